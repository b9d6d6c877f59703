"""Single-element parametric study with the closed-form Neo-Hookean energy and the
classical Ostwald loading function (G(q) = q): one HEX8 element of unit size,
E = 42, nu = 0.45, pulled to 50% strain, over the damage parameters eta_d and
kappa_d the paper varies (eta_d 1..100, kappa_d 0..2): device reactions and history
against the FP64 oracle's LU path at every step."""
import numpy as np
import pytest

from gpu_common import rel_err
from paper_2604_03411_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_03411_gb300 import build as build_mod
    build_mod.build()
    import oracle
    import paper_2604_03411_gb300.binding as B
    return torch, B, oracle


def element_problem(eta_d, kappa_d, steps=10):
    """Unit HEX8 element, uniaxial pull to 50% strain in `steps` steps."""
    mesh = I.uniaxial_bc_3d(I.structured_hex8(1, 1, 1))
    E, nu = 42.0, 0.45
    mat = I.Material(mu_e=E / (2.0 * (1.0 + nu)), lambda_e=E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), eta_d=eta_d,
                     kappa_d=kappa_d, beta_d=10.0, c_d=1.0, energy=I.ENERGY_NEO_HOOKE)
    psi = I.icnn_weights(np.random.default_rng(1), 3, 4)          # not read by the closed-form energy
    yld = I.ICNN(1, 0, np.zeros(1))                               # G(q) = q
    return I.Problem("element", mesh, psi, yld, mat, np.linspace(0.0, 0.5, steps + 1)[1:])


# (eta_d, kappa_d, final strain): gradual softening, onset then near-total loss of
# stiffness, a brittle drop, and a threshold the loading never reaches (elastic)
@pytest.mark.parametrize("eta_d,kappa_d,u_max", [(1.0, 0.0, 0.5), (3.0, 0.5, 0.4), (20.0, 1.2, 0.3),
                                                 (100.0, 0.5, 0.12)])
def test_single_element_sweep(env, eta_d, kappa_d, u_max):
    torch, B, oracle = env
    p = element_problem(eta_d, kappa_d)
    p.load = np.linspace(0.0, u_max, 11)[1:]
    h = B.gd_create(p, B.gd_default_options(newton_rtol=1e-12, newton_atol=1e-14, krylov_rtol=1e-14))
    reac, rep = B.gd_run_load_path(h)
    m = oracle.Model.from_problem(p)
    ro = oracle.run_load_path(m, p.mesh, p.load, rtol=1e-12, atol=1e-14)
    assert rel_err(reac, ro["reaction"]) < 1e-9, (eta_d, kappa_d, reac, ro["reaction"])
    _, kappa = B.gd_get_fields(h)
    assert rel_err(np.ravel(kappa), np.ravel(ro["kappa"])) < 1e-8
    assert np.all(np.ravel(kappa) >= 0.0)
