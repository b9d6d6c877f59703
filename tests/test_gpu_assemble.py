"""Parity of the FP64 element kernel (through gd_assemble) with the FP64 oracle,
element by element: residual, CSR tangent values, updated history, loading flags.
Bar: max|gpu - oracle| / max|oracle| <= 1e-10 per array (FP64 mode)."""
import numpy as np
import pytest

from gpu_common import compare_assembly, gpu_assemble, oracle_assemble
from paper_2604_03411_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10


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


def make_problem(dim, shape, w_psi, w_y, energy=I.ENERGY_ICNN_RAW, seed=7, **mat):
    if dim == 2:
        mesh = I.uniaxial_bc_2d(I.structured_q4(*shape))
    else:
        mesh = I.biaxial_bc_3d(I.structured_hex8(*shape))
    rng = np.random.default_rng(seed)
    psi = I.icnn_weights(rng, 3, w_psi)
    yld = I.icnn_weights(rng, 1, w_y) if w_y > 0 else I.ICNN(1, 0, np.zeros(1))
    m = I.Material(energy=energy, **mat)
    if energy == I.ENERGY_NEO_HOOKE:
        m.mu_e, m.lambda_e = 1.2, 5.0
    return I.Problem("t", mesh, psi, yld, m, np.array([0.1]))


def run_case(env, prob, seed=3, u_amp=0.08, phi_amp=0.3, kappa_amp=0.3, distort=0.0):
    torch, B, oracle = env
    rng = np.random.default_rng(seed)
    if distort:
        prob.mesh.coords = prob.mesh.coords + distort * rng.uniform(-1, 1, prob.mesh.coords.shape) / np.sqrt(
            prob.mesh.n_elems ** (1.0 / prob.mesh.dim))
    dofs, kappa = I.random_state(prob.mesh, rng, u_amp=u_amp, phi_amp=phi_amp, kappa_amp=kappa_amp)
    h = B.gd_create(prob, B.gd_default_options())
    Rg, Kg, kg, lg = gpu_assemble(B, torch, h, dofs, kappa)
    Ro, Ko, ko, qi = oracle_assemble(oracle, prob, dofs, kappa)
    eR, eK, ek, fl = compare_assembly(Rg, Kg, kg, lg, Ro, Ko, ko, qi)
    return eR, eK, ek, fl, qi


@pytest.mark.parametrize("w_psi,w_y", [(16, 8), (8, 0), (24, 32), (32, 64), (64, 16)])
def test_q4_widths(env, w_psi, w_y):
    prob = make_problem(2, (7, 5), w_psi, w_y)
    eR, eK, ek, fl, qi = run_case(env, prob, distort=0.15)
    assert qi[..., 5].sum() > 0 and (qi[..., 5] == 0).sum() > 0, "want both loading and elastic points"
    assert eR < TOL and eK < TOL and ek < TOL and fl, (eR, eK, ek, fl)


@pytest.mark.parametrize("energy", [I.ENERGY_ICNN_RAW, I.ENERGY_ICNN_ISO, I.ENERGY_NEO_HOOKE])
@pytest.mark.parametrize("dim", [2, 3])
def test_energies(env, dim, energy):
    prob = make_problem(dim, (5, 3) if dim == 2 else (3, 2, 2), 16, 8, energy=energy)
    eR, eK, ek, fl, _ = run_case(env, prob, distort=0.1)
    assert eR < TOL and eK < TOL and ek < TOL and fl, (eR, eK, ek, fl)


def test_hex8_wide_networks_ragged(env):
    """27 HEX8 elements (6 full batches of 4 + a tail of 3), both networks width 64."""
    prob = make_problem(3, (3, 3, 3), 64, 64)
    eR, eK, ek, fl, qi = run_case(env, prob, distort=0.1, u_amp=0.05)
    assert eR < TOL and eK < TOL and ek < TOL and fl, (eR, eK, ek, fl)


def test_many_ctas_q4(env):
    """340 Q4 elements: several thread blocks per launch and a ragged last batch."""
    prob = make_problem(2, (20, 17), 16, 16, seed=11)
    eR, eK, ek, fl, _ = run_case(env, prob, seed=5)
    assert eR < TOL and eK < TOL and ek < TOL and fl, (eR, eK, ek, fl)


def test_all_elastic_and_all_loading(env):
    torch, B, oracle = env
    prob = make_problem(2, (6, 6), 16, 8)
    rng = np.random.default_rng(4)
    dofs, _ = I.random_state(prob.mesh, rng, u_amp=0.05, phi_amp=0.3)
    kappa = 5.0 + rng.random((prob.mesh.n_elems, 4))          # far above the yield surface: all elastic
    h = B.gd_create(prob, B.gd_default_options())
    Rg, Kg, kg, lg = gpu_assemble(B, torch, h, dofs, kappa)
    Ro, Ko, ko, qi = oracle_assemble(oracle, prob, dofs, kappa)
    assert qi[..., 5].sum() == 0 and lg.sum() == 0
    eR, eK, ek, fl = compare_assembly(Rg, Kg, kg, lg, Ro, Ko, ko, qi)
    assert eR < TOL and eK < TOL and ek == 0.0 and fl, (eR, eK, ek)
    prob2 = make_problem(2, (6, 6), 16, 8, kappa_d=0.0)
    eR, eK, ek, fl, qi = run_case(env, prob2, kappa_amp=1e-6, u_amp=0.1, phi_amp=0.5)
    assert qi[..., 5].mean() > 0.5
    assert eR < TOL and eK < TOL and ek < TOL and fl, (eR, eK, ek, fl)


def test_undeformed_state_is_stress_free(env):
    torch, B, oracle = env
    prob = make_problem(3, (2, 2, 2), 32, 16)
    h = B.gd_create(prob, B.gd_default_options())
    n = prob.mesh.n_nodes * 4
    Rg, Kg, kg, lg = gpu_assemble(B, torch, h, np.zeros(n), np.zeros((prob.mesh.n_elems, 8)))
    assert np.abs(Rg).max() < 1e-14 and np.all(kg == 0.0) and np.all(lg == 0)
