"""GD_MIXED parity: FP32 element math and networks, FP32 tangent values, FP64
history test, history storage and residual accumulation.

Stated tolerances (max-norm relative to the oracle's max unless noted), derived
from FP32 arithmetic (unit roundoff 6e-8) through the element chain (~1e3
operations per entry) and then measured:
  residual 2e-5, tangent 2e-5, kappa 2e-5 (absolute on kappa ~ O(1)),
  reaction curve 1e-4, converged fields 1e-4."""
import numpy as np
import pytest

from gpu_common import gpu_assemble, oracle_assemble, rel_err
from paper_2604_03411_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL_R = 2e-5
TOL_K = 2e-5
TOL_KAPPA = 2e-5


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


def mixed_opts(B, **kw):
    return B.gd_default_options(precision=B.GD_MIXED, **kw)


@pytest.mark.parametrize("dim,shape,w", [(2, (7, 5), (16, 8)), (2, (9, 6), (32, 32)), (3, (3, 3, 2), (64, 64))])
def test_mixed_assembly_vs_oracle(env, dim, shape, w):
    torch, B, oracle = env
    rng = np.random.default_rng(5)
    mesh = I.uniaxial_bc_2d(I.structured_q4(*shape)) if dim == 2 else I.biaxial_bc_3d(I.structured_hex8(*shape))
    psi = I.icnn_weights(rng, 3, w[0])
    yld = I.icnn_weights(rng, 1, w[1])
    prob = I.Problem("m", mesh, psi, yld, I.Material(), np.array([0.1]))
    dofs, kappa = I.random_state(mesh, rng, u_amp=0.06, phi_amp=0.3, kappa_amp=0.3)
    h = B.gd_create(prob, mixed_opts(B))
    Rg, Kg, kg, lg = gpu_assemble(B, torch, h, dofs, kappa, precision="mixed")
    Ro, Ko, ko, qi = oracle_assemble(oracle, prob, dofs, kappa)
    eR = rel_err(Rg, Ro)
    dK = (Kg - Ko).tocoo()
    eK = float(np.abs(dK.data).max() / np.abs(Ko.data).max())
    ek = float(np.abs(kg - ko).max())
    # history never decreases and elastic points keep it exactly
    assert np.all(kg >= kappa)
    el = qi[..., 5] < 0.5
    clear = el & (np.abs(qi[..., 3]) > 1e-4)
    assert np.all(kg[clear] == kappa[clear])
    assert eR < TOL_R and eK < TOL_K and ek < TOL_KAPPA, (eR, eK, ek)


def test_mixed_cfg1_path_vs_oracle(env):
    torch, B, oracle = env
    prob = I.config1()
    h = B.gd_create(prob, mixed_opts(B))
    reac, rep = B.gd_run_load_path(h)
    assert rep.steps_done == 40
    dofs, kappa = B.gd_get_fields(h)
    model = oracle.Model.from_problem(prob)
    ref = oracle.run_load_path(model, prob.mesh, prob.load)
    assert rel_err(reac, ref["reaction"]) < 1e-4
    assert rel_err(dofs, ref["dofs"]) < 1e-4
    assert rel_err(kappa, ref["kappa"]) < 1e-4
