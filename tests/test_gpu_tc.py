"""Tensor-core networks of the mixed element kernel (gd_options.icnn_mma): the
second layers of both ICNNs (Sec. 4.2) as tcgen05 matrix products over the 128
points of a thread block, BF16 operands with FP32 accumulation, in two forms:

  GD_ICNN_BF16    one product per column; the operands' 8-bit mantissas (unit
                  roundoff 2^-9) give ~3e-4 relative errors in the network outputs
                  and so in the residual, tangent and history (measured up to 1.7e-3
                  on the tangent with width-64 networks);
  GD_ICNN_BF16X3  every operand split into a BF16 high part and a BF16 residual,
                  three products hi*hi + hi*lo + lo*hi (about 16 significant bits,
                  ~2^-17 per product) -- measured within 4e-6 of the oracle.

Stated tolerances against the FP64 oracle (max-norm relative; kappa absolute on
kappa ~ O(1)): BF16X3 2e-5 on R, K and kappa (as the FP32 CUDA-core path), 1e-4 on
reaction curves; BF16 5e-3 on R, K and kappa, 5e-2 on reaction curves (the local
damage solve stops at the BF16 noise level, 4e-3 relative, and the Newton iteration
at the residual's noise floor).  Every case runs the tensor-core kernel: ragged
thread-block batches, padded widths (24, 40 -> 32, 48), isochoric and Neo-Hookean
energies, the closed-form loading function, frozen history (staggered scheme), many
batches per thread block (capped grid), the whole notched plate and the 64^3 cube."""
import numpy as np
import pytest

from gpu_common import compare_assembly, gpu_assemble, oracle_assemble, rel_err, smooth_state
from paper_2604_03411_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = {"bf16x3": 2e-5, "bf16": 5e-3}
TOL_PATH = {"bf16x3": 1e-4, "bf16": 5e-2}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_03411_gb300 import build as build_mod
    build_mod.build()
    import oracle
    import paper_2604_03411_gb300.binding as B
    oracle.threads(0)
    return torch, B, oracle


def mode(B, name):
    return {"bf16": B.GD_ICNN_BF16, "bf16x3": B.GD_ICNN_BF16X3}[name]


def opts(B, name, **kw):
    return B.gd_default_options(precision=B.GD_MIXED, icnn_mma=mode(B, name), **kw)


def make(dim, shape, w_psi, w_y, energy=I.ENERGY_ICNN_RAW, seed=7):
    mesh = I.uniaxial_bc_2d(I.structured_q4(*shape)) if dim == 2 else I.biaxial_bc_3d(I.structured_hex8(*shape))
    rng = np.random.default_rng(seed)
    psi = I.icnn_weights(rng, 3, w_psi)
    yld = I.icnn_weights(rng, 1, w_y) if w_y > 0 else I.ICNN(1, 0, np.zeros(1))
    m = I.Material(energy=energy)
    if energy == I.ENERGY_NEO_HOOKE:
        m.mu_e, m.lambda_e = 1.2, 5.0
    return I.Problem("tc", mesh, psi, yld, m, np.array([0.1]))


def state(mesh, seed, u_amp=0.06):
    return smooth_state(mesh, np.random.default_rng(seed), u_amp=u_amp)


def check(env, prob, name, seed=5, **kw):
    torch, B, oracle = env
    dofs, kappa = state(prob.mesh, seed)
    h = B.gd_create(prob, opts(B, name, **kw))
    Rg, Kg, kg, lg = gpu_assemble(B, torch, h, dofs, kappa, precision="mixed")
    Ro, Ko, ko, qi = oracle_assemble(oracle, prob, dofs, kappa)
    eR, eK, _, _ = compare_assembly(Rg, Kg, kg, lg, Ro, Ko, ko, qi)
    ek = float(np.abs(kg - ko).max())
    # history never decreases; points clearly below the yield surface keep it exactly
    assert np.all(kg >= kappa)
    clear = (qi[..., 5] < 0.5) & (np.abs(qi[..., 3]) > (1e-4 if name == "bf16x3" else 5e-2))
    assert np.all(kg[clear] == kappa[clear])
    tol = TOL[name]
    assert eR < tol and eK < tol and ek < tol, (name, eR, eK, ek)
    return qi


CASES = [
    ("q4 w16/8", (2, (7, 5), 16, 8), {}),
    ("q4 w24/40 padded", (2, (6, 5), 24, 40), {}),
    ("q4 w32/32", (2, (9, 6), 32, 32), {}),
    ("hex8 w64/64 ragged", (3, (3, 3, 2), 64, 64), {}),
    ("hex8 w32/16", (3, (5, 4, 3), 32, 16), {}),
    ("q4 isochoric", (2, (5, 3), 16, 8), {"energy": I.ENERGY_ICNN_ISO}),
    ("hex8 neo-hooke", (3, (3, 2, 2), 16, 8), {"energy": I.ENERGY_NEO_HOOKE}),
    ("q4 loading function G(q) = q", (2, (5, 4), 16, 0), {}),
]


@pytest.mark.parametrize("name", ["bf16x3", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_tc_assembly_vs_oracle(env, case, name):
    _, args, kw = case
    qi = check(env, make(*args, **kw), name)
    assert qi[..., 5].sum() > 0 and (qi[..., 5] == 0).sum() > 0


@pytest.mark.parametrize("name", ["bf16x3", "bf16"])
def test_tc_many_batches_per_cta(env, name):
    """One and two thread blocks for 480 Q4 / 180 HEX8 elements: every block takes
    15-45 batches of 128 points in turn (tensor memory and barriers reused)."""
    for cap in (1, 2):
        check(env, make(2, (24, 20), 32, 32), name, asm_grid_max=cap)
        check(env, make(3, (6, 6, 5), 64, 64), name, asm_grid_max=cap)


def test_tc_frozen_history_matches_cuda_cores(env):
    """Staggered scheme: with the history frozen the tensor-core kernel skips the local
    solve; its path matches the CUDA-core kernel's to the BF16x3 tolerance."""
    torch, B, oracle = env
    prob = I.config2(n_long=40, n_wide=16)
    prob.load = prob.load[:3]
    r = {}
    for m in (B.GD_ICNN_CUDA_CORES, B.GD_ICNN_BF16X3):
        h = B.gd_create(prob, B.gd_default_options(precision=B.GD_MIXED, icnn_mma=m, scheme=B.GD_STAGGERED,
                                                   stagger_max=1000))
        r[m], _ = B.gd_run_load_path(h)
    assert rel_err(r[B.GD_ICNN_BF16X3], r[B.GD_ICNN_CUDA_CORES]) < 1e-4


@pytest.mark.parametrize("name", ["bf16x3", "bf16"])
def test_tc_cfg1_path_vs_oracle(env, name):
    """The 8x8 load-unload-reload path (40 steps) against the oracle's LU path."""
    torch, B, oracle = env
    prob = I.config1()
    h = B.gd_create(prob, opts(B, name))
    reac, rep = B.gd_run_load_path(h)
    assert rep.steps_done == 40
    dofs, kappa = B.gd_get_fields(h)
    ref = oracle.run_load_path(oracle.Model.from_problem(prob), prob.mesh, prob.load)
    e = (rel_err(reac, ref["reaction"]), rel_err(dofs, ref["dofs"]), rel_err(kappa, ref["kappa"]))
    print(f"cfg1 path {name}: reaction {e[0]:.2e} dofs {e[1]:.2e} kappa {e[2]:.2e}")
    assert max(e) < TOL_PATH[name], e


def test_tc_notched_plate_full_size(env):
    """The whole 39,936-element notched plate (widths 32) against the oracle."""
    prob = I.config2()
    check(env, prob, "bf16x3", seed=24)


@pytest.mark.parametrize("name", ["bf16x3", "bf16"])
def test_tc_cube64_path_vs_material_point(env, name):
    """The 64^3 cube (widths 64), first 10 steps of its biaxial path, against the
    homogeneous material point; per-result errors printed."""
    torch, B, oracle = env
    prob = I.config3()
    prob.load = prob.load[:10]
    h = B.gd_create(prob, opts(B, name))
    m = oracle.Model.from_problem(prob)
    P11, lam3, kap = oracle.material_point_biaxial(m, 1.0 + prob.load)
    err = {"reaction": 0.0, "kappa": 0.0, "d": 0.0}
    for s in range(10):
        rep = B.gd_newton_step(h)
        assert rep.converged == 1
        dofs, kappa, dmg = B.gd_get_fields(h, damage=True)
        err["reaction"] = max(err["reaction"], abs(rep.reaction - P11[s]) / np.abs(P11).max())
        err["kappa"] = max(err["kappa"], np.abs(kappa - kap[s]).max() / max(1.0, kap[s]))
        dref = 1.0 - np.exp(-prob.mat.eta_d * max(kap[s] - prob.mat.kappa_d, 0.0))
        err["d"] = max(err["d"], np.abs(dmg - dref).max())
    print(f"cube64 {name} vs material point:", {k: f"{v:.2e}" for k, v in err.items()})
    assert max(err.values()) < TOL_PATH[name], err
