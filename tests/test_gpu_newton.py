"""Parity of the device Newton iteration over a load path (gd_newton_step /
gd_run_load_path) with the oracle's LU-based Newton, and of the homogeneous
patch with the material-point driver (any mesh size)."""
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


def tight(B, **kw):
    o = dict(newton_rtol=1e-12, newton_atol=1e-14, krylov_rtol=1e-13, krylov_max=50000)
    o.update(kw)
    return B.gd_default_options(**o)


def test_cfg1_load_unload_reload_path(env):
    """The 8x8 Q4 square through the 40-step load-unload-reload path: reactions,
    final fields and history against the oracle (both Newton to 1e-12)."""
    torch, B, oracle = env
    prob = I.config1()
    h = B.gd_create(prob, tight(B))
    reac, rep = B.gd_run_load_path(h)
    assert rep.steps_done == 40
    dofs, kappa, dmg = B.gd_get_fields(h, damage=True)
    model = oracle.Model.from_problem(prob)
    ref = oracle.run_load_path(model, prob.mesh, prob.load, rtol=1e-12, atol=1e-14)
    assert rel_err(reac, ref["reaction"]) < 1e-10
    assert rel_err(dofs, ref["dofs"]) < 1e-10
    assert rel_err(kappa, ref["kappa"]) < 1e-10
    # damage field: d = 1 - exp(-eta_d <kappa - kappa_d>_+) (the degradation function's definition)
    m = prob.mat
    d_ref = 1.0 - np.exp(-m.eta_d * np.maximum(ref["kappa"] - m.kappa_d, 0.0))
    assert np.abs(dmg - d_ref).max() < 1e-10 and dmg.min() >= 0.0 and dmg.max() < 1.0 and dmg.max() > 0.0


def test_homogeneous_patch_32x32_matches_material_point(env):
    torch, B, oracle = env
    prob = I.config1(n=32)
    prob.load = I.piecewise_path([0.0, 0.5, 0.1, 0.7], [5, 4, 6])
    h = B.gd_create(prob, tight(B))
    reac, rep = B.gd_run_load_path(h)
    model = oracle.Model.from_problem(prob)
    P11, lam2, kap = oracle.material_point_uniaxial(model, 1.0 + prob.load)
    assert rel_err(reac, P11) < 1e-9
    dofs, kappa = B.gd_get_fields(h)
    assert rel_err(kappa, np.full_like(kappa, kap[-1])) < 1e-9
    d = dofs.reshape(-1, 3)
    assert rel_err(d[:, 2], np.full(d.shape[0], kap[-1])) < 1e-8


def test_hex8_biaxial_path(env):
    """3x3x3 HEX8 cube, biaxial stretch, both networks width 16/8, against the oracle."""
    torch, B, oracle = env
    psi, yld = I.icnn_pair(3, 16, 8)
    mesh = I.biaxial_bc_3d(I.structured_hex8(3, 3, 3))
    # break the symmetry a little so the field is not homogeneous
    rng = np.random.default_rng(1)
    inner = np.all((mesh.coords > 1e-9) & (mesh.coords < 1 - 1e-9), axis=1)
    mesh.coords[inner] += 0.04 * rng.uniform(-1, 1, (inner.sum(), 3))
    prob = I.Problem("hex", mesh, psi, yld, I.Material(c_d=0.1), np.linspace(0, 0.25, 6)[1:])
    h = B.gd_create(prob, tight(B))
    reac, rep = B.gd_run_load_path(h)
    dofs, kappa = B.gd_get_fields(h)
    model = oracle.Model.from_problem(prob)
    ref = oracle.run_load_path(model, mesh, prob.load, rtol=1e-12, atol=1e-14)
    assert rel_err(reac, ref["reaction"]) < 1e-10
    assert rel_err(dofs, ref["dofs"]) < 1e-10
    assert rel_err(kappa, ref["kappa"]) < 1e-10


def test_newton_step_reports_and_state_roundtrip(env):
    torch, B, oracle = env
    prob = I.config1(n=4)
    h = B.gd_create(prob, tight(B))
    r1 = B.gd_newton_step(h)
    assert r1.converged == 1 and r1.iterations >= 1 and r1.reaction > 0
    d1, k1 = B.gd_get_fields(h)
    r2 = B.gd_newton_step(h)
    d2, k2 = B.gd_get_fields(h)
    # restart from the state after step 1 and redo step 2: identical result
    B.gd_set_state(h, d1, k1, next_step=1)
    r2b = B.gd_newton_step(h)
    d2b, k2b = B.gd_get_fields(h)
    # the restart has no previous increment to extrapolate, so Newton takes another
    # path to the same solution: agreement to the Newton tolerance
    assert rel_err(d2b, d2) < 1e-10 and rel_err(k2b, k2) < 1e-10
    assert abs(r2b.reaction - r2.reaction) <= 1e-10 * abs(r2.reaction)
    # a full save/restore (with the previous state for the predictor) repeats the
    # uninterrupted step: same Newton path, same result up to summation order
    h2 = B.gd_create(prob, tight(B))
    B.gd_newton_step(h2)
    saved = B.gd_get_state(h2)
    assert saved[3] == 1
    r2c = B.gd_newton_step(h2)
    d2c, dp2c, k2c, ns2c, _ = B.gd_get_state(h2)
    assert ns2c == 2 and rel_err(dp2c, saved[0]) == 0.0
    B.gd_set_state(h2, saved[0], saved[2], saved[3], dofs_prev=saved[1])
    r2d = B.gd_newton_step(h2)
    d2d, _, k2d, _, _ = B.gd_get_state(h2)
    # (the restored handle keeps its coarse inverse, whose age differs from the
    # uninterrupted run's, so the Krylov iterates agree to the Krylov tolerance)
    assert r2d.iterations == r2c.iterations
    assert rel_err(d2d, d2c) < 1e-10 and rel_err(k2d, k2c) < 1e-10
    # with the third state the quadratic predictor resumes at once: a restored handle
    # repeats the uninterrupted step's Newton path (also in mixed precision, where the
    # coarse level and the noise estimate are kept across the restore)
    for prec in (B.GD_FP64, B.GD_MIXED):
        h3 = B.gd_create(prob, tight(B, precision=prec))
        for _ in range(3):
            B.gd_newton_step(h3)
        d, dp, k, ns, dpp = B.gd_get_state(h3)
        assert ns == 3 and rel_err(dpp, dp) > 0.0
        ra = B.gd_newton_step(h3)
        da, _, ka, _, _ = B.gd_get_state(h3)
        B.gd_set_state(h3, d, k, ns, dofs_prev=dp, dofs_prev2=dpp)
        rb = B.gd_newton_step(h3)
        db, _, kb, _, _ = B.gd_get_state(h3)
        tol = 1e-10 if prec == B.GD_FP64 else 1e-5
        assert abs(rb.iterations - ra.iterations) <= (0 if prec == B.GD_FP64 else 1), (prec, ra.iterations, rb.iterations)
        assert rel_err(db, da) < tol and rel_err(kb, ka) < tol, prec


def test_errors_are_reported_not_faulted(env):
    """Host-side failures: a finished path, an invalid mesh and a NaN state give
    status codes; the handle stays usable."""
    torch, B, oracle = env
    prob = I.config1(n=2)
    prob.load = prob.load[:2]
    h = B.gd_create(prob, tight(B))
    B.gd_run_load_path(h)
    with pytest.raises(B.GDError) as ei:
        B.gd_newton_step(h)
    assert ei.value.status == 10
    bad = I.config1(n=2)
    bad.mesh.conn = bad.mesh.conn[:, ::-1].copy()
    with pytest.raises(B.GDError) as ei:
        B.gd_create(bad)
    assert ei.value.status == 2
    d, k = B.gd_get_fields(h)
    d[5] = np.nan
    B.gd_set_state(h, d, k, next_step=1)
    with pytest.raises(B.GDError) as ei:
        B.gd_newton_step(h)
    assert ei.value.status in (6, 5, 7)


def test_krylov_solve_matches_sparse_lu(env):
    """gd_solve on an assembled notched-plate tangent vs a direct sparse LU of the
    same eliminated system (scipy's SuperLU as the reference solve)."""
    torch, B, oracle = env
    import scipy.sparse.linalg as spla
    from gpu_common import gpu_assemble
    prob = I.config2(n_long=60, n_wide=24)
    h = B.gd_create(prob, B.gd_default_options(krylov_rtol=1e-12, krylov_max=20000))
    rng = np.random.default_rng(2)
    # the tangent of the first converged load step (a state the Newton solver meets)
    B.gd_newton_step(h)
    dofs, kappa = B.gd_get_fields(h)
    R, K, _, _ = gpu_assemble(B, torch, h, dofs, kappa)
    n = R.size
    bidx = prob.mesh.bc_node.astype(np.int64) * 3 + prob.mesh.bc_comp
    free = np.ones(n, bool)
    free[bidx] = False
    b = rng.standard_normal(n)
    b[~free] = 0.0
    rowptr, colidx = B.gd_csr_pattern(h)
    vals = torch.tensor(K.data, dtype=torch.float64, device="cuda")
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    it, rel = B.gd_solve(h, bt, xt, vals)
    x = xt.cpu().numpy()
    Kff = K[free][:, free].tocsc()
    xr = spla.spsolve(Kff, b[free])
    assert rel <= 1e-12 and it > 0
    assert np.all(x[~free] == 0.0)
    # BiCGStab tests its recursively updated residual; the true residual b - K x
    # drifts from it by rounding of the updates, by up to ~cond(K) eps
    true_rel = np.linalg.norm(Kff @ x[free] - b[free]) / np.linalg.norm(b[free])
    assert true_rel < 1e-10
    # forward error is bounded by cond(K) x residual; the Newton systems here have cond ~1e4-1e5
    assert rel_err(x[free], xr) < 1e-6


def test_autotune_keeps_results(env):
    """gd_autotune picks launch shapes from its own timings; a tuned handle gives the
    untuned handle's load path to the Newton tolerance."""
    torch, B, oracle = env
    prob = I.config2(n_long=40, n_wide=16)
    prob.load = prob.load[:3]
    h0 = B.gd_create(prob, tight(B))
    r0, _ = B.gd_run_load_path(h0)
    h1 = B.gd_create(prob, tight(B))
    t = B.gd_autotune(h1)
    assert t.asm_warps in (2, 4, 8) and 1 <= t.krylov_ctas_per_sm <= 4
    times = [x for x in t.asm_ms if x > 0]
    assert times and t.asm_ms[[2, 4, 8].index(t.asm_warps)] == min(times)
    assert t.krylov_us[t.krylov_ctas_per_sm - 1] > 0
    r1, _ = B.gd_run_load_path(h1)
    assert np.abs(r1 - r0).max() <= 1e-9 * np.abs(r0).max()


def test_staggered_scheme_reaches_the_monolithic_solution(env):
    """GD_STAGGERED_ITERATED (equilibrium at frozen history, then the local update, alternating
    until the residual with the updated history meets the Newton test) solves the
    same equations as the monolithic scheme: same reactions and fields, and the
    oracle's; FP64 and mixed precision."""
    torch, B, oracle = env
    prob = I.config2(n_long=40, n_wide=16)
    prob.load = prob.load[:4]
    rm, _ = B.gd_run_load_path(B.gd_create(prob, tight(B)))
    # the alternation converges linearly (measured: 100 alternations reach 7.5e-12 of a
    # 9.4e-6 residual in a damaging step), so the staggered runs use a 1e-10 test
    hs = B.gd_create(prob, tight(B, newton_rtol=1e-10, scheme=B.GD_STAGGERED_ITERATED, stagger_max=1000))
    rs, rep = B.gd_run_load_path(hs)
    assert rep.steps_done == prob.load.size
    assert rel_err(rs, rm) < 1e-7, (rs, rm)
    m = oracle.Model.from_problem(prob)
    ro = oracle.run_load_path(m, prob.mesh, prob.load, rtol=1e-12, atol=1e-14)
    assert rel_err(rs, ro["reaction"]) < 1e-7
    dofs, kappa = B.gd_get_fields(hs)
    assert rel_err(np.ravel(kappa), np.ravel(ro["kappa"])) < 1e-6
    r32, _ = B.gd_run_load_path(B.gd_create(prob, B.gd_default_options(precision=B.GD_MIXED,
                                                                        scheme=B.GD_STAGGERED_ITERATED,
                                                                        stagger_max=1000)))
    assert rel_err(r32, rm) < 1e-4
    with pytest.raises(B.GDError):
        B.gd_create_batch([prob, prob], tight(B, scheme=B.GD_STAGGERED))
    with pytest.raises(B.GDError):
        B.gd_create_batch([prob, prob], tight(B, scheme=B.GD_STAGGERED_ITERATED))


@pytest.mark.parametrize("dim", [2, 3])
def test_staggered_scheme_matches_the_oracle(env, dim):
    """GD_STAGGERED (Sec. 3.2: the nodal solve at the committed history, then one local
    update per step, no coupled iteration) against the oracle's staggered path, FP64
    (1e-9) and mixed precision (1e-4).  The lag makes it differ from the monolithic
    path, with less damage; gd_backward refuses it."""
    torch, B, oracle = env
    if dim == 2:
        prob = I.config2(n_long=40, n_wide=16)
        prob.load = prob.load[4:22:3]
    else:
        prob = I.notched_plate_3d(n_long=16, n_wide=15, n_steps=25)
        prob.load = prob.load[2:25:3]
    h = B.gd_create(prob, tight(B, scheme=B.GD_STAGGERED))
    rs, rep = B.gd_run_load_path(h)
    assert rep.steps_done == prob.load.size
    m = oracle.Model.from_problem(prob)
    ro = oracle.run_load_path(m, prob.mesh, prob.load, rtol=1e-12, atol=1e-14, scheme="staggered")
    dofs, kappa = B.gd_get_fields(h)
    assert rel_err(rs, ro["reaction"]) < 1e-9, (rs, ro["reaction"])
    assert rel_err(np.ravel(kappa), np.ravel(ro["kappa"])) < 1e-9
    assert rel_err(np.ravel(dofs), np.ravel(ro["dofs"])) < 1e-9
    assert float(np.max(ro["kappa"])) > prob.mat.kappa_d, "the path should damage the specimen"
    rm, _ = B.gd_run_load_path(B.gd_create(prob, tight(B)))
    assert rel_err(rs, rm) > 1e-6, "the staggered update should lag the monolithic one"
    h32 = B.gd_create(prob, B.gd_default_options(precision=B.GD_MIXED, scheme=B.GD_STAGGERED))
    r32, _ = B.gd_run_load_path(h32)
    assert rel_err(r32, ro["reaction"]) < 1e-4
    with pytest.raises(B.GDError):
        B.gd_backward(h, np.ones(prob.load.size))


def test_gmres_solve_matches_sparse_lu(env):
    """gd_options.krylov = GD_GMRES: restarted GMRES(gmres_m) with right node-block
    Jacobi preconditioning on a notched-plate tangent, against SuperLU; and a Newton
    path with GMRES for every solve against the BiCGStab path."""
    torch, B, oracle = env
    import scipy.sparse.linalg as spla
    from gpu_common import gpu_assemble
    prob = I.config2(n_long=60, n_wide=24)
    h = B.gd_create(prob, B.gd_default_options(krylov=B.GD_GMRES, gmres_m=40, krylov_rtol=1e-12,
                                               krylov_max=20000))
    B.gd_newton_step(h)
    dofs, kappa = B.gd_get_fields(h)
    R, K, _, _ = gpu_assemble(B, torch, h, dofs, kappa)
    n = R.size
    bidx = prob.mesh.bc_node.astype(np.int64) * 3 + prob.mesh.bc_comp
    free = np.ones(n, bool)
    free[bidx] = False
    rng = np.random.default_rng(3)
    b = rng.standard_normal(n)
    b[~free] = 0.0
    vals = torch.tensor(K.data, dtype=torch.float64, device="cuda")
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    it, rel = B.gd_solve(h, bt, xt, vals)
    x = xt.cpu().numpy()
    Kff = K[free][:, free].tocsc()
    xr = spla.spsolve(Kff, b[free])
    assert 0 < it and rel <= 1e-12
    assert np.all(x[~free] == 0.0)
    # GMRES reports the true residual of the returned x
    true_rel = np.linalg.norm(Kff @ x[free] - b[free]) / np.linalg.norm(b[free])
    assert abs(true_rel - rel) <= 1e-3 * rel + 1e-15
    assert rel_err(x[free], xr) < 1e-6
    # a short path, every Newton system by GMRES
    p2 = I.config2(n_long=40, n_wide=16)
    p2.load = p2.load[:4]
    rb, _ = B.gd_run_load_path(B.gd_create(p2, tight(B)))
    rg, _ = B.gd_run_load_path(B.gd_create(p2, tight(B, krylov=B.GD_GMRES)))
    assert rel_err(rg, rb) < 1e-9


def test_gmres_takes_over_when_bicgstab_breaks_down(env):
    """A skew-symmetric system S x = b on a mesh's pattern (zero diagonal node blocks, so
    the block-Jacobi preconditioner is the identity): BiCGStab's first step divides by
    r0^T S r0, which is zero up to rounding, so it cannot solve it; the FP64 solve then
    runs GMRES(m), which minimises the residual and solves it (m is above the 38 free
    dofs: full GMRES)."""
    torch, B, oracle = env
    import scipy.sparse as sp
    mesh = I.uniaxial_bc_2d(I.structured_q4(4, 2))
    prob = I.config1()
    prob.mesh = mesh
    prob.load = prob.load[:1]
    h = B.gd_create(prob, B.gd_default_options(krylov_rtol=1e-12, krylov_max=2000, coarse=0, gmres_m=50))
    rowptr, colidx = B.gd_csr_pattern(h)
    n = rowptr.size - 1
    rng = np.random.default_rng(7)
    A = sp.csr_matrix((rng.standard_normal(colidx.size), colidx, rowptr), shape=(n, n))
    A.sort_indices()
    S = (A - A.T).tocsr()
    node = np.arange(n) // 3
    S = S.tocoo()
    keep = node[S.row] != node[S.col]                      # zero diagonal node blocks
    S = sp.csr_matrix((S.data * keep, (S.row, S.col)), shape=(n, n))
    # values in the handle's pattern order
    vals = np.asarray(S[np.repeat(np.arange(n), np.diff(rowptr)), colidx]).ravel()
    bidx = mesh.bc_node.astype(np.int64) * 3 + mesh.bc_comp
    free = np.ones(n, bool)
    free[bidx] = False
    assert free.sum() == 38
    Sff = S[free][:, free].toarray()
    assert np.abs(Sff + Sff.T).max() == 0.0 and np.linalg.cond(Sff) < 1e8
    b = rng.standard_normal(n)
    b[~free] = 0.0
    x_ref = np.linalg.solve(Sff, b[free])
    vt = torch.tensor(vals, device="cuda")
    bt = torch.tensor(b, device="cuda")
    for krylov in (B.GD_BICGSTAB, B.GD_GMRES):
        hk = B.gd_create(prob, B.gd_default_options(krylov=krylov, krylov_rtol=1e-12, krylov_max=2000, coarse=0,
                                                    gmres_m=50))
        xt = torch.zeros_like(bt)
        it, rel = B.gd_solve(hk, bt, xt, vt)
        x = xt.cpu().numpy()
        assert rel <= 1e-12, (krylov, rel)
        assert rel_err(x[free], x_ref) < 1e-8, krylov
