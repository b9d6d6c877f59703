"""Parity at the sizes and launch shapes the benchmark runs.

The element kernels are persistent: each warp takes one batch of 32 quadrature
points (8 Q4 or 4 HEX8 elements) after another.  These tests make warps take
many batches in turn, both by capping the grid on small meshes
(gd_options.asm_grid_max) and by meshes larger than one wave of the default grid
(at least 12k Q4 or 6k HEX8 elements), and compare with the FP64 oracle element
by element.  At the benchmark's full sizes they compare the whole notched plate
(39,936 Q4 elements) and, on the 64^3 HEX8 cube (2.1 M points), every result that
the oracle can compute for a sample of nodes: the residual and tangent rows of
the sampled nodes (summed over all their elements) and the history of every point
of those elements.  The Krylov solve is checked in each of its row-cache modes
(shared-memory values and columns, columns only, none) against a direct LU
(2D notched plate) and against its own true residual (1.1 M dofs, 3D).  The
64^3 biaxial path is compared with the homogeneous material-point driver
(Sec. 5.1: phi = kappa; Sec. 5.2 uniform deformation) in FP64 and mixed precision.

Bars: FP64 1e-10 relative (max-norm over each array); mixed precision 2e-5 on
residual, tangent and history (the FP32 element chain, as in test_gpu_mixed)."""
import numpy as np
import pytest

from gpu_common import compare_assembly, gpu_assemble, node_size, oracle_assemble, rel_err, smooth_state
from paper_2604_03411_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
TOL32 = 2e-5


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


def problem(mesh, w_psi, w_y, seed=9):
    rng = np.random.default_rng(seed)
    psi = I.icnn_weights(rng, 3, w_psi)
    yld = I.icnn_weights(rng, 1, w_y)
    return I.Problem("fullsize", mesh, psi, yld, I.Material(), np.array([0.1]))


def full_compare(env, prob, precision, dofs, kappa, tune=True, **opt):
    torch, B, oracle = env
    o = B.gd_default_options(precision=B.GD_FP64 if precision == "fp64" else B.GD_MIXED, **opt)
    h = B.gd_create(prob, o)
    if tune:
        B.gd_autotune(h)
    Rg, Kg, kg, lg = gpu_assemble(B, torch, h, dofs, kappa, precision=precision)
    Ro, Ko, ko, qi = oracle_assemble(oracle, prob, dofs, kappa)
    eR, eK, ek, fl = compare_assembly(Rg, Kg, kg, lg, Ro, Ko, ko, qi)
    return eR, eK, ek, fl, qi


# ---------------------------------------------------------------------------
# many batches per warp
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dim", [2, 3])
def test_capped_grid_many_batches_per_warp(env, precision, dim):
    """One or two CTAs for the whole mesh: every warp takes 8-20 batches in turn
    (a value carried across batches would show here)."""
    if dim == 2:
        mesh = I.uniaxial_bc_2d(I.structured_q4(24, 20))          # 480 elements = 60 batches
        prob = problem(mesh, 32, 32)
    else:
        mesh = I.biaxial_bc_3d(I.structured_hex8(6, 6, 5))        # 180 elements = 45 batches
        prob = problem(mesh, 64, 64)
    rng = np.random.default_rng(21)
    dofs, kappa = smooth_state(mesh, rng)
    tol = TOL64 if precision == "fp64" else TOL32
    for cap in (1, 2):
        eR, eK, ek, fl, qi = full_compare(env, prob, precision, dofs, kappa, tune=False, asm_grid_max=cap)
        assert qi[..., 5].sum() > 0 and (qi[..., 5] == 0).sum() > 0
        assert eR < tol and eK < tol and ek < tol, (cap, eR, eK, ek)
        if precision == "fp64":
            assert fl


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_q4_mesh_beyond_one_wave(env, precision):
    """12,480 Q4 elements (one wave of the default grid covers about 9.7 k)."""
    mesh = I.uniaxial_bc_2d(I.structured_q4(120, 104, 1.2, 1.04))
    prob = problem(mesh, 32, 32, seed=12)
    dofs, kappa = smooth_state(mesh, np.random.default_rng(22))
    eR, eK, ek, fl, _ = full_compare(env, prob, precision, dofs, kappa)
    tol = TOL64 if precision == "fp64" else TOL32
    assert eR < tol and eK < tol and ek < tol, (eR, eK, ek)
    if precision == "fp64":
        assert fl


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hex8_mesh_beyond_one_wave(env, precision):
    """6,120 HEX8 elements (one wave of the default grid covers about 4.9 k), widths 64."""
    mesh = I.biaxial_bc_3d(I.structured_hex8(20, 18, 17, 1.0, 0.9, 0.85))
    prob = problem(mesh, 64, 64, seed=13)
    dofs, kappa = smooth_state(mesh, np.random.default_rng(23))
    eR, eK, ek, fl, _ = full_compare(env, prob, precision, dofs, kappa)
    tol = TOL64 if precision == "fp64" else TOL32
    assert eR < tol and eK < tol and ek < tol, (eR, eK, ek)
    if precision == "fp64":
        assert fl


# ---------------------------------------------------------------------------
# the benchmark's full sizes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_notched_plate_full_size(env, precision):
    """The whole 39,936-element notched plate, autotuned launch shape, against the
    oracle's full assembly."""
    prob = I.config2()
    dofs, kappa = smooth_state(prob.mesh, np.random.default_rng(24), u_amp=0.04)
    eR, eK, ek, fl, qi = full_compare(env, prob, precision, dofs, kappa)
    tol = TOL64 if precision == "fp64" else TOL32
    assert eR < tol and eK < tol and ek < tol, (eR, eK, ek)
    if precision == "fp64":
        assert fl


def sampled_oracle(oracle, prob, dofs, kappa, nodes):
    """Residual rows, tangent rows (as {column: value} per row) of `nodes`, and the
    history and loading flag of every point of their elements, from the oracle's
    element routine (each element once)."""
    mesh = prob.mesh
    model = oracle.Model.from_problem(prob)
    nd = mesh.ndof
    conn = mesh.conn
    elems = np.nonzero(np.isin(conn, nodes).any(axis=1))[0]
    want = {int(n): i for i, n in enumerate(nodes)}
    R = np.zeros((len(nodes), nd))
    K = [[dict() for _ in range(nd)] for _ in nodes]
    kap, load = {}, {}
    for e in elems:
        c = conn[e]
        Re, Ke, k1, qi = model.element(mesh.coords[c], dofs[c], kappa[e])
        kap[int(e)] = k1
        load[int(e)] = qi[:, 5]
        for a, n in enumerate(c):
            s = want.get(int(n))
            if s is None:
                continue
            for i in range(nd):
                R[s, i] += Re[a * nd + i]
                row = K[s][i]
                for b, m in enumerate(c):
                    for k in range(nd):
                        col = int(m) * nd + k
                        row[col] = row.get(col, 0.0) + Ke[a * nd + i, b * nd + k]
    return elems, R, K, kap, load


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cube64_sampled(env, precision):
    """64^3 HEX8 cube (262,144 elements, 2.1 M points, widths 64), autotuned launch
    shape: residual and tangent rows of 160 sampled nodes (the 8 corners among them)
    and the history of every point of their elements, against the oracle."""
    torch, B, oracle = env
    prob = I.config3(precision=precision)
    mesh = prob.mesh
    rng = np.random.default_rng(25)
    dofs, kappa = smooth_state(mesh, rng, u_amp=0.04)
    o = B.gd_default_options(precision=B.GD_FP64 if precision == "fp64" else B.GD_MIXED)
    h = B.gd_create(prob, o)
    B.gd_autotune(h)
    dev = torch.device("cuda:0")
    rowptr, colidx = B.gd_csr_pattern(h)
    d = torch.tensor(dofs.ravel(), dtype=torch.float64, device=dev)
    k = torch.tensor(kappa.ravel(), dtype=torch.float64, device=dev)
    Rt = torch.zeros_like(d)
    vals = torch.zeros(colidx.size, dtype=torch.float64 if precision == "fp64" else torch.float32, device=dev)
    k1 = torch.zeros_like(k)
    ld = torch.zeros(k.numel(), dtype=torch.int8, device=dev)
    B.gd_assemble(h, d, k, Rt, vals, k1, ld, B.GD_ASM_TANGENT)
    torch.cuda.synchronize()
    corners = [0, 64, 64 * 65, 64 * 65 + 64]
    corners = corners + [c + 64 * 65 * 65 for c in corners]
    nodes = np.unique(np.concatenate([corners, rng.choice(mesh.n_nodes, 152, replace=False)]))
    elems, Ro, Ko, ko, lo = sampled_oracle(oracle, prob, dofs, kappa, nodes)
    nd = mesh.ndof
    Rg = Rt.view(-1, nd)[torch.tensor(nodes, device=dev)].cpu().numpy()
    kg = k1.view(-1, mesh.nq)[torch.tensor(elems, device=dev)].cpu().numpy()
    lg = ld.view(-1, mesh.nq)[torch.tensor(elems, device=dev)].cpu().numpy()
    kor = np.stack([ko[int(e)] for e in elems])
    lor = np.stack([lo[int(e)] for e in elems])
    # tangent rows: gather the GPU CSR rows of the sampled nodes on the device
    rows = (nodes[:, None] * nd + np.arange(nd)[None, :]).ravel()
    starts, ends = rowptr[rows], rowptr[rows + 1]
    idx = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)])
    gv = vals[torch.tensor(idx, device=dev)].double().cpu().numpy()
    gk, ok_k, pos = [], [], 0
    for r, (a, b) in zip(rows, zip(starts, ends)):
        cols = colidx[a:b]
        s = int(np.nonzero(nodes == r // nd)[0][0])
        orow = Ko[s][int(r % nd)]
        assert set(orow.keys()) == set(int(c) for c in cols), f"pattern of row {r}"
        gk.append(gv[pos:pos + (b - a)])
        ok_k.append(np.array([orow[int(c)] for c in cols]))
        pos += b - a
    gk = np.concatenate(gk)
    ok_k = np.concatenate(ok_k)
    tol = TOL64 if precision == "fp64" else TOL32
    eR = rel_err(Rg, Ro)
    eK = rel_err(gk, ok_k)
    ek = rel_err(kg, kor)
    assert lor.sum() > 0 and (lor == 0).sum() > 0
    assert eR < tol and eK < tol and ek < tol, (eR, eK, ek)
    if precision == "fp64":
        assert np.array_equal(lg.astype(bool), lor > 0.5)


# ---------------------------------------------------------------------------
# Krylov row-cache modes
# ---------------------------------------------------------------------------
def damaged_system(env, prob, steps, **opt):
    torch, B, oracle = env
    h = B.gd_create(prob, B.gd_default_options(**opt))
    for _ in range(steps):
        B.gd_newton_step(h)
    dofs, kappa = B.gd_get_fields(h)
    R, K, _, _ = gpu_assemble(B, torch, h, dofs, kappa)
    n = R.size
    nd = prob.mesh.ndof
    bidx = prob.mesh.bc_node.astype(np.int64) * nd + prob.mesh.bc_comp
    free = np.ones(n, bool)
    free[bidx] = False
    b = np.random.default_rng(31).standard_normal(n)
    b[~free] = 0.0
    return K, b, free


@pytest.mark.parametrize("coarse", [1536, 0])
def test_krylov_row_cache_modes_vs_lu(env, coarse):
    """Full-size notched plate (121k dofs): the solve in each row-cache mode matches
    SuperLU and reaches its true residual; the modes agree with one another."""
    torch, B, oracle = env
    import scipy.sparse.linalg as spla
    prob = I.config2()
    prob.load = prob.load[:8]
    K, b, free = damaged_system(env, prob, 4)
    Kff = K[free][:, free].tocsc()
    xr = spla.spsolve(Kff, b[free])
    vals = torch.tensor(K.data, dtype=torch.float64, device="cuda")
    bt = torch.tensor(b, device="cuda")
    xs = []
    for mode in (0, 1, 2):
        h = B.gd_create(prob, B.gd_default_options(krylov_rtol=1e-12, krylov_max=40000, coarse=coarse,
                                                   krylov_row_cache=mode))
        xt = torch.zeros_like(bt)
        it, rel = B.gd_solve(h, bt, xt, vals)
        x = xt.cpu().numpy()
        assert rel <= 1e-12 and it > 0, (mode, it, rel)
        true_rel = np.linalg.norm(Kff @ x[free] - b[free]) / np.linalg.norm(b[free])
        assert true_rel < (1e-10 if coarse else 1e-9), (mode, true_rel)
        assert rel_err(x[free], xr) < 1e-6, mode
        xs.append(x)
    assert rel_err(xs[1], xs[0]) < 1e-8 and rel_err(xs[2], xs[0]) < 1e-8


def test_krylov_row_cache_modes_cube64(env):
    """64^3 cube (1.1 M dofs, ndof 4): every row-cache mode reaches the true residual
    of the tangent after two load steps, and the modes agree."""
    torch, B, oracle = env
    prob = I.config3(precision="fp64")
    prob.load = prob.load[:4]
    K, b, free = damaged_system(env, prob, 2)
    vals = torch.tensor(K.data, dtype=torch.float64, device="cuda")
    bt = torch.tensor(b, device="cuda")
    Kff = K[free][:, free].tocsr()
    xs = []
    for mode in (0, 1, 2):
        h = B.gd_create(prob, B.gd_default_options(krylov_rtol=1e-11, krylov_max=20000, krylov_row_cache=mode))
        xt = torch.zeros_like(bt)
        it, rel = B.gd_solve(h, bt, xt, vals)
        x = xt.cpu().numpy()
        true_rel = np.linalg.norm(Kff @ x[free] - b[free]) / np.linalg.norm(b[free])
        assert rel <= 1e-11 and true_rel < 1e-9, (mode, it, rel, true_rel)
        xs.append(x)
    assert rel_err(xs[1], xs[0]) < 1e-7 and rel_err(xs[2], xs[0]) < 1e-7


# ---------------------------------------------------------------------------
# 64^3 biaxial path against the homogeneous material point
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cube64_path_vs_material_point(env, precision):
    """The benchmark's cube (64^3 HEX8, widths 64, biaxial to lambda = 1.267 in the
    first 10 of its 30 steps): the FE solution is the homogeneous state, so per step
    the reaction equals P11 of the 3D material-point driver, kappa and phi equal its
    kappa at every point, d = 1 - f_d(kappa), and u_z = (lam3 - 1) z.  Errors (reaction
    and u_z relative to their largest value on the path, kappa and phi relative to
    max(1, kappa), d absolute) are printed: the per-quantity errors of the mixed path."""
    torch, B, oracle = env
    prob = I.config3(precision=precision)
    prob.load = prob.load[:10]
    o = B.gd_default_options(precision=B.GD_FP64 if precision == "fp64" else B.GD_MIXED)
    h = B.gd_create(prob, o)
    m = oracle.Model.from_problem(prob)
    P11, lam3, kap = oracle.material_point_biaxial(m, 1.0 + prob.load)
    z = prob.mesh.coords[:, 2]
    mat = prob.mat
    err = {"reaction": 0.0, "kappa": 0.0, "d": 0.0, "phi": 0.0, "u_z": 0.0}
    for s in range(10):
        rep = B.gd_newton_step(h)
        assert rep.converged == 1
        dofs, kappa, dmg = B.gd_get_fields(h, damage=True)
        d = dofs.reshape(-1, 4)
        err["reaction"] = max(err["reaction"], abs(rep.reaction - P11[s]) / np.abs(P11).max())
        err["kappa"] = max(err["kappa"], np.abs(kappa - kap[s]).max() / max(1.0, kap[s]))
        dref = 1.0 - np.exp(-mat.eta_d * max(kap[s] - mat.kappa_d, 0.0))
        err["d"] = max(err["d"], np.abs(dmg - dref).max())
        err["phi"] = max(err["phi"], np.abs(d[:, 3] - kap[s]).max() / max(1.0, kap[s]))
        err["u_z"] = max(err["u_z"], np.abs(d[:, 2] - (lam3[s] - 1.0) * z).max() / np.abs(lam3 - 1.0).max())
    print(f"cube64 {precision} vs material point:", {k: f"{v:.2e}" for k, v in err.items()})
    assert kap[-1] > 1.0
    if precision == "fp64":
        assert err["reaction"] < 1e-9 and err["kappa"] < 1e-8 and err["d"] < 1e-9, err
        assert err["phi"] < 1e-8 and err["u_z"] < 1e-8, err
    else:
        assert err["reaction"] < 1e-4 and err["kappa"] < 1e-4 and err["d"] < 1e-4, err
        assert err["phi"] < 1e-4 and err["u_z"] < 1e-4, err
