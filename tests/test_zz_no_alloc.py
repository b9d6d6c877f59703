"""gd_solve_noalloc: the Krylov solve for callers that cannot allocate device
memory (applications whose own pool owns the device memory, runtimes that forbid
allocation after start-up).  It keeps its work space in one fixed device array inside the
library instead of allocating, so its result must match gd_solve, which uses the
handle's allocated work space, on the same system -- on two calls in a row,
because the second call reuses the array the first one left behind.  This file
is collected last so a failure here does not hide the other tests."""
import numpy as np
import pytest

from paper_2604_03411_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_solve_noalloc_matches_gd_solve():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_03411_gb300 import build as build_mod
    build_mod.build()
    import paper_2604_03411_gb300.binding as B

    dev = torch.device("cuda:0")
    prob = I.config2(n_long=60, n_wide=24)
    h = B.gd_create(prob, B.gd_default_options(krylov_rtol=1e-12, krylov_max=20000))
    B.gd_newton_step(h)                       # a converged state's tangent
    dofs, kappa = B.gd_get_fields(h)
    rowptr, colidx = B.gd_csr_pattern(h)
    n = dofs.size
    d = torch.tensor(dofs, dtype=torch.float64, device=dev)
    k = torch.tensor(kappa.ravel(), dtype=torch.float64, device=dev)
    R = torch.zeros(n, dtype=torch.float64, device=dev)
    vals = torch.zeros(colidx.size, dtype=torch.float64, device=dev)
    B.gd_assemble(h, d, k, R, vals, None, None, B.GD_ASM_TANGENT)
    fixed = np.zeros(n, np.uint8)
    fixed[prob.mesh.bc_node.astype(np.int64) * 3 + prob.mesh.bc_comp] = 1
    rng = np.random.default_rng(9)
    b = rng.standard_normal(n)
    b[fixed == 1] = 0.0
    bt = torch.tensor(b, device=dev)
    x_ref = torch.zeros_like(bt)
    it_ref, rel_ref = B.gd_solve(h, bt, x_ref, vals)
    rp = torch.tensor(rowptr, device=dev)
    ci = torch.tensor(colidx, device=dev)
    fx = torch.tensor(fixed, device=dev)
    ref = x_ref.cpu().numpy()
    for call in range(2):
        x = torch.full_like(bt, 7.0)          # stale contents must not leak into the result
        it, rel = B.gd_solve_noalloc(3, prob.mesh.n_nodes, rp, ci, vals, fx, bt, x, 1e-12, 20000)
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        assert rel <= 1e-12 and it > 0
        assert np.all(got[fixed == 1] == 0.0)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), call
    # a system larger than the fixed work space is refused before any launch
    big = B.GD_NOALLOC_MAX_DOFS // 3 + 1
    with pytest.raises(B.GDError) as ei:
        B.gd_solve_noalloc(3, big, rp, ci, vals, fx, bt, x, 1e-12, 10)
    assert ei.value.status == 1


def test_solve_noalloc_hex8_on_the_callers_stream():
    """The 4-dof (HEX8) variant on torch's current stream: two calls in a row match
    gd_solve on the same 3D system."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_03411_gb300 import build as build_mod
    build_mod.build()
    import paper_2604_03411_gb300.binding as B

    dev = torch.device("cuda:0")
    prob = I.config3(n=6, precision="fp64")
    h = B.gd_create(prob, B.gd_default_options(krylov_rtol=1e-12, krylov_max=20000))
    B.gd_newton_step(h)
    dofs, kappa = B.gd_get_fields(h)
    rowptr, colidx = B.gd_csr_pattern(h)
    n = dofs.size
    d = torch.tensor(dofs, dtype=torch.float64, device=dev)
    k = torch.tensor(kappa.ravel(), dtype=torch.float64, device=dev)
    R = torch.zeros(n, dtype=torch.float64, device=dev)
    vals = torch.zeros(colidx.size, dtype=torch.float64, device=dev)
    B.gd_assemble(h, d, k, R, vals, None, None, B.GD_ASM_TANGENT)
    fixed = np.zeros(n, np.uint8)
    fixed[prob.mesh.bc_node.astype(np.int64) * 4 + prob.mesh.bc_comp] = 1
    b = np.random.default_rng(10).standard_normal(n)
    b[fixed == 1] = 0.0
    bt = torch.tensor(b, device=dev)
    x_ref = torch.zeros_like(bt)
    B.gd_solve(h, bt, x_ref, vals)
    ref = x_ref.cpu().numpy()
    rp = torch.tensor(rowptr, device=dev)
    ci = torch.tensor(colidx, device=dev)
    fx = torch.tensor(fixed, device=dev)
    stream = torch.cuda.current_stream()
    for call in range(2):
        x = torch.full_like(bt, -3.0)
        it, rel = B.gd_solve_noalloc(4, prob.mesh.n_nodes, rp, ci, vals, fx, bt, x, 1e-12, 20000,
                                     stream=stream.cuda_stream)
        got = x.cpu().numpy()
        assert rel <= 1e-12 and it > 0
        assert np.all(got[fixed == 1] == 0.0)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), call
