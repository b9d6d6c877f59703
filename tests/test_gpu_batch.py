"""Batched specimens (gd_create_batch): specimens of different sizes, network
widths and path lengths in one handle give the reactions, fields and history of
the same specimens run one by one, and of the FP64 oracle."""
import numpy as np
import pytest

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


def specimens(energy=I.ENERGY_ICNN_RAW):
    """Two notched plates and a plain bar; 3, 5 and 4 load steps."""
    mat = I.Material(c_d=10.0 * 0.08 ** 2, kappa_d=0.0, energy=energy)
    out = []
    for kind, a, b, wp, wy, steps, lmax, seed in [("notch", 12, 4, 8, 8, 3, 0.3, 11),
                                                   ("bar", 6, 3, 12, 6, 5, 0.4, 12),
                                                   ("notch", 16, 6, 16, 16, 4, 0.5, 13)]:
        m = I.notched_plate_q4(a, b) if kind == "notch" else I.structured_q4(a, b, 2.0, 1.0)
        psi, yld = I.icnn_pair(seed, wp, wy)
        out.append(I.Problem(kind, I.uniaxial_bc_2d(m), psi, yld, mat, np.linspace(0.0, lmax, steps + 1)[1:]))
    return out


def opts(B, **kw):
    base = dict(newton_rtol=1e-12, newton_atol=1e-14, krylov_rtol=1e-13, krylov_max=50000)
    base.update(kw)
    return B.gd_default_options(**base)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_batch_layout(env):
    torch, B, oracle = env
    probs = specimens()
    h = B.gd_create_batch(probs, opts(B))
    no, eo, n_steps = B.gd_batch_layout(h)
    assert n_steps == max(p.load.size for p in probs)
    assert list(np.diff(no)) == [p.mesh.n_nodes for p in probs]
    assert list(np.diff(eo)) == [p.mesh.n_elems for p in probs]
    with pytest.raises(B.GDError):
        B.gd_set_params(h, probs[0].psi.params)
    with pytest.raises(B.GDError):
        B.gd_backward(h, np.ones(n_steps * len(probs)))


@pytest.mark.parametrize("energy,coarse", [(I.ENERGY_ICNN_RAW, None), (I.ENERGY_ICNN_ISO, None),
                                           (I.ENERGY_ICNN_RAW, 0)])
def test_batch_matches_individual_runs_and_oracle(env, energy, coarse):
    """coarse None: the default two-level union solve; 0: per-specimen Jacobi
    recurrences (bicgstab3_batch_kernel)."""
    torch, B, oracle = env
    probs = specimens(energy)
    h = B.gd_create_batch(probs, opts(B) if coarse is None else opts(B, coarse=coarse))
    reac, rep = B.gd_run_load_path(h)
    no, eo, n_steps = B.gd_batch_layout(h)
    d_all, k_all = B.gd_get_fields(h)
    ndof = 3
    for s, p in enumerate(probs):
        hi = B.gd_create(p, opts(B))
        ri, repi = B.gd_run_load_path(hi)
        # a halved step commits an intermediate load; under monotonic loading the
        # history (a running maximum) ends at the same state either way
        n = p.load.size
        assert rel(reac[:n, s], ri) < 1e-9, (s, reac[:n, s], ri)
        # a finished path holds its last load: the reaction stays where it ended
        if n < n_steps:
            assert rel(reac[n:, s], np.full(n_steps - n, ri[-1])) < 1e-9
        di, ki = B.gd_get_fields(hi)
        assert rel(d_all[no[s] * ndof:no[s + 1] * ndof], di) < 1e-9
        assert rel(k_all[eo[s]:eo[s + 1]], ki) < 1e-8
        m = oracle.Model(2, p.mat, p.psi.params, p.psi.width, p.yld.params, p.yld.width)
        ro = oracle.run_load_path(m, p.mesh, p.load, rtol=1e-12, atol=1e-14)
        assert rel(reac[:n, s], ro["reaction"]) < 1e-9, (s, reac[:n, s], ro["reaction"])


@pytest.mark.parametrize("coarse", [None, 0])
def test_batch_mixed_precision(env, coarse):
    """GD_MIXED batch against the FP64 batch at the mixed path tolerance."""
    torch, B, oracle = env
    probs = specimens()
    extra = {} if coarse is None else {"coarse": coarse}
    r64, _ = B.gd_run_load_path(B.gd_create_batch(probs, opts(B, **extra)))
    h = B.gd_create_batch(probs, opts(B, precision=B.GD_MIXED, **extra))
    r32, _ = B.gd_run_load_path(h)
    for s in range(len(probs)):
        assert rel(r32[:, s], r64[:, s]) < 1e-4, (s, r32[:, s], r64[:, s])


def test_batch_step_by_step_equals_run(env):
    torch, B, oracle = env
    probs = specimens()
    h1 = B.gd_create_batch(probs, opts(B))
    r_run, _ = B.gd_run_load_path(h1)
    h2 = B.gd_create_batch(probs, opts(B))
    for _ in range(r_run.shape[0]):
        B.gd_newton_step(h2)
    d1, k1 = B.gd_get_fields(h1)
    d2, k2 = B.gd_get_fields(h2)
    # both runs converge to the Newton tolerance; FP64 atomics in the assembly may
    # order the sums differently, so the two states agree to that tolerance
    assert rel(d2, d1) < 1e-9 and rel(k2, k1) < 1e-9
    with pytest.raises(B.GDError):
        B.gd_newton_step(h2)
