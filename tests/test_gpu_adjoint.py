"""gd_backward: gradient of a reaction-curve loss through the whole quasi-static
path with history, against central finite differences (CUDA forward path and
the FP64 oracle's LU path), and invariance to the checkpoint interval.
Bar: 1e-5 relative to finite differences."""
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


def small_problem(n_long=16, n_wide=6, w=8, steps=6, energy=I.ENERGY_ICNN_RAW, seed=4):
    mesh = I.uniaxial_bc_2d(I.notched_plate_q4(n_long, n_wide))
    psi, yld = I.icnn_pair(seed, w, w)
    # kappa_d = 0 and a path to 35% nominal strain: the damage, and with it the
    # yield network's influence on the reaction, grows enough to be resolved by
    # central differences
    mat = I.Material(c_d=10.0 * 0.08 ** 2, energy=energy, kappa_d=0.0)
    load = np.linspace(0.0, 0.7, steps + 1)[1:]
    return I.Problem("adj", mesh, psi, yld, mat, load)


def opts(B, k=2):
    return B.gd_default_options(newton_rtol=1e-13, newton_atol=1e-15, krylov_rtol=1e-13, krylov_max=50000,
                                checkpoint_every=k)


def loss_and_grad_target(reac, target):
    r = reac - target
    return float(np.sum(r * r)), 2.0 * r


def gpu_loss(B, prob, theta, target, k=2):
    h = B.gd_create(prob, opts(B, k))
    n_psi = prob.psi.params.size
    B.gd_set_params(h, theta[:n_psi], theta[n_psi:])
    reac, rep = B.gd_run_load_path(h)
    # a halved step adds commits to the path; differences across runs with different
    # commit sequences would not be derivatives of one discrete path
    assert rep.step_cuts == 0
    return loss_and_grad_target(reac, target)[0], h, reac


@pytest.mark.parametrize("energy", [I.ENERGY_ICNN_RAW, I.ENERGY_ICNN_ISO])
def test_adjoint_vs_central_differences(env, energy):
    torch, B, oracle = env
    prob = small_problem(energy=energy)
    theta0 = np.concatenate([prob.psi.params, prob.yld.params])
    h = B.gd_create(prob, opts(B))
    reac0, rep0 = B.gd_run_load_path(h)
    assert rep0.step_cuts == 0
    target = 0.9 * reac0 + 0.001
    L0, dL = loss_and_grad_target(reac0, target)
    g = B.gd_backward(h, dL)
    assert g.shape == theta0.shape and np.all(np.isfinite(g))
    rng = np.random.default_rng(41)
    n_psi = prob.psi.params.size
    idx = np.concatenate([rng.choice(n_psi, 12, replace=False), n_psi + rng.choice(theta0.size - n_psi, 8, replace=False)])
    fd = []
    for i in idx:
        # fourth-order central differences: the truncation error stays far below the
        # bar with a step large enough that the loss's rounding (the Newton tolerance)
        # does not dominate the smallest gradient components
        step = 5e-4 * max(abs(theta0[i]), 1e-1)

        def L_at(m):
            th = theta0.copy()
            th[i] += m * step
            return gpu_loss(B, prob, th, target)[0]
        fd.append((8.0 * (L_at(1) - L_at(-1)) - (L_at(2) - L_at(-2))) / (12.0 * step))
    fd = np.array(fd)
    scale = np.abs(fd).max()
    assert scale > 0
    err = np.abs(g[idx] - fd) / np.maximum(np.abs(fd), 1e-3 * scale)
    assert err.max() < 1e-5, (err.max(), g[idx], fd)


def test_checkpoint_interval_does_not_change_the_gradient(env):
    torch, B, oracle = env
    prob = small_problem(steps=7)
    grads = []
    for k in (1, 3, 100):
        h = B.gd_create(prob, opts(B, k))
        reac, _ = B.gd_run_load_path(h)
        grads.append(B.gd_backward(h, np.linspace(1.0, 2.0, reac.size)))
        # the handle is back at the end of the path
        with pytest.raises(B.GDError):
            B.gd_newton_step(h)
    for g in grads[1:]:
        assert np.abs(g - grads[0]).max() <= 1e-9 * np.abs(grads[0]).max()


def test_adjoint_vs_oracle_finite_differences(env):
    """The oracle's FP64 gradient: central differences of its LU-based path."""
    torch, B, oracle = env
    prob = small_problem(n_long=6, n_wide=3, w=8, steps=4)
    theta0 = np.concatenate([prob.psi.params, prob.yld.params])
    n_psi = prob.psi.params.size
    h = B.gd_create(prob, opts(B))
    reac0, _ = B.gd_run_load_path(h)
    target = 0.95 * reac0
    _, dL = loss_and_grad_target(reac0, target)
    g = B.gd_backward(h, dL)

    def oracle_loss(theta):
        m = oracle.Model(2, prob.mat, theta[:n_psi], prob.psi.width, theta[n_psi:], prob.yld.width)
        res = oracle.run_load_path(m, prob.mesh, prob.load, rtol=1e-13, atol=1e-15)
        return loss_and_grad_target(res["reaction"], target)[0]

    for i in (3, n_psi + 5, n_psi - 2):
        step = 1e-4 * max(abs(theta0[i]), 1e-1)
        tp = theta0.copy(); tp[i] += step
        tm = theta0.copy(); tm[i] -= step
        fd = (oracle_loss(tp) - oracle_loss(tm)) / (2 * step)
        assert abs(g[i] - fd) <= 1e-5 * max(abs(fd), 1e-8), (i, g[i], fd)


def test_autograd_function_matches_backward(env):
    """GDLoadPath (torch.autograd.Function): forward gives gd_run_load_path's curve
    from the undeformed state at theta, backward gives gd_backward's gradient."""
    torch, B, oracle = env
    from paper_2604_03411_gb300.autograd import reaction_curve
    prob = small_problem(n_long=8, n_wide=4, steps=4)
    theta0 = np.concatenate([prob.psi.params, prob.yld.params])
    h = B.gd_create(prob, opts(B))
    theta = torch.tensor(theta0 * 1.01, dtype=torch.float64, device="cuda", requires_grad=True)
    reac = reaction_curve(theta, h)
    w = torch.linspace(1.0, 2.0, reac.numel(), dtype=torch.float64, device="cuda")
    (w * reac).sum().backward()
    h2 = B.gd_create(prob, opts(B))
    n_psi = prob.psi.params.size
    B.gd_set_params(h2, theta0[:n_psi] * 1.01, theta0[n_psi:] * 1.01)
    r2, _ = B.gd_run_load_path(h2)
    g2 = B.gd_backward(h2, w.cpu().numpy())
    assert np.abs(reac.detach().cpu().numpy() - r2).max() <= 1e-10 * np.abs(r2).max()
    g = theta.grad.cpu().numpy()
    assert np.abs(g - g2).max() <= 1e-8 * np.abs(g2).max()
    # a second call on the same handle restarts the path from the undeformed state
    reac_again = reaction_curve(theta.detach(), h)
    assert torch.allclose(reac_again, reac.detach(), rtol=1e-10, atol=0)


def test_autograd_refuses_a_stale_path(env):
    """The backward pass differentiates the path the handle holds; when the handle ran
    another path (or changed its state or weights) after the forward, backward raises
    instead of returning that other path's gradient."""
    torch, B, oracle = env
    from paper_2604_03411_gb300.autograd import reaction_curve
    prob = small_problem(n_long=8, n_wide=4, steps=3)
    theta0 = np.concatenate([prob.psi.params, prob.yld.params])
    h = B.gd_create(prob, opts(B))
    theta = torch.tensor(theta0, dtype=torch.float64, device="cuda", requires_grad=True)
    reac = reaction_curve(theta, h)
    reaction_curve(torch.tensor(theta0 * 1.02, dtype=torch.float64, device="cuda"), h)   # another path
    with pytest.raises(RuntimeError):
        reac.sum().backward()


@pytest.mark.parametrize("energy", [I.ENERGY_ICNN_RAW, I.ENERGY_ICNN_ISO])
def test_adjoint_vs_oracle_adjoint_every_weight(env, energy):
    """gd_backward against the oracle's FP64 discrete adjoint (all states stored,
    transposed LU solves) on every weight of both networks, along a path that loads,
    unloads, reloads below and then beyond its previous maximum (the history adjoint
    is carried through unloading points).  Bar 1e-8 of the largest component (both
    are exact derivatives of paths converged to 1e-13)."""
    torch, B, oracle = env
    mesh = I.uniaxial_bc_2d(I.structured_q4(3, 2))
    psi, yld = I.icnn_pair(11, 8, 8)
    mat = I.Material(beta_d=10.0, c_d=10.0 * 0.1 ** 2, energy=energy)
    load = np.array([0.25, 0.5, 0.35, 0.45, 0.6])
    prob = I.Problem("adj-oracle", mesh, psi, yld, mat, load)
    w = np.array([1.0, -0.5, 2.0, 0.7, 1.5])
    go, reac_o = oracle.adjoint_gradient(oracle.Model.from_problem(prob), mesh, load, w, rtol=1e-13, atol=1e-15)
    h = B.gd_create(prob, opts(B, k=2))
    reac, rep = B.gd_run_load_path(h)
    assert rep.step_cuts == 0
    assert np.abs(reac - reac_o).max() <= 1e-10 * np.abs(reac_o).max()
    g = B.gd_backward(h, w)
    assert g.size == go.size
    err = np.abs(g - go).max() / np.abs(go).max()
    print(f"adjoint vs oracle adjoint ({energy}): {err:.2e} over {g.size} weights")
    assert err < 1e-8, err


def test_adjoint_cfg4_notched_plate(env):
    """The calibration workload: notched plate of 19,980 Q4 elements, 30 load steps,
    both networks width 32 (2,500 weights), checkpoint every 5 steps; the loss is the
    squared misfit of the reaction curve against the curve at seeded 5%-perturbed
    weights.  gd_backward against central differences of the GPU path on the 20
    seeded weights, bar 1e-5 relative (to a tenth of the largest component for the
    components below it)."""
    torch, B, oracle = env
    prob = I.config4()
    theta0 = np.concatenate([prob.psi.params, prob.yld.params])
    n_psi = prob.psi.params.size
    o = B.gd_default_options(newton_rtol=1e-12, newton_atol=1e-14, krylov_rtol=1e-13, krylov_max=50000,
                             checkpoint_every=prob.extra["checkpoint_every"])

    def path(theta):
        h = B.gd_create(prob, o)
        B.gd_set_params(h, theta[:n_psi], theta[n_psi:])
        reac, rep = B.gd_run_load_path(h)
        assert rep.step_cuts == 0
        return h, reac

    _, target = path(prob.extra["theta_star"])
    h, reac = path(theta0)
    _, dL = loss_and_grad_target(reac, target)
    g = B.gd_backward(h, dL)
    assert g.size == theta0.size == 2500
    scale = np.abs(g).max()
    for i in prob.extra["fd_index"]:
        step = 1e-6 * max(abs(theta0[i]), 1e-3)
        tp = theta0.copy()
        tp[i] += step
        tm = theta0.copy()
        tm[i] -= step
        fp = loss_and_grad_target(path(tp)[1], target)[0]
        fm = loss_and_grad_target(path(tm)[1], target)[0]
        fd = (fp - fm) / (2 * step)
        # relative to the component for components above a tenth of the largest; the
        # central differences of the smaller ones carry the paths' Newton tolerance
        # (measured ~5e-9 absolute, 1e-7 of the largest), so those are held to 1e-6 of
        # the largest component
        assert abs(g[i] - fd) <= 1e-5 * max(abs(fd), 0.1 * scale), (i, g[i], fd)


def test_mixed_precision_gradient(env):
    """gd_backward on a GD_MIXED path (recomputed in mixed precision, FP64 adjoint
    systems at its states) against the FP64 path's gradient: the stated mixed
    tolerance of the gradient is 1e-3 relative to the largest component."""
    torch, B, oracle = env
    prob = small_problem()
    r = {}
    for prec in (B.GD_FP64, B.GD_MIXED):
        o = opts(B) if prec == B.GD_FP64 else B.gd_default_options(precision=B.GD_MIXED, checkpoint_every=2)
        h = B.gd_create(prob, o)
        reac, rep = B.gd_run_load_path(h)
        assert rep.step_cuts == 0
        w = np.linspace(1.0, 2.0, reac.size)
        r[prec] = (reac, B.gd_backward(h, w))
    g64, g32 = r[B.GD_FP64][1], r[B.GD_MIXED][1]
    err = np.abs(g32 - g64).max() / np.abs(g64).max()
    rerr = np.abs(r[B.GD_MIXED][0] - r[B.GD_FP64][0]).max() / np.abs(r[B.GD_FP64][0]).max()
    print(f"mixed vs FP64: reaction {rerr:.2e}, gradient {err:.2e} (largest component)")
    assert err < 1e-3, err
