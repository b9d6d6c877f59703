"""Calibration of the ICNN weights on a reaction curve, the use the paper's
gradient-based training motivates: the reaction-curve misfit to a curve made by
perturbed weights, differentiated through the whole load path with GDLoadPath
(forward: the device path; backward: the discrete adjoint), goes down along the
negative gradient at every step of a backtracking descent (Armijo condition)."""
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
    import paper_2604_03411_gb300.binding as B
    return torch, B


def test_descent_on_reaction_misfit(env):
    torch, B = env
    from paper_2604_03411_gb300.autograd import reaction_curve
    mesh = I.uniaxial_bc_2d(I.notched_plate_q4(12, 4))
    psi, yld = I.icnn_pair(21, 8, 8)
    mat = I.Material(c_d=10.0 * 0.08 ** 2, kappa_d=0.0)
    prob = I.Problem("calib", mesh, psi, yld, mat, np.linspace(0.0, 0.6, 5)[1:])
    opts = B.gd_default_options(newton_rtol=1e-12, newton_atol=1e-15, krylov_rtol=1e-13, krylov_max=50000)
    theta0 = np.concatenate([psi.params, yld.params])
    rng = np.random.default_rng(22)
    theta_star = theta0 * (1.0 + 0.05 * rng.standard_normal(theta0.size))
    h = B.gd_create(prob, opts)
    target = reaction_curve(torch.tensor(theta_star, dtype=torch.float64, device="cuda"), h).detach()

    def loss(th):
        r = reaction_curve(th, h)
        return ((r - target) ** 2).sum()

    theta = torch.tensor(theta0, dtype=torch.float64, device="cuda", requires_grad=True)
    L = loss(theta)
    L.backward()
    L0 = float(L.detach())
    assert L0 > 0.0
    for _ in range(3):
        g = theta.grad.detach().clone()
        gg = float((g * g).sum())
        alpha = float(L.detach()) / max(gg, 1e-300)      # a Newton-like first trial on the misfit
        accepted = False
        for _ls in range(40):
            trial = (theta.detach() - alpha * g).requires_grad_(True)
            Lt = loss(trial)
            if float(Lt.detach()) <= float(L.detach()) - 1e-4 * alpha * gg:
                accepted = True
                break
            alpha *= 0.5
        assert accepted, "the adjoint gradient is not a descent direction of the device path"
        Lt.backward()
        theta, L = trial, Lt
    assert float(L.detach()) < L0
