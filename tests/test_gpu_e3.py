"""The local-only model and the uniform-deformation study of Sec. 5.2.

Local model (gamma_d = 0, Sec. 4.2: q = q_loc, trainable from homogeneous data): the
device path of a notched plate, whose damage field is not uniform, against the
oracle's LU path in FP64 (1e-9) and in mixed precision (1e-4).

Sec. 5.2 study: the 10 x 10 x 1 plate with the closed-form Neo-Hookean energy and the
Ostwald loading function and the constants the paper lists (read as nondimensional),
pulled to a large stretch, in all four combinations {local, non-local} x {staggered
(Sec. 3.2: history advanced after the nodal solve), monolithic}, each run until the
largest damage reaches 0.995 or a step fails, as in the study.  On the uniform mesh
and on a graded one every completed curve matches the oracle's path of the same
scheme (FP64, 1e-8); on the uniform mesh the monolithic curves also equal the 3D
uniaxial material point's P11 x area, and the non-local staggered run stays far
below the monolithic damage (the paper's finding for a stiff penalty beta_d).  The
curves are printed side by side (the paper's figures are not available, so the
comparison between schemes is reported, not pinned)."""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_local_model_notched_plate_vs_oracle(env, precision):
    torch, B, oracle = env
    prob = I.config2(n_long=40, n_wide=16)
    prob.mat.gamma_d = 0.0
    prob.load = prob.load[:8]
    if precision == "fp64":
        h = B.gd_create(prob, tight(B))
    else:
        h = B.gd_create(prob, B.gd_default_options(precision=B.GD_MIXED))
    reac, rep = B.gd_run_load_path(h)
    dofs, kappa = B.gd_get_fields(h)
    ref = oracle.run_load_path(oracle.Model.from_problem(prob), prob.mesh, prob.load, rtol=1e-12, atol=1e-14)
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert np.ptp(ref["kappa"]) > 0.1 * ref["kappa"].max(), "the damage field should not be uniform"
    assert rel_err(reac, ref["reaction"]) < tol and rel_err(kappa, ref["kappa"]) < tol * 10, (
        rel_err(reac, ref["reaction"]), rel_err(kappa, ref["kappa"]))


def run(B, prob, scheme):
    """Steps of the path until the largest damage reaches 0.995 or a step fails to
    converge (the study's stopping rule): (reactions, max damage, failed, handle)."""
    h = B.gd_create(prob, tight(B, scheme=scheme))
    reac, dmax, failed = [], [], False
    for _ in range(prob.load.size):
        try:
            rep = B.gd_newton_step(h)
        except B.GDError as e:
            if e.status != B.GD_ERR_NOT_CONVERGED:
                raise
            failed = True
            break
        reac.append(rep.reaction)
        dmax.append(rep.max_damage)
        if rep.max_damage >= 0.995:
            break
    return np.array(reac), np.array(dmax), failed, h


def graded_plate(gamma):
    prob = I.uniform_plate_e3(n=4, n_steps=30, u_max=25.0, gamma_d=gamma)
    x = prob.mesh.coords
    prob.mesh.coords = x + np.stack([0.8 * np.sin(np.pi * x[:, 0] / 10.0) * np.sin(np.pi * x[:, 1] / 10.0),
                                     0.6 * np.sin(np.pi * x[:, 1] / 10.0) * np.sin(2 * np.pi * x[:, 0] / 10.0),
                                     np.zeros(len(x))], axis=1)
    return prob


def test_uniform_deformation_four_schemes(env):
    torch, B, oracle = env
    schemes = ((B.GD_MONOLITHIC, "monolithic"), (B.GD_STAGGERED, "staggered"))
    out = {}
    for mesh_kind in ("uniform", "graded"):
        for gamma in (1.0, 0.0):
            prob = (I.uniform_plate_e3(n=4, n_steps=30, u_max=25.0, gamma_d=gamma) if mesh_kind == "uniform"
                    else graded_plate(gamma))
            m = oracle.Model.from_problem(prob)
            for scheme, name in schemes:
                reac, dmax, failed, h = run(B, prob, scheme)
                k = reac.size
                assert k >= 5, (mesh_kind, gamma, name, "the first steps are elastic or mildly damaged")
                ref = oracle.run_load_path(m, prob.mesh, prob.load[:k], rtol=1e-12, atol=1e-14, scheme=name)
                dofs, kappa = B.gd_get_fields(h)
                key = (mesh_kind, gamma, name)
                assert rel_err(reac, ref["reaction"]) < 1e-8, (key, rel_err(reac, ref["reaction"]))
                assert rel_err(np.ravel(kappa), np.ravel(ref["kappa"])) < 1e-8, key
                out[key] = (reac, dmax, failed)
    # uniform mesh, monolithic: the homogeneous state of the material point
    prob = I.uniform_plate_e3(n=4, n_steps=30, u_max=25.0)
    P11, lt, kap = oracle.material_point_uniaxial_3d(oracle.Model.from_problem(prob), 1.0 + prob.load)
    area = 10.0 * 1.0
    for gamma in (1.0, 0.0):
        reac, dmax, failed = out[("uniform", gamma, "monolithic")]
        assert rel_err(reac, P11[:reac.size] * area) < 1e-8, (gamma, rel_err(reac, P11[:reac.size] * area))
    d_mono = out[("uniform", 1.0, "monolithic")][1]
    assert d_mono[-1] > 0.3, "the path should damage the plate"
    # non-local staggered: the penalty beta_d = 1000 holds kappa near the lagged phi
    d_stag = out[("uniform", 1.0, "staggered")][1]
    n = min(d_mono.size, d_stag.size)
    assert d_stag[n - 1] < 0.5 * d_mono[n - 1], (d_stag[n - 1], d_mono[n - 1])
    print("\nSec. 5.2 plate: steps done, final reaction, final max damage, stop reason")
    for (mesh_kind, gamma, name), (reac, dmax, failed) in out.items():
        label = f"{mesh_kind:8s} {'non-local' if gamma else 'local':9s} {name:10s}"
        why = "no convergence" if failed else ("d = 0.995" if dmax[-1] >= 0.995 else "end of path")
        print(f"  {label} {reac.size:3d}  {reac[-1]: .6e}  {dmax[-1]:.4f}  {why}")
