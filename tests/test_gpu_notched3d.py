"""The paper's 3D notched-plate geometry (thin plate, one HEX8 layer, the 241-element
mesh): the device load path against the FP64 oracle's LU path, reactions and
history, and the mixed-precision path against FP64."""
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


def problem():
    p = I.notched_plate_3d(n_long=16, n_wide=15, n_steps=50)
    p.load = p.load[:4]
    return p


def test_notched_plate_3d_vs_oracle(env):
    torch, B, oracle = env
    p = problem()
    h = B.gd_create(p, B.gd_default_options(newton_rtol=1e-12, newton_atol=1e-16, krylov_rtol=1e-13,
                                            krylov_max=50000))
    reac, rep = B.gd_run_load_path(h)
    assert rep.steps_done == p.load.size
    m = oracle.Model.from_problem(p)
    ro = oracle.run_load_path(m, p.mesh, p.load, rtol=1e-12, atol=1e-16)
    assert rel_err(reac, ro["reaction"]) < 1e-9, (reac, ro["reaction"])
    dofs, kappa = B.gd_get_fields(h)
    assert rel_err(np.ravel(kappa), np.ravel(ro["kappa"])) < 1e-8
    assert rel_err(np.ravel(dofs), np.ravel(ro["dofs"])) < 1e-8


def test_notched_plate_3d_mixed(env):
    torch, B, oracle = env
    p = problem()
    r64, _ = B.gd_run_load_path(B.gd_create(p, B.gd_default_options(newton_rtol=1e-12)))
    r32, _ = B.gd_run_load_path(B.gd_create(p, B.gd_default_options(precision=B.GD_MIXED)))
    assert rel_err(r32, r64) < 1e-4
