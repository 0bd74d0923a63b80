"""GPU parity of the back-tracking line search (nsn_config.line_search, Sec.
8.1) against the oracle's: the trials t = 1, 1/2, 1/4, 1/8, 1/16, the first
whose FP64 merit is below the current iterate's, else the damped step; per
island in island mode.  The FP64 build must take the oracle's decisions
(merit histories, stop iterations) and reach its states."""
import numpy as np
import pytest

from paper_1907_04587_gb300 import nsn, scenes
from test_gpu_islands import PRM, SCENE, TOL64, vel_error

pytestmark = pytest.mark.gpu

H = 1.0 / 60.0
G = 9.81


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    yield


def _falling_particle(vz, mass=2.0):
    b = scenes.SceneBuilder()
    i = b.add_particle((0.0, 0.0, 0.0), vel=(0.3, 0.0, vz), mass=mass)
    b.add_contact(i, -1, (0, 0, 0), (0, 0, 0), (0, 0, 1), 0.0, 0.0)
    return b.build()


def test_line_search_full_step_on_piecewise_linear_rows(orc):
    """Min-map NCP on a frictionless particle hitting a plane: the line search
    takes t = 1 and reaches the closed-form impulse m (|v_n| + g h) at once."""
    s = _falling_particle(-1.0)
    prm = dict(newton_iters=8, cr_iters=10, ncp=1, tol_rel=0.0, line_search=1)
    o = orc.Oracle(s, **{**prm, "ncp": orc.NCP_MIN})
    g = nsn.Solver(s, precision=nsn.NSN_FP64, **prm)
    ro, rg = o.step(), g.step()
    ho, hg = o.merit_history() / ro["merit0"], g.merit_history() / rg["merit0"]
    print("oracle", ho[:5], "gpu", hg[:5])
    assert hg[3] < 1e-12
    n = min(len(ho), len(hg), 3)
    np.testing.assert_allclose(hg[:n], ho[:n], rtol=1e-9, atol=1e-14)
    expect = 2.0 * (1.0 + G * H)
    assert abs(H * g.get_lambda()[0] - expect) < 1e-10 * expect


def test_line_search_global_mode_fp64(orc):
    """One system (no islands), 4-cube stack to 1e-6: the merit history and the
    state of the oracle's searched Newton iteration."""
    s = scenes.cube_stack(seed=0)
    prm = dict(newton_iters=30, cr_iters=50, tol_rel=1e-6, line_search=1)
    o = orc.Oracle(s, **prm)
    g = nsn.Solver(s, precision=nsn.NSN_FP64, **prm)
    ro, rg = o.step(), g.step()
    ho, hg = o.merit_history(), g.merit_history()
    print("newton", ro["newton_done"], rg["newton_done"])
    assert rg["newton_done"] == ro["newton_done"]
    n = rg["newton_done"]       # merits of the solved iterations, then of the returned iterate
    np.testing.assert_allclose(hg[:n], ho[:n], rtol=1e-8, atol=1e-12 * ho[0])
    np.testing.assert_allclose(hg[-1], ho[-1], rtol=1e-6, atol=1e-12 * ho[0])
    assert vel_error(o.get_state(), g.get_state_f64(), s) < TOL64


@pytest.mark.parametrize("res", [1, 0])
def test_line_search_island_mode_fp64(orc, res):
    """Island mode, each island searching by itself, on the island-resident
    and on the streamed CR path: the oracle's stop iteration of every island
    and its states."""
    s = SCENE()
    prm = dict(PRM, line_search=1)
    o = orc.Oracle(s, **prm)
    g = nsn.Solver(s, precision=nsn.NSN_FP64, cr_resident=res, **prm)
    o.step(); g.step()
    io, ig = o.island_stats(), g.island_stats()
    print("stop oracle", io["stopped_at"].tolist())
    print("stop gpu   ", ig["stopped_at"].tolist())
    assert np.array_equal(ig["stopped_at"], io["stopped_at"])
    np.testing.assert_allclose(ig["merit0"], io["merit0"], rtol=1e-9)
    done = io["stopped_at"] >= 0
    assert np.all(ig["merit_final"][done] <= 1e-6 * ig["merit0"][done] * (1 + 1e-6))
    e = vel_error(o.get_state(), g.get_state_f64(), s)
    print("velocity error", e)
    assert e < 1e-6


def test_line_search_fp32_batch():
    """FP32 production path on a batch: the searched step stops islands where
    they meet the tolerance and at least as many as the damped step does in
    the same Newton cap, in fewer iterations on average."""
    s = scenes.batched_envs(seed=81, n_envs=32)
    prm = dict(PRM, newton_iters=30, cr_iters=50)
    a = nsn.Solver(s, line_search=1, **prm)
    b = nsn.Solver(s, line_search=0, **prm)
    a.step(); b.step()
    ia, ib = a.island_stats(), b.island_stats()
    sa, sb = ia["stopped_at"], ib["stopped_at"]
    print("stopped: line search", (sa >= 0).mean(), "damped", (sb >= 0).mean(),
          "mean stop iteration", sa[sa >= 0].mean(), sb[sb >= 0].mean())
    d = sa >= 0
    assert np.all(ia["merit_final"][d] <= 1e-6 * ia["merit0"][d] * 1.001)
    assert (sa >= 0).mean() >= (sb >= 0).mean() - 0.03
    assert all(np.isfinite(v).all() for v in a.get_state().values())
