"""Island-resident CR (nsn_config.cr_resident) against the streamed CR loop and
the oracle.

An island of rigid bodies, contacts and joints small enough for shared memory
runs all CR iterations of a Newton iteration inside one thread block
(k_cr_resident); the others go through the streamed loop of four kernels per
CR iteration.  Both apply the same recurrence with the same FP64 scalars and
stop rules (Sec. 8.2), so the per-island decisions of the FP64 build must
equal the oracle's whichever path an island takes, and the two paths must
agree with each other to rounding.
"""
import numpy as np
import pytest

from paper_1907_04587_gb300 import nsn, scenes
from test_gpu_islands import PRM, SCENE, TOL64, vel_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    yield


def test_resident_covers_the_batched_islands():
    s = SCENE()
    g = nsn.Solver(s, **PRM)
    n_isl, _ = g.islands()
    info = g.resident_info()
    print(info)
    assert info["islands"] == n_isl and info["grid"] >= 1 and info["smem_bytes"] > 0
    off = nsn.Solver(s, cr_resident=0, **PRM).resident_info()
    assert off["islands"] == 0
    glob = nsn.Solver(s, **{**PRM, "island_stop": 0}).resident_info()
    assert glob["islands"] == 0


@pytest.mark.parametrize("cap", [512, 24])
def test_resident_fp64_matches_oracle(orc, cap):
    """cap 512: every island resident; cap 24: the small ones resident, chains
    and piles streamed, both paths in one Newton loop."""
    s = SCENE()
    o = orc.Oracle(s, **PRM)
    g = nsn.Solver(s, precision=nsn.NSN_FP64, res_max_rows=cap, **PRM)
    info = g.resident_info()
    n_isl, _ = g.islands()
    print(info, "of", n_isl)
    if cap == 24:
        assert 0 < info["islands"] < n_isl
    so_, sg_ = o.step(), g.step()
    io, ig = o.island_stats(), g.island_stats()
    assert np.array_equal(ig["stopped_at"], io["stopped_at"])
    np.testing.assert_allclose(ig["merit0"], io["merit0"], rtol=1e-9)
    done = io["stopped_at"] >= 0
    # an island that did not converge ends on an iterate that depends on the
    # rounding order; its merit is compared at a tenth of the stop tolerance,
    # which is relative to its zero-iterate merit (Sec. 8.1)
    np.testing.assert_array_less(np.abs(ig["merit_final"] - io["merit_final"])[~done],
                                 1e-7 * io["merit0"][~done] + 1e-300)
    assert sg_["newton_done"] == so_["newton_done"]
    # CR iterations end at the FP64 floor or when ||r||_P grows, both decided
    # at the rounding level: the totals agree to a few iterations
    assert abs(sg_["cr_total"] - so_["cr_total"]) <= 0.02 * so_["cr_total"]
    e = vel_error(o.get_state(), g.get_state_f64(), s)
    print("velocity error", e)
    assert e < TOL64


def test_resident_equals_streamed_fp64():
    """The two CR paths sum in different orders.  Nearly every island takes the
    same decisions; an island whose friction state cycles (stick/slip) stops
    where the cycle first dips under the tolerance, which rounding can move."""
    s = scenes.batched_envs(seed=77, n_envs=16)
    a = nsn.Solver(s, precision=nsn.NSN_FP64, **PRM)
    b = nsn.Solver(s, precision=nsn.NSN_FP64, cr_resident=0, **PRM)
    assert a.resident_info()["islands"] > 0
    a.step(); b.step()
    ia, ib = a.island_stats()["stopped_at"], b.island_stats()["stopped_at"]
    print("islands", len(ia), "same stop iteration", np.mean(ia == ib))
    assert np.mean(ia == ib) >= 0.97
    assert np.mean((ia >= 0) != (ib >= 0)) <= 0.02
    # islands that converged at the same iteration on both paths: the same
    # velocities to well inside the tolerance
    _, bi = a.islands()
    same = ((ia == ib) & (ia >= 0))[bi]
    va, vb = a.get_state_f64(), b.get_state_f64()
    d = max(np.abs(va["vel"] - vb["vel"])[same].max(), np.abs(va["omega"] - vb["omega"])[same].max())
    scale = max(np.abs(vb["vel"][same]).max(), 9.81 / 60.0)
    print("resident vs streamed velocity difference on equal islands", d / scale)
    assert d <= 1e-6 * scale


def test_resident_fp32_islands():
    """FP32 production path on one step: the resident CR stops as many islands
    as the streamed CR (within 3%; which ones is decided at the FP32 rounding
    level for cycling islands), and the islands meet the tolerance where they
    stop."""
    s = scenes.batched_envs(seed=78, n_envs=32)
    a = nsn.Solver(s, **PRM)
    b = nsn.Solver(s, cr_resident=0, **PRM)
    assert a.resident_info()["islands"] > 0
    a.step(); b.step()
    ia, ib = a.island_stats(), b.island_stats()
    sa, sb = ia["stopped_at"], ib["stopped_at"]
    print("stopped resident", (sa >= 0).mean(), "streamed", (sb >= 0).mean())
    assert (sa >= 0).mean() >= (sb >= 0).mean() - 0.03
    d = sa >= 0
    assert np.all(ia["merit_final"][d] <= 1e-6 * ia["merit0"][d] * 1.001)


def test_resident_advancing_batch_fp32():
    """Several advancing steps of a larger batch: the resident path converges
    the same share of islands as the streamed path (FP32 rounding differs)."""
    s = scenes.batched_envs(seed=79, n_envs=256)
    prm = dict(PRM, newton_iters=30, cr_iters=50)
    a = nsn.Solver(s, **prm)
    b = nsn.Solver(s, cr_resident=0, **prm)
    fa, fb = [], []
    for _ in range(4):
        a.step(); b.step()
        fa.append((a.island_stats()["stopped_at"] >= 0).mean())
        fb.append((b.island_stats()["stopped_at"] >= 0).mean())
    print("resident", fa, "streamed", fb)
    assert abs(np.mean(fa) - np.mean(fb)) < 0.02
    st = a.get_state()
    assert all(np.isfinite(v).all() for v in st.values())


def test_time_resident_reports_the_work():
    s = scenes.batched_envs(seed=80, n_envs=64)
    g = nsn.Solver(s, **dict(PRM, newton_iters=30, cr_iters=50))
    g.step()
    info = g.resident_info()
    ms, w = g.time_resident(3)
    print(ms, w, info)
    assert ms > 0
    assert 0 < w["islands"] <= info["islands"]
    # every listed island applies A at least once, at most cr_iters times
    sz = g.sizes()
    assert 0.9 * sz["rows"] <= w["row_iterations"] <= 50 * sz["rows"]
    # the committed state is kept: the next step runs and stays finite
    g.step()
    assert all(np.isfinite(v).all() for v in g.get_state().values())
