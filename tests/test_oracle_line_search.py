"""Pins of the oracle's back-tracking line search (Sec. 8.1; reading: t = 1,
1/2, 1/4, 1/8, 1/16, the first trial whose merit is below the current
iterate's, else the damped step t = damping; per island in island mode)."""
import numpy as np
import pytest

from paper_1907_04587_gb300 import scenes
from test_oracle_islands import sub_scene

H = 1.0 / 60.0
G = 9.81


def _falling_particle(vz, mass=2.0):
    b = scenes.SceneBuilder()
    i = b.add_particle((0.0, 0.0, 0.0), vel=(0.3, 0.0, vz), mass=mass)
    b.add_contact(i, -1, (0, 0, 0), (0, 0, 0), (0, 0, 1), 0.0, 0.0)
    return b.build()


def test_full_step_on_piecewise_linear_rows(orc):
    """A frictionless particle hitting a plane, min-map NCP with the
    effective-mass r (Sec. 7): on a fixed active set the rows and g are linear
    in (u, lambda), so the exact Newton direction d gives F(x + t d) = (1 - t)
    F(x).  The damped step therefore shrinks the merit by exactly 1/4 per
    iteration, and the line search takes t = 1 and lands on the solution; both
    reach the closed-form impulse h lambda_n = m (|v_n| + g h)."""
    m, vz = 2.0, -1.0
    s = _falling_particle(vz, m)
    prm = dict(newton_iters=12, cr_iters=10, ncp=orc.NCP_MIN, tol_rel=0.0)
    a = orc.Oracle(s, line_search=1, **prm)
    b = orc.Oracle(s, line_search=0, **prm)
    ra, rb = a.step(), b.step()
    ha, hb = a.merit_history() / ra["merit0"], b.merit_history() / rb["merit0"]
    print("line search", ha[:6], "damped", hb[:6])
    assert ha[3] < 1e-12
    r = hb[5:10] / hb[4:9]
    np.testing.assert_allclose(r, 0.25, rtol=1e-6)
    expect = m * (abs(vz) + G * H)
    assert abs(H * a.get_lambda()[0] - expect) < 1e-10 * expect
    assert abs(H * b.get_lambda()[0] - expect) < 1e-5 * expect
    assert abs(a.get_state()["vel"][0, 2]) < 1e-12


def test_line_search_is_the_damped_step_when_no_trial_decreases(orc):
    """At a converged iterate no trial can lower the merit below rounding, so
    the step taken is the damped one and the iterate stays (the Newton step is
    zero to rounding): iterating past convergence changes nothing."""
    s = _falling_particle(-1.0)
    prm = dict(cr_iters=10, ncp=orc.NCP_MIN, tol_rel=0.0, line_search=1)
    a = orc.Oracle(s, newton_iters=6, **prm)
    b = orc.Oracle(s, newton_iters=12, **prm)
    a.step(); b.step()
    np.testing.assert_allclose(a.get_lambda(), b.get_lambda(), rtol=1e-13)
    np.testing.assert_allclose(a.get_state()["vel"], b.get_state()["vel"], atol=1e-13)


def test_line_search_single_island_equals_global(orc):
    """With one island, the per-island search is the global search."""
    s = scenes.cube_stack(seed=3)
    prm = dict(newton_iters=8, cr_iters=30, tol_rel=1e-30, line_search=1)
    a = orc.Oracle(s, **prm)
    b = orc.Oracle(s, island_stop=1, **prm)
    a.step(); b.step()
    np.testing.assert_allclose(a.merit_history(), b.merit_history(), rtol=1e-12, atol=0)
    for k in ("pos", "vel", "omega"):
        np.testing.assert_allclose(a.get_state()[k], b.get_state()[k], rtol=0, atol=1e-13)


def test_line_search_islands_equal_separate_solves(orc):
    """Two environments in island mode with the line search: island by island,
    the states and stop iterations of each island searched and solved alone."""
    s = scenes.batched_envs(seed=5001, n_envs=2, links=(3, 5), boxes=(2, 20))
    prm = dict(newton_iters=25, cr_iters=60, tol_rel=1e-6, island_stop=1, cone_project=1, line_search=1)
    o = orc.Oracle(s, **prm)
    ni, bi, _ = o.islands()
    o.step()
    st = o.island_stats()
    full = o.get_state()
    for i in range(ni):
        bodies = np.nonzero(bi == i)[0]
        oi = orc.Oracle(sub_scene(s, bodies), **prm)
        oi.step()
        si = oi.island_stats()
        assert si["stopped_at"][0] == st["stopped_at"][i]
        part = oi.get_state()
        for k in ("pos", "quat", "vel", "omega"):
            np.testing.assert_allclose(part[k], full[k][bodies], rtol=0, atol=1e-11)


def test_line_search_reaches_tolerance_on_a_stack(orc):
    """On the 4-cube stack the searched Newton iteration reaches 1e-6 within the
    cap, in fewer iterations than the damped one (measured: 9 vs 15)."""
    s = scenes.cube_stack(seed=0)
    prm = dict(newton_iters=30, cr_iters=50, tol_rel=1e-6)
    a = orc.Oracle(s, line_search=1, **prm)
    b = orc.Oracle(s, line_search=0, **prm)
    ra, rb = a.step(), b.step()
    print("newton iterations: line search", ra["newton_done"], "damped", rb["newton_done"])
    assert ra["merit_final"] <= 1e-6 * ra["merit0"] * (1 + 1e-9)
    assert ra["newton_done"] < rb["newton_done"]
