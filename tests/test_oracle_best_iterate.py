"""best_iterate (a safeguard, not in the paper): an island that has not
stopped returns the least-merit iterate its Newton iterations evaluated when
the last one is worse.

Pins: on the sliding heavy stack with identity scaling (Sec. 7 / Sec. 10: r = 1
diverges, one island) the returned merit is the least of the merit history
and the returned u and lambda are the iterate at that Newton iteration, as the
linearisation stopped there exports it (a separate code path: the Newton loop
run up to a given iteration); islands that stop at the tolerance are
unchanged bit for bit; island mode is required."""
import numpy as np
import pytest

from paper_1907_04587_gb300 import scenes
from test_oracle_rscale import sliding_heavy_stack


def test_diverging_island_returns_its_least_merit_iterate(orc):
    s = sliding_heavy_stack(5.0)
    p = dict(newton_iters=40, cr_iters=40, rscale=orc.R_NONE, tol_rel=1e-6, island_stop=1)
    plain = orc.Oracle(s, **p)
    sp = plain.step()
    assert sp["merit_final"] > sp["merit0"]              # the plain iteration diverges
    o = orc.Oracle(s, best_iterate=1, **p)
    st = o.step()
    hist = o.merit_history()
    heads = hist[:-1]                                     # merits of the evaluated iterates
    k = int(np.argmin(heads))
    assert st["merit_final"] == heads[k] == hist[-1]
    assert st["merit_final"] <= st["merit0"]
    np.testing.assert_array_equal(heads, plain.merit_history()[:-1])
    ref = orc.Oracle(s, **p)
    L = ref.linearize(n_before=k)
    u = o.dofs(o.get_state()["vel"], o.get_state()["omega"])
    np.testing.assert_array_equal(u, L["u"])
    np.testing.assert_array_equal(o.get_lambda(), L["lam"])


def test_converged_islands_unchanged(orc):
    s = scenes.batched_envs(seed=5, n_envs=8)
    p = dict(newton_iters=10, cr_iters=60, tol_rel=1e-6, island_stop=1, cone_project=1, line_search=1)
    a, b = orc.Oracle(s, **p), orc.Oracle(s, best_iterate=1, **p)
    a.step(); b.step()
    sa, sb = a.island_stats(), b.island_stats()
    np.testing.assert_array_equal(sa["stopped_at"], sb["stopped_at"])
    _, bi, _ = a.islands()
    done = sa["stopped_at"][bi] >= 0
    va, vb = a.get_state(), b.get_state()
    for k in ("vel", "omega", "pos", "quat"):
        np.testing.assert_array_equal(va[k][done], vb[k][done])
    # islands that did not stop: never worse than without the safeguard
    left = sa["stopped_at"] < 0
    assert np.all(sb["merit_final"][left] <= sa["merit_final"][left])
    assert np.all(sb["merit_final"] <= np.maximum(sa["merit_final"], sb["merit0"]))


def test_requires_island_mode(orc):
    with pytest.raises(ValueError):
        orc.Oracle(scenes.cube_stack(seed=0), best_iterate=1, island_stop=0)
