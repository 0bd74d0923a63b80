"""Pins of the oracle's island mode and cone projection.

Islands are solved side by side (island_stop = 1): the Newton stop test, the
warm-start acceptance and the CR scalars are per island.  Because the Schur
operator of Eq. schur_system is block diagonal by island, the result for each
island must equal the result of solving that island by itself; that and the
connected components of a graph library are what these tests check against.
The cone projection (cone_project = 1) is not part of the paper; its pins are
that the iterates stay in the cone and that it does not move solutions.
"""
import numpy as np
import pytest

from paper_1907_04587_gb300 import scenes

BODY_KEYS = ("kind", "pos", "quat", "vel", "omega", "mass", "inertia", "env", "half")


def sub_scene(s, bodies):
    """The scene restricted to the given bodies (and the constraints on them)."""
    bodies = np.asarray(bodies)
    remap = -np.ones(len(s["mass"]), np.int64)
    remap[bodies] = np.arange(len(bodies))
    out = {k: (np.asarray(v)[bodies] if k in BODY_KEYS else v) for k, v in s.items()}
    for pre, keys in (("c", ("c_body", "c_pa", "c_pb", "c_n", "c_d", "c_mu")),
                      ("j", ("j_body", "j_pa", "j_pb", "j_axa", "j_axb", "j_compliance"))):
        ids = np.asarray(s[keys[0]])
        keep = np.isin(ids[:, 0], bodies) | np.isin(ids[:, 1], bodies)
        for k in keys:
            out[k] = np.asarray(s[k])[keep]
        ids = out[keys[0]]
        out[keys[0]] = np.where(ids >= 0, remap[np.maximum(ids, 0)], -1).astype(np.int32)
    return out


def test_islands_are_connected_components(orc):
    """Islands = connected components of the body graph (edges: constraints
    between two bodies; the static world is not a node)."""
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    s = scenes.batched_envs(seed=11, n_envs=3)
    o = orc.Oracle(s)
    ni, bi, ri = o.islands()
    nb = len(s["mass"])
    e = np.concatenate([s["c_body"], s["j_body"]])
    e = e[(e[:, 0] >= 0) & (e[:, 1] >= 0)]
    g = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(nb, nb))
    ncomp, lab = csg.connected_components(g, directed=False)
    assert ni == ncomp
    # same partition (labels may differ): bijection between label sets
    pairs = set(zip(bi.tolist(), lab.tolist()))
    assert len(pairs) == ni
    # islands are numbered by their lowest body
    firsts = [int(np.nonzero(bi == i)[0][0]) for i in range(ni)]
    assert firsts == sorted(firsts)
    # each row belongs to its constraint's island
    nc = len(s["c_body"])
    a = s["c_body"][:, 0]
    assert np.array_equal(ri[0:3 * nc:3], bi[a])


@pytest.mark.parametrize("proj", [0, 1])
def test_island_mode_equals_separate_solves(orc, proj):
    """Two environments solved together in island mode give, island by island,
    the states and stop iterations of each island solved by itself."""
    s = scenes.batched_envs(seed=5001, n_envs=2, links=(3, 5), boxes=(2, 20))
    prm = dict(newton_iters=25, cr_iters=60, tol_rel=1e-6, cr_tol_mode=1, island_stop=1, cone_project=proj)
    o = orc.Oracle(s, **prm)
    ni, bi, _ = o.islands()
    o.step()
    st = o.island_stats()
    full = o.get_state()
    assert (st["stopped_at"] >= 0).sum() >= ni // 2      # most islands converge in this budget
    for i in range(ni):
        bodies = np.nonzero(bi == i)[0]
        oi = orc.Oracle(sub_scene(s, bodies), **prm)
        assert oi.islands()[0] == 1
        oi.step()
        si = oi.island_stats()
        assert si["stopped_at"][0] == st["stopped_at"][i]
        part = oi.get_state()
        for k in ("pos", "quat", "vel", "omega"):
            np.testing.assert_allclose(part[k], full[k][bodies], rtol=0, atol=1e-12)
        np.testing.assert_allclose(si["merit0"][0], st["merit0"][i], rtol=1e-12)


def test_single_island_mode_equals_global_mode(orc):
    """With one island, island mode (per-island CR scalars) is the global method."""
    s = scenes.cube_stack(seed=3)
    prm = dict(newton_iters=6, cr_iters=15, tol_rel=1e-30)
    a = orc.Oracle(s, **prm)
    b = orc.Oracle(s, island_stop=1, **prm)
    ra, rb = a.step(), b.step()
    assert b.islands()[0] == 1
    np.testing.assert_allclose(a.merit_history(), b.merit_history(), rtol=1e-13, atol=0)
    for k in ("pos", "vel", "omega"):
        np.testing.assert_allclose(a.get_state()[k], b.get_state()[k], rtol=0, atol=1e-14)


def test_island_stop_reaches_tolerance(orc):
    """Every island that stopped did so at a merit <= tol_rel times its own
    zero-iterate merit, and its final merit (same iterate) agrees."""
    s = scenes.batched_envs(seed=5000, n_envs=2)
    o = orc.Oracle(s, newton_iters=30, cr_iters=50, tol_rel=1e-6, island_stop=1, cone_project=1)
    o.step()
    st = o.island_stats()
    done = st["stopped_at"] >= 0
    assert done.sum() >= len(done) // 2
    assert np.all(st["merit_final"][done] <= 1e-6 * st["merit0"][done] * (1 + 1e-9))


def test_cone_projection_keeps_iterates_in_cone(orc):
    s = scenes.batched_envs(seed=7, n_envs=2)
    o = orc.Oracle(s, newton_iters=8, cr_iters=40, cone_project=1)
    o.step()
    lam = o.get_lambda()
    nc = len(s["c_body"])
    ln = lam[0:3 * nc:3]
    lf = np.hypot(lam[1:3 * nc:3], lam[2:3 * nc:3])
    assert np.all(ln >= 0)
    assert np.all(lf <= s["c_mu"] * ln * (1 + 1e-12) + 1e-300)


def test_cone_projection_does_not_move_solutions(orc):
    """On a scene where the printed method converges, the projected iteration
    converges to the same state (the NCP solutions lie in the cone)."""
    s = scenes.cube_stack(seed=1)
    a = orc.Oracle(s, newton_iters=40, cr_iters=60)
    b = orc.Oracle(s, newton_iters=40, cr_iters=60, cone_project=1)
    ra, rb = a.step(), b.step()
    assert ra["merit_final"] <= 1e-12 * ra["merit0"] and rb["merit_final"] <= 1e-12 * rb["merit0"]
    for k in ("pos", "vel", "omega"):
        np.testing.assert_allclose(a.get_state()[k], b.get_state()[k], rtol=0, atol=1e-10)


def test_cone_projection_separating_slider(orc):
    """A link held by a hard revolute joint with its corners touching the
    ground (C_n = 0) spins: the contacts carry no load at the solution.  Under
    the printed damped iteration lambda_n decays geometrically while the lagged
    friction compliance grows like 1/lambda_n, so the friction residual grows;
    with the projection the merit falls at the damped rate 1 - t per
    iteration."""
    s = scenes.batched_envs(seed=5000, n_envs=1, boxes=(0, 0), links=(1, 1))
    a = orc.Oracle(s, newton_iters=10, cr_iters=100)
    b = orc.Oracle(s, newton_iters=10, cr_iters=100, cone_project=1)
    ra, rb = a.step(), b.step()
    ha, hb = a.merit_history() / ra["merit0"], b.merit_history() / rb["merit0"]
    assert ha[10] > 1.0                   # the printed iteration has diverged
    assert hb[10] < 2e-6                  # 0.25^10 ~ 1e-6
    lam = b.get_lambda()
    assert np.all(np.abs(lam[:12]) < 1e-6 * s["mass"][0] * 9.81)
