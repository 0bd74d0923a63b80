"""orc_merit_at: the merit ||[g; h]|| of Sec. 8.1 at a given iterate of a step.

Pins: a particle resting on a frictionless plane has the closed-form solution
u = 0, lambda_n = m g (g = M(u - u~) - h J^T lambda vanishes, the
Fischer-Burmeister row FB(C, r lambda) = 0 at C = 0), so the merit there is 0;
at u = 0, lambda = 0 it is |M u~| = m g h; a vertical velocity error dv adds
m dv to g.  At the zero iterate and at the iterate a step returns, the value
equals the step's own zero-iterate and final merits, per island too."""
import numpy as np

from paper_1907_04587_gb300 import scenes

H, G = 1.0 / 60.0, 9.81


def resting_particle(mass=2.0):
    b = scenes.SceneBuilder()
    i = b.add_particle((0.0, 0.0, 0.0), vel=(0.0, 0.0, 0.0), mass=mass)
    b.add_contact(i, -1, (0, 0, 0), (0, 0, 0), (0, 0, 1), 0.0, 0.0)
    return b.build()


def test_closed_form_resting_particle(orc):
    m = 2.0
    o = orc.Oracle(resting_particle(m), newton_iters=4, cr_iters=10)
    v0, w0 = np.zeros((1, 3)), np.zeros((1, 3))
    exact, _ = o.merit_at(v0, w0, [m * G, 0.0, 0.0])
    assert exact < 1e-12 * m * G * H
    zero, _ = o.merit_at(v0, w0, [0.0, 0.0, 0.0])
    assert abs(zero - m * G * H) < 1e-12 * m * G * H
    dv = 1e-3
    # moving up by dv: g = m dv e_z, and the contact row FB(C, r lambda) with
    # the gap C = h dv > 0 and lambda = m g: FB(h dv, r m g) (r > 0) -- only
    # the momentum part has a closed form, so check it bounds the merit below
    up, _ = o.merit_at(np.array([[0.0, 0.0, dv]]), w0, [m * G, 0.0, 0.0])
    assert up >= m * dv * (1 - 1e-12)
    # the state is left as it was
    st = o.get_state()
    assert np.all(st["pos"] == 0.0) and np.all(st["vel"] == 0.0)


def test_matches_the_step_merits(orc):
    s = scenes.batched_envs(seed=4, n_envs=6)
    o = orc.Oracle(s, newton_iters=8, cr_iters=60, tol_rel=1e-6, island_stop=1, cone_project=1, line_search=1)
    pre = o.get_state()
    nr = o.R
    m0, isl0 = o.merit_at(np.zeros_like(pre["vel"]), np.zeros_like(pre["omega"]), np.zeros(nr))
    st = o.step()
    stats = o.island_stats()
    post, lam = o.get_state(), o.get_lambda()
    assert abs(m0 - st["merit0"]) <= 1e-12 * st["merit0"]
    np.testing.assert_allclose(isl0, stats["merit0"], rtol=1e-12)
    o.set_state(**pre)
    mf, islf = o.merit_at(post["vel"], post["omega"], lam)
    assert abs(mf - st["merit_final"]) <= 1e-9 * st["merit0"]
    np.testing.assert_allclose(islf, stats["merit_final"], rtol=1e-9, atol=1e-12 * st["merit0"])
