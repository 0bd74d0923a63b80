"""Prismatic joints and linear Hookean tets on the GPU against the FP64 oracle.

The GPU evaluates a linear tet as two blocks of three rows in the eigenbasis
of the isotropic stiffness (its compliance is diagonal there); the oracle
keeps the paper's strain rows and 6 x 6 compliance (Sec. 9.2.1).  Velocities
and net body impulses do not depend on the basis; the multipliers are
compared after rotating the GPU's back into the strain basis."""
import numpy as np
import pytest

from paper_1907_04587_gb300 import nsn, scenes

pytestmark = pytest.mark.gpu

H = 1.0 / 60.0
G = 9.81
R3, R2, R6 = 1 / np.sqrt(3), 1 / np.sqrt(2), 1 / np.sqrt(6)
# columns: the volumetric and the two deviatoric normal-strain modes
QN = np.array([[R3, R2, R6], [R3, -R2, R6], [R3, 0.0, -2 * R6]])


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    yield


def strain_basis(lam, s):
    """The GPU's multipliers with each linear tet's six rows rotated from the
    mode basis to the paper's strain basis (normal modes by QN, shears as they are)."""
    out = np.array(lam, np.float64)
    nl = len(s.get("l_v", ()))
    l0 = len(out) - 6 * nl
    for t in range(nl):
        r = l0 + 6 * t
        out[r:r + 3] = QN @ out[r:r + 3]
    return out


def body_impulse(o, lam):
    _, J = o.eval_constraints()
    return J.T @ (H * lam)


@pytest.mark.parametrize("prec,tol", [(nsn.NSN_FP64, 1e-9), (nsn.NSN_FP32, 1e-5)])
def test_slider_under_gravity(orc, prec, tol):
    """A body on a prismatic joint to the world, axis 30 degrees below the
    horizontal, 5 steps: v = k h (g . u) u and no rotation, as the oracle."""
    th = np.radians(30.0)
    u = (np.cos(th), 0.0, -np.sin(th))
    b = scenes.SceneBuilder()
    i = b.add_rigid((0.0, 0.0, 1.0), (1, 0, 0, 0), mass=2.0, inertia=(0.1, 0.2, 0.3))
    b.add_prismatic(i, -1, (0, 0, 0), (0.0, 0.0, 1.0), u, u, 0.0)
    s = b.build()
    p = dict(newton_iters=20, cr_iters=40, line_search=1, eps=0.0)
    o = orc.Oracle(s, **p)
    g = nsn.Solver(s, precision=prec, **p)
    for k in range(5):
        o.step(); g.step()
        vo, vg = o.get_state()["vel"][0], g.get_state_f64()["vel"][0]
        assert np.linalg.norm(vg - vo) <= tol * np.linalg.norm(vo), (k, vg, vo)
        assert np.abs(g.get_state_f64()["omega"][0]).max() < 10 * tol * G * H


def test_arm_and_linear_block_fp64_step_parity(orc):
    """Prismatic carriage + two revolute links + a linear Hookean block on the
    ground (contacts): FP64 build against the oracle at equal iteration counts,
    state re-synchronised every step: velocities, net body impulses, and the
    multipliers in the strain basis."""
    s = scenes.slider_arm_block(seed=1)
    p = dict(newton_iters=8, cr_iters=80, geom_stiffness=0)
    o = orc.Oracle(s, **p)
    g = nsn.Solver(s, precision=nsn.NSN_FP64, **p)
    assert g.R == o.R
    for k in range(3):
        st = o.get_state()
        f32 = {kk: v.astype(np.float32) for kk, v in st.items()}
        o.set_state(**{kk: v.astype(np.float64) for kk, v in f32.items()})
        g.set_state(**f32)
        o.step(); g.step()
        so, sg = o.get_state(), g.get_state_f64()
        du = max(np.abs(sg["vel"] - so["vel"]).max(), np.abs(sg["omega"] - so["omega"]).max())
        lo, lg = o.get_lambda(), strain_basis(g.get_lambda(), s)
        bo, bg = body_impulse(o, lo), body_impulse(o, lg)
        el = np.linalg.norm(lg - lo) / np.linalg.norm(lo)
        eb = np.linalg.norm(bg - bo) / np.linalg.norm(bo)
        print(f"step {k}: max |du| {du:.2e} body impulse {eb:.2e} multipliers {el:.2e}")
        assert du < 1e-8 and eb < 1e-7 and el < 1e-6


def test_arm_and_linear_block_fp32_converged(orc):
    """The same scene in FP32, islands to 1e-6 with the line search: both
    islands (arm, block) converge on both sides and agree to 1e-5."""
    s = scenes.slider_arm_block(seed=2)
    p = dict(newton_iters=30, cr_iters=200, tol_rel=1e-6, island_stop=1, line_search=1)
    o = orc.Oracle(s, **p)
    g = nsn.Solver(s, precision=nsn.NSN_FP32, **p)
    for k in range(3):
        o.step(); g.step()
        io, ig = o.island_stats()["stopped_at"], g.island_stats()["stopped_at"]
        assert np.all(io >= 0) and np.all(ig >= 0), (io, ig)
        so, sg = o.get_state(), g.get_state_f64()
        v = np.concatenate([so["vel"].ravel(), so["omega"].ravel()])
        dv = np.concatenate([(sg["vel"] - so["vel"]).ravel(), (sg["omega"] - so["omega"]).ravel()])
        e = np.linalg.norm(dv) / (np.linalg.norm(v) + H * G * np.sqrt(len(s["mass"])))
        print(f"step {k}: stop {ig.tolist()} / {io.tolist()}, velocity error {e:.2e}")
        assert e < 1e-5
        o.set_state(**{kk: vv.astype(np.float32).astype(np.float64) for kk, vv in sg.items()})
