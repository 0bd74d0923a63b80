"""The FEM scenes' contacts regenerated by the oracle's collider at the start
state (Sec. 3.3: a contact wherever two features come within the margin; a
point on a deformable body is a particle position).  The generated sets must
hold the scenes' hand-built contacts and nothing that the scenes' geometry
rules out: boxes of different columns of the bin never touch, and a
deformable body meets the rigid shapes and planes through its vertices."""
import numpy as np

import oracle as orc
from paper_1907_04587_gb300 import scenes

H = 1.0 / 60.0
GRAV = np.float32(H) * np.array([0.0, 0.0, -9.81], np.float32)


def collide(s):
    jb = np.asarray(s["j_body"])
    exclude = jb[(jb[:, 0] >= 0) & (jb[:, 1] >= 0)] if len(jb) else np.zeros((0, 2), np.int32)
    return orc.collide(s["kind"], s["pos"], s["quat"], (s["vel"] + GRAV).astype(np.float32), s["omega"], s["half"],
                       s["env"], s["planes"], exclude, s["mu_env"], 0.01, H)


def separation(s, co):
    """n^T (a - b) per contact at the start state, a and b in world frame."""
    R = scenes.quat_rot(s["quat"].astype(np.float64))
    def world(body, p):
        out = p.copy()
        rig = (body >= 0)
        idx = body[rig]
        pr = s["pos"][idx].astype(np.float64)
        out[rig] = np.where((s["kind"][idx] == 0)[:, None], pr + np.einsum("kij,kj->ki", R[idx], p[rig]), pr)
        return out
    a = world(co["c_body"][:, 0], co["c_pa"])
    b = world(co["c_body"][:, 1], co["c_pb"])
    return np.einsum("ki,ki->k", co["c_n"], a - b)


def pairs(cb):
    return set(map(tuple, np.asarray(cb).tolist()))


def test_bin_columns_touch_only_within_a_column():
    n_boxes = 400
    s = scenes.mixed_bin(seed=0, n_boxes=n_boxes, n_spheres=2, sphere_res=6)
    n_cols = int(np.ceil(n_boxes / 4))
    co = collide(s)
    cb = co["c_body"]
    a, b = cb[:, 0], cb[:, 1]
    boxes = (a < n_boxes) & (b >= 0)
    assert (b[boxes] < n_boxes).all()                          # boxes touch boxes or planes only
    assert ((a[boxes] % n_cols) == (b[boxes] % n_cols)).all()  # ... of their own column
    # a box rests wholly on the one beneath: its four bottom corners are
    # generated against it, as the hand-built contacts have them
    hb = s["c_body"][s["c_body"][:, 0] < n_boxes]
    assert pairs(hb) <= pairs(cb)
    for (ai, bi) in pairs(hb):
        if bi >= 0:
            assert ((a == ai) & (b == bi)).sum() >= 4
    # the balls' vertices meet the floor and the x = 0 wall only
    balls = a >= n_boxes
    assert (b[balls] == -1).all()
    assert pairs(s["c_body"][s["c_body"][:, 0] >= n_boxes]) <= pairs(cb[balls])
    assert np.isin(co["c_n"][balls].round(6).tolist(), [0.0, 1.0]).all()
    # no box starts inside another or below the floor
    assert separation(s, co).min() > -1e-6


def test_chain_block_contacts_are_block_vertices():
    links = 7
    s = scenes.chain_block(seed=0, hexes=6, links=links)
    co = collide(s)
    cb = co["c_body"]
    assert (cb[:, 0] >= links).all()                           # a: a particle of the block
    assert ((cb[:, 1] == -1) | (cb[:, 1] < links)).all()       # b: the ground or a link
    assert pairs(s["c_body"]) <= pairs(cb)
    top = (cb[:, 1] >= 0)
    np.testing.assert_allclose(co["c_n"][top], np.tile((0.0, 0.0, -1.0), (top.sum(), 1)), atol=1e-6)
