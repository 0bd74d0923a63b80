"""Pins of the oracle's contact generation (Sec. 3.3: contacts are created
when features come within a fixed distance; Sec. 10: candidates from the
unconstrained velocity, normals between closest points at the start of the
step).  Checked against closed forms, a bounded least-squares library routine
for the closest point on a box, the hand-built contacts of the synthetic
scenes, and invariants of the generated geometry."""
import numpy as np
import pytest

import oracle
from paper_1907_04587_gb300 import scenes

H = 1.0 / 60.0
Z_PLANE = [[0.0, 0.0, 1.0, 0.0]]
FP64_DECISIONS = False


@pytest.fixture(autouse=True, params=[False, True], ids=["fp32-decisions", "fp64-decisions"])
def decisions(request):
    """Every pin below holds for both versions of the oracle's contact
    generation: decisions in FP32 (the GPU's order of rounded operations) and
    the plain FP64 definition."""
    global FP64_DECISIONS
    FP64_DECISIONS = request.param
    yield request.param
    FP64_DECISIONS = False


def run(bodies, planes=Z_PLANE, exclude=None, mu=(0.5,), margin=0.01, h=H):
    b = {k: np.asarray(v) for k, v in bodies.items()}
    nb = len(b["kind"])
    z3 = np.zeros((nb, 3))
    return oracle.collide(b["kind"], b["pos"], b.get("quat", np.tile([1.0, 0, 0, 0], (nb, 1))),
                          b.get("vel", z3), b.get("omega", z3), b.get("half", z3),
                          b.get("env", np.zeros(nb, np.int32)), planes, exclude, mu, margin, h,
                          fp64_decisions=FP64_DECISIONS)


def world(pos, quat, local):
    return np.asarray(pos, np.float64) + scenes.quat_rot(np.asarray(quat, np.float64)[None])[0] @ local


def test_unit_cube_resting_on_plane():
    """A unit cube 0.1 mm above z = 0: its 4 bottom corners and nothing else,
    each with the plane normal and the corner's foot point."""
    r = run(dict(kind=[0], pos=[[0.3, -0.2, 0.5 + 1e-4]], half=[[0.5, 0.5, 0.5]]))
    assert r["c_body"].tolist() == [[0, -1]] * 4
    np.testing.assert_array_equal(r["c_pa"], [[-.5, -.5, -.5], [.5, -.5, -.5], [-.5, .5, -.5], [.5, .5, -.5]])
    np.testing.assert_allclose(r["c_pb"], [[-.2, -.7, 0], [.8, -.7, 0], [-.2, .3, 0], [.8, .3, 0]], atol=1e-7)
    np.testing.assert_array_equal(r["c_n"], np.tile([0.0, 0.0, 1.0], (4, 1)))
    np.testing.assert_array_equal(r["c_d"], 0.0)
    np.testing.assert_allclose(r["c_mu"], 0.5)


@pytest.mark.parametrize("vz,expect", [(0.0, 0), (-6.0, 4), (-2.0, 0), (6.0, 0)])
def test_candidates_from_the_unconstrained_velocity(vz, expect):
    """A cube 5 cm above the plane, margin 1 cm: it is a candidate only if its
    predicted position p + h u comes within the margin (v h = -0.1 m yes,
    -0.033 m no)."""
    r = run(dict(kind=[0], pos=[[0, 0, 0.55]], half=[[0.5, 0.5, 0.5]], vel=[[0, 0, vz]]))
    assert len(r["c_body"]) == expect


def test_rotation_moves_only_one_side_down():
    """Spin about +x at 12 rad/s: the corner velocity w x r has z component
    12 y, so corners at y = -0.5 move down by h 6 = 0.1 m (into the 5 cm gap),
    those at y = +0.5 move up."""
    r = run(dict(kind=[0], pos=[[0, 0, 0.55]], half=[[0.5, 0.5, 0.5]], omega=[[12.0, 0, 0]]))
    assert len(r["c_pa"]) == 2
    assert np.all(r["c_pa"][:, 1] == -0.5) and np.all(r["c_pa"][:, 2] == -0.5)


def test_particle_on_plane_and_wall():
    """A particle 2 mm from the floor and 5 mm from the wall x = 0 (solid side
    x < 0): one contact per plane, foot points and normals of each plane."""
    r = run(dict(kind=[1], pos=[[0.005, 0.3, 0.002]]), planes=[[0, 0, 1, 0], [1, 0, 0, 0]])
    assert r["c_body"].tolist() == [[0, -1], [0, -1]]
    np.testing.assert_allclose(r["c_pb"], [[0.005, 0.3, 0.0], [0.0, 0.3, 0.002]], atol=1e-9)
    np.testing.assert_array_equal(r["c_n"], [[0, 0, 1], [1, 0, 0]])
    np.testing.assert_array_equal(r["c_pa"], 0.0)


def test_closest_point_on_a_rotated_box_matches_bounded_least_squares():
    """Particles around a rotated box, within the margin: the closest point is
    argmin |x_b + R u - p| over -e <= u <= e (scipy's bounded least squares),
    and the normal is the unit vector from it to the particle."""
    lsq = pytest.importorskip("scipy.optimize").lsq_linear
    rng = np.random.default_rng(3)
    q = np.array([0.9, 0.2, -0.3, 0.25]); q /= np.linalg.norm(q)
    xb, e = np.array([0.1, -0.2, 0.8]), np.array([0.3, 0.2, 0.1])
    R = scenes.quat_rot(q[None])[0]
    pts = xb + (R @ (rng.uniform(-1.6, 1.6, (400, 3)) * e).T).T
    n = len(pts)
    bodies = dict(kind=np.r_[0, np.ones(n, int)], pos=np.r_[[xb], pts],
                  quat=np.r_[[q], np.tile([1.0, 0, 0, 0], (n, 1))], half=np.r_[[e], np.zeros((n, 3))])
    r = run(bodies, planes=[], margin=0.15)
    got = {int(a): i for i, (a, b) in enumerate(r["c_body"]) if b == 0}
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    Rf = scenes.quat_rot(f32(q)[None])[0]
    checked = 0
    for k in range(n):
        p = f32(pts[k])
        sol = lsq(Rf, p - f32(xb), bounds=(-f32(e), f32(e)), method="bvls", tol=1e-14)
        dist = np.linalg.norm(Rf @ sol.x - (p - f32(xb)))
        inside = np.all(np.abs(Rf.T @ (p - f32(xb))) <= f32(e))
        if inside or abs(dist - 0.15) < 1e-4:
            continue                     # inside: pinned below; near the margin: FP32 decides
        assert (k + 1 in got) == (dist < 0.15), (k, dist)
        if dist < 0.15:
            i = got[k + 1]
            # the library solution is accurate to a few 1e-9 m
            np.testing.assert_allclose(r["c_pb"][i], sol.x, atol=1e-7)
            np.testing.assert_allclose(r["c_n"][i], (p - f32(xb) - Rf @ sol.x) / dist, atol=1e-7 / dist)
            checked += 1
    assert checked > 50


def test_inside_point_takes_the_face_of_least_penetration():
    """A particle inside a rotated box, nearest to the +y face: the contact is
    on that face, with normal R e_y and depth e_y - q_y."""
    q = scenes.quat_yaw(0.4)
    R = scenes.quat_rot(np.asarray(q, np.float64)[None])[0]
    e = np.array([0.3, 0.2, 0.1])
    loc = np.array([0.05, 0.17, -0.02])
    p = world([1, 2, 0.5], q, loc)
    r = run(dict(kind=[0, 1], pos=[[1, 2, 0.5], p], quat=[q, [1, 0, 0, 0]], half=[e, [0, 0, 0]]), planes=[])
    assert r["c_body"].tolist() == [[1, 0]]
    np.testing.assert_allclose(r["c_pb"][0], [0.05, 0.2, -0.02], atol=1e-6)
    np.testing.assert_allclose(r["c_n"][0], R[:, 1], atol=1e-7)
    bw = world([1, 2, 0.5], q, r["c_pb"][0])
    assert abs(r["c_n"][0] @ (p - bw) + 0.03) < 1e-6       # signed gap = -depth


def test_exclusions_environments_and_shapes():
    """Two overlapping boxes: contacts both ways when in one environment;
    none between them when the pair is excluded (a joint) or in different
    environments; a rigid body without a shape has no vertices."""
    bodies = dict(kind=[0, 0], pos=[[0, 0, 2.0], [0.15, 0, 2.0]], half=[[0.1, 0.1, 0.1]] * 2)
    r = run(bodies)
    assert {tuple(x) for x in r["c_body"]} == {(0, 1), (1, 0)}
    assert len(run(bodies, exclude=[[1, 0]])["c_body"]) == 0
    assert len(run(dict(bodies, env=[0, 1]), mu=(0.5, 0.5))["c_body"]) == 0
    assert run(dict(bodies, half=[[0.1, 0.1, 0.1], [0, 0, 0]]))["c_body"].tolist() == []
    # outputs are ordered by body, corner, then planes before boxes
    r = run(dict(kind=[0, 0], pos=[[0, 0, 0.1], [0.15, 0, 0.1]], half=[[0.1, 0.1, 0.1]] * 2))
    key = [(a, int(np.dot((r["c_pa"][i] > 0), [1, 2, 4])), b if b >= 0 else -9) for i, (a, b) in enumerate(r["c_body"])]
    assert key == sorted(key)


def test_scene_contacts_are_reproduced():
    """The synthetic batched scenes place every link and box bottom corner on
    the ground or on the box below: the generator finds each such contact
    (with the scenes' normal and foot point) wherever the corner lies over the
    supporting box's top face (away from its edges, where a sunk corner is
    nearer to a side face); corners overhanging it are not in contact."""
    s = scenes.batched_envs(seed=5, n_envs=8)
    jb = s["j_body"][s["j_body"][:, 1] >= 0]
    r = oracle.collide(s["kind"], s["pos"], s["quat"], s["vel"], s["omega"], s["half"], s["env"], Z_PLANE, jb,
                       np.full(8, 0.5), 0.01, H, fp64_decisions=FP64_DECISIONS)
    gen = {}
    for i, ((a, b), pa) in enumerate(zip(r["c_body"], r["c_pa"])):
        gen[(int(a), int(b), tuple(np.sign(pa).astype(int)))] = i
    found = over = 0
    R = scenes.quat_rot(s["quat"].astype(np.float64))
    for (a, b), pa, pb, n in zip(s["c_body"], s["c_pa"], s["c_pb"], s["c_n"]):
        key = (int(a), int(b), tuple(np.sign(pa).astype(int)))
        if b >= 0:
            w = s["pos"][a] + R[a] @ pa
            loc = R[b].T @ (w - s["pos"][b])
            # a corner sunk into the box below (up to 1 mm, the scenes' jitter)
            # and closer than that to a side face is nearest to the side face
            if np.any(np.abs(loc[:2]) > s["half"][b][:2] - 2e-3):
                over += 1
                if np.any(np.abs(loc[:2]) > s["half"][b][:2] + 0.02):
                    assert key not in gen
                continue
        assert key in gen, key
        i = gen[key]
        np.testing.assert_allclose(r["c_n"][i], n, atol=1e-6)
        np.testing.assert_allclose(r["c_pa"][i], pa, atol=0)
        np.testing.assert_allclose(r["c_pb"][i][:2] if b < 0 else r["c_pb"][i], pb[:2] if b < 0 else pb, atol=2e-6)
        found += 1
    print("reproduced", found, "overhanging or at an edge", over, "of", len(s["c_body"]))
    assert found > 0.6 * len(s["c_body"]) and over > 0


def test_generated_geometry_invariants():
    """Random boxes and particles with random velocities: every contact's
    normal is unit; n.(a - b) is the signed distance of the vertex to the
    shape at the start of the step (the plane's value; for a box, the distance
    to the closest point outside, minus the least penetration inside); every
    vertex within the margin at the start of the step is a candidate."""
    rng = np.random.default_rng(11)
    nb, npart = 60, 40
    pos = np.c_[rng.uniform(-0.6, 0.6, (nb + npart, 2)), rng.uniform(0.0, 0.5, nb + npart)]
    q = rng.normal(size=(nb + npart, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[nb:] = (1, 0, 0, 0)
    half = np.r_[rng.uniform(0.03, 0.12, (nb, 3)), np.zeros((npart, 3))]
    kind = np.r_[np.zeros(nb, int), np.ones(npart, int)]
    vel = rng.normal(scale=0.5, size=(nb + npart, 3))
    om = np.r_[rng.normal(scale=2.0, size=(nb, 3)), np.zeros((npart, 3))]
    r = run(dict(kind=kind, pos=pos, quat=q, half=half, vel=vel, omega=om), margin=0.02)
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    pos, q, half, R = f(pos), f(q), f(half), scenes.quat_rot(f(q))
    assert len(r["c_body"]) > 100
    np.testing.assert_allclose(np.linalg.norm(r["c_n"], axis=1), 1.0, atol=1e-12)
    for (a, b), pa, pb, n in zip(r["c_body"], r["c_pa"], r["c_pb"], r["c_n"]):
        p = pos[a] + (R[a] @ pa if kind[a] == 0 else 0)
        if b < 0:
            assert abs(n @ (p - pb) - p[2]) < 1e-12
            continue
        loc = R[b].T @ (p - pos[b])
        out = np.maximum(np.abs(loc) - half[b], 0)
        sd = np.linalg.norm(out) if out.any() else -np.min(half[b] - np.abs(loc))
        # R of an FP32 quaternion is orthogonal to ~1e-7
        assert abs(n @ (p - (pos[b] + R[b] @ pb)) - sd) < 1e-6
    # completeness at the start of the step: vertex-plane and vertex-box
    have = {(int(a), int(b), tuple(np.round(pa, 6))) for (a, b), pa in zip(r["c_body"], r["c_pa"])}
    corners = np.array([[(k >> i & 1) * 2 - 1 for i in range(3)] for k in range(8)], np.float64)
    for a in range(nb + npart):
        verts = [(half[a] * c, pos[a] + R[a] @ (half[a] * c)) for c in corners] if kind[a] == 0 else [(np.zeros(3), pos[a])]
        for pa, p in verts:
            if p[2] < 0.02 - 1e-6:
                assert (a, -1, tuple(np.round(pa, 6))) in have
            for b in range(nb):
                if b == a:
                    continue
                loc = R[b].T @ (p - pos[b])
                d = np.linalg.norm(np.maximum(np.abs(loc) - half[b], 0))
                if d < 0.02 - 1e-6:
                    assert (a, b, tuple(np.round(pa, 6))) in have


def test_relative_velocity_and_plane_offset():
    """The prediction uses the vertex's velocity relative to the shape: a
    resting particle 5 cm above a box that rises at 6 m/s is a candidate, and
    not when the box sinks; a plane n.x = 0.1 puts the foot point at z = 0.1."""
    base = dict(kind=[0, 1], pos=[[0, 0, 0.0], [0.01, 0.02, 0.15]], half=[[0.2, 0.2, 0.1], [0, 0, 0]])
    up = run(dict(base, vel=[[0, 0, 6.0], [0, 0, 0]]), planes=[])
    assert up["c_body"].tolist() == [[1, 0]]
    np.testing.assert_allclose(up["c_pb"][0], [0.01, 0.02, 0.1], atol=1e-7)
    np.testing.assert_allclose(up["c_n"][0], [0, 0, 1], atol=1e-12)
    assert len(run(dict(base, vel=[[0, 0, -6.0], [0, 0, 0]]), planes=[])["c_body"]) == 0
    r = run(dict(kind=[1], pos=[[0.3, 0.4, 0.105]]), planes=[[0, 0, 1, 0.1]])
    np.testing.assert_allclose(r["c_pb"], [[0.3, 0.4, 0.1]], atol=1e-7)
    assert len(run(dict(kind=[1], pos=[[0.3, 0.4, 0.115]]), planes=[[0, 0, 1, 0.1]])["c_body"]) == 0


@pytest.mark.parametrize("which", ["batched", "particles_and_boxes"])
def test_fp32_decisions_differ_from_the_fp64_definition_only_within_rounding(which, decisions):
    """The FP32 decisions (the GPU's) against the plain FP64 definition on
    scenes whose vertices rest on planes and boxes (many decisions sit near
    the margin or on a face tie): a pair present in one list only lies within
    4 FP32 units of the coordinates' scale of the margin, a normal that changes
    face belongs to a tie within the same band, other normals differ only by
    the rotation's rounding, and geometry of the common pairs agrees."""
    if decisions:
        pytest.skip("compares the two versions once")
    import collide_band
    if which == "batched":
        s = scenes.batched_envs(seed=1, n_envs=512)
        planes = Z_PLANE
        n_envs = 512
    else:
        rng = np.random.default_rng(11)
        b = scenes.SceneBuilder()
        for i in range(300):
            if i % 3:
                b.add_particle(rng.uniform([-1, -1, -0.01], [1, 1, 0.3]), vel=rng.normal(scale=0.3, size=3))
            else:
                q = scenes.quat_axis_angle(rng.normal(size=3), rng.uniform(0, np.pi))
                b.add_rigid(rng.uniform([-1, -1, 0.0], [1, 1, 0.3]), q, vel=rng.normal(scale=0.3, size=3),
                            omega=rng.normal(scale=1.0, size=3))
        s = b.build()
        s["half"] = np.where((s["kind"] == 0)[:, None], rng.uniform(0.05, 0.2, (len(s["kind"]), 3)), 0.0)
        planes = [[0.0, 0.0, 1.0, 0.0], [0.6, 0.0, 0.8, 0.3]]
        n_envs = 1
    ex = s["j_body"][(s["j_body"] >= 0).all(1)] if len(s["j_body"]) else None
    args = (s["kind"], s["pos"], s["quat"], s["vel"], s["omega"], s["half"], s["env"], planes, ex,
            np.full(n_envs, 0.5), 0.01, H)
    A = oracle.collide(*args)
    B = oracle.collide(*args, fp64_decisions=True)
    r = collide_band.compare(s, A, B, planes, 0.01, H)
    assert r["membership"] <= 4 and r["face"] <= 4 and r["normal"] <= 4, r
    assert r["n_common"] >= 0.999 * max(len(A["c_body"]), len(B["c_body"])), r
    ka, kb = collide_band.contact_keys(A, planes), collide_band.contact_keys(B, planes)
    same = [(ka[k], kb[k]) for k in set(ka) & set(kb)
            if np.abs(A["c_n"][ka[k]] - B["c_n"][kb[k]]).max() < 1e-6]
    ia, ib = np.array(same).T
    np.testing.assert_allclose(A["c_pb"][ia], B["c_pb"][ib], rtol=0, atol=1e-6)
    print(which, r)
