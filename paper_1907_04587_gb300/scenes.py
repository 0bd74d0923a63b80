"""Seeded synthetic scenes shaped like the paper's workloads (Sec. 10, Table 2).

This module holds input generation only -- geometry, masses and contact
generation -- and none of the solver's arithmetic.  Both the CUDA library and
the FP64 oracle consume the dictionaries it returns.  Every float is rounded to
float32 so that the FP32 device path and the FP64 oracle see identical values.

Scene dictionary (numpy arrays):
  kind[nb] (0 rigid, 1 particle), pos[nb,3], quat[nb,4] (w,x,y,z), vel[nb,3],
  omega[nb,3] (world frame), mass[nb], inertia[nb,3] (body-frame principal),
  env[nb] (environment id, 0 for single scenes), mu_env[n_envs] (friction of
  each environment, batched scenes), half[nb,3] (box half extents
  of a rigid body's collision shape; zeros: no shape, and for particles)
  c_body[nc,2] (-1 = static world), c_pa[nc,3], c_pb[nc,3] (body-local, or a
  world point for the world side), c_n[nc,3] (world normal from b to a),
  c_d[nc], c_mu[nc]
  j_body[nj,2], j_pa[nj,3], j_pb[nj,3], j_axa[nj,3], j_axb[nj,3], j_compliance[nj],
  j_kind[nj] (optional: 0 revolute, 1 prismatic)
  t_v[nt,4], t_rest[nt,4,3], t_E[nt], t_nu[nt]  (stable Neo-Hookean tets)
  l_v[nl,4], l_rest[nl,4,3], l_E[nl], l_nu[nl]  (optional: linear Hookean tets)

Workloads (the paper's scenes need URDFs and meshes that are not available, so
these stand in for them):
  cube_stack     -- 4 unit cubes stacked on a plane, 16 vertex contacts
  chain_block    -- 7-link revolute chain resting on a Neo-Hookean tet block
  batched_envs   -- thousands of uneven chain + box-pile environments
"""
from __future__ import annotations

import numpy as np

RIGID, PARTICLE = 0, 1
F32 = np.float32


def quat_yaw(theta):
    theta = np.asarray(theta, dtype=np.float64)
    return np.stack([np.cos(theta / 2), np.zeros_like(theta), np.zeros_like(theta), np.sin(theta / 2)], -1)


def quat_axis_angle(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[np.cos(angle / 2)], np.sin(angle / 2) * axis])


def quat_rot(q):
    """Rotation matrices of (..., 4) quaternions (w, x, y, z) -> (..., 3, 3)."""
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)
    return R.reshape(q.shape[:-1] + (3, 3))


def box_inertia(m, dims):
    a, b, c = dims
    return np.array([m * (b * b + c * c) / 12, m * (a * a + c * c) / 12, m * (a * a + b * b) / 12])


def box_bottom_corners(dims):
    a, b, c = np.asarray(dims, dtype=np.float64) / 2
    return np.array([[-a, -b, -c], [a, -b, -c], [a, b, -c], [-a, b, -c]])


class SceneBuilder:
    """Incremental scene assembly; ``build()`` returns the float32 dictionary."""

    def __init__(self):
        self.b = {k: [] for k in ("kind", "pos", "quat", "vel", "omega", "mass", "inertia", "env")}
        self.c = {k: [] for k in ("c_body", "c_pa", "c_pb", "c_n", "c_d", "c_mu")}
        self.j = {k: [] for k in ("j_body", "j_pa", "j_pb", "j_axa", "j_axb", "j_compliance", "j_kind")}
        self.t = {k: [] for k in ("t_v", "t_rest", "t_E", "t_nu")}
        self.l = {k: [] for k in ("l_v", "l_rest", "l_E", "l_nu")}

    @property
    def n_bodies(self):
        return len(self.b["mass"])

    def add_rigid(self, pos, quat=(1, 0, 0, 0), vel=(0, 0, 0), omega=(0, 0, 0), mass=1.0,
                  inertia=(1, 1, 1), env=0):
        self.b["kind"].append(RIGID); self.b["pos"].append(pos); self.b["quat"].append(quat)
        self.b["vel"].append(vel); self.b["omega"].append(omega); self.b["mass"].append(mass)
        self.b["inertia"].append(inertia); self.b["env"].append(env)
        return self.n_bodies - 1

    def add_particle(self, pos, vel=(0, 0, 0), mass=1.0, env=0):
        self.b["kind"].append(PARTICLE); self.b["pos"].append(pos); self.b["quat"].append((1, 0, 0, 0))
        self.b["vel"].append(vel); self.b["omega"].append((0, 0, 0)); self.b["mass"].append(mass)
        self.b["inertia"].append((1, 1, 1)); self.b["env"].append(env)
        return self.n_bodies - 1

    def add_contact(self, a, b, pa, pb, n, d=0.0, mu=0.5):
        self.c["c_body"].append((a, b)); self.c["c_pa"].append(pa); self.c["c_pb"].append(pb)
        self.c["c_n"].append(n); self.c["c_d"].append(d); self.c["c_mu"].append(mu)

    def add_revolute(self, a, b, pa, pb, axa, axb, compliance=0.0):
        self.j["j_body"].append((a, b)); self.j["j_pa"].append(pa); self.j["j_pb"].append(pb)
        self.j["j_axa"].append(axa); self.j["j_axb"].append(axb); self.j["j_compliance"].append(compliance)
        self.j["j_kind"].append(0)

    def add_prismatic(self, a, b, pa, pb, axa, axb, compliance=0.0):
        """Slider: a's anchor pa stays on the line through b's anchor pb along
        b's axis axb, with a's axis axa kept along it and no twist about it."""
        self.add_revolute(a, b, pa, pb, axa, axb, compliance)
        self.j["j_kind"][-1] = 1

    def add_tet(self, v, rest, E, nu):
        self.t["t_v"].append(v); self.t["t_rest"].append(rest); self.t["t_E"].append(E); self.t["t_nu"].append(nu)

    def add_linear_tet(self, v, rest, E, nu):
        """Constant-strain tet with a linear Hookean material (Sec. 9.2.1)."""
        self.l["l_v"].append(v); self.l["l_rest"].append(rest); self.l["l_E"].append(E); self.l["l_nu"].append(nu)

    def build(self):
        shapes = dict(kind=(0,), pos=(0, 3), quat=(0, 4), vel=(0, 3), omega=(0, 3), mass=(0,), inertia=(0, 3),
                      env=(0,), c_body=(0, 2), c_pa=(0, 3), c_pb=(0, 3), c_n=(0, 3), c_d=(0,), c_mu=(0,),
                      j_body=(0, 2), j_pa=(0, 3), j_pb=(0, 3), j_axa=(0, 3), j_axb=(0, 3), j_compliance=(0,),
                      j_kind=(0,), t_v=(0, 4), t_rest=(0, 4, 3), t_E=(0,), t_nu=(0,),
                      l_v=(0, 4), l_rest=(0, 4, 3), l_E=(0,), l_nu=(0,))
        out = {}
        for grp in (self.b, self.c, self.j, self.t, self.l):
            for k, v in grp.items():
                ints = k in ("kind", "env", "c_body", "j_body", "j_kind", "t_v", "l_v")
                dt = np.int32 if ints else np.float64
                a = np.asarray(v, dtype=dt) if len(v) else np.zeros(shapes[k], dtype=dt)
                out[k] = a
        return finalize(out)


def finalize(s):
    """Round floats to float32, normalise quaternions/normals in float32."""
    out = {}
    for k, v in s.items():
        if isinstance(v, np.ndarray) and v.dtype.kind == "f":
            out[k] = np.ascontiguousarray(v.astype(F32))
        elif isinstance(v, np.ndarray):
            out[k] = np.ascontiguousarray(v.astype(np.int32))
        else:
            out[k] = v
    if len(out["quat"]):
        q = out["quat"].astype(np.float64)
        out["quat"] = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(F32)
    if len(out["c_n"]):
        n = out["c_n"].astype(np.float64)
        out["c_n"] = (n / np.linalg.norm(n, axis=1, keepdims=True)).astype(F32)
    if "env" not in out:
        out["env"] = np.zeros(len(out["mass"]), np.int32)
    out["n_envs"] = int(out["env"].max()) + 1 if len(out["env"]) else 1
    return out


def scene_counts(s):
    return dict(nb=len(s["mass"]), nc=len(s["c_body"]), nj=len(s["j_body"]), nt=len(s["t_v"]),
                rows=3 * len(s["c_body"]) + 5 * len(s["j_body"]) + 3 * len(s["t_v"]))


# --------------------------------------------------------------------------------------
# Workload 1: stack of unit cubes (rigid contact, Fig. 13 shape)

def stack_contacts(pos, quat, edge=1.0, mu=0.5):
    """4 bottom-vertex contacts per cube against the plane or the cube below."""
    pos = np.asarray(pos, np.float64); quat = np.asarray(quat, np.float64)
    n = len(pos)
    R = quat_rot(quat)
    corners = box_bottom_corners((edge, edge, edge))
    cb, pa, pb, nn = [], [], [], []
    for i in range(n):
        for p in corners:
            w = pos[i] + R[i] @ p
            if i == 0:
                cb.append((i, -1)); pa.append(p); pb.append((w[0], w[1], 0.0)); nn.append((0, 0, 1))
            else:
                loc = R[i - 1].T @ (w - pos[i - 1])
                loc[2] = edge / 2
                cb.append((i, i - 1)); pa.append(p); pb.append(loc); nn.append(R[i - 1][:, 2])
    k = len(cb)
    return dict(c_body=np.array(cb, np.int32), c_pa=np.array(pa), c_pb=np.array(pb), c_n=np.array(nn),
                c_d=np.zeros(k), c_mu=np.full(k, mu))


def cube_stack(seed=0, n=4, edge=1.0, density=1000.0, mu=0.5, jitter=1e-3, yaw_deg=5.0):
    """Config: n unit cubes stacked on z = 0 with +-jitter offsets and +-yaw."""
    rng = np.random.default_rng(seed)
    m = density * edge ** 3
    I = box_inertia(m, (edge, edge, edge))
    pos = np.zeros((n, 3)); quat = np.zeros((n, 4))
    for i in range(n):
        pos[i] = (rng.uniform(-jitter, jitter), rng.uniform(-jitter, jitter),
                  edge / 2 + i * edge + rng.uniform(-jitter, jitter))
        quat[i] = quat_yaw(np.deg2rad(rng.uniform(-yaw_deg, yaw_deg)))
    s = dict(kind=np.zeros(n, np.int32), pos=pos, quat=quat, vel=np.zeros((n, 3)), omega=np.zeros((n, 3)),
             mass=np.full(n, m), inertia=np.tile(I, (n, 1)), env=np.zeros(n, np.int32),
             half=np.full((n, 3), edge / 2))
    s.update(stack_contacts(pos, quat, edge, mu))
    s.update(_empty_joints()); s.update(_empty_tets())
    return finalize(s)


def heavy_stack(seed=0, masses=(8.0, 64.0, 512.0, 4096.0, 32768.0), edge=1.0, mu=0.5, jitter=1e-3, yaw_deg=5.0):
    """The heavy stack of Sec. 10 (Rigid Body Contact): unit cubes whose masses
    grow geometrically from the bottom, 8 ... 32768 kg (4096:1), mu = 0.5,
    each pressing on the lighter one below; seed-jittered offsets and yaw."""
    rng = np.random.default_rng(seed)
    n = len(masses)
    pos = np.zeros((n, 3)); quat = np.zeros((n, 4))
    for i in range(n):
        pos[i] = (rng.uniform(-jitter, jitter), rng.uniform(-jitter, jitter),
                  edge / 2 + i * edge + rng.uniform(-jitter, jitter))
        quat[i] = quat_yaw(np.deg2rad(rng.uniform(-yaw_deg, yaw_deg)))
    m = np.asarray(masses, np.float64)
    s = dict(kind=np.zeros(n, np.int32), pos=pos, quat=quat, vel=np.zeros((n, 3)), omega=np.zeros((n, 3)),
             mass=m, inertia=np.stack([box_inertia(mi, (edge, edge, edge)) for mi in m]),
             env=np.zeros(n, np.int32), half=np.full((n, 3), edge / 2))
    s.update(stack_contacts(pos, quat, edge, mu))
    s.update(_empty_joints()); s.update(_empty_tets())
    return finalize(s)


def _empty_joints():
    return dict(j_body=np.zeros((0, 2), np.int32), j_pa=np.zeros((0, 3)), j_pb=np.zeros((0, 3)),
                j_axa=np.zeros((0, 3)), j_axb=np.zeros((0, 3)), j_compliance=np.zeros(0))


def _empty_tets():
    return dict(t_v=np.zeros((0, 4), np.int32), t_rest=np.zeros((0, 4, 3)), t_E=np.zeros(0), t_nu=np.zeros(0))


def _empty_contacts():
    return dict(c_body=np.zeros((0, 2), np.int32), c_pa=np.zeros((0, 3)), c_pb=np.zeros((0, 3)),
                c_n=np.zeros((0, 3)), c_d=np.zeros(0), c_mu=np.zeros(0))


# --------------------------------------------------------------------------------------
# Workload 2: revolute chain on a Neo-Hookean block (Fetch Tomato / Allegro Ball shape)

def hex_tets(n):
    """5-tet split of an n^3 hex grid with alternating parity (conforming)."""
    def vid(i, j, k):
        return (k * (n + 1) + j) * (n + 1) + i
    tets = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                c = [vid(i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1)) for b in range(8)]
                if (i + j + k) % 2 == 0:
                    tets += [(c[1], c[2], c[4], c[7]), (c[0], c[1], c[2], c[4]), (c[3], c[1], c[2], c[7]),
                             (c[5], c[1], c[4], c[7]), (c[6], c[2], c[4], c[7])]
                else:
                    tets += [(c[0], c[3], c[5], c[6]), (c[1], c[0], c[3], c[5]), (c[2], c[0], c[3], c[6]),
                             (c[4], c[0], c[5], c[6]), (c[7], c[3], c[5], c[6])]
    return np.array(tets, np.int32)


def chain_block(seed=0, hexes=24, edge=0.5, E=1e5, nu=0.45, density=1000.0, links=7,
                link_dims=(0.3, 0.1, 0.1), link_density=1000.0, mu=0.8, rest_jitter=0.03,
                margin=0.005):
    """Config: revolute chain resting on / pressing into a stable Neo-Hookean block.

    Block: hexes^3 hexes x 5 tets, edge ``edge`` m, resting on z = 0.  The rest
    shape is the grid jittered by +-rest_jitter of the spacing (seeded), so the
    initial state is mildly pre-strained and singular values are distinct.
    Chain: ``links`` boxes along +x, pinned to a world anchor, lying on the top
    face; contacts: bottom block vertices vs ground, top vertices under a link.
    ``planes`` (the ground) and ``mu_env`` let a collider regenerate the same
    kinds of contact (block vertices against the ground and the links).
    """
    rng = np.random.default_rng(seed)
    n = hexes
    sp = edge / n
    g = np.arange(n + 1) * sp - edge / 2
    # vertex order matches hex_tets' vid: ((k*(n+1)+j)*(n+1)+i)
    kk, jj, ii = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    verts = np.stack([g[ii.ravel()], g[jj.ravel()], (kk.ravel() * sp)], 1)
    rest = verts + rng.uniform(-rest_jitter, rest_jitter, verts.shape) * sp
    tets = hex_tets(n)
    nv = len(verts)
    vol = np.abs(np.einsum("ij,ij->i", np.cross(rest[tets[:, 1]] - rest[tets[:, 0]],
                                                  rest[tets[:, 2]] - rest[tets[:, 0]]),
                           rest[tets[:, 3]] - rest[tets[:, 0]])) / 6.0
    vmass = np.zeros(nv)
    np.add.at(vmass, tets.ravel(), np.repeat(vol * density / 4.0, 4))

    L = np.asarray(link_dims, np.float64)
    lm = link_density * L.prod()
    lI = box_inertia(lm, L)
    top = edge
    x0 = -0.95 * (link_dims[0] / 0.3)
    zc = top + L[2] / 2
    nb_links = links
    kind = np.concatenate([np.zeros(nb_links, np.int32), np.ones(nv, np.int32)])
    lpos = np.stack([x0 + L[0] * (np.arange(links) + 0.5), np.zeros(links), np.full(links, zc)], 1)
    pos = np.concatenate([lpos, verts])
    quat = np.zeros((nb_links + nv, 4)); quat[:, 0] = 1
    mass = np.concatenate([np.full(links, lm), vmass])
    inertia = np.concatenate([np.tile(lI, (links, 1)), np.ones((nv, 3))])
    # joints: world -> link0, link k-1 -> link k, hinge axis y
    jb, jpa, jpb = [], [], []
    for k in range(links):
        if k == 0:
            jb.append((0, -1)); jpa.append((-L[0] / 2, 0, 0)); jpb.append((x0, 0, zc))
        else:
            jb.append((k, k - 1)); jpa.append((-L[0] / 2, 0, 0)); jpb.append((L[0] / 2, 0, 0))
    joints = dict(j_body=np.array(jb, np.int32), j_pa=np.array(jpa), j_pb=np.array(jpb),
                  j_axa=np.tile((0.0, 1.0, 0.0), (links, 1)), j_axb=np.tile((0.0, 1.0, 0.0), (links, 1)),
                  j_compliance=np.zeros(links))
    # contacts
    cb, pa, pb, nn = [], [], [], []
    bottom = np.nonzero(np.abs(verts[:, 2]) < 1e-9)[0]
    for v in bottom:
        cb.append((links + v, -1)); pa.append((0, 0, 0)); pb.append((verts[v, 0], verts[v, 1], 0.0)); nn.append((0, 0, 1))
    topv = np.nonzero(np.abs(verts[:, 2] - top) < 1e-9)[0]
    for k in range(links):
        c = lpos[k]
        for v in topv:
            d = verts[v] - c
            if abs(d[0]) <= L[0] / 2 + margin and abs(d[1]) <= L[1] / 2 + margin:
                cb.append((links + v, k)); pa.append((0, 0, 0)); pb.append((d[0], d[1], -L[2] / 2)); nn.append((0, 0, -1))
    kc = len(cb)
    contacts = dict(c_body=np.array(cb, np.int32), c_pa=np.array(pa), c_pb=np.array(pb), c_n=np.array(nn),
                    c_d=np.zeros(kc), c_mu=np.full(kc, mu))
    t_rest = rest[tets]
    s = dict(kind=kind, pos=pos, quat=quat, vel=np.zeros((len(kind), 3)), omega=np.zeros((len(kind), 3)),
             mass=mass, inertia=inertia, env=np.zeros(len(kind), np.int32),
             half=np.concatenate([np.tile(L / 2, (links, 1)), np.zeros((nv, 3))]), t_v=(tets + links).astype(np.int32),
             t_rest=t_rest, t_E=np.full(len(tets), E), t_nu=np.full(len(tets), nu),
             planes=np.array([[0.0, 0.0, 1.0, 0.0]]), mu_env=np.array([mu]))
    s.update(joints); s.update(contacts)
    return finalize(s)


# --------------------------------------------------------------------------------------
# Workload 3: many uneven RL-style environments (Humanoid / Yumi shape, Table 2)

def batched_envs(seed=0, n_envs=4096, links=(3, 20), boxes=(0, 64), box_edge=(0.05, 0.2),
                 mu=(0.3, 1.0), link_dims=(0.2, 0.05, 0.05), density=1000.0, spacing=8.0):
    """Config: independent environments, each a revolute chain (link count uniform
    in ``links``) lying on the ground plus a pile of cubes (count uniform in
    ``boxes``, edge log-uniform in ``box_edge``) stacked in up to four layers,
    with per-environment friction uniform in ``mu``.  Links get random spin about
    z and boxes random horizontal velocities so contacts mix stick and slip.
    Vertices of every body bottom face contact the ground or the box beneath:
    a box above another is at most 0.7 of its edge, turned by at most 0.15 rad
    and offset by at most 15% of its half edge from it, so its bottom face lies
    on the lower box's top face.
    """
    rng = np.random.default_rng(seed)
    L = np.asarray(link_dims, np.float64)
    lm = density * L.prod()
    lI = box_inertia(lm, L)
    nl = rng.integers(links[0], links[1] + 1, n_envs)
    nbx = rng.integers(boxes[0], boxes[1] + 1, n_envs)
    mue = rng.uniform(mu[0], mu[1], n_envs)
    side = int(np.ceil(np.sqrt(n_envs)))
    origin = np.stack([(np.arange(n_envs) % side) * spacing, (np.arange(n_envs) // side) * spacing, np.zeros(n_envs)], 1)
    # bodies: per env links then boxes
    nb_env = nl + nbx
    first = np.concatenate([[0], np.cumsum(nb_env)[:-1]])
    NB = int(nb_env.sum())
    kind = np.zeros(NB, np.int32)
    env = np.repeat(np.arange(n_envs, dtype=np.int32), nb_env)
    pos = np.zeros((NB, 3)); quat = np.zeros((NB, 4)); quat[:, 0] = 1
    vel = np.zeros((NB, 3)); omega = np.zeros((NB, 3)); mass = np.zeros(NB); inertia = np.zeros((NB, 3))
    # links: lie along +x from the env origin, slightly jittered in z
    li = np.concatenate([first[e] + np.arange(nl[e]) for e in range(n_envs)])
    lk = np.concatenate([np.arange(nl[e]) for e in range(n_envs)])
    le = np.repeat(np.arange(n_envs), nl)
    pos[li] = origin[le] + np.stack([L[0] * (lk + 0.5), np.zeros_like(lk, dtype=float),
                                     L[2] / 2 + rng.uniform(-5e-4, 5e-4, len(li))], 1)
    mass[li] = lm; inertia[li] = lI
    spin = rng.uniform(-0.5, 0.5, n_envs)
    omega[li, 2] = spin[le]
    # boxes: 16 cells of 0.25 m in a 1 m square next to the chain, layer = k // 16
    bi = np.concatenate([first[e] + nl[e] + np.arange(nbx[e]) for e in range(n_envs)]).astype(np.int64)
    bk = np.concatenate([np.arange(nbx[e]) for e in range(n_envs)]).astype(np.int64)
    be = np.repeat(np.arange(n_envs), nbx)
    edge = np.exp(rng.uniform(np.log(box_edge[0]), np.log(box_edge[1]), len(bi)))
    cell = bk % 16
    layer = bk // 16
    cx = (cell % 4) * 0.25 + 0.125 + rng.uniform(-0.02, 0.02, len(bi))
    cy = (cell // 4) * 0.25 + 0.5 + rng.uniform(-0.02, 0.02, len(bi))
    yaw = rng.uniform(-0.3, 0.3, len(bi))
    # height: stack on the box of the same cell one layer below
    below = np.full(len(bi), -1, np.int64)
    zc = np.zeros(len(bi))
    # boxes of one env are consecutive and ordered by k, so the support of box k is box k-16
    has_below = layer > 0
    below[has_below] = np.nonzero(has_below)[0] - 16
    # a box above another rests with its whole bottom face on the top face of
    # the one below: edge at most 0.7 of the lower edge, yaw within 0.15 rad
    # of it, centre within 15% of its half edge (0.7 (cos 0.15 + sin 0.15)
    # + 0.15 < 1, so every bottom corner lies over the lower top face)
    rel_yaw = rng.uniform(-0.15, 0.15, len(bi))
    rel_off = rng.uniform(-0.15, 0.15, (len(bi), 2))
    for lay in range(int(layer.max()) + 1 if len(layer) else 0):
        sel = layer == lay
        if lay == 0:
            zc[sel] = edge[sel] / 2
        else:
            idx = np.nonzero(sel)[0]
            lo = below[idx]
            edge[idx] = np.minimum(edge[idx], 0.7 * edge[lo])
            yaw[idx] = yaw[lo] + rel_yaw[idx]
            cx[idx] = cx[lo] + rel_off[idx, 0] * edge[lo] / 2
            cy[idx] = cy[lo] + rel_off[idx, 1] * edge[lo] / 2
            zc[idx] = zc[lo] + edge[lo] / 2 + edge[idx] / 2
    zc += rng.uniform(-5e-4, 5e-4, len(bi))
    pos[bi] = origin[be] + np.stack([cx, cy, zc], 1)
    quat[bi] = quat_yaw(yaw)
    vel[bi, :2] = rng.uniform(-0.05, 0.05, (len(bi), 2))
    mass[bi] = density * edge ** 3
    inertia[bi] = (density * edge ** 5 / 6.0)[:, None]
    # joints: anchor world -> link 0, then link k-1 -> link k, hinge axis z
    jb = []; jpa = []; jpb = []
    for e in range(n_envs):
        f = first[e]
        jb.append((f, -1)); jpa.append((-L[0] / 2, 0, 0)); jpb.append(origin[e] + (0, 0, L[2] / 2))
        for k in range(1, nl[e]):
            jb.append((f + k, f + k - 1)); jpa.append((-L[0] / 2, 0, 0)); jpb.append((L[0] / 2, 0, 0))
    nj = len(jb)
    joints = dict(j_body=np.array(jb, np.int32), j_pa=np.array(jpa, np.float64), j_pb=np.array(jpb, np.float64),
                  j_axa=np.tile((0.0, 0.0, 1.0), (nj, 1)), j_axb=np.tile((0.0, 0.0, 1.0), (nj, 1)),
                  j_compliance=np.zeros(nj))
    # contacts: 4 bottom corners of each link vs ground, each box vs ground / box below
    R = quat_rot(quat)
    cb_l = []
    lc = box_bottom_corners(L)
    n_l = len(li)
    w_l = pos[li][:, None, :] + np.einsum("nij,cj->nci", R[li], lc)
    c_body_l = np.stack([np.repeat(li, 4), np.full(4 * n_l, -1)], 1)
    c_pa_l = np.tile(lc, (n_l, 1))
    c_pb_l = w_l.reshape(-1, 3).copy(); c_pb_l[:, 2] = 0.0
    c_n_l = np.tile((0.0, 0.0, 1.0), (4 * n_l, 1))
    c_mu_l = np.repeat(mue[le], 4)
    # boxes
    unit = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1]], np.float64) * 0.5
    bc = unit[None, :, :] * edge[:, None, None]                          # (nbx, 4, 3) local corners
    w_b = pos[bi][:, None, :] + np.einsum("nij,ncj->nci", R[bi], bc)
    sup = np.where(below >= 0, bi[np.maximum(below, 0)], -1)
    c_body_b = np.stack([np.repeat(bi, 4), np.repeat(sup, 4)], 1)
    c_pa_b = bc.reshape(-1, 3)
    c_pb_b = w_b.reshape(-1, 3).copy()
    ground = np.repeat(sup < 0, 4)
    c_pb_b[ground, 2] = 0.0
    c_n_b = np.tile((0.0, 0.0, 1.0), (4 * len(bi), 1))
    if (~ground).any():
        idx = np.nonzero(~ground)[0]
        sb = c_body_b[idx, 1]
        loc = np.einsum("nji,nj->ni", R[sb], c_pb_b[idx] - pos[sb])   # R^T (w - x)
        loc[:, 2] = (edge[np.maximum(np.repeat(below, 4)[idx], 0)] / 2)
        c_pb_b[idx] = loc
        c_n_b[idx] = R[sb][:, :, 2]
    c_mu_b = np.repeat(mue[be], 4)
    contacts = dict(c_body=np.concatenate([c_body_l, c_body_b]).astype(np.int32),
                    c_pa=np.concatenate([c_pa_l, c_pa_b]), c_pb=np.concatenate([c_pb_l, c_pb_b]),
                    c_n=np.concatenate([c_n_l, c_n_b]), c_d=np.zeros(4 * (n_l + len(bi))),
                    c_mu=np.concatenate([c_mu_l, c_mu_b]))
    half = np.zeros((NB, 3))
    half[li] = L / 2
    half[bi] = edge[:, None] / 2
    s = dict(kind=kind, pos=pos, quat=quat, vel=vel, omega=omega, mass=mass, inertia=inertia, env=env, half=half,
             mu_env=mue)
    s.update(joints); s.update(contacts); s.update(_empty_tets())
    return finalize(s)


# --------------------------------------------------------------------------------------
# Workload 5: large mixed scene, rigid boxes and Neo-Hookean spheres in a bin

def sphere_mesh(radius, res, rng, rest_jitter=0.01):
    """Tet mesh of a ball: the hexes of a res^3 grid over [-radius, radius]^3
    whose centres lie inside the ball, 5 tets each (hex_tets); vertices
    renumbered, rest shape jittered by +-rest_jitter of the spacing."""
    n = res
    sp = 2.0 * radius / n
    g = np.arange(n + 1) * sp - radius
    kk, jj, ii = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    verts = np.stack([g[ii.ravel()], g[jj.ravel()], g[kk.ravel()]], 1)
    c = (np.arange(n) + 0.5) * sp - radius
    ck, cj, ci = np.meshgrid(c, c, c, indexing="ij")
    inside = (ci ** 2 + cj ** 2 + ck ** 2 <= radius ** 2).ravel()       # hex order matches hex_tets (i fastest)
    tets = hex_tets(n).reshape(-1, 5, 4)[inside].reshape(-1, 4)
    used = np.unique(tets)
    remap = -np.ones(len(verts), np.int64)
    remap[used] = np.arange(len(used))
    verts = verts[used]
    tets = remap[tets].astype(np.int32)
    rest = verts + rng.uniform(-rest_jitter, rest_jitter, verts.shape) * sp
    return verts, rest, tets


def mixed_bin(seed=0, n_boxes=2000, n_spheres=8, sphere_radius=0.3, sphere_res=12, box_edge=(0.05, 0.3),
              E=5e4, nu=0.4, density=1000.0, mu=0.5, margin=0.01, cell=0.42):
    """Config: one environment, a bin (floor z = 0, walls x = 0 and y = 0 used)
    holding ``n_boxes`` rigid boxes (edge uniform in ``box_edge``) stacked in
    columns of up to four on a grid of ``cell`` m cells, and ``n_spheres``
    stable Neo-Hookean balls (``sphere_res``^3-hex voxel meshes, ~4,500 tets
    each at res 12) resting on the floor against the x = 0 wall.  A column has
    one random yaw (within +-0.3 rad) and centre (within +-0.01 m of its cell's
    centre), and its edges decrease upwards, so each box rests wholly on the
    one beneath; the cell (0.42 m) exceeds the widest yawed box plus the
    jitter and the margin, so neighbouring columns do not touch.  Contacts: 4
    bottom corners per box vs the floor or the box below; ball vertices within
    ``margin`` of the floor or the wall vs that plane.  ``planes`` (floor and
    the two walls) and ``mu_env`` let a collider regenerate the contacts."""
    rng = np.random.default_rng(seed)
    n_cols = int(np.ceil(n_boxes / 4))
    side = int(np.ceil(np.sqrt(n_cols)))
    x_off = 2 * sphere_radius + 0.1                   # the balls' strip along the x = 0 wall
    B = SceneBuilder()
    edges = rng.uniform(box_edge[0], box_edge[1], n_boxes)
    for col in range(n_cols):                          # box k sits in column k % n_cols, level k // n_cols
        members = np.arange(col, n_boxes, n_cols)
        edges[members] = np.sort(edges[members])[::-1]
    col_xy = rng.uniform(-0.01, 0.01, (n_cols, 2))
    col_yaw = rng.uniform(-0.3, 0.3, n_cols)
    col_top = {}
    for k in range(n_boxes):
        col = k % n_cols
        cx = x_off + (col % side + 0.5) * cell + col_xy[col, 0]
        cy = (col // side + 0.5) * cell + col_xy[col, 1]
        e = edges[k]
        below = col_top.get(col)
        z0 = 0.0 if below is None else below[1]
        yaw = col_yaw[col]
        m = density * e ** 3
        q = quat_yaw(yaw)
        bid = B.add_rigid((cx, cy, z0 + e / 2), tuple(q), mass=m, inertia=(m * e * e / 6,) * 3)
        R = quat_rot(np.asarray(q)[None])[0]
        for u in np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1]], np.float64) * 0.5 * e:
            w = np.array([cx, cy, z0 + e / 2]) + R @ u
            if below is None:
                B.add_contact(bid, -1, u, (w[0], w[1], 0.0), (0, 0, 1), 0.0, mu)
            else:
                sb, _, sR, sx, se = below
                loc = sR.T @ (w - sx)
                loc[2] = se / 2
                B.add_contact(bid, sb, u, loc, sR[:, 2], 0.0, mu)
        col_top[col] = (bid, z0 + e, R, np.array([cx, cy, z0 + e / 2]), e)
    verts, rest, tets = sphere_mesh(sphere_radius, sphere_res, rng)
    vol = np.abs(np.einsum("ij,ij->i", np.cross(rest[tets[:, 1]] - rest[tets[:, 0]], rest[tets[:, 2]] - rest[tets[:, 0]]),
                           rest[tets[:, 3]] - rest[tets[:, 0]])) / 6.0
    vmass = np.zeros(len(verts))
    np.add.at(vmass, tets.ravel(), np.repeat(vol * density / 4.0, 4))
    zmin, xmin = verts[:, 2].min(), verts[:, 0].min()
    for s_ in range(n_spheres):
        c = np.array([-xmin, (s_ + 0.5) * (2 * sphere_radius + 0.05), -zmin])
        first = None
        for v in range(len(verts)):
            bid = B.add_particle(tuple(verts[v] + c), mass=vmass[v])
            first = bid if first is None else first
            p = verts[v] + c
            if p[2] <= margin:
                B.add_contact(bid, -1, (0, 0, 0), (p[0], p[1], 0.0), (0, 0, 1), 0.0, mu)
            if p[0] <= margin:
                B.add_contact(bid, -1, (0, 0, 0), (0.0, p[1], p[2]), (1, 0, 0), 0.0, mu)
        for t in range(len(tets)):
            B.add_tet(tuple(tets[t] + first), rest[tets[t]], E, nu)
    s = B.build()
    half = np.zeros((len(s["mass"]), 3), F32)        # the boxes are bodies 0 .. n_boxes-1
    half[:n_boxes] = (edges[:, None] / 2).astype(F32)
    s["half"] = half
    s["planes"] = np.array([[0, 0, 1, 0], [1, 0, 0, 0], [0, 1, 0, 0]], F32)
    s["mu_env"] = np.array([mu], F32)
    return s


# --------------------------------------------------------------------------------------
# Prismatic and revolute joints with a linear Hookean block (the joint and
# material types of the paper's Fetch and PneuNet scenes, Sec. 9.2.1, Sec. 10)

def slider_arm_block(seed=0, hexes=2, edge=0.3, E=5e4, nu=0.3, density=1000.0, mu=0.6):
    """An arm on a horizontal prismatic joint to the world (a 0.2 m cube
    carriage, 2 kg) carrying two revolute links (0.3 x 0.05 x 0.05 m, 0.5 kg)
    that start horizontal and swing under gravity, beside a block of
    hexes^3 x 5 linear Hookean tets resting on the ground (bottom vertices in
    contact with the plane, rest shape jittered by 1%)."""
    rng = np.random.default_rng(seed)
    b = SceneBuilder()
    u = (1.0, 0.0, 0.0)
    car = b.add_rigid((0.0, 2.0, 1.0), (1, 0, 0, 0), vel=(rng.uniform(-0.2, 0.2), 0, 0), mass=2.0,
                      inertia=tuple(box_inertia(2.0, (0.2, 0.2, 0.2))))
    b.add_prismatic(car, -1, (0, 0, 0), (0.0, 2.0, 1.0), u, u, 0.0)
    L = np.array([0.3, 0.05, 0.05])
    I = tuple(box_inertia(0.5, L))
    l1 = b.add_rigid((0.15, 2.0, 1.0), (1, 0, 0, 0), mass=0.5, inertia=I)
    b.add_revolute(l1, car, (-0.15, 0, 0), (0.0, 0.0, 0.0), (0, 1, 0), (0, 1, 0), 0.0)
    l2 = b.add_rigid((0.45, 2.0, 1.0), (1, 0, 0, 0), mass=0.5, inertia=I)
    b.add_revolute(l2, l1, (-0.15, 0, 0), (0.15, 0, 0), (0, 1, 0), (0, 1, 0), 0.0)
    n = hexes
    h = edge / n
    grid = np.array([(i, j, k) for k in range(n + 1) for j in range(n + 1) for i in range(n + 1)], np.float64) * h
    X = grid + rng.uniform(-0.01, 0.01, grid.shape) * h
    X[:, 2] = np.where(grid[:, 2] == 0.0, 0.0, X[:, 2])          # bottom layer on the plane
    tets = hex_tets(n)
    vol = np.zeros(len(X))
    for t in tets:
        P = X[list(t)]
        v = abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], 1))) / 6
        vol[list(t)] += v / 4
    ids = [b.add_particle(tuple(x), mass=density * vol[i]) for i, x in enumerate(X)]
    for t in tets:
        b.add_linear_tet(tuple(ids[q] for q in t), tuple(map(tuple, X[list(t)])), E, nu)
    for i, x in enumerate(X):
        if x[2] == 0.0:
            b.add_contact(ids[i], -1, (0, 0, 0), (x[0], x[1], 0.0), (0, 0, 1), 0.0, mu)
    return b.build()
