"""Pins of the oracle's prismatic joints and linear Hookean tets.

Prismatic joints (the paper's Fetch scenes use prismatic and revolute joints,
without giving their constraint functions): a body on a frictionless slider
accelerates along the slide axis with the component of gravity along it, with
no rotation; the rows are the velocities of the constraint functions, checked
by finite differences of functions written here.

Linear Hookean tets (Sec. 9.2.1: constant-strain elements, energy
V_e s^T K_e s / 2 of the small strain, compliance E = (V_e K_e)^-1): the
compliance form of a quadratic energy with a linear constraint map is backward
Euler on linear elasticity, so one converged step equals the solution of
(M + h^2 K) v = M v~ - h grad U(x^-) assembled here from this file's own
strain and stiffness; an undeformed block falls freely.
"""
import numpy as np
import pytest

from paper_1907_04587_gb300 import scenes

H = 1.0 / 60.0
G = 9.81
GRAV = np.array([0.0, 0.0, -G])


def _slider(theta, mass=2.0):
    u = np.array([np.cos(theta), 0.0, -np.sin(theta)])
    b = scenes.SceneBuilder()
    i = b.add_rigid((0.0, 0.0, 1.0), (1, 0, 0, 0), mass=mass, inertia=(0.1, 0.2, 0.3))
    b.add_prismatic(i, -1, (0, 0, 0), (0.0, 0.0, 1.0), tuple(u), tuple(u), 0.0)
    return b.build(), u


@pytest.mark.parametrize("theta_deg", [0.0, 30.0, 60.0, 90.0])
def test_slider_accelerates_with_gravity_along_its_axis(orc, theta_deg):
    """Hard prismatic joint to the world along u at angle theta below the
    horizontal: every step adds h (g . u) u to the velocity (implicit Euler is
    exact for a constant force), the body does not turn and stays on the line."""
    s, u = _slider(np.radians(theta_deg))
    # the slide direction: orthogonal to the two positional rows t_1, t_2 built
    # from the axis as the oracle receives it (FP32, unit only to rounding)
    uf = s["j_axb"][0].astype(np.float64)
    uf /= np.linalg.norm(uf)                       # axes are directions (normalised by the rows)
    # eps = 0: the shift of Sec. 8.4 would make the hard joint compliant by ~1e-7
    o = orc.Oracle(s, newton_iters=30, cr_iters=60, line_search=1, eps=0.0)
    gu = GRAV @ uf
    x0 = s["pos"][0].astype(np.float64)
    for k in range(1, 11):
        o.step()
        st = o.get_state()
        np.testing.assert_allclose(st["vel"][0], k * H * gu * uf, rtol=0, atol=1e-9 * max(1.0, k * H * G))
        assert np.abs(st["omega"][0]).max() < 1e-10
        d = st["pos"][0] - x0
        assert np.linalg.norm(d - (d @ uf) * uf) < 1e-9
        np.testing.assert_allclose(st["quat"][0], [1, 0, 0, 0], atol=1e-12)


def _basis(n):
    """Duff et al. 2017 orthonormal basis of a unit vector (the published
    construction the row definitions name)."""
    sgn = 1.0 if n[2] >= 0.0 else -1.0
    a = -1.0 / (sgn + n[2])
    b = n[0] * n[1] * a
    return (np.array([1.0 + sgn * n[0] * n[0] * a, sgn * b, -sgn * n[0]]),
            np.array([b, sgn + n[1] * n[1] * a, -n[1]]))


def _prismatic_c(s, pos, quat, j):
    """The five constraint functions of a prismatic joint, written from their
    definition: t_k . (p_a - p_b), a_w . t_k, n_a . t_2 (axes normalised)."""
    a, b = s["j_body"][j]
    R = lambda i: scenes.quat_rot(quat[i][None])[0]
    pa = pos[a] + R(a) @ s["j_pa"][j].astype(np.float64) if a >= 0 else s["j_pa"][j].astype(np.float64)
    pb = pos[b] + R(b) @ s["j_pb"][j].astype(np.float64) if b >= 0 else s["j_pb"][j].astype(np.float64)
    ub = s["j_axb"][j].astype(np.float64)
    t1, t2 = _basis(ub / np.linalg.norm(ub))
    if b >= 0:
        t1, t2 = R(b) @ t1, R(b) @ t2
    aw = s["j_axa"][j].astype(np.float64)
    aw = aw / np.linalg.norm(aw)
    na, _ = _basis(aw)
    if a >= 0:
        aw, na = R(a) @ aw, R(a) @ na
    d = pa - pb
    return np.array([t1 @ d, t2 @ d, aw @ t1, aw @ t2, na @ t2])


def _kinematic_q(s, u, h=H):
    pos = s["pos"].astype(np.float64).copy()
    quat = s["quat"].astype(np.float64).copy()
    o = 0
    for i in range(len(pos)):
        if s["kind"][i] == 0:
            v, w = u[o:o + 3], u[o + 3:o + 6]
            pos[i] += h * v
            t = quat[i].copy()
            Q = np.array([[-t[1], -t[2], -t[3]], [t[0], t[3], -t[2]], [-t[3], t[0], t[1]], [t[2], -t[1], t[0]]])
            qq = t + h * 0.5 * Q @ w
            quat[i] = qq / np.linalg.norm(qq)
            o += 6
        else:
            pos[i] += h * u[o:o + 3]
            o += 3
    return pos, quat


def test_prismatic_rows_are_constraint_velocities(orc):
    """Two rigid bodies joined by a prismatic joint in a general pose (b turned,
    a slid along the axis and slightly misaligned): the oracle's rows equal
    h^-1 d c(q(u)) / du of the functions above, by central differences."""
    u_ax = np.array([0.3, -0.5, 0.8]); u_ax /= np.linalg.norm(u_ax)
    b = scenes.SceneBuilder()
    qb = scenes.quat_axis_angle((0.2, 1.0, -0.4), 0.7)
    ib = b.add_rigid((0.1, 0.2, 0.9), qb, mass=1.5, inertia=(0.2, 0.3, 0.25))
    Rb = scenes.quat_rot(qb[None])[0]
    qa = scenes.quat_axis_angle((1.0, 0.3, 0.1), 0.05)
    qa = scenes.quat_rot(qa[None])[0]
    xa = np.array([0.1, 0.2, 0.9]) + Rb @ (0.25 * u_ax) + np.array([2e-3, -1e-3, 1e-3])
    from scipy.spatial.transform import Rotation
    qa_full = Rotation.from_matrix(qa @ Rb).as_quat()        # x y z w
    ia = b.add_rigid(tuple(xa), (qa_full[3], qa_full[0], qa_full[1], qa_full[2]), mass=0.8, inertia=(0.05, 0.07, 0.06))
    b.add_prismatic(ia, ib, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), tuple(u_ax), tuple(u_ax), 0.0)
    s = b.build()
    o = orc.Oracle(s)
    c0, J = o.eval_constraints()
    np.testing.assert_allclose(c0, _prismatic_c(s, s["pos"].astype(np.float64), s["quat"].astype(np.float64), 0),
                               rtol=0, atol=1e-6)
    rng = np.random.default_rng(2)
    for _ in range(5):
        du = rng.normal(size=J.shape[1])
        d = 1e-6
        pp, qp = _kinematic_q(s, d * du)
        pm, qm = _kinematic_q(s, -d * du)
        fd = (_prismatic_c(s, pp, qp, 0) - _prismatic_c(s, pm, qm, 0)) / (2 * d * H)
        np.testing.assert_allclose(J @ du, fd, rtol=1e-5, atol=1e-7)


# ---------------------------------------------------------------------------------
# linear Hookean tets (Sec. 9.2.1)

def _strain(x4, rest):
    """Engineering small strain [e_xx, e_yy, e_zz, 2 e_yz, 2 e_xz, 2 e_xy] of
    F = D_s D_m^-1 (e = (F + F^T)/2 - I)."""
    Dm = np.stack([rest[q] - rest[0] for q in (1, 2, 3)], 1)
    Ds = np.stack([x4[q] - x4[0] for q in (1, 2, 3)], 1)
    F = Ds @ np.linalg.inv(Dm)
    e = 0.5 * (F + F.T) - np.eye(3)
    return np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[0, 2], 2 * e[0, 1]])


def _stiffness(E, nu):
    mu = E / (2 * (1 + nu))
    la = E * nu / ((1 + nu) * (1 - 2 * nu))
    K = np.zeros((6, 6))
    K[:3, :3] = la
    K[[0, 1, 2], [0, 1, 2]] += 2 * mu
    K[[3, 4, 5], [3, 4, 5]] = mu
    return K


def _linear_block(seed=0, E=2e4, nu=0.3, stretch=0.04, spin=0.0, lift=1.0):
    """One hex of 5 linear tets, its particles moving with a deforming
    velocity field (and a rigid spin about z), lifted by `lift` above the
    rest positions."""
    rng = np.random.default_rng(seed)
    b = scenes.SceneBuilder()
    n = 1
    edge = 0.2
    grid = [(i, j, k) for k in range(n + 1) for j in range(n + 1) for i in range(n + 1)]
    X = np.array(grid, np.float64) * edge
    for x in X:
        v = np.array([stretch * (x[0] - 0.1), -0.5 * stretch * (x[1] - 0.1), 0.0]) + rng.normal(scale=0.02, size=3)
        v += spin * np.array([-(x[1] - 0.1), x[0] - 0.1, 0.0])
        b.add_particle(tuple(x + np.array([0, 0, lift])), vel=tuple(v), mass=0.5)
    for t in scenes.hex_tets(n):
        b.add_linear_tet(tuple(int(i) for i in t), tuple(map(tuple, X[list(t)])), E, nu)
    return b.build()


def _backward_euler(s, h=H):
    """(M + h^2 K) v = M (u^- + h g) - h grad U(x^-), K and grad U assembled
    from the strain of _strain (linear in x: its derivative by central
    differences is exact to rounding) and _stiffness."""
    nb = len(s["mass"])
    x0 = s["pos"].astype(np.float64)
    Kg = np.zeros((3 * nb, 3 * nb))
    gU = np.zeros(3 * nb)
    for v, rest, E, nu in zip(s["l_v"], s["l_rest"].astype(np.float64), s["l_E"], s["l_nu"]):
        Ve = abs(np.linalg.det(np.stack([rest[q] - rest[0] for q in (1, 2, 3)], 1))) / 6
        K = Ve * _stiffness(float(E), float(nu))
        x4 = x0[list(v)]
        B = np.zeros((6, 12))
        d = 1e-4
        for j in range(12):
            xp = x4.reshape(-1).copy(); xm = xp.copy()
            xp[j] += d; xm[j] -= d
            B[:, j] = (_strain(xp.reshape(4, 3), rest) - _strain(xm.reshape(4, 3), rest)) / (2 * d)
        idx = np.concatenate([[3 * q, 3 * q + 1, 3 * q + 2] for q in v])
        Kg[np.ix_(idx, idx)] += B.T @ K @ B
        gU[idx] += B.T @ K @ _strain(x4, rest)
    M = np.repeat(s["mass"].astype(np.float64), 3)
    vt = s["vel"].astype(np.float64).reshape(-1) + h * np.tile(GRAV, nb)
    return np.linalg.solve(np.diag(M) + h * h * Kg, M * vt - h * gU).reshape(nb, 3)


@pytest.mark.parametrize("seed,spin", [(0, 0.0), (1, 0.0), (2, 0.5)])
def test_linear_tets_step_is_backward_euler(orc, seed, spin):
    s = _linear_block(seed=seed, spin=spin)
    # deform the start state so that the elastic force is not zero
    s["pos"] = (s["pos"].astype(np.float64) * np.array([1.03, 0.98, 1.0])).astype(np.float32)
    o = orc.Oracle(s, newton_iters=20, cr_iters=400, line_search=1, eps=0.0)
    o.step()
    v = o.get_state()["vel"]
    ref = _backward_euler(s)
    assert np.linalg.norm(v - ref) <= 1e-8 * np.linalg.norm(ref), (np.linalg.norm(v - ref), np.linalg.norm(ref))


def test_undeformed_linear_block_falls_freely(orc):
    """At the rest shape the strain and the elastic force are zero: every
    particle gets h g, and the multipliers stay zero."""
    s = _linear_block(seed=3, stretch=0.0, lift=0.0)   # positions equal to the rest shape, bit for bit
    s["vel"] = np.zeros_like(s["vel"])
    o = orc.Oracle(s, newton_iters=10, cr_iters=100, line_search=1)
    o.step()
    np.testing.assert_allclose(o.get_state()["vel"], np.tile(H * GRAV, (len(s["mass"]), 1)), rtol=0, atol=1e-12)
    assert np.abs(o.get_lambda()).max() < 1e-9


def test_linear_tet_rows_are_strain_derivatives(orc):
    """The linear tet rows are d s / dx (h^-1 d s(q(u)) / du through x = x^- + h u)."""
    s = _linear_block(seed=4)
    o = orc.Oracle(s)
    c0, J = o.eval_constraints()
    nl = len(s["l_v"])
    lb = o.R - 6 * nl
    x0 = s["pos"].astype(np.float64)
    for t, (v, rest) in enumerate(zip(s["l_v"], s["l_rest"].astype(np.float64))):
        np.testing.assert_allclose(c0[lb + 6 * t:lb + 6 * t + 6], _strain(x0[list(v)], rest), rtol=0, atol=1e-12)
    rng = np.random.default_rng(5)
    du = rng.normal(size=J.shape[1])
    d = 1e-2   # the small strain is linear in x: central differences are exact up to rounding
    for t, (v, rest) in enumerate(zip(s["l_v"], s["l_rest"].astype(np.float64))):
        xp = x0 + d * H * du.reshape(-1, 3)
        xm = x0 - d * H * du.reshape(-1, 3)
        fd = (_strain(xp[list(v)], rest) - _strain(xm[list(v)], rest)) / (2 * d * H)
        np.testing.assert_allclose(J[lb + 6 * t:lb + 6 * t + 6] @ du, fd, rtol=1e-7, atol=1e-9)
