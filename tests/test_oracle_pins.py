"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden), closed forms, invariants, brute force, or an
independent definition (dense linear algebra, finite differences).
"""
import os

import numpy as np
import pytest

from paper_1907_04587_gb300 import scenes

H = 1.0 / 60.0
G = 9.81
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


# ---------------------------------------------------------------------------------
# NCP functions (Sec. 4.1, 4.2, App. A.1)

def test_fb_is_ncp_function(orc):
    """phi_FB(a, b) = 0  <=>  a >= 0, b >= 0, a b = 0 (Eq. ncp, Sec. 4.2)."""
    vals = [-2.0, -0.5, -1e-3, 0.0, 1e-3, 0.5, 2.0]
    for a in vals:
        for b in vals:
            phi = orc.fb(a, b)
            comp = a >= 0 and b >= 0 and a * b == 0
            assert (abs(phi) < 1e-15) == comp, (a, b, phi)
            if a < 0 or b < 0:
                assert phi < 0


def test_fb_contact_derivatives(orc):
    """alpha, S of App. A.1 are the partial derivatives of the r-scaled FB function."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        Cn, lam, r = rng.normal(), rng.normal(), rng.uniform(0.1, 3.0)
        phi, al, S = orc.fb_contact(Cn, lam, r)
        d = 1e-6
        dphi_dC = (orc.fb_contact(Cn + d, lam, r)[0] - orc.fb_contact(Cn - d, lam, r)[0]) / (2 * d)
        dphi_dl = (orc.fb_contact(Cn, lam + d, r)[0] - orc.fb_contact(Cn, lam - d, r)[0]) / (2 * d)
        assert abs(al - dphi_dC) < 1e-6
        assert abs(S - dphi_dl) < 1e-6
    # subgradient choice at the kink (Sec. 4.2): alpha(0,0) = 0, beta(0,0) = 1 -> S = r
    phi, al, S = orc.fb_contact(0.0, 0.0, 0.7)
    assert (phi, al, S) == (0.0, 0.0, 0.7)


def test_min_map_cases(orc):
    """Minimum map and its derivatives (Sec. 4.1 / App. A.1)."""
    assert orc.min_contact(0.1, 1.0, 0.5) == (0.1, 1.0, 0.0)     # C <= r lam: active
    assert orc.min_contact(2.0, 1.0, 0.5) == (0.5, 0.0, 0.5)     # inactive: phi = r lam


def test_fig7_rscaled_min_map_one_step(orc):
    """Fig. 7: with r equal to the constraint slope, the r-scaled minimum map of
    c = lambda/4 - 1/8 is linear and Newton reaches lambda = 1/2 in one step
    from any start; Fischer-Burmeister converges to the same root."""
    g = golden("fig7_rscaling.txt")
    a, b, sol = g["slope"], g["offset"], g["solution_lambda"]
    for lam0 in [-3.0, 0.0, 0.2, 2.0, 10.0]:
        phi, al, S = orc.min_contact(a * lam0 + b, lam0, a)
        lam1 = lam0 - phi / (al * a + S)
        assert abs(lam1 - sol) < 1e-14
    lam = 5.0
    for _ in range(60):
        phi, al, S = orc.fb_contact(a * lam + b, lam, a)
        lam -= phi / (al * a + S)
    assert abs(lam - sol) < 1e-12


# ---------------------------------------------------------------------------------
# Friction compliance W (Sec. 4.3, App. A.2)

def test_fig4_cone_limit(orc):
    """Fig. 4: at the cone limit (|lambda_f| = mu lambda_n) with sliding speed
    u0 both NCP friction functions vanish: W = u0 / |lambda_f| and
    phi_f = D^T qdot + W lambda_f = 0 for a friction force opposing motion."""
    g = golden("fig4_friction.txt")
    u0, ln, mu, lim = g["u0_m_per_s"], g["lambda_n_N"], g["mu"], g["cone_limit_lambda_f_N"]
    assert mu * ln == lim
    for r in [1e-3, 0.1, 1.0, 10.0]:
        w = orc.w_fb(u0, lim, mu * ln, r)
        assert abs(w - u0 / lim) < 1e-12
        assert abs(u0 + w * (-lim)) < 1e-12
        assert abs(orc.w_min(u0, lim, mu * ln, r) - u0 / lim) < 1e-12


def test_w_stick_and_penalty(orc):
    """Inside the cone with no sliding W = 0 (stick); outside the cone W > 0
    pushes the friction force back (Fig. 4 left, past the dashed line)."""
    for r in [0.01, 1.0]:
        assert abs(orc.w_fb(0.0, 2.0, 5.0, r)) < 1e-15
        assert orc.w_min(0.0, 2.0, 5.0, r) == 0.0
        assert orc.w_fb(0.0, 6.0, 5.0, r) > 0.0
        assert orc.w_min(0.0, 6.0, 5.0, r) > 0.0


def test_w_asymptote_past_cone_limit(orc):
    """Fig. 4 (left): past the cone limit W grows to a vertical asymptote where
    the FB fixed-point friction magnitude (App. A.2) reaches zero,
    |lambda_f|* = mu lambda_n + sqrt(2 vt r mu lambda_n + r^2 (mu lambda_n)^2) / r;
    beyond it the friction rows take the inactive form (zero friction)."""
    for vt, mln, r in [(0.5, 5.0, 0.3), (0.1, 2.0, 1e-3), (0.0, 1.0, 0.05)]:
        lim = mln + np.sqrt(2 * vt * r * mln + (r * mln) ** 2) / r
        ws = [orc.w_fb(vt, f * mln, mln, r) for f in (1.0, 1.2, 1.5)]
        if vt > 0:
            assert ws[0] < ws[1] < ws[2]
        assert orc.fb_friction_active(vt, lim * (1 - 1e-9), mln, r)
        assert not orc.fb_friction_active(vt, lim * (1 + 1e-9), mln, r)
        assert not orc.fb_friction_active(vt, 0.5, 0.0, r)


# ---------------------------------------------------------------------------------
# Neo-Hookean compliance (Sec. 9.2.2, App. B)

def test_nh_rest_state_stress_free(orc):
    for E, nu in [(1e5, 0.45), (5e4, 0.4), (1e7, 0.3)]:
        C1, D1, al = orc.nh_params(E, nu)
        g, Hs = orc.nh_grad_hess([1.0, 1.0, 1.0], C1, D1, al)
        assert np.abs(g).max() < 1e-9 * E
        assert np.all(np.linalg.eigvalsh(Hs) > 0)
        # Lame parameters of the stated (E, nu)
        mu = E / (2 * (1 + nu)); la = E * nu / ((1 + nu) * (1 - 2 * nu))
        assert abs(2 * C1 - mu) < 1e-9 * E and abs(2 * D1 - la) < 1e-9 * E


def test_nh_gradient_hessian_finite_differences(orc):
    """The App. B gradient/Hessian are the derivatives of Psi (finite differences)."""
    rng = np.random.default_rng(2)
    C1, D1, al = orc.nh_params(1e5, 0.45)
    for _ in range(20):
        s = rng.uniform(0.6, 1.4, 3)
        g, Hs = orc.nh_grad_hess(s, C1, D1, al)
        d = 1e-6
        for i in range(3):
            e = np.zeros(3); e[i] = d
            fd = (orc.nh_energy(s + e, C1, D1, al) - orc.nh_energy(s - e, C1, D1, al)) / (2 * d)
            assert abs(fd - g[i]) < 1e-5 * max(1.0, abs(g[i]))
            gp, _ = orc.nh_grad_hess(s + e, C1, D1, al)
            gm, _ = orc.nh_grad_hess(s - e, C1, D1, al)
            assert np.allclose((gp - gm) / (2 * d), Hs[:, i], rtol=1e-5, atol=1e-3)


def test_svd3_signed(orc):
    rng = np.random.default_rng(3)
    for k in range(200):
        F = np.eye(3) + 0.4 * rng.normal(size=(3, 3))
        if k % 5 == 0:
            F[:, 0] *= -1  # inverted element
        U, s, V = orc.svd3(F)
        assert np.allclose(U @ np.diag(s) @ V.T, F, atol=1e-12)
        assert np.allclose(U.T @ U, np.eye(3), atol=1e-12) and np.allclose(V.T @ V, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(U) - 1) < 1e-12 and abs(np.linalg.det(V) - 1) < 1e-12
        ref = np.linalg.svd(F, compute_uv=False)
        assert np.allclose(np.abs(s), ref, atol=1e-12)
        assert s[0] >= s[1] >= abs(s[2]) - 1e-12
        assert np.sign(s[2]) == np.sign(np.linalg.det(F))


def test_basis_orthonormal(orc):
    rng = np.random.default_rng(4)
    for _ in range(100):
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        t1, t2 = orc.basis(n)
        M = np.stack([t1, t2, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.allclose(np.cross(t1, t2), n, atol=1e-12)


# ---------------------------------------------------------------------------------
# physical closed forms (Sec. 3.3-3.5, 5, 6)

def _particle_on_plane(v, mu, mass=2.0):
    b = scenes.SceneBuilder()
    i = b.add_particle((0.0, 0.0, 0.0), vel=v, mass=mass)
    b.add_contact(i, -1, (0, 0, 0), (0, 0, 0), (0, 0, 1), 0.0, mu)
    return b.build()


@pytest.mark.parametrize("v0", [0.5, 0.1, 0.05, 0.0])
def test_sliding_particle_closed_form(orc, v0):
    """Coulomb friction on a resting particle: |v+| = max(0, |v-| - h mu g)."""
    s = _particle_on_plane((0.6 * v0, 0.8 * v0, 0.0), 0.5)
    o = orc.Oracle(s, newton_iters=80, cr_iters=10, tol_rel=1e-12)
    st = o.step()
    v = o.get_state()["vel"][0].astype(np.float64)
    v_in = s["vel"][0].astype(np.float64)
    expect = max(0.0, np.hypot(v_in[0], v_in[1]) - H * 0.5 * G)
    assert abs(np.hypot(v[0], v[1]) - expect) < 1e-9
    assert abs(v[2]) < 1e-9
    if v0 > 0.1:  # sliding: velocity keeps its direction
        assert abs(v[0] * 0.8 - v[1] * 0.6) < 1e-8
    assert st["merit_final"] <= 1e-9 * st["merit0"]


def _box_on_plane(mu, m=1000.0, e=1.0):
    b = scenes.SceneBuilder()
    i = b.add_rigid((0, 0, e / 2), mass=m, inertia=(m * e * e / 6,) * 3)
    for p in scenes.box_bottom_corners((e, e, e)):
        b.add_contact(i, -1, p, (p[0], p[1], 0), (0, 0, 1), 0.0, mu)
    return b.build()


@pytest.mark.parametrize("theta_deg,slip", [(15.0, False), (20.0, False), (40.0, True), (50.0, True)])
def test_incline_stick_slip(orc, theta_deg, slip):
    """Box on an incline (gravity tilted): sticks for tan(theta) < mu, else slips
    with dv = h g (sin(theta) - mu cos(theta)) per step."""
    mu = 0.5
    th = np.deg2rad(theta_deg)
    o = orc.Oracle(_box_on_plane(mu), newton_iters=100, cr_iters=50, tol_rel=1e-10,
                   gravity=(G * np.sin(th), 0.0, -G * np.cos(th)))
    st = o.step()
    v = o.get_state()["vel"][0]
    dv = H * G * (np.sin(th) - mu * np.cos(th)) if slip else 0.0
    assert (np.tan(th) > mu) == slip
    assert abs(v[0] - dv) < 1e-8
    assert abs(v[2]) < 1e-8
    assert st["merit_final"] <= 1e-9 * st["merit0"]


def test_resting_stack_normal_impulses(orc):
    """A resting stack: the contacts under layer k carry (4 - k) m g h."""
    b = scenes.SceneBuilder(); m = 1000.0
    for k in range(4):
        i = b.add_rigid((0, 0, 0.5 + k), mass=m, inertia=(m / 6,) * 3)
        for p in scenes.box_bottom_corners((1, 1, 1)):
            if k == 0:
                b.add_contact(i, -1, p, (p[0], p[1], 0), (0, 0, 1), 0.0, 0.5)
            else:
                b.add_contact(i, k - 1, p, (p[0], p[1], 0.5), (0, 0, 1), 0.0, 0.5)
    o = orc.Oracle(b.build(), newton_iters=100, cr_iters=100, tol_rel=1e-12)
    st = o.step()
    lam = o.get_lambda()
    for k in range(4):
        assert abs(H * lam[12 * k:12 * k + 12:3].sum() - m * G * H * (4 - k)) < 1e-8
    # NCP residual zero at convergence: every contact has C = 0 and lambda_n > 0
    c, _ = o.eval_constraints(with_jacobian=False)
    assert np.abs(np.minimum(c[0::3], lam[0::3])).max() < 1e-10
    assert np.abs(o.get_state()["vel"]).max() < 1e-10
    assert st["merit_final"] <= 1e-12 * st["merit0"]


def test_lcp_brute_force_frictionless_corner(orc):
    """Frictionless particle driven into a corner of three planes (plus one plane
    it leaves): the converged Newton multipliers equal the unique solution of the
    LCP 0 <= w = q + M lam  perp  lam >= 0 found by enumerating all 2^4 active sets."""
    rng = np.random.default_rng(5)
    for trial in range(5):
        normals = [np.array([0, 0, 1.0]), np.array([1.0, 0, 0.2]), np.array([0.1, 1.0, 0]), np.array([-1.0, 0.1, 0.1])]
        normals = [n / np.linalg.norm(n) for n in normals]
        x0 = np.zeros(3)
        gaps = np.array([0.0, 1e-3, -5e-4, 0.02]) * (1 + 0.1 * trial)
        v = np.array([-0.3, -0.2, -0.5]) + 0.05 * rng.normal(size=3)
        m = 1.5
        b = scenes.SceneBuilder()
        i = b.add_particle(x0, vel=v, mass=m)
        for n, gap in zip(normals, gaps):
            b.add_contact(i, -1, (0, 0, 0), -gap * n, n, 0.0, 0.0)
        s = b.build()
        o = orc.Oracle(s, newton_iters=200, cr_iters=20, tol_rel=1e-13, geom_stiffness=0)
        o.step()
        lam_n = o.get_lambda()[0::3]
        # brute-force LCP on the float32-rounded scene values
        N = s["c_n"].astype(np.float64)
        pb = s["c_pb"].astype(np.float64)
        ut = s["vel"][0].astype(np.float64) + H * np.array([0, 0, -G])
        Cm = np.array([N[k] @ (x0 - pb[k]) for k in range(4)])
        q = Cm + H * N @ ut
        Mm = H * H * N @ N.T / float(s["mass"][0])
        found = []
        for mask in range(16):
            A = [k for k in range(4) if mask >> k & 1]
            lam = np.zeros(4)
            if A:
                sub = Mm[np.ix_(A, A)]
                if np.linalg.matrix_rank(sub) < len(A):
                    continue
                lam[A] = np.linalg.solve(sub, -q[A])
            w = q + Mm @ lam
            if lam.min() >= -1e-12 and w.min() >= -1e-12:
                found.append(lam)
        assert len(found) >= 1
        lam_ref = found[0]
        assert np.allclose(lam_n, lam_ref, atol=1e-7 * max(1.0, np.abs(lam_ref).max()))


# ---------------------------------------------------------------------------------
# linear algebra of the Newton step (Sec. 6.1, 6.2, 8.2, 8.4)

def _mixed_scene():
    """Small scene with every row type: contacts, a revolute joint, NH tets."""
    s = scenes.chain_block(seed=1, hexes=2, links=3)
    return s


def test_schur_equals_saddle_point(orc):
    """Eq. schur_system + du formula reproduce the solution of the full
    saddle-point system Eq. group_system (with C + eps I)."""
    s = _mixed_scene()
    o = orc.Oracle(s, newton_iters=4, cr_iters=30)
    L = o.linearize(n_before=2)
    J, Hi, Cm, g, hv, b = L["J"], L["Hinv"], L["C"], L["g"], L["hvec"], L["b"]
    R, D = J.shape
    eps = 1e-6
    Hm = np.linalg.inv(Hi)
    K = np.block([[Hm, -J.T], [J, Cm + eps * np.eye(R)]])
    sol = np.linalg.solve(K, -np.concatenate([g, hv]))
    du_ref, hdl_ref = sol[:D], sol[D:]
    A = J @ Hi @ J.T + Cm + eps * np.eye(R)
    assert np.allclose(A, A.T, atol=1e-9 * np.abs(A).max())
    dl = np.linalg.solve(A, b)
    du = Hi @ (J.T @ dl * H - g)
    assert np.allclose(dl * H, hdl_ref, rtol=1e-8, atol=1e-10 * np.abs(hdl_ref).max())
    assert np.allclose(du, du_ref, rtol=1e-8, atol=1e-10 * np.abs(du_ref).max())


def test_stiffness_form_equivalence(orc):
    """Compliant-only system (NH tets, no contacts/joints): the stiffness form
    [H + J^T C^-1 J] du = -g - J^T C^-1 h (Sec. 6.2) gives the Schur du."""
    s = scenes.chain_block(seed=2, hexes=2, links=1)
    keep = {k: v for k, v in s.items()}
    for k in ("c_body", "c_pa", "c_pb", "c_n", "c_d", "c_mu"):
        keep[k] = keep[k][:0]
    for k in ("j_body", "j_pa", "j_pb", "j_axa", "j_axb", "j_compliance"):
        keep[k] = keep[k][:0]
    o = orc.Oracle(keep, newton_iters=3, cr_iters=10)
    L = o.linearize(n_before=1)
    J, Hi, Cm, g, hv, b = L["J"], L["Hinv"], L["C"], L["g"], L["hvec"], L["b"]
    R = J.shape[0]
    Ce = Cm + 1e-6 * np.eye(R)
    dl = np.linalg.solve(J @ Hi @ J.T + Ce, b)
    du_schur = Hi @ (J.T @ dl * H - g)
    Ci = np.linalg.inv(Ce)
    du_stiff = np.linalg.solve(np.linalg.inv(Hi) + J.T @ Ci @ J, -g - J.T @ Ci @ hv)
    assert np.allclose(du_schur, du_stiff, rtol=1e-7, atol=1e-9 * np.abs(du_stiff).max())


def test_apply_A_and_pcr(orc):
    """Matrix-free operator = dense J Hinv J^T + C + eps I; PCR after R iterations
    equals the Cholesky solution; ||r||_P is monotone (Sec. 8.2); the k-th PCR
    iterate is the minimiser of ||b - A x||_P over the Krylov space K_k(PA, Pb)."""
    s = _mixed_scene()
    o = orc.Oracle(s, newton_iters=4, cr_iters=30)
    L = o.linearize(n_before=1)
    J, Hi, Cm, b = L["J"], L["Hinv"], L["C"], L["b"]
    R = J.shape[0]
    A = J @ Hi @ J.T + Cm + 1e-6 * np.eye(R)
    rng = np.random.default_rng(6)
    x = rng.normal(size=R)
    assert np.allclose(o.apply_A(x), A @ x, rtol=1e-10, atol=1e-10 * np.abs(A @ x).max())
    # Krylov definition check for the first iterates
    P = 1.0 / np.diag(A)
    for k in range(1, 6):
        xk, hist = o.pcr(k)
        Kb = [P * b]
        for _ in range(k - 1):
            Kb.append(P * (A @ Kb[-1]))
        Kmat = np.stack(Kb, 1)
        Ws = np.sqrt(P)[:, None]
        c, *_ = np.linalg.lstsq(Ws * (A @ Kmat), np.sqrt(P) * b, rcond=None)
        xref = Kmat @ c
        assert np.allclose(xk, xref, rtol=1e-6, atol=1e-8 * np.abs(xref).max())
    # small system: exact after R iterations (well-conditioned subproblem)
    x_chol = np.linalg.solve(A, b)
    xk, hist = o.pcr(3 * R)
    live = hist[: np.argmax(hist < 1e-12 * hist[0])] if np.any(hist < 1e-12 * hist[0]) else hist
    assert len(live) > 5
    assert np.all(np.diff(live) <= 1e-12 * hist[0])
    assert np.linalg.norm(A @ xk - b) <= 1e-6 * np.linalg.norm(b)
    assert np.allclose(xk, x_chol, rtol=1e-4, atol=1e-6 * np.abs(x_chol).max())


def _kinematic_q(s, u, h=H):
    """q(u) = q^- + h G(q^-) u with the kinematic map of Sec. 9.4 (independent restatement)."""
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


def test_geometric_rows_finite_differences(orc):
    """The geometric rows (contact normal rows, joint rows, tet ds/dx rows) are
    h^-1 d c(q(u)) / du at u = 0, by central differences through the kinematic map."""
    s = scenes.chain_block(seed=3, hexes=2, links=3)
    s["quat"][1] = scenes.quat_axis_angle((0.3, 1.0, 0.2), 0.4).astype(np.float32)
    o = orc.Oracle(s)
    c0, Jg = o.eval_constraints()
    R, D = Jg.shape
    rng = np.random.default_rng(7)
    nc = len(s["c_body"])
    rows = [r for r in range(R) if not (r < 3 * nc and r % 3 != 0)]  # skip velocity-level friction rows
    for trial in range(6):
        du = rng.normal(size=D)
        d = 1e-5
        pp, qp = _kinematic_q(s, d * du)
        pm, qm = _kinematic_q(s, -d * du)
        o.set_state(pos=pp, quat=qp)
        cp, _ = o.eval_constraints(with_jacobian=False)
        o.set_state(pos=pm, quat=qm)
        cm, _ = o.eval_constraints(with_jacobian=False)
        o.set_state(pos=s["pos"].astype(np.float64), quat=s["quat"].astype(np.float64))
        fd = (cp - cm) / (2 * d * H)
        an = Jg @ du
        err = np.abs(fd[rows] - an[rows])
        assert err.max() < 1e-5 * max(1.0, np.abs(an[rows]).max()), err.max()


def test_friction_rows_are_point_velocity(orc):
    """Friction rows D map u to the tangential relative velocity of the contact
    points (Sec. 3.4): compare with finite differences of the point positions."""
    s = scenes.cube_stack(seed=0)
    o = orc.Oracle(s)
    _, Jg = o.eval_constraints()
    rng = np.random.default_rng(8)
    du = rng.normal(size=Jg.shape[1])
    d = 1e-5
    R = scenes.quat_rot
    pp, qp = _kinematic_q(s, d * du)
    pm, qm = _kinematic_q(s, -d * du)

    def pts(pos, quat):
        out = []
        for c in range(len(s["c_body"])):
            a, bb = s["c_body"][c]
            wa = pos[a] + R(quat[a]) @ s["c_pa"][c]
            wb = s["c_pb"][c].astype(np.float64) if bb < 0 else pos[bb] + R(quat[bb]) @ s["c_pb"][c]
            out.append(wa - wb)
        return np.array(out)

    vrel = (pts(pp, qp) - pts(pm, qm)) / (2 * d * H)
    for c in range(len(s["c_body"])):
        t1, t2 = orc.basis(s["c_n"][c])
        assert abs(Jg[3 * c + 1] @ du - t1 @ vrel[c]) < 1e-6
        assert abs(Jg[3 * c + 2] @ du - t2 @ vrel[c]) < 1e-6


# ---------------------------------------------------------------------------------
# geometric stiffness (Sec. 8.3), joints, free fall

def test_geometric_stiffness_nonnegative_shift(orc):
    """H~_kk >= M_kk (the shift is clamped non-negative, Eq. mass_update_2), and
    rigid blocks are untouched (particle DOFs only, Sec. 11)."""
    s = scenes.chain_block(seed=4, hexes=3, links=2)
    o = orc.Oracle(s, newton_iters=6, cr_iters=40)
    for n in range(0, 4):
        L = o.linearize(n_before=n)
        Hi = np.diag(L["Hinv"])
        off = 0
        for i in range(len(s["mass"])):
            k = 6 if s["kind"][i] == 0 else 3
            if k == 3:
                assert np.all(Hi[off:off + 3] <= 1.0 / float(s["mass"][i]) * (1 + 1e-12))
            else:
                assert np.allclose(Hi[off:off + 3], 1.0 / float(s["mass"][i]))
            off += k


def test_free_fall_and_gyroscopic(orc):
    """No constraints: Newton with damping t converges geometrically to u = u~
    (explicit gravity, Sec. 5) -- error (1 - t)^N after N iterations."""
    b = scenes.SceneBuilder()
    b.add_particle((0, 0, 1), vel=(1.0, 0, 0), mass=1.0)
    b.add_rigid((0, 0, 2), omega=(0.0, 0.0, 2.0), mass=2.0, inertia=(1.0, 2.0, 3.0))
    s = b.build()
    o = orc.Oracle(s, newton_iters=6, cr_iters=5)
    o.step()
    st = o.get_state()
    assert abs(st["vel"][0][2] - (-G * H) * (1 - 0.25 ** 6)) < 1e-12
    assert abs(st["vel"][0][0] - 1.0 * (1 - 0.25 ** 6)) < 1e-12
    # spin about a principal axis: the gyroscopic torque w x (I w) vanishes
    assert abs(st["omega"][1][2] - 2.0 * (1 - 0.25 ** 6)) < 1e-12


def test_pendulum_drift_and_period(orc):
    """Revolute pendulum (hard joint, no index reduction, Sec. 5): the joint error
    stays bounded and the small-angle period matches 2 pi sqrt(I_p / (m g l))."""
    Lx, m = 0.5, 1.0
    I = scenes.box_inertia(m, (Lx, 0.05, 0.05))
    b = scenes.SceneBuilder()
    th0 = 0.1
    cx, cz = 0.5 * Lx * np.sin(th0), -0.5 * Lx * np.cos(th0)
    q = scenes.quat_axis_angle((0, 1, 0), np.pi / 2 - th0)  # long axis x rotated to hang down
    i = b.add_rigid((cx, 0, cz), q, mass=m, inertia=I)
    b.add_revolute(i, -1, (-Lx / 2, 0, 0), (0, 0, 0), (0, 1, 0), (0, 1, 0), 0.0)
    s = b.build()
    o = orc.Oracle(s, newton_iters=8, cr_iters=30)
    xs, drift = [], []
    for k in range(240):
        o.step()
        st = o.get_state()
        xs.append(st["pos"][0][0])
        R = scenes.quat_rot(st["quat"][0])
        drift.append(np.linalg.norm(st["pos"][0] + R @ np.array([-Lx / 2, 0, 0])))
    assert max(drift) < 2e-3
    xs = np.array(xs)
    cross = np.nonzero((xs[:-1] > 0) & (xs[1:] <= 0))[0]
    period = np.mean(np.diff(cross)) * H
    Ip = I[1] + m * (Lx / 2) ** 2
    T = 2 * np.pi * np.sqrt(Ip / (m * G * Lx / 2))
    assert abs(period - T) / T < 0.05


@pytest.mark.parametrize("e", [0.0, 1e-5, 1e-4, 1e-3, 1e6])
def test_compliant_joint_one_step_closed_form(orc, e):
    """Compliant joint rows (Sec. 3.2: C = e / h^2, h = (c + e lambda) / h): a
    body of mass m hanging at rest from a world anchor at its centre.  The
    vertical row is implicit Euler on a spring of stiffness 1/e, so one step
    gives m v = h lambda - m g h with h v + e lambda = 0, i.e.
    v = -m g h / (m + h^2 / e): 0 for a hard joint, free fall as e grows."""
    m = 3.0
    b = scenes.SceneBuilder()
    i = b.add_rigid((0.2, -0.1, 1.0), (1, 0, 0, 0), mass=m, inertia=(0.2, 0.3, 0.4))
    b.add_revolute(i, -1, (0, 0, 0), (0.2, -0.1, 1.0), (0, 1, 0), (0, 1, 0), e)
    s = b.build()
    o = orc.Oracle(s, newton_iters=30, cr_iters=30, line_search=1)
    o.step()
    v = o.get_state()["vel"][0]
    x0 = np.asarray(s["pos"][0], np.float64)
    anchor = np.asarray(s["j_pb"][0], np.float64)
    assert np.array_equal(x0, anchor)
    ef = float(np.float32(e))
    expect = 0.0 if ef == 0.0 else -m * G * H / (m + H * H / ef)
    assert abs(v[2] - expect) < 1e-9 * G * H, (v, expect)
    assert np.all(np.abs(v[:2]) < 1e-12) and np.all(np.abs(o.get_state()["omega"][0]) < 1e-12)
