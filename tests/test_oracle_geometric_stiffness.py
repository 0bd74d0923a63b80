"""Pins of the oracle's diagonal geometric stiffness (Sec. 8.3).

Eq. broyden_update asks for a diagonal H~ with H~ du = dg between consecutive
Newton iterates; with H~ = M - K~ (K~ the diagonal stiffness estimate) the
entry is c_k = [M du - dg]_k / du_k and Eq. mass_update_2 adds max(0, -c_k) to
the particle mass (particles only, Sec. 11).  The oracle reads dg at the
current multipliers (H~ approximates dg/du at fixed lambda, the block of the
Newton system that multiplies du), so that M du - dg = h (J^n - J^{n-1})^T
lambda^n, and regularises the ratio as s_k du_k / (du_k^2 + tau_k^2).

The pins below check the oracle against things other than its own formula:
  * rows whose direction does not change between iterates give no shift,
    although u and lambda both change (a dg taken across the multiplier change
    would add hundreds of times the mass here);
  * on a Neo-Hookean block, the shift equals max(0, -c_k) with c_k computed
    from stretch gradients obtained independently (numpy's SVD and central
    differences), wherever |du_k| is far above the regularisation scale, and
    never exceeds it elsewhere;
  * the shift changes the Newton matrix only, not the solution (Sec. 8.3):
    converged states with and without it agree.
"""
import numpy as np
import pytest

from paper_1907_04587_gb300 import scenes

H = 1.0 / 60.0


def _masses(s):
    """Diagonal of M (rigid: mass on the three linear DOFs, inertia blocks
    are not touched by the shift) and the DOF offset of each body."""
    nb = len(s["mass"])
    dof = np.zeros(nb, int)
    off = 0
    for i in range(nb):
        dof[i] = off
        off += 6 if s["kind"][i] == scenes.RIGID else 3
    M = np.zeros(off)
    for i in range(nb):
        M[dof[i]:dof[i] + (6 if s["kind"][i] == scenes.RIGID else 3)] = s["mass"][i]
    pidx = np.concatenate([np.arange(dof[i], dof[i] + 3) for i in range(nb) if s["kind"][i] == scenes.PARTICLE])
    return M, dof, pidx


def test_no_shift_when_rows_keep_their_direction(orc):
    """Frictionless particles pressed into a plane, min-map NCP (active rows are
    the constant normal n, Sec. 4.1): J^n = J^{n-1}, so H~ = M at every
    iteration even though du and dlambda are large (warm start far above the
    solution).  Differencing g across the multiplier change instead would give
    c_k = h [J^T dlambda]_k / du_k, hundreds of times -M_k."""
    rng = np.random.default_rng(3)
    b = scenes.SceneBuilder()
    for _ in range(6):
        p = (rng.uniform(-1, 1), rng.uniform(-1, 1), -rng.uniform(1e-4, 2e-3))
        v = (rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), -rng.uniform(0.1, 1.0))
        k = b.add_particle(p, vel=v, mass=rng.uniform(0.5, 2.0))
        b.add_contact(k, -1, (0, 0, 0), (p[0], p[1], 0.0), (0, 0, 1), 0.0, 0.0)
    s = b.build()
    o = orc.Oracle(s, newton_iters=8, cr_iters=40, ncp=orc.NCP_MIN)
    M, _, _ = _masses(s)
    lam0 = np.zeros(o.R)
    lam0[0::3] = 400.0
    for n in range(1, 6):
        Lp = o.linearize(n_before=n - 1, lambda0=lam0)
        L = o.linearize(n_before=n, lambda0=lam0)
        du, dl = L["u"] - Lp["u"], L["lam"] - Lp["lam"]
        assert np.abs(du).max() > 1e-3 and np.abs(dl).max() > 1.0
        assert np.array_equal(1.0 / np.diag(L["Hinv"]), M), n
        # the other reading: dg between the two iterates, multipliers changed too
        dg = L["g"] - Lp["g"]
        moving = np.abs(du) > 1e-12
        c_full = (M[moving] * du[moving] - dg[moving]) / du[moving]
        assert (c_full / M[moving]).min() < -100.0


def _signed_stretches(x4, rest):
    """Principal stretches of F = D_s D_m^-1 (Sec. 9.2.2), sorted s1 >= s2 >= |s3|,
    the smallest negated when det F < 0 (numpy's SVD, not the oracle's)."""
    Dm = np.stack([rest[q] - rest[0] for q in (1, 2, 3)], 1)
    Ds = np.stack([x4[q] - x4[0] for q in (1, 2, 3)], 1)
    F = Ds @ np.linalg.inv(Dm)
    s = np.linalg.svd(F, compute_uv=False)
    if np.linalg.det(F) < 0:
        s[2] = -s[2]
    return s


def _stretch_gradient(x4, rest, d=1e-6):
    """d s / d x (3 x 12) by central differences."""
    G = np.zeros((3, 12))
    for j in range(12):
        xp = x4.reshape(-1).copy()
        xm = xp.copy()
        xp[j] += d
        xm[j] -= d
        G[:, j] = (_signed_stretches(xp.reshape(4, 3), rest) - _signed_stretches(xm.reshape(4, 3), rest)) / (2 * d)
    return G


def _tet_block():
    s = scenes.chain_block(seed=2, hexes=2, links=1)
    for k in ("c_body", "c_pa", "c_pb", "c_n", "c_d", "c_mu"):
        s[k] = s[k][:0]
    for k in ("j_body", "j_pa", "j_pb", "j_axa", "j_axb", "j_compliance"):
        s[k] = s[k][:0]
    rng = np.random.default_rng(0)
    part = s["kind"] == scenes.PARTICLE
    s["vel"] = s["vel"].copy()
    s["vel"][part] += rng.normal(scale=0.5, size=(int(part.sum()), 3)).astype(np.float32)
    return s


def test_shift_is_the_secant_of_the_stretch_rows(orc):
    """A deformed Neo-Hookean block (tet rows only; one rigid body without
    constraints).  From the iterates u^{n-1}, u^n and the multipliers lambda^n
    the test forms M du - dg = h sum_i lambda_i (grad s_i(x^n) - grad s_i(x^{n-1}))
    with x = x^- + h u (Sec. 5) and its own stretch gradients, then
    c_k = [M du - dg]_k / du_k (Eq. broyden_update with H~ = M - K~).  The
    oracle's H~_kk - M_kk equals max(0, -c_k) (Eq. mass_update_2) where |du_k|
    is 100 times the regularisation scale tau_k, lies in [0, max(0, -c_k)]
    everywhere, and rigid DOFs keep their mass."""
    s = _tet_block()
    o = orc.Oracle(s, newton_iters=8, cr_iters=60)
    M, dof, pidx = _masses(s)
    pos0 = s["pos"].astype(np.float64)
    active_total = 0
    for n in range(1, 5):
        Lp = o.linearize(n_before=n - 1)
        L = o.linearize(n_before=n)
        un, up, lam = L["u"], Lp["u"], L["lam"]
        tet_row0 = o.R - 3 * len(s["t_v"])
        mdu_minus_dg = np.zeros_like(M)
        for t, (v, rest) in enumerate(zip(s["t_v"], s["t_rest"].astype(np.float64))):
            xn = np.stack([pos0[v[q]] + H * un[dof[v[q]]:dof[v[q]] + 3] for q in range(4)])
            xp = np.stack([pos0[v[q]] + H * up[dof[v[q]]:dof[v[q]] + 3] for q in range(4)])
            dG = _stretch_gradient(xn, rest) - _stretch_gradient(xp, rest)
            f = H * dG.T @ lam[tet_row0 + 3 * t:tet_row0 + 3 * t + 3]
            for q in range(4):
                mdu_minus_dg[dof[v[q]]:dof[v[q]] + 3] += f[3 * q:3 * q + 3]
        du = un - up
        c = np.zeros_like(M)
        nz = du != 0
        c[nz] = mdu_minus_dg[nz] / du[nz]
        printed = np.maximum(0.0, -c)
        shift = 1.0 / np.diag(L["Hinv"]) - M
        tau = 1e-6 + 1e-3 * np.maximum(np.abs(un), np.abs(up))
        far = pidx[np.abs(du[pidx]) > 100 * tau[pidx]]
        assert len(far) > 0
        assert np.all(np.abs(shift[far] - printed[far]) <= 2e-4 * (M[far] + printed[far])), n
        # (shift recovered as 1 / H~^-1 - M: rounding of 1e-12 M allowed)
        assert np.all(shift[pidx] >= -1e-12 * M[pidx])
        assert np.all(shift[pidx] <= printed[pidx] * (1 + 1e-9) + 1e-12 * M[pidx])
        rigid = np.setdiff1d(np.arange(len(M)), pidx)
        assert np.array_equal(np.diag(L["Hinv"])[rigid][:3], 1.0 / M[rigid][:3])
        active_total += int((printed[far] > 1e-3 * M[far]).sum())
    assert active_total > 20    # the shift is active on many DOFs of this scene


@pytest.mark.parametrize("seed,hexes,links", [(0, 3, 3), (1, 2, 3)])
def test_shift_does_not_change_the_converged_solution(orc, seed, hexes, links):
    """Sec. 8.3: the shift changes the Newton matrix, not the residual, so
    solving to a tight merit tolerance with and without it reaches the same
    state (chain on a Neo-Hookean block: contacts, joints and tets)."""
    s = scenes.chain_block(seed=seed, hexes=hexes, links=links)
    out = {}
    for gs in (orc.GS_OFF, orc.GS_PARTICLES):
        o = orc.Oracle(s, newton_iters=200, cr_iters=2000, tol_rel=1e-12, line_search=1, geom_stiffness=gs)
        st = o.step()
        assert st["merit_final"] <= 1e-12 * st["merit0"], gs
        out[gs] = (o.get_state(), o.get_lambda(), st["newton_done"])
    (a, la, na), (b, lb, nb_) = out[orc.GS_OFF], out[orc.GS_PARTICLES]
    assert na != nb_      # the iterations differ ...
    ua = np.concatenate([a["vel"].ravel(), a["omega"].ravel()])
    ub = np.concatenate([b["vel"].ravel(), b["omega"].ravel()])
    assert np.linalg.norm(ua - ub) <= 1e-6 * np.linalg.norm(ua)      # ... the solution does not
    assert np.linalg.norm(la - lb) <= 1e-6 * np.linalg.norm(la)
