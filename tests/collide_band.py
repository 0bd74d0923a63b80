"""Comparison of two contact lists of the same scene whose candidate and face
decisions were taken in different precisions (Sec. 3.3, Sec. 10: a contact
exists when a vertex is within the margin of a shape at the start of the step
or at its position predicted with the unconstrained velocity; inside a box the
normal is that of the face of least penetration).

Such lists may differ only where the decision is within rounding: a
vertex-shape pair present in one list only must have a distance within the
band of the margin (at the start or at the predicted position); a pair in
both lists whose normals differ by a face must have its two nearest faces tied
within the band.  The band is measured in FP32 units of the coordinates
involved: EPS32 * (|p| + |x_B| + |e_B| + h (|u_A| + |u_B|)), |.| the largest
component.  Everything here is FP64 numpy, written from the definition."""
import numpy as np

from paper_1907_04587_gb300 import scenes

EPS32 = 2.0 ** -24


def contact_keys(c, planes):
    """(body a, corner of a, shape) -> index: the corner is read from the
    signs of the body-frame point (bit i set for +half on axis i); the shape
    is the box's body id, or -1 - j for plane j (found from the normal)."""
    k = (np.asarray(c["c_pa"]) > 0).astype(np.int64) @ np.array([1, 2, 4])
    cb = np.asarray(c["c_body"])
    pn = np.asarray(planes, np.float64)[:, :3]
    out = {}
    for i, (a, kk, b) in enumerate(zip(cb[:, 0], k, cb[:, 1])):
        if b < 0:
            b = -1 - int(np.argmax(pn @ np.asarray(c["c_n"][i], np.float64)))
        out[(int(a), int(kk), int(b))] = i
    return out


def _unit_rot(q):
    q = np.asarray(q, np.float64)
    return scenes.quat_rot(q / np.linalg.norm(q))


def _vertex(s, a, k):
    """World vertex p, lever arm r, velocity of the point u_A(p), corner (local)."""
    half = np.asarray(s["half"], np.float64)
    if s["kind"][a] == scenes.RIGID:
        cl = np.where([(k >> i) & 1 for i in range(3)], half[a], -half[a])
        r = _unit_rot(s["quat"][a]) @ cl
    else:
        cl = np.zeros(3)
        r = np.zeros(3)
    p = np.asarray(s["pos"][a], np.float64) + r
    u = np.asarray(s["vel"][a], np.float64) + np.cross(np.asarray(s["omega"][a], np.float64), r)
    return p, r, u, cl


def _pair_geometry(s, key, planes, h):
    """Distances at the start and at the predicted position, the box-frame
    start point (None for a plane) and the band's scale."""
    a, k, b = key
    p, r, ua, cl = _vertex(s, a, k)
    if b < 0:
        raise KeyError("plane pairs are keyed by plane below")
    xb = np.asarray(s["pos"][b], np.float64)
    Rb = _unit_rot(s["quat"][b])
    e = np.asarray(s["half"][b], np.float64)
    rb = p - xb
    ub = np.asarray(s["vel"][b], np.float64) + np.cross(np.asarray(s["omega"][b], np.float64), rb)
    d = []
    q0 = Rb.T @ rb
    for rr in (rb, rb + h * (ua - ub)):
        q = Rb.T @ rr
        d.append(float(np.linalg.norm(np.maximum(np.abs(q) - e, 0.0))))
    scale = np.abs(p).max() + np.abs(xb).max() + e.max() + h * (np.abs(ua).max() + np.abs(ub).max())
    return d, q0, e, scale


def _plane_pair(s, a, k, plane, h):
    p, r, ua, cl = _vertex(s, a, k)
    n, o = np.asarray(plane[:3], np.float64), float(plane[3])
    d0 = n @ p - o
    d1 = d0 + h * (n @ ua)
    scale = np.abs(p).max() + abs(o) + h * np.abs(ua).max()
    return [d0, d1], scale


def compare(s, A, B, planes, margin, h):
    """Returns a dict of the worst band ratios (in units of EPS32 * scale):
    'membership' over pairs in one list only, 'face' over pairs whose normals
    differ by a face decision, 'normal' the worst |dn| * dist / (EPS32 |q|) of
    the other common box pairs (normals of points near an edge are sensitive
    to the rotation's rounding), and the counts."""
    ka, kb = contact_keys(A, planes), contact_keys(B, planes)
    out = dict(membership=0.0, face=0.0, normal=0.0, n_only=0, n_face=0, n_common=0)
    for key in set(ka) ^ set(kb):
        a, k, b = key
        out["n_only"] += 1
        if b < 0:
            d, scale = _plane_pair(s, a, k, planes[-1 - b], h)
        else:
            d, _, _, scale = _pair_geometry(s, key, planes, h)
        out["membership"] = max(out["membership"], min(abs(x - margin) for x in d) / (EPS32 * scale))
    common = sorted(set(ka) & set(kb))
    out["n_common"] = len(common)
    for key in common:
        if key[2] < 0:
            continue
        na, nb = np.asarray(A["c_n"][ka[key]], np.float64), np.asarray(B["c_n"][kb[key]], np.float64)
        dn = np.abs(na - nb).max()
        if dn <= 1e-9:
            continue
        _, q0, e, scale = _pair_geometry(s, key, planes, h)
        dist = float(np.linalg.norm(np.maximum(np.abs(q0) - e, 0.0)))
        if dn > 0.1:
            out["n_face"] += 1
            depth = np.sort(e - np.abs(q0))
            gap = min(depth[1] - depth[0], abs(np.max(np.abs(q0) - e)))
            out["face"] = max(out["face"], gap / (EPS32 * scale))
        elif dist > 0:
            out["normal"] = max(out["normal"], dn * dist / (EPS32 * np.linalg.norm(q0)))
        else:
            out["normal"] = max(out["normal"], dn / (4 * EPS32))
    return out
