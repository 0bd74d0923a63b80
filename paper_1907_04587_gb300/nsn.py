"""ctypes binding of libnsn (include/nsn.h): argument marshalling only.

Every step of the solver runs in the CUDA kernels of libnsn.so; this module
only converts numpy arrays / torch device pointers to the C ABI.  There is no
fallback: if the library is missing or cannot be loaded the import of
``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnsn.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "nsn.h")

NSN_OK = 0
NSN_ERR_INVALID_ARG, NSN_ERR_OUT_OF_MEMORY = 1, 2
STATUS = {0: "NSN_OK", 1: "NSN_ERR_INVALID_ARG", 2: "NSN_ERR_OUT_OF_MEMORY", 3: "NSN_ERR_CUDA",
          4: "NSN_ERR_NOT_CONVERGED", 5: "NSN_ERR_TIMEOUT", 6: "NSN_ERR_BAD_STATE", 7: "NSN_ERR_NONFINITE"}
NSN_RIGID, NSN_PARTICLE = 0, 1
NSN_CONTACT, NSN_REVOLUTE, NSN_TET_NH, NSN_PRISMATIC, NSN_TET_LINEAR = 0, 1, 2, 3, 4
NSN_FP32, NSN_FP64 = 0, 1
NSN_WARM_ZERO, NSN_WARM_PREV, NSN_WARM_LEARNED = 0, 1, 2
NSN_WARM_FRICTION = 0x100
NSN_WARM_PRECOND = 0x200
NSN_MLP_NPARAM = 128 * 16 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 4 * 128 + 4

CONTACT_DTYPE = np.dtype([("body_a", "<i4"), ("body_b", "<i4"), ("pa", "<f4", 3), ("pb", "<f4", 3),
                          ("n", "<f4", 3), ("d", "<f4"), ("mu", "<f4")])
REVOLUTE_DTYPE = np.dtype([("body_a", "<i4"), ("body_b", "<i4"), ("pa", "<f4", 3), ("pb", "<f4", 3),
                           ("axis_a", "<f4", 3), ("axis_b", "<f4", 3), ("compliance", "<f4")])
TET_DTYPE = np.dtype([("v", "<i4", 4), ("rest", "<f4", (4, 3)), ("E", "<f4"), ("nu", "<f4")])


class nsn_config(C.Structure):
    _fields_ = [("h", C.c_double), ("gravity", C.c_double * 3), ("newton_iters", C.c_int32),
                ("cr_iters", C.c_int32), ("damping", C.c_double), ("eps", C.c_double),
                ("tol_rel", C.c_double), ("cr_tol_mode", C.c_int32), ("ncp", C.c_int32),
                ("rscale", C.c_int32), ("geom_stiffness", C.c_int32), ("precision", C.c_int32),
                ("use_graph", C.c_int32), ("cone_project", C.c_int32), ("island_stop", C.c_int32),
                ("cr_resident", C.c_int32), ("res_max_rows", C.c_int32), ("line_search", C.c_int32),
                ("best_iterate", C.c_int32)]


class nsn_stats(C.Structure):
    _fields_ = [("newton_done", C.c_int32), ("cr_total", C.c_int32), ("merit0", C.c_double),
                ("merit_final", C.c_double), ("ms", C.c_float)]


class NSNError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_vp = C.c_void_p


def exported_names():
    """Function names declared in include/nsn.h."""
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:nsn_status|void|const char \*)\s*(nsn_\w+)\s*\(", src, re.M)))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libnsn.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    sig = {
        "nsn_default_config": (None, [C.POINTER(nsn_config)]),
        "nsn_create": (C.c_int, [C.POINTER(nsn_config), _vp, C.POINTER(_vp)]),
        "nsn_destroy": (C.c_int, [_vp]),
        "nsn_last_error": (C.c_char_p, [_vp]),
        "nsn_add_bodies": (C.c_int, [_vp, C.c_int32, _ip, _fp, _fp, _fp, _fp, _fp, _fp, _ip]),
        "nsn_add_constraints": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp, _ip]),
        "nsn_clear_contacts": (C.c_int, [_vp]),
        "nsn_counts": (C.c_int, [_vp, _ip, _ip]),
        "nsn_step": (C.c_int, [_vp, C.c_int32, C.POINTER(nsn_stats)]),
        "nsn_get_state": (C.c_int, [_vp, _fp, _fp, _fp, _fp]),
        "nsn_set_state": (C.c_int, [_vp, _fp, _fp, _fp, _fp]),
        "nsn_set_state_device": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "nsn_get_state_device": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "nsn_get_lambda": (C.c_int, [_vp, _dp]),
        "nsn_get_state_f64": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
        "nsn_get_merit_history": (C.c_int, [_vp, _dp, C.c_int32, _ip]),
        "nsn_linearize": (C.c_int, [_vp, C.c_int32]),
        "nsn_apply_operator": (C.c_int, [_vp, _dp, _dp]),
        "nsn_solve": (C.c_int, [_vp, C.c_int32, _dp, _dp]),
        "nsn_get_system": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
        "nsn_last_launch_count": (C.c_int, [_vp, _ip]),
        "nsn_time_operator": (C.c_int, [_vp, C.c_int32, _fp, _fp]),
        "nsn_operator_sizes": (C.c_int, [_vp, C.POINTER(C.c_int64)]),
        "nsn_apply_operator_noalloc": (C.c_int, [_vp, _vp, _vp, _vp]),
        "nsn_set_warm_start": (C.c_int, [_vp, C.c_int32]),
        "nsn_get_warm_stats": (C.c_int, [_vp, _dp, _dp, _ip]),
        "nsn_mlp_set_params": (C.c_int, [_vp, _fp, C.c_int32]),
        "nsn_mlp_get_params": (C.c_int, [_vp, _fp, _fp, C.c_int32]),
        "nsn_mlp_forward": (C.c_int, [_vp, _vp, C.c_int32, _vp]),
        "nsn_mlp_time_forward": (C.c_int, [_vp, _vp, C.c_int32, _vp, C.c_int32, C.POINTER(C.c_float)]),
        "nsn_mlp_train_step": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int32, C.c_float, C.POINTER(C.c_float)]),
        "nsn_contact_features": (C.c_int, [_vp, _vp, _vp]),
        "nsn_islands": (C.c_int, [_vp, _ip, _ip]),
        "nsn_island_stats": (C.c_int, [_vp, C.c_int32, _dp, _dp, _ip]),
        "nsn_island_stop_device": (C.c_int, [_vp, C.POINTER(_vp)]),
        "nsn_island_stop_copy": (C.c_int, [_vp, _vp]),
        "nsn_clear_warm_start": (C.c_int, [_vp]),
        "nsn_record_decisions": (C.c_int, [_vp, C.c_int32]),
        "nsn_get_prev_lambda": (C.c_int, [_vp, _dp]),
        "nsn_get_phase_times": (C.c_int, [_vp, _dp]),
        "nsn_best_restored": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
        "nsn_get_decisions": (C.c_int, [_vp, _vp, _vp, _vp]),
        "nsn_tuning": (C.c_int, [_vp, _ip, _fp]),
        "nsn_resident_info": (C.c_int, [_vp, _ip]),
        "nsn_time_resident": (C.c_int, [_vp, C.c_int32, _fp, _dp]),
        "nsn_set_body_lanes": (C.c_int, [_vp, C.c_int32]),
        "nsn_collider_create": (C.c_int, [C.c_int32, _ip, _fp, _ip, C.c_int32, _fp, C.c_int32, _fp, C.c_int32,
                                          _ip, C.c_float, C.c_float, _vp, C.POINTER(_vp)]),
        "nsn_collider_destroy": (C.c_int, [_vp]),
        "nsn_collider_run": (C.c_int, [_vp, _fp, _fp, _fp, _fp, C.c_int32, _ip, _fp, _fp, _fp, _fp, _fp, _ip]),
        "nsn_collider_run_async": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp,
                                             _vp]),
        "nsn_collider_info": (C.c_int, [_vp, _ip]),
        "nsn_collider_last_error": (C.c_char_p, [_vp]),
        "nsn_collide_and_step": (C.c_int, [_vp, _vp, C.c_int32, C.POINTER(nsn_stats)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _f32(a, shape):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(shape))


def _p(a, kind=_fp):
    return None if a is None else a.ctypes.data_as(kind)


# ---- functions with the ABI names ------------------------------------------------

def nsn_default_config():
    cfg = nsn_config()
    lib().nsn_default_config(C.byref(cfg))
    return cfg


def nsn_create(cfg, stream=None):
    ctx = _vp()
    st = lib().nsn_create(C.byref(cfg), stream, C.byref(ctx))
    if st != NSN_OK:
        raise NSNError(st, "nsn_create failed")
    return ctx


def nsn_destroy(ctx):
    return lib().nsn_destroy(ctx)


def nsn_last_error(ctx):
    m = lib().nsn_last_error(ctx)
    return m.decode() if m else ""


def _check(ctx, st, what):
    if st != NSN_OK:
        raise NSNError(st, f"{what}: {nsn_last_error(ctx)}")


def nsn_add_bodies(ctx, kind, pos, quat, vel, omega, mass, inertia):
    n = len(mass)
    first = C.c_int32()
    k = np.ascontiguousarray(np.asarray(kind, np.int32))
    arrs = [_f32(pos, (n, 3)), _f32(quat, (n, 4)), _f32(vel, (n, 3)), _f32(omega, (n, 3)), _f32(mass, (n,)),
            _f32(inertia, (n, 3))]
    _check(ctx, lib().nsn_add_bodies(ctx, n, _p(k, _ip), *[_p(a) for a in arrs], C.byref(first)), "nsn_add_bodies")
    return first.value


def nsn_add_constraints(ctx, ctype, records):
    rec = np.ascontiguousarray(records)
    first = C.c_int32()
    _check(ctx, lib().nsn_add_constraints(ctx, ctype, len(rec), rec.ctypes.data_as(_vp), C.byref(first)),
           "nsn_add_constraints")
    return first.value


def nsn_clear_contacts(ctx):
    _check(ctx, lib().nsn_clear_contacts(ctx), "nsn_clear_contacts")


def nsn_counts(ctx):
    nb, nr = C.c_int32(), C.c_int32()
    _check(ctx, lib().nsn_counts(ctx, C.byref(nb), C.byref(nr)), "nsn_counts")
    return nb.value, nr.value


def nsn_step(ctx, nsteps=1):
    st = nsn_stats()
    _check(ctx, lib().nsn_step(ctx, nsteps, C.byref(st)), "nsn_step")
    return dict(newton_done=st.newton_done, cr_total=st.cr_total, merit0=st.merit0, merit_final=st.merit_final,
                ms=st.ms)


def nsn_get_state(ctx, nb):
    out = dict(pos=np.zeros((nb, 3), np.float32), quat=np.zeros((nb, 4), np.float32),
               vel=np.zeros((nb, 3), np.float32), omega=np.zeros((nb, 3), np.float32))
    _check(ctx, lib().nsn_get_state(ctx, *[_p(out[k]) for k in ("pos", "quat", "vel", "omega")]), "nsn_get_state")
    return out


def nsn_get_state_f64(ctx, nb):
    out = dict(pos=np.zeros((nb, 3)), quat=np.zeros((nb, 4)), vel=np.zeros((nb, 3)), omega=np.zeros((nb, 3)))
    _check(ctx, lib().nsn_get_state_f64(ctx, *[_p(out[k], _dp) for k in ("pos", "quat", "vel", "omega")]),
           "nsn_get_state_f64")
    return out


def nsn_set_state(ctx, nb, pos=None, quat=None, vel=None, omega=None):
    a = [_f32(pos, (nb, 3)), _f32(quat, (nb, 4)), _f32(vel, (nb, 3)), _f32(omega, (nb, 3))]
    _check(ctx, lib().nsn_set_state(ctx, *[_p(x) for x in a]), "nsn_set_state")


def nsn_set_state_device(ctx, pos=0, quat=0, vel=0, omega=0):
    """Device pointers (ints, e.g. torch tensor data_ptr(), float32 AoS); 0 = keep."""
    args = [_vp(x) if x else None for x in (pos, quat, vel, omega)]
    _check(ctx, lib().nsn_set_state_device(ctx, *args), "nsn_set_state_device")


def nsn_get_state_device(ctx, pos=0, quat=0, vel=0, omega=0):
    args = [_vp(x) if x else None for x in (pos, quat, vel, omega)]
    _check(ctx, lib().nsn_get_state_device(ctx, *args), "nsn_get_state_device")


def nsn_get_lambda(ctx, R):
    out = np.zeros(R)
    if R:
        _check(ctx, lib().nsn_get_lambda(ctx, _p(out, _dp)), "nsn_get_lambda")
    return out


def nsn_get_merit_history(ctx, cap=1025):
    out = np.zeros(cap)
    n = C.c_int32()
    _check(ctx, lib().nsn_get_merit_history(ctx, _p(out, _dp), cap, C.byref(n)), "nsn_get_merit_history")
    return out[:min(n.value, cap)]


def nsn_linearize(ctx, n_before=0):
    _check(ctx, lib().nsn_linearize(ctx, n_before), "nsn_linearize")


def nsn_apply_operator(ctx, x):
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    y = np.zeros_like(x)
    _check(ctx, lib().nsn_apply_operator(ctx, _p(x, _dp), _p(y, _dp)), "nsn_apply_operator")
    return y


def nsn_solve(ctx, iters, R, D):
    dl = np.zeros(R)
    du = np.zeros(D)
    _check(ctx, lib().nsn_solve(ctx, iters, _p(dl, _dp), _p(du, _dp)), "nsn_solve")
    return dl, du


def nsn_get_system(ctx, R, D):
    b, diag, hv, g = np.zeros(R), np.zeros(R), np.zeros(R), np.zeros(D)
    _check(ctx, lib().nsn_get_system(ctx, _p(b, _dp), _p(diag, _dp), _p(hv, _dp), _p(g, _dp)), "nsn_get_system")
    return dict(b=b, diag=diag, hvec=hv, g=g)


def nsn_last_launch_count(ctx):
    n = C.c_int32()
    _check(ctx, lib().nsn_last_launch_count(ctx, C.byref(n)), "nsn_last_launch_count")
    return n.value


def nsn_time_operator(ctx, iters=20):
    a, b = C.c_float(), C.c_float()
    _check(ctx, lib().nsn_time_operator(ctx, iters, C.byref(a), C.byref(b)), "nsn_time_operator")
    return a.value, b.value


def nsn_apply_operator_noalloc(ctx, x_dev, y_dev, stream=None):
    """y = A x on the kept system with caller-owned float32 device buffers
    (integer device addresses) and no device allocation."""
    _check(ctx, lib().nsn_apply_operator_noalloc(ctx, _vp(x_dev), _vp(y_dev), stream), "nsn_apply_operator_noalloc")


def nsn_set_warm_start(ctx, mode):
    _check(ctx, lib().nsn_set_warm_start(ctx, mode), "nsn_set_warm_start")


def nsn_islands(ctx, nb):
    n = C.c_int32()
    bi = np.zeros(max(nb, 1), np.int32)
    _check(ctx, lib().nsn_islands(ctx, C.byref(n), _p(bi, _ip)), "nsn_islands")
    return n.value, bi[:nb]


def nsn_island_stats(ctx, ni):
    m0, mf, it = np.zeros(max(ni, 1)), np.zeros(max(ni, 1)), np.zeros(max(ni, 1), np.int32)
    _check(ctx, lib().nsn_island_stats(ctx, max(ni, 1), _p(m0, _dp), _p(mf, _dp), _p(it, _ip)), "nsn_island_stats")
    return dict(merit0=m0[:ni], merit_final=mf[:ni], stopped_at=it[:ni])


def nsn_island_stop_device(ctx):
    ptr = _vp()
    _check(ctx, lib().nsn_island_stop_device(ctx, C.byref(ptr)), "nsn_island_stop_device")
    return ptr.value


def nsn_get_warm_stats(ctx):
    mz, mw, rj = C.c_double(), C.c_double(), C.c_int32()
    _check(ctx, lib().nsn_get_warm_stats(ctx, C.byref(mz), C.byref(mw), C.byref(rj)), "nsn_get_warm_stats")
    return dict(merit_zero=mz.value, merit_warm=mw.value, rejected=int(rj.value))


def nsn_mlp_set_params(ctx, params):
    p = np.ascontiguousarray(np.asarray(params, np.float32).ravel())
    _check(ctx, lib().nsn_mlp_set_params(ctx, _p(p), len(p)), "nsn_mlp_set_params")


def nsn_mlp_get_params(ctx):
    p = np.zeros(NSN_MLP_NPARAM, np.float32)
    g = np.zeros(NSN_MLP_NPARAM, np.float32)
    _check(ctx, lib().nsn_mlp_get_params(ctx, _p(p), _p(g), NSN_MLP_NPARAM), "nsn_mlp_get_params")
    return p, g


def nsn_mlp_forward(ctx, X_dev, n, Y_dev):
    _check(ctx, lib().nsn_mlp_forward(ctx, _vp(X_dev), n, _vp(Y_dev)), "nsn_mlp_forward")


def nsn_mlp_time_forward(ctx, X_dev, n, Y_dev, reps):
    ms = C.c_float()
    _check(ctx, lib().nsn_mlp_time_forward(ctx, _vp(X_dev), n, _vp(Y_dev), int(reps), C.byref(ms)),
           "nsn_mlp_time_forward")
    return ms.value


def nsn_mlp_train_step(ctx, X_dev, T_dev, w_dev, n, lr):
    loss = C.c_float()
    _check(ctx, lib().nsn_mlp_train_step(ctx, _vp(X_dev), _vp(T_dev), _vp(w_dev), n, lr, C.byref(loss)),
           "nsn_mlp_train_step")
    return loss.value


def nsn_contact_features(ctx, X_dev, Y_dev=0):
    _check(ctx, lib().nsn_contact_features(ctx, _vp(X_dev) if X_dev else None, _vp(Y_dev) if Y_dev else None),
           "nsn_contact_features")


def nsn_operator_sizes(ctx):
    out = (C.c_int64 * 8)()
    _check(ctx, lib().nsn_operator_sizes(ctx, out), "nsn_operator_sizes")
    keys = ("rigid", "particles", "rows", "pair_rows", "tets", "rigid_entries", "particle_entries", "device_bytes")
    return dict(zip(keys, list(out)))


# ---- scene records -----------------------------------------------------------------

def contact_records(s):
    nc = len(s["c_body"])
    r = np.zeros(nc, CONTACT_DTYPE)
    if nc:
        r["body_a"], r["body_b"] = s["c_body"][:, 0], s["c_body"][:, 1]
        r["pa"], r["pb"], r["n"] = s["c_pa"], s["c_pb"], s["c_n"]
        r["d"], r["mu"] = s["c_d"], s["c_mu"]
    return r


def revolute_records(s):
    nj = len(s["j_body"])
    r = np.zeros(nj, REVOLUTE_DTYPE)
    if nj:
        r["body_a"], r["body_b"] = s["j_body"][:, 0], s["j_body"][:, 1]
        r["pa"], r["pb"], r["axis_a"], r["axis_b"] = s["j_pa"], s["j_pb"], s["j_axa"], s["j_axb"]
        r["compliance"] = s["j_compliance"]
    return r


def tet_records(s, pre="t"):
    nt = len(s.get(f"{pre}_v", ()))
    r = np.zeros(nt, TET_DTYPE)
    if nt:
        r["v"], r["rest"], r["E"], r["nu"] = s[f"{pre}_v"], s[f"{pre}_rest"], s[f"{pre}_E"], s[f"{pre}_nu"]
    return r


def joint_runs(s):
    """The scene's joints as runs of equal kind in scene order: [(type, records)]
    (added run by run, the ABI joint order is the scene's)."""
    rec = revolute_records(s)
    nj = len(rec)
    kind = np.asarray(s.get("j_kind", np.zeros(nj, np.int32)), np.int32).reshape(-1)
    runs, i = [], 0
    while i < nj:
        j = i
        while j < nj and kind[j] == kind[i]:
            j += 1
        runs.append((NSN_PRISMATIC if kind[i] == 1 else NSN_REVOLUTE, rec[i:j]))
        i = j
    return runs


DEFAULTS = dict(h=1.0 / 60.0, gravity=(0.0, 0.0, -9.81), newton_iters=4, cr_iters=20, damping=0.75, eps=1e-6,
                tol_rel=0.0, cr_tol_mode=0, ncp=0, rscale=2, geom_stiffness=1, precision=NSN_FP32, use_graph=1,
                cone_project=0, island_stop=0, cr_resident=1, res_max_rows=384,
                line_search=0, best_iterate=0)


def make_config(**params):
    p = dict(DEFAULTS)
    unknown = set(params) - set(p)
    if unknown:
        raise TypeError(f"unknown parameters {sorted(unknown)}")
    p.update(params)
    cfg = nsn_config()
    cfg.h = p["h"]
    cfg.gravity = (C.c_double * 3)(*p["gravity"])
    for k in ("newton_iters", "cr_iters", "cr_tol_mode", "ncp", "rscale", "geom_stiffness", "precision", "use_graph",
              "cone_project", "island_stop", "cr_resident", "res_max_rows", "line_search", "best_iterate"):
        setattr(cfg, k, int(p[k]))
    for k in ("damping", "eps", "tol_rel"):
        setattr(cfg, k, float(p[k]))
    return cfg


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


class Solver:
    """One libnsn context built from a scene dictionary (``scenes.py``)."""

    def __init__(self, scene, stream=None, **params):
        self.cfg = make_config(**params)
        self.ctx = nsn_create(self.cfg, stream if stream is not None else _current_stream())
        s = scene
        nb = len(s["mass"])
        self.nb = nb
        nsn_add_bodies(self.ctx, s["kind"], s["pos"], s["quat"], s["vel"], s["omega"], s["mass"], s["inertia"])
        for ctype, rec in ([(NSN_CONTACT, contact_records(s))] + joint_runs(s) +
                           [(NSN_TET_NH, tet_records(s)), (NSN_TET_LINEAR, tet_records(s, "l"))]):
            if len(rec):
                nsn_add_constraints(self.ctx, ctype, rec)
        _, self.R = nsn_counts(self.ctx)
        self.D = int(sum(6 if k == 0 else 3 for k in s["kind"]))

    def close(self):
        if getattr(self, "ctx", None):
            nsn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1):
        return nsn_step(self.ctx, nsteps)

    def collide_and_step(self, collider, nsteps=1):
        """nsteps steps, each after contact generation on the current state
        (nsn_collide_and_step; `collider` a Collider over the same bodies)."""
        st = nsn_stats()
        _check(self.ctx, lib().nsn_collide_and_step(self.ctx, collider.ptr, int(nsteps), C.byref(st)),
               "nsn_collide_and_step")
        _, self.R = nsn_counts(self.ctx)
        return dict(newton_done=st.newton_done, cr_total=st.cr_total, merit0=st.merit0,
                    merit_final=st.merit_final, ms=st.ms)

    def get_state(self):
        return nsn_get_state(self.ctx, self.nb)

    def get_state_f64(self):
        return nsn_get_state_f64(self.ctx, self.nb)

    def set_state(self, pos=None, quat=None, vel=None, omega=None):
        nsn_set_state(self.ctx, self.nb, pos, quat, vel, omega)

    def set_contacts(self, scene):
        nsn_clear_contacts(self.ctx)
        rec = contact_records(scene)
        if len(rec):
            nsn_add_constraints(self.ctx, NSN_CONTACT, rec)
        _, self.R = nsn_counts(self.ctx)

    def get_lambda(self):
        return nsn_get_lambda(self.ctx, self.R)

    def get_prev_lambda(self):
        """Multipliers the next warm start reads (carried over contact changes by key)."""
        out = np.zeros(self.R)
        _check(self.ctx, lib().nsn_get_prev_lambda(self.ctx, out.ctypes.data_as(_dp)), "nsn_get_prev_lambda")
        return out

    PHASES = ("collide", "save", "layout", "upload", "restore", "capture", "step")

    def best_restored(self):
        """Islands of the last step that returned an earlier, lower-merit iterate (best_iterate)."""
        n = C.c_int32()
        _check(self.ctx, lib().nsn_best_restored(self.ctx, C.byref(n)), "nsn_best_restored")
        return int(n.value)

    def phase_times(self):
        """Host milliseconds of the phases of the last rebuild and step (nsn_get_phase_times)."""
        out = np.zeros(len(self.PHASES))
        _check(self.ctx, lib().nsn_get_phase_times(self.ctx, out.ctypes.data_as(_dp)), "nsn_get_phase_times")
        return dict(zip(self.PHASES, out.tolist()))

    def merit_history(self):
        return nsn_get_merit_history(self.ctx)

    def linearize(self, n_before=0):
        nsn_linearize(self.ctx, n_before)

    def apply(self, x):
        return nsn_apply_operator(self.ctx, x)

    def solve(self, iters):
        return nsn_solve(self.ctx, iters, self.R, self.D)

    def system(self):
        return nsn_get_system(self.ctx, self.R, self.D)

    def launches_per_step(self):
        return nsn_last_launch_count(self.ctx)

    def set_warm_start(self, mode):
        nsn_set_warm_start(self.ctx, mode)

    def warm_stats(self):
        return nsn_get_warm_stats(self.ctx)

    def tuning(self):
        """(lanes per body in the body pass, measured times of 4 / 8 / 16 lanes in ms)."""
        g = C.c_int32()
        ms = np.zeros(3, np.float32)
        _check(self.ctx, lib().nsn_tuning(self.ctx, C.byref(g), _p(ms)), "nsn_tuning")
        return g.value, ms

    def resident_info(self):
        """Island-resident CR: dict of islands, groups, max_rows, max_entries, smem_bytes, grid."""
        v = np.zeros(6, np.int32)
        _check(self.ctx, lib().nsn_resident_info(self.ctx, _p(v, _ip)), "nsn_resident_info")
        return dict(zip(("islands", "groups", "max_rows", "max_entries", "smem_bytes", "grid"), (int(x) for x in v)))

    def time_resident(self, iters=10):
        """(mean ms of one k_cr_resident launch at full activity, dict of its work)."""
        ms = C.c_float()
        w = np.zeros(4, np.float64)
        _check(self.ctx, lib().nsn_time_resident(self.ctx, iters, C.byref(ms), _p(w, _dp)), "nsn_time_resident")
        return ms.value, dict(zip(("islands", "row_iterations", "entry_iterations", "body_iterations"), w.tolist()))

    def set_body_lanes(self, lanes):
        _check(self.ctx, lib().nsn_set_body_lanes(self.ctx, lanes), "nsn_set_body_lanes")

    def clear_warm_start(self):
        _check(self.ctx, lib().nsn_clear_warm_start(self.ctx), "nsn_clear_warm_start")

    def islands(self):
        """(number of islands, island of each body)."""
        return nsn_islands(self.ctx, self.nb)

    def island_stats(self):
        """Per island of the last step (island_stop = 1): zero-iterate merit,
        final merit, Newton iteration at which it stopped (-1: not stopped)."""
        return nsn_island_stats(self.ctx, self.islands()[0])

    def record_decisions(self, iters):
        """Log the discrete decisions of the first `iters` Newton iterations of
        the following steps (nsn_record_decisions; 0 = off)."""
        _check(self.ctx, lib().nsn_record_decisions(self.ctx, int(iters)), "nsn_record_decisions")
        self._dlog_iters = int(iters)

    def decisions(self):
        """(rows: iters x R uint8 in ABI row order, islands: iters x n_islands
        uint8, cr: iters x n_islands uint16) of the last step (nsn_get_decisions)."""
        ni = self.islands()[0]
        rows = np.zeros((self._dlog_iters, self.R), np.uint8)
        isl = np.zeros((self._dlog_iters, ni), np.uint8)
        cr = np.zeros((self._dlog_iters, ni), np.uint16)
        _check(self.ctx, lib().nsn_get_decisions(self.ctx, rows.ctypes.data, isl.ctypes.data, cr.ctypes.data),
               "nsn_get_decisions")
        return rows, isl, cr

    def time_operator(self, iters=20):
        return nsn_time_operator(self.ctx, iters)

    def sizes(self):
        return nsn_operator_sizes(self.ctx)


# ---- contact generation (Sec. 3.3, Sec. 10) ----------------------------------------

class ColliderError(NSNError):
    pass


def nsn_collider_create(kind, half, env, n_envs, mu_env, planes, exclude, margin, h, stream=None):
    kind = np.ascontiguousarray(np.asarray(kind, np.int32).ravel())
    env = np.ascontiguousarray(np.asarray(env, np.int32).ravel())
    n = len(kind)
    half = _f32(half, (n, 3))
    mu_env = _f32(mu_env, (-1,))
    planes = _f32(planes, (-1, 4)) if planes is not None and len(planes) else np.zeros((0, 4), np.float32)
    exclude = (np.ascontiguousarray(np.asarray(exclude, np.int32).reshape(-1, 2))
               if exclude is not None and len(exclude) else np.zeros((0, 2), np.int32))
    out = _vp()
    st = lib().nsn_collider_create(n, _p(kind, _ip), _p(half), _p(env, _ip), int(n_envs), _p(mu_env), len(planes),
                                   _p(planes), len(exclude), _p(exclude, _ip), float(margin), float(h), stream,
                                   C.byref(out))
    if st != NSN_OK:
        raise ColliderError(st, "nsn_collider_create failed")
    return out


def nsn_collider_destroy(col):
    return lib().nsn_collider_destroy(col)


def nsn_collider_last_error(col):
    m = lib().nsn_collider_last_error(col)
    return m.decode() if m else ""


def nsn_collider_info(col):
    v = np.zeros(4, np.int32)
    st = lib().nsn_collider_info(col, _p(v, _ip))
    if st != NSN_OK:
        raise ColliderError(st, "nsn_collider_info")
    return dict(zip(("bodies", "vertices", "planes", "blocks"), (int(x) for x in v)))


def nsn_collider_run(col, pos, quat, vel, omega, capacity):
    """Host arrays in, contact arrays (a scene's c_* keys) out; grows the
    buffers once if more than ``capacity`` contacts are found."""
    n = len(pos)
    arrs = [_f32(pos, (n, 3)), _f32(quat, (n, 4)), _f32(vel, (n, 3)), _f32(omega, (n, 3))]
    for _ in range(2):
        cap = int(capacity)
        out = dict(c_body=np.zeros((cap, 2), np.int32), c_pa=np.zeros((cap, 3), np.float32),
                   c_pb=np.zeros((cap, 3), np.float32), c_n=np.zeros((cap, 3), np.float32),
                   c_d=np.zeros(cap, np.float32), c_mu=np.zeros(cap, np.float32))
        found = C.c_int32()
        st = lib().nsn_collider_run(col, *[_p(a) for a in arrs], cap, _p(out["c_body"], _ip), _p(out["c_pa"]),
                                    _p(out["c_pb"]), _p(out["c_n"]), _p(out["c_d"]), _p(out["c_mu"]),
                                    C.byref(found))
        if st == NSN_ERR_OUT_OF_MEMORY and found.value > cap:
            capacity = found.value
            continue
        if st != NSN_OK:
            raise ColliderError(st, f"nsn_collider_run: {nsn_collider_last_error(col)}")
        return {k: v[:found.value] for k, v in out.items()}
    raise ColliderError(NSN_ERR_OUT_OF_MEMORY, "nsn_collider_run: contact count changed between calls")


def nsn_collider_run_async(col, pos, quat, vel, omega, capacity, c_body, c_pa, c_pb, c_n, c_d, c_mu, found_dev):
    """Device pointers (ints) in and out, on the collider's stream."""
    st = lib().nsn_collider_run_async(col, pos, quat, vel, omega, int(capacity), c_body, c_pa, c_pb, c_n, c_d, c_mu,
                                      found_dev)
    if st != NSN_OK:
        raise ColliderError(st, f"nsn_collider_run_async: {nsn_collider_last_error(col)}")


class Collider:
    """Contact generation for a scene dictionary with box half extents
    (``half``): body corners and particles against ``planes`` (k x 4: normal,
    offset) and the boxes of their environment; the bodies of every joint are
    excluded from each other.  ``mu_env`` defaults to 0.5 per environment."""

    def __init__(self, scene, planes=((0.0, 0.0, 1.0, 0.0),), margin=0.01, h=1.0 / 60.0, mu_env=None,
                 exclude=None, stream=None):
        s = scene
        n_envs = int(s.get("n_envs", int(np.max(s["env"])) + 1 if len(s["env"]) else 1))
        if exclude is None:
            jb = np.asarray(s.get("j_body", np.zeros((0, 2), np.int32)))
            exclude = jb[(jb[:, 0] >= 0) & (jb[:, 1] >= 0)] if len(jb) else jb
        self.mu_env = np.full(n_envs, 0.5, np.float32) if mu_env is None else np.asarray(mu_env, np.float32)
        self.planes, self.exclude = np.asarray(planes, np.float32).reshape(-1, 4), np.asarray(exclude, np.int32)
        self.margin, self.h, self.n_envs = float(margin), float(h), n_envs
        self.ptr = nsn_collider_create(s["kind"], s["half"], s["env"], n_envs, self.mu_env, self.planes,
                                       self.exclude, margin, h, stream)
        self.capacity = 8 * len(s["kind"]) + 16

    def __del__(self):
        if getattr(self, "ptr", None) is not None and _lib is not None:
            nsn_collider_destroy(self.ptr)
            self.ptr = None

    def info(self):
        return nsn_collider_info(self.ptr)

    def run(self, pos, quat, vel, omega):
        r = nsn_collider_run(self.ptr, pos, quat, vel, omega, self.capacity)
        self.capacity = max(self.capacity, len(r["c_body"]))
        return r

    def run_async(self, pos, quat, vel, omega, out, found_dev):
        """Device pointers: ``out`` maps c_body, c_pa, c_pb, c_n, c_d, c_mu to
        (pointer) with room for ``out['capacity']`` contacts."""
        nsn_collider_run_async(self.ptr, pos, quat, vel, omega, out["capacity"], out["c_body"], out["c_pa"],
                               out["c_pb"], out["c_n"], out["c_d"], out["c_mu"], found_dev)
