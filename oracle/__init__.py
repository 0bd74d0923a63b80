"""FP64 CPU oracle of the non-smooth Newton time stepper (ctypes binding).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, double-precision C
implementation in ``oracle.c`` of Macklin et al. 2019 (Algorithm 1, Sec. 6-9,
App. A-B), with contact generation (Sec. 3.3, Sec. 10) in ``collide.c``.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library in ``paper_1907_04587_gb300``; both consume the same scene
dictionaries produced by ``paper_1907_04587_gb300.scenes``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_COLLIDE = os.path.join(_HERE, "collide.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NCP_FB, NCP_MIN = 0, 1
R_NONE, R_H2, R_EFFMASS = 0, 1, 2
GS_OFF, GS_PARTICLES = 0, 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C99, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(_SRC_COLLIDE), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                               _SRC, _SRC_COLLIDE, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class _Scene(C.Structure):
    _fields_ = [
        ("n_bodies", C.c_int32), ("kind", _ip), ("pos", _dp), ("quat", _dp), ("vel", _dp),
        ("omega", _dp), ("mass", _dp), ("inertia", _dp),
        ("n_contacts", C.c_int32), ("c_body", _ip), ("c_pa", _dp), ("c_pb", _dp), ("c_n", _dp),
        ("c_d", _dp), ("c_mu", _dp),
        ("n_joints", C.c_int32), ("j_body", _ip), ("j_pa", _dp), ("j_pb", _dp), ("j_axa", _dp),
        ("j_axb", _dp), ("j_compliance", _dp), ("j_kind", _ip),
        ("n_tets", C.c_int32), ("t_v", _ip), ("t_rest", _dp), ("t_E", _dp), ("t_nu", _dp),
        ("n_ltets", C.c_int32), ("l_v", _ip), ("l_rest", _dp), ("l_E", _dp), ("l_nu", _dp),
    ]


class _Params(C.Structure):
    _fields_ = [
        ("h", C.c_double), ("gravity", C.c_double * 3), ("newton_iters", C.c_int32),
        ("cr_iters", C.c_int32), ("damping", C.c_double), ("eps", C.c_double),
        ("tol_rel", C.c_double), ("cr_tol_mode", C.c_int32), ("ncp", C.c_int32),
        ("rscale", C.c_int32), ("geom_stiffness", C.c_int32), ("cone_project", C.c_int32),
        ("island_stop", C.c_int32), ("line_search", C.c_int32), ("best_iterate", C.c_int32),
    ]


class _Stats(C.Structure):
    _fields_ = [("newton_done", C.c_int32), ("cr_total", C.c_int32), ("merit0", C.c_double),
                ("merit_first", C.c_double), ("merit_final", C.c_double)]


_fp = C.POINTER(C.c_float)


class _CollideIn(C.Structure):
    _fields_ = [
        ("n_bodies", C.c_int32), ("kind", _ip), ("pos", _fp), ("quat", _fp), ("vel", _fp), ("omega", _fp),
        ("half", _fp), ("env", _ip), ("n_planes", C.c_int32), ("planes", _fp), ("n_exclude", C.c_int32),
        ("exclude", _ip), ("mu_env", _fp), ("margin", C.c_float), ("h", C.c_float),
    ]


class _Contacts(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("c_body", _ip), ("c_pa", _dp), ("c_pb", _dp), ("c_n", _dp),
                ("c_d", _dp), ("c_mu", _dp)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Scene), C.POINTER(_Params)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_num_rows.argtypes = [C.c_void_p]
        L.orc_num_dofs.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, _dp, C.POINTER(_Stats)]
        L.orc_get_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_set_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_get_lambda.argtypes = [C.c_void_p, _dp]
        L.orc_get_merit_history.argtypes = [C.c_void_p, _dp, C.c_int32]
        L.orc_get_merit_history.restype = C.c_int32
        L.orc_linearize.argtypes = [C.c_void_p, C.c_int32, _dp] + [_dp] * 8
        L.orc_apply_A.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_pcr.argtypes = [C.c_void_p, C.c_int32, _dp, _dp]
        L.orc_pcr.restype = C.c_int32
        L.orc_eval_constraints.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_merit_at.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.orc_merit_at.restype = C.c_double
        L.orc_num_islands.argtypes = [C.c_void_p]
        L.orc_num_islands.restype = C.c_int32
        L.orc_get_islands.argtypes = [C.c_void_p, _ip, _ip]
        L.orc_get_island_stats.argtypes = [C.c_void_p, _dp, _dp, _ip]
        L.orc_record_decisions.argtypes = [C.c_void_p, C.c_int32]
        L.orc_record_decisions.restype = C.c_int
        L.orc_get_decisions.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_fb.restype = C.c_double
        L.orc_fb.argtypes = [C.c_double, C.c_double]
        for f in ("orc_fb_contact", "orc_min_contact"):
            getattr(L, f).argtypes = [C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]
        for f in ("orc_w_fb", "orc_w_min"):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [C.c_double] * 4
        L.orc_fb_friction_active.restype = C.c_int
        L.orc_fb_friction_active.argtypes = [C.c_double] * 4
        L.orc_nh_params.argtypes = [C.c_double, C.c_double, _dp, _dp, _dp]
        L.orc_nh_energy.restype = C.c_double
        L.orc_nh_energy.argtypes = [_dp, C.c_double, C.c_double, C.c_double]
        L.orc_nh_grad_hess.argtypes = [_dp, C.c_double, C.c_double, C.c_double, _dp, _dp]
        L.orc_svd3.argtypes = [_dp, _dp, _dp, _dp]
        L.orc_basis.argtypes = [_dp, _dp, _dp]
        for f in ("orc_collide", "orc_collide_f64"):
            getattr(L, f).restype = C.c_int32
            getattr(L, f).argtypes = [C.POINTER(_CollideIn), C.POINTER(_Contacts)]
    return _lib


def _d(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    return a.ctypes.data_as(_ip)


DEFAULT_PARAMS = dict(h=1.0 / 60.0, gravity=(0.0, 0.0, -9.81), newton_iters=4, cr_iters=20,
                      damping=0.75, eps=1e-6, tol_rel=0.0, cr_tol_mode=0, ncp=NCP_FB,
                      rscale=R_EFFMASS, geom_stiffness=GS_PARTICLES, cone_project=0, island_stop=0,
                      line_search=0, best_iterate=0)


class Oracle:
    """One oracle context over a scene dictionary (see ``scenes.py``)."""

    def __init__(self, scene: dict, **params):
        L = lib()
        p = dict(DEFAULT_PARAMS)
        p.update(params)
        self.params = p
        nb = len(scene["mass"])
        self._keep = {}

        def arr(name, dtype, shape):
            if name in scene and scene[name] is not None and np.size(scene[name]):
                a = np.ascontiguousarray(np.asarray(scene[name], dtype=dtype).reshape(shape))
            else:
                a = np.zeros(shape, dtype=dtype)
            self._keep[name] = a
            return a

        nc = int(np.shape(scene.get("c_body", np.zeros((0, 2))))[0])
        nj = int(np.shape(scene.get("j_body", np.zeros((0, 2))))[0])
        nt = int(np.shape(scene.get("t_v", np.zeros((0, 4))))[0])
        nl = int(np.shape(scene.get("l_v", np.zeros((0, 4))))[0])
        s = _Scene()
        s.n_bodies = nb
        s.kind = _ptr(arr("kind", np.int32, (nb,)))
        s.pos = _ptr(arr("pos", np.float64, (nb, 3)))
        s.quat = _ptr(arr("quat", np.float64, (nb, 4)))
        s.vel = _ptr(arr("vel", np.float64, (nb, 3)))
        s.omega = _ptr(arr("omega", np.float64, (nb, 3)))
        s.mass = _ptr(arr("mass", np.float64, (nb,)))
        s.inertia = _ptr(arr("inertia", np.float64, (nb, 3)))
        s.n_contacts = nc
        s.c_body = _ptr(arr("c_body", np.int32, (nc, 2)))
        s.c_pa = _ptr(arr("c_pa", np.float64, (nc, 3)))
        s.c_pb = _ptr(arr("c_pb", np.float64, (nc, 3)))
        s.c_n = _ptr(arr("c_n", np.float64, (nc, 3)))
        s.c_d = _ptr(arr("c_d", np.float64, (nc,)))
        s.c_mu = _ptr(arr("c_mu", np.float64, (nc,)))
        s.n_joints = nj
        s.j_body = _ptr(arr("j_body", np.int32, (nj, 2)))
        s.j_pa = _ptr(arr("j_pa", np.float64, (nj, 3)))
        s.j_pb = _ptr(arr("j_pb", np.float64, (nj, 3)))
        s.j_axa = _ptr(arr("j_axa", np.float64, (nj, 3)))
        s.j_axb = _ptr(arr("j_axb", np.float64, (nj, 3)))
        s.j_compliance = _ptr(arr("j_compliance", np.float64, (nj,)))
        s.j_kind = _ptr(arr("j_kind", np.int32, (nj,)))     # 0 revolute (default), 1 prismatic
        s.n_tets = nt
        s.t_v = _ptr(arr("t_v", np.int32, (nt, 4)))
        s.t_rest = _ptr(arr("t_rest", np.float64, (nt, 4, 3)))
        s.t_E = _ptr(arr("t_E", np.float64, (nt,)))
        s.t_nu = _ptr(arr("t_nu", np.float64, (nt,)))
        s.n_ltets = nl
        s.l_v = _ptr(arr("l_v", np.int32, (nl, 4)))
        s.l_rest = _ptr(arr("l_rest", np.float64, (nl, 4, 3)))
        s.l_E = _ptr(arr("l_E", np.float64, (nl,)))
        s.l_nu = _ptr(arr("l_nu", np.float64, (nl,)))
        pr = _Params()
        pr.h = p["h"]
        pr.gravity = (C.c_double * 3)(*p["gravity"])
        pr.newton_iters = p["newton_iters"]
        pr.cr_iters = p["cr_iters"]
        pr.damping = p["damping"]
        pr.eps = p["eps"]
        pr.tol_rel = p["tol_rel"]
        pr.cr_tol_mode = p["cr_tol_mode"]
        pr.ncp = p["ncp"]
        pr.rscale = p["rscale"]
        pr.geom_stiffness = p["geom_stiffness"]
        pr.cone_project = p["cone_project"]
        pr.island_stop = p["island_stop"]
        pr.line_search = p["line_search"]
        pr.best_iterate = p["best_iterate"]
        self._s, self._p = s, pr
        self.ctx = L.orc_create(C.byref(s), C.byref(pr))
        if not self.ctx:
            raise ValueError("oracle rejected the scene")
        self.nb, self.nc, self.nj, self.nt, self.nl = nb, nc, nj, nt, nl
        self.kind = self._keep["kind"].copy()
        self.R = L.orc_num_rows(self.ctx)
        self.D = L.orc_num_dofs(self.ctx)
        self.last_stats = None

    def __del__(self):
        if getattr(self, "ctx", None):
            lib().orc_destroy(self.ctx)
            self.ctx = None

    def step(self, lambda0=None):
        st = _Stats()
        l0 = None if lambda0 is None else _d(lambda0, (self.R,))
        lib().orc_step(self.ctx, _ptr(l0), C.byref(st))
        self.last_stats = dict(newton_done=st.newton_done, cr_total=st.cr_total, merit0=st.merit0,
                               merit_first=st.merit_first, merit_final=st.merit_final)
        return self.last_stats

    def get_state(self):
        pos = np.zeros((self.nb, 3)); quat = np.zeros((self.nb, 4))
        vel = np.zeros((self.nb, 3)); omega = np.zeros((self.nb, 3))
        lib().orc_get_state(self.ctx, _ptr(pos), _ptr(quat), _ptr(vel), _ptr(omega))
        return dict(pos=pos, quat=quat, vel=vel, omega=omega)

    def set_state(self, pos=None, quat=None, vel=None, omega=None):
        a = [None if x is None else _d(x) for x in (pos, quat, vel, omega)]
        lib().orc_set_state(self.ctx, *[_ptr(x) for x in a])

    def get_lambda(self):
        out = np.zeros(self.R)
        if self.R:
            lib().orc_get_lambda(self.ctx, _ptr(out))
        return out

    def islands(self):
        """(number of islands, island of each body, island of each row)."""
        n = lib().orc_num_islands(self.ctx)
        bi = np.zeros(self.nb, np.int32)
        ri = np.zeros(max(self.R, 1), np.int32)
        lib().orc_get_islands(self.ctx, _ptr(bi), _ptr(ri))
        return n, bi, ri[:self.R]

    def island_stats(self):
        """Per island of the last step: zero-iterate merit, final merit, and the
        Newton iteration at which it stopped (-1: not stopped)."""
        n = lib().orc_num_islands(self.ctx)
        m0, mf, it = np.zeros(n), np.zeros(n), np.zeros(n, np.int32)
        lib().orc_get_island_stats(self.ctx, _ptr(m0), _ptr(mf), _ptr(it))
        return dict(merit0=m0, merit_final=mf, stopped_at=it)

    def record_decisions(self, iters):
        """Keep the discrete decisions of the next steps' first `iters` Newton
        iterations (see oracle.h, orc_record_decisions)."""
        if lib().orc_record_decisions(self.ctx, int(iters)) != 0:
            raise MemoryError("orc_record_decisions")
        self._dlog_iters = int(iters)

    def decisions(self):
        """(rows: iters x R uint8, islands: iters x n_islands uint8, cr: iters x
        n_islands uint16) of the last step."""
        n = lib().orc_num_islands(self.ctx)
        rows = np.zeros((self._dlog_iters, self.R), np.uint8)
        isl = np.zeros((self._dlog_iters, n), np.uint8)
        cr = np.zeros((self._dlog_iters, n), np.uint16)
        lib().orc_get_decisions(self.ctx, rows.ctypes.data_as(C.c_void_p), isl.ctypes.data_as(C.c_void_p),
                                cr.ctypes.data_as(C.c_void_p))
        return rows, isl, cr

    def merit_history(self):
        out = np.zeros(4096)
        n = lib().orc_get_merit_history(self.ctx, _ptr(out), 4096)
        return out[:n]

    def linearize(self, n_before=0, lambda0=None):
        R, D = self.R, self.D
        out = dict(J=np.zeros((R, D)), Hinv=np.zeros((D, D)), C=np.zeros((R, R)), g=np.zeros(D),
                   hvec=np.zeros(R), b=np.zeros(R), u=np.zeros(D), lam=np.zeros(R))
        l0 = None if lambda0 is None else _d(lambda0, (R,))
        lib().orc_linearize(self.ctx, n_before, _ptr(l0), _ptr(out["J"]), _ptr(out["Hinv"]), _ptr(out["C"]),
                            _ptr(out["g"]), _ptr(out["hvec"]), _ptr(out["b"]), _ptr(out["u"]), _ptr(out["lam"]))
        return out

    def apply_A(self, x):
        x = _d(x, (self.R,))
        y = np.zeros(self.R)
        lib().orc_apply_A(self.ctx, _ptr(x), _ptr(y))
        return y

    def dofs(self, vel, omega):
        """Generalised velocity in DOF order ([v, w] per rigid body, v per particle)."""
        vel, omega = np.asarray(vel, np.float64), np.asarray(omega, np.float64)
        return np.concatenate([np.concatenate([vel[i], omega[i]]) if k == 0 else vel[i]
                               for i, k in enumerate(self.kind)]) if len(self.kind) else np.zeros(0)

    def merit_at(self, vel, omega, lam):
        """The merit of Sec. 8.1 at the iterate (u = (vel, omega), lam) of the
        step from the current state: (overall, per island)."""
        u = _d(self.dofs(vel, omega), (self.D,))
        lam = _d(lam, (self.R,))
        isl = np.zeros(max(lib().orc_num_islands(self.ctx), 1))
        m = lib().orc_merit_at(self.ctx, _ptr(u), _ptr(lam), _ptr(isl))
        return m, isl[:lib().orc_num_islands(self.ctx)]

    def eval_constraints(self, with_jacobian=True):
        c = np.zeros(self.R)
        J = np.zeros((self.R, self.D)) if with_jacobian else None
        lib().orc_eval_constraints(self.ctx, _ptr(c), _ptr(J))
        return c, J

    def pcr(self, iters):
        x = np.zeros(self.R)
        hist = np.zeros(iters + 1)
        k = lib().orc_pcr(self.ctx, iters, _ptr(x), _ptr(hist))
        return x, hist[:k + 1]


# ---- scalar helpers for pin tests ------------------------------------------------

def fb(a, b):
    return lib().orc_fb(a, b)


def fb_contact(Cn, lam, r):
    o = [C.c_double() for _ in range(3)]
    lib().orc_fb_contact(Cn, lam, r, *[C.byref(x) for x in o])
    return tuple(x.value for x in o)


def min_contact(Cn, lam, r):
    o = [C.c_double() for _ in range(3)]
    lib().orc_min_contact(Cn, lam, r, *[C.byref(x) for x in o])
    return tuple(x.value for x in o)


def w_fb(vt, lf, mu_ln, r):
    return lib().orc_w_fb(vt, lf, mu_ln, r)


def fb_friction_active(vt, lf, mu_ln, r):
    return bool(lib().orc_fb_friction_active(vt, lf, mu_ln, r))


def w_min(vt, lf, mu_ln, r):
    return lib().orc_w_min(vt, lf, mu_ln, r)


def nh_params(E, nu):
    o = [C.c_double() for _ in range(3)]
    lib().orc_nh_params(E, nu, *[C.byref(x) for x in o])
    return tuple(x.value for x in o)


def nh_energy(s, C1, D1, alpha):
    return lib().orc_nh_energy(_ptr(_d(s, (3,))), C1, D1, alpha)


def nh_grad_hess(s, C1, D1, alpha):
    g = np.zeros(3); H = np.zeros(9)
    lib().orc_nh_grad_hess(_ptr(_d(s, (3,))), C1, D1, alpha, _ptr(g), _ptr(H))
    return g, H.reshape(3, 3)


def svd3(F):
    U = np.zeros(9); s = np.zeros(3); V = np.zeros(9)
    lib().orc_svd3(_ptr(_d(F, (9,))), _ptr(U), _ptr(s), _ptr(V))
    return U.reshape(3, 3), s, V.reshape(3, 3)


def basis(n):
    t1 = np.zeros(3); t2 = np.zeros(3)
    lib().orc_basis(_ptr(_d(n, (3,))), _ptr(t1), _ptr(t2))
    return t1, t2


def collide(kind, pos, quat, vel, omega, half, env, planes, exclude, mu_env, margin, h, fp64_decisions=False):
    """Contact generation of Sec. 3.3 / Sec. 10 (collide.c): candidates of body
    vertices against static planes and the boxes of their environment within
    ``margin``, at the start of the step or at the position predicted with the
    unconstrained velocity (vel, omega), over a step h.  Inputs are rounded to
    FP32 (what the GPU path receives); returns the contact arrays of a scene
    dictionary (c_body, c_pa, c_pb, c_n, c_d, c_mu), geometry in FP64.
    fp64_decisions=False: candidate and face decisions in FP32 in a fixed
    order of rounded operations (orc_collide); True: the plain FP64 definition
    throughout (orc_collide_f64)."""
    f32 = lambda a, c: np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1, c))
    i32 = lambda a: np.ascontiguousarray(np.asarray(a, np.int32).ravel())
    kind, env = i32(kind), i32(env)
    pos, quat, vel, omega, half = f32(pos, 3), f32(quat, 4), f32(vel, 3), f32(omega, 3), f32(half, 3)
    planes = f32(planes, 4) if planes is not None and len(planes) else np.zeros((0, 4), np.float32)
    exclude = (np.ascontiguousarray(np.asarray(exclude, np.int32).reshape(-1, 2))
               if exclude is not None and len(exclude) else np.zeros((0, 2), np.int32))
    mu_env = np.ascontiguousarray(np.asarray(mu_env, np.float32).ravel())
    nb = len(kind)
    assert len(env) == nb and (nb == 0 or (np.all(np.diff(env) >= 0) and env.max() < len(mu_env)))
    fp = lambda a: a.ctypes.data_as(_fp)
    ip = lambda a: a.ctypes.data_as(_ip)
    ci = _CollideIn(nb, ip(kind), fp(pos), fp(quat), fp(vel), fp(omega), fp(half), ip(env), len(planes), fp(planes),
                    len(exclude), ip(exclude), fp(mu_env), float(margin), float(h))
    cap = 0
    while True:
        out = dict(c_body=np.zeros((cap, 2), np.int32), c_pa=np.zeros((cap, 3)), c_pb=np.zeros((cap, 3)),
                   c_n=np.zeros((cap, 3)), c_d=np.zeros(cap), c_mu=np.zeros(cap))
        dp = lambda a: a.ctypes.data_as(_dp)
        co = _Contacts(cap, ip(out["c_body"]), dp(out["c_pa"]), dp(out["c_pb"]), dp(out["c_n"]), dp(out["c_d"]),
                       dp(out["c_mu"]))
        n = (lib().orc_collide_f64 if fp64_decisions else lib().orc_collide)(C.byref(ci), C.byref(co))
        if n < 0:
            raise ValueError("orc_collide: excluded pair out of range")
        if n <= cap:
            return {k: v[:n] for k, v in out.items()}
        cap = n
