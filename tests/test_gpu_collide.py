"""GPU contact generation (Sec. 3.3, Sec. 10) against the oracle's: the same
contacts in the same order -- body pairs, corners and friction bit for bit,
since both sides take every candidate, inside/outside and nearest-face
decision in FP32 with the same rounded operations -- and closest points and
normals (FP64 on both sides, rounded to FP32 on the GPU) within half an FP32
ulp.  Scenes: the cube stack, a random box and particle scene with random
velocities, the chain on the Neo-Hookean block, the bin of 2000 boxes and 8
particle balls against three planes, the batched environments at 64 and at
the full 4096."""
import ctypes
import numpy as np
import pytest

from paper_1907_04587_gb300 import nsn, scenes

pytestmark = pytest.mark.gpu

H = 1.0 / 60.0
Z = ((0.0, 0.0, 1.0, 0.0),)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    yield


def oracle_contacts(orc, s, planes, margin, mu_env, exclude, vel=None, omega=None):
    return orc.collide(s["kind"], s["pos"], s["quat"], s["vel"] if vel is None else vel,
                       s["omega"] if omega is None else omega, s["half"], s["env"], planes, exclude, mu_env,
                       margin, H)


def compare(g, o, scale):
    assert len(g["c_body"]) == len(o["c_body"])
    np.testing.assert_array_equal(g["c_body"], o["c_body"])
    np.testing.assert_array_equal(g["c_pa"], o["c_pa"].astype(np.float32))
    np.testing.assert_array_equal(g["c_mu"], o["c_mu"].astype(np.float32))
    np.testing.assert_array_equal(g["c_d"], 0.0)
    # FP64 on both sides, then one rounding to FP32 (half an ulp, 2^-24
    # relative); FP64 rounding differences of ~1e-16 x the scene's scale
    for k in ("c_pb", "c_n"):
        np.testing.assert_allclose(g[k].astype(np.float64), o[k], rtol=2.0 ** -23, atol=1e-12 * scale)


def random_scene(seed, nb=60, npart=40):
    rng = np.random.default_rng(seed)
    n = nb + npart
    pos = np.c_[rng.uniform(-0.6, 0.6, (n, 2)), rng.uniform(0.0, 0.5, n)]
    q = rng.normal(size=(n, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[nb:] = (1, 0, 0, 0)
    s = dict(kind=np.r_[np.zeros(nb, np.int32), np.ones(npart, np.int32)], pos=pos, quat=q,
             vel=rng.normal(scale=0.5, size=(n, 3)),
             omega=np.r_[rng.normal(scale=2.0, size=(nb, 3)), np.zeros((npart, 3))],
             half=np.r_[rng.uniform(0.03, 0.12, (nb, 3)), np.zeros((npart, 3))], env=np.zeros(n, np.int32))
    return {k: (v.astype(np.float32) if v.dtype.kind == "f" else v) for k, v in s.items()}


def run_both(orc, s, planes=Z, margin=0.01, mu_env=None, exclude=None):
    n_envs = int(s["env"].max()) + 1
    mu = np.linspace(0.3, 1.0, n_envs).astype(np.float32) if mu_env is None else mu_env
    col = nsn.Collider(s, planes=planes, margin=margin, h=H, mu_env=mu, exclude=exclude)
    if exclude is None:
        exclude = col.exclude
    g = col.run(s["pos"], s["quat"], s["vel"], s["omega"])
    o = oracle_contacts(orc, s, planes, margin, mu, exclude)
    return g, o, col


@pytest.mark.parametrize("name", ["cube_stack", "random", "chain_block", "batched64", "mixed_bin"])
def test_contacts_match_oracle(orc, name):
    if name == "cube_stack":
        s, kw = scenes.cube_stack(seed=0), {}
    elif name == "random":
        s, kw = random_scene(7), dict(margin=0.02, planes=((0, 0, 1, 0), (0.6, 0.8, 0.0, -0.3)))
    elif name == "chain_block":
        s, kw = scenes.chain_block(seed=0, hexes=6), dict(margin=0.005)
    elif name == "batched64":
        s, kw = scenes.batched_envs(seed=2, n_envs=64), {}
    else:     # one environment: 2000 boxes, 8 balls of particles, floor and two walls
        s, kw = scenes.mixed_bin(seed=0), dict(planes=((0, 0, 1, 0), (1, 0, 0, 0), (0, 1, 0, 0)))
    g, o, col = run_both(orc, s, **kw)
    print(name, col.info(), "contacts", len(g["c_body"]))
    assert len(g["c_body"]) > 0
    compare(g, o, float(np.abs(s["pos"]).max()) + 1.0)


def test_full_size_batched_matches_oracle(orc):
    """The 4096-environment scene of the benchmark (178k bodies, 1.4M
    vertices): every contact the oracle finds, in its order."""
    s = scenes.batched_envs(seed=0, n_envs=4096)
    g, o, col = run_both(orc, s)
    print(col.info(), "contacts", len(g["c_body"]), "hand-built scene contacts", len(s["c_body"]))
    compare(g, o, float(np.abs(s["pos"]).max()) + 1.0)


def test_device_path_equals_host_path(orc):
    """nsn_collider_run_async on device buffers (torch's stream) writes the
    same contacts and count as the host call."""
    import torch
    s = scenes.batched_envs(seed=4, n_envs=32)
    stream = torch.cuda.current_stream()
    col = nsn.Collider(s, mu_env=np.full(32, 0.7, np.float32), stream=ctypes.c_void_p(stream.cuda_stream))
    ref = col.run(s["pos"], s["quat"], s["vel"], s["omega"])
    d = {k: torch.from_numpy(np.ascontiguousarray(s[k], dtype=np.float32)).cuda() for k in ("pos", "quat", "vel", "omega")}
    cap = len(ref["c_body"]) + 5
    out_t = dict(c_body=torch.full((cap, 2), -7, dtype=torch.int32, device="cuda"),
                 c_pa=torch.zeros((cap, 3), device="cuda"), c_pb=torch.zeros((cap, 3), device="cuda"),
                 c_n=torch.zeros((cap, 3), device="cuda"), c_d=torch.ones(cap, device="cuda"),
                 c_mu=torch.zeros(cap, device="cuda"))
    found = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = {k: v.data_ptr() for k, v in out_t.items()}
    out["capacity"] = cap
    col.run_async(*[d[k].data_ptr() for k in ("pos", "quat", "vel", "omega")], out, found.data_ptr())
    torch.cuda.synchronize()
    n = int(found.item())
    assert n == len(ref["c_body"])
    for k, v in ref.items():
        np.testing.assert_array_equal(out_t[k][:n].cpu().numpy(), v)
    assert torch.all(out_t["c_body"][n:] == -7)


def test_capacity_overflow_and_empty_scenes(orc):
    """Too small a buffer: the first `capacity` contacts, the full count and
    NSN_ERR_OUT_OF_MEMORY; a scene without vertices or without bodies: no
    contacts."""
    s = scenes.cube_stack(seed=1)
    col = nsn.Collider(s)
    full = col.run(s["pos"], s["quat"], s["vel"], s["omega"])
    cap = 3
    buf = dict(c_body=np.zeros((cap, 2), np.int32), c_pa=np.zeros((cap, 3), np.float32),
               c_pb=np.zeros((cap, 3), np.float32), c_n=np.zeros((cap, 3), np.float32),
               c_d=np.zeros(cap, np.float32), c_mu=np.zeros(cap, np.float32))
    found = ctypes.c_int32()
    f = lambda a: np.ascontiguousarray(a, np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    arrs = [np.ascontiguousarray(s[k], np.float32) for k in ("pos", "quat", "vel", "omega")]
    st = nsn.lib().nsn_collider_run(col.ptr, *[f(a) for a in arrs], cap,
                                    buf["c_body"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    *[buf[k].ctypes.data_as(ctypes.POINTER(ctypes.c_float))
                                      for k in ("c_pa", "c_pb", "c_n", "c_d", "c_mu")], ctypes.byref(found))
    assert st == nsn.NSN_ERR_OUT_OF_MEMORY and found.value == len(full["c_body"]) > cap
    for k in buf:
        np.testing.assert_array_equal(buf[k], full[k][:cap])
    shapeless = dict(s, half=np.zeros_like(s["half"]))
    assert len(nsn.Collider(shapeless).run(s["pos"], s["quat"], s["vel"], s["omega"])["c_body"]) == 0
    empty = dict(kind=np.zeros(0, np.int32), half=np.zeros((0, 3), np.float32), env=np.zeros(0, np.int32), n_envs=1)
    z = np.zeros((0, 3), np.float32)
    assert len(nsn.Collider(empty).run(z, np.zeros((0, 4), np.float32), z, z)["c_body"]) == 0


def test_generated_contacts_drive_the_solver(orc):
    """The cube stack with its contacts generated on the GPU: the FP64 step on
    them equals the oracle's step on the oracle's generated contacts."""
    s = scenes.cube_stack(seed=0)
    g, o, _ = run_both(orc, s, mu_env=np.full(1, 0.5, np.float32))
    sg = scenes.finalize({**s, **{k: v for k, v in g.items()}})
    so = scenes.finalize({**s, **{k: v for k, v in o.items()}})
    prm = dict(newton_iters=8, cr_iters=30)
    gs = nsn.Solver(sg, precision=nsn.NSN_FP64, **prm)
    os_ = orc.Oracle(so, **prm)
    gs.step(); os_.step()
    dv = np.abs(gs.get_state_f64()["vel"] - os_.get_state()["vel"]).max()
    print("contacts", len(g["c_body"]), "velocity difference", dv)
    # the two contact sets agree to FP32 rounding (a few 1e-8 m): the states
    # to far below the step's velocity change g h = 0.16 m/s
    assert dv < 1e-6


def test_trajectory_with_contacts_generated_every_step(orc):
    """Sec. 10's loop: collision detection once per step from the start-of-step
    state and the unconstrained velocity (here v + h g and omega), then the
    step.  The GPU runs its collider on its own FP64 state and refills its
    solver's contacts; the oracle does the same with its own collider and
    solver.  Over 10 steps of the cube stack (4 Newton x 20 CR) the contact
    sets stay identical and the states agree to FP64 rounding (each step
    starting from the FP32-rounded state, as the GPU context's rebuild does)."""
    s = scenes.cube_stack(seed=2)
    prm = dict(newton_iters=4, cr_iters=20)
    grav = np.array([0.0, 0.0, -9.81])
    col = nsn.Collider(s, mu_env=np.full(1, 0.5, np.float32))
    g = None
    st_g = st_o = {k: s[k].astype(np.float64) for k in ("pos", "quat", "vel", "omega")}
    worst = 0.0
    for step in range(10):
        f32 = {k: v.astype(np.float32) for k, v in st_g.items()}
        cg = col.run(f32["pos"], f32["quat"], (st_g["vel"] + H * grav).astype(np.float32), f32["omega"])
        o32 = {k: v.astype(np.float32) for k, v in st_o.items()}
        co = orc.collide(s["kind"], o32["pos"], o32["quat"], (st_o["vel"] + H * grav).astype(np.float32),
                         o32["omega"], s["half"], s["env"], Z, None, [0.5], 0.01, H)
        np.testing.assert_array_equal(cg["c_body"], co["c_body"])
        sg = scenes.finalize({**s, **cg})
        if g is None:
            g = nsn.Solver(sg, precision=nsn.NSN_FP64, **prm)
        else:
            g.set_contacts(sg)
        o = orc.Oracle(scenes.finalize({**s, **co}), **prm)
        # refilling the contacts rebuilds the GPU context from its state in
        # FP32 (the ABI's state arrays): the oracle starts from the same values
        o.set_state(**{k: v.astype(np.float32).astype(np.float64) for k, v in st_o.items()})
        g.step(); o.step()
        st_g, st_o = g.get_state_f64(), o.get_state()
        dv = np.abs(st_g["vel"] - st_o["vel"]).max()
        worst = max(worst, dv)
        print(f"step {step}: {len(cg['c_body'])} contacts, velocity difference {dv:.2e}")
    assert worst < 1e-9


@pytest.mark.parametrize("name", ["random", "batched4096"])
def test_contacts_within_rounding_of_the_fp64_definition(orc, name):
    """The GPU's contacts against the oracle's plain FP64 definition of
    contact generation (orc_collide_f64): lists differ only on vertex-shape
    pairs whose distance is within 4 FP32 units of the coordinates' scale of
    the margin, normals change face only on nearest-face ties within that
    band, and other normals differ only by the rotation's rounding."""
    import collide_band
    if name == "random":
        s, planes, margin = random_scene(7), ((0, 0, 1, 0), (0.6, 0.8, 0.0, -0.3)), 0.02
    else:
        s, planes, margin = scenes.batched_envs(seed=0, n_envs=4096), Z, 0.01
    n_envs = int(s["env"].max()) + 1
    mu = np.full(n_envs, 0.5, np.float32)
    col = nsn.Collider(s, planes=planes, margin=margin, h=H, mu_env=mu)
    g = col.run(s["pos"], s["quat"], s["vel"], s["omega"])
    o = orc.collide(s["kind"], s["pos"], s["quat"], s["vel"], s["omega"], s["half"], s["env"], planes, col.exclude,
                    mu, margin, H, fp64_decisions=True)
    r = collide_band.compare(s, g, o, [list(p) for p in planes], margin, H)
    print(name, r)
    assert r["membership"] <= 4 and r["face"] <= 4 and r["normal"] <= 8, r
    assert r["n_common"] >= 0.999 * max(len(g["c_body"]), len(o["c_body"])), r
