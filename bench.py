#!/usr/bin/env python3
"""Benchmark of the non-smooth Newton time stepper on one GB300 (per rank).

Workload (default): 4096 independent RL-style environments, each a revolute
chain of 3-20 links lying on a plane plus 0-64 cubes piled in up to four
layers, per-environment friction in [0.3, 1.0] (``scenes.batched_envs``).

A step is one time step of Algorithm 1 solved to a relative residual of 1e-6:
islands (connected components of bodies through constraints) are solved side
by side, each stops when its merit reaches 1e-6 of its own zero-iterate merit
(cap: 30 Newton iterations of at most 600 CR iterations each), and an environment-step
counts only if every island of the environment reached the tolerance.  The
trajectory advances from the seeded start state (no reset between steps).
  value     converged env-steps/s, state resident in HBM (device-timed), of
            the batched form with the previous step's multipliers as the start
            (per island, kept if not worse than zero), Newton steps with the
            back-tracking line search of Sec. 8.1 (trials t = 1 .. 1/16, else
            the damped 0.75; --line-search 0: the damped step), projected onto
            the friction cone (option cone_project), the least-merit iterate
            of an island that does not reach the tolerance (best_iterate);
            CR per island in shared memory where it fits; contacts generated
            on the GPU at the start of every step (--contacts fixed: the
            scene's contacts throughout)
  arms      the same measurement for: the learned start (per-contact BF16
            network, previous-step start as fallback; with and without its
            preconditioner scale), the headline in the FP64 build, the
            headline with the damped step, the plain batched method (zero
            start; damped and with the line search), the printed update, the
            previous-step start with the damped step, the first step after an
            environment reset with the zero / learned start, and the ablations
            of Sec. 7 (min-map NCP; r = h^2 and r = 1 instead of the
            effective-mass r), each on the first step after a reset with the
            zero start (compare after_reset_zero): on the advancing trajectory
            the min-map variant diverges, in the FP64 oracle as well
  e2e       converged env-steps/s through the C ABI with host buffers: host->
            device copy of the state, the step, device->host copy of the state
            (the state makes that round trip every step)
  roofline  the dominant kernel of the step: the island-resident CR
            (k_cr_resident), shared-memory bytes per launch from its
            algorithmic count, timed live at full activity; the streamed CR
            operator apply is reported beside it (operator_apply_roofline, HBM)
            and the network forward (network_roofline, tensor)
  cpu_baseline  the FP64 oracle (plain method: zero start) on 16-environment
            samples, one process per host core, same tolerance, caps,
            contact regeneration and accounting

``--impl reference`` times the FP64 oracle (the reference arm here) on the
host cores with the same workload definition, metric and unit.
Multi-GPU (torchrun): every rank solves its own 4096 environments (weak
scaling, no data-path collective); rank 0 prints sum(units) / max(time).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1907_04587_gb300 import scenes  # noqa: E402

METRIC = "env-steps/s at 1e-6 relative residual (batched, islands solved side by side); CR-apply HBM GB/s"
UNIT = "env-steps/s"
TOL = 1e-6
WORKLOADS = {
    # CR cap 600: the fastest cap in converged env-steps/s (measured over 100
    # steps at 100, 200, 400, 500, 600, 700, 800 and 1000); chains that do not
    # reach the floor or growth stop run to it
    "batched4096": dict(make=lambda seed: scenes.batched_envs(seed=seed, n_envs=4096), newton=30, cr=600,
                        desc="4096 chain+cube-pile environments (3-20 links, 0-64 cubes, mu 0.3-1.0)"),
    "batched2048": dict(make=lambda seed: scenes.batched_envs(seed=seed, n_envs=2048), newton=30, cr=600,
                        desc="2048 chain+cube-pile environments (profiling size: ~1.2 M rows, working set above L2)"),
    "chain_block": dict(make=lambda seed: scenes.chain_block(seed=seed), newton=30, cr=50,
                        desc="7-link revolute chain on a 24^3-hex stable Neo-Hookean block (69,120 tets)"),
    "cube_stack": dict(make=lambda seed: scenes.cube_stack(seed=seed), newton=30, cr=20,
                       desc="4 unit cubes stacked on a plane (16 contacts)"),
    "mixed_bin": dict(make=lambda seed: scenes.mixed_bin(seed=seed), newton=30, cr=50,
                      desc="2000 rigid boxes + 8 stable Neo-Hookean balls (36,480 tets) in a bin, one environment"),
}
SAMPLE_ENVS = 16      # environments per oracle process of the CPU baseline
WEIGHTS = os.path.join(ROOT, "paper_1907_04587_gb300", "weights", "warm_start_mlp.npy")


def algorithmic_bytes(sz):
    """B_apply per operator apply (FP32), per unit:
    56 per rigid (row, side) entry, 32 per particle entry (J read in both the
    scatter and the gather pass plus the row index), 12 per row (x, w, C_ii),
    24 per tet (off-diagonal C block), 76 per rigid body (inverse mass block
    and z), 36 per particle."""
    return (56 * sz["rigid_entries"] + 32 * sz["particle_entries"] + 12 * sz["rows"] + 24 * sz["tets"]
            + 76 * sz["rigid"] + 36 * sz["particles"])


def design_bytes(sz):
    """Bytes the two-pass design itself must move per apply (J read once):
    36 per rigid entry, 24 per particle entry, 36 per rigid body, 16 per
    particle, 36 per pair row, 168 per tet (3 rows)."""
    return (36 * sz["rigid_entries"] + 24 * sz["particle_entries"] + 36 * sz["rigid"] + 16 * sz["particles"]
            + 36 * sz["pair_rows"] + 168 * sz["tets"])


def weak_scaling_value(units_per_rank, seconds_per_rank):
    """Whole-job throughput: all units processed over the slowest rank's time."""
    return float(sum(units_per_rank)) / float(max(seconds_per_rank))


def measured_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured bf16_tflops (burst)"
    return 1900.0, "fallback"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.fh.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def operator_traffic(kernel_hash, name="operator_apply_batched4096.json", key="dram_bytes_per_apply"):
    """dram bytes per launch from a committed ncu summary, if it was taken on the
    current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_sha256") != kernel_hash:
        return None
    return d.get(key)


# shared-memory and FP32 peaks of the part, from its unit counts and the SM clock:
# 152 SMs x 128 B of shared memory per clock; 152 x 128 FP32 lanes x 2 flop (FMA)
SMEM_BYTES_PER_SM_CLK = 128
FP32_FLOP_PER_SM_CLK = 256


RESIDENT_TRAFFIC_ROWS = 1259819   # rows of the batched2048 scene the resident traffic was captured on


def resident_roofline(g, clk):
    """k_cr_resident timed live at full activity (the first Newton iteration
    of a zero start: every resident island iterates), with its algorithmic
    shared-memory bytes and flops per row-, entry- and body-iteration."""
    info = g.resident_info()
    if info["islands"] == 0:
        return None
    ms, w = g.time_resident(10)
    Ri, Ei, Bi = w["row_iterations"], w["entry_iterations"], w["body_iterations"]
    smem = 76 * Ri + 80 * Ei + 60 * Bi
    flop = 28 * Ri + 24 * Ei + 18 * Bi
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    summ = clk.summary() if clk is not None else None
    mhz = (summ or {}).get("sm_max_mhz") or 2070.0
    smem_peak = nsm * SMEM_BYTES_PER_SM_CLK * mhz * 1e6 / 1e9
    fp32_peak = nsm * FP32_FLOP_PER_SM_CLK * mhz * 1e6 / 1e12
    ach = smem / (ms * 1e-3) / 1e9
    traffic = operator_traffic(kernel_source_hash(), "resident_cr_batched2048.json", "dram_bytes_per_launch")
    if traffic is not None:      # captured at 2048 environments: scaled to this scene by its rows
        traffic *= g.sizes()["rows"] / RESIDENT_TRAFFIC_ROWS
    return {"bound": "smem", "achieved": ach, "peak": smem_peak, "unit": "GB/s", "frac": ach / smem_peak,
            "traffic": traffic,
            "kernel": "k_cr_resident (one thread block per group of islands, all CR iterations of a Newton iteration from shared memory)",
            "ms": ms, "islands": w["islands"], "row_iterations": Ri, "entry_iterations": Ei, "body_iterations": Bi,
            "bytes_smem": smem, "flop": flop, "tflops": flop / (ms * 1e-3) / 1e12, "fp32_peak_tflops": fp32_peak,
            "peak_kind": f"derived: {nsm} SMs x {SMEM_BYTES_PER_SM_CLK} B/clk x {mhz:.0f} MHz",
            "smem_bytes_per_block": info["smem_bytes"], "grid": info["grid"], "max_island_rows": info["max_rows"]}


# FP32 operations counted from the collider's source (every operation is a
# separately rounded instruction): the rotation of a body's quaternion, once
# per rigid body, 30; one vertex-box test -- lever arm 3, velocity at the
# vertex 12, relative prediction 12, two box-frame transforms 30, two squared
# distances 28, two compares 2 -- 87; one vertex-plane test -- two plane
# distances 12, two compares 2 -- 14, plus the prediction, 6 per vertex.
OPS_ROTATION = 30
OPS_BOX_TEST = 87
OPS_PLANE_TEST = 14
OPS_VERTEX = 6


def contact_generation(nsn, torch, s, stream, clk, rank=0, iters=20):
    """Contact generation (Sec. 3.3, Sec. 10) on the workload's bodies with
    the ground plane: the collider's five kernels timed with CUDA events on
    device buffers, and end to end through nsn_collider_run
    (host arrays in and out).  Bound: FP32 ALU (the tests are independent
    arithmetic on L2-resident body data)."""
    if "half" not in s:
        return None
    n_envs = int(s["n_envs"])
    planes = ((0.0, 0.0, 1.0, 0.0),)
    col = nsn.Collider(s, planes=planes, mu_env=np.full(n_envs, 0.5, np.float32), stream=stream.cuda_stream)
    ref = col.run(s["pos"], s["quat"], s["vel"], s["omega"])
    n = len(ref["c_body"])
    dev = torch.device("cuda", torch.cuda.current_device())
    d = {k: torch.from_numpy(np.ascontiguousarray(s[k], dtype=np.float32)).to(dev) for k in ("pos", "quat", "vel", "omega")}
    cap = n + 1024
    out_t = dict(c_body=torch.empty((cap, 2), dtype=torch.int32, device=dev),
                 **{k: torch.empty((cap, 3), device=dev) for k in ("c_pa", "c_pb", "c_n")},
                 **{k: torch.empty(cap, device=dev) for k in ("c_d", "c_mu")})
    out = {k: v.data_ptr() for k, v in out_t.items()}
    out["capacity"] = cap
    found = torch.zeros(1, dtype=torch.int32, device=dev)
    args = [d[k].data_ptr() for k in ("pos", "quat", "vel", "omega")]
    torch.cuda.synchronize()
    for _ in range(3):
        col.run_async(*args, out, found.data_ptr())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(iters):
        col.run_async(*args, out, found.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    assert int(found.item()) == n
    t0 = time.perf_counter()
    for _ in range(3):
        col.run(s["pos"], s["quat"], s["vel"], s["omega"])
    ms_e2e = (time.perf_counter() - t0) * 1e3 / 3
    # tests per vertex: every plane, and the boxes of its environment other
    # than its own body and the bodies it shares a joint with
    kind = s["kind"]
    nvert, box_tests = collide_tests(kind, s["half"], s["env"], col.exclude, n_envs)
    tests_box = float((nvert * box_tests).sum())
    tests_plane = float(nvert.sum() * len(planes))
    # the emit pass repeats the tests of the vertices with contacts
    vid = ref["c_body"][:, 0].astype(np.int64) * 8 + np.dot(ref["c_pa"] > 0, [1, 2, 4])
    hit_body = np.unique(vid) // 8
    hit = np.bincount(hit_body, minlength=len(kind))
    per_vertex = OPS_BOX_TEST * box_tests + OPS_PLANE_TEST * len(planes) + OPS_VERTEX
    ops = OPS_ROTATION * float((kind == 0).sum()) + per_vertex @ nvert + per_vertex @ hit
    orc = oracle_collide_rate(s, planes, col.exclude) if rank == 0 else None
    if orc is not None:
        orc["ms_scaled_to_scene"] = (tests_box + tests_plane) / orc["tests_per_s"] * 1e3
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    summ = clk.summary() if clk is not None else None
    mhz = (summ or {}).get("sm_max_mhz") or 2070.0
    peak = nsm * 128 * mhz * 1e6 / 1e12
    ach = ops / (ms * 1e-3) / 1e12
    info = col.info()
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tops/s", "frac": ach / peak,
            "peak_kind": f"derived: {nsm} SMs x 128 FP32 lanes x {mhz:.0f} MHz, one rounded op per lane per clock",
            "kernel": ("k_col_prep + k_col_count + k_col_scan + k_col_emit (FP32, one thread per vertex over its "
                       "environment's shapes) + k_col_geom (FP64 closest points and normals, one thread per contact); "
                       "achieved = FP32 operations of the tests over the whole call"),
            "ms": ms, "ms_e2e_host_arrays": ms_e2e, "contacts": n, "vertices": info["vertices"],
            "tests": tests_box + tests_plane, "ops_per_box_test": OPS_BOX_TEST,
            "ops_per_plane_test": OPS_PLANE_TEST, "fp32_ops": ops, "tests_per_s": (tests_box + tests_plane) / (ms * 1e-3),
            "hand_built_scene_contacts": int(len(s["c_body"])), "oracle": orc}


def collide_tests(kind, half, env, exclude, n_envs):
    """Per body: its vertex count (8 per box, 1 per particle) and the boxes
    each of its vertices is tested against (the boxes of its environment
    other than itself and its joint partners).  Plane tests are one per
    vertex and plane."""
    box = (kind == 0) & np.all(half > 0, axis=1)
    nvert = np.where(kind == 1, 1, np.where(box, 8, 0))
    nbox_env = np.bincount(env, weights=box, minlength=n_envs)
    excl = np.zeros(len(kind))
    for a, b in np.asarray(exclude).reshape(-1, 2):
        excl[a] += box[b]
        excl[b] += box[a]
    return nvert, nbox_env[env] - box - excl


def oracle_collide_rate(s, planes, exclude, margin=0.01, h=1.0 / 60.0, n_envs_sample=512):
    """The oracle's contact generation (oracle/collide.c, one host core) on the
    first ``n_envs_sample`` environments of the scene: tests per second and
    the time scaled to the whole scene by its share of the tests."""
    import oracle
    env = s["env"]
    nb = int(np.searchsorted(env, n_envs_sample))     # environments are contiguous body ranges
    ex = np.asarray(exclude).reshape(-1, 2)
    ex = ex[(ex[:, 0] < nb) & (ex[:, 1] < nb)]
    kind, half = s["kind"][:nb], s["half"][:nb]
    nvert, box_tests = collide_tests(kind, half, env[:nb], ex, n_envs_sample)
    tests = float((nvert * box_tests).sum() + nvert.sum() * len(planes))
    args = (kind, s["pos"][:nb], s["quat"][:nb], s["vel"][:nb], s["omega"][:nb], half, env[:nb], planes, ex,
            np.full(n_envs_sample, 0.5), margin, h)
    t0 = time.perf_counter()
    r = oracle.collide(*args)
    sec = time.perf_counter() - t0
    return {"kind": "oracle", "cores": 1, "tests_per_s": tests / sec, "ms_sample": sec * 1e3,
            "contacts_sample": int(len(r["c_body"])),
            "sample": f"the first {n_envs_sample} environments ({nb} bodies, {tests:.0f} tests), FP32 decisions "
                      f"and FP64 geometry in plain C; the call counts the contacts, then writes them"}


def kernel_source_hash():
    """sha256 of the kernels' source file: an ncu traffic figure counts only
    if it was taken on these kernels."""
    h = hashlib.sha256()
    h.update(open(os.path.join(ROOT, "paper_1907_04587_gb300", "csrc", "nsn_kernels.cuh"), "rb").read())
    return h.hexdigest()


def island_env_map(s, body_island, n_islands):
    """Environment of each island (that of its lowest body)."""
    nb = len(body_island)
    first = np.full(n_islands, nb, np.int64)
    np.minimum.at(first, body_island, np.arange(nb))
    env = np.asarray(s.get("env", np.zeros(nb, np.int32)))
    return env[first].astype(np.int64)


def count_converged(stops, isl_env, n_envs):
    """stops: (steps, islands) stop iterations (-1: not converged).  Returns
    (converged env-steps, converged island-steps, mean stop iteration)."""
    stops = np.asarray(stops)
    fail = np.zeros((stops.shape[0], n_envs), np.int64)
    for k in range(stops.shape[0]):
        np.add.at(fail[k], isl_env, (stops[k] < 0).astype(np.int64))
    ok = stops >= 0
    return int((fail == 0).sum()), int(ok.sum()), float(stops[ok].mean()) if ok.any() else float("nan")


def _oracle_chunk(job):
    """One host process: the FP64 oracle, as it stands, on its own sample of
    the workload for ``budget_s`` seconds.  With ``regen`` the contacts are
    regenerated at every step by the oracle's collider (candidates from
    v + h g, margin 1 cm, as the GPU step does) and a fresh oracle steps them
    from the current state (zero start).  Returns (converged env-steps,
    steps, seconds, environments)."""
    workload, seed, budget_s, newton, cr, ls, regen = job
    import oracle
    if workload.startswith("batched"):
        s = scenes.batched_envs(seed=seed, n_envs=SAMPLE_ENVS)
    else:
        s = WORKLOADS[workload]["make"](seed)
    n_envs = int(s.get("n_envs", 1))
    prm = dict(newton_iters=newton, cr_iters=cr, tol_rel=TOL, island_stop=1, cone_project=1, line_search=ls,
               best_iterate=1)
    regen = regen and "half" in s and "mu_env" in s
    h = 1.0 / 60.0
    if regen:
        jb = np.asarray(s["j_body"])
        exclude = jb[(jb[:, 0] >= 0) & (jb[:, 1] >= 0)] if len(jb) else jb
        grav = np.float32(h) * np.array([0.0, 0.0, -9.81], np.float32)
    o = oracle.Oracle(s, **prm)
    conv, n, t0 = 0, 0, time.perf_counter()
    while True:
        if regen:
            st = o.get_state()
            co = oracle.collide(s["kind"], st["pos"], st["quat"], st["vel"].astype(np.float32) + grav, st["omega"],
                                s["half"], s["env"], scene_planes(s), exclude, s["mu_env"], 0.01, h)
            o = oracle.Oracle(scenes.finalize({**s, **co}), **prm)
            o.set_state(**st)
        o.step()
        ni, bi, _ = o.islands()
        conv += count_converged([o.island_stats()["stopped_at"]], island_env_map(s, bi, ni), n_envs)[0]
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            return conv, n, el, n_envs


def scene_planes(s):
    """The static planes a scene declares (k x 4: normal, offset), else the ground."""
    return s["planes"] if "planes" in s else ((0.0, 0.0, 1.0, 0.0),)


def oracle_rate(workload, seed, budget_s, newton, cr, cores=None):
    """FP64 oracle converged env-steps/s on a bounded sample of the workload:
    one process per host core (spawned: the GPU context of the caller is not
    inherited), each stepping its own environments of the same distribution
    (seeds seed*1000 + k) for budget_s; the rate is their sum over the
    longest process's time."""
    import multiprocessing as mp
    if cores is None:
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    cores = max(1, min(int(cores), 16))
    if not workload.startswith("batched"):
        cores = 1       # one scene: a sample of one
    jobs = [(workload, seed * 1000 + k if k else seed, budget_s, newton, cr, LS, REGEN) for k in range(cores)]
    probe = WORKLOADS[workload]["make"](seed) if not workload.startswith("batched") else None
    regen_used = bool(REGEN) and (probe is None or ("half" in probe and "mu_env" in probe))
    if cores == 1:
        res = [_oracle_chunk(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_chunk, jobs)
    conv = sum(r[0] for r in res)
    el = max(r[2] for r in res)
    steps = sum(r[1] for r in res)
    if workload.startswith("batched"):
        sample = (f"{cores} x {SAMPLE_ENVS} environments of the same distribution (process k: seed "
                  f"{seed} for k = 0, else 1000 x {seed} + k), one process per host core")
    else:
        sample = "the full scene, one host core"
    return conv / el, dict(kind="oracle", cores=cores,
                           sample=f"{sample}; same tolerance, caps, Newton step ({'line search' if LS else 'damped'}) "
                                  f"and accounting, zero start, contacts "
                                  f"{'regenerated by the oracle collider every step' if regen_used else 'fixed'}; "
                                  f"{steps} advancing steps in {el:.1f} s, {conv} of "
                                  f"{sum(r[1] * r[3] for r in res)} env-steps converged")


def resident_with_apply_equivalent(resident, b_apply, sz, peak, peak_kind):
    """The resident CR's work expressed as the HBM traffic the streamed apply
    would move for it: B_apply per row per CR iteration (the algorithmic
    bytes of one apply over all rows, divided by the rows) times the resident
    row-iterations, over the resident launch time, against the measured HBM
    bandwidth.  The kernel itself runs from shared memory; this says how far
    it is from what any kernel that streams the operator from HBM could do."""
    out = dict(resident)
    per_row = b_apply / max(sz["rows"], 1)
    achieved = per_row * resident["row_iterations"] / (resident["ms"] * 1e-3) / 1e9
    out["apply_equivalent"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": achieved / peak, "bytes_per_row_iteration": per_row,
                               "peak_kind": f"{peak_kind} hbm_gbs (burst)"}
    return out


def heavy_stack_comparison(nsn, stream):
    """The complementarity preconditioners of Sec. 7 on the heavy stack of
    Sec. 10 (five unit cubes, 8 ... 32768 kg), at rest and with the boxes
    sliding at up to 5 m/s: one step to 1e-6 (cap 40 Newton iterations of 40
    CR iterations), Newton iterations taken and the final merit relative to
    the zero-iterate merit, FP32 production build."""
    out = {}
    for vx in (0.0, 5.0):
        s = scenes.heavy_stack()
        s["vel"] = s["vel"].copy()
        s["vel"][:, 0] = np.float32(vx) * np.arange(1, 6, dtype=np.float32) / 5
        row = {}
        for name, rs in (("identity", 0), ("h2", 1), ("effective_mass", 2)):
            g = nsn.Solver(s, stream=stream.cuda_stream, newton_iters=40, cr_iters=40, tol_rel=TOL, rscale=rs)
            st = g.step()
            row[name] = {"newton": int(st["newton_done"]),
                         "merit_ratio": float(st["merit_final"] / max(st["merit0"], 1e-300))}
            g.close()
        out[f"top_speed_{vx:g}_m_per_s"] = row
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    value, cb = oracle_rate(args.workload, 0, args.ref_budget, W["newton"], W["cr"])
    cb["value"] = value
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "description": W["desc"], "newton_cap": W["newton"],
                      "cr_iters": W["cr"], "tol_rel": TOL},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


EAGER = False   # --eager: launch kernel by kernel instead of the CUDA graph (for profilers)
RESIDENT = 1    # --resident 0: every island in the streamed CR loop
CR_TOL = 0      # --cr-tol 1: CR of a Newton iteration also stops at the forcing term min(0.1, m/m0)
REGEN = 1       # --contacts fixed: the scene's contacts for the whole trajectory instead of generating them each step
LS = 1          # --line-search 0: the headline arm takes the damped step of Sec. 8.1 instead


def make_solver(nsn, s, stream, newton, cr, cone, warm=0, params=None, ncp=0, rscale=2, ls=0, fp64=False):
    g = nsn.Solver(s, stream=stream.cuda_stream, newton_iters=newton, cr_iters=cr, tol_rel=TOL, island_stop=1,
                   cone_project=cone, precision=nsn.NSN_FP64 if fp64 else nsn.NSN_FP32, use_graph=0 if EAGER else 1, ncp=ncp, rscale=rscale,
                   cr_resident=RESIDENT, cr_tol_mode=CR_TOL, line_search=ls, best_iterate=1)
    if params is not None:
        nsn.nsn_mlp_set_params(g.ctx, params)
    g.set_warm_start(warm)
    return g


def measure_arm(nsn, torch, g, s, st0, stream, steps, warmup, clk=None, reset=False, collider=None):
    """Device-timed advancing trajectory: reset to the start state, warmup
    steps, then `steps` timed steps; per-step island stop iterations are copied
    on the device and counted afterwards.  reset=True: every step starts from
    the start state with no previous-step multipliers (an environment reset,
    as RL training does at episode starts).  collider: contacts regenerated
    at every step (nsn_collide_and_step: the collider on the current state,
    the layout rebuilt for the new contacts, the previous multipliers carried
    over by key), all inside the timed region; the islands then change from
    step to step, and each step's are counted with that step's stop
    iterations."""
    dev = st0["pos"].device
    ni, bi = g.islands()
    isl_env = island_env_map(s, bi, ni)
    n_envs = int(s.get("n_envs", 1))
    stops = torch.empty((steps, max(ni, 1)), dtype=torch.int32, device=dev)
    ptr = {k: v.data_ptr() for k, v in st0.items()}
    nsn.nsn_set_state_device(g.ctx, ptr["pos"], ptr["quat"], ptr["vel"], ptr["omega"])
    def restart():
        nsn.nsn_set_state_device(g.ctx, ptr["pos"], ptr["quat"], ptr["vel"], ptr["omega"])
        g.clear_warm_start()

    def one_step():
        return g.collide_and_step(collider, 1) if collider is not None else g.step(1)

    for _ in range(warmup):
        if reset:
            restart()
        one_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if clk:
        clk.__enter__()
    newton, launches, contacts, phases = [], 0, [], []
    if collider is not None:
        # islands change with the contacts: the stop iterations of each step go
        # to a buffer of the largest island count a scene of these bodies can
        # have (every body alone), with that step's island -> environment map
        stops = torch.full((steps, len(s["mass"])), -1, dtype=torch.int32, device=dev)
        maps = []
    e0.record(stream)
    for k in range(steps):
        if reset:
            restart()
        st = one_step()
        nsn.lib().nsn_island_stop_copy(g.ctx, nsn.C.c_void_p(stops[k].data_ptr()))
        if collider is not None:
            ni_k, bi_k = g.islands()
            maps.append((ni_k, island_env_map(s, bi_k, ni_k)))
            contacts.append((g.R - 5 * len(s["j_body"]) - 3 * len(s["t_v"]) - 3 * len(s.get("l_v", ()))) // 3)
            phases.append(g.phase_times())
        newton.append(st["newton_done"])
        launches += g.launches_per_step()
    e1.record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__()
    sec = e0.elapsed_time(e1) / 1e3
    if collider is None:
        conv, conv_isl, mean_stop = count_converged(stops[:, :ni].cpu().numpy(), isl_env, n_envs)
        n_isl_steps = steps * ni
    else:
        sa = stops.cpu().numpy()
        conv = conv_isl = 0
        stops_ok = []
        for k, (ni_k, env_k) in enumerate(maps):
            c1, c2, _ = count_converged(sa[k:k + 1, :ni_k], env_k, n_envs)
            conv += c1; conv_isl += c2
            stops_ok.append(sa[k, :ni_k][sa[k, :ni_k] >= 0])
        allok = np.concatenate(stops_ok) if stops_ok else np.zeros(0)
        mean_stop = float(allok.mean()) if len(allok) else float("nan")
        n_isl_steps = sum(m[0] for m in maps)
        ni = int(np.mean([m[0] for m in maps]))
    out = dict(sec=sec, env_steps=conv, env_fraction=conv / (steps * n_envs),
               island_fraction=conv_isl / max(n_isl_steps, 1), mean_newton_to_tol=mean_stop,
               newton_per_step=float(np.mean(newton)), ms_per_step=sec * 1e3 / steps,
               value=conv / sec, islands=ni, kernels=launches)
    if collider is not None:
        out["contacts_per_step"] = float(np.mean(contacts))
        # host wall time per phase of a step with regenerated contacts (mean
        # over the timed steps; the step phase waits for the GPU's work)
        out["host_phases_ms"] = {k: float(np.mean([p[k] for p in phases])) for k in phases[0]} if phases else None
    return out


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1907_04587_gb300 import nsn
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    W = WORKLOADS[args.workload]
    newton = args.newton or W["newton"]
    cr = args.cr or W["cr"]
    s = W["make"](rank)
    n_envs = int(s.get("n_envs", 1))
    stream = torch.cuda.Stream(device=dev)
    st0 = {k: torch.from_numpy(np.ascontiguousarray(s[k], dtype=np.float32)).to(dev)
           for k in ("pos", "quat", "vel", "omega")}
    params = np.load(WEIGHTS) if os.path.exists(WEIGHTS) else None
    warm_names = {"learned": nsn.NSN_WARM_LEARNED, "prev": nsn.NSN_WARM_PREV, "zero": nsn.NSN_WARM_ZERO}
    warm = args.warm
    warm_note = {"learned": "learned (per-contact BF16 network) with the previous-step start as fallback: "
                            "per island the least-merit candidate of network / previous step / zero",
                 "prev": "previous-step multipliers (per island, kept if not worse than zero)",
                 "zero": "zero (Sec. 8.1), the plain method"}[warm]
    if warm == "learned" and params is None:
        warm, warm_note = "prev", "previous-step multipliers (no trained network weights present)"
    with torch.cuda.stream(stream):
        g = make_solver(nsn, s, stream, newton, cr, cone=1, warm=warm_names[warm], params=params, ls=LS)
        # contacts regenerated at every step (Sec. 10) where the scene has
        # collision shapes and per-environment friction (every workload but
        # the cube stack, whose contacts are the paper's figure's)
        collider = None
        if REGEN and "half" in s and "mu_env" in s:
            collider = nsn.Collider(s, planes=scene_planes(s), mu_env=s["mu_env"], stream=stream.cuda_stream)
        dist = None
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        clk = ClockSampler(local_rank)
        main_arm = measure_arm(nsn, torch, g, s, st0, stream, args.steps, args.warmup, clk, collider=collider)
        if warm != "zero":
            main_arm["network_or_warm_rejected_islands_last_step"] = g.warm_stats()["rejected"]
        sec = main_arm["sec"]
        units = main_arm["env_steps"]
        if dist:
            dist.barrier()
        # e2e: host buffers through the C ABI (pinned), copies inside the timed region; the state
        # makes a round trip through the host every step (as in an RL loop) and the trajectory advances
        host_in = {k: torch.from_numpy(np.ascontiguousarray(s[k], dtype=np.float32)).pin_memory()
                   for k in ("pos", "quat", "vel", "omega")}
        host_out = {k: torch.empty_like(v).pin_memory() for k, v in host_in.items()}
        fp = lambda t: nsn.C.cast(t.data_ptr(), nsn._fp)  # noqa: E731
        L = nsn.lib()
        h2d = sum(v.numel() * 4 for v in host_in.values())
        d2h = sum(v.numel() * 4 for v in host_out.values())
        ni, bi = g.islands()
        isl_env = island_env_map(s, bi, ni)
        stops = torch.empty((args.steps, max(ni, 1)), dtype=torch.int32, device=dev)
        keys = ("pos", "quat", "vel", "omega")

        if collider is not None:
            stops = torch.full((args.steps, len(s["mass"])), -1, dtype=torch.int32, device=dev)
            e2e_maps = []

        def e2e_step(k):
            L.nsn_set_state(g.ctx, *[fp(host_in[k2]) for k2 in keys])
            if collider is not None:
                g.collide_and_step(collider, 1)
                e2e_maps.append(g.islands())
            else:
                g.step(1)
            L.nsn_island_stop_copy(g.ctx, nsn.C.c_void_p(stops[k].data_ptr()))
            L.nsn_get_state(g.ctx, *[fp(host_out[k2]) for k2 in keys])
            for k2 in keys:
                host_in[k2].copy_(host_out[k2])

        g.clear_warm_start()
        for _ in range(max(args.warmup, 1)):
            e2e_step(0)
        if collider is not None:
            e2e_maps.clear()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            e2e_step(k)
        torch.cuda.synchronize()
        sec_e2e = time.perf_counter() - t0
        if collider is None:
            units_e2e, _, _ = count_converged(stops[:, :ni].cpu().numpy(), isl_env, n_envs)
        else:
            sa = stops.cpu().numpy()
            units_e2e = sum(count_converged(sa[k:k + 1, :m[0]], island_env_map(s, m[1], m[0]), n_envs)[0]
                            for k, m in enumerate(e2e_maps))
        # roofline of the CR operator apply, timed live on the solver's stream
        ms_body, ms_row = g.time_operator(20)
        sz = g.sizes()
        resident = resident_roofline(g, clk)
        tuned_lanes, tuned_ms = g.tuning()
        # the network's forward pass over every contact (BF16 tensor cores), timed live
        mlp = None
        if params is not None:
            nc = len(s["c_body"])
            X = torch.empty((nc, 16), dtype=torch.float32, device=dev)
            Y = torch.empty((nc, 4), dtype=torch.float32, device=dev)
            nsn.nsn_contact_features(g.ctx, X.data_ptr())
            for _ in range(3):
                nsn.nsn_mlp_forward(g.ctx, X.data_ptr(), nc, Y.data_ptr())
            # CUDA events around 10 launches on the context's stream
            ms_f = nsn.nsn_mlp_time_forward(g.ctx, X.data_ptr(), nc, Y.data_ptr(), 10)
            flop = 2.0 * nc * (16 * 128 + 128 * 128 + 128 * 128 + 128 * 4)
            bf16 = measured_bf16_peak()
            mlp = {"bound": "tensor", "achieved": flop / (ms_f * 1e-3) / 1e12, "peak": bf16[0], "unit": "TFLOP/s",
                   "frac": flop / (ms_f * 1e-3) / 1e12 / bf16[0], "contacts": nc, "ms_forward": ms_f,
                   "flop_per_contact": flop / nc, "peak_kind": bf16[1],
                   "kernel": "mlp::k_forward_tc (whole network per 128-row tile, tcgen05.mma kind::f16 with BF16 operands in "
                             "shared memory and FP32 accumulators in tensor memory, weights resident, two CTAs per SM)"}
        g.close()
        # the other arms, same trajectory and accounting
        arms = {}
        if args.arms:
            # (name, cone projection, warm start, reset every step, NCP function, r strategy, line search)
            for name, cone, wm, reset, ncp, rs, ls in (("learned_warm_start", 1, nsn.NSN_WARM_LEARNED, False, 0, 2, LS),
                                                   ("learned_precond", 1, nsn.NSN_WARM_LEARNED | nsn.NSN_WARM_PRECOND,
                                                    False, 0, 2, LS),
                                                   ("fp64_bulk", 1, warm_names[warm], False, 0, 2, LS),
                                                   ("damped_update" if LS else "line_search", 1, warm_names[warm],
                                                    False, 0, 2, 0 if LS else 1),
                                                   ("plain_zero_start", 1, nsn.NSN_WARM_ZERO, False, 0, 2, 0),
                                                   ("plain_zero_start_line_search", 1, nsn.NSN_WARM_ZERO, False, 0, 2, 1),
                                                   ("as_printed", 0, nsn.NSN_WARM_ZERO, False, 0, 2, 0),
                                                   ("prev_warm_start", 1, nsn.NSN_WARM_PREV, False, 0, 2, 0),
                                                   ("prev_warm_start_line_search", 1, nsn.NSN_WARM_PREV, False, 0, 2, 1),
                                                   ("after_reset_zero", 1, nsn.NSN_WARM_ZERO, True, 0, 2, 0),
                                                   ("after_reset_learned", 1, nsn.NSN_WARM_LEARNED, True, 0, 2, 0),
                                                   ("ablation_min_map", 1, nsn.NSN_WARM_ZERO, True, 1, 2, 0),
                                                   ("ablation_r_h2", 1, nsn.NSN_WARM_ZERO, True, 0, 1, 0),
                                                   ("ablation_r_identity", 1, nsn.NSN_WARM_ZERO, True, 0, 0, 0)):
                fp64 = name == "fp64_bulk"
                # the headline's own configuration runs as an arm too: the arms time
                # fewer steps than the headline, and compare with it at equal length
                if (wm & 0xff) == nsn.NSN_WARM_LEARNED and params is None:
                    arms[name] = {"unavailable": "no trained weights (paper_1907_04587_gb300/weights)"}
                    continue
                ga = make_solver(nsn, s, stream, newton, cr, cone=cone, warm=wm, params=params, ncp=ncp, rscale=rs, ls=ls,
                                 fp64=fp64)
                try:
                    r = measure_arm(nsn, torch, ga, s, st0, stream, min(args.steps, args.arm_steps),
                                    min(args.warmup, 3), reset=reset,
                                    collider=collider)
                except nsn.NSNError as e:      # the method failing on this variant is a result
                    arms[name] = {"failed": str(e)}
                    ga.close()
                    continue
                if (wm & 0xff) != nsn.NSN_WARM_ZERO:
                    r["network_or_warm_rejected_islands_last_step"] = ga.warm_stats()["rejected"]
                ga.close()
                r.pop("sec")
                arms[name] = r
    try:      # a side measurement: a host-side failure is reported, the step's line stands
        contacts_rf = contact_generation(nsn, torch, s, stream, clk, rank)
    except (nsn.ColliderError, ValueError, MemoryError) as e:
        torch.cuda.synchronize()    # a CUDA error on the context is not a host failure: it raises here
        contacts_rf = {"failed": repr(e)}
    with torch.cuda.stream(stream):
        rscale_cmp = heavy_stack_comparison(nsn, stream)
    B = algorithmic_bytes(sz)
    peak, peak_kind = measured_peaks()
    achieved = B / ((ms_body + ms_row) * 1e-3) / 1e9
    # the streamed CR operator apply (islands above the resident cap, global mode), timed live
    apply_rf = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": operator_traffic(kernel_source_hash()),
                "kernel": "CR operator apply = k_body_pass<APPLY> + k_row_pass_isl<APPLY> (streamed CR loop)",
                "ms_body_pass": ms_body, "ms_row_pass": ms_row, "bytes_algorithmic": B,
                "bytes_design": design_bytes(sz), "peak_kind": f"{peak_kind} hbm_gbs (burst)",
                "body_pass_lanes_tuned": tuned_lanes,
                "body_pass_ms_for_4_8_16_lanes": [float(x) for x in tuned_ms]}
    if dist:
        t = torch.tensor([sec, sec_e2e, float(units), float(units_e2e)], device=dev, dtype=torch.float64)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        value = tsum[2].item() / tmax[0].item()
        value_e2e = tsum[3].item() / tmax[1].item()
    else:
        value = weak_scaling_value([units], [sec])
        value_e2e = weak_scaling_value([units_e2e], [sec_e2e])
    if rank != 0:
        return
    cb_value, cb = oracle_rate(args.workload, rank, args.cpu_budget, newton, cr)
    cb["value"] = cb_value
    cb["unit"] = UNIT
    main_arm.pop("sec")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": W["desc"], "n_envs": n_envs, "bodies": g.nb,
                   "rows": sz["rows"], "islands": main_arm["islands"], "newton_cap": newton, "cr_iters": cr,
                   "cr_stop": ("forcing term min(0.1, m/m0), floor, growth, cap" if CR_TOL else "floor, growth, cap"),
                   "newton_step": ("back-tracking line search (t = 1 .. 1/16, else the damped 0.75), per island"
                                   if LS else "damped, t = 0.75"),
                   "tol_rel": TOL, "cone_projection": True, "warm_start": warm_note,
                   "best_iterate": "an island that does not reach the tolerance returns its least-merit iterate",
                   "device_bytes": sz["device_bytes"], "launch": "kernel by kernel" if EAGER else
                   "one CUDA graph per step (Newton loop as a conditional WHILE node)",
                   "cr": ("island-resident CR (groups of small islands in shared memory, one thread block "
                          "each) + streamed CR loop for the rest" if RESIDENT else "streamed CR loop only"),
                   "l2": "working set larger than L2 (no flush between steps)",
                   "contacts": ("generated on the GPU at every step (Sec. 10: box corners and particles against the "
                                "ground and the boxes of their environment, margin 1 cm, candidates from v + h g), "
                                "the layout rebuilt for them, previous multipliers carried over by key; all inside "
                                "the timed step" if collider is not None else "the scene's contacts, fixed"),
                   "parallelism": f"weak, {world} independent replica(s)"},
        "convergence": main_arm,
        "arms": arms,
        # the dominant kernel of the step: the island-resident CR where the scene
        # has resident islands, else the streamed operator apply
        "roofline": resident_with_apply_equivalent(resident, B, sz, peak, peak_kind) if resident is not None else apply_rf,
        "operator_apply_roofline": apply_rf,
        "network_roofline": mlp,
        "contact_generation": contacts_rf,
        "heavy_stack_r_strategies": rscale_cmp,
        "cpu_baseline": cb,
        "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "the state makes a host round trip every step; the trajectory advances"},
        "gpu_launches": main_arm["kernels"],
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--arm-steps", type=int, default=20,
                    help="timed steps of each comparison arm (after min(warmup, 3) warm-up steps)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched4096", choices=list(WORKLOADS))
    ap.add_argument("--newton", type=int, default=0)
    ap.add_argument("--cr", type=int, default=0)
    ap.add_argument("--arms", type=int, default=1, help="also measure the plain, as-printed and reset arms")
    ap.add_argument("--warm", default="prev", choices=["learned", "prev", "zero"],
                    help="warm start of the headline arm (prev: the previous step's multipliers; learned: the "
                         "network with the previous-step start as fallback)")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=60.0, help="seconds of oracle work for --impl reference")
    ap.add_argument("--eager", type=int, default=0,
                    help="1: launch kernel by kernel (ncu cannot profile kernels of graphs with conditional nodes)")
    ap.add_argument("--resident", type=int, default=1,
                    help="0: no island-resident CR (every island in the streamed CR loop of four kernels per iteration)")
    ap.add_argument("--cr-tol", type=int, default=0,
                    help="1: inexact Newton, CR stops at ||r||_P <= min(0.1, merit/merit0) ||r0||_P (cap --cr)")
    ap.add_argument("--contacts", default="regen", choices=["regen", "fixed"],
                    help="regen (default): contacts generated at every step on the GPU (Sec. 10), timed with the step; "
                         "fixed: the scene's contacts throughout")
    ap.add_argument("--line-search", type=int, default=1,
                    help="1 (default): headline arm with the back-tracking line search of Sec. 8.1; 0: damped step")
    args = ap.parse_args()
    global EAGER, RESIDENT, CR_TOL, LS, REGEN
    EAGER = bool(args.eager)
    REGEN = 1 if args.contacts == "regen" else 0
    RESIDENT = int(args.resident)
    CR_TOL = int(args.cr_tol)
    LS = int(args.line_search)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
