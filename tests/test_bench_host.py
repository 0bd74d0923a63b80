"""Host-side logic of bench.py on CPU: byte counts, weak-scaling aggregation
over two gloo ranks, and the reference arm (the FP64 oracle) JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_per_unit():
    one = dict(rigid_entries=1, particle_entries=0, rows=0, tets=0, rigid=0, particles=0, pair_rows=0)
    assert bench.algorithmic_bytes(one) == 56
    sz = dict(rigid_entries=10, particle_entries=20, rows=7, tets=2, rigid=3, particles=5, pair_rows=1)
    assert bench.algorithmic_bytes(sz) == 56 * 10 + 32 * 20 + 12 * 7 + 24 * 2 + 76 * 3 + 36 * 5
    assert bench.design_bytes(sz) == 36 * 10 + 24 * 20 + 36 * 3 + 16 * 5 + 36 * 1 + 168 * 2


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, sec = 4096.0 * (rank + 1), 1.0 + rank
    t = torch.tensor([sec, float(units)], dtype=torch.float64)
    tmax = t.clone(); dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone(); dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    q.put((rank, tsum[1].item() / tmax[0].item()))
    dist.destroy_process_group()


def test_weak_scaling_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(60)
    got = dict(q.get(timeout=10) for _ in range(2))
    expect = bench.weak_scaling_value([4096.0, 8192.0], [1.0, 2.0])
    assert got[0] == pytest.approx(expect) and got[1] == pytest.approx(expect)


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "cube_stack", "--ref-budget", "0.5"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == bench.UNIT and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_collider_test_count_matches_enumeration():
    """The contact-generation roofline counts the tests in closed form
    (planes, plus the boxes of the vertex's environment other than its own
    body and its joint partners); check it against the enumeration the
    oracle's loops perform, on batched environments with particles added."""
    import numpy as np
    from paper_1907_04587_gb300 import scenes
    s = scenes.batched_envs(seed=9, n_envs=5)
    kind = s["kind"].copy()
    kind[::7] = 1                         # some particles among the bodies
    half = s["half"].copy()
    half[::11] = 0.0                      # and some rigid bodies without a shape
    env = s["env"]
    jb = s["j_body"][(s["j_body"][:, 0] >= 0) & (s["j_body"][:, 1] >= 0)]
    nvert, box_tests = bench.collide_tests(kind, half, env, jb, 5)
    pairs = {(int(a), int(b)) for a, b in jb} | {(int(b), int(a)) for a, b in jb}
    is_box = [(k == 0 and np.all(h > 0)) for k, h in zip(kind, half)]
    brute = 0
    for a in range(len(kind)):
        nv = 1 if kind[a] == 1 else (8 if is_box[a] else 0)
        for b in range(len(kind)):
            if b != a and env[b] == env[a] and is_box[b] and (a, b) not in pairs:
                brute += nv
    assert brute == int((nvert * box_tests).sum())
    r = bench.oracle_collide_rate(s, ((0.0, 0.0, 1.0, 0.0),), jb, n_envs_sample=2)
    assert r["tests_per_s"] > 0 and r["contacts_sample"] > 0
