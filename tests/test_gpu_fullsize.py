"""Parity at the full size of the batched workload (4096 environments,
2,358,981 rows), in the launch configuration bench.py times: FP32, one CUDA
graph per step, islands solved side by side, island-resident CR, the
back-tracking line search, projection onto the friction cone.

The oracle cannot solve 4096 environments in a test's time, so environments
are sampled and each is solved by the FP64 oracle alone (an environment is a
union of islands and A is block diagonal by island, so this is the same
problem); the rest is checked through properties that hold at any size."""
import numpy as np
import pytest

from paper_1907_04587_gb300 import nsn, scenes
from test_oracle_islands import sub_scene

pytestmark = pytest.mark.gpu

H = 1.0 / 60.0
G = 9.81
PRM = dict(newton_iters=30, cr_iters=400, tol_rel=1e-6, island_stop=1, cone_project=1, line_search=1, best_iterate=1)
SAMPLE = tuple(int(e) for e in np.linspace(0, 4095, 64))   # 64 environments spread over the batch


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    yield


@pytest.fixture(scope="module")
def full():
    s = scenes.batched_envs(seed=0, n_envs=4096)
    g = nsn.Solver(s, precision=nsn.NSN_FP32, use_graph=1, **PRM)
    g.step()
    return s, g


def mass_weighted(s, sel, v_a, w_a, v_b, w_b):
    """Kinetic-energy norm of (a - b) over the bodies sel, relative to b's plus g h."""
    R = scenes.quat_rot(s["quat"][sel])
    m = s["mass"][sel].astype(np.float64)
    Iw = np.einsum("nij,nj,nkj->nik", R, s["inertia"][sel].astype(np.float64), R)
    rig = s["kind"][sel] == 0
    def e(dv, dw):
        return np.sqrt((m * (dv ** 2).sum(1)).sum() + np.einsum("ni,nij,nj->", dw[rig], Iw[rig], dw[rig]))
    return e(v_a - v_b, w_a - w_b) / (e(v_b, w_b) + H * G * np.sqrt(m.sum()))


def test_sampled_environments_match_oracle(orc, full):
    s, g = full
    st = g.get_state()
    n_isl, bi_g = g.islands()
    stop_g = g.island_stats()["stopped_at"]
    lam = g.get_lambda()
    nc, nj = len(s["c_body"]), len(s["j_body"])
    lam_c, lam_j = lam[:3 * nc].reshape(nc, 3), lam[3 * nc:3 * nc + 5 * nj].reshape(nj, 5)
    agree = total = 0
    errs, ratios = [], []
    for e in SAMPLE:
        bodies = np.nonzero(s["env"] == e)[0]
        sub = sub_scene(s, bodies)
        o = orc.Oracle(sub, **PRM)
        o.step()
        so = o.get_state()
        _, bi_o, _ = o.islands()
        stop_o = o.island_stats()["stopped_at"]
        # islands of this environment on the GPU, in the oracle's island order
        isl_g = bi_g[bodies]
        conv_g = np.array([stop_g[isl_g[np.nonzero(bi_o == i)[0][0]]] >= 0 for i in range(len(stop_o))])
        conv_o = stop_o >= 0
        agree += int((conv_g == conv_o).sum())
        total += len(conv_o)
        both = conv_g & conv_o
        # the GPU's FP32 iterate in the oracle's FP64 equations: merit at it
        # over the island's zero-iterate merit (the oracle's own iterate: <= 1e-6)
        kc = np.isin(s["c_body"][:, 0], bodies) | np.isin(s["c_body"][:, 1], bodies)
        kj = np.isin(s["j_body"][:, 0], bodies) | np.isin(s["j_body"][:, 1], bodies)
        o.set_state(**{k: np.asarray(sub[k], np.float64) for k in ("pos", "quat", "vel", "omega")})
        _, m_at = o.merit_at(st["vel"][bodies], st["omega"][bodies], np.concatenate([lam_c[kc].ravel(), lam_j[kj].ravel()]))
        ratios.extend((m_at / o.island_stats()["merit0"])[both].tolist())
        sel = both[bi_o]                # bodies of islands converged on both sides
        if sel.any():
            err = mass_weighted(sub, sel, st["vel"][bodies][sel], st["omega"][bodies][sel], so["vel"][sel],
                                so["omega"][sel])
            print(f"env {e}: {len(stop_o)} islands, converged gpu {conv_g.sum()} oracle {conv_o.sum()}, "
                  f"velocity error on islands converged on both {err:.2e}")
            errs.append(err)
    errs, ratios = np.array(errs), np.array(ratios)
    print("islands with the same converged / not converged outcome:", agree, "of", total)
    print(f"oracle merit at the GPU iterate / merit0 on {len(ratios)} islands converged on both: "
          f"median {np.median(ratios):.2e} p95 {np.quantile(ratios, 0.95):.2e} p99 {np.quantile(ratios, 0.99):.2e} "
          f"max {ratios.max():.2e}")
    print(f"environments within 1e-5: {(errs < 1e-5).sum()} of {len(errs)}, worst {errs.max():.2e}")
    # FP32 converges a few islands fewer than FP64 (chains at their rounding
    # limit): the outcomes agree on 95% of the islands measured
    assert agree >= 0.9 * total
    # validity of the GPU's answer by the oracle's definition, whatever the
    # conditioning: on every island converged on both sides, the GPU's FP32
    # iterate meets the oracle's FP64 equations to about the 1e-6 tolerance
    # (measured: median 1.6e-7, p99 3.2e-6, max 9.4e-6 of the zero-iterate
    # merit -- the FP32 rounding of u, lambda and of the GPU's own evaluation
    # adds to the residual it measured on itself)
    assert np.median(ratios) <= 1e-6 and np.quantile(ratios, 0.99) <= 1e-5 and ratios.max() <= 2e-5
    # the FP32 path against FP64 on islands both solved to 1e-6 of their merit:
    # the stop test bounds the residual, so two converged iterates differ by up
    # to the island's inverse Jacobian times 1e-6 of its merit -- above 1e-5 on
    # a few near-singular islands (coplanar corner contacts and hinges,
    # regularised by eps only; measured 60 of 64 environments within 1e-5)
    assert (errs < 1e-5).mean() >= 0.9 and errs.max() < 1e-4


def test_full_size_properties(full):
    """Every contact's multipliers lie in the friction cone after the projected
    update (lambda_n >= 0, |lambda_f| <= mu lambda_n); every island that
    stopped meets the tolerance; the state is finite; most islands converge."""
    s, g = full
    lam = g.get_lambda().astype(np.float64)
    nc = len(s["c_body"])
    l3 = lam[:3 * nc].reshape(nc, 3)
    mu = s["c_mu"].astype(np.float64)
    assert np.all(l3[:, 0] >= 0.0)
    fr = np.hypot(l3[:, 1], l3[:, 2])
    bad = ~(fr <= mu * l3[:, 0] * (1 + 1e-5) + 1e-30)
    if bad.any():
        i = np.nonzero(bad)[0]
        print("outside the cone:", len(i), "contacts; first", [(int(k), float(l3[k, 0]), float(fr[k]), float(mu[k]))
                                                              for k in i[:5]])
    assert not bad.any()
    st = g.island_stats()
    done = st["stopped_at"] >= 0
    assert done.mean() > 0.8
    assert np.all(st["merit_final"][done] <= 1e-6 * st["merit0"][done] * 1.001)
    assert all(np.isfinite(v).all() for v in g.get_state().values())
