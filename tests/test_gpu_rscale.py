"""The three complementarity preconditioners of Sec. 7 (r = 1, r = h^2, the
effective-mass r) on the sliding heavy stack of Sec. 10, GPU (FP64 build)
against the FP64 oracle: the merits of the Newton iterations agree, and the
outcome the oracle pins (identity scaling diverges once the boxes slide, the
other two converge) holds on the GPU.  The linear systems of each strategy are
compared in test_gpu_parity.test_linear_system_parity."""
import numpy as np
import pytest

from paper_1907_04587_gb300 import nsn
from test_oracle_rscale import sliding_heavy_stack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    yield


@pytest.mark.parametrize("rscale", [0, 1, 2])
@pytest.mark.parametrize("vx", [0.0, 5.0])
def test_heavy_stack_merit_histories(orc, rscale, vx):
    s = sliding_heavy_stack(vx)
    p = dict(newton_iters=40, cr_iters=40, rscale=rscale, tol_rel=1e-6)
    o = orc.Oracle(s, **p)
    g = nsn.Solver(s, precision=nsn.NSN_FP64, **p)
    so, sg = o.step(), g.step()
    ho, hg = np.asarray(o.merit_history()), np.asarray(g.merit_history())
    conv = so["merit_final"] <= 1e-6 * so["merit0"]
    print(f"r strategy {rscale}, vx {vx}: newton {sg['newton_done']}/{so['newton_done']}, "
          f"merit ratio gpu {sg['merit_final'] / sg['merit0']:.2e} oracle {so['merit_final'] / so['merit0']:.2e}")
    # the sliding stack (4096:1 masses) is ill-conditioned enough that two
    # FP64 evaluation orders part after a few Newton iterations (a friction or
    # Fischer-Burmeister decision taken the other way; measured: from the seventh);
    # the first five merits agree, and so does the outcome
    n = 5 if vx > 0 else min(len(ho), len(hg))
    np.testing.assert_allclose(hg[:n], ho[:n], rtol=1e-6, atol=1e-10 * ho[0])
    if conv:
        if vx == 0:
            assert sg["newton_done"] == so["newton_done"]
        assert sg["merit_final"] <= 1e-6 * sg["merit0"]
    else:
        assert sg["merit_final"] > sg["merit0"]
