"""The complementarity preconditioner of Sec. 7 on the heavy stack of Sec. 10
(box masses 8 ... 32768 kg, 4096:1, mu = 0.5).  The paper reports that
identity scaling (r = 1) may fail with large masses or large sliding
velocities, while r = h^2 and the effective-mass r converge; with the boxes
sliding at up to 5 m/s the oracle shows exactly that, and with the stack at
rest all three strategies converge."""
import numpy as np
import pytest

from paper_1907_04587_gb300 import scenes


def sliding_heavy_stack(vx):
    s = scenes.heavy_stack()
    s["vel"] = s["vel"].copy()
    s["vel"][:, 0] = np.float32(vx) * np.arange(1, 6, dtype=np.float32) / 5
    return s


@pytest.mark.parametrize("vx", [0.0, 5.0])
def test_heavy_stack_strategies(orc, vx):
    s = sliding_heavy_stack(vx)
    out = {}
    for rs in (orc.R_NONE, orc.R_H2, orc.R_EFFMASS):
        o = orc.Oracle(s, newton_iters=40, cr_iters=40, rscale=rs, tol_rel=1e-6)
        st = o.step()
        out[rs] = st["merit_final"] / st["merit0"]
    print(vx, out)
    assert out[orc.R_H2] <= 1e-6 and out[orc.R_EFFMASS] <= 1e-6
    if vx == 0.0:
        assert out[orc.R_NONE] <= 1e-6
    else:
        assert out[orc.R_NONE] > 1.0      # identity scaling diverges on the sliding stack
