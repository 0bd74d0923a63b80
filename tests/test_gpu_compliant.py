"""GPU check of compliant joint rows (Sec. 3.2: C = e / h^2 on the joint's
rows, h = (c + e lambda) / h): the closed-form step of a body hanging from a
compliant joint, the same pin the oracle meets.  (A fixed-iteration chain is
no parity measure here: on such a scene the oracle's own iterate after 12
Newton iterations moves by 7e-6 when the positions move by 1e-15.)"""
import numpy as np
import pytest

from paper_1907_04587_gb300 import nsn, scenes

pytestmark = pytest.mark.gpu

H = 1.0 / 60.0
G = 9.81


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    yield


@pytest.mark.parametrize("e", [0.0, 1e-4, 1e-3])
def test_compliant_hanging_body_closed_form(e):
    """v = -m g h / (m + h^2 / e) after one step (FP64 build)."""
    m = 3.0
    b = scenes.SceneBuilder()
    i = b.add_rigid((0.2, -0.1, 1.0), (1, 0, 0, 0), mass=m, inertia=(0.2, 0.3, 0.4))
    b.add_revolute(i, -1, (0, 0, 0), (0.2, -0.1, 1.0), (0, 1, 0), (0, 1, 0), e)
    s = b.build()
    g = nsn.Solver(s, precision=nsn.NSN_FP64, newton_iters=30, cr_iters=30, line_search=1)
    g.step()
    v = g.get_state_f64()["vel"][0]
    ef = float(np.float32(e))
    expect = 0.0 if ef == 0.0 else -m * G * H / (m + H * H / ef)
    print("e", e, "v_z", v[2], "closed form", expect)
    assert abs(v[2] - expect) < 1e-9 * G * H

