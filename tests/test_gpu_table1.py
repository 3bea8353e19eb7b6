"""The NER methods of Sec. 5.1 on the GPU: the direct-sum mode (the "direct
FT" ground truth) and the FFT-with-linear-interpolation modes (sigma = 2, 1)
against their FP64 oracles, and the ordering of Table 1 (NER-NUFFT closest
to the direct FT, then FFT sigma = 2, then FFT sigma = 1) on a ball."""
import numpy as np
import pytest

import oracle
from oracle import comparison as C
from paper_1510_01078_gb300 import inputs
from parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nd():
    from paper_1510_01078_gb300 import build
    build.build()
    from paper_1510_01078_gb300 import nedner
    return nedner


def _problem(case):
    return oracle.Problem(sensor_xy=case["sensor_xy"], h=case["h"], Nt=case["Nt"], dt=case["dt"], c=case["c"],
                          nx=case["nx"], ny=case["ny"], nz=case["nz"], dx=case["dx"], dy=case["dy"], dz=case["dz"])


@pytest.fixture(scope="module")
def case():
    return inputs.small_case(16, 16, 32, 200, 128, seed=91, layout="disc")


def _gpu(nd, case, mode):
    plan = nd.plan_from_config(case, ner_mode=mode)
    p = plan.forward(torch.as_tensor(np.asarray(case["g"], dtype=np.float32), device="cuda")).cpu().numpy()
    plan.close()
    return p


def test_direct_mode_matches_oracle(nd, case):
    check(_gpu(nd, case, "direct"), oracle.forward(_problem(case), case["g"]), 1e-5)


@pytest.mark.parametrize("mode,sigma", [("linear2", 2), ("linear1", 1)])
def test_linear_modes_match_oracle(nd, case, mode, sigma):
    check(_gpu(nd, case, mode), C.forward_linear(_problem(case), case["g"], sigma), 1e-5)


def test_comparison_modes_refuse_transposed_calls(nd, case):
    plan = nd.plan_from_config(case, ner_mode="linear2")
    p = torch.zeros((case["nz"], case["ny"], case["nx"]), device="cuda")
    with pytest.raises(nd.NednerError):
        plan.adjoint(p)
    with pytest.raises(nd.NednerError):
        plan.grad_positions(torch.zeros((200, case["Nt"]), device="cuda"), p)
    plan.close()


def test_table1_ordering_on_a_ball(nd):
    from paper_1510_01078_gb300 import table1
    cfg = table1.ball_workload(n=32, nz=64, Nt=128, dx=0.1e-3, R=0.4e-3)
    res = table1.run(cfg, reps=2)
    d = {r["method"]: r["deficit_pct"]["3D"] for r in res["rows"]}
    assert d["NER (sigma=2, w=12)"] < d["FFT + linear (sigma=2)"] < d["FFT + linear (sigma=1)"], d
    assert d["NER (sigma=2, w=12)"] < 1e-2, d
    for r in res["rows"]:
        assert all(np.isfinite(v) for v in r["deficit_pct"].values())
