"""GPU checks of the autotuner: it settles on one of its candidates, the plan
still computes S_k to the split's tolerance afterwards (and the tuning runs
themselves leave a correct S), and a later plan of the same shape starts from
the recorded choice."""

import numpy as np
import pytest

from oracle import closed_form as CF
from oracle import evaluate as EV
from workloads import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _nm():
    import paper_2602_11843_gb300 as nm

    return nm


@pytest.mark.parametrize("dtype", ["split_bf16", "split_fp16"])
def test_autotune_single_plan(dtype):
    nm = _nm()
    pl = G.config_inputs(2)  # n = 4096, planted spectrum in [-0.9, 0.9]
    ref = EV.planted_reference(pl["V"], pl["lam"], 729, 9)
    A = torch.tensor(pl["A"], dtype=torch.float64, device="cuda")
    p = nm.Plan(4096, 729, 9, dtype)
    S = torch.empty_like(A)
    info = p.autotune(A, out=S, reps=2)
    assert info["tuned"] == 1 and info["tile_pair"] in (0, 1) and info["raster_group"] in (4, 8, 16)
    assert p.status() == 0
    assert CF.rel_fro(S.cpu().numpy(), ref) < 1e-3  # the tuning runs' own result
    S2 = p(A)
    torch.cuda.synchronize()
    assert p.status() == 0 and CF.rel_fro(S2.cpu().numpy(), ref) < 1e-3
    q = nm.Plan(4096, 81, 9, dtype)  # same padded order and dtype: starts tuned
    assert q.info["tuned"] == 1
    assert (q.info["tile_pair"], q.info["raster_group"]) == (info["tile_pair"], info["raster_group"])
    print(f"{dtype}: tuned to pair={info['tile_pair']} group={info['raster_group']}")


def test_autotune_respects_single_cta_flag_and_simt_paths():
    nm = _nm()
    rng = np.random.default_rng(3)
    A = torch.tensor(rng.standard_normal((512, 512)) * (0.4 / 512 ** 0.5), device="cuda")
    p = nm.Plan(512, 81, 9, "split_bf16", nm.FLAG_SINGLE_CTA)
    assert p.autotune(A, reps=1)["tile_pair"] == 0
    f = nm.Plan(512, 81, 9, "fp64")
    info = f.autotune(A, reps=1)
    assert info["tuned"] == 1 and info["tile_pair"] == 0


def test_autotune_batched_chunk():
    nm = _nm()
    mats = G.jacobi_batch(300, 4000)
    bp = nm.BatchedPlan(len(mats), 256, 81, 9, "split_bf16")
    As = [torch.tensor(m["A"], dtype=torch.float64, device="cuda") for m in mats]
    outs = [torch.empty_like(a) for a in As]
    info = bp.autotune(As, outs, reps=1)
    assert info["tuned"] == 1 and info["batch_chunk"] in (300, 150, 75)
    outs2 = bp(As)
    torch.cuda.synchronize()
    assert bp.status() == 0
    for i in (0, 7, 150, 299):
        ref, _ = EV.evaluate(mats[i]["A"], 81, 9)
        for S in (outs[i], outs2[i]):
            assert CF.rel_fro(S.cpu().numpy(), ref) < 2e-3  # the batched split-BF16 bound of the parity tests
    again = nm.BatchedPlan(len(mats), 256, 81, 9, "split_bf16")
    assert nm.neumann_plan_info(again.handle)["batch_chunk"] == info["batch_chunk"]
