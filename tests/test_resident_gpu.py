"""The resident batch kernel: a batch's matrices of order <= resident_max_n run
in one persistent launch, each matrix's whole level loop (Sec. 5.3, eq.
generalradix) inside one CTA's shared memory. Parity against the oracle's
matrix scheme for every matrix, for each arithmetic, next to the same batch
through the grouped launches only (NEUMANN_FLAG_NO_RESIDENT).

Tolerances as the grouped batch (tests/test_fullsize_gpu.py): FP32 1e-5,
split forms 1e-4 on these damped Jacobi matrices (rho ~ 0.9).
"""

import pytest

from oracle import closed_form as CF
from oracle import evaluate as EV
from workloads import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-4, "split_fp16": 1e-4}
SIZES = tuple(range(1, 65)) + (80, 128, 200, 256)


def _batch(count, seed, sizes=SIZES):
    return G.jacobi_batch(count, seed, sizes=sizes)


def _run(mats, k, radix, dtype, flags=0):
    import paper_2602_11843_gb300 as nm

    io = torch.float32 if dtype == "fp32" else torch.float64
    bp = nm.BatchedPlan(len(mats), 256, k, radix, dtype, flags)
    As = [torch.tensor(m["A"], dtype=io, device="cuda") for m in mats]
    outs = bp(As)
    torch.cuda.synchronize()
    return [o.double().cpu().numpy() for o in outs], bp.status(), nm.neumann_plan_info(bp.handle)


@pytest.mark.parametrize("dtype", ["fp32", "split_bf16", "split_fp16"])
@pytest.mark.parametrize("k,radix", [(81, 9), (225, 15), (81, 0), (625, 25), (2, 9), (1, 9)])
def test_resident_batch_against_oracle(dtype, k, radix):
    import paper_2602_11843_gb300 as nm

    if k in (1, 2) and radix == 9:
        radix = 2 if k == 2 else 1  # k = 1, 2: no product at all
    mats = _batch(96, 700 + k + radix)
    outs, st, info = _run(mats, k, radix, dtype)
    assert st == 0
    assert info["resident_max_n"] >= 48
    errs = []
    for m, S in zip(mats, outs):
        ref, _ = EV.evaluate(m["A"], k, radix)
        errs.append(CF.rel_fro(S, ref))
    small = [e for m, e in zip(mats, errs) if m["n"] <= info["resident_max_n"]]
    print(f"resident {dtype} k={k} radix {radix}: {len(small)} resident, max err {max(small):.3e}, "
          f"all max {max(errs):.3e}")
    assert len(small) > 40
    assert max(errs) < TOL[dtype]
    del nm


@pytest.mark.parametrize("dtype", ["fp32", "split_bf16"])
def test_resident_matches_grouped(dtype):
    """The same batch with and without the resident launch: both within the
    tolerance of the oracle, and close to each other."""
    import paper_2602_11843_gb300 as nm

    mats = _batch(64, 11, sizes=tuple(range(16, 65, 4)))
    a, st_a, info_a = _run(mats, 81, 9, dtype)
    b, st_b, info_b = _run(mats, 81, 9, dtype, nm.FLAG_NO_RESIDENT)
    assert st_a == 0 and st_b == 0
    assert info_a["resident_max_n"] == 48 and info_b["resident_max_n"] == 0
    for m, x, y in zip(mats, a, b):
        assert CF.rel_fro(x, y) < 2 * TOL[dtype], m["n"]


def test_resident_mixed_radix_and_paper_residual():
    import paper_2602_11843_gb300 as nm

    mats = _batch(40, 12, sizes=(8, 24, 40, 64))
    outs, st, info = _run(mats, 135, 0, "split_bf16", nm.FLAG_ALLOW_APPROX | nm.FLAG_RESIDUAL_PAPER)
    assert st == 0
    lv = info["levels"]
    assert lv == [9, 15]
    for m, S in zip(mats, outs):
        ref, _ = EV.evaluate(m["A"], 135, 0, levels=lv, form="paper")
        assert CF.rel_fro(S, ref) < 1e-4, m["n"]


def test_resident_nonfinite_status():
    """Undamped Jacobi matrices (rho > 1) of small order: S_k overflows in the
    resident launch, which reports NEUMANN_STATUS_NONFINITE."""
    import paper_2602_11843_gb300 as nm

    mats = G.jacobi_batch(4, 4, sizes=(32,), damped=False)
    outs, st, _ = _run(mats, 15 ** 3, 15, "fp32")
    assert st & nm.STATUS_NONFINITE


def test_resident_graph_capture_and_host_buffers():
    """A batch with resident and grouped matrices, captured in a CUDA graph and
    replayed; and the same batch through the packed host-buffer call."""
    import paper_2602_11843_gb300 as nm

    mats = _batch(48, 13, sizes=(16, 33, 64, 100, 256))
    ns = [m["n"] for m in mats]
    bp = nm.BatchedPlan(len(mats), 256, 81, 9, "split_bf16")
    As = [torch.tensor(m["A"], device="cuda") for m in mats]
    outs = [torch.empty_like(a) for a in As]
    bp.bind(As, outs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bp.launch()  # warm-up outside capture (tables, first launch)
    torch.cuda.synchronize()
    for o in outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bp.launch()
    g.replay()
    torch.cuda.synchronize()
    assert bp.status() == 0
    refs = [EV.evaluate(m["A"], 81, 9)[0] for m in mats]
    for S, ref in zip(outs, refs):
        assert CF.rel_fro(S.cpu().numpy(), ref) < 1e-4
    A_host = torch.cat([torch.tensor(m["A"]).reshape(-1) for m in mats]).pin_memory()
    S_host = torch.empty_like(A_host).pin_memory()
    bp.eval_host(ns, A_host, S_host)
    bp.host_wait()
    off = 0
    for m, ref in zip(mats, refs):
        n = m["n"]
        S = S_host[off:off + n * n].view(n, n).numpy()
        off += n * n
        assert CF.rel_fro(S, ref) < 1e-4
