"""Device failure reporting and CUDA-graph capture, through the C ABI.

* Bounded waits: a probe kernel waits, with the tensor-core product's wait
  code and a short limit, on an mbarrier nothing arrives on. The plan's status
  word must report NEUMANN_STATUS_TIMEOUT, and the context must stay usable
  (the next evaluation is correct and clean). No kernel faults or hangs.
* Graph capture: after one warm-up call (workspace, tensor maps and tile tables
  exist), an evaluation is captured into a CUDA graph and replayed on new
  inputs copied into the same buffers.
"""


import pytest

from oracle import closed_form as CF
from oracle import evaluate as EV
from workloads import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import paper_2602_11843_gb300 as nm

    g = G.gaussian_scaled(64, 0.5, 3)
    p = nm.Plan(64, 81, 9, "split_bf16")
    stream = torch.cuda.current_stream().cuda_stream
    nm.neumann_plan_selftest_timeout(p.handle, 5_000_000, stream)  # 5 ms
    assert p.status() & nm.STATUS_TIMEOUT
    A = torch.tensor(g["A"], dtype=torch.float64, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    assert p.status() == 0
    ref, _ = EV.evaluate(g["A"], 81, 9)
    assert CF.rel_fro(S.cpu().numpy(), ref) < 2e-4


@pytest.mark.parametrize("dtype,tol", [("fp64", 1e-12), ("split_bf16", 1e-3)])
def test_graph_capture_single(dtype, tol):
    import paper_2602_11843_gb300 as nm

    n, k = 300, 225
    p = nm.Plan(n, k, 15, dtype)
    first = G.planted_symmetric(n, 0.9, 31)
    A = torch.tensor(first["A"], dtype=torch.float64, device="cuda")
    S = torch.empty_like(A)
    p(A, out=S)  # warm-up: workspace and tensor maps
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        p(A, out=S)
    second = G.planted_symmetric(n, 0.9, 32)
    A.copy_(torch.tensor(second["A"], dtype=torch.float64))
    graph.replay()
    torch.cuda.synchronize()
    assert p.status() == 0
    ref = EV.planted_reference(second["V"], second["lam"], k, 15)
    assert CF.rel_fro(S.cpu().numpy(), ref) < tol


def test_timing_flag_records_nothing_under_capture():
    """A plan with NEUMANN_FLAG_TIMING captured into a CUDA graph: the captured
    evaluation records no events (they could not be timed); an evaluation
    outside the capture still records one interval per product."""
    import paper_2602_11843_gb300 as nm

    n = 256
    p = nm.Plan(n, 81, 9, "split_bf16", nm.FLAG_TIMING)
    pl = G.planted_symmetric(n, 0.9, 33)
    A = torch.tensor(pl["A"], dtype=torch.float64, device="cuda")
    S = torch.empty_like(A)
    p(A, out=S)
    torch.cuda.synchronize()
    assert len(p.timing()) == p.info["products_executed"]
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        p(A, out=S)
    graph.replay()
    torch.cuda.synchronize()
    assert p.timing() == []
    assert p.status() == 0
    ref = EV.planted_reference(pl["V"], pl["lam"], 81, 9)
    assert CF.rel_fro(S.cpu().numpy(), ref) < 1e-3


def test_graph_capture_grouped_batch():
    import paper_2602_11843_gb300 as nm

    mats = G.jacobi_batch(40, 77, sizes=(16, 64, 200))
    bp = nm.BatchedPlan(len(mats), 256, 81, 9, "split_bf16")
    As = [torch.tensor(m["A"], dtype=torch.float64, device="cuda") for m in mats]
    outs = [torch.empty_like(a) for a in As]
    bp.bind(As, outs)
    bp.launch()  # warm-up: workspace, tensor maps, tile tables
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bp.launch()
    for o in outs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert bp.status() == 0
    for m, o in zip(mats, outs):
        ref, _ = EV.evaluate(m["A"], 81, 9)
        assert CF.rel_fro(o.cpu().numpy(), ref) < 2e-3


@pytest.mark.parametrize("dtype,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("split_bf16", 2e-4)])
@pytest.mark.parametrize("radix,k", [(9, 729), (15, 225), (2, 1024)])
def test_nonnormal_upper_triangular(dtype, tol, radix, k):
    """Sec. 6's nonnormal test: upper-triangular A with eigenvalues (its diagonal)
    in [-0.9, 0.9] and O(1/sqrt(n)) strictly-upper entries; S has transient
    growth (max entry ~9); the standard bounds hold."""
    import paper_2602_11843_gb300 as nm

    inp = G.nonnormal_triangular(200, 0.9, 5)
    ref, _ = EV.evaluate(inp["A"], k, radix)
    p = nm.Plan(200, k, radix, dtype)
    A = torch.tensor(inp["A"], dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    assert p.status() == 0
    err = CF.rel_fro(S.double().cpu().numpy(), ref)
    print(f"nonnormal radix {radix} k {k} {dtype} rel err {err:.2e}")
    assert err < tol
