"""neumann_eval_host: host (pinned or pageable) inputs and outputs, copies
overlapped with evaluations through the plan's two staging sets. Several calls
are issued back to back before one wait, with distinct inputs, so a wrong
ordering between a set's copy-in, evaluation and copy-out would hand a result
to the wrong call."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,pinned", [("split_bf16", True), ("fp64", True), ("split_fp16", False),
                                          ("fp32", True)])
def test_eval_host_matches_device_path(dtype, pinned):
    import paper_2602_11843_gb300 as nm

    n, k = 300, 81
    p = nm.Plan(n, k, 9, dtype)
    dt = p.io_dtype
    rng = np.random.default_rng(42)
    As = [torch.tensor(rng.standard_normal((n, n)) * (0.45 / n ** 0.5), dtype=dt) for _ in range(5)]
    if pinned:
        As = [a.pin_memory() for a in As]
    outs = [torch.empty((n, n), dtype=dt, pin_memory=pinned) for _ in As]
    for a, o in zip(As, outs):
        p.eval_host(a, out=o)
    p.host_wait()
    assert p.status() == 0
    for a, o in zip(As, outs):
        ref = p(a.cuda()).cpu()
        torch.cuda.synchronize()
        assert torch.equal(o, ref)


def test_eval_host_leading_dimensions():
    import paper_2602_11843_gb300 as nm

    n = 200
    p = nm.Plan(n, 81, 9, "fp64")
    rng = np.random.default_rng(3)
    big = torch.tensor(rng.standard_normal((n, n + 24)) * (0.4 / n ** 0.5)).pin_memory()
    A = big[:, :n]
    Sbig = torch.full((n, n + 40), 5.0, dtype=torch.float64).pin_memory()
    S = Sbig[:, :n]
    p.eval_host(A, out=S)
    p.host_wait()
    ref = p(A.contiguous().cuda()).cpu()
    torch.cuda.synchronize()
    assert torch.equal(S, ref) and torch.all(Sbig[:, n:] == 5.0)


@pytest.mark.parametrize("dtype", ["split_bf16", "fp32"])
def test_eval_batched_host_packed(dtype):
    """Three back-to-back packed batches (different contents) before one wait,
    against the device batched call on the same matrices."""
    import paper_2602_11843_gb300 as nm
    from workloads import generators as G

    ns = [16, 48, 128, 200, 256, 33, 1]
    bp = nm.BatchedPlan(len(ns), 256, 81, 9, dtype)
    dt = torch.float32 if dtype == "fp32" else torch.float64
    total = sum(n * n for n in ns)
    batches = []
    for b in range(3):
        mats = [G.gaussian_scaled(n, 0.5, 500 + 10 * b + i)["A"] for i, n in enumerate(ns)]
        A = torch.cat([torch.tensor(m, dtype=dt).reshape(-1) for m in mats]).pin_memory()
        S = torch.empty(total, dtype=dt).pin_memory()
        batches.append((mats, A, S))
    for _, A, S in batches:
        bp.eval_host(ns, A, S)
    bp.host_wait()
    assert bp.status() == 0
    for mats, A, S in batches:
        As = [torch.tensor(m, dtype=dt, device="cuda") for m in mats]
        ref = bp(As)
        torch.cuda.synchronize()
        off = 0
        for n, r in zip(ns, ref):
            assert torch.equal(S[off:off + n * n].view(n, n), r.cpu())
            off += n * n
