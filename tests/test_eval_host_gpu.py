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
