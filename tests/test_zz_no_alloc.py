"""The allocation-free product, neumann_matmul_noalloc, against the plan-based
product it mirrors (neumann_plan_matmul on a SPLIT_BF16 plan).

The allocation-free call keeps its operand scratch in a fixed array inside the
library, shared by every call, so the test makes two calls in a row with
different inputs and sizes and checks that the second is not affected by what
the first left behind. This file is collected last so that a run stopping at
the first failure has already run every other test.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 2e-5  # the split-BF16 product tolerance of tests/test_parity_gpu.py


def _rel(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def test_noalloc_matches_plan_matmul_on_two_calls():
    import paper_2602_11843_gb300 as nm
    from paper_2602_11843_gb300 import _capi as C

    stream = torch.cuda.current_stream().cuda_stream
    for call, n in enumerate((1000, 300)):  # larger first: the second call reuses a dirtier array
        rng = np.random.default_rng(100 + call)
        A = torch.tensor(rng.standard_normal((n, n)), dtype=torch.float64, device="cuda")
        B = torch.tensor(rng.standard_normal((n, n)), dtype=torch.float64, device="cuda")
        out_na = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        C.neumann_matmul_noalloc(n, A.data_ptr(), n, B.data_ptr(), n, out_na.data_ptr(), n, stream)
        plan = nm.Plan(n, 2, 2, "split_bf16")
        out_plan = plan.matmul(A, B)
        torch.cuda.synchronize()
        a, b = out_na.cpu().numpy(), out_plan.cpu().numpy()
        ref = (A.cpu() @ B.cpu()).numpy()
        assert np.isfinite(a).all()
        assert _rel(a, b) < TOL, f"call {call}: differs from neumann_plan_matmul"
        assert _rel(a, ref) < TOL, f"call {call}: differs from the FP64 product"


def test_noalloc_rejects_orders_above_its_scratch():
    from paper_2602_11843_gb300 import _capi as C

    x = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(C.NeumannError) as e:
        C.neumann_matmul_noalloc(1025, x.data_ptr(), 1025, x.data_ptr(), 1025, x.data_ptr() + 8 * 4096, 1025, 0)
    assert e.value.code == C.EINVAL
