"""The allocation-free product, neumann_matmul_noalloc, against the plan-based
product it mirrors (neumann_plan_matmul on a SPLIT_BF16 plan).

Some callers cannot allocate device memory where they need a product: code
running under an allocator that owns all device memory, or a loop that cannot
take the synchronisation cudaFree implies. The allocation-free call serves them
from a fixed array inside the library, shared by every call, so the tests make
calls in a row with different inputs and sizes and check that a call is not
affected by what an earlier one left behind; they also check its edge orders
(1 and the 1024 limit), leading dimensions above n, its status word, and that a
call made after set-up changes no device memory figure. This file is collected
last so that a run stopping at the first failure has already run every other test.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 2e-5  # the split-BF16 product tolerance of tests/test_parity_gpu.py


def _rel(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _mats(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n)), rng.standard_normal((n, n))


def test_noalloc_matches_plan_matmul_on_two_calls():
    import paper_2602_11843_gb300 as nm
    from paper_2602_11843_gb300 import _capi as C

    stream = _stream()
    for call, n in enumerate((1000, 300)):  # larger first: the second call reuses a dirtier array
        a_np, b_np = _mats(n, 100 + call)
        A = torch.tensor(a_np, dtype=torch.float64, device="cuda")
        B = torch.tensor(b_np, dtype=torch.float64, device="cuda")
        out_na = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        C.neumann_matmul_noalloc(n, A.data_ptr(), n, B.data_ptr(), n, out_na.data_ptr(), n, stream)
        plan = nm.Plan(n, 2, 2, "split_bf16")
        out_plan = plan.matmul(A, B)
        torch.cuda.synchronize()
        assert C.neumann_matmul_noalloc_status(stream) == 0
        a, b = out_na.cpu().numpy(), out_plan.cpu().numpy()
        ref = a_np @ b_np
        assert np.isfinite(a).all()
        assert _rel(a, b) < TOL, f"call {call}: differs from neumann_plan_matmul"
        assert _rel(a, ref) < TOL, f"call {call}: differs from the FP64 product"


@pytest.mark.parametrize("n,lda,ldb,ldc", [(1, 1, 1, 1), (1024, 1024, 1024, 1024), (300, 333, 301, 320),
                                           (1, 3, 2, 5), (1024, 1040, 1031, 1027)])
def test_noalloc_edge_orders_and_leading_dimensions(n, lda, ldb, ldc):
    """Orders 1 and 1024 (the limit of the fixed array), and strided operands:
    C inside the n x n block equals the FP64 product and the plan's product of
    the same matrices; the elements between n and ldc in each row are untouched."""
    import paper_2602_11843_gb300 as nm
    from paper_2602_11843_gb300 import _capi as C

    stream = _stream()
    a_np, b_np = _mats(n, 7 * n + lda)
    A = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
    B = torch.zeros((n, ldb), dtype=torch.float64, device="cuda")
    A[:, :n] = torch.from_numpy(a_np)
    B[:, :n] = torch.from_numpy(b_np)
    Cm = torch.full((n, ldc), 7.0, dtype=torch.float64, device="cuda")
    C.neumann_matmul_noalloc(n, A.data_ptr(), lda, B.data_ptr(), ldb, Cm.data_ptr(), ldc, stream)
    out_plan = nm.Plan(n, 2, 2, "split_bf16").matmul(A[:, :n].contiguous(), B[:, :n].contiguous())
    torch.cuda.synchronize()
    assert C.neumann_matmul_noalloc_status(stream) == 0
    got = Cm.cpu().numpy()
    ref = a_np @ b_np
    assert _rel(got[:, :n], ref) < TOL
    assert _rel(got[:, :n], out_plan.cpu().numpy()) < TOL
    assert (got[:, n:] == 7.0).all(), "wrote past n in a row of C"


def test_noalloc_reports_nonfinite_through_its_status_word():
    from paper_2602_11843_gb300 import _capi as C

    stream = _stream()
    n = 64
    a_np, b_np = _mats(n, 5)
    a_np[3, 4] = np.inf
    A = torch.tensor(a_np, dtype=torch.float64, device="cuda")
    B = torch.tensor(b_np, dtype=torch.float64, device="cuda")
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    assert C.neumann_matmul_noalloc_status(stream) == 0
    C.neumann_matmul_noalloc(n, A.data_ptr(), n, B.data_ptr(), n, out.data_ptr(), n, stream)
    assert C.neumann_matmul_noalloc_status(stream) & C.STATUS_NONFINITE
    assert C.neumann_matmul_noalloc_status(stream) == 0, "the read clears the word"
    A[3, 4] = 0.0
    C.neumann_matmul_noalloc(n, A.data_ptr(), n, B.data_ptr(), n, out.data_ptr(), n, stream)
    assert C.neumann_matmul_noalloc_status(stream) == 0


def test_noalloc_call_after_setup_changes_no_device_memory():
    """After one set-up call (which loads the library's device code), a call of
    another order moves neither the device's free memory nor torch's allocator."""
    from paper_2602_11843_gb300 import _capi as C

    stream = _stream()
    tensors = {}
    for n in (900, 200):
        a_np, b_np = _mats(n, n)
        tensors[n] = (torch.tensor(a_np, dtype=torch.float64, device="cuda"),
                      torch.tensor(b_np, dtype=torch.float64, device="cuda"),
                      torch.empty((n, n), dtype=torch.float64, device="cuda"), a_np @ b_np)
    A, B, out, _ = tensors[900]
    C.neumann_matmul_noalloc(900, A.data_ptr(), 900, B.data_ptr(), 900, out.data_ptr(), 900, stream)
    assert C.neumann_matmul_noalloc_status(stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    A, B, out, ref = tensors[200]
    C.neumann_matmul_noalloc(200, A.data_ptr(), 200, B.data_ptr(), 200, out.data_ptr(), 200, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0, f"device free memory moved by {free0 - free1} bytes"
    for key in ("allocation.all.allocated", "num_alloc_retries", "segment.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    assert _rel(out.cpu().numpy(), ref) < TOL


def test_noalloc_rejects_orders_above_its_scratch():
    from paper_2602_11843_gb300 import _capi as C

    x = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(C.NeumannError) as e:
        C.neumann_matmul_noalloc(1025, x.data_ptr(), 1025, x.data_ptr(), 1025, x.data_ptr() + 8 * 4096, 1025, 0)
    assert e.value.code == C.EINVAL
