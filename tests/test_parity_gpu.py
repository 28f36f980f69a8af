"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative Frobenius error against the oracle result of the same
scheme: S_k for exact schemes, Lemma 5.7's closed form for radix 15):
  FP64        1e-12
  FP32        1e-5
  split-BF16  TOL_BF16[rho]; each operand is kept to ~2^-17 relative, so a
              product carries ~1e-5 relative error, amplified by ||S|| <= 1/(1-rho)
              across levels.
  split-FP16  TOL_FP16[rho]; operands kept to ~2^-22 relative (each matrix stored
              as x * 2^e with its own e, which keeps hi in range and lo normal
              down to ~2^-17 of the matrix's bound), the same amplification. A product's
              FP32 accumulation on the tensor cores is biased toward zero by about
              (3n/16)/4 ulp of the sum (one truncating update per MMA; 2e-6 at
              n = 513, 3-5e-5 at n = 8192), which at n = 8192 exceeds both operand
              errors: there both splits end near 1e-3 (rho = 0.97).
"""

import numpy as np
import pytest

from oracle import closed_form as CF
from oracle import evaluate as EV
from workloads import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
TOL_BF16 = {0.5: 2e-4, 0.9: 1e-3, 0.97: 3e-3}
TOL_FP16 = {0.5: 1e-5, 0.9: 5e-5, 0.97: 3e-3}


def _nm():
    import paper_2602_11843_gb300 as nm

    return nm


def _tol(dtype, rho):
    if dtype in TOL:
        return TOL[dtype]
    return TOL_FP16[rho] if dtype == "split_fp16" else TOL_BF16[rho]


def _run(A_np, k, radix, dtype, flags=0):
    nm = _nm()
    n = A_np.shape[0]
    p = nm.Plan(n, k, radix, dtype, flags)
    A = torch.tensor(A_np, dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    st = p.status()
    return S.double().cpu().numpy(), st, p


# ---------------------------------------------------------------- products

@pytest.mark.parametrize("dtype,tol", [("fp64", 1e-14), ("fp32", 2e-6), ("split_bf16", 2e-5), ("split_fp16", 5e-6)])
@pytest.mark.parametrize("n", [1, 17, 200, 256, 300, 513])
def test_matmul_against_fp64_reference(dtype, tol, n):
    """C = A B of each arithmetic against an FP64 product (torch on the CPU)."""
    nm = _nm()
    rng = np.random.default_rng(n)
    A_np, B_np = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    p = nm.Plan(n, 2, 2, dtype)
    A = torch.tensor(A_np, dtype=p.io_dtype, device="cuda")
    B = torch.tensor(B_np, dtype=p.io_dtype, device="cuda")
    C = p.matmul(A, B)
    torch.cuda.synchronize()
    ref = (A.double().cpu() @ B.double().cpu()).numpy()
    assert p.status() == 0
    assert CF.rel_fro(C.double().cpu().numpy(), ref) < tol


# ---------------------------------------------------------------- schemes, small n

SCHEMES = [(1, 81, 0), (2, 64, 0), (2, 81, 1), (3, 27, 0), (5, 125, 0), (9, 81, 0), (9, 729, 0),
           (15, 225, 0), (15, 3375, 0), (0, 360, 0)]


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "split_bf16", "split_fp16"])
@pytest.mark.parametrize("radix,k,exact", SCHEMES)
@pytest.mark.parametrize("n", [200, 300])
def test_scheme_parity_planted(dtype, radix, k, exact, n):
    nm = _nm()
    rho = 0.9
    pl = G.planted_symmetric(n, rho, 100 + n)
    ref = EV.planted_reference(pl["V"], pl["lam"], k, 15 if radix == 15 else 1)
    S, st, p = _run(pl["A"], k, radix, dtype, nm.FLAG_EXACT_K if exact else 0)
    assert st == 0
    assert CF.rel_fro(S, ref) < _tol(dtype, rho)


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "split_bf16", "split_fp16"])
@pytest.mark.parametrize("radix,k,exact", [(1, 81, 0), (2, 128, 0), (2, 81, 1), (9, 81, 0), (15, 225, 0)])
def test_scheme_parity_nonsymmetric(dtype, radix, k, exact):
    """Nonsymmetric Gaussian input (||A||_2 = 0.5) against the oracle's matrix schemes."""
    nm = _nm()
    g = G.gaussian_scaled(300, 0.5, 7)
    ref, _ = EV.evaluate(g["A"], k, radix)
    S, st, _ = _run(g["A"], k, radix, dtype, nm.FLAG_EXACT_K if exact else 0)
    assert st == 0
    assert CF.rel_fro(S, ref) < _tol(dtype, 0.5)


@pytest.mark.parametrize("n,k,radix", [(1, 81, 9), (1, 5, 1), (17, 1, 9), (17, 2, 1), (17, 2, 2), (17, 9, 9),
                                       (33, 15, 15), (5, 7, 2)])
@pytest.mark.parametrize("dtype", ["fp64", "fp32", "split_bf16", "split_fp16"])
def test_edge_cases(n, k, radix, dtype):
    nm = _nm()
    g = G.gaussian_scaled(n, 0.5, 11)
    ref, _ = EV.evaluate(g["A"], k, radix)
    S, st, _ = _run(g["A"], k, radix, dtype, nm.FLAG_EXACT_K if radix == 2 else 0)
    assert st == 0
    assert CF.rel_fro(S, ref) < _tol(dtype, 0.5)


def test_residual_paper_form_and_printed_coefficients():
    nm = _nm()
    pl = G.planted_symmetric(256, 0.9, 5)
    ref = EV.planted_reference(pl["V"], pl["lam"], 225, 15)
    S, st, _ = _run(pl["A"], 225, 15, "fp64", nm.FLAG_RESIDUAL_PAPER)
    assert st == 0 and CF.rel_fro(S, ref) < 1e-12
    refp = EV.planted_reference(pl["V"], pl["lam"], 225, 15, coef15="printed")
    S, st, _ = _run(pl["A"], 225, 15, "fp64", nm.FLAG_PRINTED_COEFFS)
    assert st == 0 and CF.rel_fro(S, refp) < 1e-12


def test_leading_dimensions_and_io_fp32():
    nm = _nm()
    g = G.gaussian_scaled(100, 0.5, 3)
    ref, _ = EV.evaluate(g["A"], 81, 9)
    p = nm.Plan(100, 81, 9, "fp64")
    big = torch.zeros((100, 160), dtype=torch.float64, device="cuda")
    big[:, :100] = torch.tensor(g["A"], device="cuda")
    out = torch.full((100, 130), 7.0, dtype=torch.float64, device="cuda")
    nm.neumann_eval(p.handle, big.data_ptr(), 160, out.data_ptr(), 130, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert CF.rel_fro(out[:, :100].cpu().numpy(), ref) < 1e-12
    assert bool((out[:, 100:] == 7.0).all())  # nothing written past n
    S, st, _ = _run(g["A"], 81, 9, "split_bf16", nm.FLAG_IO_FP32)
    assert st == 0 and CF.rel_fro(S, ref) < 2e-4


@pytest.mark.parametrize("dtype", ["fp64", "split_bf16", "split_fp16"])
@pytest.mark.parametrize("n,lda,offset", [(100, 161, 0), (100, 160, 1), (101, 104, 0), (101, 101, 0)])
def test_split_of_a_alignment(dtype, n, lda, offset):
    """The first element-wise pass reads the caller's A as 4-wide vectors when its base
    and row stride are multiples of 16 bytes, and element by element otherwise (odd
    stride, base one element in). Odd n leaves a ragged run at the end of each row."""
    nm = _nm()
    g = G.gaussian_scaled(n, 0.5, 30 + n)
    ref, _ = EV.evaluate(g["A"], 81, 9)
    p = nm.Plan(n, 81, 9, dtype)
    flat = torch.zeros(offset + n * lda + 8, dtype=torch.float64, device="cuda")
    view = flat[offset:offset + n * lda].view(n, lda)
    view[:, :n] = torch.tensor(g["A"], device="cuda")
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    nm.neumann_eval(p.handle, view.data_ptr(), lda, out.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert p.status() == 0
    assert CF.rel_fro(out.cpu().numpy(), ref) < _tol(dtype, 0.5)
    # the same arithmetic on either read path: bit-identical to a contiguous, aligned A
    S = p(torch.tensor(g["A"], device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(S, out)


def test_nonfinite_status_for_divergent_input():
    """Undamped Jacobi splitting has rho(A) > 1; S_k overflows and the epilogue
    reports NEUMANN_STATUS_NONFINITE instead of trapping."""
    nm = _nm()
    m = G.jacobi_batch(1, 4, sizes=(64,), damped=False)[0]
    for dtype in ("fp32", "split_bf16", "split_fp16"):
        S, st, _ = _run(m["A"], 15 ** 3, 15, dtype)
        assert st & nm.STATUS_NONFINITE, dtype


def test_fp16_split_scales_large_entries():
    """A nilpotent A (rho = 0, A^2 = 0) with entries of 300 and 3e6: far outside
    FP16's range, but every split-FP16 matrix is stored with its own power of
    two (the bound on max |x| mapped to <= 2^14), so S = I + A comes out exact,
    as with the BF16 split (FP32 exponent range)."""
    A = np.zeros((16, 16))
    A[0, 1] = 300.0
    A[2, 5] = 3.0e6
    for dtype in ("split_fp16", "split_bf16"):
        S, st, _ = _run(A, 81, 9, dtype)
        assert st == 0 and CF.rel_fro(S, np.eye(16) + A) < 1e-12, dtype


def test_timing_flag_reports_every_product():
    nm = _nm()
    pl = G.planted_symmetric(512, 0.9, 9)
    _, st, p = _run(pl["A"], 225, 15, "split_bf16", nm.FLAG_TIMING)
    t = p.timing()
    assert len(t) == p.info["products_executed"] == 10 and all(x > 0 for x in t)


BATCH_TOL = {"fp64": 1e-12, "fp32": 1e-5, "split_bf16": 2e-3, "split_fp16": 5e-5}


def _batch_check(bp, mats, k, radix, dtype):
    dt = torch.float32 if dtype == "fp32" else torch.float64
    As = [torch.tensor(m["A"], dtype=dt, device="cuda") for m in mats]
    outs = bp(As)
    torch.cuda.synchronize()
    assert bp.status() == 0
    for m, o in zip(mats, outs):
        ref, _ = EV.evaluate(m["A"], k, radix)
        err = CF.rel_fro(o.double().cpu().numpy(), ref)
        assert err < BATCH_TOL[dtype], (m["n"], err)


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "split_bf16", "split_fp16"])
@pytest.mark.parametrize("k,radix", [(81, 9), (225, 15), (64, 2), (81, 1)])
def test_batched_grouped_matches_oracle(dtype, k, radix):
    """Grouped launches over damped-Jacobi matrices of mixed order (cfg-4 construction)."""
    nm = _nm()
    mats = G.jacobi_batch(20, 4001, sizes=(16, 48, 128, 144, 256))
    mats += [{"n": n, "A": G.gaussian_scaled(n, 0.5, 50 + n)["A"]} for n in (1, 17, 129)]
    bp = nm.BatchedPlan(len(mats), 256, k, radix, dtype)
    _batch_check(bp, mats, k, radix, dtype)


def test_batched_reuses_dirty_slabs():
    """A second call with smaller matrices on slabs that held larger ones: every
    buffer a product reads is rewritten up to its K padding."""
    nm = _nm()
    for dtype in ("fp32", "split_bf16"):
        bp = nm.BatchedPlan(6, 256, 81, 9, dtype)
        big = [{"n": 256, "A": G.gaussian_scaled(256, 0.5, 60 + i)["A"]} for i in range(6)]
        _batch_check(bp, big, 81, 9, dtype)
        small = [{"n": n, "A": G.gaussian_scaled(n, 0.5, 70 + n)["A"]} for n in (5, 16, 31, 33, 100, 200)]
        _batch_check(bp, small, 81, 9, dtype)


def test_batched_more_than_one_chunk():
    nm = _nm()
    mats = [{"n": 16, "A": G.gaussian_scaled(16, 0.5, 9000 + i)["A"]} for i in range(2100)]
    bp = nm.BatchedPlan(len(mats), 16, 81, 9, "split_bf16")
    dt = torch.float64
    As = [torch.tensor(m["A"], dtype=dt, device="cuda") for m in mats]
    outs = bp(As)
    torch.cuda.synchronize()
    assert bp.status() == 0
    for i in (0, 1, 1000, 2047, 2048, 2099):
        ref, _ = EV.evaluate(mats[i]["A"], 81, 9)
        assert CF.rel_fro(outs[i].cpu().numpy(), ref) < BATCH_TOL["split_bf16"]


def test_batched_large_orders_fall_back_per_matrix():
    nm = _nm()
    mats = [{"n": n, "A": G.gaussian_scaled(n, 0.5, 80 + n)["A"]} for n in (300, 40)]
    bp = nm.BatchedPlan(2, 300, 81, 9, "fp32")
    _batch_check(bp, mats, 81, 9, "fp32")


# ---------------------------------------------------------------- full-size workloads

def test_cfg1_full():
    """n = 256, k = 81, ||A||_2 = 0.5: naive, squaring to 2^7, exact-k binary and radix 9, FP64."""
    nm = _nm()
    g = G.config_inputs(1)
    for radix, k, fl in ((1, 81, 0), (2, 128, 0), (2, 81, nm.FLAG_EXACT_K), (9, 81, 0)):
        ref, _ = EV.evaluate(g["A"], k, radix)
        S, st, _ = _run(g["A"], k, radix, "fp64", fl)
        assert st == 0 and CF.rel_fro(S, ref) < 1e-12
        # (I - A) S_k = I - A^k
        I = np.eye(256)
        lhs = (I - g["A"]) @ S
        rhs = I - np.linalg.matrix_power(g["A"], k)
        assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(rhs)


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
@pytest.mark.parametrize("radix,k", [(9, 729), (15, 225)])
def test_cfg2_full(dtype, radix, k):
    pl = G.config_inputs(2)
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix)
    S, st, _ = _run(pl["A"], k, radix, dtype)
    assert st == 0 and CF.rel_fro(S, ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", ["split_bf16", "split_fp16"])
@pytest.mark.parametrize("radix,k", [(15, 3375), (9, 6561)])
def test_cfg3_full_split(radix, k, dtype):
    pl = G.config_inputs(3)
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix)
    S, st, _ = _run(pl["A"], k, radix, dtype)
    assert st == 0
    err = CF.rel_fro(S, ref)
    print(f"cfg3 radix {radix} k {k} {dtype} rel err {err:.3e}")
    assert err < _tol(dtype, 0.97)
