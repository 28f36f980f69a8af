"""GPU checks of NEUMANN_FLAG_SYMMETRIC: for symmetric A every matrix of the
scheme is a polynomial in A and so symmetric; the products compute only the
tiles on or above the diagonal (256 x 256 CTA pairs for the split dtypes,
128 x 128 SIMT tiles for FP64 / FP32) and write their transposes.

Checked against the closed form at orders with ragged tiles and at full
tiles, for exact symmetry of S, against the general path, with a strided
output, for the general product call of a symmetric plan (operands need not
be symmetric there), and for a grouped batch (which ignores the flag).
"""

import numpy as np
import pytest

from oracle import closed_form as CF
from oracle import evaluate as EV
from workloads import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"split_bf16": 1e-3, "split_fp16": 3e-4}  # rho = 0.9, as for the general path at n = 4096


def _nm():
    import paper_2602_11843_gb300 as nm

    return nm


def _eval(A_np, k, radix, dtype, flags, out=None):
    nm = _nm()
    p = nm.Plan(A_np.shape[0], k, radix, dtype, flags)
    A = torch.tensor(A_np, device="cuda")
    S = p(A, out=out)
    torch.cuda.synchronize()
    assert p.status() == 0
    return S, p


@pytest.mark.parametrize("dtype", ["split_bf16", "split_fp16"])
@pytest.mark.parametrize("n,radix,k", [(300, 9, 81), (1000, 15, 225), (4000, 9, 729), (4096, 15, 225)])
def test_symmetric_matches_closed_form(dtype, n, radix, k):
    nm = _nm()
    pl = G.config_inputs(2, n=n)
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix)
    S_sym, p = _eval(pl["A"], k, radix, dtype, nm.FLAG_SYMMETRIC)
    assert p.info["tile_pair"] == 1
    S_gen, _ = _eval(pl["A"], k, radix, dtype, 0)
    e_sym = CF.rel_fro(S_sym.cpu().numpy(), ref)
    e_gen = CF.rel_fro(S_gen.cpu().numpy(), ref)
    print(f"n={n} radix {radix} k {k} {dtype}: symmetric {e_sym:.3e} general {e_gen:.3e}")
    assert torch.equal(S_sym, S_sym.T)
    assert e_sym < TOL[dtype] and e_sym < 2 * e_gen + 1e-6


@pytest.mark.parametrize("dtype,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("n,radix,k", [(300, 9, 81), (1000, 15, 225), (1024, 2, 256)])
def test_symmetric_simt_paths(dtype, tol, n, radix, k):
    """FP64 and FP32: 128 x 128 SIMT tiles on or above the diagonal."""
    nm = _nm()
    pl = G.config_inputs(2, n=n)
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix)
    p = nm.Plan(n, k, radix, dtype, nm.FLAG_SYMMETRIC)
    A = torch.tensor(pl["A"], dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    assert p.status() == 0
    assert torch.equal(S, S.T)
    err = CF.rel_fro(S.double().cpu().numpy(), ref)
    print(f"n={n} radix {radix} k {k} {dtype} symmetric: {err:.3e}")
    assert err < tol


def test_symmetric_strided_output():
    nm = _nm()
    n, ld = 1000, 1032
    pl = G.config_inputs(2, n=n)
    big = torch.full((n + 4, ld), 3.0, dtype=torch.float64, device="cuda")
    out = big[:n, :n]
    S, _ = _eval(pl["A"], 81, 9, "split_bf16", nm.FLAG_SYMMETRIC, out=out)
    assert torch.all(big[:n, n:] == 3.0) and torch.all(big[n:, :] == 3.0)
    assert torch.equal(out, out.T)
    ref = EV.planted_reference(pl["V"], pl["lam"], 81, 9)
    assert CF.rel_fro(out.cpu().numpy(), ref) < TOL["split_bf16"]


def test_symmetric_plan_product_call_is_general():
    """neumann_plan_matmul of a symmetric plan multiplies any A and B."""
    nm = _nm()
    n = 1000
    rng = np.random.default_rng(17)
    A_np, B_np = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    p = nm.Plan(n, 81, 9, "split_bf16", nm.FLAG_SYMMETRIC)
    C = p.matmul(torch.tensor(A_np, device="cuda"), torch.tensor(B_np, device="cuda"))
    torch.cuda.synchronize()
    ref = A_np @ B_np
    assert CF.rel_fro(C.cpu().numpy(), ref) < 2e-5


def test_symmetric_flag_ignored_by_grouped_batch():
    nm = _nm()
    mats = G.jacobi_batch(20, 4002, sizes=(16, 48, 128, 256))  # not symmetric
    bp = nm.BatchedPlan(len(mats), 256, 81, 9, "split_bf16", nm.FLAG_SYMMETRIC)
    As = [torch.tensor(m["A"], device="cuda") for m in mats]
    outs = bp(As)
    torch.cuda.synchronize()
    assert bp.status() == 0
    for m, o in zip(mats, outs):
        ref, _ = EV.evaluate(m["A"], 81, 9)
        assert CF.rel_fro(o.cpu().numpy(), ref) < 2e-3


def test_symmetric_and_precise_together_not_supported():
    nm = _nm()
    with pytest.raises(nm.NeumannError) as e:
        nm.Plan(1024, 81, 9, "split_bf16", nm.FLAG_SYMMETRIC | nm.FLAG_PRECISE_ACC)
    assert e.value.code == nm.ENOTSUP


@pytest.mark.parametrize("dtype", ["split_bf16", "split_fp16"])
def test_symmetric_cfg3_full(dtype):
    """The n = 8192 precision workload (radix 15, k = 3375, rho 0.97), symmetric path."""
    nm = _nm()
    pl = G.config_inputs(3)
    ref = EV.planted_reference(pl["V"], pl["lam"], 3375, 15)
    S, _ = _eval(pl["A"], 3375, 15, dtype, nm.FLAG_SYMMETRIC)
    err = CF.rel_fro(S.cpu().numpy(), ref)
    print(f"cfg3 symmetric {dtype} rel err {err:.3e}")
    assert torch.equal(S, S.T) and err < 3e-3


@pytest.mark.parametrize("dtype", ["split_bf16", "fp64"])
@pytest.mark.parametrize("radix,k,extra", [(1, 81, 0), (2, 64, 0), (2, 81, "exact"), (3, 27, 0), (5, 125, 0),
                                           (0, 360, 0), (9, 81, "paper"), (15, 225, "printed"),
                                           (9, 729, "io32")])
def test_symmetric_every_scheme(dtype, radix, k, extra):
    """Every scheme and the flags that change the ops (exact-k binary, the
    paper-form residual, printed radix-15 coefficients, FP32 input/output)."""
    nm = _nm()
    flags = nm.FLAG_SYMMETRIC | {0: 0, "exact": nm.FLAG_EXACT_K, "paper": nm.FLAG_RESIDUAL_PAPER,
                                 "printed": nm.FLAG_PRINTED_COEFFS, "io32": nm.FLAG_IO_FP32}[extra]
    if extra == "io32" and dtype == "fp64":
        flags &= ~nm.FLAG_IO_FP32
    pl = G.config_inputs(2, n=300)
    coef = "printed" if extra == "printed" else "refined"
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix, coef15=coef)
    p = nm.Plan(300, k, radix, dtype, flags)
    A = torch.tensor(pl["A"], dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    assert p.status() == 0
    assert torch.equal(S, S.T)
    err = CF.rel_fro(S.double().cpu().numpy(), ref)
    assert err < (1e-12 if dtype == "fp64" else 1e-3), err
