"""GPU parity of the five-product approximate kernels (radix 24 and 25).

Each level runs five products (the third product's epilogue writes five
outputs, among them the parts of the fifth factors over I, B, P1, P2, P3),
then the concatenation and residual products of the framework (Sec. 5.3). The reference is the oracle's
result for the same scheme: Lemma 5.7's closed form on planted symmetric
spectra, and the matrix iteration for other inputs. Tolerances are those of
the other schemes at the same spectral radius (test_parity_gpu.py).
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
DTYPES = ["fp64", "fp32", "split_bf16", "split_fp16"]


def _nm():
    import paper_2602_11843_gb300 as nm

    return nm


def _tol(dtype, rho):
    if dtype in TOL:
        return TOL[dtype]
    return TOL_FP16[rho] if dtype == "split_fp16" else TOL_BF16[rho]


def _run(A_np, k, radix, dtype, flags=0):
    nm = _nm()
    p = nm.Plan(A_np.shape[0], k, radix, dtype, flags)
    A = torch.tensor(A_np, dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    return S.double().cpu().numpy(), p.status(), p


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("radix,k", [(24, 24), (24, 576), (25, 25), (25, 625)])
@pytest.mark.parametrize("n", [200, 300])
def test_p5_parity_planted(dtype, radix, k, n):
    pl = G.planted_symmetric(n, 0.9, 100 + n)
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix)
    S, st, p = _run(pl["A"], k, radix, dtype)
    assert st == 0
    assert p.info["products_executed"] == 7 * len(p.info["levels"]) - 2
    err = CF.rel_fro(S, ref)
    assert err < _tol(dtype, 0.9), err


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("radix", [24, 25])
def test_p5_nonsymmetric(dtype, radix):
    """Gaussian input, ||A||_2 = 0.5, against the oracle's matrix iteration."""
    g = G.gaussian_scaled(300, 0.5, 7)
    ref, _ = EV.evaluate(g["A"], radix * radix, radix)
    S, st, _ = _run(g["A"], radix * radix, radix, dtype)
    assert st == 0
    assert CF.rel_fro(S, ref) < _tol(dtype, 0.5)


@pytest.mark.parametrize("dtype", ["fp64", "split_bf16"])
def test_p5_paper_residual_form(dtype):
    """R' = I - (I - A) Y' (eq. generalradix) gives the same Y_t (Lemma 5.7)."""
    nm = _nm()
    pl = G.planted_symmetric(300, 0.9, 5)
    ref = EV.planted_reference(pl["V"], pl["lam"], 625, 25)
    S, st, _ = _run(pl["A"], 625, 25, dtype, nm.FLAG_RESIDUAL_PAPER)
    assert st == 0 and CF.rel_fro(S, ref) < _tol(dtype, 0.9)


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "split_bf16"])
@pytest.mark.parametrize("radix,n", [(24, 300), (25, 1000)])
def test_p5_symmetric_flag(dtype, radix, n):
    nm = _nm()
    pl = G.config_inputs(2, n=n)
    k = radix * radix
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix)
    S, st, _ = _run(pl["A"], k, radix, dtype, nm.FLAG_SYMMETRIC)
    assert st == 0
    assert np.array_equal(S, S.T)
    assert CF.rel_fro(S, ref) < _tol(dtype, 0.9)


@pytest.mark.parametrize("dtype", ["split_bf16", "split_fp16"])
def test_p5_precise_and_io_fp32(dtype):
    """NEUMANN_FLAG_PRECISE_ACC (chunked accumulation) and FLAG_IO_FP32 (float A and S)."""
    nm = _nm()
    pl = G.planted_symmetric(1000, 0.9, 21)
    ref = EV.planted_reference(pl["V"], pl["lam"], 625, 25)
    S, st, _ = _run(pl["A"], 625, 25, dtype, nm.FLAG_PRECISE_ACC)
    assert st == 0 and CF.rel_fro(S, ref) < _tol(dtype, 0.9)
    S, st, p = _run(pl["A"], 625, 25, dtype, nm.FLAG_IO_FP32)
    assert p.io_dtype == torch.float32
    assert st == 0 and CF.rel_fro(S, ref) < max(_tol(dtype, 0.9), 1e-5)


@pytest.mark.parametrize("n,k,radix", [(1, 24, 24), (17, 25, 25), (33, 625, 25), (129, 576, 24)])
@pytest.mark.parametrize("dtype", DTYPES)
def test_p5_edge_sizes(n, k, radix, dtype):
    g = G.gaussian_scaled(n, 0.5, 11)
    ref, _ = EV.evaluate(g["A"], k, radix)
    S, st, _ = _run(g["A"], k, radix, dtype)
    assert st == 0
    assert CF.rel_fro(S, ref) < _tol(dtype, 0.5)


BATCH_TOL = {"fp64": 1e-12, "fp32": 1e-5, "split_bf16": 2e-3, "split_fp16": 5e-5}


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("radix,k", [(24, 576), (25, 625)])
def test_p5_batched_grouped(dtype, radix, k):
    """Grouped launches over damped-Jacobi matrices of mixed order (cfg-4 construction)."""
    nm = _nm()
    mats = G.jacobi_batch(20, 4001, sizes=(16, 48, 128, 144, 256))
    mats += [{"n": n, "A": G.gaussian_scaled(n, 0.5, 50 + n)["A"]} for n in (1, 17, 129)]
    bp = nm.BatchedPlan(len(mats), 256, k, radix, dtype)
    dt = torch.float32 if dtype == "fp32" else torch.float64
    outs = bp([torch.tensor(m["A"], dtype=dt, device="cuda") for m in mats])
    torch.cuda.synchronize()
    assert bp.status() == 0
    for m, o in zip(mats, outs):
        ref, _ = EV.evaluate(m["A"], k, radix)
        err = CF.rel_fro(o.double().cpu().numpy(), ref)
        assert err < BATCH_TOL[dtype], (m["n"], err)


def test_p5_timing_counts_products():
    nm = _nm()
    pl = G.planted_symmetric(512, 0.9, 9)
    _, st, p = _run(pl["A"], 15625, 25, "split_bf16", nm.FLAG_TIMING)
    t = p.timing()
    assert st == 0 and len(t) == p.info["products_executed"] == 19 and all(x > 0 for x in t)


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_p5_cfg2_full(dtype):
    """n = 4096, spectrum in [-0.9, 0.9], radix 24, k = 576."""
    pl = G.config_inputs(2)
    ref = EV.planted_reference(pl["V"], pl["lam"], 576, 24)
    S, st, _ = _run(pl["A"], 576, 24, dtype)
    assert st == 0 and CF.rel_fro(S, ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", ["split_bf16", "split_fp16"])
def test_p5_cfg3_full(dtype):
    """n = 8192, spectrum in [-0.97, 0.97], radix 25, k = 15625 (three levels, 19 products)."""
    pl = G.config_inputs(3)
    ref = EV.planted_reference(pl["V"], pl["lam"], 15625, 25)
    S, st, _ = _run(pl["A"], 15625, 25, dtype)
    assert st == 0
    err = CF.rel_fro(S, ref)
    print(f"cfg3 radix 25 k 15625 {dtype} rel err {err:.3e}")
    assert err < _tol(dtype, 0.97)
