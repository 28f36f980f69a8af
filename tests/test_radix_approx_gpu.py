"""GPU parity of the approximate-prefix five-product kernels (radix 27, 31, 33;
App. C, Table approx) inside the residual framework, against the oracle's
framework value (Lemma 5.7) for the same published circuits. Spectra stay in
each kernel's convergence region (radix 33: eigenvalues above -0.925).
Tolerances as tests/test_radix_p5_gpu.py.
"""

import pytest

from oracle import closed_form as CF
from oracle import evaluate as EV
from workloads import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
TOL_BF16 = {0.5: 2e-4, 0.9: 1e-3}
TOL_FP16 = {0.5: 1e-5, 0.9: 5e-5}
DTYPES = ["fp64", "fp32", "split_bf16", "split_fp16"]


def _tol(dtype, rho):
    if dtype in TOL:
        return TOL[dtype]
    return TOL_FP16[rho] if dtype == "split_fp16" else TOL_BF16[rho]


def _run(A_np, k, radix, dtype):
    import paper_2602_11843_gb300 as nm

    p = nm.Plan(A_np.shape[0], k, radix, dtype)
    A = torch.tensor(A_np, dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    return S.double().cpu().numpy(), p.status(), p


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("radix", [27, 31, 33])
@pytest.mark.parametrize("t", [1, 2])
def test_approx_kernel_planted(dtype, radix, t):
    pl = G.planted_symmetric(300, 0.9, 300 + radix)
    k = radix ** t
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix)
    S, st, p = _run(pl["A"], k, radix, dtype)
    assert st == 0
    assert p.info["products_executed"] == 7 * t - 2
    assert CF.rel_fro(S, ref) < _tol(dtype, 0.9)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("radix", [27, 31, 33])
def test_approx_kernel_nonsymmetric(dtype, radix):
    g = G.gaussian_scaled(200, 0.5, 40 + radix)
    ref, _ = EV.evaluate(g["A"], radix * radix, radix)
    S, st, _ = _run(g["A"], radix * radix, radix, dtype)
    assert st == 0
    assert CF.rel_fro(S, ref) < _tol(dtype, 0.5)


@pytest.mark.parametrize("dtype", ["fp32", "split_bf16"])
def test_approx_kernel_grouped_and_resident_batch(dtype):
    import paper_2602_11843_gb300 as nm

    mats = G.jacobi_batch(24, 77, sizes=(16, 40, 96, 200))
    io = torch.float32 if dtype == "fp32" else torch.float64
    bp = nm.BatchedPlan(len(mats), 256, 31 * 31, 31, dtype)
    outs = bp([torch.tensor(m["A"], dtype=io, device="cuda") for m in mats])
    torch.cuda.synchronize()
    assert bp.status() == 0
    tol = 1e-5 if dtype == "fp32" else 1e-4
    for m, S in zip(mats, outs):
        ref, _ = EV.evaluate(m["A"], 31 * 31, 31)
        assert CF.rel_fro(S.double().cpu().numpy(), ref) < tol, m["n"]
