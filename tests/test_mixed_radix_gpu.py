"""GPU parity of mixed-radix schedules with approximate levels (radix 0 with
NEUMANN_FLAG_ALLOW_APPROX) against the oracle's residual framework on the
plan's own level sequence (Sec. 5.3, eq. generalradix; Lemma 5.7 level by
level), through the C ABI.

  k = 135    = 9 . 15         levels [9, 15]
  k = 450    = 2 . 15 . 15    levels [2, 15, 15]
  k = 30375  = 9 . 15^3       levels [9, 15, 15, 15]

Tolerances as tests/test_parity_gpu.py: FP64 1e-12, FP32 1e-5, split forms by rho.
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


def _plan(n, k, dtype, flags=0):
    import paper_2602_11843_gb300 as nm

    return nm.Plan(n, k, 0, dtype, nm.FLAG_ALLOW_APPROX | flags)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("k,levels", [(135, [9, 15]), (450, [2, 15, 15]), (30375, [9, 15, 15, 15])])
def test_mixed_nonsymmetric_against_matrix_oracle(dtype, k, levels):
    g = G.gaussian_scaled(200, 0.5, 31)
    p = _plan(200, k, dtype)
    assert p.info["levels"] == levels
    ref, prods = EV.evaluate(g["A"], k, 0, levels=levels, form="error-map")
    assert p.info["products_executed"] == prods
    A = torch.tensor(g["A"], dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    assert p.status() == 0
    assert CF.rel_fro(S.double().cpu().numpy(), ref) < _tol(dtype, 0.5)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("k", [135, 450, 30375])
@pytest.mark.parametrize("n", [300, 513])
def test_mixed_planted_against_closed_form(dtype, k, n):
    """Planted spectrum |l| <= 0.9 against Lemma 5.7's closed form for the
    plan's levels; the distance to S_k is small there (the radix-15 levels act
    on powers of A of norm <= 0.9^9)."""
    pl = G.planted_symmetric(n, 0.9, 900 + n)
    p = _plan(n, k, dtype)
    lv = p.info["levels"]
    ref = EV.planted_reference(pl["V"], pl["lam"], k, 0, levels=lv)
    A = torch.tensor(pl["A"], dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    assert p.status() == 0
    got = S.double().cpu().numpy()
    assert CF.rel_fro(got, ref) < _tol(dtype, 0.9)
    sk = EV.planted_reference(pl["V"], pl["lam"], k, 1)
    assert CF.rel_fro(ref, sk) < 1e-6


@pytest.mark.parametrize("dtype", ["fp64", "split_bf16"])
def test_mixed_paper_form_residual(dtype):
    import paper_2602_11843_gb300 as nm

    g = G.gaussian_scaled(256, 0.5, 32)
    p = _plan(256, 450, dtype, nm.FLAG_RESIDUAL_PAPER)
    ref, _ = EV.evaluate(g["A"], 450, 0, levels=p.info["levels"], form="paper")
    A = torch.tensor(g["A"], dtype=p.io_dtype, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    assert p.status() == 0
    assert CF.rel_fro(S.double().cpu().numpy(), ref) < _tol(dtype, 0.5)


@pytest.mark.parametrize("dtype", ["fp32", "split_bf16"])
def test_mixed_grouped_batch(dtype):
    """A grouped batch (orders <= 256) with the mixed schedule k = 135."""
    import paper_2602_11843_gb300 as nm

    mats = G.jacobi_batch(12, 4321)
    bp = nm.BatchedPlan(len(mats), 256, 135, 0, dtype, nm.FLAG_ALLOW_APPROX)
    io = torch.float32 if dtype == "fp32" else torch.float64
    As = [torch.tensor(m["A"], dtype=io, device="cuda") for m in mats]
    outs = bp(As)
    torch.cuda.synchronize()
    assert bp.status() == 0
    lv = nm.neumann_plan_info(bp.handle)["levels"]
    assert lv == [9, 15]
    tol = 1e-5 if dtype == "fp32" else 2e-3
    for m, S in zip(mats, outs):
        ref, _ = EV.evaluate(m["A"], 135, 0, levels=lv, form="error-map")
        assert CF.rel_fro(S.double().cpu().numpy(), ref) < tol, m["n"]
