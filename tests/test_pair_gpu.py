"""GPU parity of the 2-CTA (CTA pair) tensor-core product.

Split products of padded order >= 4096 run on 2-CTA clusters with 256 x 256
tiles (cta_group::2, M = 256); NEUMANN_FLAG_SINGLE_CTA keeps them on the
single-CTA 128 x 256 tiles. Both must give an FP64-accurate product to the
split's tolerance, and the two tilings issue the same MMA sequence per output
element, so they must agree with each other far more closely than either
agrees with FP64. Orders cover an even and an odd number of 256-row pair tiles
and a ragged tail (n not a multiple of 256).
"""

import numpy as np
import pytest

from oracle import closed_form as CF
from oracle import evaluate as EV
from workloads import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# relative Frobenius error of one product at n <= 4352 (N(0,1) operands)
TOL_MM = {"split_bf16": 4e-5, "split_fp16": 3e-5}


def _nm():
    import paper_2602_11843_gb300 as nm

    return nm


def _matmul(A, B, dtype, flags):
    nm = _nm()
    p = nm.Plan(A.shape[0], 2, 2, dtype, flags)
    C = p.matmul(A, B)
    torch.cuda.synchronize()
    assert p.status() == 0
    return C


@pytest.mark.parametrize("dtype", ["split_bf16", "split_fp16"])
@pytest.mark.parametrize("n", [4096, 4000, 4352])
def test_pair_product_against_fp64(dtype, n):
    nm = _nm()
    rng = np.random.default_rng(7000 + n)
    A_np, B_np = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    A = torch.tensor(A_np, dtype=torch.float64, device="cuda")
    B = torch.tensor(B_np, dtype=torch.float64, device="cuda")
    ref = torch.tensor(A_np) @ torch.tensor(B_np)
    C_pair = _matmul(A, B, dtype, 0).cpu()
    C_single = _matmul(A, B, dtype, nm.FLAG_SINGLE_CTA).cpu()
    e_pair = float(torch.linalg.norm(C_pair - ref) / torch.linalg.norm(ref))
    e_single = float(torch.linalg.norm(C_single - ref) / torch.linalg.norm(ref))
    d = float((C_pair - C_single).abs().max() / ref.abs().max())
    print(f"n={n} {dtype}: pair {e_pair:.3e} single {e_single:.3e} max|pair-single|/max|C| {d:.3e}")
    assert e_pair < TOL_MM[dtype] and e_single < TOL_MM[dtype]
    assert d < 1e-6


def test_pair_eval_writes_nothing_outside_the_caller_block():
    """S_k on pairs into a view with a larger leading dimension (n = 4000, a
    ragged last pair tile) keeps the surrounding columns and rows untouched."""
    nm = _nm()
    n, ld, k = 4000, 4104, 81
    pl = G.config_inputs(2, n=n)
    A = torch.tensor(pl["A"], dtype=torch.float64, device="cuda")
    big = torch.full((n + 8, ld), 7.0, dtype=torch.float64, device="cuda")
    out = big[:n, :n]
    p = nm.Plan(n, k, 9, "split_bf16")
    p(A, out=out)
    torch.cuda.synchronize()
    assert p.status() == 0
    assert torch.all(big[:n, n:] == 7.0) and torch.all(big[n:, :] == 7.0)
    ref = EV.planted_reference(pl["V"], pl["lam"], k, 9)
    assert CF.rel_fro(out.cpu().numpy(), ref) < 1e-3


@pytest.mark.parametrize("dtype", ["split_bf16", "split_fp16"])
@pytest.mark.parametrize("radix,k", [(9, 729), (15, 225)])
def test_pair_scheme_matches_closed_form(dtype, radix, k):
    """A whole S_k at n = 4096 (planted spectrum in [-0.9, 0.9]) on pairs and on
    single-CTA tiles, each against the oracle's closed form."""
    nm = _nm()
    pl = G.config_inputs(2)
    ref = EV.planted_reference(pl["V"], pl["lam"], k, radix)
    A = torch.tensor(pl["A"], dtype=torch.float64, device="cuda")
    errs = []
    for flags in (0, nm.FLAG_SINGLE_CTA):
        p = nm.Plan(A.shape[0], k, radix, dtype, flags)
        S = p(A)
        torch.cuda.synchronize()
        assert p.status() == 0
        errs.append(CF.rel_fro(S.cpu().numpy(), ref))
    print(f"n=4096 radix {radix} k {k} {dtype}: pair {errs[0]:.3e} single {errs[1]:.3e}")
    # both splits are limited here by the tensor cores' FP32 accumulation
    # (a bias growing with n, ~1.5e-5 per product at n = 4096), amplified across levels
    assert max(errs) < 1e-3
