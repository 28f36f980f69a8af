"""One-call oracle: S_k(A) (or the approximate kernels' framework result) in FP64 on the CPU.

radix 1  naive (Sec. 2.1)
radix 2  repeated squaring for k = 2^t, binary digits of k otherwise (Sec. 2.1)
radix 3, 5, 9  exact radix-m splitting with kernels T_3, T_5, T_9 (Sec. 2.2, Thm 3.1)
radix 15 residual framework with the approximate T~_15 (Sec. 5.3, App. B)
radix 24, 25, 27, 31, 33  residual framework with the five-product approximate
         kernels (App. C, Table approx; circuits of radix_p5.py)
radix 0  exact kernels over the factorisation of k into 9, 5, 3 and 2 (block
         concatenation holds for any factor order, Sec. 2.2); with approx=True
         the radix-15 kernel may take part too (mixed_levels), and the whole
         sequence runs in the residual framework, whose Lemma 5.7 holds level
         by level (Sec. 5.3)
"""

from __future__ import annotations

import numpy as np

from . import circuits as C
from . import radix15 as R15
from . import radix_p5 as RP5
from . import schemes as SC


def kernels(coef15: str = "refined") -> dict:
    coef = R15.load_refined(float) if coef15 == "refined" else R15.printed(float)
    return {2: C.kernel_t2, 3: C.kernel_t3, 5: C.kernel_t5, 9: C.kernel_t9,
            15: C.kernel_t15(coef),
            24: C.kernel_p5(RP5.load_refined(24)), 25: C.kernel_p5(RP5.load_refined(25)),
            27: C.kernel_p5(RP5.load_approx(27)), 31: C.kernel_p5(RP5.load_approx(31)),
            33: C.kernel_p5(RP5.load_approx(33))}


#: Radices whose kernels are approximate: they run in the residual framework (Sec. 5.3).
APPROX = (15, 24, 25, 27, 31, 33)


def auto_levels(k: int) -> list:
    """Factor k over {9, 5, 3, 2}: a 9 for each pair of 3s, then 5s, a lone 3, 2s."""
    levels, q = [], k
    for m in (9, 5, 3, 2):
        while q % m == 0:
            levels.append(m)
            q //= m
    if q != 1:
        raise ValueError(f"k={k} has a prime factor above 5")
    return levels


def mixed_levels(k: int) -> list:
    """Radix 0 with approximate levels allowed: radices from {2, 3, 5, 9, 15}
    whose product is k and whose cost sum (mu_m + 2) (Sec. 2.2 cost model) is
    least; among equal costs, fewer radix-15 levels, then fewer levels. Found
    by trying every divisor in turn (memoised recursion). Returned in the order
    the levels run: the exact ones as 9, 5, 3, 2, then the radix-15 ones."""
    from functools import lru_cache

    @lru_cache(maxsize=None)
    def best(q):
        if q == 1:
            return (0, 0, 0, ())
        options = []
        for m in (2, 3, 5, 9, 15):
            if q % m == 0:
                sub = best(q // m)
                if sub is not None:
                    options.append((sub[0] + C.MU[m] + 2, sub[1] + (m == 15), sub[2] + 1, sub[3] + (m,)))
        return min(options) if options else None

    b = best(k)
    if b is None:
        raise ValueError(f"k={k} has a prime factor above 5")
    ms = list(b[3])
    return [m for order in (9, 5, 3, 2, 15) for m in ms if m == order]


def evaluate(A: np.ndarray, k: int, radix: int, coef15: str = "refined",
             form: str = "paper", approx: bool = False, levels=None):
    """Returns (result, products executed). `levels` (radix 0 only) overrides
    the factorisation; with approx=True (or levels given) radix 0 runs in the
    residual framework."""
    A = np.asarray(A, dtype=np.float64)
    alg = C.matrix_algebra(A.shape[0])
    ks = kernels(coef15)
    if radix == 1:
        S = SC.naive(A, k, alg)
    elif radix == 2:
        S = SC.binary_pow2(A, k, alg) if k & (k - 1) == 0 else SC.binary_exact(A, k, alg)
    elif radix in (3, 5, 9):
        S = SC.radix_exact(A, SC.pure_levels(k, radix), ks, alg)
    elif radix in APPROX:
        S = SC.radix_residual(A, SC.pure_levels(k, radix), ks, alg, form)
    elif radix == 0 and (approx or levels is not None):
        S = SC.radix_residual(A, list(levels) if levels is not None else mixed_levels(k), ks, alg, form)
    elif radix == 0:
        S = SC.radix_exact(A, auto_levels(k), ks, alg)
    else:
        raise ValueError(f"radix {radix}")
    return np.asarray(S, dtype=np.float64), alg.products


def planted_reference(V, lam, k: int, radix: int, coef15: str = "refined", rows=None, levels=None):
    """Closed form on a planted symmetric spectrum (closed_form.py): S_k for the
    exact schemes, Y_t of Lemma 5.7 for the approximate radices and for an
    explicit level sequence `levels` (radix 0). `rows` selects rows only."""
    from . import closed_form as CF

    if levels is not None:
        f = CF.radix_scalar(lam, list(levels), kernels(coef15))
    elif radix in APPROX:
        f = CF.radix_scalar(lam, SC.pure_levels(k, radix), kernels(coef15))
    else:
        f = CF.sk_scalar(lam, k)
    if rows is None:
        return CF.symmetric_function(V, lam, f)
    return CF.symmetric_function_rows(V, lam, f, rows)
