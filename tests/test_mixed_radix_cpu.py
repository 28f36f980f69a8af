"""Mixed-radix schedules that include the approximate radix-15 kernel (radix 0
with NEUMANN_FLAG_ALLOW_APPROX): the oracle's level search and residual
framework pinned to brute force and to Lemmas 5.6/5.7, and the library's plans
checked against them (host only, no GPU).

Block concatenation (Sec. 2.2, eq. decomposition) lets any level sequence whose
radices multiply to k build S_k from exact kernels; Lemma 5.7 (Sec. 5.3) holds
level by level for any kernels, so a sequence mixing exact and approximate
levels gives Y_t = (I - A)^{-1} (I - E_t(...E_1(A))), which agrees with S_k
through degree k - 1.
"""

import itertools

import pytest

from oracle import circuits as C
from oracle import evaluate as EV
from oracle import radix15 as R15
from oracle import schemes as SC
from oracle.poly import Poly


def _cost(levels):
    return (sum(C.MU[m] + 2 for m in levels), sum(m == 15 for m in levels), len(levels))


def _brute_best(k):
    """Every ordered sequence of radices from {2, 3, 5, 9, 15} with product k
    (depth-first over all of them), and the least (cost, radix-15 levels, levels)."""
    best = None

    def walk(q, seq):
        nonlocal best
        if q == 1:
            c = _cost(seq)
            best = c if best is None or c < best else best
            return
        for m in (2, 3, 5, 9, 15):
            if q % m == 0:
                walk(q // m, seq + [m])

    walk(k, [])
    return best


SMOOTH = sorted({2 ** a * 3 ** b * 5 ** c for a in range(5) for b in range(5) for c in range(4)} - {1})


@pytest.mark.parametrize("k", SMOOTH[:60])
def test_oracle_mixed_levels_is_least_cost(k):
    lv = EV.mixed_levels(k)
    prod = 1
    for m in lv:
        prod *= m
    assert prod == k
    assert _cost(lv) == _brute_best(k)
    # exact levels first (9, 5, 3, 2), then the radix-15 levels
    order = {9: 0, 5: 1, 3: 2, 2: 3, 15: 4}
    assert [order[m] for m in lv] == sorted(order[m] for m in lv)


def test_oracle_mixed_levels_examples():
    assert EV.mixed_levels(135) == [9, 15]
    assert EV.mixed_levels(450) == [2, 15, 15]
    assert EV.mixed_levels(3375 * 9) == [9, 15, 15, 15]
    assert EV.mixed_levels(45) == [9, 5]  # 9 + 5 ties with 15 + 3: the exact pair wins
    assert EV.mixed_levels(16) == [2, 2, 2, 2]
    with pytest.raises(ValueError):
        EV.mixed_levels(7 * 15)


def _leading_c_total(levels, c):
    """Leading coefficient of E_t(...E_1(z)) when exact levels map w -> w^m and
    the radix-15 level maps w -> c w^15 + O(w^16) (Lemma 5.6's propagation)."""
    coef = 1
    for m in levels:
        coef = coef ** m * (c if m == 15 else 1)
    return coef


@pytest.mark.parametrize("levels", [[9, 15], [15, 9], [2, 15, 15], [15, 2], [3, 15, 2]])
def test_mixed_schedule_on_polynomials_lemma_5_7(levels):
    """The scheme run over 50-digit polynomials: (1 - z) Y = 1 - E with E = 0
    below degree k and its degree-k coefficient the propagated spillover
    c_total (c = 1 - [T~15]_15), whatever the position of the radix-15 level."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    k = 1
    for m in levels:
        k *= m
    deg = k + 1
    coef = R15.load_refined(mp.mpf)
    num = lambda q: mp.mpf(q.numerator) / q.denominator  # noqa: E731
    alg = C.poly_algebra(deg, num=num)
    ks = {2: C.kernel_t2, 3: C.kernel_t3, 5: C.kernel_t5, 9: C.kernel_t9, 15: C.kernel_t15(coef)}
    Y = SC.radix_residual(Poly.z(deg, mp.mpf(1)), levels, ks, alg, form="error-map")
    ycs = Y.coeffs(deg)
    assert max(abs(x - 1) for x in ycs[:k]) < 1e-25
    one_minus_z = Poly({0: mp.mpf(1), 1: mp.mpf(-1)}, deg)
    E = Poly.one(deg, mp.mpf(1)) - (one_minus_z @ Y)
    ecs = E.coeffs(deg)
    assert max(abs(x) for x in ecs[:k]) < 1e-25
    c = 1 - R15.circuit_poly(R15.flatten(coef), mp.mpf(0), mp.mpf(1))[15]
    assert abs(ecs[k] - _leading_c_total(levels, c)) < 1e-25
    # and both residual forms of eq. generalradix agree on polynomials
    alg2 = C.poly_algebra(deg, num=num)
    Y2 = SC.radix_residual(Poly.z(deg, mp.mpf(1)), levels, ks, alg2, form="paper")
    assert max(abs(a - b) for a, b in zip(Y2.coeffs(deg), ycs)) < 1e-25
    # products: sum (mu_m + 2) - 2 executed (no product with Y_0 = I, no unused last residual)
    assert alg.products == sum(C.MU[m] + 2 for m in levels) - 2


nm = pytest.importorskip("paper_2602_11843_gb300", reason="library not built")


@pytest.mark.parametrize("k", SMOOTH[:60] + [135, 450, 3375 * 9, 15 ** 5 * 2])
def test_library_mixed_plan_matches_oracle_search(k):
    C_ = nm._capi
    h = C_.neumann_plan_create(64, k, 0, C_.SPLIT_BF16, C_.FLAG_ALLOW_APPROX)
    try:
        info = C_.neumann_plan_info(h)
    finally:
        C_.neumann_plan_destroy(h)
    lv = info["levels"]
    prod = 1
    for m in lv:
        prod *= m
    assert prod == k
    assert _cost(lv) == _cost(EV.mixed_levels(k))
    order = {9: 0, 5: 1, 3: 2, 2: 3, 15: 4}
    assert [order[m] for m in lv] == sorted(order[m] for m in lv)
    assert info["products_formula"] == sum(C.MU[m] + 2 for m in lv)
    assert info["products_executed"] == (info["products_formula"] - 2 if len(lv) else 0)


def test_library_radix0_without_flag_stays_exact():
    C_ = nm._capi
    h = C_.neumann_plan_create(64, 135, 0, C_.FP64, 0)
    try:
        info = C_.neumann_plan_info(h)
    finally:
        C_.neumann_plan_destroy(h)
    assert info["levels"] == EV.auto_levels(135) == [9, 5, 3]
    for k in (7 * 9, 11):
        with pytest.raises(C_.NeumannError):
            C_.neumann_plan_create(64, k, 0, C_.FP64, C_.FLAG_ALLOW_APPROX)


def test_mixed_levels_search_is_exhaustive_on_orders():
    """The cost of a level multiset does not depend on order: every permutation
    of the oracle's choice costs the same (the order is the reading's choice)."""
    lv = EV.mixed_levels(3375 * 9)
    assert {_cost(list(p)) for p in itertools.permutations(lv)} == {_cost(lv)}
