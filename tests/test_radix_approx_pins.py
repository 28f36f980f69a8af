"""Pins of the approximate-prefix five-product kernels, radix 27, 31 and 33
(App. C, Table approx).

App. C reports five-product kernels of radix 24-33 with a nonzero "kernel
residual" (the prefix objective sum_{j<m} ([T~]_j - 1)^2 of Sec. 4.2) and prints
only radix 33's polynomial. This project's kernels are least-squares points of
its own seeded search (oracle/radix_p5.py), used exactly as published. What
fixes them:
- the objective, by two evaluation paths (the numpy circuit and the circuit over
  60-digit polynomials), against the table's residual column;
- the published point is the search output of its recorded start;
- Table approx's inverse-error column on its own matrix (d = 64, eigenvalues of
  I - A geometric in [0.01, 1]): radix 33 reproduces the printed 0.722;
- Lemma 5.7 on matrices inside each kernel's convergence region.
"""

import numpy as np
import pytest

from oracle import circuits as C
from oracle import closed_form as CF
from oracle import evaluate as EV
from oracle import radix_p5 as RP5
from oracle.poly import Poly
from workloads import generators as G

APPROX = RP5.RADICES_APPROX


def _table(golden):
    return {r["radix"]: r for r in golden("paper_table_approx.json")["rows"]}


@pytest.mark.parametrize("m", APPROX)
def test_kernel_residual_two_paths_and_table(m, golden):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    x = RP5.flatten(RP5.load_approx(m))
    f_np = RP5.prefix_objective(m, x)
    # the same circuit run over 60-digit polynomials (oracle.circuits.kernel_p5)
    alg = C.poly_algebra(RP5.DEG, num=lambda q: mp.mpf(q.numerator) / q.denominator)
    coef = RP5.load_approx(m, num=lambda s: mp.mpf(s))
    T = C.kernel_p5(coef)(Poly.z(RP5.DEG, mp.mpf(1)), alg).coeffs(RP5.DEG)
    f_mp = sum((T[j] - 1) ** 2 for j in range(m))
    assert abs(float(f_mp) - f_np) < 1e-12 * max(1.0, f_np)
    assert alg.products == 5
    assert abs(f_np - RP5.SEARCH_APPROX_OBJECTIVE[m]) < 1e-6 * f_np
    # Table approx prints one significant digit: ours is at most 1.5x its value
    # (27: 4.7e-4 vs 1e-3, 31: 0.109 vs 1e-1, 33: 0.554 vs 6e-1)
    assert f_np <= 1.5 * _table(golden)[m]["kernel_residual"]
    assert RP5.growth(x) <= RP5.GROWTH_CAP


@pytest.mark.parametrize("m", APPROX)
def test_published_point_is_the_search_output(m):
    s, x, f, g = RP5.approx_start_point(m, RP5.SEARCH_APPROX_PICK[m])
    assert abs(f - RP5.SEARCH_APPROX_OBJECTIVE[m]) < 1e-6 * f
    assert g <= RP5.GROWTH_CAP


@pytest.mark.parametrize("m", APPROX)
def test_table_approx_inverse_error(m, golden):
    """One kernel application S = T~(B) on Table approx's matrix: ||S - A^-1||_2 /
    ||A^-1||_2 over the eigenvalues (A symmetric). The printed "vs Exact" ratio is
    1.000 / 1.002 / 1.007; exact S_m gives 0.99^m."""
    a = np.geomspace(0.01, 1.0, 64)
    x = RP5.flatten(RP5.load_approx(m))
    T = RP5.circuit_np(x, jacobian=False)
    inv = np.abs(np.polyval(T[::-1], 1.0 - a) - 1.0 / a).max() * a.min()
    printed = _table(golden)[m]["inv_err"]
    exact = 0.99 ** m
    print(f"radix {m}: inverse error {inv:.4f} (printed {printed}), exact S_{m} {exact:.4f}")
    assert inv <= printed + 2e-3
    assert inv / exact < 1.01
    if m == 33:  # the radix the table prints coefficients for
        assert abs(inv - printed) < 1e-3


def test_radix33_matches_the_printed_polynomial_in_kind(golden):
    """App. C prints radix 33's coefficients (two decimals): between 0.69 and 1.27,
    none beyond degree 32. Ours: degree 32 (five products), every prefix
    coefficient within the same band."""
    x = RP5.flatten(RP5.load_approx(33))
    T = RP5.circuit_np(x, jacobian=False)
    assert len(T) == 33
    assert 0.6 < T[:33].min() and T[:33].max() < 1.35


REGION = {27: (-0.999, 0.999), 31: (-0.999, 0.999), 33: (-0.925, 0.999)}


@pytest.mark.parametrize("m", APPROX)
def test_convergence_region(m):
    """|E(x)| < |x| on the stated interval (radix 33: from -0.925)."""
    lo, hi = REGION[m]
    x = np.concatenate([np.linspace(lo, -1e-3, 2000), np.linspace(1e-3, hi, 2000)])
    E = CF.error_map(EV.kernels()[m])(x)
    assert np.all(np.abs(E) < np.abs(x))


@pytest.mark.parametrize("m", APPROX)
@pytest.mark.parametrize("t", [1, 2])
def test_matrix_iteration_matches_lemma_5_7(m, t):
    p = G.planted_symmetric(64, 0.9, 9)
    ref = EV.planted_reference(p["V"], p["lam"], m ** t, m)
    for form in ("paper", "error-map"):
        S, prods = EV.evaluate(p["A"], m ** t, m, form=form)
        assert CF.rel_fro(S, ref) < 1e-12
        assert prods == 7 * t - 2
    # the framework value differs from S_k by the kernel residual: measurable, bounded
    sk = EV.planted_reference(p["V"], p["lam"], m ** t, 1)
    assert CF.rel_fro(ref, sk) < 5e-2


nm = pytest.importorskip("paper_2602_11843_gb300", reason="library not built")


@pytest.mark.parametrize("m", APPROX)
def test_library_uses_the_published_point(m):
    coef, err, spill = nm._capi.neumann_radix_p5_coefficients(m)
    x = RP5.flatten(RP5.load_approx(m))
    assert coef == [float(v) for v in x]  # the same float64 values, no refinement
    T = RP5.circuit_np(x, jacobian=False)
    assert abs(err - np.abs(T[:m] - 1).max()) < 1e-12
    h = nm._capi.neumann_plan_create(64, m * m, m, nm._capi.SPLIT_BF16, 0)
    try:
        info = nm._capi.neumann_plan_info(h)
        assert info["levels"] == [m, m] and info["products_formula"] == 14
    finally:
        nm._capi.neumann_plan_destroy(h)
