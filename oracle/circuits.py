"""Radix kernels T_m(B) = I + B + ... + B^{m-1} as product circuits.

Every circuit is written once over an `Algebra`: an identity element, a
counted product `mul`, and the host language's `+`, `-` and scalar `*` for
linear combinations. The same code therefore runs on

  * numpy FP64 matrices            (the oracle proper),
  * truncated polynomials (`Poly`) with Fraction / mpf coefficients
                                   (exact identity checks),
  * numpy arrays of eigenvalues    (scalar closed forms, `mul` = elementwise).

Scalars enter through `alg.num`, which turns an exact Fraction into the
algebra's number type.
"""

from __future__ import annotations

from fractions import Fraction as F

import numpy as np

from .poly import Poly


class Algebra:
    """Identity, counted product and scalar conversion for one number system."""

    def __init__(self, one, mul, num=float):
        self.one = one
        self._mul = mul
        self.num = num
        self.products = 0

    def mul(self, x, y):
        self.products += 1
        return self._mul(x, y)


def matrix_algebra(n: int) -> Algebra:
    return Algebra(np.eye(n), lambda x, y: x @ y, float)


def scalar_algebra(shape=()) -> Algebra:
    return Algebra(np.ones(shape), lambda x, y: x * y, float)


def poly_algebra(deg: int, num=lambda q: q) -> Algebra:
    """`num` maps a Fraction to the coefficient type (identity keeps it exact)."""
    return Algebra(Poly.one(deg, num(F(1))), lambda x, y: x @ y, num)


# --------------------------------------------------------------------------
# Exact kernels
# --------------------------------------------------------------------------

def kernel_t2(B, alg: Algebra):
    """T_2(B) = I + B, no product (binary splitting, Sec. 2.1)."""
    return alg.one + B


def kernel_t3(B, alg: Algebra):
    """T_3(B) = I + B + B^2, one product (ternary splitting, Sec. 2.1)."""
    U = alg.mul(B, B)
    return alg.one + B + U


def kernel_t5(B, alg: Algebra):
    """Quinary kernel of Gustafsson et al. (Sec. 2.3; App. A.1, eq. quinary-U/V/final).

    U = B^2;  V = U (B + U) = B^3 + B^4;  T_5 = I + B + U + V.  Two products.
    """
    U = alg.mul(B, B)
    V = alg.mul(U, B + U)
    return alg.one + B + U + V


def kernel_t9(B, alg: Algebra):
    """Exact radix-9 kernel in three products (Theorem 3.1; App. A.2).

    MM1  U = B^2
    MM2  V = U (B + 2U)            = B^3 + 2 B^4
         P = 3/20 B + 2U + V,  Q = 11/40 B - 1/8 U + 1/4 V
    MM3  W = P Q
         T_9 = W + I + B + 767/800 U + 15/32 V
    """
    n = alg.num
    U = alg.mul(B, B)
    V = alg.mul(U, B + n(F(2)) * U)
    P = n(F(3, 20)) * B + n(F(2)) * U + V
    Q = n(F(11, 40)) * B - n(F(1, 8)) * U + n(F(1, 4)) * V
    W = alg.mul(P, Q)
    return W + alg.one + B + n(F(767, 800)) * U + n(F(15, 32)) * V


def kernel_naive(m: int):
    """Radix-m kernel computed naively: powers B^2..B^{m-1}, m-2 products (Sec. 2.1)."""

    def k(B, alg: Algebra):
        T = alg.one + B
        P = B
        for _ in range(m - 2):
            P = alg.mul(P, B)
            T = T + P
        return T

    return k


# --------------------------------------------------------------------------
# Approximate radix-15 kernel
# --------------------------------------------------------------------------

def kernel_t15(coef: dict):
    """Approximate radix-15 circuit (Sec. 4.1, eq. factors and radix15kernel).

    P_1 = B^2; basis B_1 = {I, B, P_1}; for i = 2, 3, 4:
    L_i = sum_{X in B_i} l_{i,X} X,  R_i = sum_{X in B_i} r_{i,X} X,
    P_i = L_i R_i,  B_{i+1} = B_i + {P_i};
    T~_15 = I + g_1 B + g_2 P_1 + g_3 P_2 + g_4 P_3 + P_4.  Four products.

    `coef` holds sequences l2, r2 (over I, B, P1), l3, r3 (over I, B, P1, P2),
    l4, r4 (over I, B, P1, P2, P3) and gamma (for B, P1, P2, P3), already in
    the algebra's number type.
    """

    def k(B, alg: Algebra):
        P1 = alg.mul(B, B)
        basis = [alg.one, B, P1]
        prods = [P1]
        for lk, rk in (("l2", "r2"), ("l3", "r3"), ("l4", "r4")):
            L = _lincomb(coef[lk], basis)
            R = _lincomb(coef[rk], basis)
            Pi = alg.mul(L, R)
            prods.append(Pi)
            basis.append(Pi)
        g = coef["gamma"]
        P1, P2, P3, P4 = prods
        return alg.one + g[0] * B + g[1] * P1 + g[2] * P2 + g[3] * P3 + P4

    return k


def kernel_p5(coef: dict):
    """Five-product approximate circuit of radix 24 or 25 (App. C, Table approx:
    the 5-product budget; structure of Sec. 4.1 with one more product).

    P_1 = B^2; basis B_1 = {I, B, P_1}; for i = 2, 3, 4, 5:
    L_i = sum_{X in B_i} l_{i,X} X,  R_i = sum_{X in B_i} r_{i,X} X,
    P_i = L_i R_i,  B_{i+1} = B_i + {P_i};
    T~_m = I + g_1 B + g_2 P_1 + g_3 P_2 + g_4 P_3 + g_5 P_4 + P_5.  Five products.

    `coef` holds l2..l5, r2..r5 over (I, B, P1, ..., P_{i-1}) and gamma (for
    B, P1, P2, P3, P4), already in the algebra's number type (radix_p5.py).
    """

    def k(B, alg: Algebra):
        P1 = alg.mul(B, B)
        basis = [alg.one, B, P1]
        for i in range(2, 6):
            L = _lincomb(coef[f"l{i}"], basis)
            R = _lincomb(coef[f"r{i}"], basis)
            basis.append(alg.mul(L, R))
        g = coef["gamma"]
        _, _, P1, P2, P3, P4, P5 = basis
        return alg.one + g[0] * B + g[1] * P1 + g[2] * P2 + g[3] * P3 + g[4] * P4 + P5

    return k


def _lincomb(cs, xs):
    acc = cs[0] * xs[0]
    for c, x in zip(cs[1:], xs[1:]):
        acc = acc + c * x
    return acc


#: Products per kernel application, mu_m (Sec. 2.2 cost model).
MU = {2: 0, 3: 1, 5: 2, 9: 3, 15: 4, 24: 5, 25: 5}
