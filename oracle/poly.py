"""Truncated univariate polynomials with coefficients of any field type.

A polynomial in z stands for a matrix polynomial in A: every iterate of every
scheme in the paper is a polynomial in A (Sec. 2.2, block concatenation), so
running a scheme on polynomials gives the exact coefficient sequence the
matrix scheme computes. Coefficients above `deg` are dropped.

Coefficients may be int / fractions.Fraction (exact), float, or mpmath.mpf.
Storage is a dict {degree: coefficient} so monomials such as A^{81} stay cheap.
"""

from __future__ import annotations


class Poly:
    __slots__ = ("c", "deg")

    def __init__(self, coeffs: dict, deg: int):
        self.deg = deg
        self.c = {d: v for d, v in coeffs.items() if d <= deg and v != 0}

    @staticmethod
    def one(deg: int, unit=1) -> "Poly":
        return Poly({0: unit}, deg)

    @staticmethod
    def z(deg: int, unit=1) -> "Poly":
        return Poly({1: unit}, deg)

    def __add__(self, other: "Poly") -> "Poly":
        out = dict(self.c)
        for d, v in other.c.items():
            out[d] = out.get(d, 0) + v
        return Poly(out, min(self.deg, other.deg))

    def __neg__(self) -> "Poly":
        return Poly({d: -v for d, v in self.c.items()}, self.deg)

    def __sub__(self, other: "Poly") -> "Poly":
        return self + (-other)

    def __rmul__(self, s) -> "Poly":
        return Poly({d: s * v for d, v in self.c.items()}, self.deg)

    def __matmul__(self, other: "Poly") -> "Poly":
        deg = min(self.deg, other.deg)
        out: dict = {}
        for d1, v1 in self.c.items():
            for d2, v2 in other.c.items():
                d = d1 + d2
                if d <= deg:
                    out[d] = out.get(d, 0) + v1 * v2
        return Poly(out, deg)

    def coef(self, d: int):
        return self.c.get(d, 0)

    def coeffs(self, upto: int | None = None) -> list:
        upto = self.deg if upto is None else upto
        return [self.c.get(d, 0) for d in range(upto + 1)]
