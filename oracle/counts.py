"""The paper's product-count formulas.

  naive                      k - 1                     (Sec. 2.1)
  binary (experiments)       2 ceil(log2 k)            (Sec. 6, "Setup" (i))
  Lei-Nakamura               2 log2 k - 1              (Table tab:compare)
  radix-m update             C(m) = mu_m + 2           (Sec. 2.2 cost model; eq. generalcost)
  pure radix-m, k = m^t      (mu_m + 2) t              (eq. generalcost)
  asymptotic coefficient     C(m) / log2 m             (Sec. 2.1, Table tab:compare, App. A.3)
"""

from __future__ import annotations

import math

from .circuits import MU


def ilog(k: int, m: int) -> int:
    t, q = 0, k
    while q > 1:
        if q % m:
            raise ValueError(f"{k} is not a power of {m}")
        q //= m
        t += 1
    return t


def naive_formula(k: int) -> int:
    return k - 1


def binary_formula(k: int) -> int:
    return 2 * math.ceil(math.log2(k)) if k > 1 else 0


def update_cost(m: int) -> int:
    return MU[m] + 2


def radix_formula(k: int, m: int) -> int:
    return update_cost(m) * ilog(k, m)


def coefficient(m: int) -> float:
    return update_cost(m) / math.log2(m)
