"""Series schemes for S_k(A), written over an `Algebra` (see circuits.py).

Each function returns the result and leaves the number of products it
executed in `alg.products`. Products with the identity are not executed (they
are not products), and neither is a power that no later step reads; the
paper's own counts (which include both) are in counts.py.

  naive            Sec. 2.1 "Naive evaluation": accumulate I, A, A^2, ...
  binary_pow2      Sec. 2.1 "Binary splitting": A^{2n} = A^n A^n, S_{2n} = S_n (I + A^n)
  binary_exact     the same doubling plus S_{n+1} = S_n + A^n, A^{n+1} = A^n A for the
                   1-bits of k (any k)
  radix_exact      Sec. 2.2: block concatenation S_{mn} = S_n T_m(A^n) (eq. decomposition)
                   and telescoping I - A^{mn} = T_m(A^n)(I - A^n) for the next power
  radix_residual   Sec. 5.3, eq. generalradix: Y_{n+1} = Y_n f(R_n), R_{n+1} = I - M Y_{n+1},
                   M = I - A, Y_0 = I, R_0 = A; or, with form="error-map", the
                   equivalent R_{n+1} = I - (I - R_n) f(R_n) from the proof of Lemma 5.7
"""

from __future__ import annotations

from .circuits import Algebra


def naive(A, k: int, alg: Algebra):
    """S_k = I + A + ... + A^{k-1} by accumulating powers (Sec. 2.1)."""
    if k < 1:
        raise ValueError("k >= 1")
    S = alg.one
    if k == 1:
        return S
    P = A
    S = S + P
    for _ in range(k - 2):
        P = alg.mul(P, A)
        S = S + P
    return S


def binary_pow2(A, k: int, alg: Algebra):
    """Repeated squaring for k = 2^t (Sec. 2.1, binary splitting)."""
    t = k.bit_length() - 1
    if k < 1 or (1 << t) != k:
        raise ValueError("k must be a power of two")
    S = alg.one
    if t == 0:
        return S
    An = A
    for level in range(t):
        last = level == t - 1
        # (ii) S_{2n} = S_n (I + A^n)
        S = alg.one + An if level == 0 else S + alg.mul(S, An)
        # (i) A^{2n} = A^n A^n, not needed after the last level
        if not last:
            An = alg.mul(An, An)
    return S


def binary_exact(A, k: int, alg: Algebra):
    """S_k for any k >= 1 by the binary digits of k, most significant first.

    Invariant: S = S_n, P = A^n. Doubling: S_{2n} = S_n + S_n A^n, A^{2n} = A^n A^n.
    Increment (digit 1): S_{n+1} = S_n + A^n, A^{n+1} = A^n A.
    """
    if k < 1:
        raise ValueError("k >= 1")
    S, P, s_is_one = alg.one, A, True
    bits = bin(k)[3:]
    for i, b in enumerate(bits):
        last = i == len(bits) - 1
        S = alg.one + P if s_is_one else S + alg.mul(S, P)
        s_is_one = False
        if not last or b == "1":
            P = alg.mul(P, P)
        if b == "1":
            S = S + P
            if not last:
                P = alg.mul(P, A)
    return S


def radix_exact(A, levels, kernels, alg: Algebra):
    """Exact radix scheme over the given level radices (Sec. 2.2).

    levels:  radices m_1, ..., m_t (k = prod m_i); kernels: m -> exact T_m.
    Level i: T = T_{m_i}(A^n); S_{m n} = S_n T (skipped while S_n = I);
    A^{m n} = I - T (I - A^n) (telescoping), skipped at the last level.
    """
    S, An = None, A
    for i, m in enumerate(levels):
        T = kernels[m](An, alg)
        S = T if S is None else alg.mul(S, T)
        if i != len(levels) - 1:
            An = alg.one - alg.mul(T, alg.one - An)
    return alg.one if S is None else S


def radix_residual(A, levels, kernels, alg: Algebra, form: str = "paper"):
    """General radix-kernel iteration (Sec. 5.3, eq. generalradix).

    Y_0 = I, R_0 = A; per level with kernel f: Y_{n+1} = Y_n f(R_n) (skipped while
    Y_n = I), then (except at the last level)
      form="paper":     R_{n+1} = I - M Y_{n+1},           M = I - A
      form="error-map": R_{n+1} = I - (I - R_n) f(R_n)     (proof of Lemma 5.7)
    By Lemma 5.7, R_n = E^{[n]}(A) and Y_n = (I - A)^{-1} (I - R_n).
    """
    Y, R = None, A
    M = alg.one - A
    for i, m in enumerate(levels):
        Fr = kernels[m](R, alg)
        Y = Fr if Y is None else alg.mul(Y, Fr)
        if i != len(levels) - 1:
            if form == "paper":
                R = alg.one - alg.mul(M, Y)
            elif form == "error-map":
                R = alg.one - alg.mul(alg.one - R, Fr)
            else:
                raise ValueError(form)
    return alg.one if Y is None else Y


def pure_levels(k: int, m: int) -> list:
    """[m] * t for k = m^t, else ValueError."""
    t, q = 0, k
    while q > 1 and q % m == 0:
        q //= m
        t += 1
    if q != 1:
        raise ValueError(f"k={k} is not a power of {m}")
    return [m] * t
