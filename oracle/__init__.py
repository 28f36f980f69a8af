"""CPU oracle for the truncated Neumann series S_k(A) = I + A + ... + A^{k-1}.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain, FP64 (or exact
rational / multi-precision) statement of what the paper computes. Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. The library (``paper_2602_11843_gb300``) never
imports it and shares no code, constants or tables with it; both sides take
their random inputs from ``workloads`` only.

Modules
  poly        truncated polynomial ring over any number type (exact checks)
  circuits    the radix kernels T_2, T_3, T_5 (Sec. 2.3), T_9 (Thm 3.1) and the
              approximate radix-15 circuit (Sec. 4.1, eq. factors/radix15kernel)
  radix15     the radix-15 coefficients as printed (App. B) and their refinement
  schemes     naive, binary, exact-k binary, exact radix-m (Sec. 2.1-2.2) and the
              residual framework (Sec. 5.3, eq. generalradix)
  closed_form closed forms on a planted symmetric spectrum, probe-vector Horner
  counts      the paper's product-count formulas (Sec. 2.2, Table tab:compare, Sec. 6)

Parity status: every function here is pinned by a test in tests/ against a
value the paper prints, an exact identity, a closed form or brute force; none
is "parity unpinned".
"""
