"""Small, fixed workloads for profiling the library's kernels under ncu.

  python -m paper_2602_11843_gb300.profile_case matmul N REPS   split-BF16 product C = A B
  python -m paper_2602_11843_gb300.profile_case matmul32 N REPS FP32 product C = A B (SIMT kernel)
  python -m paper_2602_11843_gb300.profile_case r15 N REPS      radix-15, k = 3375, split-BF16
  python -m paper_2602_11843_gb300.profile_case batched N REPS  512 matrices of order N, radix 9,
                                                                k = 81, split-BF16, one grouped pass
  python -m paper_2602_11843_gb300.profile_case mixed C REPS    C matrices of orders 16, 32, ..., 256
                                                                in turn (the batched workload's mix),
                                                                radix 9, k = 81, split-BF16
  python -m paper_2602_11843_gb300.profile_case resident C REPS  C matrices of orders 16, 32, 48
                                                                in turn, radix 9, k = 81,
                                                                split-BF16: one resident launch

Inputs are drawn on the device (no host copies): A, B ~ N(0, 1) for the
product; for r15 and batched symmetric matrices with spectral radius about 0.45. Prints the
plan's device status at the end; exits non-zero if it is not 0.
"""

from __future__ import annotations

import sys


def main(argv):
    import torch

    import paper_2602_11843_gb300 as nm

    mode, n, reps = argv[0], int(argv[1]), int(argv[2])
    g = torch.Generator(device="cuda").manual_seed(0)
    if mode in ("matmul", "matmul32"):
        dt = torch.float32 if mode == "matmul32" else torch.float64
        A = torch.randn((n, n), dtype=dt, device="cuda", generator=g)
        B = torch.randn((n, n), dtype=dt, device="cuda", generator=g)
        p = nm.Plan(n, 2, 2, "fp32" if mode == "matmul32" else "split_bf16")
        C = torch.empty_like(A)
        for _ in range(reps):
            p.matmul(A, B, out=C)
    elif mode == "r15":
        X = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
        A = (X + X.T) * (0.45 / (2.0 * n ** 0.5))
        p = nm.Plan(n, 3375, 15, "split_bf16")
        S = torch.empty_like(A)
        for _ in range(reps):
            p(A, out=S)
    elif mode == "batched":
        count = 512
        X = torch.randn((count, n, n), dtype=torch.float64, device="cuda", generator=g)
        As = list((X + X.transpose(1, 2)) * (0.45 / (2.0 * n ** 0.5)))
        outs = [torch.empty_like(a) for a in As]
        p = nm.BatchedPlan(count, n, 81, 9, "split_bf16")
        for _ in range(reps):
            p(As, outs)
    elif mode == "resident":
        count = n
        orders = [16 * (1 + i % 3) for i in range(count)]
        As = []
        for m in orders:
            X = torch.randn((m, m), dtype=torch.float64, device="cuda", generator=g)
            As.append((X + X.T) * (0.45 / (2.0 * m ** 0.5)))
        outs = [torch.empty_like(a) for a in As]
        p = nm.BatchedPlan(count, 64, 81, 9, "split_bf16")
        for _ in range(reps):
            p(As, outs)
    elif mode == "mixed":
        count = n
        orders = [16 * (1 + i % 16) for i in range(count)]
        As = []
        for m in orders:
            X = torch.randn((m, m), dtype=torch.float64, device="cuda", generator=g)
            As.append((X + X.T) * (0.45 / (2.0 * m ** 0.5)))
        outs = [torch.empty_like(a) for a in As]
        p = nm.BatchedPlan(count, 256, 81, 9, "split_bf16")
        for _ in range(reps):
            p(As, outs)
    else:
        raise SystemExit(f"unknown case {mode}")
    torch.cuda.synchronize()
    st = p.status()
    print("profile_case", mode, n, reps, "status", st)
    return 0 if st == 0 else 1


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
