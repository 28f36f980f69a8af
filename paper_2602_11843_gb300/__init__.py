"""Truncated Neumann series S_k(A) = I + A + ... + A^{k-1} on one GB300 (sm_103a).

The computation lives in libneumann_gb300.so (C ABI in include/neumann.h);
this package is its Python binding. `Plan` and `evaluate` add PyTorch tensor
marshalling (device memory and the current stream) on top of the C calls.
"""

from __future__ import annotations

from ._capi import *  # noqa: F401,F403
from ._capi import (DTYPES, FP32, FP64, SPLIT_BF16, LIB_PATH, neumann_eval, neumann_eval_batched,  # noqa: F401
                    neumann_eval_batched_host, neumann_eval_host, neumann_last_status, neumann_plan_autotune,
                    neumann_plan_autotune_batched, neumann_plan_host_wait,
                    neumann_plan_create, neumann_plan_create_batched, neumann_plan_destroy, neumann_plan_info,
                    neumann_plan_matmul, neumann_plan_timing)


def _torch_dtype(dtype: int, flags: int):
    import torch

    from ._capi import FLAG_IO_FP32

    if dtype == FP32 or (dtype != FP64 and flags & FLAG_IO_FP32):
        return torch.float32
    return torch.float64


class Plan:
    """Owns a C plan handle; `__call__` evaluates S_k(A) for a CUDA tensor A."""

    def __init__(self, n: int, k: int, radix: int, dtype="fp64", flags: int = 0):
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.flags = flags
        self.handle = neumann_plan_create(n, k, radix, self.dtype, flags)
        self.info = neumann_plan_info(self.handle)

    @property
    def io_dtype(self):
        return _torch_dtype(self.dtype, self.flags)

    def __call__(self, A, out=None, stream=None):
        import torch

        n = self.info["n"]
        if A.device.type != "cuda" or A.dtype != self.io_dtype or A.shape != (n, n) or A.stride(1) != 1:
            raise ValueError(f"A must be a CUDA {self.io_dtype} ({n}, {n}) tensor with unit column stride")
        S = torch.empty((n, n), dtype=self.io_dtype, device=A.device) if out is None else out
        s = torch.cuda.current_stream(A.device) if stream is None else stream
        neumann_eval(self.handle, A.data_ptr(), A.stride(0), S.data_ptr(), S.stride(0), s.cuda_stream)
        return S

    def eval_host(self, A, out=None, stream=None):
        """S_k(A) for a CPU tensor A (pinned for asynchronous copies). Returns the
        CPU result tensor; it is complete after `host_wait()`."""
        import torch

        n = self.info["n"]
        if A.device.type != "cpu" or A.dtype != self.io_dtype or A.shape != (n, n) or A.stride(1) != 1:
            raise ValueError(f"A must be a CPU {self.io_dtype} ({n}, {n}) tensor with unit column stride")
        S = torch.empty((n, n), dtype=self.io_dtype, pin_memory=A.is_pinned()) if out is None else out
        s = torch.cuda.current_stream() if stream is None else stream
        neumann_eval_host(self.handle, A.data_ptr(), A.stride(0), S.data_ptr(), S.stride(0), s.cuda_stream)
        return S

    def host_wait(self):
        neumann_plan_host_wait(self.handle)

    def matmul(self, A, B, out=None, stream=None):
        import torch

        C = torch.empty_like(A) if out is None else out
        s = torch.cuda.current_stream(A.device) if stream is None else stream
        neumann_plan_matmul(self.handle, A.data_ptr(), B.data_ptr(), C.data_ptr(), s.cuda_stream)
        return C

    def autotune(self, A, out=None, reps: int = 3, stream=None):
        """Pick the fastest launch configuration for this plan on input A (writes `out`)."""
        import torch

        n = self.info["n"]
        if A.device.type != "cuda" or A.dtype != self.io_dtype or A.shape != (n, n) or A.stride(1) != 1:
            raise ValueError(f"A must be a CUDA {self.io_dtype} ({n}, {n}) tensor with unit column stride")
        S = torch.empty((n, n), dtype=self.io_dtype, device=A.device) if out is None else out
        s = torch.cuda.current_stream(A.device) if stream is None else stream
        neumann_plan_autotune(self.handle, A.data_ptr(), A.stride(0), S.data_ptr(), S.stride(0), reps, s.cuda_stream)
        self.info = neumann_plan_info(self.handle)
        return self.info

    def set_launch(self, tile_pair: int, raster_group: int):
        """Set the launch configuration by hand (split dtypes): see neumann_plan_set_launch."""
        neumann_plan_set_launch(self.handle, tile_pair, raster_group)
        self.info = neumann_plan_info(self.handle)
        return self.info

    def status(self) -> int:
        return neumann_last_status(self.handle)

    def timing(self) -> list:
        return neumann_plan_timing(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            neumann_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedPlan:
    """Batched evaluation of independent matrices with n_i <= max_n."""

    def __init__(self, count: int, max_n: int, k: int, radix: int, dtype="fp32", flags: int = 0):
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.flags = flags
        self.handle = neumann_plan_create_batched(count, max_n, k, radix, self.dtype, flags)

    def __call__(self, As, outs=None, stream=None):
        import torch

        dt = _torch_dtype(self.dtype, self.flags)
        outs = [torch.empty_like(a) for a in As] if outs is None else outs
        for a in As:
            if a.dtype != dt or not a.is_contiguous():
                raise ValueError(f"inputs must be contiguous {dt}")
        s = torch.cuda.current_stream(As[0].device) if stream is None else stream
        neumann_eval_batched(self.handle, [a.shape[0] for a in As], [a.data_ptr() for a in As],
                             [o.data_ptr() for o in outs], s.cuda_stream)
        return outs

    def bind(self, As, outs):
        """Fix the inputs and outputs of later `launch` calls (argument arrays built once)."""
        import ctypes

        dt = _torch_dtype(self.dtype, self.flags)
        for a, o in zip(As, outs):
            if a.dtype != dt or o.dtype != dt or not a.is_contiguous() or not o.is_contiguous():
                raise ValueError(f"inputs and outputs must be contiguous {dt}")
        cnt = len(As)
        self._bound = (cnt, (ctypes.c_int64 * cnt)(*[a.shape[0] for a in As]),
                       (ctypes.c_void_p * cnt)(*[a.data_ptr() for a in As]),
                       (ctypes.c_void_p * cnt)(*[o.data_ptr() for o in outs]), As, outs)

    def launch(self, stream=None):
        """Evaluate the bound batch on `stream` (default: the current stream)."""
        import torch

        from ._capi import _check, _lib

        cnt, na, aa, sa, As, _ = self._bound
        s = torch.cuda.current_stream(As[0].device) if stream is None else stream
        _check(_lib.neumann_eval_batched(self.handle, cnt, na, aa, sa, s.cuda_stream), "neumann_eval_batched")

    def eval_host(self, ns, A, S, stream=None):
        """The batch packed in the CPU tensors A and S (matrix i at element
        sum_{j<i} n_j^2; pinned for asynchronous copies); complete after host_wait()."""
        import torch

        dt = _torch_dtype(self.dtype, self.flags)
        total = sum(int(n) * int(n) for n in ns)
        for t in (A, S):
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous() or t.numel() < total:
                raise ValueError(f"A and S must be contiguous CPU {dt} tensors of at least {total} elements")
        s = torch.cuda.current_stream() if stream is None else stream
        neumann_eval_batched_host(self.handle, [int(n) for n in ns], A.data_ptr(), S.data_ptr(), s.cuda_stream)

    def host_wait(self):
        neumann_plan_host_wait(self.handle)

    def autotune(self, As, outs, reps: int = 3, stream=None):
        """Pick the fastest matrices-per-pass for this batch (writes `outs`)."""
        import torch

        dt = _torch_dtype(self.dtype, self.flags)
        for a, o in zip(As, outs):
            if a.dtype != dt or o.dtype != dt or not a.is_contiguous() or not o.is_contiguous():
                raise ValueError(f"inputs and outputs must be contiguous {dt}")
        s = torch.cuda.current_stream(As[0].device) if stream is None else stream
        neumann_plan_autotune_batched(self.handle, [a.shape[0] for a in As], [a.data_ptr() for a in As],
                                      [o.data_ptr() for o in outs], reps, s.cuda_stream)
        return neumann_plan_info(self.handle)

    def status(self) -> int:
        return neumann_last_status(self.handle)

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                neumann_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def evaluate(A, k: int, radix: int, dtype="fp64", flags: int = 0):
    """S_k(A) for a CUDA tensor A (one-shot plan)."""
    p = Plan(A.shape[0], k, radix, dtype, flags)
    S = p(A)
    return S
