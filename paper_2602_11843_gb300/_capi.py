"""ctypes binding of include/neumann.h, one Python function per C entry point.

Only argument marshalling happens here; every step of the evaluation runs in
libneumann_gb300.so. Importing this module fails (ImportError) when the
library has not been built, so no caller can silently fall back to another
implementation.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_float, c_int, c_int64, c_size_t, c_uint32, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libneumann_gb300.so")

# dtypes
FP64, FP32, SPLIT_BF16, SPLIT_FP16 = 0, 1, 2, 3
DTYPES = {"fp64": FP64, "fp32": FP32, "split_bf16": SPLIT_BF16, "split_fp16": SPLIT_FP16}

# return codes
OK, EINVAL, ENOMEM, ECUDA, ENOTSUP = 0, 1, 2, 3, 4

# device status bits
STATUS_NONFINITE, STATUS_TIMEOUT = 1, 2

# flags
FLAG_EXACT_K = 0x1
FLAG_RESIDUAL_PAPER = 0x2
FLAG_PRINTED_COEFFS = 0x4
FLAG_TIMING = 0x8
FLAG_IO_FP32 = 0x10
FLAG_SINGLE_CTA = 0x20
FLAG_PRECISE_ACC = 0x40
FLAG_SYMMETRIC = 0x80
FLAG_ALLOW_APPROX = 0x100
FLAG_NO_RESIDENT = 0x200

MAX_LEVELS = 64


class NeumannError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} ({code})")


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n", c_int64), ("k", c_int64), ("radix", c_int), ("dtype", c_int), ("flags", c_uint32),
        ("levels", c_int), ("level_radix", c_int * MAX_LEVELS),
        ("products_formula", c_int64), ("products_executed", c_int64), ("launches", c_int64),
        ("workspace_bytes", c_size_t), ("padded_n", c_int64),
        ("tile_pair", c_int), ("raster_group", c_int), ("batch_chunk", c_int), ("tuned", c_int),
        ("bytes_per_element", c_int64), ("product_bytes_per_element", c_int64),
        ("resident_max_n", c_int),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "neumann_plan_create": (c_int, [POINTER(c_void_p), c_int64, c_int64, c_int, c_int, c_uint32]),
        "neumann_plan_info": (c_int, [P, POINTER(PlanInfo)]),
        "neumann_plan_set_workspace": (c_int, [P, c_void_p, c_size_t]),
        "neumann_eval": (c_int, [P, c_void_p, c_int64, c_void_p, c_int64, c_void_p]),
        "neumann_plan_matmul": (c_int, [P, c_void_p, c_void_p, c_void_p, c_void_p]),
        "neumann_eval_host": (c_int, [P, c_void_p, c_int64, c_void_p, c_int64, c_void_p]),
        "neumann_plan_host_wait": (c_int, [P]),
        "neumann_eval_batched_host": (c_int, [P, c_int, POINTER(c_int64), c_void_p, c_void_p, c_void_p]),
        "neumann_plan_create_batched": (c_int, [POINTER(c_void_p), c_int, c_int64, c_int64, c_int, c_int, c_uint32]),
        "neumann_eval_batched": (c_int, [P, c_int, POINTER(c_int64), POINTER(c_void_p), POINTER(c_void_p), c_void_p]),
        "neumann_last_status": (c_int, [P, POINTER(c_uint32)]),
        "neumann_plan_timing": (c_int, [P, POINTER(c_float), c_int, POINTER(c_int)]),
        "neumann_radix15_coefficients": (c_int, [c_int, POINTER(c_double), POINTER(c_double), POINTER(c_double),
                                                 POINTER(c_double)]),
        "neumann_radix_p5_coefficients": (c_int, [c_int, POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
        "neumann_plan_selftest_timeout": (c_int, [P, ctypes.c_uint64, c_void_p]),
        "neumann_matmul_noalloc": (c_int, [c_int64, c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int64,
                                           c_void_p]),
        "neumann_matmul_noalloc_status": (c_int, [c_void_p, POINTER(c_uint32)]),
        "neumann_plan_autotune": (c_int, [P, c_void_p, c_int64, c_void_p, c_int64, c_int, c_void_p]),
        "neumann_plan_set_launch": (c_int, [P, c_int, c_int]),
        "neumann_plan_autotune_batched": (c_int, [P, c_int, POINTER(c_int64), POINTER(c_void_p), POINTER(c_void_p),
                                                  c_int, c_void_p]),
        "neumann_measure_fma_peak": (c_int, [c_int, POINTER(c_double), POINTER(c_int), c_void_p]),
        "neumann_plan_destroy": (None, [P]),
        "neumann_error_string": (ctypes.c_char_p, [c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _check(rc: int, where: str) -> None:
    if rc != OK:
        raise NeumannError(rc, where)


def error_string(code: int) -> str:
    return _lib.neumann_error_string(code).decode()


def neumann_plan_create(n: int, k: int, radix: int, dtype: int, flags: int = 0) -> int:
    h = c_void_p()
    _check(_lib.neumann_plan_create(byref(h), n, k, radix, dtype, flags), "neumann_plan_create")
    return h.value


def neumann_plan_create_batched(count: int, max_n: int, k: int, radix: int, dtype: int, flags: int = 0) -> int:
    h = c_void_p()
    _check(_lib.neumann_plan_create_batched(byref(h), count, max_n, k, radix, dtype, flags),
           "neumann_plan_create_batched")
    return h.value


def neumann_plan_info(plan: int) -> dict:
    info = PlanInfo()
    _check(_lib.neumann_plan_info(plan, byref(info)), "neumann_plan_info")
    return {
        "n": info.n, "k": info.k, "radix": info.radix, "dtype": info.dtype, "flags": info.flags,
        "levels": list(info.level_radix[: info.levels]),
        "products_formula": info.products_formula, "products_executed": info.products_executed,
        "launches": info.launches, "workspace_bytes": info.workspace_bytes, "padded_n": info.padded_n,
        "tile_pair": info.tile_pair, "raster_group": info.raster_group, "batch_chunk": info.batch_chunk,
        "tuned": info.tuned, "bytes_per_element": info.bytes_per_element,
        "product_bytes_per_element": info.product_bytes_per_element,
        "resident_max_n": info.resident_max_n,
    }


def neumann_plan_set_workspace(plan: int, ptr: int, nbytes: int) -> None:
    _check(_lib.neumann_plan_set_workspace(plan, ptr, nbytes), "neumann_plan_set_workspace")


def neumann_eval(plan: int, A: int, lda: int, S: int, lds: int, stream: int = 0) -> None:
    _check(_lib.neumann_eval(plan, A, lda, S, lds, stream), "neumann_eval")


def neumann_eval_host(plan: int, A: int, lda: int, S: int, lds: int, stream: int = 0) -> None:
    _check(_lib.neumann_eval_host(plan, A, lda, S, lds, stream), "neumann_eval_host")


def neumann_eval_batched_host(plan: int, n, A: int, S: int, stream: int = 0) -> None:
    cnt = len(n)
    na = (c_int64 * cnt)(*n)
    _check(_lib.neumann_eval_batched_host(plan, cnt, na, A, S, stream), "neumann_eval_batched_host")


def neumann_plan_host_wait(plan: int) -> None:
    _check(_lib.neumann_plan_host_wait(plan), "neumann_plan_host_wait")


def neumann_plan_matmul(plan: int, A: int, B: int, C: int, stream: int = 0) -> None:
    _check(_lib.neumann_plan_matmul(plan, A, B, C, stream), "neumann_plan_matmul")


def neumann_eval_batched(plan: int, n, A, S, stream: int = 0) -> None:
    cnt = len(n)
    na = (c_int64 * cnt)(*n)
    aa = (c_void_p * cnt)(*A)
    sa = (c_void_p * cnt)(*S)
    _check(_lib.neumann_eval_batched(plan, cnt, na, aa, sa, stream), "neumann_eval_batched")


def neumann_plan_autotune(plan: int, A: int, lda: int, S: int, lds: int, reps: int = 3, stream: int = 0) -> None:
    _check(_lib.neumann_plan_autotune(plan, A, lda, S, lds, reps, stream), "neumann_plan_autotune")


def neumann_plan_set_launch(plan: int, tile_pair: int, raster_group: int) -> None:
    _check(_lib.neumann_plan_set_launch(plan, tile_pair, raster_group), "neumann_plan_set_launch")


def neumann_plan_autotune_batched(plan: int, n, A, S, reps: int = 3, stream: int = 0) -> None:
    cnt = len(n)
    na = (c_int64 * cnt)(*n)
    aa = (c_void_p * cnt)(*A)
    sa = (c_void_p * cnt)(*S)
    _check(_lib.neumann_plan_autotune_batched(plan, cnt, na, aa, sa, reps, stream), "neumann_plan_autotune_batched")


def neumann_last_status(plan: int) -> int:
    st = c_uint32(0)
    _check(_lib.neumann_last_status(plan, byref(st)), "neumann_last_status")
    return st.value


def neumann_plan_timing(plan: int, cap: int = 4096) -> list:
    buf = (c_float * cap)()
    cnt = c_int(0)
    _check(_lib.neumann_plan_timing(plan, buf, cap, byref(cnt)), "neumann_plan_timing")
    return [buf[i] for i in range(min(cnt.value, cap))]


def neumann_plan_selftest_timeout(plan: int, limit_ns: int, stream: int = 0) -> None:
    _check(_lib.neumann_plan_selftest_timeout(plan, limit_ns, stream), "neumann_plan_selftest_timeout")


def neumann_radix15_coefficients(coef_set: int = 0):
    c = (c_double * 28)()
    e, a, b = c_double(), c_double(), c_double()
    _check(_lib.neumann_radix15_coefficients(coef_set, c, byref(e), byref(a), byref(b)),
           "neumann_radix15_coefficients")
    return list(c), e.value, a.value, b.value


def neumann_radix_p5_coefficients(m: int):
    c = (c_double * 41)()
    e, a = c_double(), c_double()
    _check(_lib.neumann_radix_p5_coefficients(m, c, byref(e), byref(a)), "neumann_radix_p5_coefficients")
    return list(c), e.value, a.value


def neumann_matmul_noalloc(n: int, A: int, lda: int, B: int, ldb: int, C: int, ldc: int, stream: int = 0) -> None:
    """C = A B (FP64 in/out, split-BF16 tensor-core arithmetic) with no device
    allocation; the operand scratch is a fixed array inside the library, n <= 1024."""
    _check(_lib.neumann_matmul_noalloc(n, A, lda, B, ldb, C, ldc, stream), "neumann_matmul_noalloc")


def neumann_matmul_noalloc_status(stream: int = 0) -> int:
    """Synchronise `stream`; the NEUMANN_STATUS_* bits the allocation-free
    product set on the current device since the last read (then cleared)."""
    v = c_uint32()
    _check(_lib.neumann_matmul_noalloc_status(stream, byref(v)), "neumann_matmul_noalloc_status")
    return v.value


def neumann_measure_fma_peak(dtype: int, stream: int = 0):
    """(TFLOP/s of the CUDA cores' FMA pipe for FP32 or FP64, SM count) of the current device."""
    t, n = c_double(), c_int()
    _check(_lib.neumann_measure_fma_peak(dtype, byref(t), byref(n), stream), "neumann_measure_fma_peak")
    return t.value, n.value


def neumann_plan_destroy(plan: int) -> None:
    _lib.neumann_plan_destroy(plan)
