// Fused epilogue: every product of a radix level leaves its accumulator in
// registers and this code forms the linear combinations the next product
// (and the partial-sum / residual updates) need, e.g. for Thm 3.1
//   MM2: P = 3/20 B + 2U + acc, Q = 11/40 B - 1/8 U + 1/4 acc, C = B + 767/800 U + 15/32 acc,
// writing each result in every representation its consumers read: FP32 / FP64
// row-major, and hi/lo BF16 pairs row-major (left operands) or transposed
// (right operands of the tensor-core product).
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace neumann {

__device__ __forceinline__ void split_store(const EpiSplit& s, int r, int c, float v) {
  __nv_bfloat16 hi = __float2bfloat16_rn(v);
  __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  int64_t off = s.transposed ? (int64_t)c * s.ld + r : (int64_t)r * s.ld + c;
  reinterpret_cast<__nv_bfloat16*>(s.hi)[off] = hi;
  reinterpret_cast<__nv_bfloat16*>(s.lo)[off] = lo;
}

__device__ __forceinline__ void split_store_d(const EpiSplit& s, int r, int c, double v) {
  // hi = RN_bf16(v) through FP32: v -> f32 is exact to 2^-24 relative, far below
  // the 2^-17 the hi+lo pair keeps.
  float vf = (float)v;
  __nv_bfloat16 hi = __float2bfloat16_rn(vf);
  float rem = (float)(v - (double)__bfloat162float(hi));
  __nv_bfloat16 lo = __float2bfloat16_rn(rem);
  int64_t off = s.transposed ? (int64_t)c * s.ld + r : (int64_t)r * s.ld + c;
  reinterpret_cast<__nv_bfloat16*>(s.hi)[off] = hi;
  reinterpret_cast<__nv_bfloat16*>(s.lo)[off] = lo;
}

// Write 0 to every workspace destination of element (r, c), n <= r or c < npad.
__device__ __forceinline__ void epi_padding(const EpiParams& P, int r, int c) {
#pragma unroll 1
  for (int j = 0; j < P.nout; ++j) {
    const EpiOut& o = P.out[j];
    for (int d = 0; d < o.ndst; ++d) {
      const EpiDst& ds = o.dst[d];
      if (!ds.pad) continue;
      int64_t off = (int64_t)r * ds.ld + c;
      if (ds.dt == DT_F64)
        reinterpret_cast<double*>(ds.p)[off] = 0.0;
      else
        reinterpret_cast<float*>(ds.p)[off] = 0.f;
    }
    for (int s = 0; s < o.nsplit; ++s) {
      const EpiSplit& sp = o.split[s];
      int64_t off = sp.transposed ? (int64_t)c * sp.ld + r : (int64_t)r * sp.ld + c;
      reinterpret_cast<__nv_bfloat16*>(sp.hi)[off] = __float2bfloat16_rn(0.f);
      reinterpret_cast<__nv_bfloat16*>(sp.lo)[off] = __float2bfloat16_rn(0.f);
    }
  }
}

// Apply every output of the epilogue to element (r, c) with accumulator value
// acc; r, c < npad. Inside the n x n block the outputs are formed; in the
// padding only workspace buffers are written (with 0). Returns true on a
// non-finite result. Not inlined: one copy serves every call site, and P is a
// __grid_constant__ kernel parameter, so passing it by reference copies nothing.
template <typename AccT>
__device__ __noinline__ bool epi_element(const EpiParams& P, int r, int c, AccT acc) {
  bool bad = false;
  if (r >= P.n || c >= P.n) {
    epi_padding(P, r, c);
    return false;
  }
  float fin[kMaxIn];
  double din[kMaxIn];
#pragma unroll
  for (int i = 0; i < kMaxIn; ++i) {
    fin[i] = 0.f;
    din[i] = 0.0;
    if (i < P.nin) {
      const EpiIn& in = P.in[i];
      int64_t off = (int64_t)r * in.ld + c;
      if (in.dt == DT_F64) {
        din[i] = reinterpret_cast<const double*>(in.p)[off];
      } else {
        fin[i] = reinterpret_cast<const float*>(in.p)[off];
      }
    }
  }
  const bool diag = (r == c);
#pragma unroll 1
  for (int j = 0; j < P.nout; ++j) {
    const EpiOut& o = P.out[j];
    if (o.f64) {
      double v = o.acc_d * (double)acc + (diag ? o.id_d : 0.0);
#pragma unroll
      for (int i = 0; i < kMaxIn; ++i) {
        if (i < P.nin && o.in_d[i] != 0.0)
          v += o.in_d[i] * (P.in[i].dt == DT_F64 ? din[i] : (double)fin[i]);
      }
      if (!isfinite(v)) bad = true;
      for (int d = 0; d < o.ndst; ++d) {
        const EpiDst& ds = o.dst[d];
        int64_t off = (int64_t)r * ds.ld + c;
        if (ds.dt == DT_F64)
          reinterpret_cast<double*>(ds.p)[off] = v;
        else
          reinterpret_cast<float*>(ds.p)[off] = (float)v;
      }
      for (int s = 0; s < o.nsplit; ++s) split_store_d(o.split[s], r, c, v);
    } else {
      float v = o.acc_f * (float)acc + (diag ? o.id_f : 0.f);
#pragma unroll
      for (int i = 0; i < kMaxIn; ++i) {
        if (i < P.nin && o.in_f[i] != 0.f)
          v = fmaf(o.in_f[i], P.in[i].dt == DT_F64 ? (float)din[i] : fin[i], v);
      }
      if (!isfinite(v)) bad = true;
      for (int d = 0; d < o.ndst; ++d) {
        const EpiDst& ds = o.dst[d];
        int64_t off = (int64_t)r * ds.ld + c;
        if (ds.dt == DT_F64)
          reinterpret_cast<double*>(ds.p)[off] = (double)v;
        else
          reinterpret_cast<float*>(ds.p)[off] = v;
      }
      for (int s = 0; s < o.nsplit; ++s) split_store(o.split[s], r, c, v);
    }
  }
  return bad;
}

__device__ __forceinline__ void epi_flag(const EpiParams& P, bool bad) {
  if (bad && P.status) atomicOr(P.status, 1u);
}

}  // namespace neumann
