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
  // The pair is formed from RN_fp32(v): FP32 keeps 24 bits, the hi+lo pair 16.
  split_store(s, r, c, (float)v);
}

// Write 0 to every workspace destination of element (r, c), n <= r or c < npad
// (transposed splits excepted when kSkipT).
template <bool kSkipT = false>
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
      if (kSkipT && sp.transposed) continue;
      int64_t off = sp.transposed ? (int64_t)c * sp.ld + r : (int64_t)r * sp.ld + c;
      reinterpret_cast<__nv_bfloat16*>(sp.hi)[off] = __float2bfloat16_rn(0.f);
      reinterpret_cast<__nv_bfloat16*>(sp.lo)[off] = __float2bfloat16_rn(0.f);
    }
  }
}

// Apply every output of the epilogue to element (r, c) with accumulator value
// acc; r, c < npad. Inside the n x n block the outputs are formed; in the
// padding only workspace buffers are written (with 0). Returns true on a
// non-finite result.
// kDeferT: outputs' transposed split stores are not written; the value they
// would split (RN_fp32 of the output) is left in tv[j] for the caller to write
// through a shared-memory transpose (0 in the padding).
template <typename AccT, bool kDeferT>
__device__ __forceinline__ bool epi_element_impl(const EpiParams& P, int r, int c, AccT acc, float* tv) {
  bool bad = false;
  if (r >= P.n || c >= P.n) {
    if (kDeferT)
      for (int j = 0; j < kMaxOut; ++j) tv[j] = 0.f;
    epi_padding<kDeferT>(P, r, c);
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
      double v;
      if (sizeof(AccT) == 8) {
        v = o.acc_d * (double)acc + (diag ? o.id_d : 0.0);
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i) {
          if (i < P.nin && o.in_d[i] != 0.0)
            v += o.in_d[i] * (P.in[i].dt == DT_F64 ? din[i] : (double)fin[i]);
        }
      } else {
        // FP32 terms summed in FP32 (they carry FP32 rounding already); the FP64
        // inputs (a partial sum Y or residual R) are added in FP64, one DFMA each.
        float vf = o.acc_f * (float)acc;
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i)
          if (i < P.nin && o.in_f[i] != 0.f && P.in[i].dt != DT_F64) vf = fmaf(o.in_f[i], fin[i], vf);
        v = (double)vf + (diag ? o.id_d : 0.0);
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i)
          if (i < P.nin && o.in_d[i] != 0.0 && P.in[i].dt == DT_F64) v = fma(o.in_d[i], din[i], v);
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
      for (int s = 0; s < o.nsplit; ++s) {
        if (kDeferT && o.split[s].transposed)
          tv[j] = (float)v;
        else
          split_store_d(o.split[s], r, c, v);
      }
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
      for (int s = 0; s < o.nsplit; ++s) {
        if (kDeferT && o.split[s].transposed)
          tv[j] = v;
        else
          split_store(o.split[s], r, c, v);
      }
    }
  }
  return bad;
}

// One copy serves every call site of the GEMM kernels; P is a __grid_constant__
// kernel parameter, so passing it by reference copies nothing.
template <typename AccT>
__device__ __noinline__ bool epi_element(const EpiParams& P, int r, int c, AccT acc) {
  return epi_element_impl<AccT, false>(P, r, c, acc, nullptr);
}

// ---------------------------------------------------------------------------
// Vector form: W consecutive columns c0 .. c0+W-1 of row r, c0 % W == 0.
// Every input is loaded (as W-wide vectors) before any output is formed, so a
// thread keeps all of its loads in flight at once. Requires that every input
// and every pad destination is a workspace buffer (16-byte aligned, leading
// dimension a multiple of 8); the user's output (pad == 0) is written with
// scalar stores. Rows or columns outside the n x n block fall back to
// epi_element.

template <int W>
__device__ __forceinline__ void ld_vec(const float* p, float (&v)[W]) {
#pragma unroll
  for (int q = 0; q < W; q += 4) {
    float4 t = *reinterpret_cast<const float4*>(p + q);
    v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
  }
}

template <int W>
__device__ __forceinline__ void ld_vec(const double* p, double (&v)[W]) {
#pragma unroll
  for (int q = 0; q < W; q += 2) {
    double2 t = *reinterpret_cast<const double2*>(p + q);
    v[q] = t.x; v[q + 1] = t.y;
  }
}

template <int W, typename V>
__device__ __forceinline__ void st_row(const EpiOut& o, int r, int c0, const V (&v)[W]) {
  for (int d = 0; d < o.ndst; ++d) {
    const EpiDst& ds = o.dst[d];
    const int64_t off = (int64_t)r * ds.ld + c0;
    if (!ds.pad) {  // caller's matrix: any leading dimension
      if (ds.dt == DT_F64) {
#pragma unroll
        for (int w = 0; w < W; ++w) reinterpret_cast<double*>(ds.p)[off + w] = (double)v[w];
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w) reinterpret_cast<float*>(ds.p)[off + w] = (float)v[w];
      }
    } else if (ds.dt == DT_F64) {
      double* q = reinterpret_cast<double*>(ds.p) + off;
#pragma unroll
      for (int w = 0; w < W; w += 2) *reinterpret_cast<double2*>(q + w) = make_double2((double)v[w], (double)v[w + 1]);
    } else {
      float* q = reinterpret_cast<float*>(ds.p) + off;
#pragma unroll
      for (int w = 0; w < W; w += 4)
        *reinterpret_cast<float4*>(q + w) = make_float4((float)v[w], (float)v[w + 1], (float)v[w + 2], (float)v[w + 3]);
    }
  }
  for (int s = 0; s < o.nsplit; ++s) {
    const EpiSplit& sp = o.split[s];
    __nv_bfloat16 hi[W], lo[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {  // from RN_fp32(v): FP32 keeps 24 bits, the pair 16
      const float vf = (float)v[w];
      hi[w] = __float2bfloat16_rn(vf);
      lo[w] = __float2bfloat16_rn(vf - __bfloat162float(hi[w]));
    }
    if (sp.transposed) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int64_t off = (int64_t)(c0 + w) * sp.ld + r;
        reinterpret_cast<__nv_bfloat16*>(sp.hi)[off] = hi[w];
        reinterpret_cast<__nv_bfloat16*>(sp.lo)[off] = lo[w];
      }
    } else {
      const int64_t off = (int64_t)r * sp.ld + c0;
      static_assert(W == 4 || W == 8, "vector width");
      uint32_t ph[W / 2], pl[W / 2];
#pragma unroll
      for (int q = 0; q < W / 2; ++q) {
        ph[q] = (uint32_t)__bfloat16_as_ushort(hi[2 * q]) | ((uint32_t)__bfloat16_as_ushort(hi[2 * q + 1]) << 16);
        pl[q] = (uint32_t)__bfloat16_as_ushort(lo[2 * q]) | ((uint32_t)__bfloat16_as_ushort(lo[2 * q + 1]) << 16);
      }
      __nv_bfloat16* qh = reinterpret_cast<__nv_bfloat16*>(sp.hi) + off;
      __nv_bfloat16* ql = reinterpret_cast<__nv_bfloat16*>(sp.lo) + off;
      if constexpr (W == 8) {
        *reinterpret_cast<uint4*>(qh) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
        *reinterpret_cast<uint4*>(ql) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
      } else {
        *reinterpret_cast<uint2*>(qh) = make_uint2(ph[0], ph[1]);
        *reinterpret_cast<uint2*>(ql) = make_uint2(pl[0], pl[1]);
      }
    }
  }
}

template <int W, typename AccT>
__device__ __forceinline__ bool epi_row(const EpiParams& P, int r, int c0, const AccT (&acc)[W]) {
  if (r >= P.n || c0 + W > P.n) {
    bool bad = false;
#pragma unroll
    for (int w = 0; w < W; ++w) bad |= epi_element<AccT>(P, r, c0 + w, acc[w]);
    return bad;
  }
  float fin[kMaxIn][W];
  double din[kMaxIn][W];
#pragma unroll
  for (int i = 0; i < kMaxIn; ++i) {
    if (i < P.nin) {
      const EpiIn& in = P.in[i];
      const int64_t off = (int64_t)r * in.ld + c0;
      if (in.dt == DT_F64)
        ld_vec<W>(reinterpret_cast<const double*>(in.p) + off, din[i]);
      else
        ld_vec<W>(reinterpret_cast<const float*>(in.p) + off, fin[i]);
    }
  }
  bool bad = false;
#pragma unroll 1
  for (int j = 0; j < P.nout; ++j) {
    const EpiOut& o = P.out[j];
    if (o.f64) {
      double v[W];
      if (sizeof(AccT) == 8) {
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = o.acc_d * (double)acc[w] + (r == c0 + w ? o.id_d : 0.0);
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i) {
          if (i < P.nin && o.in_d[i] != 0.0) {
            const bool f = P.in[i].dt == DT_F64;
#pragma unroll
            for (int w = 0; w < W; ++w) v[w] += o.in_d[i] * (f ? din[i][w] : (double)fin[i][w]);
          }
        }
      } else {
        // FP32 terms in FP32, then one DFMA per FP64 input (see epi_element)
        float vf[W];
#pragma unroll
        for (int w = 0; w < W; ++w) vf[w] = o.acc_f * (float)acc[w];
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i) {
          if (i < P.nin && o.in_f[i] != 0.f && P.in[i].dt != DT_F64) {
#pragma unroll
            for (int w = 0; w < W; ++w) vf[w] = fmaf(o.in_f[i], fin[i][w], vf[w]);
          }
        }
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = (double)vf[w] + (r == c0 + w ? o.id_d : 0.0);
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i) {
          if (i < P.nin && o.in_d[i] != 0.0 && P.in[i].dt == DT_F64) {
#pragma unroll
            for (int w = 0; w < W; ++w) v[w] = fma(o.in_d[i], din[i][w], v[w]);
          }
        }
      }
#pragma unroll
      for (int w = 0; w < W; ++w) bad |= !isfinite(v[w]);
      st_row<W, double>(o, r, c0, v);
    } else {
      float v[W];
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = o.acc_f * (float)acc[w] + (r == c0 + w ? o.id_f : 0.f);
#pragma unroll
      for (int i = 0; i < kMaxIn; ++i) {
        if (i < P.nin && o.in_f[i] != 0.f) {
          const bool f = P.in[i].dt == DT_F64;
#pragma unroll
          for (int w = 0; w < W; ++w) v[w] = fmaf(o.in_f[i], f ? (float)din[i][w] : fin[i][w], v[w]);
        }
      }
#pragma unroll
      for (int w = 0; w < W; ++w) bad |= !isfinite(v[w]);
      st_row<W, float>(o, r, c0, v);
    }
  }
  return bad;
}

__device__ __forceinline__ void epi_flag(const EpiParams& P, bool bad) {
  if (bad && P.status) atomicOr(P.status, 1u);
}

}  // namespace neumann
