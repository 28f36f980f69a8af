// Fused epilogue: every product of a radix level leaves its accumulator in
// registers and this code forms the linear combinations the next product
// (and the partial-sum / residual updates) need, e.g. for Thm 3.1
//   MM2: P = 3/20 B + 2U + acc, Q = 11/40 B - 1/8 U + 1/4 acc, C = B + 767/800 U + 15/32 acc,
// writing each result in every representation its consumers read: FP32 / FP64
// row-major, and hi/lo BF16 pairs row-major (left operands) or transposed
// (right operands of the tensor-core product).
//
// An EpiCtx fixes the matrix a tile belongs to: its order n and the offset of
// its slab in the workspace buffers (0 for a single evaluation).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace neumann {

struct EpiCtx {
  int n;        // order of this matrix
  int mat;      // index in the batch (0 for a single evaluation)
  int64_t off;  // element offset of its slab in every workspace buffer
};

__device__ __forceinline__ EpiCtx epi_ctx(const EpiParams& P, int mat) {
  EpiCtx x;
  x.mat = mat;
  if (P.mat_n) {
    x.n = P.mat_n[mat];
    x.off = (int64_t)mat * P.mat_stride;
  } else {
    x.n = P.n;
    x.off = 0;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ const T* in_base(const EpiIn& in, const EpiCtx& x, int64_t* ld) {
  if (in.mode == EPI_WS) {
    *ld = in.ld;
    return reinterpret_cast<const T*>(in.p) + x.off;
  }
  if (in.mode == EPI_TABLE) {
    *ld = x.n;
    return reinterpret_cast<const T*>(reinterpret_cast<const void* const*>(in.p)[x.mat]);
  }
  *ld = in.ld;
  return reinterpret_cast<const T*>(in.p);
}

template <typename T>
__device__ __forceinline__ T* dst_base(const EpiDst& ds, const EpiCtx& x, int64_t* ld) {
  if (ds.mode == EPI_WS) {
    *ld = ds.ld;
    return reinterpret_cast<T*>(ds.p) + x.off;
  }
  if (ds.mode == EPI_TABLE) {
    *ld = x.n;
    return reinterpret_cast<T*>(reinterpret_cast<void* const*>(ds.p)[x.mat]);
  }
  *ld = ds.ld;
  return reinterpret_cast<T*>(ds.p);
}

// The 16-bit hi/lo pair of v as raw bits (BF16, or FP16 of v * sc with the
// matrix's power of two sc; see EpiSplit). kF16 is a compile-time choice: a
// kernel instance serves one split type.
template <bool kF16>
__device__ __forceinline__ void split_bits(float v, float sc, unsigned short* hi, unsigned short* lo) {
  if (kF16) {
    const float w = v * sc;
    const __half h = __float2half_rn(w);
    *hi = __half_as_ushort(h);
    *lo = __half_as_ushort(__float2half_rn(w - __half2float(h)));
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *hi = __bfloat16_as_ushort(h);
    *lo = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
  }
}

// An FP16 hi that overflowed (|v| * sc beyond the FP16 range) is non-finite.
template <bool kF16>
__device__ __forceinline__ bool split_bad(float v, float sc) {
  return kF16 && !(fabsf(v) * sc < 65504.f);
}

template <bool kF16>
__device__ __forceinline__ void split_store(const EpiSplit& s, const EpiCtx& x, int r, int c, float v, float sc) {
  unsigned short hi, lo;
  split_bits<kF16>(v, sc, &hi, &lo);
  int64_t off = x.off + (s.transposed ? (int64_t)c * s.ld + r : (int64_t)r * s.ld + c);
  reinterpret_cast<unsigned short*>(s.hi)[off] = hi;
  reinterpret_cast<unsigned short*>(s.lo)[off] = lo;
}

// ---------------------------------------------------------------------------
// Split-FP16 scaling (SxParams): the scales of one launch for matrix `mat`,
// read once per tile.
__device__ __forceinline__ void sx_tile(const EpiParams& P, int mat, SxTile* t) {
  const SxParams& q = P.sx;
  const int64_t m = mat;
  t->acc = 1.f;
  if (q.active && q.rec_a >= 0)
    t->acc = ldexpf(1.f, -(q.exp[q.rec_a * (int64_t)q.nmat + m] + q.exp[q.rec_b * (int64_t)q.nmat + m]));
#pragma unroll
  for (int j = 0; j < kMaxOut; ++j) {
    const int rec = (q.active && j < P.nout) ? q.rec_out[j] : -1;
    t->sc[j] = rec >= 0 ? ldexpf(1.f, q.exp[rec * (int64_t)q.nmat + m]) : 1.f;
  }
}

// Write 0 to every workspace destination of element (r, c) outside the n x n
// block (transposed splits excepted when kSkipT).
template <bool kSkipT = false>
__device__ __forceinline__ void epi_padding(const EpiParams& P, const EpiCtx& x, int r, int c) {
#pragma unroll 1
  for (int j = 0; j < P.nout; ++j) {
    const EpiOut& o = P.out[j];
    for (int d = 0; d < o.ndst; ++d) {
      const EpiDst& ds = o.dst[d];
      if (ds.mode != EPI_WS) continue;
      const int64_t off = x.off + (int64_t)r * ds.ld + c;
      if (ds.dt == DT_F64)
        reinterpret_cast<double*>(ds.p)[off] = 0.0;
      else
        reinterpret_cast<float*>(ds.p)[off] = 0.f;
    }
    for (int s = 0; s < o.nsplit; ++s) {
      const EpiSplit& sp = o.split[s];
      if (kSkipT && sp.transposed) continue;
      const int64_t off = x.off + (sp.transposed ? (int64_t)c * sp.ld + r : (int64_t)r * sp.ld + c);
      reinterpret_cast<unsigned short*>(sp.hi)[off] = 0;  // +0 in BF16 and FP16
      reinterpret_cast<unsigned short*>(sp.lo)[off] = 0;
    }
  }
}

// Apply every output of the epilogue to element (r, c) of matrix x with
// accumulator value acc. Inside the n x n block the outputs are formed; in the
// padding only workspace buffers are written (with 0). Returns true on a
// non-finite result.
// kDeferT: outputs' transposed split stores are not written; the value they
// would split (RN_fp32 of the output) is left in tv[j] for the caller to write
// through a shared-memory transpose (0 in the padding).
// t: split-FP16 scales and records of this tile (nullptr for other dtypes).
template <typename AccT, bool kDeferT, bool kF16>
__device__ __forceinline__ bool epi_element_impl(const EpiParams& P, const EpiCtx& x, int r, int c, AccT acc,
                                                 float* tv, const SxTile* t) {
  bool bad = false;
  if (r >= x.n || c >= x.n) {
    if (kDeferT)
      for (int j = 0; j < kMaxOut; ++j) tv[j] = 0.f;
    epi_padding<kDeferT>(P, x, r, c);
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
      int64_t ld;
      if (in.dt == DT_F64)
        din[i] = in_base<double>(in, x, &ld)[(int64_t)r * ld + c];
      else
        fin[i] = in_base<float>(in, x, &ld)[(int64_t)r * ld + c];
    }
  }
  const bool diag = (r == c);
#pragma unroll 1
  for (int j = 0; j < P.nout; ++j) {
    const EpiOut& o = P.out[j];
    double v;
    float vf;
    if (o.f64) {
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
        float tt = (kF16 && t ? o.acc_f * t->acc : o.acc_f) * (float)acc;
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i)
          if (i < P.nin && o.in_f[i] != 0.f && P.in[i].dt != DT_F64) tt = fmaf(o.in_f[i], fin[i], tt);
        v = (double)tt + (diag ? o.id_d : 0.0);
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i)
          if (i < P.nin && o.in_d[i] != 0.0 && P.in[i].dt == DT_F64) v = fma(o.in_d[i], din[i], v);
      }
      vf = (float)v;
      if (!isfinite(v)) bad = true;
    } else {
      vf = (kF16 && t ? o.acc_f * t->acc : o.acc_f) * (float)acc + (diag ? o.id_f : 0.f);
#pragma unroll
      for (int i = 0; i < kMaxIn; ++i) {
        if (i < P.nin && o.in_f[i] != 0.f)
          vf = fmaf(o.in_f[i], P.in[i].dt == DT_F64 ? (float)din[i] : fin[i], vf);
      }
      v = 0.0;  // unused: no FP64 destination is written from an FP32 output
      if (!isfinite(vf)) bad = true;
    }
    const float sc = kF16 && t ? t->sc[j] : 1.f;
    for (int d = 0; d < o.ndst; ++d) {
      const EpiDst& ds = o.dst[d];
      int64_t ld;
      if (ds.dt == DT_F64)
        dst_base<double>(ds, x, &ld)[(int64_t)r * ld + c] = o.f64 ? v : (double)vf;
      else
        dst_base<float>(ds, x, &ld)[(int64_t)r * ld + c] = vf;
    }
    // hi/lo pairs are formed from RN_fp32 of the output: FP32 keeps 24 bits, the pair 16
    for (int s = 0; s < o.nsplit; ++s) {
      bad |= split_bad<kF16>(vf, sc);
      if (kDeferT && o.split[s].transposed)
        tv[j] = vf;
      else
        split_store<kF16>(o.split[s], x, r, c, vf, sc);
    }
  }
  return bad;
}

// One copy serves every call site of the GEMM kernels; P is a __grid_constant__
// kernel parameter, so passing it by reference copies nothing.
template <typename AccT, bool kF16>
__device__ __noinline__ bool epi_element(const EpiParams& P, EpiCtx x, int r, int c, AccT acc,
                                         const SxTile* t = nullptr) {
  return epi_element_impl<AccT, false, kF16>(P, x, r, c, acc, nullptr, t);
}

// ---------------------------------------------------------------------------
// Vector form: W consecutive columns c0 .. c0+W-1 of row r, c0 % W == 0.
// Every input is loaded (as W-wide vectors) before any output is formed, so a
// thread keeps all of its loads in flight at once. Used by the products,
// whose inputs are all workspace buffers (16-byte aligned, leading dimension a
// multiple of 8); caller-owned outputs are written with scalar stores. Rows or
// columns outside the n x n block fall back to epi_element.

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

// kWsOnly: write workspace destinations only (padding zeros never go to the caller).
// sc: the output's split-FP16 scale.
template <int W, typename V, bool kF16, bool kWsOnly = false>
__device__ __forceinline__ void st_row(const EpiOut& o, const EpiCtx& x, int r, int c0, const V (&v)[W],
                                       float sc = 1.f) {
  for (int d = 0; d < o.ndst; ++d) {
    const EpiDst& ds = o.dst[d];
    int64_t ld;
    if (kWsOnly && ds.mode != EPI_WS) continue;
    if (ds.mode != EPI_WS) {  // caller's matrix: any leading dimension
      if (ds.dt == DT_F64) {
        double* q = dst_base<double>(ds, x, &ld) + (int64_t)r * ld + c0;
#pragma unroll
        for (int w = 0; w < W; ++w) q[w] = (double)v[w];
      } else {
        float* q = dst_base<float>(ds, x, &ld) + (int64_t)r * ld + c0;
#pragma unroll
        for (int w = 0; w < W; ++w) q[w] = (float)v[w];
      }
    } else if (ds.dt == DT_F64) {
      double* q = dst_base<double>(ds, x, &ld) + (int64_t)r * ld + c0;
#pragma unroll
      for (int w = 0; w < W; w += 2) *reinterpret_cast<double2*>(q + w) = make_double2((double)v[w], (double)v[w + 1]);
    } else {
      float* q = dst_base<float>(ds, x, &ld) + (int64_t)r * ld + c0;
#pragma unroll
      for (int w = 0; w < W; w += 4)
        *reinterpret_cast<float4*>(q + w) = make_float4((float)v[w], (float)v[w + 1], (float)v[w + 2], (float)v[w + 3]);
    }
  }
  for (int s = 0; s < o.nsplit; ++s) {
    const EpiSplit& sp = o.split[s];
    unsigned short hi[W], lo[W];
#pragma unroll
    for (int w = 0; w < W; ++w) split_bits<kF16>((float)v[w], sc, &hi[w], &lo[w]);  // from RN_fp32(v)
    if (sp.transposed) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int64_t off = x.off + (int64_t)(c0 + w) * sp.ld + r;
        reinterpret_cast<unsigned short*>(sp.hi)[off] = hi[w];
        reinterpret_cast<unsigned short*>(sp.lo)[off] = lo[w];
      }
    } else {
      const int64_t off = x.off + (int64_t)r * sp.ld + c0;
      static_assert(W == 4 || W == 8, "vector width");
      uint32_t ph[W / 2], pl[W / 2];
#pragma unroll
      for (int q = 0; q < W / 2; ++q) {
        ph[q] = (uint32_t)hi[2 * q] | ((uint32_t)hi[2 * q + 1] << 16);
        pl[q] = (uint32_t)lo[2 * q] | ((uint32_t)lo[2 * q + 1] << 16);
      }
      unsigned short* qh = reinterpret_cast<unsigned short*>(sp.hi) + off;
      unsigned short* ql = reinterpret_cast<unsigned short*>(sp.lo) + off;
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

// Zeros for W consecutive padding elements of row r (r >= n) in every workspace
// destination.
template <int W, bool kF16>
__device__ __forceinline__ void epi_row_zero(const EpiParams& P, const EpiCtx& x, int r, int c0) {
  float z[W];
#pragma unroll
  for (int w = 0; w < W; ++w) z[w] = 0.f;
#pragma unroll 1
  for (int j = 0; j < P.nout; ++j) st_row<W, float, kF16, true>(P.out[j], x, r, c0, z);
}

// A scaled FP16 split of any of these values overflows.
template <int W, typename V, bool kF16>
__device__ __forceinline__ bool fp16_overflow(const EpiOut& o, const V (&v)[W], float sc) {
  if (!kF16 || o.nsplit == 0) return false;
  bool bad = false;
#pragma unroll
  for (int w = 0; w < W; ++w) bad |= !(fabsf((float)v[w]) * sc < 65504.f);
  return bad;
}

template <int W, typename AccT, bool kF16>
__device__ __forceinline__ bool epi_row(const EpiParams& P, const EpiCtx& x, int r, int c0,
                                        const AccT (&acc)[W]) {
  if (r >= x.n) {
    epi_row_zero<W, kF16>(P, x, r, c0);
    return false;
  }
  if (c0 + W > x.n) {
    bool bad = false;
#pragma unroll
    for (int w = 0; w < W; ++w) bad |= epi_element<AccT, kF16>(P, x, r, c0 + w, acc[w]);
    return bad;
  }
  float fin[kMaxIn][W];
  double din[kMaxIn][W];
#pragma unroll
  for (int i = 0; i < kMaxIn; ++i) {
    if (i < P.nin) {
      const EpiIn& in = P.in[i];
      const int64_t off = x.off + (int64_t)r * in.ld + c0;
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
        // FP32 terms in FP32, then one DFMA per FP64 input (see epi_element_impl)
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
      bad |= fp16_overflow<W, double, kF16>(o, v, 1.f);
      st_row<W, double, kF16>(o, x, r, c0, v);
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
      bad |= fp16_overflow<W, float, kF16>(o, v, 1.f);
      st_row<W, float, kF16>(o, x, r, c0, v);
    }
  }
  return bad;
}

// ---------------------------------------------------------------------------
// Column form: W consecutive rows r0 .. r0+W-1 of column c (r0 % W == 0). A
// warp whose lanes own consecutive columns reads and writes every row-major
// buffer one cache line per instruction; a transposed hi/lo store is one
// W x 2-byte run per lane. Requires W == 8 (16-byte transposed runs).

template <int W, bool kF16>
__device__ __forceinline__ void st_col_split(const EpiSplit& sp, const EpiCtx& x, int r0, int c, const float (&v)[W],
                                             float sc) {
  unsigned short hi[W], lo[W];
#pragma unroll
  for (int w = 0; w < W; ++w) split_bits<kF16>(v[w], sc, &hi[w], &lo[w]);
  if (sp.transposed) {
    uint32_t ph[W / 2], pl[W / 2];
#pragma unroll
    for (int q = 0; q < W / 2; ++q) {
      ph[q] = (uint32_t)hi[2 * q] | ((uint32_t)hi[2 * q + 1] << 16);
      pl[q] = (uint32_t)lo[2 * q] | ((uint32_t)lo[2 * q + 1] << 16);
    }
    const int64_t off = x.off + (int64_t)c * sp.ld + r0;
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned short*>(sp.hi) + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned short*>(sp.lo) + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int64_t off = x.off + (int64_t)(r0 + w) * sp.ld + c;
      reinterpret_cast<unsigned short*>(sp.hi)[off] = hi[w];
      reinterpret_cast<unsigned short*>(sp.lo)[off] = lo[w];
    }
  }
}

// kWsOnly: padding, workspace destinations only
template <int W, typename V, bool kF16, bool kWsOnly = false>
__device__ __forceinline__ void st_col(const EpiOut& o, const EpiCtx& x, int r0, int c, const V (&v)[W],
                                       float sc = 1.f) {
  for (int d = 0; d < o.ndst; ++d) {
    const EpiDst& ds = o.dst[d];
    if (kWsOnly && ds.mode != EPI_WS) continue;
    int64_t ld;
    if (ds.dt == DT_F64) {
      double* q = dst_base<double>(ds, x, &ld) + c;
#pragma unroll
      for (int w = 0; w < W; ++w) q[(int64_t)(r0 + w) * ld] = (double)v[w];
    } else {
      float* q = dst_base<float>(ds, x, &ld) + c;
#pragma unroll
      for (int w = 0; w < W; ++w) q[(int64_t)(r0 + w) * ld] = (float)v[w];
    }
  }
  if (o.nsplit) {
    float vf[W];
#pragma unroll
    for (int w = 0; w < W; ++w) vf[w] = (float)v[w];  // pairs from RN_fp32 of the output
    for (int s = 0; s < o.nsplit; ++s) st_col_split<W, kF16>(o.split[s], x, r0, c, vf, sc);
  }
}

template <int W, typename AccT, bool kF16>
__device__ __forceinline__ bool epi_col(const EpiParams& P, const EpiCtx& x, int r0, int c, const AccT (&acc)[W],
                                        const SxTile* t = nullptr) {
  static_assert(W == 8, "transposed runs are 16 bytes");
  static_assert(sizeof(AccT) == 4, "FP32 accumulators (tensor-core products)");
  if (c >= x.n || r0 >= x.n) {  // the whole run is padding
    float z[W];
#pragma unroll
    for (int w = 0; w < W; ++w) z[w] = 0.f;
#pragma unroll 1
    for (int j = 0; j < P.nout; ++j) st_col<W, float, kF16, true>(P.out[j], x, r0, c, z);
    return false;
  }
  if (r0 + W > x.n) {  // ragged edge
    bool bad = false;
#pragma unroll
    for (int w = 0; w < W; ++w) bad |= epi_element<AccT, kF16>(P, x, r0 + w, c, acc[w], t);
    return bad;
  }
  float fin[kMaxIn][W];
  double din[kMaxIn][W];
#pragma unroll
  for (int i = 0; i < kMaxIn; ++i) {
    if (i < P.nin) {
      const EpiIn& in = P.in[i];
      if (in.dt == DT_F64) {
        const double* q = reinterpret_cast<const double*>(in.p) + x.off + (int64_t)r0 * in.ld + c;
#pragma unroll
        for (int w = 0; w < W; ++w) din[i][w] = q[(int64_t)w * in.ld];
      } else {
        const float* q = reinterpret_cast<const float*>(in.p) + x.off + (int64_t)r0 * in.ld + c;
#pragma unroll
        for (int w = 0; w < W; ++w) fin[i][w] = q[(int64_t)w * in.ld];
      }
    }
  }
  bool bad = false;
#pragma unroll 1
  for (int j = 0; j < P.nout; ++j) {
    const EpiOut& o = P.out[j];
    if (o.f64) {
      double v[W];
      float vf[W];
      const float af = kF16 && t ? o.acc_f * t->acc : o.acc_f;
#pragma unroll
      for (int w = 0; w < W; ++w) vf[w] = af * (float)acc[w];
#pragma unroll
      for (int i = 0; i < kMaxIn; ++i) {
        if (i < P.nin && o.in_f[i] != 0.f && P.in[i].dt != DT_F64) {
#pragma unroll
          for (int w = 0; w < W; ++w) vf[w] = fmaf(o.in_f[i], fin[i][w], vf[w]);
        }
      }
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = (double)vf[w] + (r0 + w == c ? o.id_d : 0.0);
#pragma unroll
      for (int i = 0; i < kMaxIn; ++i) {
        if (i < P.nin && o.in_d[i] != 0.0 && P.in[i].dt == DT_F64) {
#pragma unroll
          for (int w = 0; w < W; ++w) v[w] = fma(o.in_d[i], din[i][w], v[w]);
        }
      }
#pragma unroll
      for (int w = 0; w < W; ++w) bad |= !isfinite(v[w]);
      const float sc = kF16 && t ? t->sc[j] : 1.f;
      bad |= fp16_overflow<W, double, kF16>(o, v, sc);
      st_col<W, double, kF16>(o, x, r0, c, v, sc);
    } else {
      float v[W];
      const float af = kF16 && t ? o.acc_f * t->acc : o.acc_f;
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = af * (float)acc[w] + (r0 + w == c ? o.id_f : 0.f);
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
      const float sc = kF16 && t ? t->sc[j] : 1.f;
      bad |= fp16_overflow<W, float, kF16>(o, v, sc);
      st_col<W, float, kF16>(o, x, r0, c, v, sc);
    }
  }
  return bad;
}

// ---------------------------------------------------------------------------
// Chunk form for the tensor-core products: rows rbase .. rbase+31 of column c,
// the accumulator of row rbase + i at stg[i * 33 + lane] (the warp's staged
// 32 x 32 chunk). Chunks of ops the host marked `fast` (at most one FP64 input,
// index f64_in) take a lean path: input addresses formed once per 8 rows, the
// identity only on the diagonal element, non-finite results (and FP16 split
// overflow) detected once per chunk, hi/lo pairs from paired RN conversions
// (cvt.rn.bf16x2 / f16x2). Boundary chunks take it too when `edge_ok` (zeros
// outside the n x n block); symmetric mirrors there, caller-owned inputs and
// rows past a grouped tile's limit go through epi_col row group by row group.

// hi/lo of (a, b) as packed pairs: low half from a, high half from b.
template <bool kF16>
__device__ __forceinline__ void split2(float a, float b, float sc, uint32_t* hi, uint32_t* lo) {
  if (kF16) {
    const float wa = a * sc, wb = b * sc;
    const __half2 h = __floats2half2_rn(wa, wb);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(wa - hf.x, wb - hf.y);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// Split stores of 8 consecutive rows r0 .. r0+7 of column c.
template <bool kF16>
__device__ __forceinline__ void st8_split(const EpiSplit& sp, const EpiCtx& x, int r0, int c, const float (&v)[8],
                                          float sc) {
  uint32_t ph[4], pl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) split2<kF16>(v[2 * q], v[2 * q + 1], sc, &ph[q], &pl[q]);
  unsigned short* hi = reinterpret_cast<unsigned short*>(sp.hi) + x.off;
  unsigned short* lo = reinterpret_cast<unsigned short*>(sp.lo) + x.off;
  if (sp.transposed) {  // row c of the stored transpose, 8 consecutive entries: one 16-byte store each
    const int64_t off = (int64_t)c * sp.ld + r0;
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
    *reinterpret_cast<uint4*>(lo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
  } else {  // row-major: the warp's lanes write 32 consecutive entries of each row
    const int64_t ld = sp.ld;
    hi += (int64_t)r0 * ld + c;
    lo += (int64_t)r0 * ld + c;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hi[(2 * q) * ld] = (unsigned short)(ph[q] & 0xffffu);
      hi[(2 * q + 1) * ld] = (unsigned short)(ph[q] >> 16);
      lo[(2 * q) * ld] = (unsigned short)(pl[q] & 0xffffu);
      lo[(2 * q + 1) * ld] = (unsigned short)(pl[q] >> 16);
    }
  }
}

// The lean path proper. Rows are taken RB at a time: every input load of the
// RB rows is issued before any output is formed, so a lane keeps RB x (inputs)
// loads in flight; the host's input count picks RB (32 rows for one FP32
// input, 16 for two, or one FP32 and one FP64, 8 otherwise) so that about 32
// loads per lane are in flight whatever the op. NF: FP32 input slots (the
// op's FP32 inputs in index order, P.f32_idx); kD: the op may have an FP64 input.
// Symmetric products: a tile above the diagonal also writes its transpose.
// The run (r0 .. r0+7, c) lands at (c, r0 .. r0+7), 8 consecutive entries of
// row c: vector stores into workspace buffers (leading dimension npad, r0 a
// multiple of 8), scalar stores into a caller's matrix.
__device__ __forceinline__ void st8_mirror_dst(const EpiOut& o, const EpiCtx& x, int r0, int c, const float (&vf)[8],
                                               const double* v) {
  for (int d = 0; d < o.ndst; ++d) {
    const EpiDst& ds = o.dst[d];
    int64_t ld;
    if (ds.dt == DT_F64) {
      double* q = dst_base<double>(ds, x, &ld) + (int64_t)c * ld + r0;
      double t[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) t[w] = v ? v[w] : (double)vf[w];
      if (ds.mode == EPI_WS) {
#pragma unroll
        for (int w = 0; w < 8; w += 2) *reinterpret_cast<double2*>(q + w) = make_double2(t[w], t[w + 1]);
      } else {
#pragma unroll
        for (int w = 0; w < 8; ++w) q[w] = t[w];
      }
    } else {
      float* q = dst_base<float>(ds, x, &ld) + (int64_t)c * ld + r0;
      if (ds.mode == EPI_WS) {
        *reinterpret_cast<float4*>(q) = make_float4(vf[0], vf[1], vf[2], vf[3]);
        *reinterpret_cast<float4*>(q + 4) = make_float4(vf[4], vf[5], vf[6], vf[7]);
      } else {
#pragma unroll
        for (int w = 0; w < 8; ++w) q[w] = vf[w];
      }
    }
  }
}

// The mirrored run of a row-major split (symmetric plans store no transposed
// splits): hi/lo of (c, r0 .. r0+7), one 16-byte store each.
template <bool kF16>
__device__ __forceinline__ void st8_split_mirror(const EpiSplit& sp, const EpiCtx& x, int r0, int c,
                                                 const float (&v)[8], float sc) {
  uint32_t ph[4], pl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) split2<kF16>(v[2 * q], v[2 * q + 1], sc, &ph[q], &pl[q]);
  const int64_t off = x.off + (int64_t)c * sp.ld + r0;
  *reinterpret_cast<uint4*>(reinterpret_cast<unsigned short*>(sp.hi) + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
  *reinterpret_cast<uint4*>(reinterpret_cast<unsigned short*>(sp.lo) + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
}

// A chunk on the diagonal of a symmetric product: the element (r, c) of the
// run r = r0 .. r0+7 is written at its place when r <= c and at (c, r) too
// when r < c, so that the result is exactly symmetric.
__device__ __forceinline__ void st8_dst_diag(const EpiOut& o, const EpiCtx& x, int r0, int c, const float (&vf)[8],
                                             const double* v) {
  for (int d = 0; d < o.ndst; ++d) {
    const EpiDst& ds = o.dst[d];
    int64_t ld;
    if (ds.dt == DT_F64) {
      double* q = dst_base<double>(ds, x, &ld);
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const double t = v ? v[w] : (double)vf[w];
        if (r0 + w <= c) q[(int64_t)(r0 + w) * ld + c] = t;
        if (r0 + w < c) q[(int64_t)c * ld + r0 + w] = t;
      }
    } else {
      float* q = dst_base<float>(ds, x, &ld);
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        if (r0 + w <= c) q[(int64_t)(r0 + w) * ld + c] = vf[w];
        if (r0 + w < c) q[(int64_t)c * ld + r0 + w] = vf[w];
      }
    }
  }
}

template <bool kF16>
__device__ __forceinline__ void st8_split_diag(const EpiSplit& sp, const EpiCtx& x, int r0, int c, const float (&v)[8],
                                               float sc) {
  uint32_t ph[4], pl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) split2<kF16>(v[2 * q], v[2 * q + 1], sc, &ph[q], &pl[q]);
  unsigned short* hi = reinterpret_cast<unsigned short*>(sp.hi) + x.off;
  unsigned short* lo = reinterpret_cast<unsigned short*>(sp.lo) + x.off;
  const int64_t ld = sp.ld;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const unsigned short h = (unsigned short)(w & 1 ? ph[w / 2] >> 16 : ph[w / 2] & 0xffffu);
    const unsigned short l = (unsigned short)(w & 1 ? pl[w / 2] >> 16 : pl[w / 2] & 0xffffu);
    if (r0 + w <= c) {
      hi[(int64_t)(r0 + w) * ld + c] = h;
      lo[(int64_t)(r0 + w) * ld + c] = l;
    }
    if (r0 + w < c) {
      hi[(int64_t)c * ld + r0 + w] = h;
      lo[(int64_t)c * ld + r0 + w] = l;
    }
  }
}

// Split-FP16 (kF16): t holds the tile's scales.
template <bool kF16, int RB, int NF, bool kD>
__device__ __forceinline__ bool epi_chunk_lean(const EpiParams& P, const EpiCtx& x, int rbase, int c, const float* stg,
                                               int lane, int sym, bool edge, const SxTile* t) {
  static_assert(RB % 8 == 0 && 32 % RB == 0, "row batch");
  const int fi = P.f64_in;  // the FP64 input, or -1
  const int nf = P.nf32;    // FP32 inputs (<= NF)
  float chk = 0.f;          // becomes NaN once any output is non-finite
  float ovf = 0.f;          // largest |value| * scale split to FP16
#pragma unroll 1
  for (int g0 = 0; g0 < 32; g0 += RB) {
    float fin[NF > 0 ? NF : 1][RB];
    double din[kD ? RB : 1];
#pragma unroll
    for (int t = 0; t < NF; ++t) {
      if (t < nf) {
        int64_t ld;
        const float* q = in_base<float>(P.in[P.f32_idx[t]], x, &ld) + (int64_t)(rbase + g0) * ld + c;
#pragma unroll
        for (int w = 0; w < RB; ++w) fin[t][w] = q[(int64_t)w * ld];
      }
    }
    if (kD && fi >= 0) {
      int64_t ld;
      const double* q = in_base<double>(P.in[fi], x, &ld) + (int64_t)(rbase + g0) * ld + c;
#pragma unroll
      for (int w = 0; w < RB; ++w) din[w] = q[(int64_t)w * ld];
    }
#pragma unroll
    for (int h = 0; h < RB; h += 8) {
      const int r0 = rbase + g0 + h;
      const bool diag = (unsigned)(c - r0) < 8u;  // this lane's column holds the diagonal in these rows
      // boundary chunk (edge, warp-uniform): bit w set where (r0 + w, c) lies in the n x n block
      unsigned live = 0xffu;
      if (edge) {
        const int nr = x.n - r0;
        live = c >= x.n || nr <= 0 ? 0u : nr >= 8 ? 0xffu : (1u << nr) - 1u;
      }
      float a8[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) a8[w] = stg[(g0 + h + w) * 33 + lane];
#pragma unroll 1
      for (int j = 0; j < P.nout; ++j) {
        const EpiOut& o = P.out[j];
        // the same terms in the same order as epi_col
        const float af = kF16 ? o.acc_f * t->acc : o.acc_f;
        const float sc = kF16 ? t->sc[j] : 1.f;
        float vf[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) vf[w] = af * a8[w];
        if (o.f64) {
          // FP32 terms summed in FP32; the identity and the FP64 input (a partial
          // sum Y or residual R) are added in FP64
#pragma unroll
          for (int t = 0; t < NF; ++t) {
            const float cf = t < nf ? o.in_f[P.f32_idx[t]] : 0.f;
            if (cf != 0.f) {
#pragma unroll
              for (int w = 0; w < 8; ++w) vf[w] = fmaf(cf, fin[t][h + w], vf[w]);
            }
          }
          double v[8];
#pragma unroll
          for (int w = 0; w < 8; ++w) v[w] = (double)vf[w];
          if (diag) {
#pragma unroll
            for (int w = 0; w < 8; ++w)
              if (r0 + w == c) v[w] += o.id_d;
          }
          if (kD && fi >= 0 && o.in_d[fi] != 0.0) {
#pragma unroll
            for (int w = 0; w < 8; ++w) v[w] = fma(o.in_d[fi], din[h + w], v[w]);
          }
          if (edge) {  // padding holds zeros
#pragma unroll
            for (int w = 0; w < 8; ++w)
              if (!((live >> w) & 1u)) v[w] = 0.0;
          }
#pragma unroll
          for (int w = 0; w < 8; ++w) vf[w] = (float)v[w];
          if (sym == 2) {
            st8_dst_diag(o, x, r0, c, vf, v);
          } else {
            for (int d = 0; d < o.ndst; ++d) {
              const EpiDst& ds = o.dst[d];
              int64_t ld;
              const unsigned keep = (edge && ds.mode != EPI_WS) ? live : 0xffu;  // caller's matrix: n x n only
              if (ds.dt == DT_F64) {
                double* q = dst_base<double>(ds, x, &ld) + (int64_t)r0 * ld + c;
                if (keep == 0xffu) {
#pragma unroll
                  for (int w = 0; w < 8; ++w) q[(int64_t)w * ld] = v[w];
                } else {
#pragma unroll
                  for (int w = 0; w < 8; ++w)
                    if ((keep >> w) & 1u) q[(int64_t)w * ld] = v[w];
                }
              } else {
                float* q = dst_base<float>(ds, x, &ld) + (int64_t)r0 * ld + c;
                if (keep == 0xffu) {
#pragma unroll
                  for (int w = 0; w < 8; ++w) q[(int64_t)w * ld] = vf[w];
                } else {
#pragma unroll
                  for (int w = 0; w < 8; ++w)
                    if ((keep >> w) & 1u) q[(int64_t)w * ld] = vf[w];
                }
              }
            }
            if (sym == 1) st8_mirror_dst(o, x, r0, c, vf, v);
          }
        } else {
          if (diag) {
#pragma unroll
            for (int w = 0; w < 8; ++w)
              if (r0 + w == c) vf[w] += o.id_f;
          }
          // FP32 inputs in index order, then an FP64 input rounded to FP32 (no
          // op of the schedules pairs an FP64 input with an FP32-only output)
#pragma unroll
          for (int t = 0; t < NF; ++t) {
            const float cf = t < nf ? o.in_f[P.f32_idx[t]] : 0.f;
            if (cf != 0.f) {
#pragma unroll
              for (int w = 0; w < 8; ++w) vf[w] = fmaf(cf, fin[t][h + w], vf[w]);
            }
          }
          if (kD && fi >= 0 && o.in_f[fi] != 0.f) {
#pragma unroll
            for (int w = 0; w < 8; ++w) vf[w] = fmaf(o.in_f[fi], (float)din[h + w], vf[w]);
          }
          if (edge) {  // padding holds zeros
#pragma unroll
            for (int w = 0; w < 8; ++w)
              if (!((live >> w) & 1u)) vf[w] = 0.f;
          }
          if (sym == 2) {
            st8_dst_diag(o, x, r0, c, vf, nullptr);
          } else {
            for (int d = 0; d < o.ndst; ++d) {
              const EpiDst& ds = o.dst[d];
              int64_t ld;
              const unsigned keep = (edge && ds.mode != EPI_WS) ? live : 0xffu;  // caller's matrix: n x n only
              if (ds.dt == DT_F64) {
                double* q = dst_base<double>(ds, x, &ld) + (int64_t)r0 * ld + c;
                if (keep == 0xffu) {
#pragma unroll
                  for (int w = 0; w < 8; ++w) q[(int64_t)w * ld] = (double)vf[w];
                } else {
#pragma unroll
                  for (int w = 0; w < 8; ++w)
                    if ((keep >> w) & 1u) q[(int64_t)w * ld] = (double)vf[w];
                }
              } else {
                float* q = dst_base<float>(ds, x, &ld) + (int64_t)r0 * ld + c;
                if (keep == 0xffu) {
#pragma unroll
                  for (int w = 0; w < 8; ++w) q[(int64_t)w * ld] = vf[w];
                } else {
#pragma unroll
                  for (int w = 0; w < 8; ++w)
                    if ((keep >> w) & 1u) q[(int64_t)w * ld] = vf[w];
                }
              }
            }
            if (sym == 1) st8_mirror_dst(o, x, r0, c, vf, nullptr);
          }
        }
#pragma unroll
        for (int w = 0; w < 8; ++w) chk = fmaf(vf[w], 0.f, chk);
        if (kF16 && o.nsplit) {
          float mx = 0.f;
#pragma unroll
          for (int w = 0; w < 8; ++w) mx = fmaxf(mx, fabsf(vf[w]));
          ovf = fmaxf(ovf, mx * sc);
        }
        for (int s2 = 0; s2 < o.nsplit; ++s2) {
          if (sym == 2) {
            st8_split_diag<kF16>(o.split[s2], x, r0, c, vf, sc);
          } else {
            st8_split<kF16>(o.split[s2], x, r0, c, vf, sc);
            if (sym == 1) st8_split_mirror<kF16>(o.split[s2], x, r0, c, vf, sc);
          }
        }
      }
    }
  }
  return chk != chk || !(ovf < 65504.f);
}

template <bool kF16>
__device__ __forceinline__ bool epi_chunk_fast(const EpiParams& P, const EpiCtx& x, int rbase, int c, const float* stg,
                                               int lane, int sym, bool edge, const SxTile* t) {
  if (P.f64_in < 0 && P.nf32 <= 1) return epi_chunk_lean<kF16, 32, 1, false>(P, x, rbase, c, stg, lane, sym, edge, t);
  if (P.f64_in < 0 && P.nf32 == 2) return epi_chunk_lean<kF16, 16, 2, false>(P, x, rbase, c, stg, lane, sym, edge, t);
  if (P.f64_in < 0) return epi_chunk_lean<kF16, 8, kMaxIn, false>(P, x, rbase, c, stg, lane, sym, edge, t);
  return epi_chunk_lean<kF16, 8, kMaxIn, true>(P, x, rbase, c, stg, lane, sym, edge, t);
}

// Boundary chunks (padding, ragged edges, grouped row limits) and ops with
// several FP64 inputs, row group by row group. Out of line: it is rare, and
// its registers then do not count against the lean path's.
template <bool kF16>
__device__ __noinline__ bool epi_chunk_generic(const EpiParams& P, EpiCtx x, int rbase, int c, const float* stg,
                                               int lane, int lim, bool mirror, const SxTile* t) {
  bool bad = false;
#pragma unroll 1
  for (int g = 0; g < 4; ++g) {
    const int r0 = rbase + 8 * g;
    if (r0 >= lim) break;
    float a8[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) a8[w] = stg[(8 * g + w) * 33 + lane];
    bad |= epi_col<8, float, kF16>(P, x, r0, c, a8, t);
    if (mirror) {  // the transposed element of a symmetric result, one at a time
#pragma unroll 1
      for (int w = 0; w < 8; ++w) bad |= epi_element<float, kF16>(P, x, c, r0 + w, a8[w], t);
    }
  }
  return bad;
}

// The epilogue of one staged 32 x 32 chunk (rows rbase .. rbase+31, this lane's
// column c). Rows at or beyond `lim` (a grouped tile's limit) are not written.
// A chunk on the diagonal of a symmetric product: each element on or above
// the diagonal is written at its place, and those above it at the transpose
// too, so that the result is exactly symmetric.
template <bool kF16>
__device__ __noinline__ bool epi_chunk_diag(const EpiParams& P, EpiCtx x, int rbase, int c, const float* stg,
                                            int lane, const SxTile* t) {
  bool bad = false;
#pragma unroll 1
  for (int i = 0; i < 32; ++i) {
    const int r = rbase + i;
    const float a = stg[i * 33 + lane];
    if (r <= c) bad |= epi_element<float, kF16>(P, x, r, c, a, t);
    if (r < c) bad |= epi_element<float, kF16>(P, x, c, r, a, t);
  }
  return bad;
}

// Symmetric products: sym = 0 for a chunk of a general product, 1 for a chunk
// above the diagonal (also writes its transpose), 2 for a chunk on it.
// Split-FP16 (kF16): t as in epi_chunk_lean (nullptr otherwise).
template <bool kF16>
__device__ __forceinline__ bool epi_chunk(const EpiParams& P, const EpiCtx& x, int rbase, int c, const float* stg,
                                          int lane, int lim, int sym, const SxTile* t) {
  if (P.fast && rbase + 32 <= lim) {
    // boundary chunk: part of it lies outside the n x n block (warp-uniform)
    const bool edge = !__all_sync(0xffffffffu, c < x.n && rbase + 32 <= x.n);
    if (!edge || (sym == 0 && P.edge_ok)) return epi_chunk_fast<kF16>(P, x, rbase, c, stg, lane, sym, edge, t);
  }
  if (sym == 2) return epi_chunk_diag<kF16>(P, x, rbase, c, stg, lane, t);
  return epi_chunk_generic<kF16>(P, x, rbase, c, stg, lane, lim, sym == 1, t);
}

// Split-FP16 statistics of a product's accumulator (its true value is the
// staged value times t.acc), measured once per staged 32 x 32 chunk whatever
// the number of outputs: this lane's column sum of |acc| over the chunk's rows
// below `lim` (lane = column c; a grouped tile's rows past its matrix's padded
// order hold values no consumer reads), added to the product's column sums;
// and, for a symmetric product, the sums of the mirrored elements, added to
// the columns they land in (lane = row rbase + lane of the chunk: its elements
// right of the diagonal). The row maxima are taken where the chunk is staged
// (sx_row_max).
__device__ __forceinline__ void sx_chunk_colsum(const EpiParams& P, int mat, const float* stg, int lane, int rbase,
                                                int cbase, int sym, int lim, float tacc) {
  float* col = P.sx.acc_col + (int64_t)mat * P.sx.npad;
  const int c = cbase + lane;
  float cs = 0.f;
#pragma unroll 8
  for (int i = 0; i < 32; ++i)
    cs += (rbase + i < lim && (sym != 2 || rbase + i <= c)) ? fabsf(stg[i * 33 + lane]) : 0.f;
  if (cs > 0.f) atomicAdd(col + c, cs * tacc);
  if (sym) {
    const int r = rbase + lane;
    float rs = 0.f;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) rs += (sym == 1 || cbase + l > r) ? fabsf(stg[lane * 33 + l]) : 0.f;
    if (rs > 0.f) atomicAdd(col + r, rs * tacc);
  }
}

// max |x| of the 32 staged values of this lane's row
__device__ __forceinline__ float sx_row_max(const uint32_t (&v)[32]) {
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < 32; ++j) m = fmaxf(m, fabsf(__uint_as_float(v[j])));
  return m;
}

// End of a tile: the warp's max |acc| into the product's record for matrix mat.
__device__ __forceinline__ void sx_tile_max(const EpiParams& P, int mat, float am, float tacc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
  if ((threadIdx.x & 31) == 0 && am > 0.f) atomicMax(P.sx.acc_amax + mat, __float_as_uint(am * tacc));
}

__device__ __forceinline__ void epi_flag(const EpiParams& P, bool bad) {
  if (bad && P.status) atomicOr(P.status, 1u);
}

}  // namespace neumann
