// The resident batch kernel: small matrices of a batch, each held whole in one
// CTA's shared memory across every level of the scheme.
//
// A grouped batch runs each op of the scheme as one launch over all its
// matrices, so every intermediate matrix goes through HBM/L2 between launches,
// and a matrix of order 16 or 64 pays the same per-launch latency as one of
// order 256. Here one persistent launch takes the batch's small matrices
// (largest first; CTA b takes matrices b, b + grid, ...). For each it runs the
// plan's op program (the level loop of Sec. 5.3, eq. generalradix: kernel
// products, concatenation, residual) with every matrix of the scheme in the
// CTA's shared memory: FP32 copies of all, FP64 copies of the partial sum and
// residual, and the program itself. Only A is read from and S written to the
// caller's memory. The host launches one grid per size class (orders up to 16,
// 32, and the largest held), each with as many threads as 4 x 1 (up to order
// 16) or 4 x 2 output blocks and as many CTAs per SM as its shared memory
// allows.
//
// Products: at n <= 64 a product is at most 0.5 MFLOP and the work is a chain
// of dependent steps, so a product is a register-blocked SIMT loop (each
// thread a 4 x 1 or 4 x 2 block of the output) rather than a tensor-core
// launch. For a split plan the operands are split once per product, as the
// tensor-core path stores them (hi = RN16(x), lo = RN16(x - hi); FP16 of
// x * 2^e with e from the operand's exact max |x|, the bound mapped to 2^14),
// into packed words in shared memory, and hi*hi + hi*lo + lo*hi is
// accumulated in FP32. The epilogue is the same linear combination as epilogue.cuh's: FP32
// terms in FP32, then the identity and FP64 inputs in FP64, outputs' split
// sources RN_fp32 of the value.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace neumann {

namespace {

constexpr int kResMaxThreads = 512;  // 16 x 32 blocks of 4 x 2 outputs cover order 64

// hi + lo of x in the mode's 16-bit type (mode 2: of x * sc)
template <int MODE>
__device__ __forceinline__ void res_split(float x, float sc, float* hi, float* lo) {
  if (MODE == 1) {
    const float h = __bfloat162float(__float2bfloat16_rn(x));
    *hi = h;
    *lo = __bfloat162float(__float2bfloat16_rn(x - h));
  } else {
    const float w = x * sc;
    const float h = __half2float(__float2half_rn(w));
    *hi = h;
    *lo = __half2float(__float2half_rn(w - h));
  }
}

// The pair as one word: hi in the upper 16 bits, lo in the lower (the 16-bit
// type's bits). Unpacking a BF16 pair is two bit operations, where splitting
// takes conversions on the XU pipe (16 lanes per clock per SM).
template <int MODE>
__device__ __forceinline__ uint32_t res_pack(float x, float sc) {
  float h, l;
  res_split<MODE>(x, sc, &h, &l);
  if (MODE == 1)
    return ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(h)) << 16) |
           (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(l));
  return ((uint32_t)__half_as_ushort(__float2half_rn(h)) << 16) | (uint32_t)__half_as_ushort(__float2half_rn(l));
}
template <int MODE>
__device__ __forceinline__ void res_unpack(uint32_t w, float* hi, float* lo) {
  if (MODE == 1) {
    *hi = __uint_as_float(w & 0xffff0000u);
    *lo = __uint_as_float(w << 16);
  } else {
    *hi = __half2float(__ushort_as_half((unsigned short)(w >> 16)));
    *lo = __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
  }
}

// max |x| over the n x n block of X (leading dimension ld); every thread calls it
__device__ float res_block_amax(const float* X, int n, int ld, float* red) {
  float v = 0.f;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) v = fmaxf(v, fabsf(X[(e / n) * ld + e % n]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
  return r;
}

// e with amax * 2^e <= 2^kSxTarget (0 for zero or non-finite)
__device__ __forceinline__ int res_exp(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 0;
  int k = 0;
  frexpf(amax, &k);
  const int e = kSxTarget - k;
  return e < -kSxMaxExp ? -kSxMaxExp : e > kSxMaxExp ? kSxMaxExp : e;
}

// CW consecutive elements of a row: vector loads and stores of 4, 2 or 1 values
template <int CW>
__device__ __forceinline__ void ld_row(const float* p, float (&v)[CW]) {
  if constexpr (CW == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  } else if constexpr (CW == 2) {
    const float2 x = *reinterpret_cast<const float2*>(p);
    v[0] = x.x;
    v[1] = x.y;
  } else {
    v[0] = *p;
  }
}
template <int CW>
__device__ __forceinline__ void ld_row(const double* p, double (&v)[CW]) {
#pragma unroll
  for (int j = 0; j < CW; j += 2) {
    if (j + 1 < CW) {
      const double2 x = *reinterpret_cast<const double2*>(p + j);
      v[j] = x.x;
      v[j + 1] = x.y;
    } else {
      v[j] = p[j];
    }
  }
}
template <int CW>
__device__ __forceinline__ void st_row(float* p, const float (&v)[CW]) {
  if constexpr (CW == 4)
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else if constexpr (CW == 2)
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  else
    *p = v[0];
}
template <int CW>
__device__ __forceinline__ void st_row(double* p, const double (&v)[CW]) {
#pragma unroll
  for (int j = 0; j < CW; j += 2) {
    if (j + 1 < CW)
      *reinterpret_cast<double2*>(p + j) = make_double2(v[j], v[j + 1]);
    else
      p[j] = v[j];
  }
}

// Each thread holds a 4 x CW block of every output: CW = 1 up to order 16, else
// 2, so that a CTA runs 64-512 threads (with 4 x 4 blocks an order-32 matrix
// had 64 threads, and the SM, at 3 CTAs for its shared memory, 6 warps; an
// order-48 matrix 144 threads at 1 CTA: too few to cover the latency of one
// matrix's chain of dependent steps).
template <int MODE, int CW>
__global__ void __launch_bounds__(kResMaxThreads) resident_kernel(const __grid_constant__ ResParams P) {
  // shared memory: FP64 copies | FP32 copies | packed operands (split modes) |
  // program (16-byte aligned sections)
  extern __shared__ __align__(16) double smd[];
  __shared__ float red[kResMaxThreads / 32];
  const int t = threadIdx.x;
  const size_t slot = (size_t)P.nmax * P.nmax;
  double* f64 = smd;
  float* sm = reinterpret_cast<float*>(smd + (size_t)P.nf64 * slot);
  // split modes: the current product's operands as packed hi/lo words (2 slots)
  uint32_t* pk = reinterpret_cast<uint32_t*>(sm + (size_t)P.nslots * slot);
  ResOp* prog = reinterpret_cast<ResOp*>(pk + (MODE != 0 ? 2 * slot : 0));
  for (int w = t; w < (int)(P.nops * sizeof(ResOp) / sizeof(int)); w += blockDim.x)
    reinterpret_cast<int*>(prog)[w] = reinterpret_cast<const int*>(P.ops)[w];
  __syncthreads();
  bool bad = false;
  for (int m = blockIdx.x; m < P.count; m += gridDim.x) {
    const int n = P.mat_n[m];
    const int ld = (n + 3) & ~3;  // rows of each matrix in its slot; padding zero
    const int nbr = ld / 4, nbc = ld / CW;  // row and column blocks
    const bool act = t < nbr * nbc;
    const int r0 = act ? (t / nbc) * 4 : 0, c0 = act ? (t % nbc) * CW : 0;
#pragma unroll 1
    for (int k = 0; k < P.nops; ++k) {
      const ResOp& op = prog[k];
      float acc[4][CW];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[i][j] = 0.f;
      if (op.gemm) {
        const float* L = sm + op.a * slot;
        const float* R = sm + op.b * slot;
        int ea = 0, eb = 0;
        if (MODE == 2) {  // each operand's own power of two
          ea = res_exp(res_block_amax(L, n, ld, red));
          eb = res_exp(res_block_amax(R, n, ld, red));
        }
        const float sa = ldexpf(1.f, ea), sb = ldexpf(1.f, eb);
        if (MODE != 0) {
          // split each operand element once, into the two packed slots, not
          // once for every thread that reads it: done in the product loop, the
          // conversions (one per three FMAs) bound the largest size class
          for (int e = t; e < ld * ld; e += blockDim.x) {
            pk[e] = res_pack<MODE>(L[e], sa);
            pk[slot + e] = res_pack<MODE>(R[e], sb);
          }
          __syncthreads();
        }
        if (act) {
          // k in steps of 4: the left operand as one 16-byte run of each of the
          // block's 4 rows (at ld = 32 a warp's row groups share one set of
          // banks, so scalar loads of a column conflict); the padding columns
          // n .. ld-1 hold zeros and add nothing
#pragma unroll 1
          for (int q4 = 0; q4 < ld; q4 += 4) {
            if (MODE == 0) {
              float4 av[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4*>(L + (r0 + i) * ld + q4);
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                float b[CW];
                ld_row<CW>(R + (q4 + qq) * ld + c0, b);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const float a = qq == 0 ? av[i].x : qq == 1 ? av[i].y : qq == 2 ? av[i].z : av[i].w;
#pragma unroll
                  for (int j = 0; j < CW; ++j) acc[i][j] = fmaf(a, b[j], acc[i][j]);
                }
              }
            } else {
              uint4 aw[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) aw[i] = *reinterpret_cast<const uint4*>(pk + (r0 + i) * ld + q4);
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                float ah[4], al[4], bh[CW], bl[CW];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  res_unpack<MODE>(qq == 0 ? aw[i].x : qq == 1 ? aw[i].y : qq == 2 ? aw[i].z : aw[i].w, &ah[i], &al[i]);
#pragma unroll
                for (int j = 0; j < CW; ++j) res_unpack<MODE>(pk[slot + (q4 + qq) * ld + c0 + j], &bh[j], &bl[j]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                  for (int j = 0; j < CW; ++j)
                    acc[i][j] = fmaf(al[i], bh[j], fmaf(ah[i], bl[j], fmaf(ah[i], bh[j], acc[i][j])));
              }
            }
          }
          if (MODE == 2) {
            const float inv = ldexpf(1.f, -(ea + eb));
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < CW; ++j) acc[i][j] *= inv;
          }
        }
      }
      __syncthreads();  // every operand read before any output is written
      if (act) {
        bool is64[kMaxIn];
#pragma unroll
        for (int ii = 0; ii < kMaxIn; ++ii)
          is64[ii] = ii < op.nin && (op.in_slot[ii] < 0 ? P.io_f64 != 0 : op.in_f64[ii] != 0);
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {  // one row of the thread's block: CW consecutive columns
          const int r = r0 + i;
          const int64_t e0 = (int64_t)r * ld + c0;
          bool live[CW];
#pragma unroll
          for (int j = 0; j < CW; ++j) live[j] = r < n && c0 + j < n;
          // every input load of the row before any output is formed: FP32
          // inputs stay in FP32 registers, FP64 inputs in FP64 ones (GB300
          // converts between the two on its FP64 pipe, at 1/64 of the FP32
          // rate; with the operand splits out of the product loop those
          // conversions were the binding unit)
          float vf32[kMaxIn][CW];
          double vf64[kMaxIn][CW];
#pragma unroll
          for (int ii = 0; ii < kMaxIn; ++ii) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              vf32[ii][j] = 0.f;
              vf64[ii][j] = 0.0;
            }
            if (ii < op.nin) {
              const int sl = op.in_slot[ii];
              if (sl < 0) {  // the caller's A, leading dimension n
#pragma unroll
                for (int j = 0; j < CW; ++j)
                  if (live[j]) {
                    if (P.io_f64)
                      vf64[ii][j] = reinterpret_cast<const double*>(P.A[m])[(int64_t)r * n + c0 + j];
                    else
                      vf32[ii][j] = reinterpret_cast<const float*>(P.A[m])[(int64_t)r * n + c0 + j];
                  }
              } else if (op.in_f64[ii]) {
                ld_row<CW>(f64 + P.f64_of[sl] * slot + e0, vf64[ii]);
              } else {
                ld_row<CW>(sm + sl * slot + e0, vf32[ii]);
              }
            }
          }
#pragma unroll 1
          for (int o = 0; o < op.nout; ++o) {
            const bool f64o = op.f64[o] != 0;
            const float af = op.acc_f[o], idf = op.id_f[o];
            const double idd = op.id_d[o];
            float vf[CW];
            double v[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const bool diag = r == c0 + j;
              if (f64o) {
                // FP32 terms in FP32, then the identity and the FP64 inputs in FP64
                float tt = af * acc[i][j];
#pragma unroll
                for (int ii = 0; ii < kMaxIn; ++ii)
                  if (ii < op.nin && !is64[ii] && op.in_f[o][ii] != 0.f) tt = fmaf(op.in_f[o][ii], vf32[ii][j], tt);
                // (FP64 runs at 1/64 of FP32: the identity is added on the
                // diagonal only, and finiteness is read from the FP32 copy)
                double d = (double)tt;
                if (diag) d += idd;
#pragma unroll
                for (int ii = 0; ii < kMaxIn; ++ii)
                  if (ii < op.nin && is64[ii] && op.in_d[o][ii] != 0.0) d = fma(op.in_d[o][ii], vf64[ii][j], d);
                v[j] = live[j] ? d : 0.0;
                vf[j] = (float)v[j];
                bad |= !isfinite(vf[j]);
              } else {
                float t2 = af * acc[i][j] + (diag ? idf : 0.f);
#pragma unroll
                for (int ii = 0; ii < kMaxIn; ++ii)
                  if (ii < op.nin && op.in_f[o][ii] != 0.f)
                    t2 = fmaf(op.in_f[o][ii], is64[ii] ? (float)vf64[ii][j] : vf32[ii][j], t2);
                vf[j] = live[j] ? t2 : 0.f;
                bad |= !isfinite(t2);
              }
            }
            const int sl = op.out_slot[o];
            if (!f64o && ((sl < 0 && P.io_f64) || (sl >= 0 && op.out_f64[o]))) {  // an FP64 copy of an FP32 value
#pragma unroll
              for (int j = 0; j < CW; ++j) v[j] = (double)vf[j];
            }
            if (sl < 0) {  // the caller's S, leading dimension n: the n x n block only
#pragma unroll
              for (int j = 0; j < CW; ++j) {
                if (!live[j]) continue;
                if (P.io_f64)
                  reinterpret_cast<double*>(P.S[m])[(int64_t)r * n + c0 + j] = v[j];
                else
                  reinterpret_cast<float*>(P.S[m])[(int64_t)r * n + c0 + j] = vf[j];
              }
            } else {  // padding stored as zeros
              if (op.out_f32[o]) st_row<CW>(sm + sl * slot + e0, vf);
              if (op.out_f64[o]) st_row<CW>(f64 + P.f64_of[sl] * slot + e0, v);
            }
          }
        }
      }
      __syncthreads();  // the op's outputs complete before the next op reads them
    }
  }
  if (bad && P.status) atomicOr(P.status, 1u);  // NEUMANN_STATUS_NONFINITE
}

}  // namespace

cudaError_t launch_resident(const ResParams& P, cudaStream_t s) {
  if (P.count <= 0) return cudaSuccess;
  const size_t smem = resident_smem(P.nslots, P.nf64, P.nops, P.nmax, P.mode != 0);
  const int threads = resident_threads(P.nmax);
  if (smem > (size_t)kResSmemBudget || threads > kResMaxThreads || P.mode < 0 || P.mode > 2)
    return cudaErrorInvalidValue;
  using K = void (*)(ResParams);
  static const K kernels[3][2] = {{resident_kernel<0, 1>, resident_kernel<0, 2>},
                                  {resident_kernel<1, 1>, resident_kernel<1, 2>},
                                  {resident_kernel<2, 1>, resident_kernel<2, 2>}};
  const int ci = resident_cw(P.nmax) == 1 ? 0 : 1;
  const K k = kernels[P.mode][ci];
  static std::atomic<int> attr[3][2][kMaxDevices];
  cudaError_t e = once_per_device(attr[P.mode][ci], [&] {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmemBudget);
  });
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long cap = (long)per_sm * sm_count();
  const int grid = (int)(P.count < cap ? P.count : cap);
  k<<<grid, threads, smem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace neumann
