// CUDA-core GEMMs for the plain FP64 and FP32 paths, with the fused epilogue.
//
// Blackwell tensor cores take no FP32 operands, and GB300's FP64 rate is the
// same on the tensor and CUDA cores, so these products run as register-tiled
// SIMT GEMMs: a 128 x 128 tile per 256-thread CTA, 8 x 8 outputs per thread,
// K staged through double-buffered shared memory 8 at a time. All workspace
// matrices are padded to a multiple of 256 in both dimensions and every
// epilogue rewrites the padding with zeros, so the main loop has no bounds
// checks.
#include <mutex>
#include <type_traits>

#include "epilogue.cuh"

namespace neumann {

namespace {

constexpr int BM = 128, BN = 128, TPB = 256;
static_assert(simt_bk(true) == 8 && simt_bk(false) == 16, "SIMT stage depth differs from the tile tables");

__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  double2 t0 = reinterpret_cast<const double2*>(p)[0];
  double2 t1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}
// Four consecutive shared-memory elements: one 16-byte store for FP32 (a warp's
// 32 consecutive runs then fill 512 bytes without a bank conflict).
__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double (&v)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) p[j] = v[j];
}

constexpr int kFlushK = 128;  // FP32: k per partial sum of the two-level accumulation

// tiles == nullptr: one matrix, CTA (blockIdx.y, blockIdx.x) computes tile
// (tm, tn) over `ktiles` K steps. Otherwise (grouped launch over a batch) CTA b
// computes tiles[b] = {matrix, tm, tn, K steps}; every operand and workspace
// buffer then holds matrix m at element offset m * P.mat_stride.
// FP32 keeps its running sums in shared memory (see below), so two CTAs fit
// per SM; FP64 is bound by the FP64 pipe and keeps them in registers.
template <typename T>
__global__ void __launch_bounds__(TPB, sizeof(T) == 4 ? 2 : 1)
    simt_gemm_kernel(const T* __restrict__ A, const T* __restrict__ B, int64_t ld, int ktiles,
                     const int4* __restrict__ tiles, int sym, const __grid_constant__ EpiParams P) {
  // K depth of a shared-memory stage: 16 for FP32 (fewer barriers per FMA), 8
  // for FP64 (static shared memory is limited to 48 KB)
  constexpr int BK = sizeof(T) == 8 ? 8 : 16;
  constexpr int V = BK / 8;  // 4-element runs a thread loads per operand and stage
  __shared__ __align__(16) T As[2][BK][BM + 4];
  __shared__ __align__(16) T Bs[2][BK][BN];
  extern __shared__ float acc_smem[];  // FP32: running sums, [64][TPB] (element e of thread t at e * TPB + t)
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // FP32: two-level accumulation (below); kFlush K steps per partial sum
  constexpr bool kTwoLevel = sizeof(T) == 4;
  constexpr int kFlush = kFlushK / BK;
  int mat = 0, tm = blockIdx.y, tn = blockIdx.x;
  if (sym) {
    // a symmetric product (every matrix of the scheme is a polynomial in the
    // symmetric A): block b takes the b-th tile on or above the diagonal, row
    // by row; `sym` is the number of tile rows
    int t = blockIdx.x;
    tm = 0;
    while (t >= sym - tm) {
      t -= sym - tm;
      ++tm;
    }
    tn = tm + t;
  }
  if (tiles) {
    const int4 t = tiles[blockIdx.x];
    mat = t.x;
    tm = t.y;
    tn = t.z;
    ktiles = t.w;
    A += (int64_t)mat * P.mat_stride;
    B += (int64_t)mat * P.mat_stride;
  }
  const EpiCtx x = epi_ctx(P, mat);
  const int m0 = tm * BM, n0 = tn * BN;
  // A tile: 128 rows x BK as runs of 4 k; run v of a thread is row tid % 128,
  // k from 4 (tid / 128 + 2 v), stored transposed (As[k][row]): a warp's 32
  // consecutive rows land in 32 banks. B tile: BK rows x 128 as runs of 4
  // columns; run v of a thread is row tid / 32 + 8 v, columns 4 (tid % 32) ..:
  // a warp reads and stores 512 contiguous bytes of one row.
  const int a_row = tid & (BM - 1), a_col = 4 * (tid / BM);
  const int b_row = tid >> 5, b_col = (tid & 31) * 4;
  const T* Ap = A + (int64_t)(m0 + a_row) * ld + a_col;
  const T* Bp = B + (int64_t)b_row * ld + n0 + b_col;

  // next stage's operands: one 4-element run of A and of B at a time (V runs a
  // stage), stored into the free buffer before the next run is fetched, which
  // keeps 8 registers in flight whatever BK is
  T ra[4], rb[4];
  auto fetch = [&](int kt, int v) {
    load4(Ap + (int64_t)kt * BK + 8 * v, ra);
    load4(Bp + ((int64_t)kt * BK + 8 * v) * ld, rb);
  };
  auto stash = [&](int buf, int v) {
#pragma unroll
    for (int j = 0; j < 4; ++j) As[buf][a_col + 8 * v + j][a_row] = ra[j];
    store4(&Bs[buf][b_row + 8 * v][b_col], rb);
  };
#pragma unroll
  for (int v = 0; v < V; ++v) {
    fetch(0, v);
    stash(0, v);
  }
  __syncthreads();

  // FP32: two-level accumulation. Products are summed into `prt` for 128
  // consecutive k and then added to the running sum, so each rounding error
  // grows with sqrt(128) + sqrt(K/128) instead of sqrt(K) (K = 4096: 17 vs 64
  // units; 64 k per partial sum gave 16 and took 3.6 % longer). The running
  // sums live in shared memory (touched once per 128 k), which keeps the
  // kernel within 128 registers.
  T acc[kTwoLevel ? 1 : 8][kTwoLevel ? 1 : 8], prt[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      prt[i][j] = T(0);
      if constexpr (kTwoLevel)
        acc_smem[(i * 8 + j) * TPB + tid] = 0.f;
      else
        acc[i][j] = T(0);
    }

  for (int kt = 0; kt < ktiles; ++kt) {
    const int cur = kt & 1;
    const bool more = kt + 1 < ktiles;
    // buffer cur ^ 1 was last read before the previous barrier: free to fill
    if (more) fetch(kt + 1, 0);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      if (V > 1 && kk > 0 && kk % 8 == 0 && more) {
        stash(cur ^ 1, kk / 8 - 1);
        fetch(kt + 1, kk / 8);
      }
      T a[8], b[8];
      T t[4];
      load4(&As[cur][kk][ty * 4], t);
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = t[q];
      load4(&As[cur][kk][64 + ty * 4], t);
#pragma unroll
      for (int q = 0; q < 4; ++q) a[4 + q] = t[q];
      load4(&Bs[cur][kk][tx * 4], t);
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = t[q];
      load4(&Bs[cur][kk][64 + tx * 4], t);
#pragma unroll
      for (int q = 0; q < 4; ++q) b[4 + q] = t[q];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if constexpr (kTwoLevel)
            prt[i][j] = fma(a[i], b[j], prt[i][j]);
          else
            acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
    if constexpr (kTwoLevel) {
      if ((kt + 1) % kFlush == 0 || !more) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            acc_smem[(i * 8 + j) * TPB + tid] += prt[i][j];
            prt[i][j] = T(0);
          }
      }
    }
    if (more) stash(cur ^ 1, V - 1);
    __syncthreads();
  }

  // A grouped launch writes each matrix below its order rounded up to 32: that
  // covers the K padding later products read; the rest feeds only discarded outputs.
  const int lim = tiles ? (x.n + 31) / 32 * 32 : (1 << 30);
  bool bad = false;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c0 = n0 + h * 64 + tx * 4;
      if (r >= lim || c0 >= lim) continue;
      T a4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if constexpr (kTwoLevel)
          a4[j] = acc_smem[(i * 8 + 4 * h + j) * TPB + tid];
        else
          a4[j] = acc[i][4 * h + j];
      }
      if (!sym) {
        bad |= epi_row<4, T, false>(P, x, r, c0, a4);
      } else if (tm != tn) {  // above the diagonal: this run, then its transpose
        bad |= epi_row<4, T, false>(P, x, r, c0, a4);
#pragma unroll 1
        for (int j = 0; j < 4; ++j) bad |= epi_element<T, false>(P, x, c0 + j, r, a4[j]);
      } else {  // on the diagonal tile: r <= c at its place, r < c at the transpose too
#pragma unroll 1
        for (int j = 0; j < 4; ++j) {
          if (r <= c0 + j) bad |= epi_element<T, false>(P, x, r, c0 + j, a4[j]);
          if (r < c0 + j) bad |= epi_element<T, false>(P, x, c0 + j, r, a4[j]);
        }
      }
    }
  }
  epi_flag(P, bad);
}

// Element-wise pass (acc = 0) over one 32 x 32 tile per 256-thread CTA.
// Row-major stores are coalesced along the warp; transposed hi/lo stores go
// through a shared-memory tile so that they are coalesced too.
// tiles != nullptr (grouped launch): CTA b handles tiles[b] = {matrix, tile row, tile column}.
template <bool kF16>
__global__ void __launch_bounds__(256) ewise_kernel(const int4* __restrict__ tiles,
                                                     const __grid_constant__ EpiParams P) {
  __shared__ float tile[kMaxOut][32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  int mat = 0, tr = blockIdx.y, tc = blockIdx.x;
  if (tiles) {
    const int4 t = tiles[blockIdx.x];
    mat = t.x;
    tr = t.y;
    tc = t.z;
  }
  const EpiCtx x = epi_ctx(P, mat);
  SxTile sxt;  // split-FP16 scales of this matrix
  if (kF16) sx_tile(P, mat, &sxt);
  const int r0 = tr * 32, c0 = tc * 32;
  bool bad = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float tv[kMaxOut];
    bad |= epi_element_impl<float, true, kF16>(P, x, r0 + ty + 8 * q, c0 + tx, 0.f, tv, kF16 ? &sxt : nullptr);
#pragma unroll
    for (int j = 0; j < kMaxOut; ++j) tile[j][ty + 8 * q][tx] = tv[j];
  }
  __syncthreads();
  for (int j = 0; j < P.nout; ++j) {
    const EpiOut& o = P.out[j];
    for (int s = 0; s < o.nsplit; ++s) {
      const EpiSplit& sp = o.split[s];
      if (!sp.transposed) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // lane tx writes element (r0 + tx, c0 + ty + 8q) at row c, column r of the stored transpose
        const float v = tile[j][tx][ty + 8 * q];
        unsigned short hi, lo;
        split_bits<kF16>(v, kF16 ? sxt.sc[j] : 1.f, &hi, &lo);
        const int64_t off = x.off + (int64_t)(c0 + ty + 8 * q) * sp.ld + (r0 + tx);
        reinterpret_cast<unsigned short*>(sp.hi)[off] = hi;
        reinterpret_cast<unsigned short*>(sp.lo)[off] = lo;
      }
    }
  }
  epi_flag(P, bad);
}

// Element-wise pass, vector form. A persistent grid walks the 32 x 32 tiles;
// in a tile each of the 256 threads takes a run of 4 consecutive columns of
// one row, and every step a thread loads the runs of two tiles before it forms
// and stores either, so its loads stay in flight together. NI (the op's input
// count) and kIn64 (some input is FP64) are compile-time, so a thread holds
// only the inputs it reads. The arithmetic is epi_row's with a zero
// accumulator: FP32 terms summed in FP32, then FP64 inputs added by FMA.
// For every op that stores no transposed split. Runs of the workspace are
// always 16-byte aligned; a caller's matrix (single, or a grouped batch's
// per-matrix table) is read as vectors where its runs are aligned.
template <int NI, bool kIn64>
using EwIn = typename std::conditional<kIn64, double, float>::type[NI][4];

// A run of 4 elements at q: one vector load when q is 16-byte aligned (always so
// in the workspace), else 4 element loads (a caller's matrix with an odd base or
// row stride).
template <typename T>
__device__ __forceinline__ void ld_run4(const T* q, T (&t)[4]) {
  if (((uintptr_t)q & 15u) == 0) {
    ld_vec<4>(q, t);
  } else {
#pragma unroll
    for (int w = 0; w < 4; ++w) t[w] = q[w];
  }
}

template <int NI, bool kIn64>
__device__ __forceinline__ void ew_load(const EpiParams& P, const EpiCtx& x, int r, int c0, EwIn<NI, kIn64>& in) {
  if (r >= x.n || c0 + 4 > x.n) return;  // padding and ragged runs: ew_emit's own paths
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const EpiIn& e = P.in[i];
    int64_t ld;
    if (kIn64 && e.dt == DT_F64) {
      double t[4];
      ld_run4(in_base<double>(e, x, &ld) + (int64_t)r * ld + c0, t);
#pragma unroll
      for (int w = 0; w < 4; ++w) in[i][w] = t[w];
    } else {
      float t[4];
      ld_run4(in_base<float>(e, x, &ld) + (int64_t)r * ld + c0, t);
#pragma unroll
      for (int w = 0; w < 4; ++w) in[i][w] = t[w];
    }
  }
}

// t: split-FP16 scales of the matrix (nullptr for other dtypes)
template <int NI, bool kIn64, bool kF16>
__device__ __forceinline__ bool ew_emit(const EpiParams& P, const EpiCtx& x, int r, int c0,
                                        const EwIn<NI, kIn64>& in, const SxTile* t) {
  constexpr int W = 4;
  if (r >= x.n) {
    epi_row_zero<W, kF16>(P, x, r, c0);
    return false;
  }
  if (c0 + W > x.n) {
    bool bad = false;
#pragma unroll
    for (int w = 0; w < W; ++w) bad |= epi_element<float, kF16>(P, x, r, c0 + w, 0.f, t);
    return bad;
  }
  bool bad = false;
#pragma unroll 1
  for (int j = 0; j < P.nout; ++j) {
    const EpiOut& o = P.out[j];
    if (o.f64) {
      // FP64 runs at 1/64 of the FP32 rate: an output that is one FP64 input
      // with coefficient 1 (plus the identity) is formed without FP64
      // arithmetic off the diagonal, where fma(1, x, 0) is x itself.
      int copy = -1, nterms = 0;
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        if (kIn64 && P.in[i].dt == DT_F64 ? o.in_d[i] != 0.0 : o.in_f[i] != 0.f) {
          ++nterms;
          if (kIn64 && P.in[i].dt == DT_F64 && o.in_d[i] == 1.0) copy = i;
        }
      }
      double v[W];
      if (kIn64 && nterms == 1 && copy >= 0) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
          if (i == copy)
#pragma unroll
            for (int w = 0; w < W; ++w) v[w] = (double)in[i][w];
        if (o.id_d != 0.0 && r >= c0 && r < c0 + W) {  // the one run that holds the diagonal element
#pragma unroll
          for (int w = 0; w < W; ++w)
            if (r == c0 + w) v[w] += o.id_d;
        }
      } else {
        float vf[W];
#pragma unroll
        for (int w = 0; w < W; ++w) vf[w] = 0.f;
#pragma unroll
        for (int i = 0; i < NI; ++i)
          if (o.in_f[i] != 0.f && (!kIn64 || P.in[i].dt != DT_F64))
#pragma unroll
            for (int w = 0; w < W; ++w) vf[w] = fmaf(o.in_f[i], (float)in[i][w], vf[w]);
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = (double)vf[w] + (r == c0 + w ? o.id_d : 0.0);
        if (kIn64) {
#pragma unroll
          for (int i = 0; i < NI; ++i)
            if (o.in_d[i] != 0.0 && P.in[i].dt == DT_F64)
#pragma unroll
              for (int w = 0; w < W; ++w) v[w] = fma(o.in_d[i], (double)in[i][w], v[w]);
        }
      }
      // finite: exponent field not all ones (integer test, no FP64 instruction)
#pragma unroll
      for (int w = 0; w < W; ++w) bad |= (__double2hiint(v[w]) & 0x7ff00000) == 0x7ff00000;
      const float sc = kF16 && t ? t->sc[j] : 1.f;
      bad |= fp16_overflow<W, double, kF16>(o, v, sc);
      st_row<W, double, kF16>(o, x, r, c0, v, sc);
    } else {
      float v[W];
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = r == c0 + w ? o.id_f : 0.f;
#pragma unroll
      for (int i = 0; i < NI; ++i)
        if (o.in_f[i] != 0.f)
#pragma unroll
          for (int w = 0; w < W; ++w) v[w] = fmaf(o.in_f[i], (float)in[i][w], v[w]);
#pragma unroll
      for (int w = 0; w < W; ++w) bad |= !isfinite(v[w]);
      const float sc = kF16 && t ? t->sc[j] : 1.f;
      bad |= fp16_overflow<W, float, kF16>(o, v, sc);
      st_row<W, float, kF16>(o, x, r, c0, v, sc);
    }
  }
  return bad;
}

// Tile t: the grouped table's entry, or row-major over tpr tiles per row.
__device__ __forceinline__ void ew_tile(const int4* tiles, int tpr, int t, int* mat, int* tr, int* tc) {
  if (tiles) {
    const int4 e = tiles[t];
    *mat = e.x;
    *tr = e.y;
    *tc = e.z;
  } else {
    *mat = 0;
    *tr = t / tpr;
    *tc = t - *tr * tpr;
  }
}

// Two tiles' inputs per thread: three CTAs per SM fit for up to two inputs,
// two CTAs (128 registers) for three or four.
template <int NI, bool kIn64, bool kF16>
__global__ void __launch_bounds__(256, NI <= 2 ? 3 : 2) ewise_vec_kernel(const int4* __restrict__ tiles, int ntiles, int tpr,
                                                            const __grid_constant__ EpiParams P) {
  const int dr = (int)(threadIdx.x >> 3), dc = 4 * (int)(threadIdx.x & 7);
  bool bad = false;
  for (int t = blockIdx.x; t < ntiles; t += 2 * gridDim.x) {
    const int u = t + gridDim.x;
    const bool two = u < ntiles;
    int ma, ra, ca, mb = 0, rb = 0, cb = 0;
    ew_tile(tiles, tpr, t, &ma, &ra, &ca);
    if (two) ew_tile(tiles, tpr, u, &mb, &rb, &cb);
    const EpiCtx xa = epi_ctx(P, ma);
    const EpiCtx xb = epi_ctx(P, mb);
    EwIn<NI, kIn64> a, b;
    ew_load<NI, kIn64>(P, xa, ra * 32 + dr, ca * 32 + dc, a);
    if (two) ew_load<NI, kIn64>(P, xb, rb * 32 + dr, cb * 32 + dc, b);
    SxTile sa, sb;  // split-FP16 scales of the two tiles' matrices
    if (kF16) {
      sx_tile(P, ma, &sa);
      if (two) sx_tile(P, mb, &sb);
    }
    bad |= ew_emit<NI, kIn64, kF16>(P, xa, ra * 32 + dr, ca * 32 + dc, a, kF16 ? &sa : nullptr);
    if (two) bad |= ew_emit<NI, kIn64, kF16>(P, xb, rb * 32 + dr, cb * 32 + dc, b, kF16 ? &sb : nullptr);
  }
  epi_flag(P, bad);
}

template <int NI, bool kIn64>
void launch_ewise_vec(const EpiParams& P, cudaStream_t s, const int4* tiles, int ntiles, int tpr) {
  const int want = (ntiles + 1) / 2;  // two tiles per CTA and step
  const int cap = (NI <= 2 ? 3 : 2) * sm_count();
  const int grid = want < cap ? want : cap;
  if (P.fp16)
    ewise_vec_kernel<NI, kIn64, true><<<grid, 256, 0, s>>>(tiles, ntiles, tpr, P);
  else
    ewise_vec_kernel<NI, kIn64, false><<<grid, 256, 0, s>>>(tiles, ntiles, tpr, P);
}

template <int NI>
void launch_ewise_vec(const EpiParams& P, cudaStream_t s, const int4* tiles, int ntiles, int tpr, bool in64) {
  if (in64)
    launch_ewise_vec<NI, true>(P, s, tiles, ntiles, tpr);
  else
    launch_ewise_vec<NI, false>(P, s, tiles, ntiles, tpr);
}

template <typename T>
cudaError_t launch_simt(const T* A, const T* B, int64_t ld, int64_t npad, const int4* tiles, int ntiles,
                        const EpiParams& P, cudaStream_t s, bool sym) {
  if (npad % BM != 0 || npad % BN != 0 || ld < npad) return cudaErrorInvalidValue;
  // FP32: 64 running sums per thread in dynamic shared memory (64 KB)
  constexpr size_t dyn = sizeof(T) == 4 ? 64 * TPB * sizeof(float) : 0;
  static std::atomic<int> attr_state[kMaxDevices];
  if (dyn) {
    const cudaError_t attr = once_per_device(attr_state, [] {
      return cudaFuncSetAttribute(simt_gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    });
    if (attr != cudaSuccess) return attr;
  }
  const int ktiles = (int)(npad / simt_bk(sizeof(T) == 8));
  if (tiles) {
    if (ntiles <= 0) return cudaSuccess;
    simt_gemm_kernel<T><<<ntiles, TPB, dyn, s>>>(A, B, ld, 0, tiles, 0, P);
  } else if (sym) {
    const int t = (int)(npad / BM);
    simt_gemm_kernel<T><<<t * (t + 1) / 2, TPB, dyn, s>>>(A, B, ld, ktiles, nullptr, t, P);
  } else {
    dim3 grid((unsigned)(npad / BN), (unsigned)(npad / BM));
    simt_gemm_kernel<T><<<grid, TPB, dyn, s>>>(A, B, ld, ktiles, nullptr, 0, P);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_simt_gemm_f64(const double* A, const double* B, int64_t ld, int64_t npad, const int4* tiles,
                                 int ntiles, const EpiParams& P, cudaStream_t s, bool sym) {
  return launch_simt<double>(A, B, ld, npad, tiles, ntiles, P, s, sym);
}

cudaError_t launch_simt_gemm_f32(const float* A, const float* B, int64_t ld, int64_t npad, const int4* tiles,
                                 int ntiles, const EpiParams& P, cudaStream_t s, bool sym) {
  return launch_simt<float>(A, B, ld, npad, tiles, ntiles, P, s, sym);
}

// ---- CUDA-core peak probe ----
// Every thread runs kChains independent FMA chains a = a * b + c for `iters`
// rounds (2 flops per FMA), so the FMA pipes see kChains independent
// instructions per warp per round; the grid holds 2048 threads per SM. The
// sum of the chains is written only if it equals a value it cannot reach,
// which keeps the compiler from removing the loop without a store per thread.
constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(T* sink, int iters, T b, T c) {
  T a[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int j = 0; j < kPeakChains; ++j) a[j] = fma(a[j], b, c);
    }
  }
  T t = 0;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) t += a[j];
  if (t == (T)-12345.678) *sink = t;
}

__device__ double g_peak_sink;

cudaError_t measure_fma_peak(int f64, double* tflops, cudaStream_t s) {
  *tflops = 0.0;
  double* sink = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&sink), g_peak_sink);
  if (e != cudaSuccess) return e;
  const int grid = sm_count() * (2048 / kPeakThreads);
  // a few ms of FMA work per launch on either pipe at GB300's rates
  const int iters = f64 ? 64 : 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return e;
  }
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run is a warm-up
    cudaEventRecord(e0, s);
    if (f64)
      fma_peak_kernel<double><<<grid, kPeakThreads, 0, s>>>(sink, iters, 0.999999, 1e-7);
    else
      fma_peak_kernel<float><<<grid, kPeakThreads, 0, s>>>(reinterpret_cast<float*>(sink), iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1, s);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * kPeakChains * 16.0 * iters * (double)grid * kPeakThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return cudaSuccess;
}

// ---- split-FP16 scaling (see SxParams) ----

// Largest column sum of a measured matrix m (column sums at col + off, npad
// per matrix): a reduction over the block. Every thread of the block calls it.
__device__ float sx_block_colmax(const SxScaleOp& q, int64_t off, int m, float* red) {
  const float* c = q.col + off + (int64_t)m * q.npad;
  float v = 0.f;
  for (int j = threadIdx.x; j < q.npad; j += blockDim.x) v = fmaxf(v, c[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
  return r;
}

// e with bound * 2^e <= 2^kSxTarget (0 for a zero or non-finite bound)
__device__ int sx_exponent(double bound) {
  if (!(bound > 0.0) || !isfinite(bound)) return 0;
  int k = 0;
  frexp(bound, &k);  // bound = f 2^k, 0.5 <= f < 1, so bound < 2^k
  const int e = kSxTarget - k;
  return e < -kSxMaxExp ? -kSxMaxExp : e > kSxMaxExp ? kSxMaxExp : e;
}

// a bound stored a hair above its computed value, so that its own rounding
// cannot make it smaller than the quantity it bounds
__device__ __forceinline__ float sx_up(double v) { return (float)v * (1.f + 1e-6f); }

__global__ void __launch_bounds__(256) sx_scale_kernel(const __grid_constant__ SxScaleOp q) {
  __shared__ float red[8];
  const int m = blockIdx.x;
  const int64_t nm = q.nmat;
  const float prev_colmax = q.prev_acc >= 0 ? sx_block_colmax(q, q.prev_col, m, red) : 0.f;
  if (threadIdx.x != 0) return;
  auto amax = [&](int rec) { return (double)__uint_as_float(q.amax[rec * nm + m]); };
  auto colmax = [&](int rec) { return (double)q.colmax[rec * nm + m]; };
  // op k-1's outputs from its measured accumulator
  if (q.prev_acc >= 0) {
    const double am = amax(q.prev_acc), cm = prev_colmax;
    for (int j = 0; j < q.prev_nout; ++j) {
      const int rec = q.prev_out[j];
      if (rec < 0) continue;
      double a = fabs((double)q.prev_a[j]) * am + fabs((double)q.prev_id[j]);
      double c = fabs((double)q.prev_a[j]) * cm + fabs((double)q.prev_id[j]);
      for (int i = 0; i < q.prev_nin; ++i) {
        a += fabs((double)q.prev_c[j][i]) * amax(q.prev_in[i]);
        c += fabs((double)q.prev_c[j][i]) * colmax(q.prev_in[i]);
      }
      q.amax[rec * nm + m] = __float_as_uint(sx_up(a));
      q.colmax[rec * nm + m] = sx_up(c);
    }
  }
  // op k's exponents, from the a priori bound on its accumulator
  const double acc = q.rec_a >= 0 ? amax(q.rec_a) * colmax(q.rec_b) : 0.0;
  for (int j = 0; j < q.nout; ++j) {
    const int rec = q.rec_out[j];
    if (rec < 0) continue;
    double a = fabs((double)q.acc[j]) * acc + fabs((double)q.id[j]);
    double c = fabs((double)q.id[j]);
    for (int i = 0; i < q.nin; ++i) {
      a += fabs((double)q.in[j][i]) * amax(q.rec_in[i]);
      c += fabs((double)q.in[j][i]) * colmax(q.rec_in[i]);
    }
    q.exp[rec * nm + m] = sx_exponent(a);
    if (q.rec_a < 0) {  // an element-wise pass: its bounds are its records
      q.amax[rec * nm + m] = __float_as_uint(sx_up(a));
      q.colmax[rec * nm + m] = sx_up(c);
    }
  }
}

// A caller's matrix: max |x| and the largest column sum, into amax[m] and
// colmax[m] (float bits, atomicMax). Block (panel of 32 columns, matrix m),
// 32 columns x 8 row lanes; each block sums its columns over all rows.
template <typename T>
__global__ void __launch_bounds__(256) sx_input_stats_kernel(const __grid_constant__ EpiIn in, const int* mat_n,
                                                              int n, unsigned* amax, unsigned* colmax) {
  __shared__ float ps[8][33];
  __shared__ float pm[8];
  const int m = blockIdx.y;
  const EpiCtx x = {mat_n ? mat_n[m] : n, m, 0};
  const int c = blockIdx.x * 32 + threadIdx.x;
  float sum = 0.f, mx = 0.f;
  if (c < x.n) {
    int64_t ld;
    const T* a = in_base<T>(in, x, &ld);
    for (int r = threadIdx.y; r < x.n; r += 8) {
      const float v = fabsf((float)a[(int64_t)r * ld + c]);
      sum += v;
      mx = fmaxf(mx, v);
    }
  }
  ps[threadIdx.y][threadIdx.x] = sum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x == 0) pm[threadIdx.y] = mx;
  __syncthreads();
  if (threadIdx.y == 0) {
    float t = 0.f;
#pragma unroll
    for (int y = 0; y < 8; ++y) t += ps[y][threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) {
      float b = 0.f;
#pragma unroll
      for (int y = 0; y < 8; ++y) b = fmaxf(b, pm[y]);
      if (b > 0.f) atomicMax(amax + m, __float_as_uint(b));
      if (t > 0.f) atomicMax(colmax + m, __float_as_uint(t));
    }
  }
}

int sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  const int n = per_device_value(cache, [] {
    const int d = current_device();
    int v = 0;
    if (d < 0 || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return v;
  });
  return n > 0 ? n : 1;
}

cudaError_t launch_sx_scale(const SxScaleOp& op, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  sx_scale_kernel<<<count, 256, 0, s>>>(op);
  return cudaGetLastError();
}

cudaError_t launch_sx_input_stats(const EpiIn& in, const int* mat_n, int n, int nmat, unsigned* amax,
                                  unsigned* colmax, cudaStream_t s) {
  if (nmat <= 0 || n <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((n + 31) / 32), (unsigned)nmat);
  if (in.dt == DT_F64)
    sx_input_stats_kernel<double><<<grid, dim3(32, 8), 0, s>>>(in, mat_n, n, amax, colmax);
  else
    sx_input_stats_kernel<float><<<grid, dim3(32, 8), 0, s>>>(in, mat_n, n, amax, colmax);
  return cudaGetLastError();
}

cudaError_t launch_ewise(const EpiParams& P, cudaStream_t s, const int4* tiles, int ntiles) {
  dim3 grid;
  if (tiles) {
    if (ntiles <= 0) return cudaSuccess;
    grid = dim3((unsigned)ntiles);
  } else {
    if (P.npad <= 0 || P.npad % 32 != 0) return P.npad <= 0 ? cudaSuccess : cudaErrorInvalidValue;
    grid = dim3((unsigned)(P.npad / 32), (unsigned)(P.npad / 32));
  }
  // the vector form serves every op without a transposed split (its loads fall
  // back to single elements where a caller's run is not 16-byte aligned)
  bool vec = true;
  for (int j = 0; j < P.nout; ++j)
    for (int k = 0; k < P.out[j].nsplit; ++k) vec &= !P.out[j].split[k].transposed;
  bool in64 = false;
  for (int i = 0; i < P.nin; ++i) in64 |= P.in[i].dt == DT_F64;
  if (vec && P.nin >= 1) {
    const int tpr = tiles ? 0 : (int)(P.npad / 32);
    const int nt = tiles ? ntiles : tpr * tpr;
    switch (P.nin) {
      case 1: launch_ewise_vec<1>(P, s, tiles, nt, tpr, in64); break;
      case 2: launch_ewise_vec<2>(P, s, tiles, nt, tpr, in64); break;
      case 3: launch_ewise_vec<3>(P, s, tiles, nt, tpr, in64); break;
      default: launch_ewise_vec<4>(P, s, tiles, nt, tpr, in64); break;
    }
  } else if (P.fp16) {
    ewise_kernel<true><<<grid, dim3(32, 8), 0, s>>>(tiles, P);
  } else {
    ewise_kernel<false><<<grid, dim3(32, 8), 0, s>>>(tiles, P);
  }
  return cudaGetLastError();
}

}  // namespace neumann
