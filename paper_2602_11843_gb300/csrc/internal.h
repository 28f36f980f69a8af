// Internal interfaces between the plan (host C++) and the CUDA kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>

namespace neumann {

// Values a launcher looks up once (SM count, resident clusters, a kernel's
// shared-memory attribute) belong to one device: a process may drive several
// GPUs from several host threads. They are cached per device index, 0 meaning
// "not looked up yet"; two threads that race on an entry compute the same value.
constexpr int kMaxDevices = 64;

inline int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return d >= 0 && d < kMaxDevices ? d : -1;
}

// The cached value for the current device, computing it with `get` (which
// returns a value > 0, or <= 0 on failure: not cached) on first use.
template <typename F>
inline int per_device_value(std::atomic<int> (&cache)[kMaxDevices], F get) {
  const int d = current_device();
  if (d < 0) return get();
  int v = cache[d].load(std::memory_order_acquire);
  if (v <= 0) {
    v = get();
    if (v > 0) cache[d].store(v, std::memory_order_release);
  }
  return v;
}

// Runs `init` (returning cudaError_t) once per device; later calls on that
// device return its first result.
template <typename F>
inline cudaError_t once_per_device(std::atomic<int> (&state)[kMaxDevices], F init) {
  const int d = current_device();
  if (d < 0) return cudaErrorInvalidDevice;
  int s = state[d].load(std::memory_order_acquire);
  if (s == 0) {
    const cudaError_t e = init();
    s = e == cudaSuccess ? 1 : 2 + (int)e;
    state[d].store(s, std::memory_order_release);
  }
  return s == 1 ? cudaSuccess : (cudaError_t)(s - 2);
}

enum : int { DT_F32 = 0, DT_F64 = 1 };

constexpr int kMaxIn = 4;
constexpr int kMaxOut = 5;
constexpr int kMaxDst = 2;
constexpr int kMaxSplit = 2;

// How an epilogue input or plain destination is addressed. The zero value is
// the caller's-matrix mode, which never writes outside the n x n block.
enum : int {
  EPI_PTR = 0,    // caller's matrix: p, leading dimension ld (single evaluation)
  EPI_WS = 1,     // workspace buffer: p + slab offset of the matrix, leading dimension ld;
                  // its padding (row or column >= n) is written as 0
  EPI_TABLE = 2,  // caller's matrices: p is a device array of per-matrix pointers,
                  // leading dimension n of that matrix (batched evaluation)
};

// An epilogue input: an n x n matrix read at the output element's (r, c).
struct EpiIn {
  const void* p;
  int64_t ld;
  int dt;
  int mode;
};

// A plain store of an output (row-major).
struct EpiDst {
  void* p;
  int64_t ld;
  int dt;
  int mode;
};

// A split store, row-major or transposed:
//   BF16: hi = RN_bf16(v), lo = RN_bf16(v - hi)
//   FP16: w = v * 2^e, hi = RN_fp16(w), lo = RN_fp16(w - hi), with the matrix's
//         own e (SxParams below)
struct EpiSplit {
  void* hi;
  void* lo;
  int64_t ld;
  int transposed;
};

// Per-matrix power-of-two scaling of the FP16 split operands. Every matrix a
// split-FP16 plan stores as a hi/lo pair is stored as x * 2^e with its own e,
// chosen before the producing launch from a bound on max |x| so that the bound
// maps to at most 2^14: hi never overflows FP16 (65504) and lo stays a normal
// FP16 number down to |x| ~ 2^-17 of the bound. A product of operands stored
// with e_A and e_B carries 2^(e_A + e_B), removed exactly in its epilogue.
// Bounds come from per-matrix "records": every op output, the caller's
// matrices and every product's accumulator have
//   amax    a bound on max |x| (IEEE bits)
//   colmax  a bound on max_j sum_i |x_ij|, the largest column sum
//   exp     the e of the output's split
// A product's epilogue measures its accumulator (max |acc| with atomicMax,
// the column sums of |acc| into `col`), once per staged chunk; the caller's
// matrices are measured by a pre-pass. For out = a acc + sum_i c_i in_i + d I,
//   |out| <= |a| amax(acc) + sum_i |c_i| amax(in_i) + |d|, and the same with colmax,
// and before the product, amax(acc) <= amax(L) colmax(R) (|(L R)_ij| <= max|L|
// sum_k |R_kj|). fp16_scale_kernel, launched before each op, turns the
// previous op's measured accumulator into its outputs' records and the bounds
// into this op's exponents.
constexpr int kSxTarget = 14;  // the bound is mapped to at most 2^14
constexpr int kSxMaxExp = 60;  // |e| <= 60 keeps every scale a normal FP32 power of two

struct SxParams {
  int active;        // split-FP16 plan: the fields below are valid
  int nmat;          // matrices per record (1, or the matrices of a grouped pass)
  int npad;          // padded order (column-sum arrays hold npad entries per matrix)
  int* exp;          // [rec * nmat + m]
  int rec_a, rec_b;  // records of a product's operands (-1: element-wise pass)
  int rec_out[kMaxOut];  // record of each output (-1: the caller's S)
  unsigned* acc_amax;    // a product's accumulator record: max |acc| per matrix (float bits)
  float* acc_col;        // and its column sums, npad per matrix
};

// The scale step before op k: finalise op k-1's output records from its
// measured accumulator (prev_*), then choose op k's exponents (and, for an
// element-wise pass, record its outputs' bounds). One block per matrix.
struct SxScaleOp {
  int nmat, npad;
  unsigned* amax;     // [rec * nmat + m]
  float* colmax;
  int* exp;
  float* col;         // column-sum arrays (offsets in floats below)
  // op k
  int rec_a, rec_b;   // product operands (-1: element-wise pass)
  int nin, nout;
  int rec_in[kMaxIn];
  int rec_out[kMaxOut];   // -1: the caller's S
  float acc[kMaxOut], id[kMaxOut], in[kMaxOut][kMaxIn];
  // op k-1, a product whose outputs' records are finalised here (prev_acc < 0: none)
  int prev_acc;          // its accumulator record
  int64_t prev_col;      // offset of its column sums
  int prev_nin, prev_nout;
  int prev_in[kMaxIn];
  int prev_out[kMaxOut];
  float prev_a[kMaxOut], prev_id[kMaxOut], prev_c[kMaxOut][kMaxIn];
};

// One launch's FP16 scales for one matrix, read at tile start.
struct SxTile {
  float acc;            // 2^-(e_A + e_B): the accumulator in true units
  float sc[kMaxOut];    // 2^e of each output's split
};

// out = acc_coef * acc + sum_i in_coef[i] * in[i] + id_coef * [r == c]
struct EpiOut {
  double acc_d, id_d, in_d[kMaxIn];
  float acc_f, id_f, in_f[kMaxIn];
  int f64;  // evaluate in double
  int ndst;
  EpiDst dst[kMaxDst];
  int nsplit;
  EpiSplit split[kMaxSplit];
};

// Everything a GEMM (or element-wise) launch writes besides its accumulator.
struct EpiParams {
  int n;     // logical order
  int npad;  // padded order of workspace buffers: padding elements of pad
             // destinations and of split stores are written as 0, so a buffer
             // never needs zeroing and the GEMM main loops need no bounds checks
  int nin;
  EpiIn in[kMaxIn];
  int nout;
  EpiOut out[kMaxOut];
  unsigned* status;  // device word, NEUMANN_STATUS_* bits are OR-ed in
  int fp16;          // split stores use the scaled FP16 pair (the kernel instance is chosen on the host)
  // Batched (grouped) launches: matrix m has order mat_n[m] and occupies
  // elements [m * mat_stride, (m + 1) * mat_stride) of every workspace buffer.
  // nullptr for a single evaluation (order n, offset 0).
  const int* mat_n;
  int64_t mat_stride;
  // Set by the host for ops with at most one FP64 input (f64_in, else -1):
  // the tensor-core epilogue may take its lean path (boundary chunks: edge_ok).
  // f32_idx[0 .. nf32-1]: the FP32 inputs in index order.
  int fast;
  int f64_in;
  int nf32;
  int f32_idx[kMaxIn];
  // Every input is a workspace buffer: reads anywhere in the padded block are
  // in bounds, so the lean path may also take boundary chunks (zeros stored
  // outside the n x n block, the caller's matrices written inside it only).
  int edge_ok;
  SxParams sx;  // split-FP16 scaling (sx.active = 0 otherwise)
};

// Split-operand tensor maps of one tensor-core product C = A B:
// A as (hi, lo) row-major, B as (hi, lo) stored transposed (row j of the
// stored matrix is column j of B), both padded_n x padded_n, BF16 or FP16.
// pair: the product runs on 2-CTA clusters (256 x 256 tiles; each CTA loads
// 128 rows of the stored B^T, so the B maps have 128-row boxes).
// group: row tiles per group of the grouped raster of a single product.
// precise: K accumulated in chunks summed with round-to-nearest (256 x 128
// tiles on CTA pairs; the B maps have 64-row boxes).
// sym: a symmetric product (pairs only): the device list of the nsym tiles
// (tile row, tile column) on or above the diagonal; the tiles above it also
// write their transpose.
struct TcMaps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
  int fp16;
  int pair;
  int group;
  int precise;
  const int2* sym;
  int nsym;
  int b_mn;  // B is read MN-major from its row-major pair (bt_* are then row-major arrays of B)
};

constexpr int kDefaultRasterGroup = 8;

// ---- launchers (kernels_simt.cu) ----
// Streaming multiprocessors of the current device (cached per device; 1 if unknown).
int sm_count();
// The CUDA cores' FMA rate (FP32, or FP64 when f64), TFLOP/s: the best of three
// timed launches of independent FMA chains on every SM (synchronises `s`).
cudaError_t measure_fma_peak(int f64, double* tflops, cudaStream_t s);
// K depth of one shared-memory stage of the SIMT product: 16 (FP32) or 8 (FP64).
constexpr int simt_bk(bool f64) { return f64 ? 8 : 16; }
// tiles == nullptr: one padded npad x npad product. Otherwise a grouped launch
// over a batch: ntiles entries {matrix, tile row, tile column, K steps of simt_bk}.
// sym (single products only): the product is symmetric; only the 128 x 128
// tiles on or above the diagonal run, writing their transposes too.
cudaError_t launch_simt_gemm_f64(const double* A, const double* B, int64_t ld, int64_t npad, const int4* tiles,
                                 int ntiles, const EpiParams& P, cudaStream_t s, bool sym = false);
cudaError_t launch_simt_gemm_f32(const float* A, const float* B, int64_t ld, int64_t npad, const int4* tiles,
                                 int ntiles, const EpiParams& P, cudaStream_t s, bool sym = false);
// Element-wise epilogue with acc = 0: over the npad x npad elements, or (grouped)
// over ntiles 32 x 32 tiles {matrix, tile row, tile column}.
cudaError_t launch_ewise(const EpiParams& P, cudaStream_t s, const int4* tiles = nullptr, int ntiles = 0);
// Split-FP16 scaling: the scale step of one op, one block for each of the
// pass's `count` matrices; and the max |x| and largest column sum of a caller's
// matrix `in` (n x n, or per matrix of a grouped pass through mat_n, n the
// largest order) into amax[m] and colmax[m] (float bits; must start at 0).
cudaError_t launch_sx_scale(const SxScaleOp& op, int count, cudaStream_t s);
cudaError_t launch_sx_input_stats(const EpiIn& in, const int* mat_n, int n, int nmat, unsigned* amax,
                                  unsigned* colmax, cudaStream_t s);

// ---- the resident small-order batch kernel (kernels_resident.cu) ----
// One op of a scheme, as the resident kernel runs it. Slots index the CTA's
// shared-memory matrices (-1: the caller's A for an input, the caller's S for
// an output): every slot has an FP32 copy, and the slots the plan keeps in
// FP64 also an FP64 copy (f64_of). Coefficients as in EpiOut.
constexpr int kResMaxN = 64;                 // largest order the resident kernel holds
constexpr int kResSmemBudget = 220 * 1024;   // dynamic shared memory of one CTA at most
struct ResOp {
  int gemm;                 // 1: product acc = a b, then the epilogue; 0: element-wise (acc = 0)
  int a, b;
  int nin, nout;
  int in_slot[kMaxIn], in_f64[kMaxIn];
  int out_slot[kMaxOut], out_f32[kMaxOut], out_f64[kMaxOut], f64[kMaxOut];
  float acc_f[kMaxOut], id_f[kMaxOut], in_f[kMaxOut][kMaxIn];
  double acc_d[kMaxOut], id_d[kMaxOut], in_d[kMaxOut][kMaxIn];
};
struct ResParams {
  const ResOp* ops;         // device program, copied into each CTA's shared memory
  int nops;
  int nslots;               // FP32 matrices, nmax x nmax each
  int nf64;                 // FP64 matrices
  int f64_of[16];           // slot -> FP64 copy index (-1: none)
  int nmax;                 // largest order of the launch (rounded up to 4)
  int count;                // matrices
  const int* mat_n;         // device: orders (largest first)
  const void* const* A;     // device: caller pointers (leading dimension n_i)
  void* const* S;
  int io_f64;               // A and S are double (else float)
  int mode;                 // 0 FP32 products, 1 split BF16, 2 split FP16 (per-matrix scale)
  unsigned* status;
};
// Shared memory of a CTA holding the program and nslots FP32 + nf64 FP64
// matrices of order nmax; split modes add the current product's two operands
// as packed hi/lo words (4 bytes an element each).
inline size_t resident_smem(int nslots, int nf64, int nops, int nmax, bool split = false) {
  return (size_t)nmax * nmax * (4 * (size_t)nslots + 8 * (size_t)nf64 + (split ? 8 : 0)) +
         (size_t)nops * sizeof(ResOp);
}
// Columns of a thread's output block for order nmax (its rows are 4): 1 up to
// order 16, else 2.
inline int resident_cw(int nmax) { return nmax <= 16 ? 1 : 2; }
// Threads of a CTA for order nmax: one per 4 x resident_cw output block,
// rounded up to warps.
inline int resident_threads(int nmax) {
  const int ld = (nmax + 3) / 4 * 4;
  return ((ld / 4) * (ld / resident_cw(nmax)) + 31) / 32 * 32;
}
// The matrices of one launch in a persistent grid (as many CTAs as fit on the
// device at once, at most one per matrix): CTA b runs matrices b, b + grid, ...,
// each through the whole op program with its state in shared memory.
cudaError_t launch_resident(const ResParams& P, cudaStream_t s);

// ---- launchers (kernels_tc.cu) ----
// Encode the four tensor maps over padded_n x padded_n BF16 arrays with leading
// dimension ld; with count > 0, over count stacked padded_n x padded_n slabs
// (3-D maps, one slab per matrix of a batch).
// pair_mode: -1 CTA pairs where tc_uses_pair says so, 0 never, 1 always (single
// products only). group: row tiles per raster group (>= 1).
bool tc_make_maps(TcMaps* m, void* a_hi, void* a_lo, void* bt_hi, void* bt_lo, int64_t npad, int64_t ld,
                  int count = 0, int fp16 = 0, int pair_mode = -1, int group = kDefaultRasterGroup,
                  int precise = 0, int b_mn = 0);
// Whether a product of padded order npad (count = 0: single matrix) runs on CTA pairs.
bool tc_uses_pair(int64_t npad, int count);
// tiles == nullptr: one npad x npad product. Otherwise a grouped launch over a
// batch (3-D maps): ntiles entries {matrix, tile row, K steps of 32, 0}; each
// tile covers 128 rows and all 256 columns of its matrix's slab.
cudaError_t launch_tc_gemm(const TcMaps& maps, int64_t npad, const EpiParams& P, cudaStream_t s,
                           const int4* tiles = nullptr, int ntiles = 0);

// One thread waits (bounded by limit_ns) on an mbarrier nothing arrives on and
// sets NEUMANN_STATUS_TIMEOUT in *status when the limit passes.
cudaError_t launch_wait_probe(unsigned* status, uint64_t limit_ns, cudaStream_t s);

// ---- approximate kernel coefficients (approx_kernels.cpp) ----
// Radix 15: set 0 refined, 1 printed. Returns false if the refinement did not converge.
bool radix15_coefficients(int set, double coef[28], double* prefix_err, double* s15, double* s16);
// Radix 24 or 25 (five products): l2, r2, l3, r3, l4, r4, l5, r5, gamma.
constexpr int kApproxP5Params = 41;
bool radix_p5_coefficients(int m, double coef[kApproxP5Params], double* prefix_err, double* spill);

}  // namespace neumann
