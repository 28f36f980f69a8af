// Internal interfaces between the plan (host C++) and the CUDA kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace neumann {

enum : int { DT_F32 = 0, DT_F64 = 1 };

constexpr int kMaxIn = 4;
constexpr int kMaxOut = 4;
constexpr int kMaxDst = 2;
constexpr int kMaxSplit = 2;

// An epilogue input: an n x n matrix read at the output element's (r, c).
struct EpiIn {
  const void* p;
  int64_t ld;
  int dt;
};

// A plain store of an output (row-major).
struct EpiDst {
  void* p;
  int64_t ld;
  int dt;
  int pad;  // workspace buffer: elements in [n, npad) are written as 0
};

// A split store: hi = RN_bf16(v), lo = RN_bf16(v - hi), row-major or transposed.
struct EpiSplit {
  void* hi;
  void* lo;
  int64_t ld;
  int transposed;
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
};

// Split-operand tensor maps of one tensor-core product C = A B:
// A as (hi, lo) row-major, B as (hi, lo) stored transposed (row j of the
// stored matrix is column j of B), both padded_n x padded_n, BF16.
struct TcMaps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

// ---- launchers (kernels_simt.cu) ----
cudaError_t launch_simt_gemm_f64(const double* A, const double* B, int64_t ld, int64_t npad,
                                 const EpiParams& P, cudaStream_t s);
cudaError_t launch_simt_gemm_f32(const float* A, const float* B, int64_t ld, int64_t npad,
                                 const EpiParams& P, cudaStream_t s);
// Element-wise epilogue with acc = 0 over the n x n elements.
cudaError_t launch_ewise(const EpiParams& P, cudaStream_t s);

// ---- launchers (kernels_tc.cu) ----
// Encode the four tensor maps over padded_n x padded_n BF16 arrays with leading dimension ld.
bool tc_make_maps(TcMaps* m, void* a_hi, void* a_lo, void* bt_hi, void* bt_lo, int64_t npad, int64_t ld);
cudaError_t launch_tc_gemm(const TcMaps& maps, int64_t npad, const EpiParams& P, cudaStream_t s);

// ---- radix-15 coefficients (radix15.cpp) ----
// set 0: refined, 1: printed. Returns false if the refinement did not converge.
bool radix15_coefficients(int set, double coef[28], double* prefix_err, double* s15, double* s16);

}  // namespace neumann
