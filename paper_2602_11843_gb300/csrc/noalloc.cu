// neumann_matmul_noalloc: the split-BF16 tensor-core product C = A B for
// callers that must not allocate device memory.
//
// Who needs it: code that cannot call cudaMalloc / cudaFree at the point where
// it wants a product. Examples are code running under an allocator that owns
// all device memory (a framework's caching allocator, or an allocation hook
// that must not re-enter the driver's allocator), and latency-critical loops
// that cannot take the device-wide synchronisation that cudaFree implies. Such
// a caller can neither create a plan workspace nor let neumann_eval allocate
// one on first use.
//
// What it does: the same two steps as neumann_plan_matmul on a SPLIT_BF16
// plan. An element-wise pass splits A and B into row-major hi/lo BF16 pairs
// (the kernel reads B's pair MN-major), then the persistent tcgen05 kernel forms
// Ahi Bhi + Ahi Blo + Alo Bhi and writes C. The only difference is where the
// scratch lives: in g_noalloc_scratch below, a file-scope device array that the
// CUDA runtime places in every device context that loads this library's code
// and keeps until the process exits. It holds a 256-byte status block (the
// device status word, NEUMANN_STATUS_* bits, read and cleared by
// neumann_matmul_noalloc_status) followed by the four operand matrices. Its
// size fixes the largest order this call accepts, kNoAllocMaxN = 1024
// (4 matrices x 1024^2 x 2 bytes = 8 MiB).
//
// Sharing: every call on a device uses the same array. The split pass rewrites
// all of the operand area (padding included) before the product reads it, so
// no operand contents need to survive between calls; the status word starts at
// zero when the module is loaded and is cleared only by its reader. Calls whose
// work overlaps on the GPU (concurrent streams, or host threads on different
// streams) race on the array; serialise them.
//
// The device address of the array is looked up on every call, with the
// caller's device current (the stream must belong to that device). Once the
// module is loaded the lookup is a runtime table query that allocates nothing;
// looking it up per call, rather than caching it, keeps a call correct after
// the primary context was reset and the module reloaded at another address.
#include <string.h>

#include "internal.h"
#include "neumann.h"

namespace neumann {
namespace {

constexpr int64_t kNoAllocMaxN = 1024;
constexpr size_t kNoAllocMatBytes = (size_t)kNoAllocMaxN * kNoAllocMaxN * 2;  // one BF16 matrix

constexpr size_t kStatusBytes = 256;  // status word, padded to keep the operands 256-byte aligned

// status block | Ahi | Alo | Bhi | Blo, each matrix padded_n x padded_n with padded_n <= 1024.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStatusBytes + 4 * kNoAllocMatBytes];

// The host symbol g_noalloc_scratch is only a handle; its device address in
// the current device's context is looked up with that device current.
int scratch_address(char** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return NEUMANN_ECUDA;
  }
  *out = reinterpret_cast<char*>(p);
  return NEUMANN_OK;
}

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* x = reinterpret_cast<const char*>(a);
  const char* y = reinterpret_cast<const char*>(b);
  return x < y + bbytes && y < x + abytes;
}

// Element-wise split of one FP64 matrix into a row-major hi/lo pair.
EpiParams split_params(int64_t n, int64_t npad, const void* X, int64_t ldx, char* hi, char* lo, unsigned* status) {
  EpiParams P;
  memset(&P, 0, sizeof(P));
  P.n = (int)n;
  P.npad = (int)npad;
  P.nin = 1;
  P.in[0] = EpiIn{X, ldx, DT_F64, EPI_PTR};
  P.nout = 1;
  EpiOut& o = P.out[0];
  o.in_d[0] = 1.0;
  o.in_f[0] = 1.0f;
  o.f64 = 1;
  o.nsplit = 1;
  o.split[0] = EpiSplit{hi, lo, npad, 0};
  P.status = status;
  P.f64_in = -1;
  return P;
}

}  // namespace
}  // namespace neumann

using namespace neumann;

extern "C" int neumann_matmul_noalloc(int64_t n, const void* A, int64_t lda, const void* B, int64_t ldb, void* C,
                                      int64_t ldc, void* stream) {
  if (n < 1 || n > kNoAllocMaxN || !A || !B || !C || lda < n || ldb < n || ldc < n) return NEUMANN_EINVAL;
  const size_t cbytes = ((size_t)(n - 1) * (size_t)ldc + (size_t)n) * 8;
  if (overlaps(A, ((size_t)(n - 1) * (size_t)lda + (size_t)n) * 8, C, cbytes) ||
      overlaps(B, ((size_t)(n - 1) * (size_t)ldb + (size_t)n) * 8, C, cbytes))
    return NEUMANN_EINVAL;
  char* ws = nullptr;
  int rc = scratch_address(&ws);
  if (rc) return rc;
  const int64_t npad = (n + 255) / 256 * 256;
  const size_t mat = (size_t)npad * (size_t)npad * 2;
  unsigned* status = reinterpret_cast<unsigned*>(ws);
  ws += kStatusBytes;
  char* a_hi = ws;
  char* a_lo = ws + mat;
  char* b_hi = ws + 2 * mat;
  char* b_lo = ws + 3 * mat;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  EpiParams pa = split_params(n, npad, A, lda, a_hi, a_lo, status);
  if (launch_ewise(pa, s) != cudaSuccess) return NEUMANN_ECUDA;
  EpiParams pb = split_params(n, npad, B, ldb, b_hi, b_lo, status);
  if (launch_ewise(pb, s) != cudaSuccess) return NEUMANN_ECUDA;

  TcMaps maps;
  if (!tc_make_maps(&maps, a_hi, a_lo, b_hi, b_lo, npad, npad, 0, 0, -1, kDefaultRasterGroup, 0, /*b_mn=*/1))
    return NEUMANN_ECUDA;
  EpiParams pc;
  memset(&pc, 0, sizeof(pc));
  pc.n = (int)n;
  pc.npad = (int)npad;
  pc.nout = 1;
  pc.out[0].acc_d = 1.0;
  pc.out[0].acc_f = 1.0f;
  pc.out[0].f64 = 1;
  pc.out[0].ndst = 1;
  pc.out[0].dst[0] = EpiDst{C, ldc, DT_F64, EPI_PTR};
  pc.status = status;
  pc.fast = 1;
  pc.f64_in = -1;
  if (launch_tc_gemm(maps, npad, pc, s) != cudaSuccess) return NEUMANN_ECUDA;
  return NEUMANN_OK;
}

extern "C" int neumann_matmul_noalloc_status(void* stream, unsigned* status) {
  if (!status) return NEUMANN_EINVAL;
  *status = 0;
  char* ws = nullptr;
  int rc = scratch_address(&ws);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned v = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemcpyAsync(&v, ws, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NEUMANN_ECUDA;
  if (v && (cudaMemsetAsync(ws, 0, sizeof(v), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
    return NEUMANN_ECUDA;
  *status = v;
  return NEUMANN_OK;
}
