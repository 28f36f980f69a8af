// Plan construction (the per-level scheduler), workspace layout, execution,
// and the C ABI declared in include/neumann.h.
//
// Every scheme is compiled at plan time into a list of operations, each a
// product (GEMM) or an element-wise pass, both ending in the fused epilogue.
// A radix level with kernel f works on the residual R (R_0 = A) and the
// partial sum Y (Y_0 = I), Sec. 5.3 eq. generalradix:
//   kernel     G = f(R) - I            mu_m products (Thm 3.1; Sec. 4.1; Sec. 2.3)
//   concat     Y <- Y + Y G            1 product; at level 1 Y = I + G, no product
//   residual   R <- R + R G - G        1 product; skipped after the last level
// The residual line is I - (I - R) f(R) (proof of Lemma 5.7), which for an
// exact kernel T_m is the next power R^m (telescoping, Sec. 2.2). With
// NEUMANN_FLAG_RESIDUAL_PAPER it is formed as I - (I - A) Y instead (eq.
// generalradix). Storing G = f(R) - I rather than f(R) keeps the identity out
// of the products and lets the residual combine small quantities.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "internal.h"
#include "neumann.h"

using namespace neumann;

namespace {

enum Rep : uint32_t { REP_W = 1, REP_F64 = 2, REP_OPA = 4, REP_OPB = 8 };
constexpr uint32_t REP_ALL = REP_W | REP_F64 | REP_OPA | REP_OPB;

// Workspace matrices ("slots"). R and Y ping-pong: a product that reads one
// of them as an operand writes the other.
// SL_P3, SL_Q5L, SL_Q5R: the five-product kernels' third product and partial fifth factors.
enum : int {
  SL_R0, SL_R1, SL_Y0, SL_Y1, SL_LF0, SL_LF1, SL_RF0, SL_RF1, SL_P1, SL_P2, SL_C, SL_G, SL_A0,
  SL_P3, SL_Q5L, SL_Q5R, SL_N
};
constexpr int SL_NONE = -1, SL_USER_A = -2, SL_USER_B = -3, SL_USER_S = -4;

struct InRef {
  int slot;
  uint32_t rep;  // REP_W or REP_F64
};

struct OutSpec {
  int slot;
  uint32_t reps;
  double acc, id;
  double in[kMaxIn];
};

enum OpKind { OP_GEMM, OP_EWISE };

struct Op {
  OpKind kind;
  int a, b;  // GEMM operands (a read as left operand, b as right operand)
  int nin;
  InRef in[kMaxIn];
  int nout;
  OutSpec out[kMaxOut];
};

enum Path { PATH_F64, PATH_F32, PATH_TC };

constexpr int kMaxTimedProducts = 1 << 16;
constexpr int64_t kGroupedMaxN = 256;  // batched orders up to this run as grouped launches
constexpr int kGroupedChunk = 2048;    // matrices per grouped pass

struct SlotBufs {
  size_t w, f64, a_hi, a_lo, b_hi, b_lo;
};
constexpr size_t NOBUF = (size_t)-1;
// Tensor-core products read B MN-major from row-major hi/lo pairs (no
// transposed pair is stored).
constexpr bool kMnMajorB = true;

Op mk_gemm(int a, int b) {
  Op op;
  memset(&op, 0, sizeof(op));
  op.kind = OP_GEMM;
  op.a = a;
  op.b = b;
  return op;
}

Op mk_ewise() {
  Op op;
  memset(&op, 0, sizeof(op));
  op.kind = OP_EWISE;
  op.a = op.b = SL_NONE;
  return op;
}

void add_in(Op& op, int slot, uint32_t rep) { op.in[op.nin++] = InRef{slot, rep}; }

OutSpec& add_out(Op& op, int slot, uint32_t reps, double acc, double id) {
  OutSpec& o = op.out[op.nout++];
  memset(&o, 0, sizeof(o));
  o.slot = slot;
  o.reps = reps;
  o.acc = acc;
  o.id = id;
  return o;
}

int mu_of(int m) {
  switch (m) {
    case 2: return 0;
    case 3: return 1;
    case 5: return 2;
    case 9: return 3;
    case 15: return 4;
    case 24:
    case 25:
    case 27:
    case 31:
    case 33: return 5;
  }
  return -1;
}

bool pure_power(int64_t k, int m, std::vector<int>* levels) {
  levels->clear();
  while (k > 1) {
    if (k % m) return false;
    k /= m;
    levels->push_back(m);
  }
  return true;
}

}  // namespace

struct neumann_plan_s {
  int64_t n = 0, k = 0, npad = 0;
  int radix = 0, dtype = 0;
  uint32_t flags = 0;
  Path path = PATH_F64;
  int dt_io = DT_F64;
  std::vector<int> levels;
  int64_t formula = 0;
  std::vector<Op> ops, mm_ops;
  uint32_t reps[SL_N];
  SlotBufs bufs[SL_N];
  size_t ws_bytes = 0;
  char* ws = nullptr;
  bool ws_owned = false;
  std::vector<TcMaps> maps, mm_maps;
  bool maps_ready = false;
  double c15[28];
  double cp5[kApproxP5Params];  // radix 24 / 25 circuit
  cudaStream_t last_stream = nullptr;
  std::vector<cudaEvent_t> events;
  // neumann_eval_host: two sets of device staging buffers, an input and an
  // output copy stream, and per set the events that order copy-in, evaluation
  // and copy-out (set i % 2 serves call i)
  struct HostStage {
    char* a = nullptr;
    char* s = nullptr;
    cudaEvent_t in = nullptr, done = nullptr, out = nullptr;
    bool used = false;
  } host[2];
  cudaStream_t cs_in = nullptr, cs_out = nullptr;
  int64_t host_calls = 0;
  // neumann_eval_batched_host: one packed staging pair (stable device pointers,
  // so the grouped tile tables stay cached). Within an evaluation, `a_free` is
  // recorded after the last op that reads A and the first op that writes S
  // waits for `s_free` (the previous call's copy-out).
  char* pk_a = nullptr;
  char* pk_s = nullptr;
  size_t pk_bytes = 0;
  cudaEvent_t pk_in = nullptr, pk_a_free = nullptr, pk_done = nullptr, pk_s_free = nullptr;
  cudaEvent_t pk_a_free_res = nullptr;  // the resident launches have read A
  bool pk_used = false;
  cudaEvent_t hook_after_a = nullptr;  // record after the last A-reading op (set during one run_ops)
  cudaEvent_t hook_before_s = nullptr;  // wait before the first S-writing op
  int timed = 0;
  // launch configuration of the tensor-core products, set by the autotuner or
  // taken from an earlier tuning of the same shape in this process
  // NEUMANN_FLAG_SYMMETRIC on a split single plan: the scheme's products run
  // only the tiles on or above the diagonal (list at off_sym, nsym entries)
  bool sym = false;
  size_t off_sym = 0;
  int nsym = 0;
  // tensor-core products read B MN-major from its row-major hi/lo pair, so no
  // transposed pair is ever stored
  bool bmn = false;
  // Split-FP16 per-matrix scaling (SxParams): every output of every op and
  // every product's accumulator is a record; records 0 and 1 are the caller's
  // A and B (measured by a pre-pass). op_sx / mm_sx give each op's operand,
  // input, output and accumulator records. The stats region
  // [amax | colmax | exp | column sums of the accumulators] is cleared before each pass.
  struct OpSx {
    int rec_a, rec_b, rec_acc;
    int rec_in[kMaxIn];
    int rec_out[kMaxOut];
  };
  bool sx = false;
  int sx_nrec = 0, sx_nmat = 1;
  std::vector<OpSx> op_sx, mm_sx;
  std::vector<int64_t> sx_col;    // per record: offset (floats) of its column sums (accumulators), or -1
  size_t off_sx = 0, sx_bytes = 0, off_sx_amax = 0, off_sx_colmax = 0, off_sx_exp = 0, off_sx_col = 0;
  int tune_pair = -1;                    // -1: CTA pairs from padded order 4096; 0 never; 1 always
  int tune_group = kDefaultRasterGroup;  // row tiles per raster group of a single product
  int chunk_run = 0;                     // grouped batches: matrices per pass (0: chunk)
  bool tuned = false;
  // batched
  bool batched = false;
  int count = 0;
  int64_t max_n = 0;
  std::map<int64_t, neumann_plan_s*> sub;  // per-order plans (max_n > 256)
  // Grouped batched evaluation (max_n <= 256): `chunk` matrices at a time sit
  // in stacked npad x npad slabs of every workspace buffer, and each operation
  // of the scheme is one launch over all of them, driven by tile tables.
  bool grouped = false;
  int chunk = 0;
  size_t slab = 0;  // elements per slab
  // device tables for every chunk of the batch (offsets into the workspace)
  size_t off_matn = 0, off_atab = 0, off_stab = 0, off_tc = 0, off_simt = 0, off_ew = 0;
  // the chunk being launched: device pointers into those tables, entry counts
  const int* cur_matn = nullptr;
  const void* cur_atab = nullptr;
  const void* cur_stab = nullptr;
  const int4 *cur_tc = nullptr, *cur_simt = nullptr, *cur_ew = nullptr;
  int n_tc = 0, n_simt = 0, n_ew = 0;
  int cur_count = 0;  // matrices in the pass being launched
  // pinned host image of the tables, the call it was built for, and the event
  // after its upload (the image is rewritten only once that copy is done)
  char* h_tab = nullptr;
  size_t h_tab_bytes = 0;
  cudaEvent_t tab_event = nullptr;
  int last_chunk_run = 0;
  std::vector<int64_t> last_n;
  std::vector<const void*> last_a;
  std::vector<void*> last_s;
  struct Chunk {
    int first, count, tc0, ntc, simt0, nsimt, ew0, new_;
  };
  std::vector<Chunk> chunks;
  // The resident kernel (kernels_resident.cu) for the batch's matrices of order
  // <= res_limit (res_maxn: the most its shared memory holds): the op program
  // with slots renumbered (res_slot_of) and FP64 copies (res_f64_of), and the
  // table of resident matrices in the workspace. The last call's resident
  // matrices (largest first) split into size classes, one launch each:
  // res_class[c] = {first, count, nmax}.
  std::vector<ResOp> res_ops;
  int res_maxn = 0, res_limit = 0, res_nslots = 0, res_nf64 = 0, res_count = 0, last_res_limit = -1;
  int res_slot_of[16];
  int res_f64_of[16];
  std::vector<int3> res_class;
  size_t off_res_ops = 0, off_res_matn = 0, off_res_atab = 0, off_res_stab = 0;
  // the resident launches run on their own stream, forked from and joined back
  // into the evaluation's stream, alongside the grouped passes
  cudaStream_t res_stream = nullptr;
  cudaEvent_t res_fork = nullptr, res_join = nullptr;
  cudaEvent_t hook_after_a_res = nullptr;  // record once the resident launches have read A (host calls)
};

namespace {

// ---------------------------------------------------------------- scheduler

struct Sched {
  neumann_plan_s* p;
  bool paper;

  std::vector<Op>& ops() { return p->ops; }

  // Kernel ops for G = f(R) - I. The last product also writes G (with greps)
  // and, when ytarget != SL_NONE, the first partial sum Y = I + G.
  void kernel(int m, int R, uint32_t greps, int ytarget, uint32_t yreps) {
    // The radix-15 and five-product circuits: after P2, C = g1 B + g2 P1 + g3 P2
    // holds P2's share, so a combination c1 B + c2 P1 + c3 P2 that P3's
    // epilogue forms equals (c1 - t g1) B + (c2 - t g2) P1 + t C with t = c3 / g3,
    // and P3 reads (B, P1, C) instead of (B, P1, P2, C). This multiplies C's FP32
    // rounding by |t| (at most 4.8 over the kernels built, 0.21 for radix 15);
    // where some |t| would exceed kSubMax, P3 reads P2 as stored.
    constexpr double kSubMax = 16.0;
    auto p2_via_c = [&](const double* g, std::initializer_list<double> c3) {
      if (g[2] == 0.0) return false;
      for (double c : c3)
        if (std::fabs(c / g[2]) > kSubMax) return false;
      return true;
    };
    // in[0..2] of an output of P3 over the inputs (B, P1, C) or (B, P1, P2, C)
    auto comb3 = [](OutSpec& o, bool via_c, const double* g, double c1, double c2, double c3) {
      if (via_c) {
        const double t = c3 / g[2];
        o.in[0] = c1 - t * g[0];
        o.in[1] = c2 - t * g[1];
        o.in[2] = t;
      } else {
        o.in[0] = c1;
        o.in[1] = c2;
        o.in[2] = c3;
      }
    };
    auto tail = [&](Op& op, double acc, std::initializer_list<double> ins) {
      // G = sum ins * inputs + acc * product; Y = I + G
      if (greps) {
        OutSpec& g = add_out(op, SL_G, greps, acc, 0.0);
        int i = 0;
        for (double c : ins) g.in[i++] = c;
      }
      if (ytarget != SL_NONE) {
        OutSpec& y = add_out(op, ytarget, yreps, acc, 1.0);
        int i = 0;
        for (double c : ins) y.in[i++] = c;
      }
    };
    if (m == 3) {  // T_3 = I + B + B^2 (Sec. 2.1): G = B + U
      Op op = mk_gemm(R, R);
      add_in(op, R, REP_W);
      tail(op, 1.0, {1.0});
      ops().push_back(op);
    } else if (m == 5) {  // quinary (Sec. 2.3): U = B^2, V = U (B + U), G = B + U + V
      Op op1 = mk_gemm(R, R);
      add_in(op1, R, REP_W);
      add_out(op1, SL_P1, REP_W | REP_OPA, 1.0, 0.0);
      add_out(op1, SL_RF0, REP_OPB, 1.0, 0.0).in[0] = 1.0;
      ops().push_back(op1);
      Op op2 = mk_gemm(SL_P1, SL_RF0);
      add_in(op2, R, REP_W);
      add_in(op2, SL_P1, REP_W);
      tail(op2, 1.0, {1.0, 1.0});
      ops().push_back(op2);
    } else if (m == 9) {  // Thm 3.1
      // MM1: U = B B; emits U (value and left operand) and X = B + 2U (right operand)
      Op op1 = mk_gemm(R, R);
      add_in(op1, R, REP_W);
      add_out(op1, SL_P1, REP_W | REP_OPA, 1.0, 0.0);
      add_out(op1, SL_RF0, REP_OPB, 2.0, 0.0).in[0] = 1.0;
      ops().push_back(op1);
      // MM2: V = U X; emits P = 3/20 B + 2U + V, Q = 11/40 B - 1/8 U + 1/4 V,
      //      C = B + 767/800 U + 15/32 V
      Op op2 = mk_gemm(SL_P1, SL_RF0);
      add_in(op2, R, REP_W);
      add_in(op2, SL_P1, REP_W);
      {
        OutSpec& P = add_out(op2, SL_LF1, REP_OPA, 1.0, 0.0);
        P.in[0] = 3.0 / 20.0;
        P.in[1] = 2.0;
        OutSpec& Q = add_out(op2, SL_RF1, REP_OPB, 0.25, 0.0);
        Q.in[0] = 11.0 / 40.0;
        Q.in[1] = -0.125;
        OutSpec& C = add_out(op2, SL_C, REP_W, 15.0 / 32.0, 0.0);
        C.in[0] = 1.0;
        C.in[1] = 767.0 / 800.0;
      }
      ops().push_back(op2);
      // MM3: W = P Q; G = W + C (T_9 = I + G)
      Op op3 = mk_gemm(SL_LF1, SL_RF1);
      add_in(op3, SL_C, REP_W);
      tail(op3, 1.0, {1.0});
      ops().push_back(op3);
    } else if (m == 15) {  // Sec. 4.1, eq. factors / radix15kernel
      const double* x = p->c15;
      const double *l2 = x, *r2 = x + 3, *l3 = x + 6, *r3 = x + 10, *l4 = x + 14, *r4 = x + 19, *g = x + 24;
      const bool via_c = p2_via_c(g, {l4[3], r4[3]});
      // P1 = B B; L2, R2 over (I, B, P1)
      Op op1 = mk_gemm(R, R);
      add_in(op1, R, REP_W);
      add_out(op1, SL_P1, REP_W, 1.0, 0.0);
      add_out(op1, SL_LF0, REP_OPA, l2[2], l2[0]).in[0] = l2[1];
      add_out(op1, SL_RF0, REP_OPB, r2[2], r2[0]).in[0] = r2[1];
      ops().push_back(op1);
      // P2 = L2 R2; L3, R3 over (I, B, P1, P2); C = g1 B + g2 P1 + g3 P2 (P2
      // itself is stored only when P3 cannot read its share from C)
      Op op2 = mk_gemm(SL_LF0, SL_RF0);
      add_in(op2, R, REP_W);
      add_in(op2, SL_P1, REP_W);
      if (!via_c) add_out(op2, SL_P2, REP_W, 1.0, 0.0);
      {
        OutSpec& L = add_out(op2, SL_LF1, REP_OPA, l3[3], l3[0]);
        L.in[0] = l3[1];
        L.in[1] = l3[2];
        OutSpec& Rr = add_out(op2, SL_RF1, REP_OPB, r3[3], r3[0]);
        Rr.in[0] = r3[1];
        Rr.in[1] = r3[2];
        OutSpec& C = add_out(op2, SL_C, REP_W, g[2], 0.0);
        C.in[0] = g[0];
        C.in[1] = g[1];
      }
      ops().push_back(op2);
      // P3 = L3 R3; L4, R4 over (I, B, P1, P2, P3); C += g4 P3
      Op op3 = mk_gemm(SL_LF1, SL_RF1);
      add_in(op3, R, REP_W);
      add_in(op3, SL_P1, REP_W);
      if (!via_c) add_in(op3, SL_P2, REP_W);
      add_in(op3, SL_C, REP_W);
      {
        comb3(add_out(op3, SL_LF0, REP_OPA, l4[4], l4[0]), via_c, g, l4[1], l4[2], l4[3]);
        comb3(add_out(op3, SL_RF0, REP_OPB, r4[4], r4[0]), via_c, g, r4[1], r4[2], r4[3]);
        add_out(op3, SL_C, REP_W, g[3], 0.0).in[via_c ? 2 : 3] = 1.0;
      }
      ops().push_back(op3);
      // P4 = L4 R4; G = C + P4 (T~15 = I + G)
      Op op4 = mk_gemm(SL_LF0, SL_RF0);
      add_in(op4, SL_C, REP_W);
      tail(op4, 1.0, {1.0});
      ops().push_back(op4);
    } else if (m == 24 || m == 25 || m == 27 || m == 31 || m == 33) {  // five-product circuit (App. C, Table approx)
      const double* x = p->cp5;
      const double *l2 = x, *r2 = x + 3, *l3 = x + 6, *r3 = x + 10, *l4 = x + 14, *r4 = x + 19;
      const double *l5 = x + 24, *r5 = x + 30, *g = x + 36;
      const bool fold = p->grouped;
      const bool via_c = fold ? p2_via_c(g, {l4[3], r4[3], l5[3], r5[3]}) : p2_via_c(g, {l4[3], r4[3]});
      // P1 = B B; L2, R2 over (I, B, P1)
      Op op1 = mk_gemm(R, R);
      add_in(op1, R, REP_W);
      add_out(op1, SL_P1, REP_W, 1.0, 0.0);
      add_out(op1, SL_LF0, REP_OPA, l2[2], l2[0]).in[0] = l2[1];
      add_out(op1, SL_RF0, REP_OPB, r2[2], r2[0]).in[0] = r2[1];
      ops().push_back(op1);
      // P2 = L2 R2; L3, R3 over (I, B, P1, P2); C = g1 B + g2 P1 + g3 P2. A
      // single plan's fourth product (or element-wise pass) reads P2; a grouped
      // batch's reads it only through C.
      Op op2 = mk_gemm(SL_LF0, SL_RF0);
      add_in(op2, R, REP_W);
      add_in(op2, SL_P1, REP_W);
      if (!(fold && via_c)) add_out(op2, SL_P2, REP_W, 1.0, 0.0);
      {
        OutSpec& L = add_out(op2, SL_LF1, REP_OPA, l3[3], l3[0]);
        L.in[0] = l3[1];
        L.in[1] = l3[2];
        OutSpec& Rr = add_out(op2, SL_RF1, REP_OPB, r3[3], r3[0]);
        Rr.in[0] = r3[1];
        Rr.in[1] = r3[2];
        OutSpec& C = add_out(op2, SL_C, REP_W, g[2], 0.0);
        C.in[0] = g[0];
        C.in[1] = g[1];
      }
      ops().push_back(op2);
      // P3 = L3 R3; L4, R4 over (I, B, P1, P2, P3); C += g4 P3. The parts of L5,
      // R5 over (I, B, P1, P2, P3) come from this epilogue in a grouped batch,
      // whose products are bound by their epilogues anyway. A single product's
      // epilogue with five outputs would no longer hide behind its main loop.
      // There, after P3, C = g1 B + g2 P1 + g3 P2 + g4 P3 holds P3's share, so
      //   sum_j l5_j X_j = l5_0 I + sum_{j=1..3} (l5_j - l5_4 g_j / g4) X_j + (l5_4 / g4) C
      // over X = (I, B, P1, P2, P3), and P4's epilogue forms L5 and R5 from
      // (B, P1, P2, C) and P4: P3 is not stored and no element-wise pass runs.
      // The substitution multiplies C's FP32 rounding by |l5_4 / g4| (6.8 at
      // most over radix 24-33); above 16, P3 is stored and a pass forms the parts.
      const bool subst = !fold && std::fabs(g[3]) > 0.0 && std::fabs(l5[4] / g[3]) <= kSubMax &&
                         std::fabs(r5[4] / g[3]) <= kSubMax;
      Op op3 = mk_gemm(SL_LF1, SL_RF1);
      add_in(op3, R, REP_W);
      add_in(op3, SL_P1, REP_W);
      if (!via_c) add_in(op3, SL_P2, REP_W);
      add_in(op3, SL_C, REP_W);
      {
        comb3(add_out(op3, SL_LF0, REP_OPA, l4[4], l4[0]), via_c, g, l4[1], l4[2], l4[3]);
        comb3(add_out(op3, SL_RF0, REP_OPB, r4[4], r4[0]), via_c, g, r4[1], r4[2], r4[3]);
        add_out(op3, SL_C, REP_W, g[3], 0.0).in[via_c ? 2 : 3] = 1.0;
        if (fold) {
          comb3(add_out(op3, SL_Q5L, REP_W, l5[4], l5[0]), via_c, g, l5[1], l5[2], l5[3]);
          comb3(add_out(op3, SL_Q5R, REP_W, r5[4], r5[0]), via_c, g, r5[1], r5[2], r5[3]);
        } else if (!subst) {
          add_out(op3, SL_P3, REP_W, 1.0, 0.0);
        }
      }
      ops().push_back(op3);
      if (subst) {
        // P4 = L4 R4; L5, R5 over (I, B, P1, P2, C) and P4; C += g5 P4
        Op op4 = mk_gemm(SL_LF0, SL_RF0);
        add_in(op4, R, REP_W);
        add_in(op4, SL_P1, REP_W);
        add_in(op4, SL_P2, REP_W);
        add_in(op4, SL_C, REP_W);
        for (int side = 0; side < 2; ++side) {
          const double* c5 = side ? r5 : l5;
          OutSpec& o = add_out(op4, side ? SL_RF1 : SL_LF1, side ? REP_OPB : REP_OPA, c5[5], c5[0]);
          const double t = c5[4] / g[3];
          for (int j = 0; j < 3; ++j) o.in[j] = c5[1 + j] - t * g[j];
          o.in[3] = t;
        }
        add_out(op4, SL_C, REP_W, g[4], 0.0).in[3] = 1.0;
        ops().push_back(op4);
        Op op5 = mk_gemm(SL_LF1, SL_RF1);
        add_in(op5, SL_C, REP_W);
        tail(op5, 1.0, {1.0});
        ops().push_back(op5);
        return;
      }
      if (!fold) {  // element-wise: the parts of L5, R5 over (I, B, P1, P2, P3)
        Op ew = mk_ewise();
        add_in(ew, R, REP_W);
        add_in(ew, SL_P1, REP_W);
        add_in(ew, SL_P2, REP_W);
        add_in(ew, SL_P3, REP_W);
        OutSpec& L = add_out(ew, SL_Q5L, REP_W, 0.0, l5[0]);
        OutSpec& Rr = add_out(ew, SL_Q5R, REP_W, 0.0, r5[0]);
        for (int j = 0; j < 4; ++j) {
          L.in[j] = l5[1 + j];
          Rr.in[j] = r5[1 + j];
        }
        ops().push_back(ew);
      }
      // P4 = L4 R4; L5 = Q5L + l5_P4 P4, R5 = Q5R + r5_P4 P4; C += g5 P4
      Op op4 = mk_gemm(SL_LF0, SL_RF0);
      add_in(op4, SL_Q5L, REP_W);
      add_in(op4, SL_Q5R, REP_W);
      add_in(op4, SL_C, REP_W);
      add_out(op4, SL_LF1, REP_OPA, l5[5], 0.0).in[0] = 1.0;
      add_out(op4, SL_RF1, REP_OPB, r5[5], 0.0).in[1] = 1.0;
      add_out(op4, SL_C, REP_W, g[4], 0.0).in[2] = 1.0;
      ops().push_back(op4);
      // P5 = L5 R5; G = C + P5 (T~ = I + G)
      Op op5 = mk_gemm(SL_LF1, SL_RF1);
      add_in(op5, SL_C, REP_W);
      tail(op5, 1.0, {1.0});
      ops().push_back(op5);
    }
  }

  void levels() {
    const std::vector<int>& lv = p->levels;
    const int L = (int)lv.size();
    int R = SL_R0, Rn = SL_R1, Y = SL_Y0, Yn = SL_Y1;
    {  // R_0 = A in every representation; A kept as left operand for the paper-form residual
      Op op = mk_ewise();
      add_in(op, SL_USER_A, 0);
      add_out(op, R, REP_ALL, 0.0, 0.0).in[0] = 1.0;
      if (paper) add_out(op, SL_A0, REP_OPA, 0.0, 0.0).in[0] = 1.0;
      ops().push_back(op);
    }
    bool y_is_I = true;
    const uint32_t yreps = REP_F64 | REP_OPA | (paper ? REP_OPB : 0u);
    for (int l = 0; l < L; ++l) {
      const int m = lv[l];
      const bool last = l == L - 1;
      const bool need_res = !last;
      const int ytarget = last ? SL_USER_S : Yn;
      const uint32_t yr = last ? 0u : yreps;
      int G = SL_G;
      if (m == 2) {
        G = R;  // f = 1 + z: G = R, no product (Sec. 5.5, Hensel)
      } else {
        uint32_t greps = 0;
        if (!y_is_I) greps |= REP_OPB;
        if (need_res && !paper) greps |= REP_OPB | REP_W;
        kernel(m, R, greps, y_is_I ? ytarget : SL_NONE, yr);
      }
      const bool fuse_first_y = y_is_I && m == 2 && need_res && !paper;
      if (!y_is_I) {  // concatenation Y <- Y + Y G
        Op op = mk_gemm(Y, G);
        add_in(op, Y, REP_F64);
        add_out(op, ytarget, yr, 1.0, 0.0).in[0] = 1.0;
        ops().push_back(op);
      } else if (m == 2 && !fuse_first_y) {  // Y_1 = I + R_0, element-wise
        Op op = mk_ewise();
        add_in(op, R, REP_F64);
        add_out(op, ytarget, yr, 0.0, 1.0).in[0] = 1.0;
        ops().push_back(op);
      }
      if (need_res) {
        if (paper) {  // R' = I - (I - A) Y' = I - Y' + A Y'
          Op op = mk_gemm(SL_A0, ytarget);
          add_in(op, ytarget, REP_F64);
          add_out(op, Rn, REP_ALL, 1.0, 1.0).in[0] = -1.0;
          ops().push_back(op);
        } else if (m == 2) {  // R' = R R
          Op op = mk_gemm(R, R);
          add_out(op, Rn, REP_ALL, 1.0, 0.0);
          if (fuse_first_y) {
            add_in(op, R, REP_F64);
            add_out(op, ytarget, yr, 0.0, 1.0).in[0] = 1.0;
          }
          ops().push_back(op);
        } else {  // R' = R + R G - G
          Op op = mk_gemm(R, G);
          add_in(op, R, REP_F64);
          add_in(op, G, REP_W);
          OutSpec& o = add_out(op, Rn, REP_ALL, 1.0, 0.0);
          o.in[0] = 1.0;
          o.in[1] = -1.0;
          ops().push_back(op);
        }
        int t = R;
        R = Rn;
        Rn = t;
      }
      if (!last) {
        int t = Y;
        Y = Yn;
        Yn = t;
      }
      y_is_I = false;
    }
  }

  // Horner-free naive chain (Sec. 2.1): S_2 = I + A, S_{i+1} = I + A S_i.
  void naive() {
    const int64_t k = p->k;
    if (k == 2) {
      Op op = mk_ewise();
      add_in(op, SL_USER_A, 0);
      add_out(op, SL_USER_S, 0, 0.0, 1.0).in[0] = 1.0;
      ops().push_back(op);
      return;
    }
    Op op = mk_ewise();
    add_in(op, SL_USER_A, 0);
    add_out(op, SL_R0, REP_OPA, 0.0, 0.0).in[0] = 1.0;
    add_out(op, SL_Y0, REP_OPB, 0.0, 1.0).in[0] = 1.0;
    ops().push_back(op);
    int cur = SL_Y0, nxt = SL_Y1;
    for (int64_t i = 3; i <= k; ++i) {
      Op g = mk_gemm(SL_R0, cur);
      add_out(g, i == k ? SL_USER_S : nxt, i == k ? 0u : REP_OPB, 1.0, 1.0);
      ops().push_back(g);
      int t = cur;
      cur = nxt;
      nxt = t;
    }
  }

  // Binary digits of k, most significant first (any k): doubling
  // S_{2n} = S_n + S_n A^n, A^{2n} = A^n A^n; digit 1: S_{n+1} = S_n + A^n, A^{n+1} = A^n A.
  void binary_digits() {
    const int64_t k = p->k;
    int nb = 0;
    while ((k >> (nb + 1)) != 0) ++nb;  // digits after the leading one
    {
      Op op = mk_ewise();
      add_in(op, SL_USER_A, 0);
      add_out(op, SL_R0, REP_ALL, 0.0, 0.0).in[0] = 1.0;
      add_out(op, SL_A0, REP_OPB, 0.0, 0.0).in[0] = 1.0;
      ops().push_back(op);
    }
    int P = SL_R0, Pn = SL_R1, S = SL_Y0, Sn = SL_Y1;
    bool s_is_I = true;
    const uint32_t sreps = REP_F64 | REP_OPA;
    size_t last_op = 0;
    int last_out = 0;
    for (int i = nb - 1; i >= 0; --i) {
      const bool b = (k >> i) & 1;
      const bool last = i == 0;
      if (s_is_I) {
        Op op = mk_ewise();
        add_in(op, P, REP_F64);
        add_out(op, Sn, sreps, 0.0, 1.0).in[0] = 1.0;
        last_op = ops().size();
        last_out = 0;
        ops().push_back(op);
      } else {
        Op op = mk_gemm(S, P);
        add_in(op, S, REP_F64);
        add_out(op, Sn, sreps, 1.0, 0.0).in[0] = 1.0;
        last_op = ops().size();
        last_out = 0;
        ops().push_back(op);
      }
      std::swap(S, Sn);
      s_is_I = false;
      if (!last || b) {
        Op op = mk_gemm(P, P);
        add_out(op, Pn, REP_ALL, 1.0, 0.0);
        if (b) {
          add_in(op, S, REP_F64);
          add_out(op, Sn, sreps, 1.0, 0.0).in[0] = 1.0;
          last_op = ops().size();
          last_out = 1;
        }
        ops().push_back(op);
        std::swap(P, Pn);
        if (b) std::swap(S, Sn);
      }
      if (b && !last) {
        Op op = mk_gemm(P, SL_A0);
        add_out(op, Pn, REP_ALL, 1.0, 0.0);
        ops().push_back(op);
        std::swap(P, Pn);
      }
    }
    OutSpec& o = ops()[last_op].out[last_out];
    o.slot = SL_USER_S;
    o.reps = 0;
  }

  void matmul() {
    std::vector<Op>& mm = p->mm_ops;
    Op a = mk_ewise();
    add_in(a, SL_USER_A, 0);
    add_out(a, SL_R0, REP_OPA, 0.0, 0.0).in[0] = 1.0;
    mm.push_back(a);
    Op b = mk_ewise();
    add_in(b, SL_USER_B, 0);
    add_out(b, SL_Y0, REP_OPB, 0.0, 0.0).in[0] = 1.0;
    mm.push_back(b);
    Op g = mk_gemm(SL_R0, SL_Y0);
    add_out(g, SL_USER_S, 0, 1.0, 0.0);
    mm.push_back(g);
  }
};

// ---------------------------------------------------------------- split-FP16 records

// Records of one op list: operands and inputs take the record of the op that
// last wrote their slot; every output of a workspace slot starts a new record.
bool assign_records(const std::vector<Op>& ops, int* next, std::vector<neumann_plan_s::OpSx>* out) {
  std::vector<int> cur(SL_N, -1);
  auto rec_of = [&](int slot) { return slot == SL_USER_A ? 0 : slot == SL_USER_B ? 1 : slot >= 0 ? cur[slot] : -1; };
  out->clear();
  for (const Op& op : ops) {
    neumann_plan_s::OpSx r;
    memset(&r, 0xff, sizeof(r));  // -1 everywhere
    if (op.kind == OP_GEMM) {
      r.rec_a = rec_of(op.a);
      r.rec_b = rec_of(op.b);
      if (r.rec_a < 0 || r.rec_b < 0) return false;
    }
    for (int i = 0; i < op.nin; ++i) {
      r.rec_in[i] = rec_of(op.in[i].slot);
      if (r.rec_in[i] < 0) return false;
    }
    for (int j = 0; j < op.nout; ++j) r.rec_out[j] = op.out[j].slot >= 0 ? (*next)++ : -1;
    if (op.kind == OP_GEMM) r.rec_acc = (*next)++;
    for (int j = 0; j < op.nout; ++j)
      if (op.out[j].slot >= 0) cur[op.out[j].slot] = r.rec_out[j];
    out->push_back(r);
  }
  return true;
}

bool build_records(neumann_plan_s* p) {
  p->sx = p->dtype == NEUMANN_SPLIT_FP16;
  if (!p->sx) return true;
  int next = 2;
  if (!assign_records(p->ops, &next, &p->op_sx) || !assign_records(p->mm_ops, &next, &p->mm_sx)) return false;
  p->sx_nrec = next;
  p->sx_nmat = p->grouped ? p->chunk : 1;
  p->sx_col.assign(next, -1);
  int64_t off = 0;  // accumulators keep column sums, npad per matrix
  for (const auto* v : {&p->op_sx, &p->mm_sx})
    for (const neumann_plan_s::OpSx& r : *v)
      if (r.rec_acc >= 0) {
        p->sx_col[r.rec_acc] = off;
        off += (int64_t)p->sx_nmat * p->npad;
      }
  return true;
}

// ---------------------------------------------------------------- resident kernel

constexpr int kResDefaultLimit = 48;  // largest resident order of an untuned plan

// The grouped plan's op program for the resident kernel: every workspace slot
// the ops touch becomes a shared-memory FP32 matrix, and the slots with an
// FP64 copy also get a shared-memory FP64 matrix. The largest order held is the
// largest multiple of 4 (<= 64) whose matrices and program fit the budget.
void build_resident(neumann_plan_s* p) {
  p->res_ops.clear();
  p->res_maxn = p->res_limit = p->res_nslots = p->res_nf64 = 0;
  if (!p->grouped || p->path == PATH_F64 || (p->flags & NEUMANN_FLAG_NO_RESIDENT)) return;
  bool used[SL_N] = {}, f64[SL_N] = {};
  for (const Op& op : p->ops) {
    if (op.kind == OP_GEMM) used[op.a] = used[op.b] = true;
    for (int i = 0; i < op.nin; ++i)
      if (op.in[i].slot >= 0) {
        used[op.in[i].slot] = true;
        f64[op.in[i].slot] |= op.in[i].rep == REP_F64;
      }
    for (int j = 0; j < op.nout; ++j)
      if (op.out[j].slot >= 0) {
        used[op.out[j].slot] = true;
        f64[op.out[j].slot] |= (op.out[j].reps & REP_F64) != 0;
      }
  }
  for (int s = 0; s < 16; ++s) p->res_slot_of[s] = p->res_f64_of[s] = -1;
  for (int s = 0; s < SL_N; ++s) {
    if (!used[s]) continue;
    p->res_slot_of[s] = p->res_nslots++;
    if (f64[s]) p->res_f64_of[p->res_slot_of[s]] = p->res_nf64++;
  }
  const int nops = (int)p->ops.size();
  int m = kResMaxN;
  while (m >= 16 && resident_smem(p->res_nslots, p->res_nf64, nops, m, p->path != PATH_F32) > (size_t)kResSmemBudget)
    m -= 4;
  if (m < 16) return;
  p->res_maxn = m;
  // untuned: up to 48. Measured on the damped Jacobi batch (k = 81, 1024 matrices
  // of one order), the resident launch beats the grouped one at every order up
  // to 48 for split-BF16 and FP32 (n = 16: 0.10 ms against 0.96); at 60 the
  // split-BF16 products no longer do. neumann_plan_autotune_batched tunes it.
  p->res_limit = m < kResDefaultLimit ? m : kResDefaultLimit;
  const bool io64 = p->dt_io == DT_F64;
  for (const Op& op : p->ops) {
    ResOp r;
    memset(&r, 0, sizeof(r));
    r.gemm = op.kind == OP_GEMM;
    r.a = r.gemm ? p->res_slot_of[op.a] : 0;
    r.b = r.gemm ? p->res_slot_of[op.b] : 0;
    r.nin = op.nin;
    bool in64[kMaxIn] = {};
    for (int i = 0; i < op.nin; ++i) {
      const InRef& x = op.in[i];
      r.in_slot[i] = x.slot == SL_USER_A ? -1 : p->res_slot_of[x.slot];
      r.in_f64[i] = x.slot >= 0 && x.rep == REP_F64;
      in64[i] = x.slot == SL_USER_A ? io64 : r.in_f64[i] != 0;
    }
    r.nout = op.nout;
    for (int j = 0; j < op.nout; ++j) {
      const OutSpec& o = op.out[j];
      const bool user = o.slot == SL_USER_S;
      r.out_slot[j] = user ? -1 : p->res_slot_of[o.slot];
      r.out_f32[j] = !user && (o.reps & (REP_W | REP_OPA | REP_OPB)) != 0;
      r.out_f64[j] = !user && (o.reps & REP_F64) != 0;
      bool f = (user && io64) || r.out_f64[j];
      for (int i = 0; i < op.nin; ++i) f |= o.in[i] != 0.0 && in64[i];
      r.f64[j] = f;
      r.acc_d[j] = o.acc;
      r.acc_f[j] = (float)o.acc;
      r.id_d[j] = o.id;
      r.id_f[j] = (float)o.id;
      for (int i = 0; i < kMaxIn; ++i) {
        r.in_d[j][i] = o.in[i];
        r.in_f[j][i] = (float)o.in[i];
      }
    }
    p->res_ops.push_back(r);
  }
}

// ---------------------------------------------------------------- layout

// sym: every matrix of the scheme is symmetric, so a product's right operand
// is read from its row-major pair (B^T = B).
void note_reps(neumann_plan_s* p, const std::vector<Op>& ops, bool sym = false) {
  for (const Op& op : ops) {
    if (op.kind == OP_GEMM) {
      p->reps[op.a] |= REP_OPA;
      p->reps[op.b] |= sym ? REP_OPA : REP_OPB;
    }
    for (int i = 0; i < op.nin; ++i)
      if (op.in[i].slot >= 0) p->reps[op.in[i].slot] |= op.in[i].rep;
    for (int j = 0; j < op.nout; ++j)
      if (op.out[j].slot >= 0) p->reps[op.out[j].slot] |= op.out[j].reps;
  }
}

void layout(neumann_plan_s* p) {
  // one matrix, or `chunk` stacked slabs in a grouped batched plan
  const size_t nn = (size_t)p->npad * (size_t)p->npad * (size_t)(p->grouped ? p->chunk : 1);
  size_t off = 256;  // device status word(s)
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  if (p->grouped) {
    const size_t c = (size_t)p->count;  // tables for every chunk of a full batch
    const size_t tiles_per = (size_t)(p->npad / 128) * (size_t)(p->npad / 128);  // per matrix, at most
    p->slab = (size_t)p->npad * (size_t)p->npad;
    p->off_matn = take(c * sizeof(int));
    p->off_atab = take(c * sizeof(void*));
    p->off_stab = take(c * sizeof(void*));
    p->off_tc = take(c * tiles_per * sizeof(int4));
    p->off_simt = take(c * tiles_per * sizeof(int4));
    p->off_ew = take(c * (size_t)(p->npad / 32) * (size_t)(p->npad / 32) * sizeof(int4));
  }
  if (p->res_maxn > 0) {
    p->off_res_ops = take(p->res_ops.size() * sizeof(ResOp));
    const size_t c = (size_t)p->count;
    p->off_res_matn = take(c * sizeof(int));
    p->off_res_atab = take(c * sizeof(void*));
    p->off_res_stab = take(c * sizeof(void*));
  }
  if (p->sym && p->path == PATH_TC) {
    const int t = (int)(p->npad / 256);
    p->nsym = t * (t + 1) / 2;
    p->off_sym = take((size_t)p->nsym * sizeof(int2));
  }
  if (p->sx) {  // one contiguous region, cleared before each pass
    const size_t per = (size_t)p->sx_nrec * (size_t)p->sx_nmat * 4;
    int64_t ncol = 0;
    for (int64_t o : p->sx_col) ncol += o >= 0;
    const size_t cols = (size_t)ncol * (size_t)p->sx_nmat * (size_t)p->npad * 4;
    p->off_sx = off;
    p->off_sx_amax = take(per);
    p->off_sx_colmax = take(per);
    p->off_sx_exp = take(per);
    p->off_sx_col = take(cols);
    p->sx_bytes = off - p->off_sx;
  }
  for (int s = 0; s < SL_N; ++s) {
    SlotBufs& b = p->bufs[s];
    b.w = b.f64 = b.a_hi = b.a_lo = b.b_hi = b.b_lo = NOBUF;
    const uint32_t r = p->reps[s];
    if (!r) continue;
    if (p->path == PATH_F64) {
      b.w = take(nn * 8);
    } else if (p->path == PATH_F32) {
      if (r & (REP_W | REP_OPA | REP_OPB)) b.w = take(nn * 4);
      if (r & REP_F64) b.f64 = take(nn * 8);
    } else {
      if (r & REP_W) b.w = take(nn * 4);
      if (r & REP_F64) b.f64 = take(nn * 8);
      if (r & REP_OPA) {
        b.a_hi = take(nn * 2);
        b.a_lo = take(nn * 2);
      }
      if (r & REP_OPB) {
        b.b_hi = take(nn * 2);
        b.b_lo = take(nn * 2);
      }
    }
  }
  p->ws_bytes = off;
}

int build(neumann_plan_s* p) {
  Sched sc{p, (p->flags & NEUMANN_FLAG_RESIDUAL_PAPER) != 0};
  p->ops.clear();
  p->mm_ops.clear();
  if (p->k == 1) {
    Op op = mk_ewise();
    add_out(op, SL_USER_S, 0, 0.0, 1.0);
    p->ops.push_back(op);
  } else if (p->radix == 1) {
    sc.naive();
  } else if (p->radix == 2 && (p->k & (p->k - 1)) != 0) {
    sc.binary_digits();
  } else {
    sc.levels();
  }
  sc.matmul();
  // Right operands come from row-major pairs: read MN-major (bmn), or, in a
  // symmetric plan's scheme, read as their own transpose.
  auto row_major_b = [](std::vector<Op>& ops) {
    for (Op& op : ops)
      for (int j = 0; j < op.nout; ++j)
        if (op.out[j].reps & REP_OPB) op.out[j].reps = (op.out[j].reps & ~REP_OPB) | REP_OPA;
  };
  if (p->sym || p->bmn) row_major_b(p->ops);
  if (p->bmn) row_major_b(p->mm_ops);
  if (!build_records(p)) return NEUMANN_ENOTSUP;
  build_resident(p);
  memset(p->reps, 0, sizeof(p->reps));
  note_reps(p, p->ops, p->sym || p->bmn);
  note_reps(p, p->mm_ops, p->bmn);
  layout(p);
  return NEUMANN_OK;
}

// Radix 0 with NEUMANN_FLAG_ALLOW_APPROX: the levels of least product count
// sum_i (mu_{m_i} + 2) (Sec. 2.2 cost model) with prod_i m_i = k, over the
// exact kernels 2, 3, 5, 9 and the approximate radix-15 kernel; among equal
// counts, fewer approximate levels, then fewer levels. Block concatenation
// (Sec. 2.2) and Lemma 5.7 (Sec. 5.3) hold level by level, so any order is
// valid; the exact levels run first (9, 5, 3, 2) and the radix-15 levels last,
// where the residual they act on is a power of A of small norm, far inside
// the kernel's convergence region. k = 2^a 3^b 5^c only (else false).
bool mixed_levels(int64_t k, std::vector<int>* levels) {
  int e[3] = {0, 0, 0};
  int64_t q = k;
  const int prime[3] = {2, 3, 5};
  for (int i = 0; i < 3; ++i)
    while (q % prime[i] == 0) {
      q /= prime[i];
      ++e[i];
    }
  if (q != 1 || k < 1) return false;
  struct Factor {
    int m, d2, d3, d5, approx;
  };
  const Factor fac[5] = {{2, 1, 0, 0, 0}, {3, 0, 1, 0, 0}, {5, 0, 0, 1, 0}, {9, 0, 2, 0, 0}, {15, 0, 1, 1, 1}};
  // cost (products, approximate levels, levels) of the best split of 2^a 3^b 5^c
  typedef std::tuple<int, int, int> Cost;
  const int A = e[0] + 1, B = e[1] + 1, Cc = e[2] + 1;
  std::vector<Cost> best((size_t)A * B * Cc, Cost(1 << 30, 0, 0));
  std::vector<int> pick((size_t)A * B * Cc, -1);
  auto at = [&](int a, int b, int c) { return ((size_t)a * B + b) * Cc + c; };
  best[at(0, 0, 0)] = Cost(0, 0, 0);
  for (int a = 0; a < A; ++a)
    for (int b = 0; b < B; ++b)
      for (int c = 0; c < Cc; ++c) {
        if (a + b + c == 0) continue;
        for (int f = 0; f < 5; ++f) {
          const Factor& x = fac[f];
          if (a < x.d2 || b < x.d3 || c < x.d5) continue;
          const Cost& prev = best[at(a - x.d2, b - x.d3, c - x.d5)];
          if (std::get<0>(prev) >= (1 << 30)) continue;
          const Cost cand(std::get<0>(prev) + mu_of(x.m) + 2, std::get<1>(prev) + x.approx, std::get<2>(prev) + 1);
          if (cand < best[at(a, b, c)]) {
            best[at(a, b, c)] = cand;
            pick[at(a, b, c)] = f;
          }
        }
      }
  std::vector<int> ms;
  for (int a = e[0], b = e[1], c = e[2]; a + b + c > 0;) {
    const Factor& x = fac[pick[at(a, b, c)]];
    ms.push_back(x.m);
    a -= x.d2;
    b -= x.d3;
    c -= x.d5;
  }
  levels->clear();
  for (int m : {9, 5, 3, 2, 15})
    for (int x : ms)
      if (x == m) levels->push_back(m);
  return true;
}

int validate_and_levels(neumann_plan_s* p) {
  const int64_t k = p->k;
  p->levels.clear();
  switch (p->radix) {
    case 1:
      p->formula = k - 1;
      return NEUMANN_OK;
    case 2: {
      const bool pow2 = (k & (k - 1)) == 0;
      if (!pow2 && !(p->flags & NEUMANN_FLAG_EXACT_K)) return NEUMANN_EINVAL;
      int c = 0;
      while ((int64_t(1) << c) < k) ++c;
      p->formula = 2 * c;  // Sec. 6: 2 ceil(log2 k)
      if (pow2) pure_power(k, 2, &p->levels);
      return NEUMANN_OK;
    }
    case 3:
    case 5:
    case 9:
    case 15:
    case 24:
    case 25:
    case 27:
    case 31:
    case 33:
      if (!pure_power(k, p->radix, &p->levels)) return NEUMANN_EINVAL;
      break;
    case 0: {
      if (p->flags & NEUMANN_FLAG_ALLOW_APPROX) {
        if (!mixed_levels(k, &p->levels)) return NEUMANN_EINVAL;
        break;
      }
      int64_t q = k;
      for (int m : {9, 5, 3, 2}) {
        while (q % m == 0) {
          p->levels.push_back(m);
          q /= m;
        }
      }
      if (q != 1) return NEUMANN_EINVAL;
      break;
    }
    default:
      return NEUMANN_EINVAL;
  }
  if ((int)p->levels.size() > NEUMANN_MAX_LEVELS) return NEUMANN_EINVAL;
  p->formula = 0;
  for (int m : p->levels) p->formula += mu_of(m) + 2;  // Sec. 2.2: C(m) = mu_m + 2
  return NEUMANN_OK;
}

int init_plan(neumann_plan_s* p, int64_t n, int64_t k, int radix, int dtype, uint32_t flags) {
  if (n < 1 || k < 1 || n > (int64_t(1) << 20)) return NEUMANN_EINVAL;
  if (dtype < NEUMANN_FP64 || dtype > NEUMANN_SPLIT_FP16) return NEUMANN_EINVAL;
  p->n = n;
  p->k = k;
  p->radix = radix;
  p->dtype = dtype;
  p->flags = flags;
  p->npad = (n + 255) / 256 * 256;
  p->path = dtype == NEUMANN_FP64 ? PATH_F64 : dtype == NEUMANN_FP32 ? PATH_F32 : PATH_TC;
  p->dt_io = (dtype == NEUMANN_FP32 || (p->path == PATH_TC && (flags & NEUMANN_FLAG_IO_FP32))) ? DT_F32 : DT_F64;
  if ((flags & NEUMANN_FLAG_SYMMETRIC) && (flags & NEUMANN_FLAG_PRECISE_ACC)) return NEUMANN_ENOTSUP;
  p->sym = (flags & NEUMANN_FLAG_SYMMETRIC) != 0;
  p->bmn = p->path == PATH_TC && kMnMajorB;
  int rc = validate_and_levels(p);
  if (rc) return rc;
  if (radix == 15 || radix == 0) {
    double e, s15, s16;
    if (!radix15_coefficients((flags & NEUMANN_FLAG_PRINTED_COEFFS) ? 1 : 0, p->c15, &e, &s15, &s16))
      return NEUMANN_ENOTSUP;
  }
  if (mu_of(radix) == 5) {
    double e, sp;
    if (!radix_p5_coefficients(radix, p->cp5, &e, &sp)) return NEUMANN_ENOTSUP;
  }
  return build(p);
}

// ---------------------------------------------------------------- execution

size_t elem_bytes(int dt) { return dt == DT_F64 ? 8 : 4; }

struct UserPtrs {
  const void* A;
  int64_t lda;
  const void* B;
  void* S;
  int64_t lds;
};

EpiIn resolve_in(const neumann_plan_s* p, const InRef& r, const UserPtrs& u) {
  EpiIn e;
  e.mode = EPI_WS;
  if (r.slot == SL_USER_A) {
    e.p = p->grouped ? p->cur_atab : u.A;
    e.ld = u.lda;
    e.dt = p->dt_io;
    e.mode = p->grouped ? EPI_TABLE : EPI_PTR;
  } else if (r.slot == SL_USER_B) {
    e.p = u.B;
    e.ld = p->n;
    e.dt = p->dt_io;
    e.mode = EPI_PTR;
  } else {
    const SlotBufs& b = p->bufs[r.slot];
    e.ld = p->npad;
    if (p->path == PATH_F64) {
      e.p = p->ws + b.w;
      e.dt = DT_F64;
    } else if (r.rep == REP_F64) {
      e.p = p->ws + b.f64;
      e.dt = DT_F64;
    } else {
      e.p = p->ws + b.w;
      e.dt = DT_F32;
    }
  }
  return e;
}

EpiOut resolve_out(const neumann_plan_s* p, const OutSpec& s, const EpiIn* ins, int nin, const UserPtrs& u) {
  EpiOut o;
  memset(&o, 0, sizeof(o));
  o.acc_d = s.acc;
  o.id_d = s.id;
  o.acc_f = (float)s.acc;
  o.id_f = (float)s.id;
  for (int i = 0; i < kMaxIn; ++i) {
    o.in_d[i] = s.in[i];
    o.in_f[i] = (float)s.in[i];
  }
  auto dst = [&](void* ptr, int64_t ld, int dt, int mode) { o.dst[o.ndst++] = EpiDst{ptr, ld, dt, mode}; };
  auto split = [&](size_t hi, size_t lo, int tr) {
    o.split[o.nsplit++] = EpiSplit{p->ws + hi, p->ws + lo, p->npad, tr};
  };
  if (s.slot == SL_USER_S) {
    if (p->grouped)
      dst(const_cast<void*>(p->cur_stab), 0, p->dt_io, EPI_TABLE);
    else
      dst(u.S, u.lds, p->dt_io, EPI_PTR);
  } else {
    const SlotBufs& b = p->bufs[s.slot];
    if (p->path == PATH_F64) {
      dst(p->ws + b.w, p->npad, DT_F64, EPI_WS);
    } else if (p->path == PATH_F32) {
      if (s.reps & (REP_W | REP_OPA | REP_OPB)) dst(p->ws + b.w, p->npad, DT_F32, EPI_WS);
      if (s.reps & REP_F64) dst(p->ws + b.f64, p->npad, DT_F64, EPI_WS);
    } else {
      if (s.reps & REP_W) dst(p->ws + b.w, p->npad, DT_F32, EPI_WS);
      if (s.reps & REP_F64) dst(p->ws + b.f64, p->npad, DT_F64, EPI_WS);
      if (s.reps & REP_OPA) split(b.a_hi, b.a_lo, 0);
      if (s.reps & REP_OPB) split(b.b_hi, b.b_lo, 1);
    }
  }
  bool f64 = p->path == PATH_F64;
  for (int d = 0; d < o.ndst; ++d) f64 |= o.dst[d].dt == DT_F64;
  for (int i = 0; i < nin; ++i) f64 |= (s.in[i] != 0.0 && ins[i].dt == DT_F64);
  o.f64 = f64;
  return o;
}

// sx: the op's split-FP16 records (nullptr for other dtypes).
void make_params(const neumann_plan_s* p, const Op& op, const UserPtrs& u, EpiParams* P,
                 const neumann_plan_s::OpSx* sx = nullptr) {
  memset(P, 0, sizeof(*P));
  if (sx) {
    SxParams& q = P->sx;
    q.active = 1;
    q.nmat = p->sx_nmat;
    q.npad = (int)p->npad;
    q.exp = reinterpret_cast<int*>(p->ws + p->off_sx_exp);
    q.rec_a = sx->rec_a;
    q.rec_b = sx->rec_b;
    for (int j = 0; j < kMaxOut; ++j) q.rec_out[j] = j < op.nout ? sx->rec_out[j] : -1;
    if (sx->rec_acc >= 0) {
      q.acc_amax = reinterpret_cast<unsigned*>(p->ws + p->off_sx_amax) + (size_t)sx->rec_acc * p->sx_nmat;
      q.acc_col = reinterpret_cast<float*>(p->ws + p->off_sx_col) + p->sx_col[sx->rec_acc];
    }
  }
  P->n = (int)p->n;
  P->npad = (int)p->npad;
  P->status = reinterpret_cast<unsigned*>(p->ws);
  P->fp16 = p->dtype == NEUMANN_SPLIT_FP16;
  if (p->grouped) {
    P->mat_n = p->cur_matn;
    P->mat_stride = (int64_t)p->slab;
  }
  P->nin = op.nin;
  for (int i = 0; i < op.nin; ++i) P->in[i] = resolve_in(p, op.in[i], u);
  P->nout = op.nout;
  for (int j = 0; j < op.nout; ++j) P->out[j] = resolve_out(p, op.out[j], P->in, op.nin, u);
  // the tensor-core epilogue's lean path handles at most one FP64 input
  int nf64 = 0;
  P->f64_in = -1;
  P->nf32 = 0;
  for (int i = 0; i < op.nin; ++i) {
    if (P->in[i].dt == DT_F64) {
      ++nf64;
      P->f64_in = i;
    } else {
      P->f32_idx[P->nf32++] = i;
    }
  }
  P->fast = nf64 <= 1;
  P->edge_ok = 1;
  for (int i = 0; i < op.nin; ++i) P->edge_ok &= P->in[i].mode == EPI_WS;
}

// Algorithmic device-memory bytes of one op per matrix element: each input
// and each output representation read or written once, plus the two operands
// of a product (hi/lo pairs on the tensor-core path). Mirrors resolve_in /
// resolve_out.
int64_t op_bytes(const neumann_plan_s* p, const Op& op) {
  const int64_t io = elem_bytes(p->dt_io);
  const int64_t w = p->path == PATH_F64 ? 8 : 4;
  int64_t b = 0;
  for (int i = 0; i < op.nin; ++i) {
    const InRef& r = op.in[i];
    b += r.slot == SL_USER_A || r.slot == SL_USER_B ? io : (r.rep & REP_F64) ? 8 : w;
  }
  for (int j = 0; j < op.nout; ++j) {
    const OutSpec& o = op.out[j];
    if (o.slot == SL_USER_S) {
      b += io;
    } else if (p->path == PATH_F64) {
      b += 8;
    } else if (p->path == PATH_F32) {
      b += ((o.reps & (REP_W | REP_OPA | REP_OPB)) ? 4 : 0) + ((o.reps & REP_F64) ? 8 : 0);
    } else {
      b += ((o.reps & REP_W) ? 4 : 0) + ((o.reps & REP_F64) ? 8 : 0) + ((o.reps & REP_OPA) ? 4 : 0) +
           ((o.reps & REP_OPB) ? 4 : 0);
    }
  }
  if (op.kind == OP_GEMM) b += p->path == PATH_TC ? 8 : 2 * w;
  return b;
}

// sym: the ops are the scheme's products of a symmetric plan (right operands
// read from their row-major pairs, only the tiles on or above the diagonal).
bool build_maps(neumann_plan_s* p, const std::vector<Op>& ops, std::vector<TcMaps>* maps, bool sym = false) {
  maps->assign(ops.size(), TcMaps());
  const bool row_b = sym || p->bmn;  // B from its row-major pair
  for (size_t i = 0; i < ops.size(); ++i) {
    const Op& op = ops[i];
    if (op.kind != OP_GEMM) continue;
    const SlotBufs& a = p->bufs[op.a];
    const SlotBufs& b = p->bufs[op.b];
    const size_t bhi = row_b ? b.a_hi : b.b_hi, blo = row_b ? b.a_lo : b.b_lo;
    if (!tc_make_maps(&(*maps)[i], p->ws + a.a_hi, p->ws + a.a_lo, p->ws + bhi, p->ws + blo, p->npad, p->npad,
                      p->grouped ? p->chunk : 0, p->dtype == NEUMANN_SPLIT_FP16,
                      sym ? 1 : (p->flags & NEUMANN_FLAG_SINGLE_CTA) ? 0 : p->tune_pair, p->tune_group,
                      (p->flags & NEUMANN_FLAG_PRECISE_ACC) != 0, p->bmn && !sym))
      return false;
    if (sym) {
      (*maps)[i].sym = reinterpret_cast<const int2*>(p->ws + p->off_sym);
      (*maps)[i].nsym = p->nsym;
    }
  }
  return true;
}

// The tiles on or above the diagonal of a symmetric product, in groups of 8
// tile rows; within a group column by column, so that neighbouring clusters
// share panels in L2.
std::vector<int2> sym_tiles(int t) {
  std::vector<int2> v;
  v.reserve((size_t)t * (t + 1) / 2);
  for (int g0 = 0; g0 < t; g0 += kDefaultRasterGroup) {
    const int g1 = std::min(t, g0 + kDefaultRasterGroup);
    for (int tn = g0; tn < t; ++tn)
      for (int tm = g0; tm < g1 && tm <= tn; ++tm) v.push_back(make_int2(tm, tn));
  }
  return v;
}

int attach(neumann_plan_s* p, void* ws) {
  p->ws = reinterpret_cast<char*>(ws);
  p->maps_ready = false;
  if (p->sym && p->path == PATH_TC) {
    const std::vector<int2> t = sym_tiles((int)(p->npad / 256));
    if (cudaMemcpy(p->ws + p->off_sym, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
      return NEUMANN_ECUDA;
  }
  if (p->path == PATH_TC) {
    if (!build_maps(p, p->ops, &p->maps, p->sym) || !build_maps(p, p->mm_ops, &p->mm_maps)) return NEUMANN_ECUDA;
  }
  if (p->res_maxn > 0 && cudaMemcpy(p->ws + p->off_res_ops, p->res_ops.data(), p->res_ops.size() * sizeof(ResOp),
                                     cudaMemcpyHostToDevice) != cudaSuccess)
    return NEUMANN_ECUDA;
  p->maps_ready = true;
  return NEUMANN_OK;
}

int ensure_workspace(neumann_plan_s* p, cudaStream_t s) {
  if (p->ws) return NEUMANN_OK;
  void* ws = nullptr;
  if (cudaMalloc(&ws, p->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    return NEUMANN_ENOMEM;
  }
  if (cudaMemsetAsync(ws, 0, 256, s) != cudaSuccess) {
    cudaFree(ws);
    return NEUMANN_ECUDA;
  }
  p->ws_owned = true;
  int rc = attach(p, ws);
  if (rc) {
    cudaFree(ws);
    p->ws = nullptr;
    p->ws_owned = false;
  }
  return rc;
}

// The split-FP16 scale step before op i of `ops`: op i's records and
// coefficients, and, when op i-1 is a product, what finalises its outputs.
SxScaleOp sx_scale_op(const neumann_plan_s* p, const std::vector<Op>& ops,
                      const std::vector<neumann_plan_s::OpSx>& rs, size_t i) {
  SxScaleOp q;
  memset(&q, 0, sizeof(q));
  q.nmat = p->sx_nmat;
  q.npad = (int)p->npad;
  q.amax = reinterpret_cast<unsigned*>(p->ws + p->off_sx_amax);
  q.colmax = reinterpret_cast<float*>(p->ws + p->off_sx_colmax);
  q.exp = reinterpret_cast<int*>(p->ws + p->off_sx_exp);
  q.col = reinterpret_cast<float*>(p->ws + p->off_sx_col);
  const Op& op = ops[i];
  const neumann_plan_s::OpSx& r = rs[i];
  q.rec_a = r.rec_a;
  q.rec_b = r.rec_b;
  q.nin = op.nin;
  for (int k = 0; k < op.nin; ++k) q.rec_in[k] = r.rec_in[k];
  q.nout = op.nout;
  for (int j = 0; j < op.nout; ++j) {
    const OutSpec& o = op.out[j];
    q.rec_out[j] = r.rec_out[j];
    q.acc[j] = op.kind == OP_GEMM ? (float)o.acc : 0.f;
    q.id[j] = (float)o.id;
    for (int k = 0; k < kMaxIn; ++k) q.in[j][k] = (float)o.in[k];
  }
  q.prev_acc = -1;
  if (i > 0 && ops[i - 1].kind == OP_GEMM) {
    const Op& pv = ops[i - 1];
    const neumann_plan_s::OpSx& pr = rs[i - 1];
    q.prev_acc = pr.rec_acc;
    q.prev_col = p->sx_col[pr.rec_acc];
    q.prev_nin = pv.nin;
    for (int k = 0; k < pv.nin; ++k) q.prev_in[k] = pr.rec_in[k];
    q.prev_nout = pv.nout;
    for (int j = 0; j < pv.nout; ++j) {
      const OutSpec& o = pv.out[j];
      q.prev_out[j] = pr.rec_out[j];
      q.prev_a[j] = (float)o.acc;
      q.prev_id[j] = (float)o.id;
      for (int k = 0; k < kMaxIn; ++k) q.prev_c[j][k] = (float)o.in[k];
    }
  }
  return q;
}

// Split-FP16: clear the stats region of this pass and measure the caller's
// matrices that the ops read (records 0 and 1).
int sx_begin(neumann_plan_s* p, const std::vector<Op>& ops, const UserPtrs& u, int count, cudaStream_t s) {
  if (cudaMemsetAsync(p->ws + p->off_sx, 0, p->sx_bytes, s) != cudaSuccess) return NEUMANN_ECUDA;
  bool need[2] = {false, false};
  for (const Op& op : ops)
    for (int i = 0; i < op.nin; ++i) {
      need[0] |= op.in[i].slot == SL_USER_A;
      need[1] |= op.in[i].slot == SL_USER_B;
    }
  for (int r = 0; r < 2; ++r) {
    if (!need[r]) continue;
    const EpiIn in = resolve_in(p, InRef{r == 0 ? SL_USER_A : SL_USER_B, 0}, u);
    unsigned* amax = reinterpret_cast<unsigned*>(p->ws + p->off_sx_amax) + (size_t)r * p->sx_nmat;
    unsigned* colmax = reinterpret_cast<unsigned*>(p->ws + p->off_sx_colmax) + (size_t)r * p->sx_nmat;
    if (launch_sx_input_stats(in, p->grouped ? p->cur_matn : nullptr, (int)p->n, count, amax, colmax, s) !=
        cudaSuccess)
      return NEUMANN_ECUDA;
  }
  return NEUMANN_OK;
}

int run_ops(neumann_plan_s* p, const std::vector<Op>& ops, const std::vector<TcMaps>& maps, const UserPtrs& u,
            cudaStream_t s, bool timing) {
  EpiParams P;
  int gi = p->timed;  // timing accumulates over evaluations until neumann_plan_timing reads it
  if (timing) {  // events recorded into a CUDA graph capture cannot be timed: no record then
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return NEUMANN_ECUDA;
    timing = cs == cudaStreamCaptureStatusNone;
  }
  if (timing) {
    int ng = 0;
    for (const Op& op : ops) ng += op.kind == OP_GEMM;
    if (p->timed + ng > kMaxTimedProducts) return NEUMANN_EINVAL;
    while ((int)p->events.size() < 2 * (p->timed + ng)) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return NEUMANN_ECUDA;
      p->events.push_back(e);
    }
  }
  // the last op reading the caller's A and the first writing the caller's S
  int a_last = -1, s_first = -1;
  if (p->hook_after_a || p->hook_before_s) {
    for (int i = 0; i < (int)ops.size(); ++i) {
      for (int j = 0; j < ops[i].nin; ++j)
        if (ops[i].in[j].slot == SL_USER_A) a_last = i;
      for (int j = 0; j < ops[i].nout; ++j)
        if (ops[i].out[j].slot == SL_USER_S && s_first < 0) s_first = i;
    }
  }
  // split-FP16: matrices of this pass, and the op list's records
  const int sx_count = p->grouped ? p->cur_count : 1;
  const std::vector<neumann_plan_s::OpSx>* sxr = !p->sx ? nullptr : &ops == &p->ops ? &p->op_sx : &p->mm_sx;
  if (sxr) {
    const int rc = sx_begin(p, ops, u, sx_count, s);
    if (rc) return rc;
  }
  for (size_t i = 0; i < ops.size(); ++i) {
    const Op& op = ops[i];
    make_params(p, op, u, &P, sxr ? &(*sxr)[i] : nullptr);
    if (sxr && launch_sx_scale(sx_scale_op(p, ops, *sxr, i), sx_count, s) != cudaSuccess) return NEUMANN_ECUDA;
    if (p->hook_before_s && (int)i == s_first && cudaStreamWaitEvent(s, p->hook_before_s, 0) != cudaSuccess)
      return NEUMANN_ECUDA;
    cudaError_t err;
    const int4* ew = p->grouped ? p->cur_ew : nullptr;
    const int4* st = p->grouped ? p->cur_simt : nullptr;
    const int4* tt = p->grouped ? p->cur_tc : nullptr;
    if (op.kind == OP_EWISE) {
      err = launch_ewise(P, s, ew, p->n_ew);
    } else {
      if (timing) cudaEventRecord(p->events[2 * gi], s);
      // the scheme's products of a symmetric plan (not the general product call)
      const bool sym = p->sym && &ops == &p->ops;
      if (p->path == PATH_F64) {
        err = launch_simt_gemm_f64(reinterpret_cast<const double*>(p->ws + p->bufs[op.a].w),
                                   reinterpret_cast<const double*>(p->ws + p->bufs[op.b].w), p->npad, p->npad, st,
                                   p->n_simt, P, s, sym);
      } else if (p->path == PATH_F32) {
        err = launch_simt_gemm_f32(reinterpret_cast<const float*>(p->ws + p->bufs[op.a].w),
                                   reinterpret_cast<const float*>(p->ws + p->bufs[op.b].w), p->npad, p->npad, st,
                                   p->n_simt, P, s, sym);
      } else {
        err = launch_tc_gemm(maps[i], p->npad, P, s, tt, p->n_tc);
      }
      if (timing) cudaEventRecord(p->events[2 * gi + 1], s);
      ++gi;
    }
    if (err != cudaSuccess) return NEUMANN_ECUDA;
    if (p->hook_after_a && (int)i == a_last && cudaEventRecord(p->hook_after_a, s) != cudaSuccess)
      return NEUMANN_ECUDA;
  }
  if (timing) p->timed = gi;
  return NEUMANN_OK;
}

bool overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* x = reinterpret_cast<const char*>(a);
  const char* y = reinterpret_cast<const char*>(b);
  return x < y + bbytes && y < x + abytes;
}

int eval_one(neumann_plan_s* p, const void* A, int64_t lda, void* S, int64_t lds, cudaStream_t s) {
  if (!A || !S || lda < p->n || lds < p->n) return NEUMANN_EINVAL;
  const size_t es = elem_bytes(p->dt_io);
  const size_t ab = ((size_t)(p->n - 1) * (size_t)lda + (size_t)p->n) * es;
  const size_t sb = ((size_t)(p->n - 1) * (size_t)lds + (size_t)p->n) * es;
  if (overlap(A, ab, S, sb)) return NEUMANN_EINVAL;
  int rc = ensure_workspace(p, s);
  if (rc) return rc;
  p->last_stream = s;
  UserPtrs u{A, lda, nullptr, S, lds};
  return run_ops(p, p->ops, p->maps, u, s, (p->flags & NEUMANN_FLAG_TIMING) != 0);
}

// True if some S_i overlaps some A_j (n x n with leading dimension n): one
// sweep over the intervals sorted by start address.
bool batch_aliases(int count, const int64_t* n, const void* const* A, void* const* S, size_t es) {
  struct Iv {
    uintptr_t lo, hi;
    bool s;
  };
  std::vector<Iv> iv;
  iv.reserve(2 * (size_t)count);
  for (int i = 0; i < count; ++i) {
    const uintptr_t b = (uintptr_t)n[i] * (uintptr_t)n[i] * es;
    iv.push_back(Iv{(uintptr_t)A[i], (uintptr_t)A[i] + b, false});
    iv.push_back(Iv{(uintptr_t)S[i], (uintptr_t)S[i] + b, true});
  }
  std::sort(iv.begin(), iv.end(), [](const Iv& a, const Iv& b) { return a.lo < b.lo; });
  uintptr_t end_a = 0, end_s = 0;
  for (const Iv& x : iv) {
    if (x.s ? x.lo < end_a : x.lo < end_s) return true;
    if (x.s)
      end_s = end_s > x.hi ? end_s : x.hi;
    else
      end_a = end_a > x.hi ? end_a : x.hi;
  }
  return false;
}

// Grouped batched evaluation. Matrices run in decreasing order (the longest
// work first, for the persistent product kernel), `chunk` at a time. The host
// builds, for the whole batch, the order table, the caller-pointer tables and
// the tile tables of every chunk, copies them into the workspace from pinned
// memory (skipped when orders and pointers repeat the previous call), and then
// runs the plan's operations once per chunk.
int eval_grouped(neumann_plan_s* p, int count, const int64_t* n, const void* const* A, void* const* S,
                 cudaStream_t s) {
  const int ck = p->chunk_run > 0 ? p->chunk_run : p->chunk;  // matrices per pass
  const bool same = (int)p->last_n.size() == count && ck == p->last_chunk_run && p->res_limit == p->last_res_limit &&
                    std::equal(n, n + count, p->last_n.begin()) && std::equal(A, A + count, p->last_a.begin()) &&
                    std::equal(S, S + count, p->last_s.begin());
  if (!same) {
    if (batch_aliases(count, n, A, S, elem_bytes(p->dt_io))) return NEUMANN_EINVAL;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    // the smallest orders (the end of `order`) run in the resident launch
    int ng = count;
    while (ng > 0 && n[order[ng - 1]] <= p->res_limit) --ng;
    const int nres = count - ng;
    // size classes of the resident matrices (largest first): orders above 32, 17..32, 1..16
    p->res_class.clear();
    for (int lo : {32, 16, 0}) {
      int first = -1, cnt = 0, top = 0;
      for (int k = 0; k < nres; ++k) {
        const int nk = (int)n[order[ng + k]];
        if (nk > lo && (lo == 32 || nk <= (lo == 16 ? 32 : 16))) {
          if (first < 0) first = k;
          ++cnt;
          top = nk > top ? nk : top;
        }
      }
      if (cnt) p->res_class.push_back(make_int3(first, cnt, (top + 3) & ~3));
    }
    std::vector<int> matn(count);
    std::vector<const void*> atab(count);
    std::vector<void*> stab(count);
    std::vector<int4> tc, simt, ew;
    const int kbk = simt_bk(p->path == PATH_F64);  // K depth of a SIMT stage
    p->chunks.clear();
    for (int k = 0; k < nres; ++k) {  // resident tables after the grouped ones' entries
      const int i = order[ng + k];
      matn[ng + k] = (int)n[i];
      atab[ng + k] = A[i];
      stab[ng + k] = S[i];
    }
    p->res_count = nres;
    for (int c0 = 0; c0 < ng; c0 += ck) {
      const int cn = ng - c0 < ck ? ng - c0 : ck;
      neumann_plan_s::Chunk ch{c0, cn, (int)tc.size(), 0, (int)simt.size(), 0, (int)ew.size(), 0};
      for (int j = 0; j < cn; ++j) {
        const int i = order[c0 + j];
        const int ni = (int)n[i];
        matn[c0 + j] = ni;
        atab[c0 + j] = A[i];
        stab[c0 + j] = S[i];
        const int mt = (ni + 127) / 128;  // 128-row tiles
        for (int tm = 0; tm < mt; ++tm) tc.push_back(make_int4(j, tm, (ni + 31) / 32, 0));
        for (int tm = 0; tm < mt; ++tm)
          for (int tn = 0; tn < mt; ++tn) simt.push_back(make_int4(j, tm, tn, (ni + kbk - 1) / kbk));
        // element-wise passes, like the products, write rows and columns below the
        // order rounded up to 32: the K padding every later product reads
        for (int tr = 0; tr < (ni + 31) / 32; ++tr)
          for (int tcol = 0; tcol < (ni + 31) / 32; ++tcol) ew.push_back(make_int4(j, tr, tcol, 0));
      }
      ch.ntc = (int)tc.size() - ch.tc0;
      ch.nsimt = (int)simt.size() - ch.simt0;
      ch.new_ = (int)ew.size() - ch.ew0;
      p->chunks.push_back(ch);
    }
    // pinned host image: [matn | atab | stab | tc | simt | ew], each 256-byte aligned
    size_t o_matn = 0, o_atab, o_stab, o_tc, o_simt, o_ew, total;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    o_atab = al(o_matn + count * sizeof(int));
    o_stab = al(o_atab + count * sizeof(void*));
    o_tc = al(o_stab + count * sizeof(void*));
    o_simt = al(o_tc + tc.size() * sizeof(int4));
    o_ew = al(o_simt + simt.size() * sizeof(int4));
    total = al(o_ew + ew.size() * sizeof(int4));
    if (p->tab_event && cudaEventSynchronize(p->tab_event) != cudaSuccess) return NEUMANN_ECUDA;
    if (total > p->h_tab_bytes) {
      if (p->h_tab) cudaFreeHost(p->h_tab);
      p->h_tab = nullptr;
      p->h_tab_bytes = 0;
      if (cudaMallocHost(reinterpret_cast<void**>(&p->h_tab), total) != cudaSuccess) {
        cudaGetLastError();
        return NEUMANN_ENOMEM;
      }
      p->h_tab_bytes = total;
    }
    if (!p->tab_event && cudaEventCreateWithFlags(&p->tab_event, cudaEventDisableTiming) != cudaSuccess)
      return NEUMANN_ECUDA;
    memcpy(p->h_tab + o_matn, matn.data(), count * sizeof(int));
    memcpy(p->h_tab + o_atab, atab.data(), count * sizeof(void*));
    memcpy(p->h_tab + o_stab, stab.data(), count * sizeof(void*));
    memcpy(p->h_tab + o_tc, tc.data(), tc.size() * sizeof(int4));
    memcpy(p->h_tab + o_simt, simt.data(), simt.size() * sizeof(int4));
    memcpy(p->h_tab + o_ew, ew.data(), ew.size() * sizeof(int4));
    char* ws = p->ws;
    if (cudaMemcpyAsync(ws + p->off_matn, p->h_tab + o_matn, count * sizeof(int), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(ws + p->off_atab, p->h_tab + o_atab, count * sizeof(void*), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(ws + p->off_stab, p->h_tab + o_stab, count * sizeof(void*), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(ws + p->off_tc, p->h_tab + o_tc, tc.size() * sizeof(int4), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(ws + p->off_simt, p->h_tab + o_simt, simt.size() * sizeof(int4), cudaMemcpyHostToDevice,
                        s) ||
        cudaMemcpyAsync(ws + p->off_ew, p->h_tab + o_ew, ew.size() * sizeof(int4), cudaMemcpyHostToDevice, s))
      return NEUMANN_ECUDA;
    if (nres > 0 &&  // the resident matrices' entries of the same image
        (cudaMemcpyAsync(ws + p->off_res_matn, p->h_tab + o_matn + ng * sizeof(int), nres * sizeof(int),
                         cudaMemcpyHostToDevice, s) ||
         cudaMemcpyAsync(ws + p->off_res_atab, p->h_tab + o_atab + ng * sizeof(void*), nres * sizeof(void*),
                         cudaMemcpyHostToDevice, s) ||
         cudaMemcpyAsync(ws + p->off_res_stab, p->h_tab + o_stab + ng * sizeof(void*), nres * sizeof(void*),
                         cudaMemcpyHostToDevice, s)))
      return NEUMANN_ECUDA;
    if (cudaEventRecord(p->tab_event, s)) return NEUMANN_ECUDA;
    p->last_chunk_run = ck;
    p->last_res_limit = p->res_limit;
    p->last_n.assign(n, n + count);
    p->last_a.assign(A, A + count);
    p->last_s.assign(S, S + count);
  }
  char* ws = p->ws;
  cudaEvent_t after_a = p->hook_after_a, before_s = p->hook_before_s;
  const int nres = p->res_count;
  if (nres > 0) {  // fork: the resident launches on their own stream
    if (!p->res_stream) {
      if (cudaStreamCreateWithFlags(&p->res_stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&p->res_fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p->res_join, cudaEventDisableTiming) != cudaSuccess)
        return NEUMANN_ECUDA;
    }
    // after the tables and the caller's A are in place; they write S, so after the previous copy-out
    if (cudaEventRecord(p->res_fork, s) != cudaSuccess || cudaStreamWaitEvent(p->res_stream, p->res_fork, 0) != cudaSuccess)
      return NEUMANN_ECUDA;
    if (before_s && cudaStreamWaitEvent(p->res_stream, before_s, 0) != cudaSuccess) return NEUMANN_ECUDA;
    for (const int3& cl : p->res_class) {  // one launch per size class
      ResParams R;
      memset(&R, 0, sizeof(R));
      R.ops = reinterpret_cast<const ResOp*>(ws + p->off_res_ops);
      R.nops = (int)p->res_ops.size();
      R.nslots = p->res_nslots;
      R.nf64 = p->res_nf64;
      for (int k = 0; k < 16; ++k) R.f64_of[k] = p->res_f64_of[k];
      R.count = cl.y;
      R.mat_n = reinterpret_cast<const int*>(ws + p->off_res_matn) + cl.x;
      R.A = reinterpret_cast<const void* const*>(ws + p->off_res_atab) + cl.x;
      R.S = reinterpret_cast<void* const*>(ws + p->off_res_stab) + cl.x;
      R.io_f64 = p->dt_io == DT_F64;
      R.mode = p->path == PATH_F32 ? 0 : p->dtype == NEUMANN_SPLIT_FP16 ? 2 : 1;
      R.status = reinterpret_cast<unsigned*>(ws);
      R.nmax = cl.z;
      if (launch_resident(R, p->res_stream) != cudaSuccess) return NEUMANN_ECUDA;
    }
    if (cudaEventRecord(p->res_join, p->res_stream) != cudaSuccess) return NEUMANN_ECUDA;
    if (p->hook_after_a_res && cudaEventRecord(p->hook_after_a_res, p->res_stream) != cudaSuccess)
      return NEUMANN_ECUDA;
  }
  for (size_t ci = 0; ci < p->chunks.size(); ++ci) {
    const neumann_plan_s::Chunk& ch = p->chunks[ci];
    // S is first written by the first chunk; A is last read by the last chunk
    p->hook_before_s = ci == 0 ? before_s : nullptr;
    p->hook_after_a = ci + 1 == p->chunks.size() ? after_a : nullptr;
    p->cur_matn = reinterpret_cast<const int*>(ws + p->off_matn) + ch.first;
    p->cur_atab = reinterpret_cast<const void* const*>(ws + p->off_atab) + ch.first;
    p->cur_stab = reinterpret_cast<void* const*>(ws + p->off_stab) + ch.first;
    p->cur_tc = reinterpret_cast<const int4*>(ws + p->off_tc) + ch.tc0;
    p->cur_simt = reinterpret_cast<const int4*>(ws + p->off_simt) + ch.simt0;
    p->cur_ew = reinterpret_cast<const int4*>(ws + p->off_ew) + ch.ew0;
    p->n_tc = ch.ntc;
    p->n_simt = ch.nsimt;
    p->n_ew = ch.new_;
    p->cur_count = ch.count;
    UserPtrs u{nullptr, 0, nullptr, nullptr, 0};
    int rc = run_ops(p, p->ops, p->maps, u, s, (p->flags & NEUMANN_FLAG_TIMING) != 0);
    if (rc) {
      p->hook_after_a = p->hook_before_s = nullptr;
      return rc;
    }
  }
  p->hook_after_a = p->hook_before_s = nullptr;
  if (nres > 0) {  // join: the evaluation ends once the resident launches have
    if (cudaStreamWaitEvent(s, p->res_join, 0) != cudaSuccess) return NEUMANN_ECUDA;
    if (p->chunks.empty() && after_a && cudaEventRecord(after_a, s) != cudaSuccess) return NEUMANN_ECUDA;
    if (p->chunks.empty() && before_s && cudaStreamWaitEvent(s, before_s, 0) != cudaSuccess) return NEUMANN_ECUDA;
  }
  return NEUMANN_OK;
}

// ---------------------------------------------------------------- autotuner
// Launch configurations chosen by timing, kept for the process so that later
// plans of the same shape start from them: single tensor-core products by
// (padded order, dtype); grouped batches by (count, max order, k, radix, dtype).
std::mutex g_tune_mu;
struct TuneSingle {
  int pair, group;
};
std::map<std::pair<int64_t, int>, TuneSingle> g_tune_single;
std::map<std::tuple<int, int64_t, int64_t, int, int>, std::pair<int, int>> g_tune_batched;  // chunk, resident limit

// Single products are keyed by padded order and dtype; precise-accumulation
// plans run another kernel and are keyed apart.
std::pair<int64_t, int> tune_key(const neumann_plan_s* p) {
  return std::make_pair(p->npad, p->dtype + ((p->flags & NEUMANN_FLAG_PRECISE_ACC) ? 16 : 0) + (p->sym ? 32 : 0));
}

void apply_tuned(neumann_plan_s* p) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (p->batched) {
    auto it = g_tune_batched.find(std::make_tuple(p->count, p->max_n, p->k, p->radix, p->dtype));
    if (it != g_tune_batched.end() && it->second.first <= p->chunk && it->second.second <= p->res_maxn) {
      p->chunk_run = it->second.first;
      p->res_limit = it->second.second;
      p->tuned = true;
    }
  } else if (p->path == PATH_TC) {
    auto it = g_tune_single.find(tune_key(p));
    if (it != g_tune_single.end()) {
      p->tune_pair = it->second.pair;
      p->tune_group = it->second.group;
      p->tuned = true;
    }
  }
}

// Median device time (ms) of `reps` back-to-back runs of `run` on stream s,
// after one untimed run.
template <typename F>
int time_runs(F run, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  int rc = run();
  if (rc) return rc;
  std::vector<float> t;
  for (int r = 0; r < reps; ++r) {
    if (cudaEventRecord(e0, s) != cudaSuccess) return NEUMANN_ECUDA;
    rc = run();
    if (rc) return rc;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return NEUMANN_ECUDA;
    float x = 0.f;
    if (cudaEventElapsedTime(&x, e0, e1) != cudaSuccess) return NEUMANN_ECUDA;
    t.push_back(x);
  }
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return NEUMANN_OK;
}

struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok() {
    return cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  }
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

int autotune_one(neumann_plan_s* p, const void* A, int64_t lda, void* S, int64_t lds, int reps, cudaStream_t s) {
  if (p->path != PATH_TC) {  // the SIMT products have one launch shape
    p->tuned = true;
    return NEUMANN_OK;
  }
  int rc = ensure_workspace(p, s);
  if (rc) return rc;
  EventPair ev;
  if (!ev.ok()) return NEUMANN_ECUDA;
  std::vector<TuneSingle> cand;
  const bool precise = (p->flags & NEUMANN_FLAG_PRECISE_ACC) != 0 || p->sym;  // always CTA pairs
  for (int pair = precise ? 1 : 0; pair <= 1; ++pair) {
    if (pair && (p->flags & NEUMANN_FLAG_SINGLE_CTA) && !precise) continue;
    for (int g : {4, 8, 16}) cand.push_back({pair, g});
  }
  float best = 0.f;
  TuneSingle pick = cand[0];
  for (size_t i = 0; i < cand.size(); ++i) {
    p->tune_pair = cand[i].pair;
    p->tune_group = cand[i].group;
    if (!build_maps(p, p->ops, &p->maps, p->sym) || !build_maps(p, p->mm_ops, &p->mm_maps)) return NEUMANN_ECUDA;
    float ms = 0.f;
    rc = time_runs([&] { return eval_one(p, A, lda, S, lds, s); }, reps, s, ev.e0, ev.e1, &ms);
    if (rc) return rc;
    if (i == 0 || ms < best) {
      best = ms;
      pick = cand[i];
    }
  }
  p->tune_pair = pick.pair;
  p->tune_group = pick.group;
  if (!build_maps(p, p->ops, &p->maps, p->sym) || !build_maps(p, p->mm_ops, &p->mm_maps)) return NEUMANN_ECUDA;
  p->timed = 0;  // tuning runs are not part of a NEUMANN_FLAG_TIMING record
  p->tuned = true;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_single[tune_key(p)] = pick;
  return NEUMANN_OK;
}

int autotune_batched(neumann_plan_s* p, int count, const int64_t* n, const void* const* A, void* const* S, int reps,
                     cudaStream_t s) {
  if (!p->grouped) {  // orders above 256: one plan per order, each tuned like a single plan
    p->tuned = true;
    return NEUMANN_OK;
  }
  int rc = ensure_workspace(p, s);
  if (rc) return rc;
  EventPair ev;
  if (!ev.ok()) return NEUMANN_ECUDA;
  // 1. the largest order the resident launch takes (none, 16, 32, 48, all it holds)
  std::vector<int> lim;
  for (int c : {0, 16, 32, 48, p->res_maxn})
    if (c <= p->res_maxn && std::find(lim.begin(), lim.end(), c) == lim.end()) lim.push_back(c);
  float best = 0.f;
  int pick_lim = p->res_limit;
  for (size_t i = 0; i < lim.size(); ++i) {
    p->res_limit = lim[i];
    float ms = 0.f;
    rc = time_runs([&] { return eval_grouped(p, count, n, A, S, s); }, reps, s, ev.e0, ev.e1, &ms);
    if (rc) return rc;
    if (i == 0 || ms < best) {
      best = ms;
      pick_lim = lim[i];
    }
  }
  p->res_limit = pick_lim;
  // 2. matrices per grouped pass: the chunk halved down to 64
  std::vector<int> cand;
  for (int c = p->chunk; c >= 64 || c == p->chunk; c /= 2) {
    cand.push_back(c);
    if (cand.size() == 6 || c < 2) break;
  }
  int pick = cand[0];
  for (size_t i = 0; i < cand.size(); ++i) {
    p->chunk_run = cand[i];
    float ms = 0.f;
    rc = time_runs([&] { return eval_grouped(p, count, n, A, S, s); }, reps, s, ev.e0, ev.e1, &ms);
    if (rc) return rc;
    if (i == 0 || ms < best) {
      best = ms;
      pick = cand[i];
    }
  }
  p->chunk_run = pick;
  p->timed = 0;
  p->tuned = true;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_batched[std::make_tuple(p->count, p->max_n, p->k, p->radix, p->dtype)] = std::make_pair(pick, pick_lim);
  return NEUMANN_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

int neumann_plan_create(neumann_plan_t* out, int64_t n, int64_t k, int radix, int dtype, uint32_t flags) {
  if (!out) return NEUMANN_EINVAL;
  *out = nullptr;
  neumann_plan_s* p = new (std::nothrow) neumann_plan_s();
  if (!p) return NEUMANN_ENOMEM;
  int rc;
  try {
    rc = init_plan(p, n, k, radix, dtype, flags);
  } catch (...) {
    rc = NEUMANN_ENOMEM;
  }
  if (rc) {
    delete p;
    return rc;
  }
  apply_tuned(p);
  *out = p;
  return NEUMANN_OK;
}

int neumann_plan_info(neumann_plan_t p, neumann_plan_info_t* info) {
  if (!p || !info) return NEUMANN_EINVAL;
  memset(info, 0, sizeof(*info));
  info->n = p->batched ? p->max_n : p->n;
  info->k = p->k;
  info->radix = p->radix;
  info->dtype = p->dtype;
  info->flags = p->flags;
  info->levels = (int)p->levels.size();
  for (size_t i = 0; i < p->levels.size() && i < NEUMANN_MAX_LEVELS; ++i) info->level_radix[i] = p->levels[i];
  info->products_formula = p->formula;
  int64_t g = 0;
  for (const Op& op : p->ops) g += op.kind == OP_GEMM;
  info->products_executed = g;
  info->launches = (int64_t)p->ops.size();
  info->workspace_bytes = p->ws_bytes;
  info->padded_n = p->npad;
  if (p->path == PATH_TC && !p->grouped && !p->batched) {
    info->tile_pair = ((p->flags & NEUMANN_FLAG_PRECISE_ACC) || p->sym) ? 1
                      : (p->flags & NEUMANN_FLAG_SINGLE_CTA) ? 0
                      : p->tune_pair < 0                     ? (int)tc_uses_pair(p->npad, 0)
                                                             : p->tune_pair;
    info->raster_group = p->tune_group;
  }
  if (p->grouped) info->batch_chunk = p->chunk_run > 0 ? p->chunk_run : p->chunk;
  info->resident_max_n = p->res_limit;
  info->tuned = p->tuned;
  for (const Op& op : p->ops) {
    const int64_t b = op_bytes(p, op);
    info->bytes_per_element += b;
    if (op.kind == OP_GEMM) info->product_bytes_per_element += b;
  }
  return NEUMANN_OK;
}

int neumann_plan_autotune(neumann_plan_t p, const void* A, int64_t lda, void* S, int64_t lds, int reps,
                          void* stream) {
  if (!p || p->batched || !A || !S || lda < p->n || lds < p->n || reps < 1) return NEUMANN_EINVAL;
  const size_t es = elem_bytes(p->dt_io);
  if (overlap(A, ((size_t)(p->n - 1) * lda + p->n) * es, S, ((size_t)(p->n - 1) * lds + p->n) * es))
    return NEUMANN_EINVAL;
  try {
    return autotune_one(p, A, lda, S, lds, reps, reinterpret_cast<cudaStream_t>(stream));
  } catch (...) {
    return NEUMANN_ENOMEM;
  }
}

int neumann_plan_set_launch(neumann_plan_t p, int tile_pair, int raster_group) {
  if (!p || p->batched || p->path != PATH_TC || tile_pair < -1 || tile_pair > 1 || raster_group < 1 ||
      raster_group > 65535)
    return NEUMANN_EINVAL;
  p->tune_pair = tile_pair;
  p->tune_group = raster_group;
  p->tuned = true;
  if (p->ws && (!build_maps(p, p->ops, &p->maps, p->sym) || !build_maps(p, p->mm_ops, &p->mm_maps)))
    return NEUMANN_ECUDA;
  return NEUMANN_OK;
}

int neumann_plan_autotune_batched(neumann_plan_t p, int count, const int64_t* n, const void* const* A,
                                  void* const* S, int reps, void* stream) {
  if (!p || !p->batched || count < 1 || count > p->count || !n || !A || !S || reps < 1) return NEUMANN_EINVAL;
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || n[i] > p->max_n || !A[i] || !S[i]) return NEUMANN_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  p->last_stream = s;
  try {
    return autotune_batched(p, count, n, A, S, reps, s);
  } catch (...) {
    return NEUMANN_ENOMEM;
  }
}

int neumann_plan_set_workspace(neumann_plan_t p, void* ws, size_t bytes) {
  if (!p || !ws || bytes < p->ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) return NEUMANN_EINVAL;
  if (p->ws_owned) {
    cudaFree(p->ws);
    p->ws_owned = false;
  }
  if (cudaMemset(ws, 0, 256) != cudaSuccess) return NEUMANN_ECUDA;
  int rc = attach(p, ws);
  if (rc) return rc;
  for (auto& kv : p->sub) {
    rc = neumann_plan_set_workspace(kv.second, ws, bytes);
    if (rc) return rc;
  }
  return NEUMANN_OK;
}

int neumann_eval(neumann_plan_t p, const void* A, int64_t lda, void* S, int64_t lds, void* stream) {
  if (!p || p->batched) return NEUMANN_EINVAL;
  try {
    return eval_one(p, A, lda, S, lds, reinterpret_cast<cudaStream_t>(stream));
  } catch (...) {
    return NEUMANN_ENOMEM;
  }
}

int neumann_eval_host(neumann_plan_t p, const void* A, int64_t lda, void* S, int64_t lds, void* stream) {
  if (!p || p->batched || !A || !S || lda < p->n || lds < p->n) return NEUMANN_EINVAL;
  const size_t es = elem_bytes(p->dt_io);
  const size_t row = (size_t)p->n * es, mat = row * (size_t)p->n;
  if (overlap(A, ((size_t)(p->n - 1) * lda) * es + row, S, ((size_t)(p->n - 1) * lds) * es + row))
    return NEUMANN_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  try {
    if (!p->cs_in) {
      if (cudaStreamCreateWithFlags(&p->cs_in, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamCreateWithFlags(&p->cs_out, cudaStreamNonBlocking) != cudaSuccess)
        return NEUMANN_ECUDA;
    }
    neumann_plan_s::HostStage& h = p->host[p->host_calls & 1];
    if (!h.a) {
      if (cudaMalloc(&h.a, mat) != cudaSuccess || cudaMalloc(&h.s, mat) != cudaSuccess) {
        cudaGetLastError();
        return NEUMANN_ENOMEM;
      }
      if (cudaEventCreateWithFlags(&h.in, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h.out, cudaEventDisableTiming) != cudaSuccess)
        return NEUMANN_ECUDA;
    }
    // copy in once this set's previous evaluation has consumed its input
    if (h.used && cudaStreamWaitEvent(p->cs_in, h.done, 0) != cudaSuccess) return NEUMANN_ECUDA;
    if (cudaMemcpy2DAsync(h.a, row, A, (size_t)lda * es, row, (size_t)p->n, cudaMemcpyHostToDevice, p->cs_in) !=
            cudaSuccess ||
        cudaEventRecord(h.in, p->cs_in) != cudaSuccess)
      return NEUMANN_ECUDA;
    // evaluate on the caller's stream once the input is in and this set's
    // previous result has been copied out
    if (cudaStreamWaitEvent(s, h.in, 0) != cudaSuccess) return NEUMANN_ECUDA;
    if (h.used && cudaStreamWaitEvent(s, h.out, 0) != cudaSuccess) return NEUMANN_ECUDA;
    int rc = eval_one(p, h.a, p->n, h.s, p->n, s);
    if (rc) return rc;
    if (cudaEventRecord(h.done, s) != cudaSuccess) return NEUMANN_ECUDA;
    // copy out while the caller's stream moves on
    if (cudaStreamWaitEvent(p->cs_out, h.done, 0) != cudaSuccess ||
        cudaMemcpy2DAsync(S, (size_t)lds * es, h.s, row, row, (size_t)p->n, cudaMemcpyDeviceToHost, p->cs_out) !=
            cudaSuccess ||
        cudaEventRecord(h.out, p->cs_out) != cudaSuccess)
      return NEUMANN_ECUDA;
    h.used = true;
    ++p->host_calls;
  } catch (...) {
    return NEUMANN_ENOMEM;
  }
  return NEUMANN_OK;
}

int neumann_eval_batched_host(neumann_plan_t p, int count, const int64_t* n, const void* A, void* S,
                              void* stream) {
  if (!p || !p->batched || count < 0 || count > p->count) return NEUMANN_EINVAL;
  if (count == 0) return NEUMANN_OK;
  if (!n || !A || !S) return NEUMANN_EINVAL;
  const size_t es = elem_bytes(p->dt_io);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > p->max_n) return NEUMANN_EINVAL;
    total += (size_t)n[i] * (size_t)n[i];
  }
  const size_t bytes = total * es;
  if (overlap(A, bytes, S, bytes)) return NEUMANN_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  try {
    if (!p->cs_in) {
      if (cudaStreamCreateWithFlags(&p->cs_in, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamCreateWithFlags(&p->cs_out, cudaStreamNonBlocking) != cudaSuccess)
        return NEUMANN_ECUDA;
    }
    if (!p->pk_in) {
      for (cudaEvent_t* e : {&p->pk_in, &p->pk_a_free, &p->pk_done, &p->pk_s_free, &p->pk_a_free_res})
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return NEUMANN_ECUDA;
    }
    if (bytes > p->pk_bytes) {  // grow the staging pair once nothing uses it
      if (p->pk_used && (cudaStreamSynchronize(p->cs_in) != cudaSuccess ||
                         cudaStreamSynchronize(p->cs_out) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
        return NEUMANN_ECUDA;
      if (p->pk_a) cudaFree(p->pk_a);
      if (p->pk_s) cudaFree(p->pk_s);
      p->pk_a = p->pk_s = nullptr;
      p->pk_bytes = 0;
      p->pk_used = false;
      if (cudaMalloc(&p->pk_a, bytes) != cudaSuccess || cudaMalloc(&p->pk_s, bytes) != cudaSuccess) {
        cudaGetLastError();
        return NEUMANN_ENOMEM;
      }
      p->pk_bytes = bytes;
    }
    std::vector<const void*> ad(count);
    std::vector<void*> sd(count);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
      ad[i] = p->pk_a + off * es;
      sd[i] = p->pk_s + off * es;
      off += (size_t)n[i] * (size_t)n[i];
    }
    // copy in once the previous evaluation has read its last A (grouped passes and resident launches)
    if (p->pk_used && (cudaStreamWaitEvent(p->cs_in, p->pk_a_free, 0) != cudaSuccess ||
                       cudaStreamWaitEvent(p->cs_in, p->pk_a_free_res, 0) != cudaSuccess))
      return NEUMANN_ECUDA;
    if (cudaMemcpyAsync(p->pk_a, A, bytes, cudaMemcpyHostToDevice, p->cs_in) != cudaSuccess ||
        cudaEventRecord(p->pk_in, p->cs_in) != cudaSuccess || cudaStreamWaitEvent(s, p->pk_in, 0) != cudaSuccess)
      return NEUMANN_ECUDA;
    int rc = ensure_workspace(p, s);
    if (rc) return rc;
    p->last_stream = s;
    p->hook_after_a = p->pk_a_free;
    p->hook_after_a_res = p->pk_a_free_res;
    p->hook_before_s = p->pk_used ? p->pk_s_free : nullptr;
    if (p->grouped) {
      rc = eval_grouped(p, count, n, ad.data(), sd.data(), s);
      p->hook_after_a_res = nullptr;
    } else {  // orders above 256: plain per-matrix evaluation, then the same copy-out
      p->hook_after_a = p->hook_before_s = nullptr;
      if (p->pk_used && cudaStreamWaitEvent(s, p->pk_s_free, 0) != cudaSuccess) return NEUMANN_ECUDA;
      rc = neumann_eval_batched(p, count, n, ad.data(), sd.data(), stream);
      if (!rc && cudaEventRecord(p->pk_a_free, s) != cudaSuccess) rc = NEUMANN_ECUDA;
    }
    p->hook_after_a = p->hook_before_s = nullptr;
    if (rc) return rc;
    // copy out while the caller's stream moves on
    if (cudaEventRecord(p->pk_done, s) != cudaSuccess || cudaStreamWaitEvent(p->cs_out, p->pk_done, 0) != cudaSuccess ||
        cudaMemcpyAsync(S, p->pk_s, bytes, cudaMemcpyDeviceToHost, p->cs_out) != cudaSuccess ||
        cudaEventRecord(p->pk_s_free, p->cs_out) != cudaSuccess)
      return NEUMANN_ECUDA;
    p->pk_used = true;
  } catch (...) {
    return NEUMANN_ENOMEM;
  }
  return NEUMANN_OK;
}

int neumann_plan_host_wait(neumann_plan_t p) {
  if (!p) return NEUMANN_EINVAL;
  if (p->cs_in && cudaStreamSynchronize(p->cs_in) != cudaSuccess) return NEUMANN_ECUDA;
  if (p->cs_out && cudaStreamSynchronize(p->cs_out) != cudaSuccess) return NEUMANN_ECUDA;
  return NEUMANN_OK;
}

int neumann_plan_matmul(neumann_plan_t p, const void* A, const void* B, void* C, void* stream) {
  if (!p || p->batched || !A || !B || !C) return NEUMANN_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)p->n * (size_t)p->n * elem_bytes(p->dt_io);
  if (overlap(A, bytes, C, bytes) || overlap(B, bytes, C, bytes)) return NEUMANN_EINVAL;
  int rc = ensure_workspace(p, s);
  if (rc) return rc;
  p->last_stream = s;
  UserPtrs u{A, p->n, B, C, p->n};
  return run_ops(p, p->mm_ops, p->mm_maps, u, s, false);
}

int neumann_plan_create_batched(neumann_plan_t* out, int count, int64_t max_n, int64_t k, int radix, int dtype,
                                uint32_t flags) {
  if (!out) return NEUMANN_EINVAL;
  *out = nullptr;
  if (count < 0) return NEUMANN_EINVAL;
  neumann_plan_t p = nullptr;
  // a grouped pass over orders <= 256 has no symmetric path (its products run whole slabs)
  const bool grouped = max_n <= kGroupedMaxN && count > 0;
  int rc = neumann_plan_create(&p, max_n, k, radix, dtype, grouped ? (flags & ~NEUMANN_FLAG_SYMMETRIC) : flags);
  if (rc) return rc;
  p->flags = flags;
  p->batched = true;
  p->count = count;
  p->max_n = max_n;
  if (max_n <= kGroupedMaxN && count > 0) {
    // one padded slab per matrix; up to kGroupedChunk matrices per grouped pass
    p->grouped = true;
    p->chunk = count < kGroupedChunk ? count : kGroupedChunk;
    p->npad = kGroupedMaxN;
    int brc = NEUMANN_OK;
    try {
      brc = build(p);  // the ops again, now for grouped launches, then the layout
    } catch (...) {
      brc = NEUMANN_ENOMEM;
    }
    if (brc != NEUMANN_OK) {
      neumann_plan_destroy(p);
      return brc;
    }
  }
  apply_tuned(p);
  *out = p;
  return NEUMANN_OK;
}

int neumann_eval_batched(neumann_plan_t p, int count, const int64_t* n, const void* const* A, void* const* S,
                         void* stream) {
  if (!p || !p->batched || count < 0 || count > p->count) return NEUMANN_EINVAL;
  if (count == 0) return NEUMANN_OK;
  if (!n || !A || !S) return NEUMANN_EINVAL;
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || n[i] > p->max_n || !A[i] || !S[i]) return NEUMANN_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  try {
    int rc = ensure_workspace(p, s);
    if (rc) return rc;
    p->last_stream = s;
    if (p->grouped) return eval_grouped(p, count, n, A, S, s);
    for (int i = 0; i < count; ++i) {
      neumann_plan_s*& sp = p->sub[n[i]];
      if (!sp) {
        rc = neumann_plan_create(&sp, n[i], p->k, p->radix, p->dtype, p->flags & ~NEUMANN_FLAG_TIMING);
        if (rc) {
          p->sub.erase(n[i]);
          return rc;
        }
        rc = attach(sp, p->ws);  // a smaller order needs no more workspace than max_n
        if (rc) return rc;
      }
      rc = eval_one(sp, A[i], n[i], S[i], n[i], s);
      if (rc) return rc;
    }
  } catch (...) {
    return NEUMANN_ENOMEM;
  }
  return NEUMANN_OK;
}

int neumann_last_status(neumann_plan_t p, unsigned* status) {
  if (!p || !status) return NEUMANN_EINVAL;
  *status = 0;
  if (!p->ws) return NEUMANN_OK;
  if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return NEUMANN_ECUDA;
  unsigned v = 0;
  if (cudaMemcpy(&v, p->ws, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return NEUMANN_ECUDA;
  if (v && cudaMemset(p->ws, 0, sizeof(v)) != cudaSuccess) return NEUMANN_ECUDA;
  *status = v;
  return NEUMANN_OK;
}

int neumann_plan_timing(neumann_plan_t p, float* ms, int cap, int* count) {
  if (!p || !count || !(p->flags & NEUMANN_FLAG_TIMING)) return NEUMANN_EINVAL;
  *count = p->timed;
  if (p->timed == 0) return NEUMANN_OK;
  if (cudaEventSynchronize(p->events[2 * p->timed - 1]) != cudaSuccess) return NEUMANN_ECUDA;
  for (int i = 0; i < p->timed && i < cap && ms; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->events[2 * i], p->events[2 * i + 1]) != cudaSuccess) return NEUMANN_ECUDA;
    ms[i] = t;
  }
  p->timed = 0;
  return NEUMANN_OK;
}

int neumann_plan_selftest_timeout(neumann_plan_t p, uint64_t limit_ns, void* stream) {
  if (!p || limit_ns > 1000000000ull) return NEUMANN_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = ensure_workspace(p, s);
  if (rc) return rc;
  p->last_stream = s;
  return launch_wait_probe(reinterpret_cast<unsigned*>(p->ws), limit_ns, s) == cudaSuccess ? NEUMANN_OK
                                                                                           : NEUMANN_ECUDA;
}

int neumann_radix15_coefficients(int set, double* coef28, double* prefix_error, double* spill15, double* spill16) {
  if ((set != 0 && set != 1) || !coef28) return NEUMANN_EINVAL;
  double e = 0, a = 0, b = 0;
  bool ok = radix15_coefficients(set, coef28, &e, &a, &b);
  if (prefix_error) *prefix_error = e;
  if (spill15) *spill15 = a;
  if (spill16) *spill16 = b;
  return ok ? NEUMANN_OK : NEUMANN_ENOTSUP;
}

int neumann_radix_p5_coefficients(int m, double* coef41, double* prefix_error, double* spill) {
  if ((m != 24 && m != 25 && m != 27 && m != 31 && m != 33) || !coef41) return NEUMANN_EINVAL;
  double e = 0, a = 0;
  const bool ok = radix_p5_coefficients(m, coef41, &e, &a);
  if (prefix_error) *prefix_error = e;
  if (spill) *spill = a;
  return ok ? NEUMANN_OK : NEUMANN_ENOTSUP;
}

void neumann_plan_destroy(neumann_plan_t p) {
  if (!p) return;
  for (auto& kv : p->sub) {
    kv.second->ws = nullptr;  // shares the parent's workspace
    neumann_plan_destroy(kv.second);
  }
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  if (p->cs_in) cudaStreamSynchronize(p->cs_in);
  if (p->cs_out) cudaStreamSynchronize(p->cs_out);
  for (auto& h : p->host) {
    if (h.a) cudaFree(h.a);
    if (h.s) cudaFree(h.s);
    for (cudaEvent_t e : {h.in, h.done, h.out})
      if (e) cudaEventDestroy(e);
  }
  if (p->pk_a) cudaFree(p->pk_a);
  if (p->pk_s) cudaFree(p->pk_s);
  for (cudaEvent_t e : {p->pk_in, p->pk_a_free, p->pk_done, p->pk_s_free, p->pk_a_free_res})
    if (e) cudaEventDestroy(e);
  if (p->res_stream) {
    cudaStreamSynchronize(p->res_stream);
    cudaStreamDestroy(p->res_stream);
  }
  for (cudaEvent_t e : {p->res_fork, p->res_join})
    if (e) cudaEventDestroy(e);
  if (p->cs_in) cudaStreamDestroy(p->cs_in);
  if (p->cs_out) cudaStreamDestroy(p->cs_out);
  if (p->tab_event) cudaEventDestroy(p->tab_event);
  if (p->h_tab) cudaFreeHost(p->h_tab);
  if (p->ws_owned) cudaFree(p->ws);
  delete p;
}

int neumann_measure_fma_peak(int dtype, double* tflops, int* sms, void* stream) {
  if (!tflops || (dtype != NEUMANN_FP32 && dtype != NEUMANN_FP64)) return NEUMANN_EINVAL;
  if (sms) *sms = sm_count();
  return measure_fma_peak(dtype == NEUMANN_FP64, tflops, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? NEUMANN_OK
             : NEUMANN_ECUDA;
}

const char* neumann_error_string(int code) {
  switch (code) {
    case NEUMANN_OK: return "ok";
    case NEUMANN_EINVAL: return "invalid argument";
    case NEUMANN_ENOMEM: return "out of memory";
    case NEUMANN_ECUDA: return "CUDA error";
    case NEUMANN_ENOTSUP: return "not supported";
  }
  return "unknown error";
}

}  // extern "C"
