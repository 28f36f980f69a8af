// tcgen05 tensor-core product for the split-BF16 / split-FP16 paths.
//
// Each operand x is stored as a pair hi = RN16(x), lo = RN16(x - hi), so
// x = hi + lo to about 2^-17 (BF16) or 2^-22 (scaled FP16) relative. A
// product A B is formed as
//   Ahi Bhi + Ahi Blo + Alo Bhi
// (the lo*lo term is dropped), all three issued as tcgen05.mma kind::f16
// instructions into one FP32 accumulator in tensor memory.
//
// The kernel is persistent and warp-specialised. A work item is a 128 x 256
// output tile (one CTA) or a 256 x 256 tile (a 2-CTA cluster, cta_group::2);
// items are taken in a grouped raster, item = first + i * stride:
//   warp 0 lane 0  TMA producer: four tiles per stage (Ahi, Alo, Bhi, Blo),
//                  K = 32 per stage (64-byte rows, 64B swizzle); 4 stages of
//                  48 KiB (single CTA) or 6 of 32 KiB (pair: each CTA loads its
//                  128 rows of A and 128 of the 256 columns of B)
//   warp 1         allocates tensor memory; lane 0 (of the even CTA of a pair)
//                  issues the MMAs: 2 K-slices x 3 products per stage, and
//                  tcgen05.commit frees the stage (in both CTAs of a pair)
//   warps 2-9      epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//                  lanes 32 (w % 4) .. +31 = 32 rows; two warps per lane
//                  quarter take alternate 32-column chunks) and the fused
//                  epilogue of epilogue.cuh
// Two 128 x 256 FP32 accumulators (all 512 TMEM columns) alternate between
// items, so the epilogue of one item runs while the next item's MMAs issue.
// A is read row-major (K-major); B is read from its transpose (row j of the
// stored array is column j of B), which makes it K-major too.
//
// Every mbarrier wait is bounded (kTimeoutNs): on expiry the kernel sets
// NEUMANN_STATUS_TIMEOUT, stops issuing, drains what it issued and frees its
// tensor memory before it returns.
#include <cuda_bf16.h>

#include <mutex>

#include "epilogue.cuh"

namespace neumann {

namespace {

constexpr int BM = 128;  // accumulator rows per CTA (TMEM lanes)
constexpr int BN = 256;  // accumulator columns (output columns of one work item)
constexpr int BK = 32;   // 16-bit elements per stage row = 64 bytes

constexpr uint32_t A_TILE = BM * BK * 2;  // 8 KiB
constexpr uint32_t STG_FLOATS = 32 * 33;  // one epilogue warp's 32 x 32 staging tile, padded
// Launch shapes.
//  * single CTA (kPair = false): a CTA owns a 128 x 256 output tile and loads
//    the full 256-row B panel per stage.
//  * CTA pair (kPair = true): a 2-CTA cluster owns a 256 x 256 tile. Each CTA
//    loads its own 128 rows of A and 128 of the 256 columns of B; the even CTA
//    issues M = 256 tcgen05.mma.cta_group::2 instructions that read B from both
//    CTAs and write each CTA's 128 rows into that CTA's tensor memory. Per
//    unit of MMA work an SM stores and reads a third less shared memory.
// Epilogue warps: 8, two per TMEM lane quarter taking alternate 32-column
// chunks. The epilogue is latency-bound (a chain of dependent loads, FMAs,
// conversions and stores per chunk), so two warps per scheduler keep it under
// the next tile's K loop.
// A grouped launch (matrices of order <= 256: K loops of at most 8 stages) is
// bound by its epilogue alone, so it runs 20 warps: warpgroup 0 holds the TMA
// and MMA warps (and two idle ones) and gives registers back (setmaxnreg 24)
// to four warpgroups of epilogue warps (112 each): 128 x 24 + 512 x 112 =
// 60416 <= 61440 = 640 threads x 96 at launch.
template <bool kGrouped, bool kPair>
struct EpiShape {
  static constexpr int kWarps = kGrouped ? 16 : 8;
  static constexpr int kEpiFirst = kGrouped ? 4 : 2;                  // first epilogue warp
  static constexpr int kThreads = 32 * (kEpiFirst + kWarps);         // TMA warp, MMA warp, (idle,) epilogue
  static constexpr int kBRows = kPair ? BN / 2 : BN;  // rows of the stored B^T panel this CTA loads
  static constexpr uint32_t kBTile = kBRows * BK * 2;
  static constexpr uint32_t kStageBytes = 2 * A_TILE + 2 * kBTile;
  static constexpr int kStages = kPair ? 6 : kGrouped ? 3 : 4;
  static constexpr int kTileM = kPair ? 2 * BM : BM;  // output rows of one work item
  // stages | barriers, TMEM address, abort flag (256 B) | staging tiles (+ alignment slack)
  static constexpr uint32_t kSmem = kStages * kStageBytes + 256 + kWarps * STG_FLOATS * 4 + 1024;
};
constexpr uint32_t ACC_COLS = BN;              // one FP32 accumulator: 128 lanes x 256 columns
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;   // double-buffered
constexpr uint64_t kTimeoutNs = 2000000000ull;  // 2 s; a whole launch normally takes < 20 ms
constexpr int64_t kPairMinN = 4096;  // padded orders from which a product runs on CTA pairs

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A and B both
// BF16 (format 1 at bits 7-9 and 10-12) or both FP16 (format 0), both K-major
// (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24 (M = 256 for a CTA pair).
__host__ __device__ constexpr uint32_t make_idesc(bool f16, int m) {
  return (1u << 4) | (f16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete; false once
// `limit_ns` has passed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns = kTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (gtimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major operand tile in shared memory with the 64-byte swizzle: rows of
// 64 bytes, 8-row atoms of 512 bytes stacked along M/N (stride byte offset
// 512), version 1 at bit 46, layout type 4 (SWIZZLE_64B) at bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// MN-major operand tile (B read from its row-major hi/lo pair, B^T never
// stored): strips of 32 columns (64-byte rows, 64B swizzle) of 32 K rows each,
// strip after strip. Leading byte offset: from one 32-column strip to the
// next along N (2048); stride byte offset: from one 8-row K group to the next
// (512).
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(2048 >> 4) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// One MMA instruction D (+)= A B^T of the launch shape: cta_group::1 with
// M = 128, or cta_group::2 with M = 256 issued by the even CTA of a pair.
template <bool kPair>
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  if constexpr (kPair) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// Arrive on `bar` once every MMA this thread issued so far has completed. For
// a pair, `both` arrives on the barrier at the same offset in both CTAs.
template <bool kPair>
__device__ __forceinline__ void umma_commit(uint32_t bar, bool both = true) {
  if constexpr (kPair) {
    if (both) {
      asm volatile(
          "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
              bar),
          "h"((uint16_t)3)
          : "memory");
    } else {
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
  } else {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
  }
}

template <bool kPair>
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
  if constexpr (kPair) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  } else {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}

template <bool kPair>
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
  if constexpr (kPair)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
  else
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// ---- clusters (CTA pairs) ----
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Address, in the cluster's shared window, of the same offset in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
// Every thread of both CTAs; orders earlier shared-memory writes (barrier
// initialisation included) before later accesses from the other CTA.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, uint32_t cluster_bar, int x,
                                                 int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(cluster_bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// TMA load into this CTA's shared memory whose completion is counted on the
// even CTA's barrier (`cluster_bar`, an address in the cluster window).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t cluster_bar, int x,
                                                 int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(cluster_bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Grouped raster: `group` row tiles form a group; work items run down the
// group's rows first, so neighbouring CTAs share column panels of B in L2.
__device__ __forceinline__ void raster(int bid, int tiles_m, int tiles_n, int group, int* tm, int* tn) {
  const int per_group = group * tiles_n;
  const int g = bid / per_group;
  const int first = g * group;
  const int gs = min(tiles_m - first, group);
  const int in = bid - g * per_group;
  *tm = first + in % gs;
  *tn = in / gs;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Work item `tile` of the launch: matrix, 128-row tile, 256-column tile and the
// number of 32-deep K stages. A single product walks the grouped raster; a
// grouped launch reads the host-built table (one 128 x 256 tile per entry,
// K stages covering that matrix's order rounded up to 32).
template <bool kGrouped>
__device__ __forceinline__ void tile_of(int tile, const int4* tiles, int ktiles, int tiles_m, int tiles_n, int group,
                                        int* mat, int* tm, int* tn, int* nk, const int2* sym = nullptr) {
  if (!kGrouped && sym) {  // a symmetric product: the host's list of tiles on or above the diagonal
    const int2 t = sym[tile];
    *mat = 0;
    *tm = t.x;
    *tn = t.y;
    *nk = ktiles;
  } else if (kGrouped) {
    const int4 t = tiles[tile];
    *mat = t.x;
    *tm = t.y;
    *tn = 0;
    *nk = t.z;
  } else {
    *mat = 0;
    raster(tile, tiles_m, tiles_n, group, tm, tn);
    *nk = ktiles;
  }
}

// The four operand tiles of K stage `kb` of a work item: rows `ra` of A
// (hi, lo) and rows `rb` of the stored B^T (hi, lo), 32 deep.
template <bool kGrouped, bool kPair>
// bmn: B is read MN-major from its row-major pair (columns rb .. of rows
// kb*32 ..) as 32-column strips; otherwise K-major from the stored B^T (rows rb ..).
__device__ __forceinline__ void load_stage(uint32_t st, const CUtensorMap* ahi, const CUtensorMap* alo,
                                           const CUtensorMap* bhi, const CUtensorMap* blo, uint32_t bar, int kb,
                                           int ra, int rb, int mat, bool bmn) {
  using S = EpiShape<kGrouped, kPair>;
  const uint32_t sb = st + 2 * A_TILE;
  if constexpr (kGrouped) {
    tma_load_3d(st, ahi, bar, kb * BK, ra, mat);
    tma_load_3d(st + A_TILE, alo, bar, kb * BK, ra, mat);
    if (bmn) {
      tma_load_4d(sb, bhi, bar, 0, kb * BK, rb / 32, mat);
      tma_load_4d(sb + S::kBTile, blo, bar, 0, kb * BK, rb / 32, mat);
    } else {
      tma_load_3d(sb, bhi, bar, kb * BK, rb, mat);
      tma_load_3d(sb + S::kBTile, blo, bar, kb * BK, rb, mat);
    }
  } else if constexpr (kPair) {
    tma_load_2d_pair(st, ahi, bar, kb * BK, ra);
    tma_load_2d_pair(st + A_TILE, alo, bar, kb * BK, ra);
    if (bmn) {
      tma_load_3d_pair(sb, bhi, bar, 0, kb * BK, rb / 32);
      tma_load_3d_pair(sb + S::kBTile, blo, bar, 0, kb * BK, rb / 32);
    } else {
      tma_load_2d_pair(sb, bhi, bar, kb * BK, rb);
      tma_load_2d_pair(sb + S::kBTile, blo, bar, kb * BK, rb);
    }
  } else {
    tma_load_2d(st, ahi, bar, kb * BK, ra);
    tma_load_2d(st + A_TILE, alo, bar, kb * BK, ra);
    if (bmn) {
      tma_load_3d(sb, bhi, bar, 0, kb * BK, rb / 32);
      tma_load_3d(sb + S::kBTile, blo, bar, 0, kb * BK, rb / 32);
    } else {
      tma_load_2d(sb, bhi, bar, kb * BK, rb);
      tma_load_2d(sb + S::kBTile, blo, bar, kb * BK, rb);
    }
  }
}

__device__ __forceinline__ void spin_ns(uint64_t ns) {
  const uint64_t t0 = gtimer();
  while (gtimer() - t0 < ns) {
  }
}

template <bool kGrouped, bool kF16, bool kPair>
__global__ void __launch_bounds__(EpiShape<kGrouped, kPair>::kThreads, 1)
    tc_split_gemm_kernel(const __grid_constant__ CUtensorMap tm_ahi, const __grid_constant__ CUtensorMap tm_alo,
                         const __grid_constant__ CUtensorMap tm_bhi, const __grid_constant__ CUtensorMap tm_blo,
                         int ktiles, int tiles_m, int tiles_n, int group, const int4* __restrict__ tiles,
                         int ntiles_grouped, const int2* __restrict__ sym, int bmn,
                         const __grid_constant__ EpiParams P) {
  static_assert(!(kGrouped && kPair), "grouped launches use single-CTA tiles");
  using S = EpiShape<kGrouped, kPair>;
  constexpr int STAGES = S::kStages;
  constexpr uint32_t STAGE_BYTES = S::kStageBytes;
  constexpr uint32_t idesc = make_idesc(kF16, S::kTileM);
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // barriers: full[S], empty[S], tfull[2], tempty[2], drain
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // a symmetric product runs only the ntiles_grouped tiles listed in `sym`
  const int ntiles = (kGrouped || sym) ? ntiles_grouped : tiles_m * tiles_n;
  // Work items: one per CTA (single) or per cluster (pair); both CTAs of a
  // pair walk the same items, the odd one owning rows 128 .. 255 of each.
  const uint32_t rank = kPair ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  const int first = kPair ? (int)cluster_index() : (int)blockIdx.x;
  const int stride = kPair ? (int)cluster_count() : (int)gridDim.x;
  const uint32_t smem_base = smem_u32(smem);
  const uint32_t bar_base = smem_u32(bars);
  auto full_bar = [&](uint32_t s) { return bar_base + 8u * s; };
  auto empty_bar = [&](uint32_t s) { return bar_base + 8u * (STAGES + s); };
  auto tfull_bar = [&](uint32_t b) { return bar_base + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](uint32_t b) { return bar_base + 8u * (2 * STAGES + 2 + b); };
  const uint32_t drain_bar = bar_base + 8u * (2 * STAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      // lane 0 of each epilogue warp (of both CTAs for a pair; only the even CTA's is used)
      mbar_init(tempty_bar(b), S::kWarps * (kPair ? 2 : 1));
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<kPair>(smem_u32(tmem_slot), TMEM_COLS);
  tc_fence_before();
  if constexpr (kPair)
    cluster_sync();
  else
    __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // Stage-full and accumulator-free barriers live in the even CTA of a pair.
  const uint32_t lead_bar_base = kPair ? cluster_addr(bar_base, 0) : bar_base;
  if (warp >= S::kEpiFirst) {
    if constexpr (kGrouped) asm volatile("setmaxnreg.inc.sync.aligned.u32 112;" ::: "memory");
    // ---------------- epilogue (warps kEpiFirst .. kEpiFirst + kWarps) ----------------
    // Each 32 x 32 chunk is read from TMEM one row per lane, staged in shared
    // memory, and processed one column per lane (epi_col), so that the warp's
    // global loads and stores of row-major buffers touch one line per instruction.
    constexpr int kStep = S::kWarps / 4;          // warps per TMEM lane quarter
    const int q = warp & 3;                       // TMEM lane quarter this warp may access
    const int half = (warp - S::kEpiFirst) >> 2;  // warps of one quarter take turns at column chunks
    float* stg = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256) + (warp - S::kEpiFirst) * STG_FLOATS;
    bool bad = false;
    int it = 0;
    SxTile sxt;        // split-FP16: the tile's scales
    float am = 0.f;    // split-FP16: max |acc| (staged units) of this lane's rows of the tile
    for (int tile = first; tile < ntiles; tile += stride, ++it) {
      const uint32_t buf = it & 1;
      const uint32_t use = (uint32_t)it >> 1;
      const bool got = mbar_wait(tfull_bar(buf), use & 1u);
      if (!__all_sync(0xffffffffu, got && !*abort_flag)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      int mat, tm, tn, nk;
      tile_of<kGrouped>(tile, tiles, ktiles, tiles_m, tiles_n, group, &mat, &tm, &tn, &nk, sym);
      const EpiCtx x = epi_ctx(P, mat);
      if constexpr (kF16) sx_tile(P, mat, &sxt);
      const int rbase = tm * S::kTileM + (int)rank * BM + q * 32;
      const uint32_t taddr = tmem + buf * ACC_COLS + ((uint32_t)(q * 32) << 16);
      // A grouped tile writes rows and columns below its matrix's order rounded
      // up to 32 (= nk x 32): with that K padding zero in both operands, later
      // rows and columns only feed accumulator entries every consumer discards.
      const int nchunks = kGrouped ? nk : BN / 32;
      const int lim = kGrouped ? nk * 32 : (1 << 30);
      // symmetric product: chunks below the diagonal are left to their transpose
      const int cdiag = kGrouped ? 0 : tn * BN - rbase;  // first column of the tile minus this warp's first row
#pragma unroll 1
      for (int chunk = half; chunk < nchunks; chunk += kStep) {
        const int rel = cdiag + chunk * 32;  // this chunk's first column minus its first row
        if (sym && rel < 0) continue;        // below the diagonal
        const int symc = !sym ? 0 : rel > 0 ? 1 : 2;
        uint32_t v[32];
        __syncwarp();
        tmem_ld32(taddr + (uint32_t)(chunk * 32), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(v[j]);
        if constexpr (kF16) {
          if (rbase + lane < lim) am = fmaxf(am, sx_row_max(v));
        }
        __syncwarp();
        if constexpr (kF16) sx_chunk_colsum(P, mat, stg, lane, rbase, tn * BN + chunk * 32, symc, lim, sxt.acc);
        bad |= epi_chunk<kF16>(P, x, rbase, tn * BN + chunk * 32 + lane, stg, lane, lim, symc,
                               kF16 ? &sxt : nullptr);
        __syncwarp();
      }
      if constexpr (kF16) {
        sx_tile_max(P, mat, am, sxt.acc);
        am = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (kPair)
          mbar_arrive_cluster(lead_bar_base + 8u * (2 * STAGES + 2 + buf));
        else
          mbar_arrive(tempty_bar(buf));
      }
    }
    epi_flag(P, bad);
  } else {
    if constexpr (kGrouped) asm volatile("setmaxnreg.dec.sync.aligned.u32 24;" ::: "memory");
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_ahi)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_alo)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_bhi)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_blo)) : "memory");
      uint32_t kg = 0;  // stage loads issued so far
      bool ok = true;
      for (int tile = first; tile < ntiles && ok; tile += stride) {
        int mat, tm, tn, nk;
        tile_of<kGrouped>(tile, tiles, ktiles, tiles_m, tiles_n, group, &mat, &tm, &tn, &nk, sym);
        const int ra = tm * S::kTileM + (int)rank * BM;
        const int rb = tn * BN + (int)rank * S::kBRows;
        for (int kb = 0; kb < nk; ++kb) {
          const uint32_t s = kg % STAGES;
          const uint32_t ph = (kg / STAGES) & 1u;
          if (kg >= STAGES && (!mbar_wait(empty_bar(s), ph ^ 1u) || *abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t st = smem_base + s * STAGE_BYTES;
          if (leader) mbar_expect_tx(full_bar(s), STAGE_BYTES * (kPair ? 2u : 1u));
          load_stage<kGrouped, kPair>(st, &tm_ahi, &tm_alo, &tm_bhi, &tm_blo, lead_bar_base + 8u * s, kb, ra, rb,
                                      mat, bmn != 0);
          ++kg;
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (leader) {
          // drain: wait (bounded) for the last load issued into each stage
          for (uint32_t q = (kg > STAGES ? kg - STAGES : 0); q < kg; ++q)
            mbar_wait(full_bar(q % STAGES), (q / STAGES) & 1u, 10000000ull);
        } else {
          // this CTA's loads complete on the even CTA's barriers: give them time to land
          spin_ns(10000000ull);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer ----------------
      uint32_t kg = 0;
      bool ok = true;
      int it = 0;
      for (int tile = first; tile < ntiles && ok; tile += stride, ++it) {
        const uint32_t buf = it & 1;
        const uint32_t use = (uint32_t)it >> 1;
        if (it >= 2 && (!mbar_wait(tempty_bar(buf), (use - 1) & 1u) || *abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        int mat, tm, tn, nk;
        tile_of<kGrouped>(tile, tiles, ktiles, tiles_m, tiles_n, group, &mat, &tm, &tn, &nk, sym);
        const uint32_t d = tmem + buf * ACC_COLS;
        for (int kb = 0; kb < nk; ++kb) {
          const uint32_t s = kg % STAGES;
          const uint32_t ph = (kg / STAGES) & 1u;
          if (!mbar_wait(full_bar(s), ph) || *abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_base + s * STAGE_BYTES;
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            const uint64_t a_hi = smem_desc(st + 32u * j);
            const uint64_t a_lo = smem_desc(st + A_TILE + 32u * j);
            const uint32_t sb = st + 2 * A_TILE;
            // MN-major B: K slice j starts 16 rows (1 KiB) into every strip
            const uint64_t b_hi = bmn ? smem_desc_mn(sb + 1024u * j) : smem_desc(sb + 32u * j);
            const uint64_t b_lo = bmn ? smem_desc_mn(sb + S::kBTile + 1024u * j) : smem_desc(sb + S::kBTile + 32u * j);
            const uint32_t id = idesc | (bmn ? (1u << 16) : 0u);  // bit 16: B is MN-major
            umma_f16<kPair>(d, a_hi, b_hi, id, (kb | j) != 0);
            umma_f16<kPair>(d, a_hi, b_lo, id, 1u);
            umma_f16<kPair>(d, a_lo, b_hi, id, 1u);
          }
          umma_commit<kPair>(empty_bar(s));  // frees the stage in both CTAs of a pair
          ++kg;
        }
        if (ok) umma_commit<kPair>(tfull_bar(buf));  // accumulator `buf` holds the finished tile
      }
      if (!ok) *abort_flag = 1;
      // no MMA may be in flight when the tensor memory is freed
      umma_commit<kPair>(drain_bar, false);
      mbar_wait(drain_bar, 0);
    }
  }
  }

  tc_fence_before();
  if constexpr (kPair)
    cluster_sync();  // the even CTA's MMAs into this CTA's tensor memory have drained
  else
    __syncthreads();
  if (threadIdx.x == 0 && *abort_flag && P.status) atomicOr(P.status, 2u);
  if (warp == 1) {
    tc_fence_after();
    tmem_free<kPair>(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// Precise accumulation (NEUMANN_FLAG_PRECISE_ACC). The tensor cores' FP32
// accumulator rounds each MMA update toward zero; over the 3K/16 updates of a
// long K loop that leaves a bias of about (3K/16)/4 ulp of the sum, which at
// K = 8192 is larger than the operand split error. Here K is taken in chunks
// of 512: chunk 0 of a tile accumulates in TMEM region S, every later chunk in
// a fresh region X, and drain warps add X into S with round-to-nearest FP32
// adds, so the truncated chain is 96 updates long whatever K is.
//   tile      256 x 128 on a CTA pair (cta_group::2, M = 256, N = 128); each
//             CTA loads its 128 rows of A and 64 of the 128 rows of the stored B^T
//   TMEM      X0 [0,128), X1 [128,256): chunk accumulators, alternating by chunk;
//             S0 [256,384), S1 [384,512): tile sums, alternating by tile
//   warps     0 TMA; 1 MMA (even CTA); 2-5 drain (one per TMEM lane quarter);
//             6-7 idle; 8-15 epilogue (two per lane quarter), as in the main kernel
//   registers the TMA / MMA / drain warpgroups give back registers
//             (setmaxnreg 56) to the two epilogue warpgroups (200):
//             2 x 128 x 56 + 2 x 128 x 200 = 65536 = 512 threads x 128 at launch
constexpr int PQ_N = 128;                                // tile columns
constexpr int PQ_BROWS = PQ_N / 2;                       // stored B^T rows per CTA
constexpr uint32_t PQ_BTILE = PQ_BROWS * BK * 2;         // 4 KiB
constexpr uint32_t PQ_STAGE = 2 * A_TILE + 2 * PQ_BTILE;  // 24 KiB
constexpr int PQ_STAGES = 8;
constexpr int PQ_KC = 16;  // 32-deep stages per K chunk (512)
constexpr int PQ_THREADS = 512;
constexpr int PQ_EPI_WARPS = 8;
constexpr uint32_t PQ_SMEM = PQ_STAGES * PQ_STAGE + 256 + PQ_EPI_WARPS * STG_FLOATS * 4 + 1024;
constexpr uint32_t PQ_X = 0, PQ_S = 256;  // TMEM column bases

__host__ __device__ constexpr uint32_t make_idesc_mn(bool f16, int m, int n) {
  return (1u << 4) | (f16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

template <bool kF16>
__global__ void __launch_bounds__(PQ_THREADS, 1)
    tc_precise_kernel(const __grid_constant__ CUtensorMap tm_ahi, const __grid_constant__ CUtensorMap tm_alo,
                      const __grid_constant__ CUtensorMap tm_bhi, const __grid_constant__ CUtensorMap tm_blo,
                      int ktiles, int tiles_m, int tiles_n, int group, int bmn,
                      const __grid_constant__ EpiParams P) {
  constexpr uint32_t idesc0 = make_idesc_mn(kF16, 2 * BM, PQ_N);
  const uint32_t idesc = idesc0 | (bmn ? (1u << 16) : 0u);  // bit 16: B is MN-major
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // barriers: full[8], empty[8], xfull[2], xempty[2], sfull[2], sempty[2], drain
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + PQ_STAGES * PQ_STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * PQ_STAGES + 9);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = tiles_m * tiles_n;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int first = (int)cluster_index(), stride = (int)cluster_count();
  const int nchunks = (ktiles + PQ_KC - 1) / PQ_KC;
  const uint32_t smem_base = smem_u32(smem);
  const uint32_t bar_base = smem_u32(bars);
  auto full_bar = [&](uint32_t i) { return bar_base + 8u * i; };
  auto empty_bar = [&](uint32_t i) { return bar_base + 8u * (PQ_STAGES + i); };
  auto xfull_bar = [&](uint32_t b) { return bar_base + 8u * (2 * PQ_STAGES + b); };
  auto xempty_bar = [&](uint32_t b) { return bar_base + 8u * (2 * PQ_STAGES + 2 + b); };
  auto sfull_bar = [&](uint32_t b) { return bar_base + 8u * (2 * PQ_STAGES + 4 + b); };
  auto sempty_bar = [&](uint32_t b) { return bar_base + 8u * (2 * PQ_STAGES + 6 + b); };
  const uint32_t drain_bar = bar_base + 8u * (2 * PQ_STAGES + 8);

  if (threadIdx.x == 0) {
    for (int i = 0; i < PQ_STAGES; ++i) {
      mbar_init(full_bar(i), 1);
      mbar_init(empty_bar(i), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(xfull_bar(b), 1);
      mbar_init(xempty_bar(b), 4 * 2);  // the drain warps of both CTAs (the even CTA's is used)
      // the MMA commit, and this CTA's drain warps when there is anything to drain
      mbar_init(sfull_bar(b), nchunks > 1 ? 1 + 4 : 1);
      mbar_init(sempty_bar(b), PQ_EPI_WARPS * 2);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<true>(smem_u32(tmem_slot), TMEM_COLS);
  tc_fence_before();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lead_bar_base = cluster_addr(bar_base, 0);

  if (warp >= 8) {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 200;" ::: "memory");
    // ---------------- epilogue (warps 8 .. 15) ----------------
    const int q = warp & 3;
    const int half = (warp - 8) >> 2;
    float* stg = reinterpret_cast<float*>(smem + PQ_STAGES * PQ_STAGE + 256) + (warp - 8) * STG_FLOATS;
    bool bad = false;
    int it = 0;
    SxTile sxt;
    float am = 0.f;
    if constexpr (kF16) sx_tile(P, 0, &sxt);
    for (int tile = first; tile < ntiles; tile += stride, ++it) {
      const uint32_t sb = it & 1;
      const uint32_t su = (uint32_t)it >> 1;
      const bool got = mbar_wait(sfull_bar(sb), su & 1u);
      if (!__all_sync(0xffffffffu, got && !*abort_flag)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      int tm, tn;
      raster(tile, tiles_m, tiles_n, group, &tm, &tn);
      const EpiCtx x = epi_ctx(P, 0);
      const int rbase = tm * 2 * BM + (int)rank * BM + q * 32;
      const uint32_t taddr = tmem + PQ_S + sb * PQ_N + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int chunk = half; chunk < PQ_N / 32; chunk += 2) {
        uint32_t v[32];
        __syncwarp();
        tmem_ld32(taddr + (uint32_t)(chunk * 32), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) stg[lane * 33 + i] = __uint_as_float(v[i]);
        if constexpr (kF16) am = fmaxf(am, sx_row_max(v));
        __syncwarp();
        if constexpr (kF16) sx_chunk_colsum(P, 0, stg, lane, rbase, tn * PQ_N + chunk * 32, 0, 1 << 30, sxt.acc);
        bad |= epi_chunk<kF16>(P, x, rbase, tn * PQ_N + chunk * 32 + lane, stg, lane, 1 << 30, 0,
                               kF16 ? &sxt : nullptr);
        __syncwarp();
      }
      if constexpr (kF16) {
        sx_tile_max(P, 0, am, sxt.acc);
        am = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_bar_base + 8u * (2 * PQ_STAGES + 6 + sb));
    }
    epi_flag(P, bad);
  } else {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 56;" ::: "memory");
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t kg = 0;
      bool ok = true;
      for (int tile = first; tile < ntiles && ok; tile += stride) {
        int tm, tn;
        raster(tile, tiles_m, tiles_n, group, &tm, &tn);
        const int ra = tm * 2 * BM + (int)rank * BM;
        const int rb = tn * PQ_N + (int)rank * PQ_BROWS;
        for (int kb = 0; kb < ktiles; ++kb) {
          const uint32_t st = kg % PQ_STAGES;
          const uint32_t ph = (kg / PQ_STAGES) & 1u;
          if (kg >= PQ_STAGES && (!mbar_wait(empty_bar(st), ph ^ 1u) || *abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t sa = smem_base + st * PQ_STAGE;
          if (leader) mbar_expect_tx(full_bar(st), 2 * PQ_STAGE);
          const uint32_t fb = lead_bar_base + 8u * st;
          tma_load_2d_pair(sa, &tm_ahi, fb, kb * BK, ra);
          tma_load_2d_pair(sa + A_TILE, &tm_alo, fb, kb * BK, ra);
          if (bmn) {
            tma_load_3d_pair(sa + 2 * A_TILE, &tm_bhi, fb, 0, kb * BK, rb / 32);
            tma_load_3d_pair(sa + 2 * A_TILE + PQ_BTILE, &tm_blo, fb, 0, kb * BK, rb / 32);
          } else {
            tma_load_2d_pair(sa + 2 * A_TILE, &tm_bhi, fb, kb * BK, rb);
            tma_load_2d_pair(sa + 2 * A_TILE + PQ_BTILE, &tm_blo, fb, kb * BK, rb);
          }
          ++kg;
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (leader) {
          for (uint32_t q = (kg > PQ_STAGES ? kg - PQ_STAGES : 0); q < kg; ++q)
            mbar_wait(full_bar(q % PQ_STAGES), (q / PQ_STAGES) & 1u, 10000000ull);
        } else {
          spin_ns(10000000ull);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer ----------------
      uint32_t kg = 0, cc = 0;
      bool ok = true;
      int it = 0;
      for (int tile = first; tile < ntiles && ok; tile += stride, ++it) {
        const uint32_t sb = it & 1;
        const uint32_t su = (uint32_t)it >> 1;
        if (it >= 2 && (!mbar_wait(sempty_bar(sb), (su - 1) & 1u) || *abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int j = 0; j < nchunks && ok; ++j) {
          uint32_t d = tmem + PQ_S + sb * PQ_N;  // chunk 0 accumulates in the tile sum itself
          uint32_t xb = 0;
          if (j > 0) {
            xb = cc & 1;
            const uint32_t xu = cc >> 1;
            if (cc >= 2 && (!mbar_wait(xempty_bar(xb), (xu - 1) & 1u) || *abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            d = tmem + PQ_X + xb * PQ_N;
          }
          const int k1 = min(ktiles, (j + 1) * PQ_KC);
          for (int kb = j * PQ_KC; kb < k1; ++kb) {
            const uint32_t st = kg % PQ_STAGES;
            const uint32_t ph = (kg / PQ_STAGES) & 1u;
            if (!mbar_wait(full_bar(st), ph) || *abort_flag) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_base + st * PQ_STAGE;
#pragma unroll
            for (int q = 0; q < BK / 16; ++q) {
              const uint64_t a_hi = smem_desc(sa + 32u * q);
              const uint64_t a_lo = smem_desc(sa + A_TILE + 32u * q);
              const uint32_t sb = sa + 2 * A_TILE;
              const uint64_t b_hi = bmn ? smem_desc_mn(sb + 1024u * q) : smem_desc(sb + 32u * q);
              const uint64_t b_lo = bmn ? smem_desc_mn(sb + PQ_BTILE + 1024u * q) : smem_desc(sb + PQ_BTILE + 32u * q);
              umma_f16<true>(d, a_hi, b_hi, idesc, (kb != j * PQ_KC || q != 0) ? 1u : 0u);
              umma_f16<true>(d, a_hi, b_lo, idesc, 1u);
              umma_f16<true>(d, a_lo, b_hi, idesc, 1u);
            }
            umma_commit<true>(empty_bar(st));
            ++kg;
          }
          if (ok && j > 0) {
            umma_commit<true>(xfull_bar(xb));  // chunk j is in X[xb] in both CTAs
            ++cc;
          }
        }
        if (ok) umma_commit<true>(sfull_bar(sb));  // every MMA of the tile has completed
      }
      if (!ok) *abort_flag = 1;
      umma_commit<true>(drain_bar, false);
      mbar_wait(drain_bar, 0);
    }
  } else if (warp < 6) {
    // ---------------- drain: S += X, FP32 round to nearest ----------------
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    uint32_t cc = 0;
    int it = 0;
    bool ok = true;
    for (int tile = first; tile < ntiles && ok; tile += stride, ++it) {
      const uint32_t sb = it & 1;
      for (int j = 1; j < nchunks; ++j) {
        const uint32_t xb = cc & 1;
        const bool got = mbar_wait(xfull_bar(xb), (cc >> 1) & 1u);
        if (!__all_sync(0xffffffffu, got && !*abort_flag)) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t xa = tmem + lane_off + PQ_X + xb * PQ_N;
        const uint32_t sa = tmem + lane_off + PQ_S + sb * PQ_N;
#pragma unroll 1
        for (int piece = 0; piece < PQ_N / 16; ++piece) {
          uint32_t xv[16], sv[16];
          tmem_ld16(xa + piece * 16, xv);
          tmem_ld16(sa + piece * 16, sv);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int i = 0; i < 16; ++i) sv[i] = __float_as_uint(__uint_as_float(sv[i]) + __uint_as_float(xv[i]));
          tmem_st16(sa + piece * 16, sv);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(lead_bar_base + 8u * (2 * PQ_STAGES + 2 + xb));
        ++cc;
      }
      if (!ok) break;
      if (nchunks > 1) {  // with one chunk the tile sum is the MMA's own result
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(sfull_bar(sb));
      }
    }
  }
  }

  tc_fence_before();
  cluster_sync();
  if (threadIdx.x == 0 && *abort_flag && P.status) atomicOr(P.status, 2u);
  if (warp == 1) {
    tc_fence_after();
    tmem_free<true>(tmem, TMEM_COLS);
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives on, with the product kernel's wait code and a caller-given limit, and
// reports the expiry through the status word exactly as the product does.
__global__ void wait_probe_kernel(unsigned* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(b, 0, limit_ns)) atomicOr(status, 2u);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// count == 0: 2-D map over one npad x npad array; count > 0: 3-D map over
// count stacked slabs.
bool make_map(CUtensorMap* m, void* base, int64_t npad, int64_t ld, uint32_t box_rows, int count, int fp16) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)npad, (cuuint64_t)npad, (cuuint64_t)(count > 0 ? count : 1)};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)npad * (cuuint64_t)ld * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, count > 0 ? 3 : 2,
             base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// MN-major B over a row-major array: dims (32 columns of a strip, K rows,
// strips[, slabs]), so that one box {32, 32, strips} is the stage's strips of
// 32 columns x 32 K rows, one after the other (64B swizzle in each).
bool make_map_mn(CUtensorMap* m, void* base, int64_t npad, int64_t ld, uint32_t strips, int count, int fp16) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[4] = {32, (cuuint64_t)npad, (cuuint64_t)(npad / 32), (cuuint64_t)(count > 0 ? count : 1)};
  cuuint64_t strides[3] = {(cuuint64_t)ld * 2, 64, (cuuint64_t)npad * (cuuint64_t)ld * 2};
  cuuint32_t box[4] = {32, (cuuint32_t)BK, strips, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, count > 0 ? 4 : 3,
             base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc_uses_pair(int64_t npad, int count) { return count == 0 && npad >= kPairMinN; }

bool tc_make_maps(TcMaps* m, void* a_hi, void* a_lo, void* bt_hi, void* bt_lo, int64_t npad, int64_t ld,
                  int count, int fp16, int pair_mode, int group, int precise, int b_mn) {
  if (npad % BN != 0 || ld < npad || (ld * 2) % 16 != 0 || group < 1) return false;
  m->fp16 = fp16;
  m->precise = precise && count == 0;
  m->sym = nullptr;  // set by the caller for a symmetric product on pairs
  m->nsym = 0;
  m->pair = count == 0 && (m->precise || (pair_mode < 0 ? tc_uses_pair(npad, count) : pair_mode > 0));
  m->group = group;
  const uint32_t brows = m->precise ? PQ_BROWS : m->pair ? BN / 2 : BN;
  m->b_mn = b_mn;
  if (!make_map(&m->a_hi, a_hi, npad, ld, BM, count, fp16) || !make_map(&m->a_lo, a_lo, npad, ld, BM, count, fp16))
    return false;
  if (b_mn)
    return make_map_mn(&m->b_hi, bt_hi, npad, ld, brows / 32, count, fp16) &&
           make_map_mn(&m->b_lo, bt_lo, npad, ld, brows / 32, count, fp16);
  return make_map(&m->b_hi, bt_hi, npad, ld, brows, count, fp16) &&
         make_map(&m->b_lo, bt_lo, npad, ld, brows, count, fp16);
}

cudaError_t launch_wait_probe(unsigned* status, uint64_t limit_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 1, 0, s>>>(status, limit_ns);
  return cudaGetLastError();
}

namespace {

cudaError_t set_smem_attributes() {
  static std::atomic<int> state[kMaxDevices];
  return once_per_device(state, [] {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e[6] = {
        cudaFuncSetAttribute(tc_split_gemm_kernel<false, false, false>, a, (int)EpiShape<false, false>::kSmem),
        cudaFuncSetAttribute(tc_split_gemm_kernel<false, true, false>, a, (int)EpiShape<false, false>::kSmem),
        cudaFuncSetAttribute(tc_split_gemm_kernel<true, false, false>, a, (int)EpiShape<true, false>::kSmem),
        cudaFuncSetAttribute(tc_split_gemm_kernel<true, true, false>, a, (int)EpiShape<true, false>::kSmem),
        cudaFuncSetAttribute(tc_split_gemm_kernel<false, false, true>, a, (int)EpiShape<false, true>::kSmem),
        cudaFuncSetAttribute(tc_split_gemm_kernel<false, true, true>, a, (int)EpiShape<false, true>::kSmem)};
    for (cudaError_t x : e)
      if (x != cudaSuccess) return x;
    return cudaSuccess;
  });
}

// Clusters of the kernel that can be resident at once on the current device.
template <typename K>
int resident_clusters(K k, cudaLaunchConfig_t cfg, std::atomic<int> (&cache)[kMaxDevices]) {
  return per_device_value(cache, [&] {
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return nc;
  });
}

// One product on CTA pairs: as many 2-CTA clusters as can be resident at once
// (one CTA per SM), each walking the 256 x 256 tiles.
template <bool kF16>
cudaError_t launch_pair(const TcMaps& maps, int64_t npad, const EpiParams& P, cudaStream_t s) {
  using Sh = EpiShape<false, true>;
  auto k = tc_split_gemm_kernel<false, kF16, true>;
  const int tiles_m = (int)(npad / Sh::kTileM), tiles_n = (int)(npad / BN);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(Sh::kThreads);
  cfg.dynamicSmemBytes = Sh::kSmem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  static std::atomic<int> cache[kMaxDevices];
  cfg.gridDim = dim3(2 * tiles_m * tiles_n);
  const int max_pairs = resident_clusters(k, cfg, cache);
  if (max_pairs <= 0) return cudaErrorInvalidConfiguration;
  const int work = maps.sym ? maps.nsym : tiles_m * tiles_n;
  const int pairs = work < max_pairs ? work : max_pairs;
  cfg.gridDim = dim3(2 * pairs);
  return cudaLaunchKernelEx(&cfg, k, maps.a_hi, maps.a_lo, maps.b_hi, maps.b_lo, (int)(npad / BK), tiles_m, tiles_n,
                            maps.group, (const int4*)nullptr, maps.nsym, maps.sym, maps.b_mn, P);
}

template <bool kF16>
cudaError_t launch_precise(const TcMaps& maps, int64_t npad, const EpiParams& P, cudaStream_t s) {
  auto k = tc_precise_kernel<kF16>;
  static std::atomic<int> attr_state[kMaxDevices];
  const cudaError_t attr_err = once_per_device(
      attr_state, [&] { return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PQ_SMEM); });
  if (attr_err != cudaSuccess) return attr_err;
  const int tiles_m = (int)(npad / (2 * BM)), tiles_n = (int)(npad / PQ_N);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(PQ_THREADS);
  cfg.dynamicSmemBytes = PQ_SMEM;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  static std::atomic<int> cache[kMaxDevices];
  cfg.gridDim = dim3(2 * tiles_m * tiles_n);
  const int max_pairs = resident_clusters(k, cfg, cache);
  if (max_pairs <= 0) return cudaErrorInvalidConfiguration;
  const int pairs = tiles_m * tiles_n < max_pairs ? tiles_m * tiles_n : max_pairs;
  cfg.gridDim = dim3(2 * pairs);
  return cudaLaunchKernelEx(&cfg, k, maps.a_hi, maps.a_lo, maps.b_hi, maps.b_lo, (int)(npad / BK), tiles_m, tiles_n,
                            maps.group, maps.b_mn, P);
}

}  // namespace

cudaError_t launch_tc_gemm(const TcMaps& maps, int64_t npad, const EpiParams& P, cudaStream_t s,
                           const int4* tiles, int ntiles) {
  if (npad % BN != 0) return cudaErrorInvalidValue;
  cudaError_t attr_err = set_smem_attributes();
  if (attr_err != cudaSuccess) return attr_err;
  const int sms = sm_count();
  if (tiles) {
    if (ntiles <= 0) return cudaSuccess;
    const int grid = ntiles < sms ? ntiles : sms;
    auto k = maps.fp16 ? tc_split_gemm_kernel<true, true, false> : tc_split_gemm_kernel<true, false, false>;
    k<<<grid, EpiShape<true, false>::kThreads, EpiShape<true, false>::kSmem, s>>>(
        maps.a_hi, maps.a_lo, maps.b_hi, maps.b_lo, 0, 0, 0, 1, tiles, ntiles, (const int2*)nullptr, maps.b_mn, P);
    return cudaGetLastError();
  }
  if (maps.precise)
    return maps.fp16 ? launch_precise<true>(maps, npad, P, s) : launch_precise<false>(maps, npad, P, s);
  if (maps.pair) return maps.fp16 ? launch_pair<true>(maps, npad, P, s) : launch_pair<false>(maps, npad, P, s);
  const int tiles_m = (int)(npad / BM), tiles_n = (int)(npad / BN);
  const int grid = tiles_m * tiles_n < sms ? tiles_m * tiles_n : sms;
  auto k = maps.fp16 ? tc_split_gemm_kernel<false, true, false> : tc_split_gemm_kernel<false, false, false>;
  k<<<grid, EpiShape<false, false>::kThreads, EpiShape<false, false>::kSmem, s>>>(
      maps.a_hi, maps.a_lo, maps.b_hi, maps.b_lo, (int)(npad / BK), tiles_m, tiles_n, maps.group, nullptr, 0,
      (const int2*)nullptr, maps.b_mn, P);
  return cudaGetLastError();
}

}  // namespace neumann
