// The split-BF16 product engine on the 5th-generation tensor cores
// (tcgen05.mma, operands staged by TMA, accumulators in tensor memory).
//
// Computes, for one OzGemm (see ozaki.h),
//   C[i, j] (op)= 2^(ea_i + eb_j) sum_{p+q<=9} 2^(-7(p+q)) sum_k A_p[i][k] B_q[j][k]
// with the same exactness argument as the rest of the split path: a BF16
// product of two 7-bit digits is an integer below 2^14, so an FP32 sum of
// at most 1024 of them (one "chunk") is exact.
//
// CTA tile 128 x 128 of C for one K slice; 18 warps (at most 96 registers a
// thread, so that five warps fit one SM sub-partition's register file):
//   warp 0      TMA producer: for every digit pair (p, q) and every 128-wide
//               K stage, loads the 128 x 128 tiles of A_p and B_q (two
//               128-byte-swizzle atoms of 64 K each) into a 3-deep
//               shared-memory ring;
//   warp 1      allocates the 512 tensor-memory columns, and one thread
//               issues the MMAs (M = 128, N = 128, K = 16; eight per stage)
//               into one of two FP32 accumulators (columns 0-127, 128-255):
//               one accumulator per chunk (at most 1024 K terms of one
//               level: one pair's K range, or several same-level pairs when
//               a pair's K is at most 512), so chunk c + 1 runs while chunk
//               c is drained;
//   warps 2-17  drain each finished chunk: four warps per TMEM lane quarter
//               (32 rows of C), each owning 32 columns in two pieces of 16,
//               one row per thread.  FP32 -> exact int32 -> times
//               2^(7 (s_g - s)) -> added into a 64-bit integer sum kept in
//               tensor memory (columns 256-383 low words, 384-511 high
//               words), one group of levels at a time:
//                 group 1 = levels 2..5 (s_g = 5), group 2 = levels 6..9
//                 (s_g = 9): G = sum over the group's pairs and chunks of
//                 2^(7 (s_g - s)) * chunk sum.
//               Integer addition is exact, so the order of pairs and chunks
//               is free; with L_s <= (s - 1) K 127^2 both groups stay below
//               2^58 for any K <= 2^20.  Store mode: group 1 leaves its raw
//               sum G1 in C, group 2 forms the exact 128-bit G1 2^28 + G2
//               and rounds it once to FP64 with the scale 2^(ea + eb - 63)
//               (C = v).  Subtract mode: each group is rounded once, scaled
//               by 2^(ea + eb - 7 s_g) and subtracted (C = C - v).  The
//               rounding is done on the integer pipe (rne_f64).
// Work order inside a CTA: group, then 1024-term K chunk, then the group's
// pairs (level order), then the chunk's 128-wide K stages, so that the digit
// planes of one chunk are reused by every pair of the group while they are
// hot in L2.  CTA order: the column tiles of one row block are consecutive
// (they share the row block's A planes), K slices outermost.
// Pipelines are tied by mbarriers: full/empty per stage, full/empty per
// accumulator.  Every wait is bounded (2 s of wall time); on expiry the
// thread records CQRRPT_TIMEOUT in *G.err, the roles stop issuing work, the
// MMA thread waits (bounded) for its MMAs, the producer for its copies, and
// the tensor memory is released before the CTA exits; CTAs that start after
// the status word is set return at once.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "ozaki.h"

namespace cqrrpt {

namespace {

constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 128, kTcStages = 3;
constexpr int kTcAtomK = 64;                                // K of one 128-byte swizzle atom
constexpr int kTcAtomBytes = kTcBM * kTcAtomK * 2;          // 16 KB: 128 rows x 64 K
constexpr int kTcTileBytes = kTcBM * kTcBK * 2;             // 32 KB, one operand tile
constexpr int kTcStageBytes = 2 * kTcTileBytes;             // A + B
constexpr int kTcChunkStages = kOzChunk / kTcBK;            // 8 stages = 1024 K terms
constexpr int kTcDrainWarps = 16;                          // 4 per TMEM lane quarter
constexpr int kTcThreads = 32 * (2 + kTcDrainWarps);        // 18 warps: <= 96 registers
constexpr int kTcAccBufs = 2;                               // FP32 accumulators in TMEM
constexpr int kTcEmitCols = 8;                              // columns per batch of C loads
constexpr uint32_t kTcTmemCols = 512;
constexpr uint32_t kTcGroupLo = kTcAccBufs * kTcBN;         // 256: low words of the sums
constexpr uint32_t kTcGroupHi = kTcGroupLo + kTcBN;         // 384: high words
constexpr int kTcBarriers = 2 * kTcStages + 2 * kTcAccBufs + 1;  // full, empty, acc full/empty, done
constexpr size_t kTcSmem = 1024 /* alignment slack */ + (size_t)kTcStages * kTcStageBytes +
                           kTcBarriers * 8 + 16 + kTcBN * 4 /* column exponents */;

// first pair index of each group of levels (2..5, 6..9), and the end
__constant__ int kTcGroupFirst[3] = {0, 10, 36};
// level order of the 36 digit pairs
__constant__ unsigned char kTcPairP[kOzPairs] = {1, 1, 2, 1, 2, 3, 1, 2, 3, 4, 1, 2,
                                                 3, 4, 5, 1, 2, 3, 4, 5, 6, 1, 2, 3,
                                                 4, 5, 6, 7, 1, 2, 3, 4, 5, 6, 7, 8};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of parity `parity` to complete: gives up after
// limit_ns of wall time (kTcWaitNs by default; a pipeline step of this
// kernel takes microseconds) or kSpinLimit polls, whichever comes first.
// A limit below the default (set by cqrrpt_set_wait_limits, a test hook of
// the timeout path) polls without blocking and reads the clock every poll,
// so that a phase that is not already complete runs the limit out.
// g_tc_wait_ns bounds the pipeline's own waits; the waits of the clean-up
// after a timeout (copies and products in flight) always take kTcWaitNs.
constexpr unsigned long long kTcWaitNs = 2000000000ull;
__device__ unsigned long long g_tc_wait_ns = kTcWaitNs;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long limit_ns = kTcWaitNs) {
  const unsigned long long t0 = global_ns();
  if (limit_ns < kTcWaitNs) {
    for (unsigned long long i = 0; i < kSpinLimit; ++i) {
      if (mbar_test_wait(bar, parity)) return true;
      if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
  }
  for (unsigned long long i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y, int z, int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(bar), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 64 BF16 (128 B), 8-row core groups 1024 B apart
// (stride byte offset), leading byte offset unused (1), descriptor version 1,
// layout type 2 = 128-byte swizzle.  The tile base is 1024-byte aligned.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcBN >> 3) << 17) |
                              ((uint32_t)(kTcBM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(kTcIdesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

#define OZ_R16(r)                                                                          \
  "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),     \
      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), \
      "=r"(r[14]), "=r"(r[15])
#define OZ_W16(r)                                                                           \
  "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),  \
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),     \
      "r"(r[15])

// 16 consecutive 32-bit columns of the thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : OZ_R16(r)
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      OZ_W16(r)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// S * 2^e rounded to the nearest double (ties to even), S = hi:lo a signed
// 128-bit integer, by integer operations on the IEEE 754 binary64 encoding:
// normalise |S| so that its leading one is bit 127, keep 53 bits, round on
// the next bit and the sticky rest, and write the exponent field directly
// (the scale 2^e costs nothing).  Results outside the normal range go
// through ldexp of the rounded 53-bit value.
__device__ __forceinline__ double rne_f64(long long hi, unsigned long long lo, int e) {
  const bool neg = hi < 0;
  unsigned long long mh = (unsigned long long)hi, ml = lo;
  if (neg) {  // two's complement negation of the 128-bit value
    ml = ~ml + 1ull;
    mh = ~mh + (ml == 0ull ? 1ull : 0ull);
  }
  if ((mh | ml) == 0ull) return 0.0;
  const int nb = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);  // bits of |S|
  const int L = 128 - nb;  // left shift that puts the leading one at bit 127
  unsigned long long nh, nl;
  if (L >= 64) {
    nh = ml << (L - 64);
    nl = 0ull;
  } else if (L > 0) {
    nh = (mh << L) | (ml >> (64 - L));
    nl = ml << L;
  } else {
    nh = mh;
    nl = ml;
  }
  unsigned long long mant = nh >> 11;  // 53 bits, leading one at bit 52
  const bool rb = (nh >> 10) & 1ull;
  const bool sticky = (nh & 0x3FFull) != 0ull || nl != 0ull;
  if (rb && (sticky || (mant & 1ull))) ++mant;
  int E = nb - 1 + e;  // exponent of the leading bit
  if (mant >> 53) {
    mant >>= 1;
    ++E;
  }
  if (E >= -1022 && E <= 1023) {
    const unsigned long long bits = ((unsigned long long)neg << 63) |
                                    ((unsigned long long)(E + 1023) << 52) |
                                    (mant & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
  }
  const double m = ldexp((double)mant, E - 52);
  return neg ? -m : m;
}

__device__ __forceinline__ void record_timeout(int* err) {
  if (err) atomicExch(err, kTimeout);
}

// One CTA's tile of one product.  tmA, tmB: the product's TMA maps (kernel
// parameters of a single launch, or device memory for a batched launch).
__device__ __forceinline__ void oz_tc_body(const CUtensorMap* tmA, const CUtensorMap* tmB,
                                           const OzGemm& G, int64_t tile,
                                           unsigned char* tc_smem_raw) {
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 128-byte swizzle tiles: 1024-aligned
  const uint32_t a_tiles = base;
  const uint32_t b_tiles = base + kTcStages * kTcTileBytes;
  const uint32_t bars = base + kTcStages * kTcStageBytes;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (kTcStages + s); };
  auto accf_bar = [&](int b) { return bars + 8u * (2 * kTcStages + b); };
  auto acce_bar = [&](int b) { return bars + 8u * (2 * kTcStages + kTcAccBufs + b); };
  const uint32_t done_bar = bars + 8u * (2 * kTcStages + 2 * kTcAccBufs);
  uint32_t* tmem_slot = (uint32_t*)(tc_smem_raw + (bars - raw) + 8u * kTcBarriers);
  int* eb_s = (int*)(tc_smem_raw + (bars - raw) + 8u * kTcBarriers + 16u);  // eb of the tile

  // tile of this CTA
  const int64_t tiles_m = (G.M + kTcBM - 1) / kTcBM;
  const int64_t tiles_n = (G.N + kTcBN - 1) / kTcBN;
  const int64_t tn = tile % tiles_n, tm = (tile / tiles_n) % tiles_m;
  const int64_t ks = tile / (tiles_m * tiles_n);
  const int64_t m0 = tm * kTcBM;
  const int n0 = (int)(tn * kTcBN);
  if (G.upper_only && m0 >= n0 + kTcBN) return;  // uniform: before any barrier
  const int64_t kbeg = ks * G.kslice;
  const int64_t kend = min64(kbeg + G.kslice, G.Kpad);
  if (kbeg >= kend) return;
  // an earlier failure (of this launch or a previous step): nothing to do
  if (G.err && *(volatile const int*)G.err != kOk) return;
  const int nk = (int)((kend - kbeg + kTcBK - 1) / kTcBK);  // K stages per pair
  const int nchunks = (nk + kTcChunkStages - 1) / kTcChunkStages;
  // pairs of one level that share an FP32 accumulator: up to 1024 terms in
  // all (when one pair's K fits a chunk several same-level pairs do)
  const int run = nchunks == 1 ? max(1, kTcChunkStages / nk) : 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long wait_ns = g_tc_wait_ns;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < kTcAccBufs; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), kTcDrainWarps);  // one arrival per drain warp
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x >= 64 && threadIdx.x < 64 + kTcBN) {
    const int col = n0 + (int)threadIdx.x - 64;
    eb_s[threadIdx.x - 64] = col < G.N ? G.eb[col] : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- producer
    // blocked operands: power-of-two block extents (shift, mask); an
    // unblocked operand is one block (shift 62: block 0, x = kx)
    const int ash = G.a_kblk > 0 && G.a_kblk < G.Kpad ? __ffsll(G.a_kblk) - 1 : 62;
    const int bsh = G.b_kblk > 0 && G.b_kblk < G.Kpad ? __ffsll(G.b_kblk) - 1 : 62;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    int issued = 0;
    for (int grp = 0; grp < 2 && ok; ++grp)
    for (int c = 0; c < nchunks && ok; ++c)
    for (int pi = kTcGroupFirst[grp]; pi < kTcGroupFirst[grp + 1] && ok; ++pi) {
      const int p = kTcPairP[pi];
      int s = 2;
      while ((s - 1) * s / 2 <= pi) ++s;
      const int q = s - p;
      const int kst_end = min(nk, (c + 1) * kTcChunkStages);
      for (int kst = c * kTcChunkStages; kst < kst_end; ++kst) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, wait_ns)) {
          record_timeout(G.err);
          ok = false;
          break;
        }
        mbar_expect_tx(full_bar(stage), kTcStageBytes);
        const int64_t kx = kbeg + (int64_t)kst * kTcBK;
        // (K within the block, block) of each operand: a stage never
        // straddles a block (block extents are multiples of kTcBK)
        const int xa = (int)(kx & ((1ll << ash) - 1)), ba = (int)(kx >> ash);
        const int xb = (int)(kx & ((1ll << bsh) - 1)), bb = (int)(kx >> bsh);
#pragma unroll
        for (int at = 0; at < kTcBK / kTcAtomK; ++at) {  // one swizzle atom per copy
          tma_load_4d(a_tiles + stage * kTcTileBytes + at * kTcAtomBytes, tmA, full_bar(stage),
                      xa + at * kTcAtomK, (int)m0, ba, p - 1);
          tma_load_4d(b_tiles + stage * kTcTileBytes + at * kTcAtomBytes, tmB, full_bar(stage),
                      xb + at * kTcAtomK, n0, bb, q - 1);
        }
        ++issued;
        if (++stage == kTcStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (!ok) {
      // copies still in flight land before the CTA exits: wait for the
      // full barrier of each of the last (up to kTcStages) issued loads
      int st = stage;
      uint32_t ph = phase;
      for (int i = 0; i < kTcStages && i < issued; ++i) {
        if (--st < 0) {
          st = kTcStages - 1;
          ph ^= 1u;
        }
        mbar_wait(full_bar(st), ph);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    int stage = 0;
    uint32_t phase = 0;
    uint32_t use = 0u;  // bit b: parity of accumulator b's next use
    int buf = 0;
    bool ok = true;
    bool any = false;
    for (int grp = 0; grp < 2 && ok; ++grp)
    for (int c = 0; c < nchunks && ok; ++c) {
      for (int pi = kTcGroupFirst[grp]; pi < kTcGroupFirst[grp + 1] && ok;) {
        int s = 2;
        while ((s - 1) * s / 2 <= pi) ++s;
        const int run_end = min(pi + run, (s - 1) * s / 2);  // same level only
        if (!mbar_wait(acce_bar(buf), ((use >> buf) & 1u) ^ 1u, wait_ns)) {
          record_timeout(G.err);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kTcBN);
        const int st_n = min(kTcChunkStages, nk - c * kTcChunkStages);
        for (int pr = pi; pr < run_end && ok; ++pr) {
          for (int j = 0; j < st_n; ++j) {
            if (!mbar_wait(full_bar(stage), phase, wait_ns)) {
              record_timeout(G.err);
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int at = 0; at < kTcBK / kTcAtomK; ++at) {
              const uint64_t ad = sw128_desc(a_tiles + stage * kTcTileBytes + at * kTcAtomBytes);
              const uint64_t bd = sw128_desc(b_tiles + stage * kTcTileBytes + at * kTcAtomBytes);
#pragma unroll
              for (int kk = 0; kk < kTcAtomK / 16; ++kk)  // K = 16 per MMA: +32 bytes
                umma_bf16(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2),
                          (pr > pi || j > 0 || at > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit(empty_bar(stage));
            any = true;
            if (++stage == kTcStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
        umma_commit(accf_bar(buf));
        use ^= 1u << buf;
        buf = (buf + 1) % kTcAccBufs;
        pi = run_end;
      }
    }
    // every MMA issued by this thread has completed before the TMEM goes
    if (any) {
      umma_commit(done_bar);
      if (!mbar_wait(done_bar, 0)) record_timeout(G.err);
    }
  } else if (warp >= 2) {
    // ---- drain: 4 warps per TMEM lane quarter (32 rows), each owning 32
    // of the tile's 128 columns (two pieces of 16), one row per thread
    const int quarter = warp & 3;
    const int cslice = (warp - 2) >> 2;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cslice * 32);
    const int64_t row = m0 + quarter * 32 + lane;
    const bool row_ok = row < G.M;
    const int ea = row_ok ? G.ea[row] : 0;
    double* Cbase = G.C + ks * G.c_slice + (row_ok ? row : 0);
    uint32_t fph = 0u;  // bit b: parity of accumulator b's next completion
    int buf = 0;
    bool ok = true;
    for (int grp = 0; grp < 2 && ok; ++grp)
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s_g = grp == 0 ? 5 : 9;  // last level of the group
      for (int pi = kTcGroupFirst[grp]; pi < kTcGroupFirst[grp + 1];) {
        int s = 2;
        while ((s - 1) * s / 2 <= pi) ++s;
        const int run_end = min(pi + run, (s - 1) * s / 2);  // same level only
        if (!mbar_wait(accf_bar(buf), (fph >> buf) & 1u, wait_ns)) {
          record_timeout(G.err);
          ok = false;
          break;
        }
        fph ^= 1u << buf;
        tc_fence_after();
        const bool fresh = c == 0 && pi == kTcGroupFirst[grp];
        const bool emit = c == nchunks - 1 && run_end == kTcGroupFirst[grp + 1];
        const int weight = 1 << (7 * (s_g - s));
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          uint32_t fa[16], lo[16], hi[16];
          tmem_ld16(lane_addr + (uint32_t)(buf * kTcBN + h * 16), fa);
          if (!fresh) {
            tmem_ld16(lane_addr + kTcGroupLo + (uint32_t)(h * 16), lo);
            tmem_ld16(lane_addr + kTcGroupHi + (uint32_t)(h * 16), hi);
          }
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            long long g = fresh ? 0ll
                                : (long long)(((unsigned long long)hi[i] << 32) |
                                              (unsigned long long)lo[i]);
            // exact: |chunk| < 2^24, |g| < 2^58
            g += (long long)__float2int_rn(__uint_as_float(fa[i])) * weight;
            lo[i] = (uint32_t)((unsigned long long)g & 0xFFFFFFFFull);
            hi[i] = (uint32_t)((unsigned long long)g >> 32);
          }
          if (emit) {
            // the group is complete.  Store mode: group 1 leaves its raw
            // 64-bit sum in C; group 2 reads it back and rounds the exact
            // 128-bit G1 2^28 + G2 once.  Subtract mode: each group is
            // rounded once and subtracted from C.  Integer pipe only, except
            // the subtraction (FP64 is scarce on this part).
            if (row_ok) {
#pragma unroll
              for (int e8 = 0; e8 < 16; e8 += kTcEmitCols) {
                const int c0 = cslice * 32 + h * 16 + e8;  // column within the tile
                double old[kTcEmitCols];
                const bool stash = G.mode == kOzStore && grp == 0;
                if (!stash) {
#pragma unroll
                  for (int i = 0; i < kTcEmitCols; ++i)
                    old[i] = n0 + c0 + i < G.N ? Cbase[(int64_t)(n0 + c0 + i) * G.ldc] : 0.0;
                }
#pragma unroll
                for (int i = 0; i < kTcEmitCols; ++i) {
                  if (n0 + c0 + i >= G.N) continue;
                  const long long g = (long long)(((unsigned long long)hi[e8 + i] << 32) |
                                                  (unsigned long long)lo[e8 + i]);
                  const int e = ea + eb_s[c0 + i] - 7 * s_g;
                  double r;
                  if (stash) {
                    r = __longlong_as_double(g);
                  } else if (G.mode == kOzStore) {
                    // S = G1 2^(7 (9 - 5)) + G2 as a 128-bit integer
                    const long long g1 = __double_as_longlong(old[i]);
                    const unsigned long long l1 = (unsigned long long)g1 << 28;
                    const unsigned long long l = l1 + (unsigned long long)g;
                    const long long hh = (g1 >> 36) + (g >> 63) + (l < l1 ? 1 : 0);
                    r = rne_f64(hh, l, e);
                  } else {
                    r = __dsub_rn(old[i], rne_f64(g >> 63, (unsigned long long)g, e));
                  }
                  Cbase[(int64_t)(n0 + c0 + i) * G.ldc] = r;
                }
              }
            }
          } else {
            tmem_st16(lane_addr + kTcGroupLo + (uint32_t)(h * 16), lo);
            tmem_st16(lane_addr + kTcGroupHi + (uint32_t)(h * 16), hi);
          }
        }
        if (!emit) tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce_bar(buf));
        buf = (buf + 1) % kTcAccBufs;
        pi = run_end;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTcTmemCols)
                 : "memory");
  }
}

__global__ void __maxnreg__(96)
    oz_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 OzGemm G) {
  extern __shared__ unsigned char tc_smem_raw[];
  oz_tc_body(&tmA, &tmB, G, blockIdx.x, tc_smem_raw);
}

// CTA b -> (job, tile) through the prefix table; maps[2 j], maps[2 j + 1]
// are job j's A and B maps.
__global__ void __maxnreg__(96)
    oz_tc_batched_kernel(const OzGemm* __restrict__ jobs, const CUtensorMap* __restrict__ maps,
                         const int64_t* __restrict__ base, int njobs) {
  extern __shared__ unsigned char tc_smem_raw[];
  int64_t t;
  const int j = find_problem(base, njobs, blockIdx.x, &t);
  oz_tc_body(maps + 2 * j, maps + 2 * j + 1, jobs[j], t, tc_smem_raw);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 4-D map over digit planes [8][kpad / kblk][rows][kblk] (BF16): K within
// the block, row, block, plane; box 64 (K) x 128 rows x 1 x 1, 128-byte
// swizzle, zero fill outside.  Unblocked planes [8][rows][kpad] are the
// case kblk = kpad (one block).
bool plane_map(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t kpad,
               int64_t kblk, int64_t plane) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  if (kblk <= 0) kblk = kpad;
  const cuuint64_t dims[4] = {(cuuint64_t)kblk, (cuuint64_t)rows, (cuuint64_t)(kpad / kblk),
                              (cuuint64_t)kOzDigits};
  const cuuint64_t strides[3] = {(cuuint64_t)kblk * 2, (cuuint64_t)(rows * kblk) * 2,
                                 (cuuint64_t)plane * 2};
  const cuuint32_t box[4] = {(cuuint32_t)kTcAtomK, (cuuint32_t)kTcBM, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Test hook of the timeout path (cqrrpt_set_wait_limits): bound of the
// engine's pipeline waits on the current device; 0 restores kTcWaitNs.
cudaError_t oz_set_wait_ns(unsigned long long ns) {
  const unsigned long long v = ns ? ns : kTcWaitNs;
  return cudaMemcpyToSymbol(g_tc_wait_ns, &v, sizeof(v));
}

static cudaError_t tc_attributes() {
  cudaError_t e = raise_smem_limit((const void*)oz_tc_kernel, (size_t)kTcSmem);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)oz_tc_batched_kernel, (size_t)kTcSmem);
  return e;
}

// TMA: 16-byte aligned bases, row strides and plane strides (several K
// slices: slice boundaries on stage boundaries; one slice may end
// mid-stage, TMA fills zeros past Kpad).  Blocked planes: power-of-two
// blocks of a whole number of stages that tile Kpad, slices on block
// boundaries.
static bool kblk_valid(int64_t kb, const OzGemm& G) {
  if (kb <= 0 || kb >= G.Kpad) return kb <= G.Kpad;
  return (kb & (kb - 1)) == 0 && kb % kTcBK == 0 && G.Kpad % kb == 0 && G.kslice % kb == 0;
}
bool oz_gemm_valid(const OzGemm& G) {
  const bool sliced = G.kslice < G.Kpad;
  return !(((uintptr_t)G.A & 15) || ((uintptr_t)G.B & 15) || (G.Kpad % 8) || (G.a_plane % 8) ||
           (G.b_plane % 8) || G.kslice <= 0 || (sliced && (G.kslice % kTcBK)) ||
           !kblk_valid(G.a_kblk, G) || !kblk_valid(G.b_kblk, G));
}

int64_t oz_gemm_tiles(const OzGemm& G) {
  const int64_t tiles_m = (G.M + kTcBM - 1) / kTcBM;
  const int64_t tiles_n = (G.N + kTcBN - 1) / kTcBN;
  const int64_t nks = (G.Kpad + G.kslice - 1) / G.kslice;
  return tiles_m * tiles_n * nks;
}

bool oz_gemm_encode_maps(const OzGemm& G, void* maps_host) {
  static_assert(sizeof(CUtensorMap) == kOzMapBytes, "tensor map size");
  CUtensorMap* m = (CUtensorMap*)maps_host;
  return plane_map(&m[0], G.A, G.M, G.Kpad, G.a_kblk, G.a_plane) &&
         plane_map(&m[1], G.B, G.N, G.Kpad, G.b_kblk, G.b_plane);
}

cudaError_t oz_gemm_tc_launch(const OzGemm& G, cudaStream_t s) {
  cudaError_t e = tc_attributes();
  if (e != cudaSuccess) return e;
  if (!oz_gemm_valid(G)) return cudaErrorInvalidValue;
  alignas(64) CUtensorMap mp[2];
  if (!oz_gemm_encode_maps(G, mp)) return cudaErrorInvalidValue;
  oz_tc_kernel<<<(unsigned)oz_gemm_tiles(G), kTcThreads, kTcSmem, s>>>(mp[0], mp[1], G);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t oz_gemm_tc_batched_launch(const OzGemm* jobs, const void* maps, const int64_t* base,
                                      int njobs, int64_t total_tiles, cudaStream_t s) {
  if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
  cudaError_t e = tc_attributes();
  if (e != cudaSuccess) return e;
  if ((uintptr_t)maps & 63) return cudaErrorInvalidValue;
  oz_tc_batched_kernel<<<(unsigned)total_tiles, kTcThreads, kTcSmem, s>>>(
      jobs, (const CUtensorMap*)maps, base, njobs);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
