// Sketch GEMMs of the Nystrom preconditioner (App. B: Y = H Omega with H = A^T D A) on
// the 5th-generation tensor cores, for BF16 storage of A:
//
//   W  = diag(D) A Omega        (n x s)   GEMM 1: M = n (rows of A), N = s, K = d
//   Y  = A^T W                  (d x s)   GEMM 2: M = d, N = s, K = n (split over K)
//
// The test matrix Omega of an FP32-class sketch holds BF16 values (the orthonormal factor
// rounded once; the rest of the Nystrom core uses that same Omega), so GEMM 1 is a plain
// BF16 x BF16 product.  W is FP32 and is written as the sum of three BF16 terms (x = t1 +
// t2 + t3 holds exactly for every float x: each term takes the next 8 significant bits),
// and A is BF16 already, so every product a * t_k is exact and the tensor core accumulates
// them in FP32: GEMM 2 is an FP32-class GEMM at tensor-core rates (3 MMAs per K step).
//
// Kernel design (one CTA = two 128-row tiles of the output sharing each staged B tile, the
// full N = s <= 256 of each in TMEM):
//   * both operands are K-major: GEMM 1 reads the rows of A directly, GEMM 2 reads a
//     transposed copy of A made once per sketch (2 GB of the 280 GB HBM for the paper's
//     largest single-GPU problem); W is written by GEMM 1 already in the K-major layout
//     GEMM 2 wants;
//   * tiles are staged by cp.async (16-byte chunks, zero-filled outside the matrix) into
//     the canonical no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix;
//     core matrices 128 B apart along K, 512 B apart along M/N), 4 stages of 32 K;
//   * one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in TMEM, M = 128,
//     N = s rounded up to 16) and tcgen05.commit to the stage's mbarrier, which frees the
//     stage for the next cp.async; all waits are bounded;
//   * the epilogue reads TMEM with tcgen05.ld (warp w reads lanes 32 (w % 4) .. + 31):
//     GEMM 1 scales row i by D_i and writes the three BF16 terms of W; GEMM 2 writes its
//     K-slice's FP32 partial, and a final kernel sums the slices in a fixed order in FP64.
#include <cuda.h>   // CUtensorMap (the encode entry point is taken from the driver at run time)
#include <cuda_bf16.h>

#include "device_util.cuh"
#include "nys_internal.cuh"
#include "solver.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>

namespace nys {
namespace {

constexpr int TC_BM = 128;      // output rows per CTA = TMEM lanes
constexpr int TC_BK = 32;       // K per stage (two MMA K-steps of 16)
constexpr int TC_THREADS = 256;
constexpr int TC_TERMS = 3;     // FP32 operand = t1 + t2 + t3 (BF16)
constexpr int TC_NMAX = 256;    // MMA N limit; TMEM columns allocated
constexpr uint32_t TC_LBO = 128;                 // K-direction core-matrix stride (bytes)
constexpr uint32_t TC_SBO = (TC_BK / 8) * 128;   // 8-row-group stride (bytes)

struct TcArgs {
  const uint16_t* A;     // row-major [AT][Mrows][lda] BF16 terms, K contiguous
  int64_t lda, Mrows, Kvalid;
  int64_t aterm;         // element stride between the A terms (AT = 3)
  const uint16_t* B;     // [TERMS][NP][ldb] BF16, K contiguous, zero outside the data
  int64_t ldb, bterm;
  int NP;                // MMA N (multiple of 16, <= 256)
  int64_t ktiles;        // K tiles of TC_BK in the whole product
  int64_t kslice;        // K tiles per split-K slice (blockIdx.y)
  // epilogue 0: Wt[t][c][i] = BF16 terms of D_i * acc(i, c), rows i < wrows (zero for i >= Mrows)
  const double* D;
  uint16_t* Wt;
  int64_t ldw, wterm, wrows;
  // epilogue 1: P[z][c][j] = acc(j, c) (FP32, slice z = blockIdx.y)
  float* P;
  int64_t ldp;
  uint32_t desc_swap;    // 0: LBO along K, SBO along M/N (the canonical K-major form)
  int* status;
};

// ---- PTX wrappers (tcgen05, cp.async, proxy fences)
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, leading (K) and stride
// (M/N) byte offsets, all in 16-byte units; bits 46-48 hold the fixed value 1.  The
// swizzled form below sets the layout field (bits 61-63; 4 = 64-byte swizzle) and takes
// only the 8-row-group stride (the leading offset is unused there, encoded as 1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) |
         (4ull << 61);
}
__host__ __device__ constexpr uint32_t mma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 lanes x 8 columns of 32 bits: thread l of the warp gets lane (base + l), 8 columns.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr)
               : "memory");
}
// the registers are operands so that no use of them is scheduled before the wait
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
               :
               : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }
// x = t[0] + t[1] + t[2] (+ a remainder below 2^-24 |x|)
__device__ __forceinline__ void split3(float x, uint16_t (&t)[3]) {
  t[0] = bf16_bits(x);
  const float r1 = x - bf16_val(t[0]);
  t[1] = bf16_bits(r1);
  const float r2 = r1 - bf16_val(t[1]);
  t[2] = bf16_bits(r2);
}

// AT, BT = number of BF16 terms of the A and B operands: 1 (BF16 values) or 3 (FP32 values
// split exactly into three BF16 terms).  A K step issues the MMAs a_i x b_j with i + j <= 2
// (0-based): with AT = BT = 3 the three dropped products are below 2^-24 of the result.
template <int AT, int BT> constexpr int tc_npairs() { return AT == 3 && BT == 3 ? 6 : (AT == 1 && BT == 1 ? 1 : 3); }
// pair pr -> (A term, B term):
//   AT = 1: (0,0) (0,1) (0,2);  BT = 1: (0,0) (1,0) (2,0);
//   AT = BT = 3: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
template <int AT, int BT> __host__ __device__ constexpr int tc_pair_a(int pr) {
  return AT == 1 ? 0 : (BT == 1 ? pr : (pr == 2 || pr == 4 ? 1 : (pr == 5 ? 2 : 0)));
}
template <int AT, int BT> __host__ __device__ constexpr int tc_pair_b(int pr) {
  return BT == 1 ? 0 : (AT == 1 ? pr : (pr == 1 || pr == 4 ? 1 : (pr == 3 ? 2 : 0)));
}
// Bytes of one pipeline stage at the largest N: BM2 accumulators of 128 rows x AT terms of
// A, and BT terms of B.  Stages fill about 224 KB of shared memory, at most 6.
template <int AT, int BT, int BM2> constexpr int tc_stage_max_bytes() {
  return BM2 * AT * TC_BM * TC_BK * 2 + BT * TC_NMAX * TC_BK * 2;
}
template <int AT, int BT, int BM2> constexpr int tc_stages() {
  return (224 * 1024) / tc_stage_max_bytes<AT, BT, BM2>() < 6 ? (224 * 1024) / tc_stage_max_bytes<AT, BT, BM2>() : 6;
}

// Epilogue of both staging forms: TMEM -> registers (tcgen05.ld; warp w reads lanes
// 32 (w % 4) .. + 31 and half the columns), then W's three BF16 terms (EPI 0, rows scaled
// by D) or the split-K slice's FP32 partial (EPI 1).
template <int EPI, int BM2>
__device__ __forceinline__ void tc_epilogue(const TcArgs& a, uint32_t tmem, int64_t m0, int nkt, int warp, int lane) {
  const int quad = warp & 3;
  const int half = a.NP / 2;
  const int cb = (warp >> 2) * half;
  for (int h = 0; h < BM2; ++h) {
    const int64_t row = m0 + h * TC_BM + 32 * quad + lane;
    const uint32_t trow = tmem + (uint32_t)(h * TC_NMAX) + ((uint32_t)(32 * quad) << 16);
    double dr = 1.0;
    if (EPI == 0 && a.D && row < a.Mrows) dr = a.D[row];
    for (int c0 = cb; c0 < cb + half; c0 += 8) {
      uint32_t v[8];
      tmem_ld8(trow + (uint32_t)c0, v);
      tmem_ld_wait(v);
      if (nkt == 0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0u;
      }
      if (EPI == 0) {
        if (row < a.wrows) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float x = row < a.Mrows ? (float)(dr * (double)__uint_as_float(v[e])) : 0.f;
            uint16_t t3[3];
            split3(x, t3);
#pragma unroll
            for (int t = 0; t < TC_TERMS; ++t) a.Wt[t * a.wterm + (int64_t)(c0 + e) * a.ldw + row] = t3[t];
          }
        }
      } else {
        if (row < a.Mrows) {
          float* P = a.P + (int64_t)blockIdx.y * a.NP * a.ldp;
#pragma unroll
          for (int e = 0; e < 8; ++e) P[(int64_t)(c0 + e) * a.ldp + row] = __uint_as_float(v[e]);
        }
      }
    }
  }
}

// BM2 accumulators per CTA (1 or 2): a CTA computes BM2 x 128 output rows, every staged
// tile of B serving both (half the B traffic from L2 per output row); accumulator h sits
// at TMEM columns [256 h, 256 h + N).
template <int EPI, int AT, int BT, int BM2>
__global__ void __launch_bounds__(TC_THREADS, 1) sketch_tc_kernel(const TcArgs a) {
  constexpr int TC_STAGES = tc_stages<AT, BT, BM2>();
  constexpr uint32_t kTmemCols = BM2 == 2 ? 2 * TC_NMAX : TC_NMAX;
  static_assert(TC_STAGES >= 2, "shared memory holds fewer than two stages");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mma_bar[TC_STAGES];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * (TC_BM * BM2);
  const int64_t kt0 = (int64_t)blockIdx.y * a.kslice;
  const int64_t kt1 = min(a.ktiles, kt0 + a.kslice);
  const int nkt = (int)max((int64_t)0, kt1 - kt0);
  const uint32_t a_bytes = TC_BM * TC_BK * 2;
  const uint32_t b_bytes = (uint32_t)a.NP * TC_BK * 2;
  const uint32_t stage_bytes = BM2 * AT * a_bytes + BT * b_bytes;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t lbo = a.desc_swap ? TC_SBO : TC_LBO, sbo = a.desc_swap ? TC_LBO : TC_SBO;
  const uint32_t idesc = mma_idesc_bf16(TC_BM, a.NP);

  if (warp == 0) {
    tmem_alloc(&tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) mbar_init(&mma_bar[s], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // Stage layout: chunk q (16 bytes = 8 elements of one row) of a tile with 4 chunks per
  // row sits at byte 16 q, with q = 32 g + 8 c + r8 for row 8 g + r8 and K chunk c: that is
  // the core-matrix layout with LBO = 128 (along K) and SBO = 512 (along rows).
  auto load_stage = [&](int ktl, int stage) {
    const int64_t k0 = (kt0 + ktl) * TC_BK;
    const uint32_t st = sbase + (uint32_t)stage * stage_bytes;
    for (int q = tid; q < BM2 * AT * TC_BM * 4; q += TC_THREADS) {
      const int ht = q / (TC_BM * 4), qa = q - ht * (TC_BM * 4);   // ht = h * AT + ta
      const int h = ht / AT, ta = ht - h * AT;
      const int r8 = qa & 7, c = (qa >> 3) & 3, g = qa >> 5;
      const int64_t row = m0 + h * TC_BM + g * 8 + r8, k = k0 + c * 8;
      uint32_t bytes = 0;
      const uint16_t* src = a.A;
      if (row < a.Mrows && k < a.Kvalid) {
        bytes = (uint32_t)min((int64_t)16, (a.Kvalid - k) * 2);
        src = a.A + ta * a.aterm + row * a.lda + k;
      }
      cp_async16(st + (uint32_t)ht * a_bytes + (uint32_t)qa * 16u, src, bytes);
    }
    const int per_term = a.NP * 4;
    for (int q = tid; q < BT * per_term; q += TC_THREADS) {
      const int t = q / per_term, qq = q - t * per_term;
      const int r8 = qq & 7, c = (qq >> 3) & 3, g = qq >> 5;
      const uint16_t* src = a.B + t * a.bterm + (int64_t)(g * 8 + r8) * a.ldb + k0 + c * 8;
      cp_async16(st + BM2 * AT * a_bytes + (uint32_t)t * b_bytes + (uint32_t)qq * 16u, src, 16u);
    }
  };

  bool ok = true;
  for (int s = 0; s < TC_STAGES - 1; ++s) {
    if (s < nkt) load_stage(s, s);
    cp_async_commit();
  }
  for (int kt = 0; kt < nkt; ++kt) {
    const int stage = kt % TC_STAGES;
    cp_async_wait<TC_STAGES - 2>();  // this thread's copies of k-tile kt have landed
    fence_proxy_async_smem();        // make them visible to the tensor core (async proxy)
    ok = __syncthreads_and(ok);
    if (tid == 0 && ok) {
      tc_fence_after();
      const uint32_t st = sbase + (uint32_t)stage * stage_bytes;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
        for (int h = 0; h < BM2; ++h) {
#pragma unroll
          for (int pr = 0; pr < tc_npairs<AT, BT>(); ++pr) {
            const uint64_t ad =
                smem_desc(st + (uint32_t)(h * AT + tc_pair_a<AT, BT>(pr)) * a_bytes + kk * 256u, lbo, sbo);
            const uint64_t bd =
                smem_desc(st + BM2 * AT * a_bytes + (uint32_t)tc_pair_b<AT, BT>(pr) * b_bytes + kk * 256u, lbo, sbo);
            mma_bf16(tmem + (uint32_t)(h * TC_NMAX), ad, bd, idesc, (kt | kk | pr) != 0 ? 1u : 0u);
          }
        }
      }
      mma_commit(&mma_bar[stage]);
    }
    // refill the stage of k-tile kt - 1 with k-tile kt + STAGES - 1 once the MMAs of kt - 1
    // are done reading it (those of kt are queued behind them, so the tensor core stays busy)
    const int kn = kt + TC_STAGES - 1;
    if (kn < nkt) {
      const int sn = kn % TC_STAGES;
      if (kn >= TC_STAGES) ok = ok && mbar_wait_bounded(&mma_bar[sn], (uint32_t)(((kn - TC_STAGES) / TC_STAGES) & 1));
      if (ok) load_stage(kn, sn);
    }
    cp_async_commit();
  }
  cp_async_wait<0>();
  // the last commit tracks every MMA this CTA issued
  if (nkt > 0) {
    const int last = nkt - 1;
    if (ok) ok = mbar_wait_bounded(&mma_bar[last % TC_STAGES], (uint32_t)((last / TC_STAGES) & 1));
  }
  ok = __syncthreads_and(ok);
  tc_fence_after();

  if (ok) {
    tc_epilogue<EPI, BM2>(a, tmem, m0, nkt, warp, lane);
  } else if (tid == 0) {
    // a wait gave up: report, give the tensor core a bounded last chance to finish
    atomicExch(a.status, (int)NYS_ETIMEOUT);
    if (nkt > 0) (void)mbar_wait_bounded(&mma_bar[(nkt - 1) % TC_STAGES], (uint32_t)(((nkt - 1) / TC_STAGES) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---- TMA staging.  One thread (warp 0, lane 0) issues, per stage, one tiled copy of the
// A box {32 K, BM2 x 128 rows, AT terms} and one of the B box {32 K, N, BT terms}
// (cp.async.bulk.tensor.3d with the 64-byte swizzle; rows and K outside the matrices arrive
// as zeros) onto the stage's full barrier; one thread (warp 1, lane 0) waits for it, issues
// the MMAs and commits them to the stage's empty barrier, which the issuing thread waits on
// before it refills the stage.  A stage holds [term][row][64 bytes] in the canonical K-major
// 64-byte-swizzle layout (8-row groups 512 B apart; the K step of 16 elements moves the
// start address 32 B).  The MMAs and their order are those of sketch_tc_kernel, so both
// forms give the same bits.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

template <int EPI, int AT, int BT, int BM2>
__global__ void __launch_bounds__(TC_THREADS, 1)
    sketch_tc_tma_kernel(const __grid_constant__ TcArgs a, const __grid_constant__ CUtensorMap tmA,
                         const __grid_constant__ CUtensorMap tmB) {
  constexpr int ST = tc_stages<AT, BT, BM2>();
  constexpr uint32_t kTmemCols = BM2 == 2 ? 2 * TC_NMAX : TC_NMAX;
  constexpr int R = TC_BM * BM2;
  static_assert(ST >= 2, "shared memory holds fewer than two stages");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[ST];
  __shared__ __align__(8) uint64_t empty_bar[ST];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * R;
  const int64_t kt0 = (int64_t)blockIdx.y * a.kslice;
  const int64_t kt1 = min(a.ktiles, kt0 + a.kslice);
  const int nkt = (int)max((int64_t)0, kt1 - kt0);
  const uint32_t a_term = (uint32_t)(R * 64), b_term = (uint32_t)(a.NP * 64);   // [row][64 B] per term
  const uint32_t a_bytes = AT * a_term, b_bytes = BT * b_term;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t idesc = mma_idesc_bf16(TC_BM, a.NP);

  if (warp == 0) {
    tmem_alloc(&tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    s_fail = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    int kt = 0;
    for (; kt < nkt && !s_fail; ++kt) {
      const int s = kt % ST;
      // the MMAs of this stage's previous use must be done reading it
      if (kt >= ST && !mbar_wait_bounded(&empty_bar[s], (uint32_t)((kt / ST - 1) & 1))) {
        s_fail = 1;
        break;
      }
      const uint32_t st = sbase + (uint32_t)s * stage_bytes;
      const int k0 = (int)((kt0 + kt) * TC_BK);
      mbar_arrive_expect_tx(&full_bar[s], stage_bytes);
      tma_load_3d(st, &tmA, k0, (int)m0, 0, &full_bar[s]);
      tma_load_3d(st + a_bytes, &tmB, k0, 0, 0, &full_bar[s]);
    }
    // copies issued but not consumed (a wait gave up): let them land before the CTA leaves
    for (int j = max(0, kt - ST); j < kt; ++j) (void)mbar_wait_bounded(&full_bar[j % ST], (uint32_t)((j / ST) & 1));
  } else if (warp == 1 && lane == 0) {
    for (int kt = 0; kt < nkt && !s_fail; ++kt) {
      const int s = kt % ST;
      if (!mbar_wait_bounded(&full_bar[s], (uint32_t)((kt / ST) & 1))) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const uint32_t st = sbase + (uint32_t)s * stage_bytes;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
        for (int h = 0; h < BM2; ++h) {
#pragma unroll
          for (int pr = 0; pr < tc_npairs<AT, BT>(); ++pr) {
            const uint64_t ad = smem_desc_sw64(
                st + (uint32_t)tc_pair_a<AT, BT>(pr) * a_term + (uint32_t)(h * TC_BM * 64 + kk * 32), 512u);
            const uint64_t bd =
                smem_desc_sw64(st + a_bytes + (uint32_t)tc_pair_b<AT, BT>(pr) * b_term + (uint32_t)(kk * 32), 512u);
            mma_bf16(tmem + (uint32_t)(h * TC_NMAX), ad, bd, idesc, (kt | kk | pr) != 0 ? 1u : 0u);
          }
        }
      }
      mma_commit(&empty_bar[s]);
    }
  }
  __syncthreads();
  bool ok = s_fail == 0;
  // the last commit tracks every MMA this CTA issued
  if (ok && nkt > 0) ok = mbar_wait_bounded(&empty_bar[(nkt - 1) % ST], (uint32_t)(((nkt - 1) / ST) & 1));
  ok = __syncthreads_and(ok);
  tc_fence_after();
  if (ok) {
    tc_epilogue<EPI, BM2>(a, tmem, m0, nkt, warp, lane);
  } else if (tid == 0) {
    atomicExch(a.status, (int)NYS_ETIMEOUT);
    if (nkt > 0) (void)mbar_wait_bounded(&empty_bar[(nkt - 1) % ST], (uint32_t)(((nkt - 1) / ST) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// Operand terms: Ot[t][c][k] (c < NP, k < KP) = t-th BF16 term of float(X[k + (c0 + c) d]),
// zero outside c < mp, k < d.  X is d x m column-major (FP64 or FP32).
// NT = 1: X holds BF16 values (the rounded test matrix of the sketch), its one term is exact.
template <typename T, int NT>
__global__ void split_operand_kernel(const T* __restrict__ X, int64_t d, int c0, int mp, int NP, int64_t KP,
                                     uint16_t* __restrict__ Ot) {
  const int64_t total = (int64_t)NP * KP;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / KP);
    const int64_t k = idx - (int64_t)c * KP;
    float x = 0.f;
    if (c < mp && k < d) x = (float)X[k + (int64_t)(c0 + c) * d];
    uint16_t t3[3];
    split3(x, t3);
#pragma unroll
    for (int t = 0; t < NT; ++t) Ot[t * total + idx] = t3[t];
  }
}

// At[j][i] = A[i][j] (BF16), j < d, i < nP (zero for i >= n).  64 x 64 tiles.
__global__ void __launch_bounds__(256) transpose_bf16_kernel(const uint16_t* __restrict__ A, int64_t n, int64_t d,
                                                             int64_t lda, uint16_t* __restrict__ At, int64_t nP) {
  __shared__ uint16_t tile[64][66];
  const int64_t i0 = (int64_t)blockIdx.x * 64, j0 = (int64_t)blockIdx.y * 64;
  const int tid = threadIdx.x;
  {
    const int r = tid >> 2, cq = (tid & 3) * 16;  // row i0 + r, columns j0 + cq .. + 15
    const int64_t i = i0 + r, j = j0 + cq;
    uint16_t v[16];
    if (i < n && j + 16 <= d) {
      const uint4* src = reinterpret_cast<const uint4*>(A + i * lda + j);
      const uint4 x0 = src[0], x1 = src[1];
      const uint32_t w[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        v[2 * e] = (uint16_t)(w[e] & 0xffffu);
        v[2 * e + 1] = (uint16_t)(w[e] >> 16);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = (i < n && j + e < d) ? A[i * lda + j + e] : (uint16_t)0;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) tile[r][cq + e] = v[e];
  }
  __syncthreads();
  {
    const int r = tid >> 2, cq = (tid & 3) * 16;  // output row j0 + r, columns i0 + cq .. + 15
    const int64_t j = j0 + r, i = i0 + cq;
    if (j < d && i < nP) {
      uint32_t w[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) w[e] = (uint32_t)tile[cq + 2 * e][r] | ((uint32_t)tile[cq + 2 * e + 1][r] << 16);
      if (i + 16 <= nP) {
        uint4* dst = reinterpret_cast<uint4*>(At + j * nP + i);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
      } else {
        for (int e = 0; e < 16 && i + e < nP; ++e) At[j * nP + i + e] = tile[cq + e][r];
      }
    }
  }
}

// Y[j + (c0 + c) d] = sum_z P[z][c][j] (fixed order, FP64) + rho X[j + (c0 + c) d], c < mp.
template <typename TY, typename TX>
__global__ void sum_slices_kernel(const float* __restrict__ P, int Z, int NP, int64_t d, int c0, int mp,
                                  double rho, const TX* __restrict__ X, TY* __restrict__ Y) {
  const int64_t total = (int64_t)mp * d;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / d);
    const int64_t j = idx - (int64_t)c * d;
    double s = 0.0;
    for (int z = 0; z < Z; ++z) s += (double)P[((int64_t)z * NP + c) * d + j];
    const int64_t o = j + (int64_t)(c0 + c) * d;
    if (X && rho != 0.0) s += rho * (double)X[o];
    Y[o] = (TY)s;
  }
}

int sm_count_tc() { return sm_count(); }

// split-K slices for GEMM 2: the count (<= 32, each slice >= 16 K tiles) whose CTA count
// fills the last wave best.
int pick_slices(int64_t mtiles, int64_t ktiles, int sms) {
  int best = 1;
  double best_fill = 0.0;
  for (int z = 1; z <= 32; ++z) {
    if (z > 1 && ktiles / z < 16) break;
    const int64_t units = mtiles * z;
    const int64_t waves = (units + sms - 1) / sms;
    const double fill = (double)units / (double)(waves * sms);
    if (fill > best_fill + 1e-9) {
      best_fill = fill;
      best = z;
    }
  }
  return best;
}

// cuTensorMapEncodeTiled from the driver (the library links only the runtime).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    (void)cudaGetLastError();
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// 3-D map of `terms` BF16 matrices (rows x K, K contiguous, row stride ld elements, term
// stride tstride elements) with the box {32, box_rows, terms} and the 64-byte swizzle: one
// K tile of every row and term per copy; rows >= rows and K >= K arrive as zeros.
cudaError_t make_tile_map(CUtensorMap* m, const uint16_t* base, int64_t K, int64_t rows, int64_t ld, int terms,
                          int64_t tstride, int box_rows) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)terms};
  // a single term: any stride past the matrix will do
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)(terms > 1 ? tstride : ld * rows) * 2};
  const cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, (cuuint32_t)terms};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// TMA staging unless NYS_TC_TMA=0 or the driver offers no tensor-map encoder (then the
// cp.async form: the same MMAs, the same bits).
bool tc_use_tma() {
  const char* e = std::getenv("NYS_TC_TMA");
  if (e && std::atoi(e) == 0) return false;
  return encode_tiled_fn() != nullptr;
}

template <int EPI, int AT, int BT, int BM2>
cudaError_t launch_tc(const TcArgs& a, dim3 grid, cudaStream_t st) {
  constexpr int ST = tc_stages<AT, BT, BM2>();
  const size_t smem = (size_t)ST * (BM2 * AT * TC_BM * TC_BK * 2 + (size_t)BT * a.NP * TC_BK * 2);
  if (tc_use_tma()) {
    CUtensorMap tmA, tmB;
    NYS_CUDA_TRY(make_tile_map(&tmA, a.A, a.Kvalid, a.Mrows, a.lda, AT, a.aterm, TC_BM * BM2));
    NYS_CUDA_TRY(make_tile_map(&tmB, a.B, a.ktiles * TC_BK, a.NP, a.ldb, BT, a.bterm, a.NP));
    NYS_CUDA_TRY(ensure_max_dyn_smem((const void*)sketch_tc_tma_kernel<EPI, AT, BT, BM2>,
                                     ST * tc_stage_max_bytes<AT, BT, BM2>()));
    count_launch();
    sketch_tc_tma_kernel<EPI, AT, BT, BM2><<<grid, TC_THREADS, smem, st>>>(a, tmA, tmB);
    return cudaGetLastError();
  }
  NYS_CUDA_TRY(ensure_max_dyn_smem((const void*)sketch_tc_kernel<EPI, AT, BT, BM2>,
                                   ST * tc_stage_max_bytes<AT, BT, BM2>()));
  count_launch();
  sketch_tc_kernel<EPI, AT, BT, BM2><<<grid, TC_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

// Output rows per CTA: two 128-row accumulators, except for FP32 x FP32 (six MMA pairs),
// whose stages leave room for one.
int tc_cta_rows(int at, int bt) { return TC_BM * (at == 3 && bt == 3 ? 1 : 2); }

template <int EPI>
cudaError_t launch_tc_at(int at, int bt, const TcArgs& a, dim3 grid, cudaStream_t st) {
  if constexpr (EPI == 1) {   // the second product's B is W, always three terms
    return at == 3 ? launch_tc<EPI, 3, 3, 1>(a, grid, st) : launch_tc<EPI, 1, 3, 2>(a, grid, st);
  } else {
    if (at == 3) return bt == 3 ? launch_tc<EPI, 3, 3, 1>(a, grid, st) : launch_tc<EPI, 3, 1, 2>(a, grid, st);
    return bt == 3 ? launch_tc<EPI, 1, 3, 2>(a, grid, st) : launch_tc<EPI, 1, 1, 2>(a, grid, st);
  }
}

// FP32 storage: A (n x lda, row-major) -> three BF16 terms As[t][i][j] (row stride ldS,
// zero for j >= d) whose sum is the FP32 value exactly.
__global__ void split_matrix_kernel(const float* __restrict__ A, int64_t n, int64_t d, int64_t lda, int64_t ldS,
                                    uint16_t* __restrict__ As) {
  const int64_t total = n * ldS;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / ldS, j = idx - i * ldS;
    const float x = j < d ? A[i * lda + j] : 0.f;
    uint16_t t3[3];
    split3(x, t3);
#pragma unroll
    for (int t = 0; t < TC_TERMS; ++t) As[t * total + idx] = t3[t];
  }
}

}  // namespace


namespace {
// Y (d x m, column-major) = A^T diag(D) A X (+ rho X) on the tensor cores, given the
// transposed copy At (d x nP) of A.  X and Y are FP64 (sketch) or FP32 (batched PCG).
// xterms = 1: X holds BF16 values (the sketch's rounded test matrix), so the first product
// takes one MMA term of X instead of three.
template <typename TX, typename TY>
cudaError_t tc_product(const nys_matrix* A, const TcPrepared& prep, const double* D, const TX* X, int m,
                       double rho, TY* Y, cudaStream_t st, bool trace, int xterms) {
  const int64_t n = A->n, d = A->d;
  const int64_t nP = prep.nP;
  const int64_t dP = (d + TC_BK - 1) / TC_BK * TC_BK;
  const int NPmax = std::min(TC_NMAX, (m + 15) / 16 * 16);
  const uint32_t swap = std::getenv("NYS_TC_DESC_SWAP") ? (uint32_t)std::atoi(std::getenv("NYS_TC_DESC_SWAP")) : 0u;
  const int sms = sm_count_tc();
  const int rows1 = tc_cta_rows(prep.at, xterms), rows2 = tc_cta_rows(prep.at, TC_TERMS);
  const int64_t mt2 = (d + rows2 - 1) / rows2;
  const int64_t kt2 = nP / TC_BK;
  const int Z = pick_slices(mt2, kt2, sms);
  const int64_t kslice2 = (kt2 + Z - 1) / Z;
  const int Zeff = (int)((kt2 + kslice2 - 1) / kslice2);

  cudaEvent_t ev[8] = {};
  int nev = 0;
  auto mark = [&]() {
    if (!trace || nev >= 8) return;
    if (cudaEventCreate(&ev[nev]) == cudaSuccess) cudaEventRecord(ev[nev], st);
    ++nev;
  };
  mark();
  Pool pool(st);
  uint16_t* Ot = pool.alloc<uint16_t>((size_t)xterms * NPmax * dP);
  uint16_t* Wt = pool.alloc<uint16_t>((size_t)TC_TERMS * NPmax * nP);
  float* P = pool.alloc<float>((size_t)Zeff * NPmax * d);
  int* status = pool.alloc<int>(1);
  if (!pool.ok()) return cudaErrorMemoryAllocation;
  NYS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  mark();
  for (int c0 = 0; c0 < m; c0 += TC_NMAX) {
    const int mp = std::min(TC_NMAX, m - c0);
    const int NP = (mp + 15) / 16 * 16;
    count_launch();
    const unsigned sgrid = (unsigned)std::min<int64_t>(4096, ((int64_t)NP * dP + 255) / 256);
    if (xterms == 1)
      split_operand_kernel<TX, 1><<<sgrid, 256, 0, st>>>(X, d, c0, mp, NP, dP, Ot);
    else
      split_operand_kernel<TX, TC_TERMS><<<sgrid, 256, 0, st>>>(X, d, c0, mp, NP, dP, Ot);
    NYS_CUDA_TRY(cudaGetLastError());
    if (c0 == 0) mark();

    TcArgs g1 = {};
    g1.A = prep.A;
    g1.lda = prep.lda;
    g1.aterm = prep.aterm;
    g1.Mrows = n;
    g1.Kvalid = d;
    g1.B = Ot;
    g1.ldb = dP;
    g1.bterm = (int64_t)NP * dP;
    g1.NP = NP;
    g1.ktiles = dP / TC_BK;
    g1.kslice = g1.ktiles;
    g1.D = D;
    g1.Wt = Wt;
    g1.ldw = nP;
    g1.wterm = (int64_t)NP * nP;
    g1.wrows = nP;
    g1.desc_swap = swap;
    g1.status = status;
    NYS_CUDA_TRY(launch_tc_at<0>(prep.at, xterms, g1, dim3((unsigned)((n + rows1 - 1) / rows1), 1), st));
    if (c0 == 0) mark();

    TcArgs g2 = {};
    g2.A = prep.At;
    g2.lda = nP;
    g2.aterm = prep.atterm;
    g2.Mrows = d;
    g2.Kvalid = nP;
    g2.B = Wt;
    g2.ldb = nP;
    g2.bterm = (int64_t)NP * nP;
    g2.NP = NP;
    g2.ktiles = kt2;
    g2.kslice = kslice2;
    g2.P = P;
    g2.ldp = d;
    g2.desc_swap = swap;
    g2.status = status;
    NYS_CUDA_TRY(launch_tc_at<1>(prep.at, TC_TERMS, g2, dim3((unsigned)mt2, (unsigned)Zeff), st));
    if (c0 == 0) mark();

    count_launch();
    sum_slices_kernel<TY, TX><<<(unsigned)std::min<int64_t>(4096, ((int64_t)mp * d + 255) / 256), 256, 0, st>>>(
        P, Zeff, NP, d, c0, mp, rho, X, Y);
    NYS_CUDA_TRY(cudaGetLastError());
    if (c0 == 0) mark();
  }
  int status_h = 0;
  NYS_CUDA_TRY(cudaMemcpyAsync(&status_h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NYS_CUDA_TRY(cudaStreamSynchronize(st));
  if (trace) {
    static const char* names[] = {"alloc", "split operand", "GEMM1 W = D A X", "GEMM2 A^T W", "sum slices"};
    for (int i = 1; i < nev && i < 6; ++i) {
      float ms = 0.f;
      if (ev[i - 1] && ev[i]) cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
      std::fprintf(stderr, "[nys]   tc %-18s %8.3f ms\n", names[i - 1], ms);
    }
    std::fprintf(stderr, "[nys]   tc split-K slices %d, NP %d\n", Zeff, NPmax);
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return status_h ? cudaErrorLaunchTimeout : cudaSuccess;
}
}  // namespace

namespace {
__global__ void round_bf16_kernel(double* __restrict__ X, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    X[i] = (double)bf16_val(bf16_bits((float)X[i]));
}
}  // namespace

cudaError_t round_panel_bf16(double* X, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  round_bf16_kernel<<<(unsigned)std::min<int64_t>(4096, (n + 255) / 256), 256, 0, st>>>(X, n);
  return cudaGetLastError();
}

bool sketch_tc_supported(const nys_matrix* A) {
  if (A->dtype != NYS_BF16 && A->dtype != NYS_F32) return false;
  if (const char* env = std::getenv("NYS_SKETCH_TC")) return std::atoi(env) != 0;
  return true;
}

// Scratch of the prepared operands: BF16 storage keeps A itself and adds the transposed
// copy (d x nP); FP32 storage adds its three BF16 terms (n x ldS each) and their
// transposes (d x nP each).
size_t tc_prepare_bytes(const nys_matrix* A) {
  const int64_t nP = (A->n + TC_BK - 1) / TC_BK * TC_BK;
  const int64_t ldS = (A->d + 7) / 8 * 8;
  if (A->dtype == NYS_BF16) return (size_t)A->d * nP * 2;
  return (size_t)TC_TERMS * ((size_t)A->n * ldS + (size_t)A->d * nP) * 2;
}

cudaError_t tc_prepare(const nys_matrix* A, void* scratch, TcPrepared* prep, cudaStream_t st) {
  const int64_t n = A->n, d = A->d;
  const int64_t nP = (n + TC_BK - 1) / TC_BK * TC_BK;
  const dim3 tgrid((unsigned)((nP + 63) / 64), (unsigned)((d + 63) / 64));
  uint16_t* buf = reinterpret_cast<uint16_t*>(scratch);
  prep->nP = nP;
  if (A->dtype == NYS_BF16) {
    prep->at = 1;
    prep->A = reinterpret_cast<const uint16_t*>(A->data);
    prep->lda = A->ld;
    prep->aterm = 0;
    prep->At = buf;
    prep->atterm = 0;
    count_launch();
    transpose_bf16_kernel<<<tgrid, 256, 0, st>>>(reinterpret_cast<const uint16_t*>(A->data), n, d, A->ld, buf, nP);
    return cudaGetLastError();
  }
  if (A->dtype != NYS_F32) return cudaErrorInvalidValue;
  const int64_t ldS = (d + 7) / 8 * 8;
  uint16_t* As = buf;
  uint16_t* Ats = buf + (size_t)TC_TERMS * n * ldS;
  prep->at = 3;
  prep->A = As;
  prep->lda = ldS;
  prep->aterm = n * ldS;
  prep->At = Ats;
  prep->atterm = d * nP;
  count_launch();
  split_matrix_kernel<<<(unsigned)std::min<int64_t>(8192, (n * ldS + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const float*>(A->data), n, d, A->ld, ldS, As);
  NYS_CUDA_TRY(cudaGetLastError());
  for (int t = 0; t < TC_TERMS; ++t) {
    count_launch();
    transpose_bf16_kernel<<<tgrid, 256, 0, st>>>(As + (size_t)t * n * ldS, n, d, ldS, Ats + (size_t)t * d * nP, nP);
    NYS_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t sketch_tc(const nys_matrix* A, const double* D, const double* Om, int m, double* Y, cudaStream_t st) {
  if ((A->dtype != NYS_BF16 && A->dtype != NYS_F32) || m <= 0) return cudaErrorInvalidValue;
  const bool trace = std::getenv("NYS_TRACE") != nullptr;
  Pool pool(st);
  void* scratch = pool.alloc<unsigned char>(tc_prepare_bytes(A));
  if (!pool.ok()) return cudaErrorMemoryAllocation;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (trace) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  TcPrepared prep;
  NYS_CUDA_TRY(tc_prepare(A, scratch, &prep, st));
  if (trace) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    std::fprintf(stderr, "[nys]   tc %-18s %8.3f ms\n", "prepare A", ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  return tc_product<double, double>(A, prep, D, Om, m, 0.0, Y, st, trace, 1);
}

cudaError_t sketch_tc_with(const nys_matrix* A, const TcPrepared& prep, const double* D, const double* Om, int m,
                           double* Y, cudaStream_t st) {
  if (m <= 0) return cudaErrorInvalidValue;
  return tc_product<double, double>(A, prep, D, Om, m, 0.0, Y, st, std::getenv("NYS_TRACE") != nullptr, 1);
}

cudaError_t tc_hmm(const nys_matrix* A, const TcPrepared& prep, const double* D, const float* X, int k, double rho,
                   float* Y, cudaStream_t st) {
  if (k <= 0) return cudaErrorInvalidValue;
  return tc_product<float, float>(A, prep, D, X, k, rho, Y, st, false, TC_TERMS);
}

}  // namespace nys
