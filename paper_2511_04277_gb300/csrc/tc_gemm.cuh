// tcgen05 GEMMs for sm_103a, 16-bit operands (bf16 or fp16, both K-major: row-major with K
// contiguous), fp32 accumulation in tensor memory.
//
// gemm_kernel: D[M x N] = A[M x K] * B[N x K]^T with an epilogue functor. One CTA computes
// one BM x BN tile (BM = 128). Warp roles (192 threads):
//   warp 0      TMA producer: 64-wide K blocks of A and B into a ring of smem stages
//               (128-byte swizzle), completion signalled on full[s] mbarriers;
//   warp 1      allocates TMEM, one elected thread issues tcgen05.mma (K = 16 each)
//               and commits to empty[s] (stage free) and acc_full (accumulator ready);
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM lanes
//               32*(w%4) .. +31, i.e. tile rows), then the Epi functor writes the result.
// gemm_exact_kernel: the integer-exact level product of the dense solves' refinement (see
// its comment); the same roles with 128-long K chunks in two TMEM buffers.
//
// Every mbarrier wait is bounded; on a timeout the kernel records an error word, stops
// issuing work, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"

namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;  // one 128-byte swizzle atom of 16-bit elements
constexpr int kThreads = 192;
constexpr int kGroupM = 8;  // row tiles per rasterisation group
constexpr uint64_t kWaitNs = 2000000000ull;  // a wait gives up after 2 s

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  uint32_t addr = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t i = 1;; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 255u) == 0) {
      uint64_t now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// ---- CTA pairs (cta_group::2): a cluster of two CTAs computes one 256-row tile, each CTA
// holding its 128 rows of A and half of the tile's columns of B in shared memory at the same
// offsets; one thread of the even CTA issues the MMAs, and each CTA's tensor memory receives
// its 128 rows of the product.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// one arrival on an mbarrier of another CTA of the cluster (no memory ordering: the data the
// arrival announces is already in place, in shared memory or tensor memory)
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// mbar_wait with cluster-scope acquire, for phases completed by the other CTA of the pair
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  uint32_t addr = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t i = 1;; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 255u) == 0) {
      uint64_t now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
  }
}
// tensor memory of both CTAs of the pair: one warp of each CTA takes part (the same columns
// in both)
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void umma_f16_pair(uint32_t tmem_d, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// one arrival on the barrier at this offset in both CTAs once this thread's prior tcgen05
// operations have completed
__device__ __forceinline__ void umma_commit_pair_both(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ void umma_commit_pair_local(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 columns of this warp's 32 TMEM lanes (one row per thread), as tmem_ld32: the exact
// product's epilogue, whose 128 int32 column sums per thread leave no room for 32 more.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows, 128-byte
// swizzle, 8-row core groups 1024 bytes apart (sm_100 descriptor version 1).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16 with fp32 accumulation, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n, bool bf16) {
  return (1u << 4)                                   // D format: fp32
         | ((bf16 ? 1u : 0u) << 7)                   // A format
         | ((bf16 ? 1u : 0u) << 10)                  // B format
         | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// ------------------------------------------------------------------ epilogues
// An epilogue receives, per warp and per 32-column slab, the 32 x 32 block of the tile
// owned by that warp: lane l holds row row0 + l, columns c0 .. c0+31 in v[0..31]. `stage`
// is a [32][33] shared-memory block private to the warp, used to turn the row-per-lane
// layout into coalesced row stores.

// Straight store through the staging block: out(r, c) for r in row0..row0+31 with each
// warp instruction writing 32 consecutive columns of one row.
template <class T, class F>
__device__ __forceinline__ void staged_rows(int row0, int lane, int c0, int M, int N, const T* v, T (*stage)[33],
                                            F&& put) {
#pragma unroll
  for (int i = 0; i < 32; ++i) stage[lane][i] = v[i];
  __syncwarp();
  const int c = c0 + lane;
#pragma unroll 4
  for (int rr = 0; rr < 32; ++rr) {
    const int r = row0 + rr;
    if (r < M && c < N) put(r, c, stage[rr][lane]);
  }
  __syncwarp();
}

template <class T16>
__device__ __forceinline__ T16 to_16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_16<__half>(float x) { return __float2half_rn(x); }

// Every epilogue's store() also receives `offdiag`: true for an off-diagonal tile of a
// symmetric product (GemmArgs::sym), which stands for its transposed tile as well; the
// epilogues of the Newton-Schulz steps then also write the transposed position.

// C[r][c] = beta * C[r][c] + alpha * acc   (fp32 C)
struct EpiF32 {
  float* C;
  int64_t ldc;
  float alpha, beta;
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, const float* v,
                                        float (*stage)[33], bool) const {
    staged_rows(row0, lane, c0, M, N, v, stage, [&](int r, int c, float x) {
      float* p = C + (int64_t)r * ldc + c;
      *p = (beta == 0.f ? 0.f : beta * *p) + alpha * x;
    });
  }
};

// Newton-Schulz half step: Zt[c][r] = 16-bit (2 delta_rc - acc) -- the transposed store is
// coalesced as it is (the warp's 32 rows are 32 consecutive elements of a row of Zt). A X is
// not symmetric unless X and A commute, which rounding breaks: this product is always whole.
template <class T16>
struct EpiTwoIMinusT {
  T16* Zt;
  int64_t ld;
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, const float* v,
                                        float (*)[33], bool) const {
    const int r = row0 + lane;
    if (r >= M) return;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
      const int c = c0 + i;
      if (c < N) Zt[(int64_t)c * ld + r] = to_16<T16>((r == c ? 2.f : 0.f) - v[i]);
    }
  }
};

// Newton-Schulz step result: X[r][c] and Xt[c][r] = 16-bit acc. With `sym` (Xt = X, the
// product X (2I - A X) = 2X - X A X symmetric for symmetric X and A, whatever their
// commutation) the transposed write is made for off-diagonal tiles only.
template <class T16>
struct EpiStore16Both {
  T16* X;
  T16* Xt;
  int64_t ld;
  bool sym = false;
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, const float* v,
                                        float (*stage)[33], bool offdiag) const {
    const int r = row0 + lane;
    if (r < M && (!sym || offdiag)) {
#pragma unroll 8
      for (int i = 0; i < 32; ++i) {
        const int c = c0 + i;
        if (c < N) Xt[(int64_t)c * ld + r] = to_16<T16>(v[i]);
      }
    }
    staged_rows(row0, lane, c0, M, N, v, stage, [&](int rr, int c, float x) { X[(int64_t)rr * ld + c] = to_16<T16>(x); });
  }
};

// D[r][c] = acc * colscale[c] (* rowscale[r] when given) (fp32; the refinement's correction
// M R before it is rounded to its one-slice form), with max_r |D[r][c]| folded into colmax[c]
// (float bits, atomicMax) and *nonfinite raised on an inf or NaN.
struct EpiCorrection {
  float* D;
  int64_t ld;
  const float* colscale;
  unsigned int* colmax;
  int* nonfinite;
  const float* rowscale = nullptr;
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, const float* v,
                                        float (*stage)[33], bool) const {
#pragma unroll
    for (int i = 0; i < 32; ++i) stage[lane][i] = v[i];
    __syncwarp();
    const int c = c0 + lane;
    const bool cok = c < N;
    const float cs = cok ? colscale[c] : 0.f;
    float mx = 0.f;
    bool bad = false;
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      const int r = row0 + rr;
      if (cok && r < M) {
        const float d = stage[rr][lane] * cs * (rowscale ? rowscale[r] : 1.f);
        D[(int64_t)r * ld + c] = d;
        mx = fmaxf(mx, fabsf(d));
        bad |= !isfinite(d);
      }
    }
    __syncwarp();
    if (cok) atomicMax(&colmax[c], __float_as_uint(mx));
    if (__any_sync(0xffffffffu, bad) && lane == 0 && nonfinite) atomicExch(nonfinite, 1);
  }
};

struct GemmArgs {
  int M, N, K;
  int* error_word;
  // non-null: the kernel does nothing when *skip != 0 (written by an earlier kernel on
  // the stream; a speculatively launched product the host's decision made unnecessary)
  const int* skip = nullptr;
  // > 0: the inner dimension of the product the launch stands for (kernel timer accounting)
  int alg_k = 0;
  // 1: the product is symmetric (M = N, square tiles): only the tiles on and above the
  // diagonal are computed, the epilogue writing each off-diagonal one for its transpose too
  int sym = 0;
  // Block flags of A (CTA-pair kernel only; null: every block): aflags[tile ceil(K / BK / 32) 32
  // + kb] != 0 when A's 256-row tile `tile` has a non-zero entry in K block kb; bflags the same
  // for B's 256-row tiles (the product's 256-column tiles). A block is multiplied when neither
  // flag says zero. With flags the leader CTAs add the K blocks they execute to *level_log
  // (kernel timer), else nothing.
  const uint8_t* aflags = nullptr;
  const uint8_t* bflags = nullptr;
  int* level_log = nullptr;
};

// K blocks of the CTA-pair GEMM whose A block flags it can hold (K <= 32,768).
constexpr int kGemmMaxKWords = 16;

// Tile (I, J), I <= J, of the pid-th tile on or above the diagonal of a T x T tiling, in
// bands of kGroupM tile rows, each band's tiles column by column (the CTAs running together
// share their column tiles in L2).
__device__ __forceinline__ void upper_tile(int pid, int T, int& I, int& J) {
  int r0 = 0;
  for (;;) {
    const int r1 = min(r0 + kGroupM, T);
    // band rows [r0, r1): column J holds min(r1, J + 1) - r0 tiles, J >= r0
    const int h = r1 - r0;
    const int band = h * (h + 1) / 2 + h * (T - r1);
    if (pid < band) break;
    pid -= band;
    r0 = r1;
  }
  const int r1 = min(r0 + kGroupM, T);
  for (int j = r0;; ++j) {
    const int cnt = min(r1, j + 1) - r0;
    if (pid < cnt) {
      I = r0 + pid;
      J = j;
      return;
    }
    pid -= cnt;
  }
}

template <int BN, int kStages, class Epi, bool kBF16>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                const GemmArgs args, const Epi epi) {
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
  constexpr uint32_t kABytes = BM * BK * 2, kBBytes = BN * BK * 2;
  constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;
  constexpr uint32_t kIdesc = idesc_f16(BM, BN, kBF16);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;  // [1]
  uint64_t* drain = acc_full + 1;        // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ int s_abort;
  __shared__ int s_consumed;             // K blocks whose stage the MMA thread has taken
  __shared__ float s_stage[4][32][33];   // per epilogue warp: coalescing block

  if (args.skip && *(volatile const int*)args.skip) return;  // uniform: before any barrier or allocation
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped rasterisation of the 1-D grid: kGroupM row tiles at a time, column tiles
  // innermost, so that the CTAs resident together share their A and B tiles in L2
  const int tiles_m = (args.M + BM - 1) / BM, tiles_n = (args.N + BN - 1) / BN;
  const int pid = blockIdx.x;
  int tile_m, tile_n;
  if (args.sym) {  // square tiles (BN == BM), those on and above the diagonal
    upper_tile(pid, tiles_m, tile_m, tile_n);
  } else {
    const int group = pid / (kGroupM * tiles_n);
    const int first_m = group * kGroupM;
    const int group_m = min(tiles_m - first_m, kGroupM);
    tile_m = first_m + (pid % (kGroupM * tiles_n)) % group_m;
    tile_n = (pid % (kGroupM * tiles_n)) / group_m;
  }
  const bool offdiag = args.sym && tile_m != tile_n;
  const int m0 = tile_m * BM, n0 = tile_n * BN;
  const int kb_total = (args.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    s_abort = 0;
    s_consumed = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < kb_total; ++kb) {
        const int s = kb % kStages;
        if (kb >= kStages && !mbar_wait(&empty[s], ((kb / kStages) - 1) & 1)) { *abort_flag = 1; break; }
        if (*abort_flag) break;
        mbar_expect_tx(&full[s], kABytes + kBBytes);
        tma_load_2d(sA + s * kABytes, &map_a, &full[s], kb * BK, m0);
        tma_load_2d(sB + s * kBBytes, &map_b, &full[s], kb * BK, n0);
        ++issued;
      }
      if (*abort_flag) {
        // let the copies this thread started land before the CTA goes away
        for (int kb = *(volatile int*)&s_consumed; kb < issued; ++kb) mbar_wait(&full[kb % kStages], (kb / kStages) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      for (int kb = 0; kb < kb_total && !*abort_flag; ++kb) {
        const int s = kb % kStages;
        if (!mbar_wait(&full[s], (kb / kStages) & 1)) { *abort_flag = 1; break; }
        *(volatile int*)&s_consumed = kb + 1;
        tc_fence_after();
        const uint32_t a_addr = smem_u32(sA + s * kABytes), b_addr = smem_u32(sB + s * kBBytes);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          umma_f16(tmem_base, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), kIdesc,
                   (kb > 0 || kk > 0) ? 1u : 0u);
        umma_commit(&empty[s]);
      }
      if (!*abort_flag) umma_commit(acc_full);
      // every MMA this thread issued has completed once `drain` fires
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
  } else {
    // ---------------- epilogue warps 2 .. 5
    const int ew = warp - 2;
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int row0 = m0 + quarter * 32;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    float(*stage)[33] = s_stage[ew];
    if (mbar_wait(acc_full, 0)) {
      tc_fence_after();
      float v[32];
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        tmem_ld32(tmem_base + lane_addr + (uint32_t)c0, v);
        epi.store(row0, lane, n0 + c0, args.M, args.N, v, stage, offdiag);
      }
    } else {
      *abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag && args.error_word) atomicExch(args.error_word, 1);
}

template <int BN, int kStages>
constexpr size_t smem_bytes() {
  return 1024 + (size_t)kStages * (BM * BK * 2 + BN * BK * 2) + (2 * kStages + 3) * 8 + 16;
}

// gemm_kernel on CTA pairs (cluster of 2, cta_group::2): the pair computes a 256 x 256 tile;
// each CTA loads its 128 rows of A and 128 of the tile's 256 rows of B per K block (32 KB a
// stage instead of 48 KB, so kStages = 6 fit where the one-CTA kernel holds 4: the deeper
// ring hides more of the L2 latency, and the pair reads B once for both row halves). Warp
// roles as gemm_kernel, with:
//   warp 0 (both CTAs)   TMA into its own stage ring, completion on its own full[s];
//   warp 1, even CTA     the MMAs of the pair (M = 256, N = 256) once full[s] has both its
//                        own bytes and the odd CTA's arrival, committing to empty[s] and
//                        acc_full of both CTAs;
//   warp 1, odd CTA      relays each of its full stages to the even CTA's full[s];
//   warps 2..5           the epilogue of the CTA's own 128 rows (tensor memory of its own).
// Grid: two CTAs per tile, grouped rasterisation over the tiles as gemm_kernel.
template <int kStages, class Epi, bool kBF16>
__global__ void __launch_bounds__(kThreads, 1) __cluster_dims__(2, 1, 1)
    gemm_pair_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                     const GemmArgs args, const Epi epi) {
  constexpr int PN = 256;  // columns of the pair's tile
  constexpr uint32_t kABytes = BM * BK * 2, kBBytes = (PN / 2) * BK * 2;
  constexpr uint32_t kTmemCols = PN;
  constexpr uint32_t kIdesc = idesc_f16(2 * BM, PN, kBF16);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;  // [1]
  uint64_t* drain = acc_full + 1;        // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ int s_abort;
  __shared__ float s_stage[4][32][33];
  __shared__ uint32_t s_kmask[kGemmMaxKWords];  // the tile's K blocks of A holding non-zeros

  // uniform over the pair (both read the same word): before any barrier or allocation
  if (args.skip && *(volatile const int*)args.skip) return;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (args.M + 2 * BM - 1) / (2 * BM), tiles_n = (args.N + PN - 1) / PN;
  const int pid = blockIdx.x >> 1;
  int tile_m, tile_n;
  if (args.sym) {  // 256 x 256 tiles on and above the diagonal
    upper_tile(pid, tiles_m, tile_m, tile_n);
  } else {
    const int group = pid / (kGroupM * tiles_n);
    const int first_m = group * kGroupM;
    const int group_m = min(tiles_m - first_m, kGroupM);
    tile_m = first_m + (pid % (kGroupM * tiles_n)) % group_m;
    tile_n = (pid % (kGroupM * tiles_n)) / group_m;
  }
  const bool offdiag = args.sym && tile_m != tile_n;
  const int m0 = tile_m * 2 * BM + (int)rank * BM;         // this CTA's rows
  const int nb0 = tile_n * PN + (int)rank * (PN / 2);      // this CTA's half of B's rows
  const int n0 = tile_n * PN;                              // the tile's columns
  const int kb_total = (args.K + BK - 1) / BK;
  // K blocks this tile multiplies: every block, or with A's block flags only those where the
  // pair's 256 rows of A hold a non-zero (both CTAs read the same flags; at least one block
  // is kept, so that the accumulator is written)
  const int kwords = (kb_total + 31) / 32;
  const bool use_flags = (args.aflags != nullptr || args.bflags != nullptr) && kwords <= kGemmMaxKWords;
  // the 32 flags of word w of a flag row as bits
  auto flag_bits = [&](const uint8_t* row, int w) -> uint32_t {
    const uint4* fp = reinterpret_cast<const uint4*>(row + (int64_t)w * 32);
    const uint4 f0 = __ldg(fp), f1 = __ldg(fp + 1);
    const uint32_t fw[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
    uint32_t bits = 0u;
#pragma unroll
    for (int q = 0; q < 32; ++q) bits |= ((fw[q >> 2] >> (8 * (q & 3))) & 0xffu) ? (1u << q) : 0u;
    return bits;
  };
  for (int w = threadIdx.x; w < kwords && w < kGemmMaxKWords; w += blockDim.x) {
    uint32_t m = kb_total - 32 * w >= 32 ? ~0u : ((1u << (kb_total - 32 * w)) - 1u);
    if (use_flags && args.aflags) m &= flag_bits(args.aflags + (int64_t)tile_m * kwords * 32, w);
    if (use_flags && args.bflags) m &= flag_bits(args.bflags + (int64_t)tile_n * kwords * 32, w);
    s_kmask[w] = m;
  }

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], leader ? 2 : 1);  // even CTA: its own expect_tx and the odd CTA's relay
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc_pair(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers exist before any arrival from the other
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;
  // the K block of the t-th multiplied block (t < n_mult), from the mask table
  int n_mult = 0;
  if (use_flags)
    for (int w = 0; w < kwords; ++w) n_mult += __popc(s_kmask[w]);
  const bool none = use_flags && n_mult == 0;
  if (!use_flags) n_mult = kb_total;
  if (none) n_mult = 1;  // an all-zero row of tiles: one (zero) block initialises the accumulator
  int it_w = 0;
  uint32_t it_m = use_flags ? s_kmask[0] : 0u;
  auto next_kb = [&](int t) -> int {  // called with t = 0, 1, 2, ... in order
    if (!use_flags || none) return t;
    while (!it_m) it_m = s_kmask[++it_w];
    const int kb = 32 * it_w + __ffs(it_m) - 1;
    it_m &= it_m - 1u;
    return kb;
  };

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs)
    if (lane == 0) {
      for (int t = 0; t < n_mult; ++t) {
        const int s = t % kStages;
        if (t >= kStages && !mbar_wait_cluster(&empty[s], ((t / kStages) - 1) & 1)) { *abort_flag = 1; break; }
        if (*abort_flag) break;
        const int kb = next_kb(t);
        mbar_expect_tx(&full[s], kABytes + kBBytes);
        tma_load_2d(sA + s * kABytes, &map_a, &full[s], kb * BK, m0);
        tma_load_2d(sB + s * kBBytes, &map_b, &full[s], kb * BK, nb0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (leader) {
        // ---------------- MMA issuer of the pair
        for (int t = 0; t < n_mult && !*abort_flag; ++t) {
          const int s = t % kStages;
          if (!mbar_wait_cluster(&full[s], (t / kStages) & 1)) { *abort_flag = 1; break; }
          tc_fence_after();
          const uint32_t a_addr = smem_u32(sA + s * kABytes), b_addr = smem_u32(sB + s * kBBytes);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            umma_f16_pair(tmem_base, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), kIdesc,
                          (t > 0 || kk > 0) ? 1u : 0u);
          umma_commit_pair_both(&empty[s]);
        }
        if (use_flags && args.level_log) atomicAdd(args.level_log, n_mult);
        if (!*abort_flag) umma_commit_pair_both(acc_full);
        // every MMA this thread issued has completed once `drain` fires
        umma_commit_pair_local(drain);
        mbar_wait(drain, 0);
      } else {
        // ---------------- relay: this CTA's stage s is full -> one arrival on the even CTA's full[s]
        const uint32_t leader_full = mapa_shared(smem_u32(full), 0);
        for (int t = 0; t < n_mult; ++t) {
          const int s = t % kStages;
          if (!mbar_wait(&full[s], (t / kStages) & 1)) { *abort_flag = 1; break; }
          mbar_arrive_remote(leader_full + 8u * (uint32_t)s);
        }
      }
    }
  } else {
    // ---------------- epilogue warps 2 .. 5: this CTA's 128 rows
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int row0 = m0 + quarter * 32;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    float(*stage)[33] = s_stage[ew];
    if (mbar_wait_cluster(acc_full, 0)) {
      tc_fence_after();
      float v[32];
#pragma unroll 1
      for (int c0 = 0; c0 < PN; c0 += 32) {
        tmem_ld32(tmem_base + lane_addr + (uint32_t)c0, v);
        epi.store(row0, lane, n0 + c0, args.M, args.N, v, stage, offdiag);
      }
    } else {
      *abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // the pair's MMAs and relays no longer touch either CTA's shared memory
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag && args.error_word) atomicExch(args.error_word, 1);
}

template <int kStages>
constexpr size_t pair_smem_bytes() {
  return 1024 + (size_t)kStages * (BM * BK * 2 + 128 * BK * 2) + (2 * kStages + 2) * 8 + 16;
}
constexpr int kPairStages = 6;

// ------------------------------------------------------------------ exact level GEMM
// The product of the exact refinement (solve.cu): for levels a = 0 .. L-1,
//   S_a[i][j] = sum_k A[i][a np + k] B[j][k],   A [M][Lmax np], B [N][np], both bf16 K-major,
// where every element of A is an integer of magnitude <= 128 and every element of B one of
// magnitude <= 127 (exact in bf16). Each product is then an integer of magnitude below 2^14
// and the sum of one 256-long chunk stays below 2^22, so the fp32 tensor-memory accumulator
// holds every chunk sum exactly whatever the order of its additions. The epilogue adds the
// chunk sums as int32 (exact for level sums below 2^31, i.e. np <= 131,072) and stores each
// level's sums as int32 to
// lev + (z Lmax + a) plane, row i at i ldl (z: the CTA's K split). L is read from device
// memory (written by an earlier kernel on the stream), so that the level count can be
// decided on the device. Warp roles as gemm_kernel; the epilogue has one group of four
// warps per 128 columns (a thread keeps its row's 128 int32 sums).
// Level count of an exact product from max|X| and max|D| (bits of non-negative doubles in
// words[1] and words[2]): the dropped levels (each 2^-8 of the previous) stay below 2^-bits of
// max|A| max|X|. Every kernel that needs the count evaluates it from the same words.
__device__ __forceinline__ int exact_level_count(const unsigned long long* words, int bits, int max_levels) {
  const unsigned long long xb = words[1], db = words[2];
  if (db == 0ull) return 1;
  if (xb == 0ull || xb >= 0x7ff0000000000000ull || db >= 0x7ff0000000000000ull) return max_levels;
  const int ed = (int)(db >> 52), ex = (int)(xb >> 52);  // biased exponents (0 for subnormals)
  const int L = (bits + (ed - ex) + 7) / 8;
  return L < 1 ? 1 : (L > max_levels ? max_levels : L);
}

struct ExactArgs {
  int M, N, np;          // rows and columns of S, K length of one level (multiple of 128)
  const int* levels;     // device int L (1 <= L <= max_levels), or null: L from level_words
  const unsigned long long* level_words;  // see exact_level_count
  int level_bits;
  int max_levels;
  int32_t* lev;          // [splits][max_levels][rows >= tiles_m BM][ldl]
  int64_t ldl, plane;    // row stride; stride of one (split, level) plane; ldl >= tiles_n BN
  int split_blocks;      // K blocks of one level per CTA z (0: all)
  int* error_word;
  const int* skip = nullptr;
  int* level_log = nullptr;  // kernel timer: the launch records L here (CTA 0, thread 0), or with
                             // flags the executed 256 x 256 x BK blocks (summed by the pairs)
  // Block flags of A (CTA-pair kernel only; null: every block): flags[(a flag_rows + tile) flag_ld
  // + kb] != 0 when the 256-row tile `tile` of level a's slice has a non-zero entry in K block kb;
  // flag_ld is a multiple of 16 (one chunk's flags are one 16-byte word).
  const uint8_t* flags = nullptr;
  int flag_rows = 0, flag_ld = 0;
};

// Chunks of a level in the CTA-pair kernel with block flags: at most kExactMaxChunks per level
// (np <= 32,768), and at most 8 levels.
constexpr int kExactMaxChunks = 32;

// 1,024-long K chunks (the last one of a level may be shorter): with operands |a| <= 128 and
// |b| <= 127 every partial sum of a chunk is an integer below 1,024 x 16,256 = 16,646,144 < 2^24,
// so the fp32 accumulation in tensor memory is exact, and the epilogue drains each chunk while
// the MMAs of the next one run.
constexpr int kExactChunkBlocks = 16;
__host__ __device__ constexpr int exact_groups(int BN) { return BN > 128 ? BN / 128 : 1; }
__host__ __device__ constexpr int exact_threads(int BN) { return 64 + 128 * exact_groups(BN); }

template <int BN, int kStages>
__global__ void __launch_bounds__(exact_threads(BN), 1)
    gemm_exact_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                      const ExactArgs args) {
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
  constexpr int kGroups = exact_groups(BN);
  constexpr int kCols = BN / kGroups;  // columns of one epilogue thread
  constexpr uint32_t kABytes = BM * BK * 2, kBBytes = BN * BK * 2;
  constexpr uint32_t kTmemCols = 2 * BN < 32 ? 32 : 2 * BN;
  constexpr uint32_t kIdesc = idesc_f16(BM, BN, true);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;  // [2]
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint64_t* drain = acc_empty + 2;       // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ int s_abort;
  __shared__ int s_consumed;

  const bool skipped = args.skip && *(volatile const int*)args.skip;
  const int L = skipped ? 0
                        : (args.levels ? *(volatile const int*)args.levels
                                       : exact_level_count(args.level_words, args.level_bits, args.max_levels));
  // the kernel timer's record of the levels this launch ran (0 when it skipped itself)
  if (args.level_log && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.z == 0) *args.level_log = L;
  if (skipped) return;  // uniform: before any barrier or allocation
  if (L < 1 || L > args.max_levels) {
    if (threadIdx.x == 0 && args.error_word) atomicExch(args.error_word, 1);
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (args.M + BM - 1) / BM, tiles_n = (args.N + BN - 1) / BN;
  const int pid = blockIdx.x;
  const int group = pid / (kGroupM * tiles_n);
  const int first_m = group * kGroupM;
  const int group_m = min(tiles_m - first_m, kGroupM);
  const int tile_m = first_m + (pid % (kGroupM * tiles_n)) % group_m;
  const int tile_n = (pid % (kGroupM * tiles_n)) / group_m;
  const int m0 = tile_m * BM, n0 = tile_n * BN;
  const int kb_level = args.np / BK;  // K blocks of one level
  const int kb_first = args.split_blocks > 0 ? blockIdx.z * args.split_blocks : 0;
  const int kb_per = args.split_blocks > 0 ? min(args.split_blocks, kb_level - kb_first) : kb_level;
  const int chunks_per_level = (kb_per + kExactChunkBlocks - 1) / kExactChunkBlocks;
  const int n_chunks = L * chunks_per_level;
  const int total_kb = L * kb_per;

  if (threadIdx.x == 0) {
    s_abort = 0;
    s_consumed = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128 * kGroups);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    // ---------------- TMA producer: level a, block kb of the CTA's K range
    if (lane == 0) {
      int issued = 0;
      for (int t = 0; t < total_kb; ++t) {
        const int s = t % kStages;
        if (t >= kStages && !mbar_wait(&empty[s], ((t / kStages) - 1) & 1)) { *abort_flag = 1; break; }
        if (*abort_flag) break;
        const int a = t / kb_per, kb = kb_first + t % kb_per;
        mbar_expect_tx(&full[s], kABytes + kBBytes);
        tma_load_2d(sA + s * kABytes, &map_a, &full[s], a * args.np + kb * BK, m0);
        tma_load_2d(sB + s * kBBytes, &map_b, &full[s], kb * BK, n0);
        ++issued;
      }
      if (*abort_flag) {
        for (int t = *(volatile int*)&s_consumed; t < issued; ++t) mbar_wait(&full[t % kStages], (t / kStages) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: one accumulation per chunk, two TMEM buffers
    if (lane == 0) {
      int t = 0;
      for (int c = 0; c < n_chunks && !*abort_flag; ++c) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(&acc_empty[b], ((c >> 1) - 1) & 1)) { *abort_flag = 1; break; }
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
        const int c_in = c % chunks_per_level;
        const int nq = min(kExactChunkBlocks, kb_per - c_in * kExactChunkBlocks);
        for (int q = 0; q < nq; ++q, ++t) {
          const int s = t % kStages;
          if (!mbar_wait(&full[s], (t / kStages) & 1)) { *abort_flag = 1; break; }
          *(volatile int*)&s_consumed = t + 1;
          tc_fence_after();
          const uint32_t a_addr = smem_u32(sA + s * kABytes), b_addr = smem_u32(sB + s * kBBytes);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            umma_f16(d_tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), kIdesc,
                     (q > 0 || kk > 0) ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (*abort_flag) break;
        umma_commit(&acc_full[b]);
      }
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
  } else {
    // ---------------- epilogue: int32 level sums, one row per thread
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int cbase = (ew >> 2) * kCols;
    const int row = m0 + quarter * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint32_t acc[kCols];
#pragma unroll
    for (int i = 0; i < kCols; ++i) acc[i] = 0u;
    int in_level = 0;
    for (int c = 0; c < n_chunks; ++c) {
      const int b = c & 1;
      if (!mbar_wait(&acc_full[b], (c >> 1) & 1)) { *abort_flag = 1; break; }
      tc_fence_after();
#pragma unroll
      for (int c0 = 0; c0 < kCols; c0 += 32) {
        float v[32];
        tmem_ld32(tmem_base + lane_addr + (uint32_t)(b * BN + cbase + c0), v);
        // v is an integer of magnitude below 2^24, exact in fp32: converted exactly
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[c0 + i] += (uint32_t)__float2int_rn(v[i]);
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[b]);
      if (++in_level == chunks_per_level) {
        const int a = c / chunks_per_level;
        int32_t* dst = args.lev + ((int64_t)blockIdx.z * args.max_levels + a) * args.plane + (int64_t)row * args.ldl +
                       n0 + cbase;
#pragma unroll
        for (int i = 0; i < kCols; i += 4) {
          int4 w;
          w.x = (int32_t)acc[i];
          w.y = (int32_t)acc[i + 1];
          w.z = (int32_t)acc[i + 2];
          w.w = (int32_t)acc[i + 3];
          *reinterpret_cast<int4*>(dst + i) = w;
          acc[i] = acc[i + 1] = acc[i + 2] = acc[i + 3] = 0u;
        }
        in_level = 0;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag && args.error_word) atomicExch(args.error_word, 1);
}

template <int BN, int kStages>
constexpr size_t exact_smem_bytes() {
  return 1024 + (size_t)kStages * (BM * BK * 2 + BN * BK * 2) + (2 * kStages + 5) * 8 + 16;
}

// gemm_exact_kernel on CTA pairs (cluster of 2, cta_group::2), 256 x 256 tiles: each CTA
// loads its 128 rows of the slices and 128 of the tile's 256 rows of B per K block (32 KB a
// stage, kPairStages of them), the even CTA's thread issues the MMAs of the pair into both
// CTAs' two chunk accumulators (512 tensor-memory columns in each), and each CTA's epilogue
// adds and stores the level sums of its own 128 rows. A chunk buffer is free again once all
// eight epilogue warps of the pair have drained it (one arrival per warp on the even CTA's
// acc_empty; the odd CTA's warps arrive remotely). Level count, chunking, splits and stores
// as gemm_exact_kernel.
template <int kStages>
__global__ void __launch_bounds__(exact_threads(256), 1) __cluster_dims__(2, 1, 1)
    gemm_exact_pair_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                           const ExactArgs args) {
  constexpr int PN = 256;
  constexpr int kGroups = exact_groups(PN);  // 2 epilogue groups of four warps (128 columns each)
  constexpr int kCols = PN / kGroups;
  constexpr int kEpiWarps = 4 * kGroups;
  constexpr uint32_t kABytes = BM * BK * 2, kBBytes = (PN / 2) * BK * 2;
  constexpr uint32_t kTmemCols = 2 * PN;
  constexpr uint32_t kIdesc = idesc_f16(2 * BM, PN, true);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;  // [2]
  uint64_t* acc_empty = acc_full + 2;    // [2] (even CTA)
  uint64_t* drain = acc_empty + 2;       // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ int s_abort;
  __shared__ uint16_t s_mask[kExactMaxChunks * 8];  // [level][chunk]: the chunk's non-zero blocks
  // per epilogue warp: 32 rows x 16 columns of level sums on their way to HBM (rows 80 bytes
  // apart: 16-byte aligned, and the eight rows of a quarter-warp's stores in distinct banks)
  __shared__ __align__(16) uint32_t s_out[8][32][20];

  const bool skipped = args.skip && *(volatile const int*)args.skip;
  const int L = skipped ? 0
                        : (args.levels ? *(volatile const int*)args.levels
                                       : exact_level_count(args.level_words, args.level_bits, args.max_levels));
  const bool flagged = args.flags != nullptr;
  if (args.level_log && !flagged && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.z == 0) *args.level_log = L;
  if (skipped) return;  // uniform over the pair: before any barrier or allocation
  if (L < 1 || L > args.max_levels) {
    if (threadIdx.x == 0 && args.error_word) atomicExch(args.error_word, 1);
    return;
  }
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (args.M + 2 * BM - 1) / (2 * BM), tiles_n = (args.N + PN - 1) / PN;
  const int pid = blockIdx.x >> 1;
  const int group = pid / (kGroupM * tiles_n);
  const int first_m = group * kGroupM;
  const int group_m = min(tiles_m - first_m, kGroupM);
  const int tile_m = first_m + (pid % (kGroupM * tiles_n)) % group_m;
  const int tile_n = (pid % (kGroupM * tiles_n)) / group_m;
  const int m0 = tile_m * 2 * BM + (int)rank * BM;
  const int nb0 = tile_n * PN + (int)rank * (PN / 2);
  const int n0 = tile_n * PN;
  const int kb_level = args.np / BK;
  const int kb_first = args.split_blocks > 0 ? blockIdx.z * args.split_blocks : 0;
  const int kb_per = args.split_blocks > 0 ? min(args.split_blocks, kb_level - kb_first) : kb_level;
  const int chunks_per_level = (kb_per + kExactChunkBlocks - 1) / kExactChunkBlocks;
  if (L * chunks_per_level > kExactMaxChunks * 8) {  // the mask table holds 8 levels of 32 chunks
    if (threadIdx.x == 0 && args.error_word) atomicExch(args.error_word, 1);
    return;  // uniform over the pair: before any barrier or allocation
  }
  // the blocks of chunk c of level a that hold non-zero entries of A (bit q: block 16 c + q);
  // both CTAs of a pair read the same flags (the pair's 256-row tile), so every role of both
  // walks the same sequence of blocks. An accumulation takes up to kExactChunkBlocks of a
  // level's flagged blocks in K order, wherever they lie: the bound on its partial sums
  // counts the products it adds, not the K range they span
  for (int idx = threadIdx.x; idx < L * chunks_per_level; idx += blockDim.x) {
    const int a = idx / chunks_per_level, c = idx % chunks_per_level;
    const int nq = min(kExactChunkBlocks, kb_per - c * kExactChunkBlocks);
    unsigned msk = (1u << nq) - 1u;
    if (flagged) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(
          args.flags + ((int64_t)a * args.flag_rows + tile_m) * args.flag_ld + c * kExactChunkBlocks));
      const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
      unsigned f = 0u;
#pragma unroll
      for (int q = 0; q < 16; ++q) f |= ((wd[q >> 2] >> (8 * (q & 3))) & 0xffu) ? (1u << q) : 0u;
      msk &= f;
    }
    s_mask[idx] = (uint16_t)msk;
  }
  auto chunk_mask = [&](int a, int c) -> unsigned { return s_mask[a * chunks_per_level + c]; };
  // flagged blocks of level a (the accumulations of the level: ceil(/ kExactChunkBlocks))
  auto level_blocks = [&](int a) -> int {
    int k = 0;
    for (int c = 0; c < chunks_per_level; ++c) k += __popc(chunk_mask(a, c));
    return k;
  };

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], leader ? 2 : 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 2 * kEpiWarps);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc_pair(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs): level a, block kb of the CTA's K range
    if (lane == 0) {
      int t = 0;
      for (int g = 0; g < L * chunks_per_level && !*abort_flag; ++g) {
        const int a = g / chunks_per_level, c = g % chunks_per_level;
        for (unsigned msk = chunk_mask(a, c); msk; msk &= msk - 1u, ++t) {
          const int s = t % kStages;
          if (t >= kStages && !mbar_wait_cluster(&empty[s], ((t / kStages) - 1) & 1)) { *abort_flag = 1; break; }
          if (*abort_flag) break;
          const int kb = kb_first + c * kExactChunkBlocks + (__ffs(msk) - 1);
          mbar_expect_tx(&full[s], kABytes + kBBytes);
          tma_load_2d(sA + s * kABytes, &map_a, &full[s], a * args.np + kb * BK, m0);
          tma_load_2d(sB + s * kBBytes, &map_b, &full[s], kb * BK, nb0);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (leader) {
        // ---------------- MMA issuer of the pair: one accumulation per chunk, two buffers
        // accumulations of up to kExactChunkBlocks flagged blocks of one level; cc counts them
        // (the accumulator buffers and their phases follow cc)
        int t = 0, cc = 0;
        for (int a = 0; a < L && !*abort_flag; ++a) {
          int q = 0;  // blocks in the open accumulation
          uint32_t d_tmem = 0;
          for (int c = 0; c < chunks_per_level && !*abort_flag; ++c)
            for (unsigned msk = chunk_mask(a, c); msk; msk &= msk - 1u, ++t) {
              if (q == 0) {
                const int b = cc & 1;
                if (cc >= 2 && !mbar_wait_cluster(&acc_empty[b], ((cc >> 1) - 1) & 1)) { *abort_flag = 1; break; }
                d_tmem = tmem_base + (uint32_t)(b * PN);
              }
              const int s = t % kStages;
              if (!mbar_wait_cluster(&full[s], (t / kStages) & 1)) { *abort_flag = 1; break; }
              tc_fence_after();
              const uint32_t a_addr = smem_u32(sA + s * kABytes), b_addr = smem_u32(sB + s * kBBytes);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                umma_f16_pair(d_tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), kIdesc,
                              (q > 0 || kk > 0) ? 1u : 0u);
              umma_commit_pair_both(&empty[s]);
              if (++q == kExactChunkBlocks) {
                umma_commit_pair_both(&acc_full[cc & 1]);
                ++cc;
                q = 0;
              }
            }
          if (*abort_flag) break;
          if (q > 0) {
            umma_commit_pair_both(&acc_full[cc & 1]);
            ++cc;
          }
        }
        if (flagged && args.level_log) atomicAdd(args.level_log, t);
        if (t > 0) {  // a tile without flagged blocks issued no MMA: nothing to wait for
          umma_commit_pair_local(drain);
          mbar_wait(drain, 0);
        }
      } else {
        // ---------------- relay of this CTA's full stages to the even CTA
        const uint32_t leader_full = mapa_shared(smem_u32(full), 0);
        int total = 0;
        for (int g = 0; g < L * chunks_per_level; ++g)
          total += __popc(chunk_mask(g / chunks_per_level, g % chunks_per_level));
        for (int t = 0; t < total; ++t) {
          const int s = t % kStages;
          if (!mbar_wait(&full[s], (t / kStages) & 1)) { *abort_flag = 1; break; }
          mbar_arrive_remote(leader_full + 8u * (uint32_t)s);
        }
      }
    }
  } else {
    // ---------------- epilogue: int32 level sums of this CTA's rows, one row per thread
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int cbase = (ew >> 2) * kCols;
    const int row = m0 + quarter * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    const uint32_t empty_addr = mapa_shared(smem_u32(acc_empty), 0);  // the even CTA's, from either CTA
    uint32_t acc[kCols];
#pragma unroll
    for (int i = 0; i < kCols; ++i) acc[i] = 0u;
    int cc = 0;
    for (int a = 0; a < L && !*abort_flag; ++a) {
      const int groups = (level_blocks(a) + kExactChunkBlocks - 1) / kExactChunkBlocks;
      for (int gi = 0; gi < groups; ++gi) {  // a level without blocks: nothing to drain, zero sums
        const int b = cc & 1;
        if (!mbar_wait_cluster(&acc_full[b], (cc >> 1) & 1)) { *abort_flag = 1; break; }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < kCols; c0 += 16) {
          float v[16];
          tmem_ld16(tmem_base + lane_addr + (uint32_t)(b * PN + cbase + c0), v);
          // v is an integer of magnitude below 2^24, exact in fp32: converted exactly
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[c0 + i] += (uint32_t)__float2int_rn(v[i]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_remote(empty_addr + 8u * (uint32_t)b);
        ++cc;
      }
      if (*abort_flag) break;
      {
        // the warp's 32 rows go out 16 columns at a time through shared memory, so that each
        // store instruction writes eight rows' 64 contiguous bytes (rows at and beyond M land
        // in the plane's padding: exact_plane rounds M up to 256); streaming stores, so that
        // the level sums (gigabytes per launch) do not evict the operand tiles from L2
        uint32_t(*buf)[20] = s_out[ew];
        int32_t* plane = args.lev + ((int64_t)blockIdx.z * args.max_levels + a) * args.plane +
                         (int64_t)(m0 + quarter * 32) * args.ldl + n0 + cbase;
#pragma unroll
        for (int i0 = 0; i0 < kCols; i0 += 16) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            *reinterpret_cast<uint4*>(&buf[lane][4 * q]) =
                make_uint4(acc[i0 + 4 * q], acc[i0 + 4 * q + 1], acc[i0 + 4 * q + 2], acc[i0 + 4 * q + 3]);
            acc[i0 + 4 * q] = acc[i0 + 4 * q + 1] = acc[i0 + 4 * q + 2] = acc[i0 + 4 * q + 3] = 0u;
          }
          __syncwarp();
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int v = lane + 32 * k, r = v >> 2, q = v & 3;
            __stcs(reinterpret_cast<uint4*>(plane + (int64_t)r * args.ldl + i0 + 4 * q),
                   *reinterpret_cast<const uint4*>(&buf[r][4 * q]));
          }
          __syncwarp();
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag && args.error_word) atomicExch(args.error_word, 1);
}

template <int kStages>
constexpr size_t exact_pair_smem_bytes() {
  return 1024 + (size_t)kStages * (BM * BK * 2 + 128 * BK * 2) + (2 * kStages + 5) * 8 + 16;
}


// ------------------------------------------------------------------ host side
// Launch D = A B^T (A [M x K], B [N x K], 16-bit K-major) with the epilogue `epi`;
// instantiated in gemm.cu for the epilogues above (bf16 selects the operand type).
// sym: the product is symmetric (A B^T with M = N, e.g. two commuting symmetric matrices);
// where the tiles are square only those on and above the diagonal are computed and the
// epilogue writes the off-diagonal ones for their transposes too (the Newton-Schulz epilogues
// with their own `sym` set), else the whole product is computed.
// aflags, bflags (optional): A's and B's block flags, [ceil(M / 256)] and [ceil(N / 256)] rows of
// ceil(K / 64 / 32) 32 bytes (GemmArgs); the CTA-pair kernel skips the K blocks where either
// operand's tile is all zero (the others ignore the flags).
template <class Epi>
rg_status gemm(rg_ctx* ctx, bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
               const Epi& epi, cudaStream_t s, const int* skip = nullptr, bool sym = false,
               const uint8_t* aflags = nullptr, const uint8_t* bflags = nullptr);

// C (fp32, ldc) = alpha * A B^T + beta * C with A [M x K] (lda), B [N x K] (ldb), 16-bit
// K-major operands (bf16 when `bf16`, else fp16). lda, ldb: multiples of 8 elements;
// A, B: 16-byte aligned.
rg_status gemm_f32(rg_ctx* ctx, bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N,
                   int K, float* C, int64_t ldc, float alpha, float beta, cudaStream_t s);

// The exact level product of the refinement (gemm_exact_kernel): S_a = A_a B^T for the
// L levels that *levels_d names, int32 sums to lev (see ExactArgs); tiles of 128 x 256 where
// they give every SM a tile, else narrower; K split over up to split_max CTAs per tile when
// the tiles leave SMs idle. lev needs split_max x max_levels planes of
// exact_plane(M, N) int32 (rows rounded up to 256); *splits_out receives the splits used. alg_k: the inner dimension of
// the product the launch stands for (kernel timer accounting).
int64_t exact_ld(int N);
int64_t exact_plane(int M, int N);
// The level count comes from levels_d (device int) or, when that is null, from
// exact_level_count(level_words, level_bits, max_levels).
// flags (optional, see ExactArgs): block flags of A, [max_levels][flag_rows >= ceil(M / 256)]
// [flag_ld >= np / BK rounded up to 16] bytes; the CTA-pair kernel skips the blocks of A that
// hold only zeros (the others ignore the flags).
rg_status gemm_exact(rg_ctx* ctx, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int np,
                     const int* levels_d, const unsigned long long* level_words, int level_bits, int max_levels,
                     int32_t* lev, int split_max, int* splits_out, cudaStream_t s, const int* skip = nullptr,
                     int alg_k = 0, const uint8_t* flags = nullptr, int flag_rows = 0, int flag_ld = 0);

// Device error word the GEMM kernels raise on a timed-out wait (ctx scratch slot).
constexpr int kGemmErrorSlot = 16;

}  // namespace tc
