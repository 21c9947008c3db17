// tcgen05 GEMM for sm_103a: D[M x N] = A[M x K] * B[N x K]^T, 16-bit operands (bf16 or
// fp16, both K-major: row-major with K contiguous), fp32 accumulation in tensor memory.
//
// One CTA computes one BM x BN tile (BM = 128). Warp roles (192 threads; 320 for
// compensated 128-wide tiles):
//   warp 0      TMA producer: 64-wide K blocks of A and B into a ring of smem stages
//               (128-byte swizzle), completion signalled on full[s] mbarriers;
//   warp 1      allocates TMEM, one elected thread issues tcgen05.mma (K = 16 each)
//               and commits to empty[s] (stage free) and acc_full[b] (accumulator ready);
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM lanes
//               32*(w%4) .. +31, i.e. tile rows), then the Epi functor writes the result;
//               a compensated tile wider than 64 columns has one group of four epilogue
//               warps per 64 columns (warps 6..9 take columns 64..127), so that a thread
//               keeps 64 compensated sums.
// The K loop can be cut into chunks of kChunkBlocks K blocks: each chunk is accumulated
// in fp32 in one of two TMEM buffers and handed to the epilogue, which folds it into a
// compensated (Kahan) fp32 sum; this keeps the long reductions of the refinement
// residual accurate to ~1e-7 relative while the tensor cores run in 16-bit.
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
// epilogue warp groups of a tile: compensated tiles give every group 64 columns
template <int BN, bool kCompensated>
__host__ __device__ constexpr int epi_groups() { return (kCompensated && BN > 64) ? BN / 64 : 1; }
template <int BN, bool kCompensated>
__host__ __device__ constexpr int cta_threads() { return 64 + 128 * epi_groups<BN, kCompensated>(); }
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

// 16 columns of fp32 accumulator for the warp's 32 TMEM lanes (the compensated drain of
// wide tiles reads half-slabs: 16 fewer registers in flight next to its Kahan state).
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

// ------------------------------------------------------------------ fp64 maxima on the bit pattern
// GB300 runs fp64 min/max on a pipe far slower than its integer ALU; the compensated
// epilogue folds two maxima per element, as the bit patterns of |x|.

// |x| as its bit pattern, 0 for a NaN: the maximum of these orders like fmax of |x|.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  return a > 0x7ff0000000000000ull ? 0ull : a;
}
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

template <class T16>
__device__ __forceinline__ T16 to_16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_16<__half>(float x) { return __float2half_rn(x); }

// C[r][c] = beta * C[r][c] + alpha * acc   (fp32 C)
struct EpiF32 {
  float* C;
  int64_t ldc;
  float alpha, beta;
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, const float* v,
                                        float (*stage)[33]) const {
    staged_rows(row0, lane, c0, M, N, v, stage, [&](int r, int c, float x) {
      float* p = C + (int64_t)r * ldc + c;
      *p = (beta == 0.f ? 0.f : beta * *p) + alpha * x;
    });
  }
};

// Newton-Schulz half step: Zt[c][r] = 16-bit (2 delta_rc - acc) -- the transposed store is
// coalesced as it is (the warp's 32 rows are 32 consecutive elements of a row of Zt).
template <class T16>
struct EpiTwoIMinusT {
  T16* Zt;
  int64_t ld;
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, const float* v,
                                        float (*)[33]) const {
    const int r = row0 + lane;
    if (r >= M) return;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
      const int c = c0 + i;
      if (c < N) Zt[(int64_t)c * ld + r] = to_16<T16>((r == c ? 2.f : 0.f) - v[i]);
    }
  }
};

// Newton-Schulz step result: X[r][c] and Xt[c][r] = 16-bit acc.
template <class T16>
struct EpiStore16Both {
  T16* X;
  T16* Xt;
  int64_t ld;
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, const float* v,
                                        float (*stage)[33]) const {
    const int r = row0 + lane;
    if (r < M) {
#pragma unroll 8
      for (int i = 0; i < 32; ++i) {
        const int c = c0 + i;
        if (c < N) Xt[(int64_t)c * ld + r] = to_16<T16>(v[i]);
      }
    }
    staged_rows(row0, lane, c0, M, N, v, stage, [&](int rr, int c, float x) { X[(int64_t)rr * ld + c] = to_16<T16>(x); });
  }
};

// Epilogues that read fp64 operands of the output tile go through the staging block in
// batches of kRowBatch rows: the loads of a batch are issued together, so a warp waits
// for one memory latency per batch rather than one per row.
constexpr int kRowBatch = 8;

// X64[r][c] = (first ? 0 : X64[r][c]) + acc * colscale[c]   (the refinement correction)
struct EpiAddF64 {
  double* X;
  int64_t ld;
  const float* colscale;
  int first;
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, const float* v,
                                        float (*stage)[33]) const {
#pragma unroll
    for (int i = 0; i < 32; ++i) stage[lane][i] = v[i];
    __syncwarp();
    const int c = c0 + lane;
    const bool cok = c < N;
    const double cs = cok ? (double)colscale[c] : 0.0;
#pragma unroll 1
    for (int rb = 0; rb < 32; rb += kRowBatch) {
      double old[kRowBatch];
#pragma unroll
      for (int q = 0; q < kRowBatch; ++q) {
        const int r = row0 + rb + q;
        old[q] = (!first && cok && r < M) ? X[(int64_t)r * ld + c] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < kRowBatch; ++q) {
        const int r = row0 + rb + q;
        if (cok && r < M) {
          const double d = (double)stage[rb + q][lane] * cs;
          X[(int64_t)r * ld + c] = first ? d : old[q] + d;
        }
      }
    }
    __syncwarp();
  }
};

// Largest non-negative double into *dst (its bit pattern orders like the value).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* dst, double x) {
  atomicMax(dst, (unsigned long long)__double_as_longlong(x));
}

// out[r][c] = E[r][c] - X[r][c] + dl[r] * acc   (fp64; the refinement residual), or
// out[r][c] = dl[r] * acc when E is null (an fp64-accurate product). With `red` set it
// also folds max|out| into red[0], max|X| into red[1], max_r |out[r][c]| into
// colmax[c] (all as double bits) and raises *nonfinite on an inf or NaN.
struct EpiResidual {
  double* out;
  const double* E;   // may be null together with X
  const double* X;
  const double* dl;  // may be null (identity)
  int64_t ld;        // shared leading dimension of out, E and X
  unsigned long long* red = nullptr;     // [2], zeroed by the caller
  unsigned long long* colmax = nullptr;  // [N], zeroed by the caller (may be null)
  int* nonfinite = nullptr;
  double* partial = nullptr;             // split K: CTA z writes its raw sum to partial + z * split_stride
  int64_t split_stride = 0;
  // The caller has written the warp's 32 x 32 block into stage (stage[l][i]: row
  // row0 + l, column c0 + i), so that no register array of it stays live here.
  __device__ __forceinline__ void store(int row0, int lane, int c0, int M, int N, double (*stage)[33], int z) const {
    __syncwarp();
    const int c = c0 + lane;
    if (partial) {
      double* dst = partial + (int64_t)z * split_stride;
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr) {
        const int r = row0 + rr;
        if (r < M && c < N) dst[(int64_t)r * ld + c] = stage[rr][lane];
      }
      __syncwarp();
      return;
    }
    unsigned long long m_out = 0ull, m_x = 0ull;  // bit patterns of the maxima (abs_bits)
    bool bad = false;
    const bool cok = c < N;
#pragma unroll 1
    for (int rb = 0; rb < 32; rb += kRowBatch) {
      double e[kRowBatch], xo[kRowBatch], s[kRowBatch];
#pragma unroll
      for (int q = 0; q < kRowBatch; ++q) {
        const int r = row0 + rb + q;
        const bool ok = cok && r < M;
        const int64_t i = (int64_t)r * ld + c;
        e[q] = (ok && E) ? E[i] : 0.0;
        xo[q] = (ok && E) ? X[i] : 0.0;
        s[q] = (r < M && dl) ? dl[r] : 1.0;
      }
#pragma unroll
      for (int q = 0; q < kRowBatch; ++q) {
        const int r = row0 + rb + q;
        if (!(cok && r < M)) continue;
        const double x = stage[rb + q][lane];
        const double o = E ? (e[q] - xo[q]) + s[q] * x : s[q] * x;
        out[(int64_t)r * ld + c] = o;
        m_out = max(m_out, abs_bits(o));
        m_x = max(m_x, abs_bits(xo[q]));
        bad |= !finite_bits(o) || !finite_bits(xo[q]);
      }
    }
    __syncwarp();
    if (red) {
      // this lane saw column c0 + lane of the warp's 32 rows
      if (colmax && c0 + lane < N) atomicMax(&colmax[c0 + lane], m_out);
      for (int o = 16; o > 0; o >>= 1) {
        m_out = max(m_out, __shfl_xor_sync(0xffffffffu, m_out, o));
        m_x = max(m_x, __shfl_xor_sync(0xffffffffu, m_x, o));
      }
      bad = __any_sync(0xffffffffu, bad);
      if (lane == 0) {
        atomicMax(&red[0], m_out);
        atomicMax(&red[1], m_x);
        if (bad && nonfinite) atomicExch(nonfinite, 1);
      }
    }
  }
};

struct GemmArgs {
  int M, N, K;
  int chunk_blocks;  // 0: one fp32 accumulation over all of K; > 0: compensated chunks
  int* error_word;
  int split_blocks = 0;  // > 0: CTA z covers K blocks [z * split_blocks, (z + 1) * split_blocks)
  // > 0 (compensated, unsplit): only the first lead_blocks K blocks use chunks of
  // chunk_blocks; the rest use chunks of tail_chunk_blocks
  int lead_blocks = 0;
  int tail_chunk_blocks = 0;
  // non-null: the kernel does nothing when *skip != 0 (written by an earlier kernel on
  // the stream; a speculatively launched product the host's decision made unnecessary)
  const int* skip = nullptr;
  // > 0: the inner dimension of the product the launch stands for (kernel timer accounting)
  int alg_k = 0;
};

template <int BN, int kStages, class Epi, bool kCompensated, bool kBF16>
__global__ void __launch_bounds__(cta_threads<BN, kCompensated>(), 1)
    gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                const GemmArgs args, const Epi epi) {
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
  constexpr int kGroups = epi_groups<BN, kCompensated>();
  constexpr int kEpiCols = BN / kGroups;  // columns of one epilogue thread
  static_assert(!kCompensated || kEpiCols == 64, "the compensated epilogue keeps 2 x 64 registers per thread");
  constexpr uint32_t kABytes = BM * BK * 2, kBBytes = BN * BK * 2;
  constexpr uint32_t kAccCols = kCompensated ? 2 * BN : BN;
  constexpr uint32_t kTmemCols = kAccCols <= 32 ? 32 : (kAccCols <= 64 ? 64 : (kAccCols <= 128 ? 128 : (kAccCols <= 256 ? 256 : 512)));
  constexpr uint32_t kIdesc = idesc_f16(BM, BN, kBF16);
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
  __shared__ int s_consumed;             // K blocks whose stage the MMA thread has taken
  using StageT = typename std::conditional<kCompensated, double, float>::type;
  __shared__ StageT s_stage[4 * kGroups][32][33];  // per epilogue warp: coalescing block

  if (args.skip && *(volatile const int*)args.skip) return;  // uniform: before any barrier or allocation
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped rasterisation of the 1-D grid: kGroupM row tiles at a time, column tiles
  // innermost, so that the CTAs resident together share their A and B tiles in L2
  const int tiles_m = (args.M + BM - 1) / BM, tiles_n = (args.N + BN - 1) / BN;
  const int pid = blockIdx.x;
  const int group = pid / (kGroupM * tiles_n);
  const int first_m = group * kGroupM;
  const int group_m = min(tiles_m - first_m, kGroupM);
  const int tile_m = first_m + (pid % (kGroupM * tiles_n)) % group_m;
  const int tile_n = (pid % (kGroupM * tiles_n)) / group_m;
  const int m0 = tile_m * BM, n0 = tile_n * BN;
  const int kb_all = (args.K + BK - 1) / BK;
  // split K: this CTA's K blocks are kb_first .. kb_first + kb_total - 1
  const int kb_first = args.split_blocks > 0 ? blockIdx.z * args.split_blocks : 0;
  const int kb_total = args.split_blocks > 0 ? min(args.split_blocks, kb_all - kb_first) : kb_all;
  const int chunk = (kCompensated && args.chunk_blocks > 0) ? args.chunk_blocks : kb_total;
  // chunk schedule: n_lead chunks of `chunk` K blocks, then chunks of `tail` blocks
  const bool two_part = kCompensated && args.chunk_blocks > 0 && args.lead_blocks > 0 &&
                        args.tail_chunk_blocks > 0 && args.lead_blocks < kb_total;
  const int n_lead = two_part ? args.lead_blocks / chunk : 0;
  const int tail = two_part ? args.tail_chunk_blocks : chunk;
  const int n_chunks = n_lead + (kb_total - n_lead * chunk + tail - 1) / tail;

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
    // ---------------- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < kb_total; ++kb) {
        const int s = kb % kStages;
        if (kb >= kStages && !mbar_wait(&empty[s], ((kb / kStages) - 1) & 1)) { *abort_flag = 1; break; }
        if (*abort_flag) break;
        mbar_expect_tx(&full[s], kABytes + kBBytes);
        tma_load_2d(sA + s * kABytes, &map_a, &full[s], (kb_first + kb) * BK, m0);
        tma_load_2d(sB + s * kBBytes, &map_b, &full[s], (kb_first + kb) * BK, n0);
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
      int kb = 0;
      for (int c = 0; c < n_chunks && !*abort_flag; ++c) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(&acc_empty[b], ((c >> 1) - 1) & 1)) { *abort_flag = 1; break; }
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
        const int first = kb, kb_end = min(kb_total, kb + (c < n_lead ? chunk : tail));
        for (; kb < kb_end; ++kb) {
          const int s = kb % kStages;
          if (!mbar_wait(&full[s], (kb / kStages) & 1)) { *abort_flag = 1; break; }
          *(volatile int*)&s_consumed = kb + 1;
          tc_fence_after();
          const uint32_t a_addr = smem_u32(sA + s * kABytes), b_addr = smem_u32(sB + s * kBBytes);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            umma_f16(d_tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), kIdesc,
                     (kb > first || kk > 0) ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (*abort_flag) break;
        umma_commit(&acc_full[b]);
      }
      // every MMA this thread issued has completed once `drain` fires
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
  } else {
    // ---------------- epilogue warps 2 .. 1 + 4 kGroups
    const int ew = warp - 2;
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int cbase = (ew >> 2) * kEpiCols;
    const int row0 = m0 + quarter * 32;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    StageT (*stage)[33] = s_stage[ew];
    if constexpr (!kCompensated) {
      if (mbar_wait(&acc_full[0], 0)) {
        tc_fence_after();
        float v[32];
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
          tmem_ld32(tmem_base + lane_addr + (uint32_t)c0, v);
          epi.store(row0, lane, n0 + c0, args.M, args.N, v, stage);
        }
      } else {
        *abort_flag = 1;
      }
    } else {
      float sum[kEpiCols], comp[kEpiCols];
#pragma unroll
      for (int i = 0; i < kEpiCols; ++i) {
        sum[i] = 0.f;
        comp[i] = 0.f;
      }
      bool ok = true;
      for (int c = 0; c < n_chunks; ++c) {
        const int b = c & 1;
        if (!mbar_wait(&acc_full[b], (c >> 1) & 1)) { *abort_flag = 1; ok = false; break; }
        tc_fence_after();
        // drain in 32-column loads, or 16-column ones where the CTA's 10 warps leave each
        // thread 168 registers (wide tiles) and the Kahan state of 64 columns needs 128
        constexpr int kDrain = BN > 64 ? 16 : 32;
#pragma unroll
        for (int c0 = 0; c0 < kEpiCols; c0 += kDrain) {
          float v[kDrain];
          if constexpr (kDrain == 16)
            tmem_ld16(tmem_base + lane_addr + (uint32_t)(b * BN + cbase + c0), v);
          else
            tmem_ld32(tmem_base + lane_addr + (uint32_t)(b * BN + cbase + c0), v);
#pragma unroll
          for (int i = 0; i < kDrain; ++i) {  // Kahan: sum + v, the lost low part kept in comp
            float y = v[i] - comp[c0 + i];
            float t = sum[c0 + i] + y;
            comp[c0 + i] = (t - sum[c0 + i]) - y;
            sum[c0 + i] = t;
          }
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[b]);
      }
      if (ok) {
#pragma unroll
        for (int c0 = 0; c0 < kEpiCols; c0 += 32) {
#pragma unroll
          for (int i = 0; i < 32; ++i) stage[lane][i] = (double)sum[c0 + i] - (double)comp[c0 + i];
          epi.store(row0, lane, n0 + cbase + c0, args.M, args.N, stage, blockIdx.z);
        }
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
constexpr size_t smem_bytes() {
  return 1024 + (size_t)kStages * (BM * BK * 2 + BN * BK * 2) + (2 * kStages + 5) * 8 + 16;
}

// ------------------------------------------------------------------ host side
// Launch D = A B^T (A [M x K], B [N x K], 16-bit K-major) with the epilogue `epi`;
// instantiated in gemm.cu for the epilogues above (bf16 selects the operand type).
template <class Epi>
rg_status gemm(rg_ctx* ctx, bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
               const Epi& epi, cudaStream_t s, const int* skip = nullptr);

// C (fp32, ldc) = alpha * A B^T + beta * C with A [M x K] (lda), B [N x K] (ldb), 16-bit
// K-major operands (bf16 when `bf16`, else fp16). lda, ldb: multiples of 8 elements;
// A, B: 16-byte aligned.
rg_status gemm_f32(rg_ctx* ctx, bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N,
                   int K, float* C, int64_t ldc, float alpha, float beta, cudaStream_t s);

// out (fp64, ld) = E - X + dl o (A B^T) (or dl o (A B^T) when E is null), bf16 operands,
// fp32 tensor-core accumulation in chunks of `chunk_blocks` x 64 of K folded into a
// compensated sum.
// With split_ws (room for split_max x M x ld doubles) and too few 128 x 64 tiles to fill
// the GPU, K is split over up to split_max CTAs per tile (in whole chunks); their sums go
// to split_ws and one more kernel adds them in a fixed order and applies the epilogue.
//
// lead_blocks / tail_chunk_blocks (unsplit products only): after the first lead_blocks
// K blocks the chunks grow to tail_chunk_blocks (the refinement residual's leading slice
// pair needs the short compensated chunks; the pairs after it are 2^8 smaller and do with
// long ones).
rg_status gemm_residual(rg_ctx* ctx, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
                        int chunk_blocks, double* out, const double* E, const double* X, const double* dl,
                        int64_t ld, cudaStream_t s, unsigned long long* red = nullptr,
                        unsigned long long* colmax = nullptr, int* nonfinite = nullptr, double* split_ws = nullptr,
                        int split_max = 0, int lead_blocks = 0, int tail_chunk_blocks = 0, int alg_k = 0);

// K splits gemm_residual uses for an M x N product (1: none).
int residual_splits(const rg_ctx* ctx, int M, int N, int K, int chunk_blocks, int split_max);

// Device error word the GEMM kernels raise on a timed-out wait (ctx scratch slot).
constexpr int kGemmErrorSlot = 16;

}  // namespace tc
