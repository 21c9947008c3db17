// Host launchers of the tcgen05 GEMM (tc_gemm.cuh): tensor-map encoding and dispatch.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_gemm.cuh"

namespace tc {
namespace {

rg_status encode_kmajor(rg_ctx* ctx, CUtensorMap* map, const void* base, bool bf16, int64_t rows, int64_t cols,
                        int64_t ld, int box_rows);

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;

rg_status get_encoder(rg_ctx* ctx) {
  std::call_once(g_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) return rg::fail(ctx, RG_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  return RG_OK;
}

// 2-D K-major tile map: box of 64 (K) x box_rows, 128-byte swizzle, zero fill outside.
rg_status encode_kmajor(rg_ctx* ctx, CUtensorMap* map, const void* base, bool bf16, int64_t rows, int64_t cols,
                        int64_t ld, int box_rows) {
  rg_status st = get_encoder(ctx);
  if (st != RG_OK) return st;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16 || rows <= 0 || cols <= 0)
    return rg::fail(ctx, RG_ERR_ARG, "GEMM operand layout: base %p ld %lld", base, (long long)ld);
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return rg::fail(ctx, RG_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return RG_OK;
}

template <int BN, int kStages, class Epi, bool kComp, bool kBF16>
rg_status launch(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& args, const Epi& epi,
                 cudaStream_t s, int grid_z = 1);

// Tile width: the widest of 256 / 128 / 64 that still gives every SM two tiles. A wider
// tile reuses each A tile over more columns: a 128 x 128 x 64 step moves 32 KB for 2.1
// MFLOP (64 FLOP/B, ~35 TB/s from L2 at the tensor peak), a 128 x 256 x 64 step 48 KB
// for 4.2 MFLOP (87 FLOP/B).
int tile_width(const rg_ctx* ctx, int M, int N) {
  const int64_t tm = (M + BM - 1) / BM, want = 2 * (int64_t)ctx->sm_count;
  if (tm * ((N + 255) / 256) >= want) return 256;
  if (tm * ((N + 127) / 128) >= want) return 128;
  return 64;
}

}  // namespace

template <class Epi>
rg_status gemm(rg_ctx* ctx, bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
               const Epi& epi, cudaStream_t s, const int* skip) {
  if (M <= 0 || N <= 0) return RG_OK;
  if (K <= 0) return rg::fail(ctx, RG_ERR_ARG, "gemm: K = %d", K);
  const int bn = tile_width(ctx, M, N);
  CUtensorMap ma, mb;
  rg_status st = encode_kmajor(ctx, &ma, A, bf16, M, K, lda, BM);
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, bf16, N, K, ldb, bn);
  if (st != RG_OK) return st;
  GemmArgs args{M, N, K, 0, ctx->d_scratch + kGemmErrorSlot};
  args.skip = skip;
  if (bn == 64)
    return bf16 ? launch<64, 6, Epi, false, true>(ctx, ma, mb, args, epi, s)
                : launch<64, 6, Epi, false, false>(ctx, ma, mb, args, epi, s);
  if (bn == 128)
    return bf16 ? launch<128, 4, Epi, false, true>(ctx, ma, mb, args, epi, s)
                : launch<128, 4, Epi, false, false>(ctx, ma, mb, args, epi, s);
  return bf16 ? launch<256, 4, Epi, false, true>(ctx, ma, mb, args, epi, s)
              : launch<256, 4, Epi, false, false>(ctx, ma, mb, args, epi, s);
}

template rg_status gemm<EpiTwoIMinusT<__nv_bfloat16>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int,
                                                      int, int, const EpiTwoIMinusT<__nv_bfloat16>&, cudaStream_t, const int*);
template rg_status gemm<EpiTwoIMinusT<__half>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int,
                                               int, const EpiTwoIMinusT<__half>&, cudaStream_t, const int*);
template rg_status gemm<EpiStore16Both<__nv_bfloat16>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int,
                                                       int, int, const EpiStore16Both<__nv_bfloat16>&, cudaStream_t, const int*);
template rg_status gemm<EpiStore16Both<__half>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int,
                                                int, const EpiStore16Both<__half>&, cudaStream_t, const int*);
template rg_status gemm<EpiAddF64>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int, int,
                                   const EpiAddF64&, cudaStream_t, const int*);

namespace {

template <int BN, int kStages, class Epi, bool kComp, bool kBF16>
rg_status launch(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& args, const Epi& epi,
                 cudaStream_t s, int grid_z) {
  auto kern = gemm_kernel<BN, kStages, Epi, kComp, kBF16>;
  constexpr size_t smem = smem_bytes<BN, kStages>();
  static thread_local int configured_device = -1;
  if (configured_device != ctx->device) {
    RG_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured_device = ctx->device;
  }
  dim3 grid(((args.N + BN - 1) / BN) * ((args.M + BM - 1) / BM), 1, grid_z);
  const double executed = 2.0 * args.M * (double)args.N * args.K;
  const int tok = rg::timer_begin(ctx, kComp ? rg::kTimeResidualGemm : rg::kTimeGemm, s, executed,
                                  args.alg_k > 0 ? 2.0 * args.M * (double)args.N * args.alg_k : executed);
  kern<<<grid, cta_threads<BN, kComp>(), smem, s>>>(ma, mb, args, epi);
  rg::timer_end(ctx, tok, s);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  return RG_OK;
}

}  // namespace

rg_status gemm_f32(rg_ctx* ctx, bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N,
                   int K, float* C, int64_t ldc, float alpha, float beta, cudaStream_t s) {
  if (M <= 0 || N <= 0) return RG_OK;
  if (K <= 0) return rg::fail(ctx, RG_ERR_ARG, "gemm_f32: K = %d", K);
  const int bn = tile_width(ctx, M, N) == 256 ? 256 : 128;
  CUtensorMap ma, mb;
  rg_status st = encode_kmajor(ctx, &ma, A, bf16, M, K, lda, BM);
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, bf16, N, K, ldb, bn);
  if (st != RG_OK) return st;
  GemmArgs args{M, N, K, 0, ctx->d_scratch + kGemmErrorSlot};
  EpiF32 epi{C, ldc, alpha, beta};
  if (bn == 256)
    return bf16 ? launch<256, 4, EpiF32, false, true>(ctx, ma, mb, args, epi, s)
                : launch<256, 4, EpiF32, false, false>(ctx, ma, mb, args, epi, s);
  return bf16 ? launch<128, 4, EpiF32, false, true>(ctx, ma, mb, args, epi, s)
              : launch<128, 4, EpiF32, false, false>(ctx, ma, mb, args, epi, s);
}

namespace {

// out = E - X + dl o (sum_z partial[z]) (or dl o sum when E is null), the sum over the K
// splits in order z = 0, 1, ...; with red: max|out| -> red[0], max|X| -> red[1], column
// maxima of out -> colmax, inf / NaN -> *nonfinite. Block (32 x 8) per 32 columns x 16 rows
// (two rows per thread: many small blocks keep the independent loads in flight).
__global__ void residual_finish(const double* __restrict__ partial, int64_t stride, int splits, int M, int N,
                                int64_t ld, double* __restrict__ out, const double* __restrict__ E,
                                const double* __restrict__ X, const double* __restrict__ dl, unsigned long long* red,
                                unsigned long long* colmax, int* nonfinite) {
  __shared__ double s_out[8][33], s_x[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int r0 = blockIdx.y * 16;
  double m_out = 0.0, m_x = 0.0;
  bool bad = false;
  if (c < N) {
    for (int r = r0 + threadIdx.y; r < min(M, r0 + 16); r += 8) {
      const int64_t i = (int64_t)r * ld + c;
      double acc = 0.0;
      for (int z = 0; z < splits; ++z) acc += partial[(int64_t)z * stride + i];
      const double sc = dl ? dl[r] : 1.0;
      double o;
      if (E) {
        const double xi = X[i];
        o = (E[i] - xi) + sc * acc;
        m_x = fmax(m_x, fabs(xi));
        bad |= !isfinite(xi);
      } else {
        o = sc * acc;
      }
      out[i] = o;
      m_out = fmax(m_out, fabs(o));
      bad |= !isfinite(o);
    }
  }
  if (!red) return;
  s_out[threadIdx.y][threadIdx.x] = m_out;
  s_x[threadIdx.y][threadIdx.x] = m_x;
  if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0 && nonfinite) atomicExch(nonfinite, 1);
  if (threadIdx.y == 0) {
    for (int y = 1; y < 8; ++y) {
      m_out = fmax(m_out, s_out[y][threadIdx.x]);
      m_x = fmax(m_x, s_x[y][threadIdx.x]);
    }
    if (colmax && c < N) atomic_max_nonneg(&colmax[c], m_out);
    for (int o = 16; o > 0; o >>= 1) {
      m_out = fmax(m_out, __shfl_xor_sync(0xffffffffu, m_out, o));
      m_x = fmax(m_x, __shfl_xor_sync(0xffffffffu, m_x, o));
    }
    if (threadIdx.x == 0) {
      atomic_max_nonneg(&red[0], m_out);
      atomic_max_nonneg(&red[1], m_x);
    }
  }
}

}  // namespace

// Failure-detection check of the GEMM's mbarrier wait: a barrier nobody arrives on.
__global__ void mbarrier_timeout_probe(int* error_word, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) atomicExch(error_word, 1);
}

int residual_splits(const rg_ctx* ctx, int M, int N, int K, int chunk_blocks, int split_max) {
  const int tiles = ((M + BM - 1) / BM) * ((N + 63) / 64);
  const int kb = (K + BK - 1) / BK;
  const int chunk = chunk_blocks > 0 ? chunk_blocks : 1;
  int best = 1;
  // enough splits to give every SM a tile, in whole chunks
  for (int z = 2; z <= split_max; ++z) {
    if (tiles * (z - 1) >= ctx->sm_count) break;
    if (kb % z == 0 && (kb / z) % chunk == 0) best = z;
  }
  return best;
}

rg_status gemm_residual(rg_ctx* ctx, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
                        int chunk_blocks, double* out, const double* E, const double* X, const double* dl,
                        int64_t ld, cudaStream_t s, unsigned long long* red, unsigned long long* colmax,
                        int* nonfinite, double* split_ws, int split_max, int lead_blocks, int tail_chunk_blocks,
                        int alg_k) {
  if (M <= 0 || N <= 0) return RG_OK;
  if (K <= 0) return rg::fail(ctx, RG_ERR_ARG, "gemm_residual: K = %d", K);
  constexpr int BN = 64;
  // 128-wide tiles (two epilogue groups) where they still give every SM two tiles
  const bool wide = (int64_t)((M + BM - 1) / BM) * ((N + 127) / 128) >= 2 * (int64_t)ctx->sm_count;
  CUtensorMap ma, mb;
  rg_status st = encode_kmajor(ctx, &ma, A, true, M, K, lda, BM);
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, true, N, K, ldb, wide ? 128 : BN);
  if (st != RG_OK) return st;
  GemmArgs args{M, N, K, chunk_blocks, ctx->d_scratch + kGemmErrorSlot};
  args.alg_k = alg_k;
  const int splits = (split_ws && !wide) ? residual_splits(ctx, M, N, K, chunk_blocks, split_max) : 1;
  if (splits <= 1) {
    if (lead_blocks > 0 && tail_chunk_blocks > 0 && chunk_blocks > 0 && lead_blocks % chunk_blocks == 0) {
      args.lead_blocks = lead_blocks;
      args.tail_chunk_blocks = tail_chunk_blocks;
    }
    EpiResidual epi{out, E, X, dl, ld, red, colmax, nonfinite};
    if (wide) return launch<128, 4, EpiResidual, true, true>(ctx, ma, mb, args, epi, s, 1);
    return launch<BN, 6, EpiResidual, true, true>(ctx, ma, mb, args, epi, s, 1);
  }
  const int kb = (K + BK - 1) / BK;
  args.split_blocks = kb / splits;
  const int64_t stride = (int64_t)M * ld;
  EpiResidual epi{nullptr, nullptr, nullptr, nullptr, ld};
  epi.partial = split_ws;
  epi.split_stride = stride;
  st = launch<BN, 6, EpiResidual, true, true>(ctx, ma, mb, args, epi, s, splits);
  if (st != RG_OK) return st;
  dim3 grid((N + 31) / 32, (M + 15) / 16);
  residual_finish<<<grid, dim3(32, 8), 0, s>>>(split_ws, stride, splits, M, N, ld, out, E, X, dl, red, colmax,
                                               nonfinite);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  return RG_OK;
}

}  // namespace tc

extern "C" {

rg_status rg_debug_mbarrier_timeout(rg_ctx* ctx, double limit_s, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, limit_s > 0.0 && limit_s <= 2.0, "rg_debug_wait_timeout: limit %.3g s outside (0, 2]", limit_s);
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch + tc::kGemmErrorSlot, 0, sizeof(int), s));
  tc::mbarrier_timeout_probe<<<1, 32, 0, s>>>(ctx->d_scratch + tc::kGemmErrorSlot,
                                              (unsigned long long)(limit_s * 1e9));
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  int h = 0;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_scratch + tc::kGemmErrorSlot, sizeof(int), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h) return rg::fail(ctx, RG_ERR_CUDA, "mbarrier wait timed out after %.3g s", limit_s);
  return RG_OK;
}

rg_status rg_tc_gemm(rg_ctx* ctx, int32_t M, int32_t N, int32_t K, const void* A_d, int64_t lda, const void* B_d,
                     int64_t ldb, int32_t fp16, float* C_d, int64_t ldc, float alpha, float beta, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, M >= 0 && N >= 0 && K > 0 && A_d && B_d && C_d && ldc >= N, "rg_tc_gemm: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch + tc::kGemmErrorSlot, 0, sizeof(int), s));
  rg_status st = tc::gemm_f32(ctx, !fp16, A_d, lda, B_d, ldb, M, N, K, C_d, ldc, alpha, beta, s);
  if (st != RG_OK) return st;
  int h = 0;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_scratch + tc::kGemmErrorSlot, sizeof(int), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h) return rg::fail(ctx, RG_ERR_CUDA, "rg_tc_gemm: a barrier wait timed out");
  return RG_OK;
}

rg_status rg_tc_gemm_residual(rg_ctx* ctx, int32_t M, int32_t N, int32_t K, const void* A_d, int64_t lda,
                              const void* B_d, int64_t ldb, int32_t chunk_k, double* out_d, const double* E_d,
                              const double* X_d, const double* dl_d, int64_t ld, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, M >= 0 && N >= 0 && K > 0 && A_d && B_d && out_d && ld >= N && chunk_k >= 64 && chunk_k % 64 == 0,
               "rg_tc_gemm_residual: bad argument");
  RG_ARG_CHECK(ctx, (E_d == nullptr) == (X_d == nullptr), "rg_tc_gemm_residual: E and X go together");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch + tc::kGemmErrorSlot, 0, sizeof(int), s));
  rg_status st = tc::gemm_residual(ctx, A_d, lda, B_d, ldb, M, N, K, chunk_k / 64, out_d, E_d, X_d, dl_d, ld, s);
  if (st != RG_OK) return st;
  int h = 0;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_scratch + tc::kGemmErrorSlot, sizeof(int), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h) return rg::fail(ctx, RG_ERR_CUDA, "rg_tc_gemm_residual: a barrier wait timed out");
  return RG_OK;
}

}  // extern "C"
