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

template <int BN, int kStages, class Epi, bool kBF16>
rg_status launch(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& args, const Epi& epi,
                 cudaStream_t s);
template <class Epi, bool kBF16>
rg_status launch_pair(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& args,
                      const Epi& epi, cudaStream_t s);

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
               const Epi& epi, cudaStream_t s, const int* skip, bool sym, const uint8_t* aflags,
               const uint8_t* bflags) {
  if (M <= 0 || N <= 0) return RG_OK;
  if (K <= 0) return rg::fail(ctx, RG_ERR_ARG, "gemm: K = %d", K);
  const int bn = tile_width(ctx, M, N);
  CUtensorMap ma, mb;
  // 256-wide tiles go to CTA pairs (gemm_pair_kernel): each CTA loads 128 of B's rows
  rg_status st = encode_kmajor(ctx, &ma, A, bf16, M, K, lda, BM);
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, bf16, N, K, ldb, bn == 256 ? 128 : bn);
  if (st != RG_OK) return st;
  GemmArgs args{M, N, K, ctx->d_scratch + kGemmErrorSlot};
  args.skip = skip;
  // a symmetric product computes the upper tiles only where the tiles are square
  args.sym = (sym && M == N && (bn == 256 || bn == 128)) ? 1 : 0;
  if (bn == 256 && !args.sym && (aflags || bflags)) {
    if ((reinterpret_cast<uintptr_t>(aflags) | reinterpret_cast<uintptr_t>(bflags)) & 15)
      return rg::fail(ctx, RG_ERR_ARG, "gemm: block flags not 16-byte aligned");
    args.aflags = aflags;
    args.bflags = bflags;
  }
  if (bn == 256)
    return bf16 ? launch_pair<Epi, true>(ctx, ma, mb, args, epi, s) : launch_pair<Epi, false>(ctx, ma, mb, args, epi, s);
  if (bn == 64)
    return bf16 ? launch<64, 6, Epi, true>(ctx, ma, mb, args, epi, s) : launch<64, 6, Epi, false>(ctx, ma, mb, args, epi, s);
  return bf16 ? launch<128, 4, Epi, true>(ctx, ma, mb, args, epi, s)
              : launch<128, 4, Epi, false>(ctx, ma, mb, args, epi, s);
}

template rg_status gemm<EpiTwoIMinusT<__nv_bfloat16>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int,
                                                      int, int, const EpiTwoIMinusT<__nv_bfloat16>&, cudaStream_t, const int*, bool, const uint8_t*, const uint8_t*);
template rg_status gemm<EpiTwoIMinusT<__half>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int,
                                               int, const EpiTwoIMinusT<__half>&, cudaStream_t, const int*, bool, const uint8_t*, const uint8_t*);
template rg_status gemm<EpiStore16Both<__nv_bfloat16>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int,
                                                       int, int, const EpiStore16Both<__nv_bfloat16>&, cudaStream_t, const int*, bool, const uint8_t*, const uint8_t*);
template rg_status gemm<EpiStore16Both<__half>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int,
                                                int, const EpiStore16Both<__half>&, cudaStream_t, const int*, bool, const uint8_t*, const uint8_t*);
template rg_status gemm<EpiCorrection>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int, int,
                                       const EpiCorrection&, cudaStream_t, const int*, bool, const uint8_t*, const uint8_t*);

namespace {

template <int BN, int kStages, class Epi, bool kBF16>
rg_status launch(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& args, const Epi& epi,
                 cudaStream_t s) {
  auto kern = gemm_kernel<BN, kStages, Epi, kBF16>;
  constexpr size_t smem = smem_bytes<BN, kStages>();
  static thread_local int configured_device = -1;
  if (configured_device != ctx->device) {
    RG_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured_device = ctx->device;
  }
  const int64_t tiles_m = (args.M + BM - 1) / BM;
  const int64_t tiles = args.sym ? tiles_m * (tiles_m + 1) / 2 : ((args.N + BN - 1) / BN) * tiles_m;
  dim3 grid((unsigned)tiles);
  const double executed = args.sym ? 2.0 * (double)tiles * BM * BN * args.K : 2.0 * args.M * (double)args.N * args.K;
  const int tok = rg::timer_begin(ctx, rg::kTimeGemm, s, executed,
                                  args.alg_k > 0 ? 2.0 * args.M * (double)args.N * args.alg_k : executed);
  kern<<<grid, kThreads, smem, s>>>(ma, mb, args, epi);
  rg::timer_end(ctx, tok, s);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  return RG_OK;
}

template <class Epi, bool kBF16>
rg_status launch_pair(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& args,
                      const Epi& epi, cudaStream_t s) {
  auto kern = gemm_pair_kernel<kPairStages, Epi, kBF16>;
  constexpr size_t smem = pair_smem_bytes<kPairStages>();
  static thread_local int configured_device = -1;
  if (configured_device != ctx->device) {
    RG_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured_device = ctx->device;
  }
  // two CTAs (one cluster) per 256 x 256 tile
  const int64_t tiles_m = (args.M + 2 * BM - 1) / (2 * BM);
  const int64_t tiles = args.sym ? tiles_m * (tiles_m + 1) / 2 : ((args.N + 255) / 256) * tiles_m;
  dim3 grid((unsigned)(2 * tiles));
  const double executed =
      args.sym ? 2.0 * (double)tiles * 256 * 256 * args.K : 2.0 * args.M * (double)args.N * args.K;
  // with A's block flags the pairs add up the K blocks they execute (flops per block)
  const bool flagged = args.aflags || args.bflags;
  const int tok = rg::timer_begin(ctx, rg::kTimeGemm, s, flagged ? 2.0 * 256 * 256 * BK : executed,
                                  args.alg_k > 0 ? 2.0 * args.M * (double)args.N * args.alg_k : executed);
  GemmArgs a = args;
  if (flagged) {
    a.level_log = rg::timer_level_slot(ctx, tok);
    if (a.level_log) RG_CUDA_TRY(ctx, cudaMemsetAsync(a.level_log, 0, sizeof(int), s));
  }
  kern<<<grid, kThreads, smem, s>>>(ma, mb, a, epi);
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
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, bf16, N, K, ldb, 128);
  if (st != RG_OK) return st;
  GemmArgs args{M, N, K, ctx->d_scratch + kGemmErrorSlot};
  EpiF32 epi{C, ldc, alpha, beta};
  if (bn == 256)
    return bf16 ? launch_pair<EpiF32, true>(ctx, ma, mb, args, epi, s)
                : launch_pair<EpiF32, false>(ctx, ma, mb, args, epi, s);
  return bf16 ? launch<128, 4, EpiF32, true>(ctx, ma, mb, args, epi, s)
              : launch<128, 4, EpiF32, false>(ctx, ma, mb, args, epi, s);
}

int64_t exact_ld(int N) { return ((int64_t)N + 255) / 256 * 256; }
// rows rounded up to 256: a CTA pair's tile reaches that far
int64_t exact_plane(int M, int N) { return ((int64_t)M + 2 * BM - 1) / (2 * BM) * (2 * BM) * exact_ld(N); }

namespace {

template <int BN, int kStages>
rg_status launch_exact(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, ExactArgs args, int splits,
                       cudaStream_t s, double flops_per_level, double alg) {
  auto kern = gemm_exact_kernel<BN, kStages>;
  constexpr size_t smem = exact_smem_bytes<BN, kStages>();
  static thread_local int configured_device = -1;
  if (configured_device != ctx->device) {
    RG_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured_device = ctx->device;
  }
  dim3 grid(((args.N + BN - 1) / BN) * ((args.M + BM - 1) / BM), 1, splits);
  const int tok = rg::timer_begin(ctx, rg::kTimeResidualGemm, s, flops_per_level, alg);
  args.level_log = rg::timer_level_slot(ctx, tok);
  kern<<<grid, exact_threads(BN), smem, s>>>(ma, mb, args);
  rg::timer_end(ctx, tok, s);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  return RG_OK;
}

rg_status launch_exact_pair(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, ExactArgs args, cudaStream_t s,
                            double flops_per_level, double alg) {
  auto kern = gemm_exact_pair_kernel<kPairStages>;
  constexpr size_t smem = exact_pair_smem_bytes<kPairStages>();
  static thread_local int configured_device = -1;
  if (configured_device != ctx->device) {
    RG_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured_device = ctx->device;
  }
  // two CTAs (one cluster) per 256 x 256 tile, no K splits
  dim3 grid(2 * ((args.N + 255) / 256) * ((args.M + 2 * BM - 1) / (2 * BM)), 1, 1);
  // with block flags the pairs add up the blocks they execute (flops per block), else the
  // launch records its level count (flops per level)
  const double flops = args.flags ? 2.0 * (2 * BM) * 256 * BK : flops_per_level;
  const int tok = rg::timer_begin(ctx, rg::kTimeResidualGemm, s, flops, alg);
  args.level_log = rg::timer_level_slot(ctx, tok);
  if (args.flags && args.level_log) RG_CUDA_TRY(ctx, cudaMemsetAsync(args.level_log, 0, sizeof(int), s));
  kern<<<grid, exact_threads(256), smem, s>>>(ma, mb, args);
  rg::timer_end(ctx, tok, s);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  return RG_OK;
}

}  // namespace

rg_status gemm_exact(rg_ctx* ctx, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int np,
                     const int* levels_d, const unsigned long long* level_words, int level_bits, int max_levels,
                     int32_t* lev, int split_max, int* splits_out, cudaStream_t s, const int* skip, int alg_k,
                     const uint8_t* flags, int flag_rows, int flag_ld) {
  if (M <= 0 || N <= 0) return RG_OK;
  if (np <= 0 || np % (2 * BK) || max_levels < 1)
    return rg::fail(ctx, RG_ERR_ARG, "gemm_exact: level length %d, %d levels", np, max_levels);
  // the widest tile that still gives every SM a tile
  const int64_t tm = (M + BM - 1) / BM;
  const int bn = tm * ((N + 255) / 256) >= ctx->sm_count ? 256 : (tm * ((N + 127) / 128) >= ctx->sm_count ? 128 : 64);
  const int tiles = (int)(tm * ((N + bn - 1) / bn));
  // CTA pairs (256 x 256 tiles) when the 256-wide tiles fill the GPU twice over
  const bool pair = bn == 256 && tiles >= 2 * ctx->sm_count;
  // K splits (whole chunks per CTA and level) while the tiles leave SMs idle
  const int kb_level = np / BK;
  int splits = 1;
  for (int z = 2; z <= split_max && !pair; ++z) {
    if ((int64_t)tiles * (z - 1) >= ctx->sm_count) break;
    if (kb_level % (2 * z) == 0) splits = z;
  }
  if (splits_out) *splits_out = splits;
  CUtensorMap ma, mb;
  rg_status st = encode_kmajor(ctx, &ma, A, true, M, (int64_t)max_levels * np, lda, BM);
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, true, N, np, ldb, pair ? 128 : bn);
  if (st != RG_OK) return st;
  ExactArgs args{M,   N,        np, levels_d, level_words, level_bits, max_levels, lev, exact_ld(N), exact_plane(M, N),
                 splits > 1 ? kb_level / splits : 0, ctx->d_scratch + kGemmErrorSlot, skip};
  if (pair && flags) {
    if (flag_rows < (M + 2 * BM - 1) / (2 * BM) || flag_ld < (kb_level + 15) / 16 * 16 || flag_ld % 16 ||
        max_levels > 8 || (reinterpret_cast<uintptr_t>(flags) & 15))
      return rg::fail(ctx, RG_ERR_ARG, "gemm_exact: block flags %d x %d for %d rows, %d blocks", flag_rows, flag_ld, M,
                      kb_level);
    args.flags = flags;
    args.flag_rows = flag_rows;
    args.flag_ld = flag_ld;
  }
  const double per_level = 2.0 * M * (double)N * np;
  const double alg = 2.0 * M * (double)N * (alg_k > 0 ? alg_k : np);
  if (pair) return launch_exact_pair(ctx, ma, mb, args, s, per_level, alg);
  if (bn == 256) return launch_exact<256, 4>(ctx, ma, mb, args, splits, s, per_level, alg);
  if (bn == 128) return launch_exact<128, 4>(ctx, ma, mb, args, splits, s, per_level, alg);
  return launch_exact<64, 6>(ctx, ma, mb, args, splits, s, per_level, alg);
}

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

namespace {
// lev planes [level][rows][exact_ld(N)] -> S [level][M][N]
__global__ void compact_levels(const int32_t* __restrict__ lev, int64_t ldl, int64_t plane, int levels, int M, int N,
                               int32_t* __restrict__ S) {
  const int64_t total = (int64_t)levels * M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / ((int64_t)M * N));
    const int64_t r = e % ((int64_t)M * N);
    const int i = (int)(r / N), j = (int)(r % N);
    S[e] = lev[(int64_t)a * plane + (int64_t)i * ldl + j];
  }
}
}  // namespace

rg_status rg_tc_gemm_exact(rg_ctx* ctx, int32_t M, int32_t N, int32_t np, int32_t levels, const void* A_d,
                           int64_t lda, const void* B_d, int32_t* S_d, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, M > 0 && N > 0 && np > 0 && np % 128 == 0 && levels >= 1 && levels <= 5 && A_d && B_d && S_d &&
                        lda >= 5LL * np,
               "rg_tc_gemm_exact: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t plane = tc::exact_plane(M, N);
  void* ws = nullptr;
  rg_status st = rg::workspace(ctx, (size_t)levels * plane * sizeof(int32_t), &ws);
  if (st != RG_OK) return st;
  int32_t* lev = static_cast<int32_t*>(ws);
  // the level count and the error word in the context scratch
  int* lv = ctx->d_scratch + 64;
  ctx->h_scratch[64] = levels;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(lv, ctx->h_scratch + 64, sizeof(int), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch + tc::kGemmErrorSlot, 0, sizeof(int), s));
  int splits = 1;
  st = tc::gemm_exact(ctx, A_d, lda, B_d, np, M, N, np, lv, nullptr, 0, levels, lev, 1, &splits, s);
  if (st != RG_OK) return st;
  compact_levels<<<256, 256, 0, s>>>(lev, tc::exact_ld(N), plane, levels, M, N, S_d);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  int h = 0;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_scratch + tc::kGemmErrorSlot, sizeof(int), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h) return rg::fail(ctx, RG_ERR_CUDA, "rg_tc_gemm_exact: a barrier wait timed out or the level count was bad");
  return RG_OK;
}

}  // extern "C"
