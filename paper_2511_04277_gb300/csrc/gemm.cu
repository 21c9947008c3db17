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
                 cudaStream_t s);

}  // namespace

template <class Epi>
rg_status gemm(rg_ctx* ctx, bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
               const Epi& epi, cudaStream_t s) {
  if (M <= 0 || N <= 0) return RG_OK;
  if (K <= 0) return rg::fail(ctx, RG_ERR_ARG, "gemm: K = %d", K);
  // 64-wide tiles when 128-wide ones would leave most SMs idle
  const bool narrow = (int64_t)((M + BM - 1) / BM) * ((N + 127) / 128) < 2 * ctx->sm_count;
  CUtensorMap ma, mb;
  rg_status st = encode_kmajor(ctx, &ma, A, bf16, M, K, lda, BM);
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, bf16, N, K, ldb, narrow ? 64 : 128);
  if (st != RG_OK) return st;
  GemmArgs args{M, N, K, 0, ctx->d_scratch + kGemmErrorSlot};
  if (narrow)
    return bf16 ? launch<64, 6, Epi, false, true>(ctx, ma, mb, args, epi, s)
                : launch<64, 6, Epi, false, false>(ctx, ma, mb, args, epi, s);
  return bf16 ? launch<128, 4, Epi, false, true>(ctx, ma, mb, args, epi, s)
              : launch<128, 4, Epi, false, false>(ctx, ma, mb, args, epi, s);
}

template rg_status gemm<EpiTwoIMinusT<__nv_bfloat16>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int,
                                                      int, int, const EpiTwoIMinusT<__nv_bfloat16>&, cudaStream_t);
template rg_status gemm<EpiTwoIMinusT<__half>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int,
                                               int, const EpiTwoIMinusT<__half>&, cudaStream_t);
template rg_status gemm<EpiStore16Both<__nv_bfloat16>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int,
                                                       int, int, const EpiStore16Both<__nv_bfloat16>&, cudaStream_t);
template rg_status gemm<EpiStore16Both<__half>>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int,
                                                int, const EpiStore16Both<__half>&, cudaStream_t);
template rg_status gemm<EpiAddF64>(rg_ctx*, bool, const void*, int64_t, const void*, int64_t, int, int, int,
                                   const EpiAddF64&, cudaStream_t);

namespace {

template <int BN, int kStages, class Epi, bool kComp, bool kBF16>
rg_status launch(rg_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& args, const Epi& epi,
                 cudaStream_t s) {
  auto kern = gemm_kernel<BN, kStages, Epi, kComp, kBF16>;
  constexpr size_t smem = smem_bytes<BN, kStages>();
  static thread_local int configured_device = -1;
  if (configured_device != ctx->device) {
    RG_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured_device = ctx->device;
  }
  dim3 grid((args.N + BN - 1) / BN, (args.M + BM - 1) / BM);
  kern<<<grid, kThreads, smem, s>>>(ma, mb, args, epi);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  return RG_OK;
}

}  // namespace

rg_status gemm_f32(rg_ctx* ctx, bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N,
                   int K, float* C, int64_t ldc, float alpha, float beta, cudaStream_t s) {
  if (M <= 0 || N <= 0) return RG_OK;
  if (K <= 0) return rg::fail(ctx, RG_ERR_ARG, "gemm_f32: K = %d", K);
  constexpr int BN = 128;
  CUtensorMap ma, mb;
  rg_status st = encode_kmajor(ctx, &ma, A, bf16, M, K, lda, BM);
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, bf16, N, K, ldb, BN);
  if (st != RG_OK) return st;
  GemmArgs args{M, N, K, 0, ctx->d_scratch + kGemmErrorSlot};
  EpiF32 epi{C, ldc, alpha, beta};
  return bf16 ? launch<BN, 4, EpiF32, false, true>(ctx, ma, mb, args, epi, s)
              : launch<BN, 4, EpiF32, false, false>(ctx, ma, mb, args, epi, s);
}

rg_status gemm_residual(rg_ctx* ctx, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
                        int chunk_blocks, double* out, const double* E, const double* X, const double* dl,
                        int64_t ld, cudaStream_t s, unsigned long long* red, unsigned long long* colmax,
                        int* nonfinite) {
  if (M <= 0 || N <= 0) return RG_OK;
  if (K <= 0) return rg::fail(ctx, RG_ERR_ARG, "gemm_residual: K = %d", K);
  constexpr int BN = 64;
  CUtensorMap ma, mb;
  rg_status st = encode_kmajor(ctx, &ma, A, true, M, K, lda, BM);
  if (st == RG_OK) st = encode_kmajor(ctx, &mb, B, true, N, K, ldb, BN);
  if (st != RG_OK) return st;
  GemmArgs args{M, N, K, chunk_blocks, ctx->d_scratch + kGemmErrorSlot};
  EpiResidual epi{out, E, X, dl, ld, red, colmax, nonfinite};
  return launch<BN, 6, EpiResidual, true, true>(ctx, ma, mb, args, epi, s);
}

}  // namespace tc

extern "C" {

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
