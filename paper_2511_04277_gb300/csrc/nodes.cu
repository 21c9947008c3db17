// Node relations of two-sided surfaces (Sec. 5.2.4-5.2.5, App. C), fp64.
//
// Input matrices use the side-resolved layout of rg_trace_sided: row 2i+X is side X of
// face i (X = 0: side A, 1: side B), column 2j+Y side Y of face j, column 2N the
// environment, row-major with leading dimension 2N+1. Node i has C_i faces (1 or 2; a
// one-faced node's side-B row is zero).
//
// Both kernels work on node pairs: thread (i, j) reads the 2 x 2 block of side pairs
// (2 x 1 for the environment column j = N) and writes the pair's node quantities. A warp
// covers 32 consecutive j of two adjacent rows, i.e. 512 contiguous bytes per row, so
// every loaded sector is used; the work is one pass over the side matrix, bound by HBM.
#include <cmath>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t total, int sm_count) {
  const int64_t want = (total + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sm_count * 8;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

// Eq. 5.17 (node view factors, C_i F_ij = sum over the four side pairs) and Eq. 5.29
// (view fractions f^{X->Y} = F^{X->Y} / sum over the side pairs; 0 where the sum is 0).
__global__ void __launch_bounds__(kThreads) node_view_factors_kernel(const double* __restrict__ F2, int32_t n,
                                                                     const int32_t* __restrict__ C,
                                                                     double* __restrict__ Fn,
                                                                     double* __restrict__ frac, int32_t* err) {
  const int64_t ld2 = 2 * (int64_t)n + 1, ldn = (int64_t)n + 1;
  const int64_t total = (int64_t)n * ldn;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / ldn, j = k - i * ldn;
    const int32_t c = C[i];
    if (c != 1 && c != 2) {
      atomicExch(err, 1);
      continue;
    }
    const double* rA = F2 + 2 * i * ld2;
    const double* rB = rA + ld2;
    if (j < n) {
      const double aa = rA[2 * j], ab = rA[2 * j + 1], ba = rB[2 * j], bb = rB[2 * j + 1];
      const double sum = (aa + ab) + (ba + bb);
      Fn[k] = sum / c;
      if (frac) {
        const double r = sum > 0.0 ? 1.0 / sum : 0.0;
        double* fA = frac + 2 * i * ld2;
        fA[2 * j] = aa * r;
        fA[2 * j + 1] = ab * r;
        fA[ld2 + 2 * j] = ba * r;
        fA[ld2 + 2 * j + 1] = bb * r;
      }
    } else {
      const double ea = rA[2 * n], eb = rB[2 * n];
      const double sum = ea + eb;
      Fn[k] = sum / c;
      if (frac) {
        const double r = sum > 0.0 ? 1.0 / sum : 0.0;
        frac[2 * i * ld2 + 2 * n] = ea * r;
        frac[(2 * i + 1) * ld2 + 2 * n] = eb * r;
      }
    }
  }
}

// App. C: GR_ij = S_i (eps^A_i sum_Y B^{A->Y}_ij + eps^B_i sum_Y B^{B->Y}_ij) (Eq. C.3),
// the node REF B_ij = sum over the side pairs / C_i (Eq. C.3, first line) and the pair's
// node emissivity eps_ij = GR_ij / (C_i S_i B_ij) (Eq. C.4; 0 where B_ij = 0).
__global__ void __launch_bounds__(kThreads) node_couplings_kernel(const double* __restrict__ B2, int32_t n,
                                                                  const double* __restrict__ eps2,
                                                                  const double* __restrict__ S,
                                                                  const int32_t* __restrict__ C,
                                                                  double* __restrict__ GR, double* __restrict__ Bn,
                                                                  double* __restrict__ epsn, int32_t* err) {
  const int64_t ld2 = 2 * (int64_t)n + 1, ldn = (int64_t)n + 1;
  const int64_t total = (int64_t)n * ldn;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / ldn, j = k - i * ldn;
    const int32_t c = C[i];
    if (c != 1 && c != 2) {
      atomicExch(err, 1);
      continue;
    }
    const double* rA = B2 + 2 * i * ld2;
    const double* rB = rA + ld2;
    double sA, sB;
    if (j < n) {
      sA = rA[2 * j] + rA[2 * j + 1];
      sB = rB[2 * j] + rB[2 * j + 1];
    } else {
      sA = rA[2 * n];
      sB = rB[2 * n];
    }
    const double emitted = eps2[2 * i] * sA + eps2[2 * i + 1] * sB;
    const double sum = sA + sB;
    GR[k] = S[i] * emitted;
    if (Bn) Bn[k] = sum / c;
    if (epsn) epsn[k] = sum > 0.0 ? emitted / sum : 0.0;
  }
}

rg_status finish(rg_ctx* ctx, cudaStream_t s, const char* what) {
  RG_CUDA_TRY(ctx, cudaGetLastError());
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, ctx->d_scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (ctx->h_scratch[0]) return rg::fail(ctx, RG_ERR_ARG, "%s: a face count C_i is not 1 or 2", what);
  return RG_OK;
}

}  // namespace

extern "C" {

rg_status rg_node_view_factors(rg_ctx* ctx, int32_t n, const double* F2_d, const int32_t* faces_per_node_d,
                               double* F_node_d, double* frac_d, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n > 0 && n < (1 << 29) && F2_d && faces_per_node_d && F_node_d,
               "rg_node_view_factors: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch, 0, sizeof(int32_t), s));
  const int64_t total = (int64_t)n * (n + 1);
  node_view_factors_kernel<<<grid_for(total, ctx->sm_count), kThreads, 0, s>>>(F2_d, n, faces_per_node_d, F_node_d,
                                                                             frac_d, ctx->d_scratch);
  ++ctx->launches;
  return finish(ctx, s, "rg_node_view_factors");
}

rg_status rg_node_couplings(rg_ctx* ctx, int32_t n, const double* B2_d, const double* eps2_d,
                            const double* face_area_d, const int32_t* faces_per_node_d, double* GR_d,
                            double* B_node_d, double* eps_node_d, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n > 0 && n < (1 << 29) && B2_d && eps2_d && face_area_d && faces_per_node_d && GR_d,
               "rg_node_couplings: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch, 0, sizeof(int32_t), s));
  const int64_t total = (int64_t)n * (n + 1);
  node_couplings_kernel<<<grid_for(total, ctx->sm_count), kThreads, 0, s>>>(
      B2_d, n, eps2_d, face_area_d, faces_per_node_d, GR_d, B_node_d, eps_node_d, ctx->d_scratch);
  ++ctx->launches;
  return finish(ctx, s, "rg_node_couplings");
}

}  // extern "C"
