// Context lifetime, error reporting and workspace management.
#include "common.cuh"

namespace rg {

rg_status fail(rg_ctx* ctx, rg_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return st;
}

rg_status cuda_fail(rg_ctx* ctx, cudaError_t e, const char* what) {
  rg_status st = (e == cudaErrorMemoryAllocation) ? RG_ERR_OOM : RG_ERR_CUDA;
  return fail(ctx, st, "%s: %s", what, cudaGetErrorString(e));
}

rg_status workspace(rg_ctx* ctx, size_t bytes, void** out) {
  bytes = align_up(bytes < 256 ? 256 : bytes, 1 << 20);
  if (bytes > ctx->ws_bytes) {
    if (ctx->ws) {
      // the old buffer may still be in use by queued work
      RG_CUDA_TRY(ctx, cudaDeviceSynchronize());
      RG_CUDA_TRY(ctx, cudaFree(ctx->ws));
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
    }
    RG_CUDA_TRY(ctx, cudaMalloc(&ctx->ws, bytes));
    ctx->ws_bytes = bytes;
  }
  *out = ctx->ws;
  return RG_OK;
}

}  // namespace rg

extern "C" {

const char* rg_version(void) { return "radgeb 0.1 (sm_103a)"; }

rg_status rg_create(rg_ctx** ctx_out, int device) {
  if (!ctx_out) return RG_ERR_ARG;
  *ctx_out = nullptr;
  rg_ctx* ctx = new (std::nothrow) rg_ctx();
  if (!ctx) return RG_ERR_OOM;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) {
    delete ctx;
    return e != cudaSuccess ? RG_ERR_CUDA : RG_ERR_ARG;
  }
  cudaDeviceProp prop;
  if (cudaSetDevice(device) != cudaSuccess || cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return RG_ERR_CUDA;
  }
  if (prop.major != 10 || prop.minor != 3) {
    delete ctx;
    return RG_ERR_UNSUPPORTED;  // the kernels are built for sm_103a only
  }
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  ctx->smem_optin = (int)prop.sharedMemPerBlockOptin;
  if (cudaMalloc(&ctx->d_scratch, rg::kScratchInts * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_scratch, rg::kScratchInts * sizeof(int)) != cudaSuccess) {
    if (ctx->d_scratch) cudaFree(ctx->d_scratch);
    delete ctx;
    return RG_ERR_OOM;
  }
  if (cudaEventCreateWithFlags(&ctx->ev_read, cudaEventDisableTiming) != cudaSuccess) {
    cudaFree(ctx->d_scratch);
    cudaFreeHost(ctx->h_scratch);
    delete ctx;
    return RG_ERR_CUDA;
  }
  *ctx_out = ctx;
  return RG_OK;
}

void rg_destroy(rg_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_scratch) cudaFree(ctx->d_scratch);
  if (ctx->h_scratch) cudaFreeHost(ctx->h_scratch);
  if (ctx->ev_read) cudaEventDestroy(ctx->ev_read);
  delete ctx;
}

const char* rg_last_error(const rg_ctx* ctx) {
  if (!ctx) return "no context";
  return ctx->last_error.c_str();
}

}  // extern "C"
