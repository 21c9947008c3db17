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

namespace {
int timer_event(rg_ctx* ctx) {
  if (ctx->timer_used == ctx->timer_events.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    ctx->timer_events.push_back(e);
  }
  return (int)ctx->timer_used++;
}
}  // namespace

int timer_begin(rg_ctx* ctx, int kind, cudaStream_t s, double flops, double alg) {
  if (!ctx->timer_on) return -1;
  const int a = timer_event(ctx), b = timer_event(ctx);
  if (a < 0 || b < 0 || cudaEventRecord(ctx->timer_events[a], s) != cudaSuccess) return -1;
  ctx->timed.push_back({kind, a, b, flops, alg});
  return (int)ctx->timed.size() - 1;
}

int* timer_level_slot(rg_ctx* ctx, int token) {
  if (token < 0 || !ctx->timer_levels_d || ctx->timer_levels_used >= kTimerLevelSlots) return nullptr;
  ctx->timed[token].level_slot = ctx->timer_levels_used;
  return ctx->timer_levels_d + ctx->timer_levels_used++;
}

void timer_end(rg_ctx* ctx, int token, cudaStream_t s) {
  if (token < 0) return;
  if (cudaEventRecord(ctx->timer_events[ctx->timed[token].b], s) != cudaSuccess) ctx->timed[token].b = -1;
}

rg_status workspace_or(rg_ctx* ctx, void* user, size_t user_bytes, size_t bytes, void** out, const char* fn) {
  if (!user) return workspace(ctx, bytes, out);
  if (reinterpret_cast<uintptr_t>(user) & 255)
    return fail(ctx, RG_ERR_ARG, "%s: the caller's workspace must be 256-byte aligned", fn);
  if (user_bytes < bytes)
    return fail(ctx, RG_ERR_ARG, "%s: the caller's workspace holds %zu bytes, the call needs %zu", fn, user_bytes,
                bytes);
  *out = user;
  return RG_OK;
}

}  // namespace rg

extern "C" {

rg_status rg_workspace_bytes(const rg_ctx* ctx, size_t* bytes_out) {
  if (!ctx || !bytes_out) return RG_ERR_ARG;
  *bytes_out = ctx->ws_bytes;
  return RG_OK;
}

rg_status rg_kernel_timer(rg_ctx* ctx, int32_t enable) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, enable == 0 || enable == 1, "rg_kernel_timer: enable = %d", enable);
  if (enable) {
    RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    ctx->timed.clear();
    ctx->timer_used = 0;
    ctx->timer_levels_used = 0;
    if (!ctx->timer_levels_d)
      RG_CUDA_TRY(ctx, cudaMalloc(&ctx->timer_levels_d, rg::kTimerLevelSlots * sizeof(int)));
  }
  ctx->timer_on = enable != 0;
  return RG_OK;
}

rg_status rg_kernel_timer_read(rg_ctx* ctx, int32_t kind, int64_t* launches_out_h, double* ms_out_h,
                               double* flops_out_h, double* alg_flops_out_h) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, kind >= 0 && kind < rg::kTimeClasses && launches_out_h && ms_out_h,
               "rg_kernel_timer_read: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  int64_t n = 0;
  double ms = 0.0, flops = 0.0, alg = 0.0;
  std::vector<int> levels;
  for (const auto& t : ctx->timed) {
    if (t.kind != kind) continue;
    if (t.b < 0) return rg::fail(ctx, RG_ERR_CUDA, "rg_kernel_timer_read: an end event was not recorded");
    RG_CUDA_TRY(ctx, cudaEventSynchronize(ctx->timer_events[t.b]));
    float e = 0.f;
    RG_CUDA_TRY(ctx, cudaEventElapsedTime(&e, ctx->timer_events[t.a], ctx->timer_events[t.b]));
    double f = t.flops;
    if (t.level_slot >= 0) {
      if (levels.empty()) {
        levels.resize(ctx->timer_levels_used);
        RG_CUDA_TRY(ctx, cudaMemcpy(levels.data(), ctx->timer_levels_d, levels.size() * sizeof(int),
                                    cudaMemcpyDeviceToHost));
      }
      f *= levels[t.level_slot];
    }
    ++n;
    ms += e;
    flops += f;
    alg += t.alg;
  }
  *launches_out_h = n;
  *ms_out_h = ms;
  if (flops_out_h) *flops_out_h = flops;
  if (alg_flops_out_h) *alg_flops_out_h = alg;
  return RG_OK;
}


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
  if (cudaEventCreateWithFlags(&ctx->ev_read[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_read[1], cudaEventDisableTiming) != cudaSuccess) {
    if (ctx->ev_read[0]) cudaEventDestroy(ctx->ev_read[0]);
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
  for (cudaEvent_t e : ctx->ev_read)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->timer_events) cudaEventDestroy(e);
  if (ctx->timer_levels_d) cudaFree(ctx->timer_levels_d);
  delete ctx;
}

const char* rg_last_error(const rg_ctx* ctx) {
  if (!ctx) return "no context";
  return ctx->last_error.c_str();
}

}  // extern "C"
