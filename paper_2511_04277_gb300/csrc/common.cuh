// Internal declarations shared by the translation units of libradgeb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "radgeb.h"

struct rg_ctx {
  int device = 0;
  int sm_count = 0;
  int smem_optin = 0;
  std::string last_error;
  // device workspace owned by the context, grown on demand (never shrunk)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // small device scratch: error words, counters, flags (zeroed per call as needed)
  int* d_scratch = nullptr;
  // pinned host scratch for scalar read-backs
  int* h_scratch = nullptr;
  // recorded after a read-back copy, so that the host can wait for it while later
  // launches on the stream keep the GPU busy (two: the refinement alternates them)
  cudaEvent_t ev_read[2] = {nullptr, nullptr};
  // kernels this context has launched (rg_launch_count)
  int64_t launches = 0;
  // kernel timer (rg_kernel_timer): while on, an event pair is recorded on the launching
  // stream around every launch of the timed kernel classes
  struct TimedLaunch {
    int kind;
    int a, b;      // indices into timer_events
    double flops;  // tensor-core flops the launch executes (2 M N K), 0 for non-GEMM kernels
    double alg;    // algorithmic flops of the product it stands for (the fp64 residual for the
                   // sliced refinement product), 0 for non-GEMM kernels
    int level_slot = -1;  // >= 0: flops are per level, the level count is timer_levels_d[slot]
  };
  bool timer_on = false;
  std::vector<cudaEvent_t> timer_events;
  size_t timer_used = 0;
  std::vector<TimedLaunch> timed;
  // device log of the level counts of timed exact-product launches (decided on the device)
  int* timer_levels_d = nullptr;
  int timer_levels_used = 0;
};

namespace rg {

constexpr int kScratchInts = 1024;

rg_status fail(rg_ctx* ctx, rg_status st, const char* fmt, ...);
rg_status cuda_fail(rg_ctx* ctx, cudaError_t e, const char* what);

// Device workspace of at least `bytes` (256-byte aligned), owned by ctx.
rg_status workspace(rg_ctx* ctx, size_t bytes, void** out);
// The caller's workspace (user, user_bytes) when user is not null -- 256-byte aligned and at
// least `bytes` long, else RG_ERR_ARG naming `fn` and the size needed -- or the context's.
rg_status workspace_or(rg_ctx* ctx, void* user, size_t user_bytes, size_t bytes, void** out, const char* fn);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Kernel classes of the kernel timer (values of rg_kernel_class in radgeb.h).
enum KernelClass {
  kTimeTrace = 0,
  kTimeResidualGemm = 1,
  kTimeGemm = 2,
  kTimeEnforce = 3,
  kTimeFactor = 4,
  kTimeClasses = 5
};
// Records the start event of a launch of class `kind` on stream s when the timer is on;
// returns the token timer_end takes (-1: not recorded).
int timer_begin(rg_ctx* ctx, int kind, cudaStream_t s, double flops = 0.0, double alg = 0.0);
constexpr int kTimerLevelSlots = 8192;
// For a timed launch whose flops count per level (token from timer_begin): the device slot the
// launch writes its level count to, or nullptr (timer off, or the log is full).
int* timer_level_slot(rg_ctx* ctx, int token);
void timer_end(rg_ctx* ctx, int token, cudaStream_t s);

// Carves consecutive 256-byte aligned sub-buffers out of one allocation.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off = align_up(off + count * sizeof(T), 256);
    return p;
  }
};
// Bytes a sequence of takes needs.
struct Sizer {
  size_t off = 0;
  template <class T>
  void take(size_t count) { off = align_up(off + count * sizeof(T), 256); }
};

}  // namespace rg

#define RG_CUDA_TRY(ctx, call)                                   \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return rg::cuda_fail((ctx), e_, #call); \
  } while (0)

#define RG_ARG_CHECK(ctx, cond, ...)                                   \
  do {                                                                 \
    if (!(cond)) return rg::fail((ctx), RG_ERR_ARG, __VA_ARGS__);      \
  } while (0)
