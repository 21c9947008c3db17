// placeholder: dense solves are being written
#include "common.cuh"
extern "C" {
rg_status rg_enforce_lsq(rg_ctx* ctx, int32_t, const double*, double*, int32_t, int32_t, int32_t, int32_t*, void*) {
  return rg::fail(ctx, RG_ERR_UNSUPPORTED, "not built yet");
}
rg_status rg_gebhart(rg_ctx* ctx, int32_t, const double*, int32_t, const double*, const double*, int32_t, double,
                     int32_t, double*, int32_t*, double*, void*) {
  return rg::fail(ctx, RG_ERR_UNSUPPORTED, "not built yet");
}
rg_status rg_gebhart_adjoint(rg_ctx* ctx, int32_t, const double*, int32_t, const double*, const double*, const double*,
                             const double*, int32_t, double, int32_t, double*, double*, void*) {
  return rg::fail(ctx, RG_ERR_UNSUPPORTED, "not built yet");
}
rg_status rg_temperatures(rg_ctx* ctx, int32_t, const double*, const double*, const double*, const double*, double,
                          double, int32_t, double, double*, void*) {
  return rg::fail(ctx, RG_ERR_UNSUPPORTED, "not built yet");
}
rg_status rg_temperatures_adjoint(rg_ctx* ctx, int32_t, const double*, const double*, const double*, double, double,
                                  const double*, const double*, int32_t, double, double*, double*, void*) {
  return rg::fail(ctx, RG_ERR_UNSUPPORTED, "not built yet");
}
}
