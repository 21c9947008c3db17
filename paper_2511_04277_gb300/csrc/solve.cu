// Dense mixed-precision solves on sm_103a: REFs (App. B, Eq. B.8-B.11), the steady
// radiative balance (Eq. 3.13, 4.1-4.2) and their adjoints.
//
// Every system has the form  (I - Dl P Dr) X = R  with P an N x N fp64 matrix (read
// directly or transposed from the caller's buffer), Dl / Dr diagonal and R an N x m
// right-hand side:
//   REFs            P = F_NN,        Dr = diag(rho), R = [F_NN diag(eps) | F_inf]
//   REF adjoint     P = F_NN^T,      Dl = diag(rho), R = dL/dB
//   balance         P = B_NN,        Dl = diag(1/t), R = (Q + g B_inf T_sink^4) / (g t)
//   balance adjoint P = B_NN^T,      Dl = diag(1/t), R = (dL/du) / t
// with t_i = sum_j B_ij (env included) and g_i = sigma eps_i A_i. I - Dl P Dr is strictly
// diagonally dominant in all four cases, so Gaussian elimination needs no pivoting.
//
// Algorithm (per set):
//   1. A = I - Dl P Dr in fp32, padded to a multiple of 128 with the identity.
//   2. Blocked LU, 128-wide panels: the diagonal block is factored and its triangular
//      inverses formed by one block (fp32); the row and column panels are multiplied by
//      those inverses (fp32); the trailing update A22 -= L21 U12 runs on tcgen05 with
//      16-bit (bf16 or fp16) copies of the panels and fp32 accumulation.
//   3. Triangular solves, block by block: the diagonal inverse (fp32) then a tcgen05
//      update of the remaining rows.
//   4. Iterative refinement: R = R0 - X + Dl (P (Dr X)) with P and Dr X each split into
//      three bf16 slices (24 bits) and the six leading slice products summed by one
//      tcgen05 GEMM over a 6N-long K with compensated fp32 chunks (fp64-accurate); the
//      correction comes from the 16-bit factors. It stops when max|R| <= tol max|X|.
#include <cmath>
#include <utility>

#include "tc_gemm.cuh"

namespace {

constexpr int NB = 128;          // panel width == GEMM tile height
constexpr int kSlices = 6;       // slice pairs of the refinement product
constexpr int kResidualChunk = 2;  // K blocks (of 64) per compensated fp32 chunk
constexpr int kThreads = 256;
// Below this relative residual a sweep that no longer halves it ends the refinement:
// the residual product itself is only accurate to ~1e-8 relative.
constexpr double kStallFloor = 1e-9;

__device__ __forceinline__ double p_elem(const double* P, int64_t ldp, bool trans, int i, int k) {
  return trans ? P[(int64_t)k * ldp + i] : P[(int64_t)i * ldp + k];
}

template <class T>
__device__ __forceinline__ T to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }

// Split x into three bf16 slices whose sum carries ~24 significant bits.
__device__ __forceinline__ void split3(double x, __nv_bfloat16* s) {
  __nv_bfloat16 a = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(a);
  __nv_bfloat16 b = __double2bfloat16(r);
  r -= (double)__bfloat162float(b);
  s[0] = a;
  s[1] = b;
  s[2] = __double2bfloat16(r);
}
// K-concatenated pair order of the refinement product: (P_a, Y_b) for
// (0,0) (0,1) (1,0) (0,2) (1,1) (2,0).
__constant__ int kPairA[kSlices] = {0, 0, 1, 0, 1, 2};
__constant__ int kPairB[kSlices] = {0, 1, 0, 2, 1, 0};

// A_ext[i][q * Np + k] = slice kPairA[q] of P(i, k); zero in the padding.
__global__ void build_p_slices(const double* __restrict__ P, int64_t ldp, bool trans, int n, int np,
                               __nv_bfloat16* __restrict__ Aext) {
  const int64_t total = (int64_t)np * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / np), k = (int)(e % np);
    __nv_bfloat16 s[3];
    double x = (i < n && k < n) ? p_elem(P, ldp, trans, i, k) : 0.0;
    split3(x, s);
    __nv_bfloat16* row = Aext + (int64_t)i * (kSlices * (int64_t)np);
#pragma unroll
    for (int q = 0; q < kSlices; ++q) row[(int64_t)q * np + k] = s[kPairA[q]];
  }
}

// B_ext[j][q * Np + k] = slice kPairB[q] of (Dr X)(k, j); the refinement product's B operand.
// Tiled transpose through shared memory: block (32 x 8) covers a 32 x 32 tile of X.
__global__ void build_x_slices(const double* __restrict__ X, int64_t ldx, const double* __restrict__ dr, int n,
                               int m, int np, int mp, __nv_bfloat16* __restrict__ Bext) {
  __shared__ __nv_bfloat16 tile[3][32][33];
  const int k0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    int k = k0 + r, j = j0 + threadIdx.x;
    double x = (k < n && j < m) ? X[(int64_t)k * ldx + j] * (dr ? dr[k] : 1.0) : 0.0;
    __nv_bfloat16 s[3];
    split3(x, s);
    tile[0][r][threadIdx.x] = s[0];
    tile[1][r][threadIdx.x] = s[1];
    tile[2][r][threadIdx.x] = s[2];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    int j = j0 + r, k = k0 + threadIdx.x;
    if (j >= mp || k >= np) continue;
    __nv_bfloat16* row = Bext + (int64_t)j * (kSlices * (int64_t)np);
#pragma unroll
    for (int q = 0; q < kSlices; ++q) row[(int64_t)q * np + k] = tile[kPairB[q]][threadIdx.x][r];
  }
}

// A = I - Dl P Dr (fp32), identity in the padding.
__global__ void build_a32(const double* __restrict__ P, int64_t ldp, bool trans, const double* __restrict__ dl,
                          const double* __restrict__ dr, int n, int np, float* __restrict__ A) {
  const int64_t total = (int64_t)np * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / np), k = (int)(e % np);
    double v = (i == k) ? 1.0 : 0.0;
    if (i < n && k < n) v -= (dl ? dl[i] : 1.0) * p_elem(P, ldp, trans, i, k) * (dr ? dr[k] : 1.0);
    A[e] = (float)v;
  }
}

// Factor the 128 x 128 diagonal block at (k0, k0) in place (no pivoting) and form the
// inverses of its unit-lower and upper triangles. One block of 1024 threads.
template <class T16>
__global__ void __launch_bounds__(1024) panel_factor(float* __restrict__ A, int np, int k0, float* __restrict__ Linv,
                                                     float* __restrict__ Uinv, T16* __restrict__ Abf,
                                                     int* __restrict__ err) {
  extern __shared__ float sm[];
  float* a = sm;               // [NB][NB + 1]
  float* w = sm + NB * (NB + 1);  // [NB][NB + 1] scratch for the inverses
  constexpr int ld = NB + 1;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    a[r * ld + c] = A[(int64_t)(k0 + r) * np + k0 + c];
  }
  __syncthreads();
  for (int p = 0; p < NB; ++p) {
    float piv = a[p * ld + p];
    if (!(fabsf(piv) > 0.f) || !isfinite(piv)) {
      if (tid == 0) atomicExch(err, 1);
      piv = 1.f;
    }
    for (int r = p + 1 + tid; r < NB; r += blockDim.x) a[r * ld + p] /= piv;
    __syncthreads();
    const int rows = NB - p - 1;
    for (int e = tid; e < rows * rows; e += blockDim.x) {
      int r = p + 1 + e / rows, c = p + 1 + e % rows;
      a[r * ld + c] -= a[r * ld + p] * a[p * ld + c];
    }
    __syncthreads();
  }
  // Linv: inverse of the unit lower triangle, column by column (forward substitution)
  for (int c = tid; c < NB; c += blockDim.x) {
    for (int r = 0; r < NB; ++r) {
      float s = (r == c) ? 1.f : 0.f;
      for (int q = c; q < r; ++q) s -= a[r * ld + q] * w[q * ld + c];
      w[r * ld + c] = (r < c) ? 0.f : s;
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) Linv[e] = w[(e / NB) * ld + e % NB];
  __syncthreads();
  // Uinv: inverse of the upper triangle (back substitution), column by column
  for (int c = tid; c < NB; c += blockDim.x) {
    for (int r = NB - 1; r >= 0; --r) {
      float s = (r == c) ? 1.f : 0.f;
      for (int q = r + 1; q <= c; ++q) s -= a[r * ld + q] * w[q * ld + c];
      w[r * ld + c] = (r > c) ? 0.f : s / a[r * ld + r];
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    Uinv[e] = w[r * ld + c];
    float v = a[r * ld + c];
    A[(int64_t)(k0 + r) * np + k0 + c] = v;
    Abf[(int64_t)(k0 + r) * np + k0 + c] = to16<T16>(v);
  }
}

// Row panel: A[k-block rows, c] <- Linv * A[k-block rows, c] for columns c >= k0 + NB;
// also writes its 16-bit copy and the transposed copy Ut[c - (k0+NB)][r].
template <class T16>
__global__ void __launch_bounds__(kThreads) row_panel(float* __restrict__ A, int np, int k0,
                                                      const float* __restrict__ Linv, T16* __restrict__ Abf,
                                                      T16* __restrict__ Ut) {
  __shared__ float col[NB][33];
  const int c0 = k0 + NB + blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int r = ty; r < NB; r += 8) col[r][tx] = A[(int64_t)(k0 + r) * np + c0 + tx];
  __syncthreads();
  float out[NB / 8];
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    int r = ty + 8 * q;
    float s = 0.f;
    for (int p = 0; p <= r; ++p) s += Linv[r * NB + p] * col[p][tx];
    out[q] = s;
  }
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    int r = ty + 8 * q;
    A[(int64_t)(k0 + r) * np + c0 + tx] = out[q];
    Abf[(int64_t)(k0 + r) * np + c0 + tx] = to16<T16>(out[q]);
    Ut[(int64_t)(c0 - k0 - NB + tx) * NB + r] = to16<T16>(out[q]);
  }
}

// Column panel: A[r, k-block cols] <- A[r, k-block cols] * Uinv for rows r >= k0 + NB.
template <class T16>
__global__ void __launch_bounds__(kThreads) col_panel(float* __restrict__ A, int np, int k0,
                                                      const float* __restrict__ Uinv, T16* __restrict__ Abf) {
  __shared__ float rowv[32][NB + 1];
  const int r0 = k0 + NB + blockIdx.x * 32;
  for (int e = threadIdx.x; e < 32 * NB; e += kThreads) {
    int r = e / NB, c = e % NB;
    rowv[r][c] = A[(int64_t)(r0 + r) * np + k0 + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * NB; e += kThreads) {
    int r = e / NB, c = e % NB;
    float s = 0.f;
    for (int p = 0; p <= c; ++p) s += rowv[r][p] * Uinv[p * NB + c];
    A[(int64_t)(r0 + r) * np + k0 + c] = s;
    Abf[(int64_t)(r0 + r) * np + k0 + c] = to16<T16>(s);
  }
}

// Largest |x| of every column j < m of an fp64 matrix -> power-of-two scale 2^-e with
// max * 2^-e in [0.5, 1) (1 for an all-zero column).
__global__ void column_scales(const double* __restrict__ X, int64_t ld, int n, int m, float* __restrict__ scale,
                              float* __restrict__ inv_scale) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double mx = 0.0;
  for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(X[(int64_t)i * ld + j]));
  int e = 0;
  if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
  scale[j] = ldexpf(1.f, -e);
  inv_scale[j] = ldexpf(1.f, e);
}

// W[i][j] = (float)(R[i][j] * scale[j]) for i < n, j < m; zero elsewhere (padding).
__global__ void to_w32(const double* __restrict__ R, int64_t ldr, int n, int m, const float* __restrict__ scale,
                       float* __restrict__ W, int np, int mp) {
  const int64_t total = (int64_t)np * mp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / mp), j = (int)(e % mp);
    W[e] = (i < n && j < m) ? (float)(R[(int64_t)i * ldr + j] * (double)scale[j]) : 0.f;
  }
}

// X[i][j] (+)= W[i][j] * inv_scale[j]  (first = overwrite).
__global__ void add_w32(double* __restrict__ X, int64_t ldx, int n, int m, const float* __restrict__ W, int mp,
                        const float* __restrict__ inv_scale, bool first) {
  const int64_t total = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), j = (int)(e % m);
    double d = (double)W[(int64_t)i * mp + j] * (double)inv_scale[j];
    double* x = X + (int64_t)i * ldx + j;
    *x = first ? d : *x + d;
  }
}

// In place W[k-block] <- T * W[k-block] (T = 128 x 128 triangular inverse, lower or
// upper), and Yt[j][r] = 16-bit copy of the result, transposed (the update's B operand).
template <class T16, bool kLower>
__global__ void __launch_bounds__(kThreads) diag_apply(float* __restrict__ W, int mp, int k0,
                                                       const float* __restrict__ T, T16* __restrict__ Yt) {
  __shared__ float col[NB][33];
  const int j0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < NB; r += 8) col[r][tx] = W[(int64_t)(k0 + r) * mp + j0 + tx];
  __syncthreads();
  float out[NB / 8];
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    int r = ty + 8 * q;
    float s = 0.f;
    if (kLower) {
      for (int p = 0; p <= r; ++p) s += T[r * NB + p] * col[p][tx];
    } else {
      for (int p = r; p < NB; ++p) s += T[r * NB + p] * col[p][tx];
    }
    out[q] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB / 8; ++q) {
    int r = ty + 8 * q;
    W[(int64_t)(k0 + r) * mp + j0 + tx] = out[q];
    col[r][tx] = out[q];
  }
  __syncthreads();
  // transposed 16-bit copy: Yt[j0 + c][r]
  for (int e = threadIdx.x; e < 32 * NB; e += kThreads) {
    int c = e / NB, r = e % NB;
    Yt[(int64_t)(j0 + c) * NB + r] = to16<T16>(col[r][c]);
  }
}

// max |x| over an n x m fp64 matrix -> bits in *out (atomicMax on non-negative doubles).
__global__ void max_abs(const double* __restrict__ X, int64_t ld, int n, int m, unsigned long long* out,
                        int* nonfinite) {
  __shared__ double red[kThreads];
  double mx = 0.0;
  bool bad = false;
  const int64_t total = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < total; e += (int64_t)gridDim.x * kThreads) {
    double v = X[(e / m) * ld + e % m];
    if (!isfinite(v)) bad = true;
    mx = fmax(mx, fabs(v));
  }
  if (bad) atomicExch(nonfinite, 1);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}

inline int grid_for(int64_t total, int sm) {
  int64_t b = (total + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sm * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// ------------------------------------------------------------------ solver object
struct Layout {
  int n, m, np, mp, nblk;
};

struct Buffers {
  float* A32;
  void* Abf;
  void* Ut;
  float* Linv;
  float* Uinv;
  float* W;
  void* Yt;
  float* scale;
  float* inv_scale;
  __nv_bfloat16* Aext;
  __nv_bfloat16* Bext;
  double* R0;   // right-hand side (padded, ld = mp)
  double* X;    // solution (ld = mp)
  double* R;    // residual (ld = mp)
  double* vec;  // [2][np] per-row scratch (row sums, diagonal scalings)
  unsigned long long* red;  // [2] max|R|, max|X| bits
};

template <class Take>
void plan(const Layout& L, Take&& t) {
  t.template take<float>((size_t)L.np * L.np);                    // A32
  t.template take<uint16_t>((size_t)L.np * L.np);                 // Abf
  t.template take<uint16_t>((size_t)L.np * NB);                   // Ut
  t.template take<float>((size_t)L.nblk * NB * NB);               // Linv
  t.template take<float>((size_t)L.nblk * NB * NB);               // Uinv
  t.template take<float>((size_t)L.np * L.mp);                    // W
  t.template take<uint16_t>((size_t)L.mp * NB);                   // Yt
  t.template take<float>((size_t)L.mp);                           // scale
  t.template take<float>((size_t)L.mp);                           // inv_scale
  t.template take<__nv_bfloat16>((size_t)L.np * kSlices * L.np);  // Aext
  t.template take<__nv_bfloat16>((size_t)L.mp * kSlices * L.np);  // Bext
  t.template take<double>((size_t)L.np * L.mp);                   // R0
  t.template take<double>((size_t)L.np * L.mp);                   // X
  t.template take<double>((size_t)L.np * L.mp);                   // R
  t.template take<double>((size_t)2 * L.np);                      // vec
  t.template take<unsigned long long>(2);                         // red
}

struct Solver {
  rg_ctx* ctx;
  Layout L;
  Buffers b;
  bool bf16;
  cudaStream_t s;
  int* err;          // device error words: [0] zero pivot, [1] non-finite
  const double* P;
  int64_t ldp;
  bool transP;

  // Carves the solver's buffers out of the context workspace, after `extra_bytes`
  // reserved for the caller (returned in *extra).
  rg_status setup(int n, int m, bool use_bf16, cudaStream_t stream, size_t extra_bytes = 0, void** extra = nullptr) {
    L.n = n;
    L.m = m;
    L.np = (n + NB - 1) / NB * NB;
    L.mp = (m + NB - 1) / NB * NB;
    L.nblk = L.np / NB;
    bf16 = use_bf16;
    s = stream;
    extra_bytes = rg::align_up(extra_bytes, 256);
    rg::Sizer sz;
    plan(L, sz);
    void* ws = nullptr;
    rg_status st = rg::workspace(ctx, extra_bytes + sz.off, &ws);
    if (st != RG_OK) return st;
    if (extra) *extra = ws;
    rg::Carver cv(static_cast<char*>(ws) + extra_bytes);
    b.A32 = cv.take<float>((size_t)L.np * L.np);
    b.Abf = cv.take<uint16_t>((size_t)L.np * L.np);
    b.Ut = cv.take<uint16_t>((size_t)L.np * NB);
    b.Linv = cv.take<float>((size_t)L.nblk * NB * NB);
    b.Uinv = cv.take<float>((size_t)L.nblk * NB * NB);
    b.W = cv.take<float>((size_t)L.np * L.mp);
    b.Yt = cv.take<uint16_t>((size_t)L.mp * NB);
    b.scale = cv.take<float>(L.mp);
    b.inv_scale = cv.take<float>(L.mp);
    b.Aext = cv.take<__nv_bfloat16>((size_t)L.np * kSlices * L.np);
    b.Bext = cv.take<__nv_bfloat16>((size_t)L.mp * kSlices * L.np);
    b.R0 = cv.take<double>((size_t)L.np * L.mp);
    b.X = cv.take<double>((size_t)L.np * L.mp);
    b.R = cv.take<double>((size_t)L.np * L.mp);
    b.vec = cv.take<double>((size_t)2 * L.np);
    b.red = cv.take<unsigned long long>(2);
    err = ctx->d_scratch + 32;
    RG_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
    RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch + tc::kGemmErrorSlot, 0, sizeof(int), s));
    return RG_OK;
  }

  // P (shared by every set): its bf16 slices for the refinement product.
  rg_status set_matrix(const double* P_, int64_t ldp_, bool trans) {
    P = P_;
    ldp = ldp_;
    transP = trans;
    build_p_slices<<<grid_for((int64_t)L.np * L.np, ctx->sm_count), kThreads, 0, s>>>(P, ldp, transP, L.n, L.np,
                                                                                      b.Aext);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    return RG_OK;
  }

  template <class T16>
  rg_status factor_t(const double* dl, const double* dr) {
    build_a32<<<grid_for((int64_t)L.np * L.np, ctx->sm_count), kThreads, 0, s>>>(P, ldp, transP, dl, dr, L.n, L.np,
                                                                                 b.A32);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    T16* Abf = static_cast<T16*>(b.Abf);
    T16* Ut = static_cast<T16*>(b.Ut);
    const size_t psmem = 2 * NB * (NB + 1) * sizeof(float);
    RG_CUDA_TRY(ctx, cudaFuncSetAttribute(panel_factor<T16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
    for (int k = 0; k < L.nblk; ++k) {
      const int k0 = k * NB;
      panel_factor<T16><<<1, 1024, psmem, s>>>(b.A32, L.np, k0, b.Linv + (size_t)k * NB * NB,
                                               b.Uinv + (size_t)k * NB * NB, Abf, err);
      ++ctx->launches;
      const int rest = L.np - k0 - NB;
      if (rest > 0) {
        row_panel<T16><<<rest / 32, kThreads, 0, s>>>(b.A32, L.np, k0, b.Linv + (size_t)k * NB * NB, Abf, Ut);
        ++ctx->launches;
        col_panel<T16><<<rest / 32, kThreads, 0, s>>>(b.A32, L.np, k0, b.Uinv + (size_t)k * NB * NB, Abf);
        ++ctx->launches;
        RG_CUDA_TRY(ctx, cudaGetLastError());
        rg_status st = tc::gemm_f32(ctx, bf16, Abf + (size_t)(k0 + NB) * L.np + k0, L.np, Ut, NB, rest, rest, NB,
                                    b.A32 + (size_t)(k0 + NB) * L.np + k0 + NB, L.np, -1.f, 1.f, s);
        if (st != RG_OK) return st;
      }
      RG_CUDA_TRY(ctx, cudaGetLastError());
    }
    return RG_OK;
  }
  rg_status factor(const double* dl, const double* dr) {
    return bf16 ? factor_t<__nv_bfloat16>(dl, dr) : factor_t<__half>(dl, dr);
  }

  // X (+)= A^-1 src, where src is an fp64 n x m matrix (ld = mp), through the 16-bit factors.
  template <class T16>
  rg_status solve_t(const double* src, bool first) {
    const int cs_blocks = (L.m + 127) / 128;
    column_scales<<<cs_blocks, 128, 0, s>>>(src, L.mp, L.n, L.m, b.scale, b.inv_scale);
    ++ctx->launches;
    to_w32<<<grid_for((int64_t)L.np * L.mp, ctx->sm_count), kThreads, 0, s>>>(src, L.mp, L.n, L.m, b.scale, b.W,
                                                                               L.np, L.mp);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    const T16* Abf = static_cast<const T16*>(b.Abf);
    T16* Yt = static_cast<T16*>(b.Yt);
    const int jb = L.mp / 32;
    for (int k = 0; k < L.nblk; ++k) {  // forward: L y = w
      const int k0 = k * NB;
      diag_apply<T16, true><<<jb, kThreads, 0, s>>>(b.W, L.mp, k0, b.Linv + (size_t)k * NB * NB, Yt);
      ++ctx->launches;
      RG_CUDA_TRY(ctx, cudaGetLastError());
      const int rest = L.np - k0 - NB;
      if (rest > 0) {
        rg_status st = tc::gemm_f32(ctx, bf16, Abf + (size_t)(k0 + NB) * L.np + k0, L.np, Yt, NB, rest, L.mp, NB,
                                    b.W + (size_t)(k0 + NB) * L.mp, L.mp, -1.f, 1.f, s);
        if (st != RG_OK) return st;
      }
    }
    for (int k = L.nblk - 1; k >= 0; --k) {  // backward: U x = y
      const int k0 = k * NB;
      diag_apply<T16, false><<<jb, kThreads, 0, s>>>(b.W, L.mp, k0, b.Uinv + (size_t)k * NB * NB, Yt);
      ++ctx->launches;
      RG_CUDA_TRY(ctx, cudaGetLastError());
      if (k0 > 0) {
        rg_status st = tc::gemm_f32(ctx, bf16, Abf + k0, L.np, Yt, NB, k0, L.mp, NB, b.W, L.mp, -1.f, 1.f, s);
        if (st != RG_OK) return st;
      }
    }
    add_w32<<<grid_for((int64_t)L.n * L.m, ctx->sm_count), kThreads, 0, s>>>(b.X, L.mp, L.n, L.m, b.W, L.mp,
                                                                              b.inv_scale, first);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    return RG_OK;
  }
  rg_status solve(const double* src, bool first) {
    return bf16 ? solve_t<__nv_bfloat16>(src, first) : solve_t<__half>(src, first);
  }

  // R = R0 - X + Dl (P (Dr X)); returns max|R| / max|X| (synchronises the stream).
  rg_status residual(const double* dl, const double* dr, double* rel) {
    dim3 tg((L.mp + 31) / 32, (L.np + 31) / 32);
    build_x_slices<<<tg, dim3(32, 8), 0, s>>>(b.X, L.mp, dr, L.n, L.m, L.np, L.mp, b.Bext);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    rg_status st = tc::gemm_residual(ctx, b.Aext, (int64_t)kSlices * L.np, b.Bext, (int64_t)kSlices * L.np, L.n, L.m,
                                     kSlices * L.np, kResidualChunk, b.R, b.R0, b.X, dl, L.mp, s);
    if (st != RG_OK) return st;
    RG_CUDA_TRY(ctx, cudaMemsetAsync(b.red, 0, 2 * sizeof(unsigned long long), s));
    max_abs<<<grid_for((int64_t)L.n * L.m, ctx->sm_count), kThreads, 0, s>>>(b.R, L.mp, L.n, L.m, b.red, err + 1);
    ++ctx->launches;
    max_abs<<<grid_for((int64_t)L.n * L.m, ctx->sm_count), kThreads, 0, s>>>(b.X, L.mp, L.n, L.m, b.red + 1, err + 1);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    unsigned long long h[2];
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(h, b.red, sizeof(h), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    double r, x;
    memcpy(&r, &h[0], 8);
    memcpy(&x, &h[1], 8);
    *rel = x > 0 ? r / x : r;
    return check_errors();
  }

  rg_status check_errors() {
    int h[2] = {0, 0}, g = 0;
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(&g, ctx->d_scratch + tc::kGemmErrorSlot, sizeof(int), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (g) return rg::fail(ctx, RG_ERR_CUDA, "tensor-core GEMM timed out waiting on a barrier");
    if (h[0]) return rg::fail(ctx, RG_ERR_NUMERIC, "zero or non-finite pivot in the factorisation");
    if (h[1]) return rg::fail(ctx, RG_ERR_NUMERIC, "non-finite value in the solution or residual");
    return RG_OK;
  }

  // Factor, solve and refine one set whose right-hand side is already in b.R0.
  rg_status run(const double* dl, const double* dr, double tol, int max_sweeps, int* sweeps, double* rel_out) {
    rg_status st = factor(dl, dr);
    if (st == RG_OK) st = solve(b.R0, true);
    if (st != RG_OK) return st;
    double rel = INFINITY, prev = INFINITY;
    int sw = 0;
    bool done = false;
    for (; sw < max_sweeps; ++sw) {
      st = residual(dl, dr, &rel);
      if (st != RG_OK) return st;
      // converged, or stalled at the accuracy floor of the fp32-chunked residual product
      if (rel <= tol || (rel <= kStallFloor && rel > 0.5 * prev)) { done = true; break; }
      prev = rel;
      st = solve(b.R, false);
      if (st != RG_OK) return st;
    }
    *sweeps = sw + (done ? 1 : 0);
    *rel_out = rel;
    if (!done) return rg::fail(ctx, RG_ERR_NOT_CONVERGED, "refinement: residual %.3e > tol %.3e", rel, tol);
    return RG_OK;
  }
};

// ------------------------------------------------------------------ problem-specific kernels
// R0 = [F_NN diag(eps) | F_inf] (ld = mp), zero padding rows are never read.
__global__ void gebhart_rhs(const double* __restrict__ F, const double* __restrict__ eps, int n, int mp,
                            double* __restrict__ R0) {
  const int64_t total = (int64_t)n * (n + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / (n + 1)), j = (int)(e % (n + 1));
    R0[(int64_t)i * mp + j] = F[e] * (j < n ? eps[j] : 1.0);
  }
}

__global__ void copy_in(const double* __restrict__ src, int64_t lds, int n, int m, double* __restrict__ dst,
                        int64_t ldd) {
  const int64_t total = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), j = (int)(e % m);
    dst[(int64_t)i * ldd + j] = src[(int64_t)i * lds + j];
  }
}

// dL/deps_j = sum_i Lam_ij F_ij (j < n): one thread per column, fixed order.
__global__ void grad_eps(const double* __restrict__ Lam, int64_t ldl, const double* __restrict__ F, int n,
                         double* __restrict__ deps) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += Lam[(int64_t)i * ldl + j] * F[(int64_t)i * (n + 1) + j];
  deps[j] = s;
}

// dL/drho_k = sum_j B_kj Q_kj with Q = F^T Lam (row k): one warp per row.
__global__ void grad_rho(const double* __restrict__ B, const double* __restrict__ Q, int64_t ldq, int n,
                         double* __restrict__ drho) {
  const int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  double s = 0.0;
  for (int j = lane; j <= n; j += 32) s += B[(int64_t)k * (n + 1) + j] * Q[(int64_t)k * ldq + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) drho[k] = s;
}

// Radiative balance set-up: t_i = sum_j B_ij (env included), g_i = sigma eps_i A_i,
// dl_i = 1 / t_i, R0_i = (Q_i + g_i B_i,inf T_sink^4) / (g_i t_i).
__global__ void balance_setup(const double* __restrict__ B, const double* __restrict__ eps,
                              const double* __restrict__ area, const double* __restrict__ Q, double u_sink,
                              double sigma, int n, int mp, double* __restrict__ t, double* __restrict__ dl,
                              double* __restrict__ R0, int* err) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int j = lane; j <= n; j += 32) s += B[(int64_t)i * (n + 1) + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double g = sigma * eps[i] * area[i];
    if (!(s > 0.0) || !(g > 0.0)) atomicExch(err, 1);
    t[i] = s;
    dl[i] = 1.0 / s;
    if (R0) R0[(int64_t)i * mp] = (Q[i] + g * B[(int64_t)i * (n + 1) + n] * u_sink) / (g * s);
  }
}

__global__ void quartic_root(const double* __restrict__ u, int64_t ldu, int n, double* __restrict__ T, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = u[(int64_t)i * ldu];
  if (!(v > 0.0)) atomicExch(err, 1);
  T[i] = sqrt(sqrt(v));
}

// Adjoint balance right-hand side: R0_i = (dT_i / (4 T_i^3)) / t_i.
__global__ void balance_adj_rhs(const double* __restrict__ T, const double* __restrict__ dT,
                                const double* __restrict__ t, int n, int mp, double* __restrict__ R0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double Ti = T[i];
  R0[(int64_t)i * mp] = dT[i] / (4.0 * Ti * Ti * Ti) / t[i];
}

// dB_ij = -nu_i (u_i - u_j) (u_{n} = T_sink^4), deps_i = -(nu_i / eps_i) sum_j B_ij (u_i - u_j)
// with nu = g o mu the solution of the transposed balance. One warp per row.
__global__ void balance_adj_out(const double* __restrict__ B, const double* __restrict__ eps,
                                const double* __restrict__ T, const double* __restrict__ nu, int64_t ldnu,
                                double u_sink, int n, double* __restrict__ dB, double* __restrict__ deps) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double Ti = T[i];
  const double ui = Ti * Ti * Ti * Ti;
  const double v = nu[(int64_t)i * ldnu];
  double s = 0.0;
  for (int j = lane; j <= n; j += 32) {
    double uj;
    if (j < n) {
      double Tj = T[j];
      uj = Tj * Tj * Tj * Tj;
    } else {
      uj = u_sink;
    }
    dB[(int64_t)i * (n + 1) + j] = -v * (ui - uj);
    s += B[(int64_t)i * (n + 1) + j] * (ui - uj);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) deps[i] = -(v / eps[i]) * s;
}


// ------------------------------------------------------------------ least-squares optimum
// Restrictions on the active entries x_ij of F (Sec. 3.5.5, Eq. 3.41-3.43):
//   closure     C_i:  sum_j a_ij x_ij = 1
//   reciprocity R_ij: Omega_i a_ij x_ij - Omega_j a_ji x_ji = 0   (i < j)
// (a = active mask). With mu = (A A^T)^-1 (A x - b) and x-hat = x - A^T mu, eliminating
// the diagonal reciprocity block d_ij = Omega_i^2 a_ij + Omega_j^2 a_ji leaves
//   S mu_C = r_C - sum_j Omega_i a_ij rho_ij / d_ij,
//   S_ii = n_i - sum_j Omega_i^2 a_ij / d_ij,   S_ij = Omega_i Omega_j a_ij a_ji / d_ij,
// with rho_ij = Omega_i a_ij x_ij - Omega_j a_ji x_ji and r_C,i = sum_j a_ij x_ij - 1, and
//   x-hat_ij = x_ij - mu_i - Omega_i nu_ij,  nu_ij = (rho_ij - Omega_i a_ij mu_i + Omega_j a_ji mu_j) / d_ij
// for active pairs (x-hat = x - mu_i on the environment column and the diagonal).
// A closure row without active entries is dropped (mu_i = 0), as are pairs with d = 0.

__global__ void lsq_init(const double* __restrict__ F, int n, int spva, double* __restrict__ F0,
                         uint8_t* __restrict__ mask) {
  const int64_t total = (int64_t)n * (n + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    double x = F[e];
    F0[e] = x;
    mask[e] = (!spva || x != 0.0) ? 1 : 0;
  }
}

// One warp per row i: the diagonal of S and the right-hand side, scaled by 1/S_ii for
// the solver (which sees I - Dl P with Dl = 1/S_ii and P = -offdiag(S)).
__global__ void lsq_rows(const double* __restrict__ F0, const uint8_t* __restrict__ mask,
                         const double* __restrict__ om, int n, double* __restrict__ dl, double* __restrict__ R0,
                         int64_t ldr) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int64_t ld = n + 1;
  const double oi = om[i];
  double cnt = 0.0, rc = 0.0, sd = 0.0, sr = 0.0;
  for (int j = lane; j <= n; j += 32) {
    const double a = mask[i * ld + j];
    const double x = a * F0[i * ld + j];
    cnt += a;
    rc += x;
    if (j < n && j != i && a != 0.0) {
      const double oj = om[j];
      const double at = mask[(int64_t)j * ld + i];
      const double xt = at * F0[(int64_t)j * ld + i];
      const double d = oi * oi + oj * oj * at;
      const double rho = oi * x - oj * xt;
      sd += oi * oi / d;
      sr += oi * rho / d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    rc += __shfl_xor_sync(0xffffffffu, rc, o);
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
  }
  if (lane == 0) {
    double sii = cnt - sd, rhs = (rc - 1.0) - sr;
    if (cnt == 0.0) { sii = 1.0; rhs = 0.0; }
    dl[i] = 1.0 / sii;
    R0[(int64_t)i * ldr] = rhs / sii;
  }
}

// P_ij = -S_ij (i != j), 0 on the diagonal.
__global__ void lsq_offdiag(const uint8_t* __restrict__ mask, const double* __restrict__ om, int n,
                            double* __restrict__ P) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    double v = 0.0;
    if (i != j) {
      const int64_t ld = n + 1;
      const double a = mask[i * ld + j], at = mask[(int64_t)j * ld + i];
      if (a != 0.0 && at != 0.0) {
        const double oi = om[i], oj = om[j];
        v = -(oi * oj) / (oi * oi + oj * oj);
      }
    }
    P[e] = v;
  }
}

// x-hat from the closure multipliers mu; negative results are counted and dropped from
// the next mask (NNR).
__global__ void lsq_apply(const double* __restrict__ F0, const uint8_t* __restrict__ mask,
                          const double* __restrict__ om, const double* __restrict__ mu, int64_t ldmu, int n,
                          double* __restrict__ F, uint8_t* __restrict__ mask_next, int* __restrict__ negatives) {
  const int64_t ld = n + 1;
  const int64_t total = (int64_t)n * ld;
  int neg = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e % ld);
    const uint8_t a = mask[e];
    double xh = 0.0;
    if (a) {
      const double mi = mu[(int64_t)i * ldmu];
      xh = F0[e] - mi;
      if (j < n && j != i) {
        const double oi = om[i], oj = om[j];
        const double at = mask[(int64_t)j * ld + i];
        const double xt = at * F0[(int64_t)j * ld + i];
        const double d = oi * oi + oj * oj * at;
        const double rho = oi * F0[e] - oj * xt;
        const double nu = (rho - oi * mi + oj * at * mu[(int64_t)j * ldmu]) / d;
        xh -= oi * nu;
      }
    }
    F[e] = xh;
    const bool drop = a && xh < 0.0;
    mask_next[e] = (a && !drop) ? 1 : 0;
    neg += drop ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) neg += __shfl_xor_sync(0xffffffffu, neg, o);
  if ((threadIdx.x & 31) == 0 && neg) atomicAdd(negatives, neg);
}

rg_status check_common(rg_ctx* ctx, int32_t n, int32_t precision, double tol, int32_t max_sweeps) {
  RG_ARG_CHECK(ctx, n > 0 && n <= 32768, "dense solve: n = %d outside [1, 32768]", n);
  RG_ARG_CHECK(ctx, precision == RG_PREC_BF16_IR || precision == RG_PREC_FP16_IR, "unknown precision %d", precision);
  RG_ARG_CHECK(ctx, tol >= 1e-13 && tol < 1.0, "tolerance %.3e outside [1e-13, 1)", tol);
  RG_ARG_CHECK(ctx, max_sweeps >= 1, "max_sweeps must be >= 1");
  return RG_OK;
}

}  // namespace

extern "C" {

rg_status rg_enforce_lsq(rg_ctx* ctx, int32_t n, const double* omega_d, double* F_d, int32_t nnr, int32_t spva,
                         int32_t max_passes, int32_t* passes_out_h, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n > 0 && n <= 4096 && omega_d && F_d && max_passes >= 1, "rg_enforce_lsq: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn1 = (size_t)n * (n + 1);
  rg::Sizer ex;
  ex.take<double>(nn1);            // F0
  ex.take<uint8_t>(nn1);           // mask
  ex.take<uint8_t>(nn1);           // next mask
  ex.take<double>((size_t)n * n);  // P
  ex.take<double>(n);              // dl
  ex.take<int>(4);                 // negative counter
  Solver sv{ctx};
  void* extra = nullptr;
  rg_status st = sv.setup(n, 1, false, s, ex.off, &extra);
  if (st != RG_OK) return st;
  rg::Carver cv(extra);
  double* F0 = cv.take<double>(nn1);
  uint8_t* mask = cv.take<uint8_t>(nn1);
  uint8_t* mask2 = cv.take<uint8_t>(nn1);
  double* P = cv.take<double>((size_t)n * n);
  double* dl = cv.take<double>(n);
  int* negs = cv.take<int>(4);
  const int g = grid_for((int64_t)nn1, ctx->sm_count);
  lsq_init<<<g, kThreads, 0, s>>>(F_d, n, spva, F0, mask);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  int passes = 0;
  while (true) {
    ++passes;
    lsq_rows<<<(n + 7) / 8, 256, 0, s>>>(F0, mask, omega_d, n, dl, sv.b.R0, sv.L.mp);
    ++ctx->launches;
    lsq_offdiag<<<grid_for((int64_t)n * n, ctx->sm_count), kThreads, 0, s>>>(mask, omega_d, n, P);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    st = sv.set_matrix(P, n, false);
    int sw = 0;
    double rel = 0.0;
    if (st == RG_OK) st = sv.run(dl, nullptr, 1e-13, 40, &sw, &rel);
    if (st != RG_OK) return st;
    RG_CUDA_TRY(ctx, cudaMemsetAsync(negs, 0, sizeof(int), s));
    lsq_apply<<<g, kThreads, 0, s>>>(F0, mask, omega_d, sv.b.X, sv.L.mp, n, F_d, mask2, negs);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    int h = 0;
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, negs, sizeof(int), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (!nnr || h == 0) break;
    if (passes >= max_passes) {
      if (passes_out_h) *passes_out_h = passes;
      return rg::fail(ctx, RG_ERR_NOT_CONVERGED, "rg_enforce_lsq: %d negative entries after %d passes", h, passes);
    }
    std::swap(mask, mask2);
  }
  if (passes_out_h) *passes_out_h = passes;
  return RG_OK;
}

rg_status rg_gebhart(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets, const double* eps_d,
                     const double* rho_d, int32_t precision, double tol, int32_t max_sweeps, double* B_d,
                     int32_t* sweeps_out_h, double* resid_out_h, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, max_sweeps);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, F_d && eps_d && rho_d && B_d && n_sets > 0, "rg_gebhart: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Solver sv{ctx};
  st = sv.setup(n, n + 1, precision == RG_PREC_BF16_IR, s);
  if (st == RG_OK) st = sv.set_matrix(F_d, n + 1, false);
  if (st != RG_OK) return st;
  int max_sw = 0;
  double max_rel = 0.0;
  for (int set = 0; set < n_sets; ++set) {
    const double* eps = eps_d + (size_t)set * n;
    const double* rho = rho_d + (size_t)set * n;
    gebhart_rhs<<<grid_for((int64_t)n * (n + 1), ctx->sm_count), kThreads, 0, s>>>(F_d, eps, n, sv.L.mp, sv.b.R0);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    int sw = 0;
    double rel = 0.0;
    st = sv.run(nullptr, rho, tol, max_sweeps, &sw, &rel);
    if (st != RG_OK && st != RG_ERR_NOT_CONVERGED) return st;
    copy_in<<<grid_for((int64_t)n * (n + 1), ctx->sm_count), kThreads, 0, s>>>(
        sv.b.X, sv.L.mp, n, n + 1, B_d + (size_t)set * n * (n + 1), n + 1);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    max_sw = sw > max_sw ? sw : max_sw;
    max_rel = rel > max_rel ? rel : max_rel;
    if (st != RG_OK) {
      if (sweeps_out_h) *sweeps_out_h = max_sw;
      if (resid_out_h) *resid_out_h = max_rel;
      return st;
    }
  }
  if (sweeps_out_h) *sweeps_out_h = max_sw;
  if (resid_out_h) *resid_out_h = max_rel;
  return RG_OK;
}

rg_status rg_gebhart_adjoint(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets, const double* eps_d,
                             const double* rho_d, const double* B_d, const double* dB_d, int32_t precision,
                             double tol, int32_t max_sweeps, double* deps_d, double* drho_d, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, max_sweeps);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, F_d && eps_d && rho_d && B_d && dB_d && deps_d && drho_d && n_sets > 0,
               "rg_gebhart_adjoint: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Solver sv{ctx};
  // K^T = I - diag(rho) F_NN^T
  st = sv.setup(n, n + 1, precision == RG_PREC_BF16_IR, s);
  if (st == RG_OK) st = sv.set_matrix(F_d, n + 1, true);
  if (st != RG_OK) return st;
  for (int set = 0; set < n_sets; ++set) {
    const double* rho = rho_d + (size_t)set * n;
    const size_t off = (size_t)set * n * (n + 1);
    copy_in<<<grid_for((int64_t)n * (n + 1), ctx->sm_count), kThreads, 0, s>>>(dB_d + off, n + 1, n, n + 1,
                                                                                sv.b.R0, sv.L.mp);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    int sw = 0;
    double rel = 0.0;
    st = sv.run(rho, nullptr, tol, max_sweeps, &sw, &rel);
    if (st != RG_OK) return st;
    // deps_j = sum_i Lam_ij F_ij
    grad_eps<<<(n + 127) / 128, 128, 0, s>>>(sv.b.X, sv.L.mp, F_d, n, deps_d + (size_t)set * n);
    ++ctx->launches;
    // Q = F^T Lam (fp64-accurate sliced product), then drho_k = sum_j B_kj Q_kj
    dim3 tg((sv.L.mp + 31) / 32, (sv.L.np + 31) / 32);
    build_x_slices<<<tg, dim3(32, 8), 0, s>>>(sv.b.X, sv.L.mp, nullptr, n, n + 1, sv.L.np, sv.L.mp, sv.b.Bext);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    st = tc::gemm_residual(ctx, sv.b.Aext, (int64_t)kSlices * sv.L.np, sv.b.Bext, (int64_t)kSlices * sv.L.np, n,
                           n + 1, kSlices * sv.L.np, kResidualChunk, sv.b.R, nullptr, nullptr, nullptr, sv.L.mp, s);
    if (st != RG_OK) return st;
    grad_rho<<<(n + 7) / 8, 256, 0, s>>>(B_d + off, sv.b.R, sv.L.mp, n, drho_d + (size_t)set * n);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
  }
  return sv.check_errors();
}

rg_status rg_temperatures(rg_ctx* ctx, int32_t n, const double* B_d, const double* eps_d, const double* area_d,
                          const double* Q_d, double T_sink, double sigma, int32_t precision, double tol, double* T_d,
                          void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, 1);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, B_d && eps_d && area_d && Q_d && T_d && T_sink >= 0.0 && sigma > 0.0,
               "rg_temperatures: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Solver sv{ctx};
  st = sv.setup(n, 1, precision == RG_PREC_BF16_IR, s);
  if (st == RG_OK) st = sv.set_matrix(B_d, n + 1, false);
  if (st != RG_OK) return st;
  double* t = sv.b.vec;
  double* dl = sv.b.vec + sv.L.np;
  const double u_sink = T_sink * T_sink * T_sink * T_sink;
  balance_setup<<<(n + 7) / 8, 256, 0, s>>>(B_d, eps_d, area_d, Q_d, u_sink, sigma, n, sv.L.mp, t, dl, sv.b.R0,
                                             sv.err);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  st = sv.check_errors();
  int sw = 0;
  double rel = 0.0;
  if (st == RG_OK) st = sv.run(dl, nullptr, tol, 16, &sw, &rel);
  if (st == RG_OK) {
    quartic_root<<<(n + 127) / 128, 128, 0, s>>>(sv.b.X, sv.L.mp, n, T_d, sv.err);
    ++ctx->launches;
    st = sv.check_errors();
  }
  return st;
}

rg_status rg_temperatures_adjoint(rg_ctx* ctx, int32_t n, const double* B_d, const double* eps_d,
                                  const double* area_d, double T_sink, double sigma, const double* T_d,
                                  const double* dT_d, int32_t precision, double tol, double* dB_d, double* deps_d,
                                  void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, 1);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, B_d && eps_d && area_d && T_d && dT_d && dB_d && deps_d && sigma > 0.0,
               "rg_temperatures_adjoint: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Solver sv{ctx};
  st = sv.setup(n, 1, precision == RG_PREC_BF16_IR, s);
  if (st == RG_OK) st = sv.set_matrix(B_d, n + 1, true);
  if (st != RG_OK) return st;
  double* t = sv.b.vec;
  double* dl = sv.b.vec + sv.L.np;
  const double u_sink = T_sink * T_sink * T_sink * T_sink;
  balance_setup<<<(n + 7) / 8, 256, 0, s>>>(B_d, eps_d, area_d, eps_d, u_sink, sigma, n, sv.L.mp, t, dl, nullptr,
                                             sv.err);
  ++ctx->launches;
  balance_adj_rhs<<<(n + 127) / 128, 128, 0, s>>>(T_d, dT_d, t, n, sv.L.mp, sv.b.R0);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  st = sv.check_errors();
  int sw = 0;
  double rel = 0.0;
  if (st == RG_OK) st = sv.run(dl, nullptr, tol, 16, &sw, &rel);
  if (st == RG_OK) {
    balance_adj_out<<<(n + 7) / 8, 256, 0, s>>>(B_d, eps_d, T_d, sv.b.X, sv.L.mp, u_sink, n, dB_d, deps_d);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    st = sv.check_errors();
  }
  return st;
}

}  // extern "C"
