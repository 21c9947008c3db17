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
//   1. A = I - Dl P Dr in 16-bit (bf16 or fp16), padded to a multiple of 128 with the
//      identity, and e0 = ||Dl P Dr||_inf.
//   2. Approximate inverse by Newton-Schulz iteration X <- X (2I - A X) from X = I: the
//      error I - A X squares every step (its inf-norm starts at e0 < 1), so
//      ceil(log2(log(tol16) / log(e0))) + 1 steps reach the 16-bit floor. Each step is two
//      tcgen05 GEMMs whose epilogues write the 16-bit operands of the next one (the
//      transposed copies the K-major layout needs included).
//   3. Solve and refine: X64 = M R0, then R = R0 - X + Dl (P (Dr X)) with P and Dr X each
//      split into three bf16 slices (24 bits) and the six leading slice products summed by
//      one tcgen05 GEMM over a 6N-long K with compensated fp32 chunks (fp64-accurate);
//      X64 += M R is one more GEMM. It stops when max|R| <= tol max|X| (or stalls below
//      1e-8, above the accuracy floor of that product).
// The transposed systems reuse the same code with P read transposed.
#include <cmath>
#include <utility>

#include "tc_gemm.cuh"

namespace {

constexpr int NB = 128;          // panel width == GEMM tile height
constexpr int kSlices = 6;       // slice pairs of the refinement product
constexpr int kResidualChunk = 2;  // K blocks (of 64) per compensated fp32 chunk (leading pair)
constexpr int kResidualTailChunk = 16;  // K blocks per chunk for the pairs after the leading one
constexpr int kThreads = 256;
// Below this relative residual a sweep that no longer halves it ends the refinement.
// The residual product's own accuracy floor (fp32 accumulation inside each 128-long
// chunk) was measured between 1e-10 and 1.3e-9 for N = 512 ... 10,240.
constexpr double kStallFloor = 1e-8;
constexpr int kMaxNewtonSchulz = 24;
// Sweeps whose previous relative residual is above this use half of the slice pairs.
constexpr double kCoarseAbove = 1e-3;

__device__ __forceinline__ double p_elem(const double* P, int64_t ldp, bool trans, int i, int k) {
  return trans ? P[(int64_t)k * ldp + i] : P[(int64_t)i * ldp + k];
}

template <class T>
__device__ __forceinline__ T to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }

// Split x into three bf16 slices whose sum carries ~24 significant bits:
// s0 = bf16(x), s1 = bf16(x - s0), s2 = bf16(x - s0 - s1), each rounding to nearest, ties to
// even, and each difference exact. GB300 runs fp64 (conversions included) at a small
// fraction of its integer rate, so the hot callers take the split on the bit pattern
// (split3_bits) and fall back to the fp64 definition (split3_fp64) only where an input or
// an intermediate leaves the ranges the integer path covers. Both give the same slices
// for every input.
__device__ __forceinline__ void split3_fp64(double x, __nv_bfloat16* s) {
  s[0] = __double2bfloat16(x);
  const double r = x - (double)__bfloat162float(s[0]);
  s[1] = __double2bfloat16(r);
  s[2] = __double2bfloat16(r - (double)__bfloat162float(s[1]));
}

// Bits 31..24 of the normalised magnitude h (leading one at bit 31; l holds the bits
// below h's) rounded to nearest, ties to even, as a bf16 of sign sg (bit 31) and biased
// exponent be; (h, l) becomes the remainder's magnitude in the same frame and sg its sign.
__device__ __forceinline__ __nv_bfloat16 round8_bits(uint32_t& h, uint32_t& l, uint32_t& sg, int be) {
  const uint32_t up = ((h >> 23) & 1u) & ((((h & 0x007fffffu) | l) != 0u) | ((h >> 24) & 1u));
  const __nv_bfloat16 v =
      __ushort_as_bfloat16((unsigned short)((sg >> 16) | (((uint32_t)be << 7) + ((h >> 24) + up - 128u))));
  h &= 0x00ffffffu;
  if (up) {  // the remainder is negative: 2^24 (in units of h's bit 0) minus the dropped bits
    h = 0x01000000u - h - (l != 0u);
    l = 0u - l;
    sg ^= 0x80000000u;
  }
  return v;
}

// Shift the 64-bit magnitude (h, l) != 0 left until its leading one is bit 31 of h;
// returns the leading bit's position before the shift (0 .. 63).
__device__ __forceinline__ int normalise_bits(uint32_t& h, uint32_t& l) {
  if (h != 0u) {
    const int sh = __clz((int)h);
    if (sh) {
      h = (h << sh) | (l >> (32 - sh));
      l <<= sh;
    }
    return 63 - sh;
  }
  const int sh = __clz((int)l);
  h = l << sh;
  l = 0u;
  return 31 - sh;
}

// split3 on the two 32-bit words of x, for x zero or 2^-126 <= |x| < 2^127 with normal
// slices; false elsewhere (the slices are then unusable). The significand M of x (53 bits,
// unit ulp(x) = 2^(E - 1075)) is rounded to 8 bits at bit 45; the remainder, a signed
// integer of at most 45 bits in the same unit, is normalised and rounded to 8 bits; what
// that leaves is normalised and rounded once more.
__device__ __forceinline__ bool split3_bits(double x, __nv_bfloat16* s) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  uint32_t sg = hi & 0x80000000u;
  const uint32_t t = hi & 0x7fffffffu;
  const __nv_bfloat16 zero = __ushort_as_bfloat16((unsigned short)0);
  if ((t | lo) == 0u) {
    s[0] = __ushort_as_bfloat16((unsigned short)(sg >> 16));
    s[1] = s[2] = zero;
    return true;
  }
  const int E = (int)(t >> 20);
  bool ok = E >= 897 && E <= 1149;
  // s0: the 7 leading mantissa bits, rounded at bit 12 of the high word (bit 44 of x)
  const uint32_t up = ((t & 0x1fffu) + 0xfffu + ((lo != 0u) | ((t >> 13) & 1u))) >> 13;
  s[0] = __ushort_as_bfloat16((unsigned short)((sg >> 16) | ((((t & ~0x1fffu) + (up << 13)) >> 13) - (896u << 7))));
  // D = M - s0 in units of ulp(x): the dropped 45 bits, or 2^45 minus them when rounded up
  uint32_t h = t & 0x1fffu, l = lo;
  if (up) {
    h = 0x2000u - h - (l != 0u);
    l = 0u - l;
    sg ^= 0x80000000u;
  }
  if ((h | l) == 0u) {
    s[1] = s[2] = zero;
    return ok;
  }
  const int p1 = normalise_bits(h, l);  // bf16 exponent of D's bit 0: E - 1075 + 127
  const int be1 = E - 948 + p1;
  s[1] = round8_bits(h, l, sg, be1);
  if ((h | l) == 0u) {
    s[2] = zero;
    return ok && be1 >= 1;
  }
  const int be2 = be1 - 63 + normalise_bits(h, l);  // the frame was shifted by 63 - p1
  s[2] = round8_bits(h, l, sg, be2);
  return ok && be1 >= 1 && be2 >= 1;
}

// The split of x_d[i] into slices_d[3 i .. 3 i + 2] (rg_refinement_slices). The loop's
// trip count is the same for every thread of a block, so the vote sees whole warps.
__global__ void split_slices(const double* __restrict__ x, int64_t n, __nv_bfloat16* __restrict__ out) {
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < n;
    const double v = in ? x[i] : 0.0;
    __nv_bfloat16 s[3];
    const bool ok = split3_bits(v, s);
    if (__any_sync(0xffffffffu, !ok)) {
      if (!ok) split3_fp64(v, s);
    }
    if (in) {
      out[3 * i] = s[0];
      out[3 * i + 1] = s[1];
      out[3 * i + 2] = s[2];
    }
  }
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
    if (!split3_bits(x, s)) split3_fp64(x, s);
    __nv_bfloat16* row = Aext + (int64_t)i * (kSlices * (int64_t)np);
#pragma unroll
    for (int q = 0; q < kSlices; ++q) row[(int64_t)q * np + k] = s[kPairA[q]];
  }
}

// B_ext[j][q * Np + k] = slice kPairB[q] of (Dr X)(k, j); the refinement product's B operand.
// Tiled transpose through shared memory: block (32 x 8) covers a 32 x 32 tile of X. With
// red / colmax set it also zeroes red[0..1] and colmax[0 .. mp) for the residual GEMM that
// follows it on the stream (no separate memset).
__global__ void build_x_slices(const double* __restrict__ X, int64_t ldx, const double* __restrict__ dr, int n,
                               int m, int np, int mp, __nv_bfloat16* __restrict__ Bext,
                               unsigned long long* red = nullptr, unsigned long long* colmax = nullptr) {
  __shared__ __nv_bfloat16 tile[3][32][33];
  const int k0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  if (blockIdx.y == 0 && threadIdx.y == 0) {
    if (colmax && j0 + (int)threadIdx.x < mp) colmax[j0 + threadIdx.x] = 0ull;
    if (red && blockIdx.x == 0 && threadIdx.x < 2) red[threadIdx.x] = 0ull;
  }
  for (int r = threadIdx.y; r < 32; r += 8) {  // warp-uniform: threadIdx.y is the warp
    const int k = k0 + r, j = j0 + threadIdx.x;
    const bool in = k < n && j < m;
    double xv = 0.0, dv = 1.0;
    if (in) {
      xv = X[(int64_t)k * ldx + j];
      if (dr) dv = dr[k];
    }
    const double x = in ? xv * dv : 0.0;
    __nv_bfloat16 s[3];
    const bool ok = split3_bits(x, s);
    if (__any_sync(0xffffffffu, !ok)) {  // the fp64 definition, for the lanes that need it
      if (!ok) split3_fp64(x, s);
    }
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

// (float)(x * 2^-e) on the two 32-bit words of x, for x zero, or normal with x 2^-e and
// its float normal: the exponent moves by -e (exact), the 52-bit mantissa is rounded to 23
// bits, to nearest, ties to even (a carry moves up the exponent). Clears ok elsewhere.
__device__ __forceinline__ float scaled_bits(double x, int e, bool& ok) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u, t = hi & 0x7fffffffu;
  if ((t | lo) == 0u) return __uint_as_float(sign);
  const int E = (int)(t >> 20);
  const int fe = E - e - 896;  // float biased exponent: E - 1023 - e + 127
  const uint32_t m = ((t & 0xfffffu) << 3) | (lo >> 29), rem = lo & 0x1fffffffu;
  const uint32_t up = (rem > 0x10000000u) | ((rem == 0x10000000u) & m);
  const uint32_t bits = ((uint32_t)fe << 23) + m + (up & 1u);
  ok = ok && E >= 1 && E <= 2046 && fe >= 1 && fe <= 254 && bits < 0x7f800000u;
  return __uint_as_float(sign | bits);
}

// A16 = I - Dl P Dr (16-bit, identity padding), the first Newton-Schulz iterate
// X16 = 2I - A = I + Dl P Dr (the step from X = I, done here instead of by two GEMMs) and
// its transpose Xt16, and the largest row and column sums of |Dl P Dr| (||E||_inf into
// e0_bits[0], ||E||_1 into e0_bits[1], atomicMax on their bits). One warp per row; the grid
// has at least mp threads.
template <class T16>
__global__ void build_ns_start(const double* __restrict__ P, int64_t ldp, bool trans, const double* __restrict__ dl,
                               const double* __restrict__ dr, int n, int np, T16* __restrict__ A16,
                               T16* __restrict__ X16, T16* __restrict__ Xt16, unsigned long long* e0_bits,
                               unsigned long long* colmax, int mp) {
  // colmax[0 .. mp) = 0 for the column maxima of the first correction (no separate memset)
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < mp) colmax[tid] = 0ull;
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= np) return;
  double rs = 0.0, cs = 0.0;  // row i and column i of |E|
  const double li = (i < n && dl) ? dl[i] : 1.0;
  const double ri = (i < n && dr) ? dr[i] : 1.0;
  for (int k = lane; k < np; k += 32) {
    double e = 0.0, et = 0.0;  // (Dl P Dr)_ik and (Dl P Dr)_ki
    if (i < n && k < n) {
      e = li * p_elem(P, ldp, trans, i, k) * (dr ? dr[k] : 1.0);
      et = (dl ? dl[k] : 1.0) * p_elem(P, ldp, trans, k, i) * ri;
    }
    rs += fabs(e);
    cs += fabs(et);
    const double one = (i == k) ? 1.0 : 0.0;
    const int64_t o = (int64_t)i * np + k;
    A16[o] = to16<T16>((float)(one - e));
    X16[o] = to16<T16>((float)(one + e));
    Xt16[o] = to16<T16>((float)(one + et));
  }
  for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
  for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
  if (lane == 0) {
    atomicMax(e0_bits, (unsigned long long)__double_as_longlong(rs));
    atomicMax(e0_bits + 1, (unsigned long long)__double_as_longlong(cs));
  }
}

// Largest |R_ij| of each column j < m (bits, atomicMax); block (32 x 8) per 32 columns x 256 rows.
__global__ void column_max(const double* __restrict__ R, int64_t ld, int n, int m, unsigned long long* colmax) {
  __shared__ double red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int r0 = blockIdx.y * 256;
  double mx = 0.0;
  if (c < m)
    for (int r = r0 + threadIdx.y; r < min(n, r0 + 256); r += 8) mx = fmax(mx, fabs(R[(int64_t)r * ld + c]));
  red[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && c < m) {
    for (int y = 1; y < 8; ++y) mx = fmax(mx, red[y][threadIdx.x]);
    atomicMax(&colmax[c], (unsigned long long)__double_as_longlong(mx));
  }
}

// The refinement's stopping rule evaluated on the device, for a correction launched
// before the host has read the residual it corrects: status = the solver's status words
// (null: no guard), tol / prev / coarse as the host's loop has them. When the sweep ends
// the refinement (converged or stalled) or reported an error, the correction is skipped:
// the transposition returns at once and sets *skip, which its GEMM reads.
struct SweepGuard {
  const int* status = nullptr;
  double tol = 0.0, prev = 0.0;
  int coarse = 0;
  int* skip = nullptr;
};

__device__ __forceinline__ bool sweep_ends(const SweepGuard& g) {
  const volatile int* w = g.status;
  const double r = __hiloint2double(w[7], w[6]), x = __hiloint2double(w[9], w[8]);
  const double rel = x > 0 ? r / x : r;
  const bool done = !g.coarse && (rel <= g.tol || (rel <= kStallFloor && rel > 0.5 * g.prev));
  return done || w[0] || w[1] || w[4];
}

// Rt16[j][i] = 16-bit (R_ij * 2^-e_j) with max_i |R_ij| 2^-e_j in [0.5, 1), zero padding;
// colscale[j] = 2^e_j. Tiled transpose through shared memory, block (32 x 8).
template <class T16>
__global__ void scaled_transpose16(const double* __restrict__ R, int64_t ld, int n, int m, int np, int mp,
                                   const unsigned long long* __restrict__ colmax, T16* __restrict__ Rt,
                                   float* __restrict__ colscale, const SweepGuard guard) {
  __shared__ float tile[32][33];
  if (guard.status) {  // one thread per block evaluates the rule (an fp64 division), the block follows
    __shared__ int s_end;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      s_end = sweep_ends(guard) ? 1 : 0;
      if (blockIdx.x == 0 && blockIdx.y == 0) *guard.skip = s_end;
    }
    __syncthreads();
    if (s_end) return;
  }
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int j = j0 + threadIdx.x;
  // e_j from the bits of max_i |R_ij| (a non-negative double): frexp's exponent, or 0
  // when the maximum is 0 or not finite
  int e = 0;
  if (j < m) {
    const unsigned long long mb = colmax[j];
    const int E = (int)(mb >> 52);  // 2048 and up: the sign bit is set
    if (mb != 0ull && E < 2047) e = E >= 1 ? E - 1022 : (63 - __clzll((long long)mb)) - 1073;
  }
  const double sc = ldexp(1.0, -e);
  if (blockIdx.y == 0 && j < mp) colscale[j] = ldexpf(1.f, e);
  for (int r = threadIdx.y; r < 32; r += 8) {  // warp-uniform: threadIdx.y is the warp
    const int i = i0 + r;
    const bool in = i < n && j < m;
    const double x = in ? R[(int64_t)i * ld + j] : 0.0;
    bool ok = true;
    float v = in ? scaled_bits(x, e, ok) : 0.f;
    if (__any_sync(0xffffffffu, !ok)) {  // fp64, for the lanes that need it
      if (!ok) v = (float)(x * sc);
    }
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int jj = j0 + r, ii = i0 + threadIdx.x;
    if (jj < mp && ii < np) Rt[(int64_t)jj * np + ii] = to16<T16>(tile[threadIdx.x][r]);
  }
}

inline int grid_for(int64_t total, int sm) {
  int64_t b = (total + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sm * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// ------------------------------------------------------------------ solver object
struct Layout {
  int n, m, np, mp;
  int splits;  // room for this many K splits of the residual GEMM (0: none)
};

// Most K splits of the refinement residual GEMM (used when its tiles leave SMs idle).
constexpr int kMaxResidualSplits = 4;

struct Buffers {
  void* A16;      // np x np
  void* X16[2];   // np x np, Newton-Schulz iterates (ping-pong)
  void* Xt16;     // np x np, transpose of the current iterate
  void* Zt16;     // np x np, (2I - A X)^T
  void* Rt16;     // mp x np, scaled transposed right-hand side / residual
  float* colscale;               // mp
  unsigned long long* colmax;    // mp
  __nv_bfloat16* Aext;           // np x 6np
  __nv_bfloat16* Bext;           // mp x 6np
  double* R0;   // right-hand side (ld = mp)
  double* X;    // solution (ld = mp)
  double* R;    // residual (ld = mp)
  double* vec;  // [2][np] per-row scratch (row sums, diagonal scalings)
  unsigned long long* red;  // [4] max|R|, max|X|, ||E||_inf, ||E||_1 bits (context status words, see Solver)
  double* split;  // [splits][np][mp] partial sums of a split residual GEMM (or null)
};

template <class Take>
void plan(const Layout& L, Take&& t) {
  for (int k = 0; k < 5; ++k) t.template take<uint16_t>((size_t)L.np * L.np);  // A16, X16 x2, Xt16, Zt16
  t.template take<uint16_t>((size_t)L.mp * L.np);                 // Rt16
  t.template take<float>((size_t)L.mp);                           // colscale
  t.template take<unsigned long long>((size_t)L.mp);              // colmax
  t.template take<__nv_bfloat16>((size_t)L.np * kSlices * L.np);  // Aext
  t.template take<__nv_bfloat16>((size_t)L.mp * kSlices * L.np);  // Bext
  t.template take<double>((size_t)L.np * L.mp);                   // R0
  t.template take<double>((size_t)L.np * L.mp);                   // X
  t.template take<double>((size_t)L.np * L.mp);                   // R
  t.template take<double>((size_t)2 * L.np);                      // vec
  t.template take<double>((size_t)L.splits * L.np * L.mp);        // split
}

// The solver's status words in the context scratch (ints), laid out so that one copy
// returns everything a sweep's decision needs: [0] input error of the calling kernels,
// [1] non-finite solution or residual, [4] the GEMM wait time-out word, [5] the skip word
// of a speculatively launched correction (SweepGuard), [6..7] max|R|,
// [8..9] max|X|, [10..11] ||E||_inf and [12..13] ||E||_1 of the first Newton-Schulz
// iterate's E (doubles as bits).
constexpr int kStatus = 12;
static_assert(kStatus + 4 == tc::kGemmErrorSlot, "the GEMM error word sits in the status block");

struct Solver {
  rg_ctx* ctx;
  Layout L;
  Buffers b;
  bool bf16;
  cudaStream_t s;
  int* err;          // device status words (kStatus): [0] input error, [1] non-finite
  const char* input_error = "invalid input to the solver";  // what err[0] means for the caller
  const double* P;
  int64_t ldp;
  bool transP;
  int cur = 0;       // which X16 buffer holds the current inverse
  int ns_steps = 0;

  // Carves the solver's buffers out of the context workspace, after `extra_bytes`
  // reserved for the caller (returned in *extra).
  rg_status setup(int n, int m, bool use_bf16, cudaStream_t stream, size_t extra_bytes = 0, void** extra = nullptr) {
    L.n = n;
    L.m = m;
    L.np = (n + NB - 1) / NB * NB;
    L.mp = (m + NB - 1) / NB * NB;
    L.splits = tc::residual_splits(ctx, L.n, L.m, kSlices * L.np, kResidualChunk, kMaxResidualSplits) > 1
                   ? kMaxResidualSplits
                   : 0;
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
    b.A16 = cv.take<uint16_t>((size_t)L.np * L.np);
    b.X16[0] = cv.take<uint16_t>((size_t)L.np * L.np);
    b.X16[1] = cv.take<uint16_t>((size_t)L.np * L.np);
    b.Xt16 = cv.take<uint16_t>((size_t)L.np * L.np);
    b.Zt16 = cv.take<uint16_t>((size_t)L.np * L.np);
    b.Rt16 = cv.take<uint16_t>((size_t)L.mp * L.np);
    b.colscale = cv.take<float>(L.mp);
    b.colmax = cv.take<unsigned long long>(L.mp);
    b.Aext = cv.take<__nv_bfloat16>((size_t)L.np * kSlices * L.np);
    b.Bext = cv.take<__nv_bfloat16>((size_t)L.mp * kSlices * L.np);
    b.R0 = cv.take<double>((size_t)L.np * L.mp);
    b.X = cv.take<double>((size_t)L.np * L.mp);
    b.R = cv.take<double>((size_t)L.np * L.mp);
    b.vec = cv.take<double>((size_t)2 * L.np);
    b.split = L.splits ? cv.take<double>((size_t)L.splits * L.np * L.mp) : nullptr;
    err = ctx->d_scratch + kStatus;
    b.red = reinterpret_cast<unsigned long long*>(ctx->d_scratch + kStatus + 6);
    RG_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 6 * sizeof(int), s));  // error words and the GEMM's
    return RG_OK;
  }

  // P (shared by every set): its bf16 slices for the refinement product.
  rg_status set_matrix(const double* P_, int64_t ldp_, bool trans) {
    P = P_;
    ldp = ldp_;
    transP = trans;
    build_p_slices<<<grid_for((int64_t)L.np * L.np, ctx->sm_count), kThreads, 0, s>>>(P, ldp, transP, L.n, L.np,
                                                                                      b.Aext);
    RG_CUDA_TRY(ctx, cudaGetLastError());
    return RG_OK;
  }

  // Newton-Schulz approximate inverse of A = I - Dl P Dr into b.X16[cur].
  template <class T16>
  rg_status factor_t(const double* dl, const double* dr) {
    RG_CUDA_TRY(ctx, cudaMemsetAsync(b.red + 2, 0, 2 * sizeof(unsigned long long), s));
    T16* A16 = static_cast<T16*>(b.A16);
    T16* X[2] = {static_cast<T16*>(b.X16[0]), static_cast<T16*>(b.X16[1])};
    T16* Xt = static_cast<T16*>(b.Xt16);
    T16* Zt = static_cast<T16*>(b.Zt16);
    build_ns_start<T16><<<(L.np + 7) / 8, 256, 0, s>>>(P, ldp, transP, dl, dr, L.n, L.np, A16, X[0], Xt, b.red + 2,
                                                        b.colmax, L.mp);
    RG_CUDA_TRY(ctx, cudaGetLastError());
    // the status words and e0 in one pinned read-back: one wait on the stream
    int* hs = ctx->h_scratch;
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(hs + kStatus, err, 14 * sizeof(int), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hs[kStatus]) return rg::fail(ctx, RG_ERR_NUMERIC, "%s", input_error);
    double e_inf, e_one;
    memcpy(&e_inf, hs + kStatus + 10, sizeof(e_inf));
    memcpy(&e_one, hs + kStatus + 12, sizeof(e_one));
    if (!std::isfinite(e_inf) || !std::isfinite(e_one)) return rg::fail(ctx, RG_ERR_NUMERIC, "non-finite system matrix");
    // The residual of the Newton-Schulz iterate X_k is I - A X_k = E^(2^(k-1)), so any
    // norm of E with ||E|| < 1 bounds it. ||E||_inf (row sums) suits the Gebhart matrix
    // K = I - F diag(rho); its transpose, solved by the adjoint, has ||E||_1 < 1 instead
    // while its row sums (the column sums of F) can exceed 1: the smaller bound sets the
    // step count.
    const double e0 = std::min(e_inf, e_one);
    const double floor16 = bf16 ? 0x1p-10 : 0x1p-13;
    int steps = kMaxNewtonSchulz;
    if (e0 < 1.0) {
      steps = 1;
      if (e0 > 0.0) steps = (int)std::ceil(std::log2(std::log(floor16) / std::log(e0))) + 1;
      steps = std::max(1, std::min(steps, kMaxNewtonSchulz));
    }
    ns_steps = steps;
    cur = 0;
    for (int k = 1; k < steps; ++k) {  // step 1 was taken by build_ns_start
      // Zt = (2I - A X)^T : A operand A16 [i][k], B operand X^T rows = X columns
      rg_status st = tc::gemm(ctx, bf16, A16, L.np, Xt, L.np, L.np, L.np, L.np, tc::EpiTwoIMinusT<T16>{Zt, L.np}, s);
      if (st != RG_OK) return st;
      // X' = X (2I - A X) : A operand X [i][k], B operand Z^T
      st = tc::gemm(ctx, bf16, X[cur], L.np, Zt, L.np, L.np, L.np, L.np, tc::EpiStore16Both<T16>{X[cur ^ 1], Xt, L.np},
                    s);
      if (st != RG_OK) return st;
      cur ^= 1;
    }
    return RG_OK;
  }
  rg_status factor(const double* dl, const double* dr) {
    return bf16 ? factor_t<__nv_bfloat16>(dl, dr) : factor_t<__half>(dl, dr);
  }

  // X (+)= M src, where src is an fp64 n x m matrix (ld = mp): one tensor-core GEMM with
  // src scaled column by column into 16 bits. `have_colmax`: b.colmax already holds the
  // column maxima of src (the residual GEMM folds them in).
  template <class T16>
  rg_status apply_t(const double* src, bool first, bool have_colmax, const SweepGuard& guard) {
    if (!have_colmax) {  // colmax was zeroed by build_ns_start (apply(.., true) follows a factorisation)
      dim3 cg((L.m + 31) / 32, (L.n + 255) / 256);
      column_max<<<cg, dim3(32, 8), 0, s>>>(src, L.mp, L.n, L.m, b.colmax);
    }
    dim3 tg(L.mp / 32, L.np / 32);
    T16* Rt = static_cast<T16*>(b.Rt16);
    scaled_transpose16<T16><<<tg, dim3(32, 8), 0, s>>>(src, L.mp, L.n, L.m, L.np, L.mp, b.colmax, Rt, b.colscale,
                                                        guard);
    RG_CUDA_TRY(ctx, cudaGetLastError());
    return tc::gemm(ctx, bf16, b.X16[cur], L.np, Rt, L.np, L.n, L.m, L.np,
                    tc::EpiAddF64{b.X, L.mp, b.colscale, first ? 1 : 0}, s, guard.status ? guard.skip : nullptr);
  }
  rg_status apply(const double* src, bool first, bool have_colmax = false, const SweepGuard& guard = SweepGuard{}) {
    return bf16 ? apply_t<__nv_bfloat16>(src, first, have_colmax, guard)
                : apply_t<__half>(src, first, have_colmax, guard);
  }

  // R = R0 - X + Dl (P (Dr X)) from the first `pairs` slice pairs (3: 16-bit operands,
  // 6: 24-bit), and the copy of max|R|, max|X| and the error words to the pinned scratch,
  // after which ctx->ev_read is recorded (read_residual waits for it).
  rg_status launch_residual(const double* dl, const double* dr, int pairs) {
    dim3 tg((L.mp + 31) / 32, (L.np + 31) / 32);
    // also zeroes max|R|, max|X| and the column maxima that the residual GEMM folds
    build_x_slices<<<tg, dim3(32, 8), 0, s>>>(b.X, L.mp, dr, L.n, L.m, L.np, L.mp, b.Bext, b.red, b.colmax);
    RG_CUDA_TRY(ctx, cudaGetLastError());
    // max|R|, max|X|, the column maxima of R and the non-finite flag come from the epilogue
    rg_status st = tc::gemm_residual(ctx, b.Aext, (int64_t)kSlices * L.np, b.Bext, (int64_t)kSlices * L.np, L.n, L.m,
                                     pairs * L.np, kResidualChunk, b.R, b.R0, b.X, dl, L.mp, s, b.red, b.colmax,
                                     err + 1, b.split, L.splits, L.np / tc::BK, kResidualTailChunk, L.n);
    if (st != RG_OK) return st;
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch + kStatus, err, 10 * sizeof(int), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_read, s));
    return RG_OK;
  }

  // Waits for the read-back of launch_residual (not for later launches); max|R| / max|X|.
  rg_status read_residual(double* rel) {
    RG_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev_read));
    const int* hs = ctx->h_scratch + kStatus;
    double r, x;
    memcpy(&r, hs + 6, 8);
    memcpy(&x, hs + 8, 8);
    *rel = x > 0 ? r / x : r;
    return status_of(hs);
  }

  rg_status status_of(const int* w) {
    if (w[4]) return rg::fail(ctx, RG_ERR_CUDA, "tensor-core GEMM timed out waiting on a barrier");
    if (w[0]) return rg::fail(ctx, RG_ERR_NUMERIC, "%s", input_error);
    if (w[1]) return rg::fail(ctx, RG_ERR_NUMERIC, "non-finite value in the solution or residual");
    return RG_OK;
  }

  rg_status check_errors() {
    int* hs = ctx->h_scratch;
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(hs + kStatus, err, 6 * sizeof(int), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return status_of(hs + kStatus);
  }

  // Factor, solve and refine one set whose right-hand side is already in b.R0.
  rg_status run(const double* dl, const double* dr, double tol, int max_sweeps, int* sweeps, double* rel_out) {
    rg_status st = factor(dl, dr);
    if (st == RG_OK) st = apply(b.R0, true);
    if (st != RG_OK) return st;
    double rel = INFINITY, prev = INFINITY;
    int sw = 0;
    bool done = false;
    for (; sw < max_sweeps; ++sw) {
      // while the residual is large, the three leading slice pairs (16-bit operands,
      // error ~2^-16 max|X|) resolve it; those sweeps correct but never stop
      const bool coarse = prev > kCoarseAbove && tol < kCoarseAbove;
      st = launch_residual(dl, dr, coarse ? 3 : kSlices);
      if (st != RG_OK) return st;
      // the correction goes in behind the residual before the host has read it, so the GPU
      // works while the read-back travels; it evaluates the stopping rule below on the
      // device and does nothing when this sweep ends the refinement (X then stays as the
      // residual saw it, as if it had not been launched)
      SweepGuard g;
      g.status = err;
      g.tol = tol;
      g.prev = prev;
      g.coarse = coarse ? 1 : 0;
      g.skip = err + 5;
      st = apply(b.R, false, true, g);
      if (st != RG_OK) return st;
      st = read_residual(&rel);
      if (st != RG_OK) return st;
      // converged, or stalled at the accuracy floor of the fp32-chunked residual product
      if (!coarse && (rel <= tol || (rel <= kStallFloor && rel > 0.5 * prev))) { done = true; break; }
      prev = rel;
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

// dL/deps_j = sum_i Lam_ij F_ij (j < n). Block (32 x 8) per 32 columns: thread (x, y)
// sums rows y, y + 8, ... of column 32 b + x (coalesced along x), then the eight partial
// sums are added in a fixed order.
__global__ void grad_eps(const double* __restrict__ Lam, int64_t ldl, const double* __restrict__ F, int n,
                         double* __restrict__ deps) {
  __shared__ double part[8][33];
  const int j = blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (j < n)
    for (int i = threadIdx.y; i < n; i += 8) s += Lam[(int64_t)i * ldl + j] * F[(int64_t)i * (n + 1) + j];
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && j < n) {
    for (int y = 1; y < 8; ++y) s += part[y][threadIdx.x];
    deps[j] = s;
  }
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
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, negs, sizeof(int), cudaMemcpyDeviceToHost, s));  // pinned
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const int h = ctx->h_scratch[0];
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

rg_status rg_refinement_slices(rg_ctx* ctx, int64_t n, const double* x_d, uint16_t* slices_d, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n >= 0 && (n == 0 || (x_d && slices_d)), "rg_refinement_slices: bad argument");
  if (n == 0) return RG_OK;
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)ctx->sm_count * 8);
  split_slices<<<(int)blocks, 256, 0, s>>>(x_d, n, reinterpret_cast<__nv_bfloat16*>(slices_d));
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
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
    grad_eps<<<(n + 31) / 32, dim3(32, 8), 0, s>>>(sv.b.X, sv.L.mp, F_d, n, deps_d + (size_t)set * n);
    ++ctx->launches;
    // Q = F^T Lam (fp64-accurate sliced product), then drho_k = sum_j B_kj Q_kj
    dim3 tg((sv.L.mp + 31) / 32, (sv.L.np + 31) / 32);
    build_x_slices<<<tg, dim3(32, 8), 0, s>>>(sv.b.X, sv.L.mp, nullptr, n, n + 1, sv.L.np, sv.L.mp, sv.b.Bext);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    st = tc::gemm_residual(ctx, sv.b.Aext, (int64_t)kSlices * sv.L.np, sv.b.Bext, (int64_t)kSlices * sv.L.np, n,
                           n + 1, kSlices * sv.L.np, kResidualChunk, sv.b.R, nullptr, nullptr, nullptr, sv.L.mp, s,
                           nullptr, nullptr, nullptr, sv.b.split, sv.L.splits, sv.L.np / tc::BK, kResidualTailChunk,
                           n);
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
  sv.input_error = "rg_temperatures: a face with no radiative exchange, sigma eps A <= 0, or a non-positive T^4";
  balance_setup<<<(n + 7) / 8, 256, 0, s>>>(B_d, eps_d, area_d, Q_d, u_sink, sigma, n, sv.L.mp, t, dl, sv.b.R0,
                                             sv.err);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  // err[0] of balance_setup comes back with the factorisation's read-back
  int sw = 0;
  double rel = 0.0;
  st = sv.run(dl, nullptr, tol, 16, &sw, &rel);
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
  sv.input_error = "rg_temperatures_adjoint: a face with no radiative exchange or sigma eps A <= 0";
  balance_setup<<<(n + 7) / 8, 256, 0, s>>>(B_d, eps_d, area_d, eps_d, u_sink, sigma, n, sv.L.mp, t, dl, nullptr,
                                             sv.err);
  ++ctx->launches;
  balance_adj_rhs<<<(n + 127) / 128, 128, 0, s>>>(T_d, dT_d, t, n, sv.L.mp, sv.b.R0);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  // err[0] of balance_setup comes back with the factorisation's read-back
  int sw = 0;
  double rel = 0.0;
  st = sv.run(dl, nullptr, tol, 16, &sw, &rel);
  if (st == RG_OK) {
    balance_adj_out<<<(n + 7) / 8, 256, 0, s>>>(B_d, eps_d, T_d, sv.b.X, sv.L.mp, u_sink, n, dB_d, deps_d);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    st = sv.check_errors();
  }
  return st;
}

}  // extern "C"
