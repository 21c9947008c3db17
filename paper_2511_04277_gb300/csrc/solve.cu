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
//   2. Approximate inverse M by Newton-Schulz iteration X <- X (2I - A X) from X = I: the
//      error I - A X squares every step (its inf-norm starts at e0 < 1), so
//      ceil(log2(log(tol16) / log(e0))) + 1 steps reach the 16-bit floor. Each step is two
//      tcgen05 GEMMs whose epilogues write the 16-bit operands of the next one (the
//      transposed copies the K-major layout needs included).
//   3. Refinement with an exactly tracked residual. P' = P Dr is split once into five
//      fixed-point slices per row, P'_ik = 2^(e_i - 7) sum_a s_a,ik 2^(-8a) with integers
//      |s_a| <= 128 (40 bits below the row maximum). Starting from R = R0, X = 0, every
//      sweep takes the correction D = M R (one tensor-core GEMM), rounds each column of D to
//      one 8-bit fixed-point slice (integers |d| <= 127 times 2^(f_j - 7)), adds it to X
//      exactly and updates R <- R - D + Dl (P' D). The product P' D is a sum of integer
//      products; every 1,024-long chunk of it is exact in the fp32 tensor-core accumulator and
//      the chunks are added as integers, so the only error of the update is the truncation
//      of P' to the levels used (L levels: 2^-(8L-1) of |P'| |D|, L chosen per sweep from
//      max|D| / max|X| so that it stays below 2^-38 of |P'| |X|). The residual is thus known
//      to ~1e-12 whatever the tensor cores' rounding, and the refinement converges to the
//      fp64 solution instead of a biased one. It stops when max|R| <= tol max|X| (or stalls
//      below 1e-8).
// The transposed systems reuse the same code with P read transposed; the REF adjoint also
// accumulates sum_k P' D_k = F^T Lambda, the product its rho gradient needs.
#include <cmath>
#include <utility>

#include "tc_gemm.cuh"

namespace {

constexpr int NB = 128;          // panel width == GEMM tile height
constexpr int kThreads = 256;
// Below this relative residual a sweep that no longer halves it ends the refinement.
constexpr double kStallFloor = 1e-8;
constexpr int kMaxNewtonSchulz = 24;
// Fixed-point levels of P' (8 bits each) and the resolution the level count of a sweep
// keeps: the levels dropped from P' D stay below 2^-kLevelBits of max|P'| max|X|.
constexpr int kLevels = 5;
constexpr int kLevelBits = 38;
// Most K splits of the exact product (used when its tiles leave SMs idle).
constexpr int kMaxExactSplits = 4;
// K splits the workspace makes room for: a product whose level planes are small has few
// tiles and may split; a large one has tiles for every SM and never does (its int32 level
// sums then take one set of planes, not four).
inline int exact_splits(int n, int m) {
  return tc::exact_plane(n, m) * (int64_t)sizeof(int32_t) <= (64ll << 20) ? kMaxExactSplits : 1;
}

template <class T>
__device__ __forceinline__ T to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }

// ------------------------------------------------------------------ exact refinement kernels
// x 2^k (exact unless the result leaves the normal range).
__device__ __forceinline__ double scale2(double x, int k) {
  if (k >= -1022 && k <= 1023) return x * __longlong_as_double((long long)(k + 1023) << 52);
  return ldexp(x, k);
}

// int_scale2 for results outside the normal range, out of line so that its fp64 arithmetic
// stays off the common path.
__device__ __noinline__ double int_scale2_outside(long long q, int k) { return scale2((double)q, k); }

// q 2^k for an integer q (|q| < 2^63), rounded to nearest, ties to even, when q needs more
// than 53 bits: the same double as scale2((double)q, k), formed with integer operations
// (GB300 runs fp64 arithmetic and conversions on a pipe far slower than its integer ALU).
__device__ __forceinline__ double int_scale2(long long q, int k) {
  if (q == 0) return 0.0;
  const unsigned long long sgn = q < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long a = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
  const int lz = __clzll((long long)a);
  int e = 63 - lz + k;                       // exponent of the leading bit
  const unsigned long long m = a << lz;      // leading bit at 63
  unsigned long long mant = m >> 11;         // 53 bits
  const unsigned long long rem = m & 0x7ffull;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++e;
    }
  }
  if (e < -1022 || e > 1023) return int_scale2_outside(q, k);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 1023) << 52) | (mant & 0xfffffffffffffull)));
}

// Levels of P' that a sweep uses: the dropped ones stay below 2^-kLevelBits of
// max|P'| max|X|, with max|X| and max|D| in red[1] and red[2] (the sweep's status words).
__device__ __forceinline__ int exact_levels(const unsigned long long* red) {
  return tc::exact_level_count(red, kLevelBits, kLevels);
}

// round(x 2^s) to the nearest integer, ties to even, for |x 2^s| < 2^62, on the bit pattern of x
// (the value llrint(ldexp(x, s)) gives, without the fp64 pipe).
__device__ __forceinline__ long long round_scaled(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0) return 0;  // zero or subnormal: |x 2^s| < 2^-1022 2^s, below 1/2 here
  const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;  // 53-bit significand
  const int sh = E - 1075 + s;  // x 2^s = m 2^sh
  long long q;
  if (sh >= 0) {
    q = (long long)(m << sh);
  } else if (sh <= -54) {
    q = 0;  // below 1/2
  } else {
    const int r = -sh;
    const unsigned long long keep = m >> r, rem = m & ((1ull << r) - 1ull), half = 1ull << (r - 1);
    q = (long long)(keep + ((rem > half || (rem == half && (keep & 1ull))) ? 1ull : 0ull));
  }
  return (b >> 63) ? -q : q;
}

// bf16 bit pattern of an integer |d| <= 255 (exact): the float is formed by the magic-number
// subtraction (fp32, exact) and its upper half is the bf16 value.
__device__ __forceinline__ uint32_t bf16_bits_of_int(int d) {
  return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
}

// frexp's exponent of the double whose bit pattern (sign cleared) is b > 0, finite.
__device__ __forceinline__ int frexp_exponent_bits(unsigned long long b) {
  const int E = (int)(b >> 52);
  return E >= 1 ? E - 1022 : (63 - __clzll((long long)b)) - 1073;
}

// The split of one entry: q = round(x 2^s) (to nearest, ties to even) and its balanced
// base-256 digits s_0 .. s_4 (q = sum_a s_a 256^(4 - a)) as bf16 bit patterns.
__device__ __forceinline__ void split_digits(double x, int s, bool nonzero, uint32_t (&dbits)[kLevels]) {
  long long q = nonzero ? round_scaled(x, s) : 0;
#pragma unroll
  for (int a = kLevels - 1; a > 0; --a) {
    const int d = (int)((q + 128) & 255) - 128;
    dbits[a] = bf16_bits_of_int(d);
    q = (q - d) >> 8;
  }
  dbits[0] = bf16_bits_of_int((int)q);
}

// Block flags of the slices for the exact product (tc::ExactArgs): flags[(a rows + i / 256)
// ld + kb] = 1 when slice a has a non-zero digit in rows [256 (i / 256), + 256) and columns
// [64 kb, 64 kb + 64); the buffer is zeroed before the split. `bits` has bit a set for each
// level with a non-zero digit in the caller's block.
struct SliceFlags {
  uint8_t* f = nullptr;
  int rows = 0, ld = 0;
};
inline SliceFlags slice_flags(uint8_t* f, int np) {
  return SliceFlags{f, (np + 255) / 256, ((np / 64) + 15) / 16 * 16};
}
inline size_t slice_flag_bytes(int np) {
  const SliceFlags g = slice_flags(nullptr, np);
  return (size_t)kLevels * g.rows * g.ld;
}
__device__ __forceinline__ void mark_blocks(const SliceFlags& g, int i, int kb, unsigned bits) {
#pragma unroll
  for (int a = 0; a < kLevels; ++a)
    if (bits >> a & 1u) g.f[((int64_t)a * g.rows + i / 256) * g.ld + kb] = 1;
}
__device__ __forceinline__ unsigned nonzero_levels(const uint32_t (&d0)[kLevels], const uint32_t (&d1)[kLevels]) {
  unsigned bits = 0u;
#pragma unroll
  for (int a = 0; a < kLevels; ++a) bits |= ((d0[a] | d1[a]) != 0u) ? (1u << a) : 0u;
  return bits;
}

// Fixed-point split of P' = P Dr (Dr may be null) into kLevels slices per row: with e_i the
// exponent of max_k |P'_ik| and q = round(P'_ik 2^(39 - e_i)) (|q| < 2^39, to nearest, ties
// to even), the slices are q's balanced base-256 digits, q = sum_a s_a 256^(4 - a) with
// s_1..s_4 in [-128, 127] and |s_0| <= 128, so that P'_ik = 2^(e_i - 7) sum_a s_a 2^(-8a)
// up to 2^(e_i - 40). Aex[i][a np + k] = s_a (exact in bf16), zero in the padding;
// rowexp[i] = e_i (0 for a zero row). A non-finite entry raises *err. One warp per row, two
// adjacent columns per lane (the slices written as bf16 pairs); the row maximum is taken on
// the bit patterns and the only fp64 arithmetic is the product with Dr (GB300's fp64 pipe is
// narrow).
__global__ void build_p_exact(const double* __restrict__ P, int64_t ldp, const double* __restrict__ dr, int n,
                              int np, __nv_bfloat16* __restrict__ Aex, int* __restrict__ rowexp, int* err,
                              SliceFlags flags) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= np) return;
  uint32_t* row = reinterpret_cast<uint32_t*>(Aex + (int64_t)i * kLevels * np);  // bf16 pairs
  const int half = np / 2;
  if (i >= n) {
    for (int k2 = lane; k2 < half; k2 += 32)
#pragma unroll
      for (int a = 0; a < kLevels; ++a) row[(int64_t)a * half + k2] = 0u;
    if (lane == 0) rowexp[i] = 0;
    return;
  }
  const double* prow = P + (int64_t)i * ldp;
  unsigned long long mx = 0ull;
  bool bad = false;
  for (int k = lane; k < n; k += 32) {
    const double x = dr ? prow[k] * dr[k] : prow[k];
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    bad |= bx >= 0x7ff0000000000000ull;
    mx = max(mx, bx);
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) atomicExch(err, 1);
    mx = 0ull;  // the slices are not used once the error is raised
  }
  const int e = mx ? frexp_exponent_bits(mx) : 0;
  for (int k2 = lane; k2 < half; k2 += 32) {
    const int k = 2 * k2;
    uint32_t d0[kLevels], d1[kLevels];
    split_digits(k < n ? (dr ? prow[k] * dr[k] : prow[k]) : 0.0, 39 - e, k < n && mx, d0);
    split_digits(k + 1 < n ? (dr ? prow[k + 1] * dr[k + 1] : prow[k + 1]) : 0.0, 39 - e, k + 1 < n && mx, d1);
#pragma unroll
    for (int a = 0; a < kLevels; ++a) row[(int64_t)a * half + k2] = d0[a] | (d1[a] << 16);
    if (flags.f) {  // the warp's 64 columns are K block k2 / 32 (half is a multiple of 32)
      const unsigned bits = __reduce_or_sync(0xffffffffu, nonzero_levels(d0, d1));
      if (lane == 0 && bits) mark_blocks(flags, i, k2 / 32, bits);
    }
  }
  if (lane == 0) rowexp[i] = e;
}

// build_p_exact with the row in shared memory (n <= kRowSmem): one block of 512 threads per
// row of P', which is read from HBM once (the warp-per-row form reads it twice, the second
// time from HBM again when thousands of rows are in flight).
constexpr int kRowSmem = 12288;
__global__ void __launch_bounds__(512) build_p_exact_row(const double* __restrict__ P, int64_t ldp,
                                                         const double* __restrict__ dr, int n, int np,
                                                         __nv_bfloat16* __restrict__ Aex, int* __restrict__ rowexp,
                                                         int* err, SliceFlags flags) {
  extern __shared__ double xs[];  // [n]: the row of P'
  __shared__ unsigned long long s_mx[16];
  const int i = blockIdx.x, t = threadIdx.x;
  uint32_t* row = reinterpret_cast<uint32_t*>(Aex + (int64_t)i * kLevels * np);  // bf16 pairs
  const int half = np / 2;
  if (i >= n) {  // uniform over the block
    for (int k2 = t; k2 < half; k2 += 512)
#pragma unroll
      for (int a = 0; a < kLevels; ++a) row[(int64_t)a * half + k2] = 0u;
    if (t == 0) rowexp[i] = 0;
    return;
  }
  const double* prow = P + (int64_t)i * ldp;
  unsigned long long mx = 0ull;
  bool bad = false;
  for (int k0 = t; k0 < n; k0 += 4 * 512) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + 512 * u;
      v[u] = k < n ? (dr ? prow[k] * dr[k] : prow[k]) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + 512 * u;
      if (k < n) {
        xs[k] = v[u];
        const unsigned long long bx = (unsigned long long)__double_as_longlong(v[u]) & 0x7fffffffffffffffull;
        bad |= bx >= 0x7ff0000000000000ull;
        mx = max(mx, bx);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) s_mx[t >> 5] = mx;
  if (__syncthreads_or(bad)) {
    if (t == 0) atomicExch(err, 1);
    for (int w = 0; w < 16; ++w) s_mx[w] = 0ull;  // every thread writes the same: no race on the value
  }
  __syncthreads();
  unsigned long long m = s_mx[0];
#pragma unroll
  for (int w = 1; w < 16; ++w) m = max(m, s_mx[w]);
  const int e = m ? frexp_exponent_bits(m) : 0;
  for (int k2 = t; k2 < half; k2 += 512) {
    const int k = 2 * k2;
    uint32_t d0[kLevels], d1[kLevels];
    split_digits(k < n ? xs[k] : 0.0, 39 - e, k < n && m, d0);
    split_digits(k + 1 < n ? xs[k + 1] : 0.0, 39 - e, k + 1 < n && m, d1);
#pragma unroll
    for (int a = 0; a < kLevels; ++a) row[(int64_t)a * half + k2] = d0[a] | (d1[a] << 16);
    if (flags.f) {  // the warp's 64 columns are K block k2 / 32 (half is a multiple of 32)
      const unsigned bits = __reduce_or_sync(0xffffffffu, nonzero_levels(d0, d1));
      if ((t & 31) == 0 && bits) mark_blocks(flags, i, k2 / 32, bits);
    }
  }
  if (t == 0) rowexp[i] = e;
}

// Row maxima of P' for P read transposed (P'_ik = P_ki Dr_k), from P's rows (coalesced): block
// (32 x 8) per 32 columns i of P and 256 of its rows k, the bit patterns of |P'_ik| folded into
// colmax[i] by atomicMax (zeroed by the caller); a non-finite entry raises *err.
__global__ void __launch_bounds__(256) p_colmax_t(const double* __restrict__ P, int64_t ldp,
                                                  const double* __restrict__ dr, int n,
                                                  unsigned long long* __restrict__ colmax, int* err) {
  __shared__ unsigned long long s_mx[8][32];
  const int x = threadIdx.x, y = threadIdx.y;
  const int i = blockIdx.x * 32 + x;
  const int k0 = blockIdx.y * 256;
  unsigned long long mx = 0ull;
  bool bad = false;
  if (i < n) {
#pragma unroll
    for (int j0 = 0; j0 < 32; j0 += 8) {
      double v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int k = k0 + y + 8 * (j0 + r);
        v[r] = k < n ? P[(int64_t)k * ldp + i] : 0.0;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int k = k0 + y + 8 * (j0 + r);
        const double xv = (dr && k < n) ? v[r] * dr[k] : v[r];
        const unsigned long long bx = (unsigned long long)__double_as_longlong(xv) & 0x7fffffffffffffffull;
        const bool fin = bx < 0x7ff0000000000000ull;
        bad |= !fin;
        mx = max(mx, fin ? bx : 0ull);
      }
    }
  }
  s_mx[y][x] = mx;
  if (__syncthreads_or(bad) && x == 0 && y == 0) atomicExch(err, 1);
  if (y == 0 && i < n) {
    unsigned long long m = s_mx[0][x];
#pragma unroll
    for (int yy = 1; yy < 8; ++yy) m = max(m, s_mx[yy][x]);
    if (m) atomicMax(&colmax[i], m);
  }
}

// The transposed split's digits: block (32 x 8) per 32 rows i of P' and 64 columns k, the
// exponents from p_colmax_t's maxima; reads of P along its rows (coalesced), the digits
// through shared memory and written along k (64-byte rows per slice).
__global__ void __launch_bounds__(256) build_p_exact_t(const double* __restrict__ P, int64_t ldp,
                                                       const double* __restrict__ dr, int n, int np,
                                                       const unsigned long long* __restrict__ colmax,
                                                       __nv_bfloat16* __restrict__ Aex, int* __restrict__ rowexp,
                                                       SliceFlags flags) {
  __shared__ __align__(16) uint16_t tile[kLevels][32][66];  // [a][row of P'][column k]
  __shared__ unsigned s_bits;
  const int x = threadIdx.x, y = threadIdx.y;
  const int i0 = blockIdx.x * 32, i = i0 + x;
  const int k0 = blockIdx.y * 64;
  const unsigned long long m = i < n ? colmax[i] : 0ull;
  const int e = m ? frexp_exponent_bits(m) : 0;
  if (blockIdx.y == 0 && y == 0 && i < np) rowexp[i] = e;
  if (x == 0 && y == 0) s_bits = 0u;
  unsigned bits = 0u;
  double v[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int k = k0 + y + 8 * r;
    v[r] = (i < n && k < n) ? P[(int64_t)k * ldp + i] : 0.0;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int kl = y + 8 * r, k = k0 + kl;
    const bool in = i < n && k < n;
    const double xv = (dr && in) ? v[r] * dr[k] : v[r];
    uint32_t d[kLevels];
    split_digits(xv, 39 - e, in && m, d);
#pragma unroll
    for (int a = 0; a < kLevels; ++a) {
      tile[a][x][kl] = (uint16_t)d[a];
      bits |= d[a] ? (1u << a) : 0u;
    }
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  __syncthreads();  // s_bits is zeroed
  if (x == 0 && bits) atomicOr(&s_bits, bits);
  __syncthreads();
  // the block's 32 rows and 64 columns lie in one 256-row tile and K block (k0 = 64 blockIdx.y)
  if (flags.f && x == 0 && y == 0 && s_bits) mark_blocks(flags, i0, blockIdx.y, s_bits);
  // warp y writes rows i0 + y + 8 c, lane x the columns k0 + 2 x, k0 + 2 x + 1
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int il = y + 8 * c, ii = i0 + il;
    if (ii < np) {
      uint32_t* row = reinterpret_cast<uint32_t*>(Aex + (int64_t)ii * kLevels * np + k0);
#pragma unroll
      for (int a = 0; a < kLevels; ++a)
        row[(int64_t)a * (np / 2) + x] = *reinterpret_cast<const uint32_t*>(&tile[a][il][2 * x]);
    }
  }
}

// The fixed-point split of P' = P Dr (P^T Dr with trans) into Aex / rowexp (build_p_exact's
// definition): the transposed form as a column-maximum pass and a tiled digit pass (colmax:
// np words of scratch), the row form with the row in shared memory up to kRowSmem columns.
rg_status launch_build_p(rg_ctx* ctx, const double* P, int64_t ldp, bool trans, const double* dr, int n, int np,
                         __nv_bfloat16* Aex, int* rowexp, int* err, unsigned long long* colmax, cudaStream_t s,
                         uint8_t* flag_buf = nullptr) {
  const SliceFlags flags = slice_flags(flag_buf, np);
  if (flag_buf) RG_CUDA_TRY(ctx, cudaMemsetAsync(flag_buf, 0, slice_flag_bytes(np), s));
  if (trans) {
    RG_CUDA_TRY(ctx, cudaMemsetAsync(colmax, 0, (size_t)np * sizeof(unsigned long long), s));
    p_colmax_t<<<dim3((n + 31) / 32, (n + 255) / 256), dim3(32, 8), 0, s>>>(P, ldp, dr, n, colmax, err);
    build_p_exact_t<<<dim3(np / 32, np / 64), dim3(32, 8), 0, s>>>(P, ldp, dr, n, np, colmax, Aex, rowexp, flags);
    ctx->launches += 2;
  } else if (n <= kRowSmem) {
    static thread_local int configured_device = -1;
    if (configured_device != ctx->device) {
      RG_CUDA_TRY(ctx, cudaFuncSetAttribute(build_p_exact_row, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(kRowSmem * sizeof(double))));
      configured_device = ctx->device;
    }
    build_p_exact_row<<<np, 512, (size_t)n * sizeof(double), s>>>(P, ldp, dr, n, np, Aex, rowexp, err, flags);
    ++ctx->launches;
  } else {
    build_p_exact<<<(np + 7) / 8, 256, 0, s>>>(P, ldp, dr, n, np, Aex, rowexp, err, flags);
    ++ctx->launches;
  }
  RG_CUDA_TRY(ctx, cudaGetLastError());
  return RG_OK;
}

// Rounds each column j < m of the correction D (fp32, ld = mp) to one 8-bit fixed-point slice:
// f_j = the exponent of max_k |D_kj| (colmax, float bits), d = round(D_kj 2^(7 - f_j)) clamped to
// [-127, 127]. Writes Bq[j][k] = d (bf16, the exact product's B operand, zero in the padding),
// Dn[k][j] = d, dexp[j] = f_j and adds d 2^(f_j - 7) to X (first: X = that); folds max|X| into
// red[1], max_j colmax_j into red[2] (as doubles; both zeroed by the sweep's first kernel) and
// zeroes the column maxima of R for the residual that follows. Block (32 x 8) per 64 rows x 64
// columns, two columns per lane (8- and 16-byte loads), the transposed rows written as bf16
// pairs through shared memory; the one fp64 operation per entry is the addition to X.
__global__ void quantize_correction(const float* __restrict__ D, int n, int m, int np, int mp,
                                    const unsigned int* __restrict__ dcolmax, __nv_bfloat16* __restrict__ Bq,
                                    int16_t* __restrict__ Dn, int* __restrict__ dexp, double* __restrict__ X,
                                    int first, unsigned long long* red, unsigned long long* rcolmax, int* nonfinite,
                                    const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  __shared__ __align__(16) __nv_bfloat16 tile[64][66];  // [column][row]
  __shared__ unsigned long long s_xmax;
  if (threadIdx.x == 0 && threadIdx.y == 0) s_xmax = 0ull;
  const int k0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int jl = 2 * threadIdx.x, j = j0 + jl;  // this lane's columns j, j + 1
  int f[2];
  float sc[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const unsigned int cb = j + c < m ? dcolmax[j + c] : 0u;
    const bool cfin = cb < 0x7f800000u;
    f[c] = 0;
    if (cb != 0u && cfin) f[c] = (int)(cb >> 23) != 0 ? (int)(cb >> 23) - 126 : (31 - __clz((int)cb)) - 148;
    sc[c] = ldexpf(1.f, 7 - f[c]);
    if (blockIdx.y == 0 && threadIdx.y == 0) {
      if (j + c < mp) {
        dexp[j + c] = f[c];
        rcolmax[j + c] = 0ull;
      }
      if (j + c < m && cfin && cb) atomicMax(&red[2], (unsigned long long)__double_as_longlong((double)__uint_as_float(cb)));
      if (j + c < m && !cfin) atomicExch(nonfinite, 1);
    }
  }
  __syncthreads();
  unsigned long long xmax = 0ull;
  const bool c1 = j + 1 < m;
  if (j < m) {
#pragma unroll 4
    for (int r = 0; r < 8; ++r) {
      const int k = k0 + threadIdx.y + 8 * r;
      if (k >= n) break;
      const int64_t o = (int64_t)k * mp + j;
      const float2 dv = *reinterpret_cast<const float2*>(D + o);
      int q0 = __float2int_rn(dv.x * sc[0]), q1 = c1 ? __float2int_rn(dv.y * sc[1]) : 0;
      q0 = q0 > 127 ? 127 : (q0 < -127 ? -127 : q0);
      q1 = q1 > 127 ? 127 : (q1 < -127 ? -127 : q1);
      *reinterpret_cast<uint32_t*>(Dn + o) = (uint32_t)(uint16_t)(int16_t)q0 | ((uint32_t)(uint16_t)(int16_t)q1 << 16);
      double2 xv = first ? make_double2(0.0, 0.0) : *reinterpret_cast<const double2*>(X + o);
      if (!c1) xv.y = 0.0;  // column m is padding
      xv.x += int_scale2(q0, f[0] - 7);
      xv.y += int_scale2(q1, f[1] - 7);
      if (c1) {
        *reinterpret_cast<double2*>(X + o) = xv;
      } else {
        X[o] = xv.x;
      }
      xmax = max(xmax, (unsigned long long)__double_as_longlong(xv.x) & 0x7fffffffffffffffull);
      xmax = max(xmax, (unsigned long long)__double_as_longlong(xv.y) & 0x7fffffffffffffffull);
      tile[jl][threadIdx.y + 8 * r] = __float2bfloat16_rz((float)q0);
      tile[jl + 1][threadIdx.y + 8 * r] = __float2bfloat16_rz((float)q1);
    }
  }
  // rows k >= n and columns j >= m are zero in Bq
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int kl = threadIdx.y + 8 * r;
    if (j >= m || k0 + kl >= n) {
      tile[jl][kl] = __float2bfloat16_rz(0.f);
      tile[jl + 1][kl] = __float2bfloat16_rz(0.f);
    } else if (!c1) {
      tile[jl + 1][kl] = __float2bfloat16_rz(0.f);
    }
  }
  for (int o = 16; o > 0; o >>= 1) xmax = max(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  if (threadIdx.x == 0 && xmax) atomicMax(&s_xmax, xmax);
  __syncthreads();
  // warp w writes columns j0 + w + 8 c, lane l the rows k0 + 2 l, k0 + 2 l + 1
  const int kk = k0 + 2 * threadIdx.x;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cl = threadIdx.y + 8 * c, jj = j0 + cl;
    if (jj < mp && kk < np)
      *reinterpret_cast<uint32_t*>(Bq + (int64_t)jj * np + kk) = *reinterpret_cast<const uint32_t*>(&tile[cl][2 * threadIdx.x]);
  }
  if (threadIdx.x == 0 && threadIdx.y == 0 && s_xmax) atomicMax(&red[1], s_xmax);
}

// The residual update after the exact product: with S = P' D assembled from the integer level
// sums (T = sum_z sum_a lev[z][a] 256^(L - 1 - a), S_ij = T 2^(e_i + f_j - 14 - 8(L - 1))),
//   R_ij <- (first ? R0_ij : R_ij) - D_ij + dl_i S_ij,   D_ij = Dn_ij 2^(f_j - 7),
// and, with Q, Q_ij <- (first ? 0 : Q_ij) + S_ij. Without dl and Q, S - D = (T - Dn 2^sh) 2^a
// with sh = 7 - e_i + 8(L - 1) is formed exactly in int64 (|T| < 2^61.01 and |Dn 2^sh| < 2^60
// for e_i >= -14, so the difference fits) and rounded once, leaving one fp64 addition per
// entry (GB300's fp64 pipe issues about 2 lanes per clock per SM). Folds max|R| into red[0],
// max_i |R_ij| into colmax[j] (as doubles) and raises *nonfinite on an inf or NaN.
// Block (32 x 8) per 128 columns x 128 rows: lane l owns the block's columns 4 l .. 4 l + 3
// (16-byte loads of the level sums, the residual and Dn), warp w the rows w, w + 8, ...
__global__ void __launch_bounds__(256, 3) finish_residual(
    const int32_t* __restrict__ lev, int64_t ldl, int64_t plane, int splits, const int* __restrict__ rowexp,
    const int* __restrict__ dexp, const int16_t* __restrict__ Dn, const double* __restrict__ dl, int n, int m, int mp,
    const double* __restrict__ R0, double* __restrict__ R, double* __restrict__ Q, int first, unsigned long long* red,
    unsigned long long* colmax, int* nonfinite, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  __shared__ unsigned long long s_col[8][128];
  const int L = exact_levels(red);
  const int jb = blockIdx.x * 128, j = jb + 4 * threadIdx.x;
  const int i0 = blockIdx.y * 128;
  const double* src = first ? R0 : R;
  const bool plain = !dl && !Q;
  unsigned long long cmax[4] = {0ull, 0ull, 0ull, 0ull};
  bool bad = false;
  if (j < m) {
    const int4 fv = *reinterpret_cast<const int4*>(dexp + j);  // dexp holds mp >= j + 4 entries
    const int f[4] = {fv.x, fv.y, fv.z, fv.w};
    const int nc = min(4, m - j);  // valid columns of this lane
#pragma unroll 1
    for (int i = i0 + threadIdx.y; i < min(n, i0 + 128); i += 8) {
      const int64_t o = (int64_t)i * ldl + j;
      long long T[4] = {0ll, 0ll, 0ll, 0ll};
      for (int z = 0; z < splits; ++z) {
        int4 lv[kLevels];
#pragma unroll
        for (int a = 0; a < kLevels; ++a)
          lv[a] = a < L ? *reinterpret_cast<const int4*>(lev + ((int64_t)z * kLevels + a) * plane + o)
                        : make_int4(0, 0, 0, 0);
        long long t[4] = {0ll, 0ll, 0ll, 0ll};
#pragma unroll
        for (int a = 0; a < kLevels; ++a)
          if (a < L) {
            t[0] = t[0] * 256 + lv[a].x;
            t[1] = t[1] * 256 + lv[a].y;
            t[2] = t[2] * 256 + lv[a].z;
            t[3] = t[3] * 256 + lv[a].w;
          }
#pragma unroll
        for (int c = 0; c < 4; ++c) T[c] += t[c];
      }
      const int64_t e = (int64_t)i * mp + j;
      const double2 s01 = *reinterpret_cast<const double2*>(src + e);
      const double2 s23 = *reinterpret_cast<const double2*>(src + e + 2);
      const uint2 dnv = *reinterpret_cast<const uint2*>(Dn + e);
      const double sv[4] = {s01.x, s01.y, s23.x, s23.y};
      const int dn[4] = {(int)(int16_t)(dnv.x & 0xffffu), (int)(int16_t)(dnv.x >> 16), (int)(int16_t)(dnv.y & 0xffffu),
                         (int)(int16_t)(dnv.y >> 16)};
      const int re = rowexp[i];
      const int sh = 7 - re + 8 * (L - 1);
      double r[4];
      if (plain && re >= -14 && sh >= 0) {  // warp-uniform: the warp shares row i
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const long long U = T[c] - (long long)((unsigned long long)(long long)dn[c] << sh);
          r[c] = sv[c] + int_scale2(U, re + f[c] - 14 - 8 * (L - 1));
        }
      } else {
        const double w = dl ? dl[i] : 1.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double S = int_scale2(T[c], re + f[c] - 14 - 8 * (L - 1));
          r[c] = (sv[c] - int_scale2(dn[c], f[c] - 7)) + w * S;
          if (Q && c < nc) Q[e + c] = (first ? 0.0 : Q[e + c]) + S;
        }
      }
      if (nc == 4) {
        *reinterpret_cast<double2*>(R + e) = make_double2(r[0], r[1]);
        *reinterpret_cast<double2*>(R + e + 2) = make_double2(r[2], r[3]);
      } else {
        for (int c = 0; c < nc; ++c) R[e + c] = r[c];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const unsigned long long rb = (unsigned long long)__double_as_longlong(r[c]) & 0x7fffffffffffffffull;
        const bool fin = rb < 0x7ff0000000000000ull;
        if (c < nc) {
          bad |= !fin;
          cmax[c] = max(cmax[c], fin ? rb : 0ull);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) s_col[threadIdx.y][4 * threadIdx.x + c] = cmax[c];
  if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicExch(nonfinite, 1);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid < 128) {  // warps 0 .. 3: one column each
    unsigned long long cm = s_col[0][tid];
#pragma unroll
    for (int y = 1; y < 8; ++y) cm = max(cm, s_col[y][tid]);
    if (jb + tid < m && cm) atomicMax(&colmax[jb + tid], cm);
    for (int o = 16; o > 0; o >>= 1) cm = max(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    if (threadIdx.x == 0 && cm) atomicMax(&red[0], cm);
  }
}

// finish_residual for an unsplit level product (splits == 1), the spacecraft-sized case:
// the same arithmetic, with each warp's rows brought into shared memory by cp.async
// kFinStages rows ahead of the one it computes, so that the bytes in flight per SM are not
// bounded by the registers that would hold them. Block (32 x 8) per 128 columns x
// kFinRows rows; warp w owns the rows w, w + 8, ...; lane l the columns 4 l .. 4 l + 3.
// A lane reads back only what it copied itself, so the stages need no barrier.
constexpr int kFinStages = 3;
constexpr int kFinRows = 256;
struct FinStage {
  int4 lev[kLevels][32];
  double2 src[2][32];
  uint2 dn[32];
};
constexpr size_t kFinSmem = (size_t)8 * kFinStages * sizeof(FinStage);

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}

__global__ void __launch_bounds__(256, 2) finish_residual_staged(
    const int32_t* __restrict__ lev, int64_t ldl, int64_t plane, const int* __restrict__ rowexp,
    const int* __restrict__ dexp, const int16_t* __restrict__ Dn, const double* __restrict__ dl, int n, int m, int mp,
    const double* __restrict__ R0, double* __restrict__ R, double* __restrict__ Q, int first, unsigned long long* red,
    unsigned long long* colmax, int* nonfinite, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  extern __shared__ __align__(16) unsigned char fin_smem[];
  __shared__ unsigned long long s_col[8][128];
  FinStage* stages = reinterpret_cast<FinStage*>(fin_smem) + threadIdx.y * kFinStages;
  const int L = exact_levels(red);
  const int lane = threadIdx.x;
  const int jb = blockIdx.x * 128, j = jb + 4 * lane;
  const int i0 = blockIdx.y * kFinRows + threadIdx.y;
  const int i_end = min(n, (int)(blockIdx.y + 1) * kFinRows);
  const int rows = i0 < i_end ? (i_end - i0 + 7) / 8 : 0;  // rows of this warp
  const double* src = first ? R0 : R;
  const bool plain = !dl && !Q;
  const bool live = j < m;
  // copies of the warp's k-th row into stage k % kFinStages (an empty group past the end,
  // so that every lane commits the same number of groups)
  auto issue = [&](int k) {
    if (k < rows && live) {
      FinStage& st = stages[k % kFinStages];
      const int i = i0 + 8 * k;
      const int64_t o = (int64_t)i * ldl + j, e = (int64_t)i * mp + j;
      for (int a = 0; a < L; ++a) cp_async16(&st.lev[a][lane], lev + a * plane + o);
      cp_async16(&st.src[0][lane], src + e);
      cp_async16(&st.src[1][lane], src + e + 2);
      cp_async8(&st.dn[lane], Dn + e);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  unsigned long long cmax[4] = {0ull, 0ull, 0ull, 0ull};
  bool bad = false;
  int f[4] = {0, 0, 0, 0};
  if (live) {
    const int4 fv = *reinterpret_cast<const int4*>(dexp + j);  // dexp holds mp >= j + 4 entries
    f[0] = fv.x;
    f[1] = fv.y;
    f[2] = fv.z;
    f[3] = fv.w;
  }
  const int nc = live ? min(4, m - j) : 0;  // valid columns of this lane
#pragma unroll
  for (int k = 0; k < kFinStages - 1; ++k) issue(k);
  for (int k = 0; k < rows; ++k) {
    issue(k + kFinStages - 1);
    asm volatile("cp.async.wait_group %0;" ::"n"(kFinStages - 1) : "memory");
    if (!live) continue;
    const FinStage& st = stages[k % kFinStages];
    const int i = i0 + 8 * k;
    long long T[4] = {0ll, 0ll, 0ll, 0ll};
#pragma unroll
    for (int a = 0; a < kLevels; ++a)
      if (a < L) {
        const int4 lv = st.lev[a][lane];
        T[0] = T[0] * 256 + lv.x;
        T[1] = T[1] * 256 + lv.y;
        T[2] = T[2] * 256 + lv.z;
        T[3] = T[3] * 256 + lv.w;
      }
    const double2 s01 = st.src[0][lane], s23 = st.src[1][lane];
    const uint2 dnv = st.dn[lane];
    const double sv[4] = {s01.x, s01.y, s23.x, s23.y};
    const int dn[4] = {(int)(int16_t)(dnv.x & 0xffffu), (int)(int16_t)(dnv.x >> 16), (int)(int16_t)(dnv.y & 0xffffu),
                       (int)(int16_t)(dnv.y >> 16)};
    const int re = rowexp[i];
    const int sh = 7 - re + 8 * (L - 1);
    const int64_t e = (int64_t)i * mp + j;
    double r[4];
    if (plain && re >= -14 && sh >= 0) {  // warp-uniform: the warp shares row i
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const long long U = T[c] - (long long)((unsigned long long)(long long)dn[c] << sh);
        r[c] = sv[c] + int_scale2(U, re + f[c] - 14 - 8 * (L - 1));
      }
    } else {
      const double w = dl ? dl[i] : 1.0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double S = int_scale2(T[c], re + f[c] - 14 - 8 * (L - 1));
        r[c] = (sv[c] - int_scale2(dn[c], f[c] - 7)) + w * S;
        if (Q && c < nc) Q[e + c] = (first ? 0.0 : Q[e + c]) + S;
      }
    }
    if (nc == 4) {
      *reinterpret_cast<double2*>(R + e) = make_double2(r[0], r[1]);
      *reinterpret_cast<double2*>(R + e + 2) = make_double2(r[2], r[3]);
    } else {
      for (int c = 0; c < nc; ++c) R[e + c] = r[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const unsigned long long rb = (unsigned long long)__double_as_longlong(r[c]) & 0x7fffffffffffffffull;
      const bool fin = rb < 0x7ff0000000000000ull;
      if (c < nc) {
        bad |= !fin;
        cmax[c] = max(cmax[c], fin ? rb : 0ull);
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 4; ++c) s_col[threadIdx.y][4 * lane + c] = cmax[c];
  if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicExch(nonfinite, 1);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid < 128) {  // warps 0 .. 3: one column each
    unsigned long long cm = s_col[0][tid];
#pragma unroll
    for (int y = 1; y < 8; ++y) cm = max(cm, s_col[y][tid]);
    if (jb + tid < m && cm) atomicMax(&colmax[jb + tid], cm);
    for (int o = 16; o > 0; o >>= 1) cm = max(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    if (threadIdx.x == 0 && cm) atomicMax(&red[0], cm);
  }
}

// ------------------------------------------------------------------ narrow systems
// quantize_correction and finish_residual for m <= kNarrow right-hand sides (the balance's one
// column, a factored cotangent's few): one thread per row and a loop over the columns, so
// that no lane idles on a column that does not exist; the same arithmetic and status words.
// The B operands' rows j >= m (Bq, Rt16) are left unwritten: the GEMMs read N = m rows.
constexpr int kNarrow = 8;

__global__ void __launch_bounds__(256) quantize_correction_narrow(
    const float* __restrict__ D, int n, int m, int np, int mp, const unsigned int* __restrict__ dcolmax,
    __nv_bfloat16* __restrict__ Bq, int16_t* __restrict__ Dn, int* __restrict__ dexp, double* __restrict__ X,
    int first, unsigned long long* red, unsigned long long* rcolmax, int* nonfinite, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  __shared__ unsigned long long s_xmax;
  if (threadIdx.x == 0) s_xmax = 0ull;
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x < mp) {
    rcolmax[threadIdx.x] = 0ull;
    if (threadIdx.x >= m) dexp[threadIdx.x] = 0;
  }
  unsigned long long xmax = 0ull;
#pragma unroll
  for (int j = 0; j < kNarrow; ++j) {
    if (j >= m) break;
    const unsigned int cb = dcolmax[j];
    const bool cfin = cb < 0x7f800000u;
    int f = 0;
    if (cb != 0u && cfin) f = (int)(cb >> 23) != 0 ? (int)(cb >> 23) - 126 : (31 - __clz((int)cb)) - 148;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      dexp[j] = f;
      if (cfin && cb) atomicMax(&red[2], (unsigned long long)__double_as_longlong((double)__uint_as_float(cb)));
      if (!cfin) atomicExch(nonfinite, 1);
    }
    int q = 0;
    if (k < n) {
      const int64_t o = (int64_t)k * mp + j;
      q = __float2int_rn(D[o] * ldexpf(1.f, 7 - f));
      q = q > 127 ? 127 : (q < -127 ? -127 : q);
      Dn[o] = (int16_t)q;
      const double v = (first ? 0.0 : X[o]) + int_scale2(q, f - 7);
      X[o] = v;
      xmax = max(xmax, (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull);
    }
    if (k < np) Bq[(int64_t)j * np + k] = __float2bfloat16_rz((float)q);
  }
  for (int o = 16; o > 0; o >>= 1) xmax = max(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && xmax) atomicMax(&s_xmax, xmax);
  __syncthreads();
  if (threadIdx.x == 0 && s_xmax) atomicMax(&red[1], s_xmax);
}

// The exact level product for m <= kNarrow right-hand sides, on the CUDA cores: a matrix-vector
// product is bound by reading the slices, which a tensor-core tile of 64 columns would read
// no faster. lev[a][i][j] = sum_k Aex[i][a np + k] Bq[j][k] for a < L (the level count from
// the sweep's words), the layout of gemm_exact with one split. Exact: lane l sums the np / 32
// products of its k (|s| <= 128, |d| <= 127, so |sum| <= 1,024 x 16,256 < 2^24 for np <= 32,768)
// in fp32, and the lanes' sums are added as int32. One warp per row i, eight k per 16-byte
// load and eight loads of the slices in flight per lane; bf16 widens to fp32 by a shift.
// M = m (1 .. kNarrow).
template <int M>
__global__ void __launch_bounds__(256) exact_gemv_narrow(const __nv_bfloat16* __restrict__ Aex,
                                                         const __nv_bfloat16* __restrict__ Bq, int n, int np,
                                                         int32_t* __restrict__ lev, int64_t ldl, int64_t plane,
                                                         const unsigned long long* red, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  constexpr int kU = 8;  // loads in flight per lane
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int L = exact_levels(red);
  const int groups = np / 8;  // uint4 groups of a row
  for (int a = 0; a < L; ++a) {
    const uint4* arow = reinterpret_cast<const uint4*>(Aex + ((int64_t)i * kLevels + a) * np);
    float acc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = 0.f;
    for (int g0 = lane; g0 < groups; g0 += 32 * kU) {
      uint4 av[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int g = g0 + 32 * u;
        av[u] = g < groups ? __ldcs(arow + g) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int g = g0 + 32 * u;
        if (g >= groups) break;
        const uint32_t aw[4] = {av[u].x, av[u].y, av[u].z, av[u].w};
#pragma unroll
        for (int j = 0; j < M; ++j) {
          const uint4 bv = reinterpret_cast<const uint4*>(Bq + (int64_t)j * np)[g];
          const uint32_t bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc[j] = fmaf(__uint_as_float(aw[q] << 16), __uint_as_float(bw[q] << 16), acc[j]);
            acc[j] = fmaf(__uint_as_float(aw[q] & 0xffff0000u), __uint_as_float(bw[q] & 0xffff0000u), acc[j]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
      int v = __float2int_rn(acc[j]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) lev[(int64_t)a * plane + (int64_t)i * ldl + j] = v;
    }
  }
}

__global__ void __launch_bounds__(256) finish_residual_narrow(
    const int32_t* __restrict__ lev, int64_t ldl, int64_t plane, int splits, const int* __restrict__ rowexp,
    const int* __restrict__ dexp, const int16_t* __restrict__ Dn, const double* __restrict__ dl, int n, int m, int mp,
    const double* __restrict__ R0, double* __restrict__ R, double* __restrict__ Q, int first, unsigned long long* red,
    unsigned long long* colmax, int* nonfinite, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  __shared__ unsigned long long s_col[8][kNarrow];
  const int L = exact_levels(red);
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* src = first ? R0 : R;
  unsigned long long cmax[kNarrow];
  bool bad = false;
  const int re = i < n ? rowexp[i] : 0;
  const int sh = 7 - re + 8 * (L - 1);
  const bool fast = !dl && !Q && re >= -14 && sh >= 0;
  const double w = (dl && i < n) ? dl[i] : 1.0;
#pragma unroll
  for (int j = 0; j < kNarrow; ++j) {
    cmax[j] = 0ull;
    if (j < m && i < n) {
      const int64_t o = (int64_t)i * ldl + j;
      long long T = 0;
      for (int z = 0; z < splits; ++z) {
        int32_t lv[kLevels];
#pragma unroll
        for (int a = 0; a < kLevels; ++a) lv[a] = a < L ? lev[((int64_t)z * kLevels + a) * plane + o] : 0;
        long long t = 0;
#pragma unroll
        for (int a = 0; a < kLevels; ++a)
          if (a < L) t = t * 256 + lv[a];
        T += t;
      }
      const int64_t e = (int64_t)i * mp + j;
      const int f = dexp[j], dn = Dn[e];
      const int ex = re + f - 14 - 8 * (L - 1);
      double r;
      if (fast) {
        r = src[e] + int_scale2(T - (long long)((unsigned long long)(long long)dn << sh), ex);
      } else {
        const double S = int_scale2(T, ex);
        r = (src[e] - int_scale2(dn, f - 7)) + w * S;
        if (Q) Q[e] = (first ? 0.0 : Q[e]) + S;
      }
      R[e] = r;
      const unsigned long long rb = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;
      const bool fin = rb < 0x7ff0000000000000ull;
      bad |= !fin;
      cmax[j] = fin ? rb : 0ull;
    }
  }
  unsigned long long all = 0ull;
#pragma unroll
  for (int j = 0; j < kNarrow; ++j) {
    unsigned long long c = cmax[j];
    for (int o = 16; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
    if (lane == 0) s_col[warp][j] = c;
    all = max(all, c);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(nonfinite, 1);
  if (threadIdx.x < kNarrow && threadIdx.x < m) {
    unsigned long long c = s_col[0][threadIdx.x];
#pragma unroll
    for (int y = 1; y < 8; ++y) c = max(c, s_col[y][threadIdx.x]);
    if (c) atomicMax(&colmax[threadIdx.x], c);
  }
  if (lane == 0 && all) atomicMax(&red[0], all);
}

// out[e] = (int16) of the integer-valued bf16 in[e] (rg_exact_split's output form).
__global__ void bf16_rows_to_int16(const __nv_bfloat16* __restrict__ in, int64_t total, int16_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (int16_t)__float2int_rz(__bfloat162float(in[e]));
}

// A16 = I - Dl P Dr (16-bit, identity padding), the first Newton-Schulz iterate
// X16 = 2I - A = I + Dl P Dr (the step from X = I, done here instead of by two GEMMs) and its
// transpose Xt16, with the row and column sums of |Dl P Dr| (in fp32) added into rowsum /
// colsum (zeroed by the caller); with gen, those of |P diag(gdr)| instead (gdr null: 1), the
// unscaled matrix whose residual the refinement sees when Dl P Dr is its symmetric form. One block (32 x 8) per 32 x 32 tile: P's tile is read coalesced in its own
// layout (directly or transposed) through shared memory, and Xt16's tile is written from a
// transposed copy.
template <class T16>
__global__ void build_ns_start(const double* __restrict__ P, int64_t ldp, bool trans, const double* __restrict__ dl,
                               const double* __restrict__ dr, int n, int np, T16* __restrict__ A16,
                               T16* __restrict__ X16, T16* __restrict__ Xt16, double* __restrict__ rowsum,
                               double* __restrict__ colsum, bool gen, const double* __restrict__ gdr,
                               uint8_t* __restrict__ aflags) {
  __shared__ double raw[32][33];
  __shared__ float xs[32][33];
  __shared__ float cpart[8][33];
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int r0 = trans ? k0 : i0, c0 = trans ? i0 : k0;  // tile origin in P's own layout
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int a = ty; a < 32; a += 8) {
    const int r = r0 + a, c = c0 + tx;
    raw[a][tx] = (r < n && c < n) ? P[(int64_t)r * ldp + c] : 0.0;
  }
  __syncthreads();
  // fp32 arithmetic from here: A16 and X16 are 16-bit, and the norms only set the step count
  // (GB300's fp64 pipe, conversions included, is far slower than its fp32 one)
  const int k = k0 + tx;
  const float rk = (k < n && dr) ? (float)dr[k] : 1.f;
  const float gk = (k < n && gdr) ? (float)gdr[k] : 1.f;
  float cs = 0.f;
  bool nonzero = false;  // a non-zero 16-bit entry of A in this 32 x 32 tile
  for (int a = ty; a < 32; a += 8) {
    const int i = i0 + a;
    const float p = (float)(trans ? raw[tx][a] : raw[a][tx]);
    float e = 0.f;
    if (i < n && k < n) e = (dl ? (float)dl[i] : 1.f) * p * rk;
    const float one = (i == k) ? 1.f : 0.f;
    const int64_t o = (int64_t)i * np + k;
    const T16 av = to16<T16>(one - e);
    A16[o] = av;
    nonzero |= (*reinterpret_cast<const uint16_t*>(&av) & 0x7fffu) != 0u;
    X16[o] = to16<T16>(one + e);
    xs[a][tx] = one + e;
    const float ae = gen ? ((i < n && k < n) ? fabsf(p * gk) : 0.f) : fabsf(e);
    cs += ae;
    float rs = ae;
    for (int q = 16; q > 0; q >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, q);
    if (tx == 0 && rs != 0.f) atomicAdd(&rowsum[i], (double)rs);
  }
  cpart[ty][tx] = cs;
  // the tile lies in one 256-row tile of A and one 64-wide K block (the pair GEMM's flags)
  if (__syncthreads_or(nonzero) && aflags && tx == 0 && ty == 0)
    aflags[(int64_t)(i0 / 256) * ((np / 64 + 31) / 32 * 32) + k0 / 64] = 1;
  if (ty == 0) {
    for (int y = 1; y < 8; ++y) cs += cpart[y][tx];
    if (cs != 0.f) atomicAdd(&colsum[k], (double)cs);
  }
  for (int a = ty; a < 32; a += 8) Xt16[(int64_t)(k0 + a) * np + i0 + tx] = to16<T16>(xs[tx][a]);
}

// Bytes of the Newton-Schulz matrix's block flags (tc::GemmArgs::aflags) for np unknowns.
inline size_t a16_flag_bytes(int np) { return (size_t)((np + 255) / 256) * ((np / 64 + 31) / 32 * 32); }
// Bytes of the first correction's B block flags (mp right-hand sides, np unknowns).
inline size_t rt_flag_bytes(int mp, int np) { return (size_t)((mp + 255) / 256) * ((np / 64 + 31) / 32 * 32); }

// ||E||_inf = max_i rowsum_i into e0_bits[0], ||E||_1 = max_k colsum_k into e0_bits[1] (bits,
// atomicMax; zeroed by the caller), and colmax[0 .. mp) = 0 for the first correction.
__global__ void ns_norms(const double* __restrict__ rowsum, const double* __restrict__ colsum, int np,
                         unsigned long long* e0_bits, unsigned long long* colmax, int mp) {
  unsigned long long r = 0ull, c = 0ull;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(np, mp); i += gridDim.x * blockDim.x) {
    if (i < np) {
      r = max(r, (unsigned long long)__double_as_longlong(rowsum[i]));
      c = max(c, (unsigned long long)__double_as_longlong(colsum[i]));
    }
    if (i < mp) colmax[i] = 0ull;
  }
  for (int q = 16; q > 0; q >>= 1) {
    r = max(r, __shfl_xor_sync(0xffffffffu, r, q));
    c = max(c, __shfl_xor_sync(0xffffffffu, c, q));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(e0_bits, r);
    atomicMax(e0_bits + 1, c);
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

// The refinement's stopping rule evaluated on the device, for a sweep launched before the
// host has read the residual of the sweep before it: err = the solver's error words, red =
// that sweep's status words (max|R|, max|X|), tol / prev as the host's loop has them. When
// that sweep ended the refinement (converged or stalled) or an error was reported, the new
// sweep is skipped: its first kernel returns at once and sets *skip, which the others read.
struct SweepGuard {
  const int* err = nullptr;
  const unsigned long long* red = nullptr;
  double tol = 0.0, prev = 0.0;
  int* skip = nullptr;
};

__device__ __forceinline__ bool sweep_ends(const SweepGuard& g) {
  const volatile int* w = g.err;
  const volatile unsigned long long* red = g.red;
  const double r = __longlong_as_double((long long)red[0]), x = __longlong_as_double((long long)red[1]);
  const double rel = x > 0 ? r / x : r;
  const bool done = rel <= g.tol || (rel <= kStallFloor && rel > 0.5 * g.prev);
  return done || w[0] || w[1] || w[4];
}

// 16-bit pair (lo, hi) as one 32-bit word, lo in the lower half.
template <class T16>
__device__ __forceinline__ uint32_t pack16(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack16<__nv_bfloat16>(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}
template <>
__device__ __forceinline__ uint32_t pack16<__half>(float lo, float hi) {
  const __half2 p = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}

// (float)(x 2^-e) for |x 2^-e| < 2^128, on the two 32-bit words of x (no fp64 arithmetic):
// the exponent moves by -e, the 52-bit mantissa is rounded to 23 bits to nearest, ties to
// even (a carry moves up the exponent). Results below 2^-126 in magnitude, and subnormal x,
// give a signed zero (the value is bound for a 16-bit operand scaled to [0.5, 1), whose
// resolution is far coarser); inf and NaN stay inf and NaN.
__device__ __forceinline__ float scaled_float(double x, int e) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u, t = hi & 0x7fffffffu;
  const int E = (int)(t >> 20);
  if (E == 2047) return __uint_as_float(sign | 0x7f800000u | (((t & 0xfffffu) | lo) ? 0x400000u : 0u));
  const int fe = E - e - 896;  // float biased exponent: E - 1023 - e + 127
  if (E == 0 || fe < 1) return __uint_as_float(sign);
  if (fe > 254) return __uint_as_float(sign | 0x7f800000u);
  const uint32_t m = ((t & 0xfffffu) << 3) | (lo >> 29), rem = lo & 0x1fffffffu;
  const uint32_t up = (rem > 0x10000000u) | ((rem == 0x10000000u) & m);
  const uint32_t bits = ((uint32_t)fe << 23) + m + (up & 1u);
  return __uint_as_float(sign | (bits < 0x7f800000u ? bits : 0x7f800000u));
}

// Rt16[j][i] = 16-bit (R_ij * 2^-e_j) with max_i |R_ij| 2^-e_j in [0.5, 1), zero padding
// (values below 2^-126 of the column maximum flushed to zero); colscale[j] = 2^e_j. Block
// (32 x 8) per 64 rows x 32 columns: eight row loads in flight per thread, the transposed
// rows written as 16-bit pairs (128 bytes per warp) through shared memory; integer
// arithmetic only (GB300's fp64 pipe is far narrower than its integer ALU).
// The first kernel of a sweep: it also zeroes the sweep's status words (red_cur: max|R|,
// max|X|, max|D|) and the column maxima of the correction (dcolmax[0 .. mp)).
template <class T16>
__global__ void scaled_transpose16(const double* __restrict__ R, int64_t ld, int n, int m, int np, int mp,
                                   const unsigned long long* __restrict__ colmax, T16* __restrict__ Rt,
                                   float* __restrict__ colscale, const SweepGuard guard,
                                   unsigned long long* red_cur, unsigned int* dcolmax,
                                   const float* __restrict__ rs, uint8_t* __restrict__ bflags) {
  __shared__ __align__(16) float tile[32][66];  // [column][row]: a row pair is one 8-byte read
  if (guard.err) {  // one thread per block evaluates the rule (an fp64 division), the block follows
    __shared__ int s_end;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      s_end = sweep_ends(guard) ? 1 : 0;
      if (blockIdx.x == 0 && blockIdx.y == 0) *guard.skip = s_end;
    }
    __syncthreads();
    if (s_end) return;
  }
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 32;
  const int j = j0 + threadIdx.x;
  if (blockIdx.y == 0 && threadIdx.y == 0 && j < mp) dcolmax[j] = 0u;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.y == 0 && threadIdx.x < 3) red_cur[threadIdx.x] = 0ull;
  // e_j from the bits of max_i |R_ij| (a non-negative double): frexp's exponent, or 0
  // when the maximum is 0 or not finite
  int e = 0;
  if (j < m) {
    const unsigned long long mb = colmax[j];
    const int E = (int)(mb >> 52);  // 2048 and up: the sign bit is set
    if (mb != 0ull && E < 2047) e = E >= 1 ? E - 1022 : (63 - __clzll((long long)mb)) - 1073;
  }
  if (blockIdx.y == 0 && threadIdx.y == 0 && j < mp) colscale[j] = ldexpf(1.f, e);
  double x[8];
  bool nonzero = false;
#pragma unroll
  for (int r = 0; r < 8; ++r) {  // warp-uniform rows: threadIdx.y is the warp
    const int i = i0 + threadIdx.y + 8 * r;
    x[r] = (i < n && j < m) ? R[(int64_t)i * ld + j] : 0.0;
    nonzero |= x[r] != 0.0;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + threadIdx.y + 8 * r;  // rs (a symmetric factorisation's row scale, <= 2^10) is 0 beyond n
    tile[threadIdx.x][threadIdx.y + 8 * r] = scaled_float(x[r], e) * (rs ? rs[i] : 1.f);
  }
  // with bflags: the block's 32 columns of Rt16 lie in one 256-row tile of the correction
  // GEMM's B and its 64 rows in one K block (tc::GemmArgs::bflags)
  if (__syncthreads_or(nonzero) && bflags && threadIdx.x == 0 && threadIdx.y == 0)
    bflags[(int64_t)(j0 / 256) * ((np / 64 + 31) / 32 * 32) + i0 / 64] = 1;
  // warp w writes columns j0 + w + 8 c, lane l the rows i0 + 2 l, i0 + 2 l + 1
  const int ii = i0 + 2 * threadIdx.x;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int jl = threadIdx.y + 8 * c, jj = j0 + jl;
    const float2 p = *reinterpret_cast<const float2*>(&tile[jl][2 * threadIdx.x]);
    if (jj < mp && ii < np) *reinterpret_cast<uint32_t*>(Rt + (int64_t)jj * np + ii) = pack16<T16>(p.x, p.y);
  }
}

// scaled_transpose16 for m <= kNarrow columns: one thread per row i (the writes Rt16[j][i]
// are consecutive along i); the same outputs and status words, rows j >= m of Rt16 left
// unwritten (the GEMM reads N = m rows).
template <class T16>
__global__ void __launch_bounds__(256) scaled_transpose16_narrow(
    const double* __restrict__ R, int64_t ld, int n, int m, int np, int mp,
    const unsigned long long* __restrict__ colmax, T16* __restrict__ Rt, float* __restrict__ colscale,
    const SweepGuard guard, unsigned long long* red_cur, unsigned int* dcolmax, const float* __restrict__ rs) {
  if (guard.err) {
    __shared__ int s_end;
    if (threadIdx.x == 0) {
      s_end = sweep_ends(guard) ? 1 : 0;
      if (blockIdx.x == 0) *guard.skip = s_end;
    }
    __syncthreads();
    if (s_end) return;
  }
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x < 3) red_cur[threadIdx.x] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x < mp) {
    dcolmax[threadIdx.x] = 0u;
    if (threadIdx.x >= m) colscale[threadIdx.x] = 1.f;
  }
#pragma unroll
  for (int j = 0; j < kNarrow; ++j) {
    if (j >= m) break;
    const unsigned long long mb = colmax[j];
    const int E = (int)(mb >> 52);
    int e = 0;
    if (mb != 0ull && E < 2047) e = E >= 1 ? E - 1022 : (63 - __clzll((long long)mb)) - 1073;
    if (blockIdx.x == 0 && threadIdx.x == 0) colscale[j] = ldexpf(1.f, e);
    if (i < np)
      Rt[(int64_t)j * np + i] =
          to16<T16>(i < n ? scaled_float(R[(int64_t)i * ld + j], e) * (rs ? rs[i] : 1.f) : 0.f);
  }
}

inline int grid_for(int64_t total, int sm) {
  int64_t b = (total + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sm * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// ------------------------------------------------------------------ shared balance preconditioner
// For the steady balance of opaque faces (rho = 1 - eps) with REFs that close (t = 1),
// diag(t) - B_NN = K^-1 (I - F_NN) with K = I - F_NN diag(rho), so one approximate inverse W of
// I - F_NN, shared by every (eps, rho) set, gives each set's correction as
//   forward  D = W K diag(t) R,          adjoint  D = K^T W^T diag(t) R
// (two matrix-vector products; the balance has one right-hand side). The residual stays the
// exact residual of the set's own balance, so W only sets the convergence rate.
struct BalancePre {
  const void* W = nullptr;    // 16-bit np x np, row-major (the Newton-Schulz iterate)
  const void* Wt = nullptr;   // its transpose
  const double* rho = nullptr;
  const double* t = nullptr;  // row sums of the set's B
  bool trans = false;         // the adjoint (transposed) balance
  bool fp16 = true;
  float* y = nullptr;         // [np] scratch vectors, zero beyond n
  float* yr = nullptr;        // the product's input vector
  float* z = nullptr;
  const float* gin = nullptr;   // W symmetric (W = D^-1 W_sym D): the product's input and
  const float* gout = nullptr;  // output row scales (d and 1 / d, the adjoint the other way)
};

// The first kernel of a preconditioned sweep, in fp32: y = diag(t) src (the residual column),
// z = rho o y and the product's input yr = (1 - rho) o y (forward) or y (adjoint), times gin
// when given; also zeroes the sweep's status words and the correction's column maximum.
__global__ void pre_first(const double* __restrict__ src, int64_t ld, const double* __restrict__ t,
                          const double* __restrict__ rho, int n, bool trans, float* __restrict__ y,
                          float* __restrict__ yr, float* __restrict__ z, const float* __restrict__ gin,
                          const SweepGuard guard, unsigned long long* red_cur, unsigned int* dcolmax) {
  if (guard.err) {
    __shared__ int s_end;
    if (threadIdx.x == 0) {
      s_end = sweep_ends(guard) ? 1 : 0;
      if (blockIdx.x == 0) *guard.skip = s_end;
    }
    __syncthreads();
    if (s_end) return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x < 3) red_cur[threadIdx.x] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x == 0) dcolmax[0] = 0u;
  if (i < n) {
    const double v = t[i] * src[(int64_t)i * ld];
    const double r = rho[i];
    y[i] = (float)v;
    z[i] = (float)(r * v);
    yr[i] = (float)(trans ? v : (1.0 - r) * v) * (gin ? gin[i] : 1.f);
  }
}

// D_k = (rho ? 1 - rho_k : 1) sum_i W[k][i] v_i + z_k, to D[k][0] (fp32), max_k |D_k| to
// dcolmax[0]: the balance correction W K y = W ((1 - rho) o y) + rho o y (forward: v = yr, no
// scale) or its transpose (1 - rho) o (W^T y) + rho o y (adjoint: W^T's rows, v = y, scale
// 1 - rho), which hold because W (I - F_NN) = I for the exact inverse W of I - F_NN. One warp
// per row of W, the 16-bit W read eight elements at a time, fp32 sums (W is a 16-bit
// approximate inverse, so fp32 is far more accurate than needed). v is zero beyond n, so the
// rows' padding (np is a multiple of 128) adds nothing.
template <class T16>
__global__ void pre_w_apply(const void* __restrict__ W, int np, int n, const float* __restrict__ v,
                            const double* __restrict__ rho, const float* __restrict__ z,
                            const float* __restrict__ gout, float* __restrict__ D, int64_t ldd,
                            unsigned int* dcolmax, int* nonfinite, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  const int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  const uint4* row = reinterpret_cast<const uint4*>(reinterpret_cast<const T16*>(W) + (int64_t)k * np);
  const float4* v4 = reinterpret_cast<const float4*>(v);
  float acc = 0.f, acc2 = 0.f;
  int g = lane;
  for (; g + 32 < np / 8; g += 64) {
    const uint4 w = row[g], w2 = row[g + 32];
    const T16* h = reinterpret_cast<const T16*>(&w);
    const T16* h2 = reinterpret_cast<const T16*>(&w2);
    const float4 a = v4[2 * g], b = v4[2 * g + 1], a2 = v4[2 * (g + 32)], b2 = v4[2 * (g + 32) + 1];
    acc = fmaf((float)h[0], a.x, acc);
    acc = fmaf((float)h[1], a.y, acc);
    acc = fmaf((float)h[2], a.z, acc);
    acc = fmaf((float)h[3], a.w, acc);
    acc = fmaf((float)h[4], b.x, acc);
    acc = fmaf((float)h[5], b.y, acc);
    acc = fmaf((float)h[6], b.z, acc);
    acc = fmaf((float)h[7], b.w, acc);
    acc2 = fmaf((float)h2[0], a2.x, acc2);
    acc2 = fmaf((float)h2[1], a2.y, acc2);
    acc2 = fmaf((float)h2[2], a2.z, acc2);
    acc2 = fmaf((float)h2[3], a2.w, acc2);
    acc2 = fmaf((float)h2[4], b2.x, acc2);
    acc2 = fmaf((float)h2[5], b2.y, acc2);
    acc2 = fmaf((float)h2[6], b2.z, acc2);
    acc2 = fmaf((float)h2[7], b2.w, acc2);
  }
  if (g < np / 8) {
    const uint4 w = row[g];
    const T16* h = reinterpret_cast<const T16*>(&w);
    const float4 a = v4[2 * g], b = v4[2 * g + 1];
    acc = fmaf((float)h[0], a.x, acc);
    acc = fmaf((float)h[1], a.y, acc);
    acc = fmaf((float)h[2], a.z, acc);
    acc = fmaf((float)h[3], a.w, acc);
    acc = fmaf((float)h[4], b.x, acc);
    acc = fmaf((float)h[5], b.y, acc);
    acc = fmaf((float)h[6], b.z, acc);
    acc = fmaf((float)h[7], b.w, acc);
  }
  acc += acc2;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const float d = (rho ? (float)(1.0 - rho[k]) : 1.f) * (gout ? gout[k] : 1.f) * acc + z[k];
    D[(int64_t)k * ldd] = d;
    if (!isfinite(d)) atomicExch(nonfinite, 1);
    else atomicMax(dcolmax, __float_as_uint(fabsf(d)));
  }
}

// ------------------------------------------------------------------ symmetric factorisation
// With reciprocity, A_i F_ij = A_j F_ji, the system matrix I - F_NN diag(rho) is similar to the
// symmetric I - G, G_ij = d_i F_ij rho_j / d_j with d_i = sqrt(A_i rho_i) (rho = 1 for the
// balance's I - F_NN): (I - G) = D (I - F diag(rho)) D^-1. Its Newton-Schulz iterates
// X (2I - A X) = 2X - X A X are symmetric, so the second product of each step computes the tiles
// on and above the diagonal only (the first, A X, is symmetric only where X and A commute,
// which rounding breaks: mirroring it lets the error grow step after step). The inverse
// M = D^-1 M_sym D is applied by scaling the correction's input rows by d and its output rows
// by 1/d (the transposed system: the other way round). d is normalised to max 1.

// words: [0] bad (a non-positive or non-finite A_i rho_i), [1] / [2] min / max of A_i rho_i
// (double bits, atomicMin / atomicMax; zeroed / set by the caller).
__global__ void sym_check(const double* __restrict__ area, const double* __restrict__ rho, int n,
                          unsigned long long* words) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double w = area[i] * (rho ? rho[i] : 1.0);
  if (!(w > 0.0) || !isfinite(w)) {
    atomicExch(&words[0], 1ull);
    return;
  }
  const unsigned long long b = (unsigned long long)__double_as_longlong(w);
  atomicMin(&words[1], b);
  atomicMax(&words[2], b);
}

// d_i = sqrt(A_i rho_i / wmax): dl = d, dr = rho / d (the Newton-Schulz start's scalings), and
// the correction's row scales fin = d, fout = 1 / d (forward) in fp32; zero beyond n.
__global__ void sym_fill(const double* __restrict__ area, const double* __restrict__ rho, int n, int np,
                         double wmax, double* __restrict__ dl, double* __restrict__ dr, float* __restrict__ fin,
                         float* __restrict__ fout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  if (i >= n) {
    dl[i] = dr[i] = 0.0;
    fin[i] = fout[i] = 0.f;
    return;
  }
  const double r = rho ? rho[i] : 1.0;
  const double d = sqrt(area[i] * r / wmax);
  dl[i] = d;
  dr[i] = r / d;
  fin[i] = (float)d;
  fout[i] = (float)(1.0 / d);
}

// the transposed system's row scales from a stored d: fin = 1 / d, fout = d (1 where d = 0: a
// general inverse, stored transposed, needs none)
__global__ void sym_scales_t(const double* __restrict__ d, int n, int np, float* __restrict__ fin,
                             float* __restrict__ fout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const double v = i < n ? d[i] : 0.0;
  fin[i] = i >= n ? 0.f : (v > 0.0 ? (float)(1.0 / v) : 1.f);
  fout[i] = i >= n ? 0.f : (v > 0.0 ? (float)v : 1.f);
}

// ------------------------------------------------------------------ solver object
struct Layout {
  int n, m, np, mp;
  bool want_q;  // accumulate Q = P' X (the REF adjoint's F^T Lambda)
};

struct Buffers {
  void* A16;      // np x np
  void* X16[2];   // np x np, Newton-Schulz iterates (ping-pong)
  void* Xt16;     // np x np, transpose of the current iterate
  void* Zt16;     // np x np, (2I - A X)^T
  void* Rt16;     // mp x np, scaled transposed right-hand side / residual
  float* colscale;               // mp
  unsigned long long* colmax;    // mp, column maxima of R (double bits)
  __nv_bfloat16* Aex;            // np x kLevels np, fixed-point slices of P'
  int* rowexp;                   // np
  uint8_t* flags;                // the slices' non-zero 256 x 64 blocks (SliceFlags)
  uint8_t* aflags;               // A16's non-zero 256 x 64 blocks (the first Newton-Schulz product)
  uint8_t* bflags;               // Rt16's non-zero 256 x 64 blocks (the first sweep's correction)
  float* Dbuf;                   // np x mp, correction M R before rounding
  unsigned int* dcolmax;         // mp, its column maxima (float bits)
  __nv_bfloat16* Bq;             // mp x np, the rounded correction, transposed
  int16_t* Dn;                   // np x mp, the rounded correction's integers
  int* dexp;                     // mp, its column exponents
  int32_t* lev;                  // exact_splits(n, m) x kLevels planes of exact_plane(n, m)
  double* R0;   // right-hand side (ld = mp)
  double* X;    // solution (ld = mp)
  double* R;    // residual (ld = mp)
  double* Q;    // P' X (ld = mp) when want_q, else null
  double* vec;  // [2][np] per-row scratch (row sums, diagonal scalings)
  double* nsum; // [2][np] row and column sums of |Dl P Dr| (Newton-Schulz start)
  double* symdl;  // [np] symmetric factorisation: d, and rho / d (its start's scalings)
  double* symdr;
  float* sfin;    // [np] the correction's row scales: input d, output 1 / d (or as set)
  float* sfout;
};

template <class Take>
void plan(const Layout& L, Take&& t) {
  for (int k = 0; k < 5; ++k) t.template take<uint16_t>((size_t)L.np * L.np);  // A16, X16 x2, Xt16, Zt16
  t.template take<uint16_t>((size_t)L.mp * L.np);                 // Rt16
  t.template take<float>((size_t)L.mp);                           // colscale
  t.template take<unsigned long long>((size_t)L.mp);              // colmax
  t.template take<__nv_bfloat16>((size_t)L.np * kLevels * L.np);  // Aex
  t.template take<int>((size_t)L.np);                             // rowexp
  t.template take<float>((size_t)L.np * L.mp);                    // Dbuf
  t.template take<unsigned int>((size_t)L.mp);                    // dcolmax
  t.template take<__nv_bfloat16>((size_t)L.mp * L.np);            // Bq
  t.template take<int16_t>((size_t)L.np * L.mp);                  // Dn
  t.template take<int>((size_t)L.mp);                             // dexp
  t.template take<int32_t>((size_t)exact_splits(L.n, L.m) * kLevels * tc::exact_plane(L.n, L.m));  // lev
  t.template take<double>((size_t)L.np * L.mp);                   // R0
  t.template take<double>((size_t)L.np * L.mp);                   // X
  t.template take<double>((size_t)L.np * L.mp);                   // R
  t.template take<double>(L.want_q ? (size_t)L.np * L.mp : 0);    // Q
  t.template take<double>((size_t)2 * L.np);                      // vec
  t.template take<double>((size_t)2 * L.np);                      // nsum
  t.template take<double>((size_t)L.np);                          // symdl
  t.template take<double>((size_t)L.np);                          // symdr
  t.template take<float>((size_t)L.np);                           // sfin
  t.template take<float>((size_t)L.np);                           // sfout
  t.template take<uint8_t>(slice_flag_bytes(L.np));               // slice flags
  t.template take<uint8_t>(a16_flag_bytes(L.np));                 // A16 flags
  t.template take<uint8_t>(rt_flag_bytes(L.mp, L.np));            // Rt16 flags
}

// The solver's status words in the context scratch (ints), laid out so that one copy
// returns everything a sweep's decision needs: [0] input error of the calling kernels,
// [1] non-finite value, [4] the GEMM wait time-out word, [5] the skip word of a
// speculatively launched sweep (SweepGuard), [6..7] ||E||_inf and [8..9] ||E||_1 of the
// first Newton-Schulz iterate's E, then per sweep parity p the sweep's words at [10 + 6p ..]:
// max|R|, max|X|, max|D| (doubles as bits).
constexpr int kStatus = 12;
constexpr int kStatusInts = 22;
static_assert(kStatus + 4 == tc::kGemmErrorSlot, "the GEMM error word sits in the status block");

struct Solver {
  rg_ctx* ctx;
  Layout L;
  Buffers b;
  bool bf16;
  cudaStream_t s;
  int* err;          // device status words (kStatus)
  const char* input_error = "invalid input to the solver";  // what err[0] means for the caller
  const double* P;
  int64_t ldp;
  bool transP;
  int cur = 0;       // which X16 buffer holds the current inverse
  int ns_steps = 0;
  int splits = 1;    // K splits of the last exact product
  const BalancePre* pre = nullptr;  // set: corrections from the shared balance preconditioner
  const void* minv = nullptr;       // set: a stored inverse (16-bit np x np, row-major) replaces factor()
  const double* sym_area = nullptr; // set: try the symmetric factorisation with these areas (factor_sym)
  bool sym = false;                 // the last factorisation was the symmetric one
  const float* rs_in = nullptr;     // the correction's row scales (symmetric inverse), or null
  const float* rs_out = nullptr;

  unsigned long long* red(int parity) { return reinterpret_cast<unsigned long long*>(err + 10 + 6 * parity); }

  // Workspace bytes of a solver of n unknowns and m right-hand sides after `extra_bytes`
  // reserved for the calling entry point (the sizes every call and the size queries use).
  static size_t bytes(int n, int m, bool want_q, size_t extra_bytes) {
    Layout L{n, m, (n + NB - 1) / NB * NB, (m + NB - 1) / NB * NB, want_q};
    rg::Sizer sz;
    plan(L, sz);
    return rg::align_up(extra_bytes, 256) + sz.off;
  }

  // Carves the solver's buffers out of the caller's workspace (user, user_bytes) or the
  // context's, after `extra_bytes` reserved for the calling entry point (returned in *extra).
  rg_status setup(int n, int m, bool use_bf16, cudaStream_t stream, size_t extra_bytes = 0, void** extra = nullptr,
                  bool want_q = false, void* user = nullptr, size_t user_bytes = 0, const char* fn = "solver") {
    L.n = n;
    L.m = m;
    L.np = (n + NB - 1) / NB * NB;
    L.mp = (m + NB - 1) / NB * NB;
    L.want_q = want_q;
    bf16 = use_bf16;
    s = stream;
    extra_bytes = rg::align_up(extra_bytes, 256);
    void* ws = nullptr;
    rg_status st = rg::workspace_or(ctx, user, user_bytes, bytes(n, m, want_q, extra_bytes), &ws, fn);
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
    b.Aex = cv.take<__nv_bfloat16>((size_t)L.np * kLevels * L.np);
    b.rowexp = cv.take<int>(L.np);
    b.Dbuf = cv.take<float>((size_t)L.np * L.mp);
    b.dcolmax = cv.take<unsigned int>(L.mp);
    b.Bq = cv.take<__nv_bfloat16>((size_t)L.mp * L.np);
    b.Dn = cv.take<int16_t>((size_t)L.np * L.mp);
    b.dexp = cv.take<int>(L.mp);
    b.lev = cv.take<int32_t>((size_t)exact_splits(L.n, L.m) * kLevels * tc::exact_plane(L.n, L.m));
    b.R0 = cv.take<double>((size_t)L.np * L.mp);
    b.X = cv.take<double>((size_t)L.np * L.mp);
    b.R = cv.take<double>((size_t)L.np * L.mp);
    b.Q = want_q ? cv.take<double>((size_t)L.np * L.mp) : nullptr;
    b.vec = cv.take<double>((size_t)2 * L.np);
    b.nsum = cv.take<double>((size_t)2 * L.np);
    b.symdl = cv.take<double>((size_t)L.np);
    b.symdr = cv.take<double>((size_t)L.np);
    b.sfin = cv.take<float>((size_t)L.np);
    b.sfout = cv.take<float>((size_t)L.np);
    b.flags = cv.take<uint8_t>(slice_flag_bytes(L.np));
    b.aflags = cv.take<uint8_t>(a16_flag_bytes(L.np));
    b.bflags = cv.take<uint8_t>(rt_flag_bytes(L.mp, L.np));
    err = ctx->d_scratch + kStatus;
    RG_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 6 * sizeof(int), s));  // error words and the GEMM's
    return RG_OK;
  }

  // The matrix P of every set (read directly or transposed); its fixed-point slices are
  // built by build_slices (they include Dr).
  rg_status set_matrix(const double* P_, int64_t ldp_, bool trans) {
    P = P_;
    ldp = ldp_;
    transP = trans;
    return RG_OK;
  }

  // Fixed-point slices of P' = P Dr (Dr may be null), with their block flags where the
  // right-hand sides are wide enough for the tensor-core level product (the narrow GEMV
  // reads no flags).
  rg_status build_slices(const double* dr) {
    // nsum (the Newton-Schulz start's sums, read before this) serves as the column maxima
    return launch_build_p(ctx, P, ldp, transP, dr, L.n, L.np, b.Aex, b.rowexp, err,
                          reinterpret_cast<unsigned long long*>(b.nsum), s, L.m > kNarrow ? b.flags : nullptr);
  }

  // Newton-Schulz approximate inverse of A = I - Dl P Dr into b.X16[cur].
  template <class T16>
  rg_status factor_t(const double* dl, const double* dr, bool symm, const double* gen_dr) {
    unsigned long long* e0 = reinterpret_cast<unsigned long long*>(err + 6);
    RG_CUDA_TRY(ctx, cudaMemsetAsync(e0, 0, 2 * sizeof(unsigned long long), s));
    T16* A16 = static_cast<T16*>(b.A16);
    T16* X[2] = {static_cast<T16*>(b.X16[0]), static_cast<T16*>(b.X16[1])};
    T16* Xt = static_cast<T16*>(b.Xt16);
    T16* Zt = static_cast<T16*>(b.Zt16);
    RG_CUDA_TRY(ctx, cudaMemsetAsync(b.nsum, 0, 2 * L.np * sizeof(double), s));
    RG_CUDA_TRY(ctx, cudaMemsetAsync(b.aflags, 0, a16_flag_bytes(L.np), s));
    build_ns_start<T16><<<dim3(L.np / 32, L.np / 32), dim3(32, 8), 0, s>>>(
        P, ldp, transP, dl, dr, L.n, L.np, A16, X[0], Xt, b.nsum, b.nsum + L.np, symm, gen_dr, b.aflags);
    ns_norms<<<std::max(1, std::min(ctx->sm_count, (std::max(L.np, L.mp) + 255) / 256)), 256, 0, s>>>(
        b.nsum, b.nsum + L.np, L.np, e0, b.colmax, L.mp);
    ctx->launches += 2;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    // the status words and e0 in one pinned read-back: one wait on the stream
    int* hs = ctx->h_scratch;
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(hs + kStatus, err, 10 * sizeof(int), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hs[kStatus]) return rg::fail(ctx, RG_ERR_NUMERIC, "%s", input_error);
    double e_inf, e_one;
    memcpy(&e_inf, hs + kStatus + 6, sizeof(e_inf));
    memcpy(&e_one, hs + kStatus + 8, sizeof(e_one));
    if (!std::isfinite(e_inf) || !std::isfinite(e_one)) return rg::fail(ctx, RG_ERR_NUMERIC, "non-finite system matrix");
    // build_ns_start writes X_1 = I + E (E = Dl P Dr), whose residual is I - A X_1 = E^2, and
    // each step X <- X (2I - A X) squares the residual: X_k has residual E^(2^k), bounded by
    // ||E||^(2^k) in any norm with ||E|| < 1. ||E||_inf (row sums) suits the Gebhart matrix
    // K = I - F diag(rho); its transpose, solved by the adjoint, has ||E||_1 < 1 instead
    // while its row sums (the column sums of F) can exceed 1: the smaller bound sets the
    // step count, the least k with ||E||^(2^k) <= the 16-bit floor.
    const double e0v = std::min(e_inf, e_one);
    const double floor16 = bf16 ? 0x1p-10 : 0x1p-13;
    int steps = kMaxNewtonSchulz;
    if (e0v < 1.0) {
      steps = 1;
      if (e0v > 0.0) steps = (int)std::ceil(std::log2(std::log(floor16) / std::log(e0v)));
      steps = std::max(1, std::min(steps, kMaxNewtonSchulz));
    }
    ns_steps = steps;
    cur = 0;
    for (int k = 1; k < steps; ++k) {  // step 1 was taken by build_ns_start
      // Zt = (2I - A X)^T : A operand A16 [i][k], B operand X^T rows = X columns (X itself
      // when symmetric); the whole product
      rg_status st = tc::gemm(ctx, bf16, A16, L.np, symm ? X[cur] : Xt, L.np, L.np, L.np, L.np,
                              tc::EpiTwoIMinusT<T16>{Zt, L.np}, s, nullptr, false, b.aflags);
      if (st != RG_OK) return st;
      // X' = X (2I - A X) : A operand X [i][k], B operand Z^T; symmetric when X and A are, so
      // then only its upper tiles are computed
      st = tc::gemm(ctx, bf16, X[cur], L.np, Zt, L.np, L.np, L.np, L.np,
                    tc::EpiStore16Both<T16>{X[cur ^ 1], symm ? X[cur ^ 1] : Xt, L.np, symm}, s, nullptr, symm);
      if (st != RG_OK) return st;
      cur ^= 1;
    }
    return RG_OK;
  }
  // symm: Dl P Dr is the symmetric form of P diag(gen_dr); the step count then comes from the
  // latter's norms (the residual the refinement sees is D^-1 (its residual) D)
  rg_status factor(const double* dl, const double* dr, bool symm = false, const double* gen_dr = nullptr) {
    const int tok = rg::timer_begin(ctx, rg::kTimeFactor, s);
    const rg_status st =
        bf16 ? factor_t<__nv_bfloat16>(dl, dr, symm, gen_dr) : factor_t<__half>(dl, dr, symm, gen_dr);
    rg::timer_end(ctx, tok, s);
    return st;
  }

  // The factorisation of I - P diag(rho) (rho null: 1) in its symmetric form when the areas
  // make A P symmetric and every A_i rho_i is positive, within 2^20 of the largest (sym set,
  // the correction's row scales in rs_in / rs_out); the general one otherwise.
  rg_status factor_sym(const double* area, const double* rho) {
    unsigned long long* words = reinterpret_cast<unsigned long long*>(b.nsum);  // free before the start
    RG_CUDA_TRY(ctx, cudaMemsetAsync(words, 0, 3 * sizeof(unsigned long long), s));
    RG_CUDA_TRY(ctx, cudaMemsetAsync(words + 1, 0xff, sizeof(unsigned long long), s));
    sym_check<<<(L.n + 255) / 256, 256, 0, s>>>(area, rho, L.n, words);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    int* hs = ctx->h_scratch;
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(hs, words, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    unsigned long long w[3];
    memcpy(w, hs, sizeof(w));
    double wmin, wmax;
    memcpy(&wmin, &w[1], sizeof(double));
    memcpy(&wmax, &w[2], sizeof(double));
    sym = w[0] == 0ull && wmax > 0.0 && wmin >= wmax * 0x1p-20;
    if (!sym) {
      rs_in = rs_out = nullptr;
      return factor(nullptr, rho, false);
    }
    sym_fill<<<(L.np + 255) / 256, 256, 0, s>>>(area, rho, L.n, L.np, wmax, b.symdl, b.symdr, b.sfin, b.sfout);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    rs_in = b.sfin;
    rs_out = b.sfout;
    return factor(b.symdl, b.symdr, true, rho);
  }

  // The staged finish_residual's shared memory is above the default limit: raised once per
  // device and thread.
  rg_status finish_staged_ready() {
    static thread_local int configured_device = -1;
    if (configured_device != ctx->device) {
      RG_CUDA_TRY(ctx, cudaFuncSetAttribute(finish_residual_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kFinSmem));
      configured_device = ctx->device;
    }
    return RG_OK;
  }

  // One sweep: D = M src (src = R0 for the first, R after), D rounded to its one-slice form and
  // added to X, R = src - D + Dl P' D exactly, then the sweep's words copied to the pinned
  // slot of its parity (ctx->ev_read[parity] recorded after the copy). With a guard the sweep
  // skips itself when the sweep before it ended the refinement.
  template <class T16>
  rg_status launch_sweep_t(int parity, bool first, const double* dl, const SweepGuard& g) {
    const double* src = first ? b.R0 : b.R;
    unsigned long long* rc = red(parity);
    const int* skip = g.err ? g.skip : nullptr;
    dim3 tg(L.mp / 32, L.np / 64), qg(L.mp / 64, L.np / 64);
    const int nb = L.np / 256 + (L.np % 256 ? 1 : 0);  // narrow kernels: one thread per row < np
    rg_status st = RG_OK;
    if (pre) {
      // D = W K diag(t) R (forward) or K^T W^T diag(t) R (adjoint), one column, as
      // W ((1 - rho) o y) + rho o y or (1 - rho) o (W^T y) + rho o y with y = diag(t) R
      const int rb = (L.n + 255) / 256, wb = (L.n + 7) / 8;
      pre_first<<<rb, 256, 0, s>>>(src, L.mp, pre->t, pre->rho, L.n, pre->trans, pre->y, pre->yr, pre->z, pre->gin,
                                   g, rc, b.dcolmax);
      auto wapply = pre->fp16 ? pre_w_apply<__half> : pre_w_apply<__nv_bfloat16>;
      if (!pre->trans)
        wapply<<<wb, 256, 0, s>>>(pre->W, L.np, L.n, pre->yr, nullptr, pre->z, pre->gout, b.Dbuf, L.mp, b.dcolmax,
                                  err + 1, skip);
      else
        wapply<<<wb, 256, 0, s>>>(pre->Wt, L.np, L.n, pre->yr, pre->rho, pre->z, pre->gout, b.Dbuf, L.mp, b.dcolmax,
                                  err + 1, skip);
      ctx->launches += 2;
      RG_CUDA_TRY(ctx, cudaGetLastError());
    } else {
      T16* Rt = static_cast<T16*>(b.Rt16);
      if (L.m <= kNarrow)
        scaled_transpose16_narrow<T16><<<nb, 256, 0, s>>>(src, L.mp, L.n, L.m, L.np, L.mp, b.colmax, Rt, b.colscale,
                                                          g, rc, b.dcolmax, rs_in);
      else {
        // the first sweep's right-hand side keeps F's zero blocks (the REFs' E = [F diag(eps) |
        // F_inf]): its correction GEMM skips them; the residuals after it are dense
        if (first) RG_CUDA_TRY(ctx, cudaMemsetAsync(b.bflags, 0, rt_flag_bytes(L.mp, L.np), s));
        scaled_transpose16<T16><<<tg, dim3(32, 8), 0, s>>>(src, L.mp, L.n, L.m, L.np, L.mp, b.colmax, Rt,
                                                            b.colscale, g, rc, b.dcolmax, rs_in,
                                                            first ? b.bflags : nullptr);
      }
      ++ctx->launches;
      RG_CUDA_TRY(ctx, cudaGetLastError());
      st = tc::gemm(ctx, bf16, minv ? minv : b.X16[cur], L.np, Rt, L.np, L.n, L.m, L.np,
                    tc::EpiCorrection{b.Dbuf, L.mp, b.colscale, b.dcolmax, err + 1, rs_out}, s, skip, false,
                    nullptr, (first && L.m > kNarrow) ? b.bflags : nullptr);
      if (st != RG_OK) return st;
    }
    if (L.m <= kNarrow)
      quantize_correction_narrow<<<nb, 256, 0, s>>>(b.Dbuf, L.n, L.m, L.np, L.mp, b.dcolmax, b.Bq, b.Dn, b.dexp,
                                                     b.X, first ? 1 : 0, rc, b.colmax, err + 1, skip);
    else
      quantize_correction<<<qg, dim3(32, 8), 0, s>>>(b.Dbuf, L.n, L.m, L.np, L.mp, b.dcolmax, b.Bq, b.Dn, b.dexp,
                                                     b.X, first ? 1 : 0, rc, b.colmax, err + 1, skip);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    // levels from max|D| / max|X| of this sweep (rc[2] / rc[1]), read on the device
    if (L.m <= kNarrow) {
      using Gemv = void (*)(const __nv_bfloat16*, const __nv_bfloat16*, int, int, int32_t*, int64_t, int64_t,
                            const unsigned long long*, const int*);
      static constexpr Gemv kGemv[kNarrow] = {exact_gemv_narrow<1>, exact_gemv_narrow<2>, exact_gemv_narrow<3>,
                                              exact_gemv_narrow<4>, exact_gemv_narrow<5>, exact_gemv_narrow<6>,
                                              exact_gemv_narrow<7>, exact_gemv_narrow<8>};
      kGemv[L.m - 1]<<<(L.n + 7) / 8, 256, 0, s>>>(b.Aex, b.Bq, L.n, L.np, b.lev, tc::exact_ld(L.m),
                                                    tc::exact_plane(L.n, L.m), rc, skip);
      ++ctx->launches;
      RG_CUDA_TRY(ctx, cudaGetLastError());
      splits = 1;
    } else {
      const SliceFlags fl = slice_flags(b.flags, L.np);
      st = tc::gemm_exact(ctx, b.Aex, (int64_t)kLevels * L.np, b.Bq, L.np, L.n, L.m, L.np, nullptr, rc, kLevelBits,
                          kLevels, b.lev, exact_splits(L.n, L.m), &splits, s, skip, L.n, fl.f, fl.rows, fl.ld);
      if (st != RG_OK) return st;
    }
    dim3 fg((L.m + 127) / 128, (L.n + 127) / 128);
    if (L.m > kNarrow && splits == 1) {
      st = finish_staged_ready();
      if (st != RG_OK) return st;
    }
    if (L.m <= kNarrow)
      finish_residual_narrow<<<nb, 256, 0, s>>>(b.lev, tc::exact_ld(L.m), tc::exact_plane(L.n, L.m), splits,
                                                 b.rowexp, b.dexp, b.Dn, dl, L.n, L.m, L.mp, b.R0, b.R, b.Q,
                                                 first ? 1 : 0, rc, b.colmax, err + 1, skip);
    else if (splits == 1)
      finish_residual_staged<<<dim3((L.m + 127) / 128, (L.n + kFinRows - 1) / kFinRows), dim3(32, 8), kFinSmem, s>>>(
          b.lev, tc::exact_ld(L.m), tc::exact_plane(L.n, L.m), b.rowexp, b.dexp, b.Dn, dl, L.n, L.m, L.mp, b.R0, b.R,
          b.Q, first ? 1 : 0, rc, b.colmax, err + 1, skip);
    else
      finish_residual<<<fg, dim3(32, 8), 0, s>>>(b.lev, tc::exact_ld(L.m), tc::exact_plane(L.n, L.m), splits,
                                                 b.rowexp, b.dexp, b.Dn, dl, L.n, L.m, L.mp, b.R0, b.R, b.Q,
                                                 first ? 1 : 0, rc, b.colmax, err + 1, skip);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    int* slot = ctx->h_scratch + kStatus + 32 * parity;
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(slot, err, kStatusInts * sizeof(int), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_read[parity], s));
    return RG_OK;
  }
  rg_status launch_sweep(int parity, bool first, const double* dl, const SweepGuard& g = SweepGuard{}) {
    return bf16 ? launch_sweep_t<__nv_bfloat16>(parity, first, dl, g) : launch_sweep_t<__half>(parity, first, dl, g);
  }

  // Waits for the read-back of the sweep of this parity (not for later launches).
  rg_status read_sweep(int parity, double* rel) {
    RG_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev_read[parity]));
    const int* hs = ctx->h_scratch + kStatus + 32 * parity;
    double r, x;
    memcpy(&r, hs + 10 + 6 * parity, 8);
    memcpy(&x, hs + 12 + 6 * parity, 8);
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

  // Factor, solve and refine one set whose right-hand side is already in b.R0. The
  // fixed-point slices of P' are rebuilt when `slices` (they depend on dr).
  rg_status run(const double* dl, const double* dr, double tol, int max_sweeps, int* sweeps, double* rel_out,
                bool slices = true) {
    rg_status st = RG_OK;
    if (minv) {
      // the stored inverse stands in for the factorisation; refine() wants the column maxima
      // zeroed, which the factorisation's norm kernel does otherwise
      RG_CUDA_TRY(ctx, cudaMemsetAsync(b.colmax, 0, L.mp * sizeof(unsigned long long), s));
    } else if (sym_area && !dl) {
      st = factor_sym(sym_area, dr);
    } else {
      st = factor(dl, dr);
    }
    if (st == RG_OK && slices) st = build_slices(dr);
    if (st != RG_OK) return st;
    return refine(dl, tol, max_sweeps, sweeps, rel_out);
  }

  // The refinement of run(), with the inverse (or the preconditioner) and the slices in place.
  rg_status refine(const double* dl, double tol, int max_sweeps, int* sweeps, double* rel_out) {
    rg_status st = RG_OK;
    if (!pre) {
      dim3 cg((L.m + 31) / 32, (L.n + 255) / 256);  // colmax was zeroed by build_ns_start
      column_max<<<cg, dim3(32, 8), 0, s>>>(b.R0, L.mp, L.n, L.m, b.colmax);
      ++ctx->launches;
      RG_CUDA_TRY(ctx, cudaGetLastError());
    }
    st = launch_sweep(0, true, dl);
    if (st != RG_OK) return st;
    double rel = INFINITY, prev = INFINITY;
    int sw = 0;
    bool done = false;
    for (; sw < max_sweeps; ++sw) {
      const int p = sw & 1;
      // the next sweep goes in before the host has read this one, so the GPU works while the
      // read-back travels; it evaluates the stopping rule on the device and does nothing when
      // this sweep ends the refinement
      if (sw + 1 < max_sweeps) {
        SweepGuard g;
        g.err = err;
        g.red = red(p);
        g.tol = tol;
        g.prev = prev;
        g.skip = err + 5;
        st = launch_sweep(p ^ 1, false, dl, g);
        if (st != RG_OK) return st;
      }
      st = read_sweep(p, &rel);
      if (st != RG_OK) return st;
      if (rel <= tol || (rel <= kStallFloor && rel > 0.5 * prev)) { done = true; break; }
      prev = rel;
    }
    *sweeps = sw + (done ? 1 : 0);
    *rel_out = rel;
    if (!done) {
      // the last speculative sweep (if any) was skipped by its guard only when it saw an
      // ending; wait for the stream before reporting
      RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
      return rg::fail(ctx, RG_ERR_NOT_CONVERGED, "refinement: residual %.3e > tol %.3e", rel, tol);
    }
    return RG_OK;
  }
};

// ------------------------------------------------------------------ stored factors
// The factor store rg_gebhart fills for the REF adjoints: a header, then per set the
// transpose of that set's Newton-Schulz inverse M of K = I - F diag(rho) (16-bit np x np,
// row-major). K^T = I - diag(rho) F^T is K transposed, and M is a polynomial in K, so M^T is
// as good an inverse of K^T as M is of K; stored transposed it is the correction GEMM's
// operand as it stands. The refinement computes its residual exactly, so a stored inverse
// decides only how fast the sweeps converge, never what they converge to.
constexpr uint32_t kFactorMagic = 0x31464752u;  // "RGF1"
constexpr size_t kFactorHeader = 256;
struct FactorHeader {
  uint32_t magic;
  int32_t n, n_sets, precision, np, filled;
};

size_t factor_store_bytes(int n, int n_sets) {
  const size_t np = (size_t)(n + NB - 1) / NB * NB;
  return kFactorHeader + (size_t)n_sets * np * np * sizeof(uint16_t) + (size_t)n_sets * np * sizeof(double);
}

void* factor_slice(const void* store, int n, int set) {
  const size_t np = (size_t)(n + NB - 1) / NB * NB;
  return static_cast<char*>(const_cast<void*>(store)) + kFactorHeader + (size_t)set * np * np * sizeof(uint16_t);
}

// the set's scale vector d after all the inverses (store_sets: the sets the store was made
// for): d > 0 when the set's inverse is the symmetric one (M_sym, with M = D^-1 M_sym D),
// zeros when it is the transpose of a general inverse
double* factor_dvec(const void* store, int n, int store_sets, int set) {
  const size_t np = (size_t)(n + NB - 1) / NB * NB;
  return reinterpret_cast<double*>(static_cast<char*>(const_cast<void*>(store)) + kFactorHeader +
                                   (size_t)store_sets * np * np * sizeof(uint16_t)) +
         (size_t)set * np;
}

__global__ void write_factor_header(FactorHeader* h, FactorHeader v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *h = v;
}

rg_status check_store_layout(rg_ctx* ctx, const void* store, size_t bytes, int n, int n_sets, const char* fn) {
  if (reinterpret_cast<uintptr_t>(store) & 255)
    return rg::fail(ctx, RG_ERR_ARG, "%s: the factor store must be 256-byte aligned", fn);
  if (bytes < factor_store_bytes(n, n_sets))
    return rg::fail(ctx, RG_ERR_ARG, "%s: the factor store holds %zu bytes, %d sets of n = %d need %zu", fn, bytes,
                    n_sets, n, factor_store_bytes(n, n_sets));
  return RG_OK;
}

// Reads the store's header and checks that it holds factors of n unknowns, in `precision`
// (the inverse is an operand of a GEMM whose other operand has that type), for n_sets sets;
// *store_sets receives the sets the store was made for.
rg_status check_stored_factors(rg_ctx* ctx, const void* store, size_t bytes, int n, int n_sets, int precision,
                               cudaStream_t s, const char* fn, int* store_sets) {
  rg_status st = check_store_layout(ctx, store, bytes, n, n_sets, fn);
  if (st != RG_OK) return st;
  FactorHeader h;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, store, sizeof(h), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  memcpy(&h, ctx->h_scratch, sizeof(h));
  if (h.magic != kFactorMagic || h.n != n || h.np != (n + NB - 1) / NB * NB)
    return rg::fail(ctx, RG_ERR_ARG, "%s: the factor store holds no factors of an n = %d system", fn, n);
  if (h.precision != precision)
    return rg::fail(ctx, RG_ERR_ARG, "%s: the factors were made in precision %d, the call asks for %d", fn,
                    h.precision, precision);
  if (h.filled < n_sets || h.n_sets < h.filled)
    return rg::fail(ctx, RG_ERR_ARG, "%s: the factor store holds %d sets, the call has %d", fn, h.filled, n_sets);
  if (bytes < factor_store_bytes(n, h.n_sets))
    return rg::fail(ctx, RG_ERR_ARG, "%s: the factor store is shorter than its %d sets", fn, h.n_sets);
  *store_sets = h.n_sets;
  return RG_OK;
}

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

// u_i = T_i^4 (once per set, so that the adjoint's row pass reads it instead of recomputing it
// per entry on the fp64 pipe).
__global__ void quartic_powers(const double* __restrict__ T, int n, double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double Ti = T[i];
  u[i] = Ti * Ti * Ti * Ti;
}

// dB_ij = -nu_i (u_i - u_j) (u_{n} = T_sink^4), deps_i = -(nu_i / eps_i) sum_j B_ij (u_i - u_j)
// with nu = g o mu the solution of the transposed balance and u = T^4 (quartic_powers). One
// warp per row.
// dB may be null; with fa / fb set, dB = fa_0 fb_0^T + fa_1 fb_1^T is also written in that
// factored form: fa_0 = -nu o u, fb_0 = 1; fa_1 = nu, fb_1 = (u, u_sink) (fa [2][n], fb [2][n+1]).
__global__ void balance_adj_out(const double* __restrict__ B, const double* __restrict__ eps,
                                const double* __restrict__ u, const double* __restrict__ nu, int64_t ldnu,
                                double u_sink, int n, double* __restrict__ dB, double* __restrict__ deps,
                                double* __restrict__ fa, double* __restrict__ fb) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double ui = u[i];
  const double v = nu[(int64_t)i * ldnu];
  double s = 0.0;
  for (int j = lane; j <= n; j += 32) {
    const double uj = j < n ? u[j] : u_sink;
    if (dB) dB[(int64_t)i * (n + 1) + j] = -v * (ui - uj);
    s += B[(int64_t)i * (n + 1) + j] * (ui - uj);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    deps[i] = -(v / eps[i]) * s;
    if (fa) {
      fa[i] = -v * ui;
      fa[n + i] = v;
      fb[i] = 1.0;
      fb[(n + 1) + i] = ui;
      if (i == 0) {
        fb[n] = 1.0;
        fb[(n + 1) + n] = u_sink;
      }
    }
  }
}

// Factored REF adjoint outputs (rg_gebhart_adjoint_factored), one warp per row k:
//   deps_k = sum_r b_r,k Q_kr,   drho_k = sum_r Q_kr (B b_r)_k,   Q = F^T X (ld = ldq).
__global__ void factored_grads(const double* __restrict__ B, const double* __restrict__ Q, int64_t ldq,
                               const double* __restrict__ b, int rank, int n, double* __restrict__ deps,
                               double* __restrict__ drho) {
  const int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  double de = 0.0, dr = 0.0;
  for (int r = 0; r < rank; ++r) {
    const double* br = b + (int64_t)r * (n + 1);
    double bb = 0.0;
    for (int j = lane; j <= n; j += 32) bb += B[(int64_t)k * (n + 1) + j] * br[j];
    for (int o = 16; o > 0; o >>= 1) bb += __shfl_xor_sync(0xffffffffu, bb, o);
    const double q = Q[(int64_t)k * ldq + r];
    de += br[k] * q;
    dr += q * bb;
  }
  if (lane == 0) {
    deps[k] = de;
    drho[k] = dr;
  }
}

// R0[i][r] = a_r,i (the factored cotangent's left factors as right-hand sides).
__global__ void factors_in(const double* __restrict__ a, int rank, int n, double* __restrict__ R0, int64_t ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int r = 0; r < rank; ++r) R0[(int64_t)i * ld + r] = a[(int64_t)r * n + i];
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

// Bytes rg_enforce_lsq reserves ahead of its solver.
size_t lsq_extra_bytes(int n) {
  const size_t nn1 = (size_t)n * (n + 1);
  rg::Sizer ex;
  ex.take<double>(nn1);            // F0
  ex.take<uint8_t>(nn1);           // mask
  ex.take<uint8_t>(nn1);           // next mask
  ex.take<double>((size_t)n * n);  // P
  ex.take<double>(n);              // dl
  ex.take<int>(4);                 // negative counter
  return ex.off;
}

// Bytes rg_temperatures_sets reserves ahead of its solver (the preconditioner's vectors).
size_t balance_sets_extra_bytes(int n) {
  const size_t np = (size_t)(n + NB - 1) / NB * NB;
  rg::Sizer ex;
  ex.take<float>(np);   // y
  ex.take<float>(np);   // yr
  ex.take<float>(np);   // z
  ex.take<double>(np);  // u = T^4 (adjoint)
  return ex.off;
}

}  // namespace

extern "C" {

rg_status rg_enforce_lsq(rg_ctx* ctx, int32_t n, const double* omega_d, double* F_d, int32_t nnr, int32_t spva,
                         int32_t max_passes, int32_t* passes_out_h, void* workspace_d, size_t workspace_bytes,
                         void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n > 0 && n <= 4096 && omega_d && F_d && max_passes >= 1, "rg_enforce_lsq: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn1 = (size_t)n * (n + 1);
  Solver sv{ctx};
  void* extra = nullptr;
  rg_status st = sv.setup(n, 1, false, s, lsq_extra_bytes(n), &extra, false, workspace_d, workspace_bytes,
                          "rg_enforce_lsq");
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

rg_status rg_exact_split(rg_ctx* ctx, int32_t n, const double* P_d, int64_t ldp, int32_t trans, const double* dr_d,
                         int16_t* slices_d, int32_t* rowexp_d, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n > 0 && n <= 32768 && P_d && slices_d && rowexp_d && ldp >= (trans ? n : n),
               "rg_exact_split: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int np = (n + NB - 1) / NB * NB;
  rg::Sizer sz;
  sz.take<__nv_bfloat16>((size_t)np * kLevels * np);
  sz.take<int>(np);
  sz.take<unsigned long long>(np);
  void* ws = nullptr;
  rg_status st = rg::workspace(ctx, sz.off, &ws);
  if (st != RG_OK) return st;
  rg::Carver cv(ws);
  __nv_bfloat16* Aex = cv.take<__nv_bfloat16>((size_t)np * kLevels * np);
  int* rowexp = cv.take<int>(np);
  unsigned long long* colmax = cv.take<unsigned long long>(np);
  int* e = ctx->d_scratch + kStatus;
  RG_CUDA_TRY(ctx, cudaMemsetAsync(e, 0, sizeof(int), s));
  st = launch_build_p(ctx, P_d, ldp, trans != 0, dr_d, n, np, Aex, rowexp, e, colmax, s);
  if (st != RG_OK) return st;
  bf16_rows_to_int16<<<grid_for((int64_t)n * kLevels * np, ctx->sm_count), kThreads, 0, s>>>(
      Aex, (int64_t)n * kLevels * np, slices_d);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(rowexp_d, rowexp, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
  RG_CUDA_TRY(ctx, cudaGetLastError());
  int h = 0;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, e, sizeof(int), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  h = ctx->h_scratch[0];
  if (h) return rg::fail(ctx, RG_ERR_NUMERIC, "rg_exact_split: non-finite entry");
  return RG_OK;
}

rg_status rg_gebhart(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets, const double* eps_d,
                     const double* rho_d, const double* area_d, int32_t precision, double tol, int32_t max_sweeps,
                     double* B_d,
                     int32_t* sweeps_out_h, double* resid_out_h, void* factors_d, size_t factors_bytes,
                     void* workspace_d, size_t workspace_bytes, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, max_sweeps);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, F_d && eps_d && rho_d && B_d && n_sets > 0, "rg_gebhart: bad argument");
  if (factors_d) {
    st = check_store_layout(ctx, factors_d, factors_bytes, n, n_sets, "rg_gebhart");
    if (st != RG_OK) return st;
  }
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Solver sv{ctx};
  st = sv.setup(n, n + 1, precision == RG_PREC_BF16_IR, s, 0, nullptr, false, workspace_d, workspace_bytes,
                "rg_gebhart");
  if (st == RG_OK) st = sv.set_matrix(F_d, n + 1, false);
  if (st != RG_OK) return st;
  sv.sym_area = area_d;  // with areas: the symmetric factorisation where it applies
  int max_sw = 0;
  double max_rel = 0.0;
  // the header says "no sets" until every set has been factorised
  auto header = [&](int filled) -> rg_status {
    if (!factors_d) return RG_OK;
    const FactorHeader h{kFactorMagic, n, n_sets, precision, sv.L.np, filled};
    write_factor_header<<<1, 32, 0, s>>>(static_cast<FactorHeader*>(factors_d), h);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    return RG_OK;
  };
  st = header(0);
  if (st != RG_OK) return st;
  for (int set = 0; set < n_sets; ++set) {
    const double* eps = eps_d + (size_t)set * n;
    const double* rho = rho_d + (size_t)set * n;
    gebhart_rhs<<<grid_for((int64_t)n * (n + 1), ctx->sm_count), kThreads, 0, s>>>(F_d, eps, n, sv.L.mp, sv.b.R0);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    // the factorisation keeps the transpose of its iterate in b.Xt16: with a store, that is
    // the set's slice of the store, which then holds M^T when the set is done
    if (factors_d) sv.b.Xt16 = factor_slice(factors_d, n, set);
    int sw = 0;
    double rel = 0.0;
    st = sv.run(nullptr, rho, tol, max_sweeps, &sw, &rel);
    if (st != RG_OK && st != RG_ERR_NOT_CONVERGED) return st;
    if (factors_d) {
      // the symmetric inverse itself and its scales; a general one is already there (its
      // transpose, kept by the factorisation) with zero scales
      double* dv = factor_dvec(factors_d, n, n_sets, set);
      if (sv.sym) {
        RG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.b.Xt16, sv.b.X16[sv.cur], (size_t)sv.L.np * sv.L.np * sizeof(uint16_t),
                                         cudaMemcpyDeviceToDevice, s));
        RG_CUDA_TRY(ctx, cudaMemcpyAsync(dv, sv.b.symdl, (size_t)sv.L.np * sizeof(double), cudaMemcpyDeviceToDevice, s));
      } else {
        RG_CUDA_TRY(ctx, cudaMemsetAsync(dv, 0, (size_t)sv.L.np * sizeof(double), s));
      }
    }
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
  return header(n_sets);
}

rg_status rg_gebhart_adjoint(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets, const double* eps_d,
                             const double* rho_d, const double* B_d, const double* dB_d, int32_t precision,
                             double tol, int32_t max_sweeps, double* deps_d, double* drho_d, const void* factors_d,
                             size_t factors_bytes, void* workspace_d, size_t workspace_bytes, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, max_sweeps);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, F_d && eps_d && rho_d && B_d && dB_d && deps_d && drho_d && n_sets > 0,
               "rg_gebhart_adjoint: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  int store_sets = 0;
  if (factors_d) {
    st = check_stored_factors(ctx, factors_d, factors_bytes, n, n_sets, precision, s, "rg_gebhart_adjoint", &store_sets);
    if (st != RG_OK) return st;
  }
  Solver sv{ctx};
  // K^T = I - diag(rho) F_NN^T: P' = F^T for every set; the refinement also accumulates
  // Q = F^T Lambda (the sum of its exact products), which the rho gradient needs
  st = sv.setup(n, n + 1, precision == RG_PREC_BF16_IR, s, 0, nullptr, true, workspace_d, workspace_bytes,
                "rg_gebhart_adjoint");
  if (st == RG_OK) st = sv.set_matrix(F_d, n + 1, true);
  if (st != RG_OK) return st;
  for (int set = 0; set < n_sets; ++set) {
    const double* rho = rho_d + (size_t)set * n;
    const size_t off = (size_t)set * n * (n + 1);
    copy_in<<<grid_for((int64_t)n * (n + 1), ctx->sm_count), kThreads, 0, s>>>(dB_d + off, n + 1, n, n + 1,
                                                                                sv.b.R0, sv.L.mp);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    if (factors_d) {
      sv.minv = factor_slice(factors_d, n, set);
      sym_scales_t<<<(sv.L.np + 255) / 256, 256, 0, s>>>(factor_dvec(factors_d, n, store_sets, set), n, sv.L.np,
                                                           sv.b.sfin, sv.b.sfout);
      ++ctx->launches;
      RG_CUDA_TRY(ctx, cudaGetLastError());
      sv.rs_in = sv.b.sfin;
      sv.rs_out = sv.b.sfout;
    }
    int sw = 0;
    double rel = 0.0;
    st = sv.run(rho, nullptr, tol, max_sweeps, &sw, &rel, set == 0);
    if (st != RG_OK) return st;
    // deps_j = sum_i Lam_ij F_ij
    grad_eps<<<(n + 31) / 32, dim3(32, 8), 0, s>>>(sv.b.X, sv.L.mp, F_d, n, deps_d + (size_t)set * n);
    ++ctx->launches;
    // drho_k = sum_j B_kj Q_kj with Q = F^T Lam
    grad_rho<<<(n + 7) / 8, 256, 0, s>>>(B_d + off, sv.b.Q, sv.L.mp, n, drho_d + (size_t)set * n);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
  }
  return sv.check_errors();
}

rg_status rg_temperatures(rg_ctx* ctx, int32_t n, const double* B_d, const double* eps_d, const double* area_d,
                          const double* Q_d, double T_sink, double sigma, int32_t precision, double tol, double* T_d,
                          void* workspace_d, size_t workspace_bytes, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, 1);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, B_d && eps_d && area_d && Q_d && T_d && T_sink >= 0.0 && sigma > 0.0,
               "rg_temperatures: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Solver sv{ctx};
  st = sv.setup(n, 1, precision == RG_PREC_BF16_IR, s, 0, nullptr, false, workspace_d, workspace_bytes,
                "rg_temperatures");
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
                                  void* workspace_d, size_t workspace_bytes, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, 1);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, B_d && eps_d && area_d && T_d && dT_d && dB_d && deps_d && sigma > 0.0,
               "rg_temperatures_adjoint: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Solver sv{ctx};
  st = sv.setup(n, 1, precision == RG_PREC_BF16_IR, s, 0, nullptr, false, workspace_d, workspace_bytes,
                "rg_temperatures_adjoint");
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
    // u = T^4 in the right-hand side's buffer, which the finished solve no longer reads
    double* u4 = sv.b.R0;
    quartic_powers<<<(n + 255) / 256, 256, 0, s>>>(T_d, n, u4);
    balance_adj_out<<<(n + 7) / 8, 256, 0, s>>>(B_d, eps_d, u4, sv.b.X, sv.L.mp, u_sink, n, dB_d, deps_d, nullptr,
                                                 nullptr);
    ctx->launches += 2;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    st = sv.check_errors();
  }
  return st;
}

// Steady temperatures of n_sets (eps, rho) sets through the shared preconditioner
// (BalancePre): one factorisation of I - F_NN for all sets, then per set the refinement of its
// own balance. adjoint: the transposed balance and its outputs (rg_temperatures_adjoint).
static rg_status temperatures_sets(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets, const double* B_d,
                                   const double* eps_d, const double* rho_d, const double* area_d, const double* Q_d,
                                   double T_sink, double sigma, int32_t precision, double tol, const double* T_in,
                                   const double* dT_d, double* T_d, double* dB_d, double* deps_d, double* fa_d,
                                   double* fb_d, void* workspace_d, size_t workspace_bytes, void* stream,
                                   bool adjoint) {
  const char* fn = adjoint ? "rg_temperatures_adjoint_sets" : "rg_temperatures_sets";
  rg_status st = check_common(ctx, n, precision, tol, 1);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, F_d && B_d && eps_d && rho_d && area_d && n_sets > 0 && sigma > 0.0 && T_sink >= 0.0 &&
                        (adjoint ? (T_in && dT_d && (dB_d || (fa_d && fb_d)) && deps_d) : (Q_d && T_d)),
               "%s: bad argument", fn);
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Solver sv{ctx};
  void* extra = nullptr;
  st = sv.setup(n, 1, precision == RG_PREC_BF16_IR, s, balance_sets_extra_bytes(n), &extra, false, workspace_d,
                workspace_bytes, fn);
  if (st != RG_OK) return st;
  rg::Carver cv(extra);
  BalancePre pre;
  pre.y = cv.take<float>(sv.L.np);
  pre.yr = cv.take<float>(sv.L.np);
  pre.z = cv.take<float>(sv.L.np);
  double* u4 = cv.take<double>(sv.L.np);
  // only entries below n are ever written: the padding stays zero for the row products
  RG_CUDA_TRY(ctx, cudaMemsetAsync(pre.y, 0, sv.L.np * sizeof(float), s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(pre.yr, 0, sv.L.np * sizeof(float), s));
  // W ~ (I - F_NN)^-1, shared by every set (symmetric via sqrt(A) when the areas allow)
  st = sv.set_matrix(F_d, n + 1, false);
  if (st == RG_OK) st = sv.factor_sym(area_d, nullptr);
  if (st != RG_OK) return st;
  pre.W = sv.b.X16[sv.cur];
  pre.Wt = sv.sym ? sv.b.X16[sv.cur] : sv.b.Xt16;
  if (sv.sym) {
    pre.gin = adjoint ? sv.b.sfout : sv.b.sfin;
    pre.gout = adjoint ? sv.b.sfin : sv.b.sfout;
  }
  sv.rs_in = sv.rs_out = nullptr;  // the corrections come from the preconditioner
  pre.trans = adjoint;
  pre.fp16 = precision == RG_PREC_FP16_IR;
  sv.pre = &pre;
  double* t = sv.b.vec;
  double* dl = sv.b.vec + sv.L.np;
  pre.t = t;
  const double u_sink = T_sink * T_sink * T_sink * T_sink;
  sv.input_error = adjoint ? "rg_temperatures_adjoint_sets: a face with no radiative exchange or sigma eps A <= 0"
                           : "rg_temperatures_sets: a face with no radiative exchange, sigma eps A <= 0, or a "
                             "non-positive T^4";
  for (int set = 0; set < n_sets; ++set) {
    const double* B = B_d + (size_t)set * n * (n + 1);
    const double* eps = eps_d + (size_t)set * n;
    pre.rho = rho_d + (size_t)set * n;
    st = sv.set_matrix(B, n + 1, adjoint);
    if (st == RG_OK) st = sv.build_slices(nullptr);
    if (st != RG_OK) return st;
    balance_setup<<<(n + 7) / 8, 256, 0, s>>>(B, eps, area_d, adjoint ? eps : Q_d + (size_t)set * n, u_sink, sigma, n,
                                               sv.L.mp, t, dl, adjoint ? nullptr : sv.b.R0, sv.err);
    ++ctx->launches;
    if (adjoint) {
      balance_adj_rhs<<<(n + 127) / 128, 128, 0, s>>>(T_in + (size_t)set * n, dT_d + (size_t)set * n, t, n, sv.L.mp,
                                                      sv.b.R0);
      ++ctx->launches;
    }
    RG_CUDA_TRY(ctx, cudaGetLastError());
    int sw = 0;
    double rel = 0.0;
    st = sv.refine(dl, tol, 24, &sw, &rel);
    if (st != RG_OK) return st;
    if (adjoint) {
      quartic_powers<<<(n + 255) / 256, 256, 0, s>>>(T_in + (size_t)set * n, n, u4);
      ++ctx->launches;
      balance_adj_out<<<(n + 7) / 8, 256, 0, s>>>(
          B, eps, u4, sv.b.X, sv.L.mp, u_sink, n, dB_d ? dB_d + (size_t)set * n * (n + 1) : nullptr,
          deps_d + (size_t)set * n, fa_d ? fa_d + (size_t)set * 2 * n : nullptr,
          fb_d ? fb_d + (size_t)set * 2 * (n + 1) : nullptr);
    } else {
      quartic_root<<<(n + 127) / 128, 128, 0, s>>>(sv.b.X, sv.L.mp, n, T_d + (size_t)set * n, sv.err);
    }
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
  }
  return sv.check_errors();
}

rg_status rg_temperatures_sets(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets, const double* B_d,
                               const double* eps_d, const double* rho_d, const double* area_d, const double* Q_d,
                               double T_sink, double sigma, int32_t precision, double tol, double* T_d,
                               void* workspace_d, size_t workspace_bytes, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  return temperatures_sets(ctx, n, F_d, n_sets, B_d, eps_d, rho_d, area_d, Q_d, T_sink, sigma, precision, tol,
                           nullptr, nullptr, T_d, nullptr, nullptr, nullptr, nullptr, workspace_d, workspace_bytes,
                           stream, false);
}

rg_status rg_temperatures_adjoint_sets(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets,
                                       const double* B_d, const double* eps_d, const double* rho_d,
                                       const double* area_d, double T_sink, double sigma, const double* T_d,
                                       const double* dT_d, int32_t precision, double tol, double* dB_d,
                                       double* dB_a_d, double* dB_b_d, double* deps_d, void* workspace_d,
                                       size_t workspace_bytes, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  return temperatures_sets(ctx, n, F_d, n_sets, B_d, eps_d, rho_d, area_d, nullptr, T_sink, sigma, precision, tol,
                           T_d, dT_d, nullptr, dB_d, deps_d, dB_a_d, dB_b_d, workspace_d, workspace_bytes, stream,
                           true);
}

rg_status rg_gebhart_adjoint_factored(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets,
                                      const double* eps_d, const double* rho_d, const double* B_d, int32_t rank,
                                      const double* a_d, const double* b_d, int32_t precision, double tol,
                                      int32_t max_sweeps, double* deps_d, double* drho_d, const void* factors_d,
                                      size_t factors_bytes, void* workspace_d, size_t workspace_bytes, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  rg_status st = check_common(ctx, n, precision, tol, max_sweeps);
  if (st != RG_OK) return st;
  RG_ARG_CHECK(ctx, F_d && eps_d && rho_d && B_d && a_d && b_d && deps_d && drho_d && n_sets > 0 && rank >= 1 &&
                        rank <= 64,
               "rg_gebhart_adjoint_factored: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  int store_sets = 0;
  if (factors_d) {
    st = check_stored_factors(ctx, factors_d, factors_bytes, n, n_sets, precision, s, "rg_gebhart_adjoint_factored",
                              &store_sets);
    if (st != RG_OK) return st;
  }
  Solver sv{ctx};
  // K^T X = A (rank right-hand sides), P' = F^T for every set, Q = F^T X accumulated
  st = sv.setup(n, rank, precision == RG_PREC_BF16_IR, s, 0, nullptr, true, workspace_d, workspace_bytes,
                "rg_gebhart_adjoint_factored");
  if (st == RG_OK) st = sv.set_matrix(F_d, n + 1, true);
  if (st != RG_OK) return st;
  for (int set = 0; set < n_sets; ++set) {
    const double* rho = rho_d + (size_t)set * n;
    factors_in<<<(n + 255) / 256, 256, 0, s>>>(a_d + (size_t)set * rank * n, rank, n, sv.b.R0, sv.L.mp);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    if (factors_d) {
      sv.minv = factor_slice(factors_d, n, set);
      sym_scales_t<<<(sv.L.np + 255) / 256, 256, 0, s>>>(factor_dvec(factors_d, n, store_sets, set), n, sv.L.np,
                                                           sv.b.sfin, sv.b.sfout);
      ++ctx->launches;
      RG_CUDA_TRY(ctx, cudaGetLastError());
      sv.rs_in = sv.b.sfin;
      sv.rs_out = sv.b.sfout;
    }
    int sw = 0;
    double rel = 0.0;
    st = sv.run(rho, nullptr, tol, max_sweeps, &sw, &rel, set == 0);
    if (st != RG_OK) return st;
    factored_grads<<<(n + 7) / 8, 256, 0, s>>>(B_d + (size_t)set * n * (n + 1), sv.b.Q, sv.L.mp,
                                                b_d + (size_t)set * rank * (n + 1), rank, n, deps_d + (size_t)set * n,
                                                drho_d + (size_t)set * n);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
  }
  return sv.check_errors();
}

rg_status rg_solver_workspace(int32_t kind, int32_t n, int32_t rank, size_t* bytes_out) {
  if (!bytes_out || n <= 0 || n > 32768) return RG_ERR_ARG;
  switch (kind) {
    case RG_WS_GEBHART: *bytes_out = Solver::bytes(n, n + 1, false, 0); return RG_OK;
    case RG_WS_GEBHART_ADJOINT: *bytes_out = Solver::bytes(n, n + 1, true, 0); return RG_OK;
    case RG_WS_GEBHART_ADJOINT_FACTORED:
      if (rank < 1 || rank > 64) return RG_ERR_ARG;
      *bytes_out = Solver::bytes(n, rank, true, 0);
      return RG_OK;
    case RG_WS_TEMPERATURES: *bytes_out = Solver::bytes(n, 1, false, 0); return RG_OK;
    case RG_WS_TEMPERATURES_SETS: *bytes_out = Solver::bytes(n, 1, false, balance_sets_extra_bytes(n)); return RG_OK;
    case RG_WS_ENFORCE_LSQ:
      if (n > 4096) return RG_ERR_ARG;
      *bytes_out = Solver::bytes(n, 1, false, lsq_extra_bytes(n));
      return RG_OK;
    default: return RG_ERR_ARG;
  }
}

rg_status rg_gebhart_workspace(int32_t n, int32_t n_sets, int32_t precision, int32_t keep_factors, size_t* bytes_out) {
  if (!bytes_out || n_sets <= 0 || (precision != RG_PREC_BF16_IR && precision != RG_PREC_FP16_IR)) return RG_ERR_ARG;
  if (n <= 0 || n > 32768) return RG_ERR_ARG;
  if (keep_factors) {
    *bytes_out = factor_store_bytes(n, n_sets);
    return RG_OK;
  }
  return rg_solver_workspace(RG_WS_GEBHART, n, 0, bytes_out);
}

}  // extern "C"
