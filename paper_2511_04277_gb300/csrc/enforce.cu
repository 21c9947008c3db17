// F from counts (Eq. 3.15), the iterative closure + reciprocity enforcer (Sec. 3.5.5)
// and the multi-node aggregation (Eq. 5.6-5.7), fp64 values.
//
// Iterative enforcer layout: the caller's F (N x (N+1), row-major, ld = N+1) is turned
// into H = Omega_i F_ij in place, and a row scale s (initially 1) is kept beside it, so
// that the current iterate is eta_ij = s_i H_ij. An iteration has two steps:
//   tiles  per tile pair (I, J), I <= J, of 32 x 32 tiles (64 x 64 for N > 2,048): loads
//          eta on both sides of the diagonal, writes H'_ij = kappa_ij eta_ij + (1 -
//          kappa_ij) eta_ji (kappa = 1/2, or per pair from a kappa matrix), records the
//          largest |eta_ij - eta_ji|/2 and per-tile row sums;
//   rows   carries the environment column (eta_i,inf = s_i H_i,inf), adds the row sums,
//          records |r_i - Omega_i| and sets s_i = Omega_i / r_i (Eq. 3.39-3.40 with
//          w = eta), then applies the stopping rule.
// On GB300 all iterations run in one cooperative launch (enforce_persistent), and with
// equal weights every iteration after the first works on the symmetric matrix, reading
// and writing only the tiles on and above the diagonal (see "symmetric iterations"
// below). The first iteration reads and writes every entry once: 16 bytes of HBM traffic
// (24 with a kappa matrix); the symmetric ones 16 bytes per stored entry of the upper
// triangle. sym_pass and row_pass are the same two steps as separate kernels, for
// devices without cooperative launches and for the allocation-free entry point.
#include <cfloat>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace {

constexpr int kT = 64;        // tile edge for n > kSmallN (and the allocation-free variant's sizing)
constexpr int kTSmall = 32;   // tile edge for n <= kSmallN: four times the blocks at N = 512
constexpr int kSmallN = 2048;

inline int tile_edge(int32_t n) { return n <= kSmallN ? kTSmall : kT; }
constexpr int kThreads = 256;

__global__ void counts_to_F_kernel(const long long* __restrict__ c, const long long* __restrict__ rays,
                                   double* __restrict__ F, int32_t n, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / (n + 1);
    F[e] = (double)c[e] / (double)rays[i];
  }
}

__global__ void to_exchange_kernel(double* __restrict__ H, const double* __restrict__ omega, double* __restrict__ s,
                                   int32_t n, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / (n + 1);
    H[e] = omega[i] * H[e];
    if (e % (n + 1) == 0) s[i] = 1.0;
  }
}

// q_i = s_i / Omega_i in place of s_i, and the environment column F_i,inf = q_i H_i,inf
__global__ void row_quotients(double* __restrict__ H, const double* __restrict__ omega, double* __restrict__ s,
                              int32_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double q = s[i] / omega[i];
    s[i] = q;
    H[i * (n + 1) + n] *= q;
  }
}

// F = q_i H on the N x N block (one fp64 multiplication per entry: GB300's fp64 divide
// costs several)
__global__ void from_exchange_kernel(double* __restrict__ H, const double* __restrict__ q, int32_t n, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n;
    H[i * (n + 1) + e % n] *= q[i];
  }
}

struct EnforceState {
  unsigned long long d_recip;  // bits of the largest reciprocity defect this iteration
  unsigned long long d_close;  // bits of the largest closure defect this iteration
  int32_t done;                // 0 running, 1 converged, 2 iteration limit, 3 non-finite
  int32_t iters;
  int32_t blocks_seen;
  int32_t pad;
};

// 8-byte asynchronous global -> shared copy (rows of H, ld = n + 1 doubles, are only
// 8-byte aligned, so neither 16-byte copies nor TMA apply): every thread keeps its
// 2 T^2 / kThreads copies in flight at once.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}

// Symmetrisation of the tile pair (I, J), I <= J (one block): T is the tile edge; kW:
// weights from kappa [n][n] (kappa_ij multiplies eta_ij), else 1/2. Folds the block's
// largest reciprocity defect into *d_recip and writes the tiles' row sums to P.
//
// GB300 runs fp64 at a small fraction of its fp32 rate, and this pass is bound by it
// unless the fp64 work per entry is small, so with equal weights a pair of entries
// costs six fp64 operations: the tiles hold e_ij = (s_i / 2) H_ij = eta_ij / 2 exactly
// (halving commutes with rounding; the raw tiles arrive by asynchronous copies and each
// entry is scaled once, where the values are formed), the symmetrised value is the single sum
// v_ij = e_ij + e_ji (= (eta_ij + eta_ji) / 2 bit for bit), the defect |e_ij - e_ji| is
// maximised on its bit pattern, and since v_ji = e_ji + e_ij = v_ij the tile (J, I) is
// the transpose of (I, J): its values are read transposed from shared memory. With
// weights both tiles are computed. The values pass through registers into the tile
// arrays, which the global writes and the row sums then read; the row sums run over a
// rotated column order so that the 16 lanes of a half-warp read 16 different banks (the
// row stride is T + 1 doubles: bank of (r, c) = (r + c) mod 16), in a fixed order that
// is the same on both paths (kappa = 1/2 given as weights gives the same bits). A
// negative symmetrised value raises *neg (when given): the symmetric iterations below
// need non-negative entries. With `nz`, *nz records whether the pair's symmetrised tiles
// hold a non-zero (a zero pair stays zero in every later symmetric iteration).
template <int T>
struct TileSmem {
  double A[T][T + 1];
  double B[T][T + 1];
  double sI[T], sJ[T];  // the tiles' row scales, halved for equal weights
  unsigned long long red[kThreads / 32];
};

template <int T, bool kW>
__device__ __forceinline__ void sym_tile(double* __restrict__ H, const double* __restrict__ s,
                                         const double* __restrict__ kappa, int32_t n, double* __restrict__ P, int I,
                                         int J, unsigned long long* d_recip, TileSmem<T>& sm, int* neg = nullptr,
                                         uint8_t* nz = nullptr) {
  static_assert(T == 64 || T == 32, "bank rotation for 64- and 32-wide tiles");
  constexpr int kPer = T * T / kThreads;  // entries per thread
  auto& A = sm.A;
  auto& B = sm.B;
  auto& sI = sm.sI;
  auto& sJ = sm.sJ;
  auto& red = sm.red;
  const int64_t ld = n + 1;
  const int tid = threadIdx.x;
  const bool off = I != J;
  const double h = kW ? 1.0 : 0.5;
  for (int e = tid; e < T * T; e += kThreads) {
    int r = e / T, c = e % T;
    int64_t i = (int64_t)I * T + r, j = (int64_t)J * T + c;
    if (i < n && j < n) cp_async8(&A[r][c], H + i * ld + j); else A[r][c] = 0.0;
    if (off) {
      int64_t i2 = (int64_t)J * T + r, j2 = (int64_t)I * T + c;
      if (i2 < n && j2 < n) cp_async8(&B[r][c], H + i2 * ld + j2); else B[r][c] = 0.0;
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (tid < T) {
    const int64_t i = (int64_t)I * T + tid, j = (int64_t)J * T + tid;
    sI[tid] = i < n ? h * __ldcg(s + i) : 0.0;
    sJ[tid] = j < n ? h * __ldcg(s + j) : 0.0;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // scaled entries: ea(r, c) = e_{I r, J c}, eb(r, c) = e_{J r, I c} (rounded products,
  // not fused into the sums that use them)
  auto ea = [&](int r, int c) { return __dmul_rn(sI[r], A[r][c]); };
  auto eb = [&](int r, int c) { return off ? __dmul_rn(sJ[r], B[r][c]) : __dmul_rn(sI[r], A[r][c]); };
  auto pair = [&](double a, double b, int64_t i, int64_t j) {
    if constexpr (kW) {
      const double k = kappa[i * n + j];
      return k * a + (1.0 - k) * b;
    } else {
      return a + b;
    }
  };
  double v1[kPer], v2[kW ? kPer : 1];
  unsigned long long dmax = 0ull;  // bit pattern of the largest defect (non-negative)
  bool negative = false, any = false;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int e = tid + k * kThreads, r = e / T, c = e % T;
    const int64_t i = (int64_t)I * T + r, j = (int64_t)J * T + c;
    const double a = ea(r, c), b = eb(c, r);
    v1[k] = (i < n && j < n) ? pair(a, b, i, j) : 0.0;
    negative |= v1[k] < 0.0;
    any |= v1[k] != 0.0;
    const double d = kW ? 0.5 * fabs(a - b) : fabs(a - b);
    dmax = max(dmax, (unsigned long long)__double_as_longlong(d));
    if constexpr (kW) {
      const int64_t i2 = (int64_t)J * T + r, j2 = (int64_t)I * T + c;
      v2[k] = (off && i2 < n && j2 < n) ? pair(eb(r, c), ea(c, r), i2, j2) : 0.0;
    }
  }
  __syncthreads();  // every read of the scaled tiles is done
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int e = tid + k * kThreads, r = e / T, c = e % T;
    A[r][c] = v1[k];
    if constexpr (kW) B[r][c] = v2[k];
    const int64_t i = (int64_t)I * T + r, j = (int64_t)J * T + c;
    if (i < n && j < n) H[i * ld + j] = v1[k];
  }
  __syncthreads();
  // value of the entry (J r, I c) of the tile (J, I)
  auto w2 = [&](int r, int c) { return kW ? B[r][c] : A[c][r]; };
  if (off) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int e = tid + k * kThreads, r = e / T, c = e % T;
      const int64_t i2 = (int64_t)J * T + r, j2 = (int64_t)I * T + c;
      if (i2 < n && j2 < n) H[i2 * ld + j2] = w2(r, c);
    }
  }
  // row sums of (I, J) and (J, I); kTpr threads per row, kCpt columns each
  constexpr int kTpr = kThreads / T, kCpt = T / kTpr;
  const int row = tid / kTpr, part = tid % kTpr;
  const int rot = T == 64 ? 4 * part : 2 * (part >> 2);
  double acc = 0.0, acc2 = 0.0;
  for (int it = 0; it < kCpt; ++it) {
    const int c = part * kCpt + ((it + rot) & (kCpt - 1));
    acc += A[row][c];
    if (off) acc2 += w2(row, c);
  }
#pragma unroll
  for (int o = 1; o < kTpr; o <<= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  }
  const int64_t ri = (int64_t)I * T + row, rj = (int64_t)J * T + row;
  const int nt = (n + T - 1) / T;
  if (part == 0) {
    if (ri < n) P[ri * nt + J] = acc;
    if (off && rj < n) P[rj * nt + I] = acc2;
  }
  for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((tid & 31) == 0) red[tid >> 5] = dmax;
  __syncthreads();
  if (tid == 0) {
    unsigned long long m = red[0];
    for (int w = 1; w < kThreads / 32; ++w) m = max(m, red[w]);
    atomicMax(d_recip, m);
  }
  if (__syncthreads_or(negative) && neg && tid == 0) atomicExch(neg, 1);  // also: the tiles are reused next
  if (nz) {
    const int a = __syncthreads_or(any);
    if (tid == 0) *nz = (uint8_t)(a != 0);
  }
}

template <int T, bool kW>
__global__ void __launch_bounds__(kThreads, 3) sym_pass(double* __restrict__ H, const double* __restrict__ s,
                                                     const double* __restrict__ kappa, int32_t n,
                                                     double* __restrict__ P, EnforceState* st) {
  if (st->done) return;
  const int I = blockIdx.y, J = blockIdx.x;
  if (I > J) return;
  __shared__ TileSmem<T> sm;
  sym_tile<T, kW>(H, s, kappa, n, P, I, J, &st->d_recip, sm);
}

// ---------------------------------------------------------------- persistent enforcer
// All iterations in one cooperative launch (every block resident): per iteration the
// blocks share the tile pairs (sym_tile), meet at a grid barrier, share the rows (the
// row_pass step), meet again and apply the stop rule, each block reaching the same
// decision. The defect accumulators alternate by iteration parity, so the ones an
// iteration reads are never reset under it. Every block owns the same tile pairs and
// rows in every iteration; what crosses blocks (row scales, per-tile row sums) is read
// through L2 (__ldcg), never from a block's L1.
struct PersistState {
  unsigned long long d_recip[2], d_close[2], smax[2];
  unsigned int d_recip_f[2];
  int32_t bad[2];
  unsigned int arrive, gen;
  int32_t done, iters, timeout;
  int32_t neg;    // a negative entry or non-positive row scale: every iteration on the full path
  int32_t sym;    // symmetric iterations ran: the tiles below the diagonal are stale
  int32_t range;  // a fixed-point row-sum term outside its bound (not expected)
};

constexpr unsigned long long kBarrierNs = 2000000000ull;  // a barrier wait gives up after 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch; false (and st->timeout set) if the wait
// exceeded limit_ns, after which the caller's block returns.
__device__ bool grid_barrier(PersistState* st, int* s_ok, unsigned long long limit_ns = kBarrierNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &st->gen;
    const unsigned int g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&st->arrive, 1u) + 1u == gridDim.x) {
      st->arrive = 0u;
      __threadfence();
      atomicAdd(&st->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      for (unsigned int it = 1; *gen == g; ++it) {
        if ((it & 255u) == 0 && global_ns() - t0 > limit_ns) {
          ok = 0;
          atomicExch(&st->timeout, 1);
          break;
        }
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// ---------------------------------------------------------------- symmetric iterations
// With equal weights the first iteration leaves the N x N block of H symmetric bit for
// bit (v_ij = e_ij + e_ji = v_ji), and it stays so: the next iterate is e_ij + e_ji with
// e_ij = h_i v_ij, that is (h_i + h_j) v_ij with h = s / 2. So from the second iteration
// on the blocks read and write only the tiles on and above the diagonal (8 bytes of HBM
// traffic per entry instead of 16), at one fp64 addition and one fp64 multiplication per
// stored entry. GB300 issues fp64 at about two lanes per clock per SM, so the row sums,
// which would cost two more fp64 additions per stored entry, are accumulated in 64-bit
// fixed point: the term of row i is v' 2^-U_i truncated to an integer, U_i = e_H + e_R,i
// - 61, where 2^e_H bounds max_j h_j and 2^e_R,i bounds the row's previous sum with its
// slack. Then sum_j v'_ij <= (h_i + h_max) R_i < 2^(U_i + 62): no term or sum reaches
// 2^63, the integer sum is exact, and each term is short of v' 2^-U_i by less than one
// unit, 2^-62 of the row's bound (subnormal terms count as zero). The reciprocity defect
// |eta_ij - eta_ji| / 2 = |h_i - h_j| v_ij only matters to the stop rule in an iteration
// whose closure defect is already within the tolerance; only then a separate pass takes
// it, in fp32, as |h_i - h_j| v'_ij / (h_i + h_j) from the fp32 (hi, lo) splits of the
// iteration's h and a truncated fp32 copy of v' scaled by 2^-e_Omega (e_Omega: the
// exponent of max Omega), so the stop decisions are those of a defect taken every
// iteration. The entries must be non-negative: a negative value after the first
// iteration (or a non-positive row scale) keeps every iteration on the full path.

// e with x < 2^e, for a finite x >= 0 (2^-1022 bounds zero and the subnormals)
__device__ __forceinline__ int bound_exp(double x) {
  const int e = (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF;
  return e ? e - 1022 : -1022;
}

// x >> s with the shift count clamped to 64 (PTX shr semantics: the result is 0 for s >= 64)
__device__ __forceinline__ unsigned long long shr_clamped(unsigned long long x, unsigned s) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}

// v 2^-eoff as a truncated fp32 (0 below the fp32 normal range), v >= 0 finite
__device__ __forceinline__ float scaled_f32(unsigned long long b, int eoff) {
  const int e = (int)(b >> 52) - 896 - eoff;
  if (e <= 0) return 0.0f;
  return __uint_as_float(((unsigned)min(e, 254) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
}

// RN(h_i + h_j) from the fixed-point values X = h 2^54, exact integers for h in [1/4, 1):
// the exact sum C lies in [2^53, 2^55) and is rounded to 53 bits, ties to even, so the
// result has the bits of the fp64 addition while GB300's fp64 pipe stays free.
__device__ __forceinline__ double fixed_sum_rn(unsigned long long Xi, unsigned long long Xj) {
  const unsigned long long C = Xi + Xj;
  const unsigned k = 1u + (unsigned)(C >> 54);  // bits below the 53-bit significand
  const unsigned long long q = (C + (k - 1u) + ((C >> k) & 1ull)) >> k;
  return __longlong_as_double((long long)(((unsigned long long)(1021u + k) << 52) + q - (1ull << 52)));
}

// Per-row data of the tile pair a block works on: h = s / 2, its fixed-point form h 2^54
// (fixed_sum_rn) and K = 1086 + U (the shift of a term is K minus the biased exponent of
// v'); the fp32 splits of h for the defect pass; column partial sums of the tile.
template <int T>
struct SymMeta {
  double hI[T], hJ[T];
  unsigned long long xI[T], xJ[T];
  int KI[T], KJ[T];
  float2 pI[T], pJ[T];
  unsigned long long colred[kThreads];
};

// Tile (I, J) of H into X by asynchronous 8-byte copies (zeros outside the matrix).
template <int T>
__device__ __forceinline__ void load_tile(const double* __restrict__ H, int32_t n, int I, int J, double (*X)[T + 1]) {
  const int64_t ld = n + 1;
  for (int e = threadIdx.x; e < T * T; e += kThreads) {
    const int r = e / T, c = e % T;
    const int64_t i = (int64_t)I * T + r, j = (int64_t)J * T + c;
    if (i < n && j < n) cp_async8(&X[r][c], H + i * ld + j);
    else X[r][c] = 0.0;
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// h, h 2^54 and K of the tile pair's rows (I) and columns (J); rows outside the matrix
// get h = 1/4 and a shift that clears every term. False when some h of the tile lies
// outside [1/4, 1), where h 2^54 is not an integer of the fixed-point sum (a per-thread
// answer: the caller combines them at its barrier).
template <int T>
__device__ __forceinline__ bool load_meta(const double* __restrict__ s, const int* __restrict__ eR, int eH,
                                          int32_t n, int I, int J, SymMeta<T>& m) {
  const int t = threadIdx.x;
  bool ok = true;
  if (t < 2 * T) {
    const bool col = t >= T;
    const int q = t & (T - 1);
    const int64_t i = (int64_t)(col ? J : I) * T + q;
    double h = 0.25;
    int K = 4096;
    if (i < n) {  // written by other blocks' row steps: read through L2
      h = 0.5 * __ldcg(s + i);
      K = 1086 + eH + __ldcg(eR + i) - 61;
    }
    const unsigned long long b = (unsigned long long)__double_as_longlong(h);
    const int e = (int)(b >> 52);
    ok = e == 1021 || e == 1022;
    (col ? m.hJ : m.hI)[q] = h;
    (col ? m.xJ : m.xI)[q] = ok ? ((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << (e - 1021) : 0ull;
    (col ? m.KJ : m.KI)[q] = K;
  }
  return ok;
}

// One symmetric iteration on the tile (I, J), I <= J, held in X: v' = (h_i + h_j) v is
// written to H; the fixed-point row sums go to P[rows of I][J] and (off the diagonal)
// P[rows of J][I]. emax collects the largest biased exponent of v' (2047: not finite),
// smin the smallest term shift (below 1: a bound violated). The diagonal tile is
// processed whole (both of its triangles).
template <int T, bool kFix>
__device__ __forceinline__ void sym_tile_fast(double* __restrict__ H, int32_t n, unsigned long long* __restrict__ P,
                                              int I, int J, double (*X)[T + 1], SymMeta<T>& m, unsigned& emax,
                                              int& smin) {
  constexpr int kPer = T * T / kThreads, kStep = kThreads / T;
  const int tid = threadIdx.x, c = tid % T, r0 = tid / T;
  const bool off = I != J;
  const bool inner = (int64_t)(I + 1) * T <= n && (int64_t)(J + 1) * T <= n;
  const int64_t ld = n + 1;
  const int64_t j = (int64_t)J * T + c;
  const double hc = m.hJ[c];
  const unsigned long long xc = m.xJ[c];
  const int Kc = m.KJ[c];
  double* hrow = H + ((int64_t)I * T + r0) * ld + j;
  unsigned long long colacc = 0;
#pragma unroll 4
  for (int k = 0; k < kPer; ++k) {
    const int r = r0 + k * kStep;
    const double cij = kFix ? fixed_sum_rn(m.xI[r], xc) : __dadd_rn(m.hI[r], hc);
    const double w = __dmul_rn(cij, X[r][c]);
    if (inner || ((int64_t)I * T + r < n && j < n)) hrow[(int64_t)k * kStep * ld] = w;
    const unsigned hi = (unsigned)__double2hiint(w), lo = (unsigned)__double2loint(w);
    const int e = (int)(hi >> 20);  // the sign bit (never set here) would make it >= 2048
    emax = max(emax, (unsigned)e);
    // the 53-bit significand moved to the top of 64 bits
    const unsigned long long M = ((unsigned long long)(__funnelshift_l(lo, hi, 11) | 0x80000000u) << 32) | (lo << 11);
    const int ee = e ? e : -4096;  // zero and subnormal: shifted out entirely
    const int sr = m.KI[r] - ee, sc = Kc - ee;
    smin = min(smin, min(sr, sc));
    if (off) colacc += shr_clamped(M, (unsigned)sc);
    X[r][c] = __longlong_as_double((long long)shr_clamped(M, (unsigned)sr));  // only this thread reads the slot
  }
  __syncthreads();
  // row sums over the rotated column order of sym_tile (16 distinct banks per half-warp)
  constexpr int kTpr = kThreads / T, kCpt = T / kTpr;
  const int row = tid / kTpr, part = tid % kTpr;
  const int rot = T == 64 ? 4 * part : 2 * (part >> 2);
  unsigned long long acc = 0;
  for (int it = 0; it < kCpt; ++it)
    acc += (unsigned long long)__double_as_longlong(X[row][part * kCpt + ((it + rot) & (kCpt - 1))]);
#pragma unroll
  for (int o = 1; o < kTpr; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int64_t ri = (int64_t)I * T + row;
  const int nt = (n + T - 1) / T;
  if (part == 0 && ri < n) P[ri * nt + J] = acc;
  if (off) {
    m.colred[tid] = colacc;
    __syncthreads();
    if (tid < T && j < n) {
      unsigned long long t = 0;
      for (int q = 0; q < kStep; ++q) t += m.colred[tid + q * T];
      P[j * nt + I] = t;
    }
  }
  __syncthreads();  // X and the row data are reused by the next pair
}

// Largest |h_i - h_j| v_ij = |h_i - h_j| v'_ij / (h_i + h_j) over the tile (I, J) in X
// (fp32 bits of a non-negative value), from the fp32 splits of the iteration's h.
template <int T>
__device__ __forceinline__ unsigned tile_defect(int32_t n, int I, int J, double (*X)[T + 1], const SymMeta<T>& m,
                                                int eoff) {
  unsigned dmax = 0u;
  for (int e = threadIdx.x; e < T * T; e += kThreads) {
    const int r = e / T, c = e % T;
    if ((int64_t)I * T + r >= n || (int64_t)J * T + c >= n) continue;
    const float2 a = m.pI[r], b = m.pJ[c];
    const float d = fabsf((a.x - b.x) + (a.y - b.y)) *
                    __fdividef(scaled_f32((unsigned long long)__double_as_longlong(X[r][c]), eoff), a.x + b.x);
    dmax = max(dmax, __float_as_uint(d));
  }
  return dmax;
}

// Walks the tile pairs p, p + stride, ... (numbered row by row over I <= J) without
// recounting from the first row at every step.
struct PairWalker {
  int I, q, nt, p;  // p: the pair's number
  __device__ PairWalker(int p0, int n_tiles) : I(0), q(p0), nt(n_tiles), p(p0) { settle(); }
  __device__ void settle() {
    while (I < nt && q >= nt - I) {
      q -= nt - I;
      ++I;
    }
  }
  __device__ void advance(int stride) {
    q += stride;
    p += stride;
    settle();
  }
  __device__ bool valid() const { return I < nt; }
  __device__ int J() const { return I + q; }
  // on to the next pair (this one included) whose flag is non-zero; flags written by this
  // block in an earlier iteration or by an earlier kernel, read through L2
  __device__ void skip_zero(const uint8_t* nz, int stride) {
    if (!nz) return;
    while (valid() && !__ldcg(nz + p)) advance(stride);
  }
};

// fp32 (hi, lo) split of h: h - hi is exact in fp64, lo its rounding
__device__ __forceinline__ float2 split_f32(double h) {
  const float hi = __double2float_rn(h);
  return make_float2(hi, __double2float_rn(h - (double)hi));
}

// hp holds two buffers of N splits: the row step of iteration k writes buffer k & 1, the
// next tile step reads the same h through s, and the defect pass of iteration k reads
// buffer (k - 1) & 1 (the h its tile step used).
template <int T, bool kW>
__global__ void __launch_bounds__(kThreads, 3) enforce_persistent(double* __restrict__ H, double* __restrict__ s,
                                                               float2* __restrict__ hp, int* __restrict__ eR,
                                                               const double* __restrict__ kappa,
                                                               const double* __restrict__ omega, int32_t n,
                                                               int32_t n_tiles, double* __restrict__ P,
                                                               PersistState* st, double tol_abs, int32_t maxit,
                                                               int eoff, uint8_t* __restrict__ tile_nz) {
  __shared__ TileSmem<T> sm;
  __shared__ SymMeta<T> meta;
  __shared__ double red[kThreads];
  __shared__ int s_ok;
  const int64_t ld = n + 1;
  unsigned long long* Pu = reinterpret_cast<unsigned long long*>(P);
  bool fast = false;  // the symmetric iterations (decided after the first, the same in every block)
  int eH = 0;
  for (int k = 0;; ++k) {
    const int par = k & 1;
    // (1) reciprocity on the tile pairs (I, J), I <= J, numbered row by row
    if (!fast) {
      for (PairWalker w(blockIdx.x, n_tiles); w.valid(); w.advance(gridDim.x))
        sym_tile<T, kW>(H, s, kappa, n, P, w.I, w.J(), &st->d_recip[par], sm, k == 0 ? &st->neg : nullptr,
                        (k == 0 && !kW) ? tile_nz + w.p : nullptr);
    } else if constexpr (!kW) {
      unsigned emax = 0u;
      int smin = 64;
      // the zero pairs (flagged by the first iteration) stay zero, their row sums 0
      PairWalker w(blockIdx.x, n_tiles);
      w.skip_zero(tile_nz, gridDim.x);
      if (w.valid()) load_tile<T>(H, n, w.I, w.J(), sm.A);
      for (int cur = 0; w.valid(); cur ^= 1) {
        const int I = w.I, J = w.J();
        w.advance(gridDim.x);
        w.skip_zero(tile_nz, gridDim.x);
        if (w.valid()) {  // prefetch the next pair's tile into the other buffer
          load_tile<T>(H, n, w.I, w.J(), cur ? sm.A : sm.B);
          asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
          asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        const bool fixed = !__syncthreads_or(!load_meta<T>(s, eR, eH, n, I, J, meta));
        if (fixed) sym_tile_fast<T, true>(H, n, Pu, I, J, cur ? sm.B : sm.A, meta, emax, smin);
        else sym_tile_fast<T, false>(H, n, Pu, I, J, cur ? sm.B : sm.A, meta, emax, smin);
      }
      if (__syncthreads_or(emax >= 2047u) && threadIdx.x == 0) atomicExch(&st->bad[par], 1);
      if (__syncthreads_or(smin < 1) && threadIdx.x == 0) atomicExch(&st->range, 1);
    }
    if (!grid_barrier(st, &s_ok)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // last read before the barrier just passed
      st->d_recip[par ^ 1] = 0ull;
      st->d_close[par ^ 1] = 0ull;
      st->smax[par ^ 1] = 0ull;
      st->d_recip_f[par ^ 1] = 0u;
      st->bad[par ^ 1] = 0;
    }
    // (2) environment column carried over, closure by row scaling: one warp per row, its
    // lanes adding the row's per-tile partial sums (contiguous: P[row][tile])
    double dc = 0.0;
    unsigned long long smax = 0ull;
    bool bad = false, nonpos = false;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t i = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; i < n; i += nwarps) {
      double R = 0.0, slack = 0.0;
      if (!fast) {
        for (int J = lane; J < n_tiles; J += 32) R += __ldcg(P + i * n_tiles + J);  // written by other blocks
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) R += __shfl_xor_sync(0xffffffffu, R, o);
      } else {
        unsigned long long t = 0;
        for (int J = lane; J < n_tiles; J += 32) t += __ldcg(Pu + i * n_tiles + J);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        const int U = eH + eR[i] - 61;  // the unit the tile step used for this row
        R = ldexp((double)t, U);
        slack = (double)n * (ldexp(1.0, U) + 0x1p-1022);  // truncation: under a unit per term
      }
      __syncwarp();  // every lane has read eR[i] before lane 0 rewrites it
      if (lane == 0) {
        const double env = s[i] * H[i * ld + n];
        H[i * ld + n] = env;
        const double r = R + env;
        dc = fmax(dc, fabs(r - omega[i]));
        const double sn = (r > 0.0) ? omega[i] / r : 1.0;
        s[i] = sn;
        if constexpr (!kW) {
          hp[(int64_t)par * n + i] = split_f32(0.5 * sn);
          eR[i] = bound_exp(R * (1.0 + 0x1p-30) + slack);
          smax = max(smax, (unsigned long long)__double_as_longlong(sn));
          nonpos |= !(sn > 0.0);
        }
        bad |= !isfinite(r);
      }
    }
    red[threadIdx.x] = dc;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&st->bad[par], 1);
    if (__syncthreads_or(nonpos) && threadIdx.x == 0) atomicExch(&st->neg, 1);
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(&st->d_close[par], (unsigned long long)__double_as_longlong(red[0]));
    for (int o = 16; o > 0; o >>= 1) smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    if ((threadIdx.x & 31) == 0 && smax) atomicMax(&st->smax[par], smax);
    if (!grid_barrier(st, &s_ok)) return;
    // (3) stop rule on this iteration's defects; on the symmetric path the reciprocity
    // defect is taken only when the closure defect already meets the tolerance
    volatile PersistState* v = st;
    const double dcl = __longlong_as_double((long long)v->d_close[par]);
    double dr = __longlong_as_double((long long)v->d_recip[par]);
    if constexpr (!kW) {
      if (fast) {
        dr = INFINITY;
        if (!v->bad[par] && dcl <= tol_abs) {
          unsigned dmax = 0u;
          for (PairWalker w(blockIdx.x, n_tiles); w.skip_zero(tile_nz, gridDim.x), w.valid();
               w.advance(gridDim.x)) {
            const int I = w.I, J = w.J();
            load_tile<T>(H, n, I, J, sm.A);
            if (threadIdx.x < 2 * T) {
              const int q = threadIdx.x & (T - 1);
              const int64_t i = (int64_t)(threadIdx.x < T ? I : J) * T + q;
              (threadIdx.x < T ? meta.pI : meta.pJ)[q] =
                  i < n ? __ldcg(hp + (int64_t)(par ^ 1) * n + i) : make_float2(0.0f, 0.0f);
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            dmax = max(dmax, tile_defect<T>(n, I, J, sm.A, meta, eoff));
            __syncthreads();
          }
          for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
          if ((threadIdx.x & 31) == 0 && dmax) atomicMax(&st->d_recip_f[par], dmax);
          if (!grid_barrier(st, &s_ok)) return;
          dr = ldexp((double)__uint_as_float(v->d_recip_f[par]), eoff);
        }
      }
    }
    const int done = v->bad[par] ? 3 : (fmax(dr, dcl) <= tol_abs ? 1 : (k + 1 >= maxit ? 2 : 0));
    if (done) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->done = done;
        st->iters = k + 1;
      }
      return;
    }
    if (k == 0 && !kW && !v->neg) {
      fast = true;
      if (blockIdx.x == 0 && threadIdx.x == 0) st->sym = 1;
    }
    if (fast) eH = bound_exp(0.5 * __longlong_as_double((long long)v->smax[par]));
  }
}

// F = q_i H from the tiles on and above the diagonal after symmetric iterations (the
// tiles below it are stale): one block per tile pair, the tile (J, I) written as the
// transpose of (I, J) through shared memory. q_i = s_i / Omega_i (row_quotients).
template <int T>
__global__ void __launch_bounds__(kThreads) from_exchange_sym(double* __restrict__ H, const double* __restrict__ q,
                                                              int32_t n, int32_t n_tiles,
                                                              const uint8_t* __restrict__ tile_nz) {
  __shared__ double X[T][T + 1];
  __shared__ double qI[T], qJ[T];
  const int64_t ld = n + 1;
  // a zero pair's tiles hold zeros, which q_i H leaves as they are
  for (PairWalker w(blockIdx.x, n_tiles); w.skip_zero(tile_nz, gridDim.x), w.valid(); w.advance(gridDim.x)) {
    const int I = w.I, J = w.J();
    load_tile<T>(H, n, I, J, X);
    if (threadIdx.x < 2 * T) {
      const int t = threadIdx.x & (T - 1);
      const int64_t i = (int64_t)(threadIdx.x < T ? I : J) * T + t;
      (threadIdx.x < T ? qI : qJ)[t] = i < n ? q[i] : 0.0;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int e = threadIdx.x; e < T * T; e += kThreads) {
      const int r = e / T, c = e % T;
      const int64_t i = (int64_t)I * T + r, j = (int64_t)J * T + c;
      if (i < n && j < n) H[i * ld + j] = qI[r] * X[r][c];
    }
    if (I != J) {
      for (int e = threadIdx.x; e < T * T; e += kThreads) {
        const int r = e / T, c = e % T;
        const int64_t i = (int64_t)J * T + r, j = (int64_t)I * T + c;
        if (i < n && j < n) H[i * ld + j] = qJ[r] * X[c][r];
      }
    }
    __syncthreads();
  }
}

// Failure-detection check of the grid barrier: every block but block 0 waits at a barrier
// that block 0 never reaches, so the wait runs out after limit_ns and sets st->timeout.
__global__ void barrier_timeout_probe(PersistState* st, unsigned long long limit_ns) {
  __shared__ int s_ok;
  if (blockIdx.x == 0) return;
  grid_barrier(st, &s_ok, limit_ns);
}

// kappa_ij (rg_kappa): matrix triangulation (Eq. 3.21-3.22) or fractional variance
// (Eq. 3.23-3.25). *bad is raised for a non-positive ray count or Omega.
__global__ void kappa_kernel(int32_t mode, const double* __restrict__ F, const long long* __restrict__ rays,
                             const double* __restrict__ omega, double param, int32_t n, double* __restrict__ K,
                             int* bad) {
  const int64_t total = (int64_t)n * n;
  const int64_t ld = n + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    const double Ni = (double)rays[i], Nj = (double)rays[j], oi = omega[i], oj = omega[j];
    if (!(Ni > 0.0 && Nj > 0.0 && oi > 0.0 && oj > 0.0)) {
      atomicExch(bad, 1);
      K[e] = 0.5;
      continue;
    }
    double k = 0.5;
    if (i != j) {
      if (mode == RG_KAPPA_TRIANGULATION) {
        const double ri = oi / Ni, rj = oj / Nj;
        const double Y = (rj - ri) / (rj + ri);
        const double sg = Y > 0.0 ? 1.0 : (Y < 0.0 ? -1.0 : 0.0);
        k = 0.5 * (1.0 + sg * pow(fabs(Y), param));
      } else {
        const double fij = F[i * ld + j], fji = F[j * ld + i];
        const double zz = param * param;
        const bool zi = !(fij > 0.0), zj = !(fji > 0.0);
        if (zi && zj) {
          k = 0.5;
        } else if (zi) {
          k = 0.0;
        } else if (zj) {
          k = 1.0;
        } else {
          const double vij = zz * oi * oi * (1.0 - fij) / (Ni * fij);
          const double vji = zz * oj * oj * (1.0 - fji) / (Nj * fji);
          k = vji / (vij + vji);
        }
      }
    }
    K[e] = k;
  }
}

__global__ void __launch_bounds__(kThreads) row_pass(double* __restrict__ H, double* __restrict__ s,
                                                     const double* __restrict__ omega, const double* __restrict__ P,
                                                     int32_t n, int32_t n_tiles, EnforceState* st, double tol_abs,
                                                     int32_t maxit) {
  if (st->done) return;
  __shared__ double red[kThreads];
  __shared__ int s_last;
  const int64_t ld = n + 1;
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  double dc = 0.0;
  bool bad = false;
  if (i < n) {
    double env = s[i] * H[i * ld + n];
    H[i * ld + n] = env;
    double r = 0.0;
    for (int J = 0; J < n_tiles; ++J) r += P[i * n_tiles + J];
    r += env;
    dc = fabs(r - omega[i]);
    s[i] = (r > 0.0) ? omega[i] / r : 1.0;
    bad = !isfinite(r);
  }
  red[threadIdx.x] = dc;
  if (bad) st->done = 3;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicMax(&st->d_close, (unsigned long long)__double_as_longlong(red[0]));
    __threadfence();
    s_last = (atomicAdd(&st->blocks_seen, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    volatile EnforceState* v = st;
    double dr = __longlong_as_double((long long)v->d_recip);
    double dcl = __longlong_as_double((long long)v->d_close);
    int it = v->iters + 1;
    v->iters = it;
    if (v->done == 0) {
      if (fmax(dr, dcl) <= tol_abs) v->done = 1;
      else if (it >= maxit) v->done = 2;
    }
    v->d_recip = 0ull;
    v->d_close = 0ull;
    v->blocks_seen = 0;
  }
}

__global__ void max_kernel(const double* __restrict__ x, int32_t n, unsigned long long* out) {
  __shared__ double red[kThreads];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) m = fmax(m, fabs(x[i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (unsigned long long)__double_as_longlong(red[0]);
}

// ---------------------------------------------------------------- aggregation
__global__ void group_area_kernel(const double* __restrict__ S, const int32_t* __restrict__ g, int32_t n_sub,
                                  double* __restrict__ Sg, int32_t n_group, int32_t* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_sub; i += gridDim.x * blockDim.x) {
    int32_t k = g[i];
    if (k < 0 || k >= n_group) { atomicExch(err, 1); continue; }
    atomicAdd(&Sg[k], S[i]);
  }
}

// One block per sub-surface row i: T[m] = sum_{j in group m} F_ij (shared memory), then
// out[g(i)][m] += T[m] * S_i / S_g(i).
__global__ void __launch_bounds__(kThreads) aggregate_rows(const double* __restrict__ F, const double* __restrict__ S,
                                                           const int32_t* __restrict__ g, int32_t n_sub,
                                                           const double* __restrict__ Sg, int32_t n_group,
                                                           double* __restrict__ out) {
  extern __shared__ double acc[];
  const int cols = n_group + 1;
  const int64_t ld = n_sub + 1;
  for (int i = blockIdx.x; i < n_sub; i += gridDim.x) {
    for (int m = threadIdx.x; m < cols; m += kThreads) acc[m] = 0.0;
    __syncthreads();
    for (int j = threadIdx.x; j <= n_sub; j += kThreads) {
      int m = (j == n_sub) ? n_group : g[j];
      if ((unsigned)m > (unsigned)n_group) continue;  // reported by group_area_kernel
      double f = F[i * ld + j];
      if (f != 0.0) atomicAdd(&acc[m], f);
    }
    __syncthreads();
    const int gi = g[i];
    if ((unsigned)gi < (unsigned)n_group) {
      const double w = S[i] / Sg[gi];
      for (int m = threadIdx.x; m < cols; m += kThreads)
        if (acc[m] != 0.0) atomicAdd(&out[(int64_t)gi * cols + m], acc[m] * w);
    }
    __syncthreads();
  }
}

inline int blocks_for(int64_t total, int sm) {
  int64_t b = (total + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sm * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

extern "C" {

rg_status rg_counts_to_F(rg_ctx* ctx, int32_t n, const int64_t* counts_d, const int64_t* rays_d, double* F_d,
                         void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n > 0 && counts_d && rays_d && F_d, "rg_counts_to_F: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  int64_t total = (int64_t)n * (n + 1);
  counts_to_F_kernel<<<blocks_for(total, ctx->sm_count), kThreads, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const long long*>(counts_d), reinterpret_cast<const long long*>(rays_d), F_d, n, total);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  return RG_OK;
}

}  // extern "C"

namespace {

rg_status enforce_iterative(rg_ctx* ctx, int32_t n, const double* omega_d, const double* kappa_d, double* F_d,
                            double tol, int32_t maxit, int32_t* iters_out_h, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n > 0 && omega_d && F_d && maxit > 0 && tol >= 0.0, "rg_enforce_iterative: bad argument");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int tile = tile_edge(n);
  const int n_tiles = (n + tile - 1) / tile;
  rg::Sizer sz;
  sz.take<double>(n);                          // s
  sz.take<double>((size_t)n_tiles * n);        // P
  sz.take<EnforceState>(1);
  sz.take<PersistState>(1);
  sz.take<float2>(2 * (size_t)n);              // fp32 splits of s / 2, two iterations
  sz.take<int>(n);                             // row-sum bound exponents
  sz.take<uint8_t>((size_t)n_tiles * (n_tiles + 1) / 2);  // non-zero tile pairs
  void* ws = nullptr;
  rg_status rs = rg::workspace(ctx, sz.off, &ws);
  if (rs != RG_OK) return rs;
  rg::Carver cv(ws);
  double* sc = cv.take<double>(n);
  double* P = cv.take<double>((size_t)n_tiles * n);
  EnforceState* st = cv.take<EnforceState>(1);
  PersistState* pst = cv.take<PersistState>(1);
  float2* hsplit = cv.take<float2>(2 * (size_t)n);
  int* eR = cv.take<int>(n);
  uint8_t* tile_nz = cv.take<uint8_t>((size_t)n_tiles * (n_tiles + 1) / 2);
  const int64_t total = (int64_t)n * (n + 1);
  RG_CUDA_TRY(ctx, cudaMemsetAsync(st, 0, sizeof(EnforceState), s));
  // tolerance scale: max Omega
  max_kernel<<<1, kThreads, 0, s>>>(omega_d, n, reinterpret_cast<unsigned long long*>(ctx->d_scratch));
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, ctx->d_scratch, 8, cudaMemcpyDeviceToHost, s));
  to_exchange_kernel<<<blocks_for(total, ctx->sm_count), kThreads, 0, s>>>(F_d, omega_d, sc, n, total);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  double om_max;
  memcpy(&om_max, ctx->h_scratch, 8);
  const double tol_abs = tol * om_max;
  const int eoff = (om_max > 0.0 && std::isfinite(om_max)) ? std::ilogb(om_max) : 0;
  dim3 sym_grid(n_tiles, n_tiles);
  const int row_blocks = (n + kThreads - 1) / kThreads;
  EnforceState h{};
  // one cooperative launch for all iterations (the two-kernel loop below is the same
  // computation, kept for devices without cooperative launches)
  int coop = 0;
  bool sym = false;
  RG_CUDA_TRY(ctx, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  if (coop) {
    void (*kern)(double*, double*, float2*, int*, const double*, const double*, int32_t, int32_t, double*,
                 PersistState*, double, int32_t, int, uint8_t*);
    if (tile == kTSmall) kern = kappa_d ? enforce_persistent<kTSmall, true> : enforce_persistent<kTSmall, false>;
    else kern = kappa_d ? enforce_persistent<kT, true> : enforce_persistent<kT, false>;
    int per_sm = 0;
    RG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
    const int n_pairs = n_tiles * (n_tiles + 1) / 2;
    const int grid = std::max(1, std::min(n_pairs, per_sm * ctx->sm_count));
    RG_CUDA_TRY(ctx, cudaMemsetAsync(pst, 0, sizeof(PersistState), s));
    int32_t nn = n, nt = n_tiles, mi = maxit;
    int eo = eoff;
    double ta = tol_abs;
    double* Fp = F_d;
    const double* kp = kappa_d;
    const double* op = omega_d;
    void* args[] = {&Fp, &sc, &hsplit, &eR, &kp, &op, &nn, &nt, &P, &pst, &ta, &mi, &eo, &tile_nz};
    const int tok = rg::timer_begin(ctx, rg::kTimeEnforce, s);
    RG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kThreads), args, 0, s));
    rg::timer_end(ctx, tok, s);
    ++ctx->launches;
    PersistState hp{};
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(&hp, pst, sizeof(PersistState), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hp.timeout) return rg::fail(ctx, RG_ERR_CUDA, "rg_enforce_iterative: a grid barrier timed out");
    if (hp.range)
      return rg::fail(ctx, RG_ERR_NUMERIC, "rg_enforce_iterative: a fixed-point row-sum term left its bound");
    h.done = hp.done;
    h.iters = hp.iters;
    sym = hp.sym != 0;
  }
  for (int launched = 0; !coop && launched < maxit;) {
    int batch = std::min(8, maxit - launched);
    for (int b = 0; b < batch; ++b) {
      if (tile == kTSmall) {
        if (kappa_d) sym_pass<kTSmall, true><<<sym_grid, kThreads, 0, s>>>(F_d, sc, kappa_d, n, P, st);
        else sym_pass<kTSmall, false><<<sym_grid, kThreads, 0, s>>>(F_d, sc, nullptr, n, P, st);
      } else {
        if (kappa_d) sym_pass<kT, true><<<sym_grid, kThreads, 0, s>>>(F_d, sc, kappa_d, n, P, st);
        else sym_pass<kT, false><<<sym_grid, kThreads, 0, s>>>(F_d, sc, nullptr, n, P, st);
      }
      ++ctx->launches;
      row_pass<<<row_blocks, kThreads, 0, s>>>(F_d, sc, omega_d, P, n, n_tiles, st, tol_abs, maxit);
      ++ctx->launches;
    }
    launched += batch;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, st, sizeof(EnforceState), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (h.done) break;
  }
  row_quotients<<<blocks_for(n, ctx->sm_count), kThreads, 0, s>>>(F_d, omega_d, sc, n);
  ++ctx->launches;
  if (sym) {
    const int n_pairs = n_tiles * (n_tiles + 1) / 2;
    const int grid = std::min(n_pairs, 4 * ctx->sm_count);
    if (tile == kTSmall) from_exchange_sym<kTSmall><<<grid, kThreads, 0, s>>>(F_d, sc, n, n_tiles, tile_nz);
    else from_exchange_sym<kT><<<grid, kThreads, 0, s>>>(F_d, sc, n, n_tiles, tile_nz);
  } else {
    from_exchange_kernel<<<blocks_for((int64_t)n * n, ctx->sm_count), kThreads, 0, s>>>(F_d, sc, n, (int64_t)n * n);
  }
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  if (iters_out_h) *iters_out_h = h.iters;
  if (h.done == 3) return rg::fail(ctx, RG_ERR_NUMERIC, "rg_enforce_iterative: non-finite row sum");
  if (h.done != 1) return rg::fail(ctx, RG_ERR_NOT_CONVERGED, "rg_enforce_iterative: no convergence in %d iterations", maxit);
  return RG_OK;
}

}  // namespace

extern "C" {

rg_status rg_enforce_iterative(rg_ctx* ctx, int32_t n, const double* omega_d, double* F_d, double tol, int32_t maxit,
                               int32_t* iters_out_h, void* stream) {
  return enforce_iterative(ctx, n, omega_d, nullptr, F_d, tol, maxit, iters_out_h, stream);
}

rg_status rg_enforce_iterative_kappa(rg_ctx* ctx, int32_t n, const double* omega_d, const double* kappa_d,
                                     double* F_d, double tol, int32_t maxit, int32_t* iters_out_h, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, kappa_d != nullptr, "rg_enforce_iterative_kappa: NULL kappa");
  return enforce_iterative(ctx, n, omega_d, kappa_d, F_d, tol, maxit, iters_out_h, stream);
}

rg_status rg_debug_barrier_timeout(rg_ctx* ctx, double limit_s, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, limit_s > 0.0 && limit_s <= 2.0, "rg_debug_wait_timeout: limit %.3g s outside (0, 2]", limit_s);
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  rg_status rs = rg::workspace(ctx, sizeof(PersistState), &ws);
  if (rs != RG_OK) return rs;
  PersistState* st = static_cast<PersistState*>(ws);
  RG_CUDA_TRY(ctx, cudaMemsetAsync(st, 0, sizeof(PersistState), s));
  unsigned long long lim = (unsigned long long)(limit_s * 1e9);
  void* args[] = {&st, &lim};
  // two co-resident blocks (a cooperative launch): block 1 waits for block 0, which returns
  RG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)barrier_timeout_probe, dim3(2), dim3(32), args, 0, s));
  ++ctx->launches;
  PersistState h{};
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, st, sizeof(PersistState), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h.timeout) return rg::fail(ctx, RG_ERR_CUDA, "grid barrier timed out after %.3g s", limit_s);
  return RG_OK;
}

rg_status rg_kappa(rg_ctx* ctx, int32_t n, int32_t mode, const double* F_d, const int64_t* rays_d,
                   const double* omega_d, double param, double* kappa_d, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n > 0 && rays_d && omega_d && kappa_d, "rg_kappa: bad argument");
  RG_ARG_CHECK(ctx, mode == RG_KAPPA_TRIANGULATION || (mode == RG_KAPPA_FRACTIONAL_VARIANCE && F_d),
               "rg_kappa: unknown mode %d (or NULL F for fractional variance)", mode);
  RG_ARG_CHECK(ctx, std::isfinite(param) && param > 0.0, "rg_kappa: parameter %.3e must be positive", param);
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch, 0, sizeof(int32_t), s));
  kappa_kernel<<<blocks_for((int64_t)n * n, ctx->sm_count), kThreads, 0, s>>>(
      mode, F_d, reinterpret_cast<const long long*>(rays_d), omega_d, param, n, kappa_d, ctx->d_scratch);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, ctx->d_scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (ctx->h_scratch[0]) return rg::fail(ctx, RG_ERR_ARG, "rg_kappa: a ray count or Omega is not positive");
  return RG_OK;
}

rg_status rg_aggregate(rg_ctx* ctx, int32_t n_sub, const double* F_sub_d, const double* sub_area_d,
                       const int32_t* sub_group_d, int32_t n_group, double* F_group_d, double* group_area_d,
                       void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, n_sub > 0 && n_group > 0 && F_sub_d && sub_area_d && sub_group_d && F_group_d,
               "rg_aggregate: bad argument");
  const size_t smem = (size_t)(n_group + 1) * sizeof(double);
  RG_ARG_CHECK(ctx, (int)smem <= ctx->smem_optin - 1024, "rg_aggregate: too many groups (%d)", n_group);
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  rg_status rs = rg::workspace(ctx, (size_t)n_group * sizeof(double), &ws);
  if (rs != RG_OK) return rs;
  double* Sg = group_area_d ? group_area_d : static_cast<double*>(ws);
  RG_CUDA_TRY(ctx, cudaMemsetAsync(Sg, 0, (size_t)n_group * sizeof(double), s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(F_group_d, 0, (size_t)n_group * (n_group + 1) * sizeof(double), s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch, 0, sizeof(int32_t), s));
  group_area_kernel<<<blocks_for(n_sub, ctx->sm_count), kThreads, 0, s>>>(sub_area_d, sub_group_d, n_sub, Sg, n_group,
                                                                         ctx->d_scratch);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaFuncSetAttribute(aggregate_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int grid = std::min(n_sub, ctx->sm_count * 4);
  aggregate_rows<<<grid, kThreads, smem, s>>>(F_sub_d, sub_area_d, sub_group_d, n_sub, Sg, n_group, F_group_d);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, ctx->d_scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (ctx->h_scratch[0]) return rg::fail(ctx, RG_ERR_ARG, "rg_aggregate: group index out of range");
  return RG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free variant
// The iterative enforcer for callers that may not allocate device memory at call time:
// the same kernels as rg_enforce_iterative, with their scratch in this file-scope
// device array instead of the context workspace. Every GPU that loads the library holds
// the array until the process exits.
namespace {

constexpr int32_t kNoallocMaxN = 4096;
constexpr int32_t kNoallocMaxTiles = (kNoallocMaxN + kT - 1) / kT;
constexpr size_t kNoallocScaleBytes = (size_t)kNoallocMaxN * sizeof(double);
constexpr size_t kNoallocRowSumBytes = (size_t)kNoallocMaxTiles * kNoallocMaxN * sizeof(double);
constexpr size_t kNoallocBytes = kNoallocScaleBytes + kNoallocRowSumBytes + 256 + 256;

// Layout: [row scales s: N doubles][per-tile row sums: N x tiles doubles]
//         [EnforceState, 256 B][tolerance scale max|Omega|, 256 B]
static __device__ __align__(256) unsigned char g_enforce_scratch[kNoallocBytes];

// Device address of g_enforce_scratch on the current device. Looked up on every call (the
// lookup is cheap next to the call's synchronisations), so that no address outlives the
// context it was taken in.
cudaError_t scratch_address(void** out) { return cudaGetSymbolAddress(out, g_enforce_scratch); }

}  // namespace

extern "C" rg_status rg_enforce_iterative_noalloc(int32_t n, const double* omega_d, double* F_d, double tol,
                                                  int32_t maxit, int32_t* iters_out_h, void* stream) {
  if (n <= 0 || !omega_d || !F_d || maxit <= 0 || !(tol >= 0.0)) return RG_ERR_ARG;
  if (n > kNoallocMaxN) return RG_ERR_UNSUPPORTED;  // the static scratch holds N <= 4096
  // an error the caller's own earlier work left pending is reported, not consumed: the
  // checks below would otherwise take it for one of this call's launches
  if (cudaPeekAtLastError() != cudaSuccess) return RG_ERR_CUDA;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return RG_ERR_CUDA;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return RG_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  char* b = static_cast<char*>(base);
  double* sc = reinterpret_cast<double*>(b);
  double* P = reinterpret_cast<double*>(b + kNoallocScaleBytes);
  EnforceState* st = reinterpret_cast<EnforceState*>(b + kNoallocScaleBytes + kNoallocRowSumBytes);
  unsigned long long* om_max = reinterpret_cast<unsigned long long*>(b + kNoallocScaleBytes + kNoallocRowSumBytes + 256);
  const int tile = tile_edge(n);  // n_tiles * n <= kNoallocMaxTiles * kNoallocMaxN either way
  const int n_tiles = (n + tile - 1) / tile;
  const int64_t total = (int64_t)n * (n + 1);
  int sm = 0;
  if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return RG_ERR_CUDA;
  // the state keeps the previous call's contents: clear it
  if (cudaMemsetAsync(st, 0, sizeof(EnforceState), s) != cudaSuccess) return RG_ERR_CUDA;
  max_kernel<<<1, kThreads, 0, s>>>(omega_d, n, om_max);
  to_exchange_kernel<<<blocks_for(total, sm), kThreads, 0, s>>>(F_d, omega_d, sc, n, total);
  if (cudaGetLastError() != cudaSuccess) return RG_ERR_CUDA;
  unsigned long long om_bits = 0;
  if (cudaMemcpyAsync(&om_bits, om_max, sizeof(om_bits), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RG_ERR_CUDA;
  double om;
  memcpy(&om, &om_bits, sizeof(om));
  const double tol_abs = tol * om;
  dim3 sym_grid(n_tiles, n_tiles);
  const int row_blocks = (n + kThreads - 1) / kThreads;
  EnforceState h{};
  for (int launched = 0; launched < maxit;) {
    int batch = std::min(8, maxit - launched);
    for (int k = 0; k < batch; ++k) {
      if (tile == kTSmall) sym_pass<kTSmall, false><<<sym_grid, kThreads, 0, s>>>(F_d, sc, nullptr, n, P, st);
      else sym_pass<kT, false><<<sym_grid, kThreads, 0, s>>>(F_d, sc, nullptr, n, P, st);
      row_pass<<<row_blocks, kThreads, 0, s>>>(F_d, sc, omega_d, P, n, n_tiles, st, tol_abs, maxit);
    }
    launched += batch;
    if (cudaGetLastError() != cudaSuccess) return RG_ERR_CUDA;
    if (cudaMemcpyAsync(&h, st, sizeof(EnforceState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return RG_ERR_CUDA;
    if (h.done) break;
  }
  row_quotients<<<blocks_for(n, sm), kThreads, 0, s>>>(F_d, omega_d, sc, n);
  from_exchange_kernel<<<blocks_for((int64_t)n * n, sm), kThreads, 0, s>>>(F_d, sc, n, (int64_t)n * n);
  if (cudaGetLastError() != cudaSuccess) return RG_ERR_CUDA;
  if (iters_out_h) *iters_out_h = h.iters;
  if (h.done == 3) return RG_ERR_NUMERIC;
  if (h.done != 1) return RG_ERR_NOT_CONVERGED;
  return RG_OK;
}

