// Monte Carlo ray tracing of view factors (Sec. 3.5.1, Eq. 3.15) on sm_103a.
//
// One persistent kernel: each block repeatedly takes a work item (one face, a range
// of its rays) and keeps a shared-memory tally row of N+1 16-bit counters for that face. The
// warps of the block share the item's rays through a counter. Two schedules (chosen per
// mesh, identical counts):
//   lock-step (shallow BVHs): the warp samples 32 rays in step, gives each one root
//     visit, tallies the rays already finished (most rays leaving the scene) and queues
//     the rest; queued rays are traced to completion 32 at a time;
//   refill (deep BVHs): each warp runs one warp-synchronous loop whose iteration is one
//     BVH node visit per lane (child-box slab tests, Moller-Trumbore tests of leaf
//     triangles, stack push/pop). Lanes whose ray is finished wait until 24 of the 32
//     lanes are; then their rays go to the tally row
// (aggregated per target face) and they take new rays from a private 64-ray ring in
// shared memory, which the whole warp refills 32 rays at a time, in step, when it runs
// short (one Philox4x32-10 draw per ray: area-CDF triangle choice, uniform point lifted
// off the face, cosine-weighted direction). Sampling thus stays convergent and lanes do
// not wait for the slowest ray of their warp. At the end of an item the non-zero
// counters are flushed to the int64 count matrix in HBM. The closest
// hit is the smallest (t > 0, triangle index), so the counts do not depend on the order
// in which rays are traced.
//
// Side-resolved variant (two-sided faces, Sec. 5.2.4-5.2.5): work item rows are the
// sides 2f+X of the faces (X = 0: side A, the side the face normal points to; 1: side B),
// side B emits with the frame (t, -b, -n) and counter word 2 = f + 2^31, and a hit counts
// for column 2g+Y with Y = 0 when the Moller-Trumbore determinant is positive (the ray
// runs against the triangle normal) and 1 otherwise; column 2N is the environment.
//
// kExact = true rounds every float operation of sampling and intersection on its
// own (no fused multiply-add), which makes the counts bit-identical to any other
// implementation of the same ray definition that does the same.
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "mesh.cuh"

// Resident blocks per SM the two schedules are compiled for (register caps: 3 blocks of
// 256 threads allow 85 registers, 4 allow 64). Measured on GB300: the lock-step kernel
// runs 2.6 % faster with 3 (no spills), the refill kernel 3 % faster with 4.
#ifndef RG_LOCKSTEP_MIN_BLOCKS
#define RG_LOCKSTEP_MIN_BLOCKS 3
#endif
#ifndef RG_REFILL_MIN_BLOCKS
#define RG_REFILL_MIN_BLOCKS 4
#endif

namespace {

struct WorkItem {
  int64_t begin;
  int32_t face;
  int32_t count;
};

struct TraceParams {
  DevMesh m;
  const WorkItem* items;
  int32_t n_items;
  int32_t* item_counter;  // next item to take (zeroed before the launch)
  int32_t* error_word;    // non-zero: a ray overflowed the traversal stack
  uint32_t key0, key1;
  uint64_t ray_offset;
  unsigned long long* counts;  // [N][N+1]
  int32_t n_bins;              // N + 1
  unsigned long long* stats;   // [3]: rays, box tests, triangle tests (statistics kernels only);
                               // [4] for the reflection kernel: rays, hits, lost, overflow
  // reflection kernel only: per-face floor(eps 2^32) and floor((eps + rho) 2^32)
  const unsigned long long* thr_absorb;
  const unsigned long long* thr_reflect;
  int32_t max_bounces;
};

template <bool kExact>
struct Ar;
template <>
struct Ar<true> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
};
template <>
struct Ar<false> {
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
};

struct V3 {
  float x, y, z;
};

template <bool E>
__device__ __forceinline__ V3 cross3(V3 a, V3 b) {
  using A = Ar<E>;
  return {A::sub(A::mul(a.y, b.z), A::mul(a.z, b.y)), A::sub(A::mul(a.z, b.x), A::mul(a.x, b.z)),
          A::sub(A::mul(a.x, b.y), A::mul(a.y, b.x))};
}
template <bool E>
__device__ __forceinline__ float dot3(V3 a, V3 b) {
  using A = Ar<E>;
  return A::add(A::add(A::mul(a.x, b.x), A::mul(a.y, b.y)), A::mul(a.z, b.z));
}

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    // one 32 x 32 -> 64-bit product gives both halves
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p2 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p2 >> 32) ^ c.y ^ k0, (uint32_t)p2, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
  }
  return c;
}

__device__ __forceinline__ float unit24(uint32_t x) { return __uint2float_rn(x >> 8) * 5.9604644775390625e-08f; }

// cos and sin of 2 pi t 2^-24 (t < 2^24): the quadrant from t's top two bits; in it the
// angle (pi/2) w 2^-22 folded to alpha = (pi/4) w' 2^-21 in [0, pi/4] (w' = w, or 2^22 - w
// with cos and sin swapped) and the Taylor polynomials of degree 9 (sin) and 10 (cos) in
// z = alpha^2, coefficients (-1)^k / (2k+1)! and (-1)^k / (2k)! rounded to float. Every
// operation rounds on its own (A = Ar<true>) in the FMA-free mode.
template <bool E>
__device__ __forceinline__ void unit_circle(uint32_t t, float* pc, float* ps) {
  using A = Ar<E>;
  const uint32_t q = t >> 22, w = t & 0x3fffffu;
  const bool swap = w >= 0x200000u;
  const float a = __uint2float_rn(swap ? 0x400000u - w : w) * 0x1p-21f;  // exact
  const float al = A::mul(a, 0x1.921fb6p-1f);                              // pi/4
  const float z = A::mul(al, al);
  float sp = 0x1.71de3ap-19f;
  sp = A::add(-0x1.a01a02p-13f, A::mul(z, sp));
  sp = A::add(0x1.111112p-7f, A::mul(z, sp));
  sp = A::add(-0x1.555556p-3f, A::mul(z, sp));
  const float sn = A::add(al, A::mul(A::mul(al, z), sp));
  float cp = -0x1.27e4fcp-22f;
  cp = A::add(0x1.a01a02p-16f, A::mul(z, cp));
  cp = A::add(-0x1.6c16c2p-10f, A::mul(z, cp));
  cp = A::add(0x1.555556p-5f, A::mul(z, cp));
  cp = A::add(-0.5f, A::mul(z, cp));
  const float cs = A::add(1.0f, A::mul(z, cp));
  const float c = swap ? sn : cs, s = swap ? cs : sn;  // cos, sin of the angle in the quadrant
  *pc = q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
  *ps = q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
}

// Every quantity is computed whatever the outcome and the hit is one predicate at the
// end: the lanes of a warp testing different triangles then stay converged (a miss found
// early saves no warp instruction while another lane still tests). The arithmetic is
// that of the early-exit form, so the hits are the same; det = 0 gives inv = inf and
// NaN or infinite u, v, t, which fail their tests.
template <bool E>
__device__ __forceinline__ bool moller_trumbore(const float4 r0, const float4 r1, const float4 r2, V3 o, V3 d,
                                                float* t_out, float* det_out) {
  using A = Ar<E>;
  const float lo = -9.5367431640625e-07f, hi = 1.00000095367431640625f;  // -2^-20, 1 + 2^-20
  V3 v0{r0.x, r0.y, r0.z}, e1{r0.w, r1.x, r1.y}, e2{r1.z, r1.w, r2.x};
  V3 p = cross3<E>(d, e2);
  const float det = dot3<E>(e1, p);
  const float inv = __frcp_rn(det);
  V3 tv{A::sub(o.x, v0.x), A::sub(o.y, v0.y), A::sub(o.z, v0.z)};
  const float u = A::mul(dot3<E>(tv, p), inv);
  V3 q = cross3<E>(tv, e1);
  const float v = A::mul(dot3<E>(d, q), inv);
  const float t = A::mul(dot3<E>(e2, q), inv);
  *t_out = t;
  *det_out = det;
  return det != 0.0f && u >= lo && u <= hi && v >= lo && A::add(u, v) <= hi && t > 0.0f;
}

struct NoStats {
  __device__ __forceinline__ void box(int) {}
  __device__ __forceinline__ void tri() {}
};
struct Stats {
  unsigned long long n_box = 0, n_tri = 0;
  __device__ __forceinline__ void box(int k) { n_box += k; }
  __device__ __forceinline__ void tri() { ++n_tri; }
};

// S (side-resolved): best_face receives the tally column 2 * face + side instead of the face.
template <bool E, bool S>
__device__ __forceinline__ void test_record(const float4* __restrict__ rec, int32_t src, V3 o, V3 d, float& best_t,
                                            int32_t& best_id, int32_t& best_face) {
  float4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
  int32_t id = __float_as_int(r2.y);
  float t, det;
  const bool hit = moller_trumbore<E>(r0, r1, r2, o, d, &t, &det) && id != src;
  if (hit && (t < best_t || (t == best_t && id < best_id))) {
    best_t = t;
    best_id = id;
    const int32_t face = __float_as_int(r2.z);
    best_face = S ? 2 * face + (det > 0.0f ? 0 : 1) : face;
  }
}

// Reciprocal of a direction component for the slab tests t = box * (1/d) - o * (1/d).
// The boxes are padded far beyond the error of the approximate reciprocal. Components
// are kept at least 1e-30 in magnitude so that 1/d stays finite: with 1/d = inf the fused
// form would give fma(box, inf, -inf) = NaN on one side of the slab and -inf on the
// other, and cull a box the ray lies in (a component is exactly 0 for about one ray in
// 2^24).
__device__ __forceinline__ float rcp_approx(float x) {
  x = fabsf(x) < 1e-30f ? copysignf(1e-30f, x) : x;
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Three-input min / max (one instruction each on sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Entry and exit parameters of the ray in a box given the slab parameters of its faces:
// [max(min x, min y, min z, lo), min(max x, max y, max z, hi)].
__device__ __forceinline__ void slab_window(float x0, float x1, float y0, float y1, float z0, float z1, float lo,
                                            float hi, float& tmin, float& tmax) {
  tmin = max3f(fminf(x0, x1), fminf(y0, y1), fmaxf(fminf(z0, z1), lo));
  tmax = min3f(fmaxf(x0, x1), fmaxf(y0, y1), fminf(fmaxf(z0, z1), hi));
}

// Closest hit; returns the tally column of the hit (the face, or 2 face + side when S)
// or `env`. Sets *overflow on a traversal stack overflow.
template <bool E, bool kBVH, bool S, class St>
__device__ int32_t closest_face(const DevMesh& m, int32_t src, V3 o, V3 d, bool* overflow, St& st, int32_t env) {
  float best_t = __int_as_float(0x7f800000);
  int32_t best_id = INT_MAX, best_face = env;
  if (!kBVH) {
    for (int64_t k = 0; k < m.nt; ++k) {
      test_record<E, S>(m.tris + 3 * k, src, o, d, best_t, best_id, best_face);
      st.tri();
    }
    return best_face;
  }
  // slab tests in the form t = box * (1/d) - o/d; the boxes are padded far beyond the
  // rounding of this form, so it needs neither IEEE reciprocals nor separate roundings
  const float ix = rcp_approx(d.x), iy = rcp_approx(d.y), iz = rcp_approx(d.z);
  const float ox = o.x * ix, oy = o.y * iy, oz = o.z * iz;
  int32_t stack[kTraceStack];
  int sp = 0;
  int32_t node = 0;
  while (true) {
    const float4* nd = m.nodes + 4 * node;
    float4 a = __ldg(nd), b = __ldg(nd + 1), c = __ldg(nd + 2), w = __ldg(nd + 3);
    int32_t refL = __float_as_int(w.x), refR = __float_as_int(w.y);
    int32_t cntL = __float_as_int(w.z), cntR = __float_as_int(w.w);
    float limit = best_t + m.slack;
    float lmin, lmax, rmin, rmax;
    slab_window(fmaf(a.x, ix, -ox), fmaf(a.y, ix, -ox), fmaf(a.z, iy, -oy), fmaf(a.w, iy, -oy), fmaf(c.x, iz, -oz),
                fmaf(c.y, iz, -oz), m.t_lo, limit, lmin, lmax);
    slab_window(fmaf(b.x, ix, -ox), fmaf(b.y, ix, -ox), fmaf(b.z, iy, -oy), fmaf(b.w, iy, -oy), fmaf(c.z, iz, -oz),
                fmaf(c.w, iz, -oz), m.t_lo, limit, rmin, rmax);
    bool hl = lmin <= lmax, hr = rmin <= rmax;
    st.box(2);
    if (hl && cntL > 0) {
      for (int q = 0; q < cntL; ++q) {
        test_record<E, S>(m.tris + 3 * (int64_t)(refL + q), src, o, d, best_t, best_id, best_face);
        st.tri();
      }
      hl = false;
    }
    if (hr && cntR > 0) {
      for (int q = 0; q < cntR; ++q) {
        test_record<E, S>(m.tris + 3 * (int64_t)(refR + q), src, o, d, best_t, best_id, best_face);
        st.tri();
      }
      hr = false;
    }
    if (hl && hr) {
      bool left_first = lmin <= rmin;
      if (sp >= kTraceStack) { *overflow = true; break; }
      stack[sp++] = left_first ? refR : refL;
      node = left_first ? refL : refR;
    } else if (hl) {
      node = refL;
    } else if (hr) {
      node = refR;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  return best_face;
}

// Emission from `face` with the one draw of counter (ray lo, ray hi, stream, base):
// triangle, point and direction. Emission proper uses stream = face and base = 0; the
// reflection of bounce b of a path from face i uses stream = i and base = 128 b
// (re-emission from the hit face). side_b: emission from side B, with the frame
// (t, -b, -n) (stream = face + 2^31).
template <bool E>
__device__ __forceinline__ void sample_ray(const DevMesh& m, uint32_t k0, uint32_t k1, uint64_t ray, int32_t face,
                                           V3* o, V3* d, int32_t* src, uint32_t stream, uint32_t base,
                                           bool side_b = false) {
  using A = Ar<E>;
  const uint32_t rlo = (uint32_t)ray, rhi = (uint32_t)(ray >> 32);
  uint4 x = philox(make_uint4(rlo, rhi, stream, base), k0, k1);
  // first record whose threshold exceeds x.x (thresholds are non-decreasing; meshes
  // have fewer than 2^30 triangles)
  int32_t a = (int32_t)m.face_start[face], b = (int32_t)m.face_start[face + 1] - 1;
  while (a < b) {
    const int32_t mid = (a + b) >> 1;
    if (x.x < __ldg(m.ethr + mid)) b = mid; else a = mid + 1;
  }
  const float4* rec = m.etris + 3 * (int64_t)a;
  float4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
  *src = __float_as_int(r2.y);
  float u = unit24(x.y), v = unit24(x.z);
  if (A::add(u, v) > 1.0f) {
    u = A::sub(1.0f, u);
    v = A::sub(1.0f, v);
  }
  // pull (u, v) toward the centroid by 2^-20 so that no origin lies on an edge
  u = A::add(A::mul(u, 0x1.ffffep-1f), 0x1.555556p-22f);
  v = A::add(A::mul(v, 0x1.ffffep-1f), 0x1.555556p-22f);
  const float* fr = m.frames + 9 * (int64_t)face;
  float tx = __ldg(fr), ty = __ldg(fr + 1), tz = __ldg(fr + 2), bx = __ldg(fr + 3), by = __ldg(fr + 4),
        bz = __ldg(fr + 5), nx = __ldg(fr + 6), ny = __ldg(fr + 7), nz = __ldg(fr + 8);
  if (side_b) {
    bx = -bx; by = -by; bz = -bz;
    nx = -nx; ny = -ny; nz = -nz;
  }
  // point on the triangle, lifted off the face along its normal
  o->x = A::add(A::add(A::add(r0.x, A::mul(u, r0.w)), A::mul(v, r1.z)), A::mul(m.lift, nx));
  o->y = A::add(A::add(A::add(r0.y, A::mul(u, r1.x)), A::mul(v, r1.w)), A::mul(m.lift, ny));
  o->z = A::add(A::add(A::add(r0.z, A::mul(u, r1.y)), A::mul(v, r2.x)), A::mul(m.lift, nz));
  // cosine-weighted direction from the same draw, no rejection: the unit-disc point at
  // radius sqrt(s), angle 2 pi (x.w >> 8) 2^-24, lifted to the hemisphere; s takes 24
  // bits from the low bytes of words 3, 1, 2 (the point used the top 24 bits of 1, 2)
  const float s2 = unit24(((x.w & 0xffu) << 24) | ((x.y & 0xffu) << 16) | ((x.z & 0xffu) << 8));
  float cph, sph;
  unit_circle<E>(x.w >> 8, &cph, &sph);
  const float rad = __fsqrt_rn(s2);
  const float dx = A::mul(rad, cph), dy = A::mul(rad, sph);
  const float dz = __fsqrt_rn(A::sub(1.0f, s2));
  d->x = A::add(A::add(A::mul(dx, tx), A::mul(dy, bx)), A::mul(dz, nx));
  d->y = A::add(A::add(A::mul(dx, ty), A::mul(dy, by)), A::mul(dz, ny));
  d->z = A::add(A::add(A::mul(dx, tz), A::mul(dy, bz)), A::mul(dz, nz));
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRing = 64;         // rays per warp ring (two sampling rounds)
#ifndef RG_REFILL_LANES
#define RG_REFILL_LANES 24
#endif
constexpr int kRefillLanes = RG_REFILL_LANES;  // finished lanes of a warp that trigger a refill

struct Ring {  // one warp's sampled rays, structure of arrays in shared memory
  float ox[kRing], oy[kRing], oz[kRing], dx[kRing], dy[kRing], dz[kRing];
  int32_t src[kRing];
};

struct Walker {
  V3 o, d;
  float ix, iy, iz;
  int32_t src;
  float best_t;
  int32_t best_id, best_face;
  int32_t node;
  int sp;
};

// One BVH node visit. Returns false once the ray's traversal is complete.
template <bool E, bool S, class St>
__device__ __forceinline__ bool visit(const DevMesh& m, Walker& w, int32_t* stack, bool* overflow, St& st) {
  const float4* nd = m.nodes + 4 * w.node;
  const float4 a = __ldg(nd), b = __ldg(nd + 1), c = __ldg(nd + 2), q = __ldg(nd + 3);
  const int32_t refL = __float_as_int(q.x), refR = __float_as_int(q.y);
  const int32_t cntL = __float_as_int(q.z), cntR = __float_as_int(q.w);
  const float limit = w.best_t + m.slack;
  const float ox = w.o.x * w.ix, oy = w.o.y * w.iy, oz = w.o.z * w.iz;
  float lmin, lmax, rmin, rmax;
  slab_window(fmaf(a.x, w.ix, -ox), fmaf(a.y, w.ix, -ox), fmaf(a.z, w.iy, -oy), fmaf(a.w, w.iy, -oy),
              fmaf(c.x, w.iz, -oz), fmaf(c.y, w.iz, -oz), m.t_lo, limit, lmin, lmax);
  slab_window(fmaf(b.x, w.ix, -ox), fmaf(b.y, w.ix, -ox), fmaf(b.z, w.iy, -oy), fmaf(b.w, w.iy, -oy),
              fmaf(c.z, w.iz, -oz), fmaf(c.w, w.iz, -oz), m.t_lo, limit, rmin, rmax);
  bool hl = lmin <= lmax, hr = rmin <= rmax;
  st.box(2);
  // the hit leaf children, tested through one loop so that lanes at different leaves
  // run the same instructions: records [r0, r0 + c0) then [r1, r1 + c1), nearer first
  const bool ll = hl && cntL > 0, lr = hr && cntR > 0;
  if (ll || lr) {  // skipped by whole warps on the inner levels
    const bool right_first = lr && (!ll || rmin < lmin);
    const int32_t r0 = right_first ? refR : refL, c0 = right_first ? (lr ? cntR : 0) : (ll ? cntL : 0);
    const int32_t r1 = right_first ? refL : refR, c1 = right_first ? (ll ? cntL : 0) : (lr ? cntR : 0);
    for (int q = 0; q < c0 + c1; ++q) {
      const int32_t rec = q < c0 ? r0 + q : r1 + (q - c0);
      test_record<E, S>(m.tris + 3 * (int64_t)rec, w.src, w.o, w.d, w.best_t, w.best_id, w.best_face);
      st.tri();
    }
    if (ll) hl = false;
    if (lr) hr = false;
  }
  if (hl && hr) {
    const bool left_first = lmin <= rmin;
    if (w.sp >= kTraceStack) { *overflow = true; return false; }
    stack[w.sp++] = left_first ? refR : refL;
    w.node = left_first ? refL : refR;
  } else if (hl) {
    w.node = refL;
  } else if (hr) {
    w.node = refR;
  } else {
    if (w.sp == 0) return false;
    w.node = stack[--w.sp];
  }
  return true;
}

__device__ __forceinline__ void start_ray(Walker& w, const Ring& r, int k, int32_t env) {
  w.o = V3{r.ox[k], r.oy[k], r.oz[k]};
  w.d = V3{r.dx[k], r.dy[k], r.dz[k]};
  w.ix = rcp_approx(w.d.x);
  w.iy = rcp_approx(w.d.y);
  w.iz = rcp_approx(w.d.z);
  w.src = r.src[k];
  w.best_t = __int_as_float(0x7f800000);
  w.best_id = INT_MAX;
  w.best_face = env;
  w.node = 0;
  w.sp = 0;
}

// The block's tally row in shared memory: two 16-bit counters per 32-bit word (bin b in the
// low half of word b / 2 when b is even, the high half when odd). A work item holds at most
// kMaxItemRays rays (paths), so no counter can pass 65,535 and spill into its neighbour.
// Halving the row leaves more of the SM's unified L1 / shared memory to the per-thread
// traversal stacks.
constexpr int64_t kMaxItemRays = 1 << 15;
__device__ __forceinline__ void tally_clear(uint32_t* hist, int n_bins) {
  for (int w = threadIdx.x; w < (n_bins + 1) / 2; w += kThreads) hist[w] = 0u;
}
__device__ __forceinline__ void tally_add(uint32_t* hist, int b, uint32_t c) {
  atomicAdd(&hist[b >> 1], c << ((b & 1) * 16));
}
__device__ __forceinline__ void tally_flush(const uint32_t* hist, int n_bins, unsigned long long* row) {
  for (int w = threadIdx.x; w < (n_bins + 1) / 2; w += kThreads) {
    const uint32_t v = hist[w];
    if (v & 0xffffu) atomicAdd(row + 2 * w, (unsigned long long)(v & 0xffffu));
    if ((v >> 16) && 2 * w + 1 < n_bins) atomicAdd(row + 2 * w + 1, (unsigned long long)(v >> 16));
  }
}

// Refill variant (see the file comment). Best when traversals are long and uneven.
template <bool E, bool kBVH, bool S, class St>
__global__ void __launch_bounds__(kThreads, RG_REFILL_MIN_BLOCKS) trace_kernel_refill(const TraceParams p) {
  extern __shared__ __align__(16) uint32_t hist[];
  __shared__ Ring s_ring[kWarps];
  __shared__ int32_t s_item;
  __shared__ int32_t s_next;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  Ring& ring = s_ring[threadIdx.x >> 5];
  bool overflow = false;
  St st;
  unsigned long long n_rays = 0;
  int32_t stack[kTraceStack];
  const DevMesh& m = p.m;
  while (true) {
    if (threadIdx.x == 0) {
      s_item = atomicAdd(p.item_counter, 1);
      s_next = 0;
    }
    tally_clear(hist, p.n_bins);
    __syncthreads();
    const int32_t item = s_item;
    if (item >= p.n_items) break;
    const WorkItem wi = p.items[item];
    // the item's row: a face, or side (wi.face & 1) of face (wi.face >> 1) when S
    const int32_t face = S ? wi.face >> 1 : wi.face;
    const bool side_b = S && (wi.face & 1);
    const uint32_t stream = (uint32_t)face | (side_b ? 0x80000000u : 0u);
    const int32_t env = p.n_bins - 1;
    // warp-uniform ring state: `avail` sampled rays from position `head`
    int head = 0, avail = 0;
    bool more = true;  // rays of the item left to sample
    bool has_ray = false, done = false;
    Walker w;
    while (true) {
      if (has_ray && !done) {
        if (kBVH) {
          done = !visit<E, S>(m, w, stack, &overflow, st);
        } else {
          for (int64_t t = 0; t < m.nt; ++t) {
            test_record<E, S>(m.tris + 3 * t, w.src, w.o, w.d, w.best_t, w.best_id, w.best_face);
            st.tri();
          }
          done = true;
        }
      }
      const unsigned tracing = __ballot_sync(0xffffffffu, has_ray && !done);
      const unsigned idle = ~tracing;
      if (tracing && __popc(idle) < kRefillLanes) continue;
      // ---- refill: tally finished rays, then hand out new ones
      const unsigned fin = __ballot_sync(0xffffffffu, has_ray && done);
      if (has_ray && done) {
        const unsigned peers = __match_any_sync(fin, w.best_face);
        if (lane == __ffs(peers) - 1) tally_add(hist, w.best_face, (uint32_t)__popc(peers));
        ++n_rays;
        has_ray = false;
      }
      const int need = __popc(idle);
      if (avail < need && more) {  // sample 32 rays, all lanes in step
        int base = 0;
        if (lane == 0) base = atomicAdd(&s_next, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        const int r = base + lane;
        const bool valid = r < wi.count;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (valid) {
          V3 o, d;
          int32_t src;
          sample_ray<E>(m, p.key0, p.key1, p.ray_offset + (uint64_t)(wi.begin + r), face, &o, &d, &src, stream, 0u,
                        side_b);
          const int slot = (head + avail + lane) & (kRing - 1);
          ring.ox[slot] = o.x; ring.oy[slot] = o.y; ring.oz[slot] = o.z;
          ring.dx[slot] = d.x; ring.dy[slot] = d.y; ring.dz[slot] = d.z;
          ring.src[slot] = src;
        }
        avail += __popc(vm);
        if (base + 32 >= wi.count) more = false;
        __syncwarp();
      }
      const int rank = __popc(idle & lt_mask);
      if (!(tracing >> lane & 1u) && rank < avail) {
        start_ray(w, ring, (head + rank) & (kRing - 1), env);
        has_ray = true;
        done = false;
      }
      const int used = min(need, avail);
      head = (head + used) & (kRing - 1);
      avail -= used;
      __syncwarp();
      if (!__any_sync(0xffffffffu, has_ray)) break;  // ring empty and nothing left to sample
    }
    __syncthreads();
    tally_flush(hist, p.n_bins, p.counts + (int64_t)wi.face * p.n_bins);
    __syncthreads();
  }
  if (overflow) atomicExch(p.error_word, 1);
  if constexpr (sizeof(St) > 1) {
    for (int o = 16; o > 0; o >>= 1) {
      n_rays += __shfl_xor_sync(0xffffffffu, n_rays, o);
      st.n_box += __shfl_xor_sync(0xffffffffu, st.n_box, o);
      st.n_tri += __shfl_xor_sync(0xffffffffu, st.n_tri, o);
    }
    if (lane == 0) {
      atomicAdd(p.stats, n_rays);
      atomicAdd(p.stats + 1, st.n_box);
      atomicAdd(p.stats + 2, st.n_tri);
    }
  } else {
    (void)n_rays;
  }
}

// Lock-step variant for shallow BVHs. Each round the warp samples 32 rays in step and
// gives every ray one node visit (the root); rays that are finished by then (typically
// those leaving the scene) go straight to the tally, and the others are queued, with
// their traversal state, in a per-warp shared-memory queue. Whenever 32 rays are queued
// the warp continues them to completion in step, so the long traversals run with full
// warps instead of next to lanes that finished after one visit.
template <bool E, bool kBVH, bool S, class St>
__global__ void __launch_bounds__(kThreads, RG_LOCKSTEP_MIN_BLOCKS) trace_kernel_lockstep(const TraceParams p) {
  extern __shared__ __align__(16) uint32_t hist[];
  __shared__ Ring s_queue[kWarps];
  __shared__ int32_t s_item;
  __shared__ int32_t s_next;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  Ring& q = s_queue[threadIdx.x >> 5];
  bool overflow = false;
  St st;
  unsigned long long n_rays = 0;
  int32_t stack[kTraceStack];
  const DevMesh& m = p.m;
  const int32_t env = p.n_bins - 1;

  auto tally = [&](bool fin, int32_t face) {
    const unsigned fm = __ballot_sync(0xffffffffu, fin);
    if (fin) {
      const unsigned peers = __match_any_sync(fm, face);
      if (lane == __ffs(peers) - 1) tally_add(hist, face, (uint32_t)__popc(peers));
      ++n_rays;
    }
  };
  // Trace the queued rays q[0 .. count) (count <= 32) to completion.
  auto drain = [&](int count) {
    const bool has = lane < count;
    Walker w;
    if (has) start_ray(w, q, lane, env);
    bool more = has;
    while (__any_sync(0xffffffffu, more)) {
      if (more) more = visit<E, S>(m, w, stack, &overflow, st);
    }
    tally(has, has ? w.best_face : 0);
  };

  while (true) {
    if (threadIdx.x == 0) {
      s_item = atomicAdd(p.item_counter, 1);
      s_next = 0;
    }
    tally_clear(hist, p.n_bins);
    __syncthreads();
    const int32_t item = s_item;
    if (item >= p.n_items) break;
    const WorkItem wi = p.items[item];
    // the item's row: a face, or side (wi.face & 1) of face (wi.face >> 1) when S
    const int32_t face_i = S ? wi.face >> 1 : wi.face;
    const bool side_b = S && (wi.face & 1);
    const uint32_t stream = (uint32_t)face_i | (side_b ? 0x80000000u : 0u);
    int queued = 0;  // warp-uniform
    while (true) {
      int base = 0;
      if (lane == 0) base = atomicAdd(&s_next, 32);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= wi.count) break;
      const int r = base + lane;
      const bool valid = r < wi.count;
      V3 o, d;
      int32_t src = -1;
      if (valid) sample_ray<E>(m, p.key0, p.key1, p.ray_offset + (uint64_t)(wi.begin + r), face_i, &o, &d, &src,
                              stream, 0u, side_b);
      bool more = false;
      int32_t face = env;
      if (valid) {
        if (kBVH) {
          // escape test: does the ray enter either child box of the root? Rays that do
          // are traced from the root by drain(); the others leave the scene.
          const float ix = rcp_approx(d.x), iy = rcp_approx(d.y), iz = rcp_approx(d.z);
          const float ox = o.x * ix, oy = o.y * iy, oz = o.z * iz;
          const float4 a = __ldg(m.nodes), b = __ldg(m.nodes + 1), c = __ldg(m.nodes + 2);
          const float lim = __int_as_float(0x7f800000);
          float lmin, lmax, rmin, rmax;
          slab_window(fmaf(a.x, ix, -ox), fmaf(a.y, ix, -ox), fmaf(a.z, iy, -oy), fmaf(a.w, iy, -oy),
                      fmaf(c.x, iz, -oz), fmaf(c.y, iz, -oz), m.t_lo, lim, lmin, lmax);
          slab_window(fmaf(b.x, ix, -ox), fmaf(b.y, ix, -ox), fmaf(b.z, iy, -oy), fmaf(b.w, iy, -oy),
                      fmaf(c.z, iz, -oz), fmaf(c.w, iz, -oz), m.t_lo, lim, rmin, rmax);
          st.box(2);
          more = lmin <= lmax || rmin <= rmax;
        } else {
          face = closest_face<E, false, S>(m, src, o, d, &overflow, st, env);
        }
      }
      if (kBVH) {
        // with a BVH every ray finished here left the scene: one count for all of them
        const unsigned esc = __ballot_sync(0xffffffffu, valid && !more);
        if (lane == 0 && esc) tally_add(hist, env, (uint32_t)__popc(esc));
        if (valid && !more) ++n_rays;
      } else {
        tally(valid && !more, face);
      }
      // queue the rays that need more visits; they restart from the root
      const unsigned sm = __ballot_sync(0xffffffffu, more);
      if (more) {
        const int slot = queued + __popc(sm & lt_mask);
        q.ox[slot] = o.x; q.oy[slot] = o.y; q.oz[slot] = o.z;
        q.dx[slot] = d.x; q.dy[slot] = d.y; q.dz[slot] = d.z;
        q.src[slot] = src;
      }
      queued += __popc(sm);
      __syncwarp();
      if (queued >= 32) {
        drain(32);
        __syncwarp();
        const int rest = queued - 32;
        float ox = 0.f, oy = 0.f, oz = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
        int32_t sr = 0;
        if (lane < rest) {
          ox = q.ox[32 + lane]; oy = q.oy[32 + lane]; oz = q.oz[32 + lane];
          dx = q.dx[32 + lane]; dy = q.dy[32 + lane]; dz = q.dz[32 + lane];
          sr = q.src[32 + lane];
        }
        __syncwarp();
        if (lane < rest) {
          q.ox[lane] = ox; q.oy[lane] = oy; q.oz[lane] = oz;
          q.dx[lane] = dx; q.dy[lane] = dy; q.dz[lane] = dz;
          q.src[lane] = sr;
        }
        __syncwarp();
        queued = rest;
      }
    }
    if (queued > 0) {
      drain(queued);
      __syncwarp();
    }
    __syncthreads();
    tally_flush(hist, p.n_bins, p.counts + (int64_t)wi.face * p.n_bins);
    __syncthreads();
  }
  if (overflow) atomicExch(p.error_word, 1);
  if constexpr (sizeof(St) > 1) {
    for (int o = 16; o > 0; o >>= 1) {
      n_rays += __shfl_xor_sync(0xffffffffu, n_rays, o);
      st.n_box += __shfl_xor_sync(0xffffffffu, st.n_box, o);
      st.n_tri += __shfl_xor_sync(0xffffffffu, st.n_tri, o);
    }
    if (lane == 0) {
      atomicAdd(p.stats, n_rays);
      atomicAdd(p.stats + 1, st.n_box);
      atomicAdd(p.stats + 2, st.n_tri);
    }
  } else {
    (void)n_rays;
  }
}

// REFs directly from MCRT (Sec. 4.2.2): every lane follows its own path through its
// bounces (closest hit, Philox decision between absorption, diffuse re-emission from the
// hit face and loss); finished paths are tallied per absorbing face (column N: escaped)
// in the block's shared-memory row of the item's source face.
template <bool E, bool kBVH>
__global__ void __launch_bounds__(kThreads) trace_kernel_reflect(const TraceParams p) {
  extern __shared__ __align__(16) uint32_t hist[];
  __shared__ int32_t s_item;
  __shared__ int32_t s_next;
  const int lane = threadIdx.x & 31;
  bool overflow = false;
  NoStats st;
  unsigned long long n_rays = 0, n_hits = 0, n_lost = 0, n_over = 0;
  const DevMesh& m = p.m;
  while (true) {
    if (threadIdx.x == 0) {
      s_item = atomicAdd(p.item_counter, 1);
      s_next = 0;
    }
    tally_clear(hist, p.n_bins);
    __syncthreads();
    const int32_t item = s_item;
    if (item >= p.n_items) break;
    const WorkItem wi = p.items[item];
    while (true) {
      int base = 0;
      if (lane == 0) base = atomicAdd(&s_next, 32);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= wi.count) break;
      const int r = base + lane;
      int32_t col = -1;  // absorbing face, N (escaped) or -1 (lost / overflow / no ray)
      if (r < wi.count) {
        const uint64_t ray = p.ray_offset + (uint64_t)(wi.begin + r);
        const uint32_t stream = (uint32_t)wi.face;
        V3 o, d;
        int32_t src;
        sample_ray<E>(m, p.key0, p.key1, ray, wi.face, &o, &d, &src, stream, 0u);
        ++n_rays;
        for (int32_t bounce = 1;; ++bounce) {
          const int32_t j = closest_face<E, kBVH, false>(m, src, o, d, &overflow, st, m.n_faces);
          if (j == m.n_faces) { col = j; break; }
          ++n_hits;
          const uint32_t cb = (uint32_t)bounce << 7;
          // the decision draws counter cb + 1; cb itself is the re-emission's draw
          const uint4 x =
              philox(make_uint4((uint32_t)ray, (uint32_t)(ray >> 32), stream, cb + 1u), p.key0, p.key1);
          const unsigned long long dec = x.w;
          if (dec < p.thr_absorb[j]) { col = j; break; }
          if (dec >= p.thr_reflect[j]) { ++n_lost; break; }
          if (bounce >= p.max_bounces) { ++n_over; break; }
          sample_ray<E>(m, p.key0, p.key1, ray, j, &o, &d, &src, stream, cb);
        }
      }
      const bool fin = col >= 0;
      const unsigned fm = __ballot_sync(0xffffffffu, fin);
      if (fin) {
        const unsigned peers = __match_any_sync(fm, col);
        if (lane == __ffs(peers) - 1) tally_add(hist, col, (uint32_t)__popc(peers));
      }
    }
    __syncthreads();
    tally_flush(hist, p.n_bins, p.counts + (int64_t)wi.face * p.n_bins);
    __syncthreads();
  }
  if (overflow) atomicExch(p.error_word, 1);
  for (int o = 16; o > 0; o >>= 1) {
    n_rays += __shfl_xor_sync(0xffffffffu, n_rays, o);
    n_hits += __shfl_xor_sync(0xffffffffu, n_hits, o);
    n_lost += __shfl_xor_sync(0xffffffffu, n_lost, o);
    n_over += __shfl_xor_sync(0xffffffffu, n_over, o);
  }
  if (lane == 0) {
    atomicAdd(p.stats, n_rays);
    atomicAdd(p.stats + 1, n_hits);
    atomicAdd(p.stats + 2, n_lost);
    atomicAdd(p.stats + 3, n_over);
  }
}

// Shared memory of the tally row: (n_bins + 1) / 2 words, rounded up to 16 bytes.
inline size_t trace_smem_bytes(int n_bins) { return (size_t)((((n_bins + 1) / 2) + 3) & ~3) * sizeof(uint32_t); }

template <bool E, bool B, class St, bool S = false>
cudaError_t launch(const TraceParams& p, int sm_count, size_t smem, cudaStream_t s) {
  auto k = p.m.refill ? trace_kernel_refill<E, B, S, St> : trace_kernel_lockstep<E, B, S, St>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = sm_count * per_sm;
  if (grid > p.n_items) grid = p.n_items;
  k<<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// Reflection launches: one persistent block per resident slot.
template <bool E, bool B>
cudaError_t launch_reflect(const TraceParams& p, int sm_count, size_t smem, cudaStream_t s) {
  auto k = trace_kernel_reflect<E, B>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = sm_count * per_sm;
  if (grid > p.n_items) grid = p.n_items;
  k<<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// sided = true: side-resolved counts, rows and columns 2f + side (see the file comment).
rg_status trace_impl(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_face_h, uint64_t seed,
                     uint64_t ray_offset, int32_t fma_free, int64_t* counts_d, uint64_t* stats_h, void* stream,
                     bool sided = false) {
  if (!ctx) return RG_ERR_ARG;
  const char* fn = sided ? "rg_trace_sided" : "rg_trace";
  RG_ARG_CHECK(ctx, mesh && rays_per_face_h && counts_d, "%s: NULL argument", fn);
  const DevMesh& m = mesh_device_view(mesh);
  RG_ARG_CHECK(ctx, mesh_device(mesh) == ctx->device, "%s: mesh belongs to another device", fn);
  RG_ARG_CHECK(ctx, !sided || m.wound_like_face,
               "rg_trace_sided: a triangle is wound against its face (its normal e1 x e2 points to side B)");
  const int32_t N = m.n_faces;
  RG_ARG_CHECK(ctx, !sided || N < (1 << 29), "rg_trace_sided: %d faces", N);
  const int32_t n_rows = sided ? 2 * N : N;
  const int32_t n_bins = n_rows + 1;
  const size_t smem = trace_smem_bytes(n_bins);
  if (n_bins > 49152 || (int)smem > ctx->smem_optin - 1024)
    return rg::fail(ctx, RG_ERR_UNSUPPORTED, "%s: %d tally columns exceed the shared-memory tally row", fn, n_bins);
  // work items: chunks of at most `chunk` rays of one row. Blocks take items dynamically,
  // so the last ones set the tail of the launch: the chunk halves from 32,768 rays (the
  // most a 16-bit tally counter can take) while the launch would give its resident blocks
  // fewer than 32 items each, down to 16,384 (measured on GB300: the 1e8-ray small-
  // satellite trace 4.20 -> 4.75 G rays/s; below that the per-item clearing and flushing
  // of the tally row starts to show)
  int64_t total = 0;
  for (int32_t f = 0; f < n_rows; ++f) total += std::max<int64_t>(rays_per_face_h[f], 0);
  const int64_t resident = (int64_t)ctx->sm_count * (m.refill ? RG_REFILL_MIN_BLOCKS : RG_LOCKSTEP_MIN_BLOCKS);
  int64_t kChunk = kMaxItemRays;
  while (kChunk > (1 << 14) && total / kChunk < 32 * resident) kChunk /= 2;
  std::vector<WorkItem> items;
  for (int32_t f = 0; f < n_rows; ++f) {
    int64_t n = rays_per_face_h[f];
    RG_ARG_CHECK(ctx, n >= 0, "%s: negative ray count for row %d", fn, f);
    for (int64_t b = 0; b < n; b += kChunk) items.push_back({b, f, (int32_t)std::min(kChunk, n - b)});
  }
  if (stats_h) stats_h[0] = stats_h[1] = stats_h[2] = 0;
  if (items.empty()) return RG_OK;
  RG_ARG_CHECK(ctx, items.size() < (size_t)INT32_MAX, "%s: too many rays", fn);
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  rg_status st = rg::workspace(ctx, items.size() * sizeof(WorkItem) + 256, &ws);
  if (st != RG_OK) return st;
  unsigned long long* d_stats = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws)) ;
  WorkItem* d_items = reinterpret_cast<WorkItem*>(static_cast<char*>(ws) + 256);
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch, 0, 2 * sizeof(int32_t), s));
  if (stats_h) RG_CUDA_TRY(ctx, cudaMemsetAsync(d_stats, 0, 3 * sizeof(unsigned long long), s));
  TraceParams p;
  p.m = m;
  p.items = d_items;
  p.n_items = (int32_t)items.size();
  p.item_counter = ctx->d_scratch;
  p.error_word = ctx->d_scratch + 1;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  p.ray_offset = ray_offset;
  p.counts = reinterpret_cast<unsigned long long*>(counts_d);
  p.n_bins = n_bins;
  p.stats = d_stats;
  cudaError_t e;
  const int sm = ctx->sm_count;
  const int tok = rg::timer_begin(ctx, rg::kTimeTrace, s);
  if (sided) {
    if (fma_free)
      e = m.use_bvh ? launch<true, true, NoStats, true>(p, sm, smem, s) : launch<true, false, NoStats, true>(p, sm, smem, s);
    else
      e = m.use_bvh ? launch<false, true, NoStats, true>(p, sm, smem, s)
                    : launch<false, false, NoStats, true>(p, sm, smem, s);
  } else if (stats_h) {
    if (fma_free)
      e = m.use_bvh ? launch<true, true, Stats>(p, sm, smem, s) : launch<true, false, Stats>(p, sm, smem, s);
    else
      e = m.use_bvh ? launch<false, true, Stats>(p, sm, smem, s) : launch<false, false, Stats>(p, sm, smem, s);
  } else {
    if (fma_free)
      e = m.use_bvh ? launch<true, true, NoStats>(p, sm, smem, s) : launch<true, false, NoStats>(p, sm, smem, s);
    else
      e = m.use_bvh ? launch<false, true, NoStats>(p, sm, smem, s) : launch<false, false, NoStats>(p, sm, smem, s);
  }
  rg::timer_end(ctx, tok, s);
  if (e != cudaSuccess) return rg::cuda_fail(ctx, e, sided ? "rg_trace_sided: launch" : "rg_trace: launch");
  ++ctx->launches;
  // the host copy of the items must outlive the async upload, and the error word is read back
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, ctx->d_scratch + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (stats_h) RG_CUDA_TRY(ctx, cudaMemcpyAsync(stats_h, d_stats, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (ctx->h_scratch[0]) return rg::fail(ctx, RG_ERR_STACK, "%s: traversal stack overflow", fn);
  return RG_OK;
}

}  // namespace

extern "C" {

rg_status rg_trace(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_face_h, uint64_t seed,
                   uint64_t ray_offset, int32_t fma_free, int64_t* counts_d, void* stream) {
  return trace_impl(ctx, mesh, rays_per_face_h, seed, ray_offset, fma_free, counts_d, nullptr, stream);
}

rg_status rg_trace_sided(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_side_h, uint64_t seed,
                         uint64_t ray_offset, int32_t fma_free, int64_t* counts_d, void* stream) {
  return trace_impl(ctx, mesh, rays_per_side_h, seed, ray_offset, fma_free, counts_d, nullptr, stream, true);
}

rg_status rg_trace_stats(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_face_h, uint64_t seed,
                         uint64_t ray_offset, int32_t fma_free, int64_t* counts_d, uint64_t* stats_out_h,
                         void* stream) {
  if (!stats_out_h) return rg::fail(ctx, RG_ERR_ARG, "rg_trace_stats: NULL stats");
  return trace_impl(ctx, mesh, rays_per_face_h, seed, ray_offset, fma_free, counts_d, stats_out_h, stream);
}

rg_status rg_trace_reflect(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_face_h, const double* eps_h,
                           const double* rho_h, int32_t max_bounces, uint64_t seed, uint64_t ray_offset,
                           int32_t fma_free, int64_t* counts_d, uint64_t* stats_out_h, void* stream) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, mesh && rays_per_face_h && eps_h && rho_h && counts_d, "rg_trace_reflect: NULL argument");
  RG_ARG_CHECK(ctx, max_bounces >= 1 && max_bounces < (1 << 25), "rg_trace_reflect: max_bounces %d outside [1, 2^25)",
               max_bounces);
  const DevMesh& m = mesh_device_view(mesh);
  RG_ARG_CHECK(ctx, mesh_device(mesh) == ctx->device, "rg_trace_reflect: mesh belongs to another device");
  const int32_t N = m.n_faces;
  const int32_t n_bins = N + 1;
  const size_t smem = trace_smem_bytes(n_bins);
  if (n_bins > 49152 || (int)smem > ctx->smem_optin - 1024)
    return rg::fail(ctx, RG_ERR_UNSUPPORTED, "rg_trace_reflect: %d faces exceed the shared-memory tally row", N);
  // per-face decision thresholds: x < floor(eps 2^32) absorbs, x < floor((eps + rho) 2^32) reflects
  std::vector<unsigned long long> thr(2 * (size_t)N);
  for (int32_t f = 0; f < N; ++f) {
    const double a = eps_h[f], r = rho_h[f];
    RG_ARG_CHECK(ctx, a >= 0.0 && r >= 0.0 && a + r <= 1.0, "rg_trace_reflect: face %d has eps %.17g, rho %.17g", f,
                 a, r);
    thr[f] = (unsigned long long)std::floor(a * 4294967296.0);
    thr[N + f] = (unsigned long long)std::floor((a + r) * 4294967296.0);
  }
  constexpr int64_t kChunk = 1 << 14;  // paths are long and uneven: smaller items balance the blocks
  static_assert(kChunk <= kMaxItemRays, "an item's tally counters are 16-bit");
  std::vector<WorkItem> items;
  for (int32_t f = 0; f < N; ++f) {
    int64_t n = rays_per_face_h[f];
    RG_ARG_CHECK(ctx, n >= 0, "rg_trace_reflect: negative ray count for face %d", f);
    for (int64_t b = 0; b < n; b += kChunk) items.push_back({b, f, (int32_t)std::min(kChunk, n - b)});
  }
  uint64_t h_stats[4] = {0, 0, 0, 0};
  if (items.empty()) {
    if (stats_out_h) memcpy(stats_out_h, h_stats, sizeof(h_stats));
    return RG_OK;
  }
  RG_ARG_CHECK(ctx, items.size() < (size_t)INT32_MAX, "rg_trace_reflect: too many rays");
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t thr_off = 256 + rg::align_up(items.size() * sizeof(WorkItem), 256);
  void* ws = nullptr;
  rg_status st = rg::workspace(ctx, thr_off + thr.size() * sizeof(unsigned long long), &ws);
  if (st != RG_OK) return st;
  char* wb = static_cast<char*>(ws);
  unsigned long long* d_stats = reinterpret_cast<unsigned long long*>(wb);
  WorkItem* d_items = reinterpret_cast<WorkItem*>(wb + 256);
  unsigned long long* d_thr = reinterpret_cast<unsigned long long*>(wb + thr_off);
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(d_thr, thr.data(), thr.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                   s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scratch, 0, 2 * sizeof(int32_t), s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(d_stats, 0, 4 * sizeof(unsigned long long), s));
  TraceParams p;
  p.m = m;
  p.items = d_items;
  p.n_items = (int32_t)items.size();
  p.item_counter = ctx->d_scratch;
  p.error_word = ctx->d_scratch + 1;
  p.key0 = (uint32_t)seed;
  p.key1 = (uint32_t)(seed >> 32);
  p.ray_offset = ray_offset;
  p.counts = reinterpret_cast<unsigned long long*>(counts_d);
  p.n_bins = n_bins;
  p.stats = d_stats;
  p.thr_absorb = d_thr;
  p.thr_reflect = d_thr + N;
  p.max_bounces = max_bounces;
  const int sm = ctx->sm_count;
  cudaError_t e;
  if (fma_free)
    e = m.use_bvh ? launch_reflect<true, true>(p, sm, smem, s) : launch_reflect<true, false>(p, sm, smem, s);
  else
    e = m.use_bvh ? launch_reflect<false, true>(p, sm, smem, s) : launch_reflect<false, false>(p, sm, smem, s);
  if (e != cudaSuccess) return rg::cuda_fail(ctx, e, "rg_trace_reflect: launch");
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, ctx->d_scratch + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(h_stats, d_stats, sizeof(h_stats), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (stats_out_h) memcpy(stats_out_h, h_stats, sizeof(h_stats));
  if (ctx->h_scratch[0]) return rg::fail(ctx, RG_ERR_STACK, "rg_trace_reflect: traversal stack overflow");
  return RG_OK;
}

rg_status rg_launch_count(const rg_ctx* ctx, int64_t* launches_out_h) {
  if (!ctx || !launches_out_h) return RG_ERR_ARG;
  *launches_out_h = ctx->launches;
  return RG_OK;
}

}  // extern "C"
