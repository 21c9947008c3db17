/*
 * Oracle for Monte Carlo ray tracing (MCRT) of view factors.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow CPU reference that the
 * CUDA path is checked against. Only tests/, __graft_entry__.smoke() and the
 * bench's cpu_baseline / reference arm may load it. It shares no code with the
 * library under paper_2511_04277_gb300/.
 *
 * What it computes (Sec. 3.5.1, Eq. 3.15): for every source face i, N_i rays are
 * emitted and N_ij counts the rays whose closest hit lies on face j (column N =
 * the environment, Sec. 2.4.12 "N x (N+1)" matrix). F_ij = N_ij / N_i.
 * Emission is diffuse (Sec. 2.4.12: view factors assume diffuse emission), so the
 * direction is cosine-weighted about the face normal; origins are uniform over
 * the face area (Sec. 5.2.1, assumption 1).
 *
 * The paper gives no ray definition, so one is fixed here and in the library:
 *   RNG        Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed lo,
 *              seed hi), counter = (ray lo, ray hi, face, 0): one draw per ray.
 *   uniform    u = (x >> 8) * 2^-24.
 *   triangle   first k with x0 < thr[k] (uint32 area CDF of the face), else last.
 *   point      (u,v) = draws 1,2; folded to (1-u,1-v) if u+v > 1; pulled toward
 *              the centroid, u' = u*k + w with k = 1 - 2^-20 and w = float(2^-20/3),
 *              so that no origin lies on an edge; p = (v0 + u'*e1) + v'*e2, then
 *              lifted off the face: o = p + lift*n.
 *   direction  cosine-weighted from the same draw (one draw per ray): the point of
 *              the unit disc at radius sqrt(s) and angle 2 pi a projects to the
 *              direction (x, y, z) = (sqrt(s) cos, sqrt(s) sin, sqrt(1 - s)), which is
 *              Malley's method without rejection (s and a uniform make the disc
 *              point uniform). a = (word 3 >> 8) 2^-24; s = u-style 24 bits made of
 *              the low bytes of words 3, 1, 2 (the point used the top 24 bits of
 *              words 1, 2). cos and sin: a's top two bits pick the quadrant, the
 *              rest the angle in it, folded to [0, pi/4] and evaluated by the
 *              Taylor polynomials of degree 9 (sin) and 10 (cos) in float
 *              (disc_direction below, the order of every operation fixed).
 *              d = (x*t + y*b) + z*n in the face frame (t, b, n).
 *   hit        Moller-Trumbore, every operation rounded to float (no FMA),
 *              u,v >= -eb, u+v <= 1+eb with eb = 2^-20, t > 0, the source
 *              triangle skipped; closest = lexicographically smallest (t, tri).
 *   lift       1e-6 * length of the diagonal of the vertex bounding box. The
 *              lifted origin puts the source plane strictly behind the ray, so
 *              hits on an adjacent face at t ~ 1e-7 (rays born next to an edge of
 *              an enclosure) are kept and a closed enclosure loses no ray.
 * Face frame: from the face's lowest-index triangle (v0,v1,v2):
 *   n = c/|c| with c = cross(v1-v0, v2-v0); t = e1/|e1|; b = cross(n, t).
 *
 * Diffuse reflections (Sec. 4.2.2, REFs directly from MCRT): a random walk whose
 * expectation is B_ij of Eq. 4.5, the fraction of the energy emitted by i that is
 * absorbed by j. A ray emitted from face i as above is followed through bounces
 * b = 1, 2, ...: at its closest hit on face j, word 3 of the draw of counter
 * (ray lo, ray hi, i, b*128 + 1) decides
 *   x < floor(eps_j 2^32)            absorbed: counted for column j, path ends;
 *   x < floor((eps_j + rho_j) 2^32)  reflected diffusely;
 *   otherwise                        lost (neither absorbed nor reflected), path ends;
 * a miss is counted for the environment column. A reflection re-emits from face j
 * exactly as an emission of face j would, with the draw of counter
 * (ray lo, ray hi, i, b*128) in place of the emission draw (triangle, point and
 * direction). Re-emitting from a
 * uniform point of the face is the face-level model of Eq. 4.5 (each face reflects
 * with one uniform radiosity), so the walk estimates the same B as Gebhart's method
 * for the same faces. A path still reflecting after max_bounces counts as overflow.
 *
 * Two-sided faces (Sec. 5.2.4-5.2.5, side-resolved factors F^{X->Y}): face f has side
 * A, the side its normal n points to, and side B. Row 2f+X of the side-resolved count
 * matrix [2N x (2N+1)] counts the rays emitted from side X of face f: the triangle and
 * point draws of face f, the origin lifted along n_X and the direction
 * (x*t + y*b_X) + z*n_X, with n_A = n, b_A = b, n_B = -n, b_B = -b, and counter word
 * 2 = f for side A, f + 2^31 for side B. Side A's rays are thus exactly face f's rays
 * of the one-sided definition above. A hit on triangle k lies on side A of its face
 * when det > 0 in Moller-Trumbore (the ray runs against the triangle normal e1 x e2)
 * and on side B when det < 0; it is counted in column 2g+Y, a miss in column 2N.
 * This needs every triangle of a face wound like the face's first triangle:
 * dot(e1 x e2, n) > 0 for each of them (checked).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no fast-math), so
 * every float operation is one IEEE-rounded operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of the 4x32 S-box with the  */
/* multipliers and Weyl key increments published with the generator.        */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p2 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi2 = (uint32_t)(p2 >> 32), lo2 = (uint32_t)p2;
    uint32_t n0 = hi2 ^ c[1] ^ k0;
    uint32_t n1 = lo2;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void draw(uint64_t seed, uint64_t ray, uint32_t face, uint32_t word3,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)ray, (uint32_t)(ray >> 32), face, word3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, out);
}

/* u in [0,1) with 24 random bits. */
static float unit_float(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }

/* ------------------------------------------------------------------------ */
/* Float vector helpers, written out so that the operation order is visible. */
/* ------------------------------------------------------------------------ */
typedef struct { float x, y, z; } v3;

static v3 vsub(v3 a, v3 b) { v3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static v3 vcross(v3 a, v3 b) {
  v3 r;
  r.x = a.y * b.z - a.z * b.y;
  r.y = a.z * b.x - a.x * b.z;
  r.z = a.x * b.y - a.y * b.x;
  return r;
}
static float vdot(v3 a, v3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
static v3 vnormalize(v3 a) {
  float len = sqrtf(vdot(a, a));
  v3 r = {a.x / len, a.y / len, a.z / len};
  return r;
}
static v3 vert(const float* verts, int32_t i) {
  v3 r = {verts[3 * (int64_t)i], verts[3 * (int64_t)i + 1], verts[3 * (int64_t)i + 2]};
  return r;
}

/* ------------------------------------------------------------------------ */
/* Mesh preprocessing: per-face frame, area CDF, first triangle.             */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n_faces;
  int64_t nt;
  const float* verts;
  const int32_t* tris;
  const int32_t* tri_face;
  /* per triangle (float): v0, e1 = v1 - v0, e2 = v2 - v0 */
  v3* tv0; v3* te1; v3* te2;
  /* per face: triangle list (ascending), thresholds, frame */
  int64_t* face_start;   /* n_faces + 1 */
  int32_t* face_tris;    /* nt */
  uint32_t* face_thr;    /* nt, aligned with face_tris */
  v3* fn; v3* ft; v3* fb;
  double* face_area;
  float lift;
  int wound_like_face;  /* 1: every triangle's e1 x e2 points to its face's side A */
} omesh;

static double tri_area_d(const float* verts, const int32_t* t) {
  double a[3], b[3];
  for (int k = 0; k < 3; ++k) {
    double p0 = verts[3 * (int64_t)t[0] + k];
    a[k] = (double)verts[3 * (int64_t)t[1] + k] - p0;
    b[k] = (double)verts[3 * (int64_t)t[2] + k] - p0;
  }
  double cx = a[1] * b[2] - a[2] * b[1];
  double cy = a[2] * b[0] - a[0] * b[2];
  double cz = a[0] * b[1] - a[1] * b[0];
  return 0.5 * sqrt((cx * cx + cy * cy) + cz * cz);
}

static void omesh_free(omesh* m) {
  free(m->tv0); free(m->te1); free(m->te2);
  free(m->face_start); free(m->face_tris); free(m->face_thr);
  free(m->fn); free(m->ft); free(m->fb); free(m->face_area);
}

static int omesh_init(omesh* m, const float* verts, int64_t nv, const int32_t* tris,
                      int64_t nt, const int32_t* tri_face, int32_t n_faces) {
  memset(m, 0, sizeof(*m));
  if (!verts || !tris || !tri_face || nv <= 0 || nt <= 0 || n_faces <= 0) return ORC_ERR_ARG;
  m->n_faces = n_faces; m->nt = nt; m->verts = verts; m->tris = tris; m->tri_face = tri_face;
  for (int64_t k = 0; k < nt; ++k) {
    if (tri_face[k] < 0 || tri_face[k] >= n_faces) return ORC_ERR_ARG;
    for (int c = 0; c < 3; ++c)
      if (tris[3 * k + c] < 0 || tris[3 * k + c] >= nv) return ORC_ERR_ARG;
  }
  m->tv0 = malloc(sizeof(v3) * nt); m->te1 = malloc(sizeof(v3) * nt); m->te2 = malloc(sizeof(v3) * nt);
  m->face_start = calloc(n_faces + 1, sizeof(int64_t));
  m->face_tris = malloc(sizeof(int32_t) * nt);
  m->face_thr = malloc(sizeof(uint32_t) * nt);
  m->fn = malloc(sizeof(v3) * n_faces); m->ft = malloc(sizeof(v3) * n_faces); m->fb = malloc(sizeof(v3) * n_faces);
  m->face_area = calloc(n_faces, sizeof(double));
  if (!m->tv0 || !m->te1 || !m->te2 || !m->face_start || !m->face_tris || !m->face_thr ||
      !m->fn || !m->ft || !m->fb || !m->face_area) { omesh_free(m); return ORC_ERR_OOM; }

  for (int64_t k = 0; k < nt; ++k) {
    v3 p0 = vert(verts, tris[3 * k]), p1 = vert(verts, tris[3 * k + 1]), p2 = vert(verts, tris[3 * k + 2]);
    m->tv0[k] = p0; m->te1[k] = vsub(p1, p0); m->te2[k] = vsub(p2, p0);
  }
  /* counting sort of triangles by face, ascending triangle index within a face */
  for (int64_t k = 0; k < nt; ++k) m->face_start[tri_face[k] + 1]++;
  for (int32_t f = 0; f < n_faces; ++f) m->face_start[f + 1] += m->face_start[f];
  int64_t* fill = malloc(sizeof(int64_t) * n_faces);
  if (!fill) { omesh_free(m); return ORC_ERR_OOM; }
  for (int32_t f = 0; f < n_faces; ++f) fill[f] = m->face_start[f];
  for (int64_t k = 0; k < nt; ++k) m->face_tris[fill[tri_face[k]]++] = (int32_t)k;
  free(fill);

  for (int32_t f = 0; f < n_faces; ++f) {
    int64_t s = m->face_start[f], e = m->face_start[f + 1];
    if (e == s) { omesh_free(m); return ORC_ERR_ARG; }  /* a face with no triangle */
    double total = 0.0;
    for (int64_t q = s; q < e; ++q) total += tri_area_d(verts, &tris[3 * (int64_t)m->face_tris[q]]);
    if (!(total > 0.0)) { omesh_free(m); return ORC_ERR_ARG; }
    m->face_area[f] = total;
    double cum = 0.0;
    for (int64_t q = s; q < e; ++q) {
      cum += tri_area_d(verts, &tris[3 * (int64_t)m->face_tris[q]]);
      double scaled = floor(cum / total * 4294967296.0);
      m->face_thr[q] = (q == e - 1 || scaled >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)scaled;
    }
    int32_t k0 = m->face_tris[s];
    v3 c = vcross(m->te1[k0], m->te2[k0]);
    v3 n = vnormalize(c);
    v3 t = vnormalize(m->te1[k0]);
    m->fn[f] = n; m->ft[f] = t; m->fb[f] = vcross(n, t);
  }
  m->wound_like_face = 1;
  for (int64_t k = 0; k < nt; ++k)
    if (!(vdot(vcross(m->te1[k], m->te2[k]), m->fn[tri_face[k]]) > 0.0f)) m->wound_like_face = 0;
  /* origin lift from the bounding box diagonal */
  double lo[3] = {verts[0], verts[1], verts[2]}, hi[3] = {verts[0], verts[1], verts[2]};
  for (int64_t i = 0; i < nv; ++i)
    for (int c = 0; c < 3; ++c) {
      double x = verts[3 * i + c];
      if (x < lo[c]) lo[c] = x;
      if (x > hi[c]) hi[c] = x;
    }
  double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
  m->lift = (float)(1e-6 * sqrt((dx * dx + dy * dy) + dz * dz));
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Ray generation for ray `ray` of face `f`.                                  */
/* ------------------------------------------------------------------------ */
/* cos and sin of 2 pi t 2^-24 for t = 0 .. 2^24 - 1. The quadrant is t >> 22; in it the
   angle theta = (pi/2) w 2^-22, w = t mod 2^22, is folded to alpha = (pi/4) w' 2^-21 in
   [0, pi/4] (w' = w, or 2^22 - w with cos and sin swapped, theta = pi/2 - alpha), where
   sin alpha = alpha + alpha z (S1 + z (S2 + z (S3 + z S4))) and
   cos alpha = 1 + z (C1 + z (C2 + z (C3 + z (C4 + z C5)))), z = alpha^2, with the Taylor
   coefficients S_k = (-1)^k / (2k+1)!, C_k = (-1)^k / (2k)! rounded to float. */
static void unit_circle(uint32_t t, float* pc, float* ps) {
  uint32_t q = t >> 22, w = t & 0x3fffffu;
  int swap = w >= 0x200000u;
  float a = (float)(swap ? 0x400000u - w : w) * 0x1p-21f;   /* exact */
  float al = a * 0x1.921fb6p-1f;                             /* pi/4 */
  float z = al * al;
  float sp = 0x1.71de3ap-19f;
  sp = -0x1.a01a02p-13f + z * sp;
  sp = 0x1.111112p-7f + z * sp;
  sp = -0x1.555556p-3f + z * sp;
  float sn = al + (al * z) * sp;
  float cp = -0x1.27e4fcp-22f;
  cp = 0x1.a01a02p-16f + z * cp;
  cp = -0x1.6c16c2p-10f + z * cp;
  cp = 0x1.555556p-5f + z * cp;
  cp = -0.5f + z * cp;
  float cs = 1.0f + z * cp;
  float c = swap ? sn : cs, s = swap ? cs : sn;   /* cos, sin of theta */
  switch (q) {
    case 0: *pc = c; *ps = s; break;
    case 1: *pc = -s; *ps = c; break;
    case 2: *pc = -c; *ps = -s; break;
    default: *pc = s; *ps = -c; break;
  }
}

/* cos and sin of 2 pi t 2^-24 for t = t0 .. t0 + n - 1 (the sampling's unit circle, for
   its accuracy pin). */
int oracle_unit_circle(uint32_t t0, int64_t n, float* c_out, float* s_out) {
  if (n < 0 || (uint64_t)t0 + (uint64_t)n > (1ull << 24)) return ORC_ERR_ARG;
  for (int64_t k = 0; k < n; ++k) unit_circle(t0 + (uint32_t)k, &c_out[k], &s_out[k]);
  return ORC_OK;
}

/* Cosine-weighted (x, y, z) about +z from the emission draw x[0..3] (see the header). */
static void disc_direction(const uint32_t x[4], float* px, float* py, float* pz) {
  uint32_t sb = ((x[3] & 0xffu) << 24) | ((x[1] & 0xffu) << 16) | ((x[2] & 0xffu) << 8);
  float s = unit_float(sb);
  float c, sn;
  unit_circle(x[3] >> 8, &c, &sn);
  float r = sqrtf(s);
  *px = r * c;
  *py = r * sn;
  *pz = sqrtf(1.0f - s);
}

/* Emission from side `side` (0 = A, 1 = B) of face f with the draw of counter
   (ray, stream, base): triangle, point and direction. Side B uses the frame (t, -b, -n). Emission proper uses stream = f (side A)
   or f + 2^31 (side B) and base = 0; a reflection of bounce b uses stream = the path's
   source face and base = b*128. */
static void emit_side(const omesh* m, uint64_t seed, int32_t f, int side, uint32_t stream, uint32_t base,
                      uint64_t ray, v3* o, v3* d, int32_t* src_tri, int32_t* attempts_used) {
  uint32_t x[4];
  draw(seed, ray, stream, base, x);
  int64_t s = m->face_start[f], e = m->face_start[f + 1];
  int64_t q = e - 1;
  for (int64_t k = s; k < e; ++k) {
    if (x[0] < m->face_thr[k]) { q = k; break; }
  }
  int32_t tri = m->face_tris[q];
  float u = unit_float(x[1]), v = unit_float(x[2]);
  if (u + v > 1.0f) { u = 1.0f - u; v = 1.0f - v; }
  u = u * 0x1.ffffep-1f + 0x1.555556p-22f;   /* k = 1 - 2^-20, w = float(2^-20 / 3) */
  v = v * 0x1.ffffep-1f + 0x1.555556p-22f;
  v3 v0 = m->tv0[tri], e1 = m->te1[tri], e2 = m->te2[tri];
  v3 p;
  p.x = v0.x + u * e1.x; p.x = p.x + v * e2.x;
  p.y = v0.y + u * e1.y; p.y = p.y + v * e2.y;
  p.z = v0.z + u * e1.z; p.z = p.z + v * e2.z;
  v3 nf = m->fn[f];
  if (side) { nf.x = -nf.x; nf.y = -nf.y; nf.z = -nf.z; }
  p.x = p.x + m->lift * nf.x;
  p.y = p.y + m->lift * nf.y;
  p.z = p.z + m->lift * nf.z;

  float dx, dy, dz;
  int used = 0;  /* draws after the emission draw: none */
  disc_direction(x, &dx, &dy, &dz);
  v3 t = m->ft[f], b = m->fb[f], n = nf;
  if (side) { b.x = -b.x; b.y = -b.y; b.z = -b.z; }
  v3 dir;
  dir.x = dx * t.x + dy * b.x; dir.x = dir.x + dz * n.x;
  dir.y = dx * t.y + dy * b.y; dir.y = dir.y + dz * n.y;
  dir.z = dx * t.z + dy * b.z; dir.z = dir.z + dz * n.z;
  *o = p; *d = dir; *src_tri = tri;
  if (attempts_used) *attempts_used = used;
}

static void emit_from(const omesh* m, uint64_t seed, int32_t f, uint32_t stream, uint32_t base, uint64_t ray,
                      v3* o, v3* d, int32_t* src_tri, int32_t* attempts_used) {
  emit_side(m, seed, f, 0, stream, base, ray, o, d, src_tri, attempts_used);
}

static void sample_ray(const omesh* m, uint64_t seed, int32_t f, uint64_t ray, v3* o, v3* d,
                       int32_t* src_tri, int32_t* attempts_used) {
  emit_from(m, seed, f, (uint32_t)f, 0u, ray, o, d, src_tri, attempts_used);
}

/* Moller-Trumbore; returns 1 and t if the ray hits triangle k. */
static int intersect(const omesh* m, int32_t k, v3 o, v3 d, float* t_out) {
  const float eb_lo = -9.5367431640625e-07f;  /* -2^-20 */
  const float eb_hi = 1.00000095367431640625f; /* 1 + 2^-20 */
  v3 e1 = m->te1[k], e2 = m->te2[k];
  v3 pvec = vcross(d, e2);
  float det = vdot(e1, pvec);
  if (det == 0.0f) return 0;
  float inv = 1.0f / det;
  v3 tvec = vsub(o, m->tv0[k]);
  float u = vdot(tvec, pvec) * inv;
  if (!(u >= eb_lo && u <= eb_hi)) return 0;
  v3 qvec = vcross(tvec, e1);
  float v = vdot(d, qvec) * inv;
  if (!(v >= eb_lo && u + v <= eb_hi)) return 0;
  float t = vdot(e2, qvec) * inv;
  if (!(t > 0.0f)) return 0;
  *t_out = t;
  return 1;
}

/* Side of triangle k that a ray of direction d hits: 0 (A) when det = e1 . (d x e2) > 0,
   1 (B) otherwise; det is computed as in intersect(), where it is non-zero for a hit. */
static int hit_side(const omesh* m, int32_t k, v3 d) {
  return vdot(m->te1[k], vcross(d, m->te2[k])) > 0.0f ? 0 : 1;
}

static void consider(const omesh* m, int32_t k, int32_t src, v3 o, v3 d, float* best_t, int32_t* best_k) {
  if (k == src) return;
  float t;
  if (!intersect(m, k, o, d, &t)) return;
  if (t < *best_t || (t == *best_t && k < *best_k)) { *best_t = t; *best_k = k; }
}

/* ------------------------------------------------------------------------ */
/* Median-split BVH over triangle centroids (double boxes, padded).          */
/* ------------------------------------------------------------------------ */
typedef struct { double lo[3], hi[3]; int32_t left, right, first, count; } onode;
typedef struct { onode* nodes; int32_t n_nodes; int32_t* order; double pad; } obvh;

static const double* g_cent;  /* qsort context */
static int g_axis;
static int cmp_cent(const void* a, const void* b) {
  int32_t i = *(const int32_t*)a, j = *(const int32_t*)b;
  double ci = g_cent[3 * (int64_t)i + g_axis], cj = g_cent[3 * (int64_t)j + g_axis];
  if (ci < cj) return -1;
  if (ci > cj) return 1;
  return (i < j) ? -1 : (i > j);
}

static int32_t bvh_build_rec(obvh* b, const omesh* m, const double* cent, int32_t first, int32_t count) {
  int32_t id = b->n_nodes++;
  onode* nd = &b->nodes[id];
  for (int c = 0; c < 3; ++c) { nd->lo[c] = INFINITY; nd->hi[c] = -INFINITY; }
  for (int32_t q = first; q < first + count; ++q) {
    int32_t k = b->order[q];
    for (int v = 0; v < 3; ++v)
      for (int c = 0; c < 3; ++c) {
        double x = m->verts[3 * (int64_t)m->tris[3 * (int64_t)k + v] + c];
        if (x < nd->lo[c]) nd->lo[c] = x;
        if (x > nd->hi[c]) nd->hi[c] = x;
      }
  }
  for (int c = 0; c < 3; ++c) { nd->lo[c] -= b->pad; nd->hi[c] += b->pad; }
  if (count <= 4) {
    nd->left = nd->right = -1; nd->first = first; nd->count = count;
    return id;
  }
  double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int32_t q = first; q < first + count; ++q)
    for (int c = 0; c < 3; ++c) {
      double x = cent[3 * (int64_t)b->order[q] + c];
      if (x < clo[c]) clo[c] = x;
      if (x > chi[c]) chi[c] = x;
    }
  int axis = 0;
  for (int c = 1; c < 3; ++c) if (chi[c] - clo[c] > chi[axis] - clo[axis]) axis = c;
  g_cent = cent; g_axis = axis;
  qsort(&b->order[first], (size_t)count, sizeof(int32_t), cmp_cent);
  int32_t half = count / 2;
  int32_t l = bvh_build_rec(b, m, cent, first, half);
  int32_t r = bvh_build_rec(b, m, cent, first + half, count - half);
  nd = &b->nodes[id];
  nd->left = l; nd->right = r; nd->first = -1; nd->count = 0;
  return id;
}

static int bvh_build(obvh* b, const omesh* m) {
  int64_t nt = m->nt;
  b->nodes = malloc(sizeof(onode) * (size_t)(2 * nt + 1));
  b->order = malloc(sizeof(int32_t) * (size_t)nt);
  double* cent = malloc(sizeof(double) * 3 * (size_t)nt);
  if (!b->nodes || !b->order || !cent) { free(b->nodes); free(b->order); free(cent); return ORC_ERR_OOM; }
  for (int64_t k = 0; k < nt; ++k) {
    b->order[k] = (int32_t)k;
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int v = 0; v < 3; ++v) s += m->verts[3 * (int64_t)m->tris[3 * k + v] + c];
      cent[3 * k + c] = s / 3.0;
    }
  }
  /* padding: 1e-4 of the scene diagonal, far above float rounding of the hit point */
  b->pad = 1e-4 * ((double)m->lift / 1e-6);
  b->n_nodes = 0;
  bvh_build_rec(b, m, cent, 0, (int32_t)nt);
  free(cent);
  return ORC_OK;
}

/* slab test in double; returns the entry distance or +inf on a miss */
static double slab(const onode* nd, const double o[3], const double d[3], double t_lo, double t_hi) {
  double t0 = t_lo, t1 = t_hi;
  for (int c = 0; c < 3; ++c) {
    if (d[c] == 0.0) {
      if (o[c] < nd->lo[c] || o[c] > nd->hi[c]) return INFINITY;
      continue;
    }
    double a = (nd->lo[c] - o[c]) / d[c], b = (nd->hi[c] - o[c]) / d[c];
    if (a > b) { double tmp = a; a = b; b = tmp; }
    if (a > t0) t0 = a;
    if (b < t1) t1 = b;
    if (t0 > t1) return INFINITY;
  }
  return t0;
}

static void closest_bvh(const omesh* m, const obvh* b, int32_t src, v3 o, v3 d, float* best_t, int32_t* best_k) {
  int32_t stack[128];
  int sp = 0;
  stack[sp++] = 0;
  double od[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  while (sp > 0) {
    const onode* nd = &b->nodes[stack[--sp]];
    /* a node is skipped only if its padded box is entered strictly beyond the
       current best hit: every point within `pad` of a triangle is inside its
       box, so the box is entered at least `pad` before the triangle's t */
    double limit = isinf(*best_t) ? INFINITY : (double)*best_t;
    /* boxes left behind the origin by more than the padding cannot hold a hit */
    if (slab(nd, od, dd, -b->pad, limit) == INFINITY) continue;
    if (nd->left < 0) {
      for (int32_t q = nd->first; q < nd->first + nd->count; ++q)
        consider(m, b->order[q], src, o, d, best_t, best_k);
    } else {
      stack[sp++] = nd->left;
      stack[sp++] = nd->right;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Public entry points (C ABI, loaded through ctypes by the tests).           */
/* ------------------------------------------------------------------------ */

/* Face areas (double) and frames (float, 9 per face: t, b, n). */
int oracle_face_geometry(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                         const int32_t* tri_face, int32_t n_faces, double* area_out,
                         float* frame_out, uint32_t* thr_out, float* lift_out) {
  omesh m;
  int st = omesh_init(&m, verts, nv, tris, nt, tri_face, n_faces);
  if (st) return st;
  for (int32_t f = 0; f < n_faces; ++f) {
    if (area_out) area_out[f] = m.face_area[f];
    if (frame_out) {
      float* fr = &frame_out[9 * (int64_t)f];
      fr[0] = m.ft[f].x; fr[1] = m.ft[f].y; fr[2] = m.ft[f].z;
      fr[3] = m.fb[f].x; fr[4] = m.fb[f].y; fr[5] = m.fb[f].z;
      fr[6] = m.fn[f].x; fr[7] = m.fn[f].y; fr[8] = m.fn[f].z;
    }
  }
  if (thr_out) for (int64_t q = 0; q < nt; ++q) thr_out[m.face_tris[q]] = m.face_thr[q];
  if (lift_out) *lift_out = m.lift;
  omesh_free(&m);
  return ORC_OK;
}

/* Origins, directions and source triangles of rays [ray0, ray0+n) of face f. */
int oracle_sample_rays(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                       const int32_t* tri_face, int32_t n_faces, int32_t f, uint64_t seed,
                       uint64_t ray0, int64_t n, float* o_out, float* d_out, int32_t* tri_out,
                       int32_t* attempts_out) {
  omesh m;
  int st = omesh_init(&m, verts, nv, tris, nt, tri_face, n_faces);
  if (st) return st;
  if (f < 0 || f >= n_faces || n < 0) { omesh_free(&m); return ORC_ERR_ARG; }
  for (int64_t r = 0; r < n; ++r) {
    v3 o, d; int32_t tri, used;
    sample_ray(&m, seed, f, ray0 + (uint64_t)r, &o, &d, &tri, &used);
    o_out[3 * r] = o.x; o_out[3 * r + 1] = o.y; o_out[3 * r + 2] = o.z;
    d_out[3 * r] = d.x; d_out[3 * r + 1] = d.y; d_out[3 * r + 2] = d.z;
    tri_out[r] = tri;
    if (attempts_out) attempts_out[r] = used;
  }
  omesh_free(&m);
  return ORC_OK;
}

/* Closest hit of arbitrary rays by brute force (tri index or -1, and t). */
int oracle_closest_hits(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                        const int32_t* tri_face, int32_t n_faces, const float* o_in,
                        const float* d_in, const int32_t* src_tri, int64_t n, int32_t* hit_out,
                        float* t_out) {
  omesh m;
  int st = omesh_init(&m, verts, nv, tris, nt, tri_face, n_faces);
  if (st) return st;
  for (int64_t r = 0; r < n; ++r) {
    v3 o = {o_in[3 * r], o_in[3 * r + 1], o_in[3 * r + 2]};
    v3 d = {d_in[3 * r], d_in[3 * r + 1], d_in[3 * r + 2]};
    float bt = INFINITY; int32_t bk = -1;
    for (int64_t k = 0; k < nt; ++k) consider(&m, (int32_t)k, src_tri ? src_tri[r] : -1, o, d, &bt, &bk);
    hit_out[r] = bk; t_out[r] = bt;
  }
  omesh_free(&m);
  return ORC_OK;
}

/*
 * Hit counts N_ij (Eq. 3.15 numerators), accumulated into counts[n_faces*(n_faces+1)]
 * (row-major, column n_faces = environment). Rays of face f use ray indices
 * ray_offset .. ray_offset + rays_per_face[f] - 1. use_bvh = 0: every ray against
 * every triangle; 1: through the median-split BVH (same result by construction).
 * Rows are independent, so faces are spread over n_threads OpenMP threads.
 */
int oracle_trace_counts(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                        const int32_t* tri_face, int32_t n_faces, const int64_t* rays_per_face,
                        uint64_t seed, uint64_t ray_offset, int use_bvh, int n_threads,
                        const int32_t* face_subset, int32_t n_subset, int64_t* counts) {
  omesh m;
  int st = omesh_init(&m, verts, nv, tris, nt, tri_face, n_faces);
  if (st) return st;
  for (int32_t f = 0; f < n_faces; ++f)
    if (rays_per_face[f] < 0) { omesh_free(&m); return ORC_ERR_ARG; }
  obvh b; memset(&b, 0, sizeof(b));
  if (use_bvh) {
    st = bvh_build(&b, &m);
    if (st) { omesh_free(&m); return st; }
  }
  int32_t n_rows = face_subset ? n_subset : n_faces;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int32_t q = 0; q < n_rows; ++q) {
    int32_t f = face_subset ? face_subset[q] : q;
    int64_t* row = &counts[(int64_t)f * (n_faces + 1)];
    for (int64_t r = 0; r < rays_per_face[f]; ++r) {
      v3 o, d; int32_t src;
      sample_ray(&m, seed, f, ray_offset + (uint64_t)r, &o, &d, &src, NULL);
      float bt = INFINITY; int32_t bk = -1;
      if (use_bvh) closest_bvh(&m, &b, src, o, d, &bt, &bk);
      else for (int64_t k = 0; k < nt; ++k) consider(&m, (int32_t)k, src, o, d, &bt, &bk);
      row[bk < 0 ? n_faces : m.tri_face[bk]] += 1;
    }
  }
  free(b.nodes); free(b.order);
  omesh_free(&m);
  return ORC_OK;
}

/* Origins, directions and source triangles of rays [ray0, ray0+n) of side `side` of face f. */
int oracle_sample_rays_side(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                            const int32_t* tri_face, int32_t n_faces, int32_t f, int32_t side, uint64_t seed,
                            uint64_t ray0, int64_t n, float* o_out, float* d_out, int32_t* tri_out) {
  omesh m;
  int st = omesh_init(&m, verts, nv, tris, nt, tri_face, n_faces);
  if (st) return st;
  if (f < 0 || f >= n_faces || n < 0 || (side != 0 && side != 1)) { omesh_free(&m); return ORC_ERR_ARG; }
  const uint32_t stream = (uint32_t)f | ((uint32_t)side << 31);
  for (int64_t r = 0; r < n; ++r) {
    v3 o, d; int32_t tri;
    emit_side(&m, seed, f, side, stream, 0u, ray0 + (uint64_t)r, &o, &d, &tri, NULL);
    o_out[3 * r] = o.x; o_out[3 * r + 1] = o.y; o_out[3 * r + 2] = o.z;
    d_out[3 * r] = d.x; d_out[3 * r + 1] = d.y; d_out[3 * r + 2] = d.z;
    tri_out[r] = tri;
  }
  omesh_free(&m);
  return ORC_OK;
}

/*
 * Side-resolved hit counts (see the header), accumulated into
 * counts[2 n_faces * (2 n_faces + 1)]: row 2f+X = side X of face f, column 2g+Y = side Y
 * of face g, column 2 n_faces = environment. Side X of face f emits rays_per_side[2f+X]
 * rays with ray indices ray_offset, ray_offset + 1, ... Returns ORC_ERR_ARG when a
 * triangle is wound against its face.
 */
int oracle_trace_sided(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                       const int32_t* tri_face, int32_t n_faces, const int64_t* rays_per_side,
                       uint64_t seed, uint64_t ray_offset, int use_bvh, int n_threads,
                       const int32_t* row_subset, int32_t n_subset, int64_t* counts) {
  omesh m;
  int st = omesh_init(&m, verts, nv, tris, nt, tri_face, n_faces);
  if (st) return st;
  if (!m.wound_like_face || n_faces > (1 << 29)) { omesh_free(&m); return ORC_ERR_ARG; }
  const int32_t n_rows = 2 * n_faces, n_cols = 2 * n_faces + 1;
  for (int32_t q = 0; q < n_rows; ++q)
    if (rays_per_side[q] < 0) { omesh_free(&m); return ORC_ERR_ARG; }
  obvh b; memset(&b, 0, sizeof(b));
  if (use_bvh) {
    st = bvh_build(&b, &m);
    if (st) { omesh_free(&m); return st; }
  }
  int32_t n_work = row_subset ? n_subset : n_rows;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int32_t q = 0; q < n_work; ++q) {
    int32_t row = row_subset ? row_subset[q] : q;
    int32_t f = row >> 1, side = row & 1;
    const uint32_t stream = (uint32_t)f | ((uint32_t)side << 31);
    int64_t* out = &counts[(int64_t)row * n_cols];
    for (int64_t r = 0; r < rays_per_side[row]; ++r) {
      v3 o, d; int32_t src;
      emit_side(&m, seed, f, side, stream, 0u, ray_offset + (uint64_t)r, &o, &d, &src, NULL);
      float bt = INFINITY; int32_t bk = -1;
      if (use_bvh) closest_bvh(&m, &b, src, o, d, &bt, &bk);
      else for (int64_t k = 0; k < nt; ++k) consider(&m, (int32_t)k, src, o, d, &bt, &bk);
      out[bk < 0 ? n_rows : 2 * m.tri_face[bk] + hit_side(&m, bk, d)] += 1;
    }
  }
  free(b.nodes); free(b.order);
  omesh_free(&m);
  return ORC_OK;
}

/*
 * Direct Monte Carlo of Gebhart factors with diffuse reflections (see the header):
 * counts[i][j] += rays of face i absorbed on face j (column n_faces: escaped), with
 * per-face absorptivity eps[j] and diffuse reflectivity rho[j] (eps + rho <= 1).
 * stats (may be NULL) += {rays, bounces (hits), lost, overflow}.
 */
int oracle_trace_reflect(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                         const int32_t* tri_face, int32_t n_faces, const int64_t* rays_per_face,
                         const double* eps, const double* rho, int32_t max_bounces, uint64_t seed,
                         uint64_t ray_offset, int use_bvh, int n_threads, const int32_t* face_subset,
                         int32_t n_subset, int64_t* counts, int64_t* stats) {
  if (!eps || !rho || max_bounces < 1 || max_bounces >= (1 << 25)) return ORC_ERR_ARG;
  omesh m;
  int st = omesh_init(&m, verts, nv, tris, nt, tri_face, n_faces);
  if (st) return st;
  uint64_t* thr_a = malloc(sizeof(uint64_t) * n_faces);
  uint64_t* thr_r = malloc(sizeof(uint64_t) * n_faces);
  if (!thr_a || !thr_r) { free(thr_a); free(thr_r); omesh_free(&m); return ORC_ERR_OOM; }
  for (int32_t f = 0; f < n_faces; ++f) {
    double a = eps[f], r = rho[f];
    if (rays_per_face[f] < 0 || !(a >= 0.0 && r >= 0.0 && a + r <= 1.0)) {
      free(thr_a); free(thr_r); omesh_free(&m); return ORC_ERR_ARG;
    }
    thr_a[f] = (uint64_t)floor(a * 4294967296.0);
    thr_r[f] = (uint64_t)floor((a + r) * 4294967296.0);
  }
  obvh b; memset(&b, 0, sizeof(b));
  if (use_bvh) {
    st = bvh_build(&b, &m);
    if (st) { free(thr_a); free(thr_r); omesh_free(&m); return st; }
  }
  int32_t n_rows = face_subset ? n_subset : n_faces;
  int64_t n_rays = 0, n_hits = 0, n_lost = 0, n_over = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_rays, n_hits, n_lost, n_over)
#endif
  for (int32_t q = 0; q < n_rows; ++q) {
    int32_t f = face_subset ? face_subset[q] : q;
    int64_t* row = &counts[(int64_t)f * (n_faces + 1)];
    for (int64_t r = 0; r < rays_per_face[f]; ++r) {
      uint64_t ray = ray_offset + (uint64_t)r;
      v3 o, d; int32_t src;
      sample_ray(&m, seed, f, ray, &o, &d, &src, NULL);
      ++n_rays;
      for (int32_t bounce = 1;; ++bounce) {
        float bt = INFINITY; int32_t bk = -1;
        if (use_bvh) closest_bvh(&m, &b, src, o, d, &bt, &bk);
        else for (int64_t k = 0; k < nt; ++k) consider(&m, (int32_t)k, src, o, d, &bt, &bk);
        if (bk < 0) { row[n_faces] += 1; break; }
        ++n_hits;
        int32_t j = m.tri_face[bk];
        uint32_t x[4];
        const uint32_t base = (uint32_t)bounce << 7;
        draw(seed, ray, (uint32_t)f, base + 1u, x);  /* the decision; base itself re-emits */
        if ((uint64_t)x[3] < thr_a[j]) { row[j] += 1; break; }
        if ((uint64_t)x[3] >= thr_r[j]) { ++n_lost; break; }
        if (bounce >= max_bounces) { ++n_over; break; }
        /* diffuse reflection: re-emission from face j */
        emit_from(&m, seed, j, (uint32_t)f, base, ray, &o, &d, &src, NULL);
      }
    }
  }
  if (stats) { stats[0] += n_rays; stats[1] += n_hits; stats[2] += n_lost; stats[3] += n_over; }
  free(b.nodes); free(b.order); free(thr_a); free(thr_r);
  omesh_free(&m);
  return ORC_OK;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
