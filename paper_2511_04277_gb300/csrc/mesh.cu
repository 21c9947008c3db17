// Mesh upload: per-face emission data (area CDF, frame), a binned-SAH BVH built on
// the host, and the device records the trace kernel reads.
//
// The per-face data follow the ray definition of the MCRT estimator (Sec. 3.5.1):
//   - triangle areas in fp64: 0.5 |(v1-v0) x (v2-v0)| with the differences taken in fp64;
//   - CDF thresholds floor(cum_k / total * 2^32) over the face's triangles in index
//     order (the last one 0xFFFFFFFF); a ray takes the first triangle whose threshold
//     exceeds its 32-bit draw;
//   - frame from the face's lowest-index triangle: n = c/|c| with c = e1 x e2,
//     t = e1/|e1|, b = n x t, every float operation rounded on its own;
//   - origin lift off the face: 1e-6 of the bounding-box diagonal (float).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>

#include "mesh.cuh"

struct rg_mesh {
  rg_ctx* ctx = nullptr;
  DevMesh dev;
  std::vector<double> face_area;
  int64_t nt = 0;
  void* d_buf = nullptr;  // one allocation holding every device array
  void* d_bvh = nullptr;  // nodes and leaf-ordered records when the BVH was built on the device
};

const DevMesh& mesh_device_view(const rg_mesh* m) { return m->dev; }

// BVH depth from which the trace kernel refills finished lanes (measured on GB300: the
// 1,024-triangle plates, depth 8, run 1.5x faster lock-step; the 20,736- and
// 204,512-triangle spacecraft meshes, depths 14 and 19, run 3-7 % faster with refills).
constexpr int kRefillDepth = 12;
int mesh_device(const rg_mesh* m) { return m->ctx->device; }

namespace {

struct F3 {
  float x, y, z;
};
inline F3 f3sub(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline F3 f3cross(F3 a, F3 b) {
  F3 r;
  float p, q;
  p = a.y * b.z; q = a.z * b.y; r.x = p - q;
  p = a.z * b.x; q = a.x * b.z; r.y = p - q;
  p = a.x * b.y; q = a.y * b.x; r.z = p - q;
  return r;
}
inline float f3dot(F3 a, F3 b) {
  float s = a.x * b.x;
  float t = a.y * b.y;
  s = s + t;
  t = a.z * b.z;
  return s + t;
}
inline F3 f3unit(F3 a) {
  float len = std::sqrt(f3dot(a, a));
  return {a.x / len, a.y / len, a.z / len};
}

double area64(const float* v, const int32_t* t) {
  double d1[3], d2[3];
  for (int k = 0; k < 3; ++k) {
    double base = v[3 * (int64_t)t[0] + k];
    d1[k] = (double)v[3 * (int64_t)t[1] + k] - base;
    d2[k] = (double)v[3 * (int64_t)t[2] + k] - base;
  }
  double cx = d1[1] * d2[2] - d1[2] * d2[1];
  double cy = d1[2] * d2[0] - d1[0] * d2[2];
  double cz = d1[0] * d2[1] - d1[1] * d2[0];
  return 0.5 * std::sqrt((cx * cx + cy * cy) + cz * cz);
}

// ---------------------------------------------------------------- binned SAH BVH
struct Box {
  double lo[3], hi[3];
  void reset() {
    for (int c = 0; c < 3; ++c) { lo[c] = std::numeric_limits<double>::infinity(); hi[c] = -lo[c]; }
  }
  void grow(const Box& b) {
    for (int c = 0; c < 3; ++c) { lo[c] = std::min(lo[c], b.lo[c]); hi[c] = std::max(hi[c], b.hi[c]); }
  }
  void grow(const double* p) {
    for (int c = 0; c < 3; ++c) { lo[c] = std::min(lo[c], p[c]); hi[c] = std::max(hi[c], p[c]); }
  }
  double half_area() const {
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = std::max(0.0, hi[c] - lo[c]);
    return d[0] * d[1] + d[1] * d[2] + d[2] * d[0];
  }
};

struct BuildNode {
  Box box[2];
  int32_t ref[2];
  int32_t count[2];
};

// Binned SAH split of a range of triangles. The binning is float arithmetic, the cost
// fp64; bvh_gpu.cu evaluates the same expressions in the same order, so both builders
// make the same splits and build the same tree:
//   centroid c = 0.5f * (lo + hi) per axis (float box of the float vertices);
//   per axis with extent x = max c - min c > 0 (float): scale = 16.0f / x and bin
//   k = (int)((c - min c) * scale), clamped to [0, 15];
//   cost of the split before bin k: area(left) * n_left + area(right) * n_right with
//   area = dx dy + dy dz + dz dx of the fp64 box, bins swept from 15 down to 1, axes
//   0..2, the first strictly smallest cost taken;
//   the left side takes the bins below the chosen one; when no split separates the
//   range, its (e - b) / 2 smallest (centroid on the widest axis, triangle index).
inline float bin_scale(float ext) { return 16.0f / ext; }
inline int bin_of(float c, float lo, float scale) {
  int k = (int)((c - lo) * scale);
  return std::min(std::max(k, 0), 15);
}

struct Builder {
  const std::vector<Box>& tbox;
  const std::vector<float>& cent;  // 3 per triangle
  std::vector<int32_t>& order;
  std::vector<BuildNode> nodes;
  int max_depth = 0;
  Builder(const std::vector<Box>& tb, const std::vector<float>& c, std::vector<int32_t>& o)
      : tbox(tb), cent(c), order(o) {}

  Box range_box(int32_t b, int32_t e) const {
    Box r; r.reset();
    for (int32_t q = b; q < e; ++q) r.grow(tbox[order[q]]);
    return r;
  }

  // Split [b, e) and return the split index.
  int32_t split(int32_t b, int32_t e) {
    constexpr int kBins = 16;
    float clo[3], chi[3];
    for (int c = 0; c < 3; ++c) { clo[c] = std::numeric_limits<float>::infinity(); chi[c] = -clo[c]; }
    for (int32_t q = b; q < e; ++q)
      for (int c = 0; c < 3; ++c) {
        const float x = cent[3 * (size_t)order[q] + c];
        clo[c] = std::min(clo[c], x); chi[c] = std::max(chi[c], x);
      }
    float ext[3], scale[3];
    for (int c = 0; c < 3; ++c) {
      ext[c] = chi[c] - clo[c];
      scale[c] = ext[c] > 0.0f ? bin_scale(ext[c]) : 0.0f;
    }
    double best = std::numeric_limits<double>::infinity();
    int best_axis = -1, best_bin = -1;
    for (int ax = 0; ax < 3; ++ax) {
      if (!(ext[ax] > 0.0f)) continue;
      Box bb[kBins];
      int cnt[kBins] = {0};
      for (int k = 0; k < kBins; ++k) bb[k].reset();
      for (int32_t q = b; q < e; ++q) {
        const int k = bin_of(cent[3 * (size_t)order[q] + ax], clo[ax], scale[ax]);
        cnt[k]++;
        bb[k].grow(tbox[order[q]]);
      }
      double left_area[kBins];
      int left_cnt[kBins];
      Box acc; acc.reset();
      int c = 0;
      for (int k = 0; k < kBins; ++k) {
        acc.grow(bb[k]); c += cnt[k];
        left_area[k] = acc.half_area(); left_cnt[k] = c;
      }
      acc.reset(); c = 0;
      for (int k = kBins - 1; k >= 1; --k) {
        acc.grow(bb[k]); c += cnt[k];
        if (left_cnt[k - 1] == 0 || c == 0) continue;
        double cost = left_area[k - 1] * left_cnt[k - 1] + acc.half_area() * c;
        if (cost < best) { best = cost; best_axis = ax; best_bin = k; }
      }
    }
    int32_t mid;
    if (best_axis >= 0) {
      auto it = std::partition(order.begin() + b, order.begin() + e, [&](int32_t t) {
        return bin_of(cent[3 * (size_t)t + best_axis], clo[best_axis], scale[best_axis]) < best_bin;
      });
      mid = (int32_t)(it - order.begin());
      if (mid > b && mid < e) return mid;
    }
    // degenerate centroids: median split along the widest axis
    int ax = 0;
    for (int c2 = 1; c2 < 3; ++c2)
      if (ext[c2] > ext[ax]) ax = c2;
    mid = b + (e - b) / 2;
    std::nth_element(order.begin() + b, order.begin() + mid, order.begin() + e, [&](int32_t x, int32_t y) {
      const float cx = cent[3 * (size_t)x + ax], cy = cent[3 * (size_t)y + ax];
      return cx < cy || (cx == cy && x < y);
    });
    return mid;
  }

  // Build the subtree over [b, e) (e - b > 4) and return its node index.
  int32_t build(int32_t b, int32_t e, int depth) {
    max_depth = std::max(max_depth, depth);
    int32_t id = (int32_t)nodes.size();
    nodes.emplace_back();
    int32_t mid = split(b, e);
    int32_t rb[2] = {b, mid}, re[2] = {mid, e};
    for (int s = 0; s < 2; ++s) {
      Box bx = range_box(rb[s], re[s]);
      int32_t ref, cnt;
      if (re[s] - rb[s] <= 4) {
        ref = rb[s]; cnt = re[s] - rb[s];
      } else {
        ref = build(rb[s], re[s], depth + 1); cnt = 0;
      }
      nodes[id].box[s] = bx;
      nodes[id].ref[s] = ref;
      nodes[id].count[s] = cnt;
    }
    return id;
  }
};

inline float round_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
  return f;
}
inline float round_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, std::numeric_limits<float>::infinity());
  return f;
}

void pack_tri(float4* dst, F3 v0, F3 e1, F3 e2, int32_t id, int32_t face) {
  dst[0] = make_float4(v0.x, v0.y, v0.z, e1.x);
  dst[1] = make_float4(e1.y, e1.z, e2.x, e2.y);
  float idf, ff;
  std::memcpy(&idf, &id, 4);
  std::memcpy(&ff, &face, 4);
  dst[2] = make_float4(e2.z, idf, ff, 0.f);
}

}  // namespace

// on_device: build the BVH on the GPU (bvh_gpu.cu), the same tree as the host builder's.
static rg_status mesh_create(rg_ctx* ctx, const float* verts_h, int64_t nv, const int32_t* tris_h, int64_t nt,
                             const int32_t* tri_face_h, int32_t n_faces, int32_t use_bvh, bool on_device,
                             rg_mesh** mesh_out) {
  if (!ctx) return RG_ERR_ARG;
  RG_ARG_CHECK(ctx, mesh_out && verts_h && tris_h && tri_face_h, "rg_mesh_create: NULL argument");
  RG_ARG_CHECK(ctx, nv > 0 && nt > 0 && n_faces > 0, "rg_mesh_create: empty mesh");
  RG_ARG_CHECK(ctx, nt < (int64_t)1 << 30 && nv < (int64_t)1 << 31, "rg_mesh_create: mesh too large");
  *mesh_out = nullptr;
  for (int64_t k = 0; k < nt; ++k) {
    RG_ARG_CHECK(ctx, tri_face_h[k] >= 0 && tri_face_h[k] < n_faces, "triangle %lld: face %d out of range",
                 (long long)k, tri_face_h[k]);
    for (int c = 0; c < 3; ++c)
      RG_ARG_CHECK(ctx, tris_h[3 * k + c] >= 0 && tris_h[3 * k + c] < nv, "triangle %lld: bad vertex index",
                   (long long)k);
  }
  auto V = [&](int32_t i) { return F3{verts_h[3 * (int64_t)i], verts_h[3 * (int64_t)i + 1], verts_h[3 * (int64_t)i + 2]}; };
  std::vector<F3> tv0(nt), te1(nt), te2(nt);
  for (int64_t k = 0; k < nt; ++k) {
    F3 a = V(tris_h[3 * k]), b = V(tris_h[3 * k + 1]), c = V(tris_h[3 * k + 2]);
    tv0[k] = a; te1[k] = f3sub(b, a); te2[k] = f3sub(c, a);
  }
  // faces: triangles in ascending index order
  std::vector<int64_t> fstart(n_faces + 1, 0);
  for (int64_t k = 0; k < nt; ++k) fstart[tri_face_h[k] + 1]++;
  for (int32_t f = 0; f < n_faces; ++f) fstart[f + 1] += fstart[f];
  std::vector<int32_t> ftris(nt);
  {
    std::vector<int64_t> fill(fstart.begin(), fstart.end() - 1);
    for (int64_t k = 0; k < nt; ++k) ftris[fill[tri_face_h[k]]++] = (int32_t)k;
  }
  std::vector<uint32_t> thr(nt);
  std::vector<float> frames(9 * (size_t)n_faces);
  std::vector<double> farea(n_faces);
  for (int32_t f = 0; f < n_faces; ++f) {
    int64_t s = fstart[f], e = fstart[f + 1];
    RG_ARG_CHECK(ctx, e > s, "face %d has no triangle", f);
    double total = 0.0;
    for (int64_t q = s; q < e; ++q) total += area64(verts_h, &tris_h[3 * (int64_t)ftris[q]]);
    RG_ARG_CHECK(ctx, total > 0.0, "face %d has zero area", f);
    farea[f] = total;
    double cum = 0.0;
    for (int64_t q = s; q < e; ++q) {
      cum += area64(verts_h, &tris_h[3 * (int64_t)ftris[q]]);
      double scaled = std::floor(cum / total * 4294967296.0);
      thr[q] = (q == e - 1 || scaled >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)scaled;
    }
    int32_t k0 = ftris[s];
    F3 n = f3unit(f3cross(te1[k0], te2[k0]));
    F3 t = f3unit(te1[k0]);
    F3 b = f3cross(n, t);
    float* fr = &frames[9 * (size_t)f];
    fr[0] = t.x; fr[1] = t.y; fr[2] = t.z; fr[3] = b.x; fr[4] = b.y; fr[5] = b.z;
    fr[6] = n.x; fr[7] = n.y; fr[8] = n.z;
  }
  // side-resolved tracing takes the side of a hit from the triangle's own winding, so it
  // needs every triangle's normal e1 x e2 on its face's side A
  int32_t wound_like_face = 1;
  for (int64_t k = 0; k < nt; ++k) {
    const float* fr = &frames[9 * (size_t)tri_face_h[k]];
    if (!(f3dot(f3cross(te1[k], te2[k]), F3{fr[6], fr[7], fr[8]}) > 0.0f)) wound_like_face = 0;
  }
  // scene scale
  double lo[3], hi[3];
  for (int c = 0; c < 3; ++c) lo[c] = hi[c] = verts_h[c];
  for (int64_t i = 0; i < nv; ++i)
    for (int c = 0; c < 3; ++c) {
      double x = verts_h[3 * i + c];
      lo[c] = std::min(lo[c], x); hi[c] = std::max(hi[c], x);
    }
  double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
  double diag = std::sqrt((dx * dx + dy * dy) + dz * dz);
  float lift = (float)(1e-6 * diag);

  RG_ARG_CHECK(ctx, use_bvh >= -1 && use_bvh <= 3, "rg_mesh_create: use_bvh = %d", use_bvh);
  const int schedule = use_bvh;  // 2: force lock-step, 3: force refill
  if (use_bvh < 0) use_bvh = nt > 64 ? 1 : 0;
  if (use_bvh > 1) use_bvh = 1;
  if (nt <= 4) use_bvh = 0;

  // triangle records in traversal order
  std::vector<int32_t> order(nt);
  std::iota(order.begin(), order.end(), 0);
  std::vector<BuildNode> nodes;
  int depth = 0;
  float sah_visits = 0.f;
  GpuBvh gb;
  const bool on_gpu = use_bvh && on_device;
  if (on_gpu) {
    for (int64_t i = 0; i < 3 * nv; ++i)
      RG_ARG_CHECK(ctx, std::isfinite(verts_h[i]), "rg_mesh_create_gpu_bvh: vertex %lld is not finite",
                   (long long)(i / 3));
    rg_status st = gpu_bvh_build(ctx, verts_h, nv, tris_h, tri_face_h, nt, diag, &gb);
    if (st != RG_OK) {
      if (gb.buf) cudaFree(gb.buf);
      return st;
    }
    depth = gb.depth;
    sah_visits = gb.sah_visits;
  } else if (use_bvh) {
    std::vector<Box> tbox(nt);
    std::vector<float> cent(3 * (size_t)nt);
    for (int64_t k = 0; k < nt; ++k) {
      tbox[k].reset();
      for (int v = 0; v < 3; ++v) {
        double p[3];
        for (int c = 0; c < 3; ++c) p[c] = verts_h[3 * (int64_t)tris_h[3 * k + v] + c];
        tbox[k].grow(p);
      }
      for (int c = 0; c < 3; ++c) cent[3 * k + c] = 0.5f * ((float)tbox[k].lo[c] + (float)tbox[k].hi[c]);
    }
    Builder bld(tbox, cent, order);
    bld.build(0, (int32_t)nt, 1);
    depth = bld.max_depth;
    nodes.swap(bld.nodes);
    // expected node visits of a random line: a box is hit with probability proportional
    // to its surface area (Cauchy); the root is always visited
    Box root = nodes[0].box[0];
    root.grow(nodes[0].box[1]);
    const double sa_root = root.half_area();
    double visits = 1.0;
    for (const BuildNode& nd : nodes)
      for (int c = 0; c < 2; ++c)
        if (nd.count[c] == 0 && sa_root > 0) visits += nd.box[c].half_area() / sa_root;
    sah_visits = (float)visits;
    if (depth + 1 > kTraceStack)
      return rg::fail(ctx, RG_ERR_STACK, "BVH depth %d exceeds the traversal stack (%d)", depth, kTraceStack);
  }
  // padded float boxes: axes along which a child's triangles have extent get a wide
  // pad (1e-4 of the scene diagonal, far above the rounding of the accepted hit
  // points); axes where the child is flat get a tight one (outward rounding), so
  // that a flat child holding the ray's own face lies behind the lifted origin and
  // falls outside the traversal window [-lift/2, best_t + slack]
  const double pad_wide = 1e-4 * diag, pad_flat = 1e-9 * diag;
  std::vector<float4> hnodes(on_gpu ? 0 : 4 * nodes.size());
  for (size_t i = 0; i < hnodes.size() / 4; ++i) {
    float l[2][3], h[2][3];
    for (int s = 0; s < 2; ++s)
      for (int c = 0; c < 3; ++c) {
        const Box& bx = nodes[i].box[s];
        double pad = (bx.hi[c] - bx.lo[c] > 0) ? pad_wide : pad_flat;
        l[s][c] = round_down(bx.lo[c] - pad);
        h[s][c] = round_up(bx.hi[c] + pad);
      }
    hnodes[4 * i + 0] = make_float4(l[0][0], h[0][0], l[0][1], h[0][1]);
    hnodes[4 * i + 1] = make_float4(l[1][0], h[1][0], l[1][1], h[1][1]);
    hnodes[4 * i + 2] = make_float4(l[0][2], h[0][2], l[1][2], h[1][2]);
    int32_t iv[4] = {nodes[i].ref[0], nodes[i].ref[1], nodes[i].count[0], nodes[i].count[1]};
    float fv[4];
    std::memcpy(fv, iv, 16);
    hnodes[4 * i + 3] = make_float4(fv[0], fv[1], fv[2], fv[3]);
  }
  std::vector<float4> htris(on_gpu ? 0 : 3 * (size_t)nt), hetris(3 * (size_t)nt);
  for (int64_t q = 0; q < nt; ++q) {
    int32_t k = order[q];
    if (!on_gpu) pack_tri(&htris[3 * q], tv0[k], te1[k], te2[k], k, tri_face_h[k]);
    int32_t kf = ftris[q];
    pack_tri(&hetris[3 * q], tv0[kf], te1[kf], te2[kf], kf, tri_face_h[kf]);
  }

  rg_mesh* m = new (std::nothrow) rg_mesh();
  if (!m) {
    if (gb.buf) cudaFree(gb.buf);
    return rg::fail(ctx, RG_ERR_OOM, "rg_mesh_create: host allocation");
  }
  m->ctx = ctx;
  m->d_bvh = gb.buf;
  m->nt = nt;
  m->face_area = farea;
  rg::Sizer sz;
  sz.take<float4>(hnodes.size()); sz.take<float4>(htris.size()); sz.take<float4>(hetris.size());
  sz.take<uint32_t>(nt); sz.take<int64_t>(n_faces + 1); sz.take<float>(frames.size());
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_buf, sz.off);
  if (e != cudaSuccess) {
    if (m->d_bvh) cudaFree(m->d_bvh);
    delete m;
    return rg::cuda_fail(ctx, e, "rg_mesh_create: cudaMalloc");
  }
  rg::Carver cv(m->d_buf);
  float4* d_nodes = cv.take<float4>(hnodes.size());
  float4* d_tris = cv.take<float4>(htris.size());
  float4* d_etris = cv.take<float4>(hetris.size());
  uint32_t* d_thr = cv.take<uint32_t>(nt);
  int64_t* d_fstart = cv.take<int64_t>(n_faces + 1);
  float* d_frames = cv.take<float>(frames.size());
  struct Up { void* d; const void* h; size_t n; } ups[] = {
      {d_nodes, hnodes.data(), hnodes.size() * sizeof(float4)},
      {d_tris, htris.data(), htris.size() * sizeof(float4)},
      {d_etris, hetris.data(), hetris.size() * sizeof(float4)},
      {d_thr, thr.data(), thr.size() * sizeof(uint32_t)},
      {d_fstart, fstart.data(), fstart.size() * sizeof(int64_t)},
      {d_frames, frames.data(), frames.size() * sizeof(float)}};
  for (auto& u : ups) {
    if (u.n == 0) continue;
    e = cudaMemcpy(u.d, u.h, u.n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(m->d_buf);
      if (m->d_bvh) cudaFree(m->d_bvh);
      delete m;
      return rg::cuda_fail(ctx, e, "rg_mesh_create: upload");
    }
  }
  DevMesh& d = m->dev;
  d.n_faces = n_faces; d.nt = nt; d.use_bvh = use_bvh;
  d.n_nodes = on_gpu ? gb.n_nodes : (int32_t)nodes.size();
  d.depth = depth;
  d.lift = lift; d.t_lo = -0.5f * lift; d.slack = (float)(1e-5 * diag);
  d.sah_visits = sah_visits;
  d.wound_like_face = wound_like_face;
  // refill scheduling pays off when traversals are long; short ones run lock-step
  d.refill = schedule == 3 ? 1 : (schedule == 2 ? 0 : (depth >= kRefillDepth ? 1 : 0));
  d.nodes = on_gpu ? gb.nodes : d_nodes;
  d.tris = on_gpu ? gb.tris : d_tris;
  d.etris = d_etris; d.ethr = d_thr; d.face_start = d_fstart;
  d.frames = d_frames;
  *mesh_out = m;
  return RG_OK;
}

extern "C" {

rg_status rg_mesh_create(rg_ctx* ctx, const float* verts_h, int64_t nv, const int32_t* tris_h, int64_t nt,
                         const int32_t* tri_face_h, int32_t n_faces, int32_t use_bvh, rg_mesh** mesh_out) {
  return mesh_create(ctx, verts_h, nv, tris_h, nt, tri_face_h, n_faces, use_bvh, false, mesh_out);
}

rg_status rg_mesh_create_gpu_bvh(rg_ctx* ctx, const float* verts_h, int64_t nv, const int32_t* tris_h, int64_t nt,
                                 const int32_t* tri_face_h, int32_t n_faces, int32_t use_bvh, rg_mesh** mesh_out) {
  return mesh_create(ctx, verts_h, nv, tris_h, nt, tri_face_h, n_faces, use_bvh, true, mesh_out);
}

rg_status rg_mesh_get_bvh(const rg_mesh* mesh, float* nodes_h, int32_t* record_tri_h) {
  if (!mesh) return RG_ERR_ARG;
  const DevMesh& d = mesh->dev;
  if (cudaSetDevice(mesh->ctx->device) != cudaSuccess) return RG_ERR_CUDA;
  if (nodes_h && d.use_bvh && d.n_nodes > 0 &&
      cudaMemcpy(nodes_h, d.nodes, 4 * (size_t)d.n_nodes * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RG_ERR_CUDA;
  if (record_tri_h) {
    std::vector<float4> rec(3 * (size_t)d.nt);
    if (cudaMemcpy(rec.data(), d.tris, rec.size() * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess)
      return RG_ERR_CUDA;
    for (int64_t q = 0; q < d.nt; ++q) std::memcpy(&record_tri_h[q], &rec[3 * q + 2].y, sizeof(int32_t));
  }
  return RG_OK;
}

rg_status rg_mesh_destroy(rg_mesh* mesh) {
  if (!mesh) return RG_ERR_ARG;
  cudaSetDevice(mesh->ctx->device);
  cudaDeviceSynchronize();
  if (mesh->d_buf) cudaFree(mesh->d_buf);
  if (mesh->d_bvh) cudaFree(mesh->d_bvh);
  delete mesh;
  return RG_OK;
}

rg_status rg_mesh_get_info(const rg_mesh* mesh, rg_mesh_info* info) {
  if (!mesh || !info) return RG_ERR_ARG;
  info->n_faces = mesh->dev.n_faces;
  info->n_tris = mesh->nt;
  info->bvh_nodes = mesh->dev.use_bvh ? mesh->dev.n_nodes : 0;
  info->bvh_depth = mesh->dev.use_bvh ? mesh->dev.depth : 0;
  info->lift = mesh->dev.lift;
  info->sah_visits = mesh->dev.sah_visits;
  info->refill = mesh->dev.refill;
  return RG_OK;
}

rg_status rg_face_areas(const rg_mesh* mesh, double* areas_out_h) {
  if (!mesh || !areas_out_h) return RG_ERR_ARG;
  std::memcpy(areas_out_h, mesh->face_area.data(), mesh->face_area.size() * sizeof(double));
  return RG_OK;
}

}  // extern "C"
