// Device-side mesh layout shared by mesh.cu (builder/upload) and trace.cu (kernel).
#pragma once
#include "common.cuh"

// Triangle record used by intersection: three float4 =
//   (v0.x, v0.y, v0.z, e1.x) (e1.y, e1.z, e2.x, e2.y) (e2.z, id bits, face bits, 0)
// with e1 = v1 - v0 and e2 = v2 - v0 in float32.
//
// BVH node (two children per node, child boxes stored in the parent), four float4:
//   n0 = (L.lo.x, L.hi.x, L.lo.y, L.hi.y)   n1 = (R.lo.x, R.hi.x, R.lo.y, R.hi.y)
//   n2 = (L.lo.z, L.hi.z, R.lo.z, R.hi.z)   n3 = int(L.ref, R.ref, L.count, R.count)
// count == 0: ref is an inner node index; count > 0: ref is the first triangle record
// of a leaf of `count` records.
struct DevMesh {
  int32_t n_faces = 0;
  int64_t nt = 0;
  int32_t use_bvh = 0;
  int32_t n_nodes = 0;
  int32_t depth = 0;
  float lift = 0.f;       // origins are lifted this far off the face along its normal
  float t_lo = 0.f;       // lower end of the traversal window (-lift / 2)
  float slack = 0.f;      // the window's upper end is best_t + slack
  int32_t refill = 0;     // 1: refill scheduling of the trace kernel, 0: lock-step
  float sah_visits = 0.f; // expected node visits of a random line (surface-area heuristic)
  int32_t wound_like_face = 0;  // 1: every triangle's e1 x e2 points to its face's side A
  const float4* nodes = nullptr;
  const float4* tris = nullptr;     // nt records in leaf order (BVH) or index order
  const float4* etris = nullptr;    // nt records in face order (emission)
  const uint32_t* ethr = nullptr;   // area-CDF threshold of each face-ordered record
  const int64_t* face_start = nullptr;  // [N+1] offsets into etris/ethr
  const float* frames = nullptr;    // [N][9]: t, b, n
};

constexpr int kTraceStack = 64;

// BVH built on the device (bvh_gpu.cu): n_nodes nodes in the layout above and nt
// triangle records in leaf order, both in `buf` (cudaMalloc'd, owned by the mesh).
struct GpuBvh {
  int32_t n_nodes = 0;
  int32_t depth = 0;
  float sah_visits = 0.f;
  void* buf = nullptr;
  float4* nodes = nullptr;
  float4* tris = nullptr;
};
rg_status gpu_bvh_build(rg_ctx* ctx, const float* verts_h, int64_t nv, const int32_t* tris_h,
                        const int32_t* tri_face_h, int64_t nt, double diag, GpuBvh* out);

struct rg_mesh_impl;
const DevMesh& mesh_device_view(const rg_mesh* m);
int mesh_device(const rg_mesh* m);
