// Device construction of the triangle BVH that the trace kernels traverse (the
// acceleration structure of the MCRT estimator, Sec. 3.5.1): the alternative to the
// host binned-SAH builder of mesh.cu, for large meshes.
//
// Algorithm: parallel locally-ordered clustering (PLOC; Meister and Bittner, IEEE TVCG
// 24(3), 2018), whose merge criterion is the surface area of a node's box, the cost the
// surface-area heuristic charges for visiting it:
//   1. triangle boxes (exact float min/max of the vertices) and the bounds of their
//      centroids;
//   2. 30-bit Morton codes of the centroids, sorted together with the triangle indices
//      by a stable LSD radix sort (four 8-bit digits), so equal codes keep index order;
//   3. the sorted triangles are the initial clusters. In every iteration each cluster
//      takes as its nearest neighbour the cluster, among the `radius` on either side in
//      the current list, whose union box has the smallest surface area, comparing pairs
//      by (area, lower position, higher position); under that total order the smallest
//      pair in the list is mutual, so every iteration merges at least one pair. Mutual
//      neighbours merge into a new node at the lower position (left child = the lower
//      one), the other one leaves the list, and the list is compacted. Nodes are numbered
//      n, n+1, ... in creation order; the last one is the root;
//   4. newest nodes first, every node hands its children their first record (left child
//      first) and their depth, so that the triangles of every subtree are contiguous
//      records;
//   5. nodes holding more than 4 triangles become BVH nodes in the traversal layout of
//      mesh.cuh, numbered in depth-first preorder (root 0, a left subtree before its
//      right sibling, as the host builder numbers them: a subtree's nodes are
//      contiguous); smaller subtrees become leaves of their parent. Child boxes get the host builder's padding (1e-4 of the scene
//      diagonal on axes with extent, 1e-9 on flat ones, rounded outward).
// Every step is deterministic: sums are integer scans in a fixed order and the only
// atomics are integer min / max, so a mesh always gets the same BVH.
#include <climits>
#include <cmath>
#include <utility>
#include <vector>

#include "mesh.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 1024;        // radix-sort keys per block: four rounds of 256
constexpr int kScanItems = 4;      // prefix sums: items per thread, 1,024 per block
constexpr int kScanBlock = kThreads * kScanItems;
static_assert(kThreads == 256, "one thread per radix digit");

inline int grid_of(int64_t n, int per) {
  const int64_t g = (n + per - 1) / per;
  return (int)(g < 1 ? 1 : g);
}
inline int grid_capped(int64_t n, int sm) {
  const int64_t g = (n + kThreads - 1) / kThreads, cap = (int64_t)sm * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// float <-> unsigned with the same order (for integer atomic min / max)
__device__ __forceinline__ unsigned f2ord(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ---------------------------------------------------------------- prefix sums
// Exclusive prefix of v over the block's threads; *total = the block's sum.
__device__ int32_t block_exclusive_scan(int32_t v, int32_t* s_warp, int32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t t = lane < kThreads / 32 ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kThreads / 32) s_warp[lane] = t;
  }
  __syncthreads();
  const int32_t before = w ? s_warp[w - 1] : 0;
  *total = s_warp[kThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// Block-local exclusive prefix of 1,024 items per block; bsum[b] = the block's sum.
// In place (in == out) is allowed: a thread reads its items before writing them.
__global__ void __launch_bounds__(kThreads) scan_local(const int32_t* in, int32_t* out, int64_t n, int32_t* bsum) {
  __shared__ int32_t s_warp[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems], sum = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    sum += v[k];
  }
  int32_t total;
  int32_t run = block_exclusive_scan(sum, s_warp, &total);
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void scan_add(int32_t* out, int64_t n, const int32_t* bsum) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] += bsum[i / kScanBlock];
}

__global__ void scan_total(const int32_t* in, const int32_t* out, int64_t n, int32_t* total) {
  *total = out[n - 1] + in[n - 1];
}

struct Scanner {
  int32_t* ws;  // room for the block sums of every level
  int sm;
  int64_t* launches;
  // out = exclusive prefix sums of in (in != out), *total_d = their sum (device)
  void run(const int32_t* in, int32_t* out, int64_t n, int32_t* total_d, cudaStream_t s) {
    level(in, out, n, ws, s);
    scan_total<<<1, 1, 0, s>>>(in, out, n, total_d);
    ++*launches;
  }
  void level(const int32_t* in, int32_t* out, int64_t n, int32_t* bs, cudaStream_t s) {
    const int nb = grid_of(n, kScanBlock);
    scan_local<<<nb, kThreads, 0, s>>>(in, out, n, bs);
    ++*launches;
    if (nb > 1) {
      level(bs, bs, nb, bs + ((nb + 63) & ~63), s);
      scan_add<<<grid_capped(n, sm), kThreads, 0, s>>>(out, n, bs);
      ++*launches;
    }
  }
  static int64_t ints_needed(int64_t n) {
    int64_t t = 0;
    while (true) {
      const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
      t += (nb + 63) & ~63;
      if (nb <= 1) break;
      n = nb;
    }
    return t + 64;
  }
};

// ---------------------------------------------------------------- boxes and codes
__global__ void tri_bounds(const float* __restrict__ V, const int32_t* __restrict__ T, int64_t nt,
                           float4* __restrict__ tlo, float4* __restrict__ thi, unsigned* __restrict__ cb) {
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    float p[3][3];
    for (int v = 0; v < 3; ++v) {
      const int64_t vi = 3 * (int64_t)T[3 * i + v];
      p[v][0] = V[vi]; p[v][1] = V[vi + 1]; p[v][2] = V[vi + 2];
    }
    float lo[3], hi[3];
    for (int c = 0; c < 3; ++c) {
      lo[c] = fminf(fminf(p[0][c], p[1][c]), p[2][c]);
      hi[c] = fmaxf(fmaxf(p[0][c], p[1][c]), p[2][c]);
      const float ce = __fmul_rn(0.5f, __fadd_rn(lo[c], hi[c]));
      mn[c] = fminf(mn[c], ce);
      mx[c] = fmaxf(mx[c], ce);
    }
    tlo[i] = make_float4(lo[0], lo[1], lo[2], 0.f);
    thi[i] = make_float4(hi[0], hi[1], hi[2], 0.f);
  }
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) {
      mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
      mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
    }
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 3; ++c) {
      if (mn[c] <= mx[c]) {
        atomicMin(cb + c, f2ord(mn[c]));
        atomicMax(cb + 3 + c, f2ord(mx[c]));
      }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {  // bit k of x -> bit 3k
  x &= 1023u;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__global__ void morton_codes(const float4* __restrict__ tlo, const float4* __restrict__ thi, int64_t nt,
                             const unsigned* __restrict__ cb, uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  float mn[3], sc[3];
  for (int c = 0; c < 3; ++c) {
    mn[c] = ord2f(cb[c]);
    const float ext = ord2f(cb[3 + c]) - mn[c];
    sc[c] = ext > 0.f ? 1024.f / ext : 0.f;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = tlo[i], b = thi[i];
    const float ce[3] = {__fmul_rn(0.5f, __fadd_rn(a.x, b.x)), __fmul_rn(0.5f, __fadd_rn(a.y, b.y)),
                         __fmul_rn(0.5f, __fadd_rn(a.z, b.z))};
    uint32_t q[3];
    for (int c = 0; c < 3; ++c) {
      const float t = __fmul_rn(__fsub_rn(ce[c], mn[c]), sc[c]);
      q[c] = t <= 0.f ? 0u : (t >= 1023.f ? 1023u : (uint32_t)t);
    }
    keys[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    vals[i] = (int32_t)i;
  }
}

// ---------------------------------------------------------------- radix sort
__global__ void __launch_bounds__(kThreads) rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                    int32_t n_tiles, int32_t* __restrict__ hist) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int k = threadIdx.x; k < kTile; k += kThreads) {
    const int64_t i = base + k;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: four rounds of 256 keys in index order; within a round a
// key's rank is the number of equal digits before it (earlier warps, then earlier lanes).
__global__ void __launch_bounds__(kThreads) rs_scatter(const uint32_t* __restrict__ kin,
                                                       const int32_t* __restrict__ vin, int64_t n, int shift,
                                                       int32_t n_tiles, const int32_t* __restrict__ offs,
                                                       uint32_t* __restrict__ kout, int32_t* __restrict__ vout,
                                                       int32_t* err) {
  __shared__ int32_t s_cnt[kThreads / 32][256];
  __shared__ int32_t s_run[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  s_run[threadIdx.x] = offs[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int r = 0; r < kTile / kThreads; ++r) {
    for (int q = threadIdx.x; q < (kThreads / 32) * 256; q += kThreads) (&s_cnt[0][0])[q] = 0;
    __syncthreads();
    const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
    const bool has = i < n;
    const uint32_t key = has ? kin[i] : 0u;
    const int32_t val = has ? vin[i] : 0;
    const uint32_t d = (key >> shift) & 255u;
    const unsigned act = __ballot_sync(0xffffffffu, has);
    int rank = 0;
    if (has) {
      const unsigned peers = __match_any_sync(act, d);
      rank = __popc(peers & lt);
      if (rank == 0) s_cnt[w][d] = __popc(peers);
    }
    __syncthreads();
    {  // thread t turns digit t's per-warp counts into output positions
      int32_t run = s_run[threadIdx.x];
      for (int ww = 0; ww < kThreads / 32; ++ww) {
        const int32_t c = s_cnt[ww][threadIdx.x];
        s_cnt[ww][threadIdx.x] = run;
        run += c;
      }
      s_run[threadIdx.x] = run;
    }
    __syncthreads();
    if (has) {
      const int32_t pos = s_cnt[w][d] + rank;
      if (pos >= 0 && pos < n) {
        kout[pos] = key;
        vout[pos] = val;
      } else {
        atomicExch(err, 1);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- clustering
__global__ void gather_leaves(const int32_t* __restrict__ perm, int64_t n, const float4* __restrict__ tlo,
                              const float4* __restrict__ thi, float4* __restrict__ blo, float4* __restrict__ bhi,
                              int32_t* __restrict__ size, int32_t* __restrict__ ecount, int32_t* __restrict__ C) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = perm[q];
    blo[q] = tlo[t];
    bhi[q] = thi[t];
    size[q] = 1;
    ecount[q] = 0;
    C[q] = (int32_t)q;
  }
}

__device__ __forceinline__ float union_half_area(float4 alo, float4 ahi, float4 blo, float4 bhi) {
  const float dx = __fsub_rn(fmaxf(ahi.x, bhi.x), fminf(alo.x, blo.x));
  const float dy = __fsub_rn(fmaxf(ahi.y, bhi.y), fminf(alo.y, blo.y));
  const float dz = __fsub_rn(fmaxf(ahi.z, bhi.z), fminf(alo.z, blo.z));
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
}

__global__ void ploc_nearest(const int32_t* __restrict__ C, int32_t count, const float4* __restrict__ blo,
                             const float4* __restrict__ bhi, int32_t radius, int32_t* __restrict__ nn) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const int32_t ci = C[i];
    const float4 alo = blo[ci], ahi = bhi[ci];
    float best = INFINITY;
    int32_t bj = -1, blo_i = INT_MAX, bhi_i = INT_MAX;
    const int32_t j0 = max(0, i - radius), j1 = min(count - 1, i + radius);
    for (int32_t j = j0; j <= j1; ++j) {
      if (j == i) continue;
      const int32_t cj = C[j];
      const float d = union_half_area(alo, ahi, blo[cj], bhi[cj]);
      const int32_t pl = min(i, j), ph = max(i, j);
      if (d < best || (d == best && (pl < blo_i || (pl == blo_i && ph < bhi_i)))) {
        best = d;
        bj = j;
        blo_i = pl;
        bhi_i = ph;
      }
    }
    nn[i] = bj;
  }
}

__global__ void ploc_flags(const int32_t* __restrict__ nn, int32_t count, int32_t* __restrict__ created,
                           int32_t* __restrict__ removed) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const int32_t j = nn[i];
    const bool mutual = nn[j] == i;
    created[i] = mutual && i < j;
    removed[i] = mutual && i > j;
  }
}

__global__ void ploc_merge(const int32_t* __restrict__ C, int32_t count, const int32_t* __restrict__ nn,
                           const int32_t* __restrict__ created, const int32_t* __restrict__ crank,
                           const int32_t* __restrict__ removed, const int32_t* __restrict__ rprefix, int32_t n,
                           int32_t next_id, float4* __restrict__ blo, float4* __restrict__ bhi,
                           int32_t* __restrict__ size, int32_t* __restrict__ ecount, int32_t* __restrict__ child,
                           int32_t* __restrict__ Cout) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    if (removed[i]) continue;
    const int32_t pos = i - rprefix[i];
    if (created[i]) {
      const int32_t id = next_id + crank[i];
      const int32_t a = C[i], b = C[nn[i]];
      const float4 al = blo[a], ah = bhi[a], bl = blo[b], bh = bhi[b];
      blo[id] = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.f);
      bhi[id] = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.f);
      size[id] = size[a] + size[b];
      // BVH nodes in the new subtree: itself (when it holds more than 4 triangles) and its children's
      ecount[id] = (size[id] > 4 ? 1 : 0) + ecount[a] + ecount[b];
      child[2 * (int64_t)(id - n)] = a;
      child[2 * (int64_t)(id - n) + 1] = b;
      Cout[pos] = id;
    } else {
      Cout[pos] = C[i];
    }
  }
}

// ---------------------------------------------------------------- layout
__global__ void set_root(int32_t root, int32_t* off, int32_t* depth, int32_t* pre) {
  off[root] = 0;
  depth[root] = 1;
  pre[root] = 0;
}

// A node hands its children their first record, depth and preorder number (meaningful
// for the children that become BVH nodes: the left one follows its parent, the right
// one follows the left one's subtree).
__global__ void top_down(int32_t id0, int32_t id1, int32_t n, const int32_t* __restrict__ child,
                         const int32_t* __restrict__ size, const int32_t* __restrict__ ecount,
                         int32_t* __restrict__ off, int32_t* __restrict__ depth, int32_t* __restrict__ pre) {
  for (int32_t x = id0 + blockIdx.x * blockDim.x + threadIdx.x; x < id1; x += gridDim.x * blockDim.x) {
    const int32_t l = child[2 * (int64_t)(x - n)], r = child[2 * (int64_t)(x - n) + 1];
    const int32_t o = off[x], d = depth[x] + 1, p = pre[x] + 1;
    off[l] = o;
    off[r] = o + size[l];
    depth[l] = d;
    depth[r] = d;
    pre[l] = p;
    pre[r] = p + ecount[l];
  }
}

// Depth of the deepest internal node that becomes a BVH node (more than 4 triangles).
__global__ void max_node_depth(int32_t n, const int32_t* __restrict__ size, const int32_t* __restrict__ depth,
                               int32_t* __restrict__ max_depth) {
  for (int32_t id = n + blockIdx.x * blockDim.x + threadIdx.x; id < 2 * n - 1; id += gridDim.x * blockDim.x)
    if (size[id] > 4) atomicMax(max_depth, depth[id]);
}

__device__ __forceinline__ void pad_box(float4 lo, float4 hi, double wide, double flat, float* l, float* h) {
  const float a[3] = {lo.x, lo.y, lo.z}, b[3] = {hi.x, hi.y, hi.z};
  for (int c = 0; c < 3; ++c) {
    const double dl = a[c], dh = b[c];
    const double pad = dh - dl > 0.0 ? wide : flat;
    l[c] = __double2float_rd(dl - pad);
    h[c] = __double2float_ru(dh + pad);
  }
}

__global__ void emit_nodes(int32_t n, const int32_t* __restrict__ size, const int32_t* __restrict__ child,
                           const int32_t* __restrict__ off, const int32_t* __restrict__ pre,
                           const float4* __restrict__ blo, const float4* __restrict__ bhi, double wide, double flat,
                           int32_t n_emit, float4* __restrict__ nodes, int32_t* err) {
  for (int32_t id = n + blockIdx.x * blockDim.x + threadIdx.x; id < 2 * n - 1; id += gridDim.x * blockDim.x) {
    if (size[id] <= 4) continue;
    const int32_t me = pre[id];
    if (me < 0 || me >= n_emit) {
      atomicExch(err, 1);
      continue;
    }
    float l[2][3], h[2][3];
    int32_t ref[2], cnt[2];
    for (int s = 0; s < 2; ++s) {
      const int32_t c = child[2 * (int64_t)(id - n) + s];
      if (size[c] <= 4) {
        ref[s] = off[c];
        cnt[s] = size[c];
      } else {
        ref[s] = pre[c];
        cnt[s] = 0;
      }
      pad_box(blo[c], bhi[c], wide, flat, l[s], h[s]);
    }
    float4* o = nodes + 4 * (int64_t)me;
    o[0] = make_float4(l[0][0], h[0][0], l[0][1], h[0][1]);
    o[1] = make_float4(l[1][0], h[1][0], l[1][1], h[1][1]);
    o[2] = make_float4(l[0][2], h[0][2], l[1][2], h[1][2]);
    o[3] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(cnt[0]), __int_as_float(cnt[1]));
  }
}

// Triangle records (v0, e1, e2, id, face) at the positions the layout gave the leaves.
__global__ void emit_records(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ off,
                             const float* __restrict__ V, const int32_t* __restrict__ T,
                             const int32_t* __restrict__ TF, float4* __restrict__ rec, int32_t* err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = perm[q];
    const int64_t pos = off[q];
    if (pos < 0 || pos >= n || t < 0 || t >= n) {
      atomicExch(err, 1);
      continue;
    }
    float p[3][3];
    for (int v = 0; v < 3; ++v) {
      const int64_t vi = 3 * (int64_t)T[3 * (int64_t)t + v];
      p[v][0] = V[vi]; p[v][1] = V[vi + 1]; p[v][2] = V[vi + 2];
    }
    float e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
      e1[c] = __fsub_rn(p[1][c], p[0][c]);
      e2[c] = __fsub_rn(p[2][c], p[0][c]);
    }
    rec[3 * pos] = make_float4(p[0][0], p[0][1], p[0][2], e1[0]);
    rec[3 * pos + 1] = make_float4(e1[1], e1[2], e2[0], e2[1]);
    rec[3 * pos + 2] = make_float4(e2[2], __int_as_float(t), __int_as_float(TF[t]), 0.f);
  }
}

__device__ __forceinline__ double half_area_d(float4 lo, float4 hi) {
  const double dx = fmax(0.0, (double)hi.x - lo.x), dy = fmax(0.0, (double)hi.y - lo.y),
               dz = fmax(0.0, (double)hi.z - lo.z);
  return dx * dy + dy * dz + dz * dx;
}

// 1 + sum over BVH-node children that are BVH nodes of area(child) / area(root): the
// expected node visits of a random line, summed in a fixed order (one block).
__global__ void __launch_bounds__(1024) sah_visits_kernel(int32_t n, const int32_t* __restrict__ size,
                                                          const int32_t* __restrict__ child,
                                                          const float4* __restrict__ blo,
                                                          const float4* __restrict__ bhi, double* out) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int32_t id = n + threadIdx.x; id < 2 * n - 1; id += blockDim.x) {
    if (size[id] <= 4) continue;
    for (int s = 0; s < 2; ++s) {
      const int32_t c = child[2 * (int64_t)(id - n) + s];
      if (size[c] > 4) acc += half_area_d(blo[c], bhi[c]);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int32_t root = 2 * n - 2;
    const double ra = half_area_d(blo[root], bhi[root]);
    out[0] = ra > 0.0 ? 1.0 + red[0] / ra : 1.0;
  }
}

}  // namespace

rg_status gpu_bvh_build(rg_ctx* ctx, const float* verts_h, int64_t nv, const int32_t* tris_h,
                        const int32_t* tri_face_h, int64_t nt, double diag, int32_t radius, GpuBvh* out) {
  *out = GpuBvh{};
  RG_ARG_CHECK(ctx, nt > 4 && nt < (int64_t)1 << 30, "gpu BVH: %lld triangles", (long long)nt);
  RG_ARG_CHECK(ctx, radius >= 1 && radius <= 256, "gpu BVH: radius %d outside [1, 256]", radius);
  const int32_t n = (int32_t)nt;
  const int32_t n_nodes_all = 2 * n - 1;
  const int32_t n_tiles = (int32_t)((nt + kTile - 1) / kTile);
  cudaStream_t s = 0;
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // the context workspace may still be read by queued work of earlier calls
  RG_CUDA_TRY(ctx, cudaDeviceSynchronize());

  rg::Sizer sz;
  sz.take<float>(3 * (size_t)nv); sz.take<int32_t>(3 * (size_t)nt); sz.take<int32_t>(nt);
  sz.take<float4>(nt); sz.take<float4>(nt); sz.take<unsigned>(8);
  sz.take<uint32_t>(nt); sz.take<uint32_t>(nt); sz.take<int32_t>(nt); sz.take<int32_t>(nt);
  sz.take<int32_t>(256 * (size_t)n_tiles); sz.take<int32_t>(256 * (size_t)n_tiles);
  sz.take<float4>(n_nodes_all); sz.take<float4>(n_nodes_all);
  for (int k = 0; k < 5; ++k) sz.take<int32_t>(n_nodes_all);  // size, off, depth, ecount, pre
  sz.take<int32_t>(2 * (size_t)n);                             // child
  for (int k = 0; k < 7; ++k) sz.take<int32_t>(nt);            // C0, C1, nn, created, removed, crank, rprefix
  sz.take<int32_t>(Scanner::ints_needed(256 * (int64_t)n_tiles > nt ? 256 * (int64_t)n_tiles : nt));
  sz.take<int32_t>(8); sz.take<double>(1);
  void* ws = nullptr;
  rg_status st = rg::workspace(ctx, sz.off, &ws);
  if (st != RG_OK) return st;
  rg::Carver cv(ws);
  float* dV = cv.take<float>(3 * (size_t)nv);
  int32_t* dT = cv.take<int32_t>(3 * (size_t)nt);
  int32_t* dTF = cv.take<int32_t>(nt);
  float4* tlo = cv.take<float4>(nt);
  float4* thi = cv.take<float4>(nt);
  unsigned* cb = cv.take<unsigned>(8);
  uint32_t* k0 = cv.take<uint32_t>(nt);
  uint32_t* k1 = cv.take<uint32_t>(nt);
  int32_t* v0 = cv.take<int32_t>(nt);
  int32_t* v1 = cv.take<int32_t>(nt);
  int32_t* hist = cv.take<int32_t>(256 * (size_t)n_tiles);
  int32_t* offs = cv.take<int32_t>(256 * (size_t)n_tiles);
  float4* blo = cv.take<float4>(n_nodes_all);
  float4* bhi = cv.take<float4>(n_nodes_all);
  int32_t* size = cv.take<int32_t>(n_nodes_all);
  int32_t* off = cv.take<int32_t>(n_nodes_all);
  int32_t* depth = cv.take<int32_t>(n_nodes_all);
  int32_t* ecount = cv.take<int32_t>(n_nodes_all);
  int32_t* pre = cv.take<int32_t>(n_nodes_all);
  int32_t* child = cv.take<int32_t>(2 * (size_t)n);
  int32_t* C0 = cv.take<int32_t>(nt);
  int32_t* C1 = cv.take<int32_t>(nt);
  int32_t* nn = cv.take<int32_t>(nt);
  int32_t* created = cv.take<int32_t>(nt);
  int32_t* removed = cv.take<int32_t>(nt);
  int32_t* crank = cv.take<int32_t>(nt);
  int32_t* rprefix = cv.take<int32_t>(nt);
  int32_t* scan_ws = cv.take<int32_t>(Scanner::ints_needed(256 * (int64_t)n_tiles > nt ? 256 * (int64_t)n_tiles : nt));
  int32_t* tot = cv.take<int32_t>(8);
  double* d_sah = cv.take<double>(1);
  Scanner scan{scan_ws, ctx->sm_count, &ctx->launches};
  const int sm = ctx->sm_count;

  RG_CUDA_TRY(ctx, cudaMemcpyAsync(dV, verts_h, 3 * (size_t)nv * sizeof(float), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(dT, tris_h, 3 * (size_t)nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(dTF, tri_face_h, (size_t)nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  // centroid bounds start at (+max, -max) in the ordered encoding
  const unsigned init[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0u, 0u};
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(cb, init, sizeof(init), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(tot, 0, 8 * sizeof(int32_t), s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(off, 0xff, (size_t)n_nodes_all * sizeof(int32_t), s));  // -1: not placed

  tri_bounds<<<grid_capped(nt, sm), kThreads, 0, s>>>(dV, dT, nt, tlo, thi, cb);
  morton_codes<<<grid_capped(nt, sm), kThreads, 0, s>>>(tlo, thi, nt, cb, k0, v0);
  ctx->launches += 2;
  for (int shift = 0; shift < 30; shift += 8) {
    rs_hist<<<n_tiles, kThreads, 0, s>>>(k0, nt, shift, n_tiles, hist);
    scan.run(hist, offs, 256 * (int64_t)n_tiles, tot + 7, s);
    rs_scatter<<<n_tiles, kThreads, 0, s>>>(k0, v0, nt, shift, n_tiles, offs, k1, v1, tot + 5);
    ctx->launches += 2;
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  int32_t* perm = v0;  // triangle index of sorted position q
  gather_leaves<<<grid_capped(nt, sm), kThreads, 0, s>>>(perm, nt, tlo, thi, blo, bhi, size, ecount, C0);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());

  std::vector<int32_t> bases{n};
  int32_t count = n, next_id = n;
  while (count > 1) {
    const int g = grid_capped(count, sm);
    ploc_nearest<<<g, kThreads, 0, s>>>(C0, count, blo, bhi, radius, nn);
    ploc_flags<<<g, kThreads, 0, s>>>(nn, count, created, removed);
    ctx->launches += 2;
    scan.run(created, crank, count, tot, s);
    scan.run(removed, rprefix, count, tot + 1, s);
    ploc_merge<<<g, kThreads, 0, s>>>(C0, count, nn, created, crank, removed, rprefix, n, next_id, blo, bhi, size,
                                      ecount, child, C1);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, tot, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const int32_t made = ctx->h_scratch[0];
    if (made <= 0 || made > count / 2)
      return rg::fail(ctx, RG_ERR_NUMERIC, "gpu BVH: an iteration merged %d of %d clusters", made, count);
    next_id += made;
    count -= made;
    bases.push_back(next_id);
    std::swap(C0, C1);
  }
  const int32_t root = next_id - 1;
  if (root != 2 * n - 2) return rg::fail(ctx, RG_ERR_NUMERIC, "gpu BVH: %d nodes for %d triangles", root + 1, n);
  set_root<<<1, 1, 0, s>>>(root, off, depth, pre);
  ++ctx->launches;
  for (size_t k = bases.size() - 1; k-- > 0;) {
    const int32_t a = bases[k], b = bases[k + 1];
    top_down<<<grid_capped(b - a, sm), kThreads, 0, s>>>(a, b, n, child, size, ecount, off, depth, pre);
    ++ctx->launches;
  }
  max_node_depth<<<grid_capped(n - 1, sm), kThreads, 0, s>>>(n, size, depth, tot + 2);
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(tot + 3, ecount + root, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  sah_visits_kernel<<<1, 1024, 0, s>>>(n, size, child, blo, bhi, d_sah);
  ctx->launches += 2;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  int32_t h_tot[4];
  double h_sah = 0.0;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(h_tot, tot, sizeof(h_tot), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h_sah, d_sah, sizeof(double), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  const int32_t n_emit = h_tot[3];
  out->n_nodes = n_emit;
  out->depth = h_tot[2];
  out->sah_visits = (float)h_sah;
  if (n_emit < 1) return rg::fail(ctx, RG_ERR_NUMERIC, "gpu BVH: no node");
  if (out->depth + 1 > kTraceStack)
    return rg::fail(ctx, RG_ERR_STACK, "BVH depth %d exceeds the traversal stack (%d)", out->depth, kTraceStack);

  RG_CUDA_TRY(ctx, cudaMalloc(&out->buf, (4 * (size_t)n_emit + 3 * (size_t)nt) * sizeof(float4)));
  out->nodes = static_cast<float4*>(out->buf);
  out->tris = out->nodes + 4 * (size_t)n_emit;
  emit_nodes<<<grid_capped(n - 1, sm), kThreads, 0, s>>>(n, size, child, off, pre, blo, bhi, 1e-4 * diag,
                                                          1e-9 * diag, n_emit, out->nodes, tot + 5);
  emit_records<<<grid_capped(nt, sm), kThreads, 0, s>>>(nt, perm, off, dV, dT, dTF, out->tris, tot + 5);
  ctx->launches += 2;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, tot + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (ctx->h_scratch[0]) return rg::fail(ctx, RG_ERR_NUMERIC, "gpu BVH: a layout index fell out of range");
  return RG_OK;
}
