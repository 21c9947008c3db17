// Device construction of the triangle BVH that the trace kernels traverse (the
// acceleration structure of the MCRT estimator, Sec. 3.5.1): the host builder of mesh.cu
// (binned surface-area heuristic, 16 bins, leaves of at most 4 triangles) run on the GPU,
// level by level.
//
// Every level is one launch with one block per range of triangles still to split. The
// block takes the range's centroid bounds, fills the 3 x 16 bins (count and box, warp
// lanes of one bin combined before the shared-memory atomics), evaluates the split costs
// in one thread in the host builder's order and arithmetic (float binning, fp64 costs,
// no contraction), partitions the range stably into the second triangle-order array
// (block prefix sums), takes the two children's boxes, and finishes children of at most 4
// triangles as leaves. A prefix sum over the ranges numbers the next level's ranges. The
// splits are the host's, and a child's records occupy the same positions as there (only
// the order inside a leaf may differ, the host partition being unstable), so the node
// array equals the host builder's bit for bit. Nodes are numbered depth-first (root 0, a
// left subtree before its right sibling) from subtree sizes summed bottom-up; boxes get
// the host's padding. Deterministic: no floating-point atomics, no order-dependent sums.
#include <cmath>
#include <utility>
#include <vector>

#include "mesh.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kScanItems = 4;      // prefix sums: items per thread, 1,024 per block
constexpr int kScanBlock = kThreads * kScanItems;
constexpr int kBins = 16;
constexpr int kMaxLevels = kTraceStack - 1;  // the root is level 1; depth + 1 <= the traversal stack

inline int grid_of(int64_t n, int per) {
  const int64_t g = (n + per - 1) / per;
  return (int)(g < 1 ? 1 : g);
}
inline int grid_capped(int64_t n, int sm) {
  const int64_t g = (n + kThreads - 1) / kThreads, cap = (int64_t)sm * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// float <-> unsigned with the same order (for integer min / max reductions and atomics)
__device__ __forceinline__ unsigned f2ord(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
constexpr unsigned kOrdPosInf = 0xff800000u;  // f2ord(+inf)
constexpr unsigned kOrdNegInf = 0x007fffffu;  // f2ord(-inf)

// ---------------------------------------------------------------- prefix sums
// Exclusive prefix of v over the block's TB threads; *total = the block's sum.
template <int TB = kThreads>
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
    int32_t t = lane < TB / 32 ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < TB / 32) s_warp[lane] = t;
  }
  __syncthreads();
  const int32_t before = w ? s_warp[w - 1] : 0;
  *total = s_warp[TB / 32 - 1];
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


// ---------------------------------------------------------------- per-triangle data
__global__ void tri_boxes(const float* __restrict__ V, const int32_t* __restrict__ T, int64_t nt,
                          float4* __restrict__ tlo, float4* __restrict__ thi, float4* __restrict__ cen,
                          int32_t* __restrict__ ord) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    float p[3][3];
    for (int v = 0; v < 3; ++v) {
      const int64_t vi = 3 * (int64_t)T[3 * i + v];
      p[v][0] = V[vi]; p[v][1] = V[vi + 1]; p[v][2] = V[vi + 2];
    }
    float lo[3], hi[3], c[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(fminf(p[0][a], p[1][a]), p[2][a]);
      hi[a] = fmaxf(fmaxf(p[0][a], p[1][a]), p[2][a]);
      c[a] = __fmul_rn(0.5f, __fadd_rn(lo[a], hi[a]));
    }
    tlo[i] = make_float4(lo[0], lo[1], lo[2], 0.f);
    thi[i] = make_float4(hi[0], hi[1], hi[2], 0.f);
    cen[i] = make_float4(c[0], c[1], c[2], 0.f);
    ord[i] = (int32_t)i;
  }
}

// ---------------------------------------------------------------- one level of splits
struct Seg {
  int32_t b, e;   // triangle-order range, e - b > 4
  int32_t node;   // breadth-first node number
  int32_t depth;  // root 1
};

struct BNode {  // a node as the host builder makes it, before numbering and padding
  float lo[2][3], hi[2][3];  // child boxes (union of their triangles' boxes)
  int32_t ref[2], cnt[2];    // leaf child: first record and count; inner child: its node number, 0
  int32_t mid;               // first record of the right child
};

__device__ __forceinline__ int bin_of(float c, float lo, float scale) {
  const int k = (int)__fmul_rn(__fsub_rn(c, lo), scale);
  return min(max(k, 0), kBins - 1);
}

__device__ __forceinline__ double half_area(const double lo[3], const double hi[3]) {
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = fmax(0.0, __dsub_rn(hi[a], lo[a]));
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[1]), __dmul_rn(d[1], d[2])), __dmul_rn(d[2], d[0]));
}

// Block-wide min and max of six ordered-float values (lo xyz, hi xyz); result in out[6].
template <int TB>
__device__ void block_minmax6(unsigned v[6], unsigned* s_red /* [TB/32][6] */, unsigned* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < 6; ++k) {
    unsigned x = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned y = __shfl_xor_sync(0xffffffffu, x, o);
      x = k < 3 ? min(x, y) : max(x, y);
    }
    if (lane == 0) s_red[w * 6 + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    unsigned x = s_red[k];
    for (int ww = 1; ww < TB / 32; ++ww) x = k < 3 ? min(x, s_red[ww * 6 + k]) : max(x, s_red[ww * 6 + k]);
    out[k] = x;
  }
  __syncthreads();
}

// TB threads per block: 1,024 on the top levels (few, large ranges), 256 below.
template <int TB>
__global__ void __launch_bounds__(TB, 1) sah_split_level(
    const Seg* __restrict__ segs, const float4* __restrict__ tlo, const float4* __restrict__ thi,
    const float4* __restrict__ cen, const int32_t* __restrict__ ord_in, int32_t* __restrict__ ord_out,
    int32_t* __restrict__ ord_final, uint8_t* __restrict__ flag, BNode* __restrict__ nodes,
    int32_t* __restrict__ n_inner, int32_t* __restrict__ err) {
  __shared__ int32_t s_cnt[3][kBins];
  __shared__ unsigned s_box[3][kBins][6];  // ordered lo xyz, hi xyz
  __shared__ unsigned s_red[(TB / 32) * 6];
  __shared__ unsigned s_cb[6], s_child[2][6];
  __shared__ int32_t s_warp[TB / 32];
  __shared__ int s_axis, s_bin, s_mode, s_left;
  __shared__ float s_clo[3], s_scale[3], s_ext[3];
  __shared__ double s_cost[3];
  __shared__ int s_cbin[3];
  const Seg sg = segs[blockIdx.x];
  const int32_t b = sg.b, e = sg.e, n = e - b;
  const int lane = threadIdx.x & 31;

  // centroid bounds of the range
  {
    unsigned v[6] = {kOrdPosInf, kOrdPosInf, kOrdPosInf, kOrdNegInf, kOrdNegInf, kOrdNegInf};
    for (int32_t q = b + threadIdx.x; q < e; q += TB) {
      const float4 c = cen[ord_in[q]];
      const float cc[3] = {c.x, c.y, c.z};
      for (int a = 0; a < 3; ++a) {
        v[a] = min(v[a], f2ord(cc[a]));
        v[3 + a] = max(v[3 + a], f2ord(cc[a]));
      }
    }
    block_minmax6<TB>(v, s_red, s_cb);
  }
  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    const float lo = ord2f(s_cb[a]), ext = __fsub_rn(ord2f(s_cb[3 + a]), lo);
    s_clo[a] = lo;
    s_ext[a] = ext;
    s_scale[a] = ext > 0.0f ? __fdiv_rn(16.0f, ext) : 0.0f;
  }
  for (int k = threadIdx.x; k < 3 * kBins; k += TB) {
    (&s_cnt[0][0])[k] = 0;
    for (int j = 0; j < 6; ++j) (&s_box[0][0][0])[6 * k + j] = j < 3 ? kOrdPosInf : kOrdNegInf;
  }
  __syncthreads();

  // bins: lanes of a warp that fall into the same bin are combined first
  for (int32_t base = b; base < e; base += TB) {
    const int32_t q = base + threadIdx.x;
    const bool has = q < e;
    const unsigned act = __ballot_sync(0xffffffffu, has);
    if (has) {
      const int32_t t = ord_in[q];
      const float4 c = cen[t], lo = tlo[t], hi = thi[t];
      const float cc[3] = {c.x, c.y, c.z};
      const unsigned bx[6] = {f2ord(lo.x), f2ord(lo.y), f2ord(lo.z), f2ord(hi.x), f2ord(hi.y), f2ord(hi.z)};
      for (int a = 0; a < 3; ++a) {
        if (!(s_ext[a] > 0.0f)) continue;
        const int k = bin_of(cc[a], s_clo[a], s_scale[a]);
        const unsigned peers = __match_any_sync(act, k);
        unsigned r[6];
        for (int j = 0; j < 3; ++j) r[j] = __reduce_min_sync(peers, bx[j]);
        for (int j = 3; j < 6; ++j) r[j] = __reduce_max_sync(peers, bx[j]);
        if (lane == __ffs(peers) - 1) {
          atomicAdd(&s_cnt[a][k], __popc(peers));
          for (int j = 0; j < 3; ++j) atomicMin(&s_box[a][k][j], r[j]);
          for (int j = 3; j < 6; ++j) atomicMax(&s_box[a][k][j], r[j]);
        }
      }
    }
  }
  __syncthreads();

  // split costs: warp a takes axis a, lane k bin k; box unions and counts by prefix
  // (bins 0..k) and suffix (bins k..15) shuffles; lane k costs the split before bin k
  // with the host builder's expression. The host takes, over axes 0..2 and bins 15..1,
  // the first strictly smallest cost: per axis the largest bin among equal costs, then
  // the smallest axis.
  {
    const int w = threadIdx.x >> 5;
    if (w < 3) {
      const int a = w;
      const bool axis_ok = s_ext[a] > 0.0f;
      const bool in = lane < kBins;
      int c = 0;
      float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      if (axis_ok && in && s_cnt[a][lane] > 0) {
        c = s_cnt[a][lane];
        for (int j = 0; j < 3; ++j) {
          lo[j] = ord2f(s_box[a][lane][j]);
          hi[j] = ord2f(s_box[a][lane][3 + j]);
        }
      }
      int pc = c, sc = c;
      float plo[3], phi[3], slo[3], shi[3];
      for (int j = 0; j < 3; ++j) { plo[j] = slo[j] = lo[j]; phi[j] = shi[j] = hi[j]; }
      for (int o = 1; o < kBins; o <<= 1) {
        const int yp = __shfl_up_sync(0xffffffffu, pc, o), ys = __shfl_down_sync(0xffffffffu, sc, o);
        float ylo[3], yhi[3], zlo[3], zhi[3];
        for (int j = 0; j < 3; ++j) {
          ylo[j] = __shfl_up_sync(0xffffffffu, plo[j], o);
          yhi[j] = __shfl_up_sync(0xffffffffu, phi[j], o);
          zlo[j] = __shfl_down_sync(0xffffffffu, slo[j], o);
          zhi[j] = __shfl_down_sync(0xffffffffu, shi[j], o);
        }
        if (lane >= o) {
          pc += yp;
          for (int j = 0; j < 3; ++j) { plo[j] = fminf(plo[j], ylo[j]); phi[j] = fmaxf(phi[j], yhi[j]); }
        }
        if (lane + o < kBins) {
          sc += ys;
          for (int j = 0; j < 3; ++j) { slo[j] = fminf(slo[j], zlo[j]); shi[j] = fmaxf(shi[j], zhi[j]); }
        }
      }
      // left side of the split before bin k = prefix of bin k - 1
      const int lc = __shfl_up_sync(0xffffffffu, pc, 1);
      double llo[3], lhi[3], rlo[3], rhi[3];
      for (int j = 0; j < 3; ++j) {
        llo[j] = __shfl_up_sync(0xffffffffu, plo[j], 1);
        lhi[j] = __shfl_up_sync(0xffffffffu, phi[j], 1);
        rlo[j] = slo[j];
        rhi[j] = shi[j];
      }
      const bool valid = axis_ok && in && lane >= 1 && lc > 0 && sc > 0;
      double cost = INFINITY;
      if (valid)
        cost = __dadd_rn(__dmul_rn(half_area(llo, lhi), (double)lc), __dmul_rn(half_area(rlo, rhi), (double)sc));
      int bin = valid ? lane : -1;
      for (int o = 16; o > 0; o >>= 1) {
        const double oc = __shfl_xor_sync(0xffffffffu, cost, o);
        const int ob = __shfl_xor_sync(0xffffffffu, bin, o);
        if (oc < cost || (oc == cost && ob > bin)) { cost = oc; bin = ob; }
      }
      if (lane == 0) {
        s_cost[a] = cost;
        s_cbin[a] = bin;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double best = INFINITY;
    int best_axis = -1, best_bin = -1;
    for (int a = 0; a < 3; ++a)
      if (s_cbin[a] >= 0 && s_cost[a] < best) {
        best = s_cost[a];
        best_axis = a;
        best_bin = s_cbin[a];
      }
    int widest = 0;
    for (int c2 = 1; c2 < 3; ++c2)
      if (s_ext[c2] > s_ext[widest]) widest = c2;
    s_mode = best_axis >= 0 ? 0 : 1;
    s_axis = best_axis >= 0 ? best_axis : widest;
    s_bin = best_bin;
  }
  __syncthreads();

  // side of every triangle: the chosen bin split, else (no split separates the range)
  // the (e - b) / 2 smallest (centroid on the widest axis, index) go left
  for (int pass = 0; pass < 2; ++pass) {
    int32_t cnt = 0;
    const int a = s_axis, mode = s_mode, kb = s_bin;
    const int32_t half = n / 2;
    for (int32_t q = b + threadIdx.x; q < e; q += TB) {
      const int32_t t = ord_in[q];
      const float4 c4 = cen[t];
      const float ct = a == 0 ? c4.x : (a == 1 ? c4.y : c4.z);
      bool left;
      if (mode == 0) {
        left = bin_of(ct, s_clo[a], s_scale[a]) < kb;
      } else {
        int32_t rank = 0;  // position of (ct, t) among the range's keys
        for (int32_t j = b; j < e; ++j) {
          const int32_t u = ord_in[j];
          const float4 d4 = cen[u];
          const float cu = a == 0 ? d4.x : (a == 1 ? d4.y : d4.z);
          rank += (cu < ct || (cu == ct && u < t)) ? 1 : 0;
        }
        left = rank < half;
      }
      flag[q] = left;
      cnt += left;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) s_warp[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t t = 0;
      for (int w = 0; w < TB / 32; ++w) t += s_warp[w];
      s_left = t;
    }
    __syncthreads();
    const bool separated = s_left > 0 && s_left < n;
    if (s_mode == 1 || separated) break;
    __syncthreads();  // every thread has read s_mode and s_left
    if (threadIdx.x == 0) {  // the bin split left one side empty: median split on the widest axis
      int widest = 0;
      for (int c2 = 1; c2 < 3; ++c2)
        if (s_ext[c2] > s_ext[widest]) widest = c2;
      s_mode = 1;
      s_axis = widest;
    }
    __syncthreads();
  }
  const int32_t L = s_left;
  if (L <= 0 || L >= n) {  // cannot happen: the median split always separates
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }

  // stable partition into ord_out[b, e)
  int32_t run_l = 0, run_r = 0;
  for (int32_t base = b; base < e; base += TB) {
    const int32_t q = base + threadIdx.x;
    const bool has = q < e;
    const int32_t t = has ? ord_in[q] : 0;
    const int f = has ? flag[q] : 0;
    int32_t tot;
    const int32_t pre = block_exclusive_scan<TB>(f, s_warp, &tot);
    if (has) ord_out[f ? b + run_l + pre : b + L + run_r + (q - base - pre)] = t;
    run_l += tot;
    run_r += min(TB, e - base) - tot;
  }
  __syncthreads();

  // children: boxes, leaves finished
  const int32_t cb_[2] = {b, b + L}, ce_[2] = {b + L, e};
  for (int s = 0; s < 2; ++s) {
    unsigned v[6] = {kOrdPosInf, kOrdPosInf, kOrdPosInf, kOrdNegInf, kOrdNegInf, kOrdNegInf};
    for (int32_t q = cb_[s] + threadIdx.x; q < ce_[s]; q += TB) {
      const int32_t t = ord_out[q];
      const float4 lo = tlo[t], hi = thi[t];
      v[0] = min(v[0], f2ord(lo.x)); v[1] = min(v[1], f2ord(lo.y)); v[2] = min(v[2], f2ord(lo.z));
      v[3] = max(v[3], f2ord(hi.x)); v[4] = max(v[4], f2ord(hi.y)); v[5] = max(v[5], f2ord(hi.z));
      if (ce_[s] - cb_[s] <= 4) ord_final[q] = t;
    }
    block_minmax6<TB>(v, s_red, s_child[s]);
  }
  if (threadIdx.x == 0) {
    BNode nd;
    int inner = 0;
    for (int s = 0; s < 2; ++s) {
      for (int j = 0; j < 3; ++j) {
        nd.lo[s][j] = ord2f(s_child[s][j]);
        nd.hi[s][j] = ord2f(s_child[s][3 + j]);
      }
      const int32_t sz = ce_[s] - cb_[s];
      nd.ref[s] = sz <= 4 ? cb_[s] : -1;
      nd.cnt[s] = sz <= 4 ? sz : 0;
      inner += sz > 4;
    }
    nd.mid = b + L;
    nodes[sg.node] = nd;
    n_inner[blockIdx.x] = inner;
  }
}

// Next level's ranges (numbered by the prefix sum of inner children per range) and the
// parents' references to them.
__global__ void next_level(const Seg* __restrict__ segs, int32_t n_segs, const int32_t* __restrict__ n_inner,
                           const int32_t* __restrict__ first, int32_t node_base, BNode* __restrict__ nodes,
                           Seg* __restrict__ next) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_segs; i += gridDim.x * blockDim.x) {
    const Seg sg = segs[i];
    BNode& nd = nodes[sg.node];
    int32_t k = first[i];
    const int32_t split = nd.mid;
    for (int s = 0; s < 2; ++s) {
      if (nd.cnt[s] > 0) continue;
      Seg c;
      c.depth = sg.depth + 1;
      c.node = node_base + k;
      if (s == 0) { c.b = sg.b; c.e = split; } else { c.b = split; c.e = sg.e; }
      next[k] = c;
      nd.ref[s] = c.node;
      ++k;
    }
  }
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

// ---------------------------------------------------------------- numbering and layout
// sub[x] = inner nodes in x's subtree (x included), bottom-up one level at a time.
__global__ void subtree_sizes(int32_t id0, int32_t id1, const BNode* __restrict__ nodes, int32_t* __restrict__ sub) {
  for (int32_t x = id0 + blockIdx.x * blockDim.x + threadIdx.x; x < id1; x += gridDim.x * blockDim.x) {
    const BNode& nd = nodes[x];
    int32_t s = 1;
    for (int c = 0; c < 2; ++c)
      if (nd.cnt[c] == 0) s += sub[nd.ref[c]];
    sub[x] = s;
  }
}

// pre[x] = depth-first number: the left child follows its parent, the right child
// follows the left one's subtree.
__global__ void preorder(int32_t id0, int32_t id1, const BNode* __restrict__ nodes, const int32_t* __restrict__ sub,
                         int32_t* __restrict__ pre) {
  for (int32_t x = id0 + blockIdx.x * blockDim.x + threadIdx.x; x < id1; x += gridDim.x * blockDim.x) {
    const BNode& nd = nodes[x];
    const int32_t p = pre[x] + 1;
    if (nd.cnt[0] == 0) pre[nd.ref[0]] = p;
    if (nd.cnt[1] == 0) pre[nd.ref[1]] = p + (nd.cnt[0] == 0 ? sub[nd.ref[0]] : 0);
  }
}

__global__ void emit_nodes(int32_t n_nodes, const BNode* __restrict__ nodes, const int32_t* __restrict__ pre,
                           double wide, double flat, float4* __restrict__ out, int32_t* err) {
  for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n_nodes; x += gridDim.x * blockDim.x) {
    const BNode nd = nodes[x];
    const int32_t me = pre[x];
    if (me < 0 || me >= n_nodes) {
      atomicExch(err, 1);
      continue;
    }
    float l[2][3], h[2][3];
    int32_t ref[2];
    for (int s = 0; s < 2; ++s) {
      pad_box(make_float4(nd.lo[s][0], nd.lo[s][1], nd.lo[s][2], 0.f),
              make_float4(nd.hi[s][0], nd.hi[s][1], nd.hi[s][2], 0.f), wide, flat, l[s], h[s]);
      ref[s] = nd.cnt[s] > 0 ? nd.ref[s] : pre[nd.ref[s]];
    }
    float4* o = out + 4 * (int64_t)me;
    o[0] = make_float4(l[0][0], h[0][0], l[0][1], h[0][1]);
    o[1] = make_float4(l[1][0], h[1][0], l[1][1], h[1][1]);
    o[2] = make_float4(l[0][2], h[0][2], l[1][2], h[1][2]);
    o[3] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(nd.cnt[0]),
                       __int_as_float(nd.cnt[1]));
  }
}

// Triangle records (v0, e1, e2, id, face) at the positions the layout gave the leaves.
__global__ void emit_records(int64_t n, const int32_t* __restrict__ ord_final, const float* __restrict__ V,
                             const int32_t* __restrict__ T, const int32_t* __restrict__ TF, float4* __restrict__ rec,
                             int32_t* err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = ord_final[q];
    const int64_t pos = q;
    if (t < 0 || t >= n) {
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


// 1 + sum over inner children of area(child) / area(root): the expected node visits of
// a random line (one block, fixed order).
__global__ void __launch_bounds__(1024) sah_visits_kernel(int32_t n_nodes, const BNode* __restrict__ nodes,
                                                          double* out) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int32_t x = threadIdx.x; x < n_nodes; x += blockDim.x) {
    const BNode& nd = nodes[x];
    for (int s = 0; s < 2; ++s)
      if (nd.cnt[s] == 0) {
        const double lo[3] = {nd.lo[s][0], nd.lo[s][1], nd.lo[s][2]}, hi[3] = {nd.hi[s][0], nd.hi[s][1], nd.hi[s][2]};
        acc += half_area(lo, hi);
      }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const BNode& r = nodes[0];
    double lo[3], hi[3];
    for (int j = 0; j < 3; ++j) {
      lo[j] = fmin(r.lo[0][j], r.lo[1][j]);
      hi[j] = fmax(r.hi[0][j], r.hi[1][j]);
    }
    const double ra = half_area(lo, hi);
    out[0] = ra > 0.0 ? 1.0 + red[0] / ra : 1.0;
  }
}

}  // namespace

rg_status gpu_bvh_build(rg_ctx* ctx, const float* verts_h, int64_t nv, const int32_t* tris_h,
                        const int32_t* tri_face_h, int64_t nt, double diag, GpuBvh* out) {
  *out = GpuBvh{};
  RG_ARG_CHECK(ctx, nt > 4 && nt < (int64_t)1 << 30, "gpu BVH: %lld triangles", (long long)nt);
  const int32_t n = (int32_t)nt;
  const int32_t max_nodes = n;          // a binary tree over n triangles has fewer inner nodes
  const int32_t max_segs = n / 5 + 2;   // ranges of more than 4 triangles on one level
  cudaStream_t s = 0;
  RG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // the context workspace may still be read by queued work of earlier calls
  RG_CUDA_TRY(ctx, cudaDeviceSynchronize());

  rg::Sizer sz;
  sz.take<float>(3 * (size_t)nv); sz.take<int32_t>(3 * (size_t)nt); sz.take<int32_t>(nt);
  for (int k = 0; k < 3; ++k) sz.take<float4>(nt);          // tlo, thi, cen
  for (int k = 0; k < 3; ++k) sz.take<int32_t>(nt);         // ord0, ord1, ord_final
  sz.take<uint8_t>(nt);
  sz.take<BNode>(max_nodes);
  for (int k = 0; k < 2; ++k) sz.take<int32_t>(max_nodes);  // sub, pre
  for (int k = 0; k < 2; ++k) sz.take<Seg>(max_segs);
  for (int k = 0; k < 2; ++k) sz.take<int32_t>(max_segs);   // n_inner, first
  sz.take<int32_t>(Scanner::ints_needed(max_segs));
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
  float4* cen = cv.take<float4>(nt);
  int32_t* ord0 = cv.take<int32_t>(nt);
  int32_t* ord1 = cv.take<int32_t>(nt);
  int32_t* ord_final = cv.take<int32_t>(nt);
  uint8_t* flag = cv.take<uint8_t>(nt);
  BNode* nodes = cv.take<BNode>(max_nodes);
  int32_t* sub = cv.take<int32_t>(max_nodes);
  int32_t* pre = cv.take<int32_t>(max_nodes);
  Seg* seg0 = cv.take<Seg>(max_segs);
  Seg* seg1 = cv.take<Seg>(max_segs);
  int32_t* n_inner = cv.take<int32_t>(max_segs);
  int32_t* first = cv.take<int32_t>(max_segs);
  int32_t* scan_ws = cv.take<int32_t>(Scanner::ints_needed(max_segs));
  int32_t* tot = cv.take<int32_t>(8);
  double* d_sah = cv.take<double>(1);
  Scanner scan{scan_ws, ctx->sm_count, &ctx->launches};
  const int sm = ctx->sm_count;

  RG_CUDA_TRY(ctx, cudaMemcpyAsync(dV, verts_h, 3 * (size_t)nv * sizeof(float), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(dT, tris_h, 3 * (size_t)nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(dTF, tri_face_h, (size_t)nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(tot, 0, 8 * sizeof(int32_t), s));
  RG_CUDA_TRY(ctx, cudaMemsetAsync(ord_final, 0xff, (size_t)nt * sizeof(int32_t), s));  // -1: not placed
  const Seg root{0, n, 0, 1};
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(seg0, &root, sizeof(Seg), cudaMemcpyHostToDevice, s));
  tri_boxes<<<grid_capped(nt, sm), kThreads, 0, s>>>(dV, dT, nt, tlo, thi, cen, ord0);
  ++ctx->launches;

  std::vector<int32_t> level_start{0};
  int32_t n_segs = 1, n_nodes = 1;
  while (n_segs > 0) {
    if ((int)level_start.size() > kMaxLevels)
      return rg::fail(ctx, RG_ERR_STACK, "BVH depth exceeds the traversal stack (%d)", kTraceStack);
    if (n_segs < sm)
      sah_split_level<1024><<<n_segs, 1024, 0, s>>>(seg0, tlo, thi, cen, ord0, ord1, ord_final, flag, nodes, n_inner,
                                                    tot + 5);
    else
      sah_split_level<kThreads><<<n_segs, kThreads, 0, s>>>(seg0, tlo, thi, cen, ord0, ord1, ord_final, flag, nodes,
                                                            n_inner, tot + 5);
    ++ctx->launches;
    scan.run(n_inner, first, n_segs, tot, s);
    next_level<<<grid_capped(n_segs, sm), kThreads, 0, s>>>(seg0, n_segs, n_inner, first, n_nodes, nodes, seg1);
    ++ctx->launches;
    RG_CUDA_TRY(ctx, cudaGetLastError());
    RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, tot, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const int32_t next = ctx->h_scratch[0];
    if (next < 0 || next > max_segs || n_nodes + next > max_nodes)
      return rg::fail(ctx, RG_ERR_NUMERIC, "gpu BVH: %d ranges on a level", next);
    level_start.push_back(n_nodes);
    n_nodes += next;
    n_segs = next;
    std::swap(seg0, seg1);
    std::swap(ord0, ord1);
  }
  level_start.push_back(n_nodes);
  const int n_levels = (int)level_start.size() - 2;  // the last entry closes the deepest level
  for (int k = n_levels; k-- > 0;) {
    const int32_t a = level_start[k], bb = level_start[k + 1];
    subtree_sizes<<<grid_capped(bb - a, sm), kThreads, 0, s>>>(a, bb, nodes, sub);
    ++ctx->launches;
  }
  RG_CUDA_TRY(ctx, cudaMemsetAsync(pre, 0, sizeof(int32_t), s));
  for (int k = 0; k < n_levels; ++k) {
    const int32_t a = level_start[k], bb = level_start[k + 1];
    preorder<<<grid_capped(bb - a, sm), kThreads, 0, s>>>(a, bb, nodes, sub, pre);
    ++ctx->launches;
  }
  sah_visits_kernel<<<1, 1024, 0, s>>>(n_nodes, nodes, d_sah);
  ++ctx->launches;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  double h_sah = 0.0;
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(&h_sah, d_sah, sizeof(double), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  out->n_nodes = n_nodes;
  out->depth = n_levels;
  out->sah_visits = (float)h_sah;

  RG_CUDA_TRY(ctx, cudaMalloc(&out->buf, (4 * (size_t)n_nodes + 3 * (size_t)nt) * sizeof(float4)));
  out->nodes = static_cast<float4*>(out->buf);
  out->tris = out->nodes + 4 * (size_t)n_nodes;
  emit_nodes<<<grid_capped(n_nodes, sm), kThreads, 0, s>>>(n_nodes, nodes, pre, 1e-4 * diag, 1e-9 * diag,
                                                           out->nodes, tot + 5);
  emit_records<<<grid_capped(nt, sm), kThreads, 0, s>>>(nt, ord_final, dV, dT, dTF, out->tris, tot + 5);
  ctx->launches += 2;
  RG_CUDA_TRY(ctx, cudaGetLastError());
  RG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scratch, tot + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (ctx->h_scratch[0]) return rg::fail(ctx, RG_ERR_NUMERIC, "gpu BVH: a layout index fell out of range");
  return RG_OK;
}
