/*
 * radgeb.h -- C ABI of the GB300 (sm_103a) radiative hot path:
 *   Monte Carlo ray tracing (MCRT) of view factors  ->  closure / reciprocity
 *   enforcement  ->  multi-node aggregation  ->  Gebhart radiative exchange
 *   factors (REFs)  ->  steady radiative balance, with adjoint gradients.
 *
 * Thesis: "Novel Numerical Methods for Accurate Space Thermal Analysis"
 * (arXiv:2511.04277). Section, equation and appendix numbers below are the
 * thesis's.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Status: every call returns an rg_status; nothing throws or aborts across the
 *   ABI. rg_last_error(ctx) gives a human-readable message for the last failure
 *   on that context (never NULL).
 * - Ownership: the caller owns every buffer it passes (host or device, as each
 *   argument says). The library owns only the opaque rg_ctx and rg_mesh objects
 *   and the device workspace held by a context. Every dense-solve call (REFs,
 *   balances, adjoints, least-squares enforcement) also takes an optional
 *   caller-owned workspace (workspace_d, workspace_bytes): device memory, 256-byte
 *   aligned, at least the size rg_solver_workspace / rg_gebhart_workspace report, used
 *   for the call's duration only; with workspace_d = NULL the call uses (and grows on
 *   demand) the context's workspace. A workspace smaller than needed is RG_ERR_ARG.
 * - Layout: matrices are dense, row-major, fp64 unless stated. A view-factor or
 *   REF matrix of N faces is N x (N+1): column N is the environment (deep space),
 *   Sec. 2.4.12. Batched data of S sets is set-major ([S][...]).
 * - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream). Work
 *   is enqueued on it; calls that return a host-side scalar (iteration counts,
 *   residuals) synchronise that stream before returning.
 * - Devices: a context is bound to one device; device pointers must belong to it.
 * - Errors detected on the device (traversal stack overflow, non-finite values,
 *   non-convergence) are reported through the status of the call that detected
 *   them; the context stays usable.
 * - No call traps, asserts or waits without a bound on the device.
 */
#ifndef RADGEB_H
#define RADGEB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RG_OK = 0,
  RG_ERR_ARG = -1,            /* invalid argument (NULL pointer, size, layout)       */
  RG_ERR_CUDA = -2,           /* a CUDA runtime/driver call failed                   */
  RG_ERR_OOM = -3,            /* host or device allocation failed                    */
  RG_ERR_NOT_CONVERGED = -4,  /* an iteration hit its limit; outputs hold the last iterate */
  RG_ERR_STACK = -5,          /* BVH deeper than the traversal stack                  */
  RG_ERR_NUMERIC = -6,        /* non-finite value, zero pivot or singular system      */
  RG_ERR_UNSUPPORTED = -7     /* device is not sm_103 or size exceeds a stated limit   */
} rg_status;

typedef struct rg_ctx rg_ctx;
typedef struct rg_mesh rg_mesh;

/* Precision of the dense solves (Gebhart, adjoints, radiative balance). The
 * approximate inverse (Newton-Schulz iteration) and the corrections run on tcgen05
 * tensor cores in 16-bit floating point with fp32 accumulation; iterative refinement
 * with an exactly tracked residual (integer-exact bf16 products of fixed-point slices)
 * brings the result to the requested tolerance. */
typedef enum {
  RG_PREC_BF16_IR = 1,
  RG_PREC_FP16_IR = 2
} rg_precision;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (must be sm_103). *ctx_out receives a
 * library-owned handle; free it with rg_destroy. */
rg_status rg_create(rg_ctx** ctx_out, int device);
void rg_destroy(rg_ctx* ctx);
const char* rg_last_error(const rg_ctx* ctx);
const char* rg_version(void);
/* Number of kernels this context has launched so far (host counter, for accounting). */
rg_status rg_launch_count(const rg_ctx* ctx, int64_t* launches_out_h);
/* Bytes of device workspace the context holds (grown on demand by calls made without a
 * caller-owned workspace; never shrunk before rg_destroy). */
rg_status rg_workspace_bytes(const rg_ctx* ctx, size_t* bytes_out);

/* Device workspace a dense-solve call needs when the caller provides it (no device, no
 * context: sizes only). kind: which call; n the number of faces; rank the number of
 * cotangent factors for RG_WS_GEBHART_ADJOINT_FACTORED (ignored otherwise). The sets of a
 * batched call are solved one after another in the same workspace, so the size does not
 * depend on n_sets. Errors: RG_ERR_ARG (unknown kind, n outside the call's limits). */
typedef enum {
  RG_WS_GEBHART = 1,                  /* rg_gebhart */
  RG_WS_GEBHART_ADJOINT = 2,          /* rg_gebhart_adjoint */
  RG_WS_GEBHART_ADJOINT_FACTORED = 3, /* rg_gebhart_adjoint_factored */
  RG_WS_TEMPERATURES = 4,             /* rg_temperatures, rg_temperatures_adjoint */
  RG_WS_TEMPERATURES_SETS = 5,        /* rg_temperatures_sets, rg_temperatures_adjoint_sets */
  RG_WS_ENFORCE_LSQ = 6               /* rg_enforce_lsq */
} rg_solver_kind;
rg_status rg_solver_workspace(int32_t kind, int32_t n, int32_t rank, size_t* bytes_out);
/* The REF solve's memory (App. B, Eq. B.8-B.11) for n faces and n_sets sets in `precision`.
 * keep_factors = 0: the workspace of one rg_gebhart call, as
 * rg_solver_workspace(RG_WS_GEBHART, n, 0, ...). keep_factors != 0: the size of the factor
 * store (factors_d) that rg_gebhart fills and rg_gebhart_adjoint / rg_gebhart_adjoint_factored
 * read: a 256-byte header, one 16-bit np x np inverse per set (np = n rounded up to 128) and
 * one fp64 scale vector of np per set (the symmetric form's D, zeros for a general inverse),
 * about 2 n^2 n_sets bytes. Errors: RG_ERR_ARG. */
rg_status rg_gebhart_workspace(int32_t n, int32_t n_sets, int32_t precision, int32_t keep_factors, size_t* bytes_out);

/* Kernel timer, for measurement (no counterpart in the thesis). While it is on, the
 * context records a CUDA event pair on the launching stream around every launch of
 * these kernel classes:
 *   RG_TIME_TRACE     the MCRT trace kernel of rg_trace, rg_trace_stats, rg_trace_sided;
 *   RG_TIME_RESIDUAL  the exact level products of the dense solves' refinement (and of
 *                     rg_tc_gemm_exact);
 *   RG_TIME_GEMM      the other tensor-core GEMMs (Newton-Schulz steps, corrections);
 *   RG_TIME_ENFORCE   the persistent iterative enforcer;
 *   RG_TIME_FACTOR    one region per factorisation of a dense solve: the Newton-Schulz
 *                     inverse from its start iterate through its last step, including the
 *                     read-back of the start norms that fixes the step count (its GEMMs
 *                     are also counted under RG_TIME_GEMM).
 * rg_kernel_timer(ctx, 1) clears the records and starts recording, rg_kernel_timer(ctx, 0)
 * stops. rg_kernel_timer_read synchronises on the recorded events of `kind` and returns
 * their number, the sum of their durations (ms) and, for the GEMM classes, the tensor-core
 * flops the launches executed (2 M N K each, times the levels an exact product ran) and the
 * algorithmic flops of the products they stand for (for the refinement's level product,
 * 2 n n m of the one-slice product P' D it computes exactly; otherwise equal to the executed
 * flops); both are 0 for the other classes. The two flop outputs may be NULL. The records grow by one event pair per timed launch until the next
 * rg_kernel_timer(ctx, 1). Errors: RG_ERR_ARG, RG_ERR_CUDA. */
typedef enum {
  RG_TIME_TRACE = 0,
  RG_TIME_RESIDUAL = 1,
  RG_TIME_GEMM = 2,
  RG_TIME_ENFORCE = 3,
  RG_TIME_FACTOR = 4
} rg_kernel_class;
rg_status rg_kernel_timer(rg_ctx* ctx, int32_t enable);
rg_status rg_kernel_timer_read(rg_ctx* ctx, int32_t kind, int64_t* launches_out_h, double* ms_out_h,
                               double* flops_out_h, double* alg_flops_out_h);

/* ---------------------------------------------------------------- mesh (P1) */

/* Upload a triangle mesh and build its bounding-volume hierarchy (host binned
 * SAH, leaves of at most 4 triangles, boxes padded so that the traversal never
 * rejects a triangle the brute-force test would accept).
 *   verts_h     host float32 [nv][3]       vertex positions
 *   tris_h      host int32   [nt][3]       vertex indices; the winding (v1-v0) x
 *                                          (v2-v0) gives the emitting side
 *   tri_face_h  host int32   [nt]          face (row of F) of every triangle;
 *                                          the triangles of a face must be coplanar
 *   n_faces     number of faces N (every face needs >= 1 triangle of area > 0)
 *   use_bvh     1 = traverse the BVH, 0 = test every triangle (tiny meshes),
 *               -1 = choose (brute force when nt <= 64); 2 / 3 = traverse the BVH
 *               with the lock-step / refill schedule of the trace kernel (1 and -1
 *               take refill for BVHs of depth >= 12, lock-step otherwise).
 *               All choices give bit-identical counts.
 * The host arrays are copied; they may be freed after the call.
 * Errors: RG_ERR_ARG (bad index, empty or degenerate face), RG_ERR_STACK (BVH
 * deeper than the 64-entry traversal stack), RG_ERR_OOM, RG_ERR_CUDA. */
rg_status rg_mesh_create(rg_ctx* ctx, const float* verts_h, int64_t nv, const int32_t* tris_h,
                         int64_t nt, const int32_t* tri_face_h, int32_t n_faces, int32_t use_bvh,
                         rg_mesh** mesh_out);

/* rg_mesh_create with the BVH built on the device: the host builder's binned
 * surface-area heuristic (16 bins per axis, float binning and fp64 costs, leaves of at
 * most 4 triangles, median split where no bin split separates a range) evaluated level
 * by level, one block per range. It makes the host builder's splits, so the node array
 * is the one rg_mesh_create builds, bit for bit; within a leaf the records may come in
 * another order (the host partition is not stable). Counts are therefore bit-identical
 * too. Everything else, including the per-face emission data (built on the host), as
 * rg_mesh_create. Errors: RG_ERR_ARG (also a non-finite vertex), RG_ERR_STACK (depth
 * above the traversal stack), RG_ERR_NUMERIC (an inconsistent layout, a defect),
 * RG_ERR_CUDA. */
rg_status rg_mesh_create_gpu_bvh(rg_ctx* ctx, const float* verts_h, int64_t nv, const int32_t* tris_h, int64_t nt,
                                 const int32_t* tri_face_h, int32_t n_faces, int32_t use_bvh, rg_mesh** mesh_out);

/* Copy a mesh's BVH to the host for inspection (either builder):
 *   nodes_h       host float [bvh_nodes][16] (may be NULL): the traversal layout, per node
 *                 (L.lo.x, L.hi.x, L.lo.y, L.hi.y) (R.lo.x, R.hi.x, R.lo.y, R.hi.y)
 *                 (L.lo.z, L.hi.z, R.lo.z, R.hi.z) and the int32 bits of (L.ref, R.ref,
 *                 L.count, R.count): count > 0 makes the child a leaf of `count` records
 *                 from record `ref`, count = 0 an inner node `ref`; node 0 is the root
 *   record_tri_h  host int32 [n_tris] (may be NULL): the triangle of every traversal-order
 *                 record
 * bvh_nodes is rg_mesh_get_info's; nothing is written for nodes_h without a BVH. */
rg_status rg_mesh_get_bvh(const rg_mesh* mesh, float* nodes_h, int32_t* record_tri_h);
rg_status rg_mesh_destroy(rg_mesh* mesh);

typedef struct {
  int32_t n_faces;
  int64_t n_tris;
  int32_t bvh_nodes;   /* 0 when brute force is used */
  int32_t bvh_depth;
  float lift;          /* ray origins sit this far off their face: 1e-6 x bounding-box diagonal */
  float sah_visits;    /* expected BVH node visits of a random line (surface-area heuristic) */
  int32_t refill;      /* 1: the trace kernel refills finished lanes, 0: lock-step rays */
} rg_mesh_info;
rg_status rg_mesh_get_info(const rg_mesh* mesh, rg_mesh_info* info_out);

/* Face areas A_i (fp64 sum of the triangle areas), written to host double[N]. */
rg_status rg_face_areas(const rg_mesh* mesh, double* areas_out_h);

/* ---------------------------------------------------------------- MCRT (P2) */

/* Hit counts N_ij of the MCRT estimator F_ij = N_ij / N_i (Sec. 3.5.1, Eq. 3.15).
 *   rays_per_face_h  host int64 [N]: rays emitted from face i (N_i >= 0)
 *   seed             Philox4x32-10 key; ray r of face i is made from the one draw
 *                    of counter (ray_offset + r, i, 0), so disjoint ray ranges of
 *                    separate calls are independent and their counts add up
 *   fma_free         1: every float operation of sampling and intersection is
 *                    individually rounded (bit-exact with the reference ray
 *                    definition); 0: the compiler may fuse multiply-adds
 *   counts_d         device int64 [N][N+1], ACCUMULATED into (zero it first);
 *                    column N counts rays that escape to the environment
 * Emission is diffuse (cosine-weighted about the face normal, Sec. 2.4.12) from
 * points uniform over the face area (Sec. 5.2.1), lifted off the face by `lift`
 * along its normal. The closest hit with t > 0 (smallest t, then smallest
 * triangle index) receives the ray; the source triangle is ignored.
 * Limit: N + 1 <= 49152 (one shared-memory tally row per block).
 * Errors: RG_ERR_ARG, RG_ERR_STACK, RG_ERR_CUDA, RG_ERR_UNSUPPORTED. */
rg_status rg_trace(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_face_h, uint64_t seed,
                   uint64_t ray_offset, int32_t fma_free, int64_t* counts_d, void* stream);

/* rg_trace with traversal statistics: the same counts (bit-identical), and
 * stats_out_h = host uint64[3] {rays traced, ray-box tests, ray-triangle tests}
 * summed over the launch; the statistics cost extra atomics, so time rg_trace. */
rg_status rg_trace_stats(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_face_h, uint64_t seed,
                         uint64_t ray_offset, int32_t fma_free, int64_t* counts_d, uint64_t* stats_out_h,
                         void* stream);

/* Side-resolved hit counts of two-sided faces (Sec. 5.2.4-5.2.5: the factors
 * F^{X->Y}_{n_i m_j} between the faces A and B of the nodes). Side A of face f is the
 * side its normal n points to (n from the face's first triangle, as in rg_trace), side
 * B the other one. Row 2f+X counts the rays emitted from side X of face f, column 2g+Y
 * the rays whose closest hit lies on side Y of face g, column 2N the environment; F^{X->Y}
 * = counts / rays of the row (Eq. 3.15 per side).
 *   Side A emits exactly the rays of face f in rg_trace (counter word 2 = f), so summing
 *   a side-A row over the target sides gives rg_trace's row bit for bit. Side B uses
 *   counter word 2 = f + 2^31, the origin lifted along -n and the cosine-weighted
 *   direction in the frame (t, -b, -n). A hit on a triangle is on side A when the Moller-Trumbore
 *   determinant e1 . (d x e2) is positive (the ray runs against the triangle normal
 *   e1 x e2), on side B otherwise; the closest-hit and tie rules are rg_trace's.
 *   rays_per_side_h  host int64 [2N]: rays of side X of face f at index 2f+X (0 for a
 *             face whose side B does not radiate)
 *   counts_d  device int64 [2N][2N+1], row-major, ADDED to
 * Errors: RG_ERR_ARG when a triangle's e1 x e2 points to its face's side B (every
 * triangle of a face must be wound like the face's first one) or N >= 2^29;
 * RG_ERR_UNSUPPORTED when 2N+1 tally columns exceed the shared-memory tally row
 * (N > 24,575 on GB300); otherwise as rg_trace. */
rg_status rg_trace_sided(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_side_h, uint64_t seed,
                         uint64_t ray_offset, int32_t fma_free, int64_t* counts_d, void* stream);

/* REFs directly from MCRT (Sec. 4.2.2): rays emitted as in rg_trace are followed
 * through diffuse reflections. At bounce b (b = 1, 2, ...) the closest hit on face j
 * is decided by word 3 of the Philox draw of counter (ray lo, ray hi, i, 128 b + 1), i
 * the path's source face: below floor(eps_j 2^32) the ray is absorbed and counted for
 * column j; below floor((eps_j + rho_j) 2^32) it is reflected, i.e. re-emitted from
 * face j exactly as an emission of face j, with the draw of counter
 * (ray lo, ray hi, i, 128 b) in place of the emission draw; otherwise it is lost. A miss is counted for the environment column. Re-emission
 * from a uniform point of the hit face is the face-level model of Eq. 4.5, so
 * counts_ij / N_i estimates the B_ij that rg_gebhart solves for from the exact view
 * factors of the same faces.
 *   eps_h, rho_h host fp64 [n_faces]: absorptivity and diffuse reflectivity,
 *             eps, rho >= 0 and eps + rho <= 1 (the rest is lost)
 *   max_bounces  a path still reflecting after this many hits ends as overflow
 *             (1 <= max_bounces < 2^25)
 *   counts_d  device int64 [N][N+1], ADDED to (absorbed on face j; column N escaped)
 *   stats_out_h  host uint64[4] (may be NULL): rays, hits, lost, overflow
 * fma_free, seed, ray_offset and the errors as rg_trace. */
rg_status rg_trace_reflect(rg_ctx* ctx, const rg_mesh* mesh, const int64_t* rays_per_face_h, const double* eps_h,
                           const double* rho_h, int32_t max_bounces, uint64_t seed, uint64_t ray_offset,
                           int32_t fma_free, int64_t* counts_d, uint64_t* stats_out_h, void* stream);

/* F_ij = N_ij / N_i (Eq. 3.15) for N x (N+1) counts.
 *   counts_d  device int64 [n][n+1];  rays_d device int64 [n] (N_i > 0)
 *   F_d       device fp64 [n][n+1] (output) */
rg_status rg_counts_to_F(rg_ctx* ctx, int32_t n, const int64_t* counts_d, const int64_t* rays_d,
                         double* F_d, void* stream);

/* ---------------------------------------------------------------- enforcement (P3) */

/* Iterative closure + reciprocity enforcer for open systems (Sec. 3.5.5), in place.
 * With eta_ij = Omega_i F_ij (Eq. 3.18) each iteration
 *   (1) averages eta_ij and eta_ji on the N x N block (Eq. 3.20, kappa = 1/2), the
 *       environment column carried over from the previous iterate, then
 *   (2) enforces closure by open-system least squares with w = eta (Eq. 3.39-3.40),
 *       i.e. scales row i to sum Omega_i.
 * It stops after the first iteration whose reciprocity defect of the previous
 * iterate and closure defect after step (1) are both <= tol * max_i Omega_i.
 * Arithmetic: the first iteration in fp64. The N x N block is symmetric after it, so every
 * later iteration updates the entries on and above the diagonal in fp64 (the sum of the
 * two halved row scales carries the fp64 addition's bits), accumulates the row sums exactly
 * in 64-bit fixed point (to 2^-62 of each row's bound) and takes the stop rule's
 * reciprocity defect in fp32; tile pairs that are zero after the first iteration stay zero
 * and are skipped. A negative entry keeps every iteration in fp64 on both triangles.
 *   omega_d   device fp64 [n]: Omega_i (A_i for view factors, eps_i A_i for REFs)
 *   F_d       device fp64 [n][n+1], in: F, out: enforced F
 *   iters_out_h  host int32 (may be NULL): iterations performed
 * Rows with a zero sum are left unchanged. Errors: RG_ERR_NOT_CONVERGED (after
 * maxit iterations; F_d holds the last iterate), RG_ERR_NUMERIC (a non-finite row sum, or
 * a fixed-point term outside its bound, which the bound's construction rules out),
 * RG_ERR_ARG. */
rg_status rg_enforce_iterative(rg_ctx* ctx, int32_t n, const double* omega_d, double* F_d, double tol,
                               int32_t maxit, int32_t* iters_out_h, void* stream);

/* Reciprocity weights kappa_ij of Eq. 3.20 for rg_enforce_iterative_kappa (Sec. 3.5.3).
 *   mode RG_KAPPA_TRIANGULATION (matrix triangulation, Eq. 3.21-3.22):
 *       kappa_ij = (1 + sign(Y_ij) |Y_ij|^param) / 2,
 *       Y_ij = (Omega_j/N_j - Omega_i/N_i) / (Omega_j/N_j + Omega_i/N_i);
 *       param = the exponent n (0.4 in the thesis). F_d is not read (may be NULL).
 *   mode RG_KAPPA_FRACTIONAL_VARIANCE (Eq. 3.23-3.25):
 *       kappa_ij = var_ji / (var_ij + var_ji),
 *       var_ij = param^2 Omega_i^2 (1 - F_ij) / (N_i F_ij)  (param = z; it cancels).
 *       An estimate F_ij = 0 has infinite variance, so the other side is taken
 *       (kappa_ij = 0, kappa_ji = 1); both zero give 1/2.
 *   F_d       device fp64 [n][n+1]: the MCRT view factors (Eq. 3.15)
 *   rays_d    device int64 [n]: N_i, rays emitted per face (> 0)
 *   omega_d   device fp64 [n]: Omega_i (> 0)
 *   kappa_d   device fp64 [n][n] (output, caller-owned); kappa_ji = 1 - kappa_ij up to
 *             rounding, the diagonal is 1/2.
 * Errors: RG_ERR_ARG (bad mode or pointers; a non-positive N_i or Omega_i, found on
 * the device and reported after the call synchronises `stream`). */
typedef enum { RG_KAPPA_TRIANGULATION = 1, RG_KAPPA_FRACTIONAL_VARIANCE = 2 } rg_kappa_mode;
rg_status rg_kappa(rg_ctx* ctx, int32_t n, int32_t mode, const double* F_d, const int64_t* rays_d,
                   const double* omega_d, double param, double* kappa_d, void* stream);

/* rg_enforce_iterative with per-pair weights in step (1) (Eq. 3.20):
 *   eta-hat_ij = kappa_ij eta_ij + (1 - kappa_ij) eta_ji,
 * kappa_d device fp64 [n][n] as rg_kappa writes it (the thesis combines the
 * fractional-variance weights with the open-system closure, Sec. 3.5.5). Every iteration
 * runs in fp64 on both triangles; with every kappa_ij = 1/2 the iterates are those of
 * rg_enforce_iterative up to rounding. The same stop rule, arguments and errors as
 * rg_enforce_iterative. One iteration reads kappa once more than the first iteration of
 * the unweighted enforcer (24 instead of 16 bytes per matrix entry). */
rg_status rg_enforce_iterative_kappa(rg_ctx* ctx, int32_t n, const double* omega_d, const double* kappa_d,
                                     double* F_d, double tol, int32_t maxit, int32_t* iters_out_h, void* stream);

/* rg_enforce_iterative without allocation, for callers that must not allocate
 * device memory when they call in -- for instance flight or embedded software that
 * plans all of its memory up front, or a host application that owns the device's
 * memory pool and forbids its plug-ins from allocating. The thesis has no counterpart
 * of this entry point; it computes exactly what rg_enforce_iterative computes.
 *   - No context: it runs on the CURRENT device and allocates nothing (no cudaMalloc,
 *     no cudaFree, no allocating library call). Its scratch is a file-scope device
 *     array of about 2.1 MB that every GPU loading the library holds until exit.
 *   - Limit: n <= 4096; larger n returns RG_ERR_UNSUPPORTED.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress).
 *   - Every call shares the one array and clears the part that must start at zero;
 *     calls that overlap on the GPU (other streams, other host threads) race.
 *   - It synchronises `stream` to read its iteration state back, so it must not be
 *     called while `stream` is being captured into a CUDA graph.
 *   - A CUDA error already pending on the calling thread when it is called (left by the
 *     caller's own earlier work) makes it return RG_ERR_CUDA at once, without running
 *     and without clearing that error.
 * Arguments, results and other errors as rg_enforce_iterative (no rg_last_error:
 * the status code is the whole report). */
rg_status rg_enforce_iterative_noalloc(int32_t n, const double* omega_d, double* F_d, double tol,
                                       int32_t maxit, int32_t* iters_out_h, void* stream);

/* Least-squares optimum for open systems (Sec. 3.5.5, Eq. 3.41-3.52) with
 * non-negativity rectification (App. A.1) and small-positive-value avoidance
 * (App. A.2), in place. The unknowns are the entries of F; the restrictions are
 * sum_j F_ij = 1 and Omega_i F_ij - Omega_j F_ji = 0 (i < j); the result is the
 * orthogonal projection of the active entries of F onto them.
 *   spva = 1: MCRT zeros stay 0 and are not unknowns; restrictions left without
 *             unknowns are dropped (App. A.2).
 *   nnr  = 1: negative results are set to 0, removed from the unknowns and the
 *             original values of the remaining unknowns projected again, until no
 *             entry is negative (App. A.1); at most max_passes projections.
 *   passes_out_h host int32 (may be NULL): projections performed.
 * Limit: n <= 4096 (one dense n x n Schur complement is factorised).
 * Errors: RG_ERR_NUMERIC (singular restriction system), RG_ERR_NOT_CONVERGED. */
rg_status rg_enforce_lsq(rg_ctx* ctx, int32_t n, const double* omega_d, double* F_d, int32_t nnr,
                         int32_t spva, int32_t max_passes, int32_t* passes_out_h, void* workspace_d,
                         size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- multi-node (P4) */

/* Group view factors from sub-surface view factors (Eq. 5.6-5.7, 5.28):
 *   F_group[n][m] = sum_{i in n} sum_{j in m} F_sub[i][j] * S_i / S_n
 *   F_group[n][G] = sum_{i in n} F_sub[i][n_sub] * S_i / S_n   (environment)
 * with S_n = sum_{i in n} S_i. With groups = the faces of one node (equal-area
 * sides A and B) this is the node relation C_n F_ij = sum_{X,Y} F^{X->Y} of
 * Eq. 5.17; with singleton groups it is the identity.
 *   F_sub_d       device fp64 [n_sub][n_sub+1]
 *   sub_area_d    device fp64 [n_sub]
 *   sub_group_d   device int32 [n_sub], values in [0, n_group)
 *   F_group_d     device fp64 [n_group][n_group+1] (output)
 *   group_area_d  device fp64 [n_group] (output, may be NULL) */
rg_status rg_aggregate(rg_ctx* ctx, int32_t n_sub, const double* F_sub_d, const double* sub_area_d,
                       const int32_t* sub_group_d, int32_t n_group, double* F_group_d,
                       double* group_area_d, void* stream);

/* Node view factors and view fractions of two-sided surfaces (Sec. 5.2.4-5.2.5).
 * F2_d is a side-resolved matrix in the layout of rg_trace_sided (row 2i+X = side X of
 * face i, column 2j+Y, column 2n = environment; leading dimension 2n+1), e.g. the view
 * factors of the nodes' faces; node i has C_i faces.
 *   F_node_d  device fp64 [n][n+1] (output): C_i F_ij = F^{AA}_ij + F^{AB}_ij + F^{BA}_ij
 *             + F^{BB}_ij, C_i F_i,inf = F^{A,inf}_i + F^{B,inf}_i (Eq. 5.17 / 5.28)
 *   frac_d    device fp64 [2n][2n+1] (output, may be NULL): the view fractions
 *             f^{X->Y}_ij = F^{X->Y}_ij / (sum of the four) and f^{X,inf}_i =
 *             F^{X,inf}_i / (sum of the two) (Eq. 5.27 / 5.29), 0 where the sum is 0
 *   faces_per_node_d  device int32 [n]: C_i in {1, 2}; a one-faced node's side-B row of
 *             F2 holds zeros (its rays are not traced)
 * With singleton nodes of one face this is the identity. Errors: RG_ERR_ARG (bad
 * argument, a C_i outside {1, 2}). */
rg_status rg_node_view_factors(rg_ctx* ctx, int32_t n, const double* F2_d, const int32_t* faces_per_node_d,
                               double* F_node_d, double* frac_d, void* stream);

/* Radiative couplings of nodes whose two faces have different optical properties
 * (App. C). B2_d holds the REFs of the system whose faces are the nodes' sides
 * (rg_gebhart on 2n faces with per-side eps and rho), in the layout of
 * rg_node_view_factors.
 *   eps2_d       device fp64 [2n]: eps^X_i at 2i+X
 *   face_area_d  device fp64 [n]: S_i, the area of each face of node i (A_i = C_i S_i)
 *   faces_per_node_d  device int32 [n]: C_i in {1, 2}
 *   GR_d         device fp64 [n][n+1] (output): GR_ij = S_i (eps^A_i (B^{AA}_ij +
 *                B^{AB}_ij) + eps^B_i (B^{BA}_ij + B^{BB}_ij)) (Eq. C.3; column n the
 *                environment, B^{X,inf}); the coupling sigma GR_ij (T_i^4 - T_j^4) of
 *                Eq. 4.2 without sigma
 *   B_node_d     device fp64 [n][n+1] (output, may be NULL): node REFs, C_i B_ij = sum
 *                of the four side pairs (Eq. C.3, first line)
 *   eps_node_d   device fp64 [n][n+1] (output, may be NULL): the node emissivity of each
 *                pair, eps_ij = GR_ij / (C_i S_i B_ij) = eps^A_i (f^{AA} + f^{AB}) +
 *                eps^B_i (f^{BA} + f^{BB}) with the view fractions of B (Eq. C.4); 0 where
 *                B_ij = 0
 * Errors: RG_ERR_ARG (bad argument, a C_i outside {1, 2}). */
rg_status rg_node_couplings(rg_ctx* ctx, int32_t n, const double* B2_d, const double* eps2_d,
                            const double* face_area_d, const int32_t* faces_per_node_d, double* GR_d,
                            double* B_node_d, double* eps_node_d, void* stream);

/* ---------------------------------------------------------------- Gebhart REFs (P5) */

/* Radiative exchange factors of an open system (Eq. 4.5, App. B.2, Eq. B.6-B.11):
 *   K B = E,  K = I - F_NN diag(rho),  E = [F_NN diag(eps) | F_inf]
 * for n_sets independent (eps, rho) sets sharing F.
 *   F_d      device fp64 [n][n+1]
 *   eps_d    device fp64 [n_sets][n];  rho_d device fp64 [n_sets][n], 0 <= rho < 1
 *   area_d   device fp64 [n] face areas, or NULL. Given, and with F reciprocal (A_i F_ij =
 *            A_j F_ji, as the enforcers leave it), the 16-bit inverse is built in the
 *            symmetric form of K, D K D^-1 with D = diag(sqrt(A rho)), whose Newton-Schulz
 *            steps compute the second of their two products, X (2I - A X) (symmetric), on
 *            the tiles on and above the diagonal only; a set with a non-positive A_i rho_i, or one
 *            below 2^-20 of the largest, takes the general factorisation. The refinement's
 *            residual is exact for the F given either way: areas of a non-reciprocal F only
 *            make the inverse a poorer preconditioner (more sweeps).
 *   B_d      device fp64 [n_sets][n][n+1] (output)
 *   tol      refinement stops when max_ij |R_ij| <= tol * max_ij |B_ij| for the
 *            residual R = E - K B of every set (tol >= 1e-13). The residual is tracked
 *            exactly: each correction is rounded to 8 bits per column and added to B
 *            exactly, and its product with the fixed-point slices of F diag(rho) is an
 *            exact integer sum on the tensor cores; the only error is the truncation of
 *            those slices (below 2^-38 of max|K| max|B| per sweep), so residuals of about
 *            1e-12 relative are attainable. Below 1e-8 a sweep that fails to halve the
 *            residual also ends the refinement (counted as converged; resid_out_h reports
 *            where it stopped).
 *   max_sweeps  refinement sweeps at most (>= 1)
 *   sweeps_out_h host int32 (may be NULL); resid_out_h host fp64 (may be NULL):
 *            the final relative residual (max over sets)
 *   factors_d   device buffer of factors_bytes (may be NULL: nothing kept), 256-byte
 *            aligned, at least rg_gebhart_workspace(n, n_sets, precision, 1) bytes: the
 *            call stores there, per set, the transpose of its 16-bit approximate inverse of
 *            K, which is an approximate inverse of K^T, so that the adjoint calls need not
 *            factorise K^T again (the thesis has no adjoint; this is the usual reuse of a
 *            forward factorisation by a backward pass). Owned by the caller; the store is
 *            marked complete only when every set has been solved, and an adjoint given an
 *            incomplete store fails with RG_ERR_ARG.
 * K must be strictly diagonally dominant (rows of F_NN sum to <= 1 and rho < 1), which
 * is what makes the factorisation without pivoting stable.
 * Limit: n <= 32768. Errors: RG_ERR_ARG (also a factor store that is short or misaligned),
 * RG_ERR_NOT_CONVERGED, RG_ERR_NUMERIC, RG_ERR_OOM. */
rg_status rg_gebhart(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets, const double* eps_d,
                     const double* rho_d, const double* area_d, int32_t precision, double tol, int32_t max_sweeps,
                     double* B_d, int32_t* sweeps_out_h, double* resid_out_h, void* factors_d,
                     size_t factors_bytes, void* workspace_d, size_t workspace_bytes, void* stream);

/* Adjoint of rg_gebhart: given dB = dL/dB, the gradients of L with respect to eps
 * and rho. It solves K^T Lambda = dB and forms dL/deps_j = sum_i Lambda_ij F_ij and
 * dL/drho_k = sum_i F_ik (Lambda B^T)_ik.
 *   B_d, dB_d  device fp64 [n_sets][n][n+1];  deps_d, drho_d device fp64 [n_sets][n]
 *   factors_d  NULL: K^T is factorised afresh for every set. Otherwise the factor store a
 *              completed rg_gebhart call filled (factors_bytes its size) for the same n,
 *              precision and at least n_sets sets, whose set s then stands in for the
 *              factorisation of set s. Its header is read on the host (the call waits for
 *              the stream once), so a store written on another stream must be ordered before
 *              this call. The residual is refined exactly against this call's F and rho, so
 *              the results do not depend on the store; factors of another system only slow
 *              the sweeps (RG_ERR_NOT_CONVERGED when they no longer converge).
 * Errors as rg_gebhart; RG_ERR_ARG for a store of another n, precision or fewer sets, or one
 * that is short, misaligned or not filled. */
rg_status rg_gebhart_adjoint(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets,
                             const double* eps_d, const double* rho_d, const double* B_d,
                             const double* dB_d, int32_t precision, double tol, int32_t max_sweeps,
                             double* deps_d, double* drho_d, const void* factors_d, size_t factors_bytes,
                             void* workspace_d, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- radiative balance (P6) */

/* Steady node temperatures of the radiative network (Eq. 3.13, 4.1-4.2):
 *   sum_j GR_ij (T_i^4 - T_j^4) + GR_i,inf (T_i^4 - T_sink^4) = Q_i,
 *   GR_ij = sigma eps_i A_i B_ij,
 * solved in u = T^4 (fp64-accurate refinement) and T = u^(1/4).
 *   B_d device fp64 [n][n+1]; eps_d, area_d, Q_d device fp64 [n]; T_d output [n]
 * Errors: RG_ERR_NUMERIC (a node with no path to the environment makes the
 * system singular; a face with sigma eps_i A_i <= 0 or a B row that sums to 0 has no
 * balance; a heat load that drives u_i = T_i^4 to 0 or below has no temperature),
 * RG_ERR_NOT_CONVERGED. */
rg_status rg_temperatures(rg_ctx* ctx, int32_t n, const double* B_d, const double* eps_d,
                          const double* area_d, const double* Q_d, double T_sink, double sigma,
                          int32_t precision, double tol, double* T_d, void* workspace_d, size_t workspace_bytes,
                          void* stream);

/* Adjoint of rg_temperatures: given dT = dL/dT, writes dB = dL/dB (device fp64
 * [n][n+1]) and the direct part of dL/deps (device fp64 [n]); the part through B
 * follows from rg_gebhart_adjoint with dB. Errors as rg_temperatures (but for the heat-load
 * case, which the adjoint does not see). */
rg_status rg_temperatures_adjoint(rg_ctx* ctx, int32_t n, const double* B_d, const double* eps_d,
                                  const double* area_d, double T_sink, double sigma,
                                  const double* T_d, const double* dT_d, int32_t precision, double tol,
                                  double* dB_d, double* deps_d, void* workspace_d, size_t workspace_bytes,
                                  void* stream);

/* rg_temperatures and rg_temperatures_adjoint for n_sets (eps, rho) sets sharing F, in one
 * call: the same equations and results (each set's balance is refined to tol against its own
 * exact residual), solved faster. For opaque faces (rho = 1 - eps) whose REFs close, the
 * balance matrix of every set is K^-1 (I - F_NN) up to diagonal scalings (K = I - F_NN
 * diag(rho), Eq. B.9), so one 16-bit approximate inverse of I - F_NN, built once per call,
 * preconditions the refinement of all sets; F and rho enter only this preconditioner (with
 * other properties the refinement converges more slowly, and RG_ERR_NOT_CONVERGED reports a
 * failure to reach tol in 24 sweeps).
 *   F_d       device fp64 [n][n+1], the view factors the REFs were solved from
 *   B_d       device fp64 [n_sets][n][n+1]; eps_d, rho_d device fp64 [n_sets][n]
 *   area_d    device fp64 [n];  Q_d device fp64 [n_sets][n];  T_d device fp64 [n_sets][n] (output)
 * adjoint:  T_d, dT_d device fp64 [n_sets][n] in; deps_d [n_sets][n] out (the direct part of
 *           dL/deps) and dL/dB, in full in dB_d [n_sets][n][n+1] and/or in its factored form
 *           dL/dB_ij = -nu_i (u_i - u_j) = sum_r a_r,i b_r,j (r = 0, 1; u = T^4, u_n = T_sink^4):
 *           dB_a_d [n_sets][2][n] = (-nu o u, nu), dB_b_d [n_sets][2][n+1] = (1, u); dB_d may
 *           be NULL when dB_a_d and dB_b_d are given, and those two may be NULL when dB_d is.
 * Errors as rg_temperatures / rg_temperatures_adjoint. */
rg_status rg_temperatures_sets(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets, const double* B_d,
                               const double* eps_d, const double* rho_d, const double* area_d, const double* Q_d,
                               double T_sink, double sigma, int32_t precision, double tol, double* T_d,
                               void* workspace_d, size_t workspace_bytes, void* stream);
rg_status rg_temperatures_adjoint_sets(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets,
                                       const double* B_d, const double* eps_d, const double* rho_d,
                                       const double* area_d, double T_sink, double sigma, const double* T_d,
                                       const double* dT_d, int32_t precision, double tol, double* dB_d,
                                       double* dB_a_d, double* dB_b_d, double* deps_d, void* workspace_d,
                                       size_t workspace_bytes, void* stream);

/* rg_gebhart_adjoint for a cotangent given in factored form, dB = sum_r a_r b_r^T (for
 * instance the one rg_temperatures_adjoint_sets writes: rank 2). Lambda = K^-T dB =
 * sum_r x_r b_r^T with K^T x_r = a_r, so the transposed system (factorised afresh, or with the
 * stored factors of rg_gebhart, as in rg_gebhart_adjoint) is solved for `rank` right-hand
 * sides instead of N+1, and (derived from Eq. B.11)
 *   dL/deps_j = sum_r b_r,j (F^T x_r)_j,    dL/drho_k = sum_r (F^T x_r)_k (B b_r)_k.
 *   a_d  device fp64 [n_sets][rank][n];  b_d device fp64 [n_sets][rank][n+1];  1 <= rank <= 64
 * The other arguments and the errors as rg_gebhart_adjoint. */
rg_status rg_gebhart_adjoint_factored(rg_ctx* ctx, int32_t n, const double* F_d, int32_t n_sets,
                                      const double* eps_d, const double* rho_d, const double* B_d, int32_t rank,
                                      const double* a_d, const double* b_d, int32_t precision, double tol,
                                      int32_t max_sweeps, double* deps_d, double* drho_d, const void* factors_d,
                                      size_t factors_bytes, void* workspace_d, size_t workspace_bytes,
                                      void* stream);

/* ---------------------------------------------------------------- tensor-core GEMM */

/* The tcgen05 GEMM the dense solves are built on (no counterpart in the thesis; it
 * carries the factorisation updates of App. B's K B = E solve), exposed for testing:
 *   C = alpha * A B^T + beta * C
 *   A_d  device 16-bit [M][lda] (bf16, or fp16 when fp16 = 1), K-major (row-major, K
 *        contiguous); B_d device 16-bit [N][ldb], K-major; lda, ldb multiples of 8 and
 *        A_d, B_d 16-byte aligned;  C_d device fp32 [M][ldc].
 * fp32 accumulation in tensor memory. Errors: RG_ERR_ARG (layout), RG_ERR_CUDA. */
rg_status rg_tc_gemm(rg_ctx* ctx, int32_t M, int32_t N, int32_t K, const void* A_d, int64_t lda,
                     const void* B_d, int64_t ldb, int32_t fp16, float* C_d, int64_t ldc, float alpha,
                     float beta, void* stream);

/* The two pieces of the dense solves' exact refinement (App. B.2 mixed precision: the
 * residual R = E - K B is tracked exactly while the tensor cores run in bf16), exposed for
 * testing; no counterpart in the thesis.
 *
 * rg_exact_split: the fixed-point split of P' = P diag(dr) (dr may be NULL) row by row. With
 *   e_i the exponent of max_k |P'_ik| (max = m 2^e_i, m in [0.5, 1); e_i = 0 for a zero row)
 *   and q_ik = round(P'_ik 2^(39 - e_i)) (to nearest, ties to even; |q| < 2^39), the five
 *   slices are the balanced base-256 digits of q: q = sum_a s_a 256^(4 - a), s_1..s_4 in
 *   [-128, 127], |s_0| <= 128, so that P'_ik = 2^(e_i - 7) sum_a s_a 2^(-8a) to 2^(e_i - 40).
 *   P_d       device fp64 [n][ldp] (or, with trans = 1, P_ik read as P_d[k][i])
 *   dr_d      device fp64 [n] or NULL
 *   slices_d  device int16 [n][5][np] (output): s_a of P'_ik at [i][a][k], zero for k >= n;
 *             np = n rounded up to a multiple of 128
 *   rowexp_d  device int32 [n] (output): e_i
 *   Errors: RG_ERR_ARG; RG_ERR_NUMERIC for a non-finite P'.
 *
 * rg_tc_gemm_exact: the level product on tcgen05 for integer operands:
 *   S_a[i][j] = sum_k A[i][a np + k] B[j][k]  for a = 0 .. levels-1,
 *   A_d  device bf16 [M][lda] (lda >= 5 np), every element an integer of magnitude <= 128;
 *   B_d  device bf16 [N][np], every element an integer of magnitude <= 127 (then every
 *        product is at most 16,256 and every partial sum of a 1,024-long chunk is an integer
 *        below 2^24, exact in the fp32 tensor-core accumulator); np a multiple of 128
 *   S_d  device int32 [levels][M][N] (output), exact for |S| < 2^31
 *   Errors: RG_ERR_ARG (layout, levels outside 1..5), RG_ERR_CUDA. */
rg_status rg_exact_split(rg_ctx* ctx, int32_t n, const double* P_d, int64_t ldp, int32_t trans, const double* dr_d,
                         int16_t* slices_d, int32_t* rowexp_d, void* stream);
rg_status rg_tc_gemm_exact(rg_ctx* ctx, int32_t M, int32_t N, int32_t np, int32_t levels, const void* A_d,
                           int64_t lda, const void* B_d, int32_t* S_d, void* stream);

/* ---------------------------------------------------------------- failure-detection checks */

/* Test support with no counterpart in the thesis: each runs one of the library's bounded
 * device waits against a flag that nothing sets, so that the wait runs out after
 * limit_s seconds (0 < limit_s <= 2), and returns the status a real timeout produces.
 *   rg_debug_mbarrier_timeout  the mbarrier wait of the tensor-core GEMM (one block waits
 *                              on a barrier no one arrives on);
 *   rg_debug_barrier_timeout   the grid barrier of the persistent iterative enforcer (a
 *                              cooperative launch of two blocks, one of which never
 *                              arrives).
 * Expected result: RG_ERR_CUDA with rg_last_error naming the timeout; the kernel ends
 * on its own, nothing traps, and the context stays usable. RG_OK means the wait did
 * not run out (a defect). */
rg_status rg_debug_mbarrier_timeout(rg_ctx* ctx, double limit_s, void* stream);
rg_status rg_debug_barrier_timeout(rg_ctx* ctx, double limit_s, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RADGEB_H */
