/*
 * pdg.h - C ABI of the GB300 (sm_103a) per-iteration step of
 *         Preconditioned Deformation Grids (arXiv 2509.18097).
 *
 * The library fits, frame by frame, a multi-resolution displacement grid G_t that maps
 * the previous frame's template vertices X_{t-1} and source points P_{t-1} onto the
 * target cloud P_t (Sec. 3, problem statement).  One optimisation iteration (a "step")
 * is:
 *   (a) y = x + (1/L) sum_l trilerp(G^l, x) on Q = X_{t-1} u P_{t-1}       (Sec. 3.1, Eq. 1)
 *   (b) exact bidirectional robust-Chamfer nearest neighbours + gradient    (Sec. 3.4)
 *   (c) weak edge isometry + gradient                                      (Sec. 3.4)
 *   (d) adjoint of (a): point gradients into grid-vertex gradients         (chain rule of Eq. 1)
 *   (e) (I + lambda_l L_l)^{-2} per level, then Adam with lr_l             (Sec. 3.2 Eq. 3, Sec. 3.6)
 * Every stage runs in hand-written CUDA kernels; a step is replayed as one CUDA graph.
 *
 * Conventions (all entry points):
 *  - Errors: nothing aborts.  Every call returns a pdg_status; pdg_last_error() gives
 *    the message of the last failing call on a context.  A non-OK return leaves the
 *    context usable, except PDG_ERR_CUDA caused by a sticky device error.
 *  - Streams: `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *    work is ordered on it; calls return without synchronising unless stated.
 *  - Point arrays are float32 [n][3] (x, y, z interleaved, 12-byte stride).  Unless a
 *    call says otherwise a pointer may be device memory (used in place, stream-ordered)
 *    or host memory (pageable or pinned; copied in the call, which then synchronises
 *    `cuda_stream` before returning so the caller may free it).
 *  - Ownership: the library copies what it keeps (template, edges, current source
 *    cloud, target); caller buffers need only live for the call.  Output buffers are
 *    caller-allocated.
 *  - Grid level l (0 = coarsest) has res[l] vertices per axis spanning [lo, hi] with
 *    corners aligned; its values are float32 [res^3][C] indexed ((z*res + y)*res + x), C = 3
 *    (displacement payload) or 6 (Cayley payload, see pdg_config.payload).
 */
#ifndef PDG_H
#define PDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDG_MAX_LEVELS 8

typedef enum pdg_status {
  PDG_OK = 0,
  PDG_ERR_INVALID = 1,   /* bad argument (sizes, NULL, non-finite input, config) */
  PDG_ERR_OOM = 2,       /* device allocation failed */
  PDG_ERR_BUDGET = 3,    /* request exceeds a memory budget or a fixed capacity */
  PDG_ERR_CUDA = 4,      /* a CUDA runtime call failed */
  PDG_ERR_NONFINITE = 5, /* a loss became NaN/Inf during a fit */
  PDG_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
  PDG_ERR_STATE = 7      /* call out of order (e.g. pdg_step outside a frame) */
} pdg_status;

/* Optimisation settings.  pdg_config_default() fills the paper's values:
 * alpha = 5.56 (Sec. 3.4, w_R); w_iso = 250 (Sec. 3.4); Adam (0.9, 0.999, 1e-8),
 * lr_l = 5e-3 * 1.1^l, lambda_l = 0.25 * 1.5^l with l = 0 the coarsest level (Sec. 3.6);
 * without preconditioning the learning rate is scaled by 0.1 (Sec. 4, ablation). */
typedef struct pdg_config {
  int n_levels;               /* 1..PDG_MAX_LEVELS */
  int res[PDG_MAX_LEVELS];    /* vertices per axis, coarse -> fine: 1, or 2^a 3^b in 2..256 (the
                                 preconditioner's line transforms are radix-2/3 FFTs) */
  float lo[3], hi[3];         /* grid domain (default [-1.5, 1.5]^3); points outside are clamped */
  float alpha;                /* robust Chamfer weight exp(-alpha d^2) */
  float w_chamfer_mesh;       /* weight of CD_R(X_hat_t, P_t) (the confidence weight; 1) */
  float w_chamfer_pts;        /* weight of CD_R(P_hat_t, P_t) (1) */
  float w_iso;                /* isometry weight (250) */
  float lr0, lr_growth;       /* per-level learning rate lr0 * lr_growth^l */
  float lambda0, lambda_growth; /* per-level smoothness weight */
  float beta1, beta2, eps;    /* Adam */
  int precondition;           /* 1: (I + lambda L)^{-2} (Eq. 3); 0: raw gradient, lr x 0.1 */
  int robust_weight_stopgrad; /* 1: the robust weight is not differentiated */
  int warm_start;             /* 1: a frame starts from the previous frame's grids */
  int payload;                /* PDG_PAYLOAD_DISPLACEMENT (0) or PDG_PAYLOAD_CAYLEY (1), see below */
} pdg_config;

/* Payload of a grid vertex.  DISPLACEMENT: 3 floats u, a point moves to x + u(x) (the
 * rotation part of Sec. 3.3 held at the identity).  CAYLEY: the 6-D vector T = (z, t) of
 * Sec. 3.3; the averaged T(x) (Eq. 1) moves x to R(z) x + t with R(z) = (I + Z)(I - Z)^{-1},
 * Z the skew-symmetric matrix of z (rotation about the world origin).  Level values are then
 * float [res^3][6] ordered (z0, z1, z2, t0, t1, t2), and every level must have 1 or a power
 * of two up to 128 vertices per axis (PDG_ERR_INVALID otherwise). */
#define PDG_PAYLOAD_DISPLACEMENT 0
#define PDG_PAYLOAD_CAYLEY 1

/* Losses of the last iteration of a frame (evaluated before that iteration's update). */
typedef struct pdg_fit_stats {
  double loss_total; /* w_mesh * cd_mesh + w_pts * cd_pts + w_iso * iso */
  double cd_mesh;    /* CD_R(X_hat_t, P_t) */
  double cd_pts;     /* CD_R(P_hat_t, P_t) */
  double iso;        /* L_iso (unweighted) */
  int n_steps;       /* iterations run in the frame */
  int status;        /* pdg_status of the frame */
  int nn_ties;       /* nearest-neighbour queries of the last iteration whose neighbour was decided
                        by an exact tie of fp32 squared distances (the lowest index won; a reading,
                        the paper does not say how ties break); counted only while
                        PDG_DEBUG_COUNT_NN is set, else -1 */
} pdg_fit_stats;

typedef struct pdg_ctx pdg_ctx;
typedef struct pdg_batch pdg_batch;

/* Fills `cfg` with the paper's defaults and levels 16, 32, 64, 128 over [-1.5, 1.5]^3. */
void pdg_config_default(pdg_config* cfg);

/* Device bytes a context with these sizes allocates (max_pts bounds every source and
 * target cloud it will see).  0 on an invalid configuration. */
size_t pdg_query_bytes(const pdg_config* cfg, int n_verts, int n_edges, int max_pts);

/* Creates a fitting context for one sequence (Sec. 3, problem statement): the template
 * mesh X_0 (verts [n_verts][3], edges int32 [n_edges][2], 0-based vertex ids) and the
 * first source cloud P_0 ([n_src][3]).  max_pts (>= n_src) bounds all later clouds.
 * Allocates all device memory up front.  Errors: PDG_ERR_INVALID (sizes, edge ids out of
 * range, non-finite coordinates, config), PDG_ERR_OOM, PDG_ERR_CUDA. */
pdg_status pdg_create(const pdg_config* cfg, const float* template_xyz, int n_verts, const int32_t* edges,
                      int n_edges, const float* source_xyz, int n_src, int max_pts, void* cuda_stream,
                      pdg_ctx** out);

/* Starts fitting G_t toward the target P_t ([n_tgt][3], 1 <= n_tgt <= max_pts): per-frame
 * set-up (target cell grid, per-level point-to-vertex interpolation lists, edge rest
 * lengths from X_{t-1}, grid/Adam reset).  PDG_ERR_STATE if a frame is already open. */
pdg_status pdg_begin_frame(pdg_ctx* ctx, const float* target_xyz, int n_tgt, void* cuda_stream);

/* Runs n_steps optimisation iterations of the open frame (one CUDA-graph replay each). */
pdg_status pdg_step(pdg_ctx* ctx, int n_steps, void* cuda_stream);

/* Closes the frame: X_t = X_{t-1} + u_t(X_{t-1}) with the final grids (Sec. 3.3) and
 * P_t becomes the next source.  Synchronises `cuda_stream`; fills `stats` (may be NULL).
 * Returns PDG_ERR_NONFINITE (frame still closed and advanced) if a loss was NaN/Inf. */
pdg_status pdg_end_frame(pdg_ctx* ctx, pdg_fit_stats* stats, void* cuda_stream);

/* pdg_begin_frame + pdg_step(n_steps) + pdg_end_frame. */
pdg_status pdg_fit_frame(pdg_ctx* ctx, const float* target_xyz, int n_tgt, int n_steps, pdg_fit_stats* stats,
                         void* cuda_stream);

/* out = xyz + u(xyz) with the context's current grids (Eq. 1 / Sec. 3.3) for n arbitrary
 * points; out_xyz is [n][3] in the same memory kind rules as inputs (host outputs are
 * written before the call returns). */
pdg_status pdg_deform(pdg_ctx* ctx, const float* xyz, int n, float* out_xyz, void* cuda_stream);

/* Copies the current deformed template X_t ([n_verts][3]) to out_xyz (host or device). */
pdg_status pdg_get_vertices(pdg_ctx* ctx, float* out_xyz, void* cuda_stream);

/* Inspection of internal buffers (tests, autograd, debugging); out may be host or device.
 * `level` is used by the per-level buffers.  out_bytes must be at least the size given. */
enum pdg_buffer {
  PDG_BUF_THETA = 0,    /* level values, float [res^3][C] (C = 3, or 6 with the Cayley payload) */
  PDG_BUF_GRAD = 1,     /* dLoss/dTheta of the last step, float [res^3][C] */
  PDG_BUF_PGRAD = 2,    /* preconditioned gradient of the last step, float [res^3][C]
                           (only kept when pdg_set_debug(ctx, 1) was called) */
  PDG_BUF_Y = 3,        /* deformed query points y of the last step, float [n_verts+n_src][3] */
  PDG_BUF_POINT_GRAD = 4, /* dLoss/dy of the last step, float [n_verts+n_src][3] */
  PDG_BUF_NN_FWD = 5,   /* int32 [n_verts+n_src]: nearest target point of each query */
  PDG_BUF_NN_REV = 6,   /* int32 [2][n_tgt]: nearest template vertex / source point of each target point */
  PDG_BUF_LOSS = 7,     /* double [4]: total, cd_mesh, cd_pts, iso of the last step */
  PDG_BUF_SOURCE = 8,   /* current source cloud P_{t-1}, float [n_src][3] */
  PDG_BUF_COUNTERS = 9, /* uint64 [4] of the last step: squared distances the nearest-neighbour
                           search evaluated and queries decided by an exact tie (both counted
                           only with PDG_DEBUG_COUNT_NN, else 0), queries left to the
                           warp-cooperative ring search, 0 */
  PDG_BUF_MESH_GRAD = 10, /* dL_mesh/dX of the last pdg_fit_mesh iteration, float [n_verts][3]
                             (PDG_ERR_STATE before a fit, or once a frame has begun since) */
  PDG_BUF_MESH_PGRAD = 11 /* the same preconditioned, (I + lambda L)^{-2} dL_mesh/dX */
};
pdg_status pdg_read(pdg_ctx* ctx, int which, int level, void* out, size_t out_bytes, void* cuda_stream);

/* Overwrites level `level`'s values with theta (float [res^3][C], host or device) and
 * resets its Adam moments.  Valid inside a frame (used to start from given grids). */
pdg_status pdg_write_theta(pdg_ctx* ctx, int level, const float* theta, void* cuda_stream);

/* Profiling: runs n_steps iterations of the open frame as eager launches of the same
 * stages the step graph holds, bracketing each stage with CUDA events on `cuda_stream`,
 * and writes the summed milliseconds per stage to stage_ms[pdg_profile_stages()].
 * Synchronises the stream after every iteration.  The stages are listed by
 * pdg_profile_stage_name(i). */
int pdg_profile_stages(void);
const char* pdg_profile_stage_name(int i);
pdg_status pdg_profile_step(pdg_ctx* ctx, int n_steps, double* stage_ms, void* cuda_stream);

/* Number of kernel launches one pdg_step iteration performs: the kernel nodes of the
 * context's captured step graph, counted when the graph was captured.  *out = 0 before the
 * first pdg_step of the context (the graph is captured then).  No GPU work. */
pdg_status pdg_step_kernel_count(const pdg_ctx* ctx, int* out);

/* Evaluates the loss and its gradients at the current grids without changing them: the
 * step's forward and backward kernels (evaluation, nearest neighbours and robust-Chamfer
 * gradient, isometry gradient, adjoint into the grids), no preconditioner, no Adam, no
 * step count.  Afterwards PDG_BUF_LOSS, PDG_BUF_GRAD (dLoss/dTheta per level),
 * PDG_BUF_POINT_GRAD hold the results.  `loss` (host, may be NULL) receives total,
 * cd_mesh, cd_pts, iso (the call then synchronises).  Inside a frame only. */
pdg_status pdg_eval(pdg_ctx* ctx, double* loss, void* cuda_stream);

/* The grid Sobolev preconditioner of level `level` applied to a caller-given gradient:
 * out = (I + lambda_l L_l)^{-2} g per channel (Sec. 3.2, Eq. 3; L_l the free-boundary
 * 6-neighbour graph Laplacian of the level's vertex grid), with the same kernels as the
 * step.  g, out: float [res^3][3], host or device.  Only between frames (the level's
 * gradient buffers are used as scratch): PDG_ERR_STATE inside a frame.  Synchronises. */
pdg_status pdg_precondition(pdg_ctx* ctx, int level, const float* g, float* out, void* cuda_stream);

/* Template-mesh fit (Sec. 3.4, surface initialisation loss; Sec. 3.6): moves the context's
 * template vertices X (the mesh the next frame starts from; X_0 before the first frame) to
 * reduce L_mesh = CD_R(X, P_0) against the keyframe cloud p0_xyz ([n_p0][3], host or device,
 * 1 <= n_p0 <= max_pts), by n_steps iterations of: the exact robust Chamfer search and
 * gradient (the step's kernels, mesh term only), the gradient preconditioned by
 * (I + lambda L_mesh)^{-2} with L_mesh the combinatorial graph Laplacian of the mesh edges
 * (two Chebyshev solves, relative error below 1e-7 in exact arithmetic), then Adam with
 * learning rate lr (fresh moments each call; beta1, beta2, eps of the context's config).
 * The paper's values are lambda = 16, lr = 1e-4; lambda >= 0 with lambda times the largest
 * vertex degree at most 1e5, lr >= 0, n_steps >= 0 (PDG_ERR_INVALID otherwise; n_p0 above
 * max_pts: PDG_ERR_BUDGET).  Between frames only (PDG_ERR_STATE inside
 * a frame); the source cloud and the grids are untouched.  stats (may be NULL): loss_total =
 * cd_mesh = L_mesh of the last iteration (before its update).  Synchronises `cuda_stream`.
 * PDG_ERR_NONFINITE if a loss was NaN/Inf (the vertices are then as the fit left them). */
pdg_status pdg_fit_mesh(pdg_ctx* ctx, const float* p0_xyz, int n_p0, int n_steps, float lambda, float lr,
                        pdg_fit_stats* stats, void* cuda_stream);

/* Debug flags (bitwise or), applied to the following steps: PDG_DEBUG_KEEP_PGRAD keeps the
 * preconditioned gradient of each step readable as PDG_BUF_PGRAD; PDG_DEBUG_COUNT_NN runs the
 * nearest-neighbour search's counting instance, which counts the squared distances it
 * evaluates and the queries an exact tie decided (PDG_BUF_COUNTERS, pdg_fit_stats.nn_ties;
 * slower: leave it off while timing).  Changing PDG_DEBUG_COUNT_NN re-captures the context's
 * step graph at its next pdg_step; a batch never counts.  Unknown bits: PDG_ERR_INVALID.
 * Synchronises the device. */
#define PDG_DEBUG_KEEP_PGRAD 1
#define PDG_DEBUG_COUNT_NN 2
pdg_status pdg_set_debug(pdg_ctx* ctx, int flags);

/* Test hook: the library's next n device allocations (context arenas, batch tables) fail as
 * if the device were out of memory, so that callers can exercise their PDG_ERR_OOM paths;
 * the failing call frees whatever it had already taken.  n <= 0 turns the hook off.
 * Process-wide; no GPU work. */
void pdg_debug_fail_allocations(int n);

void pdg_destroy(pdg_ctx* ctx);
const char* pdg_status_string(pdg_status s);
const char* pdg_last_error(const pdg_ctx* ctx);

/* ---- batching (continuous batching of independent sequences) --------------------------
 * A batch runs one iteration of every member context in one CUDA-graph launch of
 * batched kernels (each kernel iterates over (job, work item) pairs of all members).
 * Members must be inside a frame (pdg_begin_frame).  Membership may change between
 * calls; results per context are the same as running it alone. */
pdg_status pdg_batch_create(int max_jobs, pdg_batch** out);
pdg_status pdg_batch_set(pdg_batch* b, pdg_ctx* const* ctxs, int n_jobs);
pdg_status pdg_batch_step(pdg_batch* b, int n_steps, void* cuda_stream);
void pdg_batch_destroy(pdg_batch* b);

/* ---- checkpoint / resume (between frames) ------------------------------------------- */
size_t pdg_state_bytes(const pdg_ctx* ctx);
pdg_status pdg_save_state(pdg_ctx* ctx, void* host_buf, size_t n, void* cuda_stream);
pdg_status pdg_load_state(pdg_ctx* ctx, const void* host_buf, size_t n, void* cuda_stream);

/* ---- allocation-free preconditioner --------------------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers that cannot
 * allocate device memory when they need the preconditioner: a service whose device-memory
 * budget was fixed at start-up, a host allocator that must not be re-entered from the
 * calling thread, or a latency-critical path on which any allocation is forbidden.
 *
 * out = (I + lambda L)^{-2} g per channel on a res^3 vertex grid (L the free-boundary
 * 6-neighbour graph Laplacian), computed by the same preconditioner kernels as
 * pdg_precondition, without a context and without allocating: its scratch lives in one
 * fixed file-scope device array of about 6.5 MB (two res^3 x 3 float buffers and the z-solve
 * pivot table at the maximum res, plus small tables and records), which every GPU that loads
 * the library keeps until the process exits.
 *  - g, out: DEVICE pointers of the current device to float [res^3][3] ((z*res + y)*res + x);
 *    host pointers or another GPU's memory give PDG_ERR_INVALID.  The call cannot check
 *    their length: each must hold res^3 * 3 floats.  res: 1 or a power of two up to
 *    PDG_STATIC_MAX_RES; larger grids give PDG_ERR_BUDGET (use pdg_precondition).
 *    lambda: finite, >= 0.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    and sets the kernels' shared-memory limits; make that first call before any stream
 *    capture.
 *  - Every call uses the same array and leaves its contents behind; each call writes its
 *    tables, job record and gradient copy before reading them, so nothing carries over.
 *    Calls in one process whose work overlaps on the GPU (other streams or threads) race on
 *    the array: serialise them.  (Each process has its own copy of the array.)
 *  - Asynchronous on `cuda_stream`: every table and record is written by a kernel from its
 *    launch arguments, so nothing is copied from host memory, allocated, freed or
 *    synchronised.  A launch error left by earlier work on the calling thread is cleared on
 *    entry, so the status returned is this call's. */
#define PDG_STATIC_MAX_RES 64
pdg_status pdg_precondition_static(int res, float lambda, const float* g, float* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PDG_H */
