// Host runtime and C ABI of libpdg: per-sequence contexts (one device arena each),
// per-frame set-up, the CUDA-graph step, batching of contexts into one graph, and
// checkpoint/resume.  See include/pdg.h for the contract of every entry point.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"

using namespace pdg;

namespace {

constexpr double PI = 3.14159265358979323846;

struct Arena {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += count * sizeof(T);
    return at;
  }
};

// Cells per axis (log2) of a nearest-neighbour grid over `count` points on a surface, with
// about `per_cell` points in an occupied cell.
int grid_bits(long count, double per_cell = 8.0) {
  const double g = std::sqrt(std::max(count, 1L) / per_cell);
  int b = (int)std::lround(std::log2(std::max(g, 1.0)));
  return std::min(std::max(b, 2), 7);
}

// Largest resolution of the levels the tile path preconditions, per size class (0: none).
// Each class is launched with its own shared-memory size, so that small tile levels keep
// several blocks per SM when a level above TILE_SPLIT shares the step (a batch).
constexpr int TILE_SPLIT = 108;
struct TileSizes {
  int small = 0;  // tile levels of at most TILE_SPLIT vertices per axis
  int big = 0;    // tile levels above TILE_SPLIT
};
TileSizes tile_sizes(int n) {
  TileSizes t;
  if (tile_level(n)) (n <= TILE_SPLIT ? t.small : t.big) = n;
  return t;
}
TileSizes tmax(TileSizes a, TileSizes b) {
  a.small = std::max(a.small, b.small);
  a.big = std::max(a.big, b.big);
  return a;
}
bool tgreater(TileSizes a, TileSizes b) { return a.small > b.small || a.big > b.big; }

// 1, or 2..256 with no prime factor but 2 and 3 (the line transforms are radix-2/3 FFTs)
bool valid_res(int n) {
  if (n < 1 || n > 256) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Test hook: the next `g_fail_allocs` device allocations of the library report failure.
std::atomic<int> g_fail_allocs{0};

cudaError_t dev_malloc(void** p, size_t bytes) {
  int n = g_fail_allocs.load();
  while (n > 0)
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  return cudaMalloc(p, bytes);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// --------------------------------------------------------------------------------- context

struct pdg_ctx {
  pdg_config cfg{};
  int dev = 0, sms = 1;
  int V = 0, E = 0, max_pts = 0, Qmax = 0;
  bool in_frame = false;
  int steps_in_frame = 0;
  std::string err;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  Job h{};                 // host mirror of the device job struct
  Job* dJ = nullptr;       // device job struct (inside the arena)
  Plan* dplan = nullptr;   // device plan holding only this job
  Job* op_job = nullptr;   // scratch job / plan for single-level operations
  Plan* op_plan = nullptr;
  int* dflag = nullptr;
  float4* mesh = nullptr;  // [7][V]: h, r, d0, d1, preconditioned gradient, Adam m, Adam v
  int max_degree = 0;      // largest vertex degree of the mesh (bounds the Laplacian's spectrum)
  bool mesh_valid = false; // a template-mesh fit has run (PDG_BUF_MESH_* readable)
  float* stage = nullptr;  // [stage_pts][3] staging of host inputs
  int stage_pts = 0;
  int nmax = 1;
  TileSizes ntile;  // largest resolutions among the levels the tile path preconditions
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_kernels = 0;   // kernel nodes of gexec
  bool plan_stale = true;  // dplan's item prefixes predate the current frame
  unsigned long long frame_gen = 0;  // frames begun (a batch recomputes its plan when one changes)
  std::vector<int> v2e_ptr, v2e;

  pdg_status fail(pdg_status s, const std::string& m) {
    err = m;
    return s;
  }
  pdg_status cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PDG_OK;
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return PDG_ERR_CUDA;
  }
};

struct pdg_batch {
  int max_jobs = 0;
  int n = 0;
  std::vector<pdg_ctx*> members;
  Plan* dplan = nullptr;
  Plan* hplan = nullptr;  // pinned host copy
  std::vector<unsigned long long> gens;  // members' frame_gen when dplan's prefixes were computed
  cudaStream_t cap = nullptr, cap2 = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_nmax = 0;
  TileSizes graph_ntile;
  bool dirty = true;  // membership changed since the last upload of the job table
  std::string err;
};

#define TRY(expr)                                  \
  do {                                             \
    pdg_status _s = (expr);                        \
    if (_s != PDG_OK) return _s;                   \
  } while (0)
#define CU(ctx, call) TRY((ctx)->cuda((call), #call))

namespace {

// sizes of every buffer of a context (used by pdg_query_bytes and pdg_create)
struct Layout {
  size_t total = 0;
  size_t job, plan, flag, stage, op_job, op_plan;
  struct Lv {
    size_t theta, theta_t, m, v, g, tmp, zmask, piv, piv_slow, mu, tw, tw4, cnt, rowptr, flag, act_v, act_ptr, ent, ccnt,
        coff, ckey, xs, n_active, csum;
    int cap;
  } lv[MAXL];
  size_t x, y, gfwd, gy, zq, uq, gz, acc, loss_fwd, loss_rev, loss_iso, nn_fwd, nn_rev, edge_d, edges, e_prev, v2e_ptr, v2e;
  size_t src4, tgt4, verts4;
  size_t t_hist, t_off, t_keys, t_pts, t_csum, m_hist, m_off, m_keys, m_pts, m_csum;
  size_t hard, hard_count, step, bias, loss, status, loss_part, gmax, counters;
  size_t mesh;  // template-mesh fit: 7 float4 [V] arrays (gradient copy, solves, Adam moments)
  int tbits, mbits;
};

Layout make_layout(const pdg_config& c, int V, int E, int max_pts) {
  Layout L;
  Arena a;
  const int Q = V + max_pts;
  const size_t C = c.payload == PDG_PAYLOAD_CAYLEY ? 6 : 3;
  L.job = a.take<Job>(1);
  L.plan = a.take<Plan>(1);
  L.op_job = a.take<Job>(1);
  L.op_plan = a.take<Plan>(1);
  L.flag = a.take<int>(4);
  const int sp = std::max(V, max_pts);
  L.stage = a.take<float>(3 * (size_t)sp);
  for (int l = 0; l < c.n_levels; ++l) {
    const size_t n = c.res[l], n3 = n * n * n;
    auto& v = L.lv[l];
    v.cap = (int)std::min<size_t>(n3, 8 * (size_t)Q);
    v.theta = a.take<float4>(n3);
    v.theta_t = a.take<float4>(C == 6 ? n3 : 1);
    v.m = a.take<float>(C * n3);
    v.v = a.take<float>(C * n3);
    v.g = a.take<float>(C * n3);
    v.tmp = a.take<float>(C * n3);
    v.zmask = a.take<int>(n);
    v.piv = a.take<float>(tile_level(n) ? 1 : (n / 2 + 1) * n * n);
    v.piv_slow = a.take<int>(1);
    v.mu = a.take<float>(n);
    v.tw = a.take<float2>(n);
    v.tw4 = a.take<float2>(n);
    v.cnt = a.take<int>(n3);
    v.rowptr = a.take<int>(n3 + 1);
    v.flag = a.take<int>(n3 + 1);
    v.act_v = a.take<int>(v.cap);
    v.act_ptr = a.take<int>(v.cap + 1);
    v.ent = a.take<int2>(8 * (size_t)Q);
    const bool fin = l == c.n_levels - 1;  // the cell order is kept for the finest level only
    const size_t cells = fin ? (n > 1 ? (n - 1) * (n - 1) * (n - 1) : 1) : 1;
    v.ccnt = a.take<int>(cells);
    v.coff = a.take<int>(cells + 1);
    v.ckey = a.take<int>(fin ? Q : 1);
    v.xs = a.take<float4>(fin ? Q : 1);
    v.n_active = a.take<int>(1);
    v.csum = a.take<int>((n3 + 1) / SCAN_CHUNK + 2);
  }
  L.x = a.take<float4>(Q);
  L.y = a.take<float4>(Q);
  L.gfwd = a.take<float4>(Q);
  L.gy = a.take<float4>(Q);
  L.zq = a.take<float4>(C == 6 ? Q : 1);
  L.uq = a.take<float4>(C == 6 ? Q : 1);
  L.gz = a.take<float4>(C == 6 ? Q : 1);
  L.acc = a.take<long long>(3 * (size_t)Q);
  L.loss_fwd = a.take<float>(Q);
  L.loss_rev = a.take<float>(2 * (size_t)max_pts);
  L.loss_iso = a.take<float>(std::max(E, 1));
  L.nn_fwd = a.take<int>(Q);
  L.nn_rev = a.take<int>(2 * (size_t)max_pts);
  L.edge_d = a.take<float4>(std::max(E, 1));
  L.edges = a.take<int2>(std::max(E, 1));
  L.e_prev = a.take<float>(std::max(E, 1));
  L.v2e_ptr = a.take<int>(V + 1);
  L.v2e = a.take<int>(std::max(2 * E, 1));
  L.src4 = a.take<float4>(max_pts);
  L.tgt4 = a.take<float4>(max_pts);
  L.verts4 = a.take<float4>(V);
  // about 32 points per occupied cell in both NN grids: during a fit the nearest neighbour is
  // often one or two spacings of a finer grid away, and the 3x3x3 box of these cells
  // certifies almost every query in the one-thread-per-query pass (the moving grid is also
  // rebuilt every step, its offsets a scan over all its cells)
  L.tbits = grid_bits(max_pts, 32.0);
  L.mbits = grid_bits(std::max(V, max_pts), 32.0);
  const size_t tG3 = size_t(1) << (3 * L.tbits), mG3 = size_t(1) << (3 * L.mbits);
  L.t_hist = a.take<int>(tG3);
  L.t_off = a.take<int>(tG3 + 1);
  L.t_keys = a.take<int>(max_pts);
  L.t_pts = a.take<float4>(max_pts);
  L.t_csum = a.take<int>(tG3 / SCAN_CHUNK + 2);
  L.m_hist = a.take<int>(2 * mG3);
  L.m_off = a.take<int>(2 * mG3 + 1);
  L.m_keys = a.take<int>(Q);
  L.m_pts = a.take<float4>(Q);
  L.m_csum = a.take<int>(2 * mG3 / SCAN_CHUNK + 2);
  L.hard = a.take<int4>(Q + 2 * (size_t)max_pts);
  L.loss_part = a.take<float>(5 * ((Q + 2 * (size_t)max_pts + std::max(E, 1)) / LOSS_CHUNK + 2));
  L.hard_count = a.take<int>(1);
  L.step = a.take<int>(1);
  L.bias = a.take<float>(2);
  L.loss = a.take<double>(4);
  L.status = a.take<int>(1);
  L.gmax = a.take<unsigned>(1);
  L.counters = a.take<unsigned long long>(4);
  L.mesh = a.take<float4>(7 * (size_t)V);
  L.total = (a.off + 255) & ~size_t(255);
  return L;
}

const char* check_config(const pdg_config* c) {
  if (!c) return "config is NULL";
  if (c->n_levels < 1 || c->n_levels > PDG_MAX_LEVELS) return "n_levels must be in 1..8";
  for (int l = 0; l < c->n_levels; ++l)
    if (!valid_res(c->res[l])) return "each res must be 1 or 2^a 3^b in 2..256";
  if (c->payload != PDG_PAYLOAD_DISPLACEMENT && c->payload != PDG_PAYLOAD_CAYLEY) return "unknown payload";
  if (c->payload == PDG_PAYLOAD_CAYLEY)
    for (int l = 0; l < c->n_levels; ++l)
      if (tile_level(c->res[l]))
        return "the Cayley payload takes levels of 1 or a power of two up to 128 vertices per axis";
  for (int a = 0; a < 3; ++a)
    if (!(std::isfinite(c->lo[a]) && std::isfinite(c->hi[a]) && c->hi[a] > c->lo[a])) return "domain must have lo < hi";
  const float f[] = {c->alpha, c->w_chamfer_mesh, c->w_chamfer_pts, c->w_iso, c->lr0, c->lr_growth, c->lambda0,
                     c->lambda_growth, c->beta1, c->beta2, c->eps};
  for (float v : f)
    if (!std::isfinite(v) || v < 0) return "config parameters must be finite and non-negative";
  if (c->beta1 >= 1 || c->beta2 >= 1) return "beta1, beta2 must be < 1";
  return nullptr;
}

// copies `n` xyz triples (host or device) into a float4 device array
pdg_status load_points(pdg_ctx* c, const float* xyz, int n, float4* dst, cudaStream_t s, bool check) {
  if (n <= 0) return PDG_OK;
  const float* src = xyz;
  if (!is_device_ptr(xyz)) {
    if (n > c->stage_pts) return c->fail(PDG_ERR_BUDGET, "point count exceeds the context capacity");
    CU(c, cudaMemcpyAsync(c->stage, xyz, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
    src = c->stage;
  }
  if (check) {
    CU(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), s));
    launch_check_finite(src, 3 * n, c->dflag, s);
    int f = 0;
    CU(c, cudaMemcpyAsync(&f, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(c, cudaStreamSynchronize(s));
    if (f) return c->fail(PDG_ERR_INVALID, "input points contain NaN or Inf");
  }
  launch_pack4(src, dst, n, s);
  return c->cuda(cudaGetLastError(), "pack points");
}

// Copies the host mirror of the job record to the device.  The mirror does not hold what the
// plan kernel writes into the device record (each level's adjoint lanes per row), so the
// plan of the context, and of any batch holding it, is recomputed before the next step.
pdg_status upload_job(pdg_ctx* c, cudaStream_t s) {
  CU(c, cudaMemcpyAsync(c->dJ, &c->h, sizeof(Job), cudaMemcpyHostToDevice, s));
  c->plan_stale = true;
  ++c->frame_gen;
  return PDG_OK;
}

// The step as an explicit list of stages; the graph capture and the profiling path launch
// exactly the same sequence.
const char* const STAGE_NAMES[] = {"interp",     "mov_scan",   "mov_scatter", "nn",          "nn_hard",
                                   "iso_edges",  "assemble",   "adjoint",     "sob_xy_fwd",  "sob_z",
                                   "sob_xy_inv", "adam",       "sobolev_256", "loss"};
constexpr int N_STAGES = sizeof(STAGE_NAMES) / sizeof(STAGE_NAMES[0]);
enum StageIndex {
  S_INTERP = 0, S_MOV_SCAN, S_MOV_SCATTER, S_NN, S_NN_HARD, S_ISO, S_ASSEMBLE, S_ADJOINT,
  S_SOB_XY_FWD, S_SOB_Z, S_SOB_XY_INV, S_ADAM, S_SOB_256, S_LOSS
};

// Stage i of a step; bump: the job_bump mode of the interpolation stage (1: optimisation
// step, 2: evaluation); count: the nearest-neighbour instances that count candidates and
// exact ties.  The plan's item prefixes must be current (refresh_plan).
// nmax: the largest level resolution; ntile: the largest ones of the levels the tile path
// preconditions, per size class
void launch_stage(int i, const Plan* plan, int nmax, TileSizes ntile, int sms, cudaStream_t s, int bump = 1,
                  bool count = false) {
  const int grid = sms * 8;
  switch (i) {
    case S_INTERP: launch_interp(plan, grid, s, bump); break;
    case S_MOV_SCAN: launch_mov_scan(plan, sms * 2, s); break;
    case S_MOV_SCATTER: launch_mov_scatter(plan, grid, s); break;
    case S_NN: launch_nn(plan, grid * 2, s, count); break;
    case S_NN_HARD: launch_nn_hard(plan, sms * 4, s, count); break;
    case S_ISO: launch_iso_edges(plan, grid, s); break;
    case S_ASSEMBLE: launch_assemble(plan, grid, s); break;
    case S_ADJOINT: launch_adjoint(plan, grid * 2, s); break;
    case S_SOB_XY_FWD:
    case S_SOB_Z:
    case S_SOB_XY_INV:
    case S_ADAM: {
      const int ps = plane_smem_max(nmax);
      const int per_sm = std::max(1, std::min(8, (227 * 1024) / ps));
      launch_sobolev_plane(plan, sms * per_sm, nmax, s, i - S_SOB_XY_FWD);
      break;
    }
    case S_SOB_256:
      if (ntile.small > 0) launch_sobolev_tiles(plan, sms, 0, TILE_SPLIT, ntile.small, s);
      if (ntile.big > 0) launch_sobolev_tiles(plan, sms, TILE_SPLIT, 256, ntile.big, s);
      break;
    case S_LOSS: launch_loss(plan, sms * 2, s); break;
  }
}
constexpr int ST_SOB_FIRST = S_SOB_XY_FWD, ST_SOB_LAST = S_SOB_256;  // preconditioner and Adam stages

// Captures one step.  Two branches: the isometry kernel runs beside the moving grid's sort
// and the nearest-neighbour passes (it needs only the deformed points), the loss reduction
// beside the adjoint and the preconditioner (nothing downstream reads it).
pdg_status capture_step(pdg_ctx* c, const Plan* plan, int nmax, TileSizes ntile, cudaStream_t cap, cudaStream_t cap2,
                        cudaGraphExec_t* out, std::string* err, int sms, int* n_kernels = nullptr) {
  cudaGraph_t g = nullptr;
  cudaEvent_t ev[4] = {};
  for (auto& e : ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      *err = "cudaEventCreate failed";
      return PDG_ERR_CUDA;
    }
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    *err = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
    for (auto& x : ev) cudaEventDestroy(x);
    return PDG_ERR_CUDA;
  }
  const bool count = c && c->h.count_nn;  // a batch graph never counts
  launch_stage(S_INTERP, plan, nmax, ntile, sms, cap);  // starts the step of every job
  cudaEventRecord(ev[0], cap);
  cudaStreamWaitEvent(cap2, ev[0], 0);
  launch_stage(S_ISO, plan, nmax, ntile, sms, cap2);
  cudaEventRecord(ev[1], cap2);
  launch_stage(S_MOV_SCAN, plan, nmax, ntile, sms, cap);
  launch_stage(S_MOV_SCATTER, plan, nmax, ntile, sms, cap);
  launch_stage(S_NN, plan, nmax, ntile, sms, cap, 1, count);
  launch_stage(S_NN_HARD, plan, nmax, ntile, sms, cap, 1, count);
  cudaStreamWaitEvent(cap, ev[1], 0);
  launch_stage(S_ASSEMBLE, plan, nmax, ntile, sms, cap);
  cudaEventRecord(ev[2], cap);
  cudaStreamWaitEvent(cap2, ev[2], 0);
  launch_stage(S_LOSS, plan, nmax, ntile, sms, cap2);
  cudaEventRecord(ev[3], cap2);
  for (int i = S_ADJOINT; i <= S_SOB_256; ++i) launch_stage(i, plan, nmax, ntile, sms, cap);  // adjoint, preconditioner, Adam
  cudaStreamWaitEvent(cap, ev[3], 0);
  e = cudaStreamEndCapture(cap, &g);
  for (auto& x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) {
    *err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
    if (g) cudaGraphDestroy(g);
    return PDG_ERR_CUDA;
  }
  if (n_kernels) {  // count the kernel nodes (what one replay launches)
    size_t nn = 0;
    *n_kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
        for (size_t i = 0; i < nn; ++i) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++*n_kernels;
        }
    }
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
    return PDG_ERR_CUDA;
  }
  (void)c;
  return PDG_OK;
}

}  // namespace

extern "C" {

void pdg_config_default(pdg_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->n_levels = 4;
  c->res[0] = 16;
  c->res[1] = 32;
  c->res[2] = 64;
  c->res[3] = 128;
  for (int a = 0; a < 3; ++a) {
    c->lo[a] = -1.5f;
    c->hi[a] = 1.5f;
  }
  c->alpha = 5.56f;
  c->w_chamfer_mesh = 1.f;
  c->w_chamfer_pts = 1.f;
  c->w_iso = 250.f;
  c->lr0 = 5e-3f;
  c->lr_growth = 1.1f;
  c->lambda0 = 0.25f;
  c->lambda_growth = 1.5f;
  c->beta1 = 0.9f;
  c->beta2 = 0.999f;
  c->eps = 1e-8f;
  c->precondition = 1;
  c->robust_weight_stopgrad = 0;
  c->warm_start = 0;
  c->payload = PDG_PAYLOAD_DISPLACEMENT;
}

size_t pdg_query_bytes(const pdg_config* cfg, int n_verts, int n_edges, int max_pts) {
  if (check_config(cfg) || n_verts < 1 || n_edges < 0 || max_pts < 1) return 0;
  return make_layout(*cfg, n_verts, n_edges, max_pts).total;
}

const char* pdg_status_string(pdg_status s) {
  switch (s) {
    case PDG_OK: return "ok";
    case PDG_ERR_INVALID: return "invalid argument";
    case PDG_ERR_OOM: return "out of device memory";
    case PDG_ERR_BUDGET: return "over budget or capacity";
    case PDG_ERR_CUDA: return "CUDA error";
    case PDG_ERR_NONFINITE: return "non-finite loss";
    case PDG_ERR_TIMEOUT: return "device wait timed out";
    case PDG_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* pdg_last_error(const pdg_ctx* c) { return c ? c->err.c_str() : "context is NULL"; }

void pdg_destroy(pdg_ctx* c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  if (c->arena) cudaFree(c->arena);
  delete c;
}

pdg_status pdg_create(const pdg_config* cfg, const float* template_xyz, int n_verts, const int32_t* edges,
                      int n_edges, const float* source_xyz, int n_src, int max_pts, void* cuda_stream,
                      pdg_ctx** out) {
  if (!out) return PDG_ERR_INVALID;
  *out = nullptr;
  if (check_config(cfg) || !template_xyz || !source_xyz || n_verts < 1 || n_src < 1 || max_pts < n_src ||
      n_edges < 0 || (n_edges > 0 && !edges))
    return PDG_ERR_INVALID;
  if ((long)n_verts + max_pts > (1L << 29) || (long)n_edges > (1L << 28)) return PDG_ERR_BUDGET;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  pdg_ctx* c = new pdg_ctx();
  c->cfg = *cfg;
  c->V = n_verts;
  c->E = n_edges;
  c->max_pts = max_pts;
  c->Qmax = n_verts + max_pts;
  auto bail = [&](pdg_status st) {
    pdg_destroy(c);
    return st;
  };
  if (cudaGetDevice(&c->dev) != cudaSuccess) return bail(PDG_ERR_CUDA);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev);
  sobolev_configure();
  sobolev_plane_configure();

  // edges to the host (validation + vertex -> edge lists)
  std::vector<int32_t> he(2 * (size_t)n_edges);
  if (n_edges) {
    if (is_device_ptr(edges)) {
      if (cudaMemcpy(he.data(), edges, he.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return bail(PDG_ERR_CUDA);
    } else {
      std::memcpy(he.data(), edges, he.size() * 4);
    }
  }
  for (size_t i = 0; i < he.size(); ++i)
    if (he[i] < 0 || he[i] >= n_verts) return bail(PDG_ERR_INVALID);
  c->v2e_ptr.assign(n_verts + 1, 0);
  for (int e = 0; e < n_edges; ++e) {
    c->v2e_ptr[he[2 * e] + 1]++;
    c->v2e_ptr[he[2 * e + 1] + 1]++;
  }
  for (int v = 0; v < n_verts; ++v) {
    c->max_degree = std::max(c->max_degree, c->v2e_ptr[v + 1]);
    c->v2e_ptr[v + 1] += c->v2e_ptr[v];
  }
  c->v2e.assign(std::max(2 * n_edges, 1), 0);
  {
    std::vector<int> fill(c->v2e_ptr.begin(), c->v2e_ptr.end() - 1);
    for (int e = 0; e < n_edges; ++e) {  // ascending edge order within each vertex
      c->v2e[fill[he[2 * e]]++] = e << 1;
      c->v2e[fill[he[2 * e + 1]]++] = (e << 1) | 1;
    }
  }

  const Layout L = make_layout(*cfg, n_verts, n_edges, max_pts);
  if (dev_malloc((void**)&c->arena, L.total) != cudaSuccess) {
    cudaGetLastError();
    c->arena = nullptr;
    return bail(PDG_ERR_OOM);
  }
  c->arena_bytes = L.total;
  if (cudaMemsetAsync(c->arena, 0, L.total, s) != cudaSuccess) return bail(PDG_ERR_CUDA);
  char* A = c->arena;
  auto P = [&](size_t off) { return (void*)(A + off); };
  Job& J = c->h;
  std::memset(&J, 0, sizeof(J));
  J.L = cfg->n_levels;
  J.C = cfg->payload == PDG_PAYLOAD_CAYLEY ? 6 : 3;
  for (int a = 0; a < 3; ++a) {
    J.lo[a] = cfg->lo[a];
    J.hi[a] = cfg->hi[a];
  }
  J.alpha = cfg->alpha;
  J.w_mesh = cfg->w_chamfer_mesh;
  J.w_pts = cfg->w_chamfer_pts;
  J.w_iso = cfg->w_iso;
  J.stopgrad = cfg->robust_weight_stopgrad ? 1 : 0;
  J.precondition = cfg->precondition ? 1 : 0;
  J.beta1 = cfg->beta1;
  J.beta2 = cfg->beta2;
  J.eps = cfg->eps;
  J.V = n_verts;
  J.N = n_src;
  J.M = 1;
  J.E = n_edges;
  J.Q = n_verts + n_src;
  J.max_pts = max_pts;
  c->dJ = (Job*)P(L.job);
  c->dplan = (Plan*)P(L.plan);
  c->op_job = (Job*)P(L.op_job);
  c->op_plan = (Plan*)P(L.op_plan);
  c->dflag = (int*)P(L.flag);
  c->mesh = (float4*)P(L.mesh);
  c->stage = (float*)P(L.stage);
  c->stage_pts = std::max(n_verts, max_pts);
  std::vector<float> mu;
  std::vector<float2> tw, tw4;
  for (int l = 0; l < J.L; ++l) {
    Level& lv = J.lev[l];
    const auto& o = L.lv[l];
    const int n = cfg->res[l];
    lv.n = n;
    lv.lg = (n & (n - 1)) == 0 ? ilog2(n) : -1;
    lv.n3 = n * n * n;
    lv.tiles = 3 * ((n * n + TILE_LINES - 1) / TILE_LINES);  // one channel per tile
    lv.lr = (float)(cfg->lr0 * std::pow((double)cfg->lr_growth, l) * (cfg->precondition ? 1.0 : 0.1));
    lv.lam = (float)(cfg->lambda0 * std::pow((double)cfg->lambda_growth, l));
    for (int a = 0; a < 3; ++a) {
      const double sc = (n - 1) / ((double)cfg->hi[a] - (double)cfg->lo[a]);
      lv.sc_hi[a] = (float)sc;
      lv.sc_lo[a] = (float)(sc - (double)lv.sc_hi[a]);
    }
    lv.theta = (float4*)P(o.theta);
    lv.theta_t = J.C == 6 ? (float4*)P(o.theta_t) : nullptr;
    lv.m = (float*)P(o.m);
    lv.v = (float*)P(o.v);
    lv.g = (float*)P(o.g);
    lv.tmp = (float*)P(o.tmp);
    lv.zmask = (int*)P(o.zmask);
    lv.piv = (float*)P(o.piv);
    lv.piv_slow = (int*)P(o.piv_slow);
    lv.mu = (float*)P(o.mu);
    lv.tw = (float2*)P(o.tw);
    lv.tw4 = (float2*)P(o.tw4);
    lv.cnt = (int*)P(o.cnt);
    lv.rowptr = (int*)P(o.rowptr);
    lv.flag = (int*)P(o.flag);
    lv.act_v = (int*)P(o.act_v);
    lv.act_ptr = (int*)P(o.act_ptr);
    lv.ent = (int2*)P(o.ent);
    lv.ccnt = (int*)P(o.ccnt);
    lv.coff = (int*)P(o.coff);
    lv.ckey = (int*)P(o.ckey);
    lv.xs = (float4*)P(o.xs);
    lv.n_active = (int*)P(o.n_active);
    lv.csum = (int*)P(o.csum);
    c->nmax = std::max(c->nmax, n);
    c->ntile = tmax(c->ntile, tile_sizes(n));
    mu.resize(n);
    tw.resize(n);
    tw4.resize(n);
    for (int k = 0; k < n; ++k) {
      const double sk = std::sin(PI * k / (2.0 * n));
      mu[k] = (float)(4.0 * sk * sk);
      tw4[k] = make_float2((float)std::cos(PI * k / (2.0 * n)), (float)-std::sin(PI * k / (2.0 * n)));
    }
    for (int k = 0; k < n; ++k)
      tw[k] = make_float2((float)std::cos(2 * PI * k / n), (float)-std::sin(2 * PI * k / n));
    // pageable sources are staged before the call returns, so the vectors may be reused
    if (cudaMemcpyAsync(lv.mu, mu.data(), n * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(lv.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(lv.tw4, tw4.data(), n * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return bail(PDG_ERR_CUDA);
    if (!tile_level(n)) launch_sobz_pivots(lv.piv, lv.piv_slow, lv.mu, n, lv.lam, s);
  }
  J.x = (float4*)P(L.x);
  J.y = (float4*)P(L.y);
  J.gfwd = (float4*)P(L.gfwd);
  J.gy = (float4*)P(L.gy);
  J.zq = J.C == 6 ? (float4*)P(L.zq) : nullptr;
  J.uq = J.C == 6 ? (float4*)P(L.uq) : nullptr;
  J.gz = J.C == 6 ? (float4*)P(L.gz) : nullptr;
  J.acc = (long long*)P(L.acc);
  J.loss_fwd = (float*)P(L.loss_fwd);
  J.loss_rev = (float*)P(L.loss_rev);
  J.loss_iso = (float*)P(L.loss_iso);
  J.nn_fwd = (int*)P(L.nn_fwd);
  J.nn_rev = (int*)P(L.nn_rev);
  J.edge_d = (float4*)P(L.edge_d);
  J.edges = (const int2*)P(L.edges);
  J.e_prev = (float*)P(L.e_prev);
  J.v2e_ptr = (const int*)P(L.v2e_ptr);
  J.v2e = (const int*)P(L.v2e);
  J.src4 = (float4*)P(L.src4);
  J.tgt4 = (float4*)P(L.tgt4);
  J.verts4 = (float4*)P(L.verts4);
  auto grid_init = [&](CellGrid& g, int bits, int nsets, size_t hist, size_t off, size_t keys, size_t pts, size_t csum) {
    g.bits = bits;
    g.nsets = nsets;
    const int G = 1 << bits;
    for (int a = 0; a < 3; ++a) {
      g.lo[a] = cfg->lo[a];
      g.inv_h[a] = (float)(G / ((double)cfg->hi[a] - cfg->lo[a]));
      g.h[a] = (float)(((double)cfg->hi[a] - cfg->lo[a]) / G);
    }
    g.hist = (int*)P(hist);
    g.off = (int*)P(off);
    g.keys = (int*)P(keys);
    g.pts = (float4*)P(pts);
    g.csum = (int*)P(csum);
  };
  grid_init(J.tgt, L.tbits, 1, L.t_hist, L.t_off, L.t_keys, L.t_pts, L.t_csum);
  grid_init(J.mov, L.mbits, 2, L.m_hist, L.m_off, L.m_keys, L.m_pts, L.m_csum);
  J.hard = (int4*)P(L.hard);
  J.loss_part = (float*)P(L.loss_part);
  J.hard_count = (int*)P(L.hard_count);
  J.step = (int*)P(L.step);
  J.bias = (float*)P(L.bias);
  J.loss = (double*)P(L.loss);
  J.status = (int*)P(L.status);
  J.gmax = (unsigned*)P(L.gmax);
  J.counters = (unsigned long long*)P(L.counters);

  if (n_edges) {
    if (cudaMemcpyAsync((void*)J.edges, he.data(), he.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync((void*)J.v2e, c->v2e.data(), c->v2e.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return bail(PDG_ERR_CUDA);
  }
  if (cudaMemcpyAsync((void*)J.v2e_ptr, c->v2e_ptr.data(), c->v2e_ptr.size() * 4, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return bail(PDG_ERR_CUDA);
  if (load_points(c, template_xyz, n_verts, J.verts4, s, true) != PDG_OK) {
    const pdg_status st = c->err.find("NaN") != std::string::npos ? PDG_ERR_INVALID : PDG_ERR_CUDA;
    return bail(st);
  }
  if (load_points(c, source_xyz, n_src, J.src4, s, true) != PDG_OK) {
    const pdg_status st = c->err.find("NaN") != std::string::npos ? PDG_ERR_INVALID : PDG_ERR_CUDA;
    return bail(st);
  }
  if (upload_job(c, s) != PDG_OK) return bail(PDG_ERR_CUDA);
  {
    Plan hp;
    std::memset(&hp, 0, sizeof(hp));
    hp.n_jobs = 1;
    hp.jobs[0] = c->dJ;
    if (cudaMemcpyAsync(c->dplan, &hp, sizeof(Plan), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return bail(PDG_ERR_CUDA);
  }
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess)
    return bail(PDG_ERR_CUDA);
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(PDG_ERR_CUDA);
  *out = c;
  return PDG_OK;
}

pdg_status pdg_set_debug(pdg_ctx* c, int flags) {
  if (!c || (flags & ~(PDG_DEBUG_KEEP_PGRAD | PDG_DEBUG_COUNT_NN))) return PDG_ERR_INVALID;
  c->h.keep_pgrad = (flags & PDG_DEBUG_KEEP_PGRAD) ? 1 : 0;
  const int count = (flags & PDG_DEBUG_COUNT_NN) ? 1 : 0;
  if (count != c->h.count_nn && c->gexec) {  // the step graph holds the other NN instances
    if (cudaDeviceSynchronize() != cudaSuccess) return PDG_ERR_CUDA;
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->h.count_nn = count;
  return upload_job(c, 0) == PDG_OK ? c->cuda(cudaDeviceSynchronize(), "set_debug") : PDG_ERR_CUDA;
}

// Recomputes the context's plan prefixes (stream-ordered) if a frame began since the last time.
pdg_status refresh_plan(pdg_ctx* c, cudaStream_t s) {
  if (!c->plan_stale) return PDG_OK;
  launch_plan(c->dplan, s);
  CU(c, cudaGetLastError());
  c->plan_stale = false;
  return PDG_OK;
}

pdg_status pdg_begin_frame(pdg_ctx* c, const float* target_xyz, int n_tgt, void* cuda_stream) {
  if (!c) return PDG_ERR_INVALID;
  if (c->in_frame) return c->fail(PDG_ERR_STATE, "a frame is already open");
  if (!target_xyz || n_tgt < 1) return c->fail(PDG_ERR_INVALID, "empty target");
  if (n_tgt > c->max_pts) return c->fail(PDG_ERR_BUDGET, "target larger than max_pts");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Job& J = c->h;
  TRY(load_points(c, target_xyz, n_tgt, J.tgt4, s, true));
  J.M = n_tgt;
  J.Q = J.V + J.N;
  TRY(upload_job(c, s));
  launch_frame_points(c->dJ, J.Q, J.E, s);
  for (int l = 0; l < J.L; ++l) {
    const Level& lv = J.lev[l];
    if (!c->cfg.warm_start) {
      CU(c, cudaMemsetAsync(lv.theta, 0, sizeof(float4) * lv.n3, s));
      if (lv.theta_t) CU(c, cudaMemsetAsync(lv.theta_t, 0, sizeof(float4) * lv.n3, s));
    }
    CU(c, cudaMemsetAsync(lv.m, 0, sizeof(float) * J.C * lv.n3, s));
    CU(c, cudaMemsetAsync(lv.v, 0, sizeof(float) * J.C * lv.n3, s));
    CU(c, cudaMemsetAsync(lv.g, 0, sizeof(float) * J.C * lv.n3, s));
  }
  CU(c, cudaMemsetAsync(J.step, 0, sizeof(int), s));
  CU(c, cudaMemsetAsync(J.status, 0, sizeof(int), s));
  // no previous neighbours in a new frame (-1: the NN search starts cold)
  CU(c, cudaMemsetAsync(J.nn_fwd, 0xff, sizeof(int) * (size_t)J.Q, s));
  CU(c, cudaMemsetAsync(J.nn_rev, 0xff, sizeof(int) * 2 * (size_t)c->max_pts, s));
  CU(c, cudaMemsetAsync(J.loss, 0, 4 * sizeof(double), s));
  launch_tgt_build(c->dJ, J, s);
  launch_csr_build(c->dJ, J, s);
  CU(c, cudaGetLastError());
  c->in_frame = true;
  c->mesh_valid = false;  // the step overwrites the mesh fit's gradient
  c->steps_in_frame = 0;
  c->plan_stale = true;
  ++c->frame_gen;
  return PDG_OK;
}

pdg_status pdg_step(pdg_ctx* c, int n_steps, void* cuda_stream) {
  if (!c) return PDG_ERR_INVALID;
  if (!c->in_frame) return c->fail(PDG_ERR_STATE, "pdg_step outside a frame");
  if (n_steps < 0) return c->fail(PDG_ERR_INVALID, "negative step count");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (!c->gexec) {
    // the captured launches must not start before this stream's pending set-up
    CU(c, cudaStreamSynchronize(s));
    TRY(capture_step(c, c->dplan, c->nmax, c->ntile, c->cap, c->cap2, &c->gexec, &c->err, c->sms, &c->graph_kernels));
  }
  TRY(refresh_plan(c, s));
  for (int i = 0; i < n_steps; ++i) CU(c, cudaGraphLaunch(c->gexec, s));
  c->steps_in_frame += n_steps;
  return PDG_OK;
}

int pdg_profile_stages(void) { return N_STAGES; }

const char* pdg_profile_stage_name(int i) { return (i >= 0 && i < N_STAGES) ? STAGE_NAMES[i] : ""; }

pdg_status pdg_step_kernel_count(const pdg_ctx* c, int* out) {
  if (!c || !out) return PDG_ERR_INVALID;
  *out = c->gexec ? c->graph_kernels : 0;
  return PDG_OK;
}

pdg_status pdg_profile_step(pdg_ctx* c, int n_steps, double* stage_ms, void* cuda_stream) {
  if (!c || !stage_ms || n_steps < 0) return PDG_ERR_INVALID;
  if (!c->in_frame) return c->fail(PDG_ERR_STATE, "pdg_profile_step outside a frame");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaEvent_t ev[N_STAGES + 1];
  for (auto& e : ev) CU(c, cudaEventCreate(&e));
  for (int i = 0; i < N_STAGES; ++i) stage_ms[i] = 0.0;
  pdg_status st = refresh_plan(c, s);
  for (int k = 0; k < n_steps && st == PDG_OK; ++k) {
    for (int i = 0; i < N_STAGES; ++i) {
      cudaEventRecord(ev[i], s);
      launch_stage(i, c->dplan, c->nmax, c->ntile, c->sms, s, 1, c->h.count_nn != 0);
    }
    cudaEventRecord(ev[N_STAGES], s);
    st = c->cuda(cudaEventSynchronize(ev[N_STAGES]), "profile step");
    for (int i = 0; i < N_STAGES && st == PDG_OK; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      stage_ms[i] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  c->steps_in_frame += n_steps;
  return st;
}

pdg_status pdg_end_frame(pdg_ctx* c, pdg_fit_stats* stats, void* cuda_stream) {
  if (!c) return PDG_ERR_INVALID;
  if (!c->in_frame) return c->fail(PDG_ERR_STATE, "no open frame");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Job& J = c->h;
  launch_end_frame(c->dJ, J.V, s);
  CU(c, cudaMemcpyAsync(J.src4, J.tgt4, sizeof(float4) * J.M, cudaMemcpyDeviceToDevice, s));
  double loss[4];
  int status = 0;
  unsigned long long cnt[4] = {0, 0, 0, 0};
  CU(c, cudaMemcpyAsync(loss, J.loss, sizeof(loss), cudaMemcpyDeviceToHost, s));
  CU(c, cudaMemcpyAsync(&status, J.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(c, cudaMemcpyAsync(cnt, J.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  CU(c, cudaStreamSynchronize(s));
  J.N = J.M;
  J.Q = J.V + J.N;
  c->in_frame = false;
  const pdg_status st = status ? PDG_ERR_NONFINITE : PDG_OK;
  if (stats) {
    stats->loss_total = loss[0];
    stats->cd_mesh = loss[1];
    stats->cd_pts = loss[2];
    stats->iso = loss[3];
    stats->n_steps = c->steps_in_frame;
    stats->status = st;
    stats->nn_ties = !J.count_nn ? -1 : c->steps_in_frame > 0 ? (int)std::min<unsigned long long>(cnt[CNT_NN_TIES], 0x7fffffff) : 0;
  }
  if (st != PDG_OK) c->err = "a loss became NaN or Inf during the frame";
  return st;
}

pdg_status pdg_fit_frame(pdg_ctx* c, const float* target_xyz, int n_tgt, int n_steps, pdg_fit_stats* stats,
                         void* cuda_stream) {
  TRY(pdg_begin_frame(c, target_xyz, n_tgt, cuda_stream));
  const pdg_status st = pdg_step(c, n_steps, cuda_stream);
  if (st != PDG_OK) {
    c->in_frame = false;
    return st;
  }
  return pdg_end_frame(c, stats, cuda_stream);
}

pdg_status pdg_deform(pdg_ctx* c, const float* xyz, int n, float* out, void* cuda_stream) {
  if (!c) return PDG_ERR_INVALID;
  if (n < 0 || (n > 0 && (!xyz || !out))) return c->fail(PDG_ERR_INVALID, "bad deform arguments");
  if (n == 0) return PDG_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool din = is_device_ptr(xyz), dout = is_device_ptr(out);
  if (din && dout) {
    launch_deform(c->dJ, xyz, out, n, s);
    return c->cuda(cudaGetLastError(), "deform");
  }
  // host buffers go through the context's staging area in chunks (no allocation): the first
  // half of the area holds the chunk's input, the second its output
  const int chunk = std::max(1, c->stage_pts / 2);
  float* sin_ = c->stage;
  float* sout = c->stage + 3 * (size_t)chunk;
  for (int b = 0; b < n; b += chunk) {
    const int m = std::min(chunk, n - b);
    const size_t bytes = sizeof(float) * 3 * (size_t)m;
    const float* in = xyz + 3 * (size_t)b;
    float* o = out + 3 * (size_t)b;
    if (!din) {
      CU(c, cudaMemcpyAsync(sin_, in, bytes, cudaMemcpyHostToDevice, s));
      in = sin_;
    }
    launch_deform(c->dJ, in, dout ? o : sout, m, s);
    if (!dout) CU(c, cudaMemcpyAsync(o, sout, bytes, cudaMemcpyDeviceToHost, s));
    // the next chunk overwrites the staging area: wait until this one has left it
    CU(c, cudaStreamSynchronize(s));
  }
  return c->cuda(cudaGetLastError(), "deform");
}

// copies `bytes` from a device buffer to `out` (host or device), synchronising for host
static pdg_status copy_out(pdg_ctx* c, void* out, const void* dsrc, size_t bytes, cudaStream_t s) {
  if (is_device_ptr(out)) {
    CU(c, cudaMemcpyAsync(out, dsrc, bytes, cudaMemcpyDeviceToDevice, s));
  } else {
    CU(c, cudaMemcpyAsync(out, dsrc, bytes, cudaMemcpyDeviceToHost, s));
    CU(c, cudaStreamSynchronize(s));
  }
  return PDG_OK;
}

pdg_status pdg_get_vertices(pdg_ctx* c, float* out, void* cuda_stream) {
  if (!c || !out) return PDG_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bytes = sizeof(float) * 3 * (size_t)c->V;
  if (is_device_ptr(out)) {
    launch_unpack4(c->h.verts4, out, c->V, s);
    return c->cuda(cudaGetLastError(), "get_vertices");
  }
  // through the staging area (it holds max(V, max_pts) points): no allocation
  launch_unpack4(c->h.verts4, c->stage, c->V, s);
  return copy_out(c, out, c->stage, bytes, s);
}

pdg_status pdg_read(pdg_ctx* c, int which, int level, void* out, size_t out_bytes, void* cuda_stream) {
  if (!c || !out) return PDG_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const Job& J = c->h;
  const bool per_level = which == PDG_BUF_THETA || which == PDG_BUF_GRAD || which == PDG_BUF_PGRAD;
  if (per_level && (level < 0 || level >= J.L)) return c->fail(PDG_ERR_INVALID, "bad level");
  size_t need = 0;
  switch (which) {
    case PDG_BUF_THETA:
    case PDG_BUF_GRAD:
    case PDG_BUF_PGRAD: need = sizeof(float) * J.C * (size_t)J.lev[level].n3; break;
    case PDG_BUF_Y:
    case PDG_BUF_POINT_GRAD: need = sizeof(float) * 3 * (size_t)J.Q; break;
    case PDG_BUF_NN_FWD: need = sizeof(int) * (size_t)J.Q; break;
    case PDG_BUF_NN_REV: need = sizeof(int) * 2 * (size_t)J.M; break;
    case PDG_BUF_LOSS: need = 4 * sizeof(double); break;
    case PDG_BUF_SOURCE: need = sizeof(float) * 3 * (size_t)J.N; break;
    case PDG_BUF_COUNTERS: need = 4 * sizeof(unsigned long long); break;
    case PDG_BUF_MESH_GRAD:
    case PDG_BUF_MESH_PGRAD:
      if (!c->mesh_valid) return c->fail(PDG_ERR_STATE, "no template-mesh fit has run");
      need = sizeof(float) * 3 * (size_t)c->V;
      break;
    default: return c->fail(PDG_ERR_INVALID, "unknown buffer");
  }
  if (out_bytes < need) return c->fail(PDG_ERR_INVALID, "output buffer too small");
  if (which == PDG_BUF_PGRAD && !J.keep_pgrad) return c->fail(PDG_ERR_STATE, "call pdg_set_debug(ctx, 1) first");
  if (which == PDG_BUF_LOSS) return copy_out(c, out, J.loss, need, s);
  if (which == PDG_BUF_NN_FWD) return copy_out(c, out, J.nn_fwd, need, s);
  if (which == PDG_BUF_NN_REV) return copy_out(c, out, J.nn_rev, need, s);
  if (which == PDG_BUF_COUNTERS) return copy_out(c, out, J.counters, need, s);
  float* tmp = nullptr;
  CU(c, cudaMallocAsync((void**)&tmp, need, s));
  switch (which) {
    case PDG_BUF_THETA:
      launch_unpack_theta(J.lev[level].theta, J.lev[level].theta_t, tmp, J.lev[level].n3, J.C, s);
      break;
    case PDG_BUF_GRAD: launch_soa_to_aos(J.lev[level].g, tmp, J.lev[level].n3, s, J.C); break;
    case PDG_BUF_PGRAD:  // without the preconditioner Adam takes the raw gradient
      launch_soa_to_aos(J.precondition ? J.lev[level].tmp : J.lev[level].g, tmp, J.lev[level].n3, s, J.C);
      break;
    case PDG_BUF_Y: launch_unpack4(J.y, tmp, J.Q, s); break;
    case PDG_BUF_POINT_GRAD: launch_unpack4(J.gy, tmp, J.Q, s); break;
    case PDG_BUF_SOURCE: launch_unpack4(J.src4, tmp, J.N, s); break;
    case PDG_BUF_MESH_GRAD: launch_unpack4(J.gy, tmp, c->V, s); break;
    case PDG_BUF_MESH_PGRAD: launch_unpack4(c->mesh + 4 * (size_t)c->V, tmp, c->V, s); break;
  }
  const pdg_status st = copy_out(c, out, tmp, need, s);
  cudaFreeAsync(tmp, s);
  return st;
}

pdg_status pdg_write_theta(pdg_ctx* c, int level, const float* theta, void* cuda_stream) {
  if (!c || !theta) return PDG_ERR_INVALID;
  if (level < 0 || level >= c->h.L) return c->fail(PDG_ERR_INVALID, "bad level");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const Level& lv = c->h.lev[level];
  const float* src = theta;
  float* tmp = nullptr;
  const int C = c->h.C;
  const size_t bytes = sizeof(float) * C * (size_t)lv.n3;
  if (!is_device_ptr(theta)) {
    CU(c, cudaMallocAsync((void**)&tmp, bytes, s));
    CU(c, cudaMemcpyAsync(tmp, theta, bytes, cudaMemcpyHostToDevice, s));
    src = tmp;
  }
  launch_pack_theta(src, lv.theta, lv.theta_t, lv.n3, C, s);
  CU(c, cudaMemsetAsync(lv.m, 0, C * sizeof(float) * lv.n3, s));
  CU(c, cudaMemsetAsync(lv.v, 0, C * sizeof(float) * lv.n3, s));
  if (tmp) {
    CU(c, cudaFreeAsync(tmp, s));
    CU(c, cudaStreamSynchronize(s));
  }
  return c->cuda(cudaGetLastError(), "write_theta");
}

pdg_status pdg_eval(pdg_ctx* c, double* loss, void* cuda_stream) {
  if (!c) return PDG_ERR_INVALID;
  if (!c->in_frame) return c->fail(PDG_ERR_STATE, "pdg_eval outside a frame");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  TRY(refresh_plan(c, s));
  for (int i = 0; i < N_STAGES; ++i)  // no preconditioner, no Adam, no step count
    if (i < ST_SOB_FIRST || i > ST_SOB_LAST) launch_stage(i, c->dplan, c->nmax, c->ntile, c->sms, s, 2, c->h.count_nn != 0);
  CU(c, cudaGetLastError());
  if (loss) {
    CU(c, cudaMemcpyAsync(loss, c->h.loss, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(c, cudaStreamSynchronize(s));
  }
  return PDG_OK;
}

pdg_status pdg_precondition(pdg_ctx* c, int level, const float* g, float* out, void* cuda_stream) {
  if (!c || !g || !out) return PDG_ERR_INVALID;
  if (c->in_frame) return c->fail(PDG_ERR_STATE, "pdg_precondition only between frames");
  if (level < 0 || level >= c->h.L) return c->fail(PDG_ERR_INVALID, "bad level");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const Level& lv = c->h.lev[level];
  const size_t bytes = sizeof(float) * 3 * (size_t)lv.n3;
  float* tmp = nullptr;
  CU(c, cudaMallocAsync((void**)&tmp, bytes, s));
  CU(c, cudaMemcpyAsync(tmp, g, bytes, is_device_ptr(g) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  launch_aos_to_soa(tmp, lv.g, lv.n3, s);
  // a one-level copy of the job that stores the preconditioned gradient instead of Adam
  Job oj = c->h;
  oj.L = 1;
  oj.C = 3;  // the entry point preconditions 3 channels whatever the payload
  oj.lev[0] = lv;
  oj.lev[0].zmask = nullptr;  // a caller's gradient may be non-zero on any plane
  oj.precondition = 1;
  oj.keep_pgrad = 1;
  oj.no_adam = 1;
  Plan op;
  std::memset(&op, 0, sizeof(op));
  op.n_jobs = 1;
  op.jobs[0] = c->op_job;
  CU(c, cudaMemcpyAsync(c->op_job, &oj, sizeof(Job), cudaMemcpyHostToDevice, s));
  CU(c, cudaMemcpyAsync(c->op_plan, &op, sizeof(Plan), cudaMemcpyHostToDevice, s));
  launch_plan(c->op_plan, s);
  for (int i = ST_SOB_FIRST; i <= ST_SOB_LAST; ++i) launch_stage(i, c->op_plan, lv.n, tile_sizes(lv.n), c->sms, s);
  launch_soa_to_aos(lv.tmp, tmp, lv.n3, s);
  CU(c, cudaGetLastError());
  const pdg_status st = copy_out(c, out, tmp, bytes, s);
  cudaFreeAsync(tmp, s);
  CU(c, cudaMemsetAsync(lv.g, 0, bytes, s));
  CU(c, cudaStreamSynchronize(s));
  return st;
}

// ------------------------------------------------------------------------------ template-mesh fit

pdg_status pdg_fit_mesh(pdg_ctx* c, const float* p0_xyz, int n_p0, int n_steps, float lambda, float lr,
                        pdg_fit_stats* stats, void* cuda_stream) {
  if (!c) return PDG_ERR_INVALID;
  if (c->in_frame) return c->fail(PDG_ERR_STATE, "pdg_fit_mesh only between frames");
  if (!p0_xyz || n_p0 < 1 || n_steps < 0 || !(lambda >= 0.f) || !(lambda < 1e30f) || !(lr >= 0.f) || !(lr < 1e30f))
    return c->fail(PDG_ERR_INVALID, "bad mesh-fit arguments");
  if (n_p0 > c->max_pts) return c->fail(PDG_ERR_BUDGET, "cloud larger than max_pts");
  // bounds the Chebyshev iteration count below (about 5000 per solve at the limit)
  if ((double)lambda * std::max(c->max_degree, 1) > 1e5)
    return c->fail(PDG_ERR_INVALID, "lambda times the largest vertex degree above 1e5");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Job& J = c->h;
  const int V = c->V;
  TRY(load_points(c, p0_xyz, n_p0, J.tgt4, s, true));
  // the step's kernels on a job whose query points are the mesh vertices alone: no source set,
  // no isometry, the mesh term with weight 1; 3 channels (the grids take no part)
  Job mj = J;
  mj.N = 0;
  mj.Q = V;
  mj.M = n_p0;
  mj.E = 0;
  mj.C = 3;
  mj.w_mesh = 1.f;
  mj.w_pts = 0.f;
  mj.w_iso = 0.f;
  mj.count_nn = 0;
  CU(c, cudaMemcpyAsync(c->op_job, &mj, sizeof(Job), cudaMemcpyHostToDevice, s));
  Plan op;
  std::memset(&op, 0, sizeof(op));
  op.n_jobs = 1;
  op.jobs[0] = c->op_job;
  CU(c, cudaMemcpyAsync(c->op_plan, &op, sizeof(Plan), cudaMemcpyHostToDevice, s));
  launch_plan(c->op_plan, s);
  float4* h = c->mesh;
  float4* r = h + V;
  float4* d0 = r + V;
  float4* d1 = d0 + V;
  float4* pg = d1 + V;
  float4* am = pg + V;
  float4* av = am + V;
  CU(c, cudaMemcpyAsync(J.x, J.verts4, sizeof(float4) * V, cudaMemcpyDeviceToDevice, s));  // X_0 being fitted
  CU(c, cudaMemsetAsync(am, 0, 2 * sizeof(float4) * (size_t)V, s));
  CU(c, cudaMemsetAsync(J.nn_fwd, 0xff, sizeof(int) * (size_t)V, s));
  CU(c, cudaMemsetAsync(J.nn_rev, 0xff, sizeof(int) * (size_t)n_p0, s));
  CU(c, cudaMemsetAsync(J.loss, 0, 4 * sizeof(double), s));
  CU(c, cudaMemsetAsync(J.status, 0, sizeof(int), s));
  launch_tgt_build(c->op_job, mj, s);
  // Chebyshev interval: the Laplacian's eigenvalues lie in [0, 2 max degree] (Gershgorin), so
  // those of I + lambda L in [1, emax]; iterations for a relative error below 1e-7 in exact
  // arithmetic, 2 sqrt(kappa) q^k <= 1e-7 with q = (sqrt(kappa) - 1) / (sqrt(kappa) + 1)
  const double emax = 1.0 + 2.0 * lambda * std::max(c->max_degree, 1);
  const double sk = std::sqrt(emax);
  const double q = (sk - 1.0) / (sk + 1.0);
  const int iters = q > 0.0 ? (int)std::ceil(std::log(1e-7 / (2.0 * sk)) / std::log(q)) : 1;
  const int2* edges = J.edges;
  for (int k = 1; k <= n_steps; ++k) {
    launch_mesh_points(c->op_job, V, s);
    for (int i = S_MOV_SCAN; i <= S_NN_HARD; ++i) launch_stage(i, c->op_plan, 1, TileSizes(), c->sms, s);
    launch_stage(S_ASSEMBLE, c->op_plan, 1, TileSizes(), c->sms, s);
    launch_stage(S_LOSS, c->op_plan, 1, TileSizes(), c->sms, s);
    // (I + lambda L)^{-2} dL/dX by two solves, then Adam on the vertices
    launch_mesh_solve(J.v2e_ptr, J.v2e, edges, J.gy, h, r, d0, d1, V, lambda, (float)emax, iters, s);
    launch_mesh_solve(J.v2e_ptr, J.v2e, edges, h, pg, r, d0, d1, V, lambda, (float)emax, iters, s);
    const float bias1 = (float)(1.0 / (1.0 - std::pow((double)J.beta1, k)));
    const float ibias2 = (float)(1.0 / std::sqrt(1.0 - std::pow((double)J.beta2, k)));
    launch_mesh_adam(J.x, pg, am, av, V, lr, J.beta1, J.beta2, J.eps, bias1, ibias2, s);
    CU(c, cudaGetLastError());
  }
  CU(c, cudaMemcpyAsync(J.verts4, J.x, sizeof(float4) * V, cudaMemcpyDeviceToDevice, s));
  double loss[4];
  int status = 0;
  CU(c, cudaMemcpyAsync(loss, J.loss, sizeof(loss), cudaMemcpyDeviceToHost, s));
  CU(c, cudaMemcpyAsync(&status, J.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(c, cudaStreamSynchronize(s));
  c->mesh_valid = n_steps > 0;
  c->plan_stale = true;  // the frame plan is recomputed at the next frame
  const pdg_status st = status ? PDG_ERR_NONFINITE : PDG_OK;
  if (stats) {
    stats->loss_total = loss[0];
    stats->cd_mesh = loss[1];
    stats->cd_pts = 0.0;
    stats->iso = 0.0;
    stats->n_steps = n_steps;
    stats->status = st;
    stats->nn_ties = -1;
  }
  if (st != PDG_OK) c->err = "a loss became NaN or Inf during the mesh fit";
  return st;
}

// ------------------------------------------------------------------------------ batching

void pdg_debug_fail_allocations(int n) { g_fail_allocs.store(n > 0 ? n : 0); }

pdg_status pdg_batch_create(int max_jobs, pdg_batch** out) {
  if (!out || max_jobs < 1 || max_jobs > MAXJ) return PDG_ERR_INVALID;
  pdg_batch* b = new pdg_batch();
  b->max_jobs = max_jobs;
  if (dev_malloc((void**)&b->dplan, sizeof(Plan)) != cudaSuccess || cudaMallocHost(&b->hplan, sizeof(Plan)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    pdg_batch_destroy(b);
    return PDG_ERR_OOM;
  }
  std::memset(b->hplan, 0, sizeof(Plan));
  *out = b;
  return PDG_OK;
}

void pdg_batch_destroy(pdg_batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
  if (b->dplan) cudaFree(b->dplan);
  if (b->hplan) cudaFreeHost(b->hplan);
  delete b;
}

pdg_status pdg_batch_set(pdg_batch* b, pdg_ctx* const* ctxs, int n_jobs) {
  if (!b || n_jobs < 0 || n_jobs > b->max_jobs || (n_jobs && !ctxs)) return PDG_ERR_INVALID;
  for (int i = 0; i < n_jobs; ++i) {
    if (!ctxs[i]) return PDG_ERR_INVALID;
    if (!ctxs[i]->in_frame) {
      b->err = "batch member outside a frame";
      return PDG_ERR_STATE;
    }
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return PDG_ERR_INVALID;
  }
  b->members.assign(ctxs, ctxs + n_jobs);
  b->n = n_jobs;
  b->dirty = true;
  return PDG_OK;
}

pdg_status pdg_batch_step(pdg_batch* b, int n_steps, void* cuda_stream) {
  if (!b || n_steps < 0) return PDG_ERR_INVALID;
  if (b->n == 0 || n_steps == 0) return PDG_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int nmax = 1, sms = 1;
  TileSizes ntile;
  for (auto* c : b->members) {
    if (!c->in_frame) {
      b->err = "batch member outside a frame";
      return PDG_ERR_STATE;
    }
    nmax = std::max(nmax, c->nmax);
    ntile = tmax(ntile, c->ntile);
    sms = c->sms;
  }
  if (b->dirty) {
    // publish the membership (stream-ordered; the pinned host copy is rewritten only after
    // the previous upload completed)
    if (cudaStreamSynchronize(s) != cudaSuccess) return PDG_ERR_CUDA;
    std::memset(b->hplan, 0, sizeof(Plan));
    b->hplan->n_jobs = b->n;
    for (int i = 0; i < b->n; ++i) b->hplan->jobs[i] = b->members[i]->dJ;
    if (cudaMemcpyAsync(b->dplan, b->hplan, sizeof(Plan), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PDG_ERR_CUDA;
    b->dirty = false;
    b->gens.clear();
  }
  // item prefixes: recomputed when the membership changed or a member began a frame
  bool stale = b->gens.size() != b->members.size();
  for (size_t i = 0; i < b->members.size() && !stale; ++i) stale = b->gens[i] != b->members[i]->frame_gen;
  if (stale) {
    launch_plan(b->dplan, s);
    if (cudaGetLastError() != cudaSuccess) return PDG_ERR_CUDA;
    b->gens.resize(b->members.size());
    for (size_t i = 0; i < b->members.size(); ++i) b->gens[i] = b->members[i]->frame_gen;
  }
  if (!b->gexec || nmax > b->graph_nmax || tgreater(ntile, b->graph_ntile)) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PDG_ERR_CUDA;
    const pdg_status st = capture_step(nullptr, b->dplan, std::max(nmax, b->graph_nmax), tmax(ntile, b->graph_ntile), b->cap, b->cap2, &b->gexec, &b->err, sms);
    if (st != PDG_OK) return st;
    b->graph_nmax = std::max(nmax, b->graph_nmax);
    b->graph_ntile = tmax(ntile, b->graph_ntile);
  }
  for (int i = 0; i < n_steps; ++i)
    if (cudaGraphLaunch(b->gexec, s) != cudaSuccess) return PDG_ERR_CUDA;
  for (auto* c : b->members) c->steps_in_frame += n_steps;
  return PDG_OK;
}

// ------------------------------------------------------------------------------ state

namespace {
struct StateHeader {
  char magic[8];
  int version, V, N, L, res[PDG_MAX_LEVELS], C;
};
}  // namespace

size_t pdg_state_bytes(const pdg_ctx* c) {
  if (!c) return 0;
  size_t b = sizeof(StateHeader) + sizeof(float4) * (size_t)c->V + sizeof(float4) * (size_t)c->max_pts;
  for (int l = 0; l < c->h.L; ++l) b += sizeof(float4) * (size_t)c->h.lev[l].n3 * (c->h.C / 3);
  return b;
}

pdg_status pdg_save_state(pdg_ctx* c, void* host_buf, size_t n, void* cuda_stream) {
  if (!c || !host_buf) return PDG_ERR_INVALID;
  if (c->in_frame) return c->fail(PDG_ERR_STATE, "save only between frames");
  if (n < pdg_state_bytes(c)) return c->fail(PDG_ERR_INVALID, "state buffer too small");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  StateHeader hd{};
  std::memcpy(hd.magic, "PDGSTAT", 8);
  hd.version = 2;
  hd.V = c->V;
  hd.C = c->h.C;
  hd.N = c->h.N;
  hd.L = c->h.L;
  for (int l = 0; l < c->h.L; ++l) hd.res[l] = c->h.lev[l].n;
  char* p = (char*)host_buf;
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  CU(c, cudaMemcpyAsync(p, c->h.verts4, sizeof(float4) * c->V, cudaMemcpyDeviceToHost, s));
  p += sizeof(float4) * c->V;
  CU(c, cudaMemcpyAsync(p, c->h.src4, sizeof(float4) * c->max_pts, cudaMemcpyDeviceToHost, s));
  p += sizeof(float4) * c->max_pts;
  for (int l = 0; l < c->h.L; ++l) {
    CU(c, cudaMemcpyAsync(p, c->h.lev[l].theta, sizeof(float4) * c->h.lev[l].n3, cudaMemcpyDeviceToHost, s));
    p += sizeof(float4) * c->h.lev[l].n3;
    if (c->h.C == 6) {
      CU(c, cudaMemcpyAsync(p, c->h.lev[l].theta_t, sizeof(float4) * c->h.lev[l].n3, cudaMemcpyDeviceToHost, s));
      p += sizeof(float4) * c->h.lev[l].n3;
    }
  }
  CU(c, cudaStreamSynchronize(s));
  return PDG_OK;
}

pdg_status pdg_load_state(pdg_ctx* c, const void* host_buf, size_t n, void* cuda_stream) {
  if (!c || !host_buf) return PDG_ERR_INVALID;
  if (c->in_frame) return c->fail(PDG_ERR_STATE, "load only between frames");
  if (n < pdg_state_bytes(c)) return c->fail(PDG_ERR_INVALID, "state buffer too small");
  StateHeader hd;
  std::memcpy(&hd, host_buf, sizeof(hd));
  if (std::memcmp(hd.magic, "PDGSTAT", 8) != 0 || hd.version != 2 || hd.V != c->V || hd.L != c->h.L || hd.C != c->h.C ||
      hd.N < 1 || hd.N > c->max_pts)
    return c->fail(PDG_ERR_INVALID, "state does not match this context");
  for (int l = 0; l < c->h.L; ++l)
    if (hd.res[l] != c->h.lev[l].n) return c->fail(PDG_ERR_INVALID, "state does not match this context");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const char* p = (const char*)host_buf + sizeof(hd);
  CU(c, cudaMemcpyAsync(c->h.verts4, p, sizeof(float4) * c->V, cudaMemcpyHostToDevice, s));
  p += sizeof(float4) * c->V;
  CU(c, cudaMemcpyAsync(c->h.src4, p, sizeof(float4) * c->max_pts, cudaMemcpyHostToDevice, s));
  p += sizeof(float4) * c->max_pts;
  for (int l = 0; l < c->h.L; ++l) {
    CU(c, cudaMemcpyAsync(c->h.lev[l].theta, p, sizeof(float4) * c->h.lev[l].n3, cudaMemcpyHostToDevice, s));
    p += sizeof(float4) * c->h.lev[l].n3;
    if (c->h.C == 6) {
      CU(c, cudaMemcpyAsync(c->h.lev[l].theta_t, p, sizeof(float4) * c->h.lev[l].n3, cudaMemcpyHostToDevice, s));
      p += sizeof(float4) * c->h.lev[l].n3;
    }
  }
  c->h.N = hd.N;
  c->h.Q = c->V + hd.N;
  TRY(upload_job(c, s));
  CU(c, cudaStreamSynchronize(s));
  return PDG_OK;
}

}  // extern "C"
