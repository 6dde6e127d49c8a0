// A variant of the grid Sobolev preconditioner entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need the
// preconditioner: code running under a strict device-memory budget that was fixed up front,
// hosts whose allocator must not be re-entered from the calling thread, and pipelines that
// forbid allocation on their hot path to keep latency predictable.  pdg_precondition needs
// a context (its arena) and a temporary buffer; this entry point instead keeps all of its
// scratch in one file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace pdg {

constexpr int STATIC_MAX_RES = PDG_STATIC_MAX_RES;
constexpr size_t STATIC_N3 = (size_t)STATIC_MAX_RES * STATIC_MAX_RES * STATIC_MAX_RES;
// layout: g (SoA, 3 n^3 floats) | tmp (3 n^3) | z-solve pivots ((n/2 + 1) n^2) | mu (n) | tw (n float2) | tw4 (n float2) |
//         n_active (int) + bias (2 floats, read by the pass even when it skips Adam) | pivot flag | job | plan
constexpr size_t SO_G = 0;
constexpr size_t SO_TMP = SO_G + 3 * STATIC_N3 * sizeof(float);
constexpr size_t SO_PIV = SO_TMP + 3 * STATIC_N3 * sizeof(float);
constexpr size_t SO_MU =
    SO_PIV + (size_t)(STATIC_MAX_RES / 2 + 1) * STATIC_MAX_RES * STATIC_MAX_RES * sizeof(float);
constexpr size_t SO_TW = SO_MU + STATIC_MAX_RES * sizeof(float);
constexpr size_t SO_TW4 = SO_TW + STATIC_MAX_RES * sizeof(float2);
constexpr size_t SO_NA = SO_TW4 + STATIC_MAX_RES * sizeof(float2);
constexpr size_t SO_SLOW = SO_NA + 4 * sizeof(int);  // after n_active and the two bias floats
constexpr size_t SO_BIAS = SO_NA + sizeof(int);
constexpr size_t SO_JOB = (SO_SLOW + sizeof(int) + 255) & ~size_t(255);
constexpr size_t SO_PLAN = (SO_JOB + sizeof(Job) + 255) & ~size_t(255);
constexpr size_t SO_BYTES = (SO_PLAN + sizeof(Plan) + 255) & ~size_t(255);

static __device__ __align__(256) unsigned char g_static_scratch[SO_BYTES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (the symbol name itself is
// only a host-side stand-in).  Looked up once per device.
unsigned char* scratch_address(pdg_status* st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    *st = PDG_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      *st = PDG_ERR_CUDA;
      return nullptr;
    }
    sobolev_plane_configure();
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *st = PDG_OK;
  return g_scratch_addr[dev];
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

}  // namespace pdg

using namespace pdg;

extern "C" pdg_status pdg_precondition_static(int res, float lambda, const float* g, float* out,
                                              void* cuda_stream) {
  if (!g || !out || !(lambda >= 0.f) || !(lambda < 3.0e38f)) return PDG_ERR_INVALID;
  if (res < 1 || (res & (res - 1)) != 0) return PDG_ERR_INVALID;
  if (res > STATIC_MAX_RES) return PDG_ERR_BUDGET;
  if (!on_device(g) || !on_device(out)) return PDG_ERR_INVALID;
  pdg_status st = PDG_OK;
  unsigned char* base = scratch_address(&st);
  if (st != PDG_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int n = res;
  const int n3 = n * n * n;
  // one-level job that stops at the preconditioned gradient (Adam is skipped)
  Job J;
  std::memset(&J, 0, sizeof(J));
  J.L = 1;
  J.precondition = 1;
  J.keep_pgrad = 1;
  J.no_adam = 1;
  Level& lv = J.lev[0];
  lv.n = n;
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  lv.lg = lg;
  lv.n3 = n3;
  lv.tiles = (n * n + TILE_LINES - 1) / TILE_LINES;
  lv.lam = lambda;
  lv.g = reinterpret_cast<float*>(base + SO_G);
  lv.tmp = reinterpret_cast<float*>(base + SO_TMP);
  lv.piv = reinterpret_cast<float*>(base + SO_PIV);
  lv.piv_slow = reinterpret_cast<int*>(base + SO_SLOW);
  lv.mu = reinterpret_cast<float*>(base + SO_MU);
  lv.tw = reinterpret_cast<float2*>(base + SO_TW);
  lv.tw4 = reinterpret_cast<float2*>(base + SO_TW4);
  lv.n_active = reinterpret_cast<int*>(base + SO_NA);
  J.bias = reinterpret_cast<float*>(base + SO_BIAS);
  Plan P;
  std::memset(&P, 0, sizeof(P));
  P.n_jobs = 1;
  P.jobs[0] = reinterpret_cast<Job*>(base + SO_JOB);
  // tables and structs in one host block (pageable copies are staged before the call returns)
  struct Tables {
    float mu[STATIC_MAX_RES];
    float2 tw[STATIC_MAX_RES];
    float2 tw4[STATIC_MAX_RES];
    int n_active;
    float bias[2];
  } T;
  const double PI = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double sk = std::sin(PI * k / (2.0 * n));
    T.mu[k] = (float)(4.0 * sk * sk);
    T.tw[k] = make_float2((float)std::cos(2 * PI * k / n), (float)-std::sin(2 * PI * k / n));
    T.tw4[k] = make_float2((float)std::cos(PI * k / (2.0 * n)), (float)-std::sin(PI * k / (2.0 * n)));
  }
  T.n_active = 0;
  T.bias[0] = T.bias[1] = 1.f;
  if (cudaMemcpyAsync(lv.mu, T.mu, sizeof(float) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(lv.tw, T.tw, sizeof(float2) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(lv.tw4, T.tw4, sizeof(float2) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(lv.n_active, &T.n_active, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(J.bias, T.bias, 2 * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(P.jobs[0], &J, sizeof(Job), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + SO_PLAN, &P, sizeof(Plan), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PDG_ERR_CUDA;
  launch_sobz_pivots(lv.piv, lv.piv_slow, lv.mu, n, lambda, s);
  const Plan* dP = reinterpret_cast<const Plan*>(base + SO_PLAN);
  launch_aos_to_soa(g, lv.g, n3, s);
  launch_plan(const_cast<Plan*>(dP), s);
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = (227 * 1024) / plane_smem_max(n) < 8 ? (227 * 1024) / plane_smem_max(n) : 8;
  launch_sobolev_plane(dP, sms * (per_sm > 0 ? per_sm : 1), n, s);
  launch_soa_to_aos(lv.tmp, out, n3, s);
  return cudaGetLastError() == cudaSuccess ? PDG_OK : PDG_ERR_CUDA;
}
