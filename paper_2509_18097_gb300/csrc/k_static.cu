// A variant of the grid Sobolev preconditioner entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need the
// preconditioner: code running under a strict device-memory budget that was fixed up front,
// hosts whose allocator must not be re-entered from the calling thread, and pipelines that
// forbid allocation on their hot path to keep latency predictable.  pdg_precondition needs
// a context (its arena) and a temporary buffer; this entry point instead keeps all of its
// scratch in one file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
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

// Device memory (or managed memory) of the current device: a pointer into another GPU's
// memory would need peer access, which this entry point does not set up.
bool on_current_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && (a.type == cudaMemoryTypeManaged || a.device == dev);
}
}  // namespace

// Writes the level's tables (path-Laplacian eigenvalues, FFT and DCT twiddles), the
// one-level job that stops at the preconditioned gradient, and its plan into the scratch
// array.  Everything comes in as kernel arguments, so the call copies nothing from host
// memory.  One block.
__global__ void k_static_setup(unsigned char* base, int n, int lg, float lam) {
  float* mu = reinterpret_cast<float*>(base + SO_MU);
  float2* tw = reinterpret_cast<float2*>(base + SO_TW);
  float2* tw4 = reinterpret_cast<float2*>(base + SO_TW4);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double sh, ch, s2, c2;
    sincospi((double)k / (2.0 * n), &sh, &ch);  // angle pi k / 2n
    sincospi(2.0 * k / n, &s2, &c2);            // angle 2 pi k / n
    mu[k] = (float)(4.0 * sh * sh);
    tw[k] = make_float2((float)c2, (float)-s2);
    tw4[k] = make_float2((float)ch, (float)-sh);
  }
  // zero the job and plan records word by word, then fill the fields that matter
  unsigned* jw = reinterpret_cast<unsigned*>(base + SO_JOB);
  for (size_t i = threadIdx.x; i < sizeof(Job) / 4; i += blockDim.x) jw[i] = 0u;
  unsigned* pw = reinterpret_cast<unsigned*>(base + SO_PLAN);
  for (size_t i = threadIdx.x; i < sizeof(Plan) / 4; i += blockDim.x) pw[i] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    Job& J = *reinterpret_cast<Job*>(base + SO_JOB);
    J.L = 1;
    J.C = 3;
    J.precondition = 1;
    J.keep_pgrad = 1;
    J.no_adam = 1;
    Level& lv = J.lev[0];
    lv.n = n;
    lv.lg = lg;
    lv.n3 = n * n * n;
    lv.tiles = 3 * ((n * n + TILE_LINES - 1) / TILE_LINES);  // one channel per tile
    lv.lam = lam;
    lv.g = reinterpret_cast<float*>(base + SO_G);
    lv.tmp = reinterpret_cast<float*>(base + SO_TMP);
    lv.piv = reinterpret_cast<float*>(base + SO_PIV);
    lv.piv_slow = reinterpret_cast<int*>(base + SO_SLOW);
    lv.mu = mu;
    lv.tw = tw;
    lv.tw4 = tw4;
    lv.n_active = reinterpret_cast<int*>(base + SO_NA);
    *lv.n_active = 0;
    J.bias = reinterpret_cast<float*>(base + SO_BIAS);
    J.bias[0] = J.bias[1] = 1.f;
    Plan& P = *reinterpret_cast<Plan*>(base + SO_PLAN);
    P.n_jobs = 1;
    P.jobs[0] = &J;
  }
}

}  // namespace pdg

using namespace pdg;

extern "C" pdg_status pdg_precondition_static(int res, float lambda, const float* g, float* out,
                                              void* cuda_stream) {
  if (!g || !out || !(lambda >= 0.f) || !(lambda < 3.0e38f)) return PDG_ERR_INVALID;
  if (res < 1 || (res & (res - 1)) != 0) return PDG_ERR_INVALID;
  if (res > STATIC_MAX_RES) return PDG_ERR_BUDGET;
  if (!on_current_device(g) || !on_current_device(out)) return PDG_ERR_INVALID;
  // a launch error left behind by earlier, unrelated work would otherwise be reported as
  // this call's
  cudaGetLastError();
  pdg_status st = PDG_OK;
  unsigned char* base = scratch_address(&st);
  if (st != PDG_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int n = res;
  const int n3 = n * n * n;
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  k_static_setup<<<1, 256, 0, s>>>(base, n, lg, lambda);
  float* lv_g = reinterpret_cast<float*>(base + SO_G);
  float* lv_tmp = reinterpret_cast<float*>(base + SO_TMP);
  launch_sobz_pivots(reinterpret_cast<float*>(base + SO_PIV), reinterpret_cast<int*>(base + SO_SLOW),
                     reinterpret_cast<const float*>(base + SO_MU), n, lambda, s);
  Plan* dP = reinterpret_cast<Plan*>(base + SO_PLAN);
  launch_aos_to_soa(g, lv_g, n3, s);
  launch_plan(dP, s);
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = (227 * 1024) / plane_smem_max(n) < 8 ? (227 * 1024) / plane_smem_max(n) : 8;
  launch_sobolev_plane(dP, sms * (per_sm > 0 ? per_sm : 1), n, s);
  launch_soa_to_aos(lv_tmp, out, n3, s);
  return cudaGetLastError() == cudaSuccess ? PDG_OK : PDG_ERR_CUDA;
}

