// Template-mesh fit (Sec. 3.4, surface initialisation loss L_mesh = CD_R(X_0, P_0); Sec. 3.6,
// lambda = 16, lr = 1e-4): the kernels of one iteration that the frame step does not have.
// The robust Chamfer search and gradient are the step's own kernels, run on a job record
// whose query points are the mesh vertices alone (no source set, no isometry term).  The
// vertex gradient is then preconditioned by (I + lambda L)^{-2}, L the combinatorial graph
// Laplacian of the mesh edges, by two Chebyshev solves (no inner products, one kernel per
// iteration), and Adam moves the vertices.
#include "kernels.h"

namespace pdg {

// y = x for the mesh vertices (the query points of the fit), their moving-grid keys and
// counts, cleared reverse-Chamfer accumulators; the first thread clears the step's counters.
__global__ void k_mesh_points(Job* __restrict__ Jp) {
  const Job& J = *Jp;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *J.hard_count = 0;
    *J.gmax = 0u;
    J.counters[CNT_NN_CANDIDATES] = 0ull;
    J.counters[CNT_NN_TIES] = 0ull;
    J.counters[CNT_NN_HARD] = 0ull;
  }
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J.V; p += gridDim.x * blockDim.x) {
    const float4 x = J.x[p];
    J.y[p] = make_float4(x.x, x.y, x.z, 0.f);
    const int key = cell_key(J.mov, x.x, x.y, x.z, 0);
    J.mov.keys[p] = key;
    atomicAdd(&J.mov.hist[key], 1);
    J.acc[3 * p + 0] = 0;
    J.acc[3 * p + 1] = 0;
    J.acc[3 * p + 2] = 0;
  }
}

// Chebyshev iteration for A h = b, A = I + lambda L (symmetric, eigenvalues in [1, emax]),
// as the three-term recurrence: h_{k+1} = h_k + d_k, r_{k+1} = r_k - A d_k,
// d_{k+1} = c1 d_k + c2 r_{k+1}, started from h_0 = 0, r_0 = b, d_0 = b / theta.
// Set-up of the recurrence.
__global__ void k_cheb_init(const float4* __restrict__ b, float4* __restrict__ h, float4* __restrict__ r,
                            float4* __restrict__ d, int V, float inv_theta) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const float4 v = b[i];
    h[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    r[i] = make_float4(v.x, v.y, v.z, 0.f);
    d[i] = make_float4(v.x * inv_theta, v.y * inv_theta, v.z * inv_theta, 0.f);
  }
}

// One iteration: (A d)_i = d_i + lambda sum_{j ~ i} (d_i - d_j) over the vertex's edges (the
// vertex -> edge lists of the context, the other end from the edge record); d is read from
// `din` (complete from the previous launch) and the next d written to `dout`.
__global__ void k_cheb_iter(const int* __restrict__ v2e_ptr, const int* __restrict__ v2e, const int2* __restrict__ edges,
                            const float4* __restrict__ din, float4* __restrict__ dout, float4* __restrict__ h,
                            float4* __restrict__ r, int V, float lam, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const float4 di = din[i];
    float lx = 0.f, ly = 0.f, lz = 0.f;
    for (int k = __ldg(v2e_ptr + i); k < __ldg(v2e_ptr + i + 1); ++k) {
      const int ent = __ldg(v2e + k);
      const int2 e = __ldg(edges + (ent >> 1));
      const float4 dj = din[(ent & 1) ? e.x : e.y];
      lx += di.x - dj.x;
      ly += di.y - dj.y;
      lz += di.z - dj.z;
    }
    const float ax = di.x + lam * lx, ay = di.y + lam * ly, az = di.z + lam * lz;
    float4 hi = h[i], ri = r[i];
    hi.x += di.x; hi.y += di.y; hi.z += di.z;
    ri.x -= ax; ri.y -= ay; ri.z -= az;
    h[i] = hi;
    r[i] = ri;
    dout[i] = make_float4(c1 * di.x + c2 * ri.x, c1 * di.y + c2 * ri.y, c1 * di.z + c2 * ri.z, 0.f);
  }
}

// Adam (PyTorch semantics) on the mesh vertices with the preconditioned gradient g;
// bias1 = 1 / (1 - beta1^k), ibias2 = 1 / sqrt(1 - beta2^k)
__global__ void k_mesh_adam(float4* __restrict__ x, const float4* __restrict__ g, float4* __restrict__ m,
                            float4* __restrict__ v, int V, float lr, float b1, float b2, float eps, float bias1,
                            float ibias2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const float4 gi = g[i];
    float4 mi = m[i], vi = v[i], xi = x[i];
    const float gg[3] = {gi.x, gi.y, gi.z};
    float* mm = &mi.x;
    float* vv = &vi.x;
    float* xx = &xi.x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mm[c] = b1 * mm[c] + (1.f - b1) * gg[c];
      vv[c] = b2 * vv[c] + (1.f - b2) * gg[c] * gg[c];
      xx[c] -= lr * bias1 * mm[c] / (sqrtf(vv[c]) * ibias2 + eps);
    }
    m[i] = mi;
    v[i] = vi;
    x[i] = xi;
  }
}

static inline int mesh_blocks(int n) { return max(1, min((n + 255) / 256, 4096)); }

void launch_mesh_points(Job* J, int V, cudaStream_t s) { k_mesh_points<<<mesh_blocks(V), 256, 0, s>>>(J); }

void launch_mesh_solve(const int* v2e_ptr, const int* v2e, const int2* edges, const float4* b, float4* h, float4* r,
                       float4* d0, float4* d1, int V, float lam, float emax, int iters, cudaStream_t s) {
  // Chebyshev constants for the interval [1, emax] (theta its centre, delta its half-width)
  const double theta = 0.5 * (emax + 1.0), delta = 0.5 * (emax - 1.0);
  const int nb = mesh_blocks(V);
  k_cheb_init<<<nb, 256, 0, s>>>(b, h, r, d0, V, (float)(1.0 / theta));
  if (delta <= 0.0) {  // lambda = 0: A = I, the set-up already holds h + d = b after one update
    k_cheb_iter<<<nb, 256, 0, s>>>(v2e_ptr, v2e, edges, d0, d1, h, r, V, 0.f, 0.f, 0.f);
    return;
  }
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  float4* din = d0;
  float4* dout = d1;
  for (int k = 0; k < iters; ++k) {
    const double rho_n = 1.0 / (2.0 * sigma - rho);
    k_cheb_iter<<<nb, 256, 0, s>>>(v2e_ptr, v2e, edges, din, dout, h, r, V, lam, (float)(rho_n * rho),
                                   (float)(2.0 * rho_n / delta));
    rho = rho_n;
    float4* t = din;
    din = dout;
    dout = t;
  }
}

void launch_mesh_adam(float4* x, const float4* g, float4* m, float4* v, int V, float lr, float b1, float b2, float eps,
                      float bias1, float ibias2, cudaStream_t s) {
  k_mesh_adam<<<mesh_blocks(V), 256, 0, s>>>(x, g, m, v, V, lr, b1, b2, eps, bias1, ibias2);
}

}  // namespace pdg
