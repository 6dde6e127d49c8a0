// Adjoint of the multi-level trilinear evaluation (chain rule of Eq. 1):
//   dLoss/dTheta_l[v] = (1/L) sum_{p : v is a corner of p in level l} w_{l,v}(x_p) dLoss/dy_p.
// The query points x are fixed for a whole frame, so the per-level point -> vertex lists
// (point id, weight / L) are built once per frame by a counting sort keyed by vertex, and
// compacted to the vertices that some point touches.  Each step then gathers every active
// vertex's row.  A row is summed in 64-bit fixed point with a scale chosen from the step's
// bound on |dLoss/dy| (taken in the assembly kernel): integer addition is associative, so
// the result does not depend on
// the (atomic, unordered) order in which the lists were filled, nor on how the row is split
// across lanes.  No floating-point atomics are used.
#include "kernels.h"

namespace pdg {

// corners of point p in level lv: flat vertex ids and trilinear weights (Eq. 1)
__device__ __forceinline__ int corners(const Job& J, const Level& lv, float px, float py, float pz, int vid[8],
                                       float w[8]) {
  const int n = lv.n;
  if (n == 1) {
    vid[0] = 0;
    w[0] = 1.f;
    return 1;
  }
  int ix, iy, iz;
  float fx, fy, fz;
  grid_coord(px, J.lo[0], lv.sc_hi[0], lv.sc_lo[0], n, ix, fx);
  grid_coord(py, J.lo[1], lv.sc_hi[1], lv.sc_lo[1], n, iy, fy);
  grid_coord(pz, J.lo[2], lv.sc_hi[2], lv.sc_lo[2], n, iz, fz);
  const int b = (iz * n + iy) * n + ix;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
    vid[c] = b + dx + dy * n + dz * n * n;
    w[c] = (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy) * (dz ? fz : 1.f - fz);
  }
  return 8;
}

__global__ void k_csr_count(Job* __restrict__ Jp) {
  const Job& J = *Jp;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J.Q; p += gridDim.x * blockDim.x) {
    const float4 x = J.x[p];
    for (int l = 0; l < J.L; ++l) {
      int vid[8];
      float w[8];
      const int K = corners(J, J.lev[l], x.x, x.y, x.z, vid, w);
      for (int c = 0; c < K; ++c) atomicAdd(&J.lev[l].cnt[vid[c]], 1);
    }
  }
}

__global__ void k_csr_fill(Job* __restrict__ Jp) {
  const Job& J = *Jp;
  const float invL = 1.f / (float)J.L;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J.Q; p += gridDim.x * blockDim.x) {
    const float4 x = J.x[p];
    for (int l = 0; l < J.L; ++l) {
      const Level& lv = J.lev[l];
      int vid[8];
      float w[8];
      const int K = corners(J, lv, x.x, x.y, x.z, vid, w);
      for (int c = 0; c < K; ++c) {
        const int pos = lv.rowptr[vid[c]] + atomicSub(&lv.cnt[vid[c]], 1) - 1;
        lv.ent_p[pos] = p;
        lv.ent_w[pos] = w[c] * invL;
      }
    }
  }
}

__global__ void k_csr_flags(Job* __restrict__ Jp, int l) {
  const Level& lv = Jp->lev[l];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < lv.n3; v += gridDim.x * blockDim.x)
    lv.flag[v] = lv.rowptr[v + 1] > lv.rowptr[v] ? 1 : 0;
}

__global__ void k_csr_compact(Job* __restrict__ Jp, int l) {
  const Level& lv = Jp->lev[l];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < lv.n3; v += gridDim.x * blockDim.x) {
    if (lv.rowptr[v + 1] > lv.rowptr[v]) {
      const int i = lv.flag[v];
      lv.act_v[i] = v;
      lv.act_ptr[i] = lv.rowptr[v];
    }
    if (v == 0) {
      const int na = lv.flag[lv.n3];
      *lv.n_active = na;
      lv.act_ptr[na] = lv.rowptr[lv.n3];
    }
  }
}

void launch_csr_build(Job* J, const Job& hJ, cudaStream_t s) {
  const int grid = max(1, min((hJ.Q + 255) / 256, 4096));
  k_csr_count<<<grid, 256, 0, s>>>(J);
  for (int l = 0; l < hJ.L; ++l) {
    const Level& lv = hJ.lev[l];
    ScanSeg seg{lv.cnt, lv.rowptr, lv.n3, lv.csum};
    launch_scan_segments(&seg, 1, nullptr, nullptr, s);
  }
  k_csr_fill<<<grid, 256, 0, s>>>(J);
  for (int l = 0; l < hJ.L; ++l) {
    const Level& lv = hJ.lev[l];
    const int g2 = max(1, min((lv.n3 + 255) / 256, 4096));
    k_csr_flags<<<g2, 256, 0, s>>>(J, l);
    ScanSeg seg{lv.flag, lv.flag, lv.n3, lv.csum};
    launch_scan_segments(&seg, 1, nullptr, nullptr, s);
    k_csr_compact<<<g2, 256, 0, s>>>(J, l);
  }
}

// ------------------------------------------------------------------------------ per step

// All levels of all jobs in one launch.  Levels of 128^3 and finer (a few dozen entries per
// row) give each warp 4 rows, 8 lanes per row; coarser levels (hundreds to thousands of
// entries per row) give each warp one row.  Every lane keeps 8 gathers in flight.  All
// partial sums are 64-bit fixed point, so the result does not depend on the split.
__device__ __forceinline__ void row_sum(const Level& lv, const float4* __restrict__ gy, int s, int e, int step,
                                        float sc, long long& ax, long long& ay, long long& az) {
  const int* __restrict__ ep = lv.ent_p;
  const float* __restrict__ ew = lv.ent_w;
  constexpr int B = 8;  // entries in flight per lane: all index loads, then all gathers
  int k = s;
  for (; k + (B - 1) * step < e; k += B * step) {
    int p[B];
    float wt[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      p[u] = __ldg(ep + k + u * step);
      wt[u] = __ldg(ew + k + u * step) * sc;  // exact: sc is a power of two
    }
    float4 g[B];
#pragma unroll
    for (int u = 0; u < B; ++u) g[u] = __ldg(gy + p[u]);
#pragma unroll
    for (int u = 0; u < B; ++u) {
      ax += __float2ll_rn(wt[u] * g[u].x);
      ay += __float2ll_rn(wt[u] * g[u].y);
      az += __float2ll_rn(wt[u] * g[u].z);
    }
  }
  for (; k < e; k += step) {
    const float w1 = __ldg(ew + k) * sc;
    const float4 g = __ldg(gy + __ldg(ep + k));
    ax += __float2ll_rn(w1 * g.x);
    ay += __float2ll_rn(w1 * g.y);
    az += __float2ll_rn(w1 * g.z);
  }
}

__global__ void __launch_bounds__(256) k_adjoint(const Plan* __restrict__ P) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_ADJ][nj];
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
    const int j = find_job(P->pre[ST_ADJ], nj, w);
    const Job& J = *P->jobs[j];
    int gi = w - P->pre[ST_ADJ][j];
    int l = 0, na = 0;
    for (; l < J.L; ++l) {
      na = *J.lev[l].n_active;
      const int ng = J.lev[l].n >= 128 ? (na + 3) >> 2 : na;
      if (gi < ng) break;
      gi -= ng;
    }
    if (l >= J.L) continue;
    const Level& lv = J.lev[l];
    const bool fine = lv.n >= 128;
    const int lpr = fine ? 8 : 32;             // lanes per row
    const int r = fine ? (gi << 2) + (lane >> 3) : gi;
    const int sub = fine ? (lane & 7) : lane;
    // fixed-point scale from the step's bound on |dL/dy|: every term |w g| < 2^ex and a row
    // has at most Q terms, so partial sums stay below 2^62
    const float gm = __uint_as_float(*J.gmax);
    const bool finite = gm <= 3.0e38f;
    int sh = 0;
    if (gm > 0.f && finite) {
      int ex;
      frexpf(gm, &ex);
      sh = min(62 - ex - (32 - __clz(J.Q)), 126);
    }
    const float sc = exp2f((float)sh), isc = exp2f((float)-sh);
    long long ax = 0, ay = 0, az = 0;
    if (r < na && gm > 0.f && finite)
      row_sum(lv, J.gy, __ldg(lv.act_ptr + r) + sub, __ldg(lv.act_ptr + r + 1), lpr, sc, ax, ay, az);
    // reduce within the row's lanes (aligned groups of lpr lanes)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long tx = __shfl_xor_sync(0xffffffffu, ax, o);
      const long long ty = __shfl_xor_sync(0xffffffffu, ay, o);
      const long long tz = __shfl_xor_sync(0xffffffffu, az, o);
      if (o < lpr) {
        ax += tx;
        ay += ty;
        az += tz;
      }
    }
    if (sub == 0 && r < na) {
      const int v = __ldg(lv.act_v + r);
      const float nan = __int_as_float(0x7fc00000);
      lv.g[v] = finite ? __ll2float_rn(ax) * isc : nan;
      lv.g[lv.n3 + v] = finite ? __ll2float_rn(ay) * isc : nan;
      lv.g[2 * lv.n3 + v] = finite ? __ll2float_rn(az) * isc : nan;
    }
  }
}

void launch_adjoint(const Plan* P, int grid, cudaStream_t s) { k_adjoint<<<grid, 256, 0, s>>>(P); }

}  // namespace pdg
