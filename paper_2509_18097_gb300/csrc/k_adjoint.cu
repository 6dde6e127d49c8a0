// Adjoint of the multi-level trilinear evaluation (chain rule of Eq. 1):
//   dLoss/dTheta_l[v] = (1/L) sum_{p : v is a corner of p in level l} w_{l,v}(x_p) dLoss/dy_p.
// The query points x are fixed for a whole frame, so the per-level point -> vertex lists
// (point id, weight / L) are built once per frame by a counting sort keyed by vertex, and
// compacted to the vertices that some point touches.  Each step then gathers every active
// vertex's row.  A row is summed in 64-bit fixed point with a per-row scale chosen from the
// row's largest term: integer addition is associative, so the result does not depend on
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

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// one warp per active vertex row; all levels of all jobs in one launch
__global__ void __launch_bounds__(256) k_adjoint(const Plan* __restrict__ P) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_ADJ][nj];
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
    const int j = find_job(P->pre[ST_ADJ], nj, w);
    const Job& J = *P->jobs[j];
    int r = w - P->pre[ST_ADJ][j];
    int l = 0;
    for (; l < J.L - 1; ++l) {
      const int na = *J.lev[l].n_active;
      if (r < na) break;
      r -= na;
    }
    const Level& lv = J.lev[l];
    const int v = lv.act_v[r];
    const int s = lv.act_ptr[r], e = lv.act_ptr[r + 1];
    // pass 1: largest |w g| of the row
    float mx = 0.f;
    for (int k = s + lane; k < e; k += 32) {
      const float wt = lv.ent_w[k];
      const float4 g = J.gy[lv.ent_p[k]];
      mx = fmaxf(mx, fmaxf(fabsf(wt * g.x), fmaxf(fabsf(wt * g.y), fabsf(wt * g.z))));
    }
    mx = warp_max(mx);
    float ox = 0.f, oy = 0.f, oz = 0.f;
    if (mx > 0.f && mx <= 3.0e38f) {
      int ex;
      frexpf(mx, &ex);                  // mx < 2^ex
      const int lg = 32 - __clz(e - s);  // row length < 2^lg
      const int sh = 62 - ex - lg;      // every partial sum stays below 2^62
      long long ax = 0, ay = 0, az = 0;
      for (int k = s + lane; k < e; k += 32) {
        const float wt = lv.ent_w[k];
        const float4 g = J.gy[lv.ent_p[k]];
        ax += __float2ll_rn(ldexpf(wt * g.x, sh));
        ay += __float2ll_rn(ldexpf(wt * g.y, sh));
        az += __float2ll_rn(ldexpf(wt * g.z, sh));
      }
      ax = warp_sum(ax);
      ay = warp_sum(ay);
      az = warp_sum(az);
      ox = ldexpf(__ll2float_rn(ax), -sh);
      oy = ldexpf(__ll2float_rn(ay), -sh);
      oz = ldexpf(__ll2float_rn(az), -sh);
    } else if (!(mx <= 3.0e38f)) {
      ox = oy = oz = __int_as_float(0x7fc00000);  // propagate a non-finite gradient
    }
    if (lane == 0) {
      lv.g[v] = ox;
      lv.g[lv.n3 + v] = oy;
      lv.g[2 * lv.n3 + v] = oz;
    }
  }
}

void launch_adjoint(const Plan* P, int grid, cudaStream_t s) { k_adjoint<<<grid, 256, 0, s>>>(P); }

}  // namespace pdg
