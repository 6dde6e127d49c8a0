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
        lv.ent[pos] = make_int2(p, __float_as_int(w[c] * invL));
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
  launch_zmask(J, hJ, s);
}

// ------------------------------------------------------------------------------ per step

// All levels of all jobs in one launch of 256-thread blocks.  Rows are summed by groups of
// 2^adj_lg lanes, set by the plan kernel from the level's mean row length (a few dozen
// entries per row on 128^3, thousands on 16^3): 32 >> adj_lg rows per warp, or a whole
// block per row on levels whose rows average 512 entries or more.  A job's items are its
// block rows first, then its warp groups, 8 to a block.  Each lane takes its entries in
// batches of 8: the 8 index and weight loads, then the 8 gathers, all issued before any of
// them is used (entries past the row's end get weight 0), so a lane waits for memory twice
// per batch however short its row.  All partial sums are 64-bit fixed point, so the result
// does not depend on the split.
// Round-to-nearest-even of x to an integer, exactly as a float -> int64 conversion, for
// |x| < 2^44, using only FP32 adds and integer subtracts (the direct conversion runs on
// the FP64 pipe, which is narrow on this part).  x + 1.5 2^45 lies in [2^45, 2^46), where
// the spacing of floats is 2^22, so hi = (x + 1.5 2^45) - 1.5 2^45 is x rounded to a
// multiple of 2^22 and lo = x - hi (|lo| <= 2^21) is exact.  For |v| <= 2^22, v + 1.5 2^23
// lies in [2^23, 2^24) with spacing 1, so its bit pattern minus that of 1.5 2^23 is v
// rounded to an integer.  hi is even, so rounding lo rounds x the same way on ties.
__device__ __forceinline__ long long round_to_ll(float x) {
  const float kHi = 52776558133248.0f;  // 1.5 * 2^45
  const float kLo = 12582912.0f;        // 1.5 * 2^23
  const float hi = __fsub_rn(__fadd_rn(x, kHi), kHi);
  const float lo = __fsub_rn(x, hi);
  const int li = __float_as_int(__fadd_rn(lo, kLo)) - __float_as_int(kLo);
  const int hq = __float_as_int(__fadd_rn(__fmul_rn(hi, 2.384185791015625e-07f), kLo)) - __float_as_int(kLo);
  return ((long long)hq << 22) + li;
}

__device__ __forceinline__ void row_sum(const Level& lv, const float4* __restrict__ gy, int s, int e, int step,
                                        float sc, long long& ax, long long& ay, long long& az) {
  const int2* __restrict__ en = lv.ent;
  constexpr int B = 8;
  if (s >= e) return;
  int p[B];
  float wt[B];
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const int kk = min(s + u * step, e - 1);  // past the end: reload the last entry, weight 0
    const int2 t = __ldg(en + kk);
    p[u] = t.x;
    wt[u] = s + u * step < e ? __int_as_float(t.y) * sc : 0.f;  // exact: sc is a power of two
  }
  for (int k = s; k < e; k += B * step) {
    float4 g[B];
#pragma unroll
    for (int u = 0; u < B; ++u) g[u] = __ldg(gy + p[u]);
    // the next batch's entries are loaded while this batch's gathers are in flight
    const int kn = k + B * step;
    int pn[B];
    float wn[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int kk = min(kn + u * step, e - 1);
      const int2 t = __ldg(en + kk);
      pn[u] = t.x;
      wn[u] = kn + u * step < e ? __int_as_float(t.y) * sc : 0.f;
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      ax += round_to_ll(__fmul_rn(wt[u], g[u].x));
      ay += round_to_ll(__fmul_rn(wt[u], g[u].y));
      az += round_to_ll(__fmul_rn(wt[u], g[u].z));
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      p[u] = pn[u];
      wt[u] = wn[u];
    }
  }
}

// sum over aligned groups of `width` lanes (a power of two); every lane gets its group's sum
__device__ __forceinline__ void group_sum(long long& ax, long long& ay, long long& az, int width) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long tx = __shfl_xor_sync(0xffffffffu, ax, o);
    const long long ty = __shfl_xor_sync(0xffffffffu, ay, o);
    const long long tz = __shfl_xor_sync(0xffffffffu, az, o);
    if (o < width) {
      ax += tx;
      ay += ty;
      az += tz;
    }
  }
}

__device__ __forceinline__ void store_row(const Level& lv, int r, bool finite, float isc, long long ax, long long ay,
                                          long long az) {
  const int v = __ldg(lv.act_v + r);
  const float nan = __int_as_float(0x7fc00000);
  lv.g[v] = finite ? __ll2float_rn(ax) * isc : nan;
  lv.g[lv.n3 + v] = finite ? __ll2float_rn(ay) * isc : nan;
  lv.g[2 * lv.n3 + v] = finite ? __ll2float_rn(az) * isc : nan;
}

__global__ void __launch_bounds__(256, 4) k_adjoint(const Plan* __restrict__ P) {
  __shared__ long long red[3][8];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_ADJ][nj];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {  // block-uniform
    const int j = find_job(P->pre[ST_ADJ], nj, it);
    const Job& J = *P->jobs[j];
    int i = it - P->pre[ST_ADJ][j];
    // fixed-point scale from the step's bound on |dL/dy|: every term |w g| < 2^ex, so a
    // scaled term is below 2^44 (the range of round_to_ll), and a row has at most Q terms,
    // so partial sums stay below 2^62
    const float gm = __uint_as_float(*J.gmax);
    const bool finite = gm <= 3.0e38f;
    const bool live = gm > 0.f && finite;
    int sh = 0;
    if (live) {  // ex: gm = m 2^ex with m in [0.5, 1), as frexp
      const unsigned gb = __float_as_uint(gm);
      const int be = (int)(gb >> 23);
      const int ex = be ? be - 126 : (31 - __clz((int)(gb & 0x7fffffu))) - 148;
      sh = min(min(62 - (32 - __clz(J.Q)), 44) - ex, 126);
    }
    const float sc = exp2f((float)sh), isc = exp2f((float)-sh);
    // block rows
    int l = 0;
    for (; l < J.L; ++l) {
      if (J.lev[l].adj_lg != 6) continue;
      const int na = *J.lev[l].n_active;
      if (i < na) break;
      i -= na;
    }
    if (l < J.L) {
      const Level& lv = J.lev[l];
      long long ax = 0, ay = 0, az = 0;
      if (live) row_sum(lv, J.gy, __ldg(lv.act_ptr + i) + threadIdx.x, __ldg(lv.act_ptr + i + 1), 256, sc, ax, ay, az);
      group_sum(ax, ay, az, 32);
      if (lane == 0) {
        red[0][warp] = ax;
        red[1][warp] = ay;
        red[2][warp] = az;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int k = 1; k < 8; ++k) {
          ax += red[0][k];
          ay += red[1][k];
          az += red[2][k];
        }
        store_row(lv, i, finite, isc, ax, ay, az);
      }
      __syncthreads();
      continue;
    }
    // warp groups
    int gi = i * 8 + warp, na = 0, lg = 0;
    for (l = 0; l < J.L; ++l) {
      lg = J.lev[l].adj_lg;
      if (lg == 6) continue;
      na = *J.lev[l].n_active;
      const int ng = (na + (32 >> lg) - 1) >> (5 - lg);
      if (gi < ng) break;
      gi -= ng;
    }
    if (l >= J.L) continue;  // past the last group (whole warp)
    const Level& lv = J.lev[l];
    const int lpr = 1 << lg;
    const int r = (gi << (5 - lg)) + (lane >> lg);
    const int sub = lane & (lpr - 1);
    long long ax = 0, ay = 0, az = 0;
    if (r < na && live) row_sum(lv, J.gy, __ldg(lv.act_ptr + r) + sub, __ldg(lv.act_ptr + r + 1), lpr, sc, ax, ay, az);
    group_sum(ax, ay, az, lpr);
    if (sub == 0 && r < na) store_row(lv, r, finite, isc, ax, ay, az);
  }
}

void launch_adjoint(const Plan* P, int grid, cudaStream_t s) { k_adjoint<<<grid, 256, 0, s>>>(P); }

}  // namespace pdg
