// Adjoint of the multi-level trilinear evaluation (chain rule of Eq. 1):
//   dLoss/dTheta_l[v] = (1/L) sum_{p : v is a corner of p in level l} w_{l,v}(x_p) dLoss/dy_p.
// The query points x are fixed for a whole frame, so the per-level point -> vertex lists
// (point id, weight / L) are built once per frame by a counting sort keyed by vertex, and
// compacted to the vertices that some point touches.  Each step then gathers every active
// vertex's row (with the Cayley payload, both the dLoss/dz and the dLoss/dt halves).  A row is summed in 64-bit fixed point with a scale chosen from the step's
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


// The finest level's cell order of the query points (per frame): counting sort of the points
// by interpolation cell (iz (n-1) + iy)(n-1) + ix, storing each point's fractions and index.
// The interpolation takes its points in this order, so the lanes of a warp interpolate
// between the same or neighbouring grid vertices.
__device__ __forceinline__ int point_cell(const Job& J, const Level& lv, float px, float py, float pz, float& fx,
                                          float& fy, float& fz) {
  const int n = lv.n;
  if (n == 1) {
    fx = fy = fz = 0.f;
    return 0;
  }
  int ix, iy, iz;
  grid_coord(px, J.lo[0], lv.sc_hi[0], lv.sc_lo[0], n, ix, fx);
  grid_coord(py, J.lo[1], lv.sc_hi[1], lv.sc_lo[1], n, iy, fy);
  grid_coord(pz, J.lo[2], lv.sc_hi[2], lv.sc_lo[2], n, iz, fz);
  return (iz * (n - 1) + iy) * (n - 1) + ix;
}

__global__ void k_cell_count(Job* __restrict__ Jp) {
  const Job& J = *Jp;
  const Level& lv = J.lev[J.L - 1];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J.Q; p += gridDim.x * blockDim.x) {
    const float4 x = J.x[p];
    float fx, fy, fz;
    const int c = point_cell(J, lv, x.x, x.y, x.z, fx, fy, fz);
    lv.ckey[p] = c;
    atomicAdd(&lv.ccnt[c], 1);
  }
}

__global__ void k_cell_fill(Job* __restrict__ Jp) {
  const Job& J = *Jp;
  const Level& lv = J.lev[J.L - 1];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J.Q; p += gridDim.x * blockDim.x) {
    const float4 x = J.x[p];
    float fx, fy, fz;
    point_cell(J, lv, x.x, x.y, x.z, fx, fy, fz);
    const int c = lv.ckey[p];
    const int pos = lv.coff[c] + atomicSub(&lv.ccnt[c], 1) - 1;  // counts return to zero
    lv.xs[pos] = make_float4(fx, fy, fz, __int_as_float(p));
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
  // the finest level's cell order
  const Level& lf = hJ.lev[hJ.L - 1];
  const int nc = lf.n > 1 ? (lf.n - 1) * (lf.n - 1) * (lf.n - 1) : 1;
  k_cell_count<<<grid, 256, 0, s>>>(J);
  ScanSeg seg{lf.ccnt, lf.coff, nc, lf.csum};
  launch_scan_segments(&seg, 1, nullptr, nullptr, s);
  k_cell_fill<<<grid, 256, 0, s>>>(J);
  launch_zmask(J, hJ, s);
}

// ------------------------------------------------------------------------------ per step

// All levels of all jobs in one launch of 256-thread blocks.  Rows are summed by groups of
// 2^adj_lg lanes, set by the plan kernel from the level's mean row length (a few dozen
// entries per row on 128^3, thousands on 16^3): 32 >> adj_lg rows per warp, or a whole
// block per row on levels whose rows average 512 entries or more.  A job's items are its
// block rows first, then its warp groups, 8 to a block.  Each lane takes its entries in
// batches of B: the B index and weight loads, then the B gathers (of dLoss/dz and dLoss/dt
// with the Cayley payload), all issued before any of them is used (entries past the row's end
// get weight 0), and loads its next batch's entries while those gathers are in flight.  All
// partial sums are 64-bit fixed point, so the result does not depend on the split.
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


// Fixed-point sums of one row: a = weights times dLoss/dy (dLoss/dz with the Cayley payload),
// b = weights times dLoss/dt (Cayley payload only).
struct RowAcc {
  long long a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;
};

template <int C>
__device__ __forceinline__ void row_sum(const Level& lv, const float4* __restrict__ gy, const float4* __restrict__ gz,
                                        int s, int e, int step, float sc, RowAcc& A) {
  const int2* __restrict__ en = lv.ent;
  constexpr int B = C == 6 ? 4 : 8;
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
    float4 g[B], h[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      if (C == 6) {
        g[u] = __ldg(gz + p[u]);
        h[u] = __ldg(gy + p[u]);
      } else {
        g[u] = __ldg(gy + p[u]);
      }
    }
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
      A.a0 += round_to_ll(__fmul_rn(wt[u], g[u].x));
      A.a1 += round_to_ll(__fmul_rn(wt[u], g[u].y));
      A.a2 += round_to_ll(__fmul_rn(wt[u], g[u].z));
      if (C == 6) {
        A.b0 += round_to_ll(__fmul_rn(wt[u], h[u].x));
        A.b1 += round_to_ll(__fmul_rn(wt[u], h[u].y));
        A.b2 += round_to_ll(__fmul_rn(wt[u], h[u].z));
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      p[u] = pn[u];
      wt[u] = wn[u];
    }
  }
}

// sum over aligned groups of `width` lanes (a power of two); every lane gets its group's sum
__device__ __forceinline__ void group_sum(long long& v, int width) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long t = __shfl_xor_sync(0xffffffffu, v, o);
    if (o < width) v += t;
  }
}

template <int C>
__device__ __forceinline__ void group_sum(RowAcc& A, int width) {
  group_sum(A.a0, width);
  group_sum(A.a1, width);
  group_sum(A.a2, width);
  if (C == 6) {
    group_sum(A.b0, width);
    group_sum(A.b1, width);
    group_sum(A.b2, width);
  }
}

// channels 0..2 from the a sums, 3..5 (Cayley t) from the b sums
template <int C>
__device__ __forceinline__ void store_row(const Level& lv, int r, bool finite, float isc, const RowAcc& A) {
  const int v = __ldg(lv.act_v + r);
  const float nan = __int_as_float(0x7fc00000);
  const size_t n3 = lv.n3;
  lv.g[v] = finite ? __ll2float_rn(A.a0) * isc : nan;
  lv.g[n3 + v] = finite ? __ll2float_rn(A.a1) * isc : nan;
  lv.g[2 * n3 + v] = finite ? __ll2float_rn(A.a2) * isc : nan;
  if (C == 6) {
    lv.g[3 * n3 + v] = finite ? __ll2float_rn(A.b0) * isc : nan;
    lv.g[4 * n3 + v] = finite ? __ll2float_rn(A.b1) * isc : nan;
    lv.g[5 * n3 + v] = finite ? __ll2float_rn(A.b2) * isc : nan;
  }
}

// a whole block sums row i of level lv, thread 0 stores it
template <int C>
__device__ __forceinline__ void block_row(const Job& J, const Level& lv, int i, bool live, bool finite, float sc,
                                          float isc, long long (*red)[8]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RowAcc A;
  if (live) row_sum<C>(lv, J.gy, J.gz, __ldg(lv.act_ptr + i) + threadIdx.x, __ldg(lv.act_ptr + i + 1), 256, sc, A);
  group_sum<C>(A, 32);
  if (lane == 0) {
    red[0][warp] = A.a0; red[1][warp] = A.a1; red[2][warp] = A.a2;
    if (C == 6) {
      red[3][warp] = A.b0; red[4][warp] = A.b1; red[5][warp] = A.b2;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; ++k) {
      A.a0 += red[0][k]; A.a1 += red[1][k]; A.a2 += red[2][k];
      if (C == 6) {
        A.b0 += red[3][k]; A.b1 += red[4][k]; A.b2 += red[5][k];
      }
    }
    store_row<C>(lv, i, finite, isc, A);
  }
  __syncthreads();
}

// a group of 2^lg lanes sums row r of level lv
template <int C>
__device__ __forceinline__ void group_row(const Job& J, const Level& lv, int r, int na, int lg, bool live, bool finite,
                                          float sc, float isc) {
  const int lane = threadIdx.x & 31;
  const int lpr = 1 << lg;
  const int sub = lane & (lpr - 1);
  RowAcc A;
  if (r < na && live) row_sum<C>(lv, J.gy, J.gz, __ldg(lv.act_ptr + r) + sub, __ldg(lv.act_ptr + r + 1), lpr, sc, A);
  group_sum<C>(A, lpr);
  if (sub == 0 && r < na) store_row<C>(lv, r, finite, isc, A);
}

__global__ void __launch_bounds__(256, 4) k_adjoint(const Plan* __restrict__ P) {
  __shared__ long long red[6][8];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_ADJ][nj];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {  // block-uniform
    const int j = find_job(P->pre[ST_ADJ], nj, it);
    const Job& J = *P->jobs[j];
    int i = it - P->pre[ST_ADJ][j];
    // fixed-point scale from the step's bound on the point gradients: every term |w g| < 2^ex,
    // so a scaled term is below 2^44 (the range of round_to_ll), and a row has at most Q
    // terms, so partial sums stay below 2^62
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
      if (J.C == 6) block_row<6>(J, J.lev[l], i, live, finite, sc, isc, red);
      else block_row<3>(J, J.lev[l], i, live, finite, sc, isc, red);
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
    const int r = (gi << (5 - lg)) + (lane >> lg);
    if (J.C == 6) group_row<6>(J, J.lev[l], r, na, lg, live, finite, sc, isc);
    else group_row<3>(J, J.lev[l], r, na, lg, live, finite, sc, isc);
  }
}

void launch_adjoint(const Plan* P, int grid, cudaStream_t s) { k_adjoint<<<grid, 256, 0, s>>>(P); }

}  // namespace pdg
