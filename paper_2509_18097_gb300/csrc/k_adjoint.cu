// Adjoint of the multi-level trilinear evaluation (chain rule of Eq. 1):
//   dLoss/dTheta_l[v] = (1/L) sum_{p : v is a corner of p in level l} w_{l,v}(x_p) dLoss/dy_p.
// The query points x are fixed for a whole frame, so once per frame each level counting-sorts
// them by their interpolation cell and stores, in cell order, each point's index and its
// fractional position in the cell.  Each step then gathers every active vertex (a corner of
// a non-empty cell) over the points of its (at most 8) adjacent cells, recomputing the
// trilinear weight of the vertex from the stored fractions.  In row-major cell order the two
// cells of a vertex that differ in x are neighbours, so the 8 cells are 4 contiguous ranges.
// A row is summed in 64-bit fixed point with a scale chosen from the step's bound on
// |dLoss/dy| (taken in the assembly kernel): integer addition is associative, so the result
// does not depend on the (atomic, unordered) order of the points within a cell, nor on how
// the row is split across lanes.  No floating-point atomics are used.
#include "kernels.h"

namespace pdg {

// interpolation cell and in-cell fractions of point p in level lv (Eq. 1; grid_coord clamps
// and closes the last cell); n = 1: the single cell 0
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

__device__ __forceinline__ int level_cells(const Level& lv) {
  return lv.n > 1 ? (lv.n - 1) * (lv.n - 1) * (lv.n - 1) : 1;
}

__global__ void k_cell_count(Job* __restrict__ Jp) {
  const Job& J = *Jp;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J.Q; p += gridDim.x * blockDim.x) {
    const float4 x = J.x[p];
    for (int l = 0; l < J.L; ++l) {
      const Level& lv = J.lev[l];
      float fx, fy, fz;
      const int c = point_cell(J, lv, x.x, x.y, x.z, fx, fy, fz);
      lv.ckey[p] = c;
      atomicAdd(&lv.ccnt[c], 1);
    }
  }
}

__global__ void k_cell_fill(Job* __restrict__ Jp) {
  const Job& J = *Jp;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J.Q; p += gridDim.x * blockDim.x) {
    const float4 x = J.x[p];
    for (int l = 0; l < J.L; ++l) {
      const Level& lv = J.lev[l];
      float fx, fy, fz;
      point_cell(J, lv, x.x, x.y, x.z, fx, fy, fz);
      const int c = lv.ckey[p];
      const int pos = lv.coff[c] + atomicSub(&lv.ccnt[c], 1) - 1;  // counts return to zero
      lv.xs[pos] = make_float4(fx, fy, fz, __int_as_float(p));
    }
  }
}

// flag[v] = 1 for the corners of every non-empty cell (flag is zero before)
__global__ void k_vertex_flags(Job* __restrict__ Jp, int l) {
  const Level& lv = Jp->lev[l];
  const int n = lv.n, nc = level_cells(lv);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    if (lv.coff[c + 1] == lv.coff[c]) continue;
    if (n == 1) {
      lv.flag[0] = 1;
      continue;
    }
    const int m = n - 1;
    const int ix = c % m, iy = (c / m) % m, iz = c / (m * m);
    const int v0 = (iz * n + iy) * n + ix;
#pragma unroll
    for (int k = 0; k < 8; ++k) lv.flag[v0 + (k & 1) + ((k >> 1) & 1) * n + (k >> 2) * n * n] = 1;
  }
}

// active vertices in ascending order from the exclusive prefix of the flags
__global__ void k_vertex_compact(Job* __restrict__ Jp, int l) {
  const Level& lv = Jp->lev[l];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < lv.n3; v += gridDim.x * blockDim.x) {
    const int i = lv.flag[v];
    if (lv.flag[v + 1] > i) lv.act_v[i] = v;
    if (v == 0) *lv.n_active = lv.flag[lv.n3];
  }
}

void launch_csr_build(Job* J, const Job& hJ, cudaStream_t s) {
  const int grid = max(1, min((hJ.Q + 255) / 256, 4096));
  k_cell_count<<<grid, 256, 0, s>>>(J);
  for (int l = 0; l < hJ.L; ++l) {
    const Level& lv = hJ.lev[l];
    const int nc = lv.n > 1 ? (lv.n - 1) * (lv.n - 1) * (lv.n - 1) : 1;
    ScanSeg seg{lv.ccnt, lv.coff, nc, lv.csum};
    launch_scan_segments(&seg, 1, nullptr, nullptr, s);
  }
  k_cell_fill<<<grid, 256, 0, s>>>(J);
  for (int l = 0; l < hJ.L; ++l) {
    const Level& lv = hJ.lev[l];
    const int nc = lv.n > 1 ? (lv.n - 1) * (lv.n - 1) * (lv.n - 1) : 1;
    cudaMemsetAsync(lv.flag, 0, sizeof(int) * ((size_t)lv.n3 + 1), s);
    k_vertex_flags<<<max(1, min((nc + 255) / 256, 4096)), 256, 0, s>>>(J, l);
    ScanSeg seg{lv.flag, lv.flag, lv.n3, lv.csum};
    launch_scan_segments(&seg, 1, nullptr, nullptr, s);
    k_vertex_compact<<<max(1, min((lv.n3 + 255) / 256, 4096)), 256, 0, s>>>(J, l);
  }
  launch_zmask(J, hJ, s);
}

// ------------------------------------------------------------------------------ per step

// All levels of all jobs in one launch of 256-thread blocks.  Rows are summed by groups of
// 2^adj_lg lanes, set by the plan kernel from the level's mean row length (a few dozen
// terms per row on 128^3, thousands on 16^3): 32 >> adj_lg rows per warp, or a whole
// block per row on levels whose rows average 512 terms or more.  A job's items are its
// block rows first, then its warp groups, 8 to a block.  A row's terms are the points of its
// 4 cell ranges (row_sum); all partial sums are 64-bit fixed point, so the result does not
// depend on the split.
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

// Fixed-point sums of one row: a = weights times the first gradient (dLoss/dy, or dLoss/dz of
// the Cayley payload), b = weights times dLoss/dt (Cayley payload only).
struct RowAcc {
  long long a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;
};

// Sums the terms of one cell range of the row: the lane takes the points s, s + step, ... of
// the range in batches of 4 (the 4 cell-order loads, the weights formed from them, then the 4
// gradient gathers, all issued before any is used; terms past the end get weight 0).  The
// weight of the vertex for a point is (wx wy wz) / L times the fixed-point scale sc (a power
// of two, so the product is exact), with wx = f or 1 - f by the point's x-cell.
template <int C>
__device__ __forceinline__ void range_sum(const Level& lv, const float4* __restrict__ gy, const float4* __restrict__ gz,
                                          int st, int split, int end, bool ylow, bool zlow, int xlo, int i, int s,
                                          int step, float invL, float sc, RowAcc& A) {
  constexpr int B = 4;
  for (int k = st + s; k < end; k += B * step) {
    int p[B];
    float wt[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int kk = k + u * step;
      const bool live = kk < end;
      const float4 e = __ldg(lv.xs + (live ? kk : end - 1));
      p[u] = __float_as_int(e.w);
      const bool xl = (live ? kk : end - 1) < split ? xlo == i - 1 : xlo + 1 == i - 1;
      const float wx = xl ? e.x : __fsub_rn(1.f, e.x);
      const float wy = ylow ? e.y : __fsub_rn(1.f, e.y);
      const float wz = zlow ? e.z : __fsub_rn(1.f, e.z);
      const float w = __fmul_rn(__fmul_rn(__fmul_rn(wx, wy), wz), invL);
      wt[u] = live ? __fmul_rn(w, sc) : 0.f;
    }
    if (C == 6) {  // channels z (from dLoss/dz) then t (from dLoss/dy)
      float4 g[B], h[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        g[u] = __ldg(gz + p[u]);
        h[u] = __ldg(gy + p[u]);
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        A.a0 += round_to_ll(__fmul_rn(wt[u], g[u].x));
        A.a1 += round_to_ll(__fmul_rn(wt[u], g[u].y));
        A.a2 += round_to_ll(__fmul_rn(wt[u], g[u].z));
        A.b0 += round_to_ll(__fmul_rn(wt[u], h[u].x));
        A.b1 += round_to_ll(__fmul_rn(wt[u], h[u].y));
        A.b2 += round_to_ll(__fmul_rn(wt[u], h[u].z));
      }
    } else {
      float4 g[B];
#pragma unroll
      for (int u = 0; u < B; ++u) g[u] = __ldg(gy + p[u]);
#pragma unroll
      for (int u = 0; u < B; ++u) {
        A.a0 += round_to_ll(__fmul_rn(wt[u], g[u].x));
        A.a1 += round_to_ll(__fmul_rn(wt[u], g[u].y));
        A.a2 += round_to_ll(__fmul_rn(wt[u], g[u].z));
      }
    }
  }
}

// The terms of the row of vertex v: the points of the (at most 8) cells around it, as 4
// ranges of the cell-ordered points.  Range r takes the cells at y-index j - (r & 1) and
// z-index k - (r >> 1) (along an axis where the cell index is j - 1 the vertex is the cell's
// upper corner, so its weight there is f, else 1 - f) and, along x, the cells
// max(i - 1, 0) .. min(i, n - 2), which are neighbours in row-major cell order.
template <int C>
__device__ __forceinline__ void row_sum(const Level& lv, int v, const float4* __restrict__ gy,
                                        const float4* __restrict__ gz, int s, int step, float invL, float sc,
                                        RowAcc& A) {
  const int n = lv.n;
  if (n == 1) {  // one cell holding every point, weight 1 / L
    const int q = __ldg(lv.coff + 1);
    range_sum<C>(lv, gy, gz, 0, q, q, false, false, 0, 0, s, step, invL, sc, A);
    return;
  }
  const int m = n - 1;
  const int i = v % n, j = (v / n) % n, k = v / (n * n);
  const int xlo = max(i - 1, 0), xhi = min(i, m - 1);
#pragma unroll 1
  for (int r = 0; r < 4; ++r) {
    const int cy = j - (r & 1), cz = k - (r >> 1);
    if (cy < 0 || cy >= m || cz < 0 || cz >= m) continue;
    const int cb = (cz * m + cy) * m;
    const int st = __ldg(lv.coff + cb + xlo), split = __ldg(lv.coff + cb + xlo + 1);
    const int end = __ldg(lv.coff + cb + xhi + 1);
    range_sum<C>(lv, gy, gz, st, split, end, (r & 1) != 0, (r >> 1) != 0, xlo, i, s, step, invL, sc, A);
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

// the block-wide sum of one row (a block per row) and its store by thread 0
template <int C>
__device__ __forceinline__ void block_row(const Job& J, const Level& lv, int i, bool live, bool finite, float invL,
                                          float sc, float isc, long long (*red)[8]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RowAcc A;
  if (live) row_sum<C>(lv, __ldg(lv.act_v + i), J.gy, J.gz, threadIdx.x, 256, invL, sc, A);
  group_sum<C>(A, 32);
  if (lane == 0) {
    red[0][warp] = A.a0; red[1][warp] = A.a1; red[2][warp] = A.a2;
    red[3][warp] = A.b0; red[4][warp] = A.b1; red[5][warp] = A.b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; ++k) {
      A.a0 += red[0][k]; A.a1 += red[1][k]; A.a2 += red[2][k];
      A.b0 += red[3][k]; A.b1 += red[4][k]; A.b2 += red[5][k];
    }
    store_row<C>(lv, i, finite, isc, A);
  }
  __syncthreads();
}

template <int C>
__device__ __forceinline__ void group_row(const Job& J, const Level& lv, int r, int na, int lg, bool live, bool finite,
                                          float invL, float sc, float isc) {
  const int lane = threadIdx.x & 31;
  const int lpr = 1 << lg;
  const int sub = lane & (lpr - 1);
  RowAcc A;
  if (r < na && live) row_sum<C>(lv, __ldg(lv.act_v + r), J.gy, J.gz, sub, lpr, invL, sc, A);
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
    const float invL = 1.f / (float)J.L;
    // block rows
    int l = 0;
    for (; l < J.L; ++l) {
      if (J.lev[l].adj_lg != 6) continue;
      const int na = *J.lev[l].n_active;
      if (i < na) break;
      i -= na;
    }
    if (l < J.L) {
      if (J.C == 6) block_row<6>(J, J.lev[l], i, live, finite, invL, sc, isc, red);
      else block_row<3>(J, J.lev[l], i, live, finite, invL, sc, isc, red);
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
    if (J.C == 6) group_row<6>(J, J.lev[l], r, na, lg, live, finite, invL, sc, isc);
    else group_row<3>(J, J.lev[l], r, na, lg, live, finite, invL, sc, isc);
  }
}

void launch_adjoint(const Plan* P, int grid, cudaStream_t s) { k_adjoint<<<grid, 256, 0, s>>>(P); }

}  // namespace pdg
