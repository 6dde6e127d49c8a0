// Exact nearest neighbours for the bidirectional robust Chamfer distance (Sec. 3.4) and
// its gradient.  Four searches per step: template vertices and source points (the moving
// sets) against the target cloud, and the target cloud against each moving set.
//
// The target (per frame) and the moving sets (per step) are counting-sorted into uniform
// cell grids (see CellGrid, about 32 points per occupied cell).  A first kernel searches
// every query's 3x3x3 cell box with one thread per query, starting from the query's
// neighbour of the previous step, queries taken in cell order so neighbouring lanes read the
// same cells (cells that cannot beat the best distance found so far are skipped).  The
// answer is certified when the best squared distance is below the squared distance from the
// query to the searched box's open faces (with a margin covering the rounding of the cell
// assignment); otherwise the same thread searches the next shell (up to NN_RTHREAD), and a
// query still uncertified is appended to a per-job list that a second, warp-cooperative
// kernel searches ring by ring (lanes split the rows of each shell, a
// __shfl min-reduction over (d^2, index) packed in 64 bits picks the lexicographic minimum,
// i.e. the lowest index on ties), falling back to an exhaustive scan of the set beyond
// NN_RMAX rings.  Both kernels compare candidates with the same fp32 expression, so the
// result is the exact lexicographic minimum of (fp32 d^2, index) over the whole set.
#include <float.h>

#include "kernels.h"

namespace pdg {

// Best candidate so far; `tie` (counting instance only): another point had exactly the same
// squared distance (the lowest index decided), which the step reports as a count.
struct Best {
  float d2;
  int idx;
  bool tie;
};

// COUNT: the instance used when the context counts (PDG_DEBUG_COUNT_NN); it also tracks
// exact ties.  The two instances take the same minimum.
template <bool COUNT>
__device__ __forceinline__ void consider(Best& b, const float4 p, float qx, float qy, float qz) {
  const float d2 = sqdist(qx, qy, qz, p.x, p.y, p.z);
  if (d2 <= b.d2) {  // rarely taken; the index decides only between equal distances
    const int id = __float_as_int(p.w);
    if (COUNT) {
      if (d2 < b.d2) {
        b.d2 = d2;
        b.idx = id;
        b.tie = false;
      } else if (id != b.idx) {
        b.tie = true;
        b.idx = min(b.idx, id);
      }
    } else if (d2 < b.d2 || id < b.idx) {
      b.d2 = d2;
      b.idx = id;
    }
  }
}

// Squared lower bound on the distance from q to any point assigned to a cell outside the
// box [c - r, c + r] (per axis, clipped to the grid).  FLT_MAX if the box covers the grid.
__device__ __forceinline__ float outside_bound2(const CellGrid& g, float qx, float qy, float qz, int cx, int cy,
                                                int cz, int r) {
  const int G = 1 << g.bits;
  const float q[3] = {qx, qy, qz};
  const int c[3] = {cx, cy, cz};
  float d = FLT_MAX;
  float hmin = FLT_MAX;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hmin = fminf(hmin, g.h[a]);
    if (c[a] - r > 0) d = fminf(d, q[a] - (g.lo[a] + (float)(c[a] - r) * g.h[a]));
    if (c[a] + r < G - 1) d = fminf(d, (g.lo[a] + (float)(c[a] + r + 1) * g.h[a]) - q[a]);
  }
  if (d == FLT_MAX) return FLT_MAX;
  d -= 1e-4f * hmin;  // cell assignment and face positions are rounded in fp32
  if (d <= 0.f) return 0.f;
  return d * d * (1.f - 4e-6f);
}

// Lower bounds on the distance from q to the points assigned to other cells of its grid.
// m[a] / p[a]: distance from q to the lower / upper face of its own cell along axis a, less
// the same rounding margin as above (negative for a query clamped into a boundary cell).
// A cell d steps away along a (d < 0 below) lies beyond that face plus |d| - 1 cells.
struct FaceBounds {
  float m[3], p[3], h[3];
};

__device__ __forceinline__ FaceBounds face_bounds(const CellGrid& g, float qx, float qy, float qz, int cx, int cy,
                                                  int cz) {
  const float q[3] = {qx, qy, qz};
  const int c[3] = {cx, cy, cz};
  const float margin = 1e-4f * fminf(g.h[0], fminf(g.h[1], g.h[2]));
  FaceBounds f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f.m[a] = q[a] - (g.lo[a] + (float)c[a] * g.h[a]) - margin;
    f.p[a] = (g.lo[a] + (float)(c[a] + 1) * g.h[a]) - q[a] - margin;
    f.h[a] = g.h[a];
  }
  return f;
}

// squared lower bound contributed by axis a for a cell d steps away (0 for d = 0), shrunk by
// the relative rounding of a squared distance; the bound of a cell is the sum over its axes
__device__ __forceinline__ float axis_lb(const FaceBounds& f, int a, int d) {
  if (d == 0) return 0.f;
  const float t = fmaxf((d < 0 ? f.m[a] : f.p[a]) + (float)(abs(d) - 1) * f.h[a], 0.f);
  return t * t * (1.f - 4e-6f);
}

// ------------------------------------------------------------------------------ finalise

// Resolves a query item of a job into its point, grid and set.
// items [0, Q): forward queries in moving-grid order; [Q, Q + 2M): reverse queries
// (set 0 then set 1) in target-grid order.
struct QueryRef {
  float x, y, z;
  int id;    // Q index (forward) or target index (reverse)
  int set;   // grid set searched
  bool fwd;
};

__device__ __forceinline__ QueryRef resolve(const Job& J, int item) {
  QueryRef q;
  float4 p;
  if (item < J.Q) {
    p = J.mov.pts[item];
    q.fwd = true;
    q.set = 0;
  } else {
    const int r = item - J.Q;
    q.set = r >= J.M ? 1 : 0;
    p = J.tgt.pts[r - q.set * J.M];
    q.fwd = false;
  }
  q.x = p.x; q.y = p.y; q.z = p.z;
  q.id = __float_as_int(p.w);
  return q;
}

// The loss term phi(s) = s e^{-alpha s} and the gradient 2 phi'(s) (a - b) of a matched
// pair (Sec. 3.4); phi'(s) = e^{-alpha s}(1 - alpha s), or e^{-alpha s} with the stop-gradient.
template <bool COUNT>
__device__ __forceinline__ void finalize(const Job& J, const QueryRef& q, const Best& b) {
  if (COUNT && b.tie) atomicAdd(J.counters + CNT_NN_TIES, 1ull);
  if (b.idx == 0x7fffffff || !(b.d2 < FLT_MAX)) {  // nothing found (non-finite coordinates)
    if (q.fwd) {
      J.loss_fwd[q.id] = __int_as_float(0x7fc00000);
      J.gfwd[q.id] = make_float4(0.f, 0.f, 0.f, 0.f);
      J.nn_fwd[q.id] = -1;
    } else {
      J.loss_rev[q.set * J.M + q.id] = __int_as_float(0x7fc00000);
      J.nn_rev[q.set * J.M + q.id] = -1;
    }
    return;
  }
  const float s = b.d2;
  const float e = expf(-J.alpha * s);
  const float phi = s * e;
  const float dphi = J.stopgrad ? e : e * (1.f - J.alpha * s);
  if (q.fwd) {  // moving point a = q -> target point b
    const float4 t = J.tgt4[b.idx];
    const bool mesh = q.id < J.V;
    const float coef = 2.f * dphi * (mesh ? J.w_mesh / (float)J.V : J.w_pts / (float)(J.Q - J.V));
    J.loss_fwd[q.id] = phi;
    J.gfwd[q.id] = make_float4(coef * (q.x - t.x), coef * (q.y - t.y), coef * (q.z - t.z), 0.f);
    J.nn_fwd[q.id] = b.idx;
  } else {  // target point q -> moving point a of set q.set; the gradient goes to a
    const float4 a = J.y[b.idx];
    J.loss_rev[q.set * J.M + q.id] = phi;
    J.nn_rev[q.set * J.M + q.id] = b.idx - (q.set ? J.V : 0);
    const float c = 2.f * dphi;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(J.acc + 3 * (size_t)b.idx);
    atomicAdd(acc + 0, (unsigned long long)to_fx(c * (a.x - q.x)));
    atomicAdd(acc + 1, (unsigned long long)to_fx(c * (a.y - q.y)));
    atomicAdd(acc + 2, (unsigned long long)to_fx(c * (a.z - q.z)));
  }
}

// ------------------------------------------------------------------------------ shells

template <bool COUNT>
__device__ __forceinline__ void scan_range(const CellGrid& g, int s, int e, float qx, float qy, float qz, Best& b,
                                           int& nc) {
  if (COUNT) nc += e - s;
  for (int k = s; k < e; ++k) consider<COUNT>(b, __ldg(g.pts + k), qx, qy, qz);
}

// adds the candidate counts of the lanes of one job to its counter (counting instance)
__device__ __forceinline__ void count_candidates(const Job& J, int j, int nc) {
  const unsigned act = __activemask();
  const unsigned same = __match_any_sync(act, j);
  const unsigned s = __reduce_add_sync(same, (unsigned)nc);
  if ((threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(J.counters + CNT_NN_CANDIDATES, (unsigned long long)s);
}

// Candidates of row (dy, dz) of shell r around cell (cx, cy, cz): rows on the shell's
// y/z boundary over the x range [cx - r, cx + r], the others only at x = cx -/+ r.  Cells
// whose lower bound is above min(cap, best so far) are skipped (strictly above: an equal
// distance with a lower index must still be seen).
template <bool COUNT>
__device__ __forceinline__ void scan_shell_row(const CellGrid& g, int base, int G, int cx, int cy, int cz, int r,
                                               int dy, int dz, float qx, float qy, float qz, const FaceBounds& fb,
                                               float cap, Best& b, int& nc) {
  const int yy = cy + dy, zz = cz + dz;
  if (yy < 0 || yy >= G || zz < 0 || zz >= G) return;
  const float lim = fminf(cap, b.d2);
  const float lyz = axis_lb(fb, 1, dy) + axis_lb(fb, 2, dz);
  if (lyz > lim) return;
  const int rk = base + row_key(yy, zz, g.bits);
  if (max(abs(dy), abs(dz)) == r) {
    int x0 = max(cx - r, 0), x1 = min(cx + r, G - 1);
    while (x0 < cx && lyz + axis_lb(fb, 0, x0 - cx) > lim) ++x0;
    while (x1 > cx && lyz + axis_lb(fb, 0, x1 - cx) > lim) --x1;
    scan_range<COUNT>(g, __ldg(g.off + rk + x0), __ldg(g.off + rk + x1 + 1), qx, qy, qz, b, nc);
  } else {
    if (cx - r >= 0 && !(lyz + axis_lb(fb, 0, -r) > fminf(cap, b.d2)))
      scan_range<COUNT>(g, __ldg(g.off + rk + cx - r), __ldg(g.off + rk + cx - r + 1), qx, qy, qz, b, nc);
    if (cx + r < G && !(lyz + axis_lb(fb, 0, r) > fminf(cap, b.d2)))
      scan_range<COUNT>(g, __ldg(g.off + rk + cx + r), __ldg(g.off + rk + cx + r + 1), qx, qy, qz, b, nc);
  }
}

// ------------------------------------------------------------------------------ thread pass

template <bool COUNT>
__global__ void __launch_bounds__(256) k_nn(const Plan* __restrict__ P) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_NNQ][nj];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int j = find_job(P->pre[ST_NNQ], nj, it);
    const Job& J = *P->jobs[j];
    const int item = it - P->pre[ST_NNQ][j];
    const QueryRef q = resolve(J, item);
    const CellGrid& g = q.fwd ? J.tgt : J.mov;
    const int G = 1 << g.bits;
    const int base = q.set * G * G * G;
    const int cx = cell_coord(q.x, g.lo[0], g.inv_h[0], G);
    const int cy = cell_coord(q.y, g.lo[1], g.inv_h[1], G);
    const int cz = cell_coord(q.z, g.lo[2], g.inv_h[2], G);
    Best b{FLT_MAX, 0x7fffffff, false};
    int nc = 0;  // candidates evaluated (profiling)
    // warm start: the query's neighbour of the previous step (of this frame), at its current
    // position, compared with the same expression as every other candidate.  It is one of
    // the set's points, so the search below, which skips only cells that cannot hold a
    // distance <= the best, still ends at the exact lexicographic minimum; starting close to
    // it lets that pruning work from the first cell.
    {
      const int w = q.fwd ? J.nn_fwd[q.id] : J.nn_rev[q.set * J.M + q.id];
      if (w >= 0) {
        const int gid = q.fwd ? w : w + (q.set ? J.V : 0);
        const float4 p = q.fwd ? J.tgt4[w] : J.y[gid];
        b.d2 = sqdist(q.x, q.y, q.z, p.x, p.y, p.z);
        b.idx = gid;
      }
    }
    // ring 1: the 3x3x3 box, the query's own cell first.  A neighbouring cell is skipped
    // when a lower bound on the squared distance to anything assigned to it is already above
    // the best one: it can hold neither the minimum nor an equal distance with a lower index.
    const FaceBounds fb = face_bounds(g, q.x, q.y, q.z, cx, cy, cz);
    {
      int rk = base + row_key(cy, cz, g.bits);
      scan_range<COUNT>(g, __ldg(g.off + rk + cx), __ldg(g.off + rk + cx + 1), q.x, q.y, q.z, b, nc);
      if (cx > 0 && !(axis_lb(fb, 0, -1) > b.d2))
        scan_range<COUNT>(g, __ldg(g.off + rk + cx - 1), __ldg(g.off + rk + cx), q.x, q.y, q.z, b, nc);
      if (cx < G - 1 && !(axis_lb(fb, 0, 1) > b.d2))
        scan_range<COUNT>(g, __ldg(g.off + rk + cx + 1), __ldg(g.off + rk + cx + 2), q.x, q.y, q.z, b, nc);
      // the other 8 x-rows: the 4 sharing a face with the query's row, then the 4 diagonal
      for (int k = 0; k < 8; ++k) {
        int dy, dz;
        if (k < 4) {
          dy = k < 2 ? (k & 1 ? 1 : -1) : 0;
          dz = k < 2 ? 0 : (k & 1 ? 1 : -1);
        } else {
          dy = k & 1 ? 1 : -1;
          dz = k & 2 ? 1 : -1;
        }
        const int yy = cy + dy, zz = cz + dz;
        if (yy < 0 || yy >= G || zz < 0 || zz >= G) continue;
        const float lyz = axis_lb(fb, 1, dy) + axis_lb(fb, 2, dz);
        if (lyz > b.d2) continue;
        const int x0 = cx > 0 && !(lyz + axis_lb(fb, 0, -1) > b.d2) ? cx - 1 : cx;
        const int x1 = cx < G - 1 && !(lyz + axis_lb(fb, 0, 1) > b.d2) ? cx + 1 : cx;
        rk = base + row_key(yy, zz, g.bits);
        scan_range<COUNT>(g, __ldg(g.off + rk + x0), __ldg(g.off + rk + x1 + 1), q.x, q.y, q.z, b, nc);
      }
    }
    int r = 1;
    bool done = b.d2 < outside_bound2(g, q.x, q.y, q.z, cx, cy, cz, 1);
    while (!done && r < NN_RTHREAD) {
      ++r;
      for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
          scan_shell_row<COUNT>(g, base, G, cx, cy, cz, r, dy, dz, q.x, q.y, q.z, fb, FLT_MAX, b, nc);
      done = b.d2 < outside_bound2(g, q.x, q.y, q.z, cx, cy, cz, r);
    }
    if (COUNT) count_candidates(J, j, nc);
    if (done) {
      finalize<COUNT>(J, q, b);
    } else {  // ring reached in the low 16 bits, the tie flag above them
      const int slot = atomicAdd(J.hard_count, 1);
      J.hard[slot] = make_int4(item, r | (COUNT && b.tie ? 0x10000 : 0), __float_as_int(b.d2), b.idx);
    }
  }
}

// ------------------------------------------------------------------------------ warp pass

__device__ __forceinline__ unsigned long long pack(const Best& b) {
  return ((unsigned long long)__float_as_uint(b.d2) << 32) | (unsigned)b.idx;
}

// lexicographic (d2, idx) minimum over the warp; every lane receives it
template <bool COUNT>
__device__ __forceinline__ Best warp_min(const Best& b) {
  unsigned long long m = pack(b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t < m ? t : m;
  }
  Best r;
  r.d2 = __uint_as_float((unsigned)(m >> 32));
  r.idx = (int)(unsigned)(m & 0xffffffffu);
  // an exact tie: a lane saw a tie at the minimum, or another lane's best has the same
  // distance with another index
  r.tie = COUNT && __any_sync(0xffffffffu, b.d2 == r.d2 && (b.tie || b.idx != r.idx));
  return r;
}

template <bool COUNT>
__global__ void __launch_bounds__(256) k_nn_hard(const Plan* __restrict__ P) {
  __shared__ int hpre[MAXJ + 1];
  const int nj = P->n_jobs;
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int j = 0; j < nj; ++j) {
      hpre[j] = acc;
      acc += *P->jobs[j]->hard_count;
    }
    hpre[nj] = acc;
    if (blockIdx.x == 0)
      for (int j = 0; j < nj; ++j) P->jobs[j]->counters[CNT_NN_HARD] = (unsigned long long)(hpre[j + 1] - hpre[j]);
  }
  __syncthreads();
  const int total = hpre[nj];
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nwarps) {
    int lo = 0, hi = nj;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (hpre[mid] <= w) lo = mid; else hi = mid;
    }
    const Job& J = *P->jobs[lo];
    const int4 h = J.hard[w - hpre[lo]];
    const QueryRef q = resolve(J, h.x);
    const CellGrid& g = q.fwd ? J.tgt : J.mov;
    const int G = 1 << g.bits;
    const int base = q.set * G * G * G;
    const int cx = cell_coord(q.x, g.lo[0], g.inv_h[0], G);
    const int cy = cell_coord(q.y, g.lo[1], g.inv_h[1], G);
    const int cz = cell_coord(q.z, g.lo[2], g.inv_h[2], G);
    const FaceBounds fb = face_bounds(g, q.x, q.y, q.z, cx, cy, cz);
    // continue from the thread pass: its best is lane 0's starting candidate, and the best
    // of the warp after each ring bounds what every lane still has to look at
    Best b{FLT_MAX, 0x7fffffff, false};
    if (lane == 0) {
      b.d2 = __int_as_float(h.z);
      b.idx = h.w;
      b.tie = (h.y & 0x10000) != 0;
    }
    Best best{__int_as_float(h.z), h.w, false};
    bool done = false;
    int nc = 0;
    for (int r = (h.y & 0xffff) + 1; r <= NN_RMAX && !done; ++r) {
      const int side = 2 * r + 1;
      for (int ri = lane; ri < side * side; ri += 32)
        scan_shell_row<COUNT>(g, base, G, cx, cy, cz, r, ri % side - r, ri / side - r, q.x, q.y, q.z, fb, best.d2,
                              b, nc);
      best = warp_min<COUNT>(b);
      done = best.d2 < outside_bound2(g, q.x, q.y, q.z, cx, cy, cz, r);
    }
    if (!done) {  // exhaustive scan of the set
      const int s = __ldg(g.off + base), e = __ldg(g.off + base + G * G * G);
      for (int k = s + lane; k < e; k += 32) consider<COUNT>(b, __ldg(g.pts + k), q.x, q.y, q.z);
      if (COUNT) nc += (e - s + 31 - lane) / 32;
      best = warp_min<COUNT>(b);
    }
    if (COUNT) {
      const unsigned s = __reduce_add_sync(0xffffffffu, (unsigned)nc);
      if (lane == 0) atomicAdd(J.counters + CNT_NN_CANDIDATES, (unsigned long long)s);
    }
    if (lane == 0) finalize<COUNT>(J, q, best);
  }
}

void launch_nn(const Plan* P, int grid, cudaStream_t s, bool count) {
  if (count) k_nn<true><<<grid, 256, 0, s>>>(P);
  else k_nn<false><<<grid, 256, 0, s>>>(P);
}
void launch_nn_hard(const Plan* P, int grid, cudaStream_t s, bool count) {
  if (count) k_nn_hard<true><<<grid, 256, 0, s>>>(P);
  else k_nn_hard<false><<<grid, 256, 0, s>>>(P);
}

}  // namespace pdg
