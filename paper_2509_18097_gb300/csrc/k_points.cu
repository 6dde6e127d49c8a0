// Point- and edge-parallel kernels of the step: the plan, multi-level trilinear
// evaluation (Eq. 1), the moving-set cell keys, edge isometry (Sec. 3.4), gradient
// assembly and the loss reduction; plus the per-frame set-up kernels.
#include "kernels.h"

namespace pdg {

// ------------------------------------------------------------------------------ plan

// Start of a step for one job, done by the thread of the job's first point in k_interp.
// bump = 1: a new optimisation step (advances the Adam step count and its bias corrections
// and clears the per-step counters); bump = 2: an evaluation (clears the counters only).
__device__ __forceinline__ void job_bump(const Job& J, int bump) {
  *J.hard_count = 0;
  *J.gmax = 0u;
  J.counters[CNT_NN_CANDIDATES] = 0ull;
  J.counters[CNT_NN_TIES] = 0ull;
  J.counters[CNT_NN_HARD] = 0ull;
  if (bump == 1) {
    const int k = *J.step + 1;
    *J.step = k;
    // 1 - beta^k = -expm1(k log1p(beta - 1)): no cancellation for small k (beta - 1 is exact)
    J.bias[0] = 1.f / -expm1f((float)k * log1pf(J.beta1 - 1.f));
    J.bias[1] = rsqrtf(-expm1f((float)k * log1pf(J.beta2 - 1.f)));
  }
}

// Computes, on the device, the per-stage item prefixes over the jobs of a plan.  They change
// only when a job starts a frame (its active-vertex counts) or the membership changes, so
// the host launches this outside the per-step graph, when the plan is stale.  One block.
__global__ void k_plan(Plan* P) {
  __shared__ int cnt[NSTAGE][MAXJ];
  const int nj = P->n_jobs;
  for (int j = threadIdx.x; j < nj; j += blockDim.x) {
    Job* J = P->jobs[j];
    const int G = 1 << J->mov.bits;
    cnt[ST_Q][j] = J->Q;
    // reverse queries into the source set only when there is one (a template-mesh fit has none)
    const int nrs = J->N > 0 ? 2 : 1;
    cnt[ST_NNQ][j] = J->Q + nrs * J->M;
    cnt[ST_E][j] = J->E;
    cnt[ST_MOVCH][j] = (2 * G * G * G + SCAN_CHUNK - 1) / SCAN_CHUNK;
    int a = 0, t = 0, p3 = 0, cols = 0, ad = 0;
    int aw = 0;
    // the levels' loads are independent: issue them level-parallel (a dependent chain of
    // global loads per level would put a dozen memory latencies on the step's critical path)
    const int L = J->L;
    int na_l[MAXL], ne_l[MAXL];
#pragma unroll
    for (int l = 0; l < MAXL; ++l) na_l[l] = l < L ? *J->lev[l].n_active : 0;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) ne_l[l] = na_l[l] > 0 ? J->lev[l].act_ptr[na_l[l]] : 0;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
      if (l >= L) break;
      // adjoint (in blocks of 8 warps): 2^adj_lg lanes per row, 8 to 16 entries per lane
      // (a row holds one entry per point in the 8 cells around its vertex: a few dozen on
      // fine levels, thousands on coarse ones), so a warp sums 32 >> adj_lg rows; rows of
      // 512 entries or more on average (adj_lg = 6) get a whole block each
      Level& lv = J->lev[l];
      const int na = na_l[l];
      const int ne = ne_l[l];
      const int avg = ne / max(na, 1);
      int lg = 0;
      while (lg < 6 && (16 << lg) <= avg) ++lg;
      lv.adj_lg = lg;
      if (lg == 6) a += na;
      else aw += (na + (32 >> lg) - 1) >> (5 - lg);
      if (tile_level(J->lev[l].n)) t += J->lev[l].tiles;
      else {
        p3 += J->lev[l].n;
        cols += J->C * ((J->lev[l].n * J->lev[l].n + 63) / 64);  // blocks of 64 columns (two threads each)
        ad += (J->lev[l].n3 + 3) >> 2;
      }
    }
    cnt[ST_ADJ][j] = a + ((aw + 7) >> 3);
    cnt[ST_TILE][j] = t;
    cnt[ST_PLANE][j] = J->C * p3;
    cnt[ST_COL][j] = cols;
    cnt[ST_ADAM][j] = ad;
    cnt[ST_JOB][j] = 1;
    cnt[ST_LOSSCH][j] = (J->Q + nrs * J->M + J->E + LOSS_CHUNK - 1) / LOSS_CHUNK;
  }
  __syncthreads();
  if (threadIdx.x < NSTAGE) {
    const int s = threadIdx.x;
    int acc = 0;
    P->pre[s][0] = 0;
    for (int j = 0; j < nj; ++j) {
      acc += cnt[s][j];
      P->pre[s][j + 1] = acc;
    }
  }
}

// ------------------------------------------------------------------------------ (a) eval

// Trilinear interpolation of one level's values at a point (Eq. 1; vertex-aligned levels,
// coordinates clamped to the domain, last cell closed): the cell's first vertex and the
// fractional coordinates, computed once and used for each payload array of the level.  A
// level of one vertex has the constant value v[0].
struct LevelCoord {
  int base;  // flat index of the cell's (0, 0, 0) corner
  int n;
  float fx, fy, fz;
};

__device__ __forceinline__ LevelCoord level_coord(const Job& J, const Level& lv, float px, float py, float pz) {
  LevelCoord c;
  c.n = lv.n;
  if (lv.n == 1) {
    c.base = 0;
    c.fx = c.fy = c.fz = 0.f;
    return c;
  }
  int ix, iy, iz;
  grid_coord(px, J.lo[0], lv.sc_hi[0], lv.sc_lo[0], lv.n, ix, c.fx);
  grid_coord(py, J.lo[1], lv.sc_hi[1], lv.sc_lo[1], lv.n, iy, c.fy);
  grid_coord(pz, J.lo[2], lv.sc_hi[2], lv.sc_lo[2], lv.n, iz, c.fz);
  c.base = (iz * lv.n + iy) * lv.n + ix;
  return c;
}

// adds sum_corners w * v[corner] to u (all 8 corner loads issued before any is used)
__device__ __forceinline__ void level_add(const LevelCoord& L, const float4* __restrict__ v, float& ux, float& uy,
                                          float& uz) {
  if (L.n == 1) {
    const float4 c = v[0];
    ux += c.x; uy += c.y; uz += c.z;
    return;
  }
  const int n = L.n;
  const float4* t0 = v + L.base;
  const float4* t1 = t0 + (size_t)n * n;
  const float4 c000 = t0[0], c100 = t0[1], c010 = t0[n], c110 = t0[n + 1];
  const float4 c001 = t1[0], c101 = t1[1], c011 = t1[n], c111 = t1[n + 1];
  const float fx = L.fx, fy = L.fy, fz = L.fz;
  const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
  const float w000 = gx * gy * gz, w100 = fx * gy * gz, w010 = gx * fy * gz, w110 = fx * fy * gz;
  const float w001 = gx * gy * fz, w101 = fx * gy * fz, w011 = gx * fy * fz, w111 = fx * fy * fz;
  ux += w000 * c000.x + w100 * c100.x + w010 * c010.x + w110 * c110.x + w001 * c001.x + w101 * c101.x +
        w011 * c011.x + w111 * c111.x;
  uy += w000 * c000.y + w100 * c100.y + w010 * c010.y + w110 * c110.y + w001 * c001.y + w101 * c101.y +
        w011 * c011.y + w111 * c111.y;
  uz += w000 * c000.z + w100 * c100.z + w010 * c010.z + w110 * c110.z + w001 * c001.z + w101 * c101.z +
        w011 * c011.z + w111 * c111.z;
}

// The payload averaged over the levels at p (Eq. 1): a = the displacement (or z of the
// Cayley payload), t = the Cayley translation (zero for the displacement payload)
__device__ void eval_payload(const Job& J, float px, float py, float pz, float3& a, float3& t) {
  float ax = 0.f, ay = 0.f, az = 0.f, tx = 0.f, ty = 0.f, tz = 0.f;
  for (int l = 0; l < J.L; ++l) {
    const Level& lv = J.lev[l];
    const LevelCoord c = level_coord(J, lv, px, py, pz);
    level_add(c, lv.theta, ax, ay, az);
    if (J.C == 6) level_add(c, lv.theta_t, tx, ty, tz);
  }
  const float invL = 1.f / (float)J.L;
  a = make_float3(ax * invL, ay * invL, az * invL);
  t = make_float3(tx * invL, ty * invL, tz * invL);
}

// the deformed position of x (Sec. 3.3): x + u(x), or R(z(x)) x + t(x) with the Cayley
// payload (then also z and u = (I - Z)^{-1} x for the backward)
__device__ __forceinline__ float3 deform_point(const Job& J, float3 x, float3& z, float3& u) {
  float3 a, t;
  eval_payload(J, x.x, x.y, x.z, a, t);
  if (J.C != 6) return make_float3(x.x + a.x, x.y + a.y, x.z + a.z);
  z = a;
  u = cayley_u(z, x);
  return make_float3(2.f * u.x - x.x + t.x, 2.f * u.y - x.y + t.y, 2.f * u.z - x.z + t.z);
}

// y = x + u(x) on Q; the cell key of y in the moving grid (set 0: template, set 1: source)
// and its count; clears the point's fixed-point reverse-Chamfer accumulator.  The thread of
// a job's first point also starts the job's step (job_bump; bump 0: none).  Points are taken
// in the finest level's cell order (the per-frame sort of the adjoint), so the lanes of a
// warp interpolate between the same or neighbouring grid vertices.
__global__ void k_interp(const Plan* __restrict__ P, int bump) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_Q][nj];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int j = find_job(P->pre[ST_Q], nj, it);
    const Job& J = *P->jobs[j];
    const int p = __float_as_int(__ldg(&J.lev[J.L - 1].xs[it - P->pre[ST_Q][j]].w));
    if (bump && p == 0) job_bump(J, bump);
    const float4 x = J.x[p];
    float3 z, u;
    const float3 yy = deform_point(J, make_float3(x.x, x.y, x.z), z, u);
    const float4 y = make_float4(yy.x, yy.y, yy.z, 0.f);
    J.y[p] = y;
    if (J.C == 6) {
      J.zq[p] = make_float4(z.x, z.y, z.z, 0.f);
      J.uq[p] = make_float4(u.x, u.y, u.z, 0.f);
    }
    const int key = cell_key(J.mov, y.x, y.y, y.z, p < J.V ? 0 : 1);
    J.mov.keys[p] = key;
    atomicAdd(&J.mov.hist[key], 1);
    J.acc[3 * p + 0] = 0;
    J.acc[3 * p + 1] = 0;
    J.acc[3 * p + 2] = 0;
  }
}

// scatter of the moving points into key order (counts return to zero)
__global__ void k_mov_scatter(const Plan* __restrict__ P) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_Q][nj];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int j = find_job(P->pre[ST_Q], nj, it);
    const Job& J = *P->jobs[j];
    const int p = it - P->pre[ST_Q][j];
    const int key = J.mov.keys[p];
    const int pos = J.mov.off[key] + atomicSub(&J.mov.hist[key], 1) - 1;
    const float4 y = J.y[p];
    J.mov.pts[pos] = make_float4(y.x, y.y, y.z, __int_as_float(p));
  }
}

// ------------------------------------------------------------------------------ (c) isometry

// |a - b| with explicit rounding so every kernel computes it bit-identically
__device__ __forceinline__ float edge_len(float4 a, float4 b) {
  return __fsqrt_rn(sqdist(a.x, a.y, a.z, b.x, b.y, b.z));
}

// per edge: |r| with r = |y_i - y_j| - e_prev, and sgn(r)(y_i - y_j)/(|y_i - y_j| |E|)
// (Sec. 3.4; sgn(0) = 0, zero-length edges contribute no gradient)
__global__ void k_iso_edges(const Plan* __restrict__ P) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_E][nj];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int j = find_job(P->pre[ST_E], nj, it);
    const Job& J = *P->jobs[j];
    const int e = it - P->pre[ST_E][j];
    const int2 ij = J.edges[e];
    const float4 a = J.y[ij.x], b = J.y[ij.y];
    const float len = edge_len(a, b);
    const float r = len - J.e_prev[e];
    J.loss_iso[e] = fabsf(r);
    float c = 0.f;
    if (len > 0.f && r != 0.f) c = copysignf(1.f, r) / (len * (float)J.E);
    J.edge_d[e] = make_float4(c * (a.x - b.x), c * (a.y - b.y), c * (a.z - b.z), 0.f);
  }
}

// dLoss/dy = forward Chamfer term + (w/M) * reverse Chamfer sums + w_iso * isometry
// gradient gathered over the vertex's edges in a fixed order.
__global__ void k_assemble(const Plan* __restrict__ P) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_Q][nj];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int j = find_job(P->pre[ST_Q], nj, it);
    const Job& J = *P->jobs[j];
    const int p = it - P->pre[ST_Q][j];
    float4 g = J.gfwd[p];
    const float wr = (p < J.V ? J.w_mesh : J.w_pts) / (float)J.M;
    g.x += wr * from_fx(J.acc[3 * p + 0]);
    g.y += wr * from_fx(J.acc[3 * p + 1]);
    g.z += wr * from_fx(J.acc[3 * p + 2]);
    if (p < J.V && J.w_iso != 0.f) {
      float ix = 0.f, iy = 0.f, iz = 0.f;
      for (int k = J.v2e_ptr[p]; k < J.v2e_ptr[p + 1]; ++k) {
        const int ent = J.v2e[k];
        const float4 d = J.edge_d[ent >> 1];
        if (ent & 1) { ix -= d.x; iy -= d.y; iz -= d.z; }
        else { ix += d.x; iy += d.y; iz += d.z; }
      }
      g.x += J.w_iso * ix;
      g.y += J.w_iso * iy;
      g.z += J.w_iso * iz;
    }
    J.gy[p] = g;
    float gm = fmaxf(fabsf(g.x), fmaxf(fabsf(g.y), fabsf(g.z)));
    if (J.C == 6) {  // the point's gradient with respect to its averaged Cayley z
      const float4 z4 = J.zq[p], u4 = J.uq[p];
      const float3 gzv = cayley_grad_z(make_float3(z4.x, z4.y, z4.z), make_float3(u4.x, u4.y, u4.z),
                                       make_float3(g.x, g.y, g.z));
      J.gz[p] = make_float4(gzv.x, gzv.y, gzv.z, 0.f);
      gm = fmaxf(gm, fmaxf(fabsf(gzv.x), fmaxf(fabsf(gzv.y), fabsf(gzv.z))));
    }
    // running bound on the point gradients of the job (order-independent max, one atomic per
    // job per warp); it sets the adjoint's fixed-point scale
    unsigned bits = __float_as_uint(gm);
    if (!(gm <= 3.0e38f)) bits = 0x7f800000u;
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, j);
    const unsigned m = __reduce_max_sync(same, bits);
    if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMax(J.gmax, m);
  }
}

// ------------------------------------------------------------------------------ loss

// Loss record.  The per-query and per-edge terms of a job form one virtual array
// [phi fwd (Q) | phi rev set 0 (M) | phi rev set 1 (M, if N > 0) | |r| (E)], cut into fixed chunks of
// LOSS_CHUNK; each chunk is summed by one block in a fixed fp32 tree per term, and a second
// kernel adds a job's chunk partials in order in FP64.  The partition depends only on the
// job, so a job's loss is bitwise the same alone or in a batch.
__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  if (w == 0) {
    t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(256) k_loss_chunks(const Plan* __restrict__ P) {
  __shared__ float red[32];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_LOSSCH][nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_LOSSCH], nj, it);
    const Job& J = *P->jobs[j];
    const int c = it - P->pre[ST_LOSSCH][j];
    const int b0 = c * LOSS_CHUNK;
    const int Q = J.Q, V = J.V, M = J.M;
    const int rev_end = Q + (J.N > 0 ? 2 : 1) * M;
    const int n_all = rev_end + J.E;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
    for (int i = b0 + threadIdx.x; i < min(b0 + LOSS_CHUNK, n_all); i += blockDim.x) {
      if (i < V) s0 += J.loss_fwd[i];
      else if (i < Q) s1 += J.loss_fwd[i];
      else if (i < Q + M) s2 += J.loss_rev[i - Q];
      else if (i < rev_end) s3 += J.loss_rev[i - Q];
      else s4 += J.loss_iso[i - rev_end];
    }
    const float t0 = block_sum(s0, red), t1 = block_sum(s1, red), t2 = block_sum(s2, red);
    const float t3 = block_sum(s3, red), t4 = block_sum(s4, red);
    if (threadIdx.x == 0) {
      float* o = J.loss_part + 5 * c;
      o[0] = t0; o[1] = t1; o[2] = t2; o[3] = t3; o[4] = t4;
    }
  }
}

__global__ void __launch_bounds__(256) k_loss_final(const Plan* __restrict__ P) {
  __shared__ float red[32];
  const int nj = P->n_jobs;
  for (int j = blockIdx.x; j < nj; j += gridDim.x) {
    const Job& J = *P->jobs[j];
    const int nch = (J.Q + (J.N > 0 ? 2 : 1) * J.M + J.E + LOSS_CHUNK - 1) / LOSS_CHUNK;
    float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
#pragma unroll
      for (int k = 0; k < 5; ++k) s[k] += J.loss_part[5 * c + k];
    }
    double t[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) t[k] = (double)block_sum(s[k], red);  // all terms are >= 0
    if (threadIdx.x == 0) {
      const double cdm = t[0] / J.V + t[2] / J.M;
      const double cdp = J.N > 0 ? t[1] / (J.Q - J.V) + t[3] / J.M : 0.0;
      const double iso = J.E > 0 ? t[4] / J.E : 0.0;
      const double tot = (double)J.w_mesh * cdm + (double)J.w_pts * cdp + (double)J.w_iso * iso;
      J.loss[0] = tot;
      J.loss[1] = cdm;
      J.loss[2] = cdp;
      J.loss[3] = iso;
      if (!isfinite(tot)) *J.status |= 1;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ per frame

__global__ void k_pack4(const float* __restrict__ in, float4* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = make_float4(in[3 * i], in[3 * i + 1], in[3 * i + 2], 0.f);
}

__global__ void k_unpack4(const float4* __restrict__ in, float* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 v = in[i];
    out[3 * i] = v.x;
    out[3 * i + 1] = v.y;
    out[3 * i + 2] = v.z;
  }
}

__global__ void k_check_finite(const float* __restrict__ in, int n, int* flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (!isfinite(in[i])) atomicOr(flag, 1);
}

// Q = X_{t-1} u P_{t-1}; rest lengths e_prev from X_{t-1} (same expression as k_iso_edges
// so that zero grids give r == 0 exactly).
__global__ void k_frame_points(Job* J) {
  const int Q = J->Q, V = J->V;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < Q; p += gridDim.x * blockDim.x)
    J->x[p] = p < V ? J->verts4[p] : J->src4[p - V];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < J->E; e += gridDim.x * blockDim.x) {
    const int2 ij = J->edges[e];
    J->e_prev[e] = edge_len(J->verts4[ij.x], J->verts4[ij.y]);
  }
}

__global__ void k_tgt_keys(Job* J) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J->M; p += gridDim.x * blockDim.x) {
    const float4 t = J->tgt4[p];
    const int key = cell_key(J->tgt, t.x, t.y, t.z, 0);
    J->tgt.keys[p] = key;
    atomicAdd(&J->tgt.hist[key], 1);
  }
}

__global__ void k_tgt_scatter(Job* J) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J->M; p += gridDim.x * blockDim.x) {
    const int key = J->tgt.keys[p];
    const int pos = J->tgt.off[key] + atomicSub(&J->tgt.hist[key], 1) - 1;
    const float4 t = J->tgt4[p];
    J->tgt.pts[pos] = make_float4(t.x, t.y, t.z, __int_as_float(p));
  }
}

// frame end: X_t = M(T_t(X_{t-1})) X_{t-1} with the final grids (Sec. 3.3)
__global__ void k_end_frame(Job* J) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J->V; p += gridDim.x * blockDim.x) {
    const float4 x = J->x[p];
    float3 z, u;
    const float3 y = deform_point(*J, make_float3(x.x, x.y, x.z), z, u);
    J->verts4[p] = make_float4(y.x, y.y, y.z, 0.f);
  }
}

// the frame's deformation applied to arbitrary points ([n][3] float in/out, device)
__global__ void k_deform(const Job* __restrict__ J, const float* __restrict__ in, float* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float3 z, u;
    const float3 y = deform_point(*J, make_float3(in[3 * i], in[3 * i + 1], in[3 * i + 2]), z, u);
    out[3 * i] = y.x;
    out[3 * i + 1] = y.y;
    out[3 * i + 2] = y.z;
  }
}

// ------------------------------------------------------------------------------ launchers

static inline int blocks_for(int n, int threads) { return max(1, min((n + threads - 1) / threads, 4096)); }

void launch_plan(Plan* P, cudaStream_t s) { k_plan<<<1, 256, 0, s>>>(P); }
void launch_interp(const Plan* P, int grid, cudaStream_t s, int bump) { k_interp<<<grid, 256, 0, s>>>(P, bump); }
void launch_mov_scatter(const Plan* P, int grid, cudaStream_t s) { k_mov_scatter<<<grid, 256, 0, s>>>(P); }
void launch_iso_edges(const Plan* P, int grid, cudaStream_t s) { k_iso_edges<<<grid, 256, 0, s>>>(P); }
void launch_assemble(const Plan* P, int grid, cudaStream_t s) { k_assemble<<<grid, 256, 0, s>>>(P); }
void launch_loss(const Plan* P, int grid, cudaStream_t s) {
  k_loss_chunks<<<grid, 256, 0, s>>>(P);
  k_loss_final<<<MAXJ, 256, 0, s>>>(P);
}

void launch_pack4(const float* in, float4* out, int n, cudaStream_t s) {
  k_pack4<<<blocks_for(n, 256), 256, 0, s>>>(in, out, n);
}
void launch_unpack4(const float4* in, float* out, int n, cudaStream_t s) {
  k_unpack4<<<blocks_for(n, 256), 256, 0, s>>>(in, out, n);
}
void launch_check_finite(const float* in, int n, int* flag, cudaStream_t s) {
  k_check_finite<<<blocks_for(n, 256), 256, 0, s>>>(in, n, flag);
}
void launch_frame_points(Job* J, int Q, int E, cudaStream_t s) {
  k_frame_points<<<blocks_for(max(Q, E), 256), 256, 0, s>>>(J);
}
void launch_end_frame(Job* J, int V, cudaStream_t s) { k_end_frame<<<blocks_for(V, 256), 256, 0, s>>>(J); }
void launch_deform(const Job* J, const float* in, float* out, int n, cudaStream_t s) {
  k_deform<<<blocks_for(n, 256), 256, 0, s>>>(J, in, out, n);
}

// channel-planar [C][n3] <-> interleaved [n3][C]
__global__ void k_soa_to_aos(const float* __restrict__ in, float* __restrict__ out, int n3, int C) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x)
    for (int c = 0; c < C; ++c) out[(size_t)C * i + c] = in[(size_t)c * n3 + i];
}
__global__ void k_aos_to_soa(const float* __restrict__ in, float* __restrict__ out, int n3, int C) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x)
    for (int c = 0; c < C; ++c) out[(size_t)c * n3 + i] = in[(size_t)C * i + c];
}
void launch_aos_to_soa(const float* in, float* out, int n3, cudaStream_t s, int C) {
  k_aos_to_soa<<<blocks_for(n3, 256), 256, 0, s>>>(in, out, n3, C);
}
void launch_soa_to_aos(const float* in, float* out, int n3, cudaStream_t s, int C) {
  k_soa_to_aos<<<blocks_for(n3, 256), 256, 0, s>>>(in, out, n3, C);
}

// level values [n3][C] <-> the float4 arrays of a level (theta; theta_t holds channels 3..5)
__global__ void k_pack_theta(const float* __restrict__ in, float4* __restrict__ th, float4* __restrict__ tht, int n3,
                             int C) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
    const float* r = in + (size_t)C * i;
    th[i] = make_float4(r[0], r[1], r[2], 0.f);
    if (C == 6) tht[i] = make_float4(r[3], r[4], r[5], 0.f);
  }
}
__global__ void k_unpack_theta(const float4* __restrict__ th, const float4* __restrict__ tht, float* __restrict__ out,
                               int n3, int C) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
    float* r = out + (size_t)C * i;
    const float4 a = th[i];
    r[0] = a.x; r[1] = a.y; r[2] = a.z;
    if (C == 6) {
      const float4 b = tht[i];
      r[3] = b.x; r[4] = b.y; r[5] = b.z;
    }
  }
}
void launch_pack_theta(const float* in, float4* th, float4* tht, int n3, int C, cudaStream_t s) {
  k_pack_theta<<<blocks_for(n3, 256), 256, 0, s>>>(in, th, tht, n3, C);
}
void launch_unpack_theta(const float4* th, const float4* tht, float* out, int n3, int C, cudaStream_t s) {
  k_unpack_theta<<<blocks_for(n3, 256), 256, 0, s>>>(th, tht, out, n3, C);
}

__global__ void k_copy_int(const int* __restrict__ in, int* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = in[i];
}
void launch_aos_to_float4(const float* in, float4* out, int n, cudaStream_t s) { launch_pack4(in, out, n, s); }
void launch_copy_int(const int* in, int* out, int n, cudaStream_t s) {
  k_copy_int<<<blocks_for(n, 256), 256, 0, s>>>(in, out, n);
}

// target cell grid of the frame: keys + counts, exclusive scan, scatter
void launch_tgt_build(Job* J, const Job& hJ, cudaStream_t s) {
  k_tgt_keys<<<blocks_for(hJ.M, 256), 256, 0, s>>>(J);
  const int G = 1 << hJ.tgt.bits;
  ScanSeg seg{hJ.tgt.hist, hJ.tgt.off, G * G * G, hJ.tgt.csum};
  launch_scan_segments(&seg, 1, nullptr, nullptr, s);
  k_tgt_scatter<<<blocks_for(hJ.M, 256), 256, 0, s>>>(J);
}

}  // namespace pdg
