// Internal device-side data structures and helpers shared by the kernels and the host
// runtime of libpdg (Preconditioned Deformation Grids, arXiv 2509.18097).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pdg.h"

namespace pdg {

constexpr int MAXJ = 256;            // jobs (contexts) per batch
constexpr int MAXL = PDG_MAX_LEVELS; // grid levels
constexpr int SCAN_CHUNK = 4096;     // elements per scan chunk (1024 threads x 4)
constexpr int SCAN_THREADS = 1024;
constexpr int TILE_LINES = 32;       // lines per Sobolev tile (per channel)
constexpr int SOB_WARPS = 8;
constexpr int SOB_THREADS = SOB_WARPS * 32;
constexpr int NN_RMAX = 8;           // ring radius after which a query is searched exhaustively
constexpr int NN_RTHREAD = 2;        // rings searched by the one-thread-per-query pass
constexpr int LOSS_CHUNK = 2048;     // elements per loss-reduction chunk
constexpr double FX_SCALE = 1099511627776.0;  // 2^40: fixed-point scale of the reverse Chamfer sums

// A uniform cell grid over the domain used by the exact nearest-neighbour search.
// G = 2^bits cells per axis.  Keys are (interleave(cy, cz) << bits) | cx, so the cells of
// one x-row are contiguous and rows follow a 2-D Morton order in (y, z).  A grid may hold
// `nsets` point sets in one key space (set s occupies keys [s G^3, (s+1) G^3)).
struct CellGrid {
  int bits;
  int nsets;
  float lo[3];
  float inv_h[3];  // G / (hi - lo)
  float h[3];      // (hi - lo) / G
  int* hist;       // [nsets G^3] per-cell counts; all zero between builds
  int* off;        // [nsets G^3 + 1] exclusive prefix of hist
  int* keys;       // [points] key of each point (scratch of the build)
  float4* pts;     // [points] points sorted by key; .w = original index (int bits)
  int* csum;       // scan chunk sums scratch
};

struct Level {
  int n;       // vertices per axis (1 or a power of two)
  int lg;      // log2(n)
  int n3;      // n^3
  int tiles;   // tile-path Sobolev tiles: 3 channels x ceil(n^2 / 32) lines of 32
  float sc_hi[3], sc_lo[3];  // (n - 1) / (hi - lo) per axis as a float pair (hi + lo)
  float lr;    // learning rate of the level (already x0.1 without preconditioning)
  float lam;   // lambda of the level
  float4* theta;  // [n3] values (x, y, z, 0): the displacement, or z of the Cayley payload
  float4* theta_t;  // [n3] translation t of the Cayley payload (null for the displacement payload)
  float* m;       // [C][n3] Adam first moment (channel-planar; C = 3, or 6: z then t)
  float* v;       // [C][n3] Adam second moment
  float* g;       // [C][n3] dLoss/dTheta (zero at vertices no point touches)
  float* tmp;     // [C][n3] spectral work array (and preconditioned gradient in debug mode)
  int* zmask;     // [n] 1 for z-planes that hold an active vertex (per frame); null: all planes
  float* piv;     // [(n/2 + 1) n^2] pivots of the z-direction twisted solves (n <= 128), per context
  int* piv_slow;  // device flag: some pivot past the first 16 differs from the limit (no register path)
  float* mu;      // [n] eigenvalues 4 sin^2(pi k / 2n) of the 1-D path Laplacian
  float2* tw;     // [n] FFT twiddles exp(-2 pi i k / n)
  float2* tw4;    // [n] DCT twiddles exp(-i pi k / 2n)
  // point -> vertex interpolation lists, built once per frame (x is fixed in a frame)
  int* cnt;       // [n3] per-vertex entry counts (zero between builds)
  int* rowptr;    // [n3 + 1]
  int* flag;      // [n3 + 1] active-vertex flags, then their exclusive prefix
  int* act_v;     // [cap] active vertices (ascending)
  int* act_ptr;   // [cap + 1] entry range of each active vertex
  int2* ent;      // [8 Q] entries: (point, bits of the trilinear weight / L)
  // finest level only: the query points in cell order, (iz (n-1) + iy)(n-1) + ix (per frame)
  int* ccnt;      // [cells] points per cell (zero between builds)
  int* coff;      // [cells + 1] exclusive prefix of ccnt
  int* ckey;      // [Q] cell of each point (scratch of the build)
  float4* xs;     // [Q] points in cell order: (fx, fy, fz, point index bits)
  int* n_active;  // device scalar
  int* csum;      // scan scratch
  int adj_lg;     // adjoint: log2 of the lanes per row, 6 = a block per row (set by the plan kernel)
};

struct Job {
  int L;
  int C;                   // channels of the payload: 3 (displacement) or 6 (Cayley z, t)
  Level lev[MAXL];
  float lo[3], hi[3];
  float alpha, w_mesh, w_pts, w_iso;
  int stopgrad, precondition, keep_pgrad;
  int no_adam;             // 1: pass C stores the preconditioned gradient and skips Adam
  float beta1, beta2, eps;
  int V, N, M, E, Q;       // template verts, source pts, target pts, edges, V + N
  int max_pts;
  float4* x;               // [Q] undeformed query points (template first), fixed in a frame
  float4* y;               // [Q] deformed points
  float4* gfwd;            // [Q] forward Chamfer gradient
  long long* acc;          // [Q][3] reverse Chamfer sums, fixed point (2^-40)
  float4* gy;              // [Q] dLoss/dy (= dLoss/dt with the Cayley payload)
  float4* zq;              // [Q] Cayley payload: the point's averaged z (null otherwise)
  float4* uq;              // [Q] Cayley payload: u = (I - Z)^{-1} x, so that R(z) x = 2 u - x
  float4* gz;              // [Q] Cayley payload: dLoss/dz of the point
  float* loss_fwd;         // [Q] phi(d^2) of each forward query
  float* loss_rev;         // [2 max_pts] phi(d^2) of each reverse query (set 0 then set 1)
  float* loss_iso;         // [E] |r_e|
  int* nn_fwd;             // [Q] (-1 before the first search of a frame)
  int* nn_rev;             // [2 max_pts] (-1 before the first search of a frame)
  float4* edge_d;          // [E] sgn(r) (y_i - y_j) / (|y_i - y_j| E)
  const int2* edges;       // [E]
  float* e_prev;           // [E] rest lengths from X_{t-1}
  const int* v2e_ptr;      // [V + 1]
  const int* v2e;          // [2E] (edge << 1) | (1 if the vertex is the edge's second end)
  float4* src4;            // [max_pts] current source cloud P_{t-1}
  float4* tgt4;            // [max_pts] target P_t
  float4* verts4;          // [V] current deformed template X_{t-1}
  CellGrid tgt;            // target grid, one set, built per frame
  CellGrid mov;            // moving grid, two sets (template, source), rebuilt every step
  int4* hard;              // [Q + 2 max_pts] queries left by the thread pass: (item, ring, d2 bits, idx)
  float* loss_part;        // [loss chunks][5] partial sums
  unsigned* gmax;          // max |dLoss/dy| component of the step (float bits; sets the adjoint's fixed-point scale)
  int* hard_count;         // device scalar
  int* step;               // Adam step count k
  float* bias;             // [2] 1 / (1 - beta1^k), 1 / sqrt(1 - beta2^k) of the current step
  double* loss;            // [4] total, cd_mesh, cd_pts, iso of the last step
  int* status;             // sticky error flags (1: non-finite loss)
  unsigned long long* counters;  // [4] of the last step: NN candidates evaluated (counted only
                                 // when count_nn), NN queries decided by an exact tie,
                                 // queries left to the warp pass, reserved
  int count_nn;            // 1: k_nn / k_nn_hard add their candidate counts to counters[0]
};

enum Counter { CNT_NN_CANDIDATES = 0, CNT_NN_TIES = 1, CNT_NN_HARD = 2 };

enum Stage { ST_Q = 0, ST_NNQ, ST_E, ST_MOVCH, ST_ADJ, ST_TILE, ST_JOB, ST_LOSSCH, ST_PLANE, ST_COL, ST_ADAM, NSTAGE };

struct Plan {
  int n_jobs;
  int pad_[3];
  Job* jobs[MAXJ];
  int pre[NSTAGE][MAXJ + 1];
};

// ------------------------------------------------------------------------------ helpers

// Which preconditioner path takes a level of n vertices per axis: powers of two up to 128
// (and n = 1) take the shared-memory plane path, 256 and the sizes with a factor 3 the
// tile path with mixed radix-2/3 line transforms.
__host__ __device__ __forceinline__ bool tile_level(int n) { return n > 128 || (n & (n - 1)) != 0; }

__device__ __forceinline__ int find_job(const int* pre, int n_jobs, int item) {
  int lo = 0, hi = n_jobs;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(pre + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

__host__ __device__ __forceinline__ uint32_t part1by1(uint32_t v) {
  v &= 0xFFu;
  v = (v | (v << 4)) & 0x0F0Fu;
  v = (v | (v << 2)) & 0x3333u;
  v = (v | (v << 1)) & 0x5555u;
  return v;
}

__host__ __device__ __forceinline__ int row_key(int cy, int cz, int bits) {
  return (int)((part1by1((uint32_t)cy) | (part1by1((uint32_t)cz) << 1)) << bits);
}

__device__ __forceinline__ int cell_coord(float p, float lo, float inv_h, int G) {
  float t = (p - lo) * inv_h;
  t = fminf(fmaxf(t, -1.0f), (float)G);
  int c = (int)floorf(t);
  return min(max(c, 0), G - 1);
}

__device__ __forceinline__ int cell_key(const CellGrid& g, float x, float y, float z, int set) {
  int G = 1 << g.bits;
  int cx = cell_coord(x, g.lo[0], g.inv_h[0], G);
  int cy = cell_coord(y, g.lo[1], g.inv_h[1], G);
  int cz = cell_coord(z, g.lo[2], g.inv_h[2], G);
  return set * (G * G * G) + row_key(cy, cz, g.bits) + cx;
}

// squared distance, difference form; the same expression everywhere so that candidate
// comparisons are consistent between kernels
__device__ __forceinline__ float sqdist(float ax, float ay, float az, float bx, float by, float bz) {
  const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Grid coordinate of x in a level with n >= 2 vertices per axis (Eq. 1, vertex-aligned,
// clamped, last cell closed): u = (x - lo) (n - 1) / (hi - lo), i0 = min(floor(u), n - 2),
// f = u - i0.  x - lo is formed exactly (TwoSum) and multiplied by the scale held as a
// float pair with an FMA two-product, so f carries ~1 ulp of error instead of
// ulp(hi - lo) * (n - 1) (which would reach 1e-5 of a weight on 128^3 grids).
__device__ __forceinline__ void grid_coord(float x, float lo, float s_hi, float s_lo, int n, int& i0, float& f) {
  const float d = __fsub_rn(x, lo);
  const float bv = __fsub_rn(d, x);
  const float dl = __fadd_rn(__fsub_rn(x, __fsub_rn(d, bv)), __fsub_rn(-lo, bv));  // x - lo = d + dl exactly
  const float p = __fmul_rn(d, s_hi);
  const float e = __fmaf_rn(d, s_hi, -p);
  const float ul = __fadd_rn(e, __fmaf_rn(d, s_lo, __fmul_rn(dl, s_hi)));       // u = p + ul
  if (!(p > 0.f) && !(p == 0.f && ul > 0.f)) {  // u <= 0 (or NaN): clamp to vertex 0
    i0 = 0;
    f = 0.f;
    return;
  }
  if (p > (float)(n - 1) || (p == (float)(n - 1) && ul >= 0.f)) {  // u >= n - 1: clamp to the last vertex
    i0 = n - 2;
    f = 1.f;
    return;
  }
  float fl = floorf(p);
  if (fl == p && ul < 0.f) fl -= 1.f;
  int i = (int)fl;
  float fr = __fadd_rn(__fsub_rn(p, fl), ul);
  if (fr >= 1.f && i < n - 2) {
    i += 1;
    fr = __fsub_rn(fr, 1.f);
  }
  if (fr < 0.f && i > 0) {
    i -= 1;
    fr = __fadd_rn(fr, 1.f);
  }
  if (i > n - 2) {
    i = n - 2;
    fr = 1.f;
  }
  i0 = i;
  f = fminf(fmaxf(fr, 0.f), 1.f);
}

// The Cayley rotation of Sec. 3.3 applied to x without forming R(z) = (I + Z)(I - Z)^{-1}:
// (I - Z)^{-1} = (I + Z + z z^T) / (1 + |z|^2) (multiply out with Z^2 = z z^T - |z|^2 I), and
// R = 2 (I - Z)^{-1} - I, so R(z) x = 2 u - x with u = (x + z x x + z (z . x)) / (1 + |z|^2).
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float3 cayley_u(float3 z, float3 x) {
  const float s = 1.f / (1.f + (z.x * z.x + z.y * z.y + z.z * z.z));
  const float zx = z.x * x.x + z.y * x.y + z.z * x.z;
  const float3 c = cross3(z, x);
  return make_float3((x.x + c.x + z.x * zx) * s, (x.y + c.y + z.y * zx) * s, (x.z + c.z + z.z * zx) * s);
}

// dLoss/dz for y = R(z) x + t and g = dLoss/dy: d(R x) = 2 (I - Z)^{-1} dZ u = -2 (I - Z)^{-1} [u]x dz,
// so dLoss/dz = 2 u x w with w = (I - Z)^{-T} g = (I + Z)^{-1} g = (g - z x g + z (z . g)) / (1 + |z|^2).
__device__ __forceinline__ float3 cayley_grad_z(float3 z, float3 u, float3 g) {
  const float s = 1.f / (1.f + (z.x * z.x + z.y * z.y + z.z * z.z));
  const float zg = z.x * g.x + z.y * g.y + z.z * g.z;
  const float3 c = cross3(z, g);
  const float3 w = make_float3((g.x - c.x + z.x * zg) * s, (g.y - c.y + z.y * zg) * s, (g.z - c.z + z.z * zg) * s);
  const float3 r = cross3(u, w);
  return make_float3(2.f * r.x, 2.f * r.y, 2.f * r.z);
}

__device__ __forceinline__ long long to_fx(float v) { return __float2ll_rn(v * 1099511627776.0f); }
__device__ __forceinline__ float from_fx(long long a) { return __ll2float_rn(a) * (1.0f / 1099511627776.0f); }

}  // namespace pdg
