// Grid Sobolev preconditioning (Sec. 3.2, Eq. 3) and the Adam update (Sec. 3.6) for levels
// of up to 128^3 vertices, in four kernels:
//   A     per (z-plane, channel): DCT-II along x, then along y                    g   -> tmp
//   B     per (kx, ky) column along z and channel, in registers: two tridiagonal solves with
//         T = (1 + lambda (mu_kx + mu_ky)) I + lambda L_z (T^{-2}), and the 1/n^2 of the
//         x and y inverse transforms                                                tmp -> tmp
//   C     per (z-plane, channel): inverse along y, then along x                    tmp -> tmp
//   Adam  elementwise on theta, m, v with the preconditioned gradient             tmp -> theta
// Why: L_l, the free-boundary 6-neighbour Laplacian, is the Kronecker sum of three
// path-graph Laplacians whose eigenvectors are the DCT-II basis vectors
// cos(pi k (i + 1/2) / n) with eigenvalues mu_k = 4 sin^2(pi k / 2n).  After the x and y DCTs
// the operator (I + lambda L)^{-2} acts on each (kx, ky) column along z as T^{-2} with the
// tridiagonal T above, which the Thomas algorithm inverts exactly in O(n) per column.
//
// A line transform handles two lines at once (packed as the real and imaginary parts of one
// complex sequence after the even/odd reordering that turns a DCT-II into a DFT).  The
// length-n complex FFT is a two-stage Cooley-Tukey split n = N1 x N2 done by a group of N1
// threads: each thread runs an N2-point DFT in registers, applies the twiddles, the group
// transposes through a small shared scratch, and each thread runs N2/N1 DFTs of N1 points.
// The pairing of Z_k with Z_{n-k} that separates the two packed lines is a register
// exchange between the lanes t and N1 - t of a group.
//
// Data movement of A and C: the first direction reads its lines straight from global
// memory into registers and leaves its result in a shared-memory plane; the second
// direction reads the plane and writes straight to global memory.  The shared plane is
// unpadded for n >= 32 with an XOR swizzle of the column index, chosen so that both access
// shapes of the passes (4 rows x 8 consecutive columns, and 8 rows x 4 consecutive columns)
// touch 32 distinct banks.  z-planes without an active vertex (the gradient lives on the
// vertices near the data) are skipped by A and read as zero by B.
#include "kernels.h"

namespace pdg {

// exp(-2 pi i k / 16), k < 8
__device__ __forceinline__ float2 tw16(int k) {
  switch (k) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(0.923879532511286756f, -0.382683432365089772f);
    case 2: return make_float2(0.707106781186547524f, -0.707106781186547524f);
    case 3: return make_float2(0.382683432365089772f, -0.923879532511286756f);
    case 4: return make_float2(0.f, -1.f);
    case 5: return make_float2(-0.382683432365089772f, -0.923879532511286756f);
    case 6: return make_float2(-0.707106781186547524f, -0.707106781186547524f);
    default: return make_float2(-0.923879532511286756f, -0.382683432365089772f);
  }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int R>
__host__ __device__ constexpr int bitrev(int k) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) r = (r << 1) | ((k & b) ? 1 : 0);
  return r;
}

// In-register DFT of R <= 16 points (natural order in and out): radix-2 decimation in
// frequency with constant twiddles, then the bit-reversal permutation.
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&a)[R]) {
#pragma unroll
  for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int start = 0; start < R; start += 2 * span) {
#pragma unroll
      for (int k = 0; k < span; ++k) {
        const int i = start + k, j = i + span;
        const float2 t = make_float2(a[i].x - a[j].x, a[i].y - a[j].y);
        a[i] = make_float2(a[i].x + a[j].x, a[i].y + a[j].y);
        if (k == 0) {
          a[j] = t;
        } else {
          float2 w = tw16((k * 16) / (2 * span));
          if (INV) w.y = -w.y;
          a[j] = cmul(t, w);
        }
      }
    }
  }
  float2 b[R];
#pragma unroll
  for (int k = 0; k < R; ++k) b[k] = a[bitrev<R>(k)];
#pragma unroll
  for (int k = 0; k < R; ++k) a[k] = b[k];
}

// Complex FFT of n = N1 * N2 points by a group of N1 threads (thread t).  In: reg[m] =
// x[t + N1 m].  Out: reg[jj N1 + k1] = X[k2 + N2 k1] with k2 = t + N1 jj.  sc: the group's
// scratch of N1 (N2 + 1) complex; twn[m] = exp(-2 pi i m / n).  All threads of the warp
// must call it together (it synchronises the warp).
template <int N1, int N2, bool INV>
__device__ __forceinline__ void fft2(float2 (&reg)[N2], float2* sc, int t, const float2* __restrict__ twn) {
  constexpr int n = N1 * N2;
  dft_reg<N2, INV>(reg);
  if (N1 > 1) {
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) {
      float2 w = __ldg(twn + ((t * k2) & (n - 1)));
      if (INV) w.y = -w.y;
      reg[k2] = cmul(reg[k2], w);
    }
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) sc[t * (N2 + 1) + k2] = reg[k2];
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < N2 / N1; ++jj) {
      float2 r2[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) r2[n1] = sc[n1 * (N2 + 1) + t + N1 * jj];
      dft_reg<N1, INV>(r2);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) reg[jj * N1 + k1] = r2[k1];
    }
    __syncwarp();
  }
}

__device__ __forceinline__ int dsrc(int j, int n) { return j < (n >> 1) ? 2 * j : 2 * (n - 1 - j) + 1; }

// index (frequency or position) held in output register idx of thread t after fft2
template <int N1, int N2>
__device__ __forceinline__ int out_index(int idx, int t) {
  if (N1 == 1) return idx;
  return t + N1 * (idx / N1) + N2 * (idx % N1);
}

constexpr int PL_THREADS = 256;

__host__ __device__ constexpr int plane_n1(int n) { return n <= 16 ? 1 : (n == 32 ? 4 : 8); }

// Shared plane of n x n floats: unpadded and column-swizzled for n >= 32 (the swizzle
// keeps even/odd column pairs adjacent), row stride n + 1 below.
template <int n>
__device__ __forceinline__ int pidx(int r, int x) {
  if (n >= 32) {
    const int u = (r >> 1) & 7;
    return r * n + (x ^ (((u & 3) << 3) | ((u >> 2) << 2)));
  } else {
    return r * (n + 1) + x;
  }
}

__host__ __device__ constexpr int plane_floats(int n) { return n >= 32 ? n * n : n * (n + 1); }
__host__ __device__ constexpr int group_scratch(int n) {
  return plane_n1(n) > 1 ? plane_n1(n) * (n / plane_n1(n) + 1) : 0;  // float2 per group
}
int scratch_bytes(int n) { return (PL_THREADS / plane_n1(n)) * group_scratch(n) * 8; }

// shared memory of a plane pass for resolution n: plane + per-group FFT scratch
int plane_smem_bytes(int n) { return ((plane_floats(n) + 1) & ~1) * 4 + scratch_bytes(n); }

template <int n>
__device__ __forceinline__ float2 plane_read2(const float* plane, int r, int x) {
  if (n >= 32) return *reinterpret_cast<const float2*>(plane + pidx<n>(r, x));
  return make_float2(plane[pidx<n>(r, x)], plane[pidx<n>(r, x + 1)]);
}

template <int n>
__device__ __forceinline__ void plane_write2(float* plane, int r, int x, float2 v) {
  if (n >= 32) {
    *reinterpret_cast<float2*>(plane + pidx<n>(r, x)) = v;
  } else {
    plane[pidx<n>(r, x)] = v.x;
    plane[pidx<n>(r, x + 1)] = v.y;
  }
}

// Forward input of rows A, B (global, n contiguous floats each): reg[m] = (a, b) at position
// j = t + N1 m of the even/odd reordering v[j] = x[dsrc(j)].  Each thread loads the pairs
// (x[2s], x[2s+1]) at s = t + N1 m' (m' < N2/2): the even element is its own v[s], the odd
// one is v[n - 1 - s] of lane t ^ (N1 - 1).
template <int N1, int N2>
__device__ __forceinline__ void load_fwd_rows(const float* __restrict__ rowA, const float* __restrict__ rowB, int t,
                                              float2 (&reg)[N2]) {
  constexpr int H = N2 / 2;
  float2 ea[H], eb[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    ea[m] = __ldg(reinterpret_cast<const float2*>(rowA) + t + N1 * m);
    eb[m] = __ldg(reinterpret_cast<const float2*>(rowB) + t + N1 * m);
  }
#pragma unroll
  for (int m = 0; m < H; ++m) reg[m] = make_float2(ea[m].x, eb[m].x);
#pragma unroll
  for (int m = H; m < N2; ++m) {
    float oa = ea[N2 - 1 - m].y, ob = eb[N2 - 1 - m].y;
    if (N1 > 1) {
      oa = __shfl_xor_sync(0xffffffffu, oa, N1 - 1);
      ob = __shfl_xor_sync(0xffffffffu, ob, N1 - 1);
    }
    reg[m] = make_float2(oa, ob);
  }
}

// Separates the two packed spectra after a forward fft2 and applies the DCT-II twiddle:
// X_A[k] = Re(w_k (Z_k + conj Z_{n-k}) / 2), X_B[k] = Re(w_k (Z_k - conj Z_{n-k}) / 2i),
// w_k = exp(-i pi k / 2n).  Z_{n-k} of lane t != 0 sits in lane N1 - t at the mirrored
// register; lane 0 holds both ends itself.
template <int N1, int N2>
__device__ __forceinline__ void dct2_post(const float2 (&reg)[N2], int t, int lbase, const float2* __restrict__ tw4,
                                          float (&XA)[N2], float (&XB)[N2]) {
  constexpr int n = N1 * N2, J = N2 / N1;
  const int src = lbase + ((N1 - t) & (N1 - 1));
#pragma unroll
  for (int idx = 0; idx < N2; ++idx) {
    float2 zc;
    if (N1 == 1) {
      zc = reg[(n - idx) & (n - 1)];
    } else {
      const int jj = idx / N1, k1 = idx % N1;
      const int it = (J - 1 - jj) * N1 + (N1 - 1 - k1);
      const int i0 = jj == 0 ? ((N1 - k1) & (N1 - 1)) : (J - jj) * N1 + (N1 - 1 - k1);
      float2 s;
      s.x = __shfl_sync(0xffffffffu, reg[it].x, src);
      s.y = __shfl_sync(0xffffffffu, reg[it].y, src);
      zc = t == 0 ? reg[i0] : s;
    }
    const float2 zk = reg[idx];
    const float2 va = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
    const float2 vb = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
    const float2 w = __ldg(tw4 + out_index<N1, N2>(idx, t));
    XA[idx] = w.x * va.x - w.y * va.y;
    XB[idx] = w.x * vb.x - w.y * vb.y;
  }
}

// Input of an inverse fft2 from two spectra X[m] = (X_A[k], X_B[k]), k = t + N1 m:
// V = exp(+i pi k / 2n) (X_k - i X_{n-k}) per line (X_n = 0), Z = V_A + i V_B.
template <int N1, int N2>
__device__ __forceinline__ void dct3_pre(const float2 (&X)[N2], int t, int lbase, const float2* __restrict__ tw4,
                                         float2 (&reg)[N2]) {
  constexpr int n = N1 * N2;
  const int src = lbase + ((N1 - t) & (N1 - 1));
#pragma unroll
  for (int m = 0; m < N2; ++m) {
    float2 xn;
    if (N1 == 1) {
      xn = m == 0 ? make_float2(0.f, 0.f) : X[n - m];
    } else {
      float2 s;
      s.x = __shfl_sync(0xffffffffu, X[N2 - 1 - m].x, src);
      s.y = __shfl_sync(0xffffffffu, X[N2 - 1 - m].y, src);
      const float2 own = m == 0 ? make_float2(0.f, 0.f) : X[(N2 - m) & (N2 - 1)];
      xn = t == 0 ? own : s;
    }
    const int k = t + N1 * m;
    float2 w = __ldg(tw4 + k);
    w.y = -w.y;  // exp(+i pi k / 2n)
    const float a = X[m].x, an = xn.x, b = X[m].y, bn = xn.y;
    const float2 va = make_float2(w.x * a + w.y * an, w.y * a - w.x * an);
    const float2 vb = make_float2(w.x * b + w.y * bn, w.y * b - w.x * bn);
    reg[m] = make_float2(va.x - vb.y, va.y + vb.x);
  }
}

// maps a plane item of a job to (level, index); C n items per level (plane major, then
// channel), only the plane-path levels (powers of two up to 128) take part
__device__ __forceinline__ bool plane_item(const Job& J, int r, int& l, int& idx) {
  for (l = 0; l < J.L; ++l) {
    const int n = J.lev[l].n;
    if (tile_level(n)) continue;
    if (r < J.C * n) {
      idx = r;
      return true;
    }
    r -= J.C * n;
  }
  return false;
}

// ------------------------------------------------------------------------------ pass A

// DCT-II along x (rows, from global memory) then y (columns of the shared plane, to global
// memory) of the z-plane `in` (n x n floats) into `out`.
template <int N1, int N2>
__device__ void plane_fwd(const Level& lv, const float* __restrict__ in, float* __restrict__ out, float* plane,
                          float2* scr) {
  constexpr int n = N1 * N2, GB = PL_THREADS / N1;
  const int gi = threadIdx.x / N1, t = threadIdx.x % N1;
  const int lbase = (threadIdx.x & 31) & ~(N1 - 1);
  float2* sc = scr + gi * group_scratch(n);
  // a group's line pairs: the condition is uniform over each warp when N1 > 1 (n N1 / 2 is a
  // multiple of 32), and N1 = 1 has no warp-collective step
  for (int p = gi; p < n / 2; p += GB) {  // x-lines: rows 2p, 2p + 1
    float2 reg[N2];
    load_fwd_rows<N1, N2>(in + (2 * p) * n, in + (2 * p + 1) * n, t, reg);
    fft2<N1, N2, false>(reg, sc, t, lv.tw);
    float XA[N2], XB[N2];
    dct2_post<N1, N2>(reg, t, lbase, lv.tw4, XA, XB);
#pragma unroll
    for (int idx = 0; idx < N2; ++idx) {
      const int k = out_index<N1, N2>(idx, t);
      plane[pidx<n>(2 * p, k)] = XA[idx];
      plane[pidx<n>(2 * p + 1, k)] = XB[idx];
    }
  }
  __syncthreads();
  for (int p = gi; p < n / 2; p += GB) {  // y-lines: columns 2p, 2p + 1
    float2 reg[N2];
#pragma unroll
    for (int m = 0; m < N2; ++m) reg[m] = plane_read2<n>(plane, dsrc(t + N1 * m, n), 2 * p);
    fft2<N1, N2, false>(reg, sc, t, lv.tw);
    float XA[N2], XB[N2];
    dct2_post<N1, N2>(reg, t, lbase, lv.tw4, XA, XB);
#pragma unroll
    for (int idx = 0; idx < N2; ++idx)
      *reinterpret_cast<float2*>(out + out_index<N1, N2>(idx, t) * n + 2 * p) = make_float2(XA[idx], XB[idx]);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(PL_THREADS, 2) k_sobp(const Plan* __restrict__ P) {
  extern __shared__ float smem[];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_PLANE][nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_PLANE], nj, it);
    const Job& J = *P->jobs[j];
    if (!J.precondition) continue;
    int l, idx;
    if (!plane_item(J, it - P->pre[ST_PLANE][j], l, idx)) continue;
    const Level& lv = J.lev[l];
    const int n = lv.n, n3 = lv.n3;
    const int q = idx / J.C, c = idx - J.C * q;  // z-plane, channel
    if (n == 1) {  // no transform: copy g to tmp (the scale is 1)
      if (threadIdx.x == 0) lv.tmp[c] = lv.g[c];
      continue;
    }
    // the gradient lives on the vertices near the data: a z-plane without an active vertex
    // stays zero, and pass B reads it as zero without loading it
    if (lv.zmask && !__ldg(lv.zmask + q)) continue;
    const size_t off = (size_t)c * n3 + (size_t)q * n * n;
    float* plane = smem;
    float2* scr = reinterpret_cast<float2*>(smem + ((plane_floats(n) + 1) & ~1));
    switch (n) {
      case 2: plane_fwd<1, 2>(lv, lv.g + off, lv.tmp + off, plane, scr); break;
      case 4: plane_fwd<1, 4>(lv, lv.g + off, lv.tmp + off, plane, scr); break;
      case 8: plane_fwd<1, 8>(lv, lv.g + off, lv.tmp + off, plane, scr); break;
      case 16: plane_fwd<1, 16>(lv, lv.g + off, lv.tmp + off, plane, scr); break;
      case 32: plane_fwd<4, 8>(lv, lv.g + off, lv.tmp + off, plane, scr); break;
      case 64: plane_fwd<8, 8>(lv, lv.g + off, lv.tmp + off, plane, scr); break;
      default: plane_fwd<8, 16>(lv, lv.g + off, lv.tmp + off, plane, scr); break;
    }
  }
}

// ------------------------------------------------------------------------------ pass B

// The two tridiagonal solves T^2 h = g of each (kx, ky) column of one channel.  T has
// diagonal b_i = a + lambda deg(i) (deg 1 at the two ends, 2 inside), off-diagonal -lambda,
// a = 1 + lambda (mu_kx + mu_ky).  Each solve is twisted (eliminated from both ends toward
// the middle row m = n/2): the top thread of a column holds rows 0 .. m-1 and eliminates
// downward, g'_i = (g_i + lambda g'_{i-1}) r_i; the bottom thread holds rows n-1 .. m and
// eliminates upward with the mirrored pivots (T is persymmetric: the pivots from the bottom
// are r_{n-1-i}); the middle row takes both neighbours,
//   h_m = (g_m + lambda g'_{m-1} + lambda g''_{m+1}) / (b_m - lambda^2 (r_{m-1} + r_{m-2})),
// and each thread back-substitutes toward its end, h_i = g'_i + lambda r_i h_{i +- 1}.  A
// thread's chain is n/2 long, its half column lives in registers and its pivots are read
// from the block's slice of a per-context table, staged in shared memory (volatile reads,
// so the compiler keeps them out of registers).  The two threads of a column are lanes l and l + 16
// of a warp (one value crosses between them, twice per solve); a warp covers 16 neighbouring
// columns, so each row access is 64 contiguous bytes.  Rows of z-planes without an active
// vertex are read as zero (the bit comes from a register mask, not from memory).
constexpr int COL_THREADS = 128;
constexpr int COLS_PER_ITEM = COL_THREADS / 2;
constexpr int PIV_REGS = 16;  // pivots held in registers on the fast path (then the limit)

// Pivot table of a level: piv[j n^2 + col] = r_j for j < n/2 (downward Thomas pivots of T,
// r_0 = 1 / b_0, r_j = 1 / (b_j - lambda^2 r_{j-1})) and, at j = n/2, the reciprocal of the
// middle row's twisted pivot.  Computed in FP64 once per context (lambda and n are fixed).
__global__ void k_sobz_pivots(float* __restrict__ piv, const float* __restrict__ mu, int n, float lam,
                              int* __restrict__ slow) {
  const int n2 = n * n, m = n / 2;
  const double L = lam, L2 = (double)lam * lam;
  for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < n2; col += gridDim.x * blockDim.x) {
    const double a = 1.0 + L * ((double)mu[col % n] + (double)mu[col / n]);
    double r = 0.0, rm1 = 0.0, rm2 = 0.0;
    for (int j = 0; j < m; ++j) {
      const double b = a + L * ((j == 0 || j == n - 1) ? 1.0 : 2.0);
      r = 1.0 / (b - L2 * r);
      piv[(size_t)j * n2 + col] = (float)r;
      if (j == m - 1) rm1 = r;
      if (j == m - 2) rm2 = r;
    }
    // row m: deg 1 only when it is the last row (n = 2); its lower neighbour exists for n >= 4
    const double bm = a + L * ((m == n - 1) ? 1.0 : 2.0);
    piv[(size_t)m * n2 + col] = (float)(1.0 / (bm - L2 * (rm1 + (n >= 4 ? rm2 : 0.0))));
    // the pivots converge geometrically; the register path holds r_0 .. r_15 and the last one
    // and needs every r_j, j >= 16, to equal the last one in FP32
    bool same = true;
    for (int j = PIV_REGS; j < m; ++j) same = same && piv[(size_t)j * n2 + col] == piv[(size_t)(m - 1) * n2 + col];
    if (!same) atomicOr(slow, 1);
  }
}

void launch_sobz_pivots(float* piv, int* slow, const float* mu, int n, float lam, cudaStream_t s) {
  if (n < 2 || n > 128) return;
  const int n2 = n * n;
  cudaMemsetAsync(slow, 0, sizeof(int), s);
  k_sobz_pivots<<<(n2 + 127) / 128, 128, 0, s>>>(piv, mu, n, lam, slow);
}

// FAST: pivots r_0 .. r_{K-1} and the limit in registers, read once from the table `pg`;
// otherwise each use reads the staged slice `pv` (stride COLS_PER_ITEM).
template <int N, bool FAST>
__device__ __forceinline__ void column_solve(float* __restrict__ t, const float* __restrict__ pg, volatile const float* pv,
                                             const unsigned (&zb)[4], float lam, float scale, bool top, bool act) {
  constexpr int M = N / 2;
  constexpr int n2 = N * N;
  constexpr int K = M < PIV_REGS ? M : PIV_REGS;
  float rp[K], rinf = 0.f;
  if (FAST) {
#pragma unroll
    for (int k = 0; k < K; ++k) rp[k] = act ? __ldg(pg + k * n2) : 0.f;
    rinf = act ? __ldg(pg + (M - 1) * n2) : 0.f;
  }
  auto piv = [&](int j) -> float { return FAST ? (j < K ? rp[j < K ? j : 0] : rinf) : pv[j * COLS_PER_ITEM]; };
  const int J = top ? M : M - 1;  // rows this thread eliminates
  float v[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const int i = top ? j : N - 1 - j;
    v[j] = (act && ((zb[i >> 5] >> (i & 31)) & 1u)) ? t[i * n2] : 0.f;
  }
  const float rm = act ? (FAST ? __ldg(pg + M * n2) : pv[M * COLS_PER_ITEM]) : 0.f;
#pragma unroll
  for (int solve = 0; solve < 2; ++solve) {
    float g = 0.f;
#pragma unroll
    for (int j = 0; j < M; ++j) {  // elimination toward the middle
      if (j < J) {
        g = (v[j] + lam * g) * piv(j);
        v[j] = g;
      }
    }
    // middle row (held by the bottom thread): both eliminated neighbours
    const float e_top = __shfl_xor_sync(0xffffffffu, v[M - 1], 16);  // top's g'_{m-1}
    const float e_bot = M >= 2 ? v[M >= 2 ? M - 2 : 0] : 0.f;        // bottom's g''_{m+1}
    float hm = (v[M - 1] + lam * e_top + lam * e_bot) * rm;  // meaningful in the bottom thread
    const float hb = __shfl_xor_sync(0xffffffffu, hm, 16);
    if (top) hm = hb;
    else v[M - 1] = hm;
    float h = hm;
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {  // back substitution toward this thread's end
      if (j < J) {
        v[j] = v[j] + lam * piv(j) * h;
        h = v[j];
      }
    }
  }
  if (act) {
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const int i = top ? j : N - 1 - j;
      t[i * n2] = v[j] * scale;
    }
  }
}

// an item is COLS_PER_ITEM consecutive columns (col = y n + x) of one channel of one level
__device__ __forceinline__ bool column_item(const Job& J, int r, int& l, int& c, int& col0) {
  for (l = 0; l < J.L; ++l) {
    const int n = J.lev[l].n;
    if (tile_level(n)) continue;
    const int per = (n * n + COLS_PER_ITEM - 1) / COLS_PER_ITEM;
    if (r < J.C * per) {
      c = r / per;
      col0 = (r - c * per) * COLS_PER_ITEM;
      return true;
    }
    r -= J.C * per;
  }
  return false;
}

// One block of COL_THREADS per item: warp w covers columns col0 + 16 w .. + 15, lane l < 16
// the top half of column l, lane l + 16 its bottom half.
__global__ void __launch_bounds__(COL_THREADS, 4) k_sobz(const Plan* __restrict__ P) {
  __shared__ unsigned zbits[4];
  __shared__ float rs[(128 / 2 + 1) * COLS_PER_ITEM];  // pivots [j][column of the item]
  const int nj = P->n_jobs;
  const int total = P->pre[ST_COL][nj];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_COL], nj, it);
    const Job& J = *P->jobs[j];
    if (!J.precondition) continue;
    int l, c, col0;
    if (!column_item(J, it - P->pre[ST_COL][j], l, c, col0)) continue;
    const Level& lv = J.lev[l];
    const int n = lv.n;
    if (n == 1) continue;  // a single vertex: T = 1
    const bool fast = !__ldg(lv.piv_slow);  // block-uniform
    // bit i: z-plane i holds an active vertex (else it is zero and pass A did not write it)
    __syncthreads();  // the previous item has read zbits and rs
    {
      const bool nz = threadIdx.x >= n || !lv.zmask || __ldg(lv.zmask + threadIdx.x);
      const unsigned b = __ballot_sync(0xffffffffu, nz);
      if (lane == 0) zbits[warp] = b;
      const int n2 = n * n, rows = fast ? 0 : n / 2 + 1;
      for (int k = threadIdx.x; k < rows * COLS_PER_ITEM; k += COL_THREADS) {
        const int cl = col0 + (k % COLS_PER_ITEM);
        rs[k] = cl < n2 ? __ldg(lv.piv + (size_t)(k / COLS_PER_ITEM) * n2 + cl) : 0.f;
      }
    }
    __syncthreads();
    const unsigned zb[4] = {zbits[0], zbits[1], zbits[2], zbits[3]};
    const int col = col0 + warp * 16 + (lane & 15);
    const bool act = col < n * n, top = lane < 16;
    const int cc = act ? col : 0;
    const float lam = lv.lam;
    const float scale = 1.f / (float)(n * n);
    float* t = lv.tmp + (size_t)c * lv.n3 + cc;
    const float* pg = lv.piv + cc;
    volatile const float* pv = rs + warp * 16 + (lane & 15);
#define PDG_SOLVE(NN)                                               \
  if (fast) column_solve<NN, true>(t, pg, pv, zb, lam, scale, top, act); \
  else column_solve<NN, false>(t, pg, pv, zb, lam, scale, top, act);
    switch (n) {  // warp-uniform: every lane takes part in the exchanges
      case 2: PDG_SOLVE(2) break;
      case 4: PDG_SOLVE(4) break;
      case 8: PDG_SOLVE(8) break;
      case 16: PDG_SOLVE(16) break;
      case 32: PDG_SOLVE(32) break;
      case 64: PDG_SOLVE(64) break;
      default: PDG_SOLVE(128) break;
    }
#undef PDG_SOLVE
  }
}

// ------------------------------------------------------------------------------ pass C

// Inverse DCT along y (columns, from global memory) then x (rows of the shared plane) of
// z-plane q, channel c; the preconditioned gradient goes back to tmp (coalesced pairs of
// neighbouring columns) for the Adam kernel.
template <int N1, int N2>
__device__ void plane_inv(const Job& J, const Level& lv, int c, int q, float* plane, float2* scr) {
  constexpr int n = N1 * N2, GB = PL_THREADS / N1, H = N2 / 2;
  const int gi = threadIdx.x / N1, t = threadIdx.x % N1;
  const int lbase = (threadIdx.x & 31) & ~(N1 - 1);
  float2* sc = scr + gi * group_scratch(n);
  const size_t poff = (size_t)q * n * n;
  const float* tp = lv.tmp + (size_t)c * lv.n3 + poff;
  for (int p = gi; p < n / 2; p += GB) {  // y-lines: columns 2p, 2p + 1
    float2 X[N2];
#pragma unroll
    for (int m = 0; m < N2; ++m) X[m] = *reinterpret_cast<const float2*>(tp + (t + N1 * m) * n + 2 * p);
    float2 reg[N2];
    dct3_pre<N1, N2>(X, t, lbase, lv.tw4, reg);
    fft2<N1, N2, true>(reg, sc, t, lv.tw);
#pragma unroll
    for (int idx = 0; idx < N2; ++idx) plane_write2<n>(plane, dsrc(out_index<N1, N2>(idx, t), n), 2 * p, reg[idx]);
  }
  __syncthreads();
  float* out = lv.tmp + (size_t)c * lv.n3;
  for (int p = gi; p < n / 2; p += GB) {  // x-lines: rows 2p, 2p + 1
    float2 X[N2];
#pragma unroll
    for (int m = 0; m < N2; ++m) {
      const int k = t + N1 * m;
      X[m] = make_float2(plane[pidx<n>(2 * p, k)], plane[pidx<n>(2 * p + 1, k)]);
    }
    float2 reg[N2];
    dct3_pre<N1, N2>(X, t, lbase, lv.tw4, reg);
    fft2<N1, N2, true>(reg, sc, t, lv.tw);
    // z[j] is the value at x = dsrc(j): for j < n/2 the even column 2j, whose odd neighbour
    // 2j + 1 = dsrc(n - 1 - j) sits in lane t ^ (N1 - 1) at the mirrored register
    float2 ga[H], gb[H];
    int xs[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int jj = N1 == 1 ? h : h / (N1 / 2), k1 = N1 == 1 ? 0 : h % (N1 / 2);
      const int idx = N1 == 1 ? h : jj * N1 + k1;
      const int mir = N1 == 1 ? n - 1 - h : (N2 / N1 - 1 - jj) * N1 + (N1 - 1 - k1);
      float2 o = reg[mir];
      if (N1 > 1) {
        o.x = __shfl_xor_sync(0xffffffffu, o.x, N1 - 1);
        o.y = __shfl_xor_sync(0xffffffffu, o.y, N1 - 1);
      }
      xs[h] = 2 * out_index<N1, N2>(idx, t);
      ga[h] = make_float2(reg[idx].x, o.x);
      gb[h] = make_float2(reg[idx].y, o.y);
    }
    const size_t rowA = poff + (size_t)(2 * p) * n, rowB = rowA + n;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      *reinterpret_cast<float2*>(out + rowA + xs[h]) = ga[h];
      *reinterpret_cast<float2*>(out + rowB + xs[h]) = gb[h];
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(PL_THREADS, 2) k_sobp_inv(const Plan* __restrict__ P) {
  extern __shared__ float smem[];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_PLANE][nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_PLANE], nj, it);
    const Job& J = *P->jobs[j];
    if (!J.precondition) continue;  // the Adam kernel reads the raw gradient
    int l, idx;
    if (!plane_item(J, it - P->pre[ST_PLANE][j], l, idx)) continue;
    const Level& lv = J.lev[l];
    const int n = lv.n;
    const int q = idx / J.C, c = idx - J.C * q;
    if (n == 1) continue;  // tmp already holds the preconditioned gradient (the operator is 1)
    float* plane = smem;
    float2* scr = reinterpret_cast<float2*>(smem + ((plane_floats(n) + 1) & ~1));
    switch (n) {
      case 2: plane_inv<1, 2>(J, lv, c, q, plane, scr); break;
      case 4: plane_inv<1, 4>(J, lv, c, q, plane, scr); break;
      case 8: plane_inv<1, 8>(J, lv, c, q, plane, scr); break;
      case 16: plane_inv<1, 16>(J, lv, c, q, plane, scr); break;
      case 32: plane_inv<4, 8>(J, lv, c, q, plane, scr); break;
      case 64: plane_inv<8, 8>(J, lv, c, q, plane, scr); break;
      default: plane_inv<8, 16>(J, lv, c, q, plane, scr); break;
    }
  }
}

// ------------------------------------------------------------------------------ Adam

// Adam (PyTorch semantics) on every vertex of every level (n <= 128) from the preconditioned
// gradient in tmp (or the raw gradient without preconditioning): 4 vertices per thread,
// float4 loads of the three channel planes of g, m and v, float4 theta.
__device__ __forceinline__ bool adam_item(const Job& J, int r, int& l, int& q) {
  for (l = 0; l < J.L; ++l) {
    const int n = J.lev[l].n;
    if (tile_level(n)) continue;
    const int cnt = (J.lev[l].n3 + 3) >> 2;
    if (r < cnt) {
      q = r;
      return true;
    }
    r -= cnt;
  }
  return false;
}

// Adam on one channel of 4 consecutive vertices e .. e + 3: th[k] is channel c of vertex e + k
__device__ __forceinline__ void adam4(const float* __restrict__ gsrc, float* __restrict__ m, float* __restrict__ v,
                                      size_t off, float b1, float b2, float eps, float step, float ib2, float (&th)[4]) {
  const float4 g4 = *reinterpret_cast<const float4*>(gsrc + off);
  float4 m4 = *reinterpret_cast<const float4*>(m + off);
  float4 v4 = *reinterpret_cast<const float4*>(v + off);
  const float g[4] = {g4.x, g4.y, g4.z, g4.w};
  float* mm = &m4.x;
  float* vv = &v4.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    mm[k] = b1 * mm[k] + (1.f - b1) * g[k];
    vv[k] = b2 * vv[k] + (1.f - b2) * g[k] * g[k];
    th[k] -= step * mm[k] / (sqrtf(vv[k]) * ib2 + eps);
  }
  *reinterpret_cast<float4*>(m + off) = m4;
  *reinterpret_cast<float4*>(v + off) = v4;
}

// Adam on the float4 array `t` (3 channels starting at channel c0 of the planar arrays)
__device__ __forceinline__ void adam_float4(float4* __restrict__ t, const float* __restrict__ gsrc, float* m, float* v,
                                            size_t n3, int c0, size_t e, float b1, float b2, float eps, float step,
                                            float ib2) {
  float4 th[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) th[k] = t[e + k];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float tc[4] = {(&th[0].x)[c], (&th[1].x)[c], (&th[2].x)[c], (&th[3].x)[c]};
    adam4(gsrc, m, v, (size_t)(c0 + c) * n3 + e, b1, b2, eps, step, ib2, tc);
#pragma unroll
    for (int k = 0; k < 4; ++k) (&th[k].x)[c] = tc[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) t[e + k] = th[k];
}

__global__ void __launch_bounds__(256) k_adam(const Plan* __restrict__ P) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_ADAM][nj];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int j = find_job(P->pre[ST_ADAM], nj, it);
    const Job& J = *P->jobs[j];
    if (J.no_adam) continue;
    int l, q;
    if (!adam_item(J, it - P->pre[ST_ADAM][j], l, q)) continue;
    const Level& lv = J.lev[l];
    const size_t n3 = lv.n3;
    const float* __restrict__ gsrc = J.precondition ? lv.tmp : lv.g;
    const float b1 = J.beta1, b2 = J.beta2, eps = J.eps;
    const float step = lv.lr * J.bias[0];
    const float ib2 = J.bias[1];
    if (n3 >= 4) {
      const size_t e = (size_t)q << 2;
      adam_float4(lv.theta, gsrc, lv.m, lv.v, n3, 0, e, b1, b2, eps, step, ib2);
      if (J.C == 6) adam_float4(lv.theta_t, gsrc, lv.m, lv.v, n3, 3, e, b1, b2, eps, step, ib2);
    } else {  // n == 1
      for (int half = 0; half < J.C / 3; ++half) {
        float4* t = half ? lv.theta_t : lv.theta;
        float4 th = t[0];
        for (int c = 0; c < 3; ++c) {
          const int cc = 3 * half + c;
          const float g = gsrc[cc * n3];
          float m = b1 * lv.m[cc * n3] + (1.f - b1) * g;
          float v = b2 * lv.v[cc * n3] + (1.f - b2) * g * g;
          lv.m[cc * n3] = m;
          lv.v[cc * n3] = v;
          (&th.x)[c] -= step * m / (sqrtf(v) * ib2 + eps);
        }
        t[0] = th;
      }
    }
  }
}

// ------------------------------------------------------------------------------ per frame

// zmask[z] = 1 for the z-planes of a level that hold an active vertex (per frame)
__global__ void k_zmask(Job* __restrict__ Jp, int l) {
  const Level& lv = Jp->lev[l];
  const int na = *lv.n_active;
  const int sh = 2 * lv.lg;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x)
    lv.zmask[lv.act_v[i] >> sh] = 1;
}

void launch_zmask(Job* J, const Job& hJ, cudaStream_t s) {
  for (int l = 0; l < hJ.L; ++l) {
    const Level& lv = hJ.lev[l];
    if (!lv.zmask) continue;
    cudaMemsetAsync(lv.zmask, 0, sizeof(int) * lv.n, s);
    const int grid = lv.n3 / 256 + 1 < 1024 ? lv.n3 / 256 + 1 : 1024;
    k_zmask<<<grid, 256, 0, s>>>(J, l);
  }
}

// largest shared memory a plane pass needs over the levels n <= nmax it may meet
int plane_smem_max(int nmax) {
  int m = 0;
  for (int n = 2; n <= 128 && n <= (nmax < 2 ? 2 : nmax); n <<= 1) m = plane_smem_bytes(n) > m ? plane_smem_bytes(n) : m;
  return m;
}

void sobolev_plane_configure() {
  const int smem = plane_smem_max(128);
  cudaFuncSetAttribute(k_sobp, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_sobp_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// part: 0 xy-forward, 1 z solve, 2 xy-inverse, 3 Adam, -1 all four
void launch_sobolev_plane(const Plan* P, int grid, int nmax, cudaStream_t s, int part) {
  const int smem = plane_smem_max(nmax);
  if (part < 0 || part == 0) k_sobp<<<grid, PL_THREADS, smem, s>>>(P);
  if (part < 0 || part == 1) k_sobz<<<grid * 3, COL_THREADS, 0, s>>>(P);
  if (part < 0 || part == 2) k_sobp_inv<<<grid, PL_THREADS, smem, s>>>(P);
  if (part < 0 || part == 3) k_adam<<<grid * 8, 256, 0, s>>>(P);
}

}  // namespace pdg
