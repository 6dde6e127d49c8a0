// Grid Sobolev preconditioning (Sec. 3.2, Eq. 3) and the Adam update (Sec. 3.6) for levels
// of up to 128^3 vertices, in four kernels:
//   A     per (z-plane, channel), in shared memory: DCT-II along x, then along y    g   -> tmp
//   B     per (kx, ky) column along z and channel, in registers: two tridiagonal solves with
//         T = (1 + lambda (mu_kx + mu_ky)) I + lambda L_z (T^{-2}), and the 1/n^2 of the
//         x and y inverse transforms                                                 tmp -> tmp
//   C     per (z-plane, channel), in shared memory: inverse along y, then along x   tmp -> tmp
//   Adam  elementwise on theta, m, v with the preconditioned gradient              tmp -> theta
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
// transposes through padded shared memory, and each thread runs N2/N1 DFTs of N1 points.
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

// Forward DCT-II (unnormalised) of lines A, B (element stride es) by a group; `act` false
// groups take part in the synchronisation only.
template <int N1, int N2>
__device__ __forceinline__ void dct2_lines(float* A, float* B, int es, float2* sc, int t, bool act,
                                          const float2* __restrict__ twn, const float2* __restrict__ tw4) {
  constexpr int n = N1 * N2;
  float2 reg[N2];
#pragma unroll
  for (int m = 0; m < N2; ++m) {
    const int s = dsrc(t + N1 * m, n) * es;
    reg[m] = act ? make_float2(A[s], B[s]) : make_float2(0.f, 0.f);
  }
  fft2<N1, N2, false>(reg, sc, t, twn);
#pragma unroll
  for (int jj = 0; jj < N2 / N1; ++jj)
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) sc[t + N1 * jj + N2 * k1] = reg[jj * N1 + k1];
  __syncwarp();
  if (act) {
#pragma unroll
    for (int m = 0; m < N2; ++m) {
      const int k = t + N1 * m;
      const float2 zk = sc[k];
      const float2 zc = sc[(n - k) & (n - 1)];
      // V_A = (Z_k + conj Z_{n-k}) / 2, V_B = (Z_k - conj Z_{n-k}) / 2i, X = Re(exp(-i pi k/2n) V)
      const float2 va = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
      const float2 vb = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
      const float2 w = __ldg(tw4 + k);
      A[k * es] = w.x * va.x - w.y * va.y;
      B[k * es] = w.x * vb.x - w.y * vb.y;
    }
  }
  __syncwarp();
}

// Inverse: A, B <- n C^{-1} A, n C^{-1} B (the 1/n per axis is folded into the scale).
template <int N1, int N2>
__device__ __forceinline__ void dct3_lines(float* A, float* B, int es, float2* sc, int t, bool act,
                                          const float2* __restrict__ twn, const float2* __restrict__ tw4) {
  constexpr int n = N1 * N2;
  if (act) {
#pragma unroll
    for (int m = 0; m < N2; ++m) {
      const int k = t + N1 * m;
      const float a = A[k * es], an = k ? A[(n - k) * es] : 0.f;
      const float b = B[k * es], bn = k ? B[(n - k) * es] : 0.f;
      float2 w = __ldg(tw4 + k);
      w.y = -w.y;  // exp(+i pi k / 2n);  V = w (X_k - i X_{n-k});  Z = V_A + i V_B
      const float2 va = make_float2(w.x * a + w.y * an, w.y * a - w.x * an);
      const float2 vb = make_float2(w.x * b + w.y * bn, w.y * b - w.x * bn);
      sc[k] = make_float2(va.x - vb.y, va.y + vb.x);
    }
  }
  __syncwarp();
  float2 reg[N2];
#pragma unroll
  for (int m = 0; m < N2; ++m) reg[m] = sc[t + N1 * m];
  __syncwarp();
  fft2<N1, N2, true>(reg, sc, t, twn);
  if (act) {
#pragma unroll
    for (int jj = 0; jj < N2 / N1; ++jj)
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int s = dsrc(t + N1 * jj + N2 * k1, n) * es;
        A[s] = reg[jj * N1 + k1].x;
        B[s] = reg[jj * N1 + k1].y;
      }
  }
  __syncwarp();
}

constexpr int PL_THREADS = 256;

__host__ __device__ constexpr int plane_n1(int n) { return n <= 16 ? 1 : (n == 32 ? 4 : (n == 64 ? 8 : (n == 128 ? 8 : 16))); }

// Row stride of a plane in shared memory.  n + 4 keeps rows 16-byte aligned (float4 copies
// from and to global memory) and spreads the strided line accesses of the transforms over
// the banks: for n = 128 a warp's loads take about 1.7 times the conflict-free number of
// shared-memory wavefronts, against 4 with a stride of n + 1.
__host__ __device__ constexpr int plane_stride(int n) { return n >= 4 ? n + 4 : n + 1; }

// shared memory of a plane pass for resolution n: plane [n][plane_stride(n)] floats +
// per-group scratch
int plane_smem_bytes(int n) {
  const int N1 = plane_n1(n), N2 = n / N1;
  const int groups = PL_THREADS / N1;
  const int sc = N1 > 1 ? N1 * (N2 + 1) : 1;
  return ((n * plane_stride(n) + 1) & ~1) * 4 + groups * (sc > n ? sc : n) * 8;
}

// Transforms the lines of a plane held in shared memory.  Line l starts at plane + l * ls
// and has element stride es.  DIR: 0 forward, 1 inverse, 2 forward + scale + inverse (scale
// uses the z-line's (kx, ky) = (line, y) and mu of the level).
template <int N1, int N2, int DIR>
__device__ void plane_lines(float* plane, int ls, int es, float2* scr, const Level& lv, int y_slab) {
  constexpr int n = N1 * N2;
  constexpr int groups = PL_THREADS / N1;
  const int g = threadIdx.x / N1, t = threadIdx.x % N1;
  float2* sc = scr + g * ((N1 > 1 && N1 * (N2 + 1) > n) ? N1 * (N2 + 1) : n);
  for (int base = 0; base < n / 2; base += groups) {
    const int p = base + g;
    const bool act = p < n / 2;
    const int pl = act ? p : 0;
    float* A = plane + (2 * pl) * ls;
    float* B = A + ls;
    if (DIR == 0 || DIR == 2) dct2_lines<N1, N2>(A, B, es, sc, t, act, lv.tw, lv.tw4);
    if (DIR == 2) {
      if (act) {
        const float inv_n3 = 1.f / (float)lv.n3;
        const float my = __ldg(lv.mu + y_slab);
        const float ma = __ldg(lv.mu + 2 * pl) + my, mb = __ldg(lv.mu + 2 * pl + 1) + my;
#pragma unroll
        for (int m = 0; m < N2; ++m) {
          const int k = t + N1 * m;
          const float me = __ldg(lv.mu + k);
          const float ia = 1.f / (1.f + lv.lam * (ma + me));
          const float ib = 1.f / (1.f + lv.lam * (mb + me));
          A[k * es] *= ia * ia * inv_n3;
          B[k * es] *= ib * ib * inv_n3;
        }
      }
      __syncwarp();
    }
    if (DIR == 1 || DIR == 2) dct3_lines<N1, N2>(A, B, es, sc, t, act, lv.tw, lv.tw4);
  }
}

template <int DIR>
__device__ void plane_lines_n(int n, float* plane, int ls, int es, float2* scr, const Level& lv, int y_slab) {
  switch (n) {
    case 2: plane_lines<1, 2, DIR>(plane, ls, es, scr, lv, y_slab); break;
    case 4: plane_lines<1, 4, DIR>(plane, ls, es, scr, lv, y_slab); break;
    case 8: plane_lines<1, 8, DIR>(plane, ls, es, scr, lv, y_slab); break;
    case 16: plane_lines<1, 16, DIR>(plane, ls, es, scr, lv, y_slab); break;
    case 32: plane_lines<4, 8, DIR>(plane, ls, es, scr, lv, y_slab); break;
    case 64: plane_lines<8, 8, DIR>(plane, ls, es, scr, lv, y_slab); break;
    case 128: plane_lines<8, 16, DIR>(plane, ls, es, scr, lv, y_slab); break;
    default: break;
  }
}

// Copies an n x n plane between global rows (row r at src + r * rstride, n contiguous
// floats) and the padded shared plane, 16 bytes per access for n >= 4, with several loads
// in flight per thread.
__device__ __forceinline__ void plane_load(float* __restrict__ plane, const float* __restrict__ src, int n, int lg,
                                           size_t rstride) {
  const int S = plane_stride(n);
  if (n >= 4) {
    const int nq = (n * n) >> 2;
#pragma unroll 16
    for (int i = threadIdx.x; i < nq; i += PL_THREADS) {
      const int e = i << 2, r = e >> lg, x = e & (n - 1);
      *reinterpret_cast<float4*>(plane + r * S + x) = __ldg(reinterpret_cast<const float4*>(src + r * rstride + x));
    }
  } else {
    for (int e = threadIdx.x; e < n * n; e += PL_THREADS) plane[(e >> lg) * S + (e & (n - 1))] = src[(e >> lg) * rstride + (e & (n - 1))];
  }
}

__device__ __forceinline__ void plane_store(float* __restrict__ dst, const float* __restrict__ plane, int n, int lg,
                                            size_t rstride) {
  const int S = plane_stride(n);
  if (n >= 4) {
    const int nq = (n * n) >> 2;
#pragma unroll 4
    for (int i = threadIdx.x; i < nq; i += PL_THREADS) {
      const int e = i << 2, r = e >> lg, x = e & (n - 1);
      *reinterpret_cast<float4*>(dst + r * rstride + x) = *reinterpret_cast<const float4*>(plane + r * S + x);
    }
  } else {
    for (int e = threadIdx.x; e < n * n; e += PL_THREADS) dst[(e >> lg) * rstride + (e & (n - 1))] = plane[(e >> lg) * S + (e & (n - 1))];
  }
}

// maps a plane item of a job to (level, index); `per` items per level (3n or n), only levels
// with 1 <= n <= 128 take part
__device__ __forceinline__ bool plane_item(const Job& J, int r, bool three, int& l, int& idx) {
  for (l = 0; l < J.L; ++l) {
    const int n = J.lev[l].n;
    if (n > 128) continue;
    const int c = three ? 3 * n : n;
    if (r < c) {
      idx = r;
      return true;
    }
    r -= c;
  }
  return false;
}

// Pass B: the two tridiagonal solves T^2 h = g of one (kx, ky) column of one channel, with
// the whole column in registers (N steps unrolled) and its reciprocal pivots in shared
// memory.  T has diagonal b_i = a + lambda deg(i) (deg 1 at the two ends, 2 inside) and
// off-diagonal -lambda, a = 1 + lambda (mu_kx + mu_ky).  Thomas: forward
// r_i = 1 / (b_i + lambda c_{i-1}) with c_i = -lambda r_i, g'_i = (g_i + lambda g'_{i-1}) r_i;
// backward h_{n-1} = g'_{n-1}, h_i = g'_i + lambda r_i h_{i+1}.  The column is read from
// global memory once and written once (scaled by the 1/n^2 of the inverse x and y
// transforms).  rs: this thread's pivots, stride COL_THREADS floats; volatile, so that the
// compiler reloads them in every sweep instead of holding all N in registers beside the
// column.  Consecutive threads take consecutive x, so every global access along z is
// coalesced and every shared access conflict-free.
constexpr int COL_THREADS = 128;

template <int N>
__device__ __forceinline__ void column_solve(float* __restrict__ t, volatile float* rs, float a, float lam,
                                             float scale) {
  constexpr int n2 = N * N;
  float v[N];
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = t[i * n2];
  float cp = 0.f, g = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {  // solve 1, forward (pivots)
    const float b = a + lam * ((i == 0 || i == N - 1) ? 1.f : 2.f);
    const float r = __frcp_rn(b + lam * cp);
    rs[i * COL_THREADS] = r;
    g = (v[i] + lam * g) * r;
    v[i] = g;
    cp = -lam * r;
  }
#pragma unroll
  for (int i = N - 2; i >= 0; --i) v[i] = v[i] + lam * rs[i * COL_THREADS] * v[i + 1];  // solve 1, backward
  g = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {  // solve 2, forward
    g = (v[i] + lam * g) * rs[i * COL_THREADS];
    v[i] = g;
  }
  t[(N - 1) * n2] = v[N - 1] * scale;
#pragma unroll
  for (int i = N - 2; i >= 0; --i) {  // solve 2, backward
    v[i] = v[i] + lam * rs[i * COL_THREADS] * v[i + 1];
    t[i * n2] = v[i] * scale;
  }
}

// an item is COL_THREADS consecutive columns (col = y n + x) of one channel of one level
__device__ __forceinline__ bool column_item(const Job& J, int r, int& l, int& c, int& col0) {
  for (l = 0; l < J.L; ++l) {
    const int n = J.lev[l].n;
    if (n > 128) continue;
    const int per = (n * n + COL_THREADS - 1) / COL_THREADS;
    if (r < 3 * per) {
      c = r / per;
      col0 = (r - c * per) * COL_THREADS;
      return true;
    }
    r -= 3 * per;
  }
  return false;
}

// One block of COL_THREADS per item.
__global__ void __launch_bounds__(COL_THREADS, 3) k_sobz(const Plan* __restrict__ P) {
  __shared__ float rs[128 * COL_THREADS];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_COL][nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_COL], nj, it);
    const Job& J = *P->jobs[j];
    if (!J.precondition) continue;
    int l, c, col0;
    if (!column_item(J, it - P->pre[ST_COL][j], l, c, col0)) continue;
    const Level& lv = J.lev[l];
    const int n = lv.n;
    const int col = col0 + threadIdx.x;
    if (n == 1 || col >= n * n) continue;  // a single vertex: T = 1
    const int x = col & (n - 1), y = col >> lv.lg;
    const float lam = lv.lam;
    const float a = 1.f + lam * (__ldg(lv.mu + x) + __ldg(lv.mu + y));
    const float scale = 1.f / (float)(n * n);
    float* t = lv.tmp + (size_t)c * lv.n3 + col;
    volatile float* r = rs + threadIdx.x;
    switch (n) {
      case 2: column_solve<2>(t, r, a, lam, scale); break;
      case 4: column_solve<4>(t, r, a, lam, scale); break;
      case 8: column_solve<8>(t, r, a, lam, scale); break;
      case 16: column_solve<16>(t, r, a, lam, scale); break;
      case 32: column_solve<32>(t, r, a, lam, scale); break;
      case 64: column_solve<64>(t, r, a, lam, scale); break;
      default: column_solve<128>(t, r, a, lam, scale); break;
    }
  }
}

// pass A: per (z-plane, channel), DCT-II along x then y
template <int PASS>
__global__ void __launch_bounds__(PL_THREADS, 2) k_sobp(const Plan* __restrict__ P) {
  static_assert(PASS == 0, "the z direction is solved by k_sobp_z");
  extern __shared__ float smem[];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_PLANE][nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_PLANE], nj, it);
    const Job& J = *P->jobs[j];
    if (!J.precondition) continue;
    int l, idx;
    if (!plane_item(J, it - P->pre[ST_PLANE][j], true, l, idx)) continue;
    const Level& lv = J.lev[l];
    const int n = lv.n, n3 = lv.n3, lg = lv.lg;
    if (n == 1) {  // no transform: copy g to tmp (the scale is 1)
      if (PASS == 0 && threadIdx.x == 0) lv.tmp[idx] = lv.g[idx];
      continue;
    }
    const int c = idx >> lg, q = idx & (n - 1);  // channel, plane index (z for A, y for B)
    const int S = plane_stride(n);
    float* plane = smem;
    float2* scr = reinterpret_cast<float2*>(smem + ((n * S + 1) & ~1));
    // A: rows y of z-plane q (row stride n);  B: rows z of the y-slab q (row stride n^2)
    const size_t off = (size_t)c * n3 + (PASS == 0 ? (size_t)q * n * n : (size_t)q * n);
    const size_t rstride = PASS == 0 ? (size_t)n : (size_t)n * n;
    plane_load(plane, (PASS == 0 ? lv.g : lv.tmp) + off, n, lg, rstride);
    __syncthreads();
    // the gradient lives on the vertices near the data: a plane that is all zero stays zero
    bool any = false;
    for (int e = threadIdx.x; e < n * n && !any; e += PL_THREADS) any = plane[(e >> lg) * S + (e & (n - 1))] != 0.f;
    if (!__syncthreads_or(any)) {
      plane_store(lv.tmp + off, plane, n, lg, rstride);
      __syncthreads();
      continue;
    }
    if (PASS == 0) {
      plane_lines_n<0>(n, plane, S, 1, scr, lv, 0);  // x-lines (rows)
      __syncthreads();
      plane_lines_n<0>(n, plane, 1, S, scr, lv, 0);  // y-lines (columns)
    } else {
      plane_lines_n<2>(n, plane, 1, S, scr, lv, q);  // z-lines (columns): forward, scale, inverse
    }
    __syncthreads();
    plane_store(lv.tmp + off, plane, n, lg, rstride);
    __syncthreads();
  }
}

// pass C: per (z-plane, channel): inverse along y and x; the preconditioned gradient goes
// back to tmp for the Adam kernel
__global__ void __launch_bounds__(PL_THREADS, 2) k_sobp_inv(const Plan* __restrict__ P) {
  extern __shared__ float smem[];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_PLANE][nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_PLANE], nj, it);
    const Job& J = *P->jobs[j];
    int l, idx;
    if (!plane_item(J, it - P->pre[ST_PLANE][j], true, l, idx)) continue;
    const Level& lv = J.lev[l];
    if (!J.precondition) continue;  // Adam then reads the raw gradient
    const int n = lv.n, n3 = lv.n3, lg = lv.lg;
    const int c = idx >> lg, z = idx & (n - 1);
    const int S = plane_stride(n);
    float* plane = smem;
    float2* scr = reinterpret_cast<float2*>(smem + ((n * S + 1) & ~1));
    const size_t base = (size_t)z * n * n;
    plane_load(plane, lv.tmp + (size_t)c * n3 + base, n, lg, n);
    __syncthreads();
    if (n > 1) {
      plane_lines_n<1>(n, plane, 1, S, scr, lv, 0);  // y-lines
      __syncthreads();
      plane_lines_n<1>(n, plane, S, 1, scr, lv, 0);  // x-lines
      __syncthreads();
    }
    plane_store(lv.tmp + (size_t)c * n3 + base, plane, n, lg, n);  // the preconditioned gradient
    __syncthreads();
  }
}

// Adam (PyTorch semantics) on every vertex of every level (n <= 128) from the preconditioned
// gradient in tmp (or the raw gradient without preconditioning): 4 vertices per thread,
// float4 loads of the three channel planes of g, m and v, float4 theta.
__device__ __forceinline__ bool adam_item(const Job& J, int r, int& l, int& q) {
  for (l = 0; l < J.L; ++l) {
    const int n = J.lev[l].n;
    if (n > 128) continue;
    const int cnt = (J.lev[l].n3 + 3) >> 2;
    if (r < cnt) {
      q = r;
      return true;
    }
    r -= cnt;
  }
  return false;
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
      float4 th[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) th[k] = lv.theta[e + k];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 g4 = *reinterpret_cast<const float4*>(gsrc + c * n3 + e);
        float4 m4 = *reinterpret_cast<const float4*>(lv.m + c * n3 + e);
        float4 v4 = *reinterpret_cast<const float4*>(lv.v + c * n3 + e);
        const float g[4] = {g4.x, g4.y, g4.z, g4.w};
        float* mm = &m4.x;
        float* vv = &v4.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          mm[k] = b1 * mm[k] + (1.f - b1) * g[k];
          vv[k] = b2 * vv[k] + (1.f - b2) * g[k] * g[k];
          (&th[k].x)[c] -= step * mm[k] / (sqrtf(vv[k]) * ib2 + eps);
        }
        *reinterpret_cast<float4*>(lv.m + c * n3 + e) = m4;
        *reinterpret_cast<float4*>(lv.v + c * n3 + e) = v4;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) lv.theta[e + k] = th[k];
    } else {  // n == 1
      float4 th = lv.theta[0];
      for (int c = 0; c < 3; ++c) {
        const float g = gsrc[c * n3];
        float m = b1 * lv.m[c * n3] + (1.f - b1) * g;
        float v = b2 * lv.v[c * n3] + (1.f - b2) * g * g;
        lv.m[c * n3] = m;
        lv.v[c * n3] = v;
        (&th.x)[c] -= step * m / (sqrtf(v) * ib2 + eps);
      }
      lv.theta[0] = th;
    }
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
  cudaFuncSetAttribute(k_sobp<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_sobp_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// part: 0 xy-forward, 1 z solve, 2 xy-inverse, 3 Adam, -1 all four
void launch_sobolev_plane(const Plan* P, int grid, int nmax, cudaStream_t s, int part) {
  const int smem = plane_smem_max(nmax);
  if (part < 0 || part == 0) k_sobp<0><<<grid, PL_THREADS, smem, s>>>(P);
  if (part < 0 || part == 1) k_sobz<<<grid * 3, COL_THREADS, 0, s>>>(P);
  if (part < 0 || part == 2) k_sobp_inv<<<grid, PL_THREADS, smem, s>>>(P);
  if (part < 0 || part == 3) k_adam<<<grid * 8, 256, 0, s>>>(P);
}

}  // namespace pdg
