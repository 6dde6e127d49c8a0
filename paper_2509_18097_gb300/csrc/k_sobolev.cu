// Grid Sobolev preconditioning (Sec. 3.2, Eq. 3) fused with the Adam update (Sec. 3.6) for
// levels of 256^3 vertices, whose planes do not fit in shared memory, and for levels whose
// resolution has a factor 3 (2^a 3^b vertices per axis; powers of two up to 128 use the
// three-pass plane path of k_sobolev_plane.cu).
//
// L_l is the 6-neighbour graph Laplacian of the level's vertex grid with a free
// boundary; it is the Kronecker sum of three path-graph Laplacians whose eigenvectors are
// the DCT-II basis vectors cos(pi k (i + 1/2) / n) with eigenvalues mu_k = 4 sin^2(pi k / 2n).
// Hence (I + lambda L)^{-2} g = C^{-1} diag((1 + lambda (mu_kx + mu_ky + mu_kz))^{-2}) C g
// with C the separable (unnormalised) 3-D DCT-II.  It is applied in five passes over the
// level, each pass loading tiles of 32 lines x 3 channels into shared memory:
//   1: x-lines of g, DCT-II                   -> tmp
//   2: y-lines,      DCT-II                   -> tmp
//   3: z-lines,      DCT-II, spectral scale (incl. 1/n^3), inverse -> tmp
//   4: y-lines,      inverse
//   5: x-lines,      inverse, then Adam on theta/m/v of those vertices.
// A line transform of length n = 2^a 3^b is done two lines at a time by one warp: the lines
// are packed as the real and imaginary parts of one complex sequence (after the
// even/odd reordering that turns a DCT-II into a DFT, valid for odd n too), transformed by
// a mixed radix-2/3 Stockham FFT in shared memory (a radix-2 stages, then b radix-3
// stages), and separated with the conjugate-symmetry of real spectra.
#include "kernels.h"

namespace pdg {

constexpr int TS = 33;  // padded tile stride (floats) between consecutive elements of a line

// floats of a tile (one channel: n elements x TS lines), rounded up to an even count so that
// the float2 FFT scratch after it is 8-byte aligned for odd n too
__host__ __device__ constexpr int tile_floats(int n) { return (n * TS + 1) & ~1; }

int sobolev_smem_bytes(int n) { return tile_floats(n) * 4 + SOB_WARPS * 2 * n * 8; }

// Stockham autosort FFT of n = 2^a 3^b points, one warp, ping-ponging between src and dst;
// returns the buffer holding the result (natural order).  Stage with radix R after Ns
// points' worth of earlier radices: for j < n / R, k = j mod Ns, the R inputs
// src[j + r n / R] times exp(-2 pi i r k / (Ns R)) go through an R-point DFT into
// dst[(j - k) R + k + r Ns].  tw[m] = exp(-2 pi i m / n).
template <bool INV>
__device__ __forceinline__ float2* fft_warp(float2* src, float2* dst, const float2* __restrict__ tw, int n,
                                            int lane) {
  const int half = n >> 1;
  const int p2 = n & -n;  // 2^a
  for (int Ns = 1; Ns < p2; Ns <<= 1) {
    const int step = half / Ns;
    for (int j = lane; j < half; j += 32) {
      const int k = j & (Ns - 1);
      float2 w = __ldg(tw + k * step);
      if (INV) w.y = -w.y;
      const float2 v0 = src[j], v1 = src[j + half];
      const float2 t = make_float2(v1.x * w.x - v1.y * w.y, v1.x * w.y + v1.y * w.x);
      const int d = ((j - k) << 1) + k;
      dst[d] = make_float2(v0.x + t.x, v0.y + t.y);
      dst[d + Ns] = make_float2(v0.x - t.x, v0.y - t.y);
    }
    __syncwarp();
    float2* sw = src;
    src = dst;
    dst = sw;
  }
  // radix 3: y_0 = a + s, y_{1,2} = a - s / 2 -+ i (sqrt(3) / 2) (b - c), s = b + c (forward);
  // the inverse conjugates the twiddles and the sign of the i term
  const int third = n / 3;
  const float h3 = INV ? -0.866025403784438647f : 0.866025403784438647f;
  for (int Ns = p2; Ns < n; Ns *= 3) {
    const int step = n / (3 * Ns);
    for (int j = lane; j < third; j += 32) {
      const int k = j % Ns;
      float2 w1 = __ldg(tw + k * step), w2 = __ldg(tw + 2 * k * step);
      if (INV) {
        w1.y = -w1.y;
        w2.y = -w2.y;
      }
      const float2 a = src[j], b0 = src[j + third], c0 = src[j + 2 * third];
      const float2 b = make_float2(b0.x * w1.x - b0.y * w1.y, b0.x * w1.y + b0.y * w1.x);
      const float2 c = make_float2(c0.x * w2.x - c0.y * w2.y, c0.x * w2.y + c0.y * w2.x);
      const float2 sm = make_float2(b.x + c.x, b.y + c.y), df = make_float2(b.x - c.x, b.y - c.y);
      const float2 m = make_float2(a.x - 0.5f * sm.x, a.y - 0.5f * sm.y);
      const int d = (j - k) * 3 + k;
      dst[d] = make_float2(a.x + sm.x, a.y + sm.y);
      dst[d + Ns] = make_float2(m.x + h3 * df.y, m.y - h3 * df.x);
      dst[d + 2 * Ns] = make_float2(m.x - h3 * df.y, m.y + h3 * df.x);
    }
    __syncwarp();
    float2* sw = src;
    src = dst;
    dst = sw;
  }
  return src;
}

// even/odd reordering of a DCT-II input (any n): v[j] = x[2j] for j < ceil(n / 2), then
// the odd elements in reverse
__device__ __forceinline__ int dct_src(int j, int n) { return j < ((n + 1) >> 1) ? 2 * j : 2 * (n - 1 - j) + 1; }

// A, B <- C A, C B (unnormalised DCT-II), lines with element stride TS
__device__ void dct2_pair(float* A, float* B, int n, float2* b0, float2* b1, const float2* __restrict__ tw,
                          const float2* __restrict__ tw4, int lane) {
  for (int j = lane; j < n; j += 32) {
    const int s = dct_src(j, n) * TS;
    b0[j] = make_float2(A[s], B[s]);
  }
  __syncwarp();
  const float2* Z = fft_warp<false>(b0, b1, tw, n, lane);
  for (int k = lane; k < n; k += 32) {
    const float2 zk = Z[k];
    const float2 zc = Z[k ? n - k : 0];
    // V_A = (Z_k + conj Z_{n-k}) / 2,  V_B = (Z_k - conj Z_{n-k}) / (2i)
    const float2 va = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
    const float2 vb = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
    const float2 w = __ldg(tw4 + k);  // exp(-i pi k / 2n)
    A[k * TS] = w.x * va.x - w.y * va.y;
    B[k * TS] = w.x * vb.x - w.y * vb.y;
  }
  __syncwarp();
}

// A, B <- n C^{-1} A, n C^{-1} B (the 1/n is folded into the spectral scale)
__device__ void dct3_pair(float* A, float* B, int n, float2* b0, float2* b1, const float2* __restrict__ tw,
                          const float2* __restrict__ tw4, int lane) {
  for (int k = lane; k < n; k += 32) {
    const float a = A[k * TS], an = k ? A[(n - k) * TS] : 0.f;
    const float b = B[k * TS], bn = k ? B[(n - k) * TS] : 0.f;
    float2 w = __ldg(tw4 + k);
    w.y = -w.y;  // exp(+i pi k / 2n)
    // V = w (X_k - i X_{n-k});  Z = V_A + i V_B
    const float2 va = make_float2(w.x * a + w.y * an, w.y * a - w.x * an);
    const float2 vb = make_float2(w.x * b + w.y * bn, w.y * b - w.x * bn);
    b0[k] = make_float2(va.x - vb.y, va.y + vb.x);
  }
  __syncwarp();
  const float2* z = fft_warp<true>(b0, b1, tw, n, lane);
  for (int j = lane; j < n; j += 32) {
    const int s = dct_src(j, n) * TS;
    A[s] = z[j].x;
    B[s] = z[j].y;
  }
  __syncwarp();
}

// flat vertex index of element e of line r of a level (axis 0: x-lines, r = z n + y;
// axis 1: y-lines, r = z n + x; axis 2: z-lines, r = y n + x); lg = log2(n), or -1 when n
// is not a power of two
template <int AXIS>
__device__ __forceinline__ int eaddr(int n, int lg, int r, int e) {
  if (lg >= 0) {
    if (AXIS == 0) return (r << lg) + e;
    const int lo = r & (n - 1), hi = r >> lg;
    if (AXIS == 1) return (((hi << lg) + e) << lg) + lo;
    return (((e << lg) + hi) << lg) + lo;
  }
  if (AXIS == 0) return r * n + e;
  const int hi = r / n, lo = r - hi * n;
  if (AXIS == 1) return (hi * n + e) * n + lo;
  return (e * n + hi) * n + lo;
}

// (quotient, remainder) of i by n, by shifts when n = 2^lg
__device__ __forceinline__ void divmod_n(int i, int n, int lg, int& q, int& rm) {
  q = lg >= 0 ? i >> lg : i / n;
  rm = i - q * n;
}

// One pass over the tiles of the tile-path levels with nlo < n <= nhi (a size class, launched
// with the shared memory of its largest level); tiles of the other class are skipped.
template <int PASS>
__global__ void __launch_bounds__(SOB_THREADS) k_sob(const Plan* __restrict__ P, int nlo, int nhi) {
  constexpr int AXIS = (PASS == 1 || PASS == 5) ? 0 : (PASS == 2 || PASS == 4) ? 1 : 2;
  extern __shared__ float smem[];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_TILE][nj];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_TILE], nj, it);
    const Job& J = *P->jobs[j];
    const bool pre = J.precondition != 0;
    if (PASS < 5 && !pre) continue;
    int t = it - P->pre[ST_TILE][j];
    int l = 0;
    for (; l < J.L; ++l) {
      if (!tile_level(J.lev[l].n)) continue;
      if (t < J.lev[l].tiles) break;
      t -= J.lev[l].tiles;
    }
    if (l >= J.L || J.lev[l].n <= nlo || J.lev[l].n > nhi) continue;
    const Level& lv = J.lev[l];
    const int n = lv.n, lg = lv.lg, n3 = lv.n3, nl = n * n;
    // a tile: TILE_LINES lines of one channel (channel-major over the level's tiles)
    const int lt = (nl + TILE_LINES - 1) / TILE_LINES;
    const int c = t / lt;
    const int r0 = (t - c * lt) * TILE_LINES;
    float* tl = smem;
    float2* b0 = reinterpret_cast<float2*>(smem + tile_floats(n)) + warp * 2 * n;
    float2* b1 = b0 + n;
    const float* src = ((PASS == 1 || (PASS == 5 && !pre)) ? lv.g : lv.tmp) + (size_t)c * n3;

    for (int idx = threadIdx.x; idx < TILE_LINES * n; idx += SOB_THREADS) {
      int tt, e;
      if (AXIS == 0) divmod_n(idx, n, lg, tt, e);
      else { e = idx >> 5; tt = idx & 31; }
      const int r = r0 + tt;
      tl[e * TS + tt] = r < nl ? src[eaddr<AXIS>(n, lg, r, e)] : 0.f;
    }
    __syncthreads();

    if (n > 1 && pre) {
      for (int pp = warp; pp < TILE_LINES / 2; pp += SOB_WARPS) {
        const int tt = pp * 2;
        float* A = tl + tt;
        float* B = A + 1;
        if (PASS == 1 || PASS == 2 || PASS == 3) dct2_pair(A, B, n, b0, b1, lv.tw, lv.tw4, lane);
        if (PASS == 3) {
          // spectral scale (1 + lambda (mu_kx + mu_ky + mu_kz))^{-2} / n^3; lines are
          // z-lines r = ky n + kx
          const int ra = r0 + tt, rb = ra + 1;
          // (lines past n^2 in the last tile are padding: their indices are wrapped into range)
          int qa, xa, qb, xb;
          divmod_n(ra, n, lg, qa, xa);
          divmod_n(rb, n, lg, qb, xb);
          const float ma = __ldg(lv.mu + xa) + __ldg(lv.mu + qa % n);
          const float mb = __ldg(lv.mu + xb) + __ldg(lv.mu + qb % n);
          const float inv_n3 = 1.f / (float)n3;
          for (int e = lane; e < n; e += 32) {
            const float me = __ldg(lv.mu + e);
            const float ia = 1.f / (1.f + lv.lam * (ma + me));
            const float ib = 1.f / (1.f + lv.lam * (mb + me));
            A[e * TS] *= ia * ia * inv_n3;
            B[e * TS] *= ib * ib * inv_n3;
          }
          __syncwarp();
        }
        if (PASS >= 3) dct3_pair(A, B, n, b0, b1, lv.tw, lv.tw4, lane);
      }
    }
    __syncthreads();

    if (PASS < 5) {
      float* dst = lv.tmp + (size_t)c * n3;
      for (int idx = threadIdx.x; idx < TILE_LINES * n; idx += SOB_THREADS) {
        int tt, e;
        if (AXIS == 0) divmod_n(idx, n, lg, tt, e);
        else { e = idx >> 5; tt = idx & 31; }
        const int r = r0 + tt;
        if (r < nl) dst[eaddr<AXIS>(n, lg, r, e)] = tl[e * TS + tt];
      }
    } else {
      // Adam (PyTorch semantics) on channel c of the vertices of these x-lines (the other
      // channels' tiles write the other components of theta: disjoint 4-byte words)
      const float b1f = J.beta1, b2f = J.beta2;
      const float step = lv.lr * J.bias[0];
      const float ib2 = J.bias[1];
      float* tmpc = lv.tmp + (size_t)c * n3;
      float* mc = lv.m + (size_t)c * n3;
      float* vc = lv.v + (size_t)c * n3;
      for (int idx = threadIdx.x; idx < TILE_LINES * n; idx += SOB_THREADS) {
        int tt, x;
        divmod_n(idx, n, lg, tt, x);
        const int r = r0 + tt;
        if (r >= nl) continue;
        const int v = r * n + x;
        const float g = tl[x * TS + tt];
        if (J.no_adam) {
          tmpc[v] = g;
          continue;
        }
        if (J.keep_pgrad) tmpc[v] = g;
        float m = mc[v], vv = vc[v];
        m = b1f * m + (1.f - b1f) * g;
        vv = b2f * vv + (1.f - b2f) * g * g;
        mc[v] = m;
        vc[v] = vv;
        float* th = reinterpret_cast<float*>(lv.theta + v) + c;
        *th -= step * m / (sqrtf(vv) * ib2 + J.eps);
      }
    }
    __syncthreads();
  }
}

void sobolev_configure() {
  const int smem = sobolev_smem_bytes(256);
  cudaFuncSetAttribute(k_sob<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_sob<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_sob<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_sob<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_sob<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// the five passes over the tile levels with nlo < n <= nhi; nsmem: the largest of them
// (sets the shared memory per block and so the blocks per SM)
void launch_sobolev_tiles(const Plan* P, int sms, int nlo, int nhi, int nsmem, cudaStream_t s) {
  const int smem = sobolev_smem_bytes(nsmem);
  const int grid = sms * std::max(1, std::min(8, (227 * 1024) / smem));
  k_sob<1><<<grid, SOB_THREADS, smem, s>>>(P, nlo, nhi);
  k_sob<2><<<grid, SOB_THREADS, smem, s>>>(P, nlo, nhi);
  k_sob<3><<<grid, SOB_THREADS, smem, s>>>(P, nlo, nhi);
  k_sob<4><<<grid, SOB_THREADS, smem, s>>>(P, nlo, nhi);
  k_sob<5><<<grid, SOB_THREADS, smem, s>>>(P, nlo, nhi);
}

}  // namespace pdg
