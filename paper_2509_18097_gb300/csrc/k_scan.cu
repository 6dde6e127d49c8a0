// Exclusive prefix sums used by the counting sorts: cell offsets of the nearest-neighbour
// grids and row pointers of the per-level point -> vertex lists, over chunks of SCAN_CHUNK
// elements.  Per frame: chunk sums, a scan of the chunk sums, chunk scans.  Per step (the
// moving grid): chunk sums, then chunk scans that add up their preceding chunk sums.
#include "kernels.h"

namespace pdg {

// exclusive scan across a block of SCAN_THREADS (= 1024) threads; *total = block sum
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  const int pre = (w > 0 ? ws[w - 1] : 0) + x - v;
  if (total) *total = ws[31];
  __syncthreads();
  return pre;
}

__device__ __forceinline__ void load4(const int* in, int len, int base, int v[4]) {
  if (base + 3 < len) {
    const int4 q = *reinterpret_cast<const int4*>(in + base);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (base + k < len) ? in[base + k] : 0;
  }
}

__device__ void chunk_sum(const int* in, int len, int chunk, int* csum) {
  int v[4];
  load4(in, len, chunk * SCAN_CHUNK + threadIdx.x * 4, v);
  int tot;
  block_excl_scan(v[0] + v[1] + v[2] + v[3], &tot);
  if (threadIdx.x == 0) csum[chunk] = tot;
}

// Exclusive scan of one chunk starting from `prefix`; `last`: also out[len] = the total.
__device__ void chunk_scan_from(const int* in, int* out, int len, int chunk, int prefix, bool last) {
  int v[4];
  const int base = chunk * SCAN_CHUNK + threadIdx.x * 4;
  load4(in, len, base, v);
  int tot;
  int e = block_excl_scan(v[0] + v[1] + v[2] + v[3], &tot) + prefix;
  if (last && threadIdx.x == 0) out[len] = prefix + tot;
  if (base + 3 < len) {
    int4 q;
    q.x = e; e += v[0];
    q.y = e; e += v[1];
    q.z = e; e += v[2];
    q.w = e;
    *reinterpret_cast<int4*>(out + base) = q;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (base + k < len) out[base + k] = e;
      e += v[k];
    }
  }
}

__device__ void chunk_scan(const int* in, int* out, int len, int chunk, const int* csum) {
  int v[4];
  const int base = chunk * SCAN_CHUNK + threadIdx.x * 4;
  load4(in, len, base, v);
  int e = block_excl_scan(v[0] + v[1] + v[2] + v[3], nullptr) + csum[chunk];
  if (base + 3 < len) {
    int4 q;
    q.x = e; e += v[0];
    q.y = e; e += v[1];
    q.z = e; e += v[2];
    q.w = e;
    *reinterpret_cast<int4*>(out + base) = q;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (base + k < len) out[base + k] = e;
      e += v[k];
    }
  }
}

// exclusive scan of the chunk sums in place (one block); out[len] = total
__device__ void scan_sums(int* csum, int nch, int* out, int len) {
  int carry = 0;
  for (int b = 0; b < nch; b += SCAN_THREADS) {
    const int i = b + threadIdx.x;
    const int v = i < nch ? csum[i] : 0;
    int tot;
    const int e = block_excl_scan(v, &tot);
    if (i < nch) csum[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) out[len] = carry;
}

// ---- moving grid of every job of a plan (per step) ------------------------------------

__device__ __forceinline__ int mov_len(const Job& J) {
  const int G = 1 << J.mov.bits;
  return 2 * G * G * G;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_mov_scan_a(const Plan* __restrict__ P) {
  const int nj = P->n_jobs;
  const int total = P->pre[ST_MOVCH][nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_MOVCH], nj, it);
    const Job& J = *P->jobs[j];
    chunk_sum(J.mov.hist, mov_len(J), it - P->pre[ST_MOVCH][j], J.mov.csum);
  }
}

// Second phase of the moving grid's scan: every block adds up the chunk sums before its
// own chunk itself (at most a few thousand, read from L2) instead of waiting for a separate
// scan of the chunk sums, then scans its chunk; the last chunk also writes the total.
__global__ void __launch_bounds__(SCAN_THREADS) k_mov_scan_c(const Plan* __restrict__ P) {
  __shared__ int red[32];
  const int nj = P->n_jobs;
  const int total = P->pre[ST_MOVCH][nj];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int j = find_job(P->pre[ST_MOVCH], nj, it);
    const Job& J = *P->jobs[j];
    const int chunk = it - P->pre[ST_MOVCH][j];
    const int len = mov_len(J);
    const int nch = (len + SCAN_CHUNK - 1) / SCAN_CHUNK;
    int part = 0;
    for (int c = threadIdx.x; c < chunk; c += SCAN_THREADS) part += __ldg(J.mov.csum + c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    int prefix = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) prefix += red[w];
    __syncthreads();
    chunk_scan_from(J.mov.hist, J.mov.off, len, chunk, prefix, chunk == nch - 1);
  }
}

void launch_mov_scan(const Plan* P, int grid, cudaStream_t s) {
  k_mov_scan_a<<<grid, SCAN_THREADS, 0, s>>>(P);
  k_mov_scan_c<<<grid, SCAN_THREADS, 0, s>>>(P);
}

// ---- one explicit segment (per-frame structures) --------------------------------------

__global__ void __launch_bounds__(SCAN_THREADS) k_seg_scan_a(ScanSeg g) {
  const int nch = (g.len + SCAN_CHUNK - 1) / SCAN_CHUNK;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) chunk_sum(g.in, g.len, c, g.csum);
}
__global__ void __launch_bounds__(SCAN_THREADS) k_seg_scan_b(ScanSeg g) {
  scan_sums(g.csum, (g.len + SCAN_CHUNK - 1) / SCAN_CHUNK, g.out, g.len);
}
__global__ void __launch_bounds__(SCAN_THREADS) k_seg_scan_c(ScanSeg g) {
  const int nch = (g.len + SCAN_CHUNK - 1) / SCAN_CHUNK;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) chunk_scan(g.in, g.out, g.len, c, g.csum);
}

void launch_scan_segments(const ScanSeg* hsegs, int nseg, ScanSeg*, int*, cudaStream_t s) {
  for (int i = 0; i < nseg; ++i) {
    const ScanSeg g = hsegs[i];
    const int nch = (g.len + SCAN_CHUNK - 1) / SCAN_CHUNK;
    const int grid = nch < 2048 ? nch : 2048;
    k_seg_scan_a<<<grid, SCAN_THREADS, 0, s>>>(g);
    k_seg_scan_b<<<1, SCAN_THREADS, 0, s>>>(g);
    k_seg_scan_c<<<grid, SCAN_THREADS, 0, s>>>(g);
  }
}

}  // namespace pdg
