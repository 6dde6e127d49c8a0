// Host-side launchers of the libpdg kernels (each defined next to its kernels).
#pragma once
#include "pdg_internal.cuh"

namespace pdg {

// per step (plan-driven; `grid` = blocks of the persistent launch)
void launch_plan(Plan* P, cudaStream_t s);
void launch_interp(const Plan* P, int grid, cudaStream_t s, int bump);
void launch_mov_scan(const Plan* P, int grid, cudaStream_t s);
void launch_mov_scatter(const Plan* P, int grid, cudaStream_t s);
// count: the instance that counts candidates and exact ties
void launch_nn(const Plan* P, int grid, cudaStream_t s, bool count);
void launch_nn_hard(const Plan* P, int grid, cudaStream_t s, bool count);
void launch_iso_edges(const Plan* P, int grid, cudaStream_t s);
void launch_assemble(const Plan* P, int grid, cudaStream_t s);
void launch_adjoint(const Plan* P, int grid, cudaStream_t s);
void launch_sobolev_tiles(const Plan* P, int sms, int nlo, int nhi, int nsmem, cudaStream_t s);
void launch_sobolev_plane(const Plan* P, int grid, int nmax, cudaStream_t s, int part = -1);
void launch_loss(const Plan* P, int grid, cudaStream_t s);

// per frame / per call (one job)
void launch_pack4(const float* in, float4* out, int n, cudaStream_t s);
void launch_unpack4(const float4* in, float* out, int n, cudaStream_t s);
void launch_check_finite(const float* in, int n, int* flag, cudaStream_t s);
void launch_frame_points(Job* J, int Q, int E, cudaStream_t s);
void launch_tgt_build(Job* J, const Job& hJ, cudaStream_t s);
void launch_csr_build(Job* J, const Job& hJ, cudaStream_t s);
void launch_end_frame(Job* J, int V, cudaStream_t s);
void launch_deform(const Job* J, const float* in, float* out, int n, cudaStream_t s);

// generic exclusive scans over explicit segments (per-frame structures)
struct ScanSeg {
  const int* in;
  int* out;   // [len + 1]
  int len;
  int* csum;  // [ceil(len / SCAN_CHUNK)]
};
void launch_scan_segments(const ScanSeg* hsegs, int nseg, ScanSeg* dsegs_scratch, int* dpre_scratch,
                          cudaStream_t s);

int sobolev_smem_bytes(int n);
void sobolev_configure();
void sobolev_plane_configure();
int plane_smem_bytes(int n);
int plane_smem_max(int nmax);
void launch_aos_to_soa(const float* in, float* out, int n3, cudaStream_t s, int C = 3);
void launch_zmask(Job* J, const Job& hJ, cudaStream_t s);
void launch_sobz_pivots(float* piv, int* slow, const float* mu, int n, float lam, cudaStream_t s);

// template-mesh fit (k_mesh.cu)
void launch_mesh_points(Job* J, int V, cudaStream_t s);
void launch_mesh_solve(const int* v2e_ptr, const int* v2e, const int2* edges, const float4* b, float4* h, float4* r,
                       float4* d0, float4* d1, int V, float lam, float emax, int iters, cudaStream_t s);
void launch_mesh_adam(float4* x, const float4* g, float4* m, float4* v, int V, float lr, float b1, float b2, float eps,
                      float bias1, float ibias2, cudaStream_t s);

// misc conversions
void launch_soa_to_aos(const float* in, float* out, int n3, cudaStream_t s, int C = 3);
void launch_pack_theta(const float* in, float4* th, float4* tht, int n3, int C, cudaStream_t s);
void launch_unpack_theta(const float4* th, const float4* tht, float* out, int n3, int C, cudaStream_t s);
void launch_aos_to_float4(const float* in, float4* out, int n, cudaStream_t s);
void launch_copy_int(const int* in, int* out, int n, cudaStream_t s);

}  // namespace pdg
