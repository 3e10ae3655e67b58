// Surrogate-guided bisection (not in the paper): the N_b bisection steps of
// every candidate of a round are first taken on the learned signed distance
// (predicted collision iff sd_hat < margin), all of them in one launch of the
// tensor-core forward kernel (ezo_mlp_tc.cu) on the brackets set up here; the
// bisection kernel then verifies each end point with one exact check and
// redoes the exact bisection of Sec. IV-B for candidates whose end point is
// not in collision.
//
// Row r of the MLP batch is candidate tile.y + (r % kTile) of bisection tile
// r / kTile (the same numbering the bisection kernel uses).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ezo_kernels_common.cuh"

namespace ezo {

// c_proj and c - c_proj per row (FP64 projection, stored in FP32), bracket [0, 1]
template <int NDOF>
__global__ void k_sbis_init(BatchView v) {
  const int n_tiles = v.summary->n_bisect_tiles;
  const int rows = n_tiles * kTile;
  if (blockIdx.x == 0 && threadIdx.x == 0) *v.s_rows = rows;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const int2 tile = v.bisect_tiles[r / kTile];
    const int c = tile.y + r % kTile;
    const SegState& st = v.st[tile.x];
    v.s_lo[r] = 0.f;
    v.s_hi[r] = 1.f;
    v.s_bits[r] = 0u;
    v.s_ok[r] = 0;
    if (c >= st.n_cand) {
      for (int j = 0; j < 8; ++j) v.s_p32[r * 8 + j] = v.s_d32[r * 8 + j] = 0.f;
      continue;
    }
    const int n = v.n;
    const int si = v.cand_idx[st.cand_off + c];
    const float* S = v.S + (long long)n * st.sample_off;
    double cs[NDOF], p[NDOF];
#pragma unroll
    for (int j = 0; j < NDOF; ++j) cs[j] = (j < n) ? (double)S[(long long)j * st.s_cap + si] : 0.0;
    project_fp64<NDOF>(cs, v.v1 + (long long)tile.x * n, v.v2 + (long long)tile.x * n, n, p);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v.s_p32[r * 8 + j] = (j < n && j < NDOF) ? (float)p[j] : 0.f;
      v.s_d32[r * 8 + j] = (j < n && j < NDOF) ? (float)(cs[j] - p[j]) : 0.f;
    }
  }
}

cudaError_t launch_sbis_init(const BatchView& v, int grid, cudaStream_t s) {
  EZO_DISPATCH_NDOF(v.n, { k_sbis_init<ND><<<grid, 256, 0, s>>>(v); });
  return cudaGetLastError();
}

}  // namespace ezo
