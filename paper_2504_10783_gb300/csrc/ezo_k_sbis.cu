// Surrogate-guided bisection (not in the paper): the N_b bisection steps of
// every candidate of a round are first taken on the learned signed distance
// (predicted collision iff sd_hat < margin), evaluated for all candidates at
// once as one MLP batch per step; the bisection kernel then verifies each end
// point with one exact check and redoes the exact bisection of Sec. IV-B for
// candidates whose end point is not in collision.
//
// Row r of the MLP batch is candidate tile.y + (r % kTile) of bisection tile
// r / kTile (the same numbering the bisection kernel uses).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ezo_kernels_common.cuh"

namespace ezo {

constexpr int kFeat = 64;

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

// features [sin q, cos q, 0..] of the midpoint of each row's bracket
__global__ void k_sbis_mid(BatchView v, __nv_bfloat16* __restrict__ X) {
  const int rows = *v.s_rows;
  const int n = v.n;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const float f = 0.5f * (v.s_lo[r] + v.s_hi[r]);
    for (int k = 0; k < kFeat; ++k) {
      float val = 0.f;
      if (k < n) val = sinf(fmaf(f, v.s_d32[r * 8 + k], v.s_p32[r * 8 + k]));
      else if (k < 2 * n) val = cosf(fmaf(f, v.s_d32[r * 8 + k - n], v.s_p32[r * 8 + k - n]));
      X[(long long)r * kFeat + k] = __float2bfloat16(val);
    }
  }
}

// one surrogate bisection step: keep the end predicted in collision
__global__ void k_sbis_update(BatchView v, const float* __restrict__ yhat, int step) {
  const int rows = *v.s_rows;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const float lo = v.s_lo[r], hi = v.s_hi[r];
    const float f = 0.5f * (lo + hi);
    if (yhat[r] < v.sbis_margin) {
      v.s_hi[r] = f;
      v.s_bits[r] |= 1u << step;
    } else {
      v.s_lo[r] = f;
    }
  }
}

cudaError_t launch_sbis_init(const BatchView& v, int grid, cudaStream_t s) {
  EZO_DISPATCH_NDOF(v.n, { k_sbis_init<ND><<<grid, 256, 0, s>>>(v); });
  return cudaGetLastError();
}

cudaError_t launch_sbis_mid(const BatchView& v, void* X, int grid, cudaStream_t s) {
  k_sbis_mid<<<grid, 256, 0, s>>>(v, static_cast<__nv_bfloat16*>(X));
  return cudaGetLastError();
}

cudaError_t launch_sbis_update(const BatchView& v, const float* yhat, int step, int grid, cudaStream_t s) {
  k_sbis_update<<<grid, 256, 0, s>>>(v, yhat, step);
  return cudaGetLastError();
}

}  // namespace ezo
