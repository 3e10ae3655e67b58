// Learned signed-distance surrogate: a small MLP sd_hat(q) from the features
// [sin q_1 .. sin q_n, cos q_1 .. cos q_n] (zero-padded to F = 64) through
// three hidden layers of width H = 256 with SiLU to one output. Not part of
// the paper: it only orders and prefilters bisection candidates; every
// certification sample is still checked exactly.
//
// Weights are kept in FP32 (master, Adam moments) and in BF16 copies that
// feed the tensor cores: every hidden-layer product of training is a
// BF16 x BF16 -> FP32 GEMM on tcgen05.mma with the accumulator in tensor
// memory (ezo_mlp_gemm_tc.cu), bias/SiLU (forward) and SiLU' (backward) fused
// into its epilogue; inference runs the whole network in one tensor-core
// kernel (ezo_mlp_tc.cu). The output layer (H -> 1), the column sums and Adam
// are small CUDA-core kernels.
//
// GEMM convention ("NT"): C[M x N] = A[M x K] B[N x K]^T, both operands
// K-contiguous (row-major with leading dimensions lda, ldb). Forward
// activations are also written transposed so that the weight gradients are
// NT products too.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ezo.h"
#include "ezo_engine.cuh"
#include "ezo_mlp.cuh"

namespace ezo {

// tensor-core forward pass (ezo_mlp_tc.cu)
size_t mlp_tc_image_bytes();
cudaError_t mlp_tc_build_image(const void* W1, const void* W2, const void* W3, void* img, cudaStream_t s);
cudaError_t mlp_tc_forward(const float* q, long long ldq, int n, long long rows_cap, const int* m_dev,
                           const void* img, const float* b1, const float* b2, const float* b3, const float* w4,
                           const float* b4, float* y, int* err, cudaStream_t s);
cudaError_t mlp_tc_bisect(int n, long long rows_cap, const int* m_dev, const void* img, const float* b1,
                          const float* b2, const float* b3, const float* w4, const float* b4, const float* s_p32,
                          const float* s_d32, float* s_lo, float* s_hi, uint32_t* s_bits, int n_b, float margin,
                          int* err, cudaStream_t s);

constexpr int kF = 64;   // padded input features
constexpr int kH = 256;  // hidden width


__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// ------------------------------------------------------------ small kernels --
// features of configuration i: sin q_j, cos q_j (j < n), zero padding to kF;
// row-major [rows x kF] and transposed [kF x ldt]. A block takes 64 rows at a
// time through a shared-memory tile, so both outputs are written along their
// contiguous dimension.
__global__ void __launch_bounds__(256) k_features(const float* __restrict__ q, long long ldq, int n, long long N,
                                                  __nv_bfloat16* __restrict__ X, __nv_bfloat16* __restrict__ Xt,
                                                  int ldt) {
  __shared__ float tile[64][kF + 1];
  for (long long r0 = (long long)blockIdx.x * 64; r0 < N; r0 += (long long)gridDim.x * 64) {
    for (int e = threadIdx.x; e < 64 * kF; e += blockDim.x) {
      const int rr = e & 63, f = e >> 6;
      const long long i = r0 + rr;
      float v = 0.f;
      if (i < N) {
        if (f < n) v = sinf(q[(long long)f * ldq + i]);
        else if (f < 2 * n) v = cosf(q[(long long)(f - n) * ldq + i]);
      }
      tile[rr][f] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * kF; e += blockDim.x) {
      const int rr = e / kF, f = e % kF;
      if (r0 + rr < N) X[(r0 + rr) * kF + f] = __float2bfloat16(tile[rr][f]);
    }
    if (Xt) {
      for (int e = threadIdx.x; e < 64 * kF; e += blockDim.x) {
        const int f = e >> 6, rr = e & 63;
        if (r0 + rr < N) Xt[(long long)f * ldt + r0 + rr] = __float2bfloat16(tile[rr][f]);
      }
    }
    __syncthreads();
  }
}

// y_i = H3_i . w4 + b4, one warp per row
__global__ void k_out(const __nv_bfloat16* __restrict__ H3, const float* __restrict__ w4, const float* __restrict__ b4,
                      long long N, const int* m_dev, float* __restrict__ y) {
  const long long lim = m_dev ? min((long long)*m_dev, N) : N;
  const int lane = threadIdx.x & 31;
  for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < lim;
       i += ((long long)gridDim.x * blockDim.x) >> 5) {
    float s = 0.f;
    for (int c = lane; c < kH; c += 32) s = fmaf(__bfloat162float(H3[i * kH + c]), w4[c], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = s + b4[0];
  }
}

// loss 1/N sum (y - t)^2, dy = 2 (y - t) / N, dZ3 = dy w4 * SiLU'(Z3)
// (row-major and transposed BF16); the block's partial sums of dw4 = sum_i
// dy_i H3_i, db4 = sum_i dy_i and the loss go to part[blockIdx.x] (kOutPart
// floats: kH columns, then db4 and the loss), summed per warp and then over
// the warps in a fixed order; k_out_reduce adds the blocks' partials in a
// fixed order, so training is reproducible bit for bit.
constexpr int kOutPart = kH + 2;
constexpr int kOutBlocks = 256;

__global__ void __launch_bounds__(256) k_out_backward(const float* __restrict__ y, const float* __restrict__ t,
                                                      const float* __restrict__ Z3, const __nv_bfloat16* __restrict__ H3,
                                                      const float* __restrict__ w4, int N,
                                                      __nv_bfloat16* __restrict__ dZ3, __nv_bfloat16* __restrict__ dZ3t,
                                                      float* __restrict__ part_out) {
  __shared__ float sw[8][kH];
  __shared__ float sbl[8][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float part[kH / 32];
#pragma unroll
  for (int k = 0; k < kH / 32; ++k) part[k] = 0.f;
  float pb = 0.f, pl = 0.f;  // the same on every lane of the warp (one row per warp step)
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += (gridDim.x * blockDim.x) >> 5) {
    const float e = y[i] - t[i];
    const float dy = 2.f * e / (float)N;
    pb += dy;
    pl += e * e / (float)N;
#pragma unroll
    for (int k = 0; k < kH / 32; ++k) {
      const int c = lane + 32 * k;
      part[k] = fmaf(dy, __bfloat162float(H3[(long long)i * kH + c]), part[k]);
      const float d = dy * w4[c] * dsilu(Z3[(long long)i * kH + c]);
      const __nv_bfloat16 h = __float2bfloat16(d);
      dZ3[(long long)i * kH + c] = h;
      dZ3t[(long long)c * N + i] = h;
    }
  }
#pragma unroll
  for (int k = 0; k < kH / 32; ++k) sw[warp][lane + 32 * k] = part[k];
  if (lane == 0) {
    sbl[warp][0] = pb;
    sbl[warp][1] = pl;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  float* out = part_out + (long long)blockIdx.x * kOutPart;
  for (int c = threadIdx.x; c < kOutPart; c += blockDim.x) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) v += c < kH ? sw[w][c] : sbl[w][c - kH];
    out[c] = v;
  }
}

// dw4, db4 and the loss: the blocks' partials added in block order
__global__ void k_out_reduce(const float* __restrict__ part, int blocks, float* __restrict__ gw4,
                             float* __restrict__ gb4, float* __restrict__ loss) {
  for (int c = threadIdx.x; c < kOutPart; c += blockDim.x) {
    float v = 0.f;
    for (int b = 0; b < blocks; ++b) v += part[(long long)b * kOutPart + c];
    if (c < kH) gw4[c] = v;
    else if (c == kH) gb4[0] = v;
    else loss[0] = v;
  }
}

__global__ void k_rowsum(const __nv_bfloat16* __restrict__ Mt, int rows, int N, float* __restrict__ out) {
  const int r = blockIdx.x;
  if (r >= rows) return;
  float s = 0.f;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += __bfloat162float(Mt[(long long)r * N + i]);
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[r] = s;
  }
}

// Adam on FP32 masters (Kingma and Ba, 2015, Algorithm 1) and the BF16
// copies the GEMMs read, over the whole flat parameter vector in one launch:
// segment k covers
// [begin[k], end[k]); a segment with a matrix W (rows x cols, row major) also
// receives the BF16 copy of the new value, and its transpose when Wt is set.
struct AdamSegs {
  long long begin[6], end[6];
  __nv_bfloat16* W[6];
  __nv_bfloat16* Wt[6];
  int rows[6], cols[6];
};

__global__ void k_adam_all(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, long long count, float lr, float b1, float b2, float eps, float c1,
                           float c2, AdamSegs segs) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    int k = 0;
    while (k < 5 && i >= segs.end[k]) ++k;
    if (segs.W[k]) {
      const long long j = i - segs.begin[k];
      const int r = (int)(j / segs.cols[k]), c = (int)(j % segs.cols[k]);
      const __nv_bfloat16 h = __float2bfloat16(pi);
      segs.W[k][j] = h;
      if (segs.Wt[k]) segs.Wt[k][(long long)c * segs.rows[k] + r] = h;
    }
  }
}

__global__ void k_to_bf16(const float* __restrict__ p, long long count, __nv_bfloat16* __restrict__ W,
                          __nv_bfloat16* __restrict__ Wt, int rows, int cols) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const __nv_bfloat16 h = __float2bfloat16(p[i]);
    W[i] = h;
    if (Wt) Wt[(long long)(i % cols) * rows + i / cols] = h;
  }
}

__global__ void k_clamp_labels(float* __restrict__ t, long long N, float lo, float hi) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    t[i] = fminf(fmaxf(t[i], lo), hi);
}

// configuration i of a training set: uniform in the joint box from Philox
// (counter (i, j, 0x5355, seed word), key (seed low, seed high))
__global__ void k_uniform_q(float* __restrict__ q, long long N, int n, const float* __restrict__ lo,
                            const float* __restrict__ hi, uint32_t k0, uint32_t k1) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    for (int j = 0; j < n; j += 4) {
      const u32x4 r = philox4x32_10(u32x4{(uint32_t)i, (uint32_t)(i >> 32), (uint32_t)j, 0x5355u}, k0, k1);
      const uint32_t w[4] = {r.x, r.y, r.z, r.w};
      for (int c = 0; c < 4 && j + c < n; ++c) q[(long long)(j + c) * N + i] = lo[j + c] + (hi[j + c] - lo[j + c]) * u01_co(w[c]);
    }
  }
}


}  // namespace ezo

// ------------------------------------------------------------------ host side --
namespace {

using namespace ezo;

// flat parameter layout: W1 [H x F] | b1 [H] | W2 [H x H] | b2 | W3 [H x H] | b3 | w4 [H] | b4 [1]
constexpr long long kOffW1 = 0, kOffB1 = kOffW1 + (long long)kH * kF, kOffW2 = kOffB1 + kH,
                    kOffB2 = kOffW2 + (long long)kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + (long long)kH * kH,
                    kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH, kNumParams = kOffB4 + 1;

template <typename T>
cudaError_t dal(T** p, size_t n) {
  return cudaMalloc((void**)p, std::max<size_t>(1, n) * sizeof(T));
}

}  // namespace

extern "C" int ezo_internal_robot_boxes(const ezo_robot* r);
extern "C" int ezo_internal_env_boxes(const ezo_env* e);
extern "C" int ezo_internal_robot_prismatic(const ezo_robot* r);
extern "C" void ezo_internal_set_error(const char* msg);
extern "C" const ezo::RobotDev* ezo_internal_robot_dev(const ezo_robot* r, int* n, int* nsp_pad, double* q_lo,
                                                       double* q_hi);
extern "C" int ezo_internal_env_dev(const ezo_robot* r, const ezo_env* e, ezo::EnvDevFull* out);

struct ezo_surrogate {
  int n = 0;
  const ezo_robot* robot = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // flat FP32
  __nv_bfloat16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W2t = nullptr, *W3t = nullptr;
  long long step = 0;
  // activations for a training batch of up to cap rows
  int cap = 0;
  __nv_bfloat16 *X = nullptr, *Xt = nullptr, *H1 = nullptr, *H1t = nullptr, *H2 = nullptr, *H2t = nullptr,
                *H3 = nullptr, *H3t = nullptr, *dZ3 = nullptr, *dZ3t = nullptr, *dZ2 = nullptr, *dZ2t = nullptr,
                *dZ1 = nullptr, *dZ1t = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *y = nullptr, *loss = nullptr;
  float* ws = nullptr;  // partial products of the weight gradients (K split over blocks)
  float* ows = nullptr;  // the output layer's per-block gradient and loss partials
  // inference: the swizzled weight image of the tensor-core forward kernel
  // and its error flag
  void* wimg = nullptr;
  int* tc_err = nullptr;
};

namespace {

using namespace ezo;

// every hidden-layer product of training on the tensor cores (tcgen05, FP32
// accumulators in tensor memory); the weight gradients split the batch
// dimension over blocks and add the partial products in a fixed order
cudaError_t gemm(ezo_surrogate* S, int epi, const GemmArgs& a, cudaStream_t s) {
  return gemm_tc(epi, a, epi == EPI_F32 ? S->ws : nullptr, S->tc_err, s);
}

int blocks_for(long long n, int t) { return (int)std::max<long long>(1, std::min<long long>((n + t - 1) / t, 4096)); }

cudaError_t sync_bf16(ezo_surrogate* S, cudaStream_t s) {
  k_to_bf16<<<blocks_for((long long)kH * kF, 256), 256, 0, s>>>(S->p + kOffW1, (long long)kH * kF, S->W1, nullptr, kH, kF);
  k_to_bf16<<<blocks_for((long long)kH * kH, 256), 256, 0, s>>>(S->p + kOffW2, (long long)kH * kH, S->W2, S->W2t, kH, kH);
  k_to_bf16<<<blocks_for((long long)kH * kH, 256), 256, 0, s>>>(S->p + kOffW3, (long long)kH * kH, S->W3, S->W3t, kH, kH);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = mlp_tc_build_image(S->W1, S->W2, S->W3, S->wimg, s);
  return e;
}

cudaError_t ensure_train_cap(ezo_surrogate* S, int B) {
  if (B <= S->cap) return cudaSuccess;
  __nv_bfloat16** bufs[] = {&S->X, &S->Xt, &S->H1, &S->H1t, &S->H2, &S->H2t, &S->H3, &S->H3t,
                            &S->dZ3, &S->dZ3t, &S->dZ2, &S->dZ2t, &S->dZ1, &S->dZ1t};
  for (auto b : bufs) {
    cudaFree(*b);
    *b = nullptr;
  }
  cudaFree(S->Z1);
  cudaFree(S->Z2);
  cudaFree(S->Z3);
  cudaFree(S->y);
  cudaFree(S->ws);
  S->ws = nullptr;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 14 && e == cudaSuccess; ++i) e = dal(bufs[i], (size_t)B * (i < 2 ? kF : kH));
  if (e == cudaSuccess) e = dal(&S->ws, gemm_tc_ws_floats(kH, kH, B));
  if (e == cudaSuccess) e = dal(&S->Z1, (size_t)B * kH);
  if (e == cudaSuccess) e = dal(&S->Z2, (size_t)B * kH);
  if (e == cudaSuccess) e = dal(&S->Z3, (size_t)B * kH);
  if (e == cudaSuccess) e = dal(&S->y, (size_t)B);
  if (e == cudaSuccess) S->cap = B;
  return e;
}

// forward + backward of one batch (q: n x B, stride ldq; t: B targets);
// gradients into S->g, loss into S->loss (both zeroed here)
cudaError_t train_grad(ezo_surrogate* S, const float* q, long long ldq, const float* t, int B, cudaStream_t s) {
  cudaError_t e = ensure_train_cap(S, B);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(S->g, 0, sizeof(float) * kNumParams, s);
  cudaMemsetAsync(S->loss, 0, sizeof(float), s);
  k_features<<<blocks_for(B, 64), 256, 0, s>>>(q, ldq, S->n, B, S->X, S->Xt, B);
  GemmArgs a{};
  a.M = B;
  a.N = kH;
  a.ldt = B;
  // forward
  a.A = S->X; a.lda = kF; a.B = S->W1; a.ldb = kF; a.K = kF; a.bias = S->p + kOffB1; a.Z = S->Z1; a.H = S->H1; a.Ht = S->H1t;
  if ((e = gemm(S, EPI_BIAS_SILU, a, s)) != cudaSuccess) return e;
  a.A = S->H1; a.lda = kH; a.B = S->W2; a.ldb = kH; a.K = kH; a.bias = S->p + kOffB2; a.Z = S->Z2; a.H = S->H2; a.Ht = S->H2t;
  if ((e = gemm(S, EPI_BIAS_SILU, a, s)) != cudaSuccess) return e;
  a.A = S->H2; a.B = S->W3; a.bias = S->p + kOffB3; a.Z = S->Z3; a.H = S->H3; a.Ht = S->H3t;
  if ((e = gemm(S, EPI_BIAS_SILU, a, s)) != cudaSuccess) return e;
  k_out<<<blocks_for((long long)B * 32, 256), 256, 0, s>>>(S->H3, S->p + kOffW4, S->p + kOffB4, B, nullptr, S->y);
  // backward
  const int ob = std::min(kOutBlocks, blocks_for((long long)B * 32, 256));
  k_out_backward<<<ob, 256, 0, s>>>(S->y, t, S->Z3, S->H3, S->p + kOffW4, B, S->dZ3, S->dZ3t, S->ows);
  k_out_reduce<<<1, 288, 0, s>>>(S->ows, ob, S->g + kOffW4, S->g + kOffB4, S->loss);
  GemmArgs w{};
  // dW3 = dZ3^T H2, db3 = column sums of dZ3
  w.A = S->dZ3t; w.lda = B; w.B = S->H2t; w.ldb = B; w.M = kH; w.N = kH; w.K = B; w.C = S->g + kOffW3; w.ldc = kH;
  if ((e = gemm(S, EPI_F32, w, s)) != cudaSuccess) return e;
  k_rowsum<<<kH, 256, 0, s>>>(S->dZ3t, kH, B, S->g + kOffB3);
  // dZ2 = (dZ3 W3) * SiLU'(Z2)
  GemmArgs d{};
  d.M = B; d.N = kH; d.K = kH; d.ldt = B;
  d.A = S->dZ3; d.lda = kH; d.B = S->W3t; d.ldb = kH; d.Z = S->Z2; d.H = S->dZ2; d.Ht = S->dZ2t;
  if ((e = gemm(S, EPI_DSILU, d, s)) != cudaSuccess) return e;
  w.A = S->dZ2t; w.B = S->H1t; w.C = S->g + kOffW2;
  if ((e = gemm(S, EPI_F32, w, s)) != cudaSuccess) return e;
  k_rowsum<<<kH, 256, 0, s>>>(S->dZ2t, kH, B, S->g + kOffB2);
  d.A = S->dZ2; d.B = S->W2t; d.Z = S->Z1; d.H = S->dZ1; d.Ht = S->dZ1t;
  if ((e = gemm(S, EPI_DSILU, d, s)) != cudaSuccess) return e;
  // dW1 = dZ1^T X
  w.A = S->dZ1t; w.B = S->Xt; w.N = kF; w.C = S->g + kOffW1; w.ldc = kF;
  if ((e = gemm(S, EPI_F32, w, s)) != cudaSuccess) return e;
  k_rowsum<<<kH, 256, 0, s>>>(S->dZ1t, kH, B, S->g + kOffB1);
  return cudaGetLastError();
}

cudaError_t adam_step(ezo_surrogate* S, float lr, cudaStream_t s) {
  S->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - std::pow(b1, (float)S->step), c2 = 1.f - std::pow(b2, (float)S->step);
  // one launch over the flat parameter vector; the BF16 copies (and
  // transposes) of W1..W3 are refreshed on the way
  AdamSegs segs{};
  segs.end[0] = kOffB1;  segs.W[0] = S->W1; segs.Wt[0] = nullptr; segs.rows[0] = kH; segs.cols[0] = kF;
  segs.end[1] = kOffW2;  segs.W[1] = nullptr;
  segs.end[2] = kOffB2;  segs.W[2] = S->W2; segs.Wt[2] = S->W2t; segs.rows[2] = kH; segs.cols[2] = kH;
  segs.end[3] = kOffW3;  segs.W[3] = nullptr;
  segs.end[4] = kOffB3;  segs.W[4] = S->W3; segs.Wt[4] = S->W3t; segs.rows[4] = kH; segs.cols[4] = kH;
  segs.end[5] = kNumParams; segs.W[5] = nullptr;
  const long long starts[6] = {kOffW1, kOffB1, kOffW2, kOffB2, kOffW3, kOffB3};
  for (int k = 0; k < 6; ++k) segs.begin[k] = starts[k];
  k_adam_all<<<blocks_for(kNumParams, 256), 256, 0, s>>>(S->p, S->g, S->m, S->v, kNumParams, lr, b1, b2, eps, c1, c2,
                                                          segs);
  return cudaGetLastError();
}

}  // namespace

// n_b surrogate bisection steps on the brackets of the rows below the device
// count *m_dev, in one tensor-core launch. Internal.
extern "C" __attribute__((visibility("hidden"))) cudaError_t ezo_internal_mlp_bisect(
    ezo_surrogate* S, long long rows_cap, const int* m_dev, const float* s_p32, const float* s_d32, float* s_lo,
    float* s_hi, uint32_t* s_bits, int n_b, float margin, cudaStream_t s) {
  return mlp_tc_bisect(S->n, rows_cap, m_dev, S->wimg, S->p + kOffB1, S->p + kOffB2, S->p + kOffB3, S->p + kOffW4,
                       S->p + kOffB4, s_p32, s_d32, s_lo, s_hi, s_bits, n_b, margin, S->tc_err, s);
}

extern "C" __attribute__((visibility("hidden"))) int ezo_internal_surrogate_dof(const ezo_surrogate* S) {
  return S ? S->n : 0;
}

extern "C" {

int64_t ezo_surrogate_num_params(void) { return kNumParams; }

ezo_status ezo_surrogate_create(const ezo_robot* robot, uint64_t seed, ezo_surrogate** out) {
  if (!robot || !out) {
    ezo_internal_set_error("ezo_surrogate_create: null argument");
    return EZO_ERR_INVALID_ARG;
  }
  int n = 0, nsp = 0;
  double lo[EZO_MAX_DOF], hi[EZO_MAX_DOF];
  ezo_internal_robot_dev(robot, &n, &nsp, lo, hi);
  if (2 * n > kF) {
    ezo_internal_set_error("ezo_surrogate_create: 2 n features must fit in 64");
    return EZO_ERR_INVALID_ARG;
  }
  if (ezo_internal_robot_prismatic(robot)) {
    // the features sin q, cos q identify revolute joint angles only
    ezo_internal_set_error("ezo_surrogate_create: prismatic joints are not supported by the [sin q, cos q] features");
    return EZO_ERR_INVALID_ARG;
  }
  ezo_surrogate* S = new ezo_surrogate();
  S->n = n;
  S->robot = robot;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dal(&S->p, kNumParams);
  if (e == cudaSuccess) e = dal(&S->g, kNumParams);
  if (e == cudaSuccess) e = dal(&S->m, kNumParams);
  if (e == cudaSuccess) e = dal(&S->v, kNumParams);
  if (e == cudaSuccess) e = dal(&S->W1, (size_t)kH * kF);
  if (e == cudaSuccess) e = dal(&S->W2, (size_t)kH * kH);
  if (e == cudaSuccess) e = dal(&S->W3, (size_t)kH * kH);
  if (e == cudaSuccess) e = dal(&S->W2t, (size_t)kH * kH);
  if (e == cudaSuccess) e = dal(&S->W3t, (size_t)kH * kH);
  if (e == cudaSuccess) e = dal(&S->loss, 1);
  if (e == cudaSuccess) e = dal(&S->ows, (size_t)kOutBlocks * kOutPart);
  if (e == cudaSuccess) e = cudaMalloc(&S->wimg, mlp_tc_image_bytes());
  if (e == cudaSuccess) e = dal(&S->tc_err, 1);
  if (e == cudaSuccess) e = cudaMemset(S->tc_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    ezo_surrogate_free(S);
    ezo_internal_set_error((std::string("ezo_surrogate_create: ") + cudaGetErrorString(e)).c_str());
    return EZO_ERR_CUDA;
  }
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases from a
  // 64-bit LCG (Knuth's MMIX constants), so the start is reproducible
  std::vector<float> h(kNumParams);
  uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((st >> 40) * (1.0 / 16777216.0));
  };
  auto fill = [&](long long off, long long cnt, int fan_in) {
    const float a = 1.f / std::sqrt((float)fan_in);
    for (long long i = 0; i < cnt; ++i) h[off + i] = (2.f * uni() - 1.f) * a;
  };
  fill(kOffW1, (long long)kH * kF, 2 * n);
  fill(kOffB1, kH, 2 * n);
  for (long long i = 0; i < kH; ++i)
    for (int c = 2 * n; c < kF; ++c) h[kOffW1 + i * kF + c] = 0.f;  // padding features carry no weight
  fill(kOffW2, (long long)kH * kH, kH);
  fill(kOffB2, kH, kH);
  fill(kOffW3, (long long)kH * kH, kH);
  fill(kOffB3, kH, kH);
  fill(kOffW4, kH, kH);
  h[kOffB4] = 0.f;
  cudaMemcpy(S->p, h.data(), sizeof(float) * kNumParams, cudaMemcpyHostToDevice);
  cudaMemset(S->m, 0, sizeof(float) * kNumParams);
  cudaMemset(S->v, 0, sizeof(float) * kNumParams);
  sync_bf16(S, nullptr);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    ezo_surrogate_free(S);
    ezo_internal_set_error((std::string("ezo_surrogate_create: ") + cudaGetErrorString(e)).c_str());
    return EZO_ERR_CUDA;
  }
  *out = S;
  return EZO_OK;
}

void ezo_surrogate_free(ezo_surrogate* S) {
  if (!S) return;
  void* ps[] = {S->p,  S->g,   S->m,   S->v,   S->W1,  S->W2,  S->W3,   S->W2t,  S->W3t, S->X,   S->Xt,  S->H1,
                S->H1t, S->H2, S->H2t, S->H3, S->H3t, S->dZ3, S->dZ3t, S->dZ2, S->dZ2t, S->dZ1, S->dZ1t, S->Z1, S->Z2,
                S->Z3, S->y,   S->loss, S->wimg, S->tc_err, S->ws, S->ows};
  for (void* q : ps)
    if (q) cudaFree(q);
  delete S;
}

ezo_status ezo_surrogate_get_params(const ezo_surrogate* S, float* out) {
  if (!S || !out) return EZO_ERR_INVALID_ARG;
  if (cudaMemcpy(out, S->p, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost) != cudaSuccess) return EZO_ERR_CUDA;
  return EZO_OK;
}

ezo_status ezo_surrogate_set_params(ezo_surrogate* S, const float* in) {
  if (!S || !in) return EZO_ERR_INVALID_ARG;
  if (cudaMemcpy(S->p, in, sizeof(float) * kNumParams, cudaMemcpyHostToDevice) != cudaSuccess) return EZO_ERR_CUDA;
  sync_bf16(S, nullptr);
  return cudaDeviceSynchronize() == cudaSuccess ? EZO_OK : EZO_ERR_CUDA;
}

ezo_status ezo_surrogate_grad(ezo_surrogate* S, const float* q_dev, int64_t ldq, const float* t_dev, int32_t N,
                              float* grad, float* loss, void* stream) {
  if (!S || !q_dev || !t_dev || N < 64 || N % 64 || ldq < N) {
    ezo_internal_set_error("ezo_surrogate_grad: need N a positive multiple of 64 and ldq >= N");
    return EZO_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = train_grad(S, q_dev, ldq, t_dev, N, s);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, S->g, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, S->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ezo_internal_set_error((std::string("ezo_surrogate_grad: ") + cudaGetErrorString(e)).c_str());
    return EZO_ERR_CUDA;
  }
  return EZO_OK;
}

ezo_status ezo_surrogate_predict(ezo_surrogate* S, const float* q_dev, int64_t ldq, int64_t N, float* out_dev,
                                 void* stream) {
  if (!S || (N > 0 && (!q_dev || !out_dev)) || N < 0 || ldq < N) {
    ezo_internal_set_error("ezo_surrogate_predict: bad argument");
    return EZO_ERR_INVALID_ARG;
  }
  if (N == 0) return EZO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // features computed inside the forward kernel from the configurations
  mlp_tc_forward(q_dev, ldq, S->n, N, nullptr, S->wimg, S->p + kOffB1, S->p + kOffB2, S->p + kOffB3, S->p + kOffW4, S->p + kOffB4,
                 out_dev, S->tc_err, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ezo_internal_set_error((std::string("ezo_surrogate_predict: ") + cudaGetErrorString(e)).c_str());
    return EZO_ERR_CUDA;
  }
  return EZO_OK;
}

ezo_status ezo_surrogate_status(ezo_surrogate* S, int32_t* timed_out, int32_t reset, void* stream) {
  if (!S || !timed_out) {
    ezo_internal_set_error("ezo_surrogate_status: null argument");
    return EZO_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, S->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(S->tc_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ezo_internal_set_error((std::string("ezo_surrogate_status: ") + cudaGetErrorString(e)).c_str());
    return EZO_ERR_CUDA;
  }
  *timed_out = v != 0 ? 1 : 0;
  ezo_internal_set_error("");
  return EZO_OK;
}

ezo_status ezo_surrogate_train(ezo_surrogate* S, const ezo_env* env, int64_t n_samples, int32_t epochs, int32_t batch,
                               float lr, uint64_t data_seed, float label_lo, float label_hi, float* epoch_loss,
                               void* stream) {
  if (!S || !env || n_samples < batch || batch < 64 || batch % 64 || epochs < 1 || !(lr > 0.f)) {
    ezo_internal_set_error("ezo_surrogate_train: need batch a multiple of 64, n_samples >= batch, epochs >= 1");
    return EZO_ERR_INVALID_ARG;
  }
  if (ezo_internal_robot_boxes(S->robot) || ezo_internal_env_boxes(env)) {
    // the labels come from the sphere signed-distance kernel
    ezo_internal_set_error("ezo_surrogate_train: sphere geometries only (the robot or env has boxes)");
    return EZO_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int n = 0, nsp = 0;
  double lo[EZO_MAX_DOF], hi[EZO_MAX_DOF];
  const RobotDev* rd = ezo_internal_robot_dev(S->robot, &n, &nsp, lo, hi);
  EnvDevFull ef{};
  ezo_internal_env_dev(S->robot, env, &ef);
  const long long N = n_samples / batch * batch;
  float *q = nullptr, *t = nullptr, *bnd = nullptr;
  cudaError_t e = dal(&q, (size_t)n * N);
  if (e == cudaSuccess) e = dal(&t, (size_t)N);
  if (e == cudaSuccess) e = dal(&bnd, 2 * EZO_MAX_DOF);
  if (e == cudaSuccess) {
    float hb[2 * EZO_MAX_DOF];
    for (int j = 0; j < n; ++j) {
      hb[j] = (float)lo[j];
      hb[EZO_MAX_DOF + j] = (float)hi[j];
    }
    cudaMemcpyAsync(bnd, hb, sizeof(hb), cudaMemcpyHostToDevice, s);
    // training set: uniform configurations labelled by the exact FP32
    // signed distance, clamped to [label_lo, label_hi]
    k_uniform_q<<<blocks_for(N, 256), 256, 0, s>>>(q, N, n, bnd, bnd + EZO_MAX_DOF, (uint32_t)data_seed,
                                                     (uint32_t)(data_seed >> 32));
    e = launch_sd_flat(rd, n, nsp, ef.e, q, N, N, t, s, label_hi);
    k_clamp_labels<<<blocks_for(N, 256), 256, 0, s>>>(t, N, label_lo, label_hi);
  }
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    float sum = 0.f;
    const long long steps = N / batch;
    for (long long st = 0; st < steps && e == cudaSuccess; ++st) {
      e = train_grad(S, q + st * batch, N, t + st * batch, batch, s);
      if (e == cudaSuccess) e = adam_step(S, lr, s);
      if (epoch_loss && e == cudaSuccess && (st % 64 == 63 || st == steps - 1)) {
        float l = 0.f;
        cudaMemcpyAsync(&l, S->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        sum = l;  // loss of the latest batch
      }
    }
    if (epoch_loss) epoch_loss[ep] = sum;
  }
  // the tensor-core forward pass reads the updated BF16 weights from its image
  if (e == cudaSuccess) e = mlp_tc_build_image(S->W1, S->W2, S->W3, S->wimg, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(q);
  cudaFree(t);
  cudaFree(bnd);
  if (e != cudaSuccess) {
    ezo_internal_set_error((std::string("ezo_surrogate_train: ") + cudaGetErrorString(e)).c_str());
    return EZO_ERR_CUDA;
  }
  return EZO_OK;
}

}  // extern "C"
