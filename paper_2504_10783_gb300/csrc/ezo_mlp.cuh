// Training GEMMs of the learned surrogate: arguments shared by the kernels
// that compute C[M x N] = A[M x K] B[N x K]^T (both operands BF16, K
// contiguous, row-major with leading dimensions lda, ldb; FP32 accumulation)
// with the epilogues of the forward and backward passes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ezo {

enum Epi : int {
  EPI_F32 = 0,        // C (FP32) = acc
  EPI_BIAS_SILU = 1,  // Z = acc + bias (FP32), H = SiLU(Z) (BF16, and transposed)
  EPI_DSILU = 2       // D = acc * SiLU'(Z) (BF16, and transposed)
};

struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  int M, N, K, lda, ldb;
  const int* m_dev;  // optional device row count (rows >= *m_dev are skipped)
  float* C;          // EPI_F32 output, ldc
  int ldc;
  const float* bias;
  float* Z;          // EPI_BIAS_SILU: pre-activation out; EPI_DSILU: pre-activation in (ldz = N)
  __nv_bfloat16* H;  // BF16 output, row-major (ldh = N)
  __nv_bfloat16* Ht; // BF16 output, transposed [N x ldt]
  int ldt;
};

// The same products on tcgen05 (ezo_mlp_gemm_tc.cu): K and lda, ldb multiples
// of 64; M any; N a multiple of 64 up to 256. EPI_F32 splits K over blocks
// when `ws` (FP32 workspace of gemm_tc_ws_floats(M, N, K) values) is given and
// adds the partial products in a fixed order, so results are reproducible.
// `err` (device int) is set when a bounded wait gave up.
size_t gemm_tc_ws_floats(int M, int N, int K);
cudaError_t gemm_tc(int epi, const GemmArgs& a, float* ws, int* err, cudaStream_t s);

}  // namespace ezo
