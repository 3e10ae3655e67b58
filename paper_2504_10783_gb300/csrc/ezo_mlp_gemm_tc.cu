// Training GEMMs of the learned surrogate on the 5th-generation tensor
// cores: C[M x N] = A[M x K] B[N x K]^T in BF16 with the FP32 accumulator in
// tensor memory, and the forward (bias + SiLU) and backward (SiLU')
// epilogues read from it with tcgen05.ld.
//
// One block of 128 threads computes a 128 x 64 tile of C over a range of K: for each 64-wide chunk of K every thread copies its
// share of the A rows (128 x 128 bytes) and B rows (Nt x 128 bytes) into
// shared memory in the K-major 128-byte swizzled layout with 16-byte
// asynchronous copies (rows beyond M or N are zero-filled), then thread 0
// issues four tcgen05.mma (M = 128, N = 64, K = 16) and commits them to the
// stage's mbarrier. Two stages let the copies of chunk c + 1 overlap the MMAs
// of chunk c. The epilogue thread t reads row t of the tile, which is lane t
// of the accumulator in tensor memory, and the outputs leave through shared
// memory as whole row segments.
//
// The weight gradients (M = 256 rows of a layer, K = the batch) split K over
// blocks, each writing its partial product to a workspace, and a second
// kernel adds the partials in a fixed order. Every mbarrier wait is bounded
// (about two seconds); a wait that gives up sets the error flag, the block
// skips its outputs and still frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ezo_mlp.cuh"
#include "ezo_tc.cuh"

namespace ezo {

namespace {

using namespace tc;

constexpr int kGM = 128;         // rows of a tile (UMMA M)
constexpr int kGK = 64;          // K of a chunk: 64 BF16 = one 128-byte swizzled row
constexpr int kGThreads = 128;   // four warps: warp w reads tensor-memory lanes 32 w .. 32 w + 31
constexpr int kGStages = 2;
constexpr int kSplitChunks = 2;  // K chunks per block of a split product

__device__ __forceinline__ float silu_g(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu_g(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

struct TcGemm {
  GemmArgs g;
  int nt;        // columns per tile: 64 or 128
  int chunks;    // K chunks per block
  float* ws;     // split-K partials [splits x M x N], or null
  int* err;
};

template <int EPI>
__global__ void __launch_bounds__(kGThreads, 1) k_gemm_tc(TcGemm p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t mma_bar[kGStages], done_bar;
  __shared__ uint32_t tmem_slot;
  const GemmArgs& g = p.g;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m_lim = g.m_dev ? min(g.M, *g.m_dev) : g.M;
  const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * p.nt;
  if (m0 >= m_lim) return;  // the whole block, before any barrier or allocation
  const int nt = p.nt;
  const int k_chunks = g.K / kGK;
  const int c0 = blockIdx.z * p.chunks, c1 = min(k_chunks, c0 + p.chunks);

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t stage_bytes = (uint32_t)(kGM + nt) * 128u;

  if (tid == 0) {
    for (int s = 0; s < kGStages; ++s) mbar_init(&mma_bar[s], 1);
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(nt)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_slot;
  const uint32_t idesc = idesc_bf16(kGM, nt);
  bool ok = true;

  for (int c = c0, i = 0; c < c1; ++c, ++i) {
    const int s = i & 1;
    // the MMAs that read this stage two chunks ago have completed
    if (i >= kGStages && !mbar_wait(&mma_bar[s], (uint32_t)((i / kGStages - 1) & 1))) ok = false;
    ok = __syncthreads_and(ok);
    if (!ok) break;
    const uint32_t sA = base + (uint32_t)s * stage_bytes, sB = sA + kGM * 128u;
    const int k0 = c * kGK;
    for (int idx = tid; idx < kGM * 8; idx += kGThreads) {
      const int r = idx >> 3, cc = idx & 7;
      const int gm = m0 + r;
      const bool v = gm < m_lim;
      cp_async16(sA + sw128(r, cc), g.A + (long long)(v ? gm : 0) * g.lda + k0 + cc * 8, v);
    }
    for (int idx = tid; idx < nt * 8; idx += kGThreads) {
      const int r = idx >> 3, cc = idx & 7;
      const int gn = n0 + r;
      const bool v = gn < g.N;
      cp_async16(sB + sw128(r, cc), g.B + (long long)(v ? gn : 0) * g.ldb + k0 + cc * 8, v);
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    proxy_fence();  // the copies are visible to the tensor cores' (async) proxy
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < kGK / 16; ++kk)
        umma_f16(tbase, sdesc(sA + kk * 32), sdesc(sB + kk * 32), idesc, (i | kk) != 0);
      umma_commit(&mma_bar[s]);
    }
  }
  if (tid == 0) umma_commit(&done_bar);  // arrives when every MMA issued above has completed
  if (!mbar_wait(&done_bar, 0)) ok = false;
  ok = __syncthreads_and(ok);
  tc_fence_after();

  // epilogue: row m0 + tid is tensor-memory lane tid. The values of a
  // 16-column slice pass through shared memory (the operand stages are free
  // now) so that the row-major outputs, and the pre-activations the backward
  // epilogue reads, move as whole 64-byte row segments; the transposed BF16
  // output is written directly (consecutive rows are consecutive addresses).
  constexpr int LD = 17;  // floats per staged row (odd: conflict-free row writes)
  float* sv = reinterpret_cast<float*>(smem_raw + (base - raw));  // 128 x LD: values / pre-activations
  float* sh = sv + kGM * LD;                                      // 128 x LD: BF16 outputs as floats
  const int r = m0 + tid;
  const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
  for (int cb = 0; cb < nt; cb += 16) {
    const int col0 = n0 + cb;
    uint32_t v[16];
    tmem_ld16(lane_addr + (uint32_t)cb, v);
    tmem_wait_ld();
    if (EPI == EPI_DSILU) {
      // Z[m0 .. m0 + 127][col0 .. col0 + 15] into the staging tile, coalesced
      for (int i = tid; i < kGM * 4; i += kGThreads) {
        const int rr = i >> 2, q4 = (i & 3) * 4, gr = m0 + rr;
        float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gr < m_lim) z4 = *reinterpret_cast<const float4*>(g.Z + (long long)gr * g.N + col0 + q4);
        sv[rr * LD + q4] = z4.x;
        sv[rr * LD + q4 + 1] = z4.y;
        sv[rr * LD + q4 + 2] = z4.z;
        sv[rr * LD + q4 + 3] = z4.w;
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float acc = __uint_as_float(v[j]);
      if (EPI == EPI_F32) {
        sv[tid * LD + j] = acc;
      } else if (EPI == EPI_BIAS_SILU) {
        const float z = acc + g.bias[col0 + j];
        const __nv_bfloat16 h = __float2bfloat16(silu_g(z));
        sv[tid * LD + j] = z;
        sh[tid * LD + j] = __bfloat162float(h);
        if (ok && r < m_lim) g.Ht[(long long)(col0 + j) * g.ldt + r] = h;
      } else {
        const __nv_bfloat16 h = __float2bfloat16(acc * dsilu_g(sv[tid * LD + j]));
        sh[tid * LD + j] = __bfloat162float(h);
        if (ok && r < m_lim) g.Ht[(long long)(col0 + j) * g.ldt + r] = h;
      }
    }
    __syncthreads();
    if (ok) {
      // FP32 rows: 4 float4 per row segment
      if (EPI != EPI_DSILU) {
        float* dst = EPI == EPI_F32 ? (p.ws ? p.ws + (long long)blockIdx.z * g.M * g.N : g.C) : g.Z;
        const int ld = EPI == EPI_F32 ? (p.ws ? g.N : g.ldc) : g.N;
        for (int i = tid; i < kGM * 4; i += kGThreads) {
          const int rr = i >> 2, q4 = (i & 3) * 4, gr = m0 + rr;
          if (gr < m_lim)
            *reinterpret_cast<float4*>(dst + (long long)gr * ld + col0 + q4) =
                make_float4(sv[rr * LD + q4], sv[rr * LD + q4 + 1], sv[rr * LD + q4 + 2], sv[rr * LD + q4 + 3]);
        }
      }
      // BF16 rows: 2 x 16 bytes per row segment
      if (EPI != EPI_F32) {
        for (int i = tid; i < kGM * 2; i += kGThreads) {
          const int rr = i >> 1, h8 = (i & 1) * 8, gr = m0 + rr;
          if (gr < m_lim) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(sh[rr * LD + h8 + 2 * k], sh[rr * LD + h8 + 2 * k + 1]);
              w[k] = *reinterpret_cast<const uint32_t*>(&b2);
            }
            *reinterpret_cast<uint4*>(g.H + (long long)gr * g.N + col0 + h8) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      }
    }
    __syncthreads();
  }
  if (!ok && tid == 0) atomicExch(p.err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(nt) : "memory");
}

// C[r][c] = sum over splits z (in order) of ws[z][r][c]
__global__ void k_splitk_sum(const float* __restrict__ ws, int splits, int M, int N, float* __restrict__ C, int ldc) {
  const long long total = (long long)M * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += ws[(long long)z * total + i];
    C[(i / N) * ldc + i % N] = s;
  }
}

int split_count(int K) { return (K / kGK + kSplitChunks - 1) / kSplitChunks; }

}  // namespace

size_t gemm_tc_ws_floats(int M, int N, int K) { return (size_t)split_count(K) * M * N; }

cudaError_t gemm_tc(int epi, const GemmArgs& a, float* ws, int* err, cudaStream_t s) {
  if (a.K <= 0 || a.K % kGK || a.lda % kGK || a.ldb % kGK || a.N % 64 || a.N > 256 || a.M <= 0)
    return cudaErrorInvalidValue;
  const int nt = 64;  // more blocks than 128-column tiles for the batch sizes of training
  const int m_tiles = (a.M + kGM - 1) / kGM, n_tiles = a.N / nt;
  const bool split = epi == EPI_F32 && ws != nullptr;
  const int splits = split ? split_count(a.K) : 1;
  TcGemm p{a, nt, split ? kSplitChunks : a.K / kGK, split ? ws : nullptr, err};
  const size_t smem = (size_t)kGStages * (kGM + nt) * 128 + 1024;
  dim3 grid((unsigned)m_tiles, (unsigned)n_tiles, (unsigned)splits);
  // the dynamic shared-memory limit is raised once per device and kernel
  static int attr_dev[3] = {-1, -1, -1};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  const void* kern = epi == EPI_F32 ? (const void*)k_gemm_tc<EPI_F32>
                     : (epi == EPI_BIAS_SILU ? (const void*)k_gemm_tc<EPI_BIAS_SILU> : (const void*)k_gemm_tc<EPI_DSILU>);
  const int ki = epi == EPI_F32 ? 0 : (epi == EPI_BIAS_SILU ? 1 : 2);
  if (e == cudaSuccess && attr_dev[ki] != dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess) attr_dev[ki] = dev;
  }
  if (e == cudaSuccess) {
    switch (epi) {
      case EPI_F32: k_gemm_tc<EPI_F32><<<grid, kGThreads, smem, s>>>(p); break;
      case EPI_BIAS_SILU: k_gemm_tc<EPI_BIAS_SILU><<<grid, kGThreads, smem, s>>>(p); break;
      default: k_gemm_tc<EPI_DSILU><<<grid, kGThreads, smem, s>>>(p); break;
    }
  }
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e == cudaSuccess && split) {
    const long long total = (long long)a.M * a.N;
    k_splitk_sum<<<(unsigned)std::min<long long>((total + 255) / 256, 4096), 256, 0, s>>>(ws, splits, a.M, a.N, a.C,
                                                                                         a.ldc);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace ezo
