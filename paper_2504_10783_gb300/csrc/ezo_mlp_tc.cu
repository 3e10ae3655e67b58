// Forward pass of the learned signed-distance surrogate on the 5th-generation
// tensor cores: one persistent kernel runs all three hidden layers of a
// 128-row tile (features [128 x 64] -> 256 -> 256 -> 256 -> 1) with the
// accumulators in tensor memory and the activations in shared memory, so a
// row costs its configuration and 4 bytes of output in HBM. In its
// bisection mode the kernel runs all N_b surrogate bisection steps of a tile
// in one launch: each step's features are those of the midpoints of the
// rows' brackets, and the step's prediction halves the brackets in shared
// memory before the next step.
//
// Roles (576 threads):
//   warps 0-15 epilogue: warp w owns rows 32 (w % 4) .. +31 of the tile (the
//              tensor-memory lanes it may read) and, in each K-chunk c of 64
//              columns, the 16 columns 64 c + 16 (w / 4) .. +15. It stages
//              the feature tile, then for each layer reads its 64 accumulator
//              columns, adds the bias, applies SiLU, rounds to BF16 and writes
//              the next layer's input to shared memory chunk by chunk; the
//              last layer is reduced against w4 into y (or into the bisection
//              step).
//   warp 16    lane 0 issues the tcgen05.mma instructions (M = 128,
//              N = 256, K = 16, BF16 x BF16 -> FP32); the whole warp
//              allocates and frees the 512 tensor-memory columns.
//   warp 17    lane 0 streams the weights (nine 32 KB chunks per tile: W1,
//              then W2 and W3 in four K-chunks of 64) with bulk asynchronous
//              copies through a four-stage ring, ahead of the MMAs by the
//              depth of the ring.
// Two accumulators (columns 0-255 and 256-511) alternate from layer to
// layer, the MMAs of K-chunk c of a layer start as soon as chunk c of its
// input is written (the epilogue writes the chunks in order), and (in the
// plain forward pass) the next tile's features are staged while the current
// tile is in its second layer, so the tensor cores work on the next layer (or
// the next tile's first layer) while the epilogue is still busy with the
// current one.
//
// Shared-memory operands use the K-major 128-byte swizzled layout: a row of
// 64 BF16 values is 128 bytes, 8 rows form a 1024-byte atom, and 16-byte
// chunk c of row r sits at chunk position c ^ (r % 8). The weights are kept
// in global memory as images of that layout (built once per weight update),
// so each chunk is one contiguous bulk copy.
//
// Every wait on an mbarrier gives up after about two seconds: the kernel
// then records an error code, writes NaN for the rows it has not finished
// (in the bisection mode such rows take every later step as free) and still
// frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ezo_tc.cuh"

namespace ezo {

namespace {

using namespace tc;

constexpr int kTcRows = 128;            // rows per tile (UMMA M)
constexpr int kTcH = 256;               // hidden width (UMMA N)
constexpr int kTcF = 64;                // padded features
constexpr int kChunkBytes = kTcH * 128; // one weight chunk: 256 rows x 64 BF16
constexpr int kChunksPerTile = 9;       // W1, W2 x 4, W3 x 4
constexpr int kStages = 4;
constexpr int kXBytes = kTcRows * 128;  // feature tile
constexpr int kHBytes = kTcRows * 512;  // hidden tile: 4 K-chunks of 16 KB
constexpr int kSmemBytes = kXBytes + kHBytes + kStages * kChunkBytes + 1024;  // + alignment slack
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = kEpiThreads + 64;  // + the MMA warp and the weight producer warp
constexpr int kTmemCols = 2 * kTcH;  // two accumulators

constexpr uint32_t kIdesc = tc::idesc_bf16(kTcRows, kTcH);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  tc::umma_f16(d_tmem, a, b, kIdesc, accumulate);
}

// SiLU(z) = z sigmoid(z) = h + h tanh(h) with h = z / 2, on the hardware
// tanh approximation (relative error about 2^-11, below the BF16 rounding of
// the result)
__device__ __forceinline__ float silu_tc(float z) {
  const float h = 0.5f * z;
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
  return fmaf(h, t, h);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

struct TcArgs {
  const float* q;          // configurations, n x rows_cap with stride ldq (plain forward pass)
  long long ldq;
  int n;
  long long rows_cap;
  const int* m_dev;        // optional device row count
  const uint8_t* wimg;     // 9 swizzled weight chunks
  const float* b1;
  const float* b2;
  const float* b3;
  const float* w4;
  const float* b4;
  float* y;
  int* err;                // set to 1 when a wait gave up
  // surrogate bisection (when s_p32 is set): n_b steps per row on the
  // bracket [lo, hi] of c_proj + f (c - c_proj); y is not written
  const float* s_p32;      // rows x 8: c_proj
  const float* s_d32;      // rows x 8: c - c_proj
  float* s_lo;
  float* s_hi;
  uint32_t* s_bits;        // bit k: step k predicted a collision
  int n_b;
  float margin;            // predicted collision iff sd_hat < margin
};

// this thread's share of one feature row: the features of joints sc, sc + 4,
// .. (sin q_j at column j, cos q_j at column n + j, as in training; the zero
// padding columns were written once at the start)
__device__ __forceinline__ void stage_features(const TcArgs& g, uint8_t* sX, int row, int sc, long long grow,
                                               bool live) {
  for (int j = sc; j < g.n; j += 4) {
    float sn = 0.f, cs = 0.f;
    if (live) {
      const float qj = g.q[(long long)j * g.ldq + grow];
      sn = sinf(qj);
      cs = cosf(qj);
    }
    const int fc = g.n + j;
    *reinterpret_cast<__nv_bfloat16*>(sX + sw128(row, j >> 3) + (j & 7) * 2) = __float2bfloat16(sn);
    *reinterpret_cast<__nv_bfloat16*>(sX + sw128(row, fc >> 3) + (fc & 7) * 2) = __float2bfloat16(cs);
  }
}

// features of the midpoint f = (lo + hi) / 2 of a row's bracket: q_j =
// c_proj_j + f (c_j - c_proj_j), joints sc, sc + 4, ..
__device__ __forceinline__ void stage_bracket_features(const TcArgs& g, uint8_t* sX, int row, int sc,
                                                       long long grow, bool live, float lo, float hi) {
  const float f = 0.5f * (lo + hi);
  for (int j = sc; j < g.n; j += 4) {
    float sn = 0.f, cs = 0.f;
    if (live) {
      const float qj = fmaf(f, g.s_d32[grow * 8 + j], g.s_p32[grow * 8 + j]);
      sn = sinf(qj);
      cs = cosf(qj);
    }
    const int fc = g.n + j;
    *reinterpret_cast<__nv_bfloat16*>(sX + sw128(row, j >> 3) + (j & 7) * 2) = __float2bfloat16(sn);
    *reinterpret_cast<__nv_bfloat16*>(sX + sw128(row, fc >> 3) + (fc & 7) * 2) = __float2bfloat16(cs);
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_mlp_forward_tc(TcArgs g) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t w_full[kStages], w_empty[kStages], x_ready, h_ready[4], acc_full[2],
      acc_empty[2], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ float sbias[3][kTcH];
  __shared__ float sw4[kTcH];
  __shared__ float ypart[2][4][kTcRows];
  __shared__ float br_lo[kTcRows], br_hi[kTcRows];  // bisection: the brackets of the current tile
  __shared__ uint32_t br_bits[kTcRows];

  const uint32_t base_u32 = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_u32 - smem_u32(smem_raw));
  uint8_t* sX = base;
  uint8_t* sH = base + kXBytes;
  uint8_t* sW = base + kXBytes + kHBytes;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long m_lim = g.m_dev ? min((long long)*g.m_dev, g.rows_cap) : g.rows_cap;
  const long long n_tiles = (m_lim + kTcRows - 1) / kTcRows;
  // work items: (tile, bisection step), steps innermost; one step per tile
  // for a plain forward pass
  const bool bis = g.s_p32 != nullptr;
  const int n_steps = bis ? g.n_b : 1;
  long long my_items = 0;
  for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) my_items += n_steps;

  // feature tile starts zero: the padding columns stay zero when the features
  // are computed from q
  for (int i = tid; i < kXBytes / 16; i += kThreads) reinterpret_cast<uint4*>(sX)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < kTcH; i += kThreads) {
    sbias[0][i] = g.b1[i];
    sbias[1][i] = g.b2[i];
    sbias[2][i] = g.b3[i];
    sw4[i] = g.w4[i];
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&w_full[s], 1);
      mbar_init(&w_empty[s], 1);
    }
    mbar_init(&x_ready, kEpiThreads);
    for (int c = 0; c < 4; ++c) mbar_init(&h_ready[c], kEpiThreads);
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kEpiThreads);
    }
    mbar_init(&mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kEpiWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_slot;
  bool ok = true;

  if (warp == kEpiWarps + 1) {
    if (lane == 0) {
      const long long total = my_items * kChunksPerTile;
      long long wl = 0;
      for (; wl < total; ++wl) {
        const int st = (int)(wl % kStages);
        if (wl >= kStages && !mbar_wait(&w_empty[st], (uint32_t)((wl / kStages - 1) & 1))) {
          ok = false;
          break;
        }
        mbar_expect_tx(&w_full[st], kChunkBytes);
        bulk_g2s(sW + st * kChunkBytes, g.wimg + (wl % kChunksPerTile) * kChunkBytes, kChunkBytes, &w_full[st]);
      }
      if (!ok) atomicExch(g.err, 1);
      for (long long c = (wl > kStages ? wl - kStages : 0); c < wl; ++c)
        mbar_wait(&w_full[c % kStages], (uint32_t)((c / kStages) & 1));
    }
    __syncwarp();
  } else if (warp == kEpiWarps) {
    if (lane == 0) {
      // ---- MMA issuer ----
      long long wi = 0;
      for (long long tl = 0; tl < my_items && ok; ++tl) {
        for (int L = 0; L < 3 && ok; ++L) {
          const long long G = 3 * tl + L;  // layers so far: accumulator G % 2, its use G / 2
          const int a = (int)(G & 1);
          const long long use = G >> 1;
          // the accumulator's previous contents have been read by every epilogue thread
          if (use >= 1 && !mbar_wait(&acc_empty[a], (uint32_t)((use - 1) & 1))) {
            ok = false;
            break;
          }
          if (L == 0 && !mbar_wait(&x_ready, (uint32_t)(tl & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dacc = tbase + (uint32_t)(a * kTcH);
          const int nch = L == 0 ? 1 : 4;
          for (int kc = 0; kc < nch && ok; ++kc) {
            // K-chunk kc of this layer's input, written by the warps that own it
            if (L > 0 && !mbar_wait(&h_ready[kc], (uint32_t)((2 * tl + L - 1) & 1))) {
              ok = false;
              break;
            }
              const int st = (int)(wi % kStages);
            if (!mbar_wait(&w_full[st], (uint32_t)((wi / kStages) & 1))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(L == 0 ? sX : sH + kc * (kTcRows * 128));
            const uint32_t b0 = smem_u32(sW + st * kChunkBytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) umma(dacc, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), (kc | kk) != 0);
            umma_commit(&w_empty[st]);
            ++wi;
          }
          if (ok) umma_commit(&acc_full[a]);
        }
      }
      if (!ok) atomicExch(g.err, 1);
      // every MMA issued here has completed before the columns are freed
      umma_commit(&mma_done);
      if (!mbar_wait(&mma_done, 0)) atomicExch(g.err, 1);
    }
    __syncwarp();
  } else {
    // ---- epilogue warps ----
    const int lq = warp & 3, sc = warp >> 2;
    const int row = lq * 32 + lane;
    const uint32_t lane_addr = tbase + ((uint32_t)(lq * 32) << 16) + (uint32_t)(sc * 16);
    auto tile_of = [&](long long it) { return blockIdx.x + (it / n_steps) * (long long)gridDim.x; };
    // bisection: the brackets of a tile's rows, held by the sc = 0 threads
    auto load_brackets = [&](long long it) {
      const long long grow = tile_of(it) * kTcRows + row;
      if (sc == 0) {
        const bool live = grow < m_lim;
        br_lo[row] = live ? g.s_lo[grow] : 0.f;
        br_hi[row] = live ? g.s_hi[grow] : 1.f;
        br_bits[row] = live ? g.s_bits[grow] : 0u;
      }
    };
    auto stage_item = [&](long long it) {
      const long long grow = tile_of(it) * kTcRows + row;
      if (bis) stage_bracket_features(g, sX, row, sc, grow, grow < m_lim, br_lo[row], br_hi[row]);
      else stage_features(g, sX, row, sc, grow, grow < m_lim);
      proxy_fence();
      mbar_arrive(&x_ready);
    };
    if (my_items > 0) {
      if (bis) {
        load_brackets(0);
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory");
      }
      stage_item(0);
    }
    for (long long tl = 0; tl < my_items; ++tl) {
      const long long grow = tile_of(tl) * kTcRows + row;
      const bool live = grow < m_lim;
      float part = 0.f;
      for (int L = 0; L < 3; ++L) {
        const long long G = 3 * tl + L;
        const int a = (int)(G & 1);
        if (ok && !mbar_wait(&acc_full[a], (uint32_t)((G >> 1) & 1))) ok = false;
        // the tensor-memory loads below are warp-collective: the warp goes on
        // only if all its lanes saw the phase complete
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc_fence_after();
        // columns 64 c + 16 sc .. +15 of accumulator a, c = 0..3
        uint32_t r[4][16];
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(lane_addr + (uint32_t)(a * kTcH + 64 * c), r[c]);
        tmem_wait_ld();
        tc_fence_before();
        mbar_arrive(&acc_empty[a]);
        if (L == 1 && ok && !bis && tl + 1 < my_items) {
          // the first layer of this tile has finished reading the feature
          // tile: stage the next tile's features now
          stage_item(tl + 1);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float* bias = sbias[L] + 64 * c + 16 * sc;
          if (L < 2) {
            uint32_t p[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              p[j] = pack_bf16(silu_tc(__uint_as_float(r[c][2 * j]) + bias[2 * j]),
                               silu_tc(__uint_as_float(r[c][2 * j + 1]) + bias[2 * j + 1]));
            uint8_t* hk = sH + c * (kTcRows * 128);
            *reinterpret_cast<uint4*>(hk + sw128(row, 2 * sc)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(hk + sw128(row, 2 * sc + 1)) = make_uint4(p[4], p[5], p[6], p[7]);
            proxy_fence();
            mbar_arrive(&h_ready[c]);
          } else {
            const float* w4 = sw4 + 64 * c + 16 * sc;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float z = __uint_as_float(r[c][j]) + bias[j];
              part = fmaf(__bfloat162float(__float2bfloat16(silu_tc(z))), w4[j], part);
            }
          }
        }
      }
      ypart[tl & 1][sc][row] = part;
      asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory");
      float yv = __int_as_float(0x7fc00000);
      if (sc == 0 && ok) {
        const float* yp = &ypart[tl & 1][0][row];
        yv = ((yp[0] + yp[kTcRows]) + (yp[2 * kTcRows] + yp[3 * kTcRows])) + g.b4[0];
      }
      if (!bis) {
        if (sc == 0 && live) g.y[grow] = yv;
        continue;
      }
      // one bisection step: keep the end predicted in collision
      const int step = (int)(tl % n_steps);
      if (sc == 0 && live) {
        const float f = 0.5f * (br_lo[row] + br_hi[row]);
        if (yv < g.margin) {
          br_hi[row] = f;
          br_bits[row] |= 1u << step;
        } else {
          br_lo[row] = f;
        }
        if (step == n_steps - 1) {
          g.s_lo[grow] = br_lo[row];
          g.s_hi[grow] = br_hi[row];
          g.s_bits[grow] = br_bits[row];
        }
      }
      if (tl + 1 < my_items) {
        if (step == n_steps - 1) load_brackets(tl + 1);
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory");
        if (ok) stage_item(tl + 1);
      }
    }
    if (!ok) atomicExch(g.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kEpiWarps) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
  }
}

// image of the three hidden-layer weight matrices in the swizzled K-major
// layout: chunk 0 = W1 [256 x 64], chunks 1..4 = W2 columns 64 (j - 1) ..,
// chunks 5..8 = W3 likewise; element (n, k) of a chunk at byte
// sw128(n, k / 8) + 2 (k % 8)
__global__ void k_mlp_tc_image(const __nv_bfloat16* __restrict__ W1, const __nv_bfloat16* __restrict__ W2,
                               const __nv_bfloat16* __restrict__ W3, uint8_t* __restrict__ img) {
  const int total = kChunksPerTile * kTcH * 64;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int j = i / (kTcH * 64), rem = i % (kTcH * 64), n = rem / 64, k = rem % 64;
    __nv_bfloat16 w;
    if (j == 0) w = W1[n * kTcF + k];
    else if (j <= 4) w = W2[n * kTcH + (j - 1) * 64 + k];
    else w = W3[n * kTcH + (j - 5) * 64 + k];
    *reinterpret_cast<__nv_bfloat16*>(img + j * kChunkBytes + sw128(n, k >> 3) + (k & 7) * 2) = w;
  }
}

}  // namespace

size_t mlp_tc_image_bytes() { return (size_t)kChunksPerTile * kChunkBytes; }

cudaError_t mlp_tc_build_image(const void* W1, const void* W2, const void* W3, void* img, cudaStream_t s) {
  k_mlp_tc_image<<<(kChunksPerTile * kTcH * 64 + 255) / 256, 256, 0, s>>>(
      static_cast<const __nv_bfloat16*>(W1), static_cast<const __nv_bfloat16*>(W2),
      static_cast<const __nv_bfloat16*>(W3), static_cast<uint8_t*>(img));
  return cudaGetLastError();
}

// y[i] = sd_hat of configuration i (q: n x rows_cap, stride ldq) for rows
// i < min(*m_dev, rows_cap) (all rows_cap rows when m_dev is null).
cudaError_t mlp_tc_forward(const float* q, long long ldq, int n, long long rows_cap, const int* m_dev,
                           const void* img, const float* b1, const float* b2, const float* b3, const float* w4,
                           const float* b4, float* y, int* err, cudaStream_t s) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  }
  if (rows_cap <= 0) return cudaSuccess;
  const long long tiles = (rows_cap + kTcRows - 1) / kTcRows;
  TcArgs a{q, ldq, n, rows_cap, m_dev, static_cast<const uint8_t*>(img), b1, b2, b3, w4, b4, y, err, nullptr,
           nullptr, nullptr, nullptr, nullptr, 0, 0.f};
  k_mlp_forward_tc<<<(unsigned)(tiles < sms ? tiles : sms), kThreads, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

// n_b surrogate bisection steps for rows i < min(*m_dev, rows_cap) in one
// launch: row i's bracket [s_lo[i], s_hi[i]] of s_p32 + f s_d32 (rows of 8
// floats) is halved n_b times, keeping the end where sd_hat < margin, and
// bit k of s_bits[i] records step k's prediction of a collision.
cudaError_t mlp_tc_bisect(int n, long long rows_cap, const int* m_dev, const void* img, const float* b1,
                          const float* b2, const float* b3, const float* w4, const float* b4, const float* s_p32,
                          const float* s_d32, float* s_lo, float* s_hi, uint32_t* s_bits, int n_b, float margin,
                          int* err, cudaStream_t s) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  }
  if (rows_cap <= 0 || n_b <= 0 || n_b > 32) return rows_cap <= 0 || n_b <= 0 ? cudaSuccess : cudaErrorInvalidValue;
  const long long tiles = (rows_cap + kTcRows - 1) / kTcRows;
  TcArgs a{nullptr, 0, n, rows_cap, m_dev, static_cast<const uint8_t*>(img), b1, b2, b3, w4, b4, nullptr, err, s_p32,
           s_d32, s_lo, s_hi, s_bits, n_b, margin};
  k_mlp_forward_tc<<<(unsigned)(tiles < sms ? tiles : sms), kThreads, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ezo
