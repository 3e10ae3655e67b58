// Device helpers shared by the kernel translation units: hit-and-run walk,
// polytope staging, shared-memory layout of the collision kernels, FP64
// projection onto the seed segment, template dispatch.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "ezo_engine.cuh"

namespace ezo {

// ------------------------------------------------------------- hit-and-run --
struct SampleParams {
  float v1f[EZO_MAX_DOF];
  float ef[EZO_MAX_DOF];
  int n_mix;
  uint32_t stream, round_k;
  PhiloxKeys keys;
};

// The walk's approximate functions, each one PTX instruction with subnormal
// operands and results taken as zero (.ftz): reciprocal, base-2 logarithm,
// reciprocal square root, sine and cosine. The walk's values reach the
// subnormal range only in measure-zero cases (a direction component or a
// row's rate a . d within 2^-126 of zero); the flush spares the scaling that
// the non-flushing forms put around each instruction.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sin_approx(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float cos_approx(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One hit-and-run walk of `n_mix` steps inside {x : A32 x <= b32}.
// Random stream: Philox block (walk, draw, round, stream); draw 0 gives the
// start x = v1 + u (v2 - v1); step s uses draws 1 + s W .. 1 + s W + W - 1,
// W = max(1, ceil(2 ceil(n/2) / 4)), whose words w_0.. give Gaussian pair i
// from the top 24 bits of (w_2i, w_2i+1) by Box-Muller and the step length
// from the low bytes of w_0, w_1, w_2 (one 24-bit integer, w_0 lowest).
__device__ __forceinline__ float step_uniform(uint32_t w0, uint32_t w1, uint32_t w2) {
  const uint32_t t = (w0 & 0xffu) | ((w1 & 0xffu) << 8) | ((w2 & 0xffu) << 16);
  return (float)t * 5.9604644775390625e-8f;  // 2^-24
}

// One Box-Muller pair from two 32-bit words: rho = sqrt(-2 ln u1) with u1 in
// (0, 1], angle 2 pi u2 with u2 in [0, 1). -2 ln u1 = -2 ln 2 log2 u1, and the
// square root is tt times its reciprocal square root; sine and cosine are the
// hardware approximations (absolute error ~2^-21 on [-pi, pi]), so the angle
// is shifted to pi (2 u2 - 1) in [-pi, pi), which negates both.
__device__ __forceinline__ void box_muller(uint32_t w1, uint32_t w2, float& za, float& zb) {
  const float tt = lg2_approx(u01_oc(w1)) * -1.38629436f;  // -2 ln 2 in FP32
  const float rho = tt > 0.f ? tt * rsqrt_approx(tt) : 0.f;
  const float a = 3.14159265358979f * fmaf(2.f, u01_co(w2), -1.f);
  za = -rho * cos_approx(a);
  zb = -rho * sin_approx(a);
}

// Philox blocks per walk step (the W above)
__host__ __device__ constexpr int hnr_blocks_per_step(int n) {
  return (2 * ((n + 1) / 2) + 3) / 4 > 1 ? (2 * ((n + 1) / 2) + 3) / 4 : 1;
}

// Shared-memory image of a polytope for the sampler, two rows per record:
// record P holds rows 2P and 2P + 1 interleaved, -a_{2P,j} and -a_{2P+1,j} at
// floats 2j and 2j + 1 (j < NDOF, zero-padded; negated, so that the slack
// b - a . x is one FMA chain from b), then b_{2P} and b_{2P+1}. The
// record is rounded up to an odd number of float4s, so that the eight
// consecutive records which the lanes of a shared walk read at once fall in
// different shared-memory banks. One 64-bit load gives a coefficient of two
// rows as the float2 operand of a packed FP32 FMA. A missing last row of an
// odd count is a zero row (rate 0, so it bounds nothing).
template <int NDOF>
__host__ __device__ constexpr int hnr_pair_stride() {
  return ((2 * NDOF + 5) & ~3) + ((((2 * NDOF + 5) & ~3) / 4) % 2 == 0 ? 4 : 0);
}

template <int NDOF>
__host__ __device__ constexpr size_t hnr_smem_bytes(int m) {
  return (size_t)((m > 1 ? m : 1) + 1) / 2 * hnr_pair_stride<NDOF>() * sizeof(float);
}

// b of row r in the paired image
template <int NDOF>
__device__ __forceinline__ float hnr_row_b(const float* __restrict__ A32, int r) {
  return A32[(r >> 1) * hnr_pair_stride<NDOF>() + 2 * NDOF + (r & 1)];
}

// Chord bounds from the row pairs P0, P0 + step, .. < P1: for row r the slack
// s = b_r - a_r . x and the rate a_r . d give the crossing t = s / rate,
// which bounds the chord from above when the rate is positive and from below
// when it is negative. From the negated coefficients the slack is the chain
// fmaf(-a_j, x_j, .) over j = 0 .. NDOF-1 from b_r, and nr = -rate the chain
// fmaf(-a_j, d_j, .) from 0, so t = -(s / nr): s times the reciprocal of nr,
// negated. Both rows of a pair advance together in packed FP32 operations
// against x and d duplicated into both halves (xx, dd); each half is a
// row's scalar chain, so every row's slack, rate and ratio are bit for bit
// those of a row taken alone, and min/max do not depend on the order or on
// how the pairs are split between lanes. For a joint-box row (a = +-e_j) the
// chains are exact but for the one term, so the bounds equal chord_joint's.
// Four pairs per iteration let the chains overlap.
template <int NDOF>
__device__ __forceinline__ void chord_pairs(const float* __restrict__ A32, int P0, int P1, int step,
                                            const float2 (&xx)[NDOF], const float2 (&dd)[NDOF], float& t_lo,
                                            float& t_hi) {
  constexpr int PS = hnr_pair_stride<NDOF>();
#pragma unroll 4
  for (int P = P0; P < P1; P += step) {
    const float2* rec = reinterpret_cast<const float2*>(A32 + P * PS);
    float2 sl = rec[NDOF], nr = make_float2(0.f, 0.f);  // slack from b, -rate from 0
#pragma unroll
    for (int j = 0; j < NDOF; ++j) {
      const float2 na = rec[j];
      sl = __ffma2_rn(na, xx[j], sl);
      nr = __ffma2_rn(na, dd[j], nr);
    }
    const float2 q = __fmul2_rn(sl, make_float2(rcp_approx(nr.x), rcp_approx(nr.y)));  // -t
    if (nr.x < 0.f) t_hi = fminf(t_hi, -q.x);
    if (nr.x > 0.f) t_lo = fmaxf(t_lo, -q.x);
    if (nr.y < 0.f) t_hi = fminf(t_hi, -q.y);
    if (nr.y > 0.f) t_lo = fmaxf(t_lo, -q.y);
  }
}

// The chord bounds of the joint-box rows j (+e_j x <= hi_j, b = bh) and n + j
// (-e_j x <= -lo_j, b = bl) without their dot products. With a = +-e_j the
// general rows compute a . x = +-x_j and a . d = +-d_j exactly, so the
// crossings are q1 = (bh - x_j) r and q2 = (bl + x_j) (-r), r = 1 / d_j, bit for
// bit theirs (the reciprocal is odd). For d_j > 0 row j bounds from above and
// row n + j from below, for d_j < 0 the reverse, and in both cases
// q1 - q2 has the sign of d_j (bh >= -bl and rounding is monotone), so the
// upper bound is max(q1, q2) and the lower min(q1, q2); d_j = 0 bounds nothing.
__device__ __forceinline__ void chord_joint(float bh, float bl, float xj, float dj, float& t_lo, float& t_hi) {
  const float r = rcp_approx(dj);
  const float q1 = (bh - xj) * r;
  const float q2 = (bl + xj) * -r;
  if (dj != 0.f) {
    t_hi = fminf(t_hi, fmaxf(q1, q2));
    t_lo = fmaxf(t_lo, fminf(q1, q2));
  }
}

// chord_joint over every joint, the box bounds in registers (bhi[j] = b of
// row j, blo[j] = b of row n + j)
template <int NDOF>
__device__ __forceinline__ void chord_box_r(int n, const float (&bhi)[NDOF], const float (&blo)[NDOF],
                                            const float (&x)[NDOF], const float (&d)[NDOF], float& t_lo,
                                            float& t_hi) {
#pragma unroll
  for (int j = 0; j < NDOF; ++j)
    if (j < n) chord_joint(bhi[j], blo[j], x[j], d[j], t_lo, t_hi);
}

// x and d in both halves of a float2, the operands chord_pairs multiplies
// each row pair with
template <int NDOF>
__device__ __forceinline__ void dup_pairs(const float (&x)[NDOF], const float (&d)[NDOF], float2 (&xx)[NDOF],
                                          float2 (&dd)[NDOF]) {
#pragma unroll
  for (int j = 0; j < NDOF; ++j) {
    xx[j] = make_float2(x[j], x[j]);
    dd[j] = make_float2(d[j], d[j]);
  }
}

// Unit direction d (zero beyond n) and step uniform u_t of walk step s; u_t =
// -1 marks a step whose Gaussians are all zero, which does not move.
template <int NDOF>
__device__ __forceinline__ void hnr_direction(const PhiloxKeys& ks, uint32_t walk, uint32_t rk, uint32_t stream,
                                              int s, int n, int W, float (&d)[NDOF], float& ut) {
  constexpr int WMAX = hnr_blocks_per_step(NDOF);
  uint32_t w[4 * WMAX];
#pragma unroll
  for (int b = 0; b < WMAX; ++b) {
    u32x4 r = u32x4{0u, 0u, 0u, 0u};
    if (b < W) r = philox4x32_10(u32x4{walk, (uint32_t)(1 + s * W + b), rk, stream}, ks);
    w[4 * b] = r.x;
    w[4 * b + 1] = r.y;
    w[4 * b + 2] = r.z;
    w[4 * b + 3] = r.w;
  }
#pragma unroll
  for (int i = 0; i < (NDOF + 1) / 2; ++i) {
    float za = 0.f, zb = 0.f;
    if (2 * i < n) box_muller(w[2 * i], w[2 * i + 1], za, zb);
    d[2 * i] = za;
    if (2 * i + 1 < NDOF) d[2 * i + 1] = (2 * i + 1 < n) ? zb : 0.f;
  }
  float nrm2 = 0.f;
#pragma unroll
  for (int j = 0; j < NDOF; ++j) nrm2 = fmaf(d[j], d[j], nrm2);
  const float inv = nrm2 > 0.f ? rsqrt_approx(nrm2) : 0.f;
#pragma unroll
  for (int j = 0; j < NDOF; ++j) d[j] *= inv;
  ut = nrm2 > 0.f ? step_uniform(w[0], w[1], w[2]) : -1.f;
}

// The move of one step: t = t_lo + u_t (t_hi - t_lo) on the chord [t_lo, t_hi]
// (clamped to contain 0), skipped for a degenerate or unbounded chord.
template <int NDOF>
__device__ __forceinline__ void hnr_move(float ut, float t_lo, float t_hi, const float (&d)[NDOF],
                                         float (&x)[NDOF]) {
  t_hi = fmaxf(t_hi, 0.f);
  t_lo = fminf(t_lo, 0.f);
  if (ut >= 0.f && isfinite(t_hi) && isfinite(t_lo) && (t_hi - t_lo) >= 1e-12f) {
    const float t = fmaf(ut, t_hi - t_lo, t_lo);
#pragma unroll
    for (int j = 0; j < NDOF; ++j) x[j] = fmaf(t, d[j], x[j]);
  }
}

template <int NDOF>
__device__ __forceinline__ void hnr_start(const PhiloxKeys& ks, uint32_t walk, uint32_t rk, uint32_t stream, int n,
                                          const float* v1f, const float* ef, float (&x)[NDOF]) {
  const u32x4 r0 = philox4x32_10(u32x4{walk, 0u, rk, stream}, ks);
  const float u0 = u01_co(r0.x);
#pragma unroll
  for (int j = 0; j < NDOF; ++j) x[j] = (j < n) ? fmaf(u0, ef[j], v1f[j]) : 0.f;
}

// When box_rows = 2n the polytope's first 2n rows are the joint box (row j:
// +e_j x <= hi_j, row n + j: -e_j x <= -lo_j) and take the chord_joint form.
template <int NDOF>
__device__ __forceinline__ void hnr_walk(const float* __restrict__ A32, int m,
                                         int n, const float* v1f, const float* ef, int n_mix,
                                         const PhiloxKeys& ks, uint32_t walk, uint32_t rk, uint32_t stream,
                                         float (&x)[NDOF], int box_rows = 0) {
  const int W = hnr_blocks_per_step(n);
  hnr_start<NDOF>(ks, walk, rk, stream, n, v1f, ef, x);
  // the joint-box bounds, loaded once for all steps
  float bhi[NDOF], blo[NDOF];
#pragma unroll
  for (int j = 0; j < NDOF; ++j) {
    bhi[j] = (box_rows && j < n) ? hnr_row_b<NDOF>(A32, j) : 0.f;
    blo[j] = (box_rows && j < n) ? hnr_row_b<NDOF>(A32, n + j) : 0.f;
  }
  for (int s = 0; s < n_mix; ++s) {
    float d[NDOF], ut;
    hnr_direction<NDOF>(ks, walk, rk, stream, s, n, W, d, ut);
    float t_lo = -INFINITY, t_hi = INFINITY;
    if (box_rows) chord_box_r<NDOF>(n, bhi, blo, x, d, t_lo, t_hi);
    float2 xx[NDOF], dd[NDOF];
    dup_pairs<NDOF>(x, d, xx, dd);
    chord_pairs<NDOF>(A32, box_rows >> 1, (m + 1) >> 1, 1, xx, dd, t_lo, t_hi);
    hnr_move<NDOF>(ut, t_lo, t_hi, d, x);
  }
}

// The same walk as hnr_walk, shared by TS consecutive lanes of a warp (TS in
// 2, 4, 8). The steps go in groups of TS: lane lw draws the direction and
// step uniform of step s0 + lw of the group, and each step of the group takes
// its direction from its lane by shuffles. Lane lw scans the polytope row
// pairs lw, lw + TS, .. (and, from four lanes up, the joints lw, lw + TS, ..
// of the box rows; with two lanes each lane takes the whole box), and the
// chord bounds are combined with min/max shuffles. Every lane ends with the
// same x, bit-identical to hnr_walk's (same arithmetic per direction and per
// row; min and max do not depend on the order), so a segment's samples do not
// depend on how many other walks share its round. All lanes of the warp must
// call this together.
template <int NDOF, int TS>
__device__ __forceinline__ void hnr_walk_split(const float* __restrict__ A32, int m, int n, const float* v1f,
                                               const float* ef, int n_mix, const PhiloxKeys& ks,
                                               uint32_t walk, uint32_t rk, uint32_t stream, int lw,
                                               float (&x)[NDOF], int box_rows = 0) {
  constexpr int JS = TS >= 4 ? (NDOF + TS - 1) / TS : NDOF;  // box joints per lane
  const int W = hnr_blocks_per_step(n);
  hnr_start<NDOF>(ks, walk, rk, stream, n, v1f, ef, x);
  // this lane's joint-box bounds: joint jj TS + lw (TS >= 4) or jj (TS = 2)
  float bhi[JS], blo[JS];
#pragma unroll
  for (int jj = 0; jj < JS; ++jj) {
    const int j = TS >= 4 ? jj * TS + lw : jj;
    bhi[jj] = (box_rows && j < n) ? hnr_row_b<NDOF>(A32, j) : 0.f;
    blo[jj] = (box_rows && j < n) ? hnr_row_b<NDOF>(A32, n + j) : 0.f;
  }
  for (int s0 = 0; s0 < n_mix; s0 += TS) {
    float dn[NDOF], un = -1.f;
    if (s0 + lw < n_mix) {
      hnr_direction<NDOF>(ks, walk, rk, stream, s0 + lw, n, W, dn, un);
    } else {
#pragma unroll
      for (int j = 0; j < NDOF; ++j) dn[j] = 0.f;
    }
#pragma unroll 1
    for (int l = 0; l < TS && s0 + l < n_mix; ++l) {
      float d[NDOF];
#pragma unroll
      for (int j = 0; j < NDOF; ++j) d[j] = __shfl_sync(0xffffffffu, dn[j], l, TS);
      const float ut = __shfl_sync(0xffffffffu, un, l, TS);
      float t_lo = -INFINITY, t_hi = INFINITY;
      if (box_rows) {
#pragma unroll
        for (int jj = 0; jj < JS; ++jj) {
          if (TS >= 4) {
            // joint jj TS + lw: its coordinate and direction by selection
            float xs = 0.f, ds = 0.f;
#pragma unroll
            for (int l2 = 0; l2 < TS; ++l2)
              if (jj * TS + l2 < NDOF && l2 == lw) {
                xs = x[jj * TS + l2];
                ds = d[jj * TS + l2];
              }
            if (jj * TS + lw < n) chord_joint(bhi[jj], blo[jj], xs, ds, t_lo, t_hi);
          } else if (jj < n) {
            chord_joint(bhi[jj], blo[jj], x[jj], d[jj], t_lo, t_hi);
          }
        }
      }
      float2 xx[NDOF], dd[NDOF];
      dup_pairs<NDOF>(x, d, xx, dd);
      chord_pairs<NDOF>(A32, (box_rows >> 1) + lw, (m + 1) >> 1, TS, xx, dd, t_lo, t_hi);
#pragma unroll
      for (int o = 1; o < TS; o <<= 1) {
        t_hi = fminf(t_hi, __shfl_xor_sync(0xffffffffu, t_hi, o, TS));
        t_lo = fmaxf(t_lo, __shfl_xor_sync(0xffffffffu, t_lo, o, TS));
      }
      hnr_move<NDOF>(ut, t_lo, t_hi, d, x);
    }
  }
}

// The polytope {A x <= b} (FP64, m rows, row stride lda) as the sampler's
// paired FP32 image (see hnr_pair_stride; coefficients negated); an odd last
// row is paired with a zero row.
template <int NDOF>
__device__ __forceinline__ void stage_polytope(float* A32, const double* __restrict__ A,
                                               const double* __restrict__ b, int m, int lda, int n) {
  constexpr int PS = hnr_pair_stride<NDOF>();
  const int np = (m + 1) >> 1;
  for (int i = threadIdx.x; i < np * PS; i += blockDim.x) {
    const int P = i / PS, c = i - P * PS;
    const int r = 2 * P + (c & 1), j = c >> 1;
    float v = 0.f;
    if (r < m) {
      if (j < n) v = -(float)A[(long long)r * lda + j];
      else if (j == NDOF) v = (float)b[r];
    }
    A32[i] = v;
  }
}

// ------------------------------------------------------------ work queue --
// The round kernels spread a round's work units over the SMs explicitly.
// Blocks are dispatched SM by SM, so a round with fewer units than resident
// blocks would otherwise crowd its units onto the first SMs. A block first
// takes a seat on its SM (rank r = its arrival order there); only ranks below
// ceil(units / SMs) work, and rank r on SM s starts with unit r * SMs + s, so
// the units go round-robin over the SMs. Every unit is claimed once (an
// atomic flag), and a working block then takes further units in order from a
// counter, skipping claimed ones, until none is left: every unit is done
// exactly once whatever the placement. A claim holds the launch's epoch, so
// the claims need no clearing: q_claim[0] counts the launches (advanced by
// the last block of each), the launch's epoch is that count + 1, and unit u's
// claim is q_claim[1 + u] (the array starts at zero). The functions below are
// called by every thread of the block together and return a block-uniform
// value.
__device__ __forceinline__ bool queue_claim(const BatchView& v, int u) {
  if (!v.q_claim) return true;
  const int epoch = *(volatile int*)&v.q_claim[0] + 1;
  return atomicExch(&v.q_claim[1 + u], epoch) != epoch;
}

// The block's first unit, or `units` when it has no seat (it then calls
// queue_leave and returns). spread = false skips the round-robin first unit
// (the seated blocks then take units in arrival order): measured on the
// bisection's short rounds, the 16-lane check runs faster packed that way.
__device__ __forceinline__ int queue_first(const BatchView& v, int* q, int units, bool spread = true) {
  __shared__ int s_unit;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    int u = units;
    const int cap = v.n_sm > 0 ? (units + v.n_sm - 1) / v.n_sm : units;
    const int rank = (sm < (unsigned)kSeatSlots && v.sm_seats) ? atomicAdd(&v.sm_seats[sm], 1) : 0;
    if (rank < cap) {
      const long long pre = (long long)rank * v.n_sm + sm;
      if (spread && pre < units && queue_claim(v, (int)pre)) u = (int)pre;
      while (u == units) {
        const int t = atomicAdd(q, 1);
        if (t >= units) break;
        if (queue_claim(v, t)) u = t;
      }
    }
    s_unit = u;
  }
  __syncthreads();
  return s_unit;
}

// The next unclaimed unit, or `units` when none is left.
__device__ __forceinline__ int queue_take(const BatchView& v, int* q, int units) {
  __shared__ int s_unit;
  __syncthreads();  // the previous unit's value has been read by every thread
  if (threadIdx.x == 0) {
    int u = units;
    while (u == units) {
      const int t = atomicAdd(q, 1);
      if (t >= units) break;
      if (queue_claim(v, t)) u = t;
    }
    s_unit = u;
  }
  __syncthreads();
  return s_unit;
}

// Called once by every block of the launch when it takes no more units: the
// last block to leave clears the seats and the counter and advances the
// claims' epoch for the next launch (every other block of the kernel is done
// with them by then).
__device__ __forceinline__ void queue_leave(const BatchView& v, int* q, int* left, int units) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(left, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    (void)units;
    if (v.sm_seats)
      for (int i = threadIdx.x; i < kSeatSlots; i += blockDim.x) v.sm_seats[i] = 0;
    if (v.q_claim && v.q_claim[0] >= (1 << 30)) {
      // the epochs wrap: clear the claims (once in 2^30 launches)
      for (int i = 1 + threadIdx.x; i <= v.q_claim_cap; i += blockDim.x) v.q_claim[i] = 0;
      __syncthreads();
      if (threadIdx.x == 0) atomicExch(&v.q_claim[0], 0);
    } else if (v.q_claim && threadIdx.x == 0) {
      atomicAdd(&v.q_claim[0], 1);
    }
    if (threadIdx.x == 0) {
      atomicExch(q, 0);
      atomicExch(left, 0);
    }
  }
}

// ------------------------------------------------------------- round end --
// Sec. IV-C "Maximum iterations": an active segment that ran N_it rounds
// stops with EZO_SEG_MAX_ITER, the others move to the next round. Returns the
// number of this thread's segments that stay active.
__device__ __forceinline__ int round_end_segments(const BatchView& v) {
  int act = 0;
  for (int g = threadIdx.x; g < v.B; g += blockDim.x) {
    SegState& st = v.st[g];
    if (st.status == SEG_ACTIVE) {
      if (st.k >= v.n_it_max) {
        st.status = SEG_MAX_ITER;
        st.rounds = st.k;
      } else {
        st.k += 1;
        ++act;
      }
    }
  }
  return act;
}

// Round summary after a round (one thread): active segments, rounds run and,
// inside a graph, the WHILE condition.
__device__ __forceinline__ void round_summary_close(const BatchView& v, int active) {
  v.summary->active = active;
  v.summary->round += 1;
#if CUDART_VERSION >= 12040
  if (v.graph_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)v.graph_cond, active > 0 ? 1u : 0u);
#endif
}

// --------------------------------------------------------- round sizing --
// Round size of Sec. IV-B: delta_k = 6 delta / (pi^2 k^2),
// M = ceil(2 ln(1/delta_k) / (eps tau^2)), |S| = max(N_p, M).
__device__ __forceinline__ int round_test_size(int k, double eps, double delta, double tau) {
  const double dk = 6.0 * delta / (3.141592653589793 * 3.141592653589793 * (double)k * (double)k);
  return (int)ceil(2.0 * log(1.0 / dk) / (eps * tau * tau));
}

// Round size of every active segment and the round's list of sample tiles
// (block-wide exclusive scan over the segments). Runs in one block.
__device__ __forceinline__ void round_begin_block(const BatchView& v) {
  __shared__ int warp_sum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < v.B; base += blockDim.x) {
    const int g = base + threadIdx.x;
    int tiles = 0;
    if (g < v.B) {
      SegState& st = v.st[g];
      if (st.status == SEG_ACTIVE && v.edit) {
        // set editing: the given configurations are already in place
        st.m_test = 0;
        st.n_cand = 0;
        st.count = 0;
        st.n_placed = 0;
        tiles = (st.n_samples + kTile - 1) / kTile;
      } else if (st.status == SEG_ACTIVE) {
        const int M = round_test_size(st.k, v.eps, v.delta, v.tau);
        int S = M > st.n_p ? M : st.n_p;
        if (S > st.s_cap) S = st.s_cap;  // capacity is sized for M at N_it; never hit
        st.m_test = M;
        st.n_samples = S;
        // algorithmic FP32 work of this round's walks, per walk step
        // 2mn + 5m + 6n: the rate a_r . d of every row (2n), the slack update
        // s_r -= t q_r, the ratio and the two bound updates (5 per row), and
        // the direction's normalisation and the move (6n). The Gaussians'
        // transcendental functions and the random-number generator are not
        // counted, nor the second dot product per row that this kernel uses
        // instead of carrying the slack.
        st.sample_flops += (long long)S * v.n_mix * (2ll * st.m * v.n + 5ll * st.m + 6ll * v.n);
        st.n_cand = 0;
        st.count = 0;
        st.n_placed = 0;
        tiles = (S + kTile - 1) / kTile;
      }
    }
    // block exclusive scan of tiles
    int x = tiles;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) warp_sum[lane] = w;
    }
    __syncthreads();
    const int excl = carry + (wid ? warp_sum[wid - 1] : 0) + x - tiles;
    for (int t = 0; t < tiles; ++t) v.sample_tiles[excl + t] = make_int2(g, t * kTile);
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    v.summary->n_sample_tiles = carry;
    v.summary->n_bisect_tiles = 0;
  }
}

// End of a round fused with the next round's sizing, by one block: every
// active segment that reached N_it stops (Sec. IV-C), the others go to round
// k + 1, the next round's sample tiles are listed, and the round summary (and
// a graph's WHILE condition) is set.
__device__ __forceinline__ void round_close_block(const BatchView& v) {
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  const int act = round_end_segments(v);
  if (act) atomicAdd(&s_active, act);
  __syncthreads();
  round_begin_block(v);
  __syncthreads();
  if (threadIdx.x == 0) round_summary_close(v, s_active);
}

// ------------------------------------------------------- collision checks --
// Shared memory of the collision kernels: robot spheres, obstacles, per group
// sphere centres, obstacle offsets, then the boxes (robot boxes in their
// frames, obstacle boxes, per group robot boxes in the world; 4 float4 each).
__host__ __device__ inline size_t check_smem_layout(int nsp, int nobs, int threads, int T, int nrbox = 0,
                                                    int nebox = 0) {
  const int groups = threads / T;
  return (size_t)(nsp + nobs + groups * (nsp + 1)) * sizeof(float4) + (size_t)nobs * sizeof(float) +
         (size_t)4 * (nrbox + nebox + groups * nrbox) * sizeof(float4);
}

struct GeomSmem {
  float4* sph;
  float4* obs;
  float4* cen_all;
  float* nhw;
  float4* rbox_l;
  float4* ebox;
  float4* rbox_w_all;
};

// nobs is a multiple of 8, so the box arrays after the obstacle offsets stay
// 16-byte aligned
__device__ __forceinline__ GeomSmem carve_geom(float4* base, int nsp, int nobs, int groups, int nrbox, int nebox) {
  GeomSmem g;
  g.sph = base;
  g.obs = g.sph + nsp;
  g.cen_all = g.obs + nobs;
  g.nhw = reinterpret_cast<float*>(g.cen_all + groups * (nsp + 1));
  g.rbox_l = reinterpret_cast<float4*>(g.nhw + nobs);
  g.ebox = g.rbox_l + 4 * nrbox;
  g.rbox_w_all = g.ebox + 4 * nebox;
  return g;
}

__device__ __forceinline__ BoxCtx box_ctx(const GeomSmem& g, const RobotDev* robot, int nrbox, int n_ebox, int gi) {
  BoxCtx b;
  b.rbox_l = g.rbox_l;
  b.ebox = g.ebox;
  b.rbox_w = g.rbox_w_all + gi * 4 * nrbox;
  b.n_ebox = n_ebox;
  b.sb_pairs = robot->sb_pairs;
  b.bb_pairs = robot->bb_pairs;
  return b;
}


// Projection of Eqs. (6)-(7) in FP64: c_proj = (1 - alpha) v1 + alpha v2.
template <int NDOF>
__device__ __forceinline__ void project_fp64(const double (&c)[NDOF], const double* v1, const double* v2, int n,
                                             double (&p)[NDOF]) {
  double ee = 0.0, ce = 0.0;
#pragma unroll
  for (int j = 0; j < NDOF; ++j) {
    if (j < n) {
      const double e = v2[j] - v1[j];
      ee = fma(e, e, ee);
      ce = fma(c[j] - v1[j], e, ce);
    }
  }
  double alpha = 0.0;
  if (ee > 0.0) alpha = fmin(fmax(ce / ee, 0.0), 1.0);
#pragma unroll
  for (int j = 0; j < NDOF; ++j) p[j] = (j < n) ? ((ee > 0.0) ? (1.0 - alpha) * v1[j] + alpha * v2[j] : v1[j]) : 0.0;
}

// ND = the smallest compiled chain length >= n (3, 7 or 16); every kernel
// guards its loops with j < n, so shorter chains run in a longer template.
#define EZO_DISPATCH_NDOF(n, ...)            \
  do {                                       \
    if ((n) > 3 && (n) <= 7) {               \
      constexpr int ND = 7;                  \
      __VA_ARGS__;                           \
    } else if ((n) <= 3) {                   \
      constexpr int ND = 3;                  \
      __VA_ARGS__;                           \
    } else {                                 \
      constexpr int ND = EZO_MAX_DOF;        \
      __VA_ARGS__;                           \
    }                                        \
  } while (0)

// BB = whether the scene has box geometries (separate kernels keep the
// sphere-only ones at their register budget)
#define EZO_DISPATCH_BOX(flag, ...) \
  do {                              \
    if (flag) {                     \
      constexpr bool BB = true;     \
      __VA_ARGS__;                  \
    } else {                        \
      constexpr bool BB = false;    \
      __VA_ARGS__;                  \
    }                               \
  } while (0)

#define EZO_DISPATCH_T(T, ...)               \
  do {                                       \
    if ((T) == 1) {                          \
      constexpr int TT = 1;                  \
      __VA_ARGS__;                           \
    } else if ((T) == 2) {                   \
      constexpr int TT = 2;                  \
      __VA_ARGS__;                           \
    } else if ((T) == 4) {                   \
      constexpr int TT = 4;                  \
      __VA_ARGS__;                           \
    } else {                                 \
      constexpr int TT = 8;                  \
      __VA_ARGS__;                           \
    }                                        \
  } while (0)

// EZO_DISPATCH_T with the wide groups of 16 and 32 lanes (the bisection)
#define EZO_DISPATCH_T_WIDE(T, ...)          \
  do {                                       \
    if ((T) == 16) {                         \
      constexpr int TT = 16;                 \
      __VA_ARGS__;                           \
    } else if ((T) == 32) {                  \
      constexpr int TT = 32;                 \
      __VA_ARGS__;                           \
    } else {                                 \
      EZO_DISPATCH_T(T, __VA_ARGS__);        \
    }                                        \
  } while (0)

// Raises a kernel's dynamic shared memory limit once per (kernel, size).
// The cache is keyed by the kernel's address: instantiations that share a
// signature must not share an entry.
// Raises a kernel's dynamic shared-memory limit to `bytes` (cached per
// kernel). The default 48 KB limit covers static and dynamic shared memory
// together, so the attribute is set for anything above 32 KB.
inline cudaError_t set_smem_impl(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, size_t>> done;
  if (bytes <= 32 * 1024) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first == kernel && d.second >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  for (auto& d : done)
    if (d.first == kernel) {
      d.second = bytes;
      return e;
    }
  done.emplace_back(kernel, bytes);
  return e;
}

template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  return set_smem_impl(reinterpret_cast<const void*>(kernel), bytes);
}

// At most one wave of resident blocks (cached per kernel, block size, shared
// memory and device): the round kernels loop over their work units with a
// grid stride, so blocks beyond what the SMs hold at once would only be
// dispatched to find no work.
inline int resident_grid_impl(const void* kernel, int threads, size_t smem, int grid_cap) {
  struct Entry {
    const void* k;
    int threads;
    size_t smem;
    int dev;
    int blocks;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return grid_cap;
  std::lock_guard<std::mutex> lock(mu);
  for (const Entry& e : cache)
    if (e.k == kernel && e.threads == threads && e.smem == smem && e.dev == dev)
      return std::max(1, std::min(grid_cap, e.blocks));
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1 || sms < 1) {
    (void)cudaGetLastError();
    return grid_cap;
  }
  cache.push_back(Entry{kernel, threads, smem, dev, per_sm * sms});
  return std::max(1, std::min(grid_cap, per_sm * sms));
}

template <typename K>
inline int resident_grid(K kernel, int threads, size_t smem, int grid_cap) {
  return resident_grid_impl(reinterpret_cast<const void*>(kernel), threads, smem, grid_cap);
}

}  // namespace ezo
