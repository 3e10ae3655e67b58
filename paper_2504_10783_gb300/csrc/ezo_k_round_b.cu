// EI-ZO round kernels, second half (arXiv 2504.10783, Algorithm 1, Sec. VI-A):
//   bisect       - projection onto L (Eqs. 6-7) and N_b bisection steps
//                  toward it (Sec. IV-B, IV-C); with a learned surrogate
//                  attached (not in the paper) the N_b steps are first taken
//                  on its predicted signed distance (ezo_mlp_tc.cu), each end
//                  point is verified with one exact check, and the exact
//                  steps are redone where it is free
//   place        - order by distance to L, place up to N_f half spaces with
//                  step back (Eqs. 10-12), discard separated candidates
//   round_end    - round counter, iteration cap N_it (Sec. IV-C)
//   containment  - segment endpoints inside earlier polytopes (Sec. VI-A)
#include "ezo_kernels_common.cuh"

#ifndef EZO_BOX_TU
#define EZO_BOX_TU 0  // 1: this translation unit holds only the box-geometry collision kernels
#endif

namespace ezo {

// Bisection of one round in three kernels. k_bisect_prep (one thread per
// candidate) projects each candidate c onto L in FP64 (Eqs. 6-7) and keeps
// c_proj and c - c_proj in FP32; k_round_bisect takes the N_b halvings of
// Sec. IV-B toward c_proj with T lanes per candidate and records the
// decisions; k_bisect_finish (one thread per candidate) forms the end point
// c* = c_proj + f (c - c_proj), f the bracket's upper end, in FP64, with its
// distance to L and the tangent plane of Eq. (10). GB300 runs FP64 at 1/64 of
// the FP32 rate, so the FP64 steps go where every lane of a warp does useful
// work, and the halvings, which only need FP32 configurations, run without it.
//
// Row r of the round's candidate rows is candidate tile.y + (r % kTile) of
// bisection tile r / kTile (the numbering the surrogate's MLP batch uses too).
// c_proj (FP64 projection of sample si onto the segment's L, Eqs. 6-7) and
// c - c_proj, rounded to FP32
template <int NDOF>
__device__ __forceinline__ void bisect_project(const BatchView& v, const SegState& st, int g, int si,
                                               float (&p32)[NDOF], float (&dv32)[NDOF]) {
  const int n = v.n;
  const float* S = v.S + (long long)n * st.sample_off;
  double cs[NDOF], p[NDOF];
#pragma unroll
  for (int j = 0; j < NDOF; ++j) cs[j] = (j < n) ? (double)S[(long long)j * st.s_cap + si] : 0.0;
  project_fp64<NDOF>(cs, v.v1 + (long long)g * n, v.v2 + (long long)g * n, n, p);
#pragma unroll
  for (int j = 0; j < NDOF; ++j) {
    p32[j] = j < n ? (float)p[j] : 0.f;
    dv32[j] = j < n ? (float)(cs[j] - p[j]) : 0.f;
  }
}

// The bracket's upper end after the exact halvings: lo + 2^-N_b, lo the sum
// of 2^-(s+1) over the steps s whose midpoint was free
__device__ __forceinline__ double bisect_hi(uint32_t bits, int n_b) {
  uint64_t lo_u = 0;
  for (int s = 0; s < n_b; ++s)
    if (!((bits >> s) & 1u)) lo_u += 1ull << (n_b - 1 - s);
  return ldexp((double)(lo_u + 1), -n_b);
}

// c* = c_proj + hi (c - c_proj) of candidate c in FP64, its distance to L, the
// FP32 copy and its norm, and the tangent plane of Eq. (10) at c*:
// a = (c* - c_proj) / dist_L(c*), b = a^T c*
template <int NDOF>
__device__ __forceinline__ void bisect_end_point(const BatchView& v, const SegState& st, int g, int c,
                                                 double hi) {
  const int n = v.n;
  const long long co = st.cand_off;
  const int np = st.n_p;
  const double* v1 = v.v1 + (long long)g * n;
  const double* v2 = v.v2 + (long long)g * n;
  const float* S = v.S + (long long)n * st.sample_off;
  const int si = v.cand_idx[co + c];
  double cs[NDOF], p[NDOF], cst[NDOF], ps[NDOF];
#pragma unroll
  for (int j = 0; j < NDOF; ++j) cs[j] = (j < n) ? (double)S[(long long)j * st.s_cap + si] : 0.0;
  project_fp64<NDOF>(cs, v1, v2, n, p);
#pragma unroll
  for (int j = 0; j < NDOF; ++j) cst[j] = (j < n) ? fma(hi, cs[j] - p[j], p[j]) : 0.0;
  project_fp64<NDOF>(cst, v1, v2, n, ps);
  double d2 = 0.0;
  float cn2 = 0.f;
#pragma unroll
  for (int j = 0; j < NDOF; ++j) {
    if (j < n) {
      const double e = cst[j] - ps[j];
      d2 = fma(e, e, d2);
      v.cstar[(long long)n * co + (long long)j * np + c] = cst[j];
      const float f = (float)cst[j];
      v.c32[(long long)n * co + (long long)j * np + c] = f;
      cn2 = fmaf(f, f, cn2);
    }
  }
  const double dist = sqrt(d2);
  v.dist[co + c] = dist;
  v.cnorm[co + c] = sqrtf(cn2);
  const double inv = dist > 0.0 ? 1.0 / dist : 0.0;
  double bval = 0.0;
#pragma unroll
  for (int j = 0; j < NDOF; ++j) {
    if (j < n) {
      const double a = (cst[j] - ps[j]) * inv;
      v.ga[(long long)n * co + (long long)j * np + c] = a;
      bval = fma(a, cst[j], bval);
    }
  }
  v.gb[co + c] = bval;
}

#if !EZO_BOX_TU
template <int NDOF>
__global__ void __launch_bounds__(kRowBlock) k_bisect_prep(BatchView v) {
  const int n_tiles = v.summary->n_bisect_tiles;
  const int rows = n_tiles * kTile;
  const int ld = v.s_ld;
  if (v.sbis && blockIdx.x == 0 && threadIdx.x == 0) *v.s_rows = rows;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const int2 tile = v.bisect_tiles[r / kTile];
    const int c = tile.y + r % kTile;
    const SegState& st = v.st[tile.x];
    if (v.sbis) {
      // the surrogate's bracket [0, 1] and its end-point record
      v.s_lo[r] = 0.f;
      v.s_hi[r] = 1.f;
      v.s_bits[r] = 0u;
      v.s_ok[r] = 0;
    }
    if (c >= st.n_cand) {
      for (int j = 0; j < ld; ++j) v.s_p32[(long long)r * ld + j] = v.s_d32[(long long)r * ld + j] = 0.f;
      continue;
    }
    float p32[NDOF], dv32[NDOF];
    bisect_project<NDOF>(v, st, tile.x, v.cand_idx[st.cand_off + c], p32, dv32);
#pragma unroll
    for (int j = 0; j < NDOF; ++j) {
      if (j < ld) {
        v.s_p32[(long long)r * ld + j] = p32[j];
        v.s_d32[(long long)r * ld + j] = dv32[j];
      }
    }
    for (int j = NDOF; j < ld; ++j) v.s_p32[(long long)r * ld + j] = v.s_d32[(long long)r * ld + j] = 0.f;
  }
}

template <int NDOF>
__global__ void __launch_bounds__(kRowBlock) k_bisect_finish(BatchView v) {
  const int n_tiles = v.summary->n_bisect_tiles;
  const int rows = n_tiles * kTile;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const int2 tile = v.bisect_tiles[r / kTile];
    const int c = tile.y + r % kTile;
    const int g = tile.x;
    const SegState& st = v.st[g];
    if (c >= st.n_cand) continue;
    const uint32_t bits = v.bits[st.cand_off + c];
    // the surrogate's verified end point, or the exact halvings' upper end
    const double hi = (v.sbis && v.s_ok[r]) ? (double)v.s_hi[r] : bisect_hi(bits, v.n_b);
    bisect_end_point<NDOF>(v, st, g, c, hi);
  }
}
#endif  // !EZO_BOX_TU

// The halvings: the bracket [0, 1] of fractions along [c_proj, c] is kept as
// the integer lo_u in units of 2^-N_b (every midpoint of N_b <= 32 halvings
// is such a multiple, so the FP32 midpoint fraction is mid_u 2^-N_b rounded
// once, the value the FP64 bracket would give), and the configuration tested
// is c_proj + f (c - c_proj) in FP32. Bit s of the record is set when the
// midpoint of step s collides (the bracket's upper end moves there).
// bis_mode 1 instead checks the surrogate's end point once (s_ok records the
// outcome), and bis_mode 2 redoes the exact halvings for the candidates whose
// surrogate end point was free.
template <int NDOF, int T, bool BOX>
__global__ void __launch_bounds__(128) k_round_bisect(BatchView v, int max_obs_pad) {
  extern __shared__ float4 smem4[];
  __shared__ RobotSmem rs;
  __shared__ int cur_env;
  const int n_tiles = v.summary->n_bisect_tiles;
  // work units are (tile, pass), taken from this mode's work queue; a block
  // that finds none leaves before staging anything
  int* q = &v.summary->q_bisect[v.bis_mode];
  int* left = &v.summary->left_bisect[v.bis_mode];
  const int units = n_tiles * T;
  int u = queue_first(v, q, units, false);
  if (u >= units) {
    queue_leave(v, q, left, units);
    return;
  }
  const RobotDev* robot = v.robot;
  const int nsp = robot->n_spheres_pad, nrbox = robot->n_box;
  const int groups = blockDim.x / T;
  const GeomSmem gs = carve_geom(smem4, nsp, max_obs_pad, groups, nrbox, v.max_ebox);
  float4* sph_s = gs.sph;
  float4* obs_s = gs.obs;
  float* nhw_s = gs.nhw;
  stage_robot(rs, sph_s, robot);
  stage_robot_boxes(gs.rbox_l, robot);
  if (threadIdx.x == 0) cur_env = -1;
  __syncthreads();
  const int gi = threadIdx.x / T, lg = threadIdx.x % T;
  float4* cen = gs.cen_all + gi * (nsp + 1);
  const int ld = v.s_ld;
  const float scale = ldexpf(1.f, -v.n_b);
  static_assert(kTile % (128 / T) == 0, "tile must be a whole number of passes");
  for (; u < units; u = queue_take(v, q, units)) {
    const int2 tile = v.bisect_tiles[u / T];
    const int sub = (u % T) * groups;
    const int g = tile.x;
    const SegState& st = v.st[g];
    const EnvDevFull& ef = v.envs[st.env];
    if (st.env != cur_env) {
      __syncthreads();
      stage_env(obs_s, nhw_s, ef.e);
      stage_env_boxes(gs.ebox, ef.e);
      if (threadIdx.x == 0) cur_env = st.env;
      __syncthreads();
    }
    const BoxCtx bx = box_ctx(gs, robot, nrbox, ef.e.n_box, gi);
    // the scene's scalars in registers for the N_b checks
    const int n_obs = ef.e.n_obs, n_obs_pad = ef.e.n_obs_pad, s_first = ef.e.s_first;
    const float E = ef.E;
    const ushort2* self_pairs = robot->self_pairs;
    const float* self_rr = robot->self_rr;
    const int c = tile.y + sub + gi;
    const int row = (u / T) * kTile + sub + gi;
    bool valid = c < st.n_cand;
    if (v.bis_mode == 2) {
      // exact halvings only where the surrogate end point failed; a warp
      // whose candidates all passed skips the work together
      const bool need = valid && !v.s_ok[row];
      if (!__any_sync(0xffffffffu, need)) continue;
      valid = need;
    }
    float p32[NDOF], dv32[NDOF];
#pragma unroll
    for (int j = 0; j < NDOF; ++j) {
      p32[j] = j < ld ? v.s_p32[(long long)row * ld + j] : 0.f;
      dv32[j] = j < ld ? v.s_d32[(long long)row * ld + j] : 0.f;
    }
    uint32_t lo_u = 0u, bits = 0u;
    if (v.bis_mode == 1) {
      bits = v.s_bits[row];
    } else if (v.bis_mode == 2 && valid && lg == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&v.st[g].checks), (unsigned long long)v.n_b);
      atomicAdd(reinterpret_cast<unsigned long long*>(&v.st[g].checks_bisect), (unsigned long long)v.n_b);
    }
    // one call site of the collision test for both modes keeps the kernel
    // small enough for the instruction cache
    const int steps = v.bis_mode == 1 ? 1 : v.n_b;
    for (int s = 0; s < steps; ++s) {
      const uint32_t mid_u = v.bis_mode == 1 ? 0u : lo_u + (1u << (v.n_b - 1 - s));
      const float f = v.bis_mode == 1 ? v.s_hi[row] : __uint2float_rn(mid_u) * scale;
      float qq[NDOF];
#pragma unroll
      for (int j = 0; j < NDOF; ++j) qq[j] = fmaf(f, dv32[j], p32[j]);
      bool hit;
      if constexpr (T > 8)
        hit = collide_wide<NDOF, T>(qq, rs, sph_s, obs_s, nhw_s, n_obs, n_obs_pad, s_first, self_pairs, self_rr, E, cen,
                                    lg, bx);
      else
        hit = collide_group<NDOF, T, BOX>(qq, rs, sph_s, obs_s, nhw_s, n_obs, n_obs_pad, s_first, self_pairs, self_rr, E,
                                          cen, lg, bx);
      if (v.bis_mode == 1) {
        if (valid && lg == 0) {
          v.s_ok[row] = hit ? 1 : 0;
          atomicAdd(reinterpret_cast<unsigned long long*>(&v.st[g].checks), 1ull);
          atomicAdd(reinterpret_cast<unsigned long long*>(&v.st[g].checks_bisect), 1ull);
        }
        if (!hit) valid = false;  // no record: the exact pass (mode 2) redoes this candidate
      } else if (hit) {
        bits |= 1u << s;
      } else {
        lo_u = mid_u;
      }
    }
    if (valid && lg == 0) v.bits[st.cand_off + c] = bits;
  }
  queue_leave(v, q, left, units);
}

#if !EZO_BOX_TU
// Two halvings at a time, three warps per candidate (sphere scenes; bisection
// modes 0 and 2). Halving s tests the bracket's midpoint lo + 2h and halving
// s + 1 then tests lo + h if that collided, else lo + 3h (h = 2^(N_b-2-s) in
// units of 2^-N_b): warps 0, 1, 2 test lo + h, lo + 2h, lo + 3h together, each
// with the 32-lane check, and the two decisions follow from the three labels
// exactly as the two halvings would take them, so the record and the end
// point are the sequential halvings' bit for bit. Half the dependent checks
// for half again the checks; an odd last halving is warp 1's alone.
template <int NDOF>
__global__ void __launch_bounds__(96) k_round_bisect_pair(BatchView v, int max_obs_pad) {
  extern __shared__ float4 smem4[];
  __shared__ RobotSmem rs;
  __shared__ int cur_env;
  __shared__ int s_hit[3];
  const int n_tiles = v.summary->n_bisect_tiles;
  int* q = &v.summary->q_bisect[v.bis_mode];
  int* left = &v.summary->left_bisect[v.bis_mode];
  const int units = n_tiles * kTile;  // one candidate row per unit
  int u = queue_first(v, q, units, false);
  if (u >= units) {
    queue_leave(v, q, left, units);
    return;
  }
  const RobotDev* robot = v.robot;
  const int nsp = robot->n_spheres_pad;
  const GeomSmem gs = carve_geom(smem4, nsp, max_obs_pad, 3, 0, 0);
  float4* sph_s = gs.sph;
  float4* obs_s = gs.obs;
  float* nhw_s = gs.nhw;
  stage_robot(rs, sph_s, robot);
  if (threadIdx.x == 0) cur_env = -1;
  __syncthreads();
  const int w = threadIdx.x >> 5, lg = threadIdx.x & 31;
  float4* cen = gs.cen_all + w * (nsp + 1);
  const BoxCtx bx{};
  const int ld = v.s_ld;
  const int nb = v.n_b;
  const float scale = ldexpf(1.f, -nb);
  for (; u < units; u = queue_take(v, q, units)) {
    const int2 tile = v.bisect_tiles[u / kTile];
    const int c = tile.y + u % kTile;
    const int g = tile.x;
    const SegState& st = v.st[g];
    const EnvDevFull& ef = v.envs[st.env];
    if (st.env != cur_env) {
      __syncthreads();
      stage_env(obs_s, nhw_s, ef.e);
      if (threadIdx.x == 0) cur_env = st.env;
      __syncthreads();
    }
    const int n_obs = ef.e.n_obs, n_obs_pad = ef.e.n_obs_pad, s_first = ef.e.s_first;
    const float E = ef.E;
    const ushort2* self_pairs = robot->self_pairs;
    const float* self_rr = robot->self_rr;
    bool valid = c < st.n_cand;
    if (v.bis_mode == 2) valid = valid && !v.s_ok[u];
    if (!valid) continue;  // the whole block: u is the block's
    float p32[NDOF], dv32[NDOF];
#pragma unroll
    for (int j = 0; j < NDOF; ++j) {
      p32[j] = j < ld ? v.s_p32[(long long)u * ld + j] : 0.f;
      dv32[j] = j < ld ? v.s_d32[(long long)u * ld + j] : 0.f;
    }
    if (v.bis_mode == 2 && threadIdx.x == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&v.st[g].checks), (unsigned long long)nb);
      atomicAdd(reinterpret_cast<unsigned long long*>(&v.st[g].checks_bisect), (unsigned long long)nb);
    }
    uint32_t lo_u = 0u, bits = 0u;
    for (int s = 0; s < nb; s += 2) {
      const bool pair = s + 1 < nb;
      const uint32_t h = pair ? 1u << (nb - 2 - s) : 0u;
      // pair: warp w tests lo + (w + 1) h; single: warp 1 tests the midpoint
      const uint32_t mid_u = pair ? lo_u + (uint32_t)(w + 1) * h : lo_u + (1u << (nb - 1 - s));
      if (pair || w == 1) {
        const float f = __uint2float_rn(mid_u) * scale;
        float qq[NDOF];
#pragma unroll
        for (int j = 0; j < NDOF; ++j) qq[j] = fmaf(f, dv32[j], p32[j]);
        const bool hit =
            collide_wide<NDOF, 32>(qq, rs, sph_s, obs_s, nhw_s, n_obs, n_obs_pad, s_first, self_pairs, self_rr, E, cen, lg,
                                   bx);
        if (lg == 0) s_hit[w] = hit ? 1 : 0;
      }
      __syncthreads();
      const bool h1 = s_hit[0] != 0, h2 = s_hit[1] != 0, h3 = s_hit[2] != 0;
      __syncthreads();  // read before the next step's labels are written
      if (!pair) {
        if (h2) bits |= 1u << s;
        else lo_u += 1u << (nb - 1 - s);
      } else if (h2) {
        bits |= 1u << s;
        if (h1) bits |= 1u << (s + 1);
        else lo_u += h;
      } else {
        lo_u += 2u * h;
        if (h3) bits |= 1u << (s + 1);
        else lo_u += h;
      }
    }
    if (threadIdx.x == 0) v.bits[st.cand_off + c] = bits;
  }
  queue_leave(v, q, left, units);
}
#endif  // !EZO_BOX_TU

#if !EZO_BOX_TU

// Greedy placement: repeatedly take the closest surviving candidate (ties by
// sample index), place a_i^T x <= b_i - Delta_i, discard candidates with
// a_i^T c_j > b_i - Delta_i; at most N_f planes. One block per segment.
// The discard test runs in FP32 with a rounding bound and falls back to FP64
// inside the bound, so every decision equals the FP64 decision.
// CLOSE: the run loops' form, whose last block to finish also closes the
// round (round_close_block), one launch fewer per round.
template <int NDOF>
__device__ __forceinline__ void place_segment(const BatchView& v) {
  const int g = blockIdx.x;
  SegState& st = v.st[g];
  if (st.status != SEG_ACTIVE) return;
  const int nc = st.n_cand;
  const int n = v.n;
  const int np = st.n_p;
  const long long co = st.cand_off;
  extern __shared__ uint32_t alive[];  // nc bits
  __shared__ unsigned long long red_key[32];
  __shared__ int red_sidx[32];
  __shared__ int red_idx[32];
  __shared__ int s_best;
  __shared__ double s_a[EZO_MAX_DOF];
  __shared__ float s_a32[EZO_MAX_DOF];
  __shared__ double s_beta;
  __shared__ float s_beta32;
  __shared__ int s_stop;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nwords = (nc + 31) >> 5;
  for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
    const int rem = nc - (w << 5);
    alive[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
  }
  if (threadIdx.x == 0) s_stop = 0;
  __syncthreads();
  const double* dist = v.dist + co;
  const int* cidx = v.cand_idx + co;
  const double* v1 = v.v1 + (long long)g * n;
  const double* v2 = v.v2 + (long long)g * n;
  double* A = v.A + (long long)g * v.m_cap * n;
  double* bb = v.b + (long long)g * v.m_cap;
  int placed = 0;
  const float u = 5.9604644775390625e-8f;
  // per-thread best survivor (distance bits, sample index, candidate)
  unsigned long long best_key = ~0ull;
  int best_i = 0x7fffffff;
  int best_c = -1;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const unsigned long long key = (unsigned long long)__double_as_longlong(dist[c]);
    const int si = cidx[c];
    if (key < best_key || (key == best_key && si < best_i)) {
      best_key = key;
      best_i = si;
      best_c = c;
    }
  }
  // warp 0's lane j < n keeps the segment's endpoints' coordinate j
  const double my_v1 = (wid == 0 && lane < n) ? v1[lane] : 0.0;
  const double my_v2 = (wid == 0 && lane < n) ? v2[lane] : 0.0;
  for (int f = 0; f < v.n_f; ++f) {
    // block arg-min of (distance, sample index) over the survivors
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, best_key, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, best_i, o);
      const int c2 = __shfl_xor_sync(0xffffffffu, best_c, o);
      if (k2 < best_key || (k2 == best_key && i2 < best_i)) {
        best_key = k2;
        best_i = i2;
        best_c = c2;
      }
    }
    if (lane == 0) {
      red_key[wid] = best_key;
      red_sidx[wid] = best_i;
      red_idx[wid] = best_c;
    }
    __syncthreads();
    if (wid == 0) {
      unsigned long long bk = lane < nw ? red_key[lane] : ~0ull;
      int bi = lane < nw ? red_sidx[lane] : 0x7fffffff;
      int bc = lane < nw ? red_idx[lane] : -1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        const int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
        if (k2 < bk || (k2 == bk && i2 < bi)) {
          bk = k2;
          bi = i2;
          bc = c2;
        }
      }
      // the plane, with the loads of warp 0's lanes in flight together: lane
      // j < n holds a_j = (grad dist_L(c*))_j (Eq. 10, from the bisection
      // kernel) and v1_j, v2_j; lane 0 the distance and b = a^T c*
      const bool have = bc >= 0;
      double a = 0.0, dbc = 0.0, bval = 0.0;
      if (have && lane < n) a = v.ga[(long long)n * co + (long long)lane * np + bc];
      if (have && lane == 0) {
        dbc = dist[bc];
        bval = v.gb[co + bc];
      }
      double av1 = a * my_v1, av2 = a * my_v2;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        av1 += __shfl_xor_sync(0xffffffffu, av1, o);
        av2 += __shfl_xor_sync(0xffffffffu, av2, o);
      }
      int stop = 0;
      double beta = 0.0, delta = 0.0;
      int row = 0;
      if (lane == 0) {
        if (!have) {
          stop = 1;
        } else if (dbc <= v.t_col) {
          stop = 2;  // segment likely in collision (Sec. IV-C)
        } else if (st.m >= v.m_cap) {
          stop = 3;
        } else {
          // step back (Eqs. 11-12): r = max(a^T v1, a^T v2) - b + Delta_max
          const double r = fmax(av1, av2) - bval + v.step_back_max;
          delta = r > 0.0 ? v.step_back_max - r : v.step_back_max;
          beta = bval - delta;
          row = st.m;
        }
      }
      stop = __shfl_sync(0xffffffffu, stop, 0);
      row = __shfl_sync(0xffffffffu, row, 0);
      if (stop == 0 && lane < n) {
        s_a[lane] = a;
        s_a32[lane] = (float)a;
        A[(long long)row * n + lane] = a;
      }
      if (lane == 0) {
        s_best = bc;
        s_stop = stop;
        if (stop == 0) {
          s_beta = beta;
          s_beta32 = (float)beta;
          bb[row] = beta;
          st.m = row + 1;
          v.placed_idx[g * v.n_f + f] = bc;
          v.placed_delta[g * v.n_f + f] = delta;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    ++placed;
    const int bc = s_best;
    const double beta = s_beta;
    const float beta32 = s_beta32;
    // one pass: discard candidates outside the new half space and find the
    // best survivor for the next plane
    best_key = ~0ull;
    best_i = 0x7fffffff;
    best_c = -1;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      if (!((alive[c >> 5] >> (c & 31)) & 1u)) continue;
      bool out;
      if (c == bc) {
        out = true;
      } else {
        // the candidate's coordinates in one batch of loads, then the dot product
        float cj[NDOF];
#pragma unroll
        for (int j = 0; j < NDOF; ++j) cj[j] = (j < n) ? v.c32[(long long)n * co + (long long)j * np + c] : 0.f;
        float s32 = 0.f;
#pragma unroll
        for (int j = 0; j < NDOF; ++j)
          if (j < n) s32 = fmaf(s_a32[j], cj[j], s32);
        const float bound = 2.f * (float)(n + 4) * u * (v.cnorm[co + c] + fabsf(beta32)) + 1e-30f;
        if (fabsf(s32 - beta32) > bound) {
          out = s32 > beta32;
        } else {
          double sd = 0.0;
          for (int j = 0; j < n; ++j) sd = fma(s_a[j], v.cstar[(long long)n * co + (long long)j * np + c], sd);
          out = sd > beta;
        }
      }
      if (out) {
        atomicAnd(&alive[c >> 5], ~(1u << (c & 31)));
      } else {
        const unsigned long long key = (unsigned long long)__double_as_longlong(dist[c]);
        const int si = cidx[c];
        if (key < best_key || (key == best_key && si < best_i)) {
          best_key = key;
          best_i = si;
          best_c = c;
        }
      }
    }
    // no barrier needed here: warp 0 read red_* before the barrier above, and
    // the shared plane is rewritten only after the next iteration's first
    // barrier, which every thread reaches after this pass
  }
  if (threadIdx.x == 0) {
    st.n_placed = placed;
    st.planes += placed;
    if (s_stop == 2) {
      st.status = SEG_IN_COLLISION;
      st.rounds = st.k;
    } else if (s_stop == 3) {
      st.status = SEG_CAPACITY;
      st.rounds = st.k;
    }
  }
}

template <int NDOF, bool CLOSE>
__global__ void __launch_bounds__(1024) k_round_place(BatchView v) {
  place_segment<NDOF>(v);
  if constexpr (CLOSE) {
    // every block reports when its segment is placed; the last one closes
    // the round for all of them
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(&v.summary->left_place, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      if (threadIdx.x == 0) v.summary->left_place = 0;
      round_close_block(v);
    }
  }
}

__global__ void k_round_end(BatchView v) {
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  const int act = round_end_segments(v);
  if (act) atomicAdd(&s_active, act);
  __syncthreads();
  if (threadIdx.x == 0) round_summary_close(v, s_active);
}

__global__ void k_containment(BatchView v, uint8_t* contained, double tol) {
  // one block per (k, j) pair of the same path with j < k
  const int k = blockIdx.x;
  const int j = v.path_first[k] + (int)blockIdx.y;
  if (j >= k) return;
  const int n = v.n;
  const SegState& sj = v.st[j];
  __shared__ int s_out;
  if (threadIdx.x == 0) s_out = 0;
  __syncthreads();
  const double* A = v.A + (long long)j * v.m_cap * n;
  const double* b = v.b + (long long)j * v.m_cap;
  const double* p1 = v.v1 + (long long)k * n;
  const double* p2 = v.v2 + (long long)k * n;
  for (int r = threadIdx.x; r < sj.m; r += blockDim.x) {
    double s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < n; ++c) {
      s1 = fma(A[(long long)r * n + c], p1[c], s1);
      s2 = fma(A[(long long)r * n + c], p2[c], s2);
    }
    if (s1 > b[r] + tol || s2 > b[r] + tol) s_out = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) contained[(long long)k * v.max_path_len + blockIdx.y] = s_out ? 0 : 1;
}

// The skip rule of Sec. VI-A after a speculative run, on the device: one
// warp per path (its segments are consecutive, from path_first) walks the
// segments in order; a segment is skipped when both its endpoints lie in the
// polytope of an earlier kept segment of the path (contained), and every
// segment after one reported in collision goes idle. For paths of up to 32
// segments lane j holds segment j's status and column j of the containment
// flags, all loaded at once, and each segment's test is a ballot over the
// lanes; longer paths take lane 0's sequential walk over global memory.
__global__ void __launch_bounds__(128) k_path_skip(BatchView v, const uint8_t* __restrict__ contained) {
  const int L = v.max_path_len;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int g0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g0 < v.B; g0 += warps) {
    if (v.path_first[g0] != g0) continue;  // the whole warp
    // path length (up to 33 read here; longer paths take the fallback)
    const bool in = g0 + lane < v.B && v.path_first[g0 + lane] == g0;
    const unsigned run = __ballot_sync(0xffffffffu, in);
    const int K = (~run == 0u) ? 33 : __ffs(~run) - 1;
    if (K <= 32) {
      const int st_l = lane < K ? v.st[g0 + lane].status : 0;
      unsigned col = 0u;  // bit k: segment k's endpoints lie in segment `lane`'s polytope
      for (int k = lane + 1; k < K; ++k)
        if (contained[(long long)(g0 + k) * L + lane]) col |= 1u << k;
      unsigned kept = 0u;
      bool stopped = false;
      for (int k = 0; k < K; ++k) {
        const bool in_kept = lane < k && ((kept >> lane) & 1u) && st_l != SEG_SKIPPED && st_l != SEG_IDLE &&
                             ((col >> k) & 1u);
        const bool skip = stopped || __ballot_sync(0xffffffffu, in_kept) != 0u;
        const int st_k = __shfl_sync(0xffffffffu, st_l, k);
        if (skip) {
          if (lane == 0) v.st[g0 + k].status = stopped ? SEG_IDLE : SEG_SKIPPED;
        } else {
          kept |= 1u << k;
          if (st_k == SEG_IN_COLLISION) stopped = true;
        }
      }
    } else if (lane == 0) {
      bool stopped = false;
      for (int g = g0; g < v.B && v.path_first[g] == g0; ++g) {
        bool skip = stopped;
        for (int j = g0; j < g && !skip; ++j) {
          const int sj = v.st[j].status;
          if (sj != SEG_SKIPPED && sj != SEG_IDLE && contained[(long long)g * L + (j - g0)]) skip = true;
        }
        if (skip) {
          v.st[g].status = stopped ? SEG_IDLE : SEG_SKIPPED;
          continue;
        }
        if (v.st[g].status == SEG_IN_COLLISION) stopped = true;
      }
    }
  }
}

// The wavefront order of Sec. VI-A on the device, one wave per call: every
// path runs its segments in order, the current segment of every path in the
// same batched run. Per path (indexed by its first segment g0): w_next[g0] is
// the next segment to consider (-1 when the path is done), w_last[g0] the
// segment the previous wave ran (-1 if none), w_kept[g] = 1 for a segment
// that ran. The previous wave's segment ends the path when it reports a
// collision (t_col, Sec. IV-C); otherwise the next segments whose endpoints
// lie in the polytope of a kept earlier segment of the path (contained, from
// k_containment) are skipped and the first other one becomes active. One
// block; the block's count of active segments sets both WHILE conditions of
// the wave graph (waves and rounds).
__global__ void k_wave_init(BatchView v, int* w_next, int* w_last, uint8_t* w_kept) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < v.B; g += gridDim.x * blockDim.x) {
    v.st[g].status = SEG_IDLE;
    w_kept[g] = 0;
    w_next[g] = v.path_first[g] == g ? g : -1;
    w_last[g] = -1;
  }
}

__global__ void k_wave_select(BatchView v, const uint8_t* __restrict__ contained, int* w_next, int* w_last,
                              uint8_t* w_kept, unsigned long long cond_waves, unsigned long long cond_rounds) {
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  const int L = v.max_path_len;
  int act = 0;
  for (int g0 = threadIdx.x; g0 < v.B; g0 += blockDim.x) {
    if (v.path_first[g0] != g0) continue;
    int g = w_next[g0];
    const int last = w_last[g0];
    if (last >= 0 && v.st[last].status == SEG_IN_COLLISION) g = -1;
    if (g < 0) {
      w_next[g0] = -1;
      w_last[g0] = -1;
      continue;
    }
    while (g < v.B && v.path_first[g] == g0) {
      bool skip = false;
      for (int j = g0; j < g && !skip; ++j)
        if (w_kept[j] && contained[(long long)g * L + (j - g0)]) skip = true;
      if (!skip) break;
      v.st[g].status = SEG_SKIPPED;
      ++g;
    }
    if (g < v.B && v.path_first[g] == g0) {
      v.st[g].status = SEG_ACTIVE;
      w_kept[g] = 1;
      w_last[g0] = g;
      w_next[g0] = g + 1;
      ++act;
    } else {
      w_next[g0] = -1;
      w_last[g0] = -1;
    }
  }
  if (act) atomicAdd(&s_active, act);
  __syncthreads();
#if CUDART_VERSION >= 12040
  if (threadIdx.x == 0) {
    const unsigned c = s_active > 0 ? 1u : 0u;
    if (cond_waves) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_waves, c);
    if (cond_rounds) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_rounds, c);
  }
#endif
}

#endif  // !EZO_BOX_TU

#if EZO_BOX_TU
cudaError_t launch_round_bisect_box(const BatchView& v, int T, int grid, cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  const size_t smem = check_smem_layout(v.nsp_pad, v.max_obs_pad, 128, T, v.n_rbox, v.max_ebox);
  constexpr bool BB = EZO_BOX_TU != 0;
  EZO_DISPATCH_NDOF(v.n, EZO_DISPATCH_T(T, {
    auto kern = k_round_bisect<ND, TT, BB>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<resident_grid(kern, 128, smem, grid), 128, smem, s>>>(v, v.max_obs_pad);
  }));
  return cudaGetLastError();
}
#else
// T = 16 or 32 lanes per candidate take the wide check (sphere scenes; box
// scenes run at 8)
cudaError_t launch_round_bisect(const BatchView& v, int T, int grid, cudaStream_t s) {
  if (v.n_rbox || v.max_ebox) return launch_round_bisect_box(v, T > 8 ? 8 : T, grid, s);
  if (T == kBisectPairLanes && v.bis_mode == 1) T = 32;  // one check per candidate: the 32-lane kernel
  if (T == kBisectPairLanes) {
    cudaError_t err = cudaSuccess;
    const size_t smem = check_smem_layout(v.nsp_pad, v.max_obs_pad, 96, 32, 0, 0);
    EZO_DISPATCH_NDOF(v.n, {
      auto kern = k_round_bisect_pair<ND>;
      err = set_smem(kern, smem);
      if (err != cudaSuccess) return err;
      kern<<<resident_grid(kern, 96, smem, std::max(grid, 1) * 4), 96, smem, s>>>(v, v.max_obs_pad);
    });
    return cudaGetLastError();
  }
  cudaError_t err = cudaSuccess;
  const size_t smem = check_smem_layout(v.nsp_pad, v.max_obs_pad, 128, T, v.n_rbox, v.max_ebox);
  constexpr bool BB = EZO_BOX_TU != 0;
  EZO_DISPATCH_NDOF(v.n, EZO_DISPATCH_T_WIDE(T, {
    auto kern = k_round_bisect<ND, TT, BB>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<resident_grid(kern, 128, smem, grid), 128, smem, s>>>(v, v.max_obs_pad);
  }));
  return cudaGetLastError();
}
#endif

#if !EZO_BOX_TU

cudaError_t launch_bisect_prep(const BatchView& v, int grid, cudaStream_t s) {
  EZO_DISPATCH_NDOF(v.n, { k_bisect_prep<ND><<<grid, kRowBlock, 0, s>>>(v); });
  return cudaGetLastError();
}

cudaError_t launch_bisect_finish(const BatchView& v, int grid, cudaStream_t s) {
  EZO_DISPATCH_NDOF(v.n, { k_bisect_finish<ND><<<grid, kRowBlock, 0, s>>>(v); });
  return cudaGetLastError();
}

cudaError_t launch_bisect_exact(const BatchView& v, int T, int grid, int grid_rows, cudaStream_t s) {
  BatchView w = v;
  w.bis_mode = 0;
  cudaError_t e = launch_bisect_prep(w, grid_rows, s);
  if (e == cudaSuccess) e = launch_round_bisect(w, T, grid, s);
  if (e == cudaSuccess) e = launch_bisect_finish(w, grid_rows, s);
  return e;
}

cudaError_t launch_round_place(const BatchView& v, cudaStream_t s, bool close) {
  // alive bitmask for the largest N_p of the batch
  const size_t smem = (size_t)((v.np_max + 31) / 32) * sizeof(uint32_t);
  cudaError_t err = cudaSuccess;
  EZO_DISPATCH_NDOF(v.n, {
    if (close) {
      err = set_smem(k_round_place<ND, true>, smem);
      if (err != cudaSuccess) return err;
      k_round_place<ND, true><<<v.B, 1024, smem, s>>>(v);
    } else {
      err = set_smem(k_round_place<ND, false>, smem);
      if (err != cudaSuccess) return err;
      k_round_place<ND, false><<<v.B, 1024, smem, s>>>(v);
    }
  });
  return cudaGetLastError();
}


cudaError_t launch_round_end(const BatchView& v, cudaStream_t s) {
  k_round_end<<<1, 256, 0, s>>>(v);
  return cudaGetLastError();
}


cudaError_t launch_containment(const BatchView& v, uint8_t* contained, double tol, cudaStream_t s) {
  dim3 grid(v.B, v.max_path_len);
  k_containment<<<grid, 128, 0, s>>>(v, contained, tol);
  return cudaGetLastError();
}

cudaError_t launch_path_skip(const BatchView& v, const uint8_t* contained, cudaStream_t s) {
  k_path_skip<<<(v.B + 3) / 4, 128, 0, s>>>(v, contained);  // one warp per segment index
  return cudaGetLastError();
}

cudaError_t launch_wave_init(const BatchView& v, int* w_next, int* w_last, uint8_t* w_kept, cudaStream_t s) {
  k_wave_init<<<(v.B + 255) / 256, 256, 0, s>>>(v, w_next, w_last, w_kept);
  return cudaGetLastError();
}

cudaError_t launch_wave_select(const BatchView& v, const uint8_t* contained, int* w_next, int* w_last,
                               uint8_t* w_kept, unsigned long long cond_waves, unsigned long long cond_rounds,
                               cudaStream_t s) {
  k_wave_select<<<1, 1024, 0, s>>>(v, contained, w_next, w_last, w_kept, cond_waves, cond_rounds);
  return cudaGetLastError();
}


#endif  // !EZO_BOX_TU

}  // namespace ezo
