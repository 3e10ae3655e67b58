// EI-ZO round kernels, first half (arXiv 2504.10783, Algorithm 1):
//   round_begin  - round size: delta_k (Eq. 9), M and |S| = max(N_p, M)
//   sample       - hit-and-run, one walk per sample (Sec. IV-B, IV-D)
//   check        - forward kinematics + sphere collision pairs (Sec. IV-D)
//   certify      - unadaptive test on the first M samples and stable
//                  selection of the first N_p colliding samples (Sec. IV-B)
#include "ezo_kernels_common.cuh"

#ifndef EZO_BOX_TU
#define EZO_BOX_TU 0  // 1: this translation unit holds only the box-geometry collision kernels
#endif

namespace ezo {

#if !EZO_BOX_TU

// ------------------------------------------------------------ round kernels --
__global__ void __launch_bounds__(1024) k_round_begin(BatchView v) { round_begin_block(v); }

// Reset of a batch in one launch: every segment's state and the rows of its
// starting polytope (st0[g].m rows; rows past a segment's m are never read),
// and the round summary's public part. One block per segment.
__global__ void __launch_bounds__(256) k_batch_reset(BatchView v, const SegState* __restrict__ st0,
                                                     const double* __restrict__ A0, const double* __restrict__ b0) {
  const int g = blockIdx.x;
  if (g >= v.B) return;
  const int m = st0[g].m;
  const long long base = (long long)g * v.m_cap;
  for (int i = threadIdx.x; i < m * v.n; i += blockDim.x) v.A[base * v.n + i] = A0[base * v.n + i];
  for (int i = threadIdx.x; i < m; i += blockDim.x) v.b[base + i] = b0[base + i];
  if (threadIdx.x == 0) v.st[g] = st0[g];
  if (g == 0 && threadIdx.x == 0) {
    v.summary->active = 0;
    v.summary->round = 0;
    v.summary->n_sample_tiles = 0;
    v.summary->n_bisect_tiles = 0;
  }
}

// End of a round fused with the next round's sizing (one launch fewer per
// round in the run loops): every active segment that reached N_it stops
// (Sec. IV-C), the others go to round k + 1, the next round's sample tiles are
// listed, and the round summary (and a graph's WHILE condition) is set.
__global__ void __launch_bounds__(1024) k_round_close(BatchView v) { round_close_block(v); }

// One pass of a 128-thread block over a tile of kTile walks at TSS lanes per
// walk (a tile takes TSS passes); writes the samples dimension-major.
template <int NDOF, int TSS>
__device__ __forceinline__ void sample_pass(const BatchView& v, const SegState& st, const float* A32,
                                            const SampleParams& p, int2 tile, int pass) {
  constexpr int WPB = 128 / TSS;
  const int gi = threadIdx.x / TSS, lw = threadIdx.x % TSS;
  float* S = v.S + (long long)v.n * st.sample_off;
  const int i = tile.y + pass * WPB + gi;
  float x[NDOF];
  // one lane per walk: a chain of exactly NDOF joints (the usual case) takes
  // n as a constant, which removes the walk's j < n tests (the arithmetic is
  // the same); the shared-walk kernel keeps one form, for its register budget
  if (TSS == 1) {
    if (i >= st.n_samples) return;
    if (v.n == NDOF)
      hnr_walk<NDOF>(A32, st.m, NDOF, p.v1f, p.ef, p.n_mix, v.keys, (uint32_t)i, p.round_k, p.stream, x,
                     st.box_rows);
    else
      hnr_walk<NDOF>(A32, st.m, v.n, p.v1f, p.ef, p.n_mix, v.keys, (uint32_t)i, p.round_k, p.stream, x,
                     st.box_rows);
  } else {
    const int ic = i < st.n_samples ? i : tile.y;
    hnr_walk_split<NDOF, TSS>(A32, st.m, v.n, p.v1f, p.ef, p.n_mix, v.keys, (uint32_t)ic, p.round_k, p.stream,
                              lw, x, st.box_rows);
    if (i >= st.n_samples || lw != 0) return;
  }
#pragma unroll
  for (int j = 0; j < NDOF; ++j)
    if (j < v.n) S[(long long)j * st.s_cap + i] = x[j];
}

// Lanes per walk for a round of n_tiles sample tiles: S = split_below_tiles
// tiles of 128 walks put one warp on every scheduler at one lane per walk;
// measured on the 7-DOF arm (1e4 to 1e5 walks, 14 to 54 rows), one lane is
// fastest from about 2 S tiles up, two from S, four from S / 4, and eight
// below. A nonzero sample_lanes fixes the count.
__device__ __forceinline__ int sample_passes(const BatchView& v, int n_tiles, int S) {
  if (v.sample_lanes) return v.sample_lanes;
  return n_tiles >= 2 * S ? 1 : (n_tiles >= S ? 2 : (4 * n_tiles >= S ? 4 : 8));
}

// Hit-and-run for every active segment. When the round has few walks (few
// active segments) several lanes share each walk, which cuts the latency of
// the sequential N_ms steps and fills the GPU; with many walks each lane runs
// one. The choice is made on the device from the round's tile count, so it
// also works inside a graph: the one-lane form (SPLIT = false) and the shared
// forms (SPLIT = true) are separate kernels, each with its own register
// budget, launched one after the other, and the one not chosen returns at
// once. Work units are (tile, pass) pairs: a tile of kTile walks takes one
// pass at one lane per walk, or 2, 4 or 8 passes at 2, 4 or 8 lanes per walk;
// blocks take them from the round's work queue.
// Register budgets: the one-lane form of chains up to 7 joints is held to 72
// registers (seven blocks per SM, no spills), which a round of ten segments'
// 1e4 walks fills in one wave; the shared forms to five blocks per SM.
template <int NDOF, bool SPLIT>
__global__ void __launch_bounds__(128, NDOF <= 7 ? (SPLIT ? 5 : 7) : 4)
    k_round_sample(BatchView v, int split_below_tiles) {
  extern __shared__ float4 smf4[];
  __shared__ SampleParams p;
  __shared__ int cur_seg;
  const int n_tiles = v.summary->n_sample_tiles;
  const int passes = sample_passes(v, n_tiles, split_below_tiles);
  if ((passes > 1) != SPLIT) return;
  float* A32 = reinterpret_cast<float*>(smf4);
  if (threadIdx.x == 0) cur_seg = -1;
  __syncthreads();
  int* q = &v.summary->q_sample;
  const int units = n_tiles * passes;
  for (int u = queue_first(v, q, units); u < units; u = queue_take(v, q, units)) {
    const int2 tile = v.sample_tiles[u / passes];
    const SegState& st = v.st[tile.x];
    if (tile.x != cur_seg) {
      __syncthreads();
      stage_polytope<NDOF>(A32, v.A + (long long)tile.x * v.m_cap * v.n, v.b + (long long)tile.x * v.m_cap, st.m,
                           v.n, v.n);
      if (threadIdx.x < EZO_MAX_DOF) {
        const int j = threadIdx.x;
        const double a1 = j < v.n ? v.v1[tile.x * v.n + j] : 0.0;
        const double a2 = j < v.n ? v.v2[tile.x * v.n + j] : 0.0;
        p.v1f[j] = (float)a1;
        p.ef[j] = (float)(a2 - a1);
      }
      if (threadIdx.x == 0) {
        p.n_mix = v.n_mix;
        p.stream = st.stream;
        p.round_k = (uint32_t)st.k;
        cur_seg = tile.x;
      }
      __syncthreads();
    }
    if (!SPLIT) sample_pass<NDOF, 1>(v, st, A32, p, tile, 0);
    else if (passes == 8) sample_pass<NDOF, 8>(v, st, A32, p, tile, u % passes);
    else if (passes == 4) sample_pass<NDOF, 4>(v, st, A32, p, tile, u % passes);
    else sample_pass<NDOF, 2>(v, st, A32, p, tile, u % passes);
  }
  queue_leave(v, q, &v.summary->left_sample, units);
}

#endif  // !EZO_BOX_TU

template <int NDOF, int T, bool BOX>
__global__ void __launch_bounds__(128) k_round_check(BatchView v, int max_obs_pad) {
  extern __shared__ float4 smem4[];
  __shared__ RobotSmem rs;
  __shared__ int cur_env;
  const int n_tiles = v.summary->n_sample_tiles;
  constexpr int PASSES = kTile / (128 / T);
  // work units are (tile, pass), taken from the round's work queue; a block
  // that finds none leaves before staging anything
  int* q = &v.summary->q_check;
  const int units = n_tiles * PASSES;
  int u = queue_first(v, q, units);
  if (u >= units) {
    queue_leave(v, q, &v.summary->left_check, units);
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
  for (; u < units; u = queue_take(v, q, units)) {
    const int2 tile = v.sample_tiles[u / PASSES];
    const int sub = (u % PASSES) * groups;
    const SegState& st = v.st[tile.x];
    const EnvDevFull& ef = v.envs[st.env];
    if (st.env != cur_env) {
      __syncthreads();
      stage_env(obs_s, nhw_s, ef.e);
      stage_env_boxes(gs.ebox, ef.e);
      if (threadIdx.x == 0) cur_env = st.env;
      __syncthreads();
    }
    const BoxCtx bx = box_ctx(gs, robot, nrbox, ef.e.n_box, gi);
    const float* S = v.S + (long long)v.n * st.sample_off;
    uint8_t* fl = v.flags + st.sample_off;
    {
      const int i = tile.y + sub + gi;
      const bool valid = i < st.n_samples;
      const int ic = valid ? i : tile.y;
      float qq[NDOF];
#pragma unroll
      for (int j = 0; j < NDOF; ++j) qq[j] = (j < v.n) ? S[(long long)j * st.s_cap + ic] : 0.f;
      const bool hit = collide_group<NDOF, T, BOX>(qq, rs, sph_s, obs_s, nhw_s, ef.e.n_obs, ef.e.n_obs_pad,
                                              ef.e.s_first, robot->self_pairs, robot->self_rr, ef.E, cen, lg, bx);
      if (valid && lg == 0) fl[i] = hit ? 1 : 0;
    }
  }
  queue_leave(v, q, &v.summary->left_check, units);
}

#if !EZO_BOX_TU

// Set editing (Sec. VI-B): configuration x is a candidate when it collides
// and lies in the current polytope, A x <= b + 1e-9 in FP64.
__device__ __forceinline__ bool edit_inside(const BatchView& v, int g, const SegState& st, int i) {
  const int n = v.n;
  const double* A = v.A + (long long)g * v.m_cap * n;
  const double* b = v.b + (long long)g * v.m_cap;
  const float* S = v.S + (long long)n * st.sample_off;
  double x[EZO_MAX_DOF];
  for (int j = 0; j < n; ++j) x[j] = (double)S[(long long)j * st.s_cap + i];
  for (int r = 0; r < st.m; ++r) {
    double ax = 0.0;
    for (int j = 0; j < n; ++j) ax = fma(A[(long long)r * n + j], x[j], ax);
    if (ax > b[r] + 1e-9) return false;
  }
  return true;
}

// Unadaptive test on the first M samples and stable compaction of the first
// N_p colliding samples (lowest sample index first). One block per segment.
// In set editing there is no test and a candidate must also lie in P.
__global__ void __launch_bounds__(1024) k_round_certify(BatchView v) {
  const int g = blockIdx.x;
  SegState& st = v.st[g];
  if (st.status != SEG_ACTIVE) return;
  __shared__ int warp_cnt[32];
  __shared__ int warp_col[32];
  __shared__ int s_running;
  __shared__ int s_count;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int S = st.n_samples, M = st.m_test, np = st.n_p;
  const uint8_t* fl = v.flags + st.sample_off;
  int* cidx = v.cand_idx + st.cand_off;
  if (threadIdx.x == 0) {
    s_running = 0;
    s_count = 0;
  }
  __syncthreads();
  int my_count = 0;
  // four consecutive samples per thread and pass (fewer block barriers)
  constexpr int PER = 4;
  for (int base = 0; base < S; base += PER * (int)blockDim.x) {
    const int i0 = base + PER * (int)threadIdx.x;
    int f[PER];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = i0 + k;
      f[k] = (i < S) ? (fl[i] != 0) : 0;
      if (v.edit && f[k]) f[k] = edit_inside(v, g, st, i) ? 1 : 0;
      if (i < M) my_count += f[k];
      cnt += f[k];
    }
    // stable positions: warp scan of the per-thread counts, then the warps
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_col[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = lane < nw ? warp_col[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) warp_cnt[lane] = w;  // inclusive
    }
    __syncthreads();
    const int running = s_running;
    int pos = running + (wid ? warp_cnt[wid - 1] : 0) + x - cnt;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      if (f[k]) {
        if (pos < np) cidx[pos] = i0 + k;
        ++pos;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_running = running + warp_cnt[nw - 1];
    __syncthreads();
    if (!v.edit && s_running >= np && base + PER * (int)blockDim.x >= M) break;
  }
  // block reduction of the count over the first M samples
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_count += __shfl_xor_sync(0xffffffffu, my_count, o);
  if (lane == 0) atomicAdd(&s_count, my_count);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int cnt = v.edit ? s_running : s_count;  // editing: colliding configurations in P
    st.count = cnt;
    st.checks += S;
    const bool accept = !v.edit && (double)cnt <= (double)M * (1.0 - v.tau) * v.eps;
    if (accept) {
      st.status = SEG_ACCEPTED;
      st.rounds = st.k;
      st.n_cand = 0;
    } else {
      const int nc = s_running < np ? s_running : np;
      st.n_cand = nc;
      if (v.sbis) {
        st.sur_evals += (long long)nc * v.n_b;  // exact checks are counted where they run
      } else {
        st.checks += (long long)nc * v.n_b;
        st.checks_bisect += (long long)nc * v.n_b;
      }
      const int nt = (nc + kTile - 1) / kTile;
      const int t0 = atomicAdd(&v.summary->n_bisect_tiles, nt);
      for (int t = 0; t < nt; ++t) v.bisect_tiles[t0 + t] = make_int2(g, t * kTile);
    }
  }
}

cudaError_t launch_round_begin(const BatchView& v, cudaStream_t s) {
  k_round_begin<<<1, 1024, 0, s>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_batch_reset(const BatchView& v, const SegState* st0, const double* A0, const double* b0,
                               cudaStream_t s) {
  if (v.B <= 0) return cudaSuccess;
  k_batch_reset<<<v.B, 256, 0, s>>>(v, st0, A0, b0);
  return cudaGetLastError();
}

cudaError_t launch_round_close(const BatchView& v, cudaStream_t s) {
  k_round_close<<<1, 1024, 0, s>>>(v);
  return cudaGetLastError();
}


cudaError_t launch_round_sample(const BatchView& v, int split_below_tiles, int grid, cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  EZO_DISPATCH_NDOF(v.n, {
    const size_t smem = hnr_smem_bytes<ND>(v.m_cap);
    auto kern1 = k_round_sample<ND, false>;
    auto kern2 = k_round_sample<ND, true>;
    err = set_smem(kern1, smem);
    if (err == cudaSuccess) err = set_smem(kern2, smem);
    if (err != cudaSuccess) return err;
    kern1<<<resident_grid(kern1, 128, smem, grid), 128, smem, s>>>(v, split_below_tiles);
    kern2<<<resident_grid(kern2, 128, smem, grid), 128, smem, s>>>(v, split_below_tiles);
  });
  return cudaGetLastError();
}

#endif  // !EZO_BOX_TU

#if EZO_BOX_TU
cudaError_t launch_round_check_box(const BatchView& v, int T, int grid, cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  const size_t smem = check_smem_layout(v.nsp_pad, v.max_obs_pad, 128, T, v.n_rbox, v.max_ebox);
  constexpr bool BB = EZO_BOX_TU != 0;
  EZO_DISPATCH_NDOF(v.n, EZO_DISPATCH_T(T, {
    auto kern = k_round_check<ND, TT, BB>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<resident_grid(kern, 128, smem, grid), 128, smem, s>>>(v, v.max_obs_pad);
  }));
  return cudaGetLastError();
}
#else
cudaError_t launch_round_check(const BatchView& v, int T, int grid, cudaStream_t s) {
  if (v.n_rbox || v.max_ebox) return launch_round_check_box(v, T, grid, s);
  cudaError_t err = cudaSuccess;
  const size_t smem = check_smem_layout(v.nsp_pad, v.max_obs_pad, 128, T, v.n_rbox, v.max_ebox);
  constexpr bool BB = EZO_BOX_TU != 0;
  EZO_DISPATCH_NDOF(v.n, EZO_DISPATCH_T(T, {
    auto kern = k_round_check<ND, TT, BB>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<resident_grid(kern, 128, smem, grid), 128, smem, s>>>(v, v.max_obs_pad);
  }));
  return cudaGetLastError();
}
#endif

#if !EZO_BOX_TU


cudaError_t launch_round_certify(const BatchView& v, cudaStream_t s) {
  k_round_certify<<<v.B, 1024, 0, s>>>(v);
  return cudaGetLastError();
}


#endif  // !EZO_BOX_TU

}  // namespace ezo
