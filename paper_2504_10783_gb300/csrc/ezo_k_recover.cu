// Kernels for recovering from detected collisions (arXiv 2504.10783,
// Sec. VI-B):
//   k_check_path - a piecewise-linear path checked at fine steps: each point
//                  is interpolated in FP64 on its edge, rounded to FP32 and
//                  checked with the same FK and sphere test as the samples
//   k_coverage   - whether each segment of a seed path lies in some polytope
//                  of the same path (both endpoints, A x <= b + tol)
// Set editing itself runs the batch's round kernels (labels, selection,
// bisection, placement) on the given configurations.
#include "ezo_kernels_common.cuh"

#ifndef EZO_BOX_TU
#define EZO_BOX_TU 0  // 1: this translation unit holds only the box-geometry collision kernels
#endif

namespace ezo {

#if !EZO_BOX_TU

// Point i of the discretised path: edge k with off[k] <= i < off[k + 1],
// t = (i - off[k]) / N_k with N_k = off[k + 1] - off[k] - 1 pieces, and
// q = v_k + t (v_{k+1} - v_k) with separately rounded FP64 products and sums.
#endif  // !EZO_BOX_TU

template <int NDOF, int T, bool BOX>
__global__ void __launch_bounds__(128) k_check_path(const RobotDev* __restrict__ robot, EnvDev env, float E,
                                                    const double* __restrict__ verts, int n_edges,
                                                    const long long* __restrict__ off, long long N,
                                                    uint8_t* __restrict__ point_flags,
                                                    uint8_t* __restrict__ edge_flags) {
  extern __shared__ float4 smem4[];
  __shared__ RobotSmem rs;
  const int nsp = robot->n_spheres_pad, nrbox = robot->n_box;
  const int groups = blockDim.x / T;
  const GeomSmem gs = carve_geom(smem4, nsp, env.n_obs_pad, groups, nrbox, env.n_box);
  float4* sph_s = gs.sph;
  float4* obs_s = gs.obs;
  float* nhw_s = gs.nhw;
  stage_robot(rs, sph_s, robot);
  stage_robot_boxes(gs.rbox_l, robot);
  stage_env(obs_s, nhw_s, env);
  stage_env_boxes(gs.ebox, env);
  __syncthreads();
  const int gi = threadIdx.x / T, lg = threadIdx.x % T;
  float4* cen = gs.cen_all + gi * (nsp + 1);
  const BoxCtx bx = box_ctx(gs, robot, nrbox, env.n_box, gi);
  const int n = rs.n;
  for (long long base = (long long)blockIdx.x * groups; base < N; base += (long long)gridDim.x * groups) {
    const long long i = base + gi;
    const long long ic = i < N ? i : N - 1;
    int lo = 0, hi = n_edges - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= ic) lo = mid;
      else hi = mid - 1;
    }
    const int k = lo;
    const long long pieces = off[k + 1] - off[k] - 1;
    const double t = (double)(ic - off[k]) / (double)pieces;
    const double* va = verts + (long long)k * n;
    const double* vb = va + n;
    float qq[NDOF];
#pragma unroll
    for (int j = 0; j < NDOF; ++j)
      qq[j] = (j < n) ? (float)__dadd_rn(va[j], __dmul_rn(t, __dsub_rn(vb[j], va[j]))) : 0.f;
    const bool hit = collide_group<NDOF, T, BOX>(qq, rs, sph_s, obs_s, nhw_s, env.n_obs, env.n_obs_pad,
                                            env.s_first, robot->self_pairs, robot->self_rr, E, cen, lg, bx);
    if (i < N && lg == 0) {
      if (point_flags) point_flags[i] = hit ? 1 : 0;
      if (hit) edge_flags[k] = 1;  // every writer stores the same value
    }
  }
}

#if EZO_BOX_TU
cudaError_t launch_check_path_box(const RobotDev* robot, int n, int nsp_pad, int n_rbox, const EnvDev& env, float E,
                              const double* verts, int n_edges, const long long* off, long long N,
                              uint8_t* point_flags, uint8_t* edge_flags, int T, int grid_cap, cudaStream_t s) {
  if (N <= 0 || n_edges <= 0) return cudaSuccess;
  cudaError_t err = cudaSuccess;
  const int threads = 128;
  const size_t smem = check_smem_layout(nsp_pad, env.n_obs_pad, threads, T, n_rbox, env.n_box);
  const long long groups = threads / T;
  long long grid = (N + groups - 1) / groups;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  constexpr bool BB = EZO_BOX_TU != 0;
  EZO_DISPATCH_NDOF(n, EZO_DISPATCH_T(T, {
    auto kern = k_check_path<ND, TT, BB>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(robot, env, E, verts, n_edges, off, N, point_flags, edge_flags);
  }));
  return cudaGetLastError();
}
#else
cudaError_t launch_check_path(const RobotDev* robot, int n, int nsp_pad, int n_rbox, const EnvDev& env, float E,
                              const double* verts, int n_edges, const long long* off, long long N,
                              uint8_t* point_flags, uint8_t* edge_flags, int T, int grid_cap, cudaStream_t s) {
  if (n_rbox || env.n_box) return launch_check_path_box(robot, n, nsp_pad, n_rbox, env, E, verts, n_edges, off, N, point_flags, edge_flags, T, grid_cap, s);
  if (N <= 0 || n_edges <= 0) return cudaSuccess;
  cudaError_t err = cudaSuccess;
  const int threads = 128;
  const size_t smem = check_smem_layout(nsp_pad, env.n_obs_pad, threads, T, n_rbox, env.n_box);
  const long long groups = threads / T;
  long long grid = (N + groups - 1) / groups;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  constexpr bool BB = EZO_BOX_TU != 0;
  EZO_DISPATCH_NDOF(n, EZO_DISPATCH_T(T, {
    auto kern = k_check_path<ND, TT, BB>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(robot, env, E, verts, n_edges, off, N, point_flags, edge_flags);
  }));
  return cudaGetLastError();
}
#endif

#if !EZO_BOX_TU

// One block per (segment k, polytope j of the same path): covered[k] = 1 when
// polytope j exists (its segment was accepted or ran N_it rounds) and holds
// both endpoints of segment k.
__global__ void k_coverage(BatchView v, uint8_t* covered, double tol) {
  const int k = blockIdx.x;
  const int j = v.path_first[k] + (int)blockIdx.y;
  if (j >= v.B || v.path_first[j] != v.path_first[k]) return;
  const SegState& sj = v.st[j];
  if (sj.status != SEG_ACCEPTED && sj.status != SEG_MAX_ITER) return;
  const int n = v.n;
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
  if (threadIdx.x == 0 && !s_out) covered[k] = 1;
}

cudaError_t launch_coverage(const BatchView& v, uint8_t* covered, double tol, cudaStream_t s) {
  dim3 grid(v.B, v.max_path_len);
  k_coverage<<<grid, 128, 0, s>>>(v, covered, tol);
  return cudaGetLastError();
}

#endif  // !EZO_BOX_TU

}  // namespace ezo
