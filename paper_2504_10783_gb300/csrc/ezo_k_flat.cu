// EI-ZO kernels on caller buffers (arXiv 2504.10783):
//   k_sample_flat - hit-and-run walks inside {A x <= b} (Sec. IV-B, IV-D)
//   k_check_flat  - forward kinematics + sphere collision labels (Sec. IV-D)
//   k_sd_flat     - signed distance over the same pairs (labels for data)
#include "ezo_kernels_common.cuh"

#ifndef EZO_BOX_TU
#define EZO_BOX_TU 0  // 1: this translation unit holds only the box-geometry collision kernels
#endif

namespace ezo {

#if !EZO_BOX_TU

template <int NDOF>
__global__ void __launch_bounds__(128) k_sample_flat(const double* __restrict__ A, const double* __restrict__ b,
                                                     int m, int lda, int n, SampleParams p,
                                                     float* __restrict__ out, long long ldo, long long N) {
  extern __shared__ float4 smf4[];
  float* A32 = reinterpret_cast<float*>(smf4);
  stage_polytope<NDOF>(A32, A, b, m, lda, n);
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    float x[NDOF];
    hnr_walk<NDOF>(A32, m, n, p.v1f, p.ef, p.n_mix, p.key0, p.key1, (uint32_t)i, p.round_k, p.stream, x);
#pragma unroll
    for (int j = 0; j < NDOF; ++j)
      if (j < n) out[(long long)j * ldo + i] = x[j];
  }
}

#endif  // !EZO_BOX_TU

template <int NDOF, int T, bool BOX>
__global__ void __launch_bounds__(128) k_check_flat(const RobotDev* __restrict__ robot, EnvDev env, float E,
                                                    const float* __restrict__ q, long long ldq, long long N,
                                                    uint8_t* __restrict__ flags) {
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
  const ushort2* sp = robot->self_pairs;
  const float* srr = robot->self_rr;
  for (long long base = (long long)blockIdx.x * groups; base < N; base += (long long)gridDim.x * groups) {
    const long long i = base + gi;
    const long long ic = i < N ? i : N - 1;
    float qq[NDOF];
#pragma unroll
    for (int j = 0; j < NDOF; ++j) qq[j] = (j < rs.n) ? q[j * ldq + ic] : 0.f;
    const bool hit =
        collide_group<NDOF, T, BOX>(qq, rs, sph_s, obs_s, nhw_s, env.n_obs, env.n_obs_pad, sp, srr, E, cen, lg, bx);
    if (i < N && lg == 0) flags[i] = hit ? 1 : 0;
  }
}

#if !EZO_BOX_TU

template <int NDOF>
__global__ void __launch_bounds__(128) k_sd_flat(const RobotDev* __restrict__ robot, EnvDev env,
                                                 const float* __restrict__ q, long long ldq, long long N,
                                                 float* __restrict__ sd, float cap) {
  extern __shared__ float4 smem4[];
  __shared__ RobotSmem rs;
  const int nsp = robot->n_spheres_pad;
  float4* sph_s = smem4;
  float4* obs_s = sph_s + nsp;
  float4* cen_all = obs_s + env.n_obs_pad;
  float* nhw_s = reinterpret_cast<float*>(cen_all + blockDim.x * (nsp + 1));
  stage_robot(rs, sph_s, robot);
  stage_env(obs_s, nhw_s, env);
  __syncthreads();
  float4* cen = cen_all + threadIdx.x * (nsp + 1);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    float qq[NDOF];
#pragma unroll
    for (int j = 0; j < NDOF; ++j) qq[j] = (j < rs.n) ? q[j * ldq + i] : 0.f;
    sd[i] = signed_distance_one<NDOF>(qq, rs, sph_s, obs_s, env.n_obs, robot->self_pairs, robot->self_rr, cen, cap);
  }
}

size_t check_smem_bytes(int n_spheres_pad, int n_obs_pad, int threads, int T, int n_rbox, int n_ebox) {
  return check_smem_layout(n_spheres_pad, n_obs_pad, threads, T, n_rbox, n_ebox);
}

#endif  // !EZO_BOX_TU

#if EZO_BOX_TU
cudaError_t launch_check_flat_box(const RobotDev* robot, int n, int nsp_pad, int n_rbox, const EnvDev& env, float E,
                              const float* q, long long ldq, long long N, uint8_t* flags, int T, int grid_cap,
                              cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  cudaError_t err = cudaSuccess;
  const int threads = 128;
  const size_t smem = check_smem_layout(nsp_pad, env.n_obs_pad, threads, T, n_rbox, env.n_box);
  const long long groups = threads / T;
  long long grid = (N + groups - 1) / groups;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  constexpr bool BB = EZO_BOX_TU != 0;
  EZO_DISPATCH_NDOF(n, EZO_DISPATCH_T(T, {
    auto kern = k_check_flat<ND, TT, BB>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(robot, env, E, q, ldq, N, flags);
  }));
  return cudaGetLastError();
}
#else
cudaError_t launch_check_flat(const RobotDev* robot, int n, int nsp_pad, int n_rbox, const EnvDev& env, float E,
                              const float* q, long long ldq, long long N, uint8_t* flags, int T, int grid_cap,
                              cudaStream_t s) {
  if (n_rbox || env.n_box) return launch_check_flat_box(robot, n, nsp_pad, n_rbox, env, E, q, ldq, N, flags, T, grid_cap, s);
  if (N <= 0) return cudaSuccess;
  cudaError_t err = cudaSuccess;
  const int threads = 128;
  const size_t smem = check_smem_layout(nsp_pad, env.n_obs_pad, threads, T, n_rbox, env.n_box);
  const long long groups = threads / T;
  long long grid = (N + groups - 1) / groups;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  constexpr bool BB = EZO_BOX_TU != 0;
  EZO_DISPATCH_NDOF(n, EZO_DISPATCH_T(T, {
    auto kern = k_check_flat<ND, TT, BB>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(robot, env, E, q, ldq, N, flags);
  }));
  return cudaGetLastError();
}
#endif

#if !EZO_BOX_TU


cudaError_t launch_sd_flat(const RobotDev* robot, int n, int nsp_pad, const EnvDev& env, const float* q, long long ldq,
                           long long N, float* sd, cudaStream_t s, float cap) {
  if (N <= 0) return cudaSuccess;
  cudaError_t err = cudaSuccess;
  const int threads = 64;
  const size_t smem = check_smem_layout(nsp_pad, env.n_obs_pad, threads, 1);
  const long long grid = (N + threads - 1) / threads;
  EZO_DISPATCH_NDOF(n, {
    auto kern = k_sd_flat<ND>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(robot, env, q, ldq, N, sd, cap);
  });
  return cudaGetLastError();
}


cudaError_t launch_sample_flat(const double* A, const double* b, int m, int lda, int n, const double* v1h,
                               const double* v2h, long long N, int n_mix, uint64_t seed, uint32_t stream, int k,
                               float* out, long long ldo, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  SampleParams p{};
  for (int j = 0; j < n; ++j) {
    p.v1f[j] = (float)v1h[j];
    p.ef[j] = (float)(v2h[j] - v1h[j]);
  }
  p.n_mix = n_mix;
  p.key0 = (uint32_t)(seed & 0xffffffffu);
  p.key1 = (uint32_t)(seed >> 32);
  p.stream = stream;
  p.round_k = (uint32_t)k;
  const int threads = 128;
  const long long grid = (N + threads - 1) / threads;
  cudaError_t err = cudaSuccess;
  EZO_DISPATCH_NDOF(n, {
    const size_t smem = (size_t)std::max(1, m) * hnr_row_stride<ND>() * sizeof(float);
    auto kern = k_sample_flat<ND>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(A, b, m, lda, n, p, out, ldo, N);
  });
  return cudaGetLastError();
}


#endif  // !EZO_BOX_TU

}  // namespace ezo
