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
    hnr_walk<NDOF>(A32, m, n, p.v1f, p.ef, p.n_mix, p.keys, (uint32_t)i, p.round_k, p.stream, x);
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
        collide_group<NDOF, T, BOX>(qq, rs, sph_s, obs_s, nhw_s, env.n_obs, env.n_obs_pad, env.s_first, sp, srr, E, cen,
                                    lg, bx);
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

// Forward kinematics of N configurations (one thread each): the FP32 sphere
// centres exactly as the collision kernels compute them (fk_group), and the
// centres of the same chain in FP64 from the FP64 constants, the joint
// values widened from FP32. mode 0 writes the FP32 centres and mode 1 the
// FP64 centres to out_c[(3 s + c) * N + i] (s sorted by frame, as RobotDev
// keeps them); mode 2 writes err[i] = max_s |c32_s - c64_s| in metres.
template <int NDOF>
__global__ void __launch_bounds__(64) k_fk_centres(const RobotDev* __restrict__ robot,
                                                   const RobotFK64* __restrict__ r64, const float* __restrict__ q,
                                                   long long ldq, long long N, int mode, double* __restrict__ out_c,
                                                   float* __restrict__ err) {
  extern __shared__ float4 smem4[];
  __shared__ RobotSmem rs;
  const int nsp = robot->n_spheres_pad;
  float4* sph_s = smem4;
  float4* cen = smem4 + nsp + threadIdx.x * (nsp + 1);
  stage_robot(rs, sph_s, robot);
  __syncthreads();
  const BoxCtx nobox{};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    float qq[NDOF];
#pragma unroll
    for (int j = 0; j < NDOF; ++j) qq[j] = (j < rs.n) ? q[j * ldq + i] : 0.f;
    fk_group<NDOF, 1, false>(qq, rs, sph_s, cen, 0, nobox);
    if (mode == 0) {
      for (int s = 0; s < rs.n_spheres; ++s) {
        out_c[(3ll * s) * N + i] = cen[s].x;
        out_c[(3ll * s + 1) * N + i] = cen[s].y;
        out_c[(3ll * s + 2) * N + i] = cen[s].z;
      }
      continue;
    }
    // FP64 chain: T_j = T_{j-1} Rz(kth q + toff) Tz(d + kd q) Tx(a) Rx(alpha)
    double c0x = 1.0, c0y = 0.0, c0z = 0.0, c1x = 0.0, c1y = 1.0, c1z = 0.0, c2x = 0.0, c2y = 0.0, c2z = 1.0;
    double px = 0.0, py = 0.0, pz = 0.0;
    double worst = 0.0;
    for (int f = 0; f <= r64->n; ++f) {
      if (f > 0) {
        const int j = f - 1;
        const double qj = (double)qq[j < NDOF ? j : 0];
        double sn, cs;
        sincos(fma(qj, r64->kth[j], r64->toff[j]), &sn, &cs);
        const double n0x = cs * c0x + sn * c1x, n0y = cs * c0y + sn * c1y, n0z = cs * c0z + sn * c1z;
        const double n1x = cs * c1x - sn * c0x, n1y = cs * c1y - sn * c0y, n1z = cs * c1z - sn * c0z;
        const double aj = r64->a[j], dj = r64->d[j] + r64->kd[j] * qj;
        px += aj * n0x + dj * c2x;
        py += aj * n0y + dj * c2y;
        pz += aj * n0z + dj * c2z;
        const double ca = r64->ca[j], sa = r64->sa[j];
        const double m1x = ca * n1x + sa * c2x, m1y = ca * n1y + sa * c2y, m1z = ca * n1z + sa * c2z;
        const double m2x = ca * c2x - sa * n1x, m2y = ca * c2y - sa * n1y, m2z = ca * c2z - sa * n1z;
        c0x = n0x; c0y = n0y; c0z = n0z;
        c1x = m1x; c1y = m1y; c1z = m1z;
        c2x = m2x; c2y = m2y; c2z = m2z;
      }
      for (int s = r64->frame_first[f]; s < r64->frame_first[f + 1]; ++s) {
        const double lx = r64->sx[s], ly = r64->sy[s], lz = r64->sz[s];
        const double x = c0x * lx + c1x * ly + c2x * lz + px;
        const double y = c0y * lx + c1y * ly + c2y * lz + py;
        const double z = c0z * lx + c1z * ly + c2z * lz + pz;
        if (mode == 1) {
          out_c[(3ll * s) * N + i] = x;
          out_c[(3ll * s + 1) * N + i] = y;
          out_c[(3ll * s + 2) * N + i] = z;
        } else {
          const double dx = (double)cen[s].x - x, dy = (double)cen[s].y - y, dz = (double)cen[s].z - z;
          worst = fmax(worst, sqrt(dx * dx + dy * dy + dz * dz));
        }
      }
    }
    if (mode == 2) err[i] = (float)worst;
  }
}

cudaError_t launch_fk_centres(const RobotDev* robot, const RobotFK64* r64, int n, int nsp_pad, const float* q,
                              long long ldq, long long N, int mode, double* out_c, float* err, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  // one slot of sphere centres per thread; 32 threads for the largest robots
  const int threads = (size_t)64 * (nsp_pad + 1) * sizeof(float4) <= 160 * 1024 ? 64 : 32;
  const size_t smem = (size_t)(nsp_pad + threads * (nsp_pad + 1)) * sizeof(float4);
  const long long grid = std::min<long long>((N + threads - 1) / threads, 1ll << 20);
  EZO_DISPATCH_NDOF(n, {
    auto kern = k_fk_centres<ND>;
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, threads, smem, s>>>(robot, r64, q, ldq, N, mode, out_c, err);
  });
  return cudaGetLastError();
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
  p.keys = philox_keys(seed);
  p.stream = stream;
  p.round_k = (uint32_t)k;
  const int threads = 128;
  const long long grid = (N + threads - 1) / threads;
  cudaError_t err = cudaSuccess;
  EZO_DISPATCH_NDOF(n, {
    const size_t smem = hnr_smem_bytes<ND>(m);
    auto kern = k_sample_flat<ND>;
    err = set_smem(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(A, b, m, lda, n, p, out, ldo, N);
  });
  return cudaGetLastError();
}


#endif  // !EZO_BOX_TU

}  // namespace ezo
