// Autotuner for the launch shape of the collision kernels: how many lanes of
// a warp cooperate on one configuration (1, 2, 4 or 8). Fewer lanes do less
// redundant forward kinematics; more lanes give more warps per SM when the
// batch is small and the per-configuration shared memory limits occupancy.
// The tuner times the flat collision kernel on uniform configurations of the
// robot's joint box at the requested batch size, picks the fastest, and
// caches it per (robot shape, obstacle count, batch size class) for the
// process lifetime.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "../../include/ezo.h"
#include "ezo_engine.cuh"

using namespace ezo;

extern "C" const ezo::RobotDev* ezo_internal_robot_dev(const ezo_robot* r, int* n, int* nsp_pad, double* q_lo,
                                                       double* q_hi);
extern "C" int ezo_internal_env_dev(const ezo_robot* r, const ezo_env* e, ezo::EnvDevFull* out);
extern "C" void ezo_internal_set_error(const char* msg);
extern "C" int ezo_internal_robot_boxes(const ezo_robot* r);

namespace {

// configuration i, coordinate j: lo_j + (hi_j - lo_j) u, u from Philox (i, j)
__global__ void k_uniform_configs(float* q, long long N, int n, const float* lo, const float* hi) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    for (int j = 0; j < n; ++j) {
      const u32x4 r = philox4x32_10(u32x4{(uint32_t)i, (uint32_t)j, 0x7475u, 0x6e65u}, 0x1234u, 0x5678u);
      q[(long long)j * N + i] = lo[j] + (hi[j] - lo[j]) * u01_co(r.x);
    }
  }
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int, int>, int> g_tune_cache;
bool g_autotune = true;

int size_class(long long N) {
  int c = 0;
  while ((1ll << c) < N && c < 40) ++c;
  return c;
}

}  // namespace

// Used by ezo_capi.cu; returns the tuned lane count (or a size rule when the
// tuner is off or fails).
extern "C" __attribute__((visibility("hidden"))) int ezo_internal_tuned_lanes(const ezo_robot* robot, const ezo_env* env,
                                                                    long long N, cudaStream_t s) {
  auto rule = [&](long long M) {
    if (M >= (1ll << 20)) return 1;
    if (M >= (1ll << 17)) return 2;
    if (M >= (1ll << 15)) return 4;
    return 8;
  };
  int n = 0, nsp = 0;
  double lo[EZO_MAX_DOF], hi[EZO_MAX_DOF];
  const RobotDev* rd = ezo_internal_robot_dev(robot, &n, &nsp, lo, hi);
  EnvDevFull ef{};
  if (!rd || ezo_internal_env_dev(robot, env, &ef) != 0) return rule(N);
  const int nrbox = ezo_internal_robot_boxes(robot);
  // only lane counts whose sphere centres fit in shared memory (more lanes,
  // fewer groups per block, less memory); 8 when none does, which the entry
  // points reject before launching
  auto fits = [&](int T) {
    return check_smem_bytes(nsp, ef.e.n_obs_pad, 128, T, nrbox, ef.e.n_box) <= kSmemBudget;
  };
  auto fit_up = [&](int T) {
    while (T < 8 && !fits(T)) T *= 2;
    return T;
  };
  if (!g_autotune || N <= 0) return fit_up(rule(N));
  RobotDev head;
  if (cudaMemcpy(&head, rd, sizeof(int) * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return fit_up(rule(N));
  int dev = 0;
  cudaGetDevice(&dev);
  const int cls = size_class(N);
  const auto key = std::make_tuple(dev, n, nsp, head.n_self, ef.e.n_obs_pad, cls, nrbox, ef.e.n_box);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
  }
  const long long M = 1ll << std::min(cls, 22);
  float* q = nullptr;
  uint8_t* flags = nullptr;
  float* bounds = nullptr;
  int best = fit_up(rule(N));
  if (cudaMalloc(&q, sizeof(float) * n * M) == cudaSuccess && cudaMalloc(&flags, M) == cudaSuccess &&
      cudaMalloc(&bounds, sizeof(float) * 2 * EZO_MAX_DOF) == cudaSuccess) {
    float hb[2 * EZO_MAX_DOF];
    for (int j = 0; j < n; ++j) {
      hb[j] = (float)lo[j];
      hb[EZO_MAX_DOF + j] = (float)hi[j];
    }
    cudaMemcpyAsync(bounds, hb, sizeof(hb), cudaMemcpyHostToDevice, s);
    k_uniform_configs<<<(unsigned)std::min<long long>((M + 255) / 256, 4096), 256, 0, s>>>(q, M, n, bounds,
                                                                                          bounds + EZO_MAX_DOF);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float best_ms = 1e30f;
    const int lanes[4] = {1, 2, 4, 8};
    for (int li = 0; li < 4; ++li) {
      const int T = lanes[li];
      if (!fits(T)) continue;
      // one warm-up launch, then the best of three
      if (launch_check_flat(rd, n, nsp, nrbox, ef.e, ef.E, q, M, M, flags, T, sms * 32, s) != cudaSuccess) continue;
      float t_best = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        launch_check_flat(rd, n, nsp, nrbox, ef.e, ef.E, q, M, M, flags, T, sms * 32, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t_best = std::min(t_best, ms);
      }
      if (t_best < best_ms) {
        best_ms = t_best;
        best = T;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaStreamSynchronize(s);
  cudaFree(q);
  cudaFree(flags);
  cudaFree(bounds);
  cudaGetLastError();
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best;
  return best;
}

extern "C" ezo_status ezo_set_autotune(int32_t on) {
  g_autotune = on != 0;
  return EZO_OK;
}

extern "C" ezo_status ezo_tune_lanes(const ezo_robot* robot, const ezo_env* env, int64_t N, int32_t* lanes,
                                     void* cuda_stream) {
  if (!robot || !env || N < 1 || !lanes) {
    ezo_internal_set_error("ezo_tune_lanes: bad argument");
    return EZO_ERR_INVALID_ARG;
  }
  const bool was = g_autotune;
  g_autotune = true;
  *lanes = ezo_internal_tuned_lanes(robot, env, N, (cudaStream_t)cuda_stream);
  g_autotune = was;
  ezo_internal_set_error("");
  return EZO_OK;
}

// ---- FP32 FMA calibration: independent FMA chains on every SM ----
namespace {

constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(256) k_fma_probe(float* out, int reps, float a, float c) {
  float x[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) x[i] = threadIdx.x * 1e-3f + (float)i;
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) x[i] = fmaf(x[i], a, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += x[i];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" ezo_status ezo_probe_fp32_fma(double* tflops, void* cuda_stream) {
  if (!tflops) {
    ezo_internal_set_error("ezo_probe_fp32_fma: tflops is NULL");
    return EZO_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // 8 blocks of 256 threads per SM: every warp slot filled
  const int blocks = sms * 8, threads = 256, reps = 20000;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads) != cudaSuccess) {
    cudaGetLastError();
    ezo_internal_set_error("ezo_probe_fp32_fma: cudaMalloc failed");
    return EZO_ERR_CUDA;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  k_fma_probe<<<blocks, threads, 0, s>>>(out, reps, 0.999f, 1e-3f);  // warm-up
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_probe<<<blocks, threads, 0, s>>>(out, reps, 0.999f, 1e-3f);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) {
    ezo_internal_set_error(cudaGetErrorString(err));
    return EZO_ERR_CUDA;
  }
  const double flops = 2.0 * kProbeChains * (double)reps * blocks * threads;
  *tflops = flops / (best * 1e-3) * 1e-12;
  ezo_internal_set_error("");
  return EZO_OK;
}
