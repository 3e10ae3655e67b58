// Single-segment inflation that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need a
// region: a real-time control loop that must not block in cudaMalloc (it may
// synchronise the device and has no latency bound), or a host application
// that hands the library a fixed memory budget at start-up and forbids later
// device allocations. For them, ezo_inflate_segment_noalloc runs the same
// round kernels as ezo_batch_run on one segment, with every working buffer
// (segment state, polytope, samples, labels, candidates, work lists, round
// summary) carved out of the file-scope array below instead of cudaMalloc'd
// memory. The robot and obstacle handles are created beforehand, outside the
// constrained section.
//
// The array holds EZO_NOALLOC_SCRATCH_BYTES on every GPU that loads the
// library, until the process exits. Every call shares it and it keeps the
// last call's contents; each call re-initialises what it reads before writing
// it. Calls whose work overlaps on the GPU (other streams, other host threads)
// race on the array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ezo.h"
#include "ezo_engine.cuh"

using namespace ezo;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[EZO_NOALLOC_SCRATCH_BYTES];

std::mutex g_addr_mu;
void* g_addr[64] = {nullptr};

}  // namespace

extern "C" void ezo_internal_set_error(const char* msg);

namespace {

ezo_status na_fail(ezo_status s, const std::string& msg) {
  ezo_internal_set_error(("ezo_inflate_segment_noalloc: " + msg).c_str());
  return s;
}

// Device address of the scratch array on the current device, looked up once
// per device (host code sees only a host-side stand-in under the array's name).
ezo_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(EZO_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return na_fail(EZO_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(EZO_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return EZO_OK;
}

struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += std::max<size_t>(1, count) * sizeof(T);
    return p;
  }
};

int na_test_size(int k, double eps, double delta, double tau) {
  const double dk = 6.0 * delta / (M_PI * M_PI * k * (double)k);
  return (int)std::ceil(2.0 * std::log(1.0 / dk) / (eps * tau * tau));
}

// Lanes per configuration of the label and bisection kernels: the rule of
// ezo_batch_create for rounds of this size (two lanes per configuration below
// 2^20 samples, sixteen per bisection candidate below 2^20 candidates, eight
// with boxes; labels do not depend on the choice); above that, the size rule
// of the collision checker, since the tuner would allocate.
int lanes_for(long long N) {
  if (N >= (1ll << 20)) return 1;
  if (N >= (1ll << 17)) return 2;
  if (N >= (1ll << 15)) return 4;
  return 8;
}
int check_lanes(long long s_cap) { return s_cap < (1ll << 20) ? 2 : lanes_for(s_cap); }
int bisect_lanes(long long np, bool boxes) { return np >= (1ll << 20) ? lanes_for(np / 4) : (boxes ? 8 : 16); }

}  // namespace

// The robot and env handles are defined in ezo_capi.cu; these accessors give
// this file the device images it needs without touching that code path.
extern "C" int ezo_internal_robot_boxes(const ezo_robot* r);
extern "C" const ezo::RobotDev* ezo_internal_robot_dev(const ezo_robot* r, int* n, int* nsp_pad, double* q_lo,
                                                       double* q_hi);
extern "C" int ezo_internal_env_dev(const ezo_robot* r, const ezo_env* e, ezo::EnvDevFull* out);

extern "C" ezo_status ezo_inflate_segment_noalloc(const ezo_robot* robot, const ezo_env* env, const double* v1,
                                                  const double* v2, const ezo_params* prm, uint32_t stream_id,
                                                  double* A_out, double* b_out, int32_t* m_out, int32_t* status_out,
                                                  int32_t* rounds_out, int64_t* checks_out, void* cuda_stream) {
  if (!robot || !env || !v1 || !v2 || !prm || !A_out || !b_out || !m_out)
    return na_fail(EZO_ERR_INVALID_ARG, "null argument");
  if (!(prm->eps > 0.0 && prm->eps < 1.0) || !(prm->delta > 0.0 && prm->delta < 1.0) ||
      !(prm->tau > 0.0 && prm->tau < 1.0) || !(prm->step_back_max >= 0.0) || !(prm->t_col >= 0.0) ||
      prm->n_p < 1 || prm->n_f < 1 || prm->n_b < 0 || prm->n_b > 32 || prm->n_mix < 0 || prm->n_it_max < 1)
    return na_fail(EZO_ERR_INVALID_ARG, "parameter out of range");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int n = 0, nsp_pad = 0;
  double q_lo[EZO_MAX_DOF], q_hi[EZO_MAX_DOF];
  const RobotDev* rdev = ezo_internal_robot_dev(robot, &n, &nsp_pad, q_lo, q_hi);
  EnvDevFull envf{};
  if (!rdev || ezo_internal_env_dev(robot, env, &envf) != 0) return na_fail(EZO_ERR_INVALID_ARG, "bad handle");

  // sizes, checked against the fixed scratch capacity before anything runs
  const int m0 = 2 * n;
  const long long m_cap = m0 + (long long)prm->n_f * prm->n_it_max;
  if (m_cap > 2048) return na_fail(EZO_ERR_CAPACITY, "2n + n_f * n_it_max must be <= 2048 rows");
  const int np = prm->n_p;
  const long long s_cap = std::max<long long>(np, na_test_size(prm->n_it_max, prm->eps, prm->delta, prm->tau) + 16);
  const long long st_tiles = (s_cap + kTile - 1) / kTile, bi_tiles = (np + kTile - 1) / kTile;
  const size_t pad = 256;
  const int s_ld = n <= 8 ? 8 : EZO_MAX_DOF;
  const size_t rows_b = (size_t)bi_tiles * kTile;
  const size_t need = 2 * rows_b * s_ld * sizeof(float) + kSeatSlots * sizeof(int) +
                      (std::max<size_t>((size_t)st_tiles * 8, (size_t)bi_tiles * 32) + 1) * sizeof(int) + sizeof(SegState) + 2 * n * sizeof(double) + m_cap * n * sizeof(double) +
                      m_cap * sizeof(double) + s_cap * n * sizeof(float) + s_cap + (size_t)np * sizeof(int) +
                      (size_t)np * n * (2 * sizeof(double) + sizeof(float)) + (size_t)np * (2 * sizeof(double) + 8) +
                      (size_t)prm->n_f * (sizeof(int) + sizeof(double)) + (st_tiles + bi_tiles) * sizeof(int2) +
                      sizeof(RoundSummary) + sizeof(EnvDevFull) + sizeof(int) + 28 * pad;
  if (need > (size_t)EZO_NOALLOC_SCRATCH_BYTES)
    return na_fail(EZO_ERR_CAPACITY, "this segment needs " + std::to_string(need) +
                                         " bytes of working memory, more than the fixed " +
                                         std::to_string((long long)EZO_NOALLOC_SCRATCH_BYTES) +
                                         " (lower n_p or n_f * n_it_max, or use ezo_batch_create)");
  // the collision kernels stage the robot spheres, the obstacles and one set
  // of sphere centres per group of lanes in shared memory: large robots with
  // many obstacles need more lanes per configuration
  int t_min = 1;
  while (t_min <= 8 && check_smem_bytes(nsp_pad, envf.e.n_obs_pad, 128, t_min, ezo_internal_robot_boxes(robot),
                                        envf.e.n_box) > kSmemBudget)
    t_min *= 2;
  if (t_min > 8) return na_fail(EZO_ERR_INVALID_ARG, "robot spheres and obstacles exceed shared memory at 8 lanes");
  void* base = nullptr;
  ezo_status st = scratch_address(&base);
  if (st != EZO_OK) return st;

  Carver c{static_cast<unsigned char*>(base)};
  BatchView v{};
  SegState* d_st = c.take<SegState>(1);
  double* d_v1 = c.take<double>(n);
  double* d_v2 = c.take<double>(n);
  double* d_A = c.take<double>(m_cap * n);
  double* d_b = c.take<double>(m_cap);
  float* d_S = c.take<float>(s_cap * n);
  uint8_t* d_flags = c.take<uint8_t>(s_cap);
  int* d_cidx = c.take<int>(np);
  double* d_cstar = c.take<double>((size_t)np * n);
  double* d_dist = c.take<double>(np);
  float* d_c32 = c.take<float>((size_t)np * n);
  float* d_cn = c.take<float>(np);
  uint32_t* d_bits = c.take<uint32_t>(np);
  double* d_ga = c.take<double>((size_t)np * n);
  double* d_gb = c.take<double>(np);
  int* d_pidx = c.take<int>(prm->n_f);
  double* d_pdelta = c.take<double>(prm->n_f);
  int2* d_stiles = c.take<int2>(st_tiles);
  int2* d_btiles = c.take<int2>(bi_tiles);
  RoundSummary* d_sum = c.take<RoundSummary>(1);
  EnvDevFull* d_env = c.take<EnvDevFull>(1);
  int* d_pf = c.take<int>(1);
  float* d_sp = c.take<float>(rows_b * s_ld);
  float* d_sd = c.take<float>(rows_b * s_ld);
  int* d_seats = c.take<int>(kSeatSlots);
  const size_t claim_cap = std::max<size_t>((size_t)st_tiles * 8, (size_t)bi_tiles * 32);
  int* d_claim = c.take<int>(claim_cap + 1);
  if (c.off > (size_t)EZO_NOALLOC_SCRATCH_BYTES) return na_fail(EZO_ERR_CAPACITY, "scratch layout overflow");

  // initial contents: everything a kernel reads before writing it
  SegState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.k = 1;
  s0.status = SEG_ACTIVE;
  s0.m = m0;
  s0.n_p = np;
  s0.env = 0;
  s0.stream = stream_id;
  s0.box_rows = 2 * n;  // the domain built below is the joint box
  s0.s_cap = (int)s_cap;
  std::vector<double> A0((size_t)m0 * n, 0.0), b0(m0, 0.0);
  for (int j = 0; j < n; ++j) {
    A0[(size_t)j * n + j] = 1.0;
    b0[j] = q_hi[j];
    A0[(size_t)(n + j) * n + j] = -1.0;
    b0[n + j] = -q_lo[j];
  }
  const int zero = 0;
  RoundSummary sum0{};
  cudaError_t e = cudaSuccess;
  // On a failure after work was queued, the stream is drained before the
  // error returns, so the shared array is idle when the call returns.
#define NA_CUDA(call)                                                              \
  do {                                                                             \
    e = (call);                                                                    \
    if (e != cudaSuccess) {                                                        \
      (void)cudaStreamSynchronize(s);                                              \
      return na_fail(EZO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e)); \
    }                                                                              \
  } while (0)
  NA_CUDA(cudaMemcpyAsync(d_st, &s0, sizeof(s0), cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_v1, v1, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_v2, v2, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_A, A0.data(), sizeof(double) * A0.size(), cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_b, b0.data(), sizeof(double) * b0.size(), cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_sum, &sum0, sizeof(sum0), cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_env, &envf, sizeof(envf), cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_pf, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemsetAsync(d_flags, 0, (size_t)s_cap, s));
  NA_CUDA(cudaMemsetAsync(d_seats, 0, sizeof(int) * kSeatSlots, s));
  NA_CUDA(cudaMemsetAsync(d_claim, 0, sizeof(int) * (claim_cap + 1), s));

  v.B = 1;
  v.n = n;
  v.m_cap = (int)m_cap;
  v.n_f = prm->n_f;
  v.n_b = prm->n_b;
  v.n_mix = prm->n_mix;
  v.n_it_max = prm->n_it_max;
  v.eps = prm->eps;
  v.delta = prm->delta;
  v.tau = prm->tau;
  v.step_back_max = prm->step_back_max;
  v.t_col = prm->t_col;
  v.key0 = (uint32_t)(prm->seed & 0xffffffffu);
  v.key1 = (uint32_t)(prm->seed >> 32);
  v.keys = philox_keys(prm->seed);
  v.st = d_st;
  v.v1 = d_v1;
  v.v2 = d_v2;
  v.A = d_A;
  v.b = d_b;
  v.S = d_S;
  v.flags = d_flags;
  v.cand_idx = d_cidx;
  v.cstar = d_cstar;
  v.dist = d_dist;
  v.c32 = d_c32;
  v.cnorm = d_cn;
  v.bits = d_bits;
  v.ga = d_ga;
  v.gb = d_gb;
  v.placed_idx = d_pidx;
  v.placed_delta = d_pdelta;
  v.sample_tiles = d_stiles;
  v.bisect_tiles = d_btiles;
  v.summary = d_sum;
  v.robot = rdev;
  v.envs = d_env;
  v.max_obs_pad = envf.e.n_obs_pad;
  v.max_ebox = envf.e.n_box;
  v.n_rbox = ezo_internal_robot_boxes(robot);
  v.nsp_pad = nsp_pad;
  v.np_max = np;
  v.path_first = d_pf;
  v.max_path_len = 1;
  v.graph_cond = 0;
  v.s_p32 = d_sp;
  v.s_d32 = d_sd;
  v.s_ld = s_ld;
  v.sm_seats = d_seats;
  v.q_claim = d_claim;
  v.q_claim_cap = (int)claim_cap;

  int dev = 0, sms = 1;
  NA_CUDA(cudaGetDevice(&dev));
  NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  v.n_sm = sms;
  const int T_check = std::max(check_lanes(s_cap), t_min);
  const int T_bis = std::max(bisect_lanes(np, ezo_internal_robot_boxes(robot) || envf.e.n_box), t_min);
  const int grid_s = (int)std::max<long long>(1, std::min<long long>(st_tiles * 8, (long long)sms * 16));
  const int grid_c = (int)std::max<long long>(1, std::min<long long>(st_tiles * T_check, (long long)sms * 16));
  const int grid_b = (int)std::max<long long>(1, std::min<long long>(bi_tiles * T_bis, (long long)sms * 16));
  const int grid_r = row_grid((long long)rows_b);
  RoundSummary h{};
  for (int r = 0; r <= prm->n_it_max + 1; ++r) {
    NA_CUDA(launch_round_begin(v, s));
    NA_CUDA(launch_round_sample(v, (sms * 4 * 32) / kTile, grid_s, s));
    NA_CUDA(launch_round_check(v, T_check, grid_c, s));
    NA_CUDA(launch_round_certify(v, s));
    NA_CUDA(launch_bisect_exact(v, T_bis, grid_b, grid_r, s));
    NA_CUDA(launch_round_place(v, s));
    NA_CUDA(launch_round_end(v, s));
    NA_CUDA(cudaMemcpyAsync(&h, d_sum, sizeof(h), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (h.active == 0) break;
  }
  SegState out;
  NA_CUDA(cudaMemcpyAsync(&out, d_st, sizeof(out), cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaStreamSynchronize(s));
  NA_CUDA(cudaMemcpyAsync(A_out, d_A, sizeof(double) * (size_t)out.m * n, cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaMemcpyAsync(b_out, d_b, sizeof(double) * (size_t)out.m, cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaStreamSynchronize(s));
#undef NA_CUDA
  *m_out = out.m;
  if (status_out) *status_out = out.status;
  if (rounds_out) *rounds_out = out.rounds;
  if (checks_out) *checks_out = out.checks;
  ezo_internal_set_error("");
  return EZO_OK;
}
