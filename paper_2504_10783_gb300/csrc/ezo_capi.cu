// Host side of libezo.so: handles, device memory, the round driver (host
// loop or one CUDA graph with a conditional WHILE node), path inflation with
// the containment skip (Sec. VI-A) and the C ABI declared in include/ezo.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <utility>
#include <string>
#include <vector>

#include "../../include/ezo.h"
#include "ezo_engine.cuh"

using namespace ezo;

namespace {

thread_local std::string g_err;

ezo_status fail(ezo_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

ezo_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  (void)cudaGetLastError();  // the runtime's record of a non-sticky error, which the caller's next check would see
  return EZO_ERR_CUDA;
}

#define EZO_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr double kU32 = 5.9604644775390625e-8;  // 2^-24

int round_up(int x, int m) { return (x + m - 1) / m * m; }

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

// ------------------------------------------------------------- profiling --
constexpr int kKinds = 7;
bool g_prof_on = false;
double g_prof_ms[kKinds] = {0};
long long g_prof_n[kKinds] = {0};

struct EventPool {
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  size_t used = 0;
  cudaEvent_t get() {
    if (used == ev.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
    }
    return ev[used++];
  }
};

}  // namespace

struct ezo_robot {
  RobotDev host{};
  RobotDev* d_robot = nullptr;
  RobotFK64* d_fk64 = nullptr;  // FP64 chain for the kinematics error
  ushort2* d_pairs = nullptr;
  float* d_rr = nullptr;
  ushort2 *d_sbp = nullptr, *d_bbp = nullptr;  // self pairs with a box
  std::vector<int> sphere_sorted;              // caller's sphere index -> sorted index
  int n = 0, n_spheres = 0, nsp_pad = 0, n_self = 0;
  int n_base = 0;  // sorted spheres on frame 0 (the fixed base), the first n_base
  std::vector<double> q_lo, q_hi;
  double reach = 0.0, r_max = 0.0;
  double fk_flops = 0.0;
  bool prismatic = false;  // any prismatic joint
  int n_box = 0, n_sbp = 0, n_bbp = 0;
};

struct ezo_env {
  float4* d_obs = nullptr;
  float* d_nhw = nullptr;
  int n_obs = 0, n_obs_pad = 0;
  double o_max = 0.0, R_max = 0.0;
  float4* d_box = nullptr;  // obstacle boxes, 4 float4 each
  int n_box = 0;
  std::vector<float4> h_obs;  // the obstacle spheres as uploaded (FP32)
  EnvDev dev() const { return EnvDev{d_obs, d_nhw, n_obs, n_obs_pad, d_box, n_box, 0}; }
  EnvDev dev_for(const ezo_robot* r) const;
};

// The robot spheres on the fixed base frame sit where they are for every
// configuration, so their pairs with a static obstacle set need no test per
// configuration when every such pair is clear. The sweep then starts at the
// first whole chunk of EZO_CH spheres past them; the clearance is checked in
// FP64 on the FP32 values the kernels use, against 1e-4 m, far above the
// rounding band of the FP32 test (the kernels place a base sphere exactly at
// its FP32 local coordinates), so every label is what the full sweep gives.
// Any base sphere within 1e-4 m of an obstacle keeps the full sweep.
static int sweep_first(const ezo_robot* r, const ezo_env* e) {
  const int cut = (r->n_base / EZO_CH) * EZO_CH;
  if (cut == 0) return 0;
  for (int s = 0; s < cut; ++s) {
    const float4 l = r->host.sph[s];
    for (const float4& o : e->h_obs) {
      const double dx = (double)l.x - o.x, dy = (double)l.y - o.y, dz = (double)l.z - o.z;
      if (std::sqrt(dx * dx + dy * dy + dz * dz) - (double)l.w - (double)o.w <= 1e-4) return 0;
    }
  }
  return cut;
}

EnvDev ezo_env::dev_for(const ezo_robot* r) const {
  EnvDev d = dev();
  d.s_first = sweep_first(r, this);
  return d;
}

static float band_E(const ezo_robot* r, const ezo_env* e) {
  // rounding bound of max_j t_ij - hu_i for the fast pair form (|c| <= reach,
  // |o| <= o_max, radii <= r_max, R_max), with a factor 8 of unit roundoff.
  const double a = r->reach + e->o_max, b = r->r_max + e->R_max;
  return (float)(8.0 * kU32 * (a * a + b * b));
}

extern "C" {

void ezo_params_default(ezo_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps = 0.05;
  p->delta = 0.05;
  p->tau = 0.5;
  p->step_back_max = 0.01;
  p->t_col = 1e-3;
  p->n_p = 10000;
  p->n_f = 10;
  p->n_b = 10;
  p->n_mix = 60;
  p->n_it_max = 50;
  p->seed = 1;
}

const char* ezo_last_error(void) { return g_err.c_str(); }

ezo_status ezo_robot_create(int32_t n, const double* a, const double* alpha, const double* d,
                            const double* theta_off, const double* q_lo, const double* q_hi, int32_t n_spheres,
                            const int32_t* sphere_frame, const double* sphere_xyz, const double* sphere_r,
                            int32_t n_self_pairs, const int32_t* self_pairs, const int32_t* joint_type,
                            ezo_robot** out) {
  if (!out) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: out is NULL");
  *out = nullptr;
  if (n < 1 || n > EZO_MAX_DOF) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: n must be in [1, 16]");
  if (n_spheres < 0 || n_spheres > EZO_MAX_SPHERES)
    return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: n_spheres must be in [0, 256]");
  if (n_self_pairs < 0 || n_self_pairs > 65535)
    return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: n_self_pairs must be in [0, 65535]");
  if (!a || !alpha || !d || !q_lo || !q_hi || (n_spheres && (!sphere_frame || !sphere_xyz || !sphere_r)) ||
      (n_self_pairs && !self_pairs))
    return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: null array");
  for (int s = 0; s < n_spheres; ++s) {
    if (sphere_frame[s] < 0 || sphere_frame[s] > n)
      return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: sphere_frame out of [0, n]");
    if (!(sphere_r[s] >= 0.0)) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: negative sphere radius");
  }
  for (int p = 0; p < 2 * n_self_pairs; ++p)
    if (self_pairs[p] < 0 || self_pairs[p] >= n_spheres)
      return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: self pair index out of range");
  for (int j = 0; j < n; ++j) {
    if (!(q_lo[j] <= q_hi[j])) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: q_lo > q_hi");
    if (joint_type && joint_type[j] != 0 && joint_type[j] != 1)
      return fail(EZO_ERR_INVALID_ARG, "ezo_robot_create: joint_type must be 0 (revolute) or 1 (prismatic)");
  }

  ezo_robot* r = new ezo_robot();
  r->n = n;
  r->n_spheres = n_spheres;
  r->nsp_pad = round_up(n_spheres, EZO_CH);
  r->n_self = n_self_pairs;
  r->q_lo.assign(q_lo, q_lo + n);
  r->q_hi.assign(q_hi, q_hi + n);
  RobotDev& h = r->host;
  h.n = n;
  h.n_spheres = n_spheres;
  h.n_spheres_pad = r->nsp_pad;
  h.n_self = n_self_pairs;
  double chain = 0.0;
  for (int j = 0; j < n; ++j) {
    h.ca[j] = (float)std::cos(alpha[j]);
    h.sa[j] = (float)std::sin(alpha[j]);
    h.a[j] = (float)a[j];
    h.d[j] = (float)d[j];
    h.toff[j] = theta_off ? (float)theta_off[j] : 0.f;
    const bool prism = joint_type && joint_type[j] == 1;
    h.kth[j] = prism ? 0.f : 1.f;
    h.kd[j] = prism ? 1.f : 0.f;
    r->prismatic = r->prismatic || prism;
    // the farthest a sphere can get from the base bounds the rounding band
    chain += std::fabs(a[j]) + std::fabs(d[j]) + (prism ? std::max(std::fabs(q_lo[j]), std::fabs(q_hi[j])) : 0.0);
  }
  // sort spheres by frame (stable) so the chain walk can emit them in order
  std::vector<int> order(n_spheres);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sphere_frame[x] < sphere_frame[y]; });
  std::vector<int> inv(n_spheres);
  double loc_max = 0.0;
  for (int s = 0; s < n_spheres; ++s) {
    const int o = order[s];
    inv[o] = s;
    h.sph[s] = make_float4((float)sphere_xyz[3 * o], (float)sphere_xyz[3 * o + 1], (float)sphere_xyz[3 * o + 2],
                           (float)sphere_r[o]);
    loc_max = std::max(loc_max, std::sqrt(sphere_xyz[3 * o] * sphere_xyz[3 * o] +
                                          sphere_xyz[3 * o + 1] * sphere_xyz[3 * o + 1] +
                                          sphere_xyz[3 * o + 2] * sphere_xyz[3 * o + 2]));
    r->r_max = std::max(r->r_max, sphere_r[o]);
  }
  for (int s = n_spheres; s < r->nsp_pad; ++s) h.sph[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int f = 0; f <= n + 1; ++f) h.frame_first[f] = 0;
  {
    int s = 0;
    for (int f = 0; f <= n; ++f) {
      h.frame_first[f] = s;
      while (s < n_spheres && sphere_frame[order[s]] == f) ++s;
    }
    h.frame_first[n + 1] = n_spheres;
  }
  r->n_base = h.frame_first[1];
  r->reach = chain + loc_max;
  r->sphere_sorted = inv;
  std::vector<ushort2> pairs(std::max(1, n_self_pairs));
  std::vector<float> rr(std::max(1, n_self_pairs));
  for (int p = 0; p < n_self_pairs; ++p) {
    const int i = self_pairs[2 * p], j = self_pairs[2 * p + 1];
    pairs[p] = make_ushort2((unsigned short)inv[i], (unsigned short)inv[j]);
    const float s = (float)sphere_r[i] + (float)sphere_r[j];
    rr[p] = s * s;
  }
  // self pairs as blocks [i0, i0+ni) x [k0, k0+nk) of sorted spheres when the
  // list is exactly such a union (the usual link-pair lists are)
  {
    std::vector<std::vector<int>> partners(n_spheres);
    std::vector<std::pair<int, int>> norm;
    for (int p = 0; p < n_self_pairs; ++p) {
      int i = inv[self_pairs[2 * p]], j = inv[self_pairs[2 * p + 1]];
      if (i > j) std::swap(i, j);
      norm.emplace_back(i, j);
    }
    std::sort(norm.begin(), norm.end());
    norm.erase(std::unique(norm.begin(), norm.end()), norm.end());
    for (auto& pr : norm) partners[pr.first].push_back(pr.second);
    // runs of each sphere's partner list
    std::vector<std::vector<std::pair<int, int>>> runs(n_spheres);
    for (int i = 0; i < n_spheres; ++i) {
      auto& P = partners[i];
      for (size_t a = 0; a < P.size();) {
        size_t b = a + 1;
        while (b < P.size() && P[b] == P[b - 1] + 1) ++b;
        runs[i].emplace_back(P[a], (int)(b - a));
        a = b;
      }
    }
    std::vector<int4> blocks;
    bool ok = (int)norm.size() == n_self_pairs;  // duplicates or i==j pairs: keep the list
    for (auto& pr : norm)
      if (pr.first == pr.second) ok = false;
    for (int i = 0; i < n_spheres && ok;) {
      if (runs[i].empty()) {
        ++i;
        continue;
      }
      int e = i + 1;
      while (e < n_spheres && runs[e] == runs[i]) ++e;
      for (auto& rn : runs[i]) {
        // the kernels take a block's rows in register chunks of EZO_CH
        // spheres (a short last chunk is padded): each block is oriented
        // for the fewer padded pair tests (the test is symmetric in the two
        // spheres of a pair)
        const int ni = e - i, nk = rn.second;
        const long pad_rows = (long)((ni + EZO_CH - 1) / EZO_CH) * nk;
        const long pad_cols = (long)((nk + EZO_CH - 1) / EZO_CH) * ni;
        blocks.push_back(pad_cols < pad_rows ? make_int4(rn.first, nk, i, ni) : make_int4(i, ni, rn.first, nk));
      }
      i = e;
    }
    // work items: one chunk of at most EZO_CH rows against all partners of
    // its block, sorted by partner count so that the lanes that take
    // consecutive items run loops of about the same length
    std::vector<int4> items;
    for (const int4& B : blocks)
      for (int r0 = B.x; r0 < B.x + B.y; r0 += EZO_CH)
        items.push_back(make_int4(r0, std::min(EZO_CH, B.x + B.y - r0), B.z, B.w));
    std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) { return a.w > b.w; });
    if (ok && !items.empty() && (int)items.size() <= EZO_MAX_SBLK) {
      h.n_sblk = (int)items.size();
      for (size_t b = 0; b < items.size(); ++b) h.sblk[b] = items[b];
    } else {
      h.n_sblk = 0;
    }
    const double a2 = 2.0 * (chain + loc_max), b2 = 2.0 * r->r_max;
    h.E_self = (float)(8.0 * kU32 * (a2 * a2 + b2 * b2));
  }
  // algorithmic FP32 flops: per joint ~45 (rotation and origin update), per
  // sphere 18 (centre) + 7 (half squared norm), 8 per pair
  r->fk_flops = 45.0 * n + 25.0 * n_spheres;
  RobotFK64 h64{};
  h64.n = n;
  h64.n_spheres = n_spheres;
  for (int j = 0; j < n; ++j) {
    h64.ca[j] = std::cos(alpha[j]);
    h64.sa[j] = std::sin(alpha[j]);
    h64.a[j] = a[j];
    h64.d[j] = d[j];
    h64.toff[j] = theta_off ? theta_off[j] : 0.0;
    h64.kth[j] = h.kth[j];
    h64.kd[j] = h.kd[j];
  }
  for (int f = 0; f < EZO_MAX_DOF + 2; ++f) h64.frame_first[f] = h.frame_first[f];
  for (int s = 0; s < n_spheres; ++s) {
    const int o = order[s];
    h64.sx[s] = sphere_xyz[3 * o];
    h64.sy[s] = sphere_xyz[3 * o + 1];
    h64.sz[s] = sphere_xyz[3 * o + 2];
  }
  cudaError_t e;
  if ((e = cudaMalloc(&r->d_pairs, pairs.size() * sizeof(ushort2))) != cudaSuccess ||
      (e = cudaMalloc(&r->d_rr, rr.size() * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&r->d_robot, sizeof(RobotDev))) != cudaSuccess ||
      (e = cudaMalloc(&r->d_fk64, sizeof(RobotFK64))) != cudaSuccess) {
    ezo_robot_free(r);
    return cuda_fail(e, "ezo_robot_create: cudaMalloc");
  }
  h.self_pairs = r->d_pairs;
  h.self_rr = r->d_rr;
  if ((e = cudaMemcpy(r->d_pairs, pairs.data(), pairs.size() * sizeof(ushort2), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(r->d_rr, rr.data(), rr.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(r->d_robot, &h, sizeof(RobotDev), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(r->d_fk64, &h64, sizeof(RobotFK64), cudaMemcpyHostToDevice)) != cudaSuccess) {
    ezo_robot_free(r);
    return cuda_fail(e, "ezo_robot_create: cudaMemcpy");
  }
  *out = r;
  g_err.clear();
  return EZO_OK;
}

void ezo_robot_free(ezo_robot* r) {
  if (!r) return;
  cudaFree(r->d_pairs);
  cudaFree(r->d_rr);
  cudaFree(r->d_sbp);
  cudaFree(r->d_bbp);
  cudaFree(r->d_robot);
  cudaFree(r->d_fk64);
  delete r;
}

int32_t ezo_robot_dof(const ezo_robot* r) { return r ? r->n : 0; }

ezo_status ezo_env_create(int32_t n_obs, const double* xyzr, ezo_env** out) {
  if (!out) return fail(EZO_ERR_INVALID_ARG, "ezo_env_create: out is NULL");
  *out = nullptr;
  if (n_obs < 0 || n_obs > EZO_MAX_OBS) return fail(EZO_ERR_INVALID_ARG, "ezo_env_create: n_obs must be in [0, 4096]");
  if (n_obs && !xyzr) return fail(EZO_ERR_INVALID_ARG, "ezo_env_create: xyzr is NULL");
  for (int j = 0; j < n_obs; ++j)
    if (!(xyzr[4 * j + 3] >= 0.0)) return fail(EZO_ERR_INVALID_ARG, "ezo_env_create: negative obstacle radius");
  ezo_env* e = new ezo_env();
  e->n_obs = n_obs;
  e->n_obs_pad = round_up(n_obs, EZO_CH);
  const int np = std::max(1, e->n_obs_pad);
  std::vector<float4> obs(np, make_float4(0.f, 0.f, 0.f, 0.f));
  std::vector<float> nhw(np, -1.0e30f);
  for (int j = 0; j < n_obs; ++j) {
    const double x = xyzr[4 * j], y = xyzr[4 * j + 1], z = xyzr[4 * j + 2], R = xyzr[4 * j + 3];
    obs[j] = make_float4((float)x, (float)y, (float)z, (float)R);
    e->h_obs.push_back(obs[j]);
    const double xf = (float)x, yf = (float)y, zf = (float)z, Rf = (float)R;
    nhw[j] = (float)(-0.5 * (xf * xf + yf * yf + zf * zf - Rf * Rf));
    e->o_max = std::max(e->o_max, std::sqrt(x * x + y * y + z * z));
    e->R_max = std::max(e->R_max, R);
  }
  cudaError_t err;
  if ((err = cudaMalloc(&e->d_obs, np * sizeof(float4))) != cudaSuccess ||
      (err = cudaMalloc(&e->d_nhw, np * sizeof(float))) != cudaSuccess ||
      (err = cudaMemcpy(e->d_obs, obs.data(), np * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(e->d_nhw, nhw.data(), np * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
    ezo_env_free(e);
    return cuda_fail(err, "ezo_env_create");
  }
  *out = e;
  g_err.clear();
  return EZO_OK;
}

void ezo_env_free(ezo_env* e) {
  if (!e) return;
  cudaFree(e->d_obs);
  cudaFree(e->d_nhw);
  cudaFree(e->d_box);
  delete e;
}

ezo_status ezo_robot_add_boxes(ezo_robot* r, int32_t n_box, const int32_t* box_frame, const double* box_xyz,
                               const double* box_rot, const double* box_half, int32_t n_sb, const int32_t* sb_pairs,
                               int32_t n_bb, const int32_t* bb_pairs) {
  if (!r) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: null robot");
  if (n_box < 0 || n_box > EZO_MAX_BOX) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: n_box must be in [0, 32]");
  if (n_sb < 0 || n_bb < 0 || n_sb > 65535 || n_bb > 65535)
    return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: pair counts must be in [0, 65535]");
  if (n_box && (!box_frame || !box_xyz || !box_rot || !box_half)) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: null array");
  if ((n_sb && !sb_pairs) || (n_bb && !bb_pairs)) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: null pair array");
  for (int k = 0; k < n_box; ++k) {
    if (box_frame[k] < 0 || box_frame[k] > r->n) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: box_frame out of [0, n]");
    for (int c = 0; c < 3; ++c)
      if (!(box_half[3 * k + c] >= 0.0)) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: negative half extent");
  }
  for (int p = 0; p < n_sb; ++p)
    if (sb_pairs[2 * p] < 0 || sb_pairs[2 * p] >= r->n_spheres || sb_pairs[2 * p + 1] < 0 || sb_pairs[2 * p + 1] >= n_box)
      return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: sphere-box pair index out of range");
  for (int p = 0; p < 2 * n_bb; ++p)
    if (bb_pairs[p] < 0 || bb_pairs[p] >= n_box) return fail(EZO_ERR_INVALID_ARG, "ezo_robot_add_boxes: box pair index out of range");
  RobotDev& h = r->host;
  // sort boxes by frame (stable), four float4 each: (centre, h_x), (axis k = column k of R, h_y / h_z / 0)
  std::vector<int> order(n_box), inv(n_box);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return box_frame[x] < box_frame[y]; });
  for (int k = 0; k < n_box; ++k) {
    const int o = order[k];
    inv[o] = k;
    const double* R = box_rot + 9 * o;  // row major, columns are the box axes
    const double* hh = box_half + 3 * o;
    h.box_l[4 * k] = make_float4((float)box_xyz[3 * o], (float)box_xyz[3 * o + 1], (float)box_xyz[3 * o + 2], (float)hh[0]);
    for (int a = 0; a < 3; ++a)
      h.box_l[4 * k + 1 + a] = make_float4((float)R[a], (float)R[3 + a], (float)R[6 + a], a < 2 ? (float)hh[a + 1] : 0.f);
  }
  {
    int k = 0;
    for (int f = 0; f <= r->n; ++f) {
      h.box_first[f] = k;
      while (k < n_box && box_frame[order[k]] == f) ++k;
    }
    h.box_first[r->n + 1] = n_box;
  }
  h.n_box = n_box;
  std::vector<ushort2> sb(std::max(1, n_sb)), bb(std::max(1, n_bb));
  for (int p = 0; p < n_sb; ++p)
    sb[p] = make_ushort2((unsigned short)r->sphere_sorted[sb_pairs[2 * p]], (unsigned short)inv[sb_pairs[2 * p + 1]]);
  for (int p = 0; p < n_bb; ++p)
    bb[p] = make_ushort2((unsigned short)inv[bb_pairs[2 * p]], (unsigned short)inv[bb_pairs[2 * p + 1]]);
  cudaFree(r->d_sbp);
  cudaFree(r->d_bbp);
  r->d_sbp = r->d_bbp = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc(&r->d_sbp, sb.size() * sizeof(ushort2))) != cudaSuccess ||
      (e = cudaMalloc(&r->d_bbp, bb.size() * sizeof(ushort2))) != cudaSuccess ||
      (e = cudaMemcpy(r->d_sbp, sb.data(), sb.size() * sizeof(ushort2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(r->d_bbp, bb.data(), bb.size() * sizeof(ushort2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "ezo_robot_add_boxes");
  h.n_sbp = n_sb;
  h.n_bbp = n_bb;
  h.sb_pairs = r->d_sbp;
  h.bb_pairs = r->d_bbp;
  r->n_box = n_box;
  r->n_sbp = n_sb;
  r->n_bbp = n_bb;
  // pose work per box (centre 9 + axes 27 multiply-adds)
  r->fk_flops = 45.0 * r->n + 25.0 * r->n_spheres + 72.0 * n_box;
  if ((e = cudaMemcpy(r->d_robot, &h, sizeof(RobotDev), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "ezo_robot_add_boxes");
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_env_add_boxes(ezo_env* e, int32_t n_box, const double* boxes) {
  if (!e || n_box < 0 || n_box > EZO_MAX_EBOX || (n_box && !boxes))
    return fail(EZO_ERR_INVALID_ARG, "ezo_env_add_boxes: need an env and 0 <= n_box <= 64");
  std::vector<float4> b((size_t)std::max(1, 4 * n_box));
  for (int k = 0; k < n_box; ++k) {
    const double* x = boxes + 15 * k;  // centre, half extents, R row major (columns = axes)
    for (int c = 3; c < 6; ++c)
      if (!(x[c] >= 0.0)) return fail(EZO_ERR_INVALID_ARG, "ezo_env_add_boxes: negative half extent");
    const double* R = x + 6;
    b[4 * k] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)x[3]);
    for (int a = 0; a < 3; ++a)
      b[4 * k + 1 + a] = make_float4((float)R[a], (float)R[3 + a], (float)R[6 + a], a < 2 ? (float)x[4 + a] : 0.f);
  }
  cudaFree(e->d_box);
  e->d_box = nullptr;
  cudaError_t err;
  if ((err = cudaMalloc(&e->d_box, b.size() * sizeof(float4))) != cudaSuccess ||
      (err = cudaMemcpy(e->d_box, b.data(), b.size() * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(err, "ezo_env_add_boxes");
  e->n_box = n_box;
  g_err.clear();
  return EZO_OK;
}

int ezo_internal_tuned_lanes(const ezo_robot* robot, const ezo_env* env, long long N, cudaStream_t s);

ezo_status ezo_check_collision(const ezo_robot* robot, const ezo_env* env, const float* q_dev, int64_t N,
                               int64_t ldq, uint8_t* flags_dev, int32_t lanes, void* stream) {
  if (!robot || !env) return fail(EZO_ERR_INVALID_ARG, "ezo_check_collision: null handle");
  if (N < 0 || ldq < N) return fail(EZO_ERR_INVALID_ARG, "ezo_check_collision: need 0 <= N <= ldq");
  if (N > 0 && (!q_dev || !flags_dev)) return fail(EZO_ERR_INVALID_ARG, "ezo_check_collision: null buffer");
  if (lanes == 0) lanes = ezo_internal_tuned_lanes(robot, env, N, (cudaStream_t)stream);
  if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)
    return fail(EZO_ERR_INVALID_ARG, "ezo_check_collision: lanes_per_config must be 0, 1, 2, 4 or 8");
  if (check_smem_bytes(robot->nsp_pad, env->n_obs_pad, 128, lanes, robot->n_box, env->n_box) > kSmemBudget)
    return fail(EZO_ERR_INVALID_ARG,
                "ezo_check_collision: robot and obstacle spheres exceed shared memory at this lanes_per_config");
  cudaError_t e = launch_check_flat(robot->d_robot, robot->n, robot->nsp_pad, robot->n_box, env->dev_for(robot), band_E(robot, env), q_dev, ldq, N,
                                    flags_dev, lanes, sm_count() * 32, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ezo_check_collision");
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_signed_distance(const ezo_robot* robot, const ezo_env* env, const float* q_dev, int64_t N,
                               int64_t ldq, float* sd_dev, void* stream) {
  if (!robot || !env) return fail(EZO_ERR_INVALID_ARG, "ezo_signed_distance: null handle");
  if (N < 0 || ldq < N) return fail(EZO_ERR_INVALID_ARG, "ezo_signed_distance: need 0 <= N <= ldq");
  if (N > 0 && (!q_dev || !sd_dev)) return fail(EZO_ERR_INVALID_ARG, "ezo_signed_distance: null buffer");
  if (robot->n_box || env->n_box)
    return fail(EZO_ERR_INVALID_ARG, "ezo_signed_distance: sphere geometries only (the robot or env has boxes)");
  if (check_smem_bytes(robot->nsp_pad, env->n_obs_pad, 64, 1) > kSmemBudget)
    return fail(EZO_ERR_INVALID_ARG, "ezo_signed_distance: robot and obstacle spheres exceed shared memory");
  cudaError_t e = launch_sd_flat(robot->d_robot, robot->n, robot->nsp_pad, env->dev(), q_dev, ldq, N, sd_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ezo_signed_distance");
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_sphere_centres(const ezo_robot* robot, const float* q_dev, int64_t N, int64_t ldq, int32_t fp64,
                              double* out_dev, void* cuda_stream) {
  if (!robot || (N > 0 && (!q_dev || !out_dev)) || N < 0 || ldq < N || (fp64 != 0 && fp64 != 1))
    return fail(EZO_ERR_INVALID_ARG, "ezo_sphere_centres: bad argument");
  const cudaError_t e = launch_fk_centres(robot->d_robot, robot->d_fk64, robot->n, robot->nsp_pad, q_dev, ldq, N,
                                          fp64, out_dev, nullptr, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "ezo_sphere_centres");
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_fk_error(const ezo_robot* robot, const float* q_dev, int64_t N, int64_t ldq, float* err_dev,
                        void* cuda_stream) {
  if (!robot || (N > 0 && (!q_dev || !err_dev)) || N < 0 || ldq < N)
    return fail(EZO_ERR_INVALID_ARG, "ezo_fk_error: bad argument");
  const cudaError_t e = launch_fk_centres(robot->d_robot, robot->d_fk64, robot->n, robot->nsp_pad, q_dev, ldq, N, 2,
                                          nullptr, err_dev, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "ezo_fk_error");
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_hit_and_run(const double* A_dev, const double* b_dev, int32_t m, int32_t n, int32_t lda,
                           const double* v1, const double* v2, int64_t N, int32_t n_mix, uint64_t seed,
                           uint32_t stream_id, int32_t round_k, float* x_dev, int64_t ldx, void* stream) {
  if (n < 1 || n > EZO_MAX_DOF) return fail(EZO_ERR_INVALID_ARG, "ezo_hit_and_run: n must be in [1, 16]");
  if (m < 0 || m > 2048 || lda < n) return fail(EZO_ERR_INVALID_ARG, "ezo_hit_and_run: need 0 <= m <= 2048, lda >= n");
  if (N < 0 || ldx < N || n_mix < 0) return fail(EZO_ERR_INVALID_ARG, "ezo_hit_and_run: bad N, ldx or n_mix");
  if (!v1 || !v2 || (N > 0 && !x_dev) || (m > 0 && (!A_dev || !b_dev)))
    return fail(EZO_ERR_INVALID_ARG, "ezo_hit_and_run: null pointer");
  cudaError_t e = launch_sample_flat(A_dev, b_dev, m, lda, n, v1, v2, N, n_mix, seed, stream_id, round_k, x_dev, ldx,
                                     (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ezo_hit_and_run");
  g_err.clear();
  return EZO_OK;
}

// Internal accessors for other translation units of the library (hidden).
__attribute__((visibility("hidden"))) const RobotDev* ezo_internal_robot_dev(const ezo_robot* r, int* n,
                                                                               int* nsp_pad, double* q_lo,
                                                                               double* q_hi) {
  if (!r) return nullptr;
  *n = r->n;
  *nsp_pad = r->nsp_pad;
  for (int j = 0; j < r->n; ++j) {
    q_lo[j] = r->q_lo[j];
    q_hi[j] = r->q_hi[j];
  }
  return r->d_robot;
}

__attribute__((visibility("hidden"))) int ezo_internal_env_dev(const ezo_robot* r, const ezo_env* e,
                                                                EnvDevFull* out) {
  if (!r || !e || !out) return 1;
  out->e = e->dev_for(r);
  out->E = band_E(r, e);
  out->pad = 0.f;
  return 0;
}

__attribute__((visibility("hidden"))) void ezo_internal_set_error(const char* msg) { g_err = msg ? msg : ""; }

__attribute__((visibility("hidden"))) int ezo_internal_robot_prismatic(const ezo_robot* r) {
  return r && r->prismatic ? 1 : 0;
}

__attribute__((visibility("hidden"))) int ezo_internal_robot_boxes(const ezo_robot* r) { return r ? r->n_box : 0; }

__attribute__((visibility("hidden"))) int ezo_internal_env_boxes(const ezo_env* e) { return e ? e->n_box : 0; }

double ezo_check_flops(const ezo_robot* robot, const ezo_env* env) {
  if (!robot || !env) return 0.0;
  // 8 flops per sphere pair, ~30 per sphere-box pair, ~330 per box-box pair
  return robot->fk_flops + 8.0 * ((double)robot->n_spheres * env->n_obs + robot->n_self) +
         30.0 * ((double)robot->n_spheres * env->n_box + (double)robot->n_box * env->n_obs + robot->n_sbp) +
         330.0 * ((double)robot->n_box * env->n_box + robot->n_bbp);
}

int32_t ezo_check_static_spheres(const ezo_robot* robot, const ezo_env* env) {
  return (robot && env) ? sweep_first(robot, env) : 0;
}

// ------------------------------------------------------------------ batch --
}  // extern "C"

struct ezo_batch {
  const ezo_robot* robot = nullptr;
  int B = 0, n = 0, m0 = 0, m_cap = 0, s_cap_max = 0, np_max = 0, max_path_len = 1, max_obs_pad = 0, max_ebox = 0;
  ezo_params prm{};
  std::vector<SegState> st0;
  std::vector<int> path_first;
  std::vector<EnvDevFull> envs;
  long long total_s = 0, total_c = 0;
  int max_sample_tiles = 0, max_bisect_tiles = 0;
  // device buffers
  SegState* d_st = nullptr;
  double *d_v1 = nullptr, *d_v2 = nullptr, *d_A = nullptr, *d_b = nullptr;
  float* d_S = nullptr;
  uint8_t* d_flags = nullptr;
  int* d_cidx = nullptr;
  double *d_cstar = nullptr, *d_dist = nullptr;
  float *d_c32 = nullptr, *d_cn = nullptr;
  uint32_t* d_bits = nullptr;
  double *d_ga = nullptr, *d_gb = nullptr;
  int* d_pidx = nullptr;
  double* d_pdelta = nullptr;
  int2 *d_stiles = nullptr, *d_btiles = nullptr;
  RoundSummary* d_sum = nullptr;
  RoundSummary* h_sum = nullptr;
  EnvDevFull* d_envs = nullptr;
  int* d_path_first = nullptr;
  uint8_t* d_contained = nullptr;
  SegState* d_st0 = nullptr;    // initial state, for resets
  double *d_A0 = nullptr, *d_b0 = nullptr;  // initial polytopes
  std::vector<double> v1h, v2h;
  BatchView view{};
  int T_check = 1, T_bisect = 4, split_below = 0;
  int t_min = 1;  // fewest lanes per configuration whose sphere centres fit in shared memory
  long long tot_s1 = 0, tot_np = 0;  // samples of round 1 and N_p over the batch (tuning keys)
  int sms = 1;
  int grid_sample = 1, grid_check = 1, grid_bisect = 1;
  // graph mode
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // the wavefront order in one graph (waves and rounds as nested WHILE nodes)
  cudaGraph_t wgraph = nullptr;
  cudaGraphExec_t wgexec = nullptr;
  int *d_wnext = nullptr, *d_wlast = nullptr;
  uint8_t* d_wkept = nullptr;
  cudaStream_t cap_stream = nullptr;
  EventPool events;
  // surrogate-guided bisection
  ezo_surrogate* sur = nullptr;
  long long sur_rows = 0;
  long long claim_cap = 0;  // work units of the largest round-kernel launch
};

namespace {

// The captured graphs hold the batch view and the launch shapes by value:
// dropped whenever either changes, rebuilt on the next graph run.
void drop_graphs(ezo_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->wgexec) cudaGraphExecDestroy(b->wgexec);
  if (b->wgraph) cudaGraphDestroy(b->wgraph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->wgexec = nullptr;
  b->wgraph = nullptr;
}

ezo_status batch_free_device(ezo_batch* b) {
  drop_graphs(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  void* ptrs[] = {b->d_st,    b->d_v1,    b->d_v2,   b->d_A,    b->d_b,      b->d_S,      b->d_flags,
                  b->d_cidx,  b->d_cstar, b->d_dist, b->d_c32,  b->d_cn,     b->d_bits,   b->d_pidx, b->d_ga, b->d_gb,
                  b->d_pdelta, b->d_stiles, b->d_btiles, b->d_sum, b->d_envs, b->d_path_first, b->d_contained, b->d_st0, b->d_A0, b->d_b0,
                  b->view.s_p32, b->view.s_d32, b->view.s_lo, b->view.s_hi,
                  b->view.s_bits, b->view.s_ok, b->view.s_rows, b->view.sm_seats, b->view.q_claim,
                  b->d_wnext, b->d_wlast, b->d_wkept};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_sum) cudaFreeHost(b->h_sum);
  for (auto e : b->events.ev) cudaEventDestroy(e);
  return EZO_OK;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T));
}

int host_test_size(int k, double eps, double delta, double tau) {
  const double dk = 6.0 * delta / (M_PI * M_PI * k * (double)k);
  return (int)std::ceil(2.0 * std::log(1.0 / dk) / (eps * tau * tau));
}

}  // namespace

extern "C" cudaError_t ezo_internal_mlp_bisect(ezo_surrogate* S, long long rows_cap, const int* m_dev,
                                               const float* s_p32, const float* s_d32, float* s_lo, float* s_hi,
                                               uint32_t* s_bits, int n_b, float margin, cudaStream_t s);
extern "C" int ezo_internal_surrogate_dof(const ezo_surrogate* S);

namespace {

// Step 4: the candidates' projections, then the exact halvings, then c* and
// its plane. With a surrogate, between the projections and c*: N_b surrogate
// bisection steps for every candidate (all of them in one tensor-core
// launch), one exact check of each end point, exact halvings for the
// candidates whose end point is free.
cudaError_t launch_bisect_step(ezo_batch* b, cudaStream_t s) {
  const int g = row_grid((long long)b->max_bisect_tiles * kTile);
  if (!b->sur) return launch_bisect_exact(b->view, b->T_bisect, b->grid_bisect, g, s);
  b->view.bis_mode = 0;
  cudaError_t e = launch_bisect_prep(b->view, g, s);
  if (e == cudaSuccess)
    e = ezo_internal_mlp_bisect(b->sur, b->sur_rows, b->view.s_rows, b->view.s_p32, b->view.s_d32, b->view.s_lo,
                                b->view.s_hi, b->view.s_bits, b->prm.n_b, b->view.sbis_margin, s);
  if (e == cudaSuccess) {
    b->view.bis_mode = 1;
    e = launch_round_bisect(b->view, b->T_bisect, b->grid_bisect, s);
  }
  if (e == cudaSuccess) {
    b->view.bis_mode = 2;
    e = launch_round_bisect(b->view, b->T_bisect, b->grid_bisect, s);
  }
  b->view.bis_mode = 0;
  if (e == cudaSuccess) e = launch_bisect_finish(b->view, g, s);
  return e;
}

ezo_status launch_step(ezo_batch* b, int step, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g_prof_on) {
    e0 = b->events.get();
    e1 = b->events.get();
    // the fused close counts as round end, the placement that closes the
    // round as placement
    b->events.kind.push_back(step == 7 ? 6 : (step == 8 ? 5 : step));
    cudaEventRecord(e0, s);
  }
  switch (step) {
    case 0: e = launch_round_begin(b->view, s); break;
    case 1: e = launch_round_sample(b->view, b->split_below, b->grid_sample, s); break;
    case 2: e = launch_round_check(b->view, b->T_check, b->grid_check, s); break;
    case 3: e = launch_round_certify(b->view, s); break;
    case 4: e = launch_bisect_step(b, s); break;
    case 5: e = launch_round_place(b->view, s); break;
    case 6: e = launch_round_end(b->view, s); break;
    case 7: e = launch_round_close(b->view, s); break;  // 6 fused with the next round's 0
    case 8: e = launch_round_place(b->view, s, true); break;  // 5 whose last block runs 7
    default: return fail(EZO_ERR_INVALID_ARG, "ezo_batch_step: step must be in [0, 8]");
  }
  if (g_prof_on) cudaEventRecord(e1, s);
  if (e != cudaSuccess) return cuda_fail(e, "round kernel launch");
  return EZO_OK;
}

void collect_profile(ezo_batch* b) {
  if (!g_prof_on) return;
  for (size_t i = 0; i < b->events.kind.size(); ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->events.ev[2 * i], b->events.ev[2 * i + 1]) == cudaSuccess) {
      g_prof_ms[b->events.kind[i]] += ms;
      g_prof_n[b->events.kind[i]] += 1;
    }
  }
  b->events.kind.clear();
  b->events.used = 0;
}

// The run loops size the first round once; every round then ends with the
// fused round-close kernel, which also sizes the next round.
// a round of the run loops: walks, labels, certification, bisection, and the
// placement whose last block closes the round (step 8)
const int kRoundSteps[5] = {1, 2, 3, 4, 8};

ezo_status run_host_loop(ezo_batch* b, cudaStream_t s) {
  ezo_status st0 = launch_step(b, 0, s);
  if (st0 != EZO_OK) return st0;
  for (int r = 0; r <= b->prm.n_it_max + 1; ++r) {
    for (int step : kRoundSteps) {
      ezo_status st = launch_step(b, step, s);
      if (st != EZO_OK) return st;
    }
    EZO_CUDA(cudaMemcpyAsync(b->h_sum, b->d_sum, sizeof(RoundSummary), cudaMemcpyDeviceToHost, s));
    EZO_CUDA(cudaStreamSynchronize(s));
    collect_profile(b);
    if (b->h_sum->active == 0) break;
  }
  return EZO_OK;
}

ezo_status build_graph(ezo_batch* b) {
#if CUDART_VERSION >= 12040
  EZO_CUDA(cudaGraphCreate(&b->graph, 0));
  if (!b->cap_stream) EZO_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  const bool prof = g_prof_on;
  g_prof_on = false;
  // the first round's sizing, then a WHILE node whose body runs a round and
  // sizes the next one
  EZO_CUDA(cudaStreamBeginCaptureToGraph(b->cap_stream, b->graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  ezo_status st = launch_step(b, 0, b->cap_stream);
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &captured);
  if (st != EZO_OK || ce != cudaSuccess) {
    g_prof_on = prof;
    return st != EZO_OK ? st : cuda_fail(ce, "cudaStreamEndCapture");
  }
  cudaGraphNode_t first = nullptr;
  size_t n_nodes = 1;
  EZO_CUDA(cudaGraphGetNodes(b->graph, &first, &n_nodes));
  cudaGraphConditionalHandle h;
  EZO_CUDA(cudaGraphConditionalHandleCreate(&h, b->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  EZO_CUDA(cudaGraphAddNode(&node, b->graph, &first, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  BatchView saved = b->view;
  b->view.graph_cond = (unsigned long long)h;
  EZO_CUDA(cudaStreamBeginCaptureToGraph(b->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  for (int step : kRoundSteps) {
    if (st != EZO_OK) break;
    st = launch_step(b, step, b->cap_stream);
  }
  ce = cudaStreamEndCapture(b->cap_stream, &captured);
  g_prof_on = prof;
  b->view = saved;
  if (st != EZO_OK) return st;
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
  EZO_CUDA(cudaGraphInstantiate(&b->gexec, b->graph, 0));
  return EZO_OK;
#else
  return fail(EZO_ERR_CUDA, "graph mode needs CUDA 12.4 or newer");
#endif
}

// sync = false leaves the graph running on the stream (the host loop reads
// the round summary every round, so it always ends synchronised)
ezo_status run_graph(ezo_batch* b, cudaStream_t s, bool sync = true) {
  if (!b->gexec) {
    ezo_status st = build_graph(b);
    if (st != EZO_OK) return st;
  }
  EZO_CUDA(cudaGraphLaunch(b->gexec, s));
  if (sync) EZO_CUDA(cudaStreamSynchronize(s));
  return EZO_OK;
}

#if CUDART_VERSION >= 12040
// The last node of a graph whose nodes form one chain (captured on one
// stream).
cudaError_t chain_tail(cudaGraph_t g, cudaGraphNode_t* tail) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  if ((e = cudaGraphGetNodes(g, nodes.data(), &n)) != cudaSuccess) return e;
  *tail = nullptr;
  for (cudaGraphNode_t nd : nodes) {
    size_t out = 0;
    if ((e = cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &out)) != cudaSuccess) return e;
    if (out == 0) *tail = nd;
  }
  return *tail ? cudaSuccess : cudaErrorInvalidValue;
}

// A WHILE node after `dep` in graph g; its handle (made on g) is not reset at
// launch: the kernels set it before the node runs.
cudaError_t add_while(cudaGraph_t g, cudaGraphNode_t dep, unsigned default_value, unsigned flags,
                      cudaGraphConditionalHandle* h, cudaGraph_t* body) {
  cudaError_t e = cudaGraphConditionalHandleCreate(h, g, default_value, flags);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = *h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &cp);
  if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
  return e;
}
#endif

// The wavefront order (Sec. VI-A: each path in order with the skip rule, the
// current segments of all paths in one batched run) as one graph:
//   wave_init -> WHILE(waves) { containment -> wave_select -> first sizing
//                               -> WHILE(rounds) { one round } }
// wave_select applies the skip rule and the stop after a collision, picks the
// next segment of every path and sets both conditions from the count of
// active segments; the round body is the one of build_graph.
ezo_status build_wave_graph(ezo_batch* b) {
#if CUDART_VERSION >= 12040
  const size_t B = b->B;
  if (!b->d_wnext) {
    cudaError_t e = dalloc(&b->d_wnext, B);
    if (e == cudaSuccess) e = dalloc(&b->d_wlast, B);
    if (e == cudaSuccess) e = dalloc(&b->d_wkept, B);
    if (e != cudaSuccess) return cuda_fail(e, "wave graph: allocation");
  }
  if (!b->cap_stream) EZO_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  const bool prof = g_prof_on;
  g_prof_on = false;
  const BatchView saved = b->view;
  ezo_status st = EZO_OK;
  cudaGraph_t captured = nullptr, wbody = nullptr, rbody = nullptr;
  cudaGraphNode_t tail = nullptr;
  cudaGraphConditionalHandle hw = 0, hr = 0;
  auto cap = [&](cudaGraph_t g, cudaGraphNode_t dep, auto&& fn) -> cudaError_t {
    cudaError_t e = cudaStreamBeginCaptureToGraph(b->cap_stream, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0,
                                                  cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    fn();
    return cudaStreamEndCapture(b->cap_stream, &captured);
  };
  cudaError_t e = cudaGraphCreate(&b->wgraph, 0);
  if (e == cudaSuccess)
    e = cap(b->wgraph, nullptr, [&] {
      cudaError_t le = launch_wave_init(b->view, b->d_wnext, b->d_wlast, b->d_wkept, b->cap_stream);
      if (le != cudaSuccess) st = cuda_fail(le, "wave graph: init");
    });
  if (e == cudaSuccess && st == EZO_OK) e = chain_tail(b->wgraph, &tail);
  if (e == cudaSuccess && st == EZO_OK) e = add_while(b->wgraph, tail, 1, cudaGraphCondAssignDefault, &hw, &wbody);
  if (e == cudaSuccess && st == EZO_OK) {
    hr = 0;
    e = cudaGraphConditionalHandleCreate(&hr, wbody, 0, 0);
  }
  if (e == cudaSuccess && st == EZO_OK)
    e = cap(wbody, nullptr, [&] {
      cudaError_t le = cudaMemsetAsync(b->d_contained, 0, B * (size_t)b->max_path_len, b->cap_stream);
      if (le == cudaSuccess) le = launch_containment(b->view, b->d_contained, 1e-9, b->cap_stream);
      if (le == cudaSuccess)
        le = launch_wave_select(b->view, b->d_contained, b->d_wnext, b->d_wlast, b->d_wkept,
                                (unsigned long long)hw, (unsigned long long)hr, b->cap_stream);
      if (le != cudaSuccess) st = cuda_fail(le, "wave graph: skip rule");
      if (st == EZO_OK) st = launch_step(b, 0, b->cap_stream);
    });
  if (e == cudaSuccess && st == EZO_OK) e = chain_tail(wbody, &tail);
  if (e == cudaSuccess && st == EZO_OK) {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hr;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, wbody, &tail, nullptr, 1, &cp);
    if (e == cudaSuccess) rbody = cp.conditional.phGraph_out[0];
  }
  if (e == cudaSuccess && st == EZO_OK) {
    b->view.graph_cond = (unsigned long long)hr;
    e = cap(rbody, nullptr, [&] {
      for (int step : kRoundSteps) {
        if (st != EZO_OK) break;
        st = launch_step(b, step, b->cap_stream);
      }
    });
  }
  g_prof_on = prof;
  b->view = saved;
  if (e == cudaSuccess && st == EZO_OK) e = cudaGraphInstantiate(&b->wgexec, b->wgraph, 0);
  if (st == EZO_OK && e != cudaSuccess) st = cuda_fail(e, "wave graph");
  if (st != EZO_OK) {
    if (b->wgraph) cudaGraphDestroy(b->wgraph);
    b->wgraph = nullptr;
    b->wgexec = nullptr;
  }
  return st;
#else
  return fail(EZO_ERR_CUDA, "graph mode needs CUDA 12.4 or newer");
#endif
}

ezo_status run_batch(ezo_batch* b, int mode, cudaStream_t s, bool sync = true) {
  if (mode == EZO_RUN_GRAPH) return run_graph(b, s, sync);
  return run_host_loop(b, s);
}

ezo_status set_status(ezo_batch* b, int g, int status, cudaStream_t s) {
  EZO_CUDA(cudaMemcpyAsync(&b->d_st[g].status, &status, sizeof(int), cudaMemcpyHostToDevice, s));
  EZO_CUDA(cudaStreamSynchronize(s));
  return EZO_OK;
}

ezo_status read_states(ezo_batch* b, std::vector<SegState>& out, cudaStream_t s) {
  out.resize(b->B);
  EZO_CUDA(cudaMemcpyAsync(out.data(), b->d_st, sizeof(SegState) * b->B, cudaMemcpyDeviceToHost, s));
  EZO_CUDA(cudaStreamSynchronize(s));
  return EZO_OK;
}

}  // namespace

extern "C" {

ezo_status ezo_batch_create(const ezo_robot* robot, int32_t n_env, const ezo_env* const* envs, int32_t n_seg,
                            const double* v1, const double* v2, const int32_t* seg_env, const int32_t* seg_np,
                            const uint32_t* seg_stream, const int32_t* path_first, const double* A0,
                            const double* b0, int32_t m0, const ezo_params* prm, ezo_batch** out) {
  if (!out) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: out is NULL");
  *out = nullptr;
  if (!robot || !prm || n_env < 1 || !envs) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: null argument");
  if (n_seg < 1 || !v1 || !v2) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: need n_seg >= 1 and v1, v2");
  if (!(prm->eps > 0.0 && prm->eps < 1.0) || !(prm->delta > 0.0 && prm->delta < 1.0) ||
      !(prm->tau > 0.0 && prm->tau < 1.0) || !(prm->step_back_max >= 0.0) || !(prm->t_col >= 0.0) ||
      prm->n_p < 1 || prm->n_f < 1 || prm->n_b < 0 || prm->n_b > 32 || prm->n_mix < 0 || prm->n_it_max < 1)
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: parameter out of range");
  for (int e = 0; e < n_env; ++e)
    if (!envs[e]) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: null env");
  const int n = robot->n;
  if (A0 && (m0 < 1 || !b0)) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: bad domain");
  std::vector<double> A0v, b0v;
  if (A0) {
    A0v.assign(A0, A0 + (size_t)m0 * n);
    b0v.assign(b0, b0 + m0);
  } else {
    m0 = 2 * n;
    A0v.assign((size_t)m0 * n, 0.0);
    b0v.assign(m0, 0.0);
    for (int j = 0; j < n; ++j) {
      A0v[(size_t)j * n + j] = 1.0;
      b0v[j] = robot->q_hi[j];
      A0v[(size_t)(n + j) * n + j] = -1.0;
      b0v[n + j] = -robot->q_lo[j];
    }
  }
  ezo_batch* b = new ezo_batch();
  b->robot = robot;
  b->B = n_seg;
  b->n = n;
  b->m0 = m0;
  b->prm = *prm;
  b->m_cap = m0 + prm->n_f * prm->n_it_max;
  if (b->m_cap > 2048) {
    delete b;
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: m0 + n_f * n_it_max must be <= 2048");
  }
  const int m_last = host_test_size(prm->n_it_max, prm->eps, prm->delta, prm->tau) + 16;
  b->st0.resize(n_seg);
  b->path_first.resize(n_seg);
  for (int g = 0; g < n_seg; ++g) {
    SegState& s = b->st0[g];
    std::memset(&s, 0, sizeof(s));
    s.k = 1;
    s.status = SEG_ACTIVE;
    s.m = m0;
    s.n_p = seg_np ? seg_np[g] : prm->n_p;
    if (s.n_p < 1) {
      delete b;
      return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: seg_np must be >= 1");
    }
    s.env = seg_env ? seg_env[g] : 0;
    if (s.env < 0 || s.env >= n_env) {
      delete b;
      return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: seg_env out of range");
    }
    s.stream = seg_stream ? seg_stream[g] : (uint32_t)g;
    s.box_rows = A0 ? 0 : 2 * n;  // the sampler skips the dot products of the joint-box rows
    s.s_cap = std::max(s.n_p, m_last);
    s.sample_off = b->total_s;
    s.cand_off = b->total_c;
    b->total_s += s.s_cap;
    b->total_c += s.n_p;
    b->s_cap_max = std::max(b->s_cap_max, s.s_cap);
    b->np_max = std::max(b->np_max, s.n_p);
    b->max_sample_tiles += (s.s_cap + kTile - 1) / kTile;
    b->max_bisect_tiles += (s.n_p + kTile - 1) / kTile;
    b->path_first[g] = path_first ? path_first[g] : 0;
    if (b->path_first[g] < 0 || b->path_first[g] > g) {
      delete b;
      return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: path_first[g] must be in [0, g]");
    }
    b->max_path_len = std::max(b->max_path_len, g - b->path_first[g] + 1);
  }
  if (b->np_max > (1 << 20)) {
    delete b;
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: N_p must be <= 2^20");
  }
  b->envs.resize(n_env);
  for (int e = 0; e < n_env; ++e) {
    b->envs[e].e = envs[e]->dev_for(robot);
    b->envs[e].E = band_E(robot, envs[e]);
    b->max_obs_pad = std::max(b->max_obs_pad, envs[e]->n_obs_pad);
    b->max_ebox = std::max(b->max_ebox, envs[e]->n_box);
  }
  // the collision kernels keep one set of sphere centres per group of lanes
  // in shared memory: large robots with many obstacles need more lanes per
  // configuration (and per bisection candidate)
  while (b->t_min <= 8 &&
         check_smem_bytes(robot->nsp_pad, b->max_obs_pad, 128, b->t_min, robot->n_box, b->max_ebox) > kSmemBudget)
    b->t_min *= 2;
  if (b->t_min > 8) {
    delete b;
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_create: robot spheres and obstacles exceed shared memory at 8 lanes");
  }
  const long long B = n_seg, mc = b->m_cap;
  cudaError_t e = cudaSuccess;
#define EZO_ALLOC(p, cnt) \
  if (e == cudaSuccess) e = dalloc(&(p), (size_t)(cnt))
  EZO_ALLOC(b->d_st, B);
  EZO_ALLOC(b->d_v1, B * n);
  EZO_ALLOC(b->d_v2, B * n);
  EZO_ALLOC(b->d_A, B * mc * n);
  EZO_ALLOC(b->d_b, B * mc);
  EZO_ALLOC(b->d_S, b->total_s * n);
  EZO_ALLOC(b->d_flags, b->total_s);
  EZO_ALLOC(b->d_cidx, b->total_c);
  EZO_ALLOC(b->d_cstar, b->total_c * n);
  EZO_ALLOC(b->d_dist, b->total_c);
  EZO_ALLOC(b->d_c32, b->total_c * n);
  EZO_ALLOC(b->d_cn, b->total_c);
  EZO_ALLOC(b->d_bits, b->total_c);
  EZO_ALLOC(b->d_ga, b->total_c * n);
  EZO_ALLOC(b->d_gb, b->total_c);
  EZO_ALLOC(b->d_pidx, B * prm->n_f);
  EZO_ALLOC(b->d_pdelta, B * prm->n_f);
  EZO_ALLOC(b->d_stiles, b->max_sample_tiles);
  EZO_ALLOC(b->d_btiles, b->max_bisect_tiles);
  EZO_ALLOC(b->d_sum, 1);
  EZO_ALLOC(b->d_envs, n_env);
  EZO_ALLOC(b->d_path_first, B);
  EZO_ALLOC(b->d_contained, B * b->max_path_len);
  EZO_ALLOC(b->d_st0, B);
  EZO_ALLOC(b->d_A0, B * mc * n);
  EZO_ALLOC(b->d_b0, B * mc);
  // the bisection's projected candidate rows (c_proj, c - c_proj in FP32)
  b->view.s_ld = n <= 8 ? 8 : EZO_MAX_DOF;
  EZO_ALLOC(b->view.s_p32, (long long)b->max_bisect_tiles * kTile * b->view.s_ld);
  EZO_ALLOC(b->view.s_d32, (long long)b->max_bisect_tiles * kTile * b->view.s_ld);
  EZO_ALLOC(b->view.sm_seats, kSeatSlots);
  // one claim per work unit of the largest launch: 8 passes per sample tile,
  // up to 32 per bisection tile
  b->claim_cap = std::max<long long>((long long)b->max_sample_tiles * 8, (long long)b->max_bisect_tiles * 32);
  EZO_ALLOC(b->view.q_claim, b->claim_cap + 1);
  b->view.q_claim_cap = (int)b->claim_cap;
#undef EZO_ALLOC
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_sum, sizeof(RoundSummary));
  if (e != cudaSuccess) {
    batch_free_device(b);
    delete b;
    return cuda_fail(e, "ezo_batch_create: allocation");
  }
  // initial contents
  std::vector<double> Ah((size_t)B * mc * n, 0.0), bh((size_t)B * mc, 0.0);
  for (long long g = 0; g < B; ++g) {
    std::copy(A0v.begin(), A0v.end(), Ah.begin() + g * mc * n);
    std::copy(b0v.begin(), b0v.end(), bh.begin() + g * mc);
  }
#define EZO_H2D(dst, src, bytes) \
  if (e == cudaSuccess) e = cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice)
  EZO_H2D(b->d_st, b->st0.data(), sizeof(SegState) * B);
  EZO_H2D(b->d_v1, v1, sizeof(double) * B * n);
  EZO_H2D(b->d_v2, v2, sizeof(double) * B * n);
  EZO_H2D(b->d_A, Ah.data(), sizeof(double) * Ah.size());
  EZO_H2D(b->d_b, bh.data(), sizeof(double) * bh.size());
  EZO_H2D(b->d_envs, b->envs.data(), sizeof(EnvDevFull) * n_env);
  EZO_H2D(b->d_path_first, b->path_first.data(), sizeof(int) * B);
  EZO_H2D(b->d_st0, b->st0.data(), sizeof(SegState) * B);
  EZO_H2D(b->d_A0, Ah.data(), sizeof(double) * Ah.size());
  EZO_H2D(b->d_b0, bh.data(), sizeof(double) * bh.size());
#undef EZO_H2D
  if (e == cudaSuccess) e = cudaMemset(b->d_sum, 0, sizeof(RoundSummary));
  if (e == cudaSuccess) e = cudaMemset(b->view.sm_seats, 0, sizeof(int) * kSeatSlots);
  if (e == cudaSuccess) e = cudaMemset(b->view.q_claim, 0, sizeof(int) * (b->claim_cap + 1));
  if (e == cudaSuccess) e = cudaMemset(b->d_flags, 0, (size_t)std::max<long long>(1, b->total_s));
  if (e != cudaSuccess) {
    batch_free_device(b);
    delete b;
    return cuda_fail(e, "ezo_batch_create: upload");
  }
  BatchView& v = b->view;
  v.B = n_seg;
  v.n = n;
  v.m_cap = b->m_cap;
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
  v.st = b->d_st;
  v.v1 = b->d_v1;
  v.v2 = b->d_v2;
  v.A = b->d_A;
  v.b = b->d_b;
  v.S = b->d_S;
  v.flags = b->d_flags;
  v.cand_idx = b->d_cidx;
  v.cstar = b->d_cstar;
  v.dist = b->d_dist;
  v.c32 = b->d_c32;
  v.cnorm = b->d_cn;
  v.bits = b->d_bits;
  v.ga = b->d_ga;
  v.gb = b->d_gb;
  v.placed_idx = b->d_pidx;
  v.placed_delta = b->d_pdelta;
  v.sample_tiles = b->d_stiles;
  v.bisect_tiles = b->d_btiles;
  v.summary = b->d_sum;
  v.robot = robot->d_robot;
  v.envs = b->d_envs;
  v.max_obs_pad = b->max_obs_pad;
  v.max_ebox = b->max_ebox;
  v.n_rbox = robot->n_box;
  v.nsp_pad = robot->nsp_pad;
  v.np_max = b->np_max;
  v.path_first = b->d_path_first;
  v.max_path_len = b->max_path_len;
  v.graph_cond = 0;
  // launch shapes: lanes per configuration from the work per round
  const int sms = sm_count();
  long long tot_np = 0, tot_s1 = 0;
  for (auto& s : b->st0) {
    tot_np += s.n_p;
    tot_s1 += std::max(s.n_p, host_test_size(1, prm->eps, prm->delta, prm->tau));
  }
  // lanes per configuration from the autotuner, at the first round's sample
  // count (labels) and at a quarter of the candidate capacity (bisection)
  int e_big = 0;
  for (int e2 = 1; e2 < n_env; ++e2)
    if (envs[e2]->n_obs > envs[e_big]->n_obs) e_big = e2;
  // the tuner times one flat launch of the round-1 size, but the round
  // kernel's work units and the smaller later rounds favour two lanes per
  // configuration below ~1e6 samples per round (1e5 samples per round, whole
  // inflation: 0.22 ms at 2 lanes, 0.28 at 1, 0.24 at 4, while the flat
  // tuner ranks them within its noise); larger rounds take the tuner's pick
  b->T_check = tot_s1 < (1ll << 20) ? 2 : ezo_internal_tuned_lanes(robot, envs[e_big], tot_s1, nullptr);
  // Bisection runs N_b dependent checks per candidate on the few thousand
  // candidates of a round, so it is latency bound: sixteen lanes per
  // candidate (the wide check; eight in scenes with boxes), unless a round
  // can hold enough candidates to fill the GPU at fewer lanes. Measured on
  // the 7-DOF arm's path (800 to 14,000 candidates a round), 16 lanes beat 8
  // by 5-30% in every round but the largest.
  b->T_bisect = tot_np >= (1ll << 20) ? ezo_internal_tuned_lanes(robot, envs[e_big], tot_np / 4, nullptr)
                                      : ((robot->n_box || b->max_ebox) ? 8 : 16);
  b->T_check = std::max(b->T_check, b->t_min);
  b->T_bisect = std::max(b->T_bisect, b->t_min);
  // walks share eight lanes in rounds with fewer walks than one warp per
  // scheduler would hold at one lane per walk
  b->split_below = (sms * 4 * 32) / kTile;
  b->tot_s1 = tot_s1;
  b->tot_np = tot_np;
  b->sms = sms;
  b->view.n_sm = sms;
  b->grid_sample = std::max(1, std::min(b->max_sample_tiles * 8, sms * 16));
  b->grid_check = std::max(1, std::min(b->max_sample_tiles * b->T_check, sms * 16));
  b->grid_bisect = std::max(1, std::min(b->max_bisect_tiles * b->T_bisect, sms * 16));
  *out = b;
  g_err.clear();
  return EZO_OK;
}

void ezo_batch_free(ezo_batch* b) {
  if (!b) return;
  batch_free_device(b);
  delete b;
}

ezo_status ezo_batch_set_sample_lanes(ezo_batch* b, int32_t lanes) {
  if (!b || !(lanes == 0 || lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8))
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_set_sample_lanes: lanes must be 0, 1, 2, 4 or 8");
  drop_graphs(b);  // the graphs hold the view by value
  b->view.sample_lanes = lanes;
  return EZO_OK;
}

}  // extern "C"

namespace {

void apply_shape(ezo_batch* b, const ezo_shape& sh) {
  b->split_below = sh.sample_fill_tiles;
  b->T_check = sh.check_lanes;
  b->T_bisect = sh.bisect_lanes;
  b->grid_check = std::max(1, std::min(b->max_sample_tiles * b->T_check, b->sms * 16));
  b->grid_bisect = std::max(1, std::min(b->max_bisect_tiles * b->T_bisect, b->sms * 16));
  drop_graphs(b);  // a captured graph holds the old launch shapes
}

int log2_class(long long x) {
  int c = 0;
  while ((1ll << c) < x && c < 48) ++c;
  return c;
}

std::mutex g_shape_mu;
std::map<std::vector<long long>, ezo_shape> g_shape_cache;

}  // namespace

extern "C" {

ezo_status ezo_batch_get_shape(const ezo_batch* b, ezo_shape* sh) {
  if (!b || !sh) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_get_shape: bad argument");
  sh->sample_fill_tiles = b->split_below;
  sh->check_lanes = b->T_check;
  sh->bisect_lanes = b->T_bisect;
  return EZO_OK;
}

ezo_status ezo_batch_set_shape(ezo_batch* b, const ezo_shape* sh) {
  if (!b || !sh) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_set_shape: bad argument");
  auto lanes_ok = [](int t) { return t == 1 || t == 2 || t == 4 || t == 8; };
  const bool bis_ok = lanes_ok(sh->bisect_lanes) || sh->bisect_lanes == 16 || sh->bisect_lanes == 32 ||
                      sh->bisect_lanes == kBisectPairLanes;
  if (sh->sample_fill_tiles < 1 || !lanes_ok(sh->check_lanes) || !bis_ok)
    return fail(EZO_ERR_INVALID_ARG,
                "ezo_batch_set_shape: sample_fill_tiles >= 1, check lanes 1, 2, 4 or 8, bisect lanes 1 to 32");
  if (sh->check_lanes < b->t_min || sh->bisect_lanes < b->t_min)
    return fail(EZO_ERR_INVALID_ARG,
                "ezo_batch_set_shape: fewer lanes than the robot's sphere centres need in shared memory");
  apply_shape(b, *sh);
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_batch_tune(ezo_batch* b, int32_t reps, ezo_shape* chosen, void* stream_v) {
  if (!b || reps < 1) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_tune: bad argument");
  cudaStream_t s = (cudaStream_t)stream_v;
  int dev = 0;
  EZO_CUDA(cudaGetDevice(&dev));
  std::vector<long long> key = {dev, b->n, b->robot->nsp_pad, b->robot->n_self, b->max_obs_pad, b->max_ebox,
                                b->robot->n_box, log2_class(b->tot_s1), log2_class(b->tot_np), log2_class(b->B),
                                b->prm.n_b, b->sur ? 1 : 0};
  ezo_shape best{};
  ezo_batch_get_shape(b, &best);
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_shape_mu);
    auto it = g_shape_cache.find(key);
    if (it != g_shape_cache.end()) {
      best = it->second;
      cached = true;
    }
  }
  if (!cached) {
    cudaEvent_t e0, e1;
    EZO_CUDA(cudaEventCreate(&e0));
    EZO_CUDA(cudaEventCreate(&e1));
    auto time_shape = [&](const ezo_shape& sh, float* out_ms) -> ezo_status {
      apply_shape(b, sh);
      float t = 1e30f;
      for (int r = 0; r < reps + 1; ++r) {  // the first run warms up (module loading, caches)
        ezo_status st = ezo_batch_reset(b, nullptr, nullptr, s);
        if (st != EZO_OK) return st;
        EZO_CUDA(cudaEventRecord(e0, s));
        st = run_host_loop(b, s);
        if (st != EZO_OK) return st;
        EZO_CUDA(cudaEventRecord(e1, s));
        EZO_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        EZO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) t = std::min(t, ms);
      }
      *out_ms = t;
      return EZO_OK;
    };
    // coordinate search: bisection lanes, then label lanes, then the walks'
    // fill threshold, each with the others at their current best
    float best_ms = 1e30f;
    ezo_status st = time_shape(best, &best_ms);
    const int S = (b->sms * 4 * 32) / kTile;
    const int bis[6] = {4, 8, 16, 32, kBisectPairLanes, 2}, chk[4] = {1, 2, 4, 8},
              fill[3] = {std::max(1, S / 2), S, 2 * S};
    for (int stage = 0; stage < 3 && st == EZO_OK; ++stage) {
      const int* cand = stage == 0 ? bis : (stage == 1 ? chk : fill);
      const int nc = stage == 0 ? 6 : (stage == 1 ? 4 : 3);
      for (int i = 0; i < nc && st == EZO_OK; ++i) {
        ezo_shape sh = best;
        if (stage == 0) sh.bisect_lanes = cand[i];
        if (stage == 1) sh.check_lanes = cand[i];
        if (stage == 2) sh.sample_fill_tiles = cand[i];
        if (sh.check_lanes < b->t_min || sh.bisect_lanes < b->t_min) continue;  // does not fit shared memory
        if (sh.bisect_lanes == best.bisect_lanes && sh.check_lanes == best.check_lanes &&
            sh.sample_fill_tiles == best.sample_fill_tiles)
          continue;
        float ms = 0.f;
        st = time_shape(sh, &ms);
        if (st == EZO_OK && ms < 0.98f * best_ms) {  // a clear win only
          best_ms = ms;
          best = sh;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != EZO_OK) return st;
    std::lock_guard<std::mutex> lock(g_shape_mu);
    g_shape_cache[key] = best;
  }
  apply_shape(b, best);
  ezo_status st = ezo_batch_reset(b, nullptr, nullptr, s);
  if (st != EZO_OK) return st;
  EZO_CUDA(cudaStreamSynchronize(s));
  if (chosen) *chosen = best;
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_batch_attach_surrogate(ezo_batch* b, ezo_surrogate* sur, float margin) {
  if (!b) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_attach_surrogate: null batch");
  drop_graphs(b);
  if (!sur) {
    b->sur = nullptr;
    b->view.sbis = 0;
    return EZO_OK;
  }
  if (ezo_internal_surrogate_dof(sur) != b->n || b->n > 8)
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_attach_surrogate: surrogate of another robot, or more than 8 joints");
  const long long rows = (long long)b->max_bisect_tiles * kTile;
  if (rows > b->sur_rows) {
    // the surrogate's brackets and end-point records (the projected rows
    // s_p32 / s_d32 exist from ezo_batch_create on)
    void* ps[] = {b->view.s_lo, b->view.s_hi, b->view.s_bits, b->view.s_ok, b->view.s_rows};
    for (void* p : ps)
      if (p) cudaFree(p);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&b->view.s_lo, rows);
    if (e == cudaSuccess) e = dalloc(&b->view.s_hi, rows);
    if (e == cudaSuccess) e = dalloc(&b->view.s_bits, rows);
    if (e == cudaSuccess) e = dalloc(&b->view.s_ok, rows);
    if (e == cudaSuccess) e = dalloc(&b->view.s_rows, 1);
    if (e != cudaSuccess) return cuda_fail(e, "ezo_batch_attach_surrogate: allocation");
    b->sur_rows = rows;
  }
  b->sur = sur;
  b->view.sbis = 1;
  b->view.sbis_margin = margin;
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_batch_reset(ezo_batch* b, const double* v1, const double* v2, void* stream_v) {
  if (!b) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_reset: null batch");
  cudaStream_t s = (cudaStream_t)stream_v;
  const size_t B = b->B, n = b->n;
  if (v1) EZO_CUDA(cudaMemcpyAsync(b->d_v1, v1, sizeof(double) * B * n, cudaMemcpyHostToDevice, s));
  if (v2) EZO_CUDA(cudaMemcpyAsync(b->d_v2, v2, sizeof(double) * B * n, cudaMemcpyHostToDevice, s));
  // states, starting polytopes and the summary in one kernel (the summary's
  // work-queue fields reset themselves at the end of every launch)
  EZO_CUDA(launch_batch_reset(b->view, b->d_st0, b->d_A0, b->d_b0, s));
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_batch_run(ezo_batch* b, int32_t mode, void* stream) {
  if (!b) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_run: null batch");
  ezo_status st = run_batch(b, mode, (cudaStream_t)stream);
  if (st == EZO_OK) g_err.clear();
  return st;
}

ezo_status ezo_batch_run_path(ezo_batch* b, int32_t sequential, int32_t mode, void* stream_v) {
  if (!b) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_run_path: null batch");
  cudaStream_t s = (cudaStream_t)stream_v;
  const int B = b->B, L = b->max_path_len;
  std::vector<SegState> sts;
  std::vector<uint8_t> contained((size_t)B * L);
  std::vector<int> kept(B, 0);
  if (sequential == 2 && mode == EZO_RUN_GRAPH) {
    // wavefront as one graph launch (build_wave_graph)
    if (!b->wgexec) {
      ezo_status st = build_wave_graph(b);
      if (st != EZO_OK) return st;
    }
    EZO_CUDA(cudaGraphLaunch(b->wgexec, s));
    EZO_CUDA(cudaStreamSynchronize(s));
  } else if (sequential == 2) {
    // wavefront with a host launch loop: each path runs its segments in
    // order with the skip rule; the current segments of all paths share one
    // batched run per wave
    ezo_status st = read_states(b, sts, s);
    if (st != EZO_OK) return st;
    for (int g = 0; g < B; ++g) sts[g].status = SEG_IDLE;
    EZO_CUDA(cudaMemcpyAsync(b->d_st, sts.data(), sizeof(SegState) * B, cudaMemcpyHostToDevice, s));
    std::vector<int> next(B, -1), stopped(B, 0);  // per path (indexed by its first segment)
    for (int g = 0; g < B; ++g)
      if (b->path_first[g] == g) next[g] = g;
    for (int wave = 0; wave <= B; ++wave) {
      EZO_CUDA(cudaMemsetAsync(b->d_contained, 0, (size_t)B * L, s));
      cudaError_t e = launch_containment(b->view, b->d_contained, 1e-9, s);
      if (e != cudaSuccess) return cuda_fail(e, "containment");
      EZO_CUDA(cudaMemcpyAsync(contained.data(), b->d_contained, (size_t)B * L, cudaMemcpyDeviceToHost, s));
      st = read_states(b, sts, s);
      if (st != EZO_OK) return st;
      int active = 0;
      for (int pf = 0; pf < B; ++pf) {
        if (next[pf] < 0 || stopped[pf]) continue;
        int g = next[pf];
        while (g < B && b->path_first[g] == pf) {
          bool skip = false;
          for (int j = pf; j < g && !skip; ++j)
            if (kept[j] && contained[(size_t)g * L + (j - pf)]) skip = true;
          if (!skip) break;
          sts[g].status = SEG_SKIPPED;
          ++g;
        }
        if (g < B && b->path_first[g] == pf) {
          sts[g].status = SEG_ACTIVE;
          kept[g] = 1;
          next[pf] = g + 1;
          ++active;
        } else {
          next[pf] = -1;
        }
      }
      EZO_CUDA(cudaMemcpyAsync(b->d_st, sts.data(), sizeof(SegState) * B, cudaMemcpyHostToDevice, s));
      if (!active) break;
      st = run_batch(b, mode, s);
      if (st != EZO_OK) return st;
      st = read_states(b, sts, s);
      if (st != EZO_OK) return st;
      for (int g = 0; g < B; ++g)
        if (kept[g] && sts[g].status == SEG_IN_COLLISION) stopped[b->path_first[g]] = 1;
    }
    EZO_CUDA(cudaStreamSynchronize(s));
  } else if (sequential) {
    // every segment idle; activate one at a time in path order
    for (int g = 0; g < B; ++g) {
      ezo_status st = set_status(b, g, SEG_IDLE, s);
      if (st != EZO_OK) return st;
    }
    std::vector<int> stopped(B, 0);
    for (int g = 0; g < B; ++g) {
      const int pf = b->path_first[g];
      if (stopped[pf]) continue;
      bool skip = false;
      if (g > pf) {
        EZO_CUDA(cudaMemsetAsync(b->d_contained, 0, (size_t)B * L, s));
        cudaError_t e = launch_containment(b->view, b->d_contained, 1e-9, s);
        if (e != cudaSuccess) return cuda_fail(e, "containment");
        EZO_CUDA(cudaMemcpyAsync(contained.data(), b->d_contained, (size_t)B * L, cudaMemcpyDeviceToHost, s));
        EZO_CUDA(cudaStreamSynchronize(s));
        for (int j = pf; j < g; ++j)
          if (kept[j] && contained[(size_t)g * L + (j - pf)]) skip = true;
      }
      if (skip) {
        ezo_status st = set_status(b, g, SEG_SKIPPED, s);
        if (st != EZO_OK) return st;
        continue;
      }
      ezo_status st = set_status(b, g, SEG_ACTIVE, s);
      if (st != EZO_OK) return st;
      st = run_batch(b, EZO_RUN_HOST_LOOP, s);
      if (st != EZO_OK) return st;
      kept[g] = 1;
      SegState one;
      EZO_CUDA(cudaMemcpyAsync(&one, &b->d_st[g], sizeof(SegState), cudaMemcpyDeviceToHost, s));
      EZO_CUDA(cudaStreamSynchronize(s));
      if (one.status == SEG_IN_COLLISION) stopped[pf] = 1;
    }
    (void)mode;
  } else {
    // every segment at once, then containment and the skip rule on the
    // device, behind the run on the same stream: one synchronisation
    ezo_status st = run_batch(b, mode, s, false);
    if (st != EZO_OK) return st;
    EZO_CUDA(cudaMemsetAsync(b->d_contained, 0, (size_t)B * L, s));
    cudaError_t e = launch_containment(b->view, b->d_contained, 1e-9, s);
    if (e == cudaSuccess) e = launch_path_skip(b->view, b->d_contained, s);
    if (e != cudaSuccess) return cuda_fail(e, "containment and skip rule");
    EZO_CUDA(cudaStreamSynchronize(s));
  }
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_batch_get_segment(const ezo_batch* b, int32_t seg, int32_t* status, int32_t* rounds, int32_t* m,
                                 int32_t* planes, int64_t* checks) {
  if (!b || seg < 0 || seg >= b->B) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_get_segment: bad segment");
  SegState s;
  EZO_CUDA(cudaMemcpy(&s, &b->d_st[seg], sizeof(SegState), cudaMemcpyDeviceToHost));
  if (status) *status = s.status;
  if (rounds) *rounds = s.rounds;
  if (m) *m = s.m;
  if (planes) *planes = s.planes;
  if (checks) *checks = s.checks;
  return EZO_OK;
}

ezo_status ezo_batch_get_polytope(const ezo_batch* b, int32_t seg, int32_t* m, double* A, double* bv) {
  if (!b || seg < 0 || seg >= b->B) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_get_polytope: bad segment");
  SegState s;
  EZO_CUDA(cudaMemcpy(&s, &b->d_st[seg], sizeof(SegState), cudaMemcpyDeviceToHost));
  if (m) *m = s.m;
  if (A) EZO_CUDA(cudaMemcpy(A, b->d_A + (size_t)seg * b->m_cap * b->n, sizeof(double) * s.m * b->n,
                             cudaMemcpyDeviceToHost));
  if (bv) EZO_CUDA(cudaMemcpy(bv, b->d_b + (size_t)seg * b->m_cap, sizeof(double) * s.m, cudaMemcpyDeviceToHost));
  return EZO_OK;
}

ezo_status ezo_batch_get_polytopes(const ezo_batch* b, int32_t* status, int32_t* m, double* A, double* bv,
                                   int32_t rows, int32_t* m_read, void* stream_v) {
  if (!b || !status || !m || rows < 0 || ((A || bv) && rows < 1))
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_get_polytopes: bad argument");
  cudaStream_t s = (cudaStream_t)stream_v;
  std::vector<SegState> sts(b->B);
  const size_t n = b->n, mc = b->m_cap;
  const int all_rows = (int)std::min<size_t>((size_t)rows, mc);
  // small batches: the states and every row the buffers hold in one pass
  // (one synchronisation); large ones read the states first and copy only
  // the rows in use
  const bool one_pass = (A || bv) && (size_t)b->B * all_rows * (n + 1) * sizeof(double) <= (4u << 20);
  auto copy_rows = [&](int r) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (A && r)
      e = cudaMemcpy2DAsync(A, sizeof(double) * rows * n, b->d_A, sizeof(double) * mc * n, sizeof(double) * r * n,
                            b->B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && bv && r)
      e = cudaMemcpy2DAsync(bv, sizeof(double) * rows, b->d_b, sizeof(double) * mc, sizeof(double) * r, b->B,
                            cudaMemcpyDeviceToHost, s);
    return e;
  };
  EZO_CUDA(cudaMemcpyAsync(sts.data(), b->d_st, sizeof(SegState) * b->B, cudaMemcpyDeviceToHost, s));
  if (one_pass) EZO_CUDA(copy_rows(all_rows));
  EZO_CUDA(cudaStreamSynchronize(s));
  int mmax = 0;
  for (int g = 0; g < b->B; ++g) {
    status[g] = sts[g].status;
    m[g] = sts[g].m;
    mmax = std::max(mmax, sts[g].m);
  }
  if (m_read) *m_read = one_pass ? all_rows : mmax;
  if ((A || bv) && mmax > rows) return fail(EZO_ERR_CAPACITY, "ezo_batch_get_polytopes: rows below the largest m");
  if ((A || bv) && !one_pass) {
    EZO_CUDA(copy_rows(mmax));
    EZO_CUDA(cudaStreamSynchronize(s));
  }
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_host_alloc(size_t bytes, void** out) {
  if (!out) return fail(EZO_ERR_INVALID_ARG, "ezo_host_alloc: null output");
  *out = nullptr;
  if (bytes == 0) return EZO_OK;
  EZO_CUDA(cudaMallocHost(out, bytes));
  return EZO_OK;
}

void ezo_host_free(void* p) {
  if (p) cudaFreeHost(p);
}

ezo_status ezo_batch_capacity(const ezo_batch* b, int32_t* m_cap, int32_t* s_cap) {
  if (!b) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_capacity: null batch");
  if (m_cap) *m_cap = b->m_cap;
  if (s_cap) *s_cap = b->s_cap_max;
  return EZO_OK;
}

ezo_status ezo_batch_step(ezo_batch* b, int32_t step, void* stream) {
  if (!b) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_step: null batch");
  return launch_step(b, step, (cudaStream_t)stream);
}

ezo_status ezo_batch_sync(ezo_batch* b, void* stream) {
  if (!b) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_sync: null batch");
  EZO_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  collect_profile(b);
  return EZO_OK;
}

ezo_status ezo_batch_read(const ezo_batch* b, int32_t seg, int32_t what, void* dst, int64_t bytes) {
  if (!b || seg < 0 || seg >= b->B || !dst) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_read: bad argument");
  SegState s;
  EZO_CUDA(cudaMemcpy(&s, &b->d_st[seg], sizeof(SegState), cudaMemcpyDeviceToHost));
  const int n = b->n;
  size_t need = 0;
  const void* src = nullptr;
  switch (what) {
    case 0: need = sizeof(float) * (size_t)n * s.s_cap; src = b->d_S + (size_t)n * s.sample_off; break;
    case 1: need = (size_t)s.s_cap; src = b->d_flags + s.sample_off; break;
    case 2: need = sizeof(int) * (size_t)s.n_p; src = b->d_cidx + s.cand_off; break;
    case 3: need = sizeof(double) * (size_t)n * s.n_p; src = b->d_cstar + (size_t)n * s.cand_off; break;
    case 4: need = sizeof(double) * (size_t)s.n_p; src = b->d_dist + s.cand_off; break;
    case 5: need = sizeof(uint32_t) * (size_t)s.n_p; src = b->d_bits + s.cand_off; break;
    case 6: {
      if (bytes < (int64_t)(12 * sizeof(int32_t))) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_read: buffer too small");
      int32_t* o = (int32_t*)dst;
      const int32_t vals[13] = {s.k, s.status, s.m, s.n_samples, s.m_test, s.count, s.n_cand,
                                s.planes, s.rounds, s.n_placed, s.n_p, s.env, s.s_cap};
      std::memcpy(o, vals, bytes >= (int64_t)sizeof(vals) ? sizeof(vals) : 12 * sizeof(int32_t));
      return EZO_OK;
    }
    case 9: {
      if (bytes < (int64_t)(3 * sizeof(int64_t))) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_read: buffer too small");
      const int64_t vals[3] = {s.checks - s.checks_bisect, s.checks_bisect, s.sample_flops};
      std::memcpy(dst, vals, sizeof(vals));
      return EZO_OK;
    }
    case 11: {
      if (bytes < (int64_t)sizeof(int64_t)) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_read: buffer too small");
      const int64_t val = s.sur_evals;
      std::memcpy(dst, &val, sizeof(val));
      return EZO_OK;
    }
    case 10: {
      // the public part of the summary: active, rounds, sample and bisection tiles
      if (bytes < (int64_t)(4 * sizeof(int32_t))) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_read: buffer too small");
      EZO_CUDA(cudaMemcpy(dst, b->d_sum, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost));
      return EZO_OK;
    }
    case 7: need = sizeof(int) * (size_t)b->prm.n_f; src = b->d_pidx + (size_t)seg * b->prm.n_f; break;
    case 8: need = sizeof(double) * (size_t)b->prm.n_f; src = b->d_pdelta + (size_t)seg * b->prm.n_f; break;
    default: return fail(EZO_ERR_INVALID_ARG, "ezo_batch_read: unknown buffer");
  }
  if (bytes < (int64_t)need) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_read: buffer too small");
  EZO_CUDA(cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost));
  return EZO_OK;
}

ezo_status ezo_batch_write_samples(ezo_batch* b, int32_t seg, const float* samples, int32_t count) {
  if (!b || seg < 0 || seg >= b->B || !samples || count < 0)
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_write_samples: bad argument");
  SegState s;
  EZO_CUDA(cudaMemcpy(&s, &b->d_st[seg], sizeof(SegState), cudaMemcpyDeviceToHost));
  if (count > s.s_cap) return fail(EZO_ERR_CAPACITY, "ezo_batch_write_samples: count exceeds sample capacity");
  for (int j = 0; j < b->n; ++j)
    EZO_CUDA(cudaMemcpy(b->d_S + (size_t)b->n * s.sample_off + (size_t)j * s.s_cap, samples + (size_t)j * count,
                        sizeof(float) * count, cudaMemcpyHostToDevice));
  EZO_CUDA(cudaMemcpy(&b->d_st[seg].n_samples, &count, sizeof(int), cudaMemcpyHostToDevice));
  return EZO_OK;
}

// ------------------------------------------------ recovery (Sec. VI-B) --
ezo_status ezo_batch_set_polytope(ezo_batch* b, int32_t seg, int32_t m, const double* A, const double* bb,
                                  void* stream_v) {
  if (!b || seg < 0 || seg >= b->B || m < 0 || (m > 0 && (!A || !bb)))
    return fail(EZO_ERR_INVALID_ARG, "ezo_batch_set_polytope: bad argument");
  if (m > b->m_cap) return fail(EZO_ERR_CAPACITY, "ezo_batch_set_polytope: more rows than the batch's m_cap");
  cudaStream_t s = (cudaStream_t)stream_v;
  const size_t n = b->n;
  if (m > 0) {
    EZO_CUDA(cudaMemcpyAsync(b->d_A + (size_t)seg * b->m_cap * n, A, sizeof(double) * m * n,
                             cudaMemcpyHostToDevice, s));
    EZO_CUDA(cudaMemcpyAsync(b->d_b + (size_t)seg * b->m_cap, bb, sizeof(double) * m, cudaMemcpyHostToDevice, s));
  }
  EZO_CUDA(cudaMemcpyAsync(&b->d_st[seg].m, &m, sizeof(int), cudaMemcpyHostToDevice, s));
  const int no_box = 0;  // rows 0..2n-1 are no longer known to be the joint box
  EZO_CUDA(cudaMemcpyAsync(&b->d_st[seg].box_rows, &no_box, sizeof(int), cudaMemcpyHostToDevice, s));
  EZO_CUDA(cudaStreamSynchronize(s));
  return EZO_OK;
}

ezo_status ezo_batch_edit(ezo_batch* b, int64_t n_cfg, const double* cfg, void* stream_v) {
  if (!b || n_cfg < 0 || (n_cfg > 0 && !cfg)) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_edit: bad argument");
  cudaStream_t s = (cudaStream_t)stream_v;
  std::vector<SegState> sts;
  ezo_status st = read_states(b, sts, s);
  if (st != EZO_OK) return st;
  std::vector<int> targets;
  for (int g = 0; g < b->B; ++g) {
    if (sts[g].status == SEG_ACTIVE) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_edit: the batch is still running");
    if (sts[g].status == SEG_ACCEPTED || sts[g].status == SEG_MAX_ITER) {
      if (n_cfg > sts[g].s_cap) return fail(EZO_ERR_CAPACITY, "ezo_batch_edit: more configurations than samples fit");
      targets.push_back(g);
    }
  }
  if (targets.empty() || n_cfg == 0) {
    g_err.clear();
    return EZO_OK;
  }
  const size_t n = b->n, N = (size_t)n_cfg;
  std::vector<float> soa(n * N);
  for (size_t i = 0; i < N; ++i)
    for (size_t j = 0; j < n; ++j) soa[j * N + i] = (float)cfg[i * n + j];
  std::vector<SegState> saved = sts;
  for (int g : targets) {
    EZO_CUDA(cudaMemcpy2DAsync(b->d_S + n * (size_t)sts[g].sample_off, sizeof(float) * (size_t)sts[g].s_cap,
                               soa.data(), sizeof(float) * N, sizeof(float) * N, n, cudaMemcpyHostToDevice, s));
    sts[g].status = SEG_ACTIVE;
    sts[g].n_samples = (int)n_cfg;
  }
  EZO_CUDA(cudaMemcpyAsync(b->d_st, sts.data(), sizeof(SegState) * b->B, cudaMemcpyHostToDevice, s));
  EZO_CUDA(cudaMemsetAsync(b->d_sum, 0, sizeof(RoundSummary), s));
  b->view.edit = 1;
  const int steps[5] = {0, 2, 3, 4, 5};  // round size, labels, selection, bisection, placement
  for (int k = 0; k < 5 && st == EZO_OK; ++k) st = launch_step(b, steps[k], s);
  b->view.edit = 0;
  if (st != EZO_OK) return st;
  st = read_states(b, sts, s);
  collect_profile(b);
  if (st != EZO_OK) return st;
  for (int g : targets)
    if (sts[g].status == SEG_ACTIVE) sts[g].status = saved[g].status;  // else in collision (t_col) or full
  EZO_CUDA(cudaMemcpyAsync(b->d_st, sts.data(), sizeof(SegState) * b->B, cudaMemcpyHostToDevice, s));
  EZO_CUDA(cudaStreamSynchronize(s));
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_batch_coverage(ezo_batch* b, uint8_t* covered, void* stream_v) {
  if (!b || !covered) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_coverage: bad argument");
  cudaStream_t s = (cudaStream_t)stream_v;
  EZO_CUDA(cudaMemsetAsync(b->d_contained, 0, (size_t)b->B, s));
  cudaError_t e = launch_coverage(b->view, b->d_contained, 1e-9, s);
  if (e != cudaSuccess) return cuda_fail(e, "coverage");
  EZO_CUDA(cudaMemcpyAsync(covered, b->d_contained, (size_t)b->B, cudaMemcpyDeviceToHost, s));
  EZO_CUDA(cudaStreamSynchronize(s));
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_batch_reinflate(ezo_batch* b, const uint8_t* which, int32_t mode, void* stream_v) {
  if (!b || !which) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_reinflate: bad argument");
  cudaStream_t s = (cudaStream_t)stream_v;
  std::vector<SegState> sts;
  ezo_status st = read_states(b, sts, s);
  if (st != EZO_OK) return st;
  const size_t n = b->n, mc = b->m_cap;
  int any = 0;
  for (int g = 0; g < b->B; ++g) {
    if (sts[g].status == SEG_ACTIVE) return fail(EZO_ERR_INVALID_ARG, "ezo_batch_reinflate: the batch is still running");
    if (!which[g]) continue;
    // back to round 1 with P = D, keeping the counters of earlier runs
    SegState r = b->st0[g];
    r.checks = sts[g].checks;
    r.checks_bisect = sts[g].checks_bisect;
    r.sur_evals = sts[g].sur_evals;
    r.sample_flops = sts[g].sample_flops;
    r.planes = 0;
    sts[g] = r;
    EZO_CUDA(cudaMemcpyAsync(b->d_A + g * mc * n, b->d_A0 + g * mc * n, sizeof(double) * mc * n,
                             cudaMemcpyDeviceToDevice, s));
    EZO_CUDA(cudaMemcpyAsync(b->d_b + g * mc, b->d_b0 + g * mc, sizeof(double) * mc, cudaMemcpyDeviceToDevice, s));
    any = 1;
  }
  if (!any) {
    g_err.clear();
    return EZO_OK;
  }
  EZO_CUDA(cudaMemcpyAsync(b->d_st, sts.data(), sizeof(SegState) * b->B, cudaMemcpyHostToDevice, s));
  EZO_CUDA(cudaMemsetAsync(b->d_sum, 0, sizeof(RoundSummary), s));
  st = run_batch(b, mode, s);
  if (st == EZO_OK) g_err.clear();
  return st;
}

ezo_status ezo_path_points(const double* verts, int32_t n_verts, int32_t n, double step, int64_t* edge_points,
                           int64_t* total) {
  if (!total || n_verts < 0 || n < 1 || n > EZO_MAX_DOF || (n_verts > 0 && !verts) || !(step > 0.0) ||
      !std::isfinite(step))
    return fail(EZO_ERR_INVALID_ARG, "ezo_path_points: bad argument");
  long long tot = 0;
  for (int k = 0; k + 1 < n_verts; ++k) {
    double ss = 0.0;
    for (int j = 0; j < n; ++j) {
      const double e = verts[(size_t)(k + 1) * n + j] - verts[(size_t)k * n + j];
      ss += e * e;
    }
    const double q = std::ceil(std::sqrt(ss) / step);
    if (!std::isfinite(q) || q > 1e12) return fail(EZO_ERR_INVALID_ARG, "ezo_path_points: non-finite or huge edge");
    const long long pts = std::max(1ll, (long long)q) + 1;
    if (edge_points) edge_points[k] = pts;
    tot += pts;
  }
  *total = tot;
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_check_path(const ezo_robot* robot, const ezo_env* env, const double* verts, int32_t n_verts,
                          double step, uint8_t* edge_flags, uint8_t* point_flags_dev, int64_t point_cap,
                          int64_t* n_points, void* stream_v) {
  if (!robot || !env || (n_verts > 1 && !edge_flags))
    return fail(EZO_ERR_INVALID_ARG, "ezo_check_path: bad argument");
  cudaStream_t s = (cudaStream_t)stream_v;
  const int K = std::max(0, n_verts - 1), n = robot->n;
  std::vector<int64_t> cnt((size_t)std::max(K, 1));
  std::vector<long long> off((size_t)K + 1, 0);
  int64_t N = 0;
  ezo_status st = ezo_path_points(verts, n_verts, n, step, cnt.data(), &N);
  if (st != EZO_OK) return st;
  if (n_points) *n_points = N;
  if (point_flags_dev && point_cap < N) return fail(EZO_ERR_CAPACITY, "ezo_check_path: point_cap < points");
  if (check_smem_bytes(robot->nsp_pad, env->n_obs_pad, 128, 8, robot->n_box, env->n_box) > kSmemBudget)
    return fail(EZO_ERR_INVALID_ARG, "ezo_check_path: robot and obstacle spheres exceed shared memory");
  if (K == 0) {
    g_err.clear();
    return EZO_OK;
  }
  for (int k = 0; k < K; ++k) off[k + 1] = off[k] + cnt[k];
  // one scratch block: vertices (FP64), edge offsets, edge flags
  const size_t vb = sizeof(double) * (size_t)n_verts * n, ob = sizeof(long long) * (size_t)(K + 1);
  char* scratch = nullptr;
  EZO_CUDA(cudaMallocAsync((void**)&scratch, vb + ob + (size_t)K, s));
  double* d_verts = (double*)scratch;
  long long* d_off = (long long*)(scratch + vb);
  uint8_t* d_edge = (uint8_t*)(scratch + vb + ob);
  cudaError_t e = cudaMemcpyAsync(d_verts, verts, vb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), ob, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_edge, 0, (size_t)K, s);
  if (e == cudaSuccess) {
    const int lanes = ezo_internal_tuned_lanes(robot, env, N, s);
    e = launch_check_path(robot->d_robot, n, robot->nsp_pad, robot->n_box, env->dev_for(robot), band_E(robot, env), d_verts, K, d_off, N,
                          point_flags_dev, d_edge, lanes, sm_count() * 32, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(edge_flags, d_edge, (size_t)K, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "ezo_check_path");
  g_err.clear();
  return EZO_OK;
}

ezo_status ezo_profile_enable(int32_t on) {
  g_prof_on = on != 0;
  return EZO_OK;
}

ezo_status ezo_profile_reset(void) {
  for (int i = 0; i < kKinds; ++i) {
    g_prof_ms[i] = 0.0;
    g_prof_n[i] = 0;
  }
  return EZO_OK;
}

ezo_status ezo_profile_read(double* ms, int64_t* launches, int32_t n_kinds) {
  for (int i = 0; i < n_kinds && i < kKinds; ++i) {
    if (ms) ms[i] = g_prof_ms[i];
    if (launches) launches[i] = g_prof_n[i];
  }
  return EZO_OK;
}

}  // extern "C"
