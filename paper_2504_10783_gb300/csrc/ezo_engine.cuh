// Shared declarations of the EI-ZO engine: per-segment device state, the
// batch layout and the kernel launchers (Algorithm 1 of arXiv 2504.10783,
// one kernel per step, batched over segments).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ezo_device.cuh"

namespace ezo {

enum SegStatus : int {
  SEG_ACTIVE = 0,
  SEG_ACCEPTED = 1,
  SEG_IN_COLLISION = 2,  // t_col triggered (Sec. IV-C)
  SEG_CAPACITY = 3,
  SEG_MAX_ITER = 6,      // N_it reached (Sec. IV-C), guarantee void
  SEG_IDLE = 7,          // not (yet) scheduled in this batch
  SEG_SKIPPED = 8,       // contained in an earlier polytope (Sec. VI-A)
};

constexpr int kTile = 128;  // samples / candidates per work tile
constexpr int kSeatSlots = 1024;  // bound on the SM ids of a device (work-queue seats)
// bisect_lanes value of the two-halvings-at-a-time bisection (three warps,
// 96 lanes, per candidate)
constexpr int kBisectPairLanes = 96;
// threads per block of the one-thread-per-candidate bisection kernels: small
// blocks spread their FP64 work (1/64 of the FP32 rate) over many SMs
constexpr int kRowBlock = 64;
inline int row_grid(long long rows) {
  const long long g = (rows + kRowBlock - 1) / kRowBlock;
  return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

struct SegState {
  int k;          // current round (1-based)
  int status;     // SegStatus
  int m;          // rows of A in use
  int n_samples;  // |S| of the current round
  int m_test;     // M of the current round
  int count;      // collisions among the first M samples
  int n_cand;     // candidates selected this round (<= N_p)
  int planes;     // hyperplanes added so far
  int rounds;     // rounds run
  int n_placed;   // planes added in the last round
  int n_p;        // N_p of this segment
  int env;        // obstacle set
  uint32_t stream;  // Philox stream id (counter word 3)
  int box_rows;     // 2n when rows 0..2n-1 are the joint box (+e_j <= hi_j, then -e_j <= -lo_j), else 0
  long long checks;      // exact collision checks so far
  long long sample_off;  // first sample slot of this segment
  long long cand_off;    // first candidate slot
  int s_cap;             // sample capacity
  int pad1;
  long long checks_bisect;  // of which at bisection midpoints
  long long sur_evals;      // surrogate evaluations (surrogate-guided bisection)
  long long sample_flops;   // algorithmic FP32 work of the hit-and-run walks so far
};

struct EnvDevFull {
  EnvDev e;
  float E;  // rounding band of the fast pair test for this robot/env
  float pad;
};

struct RoundSummary {
  int active;
  int round;
  int n_sample_tiles;
  int n_bisect_tiles;
  // work queues of the sampling, label and bisection launches (one per
  // bisection mode): units taken so far and blocks that have left; the last
  // block of a launch to leave resets both for the next launch
  int q_sample, left_sample;
  int q_check, left_check;
  int q_bisect[3], left_bisect[3];
  int left_place;  // placement blocks done (the fused round close)
};

// Everything a round kernel needs, by value (kernel parameter space).
struct BatchView {
  int B;      // segments
  int n;      // DOF
  int m_cap;  // row capacity per segment
  int n_f, n_b, n_mix, n_it_max;
  double eps, delta, tau, step_back_max, t_col;
  uint32_t key0, key1;
  PhiloxKeys keys;  // round keys of the seed (key0, key1)
  SegState* st;
  const double* v1;  // [B][n]
  const double* v2;  // [B][n]
  double* A;         // [B][m_cap][n]
  double* b;         // [B][m_cap]
  float* S;          // samples: segment g at S + n*sample_off, [n][s_cap]
  uint8_t* flags;    // [sample_off + i]
  int* cand_idx;     // [cand_off + c]
  double* cstar;     // [n*cand_off + d*n_p + c]
  double* dist;      // [cand_off + c]
  float* c32;        // [n*cand_off + d*n_p + c]
  float* cnorm;      // [cand_off + c]
  uint32_t* bits;    // [cand_off + c]
  double* ga;        // plane normal grad dist_L(c*): [n*cand_off + d*n_p + c]
  double* gb;        // plane offset a^T c*: [cand_off + c]
  int* placed_idx;   // [B][n_f]   candidate index of each plane of the last round
  double* placed_delta;  // [B][n_f]
  int2* sample_tiles;    // (segment, first sample)
  int2* bisect_tiles;    // (segment, first candidate)
  RoundSummary* summary;
  const RobotDev* robot;
  const EnvDevFull* envs;
  int check_projection;  // fail fast: check c_proj before bisecting (Sec. IV-C)
  int max_obs_pad;       // largest padded obstacle count over the batch's envs
  int nsp_pad;           // padded sphere count of the robot
  int np_max;            // largest N_p over the batch
  const int* path_first; // first segment of the path each segment belongs to
  int max_path_len;
  int pad;
  unsigned long long graph_cond;  // cudaGraphConditionalHandle (0 = none)
  // surrogate-guided bisection (0 = exact bisection only)
  int sbis;          // 1 when a surrogate is attached
  int bis_mode;      // bisection kernel mode: 0 exact, 1 verify surrogate end point, 2 exact for fallbacks
  float sbis_margin; // predicted collision iff sd_hat < margin
  int n_rbox;        // robot boxes
  int max_ebox;      // largest obstacle box count over the environments
  int sample_lanes;  // lanes per hit-and-run walk: 0 = chosen per round from the tile count, else 1, 2, 4 or 8
  int edit;          // set editing (Sec. VI-B): the samples are given configurations, no test
  float* s_p32;      // [row * s_ld + j] projection c_proj of the candidate onto L (FP32)
  float* s_d32;      // [row * s_ld + j] c - c_proj (FP32)
  int s_ld;          // row stride of s_p32 and s_d32: 8 for n <= 8 (the MLP's input), else EZO_MAX_DOF
  float* s_lo;       // [row] bracket (fractions along [c_proj, c])
  float* s_hi;
  uint32_t* s_bits;  // [row] surrogate decisions
  uint8_t* s_ok;     // [row] 1 when the surrogate end point was verified in collision
  int* s_rows;       // device row count of this round (n_bisect_tiles * kTile)
  // work-queue seats: working blocks per SM in the current launch
  // ([kSeatSlots], indexed by the SM id; zero between launches)
  int* sm_seats;
  int* q_claim;      // [1 + q_claim_cap]: launch count, then the epoch that claimed each work unit
  int q_claim_cap;   // work units of the largest launch
  int n_sm;          // SMs of the device
};

// Launchers (ezo_kernels.cu). T = lanes per configuration.
cudaError_t launch_check_flat(const RobotDev* robot, int n, int nsp_pad, int n_rbox, const EnvDev& env, float E,
                              const float* q, long long ldq, long long N, uint8_t* flags, int T, int grid_cap,
                              cudaStream_t s);
// signed distance, exact below cap (3e38: exact everywhere)
cudaError_t launch_sd_flat(const RobotDev* robot, int n, int nsp_pad, const EnvDev& env, const float* q, long long ldq,
                           long long N, float* sd, cudaStream_t s, float cap = 3.0e38f);
cudaError_t launch_sample_flat(const double* A, const double* b, int m, int lda, int n, const double* v1h,
                               const double* v2h, long long N, int n_mix, uint64_t seed, uint32_t stream, int k,
                               float* out, long long ldo, cudaStream_t s);

cudaError_t launch_round_begin(const BatchView& v, cudaStream_t s);
// a batch's reset to its initial states and polytopes in one launch
cudaError_t launch_batch_reset(const BatchView& v, const SegState* st0, const double* A0, const double* b0,
                               cudaStream_t s);
// Walks share eight lanes when the round has fewer than split_below_tiles
// sample tiles (0: never).
cudaError_t launch_round_sample(const BatchView& v, int split_below_tiles, int grid, cudaStream_t s);
cudaError_t launch_round_check(const BatchView& v, int T, int grid, cudaStream_t s);
cudaError_t launch_round_certify(const BatchView& v, cudaStream_t s);
// Bisection (ezo_k_round_b.cu): prep projects every candidate row (and, with
// a surrogate attached, resets its brackets), round_bisect takes the halvings
// (bis_mode 0), checks the surrogate end points (1) or redoes the failed ones
// (2), finish forms c*, its distance and the tangent plane; bisect_exact is
// prep + halvings + finish. grid_rows: row_grid(rows) for the batch's
// largest candidate row count.
cudaError_t launch_bisect_prep(const BatchView& v, int grid_rows, cudaStream_t s);
cudaError_t launch_round_bisect(const BatchView& v, int T, int grid, cudaStream_t s);
cudaError_t launch_bisect_finish(const BatchView& v, int grid_rows, cudaStream_t s);
cudaError_t launch_bisect_exact(const BatchView& v, int T, int grid, int grid_rows, cudaStream_t s);
// close = true: the last block also closes the round (the run loops' form)
cudaError_t launch_round_place(const BatchView& v, cudaStream_t s, bool close = false);
cudaError_t launch_round_end(const BatchView& v, cudaStream_t s);

// Containment of segment endpoints in earlier polytopes of the same path
// (Sec. VI-A): contained[k*max_path_len + d] = 1 iff both endpoints of
// segment k satisfy A_j x <= b_j + tol for j = path_first[k] + d < k.
cudaError_t launch_containment(const BatchView& v, uint8_t* contained, double tol, cudaStream_t s);
// the skip rule after a speculative run, from the containment flags
cudaError_t launch_path_skip(const BatchView& v, const uint8_t* contained, cudaStream_t s);
// the wavefront order on the device (one wave graph): statuses and per-path
// wave state reset, then per wave the skip rule and the next segment of
// every path, which also sets the waves' and the rounds' WHILE conditions
cudaError_t launch_wave_init(const BatchView& v, int* w_next, int* w_last, uint8_t* w_kept, cudaStream_t s);
cudaError_t launch_wave_select(const BatchView& v, const uint8_t* contained, int* w_next, int* w_last,
                               uint8_t* w_kept, unsigned long long cond_waves, unsigned long long cond_rounds,
                               cudaStream_t s);
// round end fused with the next round's sizing (the run loops' last kernel)
cudaError_t launch_round_close(const BatchView& v, cudaStream_t s);
// recovery (Sec. VI-B)
cudaError_t launch_check_path(const RobotDev* robot, int n, int nsp_pad, int n_rbox, const EnvDev& env, float E,
                              const double* verts, int n_edges, const long long* off, long long N,
                              uint8_t* point_flags, uint8_t* edge_flags, int T, int grid_cap, cudaStream_t s);
cudaError_t launch_coverage(const BatchView& v, uint8_t* covered, double tol, cudaStream_t s);
// the same collision launchers for scenes with box geometries (compiled in
// separate translation units so that the sphere-only kernels stay lean)
cudaError_t launch_check_flat_box(const RobotDev* robot, int n, int nsp_pad, int n_rbox, const EnvDev& env, float E,
                                  const float* q, long long ldq, long long N, uint8_t* flags, int T, int grid_cap,
                                  cudaStream_t s);
cudaError_t launch_check_path_box(const RobotDev* robot, int n, int nsp_pad, int n_rbox, const EnvDev& env, float E,
                                  const double* verts, int n_edges, const long long* off, long long N,
                                  uint8_t* point_flags, uint8_t* edge_flags, int T, int grid_cap, cudaStream_t s);
cudaError_t launch_round_check_box(const BatchView& v, int T, int grid, cudaStream_t s);
cudaError_t launch_round_bisect_box(const BatchView& v, int T, int grid, cudaStream_t s);

cudaError_t launch_fk_centres(const RobotDev* robot, const RobotFK64* r64, int n, int nsp_pad, const float* q,
                              long long ldq, long long N, int mode, double* out_c, float* err, cudaStream_t s);
size_t check_smem_bytes(int n_spheres_pad, int n_obs_pad, int threads, int T, int n_rbox = 0, int n_ebox = 0);
// Dynamic shared memory a collision kernel may request: the opt-in maximum
// per block (227 KB) less the static robot image and a margin. The sphere
// centres take (spheres + 1) x 16 bytes per group of lanes, so more lanes per
// configuration need less.
constexpr size_t kSmemBudget = 220 * 1024;

}  // namespace ezo
