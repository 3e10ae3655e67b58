/*
 * ezo.h - C ABI of libezo.so: GPU edge inflation (EI-ZO) of collision-free
 * configuration-space segments into probabilistically collision-free
 * H-polytopes, after "Superfast Configuration-Space Convex Set Computation on
 * GPUs for Online Motion Planning" (arXiv 2504.10783).
 *
 * Conventions shared by every entry point:
 *  - Host pointers (suffix-free) are read during the call and never kept; the
 *    caller owns them. Device pointers carry the suffix `_dev`; the caller
 *    owns them too and they must stay valid until the work queued on
 *    `cuda_stream` has finished.
 *  - `cuda_stream` is a cudaStream_t passed as void*; NULL is the legacy
 *    default stream.
 *  - Opaque handles are created and freed by the library; a handle's device
 *    memory is allocated with cudaMalloc at creation and freed by its *_free.
 *  - Every call returns an ezo_status. EZO_OK is 0. On an error the call has
 *    no effect on its outputs unless stated, and ezo_last_error() returns a
 *    message for the calling thread. No C++ exception crosses this ABI.
 *  - Configurations on the device are FP32 in dimension-major layout: value j
 *    of configuration i is q[j * ldq + i] (ldq >= N).
 *  - Polytopes are FP64, row-major: row r of A is A[r * n .. r * n + n - 1],
 *    and P = { x : A x <= b }.
 */
#ifndef EZO_H
#define EZO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EZO_OK = 0,
  EZO_ERR_INVALID_ARG = 1,
  /* Sec. IV-C: a candidate collision lies within t_col of the segment; the
   * segment is likely in collision and no region is built. */
  EZO_ERR_SEGMENT_IN_COLLISION = 2,
  EZO_ERR_CAPACITY = 3,
  EZO_ERR_TIMEOUT = 4,
  EZO_ERR_CUDA = 5,
  /* Sec. IV-C "Maximum iterations": N_it rounds ran without the test
   * accepting; the polytope is returned but carries no guarantee. */
  EZO_WARN_MAX_ITER = 6
} ezo_status;

/* Per-segment outcome codes reported by ezo_batch_get_segment. */
typedef enum {
  EZO_SEG_ACTIVE = 0,
  EZO_SEG_ACCEPTED = 1,
  EZO_SEG_IN_COLLISION = 2,
  EZO_SEG_CAPACITY = 3,
  EZO_SEG_MAX_ITER = 6,
  EZO_SEG_IDLE = 7,
  EZO_SEG_SKIPPED = 8
} ezo_segment_status;

/* Parameters of Algorithm 1 (Sec. IV-B, IV-C; parameter tables of the
 * appendix). eps: admissible fraction in collision; delta: admissible
 * uncertainty; tau: decision threshold of the unadaptive test (0 < tau < 1,
 * the paper uses 0.5); step_back_max: Delta_max; t_col: collision tolerance
 * of the fail-fast rule; n_p: samples to update (N_p); n_f: maximum faces per
 * iteration (N_f); n_b: bisection steps (N_b); n_mix: hit-and-run mixing
 * steps (N_ms); n_it_max: iteration cap (N_it); seed: Philox key. */
typedef struct {
  double eps;
  double delta;
  double tau;
  double step_back_max;
  double t_col;
  int32_t n_p;
  int32_t n_f;
  int32_t n_b;
  int32_t n_mix;
  int32_t n_it_max;
  int32_t reserved0;
  uint64_t seed;
} ezo_params;

/* Fills `p` with eps = delta = 0.05, tau = 0.5, Delta_max = 0.01,
 * t_col = 1e-3, N_p = 10000, N_f = 10, N_b = 10, N_ms = 60, N_it = 50, seed 1. */
void ezo_params_default(ezo_params* p);

typedef struct ezo_robot ezo_robot;
typedef struct ezo_env ezo_env;
typedef struct ezo_batch ezo_batch;

/* Thread-local description of the last error of this thread ("" if none). */
const char* ezo_last_error(void);

/* ------------------------------------------------------------------ robot --
 * Robot description the paper assumes (Sec. II: kinematics and collision
 * geometry, as in a URDF), restricted to a serial chain in standard DH form
 * with sphere geometries here and oriented boxes added by
 * ezo_robot_add_boxes (Sec. IV-D: sphere and box geometries). Frame 0 is the
 * base; frame i (1..n) is
 *   T_i = T_{i-1} Rz(q_i + theta_off_i) Tz(d_i) Tx(a_i) Rx(alpha_i)
 * for a revolute joint and
 *   T_i = T_{i-1} Rz(theta_off_i) Tz(d_i + q_i) Tx(a_i) Rx(alpha_i)
 * for a prismatic one (joint_type[i-1] = 1; joint_type NULL = all revolute;
 * two prismatic joints make the point robot of the Forest benchmark, Sec. V).
 * n <= 16 joints. Sphere s (n_spheres <= 256) sits at sphere_xyz[3s..3s+2] in
 * frame sphere_frame[s] (0..n) with radius sphere_r[s] >= 0. self_pairs holds
 * n_self_pairs pairs (i, j) of sphere indices tested against each other
 * (n_self_pairs <= 65535). q_lo/q_hi are the joint limits (the usual domain
 * D). All arrays are host FP64 (int32 for indices), copied at creation.
 * Errors: EZO_ERR_INVALID_ARG for sizes out of range or bad indices;
 * EZO_ERR_CUDA if device memory cannot be allocated. */
ezo_status ezo_robot_create(int32_t n, const double* a, const double* alpha, const double* d,
                            const double* theta_off, const double* q_lo, const double* q_hi,
                            int32_t n_spheres, const int32_t* sphere_frame, const double* sphere_xyz,
                            const double* sphere_r, int32_t n_self_pairs, const int32_t* self_pairs,
                            const int32_t* joint_type, ezo_robot** out);

/* Oriented boxes fixed to the robot's frames (Sec. IV-D: the checker supports
 * box and sphere geometries; Sec. VII: an arm described by 11 boxes). Box k
 * (n_box <= 32) sits in frame box_frame[k] (0..n) with centre box_xyz[3k..],
 * rotation box_rot[9k..] (3 x 3 row major; its columns are the box axes in the
 * frame) and half extents box_half[3k..] >= 0. sb_pairs lists n_sb self pairs
 * (sphere index, box index), bb_pairs n_bb pairs (box, box). A box overlaps
 * an obstacle sphere or a robot sphere when the sphere centre is strictly
 * inside it or closer than the radius; two boxes overlap when none of the 15
 * separating-axis candidates separates them (cross products of edges within
 * ~0.6 degrees of parallel, |a x b|^2 < 1e-4, are left out). Replaces boxes
 * added before; call before the robot is used. Host arrays, copied.
 * EZO_ERR_INVALID_ARG for counts or indices out of range. */
ezo_status ezo_robot_add_boxes(ezo_robot* robot, int32_t n_box, const int32_t* box_frame, const double* box_xyz,
                               const double* box_rot, const double* box_half, int32_t n_sb, const int32_t* sb_pairs,
                               int32_t n_bb, const int32_t* bb_pairs);
void ezo_robot_free(ezo_robot* robot);
int32_t ezo_robot_dof(const ezo_robot* robot);

/* -------------------------------------------------------------- obstacles --
 * Obstacle spheres (Sec. V-B: perceived voxels become circumscribing
 * spheres): n_obs rows (x, y, z, radius) of host FP64, n_obs <= 4096.
 * Errors: EZO_ERR_INVALID_ARG, EZO_ERR_CUDA. */
ezo_status ezo_env_create(int32_t n_obs, const double* xyzr, ezo_env** out);
/* Oriented obstacle boxes (at most 64): one row of 15 doubles per box,
 * centre (3), half extents (3), rotation (9, row major, columns = box axes in
 * the world). Replaces boxes added before; call before the env is used. The
 * signed-distance call and surrogate training take sphere geometries only and
 * return EZO_ERR_INVALID_ARG when boxes are present. */
ezo_status ezo_env_add_boxes(ezo_env* env, int32_t n_box, const double* boxes);
void ezo_env_free(ezo_env* env);

/* ------------------------------------------------------ collision checker --
 * The collision checker of Sec. IV-D: forward kinematics of each FP32
 * configuration q_dev (n x N, dimension-major, stride ldq) and a test of
 * every robot sphere against every obstacle sphere and of every listed self
 * pair; flags_dev[i] = 1 iff some pair overlaps (squared centre distance
 * below the squared sum of radii), else 0. Robot spheres on the fixed base
 * frame have the same centre for every configuration: when they all clear
 * every obstacle sphere by more than 1e-4 m (checked on the host at each
 * call) their obstacle pairs are not swept again; the flags are the same.
 * Stream-ordered, asynchronous.
 * lanes_per_config selects 1, 2, 4 or 8 cooperating lanes per configuration
 * (0 = choose from N, among the counts that fit). Each group of lanes keeps
 * its sphere centres in shared memory, so large robots with many obstacles
 * need more lanes: at the maximum sizes (256 spheres, 4096 obstacles) only 4
 * and 8 fit. Errors: EZO_ERR_INVALID_ARG (null handle, N < 0, ldq < N, bad
 * lanes value, spheres and obstacles beyond shared memory at that lanes
 * value; nothing is launched), EZO_ERR_CUDA (launch failure). */
ezo_status ezo_check_collision(const ezo_robot* robot, const ezo_env* env, const float* q_dev, int64_t N,
                               int64_t ldq, uint8_t* flags_dev, int32_t lanes_per_config, void* cuda_stream);

/* Signed distance per configuration: min over the same pairs of
 * ||c_i - c_j|| - r_i - r_j in FP32 (negative iff in collision). Used to
 * label data and to bound ambiguous decisions. Stream-ordered.
 * EZO_ERR_INVALID_ARG when the robot or env has boxes, or when its spheres
 * and obstacles exceed the kernel's shared memory (one lane per
 * configuration: (spheres + 1) x 64 centres plus the obstacles). */
ezo_status ezo_signed_distance(const ezo_robot* robot, const ezo_env* env, const float* q_dev, int64_t N,
                               int64_t ldq, float* sd_dev, void* cuda_stream);

/* Forward kinematics of the collision checker against FP64 (Sec. II, the
 * robot's kinematic chain; Sec. IV-D, the checker that places the collision
 * spheres). The checker computes the sphere centres in FP32 from the FP32
 * configuration and FP32 copies of the chain's constants; the reference is
 * the same chain in FP64 from the FP64 constants given to ezo_robot_create,
 * on the same configuration widened to FP64.
 * ezo_sphere_centres writes the centres of the N configurations q_dev (n x N,
 * stride ldq) to out_dev (device FP64, 3 * n_spheres * N values): coordinate
 * c of sphere s of configuration i at out_dev[(3 s + c) * N + i], spheres in
 * the order of their frames (stable in the caller's order within a frame);
 * fp64 = 0 gives the checker's FP32 centres, fp64 = 1 the FP64 ones.
 * ezo_fk_error writes err_dev[i] (device FP32, N values) = the largest
 * distance in metres between a sphere's FP32 and FP64 centre for
 * configuration i. Box geometries are not included. Stream-ordered.
 * Errors: EZO_ERR_INVALID_ARG (null handle or buffer, N < 0, ldq < N, fp64
 * not 0 or 1), EZO_ERR_CUDA. */
ezo_status ezo_sphere_centres(const ezo_robot* robot, const float* q_dev, int64_t N, int64_t ldq, int32_t fp64,
                              double* out_dev, void* cuda_stream);
ezo_status ezo_fk_error(const ezo_robot* robot, const float* q_dev, int64_t N, int64_t ldq, float* err_dev,
                        void* cuda_stream);

/* ------------------------------------------------------------- hit-and-run --
 * UniformSample of Algorithm 1 (Sec. IV-B, IV-D): N independent hit-and-run
 * walks of n_mix steps inside P = {x : A x <= b}, one walk per output
 * sample, started on the segment v1..v2 (host FP64, n values each). A_dev is
 * FP64 m x n with row stride lda, b_dev FP64 m (both device). Walk i draws
 * Philox4x32-10 blocks with counter (i, draw, round_k, stream_id) and key
 * (seed low 32 bits, seed high 32 bits). Output x_dev: FP32, n x N,
 * dimension-major with stride ldx. Stream-ordered. m <= 2048 (the FP32
 * copy of A is staged in shared memory).
 * Errors: EZO_ERR_INVALID_ARG, EZO_ERR_CUDA. */
ezo_status ezo_hit_and_run(const double* A_dev, const double* b_dev, int32_t m, int32_t n, int32_t lda,
                           const double* v1, const double* v2, int64_t N, int32_t n_mix, uint64_t seed,
                           uint32_t stream_id, int32_t round_k, float* x_dev, int64_t ldx, void* cuda_stream);

/* ------------------------------------------------------------------ batch --
 * A batch is a set of segments L_g = conv{v1_g, v2_g} inflated by Algorithm 1
 * with shared parameters, each starting from the domain D = {A0 x <= b0}
 * (m0 rows; A0 = NULL selects the robot's joint-limit box, rows +e_i <= q_hi_i
 * then -e_i <= -q_lo_i). v1, v2: host FP64 n_seg x n. seg_env (nullable, all
 * 0): obstacle set of each segment, an index into envs. seg_np (nullable):
 * per-segment N_p. seg_stream (nullable, default g): Philox stream id of each
 * segment; rounds and walks are the other counter words, so a segment's
 * result does not depend on what else is in the batch. path_first
 * (nullable): index of the first segment of the path each segment belongs
 * to (segments of a path are consecutive); used by ezo_batch_run_path.
 * The batch allocates its own device memory (state, polytopes, samples,
 * candidates) sized for m0 + n_f * n_it_max rows (at most 2048) and
 * max(N_p, M_{N_it}) samples per segment. Its label and bisection kernels
 * take at least the fewest lanes per configuration whose sphere centres fit
 * in shared memory (4 for 256 robot spheres with 4096 obstacles; 1 for the
 * usual robots); ezo_batch_set_shape refuses fewer. Errors:
 * EZO_ERR_INVALID_ARG (also when even 8 lanes do not fit), EZO_ERR_CUDA. */
ezo_status ezo_batch_create(const ezo_robot* robot, int32_t n_env, const ezo_env* const* envs, int32_t n_seg,
                            const double* v1, const double* v2, const int32_t* seg_env, const int32_t* seg_np,
                            const uint32_t* seg_stream, const int32_t* path_first, const double* A0,
                            const double* b0, int32_t m0, const ezo_params* params, ezo_batch** out);
void ezo_batch_free(ezo_batch* batch);

/* Puts every segment back to round 1 with its polytope equal to the domain
 * D, optionally replacing the segment endpoints with host arrays v1, v2
 * (n_seg x n FP64; NULL keeps the current ones). Stream-ordered; the batch's
 * device buffers are reused, nothing is allocated. */
ezo_status ezo_batch_reset(ezo_batch* batch, const double* v1, const double* v2, void* cuda_stream);

/* Run modes. HOST_LOOP launches the round kernels per round and reads a
 * small round summary back to decide whether to go on; GRAPH captures one
 * round into a CUDA graph whose conditional WHILE node repeats it on the
 * device until no segment is active (one launch, no host round trips). */
typedef enum { EZO_RUN_HOST_LOOP = 0, EZO_RUN_GRAPH = 1 } ezo_run_mode;

/* Algorithm 1 for every segment of the batch at once, until each one is
 * accepted, reported in collision (t_col) or has run N_it rounds. Returns
 * after the stream has finished. Errors: EZO_ERR_CUDA. */
ezo_status ezo_batch_run(ezo_batch* batch, int32_t mode, void* cuda_stream);

/* Sec. VI-A: the batch's segments form paths (path_first); inflate them in
 * order, skipping a segment whose endpoints lie in an earlier polytope of the
 * same path (A x <= b + 1e-9), and stop a path after a segment reported in
 * collision. sequential = 1 runs one segment at a time over all paths (the
 * paper's order, a host-driven launch loop); sequential = 2 ("wavefront")
 * keeps each path's order but runs the current segment of every path in one
 * batched run per wave (with mode EZO_RUN_GRAPH all waves, each with its
 * skip rule on the device and its rounds, run inside one graph launch; with
 * EZO_RUN_HOST_LOOP the host applies the skip rule between waves);
 * sequential = 0 inflates all segments speculatively
 * in one batched run and applies the same skip rule afterwards on the device
 * (one synchronisation at the end). Returns after the stream has finished.
 * All three
 * keep the same polytopes. Skipped segments report EZO_SEG_SKIPPED, segments
 * after a collision EZO_SEG_IDLE. Errors: EZO_ERR_CUDA. */
ezo_status ezo_batch_run_path(ezo_batch* batch, int32_t sequential, int32_t mode, void* cuda_stream);

/* Per-segment result: status (ezo_segment_status), rounds run, rows m of the
 * polytope, planes added, exact collision checks performed. Any output
 * pointer may be NULL. Synchronous (copies from the device). */
ezo_status ezo_batch_get_segment(const ezo_batch* batch, int32_t seg, int32_t* status, int32_t* rounds,
                                 int32_t* m, int32_t* planes, int64_t* checks);

/* Copies polytope `seg` (m x n row-major A, m entries of b; host buffers of
 * at least m_cap x n and m_cap doubles, m_cap from ezo_batch_capacity) and
 * writes its row count to *m. */
ezo_status ezo_batch_get_polytope(const ezo_batch* batch, int32_t seg, int32_t* m, double* A, double* b);

/* Every segment at once, for end-to-end readers: status[g] and m[g] (host,
 * n_seg entries each), and, when A / b are given, the first m_read rows of
 * every polytope into A (host, n_seg x rows x n, row major per segment:
 * segment g's row r at A[(g * rows + r) * n]) and b (n_seg x rows); rows
 * beyond m[g] are not meaningful. m_read >= max_g m[g]: when the buffers
 * hold at most 4 MiB (n_seg x min(rows, m_cap) x (n + 1) doubles) every
 * row up to min(rows, m_cap) is copied together with the states (one
 * synchronisation), otherwise the states are read first and max_g m[g] rows
 * follow. *m_read (nullable) receives m_read. One state copy and one strided
 * copy each for A and b. Synchronous. EZO_ERR_CAPACITY when rows <
 * max_g m[g]. */
ezo_status ezo_batch_get_polytopes(const ezo_batch* batch, int32_t* status, int32_t* m, double* A, double* b,
                                   int32_t rows, int32_t* m_read, void* cuda_stream);

/* Page-locked host memory (cudaMallocHost) for the host side of the copies
 * above: copies into it run at the host link's rate without staging through
 * a driver buffer. *out receives the buffer (NULL when bytes = 0); free it
 * with ezo_host_free. Errors: EZO_ERR_INVALID_ARG (out NULL), EZO_ERR_CUDA. */
ezo_status ezo_host_alloc(size_t bytes, void** out);
void ezo_host_free(void* p);

/* Row capacity per segment (m0 + n_f * n_it_max) and sample capacity. */
ezo_status ezo_batch_capacity(const ezo_batch* batch, int32_t* m_cap, int32_t* s_cap);

/* Lanes of a warp that share one hit-and-run walk (Algorithm 1, sampling
 * step): 1, 2, 4 or 8, or 0 (the default) to choose per round on the device
 * from the number of walks, eight lanes when the round has fewer walks than
 * the GPU holds threads. Every choice draws the same samples bit for bit; only
 * the speed differs. EZO_ERR_INVALID_ARG for any other value. */
ezo_status ezo_batch_set_sample_lanes(ezo_batch* batch, int32_t lanes);

/* Launch shapes of a batch's round kernels. sample_fill_tiles: the walks'
 * lane rule takes one lane per walk from 2 x this many 128-walk tiles per
 * round up, two from this many, four from a quarter, else eight (default:
 * the tiles that fill every scheduler with one warp, 4 x SMs x 32 / 128);
 * check_lanes: lanes per configuration of the label kernel (1, 2, 4 or 8);
 * bisect_lanes: lanes per bisection candidate (1, 2, 4, 8, 16 or 32), or 96:
 * three warps per candidate testing the three points of two halvings at
 * once (fewer dependent checks, half again the checks; scenes with boxes
 * run 16, 32 and 96 at 8). Every shape gives the same samples and
 * polytopes, and the same labels outside the FP32 rounding band of a
 * contact, bit for bit; only the speed differs. */
typedef struct {
  int32_t sample_fill_tiles;
  int32_t check_lanes;
  int32_t bisect_lanes;
} ezo_shape;
ezo_status ezo_batch_get_shape(const ezo_batch* batch, ezo_shape* shape);
/* Sets the shape (EZO_ERR_INVALID_ARG for values out of range, or for label
 * or bisection lanes below the fewest whose sphere centres fit in shared
 * memory, see ezo_batch_create); a captured graph is rebuilt at the next
 * graph run. The autotuner skips such shapes. */
ezo_status ezo_batch_set_shape(ezo_batch* batch, const ezo_shape* shape);
/* Autotuner of the shape: runs the whole batch (host-loop mode, best of
 * `reps` timed runs after a warm-up) for the bisection lanes 4, 8, 16, 32, 96, 2, then
 * the label lanes 1, 2, 4, 8, then sample_fill_tiles at half, one and two
 * times the default, keeping a change only when it is at least 2% faster,
 * and sets the winner. Results are cached for the process per (device, robot
 * shape, padded obstacle count, boxes, size classes of round 1's samples, of
 * N_p and of the segment count, N_b, surrogate attached), so a later batch of
 * the same class takes the cached shape without timing. The batch is left
 * reset (round 1, polytopes = D). *chosen (nullable) receives the shape.
 * Synchronous. */
ezo_status ezo_batch_tune(ezo_batch* batch, int32_t reps, ezo_shape* chosen, void* cuda_stream);

/* Step-by-step access for tests and tools. ezo_batch_step runs one kernel of
 * the current round over the batch: 0 round size (a1), 1 hit-and-run (a2),
 * 2 collision labels (a3, a4), 3 certification and selection (a5, a6),
 * 4 projection and bisection (a7, a8), 5 hyperplane placement (a9), 6 round
 * end; 7 round end fused with the next round's size, and 8 placement whose
 * last block then runs 7 (the run loops' kernels). Stream-ordered; call
 * ezo_batch_sync before reading. */
ezo_status ezo_batch_step(ezo_batch* batch, int32_t step, void* cuda_stream);
ezo_status ezo_batch_sync(ezo_batch* batch, void* cuda_stream);

/* Reads an internal per-segment buffer of the current round into host
 * memory: 0 samples (FP32, n x s_cap dimension-major), 1 labels (uint8
 * s_cap), 2 candidate sample indices (int32 N_p), 3 c* (FP64, n x N_p
 * dimension-major), 4 distance to L of c* (FP64 N_p), 5 bisection decisions
 * (uint32 N_p, bit s = midpoint s in collision), 6 round state (int32[12]:
 * k, status, m, |S|, M, count, n_cand, planes, rounds, n_placed, N_p, env,
 * and s_cap, the segment's sample capacity and the stride of its samples,
 * as a 13th value when `bytes` holds it),
 * 7 placed candidate indices of the last round (int32 n_f), 8 step backs of
 * the last round (FP64 n_f), 9 work counters int64[3] {exact checks at
 * samples, exact checks at bisection midpoints, algorithmic FP32 flops of the
 * hit-and-run walks: per walk step 2mn + 5m + 6n}, 11 surrogate evaluations (int64), 10 the batch's round summary (int32[4]: active
 * segments, rounds run since the last reset, sample tiles, bisection tiles;
 * `seg` is ignored). `bytes` is the size of `dst`. */
ezo_status ezo_batch_read(const ezo_batch* batch, int32_t seg, int32_t what, void* dst, int64_t bytes);

/* Overwrites the samples of segment `seg` for the current round (FP32,
 * n x count dimension-major, count <= s_cap) so that a round can be replayed
 * on given samples; sets |S| to count. */
ezo_status ezo_batch_write_samples(ezo_batch* batch, int32_t seg, const float* samples, int32_t count);

/* ------------------------------------------------------- one-call inflation --
 * The problem statement of Sec. IV-B (Algorithm 1): robot, obstacles, a
 * collision-free segment L = conv{v1, v2}, the domain D and (eps, delta) in;
 * a polytope P = {A x <= b} with L inside P out, which with probability at
 * least 1 - delta has at most an eps fraction of its volume in collision.
 * Path inflation (Sec. VI-A) inflates the segments of a piecewise-linear path
 * in order and skips a segment whose endpoints lie in an earlier polytope of
 * the path. Each call builds a batch (ezo_batch_create), runs it with the
 * batch kernels, copies the results into host objects owned by the caller
 * and frees the batch; it blocks until they are on the host. The device
 * memory is allocated and freed inside the call.
 *
 * Per-polytope statistics (the segment's outcome and work). */
typedef struct {
  int32_t status;   /* ezo_segment_status: ACCEPTED, IN_COLLISION, CAPACITY or MAX_ITER */
  int32_t rounds;   /* rounds of Algorithm 1 run */
  int32_t m;        /* rows of A */
  int32_t planes;   /* hyperplanes added to the domain */
  int64_t checks;   /* exact collision checks (samples and bisection midpoints) */
  int64_t checks_bisect;    /* of which at bisection midpoints */
  int64_t surrogate_evals;  /* surrogate evaluations (0 without a surrogate) */
} ezo_stats;

typedef struct ezo_polytope ezo_polytope; /* host object: A (m x n, row major), b (m), stats */
typedef struct ezo_scs ezo_scs;           /* sequence of polytopes of one path, in path order */

/* Algorithm 1 on one segment: v1, v2 (host FP64, n values each); the domain
 * D = {A0 x <= b0} (host FP64, m0 x n row major and m0 values), or the
 * robot's joint-limit box when A0 = NULL (then m0 = 0); params as in
 * ezo_batch_create; stream_id is the segment's Philox stream (the other
 * counter words are the round and the walk), so the polytope equals that of
 * the same segment in any batch with the same stream id. *out receives a new
 * polytope (free it with ezo_polytope_free) whenever the call returns
 * EZO_OK, EZO_ERR_SEGMENT_IN_COLLISION (the rows placed before the t_col rule
 * fired; no region is certified), EZO_ERR_CAPACITY (no room for another N_f
 * rows) or EZO_WARN_MAX_ITER (N_it rounds without acceptance; no
 * guarantee); stats (nullable) receives its statistics. Other errors
 * (EZO_ERR_INVALID_ARG, EZO_ERR_CUDA) leave *out NULL. */
ezo_status ezo_inflate_segment(const ezo_robot* robot, const ezo_env* env, const double* v1, const double* v2,
                               const double* A0, const double* b0, int32_t m0, const ezo_params* params,
                               uint32_t stream_id, ezo_polytope** out, ezo_stats* stats, void* cuda_stream);

/* Sec. VI-A on one path of n_verts vertices (host FP64, n_verts x n row
 * major, n_verts >= 2): segment k = (verts[k], verts[k + 1]) draws from
 * Philox stream stream_base + k. mode 0 runs the paper's order (one segment
 * at a time, host launch loop); mode 1 ("wavefront") and mode 2 (every
 * segment speculatively in one graph, the skip rule applied afterwards) keep
 * the same polytopes. *out receives the path's sequence of convex sets: one
 * polytope per segment that was inflated, in path order, each tagged with its
 * segment index (ezo_polytope_stats); the path stops after a segment reported
 * in collision. Returns the most severe outcome of its segments (an error
 * before EZO_WARN_MAX_ITER before EZO_OK); *out is set for those outcomes as
 * in ezo_inflate_segment. Free it with ezo_scs_free. */
ezo_status ezo_inflate_path(const ezo_robot* robot, const ezo_env* env, const double* verts, int32_t n_verts,
                            const double* A0, const double* b0, int32_t m0, const ezo_params* params, int32_t mode,
                            uint32_t stream_base, ezo_scs** out, void* cuda_stream);

/* Many paths over several obstacle sets at once (the batched form): path i
 * has path_len[i] >= 1 segments, its path_len[i] + 1 vertices follow those of
 * path i - 1 in verts (host FP64, row major), and it runs in obstacle set
 * envs[path_env[i]] (path_env NULL: all in envs[0]). seg_np (nullable, one
 * value per segment in path order) gives per-segment N_p. The segment with
 * global index g (counting over all paths in order) draws from Philox stream
 * stream_base + g. mode as in ezo_inflate_path; out (host array of n_path
 * pointers) receives one sequence of convex sets per path. Returns the most
 * severe outcome over all segments; on EZO_ERR_INVALID_ARG or EZO_ERR_CUDA
 * every out[i] is NULL. */
ezo_status ezo_inflate_batch(const ezo_robot* robot, int32_t n_env, const ezo_env* const* envs, int32_t n_path,
                             const int32_t* path_len, const double* verts, const int32_t* path_env,
                             const int32_t* seg_np, const double* A0, const double* b0, int32_t m0,
                             const ezo_params* params, int32_t mode, uint32_t stream_base, ezo_scs** out,
                             void* cuda_stream);

/* Rows m and dimension n of a polytope, and (each nullable) A into a host
 * buffer of m x n doubles (row major) and b into m doubles. */
ezo_status ezo_polytope_get(const ezo_polytope* p, int32_t* m, int32_t* n, double* A, double* b);
/* The segment index the polytope was inflated for (0 for ezo_inflate_segment,
 * the index within its path otherwise) and its statistics; both nullable. */
ezo_status ezo_polytope_stats(const ezo_polytope* p, int32_t* segment, ezo_stats* stats);
void ezo_polytope_free(ezo_polytope* p);
/* Number of polytopes of a sequence, polytope i (owned by the sequence; NULL
 * when i is out of range), and freeing the sequence with its polytopes. */
int32_t ezo_scs_size(const ezo_scs* scs);
const ezo_polytope* ezo_scs_get(const ezo_scs* scs, int32_t i);
void ezo_scs_free(ezo_scs* scs);

/* ------------------------------------------------------------- recovery --
 * Sec. VI-B: a trajectory planned in the sets is checked at fine steps; the
 * collisions found in a set are excluded from it by repeating the last steps
 * of Algorithm 1 (bisection toward the seed segment, ordering, hyperplane
 * placement with step back and t_col, at most N_f planes); afterwards every
 * segment of the seed path must lie in some set of its path, and segments
 * that no longer do are inflated again. */

/* Fine discretisation of a piecewise-linear path (host only): edge k, from
 * v_k to v_{k+1} (rows of `verts`, n_verts x n FP64 row-major), is cut into
 * N_k = max(1, ceil(|v_{k+1} - v_k|_2 / step)) pieces and checked at its
 * N_k + 1 points v_k + (i / N_k)(v_{k+1} - v_k), i = 0..N_k (the appendix
 * checks paths at 0.1 rad). Writes N_k + 1 to edge_points[k] (nullable,
 * n_verts - 1 entries) and the sum to *total. EZO_ERR_INVALID_ARG for
 * step <= 0, a non-finite step or edge, n outside [1, 16]. */
ezo_status ezo_path_points(const double* verts, int32_t n_verts, int32_t n, double step, int64_t* edge_points,
                           int64_t* total);

/* Collision check of those points on the GPU: each point is interpolated in
 * FP64 (product and sum rounded separately), rounded to FP32 and checked with
 * the same forward kinematics and sphere test as ezo_check_collision.
 * edge_flags (host, n_verts - 1 bytes): 1 when any point of the edge
 * collides. point_flags_dev (nullable, device, point_cap bytes): 1 per
 * colliding point, in edge order. *n_points (nullable) receives the point
 * count. Synchronous; uses stream-ordered scratch (cudaMallocAsync).
 * EZO_ERR_CAPACITY when point_cap is below the point count;
 * EZO_ERR_INVALID_ARG when spheres and obstacles exceed shared memory even at
 * 8 lanes per point (the lane count is chosen as in ezo_check_collision). */
ezo_status ezo_check_path(const ezo_robot* robot, const ezo_env* env, const double* verts, int32_t n_verts,
                          double step, uint8_t* edge_flags, uint8_t* point_flags_dev, int64_t point_cap,
                          int64_t* n_points, void* cuda_stream);

/* Replaces the current polytope of segment `seg` with m rows (A: m x n FP64
 * row-major, b: m entries; host buffers, copied), for editing sets computed
 * elsewhere. EZO_ERR_CAPACITY when m > m_cap. Synchronous. */
ezo_status ezo_batch_set_polytope(ezo_batch* batch, int32_t seg, int32_t m, const double* A, const double* b,
                                  void* cuda_stream);

/* Set editing: for every segment whose polytope P is final (accepted, or N_it
 * reached), the configurations cfg (n_cfg x n FP64 row-major, host; rounded
 * to FP32 like samples) that collide and lie in P (A c <= b + 1e-9, FP64) form
 * S_col; its first N_p by index are bisected toward the segment and planes are
 * placed as in a round of Algorithm 1, with no test; rows are appended to P.
 * Per segment, ezo_batch_read(.., 6, ..) then reports count = |S_col|,
 * n_cand and n_placed; a segment whose candidate lies within t_col of it
 * becomes EZO_SEG_IN_COLLISION, one without room for N_f more rows
 * EZO_SEG_CAPACITY. EZO_ERR_CAPACITY when n_cfg exceeds a segment's sample
 * capacity; EZO_ERR_INVALID_ARG while a segment is still active.
 * Synchronous. */
ezo_status ezo_batch_edit(ezo_batch* batch, int64_t n_cfg, const double* cfg, void* cuda_stream);

/* covered[g] (host, n_seg bytes) = 1 when both endpoints of segment g lie in
 * the final polytope (accepted or N_it reached) of some segment of the same
 * path, A x <= b + 1e-9; then the whole segment does. Synchronous. */
ezo_status ezo_batch_coverage(ezo_batch* batch, uint8_t* covered, void* cuda_stream);

/* Inflates the segments with which[g] != 0 again from round 1 with P = D (the
 * batch's domain), keeping every other segment as it is, and runs them in
 * `mode` until done. Check counters accumulate. Synchronous.
 * EZO_ERR_INVALID_ARG while a segment is still active. */
ezo_status ezo_batch_reinflate(ezo_batch* batch, const uint8_t* which, int32_t mode, void* cuda_stream);

/* ---------------------------------------------------- no-allocation path --
 * No counterpart in the paper. For callers that cannot allocate device memory
 * when they need a region: a real-time control loop that must not block in
 * cudaMalloc (which can synchronise the device and has no latency bound), or a
 * host application that fixes the library's device memory at start-up.
 * Inflates one segment v1..v2 (host FP64, n values each) from the robot's
 * joint-limit box with the same kernels, parameters and Philox stream
 * (stream_id) as a one-segment ezo_batch_run in HOST_LOOP mode, so the
 * polytope, status, rounds and check count equal that call's bit for bit. All working memory comes from one file-scope device
 * array of EZO_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits; the call itself makes no cudaMalloc, cudaFree or
 * other allocating call. Outputs: A_out (host, at least
 * (2n + n_f * n_it_max) x n doubles) and b_out (2n + n_f * n_it_max) receive
 * the polytope, *m_out its row count; status_out (ezo_segment_status),
 * rounds_out and checks_out may be NULL. The robot and env handles must have
 * been created beforehand (their creation allocates).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for that device. With CUDA's lazy module loading
 * that first call (like the first launch of each kernel) also loads the
 * library's device code and with it the array, which can allocate and
 * synchronise: make one call per device at start-up, outside the section
 * that must not allocate, and before any stream capture. Later calls make no
 * allocation. The array is shared by every call and keeps the last call's
 * contents; each call re-initialises what it reads. Calls that overlap on
 * the GPU (other streams or host threads) race on the array: serialise them.
 * A call that fails after queueing work waits for its stream before it
 * returns, so the array is idle afterwards. Blocks until the result is on the
 * host.
 * Errors: EZO_ERR_INVALID_ARG (also when the robot's spheres and the
 * obstacles do not fit the collision kernels' shared memory, checked before
 * anything runs); EZO_ERR_CAPACITY when the segment needs more
 * working memory than the array holds (roughly n_p <= 11000 for n = 16,
 * 23000 for n = 7, at n_f = 10 and n_it_max = 50) or
 * more than 2048 rows; EZO_ERR_CUDA. */
#define EZO_NOALLOC_SCRATCH_BYTES (6u * 1024u * 1024u)
ezo_status ezo_inflate_segment_noalloc(const ezo_robot* robot, const ezo_env* env, const double* v1,
                                       const double* v2, const ezo_params* params, uint32_t stream_id,
                                       double* A_out, double* b_out, int32_t* m_out, int32_t* status_out,
                                       int32_t* rounds_out, int64_t* checks_out, void* cuda_stream);

/* -------------------------------------------------------------- profiling --
 * When enabled, ezo_batch_run in HOST_LOOP mode records CUDA events around
 * every kernel launch on the launch stream; ezo_profile_read returns, for
 * kernel kind i (0 round size, 1 sample, 2 check, 3 certify, 4 bisect,
 * 5 place, 6 round end), the total milliseconds and launch count since the
 * last reset. */
ezo_status ezo_profile_enable(int32_t on);
ezo_status ezo_profile_reset(void);
ezo_status ezo_profile_read(double* ms, int64_t* launches, int32_t n_kinds);

/* ------------------------------------------------------- learned surrogate --
 * Not in the paper. A small MLP sd_hat(q) estimates the signed distance from
 * the features [sin q, cos q] (zero-padded to 64) through three hidden layers
 * of 256 SiLU units to one output. Hidden-layer products run on BF16 tensor
 * cores with FP32 accumulation (inference: one kernel per 128-row tile with
 * the accumulators in tensor memory and SiLU on the hardware tanh
 * approximation, relative error ~2^-11 before the BF16 rounding of each
 * activation); weights have FP32 masters trained with Adam
 * (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the mean squared error,
 * every hidden-layer product of training on tcgen05 tensor cores too. It
 * only orders and prefilters bisection candidates (ezo_batch_attach_surrogate);
 * labels and certification stay exact.
 * Parameters are one flat FP32 vector of ezo_surrogate_num_params() values:
 * W1 [256 x 64] | b1 [256] | W2 [256 x 256] | b2 | W3 [256 x 256] | b3 |
 * w4 [256] | b4 [1], matrices row-major (out x in).
 * create: deterministic initialisation from seed (uniform in
 * +-1/sqrt(fan_in)); device memory is allocated here.
 * train: draws n_samples configurations uniformly in the robot's joint box
 * (Philox, data_seed), labels them with the exact FP32 signed distance against
 * env clamped to [label_lo, label_hi], and runs `epochs` passes of Adam over
 * mini-batches of `batch` (a multiple of 64); epoch_loss (nullable, `epochs`
 * floats) receives the last batch loss of each epoch. Synchronous.
 * grad: one forward and backward pass on N (multiple of 64) configurations
 * q_dev (n x N, stride ldq) with targets t_dev, no update; gradient of the
 * mean squared error into grad (host, num_params floats) and the loss into
 * *loss. Synchronous.
 * predict: sd_hat for N configurations into out_dev (FP32). Stream-ordered. */
typedef struct ezo_surrogate ezo_surrogate;
int64_t ezo_surrogate_num_params(void);
ezo_status ezo_surrogate_create(const ezo_robot* robot, uint64_t seed, ezo_surrogate** out);
void ezo_surrogate_free(ezo_surrogate* sur);
ezo_status ezo_surrogate_get_params(const ezo_surrogate* sur, float* params);
ezo_status ezo_surrogate_set_params(ezo_surrogate* sur, const float* params);
ezo_status ezo_surrogate_train(ezo_surrogate* sur, const ezo_env* env, int64_t n_samples, int32_t epochs,
                               int32_t batch, float lr, uint64_t data_seed, float label_lo, float label_hi,
                               float* epoch_loss, void* cuda_stream);
ezo_status ezo_surrogate_grad(ezo_surrogate* sur, const float* q_dev, int64_t ldq, const float* t_dev, int32_t N,
                              float* grad, float* loss, void* cuda_stream);
ezo_status ezo_surrogate_predict(ezo_surrogate* sur, const float* q_dev, int64_t ldq, int64_t N, float* out_dev,
                                 void* cuda_stream);
/* Health of the tensor-core kernels (the forward pass and the training
 * GEMMs): every wait inside them is bounded (about 2 s); a wait that gave up
 * sets a flag on the device, and the forward pass writes NaN for the rows it
 * did not finish. *timed_out receives that flag (0 or 1) after the
 * work queued on cuda_stream has finished; reset != 0 clears it.
 * Synchronous. EZO_ERR_INVALID_ARG for NULL arguments. */
ezo_status ezo_surrogate_status(ezo_surrogate* sur, int32_t* timed_out, int32_t reset, void* cuda_stream);

/* Surrogate-guided bisection for a batch (not in the paper): in each round
 * the N_b bisection steps of every candidate are taken on sd_hat (predicted
 * collision iff sd_hat < margin; all steps of all candidates in one
 * tensor-core launch); each end point is
 * then checked exactly and kept when it collides, otherwise that candidate
 * gets the exact bisection of Sec. IV-B. Labels, the unadaptive test and the
 * planes use exact checks only. sur = NULL detaches. The robot must have at
 * most 8 joints. Allocates the batch's surrogate buffers on first use.
 * ezo_batch_read code 11 returns the surrogate evaluations (int64). */
ezo_status ezo_batch_attach_surrogate(ezo_batch* batch, ezo_surrogate* sur, float margin);

/* ------------------------------------------------------------- autotuner --
 * Launch shape of the collision kernels: the number of warp lanes that share
 * one configuration (1, 2, 4 or 8). ezo_tune_lanes times the collision
 * kernel on N uniform configurations of the robot's joint box (N rounded up
 * to a power of two, at most 2^22) for each choice and returns the fastest;
 * results are cached per (device, robot shape, padded obstacle count, size
 * class) for the process. ezo_check_collision with lanes_per_config = 0 and
 * ezo_batch_create use it unless ezo_set_autotune(0) switched it off, in
 * which case a size rule is used. Tuning allocates a scratch batch with
 * cudaMalloc. */
ezo_status ezo_tune_lanes(const ezo_robot* robot, const ezo_env* env, int64_t N, int32_t* lanes, void* cuda_stream);
ezo_status ezo_set_autotune(int32_t on);

/* FP32 calibration of the ALU roofline: times a kernel of independent fused
 * multiply-add chains that fills every warp slot of every SM (best of three
 * launches after one warm-up) and writes the achieved FP32 rate, two flops
 * per FMA, in TFLOP/s into *tflops. Allocates and frees a small scratch
 * buffer; synchronous on cuda_stream. EZO_ERR_INVALID_ARG for tflops = NULL,
 * EZO_ERR_CUDA on a failed allocation or launch. */
ezo_status ezo_probe_fp32_fma(double* tflops, void* cuda_stream);

/* Algorithmic FP32 work of one exact configuration check (forward kinematics
 * plus 8 flops per obstacle pair and per self pair, every pair counted), as
 * used for rooflines. */
double ezo_check_flops(const ezo_robot* robot, const ezo_env* env);
/* The robot spheres (the first ones, on the fixed base frame) whose obstacle
 * pairs the checker's sweep decides once for this obstacle set instead of per
 * configuration: every such sphere clears every obstacle sphere by more than
 * 1e-4 m, whole chunks of eight spheres; 0 when none qualifies or for NULL
 * handles. Their 8 x count x n_obs flops per configuration are part of
 * ezo_check_flops but are not executed per configuration. */
int32_t ezo_check_static_spheres(const ezo_robot* robot, const ezo_env* env);

#ifdef __cplusplus
}
#endif

#endif /* EZO_H */
