// Device-side building blocks of the EI-ZO hot path (sm_103a).
//
// * Philox4x32-10 counter-based generator (Salmon et al., SC'11), used by the
//   hit-and-run walks of Sec. IV-B / IV-D.
// * Forward kinematics of a standard DH chain in FP32 and the sphere
//   collision test (robot vs obstacle spheres and listed self pairs) that the
//   paper's GPU collision checker performs (Sec. IV-D, Sec. V-B).
//
// Collision test, per robot sphere i and obstacle j:
//   ||c_i - o_j||^2 < (r_i + R_j)^2
//   <=>  t_ij = c_i.o_j + r_i R_j - (|o_j|^2 - R_j^2)/2  >  hu_i = (|c_i|^2 - r_i^2)/2.
// t_ij is four FP32 FMAs per pair; a sphere is decided from max_j t_ij - hu_i
// when that margin exceeds a rounding bound E, and re-checked with the
// direct difference form otherwise, so labels equal the direct FP32 test.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define EZO_MAX_DOF 16
#define EZO_MAX_SPHERES 256
#define EZO_MAX_OBS 4096
#define EZO_CH 8
#define EZO_MAX_SBLK 32
#define EZO_MAX_BOX 32    // robot boxes
#define EZO_MAX_EBOX 64   // obstacle boxes per environment

namespace ezo {

// ------------------------------------------------------------------ Philox --
struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    // each 32 x 32 -> 64-bit product gives both halves at once
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// The ten round keys of Philox4x32-10 for one seed: (k0 + r 0x9E3779B9,
// k1 + r 0xBB67AE85) for r = 0..9, computed on the host and passed in kernel
// parameters, so the rounds read them as constant operands.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys ks;
  uint32_t a = (uint32_t)(seed & 0xffffffffu), b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    ks.k0[r] = a;
    ks.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return ks;
}

// philox4x32_10 with the round keys given (the same bits).
__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, const PhiloxKeys& ks) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = u32x4{hi1 ^ c.y ^ ks.k0[r], lo1, hi0 ^ c.w ^ ks.k1[r], lo0};
  }
  return c;
}

// [0, 1): top 24 bits times 2^-24 (exact in FP32).
__device__ __forceinline__ float u01_co(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-8f; }
// (0, 1]: (top 24 bits + 1) times 2^-24 (exact in FP32).
__device__ __forceinline__ float u01_oc(uint32_t x) { return (float)((x >> 8) + 1u) * 5.9604644775390625e-8f; }

// ------------------------------------------------------------------ robot --
// Device image of a robot: DH chain plus spheres sorted by the frame they are
// attached to. Lives in global memory; kernels stage the small part in smem.
struct RobotDev {
  int n;              // degrees of freedom (<= EZO_MAX_DOF)
  int n_spheres;      // real spheres
  int n_spheres_pad;  // multiple of EZO_CH; padding spheres never collide
  int n_self;         // listed self pairs
  float ca[EZO_MAX_DOF], sa[EZO_MAX_DOF], a[EZO_MAX_DOF], d[EZO_MAX_DOF], toff[EZO_MAX_DOF];
  // joint j turns by kth_j q_j + toff_j and slides by d_j + kd_j q_j:
  // (kth, kd) = (1, 0) for a revolute joint, (0, 1) for a prismatic one
  float kth[EZO_MAX_DOF], kd[EZO_MAX_DOF];
  int frame_first[EZO_MAX_DOF + 2];  // sorted spheres of frame f: [frame_first[f], frame_first[f+1])
  float4 sph[EZO_MAX_SPHERES];       // local x, y, z and radius (sorted by frame)
  const ushort2* self_pairs;         // [n_self] indices into the sorted spheres
  const float* self_rr;              // [n_self] (r_i + r_j)^2
  // Self pairs as work items (r0, nr, k0, nk): sorted spheres [r0, r0 + nr),
  // nr <= EZO_CH, each against the partners [k0, k0 + nk), when the pair
  // list is a union of such blocks (n_sblk > 0, then the n_self pairs are
  // not used); swept like obstacles with band E_self.
  int n_sblk;
  float E_self;
  int4 sblk[EZO_MAX_SBLK];
  // Oriented boxes fixed to frames (sorted by frame, box_first like
  // frame_first), four float4 each in the frame: (centre, h_x), (axis 0, h_y),
  // (axis 1, h_z), (axis 2, 0); self pairs sphere x box and box x box
  int n_box;
  int box_first[EZO_MAX_DOF + 2];
  float4 box_l[4 * EZO_MAX_BOX];
  int n_sbp, n_bbp;
  const ushort2* sb_pairs;  // (sorted sphere, sorted box)
  const ushort2* bb_pairs;  // (sorted box, sorted box)
};

// The chain and the spheres in FP64 as given at creation (spheres sorted as
// in RobotDev), for the FP64 reference kinematics that the forward-kinematics
// error of the FP32 checker is measured against.
struct RobotFK64 {
  int n, n_spheres;
  double ca[EZO_MAX_DOF], sa[EZO_MAX_DOF], a[EZO_MAX_DOF], d[EZO_MAX_DOF], toff[EZO_MAX_DOF];
  double kth[EZO_MAX_DOF], kd[EZO_MAX_DOF];
  int frame_first[EZO_MAX_DOF + 2];
  double sx[EZO_MAX_SPHERES], sy[EZO_MAX_SPHERES], sz[EZO_MAX_SPHERES];
};

// The part of RobotDev a block keeps in shared memory.
struct RobotSmem {
  float ca[EZO_MAX_DOF], sa[EZO_MAX_DOF], a[EZO_MAX_DOF], d[EZO_MAX_DOF], toff[EZO_MAX_DOF];
  float kth[EZO_MAX_DOF], kd[EZO_MAX_DOF];
  int frame_first[EZO_MAX_DOF + 2];
  int box_first[EZO_MAX_DOF + 2];
  int n_box, n_sbp, n_bbp;
  int n, n_spheres, n_spheres_pad, n_self;
  int n_sblk;
  float E_self;
  int4 sblk[EZO_MAX_SBLK];
};

__device__ __forceinline__ void stage_robot(RobotSmem& rs, float4* sph_s, const RobotDev* __restrict__ rd) {
  for (int i = threadIdx.x; i < EZO_MAX_DOF; i += blockDim.x) {
    rs.ca[i] = rd->ca[i];
    rs.sa[i] = rd->sa[i];
    rs.a[i] = rd->a[i];
    rs.d[i] = rd->d[i];
    rs.toff[i] = rd->toff[i];
    rs.kth[i] = rd->kth[i];
    rs.kd[i] = rd->kd[i];
  }
  for (int i = threadIdx.x; i < EZO_MAX_DOF + 2; i += blockDim.x) {
    rs.frame_first[i] = rd->frame_first[i];
    rs.box_first[i] = rd->box_first[i];
  }
  for (int i = threadIdx.x; i < EZO_MAX_SBLK; i += blockDim.x) rs.sblk[i] = rd->sblk[i];
  if (threadIdx.x == 0) {
    rs.n = rd->n;
    rs.n_spheres = rd->n_spheres;
    rs.n_spheres_pad = rd->n_spheres_pad;
    rs.n_self = rd->n_self;
    rs.n_sblk = rd->n_sblk;
    rs.E_self = rd->E_self;
    rs.n_box = rd->n_box;
    rs.n_sbp = rd->n_sbp;
    rs.n_bbp = rd->n_bbp;
  }
  const int np = rd->n_spheres_pad;
  for (int i = threadIdx.x; i < np; i += blockDim.x) sph_s[i] = rd->sph[i];
}

// The robot's boxes in their frames (4 float4 per box) into shared memory.
__device__ __forceinline__ void stage_robot_boxes(float4* rbox_l, const RobotDev* __restrict__ rd) {
  const int nb = 4 * rd->n_box;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) rbox_l[i] = rd->box_l[i];
}

// Obstacle set in global memory: (x, y, z, R) and -(|o|^2 - R^2)/2, padded to
// a multiple of EZO_CH with far-away spheres that can never collide.
struct EnvDev {
  const float4* obs;
  const float* nhw;
  int n_obs;
  int n_obs_pad;
  const float4* box;  // obstacle boxes, 4 float4 each: (centre, h_x), (axis 0, h_y), (axis 1, h_z), (axis 2, 0)
  int n_box;
  // first robot sphere of the obstacle sweep (a multiple of EZO_CH): the
  // spheres before it sit on the fixed base frame, so their pairs with these
  // obstacles are the same for every configuration, and they were found
  // clear of every obstacle by more than any rounding band when the pair
  // (robot, obstacle set) was set up; 0 when that does not hold
  int s_first;
};

// Shared-memory image of an obstacle set, in pairs of spheres (2p, 2p + 1):
// obs_s[2p] = (x_2p, x_2p+1, y_2p, y_2p+1), obs_s[2p + 1] = (z_2p, z_2p+1,
// R_2p, R_2p+1), and nhw_s[j] = -(|o_j|^2 - R_j^2)/2 in sphere order, so one
// 128-bit load gives a coordinate of two obstacles as the float2 operand of a
// packed FP32 FMA. n_obs_pad is a multiple of 8, so pairs never straddle the
// padding. obs_at(j) reads sphere j back as (x, y, z, R).
__device__ __forceinline__ void stage_env(float4* obs_s, float* nhw_s, const EnvDev& e) {
  for (int p = threadIdx.x; p < e.n_obs_pad / 2; p += blockDim.x) {
    const float4 a = e.obs[2 * p], b = e.obs[2 * p + 1];
    obs_s[2 * p] = make_float4(a.x, b.x, a.y, b.y);
    obs_s[2 * p + 1] = make_float4(a.z, b.z, a.w, b.w);
  }
  for (int i = threadIdx.x; i < e.n_obs_pad; i += blockDim.x) nhw_s[i] = e.nhw[i];
}

__device__ __forceinline__ float4 obs_at(const float4* __restrict__ obs_s, int j) {
  const float* A = reinterpret_cast<const float*>(obs_s + (j & ~1));
  const int h = j & 1;
  return make_float4(A[h], A[2 + h], A[4 + h], A[6 + h]);
}

__device__ __forceinline__ void stage_env_boxes(float4* ebox_s, const EnvDev& e) {
  for (int i = threadIdx.x; i < 4 * e.n_box; i += blockDim.x) ebox_s[i] = e.box[i];
}

// Box geometry of one collision group (all in shared memory).
struct BoxCtx {
  const float4* rbox_l;  // robot boxes in their frames
  const float4* ebox;    // obstacle boxes of the current environment
  float4* rbox_w;        // this group's robot boxes in the world
  int n_ebox;
  const ushort2* sb_pairs;
  const ushort2* bb_pairs;
};

// Sphere (centre c.xyz, radius r) against an oriented box B (4 float4): the
// centre in box coordinates p_k = axis_k . (c - centre), q_k = abs(p_k) - h_k;
// overlap iff the centre is strictly inside (every q_k < 0) or the squared
// norm of max(q, 0) is below r^2.
__device__ __forceinline__ bool sphere_box_hit(float4 c, float r, const float4* __restrict__ B) {
  const float4 b0 = B[0], b1 = B[1], b2 = B[2], b3 = B[3];
  const float dx = c.x - b0.x, dy = c.y - b0.y, dz = c.z - b0.z;
  const float q0 = fabsf(fmaf(dx, b1.x, fmaf(dy, b1.y, dz * b1.z))) - b0.w;
  const float q1 = fabsf(fmaf(dx, b2.x, fmaf(dy, b2.y, dz * b2.z))) - b1.w;
  const float q2 = fabsf(fmaf(dx, b3.x, fmaf(dy, b3.y, dz * b3.z))) - b2.w;
  if (q0 < 0.f && q1 < 0.f && q2 < 0.f) return true;
  const float m0 = fmaxf(q0, 0.f), m1 = fmaxf(q1, 0.f), m2 = fmaxf(q2, 0.f);
  return fmaf(m0, m0, fmaf(m1, m1, m2 * m2)) < r * r;
}

// Separating-axis test of two oriented boxes, written in A's frame: with
// t = A^T (c_B - c_A) and R = A^T B, a candidate axis L separates when
// abs(t . L) - sum_k hA_k abs(L_k) - sum_k hB_k abs(r_k . L) >= 0 (r_k the
// columns of R); the candidates are A's axes, B's axes and e_i x r_j, the
// latter skipped when abs(L)^2 < 1e-4 (nearly parallel edges). The boxes
// overlap iff no candidate separates them. Scaling L does not change the sign,
// so the cross products are not normalised.
__device__ __forceinline__ bool box_box_hit(const float4* __restrict__ A, const float4* __restrict__ B) {
  const float4 a0 = A[0], a1 = A[1], a2 = A[2], a3 = A[3];
  const float4 b0 = B[0], b1 = B[1], b2 = B[2], b3 = B[3];
  const float ha[3] = {a0.w, a1.w, a2.w}, hb[3] = {b0.w, b1.w, b2.w};
  const float Tx = b0.x - a0.x, Ty = b0.y - a0.y, Tz = b0.z - a0.z;
  const float ax[3][3] = {{a1.x, a1.y, a1.z}, {a2.x, a2.y, a2.z}, {a3.x, a3.y, a3.z}};
  const float bx[3][3] = {{b1.x, b1.y, b1.z}, {b2.x, b2.y, b2.z}, {b3.x, b3.y, b3.z}};
  float t[3], R[3][3], aR[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    t[i] = fmaf(Tx, ax[i][0], fmaf(Ty, ax[i][1], Tz * ax[i][2]));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R[i][j] = fmaf(ax[i][0], bx[j][0], fmaf(ax[i][1], bx[j][1], ax[i][2] * bx[j][2]));
      aR[i][j] = fabsf(R[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)  // A's axes
    if (fabsf(t[i]) - ha[i] - fmaf(hb[0], aR[i][0], fmaf(hb[1], aR[i][1], hb[2] * aR[i][2])) >= 0.f) return false;
#pragma unroll
  for (int j = 0; j < 3; ++j) {  // B's axes
    const float tj = fmaf(t[0], R[0][j], fmaf(t[1], R[1][j], t[2] * R[2][j]));
    if (fabsf(tj) - fmaf(ha[0], aR[0][j], fmaf(ha[1], aR[1][j], ha[2] * aR[2][j])) - hb[j] >= 0.f) return false;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // L = e_i x r_j in A's frame
      float L[3];
      L[i] = 0.f;
      L[(i + 1) % 3] = -R[(i + 2) % 3][j];
      L[(i + 2) % 3] = R[(i + 1) % 3][j];
      const float n2 = fmaf(L[0], L[0], fmaf(L[1], L[1], L[2] * L[2]));
      if (n2 < 1e-4f) continue;
      const float tl = fmaf(t[0], L[0], fmaf(t[1], L[1], t[2] * L[2]));
      const float ra = fmaf(ha[0], fabsf(L[0]), fmaf(ha[1], fabsf(L[1]), ha[2] * fabsf(L[2])));
      float rb = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        rb = fmaf(hb[k], fabsf(fmaf(R[0][k], L[0], fmaf(R[1][k], L[1], R[2][k] * L[2]))), rb);
      if (fabsf(tl) - ra - rb >= 0.f) return false;
    }
  }
  return true;
}

// max of three floats in one instruction (PTX max.f32 with three inputs).
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// World poses of the boxes [b0, b1) of one frame (rotation columns c0..c2,
// origin in the .w entries): centre o + R c, axes R a_k; boxes b with
// b % T == lg on this lane.
template <int T>
__device__ __forceinline__ void box_poses_of_frame(int b0, int b1, int lg, float4 c0, float4 c1, float4 c2,
                                                const BoxCtx& bx) {
  int b = b0 + ((lg - b0) & (T - 1));
  for (; b < b1; b += T) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 l = bx.rbox_l[4 * b + k];
      const float ox = k == 0 ? c0.w : 0.f, oy = k == 0 ? c1.w : 0.f, oz = k == 0 ? c2.w : 0.f;
      bx.rbox_w[4 * b + k] = make_float4(fmaf(c0.x, l.x, fmaf(c1.x, l.y, fmaf(c2.x, l.z, ox))),
                                         fmaf(c0.y, l.x, fmaf(c1.y, l.y, fmaf(c2.y, l.z, oy))),
                                         fmaf(c0.z, l.x, fmaf(c1.z, l.y, fmaf(c2.z, l.z, oz))), l.w);
    }
  }
}

// The pairs of one configuration that involve a box, split over the T lanes
// of its group: robot spheres x obstacle boxes, robot boxes x obstacle
// spheres and boxes, listed sphere-box and box-box self pairs. Returns this
// lane's OR.
template <int T>
__device__ __forceinline__ bool box_pairs_hit(const RobotSmem& rs, const float4* __restrict__ sph_s,
                                           const float4* __restrict__ obs_s, int n_obs, const float4* __restrict__ cen,
                                           int lg, const BoxCtx& bx) {
  bool hit = false;
  const int ns = rs.n_spheres, nb = rs.n_box, ne = bx.n_ebox;
  for (int p = lg; p < ns * ne && !hit; p += T) {  // robot spheres x obstacle boxes
    const int s = p / ne, e = p - s * ne;
    hit = sphere_box_hit(cen[s], sph_s[s].w, bx.ebox + 4 * e);
  }
  for (int p = lg; p < nb * n_obs && !hit; p += T) {  // robot boxes x obstacle spheres
    const int b = p / n_obs, o = p - b * n_obs;
    const float4 ob = obs_at(obs_s, o);
    hit = sphere_box_hit(ob, ob.w, bx.rbox_w + 4 * b);
  }
  for (int p = lg; p < nb * ne && !hit; p += T) {  // robot boxes x obstacle boxes
    const int b = p / ne, e = p - b * ne;
    hit = box_box_hit(bx.rbox_w + 4 * b, bx.ebox + 4 * e);
  }
  for (int p = lg; p < rs.n_sbp && !hit; p += T) {  // self: sphere x box
    const ushort2 pr = bx.sb_pairs[p];
    hit = sphere_box_hit(cen[pr.x], sph_s[pr.x].w, bx.rbox_w + 4 * pr.y);
  }
  for (int p = lg; p < rs.n_bbp && !hit; p += T) {  // self: box x box
    const ushort2 pr = bx.bb_pairs[p];
    hit = box_box_hit(bx.rbox_w + 4 * pr.x, bx.rbox_w + 4 * pr.y);
  }
  return hit;
}

// -------------------------------------------------- FK + collision test --
// Forward kinematics of one configuration by a group of T lanes (T in
// 1..8) of one warp, as the collision checker runs it: the group's lanes share
// the joint sines and cosines, lane lg writes the centres of spheres s with
// s % T == lg into the group's shared slot `cen` as (x, y, z, (|c|^2 - r^2)/2)
// (padding spheres get an infinite last entry), and BOX poses the robot's
// boxes. Ends with a warp barrier; every lane of the warp must call it.
template <int NDOF, int T, bool BOX = false>
__device__ __forceinline__ void fk_group(const float (&q)[NDOF], const RobotSmem& rs,
                                         const float4* __restrict__ sph_s, float4* __restrict__ cen, int lg,
                                         const BoxCtx& bx) {
  float c0x = 1.f, c0y = 0.f, c0z = 0.f;
  float c1x = 0.f, c1y = 1.f, c1z = 0.f;
  float c2x = 0.f, c2y = 0.f, c2z = 1.f;
  float px = 0.f, py = 0.f, pz = 0.f;
  const int n = rs.n;
  // sine and cosine of every joint angle. With T lanes per configuration,
  // lane lg evaluates joints lg, lg + T, .. (all lanes run the same
  // instructions on their own angle) and the group exchanges the results;
  // the values are the same as one lane evaluating all of them.
  float sj[NDOF], cj[NDOF];
  if (T == 1) {
#pragma unroll
    for (int j = 0; j < NDOF; ++j) {
      sj[j] = 0.f;
      cj[j] = 1.f;
      if (j < n) sincosf(fmaf(q[j], rs.kth[j], rs.toff[j]), &sj[j], &cj[j]);
    }
  } else {
    constexpr int JPL = (NDOF + T - 1) / T;
    float ms[JPL], mc[JPL];
#pragma unroll
    for (int k = 0; k < JPL; ++k) {
      const int jm = lg + k * T;
      float ang = 0.f;
#pragma unroll
      for (int j = 0; j < NDOF; ++j)
        if (j == jm && j < n) ang = fmaf(q[j], rs.kth[j], rs.toff[j]);
      sincosf(ang, &ms[k], &mc[k]);
    }
#pragma unroll
    for (int j = 0; j < NDOF; ++j) {
      sj[j] = __shfl_sync(0xffffffffu, ms[j / T], j % T, T);
      cj[j] = __shfl_sync(0xffffffffu, mc[j / T], j % T, T);
    }
  }
#pragma unroll
  for (int f = 0; f <= NDOF; ++f) {
    if (f > n) break;
    if (f > 0) {
      const int j = f - 1;
      const float s = sj[j], c = cj[j];
      // R_{j} Rz(theta): col0' = c col0 + s col1, col1' = -s col0 + c col1
      const float n0x = fmaf(c, c0x, s * c1x), n0y = fmaf(c, c0y, s * c1y), n0z = fmaf(c, c0z, s * c1z);
      const float n1x = fmaf(c, c1x, -s * c0x), n1y = fmaf(c, c1y, -s * c0y), n1z = fmaf(c, c1z, -s * c0z);
      // o_{j+1} = o_j + a col0' + d col2
      const float aj = rs.a[j], dj = fmaf(q[j], rs.kd[j], rs.d[j]);
      px = fmaf(aj, n0x, fmaf(dj, c2x, px));
      py = fmaf(aj, n0y, fmaf(dj, c2y, py));
      pz = fmaf(aj, n0z, fmaf(dj, c2z, pz));
      // Rx(alpha): col1'' = ca col1' + sa col2, col2'' = -sa col1' + ca col2
      const float ca = rs.ca[j], sa = rs.sa[j];
      const float m1x = fmaf(ca, n1x, sa * c2x), m1y = fmaf(ca, n1y, sa * c2y), m1z = fmaf(ca, n1z, sa * c2z);
      const float m2x = fmaf(ca, c2x, -sa * n1x), m2y = fmaf(ca, c2y, -sa * n1y), m2z = fmaf(ca, c2z, -sa * n1z);
      c0x = n0x; c0y = n0y; c0z = n0z;
      c1x = m1x; c1y = m1y; c1z = m1z;
      c2x = m2x; c2y = m2y; c2z = m2z;
    }
    const int s_end = rs.frame_first[f + 1];
    int s = rs.frame_first[f];
    s += (lg - s) & (T - 1);
    for (; s < s_end; s += T) {
      const float4 l = sph_s[s];
      const float cx = fmaf(c0x, l.x, fmaf(c1x, l.y, fmaf(c2x, l.z, px)));
      const float cy = fmaf(c0y, l.x, fmaf(c1y, l.y, fmaf(c2y, l.z, py)));
      const float cz = fmaf(c0z, l.x, fmaf(c1z, l.y, fmaf(c2z, l.z, pz)));
      const float hu = 0.5f * fmaf(cx, cx, fmaf(cy, cy, fmaf(cz, cz, -l.w * l.w)));
      cen[s] = make_float4(cx, cy, cz, hu);
    }
    if constexpr (BOX)
      box_poses_of_frame<T>(rs.box_first[f], rs.box_first[f + 1], lg, make_float4(c0x, c0y, c0z, px),
                            make_float4(c1x, c1y, c1z, py), make_float4(c2x, c2y, c2z, pz), bx);
  }
  for (int s = rs.n_spheres + lg; s < rs.n_spheres_pad; s += T) cen[s] = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
  __syncwarp();
}

// One configuration evaluated by a group of T lanes of one warp (T in 1..8);
// BOX adds the box geometries (robot boxes posed along the chain, pairs with
// a box after the sphere pairs).
// Lane lg of the group computes the centres of spheres s with s % T == lg
// (every lane walks the chain), the group shares them through smem slot
// `cen`, then lane lg sweeps the obstacle pairs p (obstacles 2p, 2p + 1) with
// p % T == lg, and the self pairs: the work items it % T == lg when the
// pairs form link blocks, else the listed pairs p % T == lg. Returns the
// group-wide OR.
// Every lane of the warp must call this together (invalid configurations are
// evaluated and discarded).
template <int NDOF, int T, bool BOX = false>
__device__ __forceinline__ bool collide_group(const float (&q)[NDOF], const RobotSmem& rs,
                                              const float4* __restrict__ sph_s,
                                              const float4* __restrict__ obs_s,
                                              const float* __restrict__ nhw_s, int n_obs, int n_obs_pad,
                                              int s_first, const ushort2* __restrict__ self_pairs,
                                              const float* __restrict__ self_rr, float E,
                                              float4* __restrict__ cen, int lg, const BoxCtx& bx) {
  fk_group<NDOF, T, BOX>(q, rs, sph_s, cen, lg, bx);

  // ---- robot spheres vs obstacle spheres: one pair of obstacles per step,
  //      both evaluated by packed FP32 FMAs (each half is an fma.rn of its
  //      own, so t_ij is bit for bit the scalar chain's) ----
  bool hit = false;
  const int n_pairs = n_obs_pad >> 1;
  const float2* __restrict__ nhw2 = reinterpret_cast<const float2*>(nhw_s);
  for (int s0 = s_first; s0 < rs.n_spheres_pad; s0 += EZO_CH) {
    float2 cx[EZO_CH], cy[EZO_CH], cz[EZO_CH], cr[EZO_CH];
    float m[EZO_CH];
#pragma unroll
    for (int k = 0; k < EZO_CH; ++k) {
      const float4 c = cen[s0 + k];
      const float r = sph_s[s0 + k].w;
      cx[k] = make_float2(c.x, c.x);
      cy[k] = make_float2(c.y, c.y);
      cz[k] = make_float2(c.z, c.z);
      cr[k] = make_float2(r, r);
      m[k] = -3.0e38f;
    }
#pragma unroll 2
    for (int p = lg; p < n_pairs; p += T) {
      const float4 xy = obs_s[2 * p], zr = obs_s[2 * p + 1];
      const float2 w = nhw2[p];
      const float2 ox = make_float2(xy.x, xy.y), oy = make_float2(xy.z, xy.w);
      const float2 oz = make_float2(zr.x, zr.y), oR = make_float2(zr.z, zr.w);
#pragma unroll
      for (int k = 0; k < EZO_CH; ++k) {
        float2 t = __ffma2_rn(cr[k], oR, w);
        t = __ffma2_rn(cz[k], oz, t);
        t = __ffma2_rn(cy[k], oy, t);
        t = __ffma2_rn(cx[k], ox, t);
        m[k] = fmax3f(m[k], t.x, t.y);
      }
    }
    // spheres inside the rounding band of the fast form, as a bit mask; the
    // rare re-check is one rolled loop (short code: the unrolled sweep
    // already fills the instruction cache)
    unsigned band = 0u;
#pragma unroll
    for (int k = 0; k < EZO_CH; ++k) {
      const float diff = m[k] - cen[s0 + k].w;
      if (diff > E) hit = true;
      else if (diff >= -E) band |= 1u << k;
    }
    while (band) {
      // decide with differences, over the same obstacles as this lane's
      // maximum (its pairs)
      const int k = __ffs(band) - 1;
      band &= band - 1u;
      const float4 c = cen[s0 + k];
      const float r = sph_s[s0 + k].w;
      for (int j = 2 * lg; j < n_obs; j += (j & 1) ? 2 * T - 1 : 1) {
        const float4 o = obs_at(obs_s, j);
        const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float sr = r + o.w;
        if (d2 < sr * sr) hit = true;
      }
    }
  }
  // ---- self pairs ----
  if (rs.n_sblk > 0) {
    // work items (r0, nr, k0, nk) of up to EZO_CH rows, lane lg of the group
    // taking items lg, lg + T, .. (the lanes run the same instructions on
    // their own items); same fast form as the obstacles with the partner's
    // (c_k, r_k) as the obstacle and -hu_k as its offset. The partners go two
    // at a time through packed FP32 FMAs; each half is the scalar fma.rn
    // chain of its pair, and a missing second partner of an odd count gets
    // offset -inf, which no maximum keeps.
    const float Es = rs.E_self;
    for (int it0 = 0; it0 < rs.n_sblk; it0 += T) {
      const int it = it0 + lg;
      const int4 I = it < rs.n_sblk ? rs.sblk[it] : make_int4(0, 0, 0, 0);
      float2 cx[EZO_CH], cy[EZO_CH], cz[EZO_CH], cr[EZO_CH];
      float hu[EZO_CH], m[EZO_CH];
#pragma unroll
      for (int k = 0; k < EZO_CH; ++k) {
        const bool in = k < I.y;
        const float4 c = in ? cen[I.x + k] : make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
        const float r = in ? sph_s[I.x + k].w : 0.f;
        cx[k] = make_float2(c.x, c.x);
        cy[k] = make_float2(c.y, c.y);
        cz[k] = make_float2(c.z, c.z);
        cr[k] = make_float2(r, r);
        hu[k] = c.w;
        m[k] = -3.0e38f;
      }
      for (int u = 0; 2 * u < I.w; ++u) {
        const int qa = I.z + 2 * u;
        const bool two = 2 * u + 1 < I.w;
        const float4 a = cen[qa];
        const float4 b = two ? cen[qa + 1] : make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
        const float2 ox = make_float2(a.x, b.x), oy = make_float2(a.y, b.y), oz = make_float2(a.z, b.z);
        const float2 oR = make_float2(sph_s[qa].w, two ? sph_s[qa + 1].w : 0.f);
        const float2 w = make_float2(-a.w, -b.w);
#pragma unroll
        for (int k = 0; k < EZO_CH; ++k) {
          float2 t = __ffma2_rn(cr[k], oR, w);
          t = __ffma2_rn(cz[k], oz, t);
          t = __ffma2_rn(cy[k], oy, t);
          t = __ffma2_rn(cx[k], ox, t);
          m[k] = fmax3f(m[k], t.x, t.y);
        }
      }
      unsigned band = 0u;
#pragma unroll
      for (int k = 0; k < EZO_CH; ++k) {
        const float diff = m[k] - hu[k];
        if (diff > Es) hit = true;
        else if (diff >= -Es) band |= 1u << k;
      }
      while (band) {
        // rounding band: direct differences over the item's partners
        const int k = __ffs(band) - 1;
        band &= band - 1u;
        const float4 c = cen[I.x + k];
        const float r = sph_s[I.x + k].w;
        for (int q = I.z; q < I.z + I.w; ++q) {
          const float4 o = cen[q];
          const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z;
          const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float sr = r + sph_s[q].w;
          if (d2 < sr * sr) hit = true;
        }
      }
    }
  } else {
    // explicit pair list (direct difference form)
    for (int p = lg; p < rs.n_self; p += T) {
      const ushort2 pr = self_pairs[p];
      const float4 a = cen[pr.x], b = cen[pr.y];
      const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (d2 < self_rr[p]) hit = true;
    }
  }
  // ---- pairs with a box (direct tests; compiled only into the kernels for
  //      scenes with boxes, so sphere-only scenes keep their register budget) ----
  if constexpr (BOX) {
    if (!hit) hit = box_pairs_hit<T>(rs, sph_s, obs_s, n_obs, cen, lg, bx);
  }
  __syncwarp();
  if (T > 1) {
    unsigned h = hit ? 1u : 0u;
#pragma unroll
    for (int off = 1; off < T; off <<= 1) h |= __shfl_xor_sync(0xffffffffu, h, off, T);
    hit = h != 0u;
  }
  return hit;
}

// One configuration evaluated by a group of T = 16 or 32 lanes (sphere
// geometries only). The kinematics are fk_group's. The obstacle pairs are
// split two ways: lane lg = sg OG + og takes the robot spheres s with
// s % SG == sg (SG = T / OG) against the obstacle pairs p with p % OG == og,
// so each lane holds a few spheres for a few pairs instead of one chunk of
// spheres per handful of pairs; the same fast form, rounding band and direct
// re-check as collide_group decide each sphere, over the lane's obstacles.
// Self pairs come from the explicit pair list, p % T == lg, in the direct
// difference form. Returns the group-wide OR; every lane of the warp must
// call this together.
template <int NDOF, int T>
__device__ __forceinline__ bool collide_wide(const float (&q)[NDOF], const RobotSmem& rs,
                                             const float4* __restrict__ sph_s, const float4* __restrict__ obs_s,
                                             const float* __restrict__ nhw_s, int n_obs, int n_obs_pad,
                                             int s_first, const ushort2* __restrict__ self_pairs,
                                             const float* __restrict__ self_rr, float E,
                                             float4* __restrict__ cen, int lg, const BoxCtx& bx) {
  static_assert(T == 16 || T == 32, "wide groups are 16 or 32 lanes");
  constexpr int OG = 8, SG = T / OG, CW = 4;
  fk_group<NDOF, T, false>(q, rs, sph_s, cen, lg, bx);
  bool hit = false;
  const int n_pairs = n_obs_pad >> 1;
  const float2* __restrict__ nhw2 = reinterpret_cast<const float2*>(nhw_s);
  const int sg = lg / OG, og = lg % OG;
  const int nsp = rs.n_spheres_pad;
  for (int s0 = s_first + sg; s0 < nsp; s0 += SG * CW) {
    float2 cx[CW], cy[CW], cz[CW], cr[CW];
    float hu[CW], m[CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) {
      const int s = s0 + k * SG;
      const float4 c = s < nsp ? cen[s] : make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
      const float r = s < nsp ? sph_s[s].w : 0.f;
      cx[k] = make_float2(c.x, c.x);
      cy[k] = make_float2(c.y, c.y);
      cz[k] = make_float2(c.z, c.z);
      cr[k] = make_float2(r, r);
      hu[k] = c.w;
      m[k] = -3.0e38f;
    }
    for (int p = og; p < n_pairs; p += OG) {
      const float4 xy = obs_s[2 * p], zr = obs_s[2 * p + 1];
      const float2 w = nhw2[p];
      const float2 ox = make_float2(xy.x, xy.y), oy = make_float2(xy.z, xy.w);
      const float2 oz = make_float2(zr.x, zr.y), oR = make_float2(zr.z, zr.w);
#pragma unroll
      for (int k = 0; k < CW; ++k) {
        float2 t = __ffma2_rn(cr[k], oR, w);
        t = __ffma2_rn(cz[k], oz, t);
        t = __ffma2_rn(cy[k], oy, t);
        t = __ffma2_rn(cx[k], ox, t);
        m[k] = fmax3f(m[k], t.x, t.y);
      }
    }
    unsigned band = 0u;
#pragma unroll
    for (int k = 0; k < CW; ++k) {
      const float diff = m[k] - hu[k];
      if (diff > E) hit = true;
      else if (diff >= -E) band |= 1u << k;
    }
    while (band) {
      // inside the rounding band: direct differences over this lane's
      // obstacles (2p, 2p + 1 for its pairs p), in one rolled loop
      const int k = __ffs(band) - 1;
      band &= band - 1u;
      const int s = s0 + k * SG;
      const float4 c = cen[s];
      const float r = sph_s[s].w;
      for (int j = 2 * og; j < n_obs; j += (j & 1) ? 2 * OG - 1 : 1) {
        const float4 o = obs_at(obs_s, j);
        const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float sr = r + o.w;
        if (d2 < sr * sr) hit = true;
      }
    }
  }
#pragma unroll 4
  for (int p = lg; p < rs.n_self; p += T) {
    const ushort2 pr = self_pairs[p];
    const float4 a = cen[pr.x], b = cen[pr.y];
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (d2 < self_rr[p]) hit = true;
  }
  __syncwarp();
  unsigned h = hit ? 1u : 0u;
#pragma unroll
  for (int off = 1; off < T; off <<= 1) h |= __shfl_xor_sync(0xffffffffu, h, off, T);
  return h != 0u;
}

// Signed distance min over pairs of ||c_i - c_j|| - r_i - r_j for one
// configuration, one lane per configuration, exact below `cap` and equal to
// cap above it (a pair whose squared distance is at least (r_i + r_j + cap)^2
// cannot bring the minimum below cap, so its square root is skipped).
template <int NDOF>
__device__ float signed_distance_one(const float* __restrict__ q, const RobotSmem& rs,
                                     const float4* __restrict__ sph_s, const float4* __restrict__ obs_s,
                                     int n_obs, const ushort2* __restrict__ self_pairs,
                                     const float* __restrict__ self_rr, float4* __restrict__ cen,
                                     float cap) {
  float c0x = 1.f, c0y = 0.f, c0z = 0.f, c1x = 0.f, c1y = 1.f, c1z = 0.f, c2x = 0.f, c2y = 0.f, c2z = 1.f;
  float px = 0.f, py = 0.f, pz = 0.f;
  const int n = rs.n;
#pragma unroll
  for (int f = 0; f <= NDOF; ++f) {
    if (f > n) break;
    if (f > 0) {
      const int j = f - 1;
      float s, c;
      sincosf(fmaf(q[j], rs.kth[j], rs.toff[j]), &s, &c);
      const float n0x = fmaf(c, c0x, s * c1x), n0y = fmaf(c, c0y, s * c1y), n0z = fmaf(c, c0z, s * c1z);
      const float n1x = fmaf(c, c1x, -s * c0x), n1y = fmaf(c, c1y, -s * c0y), n1z = fmaf(c, c1z, -s * c0z);
      const float aj = rs.a[j], dj = fmaf(q[j], rs.kd[j], rs.d[j]);
      px = fmaf(aj, n0x, fmaf(dj, c2x, px));
      py = fmaf(aj, n0y, fmaf(dj, c2y, py));
      pz = fmaf(aj, n0z, fmaf(dj, c2z, pz));
      const float ca = rs.ca[j], sa = rs.sa[j];
      const float m1x = fmaf(ca, n1x, sa * c2x), m1y = fmaf(ca, n1y, sa * c2y), m1z = fmaf(ca, n1z, sa * c2z);
      const float m2x = fmaf(ca, c2x, -sa * n1x), m2y = fmaf(ca, c2y, -sa * n1y), m2z = fmaf(ca, c2z, -sa * n1z);
      c0x = n0x; c0y = n0y; c0z = n0z;
      c1x = m1x; c1y = m1y; c1z = m1z;
      c2x = m2x; c2y = m2y; c2z = m2z;
    }
    for (int s = rs.frame_first[f]; s < rs.frame_first[f + 1]; ++s) {
      const float4 l = sph_s[s];
      cen[s] = make_float4(fmaf(c0x, l.x, fmaf(c1x, l.y, fmaf(c2x, l.z, px))),
                           fmaf(c0y, l.x, fmaf(c1y, l.y, fmaf(c2y, l.z, py))),
                           fmaf(c0z, l.x, fmaf(c1z, l.y, fmaf(c2z, l.z, pz))), l.w);
    }
  }
  float best = cap;
  for (int s = 0; s < rs.n_spheres; ++s) {
    const float4 c = cen[s];
    for (int j = 0; j < n_obs; ++j) {
      const float4 o = obs_at(obs_s, j);
      const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float lim = c.w + o.w + best;
      if (lim > 0.f && d2 < lim * lim) best = fminf(best, sqrtf(d2) - c.w - o.w);
    }
  }
  for (int p = 0; p < rs.n_self; ++p) {
    const ushort2 pr = self_pairs[p];
    const float4 a = cen[pr.x], b = cen[pr.y];
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float lim = a.w + b.w + best;
    if (lim > 0.f && d2 < lim * lim) best = fminf(best, sqrtf(d2) - a.w - b.w);
  }
  return best;
}

}  // namespace ezo
