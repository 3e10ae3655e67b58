// One-call inflation entry points shaped like the paper's problem statement
// (robot, obstacles, segment or path, eps and delta in; polytopes A, b out):
// Algorithm 1 on one segment (Sec. IV-B), path inflation with the
// containment skip (Sec. VI-A), and many paths over several obstacle sets at
// once. Each call builds a batch with the public batch calls, runs it, copies
// the polytopes to host objects and frees the batch, so the device work is
// exactly that of ezo_batch_run / ezo_batch_run_path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ezo.h"

extern "C" void ezo_internal_set_error(const char* msg);

struct ezo_polytope {
  int32_t m = 0, n = 0, segment = -1;
  std::vector<double> A, b;
  ezo_stats stats{};
};

struct ezo_scs {
  std::vector<ezo_polytope*> sets;  // in path order; sets[i]->segment is the segment it was inflated for
};

namespace {

ezo_status api_fail(ezo_status s, const char* msg) {
  ezo_internal_set_error(msg);
  return s;
}

// The status a one-call inflation returns for a segment's outcome.
ezo_status segment_outcome(int32_t seg_status) {
  switch (seg_status) {
    case EZO_SEG_ACCEPTED: return EZO_OK;
    case EZO_SEG_IN_COLLISION: return EZO_ERR_SEGMENT_IN_COLLISION;
    case EZO_SEG_CAPACITY: return EZO_ERR_CAPACITY;
    case EZO_SEG_MAX_ITER: return EZO_WARN_MAX_ITER;
    default: return EZO_OK;
  }
}

// Severity order for a path's combined status: errors, then the warning.
int severity(ezo_status s) {
  if (s == EZO_OK) return 0;
  if (s == EZO_WARN_MAX_ITER) return 1;
  return 2;
}

// Segment g of a finished batch as a host polytope with its statistics.
ezo_status take_polytope(const ezo_batch* b, int32_t g, int32_t n, int32_t m_cap, ezo_polytope** out) {
  ezo_polytope* p = new (std::nothrow) ezo_polytope();
  if (!p) return api_fail(EZO_ERR_CAPACITY, "out of host memory");
  p->n = n;
  p->segment = g;
  p->A.resize((size_t)m_cap * n);
  p->b.resize((size_t)m_cap);
  ezo_status st = ezo_batch_get_polytope(b, g, &p->m, p->A.data(), p->b.data());
  int64_t work[3] = {0, 0, 0}, evals = 0;
  if (st == EZO_OK)
    st = ezo_batch_get_segment(b, g, &p->stats.status, &p->stats.rounds, &p->stats.m, &p->stats.planes,
                               &p->stats.checks);
  if (st == EZO_OK) st = ezo_batch_read(b, g, 9, work, sizeof(work));
  if (st == EZO_OK) st = ezo_batch_read(b, g, 11, &evals, sizeof(evals));
  if (st != EZO_OK) {
    delete p;
    return st;
  }
  p->A.resize((size_t)p->m * n);
  p->b.resize((size_t)p->m);
  p->stats.checks_bisect = work[1];
  p->stats.surrogate_evals = evals;
  *out = p;
  return EZO_OK;
}

}  // namespace

extern "C" {

ezo_status ezo_inflate_segment(const ezo_robot* robot, const ezo_env* env, const double* v1, const double* v2,
                               const double* A0, const double* b0, int32_t m0, const ezo_params* params,
                               uint32_t stream_id, ezo_polytope** out, ezo_stats* stats, void* cuda_stream) {
  if (!out) return api_fail(EZO_ERR_INVALID_ARG, "ezo_inflate_segment: out is NULL");
  *out = nullptr;
  if (!robot || !env || !v1 || !v2 || !params || (A0 && (!b0 || m0 < 1)) || (!A0 && m0 != 0))
    return api_fail(EZO_ERR_INVALID_ARG, "ezo_inflate_segment: bad argument");
  ezo_batch* b = nullptr;
  const ezo_env* envs[1] = {env};
  ezo_status st = ezo_batch_create(robot, 1, envs, 1, v1, v2, nullptr, nullptr, &stream_id, nullptr, A0, b0, m0,
                                   params, &b);
  if (st != EZO_OK) return st;
  st = ezo_batch_run(b, EZO_RUN_HOST_LOOP, cuda_stream);
  int32_t m_cap = 0;
  if (st == EZO_OK) st = ezo_batch_capacity(b, &m_cap, nullptr);
  ezo_polytope* p = nullptr;
  if (st == EZO_OK) st = take_polytope(b, 0, ezo_robot_dof(robot), m_cap, &p);
  ezo_batch_free(b);
  if (st != EZO_OK) return st;
  if (stats) *stats = p->stats;
  *out = p;
  const ezo_status outcome = segment_outcome(p->stats.status);
  ezo_internal_set_error(outcome == EZO_OK ? "" : "ezo_inflate_segment: see the polytope's status");
  return outcome;
}

ezo_status ezo_inflate_batch(const ezo_robot* robot, int32_t n_env, const ezo_env* const* envs, int32_t n_path,
                             const int32_t* path_len, const double* verts, const int32_t* path_env,
                             const int32_t* seg_np, const double* A0, const double* b0, int32_t m0,
                             const ezo_params* params, int32_t mode, uint32_t stream_base, ezo_scs** out,
                             void* cuda_stream) {
  if (!out) return api_fail(EZO_ERR_INVALID_ARG, "ezo_inflate_batch: out is NULL");
  for (int32_t i = 0; i < n_path; ++i) out[i] = nullptr;
  if (!robot || n_env < 1 || !envs || n_path < 1 || !path_len || !verts || !params || mode < 0 || mode > 2 ||
      (A0 && (!b0 || m0 < 1)) || (!A0 && m0 != 0))
    return api_fail(EZO_ERR_INVALID_ARG, "ezo_inflate_batch: bad argument");
  const int32_t n = ezo_robot_dof(robot);
  std::vector<double> v1, v2;
  std::vector<int32_t> seg_env, path_first;
  std::vector<uint32_t> seg_stream;
  std::vector<int32_t> first_seg(n_path, 0);
  long long vo = 0;
  for (int32_t i = 0; i < n_path; ++i) {
    if (path_len[i] < 1) return api_fail(EZO_ERR_INVALID_ARG, "ezo_inflate_batch: a path needs at least one segment");
    const int32_t e = path_env ? path_env[i] : 0;
    if (e < 0 || e >= n_env) return api_fail(EZO_ERR_INVALID_ARG, "ezo_inflate_batch: path_env out of range");
    first_seg[i] = (int32_t)seg_env.size();
    for (int32_t k = 0; k < path_len[i]; ++k) {
      const double* a = verts + (vo + k) * n;
      v1.insert(v1.end(), a, a + n);
      v2.insert(v2.end(), a + n, a + 2 * n);
      seg_env.push_back(e);
      path_first.push_back(first_seg[i]);
      seg_stream.push_back(stream_base + (uint32_t)seg_env.size() - 1u);
    }
    vo += path_len[i] + 1;
  }
  const int32_t B = (int32_t)seg_env.size();
  ezo_batch* b = nullptr;
  ezo_status st = ezo_batch_create(robot, n_env, envs, B, v1.data(), v2.data(), seg_env.data(), seg_np,
                                   seg_stream.data(), path_first.data(), A0, b0, m0, params, &b);
  if (st != EZO_OK) return st;
  // mode 0: the paper's order (one segment at a time); 1: wavefront (the
  // current segment of every path in one graph launch per wave); 2: every
  // segment speculatively in one graph, the skip rule afterwards
  const int32_t seq = mode == 0 ? 1 : (mode == 1 ? 2 : 0);
  st = ezo_batch_run_path(b, seq, mode == 0 ? EZO_RUN_HOST_LOOP : EZO_RUN_GRAPH, cuda_stream);
  int32_t m_cap = 0;
  if (st == EZO_OK) st = ezo_batch_capacity(b, &m_cap, nullptr);
  std::vector<int32_t> status(B), mm(B);
  if (st == EZO_OK) st = ezo_batch_get_polytopes(b, status.data(), mm.data(), nullptr, nullptr, 0, nullptr, cuda_stream);
  ezo_status worst = EZO_OK;
  for (int32_t i = 0; i < n_path && st == EZO_OK; ++i) {
    ezo_scs* scs = new (std::nothrow) ezo_scs();
    if (!scs) {
      st = api_fail(EZO_ERR_CAPACITY, "out of host memory");
      break;
    }
    out[i] = scs;
    for (int32_t k = 0; k < path_len[i] && st == EZO_OK; ++k) {
      const int32_t g = first_seg[i] + k;
      if (status[g] == EZO_SEG_SKIPPED || status[g] == EZO_SEG_IDLE) continue;
      ezo_polytope* p = nullptr;
      st = take_polytope(b, g, n, m_cap, &p);
      if (st != EZO_OK) break;
      p->segment = k;
      scs->sets.push_back(p);
      const ezo_status o = segment_outcome(status[g]);
      if (severity(o) > severity(worst)) worst = o;
    }
  }
  ezo_batch_free(b);
  if (st != EZO_OK) {
    for (int32_t i = 0; i < n_path; ++i) {
      ezo_scs_free(out[i]);
      out[i] = nullptr;
    }
    return st;
  }
  ezo_internal_set_error(worst == EZO_OK ? "" : "ezo_inflate_batch: see the polytopes' status");
  return worst;
}

ezo_status ezo_inflate_path(const ezo_robot* robot, const ezo_env* env, const double* verts, int32_t n_verts,
                            const double* A0, const double* b0, int32_t m0, const ezo_params* params, int32_t mode,
                            uint32_t stream_base, ezo_scs** out, void* cuda_stream) {
  if (!out) return api_fail(EZO_ERR_INVALID_ARG, "ezo_inflate_path: out is NULL");
  *out = nullptr;
  if (n_verts < 2) return api_fail(EZO_ERR_INVALID_ARG, "ezo_inflate_path: a path needs at least two vertices");
  const ezo_env* envs[1] = {env};
  const int32_t len = n_verts - 1;
  return ezo_inflate_batch(robot, 1, envs, 1, &len, verts, nullptr, nullptr, A0, b0, m0, params, mode, stream_base,
                           out, cuda_stream);
}

ezo_status ezo_polytope_get(const ezo_polytope* p, int32_t* m, int32_t* n, double* A, double* b) {
  if (!p) return api_fail(EZO_ERR_INVALID_ARG, "ezo_polytope_get: null polytope");
  if (m) *m = p->m;
  if (n) *n = p->n;
  if (A && p->m) std::memcpy(A, p->A.data(), sizeof(double) * (size_t)p->m * p->n);
  if (b && p->m) std::memcpy(b, p->b.data(), sizeof(double) * (size_t)p->m);
  return EZO_OK;
}

ezo_status ezo_polytope_stats(const ezo_polytope* p, int32_t* segment, ezo_stats* stats) {
  if (!p) return api_fail(EZO_ERR_INVALID_ARG, "ezo_polytope_stats: null polytope");
  if (segment) *segment = p->segment;
  if (stats) *stats = p->stats;
  return EZO_OK;
}

void ezo_polytope_free(ezo_polytope* p) { delete p; }

int32_t ezo_scs_size(const ezo_scs* s) { return s ? (int32_t)s->sets.size() : 0; }

const ezo_polytope* ezo_scs_get(const ezo_scs* s, int32_t i) {
  if (!s || i < 0 || i >= (int32_t)s->sets.size()) return nullptr;
  return s->sets[i];
}

void ezo_scs_free(ezo_scs* s) {
  if (!s) return;
  for (ezo_polytope* p : s->sets) delete p;
  delete s;
}

}  // extern "C"
