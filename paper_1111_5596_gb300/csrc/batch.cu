// Batched smearing + mesons over many independent jobs of uneven size and
// iteration count (the paper's SNK + HAD stages run for many sources at
// once, Sec. 5).
//
// Jobs are grouped into classes of equal lattice and precisions.  Step k of
// the plan runs one hop for every job of a class whose iteration count
// exceeds k, in a single launch of the pipelined multi-job kernel (the work
// items of all those jobs share one persistent grid); jobs drop out as their
// own count is reached.  After the last step, jobs with an odd count copy
// their result back from the scratch buffer and the sixteen meson
// correlators at zero momentum are contracted per job.  Float16 jobs use
// the tensor-core hop and carry their per-iteration scale slots (set up
// before the first step, folded into each field's scale after the last).
// qdpg_batch_run can
// replay the whole sequence as one CUDA graph: the first run executes the
// launches directly (which also performs every lazy set-up) and captures
// them; later runs launch the graph.
#include <algorithm>
#include <new>
#include <vector>

#include "qdpg_internal.h"

extern "C" int qdpg_meson_2pt(qdpg_field_t S1, qdpg_field_t S2, const int* gamma_snk, const int* gamma_src,
                              int n_chan, const int* moms, int n_mom, const int origin[4], double* out_dev,
                              void* stream);

namespace qdpg {
namespace {

struct Job {
  qdpg_field U, psi, scratch;  // copies of the caller's headers
  float kappa;
  int n_iter;
  double* mesons;
};

struct JobClass {
  std::vector<int> jobs;
};

bool same_geom(const Geom& a, const Geom& b) {
  for (int mu = 0; mu < 4; ++mu)
    if (a.L[mu] != b.L[mu]) return false;
  return a.jd == b.jd;
}

}  // namespace
}  // namespace qdpg

struct qdpg_batch {
  std::vector<qdpg::Job> jobs;
  std::vector<qdpg::JobClass> classes;
  int j_decay;
  int max_iter;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool captured;
  uint64_t graph_kernels;  // kernel launches inside the graph
};

namespace qdpg {
namespace {

// All launches of one batch run, in order, on `s`.
int issue(qdpg_batch* b, cudaStream_t s) {
  int hop_mu[3], k = 0;
  for (int mu = 0; mu < 4; ++mu)
    if (mu != b->j_decay) hop_mu[k++] = mu;
  std::vector<const void*> in, U;
  std::vector<void*> out;
  std::vector<float> kap;
  // float16 jobs: their scale slots (slot 0 = the field's scale)
  std::vector<ScaleRecord*> recs;
  std::vector<int> niters;
  for (const Job& J : b->jobs)
    if (J.psi.prec == QDPG_F16 && J.n_iter > 0) {
      recs.push_back(J.psi.rec);
      niters.push_back(J.n_iter);
    }
  for (size_t off = 0; off < recs.size(); off += kMaxF16Jobs) {
    const int n = (int)std::min<size_t>(kMaxF16Jobs, recs.size() - off);
    int rc = f16_scale_init(recs.data() + off, niters.data() + off, n, s);
    if (rc != QDPG_OK) return rc;
  }
  std::vector<F16HopJob> hjobs;
  for (int it = 0; it < b->max_iter; ++it) {
    for (const JobClass& c : b->classes) {
      if (b->jobs[c.jobs[0]].psi.prec == QDPG_F16) {
        hjobs.clear();
        for (int j : c.jobs) {
          const Job& J = b->jobs[j];
          if (J.n_iter <= it) continue;
          void* bufs[2] = {J.psi.data, J.scratch.data};
          hjobs.push_back(F16HopJob{bufs[it & 1], bufs[(it + 1) & 1], J.U.data, J.kappa, J.psi.rec});
        }
        const Job& J0 = b->jobs[c.jobs[0]];
        for (size_t off = 0; off < hjobs.size(); off += kMaxF16Jobs) {
          const int n = (int)std::min<size_t>(kMaxF16Jobs, hjobs.size() - off);
          int rc = launch_hop_f16(hjobs.data() + off, n, J0.U.prec, J0.psi.g, it, s);
          if (rc != QDPG_OK) return rc;
        }
        continue;
      }
      in.clear();
      out.clear();
      U.clear();
      kap.clear();
      for (int j : c.jobs) {
        const Job& J = b->jobs[j];
        if (J.n_iter <= it) continue;
        void* bufs[2] = {J.psi.data, J.scratch.data};
        in.push_back(bufs[it & 1]);
        out.push_back(bufs[(it + 1) & 1]);
        U.push_back(J.U.data);
        kap.push_back(J.kappa);
      }
      if (in.empty()) continue;
      const Job& J0 = b->jobs[c.jobs[0]];
      const int cols = J0.psi.kind == QDPG_PROPAGATOR ? 12 : 1;
      int rc = QDPG_ERR_UNSUPPORTED;
      for (size_t off = 0; off < in.size();) {
        const int n = (int)std::min<size_t>(64, in.size() - off);
        rc = cols == 12 ? launch_hop_tma_batch(in.data() + off, out.data() + off, U.data() + off, kap.data() + off, n,
                                               J0.U.prec, J0.psi.prec, J0.psi.g, hop_mu, s)
                        : QDPG_ERR_UNSUPPORTED;
        if (rc == QDPG_ERR_UNSUPPORTED) break;
        if (rc != QDPG_OK) return rc;
        off += n;
      }
      if (rc == QDPG_ERR_UNSUPPORTED) {  // one launch per job with whichever kernel serves it
        for (size_t i = 0; i < in.size(); ++i) {
          rc = launch_hop_any(in[i], out[i], U[i], J0.U.prec, J0.psi.prec, cols, J0.psi.g, hop_mu, kap[i], s);
          if (rc != QDPG_OK) return rc;
        }
      }
      // FP32/BF16 jobs whose growth bound needs it: exact power-of-two rescale
      for (int j : c.jobs) {
        const Job& J = b->jobs[j];
        if (J.n_iter <= it) continue;
        const RescalePlan plan = rescale_plan(J.kappa, J.n_iter);
        if (plan.every && (it + 1) % plan.every == 0) {
          void* latest = (it + 1) & 1 ? J.scratch.data : J.psi.data;
          rc = launch_rescale(latest, J.psi.prec, J.psi.g.V * J.psi.ncomp, plan.shift, J.psi.rec, s);
          if (rc != QDPG_OK) return rc;
        }
      }
    }
  }
  for (size_t off = 0; off < recs.size(); off += kMaxF16Jobs) {
    const int n = (int)std::min<size_t>(kMaxF16Jobs, recs.size() - off);
    int rc = f16_scale_final(recs.data() + off, niters.data() + off, n, s);
    if (rc != QDPG_OK) return rc;
  }
  static const int chans[16] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15};
  static const int zero[3] = {0, 0, 0};
  for (Job& J : b->jobs) {
    if (J.n_iter & 1) {
      const size_t bytes = (size_t)J.psi.g.V * J.psi.ncomp * J.psi.esize;
      cudaError_t e = cudaMemcpyAsync(J.psi.data, J.scratch.data, bytes, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "batch: copy-back: %s", cudaGetErrorString(e));
    }
    if (J.mesons) {
      int rc = qdpg_meson_2pt(&J.psi, &J.psi, chans, chans, 16, zero, 1, nullptr, J.mesons, s);
      if (rc != QDPG_OK) return rc;
    }
  }
  return QDPG_OK;
}

}  // namespace
}  // namespace qdpg

using namespace qdpg;

extern "C" {

int qdpg_batch_create(const qdpg_job* jobs, int njobs, int j_decay, qdpg_batch_t* out) {
  if (!jobs || !out) return fail(QDPG_ERR_ARG, "batch_create: null argument");
  if (njobs < 1 || njobs > 4096) return fail(QDPG_ERR_ARG, "batch_create: njobs %d outside 1..4096", njobs);
  if (j_decay < 0 || j_decay > 3) return fail(QDPG_ERR_ARG, "batch_create: j_decay %d outside 0..3", j_decay);
  qdpg_batch* b = new (std::nothrow) qdpg_batch();
  if (!b) return fail(QDPG_ERR_NOMEM, "batch_create: out of host memory");
  b->j_decay = j_decay;
  b->max_iter = 0;
  b->graph = nullptr;
  b->exec = nullptr;
  b->captured = false;
  b->graph_kernels = 0;
  for (int i = 0; i < njobs; ++i) {
    const qdpg_job& q = jobs[i];
    if (!q.U || !q.psi || !q.scratch) {
      delete b;
      return fail(QDPG_ERR_ARG, "batch_create: job %d has a null field", i);
    }
    if (q.U->kind != QDPG_GAUGE || (q.psi->kind != QDPG_PROPAGATOR && q.psi->kind != QDPG_FERMION) ||
        q.scratch->kind != q.psi->kind || q.scratch->prec != q.psi->prec || q.scratch->data == q.psi->data ||
        !same_geom(q.U->g, q.psi->g) || !same_geom(q.scratch->g, q.psi->g) ||
        (q.psi->prec != QDPG_F32 && q.psi->prec != QDPG_BF16 && q.psi->prec != QDPG_F16)) {
      delete b;
      return fail(QDPG_ERR_SHAPE, "batch_create: job %d: fields do not match (gauge, psi, distinct scratch)", i);
    }
    if ((q.psi->prec == QDPG_F16) != is_f16(q.U->prec)) {
      delete b;
      return fail(QDPG_ERR_DTYPE, "batch_create: job %d: F16 propagators go with F16/F16_R12 links only", i);
    }
    if (q.psi->prec == QDPG_F16 && (j_decay != q.psi->g.jd || q.n_iter > QDPG_F16_MAX_ITER)) {
      delete b;
      return fail(QDPG_ERR_UNSUPPORTED, "batch_create: job %d: F16 smearing needs the lattice's decay direction "
                                        "and at most %d iterations", i, QDPG_F16_MAX_ITER);
    }
    if (q.n_iter < 0 || !(q.kappa == q.kappa)) {
      delete b;
      return fail(QDPG_ERR_ARG, "batch_create: job %d: bad iteration count or kappa", i);
    }
    if (q.mesons_out && q.psi->kind != QDPG_PROPAGATOR) {
      delete b;
      return fail(QDPG_ERR_SHAPE, "batch_create: job %d: mesons need a propagator", i);
    }
    Job J{*q.U, *q.psi, *q.scratch, (float)q.kappa, q.n_iter, q.mesons_out};
    b->jobs.push_back(J);
    b->max_iter = std::max(b->max_iter, q.n_iter);
    // class: same lattice, kind and precisions
    bool placed = false;
    for (JobClass& c : b->classes) {
      const Job& R = b->jobs[c.jobs[0]];
      if (same_geom(R.psi.g, J.psi.g) && R.psi.kind == J.psi.kind && R.psi.prec == J.psi.prec &&
          R.U.prec == J.U.prec) {
        c.jobs.push_back(i);
        placed = true;
        break;
      }
    }
    if (!placed) b->classes.push_back(JobClass{{i}});
  }
  *out = b;
  return ok();
}

int qdpg_batch_run(qdpg_batch_t b, int use_graph, void* stream) {
  if (!b) return fail(QDPG_ERR_ARG, "batch_run: null batch");
  cudaStream_t s = as_stream(stream);
  if (!use_graph) return issue(b, s);
  if (b->captured) {
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "batch_run: graph launch: %s", cudaGetErrorString(e));
    count_launches(b->graph_kernels);
    return ok();
  }
  // first run: execute directly (lazy set-up happens here), then capture.
  // The capture goes to a stream of the batch's own: the caller's stream may
  // be the legacy default stream, which cannot be captured.  Nothing runs
  // on it, so it needs no ordering with `s`.
  int rc = issue(b, s);
  if (rc != QDPG_OK) return rc;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "batch_run: capture stream: %s", cudaGetErrorString(e));
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(QDPG_ERR_CUDA, "batch_run: begin capture: %s", cudaGetErrorString(e));
  }
  const uint64_t before = qdpg_launch_count();
  rc = issue(b, cs);
  const uint64_t captured_kernels = qdpg_launch_count() - before;
  count_launches(0 - captured_kernels);  // captured, not run
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (rc != QDPG_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "batch_run: end capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(QDPG_ERR_CUDA, "batch_run: instantiate: %s", cudaGetErrorString(e));
  }
  b->graph = g;
  b->exec = x;
  b->captured = true;
  b->graph_kernels = captured_kernels;
  return ok();
}

void qdpg_batch_destroy(qdpg_batch_t b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

}  // extern "C"
