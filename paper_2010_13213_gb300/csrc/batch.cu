// batch.cu -- many independent solves as one unit of work, and its CUDA-graph capture.
//
// A batch holds N instances (each its own composite mesh, sharing the LGF table and its block size)
// and S internal streams.  A stage runs, for every instance i,
//     phi_i = L^{-1} f_i          (FLGF-AMR, Sec. 3.4)
//     g_i   = E_{alpha_i} * f_i   (FIF-AMR, Sec. 3.5; alpha_i for the finest level)
// -- the two solves a half-explicit Runge-Kutta stage needs (Sec. 2.4, Eqs. (eq:projection-1) and
// (eq:projection-2)).  Instances are dealt to the streams longest-first (a host work queue in LPT
// order), each stream runs its instances back to back, and the streams fork from / join into the
// caller's stream through events, so a stage is capturable: lgf_batch_graph_create captures a chain
// of stages (stage s reads the g written by stage s-1) into one CUDA graph, replayed by
// lgf_batch_graph_launch with a single launch.
#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.h"
#include "solver.h"

struct lgf_batch {
  lgf_table *t = nullptr;
  int n = 0, ncomp = 1, dtype = 0, nstreams = 1;
  lgf_solve_opts opts{};
  std::vector<int32_t> nb_all, ijk_all;           // concatenated mesh arrays
  std::vector<lgf_mesh> mesh;                      // per instance (pointers into the arrays above)
  std::vector<std::vector<int32_t>> nbk, ijk;      // per instance owned copies
  std::vector<double> alpha;
  std::vector<double> cost;
  std::vector<lgf_solve_opts> opts_i;             // per instance (the autotuner's DFT-pass choice)
  std::vector<double> tuned_ms;                   // per instance: measured solve time (ms), 0 before tuning
  bool tuned = false;
  std::vector<std::vector<int>> by_stream;         // instance lists per stream
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  // host transfers (lgf_batch_graph_create_io): one copy-in and one copy-out stream, per-instance events
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_done;
  cudaEvent_t ev_cin = nullptr, ev_cout = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_stages = 0;
  bool warmed = false;
};

namespace lgf {
double box_cost(int B, const int nb[3]);
}

using namespace lgf;

// Bytes of one field of instance i (ncomp components over all its blocks).
static size_t field_bytes(const lgf_batch *b, int i) {
  int64_t tot = 0;
  for (int k = 0; k < b->mesh[i].nlevels; ++k) tot += b->mesh[i].nblocks[k];
  const size_t B3 = (size_t)b->mesh[i].block * b->mesh[i].block * b->mesh[i].block;
  return (size_t)b->ncomp * (size_t)tot * B3 * (b->dtype == LGF_F64 ? 8 : 4);
}

// The copy streams and per-instance events of the host-transfer path (created once).
static int io_resources(lgf_batch *b) {
  if (b->copy_in) return LGF_OK;
  auto ev = [](cudaEvent_t *e) { return cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess; };
  b->ev_in.assign(b->n, nullptr);
  b->ev_done.assign(b->n, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->copy_in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->copy_out, cudaStreamNonBlocking) == cudaSuccess && ev(&b->ev_cin) &&
            ev(&b->ev_cout);
  for (int i = 0; i < b->n && ok; ++i) ok = ev(&b->ev_in[i]) && ev(&b->ev_done[i]);
  return ok ? LGF_OK : set_error(LGF_E_CUDA, "batch copy stream creation failed");
}

// One stage over all instances.  With f_host / phi_host (pinned host buffers): the sources are copied in on
// a copy stream in the order the solves start, each solve waits for its own source only, and the results
// are copied out on a second copy stream in the order the solves are expected to end (from the measured
// or block-count weights), so the transfers overlap the solves of the other instances.
static int batch_stage(lgf_batch *b, const void *const *f, void *const *phi, void *const *g, const double *alpha,
                       cudaStream_t st, const void *const *f_host = nullptr, void *const *phi_host = nullptr) {
  if (cudaEventRecord(b->ev_fork, st) != cudaSuccess) return set_error(LGF_E_CUDA, "batch fork event failed");
  const bool io = f_host && phi_host;
  std::vector<int> by_start, by_end;
  if (io) {
    int rc = io_resources(b);
    if (rc) return rc;
    const std::vector<double> &w = b->tuned ? b->tuned_ms : b->cost;
    std::vector<double> t0(b->n, 0.0), t1(b->n, 0.0);
    for (int s = 0; s < b->nstreams; ++s) {
      double t = 0.0;
      for (int i : b->by_stream[s]) t0[i] = t, t += w[i], t1[i] = t;
    }
    by_start.resize(b->n);
    for (int i = 0; i < b->n; ++i) by_start[i] = i;
    by_end = by_start;
    std::stable_sort(by_start.begin(), by_start.end(), [&](int a, int c) { return t0[a] < t0[c]; });
    std::stable_sort(by_end.begin(), by_end.end(), [&](int a, int c) { return t1[a] < t1[c]; });
    cudaStreamWaitEvent(b->copy_in, b->ev_fork, 0);
    for (int i : by_start) {
      if (cudaMemcpyAsync((void *)f[i], f_host[i], field_bytes(b, i), cudaMemcpyHostToDevice, b->copy_in) !=
          cudaSuccess)
        return set_error(LGF_E_CUDA, "instance %d: source copy failed", i);
      cudaEventRecord(b->ev_in[i], b->copy_in);
    }
    cudaEventRecord(b->ev_cin, b->copy_in);
  }
  for (int s = 0; s < b->nstreams; ++s) {
    cudaStream_t ss = b->streams[s];
    cudaStreamWaitEvent(ss, b->ev_fork, 0);
    for (int i : b->by_stream[s]) {
      if (io) cudaStreamWaitEvent(ss, b->ev_in[i], 0);
      int rc = lgf_poisson_solve(b->t, &b->mesh[i], b->ncomp, f[i], phi[i], b->dtype, &b->opts_i[i], nullptr, ss);
      if (rc) return rc;
      if (io) cudaEventRecord(b->ev_done[i], ss);
      if (g && g[i]) {
        rc = lgf_heat_apply(b->t, &b->mesh[i], b->ncomp, f[i], g[i], b->dtype, alpha ? alpha[i] : b->alpha[i],
                            &b->opts, nullptr, ss);
        if (rc) return rc;
      }
    }
    cudaEventRecord(b->ev_join[s], ss);
    cudaStreamWaitEvent(st, b->ev_join[s], 0);
  }
  if (io) {
    cudaStreamWaitEvent(b->copy_out, b->ev_fork, 0);
    for (int i : by_end) {
      cudaStreamWaitEvent(b->copy_out, b->ev_done[i], 0);
      if (cudaMemcpyAsync(phi_host[i], phi[i], field_bytes(b, i), cudaMemcpyDeviceToHost, b->copy_out) !=
          cudaSuccess)
        return set_error(LGF_E_CUDA, "instance %d: result copy failed", i);
    }
    cudaEventRecord(b->ev_cout, b->copy_out);
    cudaStreamWaitEvent(st, b->ev_cin, 0);
    cudaStreamWaitEvent(st, b->ev_cout, 0);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "batch stage: %s", cudaGetErrorString(e));
}

// Longest-processing-time-first assignment of the instances to `nstreams` streams (created on demand),
// by the measured solve times once the batch is tuned, else by block counts.
static int schedule(lgf_batch *b, int nstreams) {
  nstreams = std::max(1, std::min(nstreams, b->n));
  const std::vector<double> &w = b->tuned ? b->tuned_ms : b->cost;
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int c) { return w[a] > w[c]; });
  b->by_stream.assign(nstreams, {});
  std::vector<double> load(nstreams, 0.0);
  for (int i : order) {
    const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->by_stream[s].push_back(i);
    load[s] += w[i];
  }
  while ((int)b->streams.size() < nstreams) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return set_error(LGF_E_CUDA, "batch stream creation failed");
    b->streams.push_back(s);
    b->ev_join.push_back(e);
  }
  b->nstreams = nstreams;
  return LGF_OK;
}

extern "C" {

int lgf_batch_create(lgf_batch **out, lgf_table *t, int32_t ninst, const lgf_mesh *meshes, int32_t ncomp,
                     int32_t dtype, const double *alpha, const lgf_solve_opts *opts, int32_t nstreams) {
  if (!out || !t || !meshes || ninst < 1 || ncomp < 1) return set_error(LGF_E_INVALID_ARG, "bad batch arguments");
  if (dtype != LGF_F64 && dtype != LGF_F32) return set_error(LGF_E_INVALID_ARG, "dtype %d", dtype);
  if (nstreams < 1 || nstreams > 64) return set_error(LGF_E_INVALID_ARG, "nstreams %d out of [1, 64]", nstreams);
  *out = nullptr;
  lgf_batch *b = new lgf_batch();
  b->t = t;
  b->n = ninst;
  b->ncomp = ncomp;
  b->dtype = dtype;
  b->nstreams = std::min<int>(nstreams, ninst);
  if (opts) b->opts = *opts;
  b->opts.residual = 0;  // stages must stay free of synchronisation
  b->opts.timing = 0;
  b->mesh.resize(ninst);
  b->nbk.resize(ninst);
  b->ijk.resize(ninst);
  b->alpha.assign(ninst, 0.0);
  b->cost.assign(ninst, 0.0);
  for (int i = 0; i < ninst; ++i) {
    const lgf_mesh &m = meshes[i];
    if (!m.nblocks || !m.block_ijk || m.nlevels < 1 || m.block != t->B) {
      delete b;
      return set_error(LGF_E_MESH, "instance %d: invalid mesh", i);
    }
    int64_t tot = 0;
    for (int k = 0; k < m.nlevels; ++k) tot += m.nblocks[k];
    b->nbk[i].assign(m.nblocks, m.nblocks + m.nlevels);
    b->ijk[i].assign(m.block_ijk, m.block_ijk + 3 * tot);
    b->mesh[i] = m;
    b->mesh[i].nblocks = b->nbk[i].data();
    b->mesh[i].block_ijk = b->ijk[i].data();
    b->mesh[i].block_role = nullptr;
    b->alpha[i] = alpha ? alpha[i] : 0.0;
    b->cost[i] = (double)tot;
  }
  b->opts_i.assign(ninst, b->opts);
  b->tuned_ms.assign(ninst, 0.0);
  int rc = schedule(b, b->nstreams);
  if (rc) {
    delete b;
    return rc;
  }
  if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return set_error(LGF_E_CUDA, "batch event creation failed");
  }
  *out = b;
  return LGF_OK;
}

int lgf_batch_destroy(lgf_batch *b) {
  if (!b) return LGF_OK;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->ev_join) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->copy_in) cudaStreamDestroy(b->copy_in);
  if (b->copy_out) cudaStreamDestroy(b->copy_out);
  for (auto e : b->ev_in) if (e) cudaEventDestroy(e);
  for (auto e : b->ev_done) if (e) cudaEventDestroy(e);
  if (b->ev_cin) cudaEventDestroy(b->ev_cin);
  if (b->ev_cout) cudaEventDestroy(b->ev_cout);
  delete b;
  return LGF_OK;
}

int lgf_batch_stage(lgf_batch *b, const void *const *f_dev, void *const *phi_dev, void *const *g_dev,
                    const double *alpha, void *cuda_stream) {
  if (!b || !f_dev || !phi_dev) return set_error(LGF_E_INVALID_ARG, "NULL argument");
  int rc = batch_stage(b, f_dev, phi_dev, g_dev, alpha, (cudaStream_t)cuda_stream);
  if (!rc) b->warmed = true;
  return rc;
}

int lgf_batch_graph_create(lgf_batch *b, int32_t nstages, const void *const *f_dev, void *const *phi_dev,
                           void *const *g_dev, void *const *tmp_dev, const double *alpha_stages,
                           void *cuda_stream) {
  if (!b || !f_dev || !phi_dev || nstages < 1) return set_error(LGF_E_INVALID_ARG, "NULL argument");
  const bool heat = g_dev != nullptr;
  if (heat && nstages > 1 && !tmp_dev) return set_error(LGF_E_INVALID_ARG, "chained stages need tmp buffers");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  auto alpha_of = [&](int s) { return alpha_stages ? alpha_stages + (size_t)s * b->n : nullptr; };
  std::vector<const void *> src(b->n);
  std::vector<void *> dst(b->n);
  auto buffers_of = [&](int s) {
    for (int i = 0; i < b->n; ++i) {
      if (!heat || s == 0) src[i] = f_dev[i], dst[i] = heat ? g_dev[i] : nullptr;
      else if (s % 2 == 1) src[i] = g_dev[i], dst[i] = tmp_dev[i];
      else src[i] = tmp_dev[i], dst[i] = g_dev[i];
    }
  };
  // every stage once eagerly: builds each plan (the heat plans depend on the stage's alpha), spectrum and
  // workspace the captured stages use, so nothing allocates during the capture
  int rc = LGF_OK;
  for (int s = 0; s < nstages && !rc; ++s) {
    buffers_of(s);
    rc = batch_stage(b, src.data(), phi_dev, heat ? dst.data() : nullptr, alpha_of(s), st);
  }
  if (rc) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) return set_error(LGF_E_CUDA, "batch warm-up failed");
  if (b->exec) cudaGraphExecDestroy(b->exec), b->exec = nullptr;
  if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return set_error(LGF_E_CUDA, "stream capture could not begin (use a non-default stream)");
  for (int s = 0; s < nstages && !rc; ++s) {
    buffers_of(s);
    rc = batch_stage(b, src.data(), phi_dev, heat ? dst.data() : nullptr, alpha_of(s), st);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess || !graph) return set_error(LGF_E_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
  if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return set_error(LGF_E_CUDA, "graph instantiation failed");
  }
  b->graph = graph;
  b->graph_stages = nstages;
  return LGF_OK;
}

int lgf_batch_graph_create_io(lgf_batch *b, const void *const *f_host, void *const *phi_host,
                              const void *const *f_dev, void *const *phi_dev, void *cuda_stream) {
  if (!b || !f_host || !phi_host || !f_dev || !phi_dev) return set_error(LGF_E_INVALID_ARG, "NULL argument");
  for (int i = 0; i < b->n; ++i)
    for (const void *h : {f_host[i], (const void *)phi_host[i]}) {
      cudaPointerAttributes a{};
      if (!h || cudaPointerGetAttributes(&a, h) != cudaSuccess || a.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return set_error(LGF_E_INVALID_ARG, "instance %d: host buffers must be pinned (cudaHostAlloc / "
                                            "cudaHostRegister)", i);
      }
    }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // one eager stage (plans, spectra, workspaces), then the capture
  int rc = batch_stage(b, f_dev, phi_dev, nullptr, nullptr, st, f_host, phi_host);
  if (rc) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) return set_error(LGF_E_CUDA, "batch warm-up failed");
  if (b->exec) cudaGraphExecDestroy(b->exec), b->exec = nullptr;
  if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return set_error(LGF_E_CUDA, "stream capture could not begin (use a non-default stream)");
  rc = batch_stage(b, f_dev, phi_dev, nullptr, nullptr, st, f_host, phi_host);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess || !graph) return set_error(LGF_E_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
  if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return set_error(LGF_E_CUDA, "graph instantiation failed");
  }
  b->graph = graph;
  b->graph_stages = 1;
  return LGF_OK;
}

int lgf_batch_autotune(lgf_batch *b, const void *const *f_dev, void *const *phi_dev, void *cuda_stream) {
  if (!b || !f_dev || !phi_dev) return set_error(LGF_E_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // candidate evaluations of the block-index DFT passes: the CUDA-core passes, and for the FP32-hardware
  // arithmetics the tensor-core DFT-GEMM with the fewest slices that keeps the arithmetic's accuracy
  std::vector<int> cand = {0};
  if (b->opts.dft_slices == 0 && b->opts.mac_mode != LGF_MAC_PAIR) {
    if (b->opts.precision == LGF_PREC_DF32) cand.push_back(5);
    if (b->opts.precision == LGF_PREC_FP32) cand.push_back(3);
  }
  for (int i = 0; i < b->n; ++i) {
    double best = 1e300;
    int best_s = b->opts_i[i].dft_slices;
    for (int sl : cand) {
      lgf_solve_opts o = b->opts;
      o.dft_slices = sl;
      o.timing = 1;
      double t = 1e300;
      for (int rep = 0; rep < 3; ++rep) {  // the first call builds plans and spectra
        lgf_report r{};
        int rc = lgf_poisson_solve(b->t, &b->mesh[i], b->ncomp, f_dev[i], phi_dev[i], b->dtype, &o, &r, st);
        if (rc) return rc;
        if (rep) t = std::min(t, r.ms_total);
      }
      if (t < best) best = t, best_s = sl;
    }
    b->opts_i[i].dft_slices = best_s;
    b->tuned_ms[i] = best;
  }
  b->tuned = true;
  // the stream count: whole eager stages timed on the caller's stream
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_error(LGF_E_CUDA, "event creation failed");
  double best = 1e300;
  int best_n = b->nstreams;
  int rc = LGF_OK;
  // each candidate is timed as it will run: a Poisson stage captured into a graph and replayed (eager
  // stages when cuda_stream cannot capture, e.g. the legacy default stream)
  for (int ns : {1, 2, 4, 8, 16, 32}) {
    if (ns > b->n) continue;
    if ((rc = schedule(b, ns))) break;
    // one eager stage creates the workspaces of streams not used before (no allocation while capturing)
    if ((rc = batch_stage(b, f_dev, phi_dev, nullptr, nullptr, st))) break;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      rc = set_error(LGF_E_CUDA, "autotune stage failed");
      break;
    }
    cudaGraphExec_t exec = nullptr;
    if (st && cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int crc = batch_stage(b, f_dev, phi_dev, nullptr, nullptr, st);
      cudaGraph_t gr = nullptr;
      if (cudaStreamEndCapture(st, &gr) == cudaSuccess && gr && !crc) cudaGraphInstantiate(&exec, gr, 0);
      if (gr) cudaGraphDestroy(gr);
    }
    cudaGetLastError();
    float ms = 1e30f;
    for (int rep = 0; rep < 6 && !rc; ++rep) {  // the fastest of five replays after one untimed
      cudaEventRecord(e0, st);
      if (exec) {
        if (cudaGraphLaunch(exec, st) != cudaSuccess) rc = set_error(LGF_E_CUDA, "autotune graph launch failed");
      } else {
        rc = batch_stage(b, f_dev, phi_dev, nullptr, nullptr, st);
      }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(LGF_E_CUDA, "autotune stage failed");
      float m = 0.f;
      cudaEventElapsedTime(&m, e0, e1);
      if (rep) ms = std::min(ms, m);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (rc) break;
    if (ms < 0.99 * best) best = ms, best_n = ns;  // more streams only for a clear gain (replays vary ~1 %)
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  return schedule(b, best_n);
}

int lgf_batch_tuning(const lgf_batch *b, int32_t *nstreams, int32_t *slices, double *ms) {
  if (!b) return set_error(LGF_E_INVALID_ARG, "NULL batch");
  if (nstreams) *nstreams = b->nstreams;
  for (int i = 0; i < b->n; ++i) {
    if (slices) slices[i] = b->opts_i[i].dft_slices;
    if (ms) ms[i] = b->tuned_ms[i];
  }
  return LGF_OK;
}

int lgf_batch_graph_launch(lgf_batch *b, void *cuda_stream) {
  if (!b || !b->exec) return set_error(LGF_E_INVALID_ARG, "no captured graph");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)cuda_stream);
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "graph launch: %s", cudaGetErrorString(e));
}

int lgf_batch_graph_nodes(const lgf_batch *b, int64_t *nodes) {
  if (!b || !b->graph || !nodes) return set_error(LGF_E_INVALID_ARG, "no captured graph");
  size_t n = 0;
  if (cudaGraphGetNodes(b->graph, nullptr, &n) != cudaSuccess) return set_error(LGF_E_CUDA, "graph query failed");
  *nodes = (int64_t)n;
  return LGF_OK;
}

}  // extern "C"
