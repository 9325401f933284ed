// api.cu -- the C ABI (include/lgf.h): table lifetime, argument checking, workspaces, dispatch.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <set>
#include <tuple>

#include "internal.h"
#include "tc.cuh"
#include "solver.h"

namespace lgf {

static thread_local std::string g_last_error;

int set_error(int code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

// Workspaces are per (table, stream); calls without a table (heat apply) share a process-wide map
// keyed by (device, stream).
static std::mutex g_ws_mu;
static std::map<std::pair<int, void *>, Workspace *> g_ws;

Workspace *workspace_for(lgf_table *t, cudaStream_t st) {
  if (!t) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(g_ws_mu);
    auto key = std::make_pair(dev, (void *)st);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) return it->second;
    Workspace *w = new Workspace();
    g_ws[key] = w;
    return w;
  }
  std::lock_guard<std::mutex> g(t->mu);
  auto it = t->ws.find((void *)st);
  if (it != t->ws.end()) return it->second;
  Workspace *w = new Workspace();
  t->ws[(void *)st] = w;
  return w;
}

int check_mesh(const lgf_mesh *m, int B_expected) {
  if (!m) return set_error(LGF_E_INVALID_ARG, "mesh is NULL");
  if (m->nlevels < 1 || m->nlevels > 16) return set_error(LGF_E_INVALID_ARG, "nlevels %d", m->nlevels);
  if (B_expected && m->block != B_expected)
    return set_error(LGF_E_MESH, "mesh block %d differs from the table's %d", m->block, B_expected);
  if (m->block != 8 && m->block != 16) return set_error(LGF_E_UNSUPPORTED, "block size %d", m->block);
  if (!(m->h0 > 0.0)) return set_error(LGF_E_INVALID_ARG, "h0 must be > 0");
  if (!m->nblocks || !m->block_ijk) return set_error(LGF_E_INVALID_ARG, "nblocks/block_ijk NULL");
  if (m->n_ext < 0) return set_error(LGF_E_INVALID_ARG, "n_ext < 0");
  int64_t off = 0;
  for (int k = 0; k < m->nlevels; ++k) {
    if (m->nblocks[k] < 1) return set_error(LGF_E_MESH, "level %d has no blocks", k);
    std::set<std::tuple<int, int, int>> seen;
    for (int i = 0; i < m->nblocks[k]; ++i) {
      const int32_t *b = m->block_ijk + 3 * (off + i);
      if (!seen.insert(std::make_tuple(b[0], b[1], b[2])).second)
        return set_error(LGF_E_MESH, "duplicate block (%d,%d,%d) on level %d", b[0], b[1], b[2], k);
    }
    off += m->nblocks[k];
  }
  return LGF_OK;
}

}  // namespace lgf

using namespace lgf;

namespace lgf {

int check_slices(const lgf_solve_opts &o) {
  if (o.dft_slices == 0) return LGF_OK;
  if (o.dft_slices < 0 || o.dft_slices > TC_SMAX) return set_error(LGF_E_INVALID_ARG, "dft_slices %d", o.dft_slices);
  if (o.precision == LGF_PREC_FP64)
    return set_error(LGF_E_UNSUPPORTED, "the tensor-core DFT-GEMM serves the FP32 and DF32 precisions");
  if (o.precision == LGF_PREC_FP32 && o.dft_slices > 3)
    return set_error(LGF_E_INVALID_ARG, "FP32 takes 1..3 DFT-GEMM slices (got %d)", o.dft_slices);
  if (o.precision == LGF_PREC_DF32 && o.dft_slices < 4)
    return set_error(LGF_E_INVALID_ARG, "DF32 takes 4..6 DFT-GEMM slices (got %d)", o.dft_slices);
  return LGF_OK;
}

int take_device_status(lgf_table *t) {
  int v = 0;
  if (cudaMemcpy(&v, t->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_error(LGF_E_CUDA, "status word read failed");
  if (!v) return LGF_OK;
  cudaMemset(t->d_status, 0, sizeof(int));
  return set_error(LGF_E_TIMEOUT, "a bounded device-side wait gave up (tensor-core DFT-GEMM)");
}

// A wait that cannot complete: an mbarrier expecting one arrival that never comes, waited on with the
// bounded helper of the tensor-core kernels (limit 2^log2_cycles cycles).  It must give up, set the
// status word and leave the context usable.
__global__ void k_wait_selftest(int *status, long long limit) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    abort_flag = 0;
  }
  __syncthreads();
  const bool ok = tc::mbar_wait_or_abort(&bar, 0, &abort_flag, limit);
  __syncthreads();
  if (threadIdx.x == 0 && (!ok || abort_flag)) atomicExch(status, 1);
}

}  // namespace lgf

extern "C" {

int lgf_selftest_wait_timeout(lgf_table *t, int32_t log2_cycles, void *cuda_stream) {
  if (!t) return set_error(LGF_E_INVALID_ARG, "table is NULL");
  if (log2_cycles < 10 || log2_cycles > 31) return set_error(LGF_E_INVALID_ARG, "log2_cycles %d", log2_cycles);
  k_wait_selftest<<<1, 32, 0, (cudaStream_t)cuda_stream>>>(t->d_status, 1ll << log2_cycles);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "self-test launch: %s", cudaGetErrorString(e));
}

int lgf_device_status(lgf_table *t) {
  if (!t) return set_error(LGF_E_INVALID_ARG, "table is NULL");
  if (cudaDeviceSynchronize() != cudaSuccess) return set_error(LGF_E_CUDA, "device synchronisation failed");
  return take_device_status(t);
}

const char *lgf_last_error(void) { return g_last_error.c_str(); }
const char *lgf_version(void) { return "lgf-gb300 0.1 (sm_103a)"; }

int lgf_table_create(lgf_table **out, int32_t block, const int32_t max_block_offset[3], uint32_t flags,
                     void *cuda_stream) {
  if (!out || !max_block_offset) return set_error(LGF_E_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (block != 8 && block != 16) return set_error(LGF_E_UNSUPPORTED, "block size %d", block);
  for (int a = 0; a < 3; ++a)
    if (max_block_offset[a] < 0 || max_block_offset[a] > 64)
      return set_error(LGF_E_INVALID_ARG, "max_block_offset[%d] = %d out of [0, 64]", a, max_block_offset[a]);
  if ((flags & 15u) == 0) return set_error(LGF_E_INVALID_ARG, "no spectrum format requested");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  lgf_table *t = new lgf_table();
  cudaGetDevice(&t->device);
  if (cudaMalloc(&t->d_status, sizeof(int)) != cudaSuccess || cudaMemset(t->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(t->d_status);
    delete t;
    return set_error(LGF_E_OOM, "status word");
  }
  t->B = block;
  t->mo = make_int3(max_block_offset[0], max_block_offset[1], max_block_offset[2]);
  t->noff = (2 * t->mo.x + 1) * (2 * t->mo.y + 1) * (2 * t->mo.z + 1);
  int mmax = std::max(t->mo.x, std::max(t->mo.y, t->mo.z));
  t->N = block * (mmax + 1);
  t->flags = flags;
  int rc = build_lgf_octant(t->N, &t->Gd, st, &t->quad_T, &t->quad_nodes);
  if (rc) {
    cudaFree(t->d_status);
    delete t;
    return rc;
  }
  const size_t W = (size_t)(2 * block) * (2 * block) * (block + 1);
  const size_t n = W * t->noff;
  if (flags & LGF_TBL_BOX_ONLY) {
    *out = t;  // pair spectra skipped; box spectra are generated on demand from t->Gd
    return LGF_OK;
  }
  if ((flags & LGF_TBL_FP64) && cudaMalloc(&t->s64, n * 16) != cudaSuccess) rc = LGF_E_OOM;
  if (!rc && (flags & LGF_TBL_FP32) && cudaMalloc(&t->s32, n * 8) != cudaSuccess) rc = LGF_E_OOM;
  if (!rc && (flags & LGF_TBL_DF32) && cudaMalloc(&t->sdf, n * 16) != cudaSuccess) rc = LGF_E_OOM;
  if (rc) {
    cudaGetLastError();
    lgf_table_destroy(t);
    return set_error(LGF_E_OOM, "spectra allocation (%zu offsets) failed", (size_t)t->noff);
  }
  rc = build_spectra(block, t->Gd, t->N + 1, t->mo, t->noff, t->s64, t->s32, t->sdf, st);
  if (rc) {
    lgf_table_destroy(t);
    return rc;
  }
  *out = t;
  return LGF_OK;
}

int lgf_table_destroy(lgf_table *t) {
  if (!t) return LGF_OK;
  cudaDeviceSynchronize();
  if (t->Gd) cudaFree(t->Gd);
  if (t->d_status) cudaFree(t->d_status);
  if (t->s64) cudaFree(t->s64);
  if (t->s32) cudaFree(t->s32);
  if (t->sdf) cudaFree(t->sdf);
  for (auto &kv : t->ws) {
    for (auto &b : kv.second->buf) b.release();
    delete kv.second;
  }
  for (auto &kv : t->box) delete kv.second;
  delete t;
  return LGF_OK;
}

int lgf_table_lgf_values(const lgf_table *t, int32_t n, double *host_out) {
  if (!t || !host_out) return set_error(LGF_E_INVALID_ARG, "NULL argument");
  if (n < 0 || n > t->N) return set_error(LGF_E_TABLE_RANGE, "n = %d beyond the table extent %d", n, t->N);
  const size_t K = (size_t)t->N + 1, k = (size_t)n + 1;
  for (size_t c = 0; c < k; ++c)
    for (size_t b = 0; b < k; ++b)
      if (cudaMemcpy(host_out + (c * k + b) * k, t->Gd + (c * K + b) * K, k * sizeof(double),
                     cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_error(LGF_E_CUDA, "copy of the LGF octant failed");
  return LGF_OK;
}

int lgf_poisson_solve(lgf_table *t, const lgf_mesh *m, int32_t ncomp, const void *f_dev, void *phi_dev,
                      int32_t dtype, const lgf_solve_opts *opts, lgf_report *rep, void *cuda_stream) {
  if (!t) return set_error(LGF_E_INVALID_ARG, "table is NULL");
  int rc = check_mesh(m, t->B);
  if (rc) return rc;
  if (ncomp < 1) return set_error(LGF_E_INVALID_ARG, "ncomp %d", ncomp);
  if (!f_dev || !phi_dev) return set_error(LGF_E_INVALID_ARG, "field pointer NULL");
  if (f_dev == phi_dev) return set_error(LGF_E_INVALID_ARG, "f and phi alias");
  if (dtype != LGF_F64 && dtype != LGF_F32) return set_error(LGF_E_INVALID_ARG, "dtype %d", dtype);
  lgf_solve_opts o{LGF_PREC_FP64, LGF_MAC_AUTO, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (o.precision < 0 || o.precision > 2) return set_error(LGF_E_INVALID_ARG, "precision %d", o.precision);
  if (o.mac_mode < 0 || o.mac_mode > 2) return set_error(LGF_E_INVALID_ARG, "mac_mode %d", o.mac_mode);
  if ((rc = check_slices(o))) return rc;
  if (o.flags & ~LGF_SOLVE_NO_CORRECTION) return set_error(LGF_E_INVALID_ARG, "unknown solve flags 0x%x", o.flags);
  if (rep) memset(rep, 0, sizeof(*rep));
  return solve_poisson(t, m, ncomp, f_dev, phi_dev, dtype, o, rep, (cudaStream_t)cuda_stream);
}

int lgf_refinement_indicator(lgf_table *t, const lgf_mesh *m, int32_t ncomp, const void *f_dev, void *phi_dev,
                             int32_t dtype, const lgf_solve_opts *opts, const lgf_indicator *ind, lgf_report *rep,
                             void *cuda_stream) {
  if (!t) return set_error(LGF_E_INVALID_ARG, "table is NULL");
  int rc = check_mesh(m, t->B);
  if (rc) return rc;
  if (ncomp < 1) return set_error(LGF_E_INVALID_ARG, "ncomp %d", ncomp);
  if (!f_dev || !phi_dev) return set_error(LGF_E_INVALID_ARG, "field pointer NULL");
  if (f_dev == phi_dev) return set_error(LGF_E_INVALID_ARG, "f and phi alias");
  if (dtype != LGF_F64 && dtype != LGF_F32) return set_error(LGF_E_INVALID_ARG, "dtype %d", dtype);
  if (!ind || !ind->rms_dev || !ind->flags_dev || !ind->s_max_dev)
    return set_error(LGF_E_INVALID_ARG, "indicator request or one of its device pointers is NULL");
  if (!(ind->alpha > 0.0 && ind->alpha < 1.0) || !(ind->beta > 0.0 && ind->beta < 1.0))
    return set_error(LGF_E_INVALID_ARG, "indicator alpha %g / beta %g outside (0, 1)", ind->alpha, ind->beta);
  if (ind->n_levels_max < m->nlevels - 1 || ind->n_levels_max > 64)
    return set_error(LGF_E_INVALID_ARG, "n_levels_max %d below the mesh's top level %d", ind->n_levels_max,
                     m->nlevels - 1);
  lgf_solve_opts o{LGF_PREC_FP64, LGF_MAC_AUTO, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (o.precision < 0 || o.precision > 2) return set_error(LGF_E_INVALID_ARG, "precision %d", o.precision);
  if (o.mac_mode < 0 || o.mac_mode > 2) return set_error(LGF_E_INVALID_ARG, "mac_mode %d", o.mac_mode);
  if ((rc = check_slices(o))) return rc;
  if (o.flags & ~LGF_SOLVE_NO_CORRECTION) return set_error(LGF_E_INVALID_ARG, "unknown solve flags 0x%x", o.flags);
  if (rep) memset(rep, 0, sizeof(*rep));
  return solve_multi(t, m, ncomp, f_dev, phi_dev, dtype, o, rep, (cudaStream_t)cuda_stream, ind);
}

int lgf_table_prepare(lgf_table *t, const lgf_mesh *m, int32_t ncomp, int32_t dtype, const lgf_solve_opts *opts,
                      void *cuda_stream) {
  if (!t) return set_error(LGF_E_INVALID_ARG, "table is NULL");
  int rc = check_mesh(m, t->B);
  if (rc) return rc;
  if (ncomp < 1) return set_error(LGF_E_INVALID_ARG, "ncomp %d", ncomp);
  if (dtype != LGF_F64 && dtype != LGF_F32) return set_error(LGF_E_INVALID_ARG, "dtype %d", dtype);
  int64_t nblk = 0;
  for (int k = 0; k < m->nlevels; ++k) nblk += m->nblocks[k];
  const size_t bytes = (size_t)ncomp * nblk * t->B * t->B * t->B * (dtype == LGF_F32 ? 4 : 8);
  void *f = nullptr, *phi = nullptr;
  if (cudaMalloc(&f, bytes) != cudaSuccess || cudaMalloc(&phi, bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(f);
    return set_error(LGF_E_OOM, "prepare: %zu bytes of trial fields", bytes);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaMemsetAsync(f, 0, bytes, st);
  lgf_solve_opts o{LGF_PREC_FP64, LGF_MAC_AUTO, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  o.timing = 0;
  o.residual = 0;
  rc = lgf_poisson_solve(t, m, ncomp, f, phi, dtype, &o, nullptr, cuda_stream);  // builds and caches
  const cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(f);
  cudaFree(phi);
  if (rc) return rc;
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "prepare: %s", cudaGetErrorString(e));
}

int lgf_stage_projection(lgf_table *t, const lgf_mesh *m, const void *r_dev, void *u_dev, void *p_dev, int32_t dtype,
                         double alpha_finest, const lgf_solve_opts *opts, lgf_report *rep, void *cuda_stream) {
  if (!t) return set_error(LGF_E_INVALID_ARG, "table is NULL");
  int rc = check_mesh(m, t->B);
  if (rc) return rc;
  if (!r_dev || !u_dev) return set_error(LGF_E_INVALID_ARG, "field pointer NULL");
  if (r_dev == u_dev || (p_dev && (p_dev == r_dev || p_dev == u_dev)))
    return set_error(LGF_E_INVALID_ARG, "r, u and p must not alias");
  if (dtype != LGF_F64 && dtype != LGF_F32) return set_error(LGF_E_INVALID_ARG, "dtype %d", dtype);
  if (!(alpha_finest >= 0.0) || alpha_finest > 1e4)
    return set_error(LGF_E_INVALID_ARG, "alpha_finest %g", alpha_finest);
  lgf_solve_opts o{LGF_PREC_FP64, LGF_MAC_AUTO, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (o.precision < 0 || o.precision > 2) return set_error(LGF_E_INVALID_ARG, "precision %d", o.precision);
  if (o.mac_mode < 0 || o.mac_mode > 2) return set_error(LGF_E_INVALID_ARG, "mac_mode %d", o.mac_mode);
  if ((rc = check_slices(o))) return rc;
  if (o.flags & ~LGF_SOLVE_NO_CORRECTION) return set_error(LGF_E_INVALID_ARG, "unknown solve flags 0x%x", o.flags);
  if (rep) memset(rep, 0, sizeof(*rep));
  return solve_projection(t, m, r_dev, u_dev, p_dev, dtype, alpha_finest, o, rep, (cudaStream_t)cuda_stream);
}

int lgf_heat_apply(lgf_table *t, const lgf_mesh *m, int32_t ncomp, const void *f_dev, void *g_dev,
                   int32_t dtype, double alpha_finest, const lgf_solve_opts *opts, lgf_report *rep,
                   void *cuda_stream) {
  int rc = check_mesh(m, t ? t->B : 0);
  if (rc) return rc;
  if (ncomp < 1) return set_error(LGF_E_INVALID_ARG, "ncomp %d", ncomp);
  if (!f_dev || !g_dev) return set_error(LGF_E_INVALID_ARG, "field pointer NULL");
  if (f_dev == g_dev) return set_error(LGF_E_INVALID_ARG, "f and g alias");
  if (dtype != LGF_F64 && dtype != LGF_F32) return set_error(LGF_E_INVALID_ARG, "dtype %d", dtype);
  if (!(alpha_finest >= 0.0) || alpha_finest > 1e4)
    return set_error(LGF_E_INVALID_ARG, "alpha_finest %g", alpha_finest);
  lgf_solve_opts o{LGF_PREC_FP64, LGF_MAC_AUTO, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (rep) memset(rep, 0, sizeof(*rep));
  return solve_heat(t, m, ncomp, f_dev, g_dev, dtype, alpha_finest, o, rep, (cudaStream_t)cuda_stream);
}

}  // extern "C"
