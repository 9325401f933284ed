// solver.cu -- host driver of the single-level solve (Sec. 2.2): pair mode and block-index FFT mode,
// the cost model behind LGF_MAC_AUTO, and dispatch of the multi-level (Sec. 3.4) driver.
//
// Every per-mesh list (source/target blocks, their coordinates, the box maps) lives in a cached
// device-side plan, so a solve issues only kernel launches on its stream: it can be captured into a
// CUDA graph once the plan, the kernel spectra and the workspace exist (an eager call creates them).
#include <string.h>

#include <algorithm>
#include <cmath>
#include <list>
#include <string>
#include <vector>

#include "amr.cuh"
#include "box_ops.cuh"
#include "solver.h"

namespace lgf {

int solve_multi(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st, const lgf_indicator *ind);

template <class R>
static const void *spectra_of(const lgf_table *t);
template <>
const void *spectra_of<double>(const lgf_table *t) { return t->s64; }
template <>
const void *spectra_of<float>(const lgf_table *t) { return t->s32; }
template <>
const void *spectra_of<df>(const lgf_table *t) { return t->sdf; }

// Relative cost model of the two ways to evaluate the per-frequency block-pair sum (complex
// multiply-adds per real component): PAIR = nsrc * ntgt * (2B)^2 (B+1) plus the block transforms;
// BOX = block-index DFTs over the 2 nb grid plus the local transforms, shared by two components.
double box_cost(int B, const int nb[3]) {
  const double B3 = (double)B * B * B;
  const double nx = nb[0], ny = nb[1], nz = nb[2];
  const double dft = 2.0 * (ny * nz * 2 * nx * nx + 2 * nx * nz * 2 * ny * ny + 4 * nx * ny * 2 * nz * nz);
  const double local = 8.0 * nx * ny * nz * 3.0 * std::log2((double)B) * 2.0;
  return B3 * (dft + local) / 2.0;
}
double pair_cost(int B, double nsrc, double ntgt) {
  return nsrc * ntgt * (2.0 * B) * (2.0 * B) * (B + 1.0) + (nsrc + ntgt) * 8.0 * B * B * B * 3.0 * std::log2(2.0 * B);
}

// ------------------------------------------------------------------ single-level plan (cached)
struct SinglePlan {
  int nsrc = 0, ntgt = 0;
  int reach[3] = {0, 0, 0};      // largest |target - source| block offset per axis
  int lo[3] = {0, 0, 0}, nb[3] = {0, 0, 0};
  bool box_ok = false;
  int64_t nbox = 0;
  int32_t *d_idx = nullptr;      // src_idx [nsrc] | tgt_idx [ntgt] | box gather [nbox] | box scatter [nbox]
  int4 *d_c = nullptr;           // src coords [nsrc] | tgt coords [ntgt]
  // residual: target-block map over the targets' block box (caller index or -1), source flag per block
  int tlo[3] = {0, 0, 0}, tn[3] = {0, 0, 0};
  int32_t *d_tmap = nullptr;
  uint8_t *d_is_src = nullptr;
  ~SinglePlan() {
    cudaFree(d_idx);
    cudaFree(d_c);
    cudaFree(d_tmap);
    cudaFree(d_is_src);
  }
};

static std::mutex g_sp_mu;
static std::list<std::pair<std::string, SinglePlan *>> g_sp;

static int single_plan(const lgf_mesh *m, SinglePlan **out) {
  const int n = m->nblocks[0];
  std::string key;
  int dev = 0;
  cudaGetDevice(&dev);
  key.append((const char *)&dev, sizeof dev);
  key.append((const char *)&m->block, 4);
  key.append((const char *)&n, 4);
  key.append((const char *)m->block_ijk, 12 * (size_t)n);
  const char has_roles = m->block_role ? 1 : 0;
  key.append(&has_roles, 1);
  if (m->block_role) key.append((const char *)m->block_role, (size_t)n);
  std::lock_guard<std::mutex> g(g_sp_mu);
  for (auto it = g_sp.begin(); it != g_sp.end(); ++it)
    if (it->first == key) {
      g_sp.splice(g_sp.begin(), g_sp, it);
      *out = it->second;
      return LGF_OK;
    }
  SinglePlan *P = new SinglePlan();
  std::vector<int32_t> src_idx, tgt_idx;
  std::vector<int4> src_c, tgt_c;
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  int slo[3] = {1 << 30, 1 << 30, 1 << 30}, shi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  int tlo[3] = {1 << 30, 1 << 30, 1 << 30}, thi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int i = 0; i < n; ++i) {
    const int role = m->block_role ? m->block_role[i] : 3;
    const int32_t *b = m->block_ijk + 3 * i;
    const int4 c = make_int4(b[0], b[1], b[2], 0);
    if (role & 1) {
      src_idx.push_back(i);
      src_c.push_back(c);
      for (int a = 0; a < 3; ++a) slo[a] = std::min(slo[a], b[a]), shi[a] = std::max(shi[a], b[a]);
    }
    if (role & 2) {
      tgt_idx.push_back(i);
      tgt_c.push_back(c);
      for (int a = 0; a < 3; ++a) tlo[a] = std::min(tlo[a], b[a]), thi[a] = std::max(thi[a], b[a]);
    }
    if (role & 3)
      for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], b[a]), hi[a] = std::max(hi[a], b[a]);
  }
  P->nsrc = (int)src_idx.size();
  P->ntgt = (int)tgt_idx.size();
  for (int a = 0; a < 3; ++a) {
    P->reach[a] = (P->nsrc && P->ntgt) ? std::max(thi[a] - slo[a], shi[a] - tlo[a]) : 0;
    P->lo[a] = lo[a];
    P->nb[a] = hi[a] - lo[a] + 1;
  }
  P->box_ok = P->ntgt > 0;
  for (int a = 0; a < 3; ++a)
    if (P->nb[a] < 1 || P->nb[a] > BOX_NB_MAX) P->box_ok = false;
  P->nbox = P->box_ok ? (int64_t)P->nb[0] * P->nb[1] * P->nb[2] : 0;
  std::vector<int32_t> idx(src_idx);
  idx.insert(idx.end(), tgt_idx.begin(), tgt_idx.end());
  if (P->box_ok) {
    std::vector<int32_t> maps(2 * P->nbox, -1);
    for (int i = 0; i < n; ++i) {
      const int role = m->block_role ? m->block_role[i] : 3;
      const int32_t *b = m->block_ijk + 3 * i;
      const int64_t bi = ((int64_t)(b[2] - lo[2]) * P->nb[1] + (b[1] - lo[1])) * P->nb[0] + (b[0] - lo[0]);
      if (role & 1) maps[bi] = i;
      if (role & 2) maps[P->nbox + bi] = i;
    }
    idx.insert(idx.end(), maps.begin(), maps.end());
  }
  std::vector<int4> cs(src_c);
  cs.insert(cs.end(), tgt_c.begin(), tgt_c.end());
  std::vector<int32_t> tmap;
  std::vector<uint8_t> is_src(n, 0);
  if (P->ntgt) {
    int64_t nt = 1;
    for (int a = 0; a < 3; ++a) P->tlo[a] = tlo[a], P->tn[a] = thi[a] - tlo[a] + 1, nt *= P->tn[a];
    tmap.assign(nt, -1);
    for (size_t j = 0; j < tgt_idx.size(); ++j) {
      const int4 c = tgt_c[j];
      tmap[((int64_t)(c.z - tlo[2]) * P->tn[1] + (c.y - tlo[1])) * P->tn[0] + (c.x - tlo[0])] = tgt_idx[j];
    }
  }
  for (int i : src_idx) is_src[i] = 1;
  if (cudaMalloc(&P->d_idx, sizeof(int32_t) * std::max<size_t>(idx.size(), 1)) != cudaSuccess ||
      cudaMalloc(&P->d_c, sizeof(int4) * std::max<size_t>(cs.size(), 1)) != cudaSuccess ||
      cudaMalloc(&P->d_tmap, sizeof(int32_t) * std::max<size_t>(tmap.size(), 1)) != cudaSuccess ||
      cudaMalloc(&P->d_is_src, std::max<size_t>(is_src.size(), 1)) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return set_error(LGF_E_OOM, "single-level plan allocation failed");
  }
  if (!idx.empty()) cudaMemcpy(P->d_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice);
  if (!cs.empty()) cudaMemcpy(P->d_c, cs.data(), sizeof(int4) * cs.size(), cudaMemcpyHostToDevice);
  if (!tmap.empty()) cudaMemcpy(P->d_tmap, tmap.data(), sizeof(int32_t) * tmap.size(), cudaMemcpyHostToDevice);
  if (!is_src.empty()) cudaMemcpy(P->d_is_src, is_src.data(), is_src.size(), cudaMemcpyHostToDevice);
  g_sp.emplace_front(key, P);
  while (g_sp.size() > 1024) {
    delete g_sp.back().second;
    g_sp.pop_back();
  }
  *out = P;
  return LGF_OK;
}

// Method-minimum work of a single-level solve (see lgf_report): caller fields read and written once, the
// unique kernel-spectrum values, 5 M log2 M per complex transform and 8 flops per pair multiply-add.
static void alg_work_single(lgf_report *rep, const SinglePlan *P, int B, int ncomp, int dtype, size_t rsize,
                            int mode) {
  const double B3 = (double)B * B * B, W = (2.0 * B) * (2.0 * B) * (B + 1.0);
  const double w = dtype == LGF_F32 ? 4.0 : 8.0;
  double bytes = ncomp * (P->nsrc + P->ntgt) * B3 * w, flops = 0.0;
  if (mode == LGF_MAC_BOX) {
    double uniq = 1.0, M = 1.0;
    for (int a = 0; a < 3; ++a) uniq *= P->nb[a] * B + 1.0, M *= 2.0 * P->nb[a] * B;
    bytes += uniq * rsize;
    flops = 2.0 * ((ncomp + 1) / 2) * 5.0 * M * std::log2(M);
  } else {
    double noff = 1.0;
    for (int a = 0; a < 3; ++a) noff *= 2.0 * P->reach[a] + 1.0;
    bytes += noff * W * 2.0 * rsize;
    const double m = 8.0 * B3;
    flops = (P->nsrc + P->ntgt) * 0.5 * ncomp * 5.0 * m * std::log2(m) + 8.0 * W * P->nsrc * P->ntgt * ncomp;
  }
  rep->alg_bytes = (int64_t)bytes;
  rep->alg_flops = flops;
}

static void fill_report(lgf_report *rep, const SinglePlan *P, int64_t B3, const Workspace *ws, int64_t launches,
                        int mode, int64_t extra_bytes) {
  if (!rep) return;
  rep->target_cells = (int64_t)P->ntgt * B3;
  rep->source_blocks = P->nsrc;
  rep->target_blocks = P->ntgt;
  rep->pairs = mode == LGF_MAC_PAIR ? (int64_t)P->nsrc * P->ntgt : 0;
  rep->scratch_bytes = (int64_t)ws->total() + extra_bytes;
  rep->kernel_launches = launches;
  rep->mac_mode_used = mode;
}

template <class R>
static int solve_single_pair(lgf_table *t, const lgf_mesh *m, const SinglePlan *P, int ncomp, const void *f,
                             void *phi, int dtype, const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  const int B = m->block;
  const int64_t B3 = (int64_t)B * B * B;
  const int W = (2 * B) * (2 * B) * (B + 1);
  const void *Gh = spectra_of<R>(t);
  if (!Gh) return set_error(LGF_E_INVALID_ARG, "table lacks the spectra of the requested precision");
  const int nsrc = P->nsrc, ntgt = P->ntgt;
  const int mo[3] = {t->mo.x, t->mo.y, t->mo.z};
  for (int a = 0; a < 3; ++a)
    if (P->reach[a] > mo[a])
      return set_error(LGF_E_TABLE_RANGE, "block offsets reach %d along axis %d; the table covers %d", P->reach[a],
                       a, mo[a]);
  Workspace *ws = workspace_for(t, st);
  int rc;
  if ((rc = ws->buf[0].reserve(std::max<size_t>(sizeof(cx<R>) * (size_t)ncomp * nsrc * W, 16))) ||
      (rc = ws->buf[1].reserve(sizeof(cx<R>) * (size_t)ncomp * ntgt * W)))
    return rc;
  const int32_t *d_src_idx = P->d_idx, *d_tgt_idx = P->d_idx + nsrc;
  const int4 *d_src_c = P->d_c, *d_tgt_c = P->d_c + nsrc;
  PhaseTimer tm;
  tm.start(o.timing != 0, st);
  const int64_t cs = (int64_t)m->nblocks[0] * B3;
  if ((rc = PairOps<R>::forward(B, f, dtype, cs, d_src_idx, nsrc, ncomp, ws->buf[0].p, nullptr, 0, st))) return rc;
  tm.mark(PH_FORWARD);
  if ((rc = PairOps<R>::mac(B, ws->buf[0].p, nsrc, (int64_t)nsrc * W, nullptr, d_src_c, Gh, t->mo, ws->buf[1].p,
                            ntgt, (int64_t)ntgt * W, nullptr, d_tgt_c, ncomp, 0, st)))
    return rc;
  tm.mark(PH_MAC);
  const double scale = m->h0 * m->h0 / (double)((2 * B) * (2 * B) * (2 * B));
  if ((rc = PairOps<R>::inverse(B, ws->buf[1].p, (int64_t)ntgt * W, nullptr, d_tgt_idx, ntgt, ncomp, phi, dtype,
                                cs, 0, nullptr, 0, nullptr, 0, scale, st)))
    return rc;
  tm.mark(PH_INVERSE);
  tm.finish(rep);
  fill_report(rep, P, B3, ws, 2 + (ncomp + 2) / 3, LGF_MAC_PAIR, 0);
  if (rep) alg_work_single(rep, P, B, ncomp, dtype, sizeof(R), LGF_MAC_PAIR);
  if (o.timing) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(LGF_E_CUDA, "solve failed: %s", cudaGetErrorString(e));
  }
  return LGF_OK;
}

static size_t dtype_size(int dtype, size_t rsize) { return dtype == 0 ? 8 : (dtype == 1 ? 4 : rsize); }

template <class R>
static int solve_single_box(lgf_table *t, const lgf_mesh *m, const SinglePlan *P, int ncomp, const void *f,
                            void *phi, int dtype, const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  const int B = m->block, n = m->nblocks[0];
  const int64_t B3 = (int64_t)B * B * B;
  BoxSpec *S = nullptr;
  int rc = box_spectrum(t, P->nb, &S, st);
  if (rc) return rc;
  Workspace *ws = workspace_for(t, st);
  const int nf = (ncomp + 1) / 2;
  const size_t ybytes = sizeof(cx<R>) * (size_t)std::min(nf, BOX_MAXF) * (8 * P->nbox) * B3;
  if ((rc = ws->buf[0].reserve(ybytes)) || (rc = ws->buf[1].reserve(ybytes))) return rc;
  const int32_t *gmap = P->d_idx + P->nsrc + P->ntgt, *smap = gmap + P->nbox;
  PhaseTimer tm;
  tm.start(o.timing != 0, st);
  const int64_t cs = (int64_t)n * B3;
  const size_t es = dtype_size(dtype, sizeof(R));
  const double scale = m->h0 * m->h0 / (8.0 * P->nbox * (double)B3);
  // two components per complex field
  std::vector<int> nin(nf);
  std::vector<InSpec3> in(nf);
  std::vector<OutSpec<R>> ore(nf), oim(nf);
  for (int fi = 0; fi < nf; ++fi) {
    const int c0 = 2 * fi, c1 = c0 + 1;
    nin[fi] = 1;
    in[fi].s[0] = InSpec{gmap, (const char *)f + es * c0 * cs, nullptr, dtype, 0, 0};
    if (c1 < ncomp) in[fi].s[nin[fi]++] = InSpec{gmap, (const char *)f + es * c1 * cs, nullptr, dtype, 0, 1};
    ore[fi] = OutSpec<R>{smap, nullptr, phi, nullptr, nullptr, c0 * cs, dtype, 0};
    oim[fi] = c1 < ncomp ? OutSpec<R>{smap, nullptr, phi, nullptr, nullptr, c1 * cs, dtype, 0} : OutSpec<R>{};
  }
  int64_t launches = 0;
  if ((rc = BoxOps<R>::convolve(B, S, nf, nin.data(), in.data(), ore.data(), oim.data(), scale,
                                (cx<R> *)ws->buf[0].p, (cx<R> *)ws->buf[1].p, st,
                                o.timing ? phase_mark_cb : nullptr, &tm, o.dft_slices, t->d_status, &launches)))
    return rc;
  tm.finish(rep);
  fill_report(rep, P, B3, ws, launches, LGF_MAC_BOX, (int64_t)S->bytes);
  if (rep) alg_work_single(rep, P, B, ncomp, dtype, sizeof(R), LGF_MAC_BOX);
  if (o.timing) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(LGF_E_CUDA, "solve failed: %s", cudaGetErrorString(e));
    if (o.dft_slices > 0 && (rc = take_device_status(t))) return rc;
  }
  return LGF_OK;
}

// FP64 residual of a single-level solve (opts.residual): max |L phi - f| / max |f| over target cells
// with six target neighbours; LGF_E_PRECISION above opts.residual_tol.  Synchronises the stream.
static int single_residual(lgf_table *t, const lgf_mesh *m, const SinglePlan *P, int ncomp, const void *f,
                           const void *phi, int dtype, const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  Workspace *ws = workspace_for(t, st);
  int rc = ws->buf[15].reserve(sizeof(unsigned long long) * 2);
  if (rc) return rc;
  unsigned long long *racc = (unsigned long long *)ws->buf[15].p;
  cudaMemsetAsync(racc, 0, sizeof(unsigned long long) * 2, st);
  int shift = 0;
  while ((1 << shift) < m->block) ++shift;
  const int64_t cs = (int64_t)m->nblocks[0] * m->block * m->block * m->block;
  k_residual_single<<<dim3(P->ntgt, ncomp), 256, 0, st>>>(
      P->d_tmap, make_int3(P->tlo[0], P->tlo[1], P->tlo[2]), make_int3(P->tn[0], P->tn[1], P->tn[2]), shift, m->h0,
      P->d_idx + P->nsrc, P->d_c + P->nsrc, P->d_is_src, phi, f, dtype, cs, racc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(LGF_E_CUDA, "residual launch: %s", cudaGetErrorString(e));
  unsigned long long h[2] = {0, 0};
  cudaMemcpyAsync(h, racc, sizeof h, cudaMemcpyDeviceToHost, st);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
    return set_error(LGF_E_CUDA, "residual failed: %s", cudaGetErrorString(e));
  double r, s;
  memcpy(&r, &h[0], 8);
  memcpy(&s, &h[1], 8);
  const double rel = s > 0 ? r / s : r;
  if (rep) {
    rep->residual_rel = rel;
    rep->kernel_launches += 1;
  }
  if (o.residual_tol > 0 && rel > o.residual_tol)
    return set_error(LGF_E_PRECISION, "FP64 residual %.3e exceeds the tolerance %.3e", rel, o.residual_tol);
  return LGF_OK;
}

template <class R>
static int solve_single_any(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                            const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  SinglePlan *P = nullptr;
  int rc = single_plan(m, &P);
  if (rc) return rc;
  if (P->ntgt == 0) return LGF_OK;
  int mode = o.mac_mode;
  if (mode == LGF_MAC_AUTO)
    mode = (P->box_ok && (!spectra_of<R>(t) || o.dft_slices > 0 ||
                          box_cost(m->block, P->nb) < pair_cost(m->block, P->nsrc, P->ntgt)))
               ? LGF_MAC_BOX
               : LGF_MAC_PAIR;
  if (mode == LGF_MAC_BOX) {
    if (!P->box_ok) return set_error(LGF_E_UNSUPPORTED, "BOX mode needs 1..%d blocks per axis", BOX_NB_MAX);
    rc = solve_single_box<R>(t, m, P, ncomp, f, phi, dtype, o, rep, st);
  } else {
    rc = solve_single_pair<R>(t, m, P, ncomp, f, phi, dtype, o, rep, st);
  }
  if (rc || !o.residual) return rc;
  return single_residual(t, m, P, ncomp, f, phi, dtype, o, rep, st);
}

int solve_poisson(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                  const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  if (m->nlevels > 1) return solve_multi(t, m, ncomp, f, phi, dtype, o, rep, st, nullptr);
  switch (o.precision) {
    case LGF_PREC_FP64: return solve_single_any<double>(t, m, ncomp, f, phi, dtype, o, rep, st);
    case LGF_PREC_FP32: return solve_single_any<float>(t, m, ncomp, f, phi, dtype, o, rep, st);
    default: return solve_single_any<df>(t, m, ncomp, f, phi, dtype, o, rep, st);
  }
}

}  // namespace lgf
