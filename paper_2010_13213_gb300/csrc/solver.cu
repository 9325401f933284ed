// solver.cu -- host driver of the single-level solve (Sec. 2.2) in pair mode; dispatch of the
// multi-level (Sec. 3.4) and heat (Sec. 3.5) drivers.
#include <algorithm>
#include <cmath>
#include <vector>

#include "box_ops.cuh"
#include "solver.h"

namespace lgf {

int solve_multi(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st);

template <class R>
static const void *spectra_of(const lgf_table *t);
template <>
const void *spectra_of<double>(const lgf_table *t) { return t->s64; }
template <>
const void *spectra_of<float>(const lgf_table *t) { return t->s32; }
template <>
const void *spectra_of<df>(const lgf_table *t) { return t->sdf; }

template <class R>
static int solve_single(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                        const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  const int B = m->block;
  const int nb = m->nblocks[0];
  const int64_t B3 = (int64_t)B * B * B;
  const int W = (2 * B) * (2 * B) * (B + 1);
  const void *Gh = spectra_of<R>(t);
  if (!Gh) return set_error(LGF_E_INVALID_ARG, "table lacks the spectra of the requested precision");
  std::vector<int32_t> src_idx, tgt_idx;
  std::vector<int4> src_c, tgt_c;
  for (int i = 0; i < nb; ++i) {
    const int role = m->block_role ? m->block_role[i] : 3;
    const int32_t *b = m->block_ijk + 3 * i;
    int4 c = make_int4(b[0], b[1], b[2], 0);
    if (role & 1) {
      src_idx.push_back(i);
      src_c.push_back(c);
    }
    if (role & 2) {
      tgt_idx.push_back(i);
      tgt_c.push_back(c);
    }
  }
  const int nsrc = (int)src_idx.size(), ntgt = (int)tgt_idx.size();
  if (ntgt == 0) return LGF_OK;
  // every (target, source) offset must be covered by the table
  if (nsrc) {
    int lo[3], hi[3], tlo[3], thi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = tlo[a] = 1 << 30;
      hi[a] = thi[a] = -(1 << 30);
    }
    for (auto &c : src_c) {
      const int v[3] = {c.x, c.y, c.z};
      for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], v[a]), hi[a] = std::max(hi[a], v[a]);
    }
    for (auto &c : tgt_c) {
      const int v[3] = {c.x, c.y, c.z};
      for (int a = 0; a < 3; ++a) tlo[a] = std::min(tlo[a], v[a]), thi[a] = std::max(thi[a], v[a]);
    }
    const int mo[3] = {t->mo.x, t->mo.y, t->mo.z};
    for (int a = 0; a < 3; ++a)
      if (std::max(thi[a] - lo[a], hi[a] - tlo[a]) > mo[a])
        return set_error(LGF_E_TABLE_RANGE, "block offsets reach %d along axis %d; the table covers %d",
                         std::max(thi[a] - lo[a], hi[a] - tlo[a]), a, mo[a]);
  }
  Workspace *ws = workspace_for(t, st);
  const size_t specF = sizeof(cx<R>) * (size_t)ncomp * nsrc * W;
  const size_t specP = sizeof(cx<R>) * (size_t)ncomp * ntgt * W;
  const size_t idx_bytes = sizeof(int32_t) * (nsrc + ntgt) + sizeof(int4) * (nsrc + ntgt) + 64;
  int rc;
  if ((rc = ws->buf[0].reserve(std::max<size_t>(specF, 16)))) return rc;
  if ((rc = ws->buf[1].reserve(specP))) return rc;
  if ((rc = ws->buf[2].reserve(idx_bytes))) return rc;
  char *ib = (char *)ws->buf[2].p;
  int4 *d_src_c = (int4 *)ib;
  int4 *d_tgt_c = d_src_c + nsrc;
  int32_t *d_src_idx = (int32_t *)(d_tgt_c + ntgt);
  int32_t *d_tgt_idx = d_src_idx + nsrc;
  if (nsrc) {
    cudaMemcpyAsync(d_src_c, src_c.data(), sizeof(int4) * nsrc, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_src_idx, src_idx.data(), sizeof(int32_t) * nsrc, cudaMemcpyHostToDevice, st);
  }
  cudaMemcpyAsync(d_tgt_c, tgt_c.data(), sizeof(int4) * ntgt, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_tgt_idx, tgt_idx.data(), sizeof(int32_t) * ntgt, cudaMemcpyHostToDevice, st);

  PhaseTimer tm;
  tm.start(o.timing != 0, st);
  const int64_t cs = (int64_t)m->nblocks[0] * B3;
  if ((rc = PairOps<R>::forward(B, f, dtype, cs, d_src_idx, nsrc, ncomp, ws->buf[0].p, nullptr, 0, st)))
    return rc;
  tm.mark(PH_FORWARD);
  if ((rc = PairOps<R>::mac(B, ws->buf[0].p, nsrc, (int64_t)nsrc * W, nullptr, d_src_c, Gh, t->mo, ws->buf[1].p,
                            ntgt, (int64_t)ntgt * W, nullptr, d_tgt_c, ncomp, 0, st)))
    return rc;
  tm.mark(PH_MAC);
  const double h = m->h0;
  const double scale = h * h / (double)((2 * B) * (2 * B) * (2 * B));
  if ((rc = PairOps<R>::inverse(B, ws->buf[1].p, (int64_t)ntgt * W, nullptr, d_tgt_idx, ntgt, ncomp, phi, dtype,
                                cs, 0, nullptr, 0, nullptr, 0, scale, st)))
    return rc;
  tm.mark(PH_INVERSE);
  tm.finish(rep);
  if (rep) {
    rep->target_cells = (int64_t)ntgt * B3;
    rep->source_blocks = nsrc;
    rep->target_blocks = ntgt;
    rep->pairs = (int64_t)nsrc * ntgt;
    rep->scratch_bytes = (int64_t)ws->total();
    rep->kernel_launches = 2 + (ncomp + 2) / 3;
    rep->mac_mode_used = LGF_MAC_PAIR;
  }
  if (o.timing) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(LGF_E_CUDA, "solve failed: %s", cudaGetErrorString(e));
  }
  return LGF_OK;
}

// Relative cost model of the two ways to evaluate the per-frequency block-pair sum (complex
// multiply-adds per real component): PAIR = nsrc * ntgt * (2B)^2 (B+1); BOX = block-index DFTs over the
// 2 nb grid plus the local transforms, shared by two components.
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

static size_t dtype_size(int dtype, size_t rsize) { return dtype == 0 ? 8 : (dtype == 1 ? 4 : rsize); }

template <class R>
static int solve_single_box(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                            const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st, const int lo[3],
                            const int nb[3]) {
  const int B = m->block, n = m->nblocks[0];
  const int64_t B3 = (int64_t)B * B * B;
  BoxSpec *S = nullptr;
  int rc = box_spectrum(t, nb, &S, st);
  if (rc) return rc;
  const int64_t nbox = (int64_t)nb[0] * nb[1] * nb[2];
  std::vector<int32_t> maps(2 * nbox, -1);
  int64_t nsrc = 0, ntgt = 0;
  for (int i = 0; i < n; ++i) {
    const int role = m->block_role ? m->block_role[i] : 3;
    const int32_t *b = m->block_ijk + 3 * i;
    const int64_t bi = ((int64_t)(b[2] - lo[2]) * nb[1] + (b[1] - lo[1])) * nb[0] + (b[0] - lo[0]);
    if (role & 1) maps[bi] = i, ++nsrc;
    if (role & 2) maps[nbox + bi] = i, ++ntgt;
  }
  Workspace *ws = workspace_for(t, st);
  const int64_t P3 = 8 * nbox;
  const size_t ybytes = sizeof(cx<R>) * (size_t)P3 * B3;
  if ((rc = ws->buf[0].reserve(ybytes)) || (rc = ws->buf[1].reserve(ybytes)) ||
      (rc = ws->buf[2].reserve(sizeof(int32_t) * 2 * nbox)))
    return rc;
  int32_t *dmap = (int32_t *)ws->buf[2].p;
  cudaMemcpyAsync(dmap, maps.data(), sizeof(int32_t) * 2 * nbox, cudaMemcpyHostToDevice, st);
  PhaseTimer tm;
  tm.start(o.timing != 0, st);
  const int64_t cs = (int64_t)n * B3;
  const size_t es = dtype_size(dtype, sizeof(R));
  const double Pc3 = 8.0 * nb[0] * nb[1] * nb[2] * (double)B3;
  const double scale = m->h0 * m->h0 / Pc3;
  int64_t launches = 0;
  for (int c0 = 0; c0 < ncomp; c0 += 2) {
    const int c1 = c0 + 1;
    InSpec in[2];
    in[0] = InSpec{dmap, (const char *)f + es * c0 * cs, nullptr, dtype, 0, 0};
    int nspec = 1;
    if (c1 < ncomp) in[nspec++] = InSpec{dmap, (const char *)f + es * c1 * cs, nullptr, dtype, 0, 1};
    OutSpec<R> ore{dmap + nbox, nullptr, phi, nullptr, nullptr, c0 * cs, dtype, 0};
    OutSpec<R> oim{};
    if (c1 < ncomp) oim = OutSpec<R>{dmap + nbox, nullptr, phi, nullptr, nullptr, c1 * cs, dtype, 0};
    if ((rc = BoxOps<R>::convolve(B, S, nspec, in, ore, oim, scale, (cx<R> *)ws->buf[0].p, (cx<R> *)ws->buf[1].p,
                                  st, o.timing ? phase_mark_cb : nullptr, &tm)))
      return rc;
    launches += 7;
  }
  tm.finish(rep);
  if (rep) {
    rep->target_cells = ntgt * B3;
    rep->source_blocks = nsrc;
    rep->target_blocks = ntgt;
    rep->pairs = 0;
    rep->scratch_bytes = (int64_t)ws->total() + (int64_t)S->bytes;
    rep->kernel_launches = launches;
    rep->mac_mode_used = LGF_MAC_BOX;
  }
  if (o.timing) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(LGF_E_CUDA, "solve failed: %s", cudaGetErrorString(e));
  }
  return LGF_OK;
}

template <class R>
static int solve_single_any(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                            const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  double nsrc = 0, ntgt = 0;
  for (int i = 0; i < m->nblocks[0]; ++i) {
    const int role = m->block_role ? m->block_role[i] : 3;
    if (!role) continue;
    nsrc += role & 1;
    ntgt += (role >> 1) & 1;
    for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], m->block_ijk[3 * i + a]), hi[a] = std::max(hi[a], m->block_ijk[3 * i + a]);
  }
  int nb[3];
  bool box_ok = ntgt > 0;
  for (int a = 0; a < 3; ++a) {
    nb[a] = hi[a] - lo[a] + 1;
    if (nb[a] < 1 || nb[a] > BOX_NB_MAX) box_ok = false;
  }
  int mode = o.mac_mode;
  if (mode == LGF_MAC_AUTO) mode = (box_ok && box_cost(m->block, nb) < pair_cost(m->block, nsrc, ntgt)) ? LGF_MAC_BOX : LGF_MAC_PAIR;
  if (mode == LGF_MAC_BOX) {
    if (!box_ok) return set_error(LGF_E_UNSUPPORTED, "BOX mode needs 1..%d blocks per axis", BOX_NB_MAX);
    return solve_single_box<R>(t, m, ncomp, f, phi, dtype, o, rep, st, lo, nb);
  }
  return solve_single<R>(t, m, ncomp, f, phi, dtype, o, rep, st);
}

int solve_poisson(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                  const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  if (m->nlevels > 1) return solve_multi(t, m, ncomp, f, phi, dtype, o, rep, st);
  switch (o.precision) {
    case LGF_PREC_FP64: return solve_single_any<double>(t, m, ncomp, f, phi, dtype, o, rep, st);
    case LGF_PREC_FP32: return solve_single_any<float>(t, m, ncomp, f, phi, dtype, o, rep, st);
    default: return solve_single_any<df>(t, m, ncomp, f, phi, dtype, o, rep, st);
  }
}

}  // namespace lgf
