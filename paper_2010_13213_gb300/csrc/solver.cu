// solver.cu -- host driver of the single-level solve (Sec. 2.2) in pair mode; dispatch of the
// multi-level (Sec. 3.4) and heat (Sec. 3.5) drivers.
#include <algorithm>
#include <vector>

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

int solve_poisson(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                  const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  if (m->nlevels > 1) return solve_multi(t, m, ncomp, f, phi, dtype, o, rep, st);
  if (o.mac_mode == LGF_MAC_BOX) return set_error(LGF_E_UNSUPPORTED, "BOX mode not built yet");
  switch (o.precision) {
    case LGF_PREC_FP64: return solve_single<double>(t, m, ncomp, f, phi, dtype, o, rep, st);
    case LGF_PREC_FP32: return solve_single<float>(t, m, ncomp, f, phi, dtype, o, rep, st);
    default: return solve_single<df>(t, m, ncomp, f, phi, dtype, o, rep, st);
  }
}

}  // namespace lgf
