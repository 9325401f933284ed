// multi.cu -- host drivers of the composite-mesh Poisson solve (FLGF-AMR, Sec. 3.4) and of the
// heat apply (FIF-AMR, Sec. 3.5), plus the plan cache.
//
// FLGF-AMR, per call:
//   1. fine to coarse:  F_k = [Omega_k] fhat_k + P_{k+1->k} F_{k+1}            (k_restrict, k_coarsen_add)
//   2. coarse to fine, level k:
//        c_k   = P_{k-1->k} psi_{k-1}                                          (k_interp, k >= 1)
//        A_k   = [Omega_k] fhat_k + [Omega_k u Omega_k^E] S psi_{k-1}           (k_correct)
//        Fhat  = spectra of A_k (blocks SA) and of F_k on covered cells (blocks SB) (k_block_fwd)
//        Phi   = sum over pairs of Ghat * Fhat_A for all targets                (k_mac_pair)
//        psi_k = c_k + h_k^2 G * A_k on the psi targets                         (k_block_inv)
//        Phi  += sum over pairs of Ghat * Fhat_B on the Omega_k targets          (k_mac_pair)
//        phi   = c_k + h_k^2 G * (A_k + B_k) written on Omega_k                  (k_block_inv)
//   3. optional FP64 residual L_k phi - F_k - P L_{k-1} psi_{k-1}                (k_residual)
#include <string.h>

#include <algorithm>
#include <cmath>
#include <list>
#include <mutex>
#include <string>
#include <vector>

#include "amr.cuh"
#include "box_ops.cuh"
#include "indicator.cuh"
#include "plan.h"
#include "solver.h"

namespace lgf {

double box_cost(int B, const int nb[3]);
double pair_cost(int B, double nsrc, double ntgt);

// Dynamic shared memory of k_correct with the correction (the staged c cube; with the static coarse cube
// above the default 48 KB for 8-byte arithmetics, so the limit is raised once per arithmetic).
template <class R>
static size_t correct_smem(int B) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_correct<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)halo_smem<R>(16));
  });
  return halo_smem<R>(B);
}

// ------------------------------------------------------------------ plan cache (process-wide)
static std::mutex g_plan_mu;
static std::list<std::pair<std::string, Plan *>> g_plans;  // most recent first

static std::string plan_key(const lgf_mesh *m, const int *radii) {
  std::string k;
  int dev = 0;
  cudaGetDevice(&dev);
  int64_t tot = 0;
  for (int i = 0; i < m->nlevels; ++i) tot += m->nblocks[i];
  auto put = [&](const void *p, size_t n) { k.append((const char *)p, n); };
  put(&dev, sizeof dev);
  put(&m->nlevels, 4);
  put(&m->block, 4);
  put(&m->n_ext, 4);
  put(m->nblocks, 4 * (size_t)m->nlevels);
  put(m->block_ijk, 12 * (size_t)tot);
  const char h = radii ? 1 : 0;
  put(&h, 1);
  if (radii) put(radii, 4 * (size_t)m->nlevels);
  return k;
}

int get_plan(const lgf_mesh *m, const int *radii, Plan **out) {
  const std::string key = plan_key(m, radii);
  std::lock_guard<std::mutex> g(g_plan_mu);
  for (auto it = g_plans.begin(); it != g_plans.end(); ++it)
    if (it->first == key) {
      g_plans.splice(g_plans.begin(), g_plans, it);
      *out = it->second;
      return LGF_OK;
    }
  Plan *P = nullptr;
  int rc = build_plan(m, radii, &P);
  if (rc) return rc;
  g_plans.emplace_front(key, P);
  while (g_plans.size() > 1024) {
    delete g_plans.back().second;  // cudaFree inside orders against in-flight work
    g_plans.pop_back();
  }
  *out = P;
  return LGF_OK;
}

// Device view of level k; the spacing comes from the caller's mesh (plans are keyed by geometry only).
static LevelDev level_dev(const Plan *P, int k, double h0) {
  const LevelPlan &L = P->L[k];
  LevelDev d;
  d.map = L.d_map;
  d.lo = make_int3(L.bb_lo[0], L.bb_lo[1], L.bb_lo[2]);
  d.n = make_int3(L.bb_n[0], L.bb_n[1], L.bb_n[2]);
  d.cellmask = L.d_cellmask;
  d.user_of = L.d_user_of;
  int s = 0;
  while ((1 << s) < P->B) ++s;
  d.shift = s;
  d.h = h0 / (double)(1 << k);
  return d;
}

template <class R>
static const void *spectra_for(const lgf_table *t);
template <>
const void *spectra_for<double>(const lgf_table *t) { return t->s64; }
template <>
const void *spectra_for<float>(const lgf_table *t) { return t->s32; }
template <>
const void *spectra_for<df>(const lgf_table *t) { return t->sdf; }

static int check_range(const Plan *P, const lgf_table *t) {
  const int mo[3] = {t->mo.x, t->mo.y, t->mo.z};
  for (const auto &L : P->L) {
    int slo[3] = {1 << 30, 1 << 30, 1 << 30}, shi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    int tlo[3] = {1 << 30, 1 << 30, 1 << 30}, thi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    auto acc = [&](const std::vector<int32_t> &lst, int *lo, int *hi) {
      for (int b : lst) {
        const int v[3] = {L.BL[b].x, L.BL[b].y, L.BL[b].z};
        for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], v[a]), hi[a] = std::max(hi[a], v[a]);
      }
    };
    acc(L.SA, slo, shi);
    acc(L.SB, slo, shi);
    acc(L.Tall, tlo, thi);
    if (L.Tall.empty() || (L.SA.empty() && L.SB.empty())) continue;
    for (int a = 0; a < 3; ++a) {
      const int reach = std::max(thi[a] - slo[a], shi[a] - tlo[a]);
      if (reach > mo[a])
        return set_error(LGF_E_TABLE_RANGE,
                         "level %d needs block offsets up to %d along axis %d; the table covers %d", L.k, reach,
                         a, mo[a]);
    }
  }
  return LGF_OK;
}

#define LGF_LAUNCH_CHECK(what)                                                                   \
  do {                                                                                           \
    cudaError_t e_ = cudaGetLastError();                                                         \
    if (e_ != cudaSuccess) return set_error(LGF_E_CUDA, "%s launch: %s", what, cudaGetErrorString(e_)); \
    ++launches;                                                                                  \
  } while (0)

template <class R>
static int solve_multi_t(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                         const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st, const lgf_indicator *ind) {
  Plan *P = nullptr;
  int rc = get_plan(m, nullptr, &P);
  if (rc) return rc;
  if ((rc = check_range(P, t))) return rc;
  if (ind && P->K > LGF_IND_MAX_LEVELS)
    return set_error(LGF_E_UNSUPPORTED, "refinement indicator on more than %d levels", LGF_IND_MAX_LEVELS);
  const void *Gh = spectra_for<R>(t);  // null for a box-only table: every level then runs in box mode
  const int B = P->B, K = P->K;
  const int64_t B3 = (int64_t)B * B * B;
  const int W = (2 * B) * (2 * B) * (B + 1);
  int64_t total_user = 0;
  for (int k = 0; k < K; ++k) total_user += P->L[k].nU;
  const int64_t ucs = total_user * B3;
  // workspace layout
  std::vector<int64_t> Foff(K + 1, 0), cs(K);
  int64_t maxBL = 0, maxSA = 0, maxSB = 0, maxT = 0;
  for (int k = 0; k < K; ++k) {
    const LevelPlan &L = P->L[k];
    cs[k] = (int64_t)L.BL.size() * B3;
    Foff[k + 1] = Foff[k] + ncomp * cs[k];
    maxBL = std::max<int64_t>(maxBL, (int64_t)L.BL.size());
    maxSA = std::max<int64_t>(maxSA, (int64_t)L.SA.size());
    maxSB = std::max<int64_t>(maxSB, (int64_t)L.SB.size());
    maxT = std::max<int64_t>(maxT, (int64_t)L.nTall);
  }
  // per level: pair or block-index FFT (box) evaluation of the block-pair sums
  std::vector<int> use_box(K, 0);
  int64_t maxbox = 0;
  for (int k = 0; k < K; ++k) {
    const LevelPlan &L = P->L[k];
    if (!L.box_ok || L.Tall.empty()) continue;
    if (o.mac_mode == LGF_MAC_BOX || !Gh || (o.mac_mode == LGF_MAC_AUTO && o.dft_slices > 0)) {
      use_box[k] = 1;
    } else if (o.mac_mode == LGF_MAC_AUTO) {
      const bool packAB = !L.Tpsi.empty() || !L.SB.empty();
      const double cb = box_cost(B, L.box_nb) * (packAB ? 2.0 : 1.0);
      const double cp = pair_cost(B, (double)L.SA.size(), (double)L.nTall) +
                        pair_cost(B, (double)L.SB.size(), (double)L.Tphi.size());
      use_box[k] = cb < cp;
    }
    if (use_box[k]) maxbox = std::max<int64_t>(maxbox, (int64_t)std::min(ncomp, BOX_MAXF) * 8 * L.nbox * B3);
  }
  for (int k = 0; k < K; ++k)
    if (!use_box[k] && !P->L[k].Tall.empty() && (o.mac_mode == LGF_MAC_BOX || !Gh))
      return set_error(Gh ? LGF_E_UNSUPPORTED : LGF_E_INVALID_ARG,
                       "level %d needs the pair mode (box over 16 blocks per axis) and the table has no %s", k,
                       Gh ? "box support for it" : "pair spectra of this precision");
  Workspace *ws = workspace_for(t, st);
  const size_t field = sizeof(R) * (size_t)ncomp * maxBL * B3;
  const size_t ybytes = sizeof(cx<R>) * (size_t)maxbox;
  if ((rc = ws->buf[0].reserve(std::max(ybytes, sizeof(cx<R>) * (size_t)ncomp * std::max<int64_t>(maxSA, 1) * W))) ||
      (rc = ws->buf[1].reserve(std::max(ybytes, sizeof(cx<R>) * (size_t)ncomp * std::max<int64_t>(maxT, 1) * W))) ||
      (rc = ws->buf[3].reserve(sizeof(cx<R>) * (size_t)ncomp * std::max<int64_t>(maxSB, 1) * W)) ||
      (rc = ws->buf[4].reserve(sizeof(R) * (size_t)Foff[K])) || (rc = ws->buf[5].reserve(field)) ||
      (rc = ws->buf[6].reserve(field)) || (rc = ws->buf[7].reserve(sizeof(R) * (size_t)Foff[K])) ||
      (rc = ws->buf[9].reserve(sizeof(unsigned long long) * 2 * K)) || (rc = ws->buf[8].reserve(field)))
    return rc;
  cx<R> *FA = (cx<R> *)ws->buf[0].p, *Phi = (cx<R> *)ws->buf[1].p, *FB = (cx<R> *)ws->buf[3].p;
  R *Fall = (R *)ws->buf[4].p, *A = (R *)ws->buf[5].p, *c = (R *)ws->buf[6].p;
  R *Psi = (R *)ws->buf[7].p;  // psi_k of every level, [level][ncomp][nBL_k][B^3]
  R *Lpsi = (R *)ws->buf[8].p;  // L_{k-1} psi_{k-1} of the current coarse level
  unsigned long long *racc = (unsigned long long *)ws->buf[9].p;
  // refinement indicator: per level and internal block the sum of |S_k|^2 and max |S_k|
  std::vector<int64_t> ind_off(K + 1, 0);
  for (int k = 0; k < K; ++k) ind_off[k + 1] = ind_off[k] + (int64_t)P->L[k].BL.size();
  if (ind && ((rc = ws->buf[16].reserve(sizeof(double) * 2 * (size_t)std::max<int64_t>(ind_off[K], 1))) ||
              (rc = ws->buf[17].reserve(sizeof(int) * (size_t)std::max<int64_t>(total_user, 1)))))
    return rc;
  double *ind_ss = ind ? (double *)ws->buf[16].p : nullptr, *ind_mx = ind ? ind_ss + ind_off[K] : nullptr;
  int64_t launches = 0;
  PhaseTimer tm;
  tm.start(o.timing != 0, st);
  // 1. cumulative coarsening
  for (int k = K - 1; k >= 0; --k) {
    const LevelPlan &L = P->L[k];
    const LevelDev Ld = level_dev(P, k, m->h0);
    k_restrict<R><<<dim3(L.nU, ncomp), 256, 0, st>>>(Ld, f, dtype, ucs, L.user_off, Fall + Foff[k], cs[k]);
    LGF_LAUNCH_CHECK("restrict");
    if (k + 1 < K) {
      const LevelPlan &Lf = P->L[k + 1];
      k_coarsen_add<R><<<dim3(Lf.nU, ncomp), 256, 0, st>>>(Ld, Fall + Foff[k], cs[k], Lf.d_BL, Fall + Foff[k + 1],
                                                          cs[k + 1]);
      LGF_LAUNCH_CHECK("coarsen");
    }
  }
  tm.mark(PH_RESTRICT);
  int64_t target_cells = 0, nsrc_total = 0, ntgt_total = 0, pairs = 0;
  // 2. coarse to fine
  for (int k = 0; k < K; ++k) {
    const LevelPlan &L = P->L[k];
    const LevelDev Ld = level_dev(P, k, m->h0);
    const LevelDev Lc = k > 0 ? level_dev(P, k - 1, m->h0) : Ld;
    const int64_t ccs = k > 0 ? cs[k - 1] : 0;
    const R *psi_prev = k > 0 ? Psi + Foff[k - 1] : nullptr;
    R *psi_cur = Psi + Foff[k];
    const int nSA = (int)L.SA.size(), nSB = (int)L.SB.size(), nT = L.nTall, nPhi = (int)L.Tphi.size();
    const int nPsi = (int)L.Tpsi.size();
    const int32_t *lists = L.d_lists;
    if (k > 0) {
      k_interp<R><<<dim3((unsigned)L.BL.size(), ncomp), 256, sizeof(R) * (size_t)interp_sep_values(B), st>>>(
          Ld, L.d_BL, c, cs[k], Lc, psi_prev, ccs);
      LGF_LAUNCH_CHECK("interp");
      tm.mark(PH_INTERP);
    }
    const bool corr = k > 0 && !(o.flags & LGF_SOLVE_NO_CORRECTION);
    if (nSA) {
      if (corr && !L.LP.empty()) {  // L_{k-1} psi_{k-1} once per coarse cell read, then interpolated per fine cell
        k_lap<R><<<dim3((unsigned)L.LP.size(), ncomp), 512, halo_smem<R>(B), st>>>(
            Lc, P->L[k - 1].d_BL, lists + L.off_LP, psi_prev, Lpsi, ccs);
        LGF_LAUNCH_CHECK("coarse Laplacian");
      }
      k_correct<R><<<dim3(nSA, ncomp), 512, corr ? correct_smem<R>(B) : 0, st>>>(
          Ld, L.d_BL, lists + L.off_SA, f, dtype, ucs, A, cs[k], c, Lc, Lpsi, ccs, corr);
      LGF_LAUNCH_CHECK("correct");
      tm.mark(PH_CORRECT);
    }
    if (ind && !L.BL.empty()) {  // the combined source S_k = A_k + [covered] F_k, before A is reused
      k_ind_stats<R><<<(unsigned)L.BL.size(), 256, 0, st>>>(Ld, L.nU, ncomp, A, Fall + Foff[k], cs[k],
                                                             ind_ss + ind_off[k], ind_mx + ind_off[k]);
      LGF_LAUNCH_CHECK("indicator statistics");
    }
    if (use_box[k]) {
      BoxSpec *S = nullptr;
      if ((rc = box_spectrum(t, L.box_nb, &S, st))) return rc;
      const int32_t *gA = L.d_box, *gB = gA + L.nbox, *sPsi = gB + L.nbox, *sPhi = sPsi + L.nbox;
      const double hk = m->h0 / (double)(1 << k);
      const double scale = hk * hk / (8.0 * L.nbox * (double)B3);
      const bool packAB = nPsi > 0 || nSB > 0;
      const R *cadd = k > 0 ? c : nullptr;
      cx<R> *Y0 = (cx<R> *)ws->buf[0].p, *Y1 = (cx<R> *)ws->buf[1].p;
      std::vector<int> nin;
      std::vector<InSpec3> in;
      std::vector<OutSpec<R>> ore, oim;
      if (packAB) {
        // z = A + i (A + B): real part -> psi_k on the psi targets, imaginary part -> phi on Omega_k
        for (int cc = 0; cc < ncomp; ++cc) {
          InSpec sp[3];
          int ns = 0;
          if (nSA) {
            sp[ns++] = InSpec{gA, A + cc * cs[k], nullptr, 2, 0, 0};
            sp[ns++] = InSpec{gA, A + cc * cs[k], nullptr, 2, 0, 1};
          }
          if (nSB) sp[ns++] = InSpec{gB, Fall + Foff[k] + cc * cs[k], L.d_cellmask, 2, CB_COV, 1};
          nin.push_back(ns);
          in.emplace_back();
          for (int q = 0; q < 3; ++q) in.back().s[q] = sp[q];
          ore.push_back(OutSpec<R>{nPsi ? sPsi : nullptr, nullptr, Psi + Foff[k], cadd ? cadd + cc * cs[k] : nullptr,
                                   nullptr, cc * cs[k], 2, 0});
          oim.push_back(OutSpec<R>{nPhi ? sPhi : nullptr, nullptr, phi, cadd ? cadd + cc * cs[k] : nullptr,
                                   L.d_cellmask, cc * ucs + L.user_off * B3, dtype, CB_OM});
        }
      } else {
        // finest level without psi targets: two components per complex field, both to phi
        for (int c0 = 0; c0 < ncomp; c0 += 2) {
          const int c1 = c0 + 1;
          InSpec sp[3] = {};
          int ns = 0;
          sp[ns++] = InSpec{gA, A + c0 * cs[k], nullptr, 2, 0, 0};
          if (c1 < ncomp) sp[ns++] = InSpec{gA, A + c1 * cs[k], nullptr, 2, 0, 1};
          nin.push_back(ns);
          in.emplace_back();
          for (int q = 0; q < 3; ++q) in.back().s[q] = sp[q];
          ore.push_back(OutSpec<R>{sPhi, nullptr, phi, cadd ? cadd + c0 * cs[k] : nullptr, L.d_cellmask,
                                   c0 * ucs + L.user_off * B3, dtype, CB_OM});
          oim.push_back(c1 < ncomp ? OutSpec<R>{sPhi, nullptr, phi, cadd ? cadd + c1 * cs[k] : nullptr, L.d_cellmask,
                                                c1 * ucs + L.user_off * B3, dtype, CB_OM}
                                   : OutSpec<R>{});
        }
      }
      const int nf = (int)nin.size();
      if ((rc = BoxOps<R>::convolve(B, S, nf, nin.data(), in.data(), ore.data(), oim.data(), scale, Y0, Y1, st,
                                    o.timing ? phase_mark_cb : nullptr, &tm, o.dft_slices, t->d_status, &launches)))
        return rc;
      target_cells += L.n_omega;
      nsrc_total += nSA + nSB;
      ntgt_total += nT;
      continue;
    }
    if (nSA) {
      if ((rc = PairOps<R>::forward(B, A, 2, cs[k], lists + L.off_SA, nSA, ncomp, FA, nullptr, 0, st))) return rc;
      ++launches;
    }
    if (nSB) {
      if ((rc = PairOps<R>::forward(B, Fall + Foff[k], 2, cs[k], lists + L.off_SB, nSB, ncomp, FB, L.d_cellmask,
                                    CB_COV, st)))
        return rc;
      ++launches;
    }
    tm.mark(PH_FORWARD);
    const double hk = m->h0 / (double)(1 << k);
    const double scale = hk * hk / (double)((2 * B) * (2 * B) * (2 * B));
    const int64_t pcs = (int64_t)nT * W;
    if (nSA) {
      if ((rc = PairOps<R>::mac(B, FA, nSA, (int64_t)nSA * W, lists + L.off_SA, L.d_BL, Gh, t->mo, Phi, nT, pcs,
                                lists + L.off_Tall, L.d_BL, ncomp, 0, st)))
        return rc;
    } else {
      cudaMemsetAsync(Phi, 0, sizeof(cx<R>) * (size_t)ncomp * nT * W, st);
    }
    launches += (ncomp + 2) / 3;
    pairs += (int64_t)nSA * nT;
    tm.mark(PH_MAC);
    if (nPsi) {
      if ((rc = PairOps<R>::inverse(B, Phi, pcs, lists + L.off_psi, lists + L.off_Tpsi, nPsi, ncomp, psi_cur, 2,
                                    cs[k], 0, k > 0 ? c : nullptr, cs[k], nullptr, 0, scale, st)))
        return rc;
      ++launches;
    }
    tm.mark(PH_INVERSE);
    if (nSB && nPhi) {
      if ((rc = PairOps<R>::mac(B, FB, nSB, (int64_t)nSB * W, lists + L.off_SB, L.d_BL, Gh, t->mo, Phi, nPhi, pcs,
                                lists + L.off_Tall, L.d_BL, ncomp, 1, st)))
        return rc;
      launches += (ncomp + 2) / 3;
      pairs += (int64_t)nSB * nPhi;
      tm.mark(PH_MAC);
    }
    if (nPhi) {
      if ((rc = PairOps<R>::inverse(B, Phi, pcs, nullptr, lists + L.off_Tall, nPhi, ncomp, phi, dtype, ucs,
                                    L.user_off, k > 0 ? c : nullptr, cs[k], L.d_cellmask, CB_OM, scale, st)))
        return rc;
      ++launches;
    }
    tm.mark(PH_INVERSE);
    target_cells += L.n_omega;
    nsrc_total += nSA + nSB;
    ntgt_total += nT;
  }
  if (ind) {
    IndArgs a{};
    a.K = K;
    a.B3 = (int)B3;
    a.nlmax = ind->n_levels_max;
    a.alpha = ind->alpha;
    a.beta = ind->beta;
    for (int k = 0; k < K; ++k) {
      const LevelPlan &L = P->L[k];
      a.lv[k] = IndLevel{level_dev(P, k, m->h0), L.d_BL, (int)L.BL.size(), L.nU, L.user_off,
                         ind_ss + ind_off[k], ind_mx + ind_off[k]};
    }
    k_ind_flags<<<1, 1024, 0, st>>>(a, ind->rms_dev, ind->flags_dev, ind->s_max_dev, (int *)ws->buf[17].p);
    LGF_LAUNCH_CHECK("indicator flags");
  }
  // 3. residual
  double resid = 0.0;
  if (o.residual) {
    cudaMemsetAsync(racc, 0, sizeof(unsigned long long) * 2 * K, st);
    for (int k = 0; k < K; ++k) {
      const LevelPlan &L = P->L[k];
      if (L.Tphi.empty()) continue;
      const LevelDev Ld = level_dev(P, k, m->h0);
      const LevelDev Lc = k > 0 ? level_dev(P, k - 1, m->h0) : Ld;
      k_residual<R><<<dim3((unsigned)L.Tphi.size(), ncomp), 256, 0, st>>>(
          Ld, L.d_BL, L.d_lists + L.off_Tall, phi, dtype, ucs, Fall + Foff[k], cs[k], Lc,
          k > 0 ? Psi + Foff[k - 1] : nullptr, k > 0 ? cs[k - 1] : 0, k > 0, racc + 2 * k);
      LGF_LAUNCH_CHECK("residual");
    }
    std::vector<unsigned long long> h(2 * K);
    cudaMemcpyAsync(h.data(), racc, sizeof(unsigned long long) * 2 * K, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return set_error(LGF_E_CUDA, "residual failed");
    for (int k = 0; k < K; ++k) {
      double r, s;
      memcpy(&r, &h[2 * k], 8);
      memcpy(&s, &h[2 * k + 1], 8);
      if (s > 0) resid = std::max(resid, r / s);
    }
    tm.mark(PH_RESIDUAL);
  }
  tm.finish(rep);
  if (rep) {
    rep->residual_rel = resid;
    rep->target_cells = target_cells;
    rep->source_blocks = nsrc_total;
    rep->target_blocks = ntgt_total;
    rep->pairs = pairs;
    rep->scratch_bytes = (int64_t)ws->total() + (int64_t)P->device_bytes;
    rep->kernel_launches = launches;
    rep->mac_mode_used = LGF_MAC_PAIR;
    for (int k = 0; k < K; ++k)
      if (use_box[k]) rep->mac_mode_used = LGF_MAC_BOX;
    // method-minimum work (see lgf_report): per level the source cells (Omega_k, Omega_k^E and covered
    // cells) read and the target cells (Omega_k and the psi targets) written once per component, the
    // unique spectrum values, and the transforms / pair sums of the level's evaluation
    const double w = dtype == LGF_F32 ? 4.0 : 8.0, W2 = (2.0 * B) * (2.0 * B) * (B + 1.0);
    double bytes = 0.0, flops = 0.0;
    for (int k = 0; k < K; ++k) {
      const LevelPlan &L = P->L[k];
      if (L.Tall.empty()) continue;
      const double tgt = (double)L.n_omega + (double)L.Tpsi.size() * B3;
      bytes += ncomp * ((double)L.n_src + tgt) * w;
      const bool packAB = !L.Tpsi.empty() || !L.SB.empty();
      if (use_box[k]) {
        double uniq = 1.0, M = 1.0;
        for (int a = 0; a < 3; ++a) uniq *= L.box_nb[a] * B + 1.0, M *= 2.0 * L.box_nb[a] * B;
        bytes += uniq * sizeof(R);
        flops += 2.0 * (packAB ? ncomp : (ncomp + 1) / 2) * 5.0 * M * std::log2(M);
      } else {
        int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
        for (const auto &lst : {L.SA, L.SB, L.Tall})
          for (int b : lst) {
            const int v[3] = {L.BL[b].x, L.BL[b].y, L.BL[b].z};
            for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], v[a]), hi[a] = std::max(hi[a], v[a]);
          }
        double noff = 1.0;
        for (int a = 0; a < 3; ++a) noff *= 2.0 * (hi[a] - lo[a]) + 1.0;
        bytes += noff * W2 * 2.0 * sizeof(R);
        const double m = 8.0 * B3;
        flops += ((double)L.SA.size() + L.SB.size() + L.nTall) * ncomp * 0.5 * 5.0 * m * std::log2(m) +
                 8.0 * W2 * ncomp * ((double)L.SA.size() * L.nTall + (double)L.SB.size() * L.Tphi.size());
      }
    }
    rep->alg_bytes = (int64_t)bytes;
    rep->alg_flops = flops;
  }
  if (o.timing || o.residual) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(LGF_E_CUDA, "solve failed: %s", cudaGetErrorString(e));
    if (o.dft_slices > 0 && (rc = take_device_status(t))) return rc;
  }
  if (o.residual && o.residual_tol > 0 && resid > o.residual_tol)
    return set_error(LGF_E_PRECISION, "FP64 residual %.3e exceeds the tolerance %.3e", resid, o.residual_tol);
  return LGF_OK;
}

int solve_multi(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st, const lgf_indicator *ind) {
  switch (o.precision) {
    case LGF_PREC_FP64: return solve_multi_t<double>(t, m, ncomp, f, phi, dtype, o, rep, st, ind);
    case LGF_PREC_FP32: return solve_multi_t<float>(t, m, ncomp, f, phi, dtype, o, rep, st, ind);
    default: return solve_multi_t<df>(t, m, ncomp, f, phi, dtype, o, rep, st, ind);
  }
}

// ------------------------------------------------------------------ heat apply
// e^{-x} I_n(x), n <= nmax, by Miller's backward recurrence normalised with the generating-function
// sum e^{-x} (I_0 + 2 sum I_n) = 1 (host, FP64).
static void scaled_bessel(double x, int nmax, double *out) {
  for (int n = 0; n <= nmax; ++n) out[n] = 0.0;
  if (x <= 0.0) {
    out[0] = 1.0;
    return;
  }
  const int M = nmax + 60 + (int)std::sqrt(120.0 * x);
  double tot = 0.0;
  std::vector<double> v(M + 2, 0.0);
  v[M] = 1e-30;
  for (int n = M; n >= 1; --n) {
    const double lo = (2.0 * n / x) * v[n] + v[n + 1];
    v[n - 1] = lo;
    if (lo > 1e200) {
      for (int j = n - 1; j <= M; ++j) v[j] *= 1e-200;
    }
  }
  tot = v[0];
  for (int n = 1; n <= M; ++n) tot += 2.0 * v[n];
  for (int n = 0; n <= nmax; ++n) out[n] = v[n] / tot;
}

static int heat_weights(double alpha, HeatW *w) {
  double tmp[80];
  scaled_bessel(2.0 * alpha, 79, tmp);
  int r = -1;
  for (int n = 0; n < 80; ++n) {
    if (tmp[n] < 1e-18) break;
    r = n;
  }
  if (r < 0) r = 0;
  if (r > 64) return set_error(LGF_E_UNSUPPORTED, "heat kernel radius %d above 64 (alpha %.3g too large)", r, alpha);
  w->r = r;
  for (int n = 0; n <= 64; ++n) w->w[n] = n <= r ? tmp[n] : 0.0;
  return LGF_OK;
}

// One separable heat pass over a level's heat block set: the shared-memory line kernel for radii up to
// B, the block-map lookup kernel beyond.
template <class R, int BB>
static int heat_line_launch(const LevelDev &Ld, const int4 *BL, const int32_t *HB, int nHB, int ncomp, int ax,
                            const R *in, R *out, int64_t cs, const HeatW &w, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_heat_line<R, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)heat_line_smem<R, BB>(BB));
    attr = true;
  }
  k_heat_line<R, BB><<<dim3(nHB, ncomp), BB * BB, heat_line_smem<R, BB>(w.r), st>>>(Ld, BL, HB, ax, in, out, cs, w);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "heat pass launch: %s", cudaGetErrorString(e));
}
template <class R>
static int heat_pass_launch(int B, const LevelDev &Ld, const int4 *BL, const int32_t *HB, int nHB, int ncomp, int ax,
                            const R *in, R *out, int64_t cs, const HeatW &w, cudaStream_t st) {
  if (w.r <= B && B == 16) return heat_line_launch<R, 16>(Ld, BL, HB, nHB, ncomp, ax, in, out, cs, w, st);
  if (w.r <= B && B == 8) return heat_line_launch<R, 8>(Ld, BL, HB, nHB, ncomp, ax, in, out, cs, w, st);
  k_heat_pass<R><<<dim3(nHB, ncomp), 256, 0, st>>>(Ld, BL, HB, ax, in, out, cs, w);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "heat pass launch: %s", cudaGetErrorString(e));
}

template <class R>
static int heat_t(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *g, int dtype, double alpha,
                  const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  const int K = m->nlevels;
  std::vector<HeatW> W(K);
  std::vector<int> radii(K);
  int rc;
  for (int k = 0; k < K; ++k) {
    if ((rc = heat_weights(alpha * std::pow(4.0, -(double)(K - 1 - k)), &W[k]))) return rc;
    radii[k] = W[k].r;
  }
  Plan *P = nullptr;
  if ((rc = get_plan(m, radii.data(), &P))) return rc;
  const int B = P->B;
  const int64_t B3 = (int64_t)B * B * B;
  int64_t total_user = 0, maxBL = 0;
  for (int k = 0; k < K; ++k) total_user += P->L[k].nU, maxBL = std::max<int64_t>(maxBL, P->L[k].BL.size());
  const int64_t ucs = total_user * B3;
  std::vector<int64_t> Foff(K + 1, 0), cs(K);
  for (int k = 0; k < K; ++k) {
    cs[k] = (int64_t)P->L[k].BL.size() * B3;
    Foff[k + 1] = Foff[k] + ncomp * cs[k];
  }
  Workspace *ws = workspace_for(t, st);
  const size_t field = sizeof(R) * (size_t)ncomp * maxBL * B3;
  if ((rc = ws->buf[10].reserve(sizeof(R) * (size_t)Foff[K])) || (rc = ws->buf[11].reserve(field)) ||
      (rc = ws->buf[12].reserve(field)) || (rc = ws->buf[13].reserve(field)) || (rc = ws->buf[14].reserve(field)))
    return rc;
  R *Fall = (R *)ws->buf[10].p, *T0 = (R *)ws->buf[11].p, *T1 = (R *)ws->buf[12].p;
  R *Uprev = (R *)ws->buf[13].p, *Ucur = (R *)ws->buf[14].p;
  int64_t launches = 0;
  PhaseTimer tm;
  tm.start(o.timing != 0, st);
  for (int k = K - 1; k >= 0; --k) {
    const LevelPlan &L = P->L[k];
    const LevelDev Ld = level_dev(P, k, m->h0);
    k_restrict<R><<<dim3(L.nU, ncomp), 256, 0, st>>>(Ld, f, dtype, ucs, L.user_off, Fall + Foff[k], cs[k]);
    LGF_LAUNCH_CHECK("restrict");
    if (k + 1 < K) {
      const LevelPlan &Lf = P->L[k + 1];
      k_coarsen_add<R><<<dim3(Lf.nU, ncomp), 256, 0, st>>>(Ld, Fall + Foff[k], cs[k], Lf.d_BL, Fall + Foff[k + 1],
                                                          cs[k + 1]);
      LGF_LAUNCH_CHECK("coarsen");
    }
  }
  tm.mark(PH_RESTRICT);
  int64_t target_cells = 0;
  for (int k = 0; k < K; ++k) {
    const LevelPlan &L = P->L[k];
    const LevelDev Ld = level_dev(P, k, m->h0);
    const LevelDev Lc = k > 0 ? level_dev(P, k - 1, m->h0) : Ld;
    const int nHB = (int)L.HB.size();
    const int32_t *HB = L.d_lists + L.off_HB;
    const size_t bytes = sizeof(R) * (size_t)ncomp * L.BL.size() * B3;
    cudaMemsetAsync(T0, 0, bytes, st);
    cudaMemsetAsync(T1, 0, bytes, st);
    cudaMemsetAsync(Ucur, 0, bytes, st);
    // P_k fhat into Ucur: the heat passes' source, kept for the next level's interpolation
    k_heat_build<R><<<dim3(nHB, ncomp), 256, sizeof(R) * (size_t)interp_sep_values(B), st>>>(
        Ld, L.d_BL, HB, Fall + Foff[k], L.nU, Ucur, cs[k], Lc, Uprev, k > 0 ? cs[k - 1] : 0, k > 0);
    LGF_LAUNCH_CHECK("heat source");
    tm.mark(PH_INTERP);
    for (int ax = 0; ax < 3; ++ax) {  // x: Ucur -> T1, y: T1 -> T0, z: T0 -> T1
      const R *hin = ax == 0 ? Ucur : (ax == 1 ? T1 : T0);
      R *hout = ax == 1 ? T0 : T1;
      if ((rc = heat_pass_launch<R>(B, Ld, L.d_BL, HB, nHB, ncomp, ax, hin, hout, cs[k], W[k], st))) return rc;
      ++launches;
    }
    k_heat_store<R><<<dim3(L.nU, ncomp), 256, 0, st>>>(Ld, T1, cs[k], g, dtype, ucs, L.user_off);
    LGF_LAUNCH_CHECK("heat store");
    tm.mark(PH_HEAT);
    target_cells += L.n_omega;
    std::swap(Uprev, Ucur);
  }
  tm.finish(rep);
  if (rep) {
    rep->target_cells = target_cells;
    rep->kernel_launches = launches;
    rep->scratch_bytes = (int64_t)ws->total() + (int64_t)P->device_bytes;
  }
  if (o.timing) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(LGF_E_CUDA, "heat apply failed: %s", cudaGetErrorString(e));
  }
  return LGF_OK;
}

// ------------------------------------------------------------------ HERK stage projection (Sec. 2.4, Sec. 3.6)
// Staggered fields: component a of a face field at cell n sits on the face n + (1/2,1/2,1/2) + e_a/2; the
// pressure at the cell centre.  D r(n) = sum_a (r_a[n] - r_a[n - e_a]) / h, (G p)_a[n] = (p[n + e_a] - p[n]) / h.

// D^r on the Omega_k cells of the caller's level-k blocks from the reconstruction T = P_k r^ (3 components,
// internal layout); 0 on the other cells.  grid (nU_k), 256 threads; out in the caller's layout (dtype).
template <class R>
__global__ void __launch_bounds__(256) k_proj_div(LevelDev L, const int4 *blocks, const R *T, int64_t cs, void *out,
                                                  int dtype, int64_t user_off) {
  const int b = blockIdx.x, sh = L.shift, B = 1 << sh, B3 = B * B * B;
  const int4 bc = blocks[b];
  const double inv_h = 1.0 / L.h;
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    double d = 0.0;
    if (L.cellmask[(int64_t)b * B3 + off] & 1) {
      const int x = (bc.x << sh) + (off & (B - 1)), y = (bc.y << sh) + ((off >> sh) & (B - 1)),
                z = (bc.z << sh) + (off >> (2 * sh));
      const double here = RT<R>::to_d(T[(int64_t)b * B3 + off]) + RT<R>::to_d(T[cs + (int64_t)b * B3 + off]) +
                          RT<R>::to_d(T[2 * cs + (int64_t)b * B3 + off]);
      const double back = RT<R>::to_d(fetch<R>(L, T, cs, 0, x - 1, y, z)) +
                          RT<R>::to_d(fetch<R>(L, T, cs, 1, x, y - 1, z)) +
                          RT<R>::to_d(fetch<R>(L, T, cs, 2, x, y, z - 1));
      d = (here - back) * inv_h;
    }
    store_field(out, (user_off + b) * (int64_t)B3 + off, dtype, d);
  }
}

// w^ = r^ - G p on the Omega_k cells from the caller's r and the reconstruction T = P_k p^ (1 component); 0 on
// the other cells.  grid (nU_k, 3).
template <class R>
__global__ void __launch_bounds__(256) k_proj_grad(LevelDev L, const int4 *blocks, const R *T, int64_t cs,
                                                   const void *r, void *w, int dtype, int64_t ucs, int64_t user_off) {
  const int b = blockIdx.x, a = blockIdx.y, sh = L.shift, B = 1 << sh, B3 = B * B * B;
  const int4 bc = blocks[b];
  const double inv_h = 1.0 / L.h;
  const int64_t o0 = a * ucs + (user_off + b) * (int64_t)B3;
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    double v = 0.0;
    if (L.cellmask[(int64_t)b * B3 + off] & 1) {
      const int x = (bc.x << sh) + (off & (B - 1)), y = (bc.y << sh) + ((off >> sh) & (B - 1)),
                z = (bc.z << sh) + (off >> (2 * sh));
      const double pn = RT<R>::to_d(T[(int64_t)b * B3 + off]);
      const double pe = RT<R>::to_d(fetch<R>(L, T, cs, 0, x + (a == 0), y + (a == 1), z + (a == 2)));
      v = load_field<double>(r, o0 + off, dtype) - (pe - pn) * inv_h;
    }
    store_field(w, o0 + off, dtype, v);
  }
}

// P_k f^ of every level on the plan's heat block set (own values on Omega_k, interpolation of the coarser
// levels, 8-child means of the finer ones; as in FIF-AMR); consume(k, T, cs_k) runs after level k's T.
template <class R, class Consume>
static int reconstruct_levels(Plan *P, const lgf_mesh *m, int ncomp, const void *f, int dtype, Workspace *ws,
                              int64_t &launches, cudaStream_t st, Consume consume) {
  const int K = P->K, B = P->B;
  const int64_t B3 = (int64_t)B * B * B;
  int64_t total_user = 0, maxBL = 0;
  for (int k = 0; k < K; ++k) total_user += P->L[k].nU, maxBL = std::max<int64_t>(maxBL, P->L[k].BL.size());
  const int64_t ucs = total_user * B3;
  std::vector<int64_t> Foff(K + 1, 0), cs(K);
  for (int k = 0; k < K; ++k) {
    cs[k] = (int64_t)P->L[k].BL.size() * B3;
    Foff[k + 1] = Foff[k] + ncomp * cs[k];
  }
  const size_t field = sizeof(R) * (size_t)ncomp * maxBL * B3;
  int rc;
  if ((rc = ws->buf[10].reserve(sizeof(R) * (size_t)Foff[K])) || (rc = ws->buf[13].reserve(field)) ||
      (rc = ws->buf[14].reserve(field)))
    return rc;
  R *Fall = (R *)ws->buf[10].p, *Uprev = (R *)ws->buf[13].p, *Ucur = (R *)ws->buf[14].p;
  for (int k = K - 1; k >= 0; --k) {
    const LevelPlan &L = P->L[k];
    const LevelDev Ld = level_dev(P, k, m->h0);
    k_restrict<R><<<dim3(L.nU, ncomp), 256, 0, st>>>(Ld, f, dtype, ucs, L.user_off, Fall + Foff[k], cs[k]);
    LGF_LAUNCH_CHECK("restrict");
    if (k + 1 < K) {
      const LevelPlan &Lf = P->L[k + 1];
      k_coarsen_add<R><<<dim3(Lf.nU, ncomp), 256, 0, st>>>(Ld, Fall + Foff[k], cs[k], Lf.d_BL, Fall + Foff[k + 1],
                                                          cs[k + 1]);
      LGF_LAUNCH_CHECK("coarsen");
    }
  }
  for (int k = 0; k < K; ++k) {
    const LevelPlan &L = P->L[k];
    const LevelDev Ld = level_dev(P, k, m->h0);
    const LevelDev Lc = k > 0 ? level_dev(P, k - 1, m->h0) : Ld;
    const int nHB = (int)L.HB.size();
    const int32_t *HB = L.d_lists + L.off_HB;
    const size_t bytes = sizeof(R) * (size_t)ncomp * L.BL.size() * B3;
    cudaMemsetAsync(Ucur, 0, bytes, st);
    k_heat_build<R><<<dim3(nHB, ncomp), 256, sizeof(R) * (size_t)interp_sep_values(B), st>>>(
        Ld, L.d_BL, HB, Fall + Foff[k], L.nU, Ucur, cs[k], Lc, Uprev, k > 0 ? cs[k - 1] : 0, k > 0);
    LGF_LAUNCH_CHECK("reconstruction");
    if ((rc = consume(k, Ld, (const R *)Ucur, cs[k]))) return rc;
    ++launches;
    std::swap(Uprev, Ucur);
  }
  return LGF_OK;
}

template <class R>
static int projection_t(lgf_table *t, const lgf_mesh *m_in, const void *r, void *u, void *p_out, int dtype,
                        double alpha, const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  lgf_mesh m = *m_in;
  m.block_role = nullptr;  // every block carries r and receives u
  const int K = m.nlevels;
  std::vector<int> radii(K, 1);  // the reconstructions are read one cell around Omega_k
  Plan *P = nullptr;
  int rc = get_plan(&m, radii.data(), &P);
  if (rc) return rc;
  const int B = P->B;
  const int64_t B3 = (int64_t)B * B * B;
  int64_t total_user = 0;
  for (int k = 0; k < K; ++k) total_user += P->L[k].nU;
  const int64_t ucs = total_user * B3;
  const size_t es = dtype == LGF_F32 ? 4 : 8;
  Workspace *ws = workspace_for(t, st);
  if ((rc = ws->buf[18].reserve(es * (size_t)ucs)) || (rc = ws->buf[19].reserve(es * (size_t)ucs)) ||
      (rc = ws->buf[20].reserve(3 * es * (size_t)ucs)))
    return rc;
  void *d = ws->buf[18].p, *w = ws->buf[20].p;
  void *p = p_out ? p_out : ws->buf[19].p;
  int64_t launches = 0;
  PhaseTimer tm;
  tm.start(o.timing != 0, st);
  // 1. D^r on Omega_k from P_k r^
  rc = reconstruct_levels<R>(P, &m, 3, r, dtype, ws, launches, st,
                             [&](int k, const LevelDev &Ld, const R *T, int64_t cs) {
                               const LevelPlan &L = P->L[k];
                               k_proj_div<R><<<L.nU, 256, 0, st>>>(Ld, L.d_BL, T, cs, d, dtype, L.user_off);
                               cudaError_t e = cudaGetLastError();
                               return e == cudaSuccess ? LGF_OK
                                                       : set_error(LGF_E_CUDA, "divergence launch: %s",
                                                                   cudaGetErrorString(e));
                             });
  if (rc) return rc;
  tm.mark(PH_CORRECT);
  // 2. L_C p = D^r (FLGF-AMR)
  lgf_solve_opts so = o;
  so.timing = 0;
  so.residual = 0;
  lgf_report srep{};
  if ((rc = solve_poisson(t, &m, 1, d, p, dtype, so, &srep, st))) return rc;
  launches += srep.kernel_launches;
  tm.mark(PH_MAC);
  // 3. w^ = r^ - G P_k p^ on Omega_k
  rc = reconstruct_levels<R>(P, &m, 1, p, dtype, ws, launches, st,
                             [&](int k, const LevelDev &Ld, const R *T, int64_t cs) {
                               const LevelPlan &L = P->L[k];
                               k_proj_grad<R><<<dim3(L.nU, 3), 256, 0, st>>>(Ld, L.d_BL, T, cs, r, w, dtype, ucs,
                                                                            L.user_off);
                               cudaError_t e = cudaGetLastError();
                               return e == cudaSuccess ? LGF_OK
                                                       : set_error(LGF_E_CUDA, "gradient launch: %s",
                                                                   cudaGetErrorString(e));
                             });
  if (rc) return rc;
  tm.mark(PH_INTERP);
  // 4. u^ = FIF-AMR(w^)
  lgf_report hrep{};
  if ((rc = solve_heat(t, &m, 3, w, u, dtype, alpha, so, &hrep, st))) return rc;
  launches += hrep.kernel_launches;
  tm.mark(PH_HEAT);
  tm.finish(rep);
  if (rep) {
    rep->target_cells = hrep.target_cells;
    rep->kernel_launches = launches;
    rep->source_blocks = srep.source_blocks;
    rep->target_blocks = srep.target_blocks;
    rep->mac_mode_used = srep.mac_mode_used;
    rep->scratch_bytes = (int64_t)ws->total() + (int64_t)P->device_bytes;
    rep->alg_bytes = srep.alg_bytes;
    rep->alg_flops = srep.alg_flops;
  }
  if (o.timing) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(LGF_E_CUDA, "projection failed: %s", cudaGetErrorString(e));
  }
  return LGF_OK;
}

int solve_projection(lgf_table *t, const lgf_mesh *m, const void *r, void *u, void *p, int dtype, double alpha,
                     const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  switch (o.precision) {
    case LGF_PREC_FP64: return projection_t<double>(t, m, r, u, p, dtype, alpha, o, rep, st);
    case LGF_PREC_FP32: return projection_t<float>(t, m, r, u, p, dtype, alpha, o, rep, st);
    default: return projection_t<df>(t, m, r, u, p, dtype, alpha, o, rep, st);
  }
}

int solve_heat(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *g, int dtype, double alpha,
               const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st) {
  if (o.precision == LGF_PREC_FP32) return heat_t<float>(t, m, ncomp, f, g, dtype, alpha, o, rep, st);
  if (o.precision == LGF_PREC_DF32) return heat_t<df>(t, m, ncomp, f, g, dtype, alpha, o, rep, st);
  return heat_t<double>(t, m, ncomp, f, g, dtype, alpha, o, rep, st);
}

}  // namespace lgf
