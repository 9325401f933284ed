// box_ops.cuh -- host launch sequence of one block-index-FFT convolution (instantiated per arithmetic).
#pragma once
#include <algorithm>
#include <type_traits>
#include <vector>

#include "box.cuh"
#include "box_fft.cuh"
#include "box_tc.cuh"
#include "internal.h"

namespace lgf {

template <class R>
inline const R *spec_of(const BoxSpec *S);
template <>
inline const double *spec_of<double>(const BoxSpec *S) { return S->g64; }
template <>
inline const float *spec_of<float>(const BoxSpec *S) { return S->g32; }
template <>
inline const df *spec_of<df>(const BoxSpec *S) { return S->gdf; }

template <class R>
inline const cx<R> *twl_of(const BoxSpec *S);
template <>
inline const cx<double> *twl_of<double>(const BoxSpec *S) { return S->twl64; }
template <>
inline const cx<float> *twl_of<float>(const BoxSpec *S) { return S->twl32; }
template <>
inline const cx<df> *twl_of<df>(const BoxSpec *S) { return S->twldf; }

inline void btw_fill(BoxTw<double> &t, const BoxSpec *S, int a) {
  for (int i = 0; i < 2 * BOX_NB_MAX; ++i) t.w[i] = S->bw64[a][i];
}
inline void btw_fill(BoxTw<float> &t, const BoxSpec *S, int a) {
  for (int i = 0; i < 2 * BOX_NB_MAX; ++i) t.w[i] = S->bw32[a][i];
}
inline void btw_fill(BoxTw<df> &t, const BoxSpec *S, int a) {
  for (int i = 0; i < 2 * BOX_NB_MAX; ++i) t.w[i] = S->bwdf[a][i];
}
template <class R>
inline BoxTw<R> btw_of(const BoxSpec *S, int a) {
  BoxTw<R> t;
  btw_fill(t, S, a);
  return t;
}

template <class R>
struct BoxOps {
  // Convolutions of `nf` complex fields on the box: forward (gathering through in[f].s[0..nin[f])),
  // kernel, inverse (scattering through ore[f] / oim[f]).  A field whose input is real (one spec, real
  // part) and whose imaginary output is unused runs on the Hermitian half K1x <= Px/2.  Y0/Y1 hold
  // min(nf, BOX_MAXF) * P^3 B^3 complex R each.  `mark(phase)` is called after the forward, kernel and
  // inverse stages of every group of fields (phase timing; may be null).  `slices` > 0 runs the six
  // block-index DFT passes as tensor-core GEMMs with that many BF16 digit slices (float: 1-3,
  // double-float: 4-6); a bounded wait that gives up there sets *status.
  static int convolve(int B, const BoxSpec *S, int nf, const int *nin, const InSpec3 *in,
                      const OutSpec<R> *ore, const OutSpec<R> *oim, double scale, cx<R> *Y0, cx<R> *Y1,
                      cudaStream_t st, void (*mark)(void *, int) = nullptr, void *mark_ctx = nullptr,
                      int slices = 0, int *status = nullptr, int64_t *launches = nullptr);
};

// Launch of one tensor-core pass: persistent CTAs of 128 threads, as many per SM as registers, shared
// memory and the SM's 512 TMEM columns allow (shared memory is padded when TMEM is the limit, so that no
// tcgen05.alloc has to wait for a neighbour).
template <class R, int B, int SL>
static void tc_pass_launch(const cx<R> *in, cx<R> *out, int64_t fstride, const BoxGeom &g, int ax, int3 ext,
                           const TcMat &M, int gather, int final, int nfield, int lines, const FwdSpecs &sp,
                           const InvOuts<R> &outs, double sc, int *status, cudaStream_t st) {
  static int nsm = 0;
  static bool attr = false;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  if (!attr) {
    cudaFuncSetAttribute(k_bdft_tc<R, B, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  const TcSmem pl = tc_smem_plan(SL, M.Kp, M.Np);
  uint32_t cols = 32;
  while (cols < (uint32_t)(SL * M.Np)) cols <<= 1;
  const int cap = 512 / (int)cols;
  // residency from registers and shared memory; pad shared memory when TMEM would be over-subscribed
  static int regs = 0;
  if (!regs) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k_bdft_tc<R, B, SL>);
    regs = std::max(fa.numRegs, 1);
  }
  constexpr int SM_BYTES = 228 * 1024, CTA_RESERVED = 1024, SM_REGS = 65536;
  int req = pl.total;
  int fit = std::min(SM_REGS / (((regs + 7) / 8 * 8) * TC_ROWS), SM_BYTES / (req + CTA_RESERVED));
  if (fit > cap) {
    req = std::max(req, SM_BYTES / (cap + 1) - CTA_RESERVED + 16);
    fit = cap;
  }
  const int ntiles = nfield * lines * (B * B * B / TC_ROWS);
  const int grid = std::min(ntiles, nsm * std::max(fit, 1));
  k_bdft_tc<R, B, SL><<<grid, TC_ROWS, req, st>>>(in, out, fstride, g, ax, ext, M, gather, final, nfield, lines,
                                                  sp, outs, sc, cols, pl, status);
}

template <class R, int B>
static int tc_pass(int slices, const cx<R> *in, cx<R> *out, int64_t fstride, const BoxGeom &g, int ax, int3 ext,
                   const TcMat &M, int gather, int final, int nfield, int lines, const FwdSpecs &sp,
                   const InvOuts<R> &outs, double sc, int *status, cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value) {
    switch (slices) {
      case 1: tc_pass_launch<R, B, 1>(in, out, fstride, g, ax, ext, M, gather, final, nfield, lines, sp, outs, sc, status, st); return LGF_OK;
      case 2: tc_pass_launch<R, B, 2>(in, out, fstride, g, ax, ext, M, gather, final, nfield, lines, sp, outs, sc, status, st); return LGF_OK;
      case 3: tc_pass_launch<R, B, 3>(in, out, fstride, g, ax, ext, M, gather, final, nfield, lines, sp, outs, sc, status, st); return LGF_OK;
    }
  } else if constexpr (std::is_same<R, df>::value) {
    switch (slices) {
      case 4: tc_pass_launch<R, B, 4>(in, out, fstride, g, ax, ext, M, gather, final, nfield, lines, sp, outs, sc, status, st); return LGF_OK;
      case 5: tc_pass_launch<R, B, 5>(in, out, fstride, g, ax, ext, M, gather, final, nfield, lines, sp, outs, sc, status, st); return LGF_OK;
      case 6: tc_pass_launch<R, B, 6>(in, out, fstride, g, ax, ext, M, gather, final, nfield, lines, sp, outs, sc, status, st); return LGF_OK;
    }
  }
  return set_error(LGF_E_INVALID_ARG, "%d DFT-GEMM slices are not available for this precision", slices);
}

// Launch of the FFT passes for a block count 4..16; false for any other count.  The gathering first forward
// pass keeps its gathered inputs in shared memory (NB x NT values) for the odd half.
template <class R, int B, int NT>
static bool bfft_fwd(int nb, const cx<R> *in, cx<R> *out, int64_t fstride, const BoxGeom &g, int ax, int3 ext,
                     const BoxTw<R> &tw, int gather, int n, int lines, const FwdSpecs &sp, cudaStream_t st) {
  const dim3 grid(B * B * B / NT, lines, n);
  switch (nb) {
    case 4: k_bfft_fwd<R, B, NT, 4><<<grid, NT, gather ? 4 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 5: k_bfft_fwd<R, B, NT, 5><<<grid, NT, gather ? 5 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 6: k_bfft_fwd<R, B, NT, 6><<<grid, NT, gather ? 6 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 7: k_bfft_fwd<R, B, NT, 7><<<grid, NT, gather ? 7 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 8: k_bfft_fwd<R, B, NT, 8><<<grid, NT, gather ? 8 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 9: k_bfft_fwd<R, B, NT, 9><<<grid, NT, gather ? 9 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 10: k_bfft_fwd<R, B, NT, 10><<<grid, NT, gather ? 10 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 11: k_bfft_fwd<R, B, NT, 11><<<grid, NT, gather ? 11 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 12: k_bfft_fwd<R, B, NT, 12><<<grid, NT, gather ? 12 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 13: k_bfft_fwd<R, B, NT, 13><<<grid, NT, gather ? 13 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 14: k_bfft_fwd<R, B, NT, 14><<<grid, NT, gather ? 14 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 15: k_bfft_fwd<R, B, NT, 15><<<grid, NT, gather ? 15 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    case 16: k_bfft_fwd<R, B, NT, 16><<<grid, NT, gather ? 16 * NT * sizeof(cx<R>) : 0, st>>>(in, out, fstride, g, ax, ext, tw, gather, sp); return true;
    default: return false;
  }
}
template <class R, int B, int NT>
static bool bfft_inv(int nb, const cx<R> *in, cx<R> *out, int64_t fstride, const BoxGeom &g, int ax, int3 ext,
                     const BoxTw<R> &tw, int final, int n, int lines, const InvOuts<R> &outs, double sc,
                     cudaStream_t st) {
  const dim3 grid(B * B * B / NT, lines, n);
  switch (nb) {
    case 4: k_bfft_inv<R, B, NT, 4><<<grid, NT, 4 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 5: k_bfft_inv<R, B, NT, 5><<<grid, NT, 5 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 6: k_bfft_inv<R, B, NT, 6><<<grid, NT, 6 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 7: k_bfft_inv<R, B, NT, 7><<<grid, NT, 7 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 8: k_bfft_inv<R, B, NT, 8><<<grid, NT, 8 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 9: k_bfft_inv<R, B, NT, 9><<<grid, NT, 9 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 10: k_bfft_inv<R, B, NT, 10><<<grid, NT, 10 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 11: k_bfft_inv<R, B, NT, 11><<<grid, NT, 11 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 12: k_bfft_inv<R, B, NT, 12><<<grid, NT, 12 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 13: k_bfft_inv<R, B, NT, 13><<<grid, NT, 13 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 14: k_bfft_inv<R, B, NT, 14><<<grid, NT, 14 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 15: k_bfft_inv<R, B, NT, 15><<<grid, NT, 15 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    case 16: k_bfft_inv<R, B, NT, 16><<<grid, NT, 16 * NT * sizeof(cx<R>), st>>>(in, out, fstride, g, ax, ext, tw, final, outs, sc); return true;
    default: return false;
  }
}

template <class R, int B>
static int box_group(const BoxSpec *S, const std::vector<int> &fields, int nc, const int *nin,
                     const InSpec3 *in, const OutSpec<R> *ore, const OutSpec<R> *oim, double scale, cx<R> *Y0,
                     cx<R> *Y1, cudaStream_t st, void (*mark)(void *, int), void *mark_ctx, int slices,
                     int *status) {
  constexpr int B3 = B * B * B;
  BoxGeom g;
  for (int a = 0; a < 3; ++a) {
    g.nb[a] = S->nb[a];
    g.P[a] = 2 * S->nb[a];
  }
  g.bs[0] = 1;
  g.bs[1] = g.P[0];
  g.bs[2] = (int64_t)g.P[0] * g.P[1];
  g.nc = nc;
  const int *nb = g.nb, *P = g.P;
  const int64_t fstride = (int64_t)P[0] * P[1] * P[2] * B3;
  const int pxu = box_pxmax(g);  // lines of the y and z passes run over the widest K1x range
  const int64_t nmid = (int64_t)pxu * P[1] * P[2];
  const size_t sm = sizeof(cx<R>) * (size_t)B * B * (B + 1);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_box_mid<R, B, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  const int n = (int)fields.size();
  FwdSpecs sp{};
  InvOuts<R> outs{};
  for (int f = 0; f < n; ++f) {
    const int fi = fields[f];
    sp.n[f] = nin[fi];
    for (int i = 0; i < sp.n[f] && i < 3; ++i) sp.s[f][i] = in[fi].s[i];
    outs.re[f] = ore[fi];
    outs.im[f] = oim[fi];
  }
  int rc = LGF_OK;
  auto pass = [&](const cx<R> *in_, cx<R> *out_, int ax, int3 ext, int lines, int inverse, int gather, int final,
                  double sc) {
    const int nb_ax = nb[ax];
    const int nout = inverse ? nb_ax : 2 * nb_ax;
    if (slices > 0) {  // tensor-core passes: one kind of field per launch (nc = 0 or n)
      const bool realx = ax == 0 && nc == 0 && pxu < P[0];
      TcMat M = S->tcm[ax][inverse ? (realx ? 2 : 1) : 0];
      if (realx && !inverse) {  // the first pxu outputs of the forward matrix
        M.nout = pxu;
        M.Np = (2 * pxu + 15) / 16 * 16;
      }
      const int r = tc_pass<R, B>(slices, in_, out_, fstride, g, ax, ext, M, gather, final, n, lines, sp, outs, sc,
                                  status, st);
      if (r && !rc) rc = r;
      return;
    }
    // one cell per thread: more resident warps to cover the loads (the passes are latency-bound)
    // 2 <= nb <= 8: compile-time block counts, one chunk in both directions (nb 7 and 8 with chunks of
    // nb - 1 pair slots and nb outputs); wider boxes: runtime counts, chunks of CHF / CHI
    constexpr int NT = 128, CHF = 5, CHI = 6, REP = 1;
    static_assert(CHF + 1 >= 6 && CHI >= 6, "the nb <= 6 specialisations share the one-chunk sizes CHF, CHI");
    if (!inverse) {
      auto go = [&](auto kern, int nch) {
        kern<<<dim3(B3 / (NT * REP), lines, n * nch), NT, 0, st>>>(in_, out_, fstride, g, ax, ext, btw_of<R>(S, ax),
                                                                   gather, nch, sp);
      };
      if constexpr (B == 16) {  // 4..16 blocks: in-register mixed-radix FFTs (box_fft.cuh)
        if (nb_ax >= 4 && bfft_fwd<R, B, NT>(nb_ax, in_, out_, fstride, g, ax, ext, btw_of<R>(S, ax), gather, n, lines,
                                             sp, st))
          return;
      }
      switch (nb_ax) {
        case 2: go(k_bdft_fwd<R, B, CHF, NT, REP, 2>, 1); break;
        case 3: go(k_bdft_fwd<R, B, CHF, NT, REP, 3>, 1); break;
        case 4: go(k_bdft_fwd<R, B, CHF, NT, REP, 4>, 1); break;
        case 5: go(k_bdft_fwd<R, B, CHF, NT, REP, 5>, 1); break;
        case 6: go(k_bdft_fwd<R, B, CHF, NT, REP, 6>, 1); break;
        case 7: go(k_bdft_fwd<R, B, 6, NT, REP, 7>, 1); break;
        case 8: go(k_bdft_fwd<R, B, 7, NT, REP, 8>, 1); break;
        default:
          if constexpr (B == 16) {  // wide boxes: in-register mixed-radix FFTs (box_fft.cuh)
            if (bfft_fwd<R, B, NT>(nb_ax, in_, out_, fstride, g, ax, ext, btw_of<R>(S, ax), gather, n, lines, sp, st))
              break;
          }
          go(k_bdft_fwd<R, B, CHF, NT, REP, 0>, std::max(1, (nb_ax - 1 + CHF - 1) / CHF));
      }
    } else {
      auto go = [&](auto kern, int nch) {
        kern<<<dim3(B3 / (NT * REP), lines, n * nch), NT, 0, st>>>(in_, out_, fstride, g, ax, ext, btw_of<R>(S, ax),
                                                                   final, nch, outs, sc);
      };
      if constexpr (B == 16) {
        if (nb_ax >= 4 && bfft_inv<R, B, NT>(nb_ax, in_, out_, fstride, g, ax, ext, btw_of<R>(S, ax), final, n, lines,
                                             outs, sc, st))
          return;
      }
      switch (nb_ax) {
        case 2: go(k_bdft_inv<R, B, CHI, NT, REP, 2>, 1); break;
        case 3: go(k_bdft_inv<R, B, CHI, NT, REP, 3>, 1); break;
        case 4: go(k_bdft_inv<R, B, CHI, NT, REP, 4>, 1); break;
        case 5: go(k_bdft_inv<R, B, CHI, NT, REP, 5>, 1); break;
        case 6: go(k_bdft_inv<R, B, CHI, NT, REP, 6>, 1); break;
        case 7: go(k_bdft_inv<R, B, 7, NT, REP, 7>, 1); break;
        case 8: go(k_bdft_inv<R, B, 8, NT, REP, 8>, 1); break;
        default:
          if constexpr (B == 16) {
            if (bfft_inv<R, B, NT>(nb_ax, in_, out_, fstride, g, ax, ext, btw_of<R>(S, ax), final, n, lines, outs,
                                   sc, st))
              break;
          }
          go(k_bdft_inv<R, B, CHI, NT, REP, 0>, (nout + CHI - 1) / CHI);
      }
    }
  };
  // forward x (gather), y, z; kernel; inverse z, y, x (scatter)
  pass(nullptr, Y0, 0, make_int3(0, nb[1], nb[2]), nb[1] * nb[2], 0, 1, 0, 1.0);
  pass(Y0, Y1, 1, make_int3(pxu, 0, nb[2]), pxu * nb[2], 0, 0, 0, 1.0);
  pass(Y1, Y0, 2, make_int3(pxu, P[1], 0), pxu * P[1], 0, 0, 0, 1.0);
  if (mark) mark(mark_ctx, 2);
  k_box_mid<R, B, true><<<dim3((unsigned)nmid, n), mid_threads<R, B>(), sm, st>>>(
      Y0, fstride, spec_of<R>(S), g, twl_of<R>(S), S->twL, make_int3(S->twf[0], S->twf[1], S->twf[2]),
      make_tw64<R>(), nullptr);
  if (mark) mark(mark_ctx, 3);
  pass(Y0, Y1, 2, make_int3(pxu, P[1], 0), pxu * P[1], 1, 0, 0, 1.0);
  pass(Y1, Y0, 1, make_int3(pxu, 0, nb[2]), pxu * nb[2], 1, 0, 0, 1.0);
  pass(Y0, Y1, 0, make_int3(0, nb[1], nb[2]), nb[1] * nb[2], 1, 0, 1, scale);
  if (mark) mark(mark_ctx, 4);
  return rc;
}

template <class R, int B>
static int box_convolve_b(const BoxSpec *S, int nf, const int *nin, const InSpec3 *in, const OutSpec<R> *ore,
                          const OutSpec<R> *oim, double scale, cx<R> *Y0, cx<R> *Y1, cudaStream_t st,
                          void (*mark)(void *, int), void *mark_ctx, int slices, int *status, int64_t *launches) {
  std::vector<int> cplx, real;
  for (int f = 0; f < nf; ++f) {
    const bool is_real = nin[f] == 1 && in[f].s[0].part == 0 && oim[f].scatter == nullptr;
    (is_real ? real : cplx).push_back(f);
  }
  // CUDA-core passes take complex and real fields in one launch per stage (complex first); the
  // tensor-core passes keep the two kinds apart (their coefficient matrices differ)
  std::vector<std::vector<int>> lists;
  if (slices > 0) {
    lists = {cplx, real};
  } else {
    lists.push_back(cplx);
    lists[0].insert(lists[0].end(), real.begin(), real.end());
  }
  for (const std::vector<int> &lst : lists) {
    for (size_t f0 = 0; f0 < lst.size(); f0 += BOX_MAXF) {
      std::vector<int> grp(lst.begin() + f0, lst.begin() + std::min(lst.size(), f0 + BOX_MAXF));
      int nc = 0;
      for (int f : grp) nc += std::find(cplx.begin(), cplx.end(), f) != cplx.end();
      int rc = box_group<R, B>(S, grp, nc, nin, in, ore, oim, scale, Y0, Y1, st, mark, mark_ctx, slices, status);
      if (rc) return rc;
      if (launches) *launches += 7;
    }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "box convolution launch: %s", cudaGetErrorString(e));
}

template <class R>
int BoxOps<R>::convolve(int B, const BoxSpec *S, int nf, const int *nin, const InSpec3 *in,
                        const OutSpec<R> *ore, const OutSpec<R> *oim, double scale, cx<R> *Y0, cx<R> *Y1,
                        cudaStream_t st, void (*mark)(void *, int), void *mark_ctx, int slices, int *status,
                        int64_t *launches) {
  if (slices > 0 && (std::is_same<R, double>::value || !status))
    return set_error(LGF_E_UNSUPPORTED, "the tensor-core DFT-GEMM runs in FP32 or double-float only");
  if (B == 8)
    return box_convolve_b<R, 8>(S, nf, nin, in, ore, oim, scale, Y0, Y1, st, mark, mark_ctx, slices, status,
                                launches);
  if (B == 16)
    return box_convolve_b<R, 16>(S, nf, nin, in, ore, oim, scale, Y0, Y1, st, mark, mark_ctx, slices, status,
                                 launches);
  return set_error(LGF_E_UNSUPPORTED, "block size %d", B);
}

}  // namespace lgf
