// box_ops.cuh -- host launch sequence of one block-index-FFT convolution (instantiated per arithmetic).
#pragma once
#include <type_traits>
#include <vector>

#include "box.cuh"
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
inline const cx<R> *tw_of(const BoxSpec *S, int a);
template <>
inline const cx<double> *tw_of<double>(const BoxSpec *S, int a) { return S->tw64[a]; }
template <>
inline const cx<float> *tw_of<float>(const BoxSpec *S, int a) { return S->tw32[a]; }
template <>
inline const cx<df> *tw_of<df>(const BoxSpec *S, int a) { return S->twdf[a]; }

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
  // inverse stages of every group of fields (phase timing; may be null).
  static int convolve(int B, const BoxSpec *S, int nf, const int *nin, const InSpec3 *in,
                      const OutSpec<R> *ore, const OutSpec<R> *oim, double scale, cx<R> *Y0, cx<R> *Y1,
                      cudaStream_t st, void (*mark)(void *, int) = nullptr, void *mark_ctx = nullptr);
};

template <class R, int B>
static int box_group(const BoxSpec *S, const std::vector<int> &fields, bool real, const int *nin,
                     const InSpec3 *in, const OutSpec<R> *ore, const OutSpec<R> *oim, double scale, cx<R> *Y0,
                     cx<R> *Y1, cudaStream_t st, void (*mark)(void *, int), void *mark_ctx) {
  constexpr int B3 = B * B * B;
  BoxGeom g;
  for (int a = 0; a < 3; ++a) {
    g.nb[a] = S->nb[a];
    g.P[a] = 2 * S->nb[a];
  }
  g.bs[0] = 1;
  g.bs[1] = g.P[0];
  g.bs[2] = (int64_t)g.P[0] * g.P[1];
  g.pxu = real ? g.P[0] / 2 + 1 : g.P[0];
  const int *nb = g.nb, *P = g.P;
  const int64_t fstride = (int64_t)P[0] * P[1] * P[2] * B3;
  const int64_t nmid = (int64_t)g.pxu * P[1] * P[2];
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
  auto pass = [&](const cx<R> *in_, cx<R> *out_, int ax, int3 ext, int lines, int inverse, int gather, int final,
                  double sc) {
    const int nb_ax = nb[ax];
    const bool realx = ax == 0 && g.pxu < P[0];
    const int nout = inverse ? nb_ax : (realx ? g.pxu : 2 * nb_ax);
    if (nout <= 8) {
      k_bdft<R, B, 8, 2><<<dim3((B3 + 511) / 512, lines, n), 256, 0, st>>>(
          in_, out_, fstride, g, ax, ext, btw_of<R>(S, ax), inverse, gather, final, 1, sp, outs, sc);
    } else {
      const int nch = (nout + 7) / 8;
      k_bdft<R, B, 8, 1><<<dim3((B3 + 255) / 256, lines, n * nch), 256, 0, st>>>(
          in_, out_, fstride, g, ax, ext, btw_of<R>(S, ax), inverse, gather, final, nch, sp, outs, sc);
    }
  };
  const int pxu = g.pxu;
  // forward x (gather), y, z; kernel; inverse z, y, x (scatter)
  pass(nullptr, Y0, 0, make_int3(0, nb[1], nb[2]), nb[1] * nb[2], 0, 1, 0, 1.0);
  pass(Y0, Y1, 1, make_int3(pxu, 0, nb[2]), pxu * nb[2], 0, 0, 0, 1.0);
  pass(Y1, Y0, 2, make_int3(pxu, P[1], 0), pxu * P[1], 0, 0, 0, 1.0);
  if (mark) mark(mark_ctx, 2);
  k_box_mid<R, B, true><<<dim3((unsigned)nmid, n), 256, sm, st>>>(Y0, fstride, spec_of<R>(S), g, tw_of<R>(S, 0),
                                                                 tw_of<R>(S, 1), tw_of<R>(S, 2), make_tw64<R>(),
                                                                 nullptr);
  if (mark) mark(mark_ctx, 3);
  pass(Y0, Y1, 2, make_int3(pxu, P[1], 0), pxu * P[1], 1, 0, 0, 1.0);
  pass(Y1, Y0, 1, make_int3(pxu, 0, nb[2]), pxu * nb[2], 1, 0, 0, 1.0);
  pass(Y0, Y1, 0, make_int3(0, nb[1], nb[2]), nb[1] * nb[2], 1, 0, 1, scale);
  if (mark) mark(mark_ctx, 4);
  return LGF_OK;
}

template <class R, int B>
static int box_convolve_b(const BoxSpec *S, int nf, const int *nin, const InSpec3 *in, const OutSpec<R> *ore,
                          const OutSpec<R> *oim, double scale, cx<R> *Y0, cx<R> *Y1, cudaStream_t st,
                          void (*mark)(void *, int), void *mark_ctx) {
  std::vector<int> cplx, real;
  for (int f = 0; f < nf; ++f) {
    const bool is_real = nin[f] == 1 && in[f].s[0].part == 0 && oim[f].scatter == nullptr;
    (is_real ? real : cplx).push_back(f);
  }
  for (int pass = 0; pass < 2; ++pass) {
    const std::vector<int> &lst = pass ? real : cplx;
    for (size_t f0 = 0; f0 < lst.size(); f0 += BOX_MAXF) {
      std::vector<int> grp(lst.begin() + f0, lst.begin() + std::min(lst.size(), f0 + BOX_MAXF));
      int rc = box_group<R, B>(S, grp, pass == 1, nin, in, ore, oim, scale, Y0, Y1, st, mark, mark_ctx);
      if (rc) return rc;
    }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "box convolution launch: %s", cudaGetErrorString(e));
}

template <class R>
int BoxOps<R>::convolve(int B, const BoxSpec *S, int nf, const int *nin, const InSpec3 *in,
                        const OutSpec<R> *ore, const OutSpec<R> *oim, double scale, cx<R> *Y0, cx<R> *Y1,
                        cudaStream_t st, void (*mark)(void *, int), void *mark_ctx) {
  if (B == 8) return box_convolve_b<R, 8>(S, nf, nin, in, ore, oim, scale, Y0, Y1, st, mark, mark_ctx);
  if (B == 16) return box_convolve_b<R, 16>(S, nf, nin, in, ore, oim, scale, Y0, Y1, st, mark, mark_ctx);
  return set_error(LGF_E_UNSUPPORTED, "block size %d", B);
}

}  // namespace lgf
