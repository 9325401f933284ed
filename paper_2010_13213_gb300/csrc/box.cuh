// box.cuh -- block-index FFT mode: the per-frequency sum over block pairs diagonalised by a
// zero-padded DFT over the level's block grid (exact reformulation of the lattice convolution,
// Sec. 2.2 Eq. (eq:lgf_convolution)).
//
// A level box of nb = (nbx, nby, nbz) blocks of B^3 cells is embedded in a periodic lattice of
// P = 2 nb blocks per axis (Pc = P B cells), large enough that the circular convolution with the
// circularly laid out LGF equals the linear one on the box.  Writing a cell index n = B J + m (block J,
// local cell m) and a frequency K = K1 + P K2 (K1 in [0, P), K2 in [0, B)) per axis, the Pc-point DFT
// factors as ("four-step"):
//     Y[K1][m]  = sum_J x[J][m] W_P^{J.K1}                  block-index DFT   (k_bdft_fwd, per axis)
//     Y'        = Y W_Pc^{m.K1}                              twiddle          (k_box_mid)
//     X[K1][K2] = sum_m Y'[K1][m] W_B^{m.K2}                 local B^3 FFT     (k_box_mid)
// The convolution multiplies X by the (real, since G is even) spectrum Ghat[K1][K2] and runs the three
// steps backwards; the inverse block-index DFT is evaluated only on the box's blocks.  Inputs are
// complex: two real fields ride as real and imaginary part (G is real).
//
// The block-index DFTs have P = 2 nb points of which only nb inputs (forward) or outputs (inverse)
// are used; they are evaluated directly by conjugate pairs (real coefficients cos, sin of 2 pi j k / P),
// a CTA taking a chunk of pair slots (forward) or outputs (inverse); for nb <= 8 the block count is a
// compile-time constant and one chunk covers the line.
#pragma once
#include "common.cuh"

#define BOX_NB_MAX 16

template <class R>
struct BoxTw {  // W_P^n = e^{-2 pi i n / P}, n < P = 2 nb of the pass's axis
  cx<R> w[2 * BOX_NB_MAX];
};

// Layout of a box array: [bz][by][bx][B^3] with full extents (Px, Py, Pz) blocks.
struct BoxGeom {
  int nb[3];    // box blocks per axis
  int P[3];     // 2 nb
  int64_t bs[3];  // block strides (in blocks) of the full P-array: 1, Px, Px*Py
  int nc;       // fields [0, nc) of a launch are complex (K1x < Px); the others are real fields kept on
                // the Hermitian half K1x <= Px/2
};
// Per-axis members picked by selects: indexing a kernel parameter's array with a runtime axis would copy
// the whole struct to local memory.
LGF_HD int geo_nb(const BoxGeom &g, int a) { return a == 0 ? g.nb[0] : (a == 1 ? g.nb[1] : g.nb[2]); }
LGF_HD int geo_P(const BoxGeom &g, int a) { return a == 0 ? g.P[0] : (a == 1 ? g.P[1] : g.P[2]); }
LGF_HD int64_t geo_bs(const BoxGeom &g, int a) { return a == 0 ? g.bs[0] : (a == 1 ? g.bs[1] : g.bs[2]); }
// Block frequencies K1x a field keeps, and the most any field of the launch keeps.
LGF_HD int box_pxu(const BoxGeom &g, int field) { return field < g.nc ? g.P[0] : g.P[0] / 2 + 1; }
LGF_HD int box_pxmax(const BoxGeom &g) { return g.nc > 0 ? g.P[0] : g.P[0] / 2 + 1; }

// Source of the first forward pass: box block -> buffer block (gather, -1 = absent), a field
// (dtype per load_field, the component already applied to the pointer) and an optional cell mask.
// Each spec adds into the real (part 0) or the imaginary (part 1) part of the complex input.
struct InSpec {
  const int32_t *gather;
  const void *src;
  const uint8_t *mask;
  int dtype, bits, part;
};
// Destination of the last inverse pass for the real (re) or imaginary (im) part: box block ->
// output block (scatter, -1 = skip), output field (component applied) with element offset, the
// internal-R addend and mask indexed by aux (or by the output block when aux is null).
template <class R>
struct OutSpec {
  const int32_t *scatter;
  const int32_t *aux;
  void *dst;
  const R *add;
  const uint8_t *mask;
  int64_t off;
  int dtype, bits;
};

#define BOX_MAXF 4  // complex fields per launch

struct InSpec3 {  // the input specs of one complex field
  InSpec s[3];
};

struct FwdSpecs {   // per field: up to three input specs (first forward pass only)
  InSpec s[BOX_MAXF][3];
  int n[BOX_MAXF];
};

template <class R>
struct InvOuts {  // per field: destinations of the real and imaginary parts (last inverse pass)
  OutSpec<R> re[BOX_MAXF], im[BOX_MAXF];
};

template <class R>
LGF_D void box_store(const OutSpec<R> &o, int bidx, int m, int B3, R v) {
  if (!o.scatter) return;
  const int ob = o.scatter[bidx];
  if (ob < 0) return;
  const int64_t a = (int64_t)(o.aux ? o.aux[bidx] : ob) * B3 + m;
  if (o.add) v = v + o.add[a];
  if (o.mask && !(o.mask[a] & o.bits)) return;
  store_field<R>(o.dst, o.off + (int64_t)ob * B3 + m, o.dtype, v);
}

// The same with the block indices resolved by the caller: ob = scatter[bidx] (-1: skip), ab = the
// addend / mask block (aux[bidx], or ob without aux).
template <class R>
LGF_D void box_store_at(const OutSpec<R> &o, int ob, int ab, int m, int B3, R v) {
  if (ob < 0) return;
  const int64_t a = (int64_t)ab * B3 + m;
  if (o.add) v = v + o.add[a];
  if (o.mask && !(o.mask[a] & o.bits)) return;
  store_field<R>(o.dst, o.off + (int64_t)ob * B3 + m, o.dtype, v);
}

// ------------------------------------------------------------------ block-index DFTs
// Pass along axis `ax` for every line (the two other block coordinates within `ext`) and local cell m:
//   forward  X[.. k ..][m] = sum_{j < nb} W_P^{ j k} x[.. j ..][m],   k < P = 2 nb
//   inverse  y[.. j ..][m] = sum_{k < P}  W_P^{-j k} X[.. k ..][m],   j < nb (unnormalised)
// Both use the conjugate symmetry W_P^{j(P-k)} = conj(W_P^{jk}) (c = cos(2 pi jk/P), s = sin(2 pi jk/P)):
//   forward  A_k = sum_j c x_j, B_k = sum_j s x_j, X_k = A_k - i B_k, X_{P-k} = A_k + i B_k (1 <= k < P/2),
//   inverse  y_j += c (X_k + X_{P-k}) + i s (X_k - X_{P-k}) per input pair,
// so every multiply has a real coefficient: half the work of the complex products.  k = 0 and k = P/2
// (coefficients 1 and (-1)^j) are sums.  A real field keeps K1x in [0, P/2] (Hermitian half): its
// forward x pass stores X_k only and its inverse x pass takes X_{P-k} = conj(X_k) (real output).
// A CTA of NT threads owns REP groups of NT consecutive cells (taken one after the other) and a chunk of
// CH pair slots (forward) or outputs (inverse); grid = (B^3 / (NT REP), lines, field * nchunk + chunk).  The chunk's (c, s) sit in a shared table;
// the next input is fetched while the current one multiplies.  The first forward pass (gather) reads
// through the field's input specs, the last inverse pass (final) writes through its output specs.
// Field f's arrays start at in + f * fstride, out + f * fstride.
// NBT > 0 fixes nb = NBT at compile time for one-chunk passes (NBT - 1 <= CH forward, NBT <= CH inverse):
// the loops unroll, every coefficient index j q mod P is a constant, and the coefficients are read
// from the parameter table itself (no shared table, no barrier unless the gather/scatter tables need one).
template <class R>
LGF_D cx<R> box_coef(const BoxTw<R> &tw, int n) {  // (cos, sin)(2 pi n / P) from W_P^n
  return cx<R>{tw.w[n].re, -tw.w[n].im};
}

template <class R, int B, int CH, int NT, int REP, int NBT = 0>
__global__ void __launch_bounds__(NT) k_bdft_fwd(const cx<R> *__restrict__ in, cx<R> *__restrict__ out,
                                                 int64_t fstride, BoxGeom g, int ax, int3 ext, BoxTw<R> tw,
                                                 int gather, int nchunk, FwdSpecs sp) {
  constexpr int B3 = B * B * B;
  constexpr bool FIX = NBT > 0;
  __shared__ cx<R> TW[FIX ? 1 : BOX_NB_MAX][CH];  // (cos, sin)(2 pi j q / P) of the chunk's general slots
  const int nb = FIX ? NBT : geo_nb(g, ax), P = 2 * nb, half = nb;
  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
  const int e1 = ax == 0 ? ext.y : ext.x;
  const int l1 = (int)blockIdx.y % e1, l2 = (int)blockIdx.y / e1;
  const int field = FIX ? (int)blockIdx.z : (int)blockIdx.z / nchunk, chunk = FIX ? 0 : (int)blockIdx.z % nchunk;
  const int pxf = box_pxu(g, field);
  if (ax != 0 && l1 >= pxf) return;  // a line beyond this field's K1x range (l1 is K1x for y and z)
  const bool realx = ax == 0 && pxf < P;
  // general slots q = 1 .. half - 1 in chunks of CH; chunk 0 also sums the slots q = 0 and q = half
  const int q0 = 1 + chunk * CH;
  const int nq = FIX ? NBT - 1 : max(0, min(CH, half - q0));
  const bool ends = chunk == 0;
  if (!FIX)
    for (int i = threadIdx.x; i < nb * CH; i += NT) {
      const int j = i / CH, c = i % CH;
      const int n = (j * (q0 + c)) % P;  // < 32 * 32: 32-bit
      TW[j][c] = box_coef(tw, n);
    }
  const int64_t bsa = geo_bs(g, ax) * (int64_t)B3;
  const int64_t lbase = ((int64_t)l1 * geo_bs(g, a1) + (int64_t)l2 * geo_bs(g, a2)) * B3;
  const int gsa = ax == 0 ? 1 : (ax == 1 ? g.nb[0] : g.nb[0] * g.nb[1]);
  const int gbase = l1 * (a1 == 0 ? 1 : g.nb[0]) + l2 * (a2 == 1 ? g.nb[0] : g.nb[0] * g.nb[1]);
  InSpec s0{}, s1{}, s2{};
  int ns = 0;
  if (gather) {
#pragma unroll
    for (int f = 0; f < BOX_MAXF; ++f)
      if (f == field) {
        s0 = sp.s[f][0];
        s1 = sp.s[f][1];
        s2 = sp.s[f][2];
        ns = sp.n[f];
      }
  }
  // the line's source block of every input j and spec (the same for all cells of the CTA)
  __shared__ int GI[3][BOX_NB_MAX];
  if (gather)
    for (int j = threadIdx.x; j < nb; j += NT) {
      const int bidx = gbase + j * gsa;
      GI[0][j] = ns > 0 ? s0.gather[bidx] : -1;
      GI[1][j] = ns > 1 ? s1.gather[bidx] : -1;
      GI[2][j] = ns > 2 ? s2.gather[bidx] : -1;
    }
  const cx<R> *src = in + field * fstride + lbase;
  cx<R> *dst = out + field * fstride + lbase;
  if (!FIX || gather) __syncthreads();
  // REP groups of NT consecutive cells per CTA, one after the other (the table serves them all)
#pragma unroll 1
  for (int rep = 0; rep < REP; ++rep) {
  const int m = (blockIdx.x * REP + rep) * NT + threadIdx.x;
  auto fetch = [&](int j) -> cx<R> {
    if (!gather) return ld_stream(src + j * bsa + m);  // dead after this pass: keep L2 for its output
    R re = RT<R>::zero(), im = RT<R>::zero();
    auto add = [&](const InSpec &q, int si) {
      const int idx = GI[si][j];
      if (idx < 0) return;
      const int64_t e = (int64_t)idx * B3 + m;
      if (q.mask && !(q.mask[e] & q.bits)) return;
      const R v = load_field<R>(q.src, e, q.dtype);
      if (q.part) im = im + v;
      else re = re + v;
    };
    if (ns > 0) add(s0, 0);
    if (ns > 1) add(s1, 1);
    if (ns > 2) add(s2, 2);
    return cx<R>{re, im};
  };
  // j = 0: every coefficient is 1
  cx<R> x = fetch(0);
  cx<R> A[CH], Bv[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    A[k] = x;
    Bv[k] = cx_zero<R>();
  }
  // slots 0 and half (coefficients 1 and (-1)^j) from the sums over even and odd j
  cx<R> Se = x, So = cx_zero<R>();
  auto accumulate = [&](int j, const cx<R> &xj) {
    if (ends) {
      if (j & 1) So = cadd(So, xj);
      else Se = cadd(Se, xj);
    }
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      if (k < nq) {
        const cx<R> w = FIX ? box_coef(tw, (j * (q0 + k)) % P) : TW[FIX ? 0 : j][k];
        A[k] = cx<R>{rfma(A[k].re, w.re, xj.re), rfma(A[k].im, w.re, xj.im)};
        Bv[k] = cx<R>{rfma(Bv[k].re, w.im, xj.re), rfma(Bv[k].im, w.im, xj.im)};
      }
    }
  };
  if constexpr (FIX) {
    cx<R> xs[NBT];
#pragma unroll
    for (int j = 1; j < NBT; ++j) xs[j] = fetch(j);
#pragma unroll
    for (int j = 1; j < NBT; ++j) accumulate(j, xs[j]);
  } else {
    cx<R> xn = nb > 1 ? fetch(1) : cx_zero<R>();
    for (int j = 1; j < nb; ++j) {
      x = xn;
      if (j + 1 < nb) xn = fetch(j + 1);
      accumulate(j, x);
    }
  }
  if (ends) {
    dst[m] = cnorm(cadd(Se, So));
    dst[half * bsa + m] = cnorm(csub(Se, So));
  }
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    if (k < nq) {
      const int q = q0 + k;
      const cx<R> a = A[k], b = Bv[k];
      dst[q * bsa + m] = cx<R>{rnorm(a.re + b.im), rnorm(a.im - b.re)};
      if (!realx) dst[(P - q) * bsa + m] = cx<R>{rnorm(a.re - b.im), rnorm(a.im + b.re)};
    }
  }
  }
}

template <class R, int B, int CH, int NT, int REP, int NBT = 0>
__global__ void __launch_bounds__(NT) k_bdft_inv(const cx<R> *__restrict__ in, cx<R> *__restrict__ out,
                                                 int64_t fstride, BoxGeom g, int ax, int3 ext, BoxTw<R> tw,
                                                 int final, int nchunk, InvOuts<R> outs, double scale) {
  constexpr int B3 = B * B * B;
  constexpr bool FIX = NBT > 0;
  __shared__ cx<R> TW[FIX ? 1 : BOX_NB_MAX][CH];  // (cos, sin)(2 pi q o / P) for the general input slots
  const int nb = FIX ? NBT : geo_nb(g, ax), P = 2 * nb, half = nb;
  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
  const int e1 = ax == 0 ? ext.y : ext.x;
  const int l1 = (int)blockIdx.y % e1, l2 = (int)blockIdx.y / e1;
  const int field = FIX ? (int)blockIdx.z : (int)blockIdx.z / nchunk, chunk = FIX ? 0 : (int)blockIdx.z % nchunk;
  const int pxf = box_pxu(g, field);
  if (ax != 0 && l1 >= pxf) return;  // a line beyond this field's K1x range (l1 is K1x for y and z)
  const bool realx = ax == 0 && pxf < P;
  const int o0 = chunk * CH;
  const int no = FIX ? NBT : min(CH, nb - o0);
  if (!FIX)
    for (int i = threadIdx.x; i < half * CH; i += NT) {
      const int q = i / CH, c = i % CH;
      const int n = (q * (o0 + c)) % P;  // < 32 * 32: 32-bit
      TW[q][c] = box_coef(tw, n);
    }
  const int64_t bsa = geo_bs(g, ax) * (int64_t)B3;
  const int64_t lbase = ((int64_t)l1 * geo_bs(g, a1) + (int64_t)l2 * geo_bs(g, a2)) * B3;
  const int gsa = ax == 0 ? 1 : (ax == 1 ? g.nb[0] : g.nb[0] * g.nb[1]);
  const int gbase = l1 * (a1 == 0 ? 1 : g.nb[0]) + l2 * (a2 == 1 ? g.nb[0] : g.nb[0] * g.nb[1]);
  OutSpec<R> ore{}, oim{};
  if (final) {
#pragma unroll
    for (int f = 0; f < BOX_MAXF; ++f)
      if (f == field) {
        ore = outs.re[f];
        oim = outs.im[f];
      }
  }
  const R sc = RT<R>::from(scale);
  // output blocks of the chunk's outputs (the same for all cells of the CTA): scatter and addend / mask
  __shared__ int SO[2][CH], SX[2][CH];
  if (final && threadIdx.x < CH) {
    const int k = threadIdx.x, bidx = gbase + (o0 + k) * gsa;
    int ob = -1, ab = -1;
    if (k < no && ore.scatter) {
      ob = ore.scatter[bidx];
      ab = ob >= 0 ? (ore.aux ? ore.aux[bidx] : ob) : -1;
    }
    SO[0][k] = ob;
    SX[0][k] = ab;
    ob = ab = -1;
    if (k < no && oim.scatter) {
      ob = oim.scatter[bidx];
      ab = ob >= 0 ? (oim.aux ? oim.aux[bidx] : ob) : -1;
    }
    SO[1][k] = ob;
    SX[1][k] = ab;
  }
  if (!FIX || final) __syncthreads();
  // REP groups of NT consecutive cells per CTA, one after the other (the table serves them all)
#pragma unroll 1
  for (int rep = 0; rep < REP; ++rep) {
  const int m = (blockIdx.x * REP + rep) * NT + threadIdx.x;
  const cx<R> *src = in + field * fstride + lbase + m;
  // general input slot q (1 <= q < half): X_q and X_{P-q}, the latter conj(X_q) for a real field
  // the input is dead after this pass: streaming loads keep L2 for its output
  auto fetch = [&](int q, cx<R> &xa, cx<R> &xb) {
    xa = ld_stream(src + q * bsa);
    xb = realx ? conj(xa) : ld_stream(src + (P - q) * bsa);
  };
  // slots 0 and half: coefficients 1 and (-1)^o
  const cx<R> X0 = ld_stream(src), Xh = ld_stream(src + half * bsa);
  cx<R> y[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) y[k] = ((o0 + k) & 1) ? csub(X0, Xh) : cadd(X0, Xh);
  auto accumulate = [&](int q, const cx<R> &xa, const cx<R> &xb) {
    const cx<R> U = cadd(xa, xb), V = csub(xa, xb);
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      if (k < no) {
        if (o0 + k == 0) {
          y[k] = cadd(y[k], U);
        } else {
          const cx<R> w = FIX ? box_coef(tw, (q * (o0 + k)) % P) : TW[FIX ? 0 : q][k];
          y[k].re = rdot2(y[k].re, w.re, U.re, w.im, V.im, -1.0f);
          if (!realx) y[k].im = rdot2(y[k].im, w.re, U.im, w.im, V.re, 1.0f);
        }
      }
    }
  };
  if constexpr (FIX) {
    cx<R> xa[NBT], xb[NBT];
#pragma unroll
    for (int q = 1; q < NBT; ++q) fetch(q, xa[q], xb[q]);
#pragma unroll
    for (int q = 1; q < NBT; ++q) accumulate(q, xa[q], xb[q]);
  } else {
    cx<R> na = cx_zero<R>(), nbv = cx_zero<R>();
    if (half > 1) fetch(1, na, nbv);
    for (int q = 1; q < half; ++q) {
      const cx<R> xa = na, xb = nbv;
      if (q + 1 < half) fetch(q + 1, na, nbv);
      accumulate(q, xa, xb);
    }
  }
  if (!final) {
    cx<R> *dst = out + field * fstride + lbase + m;
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k < no) dst[(o0 + k) * bsa] = cnorm(y[k]);
    continue;
  }
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    if (k >= no) continue;
    const cx<R> v = cnorm(y[k]);
    box_store_at<R>(ore, SO[0][k], SX[0][k], m, B3, v.re * sc);
    if (!realx) box_store_at<R>(oim, SO[1][k], SX[1][k], m, B3, v.im * sc);
  }
  }
}

// ------------------------------------------------------------------ dense block-index DFT (kernel spectra, FP64)
// out[.. k ..][m] = sum_{j < P} W_P^{j k} in[.. j ..][m] over all P blocks; the first pass reads the
// circularly laid out unit-lattice LGF: cell n (per axis, 0 <= n < Pc) holds G(d), d = n for
// n <= Pc/2 and n - Pc above.
template <int B>
__global__ void __launch_bounds__(256) k_bdft_dense(const cx<double> *__restrict__ in, cx<double> *__restrict__ out,
                                                    BoxGeom g, int ax, const cx<double> *__restrict__ wP,
                                                    const double *__restrict__ Gd, int K) {
  constexpr int B3 = B * B * B;
  const int P = geo_P(g, ax);
  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
  const int e1 = geo_P(g, a1);
  const int64_t line = blockIdx.y;
  const int l1 = (int)(line % e1), l2 = (int)(line / e1);
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= B3) return;
  int coord[3];
  coord[a1] = l1;
  coord[a2] = l2;
  const int mloc[3] = {m % B, (m / B) % B, m / (B * B)};
  auto value = [&](int j) -> cx<double> {
    coord[ax] = j;
    if (Gd) {
      int d[3];
      for (int a = 0; a < 3; ++a) {
        const int Pc = geo_P(g, a) * B, n = coord[a] * B + mloc[a];
        d[a] = n <= Pc / 2 ? n : Pc - n;
      }
      return cx<double>{Gd[((int64_t)d[2] * K + d[1]) * K + d[0]], 0.0};
    }
    return in[((int64_t)coord[0] * g.bs[0] + coord[1] * g.bs[1] + coord[2] * g.bs[2]) * B3 + m];
  };
  for (int k = 0; k < P; ++k) {
    cx<double> acc{0.0, 0.0};
    for (int j = 0; j < P; ++j) acc = acc + value(j) * wP[(j * k) % P];
    coord[ax] = k;
    out[((int64_t)coord[0] * g.bs[0] + coord[1] * g.bs[1] + coord[2] * g.bs[2]) * B3 + m] = acc;
  }
}

// ------------------------------------------------------------------ fused twiddle + local FFT + kernel
// One CTA per (K1 block, field): Y'[m] = Y[m] W_Pc^{m.K1}; X = FFT_B^3(Y'); X *= Ghat; back.  Six
// line-FFT steps over the B^2 lines (l0, l1) of each axis, one thread per line (two for FP32, see
// MidSplit):
//   0  z lines (x, y): global Y, twiddle, FFT_z              -> shared
//   1  y lines (x, z): FFT_y                                 -> shared
//   2  x lines (y, z): FFT_x, X Ghat, conjugate              (registers)
//   3  x lines      : FFT_x                                  -> shared
//   4  y lines      : FFT_y                                  -> shared
//   5  z lines      : FFT_z, conjugate, conjugate twiddle    -> global Y
// (the inverse is conj(FFT(conj(.))), so one FFT body serves every step: small code, no
// instruction-cache stalls).  Four barriers, one shared store and load per cell and step.  Ghat is stored
// per block as [x][z][y] so the x lines of step 2 read it coalesced.  Shared memory: B^3 complex with
// rows padded to B + 1 (every line direction conflict-free).  Without MULTIPLY (kernel-spectrum
// generation) the real part of step 2 goes to `kout` in the same [x][z][y] order.  The per-cell twiddle
// is one load from a table of W_L^n, L = lcm of the three lattice periods, at an integer exponent.
template <int B>
struct MidGeom {
  static constexpr int RS = B + 1;          // padded row
  static constexpr int N = B * B * RS;      // padded elements
};

// Exchange with the lane 16 apart in the warp (the other half of the same line).
LGF_D double shfl16(double v) { return __shfl_xor_sync(0xffffffffu, v, 16); }
LGF_D float shfl16(float v) { return __shfl_xor_sync(0xffffffffu, v, 16); }
LGF_D df shfl16(df v) { return df{__shfl_xor_sync(0xffffffffu, v.hi, 16), __shfl_xor_sync(0xffffffffu, v.lo, 16)}; }
template <class R>
LGF_D cx<R> shfl16(cx<R> v) { return cx<R>{shfl16(v.re), shfl16(v.im)}; }

// Line FFT split over two threads: half h holds the points 2r + h (r < H = B/2) and runs the H-point
// FFT of its half (E: even points, O: odd points); the last radix-2 stage X_k = E_k + W_B^k O_k,
// X_{k+H} = E_k - W_B^k O_k is shared out by k, half h taking k in [hQ, hQ + Q), Q = B/4, after one
// exchange of Q values.  Output slot j of half h then holds X at mid_out_index(B, h, j).
LGF_HD constexpr int mid_out_index(int B, int h, int j) { return h * (B / 4) + j % (B / 4) + (B / 2) * (j / (B / 4)); }

template <class R, int B>
LGF_D void fft_split(cx<R> (&u)[B / 2], int h, const Tw64<R> &tw) {
  constexpr int Q = B / 4;
  fft_reg<R, B / 2, false, false>(u, tw);
#pragma unroll
  for (int r = 0; r < Q; ++r) {
    const cx<R> recv = shfl16(h ? u[r] : u[Q + r]);  // half 0 sends E_{Q+r}, half 1 sends O_r
    const cx<R> E = h ? recv : u[r], O = h ? u[Q + r] : recv;
    cx<R> t;
    if (r == 0) {  // k = 0 (W = 1) or k = B/4 (W = -i, an exact swap)
      t = h ? cx<R>{O.im, -O.re} : O;
    } else {
      const cx<R> w0 = twiddle<R, 64, false>(tw, r * (64 / B)), w1 = twiddle<R, 64, false>(tw, (Q + r) * (64 / B));
      t = cmul(O, h ? w1 : w0);
    }
    u[r] = cadd(E, t);
    u[Q + r] = csub(E, t);
  }
}

// Source of slot r (point 2r + h) of half h when the output of fft_split feeds another split FFT of the
// same line: >= 0, the half's own slot; < 0, -(s + 1) for the s-th value received from the other half,
// which sends its slots 2s + h.
LGF_HD constexpr int mid_regroup_src(int B, int h, int r) {
  const int m = 2 * r + h, H = B / 2, Q = B / 4;
  if ((m % H) / Q == h) return (m % H) % Q + Q * (m / H);
  int src = 0;
  for (int s = 0; s < H / 2; ++s)
    if (mid_out_index(B, 1 - h, 2 * s + h) == m) src = -(s + 1);
  return src;
}

template <class R, int B>
LGF_D void mid_regroup(cx<R> (&u)[B / 2], int h) {
  constexpr int H = B / 2;
  cx<R> recv[H / 2], nu[H];
#pragma unroll
  for (int s = 0; s < H / 2; ++s) recv[s] = shfl16(h ? u[2 * s] : u[2 * s + 1]);
#pragma unroll
  for (int r = 0; r < H; ++r) {
    const int c0 = mid_regroup_src(B, 0, r), c1 = mid_regroup_src(B, 1, r);
    const cx<R> v0 = c0 >= 0 ? u[c0 >= 0 ? c0 : 0] : recv[c0 < 0 ? -c0 - 1 : 0];
    const cx<R> v1 = c1 >= 0 ? u[c1 >= 0 ? c1 : 0] : recv[c1 < 0 ? -c1 - 1 : 0];
    nu[r] = h ? v1 : v0;
  }
#pragma unroll
  for (int r = 0; r < H; ++r) u[r] = nu[r];
}

// Lines per thread of k_box_mid: FP32 splits each line over two threads (half the registers per thread,
// twice the resident warps, one exchange per FFT); double-float and FP64 keep a whole line per thread,
// where the exchanges (two or four words per complex value) and the register limit of the doubled block
// cost more than the occupancy gains.
template <class R>
struct MidSplit {
  static constexpr bool value = false;
};
template <>
struct MidSplit<float> {
  static constexpr bool value = true;
};
template <class R, int B>
constexpr int mid_threads() { return (MidSplit<R>::value ? 2 : 1) * B * B; }

template <class R, int B, bool MULTIPLY>
__global__ void __launch_bounds__(mid_threads<R, B>(), 512 / (B * B)) k_box_mid(
    cx<R> *__restrict__ Y, int64_t fstride, const R *__restrict__ Gh, BoxGeom g, const cx<R> *__restrict__ twl,
    int L, int3 twf, Tw64<R> tw, R *__restrict__ kout) {
  constexpr bool SPLIT = MidSplit<R>::value;
  constexpr int B2 = B * B, B3 = B * B * B, RS = B + 1, NV = SPLIT ? B / 2 : B, Q = B / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R> *S = reinterpret_cast<cx<R> *>(smem_raw);
  // K1 block: blockIdx.x runs over K1x < the launch's widest range; a real field stops at Px/2
  const int pxm = box_pxmax(g);
  const int k1x = (int)(blockIdx.x % pxm), k1y = (int)((blockIdx.x / pxm) % g.P[1]);
  const int k1z = (int)(blockIdx.x / ((unsigned)pxm * g.P[1]));
  if (k1x >= box_pxu(g, blockIdx.y)) return;
  const int64_t kb = k1x + (int64_t)g.P[0] * (k1y + (int64_t)g.P[1] * k1z);  // linear in the full P array
  cx<R> *Yb = Y + blockIdx.y * fstride + kb * B3;  // field blockIdx.y
  // line t = (l0, l1).  SPLIT: lanes 0-15 of warp w hold the even points of the lines 16w .. 16w + 15,
  // lanes 16-31 the odd points of the same lines (each quarter-warp keeps the one-line-per-lane pattern)
  const int h = SPLIT ? (threadIdx.x >> 4) & 1 : 0;
  const int t = SPLIT ? (threadIdx.x >> 5) * 16 + (threadIdx.x & 15) : threadIdx.x, l0 = t % B, l1 = t / B;
  // point of the line in input slot r / output slot j of this thread
  auto in_idx = [h](int r) { return SPLIT ? 2 * r + h : r; };
  auto out_idx = [h](int j) { return SPLIT ? mid_out_index(B, h, j) : j; };
  // twiddle W_Pc^{m.K1} of the cell (x, y, z) = (l0, l1, i) of this z line: W_L^{e0 + i ez mod L} with
  // L = lcm(Pcx, Pcy, Pcz) (m_a K1_a < Pc_a, so each term below is below L: 32-bit)
  // (kept in shared memory between the first and the last step: no registers held across the FFTs)
  __shared__ int s_e0[B2];
  __shared__ int s_ez;
  if (h == 0) s_e0[t] = (l0 * k1x * twf.x + l1 * k1y * twf.y) % L;
  if (threadIdx.x == 0) s_ez = (k1z * twf.z) % L;
  __syncthreads();
  cx<R> v[NV];
  const int nstep = MULTIPLY ? 6 : 3;
  for (int step = 0; step < nstep; ++step) {
    const int ax = step < 3 ? 2 - step : step - 3;
    int base, stride;
    if (ax == 0) base = (l1 * B + l0) * RS, stride = 1;             // x lines: (y, z) = (l0, l1)
    else if (ax == 1) base = l1 * B * RS + l0, stride = RS;         // y lines: (x, z) = (l0, l1)
    else base = l1 * RS + l0, stride = B * RS;                      // z lines: (x, y) = (l0, l1)
    if (step == 0) {
      const int ez = s_ez, dez = SPLIT ? (2 * ez) % L : ez;
      int e = (s_e0[t] + h * ez) % L;
#pragma unroll
      for (int r = 0; r < NV; ++r) {
        const int i = in_idx(r);
        v[r] = cmul(ld_stream(Yb + (i * B + l1) * B + l0), twl[e]);
        e += dez;
        if (e >= L) e -= L;
      }
    } else if (step == 3) {
      if constexpr (SPLIT) mid_regroup<R, B>(v, h);  // the same x lines, in registers
    } else {
#pragma unroll
      for (int r = 0; r < NV; ++r) v[r] = S[base + in_idx(r) * stride];
    }
    // no renormalisation between the line FFTs: the next step's butterflies add lazily, and the kernel
    // product and the final twiddle product renormalise
    if constexpr (SPLIT) fft_split<R, B>(v, h, tw);
    else fft_reg<R, B, false, false>(v, tw);
    if (step == 2) {
      if (!MULTIPLY) {
#pragma unroll
        for (int j = 0; j < NV; ++j) kout[kb * B3 + out_idx(j) * B2 + t] = v[j].re;
      } else {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          const R gk = ld_stream(Gh + kb * B3 + out_idx(j) * B2 + t);  // read once per solve
          v[j] = cx<R>{v[j].re * gk, -(v[j].im * gk)};
        }
      }
      continue;
    }
    if (step == 5) {
      const int ez = s_ez, e0 = s_e0[t];
      int e = 0;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const int i = out_idx(j);
        if (j == 0 || (SPLIT && j == Q)) {
          e = (e0 + i * ez) % L;
        } else {
          e += ez;
          if (e >= L) e -= L;
        }
        Yb[(i * B + l1) * B + l0] = conj(cmul(v[j], twl[e]));
      }
    } else {
#pragma unroll
      for (int j = 0; j < NV; ++j) S[base + out_idx(j) * stride] = v[j];
      __syncthreads();
    }
  }
}
