// box_fft.cuh -- block-index DFT passes as in-register mixed-radix FFTs, for wide level boxes.
//
// A pass along one axis maps, per line and local cell, the nb inputs of the zero-padded length P = 2 nb
// (forward) to its P outputs, or the P inputs back to the nb box outputs (inverse).  Splitting the outputs
// (inputs) by parity turns both into two nb-point DFTs (Sec. 2.2's convolution; the block-index form of
// box.cuh):
//     forward  X_{2q} = DFT_nb(x)_q,            X_{2q+1} = DFT_nb(x_j W_P^j)_q,
//     inverse  y_j = IDFT_nb(X_even)_j + W_P^{-j} IDFT_nb(X_odd)_j,
// and each nb-point DFT runs as a mixed-radix Cooley-Tukey FFT over registers (radix 4, 2, 3, 5, 7; primes
// 11 and 13 directly by conjugate pairs), every index a compile-time constant.  For nb = 16 a pass then
// costs about a third of the direct conjugate-pair sums of box.cuh, whose work grows as nb^2.
// Twiddles W_N^m (N | P) are read from the pass's parameter table W_P^{m P / N}.
#pragma once
#include "box.cuh"

namespace lgf {

constexpr int bfft_radix(int n) {
  return n % 4 == 0 && n != 8 ? 4 : (n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : (n % 5 == 0 ? 5 : (n % 7 == 0 ? 7 : n))));
}

// W_N^m, forward e^{-2 pi i m / N} or its conjugate, from the W_P table (N divides P)
template <class R, int N, int P, bool INV>
LGF_D cx<R> bfft_w(const BoxTw<R> &tw, int m) {
  const cx<R> w = tw.w[(m % N) * (P / N)];
  return INV ? conj(w) : w;
}

// v W_N^m with the trivial angles (0, 1/4, 1/2, 3/4 turn) as swaps and sign changes
template <class R, int N, int P, bool INV>
LGF_D cx<R> bfft_twiddle(const cx<R> &v, const BoxTw<R> &tw, int m) {
  const int r = m % N;
  if (r == 0) return v;
  if (4 * r == N) return INV ? cx<R>{-v.im, v.re} : cx<R>{v.im, -v.re};  // * (+-i)
  if (2 * r == N) return cx<R>{-v.re, -v.im};
  if (4 * r == 3 * N) return INV ? cx<R>{v.im, -v.re} : cx<R>{-v.im, v.re};
  return cmul(v, bfft_w<R, N, P, INV>(tw, r));
}

// A small DFT of N points (N = 2, 4 by butterflies, odd N by conjugate pairs with real coefficients):
//   X_k = x_0 + sum_j c_jk (x_j + x_{N-j}) -+ i sum_j s_jk (x_j - x_{N-j}),  c, s = cos, sin(2 pi j k / N)
template <class R, int N, int P, bool INV>
LGF_D void bfft_small(cx<R> (&x)[N], const BoxTw<R> &tw) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2) {
    const cx<R> a = x[0], b = x[1];
    x[0] = cnorm(cadd(a, b));
    x[1] = cnorm(csub(a, b));
  } else if constexpr (N == 4) {
    const cx<R> s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    const cx<R> s13 = cadd(x[1], x[3]), d13 = csub(x[1], x[3]);
    const cx<R> jd = INV ? cx<R>{-d13.im, d13.re} : cx<R>{d13.im, -d13.re};  // (-+i) (x1 - x3)
    x[0] = cnorm(cadd(s02, s13));
    x[2] = cnorm(csub(s02, s13));
    x[1] = cnorm(cadd(d02, jd));
    x[3] = cnorm(csub(d02, jd));
  } else {
    static_assert(N % 2 == 1, "odd small DFT");
    constexpr int H = (N - 1) / 2;
    cx<R> U[H + 1], V[H + 1];
    cx<R> X0 = x[0];
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      U[j] = cadd(x[j], x[N - j]);
      V[j] = csub(x[j], x[N - j]);
      X0 = cadd(X0, U[j]);
    }
    cx<R> out[N];
    out[0] = cnorm(X0);
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      cx<R> A = x[0], Bs = cx_zero<R>();
#pragma unroll
      for (int j = 1; j <= H; ++j) {
        const cx<R> w = bfft_w<R, N, P, false>(tw, j * k);  // (cos, -sin)
        A = cx<R>{rfma(A.re, U[j].re, w.re), rfma(A.im, U[j].im, w.re)};
        Bs = cx<R>{rfma(Bs.re, V[j].re, w.im), rfma(Bs.im, V[j].im, w.im)};  // -sum sin V
      }
      // forward: X_k = A + i Bs (Bs = -sum s V), X_{N-k} = A - i Bs; inverse the other way round
      const cx<R> iB = cx<R>{-Bs.im, Bs.re};
      out[k] = cnorm(INV ? csub(A, iB) : cadd(A, iB));
      out[N - k] = cnorm(INV ? cadd(A, iB) : csub(A, iB));
    }
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = out[k];
  }
}

// In-place DFT of N points (N | P): X_k = sum_j x_j W_N^{+-jk}.  N = A Q: A sub-DFTs of size Q over
// x[a + A b], twiddles W_N^{a k2}, then Q DFTs of size A: X[k2 + Q k1].
template <class R, int N, int P, bool INV>
struct BFft {
  static LGF_D void run(cx<R> (&x)[N], const BoxTw<R> &tw) {
    constexpr int A = bfft_radix(N), Q = N / A;
    if constexpr (Q == 1) {
      bfft_small<R, N, P, INV>(x, tw);
    } else {
      cx<R> y[A][Q];
#pragma unroll
      for (int a = 0; a < A; ++a) {
#pragma unroll
        for (int b = 0; b < Q; ++b) y[a][b] = x[a + A * b];
        BFft<R, Q, P, INV>::run(y[a], tw);
#pragma unroll
        for (int k2 = 1; k2 < Q; ++k2)
          if (a > 0) y[a][k2] = bfft_twiddle<R, N, P, INV>(y[a][k2], tw, a * k2);
      }
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) {
        cx<R> z[A];
#pragma unroll
        for (int a = 0; a < A; ++a) z[a] = y[a][k2];
        bfft_small<R, A, P, INV>(z, tw);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) x[k2 + Q * k1] = z[k1];
      }
    }
  }
};

}  // namespace lgf

// Forward pass for a compile-time block count NB (P = 2 NB): one thread per (line, cell), all P outputs.
// Grid and arguments as k_bdft_fwd (one chunk: blockIdx.z = field); with gather, NB x NT values of dynamic
// shared memory.
template <class R, int B, int NT, int NB>
__global__ void __launch_bounds__(NT) k_bfft_fwd(const cx<R> *__restrict__ in, cx<R> *__restrict__ out,
                                                 int64_t fstride, BoxGeom g, int ax, int3 ext, BoxTw<R> tw,
                                                 int gather, FwdSpecs sp) {
  using namespace lgf;
  constexpr int B3 = B * B * B, P = 2 * NB;
  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
  const int e1 = ax == 0 ? ext.y : ext.x;
  const int l1 = (int)blockIdx.y % e1, l2 = (int)blockIdx.y / e1;
  const int field = (int)blockIdx.z;
  const int pxf = box_pxu(g, field);
  if (ax != 0 && l1 >= pxf) return;  // a line beyond this field's K1x range
  const bool realx = ax == 0 && pxf < P;
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
  __shared__ int GI[3][NB];
  if (gather) {
    for (int j = threadIdx.x; j < NB; j += NT) {
      const int bidx = gbase + j * gsa;
      GI[0][j] = ns > 0 ? s0.gather[bidx] : -1;
      GI[1][j] = ns > 1 ? s1.gather[bidx] : -1;
      GI[2][j] = ns > 2 ? s2.gather[bidx] : -1;
    }
    __syncthreads();
  }
  const int m = blockIdx.x * NT + threadIdx.x;
  const cx<R> *src = in + field * fstride + lbase + m;
  cx<R> *dst = out + field * fstride + lbase + m;
  auto fetch = [&](int j, bool last) -> cx<R> {
    if (!gather) return last ? ld_stream(src + j * bsa) : src[j * bsa];  // the second read is the last one
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
  // a gathering pass keeps its inputs (read and converted from the caller's fields once) in shared memory
  // for the odd half, each thread its own NB values (no barrier); the other passes re-read theirs from L1/L2
  extern __shared__ __align__(16) unsigned char bfft_smem[];
  cx<R> *SG = reinterpret_cast<cx<R> *>(bfft_smem);
  cx<R> w[NB];
  // even outputs X_{2q} = DFT_NB(x)_q
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    w[j] = fetch(j, false);
    if (gather) SG[j * NT + threadIdx.x] = w[j];
  }
  BFft<R, NB, P, false>::run(w, tw);
#pragma unroll
  for (int q = 0; q < NB; ++q)
    if (!realx || 2 * q <= NB) dst[(2 * q) * bsa] = w[q];
  // odd outputs X_{2q+1} = DFT_NB(x_j W_P^j)_q
#pragma unroll
  for (int j = 0; j < NB; ++j)
    w[j] = bfft_twiddle<R, P, P, false>(gather ? SG[j * NT + threadIdx.x] : fetch(j, true), tw, j);
  BFft<R, NB, P, false>::run(w, tw);
#pragma unroll
  for (int q = 0; q < NB; ++q)
    if (!realx || 2 * q + 1 <= NB) dst[(2 * q + 1) * bsa] = w[q];
}

// Inverse pass for a compile-time block count NB: y_j = sum_{k < P} W_P^{-jk} X_k for the NB box outputs
// (unnormalised), from the even and the odd inputs; a real field (x pass, K1x <= P/2 kept) takes
// X_{P-k} = conj(X_k) and writes the real part.  Grid and arguments as k_bdft_inv (one chunk).
template <class R, int B, int NT, int NB>
__global__ void __launch_bounds__(NT) k_bfft_inv(const cx<R> *__restrict__ in, cx<R> *__restrict__ out,
                                                 int64_t fstride, BoxGeom g, int ax, int3 ext, BoxTw<R> tw,
                                                 int final, InvOuts<R> outs, double scale) {
  using namespace lgf;
  constexpr int B3 = B * B * B, P = 2 * NB;
  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
  const int e1 = ax == 0 ? ext.y : ext.x;
  const int l1 = (int)blockIdx.y % e1, l2 = (int)blockIdx.y / e1;
  const int field = (int)blockIdx.z;
  const int pxf = box_pxu(g, field);
  if (ax != 0 && l1 >= pxf) return;
  const bool realx = ax == 0 && pxf < P;
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
  __shared__ int SO[2][NB], SX[2][NB];
  if (final) {
    for (int j = threadIdx.x; j < NB; j += NT) {
      const int bidx = gbase + j * gsa;
      int ob = -1, ab = -1;
      if (ore.scatter) {
        ob = ore.scatter[bidx];
        ab = ob >= 0 ? (ore.aux ? ore.aux[bidx] : ob) : -1;
      }
      SO[0][j] = ob;
      SX[0][j] = ab;
      ob = ab = -1;
      if (oim.scatter) {
        ob = oim.scatter[bidx];
        ab = ob >= 0 ? (oim.aux ? oim.aux[bidx] : ob) : -1;
      }
      SO[1][j] = ob;
      SX[1][j] = ab;
    }
    __syncthreads();
  }
  const int m = blockIdx.x * NT + threadIdx.x;
  const cx<R> *src = in + field * fstride + lbase + m;
  auto fetch = [&](int k) -> cx<R> {  // X_k; the input is dead after this pass
    if (realx && k > NB) return conj(ld_stream(src + (P - k) * bsa));
    return ld_stream(src + k * bsa);
  };
  // the even inputs' inverse DFT waits in shared memory (NB x NT values) while the odd inputs' runs, so
  // only one line of values is held in registers at a time
  extern __shared__ __align__(16) unsigned char bfft_smem[];
  cx<R> *SE = reinterpret_cast<cx<R> *>(bfft_smem);
  {
    cx<R> w[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) w[q] = fetch(2 * q);
    BFft<R, NB, P, true>::run(w, tw);
#pragma unroll
    for (int j = 0; j < NB; ++j) SE[j * NT + threadIdx.x] = w[j];
  }
  cx<R> y[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) y[q] = fetch(2 * q + 1);
  BFft<R, NB, P, true>::run(y, tw);
#pragma unroll
  for (int j = 0; j < NB; ++j) y[j] = cnorm(cadd(SE[j * NT + threadIdx.x], bfft_twiddle<R, P, P, true>(y[j], tw, j)));
  if (!final) {
    cx<R> *dst = out + field * fstride + lbase + m;
#pragma unroll
    for (int j = 0; j < NB; ++j) dst[j * bsa] = y[j];
    return;
  }
  const R sc = RT<R>::from(scale);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    box_store_at<R>(ore, SO[0][j], SX[0][j], m, B3, y[j].re * sc);
    if (!realx) box_store_at<R>(oim, SO[1][j], SX[1][j], m, B3, y[j].im * sc);
  }
}
