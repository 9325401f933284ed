// pair.cuh -- block transforms and the block-pair multiply-accumulate (pair mode).
//
// Sec. 2.2 (Eq. (eq:lgf_convolution)): phi(n) = h^2 sum_m G(n - m) f(m).  Split the lattice into B^3
// blocks; for a target block t and a source block s, with n = B t + p and m = B s + q
// (p, q in [0, B)^3),
//     phi_t(p) = h^2 sum_s sum_q g_{t-s}(p - q) f_s(q),   g_o(d) = G(B o + d),  d in (-B, B)^3.
// Each inner sum is a linear convolution of two length-B signals per axis, so a circular
// convolution of length 2B is exact on the output window p in [0, B)^3 when f_s is zero padded to
// (2B)^3 and g_o is laid out circularly (slot d = +-B never reaches the window and holds 0).
// In the Fourier domain (half spectrum along x, W = (2B)^2 (B+1) frequencies)
//     Phi_t(w) = sum_s Ghat_{t-s}(w) Fhat_s(w),
// the sum over block pairs evaluated per frequency (the "FFT-domain multiply-accumulate").
//
// Spectrum layout: [entity][w], w = (kz * 2B + ky) * (B+1) + kx, complex, compute precision R.
#pragma once
#include "common.cuh"

// ------------------------------------------------------------------ padded / windowed 1D pieces
// Forward DFT of length 2B of B samples followed by B zeros: X[2k] = FFT_B(x)[k],
// X[2k+1] = FFT_B(x_j W_2B^j)[k].  `put(k, v)` stores output k.
template <class R, int B, class Load, class Put>
LGF_D void dft_pad_fwd(const Tw64<R> &tw, Load load, Put put) {
  cx<R> x[B];
#pragma unroll
  for (int j = 0; j < B; ++j) x[j] = load(j);
  fft_reg<R, B, false>(x, tw);
#pragma unroll
  for (int k = 0; k < B; ++k) put(2 * k, x[k]);
#pragma unroll
  for (int j = 0; j < B; ++j) {
    x[j] = load(j);
    if (j) x[j] = cmul(x[j], twiddle<R, 2 * B, false>(tw, j));
  }
  fft_reg<R, B, false>(x, tw);
#pragma unroll
  for (int k = 0; k < B; ++k) put(2 * k + 1, x[k]);
}

// Inverse DFT of length 2B restricted to outputs j < B (unnormalised):
// x_j = IFFT_B(X_even)[j] + W_2B^{-j} IFFT_B(X_odd)[j].  `put(j, v)` stores, `add(j, v)` accumulates.
template <class R, int B, class Load, class Put, class Add>
LGF_D void dft_window_inv(const Tw64<R> &tw, Load load, Put put, Add add) {
  cx<R> x[B];
#pragma unroll
  for (int k = 0; k < B; ++k) x[k] = load(2 * k);
  fft_reg<R, B, true>(x, tw);
#pragma unroll
  for (int j = 0; j < B; ++j) put(j, x[j]);
#pragma unroll
  for (int k = 0; k < B; ++k) x[k] = load(2 * k + 1);
  fft_reg<R, B, true>(x, tw);
#pragma unroll
  for (int j = 0; j < B; ++j) {
    cx<R> v = x[j];
    if (j) v = cmul(v, twiddle<R, 2 * B, true>(tw, j));
    add(j, v);
  }
}

template <int B>
struct PairGeom {
  static constexpr int N2 = 2 * B;
  static constexpr int KX = B + 1;
  static constexpr int W = N2 * N2 * KX;                 // half-spectrum size
  static constexpr int A1 = B * B * KX;                  // [z][y][kx] after the x pass
  static constexpr int A2 = B * N2 * KX;                 // [z][ky][kx] after the y pass
  static constexpr int NT = 256;                         // threads per CTA
};

template <class R, int B>
constexpr size_t pair_fft_smem() {
  return sizeof(cx<R>) * (size_t)(PairGeom<B>::A1 + PairGeom<B>::A2);
}

// ------------------------------------------------------------------ forward: B^3 real -> spectrum
// grid (nsrc, ncomp).  Source block b = src_idx[blockIdx.x] of component blockIdx.y is read from
// f + comp * comp_stride + b * B^3 (dtype per load_field); spectrum written to
// out + (comp * nsrc + blockIdx.x) * W.
template <class R, int B>
__global__ void __launch_bounds__(256) k_block_fwd(const void *__restrict__ f, int dtype,
                                                   int64_t comp_stride,
                                                   const int32_t *__restrict__ src_idx, int nsrc,
                                                   cx<R> *__restrict__ out,
                                                   const uint8_t *__restrict__ cellmask, int bits,
                                                   Tw64<R> tw) {
  using G = PairGeom<B>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R> *A1 = reinterpret_cast<cx<R> *>(smem_raw);
  cx<R> *A2 = A1 + G::A1;
  const int comp = blockIdx.y;
  const int64_t blk = src_idx[blockIdx.x];
  const int64_t base = comp * comp_stride + blk * (B * B * B);
  const uint8_t *cm = cellmask ? cellmask + blk * (B * B * B) : nullptr;
  cx<R> *spec = out + ((int64_t)comp * nsrc + blockIdx.x) * G::W;
  auto ld = [&](int64_t cell) {  // cell index inside the block
    if (cm && !(cm[cell] & bits)) return RT<R>::zero();
    return load_field<R>(f, base + cell, dtype);
  };

  // x pass: rows y0 = 2 yp, y1 = 2 yp + 1 packed as one complex signal a + i b
  for (int t = threadIdx.x; t < B * B / 2; t += blockDim.x) {
    const int z = t / (B / 2), yp = t % (B / 2);
    const int64_t r0 = ((int64_t)z * B + 2 * yp) * B;
    cx<R> *S = A2;  // scratch: S[k * (B*B/2) + t], k < 2B
    dft_pad_fwd<R, B>(
        tw, [&](int j) { return cx<R>{ld(r0 + j), ld(r0 + B + j)}; },
        [&](int k, cx<R> v) { S[k * (B * B / 2) + t] = v; });
    cx<R> *row0 = A1 + ((z * B) + 2 * yp) * G::KX;
    cx<R> *row1 = row0 + G::KX;
#pragma unroll 1
    for (int k = 0; k <= B; ++k) {
      cx<R> zk = S[k * (B * B / 2) + t];
      cx<R> zm = S[((2 * B - k) & (2 * B - 1)) * (B * B / 2) + t];
      row0[k] = cx<R>{RT<R>::half(zk.re + zm.re), RT<R>::half(zk.im - zm.im)};
      row1[k] = cx<R>{RT<R>::half(zk.im + zm.im), RT<R>::half(zm.re - zk.re)};
    }
  }
  __syncthreads();
  // y pass: columns (z, kx), B samples -> 2B
  for (int t = threadIdx.x; t < B * G::KX; t += blockDim.x) {
    const int z = t / G::KX, kx = t % G::KX;
    dft_pad_fwd<R, B>(
        tw, [&](int j) { return A1[(z * B + j) * G::KX + kx]; },
        [&](int k, cx<R> v) { A2[(z * G::N2 + k) * G::KX + kx] = v; });
  }
  __syncthreads();
  // z pass: columns (ky, kx), B samples -> 2B, straight to the spectrum
  for (int t = threadIdx.x; t < G::N2 * G::KX; t += blockDim.x) {
    dft_pad_fwd<R, B>(
        tw, [&](int j) { return A2[j * (G::N2 * G::KX) + t]; },
        [&](int k, cx<R> v) { spec[k * (G::N2 * G::KX) + t] = v; });
  }
}

// ------------------------------------------------------------------ inverse: spectrum -> window
// grid (n, ncomp).  Target i reads spectrum row r = rows ? rows[i] : i of component `comp`
// (spec_in + comp * spec_cs + r * W), and with a = aux[i] writes
//   out[comp * out_cs + (a + out_off) * B^3 + cell] = scale * window (+ addend[comp * add_cs + a * B^3 + cell])
// for the cells whose cellmask[a * B^3 + cell] has a bit of `bits` (all cells when cellmask is null).
// The addend is an internal buffer in the arithmetic R.
template <class R, int B>
__global__ void __launch_bounds__(256) k_block_inv(const cx<R> *__restrict__ spec_in, int64_t spec_cs,
                                                   const int32_t *__restrict__ rows,
                                                   const int32_t *__restrict__ aux,
                                                   void *__restrict__ out, int dtype,
                                                   int64_t out_cs, int64_t out_off,
                                                   const R *__restrict__ addend, int64_t add_cs,
                                                   const uint8_t *__restrict__ cellmask, int bits,
                                                   double scale, Tw64<R> tw) {
  using G = PairGeom<B>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R> *A1 = reinterpret_cast<cx<R> *>(smem_raw);
  cx<R> *A2 = A1 + G::A1;
  const int comp = blockIdx.y;
  const int r = rows ? rows[blockIdx.x] : (int)blockIdx.x;
  const cx<R> *spec = spec_in + comp * spec_cs + (int64_t)r * G::W;
  const int64_t a = aux[blockIdx.x];
  const int64_t base = comp * out_cs + (a + out_off) * (B * B * B);
  const R *add = addend ? addend + comp * add_cs + a * (B * B * B) : nullptr;
  const uint8_t *cm = cellmask ? cellmask + a * (B * B * B) : nullptr;

  // z pass: columns (ky, kx): 2B -> window z < B
  for (int t = threadIdx.x; t < G::N2 * G::KX; t += blockDim.x) {
    dft_window_inv<R, B>(
        tw, [&](int k) { return spec[k * (G::N2 * G::KX) + t]; },
        [&](int j, cx<R> v) { A2[j * (G::N2 * G::KX) + t] = v; },
        [&](int j, cx<R> v) {
          cx<R> &d = A2[j * (G::N2 * G::KX) + t];
          d = d + v;
        });
  }
  __syncthreads();
  // y pass: columns (z, kx): 2B -> window y < B
  for (int t = threadIdx.x; t < B * G::KX; t += blockDim.x) {
    const int z = t / G::KX, kx = t % G::KX;
    dft_window_inv<R, B>(
        tw, [&](int k) { return A2[(z * G::N2 + k) * G::KX + kx]; },
        [&](int j, cx<R> v) { A1[(z * B + j) * G::KX + kx] = v; },
        [&](int j, cx<R> v) {
          cx<R> &d = A1[(z * B + j) * G::KX + kx];
          d = d + v;
        });
  }
  __syncthreads();
  // x pass: row pair (y0, y1) from the half spectra A, Bv via Z = A + i Bv (Hermitian extension)
  const R sc = RT<R>::from(scale);
  for (int t = threadIdx.x; t < B * B / 2; t += blockDim.x) {
    const int z = t / (B / 2), yp = t % (B / 2);
    const cx<R> *ra = A1 + (z * B + 2 * yp) * G::KX;
    const cx<R> *rb = ra + G::KX;
    cx<R> *S = A2;  // scratch S[j * (B*B/2) + t], j < B
    const int64_t o0 = ((int64_t)z * B + 2 * yp) * B;
    dft_window_inv<R, B>(
        tw,
        [&](int k) {
          if (k <= B) {
            cx<R> a = ra[k], b = rb[k];
            return cx<R>{a.re - b.im, a.im + b.re};
          }
          cx<R> a = ra[2 * B - k], b = rb[2 * B - k];
          return cx<R>{a.re + b.im, b.re - a.im};
        },
        [&](int j, cx<R> v) { S[j * (B * B / 2) + t] = v; },
        [&](int j, cx<R> v) {
          cx<R> zz = S[j * (B * B / 2) + t] + v;
          R va = zz.re * sc, vb = zz.im * sc;
          const int64_t ca = o0 + j, cb = o0 + B + j;
          if (add) {
            va = va + add[ca];
            vb = vb + add[cb];
          }
          if (!cm || (cm[ca] & bits)) store_field<R>(out, base + ca, dtype, va);
          if (!cm || (cm[cb] & bits)) store_field<R>(out, base + cb, dtype, vb);
        });
  }
}

// ------------------------------------------------------------------ block-pair MAC
// grid (ceil(ntgt / TC), ceil(W / blockDim.x)); one thread = one frequency w and TC targets.
//   Phi[c * p_cs + t * W + w] (+)= sum_s Ghat[idx(T_t - S_s)][w] * F[c * f_cs + s * W + w]
// with block coordinates S_s = coords[src_list ? src_list[s] : s] (same for targets) and
// idx(o) = ((oz + mo.z) * (2 mo.y + 1) + (oy + mo.y)) * (2 mo.x + 1) + (ox + mo.x).
template <class R, int TC, int NC>
__global__ void __launch_bounds__(128) k_mac_pair(const cx<R> *__restrict__ F, int nsrc, int64_t f_cs,
                                                  const int32_t *__restrict__ src_list,
                                                  const int4 *__restrict__ src_coords,
                                                  const cx<R> *__restrict__ Gh, int3 mo,
                                                  cx<R> *__restrict__ Phi, int ntgt, int64_t p_cs,
                                                  const int32_t *__restrict__ tgt_list,
                                                  const int4 *__restrict__ tgt_coords, int W,
                                                  int accumulate) {
  const int w = blockIdx.y * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int t0 = blockIdx.x * TC;
  int tb[TC];
  int4 tc[TC];
#pragma unroll
  for (int i = 0; i < TC; ++i) {
    tb[i] = (t0 + i < ntgt);
    tc[i] = tb[i] ? tgt_coords[tgt_list ? tgt_list[t0 + i] : t0 + i] : make_int4(0, 0, 0, 0);
  }
  const int sx = 2 * mo.x + 1, sy = 2 * mo.y + 1;
  cx<R> acc[TC][NC];
#pragma unroll
  for (int i = 0; i < TC; ++i)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[i][c] = cx_zero<R>();
  for (int s = 0; s < nsrc; ++s) {
    const int4 sc = src_coords[src_list ? src_list[s] : s];
    cx<R> fv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) fv[c] = F[c * f_cs + (int64_t)s * W + w];
#pragma unroll
    for (int i = 0; i < TC; ++i) {
      if (!tb[i]) continue;
      const int idx = ((tc[i].z - sc.z + mo.z) * sy + (tc[i].y - sc.y + mo.y)) * sx +
                      (tc[i].x - sc.x + mo.x);
      const cx<R> g = Gh[(int64_t)idx * W + w];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[i][c] = cmac(acc[i][c], g, fv[c]);
    }
  }
#pragma unroll
  for (int i = 0; i < TC; ++i) {
    if (!tb[i]) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      cx<R> *p = Phi + c * p_cs + (int64_t)(t0 + i) * W + w;
      *p = accumulate ? (*p + acc[i][c]) : acc[i][c];
    }
  }
}
