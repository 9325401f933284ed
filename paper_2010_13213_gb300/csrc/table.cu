// table.cu -- LGF table generation (FP64) and the block-offset kernel spectra.
//
// G(n) = -int_0^inf prod_i e^{-2t} I_{n_i}(2t) dt  (the 7-point LGF with L_1 G = delta, Sec. 2.2).
// Device work:
//   k_ive_nodes   one thread per quadrature node t_j: e^{-x} I_k(x), x = 2 t_j, k = 0..N, by Miller's
//                 backward recurrence normalised with e^{-x}(I_0 + 2 sum I_k) = 1;
//   k_lgf_octant  one thread per sorted triple a <= b <= c <= N: compensated sum of the quadrature
//                 plus the large-t tail, written to the six permutations of a dense octant array;
//   k_kspec_xy / k_kspec_z   for every block offset o the circular segment g_o(d) = G(B o + d),
//                 d in (-B, B)^3 (slot +-B = 0), forward-transformed on (2B)^3 (half spectrum).
// The quadrature rule is built on the host (Gauss-Legendre panels in ln t); the tail uses the
// Hankel large-argument series of e^{-x} I_nu(x) multiplied out and integrated term by term.
#include <math.h>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "pair.cuh"

namespace lgf {

// ------------------------------------------------------------------ quadrature rule (host)
// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_n with Tricomi's initial guesses.
static void gl_rule(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 1; i <= n; ++i) {
    double th = pi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
    double r = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(th);
    double pn = 0.0, dpn = 0.0;
    for (int it = 0; it < 60; ++it) {
      double pm1 = 1.0, p = r;  // P_0, P_1
      for (int k = 1; k < n; ++k) {
        double pn1 = ((2.0 * k + 1.0) * r * p - k * pm1) / (k + 1.0);
        pm1 = p;
        p = pn1;
      }
      pn = p;
      dpn = n * (pm1 - r * p) / (1.0 - r * r);
      double step = pn / dpn;
      r -= step;
      if (fabs(step) < 4e-17) break;
    }
    {
      double pm1 = 1.0, p = r;
      for (int k = 1; k < n; ++k) {
        double pn1 = ((2.0 * k + 1.0) * r * p - k * pm1) / (k + 1.0);
        pm1 = p;
        p = pn1;
      }
      dpn = n * (pm1 - r * p) / (1.0 - r * r);
    }
    x[i - 1] = r;
    w[i - 1] = 2.0 / ((1.0 - r * r) * dpn * dpn);
  }
}

struct Rule {
  std::vector<double> t, w;
  double T;
};

static Rule make_rule(int N) {
  Rule R;
  R.T = 500.0 * (double)(N > 1 ? N : 1) * (double)(N > 1 ? N : 1) + 1000.0;
  std::vector<double> x16, w16, x24, w24;
  gl_rule(16, x16, w16);
  gl_rule(24, x24, w24);
  // [0, 1/2] in t: two panels of 16 points
  for (int p = 0; p < 2; ++p) {
    double a = 0.25 * p, b = a + 0.25;
    for (int i = 0; i < 16; ++i) {
      R.t.push_back(0.5 * (a + b) + 0.5 * (b - a) * x16[i]);
      R.w.push_back(0.5 * (b - a) * w16[i]);
    }
  }
  // [1/2, T] in u = ln t, panels of width <= 0.3 with 24 points; dt = t du
  double u0 = log(0.5), u1 = log(R.T);
  int np = (int)ceil((u1 - u0) / 0.3);
  double hu = (u1 - u0) / np;
  for (int p = 0; p < np; ++p) {
    double a = u0 + p * hu, b = a + hu;
    for (int i = 0; i < 24; ++i) {
      double u = 0.5 * (a + b) + 0.5 * (b - a) * x24[i];
      double t = exp(u);
      R.t.push_back(t);
      R.w.push_back(0.5 * (b - a) * w24[i] * t);
    }
  }
  return R;
}

// ------------------------------------------------------------------ device kernels
__global__ void k_ive_nodes(const double *__restrict__ tn, int nn, int N, double *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nn) return;
  const double x = 2.0 * tn[j];
  double *o = out + (size_t)j * (N + 1);
  for (int k = 0; k <= N; ++k) o[k] = 0.0;
  if (!(x > 0.0)) {
    o[0] = 1.0;
    return;
  }
  int M = (int)ceil(sqrt((double)N * N + 100.0 * x)) + 50;
  double up = 0.0, cur = 1.0, acc = 0.0;  // b_{k+1}, b_k, sum_{i > k} b_i
  for (int k = M; k >= 1; --k) {
    if (k <= N) o[k] = cur;
    acc += cur;
    const double nxt = fma(2.0 * k / x, cur, up);
    up = cur;
    cur = nxt;
    if (cur > 1e250) {
      up *= 1e-250;
      cur *= 1e-250;
      acc *= 1e-250;
      for (int i = k; i <= N && i <= M; ++i) o[i] *= 1e-250;
    }
  }
  const double norm = cur + 2.0 * acc;
  o[0] = cur / norm;
  for (int k = 1; k <= N; ++k) o[k] /= norm;
}

// alpha_k(nu) of e^{-2t} I_nu(2t) ~ (4 pi t)^{-1/2} sum_k alpha_k t^{-k}
__device__ void hankel_coeffs(int nu, double *a, int nterm) {
  double v = 1.0;
  a[0] = 1.0;
  const double mu = 4.0 * (double)nu * nu;
  for (int k = 1; k < nterm; ++k) {
    const double odd = 2.0 * k - 1.0;
    v *= -(mu - odd * odd) / (16.0 * k);  // -(mu - (2k-1)^2) / (8k) / 2
    a[k] = v;
  }
}

#define LGF_TAIL_TERMS 12
__global__ void k_lgf_octant(const double *__restrict__ iv, const double *__restrict__ wq, int nn,
                             int N, double T, double *__restrict__ Gd) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y, c = blockIdx.z;
  if (a > b || b > c || a > N) return;
  const int K = N + 1;
  double s = 0.0, comp = 0.0;
  for (int j = 0; j < nn; ++j) {
    const double *r = iv + (size_t)j * K;
    const double v = wq[j] * (r[a] * r[b] * r[c]);
    const double t = s + v;
    comp += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  double ha[LGF_TAIL_TERMS], hb[LGF_TAIL_TERMS], hc[LGF_TAIL_TERMS];
  hankel_coeffs(a, ha, LGF_TAIL_TERMS);
  hankel_coeffs(b, hb, LGF_TAIL_TERMS);
  hankel_coeffs(c, hc, LGF_TAIL_TERMS);
  double tail = 0.0, Tp = 1.0 / sqrt(T);
  for (int j = 0; j < LGF_TAIL_TERMS; ++j) {
    double cj = 0.0;
    for (int p = 0; p <= j; ++p)
      for (int q = 0; p + q <= j; ++q) cj += ha[p] * hb[q] * hc[j - p - q];
    tail += cj * Tp / (j + 0.5);
    Tp /= T;
  }
  const double inv4pi32 = 1.0 / (8.0 * 3.14159265358979323846 * sqrt(3.14159265358979323846));
  const double g = -(s + comp + tail * inv4pi32);
  const int p3[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
  for (int q = 0; q < 6; ++q) Gd[((size_t)p3[q][2] * K + p3[q][1]) * K + p3[q][0]] = g;
}

// Full (2B)-point FFT in FP64 registers (used only for the one-off kernel spectra).
template <int N2>
__device__ __forceinline__ void fft_full(cx<double> (&x)[N2], const Tw64<double> &tw) {
  fft_reg<double, N2, false>(x, tw);
}

__device__ __forceinline__ double seg_value(const double *Gd, int K, int B, int ox, int oy, int oz,
                                            int px, int py, int pz) {
  if (px == B || py == B || pz == B) return 0.0;
  const int dx = px < B ? px : px - 2 * B;
  const int dy = py < B ? py : py - 2 * B;
  const int dz = pz < B ? pz : pz - 2 * B;
  const int nx = abs(B * ox + dx), ny = abs(B * oy + dy), nz = abs(B * oz + dz);
  return Gd[((size_t)nz * K + ny) * K + nx];
}

// grid (noff_batch, 2B); 64 threads.  Tmp[(ob * 2B + pz) * 2B * (B+1) + ky * (B+1) + kx]
template <int B>
__global__ void __launch_bounds__(64) k_kspec_xy(const double *__restrict__ Gd, int K, int off0,
                                                 int3 mo, cx<double> *__restrict__ Tmp,
                                                 Tw64<double> tw) {
  constexpr int N2 = 2 * B, KX = B + 1;
  __shared__ cx<double> slab[N2 * KX];
  const int ob = blockIdx.x, pz = blockIdx.y;
  const int o = off0 + ob;
  const int sx = 2 * mo.x + 1, sy = 2 * mo.y + 1;
  const int ox = o % sx - mo.x, oy = (o / sx) % sy - mo.y, oz = o / (sx * sy) - mo.z;
  // x pass: row pairs (2 yp, 2 yp + 1) over py in [0, 2B)
  for (int yp = threadIdx.x; yp < B; yp += blockDim.x) {
    cx<double> x[N2];
#pragma unroll
    for (int px = 0; px < N2; ++px)
      x[px] = cx<double>{seg_value(Gd, K, B, ox, oy, oz, px, 2 * yp, pz),
                         seg_value(Gd, K, B, ox, oy, oz, px, 2 * yp + 1, pz)};
    fft_full<N2>(x, tw);
#pragma unroll
    for (int k = 0; k <= B; ++k) {
      cx<double> zk = x[k], zm = x[(N2 - k) & (N2 - 1)];
      slab[(2 * yp) * KX + k] = cx<double>{0.5 * (zk.re + zm.re), 0.5 * (zk.im - zm.im)};
      slab[(2 * yp + 1) * KX + k] = cx<double>{0.5 * (zk.im + zm.im), 0.5 * (zm.re - zk.re)};
    }
  }
  __syncthreads();
  // y pass: column kx over py
  for (int kx = threadIdx.x; kx < KX; kx += blockDim.x) {
    cx<double> x[N2];
#pragma unroll
    for (int py = 0; py < N2; ++py) x[py] = slab[py * KX + kx];
    fft_full<N2>(x, tw);
#pragma unroll
    for (int ky = 0; ky < N2; ++ky) Tmp[((size_t)(ob * N2 + pz) * N2 + ky) * KX + kx] = x[ky];
  }
}

// grid ceil(noff_batch * 2B * (B+1) / 128); thread = (ob, ky, kx) column along pz.
template <int B>
__global__ void __launch_bounds__(128) k_kspec_z(const cx<double> *__restrict__ Tmp, int nob,
                                                 int off0, cx<double> *__restrict__ s64,
                                                 cx<float> *__restrict__ s32, cx<df> *__restrict__ sdf,
                                                 Tw64<double> tw) {
  constexpr int N2 = 2 * B, KX = B + 1, PL = N2 * KX, W = N2 * N2 * KX;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nob * PL) return;
  const int ob = g / PL, col = g % PL;
  cx<double> x[N2];
#pragma unroll
  for (int pz = 0; pz < N2; ++pz) x[pz] = Tmp[(size_t)(ob * N2 + pz) * PL + col];
  fft_full<N2>(x, tw);
  const size_t o = (size_t)(off0 + ob) * W;
#pragma unroll
  for (int kz = 0; kz < N2; ++kz) {
    const size_t i = o + (size_t)kz * PL + col;
    if (s64) s64[i] = x[kz];
    if (s32) s32[i] = cx<float>{(float)x[kz].re, (float)x[kz].im};
    if (sdf) sdf[i] = cx<df>{df_make(x[kz].re), df_make(x[kz].im)};
  }
}

// ------------------------------------------------------------------ host entry points
int build_lgf_octant(int N, double **Gd_out, cudaStream_t st, double *quad_T, int *quad_nodes) {
  Rule R = make_rule(N);
  const int nn = (int)R.t.size();
  double *dt = nullptr, *dw = nullptr, *div = nullptr, *Gd = nullptr;
  const size_t K = (size_t)N + 1;
  if (cudaMalloc(&dt, sizeof(double) * nn) != cudaSuccess) return LGF_E_OOM;
  if (cudaMalloc(&dw, sizeof(double) * nn) != cudaSuccess) return LGF_E_OOM;
  if (cudaMalloc(&div, sizeof(double) * nn * K) != cudaSuccess) return LGF_E_OOM;
  if (cudaMalloc(&Gd, sizeof(double) * K * K * K) != cudaSuccess) return LGF_E_OOM;
  cudaMemcpyAsync(dt, R.t.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dw, R.w.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, st);
  k_ive_nodes<<<(nn + 63) / 64, 64, 0, st>>>(dt, nn, N, div);
  dim3 grid((unsigned)((N + 1 + 63) / 64), (unsigned)(N + 1), (unsigned)(N + 1));
  k_lgf_octant<<<grid, 64, 0, st>>>(div, dw, nn, N, R.T, Gd);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(dt);
  cudaFree(dw);
  cudaFree(div);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaFree(Gd);
    return set_error(LGF_E_CUDA, "LGF quadrature kernels failed: %s", cudaGetErrorString(e));
  }
  *Gd_out = Gd;
  if (quad_T) *quad_T = R.T;
  if (quad_nodes) *quad_nodes = nn;
  return LGF_OK;
}

template <int B>
static int spectra_impl(const double *Gd, int K, int3 mo, int noff, cx<double> *s64, cx<float> *s32,
                        cx<df> *sdf, cudaStream_t st) {
  constexpr int N2 = 2 * B, KX = B + 1;
  const int batch = 512;
  cx<double> *tmp = nullptr;
  const size_t tmp_elems = (size_t)batch * N2 * N2 * KX;
  if (cudaMalloc(&tmp, sizeof(cx<double>) * tmp_elems) != cudaSuccess) return LGF_E_OOM;
  Tw64<double> tw = make_tw64<double>();
  for (int off0 = 0; off0 < noff; off0 += batch) {
    const int nob = noff - off0 < batch ? noff - off0 : batch;
    k_kspec_xy<B><<<dim3(nob, N2), 64, 0, st>>>(Gd, K, off0, mo, tmp, tw);
    const int cols = nob * N2 * KX;
    k_kspec_z<B><<<(cols + 127) / 128, 128, 0, st>>>(tmp, nob, off0, s64, s32, sdf, tw);
  }
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return set_error(LGF_E_CUDA, "kernel spectra failed: %s", cudaGetErrorString(e));
  return LGF_OK;
}

int build_spectra(int B, const double *Gd, int K, int3 mo, int noff, void *s64, void *s32, void *sdf,
                  cudaStream_t st) {
  if (B == 8)
    return spectra_impl<8>(Gd, K, mo, noff, (cx<double> *)s64, (cx<float> *)s32, (cx<df> *)sdf, st);
  if (B == 16)
    return spectra_impl<16>(Gd, K, mo, noff, (cx<double> *)s64, (cx<float> *)s32, (cx<df> *)sdf, st);
  return set_error(LGF_E_UNSUPPORTED, "block size %d not supported", B);
}

}  // namespace lgf
