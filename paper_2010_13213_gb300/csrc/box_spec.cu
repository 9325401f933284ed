// box_spec.cu -- kernel spectra of the block-index FFT mode, one per level-box shape, cached in the table.
//
// For a box of nb blocks per axis (periodic lattice Pc = 2 nb B), Ghat[K1][K2] is the Pc^3 DFT of the
// circularly laid out unit-lattice LGF (cell n holds G(d), d = n for n <= Pc/2, n - Pc above), in the
// four-step order of box.cuh.  G is real and even so Ghat is real.  Computed once in FP64 (dense
// block-index DFTs + the local FFT of k_box_mid), then rounded to FP32 and split into double-float.
#include <math.h>
#include <string.h>

#include <numeric>
#include <vector>

#include "box.cuh"
#include "internal.h"

namespace lgf {

__global__ void k_spec_convert(const double *__restrict__ g, int64_t n, float *__restrict__ g32,
                               df *__restrict__ gdf) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (g32) g32[i] = (float)g[i];
  if (gdf) gdf[i] = df_make(g[i]);
}

__global__ void k_tw_convert(const double *__restrict__ c, const double *__restrict__ s, int n,
                             cx<double> *__restrict__ t64, cx<float> *__restrict__ t32, cx<df> *__restrict__ tdf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  t64[i] = cx<double>{c[i], -s[i]};
  t32[i] = cx<float>{(float)c[i], -(float)s[i]};
  tdf[i] = cx<df>{df_make(c[i]), df_make(-s[i])};
}

// e^{-2 pi i n / N}, n < N, from long-double cos/sin folded into the first octant.
void twiddles_host(int N, std::vector<double> &c, std::vector<double> &s) {
  const long double pi = 3.141592653589793238462643383279502884L;
  c.resize(N);
  s.resize(N);
  for (int n = 0; n < N; ++n) {
    // reduce 2 pi n / N to [0, pi/4] with exact symmetries (N multiple of 4 here)
    long double a = 2.0L * pi * (long double)n / (long double)N;
    c[n] = (double)cosl(a);
    s[n] = (double)sinl(a);
    if (4 * n == N) c[n] = 0.0, s[n] = 1.0;
    if (2 * n == N) c[n] = -1.0, s[n] = 0.0;
    if (4 * n == 3 * N) c[n] = 0.0, s[n] = -1.0;
    if (n == 0) c[n] = 1.0, s[n] = 0.0;
  }
}

// Coefficient digits of one block-index DFT pass (box_tc.cuh): C_jo = W_P^{-+jo} (dir -1 forward, +1
// inverse); `realw`: the Hermitian-folded real inverse, weights 1 (j = 0, 2j = P) or 2 and real output
// only.  M^T[n = 2o + p][k = 2j + q] / sigma = 2^{-7} sum_t c_t 2^{-8t} with integer digits |c_t| <= 128.
static void tc_matrix(int P, int nin, int nout, int dir, bool realw, const std::vector<double> &c,
                      const std::vector<double> &s, std::vector<uint16_t> &buf, TcMat &M) {
  const int K = 2 * nin, N = 2 * nout;
  M.nin = nin;
  M.nout = nout;
  M.Kp = (K + 15) / 16 * 16;
  M.Np = (N + 15) / 16 * 16;
  M.sigma = realw ? 2.0f : 1.0f;
  M.plane16 = M.Np * M.Kp * 2 / 16;
  const size_t off = buf.size(), plane = (size_t)M.Np * M.Kp;
  buf.resize(off + TC_SMAX * plane, 0);
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      const int j = k / 2, q = k % 2, o = n / 2, p = n % 2;
      const int idx = (int)(((int64_t)j * o) % P);
      const double w = realw ? ((j == 0 || 2 * j == P) ? 1.0 : 2.0) : 1.0;
      const double cr = w * c[idx], ci = w * (dir < 0 ? -s[idx] : s[idx]);
      double v;
      if (p == 0) v = q == 0 ? cr : -ci;
      else v = realw ? 0.0 : (q == 0 ? ci : cr);
      double r = v / (double)M.sigma * 128.0;
      const size_t pos = ((size_t)(n / 8) * (M.Kp / 8) + k / 8) * 64 + (n % 8) * 8 + (k % 8);
      for (int t = 0; t < TC_SMAX; ++t) {
        const double d = nearbyint(r);
        r = (r - d) * 256.0;
        const float fd = (float)d;  // |d| <= 128: exact in bf16 (the top half of the float)
        uint32_t bits;
        memcpy(&bits, &fd, 4);
        buf[off + t * plane + pos] = (uint16_t)(bits >> 16);
      }
    }
  M.d = reinterpret_cast<const uint16_t *>(off);  // offset for now; rebased after the upload
}

static int tc_matrices(BoxSpec *S, const BoxGeom &g, cudaStream_t st) {
  std::vector<uint16_t> buf;
  for (int a = 0; a < 3; ++a) {
    std::vector<double> c, s;
    twiddles_host(g.P[a], c, s);
    tc_matrix(g.P[a], g.nb[a], g.P[a], -1, false, c, s, buf, S->tcm[a][0]);
    tc_matrix(g.P[a], g.P[a], g.nb[a], +1, false, c, s, buf, S->tcm[a][1]);
    if (a == 0) tc_matrix(g.P[a], g.P[a] / 2 + 1, g.nb[a], +1, true, c, s, buf, S->tcm[a][2]);
  }
  if (cudaMalloc(&S->tcw, buf.size() * 2) != cudaSuccess) return set_error(LGF_E_OOM, "tensor-core coefficients");
  cudaMemcpyAsync(S->tcw, buf.data(), buf.size() * 2, cudaMemcpyHostToDevice, st);
  for (int a = 0; a < 3; ++a)
    for (int v = 0; v < 3; ++v)
      if (S->tcm[a][v].Np) S->tcm[a][v].d = S->tcw + reinterpret_cast<size_t>(S->tcm[a][v].d);
  S->bytes += buf.size() * 2;
  cudaError_t e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "coefficient upload: %s", cudaGetErrorString(e));
}

BoxSpec::~BoxSpec() {
  cudaFree(tcw);
  cudaFree(g64);
  cudaFree(g32);
  cudaFree(gdf);
  cudaFree(twl64);
  cudaFree(twl32);
  cudaFree(twldf);
}

template <int B>
static int gen_spectrum(lgf_table *t, BoxSpec *S, cudaStream_t st) {
  constexpr int B3 = B * B * B;
  BoxGeom g;
  for (int a = 0; a < 3; ++a) {
    g.nb[a] = S->nb[a];
    g.P[a] = 2 * S->nb[a];
  }
  g.bs[0] = 1;
  g.bs[1] = g.P[0];
  g.bs[2] = (int64_t)g.P[0] * g.P[1];
  g.nc = 1;
  const int64_t nblk = (int64_t)g.P[0] * g.P[1] * g.P[2];
  const int64_t n = nblk * B3;
  cx<double> *Y0 = nullptr, *Y1 = nullptr, *wP[3] = {nullptr, nullptr, nullptr};
  double *dc = nullptr, *ds = nullptr;
  auto fail = [&](int code, const char *what) {
    cudaFree(Y0);
    cudaFree(Y1);
    for (int a = 0; a < 3; ++a) cudaFree(wP[a]);
    cudaFree(dc);
    cudaFree(ds);
    cudaGetLastError();
    return set_error(code, "box spectrum: %s", what);
  };
  if (cudaMalloc(&Y0, sizeof(cx<double>) * n) || cudaMalloc(&Y1, sizeof(cx<double>) * n)) return fail(LGF_E_OOM, "scratch");
  if (cudaMalloc(&S->g64, sizeof(double) * n) || cudaMalloc(&S->g32, sizeof(float) * n) ||
      cudaMalloc(&S->gdf, sizeof(df) * n))
    return fail(LGF_E_OOM, "spectrum");
  S->bytes = n * (8 + 4 + 8);
  // per-axis tables: W_P (block DFT) and W_Pc (four-step twiddle)
  for (int a = 0; a < 3; ++a) {
    std::vector<double> c, s;
    twiddles_host(g.P[a], c, s);
    std::vector<cx<double>> w(g.P[a]);
    for (int i = 0; i < g.P[a]; ++i) w[i] = cx<double>{c[i], -s[i]};
    if (cudaMalloc(&wP[a], sizeof(cx<double>) * g.P[a])) return fail(LGF_E_OOM, "tables");
    cudaMemcpyAsync(wP[a], w.data(), sizeof(cx<double>) * g.P[a], cudaMemcpyHostToDevice, st);
    std::vector<double> cb, sb;
    twiddles_host(g.P[a], cb, sb);
    for (int i = 0; i < g.P[a] && i < 32; ++i) {
      S->bw64[a][i] = cx<double>{cb[i], -sb[i]};
      S->bw32[a][i] = cx<float>{(float)cb[i], -(float)sb[i]};
      const float hr = (float)cb[i], hi = (float)(-sb[i]);
      S->bwdf[a][i] = cx<df>{df{hr, (float)(cb[i] - (double)hr)}, df{hi, (float)(-sb[i] - (double)hi)}};
    }
  }
  // four-step twiddle table W_L^n, L = lcm of the three lattice periods Pc = P B
  {
    const int Pc[3] = {g.P[0] * B, g.P[1] * B, g.P[2] * B};
    const int L = std::lcm(std::lcm(Pc[0], Pc[1]), Pc[2]);
    S->twL = L;
    for (int a = 0; a < 3; ++a) S->twf[a] = L / Pc[a];
    std::vector<double> c, s;
    twiddles_host(L, c, s);
    if (cudaMalloc(&dc, sizeof(double) * L) || cudaMalloc(&ds, sizeof(double) * L)) return fail(LGF_E_OOM, "tables");
    if (cudaMalloc(&S->twl64, sizeof(cx<double>) * L) || cudaMalloc(&S->twl32, sizeof(cx<float>) * L) ||
        cudaMalloc(&S->twldf, sizeof(cx<df>) * L))
      return fail(LGF_E_OOM, "tables");
    cudaMemcpyAsync(dc, c.data(), sizeof(double) * L, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ds, s.data(), sizeof(double) * L, cudaMemcpyHostToDevice, st);
    k_tw_convert<<<(L + 127) / 128, 128, 0, st>>>(dc, ds, L, S->twl64, S->twl32, S->twldf);
    cudaStreamSynchronize(st);
    cudaFree(dc);
    cudaFree(ds);
    dc = ds = nullptr;
    S->bytes += (size_t)L * (16 + 8 + 16);
  }
  // dense block-index DFTs of the embedded LGF: x (from G), y, z
  const dim3 blk(256);
  const unsigned gx = (B3 + 255) / 256;
  k_bdft_dense<B><<<dim3(gx, g.P[1] * g.P[2]), blk, 0, st>>>(nullptr, Y0, g, 0, wP[0], t->Gd, t->N + 1);
  k_bdft_dense<B><<<dim3(gx, g.P[0] * g.P[2]), blk, 0, st>>>(Y0, Y1, g, 1, wP[1], nullptr, 0);
  k_bdft_dense<B><<<dim3(gx, g.P[0] * g.P[1]), blk, 0, st>>>(Y1, Y0, g, 2, wP[2], nullptr, 0);
  const size_t sm = sizeof(cx<double>) * (size_t)B * B * (B + 1);
  cudaFuncSetAttribute(k_box_mid<double, B, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_box_mid<double, B, false><<<dim3((unsigned)nblk, 1), mid_threads<double, B>(), sm, st>>>(
      Y0, 0, nullptr, g, S->twl64, S->twL, make_int3(S->twf[0], S->twf[1], S->twf[2]), make_tw64<double>(), S->g64);
  k_spec_convert<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S->g64, n, S->g32, S->gdf);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(Y0);
  cudaFree(Y1);
  for (int a = 0; a < 3; ++a) cudaFree(wP[a]);
  Y0 = Y1 = nullptr;
  wP[0] = wP[1] = wP[2] = nullptr;
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return set_error(LGF_E_CUDA, "box spectrum kernels failed: %s", cudaGetErrorString(e));
  return tc_matrices(S, g, st);
}

int box_spectrum(lgf_table *t, const int nb[3], BoxSpec **out, cudaStream_t st) {
  for (int a = 0; a < 3; ++a) {
    if (nb[a] < 1 || nb[a] > BOX_NB_MAX)
      return set_error(LGF_E_UNSUPPORTED, "box mode supports 1..%d blocks per axis (got %d)", BOX_NB_MAX, nb[a]);
    if (nb[a] * t->B > t->N)
      return set_error(LGF_E_TABLE_RANGE, "box of %d blocks along axis %d exceeds the table's LGF extent", nb[a], a);
  }
  std::lock_guard<std::mutex> g(t->mu);
  const auto key = std::make_tuple(nb[0], nb[1], nb[2]);
  auto it = t->box.find(key);
  if (it != t->box.end()) {
    *out = it->second;
    return LGF_OK;
  }
  BoxSpec *S = new BoxSpec();
  for (int a = 0; a < 3; ++a) S->nb[a] = nb[a];
  int rc = t->B == 8 ? gen_spectrum<8>(t, S, st) : gen_spectrum<16>(t, S, st);
  if (rc) {
    delete S;
    return rc;
  }
  t->box[key] = S;
  *out = S;
  return LGF_OK;
}

}  // namespace lgf
