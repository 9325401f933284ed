// internal.h -- declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lgf.h"
#include "common.cuh"

namespace lgf {

int set_error(int code, const char *fmt, ...);
int check_slices(const lgf_solve_opts &o);
int check_mesh(const lgf_mesh *m, int B_expected);

// Twiddles W_64^j from long-double cos/sin of the first octant and exact symmetries.
template <class R>
inline R tw_from_double(double v);
template <>
inline double tw_from_double<double>(double v) { return v; }
template <>
inline float tw_from_double<float>(double v) { return (float)v; }
template <>
inline df tw_from_double<df>(double v) {
  float h = (float)v;
  return df{h, (float)(v - (double)h)};
}

inline void tw64_double(double *c, double *s) {
  const long double pi = 3.141592653589793238462643383279502884L;
  double cq[17], sq[17];
  for (int j = 0; j <= 16; ++j) {
    cq[j] = (double)cosl(2.0L * pi * (long double)j / 64.0L);
    sq[j] = (double)sinl(2.0L * pi * (long double)j / 64.0L);
  }
  cq[16] = 0.0;
  sq[16] = 1.0;
  cq[0] = 1.0;
  sq[0] = 0.0;
  for (int j = 0; j < 64; ++j) {
    const int q = j / 16, r = j % 16;
    double cr = cq[r], sr = sq[r];
    switch (q) {
      case 0: c[j] = cr; s[j] = sr; break;
      case 1: c[j] = -sr; s[j] = cr; break;
      case 2: c[j] = -cr; s[j] = -sr; break;
      default: c[j] = sr; s[j] = -cr; break;
    }
  }
}

template <class R>
inline Tw64<R> make_tw64() {
  double c[64], s[64];
  tw64_double(c, s);
  Tw64<R> t;
  for (int j = 0; j < 64; ++j) {
    t.c[j] = tw_from_double<R>(c[j]);
    t.s[j] = tw_from_double<R>(s[j]);
  }
  return t;
}

// table.cu
int build_lgf_octant(int N, double **Gd_out, cudaStream_t st, double *quad_T, int *quad_nodes);
int build_spectra(int B, const double *Gd, int K, int3 mo, int noff, void *s64, void *s32, void *sdf,
                  cudaStream_t st);

// pair_*.cu: launch wrappers, one instantiation per arithmetic
template <class R>
struct PairOps {
  // spectra of the zero-padded blocks src_idx[i] of f ([ncomp][*][B^3], dtype code of load_field),
  // cells masked by cellmask & bits when cellmask != null; out [ncomp][nsrc][W]
  static int forward(int B, const void *f, int dtype, int64_t comp_stride, const int32_t *src_idx, int nsrc,
                     int ncomp, void *spec, const uint8_t *cellmask, int bits, cudaStream_t st);
  // see k_block_inv
  static int inverse(int B, const void *spec, int64_t spec_cs, const int32_t *rows, const int32_t *aux, int n,
                     int ncomp, void *out, int dtype, int64_t out_cs, int64_t out_off, const void *addend,
                     int64_t add_cs, const uint8_t *cellmask, int bits, double scale, cudaStream_t st);
  // see k_mac_pair; strides in complex elements
  static int mac(int B, const void *F, int nsrc, int64_t f_cs, const int32_t *src_list, const int4 *src_coords,
                 const void *Gh, int3 mo, void *Phi, int ntgt, int64_t p_cs, const int32_t *tgt_list,
                 const int4 *tgt_coords, int ncomp, int accumulate, cudaStream_t st);
};

// Kernel spectrum and twiddles of the block-index FFT mode for one box shape (box_spec.cu).
#define TC_SMAX 6  // most digit slices of the tensor-core DFT-GEMM

// Digit planes of one block-index DFT pass's coefficient matrix for the tensor-core path (box_tc.cuh):
// M^T with Np rows (real output columns 2o + re/im) and Kp columns (real inputs 2j + re/im), bf16 bit
// patterns in 8 x 8 core-matrix order, TC_SMAX planes `plane16` 16-byte units apart.
struct TcMat {
  const uint16_t *d = nullptr;
  int nin = 0, nout = 0;  // complex inputs and outputs of the pass
  int Kp = 0, Np = 0;     // GEMM K and N, multiples of 16
  float sigma = 1.0f;     // power-of-two scale of the coefficient digits
  int plane16 = 0;
};

struct BoxSpec {
  int nb[3] = {0, 0, 0};
  double *g64 = nullptr;  // [P^3 blocks][B^3] real spectrum, FP64
  float *g32 = nullptr;
  df *gdf = nullptr;
  // four-step twiddles: W_L^n, n < L = lcm(Pcx, Pcy, Pcz) (Pc = P B cells per axis); the twiddle of a
  // cell m and block frequency K1 is W_L^{(sum_a m_a K1_a L / Pc_a) mod L}
  cx<double> *twl64 = nullptr;
  cx<float> *twl32 = nullptr;
  cx<df> *twldf = nullptr;
  int twL = 0;
  int twf[3] = {0, 0, 0};  // L / Pc_a
  cx<double> bw64[3][32];  // W_P^n per axis, n < P (host copies for kernel parameters)
  cx<float> bw32[3][32];
  cx<df> bwdf[3][32];
  uint16_t *tcw = nullptr;  // device storage of the tensor-core coefficient digits
  TcMat tcm[3][3];          // per axis: forward, inverse, Hermitian-folded real inverse (axis 0 only)
  size_t bytes = 0;
  ~BoxSpec();
};

// Growable device buffer (never shrinks; freed with the owner).
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  int reserve(size_t n) {
    if (n <= bytes) return LGF_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      return set_error(LGF_E_OOM, "device allocation of %zu bytes failed", n);
    }
    bytes = n;
    return LGF_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

// Per-stream scratch held by a table.
struct Workspace {
  DevBuf buf[24];
  size_t total() const {
    size_t s = 0;
    for (auto &b : buf) s += b.bytes;
    return s;
  }
};

}  // namespace lgf

namespace lgf {
int box_spectrum(lgf_table *t, const int nb[3], BoxSpec **out, cudaStream_t st);
// Synchronous read of the table's device status word; LGF_E_TIMEOUT (and the word cleared) when a
// bounded device-side wait gave up since the last read.
int take_device_status(lgf_table *t);
}

struct lgf_table {
  int B = 0;
  int3 mo{0, 0, 0};  // max block offset per axis
  int noff = 0;
  int N = 0;         // lattice octant extent: G on [0, N]^3
  double quad_T = 0.0;
  int quad_nodes = 0;
  unsigned flags = 0;
  int device = 0;
  double *Gd = nullptr;        // [N+1]^3 octant, FP64
  void *s64 = nullptr;         // [noff][W] cx<double>
  void *s32 = nullptr;         // [noff][W] cx<float>
  void *sdf = nullptr;         // [noff][W] cx<df>
  std::mutex mu;
  std::map<void *, lgf::Workspace *> ws;  // keyed by stream
  std::map<std::tuple<int, int, int>, lgf::BoxSpec *> box;  // block-index FFT spectra by box shape
  int *d_status = nullptr;  // device status word: nonzero after a bounded device wait gave up
};
