// indicator.cuh -- refinement indicator of the adaptive mesh (Sec. 4.2, Eqs. (eq:refine1), (eq:maximumS),
// (eq:refine2)) from the combined source S_k of Eq. (eq:combined_source), reduced on the device while the
// FLGF-AMR solve runs.
//
//   S_k = A_k + [covered] F_k,   A_k = [Omega_k] fhat_k + [Omega_k u Omega_k^E] S psi_{k-1} (k_correct)
//
// i.e. the correction source on Omega_k u Omega_k^E plus every source of level k and finer coarsened onto
// it (F_k = fhat_k on Omega_k, the coarsened finer sources on covered cells).  For a vector source |S_k| is
// the Euclidean norm over the components.
//   k_ind_stats  per internal block of a level: sum of |S_k|^2 and max |S_k| over all B^3 cells of a caller
//                block; over the Omega_k^E cells of a block outside the caller's blocks, max |S_k|
//   k_ind_flags  one CTA: S_max = max(previous S_max, largest block RMS), thresholds
//                alpha^(N_l - k) S_max, refine / coarsen flags per caller block, and the refine flag that an
//                Omega_k^E cell above the level-k threshold raises on the level-(k-1) block under it.
#pragma once
#include "amr.cuh"

#define LGF_IND_MAX_LEVELS 16

// grid (nBL of the level), 256 threads.  A is read only on blocks holding Omega_k or Omega_k^E cells (the
// blocks k_correct wrote); F only on covered cells (which lie in caller blocks).
template <class R>
__global__ void __launch_bounds__(256) k_ind_stats(LevelDev L, int nU, int ncomp, const R *A, const R *F, int64_t cs,
                                                   double *sumsq, double *smax) {
  constexpr uint8_t OM = 1, EX = 2, COV = 4;
  const int b = blockIdx.x, sh = L.shift, B = 1 << sh, B3 = B * B * B;
  const uint8_t *cm = L.cellmask + (int64_t)b * B3;
  int any = 0;
  for (int off = threadIdx.x; off < B3; off += blockDim.x) any |= (cm[off] & (OM | EX)) != 0;
  const int has_a = __syncthreads_or(any);
  const bool user = b < nU;
  double ss = 0.0, mx = 0.0;
  if (user || has_a) {
    for (int off = threadIdx.x; off < B3; off += blockDim.x) {
      const uint8_t c = cm[off];
      if (!user && !(c & EX)) continue;  // outside the caller's blocks only Omega_k^E counts
      double s2 = 0.0;
      for (int comp = 0; comp < ncomp; ++comp) {
        const int64_t i = comp * cs + (int64_t)b * B3 + off;
        double v = has_a ? RT<R>::to_d(A[i]) : 0.0;
        if (c & COV) v += RT<R>::to_d(F[i]);
        s2 += v * v;
      }
      ss += s2;
      mx = fmax(mx, s2);
    }
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[0][w] = ss, red[1][w] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, m = 0.0;
    for (int i = 0; i < nw; ++i) a += red[0][i], m = fmax(m, red[1][i]);
    sumsq[b] = a;
    smax[b] = sqrt(m);
  }
}

struct IndLevel {
  LevelDev L;
  const int4 *BL;        // internal block coordinates
  int nBL, nU;           // internal blocks, caller blocks (the first nU internal blocks)
  int64_t uoff;          // first caller block of the level in the caller's arrays
  const double *sumsq;   // [nBL] from k_ind_stats
  const double *smax;
};
struct IndArgs {
  IndLevel lv[LGF_IND_MAX_LEVELS];
  int K, B3, nlmax;
  double alpha, beta;
};

// one CTA of 1024 threads; pref: [caller blocks] scratch; s_max_io: in the previous S_max, out the new one
__global__ void __launch_bounds__(1024) k_ind_flags(IndArgs a, double *rms, uint8_t *flags, double *s_max_io,
                                                    int *pref) {
  __shared__ double red[32];
  const int t = threadIdx.x, nt = blockDim.x;
  double m = 0.0;
  for (int k = 0; k < a.K; ++k) {
    const IndLevel &l = a.lv[k];
    for (int i = t; i < l.nU; i += nt) {
      m = fmax(m, sqrt(l.sumsq[i] / (double)a.B3));
      pref[l.uoff + i] = 0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((t & 31) == 0) red[t >> 5] = m;
  __syncthreads();
  double smx = s_max_io[0];
  for (int i = 0; i < (nt >> 5); ++i) smx = fmax(smx, red[i]);
  // Omega_k^E cells outside the level-k blocks flag the level-(k-1) caller block under them
  for (int k = 1; k < a.K; ++k) {
    const IndLevel &l = a.lv[k], &lc = a.lv[k - 1];
    const double thr = pow(a.alpha, (double)(a.nlmax - k)) * smx;
    for (int i = l.nU + t; i < l.nBL; i += nt) {
      if (!(l.smax[i] > thr)) continue;
      const int4 c = l.BL[i];
      const int p = level_block(lc.L, c.x >> 1, c.y >> 1, c.z >> 1);
      if (p >= 0 && p < lc.nU) pref[lc.uoff + p] = 1;
    }
  }
  __syncthreads();
  for (int k = 0; k < a.K; ++k) {
    const IndLevel &l = a.lv[k];
    const double thr = pow(a.alpha, (double)(a.nlmax - k)) * smx;
    for (int i = t; i < l.nU; i += nt) {
      const int64_t g = l.uoff + i;
      rms[g] = sqrt(l.sumsq[i] / (double)a.B3);
      uint8_t fl = 0;
      if (l.smax[i] > thr || pref[g]) fl |= 1;
      if (l.smax[i] < a.beta * thr) fl |= 2;
      flags[g] = fl;
    }
  }
  if (t == 0) s_max_io[0] = smx;
}
