// box_tc.cuh -- block-index DFT passes of the block-index FFT mode as tensor-core GEMMs (BF16 operands,
// FP32 accumulation) with split-precision "digit slices" that restore FP32 or double-float accuracy.
//
// A pass along one axis maps, for every line and local cell m, nin complex values x_j to nout complex
// values y_o = sum_j C_jo x_j (C = W_P^{+-jo}; the Hermitian-folded real inverse weighs and keeps the real
// part only).  Over the 128 cells of a tile this is a real GEMM
//     Y[128 x 2 nout] = X[128 x 2 nin] * M[2 nin x 2 nout],   X[., 2j + q] = (Re, Im)_q x_j,
// with M[2j, 2o] = Re C, M[2j + 1, 2o] = -Im C, M[2j, 2o + 1] = Im C, M[2j + 1, 2o + 1] = Re C.
//
// Split precision (Ozaki-style): each row of X is scaled by a power of two 2^{7-e} (max |x| < 2^e) and
// cut into S signed integer digits x = 2^{e-7} sum_t d_t 2^{-8t}, |d_t| <= 128; M is cut the same way
// with the fixed scale sigma (M = sigma 2^{-7} sum_u c_u 2^{-8u}).  Digits are exact in BF16, each product
// d_t c_u is an integer of at most 2^14, and the level sums D_l = sum_{t+u=l} sum_k d_t c_u stay below
// 2^23: the FP32 tensor-core accumulation of every level is exact.  The levels l < S are kept (the
// dropped ones are below 2^{-(7+8(S-1))} of the row's largest value) and recombined on the CUDA cores
//     y = sigma 2^{e-14} sum_l D_l 2^{-8l}
// in the arithmetic R of the surrounding pipeline (FP32 or double-float).  S = 3 matches FP32,
// S = 5 or 6 double-float; S = 1 is a plain BF16 GEMM with FP32 accumulation.
#pragma once
#include "box.cuh"
#include "tc.cuh"

#include "internal.h"

#define TC_ROWS 128    // cells per tile = MMA M

namespace lgf {

// Row digits: v * s = sum_t d_t 2^{-8t} (+ dropped remainder), |d_t| <= 128, for a float value.
template <int S>
LGF_D void tc_digits(float v, float s, float (&d)[S]) {
  float r = __fmul_rn(v, s);
#pragma unroll
  for (int t = 0; t < S; ++t) {
    d[t] = rintf(r);
    r = __fmul_rn(__fsub_rn(r, d[t]), 256.0f);
  }
}
// The same for a double-float value hi + lo.  r_hi - d is exact (a multiple of ulp(r_hi), at most 1/2),
// and when nonzero it is at least ulp(r_hi) >= 2 |r_lo|, so a fast two-sum renormalises the remainder.
template <int S>
LGF_D void tc_digits(df v, float s, float (&d)[S]) {
  float rh = __fmul_rn(v.hi, s), rl = __fmul_rn(v.lo, s);
#pragma unroll
  for (int t = 0; t < S; ++t) {
    d[t] = rintf(rh);
    const float x = __fsub_rn(rh, d[t]);
    const float h = __fadd_rn(x, rl);
    const float l = __fsub_rn(rl, __fsub_rn(h, x));
    rh = __fmul_rn(h, 256.0f);
    rl = __fmul_rn(l, 256.0f);
  }
}
LGF_D float tc_absmax(float v) { return fabsf(v); }
LGF_D float tc_absmax(df v) { return fabsf(v.hi); }

// Recombination of the level sums: acc = sum_l D_l 2^{-8l} by Horner from the smallest level.
LGF_D void tc_horner(float &acc, float D) { acc = __fmaf_rn(acc, 0.00390625f, D); }
LGF_D void tc_horner(df &acc, float D) {
  const float ah = __fmul_rn(acc.hi, 0.00390625f), al = __fmul_rn(acc.lo, 0.00390625f);
  const float s = __fadd_rn(D, ah);
  const float bb = __fsub_rn(s, D);
  float e = __fadd_rn(__fsub_rn(D, __fsub_rn(s, bb)), __fsub_rn(ah, bb));
  e = __fadd_rn(e, al);
  const float h = __fadd_rn(s, e);
  acc = df{h, __fsub_rn(e, __fsub_rn(h, s))};
}
LGF_D void tc_init(float &acc, float D) { acc = D; }
LGF_D void tc_init(df &acc, float D) { acc = df{D, 0.0f}; }
LGF_D float tc_scale(float a, float f) { return __fmul_rn(a, f); }
LGF_D df tc_scale(df a, float f) { return df_scale2(a, f); }

// Shared-memory plan of one launch (bytes): digit planes of X (S x 128 x Kp bf16), of M^T (S x Np x Kp),
// then the mbarrier, the TMEM base address and the abort flag.
struct TcSmem {
  int a_off, a_plane, b_off, b_plane, bar_off, total;
};
inline TcSmem tc_smem_plan(int S, int Kp, int Np) {
  TcSmem p;
  p.a_plane = TC_ROWS * Kp * 2;
  p.a_off = 0;
  p.b_plane = Np * Kp * 2;
  p.b_off = S * p.a_plane;
  p.bar_off = (p.b_off + S * p.b_plane + 15) & ~15;
  p.total = p.bar_off + 32;
  return p;
}

}  // namespace lgf

// One pass.  Persistent CTAs of 128 threads (thread = row = cell of the tile) over tiles (field, line,
// 128-cell chunk).  Per tile: load the rows and cut them into digits (shared memory); one thread issues
// the S(S+1)/2 x Kp/16 MMAs (M = 128, N = Np, K = 16) into S level accumulators in TMEM and commits to
// the mbarrier; all threads wait, read the levels back, recombine and store.  Several CTAs share an SM
// (their phases overlap); each holds `tmem_cols` >= S Np columns.
// A wait that runs out (about a second) sets *status = 1 and the CTA drains, frees its TMEM and stops.
template <class R, int B, int S>
__global__ void __launch_bounds__(TC_ROWS) k_bdft_tc(const cx<R> *__restrict__ in, cx<R> *__restrict__ out,
                                                     int64_t fstride, BoxGeom g, int ax, int3 ext, lgf::TcMat M,
                                                     int gather, int final, int nfield, int lines, FwdSpecs sp,
                                                     InvOuts<R> outs, double scale, uint32_t tmem_cols,
                                                     lgf::TcSmem pl, int *status) {
  using namespace lgf;
  constexpr int B3 = B * B * B;
  constexpr int NCH = B3 / TC_ROWS;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + pl.bar_off);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + pl.bar_off + 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + pl.bar_off + 12);
  const int row = threadIdx.x, warp = threadIdx.x >> 5;
  const int nin = M.nin, nout = M.nout, Kp = M.Kp, Np = M.Np;
  const int kg = Kp / 8;  // 16-byte K groups per row
  const uint32_t sbo = (uint32_t)kg * 128u;

  {  // coefficient digit planes: the same for every tile
    const uint4 *src = reinterpret_cast<const uint4 *>(M.d);
    uint4 *dst = reinterpret_cast<uint4 *>(smem + pl.b_off);
    const int per = pl.b_plane / 16;
    for (int i = threadIdx.x; i < S * per; i += blockDim.x) dst[i] = src[(int64_t)(i / per) * M.plane16 + i % per];
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(bar, 1);
    *abort_flag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tslot, tmem_cols);
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;

  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
  const int e1 = ax == 0 ? ext.y : ext.x;
  const int64_t bsa = geo_bs(g, ax) * (int64_t)B3;
  const int gsa = ax == 0 ? 1 : (ax == 1 ? g.nb[0] : g.nb[0] * g.nb[1]);
  const int gs1 = a1 == 0 ? 1 : g.nb[0];
  const int gs2 = a2 == 1 ? g.nb[0] : g.nb[0] * g.nb[1];
  const int ntiles = nfield * lines * NCH;
  const uint32_t idesc = tc::idesc_bf16_f32(TC_ROWS, Np);
  const uint32_t a_base = tc::smem_addr(smem + pl.a_off), b_base = tc::smem_addr(smem + pl.b_off);
  const R sc = RT<R>::from(scale);

  for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
    const int chunk = tile % NCH, line = (tile / NCH) % lines, field = tile / (NCH * lines);
    const int l1 = line % e1, l2 = line / e1;
    const int pxf = box_pxu(g, field);
    if (ax != 0 && l1 >= pxf) continue;  // beyond this field's K1x range (uniform over the CTA)
    const bool realx = ax == 0 && pxf < g.P[0];
    const int64_t lbase = ((int64_t)l1 * geo_bs(g, a1) + (int64_t)l2 * geo_bs(g, a2)) * B3;
    const int gbase = l1 * gs1 + l2 * gs2;
    const int m = chunk * TC_ROWS + row;
    InSpec s0{}, s1{}, s2{};
    int ns = 0;
    OutSpec<R> ore{}, oim{};
#pragma unroll
    for (int f = 0; f < BOX_MAXF; ++f)
      if (f == field) {
        if (gather) {
          s0 = sp.s[f][0];
          s1 = sp.s[f][1];
          s2 = sp.s[f][2];
          ns = sp.n[f];
        }
        if (final) {
          ore = outs.re[f];
          oim = outs.im[f];
        }
      }
    const cx<R> *src = in + field * fstride + lbase;
    auto load = [&](int j) -> cx<R> {
      if (!gather) return src[j * bsa + m];
      const int bidx = gbase + j * gsa;
      R re = RT<R>::zero(), im = RT<R>::zero();
      auto add = [&](const InSpec &q) {
        const int idx = q.gather[bidx];
        if (idx < 0) return;
        const int64_t e = (int64_t)idx * B3 + m;
        if (q.mask && !(q.mask[e] & q.bits)) return;
        const R v = load_field<R>(q.src, e, q.dtype);
        if (q.part) im = im + v;
        else re = re + v;
      };
      if (ns > 0) add(s0);
      if (ns > 1) add(s1);
      if (ns > 2) add(s2);
      return cx<R>{re, im};
    };
    // ---- digits of the row.  Row scale max |x| < 2^e; e >= -100 keeps 2^{7-e} finite for rows of
    // denormal size (their digits then follow a looser scale: absolute error below 2^-(100+7+8(S-1))).
    unsigned char *arow = smem + pl.a_off + (row >> 3) * sbo + (row & 7) * 16;
    int e = 0;
    auto put_group = [&](int grp, const cx<R> (&x)[4], int nq, float sdown) {
      uint32_t w[S][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float dr[S], di[S];
        if (q < nq) {
          tc_digits<S>(x[q].re, sdown, dr);
          tc_digits<S>(x[q].im, sdown, di);
        } else {
#pragma unroll
          for (int t = 0; t < S; ++t) dr[t] = di[t] = 0.0f;
        }
#pragma unroll
        for (int t = 0; t < S; ++t) w[t][q] = __byte_perm(__float_as_uint(dr[t]), __float_as_uint(di[t]), 0x7632);
      }
#pragma unroll
      for (int t = 0; t < S; ++t)
        *reinterpret_cast<uint4 *>(arow + t * pl.a_plane + grp * 128) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    };
    {
      // two passes over groups of four inputs (max, then digits; the second mostly hits L1), the four
      // loads of a group issued back to back
      float mx = 0.0f;
      for (int j0 = 0; j0 < nin; j0 += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j0 + q < nin) {
            const cx<R> v = load(j0 + q);
            mx = fmaxf(mx, fmaxf(tc_absmax(v.re), tc_absmax(v.im)));
          }
      }
      if (mx > 0.0f) frexpf(mx, &e);
      e = max(e, -100);
      const float sdown = ldexpf(1.0f, 7 - e);
#pragma unroll 1
      for (int grp = 0; grp < kg; ++grp) {
        cx<R> xs[4];
        const int nq = min(4, max(0, nin - 4 * grp));
#pragma unroll
        for (int q = 0; q < 4; ++q) xs[q] = q < nq ? load(4 * grp + q) : cx_zero<R>();
        put_group(grp, xs, nq, sdown);
      }
    }
    const float fsc = ldexpf(M.sigma, e - 14);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- MMAs of all S levels over the Np output columns, then recombination 16 columns at a time
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      for (int l = 0; l < S; ++l) {
        uint32_t acc = 0;
        for (int t = 0; t <= l; ++t) {
          const uint32_t ab = a_base + t * pl.a_plane, bb = b_base + (l - t) * pl.b_plane;
          for (int ks = 0; ks < kg / 2; ++ks) {
            tc::mma_bf16(tbase + (uint32_t)(l * Np), tc::smem_desc(ab + ks * 256, 128, sbo),
                         tc::smem_desc(bb + ks * 256, 128, sbo), idesc, acc);
            acc = 1;
          }
        }
      }
      tc::mma_commit(bar);
    }
    if (!tc::mbar_wait_or_abort(bar, phase, abort_flag)) break;
    phase ^= 1u;
    tc::fence_after_sync();
    for (int c0 = 0; c0 < 2 * nout; c0 += 16) {
      R acc[16];
      float v[16];
      tc::tmem_ld16(lane_base + (uint32_t)((S - 1) * Np + c0), v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < 16; ++k) tc_init(acc[k], v[k]);
#pragma unroll
      for (int l = S - 2; l >= 0; --l) {
        tc::tmem_ld16(lane_base + (uint32_t)(l * Np + c0), v);
        tc::tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) tc_horner(acc[k], v[k]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int o = c0 / 2 + k;
        if (o >= nout) break;
        const cx<R> y{tc_scale(acc[2 * k], fsc), tc_scale(acc[2 * k + 1], fsc)};
        if (!final) {
          out[field * fstride + lbase + o * bsa + m] = y;
        } else {
          const int bidx = gbase + o * gsa;
          box_store<R>(ore, bidx, m, B3, y.re * sc);
          if (!realx) box_store<R>(oim, bidx, m, B3, y.im * sc);
        }
      }
    }
    // the next tile's MMAs overwrite the accumulators once every thread has read them
    tc::fence_before_sync();
    __syncthreads();
  }
  // drain: `bar` flips once every MMA issued so far has completed (bounded)
  if (threadIdx.x == 0) {
    tc::mma_commit(bar);
    tc::mbar_wait_bounded(bar, phase);
  }
  if (*abort_flag && threadIdx.x == 0) atomicExch(status, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, tmem_cols);
}
