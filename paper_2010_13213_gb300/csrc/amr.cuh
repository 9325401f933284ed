// amr.cuh -- stencil kernels of the composite-mesh path (Sec. 3.2-3.5), templated on the arithmetic.
//
//   k_restrict   F_k = [Omega_k] fhat_k + [covered] mean of the 8 children of F_{k+1}
//                (cumulative coarsening, step 1 of FLGF-AMR)
//   k_interp     c_k = P_{k-1->k} psi_{k-1}: cell-centred tensor-product linear interpolation
//   k_correct    A_k = [Omega_k] fhat_k + [Omega_k u Omega_k^E] (P L_{k-1} psi_{k-1} - L_k c_k)
//                (the commutation source correction S psi_{k-1}, Eq. (eq:source_correct))
//   k_residual   FP64 max |L_k phi^k - F_k - P L_{k-1} psi_{k-1}| over interior Omega_k cells
//   k_heat_*     FIF-AMR: P_k fhat and the separable discrete heat kernel (Sec. 3.5)
// Fields are stored per level as [ncomp][nBL][B^3] over the level's internal block set; a dense
// block map (block coords -> index, -1 if absent) gives neighbours across block boundaries.
#pragma once
#include "common.cuh"

struct LevelDev {
  const int32_t *map;      // [n.z][n.y][n.x] block map
  int3 lo, n;              // block-coordinate box of the map
  const uint8_t *cellmask; // [nBL][B^3] CellBits
  const int32_t *user_of;  // [nBL] caller block index or -1
  int shift;               // log2(B)
  double h;                // level spacing
};

LGF_D int level_block(const LevelDev &L, int bx, int by, int bz) {
  bx -= L.lo.x;
  by -= L.lo.y;
  bz -= L.lo.z;
  if ((unsigned)bx >= (unsigned)L.n.x || (unsigned)by >= (unsigned)L.n.y || (unsigned)bz >= (unsigned)L.n.z)
    return -1;
  return L.map[((int64_t)bz * L.n.y + by) * L.n.x + bx];
}

// Cell (gx, gy, gz) of a level -> (block index, offset inside the block); false if absent.
LGF_D bool level_cell(const LevelDev &L, int gx, int gy, int gz, int &blk, int &off) {
  const int B = 1 << L.shift, m = B - 1;
  blk = level_block(L, gx >> L.shift, gy >> L.shift, gz >> L.shift);
  off = (((gz & m) << L.shift) + (gy & m)) * B + (gx & m);
  return blk >= 0;
}

template <class R>
LGF_D R nan_of() {
  return RT<R>::from(__longlong_as_double(0x7ff8000000000000ll));
}

// value of an internal field (R storage) at a level cell; NaN when the block is absent
template <class R>
LGF_D R fetch(const LevelDev &L, const R *buf, int64_t cs, int comp, int gx, int gy, int gz) {
  int blk, off;
  if (!level_cell(L, gx, gy, gz, blk, off)) return nan_of<R>();
  return buf[comp * cs + ((int64_t)blk << (3 * L.shift)) + off];
}

// 7-point Laplacian of an internal field at a level cell
template <class R>
LGF_D R lap7(const LevelDev &L, const R *buf, int64_t cs, int comp, int x, int y, int z, R inv_h2) {
  R c = fetch<R>(L, buf, cs, comp, x, y, z);
  R s = fetch<R>(L, buf, cs, comp, x + 1, y, z) + fetch<R>(L, buf, cs, comp, x - 1, y, z);
  s = s + fetch<R>(L, buf, cs, comp, x, y + 1, z) + fetch<R>(L, buf, cs, comp, x, y - 1, z);
  s = s + fetch<R>(L, buf, cs, comp, x, y, z + 1) + fetch<R>(L, buf, cs, comp, x, y, z - 1);
  return (s - RT<R>::from(6.0) * c) * inv_h2;
}

// The values of an internal field on block b and on the one-cell face halo around it, staged in shared
// memory as a (B + 2)^3 cube S[((z + 1) W + y + 1) W + x + 1] (W = B + 2, local x, y, z in [-1, B]; edges and
// corners are not written).  Halo cells of absent blocks are NaN, as fetch gives.
template <class R>
LGF_D void stage_block_halo(R *S, const LevelDev &L, const R *buf, int64_t cs, int comp, int b, int4 bc) {
  const int sh = L.shift, B = 1 << sh, W = B + 2, B2 = B * B, B3 = B2 * B;
  const R *src = buf + comp * cs;
  for (int t = threadIdx.x; t < B3; t += blockDim.x) {
    const int x = t & (B - 1), y = (t >> sh) & (B - 1), z = t >> (2 * sh);
    S[((z + 1) * W + y + 1) * W + x + 1] = src[((int64_t)b << (3 * sh)) + t];
  }
  for (int t = threadIdx.x; t < 6 * B2; t += blockDim.x) {
    const int f = t >> (2 * sh), a = f >> 1, hi = f & 1, u = t & (B - 1), v = (t >> sh) & (B - 1);
    const int e = hi ? B : -1;  // the face's coordinate along axis a
    const int x = a == 0 ? e : u, y = a == 1 ? e : (a == 0 ? u : v), z = a == 2 ? e : v;
    const int nb = level_block(L, bc.x + (a == 0 ? (hi ? 1 : -1) : 0), bc.y + (a == 1 ? (hi ? 1 : -1) : 0),
                               bc.z + (a == 2 ? (hi ? 1 : -1) : 0));
    R val = nan_of<R>();
    if (nb >= 0)
      val = src[((int64_t)nb << (3 * sh)) + ((((z & (B - 1)) << sh) + (y & (B - 1))) << sh) + (x & (B - 1))];
    S[((z + 1) * W + y + 1) * W + x + 1] = val;
  }
}
// 7-point Laplacian at local cell (x, y, z) of a staged cube (the same sums in the same order as lap7)
template <class R>
LGF_D R lap7_staged(const R *S, int W, int x, int y, int z, R inv_h2) {
  const int i = ((z + 1) * W + y + 1) * W + x + 1, W2 = W * W;
  R s = S[i + 1] + S[i - 1];
  s = s + S[i + W] + S[i - W];
  s = s + S[i + W2] + S[i - W2];
  return (s - RT<R>::from(6.0) * S[i]) * inv_h2;
}
template <class R>
LGF_HD constexpr size_t halo_smem(int B) { return sizeof(R) * (size_t)(B + 2) * (B + 2) * (B + 2); }

// P_{k-1->k}: fine cell (fx, fy, fz) -> sum over the 8 coarse corners of prod (3/4 | 1/4) * value.  The
// weights are 27, 9, 3 or 1 / 64 (exact floats); products and sums run lazily in double-float, with one
// renormalisation at the end.
template <class R, class F>
LGF_D R interp_at(int fx, int fy, int fz, F coarse_value) {
  const int px = fx >> 1, py = fy >> 1, pz = fz >> 1;
  const int qx = (fx & 1) ? px + 1 : px - 1;
  const int qy = (fy & 1) ? py + 1 : py - 1;
  const int qz = (fz & 1) ? pz + 1 : pz - 1;
  R acc = RT<R>::zero();
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cx = (c & 1) ? qx : px, cy = (c & 2) ? qy : py, cz = (c & 4) ? qz : pz;
    const int quarters = ((c & 1) != 0) + ((c & 2) != 0) + ((c & 4) != 0);  // factors 1/4 (the others 3/4)
    const float w = quarters == 0 ? 27.0f / 64 : (quarters == 1 ? 9.0f / 64 : (quarters == 2 ? 3.0f / 64 : 1.0f / 64));
    acc = radd(acc, rscale(coarse_value(cx, cy, cz), w));
  }
  return rnorm(acc);
}

// The coarse cells the interpolation of a fine block reads: parents (B c)/2 + [0, B/2) per axis and one
// more on each side, (B/2 + 2)^3 values staged in shared memory (NaN for absent blocks, as fetch gives).
#define LGF_STAGE_MAX 1000  // (16/2 + 2)^3
template <class R>
LGF_D void stage_coarse(R *S, const LevelDev &Lc, const R *buf, int64_t cs, int comp, int4 bc, int B) {
  const int H = B >> 1, W = H + 2;
  const int x0 = bc.x * H - 1, y0 = bc.y * H - 1, z0 = bc.z * H - 1;
  for (int t = threadIdx.x; t < W * W * W; t += blockDim.x)
    S[t] = fetch<R>(Lc, buf, cs, comp, x0 + t % W, y0 + (t / W) % W, z0 + t / (W * W));
}
// P_{k-1->k} at fine cell (x, y, z) of block bc from the staged coarse cube
template <class R>
LGF_D R interp_staged(const R *S, int4 bc, int B, int x, int y, int z) {
  const int H = B >> 1, W = H + 2;
  const int x0 = bc.x * H - 1, y0 = bc.y * H - 1, z0 = bc.z * H - 1;
  return interp_at<R>(x, y, z, [&](int i, int j, int k) { return S[((k - z0) * W + (j - y0)) * W + (i - x0)]; });
}

// The same interpolation for a whole fine block by separable passes over the staged cube (the weights
// 3/4, 1/4 per axis factor the 27, 9, 3, 1 / 64 of the eight corners): x into T1[W][W][B], y into
// T2[W][B][B] (each value renormalised), and z per cell by interp_sep_z.  Three terms' worth of work per
// fine cell instead of eight.  Called by every thread of the CTA (two barriers).
template <class R>
LGF_D void interp_sep_xy(const R *S, R *T1, R *T2, int sh) {
  const int B = 1 << sh, W = (B >> 1) + 2;
  for (int t = threadIdx.x; t < W * W * B; t += blockDim.x) {
    const int lx = t & (B - 1), kj = t >> sh;  // kj = kz W + jy
    const int ip = (lx >> 1) + 1, iq = (lx & 1) ? ip + 1 : ip - 1;
    const R *row = S + kj * W;
    T1[t] = rnorm(radd(rscale(row[ip], 0.75f), rscale(row[iq], 0.25f)));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < W * B * B; t += blockDim.x) {
    const int lx = t & (B - 1), ly = (t >> sh) & (B - 1), kz = t >> (2 * sh);
    const int ip = (ly >> 1) + 1, iq = (ly & 1) ? ip + 1 : ip - 1;
    const R *col = T1 + kz * W * B + lx;
    T2[t] = rnorm(radd(rscale(col[ip * B], 0.75f), rscale(col[iq * B], 0.25f)));
  }
  __syncthreads();
}
template <class R>
LGF_D R interp_sep_z(const R *T2, int sh, int lx, int ly, int lz) {
  const int ip = (lz >> 1) + 1, iq = (lz & 1) ? ip + 1 : ip - 1, o = (ly << sh) + lx;
  return rnorm(radd(rscale(T2[(ip << (2 * sh)) + o], 0.75f), rscale(T2[(iq << (2 * sh)) + o], 0.25f)));
}
// Values of T1 and T2 for a block size B
LGF_HD constexpr int interp_sep_values(int B) { return (B / 2 + 2) * (B / 2 + 2) * B + (B / 2 + 2) * B * B; }

// ------------------------------------------------------------------ restriction (step 1)
// grid (nU_k, ncomp), 256 threads.  F_k on the caller blocks of level k (BL index = caller index).
template <class R>
__global__ void __launch_bounds__(256) k_restrict(LevelDev L, const void *f_user, int dtype, int64_t ucs,
                                                  int64_t user_off, R *F, int64_t cs) {
  const int b = blockIdx.x, comp = blockIdx.y, B3 = 1 << (3 * L.shift);
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    const uint8_t cm = L.cellmask[(int64_t)b * B3 + off];
    R v = RT<R>::zero();
    if (cm & 1) v = load_field<R>(f_user, comp * ucs + (user_off + b) * (int64_t)B3 + off, dtype);
    F[comp * cs + (int64_t)b * B3 + off] = v;
  }
}

// coarsening part: for covered cells, F_k += mean of children.  One thread per level-(k+1) caller
// cell group: each fine caller block covers one octant of its parent; grid (nU_{k+1}, ncomp).
template <class R>
__global__ void __launch_bounds__(256) k_coarsen_add(LevelDev Lc, R *Fc, int64_t ccs, const int4 *fine_blocks,
                                                     const R *Ff, int64_t fcs) {
  const int fb = blockIdx.x, comp = blockIdx.y, sh = Lc.shift, B = 1 << sh, H = B >> 1;
  const int4 c = fine_blocks[fb];
  const int B3 = B * B * B;
  for (int t = threadIdx.x; t < H * H * H; t += blockDim.x) {
    const int x = t % H, y = (t / H) % H, z = t / (H * H);
    // coarse cell = (B c + 2 (x, y, z)) / 2
    const int gx = (c.x << (sh - 1)) + x, gy = (c.y << (sh - 1)) + y, gz = (c.z << (sh - 1)) + z;
    R s = RT<R>::zero();
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int lx = 2 * x + (d & 1), ly = 2 * y + ((d >> 1) & 1), lz = 2 * z + ((d >> 2) & 1);
      s = s + Ff[comp * fcs + (int64_t)fb * B3 + (lz * B + ly) * B + lx];
    }
    int blk, off;
    if (level_cell(Lc, gx, gy, gz, blk, off)) {
      R &d = Fc[comp * ccs + (int64_t)blk * B3 + off];
      d = d + RT<R>::from(0.125) * s;
    }
  }
}

// ------------------------------------------------------------------ interpolation c_k = P psi_{k-1}
// grid (nBL_k, ncomp), interp_sep_values(B) values of dynamic shared memory (the separable passes)
template <class R>
__global__ void __launch_bounds__(256) k_interp(LevelDev L, const int4 *blocks, R *c, int64_t cs, LevelDev Lc,
                                                const R *psi, int64_t pcs) {
  __shared__ R S[LGF_STAGE_MAX];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x, comp = blockIdx.y, sh = L.shift, B = 1 << sh;
  const int B3 = B * B * B, W = (B >> 1) + 2;
  R *T1 = reinterpret_cast<R *>(smem_raw), *T2 = T1 + W * W * B;
  stage_coarse<R>(S, Lc, psi, pcs, comp, blocks[b], B);
  __syncthreads();
  interp_sep_xy<R>(S, T1, T2, sh);
  for (int off = threadIdx.x; off < B3; off += blockDim.x)
    c[comp * cs + (int64_t)b * B3 + off] =
        interp_sep_z<R>(T2, sh, off & (B - 1), (off >> sh) & (B - 1), off >> (2 * sh));
}

// ------------------------------------------------------------------ coarse Laplacian L_{k-1} psi_{k-1}
// Every cell of the listed blocks of the coarse level (NaN next to an absent block, as fetch gives); grid
// (|list|, ncomp), 512 threads, halo_smem<R>(B) bytes of dynamic shared memory (the block and its face halo;
// 512 threads keep 2048 resident per SM at four CTAs).
template <class R>
__global__ void __launch_bounds__(512) k_lap(LevelDev L, const int4 *blocks, const int32_t *list, const R *psi,
                                             R *out, int64_t cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *S = reinterpret_cast<R *>(smem_raw);
  const int b = list[blockIdx.x], comp = blockIdx.y, sh = L.shift, B = 1 << sh;
  const int B3 = B * B * B;
  const R inv_h2 = RT<R>::from(1.0 / (L.h * L.h));
  stage_block_halo<R>(S, L, psi, cs, comp, b, blocks[b]);
  __syncthreads();
  for (int off = threadIdx.x; off < B3; off += blockDim.x)
    out[comp * cs + (int64_t)b * B3 + off] =
        lap7_staged<R>(S, B + 2, off & (B - 1), (off >> sh) & (B - 1), off >> (2 * sh), inv_h2);
}

// ------------------------------------------------------------------ correction source A_k
// grid (|SA_k|, ncomp), 512 threads.  A[b] for b = SA[i].  k = 0: A = [OM] fhat.  `lpsi` = L_{k-1} psi_{k-1}
// (k_lap).  With has_coarse: halo_smem<R>(B) bytes of dynamic shared memory (c on the block and its face halo).
// The interpolation of L_{k-1} psi_{k-1} stays per cell (eight staged corners, only on Omega u Omega^E cells):
// the separable passes of k_interp would add 33 KB per CTA and halve the resident CTAs (measured slower).
template <class R>
__global__ void __launch_bounds__(512) k_correct(LevelDev L, const int4 *blocks, const int32_t *SA,
                                                 const void *f_user, int dtype, int64_t ucs, R *A, int64_t cs,
                                                 const R *c, LevelDev Lc, const R *lpsi, int64_t pcs,
                                                 int has_coarse) {
  __shared__ R S[LGF_STAGE_MAX];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *C = reinterpret_cast<R *>(smem_raw);
  const int b = SA[blockIdx.x], comp = blockIdx.y, sh = L.shift, B = 1 << sh;
  const int B3 = B * B * B;
  const int4 bc = blocks[b];
  const int u = L.user_of[b];
  const R inv_h2f = RT<R>::from(1.0 / (L.h * L.h));
  if (has_coarse) {
    stage_coarse<R>(S, Lc, lpsi, pcs, comp, bc, B);
    stage_block_halo<R>(C, L, c, cs, comp, b, bc);
    __syncthreads();
  }
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    const uint8_t cm = L.cellmask[(int64_t)b * B3 + off];
    R v = RT<R>::zero();
    if ((cm & 1) && u >= 0) v = load_field<R>(f_user, comp * ucs + (int64_t)u * B3 + off, dtype);
    if (has_coarse && (cm & 3)) {
      const int lx = off & (B - 1), ly = (off >> sh) & (B - 1), lz = off >> (2 * sh);
      const R plp = interp_staged<R>(S, bc, B, (bc.x << sh) + lx, (bc.y << sh) + ly, (bc.z << sh) + lz);
      const R lpc = lap7_staged<R>(C, B + 2, lx, ly, lz, inv_h2f);
      v = v + (plp - lpc);
    }
    A[comp * cs + (int64_t)b * B3 + off] = v;
  }
}

// ------------------------------------------------------------------ FP64 residual
// grid (|Tphi_k|, ncomp).  r = L_k phi - F_k - [k >= 1] P L_{k-1} psi_{k-1} at Omega_k cells whose six
// neighbours are Omega_k cells; out[0] = max |r|, out[1] = max |F + P L psi| (as ordered uint64 bits).
template <class R>
__global__ void __launch_bounds__(256) k_residual(LevelDev L, const int4 *blocks, const int32_t *Tphi,
                                                  const void *phi_user, int dtype, int64_t ucs, const R *F,
                                                  int64_t cs, LevelDev Lc, const R *psi, int64_t pcs,
                                                  int has_coarse, unsigned long long *out) {
  const int b = Tphi[blockIdx.x], comp = blockIdx.y, sh = L.shift, B = 1 << sh;
  const int B3 = B * B * B;
  const int4 bc = blocks[b];
  const double inv_h2f = 1.0 / (L.h * L.h), inv_h2c = 1.0 / (Lc.h * Lc.h);
  double rmax = 0.0, smax = 0.0;
  auto phi_at = [&](int x, int y, int z, bool &ok) -> double {
    int blk, off;
    if (!level_cell(L, x, y, z, blk, off)) {
      ok = false;
      return 0.0;
    }
    if (!(L.cellmask[(int64_t)blk * B3 + off] & 1)) ok = false;
    const int uu = L.user_of[blk];
    if (uu < 0) {
      ok = false;
      return 0.0;
    }
    return load_field<double>(phi_user, comp * ucs + (int64_t)uu * B3 + off, dtype);
  };
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    if (!(L.cellmask[(int64_t)b * B3 + off] & 1)) continue;
    const int x = (bc.x << sh) + (off & (B - 1)), y = (bc.y << sh) + ((off >> sh) & (B - 1)),
              z = (bc.z << sh) + (off >> (2 * sh));
    bool ok = true;
    const double c0 = phi_at(x, y, z, ok);
    double s = phi_at(x + 1, y, z, ok) + phi_at(x - 1, y, z, ok) + phi_at(x, y + 1, z, ok) +
               phi_at(x, y - 1, z, ok) + phi_at(x, y, z + 1, ok) + phi_at(x, y, z - 1, ok);
    if (!ok) continue;
    double src = RT<R>::to_d(F[comp * cs + (int64_t)b * B3 + off]);
    if (has_coarse) {  // P L_{k-1} psi_{k-1} in FP64 arithmetic on the stored psi values
      src += interp_at<double>(x, y, z, [&](int i, int j, int k) {
        auto pv = [&](int a, int bb, int c) { return RT<R>::to_d(fetch<R>(Lc, psi, pcs, comp, a, bb, c)); };
        const double nb = pv(i + 1, j, k) + pv(i - 1, j, k) + pv(i, j + 1, k) + pv(i, j - 1, k) + pv(i, j, k + 1) +
                          pv(i, j, k - 1);
        return (nb - 6.0 * pv(i, j, k)) * inv_h2c;
      });
    }
    const double ar = fabs((s - 6.0 * c0) * inv_h2f - src);
    rmax = (ar != ar) ? 1e300 : fmax(rmax, ar);
    smax = fmax(smax, fabs(src));
  }
  // block reduce via atomics on the ordered bit patterns of non-negative doubles
  if (rmax > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(rmax));
  if (smax > 0.0) atomicMax(out + 1, (unsigned long long)__double_as_longlong(smax));
}

// Single-level FP64 residual; grid (ntgt, ncomp).  r = L phi - [source block] f at cells of target
// blocks whose six neighbours lie in target blocks (tmap: block coords over the box lo + [0, n) ->
// caller block index of a target block or -1; is_src: per caller block, 1 when it carries source
// values).  out[0] = max |r|, out[1] = max |f| over the same cells (ordered uint64 bits).
static __global__ void __launch_bounds__(256)
    k_residual_single(const int32_t *tmap, int3 lo, int3 n, int shift, double h, const int32_t *tgt_idx,
                      const int4 *tgt_c, const uint8_t *is_src, const void *phi, const void *f, int dtype, int64_t cs,
                      unsigned long long *out) {
  const int comp = blockIdx.y, B = 1 << shift, B3 = B * B * B, m = B - 1;
  const int u0 = tgt_idx[blockIdx.x];
  const int4 bc = tgt_c[blockIdx.x];
  const double inv_h2 = 1.0 / (h * h);
  double rmax = 0.0, smax = 0.0;
  auto at = [&](int x, int y, int z, bool &ok) -> double {
    const int bx = (x >> shift) - lo.x, by = (y >> shift) - lo.y, bz = (z >> shift) - lo.z;
    if ((unsigned)bx >= (unsigned)n.x || (unsigned)by >= (unsigned)n.y || (unsigned)bz >= (unsigned)n.z) {
      ok = false;
      return 0.0;
    }
    const int u = tmap[((int64_t)bz * n.y + by) * n.x + bx];
    if (u < 0) {
      ok = false;
      return 0.0;
    }
    const int off = (((z & m) << shift) + (y & m)) * B + (x & m);
    return load_field<double>(phi, comp * cs + (int64_t)u * B3 + off, dtype);
  };
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    const int x = (bc.x << shift) + (off & m), y = (bc.y << shift) + ((off >> shift) & m),
              z = (bc.z << shift) + (off >> (2 * shift));
    bool ok = true;
    const double c0 = load_field<double>(phi, comp * cs + (int64_t)u0 * B3 + off, dtype);
    const double s = at(x + 1, y, z, ok) + at(x - 1, y, z, ok) + at(x, y + 1, z, ok) + at(x, y - 1, z, ok) +
                     at(x, y, z + 1, ok) + at(x, y, z - 1, ok);
    if (!ok) continue;
    const double src = is_src[u0] ? load_field<double>(f, comp * cs + (int64_t)u0 * B3 + off, dtype) : 0.0;
    const double ar = fabs((s - 6.0 * c0) * inv_h2 - src);
    rmax = (ar != ar) ? 1e300 : fmax(rmax, ar);
    smax = fmax(smax, fabs(src));
  }
  if (rmax > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(rmax));
  if (smax > 0.0) atomicMax(out + 1, (unsigned long long)__double_as_longlong(smax));
}

// ------------------------------------------------------------------ heat apply (FIF-AMR)
struct HeatW {
  double w[65];  // w[n] = e^{-2 alpha} I_n(2 alpha), n <= r
  int r;
};

// P_k fhat, the level-k reconstruction of the AMR data (Sec. 3.2, Eq. (eq:interp)); grid (|HB_k|, ncomp),
// interp_sep_values(B) values of dynamic shared memory (the separable interpolation passes).
// The regions partition space, so each cell takes the value of the region that holds it: on the caller's
// level-k blocks F_k (own values on Omega_k, 8-child means of the finer levels on covered cells); on every
// other block the interpolation of the level-(k-1) reconstruction Uc (which holds the coarsened level-k data
// on its covered cells, so interpolation next to a level boundary reads the same function on both sides).
template <class R>
__global__ void __launch_bounds__(256) k_heat_build(LevelDev L, const int4 *blocks, const int32_t *HB, const R *F,
                                                    int nU, R *out, int64_t cs, LevelDev Lc, const R *Uc,
                                                    int64_t ucs_c, int has_coarse) {
  __shared__ R S[LGF_STAGE_MAX];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = HB[blockIdx.x], comp = blockIdx.y, sh = L.shift, B = 1 << sh;
  const int B3 = B * B * B, W = (B >> 1) + 2;
  R *T1 = reinterpret_cast<R *>(smem_raw), *T2 = T1 + W * W * B;
  const bool interp = b >= nU && has_coarse;  // the same for the whole CTA
  if (interp) {
    stage_coarse<R>(S, Lc, Uc, ucs_c, comp, blocks[b], B);
    __syncthreads();
    interp_sep_xy<R>(S, T1, T2, sh);
  }
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    R v = RT<R>::zero();
    if (b < nU) v = F[comp * cs + (int64_t)b * B3 + off];
    else if (interp) v = interp_sep_z<R>(T2, sh, off & (B - 1), (off >> sh) & (B - 1), off >> (2 * sh));
    out[comp * cs + (int64_t)b * B3 + off] = v;
  }
}

// One separable pass of E_alpha along `axis` over the heat block set, for kernel radii r <= B (every
// tap reads this block or one of its two neighbours along the axis).  The CTA stages the block and the
// r cells of each neighbour block next to it (zeros where a neighbour is absent) in shared memory as
// S[t][q]: t = la + r in [0, B + 2r) the position along the axis, q in [0, B^2) the line (the other two
// coordinates); rows padded to B^2 + 1.  Thread q then sums its line's B outputs from shared memory,
// symmetric taps paired, in double-float left unnormalised until the end, and the outputs go back to
// global memory through shared memory in the block's element order (coalesced).
// grid (|HB|, ncomp), B^2 threads, (B + 2r)(B^2 + 1) values of dynamic shared memory.
template <class R, int B>
__global__ void __launch_bounds__(B * B) k_heat_line(LevelDev L, const int4 *blocks, const int32_t *HB, int axis,
                                                     const R *in, R *out, int64_t cs, HeatW w) {
  constexpr int B2 = B * B, B3 = B * B2, SH = B == 8 ? 3 : 4, QS = B2 + 1;
  static_assert(B == 8 || B == 16, "block size");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *S = reinterpret_cast<R *>(smem_raw);
  __shared__ R wt[B + 1];
  const int r = w.r, T = B + 2 * r;
  const int b = HB[blockIdx.x], comp = blockIdx.y;
  const int4 bc = blocks[b];
  for (int d = threadIdx.x; d <= r; d += B2) wt[d] = RT<R>::from(w.w[d]);
  const int ex = axis == 0, ey = axis == 1, ez = axis == 2;
  const int nbm = level_block(L, bc.x - ex, bc.y - ey, bc.z - ez);
  const int nbp = level_block(L, bc.x + ex, bc.y + ey, bc.z + ez);
  const R *src = in + comp * cs;
  // e / T for e < T B^2 <= 48 * 256 by a multiply and shift (exact: the rounding of the reciprocal adds
  // less than e / 2^20 < 1 / T)
  const unsigned invT = ((1u << 20) + (unsigned)T - 1) / (unsigned)T;
  // staging order: consecutive e are consecutive in memory (x fastest; along x the axis runs fastest)
  for (int e = threadIdx.x; e < T * B2; e += B2) {
    int t, q, x, y, z;
    if (axis == 0) {
      q = (int)(((unsigned)e * invT) >> 20);
      t = e - q * T;
      y = q & (B - 1), z = q >> SH, x = t - r;
    } else if (axis == 1) {
      const int u = e >> SH, zz = (int)(((unsigned)u * invT) >> 20);
      x = e & (B - 1), t = u - zz * T, z = zz, y = t - r;
      q = x + B * z;
    } else {
      x = e & (B - 1), y = (e >> SH) & (B - 1), t = e >> (2 * SH), z = t - r;
      q = x + B * y;
    }
    const int la = t - r;  // in [-r, B + r)
    const int blk = la < 0 ? nbm : (la >= B ? nbp : b);
    const int sh = la < 0 ? B : (la >= B ? -B : 0);  // into the neighbour's local coordinates
    if (axis == 0) x += sh;
    else if (axis == 1) y += sh;
    else z += sh;
    S[t * QS + q] = blk >= 0 ? src[(int64_t)blk * B3 + ((z * B + y) * B + x)] : RT<R>::zero();
  }
  __syncthreads();
  const int q = threadIdx.x;
  R acc[B];
  const R w0 = wt[0];
#pragma unroll
  for (int la = 0; la < B; ++la) acc[la] = w0 * S[(la + r) * QS + q];
  for (int d = 1; d <= r; ++d) {
    const R wd = wt[d];
    const R *Sp = S + (r + d) * QS + q, *Sm = S + (r - d) * QS + q;
#pragma unroll
    for (int la = 0; la < B; ++la) acc[la] = rfma(acc[la], wd, radd(Sp[la * QS], Sm[la * QS]));
  }
  __syncthreads();  // every read of the tile is done before it is overwritten
#pragma unroll
  for (int la = 0; la < B; ++la) S[la * QS + q] = rnorm(acc[la]);
  __syncthreads();
  R *dst = out + comp * cs + (int64_t)b * B3;
  for (int off = threadIdx.x; off < B3; off += B2) {
    const int x = off & (B - 1), y = (off >> SH) & (B - 1), z = off >> (2 * SH);
    const int la = axis == 0 ? x : (axis == 1 ? y : z);
    const int ql = axis == 0 ? y + B * z : (axis == 1 ? x + B * z : x + B * y);
    dst[off] = S[la * QS + ql];
  }
}
template <class R, int B>
size_t heat_line_smem(int r) { return sizeof(R) * (size_t)(B + 2 * r) * (B * B + 1); }

// The same pass for radii r > B: every tap looks its cell up in the block map; absent cells read 0.
template <class R>
__global__ void __launch_bounds__(256) k_heat_pass(LevelDev L, const int4 *blocks, const int32_t *HB, int axis,
                                                   const R *in, R *out, int64_t cs, HeatW w) {
  __shared__ R wt[65];
  const int b = HB[blockIdx.x], comp = blockIdx.y, sh = L.shift, B = 1 << sh;
  const int B3 = B * B * B;
  const int4 bc = blocks[b];
  for (int d = threadIdx.x; d <= w.r; d += blockDim.x) wt[d] = RT<R>::from(w.w[d]);
  __syncthreads();
  const R *src = in + comp * cs;
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    const int x = (bc.x << sh) + (off & (B - 1)), y = (bc.y << sh) + ((off >> sh) & (B - 1)),
              z = (bc.z << sh) + (off >> (2 * sh));
    R acc = wt[0] * src[(int64_t)b * B3 + off];
    for (int d = 1; d <= w.r; ++d) {
      int blk, o2;
      R s = RT<R>::zero();
      const int dx = axis == 0 ? d : 0, dy = axis == 1 ? d : 0, dz = axis == 2 ? d : 0;
      if (level_cell(L, x + dx, y + dy, z + dz, blk, o2)) s = src[(int64_t)blk * B3 + o2];
      if (level_cell(L, x - dx, y - dy, z - dz, blk, o2)) s = radd(s, src[(int64_t)blk * B3 + o2]);
      acc = rfma(acc, wt[d], s);
    }
    out[comp * cs + (int64_t)b * B3 + off] = rnorm(acc);
  }
}

// g_user on Omega_k cells of the caller blocks; grid (nU_k, ncomp)
template <class R>
__global__ void __launch_bounds__(256) k_heat_store(LevelDev L, const R *g, int64_t cs, void *g_user, int dtype,
                                                    int64_t ucs, int64_t user_off) {
  const int b = blockIdx.x, comp = blockIdx.y, B3 = 1 << (3 * L.shift);
  for (int off = threadIdx.x; off < B3; off += blockDim.x)
    if (L.cellmask[(int64_t)b * B3 + off] & 1)
      store_field<R>(g_user, comp * ucs + (user_off + b) * (int64_t)B3 + off, dtype,
                     g[comp * cs + (int64_t)b * B3 + off]);
}
