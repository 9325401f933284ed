// pair_ops.cuh -- host launch wrappers of the pair-mode kernels (instantiated per arithmetic).
#pragma once
#include "internal.h"
#include "pair.cuh"

namespace lgf {

template <class R, int B>
static int fwd_b(const void *f, int dtype, int64_t cs, const int32_t *src_idx, int nsrc, int ncomp,
                 void *spec, const uint8_t *cellmask, int bits, cudaStream_t st) {
  if (nsrc == 0) return LGF_OK;
  const size_t sm = pair_fft_smem<R, B>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_block_fwd<R, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  k_block_fwd<R, B><<<dim3(nsrc, ncomp), 256, sm, st>>>(f, dtype, cs, src_idx, nsrc, (cx<R> *)spec,
                                                        cellmask, bits, make_tw64<R>());
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "block forward launch: %s", cudaGetErrorString(e));
}

template <class R, int B>
static int inv_b(const void *spec, int64_t spec_cs, const int32_t *rows, const int32_t *aux, int n, int ncomp,
                 void *out, int dtype, int64_t out_cs, int64_t out_off, const void *addend, int64_t add_cs,
                 const uint8_t *cellmask, int bits, double scale, cudaStream_t st) {
  if (n == 0) return LGF_OK;
  const size_t sm = pair_fft_smem<R, B>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_block_inv<R, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  k_block_inv<R, B><<<dim3(n, ncomp), 256, sm, st>>>((const cx<R> *)spec, spec_cs, rows, aux, out, dtype, out_cs,
                                                     out_off, (const R *)addend, add_cs, cellmask, bits, scale,
                                                     make_tw64<R>());
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "block inverse launch: %s", cudaGetErrorString(e));
}

template <class R, int NC>
static int mac_nc(int W, const cx<R> *F, int nsrc, int64_t f_cs, const int32_t *sl, const int4 *sc,
                  const cx<R> *Gh, int3 mo, cx<R> *Phi, int ntgt, int64_t p_cs, const int32_t *tl, const int4 *tc,
                  int accumulate, cudaStream_t st) {
  constexpr int TC = 4;
  dim3 grid((ntgt + TC - 1) / TC, (W + 127) / 128);
  k_mac_pair<R, TC, NC><<<grid, 128, 0, st>>>(F, nsrc, f_cs, sl, sc, Gh, mo, Phi, ntgt, p_cs, tl, tc, W,
                                              accumulate);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "pair MAC launch: %s", cudaGetErrorString(e));
}

template <class R>
int PairOps<R>::forward(int B, const void *f, int dtype, int64_t cs, const int32_t *src_idx, int nsrc,
                        int ncomp, void *spec, const uint8_t *cellmask, int bits, cudaStream_t st) {
  if (B == 8) return fwd_b<R, 8>(f, dtype, cs, src_idx, nsrc, ncomp, spec, cellmask, bits, st);
  if (B == 16) return fwd_b<R, 16>(f, dtype, cs, src_idx, nsrc, ncomp, spec, cellmask, bits, st);
  return set_error(LGF_E_UNSUPPORTED, "block size %d", B);
}

template <class R>
int PairOps<R>::inverse(int B, const void *spec, int64_t spec_cs, const int32_t *rows, const int32_t *aux, int n,
                        int ncomp, void *out, int dtype, int64_t out_cs, int64_t out_off, const void *addend,
                        int64_t add_cs, const uint8_t *cellmask, int bits, double scale, cudaStream_t st) {
  if (B == 8)
    return inv_b<R, 8>(spec, spec_cs, rows, aux, n, ncomp, out, dtype, out_cs, out_off, addend, add_cs, cellmask,
                       bits, scale, st);
  if (B == 16)
    return inv_b<R, 16>(spec, spec_cs, rows, aux, n, ncomp, out, dtype, out_cs, out_off, addend, add_cs, cellmask,
                        bits, scale, st);
  return set_error(LGF_E_UNSUPPORTED, "block size %d", B);
}

template <class R>
int PairOps<R>::mac(int B, const void *F, int nsrc, int64_t f_cs, const int32_t *src_list, const int4 *src_coords,
                    const void *Gh, int3 mo, void *Phi, int ntgt, int64_t p_cs, const int32_t *tgt_list,
                    const int4 *tgt_coords, int ncomp, int accumulate, cudaStream_t st) {
  if (ntgt == 0) return LGF_OK;
  const int W = (2 * B) * (2 * B) * (B + 1);
  for (int c0 = 0; c0 < ncomp; c0 += 3) {
    const int nc = ncomp - c0 < 3 ? ncomp - c0 : 3;
    const cx<R> *Fc = (const cx<R> *)F + c0 * f_cs;
    cx<R> *Pc = (cx<R> *)Phi + c0 * p_cs;
    const cx<R> *G = (const cx<R> *)Gh;
    int rc;
    if (nc == 1)
      rc = mac_nc<R, 1>(W, Fc, nsrc, f_cs, src_list, src_coords, G, mo, Pc, ntgt, p_cs, tgt_list, tgt_coords,
                        accumulate, st);
    else if (nc == 2)
      rc = mac_nc<R, 2>(W, Fc, nsrc, f_cs, src_list, src_coords, G, mo, Pc, ntgt, p_cs, tgt_list, tgt_coords,
                        accumulate, st);
    else
      rc = mac_nc<R, 3>(W, Fc, nsrc, f_cs, src_list, src_coords, G, mo, Pc, ntgt, p_cs, tgt_list, tgt_coords,
                        accumulate, st);
    if (rc) return rc;
  }
  return LGF_OK;
}

}  // namespace lgf
