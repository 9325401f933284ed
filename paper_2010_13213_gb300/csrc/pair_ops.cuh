// pair_ops.cuh -- host launch wrappers of the pair-mode kernels (instantiated per arithmetic).
#pragma once
#include "internal.h"
#include "pair.cuh"

namespace lgf {

template <class R, int B>
static int fwd_b(const void *f, int dtype, int64_t cs, const int32_t *src_idx, int nsrc, int ncomp,
                 void *spec, cudaStream_t st) {
  if (nsrc == 0) return LGF_OK;
  const size_t sm = pair_fft_smem<R, B>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_block_fwd<R, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  k_block_fwd<R, B><<<dim3(nsrc, ncomp), 256, sm, st>>>(f, dtype, cs, src_idx, nsrc, (cx<R> *)spec,
                                                        make_tw64<R>());
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "block forward launch: %s", cudaGetErrorString(e));
}

template <class R, int B>
static int inv_b(const void *spec, int ntgt, int ncomp, const int32_t *tgt_idx, void *out, int dtype,
                 int64_t cs, const void *addend, int add_dtype, double scale, cudaStream_t st) {
  if (ntgt == 0) return LGF_OK;
  const size_t sm = pair_fft_smem<R, B>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_block_inv<R, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  k_block_inv<R, B><<<dim3(ntgt, ncomp), 256, sm, st>>>((const cx<R> *)spec, ntgt, tgt_idx, out, dtype,
                                                        cs, addend, add_dtype, scale, make_tw64<R>());
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "block inverse launch: %s", cudaGetErrorString(e));
}

template <class R, int NC>
static int mac_nc(int W, const cx<R> *F, int nsrc, const int4 *src_c, const cx<R> *Gh, int3 mo,
                  cx<R> *Phi, int ntgt, const int4 *tgt_c, int accumulate, cudaStream_t st) {
  constexpr int TC = 4;
  dim3 grid((ntgt + TC - 1) / TC, (W + 127) / 128);
  k_mac_pair<R, TC, NC><<<grid, 128, 0, st>>>(F, nsrc, src_c, Gh, mo, Phi, ntgt, tgt_c, W, accumulate);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LGF_OK : set_error(LGF_E_CUDA, "pair MAC launch: %s", cudaGetErrorString(e));
}

template <class R>
int PairOps<R>::forward(int B, const void *f, int dtype, int64_t cs, const int32_t *src_idx, int nsrc,
                        int ncomp, void *spec, cudaStream_t st) {
  if (B == 8) return fwd_b<R, 8>(f, dtype, cs, src_idx, nsrc, ncomp, spec, st);
  if (B == 16) return fwd_b<R, 16>(f, dtype, cs, src_idx, nsrc, ncomp, spec, st);
  return set_error(LGF_E_UNSUPPORTED, "block size %d", B);
}

template <class R>
int PairOps<R>::inverse(int B, const void *spec, int ntgt, int ncomp, const int32_t *tgt_idx, void *out,
                        int dtype, int64_t cs, const void *addend, int add_dtype, double scale,
                        cudaStream_t st) {
  if (B == 8) return inv_b<R, 8>(spec, ntgt, ncomp, tgt_idx, out, dtype, cs, addend, add_dtype, scale, st);
  if (B == 16) return inv_b<R, 16>(spec, ntgt, ncomp, tgt_idx, out, dtype, cs, addend, add_dtype, scale, st);
  return set_error(LGF_E_UNSUPPORTED, "block size %d", B);
}

template <class R>
int PairOps<R>::mac(int B, const void *F, int nsrc, const int4 *src_c, const void *Gh, int3 mo, void *Phi,
                    int ntgt, const int4 *tgt_c, int ncomp, int accumulate, cudaStream_t st) {
  if (ntgt == 0) return LGF_OK;
  const int W = (2 * B) * (2 * B) * (B + 1);
  const size_t cstride_F = (size_t)nsrc * W, cstride_P = (size_t)ntgt * W;
  for (int c0 = 0; c0 < ncomp; c0 += 3) {
    const int nc = ncomp - c0 < 3 ? ncomp - c0 : 3;
    const cx<R> *Fc = (const cx<R> *)F + c0 * cstride_F;
    cx<R> *Pc = (cx<R> *)Phi + c0 * cstride_P;
    int rc;
    if (nc == 1)
      rc = mac_nc<R, 1>(W, Fc, nsrc, src_c, (const cx<R> *)Gh, mo, Pc, ntgt, tgt_c, accumulate, st);
    else if (nc == 2)
      rc = mac_nc<R, 2>(W, Fc, nsrc, src_c, (const cx<R> *)Gh, mo, Pc, ntgt, tgt_c, accumulate, st);
    else
      rc = mac_nc<R, 3>(W, Fc, nsrc, src_c, (const cx<R> *)Gh, mo, Pc, ntgt, tgt_c, accumulate, st);
    if (rc) return rc;
  }
  return LGF_OK;
}

}  // namespace lgf
