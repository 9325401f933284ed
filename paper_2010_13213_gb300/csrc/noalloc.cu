// noalloc.cu -- a single-level solve that performs no device allocation.
//
// Who needs it: code that must not allocate device memory during a solve -- for example a caller
// with a device-memory budget fixed at start-up, or one running on a thread that must not block on
// the allocator (cudaMalloc can synchronise the device and may fail under memory pressure).  Such a
// caller still owns its input and output buffers and the LGF table (built once beforehand); the
// solve's scratch (source and target spectra, index lists) lives in a file-scope device array of
// fixed size instead of the table's per-stream workspace.
//
// The array is a static __device__ object: every GPU that loads the library reserves its
// LGF_STATIC_SCRATCH_BYTES until the process exits.  Host code cannot use the array's name as a
// device address; the first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it.  That first call should therefore happen before any
// stream capture.  Every call copies its block index lists from pageable host memory into the array,
// so a call on a stream that is capturing is rejected (LGF_E_UNSUPPORTED) before anything is
// enqueued.  All calls share the one array: calls whose GPU work overlaps (different streams,
// or different host threads without ordering) race on it and must be serialised by the caller.
// Nothing in the array needs to start at zero: every byte a call reads was written earlier in the
// same call.
#include <mutex>
#include <vector>

#include "internal.h"

#define LGF_STATIC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_lgf_static_scratch[LGF_STATIC_SCRATCH_BYTES];

namespace lgf {

static std::mutex g_static_mu;
static void *g_static_addr[64];

static int static_scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return set_error(LGF_E_CUDA, "no current CUDA device");
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_lgf_static_scratch);
    if (e != cudaSuccess || !p)
      return set_error(LGF_E_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                       cudaGetErrorString(e));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return LGF_OK;
}

template <class R>
static const void *table_spectra(const lgf_table *t);
template <>
const void *table_spectra<double>(const lgf_table *t) { return t->s64; }
template <>
const void *table_spectra<float>(const lgf_table *t) { return t->s32; }
template <>
const void *table_spectra<df>(const lgf_table *t) { return t->sdf; }

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

template <class R>
static int solve_static(const lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi,
                        int dtype, cudaStream_t st) {
  const int B = m->block;
  const int nb = m->nblocks[0];
  const int W = (2 * B) * (2 * B) * (B + 1);
  const void *Gh = table_spectra<R>(t);
  if (!Gh) return set_error(LGF_E_INVALID_ARG, "table lacks the spectra of the requested precision");
  std::vector<int32_t> src_idx, tgt_idx;
  std::vector<int4> src_c, tgt_c;
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  int tlo[3] = {1 << 30, 1 << 30, 1 << 30}, thi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int i = 0; i < nb; ++i) {
    const int role = m->block_role ? m->block_role[i] : 3;
    const int32_t *b = m->block_ijk + 3 * i;
    const int4 c = make_int4(b[0], b[1], b[2], 0);
    if (role & 1) {
      src_idx.push_back(i);
      src_c.push_back(c);
      for (int a = 0; a < 3; ++a) lo[a] = b[a] < lo[a] ? b[a] : lo[a], hi[a] = b[a] > hi[a] ? b[a] : hi[a];
    }
    if (role & 2) {
      tgt_idx.push_back(i);
      tgt_c.push_back(c);
      for (int a = 0; a < 3; ++a) tlo[a] = b[a] < tlo[a] ? b[a] : tlo[a], thi[a] = b[a] > thi[a] ? b[a] : thi[a];
    }
  }
  const int nsrc = (int)src_idx.size(), ntgt = (int)tgt_idx.size();
  if (ntgt == 0) return LGF_OK;
  const int mo[3] = {t->mo.x, t->mo.y, t->mo.z};
  if (nsrc)
    for (int a = 0; a < 3; ++a) {
      const int reach = (thi[a] - lo[a]) > (hi[a] - tlo[a]) ? (thi[a] - lo[a]) : (hi[a] - tlo[a]);
      if (reach > mo[a])
        return set_error(LGF_E_TABLE_RANGE, "block offsets reach %d along axis %d; the table covers %d",
                         reach, a, mo[a]);
    }
  // carve the static array: [index lists][source spectra][target spectra]
  const size_t idx_bytes = align256(sizeof(int4) * (nsrc + ntgt) + sizeof(int32_t) * (nsrc + ntgt));
  const size_t specF = align256(sizeof(cx<R>) * (size_t)ncomp * nsrc * W);
  const size_t specP = align256(sizeof(cx<R>) * (size_t)ncomp * ntgt * W);
  const size_t need = idx_bytes + specF + specP;
  if (need > LGF_STATIC_SCRATCH_BYTES)
    return set_error(LGF_E_INVALID_ARG,
                     "allocation-free solve needs %zu bytes of scratch; the static scratch holds %u "
                     "(reduce ncomp or the number of blocks, or use lgf_poisson_solve)",
                     need, (unsigned)LGF_STATIC_SCRATCH_BYTES);
  void *base = nullptr;
  int rc = static_scratch_address(&base);
  if (rc) return rc;
  char *p = (char *)base;
  int4 *d_src_c = (int4 *)p;
  int4 *d_tgt_c = d_src_c + nsrc;
  int32_t *d_src_idx = (int32_t *)(d_tgt_c + ntgt);
  int32_t *d_tgt_idx = d_src_idx + nsrc;
  void *F = p + idx_bytes;
  void *P = p + idx_bytes + specF;
  // The index lists go up from pageable host vectors: the copy returns once the data is staged, so the
  // vectors may be released when this function returns.
  struct Up {
    void *dst;
    const void *src;
    size_t n;
    const char *what;
  } ups[4] = {{d_src_c, src_c.data(), sizeof(int4) * nsrc, "source coordinates"},
              {d_src_idx, src_idx.data(), sizeof(int32_t) * nsrc, "source indices"},
              {d_tgt_c, tgt_c.data(), sizeof(int4) * ntgt, "target coordinates"},
              {d_tgt_idx, tgt_idx.data(), sizeof(int32_t) * ntgt, "target indices"}};
  for (const Up &u : ups) {
    if (u.n == 0) continue;
    const cudaError_t e = cudaMemcpyAsync(u.dst, u.src, u.n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(LGF_E_CUDA, "allocation-free solve: copy of the %s failed: %s", u.what,
                       cudaGetErrorString(e));
    }
  }
  const int64_t cs = (int64_t)nb * B * B * B;
  if ((rc = PairOps<R>::forward(B, f, dtype, cs, d_src_idx, nsrc, ncomp, F, nullptr, 0, st))) return rc;
  if ((rc = PairOps<R>::mac(B, F, nsrc, (int64_t)nsrc * W, nullptr, d_src_c, Gh, t->mo, P, ntgt, (int64_t)ntgt * W,
                            nullptr, d_tgt_c, ncomp, 0, st)))
    return rc;
  const double h = m->h0;
  const double scale = h * h / (double)((2 * B) * (2 * B) * (2 * B));
  return PairOps<R>::inverse(B, P, (int64_t)ntgt * W, nullptr, d_tgt_idx, ntgt, ncomp, phi, dtype, cs, 0, nullptr, 0,
                             nullptr, 0, scale, st);
}

int check_mesh(const lgf_mesh *m, int B_expected);

}  // namespace lgf

using namespace lgf;

extern "C" int lgf_poisson_solve_static(const lgf_table *t, const lgf_mesh *m, int32_t ncomp,
                                        const void *f_dev, void *phi_dev, int32_t dtype, int32_t precision,
                                        void *cuda_stream) {
  if (!t) return set_error(LGF_E_INVALID_ARG, "table is NULL");
  int rc = check_mesh(m, t->B);
  if (rc) return rc;
  if (m->nlevels != 1) return set_error(LGF_E_UNSUPPORTED, "the allocation-free solve is single-level only");
  if (ncomp < 1) return set_error(LGF_E_INVALID_ARG, "ncomp %d", ncomp);
  if (!f_dev || !phi_dev || f_dev == phi_dev) return set_error(LGF_E_INVALID_ARG, "bad field pointers");
  if (dtype != LGF_F64 && dtype != LGF_F32) return set_error(LGF_E_INVALID_ARG, "dtype %d", dtype);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // The index lists are copied from pageable host memory, which a capturing stream refuses (and the
  // refusal would invalidate the caller's capture): reject before anything is enqueued.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(st, &cap);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return set_error(LGF_E_CUDA, "allocation-free solve: cudaStreamIsCapturing: %s", cudaGetErrorString(ce));
  }
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(LGF_E_UNSUPPORTED,
                     "allocation-free solve called on a capturing stream: its index lists are copied from "
                     "pageable host memory, which stream capture does not accept");
  switch (precision) {
    case LGF_PREC_FP64: return solve_static<double>(t, m, ncomp, f_dev, phi_dev, dtype, st);
    case LGF_PREC_FP32: return solve_static<float>(t, m, ncomp, f_dev, phi_dev, dtype, st);
    case LGF_PREC_DF32: return solve_static<df>(t, m, ncomp, f_dev, phi_dev, dtype, st);
    default: return set_error(LGF_E_INVALID_ARG, "precision %d", precision);
  }
}
