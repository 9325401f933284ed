// refresh.cu -- velocity refresh u = -C^T L_E^{-1} omega on one level (Sec. 4.1, Eq. (eq:vel_update)).
//
// Staggered lattice (Sec. 2.1): the velocity lives on the positive faces of a cell, the vorticity and the
// streamfunction on its positive edges; component a of cell n is stored at index n (face centre
// n + (1,1,1)/2 + e_a/2, edge centre n + (1,1,1) - e_a/2, in cells).  The LGF of the edge Laplacian is
// the cell one (the lattice is shift-invariant), so L_E^{-1} is the library's three-component Poisson
// solve; C^T, the curl from edges to faces (the transpose of the face-to-edge curl C, Eq. (eq:mimetic)),
// is a backward difference:
//   (C^T psi)_x[n] = (psi_z[n] - psi_z[n - e_y] - psi_y[n] + psi_y[n - e_z]) / h   (and cyclically).
// The backward differences reach one cell below a block toward -x, -y, -z, so the streamfunction is
// solved on the caller's blocks (sources and targets) and on their -x, -y, -z neighbour blocks (targets).
#include <cuda_runtime.h>
#include <string.h>

#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "solver.h"

namespace lgf {

template <class T>
__device__ __forceinline__ double ld(const T *p, int64_t i) {
  return (double)p[i];
}

// u = -C^T psi on the caller's blocks; grid (nblocks, 3 components), 256 threads.
// psi: [3][next][B^3] over the extended block set whose first n blocks are the caller's; nbr[b][a] is the
// extended index of block b's neighbour toward -e_a.
template <class T>
__global__ void __launch_bounds__(256) k_curl_t(const T *__restrict__ psi, int64_t pcs, const int32_t *__restrict__ nbr,
                                                int shift, double inv_h, T *__restrict__ u, int64_t ucs) {
  const int b = blockIdx.x, comp = blockIdx.y, B = 1 << shift, B3 = 1 << (3 * shift);
  const int a1 = (comp + 1) % 3, a2 = (comp + 2) % 3;  // (C^T psi)_c = d_{a1} psi_{a2} - d_{a2} psi_{a1}
  const int nb1 = nbr[3 * b + a1], nb2 = nbr[3 * b + a2];
  for (int off = threadIdx.x; off < B3; off += blockDim.x) {
    const int c[3] = {off & (B - 1), (off >> shift) & (B - 1), off >> (2 * shift)};
    const int st1 = 1 << (a1 * shift), st2 = 1 << (a2 * shift);  // element strides along a1, a2
    // index of the cell one step toward -e_a1 (-e_a2): this block, or the neighbour's last layer
    const int64_t own = (int64_t)b * B3 + off;
    const int64_t m1 = c[a1] > 0 ? own - st1 : (int64_t)nb1 * B3 + off + (int64_t)(B - 1) * st1;
    const int64_t m2 = c[a2] > 0 ? own - st2 : (int64_t)nb2 * B3 + off + (int64_t)(B - 1) * st2;
    const double d1 = ld(psi, a2 * pcs + own) - ld(psi, a2 * pcs + m1);  // backward difference along a1 of psi_a2
    const double d2 = ld(psi, a1 * pcs + own) - ld(psi, a1 * pcs + m2);  // along a2 of psi_a1
    u[comp * ucs + own] = (T)(-(d1 - d2) * inv_h);
  }
}

}  // namespace lgf

using namespace lgf;

extern "C" int lgf_velocity_refresh(lgf_table *t, const lgf_mesh *m, const void *omega_dev, void *u_dev,
                                    int32_t dtype, const lgf_solve_opts *opts, lgf_report *rep, void *cuda_stream) {
  if (!t) return set_error(LGF_E_INVALID_ARG, "table is NULL");
  int rc = check_mesh(m, t->B);
  if (rc) return rc;
  if (m->nlevels != 1) return set_error(LGF_E_MESH, "the velocity refresh takes one level (got %d)", m->nlevels);
  if (!omega_dev || !u_dev) return set_error(LGF_E_INVALID_ARG, "field pointer NULL");
  if (omega_dev == u_dev) return set_error(LGF_E_INVALID_ARG, "omega and u alias");
  if (dtype != LGF_F64 && dtype != LGF_F32) return set_error(LGF_E_INVALID_ARG, "dtype %d", dtype);
  lgf_solve_opts o{LGF_PREC_FP64, LGF_MAC_AUTO, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (o.precision < 0 || o.precision > 2) return set_error(LGF_E_INVALID_ARG, "precision %d", o.precision);
  if (o.mac_mode < 0 || o.mac_mode > 2) return set_error(LGF_E_INVALID_ARG, "mac_mode %d", o.mac_mode);
  if ((rc = check_slices(o))) return rc;
  if (rep) memset(rep, 0, sizeof(*rep));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int B = m->block, n = m->nblocks[0];
  const int shift = B == 8 ? 3 : 4;
  const int64_t B3 = (int64_t)B * B * B;
  // extended block set: the caller's blocks first, then the missing -x, -y, -z neighbours
  std::map<std::tuple<int, int, int>, int> index;
  std::vector<int32_t> ijk(m->block_ijk, m->block_ijk + 3 * (size_t)n);
  for (int i = 0; i < n; ++i) index[std::make_tuple(ijk[3 * i], ijk[3 * i + 1], ijk[3 * i + 2])] = i;
  std::vector<int32_t> nbr(3 * (size_t)n);
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      int c[3] = {m->block_ijk[3 * i], m->block_ijk[3 * i + 1], m->block_ijk[3 * i + 2]};
      --c[a];
      const auto key = std::make_tuple(c[0], c[1], c[2]);
      auto it = index.find(key);
      if (it == index.end()) {
        it = index.emplace(key, (int)(ijk.size() / 3)).first;
        ijk.insert(ijk.end(), c, c + 3);
      }
      nbr[3 * i + a] = it->second;
    }
  const int next = (int)(ijk.size() / 3);
  std::vector<uint8_t> roles(next, 2);  // added blocks: targets only
  for (int i = 0; i < n; ++i) roles[i] = 3;
  lgf_mesh me = *m;
  int32_t nb_ext[1] = {next};
  me.nblocks = nb_ext;
  me.block_ijk = ijk.data();
  me.block_role = roles.data();
  // scratch (stream-ordered): omega on the extended set (the added blocks are not sources, never read),
  // psi on the extended set, the neighbour table
  const size_t es = dtype == LGF_F64 ? 8 : 4;
  const int64_t ext_cs = (int64_t)next * B3, ucs = (int64_t)n * B3;
  void *om = nullptr, *psi = nullptr, *dnbr = nullptr;
  if (cudaMallocAsync(&om, es * 3 * (size_t)ext_cs, st) != cudaSuccess ||
      cudaMallocAsync(&psi, es * 3 * (size_t)ext_cs, st) != cudaSuccess ||
      cudaMallocAsync(&dnbr, sizeof(int32_t) * nbr.size(), st) != cudaSuccess) {
    if (om) cudaFreeAsync(om, st);
    if (psi) cudaFreeAsync(psi, st);
    if (dnbr) cudaFreeAsync(dnbr, st);
    cudaGetLastError();
    return set_error(LGF_E_OOM, "velocity refresh scratch (%zu bytes)", 2 * es * 3 * (size_t)ext_cs);
  }
  for (int c = 0; c < 3; ++c)
    cudaMemcpyAsync((char *)om + es * c * ext_cs, (const char *)omega_dev + es * c * ucs, es * ucs,
                    cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(dnbr, nbr.data(), sizeof(int32_t) * nbr.size(), cudaMemcpyHostToDevice, st);
  rc = solve_poisson(t, &me, 3, om, psi, dtype, o, rep, st);
  if (rc == LGF_OK) {
    const double inv_h = 1.0 / m->h0;
    if (dtype == LGF_F64)
      k_curl_t<double><<<dim3(n, 3), 256, 0, st>>>((const double *)psi, ext_cs, (const int32_t *)dnbr, shift, inv_h,
                                                  (double *)u_dev, ucs);
    else
      k_curl_t<float><<<dim3(n, 3), 256, 0, st>>>((const float *)psi, ext_cs, (const int32_t *)dnbr, shift, inv_h,
                                                 (float *)u_dev, ucs);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = set_error(LGF_E_CUDA, "curl launch: %s", cudaGetErrorString(e));
    else if (rep) rep->kernel_launches += 1;
  }
  cudaFreeAsync(om, st);
  cudaFreeAsync(psi, st);
  cudaFreeAsync(dnbr, st);
  return rc;
}
