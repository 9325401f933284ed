// plan.cu -- host construction of the composite-mesh plan (regions -> block sets -> device lists).
#include <algorithm>
#include <map>
#include <tuple>

#include "plan.h"

namespace lgf {

static inline int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
static inline int fmod_(int a, int b) { return a - b * fdiv(a, b); }

// Region bits of the per-level cell grid.
enum : uint8_t { G_UB = 1, G_OM = 2, G_COV = 4, G_EX = 8, G_NP = 16, G_C = 32, G_HR = 64, G_NU = 128 };

struct Grid {
  int lo[3] = {0, 0, 0}, n[3] = {0, 0, 0};
  std::vector<uint8_t> v;
  size_t idx(int x, int y, int z) const {
    return ((size_t)(z - lo[2]) * n[1] + (size_t)(y - lo[1])) * n[0] + (size_t)(x - lo[0]);
  }
  bool inside(int x, int y, int z) const {
    return x >= lo[0] && y >= lo[1] && z >= lo[2] && x < lo[0] + n[0] && y < lo[1] + n[1] && z < lo[2] + n[2];
  }
  uint8_t get(int x, int y, int z) const { return inside(x, y, z) ? v[idx(x, y, z)] : 0; }
};

// out_bit |= max-norm dilation of in_mask by r (separable running windows).
static void dilate(Grid &g, uint8_t in_mask, int r, uint8_t out_bit) {
  const size_t N = g.v.size();
  std::vector<uint8_t> a(N), b(N);
  for (size_t i = 0; i < N; ++i) a[i] = (g.v[i] & in_mask) ? 1 : 0;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  auto pass = [&](std::vector<uint8_t> &src, std::vector<uint8_t> &dst, int axis) {
    const int len = g.n[axis];
    const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)nx : (size_t)nx * ny);
    const int o1 = axis == 0 ? ny : nx, o2 = axis == 2 ? ny : nz;
    std::vector<int> pre(len + 1);
    for (int j2 = 0; j2 < o2; ++j2)
      for (int j1 = 0; j1 < o1; ++j1) {
        size_t base;
        if (axis == 0) base = ((size_t)j2 * ny + j1) * nx;
        else if (axis == 1) base = (size_t)j2 * nx * ny + j1;
        else base = (size_t)j2 * nx + j1;
        pre[0] = 0;
        for (int i = 0; i < len; ++i) pre[i + 1] = pre[i] + src[base + i * stride];
        for (int i = 0; i < len; ++i) {
          const int l = std::max(0, i - r), h = std::min(len, i + r + 1);
          dst[base + i * stride] = (pre[h] - pre[l]) > 0;
        }
      }
  };
  if (r <= 0) {
    for (size_t i = 0; i < N; ++i)
      if (a[i]) g.v[i] |= out_bit;
    return;
  }
  pass(a, b, 0);
  pass(b, a, 1);
  pass(a, b, 2);
  for (size_t i = 0; i < N; ++i)
    if (b[i]) g.v[i] |= out_bit;
}

// coarse.out_bit |= footprint of fine cells having any bit of fine_mask, then dilated by r.
static void footprint_dilate(const Grid &fine, uint8_t fine_mask, Grid &coarse, int r, uint8_t out_bit,
                             uint8_t tmp_bit) {
  for (auto &v : coarse.v) v &= (uint8_t)~tmp_bit;
  for (int z = 0; z < fine.n[2]; ++z)
    for (int y = 0; y < fine.n[1]; ++y)
      for (int x = 0; x < fine.n[0]; ++x) {
        if (!(fine.v[((size_t)z * fine.n[1] + y) * fine.n[0] + x] & fine_mask)) continue;
        const int cx = fdiv(x + fine.lo[0], 2), cy = fdiv(y + fine.lo[1], 2), cz = fdiv(z + fine.lo[2], 2);
        if (coarse.inside(cx, cy, cz)) coarse.v[coarse.idx(cx, cy, cz)] |= tmp_bit;
      }
  dilate(coarse, tmp_bit, r, out_bit);
  for (auto &v : coarse.v) v &= (uint8_t)~tmp_bit;
}

Plan::~Plan() {
  for (auto &l : L) {
    cudaFree(l.d_map);
    cudaFree(l.d_BL);
    cudaFree(l.d_cellmask);
    cudaFree(l.d_octcov);
    cudaFree(l.d_lists);
    cudaFree(l.d_phi_oct);
    cudaFree(l.d_user_of);
    cudaFree(l.d_box);
  }
}

template <class T>
static int upload(T **dst, const std::vector<T> &src, size_t *acc) {
  const size_t n = std::max<size_t>(src.size(), 1) * sizeof(T);
  if (cudaMalloc(dst, n) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LGF_E_OOM, "plan upload of %zu bytes failed", n);
  }
  if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error(LGF_E_CUDA, "plan upload copy failed");
  *acc += n;
  return LGF_OK;
}

int build_plan(const lgf_mesh *m, const int *heat_radii, Plan **out) {
  const int B = m->block, K = m->nlevels, H = B / 2;
  const int ne = m->n_ext;
  Plan *P = new Plan();
  P->B = B;
  P->K = K;
  P->n_ext = ne;
  P->heat = heat_radii != nullptr;
  P->L.resize(K);
  std::vector<std::map<std::tuple<int, int, int>, int>> umap(K);
  int64_t off = 0;
  int rmax = 0;
  if (heat_radii)
    for (int k = 0; k < K; ++k) rmax = std::max(rmax, heat_radii[k]);
  for (int k = 0; k < K; ++k) {
    LevelPlan &L = P->L[k];
    L.k = k;
    L.user_off = off;
    L.nU = m->nblocks[k];
    L.heat_r = heat_radii ? heat_radii[k] : 0;
    for (int i = 0; i < L.nU; ++i) {
      const int32_t *b = m->block_ijk + 3 * (off + i);
      umap[k][std::make_tuple(b[0], b[1], b[2])] = i;
      L.BL.push_back(make_int4(b[0], b[1], b[2], 0));
    }
    off += L.nU;
  }
  // nesting and covered octants
  std::vector<std::vector<uint8_t>> cov(K);
  for (int k = 0; k < K; ++k) cov[k].assign(P->L[k].nU, 0);
  for (int k = 0; k + 1 < K; ++k) {
    for (auto &c : P->L[k + 1].BL) {
      auto it = umap[k].find(std::make_tuple(fdiv(c.x, 2), fdiv(c.y, 2), fdiv(c.z, 2)));
      if (it == umap[k].end()) {
        delete P;
        return set_error(LGF_E_MESH, "level %d block (%d,%d,%d) is not inside a level-%d block", k + 1, c.x,
                         c.y, c.z, k);
      }
      cov[k][it->second] |= (uint8_t)(1 << (fmod_(c.x, 2) + 2 * fmod_(c.y, 2) + 4 * fmod_(c.z, 2)));
    }
  }
  // level grids
  const int need = std::max(ne + 1, (ne + B) / 2 + 4 + B) + rmax + 2;
  const int D = ((need + B - 1) / B) * B;
  std::vector<Grid> G(K);
  for (int k = 0; k < K; ++k) {
    LevelPlan &L = P->L[k];
    int blo[3] = {1 << 30, 1 << 30, 1 << 30}, bhi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    for (int i = 0; i < L.nU; ++i) {
      const int v[3] = {L.BL[i].x, L.BL[i].y, L.BL[i].z};
      for (int a = 0; a < 3; ++a) blo[a] = std::min(blo[a], v[a]), bhi[a] = std::max(bhi[a], v[a]);
    }
    for (int a = 0; a < 3; ++a) {
      G[k].lo[a] = blo[a] * B - D;
      G[k].n[a] = (bhi[a] - blo[a] + 1) * B + 2 * D;
      L.bb_lo[a] = blo[a] - D / B;
      L.bb_n[a] = G[k].n[a] / B;
    }
    const size_t cells = (size_t)G[k].n[0] * G[k].n[1] * G[k].n[2];
    if (cells > ((size_t)1 << 31)) {
      delete P;
      return set_error(LGF_E_MESH, "level %d region grid too large (%zu cells)", k, cells);
    }
    G[k].v.assign(cells, 0);
    for (int i = 0; i < L.nU; ++i) {
      const int4 c = L.BL[i];
      for (int z = 0; z < B; ++z)
        for (int y = 0; y < B; ++y)
          for (int x = 0; x < B; ++x) {
            const int o = (x >= H) + 2 * (y >= H) + 4 * (z >= H);
            const bool covered = (cov[k][i] >> o) & 1;
            G[k].v[G[k].idx(c.x * B + x, c.y * B + y, c.z * B + z)] |= G_UB | (covered ? G_COV : G_OM);
          }
    }
  }
  for (int k = 1; k < K; ++k) {
    dilate(G[k], G_OM, ne, G_EX);
    for (auto &v : G[k].v)
      if (v & G_OM) v &= (uint8_t)~G_EX;
  }
  auto blocks_with = [&](int k, uint8_t mask, std::vector<int4> &res) {
    const Grid &g = G[k];
    res.clear();
    for (int bz = 0; bz < g.n[2] / B; ++bz)
      for (int by = 0; by < g.n[1] / B; ++by)
        for (int bx = 0; bx < g.n[0] / B; ++bx) {
          bool any = false;
          for (int z = 0; z < B && !any; ++z)
            for (int y = 0; y < B && !any; ++y) {
              const size_t base = ((size_t)(bz * B + z) * g.n[1] + (by * B + y)) * g.n[0] + bx * B;
              for (int x = 0; x < B; ++x)
                if (g.v[base + x] & mask) {
                  any = true;
                  break;
                }
            }
          if (any) res.push_back(make_int4(g.lo[0] / B + bx, g.lo[1] / B + by, g.lo[2] / B + bz, 0));
        }
  };
  // BL index lookup / insertion
  std::vector<std::map<std::tuple<int, int, int>, int>> blmap(K);
  for (int k = 0; k < K; ++k)
    for (int i = 0; i < P->L[k].nU; ++i)
      blmap[k][std::make_tuple(P->L[k].BL[i].x, P->L[k].BL[i].y, P->L[k].BL[i].z)] = i;
  auto bl_index = [&](int k, int4 c) {
    auto key = std::make_tuple(c.x, c.y, c.z);
    auto it = blmap[k].find(key);
    if (it != blmap[k].end()) return it->second;
    const int idx = (int)P->L[k].BL.size();
    P->L[k].BL.push_back(c);
    blmap[k][key] = idx;
    return idx;
  };
  std::vector<int4> tmp;
  // Poisson block sets, finest to coarsest
  for (int k = K - 1; k >= 0; --k) {
    LevelPlan &L = P->L[k];
    L.Tphi.clear();
    for (int i = 0; i < L.nU; ++i)
      if (cov[k][i] != 0xFF) L.Tphi.push_back(i);
    blocks_with(k, G_NP, tmp);
    std::vector<int32_t> tpsi;
    for (auto &c : tmp) tpsi.push_back(bl_index(k, c));
    L.Tpsi = tpsi;
    if (k >= 1) {
      // C_k = cells of (Tphi u Tpsi) blocks u dilate(SR_k, 1)
      dilate(G[k], G_OM | G_EX, 1, G_C);
      auto mark_block = [&](int4 c) {
        for (int z = 0; z < B; ++z)
          for (int y = 0; y < B; ++y)
            for (int x = 0; x < B; ++x) {
              const int gx = c.x * B + x, gy = c.y * B + y, gz = c.z * B + z;
              if (G[k].inside(gx, gy, gz)) G[k].v[G[k].idx(gx, gy, gz)] |= G_C;
            }
      };
      for (int i : L.Tphi) mark_block(L.BL[i]);
      for (int i : L.Tpsi) mark_block(L.BL[i]);
      footprint_dilate(G[k], G_C, G[k - 1], 2, G_NP, G_HR);  // G_HR used as scratch here
    }
  }
  // source lists
  for (int k = 0; k < K; ++k) {
    LevelPlan &L = P->L[k];
    L.SA.clear();
    L.SB.clear();
    if (k == 0) {
      for (int i = 0; i < L.nU; ++i)
        if (cov[k][i] != 0xFF) L.SA.push_back(i);
    } else {
      blocks_with(k, G_OM | G_EX, tmp);
      for (auto &c : tmp) L.SA.push_back(bl_index(k, c));
    }
    if (k + 1 < K)
      for (int i = 0; i < L.nU; ++i)
        if (cov[k][i]) L.SB.push_back(i);
    if (k >= 1) {
      blocks_with(k, G_C, tmp);
      for (auto &c : tmp) bl_index(k, c);
    }
  }
  // heat regions (after the Poisson scratch use of G_HR)
  if (heat_radii) {
    for (int k = 0; k < K; ++k)
      for (auto &v : G[k].v) v &= (uint8_t)~(G_HR | G_NU);
    for (int k = 0; k < K; ++k) dilate(G[k], G_OM, heat_radii[k], G_HR);
    for (int k = K - 2; k >= 0; --k) {
      // NU_k = dilate(footprint(HR_{k+1} u NU_{k+1}), 1); G_C of level k is free scratch now
      footprint_dilate(G[k + 1], G_HR | G_NU, G[k], 1, G_NU, G_C);
    }
    for (int k = 0; k < K; ++k) {
      blocks_with(k, G_HR | G_NU | G_UB, tmp);
      P->L[k].HB.clear();
      for (auto &c : tmp) P->L[k].HB.push_back(bl_index(k, c));
    }
  }
  // per-level finishing: maps, masks, lists, upload
  for (int k = 0; k < K; ++k) {
    LevelPlan &L = P->L[k];
    const int nBL = (int)L.BL.size();
    L.map.assign((size_t)L.bb_n[0] * L.bb_n[1] * L.bb_n[2], -1);
    for (int i = 0; i < nBL; ++i) {
      const int bx = L.BL[i].x - L.bb_lo[0], by = L.BL[i].y - L.bb_lo[1], bz = L.BL[i].z - L.bb_lo[2];
      if (bx < 0 || by < 0 || bz < 0 || bx >= L.bb_n[0] || by >= L.bb_n[1] || bz >= L.bb_n[2]) {
        delete P;
        return set_error(LGF_E_MESH, "internal: block outside the level map");
      }
      L.map[((size_t)bz * L.bb_n[1] + by) * L.bb_n[0] + bx] = i;
    }
    const size_t B3 = (size_t)B * B * B;
    L.cellmask.assign((size_t)nBL * B3, 0);
    L.octcov.assign(nBL, 0);
    for (int i = 0; i < nBL; ++i) {
      if (i < L.nU) L.octcov[i] = cov[k][i];
      const int4 c = L.BL[i];
      for (int z = 0; z < B; ++z)
        for (int y = 0; y < B; ++y)
          for (int x = 0; x < B; ++x) {
            const uint8_t g = G[k].get(c.x * B + x, c.y * B + y, c.z * B + z);
            uint8_t cb = 0;
            if (g & G_OM) cb |= CB_OM;
            if (g & G_EX) cb |= CB_EX;
            if (g & G_COV) cb |= CB_COV;
            L.cellmask[(size_t)i * B3 + ((size_t)z * B + y) * B + x] = cb;
            if ((cb & CB_OM) && i < L.nU) ++L.n_omega;
            if (cb & (CB_OM | CB_EX | CB_COV)) ++L.n_src;
          }
    }
    // Tall = Tphi then (Tpsi minus Tphi); psi rows
    L.Tall = L.Tphi;
    std::map<int, int> row_of;
    for (int r = 0; r < (int)L.Tall.size(); ++r) row_of[L.Tall[r]] = r;
    L.psi_rows.clear();
    for (int b : L.Tpsi) {
      auto it = row_of.find(b);
      if (it == row_of.end()) {
        row_of[b] = (int)L.Tall.size();
        L.Tall.push_back(b);
      }
      L.psi_rows.push_back(row_of[b]);
    }
    L.nTall = (int)L.Tall.size();
    L.phi_oct.clear();
    for (int b : L.Tphi) L.phi_oct.push_back((uint8_t)~cov[k][b]);
    std::vector<int32_t> lists;
    L.off_SA = 0;
    lists.insert(lists.end(), L.SA.begin(), L.SA.end());
    L.off_SB = (int)lists.size();
    lists.insert(lists.end(), L.SB.begin(), L.SB.end());
    L.off_Tall = (int)lists.size();
    lists.insert(lists.end(), L.Tall.begin(), L.Tall.end());
    L.off_psi = (int)lists.size();
    lists.insert(lists.end(), L.psi_rows.begin(), L.psi_rows.end());
    L.off_Tpsi = (int)lists.size();
    lists.insert(lists.end(), L.Tpsi.begin(), L.Tpsi.end());
    L.off_HB = (int)lists.size();
    lists.insert(lists.end(), L.HB.begin(), L.HB.end());
    // LP: the coarse blocks under the SA blocks' interpolation stencils (parent cells and one more on each
    // side: coarse cells B c / 2 - 1 .. B c / 2 + B / 2 per axis), as they exist on level k - 1
    L.LP.clear();
    if (k >= 1) {
      const LevelPlan &Lc = P->L[k - 1];
      std::vector<char> need(Lc.BL.size(), 0);
      auto fdiv = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
      const int H = B / 2;
      for (int b : L.SA) {
        const int v[3] = {L.BL[b].x, L.BL[b].y, L.BL[b].z};
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) lo[a] = fdiv(v[a] * H - 1, B), hi[a] = fdiv(v[a] * H + H, B);
        for (int z = lo[2]; z <= hi[2]; ++z)
          for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
              const int bx = x - Lc.bb_lo[0], by = y - Lc.bb_lo[1], bz = z - Lc.bb_lo[2];
              if (bx < 0 || by < 0 || bz < 0 || bx >= Lc.bb_n[0] || by >= Lc.bb_n[1] || bz >= Lc.bb_n[2]) continue;
              const int i = Lc.map[((size_t)bz * Lc.bb_n[1] + by) * Lc.bb_n[0] + bx];
              if (i >= 0) need[i] = 1;
            }
      }
      for (int i = 0; i < (int)need.size(); ++i)
        if (need[i]) L.LP.push_back(i);
    }
    L.off_LP = (int)lists.size();
    lists.insert(lists.end(), L.LP.begin(), L.LP.end());
    // block-index FFT box
    {
      int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
      auto acc = [&](const std::vector<int32_t> &lst) {
        for (int b : lst) {
          const int v[3] = {L.BL[b].x, L.BL[b].y, L.BL[b].z};
          for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], v[a]), hi[a] = std::max(hi[a], v[a]);
        }
      };
      acc(L.SA);
      acc(L.SB);
      acc(L.Tall);
      L.box_ok = !L.Tall.empty();
      for (int a = 0; a < 3 && L.box_ok; ++a) {
        L.box_lo[a] = lo[a];
        L.box_nb[a] = hi[a] - lo[a] + 1;
        if (L.box_nb[a] < 1 || L.box_nb[a] > 16) L.box_ok = false;
      }
      if (L.box_ok) {
        L.nbox = (int64_t)L.box_nb[0] * L.box_nb[1] * L.box_nb[2];
        std::vector<int32_t> maps(4 * L.nbox, -1);
        auto put = [&](const std::vector<int32_t> &lst, int which) {
          for (int b : lst) {
            const int x = L.BL[b].x - lo[0], y = L.BL[b].y - lo[1], z = L.BL[b].z - lo[2];
            maps[which * L.nbox + ((int64_t)z * L.box_nb[1] + y) * L.box_nb[0] + x] = b;
          }
        };
        put(L.SA, 0);
        put(L.SB, 1);
        put(L.Tpsi, 2);
        put(L.Tphi, 3);
        int rc2 = upload(&L.d_box, maps, &P->device_bytes);
        if (rc2) {
          delete P;
          return rc2;
        }
      }
    }
    std::vector<int32_t> user_of(nBL, -1);
    for (int i = 0; i < L.nU; ++i) user_of[i] = (int32_t)(L.user_off + i);
    int rc;
    if ((rc = upload(&L.d_map, L.map, &P->device_bytes)) || (rc = upload(&L.d_BL, L.BL, &P->device_bytes)) ||
        (rc = upload(&L.d_cellmask, L.cellmask, &P->device_bytes)) ||
        (rc = upload(&L.d_octcov, L.octcov, &P->device_bytes)) ||
        (rc = upload(&L.d_lists, lists, &P->device_bytes)) ||
        (rc = upload(&L.d_phi_oct, L.phi_oct, &P->device_bytes)) ||
        (rc = upload(&L.d_user_of, user_of, &P->device_bytes))) {
      delete P;
      return rc;
    }
  }
  *out = P;
  return LGF_OK;
}

}  // namespace lgf
