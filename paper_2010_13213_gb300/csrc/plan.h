// plan.h -- host plan of a composite-mesh solve: regions, block sets and their device copies.
//
// Regions (Sec. 3.1-3.4; every set is a set of level-k cells):
//   UB_k  cells of the caller's level-k blocks
//   OM_k  Omega_k = UB_k minus the cells covered by level-(k+1) blocks (Eq. (eq:partition))
//   COV_k UB_k cells covered by level k+1 (where the coarsened finer sources live)
//   EX_k  Omega_k^E = cells within n_ext (max-norm) of OM_k and not in OM_k (Eq. (eq:extended_regions)), k >= 1
//   SR_k  OM_k u EX_k: where the correction source S psi_{k-1} is kept (k >= 1); OM_0 for k = 0
//   NP_k  cells of level k where psi_k is needed by level k+1:
//         NP_k = dilate(footprint(C_{k+1}), 2), C_k = cells(T_phi u T_psi blocks) u dilate(SR_k, 1)
//   HR_k  dilate(OM_k, r_k): where the heat apply needs P_k fhat (Sec. 3.5)
//   NU_k  cells where the cumulative interpolation U_k is needed: dilate(footprint(HR_{k+1} u NU_{k+1}), 1)
// Block sets are the blocks intersecting these cell sets; per-cell masks carry the exact regions
// into the kernels (bit 1: OM, bit 2: EX, bit 4: COV).
#pragma once
#include <cstdint>
#include <vector>

#include "internal.h"

namespace lgf {

enum CellBits : uint8_t { CB_OM = 1, CB_EX = 2, CB_COV = 4 };

struct LevelPlan {
  int k = 0;
  int64_t user_off = 0;            // first block of this level in the caller's arrays
  int nU = 0;                      // caller blocks of this level
  // internal block set BL (caller blocks first, in caller order, then added blocks)
  std::vector<int4> BL;            // block coords
  int bb_lo[3] = {0, 0, 0}, bb_n[3] = {0, 0, 0};  // block-coordinate box of the block map
  std::vector<int32_t> map;        // [bb_n z][y][x] -> BL index or -1
  std::vector<uint8_t> cellmask;   // [nBL][B^3] CellBits
  std::vector<uint8_t> octcov;     // [nBL] covered octants (bit o = octant (x>=B/2)+2(y>=B/2)+4(z>=B/2))
  std::vector<int32_t> SA, SB, Tphi, Tpsi;  // lists of BL indices (Poisson)
  std::vector<int32_t> HB;         // heat block set (BL indices)
  std::vector<int32_t> LP;         // k >= 1: level-(k-1) BL indices whose L_{k-1} psi_{k-1} the correction of
                                   // the SA blocks reads (the coarse cubes k_correct stages)
  std::vector<uint8_t> phi_oct;    // [|Tphi|] octants of Omega_k (write mask)
  // device copies
  int32_t *d_map = nullptr;
  int4 *d_BL = nullptr;
  uint8_t *d_cellmask = nullptr;
  uint8_t *d_octcov = nullptr;
  int32_t *d_lists = nullptr;      // SA | SB | Tall(=Tphi then Tpsi\Tphi) | psi rows | Tpsi | HB | LP
  uint8_t *d_phi_oct = nullptr;
  int32_t *d_user_of = nullptr;    // [nBL] global caller block index or -1
  std::vector<int32_t> Tall;       // Tphi then Tpsi minus Tphi
  std::vector<int32_t> psi_rows;   // rows of Tall that are psi targets
  int nTall = 0;
  int off_SA = 0, off_SB = 0, off_Tall = 0, off_psi = 0, off_Tpsi = 0, off_HB = 0, off_LP = 0;
  int heat_r = 0;                  // heat kernel radius at this level
  int64_t n_omega = 0;             // |Omega_k| in cells
  int64_t n_src = 0;               // cells carrying a source of the level's convolutions (OM, EX or COV)
  // block-index FFT mode: box over SA u SB u Tall and its maps (box block -> BL index or -1)
  bool box_ok = false;
  int box_lo[3] = {0, 0, 0}, box_nb[3] = {0, 0, 0};
  int32_t *d_box = nullptr;        // [4][nbox]: gather A (SA), gather B (SB), scatter psi (Tpsi), scatter phi (Tphi)
  int64_t nbox = 0;
};

struct Plan {
  int B = 0, K = 0, n_ext = 0;
  bool heat = false;
  double alpha = 0.0;
  std::vector<LevelPlan> L;
  size_t device_bytes = 0;
  ~Plan();
};

// Builds the plan (host) and uploads it.  `heat_radii` may be null (Poisson plan).
int build_plan(const lgf_mesh *m, const int *heat_radii, Plan **out);

}  // namespace lgf
