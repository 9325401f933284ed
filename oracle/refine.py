"""Refinement indicator of the adaptive mesh (Sec. 4.2, Eqs. (eq:refine1), (eq:maximumS), (eq:refine2))
from the combined source S_k of Eq. (eq:combined_source).

TEST INFRASTRUCTURE ONLY (see the package docstring).

S_k = S_{k-1->k} psi_{k-1} + sum_{i >= k} P_{i->k} fhat_i is the source each level's LGF solve sees in
Eq. (eq:combine_S): F_0 on level 0, the correction s (on Omega_k and Omega_k^E) plus F_k on level k >= 1,
taken from ``amr.flgf_amr``.  A point of level k is refined where S_k > alpha^(N_l - k) S_max and
coarsened where S_k < beta alpha^(N_l - k) S_max, S_max being the largest block RMS of S up to now.

Readings (the paper states the criteria per point and the maximum per block, for a vector source):
* |S_k(n)| is the Euclidean norm over the components; the block RMS is sqrt(mean |S_k|^2) over all B^3
  cells of a level-k block (cells that a finer level covers carry the coarsened finer sources).
* A level-k block is flagged for refinement when |S_k| exceeds the level's threshold at one of its
  cells, for coarsening when |S_k| is below beta times the threshold at all of them.
* Cells of Omega_k^E outside the level-k blocks flag the level-(k-1) block that holds their parent
  cell for refinement when |S_k| exceeds the level-k threshold there.
* S_max is the largest block RMS over the levels now and the value carried from earlier times
  (``s_max_prev``), Eq. (eq:maximumS); N_l is the prescribed maximum level index.

Pins (tests/test_oracle_refine.py): block RMS against sums over the caller's input arrays (one level;
two levels with no coarse source, where S_1 is the fine input and S_0 its 8-child mean), scale
invariance of the flags, S_max carried over time, refine and coarsen never both set, and the extended
region flagging exactly the level-0 blocks under it (a mesh whose expected block set is written out in
block coordinates).
"""
import numpy as np

from .amr import flgf_amr


def combined_sources(mesh, f_levels):
    """S_k on each level's dense box ([ncomp][nz][ny][nx]), with the level boxes and the per-level
    correction internals of the FLGF-AMR oracle."""
    _, _, it = flgf_amr(mesh, f_levels, return_internals=True)
    F, steps = it["F"], it["steps"]
    S = [F[0]] + [steps[k - 1]["s"] + F[k] for k in range(1, len(F))]
    return S, it["levels"], steps


def refinement_indicator(mesh, f_levels, alpha, beta, n_levels_max, s_max_prev=0.0):
    """Per level and block: the RMS of |S_k|, the refine and coarsen flags; and S_max."""
    S, lv, steps = combined_sources(mesh, f_levels)
    B = mesh["B"]
    mag = [np.sqrt((s ** 2).sum(axis=0)) for s in S]
    rms = [np.array([np.sqrt(np.mean(mag[k][lv[k].block_slice(b, B)] ** 2)) for b in blocks])
           for k, blocks in enumerate(mesh["levels"])]
    s_max = max([float(s_max_prev)] + [float(r.max()) for r in rms])
    thr = [alpha ** (n_levels_max - k) * s_max for k in range(len(mesh["levels"]))]
    refine = [np.array([bool((mag[k][lv[k].block_slice(b, B)] > thr[k]).any()) for b in blocks])
              for k, blocks in enumerate(mesh["levels"])]
    coarsen = [np.array([bool((mag[k][lv[k].block_slice(b, B)] < beta * thr[k]).all()) for b in blocks])
               for k, blocks in enumerate(mesh["levels"])]
    for k in range(1, len(mesh["levels"])):
        hot = steps[k - 1]["ext"] & ~lv[k].user & (mag[k] > thr[k])
        parents = {tuple(int(c) for c in b): i for i, b in enumerate(np.asarray(mesh["levels"][k - 1]))}
        for z, y, x in zip(*np.nonzero(hot)):
            cell = (lv[k].origin[0] + x, lv[k].origin[1] + y, lv[k].origin[2] + z)  # level-k cell index
            i = parents.get(tuple((c // 2) // B for c in cell))
            if i is not None:
                refine[k - 1][i] = True
    return dict(rms=rms, s_max=s_max, refine=refine, coarsen=coarsen)
