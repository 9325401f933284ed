"""Full-size workloads on the GPU against the oracle: the three-level ring composite mesh (h = R/16, R/32,
R/64; 100 / 128 / 424 blocks of 16^3), the two coaxial rings (96x96x112 cells), and the uneven batch of
64 ring instances (1-3 levels, finest boxes 32..192 cells) run as one captured stage."""
import numpy as np
import pytest

import lgf_synth as S
import oracle
from oracle import amr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_13213_gb300.lgf as L
    L.load()
    return L


@pytest.fixture(scope="module")
def tbox(L):
    t = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    yield t
    L.lgf_table_destroy(t)


def level_errors(got, ref, masks, levels, comps=(0, 1)):
    errs, o = [], 0
    for k, blk in enumerate(levels):
        m = masks[k]
        for c in comps:
            r = ref[k][c][m]
            errs.append(float(np.abs(got[c, o:o + len(blk)][m] - r).max() / np.abs(r).max()))
        o += len(blk)
    return errs


@pytest.fixture(scope="module")
def ring3_full():
    mesh, f = S.three_level_ring()
    ref, masks = amr.flgf_amr(mesh, f)
    return mesh, f, ref, masks


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-10)])
def test_three_level_ring_full(L, tbox, ring3_full, precision, tol):
    mesh, f, ref, masks = ring3_full
    m = L.Mesh(mesh["levels"], 16, mesh["h0"], n_ext=mesh["n_ext"])
    ft = torch.from_numpy(np.concatenate(f, axis=1)).cuda()
    phi = torch.full_like(ft, float("nan"))
    rep = L.lgf_report()
    L.lgf_poisson_solve(tbox, m, 3, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=precision, residual=1), rep)
    torch.cuda.synchronize()
    got = phi.cpu().numpy()
    errs = level_errors(got, ref, masks, mesh["levels"])
    assert max(errs) <= tol, errs
    assert rep.mac_mode_used == L.LGF_MAC_BOX
    assert rep.target_cells == sum(int(x.sum()) for x in masks)
    assert rep.residual_rel < (1e-8 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-10), (1, 1e-5)])
def test_two_coaxial_rings(L, tbox, precision, tol):
    case = S.two_ring_single_level()
    ref = oracle.solve_box_fft(case["box"][:2], case["h"])
    m = L.Mesh([case["blocks"]], 16, case["h"])
    ft = torch.from_numpy(case["f"]).cuda()
    phi = torch.full_like(ft, float("nan"))
    L.lgf_poisson_solve(tbox, m, 3, ft.data_ptr(), phi.data_ptr(), L.LGF_F64, L.make_opts(precision=precision))
    torch.cuda.synchronize()
    got = S.blocks_to_box(phi.cpu().numpy(), case["blocks"], 16, case["shape"])
    for c in range(2):
        assert np.abs(got[c] - ref[c]).max() <= tol * np.abs(ref[c]).max()
    assert np.abs(got[2]).max() == 0.0


def test_batch_of_64_uneven_instances(L, tbox):
    params = S.batch_instances(64, B=16)
    inst = [S.ring_instance(p, B=16, n_ext=16) for p in params]
    meshes = [L.Mesh(mh["levels"], 16, mh["h0"], n_ext=16) for mh, _, _ in inst]
    fs = [torch.from_numpy(np.concatenate(f, axis=1)).cuda() for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    gs = [torch.zeros_like(f) for f in fs]
    tmps = [torch.zeros_like(f) for f in fs]
    b = L.Batch(tbox, meshes, 3, L.LGF_F64, alpha=[0.1] * 64, opts=L.make_opts(precision=2), nstreams=8)
    s = torch.cuda.Stream()
    ptr = lambda ts: [t.data_ptr() for t in ts]
    b.stage(ptr(fs), ptr(phis), ptr(gs), s.cuda_stream)
    torch.cuda.synchronize()
    # oracle parity on the smallest instance of each level count
    chosen = {}
    for i, (mh, f, roles) in enumerate(inst):
        K = len(mh["levels"])
        size = sum(len(x) for x in mh["levels"])
        if roles is None and (K not in chosen or size < chosen[K][1]):
            chosen[K] = (i, size)
    assert len(chosen) >= 2
    for K, (i, _) in chosen.items():
        mh, fl, _ = inst[i]
        ref, masks = amr.flgf_amr(mh, fl)
        errs = level_errors(phis[i].cpu().numpy(), ref, masks, mh["levels"])
        assert max(errs) <= 1e-10, (K, errs)
    # the captured three-stage graph reproduces the eager chain
    b.graph_create(3, ptr(fs), ptr(phis), ptr(gs), ptr(tmps), s.cuda_stream)
    b.graph_launch(s.cuda_stream)
    torch.cuda.synchronize()
    for i in (0, 63):
        g1, g2, phi = torch.zeros_like(fs[i]), torch.zeros_like(fs[i]), torch.zeros_like(fs[i])
        src = fs[i]
        for dst in (g1, g2, g1):
            L.lgf_poisson_solve(tbox, meshes[i], 3, src.data_ptr(), phi.data_ptr(), L.LGF_F64, L.make_opts(precision=2))
            L.lgf_heat_apply(tbox, meshes[i], 3, src.data_ptr(), dst.data_ptr(), L.LGF_F64, 0.1, L.make_opts(precision=2))
            src = dst
        torch.cuda.synchronize()
        assert torch.equal(phi, phis[i]) and torch.equal(g1, gs[i])
    b.close()
