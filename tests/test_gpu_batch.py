"""GPU tests of the batched stage (lgf_batch_*): uneven ring instances solved as one unit, the CUDA-graph
capture of chained stages, and parity of individual instances against the oracle (FLGF-AMR Sec. 3.4,
FIF-AMR Sec. 3.5)."""
import numpy as np
import pytest

import lgf_synth as S
from oracle import amr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALPHA = 0.1


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_13213_gb300.lgf as L
    L.load()
    return L


@pytest.fixture(scope="module")
def table8(L):
    t = L.lgf_table_create(8, (14, 14, 8), L.LGF_TBL_FP64 | L.LGF_TBL_DF32)
    yield t
    L.lgf_table_destroy(t)


def small_instances(n=8):
    out = []
    for p in S.batch_instances(n, B=8):
        q = dict(p)
        q["nxy"] = min(p["nxy"], 48)
        q["nz"] = max(32, 16 * int(np.ceil(q["nxy"] / 32)))
        q["h_fine"] = (2 * p["R"] + 8 * p["sigma"]) / q["nxy"]
        mesh, f, roles = S.ring_instance(q, B=8, n_ext=6)
        out.append((mesh, np.concatenate(f, axis=1), roles))
    return out


@pytest.fixture(scope="module")
def inst():
    return small_instances()


def make_batch(L, table, inst, precision=2):
    meshes = [L.Mesh(m["levels"], m["B"], m["h0"], n_ext=m["n_ext"]) for m, _, _ in inst]
    opts = L.make_opts(precision=precision)
    return L.Batch(table, meshes, 3, L.LGF_F64, alpha=[ALPHA] * len(inst), opts=opts, nstreams=4), meshes


def test_batch_stage_equals_individual_solves(L, table8, inst):
    b, meshes = make_batch(L, table8, inst)
    fs = [torch.from_numpy(f).cuda() for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    gs = [torch.zeros_like(f) for f in fs]
    s = torch.cuda.Stream()
    b.stage([f.data_ptr() for f in fs], [p.data_ptr() for p in phis], [g.data_ptr() for g in gs], s.cuda_stream)
    torch.cuda.synchronize()
    for i, (m, f) in enumerate(zip(meshes, fs)):
        phi = torch.zeros_like(f)
        g = torch.zeros_like(f)
        L.lgf_poisson_solve(table8, m, 3, f.data_ptr(), phi.data_ptr(), L.LGF_F64, L.make_opts(precision=2))
        L.lgf_heat_apply(table8, m, 3, f.data_ptr(), g.data_ptr(), L.LGF_F64, ALPHA, L.make_opts(precision=2))
        torch.cuda.synchronize()
        assert torch.equal(phi, phis[i]) and torch.equal(g, gs[i]), f"instance {i}"
    b.close()


def test_batch_instances_match_oracle(L, table8, inst):
    b, meshes = make_batch(L, table8, inst)
    fs = [torch.from_numpy(f).cuda() for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    gs = [torch.zeros_like(f) for f in fs]
    b.stage([f.data_ptr() for f in fs], [p.data_ptr() for p in phis], [g.data_ptr() for g in gs])
    torch.cuda.synchronize()
    checked = set()
    for i, (mesh, f, roles) in enumerate(inst):
        K = len(mesh["levels"])
        if K in checked or roles is not None:
            continue
        checked.add(K)
        fl, o = [], 0
        for blk in mesh["levels"]:
            fl.append(f[:, o:o + len(blk)])
            o += len(blk)
        ref, masks = amr.flgf_amr(mesh, fl)
        gref = amr.fif_amr(mesh, fl, ALPHA)
        got = phis[i].cpu().numpy()
        gg = gs[i].cpu().numpy()
        o = 0
        for k, blk in enumerate(mesh["levels"]):
            msk = masks[k]
            for c in range(2):
                r = ref[k][c][msk]
                assert np.abs(got[c, o:o + len(blk)][msk] - r).max() <= 1e-10 * np.abs(r).max()
                gr = gref[k][c][msk]
                assert np.abs(gg[c, o:o + len(blk)][msk] - gr).max() <= 1e-12 * np.abs(gr).max()
            o += len(blk)
    assert checked, "no multi-level instance in the batch"
    b.close()


def test_batch_graph_replays_chained_stages(L, table8, inst):
    b, meshes = make_batch(L, table8, inst)
    fs = [torch.from_numpy(f).cuda() for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    gs = [torch.zeros_like(f) for f in fs]
    tmps = [torch.zeros_like(f) for f in fs]
    s = torch.cuda.Stream()
    ptr = lambda ts: [t.data_ptr() for t in ts]
    b.graph_create(3, ptr(fs), ptr(phis), ptr(gs), ptr(tmps), s.cuda_stream)
    assert b.graph_nodes() > 3 * len(inst)
    for t in phis + gs + tmps:
        t.zero_()
    torch.cuda.synchronize()
    b.graph_launch(s.cuda_stream)
    torch.cuda.synchronize()
    # eager chain: f -> (phi, g); g -> (phi, tmp); tmp -> (phi, g)
    for i, (m, f) in enumerate(zip(meshes, fs)):
        g1, g2, phi = torch.zeros_like(f), torch.zeros_like(f), torch.zeros_like(f)
        src = f
        for dst in (g1, g2, g1):
            L.lgf_poisson_solve(table8, m, 3, src.data_ptr(), phi.data_ptr(), L.LGF_F64, L.make_opts(precision=2))
            L.lgf_heat_apply(table8, m, 3, src.data_ptr(), dst.data_ptr(), L.LGF_F64, ALPHA, L.make_opts(precision=2))
            src = dst
        torch.cuda.synchronize()
        assert torch.equal(phi, phis[i]), f"phi instance {i}"
        assert torch.equal(g1, gs[i]), f"g instance {i}"
    b.close()


def test_batch_graph_with_per_stage_alpha(L, table8, inst):
    # the integrating-factor argument of a HERK stage is (c~_i - c~_{i-1}) dt kappa / dx^2 (Eq.
    # (eq:composite-LGF-IF)), so it differs between the stages of one step
    b, meshes = make_batch(L, table8, inst)
    fs = [torch.from_numpy(f).cuda() for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    gs = [torch.zeros_like(f) for f in fs]
    tmps = [torch.zeros_like(f) for f in fs]
    s = torch.cuda.Stream()
    ptr = lambda ts: [t.data_ptr() for t in ts]
    stage_alpha = [0.1 / 3.0, 0.2 / 3.0, 0.05]
    table = [[a * (1.0 + 0.1 * i) for i in range(len(inst))] for a in stage_alpha]
    b.graph_create(3, ptr(fs), ptr(phis), ptr(gs), ptr(tmps), s.cuda_stream, alpha_stages=table)
    for t in phis + gs + tmps:
        t.zero_()
    torch.cuda.synchronize()
    b.graph_launch(s.cuda_stream)
    torch.cuda.synchronize()
    for i, (m, f) in enumerate(zip(meshes, fs)):
        g1, g2, phi = torch.zeros_like(f), torch.zeros_like(f), torch.zeros_like(f)
        src = f
        for st, dst in enumerate((g1, g2, g1)):
            L.lgf_poisson_solve(table8, m, 3, src.data_ptr(), phi.data_ptr(), L.LGF_F64, L.make_opts(precision=2))
            L.lgf_heat_apply(table8, m, 3, src.data_ptr(), dst.data_ptr(), L.LGF_F64, table[st][i],
                             L.make_opts(precision=2))
            src = dst
        torch.cuda.synchronize()
        assert torch.equal(g1, gs[i]), f"g instance {i}"
        assert torch.equal(g2, tmps[i]), f"tmp instance {i}"
        assert torch.equal(phi, phis[i]), f"phi instance {i}"
    b.close()


def test_batch_poisson_only_graph(L, table8, inst):
    b, meshes = make_batch(L, table8, inst)
    fs = [torch.from_numpy(f).cuda() for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    s = torch.cuda.Stream()
    ptr = lambda ts: [t.data_ptr() for t in ts]
    b.graph_create(2, ptr(fs), ptr(phis), None, None, s.cuda_stream)
    for t in phis:
        t.zero_()
    torch.cuda.synchronize()
    b.graph_launch(s.cuda_stream)
    torch.cuda.synchronize()
    for i, (m, f) in enumerate(zip(meshes, fs)):
        phi = torch.zeros_like(f)
        L.lgf_poisson_solve(table8, m, 3, f.data_ptr(), phi.data_ptr(), L.LGF_F64, L.make_opts(precision=2))
        torch.cuda.synchronize()
        assert torch.equal(phi, phis[i]), f"phi instance {i}"
    b.close()


def test_batch_rejects_mismatched_block_size(L, table8):
    m16 = L.Mesh([S.box_blocks((32, 32, 32), 16)], 16, 1.0)
    with pytest.raises(L.LgfError) as e:
        L.Batch(table8, [m16], 1)
    assert e.value.status == L.LGF_E_MESH


def test_batch_autotune_choices_and_results(L, table8, inst):
    # the autotuner times each instance's DFT-pass variants and the stream counts; afterwards every stage
    # reproduces the individual solves made with the chosen variant bit for bit, and stays within the
    # DF32 accuracy of the untuned ones
    b, meshes = make_batch(L, table8, inst)
    fs = [torch.from_numpy(f).cuda() for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    s = torch.cuda.Stream()
    ptr = lambda ts: [t.data_ptr() for t in ts]
    b.autotune(ptr(fs), ptr(phis), s.cuda_stream)
    ns, slices, ms = b.tuning()
    assert ns in (1, 2, 4, 8) and all(x in (0, 5) for x in slices) and all(m > 0 for m in ms)
    b.graph_create(1, ptr(fs), ptr(phis), None, None, s.cuda_stream)
    for t in phis:
        t.zero_()
    torch.cuda.synchronize()
    b.graph_launch(s.cuda_stream)
    torch.cuda.synchronize()
    for i, (m, f) in enumerate(zip(meshes, fs)):
        phi = torch.zeros_like(f)
        L.lgf_poisson_solve(table8, m, 3, f.data_ptr(), phi.data_ptr(), L.LGF_F64,
                            L.make_opts(precision=2, dft_slices=slices[i]))
        ref = torch.zeros_like(f)
        L.lgf_poisson_solve(table8, m, 3, f.data_ptr(), ref.data_ptr(), L.LGF_F64, L.make_opts(precision=2))
        torch.cuda.synchronize()
        assert torch.equal(phi, phis[i]), f"instance {i}"
        assert (phi - ref).abs().max() <= 1e-10 * ref.abs().max()
    b.close()


def test_graph_with_host_transfers_matches_device_graph(L, table8, inst):
    """lgf_batch_graph_create_io: the sources come from pinned host memory and the results go back to it
    inside the graph; the results equal those of the device-only graph, bit for bit, on every replay."""
    b, meshes = make_batch(L, table8, inst)
    host_f = [torch.from_numpy(f).pin_memory() for _, f, _ in inst]
    host_phi = [torch.full_like(h, float("nan")).pin_memory() for h in host_f]
    dev_f = [torch.zeros(h.shape, dtype=h.dtype, device="cuda") for h in host_f]
    dev_phi = [torch.zeros_like(d) for d in dev_f]
    s = torch.cuda.Stream()
    ptr = lambda ts: [t.data_ptr() for t in ts]
    b.graph_create_io(ptr(host_f), ptr(host_phi), ptr(dev_f), ptr(dev_phi), s.cuda_stream)
    ref_f = [h.cuda() for h in host_f]
    ref_phi = [torch.zeros_like(d) for d in ref_f]
    b2, _ = make_batch(L, table8, inst)
    b2.graph_create(1, ptr(ref_f), ptr(ref_phi), None, None, s.cuda_stream)
    b2.graph_launch(s.cuda_stream)
    s.synchronize()
    for rep in range(2):
        for h in host_phi:
            h.fill_(float("nan"))
        for d in dev_f:
            d.zero_()
        torch.cuda.synchronize()
        b.graph_launch(s.cuda_stream)
        s.synchronize()
        for i in range(len(inst)):
            assert torch.equal(host_phi[i], ref_phi[i].cpu()), (rep, i)
    b.close()
    b2.close()


def test_graph_with_host_transfers_rejects_pageable_memory(L, table8, inst):
    b, _ = make_batch(L, table8, inst)
    pageable = [torch.from_numpy(f.copy()) for _, f, _ in inst]
    dev = [torch.zeros(h.shape, dtype=h.dtype, device="cuda") for h in pageable]
    ptr = lambda ts: [t.data_ptr() for t in ts]
    s = torch.cuda.Stream()
    with pytest.raises(L.LgfError) as e:
        b.graph_create_io(ptr(pageable), ptr(pageable), ptr(dev), ptr(dev), s.cuda_stream)
    assert e.value.status == L.LGF_E_INVALID_ARG
    b.close()
