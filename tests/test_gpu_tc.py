"""GPU parity of the tensor-core DFT-GEMM: the block-index DFT passes of the box mode run as BF16 x BF16
-> FP32 tcgen05 GEMMs with split-precision digit slices (opts.dft_slices), against the CPU oracle
(lattice convolution, Sec. 2.2) and against the CUDA-core passes.  The error of a pass is about
2^-(7+8(S-1)) of each cell line's largest value, so the tolerances below follow the slice count; the
tables printed per field are the precision study of the two-ring workload (error vs the FP64 oracle)."""
import numpy as np
import pytest

import lgf_synth as S
import oracle
from oracle import amr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# relative L-infinity bound per (precision, slices); the pass error 2^-(7+8(S-1)) times a margin for
# six passes and the local FFTs
TOL = {(1, 1): 3e-2, (1, 2): 2e-4, (1, 3): 2e-5, (2, 4): 5e-8, (2, 5): 1e-10, (2, 6): 1e-12}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_13213_gb300.lgf as L
    L.load()
    return L


@pytest.fixture(scope="module")
def tables(L):
    t16 = L.lgf_table_create(16, (6, 6, 6), L.LGF_TBL_FP64 | L.LGF_TBL_FP32 | L.LGF_TBL_DF32)
    t8 = L.lgf_table_create(8, (14, 14, 8), L.LGF_TBL_BOX_ONLY)
    yield {16: t16, 8: t8}
    L.lgf_table_destroy(t16)
    L.lgf_table_destroy(t8)


def solve(L, table, levels, B, h, f_blocks, precision, slices, n_ext=16, rep=None, mode=None):
    m = L.Mesh(levels, B, h, n_ext=n_ext)
    f = torch.from_numpy(np.ascontiguousarray(f_blocks)).cuda()
    phi = torch.full_like(f, float("nan"))
    mode = L.LGF_MAC_BOX if mode is None else mode
    L.lgf_poisson_solve(table, m, f.shape[0], f.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=precision, mac_mode=mode, dft_slices=slices), rep)
    torch.cuda.synchronize()
    return phi.cpu().numpy()


def rel(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("precision,slices", sorted(TOL))
def test_tc_random_32cube(L, tables, precision, slices):
    case = S.single_level_random(n=32, B=16, seed=3, ncomp=3)
    ref = oracle.solve_box_fft(case["box"], case["h"])
    rep = L.lgf_report()
    phi = solve(L, tables[16], [case["blocks"]], 16, case["h"], case["f"], precision, slices, rep=rep)
    got = S.blocks_to_box(phi, case["blocks"], 16, case["shape"])
    assert rep.mac_mode_used == L.LGF_MAC_BOX
    errs = [rel(got[c], ref[c]) for c in range(3)]
    assert max(errs) <= TOL[(precision, slices)], errs
    L.lgf_device_status(tables[16])


@pytest.mark.parametrize("slices", [5, 6])
def test_tc_ring_matches_cuda_core_passes(L, tables, slices):
    """cfg: ring 96x96x48 (3 components: one complex field + one Hermitian-half real field)."""
    case = S.single_level_ring()
    ref = oracle.solve_box_fft(case["box"], case["h"])
    tc = solve(L, tables[16], [case["blocks"]], 16, case["h"], case["f"], 2, slices)
    cc = solve(L, tables[16], [case["blocks"]], 16, case["h"], case["f"], 2, 0)
    for c in range(2):
        r = S.blocks_to_box(tc, case["blocks"], 16, case["shape"])[c]
        assert rel(r, ref[c]) <= TOL[(2, slices)]
        assert rel(tc[c], cc[c]) <= TOL[(2, slices)]
    assert np.abs(tc[2]).max() == 0.0


def test_tc_block8_uneven_box(L, tables):
    """B = 8 and an uneven box (5 x 3 x 2 blocks, so P = 10 x 6 x 4) with a ragged-support source."""
    shape = (16, 24, 40)
    box = S.random_box(shape, 11, 2)
    blocks = S.box_blocks(shape, 8)
    ref = oracle.solve_box_fft(box, 0.5)
    for prec, sl in ((2, 5), (1, 3)):
        phi = solve(L, tables[8], [blocks], 8, 0.5, S.box_to_blocks(box, blocks, 8), prec, sl)
        got = S.blocks_to_box(phi, blocks, 8, shape)
        for c in range(2):
            assert rel(got[c], ref[c]) <= TOL[(prec, sl)]


def test_tc_three_level_ring(L):
    """Composite 3-level ring: complex A + i(A+B) packing, masked gathers, addends and masked scatters."""
    mesh, f = S.three_level_ring()
    ref, masks = amr.flgf_amr(mesh, f)
    t = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    try:
        m = L.Mesh(mesh["levels"], 16, mesh["h0"], n_ext=mesh["n_ext"])
        ft = torch.from_numpy(np.concatenate(f, axis=1)).cuda()
        phi = torch.full_like(ft, float("nan"))
        rep = L.lgf_report()
        L.lgf_poisson_solve(t, m, 3, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                            L.make_opts(precision=2, dft_slices=5, residual=1), rep)
        got = phi.cpu().numpy()
        o = 0
        for k, blk in enumerate(mesh["levels"]):
            for c in range(2):
                r = ref[k][c][masks[k]]
                assert np.abs(got[c, o:o + len(blk)][masks[k]] - r).max() <= 1e-10 * np.abs(r).max()
            o += len(blk)
        # the FP64 residual L phi - f amplifies the solution's error by the stencil's 12 / h^2 over the
        # source magnitude: about 1e6 here (FP64 gives ~1e-9, DF32 ~1e-7), so ~1e-11 error -> ~1e-5
        assert rep.residual_rel < 1e-4
    finally:
        L.lgf_table_destroy(t)


def test_tc_two_rings_error_table(L, capsys):
    """Precision study of the two coaxial rings: error per field for every slice count."""
    case = S.two_ring_single_level()
    ref = oracle.solve_box_fft(case["box"][:2], case["h"])
    t = L.lgf_table_create(16, (6, 6, 7), L.LGF_TBL_BOX_ONLY)
    rows = []
    try:
        for prec, sl in sorted(TOL):
            phi = solve(L, t, [case["blocks"]], 16, case["h"], case["f"], prec, sl)
            got = S.blocks_to_box(phi, case["blocks"], 16, case["shape"])
            errs = [rel(got[c], ref[c]) for c in range(2)]
            rows.append((prec, sl, errs))
            assert max(errs) <= TOL[(prec, sl)], (prec, sl, errs)
        # more slices never hurt within an arithmetic
        for p in (1, 2):
            e = [max(r[2]) for r in rows if r[0] == p]
            assert all(a >= b for a, b in zip(e, e[1:])), e
    finally:
        L.lgf_table_destroy(t)
    with capsys.disabled():
        for prec, sl, errs in rows:
            print(f"\n two rings  {'FP32' if prec == 1 else 'DF32'} x {sl} BF16 slices: "
                  f"omega_x {errs[0]:.2e}  omega_y {errs[1]:.2e}", end="")


def test_tc_rejects_bad_slices(L, tables):
    case = S.single_level_random(n=32, B=16, seed=1, ncomp=1)
    for prec, sl in ((0, 5), (1, 4), (2, 3), (2, 7)):
        with pytest.raises(L.LgfError) as e:
            solve(L, tables[16], [case["blocks"]], 16, case["h"], case["f"], prec, sl)
        assert e.value.status in (L.LGF_E_INVALID_ARG, L.LGF_E_UNSUPPORTED)


def test_bounded_wait_gives_up_and_context_survives(L, tables):
    """A wait on an mbarrier nothing arrives at (limit 2^24 cycles) reports LGF_E_TIMEOUT through the
    status word; the word clears and the next solve is unaffected."""
    L.lgf_device_status(tables[16])  # clean start
    L.lgf_selftest_wait_timeout(tables[16], 24)
    with pytest.raises(L.LgfError) as e:
        L.lgf_device_status(tables[16])
    assert e.value.status == L.LGF_E_TIMEOUT
    L.lgf_device_status(tables[16])  # cleared
    case = S.single_level_random(n=32, B=16, seed=5, ncomp=2)
    ref = oracle.solve_box_fft(case["box"], case["h"])
    phi = solve(L, tables[16], [case["blocks"]], 16, case["h"], case["f"], 2, 5)
    got = S.blocks_to_box(phi, case["blocks"], 16, case["shape"])
    assert max(rel(got[c], ref[c]) for c in range(2)) <= TOL[(2, 5)]
    L.lgf_device_status(tables[16])
