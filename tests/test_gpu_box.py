"""GPU parity of the block-index FFT mode (LGF_MAC_BOX): the per-frequency block-pair sums evaluated
through a zero-padded DFT over each level's block grid, against the CPU oracle and against the
direct pair mode (both are exact evaluations of the same lattice convolution, Sec. 2.2)."""
import numpy as np
import pytest

import lgf_synth as S
import oracle
from oracle import amr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 2: 1e-10, 1: 2e-5}


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
    t8 = L.lgf_table_create(8, (14, 14, 8), L.LGF_TBL_FP64 | L.LGF_TBL_FP32 | L.LGF_TBL_DF32)
    yield {16: t16, 8: t8}
    L.lgf_table_destroy(t16)
    L.lgf_table_destroy(t8)


def solve(L, table, mesh_levels, B, h, f_blocks, precision, mode, roles=None, n_ext=16, dtype=0, rep=None):
    m = L.Mesh(mesh_levels, B, h, n_ext=n_ext, roles=roles)
    tdt = torch.float64 if dtype == 0 else torch.float32
    f = torch.from_numpy(f_blocks).to("cuda", tdt)
    phi = torch.full_like(f, float("nan"))
    L.lgf_poisson_solve(table, m, f.shape[0], f.data_ptr(), phi.data_ptr(), dtype,
                        L.make_opts(precision=precision, mac_mode=mode), rep)
    torch.cuda.synchronize()
    return phi.double().cpu().numpy()


def rel(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("precision", [0, 2, 1])
@pytest.mark.parametrize("ncomp", [1, 3])
def test_box_random_32cube(L, tables, precision, ncomp):
    case = S.single_level_random(n=32, B=16, seed=ncomp, ncomp=ncomp)
    ref = oracle.solve_box_fft(case["box"], case["h"])
    rep = L.lgf_report()
    phi = solve(L, tables[16], [case["blocks"]], 16, case["h"], case["f"], precision, L.LGF_MAC_BOX, rep=rep)
    got = S.blocks_to_box(phi, case["blocks"], 16, case["shape"])
    assert rep.mac_mode_used == L.LGF_MAC_BOX
    for c in range(ncomp):
        assert rel(got[c], ref[c]) <= TOL[precision]


def test_box_ragged_roles_B8(L, tables):
    rng = np.random.default_rng(44)
    blocks = np.array([[0, 0, 0], [1, 0, 0], [3, 1, 0], [0, 2, 1], [2, 2, 1], [4, 0, 2], [1, 3, 2],
                       [3, 3, 0], [0, 1, 3], [2, 0, 3], [4, 3, 3]], np.int32)
    roles = np.array([3, 1, 2, 3, 1, 2, 3, 3, 1, 2, 3], np.uint8)
    B, h = 8, 0.25
    f = rng.standard_normal((3, len(blocks), B, B, B))
    pair = solve(L, tables[8], [blocks], B, h, f, 0, L.LGF_MAC_PAIR, roles=roles)
    box = solve(L, tables[8], [blocks], B, h, f, 0, L.LGF_MAC_BOX, roles=roles)
    tg = (roles & 2) > 0
    assert rel(box[:, tg], pair[:, tg]) <= 1e-12
    assert np.isnan(box[:, ~tg]).all()
    # and against the direct-sum oracle
    src_b = blocks[(roles & 1) > 0]
    sxyz = np.concatenate([oracle.core.box_cells((B, B, B), tuple(B * b)) for b in src_b])
    txyz = np.concatenate([oracle.core.box_cells((B, B, B), tuple(B * b)) for b in blocks[tg]])
    ref = oracle.direct_conv(oracle.lgf_octant(48), sxyz, f[:, (roles & 1) > 0].reshape(3, -1), txyz, h * h)
    assert rel(box[:, tg].reshape(3, -1), ref) <= 1e-12


@pytest.mark.parametrize("precision", [0, 2])
def test_box_ring_96x96x48(L, tables, precision):
    case = S.single_level_ring()
    ref = oracle.solve_box_fft(case["box"], case["h"])
    phi = solve(L, tables[16], [case["blocks"]], 16, case["h"], case["f"], precision, L.LGF_MAC_BOX)
    got = S.blocks_to_box(phi, case["blocks"], 16, case["shape"])
    for c in range(2):
        assert rel(got[c], ref[c]) <= TOL[precision]
    assert np.abs(got[2]).max() == 0.0


def _flat(fl):
    return np.concatenate(fl, axis=1)


def _split(a, levels):
    out, o = [], 0
    for b in levels:
        out.append(a[:, o:o + len(b)])
        o += len(b)
    return out


@pytest.mark.parametrize("precision", [0, 2])
def test_box_two_level(L, tables, precision):
    B = 8
    levels = [S.box_blocks((24, 24, 24), B), np.array([[2, 2, 2], [3, 2, 2], [2, 3, 2], [3, 3, 2], [2, 2, 3]], np.int32)]
    mesh = dict(B=B, h0=0.5, n_ext=4, levels=levels)
    rng = np.random.default_rng(12)
    f = [rng.standard_normal((2, len(b), B, B, B)) for b in levels]
    ref, masks = amr.flgf_amr(mesh, f)
    phi = _split(solve(L, tables[8], levels, B, 0.5, _flat(f), precision, L.LGF_MAC_BOX, n_ext=4), levels)
    for g, r, msk in zip(phi, ref, masks):
        assert rel(g[:, msk], r[:, msk]) <= TOL[precision]


def test_box_three_level_ring_matches_pair(L, tables):
    mesh, f = S.three_level_ring(R=1.0, sigma=0.2, B=8, n_ext=6, h_fine=1 / 32, support=(24, 24, 16), dilate0=1)
    levels = mesh["levels"]
    ref, masks = amr.flgf_amr(mesh, f)
    box = _split(solve(L, tables[8], levels, 8, mesh["h0"], _flat(f), 0, L.LGF_MAC_BOX, n_ext=6), levels)
    auto_rep = L.lgf_report()
    auto = _split(solve(L, tables[8], levels, 8, mesh["h0"], _flat(f), 2, L.LGF_MAC_AUTO, n_ext=6, rep=auto_rep),
                  levels)
    for g, a, r, msk in zip(box, auto, ref, masks):
        for c in range(2):
            assert rel(g[c][msk], r[c][msk]) <= 1e-12
            assert rel(a[c][msk], r[c][msk]) <= 1e-10


@pytest.mark.parametrize("mode", ["box", "pair"])
def test_df32_field_conversions_across_exponents(L, tables, mode):
    """Double-float solves convert the double fields they read and write: scaling the source by 2^k (with
    exact zeros mixed in) scales the solution by 2^k at the same relative accuracy."""
    case = S.single_level_random(n=32, B=16, seed=21, ncomp=2)
    f = case["f"].copy()
    f[:, :, ::7] = 0.0  # exact zeros among the source cells
    box = S.blocks_to_box(f, case["blocks"], 16, case["shape"])
    ref = oracle.solve_box_fft(box, case["h"])
    mac = L.LGF_MAC_BOX if mode == "box" else L.LGF_MAC_PAIR
    for k in (-80, -30, 0, 30, 80):
        s = 2.0 ** k
        phi = solve(L, tables[16], [case["blocks"]], 16, case["h"], f * s, 2, mac)
        got = S.blocks_to_box(phi, case["blocks"], 16, case["shape"])
        for c in range(2):
            assert rel(got[c], ref[c] * s) <= TOL[2], (k, c, rel(got[c], ref[c] * s))


@pytest.mark.parametrize("precision", [0, 2, 1])
@pytest.mark.parametrize("shape", [(8, 32, 56), (64, 96, 8)])
def test_box_block_counts_every_pass_kernel(L, tables, precision, shape):
    """Boxes of 7 x 4 x 1 and 1 x 12 x 8 blocks (B = 8; shape is [nz][ny][nx] cells): the DFT passes
    with compile-time block counts (nb <= 6) and the runtime-count passes with one to three chunks of
    pair slots / outputs (nb = 7, 8, 12), and the trivial nb = 1 axis, against the oracle; three
    components (a complex and a Hermitian-half real field)."""
    B = 8
    box = S.random_box(shape, 31 + shape[0], 3)
    blocks = S.box_blocks(shape, B)
    ref = oracle.solve_box_fft(box, 0.5)
    phi = solve(L, tables[8], [blocks], B, 0.5, S.box_to_blocks(box, blocks, B), precision, L.LGF_MAC_BOX)
    got = S.blocks_to_box(phi, blocks, B, shape)
    for c in range(3):
        assert rel(got[c], ref[c]) <= TOL[precision], (c, rel(got[c], ref[c]))
