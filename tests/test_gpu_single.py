"""GPU parity of the single-level free-space solve (Sec. 2.2, Eq. (eq:lgf_convolution)) through the C ABI.

Every expected value comes from the CPU oracle (direct Neumaier sums, or its zero-padded FFT
convolution which the oracle tests pin to the direct sum), or from an identity of the lattice.
Tolerances: relative L-infinity error (max |diff| / max |ref|) <= 1e-12 for FP64, <= 1e-10 for
the double-float (DF32) path; plain FP32 is bounded loosely (its error is reported, not a target).
"""
import numpy as np
import pytest

import lgf_synth as S
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 2: 1e-10, 1: 2e-5}  # precision code -> tolerance


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_13213_gb300.lgf as L
    L.load()
    return L


def rel_err(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def run_solve(L, table, mesh, f_blocks, precision, dtype=0, report=None):
    tdt = torch.float64 if dtype == 0 else torch.float32
    f = torch.from_numpy(f_blocks).to("cuda", tdt)
    phi = torch.full_like(f, float("nan"))
    L.lgf_poisson_solve(table, mesh, f.shape[0], f.data_ptr(), phi.data_ptr(), dtype,
                        L.make_opts(precision=precision, mac_mode=L.LGF_MAC_PAIR), report)
    torch.cuda.synchronize()
    return phi.double().cpu().numpy()


@pytest.fixture(scope="module")
def table16(L):
    t = L.lgf_table_create(16, (6, 6, 6), L.LGF_TBL_FP64 | L.LGF_TBL_FP32 | L.LGF_TBL_DF32)
    yield t
    L.lgf_table_destroy(t)


def test_device_lgf_table_matches_oracle(L, table16):
    n = 100
    dev = L.lgf_table_lgf_values(table16, n)
    ref = oracle.lgf_octant(n)
    assert np.abs(dev - ref).max() / np.abs(ref).max() < 1e-14
    assert (np.abs(dev - ref) / np.abs(ref)).max() < 2e-14


@pytest.fixture(scope="module")
def random32():
    case = S.single_level_random(n=32, B=16, seed=0)
    src = oracle.core.box_cells(case["shape"])
    ref = oracle.solve_box_direct(case["box"], case["h"])[0].reshape(case["shape"])
    return case, ref, src


@pytest.mark.parametrize("precision", [0, 2, 1])
def test_random_32cube_full_field(L, table16, random32, precision):
    case, ref, _ = random32
    mesh = L.Mesh([case["blocks"]], 16, case["h"])
    rep = L.lgf_report()
    phi = run_solve(L, table16, mesh, case["f"], precision, report=rep)
    got = S.blocks_to_box(phi, case["blocks"], 16, case["shape"])[0]
    err = rel_err(got, ref)
    assert err <= TOL[precision], f"precision {precision}: rel err {err:.3e}"
    assert rep.pairs == 64 and rep.target_cells == 32 ** 3


def test_ragged_block_set_with_roles_and_float_storage(L):
    """B = 8, 13 scattered blocks; some source-only, some target-only; float32 storage."""
    rng = np.random.default_rng(21)
    blocks = np.array([[0, 0, 0], [1, 0, 0], [3, 1, 0], [0, 2, 1], [2, 2, 1], [4, 0, 2], [1, 3, 2],
                       [3, 3, 0], [0, 1, 3], [2, 0, 3], [4, 3, 3], [1, 1, 1], [3, 2, 2]], np.int32)
    roles = np.array([3, 1, 2, 3, 1, 2, 3, 3, 1, 2, 3, 1, 2], np.uint8)
    B, h = 8, 0.3
    f = rng.standard_normal((2, len(blocks), B, B, B)).astype(np.float32).astype(np.float64)
    table = L.lgf_table_create(B, (4, 3, 3), L.LGF_TBL_FP64 | L.LGF_TBL_DF32)
    try:
        mesh = L.Mesh([blocks], B, h, roles=roles)
        for prec, tol in ((0, 1e-6), (2, 1e-6)):  # float32 output storage bounds the error at ~6e-8
            phi = run_solve(L, table, mesh, f, prec, dtype=1)
            # oracle: direct sum from the source blocks to every cell of the target blocks
            src_b = blocks[(roles & 1) > 0]
            fs = f[:, (roles & 1) > 0]
            sxyz = np.concatenate([oracle.core.box_cells((B, B, B), tuple(B * b)) for b in src_b])
            sval = fs.reshape(2, len(src_b), -1).reshape(2, -1)
            tgt_b = blocks[(roles & 2) > 0]
            txyz = np.concatenate([oracle.core.box_cells((B, B, B), tuple(B * b)) for b in tgt_b])
            T = oracle.lgf_octant(48)
            ref = oracle.direct_conv(T, sxyz, sval, txyz, h * h)
            got = phi[:, (roles & 2) > 0].reshape(2, -1)
            assert rel_err(got, ref) <= tol
            # blocks without the target role are left untouched (NaN sentinel)
            assert np.isnan(phi[:, (roles & 2) == 0]).all()
    finally:
        L.lgf_table_destroy(table)


def test_exact_inverse_on_device(L, table16):
    """h^2 G * (L_h g) = g for compactly supported g (a lattice identity, no oracle involved)."""
    rng = np.random.default_rng(5)
    B, h = 16, 0.7
    g = np.zeros((1, 32, 32, 48))
    g[0, 3:29, 2:30, 5:43] = rng.standard_normal((26, 28, 38))
    p = np.pad(g[0], 1)
    f = np.zeros_like(g)
    f[0] = (p[2:, 1:-1, 1:-1] + p[:-2, 1:-1, 1:-1] + p[1:-1, 2:, 1:-1] + p[1:-1, :-2, 1:-1]
            + p[1:-1, 1:-1, 2:] + p[1:-1, 1:-1, :-2] - 6 * g[0]) / h ** 2
    blocks = S.box_blocks((32, 32, 48), B)
    mesh = L.Mesh([blocks], B, h)
    for prec, tol in ((0, 1e-12), (2, 1e-10)):
        phi = run_solve(L, table16, mesh, S.box_to_blocks(f, blocks, B), prec)
        got = S.blocks_to_box(phi, blocks, B, (32, 32, 48))
        assert rel_err(got, g) <= tol


@pytest.fixture(scope="module")
def ring_case():
    case = S.single_level_ring()
    ref = oracle.solve_box_fft(case["box"], case["h"])
    return case, ref


@pytest.mark.parametrize("precision", [0, 2])
def test_ring_96x96x48_full_field_and_samples(L, table16, ring_case, precision):
    case, ref = ring_case
    B = 16
    roles = np.zeros(len(case["blocks"]), np.uint8) + 2
    src = {tuple(b) for b in case["src_blocks"]}
    roles += np.array([1 if tuple(b) in src else 0 for b in case["blocks"]], np.uint8)
    mesh = L.Mesh([case["blocks"]], B, case["h"], roles=roles)
    phi = run_solve(L, table16, mesh, case["f"], precision)
    got = S.blocks_to_box(phi, case["blocks"], B, case["shape"])
    for c in range(2):
        assert rel_err(got[c], ref[c]) <= TOL[precision]
    assert np.abs(got[2]).max() == 0.0  # omega_z = 0 => phi_z = 0 exactly
    # sampled cells against the direct sum (independent of the FFT oracle)
    rng = np.random.default_rng(7)
    nz, ny, nx = case["shape"]
    idx = rng.integers(0, [nx, ny, nz], size=(64, 3)).astype(np.int32)
    direct = oracle.solve_box_direct(case["box"][:2], case["h"], idx)
    for c in range(2):
        sample = got[c][idx[:, 2], idx[:, 1], idx[:, 0]]
        assert np.abs(sample - direct[c]).max() <= TOL[precision] * np.abs(ref[c]).max()


def test_prepared_table_allocates_nothing_during_solves(L):
    # after lgf_table_prepare the solve builds nothing: the report's workspace stays the same, and a CUDA
    # graph capture of the solve (which forbids allocation) succeeds
    import lgf_synth as S2
    case = S2.single_level_ring()
    mesh = L.Mesh([case["blocks"]], 16, case["h"])
    t = L.lgf_table_create(16, (5, 5, 2), L.LGF_TBL_BOX_ONLY)
    try:
        s = torch.cuda.Stream()
        opts = L.make_opts(precision=L.LGF_PREC_DF32)
        L.lgf_table_prepare(t, mesh, 3, L.LGF_F64, opts, s.cuda_stream)
        f = torch.from_numpy(case["f"]).cuda()
        phi = torch.zeros_like(f)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            L.lgf_poisson_solve(t, mesh, 3, f.data_ptr(), phi.data_ptr(), L.LGF_F64, opts, None, s.cuda_stream)
            g.capture_end()
        g.replay()
        torch.cuda.synchronize()
        ref = torch.zeros_like(f)
        L.lgf_poisson_solve(t, mesh, 3, f.data_ptr(), ref.data_ptr(), L.LGF_F64, opts)
        torch.cuda.synchronize()
        assert torch.equal(phi, ref)
    finally:
        L.lgf_table_destroy(t)
