"""Block-index DFT passes of wide boxes (9-16 blocks per axis, 16^3 blocks) as in-register mixed-radix FFTs
(box_fft.cuh): parity with the oracle's FFT convolution (Sec. 2.2, Eq. (eq:lgf_convolution)) in FP64 and
DF32, and agreement with the tensor-core DFT-GEMM passes (6 digit slices), an independent evaluation of
the same block-index DFTs, on boxes that use every block count 9..16 and the real-field (Hermitian half)
x pass."""
import numpy as np
import pytest

import lgf_synth as S
import oracle

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
def table(L):
    t = L.lgf_table_create(16, (16, 16, 16), L.LGF_TBL_BOX_ONLY)
    yield t
    L.lgf_table_destroy(t)


def _solve(L, table, mesh, f, precision, slices=0):
    phi = torch.full_like(f, float("nan"))
    L.lgf_poisson_solve(table, mesh, f.shape[0], f.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=precision, mac_mode=L.LGF_MAC_BOX, dft_slices=slices))
    torch.cuda.synchronize()
    return phi


def test_fft_passes_match_oracle(L, table):
    nb = (9, 10, 11)
    shape = tuple(16 * n for n in nb[::-1])
    blocks = S.box_blocks(shape, 16)
    box = S.random_box(shape, 71, 1)
    ref = oracle.solve_box_fft(box, 0.5)
    mesh = L.Mesh([blocks], 16, 0.5)
    f = torch.from_numpy(S.box_to_blocks(box, blocks, 16)).cuda()
    for precision, tol in ((0, 1e-12), (2, 1e-10)):
        got = S.blocks_to_box(_solve(L, table, mesh, f, precision).cpu().numpy(), blocks, 16, shape)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= tol, (precision, err)


@pytest.mark.parametrize("nb", [(12, 13, 14), (15, 16, 12)])
def test_fft_passes_match_tensor_core_passes(L, table, nb):
    shape = tuple(16 * n for n in nb[::-1])
    blocks = S.box_blocks(shape, 16)
    rng = np.random.default_rng(sum(nb))
    f = torch.from_numpy(rng.standard_normal((3, len(blocks), 16, 16, 16))).cuda()  # complex + half-range real
    mesh = L.Mesh([blocks], 16, 0.5)
    a = _solve(L, table, mesh, f, 2)
    b = _solve(L, table, mesh, f, 2, slices=6)
    scale = b.abs().max().item()
    assert torch.isfinite(a).all()
    assert (a - b).abs().max().item() <= 1e-12 * scale
