"""The FP64 residual the library reports (opts.residual) as a value, not only as a bound.

The residual is the acceptance check of the mixed-precision paths: r = L_k phi - F_k - P L_{k-1} psi_{k-1}
on interior Omega_k cells (Sec. 3.4, Eq. (eq:combine_S); L phi - f on a single level, Sec. 2.2), reported
as max |r| / max |source|.  The tests recompute it on the CPU from the phi the GPU returned:
* single level, FP32 and DF32 solves of sources that are exact in FP32: the library's residual must equal
  the recomputed one (the inputs to both are the same numbers);
* two levels, FP32 solve: the recomputation takes F_k and psi_{k-1} from the oracle, which differ from the
  library's FP32 internals by their own rounding, so the two may differ by a bounded factor;
* opts.residual_tol below the achieved residual makes the call return LGF_E_PRECISION.
"""
import numpy as np
import pytest

import lgf_synth as S
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
def table8(L):
    t = L.lgf_table_create(8, (14, 14, 8), L.LGF_TBL_FP64 | L.LGF_TBL_FP32 | L.LGF_TBL_DF32)
    yield t
    L.lgf_table_destroy(t)


def _lap_interior(box, h):
    """7-point Laplacian on the interior of a [ncomp][nz][ny][nx] box (boundary cells dropped)."""
    c = box[:, 1:-1, 1:-1, 1:-1]
    s = (box[:, 2:, 1:-1, 1:-1] + box[:, :-2, 1:-1, 1:-1] + box[:, 1:-1, 2:, 1:-1] + box[:, 1:-1, :-2, 1:-1] +
         box[:, 1:-1, 1:-1, 2:] + box[:, 1:-1, 1:-1, :-2])
    return (s - 6.0 * c) / (h * h)


@pytest.mark.parametrize("precision,mode,rtol", [(1, 1, 1e-6), (1, 2, 1e-6), (2, 2, 5e-2)])
def test_single_level_residual_value(L, table8, precision, mode, rtol):
    shape, B, h = (24, 32, 40), 8, 0.3
    blocks = S.box_blocks(shape, B)
    rng = np.random.default_rng(21)
    box = rng.standard_normal((2,) + shape).astype(np.float32).astype(np.float64)  # exact in FP32
    f = S.box_to_blocks(box, blocks, B)
    mesh = L.Mesh([blocks], B, h)
    ft = torch.from_numpy(f).cuda()
    phi = torch.zeros_like(ft)
    rep = L.lgf_report()
    L.lgf_poisson_solve(table8, mesh, 2, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=precision, mac_mode=mode, residual=1), rep)
    torch.cuda.synchronize()
    got = S.blocks_to_box(phi.cpu().numpy(), blocks, B, shape)
    r = np.abs(_lap_interior(got, h) - box[:, 1:-1, 1:-1, 1:-1]).max()
    want = r / np.abs(box[:, 1:-1, 1:-1, 1:-1]).max()
    assert want > 0 and rep.residual_rel > 0
    assert abs(rep.residual_rel - want) <= rtol * want, (rep.residual_rel, want)


def test_single_level_residual_ignores_non_source_blocks(L, table8):
    # with block roles, f counts only on source blocks: L phi = 0 on target-only blocks
    shape, B, h = (16, 16, 32), 8, 1.0
    blocks = S.box_blocks(shape, B)
    roles = np.full(len(blocks), 2, np.uint8)
    roles[:4] = 3
    rng = np.random.default_rng(22)
    box = rng.standard_normal((1,) + shape).astype(np.float32).astype(np.float64)
    f = S.box_to_blocks(box, blocks, B)
    mesh = L.Mesh([blocks], B, h, roles=roles)
    ft = torch.from_numpy(f).cuda()
    phi = torch.zeros_like(ft)
    rep = L.lgf_report()
    L.lgf_poisson_solve(table8, mesh, 1, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=1, mac_mode=1, residual=1), rep)
    torch.cuda.synchronize()
    src = f.copy()
    src[:, 4:] = 0.0
    srcbox = S.blocks_to_box(src, blocks, B, shape)
    got = S.blocks_to_box(phi.cpu().numpy(), blocks, B, shape)
    inner = srcbox[:, 1:-1, 1:-1, 1:-1]
    want = np.abs(_lap_interior(got, h) - inner).max() / np.abs(inner).max()
    assert abs(rep.residual_rel - want) <= 1e-6 * want


def test_two_level_residual_value(L, table8):
    B = 8
    mesh = dict(B=B, h0=0.5, n_ext=4, levels=[S.box_blocks((24, 24, 24), B),
                                              np.array([[2, 2, 2], [3, 2, 2], [2, 3, 2], [3, 3, 2], [2, 2, 3]],
                                                       np.int32)])
    rng = np.random.default_rng(23)
    f = [rng.standard_normal((2, len(b), B, B, B)).astype(np.float32).astype(np.float64) for b in mesh["levels"]]
    _, _, I = amr.flgf_amr(mesh, f, return_internals=True)
    m = L.Mesh(mesh["levels"], B, mesh["h0"], n_ext=mesh["n_ext"])
    ft = torch.from_numpy(np.concatenate(f, axis=1)).cuda()
    phi = torch.zeros_like(ft)
    rep = L.lgf_report()
    L.lgf_poisson_solve(table8, m, 2, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=1, mac_mode=1, residual=1), rep)
    torch.cuda.synchronize()
    got = phi.cpu().numpy()
    lv, F, psi = I["levels"], I["F"], I["psi"]
    ratios, o = [], 0
    for k, blk in enumerate(mesh["levels"]):
        box = np.zeros((2,) + lv[k].shape)
        for i, b in enumerate(blk):
            box[(slice(None),) + lv[k].block_slice(b, B)] = got[:, o + i]
        o += len(blk)
        src = F[k].copy()
        if k > 0:
            src = src + amr.interp_up(amr.laplacian_box(psi[k - 1], lv[k - 1].h), lv[k - 1], lv[k])
        om = lv[k].omega
        inner = om.copy()
        inner[1:-1, 1:-1, 1:-1] &= (om[2:, 1:-1, 1:-1] & om[:-2, 1:-1, 1:-1] & om[1:-1, 2:, 1:-1] &
                                    om[1:-1, :-2, 1:-1] & om[1:-1, 1:-1, 2:] & om[1:-1, 1:-1, :-2])
        inner[[0, -1], :, :] = inner[:, [0, -1], :] = inner[:, :, [0, -1]] = False
        lap = np.zeros_like(box)
        lap[:, 1:-1, 1:-1, 1:-1] = _lap_interior(box, lv[k].h)
        r = np.abs(lap - src)[:, inner].max()
        ratios.append(r / np.abs(src[:, inner]).max())
    want = max(ratios)
    assert want > 1e-9  # an FP32 solve leaves a residual far above FP64 rounding
    assert 0.5 * want <= rep.residual_rel <= 2.0 * want, (rep.residual_rel, ratios)


@pytest.mark.parametrize("levels", [1, 2])
def test_residual_tolerance_raises_precision_error(L, table8, levels):
    B = 8
    blk0 = S.box_blocks((24, 24, 24), B)
    lv = [blk0] if levels == 1 else [blk0, np.array([[2, 2, 2], [3, 2, 2]], np.int32)]
    m = L.Mesh(lv, B, 0.5, n_ext=4)
    rng = np.random.default_rng(24)
    ft = torch.from_numpy(rng.standard_normal((1, sum(len(b) for b in lv), B, B, B))).cuda()
    phi = torch.zeros_like(ft)
    rep = L.lgf_report()
    L.lgf_poisson_solve(table8, m, 1, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=1, mac_mode=1, residual=1, residual_tol=1.0), rep)
    achieved = rep.residual_rel
    assert 1e-9 < achieved < 1e-3
    with pytest.raises(L.LgfError) as e:
        L.lgf_poisson_solve(table8, m, 1, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                            L.make_opts(precision=1, mac_mode=1, residual=1, residual_tol=0.5 * achieved), rep)
    assert e.value.status == L.LGF_E_PRECISION
    # FP64 meets a tolerance the FP32 solve misses
    L.lgf_poisson_solve(table8, m, 1, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=0, mac_mode=1, residual=1, residual_tol=0.5 * achieved), rep)
    assert rep.residual_rel < 1e-11
