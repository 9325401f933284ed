"""GPU parity of the HERK stage projection (lgf_stage_projection: L_C p = D r, u = H(r - G p); Sec. 2.4,
Sec. 3.6) against the oracle (oracle/projection.py), on one, two and three levels, through the C ABI.

Tolerances (relative L-infinity over Omega_k, per field): 1e-12 FP64, 1e-10 DF32.  On one level the
projected field is also checked to be divergence-free inside the blocks."""
import numpy as np
import pytest

import lgf_synth as S
from oracle import amr, core, projection

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 2: 1e-10}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_13213_gb300.lgf as L
    L.load()
    return L


@pytest.fixture(scope="module")
def table8(L):
    t = L.lgf_table_create(8, (14, 14, 14), L.LGF_TBL_FP64 | L.LGF_TBL_DF32)
    yield t
    L.lgf_table_destroy(t)


def _smooth_r(mesh, seed):
    rng = np.random.default_rng(seed)
    B = mesh["B"]
    coef = rng.standard_normal((3, 4))
    out = []
    for k, blk in enumerate(mesh["levels"]):
        h = mesh["h0"] / 2 ** k
        data = np.zeros((3, len(blk), B, B, B))
        for i, (bx, by, bz) in enumerate(blk):
            z, y, x = np.meshgrid(*[(B * b + np.arange(B) + 0.5) * h - 10.0 for b in (bz, by, bx)], indexing="ij")
            env = np.exp(-(x ** 2 + y ** 2 + z ** 2) / 16.0)
            for c in range(3):
                data[c, i] = env * (coef[c, 0] * x + coef[c, 1] * y + coef[c, 2] * z + coef[c, 3])
        out.append(data)
    return out


def _gpu(L, table, mesh, r, precision, alpha, mode=0):
    m = L.Mesh(mesh["levels"], mesh["B"], mesh["h0"], n_ext=mesh["n_ext"])
    rt = torch.from_numpy(np.concatenate(r, axis=1)).cuda()
    u = torch.full_like(rt, float("nan"))
    p = torch.full((1,) + tuple(rt.shape[1:]), float("nan"), dtype=torch.float64, device="cuda")
    rep = L.lgf_report()
    L.lgf_stage_projection(table, m, rt.data_ptr(), u.data_ptr(), p.data_ptr(), L.LGF_F64, alpha,
                           L.make_opts(precision=precision, mac_mode=mode), rep)
    torch.cuda.synchronize()

    def split(a):
        out, o = [], 0
        for b in mesh["levels"]:
            out.append(a[:, o:o + len(b)])
            o += len(b)
        return out

    return split(u.cpu().numpy()), split(p.cpu().numpy()), rep


def _compare(got, ref, masks, tol):
    for k, (g, r, m) in enumerate(zip(got, ref, masks)):
        if not m.any():
            continue
        scale = np.abs(r[:, m]).max()
        err = np.abs(g[:, m] - r[:, m]).max() / scale
        assert err <= tol, (k, err)


def _masks(mesh):
    lv = amr.build_levels(mesh)
    return [projection._to_blocks(lv[k], mesh["levels"][k], lv[k].omega[None].astype(float), mesh["B"])[0] > 0.5
            for k in range(len(lv))]


@pytest.mark.parametrize("precision", [0, 2])
def test_projection_one_level(L, table8, precision):
    mesh = dict(B=8, h0=0.5, n_ext=4, levels=[S.box_blocks((32, 32, 40), 8)])
    r = _smooth_r(mesh, 51)
    for alpha in (0.1, 0.0):
        ref_u, ref_p = projection.project_amr(mesh, r, alpha)
        u, p, rep = _gpu(L, table8, mesh, r, precision, alpha)
        masks = _masks(mesh)
        _compare(u, ref_u, masks, TOL[precision])
        _compare(p, ref_p, masks, TOL[precision])
    # divergence-free inside the blocks (alpha = 0 leaves a two-cell margin)
    ub = S.blocks_to_box(u[0], mesh["levels"][0], 8, (32, 32, 40))
    rb = S.blocks_to_box(r[0], mesh["levels"][0], 8, (32, 32, 40))

    def div(a):
        return ((a[0][1:, 1:, 1:] - a[0][1:, 1:, :-1]) + (a[1][1:, 1:, 1:] - a[1][1:, :-1, 1:]) +
                (a[2][1:, 1:, 1:] - a[2][:-1, 1:, 1:]))

    assert np.abs(div(ub))[2:-2, 2:-2, 2:-2].max() < 1e2 * TOL[precision] * np.abs(div(rb)).max()


@pytest.mark.parametrize("precision", [0, 2])
def test_projection_two_levels(L, table8, precision):
    B = 8
    mesh = dict(B=B, h0=0.5, n_ext=4, levels=[S.box_blocks((40, 40, 40), B),
                                              np.array([[x, y, z] for x in (3, 4, 5, 6) for y in (3, 4, 5, 6)
                                                        for z in (4, 5)], np.int32)])
    r = _smooth_r(mesh, 52)
    ref_u, ref_p = projection.project_amr(mesh, r, 0.08)
    u, p, _ = _gpu(L, table8, mesh, r, precision, 0.08)
    masks = _masks(mesh)
    _compare(u, ref_u, masks, TOL[precision])
    _compare(p, ref_p, masks, TOL[precision])


def test_projection_three_level_ring_box_mode(L):
    mesh, f = S.three_level_ring(R=1.0, sigma=0.2, B=8, n_ext=6, h_fine=1 / 32, support=(24, 24, 16), dilate0=1)
    ref_u, ref_p = projection.project_amr(mesh, f, 0.1)
    t = L.lgf_table_create(8, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    try:
        u, p, _ = _gpu(L, t, mesh, f, 2, 0.1, mode=2)
    finally:
        L.lgf_table_destroy(t)
    masks = _masks(mesh)
    _compare(u, ref_u, masks, 1e-10)
    _compare(p, ref_p, masks, 1e-10)
