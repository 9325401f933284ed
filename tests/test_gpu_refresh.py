"""GPU parity of the velocity refresh u = -C^T L_E^{-1} omega (Sec. 4.1, Eq. (eq:vel_update)) through the
C ABI, against the CPU oracle (``oracle.refresh``) and against the lattice identities the oracle is
pinned to (C u = omega for omega = C v, D u = 0)."""
import numpy as np
import pytest

import lgf_synth as S
from oracle import refresh
from test_oracle_refresh import curl_faces_to_edges, div_faces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# u differences psi: its relative error is about 2 x (box width in cells) times the solve's
TOL = {0: 1e-12, 2: 1e-10, 1: 2e-4}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_13213_gb300.lgf as L
    L.load()
    return L


@pytest.fixture(scope="module")
def tables(L):
    flags = L.LGF_TBL_FP64 | L.LGF_TBL_FP32 | L.LGF_TBL_DF32
    t16 = L.lgf_table_create(16, (3, 3, 3), flags)
    t8 = L.lgf_table_create(8, (6, 6, 6), flags)
    yield {16: t16, 8: t8}
    L.lgf_table_destroy(t16)
    L.lgf_table_destroy(t8)


def gpu_refresh(L, table, blocks, B, h, om_blocks, precision, mode=None, rep=None):
    m = L.Mesh([blocks], B, h)
    om = torch.from_numpy(np.ascontiguousarray(om_blocks)).cuda()
    u = torch.full_like(om, float("nan"))
    L.lgf_velocity_refresh(table, m, om.data_ptr(), u.data_ptr(), L.LGF_F64,
                           L.make_opts(precision=precision, mac_mode=L.LGF_MAC_AUTO if mode is None else mode), rep)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def rel(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("precision", [0, 2, 1])
def test_refresh_random_32cube(L, tables, precision):
    shape = (32, 32, 32)
    om = S.random_box(shape, 17, 3)
    blocks = S.box_blocks(shape, 16)
    ref = refresh.velocity_refresh(om, 0.25)
    rep = L.lgf_report()
    u = gpu_refresh(L, tables[16], blocks, 16, 0.25, S.box_to_blocks(om, blocks, 16), precision, rep=rep)
    got = S.blocks_to_box(u, blocks, 16, shape)
    assert max(rel(got[c], ref[c]) for c in range(3)) <= TOL[precision]
    assert rep.kernel_launches > 0


@pytest.mark.parametrize("mode", ["pair", "box"])
def test_refresh_ragged_blocks_B8(L, tables, mode):
    """An L-shaped set of 8^3 blocks inside a 24 x 32 x 16 bounding box: sources and outputs on the blocks
    only; the oracle's box carries zero vorticity elsewhere."""
    B, h = 8, 0.5
    blocks = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0], [0, 2, 0], [0, 3, 0], [0, 0, 1], [1, 1, 1]],
                      np.int32)
    shape = (16, 32, 24)
    rng = np.random.default_rng(23)
    omb = rng.standard_normal((3, len(blocks), B, B, B))
    box = S.blocks_to_box(omb, blocks, B, shape)
    ref = refresh.velocity_refresh(box, h)
    mac = L.LGF_MAC_PAIR if mode == "pair" else L.LGF_MAC_BOX
    u = gpu_refresh(L, tables[8], blocks, B, h, omb, 0, mode=mac)
    refb = S.box_to_blocks(ref, blocks, B)
    assert rel(u, refb) <= 1e-12


def test_refresh_recovers_a_curl_on_the_gpu(L, tables):
    """omega = C v for a compact face field v: the GPU's u satisfies C u = omega and D u = 0."""
    rng = np.random.default_rng(29)
    n, h = 32, 0.5
    v = np.zeros((3, n + 1, n + 1, n + 1))
    v[:, 10:22, 9:21, 11:23] = rng.standard_normal((3, 12, 12, 12))
    omega = curl_faces_to_edges(v, h)  # [3][32][32][32]
    blocks = S.box_blocks((n, n, n), 16)
    u = S.blocks_to_box(gpu_refresh(L, tables[16], blocks, 16, h, S.box_to_blocks(omega, blocks, 16), 0),
                        blocks, 16, (n, n, n))
    assert np.abs(curl_faces_to_edges(u, h) - omega[:, :-1, :-1, :-1]).max() <= 1e-11 * np.abs(omega).max()
    assert np.abs(div_faces(u, h)).max() <= 1e-11 * np.abs(u).max() / h


def test_refresh_rejects_bad_requests(L, tables):
    blocks = S.box_blocks((16, 16, 16), 16)
    om = torch.zeros((3, 1, 16, 16, 16), dtype=torch.float64, device="cuda")
    two = L.Mesh([blocks, np.array([[0, 0, 0]], np.int32)], 16, 1.0)
    with pytest.raises(L.LgfError) as e:
        L.lgf_velocity_refresh(tables[16], two, om.data_ptr(), om.data_ptr() + 8, L.LGF_F64)
    assert e.value.status == L.LGF_E_MESH
    m = L.Mesh([blocks], 16, 1.0)
    with pytest.raises(L.LgfError) as e:
        L.lgf_velocity_refresh(tables[16], m, om.data_ptr(), om.data_ptr(), L.LGF_F64)
    assert e.value.status == L.LGF_E_INVALID_ARG
