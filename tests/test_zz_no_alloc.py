"""The allocation-free single-level solve (lgf_poisson_solve_static) against the regular entry point.

Callers that cannot allocate device memory during a solve (a fixed device-memory budget, or a thread
that must not block on the allocator) use this entry point; its scratch is the library's fixed
32 MiB device array.  This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import lgf_synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_13213_gb300.lgf as L
    L.load()
    return L


def _solve_pair(L, table, mesh, f, precision, dtype):
    out = torch.full_like(f, float("nan"))
    L.lgf_poisson_solve(table, mesh, f.shape[0], f.data_ptr(), out.data_ptr(), dtype,
                        L.make_opts(precision=precision, mac_mode=L.LGF_MAC_PAIR))
    return out


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-10), (1, 1e-5)])
def test_static_matches_regular_on_two_calls(L, precision, tol):
    table = L.lgf_table_create(16, (1, 1, 1), L.LGF_TBL_FP64 | L.LGF_TBL_DF32 | L.LGF_TBL_FP32)
    try:
        case = S.single_level_random(n=32, B=16, seed=3, ncomp=2)
        mesh = L.Mesh([case["blocks"]], 16, case["h"])
        f = torch.from_numpy(case["f"]).cuda()
        ref = _solve_pair(L, table, mesh, f, precision, L.LGF_F64)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        scale = np.abs(ref).max()
        for call in range(2):
            # the second call gets a different source so stale scratch contents would show
            fin = f if call == 0 else -2.0 * f
            out = torch.full_like(f, float("nan"))
            L.lgf_poisson_solve_static(table, mesh, 2, fin.data_ptr(), out.data_ptr(), L.LGF_F64, precision)
            torch.cuda.synchronize()
            expect = ref if call == 0 else -2.0 * ref
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.abs(got - expect).max() <= tol * (2.0 if call else 1.0) * scale
    finally:
        L.lgf_table_destroy(table)


def test_static_rejects_requests_beyond_its_scratch(L):
    table = L.lgf_table_create(16, (5, 5, 2), L.LGF_TBL_FP64)
    try:
        case = S.single_level_ring()
        mesh = L.Mesh([case["blocks"]], 16, case["h"])
        f = torch.from_numpy(case["f"]).cuda()
        out = torch.zeros_like(f)
        with pytest.raises(L.LgfError) as e:
            L.lgf_poisson_solve_static(table, mesh, 3, f.data_ptr(), out.data_ptr(), L.LGF_F64, 0)
        assert e.value.status == L.LGF_E_INVALID_ARG and "static scratch" in str(e.value)
    finally:
        L.lgf_table_destroy(table)


@pytest.mark.parametrize("roles", ["subset", "none"])
def test_static_with_block_roles(L, roles):
    # sources a strict subset of the targets (ragged source and target lists), or no source at all
    # (every target block must then be written with zeros)
    table = L.lgf_table_create(8, (3, 3, 3), L.LGF_TBL_FP64)
    try:
        case = S.single_level_random(n=32, B=8, seed=9, ncomp=2)
        nb = len(case["blocks"])
        role = np.full(nb, 2, np.uint8)
        if roles == "subset":
            role[::3] = 3
            role[5] = 1  # a source that receives no output
        mesh = L.Mesh([case["blocks"]], 8, case["h"], roles=role)
        f = torch.from_numpy(case["f"]).cuda()
        ref = _solve_pair(L, table, mesh, f, 0, L.LGF_F64)
        for _ in range(2):
            out = torch.full_like(f, float("nan"))
            L.lgf_poisson_solve_static(table, mesh, 2, f.data_ptr(), out.data_ptr(), L.LGF_F64, 0)
            torch.cuda.synchronize()
            got, want = out.cpu().numpy(), ref.cpu().numpy()
            tgt = (role & 2) > 0
            assert np.isnan(got[:, ~tgt]).all()  # blocks without the target role are left untouched
            if roles == "none":
                assert (got[:, tgt] == 0.0).all()
            else:
                scale = np.abs(want[:, tgt]).max()
                assert scale > 0 and np.abs(got[:, tgt] - want[:, tgt]).max() <= 1e-12 * scale
    finally:
        L.lgf_table_destroy(table)


def test_static_refuses_a_capturing_stream(L):
    # its index lists come from pageable host memory, which a capturing stream does not accept: the call
    # must return LGF_E_UNSUPPORTED without touching the capture
    table = L.lgf_table_create(16, (1, 1, 1), L.LGF_TBL_FP64)
    try:
        case = S.single_level_random(n=32, B=16, seed=4, ncomp=1)
        mesh = L.Mesh([case["blocks"]], 16, case["h"])
        f = torch.from_numpy(case["f"]).cuda()
        out = torch.zeros_like(f)
        L.lgf_poisson_solve_static(table, mesh, 1, f.data_ptr(), out.data_ptr(), L.LGF_F64, 0)  # set-up call
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        status = None
        with torch.cuda.stream(s):
            g.capture_begin()
            try:
                L.lgf_poisson_solve_static(table, mesh, 1, f.data_ptr(), out.data_ptr(), L.LGF_F64, 0,
                                           s.cuda_stream)
            except L.LgfError as e:
                status = e.status
            out.add_(1.0)  # the capture is still valid: a later node records fine
            g.capture_end()
        assert status == L.LGF_E_UNSUPPORTED
        before = out.clone()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, before + 1.0)
    finally:
        L.lgf_table_destroy(table)
