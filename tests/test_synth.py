"""The seeded synthetic inputs (lgf_synth) on the CPU: the batch's instance draws are reproducible and
span the stated ranges, and every generated composite mesh is properly nested (each level-(k+1) block
lies inside a level-k block, Sec. 3.1), with source arrays of the mesh's shape."""
import numpy as np

import lgf_synth as S


def _check_nested(mesh):
    B = mesh["B"]
    levels = mesh["levels"]
    for k, blk in enumerate(levels):
        assert len({tuple(b) for b in blk}) == len(blk), f"duplicate blocks on level {k}"
    for k in range(1, len(levels)):
        coarse = {tuple(b) for b in levels[k - 1]}
        for b in levels[k]:
            parent = tuple(int(v) for v in (np.asarray(b) * (B // 2)) // B)
            assert parent in coarse, (k, tuple(b))


def test_batch_draws_are_reproducible_and_in_range():
    a, b = S.batch_instances(64), S.batch_instances(64)
    assert a == b
    assert {p["levels"] for p in a} == {1, 2, 3}
    for p in a:
        assert 0.5 <= p["R"] <= 1.5 and 0.1 <= p["sigma"] / p["R"] <= 0.25
        assert 32 <= p["nxy"] <= 192 and p["nxy"] % 16 == 0
        assert p["nz"] == max(32, 16 * int(np.ceil(p["nxy"] / 32)))
        assert abs(p["h_fine"] * p["nxy"] - (2 * p["R"] + 8 * p["sigma"])) < 1e-12


def test_small_batch_instances_are_nested_with_matching_sources():
    params = S.batch_instances(64)
    smallest = {}
    for p in params:  # the smallest instance of each level count
        k = p["levels"]
        if k not in smallest or p["nxy"] < smallest[k]["nxy"]:
            smallest[k] = p
    for k, p in sorted(smallest.items()):
        mesh, f, roles = S.ring_instance(p, B=16, n_ext=16)
        assert len(mesh["levels"]) == k
        _check_nested(mesh)
        for lev, blk in zip(f, mesh["levels"]):
            assert lev.shape == (3, len(blk), 16, 16, 16) and np.isfinite(lev).all()
        assert (roles is None) == (k > 1)


def test_three_level_ring_mesh():
    mesh, f = S.three_level_ring()
    _check_nested(mesh)
    n = [len(b) for b in mesh["levels"]]
    assert sum(n) == 652  # the three-level ring's caller blocks
    # Omega_k cells: each level-(k+1) block covers one octant of its parent
    cells = sum((n[k] - (n[k + 1] if k + 1 < 3 else 0) / 8) * 16 ** 3 for k in range(3))
    assert cells == 2387968
    assert all(x.shape[1] == len(b) for x, b in zip(f, mesh["levels"]))


def test_bump_case_refines_children_only():
    for lr in range(4):
        mesh, om, ps = S.bump_case(lr)
        assert len(mesh["levels"]) == lr + 1
        _check_nested(mesh)
        assert all(o.shape[1] == len(b) for o, b in zip(om, mesh["levels"]))
