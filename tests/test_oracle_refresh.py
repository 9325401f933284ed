"""Pins of the oracle's velocity refresh u = -C^T L_E^{-1} omega (Sec. 4.1, Eq. (eq:vel_update)).

On the staggered lattice (Sec. 2.1; component a of cell n stored at index n, faces and edges on the
cell's positive side) the face-to-edge curl C takes forward differences, the face divergence D backward
ones; both are written here, independently of the oracle's C^T.  Two identities of the mimetic
operators fix the result exactly (up to rounding and the LGF table's accuracy):
  * D u = 0 for every omega (D C^T = 0: the divergence of a curl);
  * C u = omega when omega = C v (C C^T = (|s|^2 - conj(s) s^T) in Fourier symbols, and the vertex
    divergence s^T C v of a curl vanishes), so a sign, an index or a transposition slip in C^T or in
    the solve breaks one of the two."""
import numpy as np

from oracle import refresh


def curl_faces_to_edges(v, h):
    """omega_x[n] = (v_z[n + e_y] - v_z[n] - v_y[n + e_z] + v_y[n]) / h and cyclically, on the cells whose
    +e neighbours are in the box ([3][z][y][x]; the result covers [:-1, :-1, :-1])."""
    def fwd(a, axis):
        hi = [slice(0, -1)] * 3
        hi[2 - axis] = slice(1, None)
        return a[tuple(hi)] - a[:-1, :-1, :-1]
    vx, vy, vz = v
    return np.stack([fwd(vz, 1) - fwd(vy, 2), fwd(vx, 2) - fwd(vz, 0), fwd(vy, 0) - fwd(vx, 1)]) / h


def div_faces(u, h):
    """(D u)[n] = sum_a (u_a[n] - u_a[n - e_a]) / h on the cells whose -e neighbours are in the box
    (covers [1:, 1:, 1:])."""
    out = 0.0
    for a in range(3):
        lo = [slice(1, None)] * 3
        lo[2 - a] = slice(0, -1)
        out = out + u[a][1:, 1:, 1:] - u[a][tuple(lo)]
    return out / h


def test_refresh_recovers_the_curl_and_is_divergence_free():
    rng = np.random.default_rng(7)
    n, h = 14, 0.5
    v = np.zeros((3, n + 1, n + 1, n + 1))
    v[:, 4:10, 5:11, 3:9] = rng.standard_normal((3, 6, 6, 6))
    omega = curl_faces_to_edges(v, h)  # [3][n][n][n], compact inside the box
    assert np.abs(omega[:, :2]).max() == 0.0 and np.abs(omega[:, -2:]).max() == 0.0
    u = refresh.velocity_refresh(omega, h)
    cu = curl_faces_to_edges(u, h)
    assert np.abs(cu - omega[:, :-1, :-1, :-1]).max() <= 1e-11 * np.abs(omega).max()
    assert np.abs(div_faces(u, h)).max() <= 1e-11 * np.abs(u).max() / h


def test_refresh_of_random_vorticity_is_divergence_free_and_linear():
    rng = np.random.default_rng(8)
    omega = rng.standard_normal((3, 10, 12, 9))
    u = refresh.velocity_refresh(omega, 1.0)
    assert np.abs(div_faces(u, 1.0)).max() <= 1e-11 * np.abs(u).max()
    u2 = refresh.velocity_refresh(2.0 * omega, 0.5)  # psi scales with h^2 omega, C^T with 1/h
    assert np.allclose(u2, u, rtol=0, atol=1e-12 * np.abs(u).max())
