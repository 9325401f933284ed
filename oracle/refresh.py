"""Velocity refresh u = -C^T L_E^{-1} omega on one uniform level (Sec. 4.1, Eq. (eq:vel_update)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Staggered lattice (Sec. 2.1): u lives on the positive faces of a cell, omega and the streamfunction psi
on its positive edges; component a of cell n is stored at array index n.  The edge Laplacian's LGF is
the cell one (the lattice is shift-invariant), so psi = L_E^{-1} omega is ``core.solve_box_fft`` of each
component.  C^T, the discrete curl from edges to faces, is the transpose of the face-to-edge curl C
(Eq. (eq:mimetic): C-bar = C^T); with C's forward differences, C^T takes backward differences:
    (C^T psi)_x[n] = (psi_z[n] - psi_z[n - e_y] - psi_y[n] + psi_y[n - e_z]) / h   (and cyclically).

Pins (tests/test_oracle_refresh.py): for omega = C v of a compactly supported face field v (written in
the test, forward differences), the refreshed u satisfies C u = omega and D u = 0 on the lattice (the
discrete identities C C^T - (L_E - G D) = 0 and D C^T = 0); the solve itself is pinned in
``core``.
"""
import numpy as np

from .core import solve_box_fft


def _back(a: np.ndarray, axis: int) -> np.ndarray:
    """Backward difference a[n] - a[n - e_axis] on the cells that have the neighbour (the box shrinks by
    one cell at the low end of every axis); arrays are [z][y][x], axis 0 = x."""
    sl_hi = [slice(1, None)] * 3
    sl_lo = [slice(1, None)] * 3
    sl_lo[2 - axis] = slice(0, -1)
    return a[tuple(sl_hi)] - a[tuple(sl_lo)]


def velocity_refresh(omega: np.ndarray, h: float) -> np.ndarray:
    """u = -C^T L_E^{-1} omega on the box of ``omega`` ([3][nz][ny][nx], the sources): psi is solved on the
    box widened by one cell toward -x, -y, -z (no sources there), then the backward differences of C^T
    land on the original box."""
    om = np.pad(omega, ((0, 0), (1, 0), (1, 0), (1, 0)))
    psi = solve_box_fft(om, h)
    px, py, pz = psi[0], psi[1], psi[2]
    ux = _back(pz, 1) - _back(py, 2)
    uy = _back(px, 2) - _back(pz, 0)
    uz = _back(py, 0) - _back(px, 1)
    return -np.stack([ux, uy, uz]) / h
