"""Test glue: map between the oracle's interior-edge ordering and the library's device layout.

The oracle numbers all x-, y-, z-edges of the Yee grid in its own order and keeps the
interior ones; the library stores 3 blocks of nx*ny*nz entries, entry (c, i, j, k) at
c*nx*ny*nz + i + nx*(j + ny*k) for the edge of direction c leaving node (i, j, k).
"""
import numpy as np


def lib_index_of_interior(grid):
    """Library index of every interior oracle edge, in the oracle's interior order."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    nc = nx * ny * nz
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx), indexing="ij")
    ix = (0 * nc + i + nx * (j + ny * k)).ravel()
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx + 1), indexing="ij")
    iy = (1 * nc + i + nx * (j + ny * k)).ravel()
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    iz = (2 * nc + i + nx * (j + ny * k)).ravel()
    allidx = np.concatenate((ix, iy, iz))
    return allidx[grid.interior_mask()]


def to_lib(grid, v_interior):
    nc = grid.nx * grid.ny * grid.nz
    out = np.zeros(3 * nc, dtype=np.complex128)
    out[lib_index_of_interior(grid)] = v_interior
    return out


def from_lib(grid, v_lib):
    return np.asarray(v_lib)[lib_index_of_interior(grid)]
