"""GPU parity of the matrix-free shifted operator q = (K - xi M) p against the oracle's assembled K, M.

Grids span several CTA tiles (32 x 8 nodes, 32-plane z chunks) with ragged tails in every
direction; p is random on the interior edges.  FP64: the stencil sums the same 13 terms in
another order, so the bound is a few ulps of the largest term per row (1e-13 of |K| |p|).
FP32: the same operator in single precision (1e-5 of |K| |p|).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.yee import YeeGrid
from tests._layout import to_lib, from_lib

pytestmark = pytest.mark.gpu


def _grid(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    hx, hy, hz = rng.uniform(5, 20, nx), rng.uniform(5, 20, ny), rng.uniform(5, 20, nz)
    sigma = 10 ** rng.uniform(-8, 0, nx * ny * nz)
    return hx, hy, hz, sigma


@pytest.mark.parametrize("dims", [(8, 8, 8), (40, 20, 36), (33, 9, 65), (5, 3, 4)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_operator_matches_assembled(dims, prec):
    from paper_2506_11657_gb300 import tem
    nx, ny, nz = dims
    hx, hy, hz, sigma = _grid(nx, ny, nz, sum(dims))
    G = YeeGrid(hx, hy, hz)
    mask = G.interior_mask()
    K = G.stiffness()[mask][:, mask]
    M = G.mass(sigma)[mask]
    shifts = np.array([-800 + 250j, 3e4 + 1e5j, -5.0 + 0j])
    rng = np.random.default_rng(7)
    n = mask.sum()
    P = rng.standard_normal((len(shifts), n)) + 1j * rng.standard_normal((len(shifts), n))
    grid = tem.Grid(hx, hy, hz, (0, 0, 0), sigma)
    nc3 = 3 * nx * ny * nz
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    p = torch.tensor(np.stack([to_lib(G, P[i]) for i in range(len(shifts))]), dtype=dt, device="cuda")
    q = torch.full((len(shifts), nc3), float("nan"), dtype=dt, device="cuda")
    tem.apply_operator(grid, shifts, p, q, tem.PREC_FP64 if prec == "fp64" else tem.PREC_MIXED)
    torch.cuda.synchronize()
    qh = q.cpu().numpy().astype(np.complex128)
    tol = 1e-13 if prec == "fp64" else 2e-6
    for i, s in enumerate(shifts):
        ref = K @ P[i] - s * M * P[i]
        scale = abs(K) @ np.abs(P[i]) + abs(s) * M * np.abs(P[i])
        got = from_lib(G, qh[i])
        assert np.all(np.abs(got - ref) <= tol * scale + 1e-300), (i, np.max(np.abs(got - ref) / scale))
        # boundary and padding entries are written as exact zeros
        full = np.zeros(nc3, dtype=bool)
        full[__import__("tests._layout", fromlist=["x"]).lib_index_of_interior(G)] = True
        assert np.all(qh[i][~full] == 0)
