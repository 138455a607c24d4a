"""Pins of the oracle's Yee assembly against facts fixed by the mathematics (Sec. 2.2).

None of these retypes the assembly formulas: each checks an identity or a
closed form that a sign, index, length or transposition error would break.
"""
import numpy as np
import pytest

from oracle.yee import YeeGrid, MU0


def _nonuniform_grid(seed=0, n=(5, 4, 6)):
    rng = np.random.default_rng(seed)
    return YeeGrid(rng.uniform(0.5, 2.0, n[0]), rng.uniform(0.5, 2.0, n[1]), rng.uniform(0.5, 2.0, n[2]),
                   origin=(-1.0, 2.0, -3.0))


def test_curl_of_gradient_is_zero():
    """C G = 0 exactly: every face circulation of a nodal gradient vanishes."""
    g = _nonuniform_grid()
    C, _, _ = g.curl()
    phi = np.random.default_rng(1).standard_normal(g.n_nodes)
    e = g.gradient() @ phi
    assert np.abs(C @ e).max() <= 1e-12 * np.abs(e).max() * g.hx.max()


def test_stiffness_symmetric_and_semidefinite():
    g = _nonuniform_grid(2)
    K = g.stiffness()
    assert abs(K - K.T).max() <= 1e-12 * abs(K).max()
    X = np.random.default_rng(3).standard_normal((g.n_edges, 20))
    assert np.all(np.einsum("ij,ij->j", X, K @ X) >= 0)


def test_uniform_curl_patch():
    """A field with uniform curl (0, 0, B) has circ/area = B on every z-face and 0 elsewhere,
    so K e = 0 on every edge whose four faces all exist, on any tensor grid."""
    g = _nonuniform_grid(4)
    L = g.edge_lengths()
    nx, ny, nz = g.nx, g.ny, g.nz
    # edge midpoints
    xm = np.concatenate([np.broadcast_to(0.5 * (g.xn[:-1] + g.xn[1:])[None, None, :], (nz + 1, ny + 1, nx)).ravel(),
                         np.broadcast_to(g.xn[None, None, :], (nz + 1, ny, nx + 1)).ravel(),
                         np.broadcast_to(g.xn[None, None, :], (nz, ny + 1, nx + 1)).ravel()])
    ym = np.concatenate([np.broadcast_to(g.yn[None, :, None], (nz + 1, ny + 1, nx)).ravel(),
                         np.broadcast_to(0.5 * (g.yn[:-1] + g.yn[1:])[None, :, None], (nz + 1, ny, nx + 1)).ravel(),
                         np.broadcast_to(g.yn[None, :, None], (nz, ny + 1, nx + 1)).ravel()])
    B = 2.5
    e = np.zeros(g.n_edges)
    e[:g.n_ex] = -0.5 * B * ym[:g.n_ex]
    e[g.n_ex:g.n_ex + g.n_ey] = 0.5 * B * xm[g.n_ex:g.n_ex + g.n_ey]
    C, area, _ = g.curl()
    b = (C @ e) / area
    nxf = nz * ny * (nx + 1) + nz * (ny + 1) * nx
    assert np.allclose(b[nxf:], B, rtol=1e-12)
    assert np.allclose(b[:nxf], 0.0, atol=1e-12 * B)
    Ke = g.stiffness() @ e
    # interior edges (no boundary face is missing) see zero
    mask = g.interior_mask()
    assert np.abs(Ke[mask]).max() <= 1e-9 * B / MU0 * L.max()
    del L


def test_mass_total_and_interior_value():
    """Each cell hands V_c/4 to each of its 12 edges: sum M = 3 sum sigma V."""
    g = _nonuniform_grid(5)
    rng = np.random.default_rng(6)
    sigma = 10 ** rng.uniform(-3, 0, g.nx * g.ny * g.nz)
    V = (g.hz[:, None, None] * g.hy[None, :, None] * g.hx[None, None, :]).ravel()
    M = g.mass(sigma)
    assert np.isclose(M.sum(), 3.0 * (sigma * V).sum(), rtol=1e-13)
    gu = YeeGrid(np.full(4, 2.0), np.full(4, 2.0), np.full(4, 2.0))
    Mu = gu.mass(np.full(64, 0.3))
    # an interior edge of a uniform grid carries sigma * h^3
    assert np.isclose(Mu[gu.ex(1, 2, 2)], 0.3 * 8.0, rtol=1e-14)


def _closed_form_spectrum(n, h, sigma):
    """Eigenvalues of M^{-1} K on an n^3 Yee cube with n x e = 0 walls:
    (4 / (mu0 sigma h^2)) (s_a + s_b + s_c), s_q = sin^2(q pi / (2 n));
    two modes when a, b, c >= 1, one when exactly one index is 0,
    and (n-1)^3 gradient modes at 0."""
    s = np.sin(np.arange(n) * np.pi / (2 * n)) ** 2
    lam = [0.0] * (n - 1) ** 3
    for a in range(n):
        for b in range(n):
            for c in range(n):
                zeros = (a == 0) + (b == 0) + (c == 0)
                if zeros >= 2:
                    continue
                mult = 2 if zeros == 0 else 1
                lam += [4.0 / (MU0 * sigma * h * h) * (s[a] + s[b] + s[c])] * mult
    return np.sort(np.array(lam))


@pytest.mark.parametrize("n", [3, 4])
def test_uniform_cube_spectrum_closed_form(n):
    h, sigma = 1.5, 0.2
    g = YeeGrid(np.full(n, h), np.full(n, h), np.full(n, h))
    mask = g.interior_mask()
    K = g.stiffness()[mask][:, mask].toarray()
    M = g.mass(np.full(n ** 3, sigma))[mask]
    s = 1.0 / np.sqrt(M)
    lam = np.sort(np.linalg.eigvalsh(s[:, None] * K * s[None, :]))
    ref = _closed_form_spectrum(n, h, sigma)
    assert lam.size == ref.size == 3 * n * (n - 1) ** 2
    assert np.allclose(lam, ref, rtol=1e-9, atol=1e-9 * ref.max())


def test_loop_source_divergence_free_and_moment():
    """A closed loop current has zero discrete divergence (G^T f = 0 at every node)
    and magnetic moment I * area along +z when counter-clockwise."""
    g = YeeGrid(np.full(8, 10.0), np.full(8, 10.0), np.full(6, 10.0), origin=(-40.0, -40.0, -30.0))
    loop = np.array([[-20.0, -20.0], [30.0, -20.0], [30.0, 10.0], [-20.0, 10.0]])
    f = g.loop_source(loop, 0.0, current=2.0)
    assert np.abs(g.gradient().T @ f).max() <= 1e-12
    # moment m_z = 1/2 sum (x dy - y dx) I  over the loop edges
    nx, ny, nz = g.nx, g.ny, g.nz
    xm_x = np.broadcast_to(0.5 * (g.xn[:-1] + g.xn[1:])[None, None, :], (nz + 1, ny + 1, nx)).ravel()
    ym_x = np.broadcast_to(g.yn[None, :, None], (nz + 1, ny + 1, nx)).ravel()
    xm_y = np.broadcast_to(g.xn[None, None, :], (nz + 1, ny, nx + 1)).ravel()
    fx, fy = f[:g.n_ex], f[g.n_ex:g.n_ex + g.n_ey]
    mz = 0.5 * ((xm_y * fy).sum() - (ym_x * fx).sum())
    del xm_x
    assert np.isclose(mz, 2.0 * 50.0 * 30.0, rtol=1e-13)


def test_receiver_row_reads_uniform_curl():
    """d_t b_z = -(curl e)_z: a field of uniform curl B reads -B at any interior point."""
    g = _nonuniform_grid(7, n=(6, 6, 5))
    nx, ny, nz = g.nx, g.ny, g.nz
    ym = np.broadcast_to(g.yn[None, :, None], (nz + 1, ny + 1, nx)).ravel()
    xm = np.broadcast_to(g.xn[None, None, :], (nz + 1, ny, nx + 1)).ravel()
    e = np.zeros(g.n_edges)
    e[:g.n_ex] = -0.5 * 3.0 * ym
    e[g.n_ex:g.n_ex + g.n_ey] = 0.5 * 3.0 * xm
    for (x, y) in [(g.xn[2] + 0.1, g.yn[3] - 0.2), (g.xn[3], g.yn[3])]:
        q = g.receiver_row(x, y, g.zn[2] + 1e-3)
        assert np.isclose(q @ e, -3.0, rtol=1e-12)


def test_receiver_at_face_centre_uses_one_face():
    g = YeeGrid(np.full(4, 1.0), np.full(4, 2.0), np.full(3, 1.0))
    q = g.receiver_row(1.5, 3.0, 1.0)  # centre of z-face (1, 1, 1)
    nz_ = np.flatnonzero(q)
    assert len(nz_) == 4
    C, area, _ = g.curl()
    row = -C.getrow(g.zface_index(1, 1, 1)).toarray().ravel() / area[g.zface_index(1, 1, 1)]
    assert np.allclose(q, row)


def test_rejects_bad_geometry():
    g = YeeGrid(np.full(4, 1.0), np.full(4, 1.0), np.full(4, 1.0))
    with pytest.raises(ValueError):
        g.loop_source([[0.5, 0.0], [2.0, 0.0], [2.0, 2.0], [0.0, 2.0]], 1.0)
    with pytest.raises(ValueError):
        g.loop_source([[0.0, 0.0], [2.0, 1.0], [0.0, 2.0]], 1.0)
    with pytest.raises(ValueError):
        g.receiver_row(5.0, 1.0, 1.0)


def test_mass_derivative_sums_to_the_mass():
    """dM/dlog sigma_c = diag(D[:, c]) and M is linear in sigma, so sum_c D[:, c] = M, on any widths."""
    g = _nonuniform_grid(8)
    rng = np.random.default_rng(9)
    sigma = 10 ** rng.uniform(-3, 0, g.nx * g.ny * g.nz)
    D = g.mass_derivative(sigma)
    assert np.allclose(D @ np.ones(D.shape[1]), g.mass(sigma), rtol=1e-13, atol=0)
