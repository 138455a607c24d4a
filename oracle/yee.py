"""Oracle: assembled Yee (staggered edge) discretisation of the TEM problem, FP64, SciPy.

Test infrastructure only (see ``oracle/__init__.py``).

Section 2.2 discretises Eq. (pde)-(source) with lowest-order Nedelec edge
elements; on a tensor-product hexahedral grid with lumped mass these are the
staggered Yee grid (finite-integration form):

* unknowns u_e: tangential E on every edge e, length L_e;
* circulation matrix C (faces x edges): circ_f = sum_{e in f} +-L_e u_e, the
  sign given by the right-hand rule about the face normal;
* stiffness K = C^T diag(L*_f / (mu0 A_f)) C  (Eq. for [K]_ij), with A_f the
  face area and L*_f the dual edge through f (distance between the centres of
  the two cells sharing f, half a cell at the domain boundary);
* mass M = diag(sum_{cells c containing e} sigma_c V_c / 4)  (Eq. for [M]_ij,
  lumped);
* source f_e = I L_e (+-1) on the edges of a closed loop of current I
  (Eq. for [f]_i with q the loop's line current, Sec. 2.1 step-off source);
* observation -d_t b_z = (curl e)_z ~ circ_f / A_f on z-faces (Sec. 5, the
  operator Q), bilinearly interpolated to the receiver; the row returned here
  gives d_t b_z itself, i.e. it carries the minus sign.

The boundary condition n x e = 0 (Eq. (bc)) removes the edges that lie in the
boundary: only "interior" edges are unknowns.

Edge numbering (this module's own): all x-edges, then y-edges, then z-edges;
x-edge (i, j, k) joins nodes (i, j, k)-(i+1, j, k) and has index
i + nx (j + (ny+1) k); y-edges (nz+1, ny, nx+1) and z-edges (nz, ny+1, nx+1)
follow likewise, x fastest.  Cell sigma is indexed i + nx (j + ny k).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MU0 = 4e-7 * np.pi  # Vs/(Am), Sec. 2.1

__all__ = ["MU0", "YeeGrid"]


def _dual(h: np.ndarray) -> np.ndarray:
    """Dual lengths at the n+1 node planes: mean of the two adjacent cell widths."""
    hp = np.concatenate(([0.0], h, [0.0]))
    return 0.5 * (hp[:-1] + hp[1:])


class YeeGrid:
    """Tensor grid with cell widths hx, hy, hz (metres) and origin (x0, y0, z0)."""

    def __init__(self, hx, hy, hz, origin=(0.0, 0.0, 0.0)):
        self.hx = np.asarray(hx, dtype=np.float64)
        self.hy = np.asarray(hy, dtype=np.float64)
        self.hz = np.asarray(hz, dtype=np.float64)
        self.nx, self.ny, self.nz = len(self.hx), len(self.hy), len(self.hz)
        self.origin = tuple(float(v) for v in origin)
        self.xn = self.origin[0] + np.concatenate(([0.0], np.cumsum(self.hx)))
        self.yn = self.origin[1] + np.concatenate(([0.0], np.cumsum(self.hy)))
        self.zn = self.origin[2] + np.concatenate(([0.0], np.cumsum(self.hz)))
        nx, ny, nz = self.nx, self.ny, self.nz
        self.n_ex = nx * (ny + 1) * (nz + 1)
        self.n_ey = (nx + 1) * ny * (nz + 1)
        self.n_ez = (nx + 1) * (ny + 1) * nz
        self.n_edges = self.n_ex + self.n_ey + self.n_ez
        self.n_nodes = (nx + 1) * (ny + 1) * (nz + 1)

    # ---- index maps -------------------------------------------------------
    def ex(self, i, j, k):
        return i + self.nx * (j + (self.ny + 1) * k)

    def ey(self, i, j, k):
        return self.n_ex + i + (self.nx + 1) * (j + self.ny * k)

    def ez(self, i, j, k):
        return self.n_ex + self.n_ey + i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def node(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def edge_lengths(self) -> np.ndarray:
        nx, ny, nz = self.nx, self.ny, self.nz
        Lx = np.broadcast_to(self.hx[None, None, :], (nz + 1, ny + 1, nx)).ravel()
        Ly = np.broadcast_to(self.hy[None, :, None], (nz + 1, ny, nx + 1)).ravel()
        Lz = np.broadcast_to(self.hz[:, None, None], (nz, ny + 1, nx + 1)).ravel()
        return np.concatenate((Lx, Ly, Lz))

    def interior_mask(self) -> np.ndarray:
        """True for edges not lying in the boundary (Eq. (bc): n x e = 0)."""
        nx, ny, nz = self.nx, self.ny, self.nz
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx), indexing="ij")
        mx = (j > 0) & (j < ny) & (k > 0) & (k < nz)
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx + 1), indexing="ij")
        my = (i > 0) & (i < nx) & (k > 0) & (k < nz)
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        mz = (i > 0) & (i < nx) & (j > 0) & (j < ny)
        return np.concatenate((mx.ravel(), my.ravel(), mz.ravel()))

    # ---- operators --------------------------------------------------------
    def curl(self):
        """Circulation matrix C (faces x edges) and per-face (area, dual length).

        Face order: x-faces (nz, ny, nx+1), y-faces (nz, ny+1, nx), z-faces
        (nz+1, ny, nx); each row holds the four signed edge lengths.
        """
        nx, ny, nz = self.nx, self.ny, self.nz
        hx, hy, hz = self.hx, self.hy, self.hz
        rows, cols, vals, area, dual = [], [], [], [], []
        off = 0
        # x-faces: normal +x, loop y -> z
        k, j, i = (a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx + 1), indexing="ij"))
        f = off + np.arange(i.size)
        for e, v in ((self.ey(i, j, k), hy[j]), (self.ez(i, j + 1, k), hz[k]),
                     (self.ey(i, j, k + 1), -hy[j]), (self.ez(i, j, k), -hz[k])):
            rows.append(f); cols.append(e); vals.append(v)
        area.append(hy[j] * hz[k]); dual.append(_dual(hx)[i])
        off += i.size
        # y-faces: normal +y, loop z -> x
        k, j, i = (a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny + 1), np.arange(nx), indexing="ij"))
        f = off + np.arange(i.size)
        for e, v in ((self.ez(i, j, k), hz[k]), (self.ex(i, j, k + 1), hx[i]),
                     (self.ez(i + 1, j, k), -hz[k]), (self.ex(i, j, k), -hx[i])):
            rows.append(f); cols.append(e); vals.append(v)
        area.append(hz[k] * hx[i]); dual.append(_dual(hy)[j])
        off += i.size
        # z-faces: normal +z, loop x -> y
        k, j, i = (a.ravel() for a in np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij"))
        f = off + np.arange(i.size)
        for e, v in ((self.ex(i, j, k), hx[i]), (self.ey(i + 1, j, k), hy[j]),
                     (self.ex(i, j + 1, k), -hx[i]), (self.ey(i, j, k), -hy[j])):
            rows.append(f); cols.append(e); vals.append(v)
        area.append(hx[i] * hy[j]); dual.append(_dual(hz)[k])
        off += i.size
        C = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(off, self.n_edges))
        return C, np.concatenate(area), np.concatenate(dual)

    def zface_index(self, i, j, k):
        """Row of C for z-face (i, j, k)."""
        nx, ny, nz = self.nx, self.ny, self.nz
        return nz * ny * (nx + 1) + nz * (ny + 1) * nx + i + nx * (j + ny * k)

    def stiffness(self) -> sp.csr_matrix:
        """K = C^T diag(L*_f / (mu0 A_f)) C over all edges."""
        C, area, dual = self.curl()
        return (C.T @ sp.diags(dual / (MU0 * area)) @ C).tocsr()

    def mass(self, sigma) -> np.ndarray:
        """Lumped edge mass M_e = sum over the 4 cells containing e of sigma_c V_c / 4."""
        nx, ny, nz = self.nx, self.ny, self.nz
        s = np.asarray(sigma, dtype=np.float64).reshape(nz, ny, nx)
        V = self.hz[:, None, None] * self.hy[None, :, None] * self.hx[None, None, :]
        q = 0.25 * s * V
        mx = np.zeros((nz + 1, ny + 1, nx)); my = np.zeros((nz + 1, ny, nx + 1)); mz = np.zeros((nz, ny + 1, nx + 1))
        for a in (0, 1):
            for b in (0, 1):
                mx[b:b + nz, a:a + ny, :] += q
                my[b:b + nz, :, a:a + nx] += q
                mz[:, b:b + ny, a:a + nx] += q
        return np.concatenate((mx.ravel(), my.ravel(), mz.ravel()))

    def mass_derivative(self, sigma) -> sp.csr_matrix:
        """D (edges x cells) with D[e, c] = sigma_c V_c / 4 if e lies on cell c: dM/dlog sigma_c = diag(D[:, c])."""
        nx, ny, nz = self.nx, self.ny, self.nz
        s = np.asarray(sigma, dtype=np.float64).ravel()
        k, j, i = (a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"))
        c = i + nx * (j + ny * k)
        V = self.hx[i] * self.hy[j] * self.hz[k]
        q = 0.25 * s[c] * V
        rows, cols, vals = [], [], []
        for a in (0, 1):
            for b in (0, 1):
                for e in (self.ex(i, j + a, k + b), self.ey(i + a, j, k + b), self.ez(i + a, j + b, k)):
                    rows.append(e); cols.append(c); vals.append(q)
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_edges, nx * ny * nz))

    def gradient(self) -> sp.csr_matrix:
        """Nodal gradient G (edges x nodes): (G phi)_e = (phi_end - phi_start) / L_e."""
        nx, ny, nz = self.nx, self.ny, self.nz
        rows, cols, vals = [], [], []
        k, j, i = (a.ravel() for a in np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx), indexing="ij"))
        e = self.ex(i, j, k)
        rows += [e, e]; cols += [self.node(i + 1, j, k), self.node(i, j, k)]; vals += [1 / self.hx[i], -1 / self.hx[i]]
        k, j, i = (a.ravel() for a in np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx + 1), indexing="ij"))
        e = self.ey(i, j, k)
        rows += [e, e]; cols += [self.node(i, j + 1, k), self.node(i, j, k)]; vals += [1 / self.hy[j], -1 / self.hy[j]]
        k, j, i = (a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny + 1), np.arange(nx + 1), indexing="ij"))
        e = self.ez(i, j, k)
        rows += [e, e]; cols += [self.node(i, j, k + 1), self.node(i, j, k)]; vals += [1 / self.hz[k], -1 / self.hz[k]]
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_edges, self.n_nodes))

    # ---- source and receivers --------------------------------------------
    def _snap(self, coords, v, what):
        idx = int(np.argmin(np.abs(coords - v)))
        span = coords[-1] - coords[0]
        if abs(coords[idx] - v) > 1e-9 * span:
            raise ValueError(f"{what} {v} is not on a grid node plane")
        return idx

    def loop_source(self, loop_xy, z_loop, current=1.0) -> np.ndarray:
        """f_e = I L_e (+-1) along a closed axis-aligned polygon through grid nodes.

        loop_xy: (n, 2) vertices in order; the polygon is closed back to the
        first vertex.  Counter-clockwise seen from +z gives a +z moment.
        """
        P = np.asarray(loop_xy, dtype=np.float64)
        k = self._snap(self.zn, z_loop, "loop height")
        f = np.zeros(self.n_edges)
        n = len(P)
        for a in range(n):
            (xa, ya), (xb, yb) = P[a], P[(a + 1) % n]
            ia, ja = self._snap(self.xn, xa, "loop x"), self._snap(self.yn, ya, "loop y")
            ib, jb = self._snap(self.xn, xb, "loop x"), self._snap(self.yn, yb, "loop y")
            if ia != ib and ja != jb:
                raise ValueError("loop segments must be axis-aligned")
            if ja == jb:
                step = 1 if ib > ia else -1
                for i in range(min(ia, ib), max(ia, ib)):
                    f[self.ex(i, ja, k)] += current * self.hx[i] * step
            else:
                step = 1 if jb > ja else -1
                for j in range(min(ja, jb), max(ja, jb)):
                    f[self.ey(ia, j, k)] += current * self.hy[j] * step
        return f

    def receiver_row(self, xr, yr, zr) -> np.ndarray:
        """Row q with q . u = d_t b_z at (xr, yr) on the node plane nearest zr.

        (curl e)_z on each z-face is circ_f / A_f, located at the face centre;
        it is interpolated bilinearly between face centres (clamped to the
        outermost centres) and negated (Faraday: d_t b = -curl e).
        """
        if not (self.xn[0] <= xr <= self.xn[-1] and self.yn[0] <= yr <= self.yn[-1]
                and self.zn[0] <= zr <= self.zn[-1]):
            raise ValueError("receiver outside the grid")
        k = int(np.argmin(np.abs(self.zn - zr)))
        xc = 0.5 * (self.xn[:-1] + self.xn[1:])
        yc = 0.5 * (self.yn[:-1] + self.yn[1:])

        def weights(c, v):
            if v <= c[0]:
                return [(0, 1.0)]
            if v >= c[-1]:
                return [(len(c) - 1, 1.0)]
            a = int(np.searchsorted(c, v, side="right") - 1)
            t = (v - c[a]) / (c[a + 1] - c[a])
            return [(a, 1.0 - t), (a + 1, t)]

        C, area, _ = self.curl()
        q = np.zeros(self.n_edges)
        for i, wi in weights(xc, xr):
            for j, wj in weights(yc, yr):
                fidx = self.zface_index(i, j, k)
                q -= wi * wj * C.getrow(fidx).toarray().ravel() / area[fidx]
        return q
