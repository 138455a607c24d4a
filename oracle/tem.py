"""Oracle: step-off TEM forward model and its adjoint gradient (FP64 CPU).

Test infrastructure only (see ``oracle/__init__.py``).

Forward (Eq. (rmj) projected with Q as in Eq. (rmjQ)): for shifts xi_i and
channel weights c[i, k] (c = 2 alpha for one pole of a conjugate pair, alpha
for a real pole),

    d[r, k] = sum_i Re( c[i, k] q_r^T (K - xi_i M)^{-1} f ),

with q_r the receiver rows (d_t b_z) restricted to the interior edges.

Adjoint (Sec. 4, the Jacobian of Eq. (rmjQ)): with m_c = log sigma_c,
M(m) = sum_c e^{m_c} M_c and dA_i/dm_c = -xi_i e^{m_c} M_c, the product of the
Jacobian's transpose with g = dphi/dd is

    dphi/dm_c = sum_i Re( xi_i lambda_i^T (e^{m_c} M_c) x_i ),
    lambda_i = A_i^{-T} w_i = A_i^{-1} w_i,  w_i = sum_r beta[i, r] q_r,
    beta[i, r] = sum_k c[i, k] g[r, k]

(A_i is complex symmetric, so A_i^{-T} = A_i^{-1}).
"""
from __future__ import annotations

import numpy as np

from .yee import YeeGrid
from .solvers import factor_lu, solve_cocg, DenseEig

__all__ = ["TEMProblem"]


class TEMProblem:
    """Assembled interior system for one model: grid, conductivity, loop, receivers."""

    def __init__(self, hx, hy, hz, sigma, loop_xy, z_loop, rx_xyz, current=1.0, origin=(0.0, 0.0, 0.0)):
        self.grid = g = YeeGrid(hx, hy, hz, origin)
        self.sigma = np.asarray(sigma, dtype=np.float64).ravel()
        if self.sigma.size != g.nx * g.ny * g.nz:
            raise ValueError("sigma has the wrong size")
        mask = g.interior_mask()
        self.mask = mask
        Kall = g.stiffness()
        self.K = Kall[mask][:, mask].tocsr()
        self.Md = g.mass(self.sigma)[mask]
        self.f = g.loop_source(loop_xy, z_loop, current)[mask]
        rx = np.atleast_2d(np.asarray(rx_xyz, dtype=np.float64))
        self.Q = np.stack([g.receiver_row(*p)[mask] for p in rx])  # (n_rx, N)
        self._dMdm = None
        self._lu = {}

    @property
    def n(self):
        return self.K.shape[0]

    def _lu_solve(self, b, shift):
        """(K - shift M)^{-1} b by sparse LU; one factorisation per shift, kept for later right-hand
        sides of the same shift (the adjoint and linearised solves reuse the forward's)."""
        key = complex(shift)
        if key not in self._lu:
            self._lu[key] = factor_lu(self.K, self.Md, key)
        return self._lu[key].solve(np.asarray(b, dtype=np.complex128))

    def solve(self, shift, method="lu", tol=1e-13):
        if method == "lu":
            return self._lu_solve(self.f, shift)
        x, _, _ = solve_cocg(self.K, self.Md, self.f, shift, tol=tol)
        return x

    def forward(self, shifts, c, method="lu", tol=1e-13, return_solutions=False):
        """d[r, k] = sum_i Re(c[i, k] q_r^T x_i) with x_i = (K - xi_i M)^{-1} f."""
        xs = [self.solve(s, method, tol) for s in shifts]
        y = np.stack([self.Q @ x for x in xs])  # (s, n_rx) complex
        d = np.einsum("ik,ir->rk", np.asarray(c), y).real
        return (d, xs) if return_solutions else d

    def combine(self, xs, c):
        """The projection and combination alone, for given solutions x_i."""
        y = np.stack([self.Q @ np.asarray(x) for x in xs])
        return np.einsum("ik,ir->rk", np.asarray(c), y).real

    def mass_derivative(self):
        if self._dMdm is None:
            self._dMdm = self.grid.mass_derivative(self.sigma)[self.mask].tocsc()
        return self._dMdm

    def adjoint_gradient(self, shifts, c, dphi_dd, xs=None, method="lu"):
        """dphi/dlog sigma (one value per cell) for dphi/dd = dphi_dd[n_rx, K]."""
        if xs is None:
            xs = [self.solve(s, method) for s in shifts]
        beta = np.asarray(c) @ np.asarray(dphi_dd).T  # (s, n_rx)
        D = self.mass_derivative()  # edges x cells: sigma_c V_c / 4 on the cell's edges
        g = np.zeros(self.sigma.size)
        for i, s in enumerate(shifts):
            w = beta[i] @ self.Q
            if method == "lu":
                lam = self._lu_solve(w, s)
            else:
                lam, _, _ = solve_cocg(self.K, self.Md, w, s)
            g += (s * (D.T @ (lam * xs[i]))).real
        return g

    def jvp(self, shifts, c, dlogsigma, xs=None, method="lu"):
        """J dm for dm = d log sigma (one value per cell), Sec. 4: with A_i = K - xi_i M(m) and
        dA_i/dm_c = -xi_i e^{m_c} M_c,  d(A_i^{-1} f)/dm . dm = xi_i A_i^{-1} (sum_c dm_c e^{m_c} M_c) g_i,
        g_i = A_i^{-1} f, so  (J dm)[r, k] = sum_i Re(c[i, k] xi_i q_r^T A_i^{-1} (dM g_i)),
        dM = diag(D dm) with D[e, c] = sigma_c V_c / 4 on the cell's edges."""
        if xs is None:
            xs = [self.solve(s, method) for s in shifts]
        dM = self.mass_derivative() @ np.asarray(dlogsigma, dtype=np.float64).ravel()
        y = []
        for i, s in enumerate(shifts):
            b = s * (dM * xs[i])
            if method == "lu":
                dx = self._lu_solve(b, s)
            else:
                dx, _, _ = solve_cocg(self.K, self.Md, b, s)
            y.append(self.Q @ dx)
        return np.einsum("ik,ir->rk", np.asarray(c), np.stack(y)).real

    def dense(self):
        """T0 route for tiny grids."""
        return DenseEig(self.K, self.Md)

    def exact_response(self, t, eig=None):
        """Q exp(-t M^{-1} K) M^{-1} f per channel (Eq. (expm)), shape (n_rx, K)."""
        eig = eig or self.dense()
        return np.stack([self.Q @ eig.expm(tk, self.f) for tk in np.atleast_1d(t)], axis=1)
