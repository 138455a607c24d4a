"""Oracle: the three FP64 CPU routes to (K - xi M)^{-1} f and exp(-t M^{-1} K) M^{-1} f.

Test infrastructure only (see ``oracle/__init__.py``).

* T0 ``DenseEig``: the generalised symmetric eigenproblem K w = lam M w solved
  densely through M^{-1/2} K M^{-1/2} = W diag(lam) W^T (Eq. (expm)); any
  function of M^{-1} K applied to b = M^{-1} f is then a diagonal scaling.
  Tiny grids only.
* T1 ``solve_lu``: sparse direct LU (SuperLU) of the complex symmetric shifted
  matrix K - xi M, one factorisation per pole (the paper factorises one matrix
  per pole with a direct solver, Sec. 5.3).
* T2 ``solve_cocg``: conjugate orthogonal CG (the unconjugated bilinear form
  x^T y, for complex symmetric matrices) with the Jacobi preconditioner
  diag(K - xi M), stopped on the FP64 residual recomputed from scratch.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = ["DenseEig", "factor_lu", "solve_lu", "solve_cocg"]


class DenseEig:
    """T0: dense eigendecomposition of M^{-1/2} K M^{-1/2} (M diagonal, positive)."""

    def __init__(self, K, Mdiag):
        Kd = K.toarray() if sp.issparse(K) else np.asarray(K)
        self.s = 1.0 / np.sqrt(np.asarray(Mdiag))
        self.lam, self.W = np.linalg.eigh(self.s[:, None] * Kd * self.s[None, :])

    def apply(self, fn, f):
        """fn(M^{-1} K) M^{-1} f = M^{-1/2} W fn(lam) W^T M^{-1/2} f."""
        y = self.W.T @ (self.s * f)
        return self.s * (self.W @ (fn(self.lam) * y))

    def expm(self, t, f):
        """Eq. (expm): u(t) = exp(-t M^{-1} K) M^{-1} f."""
        return self.apply(lambda lam: np.exp(-t * lam), f)

    def rational(self, shifts, c_k, f):
        """sum_i Re(c_i (K - xi_i M)^{-1} f) through the eigenbasis (Eq. (rmj))."""
        def fn(lam):
            return sum((ci / (lam - xi)).real for xi, ci in zip(shifts, c_k))
        return self.apply(fn, f)


def factor_lu(K, Mdiag, shift):
    """T1: the SuperLU factorisation of K - shift M in complex128 (its .solve(b) gives A^{-1} b)."""
    A = (K.astype(np.complex128) - shift * sp.diags(np.asarray(Mdiag, dtype=np.complex128))).tocsc()
    return spla.splu(A)


def solve_lu(K, Mdiag, f, shift):
    """T1: x = (K - shift M)^{-1} f by SuperLU in complex128."""
    return factor_lu(K, Mdiag, shift).solve(np.asarray(f, dtype=np.complex128))


def solve_cocg(K, Mdiag, f, shift, tol=1e-13, maxiter=20000, x0=None):
    """T2: Jacobi-preconditioned COCG for (K - shift M) x = f.

    Iterates the textbook recurrences (van der Vorst & Melissen 1990) with the
    unconjugated form (a, b) = sum a_e b_e:
        alpha = (r, z) / (p, A p);  x += alpha p;  r -= alpha A p;
        z = D^{-1} r;  beta = (r, z)_new / (r, z)_old;  p = z + beta p,
    D = diag(K) - shift M.  Stops once the recursively updated residual drops
    below tol ||f|| and confirms with the residual recomputed from x.
    Returns (x, iterations, true relative residual).
    """
    f = np.asarray(f, dtype=np.complex128)
    A = (K.astype(np.complex128) - shift * sp.diags(np.asarray(Mdiag, dtype=np.complex128))).tocsr()
    D = A.diagonal()
    nf = np.linalg.norm(f)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.complex128)
    r = f - A @ x
    z = r / D
    p = z.copy()
    rho = r @ z
    it = 0
    while it < maxiter:
        q = A @ p
        alpha = rho / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.linalg.norm(r) <= tol * nf:
            rt = f - A @ x
            if np.linalg.norm(rt) <= tol * nf:
                break
            r = rt  # replace the drifted recursive residual and go on
        z = r / D
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, it, float(np.linalg.norm(f - A @ x) / nf)
