"""Gauss-Newton steps for the log-conductivity from TEM data (Sec. 4, "Using iterative solvers").

The rational forward d(m) (m = log sigma per cell) is linearised at the current model and
the step solves the damped least-squares problem of the paper's Tikhonov extension,

    min_dm || [W J ; sqrt(lam) I] dm - [W (d(m) - d_obs) ; sqrt(lam) (m - m_ref)] ||_2,
    m_next = m - alpha dm,

with CGLS (Bjorck), which needs only the actions J v (tem_jvp) and J^T u (tem_adjoint):
each CGLS iteration is one of each, i.e. two batched solves over the shared poles.  W is an
optional diagonal data weighting; `active` restricts the update to a subset of cells (for
example the earth below the air).  The vector algebra over cells runs on the host; every
J or J^T action runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import tem


def cgls(apply_a, apply_at, b, n_iter, tol=0.0):
    """CGLS for min ||A x - b||_2 from x = 0.  apply_a(x) -> A x, apply_at(r) -> A^T r.
    Stops after n_iter iterations or once ||A^T r|| <= tol ||A^T b||.  Returns (x, history)
    with history[k] = ||b - A x_k||_2."""
    r = np.array(b, dtype=np.float64, copy=True)
    s = apply_at(r)
    x = np.zeros_like(s)
    p = s.copy()
    gamma = float(s @ s)
    gamma0 = gamma
    hist = [float(np.linalg.norm(r))]
    for _ in range(int(n_iter)):
        if gamma == 0.0 or gamma <= (tol * tol) * gamma0:
            break
        q = apply_a(p)
        qq = float(q @ q)
        if qq == 0.0:
            break
        alpha = gamma / qq
        x += alpha * p
        r -= alpha * q
        s = apply_at(r)
        gamma_new = float(s @ s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        hist.append(float(np.linalg.norm(r)))
    return x, hist


@dataclass
class StepResult:
    m: np.ndarray            # the updated model (log sigma per cell)
    d: np.ndarray            # forward response at the model the step started from
    misfit: float            # ||W (d - d_obs)|| at that model
    cgls_residuals: list     # CGLS history of the damped linear problem


def gauss_newton_step(grid: tem.Grid, model, m, d_obs, shifts, c, options=None, lam=0.0, m_ref=None,
                      weights=None, active=None, n_cgls=10, alpha=1.0) -> StepResult:
    """One Gauss-Newton step from m (log sigma, one value per cell of `grid`).

    model supplies the loop (loop_xy, z_loop) and receivers (rx); d_obs has the forward's
    (n_rx, K) layout; weights (same layout) scales the data residual; m_ref (default m)
    is the Tikhonov reference; active (boolean per cell) masks the update."""
    m = np.asarray(m, dtype=np.float64).ravel()
    n = m.size
    mask = np.ones(n, dtype=bool) if active is None else np.asarray(active, dtype=bool).ravel()
    Wd = np.ones_like(np.asarray(d_obs, dtype=np.float64)) if weights is None else np.asarray(weights, np.float64)
    m_ref = m if m_ref is None else np.asarray(m_ref, dtype=np.float64).ravel()
    sl = float(np.sqrt(lam))
    grid.set_sigma(np.exp(m))
    res = tem.forward(grid, model.loop_xy, model.z_loop, model.rx, shifts, c, options, keep_state=True)
    try:
        if res.status != tem.TEM_OK:
            raise tem.TEMError(res.status, "gauss_newton_step forward")
        r_data = (Wd * (res.d - d_obs)).ravel()
        nd = r_data.size

        def apply_a(v):
            full = np.zeros(n)
            full[mask] = v
            jd = (Wd * res.state.jvp(full)).ravel()
            return np.concatenate((jd, sl * v)) if sl > 0 else jd

        def apply_at(u):
            g = res.state.adjoint((Wd.ravel() * u[:nd]).reshape(res.d.shape))[mask]
            return g + sl * u[nd:] if sl > 0 else g

        b = np.concatenate((r_data, sl * (m - m_ref)[mask])) if sl > 0 else r_data
        dm, hist = cgls(apply_a, apply_at, b, n_cgls)
    finally:
        if res.state is not None:
            res.state.close()
    m_new = m.copy()
    m_new[mask] -= alpha * dm
    return StepResult(m_new, res.d, float(np.linalg.norm(r_data)), hist)


def objective(grid: tem.Grid, model, m, d_obs, shifts, c, options=None, lam=0.0, m_ref=None, weights=None):
    """phi(m) = ||W (d(m) - d_obs)||^2 + lam ||m - m_ref||^2 (one forward)."""
    m = np.asarray(m, dtype=np.float64).ravel()
    grid.set_sigma(np.exp(m))
    res = tem.forward(grid, model.loop_xy, model.z_loop, model.rx, shifts, c, options)
    if res.status != tem.TEM_OK:
        raise tem.TEMError(res.status, "objective forward")
    Wd = 1.0 if weights is None else np.asarray(weights, np.float64)
    phi = float(np.sum((Wd * (res.d - d_obs)) ** 2))
    if lam > 0:
        ref = m if m_ref is None else np.asarray(m_ref, dtype=np.float64).ravel()
        phi += lam * float(np.sum((m - ref) ** 2))
    return phi, res.d


def gauss_newton(grid: tem.Grid, model, m0, d_obs, shifts, c, options=None, n_steps=1, lam=0.0, m_ref=None,
                 weights=None, active=None, n_cgls=10, alphas=(1.0, 0.5, 0.25, 0.125, 0.0625)):
    """Gauss-Newton iterations with a backtracking choice of the step length alpha (the first
    of `alphas` that lowers the objective).  Returns (m, history) with history[l] = phi(m_l);
    stops early when no alpha lowers phi."""
    m = np.asarray(m0, dtype=np.float64).ravel().copy()
    m_ref = m.copy() if m_ref is None else np.asarray(m_ref, dtype=np.float64).ravel()
    phi, _ = objective(grid, model, m, d_obs, shifts, c, options, lam, m_ref, weights)
    history = [phi]
    for _ in range(int(n_steps)):
        step = gauss_newton_step(grid, model, m, d_obs, shifts, c, options, lam, m_ref, weights, active, n_cgls,
                                 alpha=1.0)
        full = m - step.m
        for a in alphas:
            trial = m - a * full
            phi_t, _ = objective(grid, model, trial, d_obs, shifts, c, options, lam, m_ref, weights)
            if phi_t < phi:
                m, phi = trial, phi_t
                break
        else:
            break
        history.append(phi)
    grid.set_sigma(np.exp(m))
    return m, history
