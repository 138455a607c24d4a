"""Oracle: closed-form step-off response at the centre of a circular loop on a halfspace.

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 5 compares against a 1-D semi-analytic solution for a loop on a conducting
halfspace and quotes the late-time decay of d_t b_z as t^{-5/2} (Sec. 5.2).
The central-loop step-off response of a homogeneous halfspace has the
well-known closed form (Ward & Hohmann 1988, in Nabighian (ed.),
"Electromagnetic Methods in Applied Geophysics", the reference the paper cites
for the decay rates):

    d_t h_z = -I / (mu0 sigma a^3) [ 3 erf(u) - (2/sqrt(pi)) u (3 + 2 u^2) e^{-u^2} ],
    u = theta a,  theta = sqrt(mu0 sigma / (4 t)),

and d_t b_z = mu0 d_t h_z (quasi-static, non-magnetic ground).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from .yee import MU0

__all__ = ["dbzdt_central_loop", "late_time_dbzdt"]


def _bracket(u):
    """3 erf(u) - (2/sqrt(pi)) u (3 + 2u^2) e^{-u^2}.

    For small u the two terms cancel to O(u^5); there the Taylor series of erf
    and exp combine to (2/sqrt(pi)) sum_{n>=2} (-1)^n 4 n (n-1) u^{2n+1} / (n! (2n+1)).
    """
    u = np.asarray(u, dtype=np.float64)
    direct = 3.0 * erf(u) - (2.0 / np.sqrt(np.pi)) * u * (3.0 + 2.0 * u * u) * np.exp(-u * u)
    series = np.zeros_like(u)
    for n in range(2, 30):
        fact = float(np.prod(np.arange(1, n + 1)))
        series += (-1.0) ** n * 4.0 * n * (n - 1) * u ** (2 * n + 1) / (fact * (2 * n + 1))
    series *= 2.0 / np.sqrt(np.pi)
    return np.where(u < 0.5, series, direct)


def dbzdt_central_loop(t, sigma, a, current=1.0):
    """d_t b_z (T/s) at the centre of a loop of radius a (m) after step-off."""
    t = np.asarray(t, dtype=np.float64)
    u = np.sqrt(MU0 * sigma / (4.0 * t)) * a
    return MU0 * (-current / (MU0 * sigma * a ** 3)) * _bracket(u)


def late_time_dbzdt(t, sigma, a, current=1.0):
    """The t -> inf limit: -I a^2 sigma^{3/2} mu0^{5/2} / (20 sqrt(pi) t^{5/2})."""
    t = np.asarray(t, dtype=np.float64)
    return -current * a * a * sigma ** 1.5 * MU0 ** 2.5 / (20.0 * np.sqrt(np.pi) * t ** 2.5)
