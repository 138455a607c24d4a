"""Pins of the oracle's shared-pole fit (Sec. 3.2-3.3) against the paper's Table and mathematics."""
import os

import numpy as np
import pytest

from oracle import rational as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RATIOS = [1.0, 1e1, 1e2, 1e3, 1e4, 1e5]


def _table():
    rows = {}
    for line in open(os.path.join(GOLDEN, "degree_table.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        rows[float(v[0])] = [int(a) for a in v[1:]]
    return rows


def table_bound(ratio, m):
    """Accuracy the Table implies for degree m at this ratio: log-linear between its rows."""
    col = RATIOS.index(ratio)
    acc = sorted(_table().items(), key=lambda kv: kv[1][col])
    degs = np.array([r[col] for _, r in acc], dtype=float)
    logs = np.log10([a for a, _ in acc])
    return 10.0 ** np.interp(m, degs, logs)


# (ratio, degree): Table rows and the two degree/interval pairs the TEM models use
CASES = [(1e1, 9), (1e1, 14), (1e2, 14), (1e2, 16), (1e2, 20), (1e3, 18), (1e3, 20), (1e3, 27)]


@pytest.mark.parametrize("ratio,m", CASES)
def test_uniform_error_meets_table(ratio, m):
    """The Table lists, per interval ratio, the degree that reaches each accuracy.
    Our RKFIT-style family must reach that accuracy within a factor 2."""
    tau = np.logspace(-np.log10(ratio), 0.0, 31)
    xi, alpha = R.rkfit(tau, m)
    err, _ = R.uniform_error(tau, xi, alpha)
    assert err <= 2.0 * table_bound(ratio, m), (err, table_bound(ratio, m))


def test_poles_conjugate_pairs_off_spectrum():
    """Fig. 1: 28 poles in 14 exact conjugate pairs, none on [0, inf)."""
    tau = np.logspace(-3, 0, 31)
    xi, alpha = R.rkfit(tau, 28)
    up = np.sort_complex(xi[xi.imag > 0])
    lo = np.sort_complex(np.conj(xi[xi.imag < 0]))
    assert len(up) == 14 and np.array_equal(up, lo)
    # distance to [0, inf) relative to |xi| is bounded away from 0
    dist = np.where(xi.real >= 0, np.abs(xi.imag), np.abs(xi))
    assert np.all(dist > 0.3 * np.abs(xi))
    # residues of a conjugate pair are conjugate, so r^[j](x) is real on the real axis
    x = np.linspace(0, 50, 7)
    assert np.abs(R.evaluate(x, xi, alpha).imag).max() < 1e-12


def test_closest_pole_pair_fig1_not_reproduced():
    """Fig. 1 prints -7.574 +- 12.45i for the closest pair of the degree-28 family.
    The surrogate sampling and start of the paper's RKFIT run are not given; this
    fit lands in another local optimum with the same accuracy class.  Record
    both facts: our accuracy is at least as good as the Table's for degree 28,
    and our closest pair lies in the same left half-plane strip."""
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "pole_pin.txt")) if l[0] != "#")
    tau = np.logspace(np.log10(float(vals["t_min"])), 0.0, int(vals["K"]))
    xi, alpha = R.rkfit(tau, int(vals["degree"]))
    err, _ = R.uniform_error(tau, xi, alpha)
    assert err <= table_bound(1e3, 28)
    closest = xi[np.argmin(np.abs(xi))]
    assert closest.real < 0 and abs(closest.real - float(vals["closest_re"])) < 0.5 * abs(float(vals["closest_re"]))


def test_conj_reduce_identity():
    """sum_i alpha_i / (lam - xi_i) == sum_k Re(c_k / (lam - shift_k)) for real lam."""
    tau = np.logspace(-2, 0, 9)
    for m in (8, 9):
        xi, alpha = R.rkfit(tau, m, iters=6)
        sh, c = R.conj_reduce(xi, alpha)
        assert len(sh) == (m + 1) // 2
        lam = np.array([0.0, 0.3, 7.0, 1e3])
        full = (1.0 / (lam[:, None] - xi[None, :])) @ alpha
        red = ((1.0 / (lam[:, None] - sh[None, :])) @ c).real
        assert np.allclose(full.real, red, rtol=1e-12, atol=1e-14)


def test_odd_degree_has_one_real_pole():
    tau = np.logspace(-2, 0, 9)
    xi, alpha = R.rkfit(tau, 9, iters=6)
    assert np.sum(xi.imag == 0) >= 1 and np.sum(xi.imag == 0) % 2 == 1
    assert np.all(alpha[xi.imag == 0].imag == 0)


def test_residue_fit_reproduces_representable_target():
    """With poles fixed, the residue LSQ is exact when exp(-tau x) is replaced by a member of
    the family: fit the family's own values and get its residues back."""
    tau = np.logspace(-1, 0, 5)
    xi, alpha = R.rkfit(tau, 6, iters=4)
    x = R.surrogate_samples(tau.min(), 400)
    Phi = R.real_basis(x, xi, const=False)
    target = R.evaluate(x, xi, alpha).real
    coef, *_ = np.linalg.lstsq(Phi, target, rcond=None)
    assert np.allclose(Phi @ coef, target, atol=1e-12)


def test_solve_counts():
    """Sec. 3.1 / Sec. 5: K*ceil(m/2) solves for single-time approximants, ceil(m/2) for RKFIT."""
    vals = {}
    for line in open(os.path.join(GOLDEN, "solve_counts.txt")):
        if line[0] != "#" and line.strip():
            k, v = line.split()
            vals[k] = float(v)

    def single(m, K):
        return K * ((m + 1) // 2)

    def shared(m):
        return (m + 1) // 2

    assert single(14, 31) == vals["single_m14_K31"]
    assert shared(38) == vals["rkfit_m38"]
    assert single(14, 31) / shared(38) > vals["min_factor"]
    assert single(7, 31) == vals["single_m7_K31"]
    tau = np.logspace(-3, 0, 31)
    xi, alpha = R.rkfit(tau, 20, iters=4)
    assert len(R.conj_reduce(xi, alpha)[0]) == 10


def test_physical_scaling():
    """exp(-t lam) ~ sum Re(c / (lam - shift)) in physical units (Eq. (rmj) with t_max scaling)."""
    t = np.logspace(-5, -3, 11)
    sh, c, err = R.tem_poles_residues(t, 16)
    lam = np.logspace(1, 7, 50)
    approx = ((1.0 / (lam[:, None] - sh[None, :])) @ c).real
    assert np.abs(approx - np.exp(-np.outer(lam, t))).max() <= 1.01 * err + 1e-15


# Halphen's constant, the geometric rate of the best rational approximation to exp(-x) on
# [0, inf): error ~ 2 H^(-m-1/2) (Sec. 3.3, citing Trefethen, Approximation Theory and Practice).
HALPHEN = 9.289025491920819


def test_single_time_fit_follows_halphen():
    """The single-time approximant of Sec. 3.1 (the fitter on the one time t = 1, type [(m-1)/m]):
    for m = 3..10 its uniform error on [0, inf) lies between half and three times Halphen's
    2 H^(-m-1/2) (the best type-[m/m] error, which no approximant of this type can beat by more
    than the formula's asymptotic slack), falls by a factor H per degree on average, and it reaches
    each accuracy of the paper's Table (ratio-1 column: the classical best approximation) at
    that degree or one more."""
    errs = {}
    for m in range(2, 13):
        _, _, errs[m] = R.tem_poles_residues([1.0], m)
    for m in range(3, 11):
        h = 2.0 * HALPHEN ** (-m - 0.5)
        assert 0.5 * h <= errs[m] <= 3.0 * h, (m, errs[m], h)
    rate = np.exp(np.mean([np.log(errs[m] / errs[m + 1]) for m in range(3, 10)]))
    assert 7.5 <= rate <= 11.5, rate
    table = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "degree_table.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            table[float(v[0])] = int(v[1])
    for acc, m_best in table.items():
        m_ours = min(m for m in errs if errs[m] <= acc)
        assert m_best <= m_ours <= m_best + 1, (acc, m_best, m_ours)
