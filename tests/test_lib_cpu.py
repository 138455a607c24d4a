"""CPU-side checks of the C-ABI library: it builds, loads, exports every declared entry point,
and its host-only parts (argument validation, the pole fit) agree with the oracle."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_11657_gb300 import build, tem
    build.build()
    return tem


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(tem_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    import ctypes
    L = ctypes.CDLL(lib.LIB_PATH)
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert set(lib.EXPORTED) <= set(names)


def test_poles_residues_matches_oracle_fit(lib):
    """Same RKFIT steps in C++ and in the oracle: the two pole sets agree, and with the library's
    poles fixed the oracle's residue least squares reproduces the library's weights."""
    from oracle import rational as R
    for lo, hi, K, m in [(-5, -3, 21, 16), (-5, -2, 31, 20)]:
        t = np.logspace(lo, hi, K)
        sh, c, err = lib.poles_residues(t, m)
        sh2, c2, err2 = R.tem_poles_residues(t, m)
        assert len(sh) == m // 2
        assert np.max(np.abs(sh - sh2) / np.abs(sh2)) < 1e-4
        assert abs(err - err2) <= 0.01 * err2
        # residue step with the library's poles (normalised variable)
        tmax = t[-1]
        xi = np.concatenate([[z, np.conj(z)] for z in sh * tmax])
        x = R.surrogate_samples(t[0] / tmax)
        xi_o, alpha = R.fit_residues(x, t / tmax, xi)
        sh3, c3 = R.conj_reduce(xi_o, alpha)
        order = [int(np.argmin(np.abs(sh3 - z * tmax))) for z in sh]
        assert np.max(np.abs(c3[order] / tmax - c)) <= 1e-7 * np.abs(c).max()


def test_poles_residues_validation(lib):
    import ctypes as C
    t = np.array([1e-5, 1e-4, 1e-4])
    xi = np.zeros(32)
    c = np.zeros(200)
    s = C.c_int64()
    L = lib.lib()
    rc = L.tem_poles_residues(t.ctypes.data_as(lib._dp), 3, 16, None, xi.ctypes.data_as(lib._dp),
                              c.ctypes.data_as(lib._dp), C.byref(s), None)
    assert rc == lib.TEM_EINVAL
    rc = L.tem_poles_residues(t.ctypes.data_as(lib._dp), 3, 0, None, xi.ctypes.data_as(lib._dp),
                              c.ctypes.data_as(lib._dp), C.byref(s), None)
    assert rc == lib.TEM_EINVAL


def test_build_grid_validates_before_touching_the_device(lib):
    import ctypes as C
    h = np.full(4, 10.0)
    o = np.zeros(3)
    sig = np.full(64, 0.1)
    sig[3] = np.nan
    out = C.c_void_p()
    rc = lib.lib().tem_build_grid(h.ctypes.data_as(lib._dp), 4, h.ctypes.data_as(lib._dp), 4,
                                  h.ctypes.data_as(lib._dp), 4, o.ctypes.data_as(lib._dp),
                                  sig.ctypes.data_as(lib._dp), None, C.byref(out))
    assert rc == lib.TEM_EINVAL and not out.value
    rc = lib.lib().tem_build_grid(h.ctypes.data_as(lib._dp), 1, h.ctypes.data_as(lib._dp), 4,
                                  h.ctypes.data_as(lib._dp), 4, o.ctypes.data_as(lib._dp),
                                  sig.ctypes.data_as(lib._dp), None, C.byref(out))
    assert rc == lib.TEM_EINVAL


def test_status_strings(lib):
    assert lib.status_string(lib.TEM_OK) == "TEM_OK"
    assert "max_iter" in lib.status_string(lib.TEM_ENOCONV)


def test_default_options_and_struct_layout(lib):
    """tem_default_options fills every field of the binding's struct (the C struct ends with
    carry_direction; a field added on one side only would shift it)."""
    import ctypes as C
    o = lib.Options()
    C.memset(C.byref(o), 0x7f, C.sizeof(o))
    lib.lib().tem_default_options(C.byref(o))
    assert (o.precision, o.max_iter, o.tol, o.inner_tol) == (lib.PREC_FP64, 20000, 1e-12, 1e-1)
    assert (o.max_outer, o.check_every, o.keep_state, o.precond, o.carry_direction) == (40, 32, 0, 0, 1)
    assert C.sizeof(o) == 48


def test_late_time_weights_match_the_oracle_and_help_late_channels(lib):
    """Weights w_k = (t_k / t_K)^(5/2) (the late-time decay of Sec. 5.2): the C++ and oracle
    fitters agree, and the weighted family is far more accurate on the last channel than the
    unweighted one (at the cost of the first)."""
    from oracle import rational as R
    t = np.logspace(-5, -2, 31)
    w = (t / t[-1]) ** 2.5
    sh, c, err = lib.poles_residues(t, 20, w)
    sh2, c2, err2 = R.tem_poles_residues(t, 20, w=w)
    order = [int(np.argmin(np.abs(sh2 - z))) for z in sh]
    assert np.max(np.abs(sh - sh2[order]) / np.abs(sh2[order])) < 1e-4
    assert abs(err - err2) <= 0.01 * err2

    def per_channel(shifts, cc):
        tau, tm = t / t[-1], t[-1]
        x = np.concatenate([[0.0], np.logspace(-4, np.log10(1e4 / tau[0]), 20000)])
        r = np.real(np.sum(cc[:, None, :] * tm / (x[None, :, None] - (shifts * tm)[:, None, None]), axis=0))
        return np.abs(np.exp(-np.outer(x, tau)) - r).max(axis=0)

    e_w = per_channel(sh, c)
    e_u = per_channel(*lib.poles_residues(t, 20)[:2])
    assert e_w[-1] < 1e-2 * e_u[-1]
    assert e_w[0] > e_u[0]
    assert np.max(w * e_w) <= 1.01 * err


@pytest.mark.parametrize("lo,hi,K,m", [(-4, -3.5, 5, 30), (-4, -3.5, 5, 64), (-5, -3, 21, 48), (-5, -2, 31, 64)])
def test_saturated_fits_keep_poles_off_the_spectrum(lib, lo, hi, K, m):
    """Degrees far past the error floor: every shift stays off [0, inf) (the spurious real
    doublets a saturated fit can leave there are dropped) and the uniform error stays at
    rounding level."""
    t = np.logspace(lo, hi, K)
    sh, c, err = lib.poles_residues(t, m)
    assert np.all((sh.real < 0) | (sh.imag != 0))
    assert np.all(np.isfinite(c)) and err < 1e-10
