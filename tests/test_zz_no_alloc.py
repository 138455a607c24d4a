"""tem_apply_operator_noalloc against tem_apply_operator, through the C ABI.

The no-allocation entry point serves callers that may not allocate device memory (a host
framework that owns all of it, or a loop that must not risk cudaMalloc's synchronisation).
It keeps the shifts in one static device array shared by all calls.  Two calls in a row,
with different shifts and precisions, must each give the same q as the allocating entry
point (within the operator tests' tolerance), so the second call cannot be reading the
first call's shifts.  This file sorts last so that a stop-at-first-failure run has already
run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _setup(nx=40, ny=20, nz=36, seed=3):
    from paper_2506_11657_gb300 import tem
    rng = np.random.default_rng(seed)
    hx, hy, hz = rng.uniform(5, 20, nx), rng.uniform(5, 20, ny), rng.uniform(5, 20, nz)
    sigma = 10 ** rng.uniform(-8, 0, nx * ny * nz)
    grid = tem.Grid(hx, hy, hz, (0, 0, 0), sigma)
    return tem, grid, 3 * nx * ny * nz, rng


def _random_p(rng, s, n3, dtype):
    p = rng.standard_normal((s, n3)) + 1j * rng.standard_normal((s, n3))
    return torch.tensor(p, dtype=dtype, device="cuda")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    tem, grid, n3, rng = _setup()
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    pr = tem.PREC_FP64 if prec == "fp64" else tem.PREC_MIXED
    tol = 1e-13 if prec == "fp64" else 2e-6
    calls = [np.array([-800 + 250j, 3e4 + 1e5j, -5.0 + 0j]), np.array([1e5 - 4e3j, -2.5e3 + 7e2j])]
    for shifts in calls:
        p = _random_p(rng, len(shifts), n3, dt)
        # p's boundary entries must be zero: take them from the allocating call's q mask
        q_ref = torch.zeros_like(p)
        tem.apply_operator(grid, shifts, p, q_ref, pr)
        torch.cuda.synchronize()
        mask = (q_ref != 0).any(dim=0)
        p = p * mask
        tem.apply_operator(grid, shifts, p, q_ref, pr)
        q = torch.full_like(p, float("nan"))
        tem.apply_operator_noalloc(grid, shifts, p, q, pr)
        torch.cuda.synchronize()
        a, b = q.cpu().numpy(), q_ref.cpu().numpy()
        scale = np.abs(b).max()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= tol * scale


def test_noalloc_rejects_too_many_shifts():
    tem, grid, n3, rng = _setup(8, 8, 8)
    shifts = np.full(65, -100.0 + 10j)
    p = torch.zeros((65, 3 * 8 * 8 * 8), dtype=torch.complex128, device="cuda")
    q = torch.zeros_like(p)
    with pytest.raises(tem.TEMError) as e:
        tem.apply_operator_noalloc(grid, shifts, p, q, tem.PREC_FP64)
    assert e.value.code == tem.TEM_EINVAL
