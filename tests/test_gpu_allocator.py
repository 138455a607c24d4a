"""The library's device memory comes from PyTorch's caching allocator (tem_set_allocator, installed
by the binding): a grid and a forward solve show up as torch allocations on the caller's device,
and closing them gives the memory back to torch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_forward_memory_is_torch_memory():
    from paper_2506_11657_gb300 import tem
    assert tem.allocator() == "torch"
    m = W.uniform_model(24, 10.0, 6, 0.02, 80.0, 1e-5, 1e-3, 11, 12)
    shifts, c, _ = tem.poles_residues(m.t, m.degree)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    n = m.sigma.size
    assert torch.cuda.memory_allocated() - base >= n * (7 * 12 + 8)        # masses, diag K, sigma
    res = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, tem.default_options(precision="mixed"),
                      keep_state=True)
    assert res.status == tem.TEM_OK
    # the kept solutions: per shift two FP64 and five FP32 edge vectors (3 n complex each)
    assert torch.cuda.memory_allocated() - base >= len(shifts) * 3 * n * (2 * 16 + 5 * 8)
    res.state.close()
    grid.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    assert torch.cuda.max_memory_allocated() > base
