"""Seeded synthetic TEM models (inputs only; no part of the method's arithmetic).

Each builder returns a ``Model``: cell widths, origin, per-cell conductivity,
a square transmitter loop on the air-earth interface, receivers and channel
times.  Both the CUDA path and the CPU oracle consume these arrays; this module
imports neither.

Conventions: z points up; the air-earth interface is the node plane z = 0;
conductivity is stored per cell in (nz, ny, nx) order (x fastest); the loop is
counter-clockwise seen from +z (moment along +z); channel times are
log-spaced including both end points.

Named models (sizes and value ranges of the workloads they stand in for):

* ``tiny16``       16^3 cells of 20 m; top 6 layers air (1e-8 S/m), 0.01 S/m
                   halfspace; 80 m loop; 21 channels on [1e-5, 1e-3] s, degree 16.
* ``layered64``    64^3 cells: 48 core cells of 10 m plus 8 padding cells per
                   side growing by 1.15; air above; 100/10/1000 Ohm m layers
                   (0-30 m, 30-60 m, below); 100 m loop; 31 channels on
                   [1e-5, 1e-2] s, degree 20.
* ``randblock128`` 128^3 cells of 10 m; top 16 layers air; 8^3-cell blocks with
                   log10 rho ~ U[0, 3] (seed 3); 200 m loop; 31 channels on
                   [1e-5, 1e-2] s, degree 20.
* ``adjoint96``    96^3 cells of 10 m; top 16 layers air; 300 Ohm m host under a
                   30 m 100 Ohm m cover, 4 blocks of 5-50 Ohm m (seed 5); 150 m
                   loop; 64 receivers on an 8 x 8 grid at 25 m; 31 channels,
                   degree 20.
* ``serving_stream`` 256 requests (seed 4): n in {32, 48, 64, 96}, 3 layers plus
                   random blocks (log-uniform 1-1000 Ohm m), loop 50-200 m
                   snapped to the grid, degree 16-20, 31 channels, Poisson
                   arrival times.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SIGMA_AIR = 1e-8

__all__ = ["Model", "uniform_model", "tiny16", "layered64", "randblock128", "adjoint96",
           "serving_stream", "channel_times", "by_name"]


@dataclass
class Model:
    name: str
    hx: np.ndarray
    hy: np.ndarray
    hz: np.ndarray
    origin: tuple
    sigma: np.ndarray          # (nz, ny, nx) float64
    loop_xy: np.ndarray        # (n_vertices, 2)
    z_loop: float
    rx: np.ndarray             # (n_rx, 3)
    t: np.ndarray              # (K,)
    degree: int
    current: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (len(self.hx), len(self.hy), len(self.hz))

    @property
    def n_cells(self):
        return len(self.hx) * len(self.hy) * len(self.hz)


def channel_times(t_min, t_max, K):
    return np.logspace(np.log10(t_min), np.log10(t_max), K)


def _centres(h, origin):
    nodes = origin + np.concatenate(([0.0], np.cumsum(h)))
    return 0.5 * (nodes[:-1] + nodes[1:]), nodes


def _square_loop(side, nodes_x, nodes_y):
    """Square loop of about `side` metres centred on 0, snapped to grid nodes."""
    half = side / 2.0
    xa = nodes_x[np.argmin(np.abs(nodes_x + half))]
    xb = nodes_x[np.argmin(np.abs(nodes_x - half))]
    ya = nodes_y[np.argmin(np.abs(nodes_y + half))]
    yb = nodes_y[np.argmin(np.abs(nodes_y - half))]
    return np.array([[xa, ya], [xb, ya], [xb, yb], [xa, yb]], dtype=np.float64)


def uniform_model(n, h, air_layers, sigma_earth, loop_side, t_min, t_max, K, degree, name=None,
                  ny=None, nz=None):
    """Uniform cells of width h, `air_layers` top layers of air, homogeneous earth below."""
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    hx, hy, hz = np.full(nx, float(h)), np.full(ny, float(h)), np.full(nz, float(h))
    origin = (-(nx // 2) * h, -(ny // 2) * h, -(nz - air_layers) * h)
    sigma = np.full((nz, ny, nx), float(sigma_earth))
    sigma[nz - air_layers:] = SIGMA_AIR
    _, xn = _centres(hx, origin[0])
    _, yn = _centres(hy, origin[1])
    loop = _square_loop(loop_side, xn, yn)
    rx = np.array([[0.5 * (loop[0, 0] + loop[1, 0]), 0.5 * (loop[0, 1] + loop[2, 1]), 0.0]])
    return Model(name or f"uniform{nx}x{ny}x{nz}", hx, hy, hz, origin, sigma, loop, 0.0, rx,
                 channel_times(t_min, t_max, K), degree)


def tiny16():
    return uniform_model(16, 20.0, 6, 0.01, 80.0, 1e-5, 1e-3, 21, 16, name="tiny16")


def _padded(ncore, h, npad, factor):
    pad = h * factor ** np.arange(1, npad + 1)
    return np.concatenate((pad[::-1], np.full(ncore, float(h)), pad))


def layered64():
    h = 10.0
    hx = _padded(48, h, 8, 1.15)
    hy = hx.copy()
    # z: 8 padding + 40 core earth cells, interface, 8 core + 8 padding air cells
    pad = h * 1.15 ** np.arange(1, 9)
    hz = np.concatenate((pad[::-1], np.full(48, h), pad))
    origin = (-hx.sum() / 2, -hy.sum() / 2, -(pad.sum() + 40 * h))
    zc, _ = _centres(hz, origin[2])
    depth = -zc
    rho = np.where(depth < 0, 1.0 / SIGMA_AIR, np.where(depth < 30, 100.0, np.where(depth < 60, 10.0, 1000.0)))
    sigma = np.broadcast_to((1.0 / rho)[:, None, None], (len(hz), len(hy), len(hx))).copy()
    _, xn = _centres(hx, origin[0])
    _, yn = _centres(hy, origin[1])
    loop = _square_loop(100.0, xn, yn)
    rx = np.array([[0.0, 0.0, 0.0]])
    return Model("layered64", hx, hy, hz, origin, sigma, loop, 0.0, rx, channel_times(1e-5, 1e-2, 31), 20)


def _block_sigma(nz, ny, nx, air_layers, block, rng, log10_rho_range=(0.0, 3.0)):
    nbz, nby, nbx = -(-nz // block), -(-ny // block), -(-nx // block)
    lr = rng.uniform(log10_rho_range[0], log10_rho_range[1], size=(nbz, nby, nbx))
    s = 10.0 ** (-lr)
    s = np.repeat(np.repeat(np.repeat(s, block, 0), block, 1), block, 2)[:nz, :ny, :nx].copy()
    s[nz - air_layers:] = SIGMA_AIR
    return s


def randblock128(n=128, seed=3):
    h = 10.0
    air = n // 8
    hx = np.full(n, h)
    origin = (-(n // 2) * h, -(n // 2) * h, -(n - air) * h)
    rng = np.random.default_rng(seed)
    sigma = _block_sigma(n, n, n, air, 8, rng)
    _, xn = _centres(hx, origin[0])
    loop = _square_loop(200.0, xn, xn)
    rx = np.array([[0.0, 0.0, 0.0]])
    return Model(f"randblock{n}", hx, hx.copy(), hx.copy(), origin, sigma, loop, 0.0, rx,
                 channel_times(1e-5, 1e-2, 31), 20, meta={"seed": seed})


def adjoint96(n=96, seed=5, n_rx_side=8, h=10.0, blocks=True):
    """The adjoint-gradient model; n cells of h metres per side (n * h = 960 m keeps the physical
    model: n=24, h=40 is its 4x coarsening); blocks=False gives the layered background."""
    air = n // 6
    hx = np.full(n, h)
    origin = (-(n // 2) * h, -(n // 2) * h, -(n - air) * h)
    zc, _ = _centres(hx, origin[2])
    xc, xn = _centres(hx, origin[0])
    rho = np.full((n, n, n), 300.0)
    rho[(zc > -30.0) & (zc < 0.0)] = 100.0
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    for _ in range(4 if blocks else 0):
        bw = rng.integers(4, 10, size=3) * 10.0
        cx, cy = rng.uniform(-150, 150, size=2)
        top = -rng.uniform(30, 120)
        r = 10.0 ** rng.uniform(np.log10(5.0), np.log10(50.0))
        zsel = (zc <= top) & (zc >= top - bw[2])
        xy = (np.abs(X - cx) <= bw[0] / 2) & (np.abs(Y - cy) <= bw[1] / 2)
        rho[np.ix_(zsel, np.ones(n, bool), np.ones(n, bool))] = np.where(
            xy[None], r, rho[np.ix_(zsel, np.ones(n, bool), np.ones(n, bool))])
    sigma = 1.0 / rho
    sigma[zc > 0] = SIGMA_AIR
    loop = _square_loop(150.0, xn, xn)
    off = (np.arange(n_rx_side) - (n_rx_side - 1) / 2) * 25.0
    RX, RY = np.meshgrid(off, off, indexing="xy")
    rx = np.stack((RX.ravel(), RY.ravel(), np.zeros(RX.size)), axis=1)
    return Model(f"adjoint{n}", hx, hx.copy(), hx.copy(), origin, sigma, loop, 0.0, rx,
                 channel_times(1e-5, 1e-2, 31), 20, meta={"seed": seed, "h": h, "blocks": blocks})


def serving_stream(n_requests=256, seed=4, rate=1.0, sizes=(32, 48, 64, 96)):
    """Requests for the continuous-batching loop: (arrival time in s, Model)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    out = []
    for q in range(n_requests):
        n = int(rng.choice(sizes))
        h = 10.0
        air = n // 4
        hx = np.full(n, h)
        origin = (-(n // 2) * h, -(n // 2) * h, -(n - air) * h)
        zc, xn = _centres(hx, origin[2])
        _, xn = _centres(hx, origin[0])
        t1, t2 = np.sort(rng.uniform(5.0, 0.5 * (n - air) * h, size=2))
        r = 10.0 ** rng.uniform(0.0, 3.0, size=3)
        depth = -zc
        rho_l = np.where(depth < t1, r[0], np.where(depth < t2, r[1], r[2]))
        sigma = np.broadcast_to((1.0 / rho_l)[:, None, None], (n, n, n)).copy()
        blocks = 10.0 ** (-rng.uniform(0.0, 3.0, size=(n // 8, n // 8, n // 8)))
        bmask = rng.uniform(size=blocks.shape) < 0.15
        big = np.repeat(np.repeat(np.repeat(np.where(bmask, blocks, 0.0), 8, 0), 8, 1), 8, 2)
        sigma = np.where(big > 0, big, sigma)
        sigma[zc > 0] = SIGMA_AIR
        side = rng.uniform(50.0, 200.0)
        loop = _square_loop(side, xn, xn)
        if loop[1, 0] <= loop[0, 0]:
            loop = _square_loop(2 * h, xn, xn)
        m = int(rng.integers(16, 21))
        model = Model(f"req{q}_n{n}", hx, hx.copy(), hx.copy(), origin, sigma, loop, 0.0,
                      np.array([[0.0, 0.0, 0.0]]), channel_times(1e-5, 1e-2, 31), m)
        out.append((float(arrivals[q]), model))
    return out


def by_name(name):
    return {"tiny16": tiny16, "layered64": layered64, "randblock128": randblock128,
            "adjoint96": adjoint96}[name]()
