"""Thin ctypes binding of the TEM C ABI (include/tem.h).

Argument marshalling only: every step of the forward model, the adjoint and
the operator runs in libtem.so's CUDA kernels.  PyTorch supplies device memory
and streams: when torch has CUDA, loading the library installs PyTorch's caching
allocator as the library's allocator (tem_set_allocator), so every device buffer the
library creates is a torch allocation on the caller's stream (TEM_ALLOCATOR=cuda keeps
the library's own stream-ordered pool instead).  Loading fails loudly if the library
has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("TEM_LIB") or os.path.join(HERE, "libtem.so")   # TEM_LIB: another build of it

TEM_OK, TEM_EINVAL, TEM_ENOMEM, TEM_ENOCONV, TEM_EBREAKDOWN, TEM_ETIMEOUT, TEM_ECUDA, TEM_EBUSY = range(8)
PREC_FP64, PREC_MIXED = 0, 1
PRECOND_AUTO, PRECOND_JACOBI, PRECOND_NODAL = 0, 1, 2

EXPORTED = ["tem_default_options", "tem_status_string", "tem_version", "tem_set_allocator",
            "tem_build_grid", "tem_grid_set_sigma", "tem_grid_dims", "tem_grid_destroy",
            "tem_poles_residues", "tem_forward", "tem_forward_sources", "tem_forward_single_time", "tem_state_stats", "tem_state_solution", "tem_state_fields", "tem_adjoint", "tem_jvp",
            "tem_state_destroy", "tem_apply_operator", "tem_apply_operator_noalloc", "tem_launch_count",
            "tem_profile_passes", "tem_server_default_options", "tem_server_create", "tem_server_submit",
            "tem_server_step", "tem_server_poll", "tem_server_counts", "tem_server_destroy"]


class TEMError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} (code {code}) {last_error()}")


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("inner_tol", C.c_double), ("max_outer", C.c_int32), ("check_every", C.c_int32),
                ("keep_state", C.c_int32), ("precond", C.c_int32), ("carry_direction", C.c_int32)]


class ServerOptions(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32), ("iters_per_step", C.c_int32),
                ("solver", Options)]


class RequestStats(C.Structure):
    _fields_ = [("submit_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double),
                ("footprint_bytes", C.c_int64), ("status", C.c_int32), ("max_iters", C.c_int32)]


_lib = None
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)


def lib():
    """Load libtem.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    L = C.CDLL(LIB_PATH)
    L.tem_default_options.argtypes = [C.POINTER(Options)]
    L.tem_default_options.restype = None
    L.tem_status_string.argtypes = [C.c_int]
    L.tem_status_string.restype = C.c_char_p
    L.tem_last_error.argtypes = []
    L.tem_last_error.restype = C.c_char_p
    L.tem_version.restype = C.c_char_p
    L.tem_build_grid.argtypes = [_dp, C.c_int64, _dp, C.c_int64, _dp, C.c_int64, _dp, _dp, C.c_void_p,
                                 C.POINTER(C.c_void_p)]
    L.tem_grid_set_sigma.argtypes = [C.c_void_p, _dp, C.c_void_p]
    L.tem_grid_dims.argtypes = [C.c_void_p, _i64p]
    L.tem_grid_destroy.argtypes = [C.c_void_p]
    L.tem_poles_residues.argtypes = [_dp, C.c_int64, C.c_int64, _dp, _dp, _dp, _i64p, _dp]
    L.tem_forward.argtypes = [C.c_void_p, _dp, C.c_int64, C.c_double, C.c_double, _dp, C.c_int64, _dp, _dp,
                              C.c_int64, C.c_int64, C.POINTER(Options), C.c_void_p, _dp, C.POINTER(C.c_void_p)]
    L.tem_state_stats.argtypes = [C.c_void_p, _i32p, _dp]
    L.tem_forward_sources.argtypes = [C.c_void_p, _dp, _i64p, C.c_int64, _dp, _dp, _dp, C.c_int64, _dp, _dp,
                                      C.c_int64, C.c_int64, C.POINTER(Options), C.c_void_p, _dp]
    L.tem_forward_single_time.argtypes = [C.c_void_p, _dp, C.c_int64, C.c_double, C.c_double, _dp, C.c_int64, _dp,
                                          C.c_int64, _dp, _dp, C.c_int64, C.POINTER(Options), C.c_void_p, _dp, _i64p]
    L.tem_state_solution.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, _dp]
    L.tem_state_fields.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
    L.tem_adjoint.argtypes = [C.c_void_p, _dp, C.c_void_p, _dp]
    L.tem_jvp.argtypes = [C.c_void_p, _dp, C.c_void_p, _dp]
    L.tem_state_destroy.argtypes = [C.c_void_p]
    L.tem_apply_operator.argtypes = [C.c_void_p, _dp, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    L.tem_apply_operator_noalloc.argtypes = [C.c_void_p, _dp, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32,
                                             C.c_void_p]
    L.tem_server_default_options.argtypes = [C.POINTER(ServerOptions)]
    L.tem_server_default_options.restype = None
    L.tem_server_create.argtypes = [C.POINTER(ServerOptions), C.c_void_p, C.POINTER(C.c_void_p)]
    L.tem_server_submit.argtypes = [C.c_void_p, _dp, C.c_int64, _dp, C.c_int64, _dp, C.c_int64, _dp, _dp, _dp,
                                    C.c_int64, C.c_double, C.c_double, _dp, C.c_int64, _dp, _dp, C.c_int64,
                                    C.c_int64, _i64p]
    L.tem_server_step.argtypes = [C.c_void_p]
    L.tem_server_poll.argtypes = [C.c_void_p, C.c_int64, _dp, C.POINTER(RequestStats)]
    L.tem_server_counts.argtypes = [C.c_void_p, _i64p, _i64p, _i64p]
    L.tem_server_destroy.argtypes = [C.c_void_p]
    L.tem_launch_count.argtypes = []
    L.tem_launch_count.restype = C.c_int64
    L.tem_profile_passes.argtypes = [C.c_void_p, _dp, C.c_int64, C.c_double, C.c_double, _dp, C.c_int64, C.c_int32,
                                     C.c_int32, C.c_int32, C.c_void_p, _dp, _dp]
    L.tem_set_allocator.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    _lib = L
    _install_torch_allocator(L)
    return L


# ---- device memory from PyTorch's caching allocator (tem_set_allocator)
_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_allocator = "cuda"


def _torch_alloc(nbytes, stream, ctx):
    try:
        import torch
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
    except Exception:
        return None                       # NULL: the library reports TEM_ENOMEM


def _torch_free(ptr, nbytes, stream, ctx):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


_alloc_cb = _ALLOC_FN(_torch_alloc)       # kept alive for the life of the process
_free_cb = _FREE_FN(_torch_free)


def _install_torch_allocator(L):
    global _allocator
    if os.environ.get("TEM_ALLOCATOR", "torch") != "torch":
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except ImportError:
        return
    rc = L.tem_set_allocator(C.cast(_alloc_cb, C.c_void_p), C.cast(_free_cb, C.c_void_p), None)
    if rc == TEM_OK:
        _allocator = "torch"


def allocator():
    """Which allocator the library uses: "torch" (PyTorch's caching allocator) or "cuda" (its own
    cudaMallocAsync pool)."""
    lib()
    return _allocator


def status_string(code):
    return lib().tem_status_string(int(code)).decode()


def last_error():
    return lib().tem_last_error().decode()


def _check(rc, what, ok=(TEM_OK,)):
    if rc not in ok:
        raise TEMError(rc, what)
    return rc


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def default_options(**kw) -> Options:
    o = Options()
    lib().tem_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[v]
        if k == "precond" and isinstance(v, str):
            v = {"auto": PRECOND_AUTO, "jacobi": PRECOND_JACOBI, "nodal": PRECOND_NODAL}[v]
        setattr(o, k, v)
    return o


class Grid:
    """Device-resident grid and conductivity (tem_build_grid)."""

    def __init__(self, hx, hy, hz, origin, sigma, stream=None):
        self.hx, self.hy, self.hz = _f64(hx), _f64(hy), _f64(hz)
        self.origin = _f64(origin)
        sig = _f64(sigma).ravel()
        h = C.c_void_p()
        _check(lib().tem_build_grid(_ptr(self.hx), len(self.hx), _ptr(self.hy), len(self.hy), _ptr(self.hz),
                                    len(self.hz), _ptr(self.origin), _ptr(sig), _stream(stream), C.byref(h)),
               "tem_build_grid")
        self.handle = h

    @property
    def shape(self):
        return (len(self.hx), len(self.hy), len(self.hz))

    def set_sigma(self, sigma, stream=None):
        sig = _f64(sigma).ravel()
        _check(lib().tem_grid_set_sigma(self.handle, _ptr(sig), _stream(stream)), "tem_grid_set_sigma")

    def close(self):
        if getattr(self, "handle", None):
            lib().tem_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poles_residues(t, degree, weights=None):
    """tem_poles_residues: (shifts[s] complex, c[s, K] complex, uniform_err)."""
    t = _f64(t)
    K = len(t)
    xi = np.zeros(2 * degree)
    c = np.zeros(2 * degree * K)
    s = C.c_int64()
    err = C.c_double()
    w = _f64(weights) if weights is not None else None
    _check(lib().tem_poles_residues(_ptr(t), K, degree, _ptr(w) if w is not None else None, _ptr(xi), _ptr(c),
                                    C.byref(s), C.byref(err)), "tem_poles_residues")
    s = s.value
    shifts = xi[:2 * s].view(np.complex128).copy()
    cc = c[:2 * s * K].view(np.complex128).reshape(s, K).copy()
    return shifts, cc, err.value


class State:
    """Kept shifted solutions of a forward call (for the adjoint)."""

    def __init__(self, handle, s, n_rx, K, n_cells):
        self.handle, self.s, self.n_rx, self.K, self.n_cells = handle, s, n_rx, K, n_cells

    def stats(self):
        it = np.zeros(self.s, dtype=np.int32)
        rr = np.zeros(self.s)
        _check(lib().tem_state_stats(self.handle, it.ctypes.data_as(_i32p), _ptr(rr)), "tem_state_stats")
        return it, rr

    def solution(self, i, stream=None):
        """FP64 solution x_i of shift i, complex, in the library's edge layout (tem_state_solution)."""
        out = np.zeros(3 * self.n_cells, dtype=np.complex128)
        _check(lib().tem_state_solution(self.handle, int(i), _stream(stream), out.view(np.float64).ctypes.data_as(_dp)),
               "tem_state_solution")
        return out

    def adjoint(self, dphi_dd, stream=None):
        g = _f64(dphi_dd).reshape(self.n_rx, self.K)
        out = np.zeros(self.n_cells)
        rc = lib().tem_adjoint(self.handle, _ptr(g), _stream(stream), _ptr(out))
        _check(rc, "tem_adjoint", ok=(TEM_OK, TEM_ENOCONV))
        return out

    def fields(self, k0=0, nk=None, out=None, stream=None):
        """Field snapshots u_k = sum_i Re(c[i, k] x_i) for channels k0 .. k0+nk-1 (tem_state_fields),
        as a (nk, 3 * n_cells) float64 CUDA tensor in the library's edge layout."""
        import torch
        nk = self.K - k0 if nk is None else nk
        if out is None:
            out = torch.empty((nk, 3 * self.n_cells), dtype=torch.float64, device="cuda")
        if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous() or out.numel() < nk * 3 * self.n_cells:
            raise ValueError("fields: out must be a contiguous float64 CUDA tensor of nk * 3 * n_cells values")
        _check(lib().tem_state_fields(self.handle, int(k0), int(nk), _stream(stream), C.c_void_p(out.data_ptr())),
               "tem_state_fields")
        return out

    def jvp(self, dlogsigma, stream=None):
        """J dm (tem_jvp): the linearised response (n_rx, K) along a direction in log sigma."""
        dm = _f64(dlogsigma).ravel()
        if dm.size != self.n_cells:
            raise ValueError(f"jvp: {dm.size} values for {self.n_cells} cells")
        out = np.zeros((self.n_rx, self.K))
        rc = lib().tem_jvp(self.handle, _ptr(dm), _stream(stream), _ptr(out))
        _check(rc, "tem_jvp", ok=(TEM_OK, TEM_ENOCONV))
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().tem_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class ForwardResult:
    d: np.ndarray
    status: int
    state: State | None


def forward(grid: Grid, loop_xy, z_loop, rx, shifts, c, options: Options | None = None, current=1.0,
            stream=None, keep_state=False) -> ForwardResult:
    """tem_forward: d_t b_z (n_rx, K) for the given shifts and channel weights."""
    loop = _f64(loop_xy).reshape(-1, 2)
    rxa = _f64(rx).reshape(-1, 3)
    shifts = np.ascontiguousarray(shifts, dtype=np.complex128)
    cc = np.ascontiguousarray(c, dtype=np.complex128)
    s, K = cc.shape
    xi = shifts.view(np.float64)
    cf = cc.view(np.float64).ravel()
    opt = options or default_options()
    opt.keep_state = 1 if keep_state else 0
    out = np.zeros((len(rxa), K))
    h = C.c_void_p()
    rc = lib().tem_forward(grid.handle, _ptr(loop), len(loop), float(z_loop), float(current), _ptr(rxa), len(rxa),
                           _ptr(xi), _ptr(cf), s, K, C.byref(opt), _stream(stream), _ptr(out), C.byref(h))
    _check(rc, "tem_forward", ok=(TEM_OK, TEM_ENOCONV))
    st = State(h, s, len(rxa), K, int(np.prod(grid.shape))) if (keep_state and h.value) else None
    return ForwardResult(out, rc, st)


def forward_sources(grid: Grid, loops, z_loops, rx, shifts, c, options: Options | None = None, currents=None,
                    stream=None):
    """tem_forward_sources: d_t b_z (n_src, n_rx, K) for several loops solved as one batch.
    loops: sequence of (n_j, 2) vertex arrays; z_loops, currents: one value per loop."""
    loops = [_f64(l).reshape(-1, 2) for l in loops]
    n_src = len(loops)
    verts = np.ascontiguousarray(np.concatenate(loops), dtype=np.float64)
    off = np.ascontiguousarray(np.concatenate(([0], np.cumsum([len(l) for l in loops]))), dtype=np.int64)
    zl = _f64(np.broadcast_to(np.asarray(z_loops, dtype=np.float64), (n_src,)))
    cur = _f64(np.ones(n_src) if currents is None else np.broadcast_to(np.asarray(currents, np.float64), (n_src,)))
    rxa = _f64(rx).reshape(-1, 3)
    shifts = np.ascontiguousarray(shifts, dtype=np.complex128)
    cc = np.ascontiguousarray(c, dtype=np.complex128)
    s, K = cc.shape
    opt = options or default_options()
    out = np.zeros((n_src, len(rxa), K))
    rc = lib().tem_forward_sources(grid.handle, _ptr(verts), off.ctypes.data_as(_i64p), n_src, _ptr(zl), _ptr(cur),
                                   _ptr(rxa), len(rxa), _ptr(shifts.view(np.float64)), _ptr(cc.view(np.float64).ravel()),
                                   s, K, C.byref(opt), _stream(stream), _ptr(out))
    _check(rc, "tem_forward_sources", ok=(TEM_OK, TEM_ENOCONV))
    return out


def forward_single_time(grid: Grid, loop_xy, z_loop, rx, t, shifts, c, options: Options | None = None, current=1.0,
                        stream=None):
    """tem_forward_single_time: the single-time baseline of Sec. 3.1.  shifts, c: the fit of
    exp(-x) for t = 1 (poles_residues([1.0], m)); t: the K channel times.  Returns (d (n_rx, K),
    number of shifted solves)."""
    loop = _f64(loop_xy).reshape(-1, 2)
    rxa = _f64(rx).reshape(-1, 3)
    tt = _f64(t)
    shifts = np.ascontiguousarray(shifts, dtype=np.complex128)
    cc = np.ascontiguousarray(np.asarray(c).reshape(len(shifts)), dtype=np.complex128)
    opt = options or default_options()
    out = np.zeros((len(rxa), len(tt)))
    solves = C.c_int64()
    rc = lib().tem_forward_single_time(grid.handle, _ptr(loop), len(loop), float(z_loop), float(current), _ptr(rxa),
                                       len(rxa), _ptr(tt), len(tt), _ptr(shifts.view(np.float64)),
                                       _ptr(cc.view(np.float64)), len(shifts), C.byref(opt), _stream(stream), _ptr(out),
                                       C.byref(solves))
    _check(rc, "tem_forward_single_time", ok=(TEM_OK, TEM_ENOCONV))
    return out, int(solves.value)


def apply_operator(grid: Grid, shifts, p, q, precision=PREC_FP64, stream=None):
    """q[i] = (K - xi_i M) p[i] on device tensors in the library's edge layout (see tem.h)."""
    shifts = np.ascontiguousarray(shifts, dtype=np.complex128)
    xi = shifts.view(np.float64)
    _check(lib().tem_apply_operator(grid.handle, _ptr(xi), len(shifts), C.c_void_p(p.data_ptr()),
                                    C.c_void_p(q.data_ptr()), int(precision), _stream(stream)),
           "tem_apply_operator")


def apply_operator_noalloc(grid: Grid, shifts, p, q, precision=PREC_FP64, stream=None):
    """tem_apply_operator_noalloc: same result as apply_operator, no device allocation
    (at most 64 shifts; the shifts live in one array shared by all calls)."""
    shifts = np.ascontiguousarray(shifts, dtype=np.complex128)
    xi = shifts.view(np.float64)
    _check(lib().tem_apply_operator_noalloc(grid.handle, _ptr(xi), len(shifts), C.c_void_p(p.data_ptr()),
                                            C.c_void_p(q.data_ptr()), int(precision), _stream(stream)),
           "tem_apply_operator_noalloc")


def launch_count() -> int:
    """Kernels launched by libtem.so in this process so far."""
    return int(lib().tem_launch_count())


def profile_passes(grid: Grid, loop_xy, z_loop, shifts, precision=PREC_MIXED, n_iter=20, current=1.0, stream=None,
                   precond=PRECOND_AUTO):
    """Average CUDA-event time (ms) of the stencil, update and FP64 residual passes, the CTAs
    per SM the FP32 stencil keeps resident, and the interior edges x shifts one launch
    processes (tem_profile_passes)."""
    loop = _f64(loop_xy).reshape(-1, 2)
    shifts = np.ascontiguousarray(shifts, dtype=np.complex128)
    xi = shifts.view(np.float64)
    ms = np.zeros(4)
    units = np.zeros(1)
    _check(lib().tem_profile_passes(grid.handle, _ptr(loop), len(loop), float(z_loop), float(current), _ptr(xi),
                                    len(shifts), int(precision), int(precond), int(n_iter), _stream(stream), _ptr(ms),
                                    _ptr(units)),
           "tem_profile_passes")
    return {"stencil_ms": ms[0], "update_ms": ms[1], "residual_ms": ms[2],
            "stencil_ctas_per_sm": int(ms[3]), "units": units[0]}


class Server:
    """Continuous-batching server of forward models (tem_server_*)."""

    def __init__(self, hbm_budget_bytes=None, max_slots=None, iters_per_step=None, stream=None, **solver):
        o = ServerOptions()
        lib().tem_server_default_options(C.byref(o))
        if hbm_budget_bytes is not None:
            o.hbm_budget_bytes = int(hbm_budget_bytes)
        if max_slots is not None:
            o.max_slots = int(max_slots)
        if iters_per_step is not None:
            o.iters_per_step = int(iters_per_step)
        base = default_options(**solver) if solver else None
        if base is not None:
            o.solver = base
        if "precision" not in solver:
            o.solver.precision = PREC_MIXED
        h = C.c_void_p()
        _check(lib().tem_server_create(C.byref(o), _stream(stream), C.byref(h)), "tem_server_create")
        self.handle = h
        self.shapes = {}

    def submit(self, model, shifts, c):
        """Queue a workloads.Model with its shifts/weights; returns the ticket."""
        hx, hy, hz = _f64(model.hx), _f64(model.hy), _f64(model.hz)
        org, sig = _f64(model.origin), _f64(model.sigma).ravel()
        loop, rx = _f64(model.loop_xy).reshape(-1, 2), _f64(model.rx).reshape(-1, 3)
        sh = np.ascontiguousarray(shifts, dtype=np.complex128)
        cc = np.ascontiguousarray(c, dtype=np.complex128)
        s, K = cc.shape
        t = C.c_int64()
        _check(lib().tem_server_submit(self.handle, _ptr(hx), len(hx), _ptr(hy), len(hy), _ptr(hz), len(hz), _ptr(org),
                                       _ptr(sig), _ptr(loop), len(loop), float(model.z_loop), float(model.current),
                                       _ptr(rx), len(rx), _ptr(sh.view(np.float64)), _ptr(cc.view(np.float64).ravel()),
                                       s, K, C.byref(t)), "tem_server_submit")
        self.shapes[t.value] = (len(rx), K)
        return t.value

    def step(self):
        _check(lib().tem_server_step(self.handle), "tem_server_step")

    def poll(self, ticket):
        """None while queued/running; else (d, stats dict)."""
        n_rx, K = self.shapes[ticket]
        out = np.zeros((n_rx, K))
        st = RequestStats()
        rc = lib().tem_server_poll(self.handle, int(ticket), _ptr(out), C.byref(st))
        if rc == TEM_EBUSY:
            return None
        del self.shapes[ticket]
        stats = {k: getattr(st, k) for k, _ in RequestStats._fields_}
        return out, stats

    def counts(self):
        q, r, d = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().tem_server_counts(self.handle, C.byref(q), C.byref(r), C.byref(d)), "tem_server_counts")
        return q.value, r.value, d.value

    def close(self):
        if getattr(self, "handle", None):
            lib().tem_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
