"""ctypes binding of libchanfs (include/chanfs.h): argument marshalling only.

Every step of every solve runs in the library's CUDA kernels.  Fields are
torch float64 tensors of shape (Nz, Ny, Nx) (x fastest), contiguous, on the
plan's CUDA device; work is queued on torch's current stream unless a stream
is given.  If the library has not been built this module raises: there is no
CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchanfs.so")

NEUMANN, DIRICHLET = 0, 1
CENTER, FACE = 0, 1
F64, F32_REFINED = 0, 1

X_FORWARD, Y_FORWARD, Z_SOLVE, Y_INVERSE, X_INVERSE = 0, 1, 2, 3, 4

OPT_THOMAS_TILE, OPT_X_LINES, OPT_Y_TILE, OPT_PCR_PARTS, OPT_HELM_FP64 = 1, 2, 3, 4, 5
OPT_HELM_THOMAS, OPT_HELM_THOMAS32, OPT_FFT_RADIX = 6, 7, 8
OPT_F64_ADDS_X, OPT_F64_ADDS_Y, OPT_STREAM_CHUNKS = 9, 10, 11

REQ_POISSON, REQ_HELMHOLTZ = 0, 1

Y_PERIODIC, Y_NEUMANN, Y_DIRICHLET = 0, 1, 2


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("completed", ctypes.c_ulonglong),
                ("failed", ctypes.c_ulonglong), ("batches", ctypes.c_ulonglong),
                ("max_batch_seen", ctypes.c_int), ("plans_created", ctypes.c_int),
                ("plans_evicted", ctypes.c_int), ("plans_resident", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("cancelled", ctypes.c_ulonglong),
                ("workers_alive", ctypes.c_int), ("pending", ctypes.c_int)]

OK, EINVAL, ENOMEM, EUNSUPPORTED, ECUDA, ETIMEOUT, ENOTCONVERGED, ECANCELED = 0, -1, -2, -3, -4, -5, -6, -7
EGUARD = -8
FAULT_PLAN_ALLOC, FAULT_WORKER_START = 1, 2

_lib = None


class ChanfsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def lib():
    """Load libchanfs.so (built by __graft_entry__.build() / build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; "
                               f"g.build()'` first (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
        sig = {
            "cfs_version": ([], i),
            "cfs_status_string": ([i], ctypes.c_char_p),
            "cfs_plan_create": ([ctypes.POINTER(vp), i, i, i, d, d, dp, i, i], i),
            "cfs_plan_create_walls": ([ctypes.POINTER(vp), i, i, i, d, d, dp, i, i, i], i),
            "cfs_plan_destroy": ([vp], i),
            "cfs_plan_device_bytes": ([vp, ctypes.POINTER(ctypes.c_size_t)], i),
            "cfs_poisson_solve": ([vp, vp, vp, vp], i),
            "cfs_helmholtz_prepare": ([vp, d, i, i], i),
            "cfs_helmholtz_solve": ([vp, d, i, vp, vp, vp], i),
            "cfs_spectral_forward": ([vp, vp, vp, vp], i),
            "cfs_spectral_inverse": ([vp, vp, vp, vp], i),
            "cfs_poisson_solve_host": ([vp, vp, vp, vp], i),
            "cfs_helmholtz_solve_host": ([vp, d, i, vp, vp, vp], i),
            "cfs_plan_check": ([vp, ctypes.POINTER(i)], i),
            "cfs_plan_check_guards": ([vp, ctypes.POINTER(i)], i),
            "cfs_plan_debug_guard_poke": ([vp, i, i], i),
            "cfs_poisson_stage": ([vp, i, vp, vp, vp], i),
            "cfs_plan_set_refinement": ([vp, d, i], i),
            "cfs_helmholtz_solve_noalloc": ([i, i, i, dp, d, i, i, vp, vp, vp, vp], i),
            "cfs_last_info": ([vp, ctypes.POINTER(i), ctypes.POINTER(d)], i),
            "cfs_probe_fma": ([i, ctypes.c_longlong, dp, dp], i),
            "cfs_selftest_wait_timeout": ([vp, vp, ctypes.c_uint, vp], i),
            "cfs_slab_partition": ([i, i, i, ctypes.POINTER(i), ctypes.POINTER(i)], i),
            "cfs_slab_create": ([ctypes.POINTER(vp), i, i, i, d, d, dp, i, i, i], i),
            "cfs_slab_destroy": ([vp], i),
            "cfs_slab_extent": ([vp, ctypes.POINTER(i), ctypes.POINTER(i)], i),
            "cfs_slab_boundary_doubles": ([vp, i, ctypes.POINTER(ctypes.c_size_t)], i),
            "cfs_slab_poisson_reduce": ([vp, vp, vp, vp, vp], i),
            "cfs_slab_poisson_finish": ([vp, vp, vp, vp, vp], i),
            "cfs_slab_helmholtz_reduce": ([vp, d, i, vp, vp, vp, vp], i),
            "cfs_slab_helmholtz_finish": ([vp, d, i, vp, vp, vp, vp], i),
            "cfs_group_create": ([ctypes.POINTER(vp), i, ctypes.POINTER(vp)], i),
            "cfs_group_destroy": ([vp], i),
            "cfs_group_size": ([vp, ctypes.POINTER(i)], i),
            "cfs_group_poisson_solve": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp], i),
            "cfs_group_last_info": ([vp, ctypes.POINTER(i), ctypes.POINTER(d)], i),
            "cfs_group_set_graphs": ([vp, i], i),
            "cfs_group_set_trace": ([vp, i], i),
            "cfs_group_trace": ([vp, ctypes.POINTER(ctypes.c_float), i, ctypes.POINTER(i)], i),
            "cfs_solve_batch_host": ([vp, i, ctypes.POINTER(i), ctypes.POINTER(d),
                                      ctypes.POINTER(i), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      vp], i),
            "cfs_autotune_save": ([ctypes.c_char_p], i),
            "cfs_autotune_load": ([ctypes.c_char_p, ctypes.POINTER(i)], i),
            "cfs_autotune_clear": ([], i),
            "cfs_group_helmholtz_solve": ([vp, dp, ctypes.POINTER(i), ctypes.POINTER(vp),
                                           ctypes.POINTER(vp), vp], i),
            "cfs_helmholtz3d_prepare": ([vp, d, i], i),
            "cfs_helmholtz3d_solve": ([vp, d, i, vp, vp, vp], i),
            "cfs_plan_set_option": ([vp, i, i], i),
            "cfs_selfcheck_conversions": ([ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ulonglong)], i),
            "cfs_selfcheck_f64_addsub": ([ctypes.c_ulonglong, i,
                                          ctypes.POINTER(ctypes.c_ulonglong)], i),
            "cfs_probe_addsub": ([i, ctypes.c_longlong, dp, dp], i),
            "cfs_f64_addsub_host": ([ctypes.c_longlong, dp, dp, dp, dp], i),
            "cfs_group_reserve": ([ctypes.POINTER(vp), i], i),
            "cfs_group_rebind": ([vp, i, ctypes.POINTER(vp), vp], i),
            "cfs_server_create": ([ctypes.POINTER(vp), ctypes.c_size_t, i, i, i, i], i),
            "cfs_server_cancel": ([vp, ctypes.c_ulonglong], i),
            "cfs_server_pause": ([vp, i], i),
            "cfs_server_inject_fault": ([vp, i, i], i),
            "cfs_server_add_run": ([vp, i, i, i, d, d, dp, i, ctypes.POINTER(i)], i),
            "cfs_server_submit": ([vp, i, i, d, i, vp, vp, ctypes.POINTER(ctypes.c_ulonglong)], i),
            "cfs_server_wait": ([vp, ctypes.c_ulonglong, d, ctypes.POINTER(i), ctypes.POINTER(d)], i),
            "cfs_server_stats": ([vp, ctypes.POINTER(ServerStats)], i),
            "cfs_server_destroy": ([vp], i),
            "cfs_plan_autotune": ([vp, vp], i),
            "cfs_plan_get_option": ([vp, i, ctypes.POINTER(i)], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    """Names of the C-ABI entry points declared in include/chanfs.h."""
    hdr = os.path.join(os.path.dirname(HERE), "include", "chanfs.h")
    import re
    return sorted(set(re.findall(r"^\w[\w\s\*]*?\b(cfs_\w+)\s*\(", open(hdr).read(), re.M)))


def status_string(status: int) -> str:
    return lib().cfs_status_string(status).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise ChanfsError(rc, what)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """One grid: Nx x Ny x Nz cells, periodic x of length lx, y of length ly
    (periodic, or walls: ybc), and the z cell widths dz (host array).  See
    cfs_plan_create / cfs_plan_create_walls."""

    def __init__(self, nx: int, ny: int, nz: int, lx: float, ly: float, dz, bc: int = NEUMANN,
                 dtype: int = F64, ybc: int = Y_PERIODIC):
        self.dtype = dtype
        dz = np.ascontiguousarray(dz, dtype=np.float64)
        if dz.size != nz:
            raise ValueError("dz must have nz entries")
        self.nx, self.ny, self.nz, self.lx, self.ly, self.bc = nx, ny, nz, lx, ly, bc
        self.ybc = ybc
        self.dz = dz.copy()
        h = ctypes.c_void_p()
        rc = lib().cfs_plan_create_walls(ctypes.byref(h), nx, ny, nz, lx, ly,
                                         dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), bc,
                                         ybc, dtype)
        _check(rc, "cfs_plan_create_walls")
        self._h = h

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def close(self):
        if getattr(self, "_h", None):
            lib().cfs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _field(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise TypeError(f"{name} must be a float64 CUDA tensor")
        if tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {self.shape}")
        return ctypes.c_void_p(t.data_ptr())

    def _out(self, like, out):
        import torch
        return torch.empty_like(like) if out is None else out

    def device_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().cfs_plan_device_bytes(self._h, ctypes.byref(n)), "cfs_plan_device_bytes")
        return n.value

    def poisson_solve(self, f, out=None, stream=None):
        out = self._out(f, out)
        _check(lib().cfs_poisson_solve(self._h, self._field(f, "f"), self._field(out, "out"),
                                       _stream_ptr(stream)), "cfs_poisson_solve")
        return out

    def helmholtz_prepare(self, c: float, loc: int = CENTER, nparts: int = 0):
        _check(lib().cfs_helmholtz_prepare(self._h, float(c), loc, nparts), "cfs_helmholtz_prepare")

    def helmholtz_solve(self, c: float, rhs, loc: int = CENTER, out=None, stream=None):
        out = self._out(rhs, out)
        _check(lib().cfs_helmholtz_solve(self._h, float(c), loc, self._field(rhs, "rhs"),
                                         self._field(out, "out"), _stream_ptr(stream)),
               "cfs_helmholtz_solve")
        return out

    def helmholtz3d_prepare(self, c: float, loc: int = CENTER):
        _check(lib().cfs_helmholtz3d_prepare(self._h, float(c), loc), "cfs_helmholtz3d_prepare")

    def helmholtz3d_solve(self, c: float, rhs, loc: int = CENTER, out=None, stream=None):
        """(I - c L) u = rhs, the fully implicit Helmholtz solve (Eq. 8)."""
        out = self._out(rhs, out)
        _check(lib().cfs_helmholtz3d_solve(self._h, float(c), loc, self._field(rhs, "rhs"),
                                           self._field(out, "out"), _stream_ptr(stream)),
               "cfs_helmholtz3d_solve")
        return out

    def spectral_forward(self, f, out=None, stream=None):
        out = self._out(f, out)
        _check(lib().cfs_spectral_forward(self._h, self._field(f, "f"), self._field(out, "out"),
                                          _stream_ptr(stream)), "cfs_spectral_forward")
        return out

    def spectral_inverse(self, s, out=None, stream=None):
        out = self._out(s, out)
        _check(lib().cfs_spectral_inverse(self._h, self._field(s, "s"), self._field(out, "out"),
                                          _stream_ptr(stream)), "cfs_spectral_inverse")
        return out

    def poisson_stage(self, stage: int, x, out=None, stream=None):
        """Run one kernel of the Poisson solve (see cfs_poisson_stage)."""
        out = self._out(x, out)
        _check(lib().cfs_poisson_stage(self._h, stage, self._field(x, "in"), self._field(out, "out"),
                                       _stream_ptr(stream)), "cfs_poisson_stage")
        return out

    def poisson_solve_host(self, f, out, stream=None):
        """f, out: host buffers (numpy arrays or pinned CPU tensors) of the field shape."""
        _check(lib().cfs_poisson_solve_host(self._h, _host_ptr(f, self.shape), _host_ptr(out, self.shape),
                                            _stream_ptr(stream)), "cfs_poisson_solve_host")
        return out

    def helmholtz_solve_host(self, c: float, rhs, out, loc: int = CENTER, stream=None):
        _check(lib().cfs_helmholtz_solve_host(self._h, float(c), loc, _host_ptr(rhs, self.shape),
                                              _host_ptr(out, self.shape), _stream_ptr(stream)),
               "cfs_helmholtz_solve_host")
        return out

    def solve_batch_host(self, jobs, stream=None):
        """jobs: a list of (kind, c, loc, input, output) with pinned (or any)
        host arrays / CPU tensors of the plan's shape; solved in order with
        the copies overlapped (cfs_solve_batch_host)."""
        n = len(jobs)
        kinds = (ctypes.c_int * n)(*[int(j[0]) for j in jobs])
        cs = (ctypes.c_double * n)(*[float(j[1]) for j in jobs])
        locs = (ctypes.c_int * n)(*[int(j[2]) for j in jobs])
        ins = (ctypes.c_void_p * n)(*[_host_ptr(j[3], self.shape).value for j in jobs])
        outs = (ctypes.c_void_p * n)(*[_host_ptr(j[4], self.shape).value for j in jobs])
        _check(lib().cfs_solve_batch_host(self._h, n, kinds, cs, locs, ins, outs,
                                          _stream_ptr(stream)), "cfs_solve_batch_host")

    def set_refinement(self, tol: float = 1e-10, maxit: int = 4):
        """Refined plans: stop at ||r||_inf <= tol ||b||_inf or after maxit FP32 solves."""
        _check(lib().cfs_plan_set_refinement(self._h, float(tol), int(maxit)), "cfs_plan_set_refinement")

    def set_option(self, option: int, value: int):
        """Choose a kernel shape (see cfs_plan_set_option)."""
        _check(lib().cfs_plan_set_option(self._h, int(option), int(value)), "cfs_plan_set_option")

    def autotune(self, stream=None):
        """Time the kernel-shape candidates on the GPU and keep the fastest
        (cfs_plan_autotune); returns the options now in effect."""
        _check(lib().cfs_plan_autotune(self._h, _stream_ptr(stream)), "cfs_plan_autotune")
        return {name: self.get_option(opt) for name, opt in
                (("x_lines", OPT_X_LINES), ("y_tile", OPT_Y_TILE),
                 ("thomas_tile", OPT_THOMAS_TILE), ("pcr_parts", OPT_PCR_PARTS),
                 ("helm_fp64", OPT_HELM_FP64), ("helm_thomas", OPT_HELM_THOMAS),
                 ("helm_thomas32", OPT_HELM_THOMAS32), ("fft_radix", OPT_FFT_RADIX),
                 ("f64_adds_x", OPT_F64_ADDS_X), ("f64_adds_y", OPT_F64_ADDS_Y))}

    def get_option(self, option: int) -> int:
        """The kernel shape in effect, automatic choices resolved."""
        v = ctypes.c_int(0)
        _check(lib().cfs_plan_get_option(self._h, int(option), ctypes.byref(v)), "cfs_plan_get_option")
        return v.value

    def last_info(self):
        """(FP32 solves, final relative residual) of the last refined solve."""
        it, rho = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(lib().cfs_last_info(self._h, ctypes.byref(it), ctypes.byref(rho)), "cfs_last_info")
        return it.value, rho.value

    def check(self) -> int:
        """Synchronise and return the device failure bits (raises on failure)."""
        bits = ctypes.c_int(0)
        rc = lib().cfs_plan_check(self._h, ctypes.byref(bits))
        _check(rc, "cfs_plan_check")
        return bits.value

    def check_guards(self) -> int:
        """Synchronise and compare the guard words around the plan's work
        buffers (cfs_plan_check_guards); raises ChanfsError(EGUARD) if any
        was overwritten, else returns 0."""
        n = ctypes.c_int(0)
        _check(lib().cfs_plan_check_guards(self._h, ctypes.byref(n)), "cfs_plan_check_guards")
        return n.value

    def debug_guard_poke(self, buffer: int, tail: bool):
        """Overwrite one byte of a work buffer's guard (tests of the check)."""
        _check(lib().cfs_plan_debug_guard_poke(self._h, int(buffer), int(bool(tail))),
               "cfs_plan_debug_guard_poke")


def helmholtz_solve_noalloc(dz, c: float, rhs, loc: int = CENTER, nparts: int = 0, out=None,
                            status=None, stream=None):
    """cfs_helmholtz_solve_noalloc: the Helmholtz solve without a plan and
    without device allocation by the library (see include/chanfs.h).
    `status` is a CUDA int32 tensor of at least one element that receives the
    solve's failure bits (allocated here if not given); returns (u, status).
    Read status after the stream has finished: nonzero means u is invalid."""
    import torch
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    nz, ny, nx = rhs.shape
    if dz.size != nz:
        raise ValueError("dz must have nz entries")
    out = torch.empty_like(rhs) if out is None else out
    for t, name in ((rhs, "rhs"), (out, "out")):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.shape != rhs.shape:
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor of the rhs shape")
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=rhs.device)
    if status.dtype != torch.int32 or not status.is_cuda or status.numel() < 1:
        raise TypeError("status must be a CUDA int32 tensor")
    _check(lib().cfs_helmholtz_solve_noalloc(nx, ny, nz, dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             float(c), loc, nparts, ctypes.c_void_p(rhs.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(status.data_ptr()), _stream_ptr(stream)),
           "cfs_helmholtz_solve_noalloc")
    return out, status


def slab_partition(nz: int, nranks: int, rank: int):
    """Planes [z0, z1) of `rank` among `nranks` z-slabs (host arithmetic)."""
    z0, z1 = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().cfs_slab_partition(nz, nranks, rank, ctypes.byref(z0), ctypes.byref(z1)),
           "cfs_slab_partition")
    return z0.value, z1.value


class Slab:
    """One rank's z-slab of a grid distributed over several GPUs (see
    cfs_slab_create): the rank's planes of the Poisson and Helmholtz solves,
    reduce and finish around an exchange of boundary values."""

    def __init__(self, nx: int, ny: int, nz: int, lx: float, ly: float, dz, bc: int = NEUMANN,
                 nranks: int = 1, rank: int = 0):
        dz = np.ascontiguousarray(dz, dtype=np.float64)
        if dz.size != nz:
            raise ValueError("dz must have nz entries (the whole grid)")
        h = ctypes.c_void_p()
        _check(lib().cfs_slab_create(ctypes.byref(h), nx, ny, nz, float(lx), float(ly),
                                     dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), bc,
                                     nranks, rank), "cfs_slab_create")
        self._h = h
        z0, z1 = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().cfs_slab_extent(self._h, ctypes.byref(z0), ctypes.byref(z1)), "cfs_slab_extent")
        self.z0, self.z1 = z0.value, z1.value
        self.shape = (self.z1 - self.z0, ny, nx)

    def close(self):
        if getattr(self, "_h", None):
            lib().cfs_slab_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def boundary_doubles(self, kind: int) -> int:
        n = ctypes.c_size_t(0)
        _check(lib().cfs_slab_boundary_doubles(self._h, kind, ctypes.byref(n)),
               "cfs_slab_boundary_doubles")
        return n.value

    def _field(self, t, name):
        if t.dtype != _torch().float64 or not t.is_cuda or not t.is_contiguous() or \
                tuple(t.shape) != self.shape:
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor of shape {self.shape}")
        return ctypes.c_void_p(t.data_ptr())

    def poisson_reduce(self, f, work, bnd, stream=None):
        _check(lib().cfs_slab_poisson_reduce(self._h, self._field(f, "f"), self._field(work, "work"),
                                             ctypes.c_void_p(bnd.data_ptr()), _stream_ptr(stream)),
               "cfs_slab_poisson_reduce")

    def poisson_finish(self, bnd_all, work, out, stream=None):
        _check(lib().cfs_slab_poisson_finish(self._h, ctypes.c_void_p(bnd_all.data_ptr()),
                                             self._field(work, "work"), self._field(out, "out"),
                                             _stream_ptr(stream)), "cfs_slab_poisson_finish")

    def helmholtz_reduce(self, c: float, loc: int, rhs, work, bnd, stream=None):
        _check(lib().cfs_slab_helmholtz_reduce(self._h, float(c), loc, self._field(rhs, "rhs"),
                                               self._field(work, "work"),
                                               ctypes.c_void_p(bnd.data_ptr()), _stream_ptr(stream)),
               "cfs_slab_helmholtz_reduce")

    def helmholtz_finish(self, c: float, loc: int, bnd_all, work, out, stream=None):
        _check(lib().cfs_slab_helmholtz_finish(self._h, float(c), loc,
                                               ctypes.c_void_p(bnd_all.data_ptr()),
                                               self._field(work, "work"), self._field(out, "out"),
                                               _stream_ptr(stream)), "cfs_slab_helmholtz_finish")


def _torch():
    import torch
    return torch


class Group:
    """Several CFS_F32_REFINED plans solved together, one launch per stage for
    all boxes (see cfs_group_create).  The plans must outlive the group."""

    def __init__(self, plans, capacity=None):
        """capacity (default: len(plans)): the most plans a later rebind()
        may take."""
        self.plans = list(plans)
        n = len(self.plans)
        h = ctypes.c_void_p()
        if capacity is None:
            arr = (ctypes.c_void_p * n)(*[p._h for p in self.plans])
            _check(lib().cfs_group_create(ctypes.byref(h), n, arr), "cfs_group_create")
            self._h = h
        else:
            _check(lib().cfs_group_reserve(ctypes.byref(h), int(capacity)), "cfs_group_reserve")
            self._h = h
            self.rebind(self.plans)

    def rebind(self, plans, stream=None):
        """Binds the group to other plans (at most its capacity)."""
        plans = list(plans)
        n = len(plans)
        arr = (ctypes.c_void_p * n)(*[p._h for p in plans])
        _check(lib().cfs_group_rebind(self._h, n, arr, _stream_ptr(stream)), "cfs_group_rebind")
        self.plans = plans

    def close(self):
        if getattr(self, "_h", None):
            lib().cfs_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def poisson_solve(self, fs, outs=None, stream=None):
        """fs: one float64 CUDA tensor per plan; returns the solutions."""
        import torch
        if len(fs) != len(self.plans):
            raise ValueError("one right-hand side per plan")
        outs = [torch.empty_like(f) for f in fs] if outs is None else list(outs)
        n = len(self.plans)
        fp = (ctypes.c_void_p * n)(*[p._field(f, "f").value for p, f in zip(self.plans, fs)])
        pp = (ctypes.c_void_p * n)(*[p._field(o, "out").value for p, o in zip(self.plans, outs)])
        _check(lib().cfs_group_poisson_solve(self._h, fp, pp, _stream_ptr(stream)),
               "cfs_group_poisson_solve")
        return outs

    def helmholtz_solve(self, cs, rhss, locs=None, outs=None, stream=None):
        """(I - c L_z) u = rhs per box: cs, locs per plan; returns the solutions."""
        import torch
        n = len(self.plans)
        if len(cs) != n or len(rhss) != n:
            raise ValueError("one coefficient and one right-hand side per plan")
        locs = [CENTER] * n if locs is None else list(locs)
        outs = [torch.empty_like(r) for r in rhss] if outs is None else list(outs)
        ca = (ctypes.c_double * n)(*[float(c) for c in cs])
        la = (ctypes.c_int * n)(*[int(x) for x in locs])
        fp = (ctypes.c_void_p * n)(*[p._field(r, "rhs").value for p, r in zip(self.plans, rhss)])
        pp = (ctypes.c_void_p * n)(*[p._field(o, "out").value for p, o in zip(self.plans, outs)])
        _check(lib().cfs_group_helmholtz_solve(self._h, ca, la, fp, pp, _stream_ptr(stream)),
               "cfs_group_helmholtz_solve")
        return outs

    def set_graphs(self, on):
        """Graph-launched solves with the refinement loop on the device (the
        default), or direct launches with the loop on the host (on=False)."""
        _check(lib().cfs_group_set_graphs(self._h, int(bool(on))), "cfs_group_set_graphs")

    def set_trace(self, on):
        """Direct launches with an event pair around each copy and kernel
        (cfs_group_set_trace); trace() then gives their device times."""
        _check(lib().cfs_group_set_trace(self._h, int(bool(on))), "cfs_group_set_trace")

    def trace(self, capacity: int = 512):
        """Device time (ms) of each copy and kernel of the last traced solve."""
        buf = (ctypes.c_float * capacity)()
        n = ctypes.c_int(0)
        _check(lib().cfs_group_trace(self._h, buf, capacity, ctypes.byref(n)), "cfs_group_trace")
        return [float(buf[k]) for k in range(min(n.value, capacity))]

    def last_info(self):
        """Per plan: (FP32 solves, final relative residual) of the last solve."""
        n = len(self.plans)
        it = (ctypes.c_int * n)()
        rho = (ctypes.c_double * n)()
        _check(lib().cfs_group_last_info(self._h, it, rho), "cfs_group_last_info")
        return list(zip(list(it), list(rho)))


class Server:
    """Serving loop for solve requests of many runs (see cfs_server_create):
    plans resident under an HBM budget, continuous batching by worker threads
    with one CUDA stream each, FP32 + FP64-refined grouped solves."""

    def __init__(self, budget_bytes: int, workers: int = 2, max_batch: int = 16,
                 autotune: bool = True, slots_per_run: int = 1):
        h = ctypes.c_void_p()
        _check(lib().cfs_server_create(ctypes.byref(h), int(budget_bytes), int(workers),
                                       int(max_batch), int(slots_per_run), int(bool(autotune))),
               "cfs_server_create")
        self._h = h
        self._shapes = []
        self._held = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().cfs_server_destroy(self._h)
            self._h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_run(self, nx: int, ny: int, nz: int, lx: float, ly: float, dz, bc: int = NEUMANN) -> int:
        dz = np.ascontiguousarray(dz, dtype=np.float64)
        if dz.size != nz:
            raise ValueError("dz must have nz entries")
        run = ctypes.c_int(-1)
        _check(lib().cfs_server_add_run(self._h, nx, ny, nz, float(lx), float(ly),
                                        dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), bc,
                                        ctypes.byref(run)), "cfs_server_add_run")
        self._shapes.append((nz, ny, nx))
        return run.value

    def submit(self, run: int, kind: int, rhs, out, c: float = 0.0, loc: int = CENTER) -> int:
        """Queue a solve; rhs and out (float64 CUDA tensors of the run's shape)
        are held until the ticket is waited for."""
        import torch
        shape = self._shapes[run] if 0 <= run < len(self._shapes) else None
        for t, name in ((rhs, "rhs"), (out, "out")):
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda \
                    or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of the run's shape")
        ticket = ctypes.c_ulonglong(0)
        _check(lib().cfs_server_submit(self._h, run, kind, float(c), loc, ctypes.c_void_p(rhs.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.byref(ticket)),
               "cfs_server_submit")
        self._held[ticket.value] = (rhs, out)
        return ticket.value

    def wait(self, ticket: int, timeout: float = -1.0):
        """(solve status, latency in seconds) of a ticket; raises on timeout."""
        status, lat = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(lib().cfs_server_wait(self._h, ticket, float(timeout), ctypes.byref(status),
                                     ctypes.byref(lat)), "cfs_server_wait")
        self._held.pop(ticket, None)
        return status.value, lat.value

    def cancel(self, ticket: int) -> None:
        """Take a request no worker has started off the queue (it completes
        with ECANCELED); raises if it is unknown, running or done."""
        _check(lib().cfs_server_cancel(self._h, ticket), "cfs_server_cancel")

    def pause(self, paused: bool = True) -> None:
        _check(lib().cfs_server_pause(self._h, int(bool(paused))), "cfs_server_pause")

    def inject_fault(self, fault: int, count: int) -> None:
        """Host-side fault injection (FAULT_PLAN_ALLOC) for tests."""
        _check(lib().cfs_server_inject_fault(self._h, int(fault), int(count)),
               "cfs_server_inject_fault")

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().cfs_server_stats(self._h, ctypes.byref(st)), "cfs_server_stats")
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}


def autotune_save(path) -> None:
    """Write the tuner's choices of this process to a text file."""
    _check(lib().cfs_autotune_save(str(path).encode()), "cfs_autotune_save")


def autotune_load(path) -> int:
    """Take the choices of a file written by autotune_save on this kind of
    GPU; returns how many were taken."""
    n = ctypes.c_int(0)
    _check(lib().cfs_autotune_load(str(path).encode(), ctypes.byref(n)), "cfs_autotune_load")
    return n.value


def autotune_clear() -> None:
    """Forget every tuning choice of this process."""
    _check(lib().cfs_autotune_clear(), "cfs_autotune_clear")


def probe_fma(bits: int = 64, iters: int = 1 << 15):
    """(FMAs per second, launch ms) of the current GPU in FP64 or FP32
    (cfs_probe_fma)."""
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().cfs_probe_fma(int(bits), int(iters), ctypes.byref(rate), ctypes.byref(ms)),
           "cfs_probe_fma")
    return rate.value, ms.value


def selfcheck_conversions(samples: int = 1 << 22) -> int:
    """Bit mismatches of the library's FP32 <-> FP64 conversions against the
    hardware's over `samples` hashed operands (cfs_selfcheck_conversions)."""
    bad = ctypes.c_ulonglong(0)
    _check(lib().cfs_selfcheck_conversions(int(samples), ctypes.byref(bad)),
           "cfs_selfcheck_conversions")
    return bad.value


def selfcheck_f64_addsub(samples: int = 1 << 22, on_device: bool = True) -> int:
    """Bit mismatches of the library's integer-unit FP64 additions and
    subtractions against the FP64 hardware's over `samples` hashed operand
    pairs, on the GPU or, with on_device=False, on the host CPU
    (cfs_selfcheck_f64_addsub)."""
    bad = ctypes.c_ulonglong(0)
    _check(lib().cfs_selfcheck_f64_addsub(int(samples), 1 if on_device else 0, ctypes.byref(bad)),
           "cfs_selfcheck_f64_addsub")
    return bad.value


def f64_addsub_host(a, b):
    """(a + b, a - b) elementwise by the library's integer-unit FP64 additions,
    run on the host CPU (cfs_f64_addsub_host); a and b are float64 arrays of
    one shape."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError("a and b must have the same shape")
    s, d = np.empty_like(a), np.empty_like(a)
    p = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib().cfs_f64_addsub_host(a.size, p(a), p(b), p(s), p(d)), "cfs_f64_addsub_host")
    return s, d


def probe_addsub(on_integer_units: bool, iters: int = 1 << 14):
    """(butterfly pairs per second, launch ms) of (a + b, a - b) in FP64 on the
    FP64 pipe or on the integer units (cfs_probe_addsub)."""
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().cfs_probe_addsub(1 if on_integer_units else 0, int(iters), ctypes.byref(rate),
                                  ctypes.byref(ms)), "cfs_probe_addsub")
    return rate.value, ms.value


def _host_ptr(a, shape):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != int(np.prod(shape)):
            raise ValueError("host buffer must be a contiguous float64 array of the field size")
        return ctypes.c_void_p(a.ctypes.data)
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != int(np.prod(shape)):
            raise ValueError("host buffer must be a contiguous float64 CPU tensor of the field size")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("host buffer must be a numpy array or a CPU tensor")
