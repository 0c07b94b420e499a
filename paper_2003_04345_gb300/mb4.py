"""Thin ctypes binding of libmb4 (include/mb4.h).

Argument marshalling only: every step of the MB4 path runs in the library's
CUDA kernels.  There is no CPU fallback; if libmb4.so has not been built, or
no GPU is present, calls raise.

Arrays may be numpy (host memory) or torch CUDA tensors (device memory,
passed by pointer with on_device = 1).  Complex states are split into their
real and imaginary parts, S = nx*ny doubles each, row-major (k = y*nx + x).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmb4.so")

MB4_OK = 0
MB4_ERR_INVALID_ARG = -1
MB4_ERR_OUT_OF_MEMORY = -2
MB4_ERR_CUDA = -3
MB4_ERR_NEWTON_NOT_CONVERGED = -4
MB4_ERR_KRYLOV_BREAKDOWN = -5
MB4_ERR_NONFINITE = -6
MB4_ERR_TIMEOUT = -7
MB4_ERR_ADMISSION_REJECTED = -8

MB4_FP64 = 0
MB4_MIXED = 1
MAX_KRYLOV_S = 10
KERNEL_CLASSES = ("setup", "residual", "matvec", "gram", "update", "accept")

# Every entry point include/mb4.h declares.
EXPORTS = ("mb4_default_options", "mb4_create", "mb4_create_sparse", "mb4_destroy", "mb4_set_state", "mb4_get_state",
           "mb4_get_stages", "mb4_step", "mb4_step_async", "mb4_wait", "mb4_step_profiled", "mb4_energy",
           "mb4_norm", "mb4_observables", "mb4_residual", "mb4_solve_shifted", "mb4_get_launch_shape",
           "mb4_set_chi_field", "mb4_constants", "mb4_status_string", "mb4_version", "mb4_observables_noalloc",
           "mb4_batch_create", "mb4_batch_destroy", "mb4_batch_set_state", "mb4_batch_get_state", "mb4_batch_load",
           "mb4_batch_enable", "mb4_batch_step_async", "mb4_batch_wait", "mb4_batch_step", "mb4_batch_observables",
           "mb4_batch_clear_errors", "mb4_batch_get_launch_shape", "mb4_batch_set_chi_field", "mb4_batch_bytes",
           "mb4_batch_step_profiled", "mb4_fp64_fma_rate", "mb4_batch_get_tile_shape", "mb4_server_create",
           "mb4_server_destroy", "mb4_server_submit", "mb4_server_run", "mb4_server_result", "mb4_server_clock")


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("tx", C.c_double), ("ty", C.c_double),
                ("onsite", C.c_double)]


class Potential(C.Structure):
    _fields_ = [("v", C.c_void_p), ("on_device", C.c_int)]


class Nonlinearity(C.Structure):
    _fields_ = [("chi", C.c_double)]


class SparseKinetic(C.Structure):
    _fields_ = [("S", C.c_int), ("max_degree", C.c_int), ("nbr", C.c_void_p), ("t", C.c_void_p),
                ("onsite", C.c_double), ("t_im", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("newton_rtol", C.c_double), ("newton_max", C.c_int), ("krylov_s", C.c_int),
                ("precision", C.c_int), ("alpha1", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
                ("stream", C.c_void_p), ("use_graph", C.c_int), ("newton_predict", C.c_double),
                ("overlap_launches", C.c_int), ("newton_start", C.c_int), ("newton_start_adaptive", C.c_int),
                ("autotune", C.c_int), ("site_threads", C.c_int), ("precondition", C.c_int),
                ("site_chi", C.c_int), ("persistent", C.c_int), ("powers_tile", C.c_int),
                ("wait_limit", C.c_longlong)]


class Stats(C.Structure):
    _fields_ = [("steps_done", C.c_longlong), ("newton_iters_total", C.c_longlong),
                ("newton_iters_last", C.c_int), ("last_update_inf", C.c_double), ("u0_inf", C.c_double),
                ("update_hist", C.c_double * 8)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["update_hist"] = list(self.update_hist)[:max(0, self.newton_iters_last)]
        return d


class Request(C.Structure):
    _fields_ = [("grid", Grid), ("h", C.c_double), ("chi", C.c_double), ("nsteps", C.c_int),
                ("v", C.c_void_p), ("re", C.c_void_p), ("im", C.c_void_p), ("arrival", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("done", C.c_int), ("steps_done", C.c_longlong),
                ("newton_iters_total", C.c_longlong), ("arrival", C.c_double), ("admitted", C.c_double),
                ("completed", C.c_double), ("energy_start", C.c_double), ("energy_end", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MB4Error(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)


def lib():
    """Load libmb4.so (built in-tree by paper_2003_04345_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -m paper_2003_04345_gb300.build`")
        L = C.CDLL(LIB_PATH)
        L.mb4_default_options.argtypes = [C.POINTER(Options)]
        L.mb4_create_sparse.argtypes = [C.POINTER(SparseKinetic), C.POINTER(Potential), C.POINTER(Nonlinearity),
                                        C.c_double, C.POINTER(Options), C.POINTER(_P)]
        L.mb4_create.argtypes = [C.POINTER(Grid), C.POINTER(Potential), C.POINTER(Nonlinearity), C.c_double,
                                 C.POINTER(Options), C.POINTER(_P)]
        L.mb4_destroy.argtypes = [_P]
        L.mb4_destroy.restype = None
        L.mb4_set_state.argtypes = [_P, _P, _P, C.c_int]
        L.mb4_get_state.argtypes = [_P, _P, _P, C.c_int]
        L.mb4_get_stages.argtypes = [_P, _P, _P, C.c_int]
        L.mb4_step.argtypes = [_P, C.c_int, C.POINTER(Stats)]
        L.mb4_step_async.argtypes = [_P, C.c_int]
        L.mb4_get_launch_shape.argtypes = [_P, C.POINTER(C.c_int)]
        L.mb4_set_chi_field.argtypes = [_P, C.c_void_p, C.c_int]
        L.mb4_batch_set_chi_field.argtypes = [_P, C.c_int, C.c_void_p, C.c_int]
        L.mb4_batch_get_launch_shape.argtypes = [_P, C.POINTER(C.c_int)]
        L.mb4_wait.argtypes = [_P, C.POINTER(Stats)]
        L.mb4_step_profiled.argtypes = [_P, C.c_int, C.POINTER(Stats), _D, C.POINTER(C.c_longlong), _D]
        L.mb4_energy.argtypes = [_P, _D, _D]
        L.mb4_norm.argtypes = [_P, _D]
        L.mb4_observables.argtypes = [_P, _D]
        L.mb4_residual.argtypes = [_P, _P, _P, _P, _P, _P, _P, C.c_int]
        L.mb4_solve_shifted.argtypes = [_P, _P, _P, _P, _P, _P, _P, C.c_int]
        L.mb4_constants.argtypes = [C.c_double, C.c_double, C.c_double, _D, _D, _D, _D, _D, _D]
        L.mb4_status_string.argtypes = [C.c_int]
        L.mb4_status_string.restype = C.c_char_p
        L.mb4_version.restype = C.c_char_p
        L.mb4_observables_noalloc.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                              _P, _P, _P, _P, _P]
        L.mb4_batch_create.argtypes = [C.POINTER(Grid), C.c_int, C.POINTER(Potential), _D, C.c_double,
                                       C.POINTER(Options), C.POINTER(_P)]
        L.mb4_batch_destroy.argtypes = [_P]
        L.mb4_batch_destroy.restype = None
        L.mb4_batch_set_state.argtypes = [_P, C.c_int, _P, _P, C.c_int]
        L.mb4_batch_get_state.argtypes = [_P, C.c_int, _P, _P, C.c_int]
        L.mb4_batch_load.argtypes = [_P, C.c_int, _P, C.c_double, _P, _P, C.c_int]
        L.mb4_batch_enable.argtypes = [_P, C.c_int, C.c_int]
        L.mb4_batch_step_async.argtypes = [_P, C.c_int]
        L.mb4_batch_wait.argtypes = [_P, C.POINTER(Stats), C.POINTER(C.c_int)]
        L.mb4_batch_step.argtypes = [_P, C.c_int, C.POINTER(Stats), C.POINTER(C.c_int)]
        L.mb4_batch_observables.argtypes = [_P, _D]
        L.mb4_batch_step_profiled.argtypes = [_P, C.c_int, C.POINTER(Stats), C.POINTER(C.c_int), _D,
                                              C.POINTER(C.c_longlong), _D]
        L.mb4_fp64_fma_rate.argtypes = [C.c_double, _D, _D]
        L.mb4_batch_get_tile_shape.argtypes = [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.mb4_batch_clear_errors.argtypes = [_P]
        L.mb4_batch_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(Options)]
        L.mb4_batch_bytes.restype = C.c_longlong
        L.mb4_server_create.argtypes = [C.c_longlong, C.c_int, C.c_int, C.POINTER(Options), C.POINTER(_P)]
        L.mb4_server_destroy.argtypes = [_P]
        L.mb4_server_destroy.restype = None
        L.mb4_server_submit.argtypes = [_P, C.POINTER(Request), C.POINTER(C.c_longlong)]
        L.mb4_server_run.argtypes = [_P, C.c_double, C.POINTER(C.c_longlong)]
        L.mb4_server_result.argtypes = [_P, C.c_longlong, C.POINTER(Result), _P, _P]
        L.mb4_server_clock.argtypes = [_P]
        L.mb4_server_clock.restype = C.c_double
        _lib = L
    return _lib


def status_string(code):
    try:
        return lib().mb4_status_string(int(code)).decode()
    except Exception:  # the library itself failed to load
        return "unknown"


def _check(rc, what):
    if rc != MB4_OK:
        raise MB4Error(rc, what)


def constants(alpha1=-712.5, c1=1.0 / 3.0, c2=2.0 / 3.0):
    """The MB4 constants computed by the library on the host (no GPU needed)."""
    E = np.zeros(12)
    lam = np.zeros(3)
    T = np.zeros(9)
    Ti = np.zeros(9)
    gx = np.zeros(6)
    gw = np.zeros(6)
    ptr = lambda a: a.ctypes.data_as(_D)
    _check(lib().mb4_constants(alpha1, c1, c2, ptr(E), ptr(lam), ptr(T), ptr(Ti), ptr(gx), ptr(gw)),
           "mb4_constants")
    return {"E": E.reshape(3, 4), "lam": lam, "T": T.reshape(3, 3), "Tinv": Ti.reshape(3, 3),
            "gauss_x": gx, "gauss_w": gw}


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class _Planar:
    """Real/imag planes of a complex array as two contiguous float64 buffers.

    numpy input -> host buffers; torch CUDA input -> device buffers."""

    def __init__(self, z, n):
        if _is_torch(z):
            import torch
            z = z.reshape(-1)
            if z.numel() != n:
                raise ValueError(f"expected {n} complex values, got {z.numel()}")
            if z.is_complex():
                self.re = z.real.to(torch.float64).contiguous()
                self.im = z.imag.to(torch.float64).contiguous()
            else:
                raise ValueError("expected a complex tensor")
            if not self.re.is_cuda:
                raise ValueError("torch tensors must be on the GPU; pass numpy arrays for host memory")
            self.on_device = 1
            self.pre, self.pim = self.re.data_ptr(), self.im.data_ptr()
        else:
            z = np.asarray(z).reshape(-1)
            if z.size != n:
                raise ValueError(f"expected {n} complex values, got {z.size}")
            self.re = np.ascontiguousarray(z.real, dtype=np.float64)
            self.im = np.ascontiguousarray(z.imag, dtype=np.float64)
            self.on_device = 0
            self.pre, self.pim = self.re.ctypes.data, self.im.ctypes.data


class Integrator:
    """One MB4 context (mb4_create ... mb4_destroy)."""

    def __init__(self, nx, ny, V, chi, h, tx=1.0, ty=None, onsite=0.0, precision="fp64", **opts):
        """opts: the mb4_options fields (krylov_s, newton_rtol, newton_max, alpha1, c1, c2,
        stream, use_graph, newton_predict, overlap_launches, newton_start, newton_start_adaptive,
        autotune, site_threads, precondition, site_chi, persistent, powers_tile, wait_limit)."""
        L = lib()
        self.nx, self.ny = int(nx), int(ny)
        self.S = self.nx * self.ny
        self.h = float(h)
        self._ctx = _P()
        grid = Grid(self.nx, self.ny, float(tx), float(tx if ty is None else ty), float(onsite))
        if _is_torch(V):
            Vd = V.reshape(-1).to(dtype=__import__("torch").float64).contiguous()
            if Vd.numel() != self.S or not Vd.is_cuda:
                raise ValueError("V must hold nx*ny values on the GPU (or be a numpy array)")
            pot = Potential(Vd.data_ptr(), 1)
            keep = Vd
        else:
            Vh = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
            if Vh.size != self.S:
                raise ValueError("V must hold nx*ny values")
            pot = Potential(Vh.ctypes.data, 0)
            keep = Vh
        opt = _options(precision=precision, **opts)
        self.precision = precision
        _check(L.mb4_create(C.byref(grid), C.byref(pot), C.byref(Nonlinearity(float(chi))), self.h,
                            C.byref(opt), C.byref(self._ctx)), "mb4_create")
        del keep

    @classmethod
    def sparse(cls, K, V, chi, h, precision="fp64", **opts):
        """A context for a general kinetic matrix (mb4_create_sparse): K is S x S,
        Hermitian, real or complex (dense or scipy sparse).  A constant diagonal is passed
        as K's on-site term (so U_K and U_E split as for K and V); a diagonal that varies
        from site to site is folded into V (U_E then carries it)."""
        Kd = K.toarray() if hasattr(K, "toarray") else np.asarray(K)
        cplx = np.iscomplexobj(Kd) and bool(np.any(Kd.imag))
        Kd = Kd.astype(np.complex128 if cplx else np.float64)
        S = Kd.shape[0]
        off = Kd - np.diag(np.diag(Kd))
        deg = max(1, int((off != 0).sum(axis=1).max()))
        nbr = -np.ones((S, deg), dtype=np.int32)
        t = np.zeros((S, deg))
        ti = np.zeros((S, deg))
        for k in range(S):
            js = np.nonzero(off[k])[0]
            nbr[k, :len(js)] = js
            t[k, :len(js)] = off[k, js].real
            ti[k, :len(js)] = off[k, js].imag
        dg = np.diag(Kd).real
        onsite = float(dg[0]) if S and np.all(dg == dg[0]) else 0.0
        Vh = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(S) + (dg - onsite))
        self = cls.__new__(cls)
        self.nx, self.ny, self.S, self.h = S, 1, S, float(h)
        self.precision = precision
        self._ctx = _P()
        spk = SparseKinetic(S, deg, nbr.ctypes.data, t.ctypes.data, onsite, ti.ctypes.data if cplx else None)
        _check(lib().mb4_create_sparse(C.byref(spk), C.byref(Potential(Vh.ctypes.data, 0)),
                                       C.byref(Nonlinearity(float(chi))), self.h,
                                       C.byref(_options(precision=precision, **opts)), C.byref(self._ctx)),
               "mb4_create_sparse")
        return self

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().mb4_destroy(self._ctx)
            self._ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- state -----------------------------------------------------------
    def set_state(self, psi):
        p = _Planar(psi, self.S)
        _check(lib().mb4_set_state(self._ctx, p.pre, p.pim, p.on_device), "mb4_set_state")

    def get_state(self):
        re = np.empty(self.S)
        im = np.empty(self.S)
        _check(lib().mb4_get_state(self._ctx, re.ctypes.data, im.ctypes.data, 0), "mb4_get_state")
        return re + 1j * im

    def get_state_device(self, re, im):
        """Copy the state into two caller-owned float64 CUDA tensors of S elements."""
        _check(lib().mb4_get_state(self._ctx, re.data_ptr(), im.data_ptr(), 1), "mb4_get_state")

    def stages(self):
        re = np.empty(3 * self.S)
        im = np.empty(3 * self.S)
        _check(lib().mb4_get_stages(self._ctx, re.ctypes.data, im.ctypes.data, 0), "mb4_get_stages")
        return (re + 1j * im).reshape(3, self.S)

    # -- stepping --------------------------------------------------------
    def step(self, nsteps=1, check=True):
        st = Stats()
        rc = lib().mb4_step(self._ctx, int(nsteps), C.byref(st))
        if check:
            _check(rc, "mb4_step")
        return (st.as_dict(), rc) if not check else st.as_dict()

    def set_chi_field(self, chi):
        """Per-site chi (S values; the context needs site_chi=True)."""
        a = np.ascontiguousarray(np.asarray(chi, dtype=np.float64).reshape(-1))
        if a.size != self.S:
            raise ValueError("chi field must hold nx*ny values")
        _check(lib().mb4_set_chi_field(self._ctx, a.ctypes.data, 0), "mb4_set_chi_field")

    def launch_shape(self):
        """Per-site kernels (set-up/accept, residual, basis, update): threads per block,
        then blocks per instance."""
        out = (C.c_int * 8)()
        _check(lib().mb4_get_launch_shape(self._ctx, out), "mb4_get_launch_shape")
        return tuple(out)

    def tile_shape(self):
        """(tx, ty) of the FP32 matrix-powers tile in use, (0, 0) where it is not used."""
        tx, ty = C.c_int(), C.c_int()
        _check(lib().mb4_batch_get_tile_shape(self._ctx, C.byref(tx), C.byref(ty)), "mb4_batch_get_tile_shape")
        return tx.value, ty.value

    def step_async(self, nsteps=1):
        """Queue nsteps steps on the stream without waiting (see wait)."""
        _check(lib().mb4_step_async(self._ctx, int(nsteps)), "mb4_step_async")

    def wait(self, check=True):
        """Wait for queued steps; stats cover every step since the last wait/step."""
        st = Stats()
        rc = lib().mb4_wait(self._ctx, C.byref(st))
        if check:
            _check(rc, "mb4_wait")
            return st.as_dict()
        return st.as_dict(), rc

    def step_profiled(self, nsteps=1):
        """Host-driven steps with CUDA events around every kernel: returns
        (stats, {kernel class: (total ms, launches, sites computed)})."""
        st = Stats()
        ms = np.zeros(len(KERNEL_CLASSES))
        sites = np.zeros(len(KERNEL_CLASSES))
        n = (C.c_longlong * len(KERNEL_CLASSES))()
        _check(lib().mb4_step_profiled(self._ctx, int(nsteps), C.byref(st), ms.ctypes.data_as(_D), n,
                                       sites.ctypes.data_as(_D)), "mb4_step_profiled")
        return st.as_dict(), {k: (float(ms[i]), int(n[i]), float(sites[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def set_state_ptr(self, re_ptr, im_ptr, on_device):
        """Set the state from raw pointers (host pinned or device), S doubles each."""
        _check(lib().mb4_set_state(self._ctx, re_ptr, im_ptr, int(on_device)), "mb4_set_state")

    def get_state_ptr(self, re_ptr, im_ptr, on_device):
        _check(lib().mb4_get_state(self._ctx, re_ptr, im_ptr, int(on_device)), "mb4_get_state")

    # -- observables -----------------------------------------------------
    def observables(self):
        out = np.zeros(6)
        _check(lib().mb4_observables(self._ctx, out.ctypes.data_as(_D)), "mb4_observables")
        return {"H": out[0], "U_K": out[1], "U_E": out[2], "U_nl": out[3], "norm2": out[4],
                "participation": out[5]}

    def energy(self):
        H = C.c_double()
        parts = np.zeros(3)
        _check(lib().mb4_energy(self._ctx, C.byref(H), parts.ctypes.data_as(_D)), "mb4_energy")
        return H.value, parts

    def norm2(self):
        n = C.c_double()
        _check(lib().mb4_norm(self._ctx, C.byref(n)), "mb4_norm")
        return n.value

    # -- kernels on their own (testing) ------------------------------------
    def residual(self, u0, U):
        a = _Planar(u0, self.S)
        b = _Planar(np.asarray(U), 3 * self.S)
        re = np.empty(3 * self.S)
        im = np.empty(3 * self.S)
        _check(lib().mb4_residual(self._ctx, a.pre, a.pim, b.pre, b.pim, re.ctypes.data, im.ctypes.data, 0),
               "mb4_residual")
        return (re + 1j * im).reshape(3, self.S)

    def solve_shifted(self, u0, rhs):
        a = _Planar(u0, self.S)
        b = _Planar(np.asarray(rhs), 3 * self.S)
        re = np.empty(3 * self.S)
        im = np.empty(3 * self.S)
        _check(lib().mb4_solve_shifted(self._ctx, a.pre, a.pim, b.pre, b.pim, re.ctypes.data, im.ctypes.data,
                                       0), "mb4_solve_shifted")
        return (re + 1j * im).reshape(3, self.S)


def fp64_fma_rate(seconds=0.2):
    """Measured FP64 FMA throughput of the current device (flop/s, FMA = 2) and the
    duration of the timed launch (mb4_fp64_fma_rate)."""
    f = C.c_double()
    t = C.c_double()
    _check(lib().mb4_fp64_fma_rate(float(seconds), C.byref(f), C.byref(t)), "mb4_fp64_fma_rate")
    return f.value, t.value


def observables_noalloc(nx, ny, re, im, V, out6, chi, tx=1.0, ty=None, onsite=0.0, stream=None):
    """mb4_observables_noalloc on torch CUDA tensors (float64; re, im, V of nx*ny
    elements, out6 of 6): enqueues the reduction on ``stream`` without allocating."""
    sp = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().mb4_observables_noalloc(int(nx), int(ny), float(tx), float(tx if ty is None else ty),
                                         float(onsite), float(chi), re.data_ptr(), im.data_ptr(), V.data_ptr(),
                                         out6.data_ptr(), sp), "mb4_observables_noalloc")


def _options(precision="fp64", krylov_s=0, newton_rtol=1e-13, newton_max=30, alpha1=-712.5, c1=1.0 / 3.0,
             c2=2.0 / 3.0, stream=None, use_graph=True, newton_predict=0.0, overlap_launches=True,
             newton_start=None, newton_start_adaptive=None, autotune=None, site_threads=None,
             precondition=None, site_chi=None, persistent=None, wait_limit=None, powers_tile=None):
    opt = Options()
    lib().mb4_default_options(C.byref(opt))
    opt.newton_rtol = float(newton_rtol)
    opt.newton_max = int(newton_max)
    opt.krylov_s = int(krylov_s)
    opt.precision = {"fp64": MB4_FP64, "mixed": MB4_MIXED}[precision] if isinstance(precision, str) \
        else int(precision)
    opt.alpha1 = float(alpha1)
    opt.c1, opt.c2 = float(c1), float(c2)
    opt.use_graph = 1 if use_graph else 0
    opt.newton_predict = float(newton_predict)
    opt.overlap_launches = 1 if overlap_launches else 0
    if newton_start is not None:                # None keeps the library default
        opt.newton_start = int(newton_start)
    if newton_start_adaptive is not None:
        opt.newton_start_adaptive = 1 if newton_start_adaptive else 0
    if autotune is not None:
        opt.autotune = 1 if autotune else 0
    if site_threads is not None:
        opt.site_threads = int(site_threads)
    if precondition is not None:
        opt.precondition = int(precondition)
    if site_chi is not None:
        opt.site_chi = 1 if site_chi else 0
    if persistent is not None:
        opt.persistent = int(persistent)
    if wait_limit is not None:
        opt.wait_limit = int(wait_limit)
    if powers_tile is not None:
        opt.powers_tile = int(powers_tile)
    if stream is not None:
        opt.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return opt


def batch_bytes(nx, ny, batch, **opts):
    """Device bytes a batch of this shape would allocate (mb4_batch_bytes)."""
    return int(lib().mb4_batch_bytes(int(nx), int(ny), int(batch), C.byref(_options(**opts))))


class Batch:
    """B independent instances of one grid shape and h (mb4_batch_*).  V is
    (B, S) or B*S host values; chi holds B values."""

    def __init__(self, nx, ny, V, chi, h, tx=1.0, ty=None, onsite=0.0, **opts):
        L = lib()
        self.nx, self.ny = int(nx), int(ny)
        self.S = self.nx * self.ny
        chi = np.ascontiguousarray(np.asarray(chi, dtype=np.float64).reshape(-1))
        self.B = chi.size
        Vh = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
        if Vh.size != self.B * self.S:
            raise ValueError("V must hold B*nx*ny values")
        self._ctx = _P()
        grid = Grid(self.nx, self.ny, float(tx), float(tx if ty is None else ty), float(onsite))
        _check(L.mb4_batch_create(C.byref(grid), self.B, C.byref(Potential(Vh.ctypes.data, 0)),
                                  chi.ctypes.data_as(_D), float(h), C.byref(_options(**opts)),
                                  C.byref(self._ctx)), "mb4_batch_create")

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().mb4_batch_destroy(self._ctx)
            self._ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, psi, instance=-1):
        n = self.S * (self.B if instance < 0 else 1)
        p = _Planar(psi, n)
        _check(lib().mb4_batch_set_state(self._ctx, int(instance), p.pre, p.pim, p.on_device), "mb4_batch_set_state")

    def get_state(self, instance=-1):
        n = self.S * (self.B if instance < 0 else 1)
        re = np.empty(n)
        im = np.empty(n)
        _check(lib().mb4_batch_get_state(self._ctx, int(instance), re.ctypes.data, im.ctypes.data, 0),
               "mb4_batch_get_state")
        z = re + 1j * im
        return z.reshape(self.B, self.S) if instance < 0 else z

    def load(self, instance, V, chi, psi):
        Vh = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
        p = _Planar(psi, self.S)
        if p.on_device:
            raise ValueError("load takes host arrays")
        _check(lib().mb4_batch_load(self._ctx, int(instance), Vh.ctypes.data, float(chi), p.pre, p.pim, 0),
               "mb4_batch_load")

    def enable(self, instance, enabled=True):
        _check(lib().mb4_batch_enable(self._ctx, int(instance), 1 if enabled else 0), "mb4_batch_enable")

    def step_async(self, nsteps=1):
        _check(lib().mb4_batch_step_async(self._ctx, int(nsteps)), "mb4_batch_step_async")

    def wait(self):
        """(per-instance stats list, per-instance status codes)."""
        st = (Stats * self.B)()
        codes = (C.c_int * self.B)()
        rc = lib().mb4_batch_wait(self._ctx, st, codes)
        if rc not in (MB4_OK, MB4_ERR_NEWTON_NOT_CONVERGED, MB4_ERR_KRYLOV_BREAKDOWN, MB4_ERR_NONFINITE):
            _check(rc, "mb4_batch_wait")     # not a per-instance code: the call itself failed
        return [s.as_dict() for s in st], list(codes)

    def step(self, nsteps=1):
        self.step_async(nsteps)
        return self.wait()

    def step_profiled(self, nsteps=1):
        """Host-driven steps with CUDA events around every launch: returns
        (per-instance stats, status codes, {kernel class: (total ms, launches)})."""
        st = (Stats * self.B)()
        codes = (C.c_int * self.B)()
        ms = np.zeros(len(KERNEL_CLASSES))
        sites = np.zeros(len(KERNEL_CLASSES))
        n = (C.c_longlong * len(KERNEL_CLASSES))()
        rc = lib().mb4_batch_step_profiled(self._ctx, int(nsteps), st, codes, ms.ctypes.data_as(_D), n,
                                           sites.ctypes.data_as(_D))
        if rc not in (MB4_OK, MB4_ERR_NEWTON_NOT_CONVERGED, MB4_ERR_KRYLOV_BREAKDOWN, MB4_ERR_NONFINITE):
            _check(rc, "mb4_batch_step_profiled")
        return ([s.as_dict() for s in st], list(codes),
                {k: (float(ms[i]), int(n[i]), float(sites[i])) for i, k in enumerate(KERNEL_CLASSES)})

    def observables(self):
        out = np.zeros(self.B * 6)
        _check(lib().mb4_batch_observables(self._ctx, out.ctypes.data_as(_D)), "mb4_batch_observables")
        return out.reshape(self.B, 6)

    def clear_errors(self):
        _check(lib().mb4_batch_clear_errors(self._ctx), "mb4_batch_clear_errors")

    def set_chi_field(self, instance, chi):
        a = np.ascontiguousarray(np.asarray(chi, dtype=np.float64).reshape(-1))
        if a.size != self.S:
            raise ValueError("chi field must hold nx*ny values")
        _check(lib().mb4_batch_set_chi_field(self._ctx, int(instance), a.ctypes.data, 0), "mb4_batch_set_chi_field")

    def launch_shape(self):
        out = (C.c_int * 8)()
        _check(lib().mb4_batch_get_launch_shape(self._ctx, out), "mb4_batch_get_launch_shape")
        return tuple(out)

    def tile_shape(self):
        """(tx, ty) of the FP32 matrix-powers tile in use, (0, 0) where it is not used."""
        tx, ty = C.c_int(), C.c_int()
        _check(lib().mb4_batch_get_tile_shape(self._ctx, C.byref(tx), C.byref(ty)), "mb4_batch_get_tile_shape")
        return tx.value, ty.value


class Server:
    """Continuous-batching server (mb4_server_*): requests of different grids, h,
    step counts and potentials share the GPU inside an HBM budget."""

    def __init__(self, hbm_budget_bytes, max_slots=64, keep_states=False, **opts):
        self._ctx = _P()
        _check(lib().mb4_server_create(int(hbm_budget_bytes), int(max_slots), 1 if keep_states else 0,
                                       C.byref(_options(**opts)), C.byref(self._ctx)), "mb4_server_create")
        self.sizes = {}

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().mb4_server_destroy(self._ctx)
            self._ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, nx, ny, V, chi, psi, h, nsteps, arrival=0.0, tx=1.0, ty=None, onsite=0.0):
        Vh = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
        p = _Planar(psi, nx * ny)
        req = Request(Grid(int(nx), int(ny), float(tx), float(tx if ty is None else ty), float(onsite)),
                      float(h), float(chi), int(nsteps), Vh.ctypes.data, p.pre, p.pim, float(arrival))
        rid = C.c_longlong()
        _check(lib().mb4_server_submit(self._ctx, C.byref(req), C.byref(rid)), "mb4_server_submit")
        self.sizes[rid.value] = nx * ny
        return rid.value

    def run(self, until=1e300):
        n = C.c_longlong()
        _check(lib().mb4_server_run(self._ctx, float(until), C.byref(n)), "mb4_server_run")
        return n.value

    def result(self, rid, state=False):
        res = Result()
        if state:
            S = self.sizes[rid]
            re = np.empty(S)
            im = np.empty(S)
            _check(lib().mb4_server_result(self._ctx, int(rid), C.byref(res), re.ctypes.data, im.ctypes.data),
                   "mb4_server_result")
            return res.as_dict(), re + 1j * im
        _check(lib().mb4_server_result(self._ctx, int(rid), C.byref(res), None, None), "mb4_server_result")
        return res.as_dict()

    def clock(self):
        return lib().mb4_server_clock(self._ctx)


def from_workload(w, precision="fp64", **kw):
    """An Integrator for an inputs.Workload, with its potential and wavepacket set."""
    it = Integrator(w.nx, w.ny, w.potential(), w.chi, w.h, tx=w.tx, ty=w.ty, onsite=w.eps0,
                    precision=precision, **kw)
    it.set_state(w.psi0())
    return it
