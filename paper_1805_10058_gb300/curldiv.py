"""Thin ctypes binding of the C-ABI in include/curldiv.h (argument marshalling only).

Every computation runs in libcurldiv.so's CUDA kernels; there is no Python or CPU
fallback.  Device vectors are passed as torch CUDA tensors (FP64 or FP32, contiguous),
host vectors as numpy arrays.  Names follow the C entry points.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcurldiv.so")

CD_OK, CD_EINVAL, CD_ENOMEM, CD_ECUDA, CD_NOT_CONVERGED, CD_BREAKDOWN, CD_TIMEOUT, CD_CANCELLED = range(8)
CD_PREC_FP64, CD_PREC_FP32_IR = 0, 1
CD_PC_NONE, CD_PC_FD_D, CD_PC_FD_T, CD_PC_MG, CD_PC_T_BAND, CD_PC_MIM, CD_PC_WL = 0, 1, 2, 3, 4, 5, 6


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precond", ctypes.c_int), ("maxit", ctypes.c_int),
                ("rtol", ctypes.c_double), ("max_batch", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("inner_maxit", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("smoother_degree", ctypes.c_int),
                ("mg_m_min", ctypes.c_int), ("use_graphs", ctypes.c_int), ("chunk", ctypes.c_int),
                ("mixed_switch_ratio", ctypes.c_double), ("fd_tensor_cores", ctypes.c_int),
                ("autotune", ctypes.c_int), ("ext_residual", ctypes.c_int),
                ("emulated_fp64", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class Result(ctypes.Structure):
    _fields_ = [("iters_outer", ctypes.c_int), ("iters_inner", ctypes.c_int),
                ("relres", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int),
                ("relres_hi", ctypes.c_double)]

    def as_dict(self):
        return dict(iters_outer=self.iters_outer, iters_inner=self.iters_inner,
                    relres=self.relres, seconds=self.seconds, status=self.status,
                    relres_hi=self.relres_hi)


class ServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("workers", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("timeout_s", ctypes.c_double), ("solve", Options)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("solves", ctypes.c_uint64), ("p50_s", ctypes.c_double),
                ("p99_s", ctypes.c_double), ("mean_batch", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("bytes_in_use", ctypes.c_size_t), ("handles", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CurlDivError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load(path=LIB_PATH):
    """Loads libcurldiv.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i, d, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
    sig = {
        "cd_default_options": (None, [ctypes.POINTER(Options)]),
        "cd_dofs": (ctypes.c_size_t, [i, i, i]),
        "cd_strerror": (ctypes.c_char_p, [i]),
        "cd_last_error": (ctypes.c_char_p, []),
        "cd_create": (i, [ctypes.POINTER(vp), i, i, i, d, d, ctypes.POINTER(Options), vp]),
        "cd_create_aniso": (i, [ctypes.POINTER(vp), i, i, ctypes.POINTER(ctypes.c_int), d, d,
                                ctypes.POINTER(Options), vp]),
        "cd_destroy": (i, [vp]),
        "cd_apply": (i, [vp, vp, vp, i, dp, dp]),
        "cd_apply_f32": (i, [vp, vp, vp, i, dp, dp]),
        "cd_solve": (i, [vp, vp, vp, i, dp, dp, ctypes.POINTER(Result)]),
        "cd_solve_host": (i, [vp, vp, vp, i, dp, dp, ctypes.POINTER(Result)]),
        "cd_solve_ext": (i, [vp, vp, vp, vp, i, dp, dp, ctypes.POINTER(Result)]),
        "cd_precond": (i, [vp, i, vp, vp, i, dp, dp, i]),
        "cd_get_bands": (i, [vp, i, dp, dp, dp, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "cd_levels": (i, [vp]),
        "cd_get_eig": (i, [vp, i, dp, dp]),
        "cd_restrict": (i, [vp, i, vp, vp, i]),
        "cd_prolong": (i, [vp, i, vp, vp, i]),
        "cd_kernel_launches": (ctypes.c_uint64, []),
        "cd_symbol_eigs": (i, [i, i, d, d, dp, i, vp, vp, vp]),
        "cd_lanczos": (i, [vp, vp, i, i, dp, dp, dp, dp, dp, dp]),
        "cd_apply3d_static": (i, [i, i, d, d, vp, vp, i, vp]),
        "cd_setup_bands": (i, [i, i, i, dp, dp, dp, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "cd_setup_eig": (i, [i, i, i, dp, dp]),
        "cd_setup_tband": (i, [i, i, dp, dp]),
        "cd_server_default_options": (None, [ctypes.POINTER(ServerOptions)]),
        "cd_server_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(ServerOptions)]),
        "cd_server_submit": (i, [vp, i, i, i, dp, dp, dp, i, ctypes.POINTER(ctypes.c_uint64)]),
        "cd_server_poll": (i, [vp, ctypes.c_uint64, dp, ctypes.POINTER(Result), ctypes.POINTER(i)]),
        "cd_server_wait": (i, [vp, ctypes.c_uint64, dp, ctypes.POINTER(Result), d]),
        "cd_server_cancel": (i, [vp, ctypes.c_uint64]),
        "cd_server_stats_get": (i, [vp, ctypes.POINTER(ServerStats)]),
        "cd_server_destroy": (i, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st, what):
    if st != CD_OK:
        lib = load()
        raise CurlDivError(st, f"{what}: {lib.cd_strerror(st).decode()} ({lib.cd_last_error().decode()})")


def default_options(**kw):
    o = Options()
    load().cd_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def cd_dofs(d, p, n):
    return int(load().cd_dofs(d, p, n))


def cd_kernel_launches():
    return int(load().cd_kernel_launches())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def cd_setup_bands(p, n, level=0):
    """Host-only: the library's 1D bands (M, A, S) of grid level `level`, each (m, 2P+1)."""
    lib = load()
    m, P = ctypes.c_int(), ctypes.c_int()
    _check(lib.cd_setup_bands(p, n, level, None, None, None, ctypes.byref(m), ctypes.byref(P)),
           "cd_setup_bands")
    out = [np.zeros((m.value, 2 * P.value + 1)) for _ in range(3)]
    _check(lib.cd_setup_bands(p, n, level, *[_dp(x) for x in out], None, None), "cd_setup_bands")
    return out, P.value


def cd_setup_eig(p, n, which):
    """Host-only: FD eigenbasis (U, lam) of (p, n); which = 0 generalized (S, M), 1 T."""
    m = n + p - 2
    U, lam = np.zeros((m, m)), np.zeros(m)
    _check(load().cd_setup_eig(p, n, which, _dp(U), _dp(lam)), "cd_setup_eig")
    return U, lam


def cd_setup_tband(p, n):
    """Host-only: banded Cholesky factor of T (Lb of shape (m + q, q), dinv of length m)."""
    m, q = n + p - 2, p - 1
    Lb, dinv = np.zeros(max(1, (m + q) * q)), np.zeros(m)
    _check(load().cd_setup_tband(p, n, _dp(Lb), _dp(dinv)), "cd_setup_tband")
    return Lb[:(m + q) * q].reshape(m + q, q), dinv


def cd_apply3d_static(p, n, alpha, beta, w, y, stream=None, check=True):
    """y = A w (d = 3, FP64 CUDA tensors) through the allocation-free entry point."""
    import torch
    lib = load()
    N = cd_dofs(3, p, n)
    if N == 0:
        raise ValueError("cd_apply3d_static: invalid (p, n)")
    nrhs = _nrhs(N, w, y, "cd_apply3d_static")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.cd_apply3d_static(p, n, alpha, beta, _dev(w, "float64"), _dev(y, "float64"), nrhs,
                               ctypes.c_void_p(stream))
    if check:
        _check(st, "cd_apply3d_static")
    return st


def _nrhs(N, a, b, what):
    """Right-hand sides in a pair of vectors: both must hold the same whole number (>= 1) of
    N-entry right-hand sides (a short output would let the kernels write past its end)."""
    na, nb = int(a.numel() if hasattr(a, "numel") else a.size), int(b.numel() if hasattr(b, "numel") else b.size)
    if na < N or na % N or nb != na:
        raise ValueError(f"{what}: expected two vectors of the same length nrhs * {N} (nrhs >= 1), "
                         f"got {na} and {nb} entries")
    return na // N


def cd_symbol_eigs(d, p, alpha, beta, mg, lam, lap=None, nu=None, stream=None):
    """Eigenvalues of the symbol on the grid Gamma (device tensors lam [mg^d * d], lap [mg^d])."""
    import torch
    npts = mg ** d
    if lam.numel() != npts * d or (lap is not None and lap.numel() != npts):
        raise ValueError(f"cd_symbol_eigs: lam needs {npts * d} entries and lap {npts}")
    nuv = None if nu is None else np.ascontiguousarray(np.asarray(nu, dtype=np.float64))
    if nuv is not None and nuv.size != d:
        raise ValueError("cd_symbol_eigs: nu needs d entries")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = load().cd_symbol_eigs(d, p, alpha, beta, None if nuv is None else _dp(nuv), mg,
                               _dev(lam, "float64"), None if lap is None else _dev(lap, "float64"),
                               ctypes.c_void_p(stream))
    _check(st, "cd_symbol_eigs")


def _params(nrhs, alphas, betas):
    def arr(v):
        if v is None:
            return None, None
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), (nrhs,)))
        return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ka, pa = arr(alphas)
    kb, pb = arr(betas)
    return (ka, kb), pa, pb


def _dev(t, dtype_name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected torch.{dtype_name}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """Owns a cd_solver handle for (d, p, n); methods mirror the C entry points.  ``n`` is the
    number of intervals per direction, or a sequence of d per-direction counts (an anisotropic
    mesh: cd_create_aniso)."""

    def __init__(self, d, p, n, alpha=1.0, beta=1.0, stream=None, **opts):
        self.lib = load()
        self.d, self.p, self.n = d, p, n
        self.aniso = not np.isscalar(n)
        h = ctypes.c_void_p()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        if self.aniso:
            ns = [int(v) for v in n]
            if len(ns) != d:
                raise ValueError("one interval count per direction")
            self.ma = [v + p - 2 for v in ns]
            self.m = self.ma[0]
            self.N = d * int(np.prod(self.ma))
            self.opts = default_options(**opts)
            arr = (ctypes.c_int * d)(*ns)
            _check(self.lib.cd_create_aniso(ctypes.byref(h), d, p, arr, alpha, beta,
                                            ctypes.byref(self.opts), ctypes.c_void_p(stream)),
                   "cd_create_aniso")
        else:
            self.m = n + p - 2
            self.N = cd_dofs(d, p, n)
            self.opts = default_options(**opts)
            _check(self.lib.cd_create(ctypes.byref(h), d, p, n, alpha, beta, ctypes.byref(self.opts),
                                      ctypes.c_void_p(stream)), "cd_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.cd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cd_apply(self, w, y, alphas=None, betas=None):
        nrhs = _nrhs(self.N, w, y, "cd_apply")
        keep, pa, pb = _params(nrhs, alphas, betas)
        _check(self.lib.cd_apply(self.h, _dev(w, "float64"), _dev(y, "float64"), nrhs, pa, pb), "cd_apply")

    def cd_apply_f32(self, w, y, alphas=None, betas=None):
        nrhs = _nrhs(self.N, w, y, "cd_apply_f32")
        keep, pa, pb = _params(nrhs, alphas, betas)
        _check(self.lib.cd_apply_f32(self.h, _dev(w, "float32"), _dev(y, "float32"), nrhs, pa, pb),
               "cd_apply_f32")

    def cd_solve(self, b, x, alphas=None, betas=None, check=True):
        nrhs = _nrhs(self.N, b, x, "cd_solve")
        keep, pa, pb = _params(nrhs, alphas, betas)
        res = (Result * nrhs)()
        st = self.lib.cd_solve(self.h, _dev(b, "float64"), _dev(x, "float64"), nrhs, pa, pb, res)
        if check and st not in (CD_OK,):
            _check(st, "cd_solve")
        return st, [r.as_dict() for r in res]

    def cd_solve_ext(self, b, x, x_lo=None, alphas=None, betas=None, check=True):
        """Solve returning the double-FP64 solution x + x_lo (x_lo may be None)."""
        nrhs = _nrhs(self.N, b, x, "cd_solve_ext")
        if x_lo is not None:
            _nrhs(self.N, x, x_lo, "cd_solve_ext")
        keep, pa, pb = _params(nrhs, alphas, betas)
        res = (Result * nrhs)()
        lo = _dev(x_lo, "float64") if x_lo is not None else None
        st = self.lib.cd_solve_ext(self.h, _dev(b, "float64"), _dev(x, "float64"), lo, nrhs, pa, pb, res)
        if check and st not in (CD_OK,):
            _check(st, "cd_solve_ext")
        return st, [r.as_dict() for r in res]

    def cd_solve_host(self, b, x, alphas=None, betas=None):
        if not (b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous
                and x.flags.c_contiguous):
            raise TypeError("cd_solve_host: expected contiguous float64 numpy arrays")
        nrhs = _nrhs(self.N, b, x, "cd_solve_host")
        keep, pa, pb = _params(nrhs, alphas, betas)
        res = (Result * nrhs)()
        st = self.lib.cd_solve_host(self.h, ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(x.ctypes.data),
                                    nrhs, pa, pb, res)
        return st, [r.as_dict() for r in res]

    def cd_precond(self, kind, r, z, alphas=None, betas=None):
        f32 = str(r.dtype) == "torch.float32"
        nrhs = _nrhs(self.N, r, z, "cd_precond")
        keep, pa, pb = _params(nrhs, alphas, betas)
        dt = "float32" if f32 else "float64"
        _check(self.lib.cd_precond(self.h, kind, _dev(r, dt), _dev(z, dt), nrhs, pa, pb, int(f32)),
               "cd_precond")

    def cd_lanczos(self, v0, steps, alphas=None, betas=None):
        """Lanczos extremes of A for the start vectors v0 (FP64 CUDA tensor of nrhs * N)."""
        nrhs = _nrhs(self.N, v0, v0, "cd_lanczos")
        keep, pa, pb = _params(nrhs, alphas, betas)
        lmin, lmax = np.zeros(nrhs), np.zeros(nrhs)
        a, b = np.zeros((nrhs, steps)), np.zeros((nrhs, steps))
        _check(self.lib.cd_lanczos(self.h, _dev(v0, "float64"), nrhs, steps, pa, pb, _dp(lmin),
                                   _dp(lmax), _dp(a), _dp(b)), "cd_lanczos")
        return lmin, lmax, a, b

    def cd_levels(self):
        return int(self.lib.cd_levels(self.h))

    def cd_get_bands(self, level=0):
        m, P = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.cd_get_bands(self.h, level, None, None, None, ctypes.byref(m), ctypes.byref(P)),
               "cd_get_bands")
        W = 2 * P.value + 1
        arrs = [np.zeros((m.value, W)) for _ in range(3)]
        ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        _check(self.lib.cd_get_bands(self.h, level, ptr(arrs[0]), ptr(arrs[1]), ptr(arrs[2]),
                                     ctypes.byref(m), ctypes.byref(P)), "cd_get_bands")
        return arrs, P.value

    def cd_get_eig(self, which):
        U = np.zeros((self.m, self.m))
        lam = np.zeros(self.m)
        ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        _check(self.lib.cd_get_eig(self.h, which, ptr(U), ptr(lam)), "cd_get_eig")
        return U, lam

    def _transfer_nrhs(self, level, fine, coarse, what):
        if level < 0 or level + 1 >= self.cd_levels():
            raise ValueError(f"{what}: level {level} has no coarser level")
        Nf = self.d * self.level_m(level) ** self.d
        Nc = self.d * self.level_m(level + 1) ** self.d
        nf, nc = int(fine.numel()), int(coarse.numel())
        if nf < Nf or nf % Nf or nc != (nf // Nf) * Nc:
            raise ValueError(f"{what}: fine has {nf} entries and coarse {nc}; expected nrhs * {Nf} "
                             f"and nrhs * {Nc}")
        return nf // Nf

    def cd_restrict(self, level, fine, coarse):
        nrhs = self._transfer_nrhs(level, fine, coarse, "cd_restrict")
        _check(self.lib.cd_restrict(self.h, level, _dev(fine, "float64"), _dev(coarse, "float64"), nrhs),
               "cd_restrict")

    def cd_prolong(self, level, coarse, fine):
        nrhs = self._transfer_nrhs(level, fine, coarse, "cd_prolong")
        _check(self.lib.cd_prolong(self.h, level, _dev(coarse, "float64"), _dev(fine, "float64"), nrhs),
               "cd_prolong")

    def level_m(self, level):
        m = self.m
        for _ in range(level):
            m //= 2
        return m


def server_options(**kw):
    o = ServerOptions()
    load().cd_server_default_options(ctypes.byref(o))
    solve = kw.pop("solve", {})
    for k, v in kw.items():
        setattr(o, k, v)
    for k, v in solve.items():
        setattr(o.solve, k, v)
    return o


class Server:
    """Continuous-batching solve server (cd_server_*); host numpy buffers."""

    def __init__(self, **kw):
        self.lib = load()
        self.opts = server_options(**kw)
        h = ctypes.c_void_p()
        _check(self.lib.cd_server_create(ctypes.byref(h), ctypes.byref(self.opts)), "cd_server_create")
        self.h = h
        self.meta = {}

    def submit(self, d, p, n, alphas, betas, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        N = cd_dofs(d, p, n)
        if N == 0 or b.size < N or b.size % N:
            raise ValueError(f"submit: b must hold nrhs * {N} entries (nrhs >= 1), got {b.size}")
        nrhs = b.size // N
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(alphas, dtype=np.float64), (nrhs,)))
        be = np.ascontiguousarray(np.broadcast_to(np.asarray(betas, dtype=np.float64), (nrhs,)))
        t = ctypes.c_uint64()
        P = ctypes.POINTER(ctypes.c_double)
        st = self.lib.cd_server_submit(self.h, d, p, n, a.ctypes.data_as(P), be.ctypes.data_as(P),
                                       b.ctypes.data_as(P), nrhs, ctypes.byref(t))
        _check(st, "cd_server_submit")
        self.meta[t.value] = (N, nrhs)
        return t.value

    def _out(self, ticket):
        N, nrhs = self.meta[ticket]
        return np.zeros(N * nrhs), (Result * nrhs)()

    def poll(self, ticket):
        x, res = self._out(ticket)
        done = ctypes.c_int()
        st = self.lib.cd_server_poll(self.h, ticket, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     res, ctypes.byref(done))
        if not done.value:
            return None
        self.meta.pop(ticket)
        return st, x, [r.as_dict() for r in res]

    def wait(self, ticket, timeout_s=0.0):
        x, res = self._out(ticket)
        st = self.lib.cd_server_wait(self.h, ticket, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     res, timeout_s)
        if st == CD_TIMEOUT and timeout_s > 0:
            return None
        self.meta.pop(ticket, None)
        return st, x, [r.as_dict() for r in res]

    def cancel(self, ticket):
        return self.lib.cd_server_cancel(self.h, ticket)

    def stats(self):
        s = ServerStats()
        _check(self.lib.cd_server_stats_get(self.h, ctypes.byref(s)), "cd_server_stats_get")
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.cd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
