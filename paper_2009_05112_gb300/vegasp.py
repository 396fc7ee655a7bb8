"""Python binding of libvegasp (include/vegasp.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module only
converts numpy arrays and torch streams to the C-ABI's plain pointers.  It
fails loudly (ImportError) when ``libvegasp.so`` has not been built: there is
no CPU fallback.

The C entry points are exposed under their own names (``vp_map_create``,
``vp_iterate``, ``vp_adapt``, ``vp_step``, ``vp_result`` ...) through
``lib()``; :class:`Integrator` wraps one context for convenience.
"""
import ctypes
import os

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvegasp.so")

VP_OK, VP_EINVAL, VP_ENOMEM, VP_ECUDA, VP_ETIMEOUT, VP_ENONFINITE, VP_EBUSY = range(7)
VP_FP64, VP_FP32 = 0, 1
VP_GAUSS, VP_BALL, VP_EXPNORM, VP_POSTERIOR = 0, 1, 2, 3
STATUS_NAMES = {0: "VP_OK", 1: "VP_EINVAL", 2: "VP_ENOMEM", 3: "VP_ECUDA", 4: "VP_ETIMEOUT",
                5: "VP_ENONFINITE", 6: "VP_EBUSY"}


class VegasError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class vp_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("lo", ctypes.POINTER(ctypes.c_double)),
                ("hi", ctypes.POINTER(ctypes.c_double)), ("n_g", ctypes.c_int),
                ("n_ev", ctypes.c_int64), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("integral_id", ctypes.c_uint32),
                ("precision", ctypes.c_int), ("plus2", ctypes.c_int), ("n_st", ctypes.c_int),
                ("max_it", ctypes.c_int), ("n_st_axis", ctypes.POINTER(ctypes.c_int32)),
                ("mixed", ctypes.c_int), ("n_extra", ctypes.c_int),
                ("out_mono", ctypes.POINTER(ctypes.c_int32)), ("d_weighted", ctypes.c_int),
                ("nst_div", ctypes.c_int)]


class vp_integrand(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_param", ctypes.c_int),
                ("param", ctypes.POINTER(ctypes.c_double))]


class vp_result_t(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("sdev", ctypes.c_double), ("chi2", ctypes.c_double),
                ("dof", ctypes.c_int), ("n_it", ctypes.c_int), ("n_eval", ctypes.c_int64),
                ("last_i", ctypes.c_double), ("last_sdev", ctypes.c_double)]


class vp_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_int64), ("max_active", ctypes.c_int)]


class vp_request(ctypes.Structure):
    _fields_ = [("p", vp_params), ("f", vp_integrand), ("rtol", ctypes.c_double),
                ("discard", ctypes.c_int), ("min_meas", ctypes.c_int), ("tag", ctypes.c_uint64)]


class vp_served(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("converged", ctypes.c_int), ("n_iter", ctypes.c_int), ("r", vp_result_t),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class vp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("finished", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("active", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("bytes_peak", ctypes.c_int64),
                ("mem_budget", ctypes.c_int64), ("n_eval", ctypes.c_int64),
                ("busy_s", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_P = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "vp_set_allocator": [ALLOC_FN, FREE_FN, _P],
    "vp_map_create": [ctypes.POINTER(vp_params), ctypes.POINTER(vp_integrand), _P,
                      ctypes.POINTER(_P)],
    "vp_iterate": [_P, _P],
    "vp_adapt": [_P, _P],
    "vp_step": [_P, _P],
    "vp_result": [_P, ctypes.c_int, ctypes.POINTER(vp_result_t)],
    "vp_map_destroy": [_P],
    "vp_get_info": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                    ctypes.POINTER(ctypes.c_int)],
    "vp_get_strata": [_P, _P],
    "vp_get_history_multi": [_P, ctypes.c_int, _P, _P],
    "vp_result_multi": [_P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "vp_get_moments_multi": [_P, _P, _P],
    "vp_precondition": [_P, ctypes.c_int64, _P, _P, ctypes.c_int, _P],
    "vp_export_state": [_P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "vp_import_state": [_P, _P, ctypes.c_size_t],
    "vp_get_edges": [_P, _P],
    "vp_set_edges": [_P, _P],
    "vp_get_alloc": [_P, _P, _P],
    "vp_get_moments": [_P, _P, _P],
    "vp_get_hist": [_P, _P, _P],
    "vp_get_history": [_P, ctypes.c_int, _P, _P],
    "vp_get_dh": [_P, _P, ctypes.POINTER(ctypes.c_double)],
    "vp_iterate_part": [_P, ctypes.c_int, ctypes.c_int, _P],
    "vp_partials_size": [_P, ctypes.POINTER(ctypes.c_int64)],
    "vp_partials_export": [_P, _P, _P],
    "vp_partials_import": [_P, _P, _P],
    "vp_estimate": [_P, _P],
    "vp_alloc_from_dh": [_P, _P, _P],
    "vp_alloc_from_sigma": [_P, _P, _P],
    "vp_refine_from_hist": [_P, _P, _P, _P],
    "vp_eval_samples": [_P, ctypes.c_int64, _P, _P, ctypes.c_uint32, _P, _P, _P, _P],
    "vp_last_sample_ms": [_P, ctypes.POINTER(ctypes.c_float)],
    "vp_shared_atomic_rate": [ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
    "vp_alloc_static": [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _P, _P, _P],
    "vp_result_unweighted": [_P, ctypes.c_int, ctypes.POINTER(vp_result_t)],
    "vp_set_damping": [_P, ctypes.c_double, ctypes.c_double],
    "vp_get_tuning": [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                      ctypes.POINTER(ctypes.c_int)],
    "vp_set_tuning": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "vp_batch_create": [ctypes.c_int, ctypes.POINTER(vp_params), ctypes.POINTER(vp_integrand), _P,
                        ctypes.POINTER(_P)],
    "vp_batch_iterate": [_P, _P],
    "vp_batch_adapt": [_P, _P],
    "vp_batch_step": [_P, _P],
    "vp_batch_result": [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp_result_t)],
    "vp_batch_results": [_P, ctypes.c_int, _P],
    "vp_batch_size": [_P, ctypes.POINTER(ctypes.c_int)],
    "vp_batch_destroy": [_P],
    "vp_batch_history": [_P, ctypes.c_int, ctypes.c_int, _P, _P],
    "vp_step_read": [_P, _P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                     ctypes.POINTER(ctypes.c_double)],
    "vp_step_read_flush": [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double)],
    "vp_batch_result_multi": [_P, ctypes.c_int, ctypes.c_int, _P, _P,
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_int)],
    "vp_batch_history_multi": [_P, ctypes.c_int, ctypes.c_int, _P, _P],
    "vp_server_create": [ctypes.POINTER(vp_server_config), _P, ctypes.POINTER(_P)],
    "vp_server_submit": [_P, ctypes.POINTER(vp_request), ctypes.POINTER(ctypes.c_uint64)],
    "vp_server_step": [_P, ctypes.POINTER(ctypes.c_int)],
    "vp_server_start": [_P],
    "vp_server_stop": [_P],
    "vp_server_poll": [_P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int)],
    "vp_server_wait": [_P, ctypes.c_int64, ctypes.c_double],
    "vp_server_get_stats": [_P, ctypes.POINTER(vp_server_stats)],
    "vp_server_destroy": [_P],
}

_lib = None


def lib():
    """The loaded library (raises ImportError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libvegasp.so is not built (run __graft_entry__.build()); "
                              "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.vp_last_error.argtypes = []
        L.vp_last_error.restype = ctypes.c_char_p
        L.vp_server_clock.argtypes = []
        L.vp_server_clock.restype = ctypes.c_double
        _lib = L
    return _lib


def check(status):
    if status != VP_OK:
        raise VegasError(status, lib().vp_last_error().decode(errors="replace"))
    return status


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def current_stream():
    """cudaStream_t of torch's current stream (0 when torch/CUDA is absent)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


# torch's caching allocator as the library's device allocator --------------
_keep = []


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # the library reports VP_ENOMEM
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _keep[:] = [a, f]
    check(lib().vp_set_allocator(a, f, None))


def shared_atomic_rate(f32=False):
    """Shared-memory atomic adds per second on the current device in the
    sampling kernel's histogram pattern (vp_shared_atomic_rate): 32-bit integer
    adds (the counts) or, with f32, FP32 adds (the sums)."""
    r = ctypes.c_double()
    check(lib().vp_shared_atomic_rate(1 if f32 else 0, ctypes.byref(r)))
    return r.value


class Integrator:
    """One vegas+ integral on the GPU (a vp_ctx)."""

    def __init__(self, dim, lo, hi, kind, prm, n_g=1000, n_ev=10_000, alpha=0.5, beta=0.75,
                 seed=0, integral_id=0, precision=VP_FP64, plus2=False, n_st=0, max_it=0,
                 stream=None, n_st_axis=None, mixed=False, out_mono=None, d_weighted=False,
                 nst_div=0):
        self.dim, self.n_g = int(dim), int(n_g)
        self._lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (self.dim,)))
        self._hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, np.float64), (self.dim,)))
        self._prm = np.ascontiguousarray(prm, np.float64)
        if isinstance(precision, str):
            precision = {"fp64": VP_FP64, "fp32": VP_FP32}[precision]
        p = vp_params(self.dim, self._lo.ctypes.data_as(_dp), self._hi.ctypes.data_as(_dp),
                      self.n_g, int(n_ev), float(alpha), float(beta), int(seed) & (2 ** 64 - 1),
                      int(integral_id), int(precision), int(bool(plus2)), int(n_st), int(max_it))
        if n_st_axis is not None:
            self._nst = np.ascontiguousarray(n_st_axis, np.int32).reshape(self.dim)
            p.n_st_axis = self._nst.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.mixed = int(bool(mixed))
        p.d_weighted = int(bool(d_weighted))
        p.nst_div = int(nst_div)
        self.n_out = 1
        if out_mono:  # extra outputs f x^a x^b (App. B)
            self._mono = np.ascontiguousarray(np.asarray(out_mono, np.int32).reshape(-1))
            p.n_extra = self._mono.size // 2
            p.out_mono = self._mono.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            self.n_out = 1 + p.n_extra
        f = vp_integrand(int(kind), self._prm.size, self._prm.ctypes.data_as(_dp))
        self.stream = current_stream() if stream is None else ctypes.c_void_p(stream)
        h = ctypes.c_void_p()
        check(lib().vp_map_create(ctypes.byref(p), ctypes.byref(f), self.stream, ctypes.byref(h)))
        self.ctx = h
        n_st_, n_hc_, _ = self.info()
        self.n_st, self.n_hc = n_st_, n_hc_

    @classmethod
    def from_problem(cls, prob: "_inputs.Problem", precision=VP_FP64, **kw):
        args = dict(dim=prob.dim, lo=prob.lo, hi=prob.hi, kind=prob.kind, prm=prob.prm,
                    n_g=prob.n_g, n_ev=prob.n_ev, alpha=prob.alpha, beta=prob.beta,
                    seed=prob.seed, integral_id=prob.integral_id, precision=precision,
                    plus2=prob.plus2, n_st=prob.n_st, n_st_axis=prob.n_st_axis,
                    mixed=prob.mixed, d_weighted=prob.d_weighted, nst_div=prob.nst_div)
        args.update(kw)
        return cls(**args)

    def close(self):
        if getattr(self, "ctx", None):
            lib().vp_map_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # the method
    def iterate(self):
        check(lib().vp_iterate(self.ctx, self.stream))

    def adapt(self):
        check(lib().vp_adapt(self.ctx, self.stream))

    def step(self):
        check(lib().vp_step(self.ctx, self.stream))

    def run(self, n_it, graph=True):
        for _ in range(n_it):
            if graph:
                self.step()
            else:
                self.iterate()
                self.adapt()
        return self

    def step_read(self):
        """One step; returns the previous step_read call's (I_j, sigma_j^2), or
        None on the first call (vp_step_read)."""
        have, i, v = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        check(lib().vp_step_read(self.ctx, self.stream, ctypes.byref(have), ctypes.byref(i),
                                 ctypes.byref(v)))
        return (i.value, v.value) if have.value else None

    def step_read_flush(self):
        """The last step_read call's (I_j, sigma_j^2), or None."""
        have, i, v = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        check(lib().vp_step_read_flush(self.ctx, ctypes.byref(have), ctypes.byref(i),
                                       ctypes.byref(v)))
        return (i.value, v.value) if have.value else None

    def set_damping(self, alpha, beta):
        """alpha, beta for the following iterations (alpha = 0 freezes the map)."""
        check(lib().vp_set_damping(self.ctx, float(alpha), float(beta)))

    def result(self, discard=0, allow_nonfinite=False, unweighted=False):
        r = vp_result_t()
        fn = lib().vp_result_unweighted if unweighted else lib().vp_result
        st = fn(self.ctx, int(discard), ctypes.byref(r))
        if not (allow_nonfinite and st == VP_ENONFINITE):
            check(st)
        return dict(mean=r.mean, sdev=r.sdev, chi2=r.chi2, dof=r.dof, n_it=r.n_it,
                    n_eval=r.n_eval, last_i=r.last_i, last_sdev=r.last_sdev, status=st)

    # inspection
    def info(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        check(lib().vp_get_info(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def history_multi(self, n=None):
        """I_j[n][M] and cov_j[n][M][M] of the outputs (App. B)."""
        n = self.info()[2] if n is None else int(n)
        I = np.zeros((n, self.n_out))
        C = np.zeros((n, self.n_out, self.n_out))
        check(lib().vp_get_history_multi(self.ctx, n, _ptr(I), _ptr(C)))
        return I, C

    def result_multi(self, discard=0):
        """The outputs combined over iterations j >= discard (App. B, §2.5)."""
        M = self.n_out
        mean, cov = np.zeros(M), np.zeros((M, M))
        chi2, dof, n_it = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
        check(lib().vp_result_multi(self.ctx, int(discard), _ptr(mean), _ptr(cov),
                                    ctypes.byref(chi2), ctypes.byref(dof), ctypes.byref(n_it)))
        return dict(mean=mean, cov=cov, chi2=chi2.value, dof=dof.value, n_it=n_it.value)

    def moments_multi(self):
        """The latest iteration's per-hypercube sums X1[N_h][M], X2[N_h][M(M+1)/2]."""
        M = self.n_out
        x1 = np.zeros((self.n_hc, M))
        x2 = np.zeros((self.n_hc, M * (M + 1) // 2))
        check(lib().vp_get_moments_multi(self.ctx, _ptr(x1), _ptr(x2)))
        return x1, x2

    def precondition(self, x, f=None, n_iter=10):
        """§4.2: trains the map on sample data {x, f(x)} (f None: the
        integrand), n_iter refinements on the same data."""
        x = np.ascontiguousarray(x, np.float64).reshape(-1, self.dim)
        fa = None if f is None else np.ascontiguousarray(f, np.float64).reshape(-1)
        check(lib().vp_precondition(self.ctx, x.shape[0], _ptr(x), _ptr(fa), int(n_iter),
                                    self.stream))
        return self

    def export_state(self):
        """The context's state between iterations (bytes), for vp_import_state."""
        n = ctypes.c_size_t()
        check(lib().vp_export_state(self.ctx, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        check(lib().vp_export_state(self.ctx, buf, n.value, ctypes.byref(n)))
        return buf.raw

    def import_state(self, blob):
        """Resumes from a state written by export_state (same parameters)."""
        check(lib().vp_import_state(self.ctx, blob, len(blob)))
        return self

    def strata(self):
        """Strata on every axis (§3.2)."""
        out = np.zeros(self.dim, np.int32)
        check(lib().vp_get_strata(self.ctx, _ptr(out)))
        return out

    def edges(self):
        out = np.zeros((self.dim, self.n_g + 1))
        check(lib().vp_get_edges(self.ctx, _ptr(out)))
        return out

    def set_edges(self, e):
        e = np.ascontiguousarray(e, np.float64)
        assert e.shape == (self.dim, self.n_g + 1)
        check(lib().vp_set_edges(self.ctx, _ptr(e)))

    def alloc(self):
        n = np.zeros(self.n_hc, np.uint32)
        off = np.zeros(self.n_hc + 1, np.uint64)
        check(lib().vp_get_alloc(self.ctx, _ptr(n), _ptr(off)))
        return n, off

    def moments(self):
        s1, s2 = np.zeros(self.n_hc), np.zeros(self.n_hc)
        check(lib().vp_get_moments(self.ctx, _ptr(s1), _ptr(s2)))
        return s1, s2

    def hist(self):
        hs = np.zeros((self.dim, self.n_g))
        hc = np.zeros((self.dim, self.n_g))
        check(lib().vp_get_hist(self.ctx, _ptr(hs), _ptr(hc)))
        return hs, hc

    def history(self):
        n = self.info()[2]
        I, V = np.zeros(n), np.zeros(n)
        check(lib().vp_get_history(self.ctx, n, _ptr(I), _ptr(V)))
        return I, V

    # one integral over several devices: sampling in parts, the partial sums
    # exchanged by the caller, then the estimate (see vegasp.h)
    def iterate_part(self, part, n_parts):
        check(lib().vp_iterate_part(self.ctx, int(part), int(n_parts), self.stream))

    def partials_size(self):
        n = ctypes.c_int64(0)
        check(lib().vp_partials_size(self.ctx, ctypes.byref(n)))
        return n.value

    def export_partials(self, dev_ptr):
        """Packs the iteration's partial sums into the device buffer at
        dev_ptr (partials_size() doubles)."""
        check(lib().vp_partials_export(self.ctx, ctypes.c_void_p(int(dev_ptr)), self.stream))

    def import_partials(self, dev_ptr):
        check(lib().vp_partials_import(self.ctx, ctypes.c_void_p(int(dev_ptr)), self.stream))

    def estimate(self):
        check(lib().vp_estimate(self.ctx, self.stream))

    def dh(self):
        """(d_h[N_h], sum d) as the latest estimate or reallocation left them."""
        d = np.zeros(self.n_hc)
        sd = ctypes.c_double(0.0)
        check(lib().vp_get_dh(self.ctx, _ptr(d), ctypes.byref(sd)))
        return d, sd.value

    def alloc_from_dh(self, d_h):
        d = np.ascontiguousarray(d_h, np.float64)
        assert d.size == self.n_hc
        check(lib().vp_alloc_from_dh(self.ctx, _ptr(d), self.stream))

    def alloc_from_sigma(self, sigma):
        d = np.ascontiguousarray(sigma, np.float64)
        assert d.size == self.n_hc
        check(lib().vp_alloc_from_sigma(self.ctx, _ptr(d), self.stream))

    def refine_from_hist(self, hsum, hcnt):
        hs = np.ascontiguousarray(hsum, np.float64).reshape(self.dim, self.n_g)
        hc = np.ascontiguousarray(hcnt, np.float64).reshape(self.dim, self.n_g)
        check(lib().vp_refine_from_hist(self.ctx, _ptr(hs), _ptr(hc), self.stream))

    def eval_samples(self, h, j, t):
        h = np.ascontiguousarray(h, np.uint64)
        j = np.ascontiguousarray(j, np.uint32)
        n = h.size
        x = np.zeros((n, self.dim))
        idx = np.zeros((n, self.dim), np.int32)
        jac, f = np.zeros(n), np.zeros(n)
        check(lib().vp_eval_samples(self.ctx, n, _ptr(h), _ptr(j), int(t), _ptr(x), _ptr(idx),
                                    _ptr(jac), _ptr(f)))
        return x, idx, jac, f

    def tuning(self):
        v = [ctypes.c_int() for _ in range(5)]
        check(lib().vp_get_tuning(self.ctx, *[ctypes.byref(x) for x in v]))
        return dict(scheme=["static-cluster", "tasks", "static-dynamic"][v[0].value],
                    blocks=v[1].value,
                    threads=v[2].value, cluster=v[3].value, run=v[4].value)

    def set_tuning(self, scheme, blocks, threads=256, cluster=1, run=8):
        """Fixes the sampling launch shape (scheme "static-cluster", "tasks" or
        "static-dynamic")."""
        code = ({"static-cluster": 0, "tasks": 1, "static-dynamic": 2}[scheme]
                if isinstance(scheme, str) else int(scheme))
        check(lib().vp_set_tuning(self.ctx, code, int(blocks), int(threads), int(cluster),
                                  int(run)))

    def last_sample_ms(self):
        ms = ctypes.c_float()
        check(lib().vp_last_sample_ms(self.ctx, ctypes.byref(ms)))
        return ms.value


def _result_dict(r, st):
    return dict(mean=r.mean, sdev=r.sdev, chi2=r.chi2, dof=r.dof, n_it=r.n_it, n_eval=r.n_eval,
                last_i=r.last_i, last_sdev=r.last_sdev, status=st)


class Batch:
    """Many independent integrals iterated together (a vp_batch)."""

    def __init__(self, problems, precision=VP_FP32, stream=None, out_mono=None):
        """out_mono: None, or per problem None or the (a, b) pairs of its extra
        outputs f x^a x^b (App. B; FP64)."""
        self.n = len(problems)
        self._keep = []
        self.n_out = [1] * self.n
        ps = (vp_params * self.n)()
        fs = (vp_integrand * self.n)()
        for i, prob in enumerate(problems):
            lo = np.ascontiguousarray(np.broadcast_to(np.asarray(prob.lo, np.float64), (prob.dim,)))
            hi = np.ascontiguousarray(np.broadcast_to(np.asarray(prob.hi, np.float64), (prob.dim,)))
            prm = np.ascontiguousarray(prob.prm, np.float64)
            self._keep += [lo, hi, prm]
            ps[i] = vp_params(prob.dim, lo.ctypes.data_as(_dp), hi.ctypes.data_as(_dp), prob.n_g,
                              int(prob.n_ev), float(prob.alpha), float(prob.beta),
                              int(prob.seed) & (2 ** 64 - 1), int(prob.integral_id),
                              int(precision), int(bool(prob.plus2)), int(prob.n_st), 0)
            _set_strata(ps[i], prob, self._keep)
            if out_mono is not None and out_mono[i]:
                mono = np.ascontiguousarray(np.asarray(out_mono[i], np.int32).reshape(-1))
                self._keep.append(mono)
                ps[i].n_extra = mono.size // 2
                ps[i].out_mono = mono.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
                self.n_out[i] = 1 + mono.size // 2
            fs[i] = vp_integrand(int(prob.kind), prm.size, prm.ctypes.data_as(_dp))
        self.stream = current_stream() if stream is None else ctypes.c_void_p(stream)
        h = ctypes.c_void_p()
        check(lib().vp_batch_create(self.n, ps, fs, self.stream, ctypes.byref(h)))
        self.b = h

    def close(self):
        if getattr(self, "b", None):
            lib().vp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self):
        check(lib().vp_batch_iterate(self.b, self.stream))

    def adapt(self):
        check(lib().vp_batch_adapt(self.b, self.stream))

    def step(self):
        check(lib().vp_batch_step(self.b, self.stream))

    def run(self, n_it, graph=True):
        for _ in range(n_it):
            if graph:
                self.step()
            else:
                self.iterate()
                self.adapt()
        return self

    def result(self, i, discard=0):
        r = vp_result_t()
        st = lib().vp_batch_result(self.b, int(i), int(discard), ctypes.byref(r))
        if st not in (VP_OK, VP_ENONFINITE):
            check(st)
        return _result_dict(r, st)

    def history(self, i):
        n = self.result(i)["n_it"]
        I, Vv = np.zeros(n), np.zeros(n)
        check(lib().vp_batch_history(self.b, int(i), n, _ptr(I), _ptr(Vv)))
        return I, Vv

    def history_multi(self, i, n=None):
        """Integral i's I_j[n][M] and cov_j[n][M][M] (App. B)."""
        n = self.result(i)["n_it"] if n is None else int(n)
        M = self.n_out[i] if 0 <= i < self.n else 1
        I, C = np.zeros((n, M)), np.zeros((n, M, M))
        check(lib().vp_batch_history_multi(self.b, int(i), n, _ptr(I), _ptr(C)))
        return I, C

    def result_multi(self, i, discard=0):
        """Integral i's outputs combined over iterations j >= discard (App. B, §2.5)."""
        M = self.n_out[i] if 0 <= i < self.n else 1  # (the library refuses a bad index)
        mean, cov = np.zeros(M), np.zeros((M, M))
        chi2, dof, n_it = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
        check(lib().vp_batch_result_multi(self.b, int(i), int(discard), _ptr(mean), _ptr(cov),
                                          ctypes.byref(chi2), ctypes.byref(dof),
                                          ctypes.byref(n_it)))
        return dict(mean=mean, cov=cov, chi2=chi2.value, dof=dof.value, n_it=n_it.value)

    def results(self, discard=0):
        out = (vp_result_t * self.n)()
        st = lib().vp_batch_results(self.b, int(discard), out)
        if st not in (VP_OK, VP_ENONFINITE):
            check(st)
        return [_result_dict(out[i], VP_OK) for i in range(self.n)]


def _params_of(prob, precision, max_it, keep):
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(prob.lo, np.float64), (prob.dim,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(prob.hi, np.float64), (prob.dim,)))
    prm = np.ascontiguousarray(prob.prm, np.float64)
    keep += [lo, hi, prm]
    p = vp_params(prob.dim, lo.ctypes.data_as(_dp), hi.ctypes.data_as(_dp), prob.n_g,
                  int(prob.n_ev), float(prob.alpha), float(prob.beta),
                  int(prob.seed) & (2 ** 64 - 1), int(prob.integral_id), int(precision),
                  int(bool(prob.plus2)), int(prob.n_st), int(max_it))
    _set_strata(p, prob, keep)
    f = vp_integrand(int(prob.kind), prm.size, prm.ctypes.data_as(_dp))
    return p, f


def _set_strata(p, prob, keep):
    """The per-axis strata fields of vp_params from a Problem (§3.2)."""
    if getattr(prob, "n_st_axis", None) is not None:
        a = np.ascontiguousarray(prob.n_st_axis, np.int32).reshape(prob.dim)
        keep.append(a)
        p.n_st_axis = a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.mixed = int(bool(getattr(prob, "mixed", False)))
    p.d_weighted = int(bool(getattr(prob, "d_weighted", False)))
    p.nst_div = int(getattr(prob, "nst_div", 0))


def clock():
    """The server's clock (seconds, steady)."""
    return lib().vp_server_clock()


class Server:
    """A stream of integration requests iterated together (a vp_server)."""

    def __init__(self, mem_budget=0, max_active=0, stream=None):
        cfg = vp_server_config(int(mem_budget), int(max_active))
        self.stream = ctypes.c_void_p(0) if stream is None else ctypes.c_void_p(stream)
        h = ctypes.c_void_p()
        check(lib().vp_server_create(ctypes.byref(cfg), self.stream, ctypes.byref(h)))
        self.s = h

    def close(self):
        if getattr(self, "s", None):
            lib().vp_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, prob, rtol, discard=0, min_meas=1, max_it=0, precision=VP_FP32, tag=0):
        keep = []
        p, f = _params_of(prob, precision, max_it, keep)
        q = vp_request(p, f, float(rtol), int(discard), int(min_meas), int(tag) & (2 ** 64 - 1))
        rid = ctypes.c_uint64()
        check(lib().vp_server_submit(self.s, ctypes.byref(q), ctypes.byref(rid)))
        return rid.value

    def step(self):
        n = ctypes.c_int()
        check(lib().vp_server_step(self.s, ctypes.byref(n)))
        return n.value

    def start(self):
        check(lib().vp_server_start(self.s))

    def stop(self):
        check(lib().vp_server_stop(self.s))

    def poll(self, max_n=4096):
        out = (vp_served * max_n)()
        n = ctypes.c_int()
        check(lib().vp_server_poll(self.s, max_n, out, ctypes.byref(n)))
        res = []
        for k in range(n.value):
            o = out[k]
            d = _result_dict(o.r, o.status)
            d.update(id=o.id, tag=o.tag, converged=bool(o.converged), n_iter=o.n_iter,
                     t_submit=o.t_submit, t_admit=o.t_admit, t_done=o.t_done)
            res.append(d)
        return res

    def wait(self, finished, timeout_s=60.0):
        check(lib().vp_server_wait(self.s, int(finished), float(timeout_s)))

    def stats(self):
        o = vp_server_stats()
        check(lib().vp_server_get_stats(self.s, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in vp_server_stats._fields_}
