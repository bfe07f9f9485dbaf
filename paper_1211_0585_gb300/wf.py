"""ctypes binding of the C ABI declared in include/wf.h (argument marshalling
only: every step of the method runs in the CUDA library).

Device buffers are passed as integer device addresses (for example
`torch.Tensor.data_ptr()`); host buffers as numpy arrays. The library is
loaded on first use from paper_1211_0585_gb300/_build/libwf.so; if it is
missing or fails to load, every call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwf.so")

WF_OK, WF_EINVAL, WF_ENOMEM, WF_ECUDA, WF_ENOTCONVERGED, WF_ENUMERIC, WF_ETIMEOUT, WF_EBUSY, \
    WF_ECANCELLED, WF_ENOTFOUND = range(10)
WF_PREC_FP64, WF_PREC_MIXED, WF_PREC_FP64_NATIVE = 0, 1, 2
STATUS_NAMES = {0: "WF_OK", 1: "WF_EINVAL", 2: "WF_ENOMEM", 3: "WF_ECUDA", 4: "WF_ENOTCONVERGED",
                5: "WF_ENUMERIC", 6: "WF_ETIMEOUT", 7: "WF_EBUSY", 8: "WF_ECANCELLED", 9: "WF_ENOTFOUND"}

EXPORTED = ["wf_options_default", "wf_plan_create", "wf_plan_destroy", "wf_plan_info", "wf_plan_legendre_terms",
            "wf_plan_legendre_table", "wf_plan_kernels_per_iteration", "wf_plan_set_options",
            "wf_alm2map", "wf_map2alm", "wf_map2alm_noalloc", "wf_iterate", "wf_profile_iterations", "wf_solve",
            "wf_solve_history", "wf_solve_batch", "wf_constrained_realisations",
            "wf_multi_create", "wf_multi_solve", "wf_multi_destroy",
            "wf_pol_create", "wf_pol_solve", "wf_pol_alm2map", "wf_pol_map2alm", "wf_pol_destroy",
            "wf_server_create", "wf_submit", "wf_poll", "wf_cancel", "wf_server_warm", "wf_server_drain", "wf_server_stats",
            "wf_server_destroy", "wf_last_error"]


class WFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("cooling", ctypes.c_int), ("l_iter0", ctypes.c_int), ("lmax_margin", ctypes.c_int),
                ("band_limit", ctypes.c_int), ("plateau_eps", ctypes.c_double),
                ("final_dchi2", ctypes.c_double), ("min_level_iters", ctypes.c_int),
                ("max_level_iters", ctypes.c_int), ("graph_iters", ctypes.c_int),
                ("batch_slots", ctypes.c_int), ("legendre_table_bytes", ctypes.c_size_t),
                ("posterior_grad", ctypes.c_int), ("refine_iters", ctypes.c_int), ("refine_tol", ctypes.c_double), ("synthesis_table", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("levels", ctypes.c_int),
                ("lmax_sht_final", ctypes.c_int), ("lambda_final", ctypes.c_double), ("chi2", ctypes.c_double),
                ("chi2_prior", ctypes.c_double), ("chi2_noise", ctypes.c_double),
                ("chi2_per_dof", ctypes.c_double), ("rel_increment", ctypes.c_double),
                ("ms_device", ctypes.c_double), ("rel_posterior_grad", ctypes.c_double),
                ("ms_latency", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IterRecord(ctypes.Structure):
    _fields_ = [("chi2_prior", ctypes.c_double), ("chi2_noise", ctypes.c_double),
                ("chi2_lambda", ctypes.c_double), ("incr2", ctypes.c_double), ("norm2", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("lmax_sht", ctypes.c_int), ("level", ctypes.c_int)]

    def as_dict(self):
        return dict(chi2_prior=self.chi2_prior, chi2_noise=self.chi2_noise, chi2_lambda=self.chi2_lambda,
                    incr2=self.incr2, norm2=self.norm2, lam=self.lambda_, lsht=self.lmax_sht, level=self.level,
                    chi2=self.chi2_prior + self.chi2_noise)


_lib = None
_vp, _dp, _i, _d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double


def load(path: str = LIB_PATH):
    """Open libwf.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libwf.so not built ({path}); run paper_1211_0585_gb300.build.build()")
    L = ctypes.CDLL(path)
    sig = {
        "wf_options_default": [ctypes.POINTER(Options)],
        "wf_plan_create": [_i, _i, _vp, _vp, _vp, ctypes.POINTER(Options), ctypes.POINTER(_vp)],
        "wf_plan_destroy": [_vp],
        "wf_plan_info": [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _dp,
                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_size_t)],
        "wf_plan_set_options": [_vp, ctypes.POINTER(Options)],
        "wf_plan_legendre_terms": [_vp, _i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
        "wf_plan_legendre_table": [_vp, _i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
        "wf_plan_kernels_per_iteration": [_vp, ctypes.POINTER(_i)],
        "wf_alm2map": [_vp, _i, _vp, _vp],
        "wf_map2alm": [_vp, _i, _vp, _vp],
        "wf_map2alm_noalloc": [_i, _i, _vp, _vp, _vp],
        "wf_iterate": [_vp, _vp, _vp, _d, _i, _i, _i, ctypes.POINTER(IterRecord)],
        "wf_profile_iterations": [_vp, _vp, _vp, _d, _i, _i, ctypes.POINTER(ctypes.c_float)],
        "wf_solve": [_vp, _vp, _i, _vp, _i, _vp, ctypes.POINTER(Stats)],
        "wf_solve_history": [_vp, _vp, _i, _vp, _i, ctypes.POINTER(Stats), ctypes.POINTER(IterRecord), _i,
                             ctypes.POINTER(_i)],
        "wf_solve_batch": [_vp, _i, _vp, _i, _vp, _i, ctypes.POINTER(Stats)],
        "wf_constrained_realisations": [_vp, _i, ctypes.c_uint64, _vp, _i, _vp, _i, _vp, ctypes.POINTER(Stats)],
        "wf_multi_create": [_i, _i, _i, _vp, _vp, _vp, _vp, ctypes.POINTER(Options), ctypes.POINTER(_vp)],
        "wf_multi_solve": [_vp, _vp, _i, _vp, _i, ctypes.POINTER(Stats), ctypes.POINTER(IterRecord), _i,
                           ctypes.POINTER(_i)],
        "wf_multi_destroy": [_vp],
        "wf_pol_create": [_i, _i, _vp, _vp, _vp, _vp, ctypes.POINTER(Options), ctypes.POINTER(_vp)],
        "wf_pol_solve": [_vp, _vp, _i, _vp, _i, ctypes.POINTER(Stats), ctypes.POINTER(IterRecord), _i,
                         ctypes.POINTER(_i)],
        "wf_pol_alm2map": [_vp, _vp, _vp],
        "wf_pol_map2alm": [_vp, _vp, _vp],
        "wf_pol_destroy": [_vp],
        "wf_server_create": [ctypes.c_size_t, _i, ctypes.POINTER(_vp)],
        "wf_submit": [_vp, _i, _i, _vp, _vp, _vp, _vp, _d, ctypes.POINTER(ctypes.c_uint64)],
        "wf_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(_i), _vp, ctypes.POINTER(Stats)],
        "wf_cancel": [_vp, ctypes.c_uint64],
        "wf_server_drain": [_vp, _i],
        "wf_server_warm": [_vp, _i, _i, _i],
        "wf_server_stats": [_vp, _dp, _dp, ctypes.POINTER(ctypes.c_int64)],
        "wf_server_destroy": [_vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.wf_last_error.argtypes = []
    L.wf_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def last_error() -> str:
    return load().wf_last_error().decode()


def _check(st, ok=(WF_OK,)):
    if st not in ok:
        raise WFError(st, last_error())
    return st


def _host_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def map2alm_noalloc(nside: int, lmax: int, map_dev: int, alm_dev: int, stream: int = 0):
    """Plan-free map2alm that allocates no device memory (static 16 MiB scratch
    per GPU; concurrent calls on one GPU must be serialised by the caller)."""
    _check(load().wf_map2alm_noalloc(nside, lmax, ctypes.c_void_p(map_dev), ctypes.c_void_p(alm_dev),
                                     ctypes.c_void_p(stream) if stream else None))


def options(**kw) -> Options:
    o = Options()
    _check(load().wf_options_default(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Plan:
    """Owns a wf_plan_t (one nside, lmax, C_l, noise and mask)."""

    def __init__(self, nside, lmax, cl, noise_var, mask=None, opts: Options | None = None):
        L = load()
        self.nside, self.lmax = nside, lmax
        self._cl = np.ascontiguousarray(cl, dtype=np.float64)
        self._nv = np.ascontiguousarray(noise_var, dtype=np.float64)
        self._mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        if self._cl.size != lmax + 1 or self._nv.size != 12 * nside * nside:
            raise ValueError("cl / noise_var sizes do not match nside, lmax")
        if self._mask is not None and self._mask.size != self._nv.size:
            raise ValueError("mask size")
        h = ctypes.c_void_p()
        _check(L.wf_plan_create(nside, lmax, _host_ptr(self._cl), _host_ptr(self._nv), _host_ptr(self._mask),
                                ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().wf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def npix(self):
        return 12 * self.nside * self.nside

    @property
    def nalm(self):
        return (self.lmax + 1) * (self.lmax + 2) // 2

    def info(self):
        npix, nalm, nobs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        tau, nbytes = ctypes.c_double(), ctypes.c_size_t()
        _check(load().wf_plan_info(self.handle, ctypes.byref(npix), ctypes.byref(nalm), ctypes.byref(tau),
                                   ctypes.byref(nobs), ctypes.byref(nbytes)))
        return dict(npix=npix.value, nalm=nalm.value, tau=tau.value, n_obs=nobs.value, device_bytes=nbytes.value)

    def legendre_terms(self, lsht):
        """(evaluated, full) counts of (l, m, ring pair) Legendre terms at band limit lsht."""
        ev, full = ctypes.c_int64(), ctypes.c_int64()
        _check(load().wf_plan_legendre_terms(self.handle, lsht, ctypes.byref(ev), ctypes.byref(full)))
        return ev.value, full.value

    def legendre_table(self, lsht):
        """(held, per_pass) bytes of the precomputed lambda table (0 held: recurrence)."""
        held, per_pass = ctypes.c_int64(), ctypes.c_int64()
        _check(load().wf_plan_legendre_table(self.handle, lsht, ctypes.byref(held), ctypes.byref(per_pass)))
        return held.value, per_pass.value

    def kernels_per_iteration(self):
        n = _i()
        _check(load().wf_plan_kernels_per_iteration(self.handle, ctypes.byref(n)))
        return n.value

    def set_options(self, opts: Options):
        _check(load().wf_plan_set_options(self.handle, ctypes.byref(opts)))

    # device-pointer transforms
    def alm2map(self, lsht, alm_dev: int, map_dev: int):
        _check(load().wf_alm2map(self.handle, lsht, ctypes.c_void_p(alm_dev), ctypes.c_void_p(map_dev)))

    def map2alm(self, lsht, map_dev: int, alm_dev: int):
        _check(load().wf_map2alm(self.handle, lsht, ctypes.c_void_p(map_dev), ctypes.c_void_p(alm_dev)))

    def iterate(self, d_dev: int, s_dev: int, lam: float, lsht: int, niter: int, reset: bool = True):
        recs = (IterRecord * max(1, niter))()
        _check(load().wf_iterate(self.handle, ctypes.c_void_p(d_dev), ctypes.c_void_p(s_dev), float(lam), lsht,
                                 niter, 1 if reset else 0, recs))
        return [recs[i].as_dict() for i in range(niter)]

    def profile(self, d_dev: int, s_dev: int, lam: float, lsht: int, niter: int):
        """Average device ms per launch of (ring kernel, Legendre kernel, controller)."""
        ms = (ctypes.c_float * 3)()
        _check(load().wf_profile_iterations(self.handle, ctypes.c_void_p(d_dev), ctypes.c_void_p(s_dev), float(lam),
                                            lsht, niter, ms))
        return dict(ring=ms[0], legendre=ms[1], control=ms[2])

    def solve(self, d, alm_out=None, alm_init=None, on_device=False, history=0):
        """d: numpy (host) or device address (on_device=True). Returns (alm or None, stats, status, records)."""
        L = load()
        st = Stats()
        if on_device:
            dptr, aptr = ctypes.c_void_p(d), ctypes.c_void_p(alm_out)
            iptr = ctypes.c_void_p(alm_init) if alm_init else None
            out = None
        else:
            dh = np.ascontiguousarray(d, dtype=np.float64)
            out = np.empty(self.nalm, dtype=np.complex128) if alm_out is None else alm_out
            dptr, aptr = _host_ptr(dh), out.ctypes.data_as(ctypes.c_void_p)
            init = None if alm_init is None else np.ascontiguousarray(alm_init, dtype=np.complex128)
            iptr = _host_ptr(init)
        recs_out = []
        if history:
            recs = (IterRecord * history)()
            n = ctypes.c_int()
            status = L.wf_solve_history(self.handle, dptr, 1 if on_device else 0, aptr, 1 if on_device else 0,
                                        ctypes.byref(st), recs, history, ctypes.byref(n))
            recs_out = [recs[i].as_dict() for i in range(n.value)]
        else:
            status = L.wf_solve(self.handle, dptr, 1 if on_device else 0, aptr, 1 if on_device else 0, iptr,
                                ctypes.byref(st))
        _check(status, ok=(WF_OK, WF_ENOTCONVERGED))
        return out, st.as_dict(), status, recs_out

    def solve_batch(self, d, on_device=False, alm_out=None, nrhs=None):
        L = load()
        if on_device:
            stats = (Stats * nrhs)()
            status = L.wf_solve_batch(self.handle, nrhs, ctypes.c_void_p(d), 1, ctypes.c_void_p(alm_out), 1, stats)
            _check(status, ok=(WF_OK, WF_ENOTCONVERGED))
            return None, [stats[i].as_dict() for i in range(nrhs)], status
        dh = np.ascontiguousarray(d, dtype=np.float64)
        nrhs = dh.shape[0]
        out = np.empty((nrhs, self.nalm), dtype=np.complex128)
        stats = (Stats * nrhs)()
        status = L.wf_solve_batch(self.handle, nrhs, _host_ptr(dh), 0, out.ctypes.data_as(ctypes.c_void_p), 0, stats)
        _check(status, ok=(WF_OK, WF_ENOTCONVERGED))
        return out, [stats[i].as_dict() for i in range(nrhs)], status


    def constrained_realisations(self, d, nreal, seed, with_wf=True):
        """nreal constrained realisations s_WF(d) + xi_i - s_WF(Y xi_i + n_i) of host data d.
        Returns (cr [nreal, nalm] complex, s_WF(d) or None, stats of the nreal + 1 solves, status)."""
        dh = np.ascontiguousarray(d, dtype=np.float64)
        cr = np.empty((nreal, self.nalm), dtype=np.complex128)
        wfo = np.empty(self.nalm, dtype=np.complex128) if with_wf else None
        stats = (Stats * (nreal + 1))()
        status = load().wf_constrained_realisations(self.handle, nreal, ctypes.c_uint64(seed), _host_ptr(dh), 0,
                                                    cr.ctypes.data_as(ctypes.c_void_p), 0, _host_ptr(wfo), stats)
        _check(status, ok=(WF_OK, WF_ENOTCONVERGED))
        return cr, wfo, [stats[i].as_dict() for i in range(nreal + 1)], status


class Multi:
    """Owns a wf_multi_t: the joint Wiener filter of several maps of one sky
    (one messenger field per map)."""

    def __init__(self, nside, lmax, cl, noise_vars, masks=None, beams=None, opts: Options | None = None):
        self.nside, self.lmax = nside, lmax
        self._cl = np.ascontiguousarray(cl, dtype=np.float64)
        self._nv = np.ascontiguousarray(np.stack(noise_vars), dtype=np.float64)
        self.ndet = self._nv.shape[0]
        self._mask = None if masks is None else np.ascontiguousarray(np.stack(masks), dtype=np.uint8)
        self._beams = None if beams is None else np.ascontiguousarray(np.stack(beams), dtype=np.float64)
        h = ctypes.c_void_p()
        _check(load().wf_multi_create(nside, lmax, self.ndet, _host_ptr(self._cl), _host_ptr(self._beams),
                                      _host_ptr(self._nv), _host_ptr(self._mask),
                                      ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
        self.handle = h

    @property
    def nalm(self):
        return (self.lmax + 1) * (self.lmax + 2) // 2

    def solve(self, ds, history=0):
        """ds: [ndet][Npix] host maps. Returns (alm, stats, status, records)."""
        dh = np.ascontiguousarray(np.stack(ds), dtype=np.float64)
        out = np.empty(self.nalm, dtype=np.complex128)
        st = Stats()
        recs = (IterRecord * max(1, history))()
        n = ctypes.c_int()
        status = load().wf_multi_solve(self.handle, _host_ptr(dh), 0, out.ctypes.data_as(ctypes.c_void_p), 0,
                                       ctypes.byref(st), recs, history, ctypes.byref(n))
        _check(status, ok=(WF_OK, WF_ENOTCONVERGED))
        return out, st.as_dict(), status, [recs[i].as_dict() for i in range(n.value)]

    def close(self):
        if getattr(self, "handle", None):
            load().wf_multi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pol:
    """Owns a wf_pol_t: the joint Wiener filter of (T, Q, U) maps."""

    def __init__(self, nside, lmax, cls, noise, mask_t=None, mask_p=None, opts: Options | None = None):
        self.nside, self.lmax = nside, lmax
        self._cls = np.ascontiguousarray(np.stack(cls), dtype=np.float64)
        self._noise = np.ascontiguousarray(noise, dtype=np.float64)
        self._mt = None if mask_t is None else np.ascontiguousarray(mask_t, dtype=np.uint8)
        self._mp = None if mask_p is None else np.ascontiguousarray(mask_p, dtype=np.uint8)
        h = ctypes.c_void_p()
        _check(load().wf_pol_create(nside, lmax, _host_ptr(self._cls), _host_ptr(self._noise), _host_ptr(self._mt),
                                    _host_ptr(self._mp), ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(h)))
        self.handle = h

    @property
    def nalm(self):
        return (self.lmax + 1) * (self.lmax + 2) // 2

    def alm2map(self, alm_dev: int, map_dev: int):
        _check(load().wf_pol_alm2map(self.handle, ctypes.c_void_p(alm_dev), ctypes.c_void_p(map_dev)))

    def map2alm(self, map_dev: int, alm_dev: int):
        _check(load().wf_pol_map2alm(self.handle, ctypes.c_void_p(map_dev), ctypes.c_void_p(alm_dev)))

    def solve(self, d, history=0):
        """d: [3][Npix] host (T, Q, U). Returns (alm [3][nalm], stats, status, records)."""
        dh = np.ascontiguousarray(d, dtype=np.float64)
        out = np.empty((3, self.nalm), dtype=np.complex128)
        st = Stats()
        recs = (IterRecord * max(1, history))()
        n = ctypes.c_int()
        status = load().wf_pol_solve(self.handle, _host_ptr(dh), 0, out.ctypes.data_as(ctypes.c_void_p), 0,
                                     ctypes.byref(st), recs, history, ctypes.byref(n))
        _check(status, ok=(WF_OK, WF_ENOTCONVERGED))
        return out, st.as_dict(), status, [recs[i].as_dict() for i in range(n.value)]

    def close(self):
        if getattr(self, "handle", None):
            load().wf_pol_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns a wf_server_t (continuous batching of solve requests)."""

    def __init__(self, hbm_budget_bytes=0, max_batch=16):
        h = ctypes.c_void_p()
        _check(load().wf_server_create(hbm_budget_bytes, max_batch, ctypes.byref(h)))
        self.handle = h
        self._nalm = {}

    def submit(self, nside, lmax, cl, noise_var, mask, d, tol):
        t = ctypes.c_uint64()
        cl = np.ascontiguousarray(cl, dtype=np.float64)
        nv = np.ascontiguousarray(noise_var, dtype=np.float64)
        mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        dd = np.ascontiguousarray(d, dtype=np.float64)
        _check(load().wf_submit(self.handle, nside, lmax, _host_ptr(cl), _host_ptr(nv), _host_ptr(mk), _host_ptr(dd),
                                float(tol), ctypes.byref(t)))
        self._nalm[t.value] = (lmax + 1) * (lmax + 2) // 2
        return t.value

    def poll(self, ticket):
        """Returns None while running, else (alm, stats, status)."""
        done = ctypes.c_int()
        out = np.empty(self._nalm.get(ticket, 1), dtype=np.complex128)
        st = Stats()
        status = load().wf_poll(self.handle, ticket, ctypes.byref(done), out.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(st))
        if not done.value:
            _check(status, ok=(WF_OK, WF_EBUSY))
            return None
        self._nalm.pop(ticket, None)
        _check(status, ok=(WF_OK, WF_ENOTCONVERGED, WF_ECANCELLED))
        return (None if status == WF_ECANCELLED else out), st.as_dict(), status

    def cancel(self, ticket):
        """Cancel a request; returns the status (WF_OK: recorded, WF_EINVAL: it had already
        finished, WF_ENOTFOUND: unknown ticket). Raises on other errors."""
        return _check(load().wf_cancel(self.handle, ticket), ok=(WF_OK, WF_EINVAL, WF_ENOTFOUND))

    def warm(self, nside, lmax, precision):
        """Make a shape resident (WF_PREC_MIXED: its batched engine; WF_PREC_FP64: one pooled plan)."""
        _check(load().wf_server_warm(self.handle, nside, lmax, precision))

    def drain(self, timeout_ms=600000):
        _check(load().wf_server_drain(self.handle, timeout_ms))

    def stats(self):
        p50, p99, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(load().wf_server_stats(self.handle, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n)))
        return dict(p50_ms=p50.value, p99_ms=p99.value, completed=n.value)

    def close(self):
        if getattr(self, "handle", None):
            load().wf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
