"""Thin ctypes binding of libdmfe.so (include/dmfe.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. Loading fails loudly (OSError) if the library has not been built; there is
no CPU fallback. The functions keep the C names (``dmfe_create`` ...); ``Solver`` wraps
them for numpy arrays and torch device tensors.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DMFE_LIBRARY selects another build of the same ABI, e.g. the bounds-checked
# libdmfe_checked.so next to this file
LIB_PATH = os.environ.get("DMFE_LIBRARY") or os.path.join(_HERE, "libdmfe.so")
CHECKED_LIB_PATH = os.path.join(_HERE, "libdmfe_checked.so")

DMFE_OK = 0
DMFE_ERR_ARG = -1
DMFE_ERR_OOM = -2
DMFE_ERR_NONFINITE = -3
DMFE_ERR_STEP_UNDERFLOW = -4
DMFE_ERR_CAPACITY = -5
DMFE_ERR_CUDA = -6
DMFE_ERR_TIMEOUT = -7
DMFE_ERR_UNSUPPORTED = -8
DMFE_ERR_IO = -9
DMFE_FP64 = 0
DMFE_FP32_COMPENSATED = 1
DMFE_DOUBLE_FLOAT = 2
PRECISIONS = {"fp64": DMFE_FP64, "fp32": DMFE_FP32_COMPENSATED, "df": DMFE_DOUBLE_FLOAT}
DMFE_RK_AUTO = 0
DMFE_RK_DP5 = 1
DMFE_RK_SSPRK104 = 2
INTEGRATORS = {"auto": DMFE_RK_AUTO, "dp5": DMFE_RK_DP5, "ssprk104": DMFE_RK_SSPRK104}
INTERPS = {"lagrange_index": 0, "fh_index": 1, "lagrange_theta": 2, "fh_theta": 3}
DMFE_NS = 10

_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class dmfe_params(ctypes.Structure):
    _fields_ = [("n_terms", _i), ("powers", _ip), ("coefs", _dp), ("T", _d), ("beta0", _d),
                ("L", _i), ("s", _i), ("grid_t_max", _d), ("alpha", _d), ("delta", _d),
                ("history_cap", _i), ("dt0", _d), ("dt_min", _d), ("precision", _i),
                ("sparsify", _i), ("stream", _p), ("integrator", _i), ("rk_switch_dt", _d), ("hi_chunk", _i),
                ("interp", _i), ("fh_d", _i), ("log_r", _i), ("sparsify_every", _i), ("sparsify_passes", _i)]


class dmfe_stats_t(ctypes.Structure):
    _fields_ = [("t", _d), ("dt", _d), ("mu", _d), ("E", _d), ("last_eps", _d),
                ("max_eps_sparse", _d), ("steps_accepted", ctypes.c_longlong),
                ("steps_rejected", ctypes.c_longlong), ("stages", ctypes.c_longlong),
                ("sparsify_passes", ctypes.c_longlong), ("slices_removed", ctypes.c_longlong),
                ("forced_removals", ctypes.c_longlong), ("n_slices", _i), ("status", _i),
                ("L", _i), ("history_cap", _i), ("s", _i), ("precision", _i), ("method", _i),
                ("t_switch", _d), ("rk_switch_dt", _d), ("step_graph", _i), ("bounds_site", _i)]


class dmfe_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", _i), ("slot", _i), ("t_final", _d), ("E", _d), ("mu", _d),
                ("submit_s", _d), ("admit_s", _d), ("done_s", _d), ("steps_accepted", ctypes.c_longlong),
                ("steps_rejected", ctypes.c_longlong)]


class dmfe_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("admitted", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong), ("queued", _i), ("running", _i),
                ("bytes_in_use", ctypes.c_ulonglong), ("hbm_budget", ctypes.c_ulonglong),
                ("batched_steps", ctypes.c_longlong)]


_SIGS = {
    "dmfe_default_params": (None, [ctypes.POINTER(dmfe_params)]),
    "dmfe_strerror": (ctypes.c_char_p, [_i]),
    "dmfe_create": (_i, [ctypes.POINTER(dmfe_params), ctypes.POINTER(_p)]),
    "dmfe_destroy": (None, [_p]),
    "dmfe_grid": (_i, [_p, _dp, _dp, _dp]),
    "dmfe_tables": (_i, [_p, _dp, _dp, _dp]),
    "dmfe_integrate": (_i, [_p, _d, _d]),
    "dmfe_step": (_i, [_p, _i, _d, _d, _p]),
    "dmfe_get_C": (_i, [_p, _i, _dp, _dp, _dp]),
    "dmfe_get_R": (_i, [_p, _i, _dp, _dp, _dp]),
    "dmfe_get_row": (_i, [_p, _dp, _dp, _dp, _dp, _dp]),
    "dmfe_set_history": (_i, [_p, _i, _dp, _dp, _dp, _dp, _dp]),
    "dmfe_get_history": (_i, [_p, _ip, _dp, _dp, _dp, _dp, _dp]),
    "dmfe_history_integrals": (_i, [_p, _d, _dp, _dp, _dp, _dp]),
    "dmfe_history_integrals_dev": (_i, [_p, _d, _p, _p, _p]),
    "dmfe_rhs": (_i, [_p, _d, _dp, _dp, _dp, _dp, _dp, _dp]),
    "dmfe_sparsify": (_i, [_p, _d, _ip]),
    "dmfe_theta_grid": (_i, [_i, _d, _d, _d, _dp, _dp, _dp]),
    "dmfe_stats": (_i, [_p, ctypes.POINTER(dmfe_stats_t)]),
    "dmfe_checkpoint": (_i, [_p, ctypes.c_char_p]),
    "dmfe_restore": (_i, [ctypes.c_char_p, _p, ctypes.POINTER(_p)]),
    "dmfe_sync": (_i, [_p]),
    "dmfe_autotune": (_i, [_p, _ip]),
    "dmfe_batch_create": (_i, [_i, _i, _i, _i, _i, _p, ctypes.POINTER(_p)]),
    "dmfe_batch_destroy": (None, [_p]),
    "dmfe_batch_add": (_i, [_p, ctypes.POINTER(dmfe_params), _d, _d, _ip]),
    "dmfe_batch_remove": (_i, [_p, _i]),
    "dmfe_batch_solver": (_p, [_p, _i]),
    "dmfe_batch_step": (_i, [_p, _i]),
    "dmfe_batch_poll": (_i, [_p, _ip, _dp, _ip]),
    "dmfe_batch_autotune": (_i, [_p, _i, _ip, _dp]),
    "dmfe_footprint": (ctypes.c_ulonglong, [ctypes.POINTER(dmfe_params)]),
    "dmfe_server_start": (_i, [_i, _i, _i, _i, _i, ctypes.c_ulonglong, _i, ctypes.POINTER(_p)]),
    "dmfe_server_submit": (_i, [_p, ctypes.POINTER(dmfe_params), _d, _d, ctypes.POINTER(ctypes.c_longlong)]),
    "dmfe_server_poll": (_i, [_p, ctypes.POINTER(dmfe_result), _i, _ip]),
    "dmfe_server_stats": (_i, [_p, ctypes.POINTER(dmfe_server_stats_t)]),
    "dmfe_server_stop": (_i, [_p]),
    "dmfe_sparsify_select_noalloc": (_i, [_p, _p, _p, _p, _p, _i, _i, _d, _p, _p]),
    "dmfe_fma_rate": (_i, [_i, _dp]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libdmfe.so (raises OSError if it is missing) and declare the signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError("libdmfe.so not built at %s (run __graft_entry__.build())" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class DMFEError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = load().dmfe_strerror(code).decode()
        super().__init__("%s: %s (%d)" % (where, msg, code))


def _check(rc, where):
    if rc != DMFE_OK:
        raise DMFEError(rc, where)
    return rc


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def make_params(coefs, T, L, grid_t_max, s=4, beta0=0.0, alpha=0.0, delta=0.0, history_cap=None, dt0=1e-4,
                dt_min=1e-12, precision="fp64", sparsify=True, stream=None, integrator="auto", switch_dt=0.0,
                hi_chunk=0, interp="lagrange_index", fh_d=3, log_r=False, sparsify_every=0, sparsify_passes=1):
    """A dmfe_params structure; the returned tuple keeps the coefficient arrays alive."""
    lib = load()
    terms = sorted((int(p), float(c)) for p, c in dict(coefs).items())
    pw = (ctypes.c_int * len(terms))(*[p for p, _ in terms])
    cf = (ctypes.c_double * len(terms))(*[c for _, c in terms])
    prm = dmfe_params()
    lib.dmfe_default_params(ctypes.byref(prm))
    prm.n_terms = len(terms)
    prm.powers = ctypes.cast(pw, _ip)
    prm.coefs = ctypes.cast(cf, _dp)
    prm.T, prm.beta0, prm.L, prm.s = T, beta0, L, s
    prm.grid_t_max, prm.alpha, prm.delta = grid_t_max, alpha, delta
    prm.history_cap = int(history_cap) if history_cap else L
    prm.dt0, prm.dt_min = dt0, dt_min
    prm.precision = PRECISIONS[precision]
    prm.sparsify = 1 if sparsify else 0
    prm.stream = stream
    prm.integrator = INTEGRATORS[integrator]
    prm.rk_switch_dt = float(switch_dt)
    prm.hi_chunk = int(hi_chunk)
    prm.interp = INTERPS[interp]
    prm.fh_d = int(fh_d)
    prm.log_r = 1 if log_r else 0
    prm.sparsify_every = int(sparsify_every)
    prm.sparsify_passes = int(sparsify_passes)
    return prm, (pw, cf)


class Batch:
    """A dmfe_batch: many independent solves stepped together (continuous batching)."""

    def __init__(self, max_slots, max_L, max_cap, precision="fp64", s=4, stream=None):
        self._lib = load()
        self.h = _p()
        self.max_slots = max_slots
        _check(self._lib.dmfe_batch_create(max_slots, max_L, max_cap, PRECISIONS[precision], s, stream,
                                           ctypes.byref(self.h)), "dmfe_batch_create")
        self.precision, self.s = precision, s

    def add(self, coefs, T, L, grid_t_max, t_max, tol, **kw):
        prm, keep = make_params(coefs, T, L, grid_t_max, s=self.s, precision=self.precision, **kw)
        slot = _i()
        _check(self._lib.dmfe_batch_add(self.h, ctypes.byref(prm), float(t_max), float(tol), ctypes.byref(slot)),
               "dmfe_batch_add")
        return slot.value

    def remove(self, slot):
        _check(self._lib.dmfe_batch_remove(self.h, int(slot)), "dmfe_batch_remove")

    def solver(self, slot):
        """Non-owning Solver view of a slot (valid until the slot is removed)."""
        h = self._lib.dmfe_batch_solver(self.h, int(slot))
        if not h:
            raise ValueError("slot %d is free" % slot)
        return Solver._from_handle(h, owned=False)

    def step(self, nsteps):
        _check(self._lib.dmfe_batch_step(self.h, int(nsteps)), "dmfe_batch_step")

    def poll(self):
        """(status[max_slots], t[max_slots], running): status 0 running, 1 done, < 0 error, -100 free."""
        st = (ctypes.c_int * self.max_slots)()
        tt = np.empty(self.max_slots)
        run = _i()
        _check(self._lib.dmfe_batch_poll(self.h, ctypes.cast(st, _ip), _ptr(tt), ctypes.byref(run)),
               "dmfe_batch_poll")
        return np.array(st[:], dtype=int), tt, run.value

    def autotune(self, steps=4):
        """dmfe_batch_autotune: (chosen unit size, {candidate: ms per batched step}).
        The timed steps advance the slots; 0 means one unit per output index."""
        c = _i()
        ms = (_d * 5)()
        _check(self._lib.dmfe_batch_autotune(self.h, int(steps), ctypes.byref(c), ctypes.cast(ms, _dp)),
               "dmfe_batch_autotune")
        return c.value, {k: ms[q] for q, k in enumerate((0, 256, 512, 1024, 2048))}

    def run(self, poll_every=16):
        """Step until no slot is running."""
        while True:
            self.step(poll_every)
            _, _, running = self.poll()
            if running == 0:
                return

    def close(self):
        if self.h:
            self._lib.dmfe_batch_destroy(self.h)
            self.h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(coefs, T, L, grid_t_max, **kw):
    """Device bytes a solver with these parameters allocates."""
    prm, keep = make_params(coefs, T, L, grid_t_max, **kw)
    return int(load().dmfe_footprint(ctypes.byref(prm)))


def fma_rate(bits):
    """Measured FP64 (bits = 64) or FP32 (bits = 32) FMA rate of the current device, GFLOP/s."""
    g = _d()
    _check(load().dmfe_fma_rate(int(bits), ctypes.byref(g)), "dmfe_fma_rate")
    return g.value


def theta_grid(L, grid_t_max, alpha=0.0, delta=0.0):
    """(theta, omega, nu) of Eq. (theta) and Sec. 3.4 from the library's host code."""
    theta, omega, nu = np.empty(L), np.empty(L), np.empty(L)
    _check(load().dmfe_theta_grid(int(L), float(grid_t_max), float(alpha), float(delta), _ptr(theta),
                                  _ptr(omega), _ptr(nu)), "dmfe_theta_grid")
    return theta, omega, nu


class Server:
    """dmfe_server: requests admitted by device-memory footprint into a continuously
    stepped batch by a native worker thread."""

    def __init__(self, max_slots, max_L, max_cap, precision="fp64", s=4, hbm_budget=None, steps_per_round=4):
        self._lib = load()
        self.h = _p()
        self.precision, self.s = precision, s
        if hbm_budget is None:
            hbm_budget = 64 << 30
        _check(self._lib.dmfe_server_start(max_slots, max_L, max_cap, PRECISIONS[precision], s, int(hbm_budget),
                                           steps_per_round, ctypes.byref(self.h)), "dmfe_server_start")

    def submit(self, coefs, T, L, grid_t_max, t_max, tol, **kw):
        prm, keep = make_params(coefs, T, L, grid_t_max, s=self.s, precision=self.precision, **kw)
        rid = ctypes.c_longlong()
        _check(self._lib.dmfe_server_submit(self.h, ctypes.byref(prm), float(t_max), float(tol), ctypes.byref(rid)),
               "dmfe_server_submit")
        return rid.value

    def poll(self, max_out=1024):
        buf = (dmfe_result * max_out)()
        n = _i()
        _check(self._lib.dmfe_server_poll(self.h, buf, max_out, ctypes.byref(n)), "dmfe_server_poll")
        return [{f: getattr(buf[k], f) for f, _ in dmfe_result._fields_} for k in range(n.value)]

    def stats(self):
        st = dmfe_server_stats_t()
        _check(self._lib.dmfe_server_stats(self.h, ctypes.byref(st)), "dmfe_server_stats")
        return {f: getattr(st, f) for f, _ in dmfe_server_stats_t._fields_}

    def stop(self):
        if self.h:
            rc = self._lib.dmfe_server_stop(self.h)
            self.h = _p()
            _check(rc, "dmfe_server_stop")

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


class Solver:
    """A dmfe_solver handle. coefs: {power: coefficient} for f(q) = sum c_p q^p."""

    def __init__(self, coefs, T, L, grid_t_max, s=4, beta0=0.0, alpha=0.0, delta=0.0,
                 history_cap=None, dt0=1e-4, dt_min=1e-12, precision="fp64", sparsify=True,
                 stream=None, integrator="auto", switch_dt=0.0, hi_chunk=0, interp="lagrange_index", fh_d=3,
                 log_r=False, sparsify_every=0, sparsify_passes=1):
        """The fields of dmfe_params (include/dmfe.h). precision: "fp64", "df" (double-float)
        or "fp32" (FP32 with compensated sums). integrator: "auto" (Dormand-Prince, then
        SSPRK(10,4) once the step reaches switch_dt; 0 = the stability estimate), "dp5" or
        "ssprk104" (Sec. 3.5). interp: "lagrange_index", "fh_index", "lagrange_theta" or
        "fh_theta" with Floater-Hormann degree fh_d (Sec. 3.3; all but the first FP64 only).
        log_r: interpolate the response history in log R where positive (App. A; FP64).
        sparsify_every, sparsify_passes: a sparsification round also after every P-th
        accepted step (0: only on a full store), and the passes per round (Sec. 3.6)."""
        lib = load()
        self._lib = lib
        self.h = _p()
        self._owned = True
        prm, keep = make_params(coefs, T, L, grid_t_max, s=s, beta0=beta0, alpha=alpha, delta=delta,
                                history_cap=history_cap, dt0=dt0, dt_min=dt_min, precision=precision,
                                sparsify=sparsify, stream=stream, integrator=integrator, switch_dt=switch_dt,
                                hi_chunk=hi_chunk, interp=interp, fh_d=fh_d, log_r=log_r,
                                sparsify_every=sparsify_every, sparsify_passes=sparsify_passes)
        _check(lib.dmfe_create(ctypes.byref(prm), ctypes.byref(self.h)), "dmfe_create")
        self._sizes()

    def _sizes(self):
        st = self.stats()
        self.L, self.cap = st["L"], st["history_cap"]
        th, om, nu = (np.empty(self.L) for _ in range(3))
        _check(self._lib.dmfe_grid(self.h, _ptr(th), _ptr(om), _ptr(nu)), "dmfe_grid")
        self.theta, self.omega, self.nu = th, om, nu

    @classmethod
    def _from_handle(cls, h, owned):
        obj = cls.__new__(cls)
        obj._lib = load()
        obj.h = _p(h)
        obj._owned = owned
        obj._sizes()
        return obj

    @classmethod
    def restore(cls, path, stream=None):
        lib = load()
        obj = cls.__new__(cls)
        obj._lib = lib
        obj.h = _p()
        _check(lib.dmfe_restore(path.encode(), stream, ctypes.byref(obj.h)), "dmfe_restore")
        obj._sizes()
        return obj

    def close(self):
        if self.h and getattr(self, "_owned", True):
            self._lib.dmfe_destroy(self.h)
        self.h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- calls
    def integrate(self, t_max, tol, check=False):
        rc = self._lib.dmfe_integrate(self.h, float(t_max), float(tol))
        if check:
            _check(rc, "dmfe_integrate")
        return rc

    def step(self, nsteps, t_max, tol, stream_ptr=None):
        """Launch nsteps device-driven trial steps without synchronising."""
        _check(self._lib.dmfe_step(self.h, int(nsteps), float(t_max), float(tol),
                                   _p(stream_ptr) if stream_ptr else None), "dmfe_step")

    def tables(self):
        x = [np.empty((self.L, self.L)) for _ in range(3)]
        _check(self._lib.dmfe_tables(self.h, *[_ptr(a) for a in x]), "dmfe_tables")
        return x

    def _two_time(self, fn, t, tp):
        t, tp = np.broadcast_arrays(np.atleast_1d(np.asarray(t, float)), np.atleast_1d(np.asarray(tp, float)))
        t, tp = _f64(t.ravel()), _f64(tp.ravel())
        out = np.empty(t.size)
        _check(fn(self.h, t.size, _ptr(t), _ptr(tp), _ptr(out)), fn.__name__)
        return out

    def get_C(self, t, tp):
        return self._two_time(self._lib.dmfe_get_C, t, tp)

    def get_R(self, t, tp):
        return self._two_time(self._lib.dmfe_get_R, t, tp)

    def get_row(self):
        t, mu, E = _d(), _d(), _d()
        C, R = np.empty(self.L), np.empty(self.L)
        _check(self._lib.dmfe_get_row(self.h, ctypes.byref(t), _ptr(C), _ptr(R), ctypes.byref(mu),
                                      ctypes.byref(E)), "dmfe_get_row")
        return t.value, C, R, mu.value, E.value

    def set_history(self, t, C, dC, R, dR):
        t = _f64(t)
        n = t.size
        arrs = [_f64(a, n * self.L) for a in (C, dC, R, dR)]
        _check(self._lib.dmfe_set_history(self.h, n, _ptr(t), *[_ptr(a) for a in arrs]), "dmfe_set_history")

    def get_history(self):
        n = _i()
        t = np.empty(self.cap)
        arrs = [np.empty((self.cap, self.L)) for _ in range(4)]
        _check(self._lib.dmfe_get_history(self.h, ctypes.byref(n), _ptr(t), *[_ptr(a) for a in arrs]),
               "dmfe_get_history")
        k = n.value
        return (t[:k],) + tuple(a[:k] for a in arrs)

    def history_integrals(self, t, C, R):
        C, R = _f64(C, self.L), _f64(R, self.L)
        S = np.empty((DMFE_NS, self.L))
        mu = _d()
        _check(self._lib.dmfe_history_integrals(self.h, float(t), _ptr(C), _ptr(R), _ptr(S), ctypes.byref(mu)),
               "dmfe_history_integrals")
        return S, mu.value

    def history_integrals_dev(self, t, row_dev_ptr, S_dev_ptr, stream_ptr=None):
        """Device-pointer entry: row_dev [2][L] float64, S_dev [NS][L] float64 (torch data_ptr())."""
        _check(self._lib.dmfe_history_integrals_dev(self.h, float(t), _p(row_dev_ptr), _p(S_dev_ptr),
                                                    _p(stream_ptr) if stream_ptr else None),
               "dmfe_history_integrals_dev")

    def rhs(self, t, C, R):
        C, R = _f64(C, self.L), _f64(R, self.L)
        dC, dR = np.empty(self.L), np.empty(self.L)
        mu, E = _d(), _d()
        _check(self._lib.dmfe_rhs(self.h, float(t), _ptr(C), _ptr(R), _ptr(dC), _ptr(dR), ctypes.byref(mu),
                                  ctypes.byref(E)), "dmfe_rhs")
        return dC, dR, mu.value, E.value

    def sparsify(self, tol):
        """One pass (Sec. 3.6); returns a boolean mask over the slices before the pass."""
        n = self.stats()["n_slices"]
        removed = (ctypes.c_int * self.cap)()
        _check(self._lib.dmfe_sparsify(self.h, float(tol), ctypes.cast(removed, _ip)), "dmfe_sparsify")
        return np.array(removed[:n], dtype=bool)

    def stats(self):
        s = dmfe_stats_t()
        _check(self._lib.dmfe_stats(self.h, ctypes.byref(s)), "dmfe_stats")
        return {name: getattr(s, name) for name, _ in dmfe_stats_t._fields_}

    def checkpoint(self, path):
        _check(self._lib.dmfe_checkpoint(self.h, path.encode()), "dmfe_checkpoint")

    def autotune(self):
        """Pick the fastest work-unit size for this configuration; returns it."""
        c = _i()
        _check(self._lib.dmfe_autotune(self.h, ctypes.byref(c)), "dmfe_autotune")
        return c.value

    def sync(self):
        return self._lib.dmfe_sync(self.h)
