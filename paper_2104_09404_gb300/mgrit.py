"""Thin ctypes binding of libmgrit.so (C ABI declared in include/mgrit.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  The module-level functions carry the C names; ``Solver`` is a
small convenience wrapper taking torch CUDA tensors (torch supplies device
memory and streams).  If libmgrit.so is missing, loading raises: there is no
CPU fallback.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# MGRIT_DEBUG=1 selects the bounds-checked build libmgrit_debug.so
LIB_PATH = os.path.join(PKG, "libmgrit_debug.so" if os.environ.get("MGRIT_DEBUG") == "1"
                        else "libmgrit.so")

OK, EINVAL, ECUDA, ENOMEM, EDIVERGED, ENOTCONV, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
WENO5_SSPRK3, FO_FE, LF_FE = 0, 1, 2
BURGERS, ADVECTION = 0, 1
LF_SPLIT, LF_STATE, ROE = 0, 1, 2
RELAX_F, RELAX_FCF = 0, 1
GUESS_EQ17, GUESS_INJECT = 0, 1
CYCLE_V, CYCLE_F = 0, 1
SEQ_AUTO, SEQ_ONE_CTA, SEQ_CLUSTER, SEQ_GRID = 0, 1, 2, 3
COARSE_REDISC, COARSE_PSI0, COARSE_PSI1 = 0, 1, 2
STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ECUDA: "ECUDA", ENOMEM: "ENOMEM",
                EDIVERGED: "EDIVERGED", ENOTCONV: "ENOTCONV", ETIMEOUT: "ETIMEOUT"}


class mgrit_params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double), ("L", ctypes.c_double), ("relax", ctypes.c_int),
                ("cycle", ctypes.c_int), ("guess", ctypes.c_int), ("numflux", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("coarse", ctypes.c_int), ("chunk_clusters", ctypes.c_int),
                ("seq_stepper", ctypes.c_int)]


class mgrit_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("res_hist", ctypes.c_double * 256), ("t_total_ms", ctypes.c_double),
                ("cell_updates", ctypes.c_double), ("stagnated", ctypes.c_int)]


class mgrit_instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nt", ctypes.c_int), ("m", ctypes.c_int),
                ("levels", ctypes.c_int), ("scheme", ctypes.c_int), ("flux", ctypes.c_int),
                ("T", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    "mgrit_default_params": (None, [ctypes.POINTER(mgrit_params)]),
    "mgrit_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, _I]),
    "mgrit_set_params": (_I, [_P, ctypes.POINTER(mgrit_params)]),
    "mgrit_solve": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(mgrit_stats)]),
    "mgrit_run_cycles": (_I, [_P, _P, _I, _P]),
    "mgrit_copy_cpoints": (_I, [_P, _P, _P]),
    "mgrit_serial_step": (_I, [_P, _P, _P, _I, _P]),
    "mgrit_residual": (_I, [_P, _P, ctypes.POINTER(_D), _P]),
    "mgrit_launch_kernel": (_I, [_P, _I, _I, _I, _P]),
    "mgrit_residual_static": (_I, [_I, _I, _I, _I, _I, _I, _D, _D, _P, _P, _P]),
    "mgrit_fma_probe": (_I, [_I, _I, _I, ctypes.POINTER(_D), _P]),
    "mgrit_cycle_cell_updates": (_D, [_P]),
    "mgrit_query": (_I, [_P, _I]),
    "mgrit_sync_status": (_I, [_P, _P]),
    "mgrit_test_grid_timeout": (_I, [_P, _P]),
    "mgrit_step_vjp": (_I, [_P, _P, _P, _P, _P]),
    "mgrit_adjoint_serial": (_I, [_P, _P, _P, _P, _P]),
    "mgrit_adjoint": (_I, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(mgrit_stats)]),
    "mgrit_adjoint_query": (_I, [_P, _I]),
    "mgrit_last_error": (ctypes.c_char_p, [_P]),
    "mgrit_batch_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(mgrit_instance), _I,
                                ctypes.POINTER(mgrit_params)]),
    "mgrit_batch_run_cycles": (_I, [_P, _P, _I, _P]),
    "mgrit_batch_solve": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "mgrit_batch_autotune": (_I, [_P, _P, _I, _P]),
    "mgrit_batch_cycle_cell_updates": (_D, [_P]),
    "mgrit_batch_launch_relax": (_I, [_P, _I, _P]),
    "mgrit_batch_query": (_I, [_P, _I, _I]),
    "mgrit_batch_copy_cpoints": (_I, [_P, _I, _P, _P]),
    "mgrit_batch_last_error": (ctypes.c_char_p, [_P]),
    "mgrit_batch_destroy": (None, [_P]),
    "mgrit_destroy": (None, [_P]),
}


def load():
    """Load libmgrit.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libmgrit.so not built: run __graft_entry__.build() "
                          "(paper_2104_09404_gb300/build.py); there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def __getattr__(name):
    # module-level access to the C entry points under their own names
    if name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)


class MGRITError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


FMA_FP64, FMA_FP32, FMA_FP32X2 = 0, 1, 2


def fma_probe(kind, iters, blocks_per_sm=8, stream=None):
    """Multiply-add throughput (flop/s) of one SIMT pipe (mgrit_fma_probe)."""
    out = ctypes.c_double(0.0)
    st = load().mgrit_fma_probe(kind, iters, blocks_per_sm, ctypes.byref(out), _stream_handle(stream))
    if st != OK:
        raise MGRITError(st, "mgrit_fma_probe failed")
    return out.value


class Solver:
    """MGRIT solver for one problem size (wraps one mgrit_ctx)."""

    def __init__(self, nx, nt, m, levels, scheme=WENO5_SSPRK3, flux=BURGERS, **params):
        lib = load()
        h = _P()
        st = lib.mgrit_create(ctypes.byref(h), nx, nt, m, levels, scheme, flux)
        if st != OK:
            raise MGRITError(st, lib.mgrit_last_error(None).decode())
        self._h = h
        self.nx, self.nt, self.m, self.levels = nx, nt, m, levels
        self.scheme, self.flux = scheme, flux
        self.params = mgrit_params()
        lib.mgrit_default_params(ctypes.byref(self.params))
        if params:
            self.set_params(**params)

    def _check(self, st, allowed=(OK,)):
        if st not in allowed:
            raise MGRITError(st, load().mgrit_last_error(self._h).decode())
        return st

    def set_params(self, **kw):
        for k, v in kw.items():
            if not hasattr(self.params, k):
                raise KeyError(k)
            setattr(self.params, k, v)
        self._check(load().mgrit_set_params(self._h, ctypes.byref(self.params)))

    def solve(self, u0, want_uC=True, stream=None):
        """Returns (status, uT, uC or None, stats); status is OK, EDIVERGED or ENOTCONV."""
        import torch
        nC = self.nt // self.m
        uT = torch.empty(self.nx, dtype=torch.float64, device=u0.device)
        uC = torch.empty((nC + 1, self.nx), dtype=torch.float64, device=u0.device) if want_uC else None
        stats = mgrit_stats()
        st = load().mgrit_solve(self._h, _ptr(u0), _ptr(uC), _ptr(uT), _stream_handle(stream),
                                ctypes.byref(stats))
        self._check(st, (OK, EDIVERGED, ENOTCONV))
        return st, uT, uC, stats

    def run_cycles(self, u0, ncycles, stream=None):
        self._check(load().mgrit_run_cycles(self._h, _ptr(u0), ncycles, _stream_handle(stream)))

    def cpoints(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.nt // self.m + 1, self.nx), dtype=torch.float64, device="cuda")
        self._check(load().mgrit_copy_cpoints(self._h, _ptr(out), _stream_handle(stream)))
        return out

    def serial_step(self, u0, nsteps, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(u0)
        self._check(load().mgrit_serial_step(self._h, _ptr(u0), _ptr(out), nsteps,
                                             _stream_handle(stream)))
        return out

    def residual(self, uC, stream=None):
        v = ctypes.c_double(0.0)
        self._check(load().mgrit_residual(self._h, _ptr(uC), ctypes.byref(v), _stream_handle(stream)))
        return v.value

    def launch_kernel(self, which, level, reps=1, stream=None):
        self._check(load().mgrit_launch_kernel(self._h, which, level, reps, _stream_handle(stream)))

    def cycle_cell_updates(self):
        return load().mgrit_cycle_cell_updates(self._h)

    def query(self, what):
        """0: cells per thread, 1: threads per CTA, 2: cluster size of the
        sequential stepper, 3: CTAs of the grid stepper (0: not used),
        100 + l: cluster size of the level-l relaxation and interpolation
        chunks (1: one CTA per chunk; 0 before the first allocating call)."""
        return load().mgrit_query(self._h, what)

    def sync_status(self, stream=None):
        """Synchronise; MGRIT_ETIMEOUT (raised) if a grid-stepper barrier wait
        of an earlier asynchronous call gave up."""
        self._check(load().mgrit_sync_status(self._h, _stream_handle(stream)))

    def test_grid_timeout(self, stream=None):
        """Status of one grid-stepper launch whose first barrier can never
        complete (the bounded wait's test hook): MGRIT_ETIMEOUT expected."""
        return load().mgrit_test_grid_timeout(self._h, _stream_handle(stream))

    # ---- discrete adjoint ----------------------------------------------

    def step_vjp(self, u, lam, out=None, stream=None):
        """Phi'(u)^T lam for one fine step."""
        import torch
        if out is None:
            out = torch.empty_like(lam)
        self._check(load().mgrit_step_vjp(self._h, _ptr(u), _ptr(lam), _ptr(out),
                                          _stream_handle(stream)))
        return out

    def adjoint_serial(self, u0, lamT, out=None, stream=None):
        """dJ/du0 from dJ/du(T) = lamT through nt serial steps (C-point checkpoints)."""
        import torch
        if out is None:
            out = torch.empty_like(lamT)
        self._check(load().mgrit_adjoint_serial(self._h, _ptr(u0), _ptr(lamT), _ptr(out),
                                                _stream_handle(stream)))
        return out

    def adjoint(self, uC, lamT, want_lamC=False, stream=None):
        """Adjoint MGRIT from the forward C-point checkpoints uC ((nt/m+1, nx)).
        Returns (status, lam0, lamC or None, stats)."""
        import torch
        lam0 = torch.empty_like(lamT)
        lamC = torch.empty((self.nt // self.m + 1, self.nx), dtype=torch.float64,
                           device=lamT.device) if want_lamC else None
        stats = mgrit_stats()
        st = load().mgrit_adjoint(self._h, _ptr(uC), _ptr(lamT), _ptr(lam0), _ptr(lamC),
                                  _stream_handle(stream), ctypes.byref(stats))
        self._check(st, (OK, EDIVERGED, ENOTCONV))
        return st, lam0, lamC, stats

    def adjoint_query(self, what):
        """0: cells per thread, 1: threads per CTA of the one-CTA adjoint slab (0: none);
        2: CTAs per cluster of the sequential adjoint chains; 100 + l: CTAs per cluster
        of the adjoint chunks of level l (2 and 100 + l after the first adjoint call)."""
        return load().mgrit_adjoint_query(self._h, what)

    def close(self):
        if getattr(self, "_h", None):
            load().mgrit_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent instances advanced together (wraps one mgrit_batch).
    `instances` is a list of dicts with nx, nt, m, levels, flux, T (and
    optionally scheme); other parameters are shared keyword arguments."""

    def __init__(self, instances, **params):
        lib = load()
        arr = (mgrit_instance * len(instances))()
        for k, d in enumerate(instances):
            arr[k] = mgrit_instance(d["nx"], d["nt"], d["m"], d["levels"],
                                    d.get("scheme", WENO5_SSPRK3), d["flux"], d["T"])
        p = mgrit_params()
        lib.mgrit_default_params(ctypes.byref(p))
        for k, v in params.items():
            setattr(p, k, v)
        h = _P()
        st = lib.mgrit_batch_create(ctypes.byref(h), arr, len(instances), ctypes.byref(p))
        if st != OK:
            raise MGRITError(st, lib.mgrit_last_error(None).decode())
        self._h = h
        self.n = len(instances)
        self.instances = list(instances)

    def _check(self, st):
        if st != OK:
            raise MGRITError(st, load().mgrit_batch_last_error(self._h).decode())

    @staticmethod
    def _ptr_array(tensors):
        arr = (ctypes.c_void_p * len(tensors))()
        for k, t in enumerate(tensors):
            arr[k] = t.data_ptr() if t is not None else None
        return arr

    def run_cycles(self, u0s, ncycles, stream=None):
        self._check(load().mgrit_batch_run_cycles(self._h, self._ptr_array(u0s), ncycles,
                                                  _stream_handle(stream)))

    def autotune(self, u0s, reps=3, stream=None):
        self._check(load().mgrit_batch_autotune(self._h, self._ptr_array(u0s), reps,
                                                _stream_handle(stream)))

    def solve(self, u0s, stream=None):
        """Returns (uT list, status list, iters list, final residual list)."""
        import torch
        uTs = [torch.empty_like(u) for u in u0s]
        st = (ctypes.c_int * self.n)()
        it = (ctypes.c_int * self.n)()
        res = (ctypes.c_double * self.n)()
        self._check(load().mgrit_batch_solve(self._h, self._ptr_array(u0s), self._ptr_array(uTs),
                                             st, it, res, _stream_handle(stream)))
        return uTs, list(st), list(it), list(res)

    def cpoints(self, i, stream=None):
        import torch
        d = self.instances[i]
        out = torch.empty((d["nt"] // d["m"] + 1, d["nx"]), dtype=torch.float64, device="cuda")
        self._check(load().mgrit_batch_copy_cpoints(self._h, i, _ptr(out), _stream_handle(stream)))
        return out

    def cycle_cell_updates(self):
        return load().mgrit_batch_cycle_cell_updates(self._h)

    def launch_relax(self, reps=1, stream=None):
        """Profiling hook: the batched level-0 relaxation, reps times."""
        self._check(load().mgrit_batch_launch_relax(self._h, reps, _stream_handle(stream)))

    def query(self, i, what):
        """Instance i: 0 cells per thread, 1 threads per CTA, 2 levels, 3 slabs
        per CTA (always 1), 4 CTAs per cluster of its coarsest solve (1 = one CTA)."""
        return load().mgrit_batch_query(self._h, i, what)

    def close(self):
        if getattr(self, "_h", None):
            load().mgrit_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class MGRITSolve(torch.autograd.Function):
        """u(T) = MGRIT solve from u0 (to the solver's tolerance); its backward
        pass is dJ/du0 = adjoint MGRIT from the forward C-point checkpoints,
        given dJ/du(T)."""

        @staticmethod
        def forward(ctx, u0, solver):
            st, uT, uC, _ = solver.solve(u0.detach().contiguous())
            if st != OK:
                raise MGRITError(st, "forward MGRIT did not converge")
            ctx.solver = solver
            ctx.save_for_backward(uC)
            return uT

        @staticmethod
        def backward(ctx, gT):
            (uC,) = ctx.saved_tensors
            st, lam0, _, _ = ctx.solver.adjoint(uC, gT.detach().to(torch.float64).contiguous())
            if st != OK:
                raise MGRITError(st, "adjoint MGRIT did not converge")
            return lam0, None

    return MGRITSolve


_MGRITSolve = None


def mgrit_solve(u0, solver):
    """Differentiable u(T) = Phi^nt(u0) through an MGRIT Solver (FP64 CUDA
    tensors, split numerical flux): autograd's backward runs adjoint MGRIT."""
    global _MGRITSolve
    if _MGRITSolve is None:
        _MGRITSolve = _autograd_function()
    return _MGRITSolve.apply(u0, solver)
