"""ctypes wrapper around the oracle's shared library (test infrastructure only)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mgrit_oracle.c")
_LIB = os.path.join(_HERE, "liborc_mgrit.so")
# a prebuilt library to load instead (the mutation tests point this at copies
# of the oracle with a planted mistake); build() leaves it untouched
_LIB_OVERRIDE = os.environ.get("MGRIT_ORACLE_LIB")

SCHEME_WENO5_SSPRK3, SCHEME_FO_FE, SCHEME_LF_FE = 0, 1, 2
FLUX_BURGERS, FLUX_ADVECTION = 0, 1
NUMFLUX_LF_SPLIT, NUMFLUX_LF_STATE, NUMFLUX_ROE = 0, 1, 2
RELAX_F, RELAX_FCF = 0, 1
GUESS_EQ17, GUESS_INJECT = 0, 1
CYCLE_V, CYCLE_F = 0, 1
COARSE_REDISC, COARSE_PSI0, COARSE_PSI1 = 0, 1, 2
OK, EINVAL, EDIVERGED, ENOTCONV = 0, -1, -4, -5

_lib = None


def compile_oracle(src, out):
    """gcc, plain -O2, no FMA contraction (the same bits on x86 and Arm), OpenMP."""
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                           "-shared", src, "-o", out, "-lm"])


def build(force=False):
    """Compile the oracle (compile_oracle) unless it is up to date."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        compile_oracle(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        D = ctypes.c_double
        I = ctypes.c_int
        P = ctypes.c_void_p
        lib.orc_weno5_left.restype = D
        lib.orc_weno5_left.argtypes = [P, P, P, P]
        lib.orc_spatial_op.restype = None
        lib.orc_spatial_op.argtypes = [I, D, I, I, I, P, P]
        lib.orc_step.restype = None
        lib.orc_step.argtypes = [I, D, D, I, I, I, P, P]
        lib.orc_serial.restype = None
        lib.orc_serial.argtypes = [I, D, D, I, I, I, I, P, P, I]
        lib.orc_mgrit.restype = I
        lib.orc_mgrit.argtypes = [I, I, I, I, I, I, I, D, D, I, I, I, I, D, I,
                                  P, P, P, P, P, P, P]
        lib.orc_residual.restype = I
        lib.orc_residual.argtypes = [I, I, I, I, I, I, D, D, P, P]
        lib.orc_vcycles.restype = I
        lib.orc_vcycles.argtypes = [I, I, I, I, I, I, I, D, D, I, I, I, I, I, P, P, P]
        lib.orc_weno5_left_grad.restype = None
        lib.orc_weno5_left_grad.argtypes = [P, P]
        lib.orc_step_vjp.restype = None
        lib.orc_step_vjp.argtypes = [I, D, D, I, I, P, P, P]
        lib.orc_adjoint_serial.restype = None
        lib.orc_adjoint_serial.argtypes = [I, D, D, I, I, I, P, P, P]
        lib.orc_adjoint_mgrit.restype = I
        lib.orc_adjoint_mgrit.argtypes = [I, I, I, I, I, I, D, D, I, I, I, D, I,
                                          P, P, P, P, P, P]
        lib.orc_psi_step.restype = None
        lib.orc_psi_step.argtypes = [I, D, D, I, I, I, P, P]
        lib.orc_num_threads.restype = I
        lib.orc_num_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return _load().orc_num_threads()


def weno5_left(q5):
    """q^-_{i+1/2} from q_{i-2..i+2}; returns (value, p[3], beta[3], omega[3])."""
    q = _f64(q5)
    assert q.shape == (5,)
    p, b, w = np.zeros(3), np.zeros(3), np.zeros(3)
    v = _load().orc_weno5_left(_ptr(q), _ptr(p), _ptr(b), _ptr(w))
    return v, p, b, w


def spatial_op(u, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS, numflux=NUMFLUX_LF_SPLIT,
               Lx=1.0):
    u = _f64(u)
    out = np.zeros_like(u)
    _load().orc_spatial_op(u.size, Lx, scheme, flux, numflux, _ptr(u), _ptr(out))
    return out


def step(u, dt, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS, numflux=NUMFLUX_LF_SPLIT,
         Lx=1.0):
    u = _f64(u)
    out = np.zeros_like(u)
    _load().orc_step(u.size, Lx, dt, scheme, flux, numflux, _ptr(u), _ptr(out))
    return out


def serial(u0, dt, nsteps, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS,
           numflux=NUMFLUX_LF_SPLIT, Lx=1.0, store_all=False):
    u0 = _f64(u0)
    nx = u0.size
    out = np.zeros(((nsteps + 1) if store_all else 1, nx))
    _load().orc_serial(nx, Lx, dt, nsteps, scheme, flux, numflux, _ptr(u0), _ptr(out),
                       1 if store_all else 0)
    return out if store_all else out[0]


def mgrit(u0, nt, m, levels, T, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS,
          numflux=NUMFLUX_LF_SPLIT, relax=RELAX_FCF, guess=GUESS_EQ17, tol=1e-10,
          max_iter=64, Lx=1.0, uC_init=None, want_full=False, cycle=CYCLE_V,
          coarse=COARSE_REDISC):
    """Run the oracle MGRIT V-cycle.  Returns a dict with status, iters,
    res_hist, uC ((nt/m+1, nx)), uT and (optionally) the full trajectory."""
    u0 = _f64(u0)
    nx = u0.size
    nc = nt // m
    uC = np.zeros((nc + 1, nx))
    uT = np.zeros(nx)
    full = np.zeros((nt + 1, nx)) if want_full else None
    hist = np.zeros(max_iter + 2)
    iters = ctypes.c_int(0)
    init = None if uC_init is None else _f64(uC_init)
    st = _load().orc_mgrit(nx, nt, m, levels, scheme, flux, numflux, Lx, T, relax, guess,
                           cycle, coarse, tol, max_iter, _ptr(u0), _ptr(init), _ptr(uC), _ptr(full),
                           _ptr(uT), ctypes.cast(ctypes.pointer(iters), ctypes.c_void_p),
                           _ptr(hist))
    k = iters.value
    out = dict(status=st, iters=k, res_hist=hist[:k + 1].copy(), uC=uC, uT=uT)
    if want_full:
        out["u"] = full
    return out


def residual(uC, nt, m, T, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS,
             numflux=NUMFLUX_LF_SPLIT, Lx=1.0):
    uC = _f64(uC)
    nx = uC.shape[1]
    out = np.zeros(1)
    st = _load().orc_residual(nx, nt, m, scheme, flux, numflux, Lx, T, _ptr(uC), _ptr(out))
    if st != OK:
        raise ValueError("orc_residual: invalid arguments")
    return float(out[0])


def vcycles(u0, nt, m, levels, T, ncycles, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS,
            numflux=NUMFLUX_LF_SPLIT, relax=RELAX_FCF, guess=GUESS_EQ17, Lx=1.0, cycle=CYCLE_V,
            coarse=COARSE_REDISC):
    """Exactly ncycles cycles (no stopping test); returns (uC, res_hist)."""
    u0 = _f64(u0)
    nx = u0.size
    uC = np.zeros((nt // m + 1, nx))
    hist = np.zeros(max(ncycles, 1))
    st = _load().orc_vcycles(nx, nt, m, levels, scheme, flux, numflux, Lx, T, relax, guess,
                             cycle, coarse, ncycles, _ptr(u0), _ptr(uC), _ptr(hist))
    if st != OK:
        raise ValueError("orc_vcycles: invalid arguments")
    return uC, hist[:ncycles]


def weno5_left_grad(q5):
    """d q^-_{i+1/2} / d q_{i-2..i+2}."""
    q = _f64(q5)
    g = np.zeros(5)
    _load().orc_weno5_left_grad(_ptr(q), _ptr(g))
    return g


def step_vjp(u, lam, dt, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS, Lx=1.0):
    """Phi'(u)^T lam for one step (split numerical flux)."""
    u, lam = _f64(u), _f64(lam)
    out = np.zeros_like(u)
    _load().orc_step_vjp(u.size, Lx, dt, scheme, flux, _ptr(u), _ptr(lam), _ptr(out))
    return out


def adjoint_serial(u0, lamT, dt, nsteps, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS, Lx=1.0):
    """dJ/du0 given dJ/du(T) = lamT, through nsteps serial steps."""
    u0, lamT = _f64(u0), _f64(lamT)
    out = np.zeros_like(u0)
    _load().orc_adjoint_serial(u0.size, Lx, dt, nsteps, scheme, flux, _ptr(u0), _ptr(lamT),
                               _ptr(out))
    return out


def adjoint_mgrit(uC, lamT, nt, m, levels, T, scheme=SCHEME_WENO5_SSPRK3, flux=FLUX_BURGERS,
                  relax=RELAX_FCF, guess=GUESS_EQ17, tol=1e-10, max_iter=64, Lx=1.0,
                  cycle=CYCLE_V):
    """Adjoint MGRIT backward in time from the forward C-point checkpoints uC
    ((nt/m+1, nx)).  Returns a dict with status, iters, res_hist, lam0 and
    lamC (row i = lam at forward point m*i)."""
    uC, lamT = _f64(uC), _f64(lamT)
    nx = lamT.size
    lam0 = np.zeros(nx)
    lamC = np.zeros((nt // m + 1, nx))
    hist = np.zeros(max_iter + 2)
    iters = ctypes.c_int(0)
    st = _load().orc_adjoint_mgrit(nx, nt, m, levels, scheme, flux, Lx, T, relax, guess, cycle,
                                   tol, max_iter, _ptr(uC), _ptr(lamT), _ptr(lam0), _ptr(lamC),
                                   ctypes.cast(ctypes.pointer(iters), ctypes.c_void_p),
                                   _ptr(hist))
    k = iters.value
    return dict(status=st, iters=k, res_hist=hist[:k + 1].copy(), lam0=lam0, lamC=lamC)


def psi_step(u, dt, M, order, flux=FLUX_BURGERS, Lx=1.0):
    """Matched coarse step for M fine steps of the classical LF + FE scheme:
    order 0 = Psi0, order 1 = Psi1 (dt is the fine step)."""
    u = _f64(u)
    out = np.zeros_like(u)
    _load().orc_psi_step(u.size, Lx, dt, M, order, flux, _ptr(u), _ptr(out))
    return out
