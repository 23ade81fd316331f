"""Seeded synthetic inputs: exact cell averages of analytic initial conditions.

This module holds no part of the MGRIT method's arithmetic; it only turns an
initial condition u0(x) on the periodic domain [0, Lx) into the cell averages
(1/dx) * integral of u0 over cell i, which is the finite-volume unknown of
Sec. 2.1.  Both the CUDA path and the oracle receive the same arrays.

Workloads (the paper's tests use analytic initial conditions, Sec. 4):
  * ``sine_ic``     u0 = offset + amp * sin(2 pi x / Lx)          (0.5 + sin: moving shock)
  * ``fourier_ic``  u0 = offset + sum_k a_k sin(2 pi k x + phi_k), k = 1..K,
                    a_k ~ N(0,1)/k^2, phi_k ~ U[0, 2 pi), drawn in that order
                    from numpy.random.default_rng(seed).
"""
import numpy as np


def _edges(nx, Lx):
    return np.arange(nx + 1, dtype=np.float64) * (Lx / nx)


def sine_ic(nx, offset=0.5, amp=1.0, Lx=1.0):
    """Cell averages of offset + amp * sin(2 pi x / Lx)."""
    x = _edges(nx, Lx)
    dx = Lx / nx
    w = 2.0 * np.pi / Lx
    c = np.cos(w * x)
    return offset + amp * (c[:-1] - c[1:]) / (w * dx)


def fourier_coeffs(seed, K=8):
    """(a, phi) of the random Fourier initial condition for a seed."""
    rng = np.random.default_rng(seed)
    k = np.arange(1, K + 1, dtype=np.float64)
    a = rng.standard_normal(K) / k ** 2
    phi = rng.uniform(0.0, 2.0 * np.pi, K)
    return a, phi


def fourier_ic(nx, seed, K=8, offset=0.5, Lx=1.0):
    """Cell averages of offset + sum_k a_k sin(2 pi k x / Lx + phi_k)."""
    a, phi = fourier_coeffs(seed, K)
    x = _edges(nx, Lx)
    dx = Lx / nx
    u = np.full(nx, offset, dtype=np.float64)
    for kk in range(1, K + 1):
        w = 2.0 * np.pi * kk / Lx
        c = np.cos(w * x + phi[kk - 1])
        u += a[kk - 1] * (c[:-1] - c[1:]) / (w * dx)
    return u


def fourier_breaking_time(seed, K=8, Lx=1.0, samples=1 << 16):
    """Breaking time -1 / min_x u0'(x) of the Fourier initial condition for
    Burgers (inf if u0' >= 0 everywhere), sampled on a fine grid."""
    a, phi = fourier_coeffs(seed, K)
    x = np.arange(samples) * (Lx / samples)
    du = np.zeros_like(x)
    for kk in range(1, K + 1):
        w = 2.0 * np.pi * kk / Lx
        du += a[kk - 1] * w * np.cos(w * x + phi[kk - 1])
    mn = du.min()
    return np.inf if mn >= 0 else -1.0 / mn


def levels_for(nt, m, max_coarse=16):
    """Number of levels when coarsening until at most max_coarse C-points
    remain: 1 + min{k : nt / m^k <= max_coarse}."""
    k, n = 0, nt
    while n > max_coarse:
        if n % m:
            break
        n //= m
        k += 1
    return 1 + k


def batch_workload(seed=0, n=64, m=4, cfl=0.375, K=8):
    """Uneven batch of independent problems: nx drawn from {256, ..., 8192}
    and nt from {1024, ..., 16384} (powers of two, uniform), the first half
    Burgers and the second half linear advection, random Fourier u0 per
    instance (seed * 1000 + i), coarsened until at most 16 C-points remain,
    and dt = cfl * dx / max|u0| (advection: / 1), i.e. T = nt * dt.
    Returns (list of instance dicts, list of u0 arrays)."""
    rng = np.random.default_rng(seed)
    nxs = 2 ** rng.integers(8, 14, size=n)
    nts = 2 ** rng.integers(10, 15, size=n)
    insts, u0s = [], []
    for i in range(n):
        nx, nt = int(nxs[i]), int(nts[i])
        flux = 0 if i < n // 2 else 1
        u0 = fourier_ic(nx, seed=seed * 1000 + i, K=K)
        speed = float(np.abs(u0).max()) if flux == 0 else 1.0
        T = nt * cfl * (1.0 / nx) / speed
        insts.append(dict(nx=nx, nt=nt, m=m, levels=levels_for(nt, m), flux=flux, T=T))
        u0s.append(u0)
    return insts, u0s
