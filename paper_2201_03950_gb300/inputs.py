"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds input recipes only -- none of the solver's arithmetic -- so
that the CUDA path and the CPU oracle can be fed identical data without sharing
any code.  Everything is drawn with numpy's PCG64 (``default_rng(seed)``), which
gives the same stream on x86_64 and aarch64.

Coefficient recipe (diagonally dominant with margin >= 0.5, b in [0.7, 3.5]):
    a = -0.1 - 0.9 U1,   c = -0.1 - 0.9 U2,   b = |a| + |c| + 0.5 + U3,
    d = 2 U4 - 1,        U_k ~ U[0, 1) independent.
Values are drawn in float64 and rounded once to the requested dtype; the
oracle is then given exactly those rounded values widened back to float64.
"""
from __future__ import annotations

import math

import numpy as np


def dominant_system(shape, seed: int = 0, dtype=np.float32):
    """Return (a, b, c, d) arrays of ``shape`` following the recipe above."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape)) if len(shape) else 1
    u = rng.random((4, n))
    a = -0.1 - 0.9 * u[0]
    c = -0.1 - 0.9 * u[1]
    b = np.abs(a) + np.abs(c) + 0.5 + u[2]
    d = 2.0 * u[3] - 1.0
    return tuple(v.reshape(shape).astype(dtype) for v in (a, b, c, d))


def random_rhs(shape, seed: int = 0, dtype=np.float32):
    rng = np.random.default_rng(seed)
    return (2.0 * rng.random(shape) - 1.0).astype(dtype)


def sine_modes(dims, seed: int = 0, nmodes: int = 3, pmax: int = 16):
    """Draw ``nmodes`` (wave numbers, amplitude) triples for a Dirichlet mesh.

    Wave numbers are drawn from {1..min(pmax, n-2)} per axis and amplitudes
    from U(0.5, 1.5).  Returns a list of (tuple_of_wavenumbers, amplitude)."""
    rng = np.random.default_rng(seed)
    modes = []
    for _ in range(nmodes):
        ks = tuple(int(rng.integers(1, max(2, min(pmax, n - 2) + 1))) for n in dims)
        amp = float(rng.uniform(0.5, 1.5))
        modes.append((ks, amp))
    return modes


def sine_field(dims, modes, dtype=np.float64):
    """Evaluate sum_m amp_m prod_axis sin(pi k_axis i / (n_axis - 1)) on the
    column-major mesh ``dims`` (dims[0] contiguous); returns a flat array in
    that element order.  Boundary nodes (i = 0, n-1) are exactly zero."""
    total = np.zeros(tuple(reversed(dims)), dtype=np.float64)
    for ks, amp in modes:
        term = np.array(amp, dtype=np.float64)
        for axis, (n, k) in enumerate(zip(dims, ks)):
            i = np.arange(n, dtype=np.float64)
            s = np.sin(math.pi * k * i / (n - 1))
            s[0] = 0.0
            s[-1] = 0.0
            shape = [1] * len(dims)
            shape[len(dims) - 1 - axis] = n
            term = term * s.reshape(shape)
        total = total + term
    return total.reshape(-1).astype(dtype)


def loguniform_lengths(nsys: int, lo: int, hi: int, seed: int = 0):
    """System lengths L_k = round(exp(ln lo + U ln(hi/lo))), as int64."""
    rng = np.random.default_rng(seed)
    u = rng.random(nsys)
    lengths = np.rint(np.exp(math.log(lo) + u * math.log(hi / lo))).astype(np.int64)
    return np.clip(lengths, lo, hi)


def diffusivity_field(dims, seed: int = 0, sigma: float = 0.3, passes: int = 3,
                      dtype=np.float64):
    """Positive diffusivity field kappa = exp(N(0, sigma^2)) per node, smoothed
    by ``passes`` passes of a 3x3 box filter (edge nodes replicated), flat in
    column-major order (x fastest)."""
    nx, ny = int(dims[0]), int(dims[1])
    rng = np.random.default_rng(seed)
    k = np.exp(rng.normal(0.0, sigma, (ny, nx)))
    for _ in range(passes):
        p = np.pad(k, 1, mode="edge")
        k = sum(p[1 + dy: 1 + dy + ny, 1 + dx: 1 + dx + nx]
                for dy in (-1, 0, 1) for dx in (-1, 0, 1)) / 9.0
    return k.reshape(-1).astype(dtype)


def target_field(dims, seed: int = 0, dtype=np.float64):
    """Seeded smooth target field: a sum of sine eigenmodes (zero on the
    boundary) plus small uniform noise on the interior."""
    rng = np.random.default_rng(seed + 7919)
    t = sine_field(dims, sine_modes(dims, seed=seed + 1), dtype=np.float64)
    nx, ny = int(dims[0]), int(dims[1])
    noise = rng.uniform(-0.05, 0.05, (ny, nx))
    noise[0, :] = noise[-1, :] = 0.0
    noise[:, 0] = noise[:, -1] = 0.0
    return (t + noise.reshape(-1)).astype(dtype)
