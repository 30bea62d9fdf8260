"""Seeded synthetic inputs (charges and positions) for tests and benchmarks.

These generators hold none of the method's arithmetic; the CUDA path and the
oracle both read their output.  Positions are in the centred box of the
paper, x in [-Lx/2, Lx/2), y in [-Ly/2, Ly/2), z in [-Lz/2, Lz/2]; charges
are +-1 with exactly half of each sign, randomly permuted (neutral, Eq. 2.4).
"""
from __future__ import annotations

import numpy as np


def _charges(rng, N):
    q = np.ones(N, dtype=np.float64)
    q[N // 2:] = -1.0
    if N % 2:
        q[-1] = 0.0
    rng.shuffle(q)
    return q


def uniform_neutral(N: int, L, seed: int = 0, dtype=np.float64):
    """N charges +-1 at uniform positions.  With dtype=float32 the positions
    are rounded to float32 before being returned (as dtype), so that every
    consumer sees the same numbers."""
    Lx, Ly, Lz = map(float, L)
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.empty((N, 3), dtype=np.float64)
    r[:, 0] = rng.uniform(-Lx / 2, Lx / 2, N)
    r[:, 1] = rng.uniform(-Ly / 2, Ly / 2, N)
    r[:, 2] = rng.uniform(-Lz / 2, Lz / 2, N)
    q = _charges(rng, N)
    return q.astype(dtype), r.astype(dtype)


def edl_neutral(N: int, L, seed: int = 0, decay: float = 2.0, dtype=np.float64):
    """Electric double layer: N/4 cations with density ~exp(-(z+Lz/2)/decay)
    near the wall z = -Lz/2, N/4 anions ~exp(-(Lz/2-z)/decay) near z = +Lz/2
    (drawn by rejection into the box), and N/4 + N/4 uniform bulk ions."""
    Lx, Ly, Lz = map(float, L)
    rng = np.random.Generator(np.random.PCG64(seed))
    n4 = N // 4

    def wall(n):
        out = np.empty(0)
        while out.size < n:
            d = rng.exponential(decay, 2 * n)
            out = np.concatenate([out, d[d <= Lz]])
        return out[:n]

    zc = -Lz / 2 + wall(n4)
    za = Lz / 2 - wall(n4)
    nb = N - 2 * n4
    zb = rng.uniform(-Lz / 2, Lz / 2, nb)
    z = np.concatenate([zc, za, zb])
    q = np.concatenate([np.ones(n4), -np.ones(n4), _charges(rng, nb)])
    x = rng.uniform(-Lx / 2, Lx / 2, N)
    y = rng.uniform(-Ly / 2, Ly / 2, N)
    perm = rng.permutation(N)
    r = np.column_stack([x, y, z])[perm]
    return q[perm].astype(dtype), r.astype(dtype)


def batched_slabs(nsys: int, seed: int = 0, nmin: int = 500, nmax: int = 50000,
                  density: float = 0.1, amin: float = 0.05, amax: float = 10.0):
    """Independent neutral systems with N log-uniform in [nmin, nmax], aspect
    ratio a = Lz/Lx uniform in [amin, amax] and Lx = Ly chosen for the given
    number density.  Returns a list of (q, r, (Lx, Ly, Lz))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(nsys):
        N = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        N += N % 2
        a = rng.uniform(amin, amax)
        Lx = (N / (density * a)) ** (1.0 / 3.0)
        L = (Lx, Lx, a * Lx)
        q, r = uniform_neutral(N, L, int(rng.integers(1 << 31)))
        out.append((q, r, L))
    return out
