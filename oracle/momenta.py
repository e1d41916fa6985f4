"""Momentum sets and Fourier phases (Sec. 3; Eqs. 9 and 10).

Momenta are p = 2*pi*k/L with integer k (Sec. 3, where the sink and insertion
momentum ranges "k^2 = 0..8" are quoted with 93 vectors each).  The set for a
cutoff is every k in Z^3 with |k|^2 <= n2max and, if given, |k_j| <= cmax.
The order (not fixed by the paper) is ascending (|k|^2, kx, ky, kz).

The phase of site x for momentum k and source r is
exp(sign * 2*pi*i * ((k . (x - r)) mod L) / L): sign = -1 for the spectator
(Eq. 9) and +1 for the insertion (Eq. 10); the shift x -> x - r for a source
away from the origin is the one the paper states after Eq. 10.
"""
import numpy as np


def momenta(n2max: int, cmax: int | None = None) -> np.ndarray:
    """All integer k with |k|^2 <= n2max (and |k_j| <= cmax): int array [nq][3]."""
    c = int(np.floor(np.sqrt(n2max))) if cmax is None else int(cmax)
    out = []
    for kx in range(-c, c + 1):
        for ky in range(-c, c + 1):
            for kz in range(-c, c + 1):
                n2 = kx * kx + ky * ky + kz * kz
                if n2 <= n2max:
                    out.append((n2, kx, ky, kz))
    out.sort()
    return np.array([o[1:] for o in out], dtype=np.int64).reshape(-1, 3)


def site_coords(L: int) -> np.ndarray:
    """Coordinates (x, y, z) of the L^3 sites in the order site = (z*L + y)*L + x."""
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return np.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], axis=1)


def phases(L: int, k: np.ndarray, r3, sign: int) -> np.ndarray:
    """P[q, site] = exp(sign * 2 pi i ((k_q . (x - r)) mod L) / L), complex128 [nq][L^3]."""
    xs = site_coords(L) - np.asarray(r3, dtype=np.int64)[None, :]
    m = np.mod(np.asarray(k, dtype=np.int64) @ xs.T, L)          # integer k.(x-r) mod L
    return np.exp(sign * 2j * np.pi * m / L)
