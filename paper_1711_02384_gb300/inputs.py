"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the three-point method itself: it only draws
random numbers.  Both sides of every parity test (the FP64 CPU oracle and the
CUDA path) receive the very same bits from here.

Generator: Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written here from
its published definition (multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key
increments 0x9E3779B9 / 0xBB67AE85, ten rounds).  Gaussian variates come from
the Box-Muller transform of two uniforms.  Because the generator is keyed by a
counter, any slice of any field can be regenerated on its own.

Counter layout for element pair ``c`` (two complex numbers per Philox call) of
tensor ``tensor_id`` under ``seed``::

    ctr = (c mod 2^32, c div 2^32, tensor_id, 0)      key = (seed mod 2^32, seed div 2^32)

Fields are stored as complex numbers in the layouts of the library interface:

* propagator  S[t][site][12][12]   (row = sink spin*3+colour, column = source)
* solution    psi[noise][t][site][12]
* noise       eta[noise][site][12]  (Z2 x Z2: (+-1 +-1 i)/sqrt(2))

with ``site = (z*L + y)*L + x``.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# tensor ids used by the workloads (seed per workload, tensor id per field)
TID_PROP = 0      # point-to-all propagator S (also G_A for baryons)
TID_PROP_B = 1    # second baryon propagator G_B
TID_PSI = 2       # stochastic solutions psi
TID_ETA = 3       # Z2 x Z2 noise eta


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ``ctr``: uint array [..., 4] of 32-bit words; ``key``: uint array [..., 2].
    Returns uint32 array [..., 4].
    """
    c = [np.asarray(ctr[..., j], dtype=np.uint64) & _MASK for j in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & _MASK
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def _raw_words(seed: int, tensor_id: int, pair_index: np.ndarray) -> np.ndarray:
    """Four uint32 words for each pair index (uint64 array)."""
    pair_index = np.asarray(pair_index, dtype=np.uint64)
    ctr = np.empty(pair_index.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = pair_index & _MASK
    ctr[..., 1] = pair_index >> _S32
    ctr[..., 2] = np.uint64(tensor_id)
    ctr[..., 3] = 0
    key = np.empty(pair_index.shape + (2,), dtype=np.uint64)
    key[..., 0] = np.uint64(seed) & _MASK
    key[..., 1] = np.uint64(seed) >> _S32
    return philox4x32_10(ctr, key)


def _box_muller(w: np.ndarray) -> np.ndarray:
    """uint32 words [..., 4] -> complex128 [..., 2], real and imaginary parts N(0, 1)."""
    w = w.astype(np.float64)
    u1a = (w[..., 0] + 1.0) * 2.0**-32      # (0, 1]
    u2a = w[..., 1] * 2.0**-32              # [0, 1)
    u1b = (w[..., 2] + 1.0) * 2.0**-32
    u2b = w[..., 3] * 2.0**-32
    ra = np.sqrt(-2.0 * np.log(u1a))
    rb = np.sqrt(-2.0 * np.log(u1b))
    out = np.empty(w.shape[:-1] + (2,), dtype=np.complex128)
    out[..., 0] = ra * np.cos(2.0 * np.pi * u2a) + 1j * ra * np.sin(2.0 * np.pi * u2a)
    out[..., 1] = rb * np.cos(2.0 * np.pi * u2b) + 1j * rb * np.sin(2.0 * np.pi * u2b)
    return out


def gaussian_rows(seed: int, tensor_id: int, rows: np.ndarray, ncomp: int) -> np.ndarray:
    """Complex Gaussian rows: result[j, :] is row ``rows[j]`` of a field whose rows
    hold ``ncomp`` (even) complex numbers.  Rows are independent of each other, so
    a sub-block of a large field can be produced without the rest."""
    assert ncomp % 2 == 0
    rows = np.asarray(rows, dtype=np.uint64).reshape(-1)
    npair = ncomp // 2
    pair = rows[:, None] * np.uint64(npair) + np.arange(npair, dtype=np.uint64)[None, :]
    return _box_muller(_raw_words(seed, tensor_id, pair)).reshape(rows.size, ncomp)


def z2z2_rows(seed: int, tensor_id: int, rows: np.ndarray, ncomp: int) -> np.ndarray:
    """Z2 x Z2 noise rows, entries (+-1 +-1 i)/sqrt(2) (unit modulus)."""
    assert ncomp % 2 == 0
    rows = np.asarray(rows, dtype=np.uint64).reshape(-1)
    npair = ncomp // 2
    pair = rows[:, None] * np.uint64(npair) + np.arange(npair, dtype=np.uint64)[None, :]
    w = _raw_words(seed, tensor_id, pair)                 # [rows, npair, 4]
    bits = w[..., :2]                                      # one word per complex entry
    re = np.where(bits & 1, -1.0, 1.0)
    im = np.where(bits & 2, -1.0, 1.0)
    return ((re + 1j * im) / np.sqrt(2.0)).reshape(rows.size, ncomp)


# --------------------------------------------------------------------------
# whole fields in the interface layouts
# --------------------------------------------------------------------------

def propagator(seed: int, L: int, T: int, slices=None, tensor_id: int = TID_PROP,
               decay: float = 0.0, t0: int = 0) -> np.ndarray:
    """Seeded Gaussian point-to-all propagator, complex128 [len(slices)][L^3][12][12].

    ``decay`` > 0 multiplies slice t by exp(-decay*|t - t0|) (the decaying
    variant that exposes dynamic-range problems of reduced precisions)."""
    V3 = L ** 3
    slices = list(range(T)) if slices is None else [int(t) % T for t in slices]
    out = np.empty((len(slices), V3, 12, 12), dtype=np.complex128)
    for j, t in enumerate(slices):
        rows = np.arange(V3, dtype=np.uint64) + np.uint64(t * V3)
        out[j] = gaussian_rows(seed, tensor_id, rows, 144).reshape(V3, 12, 12)
        if decay:
            out[j] *= np.exp(-decay * abs(t - t0))
    return out


def solutions(seed: int, L: int, T: int, n_r: int, slices=None,
              tensor_id: int = TID_PSI) -> np.ndarray:
    """Seeded Gaussian stochastic solutions psi, complex128 [n_r][len(slices)][L^3][12]."""
    V3 = L ** 3
    slices = list(range(T)) if slices is None else [int(t) % T for t in slices]
    out = np.empty((n_r, len(slices), V3, 12), dtype=np.complex128)
    for i in range(n_r):
        for j, t in enumerate(slices):
            rows = np.arange(V3, dtype=np.uint64) + np.uint64((i * T + t) * V3)
            out[i, j] = gaussian_rows(seed, tensor_id, rows, 12)
    return out


def noise(seed: int, L: int, n_r: int, t_sink: int = 0, tensor_id: int = TID_ETA) -> np.ndarray:
    """Z2 x Z2 noise on one sink timeslice, complex128 [n_r][L^3][12]."""
    V3 = L ** 3
    out = np.empty((n_r, V3, 12), dtype=np.complex128)
    for i in range(n_r):
        rows = np.arange(V3, dtype=np.uint64) + np.uint64((i * 4096 + t_sink) * V3)
        out[i] = z2z2_rows(seed, tensor_id, rows, 12)
    return out


def gaussian_array(seed: int, tensor_id: int, shape) -> np.ndarray:
    """Any-shaped complex Gaussian array (used for small test matrices such as
    random Gamma structures)."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    m = n + (n % 2)
    flat = gaussian_rows(seed, tensor_id, np.arange(1, dtype=np.uint64), m).reshape(-1)
    return flat[:n].reshape(shape)


def source_positions(seed: int, L: int, T: int, n: int) -> np.ndarray:
    """``n`` seeded source positions r = (x, y, z, t) (int array [n][4])."""
    w = _raw_words(seed, 7, np.arange(n, dtype=np.uint64))
    out = np.empty((n, 4), dtype=np.int64)
    out[:, 0] = w[:, 0] % L
    out[:, 1] = w[:, 1] % L
    out[:, 2] = w[:, 2] % L
    out[:, 3] = w[:, 3] % T
    return out


def dirac_matrices() -> np.ndarray:
    """Euclidean Dirac matrices gamma_1..gamma_4 in a chiral basis, complex128 [4][4][4]:
    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0, 1], [1, 0]], Hermitian,
    with gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1) (the library's default
    gamma5).  Input data for the benchmark's Gamma structures."""
    sig = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]),
           np.array([[1, 0], [0, -1]], dtype=complex)]
    z, one = np.zeros((2, 2), dtype=complex), np.eye(2, dtype=complex)
    g = [np.block([[z, -1j * sk], [1j * sk, z]]) for sk in sig] + [np.block([[z, one], [one, z]])]
    return np.array(g)


def dirac_structures() -> np.ndarray:
    """The 16 products gamma_1^n1 gamma_2^n2 gamma_3^n3 gamma_4^n4 (n in {0, 1}), indexed
    by n1 + 2 n2 + 4 n3 + 8 n4, complex128 [16][4][4]."""
    g = dirac_matrices()
    out = np.empty((16, 4, 4), dtype=complex)
    for n in range(16):
        m = np.eye(4, dtype=complex)
        for mu in range(4):
            if (n >> mu) & 1:
                m = m @ g[mu]
        out[n] = m
    return out

