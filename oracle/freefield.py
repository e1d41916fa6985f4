"""Free (unit-link) Wilson fermions on a periodic L^3 x T lattice, in closed form.

Wilson-Dirac operator with unit links (Wilson parameter 1, bare mass m):

  (D psi)(x) = (m + 4) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) psi(x + mu) + (1 + gamma_mu) psi(x - mu) ].

In momentum space D(p) = M(p) + i sum_mu gamma_mu sin p_mu with
M(p) = m + sum_mu (1 - cos p_mu), hence

  S(p) = D(p)^{-1} = (M(p) - i sum_mu gamma_mu sin p_mu) / (M(p)^2 + sum_mu sin^2 p_mu),
  S(x) = (1/V) sum_p e^{i p.x} S(p),        G(x, y) = S(x - y),

periodic in all four directions, so -x wraps without a sign.  Arrays are indexed
[t][z][y][x][spin][spin]; colour is the identity (or a gauge rotation, below).
"""
import numpy as np


def wilson_propagator(L: int, T: int, m: float, gammas) -> np.ndarray:
    """Spin part of the free propagator S(x), complex128 [T][L][L][L][4][4]."""
    pt = 2 * np.pi * np.fft.fftfreq(T) * 1.0
    ps = 2 * np.pi * np.fft.fftfreq(L) * 1.0
    P4, PZ, PY, PX = np.meshgrid(pt, ps, ps, ps, indexing="ij")
    mom = [PX, PY, PZ, P4]                                    # mu = 1, 2, 3, 4 -> x, y, z, t
    M = m + sum(1 - np.cos(p) for p in mom)
    den = M ** 2 + sum(np.sin(p) ** 2 for p in mom)
    Sp = M[..., None, None] * np.eye(4)
    for mu in range(4):
        Sp = Sp - 1j * np.sin(mom[mu])[..., None, None] * gammas[mu]
    Sp = Sp / den[..., None, None]
    return np.fft.ifftn(Sp, axes=(0, 1, 2, 3))                # (1/V) sum_p e^{ipx} S(p)


def apply_wilson(psi: np.ndarray, m: float, gammas) -> np.ndarray:
    """Hopping-stencil Wilson operator on a field psi[t][z][y][x][4][...] (any trailing
    columns), unit links, periodic boundaries."""
    out = (m + 4.0) * psi
    one = np.eye(4)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}                           # mu -> array axis (x, y, z, t)
    for mu in range(4):
        ax = axes[mu]
        fwd = np.roll(psi, -1, axis=ax)                        # psi(x + mu)
        bwd = np.roll(psi, +1, axis=ax)                        # psi(x - mu)
        out = out - 0.5 * (_spin_mul(one - gammas[mu], fwd) + _spin_mul(one + gammas[mu], bwd))
    return out


def _spin_mul(m4, f):
    """Apply a 4x4 spin matrix to axis 4 of f[t][z][y][x][4][...]."""
    return np.moveaxis(np.tensordot(m4, f, axes=([1], [4])), 0, 4)


def random_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-like random SU(3) matrices (QR of a complex Gaussian, phase-fixed)."""
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


def full_propagator(Sspin_x: np.ndarray, Om_x: np.ndarray, Om_y: np.ndarray) -> np.ndarray:
    """12x12 matrices G(x, y) = S_spin(x - y) (x) Omega(x) Omega(y)^dagger for stacks
    of spin blocks [..., 4, 4] and colour rotations [..., 3, 3]."""
    col = Om_x @ np.conj(np.swapaxes(Om_y, -1, -2))
    return np.einsum("...ab,...cd->...acbd", Sspin_x, col).reshape(Sspin_x.shape[:-2] + (12, 12))
