"""Shared helpers of the GPU parity tests: seeded inputs, oracle references and
the per-correlator error measure.

Error measures (the paper fixes none):

* spectator and insertion parts: a block is one (slice, momentum) over all open
  spin-colour components and all noises; its error is ||x_gpu - x_ref||_2 / ||x_ref||_2,
  and a test reports the maximum over blocks (``block_err``);
* correlators of the combine: each scalar C[..][p][q] is checked on its own.  Its
  error is |C_gpu - C_ref| divided by the largest |C_ref| of its row (the same
  leading indices and sink momentum p, all insertion momenta q) (``corr_err``).  A
  single wrong (p, q) entry therefore fails even where one norm over the whole
  [np x nq] matrix would hide it, and the scale does not vanish where the terms of one
  correlator happen to cancel.
"""
import numpy as np

from oracle import contractions as OC
from oracle import gamma as OG
from paper_1711_02384_gb300 import inputs

FP64_TOL = 1e-12
MIXED_TOL = 1e-6


def g5_matrix(signs=(1, 1, -1, -1)):
    return np.diag(np.asarray(signs, dtype=float)).astype(complex)


def block_err(got, ref, block_axes):
    """max over blocks of ||got - ref|| / ||ref||; blocks are indexed by the leading
    ``block_axes`` axes."""
    got = np.asarray(got).reshape(int(np.prod(ref.shape[:block_axes])), -1)
    ref = np.asarray(ref).reshape(got.shape)
    num = np.linalg.norm(got - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def corr_err(got, ref):
    """max over correlators of |got - ref| / max_q |ref|: the last axis is the insertion
    momentum q, and the scale of a correlator is the largest |ref| of its row."""
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    scale = np.max(np.abs(ref), axis=-1, keepdims=True)
    return float(np.max(np.abs(got - ref) / np.maximum(scale, 1e-300)))


class Case:
    """A seeded meson/baryon workload on an L^3 x T lattice."""

    def __init__(self, L, T, n_r, kset, seed=1000, dtype=np.complex128, r=(0, 0, 0, 0)):
        self.L, self.T, self.n_r, self.k = L, T, n_r, np.asarray(kset, dtype=np.int32)
        self.V3 = L ** 3
        self.seed = seed
        self.r = np.asarray(r, dtype=np.int32)
        self.dtype = dtype
        self.S = inputs.propagator(seed, L, T).astype(dtype)                             # [T][V3][12][12]
        self.SB = inputs.propagator(seed, L, T, tensor_id=inputs.TID_PROP_B).astype(dtype)
        self.psi = inputs.solutions(seed + 2, L, T, n_r).astype(dtype)                   # [n_r][T][V3][12]

    def eta(self, t_sink):
        return inputs.noise(seed=self.seed + 3, L=self.L, n_r=self.n_r, t_sink=t_sink).astype(self.dtype)

    # ---- oracle references (complex128 inputs: the same bits the GPU reads)
    def ref_insertion(self, t_lo, t_hi, g5=None):
        g5 = g5_matrix() if g5 is None else g5
        ts = [t % self.T for t in range(t_lo, t_hi + 1)]
        S = self.S[ts].astype(np.complex128)
        psi = self.psi[:, ts].astype(np.complex128)
        return OC.insertion(S, psi, g5, self.r[:3], self.k, self.L)

    def ref_spectator_meson(self, t_sink, g5=None):
        g5 = g5_matrix() if g5 is None else g5
        return OC.spectator_meson(self.S[t_sink % self.T].astype(np.complex128),
                                  self.eta(t_sink).astype(np.complex128), g5, self.r[:3], self.k, self.L)

    def ref_spectator_baryon(self, t_sink, g5=None):
        g5 = g5_matrix() if g5 is None else g5
        t = t_sink % self.T
        return OC.spectator_baryon(self.S[t].astype(np.complex128), self.SB[t].astype(np.complex128),
                                   self.eta(t_sink).astype(np.complex128), g5, self.r[:3], self.k, self.L)


def random_gammas(seed, ng, shape):
    return inputs.gaussian_array(seed, 11, (ng,) + tuple(shape))


def gamma16():
    return OG.gamma16(OG.chiral())
