"""The per-correlator error measure of the combine parity tests, on the CPU.

A correlator C[g][p][q] is a scalar (Eqs. 5 and 8).  The measure divides the error of
each one by the largest |C| of its row (fixed g and sink momentum p, all insertion
momenta q).  A mistake planted in one entry of the oracle's result must be caught, also
where one norm over the whole [np x nq] matrix of a Gamma structure would miss it, and a
relative perturbation of every input of the size of FP32 rounding must pass."""
import numpy as np

import _cases as CS
from oracle import contractions as OC


def _parts(seed, np_, nq, n_r, ng, cols):
    rng = np.random.default_rng(seed)
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    wshape = (4, 4) if cols == 192 else (4, 4, 4)
    return c(np_, n_r, cols), c(nq, n_r, 192), c(ng, *wshape), c(ng, 4, 4), c(ng, *wshape)


def test_one_wrong_correlator_is_caught():
    spec, ins, snk, gi, src = _parts(31, 12, 14, 4, 3, 192)
    ref = OC.combine_meson(spec, ins, snk, gi, src)
    g, p, q = 1, 7, 3
    bad = ref.copy()
    bad[g, p, q] += 3e-6 * np.abs(ref[g, p]).max()
    assert CS.corr_err(bad, ref) > CS.MIXED_TOL
    # one norm per Gamma over the whole [np x nq] matrix would have let it through
    assert CS.block_err(bad, ref, 1) < CS.MIXED_TOL
    assert CS.corr_err(ref, ref) == 0.0


def test_one_wrong_baryon_correlator_is_caught():
    spec, ins, snk, gi, src = _parts(32, 5, 6, 2, 2, 3072)
    ref = OC.combine_baryon(spec, ins, snk, gi, src)
    bad = ref.copy()
    bad[1, 4, 2] -= 2e-6j * np.abs(ref[1, 4]).max()
    assert CS.corr_err(bad, ref) > CS.MIXED_TOL


def test_rounding_sized_input_errors_pass():
    """Inputs perturbed by 6e-8 relative (FP32 rounding) move every correlator by well
    under 1e-6 of its row's scale."""
    spec, ins, snk, gi, src = _parts(33, 30, 30, 4, 2, 192)
    rng = np.random.default_rng(34)
    wig = lambda a: a * (1 + 6e-8 * rng.choice([-1.0, 1.0], size=a.shape))
    ref = OC.combine_meson(spec, ins, snk, gi, src)
    got = OC.combine_meson(wig(spec), wig(ins), snk, gi, src)
    assert CS.corr_err(got, ref) < 2e-7
