"""All-momenta mode: the momentum projection as a discrete Fourier transform over the
slice (three passes of L-point sums) gives the direct sums of Eqs. 9 and 10 for every
momentum, gathered in any requested order with the source phase, against the oracle:
in FP64 within 1e-12, and in the mixed path's FP32 transform within 1e-6."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1711_02384_gb300 import lhc
    c = lhc.Context(0)
    yield c
    c.sync()
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _all_momenta(L, seed):
    lo = -(L // 2)
    ks = np.array([(x, y, z) for z in range(lo, lo + L) for y in range(lo, lo + L) for x in range(lo, lo + L)])
    return ks[np.random.default_rng(seed).permutation(len(ks))]


@pytest.mark.parametrize("prec,mode", [("fp64", "auto"), ("mixed", "auto"), ("mixed", "dft")])
def test_all_momenta(ctx, prec, mode):
    """Every momentum of a 6^3 slice, shuffled: both precisions switch to the transform by
    default (nq >= L^3/2); FP64 within 1e-12, the mixed path's FP32 transform within 1e-6."""
    c = CS.Case(6, 4, 2, _all_momenta(6, 1), seed=2400, r=(1, 4, 2, 0))
    ctx.set_projection(mode)
    try:
        gi = ctx.insertion(dev(c.S), dev(c.psi), 1, 2, c.r, c.k, prec=prec).cpu().numpy()
        gs = ctx.spectator(dev(c.S), dev(c.eta(3)), 3, c.r, c.k, prec=prec).cpu().numpy()
        ctx.sync()
    finally:
        ctx.set_projection("auto")
    tol = CS.FP64_TOL if prec == "fp64" else CS.MIXED_TOL
    assert CS.block_err(gi, c.ref_insertion(1, 2), 2) < tol
    assert CS.block_err(gs, c.ref_spectator_meson(3), 1) < tol


@pytest.mark.parametrize("L,dtype,prec", [(5, np.complex128, "fp64"), (4, np.complex64, "fp64"),
                                          (5, np.complex128, "mixed"), (4, np.complex64, "mixed")])
def test_forced_dft_any_list(ctx, L, dtype, prec):
    """A short list with duplicates, negative and out-of-range components on an odd and
    an even lattice, complex64 inputs too; meson and baryon spectators and insertion, in
    both precisions."""
    from oracle.momenta import momenta
    k = np.concatenate([momenta(2), [[7, -3, 0], [0, 0, 0], [-1, 2, 5]]])
    c = CS.Case(L, 4, 2, k, seed=2410 + L, r=(2, 0, 1, 0), dtype=dtype)
    ctx.set_projection("dft")
    try:
        gi = ctx.insertion(dev(c.S), dev(c.psi), 0, 3, c.r, c.k, prec=prec).cpu().numpy()
        gs = ctx.spectator(dev(c.S), dev(c.eta(2)), 2, c.r, c.k, prec=prec).cpu().numpy()
        gb = ctx.spectator(dev(c.S), dev(c.eta(2)), 2, c.r, c.k, prec=prec, GB=dev(c.SB)).cpu().numpy()
        ctx.sync()
    finally:
        ctx.set_projection("auto")
    # the FP64 transform of complex64 inputs is exact FP64 arithmetic on them; the
    # oracle reads the same complex64 values
    tol = CS.FP64_TOL if prec == "fp64" else CS.MIXED_TOL
    assert CS.block_err(gi, c.ref_insertion(0, 3), 2) < tol
    assert CS.block_err(gs, c.ref_spectator_meson(2), 1) < tol
    assert CS.block_err(gb, c.ref_spectator_baryon(2), 1) < tol


def test_dft_equals_gemm(ctx):
    """The two projections of the same call agree to FP64 rounding."""
    c = CS.Case(8, 2, 3, _all_momenta(8, 2)[:300], seed=2420, r=(3, 3, 7, 0))
    out = {}
    for mode in ("gemm", "dft"):
        ctx.set_projection(mode)
        out[mode] = ctx.insertion(dev(c.S), dev(c.psi), 0, 1, c.r, c.k, prec="fp64").cpu().numpy()
    ctx.set_projection("auto")
    ctx.sync()
    assert CS.block_err(out["dft"], out["gemm"], 2) < CS.FP64_TOL


def test_mixed_dft_against_fp64_at_16(ctx):
    """The mixed path's FP32 transform on every momentum of a 16^3 slice, complex128
    inputs, 4 noises: within 1e-6 per correlator of the FP64 transform of the same call
    (which the tests above pin to the oracle)."""
    c = CS.Case(16, 2, 4, _all_momenta(16, 3), seed=2430, r=(5, 9, 13, 0))
    ctx.set_projection("dft")
    try:
        f = ctx.insertion(dev(c.S), dev(c.psi), 0, 1, c.r, c.k, prec="fp64").cpu().numpy()
        m = ctx.insertion(dev(c.S), dev(c.psi), 0, 1, c.r, c.k, prec="mixed").cpu().numpy()
        ctx.sync()
    finally:
        ctx.set_projection("auto")
    assert CS.block_err(m, f, 2) < CS.MIXED_TOL
