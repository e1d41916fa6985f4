"""Parity of the mixed-precision path (FP32 contraction, split-FP16 tcgen05 projection,
FP64 reduction) against the FP64 oracle: per-correlator relative error < 1e-6."""
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


def report(name, err):
    print(f"{name}: max per-correlator relative error {err:.3e}")
    return err


@pytest.fixture(scope="module")
def c1():
    from oracle.momenta import momenta
    return CS.Case(4, 8, 4, momenta(3, 1), seed=1000)


def test_insertion_c1(ctx, c1):
    got = ctx.insertion(dev(c1.S), dev(c1.psi), 0, 4, c1.r, c1.k, prec="mixed").cpu().numpy()
    ctx.sync()
    assert report("ins c1", CS.block_err(got, c1.ref_insertion(0, 4), 2)) < CS.MIXED_TOL


def test_spectator_meson_c1(ctx, c1):
    got = ctx.spectator(dev(c1.S), dev(c1.eta(4)), 4, c1.r, c1.k, prec="mixed").cpu().numpy()
    ctx.sync()
    assert report("spec c1", CS.block_err(got, c1.ref_spectator_meson(4), 1)) < CS.MIXED_TOL


@pytest.mark.parametrize("L,n_r,n2max,r,dtype", [
    (5, 1, 0, (0, 0, 0, 0), np.complex128),      # nq = 1, n_r = 1 (half-empty column tile), V3 = 125
    (3, 3, 3, (2, 1, 1, 0), np.complex128),      # odd n_r, source off the origin
    (6, 2, 2, (5, 0, 3, 0), np.complex64),       # complex64 storage
    (6, 2, 16, (1, 2, 3, 0), np.complex128),     # 257 momenta: three momentum chunks
])
def test_edges(ctx, L, n_r, n2max, r, dtype):
    from oracle.momenta import momenta
    c = CS.Case(L, 4, n_r, momenta(n2max), seed=1400 + L, r=r, dtype=dtype)
    gi = ctx.insertion(dev(c.S), dev(c.psi), 2, 5, c.r, c.k, prec="mixed").cpu().numpy()
    gs = ctx.spectator(dev(c.S), dev(c.eta(3)), 3, c.r, c.k, prec="mixed").cpu().numpy()
    ctx.sync()
    assert report(f"ins L={L}", CS.block_err(gi, c.ref_insertion(2, 5), 2)) < CS.MIXED_TOL
    assert report(f"spec L={L}", CS.block_err(gs, c.ref_spectator_meson(3), 1)) < CS.MIXED_TOL


def test_other_gamma5(ctx):
    from oracle.momenta import momenta
    c = CS.Case(4, 4, 2, momenta(2), seed=1500, r=(1, 1, 1, 0))
    signs = (-1, 1, -1, 1)
    ctx.set_gamma5(signs)
    try:
        gi = ctx.insertion(dev(c.S), dev(c.psi), 1, 2, c.r, c.k, prec="mixed").cpu().numpy()
        gs = ctx.spectator(dev(c.S), dev(c.eta(2)), 2, c.r, c.k, prec="mixed").cpu().numpy()
    finally:
        ctx.set_gamma5((1, 1, -1, -1))
    g5 = CS.g5_matrix(signs)
    assert CS.block_err(gi, c.ref_insertion(1, 2, g5), 2) < CS.MIXED_TOL
    assert CS.block_err(gs, c.ref_spectator_meson(2, g5), 1) < CS.MIXED_TOL


def test_meson_24c48_sampled_slices(ctx):
    """The benchmark's lattice (24^3, N_r = 16, 93 momenta, complex128) at full size
    on two insertion slices and the sink slice, against the oracle."""
    from oracle.momenta import momenta
    from oracle import contractions as OC
    from paper_1711_02384_gb300 import inputs
    L, n_r, tf = 24, 16, 12
    k = momenta(8)
    S = inputs.propagator(2000, L, 48, slices=range(tf + 1))
    psi = inputs.solutions(2030, L, 48, n_r, slices=range(tf + 1))
    eta = inputs.noise(2033, L, n_r, tf)
    r = np.zeros(4, dtype=np.int32)
    g5 = CS.g5_matrix()
    gi = ctx.insertion(dev(S), dev(psi), 0, tf, r, k, prec="mixed").cpu().numpy()
    gs = ctx.spectator(dev(S), dev(eta), tf, r, k, prec="mixed").cpu().numpy()
    ctx.sync()
    for t in (0, 7):
        ref = OC.insertion(S[t:t + 1], psi[:, t:t + 1], g5, r[:3], k, L)
        assert report(f"24c48 ins t={t}", CS.block_err(gi[t:t + 1], ref, 2)) < CS.MIXED_TOL
    ref = OC.spectator_meson(S[tf], eta, g5, r[:3], k, L)
    assert report("24c48 spec", CS.block_err(gs, ref, 1)) < CS.MIXED_TOL
