"""Parity of the plain FP64 GPU path against the FP64 oracle (tolerance 1e-12 per
correlator), through the C ABI."""
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
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def c1():
    """4^3 x 8, N_r = 4, 27 momenta in {-1,0,1}^3, t_f = 4, insertion slices 0..4."""
    from oracle.momenta import momenta
    return CS.Case(4, 8, 4, momenta(3, 1), seed=1000)


def test_insertion_c1(ctx, c1):
    got = ctx.insertion(dev(c1.S), dev(c1.psi), 0, 4, c1.r, c1.k, prec="fp64").cpu().numpy()
    ref = c1.ref_insertion(0, 4)
    assert CS.block_err(got, ref, 2) < CS.FP64_TOL


def test_spectator_meson_c1(ctx, c1):
    got = ctx.spectator(dev(c1.S), dev(c1.eta(4)), 4, c1.r, c1.k, prec="fp64").cpu().numpy()
    ref = c1.ref_spectator_meson(4)
    assert CS.block_err(got, ref, 1) < CS.FP64_TOL


def test_spectator_baryon_small(ctx):
    from oracle.momenta import momenta
    c = CS.Case(3, 4, 2, momenta(2), seed=1100, r=(1, 2, 0, 0))
    got = ctx.spectator(dev(c.S), dev(c.eta(1)), 1, c.r, c.k, prec="fp64", GB=dev(c.SB)).cpu().numpy()
    ref = c.ref_spectator_baryon(1)
    assert CS.block_err(got, ref, 1) < CS.FP64_TOL


@pytest.mark.parametrize("L,n_r,kset,r", [
    (5, 1, [[0, 0, 0]], (0, 0, 0, 0)),             # nq = 1, n_r = 1, V3 = 125 (ragged tiles)
    (3, 3, "n2<=3", (2, 1, 1, 0)),                  # source away from the origin
    (6, 2, "n2<=2", (5, 0, 3, 0)),
])
def test_insertion_edges(ctx, L, n_r, kset, r):
    from oracle.momenta import momenta
    k = momenta(3) if kset == "n2<=3" else momenta(2) if kset == "n2<=2" else np.array(kset)
    c = CS.Case(L, 4, n_r, k, seed=1200 + L, r=r)
    got = ctx.insertion(dev(c.S), dev(c.psi), 2, 5, c.r, c.k, prec="fp64").cpu().numpy()   # wraps mod T
    ref = c.ref_insertion(2, 5)
    assert CS.block_err(got, ref, 2) < CS.FP64_TOL


def test_complex64_inputs_and_other_gamma5(ctx):
    from oracle.momenta import momenta
    c = CS.Case(4, 4, 2, momenta(2), seed=1300, dtype=np.complex64, r=(1, 1, 1, 0))
    signs = (-1, 1, -1, 1)
    ctx.set_gamma5(signs)
    try:
        got_i = ctx.insertion(dev(c.S), dev(c.psi), 1, 2, c.r, c.k, prec="fp64").cpu().numpy()
        got_s = ctx.spectator(dev(c.S), dev(c.eta(2)), 2, c.r, c.k, prec="fp64").cpu().numpy()
    finally:
        ctx.set_gamma5((1, 1, -1, -1))
    g5 = CS.g5_matrix(signs)
    assert CS.block_err(got_i, c.ref_insertion(1, 2, g5), 2) < CS.FP64_TOL
    assert CS.block_err(got_s, c.ref_spectator_meson(2, g5), 1) < CS.FP64_TOL


def test_host_buffers(ctx, c1):
    """Host (CPU) tensors in and out: the library stages them."""
    S = torch.from_numpy(c1.S)
    psi = torch.from_numpy(c1.psi).pin_memory()
    got = ctx.insertion(S, psi, 3, 4, c1.r, c1.k, prec="fp64").numpy()
    assert CS.block_err(got, c1.ref_insertion(3, 4), 2) < CS.FP64_TOL


@pytest.mark.parametrize("kind", ["meson", "baryon"])
def test_combine(ctx, kind):
    """The combine on oracle-made spectator/insertion tensors against the oracle combine."""
    from oracle import contractions as OC
    rng = np.random.default_rng(7)
    np_, nq, n_r, ng = 5, 7, 3, 4
    cols = 192 if kind == "meson" else 3072
    spec = rng.standard_normal((np_, n_r, cols)) + 1j * rng.standard_normal((np_, n_r, cols))
    ins = rng.standard_normal((nq, n_r, 192)) + 1j * rng.standard_normal((nq, n_r, 192))
    wshape = (4, 4) if kind == "meson" else (4, 4, 4)
    snk = CS.random_gammas(1, ng, wshape)
    gi = CS.random_gammas(2, ng, (4, 4))
    src = CS.random_gammas(3, ng, wshape)
    got = ctx.combine(dev(spec), dev(ins), dev(snk), dev(gi), dev(src)).cpu().numpy()
    fn = OC.combine_meson if kind == "meson" else OC.combine_baryon
    ref = fn(spec, ins, snk, gi, src)
    assert CS.corr_err(got, ref) < CS.FP64_TOL


@pytest.mark.parametrize("kind", ["meson", "baryon"])
@pytest.mark.parametrize("prec,tol", [("fp64", CS.FP64_TOL), ("mixed", CS.MIXED_TOL)])
def test_combine_batched(ctx, kind, prec, tol):
    """nt insertion slices in one call; the mixed combine (FP32 per-noise sums, FP64
    noise average) within 1e-6 per correlator C[t][g][p][q]."""
    from oracle import contractions as OC
    rng = np.random.default_rng(8)
    np_, nq, n_r, ng, nt = 33, 40, 5, 3, 4
    cols = 192 if kind == "meson" else 3072
    spec = rng.standard_normal((np_, n_r, cols)) + 1j * rng.standard_normal((np_, n_r, cols))
    ins = rng.standard_normal((nt, nq, n_r, 192)) + 1j * rng.standard_normal((nt, nq, n_r, 192))
    wshape = (4, 4) if kind == "meson" else (4, 4, 4)
    snk = CS.random_gammas(4, ng, wshape)
    gi = CS.random_gammas(5, ng, (4, 4))
    src = CS.random_gammas(6, ng, wshape)
    got = ctx.combine(dev(spec), dev(ins), dev(snk), dev(gi), dev(src), prec=prec).cpu().numpy()
    fn = OC.combine_meson if kind == "meson" else OC.combine_baryon
    for t in range(nt):
        ref = fn(spec, ins[t], snk, gi, src)
        assert CS.corr_err(got[t], ref) < tol
