"""Parity of the mixed-precision path (FP32 contraction, split-FP16 tcgen05 projection,
FP64 reduction) against the FP64 oracle: per-correlator relative error < 1e-6.  The
all-momenta transform that replaces the projection for large momentum lists in the
automatic mode is covered by the DFT tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1711_02384_gb300 import lhc
    c = lhc.Context(0)
    c.set_projection("gemm")   # this module covers the tensor-core projection at every momentum count
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


def _klists():
    from oracle.momenta import momenta
    rng = np.random.default_rng(77)
    full = momenta(4)
    half = np.array([k for k in full if tuple(k) > tuple(-k)])       # no partner requested
    mixed = full[rng.permutation(len(full))][:40]                    # shuffled, pairs broken
    mixed = np.concatenate([mixed, mixed[:5], -mixed[5:9]])          # duplicates and partners
    modL = np.array([[2, 0, 0], [-2, 0, 0], [2, 2, 0], [-2, 2, 0], [0, -2, 2], [1, 0, 0], [-1, 0, 0]])
    big = np.concatenate([momenta(18), np.array([[9, 0, 0], [0, 0, -9]])])   # 173 representatives: 4 chunks
    k9 = momenta(9)
    extra = np.array([k for k in k9 if k @ k == 9 and tuple(k) > tuple(-k)])[:4]
    r51 = np.concatenate([momenta(8), extra, -extra])               # 51 representatives: two chunks of 32
    r36 = np.array([k for k in momenta(8) if tuple(k) > tuple(-k)])[:36]   # one chunk of 40 (36 used)
    return [("unpaired", half), ("shuffled", mixed), ("k=-k mod L", modL), ("four chunks", big),
            ("51 representatives", r51), ("62 representatives", k9), ("36 representatives", r36),
            ("74 representatives", momenta(10))]                    # two chunks of 40


@pytest.mark.parametrize("name,k", _klists(), ids=lambda v: v if isinstance(v, str) else "")
def test_momentum_lists(ctx, name, k):
    """The projection groups the momenta into pairs {k, -k} and forms both from the same
    cos and sin sums: momentum lists with unpaired momenta, broken pairs, duplicates,
    an arbitrary order, momenta whose negatives coincide modulo L (L = 4), every chunk
    width (36 representatives: one chunk of 40; 51 and 62: two of 32; 74: two of 40;
    173: four of 48), all against the oracle."""
    c = CS.Case(4, 4, 2, k, seed=1450, r=(3, 1, 2, 0))
    gi = ctx.insertion(dev(c.S), dev(c.psi), 0, 2, c.r, c.k, prec="mixed").cpu().numpy()
    gs = ctx.spectator(dev(c.S), dev(c.eta(2)), 2, c.r, c.k, prec="mixed").cpu().numpy()
    ctx.sync()
    assert report(f"ins {name}", CS.block_err(gi, c.ref_insertion(0, 2), 2)) < CS.MIXED_TOL
    assert report(f"spec {name}", CS.block_err(gs, c.ref_spectator_meson(2), 1)) < CS.MIXED_TOL


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


def test_meson_48c_largest_served_lattice(ctx):
    """The largest lattice of the served workload (48^3, 110592 sites: the longest sums
    over sites per slice) at full size: one insertion slice and the spectator, 4 noises,
    93 momenta, complex64 inputs, against the oracle on the same complex64-rounded inputs."""
    from oracle.momenta import momenta
    from oracle import contractions as OC
    from paper_1711_02384_gb300 import inputs
    L, n_r, t = 48, 4, 1
    k = momenta(8)
    S = inputs.propagator(2600, L, 2, slices=[0, 1]).astype(np.complex64)
    psi = inputs.solutions(2601, L, 2, n_r, slices=[0, 1]).astype(np.complex64)
    eta = inputs.noise(2602, L, n_r, t).astype(np.complex64)
    r = np.array([5, 17, 40, 0], dtype=np.int32)
    g5 = CS.g5_matrix()
    gi = ctx.insertion(dev(S), dev(psi), t, t, r, k, prec="mixed").cpu().numpy()
    gs = ctx.spectator(dev(S), dev(eta), t, r, k, prec="mixed").cpu().numpy()
    ctx.sync()
    ri = OC.insertion(S[t:t + 1].astype(complex), psi[:, t:t + 1].astype(complex), g5, r[:3], k, L)
    rs = OC.spectator_meson(S[t].astype(complex), eta.astype(complex), g5, r[:3], k, L)
    assert report("48c ins", CS.block_err(gi, ri, 2)) < CS.MIXED_TOL
    assert report("48c spec", CS.block_err(gs, rs, 1)) < CS.MIXED_TOL


def test_noise_offset_beyond_int32(ctx):
    """complex64 solutions whose noise offset (noise x T x V3 x 12 elements) passes 2^31
    for the last noises: 16^3 x 1536 lattice, 32 noises, two insertion slices near the end
    of the time extent; only those slices are filled (26 GB on the device).  Both
    precisions against the oracle on the same complex64-rounded inputs."""
    from oracle.momenta import momenta
    from oracle import contractions as OC
    from paper_1711_02384_gb300 import inputs
    L, T, n_r, t0 = 16, 1536, 32, 1530
    V3 = L ** 3
    assert (n_r - 1) * T * V3 * 12 > 2 ** 31
    k = momenta(2)
    S_h = inputs.propagator(3200, L, T, slices=[t0, t0 + 1]).astype(np.complex64)
    psi_h = inputs.solutions(3201, L, T, n_r, slices=[t0, t0 + 1]).astype(np.complex64)
    S = torch.empty((T, V3, 12, 12), dtype=torch.complex64, device="cuda")
    psi = torch.empty((n_r, T, V3, 12), dtype=torch.complex64, device="cuda")
    try:
        S[t0:t0 + 2] = dev(S_h)
        psi[:, t0:t0 + 2] = dev(psi_h)
        r = np.array([2, 5, 9, 0], dtype=np.int32)
        gm = ctx.insertion(S, psi, t0, t0 + 1, r, k, prec="mixed").cpu().numpy()
        gd = ctx.insertion(S, psi, t0, t0 + 1, r, k, prec="fp64").cpu().numpy()
        ctx.sync()
    finally:
        del S, psi
        torch.cuda.empty_cache()
    ref = OC.insertion(S_h.astype(complex), psi_h.astype(complex), CS.g5_matrix(), r[:3], k, L)
    assert report("ins noise offset > 2^31 (mixed)", CS.block_err(gm, ref, 2)) < CS.MIXED_TOL
    assert report("ins noise offset > 2^31 (fp64)", CS.block_err(gd, ref, 2)) < CS.FP64_TOL


@pytest.mark.parametrize("L,n_r,n2max,cmax,r,dtype", [
    (3, 3, 2, -1, (1, 2, 0, 0), np.complex128),   # odd n_r, source off the origin
    (4, 2, 3, 1, (0, 0, 0, 0), np.complex64),     # 27 momenta, complex64 storage
])
def test_spectator_baryon(ctx, L, n_r, n2max, cmax, r, dtype):
    from oracle.momenta import momenta
    c = CS.Case(L, 4, n_r, momenta(n2max, None if cmax < 0 else cmax), seed=1600 + L, r=r, dtype=dtype)
    got = ctx.spectator(dev(c.S), dev(c.eta(1)), 1, c.r, c.k, prec="mixed", GB=dev(c.SB)).cpu().numpy()
    ctx.sync()
    assert report(f"baryon L={L}", CS.block_err(got, c.ref_spectator_baryon(1), 1)) < CS.MIXED_TOL


def test_baryon_16c_123mom_sampled_noises(ctx):
    """Baryon spectator on a 16^3 slice with 32 noises and the 123 momenta of |k|^2 <= 9
    (components <= 3), complex64 storage; two of the 32 noises against the oracle."""
    from oracle.momenta import momenta
    from oracle import contractions as OC
    from paper_1711_02384_gb300 import inputs
    L, n_r = 16, 32
    k = momenta(9, 3)
    GA = inputs.propagator(3000, L, 4, slices=[1]).astype(np.complex64)
    GB = inputs.propagator(3000, L, 4, slices=[1], tensor_id=inputs.TID_PROP_B).astype(np.complex64)
    eta = inputs.noise(3003, L, n_r, 1).astype(np.complex64)
    r = np.zeros(4, dtype=np.int32)
    got = ctx.spectator(dev(GA), dev(eta), 0, r, k, prec="mixed", GB=dev(GB)).cpu().numpy()
    ctx.sync()
    pick = [0, n_r - 1]
    ref = OC.spectator_baryon(GA[0].astype(complex), GB[0].astype(complex), eta[pick].astype(complex),
                              CS.g5_matrix(), r[:3], k, L)
    assert report("baryon 16^3 sampled", CS.block_err(got[:, pick], ref, 1)) < CS.MIXED_TOL


def test_baryon_32c_full_size_sampled_components(ctx):
    """The full 32^3 baryon workload shape (32 noises, 123 momenta, complex64): sampled
    output components, each computed by the oracle one by one, per-component relative
    error over all momenta."""
    from oracle.momenta import momenta
    from oracle import contractions as OC
    from paper_1711_02384_gb300 import inputs
    L, n_r = 32, 32
    k = momenta(9, 3)
    GA = inputs.propagator(3100, L, 64, slices=[10]).astype(np.complex64)
    GB = inputs.propagator(3100, L, 64, slices=[10], tensor_id=inputs.TID_PROP_B).astype(np.complex64)
    eta = inputs.noise(3103, L, n_r, 10).astype(np.complex64)
    r = np.array([3, 7, 11, 0], dtype=np.int32)
    got = ctx.spectator(dev(GA), dev(eta), 0, r, k, prec="mixed", GB=dev(GB)).cpu().numpy()
    ctx.sync()
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(6):
        i = int(rng.integers(n_r))
        comp = tuple(int(v) for v in rng.integers(0, 4, 5)) + (int(rng.integers(3)),)
        col = ((((comp[0] * 4 + comp[1]) * 4 + comp[2]) * 4 + comp[3]) * 4 + comp[4]) * 3 + comp[5]
        ref = OC.spectator_baryon_component(GA[0].astype(complex), GB[0].astype(complex), eta[i].astype(complex),
                                            CS.g5_matrix(), r[:3], k, L, *comp)
        err = np.linalg.norm(got[:, i, col] - ref) / np.linalg.norm(ref)
        worst = max(worst, err)
    assert report("baryon 32^3 sampled components", worst) < CS.MIXED_TOL


def test_misaligned_buffers_rejected(ctx):
    """complex64 views that start 8 bytes into an allocation are refused with LHC_EINVAL
    before any launch (the kernels copy 16-byte chunks)."""
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import lhc
    L, T, n_r = 4, 2, 2
    V3 = L ** 3
    k = momenta(1)
    S = torch.zeros(T * V3 * 144 + 1, dtype=torch.complex64, device="cuda")[1:].view(T, V3, 12, 12)
    psi = torch.zeros((n_r, T, V3, 12), dtype=torch.complex64, device="cuda")
    with pytest.raises(lhc.LhcError) as e:
        ctx.insertion(S, psi, 0, 1, (0, 0, 0, 0), k, prec="mixed")
    assert e.value.status == 1 and "aligned" in str(e.value)
    eta = torch.zeros(n_r * V3 * 12 + 1, dtype=torch.complex64, device="cuda")[1:].view(n_r, V3, 12)
    S_ok = torch.zeros((T, V3, 12, 12), dtype=torch.complex64, device="cuda")
    with pytest.raises(lhc.LhcError) as e:
        ctx.spectator(S_ok, eta, 0, (0, 0, 0, 0), k, prec="fp64")
    assert e.value.status == 1
    ctx.sync()


@pytest.mark.parametrize("name,fs,fv", [
    ("tiny", 1e-9, 1e-6),          # products near 1e-15: the unscaled FP16 split would flush them
    ("huge", 3e3, 1e3),            # products near 1e7 (1e10 for the baryon): beyond FP16
    ("decaying", None, 1.0),       # slice t scaled by exp(-0.9 |t|): 5 orders over the range
])
def test_dynamic_range(ctx, name, fs, fv):
    """The FP16 split of the contracted values is scaled per slice by a power of two
    bounded by the operands' maxima, so inputs far from unit magnitude keep the 1e-6
    per-correlator bound: insertion over slices of different magnitude, meson and baryon
    spectators, against the oracle."""
    from oracle.momenta import momenta
    from oracle import contractions as OC
    c = CS.Case(4, 8, 2, momenta(2), seed=1700, r=(1, 2, 3, 0))
    if fs is None:
        w = np.exp(-0.9 * np.arange(8))
        S, SB = c.S * w[:, None, None, None], c.SB * w[:, None, None, None]
    else:
        S, SB = c.S * fs, c.SB * fs
    psi, eta = c.psi * fv, c.eta(6) * fv
    g5 = CS.g5_matrix()
    gi = ctx.insertion(dev(S), dev(psi), 0, 6, c.r, c.k, prec="mixed").cpu().numpy()
    gs = ctx.spectator(dev(S), dev(eta), 6, c.r, c.k, prec="mixed").cpu().numpy()
    gb = ctx.spectator(dev(S), dev(eta), 6, c.r, c.k, prec="mixed", GB=dev(SB)).cpu().numpy()
    ctx.sync()
    ri = OC.insertion(S[0:7], psi[:, 0:7], g5, c.r[:3], c.k, 4)
    rs = OC.spectator_meson(S[6], eta, g5, c.r[:3], c.k, 4)
    rb = OC.spectator_baryon(S[6], SB[6], eta, g5, c.r[:3], c.k, 4)
    assert report(f"ins {name}", CS.block_err(gi, ri, 2)) < CS.MIXED_TOL
    assert report(f"spec {name}", CS.block_err(gs, rs, 1)) < CS.MIXED_TOL
    assert report(f"baryon {name}", CS.block_err(gb, rb, 1)) < CS.MIXED_TOL


def test_complex128_staging_is_the_ieee_conversion(ctx):
    """complex128 inputs are staged to complex64 (round to nearest even); the
    mixed results must equal, bit for bit, those from the same inputs converted to
    complex64 on the host by numpy (IEEE 754).  Magnitudes span 2^-12 .. 2^4, a quarter
    of the values sit exactly on a rounding tie, and a few are zero or round to binary32
    subnormals.  The results must also be finite: the baryon's products of three such
    inputs exceed the FP16 range unless the split is scaled."""
    from oracle.momenta import momenta
    g = torch.Generator(device="cuda")
    g.manual_seed(77)
    L, T, n_r = 6, 4, 3
    V3 = L ** 3

    def rough(shape):
        x = torch.randn(shape + (2,), dtype=torch.float64, device="cuda", generator=g)
        x = x * torch.exp2(torch.randint(-12, 5, shape + (2,), device="cuda", generator=g).double())
        bits = x.view(torch.int64)
        tie = torch.rand(shape + (2,), device="cuda", generator=g) < 0.25
        bits = torch.where(tie, (bits & ~0x1FFFFFFF) | 0x10000000, bits)
        x = bits.view(torch.float64)
        # exact zeros and values whose binary32 result is subnormal (the conversion's
        # other branch)
        u = torch.rand(shape + (2,), device="cuda", generator=g)
        x = torch.where(u < 0.02, torch.zeros_like(x), torch.where(u > 0.98, x * 2.0 ** -135, x))
        return torch.view_as_complex(x.contiguous())

    S, SB = rough((T, V3, 12, 12)), rough((T, V3, 12, 12))
    psi, eta = rough((n_r, T, V3, 12)), rough((n_r, V3, 12))
    k = momenta(2)
    r = (1, 0, 2, 0)
    # the reference conversion is numpy's on the host: IEEE round to nearest even with
    # gradual underflow
    c64 = lambda t: torch.from_numpy(t.cpu().numpy().astype(np.complex64)).cuda()
    a = ctx.insertion(S, psi, 0, 3, r, k, prec="mixed")
    b = ctx.insertion(c64(S), c64(psi), 0, 3, r, k, prec="mixed")
    assert torch.equal(a, b)
    a = ctx.spectator(S, eta, 2, r, k, prec="mixed")
    b = ctx.spectator(c64(S), c64(eta), 2, r, k, prec="mixed")
    assert torch.equal(a, b)
    a = ctx.spectator(S, eta, 1, r, k, prec="mixed", GB=SB)
    b = ctx.spectator(c64(S), c64(eta), 1, r, k, prec="mixed", GB=c64(SB))
    assert torch.equal(a, b)
    assert bool(torch.isfinite(torch.view_as_real(a)).all())
    ctx.sync()
