"""Pins of the FP64 oracle: each check ties an oracle function to something other
than itself and raises AssertionError when it does not hold.  The mutation tests
plant a mistake in the oracle and require that one of these checks fails.
"""
import numpy as np

from oracle import contractions as C
from oracle import direct as D
from oracle import freefield as F
from oracle import gamma as G
from oracle import momenta as M
from paper_1711_02384_gb300 import inputs


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _gammas(basis):
    return G.chiral() if basis == "chiral" else G.dirac_pauli()


def _rand(seed, shape):
    return inputs.gaussian_array(seed, 9, shape)


# ---------------------------------------------------------------- momenta / phases

def check_momentum_count(n2max, cmax, count):
    k = M.momenta(n2max, None if cmax < 0 else cmax)
    assert len(k) == count, (n2max, cmax, len(k), count)
    # independent count: for each (kx, ky) the number of kz with kz^2 <= n2max - kx^2 - ky^2
    c = int(np.floor(np.sqrt(n2max))) if cmax < 0 else cmax
    n = 0
    for kx in range(-c, c + 1):
        for ky in range(-c, c + 1):
            rest = n2max - kx * kx - ky * ky
            if rest >= 0:
                n += min(2 * int(np.floor(np.sqrt(rest))) + 1, 2 * c + 1)
    assert n == count, (n, count)


def check_k0_is_site_sum(L=4, seed=11):
    f = _rand(seed, (L ** 3, 5))
    for sign in (+1, -1):
        P = M.phases(L, np.zeros((1, 3), dtype=int), (1, 2, 3), sign)
        assert _rel(P @ f, f.sum(axis=0)[None, :]) < 1e-14


def check_all_momenta_is_fft(L=4, seed=12):
    """With k over all L^3 momenta, the spectator projection (sign -) is numpy's
    forward FFT and the insertion projection (sign +) is V3 times the inverse FFT."""
    f = _rand(seed, (L, L, L))                                  # [z][y][x]
    k = np.array([(kx, ky, kz) for kz in range(L) for ky in range(L) for kx in range(L)])
    fwd = M.phases(L, k, (0, 0, 0), -1) @ f.reshape(-1)
    bwd = M.phases(L, k, (0, 0, 0), +1) @ f.reshape(-1)
    assert _rel(fwd, np.fft.fftn(f).reshape(-1)) < 1e-13
    assert _rel(bwd, (L ** 3) * np.fft.ifftn(f).reshape(-1)) < 1e-13


def check_translation_covariance(L=4, seed=13):
    """Shifting every field by a lattice vector d and the source by d leaves the
    projected spectator and insertion unchanged (the x -> x - r rule after Eq. 10)."""
    g5 = G.gamma5(G.chiral())
    V3 = L ** 3
    S = _rand(seed, (1, V3, 12, 12))
    psi = _rand(seed + 1, (2, 1, V3, 12))
    eta = _rand(seed + 2, (2, V3, 12))
    k = M.momenta(2)
    r = np.array([1, 0, 2])
    d = np.array([3, 1, 2])
    xyz = M.site_coords(L)
    src = np.mod(xyz - d[None, :], L)                            # f'(x) = f(x - d)
    idx = (src[:, 2] * L + src[:, 1]) * L + src[:, 0]
    a = C.insertion(S, psi, g5, r, k, L)
    b = C.insertion(S[:, idx], psi[:, :, idx], g5, r + d, k, L)
    assert _rel(b, a) < 1e-13
    a = C.spectator_meson(S[0], eta, g5, r, k, L)
    b = C.spectator_meson(S[0][idx], eta[:, idx], g5, r + d, k, L)
    assert _rel(b, a) < 1e-13


# ---------------------------------------------------------------- full dilution

def _full_dilution_meson_inputs(L, basis, seed):
    gam = _gammas(basis)
    g5 = G.gamma5(gam)
    V3 = L ** 3
    S1 = _rand(seed, (V3, 12, 12))            # G1(x', r) on the sink slice
    S3 = _rand(seed + 1, (V3, 12, 12))        # G3(y, r) on the insertion slice
    G2_yx = _rand(seed + 2, (V3, V3, 12, 12)) # G2(y, x0): all-to-all, insertion slice <- sink slice
    # full dilution: noise i = (x0, spin, colour), eta_i(x) = delta_{x x0} e_{spin colour}
    N = 12 * V3
    eta = np.zeros((N, V3, 12), dtype=complex)
    for x0 in range(V3):
        for sc in range(12):
            eta[x0 * 12 + sc, x0, sc] = 1.0
    psi = np.transpose(G2_yx, (1, 3, 0, 2)).reshape(N, V3, 12)      # s_i(y) = G2(y, x0) e_sc
    G5 = np.kron(g5, np.eye(3))
    G1_rx = G5 @ np.conj(np.transpose(S1, (0, 2, 1))) @ G5           # gamma5-hermiticity of G1
    G2_xy = G5 @ np.conj(np.transpose(G2_yx, (1, 0, 3, 2))) @ G5    # G2(x', y) from G2(y, x')
    return g5, gam, S1, S3, eta, psi, G1_rx, G2_xy, N


def check_full_dilution_meson(L=2, basis="chiral", seed=21, r=(1, 0, 1)):
    """Eq. 8 is exact under full spin-colour-site dilution of the sink slice:
    N * combine(spectator, insertion) equals the brute-force trace of Eq. 1."""
    g5, gam, S1, S3, eta, psi, G1_rx, G2_xy, N = _full_dilution_meson_inputs(L, basis, seed)
    k = M.momenta(3, 1)[:9]
    ng = 3
    gs = _rand(seed + 5, (ng, 4, 4))
    gi = _rand(seed + 6, (ng, 4, 4))
    gc = _rand(seed + 7, (ng, 4, 4))
    spec = C.spectator_meson(S1, eta, g5, r, k, L)
    ins = C.insertion(S3[None], psi[:, None], g5, r, k, L)[0]
    got = N * C.combine_meson(spec, ins, gs, gi, gc)
    for g in range(ng):
        ref = D.meson_3pt(G1_rx, G2_xy, S3, gs[g], gi[g], gc[g], r, k, k, L)
        assert _rel(got[g], ref) < 1e-12, (g, _rel(got[g], ref))


def check_full_dilution_baryon(L=2, basis="chiral", seed=31, r=(0, 1, 1)):
    """The baryon analogue of the full-dilution identity against the direct
    eps-eps contraction."""
    g5, gam, S1, S3, eta, psi, G1_rx, G2_xy, N = _full_dilution_meson_inputs(L, basis, seed)
    V3 = L ** 3
    GA = _rand(seed + 10, (V3, 12, 12))
    GB = _rand(seed + 11, (V3, 12, 12))
    k = M.momenta(3, 1)[:5]
    ng = 2
    ws = _rand(seed + 12, (ng, 4, 4, 4))
    wc = _rand(seed + 13, (ng, 4, 4, 4))
    gi = _rand(seed + 14, (ng, 4, 4))
    spec = C.spectator_baryon(GA, GB, eta, g5, r, k, L)
    ins = C.insertion(S3[None], psi[:, None], g5, r, k, L)[0]
    got = N * C.combine_baryon(spec, ins, ws, gi, wc)
    for g in range(ng):
        ref = D.baryon_3pt(GA, GB, G2_xy, S3, ws[g], gi[g], wc[g], r, k, k, L)
        assert _rel(got[g], ref) < 1e-12, (g, _rel(got[g], ref))


# ---------------------------------------------------------------- free field

class FreeField:
    """Gauge-rotated free Wilson propagators on an L^3 x T lattice."""

    def __init__(self, L=4, T=8, m=0.3, basis="chiral", seed=41):
        self.L, self.T, self.gam = L, T, _gammas(basis)
        self.g5 = G.gamma5(self.gam)
        self.S = F.wilson_propagator(L, T, m, self.gam)             # [T][z][y][x][4][4]
        rng = np.random.default_rng(seed)
        self.Om = F.random_su3(rng, T * L ** 3).reshape(T, L ** 3, 3, 3)
        self.xyz = M.site_coords(L)

    def spin(self, dt, d3):
        d3 = np.mod(d3, self.L)
        return self.S[dt % self.T, d3[..., 2], d3[..., 1], d3[..., 0]]

    def G(self, tx, x_sites, ty, y_sites, rotate=True):
        """G(x, y) for sites x on slice tx and y on slice ty, broadcast over the
        leading shapes of the two site-index arrays."""
        xs, ys = self.xyz[x_sites], self.xyz[y_sites]
        Ssp = self.spin(tx - ty, xs - ys)
        if rotate:
            Ox, Oy = self.Om[tx % self.T][x_sites], self.Om[ty % self.T][y_sites]
        else:
            Ox = Oy = np.broadcast_to(np.eye(3), np.broadcast(x_sites, y_sites).shape + (3, 3))
        Ox, Oy = np.broadcast_arrays(Ox, Oy)
        return F.full_propagator(Ssp, Ox, Oy)

    def momentum_space_3pt(self, r4, r3, tf, ty, g_snk, g_ins, g_src, ks, kq):
        """Independent evaluation of the (gauge-invariant) free correlator:
        (1/V3) sum_k tr[S~(k; r4-tf) G_snk S~(k+p'; tf-ty) G_ins S~(k+p'-q; ty-r4) G_src]
        times the colour trace 3 (convolution theorem)."""
        L = self.L
        St = lambda t: np.fft.fftn(self.S[t % self.T], axes=(0, 1, 2))   # [kz][ky][kx][4][4]
        A, B, Cc = St(r4 - tf), St(tf - ty), St(ty - r4)
        allk = np.array([(kx, ky, kz) for kz in range(L) for ky in range(L) for kx in range(L)])
        out = np.empty((len(ks), len(kq)), dtype=complex)
        at = lambda X, kk: X[kk[:, 2] % L, kk[:, 1] % L, kk[:, 0] % L]
        for a, p in enumerate(ks):
            for b, q in enumerate(kq):
                m = at(A, allk) @ g_snk @ at(B, allk + p) @ g_ins @ at(Cc, allk + p - q) @ g_src
                out[a, b] = 3.0 * np.trace(m, axis1=1, axis2=2).sum() / L ** 3
        return out


def check_wilson_solves(L=4, T=8, m=0.3, basis="chiral"):
    """The closed-form propagator solves the hopping-stencil Wilson equation D S = delta."""
    gam = _gammas(basis)
    S = F.wilson_propagator(L, T, m, gam)
    DS = F.apply_wilson(S, m, gam)
    delta = np.zeros_like(S)
    delta[0, 0, 0, 0] = np.eye(4)
    assert np.max(np.abs(DS - delta)) < 1e-12


def check_g5_hermiticity(L=4, T=8, m=0.3, basis="chiral"):
    """gamma5 S(x)^dagger gamma5 = S(-x) for the free Wilson propagator."""
    gam = _gammas(basis)
    g5 = G.gamma5(gam)
    S = F.wilson_propagator(L, T, m, gam)
    Sm = np.roll(np.flip(S, axis=(0, 1, 2, 3)), shift=1, axis=(0, 1, 2, 3))    # S(-x)
    lhs = g5 @ np.conj(np.swapaxes(S, -1, -2)) @ g5
    assert np.max(np.abs(lhs - Sm)) < 1e-13


def check_freefield_direct(ff=None, r4=1, r3=(1, 2, 3), tf=5, ty=3):
    """Brute-force Eq. 1 with true (gauge-rotated) free propagators equals the
    momentum-space evaluation."""
    ff = ff or FreeField()
    V3 = ff.L ** 3
    sites = np.arange(V3)
    rsite = (r3[2] * ff.L + r3[1]) * ff.L + r3[0]
    G1_rx = ff.G(r4, np.full(V3, rsite), tf, sites)              # G(r, x')
    G2_xy = ff.G(tf, sites[:, None], ty, sites[None, :])         # G(x', y)
    G3_yr = ff.G(ty, sites, r4, np.full(V3, rsite))              # G(y, r)
    rng = np.random.default_rng(5)
    gs, gi, gc = (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)) for _ in range(3))
    k = M.momenta(2)[:7]
    got = D.meson_3pt(G1_rx, G2_xy, G3_yr, gs, gi, gc, r3, k, k, ff.L)
    ref = ff.momentum_space_3pt(r4, r3, tf, ty, gs, gi, gc, k, k)
    assert _rel(got, ref) < 1e-12, _rel(got, ref)


def check_freefield_factorized(ff=None, r4=1, r3=(1, 2, 3), tf=5, ty=3):
    """The factorized method, fed only what the library receives (point-to-all
    propagators G(x, r) and solutions s_i = D^{-1} eta_i for fully diluted noise),
    reproduces the momentum-space free correlator: this pins the use of
    gamma5-hermiticity (Eqs. 8-9) against a real propagator."""
    ff = ff or FreeField()
    L = ff.L
    V3 = L ** 3
    sites = np.arange(V3)
    rsite = (r3[2] * L + r3[1]) * L + r3[0]
    S1 = ff.G(tf, sites, r4, np.full(V3, rsite))                 # G(x', r)
    S3 = ff.G(ty, sites, r4, np.full(V3, rsite))                 # G(y, r)
    G_yx0 = ff.G(ty, sites[:, None], tf, sites[None, :])         # G(y, x0)
    N = 12 * V3
    eta = np.zeros((N, V3, 12), dtype=complex)
    for x0 in range(V3):
        for sc in range(12):
            eta[x0 * 12 + sc, x0, sc] = 1.0
    psi = np.transpose(G_yx0, (1, 3, 0, 2)).reshape(N, V3, 12)
    rng = np.random.default_rng(6)
    gs, gi, gc = (rng.standard_normal((1, 4, 4)) + 1j * rng.standard_normal((1, 4, 4)) for _ in range(3))
    k = M.momenta(2)[:7]
    spec = C.spectator_meson(S1, eta, ff.g5, r3, k, L)
    ins = C.insertion(S3[None], psi[:, None], ff.g5, r3, k, L)[0]
    got = N * C.combine_meson(spec, ins, gs, gi, gc)[0]
    ref = ff.momentum_space_3pt(r4, r3, tf, ty, gs[0], gi[0], gc[0], k, k)
    assert _rel(got, ref) < 1e-12, _rel(got, ref)


def check_baryon_colour_factor(seed=51):
    """Colour-trivial propagators A(x)1, B(x)1, M(x)1: the eps-eps sum over colours
    gives 3! = 6, leaving 6 * sum W_snk W_src A B M over spins."""
    A = _rand(seed, (4, 4))
    B = _rand(seed + 1, (4, 4))
    Mm = _rand(seed + 2, (4, 4))
    ws = _rand(seed + 3, (4, 4, 4))
    wc = _rand(seed + 4, (4, 4, 4))
    one = lambda X: np.kron(X, np.eye(3)).reshape(4, 3, 4, 3)
    got = D._baryon_site(one(A), one(B), one(Mm), ws, wc)
    ref = 0.0
    for i1 in range(4):
        for i2 in range(4):
            for e in range(4):
                for j1 in range(4):
                    for j2 in range(4):
                        for b in range(4):
                            ref += ws[i1, i2, e] * wc[j1, j2, b] * A[i1, j1] * B[i2, j2] * Mm[e, b]
    assert abs(got - 6 * ref) < 1e-12 * max(1.0, abs(ref)), (got, 6 * ref)


def check_baryon_gauge_invariance(seed=52, L=2, T=4):
    """The eps-eps colour singlet is invariant under SU(3) gauge rotations of all
    propagators (direct baryon trace, free propagators rotated vs not)."""
    ff = FreeField(L=L, T=T, seed=seed)
    V3 = L ** 3
    sites = np.arange(V3)
    r4, tf, ty = 0, 2, 1
    rsite = 0
    k = M.momenta(1)[:3]
    rng = np.random.default_rng(seed)
    ws = rng.standard_normal((4, 4, 4)) + 0j
    wc = rng.standard_normal((4, 4, 4)) + 0j
    gi = rng.standard_normal((4, 4)) + 0j
    res = []
    for rot in (True, False):
        GA = ff.G(tf, sites, r4, np.full(V3, rsite), rot)
        G2 = ff.G(tf, sites[:, None], ty, sites[None, :], rot)
        G3 = ff.G(ty, sites, r4, np.full(V3, rsite), rot)
        res.append(D.baryon_3pt(GA, GA, G2, G3, ws, gi, wc, (0, 0, 0), k, k, L))
    assert _rel(res[0], res[1]) < 1e-12
    assert np.linalg.norm(res[1]) > 1e-6


ALL_CHECKS = [
    lambda: check_momentum_count(8, -1, 93),
    check_k0_is_site_sum,
    check_all_momenta_is_fft,
    check_translation_covariance,
    check_full_dilution_meson,
    lambda: check_full_dilution_meson(basis="dirac_pauli"),
    check_full_dilution_baryon,
    check_wilson_solves,
    check_g5_hermiticity,
    check_freefield_direct,
    check_freefield_factorized,
    check_baryon_colour_factor,
    check_baryon_gauge_invariance,
]
