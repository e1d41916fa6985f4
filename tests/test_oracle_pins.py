"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import os

import numpy as np
import pytest

import _pins as P
from oracle import contractions as C
from oracle import gamma as G
from oracle import momenta as M
from paper_1711_02384_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gamma_bases():
    for gam in (G.chiral(), G.dirac_pauli()):
        for mu in range(4):
            assert np.allclose(gam[mu], gam[mu].conj().T)
            for nu in range(4):
                ac = gam[mu] @ gam[nu] + gam[nu] @ gam[mu]
                assert np.allclose(ac, 2 * np.eye(4) * (mu == nu))
        g5 = G.gamma5(gam)
        assert np.allclose(g5 @ g5, np.eye(4)) and np.allclose(g5, g5.conj().T)
    assert np.allclose(G.gamma5(G.chiral()), np.diag([1, 1, -1, -1]))
    assert not np.allclose(G.gamma5(G.dirac_pauli()), np.diag(np.diag(G.gamma5(G.dirac_pauli()))))
    g16 = G.gamma16(G.chiral())
    # the 16 structures are a basis of 4x4 matrices: tr(G_a^dagger G_b) = 4 delta_ab
    gram = np.einsum("aij,bij->ab", g16.conj(), g16)
    assert np.allclose(gram, 4 * np.eye(16))


def _golden_counts():
    rows = []
    with open(os.path.join(GOLDEN, "momentum_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n2, c, cnt, _ = line.split()
                rows.append((int(n2), int(c), int(cnt)))
    return rows


@pytest.mark.parametrize("n2max,cmax,count", _golden_counts())
def test_momentum_counts_golden(n2max, cmax, count):
    P.check_momentum_count(n2max, cmax, count)


@pytest.mark.parametrize("n2max", [4, 9, 16])
def test_momentum_counts_independent(n2max):
    k = M.momenta(n2max)
    P.check_momentum_count(n2max, -1, len(k))
    # closed under negation and permutation of components, no duplicates
    s = {tuple(v) for v in k}
    assert len(s) == len(k)
    assert all(tuple(-np.array(v)) in s for v in s)
    assert all((v[1], v[2], v[0]) in s for v in s)
    n2 = (k ** 2).sum(1)
    assert np.all(np.diff(n2) >= 0)


def test_k0_is_site_sum():
    P.check_k0_is_site_sum()


def test_all_momenta_is_fft():
    P.check_all_momenta_is_fft()


def test_translation_covariance():
    P.check_translation_covariance()


@pytest.mark.parametrize("basis", ["chiral", "dirac_pauli"])
def test_full_dilution_meson(basis):
    P.check_full_dilution_meson(basis=basis)


def test_full_dilution_meson_L4():
    P.check_full_dilution_meson(L=4, seed=22, r=(3, 1, 2))


def test_full_dilution_baryon():
    P.check_full_dilution_baryon()


def test_full_dilution_baryon_dirac_pauli():
    P.check_full_dilution_baryon(basis="dirac_pauli", seed=33)


@pytest.mark.parametrize("basis", ["chiral", "dirac_pauli"])
def test_wilson_propagator_solves_stencil(basis):
    P.check_wilson_solves(basis=basis)


@pytest.mark.parametrize("basis", ["chiral", "dirac_pauli"])
def test_wilson_gamma5_hermiticity(basis):
    P.check_g5_hermiticity(basis=basis)


def test_freefield_direct_vs_momentum_space():
    P.check_freefield_direct()


def test_freefield_factorized_vs_momentum_space():
    P.check_freefield_factorized()


def test_freefield_factorized_origin_source():
    P.check_freefield_factorized(r4=0, r3=(0, 0, 0), tf=4, ty=2)


def test_baryon_colour_factor():
    P.check_baryon_colour_factor()


def test_baryon_gauge_invariance():
    P.check_baryon_gauge_invariance()


def test_baryon_single_component_matches_full():
    """The one-component baryon helper (used for sampled checks on large lattices)
    equals the corresponding column of the full baryon spectator."""
    L, V3 = 3, 27
    GA = inputs.gaussian_array(1, 9, (V3, 12, 12))
    GB = inputs.gaussian_array(2, 9, (V3, 12, 12))
    eta = inputs.gaussian_array(3, 9, (2, V3, 12))
    g5 = G.gamma5(G.chiral())
    k = M.momenta(2)
    r = (1, 2, 0)
    full = C.spectator_baryon(GA, GB, eta, g5, r, k, L)
    for comp in [(0, 0, 0, 0, 0, 0), (3, 2, 1, 0, 2, 1), (1, 3, 2, 2, 3, 2)]:
        a1p, a1, a2p, a2, bp, c = comp
        col = ((((a1p * 4 + a1) * 4 + a2p) * 4 + a2) * 4 + bp) * 3 + c
        one = C.spectator_baryon_component(GA, GB, eta[1], g5, r, k, L, *comp)
        assert np.max(np.abs(one - full[:, 1, col])) < 1e-12


def test_noise_moments():
    """Z2 x Z2 noise: unit modulus, mean 0 and <eta eta*> = delta within the
    statistical 1/sqrt(N) of Eqs. 6-7."""
    n = 4000
    eta = inputs.noise(5, 2, n)                    # [n][8][12]
    assert np.allclose(np.abs(eta), 1.0)
    v = eta.reshape(n, -1)
    mean = v.mean(0)
    assert np.max(np.abs(mean)) < 5 / np.sqrt(n)
    cov = v.T @ v.conj() / n
    assert np.max(np.abs(cov - np.eye(v.shape[1]))) < 6 / np.sqrt(n)


def test_philox_known_answers():
    """The input generator is Philox4x32-10: its outputs on the three published
    known-answer vectors (tests/golden/philox4x32_10_kat.txt) match word for word."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        w = [int(x, 16) for x in row]
        ctr = np.array(w[0:4], dtype=np.uint64)
        key = np.array(w[4:6], dtype=np.uint64)
        got = inputs.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == w[6:10], row


def test_gaussian_generator_moments():
    g = inputs.gaussian_rows(3, 0, np.arange(2000), 12).reshape(-1)
    assert abs(g.real.mean()) < 0.03 and abs(g.imag.mean()) < 0.03
    assert abs(g.real.var() - 1) < 0.03 and abs(g.imag.var() - 1) < 0.03
    a = inputs.propagator(1, 3, 4, slices=[2])
    b = inputs.propagator(1, 3, 4)[2:3]
    assert np.array_equal(a, b)                  # any slice regenerates on its own


# ------------------------------------------------------------------ planted mistakes
# Each mutation plants one plausible mistake in the oracle (on the CPU) and requires
# that at least one pin catches it.

def _g5_no_transpose(S, g5):
    G5 = C.spin_colour(g5)
    return G5 @ np.conj(S) @ G5


def _ins_sites_no_conj(S3, psi, g5):
    s5 = C.apply_g5_vec(g5, psi).reshape(psi.shape[0], psi.shape[1], 4, 3)
    G3 = S3.reshape(S3.shape[0], 4, 3, 4, 3)
    return np.einsum("iyAc,yBcDa->yiABDa", s5, G3)


def _phases_wrong_sign(L, k, r3, sign):
    return M.phases(L, k, r3, -sign)


def _phases_plus_r(L, k, r3, sign):
    return M.phases(L, k, -np.asarray(r3), sign)


def _apply_no_g5(g5, v):
    return v


def _combine_src_transposed(spec, ins, gs, gi, gc):
    return C.__dict__["_orig_combine"](spec, ins, gs, gi, np.swapaxes(gc, -1, -2))


def _eps_wrong(monkeypatch):
    bad = C.EPS.copy()
    bad[0, 1, 2] = -1.0            # breaks total antisymmetry
    monkeypatch.setattr(C, "EPS", bad)


MUTATIONS = {
    "gamma5 conjugate without transpose": lambda mp: mp.setattr(C, "gamma5_hermitian_conjugate", _g5_no_transpose),
    "insertion without complex conjugate": lambda mp: mp.setattr(C, "insertion_sites", _ins_sites_no_conj),
    "spectator/insertion phase sign flipped": lambda mp: mp.setattr(C, "phases", _phases_wrong_sign),
    "source shift x + r instead of x - r": lambda mp: mp.setattr(C, "phases", _phases_plus_r),
    "gamma5 dropped from the noise and solution": lambda mp: mp.setattr(C, "apply_g5_vec", _apply_no_g5),
    "baryon epsilon tensor wrong": _eps_wrong,
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    failed = []
    for chk in P.ALL_CHECKS:
        try:
            chk()
        except AssertionError:
            failed.append(chk)
    assert failed, f"no pin caught the planted mistake: {name}"


def test_pins_catch_transposed_gamma_src(monkeypatch):
    monkeypatch.setitem(C.__dict__, "_orig_combine", C.combine_meson)
    monkeypatch.setattr(C, "combine_meson", _combine_src_transposed)
    with pytest.raises(AssertionError):
        P.check_full_dilution_meson()


def test_baryon_exchange_is_an_index_permutation():
    """Swapping the two spectator propagators of the eps-eps contraction (the second Wick
    topology of two identical spectator flavours) permutes the open indices
    (a1', a1) <-> (a2', a2) of the spectator: eps_{a'b'c'} eps_{abc} is invariant when
    both colour pairs are exchanged.  Checked on the oracle's spectator."""
    from oracle import contractions as OC
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import inputs
    import numpy as np
    L, n_r = 2, 2
    GA = inputs.propagator(2200, L, 1)[0]
    GB = inputs.propagator(2200, L, 1, tensor_id=inputs.TID_PROP_B)[0]
    eta = inputs.noise(2201, L, n_r, 0)
    g5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(complex)
    k, r3 = momenta(1)[:4], np.array([1, 0, 1])
    ab = OC.spectator_baryon(GA, GB, eta, g5, r3, k, L).reshape(len(k), n_r, 4, 4, 4, 4, 4, 3)
    ba = OC.spectator_baryon(GB, GA, eta, g5, r3, k, L).reshape(len(k), n_r, 4, 4, 4, 4, 4, 3)
    assert np.abs(ba - ab.transpose(0, 1, 4, 5, 2, 3, 6, 7)).max() < 1e-12 * np.abs(ab).max()


def test_benchmark_dirac_basis_is_a_clifford_basis():
    """The benchmark's Gamma structures (built in the input module, apart from the
    oracle): Hermitian gamma_mu with {gamma_mu, gamma_nu} = 2 delta, gamma5 =
    diag(1, 1, -1, -1), and 16 products that span the 4x4 matrices."""
    import numpy as np
    from paper_1711_02384_gb300 import inputs
    g = inputs.dirac_matrices()
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2 * (a == b) * np.eye(4))
    assert np.allclose(g[0] @ g[1] @ g[2] @ g[3], np.diag([1, 1, -1, -1]))
    G = inputs.dirac_structures().reshape(16, 16)
    assert np.linalg.matrix_rank(G) == 16
