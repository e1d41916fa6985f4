"""Spectator, insertion and combine in FP64: the plain definitions (Sec. 2.1).

Conventions (all complex128):

* a propagator S(x) = G(x, r) is a 12x12 matrix per site, row = sink (spin, colour)
  at x, column = source (spin, colour) at r, flattened as spin*3 + colour;
* ``g5`` is the 4x4 gamma5 matrix of the basis in use (Hermitian, squares to 1);
  spin structures act on colour as the identity;
* a timeslice holds L^3 sites ordered site = (z*L + y)*L + x.

Readings of the paper taken here (the paper is silent or inconsistent):

* Eq. 9 writes the G1 factor as [gamma5 G1^dagger(x', r) gamma5]^{alpha' alpha}_{a' a};
  Eq. 1 needs G1(r, x')^{alpha alpha'}_{a a'}.  gamma5-hermiticity gives
  G1(r, x') = gamma5 G1(x', r)^dagger gamma5, and the element used is the one Eq. 1
  needs: row (alpha, a), column (alpha', a').
* The stochastic line G2(x', y) comes from Eq. 5 by gamma5-hermiticity:
  G2(x', y) = gamma5 G2(y, x')^dagger gamma5
            ~ (1/N) sum_i [gamma5 eta_i(x')] [gamma5 s_i(y)]^dagger,
  so the spectator carries (gamma5 eta_i)^{beta'}_{b'} (the paper's row form
  eta_i gamma5 is the same vector for a symmetric gamma5) and the insertion
  carries conj(gamma5 s_i)^{alpha~}_{a~}.
* 1/N is applied only in the combine; spectator and insertion are plain sums.
* Output component orders: insertion (alpha~, beta~, beta, a), meson spectator
  (beta', alpha', alpha, a), baryon spectator (alpha1', alpha1, alpha2', alpha2,
  beta', c).
"""
import numpy as np

from .momenta import phases

EPS = np.zeros((3, 3, 3))
for _a, _b, _c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
    EPS[_a, _b, _c] = 1.0
    EPS[_a, _c, _b] = -1.0


def spin_colour(m4: np.ndarray) -> np.ndarray:
    """4x4 spin matrix -> 12x12 spin (x) colour-identity matrix."""
    return np.kron(m4, np.eye(3))


def gamma5_hermitian_conjugate(S: np.ndarray, g5: np.ndarray) -> np.ndarray:
    """gamma5 S^dagger gamma5 for a stack of 12x12 matrices [..., 12, 12]: the
    propagator in the opposite direction, G(r, x) = gamma5 G(x, r)^dagger gamma5."""
    G5 = spin_colour(g5)
    return G5 @ np.conj(np.swapaxes(S, -1, -2)) @ G5


def apply_g5_vec(g5: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(gamma5 v) for spin-colour vectors v[..., 12]."""
    return v @ spin_colour(g5).T


# ---------------------------------------------------------------- insertion, Eq. 10

def insertion_sites(S3: np.ndarray, psi: np.ndarray, g5: np.ndarray) -> np.ndarray:
    """U_i(y)[alpha~, beta~, beta, a] = sum_{a~} conj((gamma5 s_i(y))^{alpha~}_{a~})
    G3(y, r)^{beta~ beta}_{a~ a} for every site y (no momentum sum yet).

    S3: [V3][12][12]; psi: [n_r][V3][12].  Returns [V3][n_r][4][4][4][3]."""
    s5 = apply_g5_vec(g5, psi).reshape(psi.shape[0], psi.shape[1], 4, 3)   # [i, y, alpha~, a~]
    G3 = S3.reshape(S3.shape[0], 4, 3, 4, 3)                                # [y, beta~, a~, beta, a]
    return np.einsum("iyAc,yBcDa->yiABDa", np.conj(s5), G3)


def insertion(S3: np.ndarray, psi: np.ndarray, g5: np.ndarray, r3, k: np.ndarray,
              L: int) -> np.ndarray:
    """Insertion part I_i(q, y4) of Eq. 10 for each given slice.

    S3: [nt][V3][12][12] propagator G3(y, r) on the insertion slices;
    psi: [n_r][nt][V3][12] stochastic solutions on the same slices.
    Returns complex128 [nt][nq][n_r][192] (components alpha~, beta~, beta, a)."""
    P = phases(L, k, r3, +1)                                               # [nq, V3]
    nt = S3.shape[0]
    n_r = psi.shape[0]
    out = np.empty((nt, P.shape[0], n_r, 192), dtype=np.complex128)
    for t in range(nt):
        U = insertion_sites(S3[t], psi[:, t], g5).reshape(S3.shape[1], n_r * 192)
        out[t] = (P @ U).reshape(P.shape[0], n_r, 192)
    return out


# ---------------------------------------------------------------- spectator, Eq. 9

def spectator_meson_sites(S1: np.ndarray, eta: np.ndarray, g5: np.ndarray) -> np.ndarray:
    """V_i(x')[beta', alpha', alpha, a] = sum_{a'} (gamma5 eta_i(x'))^{beta'}_{a'}
    G1(r, x')^{alpha alpha'}_{a a'} with G1(r, x') = gamma5 S1(x')^dagger gamma5.

    S1: [V3][12][12] = G1(x', r); eta: [n_r][V3][12].  Returns [V3][n_r][4][4][4][3]."""
    G1 = gamma5_hermitian_conjugate(S1, g5).reshape(S1.shape[0], 4, 3, 4, 3)   # [x, alpha, a, alpha', a']
    e5 = apply_g5_vec(g5, eta).reshape(eta.shape[0], eta.shape[1], 4, 3)        # [i, x, beta', a']
    return np.einsum("ixBc,xAaPc->xiBPAa", e5, G1)


def spectator_meson(S1: np.ndarray, eta: np.ndarray, g5: np.ndarray, r3, k: np.ndarray,
                    L: int) -> np.ndarray:
    """Meson spectator part S_i(p', x'4) of Eq. 9 on the sink slice.
    Returns complex128 [nq][n_r][192] (components beta', alpha', alpha, a)."""
    P = phases(L, k, r3, -1)
    V = spectator_meson_sites(S1, eta, g5).reshape(S1.shape[0], -1)
    return (P @ V).reshape(P.shape[0], eta.shape[0], 192)


def spectator_baryon_sites(GA: np.ndarray, GB: np.ndarray, eta: np.ndarray,
                           g5: np.ndarray) -> np.ndarray:
    """Baryon spectator before the momentum sum (the paper gives no formula; this is
    our reading).  The two spectator quarks run from the source r to the sink x'
    as G_A(x', r), G_B(x', r); the third quark's sink end is the stochastic
    (gamma5 eta_i)(x'), exactly as in the meson, so the insertion part is shared:

      B_i(x')[a1', a1, a2', a2, b', c] = sum eps_{p q s} eps_{u v c}
            G_A(x')^{a1' a1}_{p u} G_B(x')^{a2' a2}_{q v} (gamma5 eta_i)^{b'}_{s}.

    Returns [V3][n_r][4][4][4][4][4][3]."""
    A = GA.reshape(GA.shape[0], 4, 3, 4, 3)      # [x, a1', p, a1, u]
    B = GB.reshape(GB.shape[0], 4, 3, 4, 3)      # [x, a2', q, a2, v]
    e5 = apply_g5_vec(g5, eta).reshape(eta.shape[0], eta.shape[1], 4, 3)   # [i, x, b', s]
    D = np.einsum("pqs,uvc,xIpJu,xKqLv->xIJKLsc", EPS, EPS, A, B)           # noise-independent diquark
    return np.einsum("xIJKLsc,ixEs->xiIJKLEc", D, e5)


def spectator_baryon(GA, GB, eta, g5, r3, k, L) -> np.ndarray:
    """Baryon spectator projected with exp(-i p'.(x'-r)).
    Returns complex128 [nq][n_r][3072] (alpha1', alpha1, alpha2', alpha2, beta', c)."""
    P = phases(L, k, r3, -1)
    Bx = spectator_baryon_sites(GA, GB, eta, g5).reshape(GA.shape[0], -1)
    return (P @ Bx).reshape(P.shape[0], eta.shape[0], 3072)


# ---------------------------------------------------------------- combine, Eqs. 5 and 8

def combine_meson(spec: np.ndarray, ins: np.ndarray, g_snk, g_ins, g_src) -> np.ndarray:
    """C[g][p'][q] = (1/N) sum_i Gamma_snk^{alpha' beta'} Gamma_ins^{alpha~ beta~}
    Gamma_src^{beta alpha} S_i(p')^{beta' alpha' alpha}_a I_i(q)^{alpha~ beta~ beta}_a.

    spec: [np][N][192]; ins: [nq][N][192]; Gammas: [ng][4][4].  Returns [ng][np][nq]."""
    n = spec.shape[1]
    S = spec.reshape(spec.shape[0], n, 4, 4, 4, 3)   # [p, i, beta', alpha', alpha, a]
    I = ins.reshape(ins.shape[0], n, 4, 4, 4, 3)     # [q, i, alpha~, beta~, beta, a]
    out = np.empty((len(g_snk), spec.shape[0], ins.shape[0]), dtype=np.complex128)
    for g in range(len(g_snk)):
        out[g] = np.einsum("PB,GH,bA,piBPAa,qiGHba->pq", g_snk[g], g_ins[g], g_src[g], S, I,
                           optimize=True) / n
    return out


def combine_baryon(spec: np.ndarray, ins: np.ndarray, w_snk, g_ins, w_src) -> np.ndarray:
    """C[g][p'][q] = (1/N) sum_{i,c} W_snk[a1',a2',b'] W_src[a1,a2,b] Gamma_ins^{a~ b~}
    B_i(p')^{a1' a1 a2' a2 b'}_c I_i(q)^{a~ b~ b}_c.

    spec: [np][N][3072]; ins: [nq][N][192]; W: [ng][4][4][4]; Gamma_ins: [ng][4][4]."""
    n = spec.shape[1]
    B = spec.reshape(spec.shape[0], n, 4, 4, 4, 4, 4, 3)
    I = ins.reshape(ins.shape[0], n, 4, 4, 4, 3)
    out = np.empty((len(w_snk), spec.shape[0], ins.shape[0]), dtype=np.complex128)
    for g in range(len(w_snk)):
        out[g] = np.einsum("IKE,JLb,GH,piIJKLEc,qiGHbc->pq", w_snk[g], w_src[g], g_ins[g], B, I,
                           optimize=True) / n
    return out


def spectator_baryon_component(GA, GB, eta_i, g5, r3, k, L, a1p, a1, a2p, a2, bp, c) -> np.ndarray:
    """One open component (alpha1', alpha1, alpha2', alpha2, beta', c) of the baryon spectator
    for one noise, at all momenta: the same sum as spectator_baryon, restricted to one
    output column so that large lattices stay cheap.  Returns complex128 [nq]."""
    A = GA.reshape(GA.shape[0], 4, 3, 4, 3)[:, a1p, :, a1, :]      # [x, a', a]
    B = GB.reshape(GB.shape[0], 4, 3, 4, 3)[:, a2p, :, a2, :]      # [x, b', b]
    e5 = apply_g5_vec(g5, eta_i).reshape(eta_i.shape[0], 4, 3)[:, bp, :]   # [x, c']
    D = np.einsum("pqs,uv,xpu,xqv->xs", EPS, EPS[:, :, c], A, B)                    # [x, c']
    return phases(L, k, r3, -1) @ np.einsum("xs,xs->x", D, e5)
