"""Brute-force three-point correlators from whole propagators (Eq. 1), for tiny lattices.

No stochastic estimate and no factorization: the trace is taken site pair by site
pair, O(V3^2), then Fourier-summed over the sink and insertion positions with the
same phase conventions as Eqs. 9 and 10.
"""
import numpy as np

from .contractions import EPS, spin_colour
from .momenta import phases


def meson_3pt(G1_rx, G2_xy, G3_yr, g_snk, g_ins, g_src, r3, k_snk, k_ins, L):
    """C(p', q) = sum_{x', y} e^{-i p'.(x'-r)} e^{+i q.(y-r)}
                  tr[G1(r,x') Gamma_snk G2(x',y) Gamma_ins G3(y,r) Gamma_src]   (Eq. 1)

    G1_rx: [V3][12][12] = G1(r, x') for x' on the sink slice;
    G2_xy: [V3 (x')][V3 (y)][12][12] = G2(x', y);
    G3_yr: [V3][12][12] = G3(y, r) for y on the insertion slice.
    Colour deltas of Eq. 1 appear as Gamma (x) 1_colour.  Returns [np][nq]."""
    Gs, Gi, Gc = spin_colour(g_snk), spin_colour(g_ins), spin_colour(g_src)
    V3 = G1_rx.shape[0]
    tr = np.empty((V3, V3), dtype=np.complex128)
    for xp in range(V3):
        for y in range(V3):
            tr[xp, y] = np.trace(G1_rx[xp] @ Gs @ G2_xy[xp, y] @ Gi @ G3_yr[y] @ Gc)
    Ps = phases(L, k_snk, r3, -1)     # [np, V3]
    Pi = phases(L, k_ins, r3, +1)     # [nq, V3]
    return Ps @ tr @ Pi.T


def baryon_3pt(GA_xr, GB_xr, G2_xy, G3_yr, w_snk, g_ins, w_src, r3, k_snk, k_ins, L):
    """Baryon analogue (our reading; the paper gives no formula):

      C(p', q) = sum_{x', y} e^{-i p'.(x'-r)} e^{+i q.(y-r)} sum eps_{a'b'c'} eps_{abc}
                 W_snk[a1', a2', b'] W_src[a1, a2, b] G_A(x',r)^{a1' a1}_{a' a}
                 G_B(x',r)^{a2' a2}_{b' b} [G2(x',y) Gamma_ins G3(y,r)]^{b' b}_{c' c}.

    Returns [np][nq]."""
    Gi = spin_colour(g_ins)
    V3 = GA_xr.shape[0]
    A = GA_xr.reshape(V3, 4, 3, 4, 3)
    B = GB_xr.reshape(V3, 4, 3, 4, 3)
    tr = np.empty((V3, V3), dtype=np.complex128)
    for xp in range(V3):
        for y in range(V3):
            M = (G2_xy[xp, y] @ Gi @ G3_yr[y]).reshape(4, 3, 4, 3)   # [b', c', b, c]
            tr[xp, y] = _baryon_site(A[xp], B[xp], M, w_snk, w_src)
    Ps = phases(L, k_snk, r3, -1)
    Pi = phases(L, k_ins, r3, +1)
    return Ps @ tr @ Pi.T


def _baryon_site(A, B, M, w_snk, w_src):
    """sum eps_{p q s} eps_{u v c} W_snk[I, K, E] W_src[J, L, b] A[I, p, J, u] B[K, q, L, v]
    M[E, s, b, c] at one site pair, taken as a chain of two-operand sums."""
    X = np.einsum("IKE,IpJu->KEpJu", w_snk, A)
    X = np.einsum("KEpJu,KqLv->EpJuqLv", X, B)
    X = np.einsum("EpJuqLv,JLb->Epuqvb", X, w_src)
    X = np.einsum("pqs,Epuqvb->Esuvb", EPS, X)
    X = np.einsum("uvc,Esuvb->Esbc", EPS, X)
    return np.sum(X * M)
