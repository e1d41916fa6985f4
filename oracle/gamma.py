"""Euclidean Dirac matrices, Hermitian, {gamma_mu, gamma_nu} = 2 delta_mu_nu.

The paper does not fix a basis (Sec. 2).  ``chiral()`` is the DeGrand-Rossi basis
in which gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1, 1, -1, -1); ``dirac_pauli()``
has a non-diagonal gamma5 and is used to show that the factorization (Eq. 8) holds
in any basis.  The index order is (mu = 1, 2, 3, 4) -> list positions 0..3.
"""
import numpy as np


def chiral():
    i = 1j
    g1 = np.array([[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]])
    g2 = np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=complex)
    g3 = np.array([[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]])
    g4 = np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=complex)
    return [g1, g2, g3, g4]


def dirac_pauli():
    s = [np.array([[0, 1], [1, 0]], dtype=complex),
         np.array([[0, -1j], [1j, 0]]),
         np.array([[1, 0], [0, -1]], dtype=complex)]
    z = np.zeros((2, 2), dtype=complex)
    one = np.eye(2, dtype=complex)
    gk = [np.block([[z, -1j * sk], [1j * sk, z]]) for sk in s]
    g4 = np.block([[one, z], [z, -one]])
    return gk + [g4]


def gamma5(gammas):
    g = gammas
    return g[0] @ g[1] @ g[2] @ g[3]


def gamma16(gammas):
    """The 16 products gamma_1^n1 gamma_2^n2 gamma_3^n3 gamma_4^n4 (n in {0,1}),
    ordered by the bit pattern n1 + 2 n2 + 4 n3 + 8 n4 (the Chroma numbering)."""
    out = []
    for n in range(16):
        m = np.eye(4, dtype=complex)
        for mu in range(4):
            if (n >> mu) & 1:
                m = m @ gammas[mu]
        out.append(m)
    return np.array(out)
