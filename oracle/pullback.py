"""Macro field A_ij^H(t)(xi) of eq. 37 through the curvilinear formalism of appendix A.

Literal transcription, per point, of
  g_i = M_,xi_i                                   (eq. 79: covariant basis = columns of J)
  g_ij = g_i . g_j,  [g^ij] = [g_ij]^-1           (eq. 81)
  C^ijkl = lam g^ij g^kl + mu (g^ik g^jl + g^il g^jk)        (eq. 84a)
  C (6x6, Voigt order 11,22,33,23,13,12)          (eq. 93)
  G_1 = [g1 0 0 0 g3 g2], G_2 = [0 g2 0 g3 0 g1], G_3 = [0 0 g3 g2 g1 0]   (eq. 91)
  A_ij = G_i C G_j^T |det J|                      (eq. 37, 97)
Output index order [i, j, alpha, beta]: A_ij[alpha, beta].
"""
from __future__ import annotations

import numpy as np

VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def lame(E: float, nu: float):
    """Lame constants of an isotropic material from Young's modulus and Poisson's ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def material_contravariant(gcon: np.ndarray, lam: float, mu: float) -> np.ndarray:
    """C^ijkl of eq. 84a as a (..., 3, 3, 3, 3) array."""
    return (lam * np.einsum("...ij,...kl->...ijkl", gcon, gcon)
            + mu * (np.einsum("...ik,...jl->...ijkl", gcon, gcon)
                    + np.einsum("...il,...jk->...ijkl", gcon, gcon)))


def voigt_matrix(C4: np.ndarray) -> np.ndarray:
    """The 6x6 matrix of eq. 93 from the 4th-order tensor."""
    out = np.empty(C4.shape[:-4] + (6, 6), dtype=C4.dtype)
    for I, (i, j) in enumerate(VOIGT):
        for K, (k, l) in enumerate(VOIGT):
            out[..., I, K] = C4[..., i, j, k, l]
    return out


def g_blocks(J: np.ndarray) -> np.ndarray:
    """G_1, G_2, G_3 of eq. 91 as (..., 3, 3, 6): [i, component, voigt column]."""
    g = [J[..., :, 0], J[..., :, 1], J[..., :, 2]]
    z = np.zeros_like(g[0])
    G1 = np.stack([g[0], z, z, z, g[2], g[1]], axis=-1)
    G2 = np.stack([z, g[1], z, g[2], z, g[0]], axis=-1)
    G3 = np.stack([z, z, g[2], g[1], g[0], z], axis=-1)
    return np.stack([G1, G2, G3], axis=-3)


def macro_field(J: np.ndarray, lam: float, mu: float) -> np.ndarray:
    """A_ij[alpha, beta] for Jacobians J (..., 3, 3) with J[p, i] = d M_p / d xi_i."""
    gcov = np.einsum("...pi,...pj->...ij", J, J)              # eq. 81 (g_i . g_j, no conjugation)
    gcon = np.linalg.inv(gcov)
    Cv = voigt_matrix(material_contravariant(gcon, lam, mu))   # eq. 84, 93
    G = g_blocks(J)                                            # eq. 91
    detJ = np.linalg.det(J)
    # |det J| (eq. 37), written as det J * sign(Re det J) so that a complex-step
    # perturbation of the control net stays analytic; equal to |det J| for real J
    detJ = detJ * np.sign(np.real(detJ))
    A = np.einsum("...iaV,...VW,...jbW->...ijab", G, Cv, G)    # eq. 37 / 97
    return A * detJ[..., None, None, None, None]


def macro_field_cartesian(J: np.ndarray, lam: float, mu: float) -> np.ndarray:
    """Independent Cartesian form used only to cross-check macro_field:
    A_ij[a,b] = |det J| (lam G_ia G_jb + mu delta_ab (G G^T)_ij + mu G_ib G_ja), G = J^-1.
    """
    G = np.linalg.inv(J)
    GGt = np.einsum("...ip,...jp->...ij", G, G)
    eye = np.eye(3)
    A = (lam * np.einsum("...ia,...jb->...ijab", G, G)
         + mu * np.einsum("...ij,ab->...ijab", GGt, eye)
         + mu * np.einsum("...ib,...ja->...ijab", G, G))
    return A * np.abs(np.linalg.det(J))[..., None, None, None, None]
