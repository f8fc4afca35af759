"""Compressible neo-Hookean material at quadrature points (oracle; test infrastructure only).

Eq. hypref (Section 3.2):  Psi(F) = mu/2 (tr C - tr I - 2 ln J) + lambda (ln J)^2,
C = F^T F, J = det F, natural logarithm.  The volumetric term is taken literally
(lambda, not lambda/2).

First Piola stress (Section 2.1, P = dPsi/dF):
    P = mu (F - F^{-T}) + 2 lambda ln J F^{-T}.
Tangent moduli (Eq. L, L = dP/dF), formed explicitly as a 3x3x3x3 array -- the "naive"
route of Section 3.2.1 that forms L and then contracts it:
    L[i,J,k,L] = mu d_ik d_JL + (mu - 2 lambda ln J) Finv[L,i] Finv[J,k]
                 + 2 lambda Finv[J,i] Finv[L,k].
All functions broadcast over leading dimensions of F (shape [..., 3, 3]).
"""
from __future__ import annotations

import numpy as np


class NonPositiveJacobian(ValueError):
    """det F <= 0 at a quadrature point: the neo-Hookean energy is undefined there."""


def _det_checked(F: np.ndarray) -> np.ndarray:
    J = np.linalg.det(F)
    if np.any(~(J > 0.0)):
        raise NonPositiveJacobian(f"det F <= 0 at {int(np.sum(~(J > 0.0)))} points")
    return J


def energy_density(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    J = np.linalg.det(F) if np.iscomplexobj(F) else _det_checked(F)
    trC = np.einsum("...ij,...ij->...", F, F)
    lnJ = np.log(J)
    return 0.5 * mu * (trC - 3.0 - 2.0 * lnJ) + lam * lnJ * lnJ


def piola(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    J = np.linalg.det(F) if np.iscomplexobj(F) else _det_checked(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(J)[..., None, None]
    return mu * (F - FinvT) + 2.0 * lam * lnJ * FinvT


def tangent_moduli(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    J = _det_checked(F)
    Fi = np.linalg.inv(F)
    lnJ = np.log(J)[..., None, None, None, None]
    eye = np.eye(3)
    term0 = np.einsum("ik,JL->iJkL", eye, eye)
    term1 = np.einsum("...Li,...Jk->...iJkL", Fi, Fi)
    term2 = np.einsum("...Ji,...Lk->...iJkL", Fi, Fi)
    return mu * term0 + (mu - 2.0 * lam * lnJ) * term1 + 2.0 * lam * term2
