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

Split (isochoric-volumetric) neo-Hookean model, Eq. hypcomplex (Section 3.3):
    Psi = mu/2 (tr Cbar - 3) + kappa/2 ((J^2 - 1)/2 - ln J),  Cbar = J^(-2/3) C,
    P   = mu a (F - I1/3 F^-T) + kappa/2 (J^2 - 1) F^-T,       a = J^(-2/3), I1 = F : F,
    L[i,J,k,L] = mu a d_ik d_JL - 2/3 mu a (F_iJ Finv_Lk + Finv_Ji F_kL)
                 + (2/9 mu a I1 + kappa J^2) Finv_Ji Finv_Lk
                 + (mu a I1/3 - kappa/2 (J^2 - 1)) Finv_Li Finv_Jk.
The functions below take the model as `model` (0 compressible, Eq. hypref; 1 split) and read
the second constant as lambda (model 0) or kappa (model 1).
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


def energy_density(F: np.ndarray, mu: float, lam: float, model: int = 0) -> np.ndarray:
    J = np.linalg.det(F) if np.iscomplexobj(F) else _det_checked(F)
    trC = np.einsum("...ij,...ij->...", F, F)
    lnJ = np.log(J)
    if model == 1:
        return 0.5 * mu * (J ** (-2.0 / 3.0) * trC - 3.0) + 0.5 * lam * (0.5 * (J * J - 1.0) - lnJ)
    return 0.5 * mu * (trC - 3.0 - 2.0 * lnJ) + lam * lnJ * lnJ


def piola(F: np.ndarray, mu: float, lam: float, model: int = 0) -> np.ndarray:
    J = np.linalg.det(F) if np.iscomplexobj(F) else _det_checked(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    if model == 1:
        I1 = np.einsum("...ij,...ij->...", F, F)[..., None, None]
        a = (J ** (-2.0 / 3.0))[..., None, None]
        J2 = (J * J)[..., None, None]
        return mu * a * (F - I1 / 3.0 * FinvT) + 0.5 * lam * (J2 - 1.0) * FinvT
    lnJ = np.log(J)[..., None, None]
    return mu * (F - FinvT) + 2.0 * lam * lnJ * FinvT


def tangent_moduli(F: np.ndarray, mu: float, lam: float, model: int = 0) -> np.ndarray:
    J = _det_checked(F)
    Fi = np.linalg.inv(F)
    eye = np.eye(3)
    term0 = np.einsum("ik,JL->iJkL", eye, eye)
    term1 = np.einsum("...Li,...Jk->...iJkL", Fi, Fi)
    term2 = np.einsum("...Ji,...Lk->...iJkL", Fi, Fi)
    if model == 1:
        x = lambda s: s[..., None, None, None, None]
        a = J ** (-2.0 / 3.0)
        I1 = np.einsum("...ij,...ij->...", F, F)
        J2 = J * J
        mixed = np.einsum("...iJ,...Lk->...iJkL", F, Fi) + np.einsum("...Ji,...kL->...iJkL", Fi, F)
        return (x(mu * a) * term0 - x(2.0 / 3.0 * mu * a) * mixed
                + x(2.0 / 9.0 * mu * a * I1 + lam * J2) * term2
                + x(mu * a * I1 / 3.0 - 0.5 * lam * (J2 - 1.0)) * term1)
    lnJ = np.log(J)[..., None, None, None, None]
    return mu * term0 + (mu - 2.0 * lam * lnJ) * term1 + 2.0 * lam * term2
