"""Pins of the oracle's neo-Hookean point functions: complex-step derivatives, closed forms,
symmetry and objectivity (Eq. hypref, Eq. F, Eq. L)."""
import json
import os

import numpy as np
import pytest

from oracle.material import NonPositiveJacobian, energy_density, piola, tangent_moduli

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(7)


def random_F(count=5, scale=0.2):
    return np.eye(3) + scale * RNG.uniform(-1, 1, size=(count, 3, 3))


@pytest.mark.parametrize("mu,lam", [(1.0, 1.5), (1.0, 49.0), (0.4225, 0.6338)])
def test_piola_is_energy_gradient(mu, lam):
    F = random_F()
    P = piola(F, mu, lam)
    for i in range(3):
        for J in range(3):
            Fc = F.astype(complex)
            Fc[:, i, J] += 1e-30j
            dpsi = np.imag(energy_density(Fc, mu, lam)) / 1e-30
            assert np.allclose(dpsi, P[:, i, J], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("mu,lam", [(1.0, 1.5), (1.0, 49.0)])
def test_moduli_are_piola_derivative(mu, lam):
    F = random_F()
    L = tangent_moduli(F, mu, lam)
    for k in range(3):
        for l in range(3):
            Fc = F.astype(complex)
            Fc[:, k, l] += 1e-30j
            dP = np.imag(piola(Fc, mu, lam)) / 1e-30
            assert np.allclose(dP, L[:, :, :, k, l], rtol=1e-13, atol=1e-12)


def test_moduli_major_symmetry():
    L = tangent_moduli(random_F(), 1.0, 1.5)
    assert np.allclose(L, np.transpose(L, (0, 3, 4, 1, 2)), atol=1e-14)


def test_moduli_at_identity_is_isotropic_elasticity_with_two_lambda():
    mu, lam = 0.7, 1.3
    L = tangent_moduli(np.eye(3)[None], mu, lam)[0]
    d = np.eye(3)
    ref = (mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
           + 2.0 * lam * np.einsum("ij,kl->ijkl", d, d))
    assert np.allclose(L, ref, atol=1e-15)


def test_piola_closed_form_diagonal():
    gold = json.load(open(os.path.join(GOLD, "piola_diag.json")))["cases"]
    for c in gold:
        P = piola(np.diag(c["F"])[None], c["mu"], c["lam"])[0]
        assert np.allclose(np.diag(P), c["P_diag"], rtol=1e-14, atol=1e-15)
        assert np.allclose(P - np.diag(np.diag(P)), 0.0, atol=1e-15)


def test_energy_zero_and_stress_free_reference():
    assert abs(energy_density(np.eye(3)[None], 1.0, 1.5)[0]) < 1e-15
    assert np.allclose(piola(np.eye(3)[None], 1.0, 1.5), 0.0, atol=1e-15)


def test_objectivity():
    F = random_F(3)
    th = 0.7
    Q = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    QF = np.einsum("ij,ejk->eik", Q, F)
    assert np.allclose(energy_density(QF, 1.0, 1.5), energy_density(F, 1.0, 1.5), atol=1e-14)
    assert np.allclose(piola(QF, 1.0, 1.5), np.einsum("ij,ejk->eik", Q, piola(F, 1.0, 1.5)), atol=1e-14)


def test_nonpositive_jacobian_raises():
    F = np.diag([1.0, 1.0, -0.5])[None]
    with pytest.raises(NonPositiveJacobian):
        piola(F, 1.0, 1.5)
    with pytest.raises(NonPositiveJacobian):
        tangent_moduli(F, 1.0, 1.5)


# ---- split (isochoric-volumetric) neo-Hookean model, Eq. hypcomplex
@pytest.mark.parametrize("mu,kappa", [(1.0, 2.0), (0.4225, 100.0)])
def test_split_model_stress_and_moduli_are_derivatives(mu, kappa):
    F = random_F()
    P = piola(F, mu, kappa, 1)
    L = tangent_moduli(F, mu, kappa, 1)
    for i in range(3):
        for J in range(3):
            Fc = F.astype(complex)
            Fc[:, i, J] += 1e-30j
            assert np.allclose(np.imag(energy_density(Fc, mu, kappa, 1)) / 1e-30, P[:, i, J], rtol=1e-13, atol=1e-13)
            assert np.allclose(np.imag(piola(Fc, mu, kappa, 1)) / 1e-30, L[:, :, :, i, J], rtol=1e-13, atol=1e-12)
    assert np.allclose(L, np.transpose(L, (0, 3, 4, 1, 2)), atol=1e-13)


def test_split_model_isochoric_invariance_and_identity():
    mu, kappa = 0.8, 3.0
    # the isochoric part does not see volume changes: Psi(s F) - Psi_vol(s^3) = Psi(F) - Psi_vol(1) for det F = 1
    F = np.array([[1.1, 0.1, 0.0], [0.0, 1.0 / 1.1, 0.05], [0.0, 0.0, 1.0]])[None]
    assert abs(np.linalg.det(F[0]) - 1.0) < 1e-15
    s = 1.2
    vol = lambda J: 0.5 * kappa * (0.5 * (J * J - 1.0) - np.log(J))
    assert abs((energy_density(s * F, mu, kappa, 1) - vol(s ** 3)) - energy_density(F, mu, kappa, 1))[0] < 1e-13
    # stress free at F = I; at F = I the tangent is isotropic linear elasticity with (mu, kappa - 2 mu / 3)
    assert np.allclose(piola(np.eye(3)[None], mu, kappa, 1), 0.0, atol=1e-15)
    L = tangent_moduli(np.eye(3)[None], mu, kappa, 1)[0]
    d = np.eye(3)
    lam_eff = kappa - 2.0 * mu / 3.0
    ref = (mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
           + lam_eff * np.einsum("ij,kl->ijkl", d, d))
    assert np.allclose(L, ref, atol=1e-14)
