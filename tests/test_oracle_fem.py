"""Pins of the oracle's finite-element operators against the mathematics (Eq. F, Eq. DF,
Section 2.4): energy gradient, residual derivative, symmetry, linear elasticity at u = 0,
rigid-body modes, the patch test and brute-force mesh bookkeeping."""
import numpy as np
import pytest

import nhmf_inputs as inp
from oracle.fem import Operator
from oracle.mesh import Mesh
from oracle.tables import element_tables

RNG = np.random.default_rng(11)


def rand_u(mesh, amp):
    return amp * mesh.h / mesh.p * RNG.uniform(-1, 1, mesh.n_dofs)


# ---------------------------------------------------------------- mesh bookkeeping
@pytest.mark.parametrize("N,p", [(2, 1), (3, 2), (2, 4)])
def test_element_nodes_brute_force(N, p):
    mesh = Mesh(N, p)
    conn = mesh.element_nodes()
    n = p + 1
    X = mesh.node_coords()
    for e in range(mesh.n_elements):
        ex, ey, ez = e % N, (e // N) % N, e // (N * N)
        for c in range(n):
            for b in range(n):
                for a in range(n):
                    node = conn[e, a + n * (b + n * c)]
                    assert node == (p * ex + a) + mesh.M * ((p * ey + b) + mesh.M * (p * ez + c))
        # all nodes of the element lie in its closed cube
        lo = np.array([ex, ey, ez]) * mesh.h
        assert np.all(X[conn[e]] >= lo - 1e-14) and np.all(X[conn[e]] <= lo + mesh.h + 1e-14)


@pytest.mark.parametrize("N,p", [(3, 1), (3, 2), (2, 3)])
def test_elements_of_node_brute_force(N, p):
    mesh = Mesh(N, p)
    conn = mesh.element_nodes()
    for node in range(mesh.n_nodes):
        ref = sorted(np.nonzero(np.any(conn == node, axis=1))[0].tolist())
        assert mesh.elements_of_node(node) == ref


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_constrained_sets_match_input_masks(bc):
    mesh = Mesh(3, 2)
    assert np.array_equal(mesh.constrained(bc), inp.dirichlet_mask(3, 2, bc).reshape(-1))


# ---------------------------------------------------------------- energy / residual / tangent
@pytest.mark.parametrize("p", [1, 2, 3])
def test_residual_is_energy_gradient(p):
    mesh = Mesh(2, p)
    op = Operator(mesh, 1.0, 1.5, bc=0)
    u = rand_u(mesh, 0.1)
    R = op.residual(u)
    idx = RNG.choice(mesh.n_dofs, size=40, replace=False)
    for i in idx:
        uc = u.astype(complex)
        uc[i] += 1e-30j
        g = np.imag(op.energy(uc)) / 1e-30
        assert abs(g - R[i]) <= 1e-13 * max(1.0, np.abs(R).max())


@pytest.mark.parametrize("p,lam", [(1, 1.5), (2, 1.5), (3, 49.0), (4, 1.5)])
def test_tangent_is_residual_derivative(p, lam):
    mesh = Mesh(2, p)
    op = Operator(mesh, 1.0, lam, bc=0)
    u = rand_u(mesh, 0.1)
    du = RNG.standard_normal(mesh.n_dofs)
    W = op.apply(u, du)
    # complex step: exact to rounding
    Rc = op.residual(u + 1e-30j * du)
    assert np.linalg.norm(np.imag(Rc) / 1e-30 - W) <= 1e-12 * np.linalg.norm(W)
    # central finite difference, relative error <= 1e-6
    eps = 1e-6
    fd = (op.residual(u + eps * du) - op.residual(u - eps * du)) / (2 * eps)
    assert np.linalg.norm(fd - W) <= 1e-6 * np.linalg.norm(W)


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_operator_symmetry(bc):
    mesh = Mesh(3, 2)
    op = Operator(mesh, 1.0, 1.5, bc=bc)
    u = rand_u(mesh, 0.1)
    u[mesh.constrained(bc)] = 0.0
    x = RNG.standard_normal(mesh.n_dofs)
    y = RNG.standard_normal(mesh.n_dofs)
    a, b = y @ op.apply(u, x), x @ op.apply(u, y)
    assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))


def voigt_elasticity_element_matrix(p, h, mu, lam_eff):
    """Independent Q_p element stiffness of isotropic linear elasticity (Voigt B-matrices)."""
    _, _, wq, B1, D1 = element_tables(p)
    n = p + 1
    nq = n ** 3
    C = np.zeros((6, 6))
    C[:3, :3] = lam_eff
    C[np.arange(3), np.arange(3)] += 2 * mu
    C[np.arange(3, 6), np.arange(3, 6)] = mu
    K = np.zeros((3 * nq, 3 * nq))
    for qz in range(n):
        for qy in range(n):
            for qx in range(n):
                Bm = np.zeros((6, 3 * nq))
                for az in range(n):
                    for ay in range(n):
                        for ax in range(n):
                            a = ax + n * (ay + n * az)
                            gx = D1[qx, ax] * B1[qy, ay] * B1[qz, az] / h
                            gy = B1[qx, ax] * D1[qy, ay] * B1[qz, az] / h
                            gz = B1[qx, ax] * B1[qy, ay] * D1[qz, az] / h
                            # engineering strains: xx, yy, zz, yz, xz, xy; dof column c*nq + a
                            Bm[0, a] = gx
                            Bm[1, nq + a] = gy
                            Bm[2, 2 * nq + a] = gz
                            Bm[3, nq + a] = gz; Bm[3, 2 * nq + a] = gy
                            Bm[4, a] = gz; Bm[4, 2 * nq + a] = gx
                            Bm[5, a] = gy; Bm[5, nq + a] = gx
                K += Bm.T @ C @ Bm * wq[qx] * wq[qy] * wq[qz] * h ** 3
    return K


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_reduces_to_linear_elasticity_at_zero(p):
    mesh = Mesh(2, p)
    mu, lam = 0.8, 1.7
    op = Operator(mesh, mu, lam, bc=0)
    Ke = op.element_matrix(np.zeros(mesh.n_dofs), 3)
    ref = voigt_elasticity_element_matrix(p, mesh.h, mu, 2.0 * lam)
    assert np.allclose(Ke, ref, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_rigid_body_modes(p):
    mesh = Mesh(2, p)
    op = Operator(mesh, 1.0, 1.5, bc=0)
    X = mesh.node_coords()
    u = rand_u(mesh, 0.1)
    scale = np.linalg.norm(op.apply(u, RNG.standard_normal(mesh.n_dofs)))
    for c in range(3):                               # translations, any u
        t = np.zeros((3, mesh.n_nodes)); t[c] = 1.0
        assert np.linalg.norm(op.apply(u, t.reshape(-1))) <= 1e-13 * scale
    Wm = np.array([[0.0, -0.3, 0.2], [0.3, 0.0, -0.5], [-0.2, 0.5, 0.0]])
    rot0 = (X @ Wm.T).T.reshape(-1)                  # infinitesimal rotation at u = 0
    assert np.linalg.norm(op.apply(np.zeros(mesh.n_dofs), rot0)) <= 1e-13 * scale
    # at u != 0: K(u)[W (X + u)] equals the integral of (W P) : Grad phi (objectivity)
    xcur = X.T + u.reshape(3, -1)
    lhs = op.apply(u, (Wm @ xcur).reshape(-1))
    conn = mesh.element_nodes()
    from oracle.material import piola
    F = np.eye(3) + op.gradients(u, conn)
    WP = np.einsum("ij,eqjd->eqid", Wm, piola(F, 1.0, 1.5))
    rhs = np.zeros(mesh.n_dofs)
    op._scatter(rhs, conn, np.einsum("eqcd,qad,q->eca", WP, op.G, op.vol))
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_patch_test_affine_deformation(p):
    mesh = Mesh(3, p)
    mu, lam = 1.0, 1.5
    op = Operator(mesh, mu, lam, bc=0)
    X = mesh.node_coords()
    F0 = np.array([[1.05, 0.02, 0.0], [0.01, 0.97, 0.03], [0.0, -0.02, 1.02]])
    u = ((F0 - np.eye(3)) @ X.T).reshape(-1)
    R = op.residual(u).reshape(3, -1)
    i = np.arange(mesh.n_nodes) % mesh.M
    j = (np.arange(mesh.n_nodes) // mesh.M) % mesh.M
    k = np.arange(mesh.n_nodes) // mesh.M ** 2
    interior = (i > 0) & (i < mesh.M - 1) & (j > 0) & (j < mesh.M - 1) & (k > 0) & (k < mesh.M - 1)
    assert np.abs(R[:, interior]).max() < 1e-13
    # reaction on face x = 1 is P(F0) N over a unit face: sum_c R_c = P_c1
    J = np.linalg.det(F0)
    Fi_T = np.linalg.inv(F0).T
    P0 = mu * (F0 - Fi_T) + 2 * lam * np.log(J) * Fi_T
    face = i == mesh.M - 1
    assert np.allclose(R[:, face].sum(axis=1), P0[:, 0], atol=1e-13)
    assert np.allclose(R[:, i == 0].sum(axis=1), -P0[:, 0], atol=1e-13)
    # the tangent applied to an affine direction vanishes on interior rows
    du = (np.array([[0.1, -0.2, 0.3], [0.0, 0.2, 0.1], [0.4, 0.0, -0.1]]) @ X.T).reshape(-1)
    W = op.apply(u, du).reshape(3, -1)
    assert np.abs(W[:, interior]).max() < 1e-13


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_assembled_matrix_and_diagonal(bc):
    mesh = Mesh(2, 2)
    op = Operator(mesh, 1.0, 1.5, bc=bc)
    u = rand_u(mesh, 0.1)
    u[mesh.constrained(bc)] = 0.0
    K = op.assemble(u)
    assert np.allclose(K, K.T, atol=1e-13)
    for j in RNG.choice(mesh.n_dofs, 12, replace=False):
        e = np.zeros(mesh.n_dofs); e[j] = 1.0
        assert np.allclose(op.apply(u, e), K[:, j], atol=1e-13)
    assert np.allclose(op.diagonal(u), np.diag(K), atol=1e-13)
    if bc != 0:
        # at u = 0 the constrained operator is linear elasticity: SPD with the Dirichlet rows
        assert np.all(np.linalg.eigvalsh(op.assemble(np.zeros(mesh.n_dofs))) > 0)


def test_row_extraction_matches_full_operators():
    mesh = Mesh(3, 2)
    op = Operator(mesh, 1.0, 1.5, bc=1)
    u = rand_u(mesh, 0.1); u[op.fixed] = 0.0
    du = RNG.standard_normal(mesh.n_dofs)
    rows = RNG.choice(mesh.n_dofs, 30, replace=False)
    assert np.allclose(op.apply_rows(u, du, rows), op.apply(u, du)[rows], atol=1e-14)
    assert np.allclose(op.residual_rows(u, rows), op.residual(u)[rows], atol=1e-14)


# ---- the split neo-Hookean model (Eq. hypcomplex) through the same operators
@pytest.mark.parametrize("p", [1, 2, 3])
def test_split_model_residual_and_tangent_are_derivatives(p):
    mesh = Mesh(2, p)
    op = Operator(mesh, 1.0, 5.0, bc=0, model=1)
    u = rand_u(mesh, 0.1)
    R = op.residual(u)
    for i in RNG.choice(mesh.n_dofs, 10, replace=False):
        uc = u.astype(complex)
        uc[i] += 1e-30j
        assert abs(np.imag(op.energy(uc)) / 1e-30 - R[i]) <= 1e-13 * max(1.0, np.abs(R).max())
    du = RNG.standard_normal(mesh.n_dofs)
    W = op.apply(u, du)
    Rc = op.residual(u + 1e-30j * du)
    assert np.linalg.norm(np.imag(Rc) / 1e-30 - W) <= 1e-12 * np.linalg.norm(W)
    x, y = RNG.standard_normal(mesh.n_dofs), RNG.standard_normal(mesh.n_dofs)
    a, b = y @ op.apply(u, x), x @ op.apply(u, y)
    assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))


# ---- heterogeneous material: per-element factors (stiff inclusions)
def test_element_factors_scale_contributions():
    mesh = Mesh(8, 1)
    f = inp.inclusion_factors(8, 100.0)
    assert set(np.unique(f)) == {1.0, 100.0}
    op = Operator(mesh, 1.0, 1.5, bc=0, factors=f)
    u = rand_u(mesh, 0.05)
    # residual = energy gradient and tangent = residual derivative still hold
    R = op.residual(u)
    for i in RNG.choice(mesh.n_dofs, 6, replace=False):
        uc = u.astype(complex); uc[i] += 1e-30j
        assert abs(np.imag(op.energy(uc)) / 1e-30 - R[i]) <= 1e-13 * np.abs(R).max()
    du = RNG.standard_normal(mesh.n_dofs)
    W = op.apply(u, du)
    assert np.linalg.norm(np.imag(op.residual(u + 1e-30j * du)) / 1e-30 - W) <= 1e-12 * np.linalg.norm(W)
    # a uniform factor scales the operator
    op2 = Operator(mesh, 1.0, 1.5, bc=0, factors=np.full(mesh.n_elements, 3.0))
    assert np.allclose(op2.apply(u, du), 3.0 * Operator(mesh, 1.0, 1.5, bc=0).apply(u, du), rtol=1e-13, atol=1e-13)


def test_diagonal_rows_match_full_diagonal():
    """The row-restricted diagonal (used at full size on sampled rows) equals rows of the full one."""
    w = inp.small(inp.WORKLOADS["q3_48_compress"], 3)
    u = inp.uniform_pm(77, w.n_dofs, 0.02)
    op = Operator(Mesh(w.n_el, w.degree), w.mu, w.lam, w.bc)
    rows = np.array([0, 5, 100, w.n_dofs // 2, w.n_dofs - 1, 2 * w.n_dofs // 3 + 7])
    assert np.allclose(op.diagonal_rows(u, rows), op.diagonal(u)[rows], rtol=1e-14, atol=0)
