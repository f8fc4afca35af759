"""Pins of the oracle's Newton solver: it reaches the residual tolerance, satisfies the
Dirichlet data, and for a tiny load it reduces to linear elasticity (first-order agreement)."""
import numpy as np
import pytest

from oracle.fem import Operator
from oracle.mesh import Mesh
from oracle.solver import newton_load_steps


def test_newton_converges_and_satisfies_bc():
    mesh = Mesh(2, 2)
    op = Operator(mesh, 1.0, 1.5, bc=2)
    u, hist = newton_load_steps(op, steps=2, compression=0.1)
    assert all(h["rel_residual"] <= 1e-8 for h in hist)
    g = mesh.prescribed_values(2, -0.1)
    assert np.array_equal(u[op.fixed], g[op.fixed])
    R = op.residual(u)
    assert np.linalg.norm(R) <= 1e-9 * np.linalg.norm(op.apply(u, u))


def test_small_load_matches_linear_elasticity():
    mesh = Mesh(2, 2)
    op = Operator(mesh, 1.0, 1.5, bc=2)
    eps = 1e-5
    u, _ = newton_load_steps(op, steps=1, compression=eps)
    # linear elasticity with the same Dirichlet data: K0 u_lin = 0 on free rows, u_lin = g on D
    raw = Operator(mesh, 1.0, 1.5, bc=0)
    K0 = raw.assemble(np.zeros(mesh.n_dofs))
    g = mesh.prescribed_values(2, -eps)
    f = op.fixed
    ul = g.copy()
    free = ~f
    ul[free] = np.linalg.solve(K0[np.ix_(free, free)], -K0[np.ix_(free, f)] @ g[f])
    # geometric nonlinearity is second order in the load
    assert np.linalg.norm(u - ul) <= 1e-3 * np.linalg.norm(ul)


def test_resume_reproduces_the_path():
    mesh = Mesh(2, 1)
    op = Operator(mesh, 1.0, 49.0, bc=2)
    u_all, _ = newton_load_steps(op, steps=3, compression=0.06)
    u_12, _ = newton_load_steps(op, steps=3, compression=0.06, last=2)
    u_3, _ = newton_load_steps(op, steps=3, compression=0.06, first=3, u0=u_12)
    assert np.array_equal(u_all, u_3)
