"""Finite-element operators of the neo-Hookean problem, plain definitions (oracle; test only).

Residual, Eq. F (Section 2.1), no traction:
    R_{c,I} = sum_e sum_q P(F_q)_{cd} dphi_I/dX_d (x_q) w_q h^3,  F = I + Grad u.
Tangent application, Eq. DF and Section 2.4 (W_i = K(u; du, phi_i)):
    W_{c,I} = sum_e sum_q L(F_q)_{c d k l} dDu_k/dX_l dphi_I/dX_d w_q h^3.
Quadrature: (p+1)^3 Gauss-Legendre points per element; the affine cube of side h has the
constant Jacobian determinant h^3.

Shape-function values and gradients at the points are evaluated directly as products of
1D Lagrange polynomials, O((p+1)^6) per element -- no sum factorisation -- and L is formed
explicitly per point (the "naive" route of Section 3.2.1).

Heterogeneous material (the paper's test has inclusions 100x stiffer, Section 3.1): an
optional per-element factor f_e multiplies mu and lambda on element e; both energies are
linear in (mu, lambda), so P, L and every element contribution scale by f_e.

Dirichlet handling (a reading; the paper does not state it for the operator): with D the
constrained DoFs, the constrained operator is  A du = P_f K P_f du + P_D du  (identity rows
and columns on D), and residual rows on D are zero.  bc = 0 gives the raw operator.
"""
from __future__ import annotations

import numpy as np

from .material import energy_density, piola, tangent_moduli
from .mesh import Mesh
from .tables import element_tables

_CHUNK = 4096


def reference_basis(p: int):
    """Phi[q, a] and Gref[q, a, d] on the unit reference cube, with quadrature weights W[q].

    q = qx + n (qy + n qz), a = ax + n (ay + n az); d = 0, 1, 2 for x, y, z.
    """
    _, _, wq, B, D = element_tables(p)
    n = p + 1
    nq = n ** 3
    Phi = np.zeros((nq, nq))
    Gref = np.zeros((nq, nq, 3))
    W = np.zeros(nq)
    for qz in range(n):
        for qy in range(n):
            for qx in range(n):
                q = qx + n * (qy + n * qz)
                W[q] = wq[qx] * wq[qy] * wq[qz]
                for az in range(n):
                    for ay in range(n):
                        for ax in range(n):
                            a = ax + n * (ay + n * az)
                            bx, by, bz = B[qx, ax], B[qy, ay], B[qz, az]
                            Phi[q, a] = bx * by * bz
                            Gref[q, a, 0] = D[qx, ax] * by * bz
                            Gref[q, a, 1] = bx * D[qy, ay] * bz
                            Gref[q, a, 2] = bx * by * D[qz, az]
    return Phi, Gref, W


class Operator:
    """Neo-Hookean operators on a structured mesh with Lame parameters (mu, lam)."""

    def __init__(self, mesh: Mesh, mu: float, lam: float, bc: int = 0, model: int = 0, factors=None):
        self.mesh = mesh
        self.mu = float(mu)
        self.lam = float(lam)
        self.bc = bc
        self.model = model
        self.factors = None if factors is None else np.asarray(factors, dtype=np.float64)
        self.Phi, self.Gref, self.W = reference_basis(mesh.p)
        self.G = self.Gref / mesh.h                     # physical gradients (affine cube)
        self.vol = self.W * mesh.h ** 3                 # w_q * J_q
        self.fixed = mesh.constrained(bc)

    # -- element-level pieces ---------------------------------------------------------
    def _local(self, vec, conn):
        """u_e[e, c, a] from a global [3 M^3] vector."""
        v = vec.reshape(3, -1)
        return np.stack([v[c][conn] for c in range(3)], axis=1)

    def gradients(self, vec, conn):
        """Grad u at every point of the listed elements: [e, q, c, d]."""
        ue = self._local(vec, conn)
        return np.einsum("eca,qad->eqcd", ue, self.G)

    def _scatter(self, out, conn, fe):
        o = out.reshape(3, -1)
        for c in range(3):
            np.add.at(o[c], conn, fe[:, c, :])

    def _chunks(self, elems=None):
        mesh = self.mesh
        if elems is None:
            elems = np.arange(mesh.n_elements)
        for s in range(0, len(elems), _CHUNK):
            sub = elems[s:s + _CHUNK]
            yield sub, mesh.element_nodes(sub)

    def _f(self, elems, shape_tail):
        """Material factors of the listed elements, shaped to broadcast over shape_tail."""
        if self.factors is None:
            return 1.0
        return self.factors[np.asarray(elems)].reshape((-1,) + (1,) * shape_tail)

    # -- global operators -------------------------------------------------------------
    def energy(self, u):
        """Discrete potential energy sum_e sum_q Psi(F_q) w_q h^3 (complex u allowed for complex-step checks)."""
        total = 0.0
        for sub, conn in self._chunks():
            F = np.eye(3) + self.gradients(u, conn)
            psi = energy_density(F, self.mu, self.lam, self.model) * self._f(sub, 1)
            total = total + np.einsum("eq,q->", psi, self.vol)
        return total

    def element_residuals(self, u, conn, elems):
        F = np.eye(3) + self.gradients(u, conn)
        P = piola(F, self.mu, self.lam, self.model)
        return np.einsum("eqcd,qad,q->eca", P, self.G, self.vol) * self._f(elems, 2)

    def residual(self, u, elems=None) -> np.ndarray:
        r = np.zeros(self.mesh.n_dofs, dtype=np.result_type(u, np.float64))
        for sub, conn in self._chunks(elems):
            self._scatter(r, conn, self.element_residuals(u, conn, sub))
        r[self.fixed] = 0.0
        return r

    def element_applies(self, u, du, conn, elems):
        F = np.eye(3) + self.gradients(u, conn)
        L = tangent_moduli(F, self.mu, self.lam, self.model)
        dH = self.gradients(du, conn)
        G = np.einsum("eqiJkL,eqkL->eqiJ", L, dH)          # G = L : Grad du
        return np.einsum("eqcd,qad,q->eca", G, self.G, self.vol) * self._f(elems, 2)

    def apply(self, u, du, elems=None) -> np.ndarray:
        """A du = P_f K(u) P_f du + P_D du."""
        dm = np.where(self.fixed, 0.0, du)
        v = np.zeros(self.mesh.n_dofs)
        for sub, conn in self._chunks(elems):
            self._scatter(v, conn, self.element_applies(u, dm, conn, sub))
        v[self.fixed] = du[self.fixed]
        return v

    def apply_rows(self, u, du, dofs) -> np.ndarray:
        """Rows `dofs` of A du, touching only the elements around those DoFs."""
        mesh = self.mesh
        dofs = np.asarray(dofs)
        nodes = dofs % mesh.n_nodes
        elems = sorted({e for nd in np.unique(nodes) for e in mesh.elements_of_node(int(nd))})
        elems = np.array(elems, dtype=np.int64)
        dm = np.where(self.fixed, 0.0, du)
        v = np.zeros(mesh.n_dofs)
        conn = mesh.element_nodes(elems)
        self._scatter(v, conn, self.element_applies(u, dm, conn, elems))
        out = v[dofs]
        fx = self.fixed[dofs]
        out[fx] = du[dofs][fx]
        return out

    def residual_rows(self, u, dofs) -> np.ndarray:
        mesh = self.mesh
        dofs = np.asarray(dofs)
        nodes = dofs % mesh.n_nodes
        elems = sorted({e for nd in np.unique(nodes) for e in mesh.elements_of_node(int(nd))})
        elems = np.array(elems, dtype=np.int64)
        r = np.zeros(mesh.n_dofs)
        conn = mesh.element_nodes(elems)
        self._scatter(r, conn, self.element_residuals(u, conn, elems))
        out = r[dofs]
        out[self.fixed[dofs]] = 0.0
        return out

    def diagonal_rows(self, u, dofs) -> np.ndarray:
        """Rows `dofs` of diag(A), touching only the elements around those DoFs."""
        mesh = self.mesh
        dofs = np.asarray(dofs)
        nodes = dofs % mesh.n_nodes
        elems = np.array(sorted({e for nd in np.unique(nodes) for e in mesh.elements_of_node(int(nd))}), dtype=np.int64)
        conn = mesh.element_nodes(elems)
        F = np.eye(3) + self.gradients(u, conn)
        L = tangent_moduli(F, self.mu, self.lam, self.model)
        de = np.einsum("eqcdcl,qal,qad,q->eca", L, self.G, self.G, self.vol) * self._f(elems, 2)
        d = np.zeros(mesh.n_dofs)
        self._scatter(d, conn, de)
        out = d[dofs]
        out[self.fixed[dofs]] = 1.0
        return out

    def element_matrix(self, u, e: int) -> np.ndarray:
        """K_e[(c,a), (k,b)] = sum_q L_{c d k l} G[q,b,l] G[q,a,d] w_q h^3 (raw, no Dirichlet)."""
        conn = self.mesh.element_nodes(np.array([e]))
        F = np.eye(3) + self.gradients(u, conn)[0]
        L = tangent_moduli(F, self.mu, self.lam, self.model)
        nq = self.G.shape[1]
        Ke = np.einsum("qcdkl,qbl,qad,q->cakb", L, self.G, self.G, self.vol)
        fe = 1.0 if self.factors is None else self.factors[e]
        return fe * Ke.reshape(3 * nq, 3 * nq)

    def assemble(self, u) -> np.ndarray:
        """Dense global matrix of the constrained operator (tiny meshes only)."""
        mesh = self.mesh
        n = mesh.n_dofs
        if n > 6000:
            raise ValueError("dense assembly is for tiny meshes")
        K = np.zeros((n, n))
        nn = mesh.n_nodes
        for e in range(mesh.n_elements):
            conn = mesh.element_nodes(np.array([e]))[0]
            gd = np.concatenate([c * nn + conn for c in range(3)])
            K[np.ix_(gd, gd)] += self.element_matrix(u, e)
        K[self.fixed, :] = 0.0
        K[:, self.fixed] = 0.0
        K[self.fixed, self.fixed] = 1.0
        return K

    def diagonal(self, u) -> np.ndarray:
        """diag(A): sum of element-matrix diagonals, 1 on constrained DoFs."""
        mesh = self.mesh
        d = np.zeros(mesh.n_dofs)
        for sub, conn in self._chunks():
            F = np.eye(3) + self.gradients(u, conn)
            L = tangent_moduli(F, self.mu, self.lam, self.model)
            de = np.einsum("eqcdcl,qal,qad,q->eca", L, self.G, self.G, self.vol) * self._f(sub, 2)
            self._scatter(d, conn, de)
        d[self.fixed] = 1.0
        return d

    def min_jacobian(self, u) -> float:
        m = np.inf
        for _, conn in self._chunks():
            F = np.eye(3) + self.gradients(u, conn)
            m = min(m, float(np.linalg.det(F).min()))
        return m
