"""Structured hexahedral Q_p mesh of the unit cube (oracle; test infrastructure only).

Section 2.2: the domain is subdivided into hexahedra carrying the continuous Q_p space with
(p n_c + 1)^d nodes (Section 3.3).  Here Omega = [0, 1]^3 with N^3 affine cubes of side
h = 1/N; M = pN + 1 nodes per direction.  Numbering (a reading: the paper does not fix it):
node (i, j, k) -> i + M (j + M k); DoF (c, node) -> c M^3 + node, component-major.
Element (ex, ey, ez) -> ex + N (ey + N ez); its local node (a, b, c) -> a + n (b + n c),
n = p + 1, which is global node (p ex + a, p ey + b, p ez + c).
"""
from __future__ import annotations

import numpy as np


class Mesh:
    def __init__(self, n_el: int, degree: int):
        if n_el < 1 or degree < 1:
            raise ValueError("need n_el >= 1 and degree >= 1")
        self.N = n_el
        self.p = degree
        self.n = degree + 1
        self.M = degree * n_el + 1
        self.h = 1.0 / n_el
        self.n_nodes = self.M ** 3
        self.n_dofs = 3 * self.n_nodes
        self.n_elements = n_el ** 3

    def node(self, i, j, k):
        return i + self.M * (j + self.M * k)

    def node_coords(self) -> np.ndarray:
        """X[node, 3] reference coordinates for GLL node positions inside each element."""
        from .tables import gll_nodes
        t = gll_nodes(self.p)
        x1 = np.empty(self.M)
        for e in range(self.N):
            x1[self.p * e:self.p * e + self.n] = (e + t) * self.h
        kk, jj, ii = np.meshgrid(x1, x1, x1, indexing="ij")
        return np.stack([ii.reshape(-1), jj.reshape(-1), kk.reshape(-1)], axis=1)

    def element_index(self, ex, ey, ez):
        return ex + self.N * (ey + self.N * ez)

    def element_nodes(self, elems=None) -> np.ndarray:
        """conn[e, a] = global node of local node a of element e (all elements by default)."""
        if elems is None:
            elems = np.arange(self.n_elements)
        elems = np.asarray(elems)
        ex = elems % self.N
        ey = (elems // self.N) % self.N
        ez = elems // (self.N * self.N)
        a = np.arange(self.n)
        la, lb, lc = np.meshgrid(a, a, a, indexing="ij")      # indexed [a, b, c]
        # local index a + n (b + n c): iterate c slowest, a fastest
        la = la.transpose(2, 1, 0).reshape(-1)
        lb = lb.transpose(2, 1, 0).reshape(-1)
        lc = lc.transpose(2, 1, 0).reshape(-1)
        gi = self.p * ex[:, None] + la[None, :]
        gj = self.p * ey[:, None] + lb[None, :]
        gk = self.p * ez[:, None] + lc[None, :]
        return self.node(gi, gj, gk)

    def elements_of_node(self, node: int) -> list[int]:
        """Elements whose closure contains the node."""
        i = node % self.M
        j = (node // self.M) % self.M
        k = node // (self.M * self.M)
        out = []
        def rng(g):
            lo = max(0, (g - 1) // self.p) if g % self.p == 0 else g // self.p
            hi = min(self.N - 1, g // self.p)
            return range(lo, hi + 1)
        for ez in rng(k):
            for ey in rng(j):
                for ex in rng(i):
                    out.append(self.element_index(ex, ey, ez))
        return out

    def constrained(self, bc: int) -> np.ndarray:
        """Boolean [3 * M^3] flags of Dirichlet DoFs for a boundary preset.

        bc 0: none.  bc 1: all components on the face x = 0.
        bc 2 (compression): all components on z = 0, the z component on z = 1.
        """
        flags = np.zeros((3, self.n_nodes), dtype=bool)
        idx = np.arange(self.n_nodes)
        i = idx % self.M
        k = idx // (self.M * self.M)
        if bc == 1:
            flags[:, i == 0] = True
        elif bc == 2:
            flags[:, k == 0] = True
            flags[2, k == self.M - 1] = True
        elif bc != 0:
            raise ValueError("unknown boundary preset")
        return flags.reshape(-1)

    def prescribed_values(self, bc: int, top_uz: float) -> np.ndarray:
        """Dirichlet values: zero everywhere except u_z = top_uz on z = 1 for the compression preset."""
        g = np.zeros((3, self.n_nodes))
        if bc == 2:
            k = np.arange(self.n_nodes) // (self.M * self.M)
            g[2, k == self.M - 1] = top_uz
        return g.reshape(-1)
