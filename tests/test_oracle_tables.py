"""Pins of the oracle's 1D tables against closed forms and polynomial exactness."""
import json
import os

import numpy as np
import pytest

from oracle.tables import element_tables, gauss_legendre, gll_nodes, lagrange_derivatives, lagrange_values

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_exact_to_degree_2n_minus_1(n):
    x, w = gauss_legendre(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-15
    # degree 2n is not integrated exactly (the rule is not over-exact by accident)
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


def test_gll_closed_forms():
    gold = json.load(open(os.path.join(GOLD, "gll_nodes.json")))["nodes"]
    for p, ref in gold.items():
        assert np.allclose(gll_nodes(int(p)), ref, atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", [1, 2])
def test_gll_equals_equispaced_low_degree(p):
    assert np.allclose(gll_nodes(p), np.linspace(0, 1, p + 1), atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_cardinal_and_reproduction(p):
    nodes = gll_nodes(p)
    assert np.allclose(lagrange_values(nodes, nodes), np.eye(p + 1), atol=1e-14)
    x = np.linspace(-0.3, 1.2, 17)
    L = lagrange_values(nodes, x)
    D = lagrange_derivatives(nodes, x)
    for m in range(p + 1):
        assert np.allclose(L @ nodes ** m, x ** m, atol=1e-12)
        dm = m * x ** (m - 1) if m > 0 else np.zeros_like(x)
        assert np.allclose(D @ nodes ** m, dm, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_element_tables_shapes_and_symmetry(p):
    nodes, xq, wq, B, D = element_tables(p)
    n = p + 1
    assert B.shape == (n, n) and D.shape == (n, n)
    # mirror symmetry of symmetric node/point sets: B[n-1-q, n-1-i] = B[q, i], D antisymmetric
    assert np.allclose(B[::-1, ::-1], B, atol=1e-14)
    assert np.allclose(D[::-1, ::-1], -D, atol=1e-12)
    assert abs(wq.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mirror_structure_used_by_the_even_odd_passes(p):
    """The GLL nodes and the Gauss points are symmetric about 1/2, so the interpolation B and
    the weighted transpose B^T w are centro-symmetric (M[n-1-r][n-1-m] = M[r][m]) and the
    collocation derivative Dc at the Gauss points is anti-centro-symmetric; for odd n the
    middle Gauss point is the middle GLL node x = 1/2, so B's centre row is e_h and the centre
    column of B^T w vanishes off the centre.  The GPU passes in even-odd form rely on these."""
    n = p + 1
    xq, wq = gauss_legendre(n)
    nodes = gll_nodes(p)
    B = lagrange_values(nodes, xq)          # B[q][i] = l_i(x_q)
    Dc = lagrange_derivatives(xq, xq)       # Dc[q][m] = l^G_m'(x_q)
    BWt = (B * wq[:, None]).T               # (B^T w)[i][q] = B[q][i] w_q
    flip = lambda M: M[::-1, ::-1]
    assert np.allclose(flip(B), B, atol=1e-14)
    assert np.allclose(flip(BWt), BWt, atol=1e-14)
    assert np.allclose(flip(Dc), -Dc, atol=1e-12)
    assert np.allclose(Dc.sum(axis=1), 0.0, atol=1e-12)          # derivative of a constant
    if n % 2 == 1:
        h = n // 2
        assert abs(xq[h] - 0.5) <= 1e-15 and abs(nodes[h] - 0.5) <= 1e-15
        e = np.zeros(n)
        e[h] = 1.0
        assert np.allclose(B[h], e, atol=1e-15)
        assert np.allclose(np.delete(BWt[:, h], h), 0.0, atol=1e-15)
