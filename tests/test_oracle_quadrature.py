"""Pins of the oracle's quadrature (oracle/quadrature.py) against library roots and closed forms."""
import itertools
import math

import numpy as np
import pytest
import scipy.special as sps

from oracle.quadrature import gauss_jacobi, simplex_rule


@pytest.mark.parametrize("n,a,b", [(1, 0, 0), (3, 0, 0), (5, 0, 0), (5, 1, 0), (5, 2, 0), (6, 1.5, 0.5)])
def test_gauss_jacobi_matches_library_roots(n, a, b):
    x, w = gauss_jacobi(n, a, b)
    xr, wr = sps.roots_jacobi(n, a, b)
    o, orr = np.argsort(x), np.argsort(xr)
    assert np.allclose(x[o], xr[orr], atol=1e-14, rtol=0)
    assert np.allclose(w[o], wr[orr], atol=1e-14, rtol=1e-13)


def _simplex_monomial(exps):
    # int over the reference simplex of prod xi_k^{e_k} = prod e_k! / (sum e_k + d)!
    d = len(exps)
    return math.prod(math.factorial(e) for e in exps) / math.factorial(sum(exps) + d)


@pytest.mark.parametrize("dim", [2, 3])
def test_simplex_rule_exact_to_degree_9(dim):
    pts, w = simplex_rule(dim, 5)
    for exps in itertools.product(range(10), repeat=dim):
        if sum(exps) > 9:
            continue
        val = float(np.sum(w * np.prod(pts ** np.array(exps), axis=1)))
        assert val == pytest.approx(_simplex_monomial(exps), rel=1e-12, abs=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_simplex_rule_not_exact_beyond_degree(dim):
    # 2 points per direction integrate degree <= 3 only: degree 4 must show an error
    pts, w = simplex_rule(dim, 2)
    exps = (4,) + (0,) * (dim - 1)
    val = float(np.sum(w * pts[:, 0] ** 4))
    assert abs(val - _simplex_monomial(exps)) > 1e-6
