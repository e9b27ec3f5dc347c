"""Pins for the oracle's Radau IIA tableau (Section 2 consistency and stability
function; Section 5 RadauIIA family, order 2s-1)."""
import numpy as np
import pytest

from oracle import tableau
from tests.golden.load import evaluate, load

G = load("radau_iia_closed_form.txt")


@pytest.mark.parametrize("s", [2, 3])
def test_matches_textbook_closed_form(s):
    A, b, c = tableau.radau_iia(s)
    np.testing.assert_allclose(c, evaluate(G[f"s{s}.c"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(A, evaluate(G[f"s{s}.A"]), rtol=0, atol=2e-15)
    np.testing.assert_allclose(b, evaluate(G[f"s{s}.b"]), rtol=0, atol=2e-15)


@pytest.mark.parametrize("s", [1, 2, 3, 4])
def test_consistency_and_order_conditions(s):
    A, b, c = tableau.radau_iia(s)
    assert tableau.check_consistency(A, b, c)
    # B(2s-1): only k <= s is imposed by the construction; k in (s, 2s-1] is not
    for k in range(1, 2 * s):
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 1e-13
    assert abs(b @ c ** (2 * s - 1) - 1.0 / (2 * s)) > 1e-6   # order is exactly 2s-1
    assert c[-1] == 1.0 and np.allclose(A[-1], b)              # stiffly accurate


def test_stability_function_closed_form_s2():
    A, b, _ = tableau.radau_iia(2)
    for z in [-0.3, -2.0, -50.0, 0.7 + 0.4j, -3 + 5j]:
        assert abs(tableau.stability_function(A, b, z) - evaluate(G["s2.R"], z=z)) < 1e-13


@pytest.mark.parametrize("s", [2, 3])
def test_l_stable_and_order(s):
    A, b, _ = tableau.radau_iia(s)
    assert abs(tableau.stability_function(A, b, -1e9)) < 1e-8   # r(-inf) = 0
    for y in np.linspace(-30, 30, 13):                            # |r(iy)| <= 1
        assert abs(tableau.stability_function(A, b, 1j * y)) <= 1 + 1e-12
    # local error of r(z) against exp(z) is O(z^(2s)) (order 2s-1)
    e1 = abs(tableau.stability_function(A, b, 0.1) - np.exp(0.1))
    e2 = abs(tableau.stability_function(A, b, 0.05) - np.exp(0.05))
    assert abs(np.log2(e1 / e2) - 2 * s) < 0.25


@pytest.mark.parametrize("fam,s", [("g", 2), ("g", 3), ("l", 2), ("l", 3)])
def test_gauss_lobatto_match_textbook(fam, s):
    A, b, c = (tableau.gauss if fam == "g" else tableau.lobatto_iiic)(s)
    np.testing.assert_allclose(c, evaluate(G[f"{fam}{s}.c"]), rtol=0, atol=2e-15)
    np.testing.assert_allclose(A, evaluate(G[f"{fam}{s}.A"]), rtol=0, atol=3e-15)
    np.testing.assert_allclose(b, evaluate(G[f"{fam}{s}.b"]), rtol=0, atol=2e-15)
    assert tableau.check_consistency(A, b, c)


@pytest.mark.parametrize("s", [2, 3, 4])
def test_gauss_order_and_stability(s):
    A, b, c = tableau.gauss(s)
    for k in range(1, 2 * s + 1):                         # order 2s
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 1e-13
    for y in np.linspace(-20, 20, 9):                     # |r(iy)| = 1: A-stable, not L-stable
        assert abs(abs(tableau.stability_function(A, b, 1j * y)) - 1.0) < 1e-12
    assert abs(abs(tableau.stability_function(A, b, -1e8)) - 1.0) < 1e-6


@pytest.mark.parametrize("s", [2, 3, 4])
def test_lobatto_iiic_order_and_stability(s):
    A, b, c = tableau.lobatto_iiic(s)
    for k in range(1, 2 * s - 1):                         # order 2s-2
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 1e-13
    assert np.allclose(A[:, 0], b[0]) and np.allclose(A[-1], b)   # a_i1 = b_1, stiffly accurate
    assert abs(tableau.stability_function(A, b, -1e9)) < 1e-7      # L-stable
