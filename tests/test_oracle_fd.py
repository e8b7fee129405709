"""Pins for the oracle's finite-difference weights and Laplacian (CPU only).

The weights are checked against (1) the order-2 stencil printed in Sec. IV-A1,
(2) an independent exact solve of the moment (Vandermonde) conditions that
define the centred second derivative, and the Laplacian against (3) its exact
discrete symbol on plane waves and (4) its measured convergence order.
"""

import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import fd, wave

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_order2_matches_printed_example():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fd_order2.txt")) if l.strip() and l[0] != "#"]
    printed = {int(j): Fraction(w) for j, w in rows}
    w = fd.fd_weights_exact(2)
    assert printed[0] == w[0]
    assert printed[1] == w[1] and printed[-1] == w[1]


def _moment_solve(R):
    """Solve sum_{j=-R..R} w_j j^(2p) = 2*[p==1], p = 0..R, for symmetric w
    by exact Gaussian elimination over the rationals."""
    n = R + 1
    A = [[Fraction(0)] * n for _ in range(n)]
    rhs = [Fraction(2 if p == 1 else 0) for p in range(n)]
    for p in range(n):
        A[p][0] = Fraction(1 if p == 0 else 0)
        for j in range(1, R + 1):
            A[p][j] = Fraction(2 * j ** (2 * p))
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        rhs[col], rhs[piv] = rhs[piv], rhs[col]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col] / A[col][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
                rhs[r] -= f * rhs[col]
    return [rhs[i] / A[i][i] for i in range(n)]


@pytest.mark.parametrize("so", fd.SPACE_ORDERS)
def test_weights_solve_moment_conditions(so):
    assert fd.fd_weights_exact(so) == _moment_solve(so // 2)


def test_known_order4_and_order8_values():
    assert fd.fd_weights_exact(4) == [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)]
    assert fd.fd_weights_exact(8) == [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5),
                                      Fraction(8, 315), Fraction(-1, 560)]


@pytest.mark.parametrize("so", [2, 8, 16])
def test_bad_orders_rejected(so):
    fd.radius(so)
    for bad in (0, 3, 18, -2):
        with pytest.raises(ValueError):
            fd.radius(bad)


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
@pytest.mark.parametrize("ndim", [2, 3])
def test_laplacian_symbol_on_plane_wave(so, ndim):
    """L sin(k.x) = -(sum_d k_eff,d^2) sin(k.x) away from the boundary, with
    k_eff^2 h^2 = -w_0 - 2 sum_j w_j cos(j k h)."""
    R = so // 2
    n = 3 * R + 8
    h = [10.0, 7.0, 12.5][:ndim]
    k = [0.031, 0.047, 0.023][:ndim]
    axes = [np.arange(n) * hd for hd in h]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    phase = sum(kd * g for kd, g in zip(k, grids))
    u = np.sin(phase + 0.3)
    L = wave.laplacian(u, so, h)
    w = fd.fd_weights(so)
    keff2 = 0.0
    for kd, hd in zip(k, h):
        keff2 += (-w[0] - 2 * sum(w[j] * np.cos(j * kd * hd) for j in range(1, R + 1))) / hd ** 2
    inner = tuple(slice(R, n - R) for _ in range(ndim))
    np.testing.assert_allclose(L[inner], -keff2 * u[inner], rtol=0, atol=1e-13 * keff2)


@pytest.mark.parametrize("so", [2, 4, 6, 8, 12, 16])
def test_laplacian_convergence_order(so):
    """Truncation error of L on a smooth field falls as h^so."""
    R = so // 2
    kappa = 1.0
    errs = []
    # high orders reach the asymptotic regime only at larger kh before round-off
    hs, tol = ([0.5, 0.25], 0.3) if so <= 8 else ([0.8, 0.5], 0.7)
    for hh in hs:
        n = 2 * R + 9
        x = np.arange(n) * hh
        u2 = np.sin(kappa * x)[None, :] * np.ones((n, 1))
        L = wave.laplacian(u2, so, [hh, hh])
        c = n // 2
        errs.append(abs(L[c, c] + kappa ** 2 * u2[c, c]) / abs(u2[c, c]))
    slope = np.log(errs[0] / errs[1]) / np.log(hs[0] / hs[1])
    assert slope > so - tol, (so, errs, slope)
