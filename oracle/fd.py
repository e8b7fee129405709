"""Central finite-difference weights for the second derivative (oracle, FP64).

Sec. IV-A1 of the paper expands ``f.dx2`` for a ``space_order`` set on the data
object and prints the order-2 case: ``(f(x-h) - 2 f(x) + f(x+h)) / h**2``.  For a
general even order ``so = 2R`` the expansion is the centred stencil over the
2R+1 points ``x + j h``, ``j = -R..R``, whose weights are the standard closed
form (Fornberg's centred second-derivative weights):

    w_0     = -2 * sum_{j=1..R} 1/j**2
    w_{+-j} =  2 * (-1)**(j+1) * (R!)**2 / (j**2 * (R-j)! * (R+j)!)

so that ``f''(x) ~= sum_j w_j f(x + j h) / h**2`` with error O(h**so).

Test infrastructure only (see the package docstring).
"""

from fractions import Fraction
from math import factorial

import numpy as np

SPACE_ORDERS = (2, 4, 6, 8, 10, 12, 14, 16)


def radius(space_order):
    """Stencil half-width R = so/2 for an even space order in [2, 16]."""
    so = int(space_order)
    if so not in SPACE_ORDERS:
        raise ValueError("space_order must be even and in [2, 16], got %r" % (space_order,))
    return so // 2


def fd_weights_exact(space_order):
    """Exact rational weights [w_0, w_1, ..., w_R] of the centred second derivative."""
    R = radius(space_order)
    w = [Fraction(0)] * (R + 1)
    for j in range(1, R + 1):
        w[j] = Fraction(2 * (-1) ** (j + 1) * factorial(R) ** 2,
                        j * j * factorial(R - j) * factorial(R + j))
    w[0] = -2 * sum(Fraction(1, j * j) for j in range(1, R + 1))
    return w


def fd_weights(space_order):
    """float64 weights [w_0, w_1, ..., w_R] (symmetric: w_{-j} = w_j)."""
    return np.array([float(x) for x in fd_weights_exact(space_order)], dtype=np.float64)
