"""Cardinal B-spline particle shapes (oracle; test infrastructure only).

Section 2.2 (the PIC charge and current densities) defines the grid quantities
through a particle shape function S; section 4.1 and section 5 state that S is a
tensor product of 1-D B-splines (quadratic in the text, higher orders in the
DIRK-2 refinement study of section 5.1).  Here the 1-D shape of degree p is the
centred cardinal B-spline W_p with unit integral, so a particle at xi = x/dx (in
cell units) gives node i the weight W_p(xi - i).

The value is computed with the Cox-de Boor recursion on the integer knots
0, 1, ..., p+1 (de Boor, "A Practical Guide to Splines", ch. 9) -- deliberately not
with the closed-form piecewise polynomials, which the tests use as the independent
check.
"""
import numpy as np


def cardinal_bspline(t, p):
    """W_p(t): centred cardinal B-spline of degree p, evaluated by Cox-de Boor.

    W_p(t) = N_{0,p}(t + (p+1)/2), where N_{i,k} are the B-splines on the integer
    knot sequence: N_{i,0}(s) = 1 on [i, i+1) and
        N_{i,k}(s) = (s - i)/k * N_{i,k-1}(s) + (i + k + 1 - s)/k * N_{i+1,k-1}(s).
    """
    t = np.asarray(t, dtype=np.float64)
    s = t + 0.5 * (p + 1)
    basis = [((s >= i) & (s < i + 1)).astype(np.float64) for i in range(p + 1)]
    for k in range(1, p + 1):
        basis = [((s - i) / k) * basis[i] + ((i + k + 1 - s) / k) * basis[i + 1]
                 for i in range(p + 1 - k)]
    return basis[0]


def first_node(xi, p):
    """Lowest grid node whose weight W_p(xi - i) can be nonzero.

    The support of W_p(xi - i) is |xi - i| < (p+1)/2, which holds for the p+1
    integers i = floor(xi - (p+1)/2) + 1, ..., floor(xi - (p+1)/2) + p + 1.
    """
    return np.floor(np.asarray(xi, dtype=np.float64) - 0.5 * (p + 1)).astype(np.int64) + 1


def node_weights(xi, p):
    """Node indices (unwrapped) and weights of a degree-p shape at positions xi.

    Returns (i0, w) with i0 of shape (n,) and w of shape (n, p+1): node i0 + a gets
    weight w[:, a] = W_p(xi - (i0 + a)).
    """
    xi = np.asarray(xi, dtype=np.float64)
    i0 = first_node(xi, p)
    w = np.stack([cardinal_bspline(xi - (i0 + a), p) for a in range(p + 1)], axis=-1)
    return i0, w
