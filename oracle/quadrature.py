"""Grundmann-Moeller quadrature on the n-simplex (oracle; test infrastructure only).

Grundmann & Moeller (1978), "Invariant integration formulas for the n-simplex
by combinatorial methods": for an integer s >= 0 the rule of degree d = 2s+1 on
the unit n-simplex is

    Q f = sum_{i=0..s} (-1)^i 2^(-2s) (d+n-2i)^d / (i! (d+n-i)!)
              * sum_{|beta| = s-i} f( (2 beta_0 + 1)/(d+n-2i), ..., (2 beta_n + 1)/(d+n-2i) ),

beta ranging over (n+1)-tuples of non-negative integers and the point given in
barycentric coordinates.  The weights of this form sum to the simplex volume
1/n!; ``gm_rule`` returns them rescaled to sum to one, so a rule is applied to
a simplex of volume V as  V * sum_q w_q f(x_q).

Pinned by tests against the closed-form simplex moments
    mean over the simplex of prod_j lambda_j^a_j = n! prod_j a_j! / (|a| + n)!.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def _compositions(total, parts):
    """All tuples of ``parts`` non-negative integers summing to ``total``."""
    for c in itertools.combinations(range(total + parts - 1), parts - 1):
        prev = -1
        out = []
        for x in c:
            out.append(x - prev - 1)
            prev = x
        out.append(total + parts - 1 - prev - 1)
        yield tuple(out)


def gm_rule(n: int, s: int):
    """Return (bary, w): barycentric points (m, n+1) and weights (m,) summing to 1."""
    d = 2 * s + 1
    pts, wts = [], []
    for i in range(s + 1):
        denom = d + n - 2 * i
        weight = ((-1) ** i) * 2.0 ** (-2 * s) * denom ** d / (math.factorial(i) * math.factorial(d + n - i))
        for beta in _compositions(s - i, n + 1):
            pts.append([(2 * b + 1) / denom for b in beta])
            wts.append(weight)
    w = np.array(wts) * math.factorial(n)
    return np.array(pts, dtype=np.float64), w


# degree-7 rules: exact for the cut-cell integrands (degree <= 6)
TET_BARY, TET_W = gm_rule(3, 3)
TRI_BARY, TRI_W = gm_rule(2, 3)
