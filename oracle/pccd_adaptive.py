"""Partial CCD with a sample density chosen per pair from the bound of
Eq. (sample_bound) -- part of the ORACLE (test infrastructure only).

Sec. 4.1: for a pair whose exact time of impact t* satisfies t* <= alpha, the
query Q(lambda) = (p2^1 - p1^1) . (p2^0 - p1^0) is at most
-(1/alpha - 1) (H^0)^2 at the contact parameters lambda*, and its gradient
in lambda is bounded by 2 sqrt(2) L (H^1 + 2L) (Eq. derivative_bound), so
Q < 0 on the disc of radius

    rho* = (1/alpha - 1) (H^0)^2 / (2 sqrt(2) L (H^1 + 2L))

around lambda*.  Here H^0 is the closest distance of the two primitives at
t = 0, H^1 an upper bound of their distance over the step (the largest
vertex-to-vertex distance at t = 0 or t = 1: distances between points of
linearly moving primitives are convex in the points and in t), and L the
longest edge of either primitive at t = 0 or t = 1.  A square lattice of
spacing h in lambda covers its domain to h / sqrt(2), so h <= sqrt(2) rho*
puts a sample inside that disc.  The samples are the t = 0 closest point plus
the lattice {(i h, j h)} over the pair's parameter domain (VT: barycentric
weights (b1, b2) of the triangle's second and third vertex, b1 + b2 <= 1;
EE: (s, t) in [0, 1]^2), with h = 1 / m, m = ceil(1 / (sqrt(2) rho*)) capped
at max_axis.  The activity test is R7's: min over samples of
Q - dhat |p2^0 - p1^0| <= 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import collide

_VT_EDGES = ((1, 2), (2, 3), (3, 1))
_EE_EDGES = ((0, 1), (2, 3))


def sample_bound(q0, q1, kind, alpha):
    """rho* of Eq. (sample_bound) for one pair (quads [4][3] at t = 0, 1)."""
    q0 = np.asarray(q0, dtype=np.float64)
    q1 = np.asarray(q1, dtype=np.float64)
    c = collide.closest_coef(q0, kind)
    h0 = float(np.linalg.norm(c @ q0))
    first, second = ((0,), (1, 2, 3)) if kind == 0 else ((0, 1), (2, 3))
    h1 = max(float(np.linalg.norm(q[j] - q[i])) for q in (q0, q1) for i in first for j in second)
    edges = _VT_EDGES if kind == 0 else _EE_EDGES
    L = max(float(np.linalg.norm(q[j] - q[i])) for q in (q0, q1) for i, j in edges)
    if L <= 0.0:
        return math.inf
    return (1.0 / alpha - 1.0) * h0 * h0 / (2.0 * math.sqrt(2.0) * L * (h1 + 2.0 * L))


def lattice(kind, m):
    """Parameter samples of spacing 1/m over the pair's domain."""
    g = np.arange(m + 1, dtype=np.float64) / m
    a, b = np.meshgrid(g, g, indexing="ij")
    a, b = a.ravel(), b.ravel()
    if kind == 0:
        keep = (np.arange(m + 1)[:, None] + np.arange(m + 1)[None, :]).ravel() <= m
        a, b = a[keep], b[keep]
    return np.stack([a, b], axis=1)


def _points(q, kind, lam):
    """p1, p2 at parameters lam [k, 2] for one configuration q [4][3]."""
    if kind == 0:
        p1 = np.repeat(q[0][None, :], len(lam), axis=0)
        p2 = q[1][None, :] + lam[:, :1] * (q[2] - q[1])[None, :] + lam[:, 1:] * (q[3] - q[1])[None, :]
    else:
        p1 = q[0][None, :] + lam[:, :1] * (q[1] - q[0])[None, :]
        p2 = q[2][None, :] + lam[:, 1:] * (q[3] - q[2])[None, :]
    return p1, p2


def partial_ccd_adaptive(X0, X1, pairs, kinds, dhat, alpha, max_axis=64):
    """Per pair: active flag, margin min_s(Q - dhat |d0|), lattice size m and
    whether m was capped at max_axis (the guarantee then no longer holds)."""
    pairs = np.asarray(pairs).reshape(-1, 4)
    n = len(pairs)
    act = np.zeros(n, dtype=bool)
    margin = np.zeros(n)
    msize = np.zeros(n, dtype=np.int64)
    capped = np.zeros(n, dtype=bool)
    X0 = np.asarray(X0, dtype=np.float64)
    X1 = np.asarray(X1, dtype=np.float64)
    for i in range(n):
        kind = int(kinds[i])
        q0, q1 = X0[pairs[i]], X1[pairs[i]]
        rho = sample_bound(q0, q1, kind, alpha)
        need = math.inf if rho <= 0.0 else 1.0 / (math.sqrt(2.0) * rho)
        m = max(1, int(math.ceil(need))) if math.isfinite(need) else max_axis
        if m > max_axis:
            m, capped[i] = max_axis, True
        msize[i] = m
        c = collide.closest_coef(q0, kind)
        lam0 = np.array([[c[2], c[3]]]) if kind == 0 else np.array([[-c[1], c[3]]])
        lam = np.concatenate([lam0, lattice(kind, m)])
        a0, b0 = _points(q0, kind, lam)
        a1, b1 = _points(q1, kind, lam)
        d0 = b0 - a0
        Q = np.sum((b1 - a1) * d0, axis=1)
        mar = float(np.min(Q - dhat * np.linalg.norm(d0, axis=1)))
        margin[i] = mar
        act[i] = mar <= 0.0
    return act, margin, msize, capped
