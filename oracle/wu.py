"""Two-point resistance of a uniform free-boundary M x N mesh (test infrastructure).

Paper Sec. II-B, Eq. 3 (Wu's closed form).  Reading of the typeset formula:
"cos(x1 + 1/2) theta_m" means cos((x1 + 1/2) * theta_m); coordinates are 0-based,
x in [0, M) along the direction of the r-segments, y in [0, N) along the
s-segments; theta_m = m pi / M, phi_n = n pi / N.

  R = (r/N)|x1-x2| + (s/M)|y1-y2|
      + 2/(MN) sum_{m=1}^{M-1} sum_{n=1}^{N-1}
        [c_m(x1) d_n(y1) - c_m(x2) d_n(y2)]^2 / (r^-1 (1-cos theta_m) + s^-1 (1-cos phi_n))
  with c_m(x) = cos((x+1/2) theta_m), d_n(y) = cos((y+1/2) phi_n).

The double sum runs in long double.  The paper evaluates the cosines with a
multiple-angle recursion instead of cos calls (Sec. III-E); `cos_half_table`
implements that recursion (the Chebyshev three-term relation
cos((x+1)a) = 2 cos(a) cos(x a) - cos((x-1) a)) and `cos_half_direct` the
plain calls, so a test can pin one against the other.
"""
from __future__ import annotations

import numpy as np

LD = np.longdouble


def cos_half_direct(M):
    """T[m, x] = cos((x + 1/2) m pi / M) for m, x in [0, M)."""
    m = np.arange(M, dtype=LD)[:, None]
    x = np.arange(M, dtype=LD)[None, :]
    return np.cos((x + LD(0.5)) * m * LD(np.pi) / LD(M))


def cos_half_table(M):
    """Same table by the multiple-angle recursion in x:
    c(0) = cos(theta/2), c(-1) = cos(-theta/2) = c(0), c(x+1) = 2 cos(theta) c(x) - c(x-1)."""
    T = np.empty((M, M), dtype=LD)
    theta = np.arange(M, dtype=LD) * LD(np.pi) / LD(M)
    two_c = LD(2) * np.cos(theta)
    prev = np.cos(theta / LD(2))
    cur = prev.copy()
    T[:, 0] = cur
    for x in range(1, M):
        nxt = two_c * cur - prev
        prev, cur = cur, nxt
        T[:, x] = cur
    return T


def reff_wu(M, N, r, s, p1, p2, recursion=False):
    """Effective resistance between p1 = (x1, y1) and p2 = (x2, y2) on the M x N mesh."""
    (x1, y1), (x2, y2) = p1, p2
    r, s = LD(r), LD(s)
    R = r / LD(N) * abs(x1 - x2) + s / LD(M) * abs(y1 - y2)
    if M < 2 or N < 2:
        return float(R)
    cx = cos_half_table(M) if recursion else cos_half_direct(M)
    cy = cos_half_table(N) if recursion else cos_half_direct(N)
    th = np.arange(1, M, dtype=LD) * LD(np.pi) / LD(M)
    ph = np.arange(1, N, dtype=LD) * LD(np.pi) / LD(N)
    den = (LD(1) - np.cos(th))[:, None] / r + (LD(1) - np.cos(ph))[None, :] / s
    num = cx[1:, x1][:, None] * cy[1:, y1][None, :] - cx[1:, x2][:, None] * cy[1:, y2][None, :]
    R = R + LD(2) / (LD(M) * LD(N)) * np.sum(num * num / den)
    return float(R)


def reff_wu_matrix(M, N, r, s, points, recursion=False):
    """All pairwise Wu resistances among `points` (list of (x, y))."""
    P = len(points)
    out = np.zeros((P, P))
    for a in range(P):
        for b in range(a + 1, P):
            out[a, b] = out[b, a] = reff_wu(M, N, r, s, points[a], points[b], recursion)
    return out
