"""B-spline basis functions in FP64 (oracle; test infrastructure only).

The paper represents every micro-block by an MFA tensor-product B-spline (Sec. 4.2:
knots, degree and NCP control points per axis; Fig. "Micro-model storage layout")
and refers to de Boor for the basis. The functions here write the textbook
definitions out:

* degree 0:  N_{i,0}(u) = 1 if t_i <= u < t_{i+1} else 0, with the right end of a
  clamped vector closed: at u = t_last the last non-empty interval is used
  (the usual convention, Piegl & Tiller A2.1);
* degree k:  N_{i,k}(u) = (u - t_i)/(t_{i+k} - t_i) N_{i,k-1}(u)
                        + (t_{i+k+1} - u)/(t_{i+k+1} - t_{i+1}) N_{i+1,k-1}(u),
  every 0/0 read as 0 (Cox-de Boor recurrence);
* derivative: N'_{i,p}(u) = p [N_{i,p-1}(u)/(t_{i+p} - t_i)
                              - N_{i+1,p-1}(u)/(t_{i+p+1} - t_{i+1})], 0/0 = 0.

Everything is vectorised over the parameter values only; no blocking, no reuse of
partial products between basis functions.
"""

import numpy as np


def _ratio(num, den):
    """num/den with the 0/0 (empty knot interval) convention: a zero denominator gives 0."""
    den = np.asarray(den, dtype=np.float64)
    if den == 0.0:
        return np.zeros_like(num)
    return num / den


def degree0(t, u):
    """Indicator functions N_{i,0}(u) for i = 0 .. len(t)-2, shape (len(u), len(t)-1)."""
    t = np.asarray(t, dtype=np.float64)
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    m = len(t) - 1
    N = np.zeros((len(u), m))
    for i in range(m):
        N[:, i] = ((t[i] <= u) & (u < t[i + 1])).astype(np.float64)
    # Closed right end: u equal to the last knot belongs to the last non-empty interval.
    last = max(i for i in range(m) if t[i] < t[i + 1])
    at_end = u == t[-1]
    N[at_end, :] = 0.0
    N[at_end, last] = 1.0
    return N


def basis_table(t, p, u):
    """All N_{i,k}(u) for k = 0..p, as a list of arrays (degree k -> shape (len(u), len(t)-1-k))."""
    t = np.asarray(t, dtype=np.float64)
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    levels = [degree0(t, u)]
    for k in range(1, p + 1):
        prev = levels[-1]
        m = len(t) - 1 - k
        N = np.zeros((len(u), m))
        for i in range(m):
            left = _ratio(u - t[i], t[i + k] - t[i]) * prev[:, i]
            right = _ratio(t[i + k + 1] - u, t[i + k + 1] - t[i + 1]) * prev[:, i + 1]
            N[:, i] = left + right
        levels.append(N)
    return levels


def basis(t, p, u):
    """N_{i,p}(u) for every i = 0 .. C-1 (C = len(t) - p - 1); shape (len(u), C)."""
    return basis_table(t, p, u)[p]


def basis_deriv(t, p, u):
    """dN_{i,p}/du for every i; shape (len(u), C). Zero for p = 0."""
    t = np.asarray(t, dtype=np.float64)
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    C = len(t) - p - 1
    if p == 0:
        return np.zeros((len(u), C))
    lower = basis_table(t, p - 1, u)[p - 1]  # shape (len(u), C + 1)
    dN = np.zeros((len(u), C))
    for i in range(C):
        a = _ratio(lower[:, i], t[i + p] - t[i])
        b = _ratio(lower[:, i + 1], t[i + p + 1] - t[i + 1])
        dN[:, i] = p * (a - b)
    return dN


def find_span(t, p, u):
    """Knot span index s with t_s <= u < t_{s+1}, p <= s <= C-1, for each u.

    At u = t_last the last non-empty span (s = C-1 for a clamped vector) is returned,
    matching the closed right end in :func:`degree0`. Binary search over the knots.
    """
    t = np.asarray(t, dtype=np.float64)
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    C = len(t) - p - 1
    out = np.empty(len(u), dtype=np.int64)
    for m, x in enumerate(u):
        if x >= t[C]:
            out[m] = C - 1
            continue
        lo, hi = p, C
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if x < t[mid]:
                hi = mid
            else:
                lo = mid
        out[m] = lo
    return out


def sample_params(n):
    """Parameter values of a micro-block's n regular samples: u_i = i/(n-1), endpoints included.

    The quotient is rounded to FP32 (the sample positions as an FP32 decoder computes
    them) and then widened: a sample can fall exactly on a knot (e.g. n = 64 with
    knots j/14 puts u_9 on 1/7), and the span there is an integer chosen by comparing
    u with that knot, so both sides must compare the same numbers.
    """
    i = np.arange(n, dtype=np.float32)
    return (i / np.float32(n - 1)).astype(np.float64)
