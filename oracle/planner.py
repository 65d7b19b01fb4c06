"""A-priori analysis of the filtered PS scheme, written out from the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every sum below is accumulated left to right in ascending index order, as
written in the paper, in plain FP64 (no fused operations).  Coefficients with
index >= N count as zero (Eq. 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

K_NORMEST = 10  # Eq. (37): exact norms up to ||Z^10||, Lemma 1 above


def ps_split(N: int, s: int = 0):
    """Eq. (6): q = floor(sqrt(N-1)), b = ceil(N/q), g = 1 iff N - q(b-1) = 1.

    ``s`` > 0 overrides q (clamped to N-1).  N = 1 returns q = 0 (the result
    is a_0 I and no product is formed).
    """
    if N <= 1:
        return 0, 1, 0
    q = math.isqrt(N - 1) if s <= 0 else min(s, N - 1)
    b = -(-N // q)
    g = 1 if N - q * (b - 1) == 1 else 0
    return q, b, g


def mult_count(N: int) -> int:
    """Eq. (5): number of matrix products of the PS scheme."""
    if N <= 2:
        return 0
    q, b, g = ps_split(N)
    return q + b - 2 - g


def z_sequence(norms, upto: int, submult: bool = False):
    """Eq. (37) with Lemma 1 (K = 10).

    ``norms[i]`` = ||Z^i||_1 for i = 0..10 (norms[0] = 1).  Returns z_0..z_upto:
    z_i = norms[i] for i <= 10 and alpha_10^i above, with
    alpha_10 = max_{k=5..10} ||Z^k||^(1/k).  ``submult`` gives the crude bound
    z_i = ||Z||^i of Sec. 2.2 instead (only norms[1] is used).
    """
    if submult:
        z1 = norms[1]
        return [1.0] + [z1 ** i for i in range(1, upto + 1)]
    alpha = max(norms[k] ** (1.0 / k) for k in range(5, K_NORMEST + 1))
    return [norms[i] if i <= K_NORMEST else alpha ** i for i in range(upto + 1)]


def tail(a, z, m: int) -> float:
    """sum_{i=m}^{M-1} |a_i| z_i over the supplied coefficients (Eq. 9/33)."""
    s = 0.0
    for i in range(m, len(a)):
        if a[i] != 0.0:
            s += abs(a[i]) * z[i]
    return s


def theta(tol: float, a, z):
    """Eq. (34): the smallest m >= 1 with tail(m) <= 0.5 tol.

    Returns None when only the empty tail (m = M) qualifies: the supplied
    coefficients then do not show the series has converged.
    """
    M = len(a)
    for m in range(1, M + 1):
        if tail(a, z, m) <= 0.5 * tol:
            return m if m < M else None
    return None


@dataclass
class Plan:
    N: int
    q: int
    b: int
    g: int
    z: list
    trunc: float  # truncation bound tail(N) (0 in polynomial mode)
    budget: float  # eps_tol - tail(N) (Eq. 35) or eps (Eq. 27)
    zeta: dict = field(default_factory=dict)  # k -> bound on ||zeta_k||, k = 2..q
    sigma: dict = field(default_factory=dict)  # j -> bound on ||Sigma_j||, j = 1+g..b-1
    d: dict = field(default_factory=dict)  # k -> d_k (Eq. 24)


def filter_bounds(a, N: int, q: int, b: int, g: int, z, budget: float):
    """Eqs. (24)-(26) and (28)/(36): d_k, then zeta_k and sigma_j."""

    def coef(idx):
        return a[idx] if idx < N and idx < len(a) else 0.0

    Mp = q + b - 2 - g
    # Eq. (25): ||B_i|| <= sum_j |a_{iq+j}| z_j
    normB = []
    for i in range(b):
        s = 0.0
        for j in range(q):
            s += abs(coef(i * q + j)) * z[j]
        normB.append(s)
    # Eq. (26): ||S_0|| = ||B_{b-1}||, ||S_i|| <= ||B_{b-1-i}|| + ||Z^q|| ||S_{i-1}||
    normS = [normB[b - 1]]
    for i in range(1, b):
        normS.append(normB[b - 1 - i] + z[q] * normS[i - 1])

    # Eq. (21): beta_{i,k} = sum_{l=k}^{q-1} |a_{iq+l}| z_{l-k}; beta_{i,q} = 0
    def beta(i, k):
        s = 0.0
        for l in range(k, q):
            s += abs(coef(i * q + l)) * z[l - k]
        return s

    d, zeta, sigma = {}, {}, {}
    for k in range(2, q + 1):
        s = 0.0
        for j in range(b):
            s_prev = normS[j - 1] if j >= 1 else 0.0  # ||S_{-1}|| = 0
            s += z[q * (b - 1 - j)] * (beta(b - 1 - j, k) + z[q - k] * s_prev)
        d[k] = s
        zeta[k] = budget / (s * Mp) if s * Mp != 0.0 else math.inf
    for j in range(1 + g, b):
        w = z[q * (b - 1 - j)] * Mp
        sigma[j] = budget / w if w != 0.0 else math.inf
    return d, zeta, sigma


def plan(a, tol: float, norms, poly: bool = False, s: int = 0, submult: bool = False,
         stride: int = 1) -> Plan:
    """Alg. 2 steps 1-3 plus the filtering-norm-thresholds.

    Series mode: N = Theta(tol, a, z) (Eq. 34), budget = tol - tail(N)
    (Eq. 35/36).  Polynomial mode: N = len(a), budget = tol (Eq. 27/28).

    ``stride`` = 2 plans the series in W = Z^2 (``split_even_odd``): the
    norms are still those of Z, and z_i of W is Eq. (37)'s z_{2i} of Z, a
    bound on ||W^i|| = ||Z^{2i}||.
    """
    a = [float(x) for x in a]
    M = len(a)
    zz = z_sequence(norms, stride * max(M, K_NORMEST + 1), submult)
    z = zz[::stride]
    if poly:
        N = M
        trunc = 0.0
        budget = tol
    else:
        N = theta(tol, a, z)
        if N is None:
            raise ValueError("series not converged within the supplied coefficients")
        trunc = tail(a, z, N)
        budget = tol - trunc
    q, b, g = ps_split(N, s)
    p = Plan(N, q, b, g, z, trunc, budget)
    if N >= 2:
        p.d, p.zeta, p.sigma = filter_bounds(a, N, q, b, g, z, budget)
    return p


def split_even_odd(a):
    """The substitution W = Z^2 for a series with only even or only odd
    powers (an adjacent variant; the paper evaluates cos with its zero odd
    coefficients in place, Eq. 40).

    Even: f(Z) = g(Z^2) with c_k = a_{2k}.  Odd: f(Z) = Z g(Z^2) with
    c_k = a_{2k+1}.  Returns (c, odd); raises ValueError when both parities
    have nonzero coefficients.  All-zero coefficients count as even.
    """
    a = [float(x) for x in a]
    even_nz = any(x != 0.0 for x in a[0::2])
    odd_nz = any(x != 0.0 for x in a[1::2])
    if even_nz and odd_nz:
        raise ValueError("the series has both even and odd powers")
    if odd_nz:
        return a[1::2], True
    return a[0::2], False
