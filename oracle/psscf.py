"""Algorithm 2 (Sec. 3.2.3): the PS scheme combined with filtering, step by
step in the paper's order, plus the unfiltered PS scheme.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import planner
from .sparse import CSR, alg1, axpy, matmul_add, norm1


@dataclass
class StepStat:
    kind: str  # "baby" (Eq. 11), "giant" (Eq. 14) or "odd" (F = Z G-hat, square mode)
    index: int  # k of Z-hat_(k) or i of S-hat_i
    threshold: float  # the bound the filter of this step must meet in Algorithm 2 (0 = unfiltered)
    nnz_pre: int
    nnz_post: int
    eps_f: float
    iters: int
    c: float


@dataclass
class Result:
    F: CSR
    plan: planner.Plan
    norms: list
    steps: list = field(default_factory=list)
    products: int = 0


def power_norms(Z: CSR):
    """||Z^i||_1 for i = 0..10, Z^i = Z Z^{i-1} unfiltered (Eq. 37 first case)."""
    norms = [1.0, norm1(Z)]
    P = Z
    for _ in range(2, planner.K_NORMEST + 1):
        P = matmul_add(Z, P)
        norms.append(norm1(P))
    return norms


def block(a, N: int, q: int, i: int, Zh: dict, n: int) -> CSR:
    """B-hat_i = sum_{j=0}^{q-1} a_{iq+j} Z-hat_(j), Z-hat_(0) = I (Eq. 13,
    Algorithm 2), accumulated in ascending j; not filtered."""
    X = None
    for j in range(q):
        idx = i * q + j
        alpha = a[idx] if idx < N and idx < len(a) else 0.0
        if alpha == 0.0:
            continue
        X = axpy(alpha, Zh[j] if j >= 1 else None, X, n)
    return X if X is not None else CSR.empty(n)


def _filter(C: CSR, bound: float, e_r: float, maxit: int):
    """Alg. 1 with eps_g chosen so that eps_g (1 + e_r) equals the bound."""
    eps_g = bound / (1.0 + e_r)
    return alg1(C, eps_g, e_r, maxit)


def psscf(Z: CSR, a, tol: float, *, poly: bool = False, filtered: bool = True, s: int = 0,
          e_r: float = 0.1, maxit: int = 1000, submult: bool = False,
          norms=None, square: bool = False) -> Result:
    """f(Z) ~ S-hat_{b-1} by Algorithm 2.

    ``filtered=False`` is the unfiltered PS scheme with the same N, q, b: every
    threshold is 0, which keeps every nonzero entry.  ``norms`` may pass
    precomputed ||Z^i||_1, i = 0..10.

    ``square=True`` substitutes W = Z^2 (``planner.split_even_odd``): W = Z Z
    unfiltered, then Algorithm 2 on g(W) with the norms z_i of W taken as
    z_{2i} of Z.  An odd series ends with the unfiltered product F = Z G-hat;
    since ||Z (g(W) - G-hat)|| <= ||Z||_1 ||g(W) - G-hat||, g is evaluated to
    eps_tol / ||Z||_1 (infinite for Z = 0).
    """
    n = Z.n
    a = [float(x) for x in a]
    if norms is None:
        norms = [1.0, norm1(Z)] if submult else power_norms(Z)  # step 1
    if not square:
        p = planner.plan(a, tol, norms, poly=poly, s=s, submult=submult)  # steps 2-3
        res = Result(CSR.empty(n), p, list(norms))
        res.F = _alg2(Z, a, p, res, filtered, e_r, maxit)
        return res
    c, odd = planner.split_even_odd(a)
    tol_g = tol
    if odd:
        tol_g = tol / norms[1] if norms[1] != 0.0 else math.inf
    p = planner.plan(c, tol_g, norms, poly=poly, s=s, submult=submult, stride=2)
    res = Result(CSR.empty(n), p, list(norms))
    W = matmul_add(Z, Z)
    res.products += 1
    G = _alg2(W, c, p, res, filtered, e_r, maxit)
    if odd:
        G = matmul_add(Z, G)
        res.products += 1
        res.steps.append(StepStat("odd", 1, 0.0, G.nnz, G.nnz, 0.0, 0, 0.0))
    res.F = G
    return res


def _alg2(Z: CSR, a, p: planner.Plan, res: Result, filtered: bool, e_r: float, maxit: int) -> CSR:
    """Steps 4-14 of Algorithm 2 with the plan ``p``; appends to ``res.steps``."""
    n = Z.n
    N, q, b, g = p.N, p.q, p.b, p.g
    if N == 1:
        return CSR.identity(n, a[0]) if a[0] != 0.0 else CSR.empty(n)

    # steps 4-7: baby steps Z-hat_(k+1) = filter(Z Z-hat_(k))
    Zh = {1: Z}
    for k in range(1, q):
        Zt = matmul_add(Z, Zh[k])
        res.products += 1
        bound = p.zeta[k + 1] if filtered else 0.0
        f = _filter(Zt, bound, e_r, maxit)
        Zh[k + 1] = f.kept
        res.steps.append(StepStat("baby", k + 1, bound, Zt.nnz, f.kept.nnz, f.eps_f, f.iters, f.c))

    # step 8: S-hat_0 = B-hat_{b-1}
    S = block(a, N, q, b - 1, Zh, n)
    # steps 9-13, i = 1..b-1 (Eq. 14)
    for i in range(1, b):
        B = block(a, N, q, b - 1 - i, Zh, n)
        if g == 1 and i == 1:
            # B_{b-1} = a_{(b-1)q} I: S_1 = B-hat_{b-2} + a_{(b-1)q} Z-hat_(q), no
            # product and no filter (Sec. 3.1.2, last sentence)
            alpha = a[(b - 1) * q]
            S = axpy(alpha, Zh[q], B, n) if alpha != 0.0 else B
            res.steps.append(StepStat("giant", i, 0.0, S.nnz, S.nnz, 0.0, 0, 0.0))
            continue
        St = matmul_add(Zh[q], S, B)
        res.products += 1
        bound = p.sigma[i] if filtered else 0.0
        f = _filter(St, bound, e_r, maxit)
        S = f.kept
        res.steps.append(StepStat("giant", i, bound, St.nnz, S.nnz, f.eps_f, f.iters, f.c))
    return S  # step 14
