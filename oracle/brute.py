"""P0: brute-force evaluation with exact Python integers (test infrastructure).

For tiny inputs only.  It evaluates the definition of the bivariate images
(paper Sect. 2.3, below Eq. 1) with unbounded integers: every term's value
a_i * prod_k (beta_k^t)^{e_ik} is formed exactly and only the final group sum
is reduced modulo p.  It shares no arithmetic with oracle.c (no modular
products at all) and so pins it independently.
"""
from __future__ import annotations

from typing import Dict, List, Tuple


def eval_exact(p: int, coeffs, exps, beta, T: int, t0: int = 1):
    """Returns (keys, rows): keys in descending lex order of (d, e); rows[r][g]
    is the coefficient of x1^d x2^e in f(x1, x2, beta^(t0+r)) mod p."""
    coeffs = [int(c) for c in coeffs]
    exps = [[int(x) for x in row] for row in exps]
    beta = [int(b) for b in beta]
    keys = sorted({(e[0], e[1]) for e in exps}, reverse=True)
    col = {k: g for g, k in enumerate(keys)}
    rows: List[List[int]] = []
    for r in range(T):
        t = t0 + r
        acc: Dict[Tuple[int, int], int] = {k: 0 for k in keys}
        for c, e in zip(coeffs, exps):
            v = c
            for k, b in enumerate(beta):
                v *= (b ** t) ** e[2 + k]          # exact, no reduction
            acc[(e[0], e[1])] += v
        rows.append([acc[k] % p for k in keys])
    return keys, rows
