"""Independent checks the oracle is pinned to (no oracle code here).

Each helper restates a fact that the paper or plain mathematics fixes, in a
formulation different from the oracle's edge loop: the dense matrix product
(M + M^T) W, exact rational arithmetic over node pairs, exact rounding of a
rational to float32.
"""
from __future__ import annotations

import json
import os
import re
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_hand_cases():
    with open(os.path.join(GOLDEN, "hand_cases.json")) as f:
        return json.load(f)["cases"]


_TERM = re.compile(r"^\s*(-?\d+)(?:/(\d+))?(?:\*sqrt\((\d+)\))?\s*$")


def parse_exact(text: str) -> float:
    """'p/q', 'p/q*sqrt(r)' or a ' + '-separated sum of those, as a float."""
    total = 0.0
    for term in text.split("+"):
        m = _TERM.match(term)
        if m is None:
            raise ValueError(f"bad exact value {text!r}")
        num = Fraction(int(m.group(1)), int(m.group(2) or 1))
        total += float(num) * (float(np.sqrt(int(m.group(3)))) if m.group(3) else 1.0)
    return total


def parse_fraction(text: str) -> Fraction:
    """Rational hand value (no square roots)."""
    m = _TERM.match(text)
    if m is None or m.group(3):
        raise ValueError(f"not rational: {text!r}")
    return Fraction(int(m.group(1)), int(m.group(2) or 1))


def dense_projection(Y, K):
    """W (n x K) with W[i, Y[i]] = 1 / count(Y = Y[i]); zero rows for -1."""
    Y = np.asarray(Y)
    W = np.zeros((Y.size, K))
    for k in range(K):
        idx = np.flatnonzero(Y == k)
        if idx.size:
            W[idx, k] = 1.0 / idx.size
    return W


def dense_adjacency(edges, n, weights=None):
    """A = M + M^T with M[u, v] = sum of weights of listed edges (u, v)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(e.shape[0]) if weights is None else np.asarray(weights, np.float64)
    M = np.zeros((n, n))
    np.add.at(M, (e[:, 0], e[:, 1]), w)
    return M + M.T


def dense_embedding(edges, Y, K, weights=None):
    """Closed form Z = (M + M^T) W."""
    n = len(Y)
    return dense_adjacency(edges, n, weights) @ dense_projection(Y, K)


def pairwise_exact(edges, Y, K):
    """Exact rational Z for unit weights by summing over node pairs:
    Z[u, k] = sum_v A[u, v] [Y[v] = k] / n_k with A = M + M^T counted as
    integers."""
    n = len(Y)
    A = [[0] * n for _ in range(n)]
    for u, v in edges:
        A[u][v] += 1
        A[v][u] += 1
    nk = [sum(1 for y in Y if y == k) for k in range(K)]
    Z = [[Fraction(0)] * K for _ in range(n)]
    for u in range(n):
        for v in range(n):
            if A[u][v] and Y[v] >= 0:
                Z[u][Y[v]] += Fraction(A[u][v], nk[Y[v]])
    return Z


def pairwise_exact_weighted(edges, w, Y, K):
    """Exact rational Z for dyadic edge weights (each w exactly a float32 of
    few bits) by summing over node pairs: A[u, v] = sum of the weights of the
    listed edges {u, v}, counted in both directions, then
    Z[u, k] = sum_v A[u, v] [Y[v] = k] / n_k."""
    n = len(Y)
    A = [[Fraction(0)] * n for _ in range(n)]
    for (u, v), x in zip(edges, w):
        q = Fraction(float(x))
        A[u][v] += q
        A[v][u] += q
    nk = [sum(1 for y in Y if y == k) for k in range(K)]
    Z = [[Fraction(0)] * K for _ in range(n)]
    for u in range(n):
        for v in range(n):
            if A[u][v] != 0 and Y[v] >= 0:
                Z[u][Y[v]] += A[u][v] / nk[Y[v]]
    return Z


def pairwise_laplacian_decimal(edges, w, Y, K, digits=40):
    """Z of the normalised adjacency D^-1/2 A D^-1/2 with non-negative
    weights, node pair by node pair, in `digits`-digit decimal arithmetic:
    A and the weighted degrees d_u = sum_v A[u, v] exactly as rationals, then
    Z[u, k] = sum_v A[u, v] / sqrt(d_u d_v) [Y[v] = k] / n_k."""
    import decimal
    ctx = decimal.Context(prec=digits)
    n = len(Y)
    A = [[Fraction(0)] * n for _ in range(n)]
    for (u, v), x in zip(edges, w):
        q = Fraction(float(x))
        A[u][v] += q
        A[v][u] += q
    d = [sum(row) for row in A]
    nk = [sum(1 for y in Y if y == k) for k in range(K)]

    def dec(q: Fraction):
        return ctx.divide(decimal.Decimal(q.numerator), decimal.Decimal(q.denominator))

    Z = [[decimal.Decimal(0)] * K for _ in range(n)]
    for u in range(n):
        for v in range(n):
            if A[u][v] != 0 and Y[v] >= 0:
                root = ctx.sqrt(dec(d[u] * d[v]))
                term = ctx.divide(dec(A[u][v] / nk[Y[v]]), root)
                Z[u][Y[v]] = ctx.add(Z[u][Y[v]], term)
    return Z


def round_fraction_to_f32(q: Fraction) -> np.float32:
    """Correctly rounded (nearest, ties to even) float32 of a non-negative
    rational, computed with exact integer arithmetic (normal range only)."""
    if q == 0:
        return np.float32(0.0)
    if q < 0:
        raise ValueError("non-negative only")
    e = q.numerator.bit_length() - q.denominator.bit_length()
    # scale so that 2^23 <= m < 2^24
    while True:
        scaled = q * (Fraction(2) ** (23 - e))
        if scaled >= 2 ** 24:
            e += 1
        elif scaled < 2 ** 23:
            e -= 1
        else:
            break
    fl = scaled.numerator // scaled.denominator
    rem = scaled - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return np.float32(float(Fraction(fl) * (Fraction(2) ** (e - 23))))
