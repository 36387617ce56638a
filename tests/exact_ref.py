"""Exact reference arithmetic for pinning the oracle on tiny inputs.

Written independently of ``oracle/`` (exact rationals and Python integers, no
floating point), straight from the definitions: Eq. (3) min1, Eq. (4) min2,
Eq. (7) diamond, the row-wise matrix product of Alg. 1, l1 normalisation
(Eq. (6)), the min-covariance of Eq. (5) and the integer fixed-point rule of
the integer storage.  Used only by the tests.
"""
from __future__ import annotations

from fractions import Fraction as Fr


def sign(x) -> int:
    return (x > 0) - (x < 0)


def term(op: str, a, b):
    if op == "min1":
        return sign(a) * sign(b) * min(abs(a), abs(b))
    if op == "min2":
        return min(abs(a), abs(b)) if sign(a) == sign(b) else 0
    if op == "diamond":
        return sign(a) * b + a * sign(b)
    if op == "dot":
        return a * b
    raise ValueError(op)


def vecprod(op, w, x):
    return sum((term(op, a, b) for a, b in zip(w, x)), Fr(0))


def matvec(op, A, w):
    return [vecprod(op, row, w) for row in A]


def l1_step(op, A, w):
    """One MAPI step without start normalisation: y/||y||_1."""
    y = matvec(op, A, w)
    s = sum(abs(v) for v in y)
    if s == 0:
        raise ZeroDivisionError("zero l1 norm")
    return [v / s for v in y]


def mapi_raw(op, A, w0, T):
    """T exact MAPI steps from w0 taken as given; returns all iterates."""
    w = [Fr(v) for v in w0]
    out = []
    for _ in range(T):
        w = l1_step(op, A, w)
        out.append(w)
    return out


def mincov(op, X, denom):
    """C_pq = sum_n term(X_pn, X_qn) / denom (X as a list of D rows)."""
    D = len(X)
    return [[vecprod(op, X[p], X[q]) / denom for q in range(D)] for p in range(D)]


def pair_step(op, X, w, denom):
    D, N = len(X), len(X[0])
    t = [sum((term(op, X[d][n], w[d]) for d in range(D)), Fr(0)) for n in range(N)]
    return [sum((term(op, X[d][n], t[n]) for n in range(N)), Fr(0)) / denom
            for d in range(D)]


def int_normalise(y, q):
    """sign(y_i) * floor((|y_i| 2^q + floor(L/2)) / L), L = sum |y_i|."""
    L = sum(abs(v) for v in y)
    if L == 0:
        raise ZeroDivisionError("zero l1 norm")
    return [sign(v) * ((abs(v) * 2 ** q + L // 2) // L) for v in y]


def mapi_int(op, Aq, q, x0, T):
    """Integer MAPI: start x0 (already integers in units 2^-q), l1-normalised
    by the integer rule, then T exact integer steps."""
    w = int_normalise(list(x0), q)
    hist = []
    for _ in range(T):
        y = [sum(term(op, a, b) for a, b in zip(row, w)) for row in Aq]
        w = int_normalise(y, q)
        hist.append(w)
    return hist


def parse_fraction_row(text: str):
    return [Fr(tok) for tok in text.split()]


def parse_matrix(text: str):
    return [parse_fraction_row(r) for r in text.split(";")]
