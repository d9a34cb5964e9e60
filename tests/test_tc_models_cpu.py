"""The exact models of the tensor-core arithmetic (tests/tc_models.py), pinned
on the CPU: the digits reconstruct the truncated fixed-point integers, and
the models stay within the error bounds the kernels document against exact
rational arithmetic and against the FP64 oracle of eq. (gram) and eq. (coords)."""
import math
from fractions import Fraction

import numpy as np

from oracle import ascg_oracle as O
from tc_models import bexp, digits55, gram_tc_model, recover_tc_model


def test_digits_reconstruct_the_truncated_integers():
    rng = np.random.default_rng(2)
    y = np.concatenate([rng.standard_normal(500) * 10.0 ** rng.uniform(-20, 0, 500), [0.0, -0.0, 5e-324, -1e-310]])
    emax = int(bexp(y).max())
    d = digits55(y, emax)
    assert all(np.all(np.abs(dk) <= 128) for dk in d)
    for i, v in enumerate(y):
        t = int(Fraction(float(v)) * Fraction(2) ** (55 - (emax - 1022)))  # truncation toward zero
        assert sum(int(d[k][i]) * 256 ** (6 - k) for k in range(7)) == t
        assert abs(t) < 2 ** 55


def _exact_gram(Y):
    w = Y.shape[0]
    F = [[Fraction(float(v)) for v in row] for row in Y]
    return [[sum(a * b for a, b in zip(F[i], F[j])) for j in range(w)] for i in range(w)]


def test_gram_model_within_its_bound():
    """|G_model - Y^T Y| <= 2^-51 (max|y_a| ||y_b||_1 + max|y_b| ||y_a||_1) +
    gamma_(parts+1) |y_a|^T |y_b| (truncation of each entry to the grid
    2^(E - 55), then FP64 rounding of the partials and their sum)."""
    rng = np.random.default_rng(5)
    w, n = 9, 3000
    Y = rng.standard_normal((w, n)) * 10.0 ** rng.uniform(-6, 0, (w, n)) * np.logspace(0, 5, w)[:, None]
    G = gram_tc_model(Y, sms=2)
    ex = _exact_gram(Y)
    a_ = np.abs(Y)
    mx, l1 = a_.max(axis=1), a_.sum(axis=1)
    eps = 2.0 ** -53
    parts = 2
    g = (parts + 2) * eps / (1 - (parts + 2) * eps)
    for i in range(w):
        for j in range(w):
            bound = 2.0 ** -51 * (mx[i] * l1[j] + mx[j] * l1[i]) + g * float(a_[i] @ a_[j])
            assert abs(Fraction(G[i, j]) - ex[i][j]) <= Fraction(bound)
    assert np.array_equal(G, G.T)


def test_recovery_model_within_its_bound():
    """|result - sum_j Y_ij c_j| <= 2^-53 |result| + 2^-54 sum_j ||y_j|| |c_j| +
    (w + 2) 2^-52 max_j ||y_j|| |c_j|, against exact rational sums; x' adds the
    rounding of x + (Y x')_i."""
    rng = np.random.default_rng(6)
    w, n = 17, 400
    Y = rng.standard_normal((w, n)) * 10.0 ** rng.uniform(-4, 0, (w, n)) * np.logspace(0, 6, w)[:, None]
    Y[5] = 0.0
    x = rng.standard_normal(n)
    cf = rng.standard_normal(3 * w) * 10.0 ** rng.uniform(-2, 2, 3 * w)
    got = recover_tc_model(Y, cf, x)
    ninf = np.abs(Y).max(axis=1)
    for v in range(3):
        c = cf[v * w:(v + 1) * w]
        bnd = 2.0 ** -54 * float(ninf @ np.abs(c)) + (w + 2) * 2.0 ** -52 * float(np.max(ninf * np.abs(c)))
        for i in range(0, n, 7):
            exact = sum(Fraction(float(Y[j, i])) * Fraction(float(c[j])) for j in range(w))
            if v == 0:
                exact += Fraction(float(x[i]))
                tol = 2.0 ** -52 * abs(got[0][i]) + bnd
            else:
                tol = 2.0 ** -53 * abs(got[v][i]) + bnd
            assert abs(Fraction(float(got[v][i])) - exact) <= Fraction(tol)
    # and the FP64 oracle of eq. (coords) agrees within the two bounds together
    xo, ro, po = O.recover(Y.T, x, cf[:w], cf[w:2 * w], cf[2 * w:])
    for g_, o_ in zip(got, (xo, ro, po)):
        assert np.allclose(g_, o_, rtol=1e-12, atol=1e-12 * float(np.abs(Y).max() * np.abs(cf).max()))
