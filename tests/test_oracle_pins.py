"""Pins for the CPU oracle: each test checks it against something other than itself.

Exact rational arithmetic, closed forms, SVD, exactly rounded sums, the
paper's rounding bounds (eq. (E) and eq. (fb)), and the qualitative claims of
Sec. 5. No GPU is needed.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import ascg_oracle as O

EPS = 2.0 ** -53
HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# helpers written here, independent of the oracle
# ---------------------------------------------------------------------------

def frac_array(a):
    out = np.empty(np.shape(a), dtype=object)
    flat = out.reshape(-1)
    for i, v in enumerate(np.asarray(a).reshape(-1)):
        flat[i] = Fraction(v.item() if hasattr(v, "item") else v)  # python ints: no overflow
    return out


def frac_solve(D, b):
    """Gaussian elimination in exact rational arithmetic (no pivoting needed: SPD)."""
    n = len(b)
    M = [[Fraction(int(D[i][j])) for j in range(n)] + [Fraction(int(b[i]))] for i in range(n)]
    for k in range(n):
        for i in range(k + 1, n):
            f = M[i][k] / M[k][k]
            for j in range(k, n + 1):
                M[i][j] -= f * M[k][j]
    x = [Fraction(0)] * n
    for i in reversed(range(n)):
        x[i] = (M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))) / M[i][i]
    return x


def small_int_spd(n, seed):
    rng = np.random.default_rng(seed)
    L = rng.integers(-2, 3, size=(n, n))
    D = L.T @ L + 3 * np.eye(n, dtype=np.int64)
    return D.astype(np.int64)


def exact_operator(D):
    return O.Operator.from_dense(frac_array(D))


# ---------------------------------------------------------------------------
# Alg. 1 / 2 / 3 in exact arithmetic
# ---------------------------------------------------------------------------

def test_classical_cg_exact_finite_termination():
    """Classical CG (Alg. 1) in rational arithmetic reaches r = 0 and x = A^{-1} b in <= n steps."""
    D = small_int_spd(6, 1)
    b = np.array([1, -2, 0, 3, 1, -1])
    A = exact_operator(D)
    res = O.classical_cg(A, frac_array(b), frac_array(np.zeros(6)), exact=True, max_iters=6)
    assert all(v == 0 for v in res.r)
    assert list(res.x) == frac_solve(D, b)
    assert res.iters <= 6


@pytest.mark.parametrize("seq", [[1], [2], [3], [5], [2, 1, 3], [1, 4], [3, 2, 1]])
@pytest.mark.parametrize("basis", ["monomial", "chebyshev", "newton", "three_term"])
def test_sstep_equals_classical_exact(seq, basis):
    """s-step CG (Alg. 2) and variable s-step CG (Alg. 3) give the classical iterates exactly.

    The paper states this in Sec. 1 and Sec. 3.2. Checked after every block, in exact
    rational arithmetic, for three polynomial bases.
    """
    n = 7
    D = small_int_spd(n, 2)
    b = frac_array(np.array([2, -1, 1, 0, 3, -2, 1]))
    x1 = frac_array(np.zeros(n))
    A = exact_operator(D)
    smax = max(seq)
    if basis == "monomial":
        bp = O.monomial_params(smax, one=Fraction(1), zero=Fraction(0))
    elif basis == "chebyshev":
        bp = O.chebyshev_params(Fraction(1, 2), Fraction(40), smax)
    elif basis == "newton":
        bp = O.BasisParams([Fraction(k + 1, 3) for k in range(smax)], [Fraction(0)] * smax,
                           [Fraction(1)] * smax, "newton")
    else:
        # a general three-term recurrence: theta_j, sigma_j and gamma_j all differ
        # with j, so an index slip anywhere in the recurrence or in B shows
        bp = O.BasisParams([Fraction(2 * k + 1, 5) for k in range(smax)],
                           [Fraction(k + 2, 7) for k in range(smax)],
                           [Fraction(k + 3, 4) for k in range(smax)], "three_term")
    total = n - 1   # stop before r = 0 exactly (finite termination at step n)
    ss = O.variable_sstep_cg(A, b, x1, seq, bp, max_iters=total, exact=True)
    assert ss.iters == total
    m = 0
    for blk in ss.blocks:
        m += blk["s_k"]
    cl = O.classical_cg(A, b, x1, exact=True, max_iters=total)
    assert list(ss.x) == list(cl.x)
    assert list(ss.r) == list(cl.r)
    assert list(ss.p) == list(cl.p)
    assert ss.alphas == cl.alphas
    assert ss.betas == cl.betas


def test_finite_termination_fp64():
    """d distinct, well separated eigenvalues: ||r_{d+1}|| / ||b|| <= 1e-10 in FP64."""
    rng = np.random.default_rng(3)
    n, d = 60, 5
    lam = np.repeat([1.0, 2.0, 3.5, 6.0, 9.0], n // d)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Dm = (Q * lam) @ Q.T
    Dm = (Dm + Dm.T) / 2
    A = O.Operator.from_dense(Dm)
    b = rng.standard_normal(n)
    b /= np.linalg.norm(b)
    cl = O.classical_cg(A, b, np.zeros(n), eps_target=0.0, max_iters=d)
    assert cl.res_hist[d] <= 1e-10
    ss = O.fixed_sstep_cg(A, b, np.zeros(n), d, O.chebyshev_params(1.0, 9.0, d), eps_target=0.0, max_iters=d)
    assert ss.res_hist[d] <= 1e-9
    assert O.norm2(O.residual(A, b, ss.x)) <= 1e-9


# ---------------------------------------------------------------------------
# inputs: closed-form Poisson eigenvalues (used for the Chebyshev interval)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,m", [(2, 3), (2, 7), (2, 10), (3, 3), (3, 5)])
def test_poisson_closed_form_eigenvalues(dim, m):
    A = W.poisson2d(m) if dim == 2 else W.poisson3d(m)
    ev = np.linalg.eigvalsh(A.to_dense())
    np.testing.assert_allclose(ev, W.poisson_eigenvalues(dim, m), rtol=0, atol=1e-13)
    lo, hi = W.poisson_eig_bounds(dim, m)
    assert abs(lo - ev[0]) <= 1e-13 and abs(hi - ev[-1]) <= 1e-13


def test_workload_sizes():
    A = W.poisson2d(32)
    assert A.n == 1024 and A.nnz == 4992
    m = 128
    assert 7 * m ** 3 - 6 * m ** 2 == 14581760   # 3D 7-point nonzeros on 128^3
    assert 5 * 2048 ** 2 - 4 * 2048 == 20963328  # 2D 5-point nonzeros on 2048^2
    F = W.fv_diffusion2d(16, 2.0, np.random.default_rng(0))
    assert F.nnz == 5 * 256 - 4 * 16
    d = F.to_dense()
    assert np.array_equal(d, d.T)
    assert np.all(np.linalg.eigvalsh(d) > 0)


# ---------------------------------------------------------------------------
# basis recurrence, eq. (polybasiscg), (AVVB), rounding bound eq. (E)
# ---------------------------------------------------------------------------

def _exact_residual_norm(Ad, Yu, Y, B):
    """|| A Yunder - Y B ||_2 of the given floating-point arrays, formed exactly."""
    AF, YuF, YF, BF = frac_array(Ad), frac_array(Yu), frac_array(Y), frac_array(B)
    E = AF @ YuF - YF @ BF
    return np.linalg.norm(E.astype(np.float64), 2)


@pytest.mark.parametrize("basis", ["monomial", "chebyshev", "newton", "three_term"])
def test_basis_recurrence_bound_E(basis):
    """||A Yunder - Y B|| <= eps((3+N_A)||A|| ||Yunder|| + 4 ||Y|| ||B||), eq. (E)."""
    c = W.scaled("poisson2d", 6, 5)
    A = O.Operator.from_csr(c["A"])
    s = 6
    if basis == "monomial":
        bp = O.monomial_params(s)
    elif basis == "chebyshev":
        bp = O.chebyshev_params(c["lam"][0], c["lam"][1], s)
    elif basis == "newton":
        bp = O.newton_params(np.linspace(1.9, 0.1, s), s)
    else:
        lo, hi = c["lam"]
        bp = O.BasisParams([(lo + hi) / 2 + 0.1 * k for k in range(s)], [0.2 + 0.05 * k for k in range(s)],
                           [0.6 + 0.1 * k for k in range(s)], "three_term")
    rng = np.random.default_rng(4)
    p = rng.standard_normal(A.n)
    r = rng.standard_normal(A.n)
    Y = O.matrix_powers(A, p, r, s, bp)
    B = O.basis_change_matrix(s, bp)
    Yu = Y.copy()
    Yu[:, s] = 0.0
    Yu[:, 2 * s] = 0.0
    Ad = A.dense()
    lhs = _exact_residual_norm(Ad, Yu, Y, B)
    nA, nY, nYu, nB = (np.linalg.norm(M, 2) for M in (Ad, Y, Yu, B))
    bound = EPS * ((3 + A.N_A) * nA * nYu + 4 * nY * nB)
    assert lhs <= bound
    # a transposed B or a dropped gamma leaves an O(||A|| ||Y||) residual
    assert _exact_residual_norm(Ad, Yu, Y, B.T) > 1e3 * bound
    Bbad = B.copy()
    Bbad[s + 2, s + 1] = 0.0
    assert _exact_residual_norm(Ad, Yu, Y, Bbad) > 1e3 * bound


@pytest.mark.parametrize("basis", ["monomial", "chebyshev", "newton"])
def test_basis_closed_form_on_diagonal(basis):
    """On A = diag(lambda), rho_j(A) v = rho_j(lambda) * v with rho_j in closed form."""
    lam = np.linspace(0.05, 1.95, 40)
    A = O.Operator.from_dense(np.diag(lam))
    v = np.random.default_rng(6).standard_normal(40)
    s = 8
    if basis == "monomial":
        bp = O.monomial_params(s)
        closed = [lam ** j * v for j in range(s + 1)]
    elif basis == "chebyshev":
        lo, hi = 0.05, 1.95
        bp = O.chebyshev_params(lo, hi, s)
        t = np.clip((lam - (hi + lo) / 2) / ((hi - lo) / 2), -1, 1)
        closed = [np.cos(j * np.arccos(t)) * v for j in range(s + 1)]
    else:
        th = [1.9, 0.1, 1.0, 1.5, 0.5, 1.7, 0.3, 1.2]
        bp = O.newton_params(th, s)
        closed = [np.prod([lam - th[i] for i in range(j)], axis=0) * v if j else v for j in range(s + 1)]
    cols = O.basis_columns(A, v, s + 1, bp)
    for j in range(s + 1):
        np.testing.assert_allclose(cols[j], closed[j], rtol=0, atol=1e-12 * max(1.0, np.abs(closed[j]).max()))


def test_basis_change_matrix_structure():
    """B is block diagonal with two tridiagonal blocks and zero last columns (eq. AVVB)."""
    s = 4
    bp = O.BasisParams([1.0, 2.0, 3.0, 4.0], [10.0, 20.0, 30.0, 40.0], [0.5, 0.25, 0.125, 0.0625])
    B = O.basis_change_matrix(s, bp)
    # column 0 of the P block: A rho_0 = gamma_0 rho_1 + theta_0 rho_0
    assert B[0, 0] == 1.0 and B[1, 0] == 0.5
    # column 2: A rho_2 = gamma_2 rho_3 + theta_2 rho_2 + sigma_1 rho_1
    assert B[2, 2] == 3.0 and B[3, 2] == 0.125 and B[1, 2] == 20.0
    assert np.all(B[:, s] == 0) and np.all(B[:, 2 * s] == 0)
    assert np.all(B[: s + 1, s + 1:] == 0) and np.all(B[s + 1:, : s + 1] == 0)
    # R block (columns s+1 .. 2s): same coefficients, one column fewer
    assert B[s + 1, s + 1] == 1.0 and B[s + 2, s + 1] == 0.5 and B[s + 2, s + 3] == 20.0


# ---------------------------------------------------------------------------
# Gram matrix
# ---------------------------------------------------------------------------

def test_gram_against_exact_sums():
    """|G - Y^T Y (exact)| <= gamma_n |Y|^T |Y| entrywise, and G is symmetric."""
    rng = np.random.default_rng(8)
    n, w = 60, 9
    Y = rng.standard_normal((n, w)) * np.logspace(0, 3, w)
    G = O.gram(Y)
    YF = frac_array(Y)
    exact = (YF.T @ YF).astype(np.float64)
    gamma_n = n * EPS / (1 - n * EPS)
    bound = gamma_n * (np.abs(Y).T @ np.abs(Y))
    assert np.all(np.abs(G - exact) <= bound)
    assert np.array_equal(G, G.T)
    # the transposed product Y Y^T has the wrong shape entirely; a wrong operand order fails
    assert G.shape == (w, w)


# ---------------------------------------------------------------------------
# condition estimates and the choice of s~ (eq. condy)
# ---------------------------------------------------------------------------

def test_submatrix_index_matches_matlab_notation():
    # sbar = 3: i_s = 5 (1-based). i = 1: cols 1:2 and 5:5; i = 2: 1:3, 5:6; i = 3: 1:4, 5:7.
    assert O.submatrix_index(3, 1) == [0, 1, 4]
    assert O.submatrix_index(3, 2) == [0, 1, 2, 4, 5]
    assert O.submatrix_index(3, 3) == [0, 1, 2, 3, 4, 5, 6]
    assert O.submatrix_index(1, 1) == [0, 1, 2]


def test_kappa_matches_svd_of_column_subset():
    """sqrt(kappa(G_{k,i})) = kappa(Y_{k,i}) (Sec. 3.2), checked with SVD of the explicit columns."""
    c = W.scaled("poisson2d", 8, 1)
    A = O.Operator.from_csr(c["A"])
    s = 5
    bp = O.chebyshev_params(c["lam"][0], c["lam"][1], s)
    rng = np.random.default_rng(2)
    Y = O.matrix_powers(A, rng.standard_normal(A.n), rng.standard_normal(A.n), s, bp)
    G = O.gram(Y)
    prev = 0.0
    for i in range(1, s + 1):
        cols = list(range(i + 1)) + list(range(s + 1, s + 1 + i))   # P 0..i, R 0..i-1
        kap, unc = O.kappa_gram(G[np.ix_(cols, cols)], A.n)
        assert not unc
        ky = np.linalg.cond(Y[:, cols])
        assert abs(math.sqrt(kap) - ky) <= 1e-6 * ky
        assert math.sqrt(kap) >= prev * (1 - 1e-12)   # interlacing: non-decreasing in i
        prev = math.sqrt(kap)


def test_kappa_uncertified_is_infinite():
    G = np.diag([1.0, 1e-20, 2.0])
    kap, unc = O.kappa_gram(G)
    assert unc and kap == math.inf
    kap, unc = O.kappa_gram(np.diag([4.0, 1.0, 2.0]))
    assert not unc and kap == 4.0
    # the floor grows with sqrt(n): 3 * sqrt(1e6) * eps * 2 ~ 6.7e-13
    kap, unc = O.kappa_gram(np.diag([2.0, 1e-12, 1.0]), nrows=10 ** 6)
    assert not unc
    kap, unc = O.kappa_gram(np.diag([2.0, 5e-13, 1.0]), nrows=10 ** 6)
    assert unc


def test_first_blocks_are_rank_limited():
    """p, r in K_{m+1}(A, r_1): Y_{k,i} is rank deficient for i > m, so s~_k <= max(m, 1)."""
    c = W.poisson2d_32()
    A = O.Operator.from_csr(c["A"])
    ad = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=8, eps_target=1e-6)
    for blk in ad.blocks:
        assert blk["stilde"] <= max(blk["m"], 1)
    assert [blk["s_k"] for blk in ad.blocks[:5]] == [1, 1, 2, 4, 8]


def test_choose_s_prefix_rule():
    """Diagonal G: kappa(G_{k,i}) is max/min over the index set, known by hand."""
    sbar = 3
    # order: P0 P1 P2 P3 | R0 R1 R2
    d = np.array([1.0, 1.0, 4.0, 100.0, 1.0, 9.0, 1e4])
    G = np.diag(d)
    # i=1: {P0,P1,R0} -> kappa 1; i=2: {P0..P2,R0,R1} -> 9; i=3: all -> 1e4
    s, ev = O.choose_s(G, sbar, threshold=3.0)      # sqrt: 1, 3, 100
    assert s == 2 and [round(e[1], 12) for e in ev] == [1.0, 3.0, 100.0]
    s, ev = O.choose_s(G, sbar, threshold=2.9)
    assert s == 1 and len(ev) == 2
    s, ev = O.choose_s(G, sbar, threshold=0.5)      # none admissible -> 1
    assert s == 1 and len(ev) == 1
    s, ev = O.choose_s(G, sbar, threshold=1e9)
    assert s == 3


# ---------------------------------------------------------------------------
# Newton basis inputs: Ritz values and Leja order
# ---------------------------------------------------------------------------

def test_ritz_values_are_eigenvalues_after_d_steps():
    lam = np.array([0.3, 0.7, 1.1, 1.6, 1.9])
    A = O.Operator.from_dense(np.diag(lam))
    b = np.ones(5) / math.sqrt(5)
    cl = O.classical_cg(A, b, np.zeros(5), eps_target=0.0, max_iters=5)
    assert len(cl.alphas) == 5
    ritz = O.ritz_values(cl.alphas, cl.betas)
    np.testing.assert_allclose(np.sort(ritz), lam, rtol=0, atol=1e-8)
    # fewer steps: Ritz values interlace inside [lam_min, lam_max]
    cl3 = O.classical_cg(A, b, np.zeros(5), eps_target=0.0, max_iters=3)
    r3 = O.ritz_values(cl3.alphas, cl3.betas)
    assert np.all(r3 >= lam[0] - 1e-12) and np.all(r3 <= lam[-1] + 1e-12)


def test_leja_order_golden():
    path = os.path.join(HERE, "golden", "leja_examples.txt")
    n = 0
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        inp, out = line.split("|")
        got = O.leja_order([float(v) for v in inp.split()])
        assert got == [float(v) for v in out.split()], line
        n += 1
    assert n >= 5


# ---------------------------------------------------------------------------
# adaptive driver (Alg. 4)
# ---------------------------------------------------------------------------

def test_adaptive_with_s1_matches_classical():
    """s_k = 1 in every block is classical CG (Sec. 3.2); histories agree to rounding."""
    c = W.poisson2d_32()
    A = O.Operator.from_csr(c["A"])
    cl = O.classical_cg(A, c["b"], c["x1"], eps_target=1e-10)
    ad = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=1, eps_target=1e-10)
    assert ad.iters == cl.iters
    assert all(bl["s_k"] == 1 for bl in ad.blocks)
    np.testing.assert_allclose(ad.res_hist, cl.res_hist, rtol=1e-9, atol=1e-14)


def test_gap_bound_fb():
    """Residual-gap growth inside each block obeys eq. (fb) with c_{k,j} = 6 N_k j kappa(A)."""
    c = W.scaled("poisson2d", 10, 3)
    A = O.Operator.from_csr(c["A"])
    Ad = A.dense()
    b = c["b"]
    ev = np.linalg.eigvalsh(Ad)
    kA, nA = ev[-1] / ev[0], ev[-1]
    xstar = np.linalg.solve(Ad, b)
    res = O.adaptive_sstep_cg(A, b, c["x1"], s_max=6, eps_target=1e-13, trace=True)
    assert res.converged
    AF, bF = frac_array(Ad), frac_array(b)

    def gap(x, r):
        return np.linalg.norm((bF - AF @ frac_array(x) - frac_array(r)).astype(np.float64))

    checked = 0
    for blk in res.blocks:
        Y, B = blk["Y"], blk["B"]
        tau = np.linalg.norm(B, 2) / nA
        Nk = 7 + 2 * A.N_A + 14 * tau
        kY = np.linalg.cond(Y)
        x0, r0 = blk["x_start"], blk["r_start"]
        d0 = gap(x0, r0)
        rmax = np.linalg.norm(r0)
        for j, (xc, rc) in enumerate(blk["inner"], start=1):
            xj = Y @ xc + x0
            rj = Y @ rc
            rmax = max(rmax, np.linalg.norm(rj))
            bound = 6 * Nk * j * kA * EPS * kY * rmax + EPS * nA * np.linalg.norm(xstar)
            dj = (bF - AF @ frac_array(xj) - frac_array(rj)) - (bF - AF @ frac_array(x0) - frac_array(r0))
            assert np.linalg.norm(dj.astype(np.float64)) <= bound
            checked += 1
        assert d0 >= 0
    assert checked > 20


def test_attains_requested_accuracy():
    c = W.poisson2d_32()
    A = O.Operator.from_csr(c["A"])
    for eps in (1e-6, 1e-10):
        ad = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=8, eps_target=eps)
        assert ad.converged and ad.true_res <= 2 * eps


def test_paper_observations_sec5():
    """Qualitative claims of Sec. 5 on the 2D Poisson stand-in.

    (1) at a tight target, fixed s = 10 monomial s-step CG does not converge while
        adaptive s_max = 10 does;
    (2) adaptive needs fewer outer loops (global synchronisations) than classical iterations;
    (3) at eps* = 1e-6 adaptive uses s_max in every block once m >= s_max (before
        that the basis is rank limited, see test_first_blocks_are_rank_limited).
    """
    c = W.poisson2d_32()
    A = O.Operator.from_csr(c["A"])
    cl = O.classical_cg(A, c["b"], c["x1"], eps_target=1e-13, max_iters=3000)
    assert cl.converged
    fx = O.fixed_sstep_cg(A, c["b"], c["x1"], 10, O.monomial_params(10), eps_target=1e-13, max_iters=1500)
    assert not fx.converged or fx.true_res > 1e-13
    ad = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=10, eps_target=1e-13, max_iters=3000)
    assert ad.converged and ad.true_res <= 2e-13
    assert len(ad.blocks) < cl.iters
    loose = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=8, eps_target=1e-6)
    late = [bl["s_k"] for bl in loose.blocks[:-1] if bl["m"] >= 8]
    assert late and all(s == 8 for s in late)


@pytest.mark.parametrize("s_max", [8, 10])
@pytest.mark.parametrize("family", ["poisson2d_32", "poisson3d_12"])
def test_sk_monotone_while_residual_decreases(family, s_max):
    """Sec. 5 observation: where the residual 2-norm decreases monotonically, the
    chosen s_k increase monotonically (the threshold of (condy) grows as the
    residual shrinks). Checked on the Poisson stand-ins at a tight target: the
    block-start residuals must fall, and s_k must not decrease, up to the last
    block, which is cut short by convergence."""
    if family == "poisson2d_32":
        c = W.poisson2d_32()
        A, b, x1 = O.Operator.from_csr(c["A"]), c["b"], c["x1"]
    else:
        A = O.Operator.from_csr(W.poisson3d(12))
        rng = np.random.default_rng(5)
        b = rng.uniform(-1.0, 1.0, A.n)
        b /= np.linalg.norm(b)
        x1 = np.zeros(A.n)
    ad = O.adaptive_sstep_cg(A, b, x1, s_max=s_max, eps_target=1e-13, max_iters=3000)
    assert ad.converged
    rn = [bl["rnorm"] for bl in ad.blocks]
    assert all(rn[i + 1] <= rn[i] for i in range(len(rn) - 1))
    body = [bl["s_k"] for bl in ad.blocks if bl["stop"] != "converged"]
    assert len(body) >= 5
    assert all(body[i + 1] >= body[i] for i in range(len(body) - 1)), body
    assert body[-1] > body[0]


@pytest.mark.parametrize("n,hbw", [(800, 20), (1500, 40)])
def test_in_loop_check_cuts_blocks_short(n, hbw):
    """Eq. (check) inside the block (Alg. 4): where the coordinate residual grows
    within a block, the threshold eps*/(c eps ||r'||) falls below the basis'
    condition estimate gamma and the block stops before s~ steps. On banded
    SPD matrices (whose CG residual norms oscillate) at eps* = 1e-12 some blocks
    must stop that way. In each, gamma lies below every earlier step's threshold
    and at or above the last one's."""
    A = O.Operator.from_csr(W.banded_spd(n, hbw, np.random.default_rng(n)))
    b = W.rhs_uniform(A.n, np.random.default_rng(1))
    ad = O.adaptive_sstep_cg(A, b, np.zeros(A.n), s_max=10, eps_target=1e-12, max_iters=20000)
    assert ad.converged
    cut = [bl for bl in ad.blocks if bl["stop"] == "break" and bl["s_k"] < bl["stilde"]]
    assert cut
    for bl in cut:
        thresholds = [t for _, t in bl["checks"]]
        assert len(thresholds) == bl["s_k"]
        assert all(bl["gamma"] < t for t in thresholds[:-1])
        assert bl["gamma"] >= thresholds[-1]


def _laplacian_1d(n):
    """tridiag(-1/2, 1, -1/2): the 1D Dirichlet Laplacian, equilibrated (Sec. 5).
    Eigenvalues 1 - cos(k pi/(n+1)), k = 1..n (closed form)."""
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -0.5), (i, 1.0), (i + 1, -0.5)):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                vals.append(v)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, np.array(rows) + 1, 1)
    return O.Operator(n, np.cumsum(rowptr), np.array(cols), np.array(vals))


def test_c_formula_mode_closed_form():
    """c_{k,j} = 6 N_k j kappa(A) (eq. (fb)) on the 1D Laplacian, where every
    ingredient is known without the oracle: N_A = 3 nonzeros per row, ||B|| = 1
    for the monomial basis (a shift), kappa(A) = cot^2(pi/(2(n+1))) and
    ||A|| = 1 + cos(pi/(n+1)). Each block's eq. (condy) threshold must use
    c_{k,s_max}, and the run must still reach its target."""
    n, s_max, eps = 40, 6, 1e-10
    A = _laplacian_1d(n)
    th = math.pi / (n + 1)
    kA = 1.0 / math.tan(th / 2) ** 2
    nA = 1.0 + math.cos(th)
    assert A.N_A == 3
    b = W.rhs_uniform(n, np.random.default_rng(0))
    res = O.adaptive_sstep_cg(A, b, np.zeros(n), s_max=s_max, eps_target=eps, c_formula=(kA, nA))
    c_step = 6 * (7 + 2 * 3 + 14 * 1.0 / nA) * kA
    for blk in res.blocks:
        assert blk["c_condy"] == pytest.approx(c_step * s_max, rel=1e-13)
        assert blk["threshold"] == pytest.approx(eps / (c_step * s_max * EPS * blk["rnorm"]), rel=1e-13)
    assert res.converged and res.true_res <= 2 * eps


def test_c_formula_is_more_conservative():
    """The bound's c_{k,j} is far above 1, so eq. (condy) admits smaller bases
    than with c = 1 (Sec. 3.2: the bound overestimates the error); the method
    still converges, to the requested accuracy."""
    c = W.poisson2d_32()
    A = O.Operator.from_csr(c["A"])
    lo, hi = W.poisson_eig_bounds(2, 32)
    base = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=8, eps_target=1e-10)
    form = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=8, eps_target=1e-10, c_formula=(hi / lo, hi))
    assert form.converged and form.true_res <= 2e-10
    mean = lambda r: r.iters / len(r.blocks)
    assert mean(form) < mean(base)
    assert len(form.blocks) > len(base.blocks)


def test_c_formula_uses_the_bases_B_norm():
    """tau_k = ||B_{k,sbar}|| / ||A||: for a Chebyshev basis ||B|| is not 1, and
    the recorded c_{k,s_max} follows the 2-norm of the block's B."""
    c = W.poisson2d_32()
    A = O.Operator.from_csr(c["A"])
    lo, hi = W.poisson_eig_bounds(2, 32)
    res = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=8, eps_target=1e-10, basis="chebyshev", lam=(lo, hi),
                              c_formula=(hi / lo, hi))
    bp = O.chebyshev_params(lo, hi, 8)
    for blk in res.blocks:
        nb = np.linalg.svd(O.basis_change_matrix(blk["sbar"], bp), compute_uv=False)[0]
        assert nb != pytest.approx(1.0, rel=1e-3)
        assert blk["c_condy"] == pytest.approx(6 * (7 + 2 * A.N_A + 14 * nb / hi) * (hi / lo) * 8, rel=1e-12)
    assert res.converged


# ---------------------------------------------------------------------------
# the Hankel-moment Gram of the monomial basis (a variant of the Gram step)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s", [1, 2, 4])
def test_gram_moments_equal_gram_in_exact_arithmetic(s):
    """With A symmetric the monomial basis' Gram blocks are Hankel matrices of
    moments: in exact (rational) arithmetic the moment form equals Y^T Y
    entry for entry, for every block (P^T P, P^T R, R^T R)."""
    D = small_int_spd(7, 5)
    A = O.Operator.from_dense(frac_array(D))
    p = frac_array(np.array([1, -2, 0, 3, 1, -1, 2]))
    r = frac_array(np.array([2, 1, -1, 0, 1, 3, -2]))
    Y = O.matrix_powers(A, p, r, s, O.monomial_params(s, one=Fraction(1), zero=Fraction(0)))
    Gm = O.gram_moments(Y, s)
    Gp = O.gram(Y)
    assert all(Gm[i, j] == Gp[i, j] for i in range(2 * s + 1) for j in range(2 * s + 1))
    if s == 1:  # every entry is its own moment: the forms agree for any Y
        return
    # from s = 2 on, a basis that is not a Krylov sequence of one symmetric matrix breaks the identity
    Y2 = Y.copy()
    Y2[0, 1] += Fraction(1)
    G2 = O.gram_moments(Y2, s)
    assert any(G2[i, j] != O.gram(Y2)[i, j] for i in range(2 * s + 1) for j in range(2 * s + 1))


def test_gram_moments_solve_reaches_target():
    """Adaptive s-step CG with the moment Gram converges to the requested
    accuracy on the 2D Poisson problem, with an s_k sequence close to the
    plain Gram's."""
    c = W.poisson2d_32()
    A = O.Operator.from_csr(c["A"])
    plain = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=8, eps_target=1e-10)
    mom = O.adaptive_sstep_cg(A, c["b"], c["x1"], s_max=8, eps_target=1e-10, gram_mode="moments")
    assert mom.converged and mom.true_res <= 2e-10
    assert abs(mom.iters - plain.iters) <= plain.iters // 10
