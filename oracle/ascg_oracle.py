"""Plain CPU oracle for the adaptive s-step conjugate gradient method.

TEST INFRASTRUCTURE ONLY. The oracle is what the CUDA path is checked
against; the solver library never imports, links or runs it. Only the tests,
`__graft_entry__.smoke()` and the CPU-baseline arm of `bench.py` use it.

Reference: E. Carson, "The Adaptive s-step Conjugate Gradient Method"
(arXiv:1701.03989). Section, equation and algorithm names below are the
paper's:
  Alg. 1  classical CG (Sec. 2)
  Alg. 2  s-step CG (Sec. 2.1)
  Alg. 3  variable s-step CG (Sec. 3)
  Alg. 4  adaptive s-step CG (Sec. 3.2)
  eq. (polybasiscg)   three-term polynomial recurrence for the basis
  eq. (cg-krylovbasis) basis matrices P_{k,s}, R_{k,s}
  eq. (AVVB)          A * Yunder = Y * B
  eq. (coords)        x, r, p as Y times coordinate vectors
  eq. (condy)         choice of s~_k from the Gram submatrices
  eq. (check)         in-loop break test

Everything is a literal, sequential restatement in numpy. Floating point is
IEEE double, and unit roundoff is eps = 2^-53 (Sec. 5). The functions that
make up Alg. 2 and Alg. 3 (basis, Gram, B, coordinate steps, recovery) also
run on numpy object arrays of `fractions.Fraction`. The tests use that to pin
the oracle against exact arithmetic.

How each part is pinned (tests/test_oracle_pins.py):
  classical CG        finite termination, exact (Fraction) solution
  s-step, variable s  identical to classical CG in exact arithmetic
  basis recurrence    eq. (E) rounding bound; closed forms on diagonal A
  Gram                exactly rounded sums (math.fsum) within the dot-product bound
  kappa / s~ choice   SVD of the explicit column subset; interlacing
  Ritz values, Leja   exact eigenvalues after d steps; hand-worked fixtures
  adaptive driver     s_k = 1 equals classical CG; gap bound eq. (fb);
                      accuracy attained at eps* >= eps_CG
The paper's Table 1 matrices are missing, so its printed synchronisation
counts and s_k sequences cannot be reproduced. Parity for those stays
unpinned; they are quoted as context only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EPS = 2.0 ** -53  # unit roundoff of IEEE double (Sec. 5)


# ---------------------------------------------------------------------------
# Sparse operator (the matrix A of Alg. 1-4)
# ---------------------------------------------------------------------------

class Operator:
    """A CSR matrix with a cached row index per nonzero."""

    def __init__(self, n, rowptr, colind, val):
        self.n = int(n)
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.colind = np.asarray(colind, dtype=np.int64)
        self.val = np.asarray(val) if np.asarray(val).dtype == object else np.asarray(val, dtype=np.float64)
        self.rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        self.N_A = int(np.max(np.diff(self.rowptr))) if self.n else 0  # max nonzeros per row (Sec. 3.1)

    @classmethod
    def from_csr(cls, A):
        return cls(A.n, A.rowptr, A.colind, A.val)

    @classmethod
    def from_dense(cls, D):
        D = np.asarray(D)
        n = D.shape[0]
        rowptr = [0]
        cols, vals = [], []
        for i in range(n):
            for j in range(n):
                if D[i, j] != 0:
                    cols.append(j)
                    vals.append(D[i, j])
            rowptr.append(len(cols))
        val = np.empty(len(vals), dtype=D.dtype)
        val[:] = vals
        return cls(n, rowptr, cols, val)

    def dense(self):
        d = np.zeros((self.n, self.n), dtype=self.val.dtype)
        d[self.rows, self.colind] = self.val
        return d


def spmv(A: Operator, x):
    """y = A x. Each row is summed in stored column order, starting from 0."""
    prods = A.val * x[A.colind]
    y = np.zeros(A.n, dtype=prods.dtype)
    np.add.at(y, A.rows, prods)
    return y


def norm2(v) -> float:
    return math.sqrt(float(v @ v))


# ---------------------------------------------------------------------------
# Basis polynomials: eq. (polybasiscg). Each basis is three lists
# theta, sigma, gamma; rho_j(z) = ((z - theta_{j-1}) rho_{j-1}(z)
#                                  - sigma_{j-2} rho_{j-2}(z)) / gamma_{j-1}.
# ---------------------------------------------------------------------------

@dataclass
class BasisParams:
    theta: list
    sigma: list
    gamma: list
    kind: str = "monomial"


def monomial_params(s: int, one=1.0, zero=0.0) -> BasisParams:
    """Monomial basis [v, Av, A^2 v, ...] (Sec. 2): theta = sigma = 0, gamma = 1."""
    return BasisParams([zero] * s, [zero] * s, [one] * s, "monomial")


def chebyshev_params(lam_min, lam_max, s: int) -> BasisParams:
    """Chebyshev basis on [lam_min, lam_max]. The paper only names this basis (Sec. 2).

    Reading: rho_j(z) = T_j((z - c) / h), c = (lam_max + lam_min)/2,
    h = (lam_max - lam_min)/2. From T_1(t) = t and T_{j+1} = 2 t T_j - T_{j-1}:
    theta_j = c for all j, gamma_0 = h, gamma_j = h/2 (j >= 1), sigma_j = h/2.
    """
    c = (lam_max + lam_min) / 2
    h = (lam_max - lam_min) / 2
    return BasisParams([c] * s, [h / 2] * s, [h] + [h / 2] * (s - 1), "chebyshev")


def newton_params(shifts, s: int) -> BasisParams:
    """Newton basis rho_{j+1}(z) = (z - theta_j) rho_j(z). The paper only names it (Sec. 2).

    Reading: theta_j = the first s Leja-ordered Ritz values, sigma = 0, gamma = 1.
    """
    shifts = list(shifts)
    if len(shifts) < s:
        raise ValueError("need at least s shifts")
    return BasisParams(shifts[:s], [0.0] * s, [1.0] * s, "newton")


def ritz_values(alphas, betas):
    """Eigenvalues of the Lanczos tridiagonal built from k CG steps.

    Standard CG/Lanczos relation (background to Sec. 2): T_jj = 1/alpha_j +
    beta_{j-1}/alpha_{j-1} (no second term for j = 1), T_{j,j+1} =
    sqrt(beta_j)/alpha_j. Eigenvalues by LAPACK (numpy.linalg.eigvalsh).
    """
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(betas[j]) / alphas[j]
    return np.linalg.eigvalsh(T)


def leja_order(values):
    """Leja ordering of a set of real numbers.

    The first value has the largest magnitude. Each next value maximises the
    product of its distances to the values already chosen. Ties go to the
    larger value, and equal values to the earlier index.
    """
    vals = [float(v) for v in values]
    remaining = list(range(len(vals)))
    chosen = []
    while remaining:
        best, best_key = None, None
        for i in remaining:
            if not chosen:
                score = abs(vals[i])
            else:
                score = 1.0
                for c in chosen:
                    score *= abs(vals[i] - vals[c])
            key = (score, vals[i])
            if best_key is None or key > best_key:
                best, best_key = i, key
        chosen.append(best)
        remaining.remove(best)
    return [vals[i] for i in chosen]


# ---------------------------------------------------------------------------
# One block of s-step CG: steps a4 .. a9
# ---------------------------------------------------------------------------

def basis_columns(A: Operator, v, ncols: int, bp: BasisParams):
    """[rho_0(A) v, ..., rho_{ncols-1}(A) v] by eq. (polybasiscg)."""
    cols = [v]
    for j in range(1, ncols):
        t = spmv(A, cols[j - 1]) - bp.theta[j - 1] * cols[j - 1]
        if j >= 2:
            t = t - bp.sigma[j - 2] * cols[j - 2]
        cols.append(t / bp.gamma[j - 1])
    return cols


def matrix_powers(A: Operator, p, r, s: int, bp: BasisParams):
    """Y_{k,s} = [P_{k,s}, R_{k,s}], eq. (cg-krylovbasis): s+1 columns from p, s from r."""
    P = basis_columns(A, p, s + 1, bp)
    R = basis_columns(A, r, s, bp)
    return np.column_stack(P + R)


def gram(Y):
    """G_{k,s} = Y^T Y (Sec. 2.1; Alg. 2, 4)."""
    return Y.T @ Y


def gram_moments(Y, s: int):
    """G_{k,s} of the monomial basis from 6s dot products (a variant of the Gram
    step; the paper forms Y^T Y).

    With A symmetric and rho_j(z) = z^j, P_i^T P_j = p^T A^(i+j) p,
    P_i^T R_j = p^T A^(i+j) r and R_i^T R_j = r^T A^(i+j) r depend on i + j
    only: each block of G is a Hankel matrix of moments. Reading (one pair of
    columns per moment, the most balanced one):
      mu_pp[k] = <P_floor(k/2), P_ceil(k/2)>,  k = 0 .. 2s
      mu_pr[k] = <P_ceil(k/2), R_floor(k/2)>,  k = 0 .. 2s-1
      mu_rr[k] = <R_floor(k/2), R_ceil(k/2)>,  k = 0 .. 2s-2
    In exact arithmetic this is Y^T Y. In floating point it differs from it by
    the rounding of the basis recurrence, which the other products of the
    same moment would see differently. Y: P columns then R columns (s+1, s).
    """
    P = Y[:, : s + 1]
    R = Y[:, s + 1:]
    mpp = [P[:, k // 2] @ P[:, (k + 1) // 2] for k in range(2 * s + 1)]
    mpr = [P[:, (k + 1) // 2] @ R[:, k // 2] for k in range(2 * s)]
    mrr = [R[:, k // 2] @ R[:, (k + 1) // 2] for k in range(2 * s - 1)]
    w = 2 * s + 1
    G = np.zeros((w, w), dtype=np.asarray(Y).dtype)
    for i in range(s + 1):
        for j in range(s + 1):
            G[i, j] = mpp[i + j]
        for j in range(s):
            G[i, s + 1 + j] = mpr[i + j]
            G[s + 1 + j, i] = mpr[i + j]
    for i in range(s):
        for j in range(s):
            G[s + 1 + i, s + 1 + j] = mrr[i + j]
    return G


def gram_of(Y, s: int, gram_mode: str):
    """G by gram_mode: "plain" (Y^T Y, the paper's step) or "moments" (gram_moments;
    monomial basis only)."""
    if gram_mode == "plain":
        return gram(Y)
    if gram_mode == "moments":
        return gram_moments(Y, s)
    raise ValueError(gram_mode)


def basis_change_matrix(s: int, bp: BasisParams, dtype=np.float64):
    """B_{k,s} with A * Yunder_{k,s} = Y_{k,s} * B_{k,s}, eq. (AVVB).

    Yunder is Y with zero columns s+1 and 2s+1 (1-based), so the last column
    of each of the two blocks is zero. In column c = start + j of a block,
    A rho_j = gamma_j rho_{j+1} + theta_j rho_j + sigma_{j-1} rho_{j-1}, so
    B[c+1, c] = gamma_j, B[c, c] = theta_j, B[c-1, c] = sigma_{j-1}.
    B is therefore block diagonal with two tridiagonal blocks.
    """
    w = 2 * s + 1
    B = np.zeros((w, w), dtype=dtype)
    for start, length in ((0, s + 1), (s + 1, s)):
        for j in range(length - 1):
            c = start + j
            B[c, c] = bp.theta[j]
            B[c + 1, c] = bp.gamma[j]
            if j >= 1:
                B[c - 1, c] = bp.sigma[j - 1]
    return B


def submatrix_index(sbar: int, i: int):
    """0-based columns of Y_{k,i} inside Y_{k,sbar} (Sec. 3.2).

    MATLAB notation in the paper: columns 1:i+1 and i_s:i_s+i-1, i_s = sbar+2.
    """
    i_s = sbar + 2
    return list(range(0, i + 1)) + list(range(i_s - 1, i_s - 1 + i))


def kappa_gram(Gsub, nrows: int = 1):
    """kappa(G_sub) = lam_max / lam_min, or +inf when lam_min is at rounding level.

    Eigenvalues by LAPACK (numpy.linalg.eigvalsh). Reading (the paper is
    silent): the computed Gram matrix carries rounding errors of typical size
    sqrt(n) * eps * ||Y||^2 (n = nrows, the length of the basis vectors). If
    lam_min <= w * sqrt(n) * eps * lam_max (w = order of G_sub), the Gram
    matrix cannot tell the basis from a rank-deficient one. kappa is then
    +inf, so the basis fails eq. (condy). One consequence: p, r lie in
    K_{m+1}(A, r_1), so Y_{k,i} is rank deficient whenever i > m. The first
    blocks therefore take s = 1, 1, 2, 4, ... Capping kappa at a finite value
    instead lets numerically singular bases through once the threshold grows,
    and the solve can then diverge. Returns (kappa, uncertified).
    """
    ev = np.linalg.eigvalsh(np.asarray(Gsub, dtype=np.float64))
    lmin, lmax = float(ev[0]), float(ev[-1])
    w = Gsub.shape[0]
    if not (lmax > 0.0) or not math.isfinite(lmax):
        return math.inf, True
    if lmin <= w * math.sqrt(nrows) * EPS * lmax:
        return math.inf, True
    return lmax / lmin, False


def choose_s(G, sbar: int, threshold: float, nrows: int = 1):
    """s~_k from eq. (condy): the largest i in 1..sbar with sqrt(kappa(G_{k,i})) <= threshold.

    kappa(Y_{k,i}) = sqrt(kappa(G_{k,i})) (Sec. 3.2). Reading: scan i = 1, 2, ... and stop
    at the first failure. Exact kappas are non-decreasing in i by interlacing,
    so this is the largest admissible prefix. If none is admissible, s~ = 1
    (Sec. 3.2: default to a classical step). Returns (s~, list of
    (i, sqrt_kappa, clamped)).
    """
    evals = []
    stilde = 0
    for i in range(1, sbar + 1):
        idx = submatrix_index(sbar, i)
        kap, clamped = kappa_gram(G[np.ix_(idx, idx)], nrows)
        sk = math.sqrt(kap)
        evals.append((i, sk, clamped))  # clamped = uncertified
        if sk <= threshold:
            stilde = i
        else:
            break
    return max(stilde, 1), evals


@dataclass
class InnerResult:
    xc: object
    rc: object
    pc: object
    steps: int
    alphas: list
    betas: list
    rGr: list            # r'^T G r' after each step
    stop: str            # "done", "converged", "break", "breakdown", "maxiter"
    trace: list = field(default_factory=list)  # (x', r') after each step, when asked


def coordinate_steps(G, B, s: int, nsteps: int, stop_test=None, trace=False, float_checks=True):
    """Inner loop of Alg. 2/3/4 on coordinate vectors of length 2s+1 (Sec. 2.1).

    p' = e_1, r' = e_{s+2}, x' = 0; for j = 1..nsteps:
      alpha = (r'^T G r') / (p'^T G B p');  q' = alpha p';  x' += q';
      r'_new = r' - B q';  beta = (r'_new^T G r'_new) / (r'^T G r');
      p' = r'_new + beta p'.
    stop_test(j, rGr_new) may return "converged" or "break" to end the loop
    after step j. Reading for breakdown (the paper is silent): if the alpha
    denominator is not positive and finite, the loop stops before step j.
    """
    w = 2 * s + 1
    pc = np.zeros(w, dtype=G.dtype)
    rc = np.zeros(w, dtype=G.dtype)
    xc = np.zeros(w, dtype=G.dtype)
    pc[0] = 1
    rc[s + 1] = 1
    rGr = rc @ (G @ rc)
    alphas, betas, hist, tr = [], [], [], []
    stop = "done"
    steps = 0
    for j in range(1, nsteps + 1):
        pGBp = pc @ (G @ (B @ pc))
        if float_checks and not (math.isfinite(float(pGBp)) and float(pGBp) > 0.0
                                 and math.isfinite(float(rGr)) and float(rGr) > 0.0):
            stop = "breakdown"
            break
        alpha = rGr / pGBp
        q = alpha * pc
        xc = xc + q
        rn = rc - B @ q
        rGr_new = rn @ (G @ rn)
        beta = rGr_new / rGr
        pc = rn + beta * pc
        rc = rn
        rGr = rGr_new
        steps = j
        alphas.append(alpha)
        betas.append(beta)
        hist.append(rGr_new)
        if trace:
            tr.append((xc.copy(), rc.copy()))
        if stop_test is not None:
            verdict = stop_test(j, rGr_new)
            if verdict:
                stop = verdict
                break
    return InnerResult(xc, rc, pc, steps, alphas, betas, hist, stop, tr)


def recover(Y, x, xc, rc, pc):
    """Recover x, r, p from coordinates, eq. (coords): x += Y x', r = Y r', p = Y p'."""
    return x + Y @ xc, Y @ rc, Y @ pc


def formula_c_step(A: Operator, B, kappa_A: float, norm_A: float) -> float:
    """6 N_k kappa(A), the factor of c_{k,j} = 6 N_k j kappa(A) that the bound
    eq. (fb) gives, with N_k = 7 + 2 N_A + 14 tau_k and tau_k = ||B|| / ||A||
    (2-norms; notation set before eq. (fb)). kappa(A) and ||A|| are the
    user's estimates. Reading: B is the block's B_{k,sbar}, since s_k is not
    known when s~_k is chosen; B_{k,s_k} is a submatrix of it, so tau_k can
    only be overestimated. For the monomial basis ||B|| = 1 either way."""
    tau = float(np.linalg.norm(B, 2)) / norm_A
    Nk = 7 + 2 * A.N_A + 14 * tau
    return 6.0 * Nk * kappa_A


def adaptive_block(G, sbar: int, bp: BasisParams, eps_star: float, c: float, nrows: int,
                   check_in_loop: bool = True, max_steps: int | None = None, trace: bool = False,
                   c_step: float | None = None, s_max: int | None = None):
    """One block of Alg. 4 (Sec. 3.2) after G is formed: the choice of s~_k, then the inner loop.

    ||r_{m+1}|| = sqrt(G[i_s, i_s]) (column i_s is r since rho_0 = 1);
    threshold = eps* / (c_{k,s_max} eps ||r_{m+1}||); s~ by eq. (condy); gamma =
    sqrt(kappa(G_{k,s~})); G and B restricted to Y_{k,s~}; inner steps with the
    eq. (check) break test, which after step j uses c_{k,j}. With c_step None,
    c_{k,j} = c for every j; else c_{k,j} = c_step * j. Returns (block record,
    InnerResult, column indices of Y_{k,s~} inside Y_{k,sbar}).
    """
    c_condy = c if c_step is None else c_step * s_max

    def c_check(j):
        return c if c_step is None else c_step * j

    i_s = sbar + 1
    rnorm = math.sqrt(max(float(G[i_s, i_s]), 0.0))
    threshold = eps_star / (c_condy * EPS * rnorm) if rnorm > 0 else math.inf
    stilde, kappas = choose_s(G, sbar, threshold, nrows)
    idx = submatrix_index(sbar, stilde)
    kap, gclamped = kappa_gram(G[np.ix_(idx, idx)], nrows)
    gamma_est = math.sqrt(kap)
    Gt = G[np.ix_(idx, idx)]
    Bt = basis_change_matrix(stilde, bp)
    nsteps = stilde if max_steps is None else min(stilde, max_steps)
    checks = []

    def stop_test(j, rGr_new):
        rn = math.sqrt(max(float(rGr_new), 0.0))
        if rn <= eps_star:
            return "converged"
        if check_in_loop:
            tj = eps_star / (c_check(j) * EPS * rn) if rn > 0 else math.inf
            checks.append((j, tj))
            if gamma_est >= tj:
                return "break"
        return None

    inner = coordinate_steps(Gt, Bt, stilde, nsteps, stop_test, trace=trace)
    blk = dict(sbar=sbar, stilde=stilde, s_k=inner.steps, threshold=threshold, rnorm=rnorm, kappas=kappas,
               gamma=gamma_est, gamma_clamped=gclamped, checks=checks, stop=inner.stop, c_condy=c_condy)
    if trace:
        blk.update(G=Gt, B=Bt, inner=inner.trace)
    return blk, inner, idx


# ---------------------------------------------------------------------------
# Drivers
# ---------------------------------------------------------------------------

@dataclass
class SolveResult:
    x: np.ndarray
    r: np.ndarray
    p: np.ndarray
    res_hist: list           # ||r_i|| / ||b||, i = 1 (initial) .. m+1
    alphas: list
    betas: list
    iters: int
    converged: bool
    status: str
    blocks: list = field(default_factory=list)
    true_res: float = float("nan")


def residual(A: Operator, b, x):
    """r = b - A x."""
    return b - spmv(A, x)


def classical_cg(A: Operator, b, x1, eps_target: float = 1e-10, max_iters: int = 10000,
                 exact: bool = False):
    """Classical CG, Alg. 1.

    alpha_i = r^T r / p^T A p; q = alpha p; x += q; r -= A q; beta = r_new^T r_new / r^T r;
    p = r_new + beta p. Reading: A q_i is formed as alpha_i (A p_i), which
    reuses the product already computed for alpha. Stop after iteration i when
    ||r_{i+1}|| <= eps* = eps_target * ||b||. In exact mode (Fraction
    arithmetic) no norms are taken, and exactly max_iters iterations run
    unless r becomes exactly zero.
    """
    x = x1.copy()
    r = residual(A, b, x)
    p = r.copy()
    rr = r @ r
    if exact:
        bnorm = None
        eps_star = None
        hist = []
    else:
        bnorm = norm2(b)
        eps_star = eps_target * bnorm
        hist = [math.sqrt(float(rr)) / bnorm]
    alphas, betas = [], []
    converged = (not exact) and math.sqrt(float(rr)) <= eps_star
    i = 0
    while not converged and i < max_iters:
        if exact and rr == 0:
            break
        Ap = spmv(A, p)
        alpha = rr / (p @ Ap)
        q = alpha * p
        x = x + q
        r = r - alpha * Ap
        rr_new = r @ r
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        i += 1
        alphas.append(alpha)
        betas.append(beta)
        if not exact:
            hist.append(math.sqrt(float(rr)) / bnorm)
            converged = math.sqrt(float(rr)) <= eps_star
    res = SolveResult(x, r, p, hist, alphas, betas, i, bool(converged),
                      "converged" if converged else ("exact" if exact else "maxiter"))
    if not exact:
        res.true_res = norm2(residual(A, b, x)) / bnorm
    return res


def variable_sstep_cg(A: Operator, b, x1, s_seq, bp: BasisParams, eps_target: float = 1e-10,
                      max_iters: int = 10000, exact: bool = False, gram_mode: str = "plain"):
    """Variable s-step CG, Alg. 3 (Alg. 2 when every s_k is the same).

    Block k: Y_{k,s_k} (eq. cg-krylovbasis), G = Y^T Y, B (eq. AVVB), s_k
    coordinate steps, recovery (eq. coords), m += s_k. s_seq gives s_0, s_1, ...;
    its last value repeats. Reading: stop after an inner step whose
    coordinate residual norm sqrt(r'^T G r') is at or below eps*. In exact
    mode no norms are taken, and blocks run until max_iters iterations are done.
    """
    x = x1.copy()
    r = residual(A, b, x)
    p = r.copy()
    m = 0
    k = 0
    bnorm = None if exact else norm2(b)
    eps_star = None if exact else eps_target * bnorm
    hist = [] if exact else [norm2(r) / bnorm]
    alphas, betas, blocks = [], [], []
    converged = (not exact) and norm2(r) <= eps_star
    while not converged and m < max_iters:
        s = int(s_seq[min(k, len(s_seq) - 1)])
        Y = matrix_powers(A, p, r, s, bp)
        G = gram_of(Y, s, gram_mode)
        B = basis_change_matrix(s, bp, dtype=G.dtype)
        nsteps = min(s, max_iters - m)

        def stop_test(j, rGr_new):
            if exact:
                return None
            return "converged" if math.sqrt(max(float(rGr_new), 0.0)) <= eps_star else None

        inner = coordinate_steps(G, B, s, nsteps, stop_test, float_checks=not exact)
        if inner.steps == 0:
            return SolveResult(x, r, p, hist, alphas, betas, m, False, "breakdown", blocks)
        x, r, p = recover(Y, x, inner.xc, inner.rc, inner.pc)
        alphas += inner.alphas
        betas += inner.betas
        if not exact:
            hist += [math.sqrt(max(float(v), 0.0)) / bnorm for v in inner.rGr]
        blocks.append(dict(sbar=s, stilde=s, s_k=inner.steps, stop=inner.stop))
        m += inner.steps
        k += 1
        converged = inner.stop == "converged"
    res = SolveResult(x, r, p, hist, alphas, betas, m, bool(converged),
                      "converged" if converged else ("exact" if exact else "maxiter"), blocks)
    if not exact:
        res.true_res = norm2(residual(A, b, x)) / bnorm
    return res


def fixed_sstep_cg(A: Operator, b, x1, s: int, bp: BasisParams, **kw):
    """s-step CG with a fixed s, Alg. 2."""
    return variable_sstep_cg(A, b, x1, [s], bp, **kw)


def adaptive_sstep_cg(A: Operator, b, x1, *, s_max: int, s0: int | None = None, f: int | None = None,
                      eps_target: float = 1e-10, c: float = 1.0, basis: str = "monomial",
                      lam=None, newton_warmup: int | None = None, check_in_loop: bool = True,
                      max_iters: int = 10000, trace: bool = False, c_formula=None, gram_mode: str = "plain"):
    """Adaptive s-step CG, Alg. 4.

    c_{k,j}: the constant c, or with c_formula = (kappa(A), ||A||) the bound's
    own c_{k,j} = 6 N_k j kappa(A) (see formula_c_step). gram_mode "moments"
    forms G from moments (gram_moments; monomial basis only).

    Per block k:
      sbar_k = s0 for k = 0, else min(s_{k-1} + f, s_max);
      Y = [P, R] for sbar_k (eq. cg-krylovbasis), G = Y^T Y;
      s~_k by eq. (condy) with threshold eps* / (c eps ||r_{m+1}||), where
      ||r_{m+1}|| = sqrt(G[i_s, i_s]) (column i_s is r, since rho_0 = 1);
      gamma = sqrt(kappa(G_{k,s~})) estimates kappa(Y_{k,s~});
      Y, G restricted to the columns of Y_{k,s~}; B for s~;
      inner steps j = 1..s~, with s_k = j; after step j, break if
      gamma >= eps* / (c eps sqrt(r'^T G r')) (eq. check);
      recovery (eq. coords); m += s_k.
    Readings (the paper is silent): eps* = eps_target * ||b||; stop after an
    inner step whose sqrt(max(r'^T G r', 0)) <= eps*; the convergence test
    comes before the break test.

    basis: "monomial", "chebyshev" (lam = (lam_min, lam_max)) or "newton"
    (newton_warmup classical iterations, default 2 s_max; Ritz values of their
    Lanczos tridiagonal, Leja-ordered). The warm-up iterations count toward
    the iteration total and the residual history.
    """
    if gram_mode == "moments" and basis != "monomial":
        raise ValueError("the moment Gram needs the monomial basis")
    s0 = s_max if s0 is None else s0
    f = s_max if f is None else f
    x = x1.copy()
    bnorm = norm2(b)
    eps_star = eps_target * bnorm
    alphas, betas, blocks = [], [], []
    m = 0
    if basis == "newton":
        nw = 2 * s_max if newton_warmup is None else newton_warmup
        warm = classical_cg(A, b, x, eps_target=eps_target, max_iters=min(nw, max_iters))
        x, r, p = warm.x, warm.r, warm.p
        hist = list(warm.res_hist)
        alphas += warm.alphas
        betas += warm.betas
        m = warm.iters
        if warm.converged or m >= max_iters:
            res = SolveResult(x, r, p, hist, alphas, betas, m, warm.converged,
                              "converged" if warm.converged else "maxiter", blocks)
            res.true_res = norm2(residual(A, b, x)) / bnorm
            return res
        shifts = leja_order(ritz_values(warm.alphas, warm.betas))
        bp = newton_params(shifts, s_max)
    else:
        r = residual(A, b, x)
        p = r.copy()
        hist = [norm2(r) / bnorm]
        if basis == "monomial":
            bp = monomial_params(s_max)
        elif basis == "chebyshev":
            bp = chebyshev_params(lam[0], lam[1], s_max)
        else:
            raise ValueError(basis)
    converged = norm2(r) <= eps_star
    k = 0
    s_prev = None
    while not converged and m < max_iters:
        sbar = s0 if k == 0 else min(s_prev + f, s_max)
        Y = matrix_powers(A, p, r, sbar, bp)
        G = gram_of(Y, sbar, gram_mode)
        c_step = None
        if c_formula is not None:
            c_step = formula_c_step(A, basis_change_matrix(sbar, bp), c_formula[0], c_formula[1])
        blk, inner, idx = adaptive_block(G, sbar, bp, eps_star, c, A.n, check_in_loop, max_iters - m,
                                         trace=trace, c_step=c_step, s_max=s_max)
        if inner.steps == 0:
            return SolveResult(x, r, p, hist, alphas, betas, m, False, "breakdown", blocks)
        Yt = Y[:, idx]
        blk.update(k=k, m=m)
        if trace:
            blk.update(Y=Yt, x_start=x.copy(), r_start=r.copy())
        x, r, p = recover(Yt, x, inner.xc, inner.rc, inner.pc)
        alphas += inner.alphas
        betas += inner.betas
        hist += [math.sqrt(max(float(v), 0.0)) / bnorm for v in inner.rGr]
        blocks.append(blk)
        m += inner.steps
        s_prev = inner.steps
        k += 1
        converged = inner.stop == "converged"
    res = SolveResult(x, r, p, hist, alphas, betas, m, bool(converged),
                      "converged" if converged else "maxiter", blocks)
    res.true_res = norm2(residual(A, b, x)) / bnorm
    return res
