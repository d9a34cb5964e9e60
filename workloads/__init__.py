"""Seeded synthetic inputs for the adaptive s-step CG solver and its CPU oracle.

This module builds matrices and right-hand sides only. It holds none of the
method's arithmetic, so that the CUDA path and the oracle can both use it
without sharing any solver code.

The paper's protocol (Sec. 5) is kept for every family:
  * double precision throughout;
  * the matrix is equilibrated, A <- D^{-1/2} A D^{-1/2}, where D holds the
    largest entry of each row (largest in magnitude; for every family here it
    is the positive diagonal);
  * the right-hand side is normalised to unit 2-norm. The paper uses
    b_i = 1/sqrt(n); the configurations here draw b_i ~ U[-1, 1] from the
    seed and then normalise, so ||b|| = 1 in both cases;
  * x_1 = 0.

The SuiteSparse matrices of the paper's Table 1 are not available here, so
these families stand in for them:
  * 2D Poisson, 5-point, Dirichlet, lexicographic order;
  * 3D Poisson, 7-point, Dirichlet, lexicographic order;
  * 2D finite-volume diffusion with log-normal cell coefficients (5-point);
  * random banded SPD.

Random numbers come from numpy's PCG64 (`numpy.random.default_rng(seed)`),
seed = 1000 + configuration number.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSRMatrix:
    """Square sparse matrix in compressed sparse row form.

    rowptr: int64[n+1], colind: int32[nnz] (sorted within each row),
    val: float64[nnz].
    """

    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=self.val.dtype)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.colind] = self.val
        return d


def _stencil_csr(shape, offsets, weights):
    """CSR of a constant-coefficient stencil on a grid with Dirichlet boundary.

    shape: grid extents (slowest first); offsets: list of integer tuples;
    weights: matching list of values. Rows are grid points in lexicographic
    order; neighbours outside the grid are dropped.
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    coords = np.indices(shape).reshape(len(shape), n)
    strides = [int(np.prod(shape[d + 1:])) for d in range(len(shape))]
    # column index of each neighbour; keep offsets sorted by column shift so
    # every row's columns come out in increasing order
    order = sorted(range(len(offsets)), key=lambda k: sum(o * s for o, s in zip(offsets[k], strides)))
    cols, vals, masks = [], [], []
    idx = np.arange(n, dtype=np.int64)
    for k in order:
        off = offsets[k]
        ok = np.ones(n, dtype=bool)
        for d, o in enumerate(off):
            if o:
                c = coords[d] + o
                ok &= (c >= 0) & (c < shape[d])
        shift = sum(o * s for o, s in zip(off, strides))
        cols.append(idx + shift)
        vals.append(np.full(n, weights[k], dtype=np.float64))
        masks.append(ok)
    cols = np.stack(cols, axis=1)
    vals = np.stack(vals, axis=1)
    masks = np.stack(masks, axis=1)
    counts = masks.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[masks].astype(np.int32)
    val = vals[masks]
    return CSRMatrix(n, rowptr, colind, val)


def equilibrate(A: CSRMatrix) -> CSRMatrix:
    """A <- D^{-1/2} A D^{-1/2}, D_ii = max_j |a_ij| (Sec. 5)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    d = np.zeros(A.n)
    np.maximum.at(d, rows, np.abs(A.val))
    if np.any(d <= 0):
        raise ValueError("equilibration needs a nonzero entry in every row")
    s = 1.0 / np.sqrt(d)
    val = A.val * (s[rows] * s[A.colind])  # product first: exactly symmetric
    return CSRMatrix(A.n, A.rowptr.copy(), A.colind.copy(), val, dict(A.meta))


def poisson2d(m: int) -> CSRMatrix:
    """5-point Laplacian on an m x m grid, Dirichlet, diag 4, off -1, then equilibrated (/4)."""
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    w = [4.0, -1.0, -1.0, -1.0, -1.0]
    A = equilibrate(_stencil_csr((m, m), offs, w))
    A.meta.update(family="poisson2d", m=m, N_A=5)
    return A


def poisson3d(m: int) -> CSRMatrix:
    """7-point Laplacian on an m^3 grid, Dirichlet, diag 6, off -1, then equilibrated (/6)."""
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    w = [6.0] + [-1.0] * 6
    A = equilibrate(_stencil_csr((m, m, m), offs, w))
    A.meta.update(family="poisson3d", m=m, N_A=7)
    return A


def poisson_eig_bounds(dim: int, m: int) -> tuple[float, float]:
    """Extreme eigenvalues of the equilibrated dim-D Poisson matrix on an m^dim grid.

    The 1D Dirichlet Laplacian tridiag(-1, 2, -1) of size m has eigenvalues
    2 - 2 cos(k pi / (m+1)), k = 1..m; the dim-D operator is the Kronecker sum,
    and equilibration divides by the diagonal 2*dim.
    """
    lo = dim * (2.0 - 2.0 * math.cos(math.pi / (m + 1)))
    hi = dim * (2.0 - 2.0 * math.cos(m * math.pi / (m + 1)))
    return lo / (2 * dim), hi / (2 * dim)


def poisson_eigenvalues(dim: int, m: int) -> np.ndarray:
    """All eigenvalues (sorted) of the equilibrated dim-D Poisson matrix, closed form."""
    one = 2.0 - 2.0 * np.cos(np.arange(1, m + 1) * np.pi / (m + 1))
    grids = np.meshgrid(*([one] * dim), indexing="ij")
    return np.sort(sum(grids).ravel() / (2 * dim))


def fv_diffusion2d(m: int, sigma: float, rng: np.random.Generator) -> CSRMatrix:
    """Cell-centred finite-volume diffusion on an m x m grid, then equilibrated.

    Cell coefficient a_c = exp(sigma * N(0,1)). Interior face coefficient is the
    harmonic mean 2 a_i a_j / (a_i + a_j); a Dirichlet boundary face of cell i
    has coefficient 2 a_i. A_ii = sum of the cell's face coefficients,
    A_ij = -face(i, j).
    """
    a = np.exp(sigma * rng.standard_normal((m, m)))
    n = m * m
    # faces between (i, j) and (i+1, j) [vertical neighbours], (i, j) and (i, j+1)
    fv = 2.0 * a[:-1, :] * a[1:, :] / (a[:-1, :] + a[1:, :])   # (m-1, m)
    fh = 2.0 * a[:, :-1] * a[:, 1:] / (a[:, :-1] + a[:, 1:])   # (m, m-1)
    diag = np.zeros((m, m))
    diag[:-1, :] += fv
    diag[1:, :] += fv
    diag[:, :-1] += fh
    diag[:, 1:] += fh
    diag[0, :] += 2.0 * a[0, :]
    diag[-1, :] += 2.0 * a[-1, :]
    diag[:, 0] += 2.0 * a[:, 0]
    diag[:, -1] += 2.0 * a[:, -1]
    # neighbour values per cell in column order: up (-m), left (-1), self, right (+1), down (+m)
    up = np.zeros((m, m)); up[1:, :] = -fv
    down = np.zeros((m, m)); down[:-1, :] = -fv
    left = np.zeros((m, m)); left[:, 1:] = -fh
    right = np.zeros((m, m)); right[:, :-1] = -fh
    idx = np.arange(n, dtype=np.int64).reshape(m, m)
    has_up = np.zeros((m, m), bool); has_up[1:, :] = True
    has_down = np.zeros((m, m), bool); has_down[:-1, :] = True
    has_left = np.zeros((m, m), bool); has_left[:, 1:] = True
    has_right = np.zeros((m, m), bool); has_right[:, :-1] = True
    cols = np.stack([idx - m, idx - 1, idx, idx + 1, idx + m], axis=-1).reshape(n, 5)
    vals = np.stack([up, left, diag, right, down], axis=-1).reshape(n, 5)
    mask = np.stack([has_up, has_left, np.ones((m, m), bool), has_right, has_down], axis=-1).reshape(n, 5)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=rowptr[1:])
    A = CSRMatrix(n, rowptr, cols[mask].astype(np.int32), vals[mask])
    A = equilibrate(A)
    A.meta.update(family="fv_diffusion2d", m=m, sigma=sigma, N_A=5)
    return A


def banded_spd(n: int, hbw: int, rng: np.random.Generator) -> CSRMatrix:
    """Random banded SPD: A_ij ~ U[-1, 0] for 0 < |i-j| <= hbw (mirrored),
    A_ii = sum_j |A_ij| + 1e-3 (strictly diagonally dominant), then equilibrated."""
    hbw = int(min(hbw, n - 1))
    upper = [-rng.random(n - k) for k in range(1, hbw + 1)]  # diagonal k: entries (i, i+k)
    offs = list(range(-hbw, hbw + 1))
    cols = np.arange(n)[:, None] + np.array(offs)[None, :]
    mask = (cols >= 0) & (cols < n)
    vals = np.zeros((n, len(offs)))
    for k in range(1, hbw + 1):
        vals[: n - k, hbw + k] = upper[k - 1]        # (i, i+k)
        vals[k:, hbw - k] = upper[k - 1]             # (i+k, i) mirrored
    vals[:, hbw] = np.abs(vals).sum(axis=1) + 1e-3
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=rowptr[1:])
    A = CSRMatrix(n, rowptr, cols[mask].astype(np.int32), vals[mask])
    A = equilibrate(A)
    A.meta.update(family="banded", hbw=hbw, N_A=2 * hbw + 1)
    return A


def rhs_uniform(n: int, rng: np.random.Generator) -> np.ndarray:
    """b_i ~ U[-1, 1], normalised to ||b||_2 = 1."""
    b = rng.uniform(-1.0, 1.0, n)
    return b / np.linalg.norm(b)


# ---------------------------------------------------------------------------
# The named workloads. Each returns dict(A=CSRMatrix, b=..., x1=..., runs=[...]).
# ---------------------------------------------------------------------------

def seed_for(config: int) -> int:
    return 1000 + int(config)


def poisson2d_32():
    """2D Poisson 5-pt, 32x32 (n=1024, nnz=4992); classical CG, fixed s=4
    monomial s-step CG, adaptive monomial s_max=8 (s0=f=8, c=1), target 1e-10."""
    rng = np.random.default_rng(seed_for(1))
    A = poisson2d(32)
    b = rhs_uniform(A.n, rng)
    lo, hi = poisson_eig_bounds(2, 32)
    return dict(name="poisson2d_32", A=A, b=b, x1=np.zeros(A.n), lam=(lo, hi),
                runs=[dict(method="classical", eps=1e-10),
                      dict(method="fixed", basis="monomial", s=4, eps=1e-10),
                      dict(method="adaptive", basis="monomial", s_max=8, s0=8, f=8, c=1.0, eps=1e-10)])


def poisson3d_128():
    """3D Poisson 7-pt, 128^3 (n=2,097,152, nnz=14,581,760); adaptive Chebyshev
    s_max=16 with the closed-form eigenvalue bounds, target 1e-12."""
    rng = np.random.default_rng(seed_for(2))
    A = poisson3d(128)
    b = rhs_uniform(A.n, rng)
    lo, hi = poisson_eig_bounds(3, 128)
    return dict(name="poisson3d_128", A=A, b=b, x1=np.zeros(A.n), lam=(lo, hi),
                runs=[dict(method="adaptive", basis="chebyshev", s_max=16, s0=16, f=16, c=1.0, eps=1e-12),
                      dict(method="classical", eps=1e-12)])


def diffusion2d_2048():
    """2D FV diffusion, 2048x2048 (n=4,194,304), log-normal sigma=2 coefficients;
    adaptive Newton s_max=12 with 24 classical warm-up iterations, target 1e-10."""
    rng = np.random.default_rng(seed_for(3))
    A = fv_diffusion2d(2048, 2.0, rng)
    b = rhs_uniform(A.n, rng)
    return dict(name="diffusion2d_2048", A=A, b=b, x1=np.zeros(A.n), lam=None,
                runs=[dict(method="adaptive", basis="newton", s_max=12, s0=12, f=12, c=1.0, eps=1e-10,
                           newton_warmup=24),
                      dict(method="classical", eps=1e-10)])


def scaled(family: str, size: int, seed: int):
    """A smaller member of a family with the same structure, for parity tests.

    family in {"poisson2d", "poisson3d", "diffusion2d", "banded"}; size is the
    grid extent m (or n for banded).
    """
    rng = np.random.default_rng(seed)
    if family == "poisson2d":
        A = poisson2d(size); lam = poisson_eig_bounds(2, size)
    elif family == "poisson3d":
        A = poisson3d(size); lam = poisson_eig_bounds(3, size)
    elif family == "diffusion2d":
        A = fv_diffusion2d(size, 2.0, rng); lam = None
    elif family == "banded":
        A = banded_spd(size, int(rng.integers(8, 65)), rng); lam = None
    else:
        raise ValueError(family)
    b = rhs_uniform(A.n, rng)
    return dict(name=f"{family}_{size}", A=A, b=b, x1=np.zeros(A.n), lam=lam)


def batch_systems(count: int = 256, seed: int | None = None, nmin: float = 1e3, nmax: float = 2e5):
    """Batch of independent SPD systems (the uneven batched workload).

    Sizes are log-uniform on [nmin, nmax]; the family is uniform over 2D
    Poisson (m = round(sqrt n)), 3D Poisson (m = round(cbrt n)) and banded SPD
    (half-bandwidth ~ U{8..64}); targets are 1e-8 or 1e-12 with probability
    1/2 each; b ~ U[-1, 1] normalised, x1 = 0. Returns a list of dicts with A,
    b, x1, eps and the family name."""
    rng = np.random.default_rng(seed_for(4) if seed is None else seed)
    out = []
    for q in range(count):
        n = int(round(float(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))))
        fam = ("poisson2d", "poisson3d", "banded")[int(rng.integers(0, 3))]
        if fam == "poisson2d":
            A = poisson2d(max(2, int(round(n ** 0.5))))
        elif fam == "poisson3d":
            A = poisson3d(max(2, int(round(n ** (1.0 / 3.0)))))
        else:
            A = banded_spd(n, int(rng.integers(8, 65)), rng)
        eps = 1e-8 if rng.random() < 0.5 else 1e-12
        b = rhs_uniform(A.n, rng)
        out.append(dict(name=f"{fam}_{A.n}", family=fam, A=A, b=b, x1=np.zeros(A.n), eps=eps))
    return out


def serve_pool(size: int = 12, seed: int | None = None, nmin: float = 1e4, nmax: float = 4e6):
    """Operators for the served workload: `size` SPD matrices whose sizes sit
    at the quantiles (i + 1/2)/size of the log-uniform law on [nmin, nmax],
    families (2D Poisson, 3D Poisson, banded with half-bandwidth ~ U{8..64})
    dealt out in a seeded random order, equal numbers of each. Returns a list
    of dicts with A, family and name."""
    rng = np.random.default_rng(seed_for(5) if seed is None else seed)
    fams = np.array(["poisson2d", "poisson3d", "banded"] * ((size + 2) // 3))[:size]
    fams = fams[rng.permutation(size)]
    out = []
    for i in range(size):
        n = int(round(float(np.exp(np.log(nmin) + (i + 0.5) / size * (np.log(nmax) - np.log(nmin))))))
        fam = str(fams[i])
        if fam == "poisson2d":
            A = poisson2d(max(2, int(round(n ** 0.5))))
        elif fam == "poisson3d":
            A = poisson3d(max(2, int(round(n ** (1.0 / 3.0)))))
        else:
            A = banded_spd(n, int(rng.integers(8, 65)), rng)
        out.append(dict(name=f"{fam}_{A.n}", family=fam, A=A))
    return out


def serve_requests(count: int, pool_size: int = 12, seed: int | None = None):
    """Request stream of the served workload: for each request the pool
    operator (uniform), the relative target (uniform over 1e-6, 1e-8, 1e-10,
    1e-12), a seed for its right-hand side, and its inter-arrival gap for a
    Poisson process of rate 1 (exponential, mean 1; scale by 1/rate).
    Returns a dict of numpy arrays: op, eps, rhs_seed, gap."""
    rng = np.random.default_rng((seed_for(5) if seed is None else seed) + 1)
    return dict(op=rng.integers(0, pool_size, count), eps=rng.choice([1e-6, 1e-8, 1e-10, 1e-12], count),
                rhs_seed=rng.integers(0, 2 ** 62, count), gap=rng.exponential(1.0, count))


def fibonacci_s_sequence(s_max: int, count: int, s0: int = 1, s1: int = 1):
    """Block sizes s_k = min(s_max, s_{k-1} + s_{k-2}) (the Fibonacci-type growth
    of Imberti and Erhel that the paper cites as related work), starting from
    s0, s1: an input sequence for variable s-step CG (Alg. 3)."""
    seq = [min(s_max, s0), min(s_max, s1)]
    while len(seq) < count:
        seq.append(min(s_max, seq[-1] + seq[-2]))
    return seq[:count]
