"""Failure paths on the GPU, in forms that fault and hang nothing.

* A bounded wait that runs out: the stall test option makes the tensor-core
  Gram's first CTA skip one tensor copy and limits every wait to a few
  milliseconds, so a wait runs out by construction (a barrier that nothing
  completes). The CTA must give up cleanly, the solve must report
  ASCG_ERR_TIMEOUT, and the GPU context must stay usable: the next solve runs
  normally and gives the same bits as before.
* Breakdown made on the host: an indefinite matrix with a positive diagonal
  and a right-hand side along an eigenvector of a negative eigenvalue, so
  p^T A p < 0 in the first step. Classical and s-step CG must stop with
  ASCG_ERR_BREAKDOWN and a finite x (the paper is silent on breakdown; the
  reading is that a block with no admissible step ends the solve).
* Non-finite data made on the host: NaN in b is refused with
  ASCG_ERR_INVALID before any iteration.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1701_03989_gb300 as P
    torch.cuda.init()
    return P, torch


def _op(P, A):
    return P.ascg_op_create_csr(A.n, A.nnz, np.ascontiguousarray(A.rowptr, np.int64),
                                np.ascontiguousarray(A.colind, np.int32), np.ascontiguousarray(A.val, np.float64), 0)


def _solve(P, torch, op, b, kw, raise_on=None):
    import paper_1701_03989_gb300 as PP
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    o = P.make_options(**kw)
    res = P.ascg_solve(op, torch.from_numpy(np.ascontiguousarray(b)).cuda(), x, o,
                       raise_on=raise_on if raise_on is not None else tuple(PP.STATUS_NAMES))
    return res, x.cpu().numpy()


def test_gram_wait_runs_out_and_context_survives(env):
    P, torch = env
    A = W.poisson3d(23)                      # w = 33 in the first block
    b = W.rhs_uniform(A.n, np.random.default_rng(11))
    lam = W.poisson_eig_bounds(3, 23)
    kw = dict(method="adaptive", basis="chebyshev", s_max=16, lam=lam, eps_target=1e-12, max_iters=5000,
              gram_tc=True)                  # the tensor-core Gram at this size too
    op = _op(P, A)
    ref, xref = _solve(P, torch, op, b, kw)
    assert ref.status == P.ASCG_OK
    res, x = _solve(P, torch, op, b, dict(kw, test_gram_stall=True))
    assert res.status == P.ASCG_ERR_TIMEOUT, P.STATUS_NAMES.get(res.status)
    assert "timeout" in P.last_error()
    assert np.all(np.isfinite(x))
    torch.cuda.synchronize()                  # the context is still usable ...
    again, x2 = _solve(P, torch, op, b, kw)
    assert again.status == P.ASCG_OK          # ... and the next solve is unchanged, bit for bit
    assert again.iters == ref.iters and np.array_equal(x2, xref)
    P.ascg_op_destroy(op)


def _indefinite(n=64, off=-0.75):
    """Tridiagonal, diagonal 1, off-diagonal `off`: symmetric with a positive
    diagonal, eigenvalues 1 + 2 off cos(k pi / (n + 1)), the smallest negative
    for off = -0.75. Returns the matrix and the unit eigenvector of that
    eigenvalue (sin(k pi j / (n + 1)), k = 1)."""
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, off), (i, 1.0), (i + 1, off)):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                vals.append(v)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, np.asarray(rows) + 1, 1)
    A = W.CSRMatrix(n, np.cumsum(rp), np.asarray(cols, np.int32), np.asarray(vals))
    v = np.sin(np.pi * np.arange(1, n + 1) / (n + 1))
    lam = 1 + 2 * off * math.cos(math.pi / (n + 1))
    assert lam < 0
    return A, v / np.linalg.norm(v)


@pytest.mark.parametrize("kw", [dict(method="classical"), dict(method="adaptive", s_max=4),
                                dict(method="fixed", s_max=3)])
def test_indefinite_matrix_breaks_down(env, kw):
    P, torch = env
    A, v = _indefinite()
    op = _op(P, A)
    res, x = _solve(P, torch, op, v, dict(kw, eps_target=1e-10, max_iters=1000))
    assert res.status == P.ASCG_ERR_BREAKDOWN, P.STATUS_NAMES.get(res.status)
    assert "breakdown" in P.last_error()
    assert np.all(np.isfinite(x))
    P.ascg_op_destroy(op)


@pytest.mark.parametrize("kw", [dict(method="classical"), dict(method="adaptive", s_max=8)])
def test_nan_in_b_is_refused(env, kw):
    P, torch = env
    A = W.poisson2d(16)
    b = W.rhs_uniform(A.n, np.random.default_rng(12))
    b[17] = np.nan
    op = _op(P, A)
    res, x = _solve(P, torch, op, b, dict(kw, eps_target=1e-10))
    assert res.status == P.ASCG_ERR_INVALID and res.iters == 0
    assert np.all(x == 0.0)                    # x_1 untouched
    P.ascg_op_destroy(op)
