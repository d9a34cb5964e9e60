"""ascg_gram_noalloc: the Gram matrix without any device allocation.

This entry point is for callers that must not call cudaMalloc or cudaFree.
Examples are code under a fixed device-memory budget owned by a host
framework, and latency-sensitive loops where cudaFree's device-wide
synchronisation would stall other streams. It keeps its partial sums in a
static device array instead. The test calls it twice in a row through the C
ABI, on different shapes, and checks each result against ascg_gram (which
allocates) within the Gram parity bound 2*gamma_n*|Y|^T|Y| used for the
oracle comparison. This file is collected last on purpose. It must pass alone
in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1701_03989_gb300 as P
    torch.cuda.init()
    return P, torch


def _basis(torch, n, w, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((w, n)) * np.logspace(0, 3, w)[:, None]
    ld = n + (32 - n % 32) % 32
    Yd = torch.zeros(w * ld, dtype=torch.float64, device="cuda")
    Yd.view(w, ld)[:, :n] = torch.from_numpy(Y).cuda()
    return Y, Yd, ld


def test_gram_noalloc_matches_gram_twice(env):
    P, torch = env
    for n, w, seed in ((70001, 33, 1), (5003, 17, 2), (70001, 33, 3)):
        Y, Yd, ld = _basis(torch, n, w, seed)
        g_ref = torch.empty(w * w, dtype=torch.float64, device="cuda")
        P.ascg_gram(n, w, Yd, ld, g_ref)
        bound = 2 * (n * EPS / (1 - n * EPS)) * (np.abs(Y) @ np.abs(Y).T)
        for _ in range(2):   # two calls in a row share the static scratch
            g = torch.full((w * w,), float("nan"), dtype=torch.float64, device="cuda")
            P.ascg_gram_noalloc(n, w, Yd, ld, g)
            torch.cuda.synchronize()
            a = g.cpu().numpy().reshape(w, w)
            b = g_ref.cpu().numpy().reshape(w, w)
            assert np.all(np.isfinite(a))
            assert np.all(np.abs(a - b) <= bound)
            assert np.array_equal(a, a.T)


def test_gram_noalloc_rejects_oversize(env):
    P, torch = env
    Y, Yd, ld = _basis(torch, 64, 3, 4)
    g = torch.empty(34 * 34, dtype=torch.float64, device="cuda")
    with pytest.raises(P.AscgError) as e:
        P.ascg_gram_noalloc(64, 34, Yd, ld, g)
    assert e.value.status == P.ASCG_ERR_INVALID and "33" in P.last_error()
