"""ascg_gram_noalloc: the Gram matrix without any device allocation.

This entry point is for callers that must not call cudaMalloc or cudaFree.
Examples are code under a fixed device-memory budget owned by a host
framework, and latency-sensitive loops where cudaFree's device-wide
synchronisation would stall other streams. It keeps its partial sums in a
static device array instead.

The test calls it twice in a row through the C ABI on each shape (the calls
share the static array) and checks each result against ascg_gram, which
allocates: the two run the same kernels in the same summation order, so the
results must be the same bits. Both are also held to the oracle's Y^T Y
within the bound of the kernel that ran: the tensor-core bound (w >= 9 with
16-byte aligned columns) or the FP64 bound 2 gamma_n |Y|^T |Y| (narrow bases,
an odd leading dimension). This file is collected last on purpose. It must
pass alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from oracle import ascg_oracle as O

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def gamma_n(k):
    return k * EPS / (1 - k * EPS)


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1701_03989_gb300 as P
    torch.cuda.init()
    return P, torch


def _basis(torch, n, w, seed, ld):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((w, n)) * np.logspace(0, 3, w)[:, None]
    Yd = torch.zeros(w * ld + 2, dtype=torch.float64, device="cuda")
    Yd[: w * ld].view(w, ld)[:, :n] = torch.from_numpy(Y).cuda()
    return Y, Yd


def _bound(Y, tensor_cores):
    absY = np.abs(Y)
    n = Y.shape[1]
    fp64 = 2 * gamma_n(n) * (absY @ absY.T)   # the oracle's own error, and the FP64 kernel's
    if not tensor_cores:
        return fp64
    mx, l1 = absY.max(axis=1), absY.sum(axis=1)
    tc = 2.0 ** -51 * (mx[:, None] * l1[None, :] + l1[:, None] * mx[None, :]) + 2 * gamma_n(168) * (absY @ absY.T)
    return tc + fp64


# (n, w, seed, leading dimension, tensor-core kernel?)
CASES = [
    (70001, 33, 1, 70016, True),
    (5003, 17, 2, 5024, True),
    (70001, 5, 3, 70016, False),    # w < 9: the FP64 kernel
    (5003, 17, 4, 5003, False),     # odd leading dimension: no tensor copies, the FP64 kernel
    (70001, 33, 5, 70016, True),
]


def test_gram_noalloc_matches_gram_twice(env):
    P, torch = env
    for n, w, seed, ld, tcores in CASES:
        Y, Yd = _basis(torch, n, w, seed, ld)
        g_ref = torch.empty(w * w, dtype=torch.float64, device="cuda")
        P.ascg_gram(n, w, Yd, ld, g_ref)
        ref = g_ref.cpu().numpy().reshape(w, w)
        want = O.gram(Y.T)
        bound = _bound(Y, tcores)
        assert np.all(np.abs(ref - want) <= bound), (n, w)
        for _ in range(2):   # two calls in a row share the static scratch
            g = torch.full((w * w,), float("nan"), dtype=torch.float64, device="cuda")
            P.ascg_gram_noalloc(n, w, Yd, ld, g)
            torch.cuda.synchronize()
            a = g.cpu().numpy().reshape(w, w)
            assert np.array_equal(a, ref), (n, w, np.max(np.abs(a - ref)))   # same kernels, same bits
            assert np.all(np.abs(a - want) <= bound), (n, w)
            assert np.array_equal(a, a.T)


def test_gram_noalloc_rejects_oversize(env):
    P, torch = env
    Y, Yd = _basis(torch, 64, 3, 4, 64)
    g = torch.empty(34 * 34, dtype=torch.float64, device="cuda")
    with pytest.raises(P.AscgError) as e:
        P.ascg_gram_noalloc(64, 34, Yd, 64, g)
    assert e.value.status == P.ASCG_ERR_INVALID and "33" in P.last_error()
