"""The parity rules themselves (tests/parity.py), pinned on the CPU.

A GPU-side block list is built from an oracle run, and disagreements are
planted in it: each must be classified as the rules say (identical, exempt
near-threshold decision, or a mismatch)."""
import copy
import math

import numpy as np
import pytest

import parity
import workloads as W
from oracle import ascg_oracle as O


STOP_CODE = {"done": 0, "converged": 1, "break": 2, "breakdown": 3, "maxiter": 4}


def as_gpu(blocks):
    out = []
    for o in blocks:
        sk = [0.0] * 16
        for i, v, _ in o["kappas"]:
            sk[i - 1] = v
        out.append(dict(sbar=o["sbar"], stilde=o["stilde"], s_k=o["s_k"], m=o["m"], rnorm=o["rnorm"],
                        threshold=o["threshold"], gamma=o["gamma"], sqrt_kappa=sk, stop=STOP_CODE[o["stop"]]))
    return out


@pytest.fixture(scope="module")
def run():
    A = W.poisson2d(12)
    b = W.rhs_uniform(A.n, np.random.default_rng(0))
    r = O.adaptive_sstep_cg(O.Operator.from_csr(A), b, np.zeros(A.n), s_max=6, eps_target=1e-8, basis="monomial",
                            max_iters=500)
    assert r.converged and len(r.blocks) > 3
    return A, r


def test_identical_sequences(run):
    A, r = run
    exempt, bad = parity.compare_block_sequences(as_gpu(r.blocks), r.blocks, A.n, r.res_hist, 1e-8)
    assert exempt is None and not bad
    assert parity.final_residual_ok(r.true_res, r.true_res, 1e-8, None)
    assert not parity.final_residual_ok(2.5 * r.true_res, r.true_res, 1e-8, None)


def test_planted_s_k_mismatch_is_caught(run):
    A, r = run
    g = as_gpu(r.blocks)
    k = next(j for j, b in enumerate(r.blocks) if b["stilde"] >= 3)
    g[k]["s_k"] -= 1
    g[k]["stilde"] -= 1
    exempt, bad = parity.compare_block_sequences(g, r.blocks, A.n, r.res_hist, 1e-8)
    assert exempt == k and bad


def test_planted_near_threshold_decision_is_exempt(run):
    """The same disagreement becomes exempt when the oracle's sqrt(kappa) at
    that size lies within the criterion's uncertainty of the threshold."""
    A, r = run
    o = copy.deepcopy(r.blocks)
    k = next(j for j, b in enumerate(o) if b["stilde"] >= 3 and b["s_k"] == b["stilde"])
    i = o[k]["stilde"]
    T = [v for j, v, _ in o[k]["kappas"] if j == i][0] * (1 + 1e-9)  # oracle passes size i, barely
    o[k]["threshold"] = T
    g = as_gpu(o)
    g[k]["sqrt_kappa"][i - 1] = T * (1 + 1e-8)  # the GPU's estimate lands just above it
    g[k]["s_k"] = g[k]["stilde"] = i - 1
    exempt, bad = parity.compare_block_sequences(g, o, A.n, r.res_hist, 1e-8)
    assert exempt == k and not bad


def test_stop_decision_one_block_apart(run):
    """One side runs a block more: exempt only when the oracle's residual at the
    shorter side's stop lies within the history tolerance of the target."""
    A, r = run
    g = as_gpu(r.blocks)
    last = r.blocks[-1]
    extra = dict(g[-1], m=last["m"] + last["s_k"])
    i = last["m"] + last["s_k"]
    h = r.res_hist[i]
    # target just below the oracle's final residual: the GPU went on one block
    near_target = h - 0.5e-10
    exempt, bad = parity.compare_block_sequences(g + [extra], r.blocks, A.n, r.res_hist, near_target)
    assert exempt == len(r.blocks) - 1 and not bad
    # far from it: a real mismatch
    exempt, bad = parity.compare_block_sequences(g + [extra], r.blocks, A.n, r.res_hist, h * 100)
    assert bad
    # GPU stopped on convergence a block early (oracle went on): the same rule from the other side
    early = g[:-1]
    early[-1] = dict(early[-1], stop=1)
    prev = r.blocks[-2]
    h_prev = r.res_hist[prev["m"] + prev["s_k"]]
    exempt, bad = parity.compare_block_sequences(early, r.blocks, A.n, r.res_hist, h_prev + 0.5e-10)
    assert exempt == len(early) - 1 and not bad
    exempt, bad = parity.compare_block_sequences(early, r.blocks, A.n, r.res_hist, h_prev / 100)
    assert bad
    # a side that ended for another reason (an iteration cap) decided nothing: prefix comparison
    capped = g[:-1]
    capped[-1] = dict(capped[-1], stop=4)
    exempt, bad = parity.compare_block_sequences(capped, r.blocks, A.n, r.res_hist, 1e-8)
    assert exempt is None and not bad


def test_final_residual_rule_after_a_flipped_stop():
    assert parity.final_residual_ok(4.7e-9, 9.87e-9, 1e-8, 3)
    assert parity.final_residual_ok(1.9e-8, 9.87e-9, 1e-8, 3)
    assert not parity.final_residual_ok(2.1e-8, 9.87e-9, 1e-8, 3)
    assert parity.final_residual_ok(4.7e-9, 9.87e-9, 1e-8, None)      # 2x lower, under the target
    assert not parity.final_residual_ok(4.7e-9, 9.87e-9, 1e-9, None)  # 2x lower, above the target
    assert not parity.final_residual_ok(2.1e-8, 1.0e-8, 1e-7, None)   # more than 2x higher
    assert math.isfinite(parity.kappa_uncertainty(10.0, 5, 100))


def test_stop_decision_after_finite_termination_is_exempt(run):
    """A stop decision after n iterations (finite termination) is on rounding
    noise: exempt whatever the residuals."""
    A, r = run
    g = as_gpu(r.blocks)
    last = r.blocks[-1]
    extra = dict(g[-1], m=last["m"] + last["s_k"])
    i = last["m"] + last["s_k"]
    exempt, bad = parity.compare_block_sequences(g + [extra], r.blocks, i, r.res_hist, r.res_hist[i] * 100)
    assert exempt == len(r.blocks) - 1 and not bad
    exempt, bad = parity.compare_block_sequences(g + [extra], r.blocks, i + 1, r.res_hist, r.res_hist[i] * 100)
    assert bad
