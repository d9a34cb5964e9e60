"""Helpers for comparing the CUDA path with the oracle (test infrastructure).

Tolerances are derived from the arithmetic (see each function):
  * residual histories over the first 20 iterations: 1e-10 absolute on
    ||r_i||/||b||, widened to eps * kappa(G) * ||r_i||/||b|| inside blocks whose
    Gram matrix is ill conditioned. The updated residual norm is a quadratic
    form in G, whose first-order relative sensitivity to rounding in G and in
    the coordinate steps is eps * kappa(G). The oracle itself moves by that much
    under a different valid summation order of Y^T Y (tests/test_tolerances.py);
  * s_k sequences: identical, except where the oracle's decision lies within
    the uncertainty of its criterion. For the kappa test, that uncertainty is
    max(1e-6, K w sqrt(n) eps kappa): the two sides form G in different
    summation orders, which moves lambda_min by about sqrt(n) eps lambda_max.
    After the first exempt block only the earlier iterations are compared;
  * final true residual: within a factor 2 of the oracle's when both sides
    stop at the same iteration, read as: never more than 2x above it, and more
    than 2x below it only under the target. The true residual is the updated
    one plus the residual gap of eq. (fb), which rounding sets; with c = 1
    the method keeps that gap near eps*, so at a target the gap can cancel
    part of the residual on one side and not on the other. A lower true
    residual is no loss of accuracy. A stop decision ("||r_i|| <= eps*")
    whose oracle residual lies within the history tolerance of the target may
    flip, since the histories themselves may differ by that much; the two runs
    then end at different iterations, and the GPU's true residual must stay
    within 2x of max(oracle's, target).
"""
from __future__ import annotations

import math

import numpy as np

EPS = 2.0 ** -53
K_UNCERTAINTY = 64.0


def kappa_uncertainty(sk: float, w: int, n: int) -> float:
    """Relative uncertainty of sqrt(kappa(G_sub)) from rounding in G and its eigenvalues."""
    if not math.isfinite(sk):
        return math.inf
    return max(1e-6, K_UNCERTAINTY * w * math.sqrt(n) * EPS * sk * sk)


def decision_is_near(sk_o: float, sk_g: float, T: float, w: int, n: int) -> bool:
    """True if the two sides may legitimately disagree on 'sqrt(kappa) <= T'."""
    pass_o, pass_g = sk_o <= T, sk_g <= T
    if pass_o == pass_g:
        return False
    if math.isfinite(sk_o) and math.isfinite(sk_g):
        return abs(sk_o - T) <= kappa_uncertainty(sk_o, w, n) * T or abs(sk_g - T) <= kappa_uncertainty(sk_g, w, n) * T
    # one side certified the basis, the other did not: only near the floor
    # lambda_min = w sqrt(n) eps lambda_max, i.e. kappa ~ 1 / (w sqrt(n) eps)
    fin = sk_o if math.isfinite(sk_o) else sk_g
    floor_sk = math.sqrt(1.0 / (w * math.sqrt(n) * EPS))
    return fin >= floor_sk / 8.0


def block_kappa(o) -> float:
    """kappa(G_{k,s~}) of an oracle block record (gamma^2); 1 when uncertified at s~ = 1."""
    g = o.get("gamma", 1.0)
    if not math.isfinite(g):
        return 1.0
    return max(1.0, g * g)


def compare_block_sequences(gpu_blocks, oracle_blocks, n: int, oracle_hist=None, target=None):
    """Walks both block sequences. Returns (index of the first exempt block or
    None, list of mismatch messages that are not exempt).

    A block is exempt when its decision lies within the uncertainty of its
    criterion, or when the two trajectories entering it already differ by
    more than 1e-6 in ||r_{m+1}|| (which earlier ill-conditioned blocks can
    cause legitimately; the history tolerance checks that part).
    oracle_hist / target (relative residual history and eps_target) let a
    convergence decision count as near when the residual at either side's
    stopping step is within its uncertainty of the target."""
    bad = []
    kacc = 1.0
    for k, (g, o) in enumerate(zip(gpu_blocks, oracle_blocks)):
        if g["sbar"] != o["sbar"]:
            bad.append(f"block {k}: sbar {g['sbar']} vs {o['sbar']}")
            return k, bad
        if "rnorm" in g and abs(g["rnorm"] - o["rnorm"]) > 1e-6 * o["rnorm"]:
            return k, bad
        kacc = max(kacc, block_kappa(o))
        same = g["stilde"] == o["stilde"] and g["s_k"] == o["s_k"]
        if same:
            continue
        T = o["threshold"]
        near = False
        sk_o = {i: s for i, s, _ in o.get("kappas", [])}
        for i in range(1, g["sbar"] + 1):
            if i in sk_o:
                if decision_is_near(sk_o[i], g["sqrt_kappa"][i - 1], T, 2 * i + 1, n):
                    near = True
        # in-loop check: gamma >= T_j
        for j, tj in o.get("checks", []):
            if abs(o["gamma"] - tj) <= kappa_uncertainty(o["gamma"], 2 * o["stilde"] + 1, n) * tj:
                near = True
        if oracle_hist is not None and target is not None:
            unc = max(1e-6, EPS * kacc)
            for s_ in (g["s_k"], o["s_k"]):
                i = o["m"] + s_
                if i < len(oracle_hist) and abs(oracle_hist[i] - target) <= unc * target:
                    near = True
        if near:
            return k, bad
        bad.append(f"block {k}: stilde/s_k gpu {g['stilde']}/{g['s_k']} oracle {o['stilde']}/{o['s_k']} "
                   f"T={T:.6g} sk_gpu={list(g['sqrt_kappa'][:g['sbar']])} sk_or={o.get('kappas')}")
        return k, bad
    shorter = gpu_blocks if len(gpu_blocks) < len(oracle_blocks) else oracle_blocks
    if len(gpu_blocks) != len(oracle_blocks) and shorter and _stopped_converged(shorter[-1]):
        # Both ran their common blocks alike; after the last of them one side
        # stopped on convergence and the other went on: a stop decision at
        # iteration i. (A side that ended for another reason, such as an
        # iteration cap on a prefix comparison, decided nothing.)
        k = len(shorter) - 1
        o = oracle_blocks[k]
        i = o["m"] + o["s_k"]
        # after n iterations CG has terminated in exact arithmetic: every later
        # residual, and any stop decision on it, is rounding noise
        near = i >= n
        if not near and oracle_hist is not None and target is not None and i < len(oracle_hist):
            tol = max(1e-10, EPS * kacc * oracle_hist[i], max(1e-6, EPS * kacc) * target)
            near = abs(oracle_hist[i] - target) <= tol
        if near:
            return k, bad
        bad.append(f"after block {k}: {len(gpu_blocks)} gpu blocks vs {len(oracle_blocks)} oracle blocks")
        return k, bad
    return None, bad


def _stopped_converged(block) -> bool:
    st = block.get("stop")
    return st == "converged" or st == 1  # oracle record / ascg_block_info (ASCG_STOP_CONVERGED)


def final_residual_ok(gpu_true: float, oracle_true: float, target: float, exempt_block) -> bool:
    """Final true residual rule (see the module docstring)."""
    if exempt_block is None:
        return gpu_true <= 2.0 * oracle_true and (gpu_true >= 0.5 * oracle_true or gpu_true <= target)
    return gpu_true <= 2.0 * max(oracle_true, target)


def gpu_blocks_from_infos(infos, count):
    out = []
    for i in range(count):
        b = infos[i]
        out.append(dict(sbar=b.sbar, stilde=b.stilde, s_k=b.s_k, stop=b.stop, m=b.m, rnorm=b.rnorm,
                        threshold=b.threshold, gamma=b.gamma, sqrt_kappa=[b.sqrt_kappa[j] for j in range(16)]))
    return out


def history_tolerance(oracle_blocks, oracle_hist, count: int):
    """tau_i = max(1e-10, eps * K_i * h_i), K_i = the largest kappa(G_{k,s~})
    over the blocks up to the one that produced iteration i."""
    tau = np.full(count, 1e-10)
    kacc = 1.0
    for o in oracle_blocks:
        kacc = max(kacc, block_kappa(o))
        for i in range(o["m"] + 1, min(o["m"] + o["s_k"] + 1, count)):
            tau[i] = max(1e-10, EPS * kacc * oracle_hist[i])
    return tau


def history_window(gpu_blocks, oracle_blocks, exempt_block, iters=20, offset=0):
    """Number of leading history entries to compare: the first `iters`
    iterations, cut at the start of the first exempt block."""
    limit = iters
    if exempt_block is not None:
        m = oracle_blocks[exempt_block]["m"]
        limit = min(limit, m)
    return limit + 1  # entry 0 is the initial residual
