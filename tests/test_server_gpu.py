"""Solve server (ascg_server_*): continuous batching over the lockstep engine.

Requests of uneven sizes and targets arrive while others run; the server
admits them in submission order as device memory and system slots free up.
Each served result must be bitwise the same as the same system solved alone
(ascg_solve_batch with one system), whatever ran beside it, and the admission
must respect the memory budget and the slot count.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ascg_oracle as O

pytestmark = pytest.mark.gpu
S_MAX = 10


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1701_03989_gb300 as P
    torch.cuda.init()
    return P, torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def make_op(P, A):
    return P.ascg_op_create_csr(A.n, A.nnz, np.ascontiguousarray(A.rowptr, np.int64),
                                np.ascontiguousarray(A.colind, np.int32), np.ascontiguousarray(A.val, np.float64), 0)


def opts(P, max_iters=4000):
    return P.make_options(method="adaptive", basis="monomial", s_max=S_MAX, eps_target=1e-10, max_iters=max_iters)


def gram_item_rows(n):
    r = 1024
    while r < 8192 and r * 16 < n:
        r *= 2
    return r


def footprint(n, s_max=S_MAX):
    """Device bytes the server counts for a system: basis rows rounded to 1024,
    FP64 Gram partials per item and tensor-core Gram partials per 8192 rows."""
    w = 2 * s_max + 1
    rows = -(-n // 1024) * 1024
    np_ = w * (w + 1) // 2
    return w * rows * 8 + -(-n // gram_item_rows(n)) * np_ * 8 + -(-rows // 8192) * np_ * 8


def solve_alone(P, torch, op, b, x1, eps, max_iters=4000):
    x = dev(torch, x1)
    res, _ = P.ascg_solve_batch([op], [dev(torch, b)], [x], opts(P, max_iters), eps_targets=[eps])
    return res[0], x.cpu().numpy()


def serve(P, torch, srv, systems, ops, waves, stats_log=None):
    """Submits the systems in waves (lists of indices), running `gap` server
    steps between waves; then steps until idle. Returns {index: (completion, x)}."""
    xs = {q: dev(torch, systems[q]["x1"]) for wave, _ in waves for q in wave}
    bs = {q: dev(torch, systems[q]["b"]) for wave, _ in waves for q in wave}
    done = {}
    order = []
    for wave, gap in waves:
        for q in wave:
            P.ascg_server_submit(srv, ops[q], bs[q], xs[q], systems[q]["eps"], q)
            order.append(q)
        for _ in range(gap):
            comps, _, _ = P.ascg_server_step(srv)
            for c in comps:
                done[c.tag] = c
            if stats_log is not None:
                stats_log.append(P.ascg_server_info(srv))
    for _ in range(100000):
        comps, nact, npend = P.ascg_server_step(srv, cap=3)
        for c in comps:
            done[c.tag] = c
        if stats_log is not None:
            stats_log.append(P.ascg_server_info(srv))
        if nact == 0 and npend == 0:
            break
    assert sorted(done) == sorted(order)
    return {q: (done[q], xs[q].cpu().numpy()) for q in order}, order


def mixed_systems(seed=21, count=10):
    sys = W.batch_systems(count, seed=seed, nmin=100, nmax=6000)
    rng = np.random.default_rng(seed)
    for s in sys:  # targets across the served range
        s["eps"] = float(rng.choice([1e-6, 1e-8, 1e-10, 1e-12]))
    return sys


def test_served_results_equal_alone(env):
    """Continuous batching: a first wave runs one step before the second
    arrives; a budget of a third of the total footprint forces queueing. Every
    served system equals its solve alone, bit for bit."""
    P, torch = env
    systems = mixed_systems()
    ops = [make_op(P, s["A"]) for s in systems]
    fp = [footprint(s["A"].n) for s in systems]
    budget = max(max(fp), sum(fp) // 3) + 65536
    srv = P.ascg_server_create(opts(P), budget, 8)
    log = []
    try:
        served, order = serve(P, torch, srv, systems, ops, [(list(range(5)), 1), (list(range(5, 10)), 0)], log)
    finally:
        P.ascg_server_destroy(srv)
    for st in log:
        assert st.basis_bytes_used <= st.basis_bytes_total
        assert st.systems_running <= 8
    # admission is FIFO: admission steps never decrease in submission order
    adm = [served[q][0].step_admitted for q in order]
    assert adm == sorted(adm)
    assert max(st.queued for st in log) > 0  # some requests had to wait
    for q in range(len(systems)):
        c, x = served[q]
        r, xa = solve_alone(P, torch, ops[q], systems[q]["b"], systems[q]["x1"], systems[q]["eps"])
        assert c.result.status == P.ASCG_OK == r.status, systems[q]["name"]
        assert c.result.iters == r.iters and c.result.blocks == r.blocks, systems[q]["name"]
        assert c.result.rel_res_true == r.rel_res_true and c.result.rel_res_updated == r.rel_res_updated
        assert np.array_equal(x, xa), systems[q]["name"]
        assert c.result.rel_res_updated <= systems[q]["eps"]
        assert c.latency_ms >= c.queue_ms >= 0.0
    for op in ops:
        P.ascg_op_destroy(op)


def test_shortest_first_admission_and_large_cap(env):
    """ASCG_ADMIT_SHORTEST_FIRST: with room for one system at a time, the
    waiting requests are admitted in increasing estimated work (rows times
    target digits), and every result is still bitwise the same as alone. A
    large-class cap of 1 keeps two large systems from running at once."""
    P, torch = env
    rng = np.random.default_rng(33)
    mats = [W.poisson2d(60), W.poisson2d(20), W.banded_spd(2000, 12, rng), W.poisson2d(30)]
    epss = [1e-10, 1e-8, 1e-6, 1e-12]
    systems = [dict(name=f"s{i}_{A.n}", A=A, b=W.rhs_uniform(A.n, rng), x1=np.zeros(A.n), eps=e)
               for i, (A, e) in enumerate(zip(mats, epss))]
    ops = [make_op(P, s["A"]) for s in systems]
    srv = P.ascg_server_create(opts(P), 1 << 30, 1)      # one slot: requests wait their turn
    P.ascg_server_set_policy(srv, P.ASCG_ADMIT_SHORTEST_FIRST, 0)
    try:
        # the first request takes the slot at once; the other three wait and are
        # then admitted shortest first
        served, order = serve(P, torch, srv, systems, ops, [([0], 1), ([1, 2, 3], 0)])
    finally:
        P.ascg_server_destroy(srv)
    work = {q: systems[q]["A"].n * max(1.0, -np.log10(systems[q]["eps"])) for q in range(4)}
    waiting = sorted([1, 2, 3], key=lambda q: work[q])
    adm = [served[q][0].step_admitted for q in waiting]
    assert adm == sorted(adm) and len(set(adm)) == 3, (adm, waiting)
    for q, s in enumerate(systems):
        c, x = served[q]
        r, xa = solve_alone(P, torch, ops[q], s["b"], s["x1"], s["eps"])
        assert c.result.status == P.ASCG_OK == r.status and np.array_equal(x, xa), s["name"]
    # large-class cap: two systems of >= 2^19 rows never run at once
    big = [W.poisson3d(81), W.poisson3d(82)]
    assert all(A.n >= 1 << 19 for A in big)
    bsys = [dict(name=f"big{i}", A=A, b=W.rhs_uniform(A.n, rng), x1=np.zeros(A.n), eps=1e-6)
            for i, A in enumerate(big)]
    bops = [make_op(P, s["A"]) for s in bsys]
    srv = P.ascg_server_create(opts(P), 1 << 32, 8)
    P.ascg_server_set_policy(srv, P.ASCG_ADMIT_FIFO, 1)
    log = []
    try:
        bserved, _ = serve(P, torch, srv, bsys, bops, [([0, 1], 0)], log)
    finally:
        P.ascg_server_destroy(srv)
    assert max(st.systems_running for st in log) == 1
    assert bserved[1][0].step_admitted >= bserved[0][0].step_done
    for q, s in enumerate(bsys):
        c, x = bserved[q]
        r, xa = solve_alone(P, torch, bops[q], s["b"], s["x1"], s["eps"])
        assert c.result.status == P.ASCG_OK == r.status and np.array_equal(x, xa), s["name"]
    # yield: with a small system running, the large class starts no block, so
    # the small system, submitted with the large one, finishes first
    ysys = [dict(name="big", A=big[0], b=W.rhs_uniform(big[0].n, rng), x1=np.zeros(big[0].n), eps=1e-6),
            dict(name="small", A=W.poisson2d(30), b=None, x1=None, eps=1e-8)]
    ysys[1]["b"], ysys[1]["x1"] = W.rhs_uniform(900, rng), np.zeros(900)
    yops = [make_op(P, q["A"]) for q in ysys]
    srv = P.ascg_server_create(opts(P), 1 << 32, 8)
    P.ascg_server_set_policy(srv, P.ASCG_ADMIT_FIFO, 0, True)
    try:
        yserved, _ = serve(P, torch, srv, ysys, yops, [([0, 1], 0)])
    finally:
        P.ascg_server_destroy(srv)
    assert yserved[1][0].step_done < yserved[0][0].step_done
    for q, sy in enumerate(ysys):
        c, x = yserved[q]
        r, xa = solve_alone(P, torch, yops[q], sy["b"], sy["x1"], sy["eps"])
        assert c.result.status == P.ASCG_OK == r.status and np.array_equal(x, xa), sy["name"]
    for op in yops:
        P.ascg_op_destroy(op)
    with pytest.raises(P.AscgError):
        srv2 = P.ascg_server_create(opts(P), 1 << 20, 2)
        try:
            P.ascg_server_set_policy(srv2, 7, 0)
        finally:
            P.ascg_server_destroy(srv2)
    for op in ops + bops:
        P.ascg_op_destroy(op)


def test_served_size_classes_equal_alone(env):
    """Systems in all three size classes (n < 2^16, < 2^19, larger), each class
    stepping on its own stream: every result equals its solve alone, bit for
    bit, and the two large lanes run the tensor-core Gram."""
    P, torch = env
    rng = np.random.default_rng(17)
    mats = [W.poisson2d(40), W.banded_spd(3000, 20, rng), W.poisson3d(65), W.poisson3d(81), W.poisson2d(60)]
    assert mats[2].n >= 1 << 18 and mats[3].n >= 1 << 19
    systems = [dict(name=f"s{i}_{A.n}", A=A, b=W.rhs_uniform(A.n, rng), x1=np.zeros(A.n), eps=e)
               for i, (A, e) in enumerate(zip(mats, [1e-10, 1e-8, 1e-8, 1e-6, 1e-12]))]
    ops = [make_op(P, s["A"]) for s in systems]
    srv = P.ascg_server_create(opts(P), 1 << 30, 16)
    try:
        served, _ = serve(P, torch, srv, systems, ops, [([0, 1, 2, 3], 2), ([4], 0)])
    finally:
        P.ascg_server_destroy(srv)
    for q, s in enumerate(systems):
        c, x = served[q]
        r, xa = solve_alone(P, torch, ops[q], s["b"], s["x1"], s["eps"])
        assert c.result.status == P.ASCG_OK == r.status, s["name"]
        assert c.result.iters == r.iters and c.result.rel_res_true == r.rel_res_true, s["name"]
        assert np.array_equal(x, xa), s["name"]
        assert c.result.rel_res_updated <= s["eps"]
    for op in ops:
        P.ascg_op_destroy(op)


def test_served_result_against_oracle(env):
    """Served systems against the FP64 oracle: each served result equals the
    system solved alone bit for bit, and that solve, with its block records,
    meets the parity rules (s_k sequence up to near-threshold decisions,
    residual history, true residual within 2x). The target 1e-8 keeps the
    true residuals well above the rounding floor eps ||A|| ||x||."""
    import parity
    from test_batch_gpu import run_batch
    P, torch = env
    systems = mixed_systems(seed=5, count=4)[:3]
    for s in systems:
        s["eps"] = 1e-8
    ops = [make_op(P, s["A"]) for s in systems]
    srv = P.ascg_server_create(opts(P), 1 << 28, 4)
    try:
        served, _ = serve(P, torch, srv, systems, ops, [([0, 1, 2], 0)])
    finally:
        P.ascg_server_destroy(srv)
    for q, s in enumerate(systems):
        g = run_batch(P, torch, [s], s_max=S_MAX)[0][0]
        c, x = served[q]
        assert np.array_equal(x, g["x"]) and c.result.iters == g["res"].iters
        orc = O.adaptive_sstep_cg(O.Operator.from_csr(s["A"]), s["b"], s["x1"], s_max=S_MAX, eps_target=s["eps"],
                                  basis="monomial", max_iters=4000)
        assert orc.converged and c.result.status == P.ASCG_OK
        exempt, bad = parity.compare_block_sequences(g["blocks"], orc.blocks, s["A"].n, orc.res_hist, s["eps"])
        assert not bad, (s["name"], bad)
        nwin = min(parity.history_window(g["blocks"], orc.blocks, exempt, iters=20), len(g["hist"]),
                   len(orc.res_hist), s["A"].n)
        ho = np.asarray(orc.res_hist[:nwin])
        tau = parity.history_tolerance(orc.blocks, ho, nwin)
        assert np.all(np.abs(g["hist"][:nwin] - ho) <= tau), s["name"]
        assert parity.final_residual_ok(c.result.rel_res_true, orc.true_res, s["eps"], exempt), (
            s["name"], c.result.rel_res_true, orc.true_res)
        if exempt is None:
            assert c.result.iters == orc.iters, (s["name"], c.result.iters, orc.iters)
    for op in ops:
        P.ascg_op_destroy(op)


def test_server_slots_and_edge_requests(env):
    """One slot: requests run one after another. A zero right-hand side and an
    exact start complete at admission with no block; a request larger than
    the budget is refused at submission."""
    P, torch = env
    A1 = W.poisson2d(9)
    A2 = W.poisson2d(12)
    b2 = W.rhs_uniform(A2.n, np.random.default_rng(1))
    xs2 = np.linalg.solve(A2.to_dense(), b2)
    A3 = W.banded_spd(700, 12, np.random.default_rng(2))
    systems = [
        dict(name="zero_rhs", A=A1, b=np.zeros(A1.n), x1=np.ones(A1.n), eps=1e-10),
        dict(name="solved", A=A2, b=b2, x1=xs2, eps=1e-8),
        dict(name="banded", A=A3, b=W.rhs_uniform(A3.n, np.random.default_rng(3)), x1=np.zeros(A3.n), eps=1e-12),
        dict(name="banded2", A=A3, b=W.rhs_uniform(A3.n, np.random.default_rng(4)), x1=np.zeros(A3.n), eps=1e-8),
    ]
    ops = [make_op(P, s["A"]) for s in systems]
    srv = P.ascg_server_create(opts(P), 1 << 26, 1)
    log = []
    try:
        served, order = serve(P, torch, srv, systems, ops, [([0, 1, 2, 3], 0)], log)
        big = W.poisson2d(64)
        opb = make_op(P, big)
        tiny = P.ascg_server_create(opts(P), footprint(big.n) - 1, 2)
        with pytest.raises(P.AscgError) as e:
            P.ascg_server_submit(tiny, opb, dev(torch, np.ones(big.n)), dev(torch, np.zeros(big.n)), 1e-8, 99)
        assert e.value.status == P.ASCG_ERR_INVALID
        P.ascg_server_destroy(tiny)
        P.ascg_op_destroy(opb)
    finally:
        P.ascg_server_destroy(srv)
    assert all(st.systems_running <= 1 for st in log)
    c0, x0 = served[0]
    assert c0.result.iters == 0 and c0.result.status == P.ASCG_OK and np.array_equal(x0, np.zeros(A1.n))
    c1, x1 = served[1]
    assert c1.result.iters == 0 and np.array_equal(x1, xs2)
    # one slot: system 3 is admitted only after system 2 completed
    assert served[3][0].step_admitted >= served[2][0].step_done
    for q in (2, 3):
        r, xa = solve_alone(P, torch, ops[q], systems[q]["b"], systems[q]["x1"], systems[q]["eps"])
        assert np.array_equal(served[q][1], xa)
    for op in ops:
        P.ascg_op_destroy(op)


def test_server_iteration_cap(env):
    """max_iters stops a served system with ASCG_NOT_CONVERGED, like a batch."""
    P, torch = env
    A = W.banded_spd(900, 30, np.random.default_rng(7))
    s = dict(name="capped", A=A, b=W.rhs_uniform(A.n, np.random.default_rng(8)), x1=np.zeros(A.n), eps=1e-12)
    op = make_op(P, A)
    srv = P.ascg_server_create(opts(P, max_iters=9), 1 << 26, 2)
    try:
        served, _ = serve(P, torch, srv, [s], [op], [([0], 0)])
    finally:
        P.ascg_server_destroy(srv)
    c, x = served[0]
    assert c.result.status == P.ASCG_NOT_CONVERGED and c.result.iters == 9
    r, xa = solve_alone(P, torch, op, s["b"], s["x1"], s["eps"], max_iters=9)
    assert np.array_equal(x, xa)
    P.ascg_op_destroy(op)


def test_served_stream_full_size_pool(env):
    """Requests drawn from the served workload's operator pool (sizes at
    log-uniform quantiles of [1e4, 4e6]) and targets, all submitted at once to a
    server with the default budget split: every request converges, and the
    three smallest are bitwise the same solved alone."""
    P, torch = env
    pool = W.serve_pool()
    req = W.serve_requests(24)
    ops = [make_op(P, p["A"]) for p in pool]
    nop = [p["A"].n for p in pool]
    rng = np.random.default_rng(99)
    systems = []
    for i in range(len(req["op"])):
        n = nop[req["op"][i]]
        systems.append(dict(name=f"req{i}_{n}", A=pool[req["op"][i]]["A"], b=W.rhs_uniform(n, rng), x1=np.zeros(n),
                            eps=float(req["eps"][i])))
    sys_ops = [ops[req["op"][i]] for i in range(len(systems))]
    srv = P.ascg_server_create(opts(P, max_iters=60000), 40 * (1 << 30), 64)
    try:
        served, _ = serve(P, torch, srv, systems, sys_ops, [(list(range(len(systems))), 0)])
    finally:
        P.ascg_server_destroy(srv)
    for q, s in enumerate(systems):
        c, _ = served[q]
        assert c.result.status == P.ASCG_OK, s["name"]
        assert c.result.rel_res_updated <= s["eps"] and c.result.rel_res_true <= 4 * s["eps"], s["name"]
    for q in sorted(range(len(systems)), key=lambda q: systems[q]["A"].n)[:3]:
        r, xa = solve_alone(P, torch, sys_ops[q], systems[q]["b"], systems[q]["x1"], systems[q]["eps"],
                            max_iters=60000)
        assert np.array_equal(served[q][1], xa), systems[q]["name"]
    for op in ops:
        P.ascg_op_destroy(op)
