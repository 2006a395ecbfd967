"""Serving engine (mb_server_*): continuous batching, admission by footprint,
and per-request results that do not depend on the other requests in flight.

Bar: each request's body velocities within 1e-6 relative of the same problem
solved alone (mb_solve_mobility) and of the oracle's direct solve.
"""
import numpy as np
import pytest
import torch

import paper_1602_02170_gb300 as mb
from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I
from tests.gpu_common import ctx, dev, host, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu
A = 0.1625


def _prob(s):
    return dict(q=dev(s.q), theta=dev(s.theta), blob_start=dev(s.blob_start, torch.int64),
                rho=dev(s.rho), F=dev(s.F), T=dev(s.T))


def _alone(ctx, P):
    U, W, lam, _ = ctx.solve_mobility(P["q"], P["theta"], P["blob_start"], P["rho"], P["F"], P["T"],
                                      A, 1.0, True, tol=1e-10, prec="mixed")
    return host(U), host(W)


def test_server_requests_join_mid_flight(ctx):
    first = [I.mixed_suspension(200 + k, nb) for k, nb in enumerate([12, 5])]
    later = [I.mixed_suspension(300 + k, nb) for k, nb in enumerate([3, 9, 1])]
    srv = mb.Server(ctx, A, tol=1e-10, prec="mixed", max_blobs=20000, max_bodies=500,
                    max_requests=16)
    probs, tickets, outs = [], [], []
    for s in first:
        P = _prob(s)
        t, o = srv.submit(P)
        probs.append((s, P)); tickets.append(t); outs.append(o)
    srv.step()
    srv.step()
    assert srv.poll(tickets[0])[0] == mb.Server.RUNNING
    for s in later:
        P = _prob(s)
        t, o = srv.submit(P)
        probs.append((s, P)); tickets.append(t); outs.append(o)
    nr, nq = srv.step()
    # the late requests were admitted while the first ones were still running
    assert nr == 5 and nq == 0
    assert srv.poll(tickets[0])[0] == mb.Server.RUNNING
    srv.run_until_idle()
    for (s, P), t, (U, W, lam) in zip(probs, tickets, outs):
        state, info, status = srv.poll(t)
        assert state == mb.Server.DONE and status == "MB_OK", (state, status, info)
        assert info["converged"] == 1 and info["rel_residual"] <= 1e-10
        Ua, Wa = _alone(ctx, P)
        assert rel_l2(host(U), Ua) <= 1e-6 and rel_l2(host(W), Wa) <= 1e-6
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Ur, Wr, lr = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, A, 1.0, True)
        assert rel_l2(host(U), Ur) <= 1e-6 and rel_l2(host(W), Wr) <= 1e-6
        assert rel_l2(host(lam), lr) <= 1e-5
    srv.close()


def test_server_admission_by_footprint(ctx):
    """An arena with room for one request at a time still serves them all,
    one after the other; a request bigger than the arena is refused."""
    susp = [I.mixed_suspension(400 + k, 6) for k in range(3)]
    cap = max(s.n_blobs for s in susp) + 10
    srv = mb.Server(ctx, A, tol=1e-10, prec="fp64", max_blobs=cap, max_bodies=64,
                    max_requests=8)
    tickets, outs = [], []
    for s in susp:
        t, o = srv.submit(_prob(s))
        tickets.append(t); outs.append(o)
    most = 0
    for _ in range(10000):
        nr, nq = srv.step()
        most = max(most, nr)
        if nr == 0 and nq == 0:
            break
    assert most == 1
    for s, t, (U, W, lam) in zip(susp, tickets, outs):
        assert srv.poll(t)[0] == mb.Server.DONE
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, A, 1.0, True)
        assert rel_l2(host(U), Ur) <= 1e-6
    big = I.mixed_suspension(9, 40)
    with pytest.raises(mb.MBError) as ei:
        srv.submit(_prob(big))
    assert ei.value.name == "MB_ENOMEM"
    srv.close()


def test_server_isolates_a_failing_request(ctx):
    good = [I.mixed_suspension(500 + k, 4) for k in range(2)]
    s = I.mixed_suspension(510, 4)
    q = s.q.copy()
    r = O.blob_positions(q, s.theta, s.blob_start, s.rho)
    q[0, 2] -= r[s.blob_start[0]:s.blob_start[1], 2].min() - 0.5 * A
    badP = _prob(s)
    badP["q"] = dev(q)
    srv = mb.Server(ctx, A, tol=1e-10, prec="mixed", max_blobs=5000, max_bodies=100,
                    max_requests=8)
    t0, o0 = srv.submit(_prob(good[0]))
    tb, _ = srv.submit(badP)
    t1, o1 = srv.submit(_prob(good[1]))
    srv.run_until_idle()
    assert srv.poll(tb)[0] == mb.Server.FAILED and srv.poll(tb)[2] == "MB_ESINGULAR"
    for g, t, (U, W, lam) in ((good[0], t0, o0), (good[1], t1, o1)):
        assert srv.poll(t)[0] == mb.Server.DONE
        rg = O.blob_positions(g.q, g.theta, g.blob_start, g.rho)
        Ur, Wr, _ = O.solve_saddle(rg, g.q, g.blob_start, g.F, g.T, A, 1.0, True)
        assert rel_l2(host(U), Ur) <= 1e-6 and rel_l2(host(W), Wr) <= 1e-6
    srv.close()


def test_server_split_matvec_matches_unsplit(ctx):
    """A small tick pair budget spreads each large FP32 Arnoldi matvec over
    several ticks; the solutions match the unsplit engine and the oracle."""
    sus = [I.mixed_suspension(500, 60), I.mixed_suspension(501, 2)]
    probs = [_prob(s) for s in sus]
    ctx.set_pair_variant(3)  # the symmetric tile shape, the one that splits
    try:
        res, ticks = {}, {}
        for budget in (-1.0, 1e5):
            srv = mb.Server(ctx, A, tol=1e-10, prec="mixed", max_blobs=20000, max_bodies=500,
                            max_requests=8, tick_pairs=budget)
            outs = [srv.submit(P) for P in probs]
            n = 0
            while True:
                nr, nq = srv.step()
                n += 1
                if nr == 0 and nq == 0:
                    break
                assert n < 100000
            ticks[budget] = n
            res[budget] = []
            for t, (U, W, lam) in outs:
                state, info, status = srv.poll(t)
                assert state == mb.Server.DONE and status == "MB_OK", (state, status, info)
                assert info["converged"] == 1 and info["rel_residual"] <= 1e-10
                res[budget].append((host(U), host(W)))
            srv.close()
    finally:
        ctx.set_pair_variant(-1)
    # the large request (1,845 blobs) takes 17 ticks per Arnoldi matvec
    assert ticks[1e5] > 3 * ticks[-1.0], ticks
    for (Ua, Wa), (Ub, Wb), s in zip(res[-1.0], res[1e5], sus):
        assert rel_l2(Ub, Ua) <= 1e-8 and rel_l2(Wb, Wa) <= 1e-8
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, A, 1.0, True)
        assert rel_l2(Ub, Ur) <= 1e-6 and rel_l2(Wb, Wr) <= 1e-6


def _head_of_line_setup():
    """A medium request A, then a large request B that cannot fit beside A,
    then small requests C, D, E that can."""
    sa, sb = I.mixed_suspension(600, 10), I.mixed_suspension(601, 30)
    small = [I.mixed_suspension(602 + k, 2) for k in range(3)]
    cap = max(sb.n_blobs, sa.n_blobs + sum(s.n_blobs for s in small)) + 5
    assert sa.n_blobs + sb.n_blobs > cap
    return sa, sb, small, cap


def _check_vs_oracle(srv, jobs):
    for s, t, (U, W, lam) in jobs:
        state, info, status = srv.poll(t)
        assert state == mb.Server.DONE and status == "MB_OK", (state, status, info)
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, A, 1.0, True)
        assert rel_l2(host(U), Ur) <= 1e-6 and rel_l2(host(W), Wr) <= 1e-6


@pytest.mark.parametrize("max_bypass", [0, -1])
def test_server_small_request_overtakes_a_waiting_large_one(ctx, max_bypass):
    """Admission scans the queue in arrival order: a small request queued
    behind a large one that does not fit yet is admitted first (max_bypass =
    0, the default limit); with max_bypass < 0 admission is strictly first
    come, first served and it waits.  Every result matches the oracle."""
    sa, sb, small, cap = _head_of_line_setup()
    srv = mb.Server(ctx, A, tol=1e-10, prec="mixed", max_blobs=cap, max_bodies=500,
                    max_requests=8, max_bypass=max_bypass)
    tA, oA = srv.submit(_prob(sa))
    srv.step()
    tB, oB = srv.submit(_prob(sb))
    tC, oC = srv.submit(_prob(small[0]))
    srv.step()
    assert srv.poll(tA)[0] == mb.Server.RUNNING
    assert srv.poll(tB)[0] == mb.Server.QUEUED
    assert srv.poll(tC)[0] == (mb.Server.RUNNING if max_bypass == 0 else mb.Server.QUEUED)
    srv.run_until_idle()
    assert sorted(srv.finished()) == sorted([tA, tB, tC])
    assert srv.finished() == []
    _check_vs_oracle(srv, [(sa, tA, oA), (sb, tB, oB), (small[0], tC, oC)])
    srv.close()


def test_server_aging_bounds_the_overtaking(ctx):
    """With max_bypass = 1, once later requests have overtaken the waiting
    large request, the next arrival queues behind it until it is admitted."""
    sa, sb, small, cap = _head_of_line_setup()
    srv = mb.Server(ctx, A, tol=1e-10, prec="mixed", max_blobs=cap, max_bodies=500,
                    max_requests=8, max_bypass=1)
    tA, oA = srv.submit(_prob(sa))
    srv.step()
    tB, oB = srv.submit(_prob(sb))
    tC, oC = srv.submit(_prob(small[0]))
    tD, oD = srv.submit(_prob(small[1]))
    srv.step()
    assert srv.poll(tB)[0] == mb.Server.QUEUED
    assert srv.poll(tC)[0] == mb.Server.RUNNING and srv.poll(tD)[0] == mb.Server.RUNNING
    tE, oE = srv.submit(_prob(small[2]))
    srv.step()
    # B has been overtaken twice: E, which would fit, waits behind it
    assert srv.poll(tB)[0] == mb.Server.QUEUED and srv.poll(tE)[0] == mb.Server.QUEUED
    order = []
    for _ in range(100000):
        nr, nq = srv.step()
        for t in (tB, tE):
            if t not in order and srv.poll(t)[0] != mb.Server.QUEUED:
                order.append(t)
        if nr == 0 and nq == 0:
            break
    assert order[0] == tB  # B is admitted before (or with) E
    _check_vs_oracle(srv, [(sa, tA, oA), (sb, tB, oB), (small[0], tC, oC),
                           (small[1], tD, oD), (small[2], tE, oE)])
    srv.close()
