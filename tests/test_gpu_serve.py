"""Serving loop (continuous batching): every request's result is the same
alone and in a concurrent mix (bit for bit), small Block GEMMs of one
precision and bucket are batched, the memory budget holds, and malformed,
oversized and cancelled requests are reported."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal

pytestmark = pytest.mark.gpu

PRECS = [128, 256, 512, 1024, 2048]


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        p = int(rng.choice(PRECS))
        if rng.random() < 0.7:
            m, l, n = (int(x) for x in rng.integers(16, 160, 3))
            algo = mp.WINOGRAD if min(m, l, n) > 100 else mp.BLOCK
            A = gen.uniform_pm1(m, l, p, 1000 + i, -16, 16)
            B = gen.uniform_pm1(l, n, p, 2000 + i, -16, 16)
            reqs.append(("gemm", i, A, B, algo))
        else:
            n = int(rng.integers(16, 90))
            A = gen.well_conditioned(n, p, 3000 + i)
            b = gen.uniform_pm1(n, 1, p, 4000 + i)
            reqs.append(("lu", i, A, b, mp.WINOGRAD if n > 64 else mp.SIMPLE))
    return reqs


def _submit(srv, r):
    kind, rid, A, B, algo = r
    if kind == "gemm":
        return srv.submit_gemm(rid, A, B, algo=algo, cutoff=32)
    return srv.submit_lu(rid, A, B, algo=algo, cutoff=16, panel=32)


def test_alone_equals_mixed():
    reqs = _requests(40, 5)
    # alone: one slot, one request at a time
    alone = {}
    srv = mp.Server(budget_bytes=8 << 30, slots=1)
    for r in reqs:
        assert _submit(srv, r) == 0
        srv.drain()
        st, ms, out = srv.results[r[1]]
        assert st == mp.REQ_DONE
        alone[r[1]] = out
    srv.close()
    # mixed: everything at once, eight slots
    srv = mp.Server(budget_bytes=8 << 30, slots=8)
    for r in reqs:
        assert _submit(srv, r) == 0
    srv.drain()
    stats = srv.stats()
    assert stats["completed"] == len(reqs)
    for r in reqs:
        st, ms, out = srv.results[r[1]]
        assert st == mp.REQ_DONE
        assert_bits_equal(out, alone[r[1]], "request %d" % r[1])
    srv.close()
    # and the results are the algorithms' own (oracle) results
    for r in reqs[:6]:
        kind, rid, A, B, algo = r
        if kind == "gemm":
            want = orc.gemm(algo, A, B, cutoff=32)
        else:
            F, piv, rc = orc.lu(A, panel=32, algo=algo, cutoff=16)
            want = orc.lu_solve(F, piv, B)
        assert_bits_equal(alone[rid], want, "oracle %d" % rid)


def test_budget_is_respected_and_oversized_rejected():
    p = 512
    A = gen.uniform_pm1(200, 200, p, 1)
    B = gen.uniform_pm1(200, 200, p, 2)
    per = mp.Server(budget_bytes=1 << 40, slots=1)
    per.close()
    budget = 3 * 200 * 200 * 73 * 2          # about two requests' operands
    srv = mp.Server(budget_bytes=budget, slots=8)
    for i in range(6):
        assert srv.submit_gemm(i, A, B, algo=mp.SIMPLE) == 0
    big = gen.uniform_pm1(600, 600, p, 3)
    assert srv.submit_gemm(99, big, big, algo=mp.SIMPLE) == -2     # never fits
    srv.drain()
    st = srv.stats()
    assert st["completed"] == 6 and st["peak_bytes"] <= budget
    outs = [srv.results[i][2] for i in range(6)]
    for o in outs[1:]:
        assert_bits_equal(o, outs[0], "same request")
    srv.close()


def test_malformed_and_cancelled():
    srv = mp.Server(budget_bytes=1 << 30, slots=1)
    A = gen.uniform_pm1(4, 4, 128, 1)
    bad = mp.HostMP(A.limb, A.exp, A.sign, 9000)          # precision out of range (> 8704)
    assert srv.submit_gemm(1, bad, bad) == -1
    # a long head request keeps the single slot busy; cancel a queued one
    H = gen.uniform_pm1(300, 300, 1024, 2)
    assert srv.submit_gemm(10, H, H, algo=mp.SIMPLE) == 0
    for i in range(11, 15):
        assert srv.submit_gemm(i, A, A, algo=mp.WINOGRAD, cutoff=2) == 0
    assert srv.cancel(13) == 0
    assert srv.cancel(13) == -1
    srv.drain()
    assert srv.results[13][0] == mp.REQ_CANCELLED
    assert all(srv.results[i][0] == mp.REQ_DONE for i in (10, 11, 12, 14))
    srv.close()


def test_queued_small_gemms_are_batched():
    """Small Block GEMMs of one precision and bucket that wait behind a long
    request run as one grouped launch, with the results they have alone."""
    p = 512
    big_A = gen.well_conditioned(400, 1024, 77)
    big_b = gen.uniform_pm1(400, 1, 1024, 78)
    small = [(gen.uniform_pm1(40 + i, 30, p, 6100 + i, -16, 16), gen.uniform_pm1(30, 50, p, 6200 + i, -16, 16))
             for i in range(6)]
    srv = mp.Server(budget_bytes=8 << 30, slots=1)
    srv.set_graphs(0)
    assert srv.submit_lu(100, big_A, big_b, algo=mp.SIMPLE, cutoff=64, panel=128) == 0   # holds the slot
    for i, (A, B) in enumerate(small):
        assert srv.submit_gemm(i, A, B, algo=mp.BLOCK) == 0
    srv.drain()
    stats = srv.stats()
    assert stats["completed"] == 7
    assert stats["batches"] >= 1 and stats["batched_requests"] >= 2
    for i, (A, B) in enumerate(small):
        st, ms, out = srv.results[i]
        assert st == mp.REQ_DONE
        assert_bits_equal(out, orc.gemm(orc.BLOCK, A, B), "batched request %d" % i)
    srv.close()


@pytest.mark.parametrize("kind", ["gemm", "lu"])
def test_graph_cache_replays_bit_exact(kind):
    """Repeated request shapes run from captured CUDA graphs; every result
    equals the uncached path's (graph cache off) bit for bit."""
    p = 256
    reqs = []
    for i in range(5):
        if kind == "gemm":
            A = gen.uniform_pm1(70, 90, p, 5100 + i, -16, 16)
            B = gen.uniform_pm1(90, 66, p, 5200 + i, -16, 16)
            reqs.append(("gemm", i, A, B, mp.WINOGRAD))
        else:
            A = gen.well_conditioned(48, p, 5300 + i)
            b = gen.uniform_pm1(48, 1, p, 5400 + i)
            reqs.append(("lu", i, A, b, mp.SIMPLE))
    outs = {}
    for graphs in (0, 8):
        srv = mp.Server(budget_bytes=8 << 30, slots=2)
        srv.set_graphs(graphs)
        for r in reqs:                     # one at a time: the cached entry is free again
            assert _submit(srv, r) == 0
            srv.drain()
        gs = srv.graph_stats()
        for r in reqs:
            st, ms, out = srv.results[r[1]]
            assert st == mp.REQ_DONE
            outs.setdefault(r[1], []).append(out)
        srv.close()
        if graphs == 0:
            assert gs["captured"] == 0 and gs["replays"] == 0
        else:
            # first sighting runs directly, the second is captured, all later ones replay
            assert gs["captured"] == 1 and gs["replays"] == len(reqs) - 1
    for rid, (plain, cached) in outs.items():
        assert_bits_equal(cached, plain, "request %d from the graph cache" % rid)


def test_same_precision_gemms_share_leaf_launches():
    """GEMMs of one precision and size class that wait behind a long request
    run as one leaf group: each request's own operand sums and combinations,
    the leaves of all of them in shared grouped launches.  Strassen,
    Winograd (odd sizes: peeled borders and rank-1 fix-ups), Block and Simple
    requests together; every result equals the oracle running the request's
    own algorithm, bit for bit, and a request of another precision waiting
    beside them is not grouped with them."""
    p = 512
    big_A = gen.well_conditioned(400, 1024, 79)
    big_b = gen.uniform_pm1(400, 1, 1024, 80)
    shapes = [(150, 131, 97, mp.WINOGRAD, 32), (140, 200, 120, mp.STRASSEN, 48), (130, 66, 140, mp.WINOGRAD, 64),
              (96, 100, 90, mp.BLOCK, 64), (77, 180, 101, mp.SIMPLE, 64), (200, 160, 170, mp.WINOGRAD, 40)]
    reqs = [(gen.uniform_pm1(m, l, p, 6300 + i, -16, 16), gen.uniform_pm1(l, n, p, 6400 + i, -16, 16), algo, cut)
            for i, (m, l, n, algo, cut) in enumerate(shapes)]
    other = (gen.uniform_pm1(90, 80, 256, 6500, -16, 16), gen.uniform_pm1(80, 70, 256, 6501, -16, 16))
    srv = mp.Server(budget_bytes=8 << 30, slots=1)
    assert srv.submit_lu(100, big_A, big_b, algo=mp.SIMPLE, cutoff=64, panel=128) == 0   # holds the slot
    for i, (A, B, algo, cut) in enumerate(reqs):
        assert srv.submit_gemm(i, A, B, algo=algo, cutoff=cut) == 0
    assert srv.submit_gemm(50, *other, algo=mp.WINOGRAD, cutoff=32) == 0
    srv.drain()
    stats = srv.stats()
    assert stats["completed"] == len(reqs) + 2
    assert stats["batches"] >= 1 and stats["batched_requests"] >= len(reqs)
    for i, (A, B, algo, cut) in enumerate(reqs):
        st, ms, out = srv.results[i]
        assert st == mp.REQ_DONE
        assert_bits_equal(out, orc.gemm(algo, A, B, cutoff=cut), "grouped request %d" % i)
    st, ms, out = srv.results[50]
    assert st == mp.REQ_DONE
    assert_bits_equal(out, orc.gemm(orc.WINOGRAD, *other, cutoff=32), "other precision")
    srv.close()


def test_leaf_group_with_empty_products():
    """A leaf group that holds degenerate products (m = 0, n = 0, l = 0) beside
    recursive ones: the empty ones return empty or +0 results, the others
    equal the oracle, bit for bit."""
    p = 256
    big_A = gen.well_conditioned(300, 1024, 81)
    big_b = gen.uniform_pm1(300, 1, 1024, 82)
    shapes = [(120, 130, 110, mp.WINOGRAD), (0, 90, 100, mp.WINOGRAD), (100, 0, 90, mp.STRASSEN),
              (80, 100, 0, mp.WINOGRAD), (140, 100, 150, mp.STRASSEN)]
    reqs = [(gen.uniform_pm1(m, l, p, 6600 + i, -16, 16), gen.uniform_pm1(l, n, p, 6700 + i, -16, 16), algo)
            for i, (m, l, n, algo) in enumerate(shapes)]
    srv = mp.Server(budget_bytes=8 << 30, slots=1)
    assert srv.submit_lu(100, big_A, big_b, algo=mp.SIMPLE, cutoff=64, panel=128) == 0   # holds the slot
    for i, (A, B, algo) in enumerate(reqs):
        assert srv.submit_gemm(i, A, B, algo=algo, cutoff=32) == 0
    srv.drain()
    stats = srv.stats()
    assert stats["completed"] == len(reqs) + 1 and stats["batches"] >= 1
    for i, (A, B, algo) in enumerate(reqs):
        st, ms, out = srv.results[i]
        assert st == mp.REQ_DONE
        m, n = A.shape[0], B.shape[1]
        assert out.exp.shape == (m, n)
        if A.shape[1] == 0:
            assert np.all(out.exp == gen.EXP_ZERO) and not out.limb.any() and not out.sign.any()
        elif m and n:
            assert_bits_equal(out, orc.gemm(algo, A, B, cutoff=32), "grouped request %d" % i)
    srv.close()
