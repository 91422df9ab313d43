"""The serving form: each result is the same alone and in a concurrent mix, and
admission by memory footprint behaves as documented."""
from __future__ import annotations

import random
import threading

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1706_05151_gb300 import build
    build.build()
    import paper_1706_05151_gb300 as lib
    return lib


def graph_pool():
    return [
        (1 << 12, synth.er(1 << 12, 8 << 12, 1)),
        (1 << 12, synth.rmat(12, 16, 2)),
        (5000, synth.chung_lu(5000, 16.0, 2.1, 3, 0)),
        (1 << 13, synth.ba(1 << 13, 16, 4)),
        (700, synth.complete(700)),
    ]


def key_of(res):
    tri = None
    if res.tri is not None:
        t = res.tri.cpu().numpy()
        tri = t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))] if len(t) else t
    return (res.status, res.triangles,
            None if res.tv is None else res.tv.cpu().numpy().tobytes(),
            None if res.cc is None else res.cc.cpu().numpy().tobytes(),
            None if tri is None else tri.tobytes())


@pytest.mark.parametrize("small_edges", [0, 1, 40000])
def test_results_same_alone_and_in_the_mix(tc, small_edges):
    # small_edges 1: every request is large (low-priority slots, tile blocks with a
    # chunk quota); 40000: a mix of both classes; 0: the default threshold
    srv = tc.Server(2 << 30, slots=6, small_edges=small_edges)
    graphs = graph_pool()
    ids = [srv.add_graph(n, e) for n, e in graphs]
    refs = {gid: oracle.count(n, e)["T"] for gid, (n, e) in zip(ids, graphs)}
    reqs = [(gid, kind) for gid in ids for kind in (tc.COUNT, tc.LOCAL, tc.LIST)]
    alone = {}
    for gid, kind in reqs:
        r = srv.wait(srv.submit(gid, kind))
        assert r.status == 0 and r.triangles == refs[gid]
        alone[(gid, kind)] = key_of(r)
    mix = reqs * 4
    random.Random(7).shuffle(mix)
    tickets = []

    def submitter():
        for gid, kind in mix:
            tickets.append((srv.submit(gid, kind), gid, kind))
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    for t, gid, kind in tickets:
        r = srv.wait(t)
        assert key_of(r) == alone[(gid, kind)], (gid, kind)
    st = srv.stats()
    assert st["completed"] == len(reqs) + len(mix) and st["rejected"] == 0
    srv.close()


def test_requests_wait_for_memory_and_complete(tc):
    n, e = 1 << 14, synth.rmat(14, 16, 9)
    srv = tc.Server(4 << 20, slots=4, admit_timeout_ms=20000)
    gid = srv.add_graph(n, e)
    ref = oracle.count(n, e, local=True)
    # each LOCAL result holds 16n bytes; the pool fits only a few at a time
    tickets = [srv.submit(gid, tc.LOCAL) for _ in range(12)]
    for t in tickets:
        r = srv.wait(t)
        assert r.status == 0 and r.triangles == ref["T"]
        assert np.array_equal(r.tv.cpu().numpy(), ref["tv"])
    srv.close()


def test_graph_too_big_for_the_pool_is_rejected(tc):
    srv = tc.Server(1 << 20, slots=2)
    with pytest.raises(tc.TcError) as ex:
        srv.add_graph(1 << 16, synth.ba(1 << 16, 16, 5))
    assert ex.value.status == 8
    srv.close()


def test_listing_larger_than_the_pool_is_rejected(tc):
    # K_200 fits, its 1.3M triples (16 MB) never can
    srv = tc.Server(4 << 20, slots=2)
    gid = srv.add_graph(200, synth.complete(200))
    r = srv.wait(srv.submit(gid, tc.LIST))
    assert r.status == 8
    r = srv.wait(srv.submit(gid, tc.COUNT))
    assert r.status == 0 and r.triangles == 200 * 199 * 198 // 6
    srv.close()


def test_invalid_requests(tc):
    srv = tc.Server(1 << 24, slots=2)
    with pytest.raises(tc.TcError) as ex:
        srv.add_graph(3, np.array([[0, 1], [1, 1]], np.int32))
    assert ex.value.status == 2
    with pytest.raises(tc.TcError) as ex:
        srv.submit(12345, tc.COUNT)
    assert ex.value.status == 1
    gid = srv.add_graph(4, synth.complete(4))
    r = srv.wait(srv.submit(gid, tc.COUNT))
    assert r.triangles == 4
    srv.remove_graph(gid)
    with pytest.raises(tc.TcError):
        srv.submit(gid, tc.COUNT)
    srv.close()


def test_small_requests_unchanged_behind_a_large_one(tc):
    # an R-MAT scale 22 listing (2.1e9 triples, 25 GB) is running when small requests arrive:
    # they are admitted beside it, finish first, and return what they return alone
    big_n, big_e = 1 << 22, synth.rmat(22, 16, 21)
    srv = tc.Server(48 << 30, slots=6, admit_timeout_ms=120000)
    big = srv.add_graph(big_n, big_e)
    smalls = [(1 << 12, synth.er(1 << 12, 8 << 12, 22)), (5000, synth.chung_lu(5000, 16.0, 2.1, 23, 0)),
              (1 << 12, synth.rmat(12, 16, 24))]
    sids = [srv.add_graph(n, e) for n, e in smalls]
    alone = {}
    for gid, (n, e) in zip(sids, smalls):
        ref = oracle.count(n, e, local=True, listing=True)
        for kind in (tc.COUNT, tc.LOCAL, tc.LIST):
            r = srv.wait(srv.submit(gid, kind))
            assert r.status == 0 and r.triangles == ref["T"]
            alone[(gid, kind)] = key_of(r)
    big_ref = srv.wait(srv.submit(big, tc.COUNT), timeout_ms=120000).triangles
    big_t = srv.submit(big, tc.LIST)
    small_t = [(srv.submit(gid, kind), gid, kind) for gid in sids for kind in (tc.COUNT, tc.LOCAL, tc.LIST)]
    small_res = [(srv.wait(t, timeout_ms=120000), gid, kind) for t, gid, kind in small_t]
    b = srv.wait(big_t, timeout_ms=300000, copy=False)
    assert b.status == 0 and b.triangles == big_ref > 10 ** 9
    for r, gid, kind in small_res:
        assert key_of(r) == alone[(gid, kind)], (gid, kind)
        assert r.latency_ms < b.latency_ms  # not held behind the large request
    srv.close()
