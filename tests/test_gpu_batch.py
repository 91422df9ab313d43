"""The batched form (tc_batch) against the oracle and against one call per graph."""
from __future__ import annotations

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


def mixed_graphs():
    gs = [
        (2000, synth.er(2000, 12000, 1)),
        (3000, synth.ba(3000, 12, 2)),
        (1 << 10, synth.rmat(10, 16, 3)),
        (5, np.zeros((0, 2), np.int32)),          # no edges
        (0, np.zeros((0, 2), np.int32)),          # no vertices
        (40, synth.complete(40)),
        (700, synth.complete(700)),               # lists longer than a tile
        (4, synth.wheel(3)),
        (1, np.zeros((0, 2), np.int32)),
    ]
    ns, ds = synth.batch_params(24, 77, nlo=100, nhi=5000)
    gs += [(int(n), synth.chung_lu(int(n), float(d), 2.1, 77, g)) for g, (n, d) in enumerate(zip(ns, ds))]
    return gs


def test_batch_matches_oracle_and_per_graph_calls(tc):
    graphs = mixed_graphs()
    b = tc.make_batch([(n, synth.shuffle_edges(e, i)) for i, (n, e) in enumerate(graphs)], "cuda")
    totals, tv, union = tc.batch(b)
    totals = totals.cpu().numpy()
    tv = tv.cpu().numpy()
    vbase = b.vbase.cpu().numpy()
    off = union.offsets.cpu().numpy()
    cols = union.cols.cpu().numpy()
    for g, (n, e) in enumerate(graphs):
        ref = oracle.count(n, e, local=True) if n > 0 else {"T": 0, "tv": np.zeros(0, np.int64)}
        assert totals[g] == ref["T"], g
        assert np.array_equal(tv[vbase[g]:vbase[g + 1]], ref["tv"]), g
        if n == 0:
            continue
        single = tc.orient(torch.from_numpy(np.ascontiguousarray(e)).cuda(), n)
        T1, tv1, _ = tc.count_local(single)
        assert T1 == ref["T"]
        # the union's lists of graph g are graph g's own lists, shifted by vbase[g]
        so = single.offsets.cpu().numpy()
        sc = single.cols.cpu().numpy()
        uo = off[vbase[g]:vbase[g + 1] + 1]
        assert np.array_equal(uo - uo[0], so)
        assert np.array_equal(cols[uo[0]:uo[-1]] - vbase[g], sc)


def test_batch_of_the_batched_configuration_shape(tc):
    # a slice of the 4096-graph Chung-Lu configuration (smaller n range)
    graphs = synth.batch_graphs(64, 2024, nhi=20000)
    b = tc.make_batch(graphs, "cuda")
    totals, tv, _ = tc.batch(b, local=False)
    assert tv is None
    totals = totals.cpu().numpy()
    for g in range(0, 64, 7):
        n, e = graphs[g]
        assert totals[g] == oracle.count(n, e)["T"]


def test_batch_rejects_bad_local_ids(tc):
    graphs = [(10, np.array([[0, 1], [1, 2]], np.int32)), (3, np.array([[0, 3]], np.int32))]
    b = tc.make_batch(graphs, "cuda")
    with pytest.raises(tc.TcError) as ex:
        tc.batch(b)
    assert ex.value.status == 2
