"""The hub side of the intersection: an edge (v, u) with a long N_u (at least
hub_min ids, longer than N_v) is counted from u's side.  Which side counts an
edge is a cost split only: every output -- T, T_v, C_v and the triangle list,
element by element and in order -- must be identical with the hub side off,
at any threshold, and equal to the oracle or to a closed form."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.brute import clique_with_pendants

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1706_05151_gb300 import build
    build.build()
    import paper_1706_05151_gb300 as lib
    return lib


def to_dev(e: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(e, dtype=np.int32)).cuda()


def run_all(tc, g, ctx, hub_min, tile_max):
    ctx.set_hub_min(hub_min)
    ctx.set_tuning(tile_max, 1)
    try:
        T = tc.count(g, ctx)
        Tl, tv, cc = tc.count_local(g, ctx=ctx)
        tri = tc.list_triangles(g, ctx)
        Ta, tva, cca, tria = tc.analyze(g, ctx=ctx)
    finally:
        ctx.set_hub_min(0)
        ctx.set_tuning(0, 1)
    assert T == Tl == Ta == tri.shape[0] == tria.shape[0]
    assert torch.equal(tv, tva) and torch.equal(cc, cca) and torch.equal(tri, tria)
    return T, tv.clone(), cc.clone(), tri.clone()


SKEWED = {
    "rmat16": lambda: (1 << 16, synth.rmat(16, 16, 11)),
    "chung_lu": lambda: (100000, synth.chung_lu(100000, 32.0, 2.1, 5)),
    "er": lambda: (20000, synth.er(20000, 200000, 3)),
}


@pytest.mark.parametrize("name", sorted(SKEWED))
def test_hub_side_changes_no_output(tc, name):
    n, e = SKEWED[name]()
    ctx = tc.Context(0)
    g = tc.orient(to_dev(synth.shuffle_edges(e, 1)), n, ctx)
    ref = oracle.count(n, e, local=True)
    base = run_all(tc, g, ctx, -1, 0)  # hub side off
    assert base[0] == ref["T"]
    assert np.array_equal(base[1].cpu().numpy(), ref["tv"])
    for hub_min, tile_max in ((0, 0), (32, 0), (200, 0), (0, 32), (1, 64)):
        got = run_all(tc, g, ctx, hub_min, tile_max)
        assert got[0] == base[0], (hub_min, tile_max)
        assert torch.equal(got[1], base[1]), (hub_min, tile_max)
        assert torch.equal(got[2], base[2]), (hub_min, tile_max)
        assert torch.equal(got[3], base[3]), (hub_min, tile_max)
    ctx.close()


def test_hub_chunked_and_segmented_counts(tc):
    # hub 0: 2199 ids (hashed in 2 chunks for T, 3 for T_v) and 1100 in-edges
    # from pendants (two work items of the hub kernel)
    n, e, T, tv = clique_with_pendants(2200, 1100)
    ctx = tc.Context(0)
    g = tc.orient(to_dev(synth.shuffle_edges(e, 2)), n, ctx)
    assert int(g.dhat[0].item()) == 2199
    for hub_min in (-1, 0, 16):
        ctx.set_hub_min(hub_min)
        assert tc.count(g, ctx) == T
        Tl, tvg, cc = tc.count_local(g, ctx=ctx)
        assert Tl == T
        assert np.array_equal(tvg.cpu().numpy(), tv)
    ctx.close()


def test_hub_chunked_listing_matches_hub_off(tc):
    # 2099 ids at hub 0: listing hashes it in two chunks; 1100 pendant edges at it
    n, e, T, tv = clique_with_pendants(2100, 1100)
    ctx = tc.Context(0)
    g = tc.orient(to_dev(synth.shuffle_edges(e, 3)), n, ctx)
    ctx.set_hub_min(-1)
    off = tc.list_triangles(g, ctx)
    assert off.shape[0] == T
    ctx.set_hub_min(0)
    on = tc.list_triangles(g, ctx)
    assert torch.equal(on, off)
    del on, off
    torch.cuda.empty_cache()
    ctx.close()
