"""The host planner of the step kernel's equal shares (md_plan_shares, host
only, no GPU): for clusters of many sizes, i-block widths, tile sizes and share
counts, the pieces of every i-block cover its cluster's sources once, in source
order and on tile boundaries; every i-block of every cluster is present, in
cluster and i-block order; the shares are contiguous runs of units whose tile
counts differ by at most one; and bad arguments are rejected."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def md():
    from paper_1307_3711_gb300 import build
    build.build()
    from paper_1307_3711_gb300 import md as m
    return m


CASES = [
    # (n_pad per cluster, per, tile, shares)
    ([200000], 1024, 256, 1824),      # the headline: 4 shares per resident CTA
    ([200000], 1024, 512, 1216),
    ([50000], 1024, 256, 1824),       # several pieces per i-block
    ([16], 128, 512, 456),            # one tile in all: one share
    ([1024, 16, 3008, 512], 512, 256, 7),
    ([1000000], 512, 256, 9728),
    ([4096] * 5 + [16] * 3, 128, 512, 100000),   # more shares than tiles
    ([13712, 2048, 29760, 176], 1024, 512, 1),  # one share: every unit in it
]


def _tiles(jn, tile):
    return (jn + tile - 1) // tile


@pytest.mark.parametrize("n_pad,per,tile,shares", CASES)
def test_pieces_cover_every_iblock_once_in_order(md, n_pad, per, tile, shares):
    units, first = md.plan_shares(n_pad, per, tile, shares)
    tiles = [-(-n // tile) for n in n_pad]
    T = sum(-(-n // per) * t for n, t in zip(n_pad, tiles))
    S = min(shares, T)
    assert len(first) == S + 1 and first[0] == 0 and first[-1] == len(units)
    assert np.all(np.diff(first) >= 1)          # no empty share
    # i-blocks in cluster and i-block order, each with its pieces 0..np-1
    expect = [(c, b) for c, n in enumerate(n_pad) for b in range(-(-n // per))]
    k = 0
    for c, b in expect:
        np_ = units[k, 3]
        assert np_ >= 1
        pieces = units[k:k + np_]
        assert np.all(pieces[:, 0] == c) and np.all(pieces[:, 1] == b)
        assert pieces[:, 2].tolist() == list(range(np_))
        assert np.all(pieces[:, 3] == np_)
        # the pieces tile [0, n_pad) in source order, on tile boundaries
        j0, jn = pieces[:, 4], pieces[:, 5]
        assert j0[0] == 0 and np.all(j0 % tile == 0) and np.all(jn > 0)
        assert np.all(j0[1:] == j0[:-1] + jn[:-1])
        assert j0[-1] + jn[-1] == n_pad[c]
        assert np.all(jn[:-1] % tile == 0)
        k += np_
    assert k == len(units)
    # shares: tile counts within one of each other, and their sum is T
    per_share = [int(sum(_tiles(u[5], tile) for u in units[first[s]:first[s + 1]]))
                 for s in range(S)]
    assert sum(per_share) == T
    assert max(per_share) - min(per_share) <= 1
    assert min(per_share) == T // S


def _plan_by_definition(n_pad, per, tile, shares):
    """The partition as md.h states it, written out: the tiles of every
    i-block end to end (cluster, then i-block order), share s = tiles
    [s T / S, (s + 1) T / S) (integer division), pieces = the non-empty
    intersections of shares and i-blocks in order."""
    blocks = []
    for c, n in enumerate(n_pad):
        tiles = -(-n // tile)
        blocks += [(c, b, tiles, n) for b in range(-(-n // per))]
    T = sum(b[2] for b in blocks)
    S = min(shares, T)
    bounds = [k * T // S for k in range(S + 1)]
    units, share_of, F = [], [], 0
    for c, b, tiles, n in blocks:
        pcs = []
        for s_ in range(S):
            lo, hi = max(F, bounds[s_]), min(F + tiles, bounds[s_ + 1])
            if lo < hi:
                j0 = (lo - F) * tile
                pcs.append([c, b, len(pcs), 0, j0, min((hi - F) * tile, n) - j0])
                share_of.append(s_)
        for p_ in pcs:
            p_[3] = len(pcs)
        units += pcs
        F += tiles
    first = [0] * (S + 1)
    for s_ in share_of:
        first[s_ + 1] += 1
    for k in range(1, S + 1):
        first[k] += first[k - 1]
    return units, first


@pytest.mark.parametrize("n_pad,per,tile,shares", CASES[:5] + CASES[6:])
def test_plan_equals_the_stated_definition(md, n_pad, per, tile, shares):
    units, first = md.plan_shares(n_pad, per, tile, shares)
    ref_units, ref_first = _plan_by_definition(n_pad, per, tile, shares)
    assert units.tolist() == ref_units
    assert first.tolist() == ref_first


def test_small_plan_by_hand(md):
    """2 clusters of 2048 records, i-blocks of 1024 targets, 512-record tiles:
    4 i-blocks of 4 tiles (T = 16) in 3 shares of tiles [0,5) [5,10) [10,16).
    A share boundary inside an i-block splits it into pieces."""
    units, first = md.plan_shares([2048, 2048], 1024, 512, 3)
    assert first.tolist() == [0, 2, 4, 6]
    assert units.tolist() == [
        [0, 0, 0, 1, 0, 2048],                          # share 0: tiles 0-3
        [0, 1, 0, 2, 0, 512],                           # share 0: tile 4
        [0, 1, 1, 2, 512, 1536],                        # share 1: tiles 5-7
        [1, 0, 0, 2, 0, 1024],                          # share 1: tiles 8-9
        [1, 0, 1, 2, 1024, 1024],                       # share 2: tiles 10-11
        [1, 1, 0, 1, 0, 2048],                          # share 2: tiles 12-15
    ]


@pytest.mark.parametrize("args", [
    ([0], 1024, 256, 8),        # an empty cluster
    ([100], 0, 256, 8),         # per < 1
    ([100], 128, 0, 8),         # tile < 1
    ([100], 128, 256, 0),       # shares < 1
    ([100], 128, 256, 1 << 31),  # shares beyond int32
    ([1 << 30, 1 << 30], 128, 256, 10),  # 2^31 or more source tiles in all
])
def test_bad_arguments(md, args):
    with pytest.raises(md.MDError) as ei:
        md.plan_shares(*args)
    assert ei.value.status == md.MD_ERR_ARG


def test_cap_below_the_unit_count(md):
    import ctypes as C
    n_pad = np.array([200000], np.int32)
    ip = C.POINTER(C.c_int32)
    units = np.zeros((10, 6), np.int32)
    first = np.zeros(1825, np.int32)
    nu, ns = C.c_int64(0), C.c_int64(0)
    st = md._lib.md_plan_shares(n_pad.ctypes.data_as(ip), 1, 1024, 256, 1824,
                                units.ctypes.data_as(ip), 10, first.ctypes.data_as(ip),
                                C.byref(nu), C.byref(ns))
    assert st == md.MD_ERR_ARG and nu.value == 2016 and ns.value == 1824
    assert not units.any()
    # the shares' first units alone need no unit capacity
    st = md._lib.md_plan_shares(n_pad.ctypes.data_as(ip), 1, 1024, 256, 1824, None, 0,
                                first.ctypes.data_as(ip), C.byref(nu), C.byref(ns))
    assert st == md.MD_OK and first[-1] == 2016 and np.all(np.diff(first) >= 1)
