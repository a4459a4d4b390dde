"""Pins of the oracle's integer passes (chunk table, per-chunk bucket offsets and order)
against numpy's own counting and stable sorting, including empty and ragged sequences."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("lens,C", [([5, 0, 12], 4), ([1], 1), ([0, 0, 7], 7), ([100, 3, 64, 65], 32),
                                    ([0], 8)])
def test_chunk_table_matches_numpy(lens, C):
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    base, seq = oracle.chunk_table(offsets, C)
    per = np.array([(n + C - 1) // C for n in lens], dtype=np.int64)
    np.testing.assert_array_equal(base, np.concatenate([[0], np.cumsum(per)]))
    np.testing.assert_array_equal(seq, np.repeat(np.arange(len(lens)), per))


@pytest.mark.parametrize("N,M,C,P", [(23, 10, 8, 3), (1000, 300, 192, 8), (1, 5, 4, 2),
                                     (0, 4, 16, 2), (257, 7, 64, 7), (130, 1, 32, 1)])
def test_bucket_order_matches_stable_sort(N, M, C, P):
    c = np.random.default_rng(N + M).integers(0, M, N).astype(np.int32)
    bs, order = oracle.bucket_order(c, M, C, P)
    for b in range((N + C - 1) // C):
        cc = c[b * C: (b + 1) * C]
        idx = np.arange(cc.shape[0])
        want = np.lexsort((idx, cc // P, cc % P))        # last key is the primary one
        np.testing.assert_array_equal(order[b * C: b * C + cc.shape[0]], want)
        blocks = np.bincount(cc % P, minlength=P)
        np.testing.assert_array_equal(bs[b], np.concatenate([[0], np.cumsum(blocks)]))


@pytest.mark.parametrize("M,density,all_entries", [(7, 0.3, False), (40, 0.05, False),
                                                   (5, 0.0, False), (9, 0.5, True)])
def test_support_rows_match_numpy(M, density, all_entries):
    rng = np.random.default_rng(M)
    a = rng.uniform(0.1, 1.0, (M, M)) * (rng.random((M, M)) < density)
    row_ptr, col = oracle.support_rows(a, all_entries)
    mask = np.ones_like(a, bool) if all_entries else a != 0
    np.testing.assert_array_equal(row_ptr, np.concatenate([[0], np.cumsum(mask.sum(1))]))
    np.testing.assert_array_equal(col, np.nonzero(mask)[1])


@pytest.mark.parametrize("N,M,L", [(100, 7, 30), (1, 3, 5), (0, 4, 8), (1000, 50, 1000), (257, 1, 16)])
def test_mark_sort_matches_stable_sort(N, M, L):
    c = np.random.default_rng(N + 3).integers(0, M, N).astype(np.int32)
    start, order = oracle.mark_sort(c, M, L)
    seg = np.arange(N) // L
    want = np.lexsort((np.arange(N), c, seg))
    np.testing.assert_array_equal(order, want)
    nseg = (N + L - 1) // L
    counts = np.zeros(nseg * M, np.int64)
    np.add.at(counts, seg * M + c, 1)
    np.testing.assert_array_equal(start, np.concatenate([[0], np.cumsum(counts)]))
