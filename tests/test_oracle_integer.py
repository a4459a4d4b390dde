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
