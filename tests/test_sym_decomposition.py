"""The block decomposition behind the symmetric pass, checked in FP64 on the CPU.

K is symmetric, so the segment sums S_ic = sum_{j in L_c} K_ij can be taken from
the 128 x 128 blocks on and above the diagonal alone: block (I, J), I <= J, gives
the row sums of its rows (slot J of the rows of block I) and, off the diagonal,
its column sums (slot I of the rows of block J).  Every (slot, cluster, row) is
written exactly once, and the slots of a row add up to S.  This test builds the
slots exactly as described (numpy, no GPU) for ragged n and compares their sum
with the plain definition, so a wrong slot, a missing block or a double-counted
diagonal would show.  It also checks the block-packed, swizzled tile layout the
K build writes and the stream's loads expect: every element of the triangle is
stored once, at a distinct offset, inside its tile.
"""
import numpy as np
import pytest

B = 128


def _slots(K, lab, k):
    n = K.shape[0]
    T = (n + B - 1) // B
    slots = np.full((T, k, n), np.nan)
    for I in range(T):
        rI = slice(I * B, min(n, I * B + B))
        for J in range(I, T):
            cJ = slice(J * B, min(n, J * B + B))
            blk = K[rI, cJ]
            for c in range(k):
                # row sums of block (I, J) over its columns of cluster c -> slot J, rows of I
                assert np.all(np.isnan(slots[J, c, rI]))
                slots[J, c, rI] = blk[:, lab[cJ] == c].sum(axis=1)
                if I != J:
                    # column sums over its rows of cluster c -> slot I, rows of J
                    assert np.all(np.isnan(slots[I, c, cJ]))
                    slots[I, c, cJ] = blk[lab[rI] == c, :].sum(axis=0)
    return slots


@pytest.mark.parametrize("n,k", [(1, 1), (97, 3), (128, 2), (300, 4), (513, 8)])
def test_slots_sum_to_segment_sums(n, k):
    rng = np.random.default_rng(n * 31 + k)
    X = rng.standard_normal((n, 3))
    K = np.exp(-((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))    # a symmetric K
    lab = rng.integers(0, k, size=n)
    slots = _slots(K, lab, k)
    assert not np.isnan(slots).any()                                 # every slot written
    S = np.stack([K[:, lab == c].sum(axis=1) for c in range(k)])     # [c][i]
    np.testing.assert_allclose(slots.sum(axis=0), S, rtol=1e-12, atol=1e-12)


def _packed_offset(tile, r, c):
    """Float offset of element (r, c) of a tile in the block-packed layout: four boxes of
    128 rows x 32 columns, 16-byte chunk j of row r stored at chunk j ^ (r mod 8)."""
    box, j, e = c // 32, (c % 32) // 4, c % 4
    return tile * B * B + box * B * 32 + r * 32 + ((j ^ (r % 8)) * 4) + e


@pytest.mark.parametrize("T", [1, 3])
def test_packed_layout_is_a_bijection_per_tile(T):
    tiles = T * (T + 1) // 2
    seen = np.zeros(tiles * B * B, dtype=np.int32)
    r, c = np.meshgrid(np.arange(B), np.arange(B), indexing="ij")
    for t in range(tiles):
        off = _packed_offset(t, r, c)
        assert off.min() == t * B * B and off.max() == (t + 1) * B * B - 1
        np.add.at(seen, off.ravel(), 1)
    assert np.all(seen == 1)


def test_packed_rows_of_a_chunk_hit_distinct_banks():
    # lanes reading rows r .. r + 7 of one 16-byte chunk (the row group's float4 loads)
    # touch 8 different 16-byte bank groups: a conflict-free quarter-warp
    for j in range(8):
        for r0 in range(0, B, 8):
            groups = {(_packed_offset(0, r, 4 * j) % 32) // 4 for r in range(r0, r0 + 8)}
            assert len(groups) == 8
