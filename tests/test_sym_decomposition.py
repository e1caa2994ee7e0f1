"""The block decomposition behind the symmetric pass, checked in FP64 on the CPU.

K is symmetric, so the segment sums S_ic = sum_{j in L_c} K_ij can be taken from
the 128 x 128 blocks on and above the diagonal alone: block (I, J), I <= J, gives
the row sums of its rows and, off the diagonal, the column sums of its columns'
rows.  The pass hands out super-tiles of a x a blocks: super-tile (Is, Js),
Is <= Js, accumulates the row sums of each of its block rows over its columns and
stores them to slot Js of those rows, and the column sums of each of its block
columns over its rows, stored to slot Is of those rows -- or, for a diagonal
super-tile with a > 1, to the extra slot Ts.  Every (slot, cluster, row) is
written exactly once, and the slots of a row add up to S.  This test builds the
slots exactly as described (numpy, no GPU) for ragged n and every super-tile edge,
and compares their sum with the plain definition, so a wrong slot, a missing block
or a double-counted diagonal would show.  It also checks the block-packed, swizzled
tile layout the K builds write and the stream's loads expect: every element of the
triangle is stored once, at a distinct offset, inside its tile.
"""
import numpy as np
import pytest

B = 128


def _slots(K, lab, k, a):
    n = K.shape[0]
    T = (n + B - 1) // B
    Ts = (T + a - 1) // a
    slots = np.full((Ts + (1 if a > 1 else 0), k, n), np.nan)

    def rows(I):
        return slice(I * B, min(n, I * B + B))

    def store(slot, I, v):
        assert np.all(np.isnan(slots[slot, :, rows(I)]))
        slots[slot, :, rows(I)] = v

    for Is in range(Ts):
        for Js in range(Is, Ts):
            I0, I1, J0, J1 = Is * a, min(Is * a + a, T), Js * a, min(Js * a + a, T)
            colacc = {J: np.zeros((k, rows(J).stop - rows(J).start)) for J in range(J0, J1)}
            for I in range(I0, I1):
                rowacc = np.zeros((k, rows(I).stop - rows(I).start))
                for J in range(max(I, J0), J1):
                    blk = K[rows(I), rows(J)]
                    for c in range(k):
                        rowacc[c] += blk[:, lab[rows(J)] == c].sum(axis=1)    # row sums
                        if I != J:
                            colacc[J][c] += blk[lab[rows(I)] == c, :].sum(axis=0)   # column sums
                    if J == J1 - 1:
                        store(Js, I, rowacc)
                    if I == min(J, I1 - 1) and (I != J or a > 1):
                        store(Ts if Is == Js else Is, J, colacc[J])
    return slots


@pytest.mark.parametrize("a", [1, 2, 4])
@pytest.mark.parametrize("n,k", [(1, 1), (97, 3), (128, 2), (300, 4), (513, 8), (1100, 16)])
def test_slots_sum_to_segment_sums(n, k, a):
    rng = np.random.default_rng(n * 31 + k)
    X = rng.standard_normal((n, 3))
    K = np.exp(-((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))    # a symmetric K
    lab = rng.integers(0, k, size=n)
    slots = _slots(K, lab, k, a)
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


# ---------------------------------------------------------------- the run form's layout and metadata

def _sw4_offset(r, c):
    """Float offset of element (r, c) of a tile in the XOR-32 packed layout: four boxes of
    128 rows x 32 columns, element c of row r stored at (c mod 32) ^ (r mod 32)."""
    return (c // 32) * B * 32 + r * 32 + ((c % 32) ^ (r % 32))


def test_sw4_layout_is_a_bijection_and_conflict_free():
    r, c = np.meshgrid(np.arange(B), np.arange(B), indexing="ij")
    off = _sw4_offset(r, c)
    assert sorted(off.ravel().tolist()) == list(range(B * B))
    for col in range(B):                  # a column read by 32 consecutive rows (the row group)
        for r0 in range(0, B, 32):
            assert len({_sw4_offset(rr, col) % 32 for rr in range(r0, r0 + 32)}) == 32
    for row in range(B):                  # a row of a box read by 32 lanes (the column group)
        for b0 in range(0, B, 32):
            assert len({_sw4_offset(row, cc) % 32 for cc in range(b0, b0 + 32)}) == 32


def test_sw4_codes_xor_keys_give_the_offsets():
    """colcode(l) ^ (32 r + r mod 32) is the offset of (row r, column l), and
    rowcode(l) ^ (4096 q + lane) that of (row l, column 32 q + lane)."""
    for l in range(B):
        colcode = ((l >> 5) << 12) | (l & 31)
        rowcode = 32 * l + (l & 31)
        for r in range(B):
            assert colcode ^ (32 * r + (r & 31)) == _sw4_offset(r, l)
        for q in range(4):
            for lane in range(32):
                assert rowcode ^ (4096 * q + lane) == _sw4_offset(l, 32 * q + lane)


def test_sw4_float4_store_of_the_simt_build():
    """Four consecutive columns cl..cl+3 (cl a multiple of 4) of row r land in one 16-byte
    chunk at (cl mod 32) ^ (r & 28), element e in slot e ^ (r mod 4)."""
    for r in range(B):
        for cl in range(0, B, 4):
            base = (cl // 32) * B * 32 + r * 32 + ((cl % 32) ^ (r & 28))
            for e in range(4):
                assert _sw4_offset(r, cl + e) == base + (e ^ (r & 3))


def _meta(labels_block):
    """The run form's metadata of one 128-block, as sym_meta_kernel defines it: the stable
    sort of the block's labels (0xFF past the block's rows, sorting last), the label at
    each sorted position, and the positions that end a run of one real label (the first
    half also ends at 63)."""
    lab = np.asarray(labels_block)
    order = np.argsort(lab, kind="stable")
    slab = lab[order]
    ends = np.zeros(B, bool)
    for p in range(B):
        if slab[p] != 0xFF and (p == B - 1 or slab[p + 1] != slab[p] or p == 63):
            ends[p] = True
    return order, slab, ends


def _sum_runs(values_in_order, slab, ends, k):
    """What one lane computes for one block: the two halves' run sums added into per-half
    cluster sums at each run end, then the halves added."""
    acc = np.zeros((2, k))
    for h in range(2):
        run = 0.0
        for p in range(64 * h, 64 * h + 64):
            run += values_in_order[p]
            if ends[p]:
                acc[h, slab[p]] += run
                run = 0.0
    return acc[0] + acc[1]


@pytest.mark.parametrize("valid,k,seed", [(128, 10, 0), (128, 1, 1), (77, 16, 2), (64, 3, 3), (63, 32, 4),
                                          (1, 5, 5), (128, 32, 6)])
def test_run_sums_are_the_cluster_sums(valid, k, seed):
    rng = np.random.default_rng(seed)
    lab = np.full(B, 0xFF, dtype=np.int64)
    lab[:valid] = rng.integers(0, k, size=valid)
    order, slab, ends = _meta(lab)
    x = rng.standard_normal(B)
    x[valid:] = np.nan                    # entries past the block's rows are never added
    got = _sum_runs(x[order], slab, ends, k)
    ref = np.array([x[:valid][lab[:valid] == c].sum() for c in range(k)])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
