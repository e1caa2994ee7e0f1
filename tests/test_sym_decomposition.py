"""The block decomposition behind the symmetric pass, checked in FP64 on the CPU.

K is symmetric, so the segment sums S_ic = sum_{j in L_c} K_ij can be taken from
the 128 x 128 blocks on and above the diagonal alone: block (I, J), I <= J, gives
the row sums of its rows and, off the diagonal, the column sums of its columns'
rows.  The pass hands out super-tiles of a x a blocks: super-tile (Is, Js),
Is <= Js, accumulates the row sums of each of its block rows over its columns and
stores them to slot Js of those rows, and the column sums of each of its block
columns over its rows, stored to slot Is of those rows -- or, for a diagonal
super-tile of the sorted form, to the extra slot Ts.  Every (slot, cluster, row) is
written exactly once, and the slots of a row add up to S.  This test builds the
slots exactly as the kernels order the blocks (numpy, no GPU) for ragged n and every
super-tile edge, and compares their sum with the plain definition, so a wrong slot,
a missing block or a double-counted diagonal would show.  It also checks the
block-packed, swizzled tile layouts the K builds write and the streams' loads expect
(every element of the triangle stored once, at a distinct offset, inside its tile),
and the sorted form's per-block lists: the header, the padded entries and a lane's
walk over them give the cluster sums of its rows and columns, with every read inside
the list and the tile.
"""
import numpy as np
import pytest

B = 128


def _slots(K, lab, k, a, extra_slot):
    """The slots as the stream kernels store them.  Super-tile (Is, Js) is taken block by
    block in the kernels' Latin-square order; row warp i keeps the row sums of block row
    I0 + i over the super-tile's columns, column warp j the column sums of block column
    J0 + j over its rows (diagonal blocks excluded), and each stores once at the end:
    rows to slot Js, columns to slot Is, or to the extra slot Ts from a diagonal
    super-tile.  The branch form (a = 1) has no extra slot and skips that store."""
    n = K.shape[0]
    T = (n + B - 1) // B
    Ts = (T + a - 1) // a
    slots = np.full((Ts + (1 if extra_slot else 0), k, n), np.nan)

    def rows(I):
        return slice(I * B, min(n, I * B + B))

    def store(slot, I, v):
        assert np.all(np.isnan(slots[slot, :, rows(I)]))
        slots[slot, :, rows(I)] = v

    for Is in range(Ts):
        for Js in range(Is, Ts):
            I0, J0 = Is * a, Js * a
            racc = {i: np.zeros((k, B)) for i in range(a)}
            cacc = {j: np.zeros((k, B)) for j in range(a)}
            seen = set()
            for m in range(a):
                for i in range(a):
                    I, J = I0 + i, J0 + (i + m) % a
                    if I >= T or J >= T or J < I:
                        continue
                    assert (I, J) not in seen
                    seen.add((I, J))
                    blk = K[rows(I), rows(J)]
                    for c in range(k):
                        racc[i][c, :blk.shape[0]] += blk[:, lab[rows(J)] == c].sum(axis=1)
                        if I != J:
                            cacc[J - J0][c, :blk.shape[1]] += blk[lab[rows(I)] == c, :].sum(axis=0)
            want = {(I, J) for I in range(I0, min(I0 + a, T)) for J in range(max(I, J0), min(J0 + a, T))}
            assert seen == want
            for i in range(a):
                if I0 + i < T:
                    store(Js, I0 + i, racc[i][:, :rows(I0 + i).stop - rows(I0 + i).start])
            for j in range(a):
                J = J0 + j
                if J < T and (Is != Js or extra_slot):
                    store(Ts if Is == Js else Is, J, cacc[j][:, :rows(J).stop - rows(J).start])
    return slots


@pytest.mark.parametrize("a,extra", [(1, False), (1, True), (2, True), (3, True), (4, True), (7, True), (8, True)])
@pytest.mark.parametrize("n,k", [(1, 1), (97, 3), (128, 2), (300, 4), (513, 8), (1100, 16), (2000, 5)])
def test_slots_sum_to_segment_sums(n, k, a, extra):
    rng = np.random.default_rng(n * 31 + k)
    X = rng.standard_normal((n, 3))
    K = np.exp(-((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))    # a symmetric K
    lab = rng.integers(0, k, size=n)
    slots = _slots(K, lab, k, a, extra)
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


# ---------------------------------------------------------------- the XOR-32 layout of the sorted form

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


def test_sorted_entries_xor_keys_give_the_offsets():
    """In bytes: the column entry of point l, 16384 (l >> 5) + 4 (l & 31), XOR 132 lane,
    plus 4096 e, is element (row lane + 32 e, column l); the row entry 128 l + 4 (l & 31),
    XOR 4 lane, plus 16384 e, is element (row l, column lane + 32 e).  All inside 64 KB."""
    for l in range(B):
        colent = 16384 * (l >> 5) + 4 * (l & 31)
        rowent = 128 * l + 4 * (l & 31)
        for lane in range(32):
            for e in range(4):
                a = (colent ^ (132 * lane)) + 4096 * e
                b = (rowent ^ (4 * lane)) + 16384 * e
                assert a == 4 * _sw4_offset(lane + 32 * e, l) and 0 <= a < 65536
                assert b == 4 * _sw4_offset(l, lane + 32 * e) and 0 <= b < 65536


def test_sw4_float4_store_of_the_simt_build():
    """Four consecutive columns cl..cl+3 (cl a multiple of 4) of row r land in one 16-byte
    chunk at (cl mod 32) ^ (r & 28), element e in slot e ^ (r mod 4)."""
    for r in range(B):
        for cl in range(0, B, 4):
            base = (cl // 32) * B * 32 + r * 32 + ((cl % 32) ^ (r & 28))
            for e in range(4):
                assert _sw4_offset(r, cl + e) == base + (e ^ (r & 3))


# ---------------------------------------------------------------- the sorted form's lists

HDR = 32        # header words (u32, one per cluster)


def _list_len(k):
    return ((B + 3 * k + 3) & ~3) + 4


def _sorted_lists(labels_block, k):
    """One 128-block's lists as sym_sort_kernel writes them: a header word per cluster,
    (start << 8) | count, then the entries cluster after cluster in stable order, each
    cluster padded to a multiple of 4 with 0; the column list holds the byte offset
    16384 (l >> 5) + 4 (l & 31) of point l as a column, the row list 128 l + 4 (l & 31)."""
    lab = np.asarray(labels_block)
    L = _list_len(k)
    cnt = [int(np.sum(lab == c)) for c in range(k)]
    start = np.concatenate([[0], np.cumsum([(m + 3) & ~3 for m in cnt])])[:k]
    colw = np.zeros(HDR + L, dtype=np.int64)
    roww = np.zeros(HDR + L, dtype=np.int64)
    for c in range(k):
        colw[c] = roww[c] = (int(start[c]) << 8) | cnt[c]
        for q, l in enumerate(np.nonzero(lab == c)[0]):
            colw[HDR + start[c] + q] = 16384 * (l >> 5) + 4 * (l & 31)
            roww[HDR + start[c] + q] = 128 * l + 4 * (l & 31)
    return colw, roww


def _sum_sorted(tile_bytes_to_value, words, k, key, stride):
    """What one lane of sum_sorted computes on one tile: for each cluster, chunks of 4
    entries (the next chunk read ahead) and a tail of 1-3; element of entry x for the
    lane's e-th row (column) at (x ^ key) + stride e.  Returns sums [k][4] and checks
    that every list read stays inside the list and every element read inside the tile."""
    L = len(words) - HDR
    acc = np.zeros((k, 4))
    for c in range(k):
        h = int(words[c])
        p0, cnt = h >> 8, h & 0xFF
        pe = p0 + (cnt & ~3)

        def chunk(p):
            assert 0 <= p and p + 4 <= L
            return [int(w) for w in words[HDR + p:HDR + p + 4]]

        cw = chunk(p0)
        p = p0
        while p < pe:
            cur, cw = cw, chunk(p + 4)
            for x in cur:
                for e in range(4):
                    acc[c, e] += tile_bytes_to_value((x ^ key) + stride * e)
            p += 4
        for x in cw[:cnt & 3]:
            for e in range(4):
                acc[c, e] += tile_bytes_to_value((x ^ key) + stride * e)
    return acc


@pytest.mark.parametrize("valid,k,seed", [(128, 10, 0), (128, 1, 1), (77, 16, 2), (64, 3, 3), (63, 32, 4),
                                          (1, 5, 5), (128, 32, 6), (112, 12, 7), (128, 4, 8)])
def test_sorted_lists_give_the_cluster_sums(valid, k, seed):
    """Row warp (key 132 lane, stride 4096) and column warp (key 4 lane, stride 16384) of
    the sorted form, on a tile in the XOR-32 layout: each lane's sums are the row
    (column) cluster sums of its 4 rows (columns)."""
    rng = np.random.default_rng(seed)
    lab = np.full(B, 0xFF, dtype=np.int64)
    lab[:valid] = rng.integers(0, k, size=valid)
    tile = rng.standard_normal((B, B))
    tile[valid:, :] = np.nan              # entries past the block's points are never read
    tile[:, valid:] = np.nan
    mem = np.full(B * B, np.nan)
    r, c = np.meshgrid(np.arange(B), np.arange(B), indexing="ij")
    mem[_sw4_offset(r, c).ravel()] = tile.ravel()

    def value(byte_off):
        assert byte_off % 4 == 0 and 0 <= byte_off < 4 * B * B
        return mem[byte_off // 4]

    colw, roww = _sorted_lists(lab, k)
    for lane in range(32):
        mine = [lane + 32 * e for e in range(4)]
        got = _sum_sorted(value, colw, k, 132 * lane, 4096)            # row warp: rows lane + 32 e
        for e, rr in enumerate(mine):
            if rr < valid:
                ref = [tile[rr, :valid][lab[:valid] == cc].sum() for cc in range(k)]
                np.testing.assert_allclose(got[:, e], ref, rtol=1e-12, atol=1e-12)
        got = _sum_sorted(value, roww, k, 4 * lane, 16384)             # column warp: columns lane + 32 e
        for e, cl in enumerate(mine):
            if cl < valid:
                ref = [tile[:valid, cl][lab[:valid] == cc].sum() for cc in range(k)]
                np.testing.assert_allclose(got[:, e], ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- the half layout (FP16 / BF16 K)
# The tensor-core form reads tiles in the 128-byte swizzle of the MMA shared-memory operands:
# within each 1024-byte group of 8 rows of 128 bytes, 16-byte chunk j of row r sits at chunk
# j ^ (r mod 8).  Below, the operand views are modelled as the canonical layouts composed
# with that swizzle, and checked to address the element the math needs.

def _sw128h_offset(r, c):
    """Byte offset of element (r, c) of a tile in the half layout kPackedSw128H: two boxes of
    128 rows x 64 columns (16 KB each), chunk (c mod 64) // 8 of row r swizzled by r mod 8."""
    return 16384 * (c // 64) + 128 * r + 16 * (((c % 64) // 8) ^ (r % 8)) + 2 * (c % 8)


def _swizzle128(addr):
    """The 128-byte swizzle on byte addresses (1024-byte aligned base): bits 4-6 ^= bits 7-9."""
    return addr ^ (((addr >> 7) & 7) << 4)


def test_half_layout_is_a_bijection_and_the_swizzle_of_row_major_boxes():
    r, c = np.meshgrid(np.arange(B), np.arange(B), indexing="ij")
    off = _sw128h_offset(r, c)
    assert sorted(off.ravel().tolist()) == list(range(0, 2 * B * B, 2))
    for rr in range(B):
        for cc in range(B):
            plain = 16384 * (cc // 64) + 128 * rr + 2 * (cc % 64)      # row-major 128 x 64 boxes
            assert _sw128h_offset(rr, cc) == _swizzle128(plain)


def test_pack_half_word_mapping():
    """pack_half_kernel's output word o (box o >> 12, row (o >> 5) & 127, column
    64 box + 8 (((o >> 2) & 7) ^ (row & 7)) + 2 (o & 3)) holds the two elements the layout
    puts at bytes 4 o and 4 o + 2; every element is written once."""
    seen = set()
    for o in range(8192):
        b, r = o >> 12, (o >> 5) & 127
        C = 64 * b + 8 * (((o >> 2) & 7) ^ (r & 7)) + 2 * (o & 3)
        assert _sw128h_offset(r, C) == 4 * o and _sw128h_offset(r, C + 1) == 4 * o + 2
        seen.add((r, C))
    assert len(seen) == 8192


def _kmajor_sw128(start, m, kidx, sbo=1024):
    """K-major operand, 128-byte swizzle: row m of 64 elements (128 bytes), 8-row groups sbo
    apart; element kidx < 16 of the K = 16 slice that starts at byte `start`."""
    return _swizzle128(start + (m // 8) * sbo + (m % 8) * 128 + 2 * kidx)


def _mnmajor_sw128(start, m, kidx, lbo, sbo):
    """MN-major operand, 128-byte swizzle: atoms of 64 elements along M (one 128-byte row) by
    8 reduction rows; atoms lbo apart along M, 8-row groups sbo apart along the reduction."""
    return _swizzle128(start + (m // 64) * lbo + (kidx // 8) * sbo + (kidx % 8) * 128 + 2 * (m % 64))


def test_tile_is_the_k_major_operand_of_the_row_sums():
    """Row sums R = K V_J^T: A[m = r][kk-th slice, element e] must be K[r][16 kk + e], from
    start = 16384 (kk >> 2) + 32 (kk & 3) (16 columns = 32 bytes along a row, box 2 at 16 KB)."""
    for kk in range(8):
        start = 16384 * (kk >> 2) + 32 * (kk & 3)
        for r in range(B):
            for e in range(16):
                assert _kmajor_sw128(start - 32 * (kk & 3), r, 16 * (kk & 3) + e) == _sw128h_offset(r, 16 * kk + e)


def test_tile_is_the_mn_major_operand_of_the_column_sums():
    """Column sums C = K^T V_I^T: A'[m = column c][kk-th slice, element e] must be
    K[16 kk + e][c], from start = 2048 kk (16 rows), atoms 16 KB apart (lbo), 8-row groups
    1 KB apart (sbo); and every byte it reads lies inside the 32 KB tile."""
    for kk in range(8):
        for c in range(B):
            for e in range(16):
                a = _mnmajor_sw128(2048 * kk, c, e, lbo=16384, sbo=1024)
                assert a == _sw128h_offset(16 * kk + e, c) and 0 <= a < 32768


def test_onehot_operand_layout():
    """sym_onehot_kernel: 16-byte chunk q = (box, c, ch) holds points 64 box + 8 (ch ^ (c mod 8))
    + 0..7 of cluster row c -- the K-major swizzled operand of N rows: B[n = c][kk-th slice,
    element e] = V[c][16 kk + e] from start (N x 128) (kk >> 2) + 32 (kk & 3)."""
    for N in (16, 32):
        where = {}
        for q in range(N * 16):
            box, c, ch = q // (N * 8), (q >> 3) % N, q & 7
            i0 = 64 * box + 8 * (ch ^ (c & 7))
            for e in range(8):
                where[(c, i0 + e)] = 16 * q + 2 * e
        assert len(where) == N * B
        for kk in range(8):
            base = N * 128 * (kk >> 2)
            for c in range(N):
                for e in range(16):
                    i = 16 * kk + e
                    assert _kmajor_sw128(base, c, 16 * (kk & 3) + e) == where[(c, i)]


def test_batched_build_half_tile_and_transpose_stores():
    """The batched FP32 build's half-tile epilogue: a thread's 4 consecutive columns of row r
    (4-aligned) are one 8-byte store at off(r, c) in tile (I, J), and its 4 consecutive rows
    of column c are one 8-byte store at off(c, r) in tile (J, I).  Every element of both tiles
    is written exactly once, each 8-byte store stays inside one 16-byte chunk, and the
    element the K-major MMA operand reads for (row, column) of tile (J, I) is K[column][row]
    of tile (I, J)."""
    def off(r, c):
        return 16384 * (c >> 6) + 128 * r + 16 * (((c >> 3) & 7) ^ (r & 7)) + 2 * (c & 7)

    direct, trans = {}, {}
    for r in range(B):
        for c0 in range(0, B, 4):
            base = off(r, c0)
            assert base % 8 == 0 and (base % 16) + 8 <= 16
            for e in range(4):
                assert off(r, c0 + e) == base + 2 * e
                direct[base + 2 * e] = (r, c0 + e)
    for c in range(B):
        for r0 in range(0, B, 4):
            base = off(c, r0)           # transposed tile: row c, columns r0 .. r0 + 3
            for e in range(4):
                assert off(c, r0 + e) == base + 2 * e
                trans[base + 2 * e] = (r0 + e, c)   # holds K[r0 + e][c] of the direct tile
    assert len(direct) == len(trans) == B * B
    for kk in range(8):                  # the MMA's K-major reads of the transposed tile
        start = 16384 * (kk >> 2)
        for m in range(B):
            for e in range(16):
                a = _kmajor_sw128(start, m, 16 * (kk & 3) + e)
                assert trans[a] == (16 * kk + e, m)   # operand (row m, column 16 kk + e) = K[16 kk + e][m]


# ---------------------------------------------------------------- the z reduction's in-block sort

def _block_sort_positions(labels, k, nw=32):
    """zreduce_body's placement of a block's rows, step by step: each warp's rank of a row
    among its earlier lanes with the same label (match + popcount), the per-warp counts, the
    cluster starts (a scan over clusters of the warps' totals), each warp's offset inside its
    cluster (a scan over warps), and the position offset + rank.  -1 labels (rows past n) are
    not placed."""
    rows = len(labels)
    cnt = np.zeros((nw, k), dtype=np.int64)
    rank = np.zeros(rows, dtype=np.int64)
    for w in range(nw):
        for lane in range(32):
            i = 32 * w + lane
            if i >= rows or labels[i] < 0:
                continue
            rank[i] = sum(1 for l2 in range(lane) if labels[32 * w + l2] == labels[i])
            cnt[w, labels[i]] += 1
    totals = cnt.sum(axis=0)
    cstart = np.concatenate([[0], np.cumsum(totals)])
    off = np.zeros((nw, k), dtype=np.int64)
    for c in range(k):
        o = cstart[c]
        for w in range(nw):
            off[w, c] = o
            o += cnt[w, c]
    pos = np.full(rows, -1)
    for i in range(rows):
        if labels[i] >= 0:
            pos[i] = off[i // 32, labels[i]] + rank[i]
    return pos, cstart


@pytest.mark.parametrize("k,valid,seed", [(10, 1024, 0), (1, 1024, 1), (64, 1000, 2), (256, 777, 3), (3, 5, 4)])
def test_zreduce_block_sort_is_a_stable_counting_sort(k, valid, seed):
    rng = np.random.default_rng(seed)
    labels = np.full(1024, -1)
    labels[:valid] = rng.integers(0, k, size=valid)
    if k > 2:
        labels[:valid][labels[:valid] == 1] = 0          # an empty cluster
    pos, cstart = _block_sort_positions(labels, k)
    placed = pos[pos >= 0]
    assert sorted(placed.tolist()) == list(range(valid))  # a permutation of the valid rows
    order = np.argsort(pos[:valid], kind="stable")
    expect = np.argsort(labels[:valid], kind="stable")    # by label, row order kept among equals
    np.testing.assert_array_equal(order, expect)
    for c in range(k):                                     # each cluster's rows sit in its range
        idx = np.nonzero(labels[:valid] == c)[0]
        assert np.all((pos[idx] >= cstart[c]) & (pos[idx] < cstart[c + 1]))
