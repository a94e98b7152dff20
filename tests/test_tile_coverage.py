"""Index arithmetic of the tensor-core GEMM, the bias-gradient column sums and the grouped LU,
checked on CPU: the work splits that csrc/gemm_tc.cu and csrc/ansatz.cu compute (restated here
formula by formula) cover every output element, every k-block and every row exactly once for
ragged shapes, and every TMA box starts on a 16-byte boundary. No GPU and no library call."""
import itertools

import pytest

TC_BK = 64
TC_MAX_UNIT_KB = 512


def tc_split_count(tiles, nkb):
    splits = 1
    while tiles * splits < 148 and splits * 2 <= nkb and splits < 64:
        splits *= 2
    while nkb // splits > TC_MAX_UNIT_KB and splits * 2 <= nkb and splits < 64:
        splits *= 2
    return splits


def host_splits(M, N, K, BN, split_ok=True):
    """gemm_tc_run: splits from 128-row tiles at tile width BN, then the ceil correction."""
    tiles = -(-N // BN) * -(-M // 128)
    nkb = -(-K // TC_BK)
    splits = tc_split_count(tiles, nkb) if split_ok else 1
    if splits > 1:
        per = -(-nkb // splits)
        splits = -(-nkb // per)
    return splits


def unit_of_pair(u, M, N, K, splits, BN):
    ntn, ntm = -(-N // BN), -(-M // 256)
    tiles = ntn * ntm
    z, t = divmod(u, tiles)
    nkb = -(-K // TC_BK)
    per = -(-nkb // splits)
    kb0 = z * per
    nk = max(0, min(nkb, kb0 + per) - kb0)
    return (t // ntn) * 256, (t % ntn) * BN, kb0, nk, z


SHAPES = [(1, 1, 1), (255, 257, 63), (256, 256, 64), (1000, 300, 200), (4096 + 77, 1000, 1024),
          (2016, 1024, 1 << 20), (1024, 88, 1 << 18), (300, 2016, 136), (1 << 20, 2016, 1024)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_paired_units_cover_every_tile_and_k_block_once(M, N, K):
    """k_gemm_tc_pair: unit u = (split z, 256-row tile, 256-column tile); CTA rank r of the pair
    owns rows m0 + 128 r .. + 128 of the tile, all its columns in tensor memory, and stages B rows
    n0 + 128 r .. + 128. Every (128-row block, column tile) gets every k-block exactly once."""
    BN = 256
    splits = host_splits(M, N, K, BN)
    nkb = -(-K // TC_BK)
    units = -(-N // BN) * -(-M // 256) * splits
    seen = {}
    for u in range(units):
        m0, n0, kb0, nk, z = unit_of_pair(u, M, N, K, splits, BN)
        assert 0 <= z < splits and nk >= 1  # no empty split after the ceil correction
        b_rows = []
        for rank in (0, 1):
            rb = m0 + 128 * rank
            key = (rb // 128, n0 // BN)
            ks = seen.setdefault(key, [])
            ks.extend(range(kb0, kb0 + nk))
            b_rows.append(range(n0 + 128 * rank, n0 + 128 * rank + 128))
        # the two halves of B make up the unit's BN columns
        assert sorted(itertools.chain(*b_rows)) == list(range(n0, n0 + BN))
    for rt in range(-(-M // 256) * 2):
        for ct in range(-(-N // BN)):
            assert sorted(seen[(rt, ct)]) == list(range(nkb)), (rt, ct)


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (1, 1), (1, 0), (0, 1)])
def test_tma_box_origins_are_16_byte_aligned(M, N, K, a_mn, b_mn):
    """The innermost coordinate of every operand box: K-major boxes start at k = 64 kb; MN-major
    boxes at m (or n) = tile origin + 128 rank + 64 j. bf16: a multiple of 8 elements."""
    BN = 256
    splits = host_splits(M, N, K, BN)
    units = -(-N // BN) * -(-M // 256) * splits
    for u in range(min(units, 4096)):
        m0, n0, kb0, nk, _ = unit_of_pair(u, M, N, K, splits, BN)
        for rank in (0, 1):
            for kb in (kb0, kb0 + nk - 1):
                xs = []
                xs += [m0 + 128 * rank + 64 * j for j in range(2)] if a_mn else [kb * TC_BK]
                xs += [n0 + 128 * rank + 64 * j for j in range(2)] if b_mn else [kb * TC_BK]
                assert all((x * 2) % 16 == 0 for x in xs)


COLSUM_ROWS = 1024


def colsum_plan(M, N):
    """colsum_bf16: threads per row group, groups per 256-thread block, partials, blocks."""
    tpr = min(((N + 7) // 8 + 31) & ~31, 256)
    groups = 256 // tpr
    nparts = -(-M // COLSUM_ROWS)
    nblocks = -(-nparts // groups)
    return tpr, groups, nparts, nblocks


@pytest.mark.parametrize("M,N", [(1, 1), (1023, 84), (1025, 1024), (4097, 2016), (65536, 1024),
                                 (1 << 20, 2016), (3000, 2048), (3000, 2056), (777, 8)])
def test_colsum_groups_cover_every_row_and_column_once(M, N):
    """k_colsum_bf16_part: thread tt of group q in block b sums columns 8 tt + 8 tpr i .. + 7 of
    rows [(b G + q) R, ...) clipped to M; k_colsum_bf16_final reads partials 0 .. nparts - 1, and
    every partial past nparts is empty."""
    tpr, groups, nparts, nblocks = colsum_plan(M, N)
    assert tpr % 32 == 0 and groups >= 1 and groups * tpr <= 256
    rows_seen = [0] * M
    for b in range(nblocks):
        for q in range(groups):
            pidx = b * groups + q
            r0 = pidx * COLSUM_ROWS
            r1 = min(r0 + COLSUM_ROWS, M)
            if pidx >= nparts:
                assert r1 <= r0  # empty: the final pass never reads it
                continue
            for r in range(r0, r1):
                rows_seen[r] += 1
    assert rows_seen == [1] * M
    cols = []
    for tt in range(tpr):
        c8 = 8 * tt
        while c8 < N:
            cols.extend(c for c in range(c8, c8 + 8) if c < N)
            c8 += 8 * tpr
    assert sorted(cols) == list(range(N))


@pytest.mark.parametrize("N", list(range(13, 25)))
def test_grouped_lu_rows_and_configurations(N):
    """k_lu_grp<N>: lane l of group g holds rows l + 8 t (t < ceil(N / 8)) of the block of
    configuration 4 w + g: the rows of a block are held once each, no lane owns more than three,
    and the warps cover every configuration once (a ragged last warp included)."""
    R = (N + 7) // 8
    assert R <= 3
    rows = sorted(l + 8 * t for l in range(8) for t in range(R) if l + 8 * t < N)
    assert rows == list(range(N))
    for M in (1, 3, 4, 5, 400, 1023):
        got = sorted(4 * w + g for w in range(-(-M // 4)) for g in range(4) if 4 * w + g < M)
        assert got == list(range(M))
