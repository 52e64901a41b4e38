"""CPU checks of the index arithmetic the CUDA kernels rely on (no GPU, no oracle).

The kernels take these facts as given, so they are checked here exactly, over every size the
kernels accept:
- F stage: pad(i) = i + floor(i / 16) splits, pad(j + r P) = pad(j) + pad(r P) for a power
  of two P and j < P, which turns every strided shared-memory index into a base plus
  compile-time offsets; the row pitches read from the kernel source hold a padded row and
  keep the transposed load phase and the stores of a warp's channels free of bank conflicts.
- Tile decode: the upper-triangle block index -> (I, J) by a float square root and integer
  correction is exact for every block count up to 128 (8192 inputs).
- Dump step: blocks over baseline row pairs (i, N - 1 - i) cover every baseline once.
"""
import pathlib
import re

import numpy as np

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_0906_1887_gb300" / "csrc"


def pad(i):
    return i + (i >> 4)


def _pitches():
    src = (CSRC / "fengine.cu").read_text()
    body = src[src.index("constexpr int f_pitch(int LG)"):]
    body = body[:body.index("}")]
    pairs = {int(a): int(b) for a, b in re.findall(r"LG == (\d+) \? (\d+)", body)}
    last = int(re.findall(r": (\d+);", body)[-1])
    return {lg: pairs.get(lg, last) for lg in range(3, 13)}


def test_pad_splits_over_every_stage():
    for lg in range(3, 13):
        L = 1 << lg
        ns, lgns = 1, 0
        while ns < L:
            lgr = min(4, lg - lgns)
            R, LR = 1 << lgr, L >> lgr
            for j in range(LR):
                k = j & (ns - 1)
                d = (j - k) * R + k
                for r in range(R):
                    assert pad(j + r * LR) == pad(j) + pad(r * LR)
                    assert pad(d + r * ns) == pad(d) + pad(r * ns)
            ns <<= lgr
            lgns += lgr


def _halfwarp_wavefronts(words):
    """Wavefronts of one 64-bit shared access by 16 lanes (word addresses of the first word)."""
    banks = {}
    for a in words:
        for w in (a, a + 1):
            banks.setdefault(w % 32, set()).add(w)
    return max(len(v) for v in banks.values())


def test_row_pitches_fit_and_are_conflict_free():
    for lg, pitch in _pitches().items():
        L = 1 << lg
        G = 4096 >> lg if lg >= 6 else 64
        assert pitch >= pad(L - 1) + 1, (L, pitch)
        # last stage / output: lanes along the inputs, one channel
        for c in range(0, L, max(1, L // 8)):
            for g0 in range(0, G, 16):
                lanes = [g for g in range(g0, min(G, g0 + 16))]
                assert _halfwarp_wavefronts([2 * (g * pitch + pad(c)) for g in lanes]) == 1, (L, c)


def test_tile_decode_exact():
    f32 = np.float32
    for nb in range(1, 129):
        tile = 0
        for I in range(nb):
            for J in range(I, nb):
                b = 2 * nb + 1
                i = int((f32(b) - np.sqrt(f32(b * b - 8 * tile))) * f32(0.5))
                i = max(0, min(i, nb - 1))
                while i > 0 and i * nb - i * (i - 1) // 2 > tile:
                    i -= 1
                while i + 1 < nb and (i + 1) * nb - (i + 1) * i // 2 <= tile:
                    i += 1
                assert (i, i + (tile - (i * nb - i * (i - 1) // 2))) == (I, J), (nb, tile)
                tile += 1


def test_dump_row_pairs_cover_every_baseline_once():
    def off(i, n):
        return i * n - i * (i - 1) // 2
    for n in list(range(1, 70)) + [255, 256, 1023, 1024]:
        seen = np.zeros(n * (n + 1) // 2, np.int64)
        for i0 in range((n + 1) // 2):
            i1 = n - 1 - i0
            len0 = n - i0
            length = len0 if i1 == i0 else n + 1
            e = np.arange(length)
            first = e < len0
            b = np.where(first, off(i0, n) + e, off(i1, n) + (e - len0))
            j = np.where(first, i0 + e, i1 + (e - len0))
            i = np.where(first, i0, i1)
            assert np.all(b == np.array([off(ii, n) for ii in i]) + (j - i))
            np.add.at(seen, b, 1)
        assert np.all(seen == 1), n


def _pairs_upto(m):
    """S(m) = sum over k = 1..m of ceil(k / 2): items of m consecutive block rows of lengths 1..m."""
    return ((m + 1) >> 1) * ((m + 2) >> 1)


def _wide_coords(tile, nb):
    """The kernel's decode of a wide work item: row I holds the items J0 = I, I + 2, ... < nb."""
    R = _pairs_upto(nb) - tile
    m = int(np.float32(2.0) * np.sqrt(np.float32(R)) - np.float32(1.5))
    m = max(0, min(m, nb))
    while m > 0 and _pairs_upto(m - 1) >= R:
        m -= 1
    while _pairs_upto(m) < R:
        m += 1
    I = nb - m
    return I, I + 2 * (tile - (_pairs_upto(nb) - _pairs_upto(m)))


def test_wide_item_decode_covers_every_tile_once():
    # wide items (block I against blocks J0 and J0 + 1 in one N = 256 MMA): every upper-triangle
    # tile of every array up to 128 blocks belongs to exactly one item, items of a row are
    # consecutive, and the second block exists unless J0 is the last block
    for nb in range(1, 129):
        seen = {}
        n_items = _pairs_upto(nb)
        assert n_items == sum((nb - i + 1) // 2 for i in range(nb))
        prev = (-1, -1)
        for tile in range(n_items):
            I, J0 = _wide_coords(tile, nb)
            assert 0 <= I <= J0 < nb and (J0 - I) % 2 == 0
            assert (I, J0) > prev
            prev = (I, J0)
            for J in range(J0, min(J0 + 2, nb)):
                assert (I, J) not in seen
                seen[(I, J)] = tile
        assert len(seen) == nb * (nb + 1) // 2
