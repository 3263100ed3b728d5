"""The Python binding's argument marshalling on the CPU (no GPU, no library
call): bivariate and univariate inputs packed into the C ABI's descriptors and
two's-complement words read back through the raw pointers, the word count,
and sign-magnitude results (gbr_bigpoly) converted to Python integers and
back.  Expected values are plain Python integer arithmetic."""

import ctypes as C
import random

import numpy as np

from paper_1103_4697_gb300 import api as A
from paper_1103_4697_gb300 import native as N


def _read_words(ptr, count):
    return [int(v) for v in np.ctypeslib.as_array((C.c_uint64 * count).from_address(int(ptr)))]


def _decode(words, W):
    """Two's-complement integers of W 64-bit words each."""
    out = []
    for k in range(0, len(words), W):
        u = sum(words[k + q] << (64 * q) for q in range(W))
        out.append(u - (1 << (64 * W)) if u >> (64 * W - 1) else u)
    return out


def _rand_int(rng, bits):
    return rng.randint(-(1 << bits) + 1, (1 << bits) - 1)


def test_word_count_holds_the_magnitude_and_a_sign_bit():
    """The least W with 64 W >= bit length of |v| + 1; -2^63 (whose two's
    complement would fit one word) is given two, which is still exact."""
    for bits in range(0, 600):
        v = (1 << bits) - 1 if bits else 0
        W = A._words_for([v, -v])
        assert 64 * W >= bits + 1 and (W == 1 or 64 * (W - 1) < bits + 1)
    assert A._words_for([1 << 63]) == 2 and A._words_for([-(1 << 63)]) == 2
    assert _decode([int(w) for w in A._to_words(np.array([-(1 << 63)], dtype=object), 2)], 2) == [-(1 << 63)]


def test_bivariate_inputs_round_trip_through_the_descriptors():
    rng = random.Random(91)
    polys = []
    for _ in range(40):
        dy, dx = rng.randint(0, 5), rng.randint(0, 5)
        bits = rng.choice([8, 40, 63, 64, 100, 300, 511])
        polys.append([[_rand_int(rng, bits) for _ in range(rng.randint(1, dx + 1))] for _ in range(dy + 1)])
    keep = A._Packed()
    desc = A.pack_bipolys(polys, keep)
    for f, d in zip(polys, desc):
        width = max(len(r) for r in f)
        dense = [list(r) + [0] * (width - len(r)) for r in f]
        assert (int(d["deg_x"]), int(d["deg_y"])) == (width - 1, len(f) - 1)
        W = int(d["words"])
        assert W == A._words_for([c for r in f for c in r])
        got = _decode(_read_words(d["coef"], width * len(f) * W), W)
        assert got == [c for r in dense for c in r]


def test_word_boundaries_and_ragged_rows():
    """Coefficients at the ends of a signed word (2^63 - 1 and -2^63 stay one word, 2^63
    and -2^63 - 1 take two), ragged rows padded with zeros, an empty polynomial, and
    numpy integers as input, each read back through the descriptor."""
    cases = [[[(1 << 63) - 1, -(1 << 63)], [1]],
             [[1 << 63], [-(1 << 63) - 1, 0, 7]],
             [[np.int64(-5), np.int64(3)], [np.int64(2)]],
             [],
             [[0]],
             [[1, 2, 3], [], [4]]]
    keep = A._Packed()
    desc = A.pack_bipolys(cases, keep)
    for f, d in zip(cases, desc):
        rows = [[int(c) for c in r] for r in f] or [[0]]
        width = max(len(r) for r in rows) or 1
        dense = [r + [0] * (width - len(r)) for r in rows]
        assert (int(d["deg_x"]), int(d["deg_y"])) == (width - 1, len(dense) - 1)
        W = int(d["words"])
        flat = [c for r in dense for c in r]
        assert W == (1 if all(-(1 << 63) <= c < (1 << 63) for c in flat) else A._words_for(flat))
        assert _decode(_read_words(d["coef"], width * len(dense) * W), W) == flat


def test_int64_batch_array_descriptors():
    rng = np.random.default_rng(92)
    arr = rng.integers(-(1 << 62), 1 << 62, size=(5, 4, 3), dtype=np.int64)
    keep = A._Packed()
    desc = A.pack_bipolys(arr, keep)
    for k, d in enumerate(desc):
        assert (int(d["deg_x"]), int(d["deg_y"]), int(d["words"])) == (2, 3, 1)
        assert _decode(_read_words(d["coef"], 12), 1) == [int(v) for v in arr[k].ravel()]


def test_univariate_inputs_int64_and_wide():
    rng = random.Random(93)
    small = [[rng.randint(-(1 << 62), 1 << 62) for _ in range(rng.randint(1, 30))] for _ in range(20)] + [[], [0]]
    keep = A._Packed()
    desc = A.pack_upolys(small, keep)
    for p, d in zip(small, desc):
        n = max(len(p), 1)
        assert int(d["deg"]) == n - 1 and int(d["words"]) == 1
        assert _decode(_read_words(d["coef"], n), 1) == (list(p) or [0])
    # with a wide polynomial in the batch, each polynomial gets its own word count
    wide = small[:3] + [[_rand_int(rng, 200) for _ in range(7)]]
    desc = A.pack_upolys(wide, keep)
    for p, d in zip(wide, desc):
        W = int(d["words"])
        assert W == A._words_for(p or [0])
        assert _decode(_read_words(d["coef"], len(p) * W), W) == list(p)


def test_sign_magnitude_results_round_trip():
    rng = random.Random(94)
    polys = [[_rand_int(rng, rng.choice([1, 31, 32, 33, 64, 500])) for _ in range(rng.randint(1, 9))]
             for _ in range(30)]
    polys += [[0, 0], [], [5, 0, 0], [-(1 << 95)]]
    keep = A._Packed()
    arr = A.pack_bigpolys(polys, keep)
    for k, p in enumerate(polys):
        want = list(p)
        while want and want[-1] == 0:
            want.pop()
        b = arr[k]
        if not want:
            assert b.deg == -1
            continue
        assert b.deg == len(want) - 1
        assert b.limbs == max(1, max((abs(v).bit_length() + 31) // 32 for v in want))
        assert A.bigpoly_to_ints(b) == want


def test_bigpoly_to_ints_trims_and_reads_signs():
    mag = (C.c_uint32 * 6)(5, 0, 0, 1, 0, 0)            # 5, 2^32, 0 with two limbs each
    sign = (C.c_int8 * 3)(-1, 1, 0)
    b = N.BigPoly(2, 2, C.cast(mag, C.POINTER(C.c_uint32)), C.cast(sign, C.POINTER(C.c_int8)))
    assert A.bigpoly_to_ints(b) == [-5, 1 << 32]
    assert A.bigpoly_to_ints(N.BigPoly(-1, 0, None, None)) == []
