"""The integer algebra behind the folded FP16 tensor-core count, checked on the CPU.

The count pass appends one 16-column chunk to each operand row: rows carry the
constants 1, 2^11, 2^15 and columns the negated digits of h_q = ceil(|v_q|^2 / 2)
(h = q0 + 2^11 q1 + 2^22 q2 with q0, q1 < 2^11), so the FP32 accumulator holds
G - h_q with G = v_p . v_q.  Columns are grouped by the parity f of |v_q|^2 and
a pair is a neighbour iff G - h_q >= ceil((|v_p|^2 - T - f) / 2), decided as
sat(acc + 1 - thr_f) in float32.  These tests restate that reading in exact
integers and float32 and check, on random and extreme vectors, that

- every chunk entry is an integer FP16 holds exactly, and the chunk's products
  sum to -h_q;
- the magnitudes of all terms of the accumulation add up to at most 2^24 while
  3 max|v|^2 + 1 <= 2^25 (so every partial sum is exact in FP32, in any order);
- the parity threshold decides D <= T exactly, and so does the float32
  saturating decision;
- a padding column (zero vector, h = 2^24) is never counted.
"""
import numpy as np

FOLD_LIMIT = ((1 << 25) - 1) // 3
ROW_CHUNK = np.array([1, 2048, 32768], dtype=np.int64)


def col_chunk(beta: int, valid: bool = True) -> np.ndarray:
    h = (beta + 1) >> 1 if valid else 1 << 24
    return np.array([-(h & 2047), -((h >> 11) & 2047), -((h >> 22) << 7)], dtype=np.int64)


def fp16_exact(x: np.ndarray) -> bool:
    return bool(np.all(np.float16(x).astype(np.float64) == x))


def f32(x) -> np.float32:
    return np.float32(x)


def vectors(rng, d: int):
    """Pairs of centred unit vectors (v = u - 512): uniform, near the norm limit
    with the grid's extreme units, and near copies (small distances)."""
    kind = rng.integers(0, 3)
    if kind == 0:
        return rng.integers(-512, 512, d), rng.integers(-512, 512, d)
    if kind == 1:
        k = min(d, 42)
        vp = np.zeros(d, np.int64)
        vq = np.zeros(d, np.int64)
        vp[:k] = rng.choice([-512, 511], k)
        vq[:k] = rng.choice([-512, 511], k)
        if d > k:
            vp[k] = rng.integers(-418, 419)
            vq[k] = rng.integers(-418, 419)
        return vp, vq
    vp = rng.integers(-512, 512, d)
    vq = vp.copy()
    j = rng.integers(0, d)
    vq[j] = np.clip(vq[j] + rng.integers(-3, 4), -512, 511)
    return vp, vq


def test_chunk_entries_are_exact_and_sum_to_minus_h():
    rng = np.random.default_rng(1)
    assert fp16_exact(ROW_CHUNK)
    for beta in list(rng.integers(0, 1 << 24, 2000)) + [0, 1, 2047, 2048, (1 << 24) - 1, 1 << 24]:
        beta = int(beta)
        c = col_chunk(beta)
        assert fp16_exact(c)
        assert int((ROW_CHUNK * c).sum()) == -((beta + 1) >> 1)
    pad = col_chunk(0, valid=False)
    assert fp16_exact(pad) and int((ROW_CHUNK * pad).sum()) == -(1 << 24)


def test_fold_decides_the_predicate_exactly_within_the_norm_limit():
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(6000):
        d = int(rng.choice([16, 32, 48, 64]))
        vp, vq = vectors(rng, d)
        bp, bq = int((vp * vp).sum()), int((vq * vq).sum())
        if 3 * max(bp, bq) + 1 > (1 << 25):
            continue
        terms = np.concatenate([vp * vq, ROW_CHUNK * col_chunk(bq)])
        assert int(np.abs(terms).sum()) <= 1 << 24  # every partial sum is exact in FP32
        acc = int(terms.sum())
        D = int(((vp - vq) ** 2).sum())
        f = bq & 1
        for T in {0, 1, D - 1, D, D + 1, 218659, (1 << 24) - 2}:
            if not 0 <= T < (1 << 24):
                continue
            thr = (bp - T - f + 1) >> 1  # ceil((|v_p|^2 - T - f) / 2)
            assert (acc >= thr) == (D <= T)
            y = np.float32(f32(acc) + f32(1 - thr))  # the epilogue's saturating add
            assert (y >= 1) == (D <= T) and (y >= 1 or y <= 0)
            checked += 1
    assert checked > 10000


def test_padding_columns_are_never_counted():
    for bp in (0, 1, 5000, FOLD_LIMIT):
        for T in (0, 218659, (1 << 24) - 2):
            for f in (0, 1):
                thr = (bp - T - f + 1) >> 1
                assert np.float32(f32(-(1 << 24)) + f32(1 - thr)) <= 0


def test_the_norm_limit_is_tight_for_the_bound():
    # 3 b + 1 <= 2^25 is what (b_p + 2 b_q + 1) / 2 <= 2^24 needs when b_p = b_q = b
    assert 3 * FOLD_LIMIT + 1 <= (1 << 25) < 3 * (FOLD_LIMIT + 1) + 1
