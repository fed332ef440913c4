"""The min-search key of the packed check body, checked exhaustively on the CPU:
one saturating binary16 multiply-add fma.rn.sat(|u|, 2^-7, j 2^-11) forms
(16 |u| + j) 2^-11 clamped to 1, and the minima start at (16 Qm + 15) 2^-11.
The claim the kernels rest on: the decoded minimum of any set of positions has
the magnitude min(|u|, Qm) of the smallest, and the first position reaching it
wherever that magnitude is below Qm (where both minima saturate, A = B and the
position does not matter), for every Qm in [1, 127] and every |u| a binary16
posterior difference can take (< 2048).

fma.rn rounds the exact a b + c once; here the exact value (16 |u| + j) / 2048
is formed in float64 (exact) and rounded once to binary16 by numpy, which
rounds to nearest even like the hardware."""
import numpy as np

S7, S11 = 2.0 ** -7, 2.0 ** -11


def key(u_abs, j):
    exact = u_abs.astype(np.float64) * S7 + np.asarray(j, np.float64) * S11
    return np.clip(exact.astype(np.float16), np.float16(0), np.float16(1))


def decode(k):
    return np.rint(k.astype(np.float64) * 2048).astype(np.int64)


def test_single_key_every_qm_u_j():
    u = np.arange(2048)
    for j in range(16):
        k = key(u, j)
        for qm in range(1, 128):
            start = np.float16((16 * qm + 15) * S11)
            assert float(start) == (16 * qm + 15) * S11  # the start is exact
            got = decode(np.minimum(k, start))
            want = np.where(u <= qm, 16 * u + j, 16 * qm + 15)
            np.testing.assert_array_equal(got, want)
            # magnitude is min(|u|, Qm); the position is exact where |u| <= Qm
            np.testing.assert_array_equal(got >> 4, np.minimum(u, qm))


def test_two_minima_random_checks():
    """min1 / min2 over random checks (degrees 2..16) against the integer
    definition, with the saturated magnitudes at the ties."""
    rng = np.random.default_rng(0)
    for _ in range(3000):
        qm = int(rng.integers(1, 128))
        d = int(rng.integers(2, 17))
        u = np.abs(rng.integers(-int(rng.choice([4, 60, 300, 2047])), 2048, size=d))
        u = np.minimum(u, 2047)
        ks = [key(np.array([u[j]]), j)[0] for j in range(d)]
        K1 = K2 = np.float16((16 * qm + 15) * S11)
        for kj in ks:
            K2 = min(K2, max(K1, kj))
            K1 = min(K1, kj)
        k1, k2 = int(decode(np.array([K1]))[0]), int(decode(np.array([K2]))[0])
        sat = np.minimum(u, qm)
        order = sorted(range(d), key=lambda j: (sat[j], j))
        assert k1 >> 4 == sat[order[0]] and k2 >> 4 == sat[order[1]]
        if sat[order[0]] < qm:  # the position of the first minimum matters only then
            assert k1 & 15 == order[0]


def _fma16(a, b, c):
    """fma.rn on binary16: the exact a b + c (float64) rounded once."""
    return np.asarray(np.asarray(a, np.float64) * np.float64(b) + np.asarray(c, np.float64)).astype(np.float16)


def test_binary16_minima_decode_degree_le_8():
    """The ping-pong row pass (checks of degree <= 8) decodes a key K = (16 m +
    j) 2^-11, j <= 7, without leaving binary16: 1024 + 128 K rounds to 1024 + m
    (j / 16 < 1/2), 2048 K + (17408 - 16 (1024 + m)) is 1024 + j, and the offset
    rule max(1024 - beta + 128 K, 1024) is 1024 + max(m - beta, 0).  The minima
    start at (16 Qm + 7) 2^-11, so that a saturated key keeps j = 7.  Every Qm,
    m <= Qm, j <= 7 and offset beta <= 127."""
    j = np.arange(8)
    for qm in range(1, 128):
        start = np.float16((16 * qm + 7) * S11)
        assert float(start) == (16 * qm + 7) * S11
        m = np.arange(qm + 1)[:, None]
        K = ((16 * m + j) * S11).astype(np.float16)
        assert np.all(K.astype(np.float64) * 2048 == 16 * m + j)  # every key is exact
        assert np.all(K <= start)
        M1 = _fma16(K, 128, 1024)
        np.testing.assert_array_equal(M1.astype(np.int64), np.broadcast_to(1024 + m, K.shape))
        n16 = _fma16(M1, -16, 17408)
        np.testing.assert_array_equal(n16.astype(np.int64), np.broadcast_to(1024 - 16 * m, K.shape))
        Ip = _fma16(K, 2048, n16)
        np.testing.assert_array_equal(Ip.astype(np.int64), np.broadcast_to(1024 + j, K.shape))
        for beta in range(128):
            Ap = np.maximum(_fma16(K, 128, np.float16(1024 - beta)).astype(np.float64), 1024.0)
            np.testing.assert_array_equal(Ap, np.broadcast_to(1024 + np.maximum(m - beta, 0), K.shape))
        # the saturated start decodes to magnitude Qm
        assert int(_fma16(start, 128, 1024)) == 1024 + qm


def test_packed_normalized_halves():
    """The normalized rule floor(m num / 2^shift) on the integer halves of a
    pattern pair: ((m_lo | m_hi << 16) num mod 2^32) >> shift holds g(m_lo) in
    byte 0 and g(m_hi) in byte 2, for m <= 127 and every num <= 2^shift,
    shift <= 8 (no carry crosses the halves: m num < 2^16)."""
    m = np.arange(128, dtype=np.uint64)
    lo, hi = np.meshgrid(m, m, indexing="ij")
    for shift in range(9):
        for num in range(1, (1 << shift) + 1):
            w = (((lo | (hi << np.uint64(16))) * np.uint64(num)) & np.uint64(0xFFFFFFFF)) >> np.uint64(shift)
            np.testing.assert_array_equal(w & np.uint64(0xFF), (lo * np.uint64(num)) >> np.uint64(shift))
            np.testing.assert_array_equal((w >> np.uint64(16)) & np.uint64(0xFF), (hi * np.uint64(num)) >> np.uint64(shift))


def _pattern_pair(lo, hi):
    """32-bit word of two binary16 values (lo in bits 0-15)."""
    return (np.asarray(lo, np.float16).view(np.uint16).astype(np.uint64)
            | (np.asarray(hi, np.float16).view(np.uint16).astype(np.uint64) << np.uint64(16)))


def test_binary16_decode_shared_check_body():
    """The shared check body's binary16 decode (checks of degree <= 8 there; the
    form holds to degree 15): keys (16 |u| + j - 7) 2^-11 without a clamp, the
    minima started at (16 Qm + 7) 2^-11.  Every key of |u| <= 127 is exact,
    every |u| > Qm keys above the start (|u| up to 2300, rounded or not), and
    the decode gives 1025 + m (fma(K, 128, 1025)), 1017 + j (fma(K, 2048,
    fma(1025 + m, -16, 17424))) and the rule's pattern 1024 + g(m):
    max(fma(K, 128, 1025 - beta), 1025), then (pattern num - 0x64016401 num)
    >> shift on the 32-bit pair, bytes 0 and 2 behind 0x64."""
    j = np.arange(15)
    u_all = np.arange(2301)
    for qm in range(1, 128):
        start = np.float16((16 * qm + 7) * S11)
        keys = _fma16(u_all[:, None], S7, (j - 7) * S11)
        exact = (16 * u_all[:, None] + j - 7) * S11
        assert np.all(keys[:128].astype(np.float64) == exact[:128])
        assert np.all(keys[qm + 1:] > start)
        m = np.arange(qm + 1)[:, None]
        K = keys[:qm + 1]
        M1 = _fma16(K, 128, 1025)
        np.testing.assert_array_equal(M1.astype(np.int64), np.broadcast_to(1025 + m, K.shape))
        In = _fma16(K, 2048, _fma16(M1, -16, 17424))
        np.testing.assert_array_equal(In.astype(np.int64), np.broadcast_to(1017 + j, K.shape))
        for beta in (0, 1, 2, 5, 127):
            a = np.maximum(_fma16(K, 128, np.float16(1025 - beta)).astype(np.float64), 1025.0)
            np.testing.assert_array_equal(a, np.broadcast_to(1025 + np.maximum(m - beta, 0), K.shape))
        assert int(_fma16(start, 128, 1025)) == 1025 + qm
    # the integer step on pattern pairs 1025 + v (v <= 127) for the normalized rule
    v = np.arange(128)
    lo, hi = np.meshgrid(v, v, indexing="ij")
    w = _pattern_pair(1025.0 + lo, 1025.0 + hi)
    for shift in range(9):
        for num in sorted({1, 2, 3, (1 << shift) - 1, 1 << shift} - {0}):
            if num > (1 << shift):
                continue
            c2 = (-0x64016401 * num) % (1 << 32)
            x = ((w * np.uint64(num) + np.uint64(c2)) % np.uint64(1 << 32)) >> np.uint64(shift)
            np.testing.assert_array_equal(x & np.uint64(0xFF), (lo * num) >> shift)
            np.testing.assert_array_equal((x >> np.uint64(16)) & np.uint64(0xFF), (hi * num) >> shift)
