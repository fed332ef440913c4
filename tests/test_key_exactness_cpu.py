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
