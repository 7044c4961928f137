"""Pins of the oracle's encoder, rate matcher and de-rate-matcher: parity-check
identities of the constituent code, linearity, termination, bijection of the
circular buffer at rate 1/3, and HARQ combining.  CPU only."""
import numpy as np
import pytest

import synth

NULL = 2


def conv2(a, b):
    return np.convolve(a.astype(np.int64), b.astype(np.int64)) % 2


G0 = np.array([1, 0, 1, 1])  # 1 + D^2 + D^3
G1 = np.array([1, 1, 0, 1])  # 1 + D + D^3


def constituent_sequences(d0, d1, d2, K, pi, c):
    """(x, z) of encoder 1 and (x', z') of encoder 2 over K+3 steps, with the
    tail values read back from the round-robin multiplexing of the 12 tail bits."""
    t = [int([d0, d1, d2][i % 3][K + i // 3]) for i in range(12)]
    cz = np.where(c == NULL, 0, c).astype(np.int64)
    x1 = np.concatenate([cz, [t[0], t[2], t[4]]])
    z1 = np.concatenate([d1[:K].astype(np.int64), [t[1], t[3], t[5]]])
    x2 = np.concatenate([cz[pi], [t[6], t[8], t[10]]])
    z2 = np.concatenate([d2[:K].astype(np.int64), [t[7], t[9], t[11]]])
    return x1, z1, x2, z2


def encode_with_parity_from(orc, c):
    d0, d1, d2 = orc.turbo_encode_cb(c)
    return d0, d1, d2


@pytest.mark.parametrize("K,F", [(40, 0), (48, 8), (1056, 0), (6144, 0), (5824, 24)])
def test_encoder_parity_check_identity_and_termination(orc, K, F):
    # For an RSC with G = [1, g1/g0] started and terminated in state 0 the
    # sequences satisfy x(D) g1(D) = z(D) g0(D) exactly as polynomials.
    c = synth.bits(11, K, K).astype(np.uint8)
    c[:F] = NULL
    d0, d1, d2 = orc.turbo_encode_cb(c)
    assert np.all(d0[:F] == NULL) and np.all(d1[:F] == NULL)
    assert np.all(d0[F:K] == c[F:K])
    pi = orc.qpp(K)
    # recompute parity at filler positions: the encoder saw zeros there
    d1f = d1.copy()
    cz = np.where(c == NULL, 0, c)
    # parity of encoder 1 over the filler prefix is 0 (state stays 0 on zeros)
    d1f[:F] = 0
    x1, z1, x2, z2 = constituent_sequences(d0, d1f, d2, K, pi, c)
    assert np.array_equal(conv2(x1, G1), conv2(z1, G0))
    assert np.array_equal(conv2(x2, G1), conv2(z2, G0))
    assert np.array_equal(x2[:K], cz[pi])


def test_encoder_linear_and_zero(orc):
    K = 104
    a = synth.bits(3, 0, K)
    b = synth.bits(3, 1, K)
    da = orc.turbo_encode_cb(a)
    db = orc.turbo_encode_cb(b)
    dab = orc.turbo_encode_cb(a ^ b)
    for i in range(3):
        assert np.array_equal(dab[i], da[i] ^ db[i])
    dz = orc.turbo_encode_cb(np.zeros(K, np.uint8))
    assert all(not d.any() for d in dz)


def test_rate_one_third_is_bijection(orc):
    # E = 3(K+4) with rv 0 and no filler: every coded bit sent exactly once.
    K = 6144
    c = synth.bits(0, 99, K)
    d0, d1, d2 = orc.turbo_encode_cb(c)
    E = 3 * (K + 4)
    e = orc.rate_match_cb(d0, d1, d2, E, 0)
    assert e.sum() == d0.sum() + d1.sum() + d2.sum()
    llr = np.where(e == 0, 100, -100).astype(np.int8)
    r0, r1, r2, soft = orc.derm_cb(llr, K, 0, 0)
    for d, r in ((d0, r0), (d1, r1), (d2, r2)):
        assert np.array_equal(r, np.where(d == 0, 100, -100))


@pytest.mark.parametrize("K,F,E,rv", [(40, 0, 100, 0), (48, 8, 70, 2), (1056, 16, 4000, 3),
                                      (512, 0, 3000, 1), (5824, 0, 6642, 0), (40, 16, 500, 0)])
def test_derm_inverts_rate_matching(orc, K, F, E, rv):
    c = synth.bits(7, K, K).astype(np.uint8)
    c[:F] = NULL
    d0, d1, d2 = orc.turbo_encode_cb(c)
    e = orc.rate_match_cb(d0, d1, d2, E, rv)
    # bit selection walks w from k0 skipping <NULL>: rebuild that walk here
    Ncb, k0 = orc.ncb(K), orc.k0(K, rv)
    walk = []
    j = 0
    while len(walk) < E:
        st, di = orc.wpos_to_d(K, (k0 + j) % Ncb)
        if di >= 0 and not (st < 2 and di < F):
            walk.append((st, di))
        j += 1
    ds = (d0, d1, d2)
    assert [int(ds[st][di]) for st, di in walk] == e.tolist()
    vals = synth.randint(3, E, E, -40, 40).astype(np.int8)
    r = orc.derm_cb(vals, K, F, rv)
    acc = [np.zeros(K + 4, np.int64) for _ in range(3)]
    for (st, di), v in zip(walk, vals):
        acc[st][di] = max(-127, min(127, acc[st][di] + int(v)))
    acc[0][:F] = 127
    acc[1][:F] = 0
    for i in range(3):
        assert np.array_equal(r[i].astype(np.int64), acc[i])


def test_harq_combining_saturates_and_accumulates(orc):
    K, E = 512, 900
    v1 = synth.randint(4, 1, E, -127, 127).astype(np.int8)
    v2 = synth.randint(4, 2, E, -127, 127).astype(np.int8)
    _, _, _, soft = orc.derm_cb(v1, K, 0, 0)
    s1 = soft.copy()
    r = orc.derm_cb(v2, K, 0, 2, soft=soft)
    _, _, _, s2 = orc.derm_cb(v2, K, 0, 2)
    want = np.clip(s1.astype(np.int64) + s2.astype(np.int64), -127, 127)
    # v2 alone (rv 2, no repetition) touches each position at most once
    assert np.array_equal(r[3].astype(np.int64), want)
    # -128 inputs saturate to -127
    _, _, _, s3 = orc.derm_cb(np.full(E, -128, np.int8), K, 0, 0)
    assert s3.min() == -127
