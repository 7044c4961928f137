"""Pins of the oracle's PUSCH front stage: the Gold scrambling sequence, the
scrambling initialisation, descrambling and the data-only channel
interleaver (TS 36.211 Sec. 5.3.1 / 7.2, TS 36.212 Sec. 5.2.2.8; the
demultiplexing ahead of the decoder in the paper's Sec. IV-B).  The
specifications are not in this repository, so conformance of the sequence
values is unpinned; these tests pin what the algebra fixes."""
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "pusch_interleaver.txt")
MERSENNE31 = (1 << 31) - 1  # prime


def berlekamp_massey(s):
    """Shortest GF(2) linear recurrence of the bit sequence s: returns the
    connection polynomial as an int (bit i = coefficient of x^i, C(0) = 1)
    and its length L."""
    C, B = 1, 1
    L, m = 0, 1
    for n in range(len(s)):
        d = s[n]
        for i in range(1, L + 1):
            d ^= ((C >> i) & 1) & s[n - i]
        if d == 0:
            m += 1
        elif 2 * L <= n:
            T = C
            C ^= B << m
            L, B, m = n + 1 - L, T, 1
        else:
            C ^= B << m
            m += 1
    return C, L


def pmulmod(a, b, f, deg):
    """a * b mod f over GF(2) (ints as polynomials)."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if (a >> deg) & 1:
            a ^= f
    return r


def xpow(n, f, deg):
    """x^n mod f over GF(2)."""
    r, base = 1, 2
    while n:
        if n & 1:
            r = pmulmod(r, base, f, deg)
        base = pmulmod(base, base, f, deg)
        n >>= 1
    return r


def characteristic(conn, L):
    """The characteristic polynomial x^L C(1/x) of a connection polynomial."""
    return sum(((conn >> i) & 1) << (L - i) for i in range(L + 1))


def recovered_polys(orc):
    x1 = [int(v) for v in orc.gold(0, 200)]            # c_init = 0: x2 vanishes
    a = 0x1234567
    x2 = [int(v) for v in orc.gold(a, 200) ^ orc.gold(0, 200)]
    return berlekamp_massey(x1), berlekamp_massey(x2)


def test_gold_components_are_maximal_length_sequences(orc):
    # each component is an LFSR sequence of degree 31 whose characteristic
    # polynomial is primitive: x has order 2^31 - 1 modulo it (a prime, so
    # x^(2^31 - 1) = 1 suffices), i.e. the sequence has the maximal period
    for conn, L in recovered_polys(orc):
        assert L == 31
        f = characteristic(conn, L)
        assert f & 1 and (f >> 31) & 1
        assert xpow(MERSENNE31, f, 31) == 1
        assert xpow(1, f, 31) != 1


def test_gold_matches_the_specified_recurrences(orc):
    # recovered recurrences: x^31 + x^3 + 1 for x1, x^31 + x^3 + x^2 + x + 1 for x2
    (c1, L1), (c2, L2) = recovered_polys(orc)
    assert characteristic(c1, L1) == (1 << 31) | (1 << 3) | 1
    assert characteristic(c2, L2) == (1 << 31) | (1 << 3) | (1 << 2) | (1 << 1) | 1


@pytest.mark.parametrize("c_init", [0, 1, 0x1234567, (1 << 31) - 1, 1639431])
def test_gold_by_jump_ahead(orc, c_init):
    # c(n) = x1(n + 1600) + x2(n + 1600); a sequence with characteristic
    # polynomial f has x(n) = sum_j r_j x(j) with r = x^n mod f, so the
    # terms at n = 1600 + k follow from the initial states (x1: 1, 0, ..., 0;
    # x2: the bits of c_init) by polynomial exponentiation -- no stepping
    f1 = (1 << 31) | (1 << 3) | 1
    f2 = (1 << 31) | (1 << 3) | (1 << 2) | (1 << 1) | 1
    got = orc.gold(c_init, 64)
    for k in range(64):
        r1 = xpow(1600 + k, f1, 31)
        r2 = xpow(1600 + k, f2, 31)
        x1 = r1 & 1
        x2 = bin(r2 & c_init).count("1") & 1
        assert got[k] == x1 ^ x2, k


def test_gold_is_affine_in_c_init(orc):
    a, b = 0x2ABCDEF, 0x1357913
    ga, gb, g0 = orc.gold(a, 5000), orc.gold(b, 5000), orc.gold(0, 5000)
    assert np.array_equal(orc.gold(a ^ b, 5000), ga ^ gb ^ g0)
    assert 0.45 < ga.mean() < 0.55


def test_pusch_cinit_fields(orc):
    # n_RNTI 2^14 + q 2^13 + floor(n_s / 2) 2^9 + N_ID^cell, by hand
    assert orc.pusch_cinit(100, 0, 4, 7) == 1639431
    assert orc.pusch_cinit(65535, 1, 19, 503) == 65535 * 16384 + 8192 + 9 * 512 + 503


def golden_cases():
    out = []
    for line in open(GOLD):
        if line.startswith("case"):
            v = [int(x) for x in line.split()[1:]]
            out.append((v[0], v[1], v[2], v[3:]))
    return out


@pytest.mark.parametrize("G,QmNL,ncol,order", golden_cases())
def test_channel_interleaver_golden(orc, G, QmNL, ncol, order):
    # mark every bit with the index of its symbol and follow it through
    marks = (np.arange(G) // QmNL).astype(np.uint8)
    tx = orc.channel_interleave(marks, QmNL, ncol).reshape(-1, QmNL)
    assert (tx == tx[:, :1]).all()  # a symbol's bits stay together
    assert list(tx[:, 0]) == order


@pytest.mark.parametrize("G,QmNL", [(86400, 6), (28800, 2), (172800, 12), (1728, 4)])
def test_channel_interleaver_is_a_bijection(orc, G, QmNL):
    # bits of distinct positions end up in distinct positions: interleave the
    # position index bit by bit (17 bit planes)
    pos = np.zeros(G, dtype=np.int64)
    for bit in range(18):
        plane = ((np.arange(G) >> bit) & 1).astype(np.uint8)
        pos |= orc.channel_interleave(plane, QmNL).astype(np.int64) << bit
    assert np.array_equal(np.sort(pos), np.arange(G))
    # the bits of one symbol stay together and in order
    assert np.array_equal(pos % QmNL, np.arange(G) % QmNL)


def test_pusch_rx_inverts_tx(orc):
    # transmit: interleave + scramble; receive: descramble + de-interleave
    G, QmNL = 4320, 6
    e = synth.bits(9, 1, G).astype(np.uint8)
    c_init = orc.pusch_cinit(4711, 0, 7, 101)
    tx = orc.pusch_tx(e, QmNL, c_init)
    llr = np.where(tx == 0, 90, -90).astype(np.int8)
    back = orc.pusch_rx(llr, QmNL, c_init)
    assert np.array_equal(back, np.where(e == 0, 90, -90).astype(np.int8))
    # the scrambling really changes the transmitted bits
    assert 0.4 < np.mean(tx != orc.channel_interleave(e, QmNL)) < 0.6


def test_descrambling_is_an_involution(orc):
    # one column: the interleaver is the identity and pusch_rx only
    # descrambles; twice gives the input back (-128 reads as -127)
    llr = synth.randint(5, 2, 3000, -128, 127).astype(np.int8)
    c_init = 0x5A5A5A5
    once = orc.pusch_rx(llr, 2, c_init, ncol=1)
    twice = orc.pusch_rx(once, 2, c_init, ncol=1)
    assert np.array_equal(twice, np.maximum(llr, -127))
    flip = orc.gold(c_init, 3000).astype(bool)
    assert np.array_equal(once, np.where(flip, -np.maximum(llr, -127), np.maximum(llr, -127)))
