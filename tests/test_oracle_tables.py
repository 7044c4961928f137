"""Pins of the oracle's tables and parameter arithmetic against what the
mathematics and published values fix (CRC, code-block sizes, QPP,
segmentation, rate-matching parameters).  CPU only."""
import math
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "params.txt")


def golden():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        out[k] = int(v, 0)
    return out


# ------------------------------------------------------------------ CRC
def poly_mod(num, g):
    """GF(2) polynomial remainder with Python ints (bit i = coeff of x^i)."""
    dg = g.bit_length() - 1
    while num and num.bit_length() - 1 >= dg:
        num ^= g << (num.bit_length() - 1 - dg)
    return num


G24A = (1 << 24) | 0x864CFB
G24B = (1 << 24) | 0x800063


def test_crc_published_check_values(orc):
    g = golden()
    msg = np.unpackbits(np.frombuffer(b"123456789", dtype=np.uint8))
    assert orc.crc24(msg, "A") == g["crc24a_check"]
    assert orc.crc24(msg, "B") == g["crc24b_check"]


@pytest.mark.parametrize("kind,g", [("A", G24A), ("B", G24B)])
def test_crc_is_polynomial_remainder(orc, kind, g):
    # crc(m) = m(x) x^24 mod g(x), computed here by long division on ints.
    for n in (1, 7, 24, 100, 333):
        m = synth.bits(5, n, n)
        val = int("".join(map(str, m)), 2)
        assert orc.crc24(m, kind) == poly_mod(val << 24, g)


@pytest.mark.parametrize("kind", ["A", "B"])
def test_crc_codeword_divisible_linear_leading_zeros(orc, kind):
    for n in (16, 40, 6120):
        a = synth.bits(1, n, n)
        b = synth.bits(2, n, n)
        ca = orc.crc24(a, kind)
        par = np.array([(ca >> (23 - i)) & 1 for i in range(24)], dtype=np.uint8)
        assert orc.crc24(np.concatenate([a, par]), kind) == 0
        assert orc.crc24(a ^ b, kind) == ca ^ orc.crc24(b, kind)
        assert orc.crc24(np.concatenate([np.zeros(37, np.uint8), a]), kind) == ca
    assert orc.crc24(np.zeros(500, np.uint8), kind) == 0


# ------------------------------------------------------------------ K table / QPP
def test_k_table_closed_form(orc):
    ks = orc.k_table()
    want = (list(range(40, 513, 8)) + list(range(528, 1025, 16)) + list(range(1056, 2049, 32))
            + list(range(2112, 6145, 64)))
    assert ks == want and len(ks) == 188


def _prime_factors(n):
    f, p = set(), 2
    while p * p <= n:
        while n % p == 0:
            f.add(p)
            n //= p
        p += 1
    if n > 1:
        f.add(n)
    return f


def test_qpp_rows_are_permutations(orc):
    for K in orc.k_table():
        f1, f2 = orc.qpp_params(K)
        # Sun & Takeshita permutation-polynomial conditions for 4 | K.
        assert f1 % 2 == 1 and f2 % 2 == 0
        for p in _prime_factors(K):
            assert f2 % p == 0 and f1 % p != 0
        i = np.arange(K, dtype=np.int64)
        pi = (f1 * i + f2 * i * i) % K
        assert len(np.unique(pi)) == K
        # parity preserving (f1 odd, f2 even): PI(i) = i mod 2
        assert np.all(pi % 2 == i % 2)
    pi40 = orc.qpp(40)
    assert sorted(pi40.tolist()) == list(range(40)) and pi40[0] == 0 and pi40[1] == (3 + 10) % 40


# ------------------------------------------------------------------ segmentation
def test_segmentation_worked_configs(orc):
    g = golden()
    s1 = orc.segment(g["cfg1_A"] + 24)
    assert (s1["B"], s1["C"], s1["Kp"], s1["F"]) == (g["cfg1_B"], g["cfg1_C"], g["cfg1_K"],
                                                     g["cfg1_F"])
    s2 = orc.segment(g["cfg2_A"] + 24)
    assert (s2["B"], s2["C"], s2["Bp"], s2["Kp"], s2["Cm"], s2["F"]) == (
        g["cfg2_B"], g["cfg2_C"], g["cfg2_Bp"], g["cfg2_K"], 0, g["cfg2_F"])
    s = orc.segment(16 + 24)
    assert (s["C"], s["Kp"], s["F"]) == (1, 40, 0)


def test_segmentation_invariants_exhaustive(orc):
    ks = orc.k_table()
    for A in range(16, 75377, 8):
        B = A + 24
        s = orc.segment(B)
        C, L = s["C"], s["L"]
        if B <= 6144:
            assert C == 1 and L == 0 and s["Bp"] == B
        else:
            assert L == 24 and C == math.ceil(B / 6120) and s["Bp"] == B + 24 * C
        # K+ is the smallest table size with C * K+ >= B'
        assert s["Kp"] in ks and C * s["Kp"] >= s["Bp"]
        idx = ks.index(s["Kp"])
        assert idx == 0 or C * ks[idx - 1] < s["Bp"]
        assert s["Cp"] + s["Cm"] == C
        if C > 1:
            assert s["Km"] == ks[idx - 1]
        # every bit lands in exactly one CB: sum K_r = B' + F, F < K gap
        assert s["Cp"] * s["Kp"] + s["Cm"] * s["Km"] == s["Bp"] + s["F"]
        gap = s["Kp"] - (ks[idx - 1] if idx else 0)
        assert 0 <= s["F"] < gap


# ------------------------------------------------------------------ rate matching parameters
def test_rate_matching_parameters(orc):
    g = golden()
    assert orc.ncb(g["cfg1_K"]) == g["cfg1_Ncb"] == 3 * 32 * g["cfg1_R"]
    assert orc.k0(g["cfg1_K"], 0) == g["cfg1_k0_rv0"]
    assert orc.ncb(g["cfg2_K"]) == g["cfg2_Ncb"] == 3 * 32 * g["cfg2_R"]
    assert orc.k0(g["cfg2_K"], 0) == g["cfg2_k0_rv0"]
    Es = [orc.e_r(g["cfg2_G"], 6, 1, 13, r) for r in range(13)]
    assert Es.count(g["cfg2_Er_small"]) == g["cfg2_Er_small_count"]
    assert Es.count(g["cfg2_Er_large"]) == g["cfg2_Er_large_count"]
    assert Es == sorted(Es) and sum(Es) == g["cfg2_G"]
    assert orc.e_r(18444, 2, 1, 1, 0) == g["cfg1_E"] == 3 * (g["cfg1_K"] + 4)


def test_e_r_sums_to_G(orc):
    for C in (1, 2, 5, 13):
        for Qm in (2, 4, 6):
            for NL in (1, 2):
                for G in (Qm * NL * 1000, Qm * NL * 4321):
                    Es = [orc.e_r(G, Qm, NL, C, r) for r in range(C)]
                    assert sum(Es) == G and all(e % (Qm * NL) == 0 for e in Es)
                    assert max(Es) - min(Es) <= Qm * NL


def test_column_permutation_is_bit_reversal(orc):
    assert orc.colperm() == [int(format(j, "05b")[::-1], 2) for j in range(32)]


@pytest.mark.parametrize("K", [40, 48, 512, 1056, 5824, 6144])
def test_circular_buffer_is_bijection_onto_d(orc, K):
    D = K + 4
    R = math.ceil(D / 32)
    ND = 32 * R - D
    seen = set()
    nulls = 0
    for w in range(orc.ncb(K)):
        st, d = orc.wpos_to_d(K, w)
        if d < 0:
            nulls += 1
            continue
        assert 0 <= d < D and (st, d) not in seen
        seen.add((st, d))
    assert nulls == 3 * ND and len(seen) == 3 * D
    # v0 starts with the dummy column entries of permuted column 0
    assert [orc.wpos_to_d(K, w)[1] for w in range(R)][0] == (-1 if ND > 0 else 0)


def test_scale_ext_values(orc):
    # (3x)>>2 with an arithmetic shift = floor(3x/4)
    for x, want in [(-1, -1), (-3, -3), (5, 3), (4, 3), (-4, -3), (0, 0), (1, 0),
                    (32767, 24575), (-32768, -24576)]:
        assert orc.scale_ext(x) == want
    for x in range(-600, 600):
        assert orc.scale_ext(x) == math.floor(3 * x / 4)
