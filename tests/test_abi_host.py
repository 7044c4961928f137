"""The C-ABI library loads without a GPU, exports every entry point that
include/crnt.h declares, its structs match the header's sizes, and its
host-side parameter arithmetic agrees with the oracle (independent code)."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "crnt.h")


def declared_functions():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(crnt_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(crnt_lib):
    names = declared_functions()
    assert "crnt_decode_batch" in names and len(names) >= 18
    lib = crnt_lib.load()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(crnt_lib.SIGNATURES)


def test_struct_sizes(crnt_lib):
    assert ctypes.sizeof(crnt_lib.TbParams) == 40
    assert ctypes.sizeof(crnt_lib.Config) == 32
    assert ctypes.sizeof(crnt_lib.TbResult) == 96
    assert ctypes.sizeof(crnt_lib.CbLayout) == 40
    assert ctypes.sizeof(crnt_lib.PlanInfo) == 64
    assert ctypes.sizeof(crnt_lib.CbTiming) == 48
    assert ctypes.sizeof(crnt_lib.ServeStats) == 128
    assert crnt_lib.version() == 2
    assert crnt_lib.strerror(-1) == "invalid argument"


def test_qpp_table_matches_oracle(crnt_lib, orc):
    for K in orc.k_table():
        assert crnt_lib.qpp_params(K) == orc.qpp_params(K), K
    with pytest.raises(crnt_lib.CrntError):
        crnt_lib.qpp_params(41)


def test_tb_layout_matches_oracle(crnt_lib, orc):
    rng_A = 8 * synth.randint(9, 0, 300, 2, 9422)
    cases = [(6120, 18444, 2, 1, 0), (75376, 86400, 6, 1, 0), (16, 132, 2, 1, 3), (6128, 13000, 2, 2, 2)]
    for t, A in enumerate(rng_A):
        Qm = (2, 4, 6)[t % 3]
        G = Qm * int(np.ceil((A + 24) * 1.3 / Qm))
        cases.append((int(A), G, Qm, 1 + (t % 2), t % 4))
    for A, G, Qm, NL, rv in cases:
        G = G - G % (Qm * NL)
        lay = crnt_lib.tb_layout(dict(A=A, G=G, Qm=Qm, NL=NL, rv=rv))
        s = orc.segment(A + 24)
        assert len(lay) == s["C"]
        eoff = soff = 0
        for r, c in enumerate(lay):
            K = s["Km"] if r < s["Cm"] else s["Kp"]
            assert c["K"] == K and c["F"] == (s["F"] if r == 0 else 0)
            assert c["E"] == orc.e_r(G, Qm, NL, s["C"], r)
            assert c["k0"] == orc.k0(K, rv) and c["Ncb"] == orc.ncb(K)
            assert c["llr_offset"] == eoff and c["soft_offset"] == soff
            assert c["crc_b"] == (s["C"] > 1)
            assert 1 <= c["P"] <= min(128, max(1, K // 8)) and c["W"] == -(-K // c["P"])
            eoff += c["E"]
            soff += c["Ncb"]
        assert eoff == G


def test_segmentation_every_tb_size(crnt_lib, orc):
    # every TB size the library accepts (A = 16..75376, multiples of 8): the
    # library's CB sizes and filler count equal the oracle's segmentation
    for A in range(16, 75377, 8):
        lay = crnt_lib.tb_layout(dict(A=A, G=6 * (3 * A + 400), Qm=6))
        s = orc.segment(A + 24)
        assert len(lay) == s["C"], A
        for r, c in enumerate(lay):
            assert c["K"] == (s["Km"] if r < s["Cm"] else s["Kp"]), (A, r)
            assert c["F"] == (s["F"] if r == 0 else 0), (A, r)


def test_invalid_params_rejected(crnt_lib):
    bad = [dict(A=15, G=100), dict(A=17, G=100), dict(A=75384, G=100000), dict(A=100, G=101),
           dict(A=100, G=300, Qm=3), dict(A=100, G=300, rv=4), dict(A=100, G=300, max_iter=0),
           dict(A=100, G=300, NL=3)]
    for b in bad:
        with pytest.raises(crnt_lib.CrntError) as ei:
            crnt_lib.tb_layout(b)
        assert ei.value.code == crnt_lib.EINVAL


def test_tune_table_drives_p0_windows(crnt_lib):
    # the process-wide window table: P = 0 requests take its entry for their
    # K (clamped like a requested P); explicit P ignores it; 0 = built-in
    ks = [crnt_lib.tb_layout(dict(A=6120, G=18444))[0]["K"]]
    assert ks == [6144]
    old = crnt_lib.tune_get()
    try:
        t = [0] * crnt_lib.NUM_K
        t[-1] = 100                       # K = 6144
        t[0] = 9                          # K = 40: clamped to K / 8 = 5
        crnt_lib.tune_set(t)
        assert crnt_lib.tune_get() == t
        assert crnt_lib.tb_layout(dict(A=6120, G=18444))[0]["P"] == 100
        assert crnt_lib.tb_layout(dict(A=6120, G=18444, P=64))[0]["P"] == 64
        assert crnt_lib.tb_layout(dict(A=16, G=132))[0]["P"] == 5
        with pytest.raises(crnt_lib.CrntError):
            crnt_lib.tune_set([200] * crnt_lib.NUM_K)
        arr = (ctypes.c_uint8 * 10)()
        assert crnt_lib.load().crnt_tune_set(arr, 10) == crnt_lib.EINVAL
        crnt_lib.tune_set([0] * crnt_lib.NUM_K)
        assert crnt_lib.tb_layout(dict(A=6120, G=18444))[0]["P"] == 128
    finally:
        crnt_lib.tune_set(old)


def test_radix_table_get_set(crnt_lib):
    # the forward-recursion radix table: 2 by default, 4 where selected; it
    # changes no decoded value, so crnt_tb_layout does not depend on it
    old = crnt_lib.tune_radix_get()
    try:
        crnt_lib.tune_radix_set([0] * crnt_lib.NUM_K)
        assert crnt_lib.tune_radix_get() == [2] * crnt_lib.NUM_K
        lay2 = crnt_lib.tb_layout(dict(A=75376, G=86400, Qm=6))
        t = [2] * crnt_lib.NUM_K
        t[-1] = 4
        t[100] = 4
        crnt_lib.tune_radix_set(t)
        assert crnt_lib.tune_radix_get() == t
        assert crnt_lib.tb_layout(dict(A=75376, G=86400, Qm=6)) == lay2
        for bad in (1, 3, 8, 255):
            with pytest.raises(crnt_lib.CrntError):
                crnt_lib.tune_radix_set([bad] * crnt_lib.NUM_K)
        assert crnt_lib.tune_radix_get() == t       # a refused table changes nothing
        arr = (ctypes.c_uint8 * 10)()
        assert crnt_lib.load().crnt_tune_radix_set(arr, 10) == crnt_lib.EINVAL
        assert crnt_lib.load().crnt_tune_radix_get(None, 188) == crnt_lib.EINVAL
    finally:
        crnt_lib.tune_radix_set(old)


@pytest.mark.parametrize("K,F,P,rv", [(40, 0, 1, 0), (40, 8, 5, 1), (512, 24, 9, 2),
                                      (1024, 0, 21, 3), (5824, 16, 121, 1),
                                      (6144, 0, 128, 0), (6144, 56, 128, 3), (2112, 40, 7, 2)])
def test_derm_map_matches_oracle_rate_matching(orc, crnt_lib, K, F, P, rv):
    # the decoder's de-rate-matching map against the oracle's circular buffer:
    # with one distinct LLR per non-NULL position (E = Nv), each received LLR k
    # must land exactly where the map says, and the map must cover every
    # non-NULL bit of the three streams once (filler bits of streams 0 and 1
    # excepted)
    Nv = 3 * (K + 4) - 2 * F
    rng = np.random.default_rng(K * 131 + F * 7 + rv)
    e = rng.integers(-127, 128, Nv).astype(np.int8)
    d = orc.derm_cb(e, K, F, rv)[:3]
    m = np.array(crnt_lib.derm_map(K, P, F, rv), dtype=np.int64)
    assert len(m) == Nv
    Pr = max(1, min(P, K // 8, 128))
    W = -(-K // Pr)
    Pe = -(-K // W)
    tp = W * Pe
    dst, pos = m & 0xFFFF, m >> 16
    tail = dst >= 3 * tp
    s = np.where(tail, (dst - 3 * tp) % 3, dst // tp)
    t = dst % tp
    di = np.where(tail, K + (dst - 3 * tp) // 3, (t % Pe) * W + t // Pe)
    got = np.array([d[si][x] for si, x in zip(s, di)], dtype=np.int8)
    assert np.array_equal(got, e)
    hit = set(zip(s.tolist(), di.tolist()))
    assert len(hit) == Nv
    want = {(si, x) for si in range(3) for x in range(K + 4) if not (si < 2 and x < F)}
    assert hit == want
    assert len(set(pos.tolist())) == Nv and pos.max() < 96 * ((K + 4 + 31) // 32)
    with pytest.raises(crnt_lib.CrntError):
        crnt_lib.derm_map(K, P, F + 4, rv)


@pytest.mark.parametrize("K,P", [(40, 1), (40, 5), (512, 9), (1024, 21), (2112, 7),
                                 (5824, 121), (6144, 128), (6144, 100)])
def test_interleaver_map_matches_oracle_qpp(orc, crnt_lib, K, P):
    # the decoder's interleaved-pass address table against the oracle's QPP
    # permutation: step j of window p reads natural position PI(p W + j),
    # stored at its transposed shared-memory index
    pi = np.asarray(orc.qpp(K), dtype=np.int64)
    m = np.array(crnt_lib.interleaver_map(K, P), dtype=np.int64)
    Pr = max(1, min(P, K // 8, 128))
    W = -(-K // Pr)
    Pe = -(-K // W)
    m = m[:W * Pe].reshape(Pe, W)
    for p in range(Pe):
        n = min(W, K - p * W)
        q, t = m[p, :n] >> 16, m[p, :n] & 0xFFFF
        assert np.array_equal(q, pi[p * W:p * W + n]), p
        assert np.array_equal(t, (q % W) * Pe + q // W), p
        assert not m[p, n:].any()


def test_load_generator_built_and_checks_its_arguments(crnt_lib):
    # the native load generator is a client of the C ABI only; argument
    # errors end it with status 2 before it touches a GPU
    import subprocess
    from paper_1905_01141_gb300 import build as crnt_build
    assert os.path.exists(crnt_build.LOADGEN)
    r = subprocess.run([crnt_build.LOADGEN], capture_output=True, text=True, timeout=60)
    assert r.returncode == 2 and "usage" in r.stderr
    r = subprocess.run([crnt_build.LOADGEN, "--threads", "2", "--poisson", "/nonexistent", "8",
                        "1", "0.1", "1", "4"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 2


def test_pusch_parameters_validated(crnt_lib):
    # CRNT_F_PUSCH: G a multiple of Qm NL n_symb, n_symb at most 14, 31-bit
    # c_init, G at most 196608 (host-side check, no GPU)
    F = crnt_lib.F_PUSCH
    for tb in (dict(A=1000, G=1202, Qm=2, flags=F),
               dict(A=1000, G=1440, Qm=2, n_symb=15, flags=F),
               dict(A=1000, G=1440, Qm=2, c_init=1 << 31, flags=F),
               dict(A=75376, G=196608 + 144 * 2, Qm=2, n_symb=1, flags=F)):
        with pytest.raises(crnt_lib.CrntError) as ei:
            crnt_lib.tb_layout(tb)
        assert ei.value.code == crnt_lib.EINVAL
    assert len(crnt_lib.tb_layout(dict(A=1000, G=1440, Qm=2, flags=F))) == 1
    assert len(crnt_lib.tb_layout(dict(A=1000, G=1202, Qm=2))) == 1  # no flag: any G
