"""Seeded synthetic workload generator shared by the tests and the benchmark.

This module holds none of the decoder's arithmetic: it draws payload bits,
channel noise and workload shapes, and it turns coded bits (produced by
whichever encoder the caller uses) into quantised int8 LLRs through a
modulator, an AWGN channel and a max-log demapper.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value i of stream (seed, sid) is mix64(key + (i + 1) * 0x9E3779B97F4A7C15)
with key = mix64(seed * 0x100000001B3 + sid).  Normals use Box-Muller on two
53-bit uniforms.

Workload recipes (sizes of the decoding workloads this library is measured
on):
  * single_cb      : A=6120 payload bits (+CRC24A -> one K=6144 CB), rate 1/3
                     without puncturing (E=18444), BPSK, AWGN at Eb/N0 dB.
  * subframe_20mhz : A=75376 (13 CBs of K=5824), G=86400 (100 PRB x 144 RE
                     x 6 bits), 64QAM, AWGN at SNR dB.
  * tti_batch      : cells x UEs TBs, A uniform over multiples of 8 in
                     [16, 75376], Qm in {2,4,6} and G drawn so that the code
                     rate stays <= 0.93 inside 100 PRB, SNR within +-3 dB of
                     a threshold for the (Qm, rate) pair: the capacity SNR plus
                     a gap measured for this decoder (about 10 % BLER there).
"""
import math

import numpy as np

_GOLD = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, sid):
    with np.errstate(over="ignore"):
        k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * np.uint64(0x100000001B3) + np.uint64(sid)
    return _mix64(k)


def u64(seed, sid, n, start=0):
    """n raw 64-bit draws of stream (seed, sid), starting at counter ``start``."""
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_key(seed, sid) + i * _GOLD)


def uniform01(seed, sid, n):
    """Uniforms in (0, 1]."""
    return ((u64(seed, sid, n) >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def bits(seed, sid, n):
    return (u64(seed, sid, n) >> np.uint64(63)).astype(np.uint8)


def normal(seed, sid, n):
    m = (n + 1) // 2
    u1 = uniform01(seed, sid, m)
    u2 = uniform01(seed, sid + 0x5A5A, m)
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    return np.concatenate([r * np.cos(t), r * np.sin(t)])[:n]


def randint(seed, sid, n, lo, hi):
    """Integers uniform in [lo, hi] (inclusive), by rejection-free scaling."""
    span = hi - lo + 1
    x = u64(seed, sid, n) >> np.uint64(11)
    return lo + ((x.astype(np.float64) * span) / 9007199254740992.0).astype(np.int64)


# ------------------------------------------------------------ channel model
def _pam_levels(m):
    """Gray-labelled PAM with 2**m levels; bit 0 picks the sign (0 -> +),
    the remaining bits pick the magnitude index through a binary-reflected
    Gray code.  Returns levels[label] for label = b0 b1 ... (b0 MSB)."""
    M = 1 << m
    lv = np.zeros(M)
    for lab in range(M):
        b = [(lab >> (m - 1 - i)) & 1 for i in range(m)]
        sign = 1.0 - 2.0 * b[0]
        g = 0
        for i in range(1, m):
            g = (g << 1) | b[i]
        j = 0
        while g:  # Gray -> binary
            j ^= g
            g >>= 1
        lv[lab] = sign * (2 * j + 1)
    return lv


def modulate(cbits, Qm):
    """Coded bits -> complex symbols with unit average energy.  Bits 2i of a
    symbol's label go to I, bits 2i+1 to Q (Qm = 1 means BPSK on I)."""
    cbits = np.asarray(cbits, dtype=np.int64)
    if Qm == 1:
        return (1.0 - 2.0 * cbits).astype(np.complex128)
    m = Qm // 2
    lv = _pam_levels(m)
    norm = math.sqrt(np.mean(lv ** 2) * 2)
    sym = cbits.reshape(-1, Qm)
    li = np.zeros(len(sym), dtype=np.int64)
    lq = np.zeros(len(sym), dtype=np.int64)
    for i in range(m):
        li = (li << 1) | sym[:, 2 * i]
        lq = (lq << 1) | sym[:, 2 * i + 1]
    return (lv[li] + 1j * lv[lq]) / norm


def demap_maxlog(y, Qm, sigma2):
    """Max-log LLRs log P(0)/P(1) for every bit, sigma2 = noise variance per
    real dimension."""
    if Qm == 1:
        return 2.0 * y.real / sigma2
    m = Qm // 2
    lv = _pam_levels(m)
    norm = math.sqrt(np.mean(lv ** 2) * 2)
    lv = lv / norm
    M = len(lv)
    out = np.zeros((len(y), Qm))
    for dim, comp in ((0, y.real), (1, y.imag)):
        d2 = (comp[:, None] - lv[None, :]) ** 2
        for i in range(m):
            bit = np.array([(lab >> (m - 1 - i)) & 1 for lab in range(M)])
            d0 = d2[:, bit == 0].min(axis=1)
            d1 = d2[:, bit == 1].min(axis=1)
            out[:, 2 * i + dim] = (d1 - d0) / (2.0 * sigma2)
    return out.reshape(-1)


def quantise(llr, scale=8.0):
    """LLR -> int8 with 3 fractional bits: round half away from zero, then
    saturate to [-127, 127]."""
    v = np.asarray(llr) * scale
    r = np.sign(v) * np.floor(np.abs(v) + 0.5)
    return np.clip(r, -127, 127).astype(np.int8)


def channel_llrs(cbits, Qm, sigma2, seed, sid):
    """Modulate coded bits, add AWGN (variance sigma2 per real dimension),
    demap and quantise to int8."""
    x = modulate(cbits, Qm)
    n = normal(seed, sid, 2 * len(x))
    y = x + math.sqrt(sigma2) * (n[0::2] + 1j * n[1::2])
    return quantise(demap_maxlog(y, Qm, sigma2))


def sigma2_ebn0(ebn0_db, rate):
    """BPSK with unit symbol energy: sigma^2 = 1 / (2 R Eb/N0)."""
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def sigma2_snr(snr_db):
    """Unit-energy complex symbols: sigma^2 per real dimension = 1/(2 SNR)."""
    return 1.0 / (2.0 * 10.0 ** (snr_db / 10.0))


# ------------------------------------------------------------ workloads
def tti_batch(seed, n_tb=320, amin=16, amax=75376):
    """Shapes of one TTI of the batched uneven load: list of dicts with A, G,
    Qm, snr_db.  40 cells x 8 UEs gives n_tb = 320."""
    A = 8 * randint(seed, 1, n_tb, amin // 8, amax // 8)
    rate_u = uniform01(seed, 2, n_tb)
    snr_u = uniform01(seed, 3, n_tb)
    out = []
    for t in range(n_tb):
        a = int(A[t])
        need = (a + 24) / (14400.0 * 0.93)
        Qm = 2 if need <= 2 else (4 if need <= 4 else 6)
        rmin = max(1.0 / 3.0, (a + 24) / (14400.0 * Qm))
        r = rmin + (0.93 - rmin) * float(rate_u[t]) if rmin < 0.93 else 0.93
        G = Qm * int(math.ceil((a + 24) / (r * Qm)))
        G = min(G, 14400 * Qm)
        r_eff = (a + 24) / G
        # threshold: capacity SNR plus an empirical gap of this decoder (max
        # 6 iterations) that grows with the modulation order and at high rate
        gap = 2.0 + 0.35 * (Qm - 2) + 10.0 * max(0.0, r_eff - 0.75)
        snr_th = 10.0 * math.log10(2.0 ** (r_eff * Qm) - 1.0) + gap
        out.append(dict(A=a, G=G, Qm=Qm, snr_db=snr_th + 6.0 * float(snr_u[t]) - 3.0))
    return out


def pusch_batch(seed, n_tb=320, amin=16, amax=75376):
    """Shapes of a TTI whose TBs arrive in PUSCH order: the TTI shapes with G
    rounded up to whole PRBs (144 resource elements of 12 SC-FDMA data
    symbols: G a multiple of 144 Qm, at most 100 PRBs), plus a seeded 31-bit
    scrambling initialisation per TB (c_init) and the interleaver's 12
    columns."""
    out = []
    cinit = randint(seed, 9, n_tb, 0, (1 << 31) - 1)
    for t, s in enumerate(tti_batch(seed, n_tb=n_tb, amin=amin, amax=amax)):
        per = 144 * s["Qm"]
        G = min(100 * per, per * int(math.ceil(s["G"] / per)))
        out.append(dict(A=s["A"], G=G, Qm=s["Qm"], snr_db=s["snr_db"], c_init=int(cinit[t]),
                        n_symb=12))
    return out
