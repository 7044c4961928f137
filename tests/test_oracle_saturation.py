"""Pins of the oracle's int16 saturation semantics (the fixed-point reading
of the max-log-MAP SISO, Sec. IV-B "Decoding function"): a hand-worked pass
where saturation decides several outputs (tests/golden/siso_saturation.txt),
and the shift invariance that normalising before saturating implies."""
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "siso_saturation.txt")


def load_golden():
    g = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        g[k] = [int(x) for x in v]
    return g


def test_saturation_golden(orc):
    g = load_golden()
    K, P = g["K"][0], g["P"][0]
    a = np.zeros((P, 8), dtype=np.int16)
    b = np.zeros((P, 8), dtype=np.int16)
    a[1], a[2] = g["aseed1"], g["aseed2"]
    b[0], b[1] = g["bseed0"], g["bseed1"]
    lam, le, an, bn = orc.siso_seeded(g["Ls"], g["Lp"], g["La"], g["ts"], g["tp"], P,
                                      aseed=a, bseed=b)
    assert len(lam) == K
    assert [int(x) for x in lam] == g["Lambda"]
    assert [int(x) for x in le] == g["Le"]
    assert [int(x) for x in an[1]] == g["aseed1_out"]
    assert [int(x) for x in an[2]] == g["aseed2_out"]
    assert [int(x) for x in bn[0]] == g["bseed0_out"]
    assert [int(x) for x in bn[1]] == g["bseed1_out"]


@pytest.mark.parametrize("seed", range(6))
def test_seed_shift_invariance(orc, seed):
    # Metrics are normalised (exact difference to state 0) before they are
    # saturated, so adding one constant to every entry of a boundary seed
    # changes no output, even when the a-priori values drive the incoming sums
    # far outside int16.  (Clamping the sums before normalising breaks this.)
    K, P = 48, 3
    rng = lambda s, n, lo, hi: synth.randint(1000 + seed, s, n, lo, hi)
    Ls = rng(1, K, -127, 127)
    Lp = rng(2, K, -127, 127)
    La = rng(3, K, -24575, 24575)
    a = rng(4, P * 8, -12000, 12000).reshape(P, 8)
    b = rng(5, P * 8, -12000, 12000).reshape(P, 8)
    a[:, 0] = 0
    b[:, 0] = 0
    ts, tp = rng(6, 3, -127, 127), rng(7, 3, -127, 127)
    base = orc.siso_seeded(Ls, Lp, La, ts, tp, P, aseed=a, bseed=b)
    for c in (-20000, 20000):
        a2 = a + c
        b2 = b - c
        out = orc.siso_seeded(Ls, Lp, La, ts, tp, P, aseed=a2, bseed=b2)
        for x, y in zip(base, out):
            assert np.array_equal(x, y), c
