"""Pins of the oracle's max-log-MAP SISO against brute force: for tiny
trellises the APP values are the exact difference of the best codeword
metrics with u_k = 0 and u_k = 1 (no saturation is reached at these
magnitudes, and normalisation cancels in the difference).  The brute force
enumerates input sequences and encodes them with its own feedback-register
recursion (a_k = u_k + a_{k-2} + a_{k-3}, z_k = a_k + a_{k-1} + a_{k-3})."""
import itertools

import numpy as np
import pytest

import synth


def rsc_path(u, s0):
    """Run the register from state s0 = (a_{-1}, a_{-2}, a_{-3}) over inputs u;
    return parities, states after each step (as (a_{k}, a_{k-1}, a_{k-2}))."""
    hist = list(s0)  # hist[0] = a_{k-1}, hist[1] = a_{k-2}, hist[2] = a_{k-3}
    zs, states = [], []
    for uk in u:
        a = uk ^ hist[1] ^ hist[2]
        z = a ^ hist[0] ^ hist[2]
        hist = [a, hist[0], hist[1]]
        zs.append(z)
        states.append(tuple(hist))
    return zs, states


def tail_path(state):
    """Terminating inputs: choose u so that the register input a is 0."""
    hist = list(state)
    xs, zs = [], []
    for _ in range(3):
        u = hist[1] ^ hist[2]
        a = 0
        z = a ^ hist[0] ^ hist[2]
        hist = [a, hist[0], hist[1]]
        xs.append(u)
        zs.append(z)
    assert hist == [0, 0, 0]
    return xs, zs


def sidx(st):
    # oracle state index: 4*r1 + 2*r2 + r3 with (r1, r2, r3) = (a_{k-1}, a_{k-2}, a_{k-3})
    return 4 * st[0] + 2 * st[1] + st[2]


def brute_window(Ls, Lp, La, lo, hi, start_metric, end_metric, tail):
    """Exact max-log APP over steps [lo, hi) of one window.  start_metric[s]
    (None = not allowed) weights the start state; end_metric[s] the end state;
    if tail = (ts, tp) the end state continues through its terminating tail."""
    w = hi - lo
    best = {k: [None, None] for k in range(lo, hi)}
    for s0 in range(8):
        if start_metric[s0] is None:
            continue
        st0 = ((s0 >> 2) & 1, (s0 >> 1) & 1, s0 & 1)
        for u in itertools.product((0, 1), repeat=w):
            zs, states = rsc_path(u, st0)
            m = start_metric[s0]
            for j in range(w):
                k = lo + j
                m += (int(Ls[k]) + int(La[k])) * (u[j] == 0) + int(Lp[k]) * (zs[j] == 0)
            send = sidx(states[-1])
            if tail is not None:
                xs, zt = tail_path(states[-1])
                ts, tp = tail
                m += sum(int(ts[j]) * (xs[j] == 0) + int(tp[j]) * (zt[j] == 0) for j in range(3))
            else:
                if end_metric[send] is None:
                    continue
                m += end_metric[send]
            for j in range(w):
                b = best[lo + j]
                if b[u[j]] is None or m > b[u[j]]:
                    b[u[j]] = m
    return {k: best[k][0] - best[k][1] for k in best}


def small_inputs(K, seed, amp=20, aamp=40):
    Ls = synth.randint(seed, 1, K, -amp, amp)
    Lp = synth.randint(seed, 2, K, -amp, amp)
    La = synth.randint(seed, 3, K, -aamp, aamp)
    ts = synth.randint(seed, 4, 3, -amp, amp)
    tp = synth.randint(seed, 5, 3, -amp, amp)
    return Ls, Lp, La, ts, tp


@pytest.mark.parametrize("K,seed", [(3, 0), (6, 1), (8, 2), (10, 3), (9, 4)])
def test_siso_p1_equals_brute_force(orc, K, seed):
    Ls, Lp, La, ts, tp = small_inputs(K, seed)
    lam, le = orc.siso_once(Ls, Lp, La, ts, tp, P=1)
    start = [0] + [None] * 7
    want = brute_window(Ls, Lp, La, 0, K, start, None, (ts, tp))
    for k in range(K):
        assert lam[k] == want[k], k
        assert le[k] == want[k] - (Ls[k] + La[k])


def test_siso_first_iteration_windows_use_zero_seeds(orc):
    # P = 2 on K = 16: windows [0,8) and [8,16).  Window 0 starts in state 0
    # and ends free (zero metrics); window 1 starts free and ends in the tail.
    K = 16
    Ls, Lp, La, ts, tp = small_inputs(K, 9)
    lam, le, aseed, bseed = orc.siso_seeded(Ls, Lp, La, ts, tp, P=2)
    w0 = brute_window(Ls, Lp, La, 0, 8, [0] + [None] * 7, [0] * 8, None)
    w1 = brute_window(Ls, Lp, La, 8, 16, [0] * 8, None, (ts, tp))
    for k in range(8):
        assert lam[k] == w0[k]
    for k in range(8, 16):
        assert lam[k] == w1[k]


def test_siso_seeds_are_normalised_boundary_metrics(orc):
    # After one pass, the alpha seed of window 1 is the forward metric at the
    # boundary (best path from state 0 into each state) minus that of state 0;
    # the beta seed of window 0 is the backward metric of window 1 at the
    # boundary, normalised the same way.  Then a second pass with those seeds
    # equals the brute force with the seeds as start / end weights.
    K = 16
    Ls, Lp, La, ts, tp = small_inputs(K, 12)
    lam, le, aseed, bseed = orc.siso_seeded(Ls, Lp, La, ts, tp, P=2)
    fwd = [None] * 8
    for u in itertools.product((0, 1), repeat=8):
        zs, states = rsc_path(u, (0, 0, 0))
        m = sum((int(Ls[j]) + int(La[j])) * (u[j] == 0) + int(Lp[j]) * (zs[j] == 0)
                for j in range(8))
        s = sidx(states[-1])
        fwd[s] = m if fwd[s] is None else max(fwd[s], m)
    assert [int(v) for v in aseed[1]] == [f - fwd[0] for f in fwd]
    bwd = [None] * 8
    for s0 in range(8):
        st0 = ((s0 >> 2) & 1, (s0 >> 1) & 1, s0 & 1)
        for u in itertools.product((0, 1), repeat=8):
            zs, states = rsc_path(u, st0)
            m = sum((int(Ls[8 + j]) + int(La[8 + j])) * (u[j] == 0) + int(Lp[8 + j]) * (zs[j] == 0)
                    for j in range(8))
            xs, zt = tail_path(states[-1])
            m += sum(int(ts[j]) * (xs[j] == 0) + int(tp[j]) * (zt[j] == 0) for j in range(3))
            bwd[s0] = m if bwd[s0] is None else max(bwd[s0], m)
    assert [int(v) for v in bseed[0]] == [b - bwd[0] for b in bwd]
    # second pass with the seeds
    lam2, _, _, _ = orc.siso_seeded(Ls, Lp, La, ts, tp, P=2, aseed=aseed, bseed=bseed)
    w0 = brute_window(Ls, Lp, La, 0, 8, [0] + [None] * 7, [int(v) for v in bseed[0]], None)
    w1 = brute_window(Ls, Lp, La, 8, 16, [int(v) for v in aseed[1]], None, (ts, tp))
    for k in range(8):
        assert lam2[k] == w0[k]
    for k in range(8, 16):
        assert lam2[k] == w1[k]


def test_siso_saturates_instead_of_wrapping(orc):
    # Extreme a-priori values drive metrics past int16: outputs stay in range
    # and keep the sign of the evidence.
    K = 64
    Ls = np.full(K, 127)
    Lp = np.full(K, 127)
    La = np.full(K, 24575)
    ts = np.full(3, 127)
    tp = np.full(3, 127)
    lam, le = orc.siso_once(Ls, Lp, La, ts, tp, P=1)
    # exact metrics would give Lambda > 32767 everywhere; saturated state
    # metrics cap the competitor distance instead of wrapping around
    assert lam.min() > 16384
    lam_n, le_n = orc.siso_once(-Ls, -Lp, -La, -ts, -tp, P=1)
    assert lam_n.max() < -16384


def test_windows_clamp(orc):
    assert orc.windows(40, 64) == 5 and orc.windows(6144, 64) == 64 and orc.windows(6144, 0) == 1
