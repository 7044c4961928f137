"""Helpers of the GPU parity tests: seeded workloads encoded by the oracle,
the library run through its C ABI with the debug outputs, and the oracle's
per-CB and per-TB expectations."""
import numpy as np

import synth


def make_tb(orc, A, G, Qm, seed, rv=0, ebn0=None, snr=None, noiseless=False, amp=100):
    """Payload bits and int8 LLRs of one TB (oracle encoder, synth channel;
    noiseless: +-amp)."""
    a = synth.bits(seed, 100, A)
    e = orc.encode_tb(a, G, Qm=Qm, rv=rv)
    if noiseless:
        llr = np.where(e == 0, amp, -amp).astype(np.int8)
    elif ebn0 is not None:
        llr = synth.channel_llrs(e, 1, synth.sigma2_ebn0(ebn0, A / G), seed, 200)
    else:
        llr = synth.channel_llrs(e, Qm, synth.sigma2_snr(snr), seed, 200)
    return a, llr


def batch(orc, specs):
    """TB parameter dicts and LLRs from specs (dicts of TB parameters plus
    seed and one of ebn0 / snr / noiseless (with amp))."""
    tbs, llrs = [], []
    for s in specs:
        s = dict(s)
        seed = s.pop("seed")
        kw = {k: s.pop(k) for k in ("ebn0", "snr", "noiseless", "amp") if k in s}
        a, llr = make_tb(orc, s["A"], s["G"], s.get("Qm", 2), seed, rv=s.get("rv", 0), **kw)
        tbs.append(s)
        llrs.append(llr)
    return tbs, llrs


def run_gpu(crnt, ctx, tbs, llr_cat, debug=True):
    """Decode a batch through crnt_plan_launch_debug; returns host copies."""
    import torch
    plan = ctx.plan(tbs)
    inf = plan.info
    dev = torch.device("cuda")
    llr_d = torch.from_numpy(np.ascontiguousarray(llr_cat)).to(dev)
    out_d = torch.zeros(max(1, inf["out_bytes"]), dtype=torch.uint8, device=dev)
    n = inf["dbg_elems"]
    stream = torch.cuda.current_stream().cuda_stream
    if debug:
        dd = torch.full((3 * n,), -99, dtype=torch.int8, device=dev)
        de = torch.zeros(n, dtype=torch.int16, device=dev)
        dh = torch.zeros(n, dtype=torch.uint8, device=dev)
        plan.launch(llr_d, out_d, stream, dbg_d=dd, dbg_ext=de, dbg_hard=dh)
    else:
        plan.launch(llr_d, out_d, stream)
    res = plan.results(stream)
    torch.cuda.synchronize()
    out = dict(res=res, out=out_d.cpu().numpy(), info=inf)
    if debug:
        out.update(d=dd.cpu().numpy(), ext=de.cpu().numpy(), hard=dh.cpu().numpy())
    plan.close()
    return out


def oracle_tb(orc, crnt, tb, llr, soft=None):
    """Oracle decode of one TB CB by CB, with the library's per-CB window
    counts (reported by crnt_tb_layout, which needs no GPU).  Returns per-CB
    (d0, d1, d2, iters, hard, ext, iterations run), the A payload bits, tb_ok
    and the soft
    buffer."""
    lay = crnt.tb_layout(tb)
    A, G, Qm, NL, rv = tb["A"], tb["G"], tb.get("Qm", 2), tb.get("NL", 1), tb.get("rv", 0)
    C = len(lay)
    L = 24 if C > 1 else 0
    new = soft is None
    if new:
        soft = np.zeros(sum(c["Ncb"] for c in lay), dtype=np.int8)
    cbs = []
    payload = []
    ok_all = True
    for r, c in enumerate(lay):
        e = llr[c["llr_offset"]:c["llr_offset"] + c["E"]]
        sb = soft[c["soft_offset"]:c["soft_offset"] + c["Ncb"]]
        if new:
            d0, d1, d2, sb2 = orc.derm_cb(e, c["K"], c["F"], rv)
        else:
            d0, d1, d2, sb2 = orc.derm_cb(e, c["K"], c["F"], rv, soft=sb.copy())
        soft[c["soft_offset"]:c["soft_offset"] + c["Ncb"]] = sb2
        it, hard, ext, ran = orc.turbo_decode_cb(d0, d1, d2, F=c["F"],
                                                 crc="B" if C > 1 else "A", P=c["P"],
                                                 max_iter=tb.get("max_iter", 6),
                                                 early_stop=tb.get("early_stop", 1), runs=True)
        ok_all &= it <= tb.get("max_iter", 6)
        cbs.append((d0, d1, d2, it, hard, ext, ran))
        payload.append(hard[c["F"]:c["K"] - L])
    b = np.concatenate(payload)
    tb_ok = bool(ok_all and orc.crc24(b, "A") == 0)
    return cbs, b[:A], tb_ok, soft


def _diff(x, y):
    """Mismatch summary: count and first few differing indices / values."""
    d = np.nonzero(np.asarray(x) != np.asarray(y))[0]
    return dict(n=len(d), first=[(int(i), int(x[i]), int(y[i])) for i in d[:4]])


def oracle_batch(orc, crnt, tbs, llrs, idx, workers=None):
    """oracle_tb of the TBs idx on a thread pool (the oracle's ctypes calls
    release the GIL); returns {t: oracle_tb(...)}."""
    import concurrent.futures as cf
    import os
    workers = workers or min(32, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {t: ex.submit(oracle_tb, orc, crnt, tbs[t], llrs[t]) for t in idx}
        return {t: f.result() for t, f in futs.items()}


def check_batch(orc, crnt, tbs, llrs, g, sample=None):
    """Compare every (or a sample of) TB of a GPU run with the oracle:
    de-rate-matched streams, hard decisions, extrinsics, iteration counts,
    CRC flags and payload bytes -- all bit-exact."""
    idx = list(range(len(tbs)) if sample is None else sample)
    want = oracle_batch(orc, crnt, tbs, llrs, idx)
    dbg_off = [0]
    for t in tbs:
        for c in crnt.tb_layout(t):
            dbg_off.append(dbg_off[-1] + c["K"] + 4)
    cb_index = []
    k = 0
    for t in tbs:
        cb_index.append(k)
        k += len(crnt.tb_layout(t))
    out_off = np.cumsum([0] + [t["A"] // 8 for t in tbs])
    for t in idx:
        tb = tbs[t]
        cbs, bits, tb_ok, _ = want[t]
        res = g["res"][t]
        assert res["C"] == len(cbs)
        for r, (d0, d1, d2, it, hard, ext, ran) in enumerate(cbs):
            K = len(hard)
            o = dbg_off[cb_index[t] + r]
            D = K + 4
            if "d" in g:
                gd = g["d"][3 * o:3 * o + 3 * D]
                assert np.array_equal(gd[:D], d0), ("d0", t, r)
                assert np.array_equal(gd[D:2 * D], d1), ("d1", t, r)
                assert np.array_equal(gd[2 * D:], d2), ("d2", t, r)
                gh, ge = g["hard"][o:o + K], g["ext"][o:o + K]
                assert np.array_equal(gh, hard), ("hard", t, r, _diff(gh, hard),
                                                  res["cb_iters"][r], it)
                assert np.array_equal(ge, ext), ("ext", t, r, _diff(ge, ext))
            assert res["cb_iters"][r] == it, ("iters", t, r, res["cb_iters"][r], it)
            assert res["cb_iters_run"][r] == ran, ("run", t, r, res["cb_iters_run"][r], ran)
            assert res["cb_crc_ok"][r] == (it <= tb.get("max_iter", 6)), ("cbok", t, r)
        assert res["tb_crc_ok"] == tb_ok, ("tbok", t)
        got = np.unpackbits(g["out"][out_off[t]:out_off[t + 1]])
        assert np.array_equal(got, bits), ("payload", t)
    return want
