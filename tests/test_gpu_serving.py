"""Serving loop (crnt_submit / crnt_poll): continuous batching gives every
TB the same result alone and in the mix, admission refuses work beyond the
in-flight limit, HARQ retransmissions combine through the serving path."""
import json
import time

import numpy as np
import pytest

import synth
from gpu_helpers import make_tb, oracle_tb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = crnt_lib.Context(0, max_inflight=2000)
    yield c
    c.close()


def drain(ctx, tickets, timeout_s=30.0):
    want = set(tickets)
    got = {}
    t0 = time.time()
    while want - set(got):
        for d, data in ctx.poll(512, 2000):
            got[d["ticket"]] = (d, data)
        assert time.time() - t0 < timeout_s, "serving did not finish"
    return got


def test_results_same_alone_and_in_the_mix(orc, crnt_lib, ctx):
    shapes = synth.tti_batch(seed=31, n_tb=48, amax=40000)
    tbs, llrs = [], []
    for i, s in enumerate(shapes):
        tbs.append(dict(A=s["A"], G=s["G"], Qm=s["Qm"], max_iter=6, early_stop=1))
        llrs.append(make_tb(orc, s["A"], s["G"], s["Qm"], 400 + i, snr=s["snr_db"])[1])
    # alone: one blocking batch decode per TB
    alone = []
    for t, l in zip(tbs, llrs):
        out = np.zeros(t["A"] // 8, dtype=np.uint8)
        r = ctx.decode_batch([t], l, out)[0]
        alone.append((r, out.tobytes()))
    # in the mix: submitted in uneven groups while earlier groups run
    tickets = []
    i = 0
    for g in (1, 7, 3, 12, 5, 20):
        tk = ctx.submit(tbs[i:i + g], llrs[i:i + g])
        assert tk is not None
        tickets += tk
        i += g
    got = drain(ctx, tickets)
    for k, tk in enumerate(tickets):
        d, data = got[tk]
        r, bits = alone[k]
        assert d["status"] == 0
        assert d["cb_iters"] == r["cb_iters"] and d["tb_crc_ok"] == r["tb_crc_ok"]
        assert data == bits
        assert d["t_submit_ns"] <= d["t_start_ns"] <= d["t_done_ns"]
    # and the serving results match the oracle on a sample
    for k in (0, 9, 30):
        _, bits, ok, _ = oracle_tb(orc, crnt_lib, tbs[k], llrs[k])
        d, data = got[tickets[k]]
        assert d["tb_crc_ok"] == ok
        assert np.array_equal(np.unpackbits(np.frombuffer(data, np.uint8)), bits)


def test_admission_refuses_beyond_inflight(crnt_lib):
    with crnt_lib.Context(0, max_inflight=4, admission=1) as c:
        t = dict(A=6120, G=18444, Qm=2)
        llr = np.zeros(18444, dtype=np.int8)
        assert c.submit([t] * 5, [llr] * 5) is None  # CRNT_EAGAIN: 5 > 4 in flight
        tk = c.submit([t] * 4, [llr] * 4)
        assert tk is not None
        got = drain(c, tk)
        assert len(got) == 4
        st = c.serve_stats()
        assert st["submit_calls"] == 2 and st["refused_calls"] == 1
        assert st["offered_tbs"] == 9 and st["admitted_tbs"] == 4 and st["done_tbs"] == 4
        assert st["refused_deadline"] == 0
        assert c.submit([t], [llr]) is not None
        assert c.poll(8, 5_000_000)


def test_admission_refuses_by_predicted_completion(crnt_lib):
    # a 50 us latency target: with work outstanding, the model (its prior
    # latency alone is 150 us) predicts any further subframe late and
    # refuses it; with nothing outstanding a subframe is always admitted
    with crnt_lib.Context(0, deadline_us=50, max_inflight=4096) as c:
        big = dict(A=75376, G=86400, Qm=6, max_iter=16, early_stop=0)  # 13 CBs x 16 iterations
        llr_big = np.zeros(86400, dtype=np.int8)
        small = dict(A=1000, G=1200, Qm=2)
        llr_small = np.zeros(1200, dtype=np.int8)
        tk = c.submit([big] * 32, [llr_big] * 32)
        assert tk is not None
        assert c.submit([small], [llr_small]) is None  # CRNT_EAGAIN
        st = c.serve_stats()
        assert st["refused_deadline"] == 1 and st["refused_calls"] == 1
        assert st["admitted_tbs"] == 32 and st["offered_tbs"] == 33
        got = drain(c, tk)
        assert all(d["status"] == 0 for d, _ in got.values())
        st = c.serve_stats()
        assert st["done_tbs"] == 32 and st["late_tbs"] == 32  # each took more than 50 us
        assert st["model_a_us"] > 0 and st["model_rate"] > 0
        tk2 = c.submit([small], [llr_small])
        assert tk2 is not None
        drain(c, tk2)


def test_poll_timeout_returns_empty(crnt_lib):
    with crnt_lib.Context(0) as c:
        t0 = time.time()
        assert c.poll(4, 20000) == []
        assert time.time() - t0 < 2.0


def test_harq_through_serving(orc, crnt_lib, ctx):
    A, G, Qm = 2000, 2400, 2
    a = synth.bits(5, 100, A)
    e0 = orc.encode_tb(a, G, Qm=Qm, rv=0)
    e2 = orc.encode_tb(a, G, Qm=Qm, rv=2)
    sig = synth.sigma2_snr(1.0)
    l0 = synth.channel_llrs(e0, 2, sig, 5, 1)
    l2 = synth.channel_llrs(e2, 2, sig, 5, 2)
    key = dict(cell=11, ue=3, harq_pid=5, flags=crnt_lib.F_HARQ)
    t0 = dict(A=A, G=G, Qm=Qm, rv=0, new_data=1, **key)
    t2 = dict(A=A, G=G, Qm=Qm, rv=2, new_data=0, **key)
    d0, _ = drain(ctx, ctx.submit([t0], [l0])).popitem()[1]
    assert not d0["tb_crc_ok"]
    d2, data = drain(ctx, ctx.submit([t2], [l2])).popitem()[1]
    _, soft = oracle_tb(orc, crnt_lib, t0, l0)[2:]
    _, bits, ok, _ = oracle_tb(orc, crnt_lib, t2, l2, soft=soft)
    assert ok and d2["tb_crc_ok"]
    assert np.array_equal(np.unpackbits(np.frombuffer(data, np.uint8)), bits)
    ctx.harq_release(11, 3, 5)
    with pytest.raises(crnt_lib.CrntError) as ei:
        ctx.submit([t2], [l2])
    assert ei.value.code == crnt_lib.ENOTFOUND


def test_native_load_generator_runs(crnt_lib):
    # crnt_loadgen (the bench's serving load generator, a C-ABI client) serves
    # a light load: every submitted TB comes back without error or refusal
    # (the latency figures are the bench's; here only a loose bound)
    import os
    import struct
    import subprocess
    import tempfile

    import numpy as np
    from paper_1905_01141_gb300 import build
    shapes = synth.tti_batch(seed=41, n_tb=16, amax=20000)
    tbs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], max_iter=6, early_stop=1) for s in shapes]
    llr = np.concatenate([synth.channel_llrs(np.zeros(s["G"], np.uint8), s["Qm"],
                                             synth.sigma2_snr(30.0), 41, i)
                          for i, s in enumerate(shapes)])
    offs = np.cumsum([0] + [s["G"] for s in shapes])[:-1].astype(np.int64)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "load.bin")
        with open(path, "wb") as f:
            f.write(struct.pack("<I", len(tbs)))
            f.write(bytes(crnt_lib.params_array(tbs)))
            f.write(offs.tobytes())
            f.write(llr.tobytes())
        out = subprocess.run([build.LOADGEN, path, "8", "0.3", "0.1", "1", "2"],
                             capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    rows = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(rows) == 1 and rows[0]["cells"] == 2
    assert rows[0]["tbs"] >= 2 * 8 * 250 and rows[0]["errors"] == 0
    assert rows[0]["refused_subframes"] == 0 and rows[0]["p99_us"] < 20000.0
