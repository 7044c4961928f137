"""GPU parity of the fused decode path (de-rate-matching + HARQ combining,
turbo decoding, CRC stop, TB reassembly, batched work queue) against the CPU
oracle, through the C ABI.  All integer work: every output is compared
bit-exactly (tolerance 0)."""
import numpy as np
import pytest

import synth
from gpu_helpers import batch, check_batch, make_tb, oracle_tb, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = crnt_lib.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("P", [1, 8, 64, 128])
def test_single_cb_workload(orc, crnt_lib, ctx, P):
    # A=6120 + CRC24A -> one K=6144 CB, rate 1/3 (E=18444), BPSK at Eb/N0 1 dB
    tbs, llrs = batch(orc, [dict(A=6120, G=18444, Qm=2, P=P, max_iter=6, seed=s, ebn0=1.0)
                            for s in range(3)])
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)
    assert all(r["P_used"] == P for r in g["res"])


@pytest.mark.parametrize("P", [1, 8, 32])
@pytest.mark.parametrize("snr", [18.0, 20.0, 22.0])
def test_20mhz_subframe_workload(orc, crnt_lib, ctx, P, snr):
    # TBS 75376 -> 13 CBs of K=5824, G=86400 (100 PRB x 144 RE x 6), 64QAM
    tbs, llrs = batch(orc, [dict(A=75376, G=86400, Qm=6, P=P, max_iter=6, seed=int(snr),
                                 snr=snr)])
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)
    assert g["res"][0]["C"] == 13 and g["res"][0]["Kp"] == 5824


def test_mixed_batch_autotuned(orc, crnt_lib, ctx):
    # uneven load: A across the whole LTE range (K 40..6144, C 1..13), mixed
    # modulation, SNR around the decoding threshold so iterations vary
    shapes = synth.tti_batch(seed=7, n_tb=40, amax=30000)
    shapes += synth.tti_batch(seed=8, n_tb=4, amin=60000)
    specs = []
    for i, s in enumerate(shapes):
        specs.append(dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=6,
                          early_stop=1 if i % 3 else 0, rv=i % 4, seed=100 + i,
                          snr=s["snr_db"]))
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)
    iters = [it for r in g["res"] for it in r["cb_iters"]]
    assert len(set(iters)) > 2  # uneven iteration counts really occurred


def test_edge_cases(orc, crnt_lib, ctx):
    specs = [
        dict(A=16, G=132, Qm=2, seed=1, snr=2.0),              # K = 40, smallest CB
        dict(A=16, G=1200, Qm=2, seed=2, snr=-4.0),            # heavy repetition E >> 3D
        dict(A=6128, G=13000, Qm=2, seed=3, snr=3.0),          # C = 2 with filler bits
        dict(A=1000, G=1400, Qm=4, seed=4, snr=30.0, max_iter=1),
        dict(A=2000, G=2600, Qm=2, seed=5, snr=6.0, early_stop=0, max_iter=3),
        dict(A=512, G=900, Qm=2, seed=6, snr=0.0, P=500),      # P beyond K/8: clamped
        dict(A=40000, G=60000, Qm=4, NL=2, rv=1, seed=7, snr=9.0, max_iter=8),
        dict(A=3000, G=3100, Qm=2, seed=8, snr=-10.0),         # undecodable: max_iter + 1
    ]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)
    assert g["res"][7]["cb_iters"] == [7] and not g["res"][7]["tb_crc_ok"]
    assert g["res"][3]["cb_iters"][0] in (1, 2)


def test_batch_invariance(orc, crnt_lib, ctx):
    # a TB's result alone equals its result inside a mixed batch
    shapes = synth.tti_batch(seed=11, n_tb=12, amax=40000)
    specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], seed=200 + i, snr=s["snr_db"])
             for i, s in enumerate(shapes)]
    tbs, llrs = batch(orc, specs)
    gall = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs), debug=False)
    off = np.cumsum([0] + [t["A"] // 8 for t in tbs])
    for t in (0, 5, 11):
        g1 = run_gpu(crnt_lib, ctx, [tbs[t]], llrs[t], debug=False)
        assert g1["res"][0]["cb_iters"] == gall["res"][t]["cb_iters"]
        assert g1["res"][0]["tb_crc_ok"] == gall["res"][t]["tb_crc_ok"]
        assert np.array_equal(g1["out"], gall["out"][off[t]:off[t + 1]])


def test_harq_combining(orc, crnt_lib, ctx):
    # first transmission (rv 0) fails; the retransmission (rv 2) combined in
    # the library-owned soft buffer decodes; both match the oracle's combine
    A, G, Qm = 2000, 2400, 2
    a = synth.bits(5, 100, A)
    e0 = orc.encode_tb(a, G, Qm=Qm, rv=0)
    e2 = orc.encode_tb(a, G, Qm=Qm, rv=2)
    sig = synth.sigma2_snr(1.0)
    l0 = synth.channel_llrs(e0, 2, sig, 5, 1)
    l2 = synth.channel_llrs(e2, 2, sig, 5, 2)
    key = dict(cell=3, ue=7, harq_pid=2, flags=crnt_lib.F_HARQ)
    t0 = dict(A=A, G=G, Qm=Qm, rv=0, new_data=1, **key)
    t2 = dict(A=A, G=G, Qm=Qm, rv=2, new_data=0, **key)
    g0 = run_gpu(crnt_lib, ctx, [t0], l0)
    cbs0, _, ok0, soft = oracle_tb(orc, crnt_lib, t0, l0)
    check_batch(orc, crnt_lib, [t0], [l0], g0)
    assert not ok0 and not g0["res"][0]["tb_crc_ok"]
    g2 = run_gpu(crnt_lib, ctx, [t2], l2)
    cbs2, bits2, ok2, _ = oracle_tb(orc, crnt_lib, t2, l2, soft=soft)
    assert ok2 and g2["res"][0]["tb_crc_ok"]
    d0, d1, d2, it, hard, ext, _ = cbs2[0]
    D = len(d0)
    assert np.array_equal(g2["d"][:D], d0) and np.array_equal(g2["d"][2 * D:3 * D], d2)
    assert g2["res"][0]["cb_iters"][0] == it
    assert np.array_equal(np.unpackbits(g2["out"]), bits2)
    assert ctx.harq_release(3, 7, 2) == 0
    assert ctx.harq_release(3, 7, 2) == crnt_lib.ENOTFOUND


def test_harq_unknown_process_rejected(crnt_lib, ctx):
    t = dict(A=2000, G=2400, Qm=2, rv=2, new_data=0, cell=9, ue=9, harq_pid=9,
             flags=crnt_lib.F_HARQ)
    with pytest.raises(crnt_lib.CrntError) as ei:
        ctx.plan([t])
    assert ei.value.code == crnt_lib.ENOTFOUND


def test_full_tti(orc, crnt_lib, ctx):
    # the benchmark's workload (40 cells x 8 UEs, A uniform over 16..75376,
    # exactly 6 iterations, window counts of the installed table) in its
    # launch configuration: every one of the 320 TBs against the oracle --
    # de-rate-matched streams, final extrinsics, hard decisions, iteration
    # counts, CRC flags and payload bytes
    shapes = synth.tti_batch(seed=1, n_tb=320)
    specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=6, early_stop=0, seed=300 + i,
                  snr=s["snr_db"]) for i, s in enumerate(shapes)]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)
    assert sum(r["C"] for r in g["res"]) == g["info"]["n_cb"] > 2000
    ok = sum(r["tb_crc_ok"] for r in g["res"])
    assert 0 < ok < len(tbs)  # SNRs around threshold: some TBs fail, most decode


def test_saturating_path_runs_bit_exact(orc, crnt_lib, ctx):
    # Window passes the decoder cannot prove clamp-free run its exact path
    # (int16 clamps after normalisation, on Lambda and on Le).  The proof
    # needs spread(alpha) + spread(beta) + 2 g <= 32767 with g = 254 + the
    # largest |a-priori| of the pass; window 0 starts from the spread 16384 of
    # the known start state, so it fails once |La| exceeds about 2086.  With
    # +-127 channel LLRs (noiseless, rate 1/3) the extrinsics climb to about
    # 2600 by the fourth iteration (a weight-2 error event keeps them there:
    # La <= 0.75 (La + 7 x 127)), so the first and last windows switch to the
    # exact path; heavy repetition (E = 9 x 3K, soft bits at +-127) does the
    # same.  sat_passes counts those passes per TB, and every output stays
    # bit-exact.  No clamp can act with int8 channel inputs (the extrinsics
    # never approach 32767): the clamp semantics themselves are pinned on the
    # CPU by the hand-worked golden (test_oracle_saturation.py).
    specs = [dict(A=6120, G=18444, Qm=2, P=P, max_iter=8, early_stop=0, seed=60 + P,
                  noiseless=True, amp=127) for P in (1, 2, 8)]
    specs += [dict(A=1000, G=9000, Qm=2, P=2, max_iter=8, early_stop=0, seed=66, snr=20.0),
              dict(A=75376, G=86400, Qm=6, P=4, max_iter=8, early_stop=0, seed=64, snr=40.0),
              dict(A=16, G=1200, Qm=2, P=1, max_iter=8, early_stop=0, seed=65, snr=30.0)]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)
    sat = [r["sat_passes"] for r in g["res"]]
    print("window passes on the saturating path per TB:", sat)
    assert all(x > 0 for x in sat[:4]), sat
    # the clamp-free path still runs where it can: a moderate-SNR TB
    tbs2, llrs2 = batch(orc, [dict(A=6120, G=18444, Qm=2, P=64, max_iter=6, seed=67, ebn0=1.0)])
    g2 = run_gpu(crnt_lib, ctx, tbs2, np.concatenate(llrs2))
    check_batch(orc, crnt_lib, tbs2, llrs2, g2)
    assert g2["res"][0]["sat_passes"] == 0


def test_window_count_capped_at_128(orc, crnt_lib, ctx):
    # The library caps the window count at CRNT_MAX_P = 128 (one thread per
    # window in a 128-thread CTA) on top of the P <= K/8 clamp that the
    # oracle applies; a request above the cap decodes exactly like P = 128,
    # checked against the oracle called directly at 128 windows.
    tb = dict(A=6120, G=18444, Qm=2, P=500, max_iter=6, early_stop=0)
    assert crnt_lib.tb_layout(tb)[0]["P"] == 128 and orc.windows(6144, 500) > 128
    a, llr = make_tb(orc, 6120, 18444, 2, 77, ebn0=1.2)
    g = run_gpu(crnt_lib, ctx, [tb], llr)
    d0, d1, d2, _ = orc.derm_cb(llr, 6144, 0, 0)
    it, hard, ext, ran = orc.turbo_decode_cb(d0, d1, d2, F=0, crc="A", P=128, max_iter=6,
                                             early_stop=0, runs=True)
    assert g["res"][0]["P_used"] == 128
    assert g["res"][0]["cb_iters"] == [it]
    assert np.array_equal(g["hard"][:6144], hard) and np.array_equal(g["ext"][:6144], ext)
    g128 = run_gpu(crnt_lib, ctx, [dict(tb, P=128)], llr)
    assert np.array_equal(g128["out"], g["out"])


@pytest.mark.parametrize("n_tb", [23, 24, 61])
def test_decode_batch_chunks_match_one_plan(orc, crnt_lib, ctx, n_tb):
    # crnt_decode_batch splits batches of >= 24 TBs into three chunks on
    # their own streams; with pageable host buffers (staged), page-locked
    # host buffers (used in place by the kernel) and device buffers every
    # TB's bits and results equal one single-plan launch of the whole batch,
    # which the other tests hold to the oracle
    shapes = synth.tti_batch(seed=17 + n_tb, n_tb=n_tb, amax=40000)
    specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], seed=700 + i, snr=s["snr_db"], max_iter=5,
                  early_stop=i % 2) for i, s in enumerate(shapes)]
    tbs, llrs = batch(orc, specs)
    llr = np.concatenate(llrs)
    want = run_gpu(crnt_lib, ctx, tbs, llr, debug=False)
    nbytes = sum(t["A"] // 8 for t in tbs)
    out_h = np.zeros(nbytes, dtype=np.uint8)
    res_h = ctx.decode_batch(tbs, llr, out_h)
    out_p = torch.zeros(nbytes, dtype=torch.uint8).pin_memory()
    res_p = ctx.decode_batch(tbs, torch.from_numpy(llr).pin_memory(), out_p)
    dev = torch.device("cuda")
    out_d = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    res_d = ctx.decode_batch(tbs, torch.from_numpy(llr).to(dev), out_d)
    assert np.array_equal(out_h, want["out"][:nbytes])
    assert np.array_equal(out_p.numpy(), want["out"][:nbytes])
    assert np.array_equal(out_d.cpu().numpy(), want["out"][:nbytes])
    for r_h, r_p, r_d, w in zip(res_h, res_p, res_d, want["res"]):
        for k in ("cb_iters", "cb_crc_ok", "tb_crc_ok", "C", "Kp", "P_used"):
            assert r_h[k] == w[k] and r_p[k] == w[k] and r_d[k] == w[k], k


def test_plan_launch_captured_in_cuda_graph(orc, crnt_lib, ctx):
    # one persistent launch per TTI can be captured once and replayed
    shapes = synth.tti_batch(seed=13, n_tb=24, amax=30000)
    tbs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], max_iter=6, early_stop=0) for s in shapes]
    llrs = [make_tb(orc, s["A"], s["G"], s["Qm"], 600 + i, snr=s["snr_db"])[1]
            for i, s in enumerate(shapes)]
    plan = ctx.plan(tbs)
    dev = torch.device("cuda")
    llr_d = torch.from_numpy(np.concatenate(llrs)).to(dev)
    out_direct = torch.zeros(plan.info["out_bytes"], dtype=torch.uint8, device=dev)
    out_graph = torch.zeros_like(out_direct)
    s = torch.cuda.current_stream().cuda_stream
    plan.launch(llr_d, out_direct, s)
    want = plan.results(s)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        plan.launch(llr_d, out_graph, torch.cuda.current_stream().cuda_stream)
    for _ in range(3):
        out_graph.zero_()
        g.replay()
    torch.cuda.synchronize()
    got = plan.results(s)
    assert torch.equal(out_graph, out_direct)
    assert [r["cb_iters"] for r in got] == [r["cb_iters"] for r in want]
    plan.close()


def test_autotuned_windows_match_oracle(orc, crnt_lib, ctx):
    # the autotuner installs a window count per K (windows of >= 32 steps
    # where K allows); P = 0 TBs then decode with it, still bit-exact with
    # the oracle run at the same window counts
    old = crnt_lib.tune_get()
    old_radix = crnt_lib.tune_radix_get()
    try:
        table = ctx.autotune(32)
        assert table == crnt_lib.tune_get()
        assert set(crnt_lib.tune_radix_get()) <= {2, 4}
        ks = list(orc.k_table())
        assert len(ks) == len(table) == 188
        for K, P in zip(ks, table):
            assert 1 <= P <= min(128, max(1, K // 8)), (K, P)
            assert -(-K // P) >= min(32, K), (K, P)
        shapes = synth.tti_batch(seed=23, n_tb=16, amax=40000)
        specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=6, seed=800 + i,
                      snr=s["snr_db"]) for i, s in enumerate(shapes)]
        tbs, llrs = batch(orc, specs)
        g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
        check_batch(orc, crnt_lib, tbs, llrs, g)
    finally:
        crnt_lib.tune_set(old)
        crnt_lib.tune_radix_set(old_radix)


@pytest.fixture
def radix4(crnt_lib):
    """The radix-4 forward recursion selected for every CB size."""
    old = crnt_lib.tune_radix_get()
    crnt_lib.tune_radix_set([4] * crnt_lib.NUM_K)
    yield
    crnt_lib.tune_radix_set(old)


@pytest.mark.parametrize("P", [1, 8, 128])
def test_radix4_forward_single_cb(orc, crnt_lib, ctx, radix4, P):
    # two trellis steps per forward update on clamp-free passes: the same
    # metrics as radix 2, so every output stays bit-exact with the oracle
    tbs, llrs = batch(orc, [dict(A=6120, G=18444, Qm=2, P=P, max_iter=6, seed=s, ebn0=1.0)
                            for s in range(3)])
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)


def test_radix4_forward_mixed_and_saturating(orc, crnt_lib, ctx, radix4):
    # every CB size class, ragged windows (K not a multiple of 4 P), both
    # the clamp-free passes (radix 4) and, with noiseless and very strong
    # inputs whose extrinsics grow large, passes that may saturate (radix 2)
    shapes = synth.tti_batch(seed=9, n_tb=30, amax=30000)
    shapes += synth.tti_batch(seed=10, n_tb=3, amin=60000)
    specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=6, early_stop=i % 2,
                  rv=i % 4, seed=300 + i, snr=s["snr_db"]) for i, s in enumerate(shapes)]
    specs += [dict(A=6120, G=18444, Qm=2, P=P, max_iter=8, early_stop=0, seed=40 + P,
                   noiseless=True) for P in (1, 3, 64)]
    specs += [dict(A=520, G=1600, Qm=2, P=7, max_iter=8, early_stop=0, seed=45, snr=40.0),
              dict(A=16, G=132, Qm=2, seed=46, snr=2.0),
              dict(A=3000, G=3100, Qm=2, seed=47, snr=-10.0)]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)


def test_purge_on_failure(orc, crnt_lib, ctx):
    # Purge on failure (Algorithm 2): with CRNT_F_PURGE a failed CB stops the
    # other CBs of its TB.  Decoded TBs are bit-exact with the oracle; every
    # failed TB still fails, and each of its CBs either matches the oracle
    # (iterations, CRC flag) or was stopped (0 iterations, CRC not passed).
    # Many undecodable 13-CB TBs spread their CBs over several waves of CTAs.
    specs = []
    for i in range(48):
        bad = i % 2 == 0
        specs.append(dict(A=75376, G=86400, Qm=6, max_iter=6, early_stop=1,
                          flags=crnt_lib.F_PURGE, seed=900 + i, snr=6.0 if bad else 22.0))
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs), debug=False)
    off = np.cumsum([0] + [t["A"] // 8 for t in tbs])
    stopped = 0
    for t in range(len(tbs)):
        cbs, bits, ok, _ = oracle_tb(orc, crnt_lib, tbs[t], llrs[t])
        r = g["res"][t]
        assert r["tb_crc_ok"] == ok
        if ok:
            assert np.array_equal(np.unpackbits(g["out"][off[t]:off[t + 1]]), bits)
            assert r["cb_iters"] == [c[3] for c in cbs]
        for c, it, crc in zip(cbs, r["cb_iters"], r["cb_crc_ok"]):
            if it == 0:
                stopped += 1
                assert not ok and not crc
            else:
                assert it == c[3] and crc == (c[3] <= 6)
    print("CBs stopped by purges:", stopped)


def test_mi_stop_rule_matches_oracle(orc, crnt_lib, ctx):
    # stop rule 2 (the paper's mutual-information rule): per CB iterations,
    # hard decisions, extrinsics and CRC results bit-exact with the oracle,
    # over SNRs where blocks decode quickly, slowly or not at all
    shapes = synth.tti_batch(seed=29, n_tb=24, amax=40000)
    specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=8, early_stop=2, seed=950 + i,
                  snr=s["snr_db"]) for i, s in enumerate(shapes)]
    specs.append(dict(A=6120, G=18444, Qm=2, P=1, max_iter=8, early_stop=2, seed=990, ebn0=0.5))
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    check_batch(orc, crnt_lib, tbs, llrs, g)
    iters = [it for r in g["res"] for it in r["cb_iters"]]
    assert min(iters) >= 2 and len(set(iters)) > 2


def test_int_issue_probe(crnt_lib):
    # the issue-rate probe behind the roofline: every kind reports a rate
    # between 1 and 4 warp-instructions per SM clock (4 schedulers); DPX
    # add-max reaches at least 1.5 (two per clock on this GPU)
    import ctypes

    from paper_1905_01141_gb300 import build as crnt_build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = crnt_build.load_probe()
    rates = []
    for kind in range(4):
        v = ctypes.c_double()
        assert L.crnt_int_issue_probe(0, kind, ctypes.byref(v)) == 0
        rates.append(v.value)
    assert all(1.0 <= r <= 4.0 for r in rates), rates
    assert rates[0] >= 1.5
    v = ctypes.c_double()
    assert L.crnt_int_issue_probe(0, 4, ctypes.byref(v)) == crnt_lib.EINVAL


@pytest.fixture(scope="module")
def ctx_pairs(crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = crnt_lib.Context(0, pair_min_cbs=1)
    yield c
    c.close()


@pytest.mark.parametrize("shape", [1, 2])
def test_cb_timestamps(orc, crnt_lib, ctx_pairs, shape):
    # the performance captor: per CB four %globaltimer stamps in order, all
    # inside the launch, iterations equal to the results' iterations run
    old = crnt_lib.tune_shape_get()
    crnt_lib.tune_shape_set([shape] * crnt_lib.NUM_K)
    try:
        shapes = synth.tti_batch(seed=31, n_tb=24, amax=40000)
        specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=6, early_stop=1,
                      seed=1100 + i, snr=s["snr_db"]) for i, s in enumerate(shapes)]
        tbs, llrs = batch(orc, specs)
        plan = ctx_pairs.plan(tbs)
        plan.set_timing(True)
        dev = torch.device("cuda")
        llr_d = torch.from_numpy(np.concatenate(llrs)).to(dev)
        out_d = torch.zeros(plan.info["out_bytes"], dtype=torch.uint8, device=dev)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        plan.launch(llr_d, out_d, s.cuda_stream)
        e1.record(s)
        tm = plan.timing(s.cuda_stream)
        res = plan.results(s.cuda_stream)
        torch.cuda.synchronize()
        assert len(tm) == plan.info["n_cb"]
        assert (plan.info["pair_items"] > 0) == (shape == 2)
        assert (tm["t_start_ns"] <= tm["t_derm_ns"]).all()
        assert (tm["t_derm_ns"] <= tm["t_iter_ns"]).all()
        assert (tm["t_iter_ns"] <= tm["t_done_ns"]).all()
        span_us = (tm["t_done_ns"].max() - tm["t_start_ns"].min()) / 1e3
        assert 0 < span_us <= e0.elapsed_time(e1) * 1e3 + 5
        runs = [x for r in res for x in r["cb_iters_run"]]
        assert list(tm["iterations"]) == runs
        assert list(tm["tb"]) == [t for t, r in enumerate(res) for _ in range(r["C"])]
        plan.close()
    finally:
        crnt_lib.tune_shape_set(old)
