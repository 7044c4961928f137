"""GPU parity of the CB-pair shape (two CBs of equal size and window count on
the same threads, window p of both in the two 16-bit lanes of each register)
against the CPU oracle.  The shape changes only the speed: every output must
stay bit-exact, including where a pass falls back to one CB at a time (a
pass that cannot be proved to stay within 16 bits, or a CB whose partner has
stopped iterating)."""
import numpy as np
import pytest

import synth
from gpu_helpers import batch, check_batch, oracle_tb, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = crnt_lib.Context(0, pair_min_cbs=1)  # pairs in batches of any size
    yield c
    c.close()


@pytest.fixture
def pairs(crnt_lib):
    """CB pairs selected for every CB size."""
    old = crnt_lib.tune_shape_get()
    crnt_lib.tune_shape_set([2] * crnt_lib.NUM_K)
    yield
    crnt_lib.tune_shape_set(old)


def test_shape_table_get_set(crnt_lib):
    old = crnt_lib.tune_shape_get()
    try:
        crnt_lib.tune_shape_set([0] * crnt_lib.NUM_K)
        assert crnt_lib.tune_shape_get() == [1] * crnt_lib.NUM_K
        crnt_lib.tune_shape_set([2] * crnt_lib.NUM_K)
        assert crnt_lib.tune_shape_get() == [2] * crnt_lib.NUM_K
        with pytest.raises(crnt_lib.CrntError):
            crnt_lib.tune_shape_set([3] * crnt_lib.NUM_K)
    finally:
        crnt_lib.tune_shape_set(old)


@pytest.mark.parametrize("P", [1, 8, 64, 128])
def test_pairs_single_cb_workload(orc, crnt_lib, ctx, pairs, P):
    # four K = 6144 CBs at Eb/N0 1 dB: two pair items, both lanes bit-exact
    tbs, llrs = batch(orc, [dict(A=6120, G=18444, Qm=2, P=P, max_iter=6, early_stop=0, seed=s,
                                 ebn0=1.0) for s in range(4)])
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    assert g["info"]["pair_items"] == 2
    check_batch(orc, crnt_lib, tbs, llrs, g)


def test_pairs_mixed_batch(orc, crnt_lib, ctx, pairs):
    # every CB size class, ragged windows, odd CB counts per (K, P) (one CB
    # of a size runs alone), early stop on some TBs and off on others -- so
    # the two CBs of a pair stop at different iterations and the survivor
    # continues on the one-CB path -- and different iteration limits
    shapes = synth.tti_batch(seed=37, n_tb=40, amax=30000)
    shapes += synth.tti_batch(seed=38, n_tb=4, amin=60000)
    specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=4 + (i % 4),
                  early_stop=1 if i % 3 else 0, rv=i % 4, seed=400 + i, snr=s["snr_db"])
             for i, s in enumerate(shapes)]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    assert g["info"]["pair_items"] > 10
    check_batch(orc, crnt_lib, tbs, llrs, g)


def test_pairs_full_tti(orc, crnt_lib, ctx, pairs):
    # the benchmark's workload with CB pairs: all 320 TBs against the oracle
    shapes = synth.tti_batch(seed=1, n_tb=320)
    specs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=6, early_stop=0, seed=300 + i,
                  snr=s["snr_db"]) for i, s in enumerate(shapes)]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    assert g["info"]["pair_items"] > 1000
    check_batch(orc, crnt_lib, tbs, llrs, g)


def test_pairs_fallback_to_one_cb(orc, crnt_lib, ctx, pairs):
    # +-127 noiseless inputs drive the extrinsics to ~2600: the first and
    # last windows can no longer be proved to fit 16-bit lanes (and later not
    # clamp-free either), so those passes run one CB at a time, some on the
    # saturating path; everything stays bit-exact
    specs = [dict(A=6120, G=18444, Qm=2, P=P, max_iter=8, early_stop=0, seed=70 + s,
                  noiseless=True, amp=127) for P in (2, 64) for s in range(2)]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    assert g["info"]["pair_items"] == 2
    check_batch(orc, crnt_lib, tbs, llrs, g)
    assert all(r["sat_passes"] > 0 for r in g["res"])


def test_pairs_purge_and_mi_rule(orc, crnt_lib, ctx, pairs):
    # purge on failure and the mutual-information stop rule inside pairs
    specs = []
    for i in range(8):
        specs.append(dict(A=75376, G=86400, Qm=6, max_iter=6, early_stop=1,
                          flags=crnt_lib.F_PURGE, seed=900 + i, snr=6.0 if i % 2 else 22.0))
    specs += [dict(A=6120, G=18444, Qm=2, P=64, max_iter=8, early_stop=2, seed=990 + i,
                   ebn0=0.5 + 0.25 * i) for i in range(4)]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs), debug=False)
    assert g["info"]["pair_items"] > 10
    off = np.cumsum([0] + [t["A"] // 8 for t in tbs])
    for t in range(len(tbs)):
        cbs, bits, ok, _ = oracle_tb(orc, crnt_lib, tbs[t], llrs[t])
        r = g["res"][t]
        assert r["tb_crc_ok"] == ok
        if ok:
            assert np.array_equal(np.unpackbits(g["out"][off[t]:off[t + 1]]), bits)
            assert r["cb_iters"] == [c[3] for c in cbs]
        for c, it, crc in zip(cbs, r["cb_iters"], r["cb_crc_ok"]):
            if it == 0:
                assert tbs[t].get("flags") and not ok and not crc
            else:
                assert it == c[3] and crc == (c[3] <= tbs[t]["max_iter"])
    mi = slice(8, 12)
    check_batch(orc, crnt_lib, tbs[mi], llrs[mi], run_gpu(crnt_lib, ctx, tbs[mi],
                                                          np.concatenate(llrs[mi])))


def test_pairs_harq(orc, crnt_lib, ctx, pairs):
    # HARQ combining into the soft buffers of two CBs decoded as a pair
    A, G, Qm = 2000, 2400, 2
    key = lambda u: dict(cell=5, ue=u, harq_pid=1, flags=crnt_lib.F_HARQ)
    a = [synth.bits(50 + u, 100, A) for u in range(2)]
    sig = synth.sigma2_snr(1.0)
    l0 = [synth.channel_llrs(orc.encode_tb(a[u], G, Qm=Qm, rv=0), 2, sig, 50 + u, 1)
          for u in range(2)]
    l2 = [synth.channel_llrs(orc.encode_tb(a[u], G, Qm=Qm, rv=2), 2, sig, 50 + u, 2)
          for u in range(2)]
    t0 = [dict(A=A, G=G, Qm=Qm, rv=0, new_data=1, P=16, **key(u)) for u in range(2)]
    t2 = [dict(A=A, G=G, Qm=Qm, rv=2, new_data=0, P=16, **key(u)) for u in range(2)]
    g0 = run_gpu(crnt_lib, ctx, t0, np.concatenate(l0))
    assert g0["info"]["pair_items"] == 1
    check_batch(orc, crnt_lib, t0, l0, g0)
    g2 = run_gpu(crnt_lib, ctx, t2, np.concatenate(l2))
    for u in range(2):
        _, _, _, soft = oracle_tb(orc, crnt_lib, t0[u], l0[u])
        _, bits2, ok2, _ = oracle_tb(orc, crnt_lib, t2[u], l2[u], soft=soft)
        assert g2["res"][u]["tb_crc_ok"] == ok2
        if ok2:
            assert np.array_equal(np.unpackbits(g2["out"][u * (A // 8):(u + 1) * (A // 8)]), bits2)
        assert ctx.harq_release(5, u, 1) == 0


def test_pairs_joint_derate_matching(orc, crnt_lib, ctx, pairs):
    # pairs whose two CBs share a de-rate-matching map are de-rate-matched in
    # one pass over it: here with different redundancy versions, with
    # repetition (E = 19200 > Nv = 18444 at K = 6144, both CBs' LLRs still
    # staged side by side), and next to a pair whose maps differ (a TB's
    # first CB with filler bits beside one without) -- every d-stream,
    # extrinsic and payload bit-exact
    specs = [dict(A=6120, G=19200, Qm=2, P=128, rv=rv, max_iter=4, early_stop=0, seed=1300 + i,
                  ebn0=1.5) for i, rv in enumerate((0, 2, 3, 1))]
    specs += [dict(A=12200, G=36000, Qm=2, P=0, max_iter=4, early_stop=0, seed=1310, ebn0=1.5)]
    tbs, llrs = batch(orc, specs)
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(llrs))
    assert g["info"]["pair_items"] >= 2
    check_batch(orc, crnt_lib, tbs, llrs, g)
