"""crnt_decode_batch_static -- the decode for callers that cannot allocate
device memory -- gives the same output as crnt_decode_batch, bit for bit, on
two calls in a row (the second call reuses the fixed workspace the first one
left behind), and the same as the CPU oracle.  Kept in a file that pytest
collects last."""
import numpy as np
import pytest

import synth
from gpu_helpers import make_tb, oracle_batch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KEYS = ("status", "tb_crc_ok", "C", "Kp", "Km", "F", "cb_iters", "cb_crc_ok", "cb_iters_run",
        "P_used", "sat_passes")


def _batch(orc, seed, n, amax):
    shapes = synth.tti_batch(seed=seed, n_tb=n, amax=amax)
    tbs, llrs = [], []
    for i, s in enumerate(shapes):
        tbs.append(dict(A=s["A"], G=s["G"], Qm=s["Qm"], max_iter=6, early_stop=i % 3))
        llrs.append(make_tb(orc, s["A"], s["G"], s["Qm"], seed * 100 + i, snr=s["snr_db"])[1])
    return tbs, llrs


def _compare(crnt_lib, ctx, tbs, llr):
    dev = torch.device("cuda")
    llr_d = torch.from_numpy(llr).to(dev)
    nbytes = sum(t["A"] // 8 for t in tbs)
    out_static = torch.full((nbytes,), 0xA5, dtype=torch.uint8, device=dev)
    out_ref = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()  # inputs in place before the library's streams read them
    res_static = crnt_lib.decode_batch_static(tbs, llr_d, out_static)
    res_ref = ctx.decode_batch(tbs, llr_d, out_ref)
    torch.cuda.synchronize()
    assert np.array_equal(out_static.cpu().numpy(), out_ref.cpu().numpy())
    for a, b in zip(res_static, res_ref):
        assert {k: a[k] for k in KEYS} == {k: b[k] for k in KEYS}
    return res_static, out_static.cpu().numpy()


def test_static_decode_matches_existing_entry_point_twice(orc, crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with crnt_lib.Context(0) as ctx:
        # first call: small and mid-size TBs, all three stop rules; second
        # call: the largest TB sizes (13 code blocks) so it overwrites more of
        # the workspace, an explicit window count that is not a divisor
        # (P = 120 at K = 6144 runs 119 windows) and purge-on-failure TBs
        tbs1, llr1 = _batch(orc, 3, 12, 20000)
        _compare(crnt_lib, ctx, tbs1, np.concatenate(llr1))
        tbs2, llr2 = _batch(orc, 4, 6, 75376)
        extra = [(dict(A=75376, G=86400, Qm=6, max_iter=6, early_stop=1), 4242, 20.0),
                 (dict(A=6120, G=18444, Qm=2, P=120, max_iter=6, early_stop=1), 4243, 3.0),
                 (dict(A=75376, G=86400, Qm=6, max_iter=4, early_stop=1,
                       flags=crnt_lib.F_PURGE), 4244, 22.0)]
        for tb, seed, snr in extra:
            tbs2.append(tb)
            llr2.append(make_tb(orc, tb["A"], tb["G"], tb["Qm"], seed, snr=snr)[1])
        res, _ = _compare(crnt_lib, ctx, tbs2, np.concatenate(llr2))
        assert res[-2]["P_used"] == 119


def test_static_decode_matches_oracle(orc, crnt_lib):
    # directly against the oracle: iteration counts, CRC flags, payload bytes
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tbs, llrs = _batch(orc, 5, 16, 40000)
    dev = torch.device("cuda")
    llr_d = torch.from_numpy(np.concatenate(llrs)).to(dev)
    nbytes = sum(t["A"] // 8 for t in tbs)
    out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    res = crnt_lib.decode_batch_static(tbs, llr_d, out)
    out = out.cpu().numpy()
    want = oracle_batch(orc, crnt_lib, tbs, llrs, range(len(tbs)))
    off = np.cumsum([0] + [t["A"] // 8 for t in tbs])
    for t, tb in enumerate(tbs):
        cbs, bits, tb_ok, _ = want[t]
        assert res[t]["tb_crc_ok"] == tb_ok, t
        assert res[t]["cb_iters"] == [c[3] for c in cbs], t
        assert res[t]["cb_iters_run"] == [c[6] for c in cbs], t
        assert np.array_equal(np.unpackbits(out[off[t]:off[t + 1]]), bits), t


def test_static_decode_rejects_beyond_its_limits(crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda")
    llr = torch.zeros(65 * 132, dtype=torch.int8, device=dev)
    out = torch.zeros(65 * 2, dtype=torch.uint8, device=dev)
    with pytest.raises(crnt_lib.CrntError) as ei:
        crnt_lib.decode_batch_static([dict(A=16, G=132)] * 65, llr, out)
    assert ei.value.code == crnt_lib.ENOMEM
    for flags in (crnt_lib.F_HARQ, crnt_lib.F_PUSCH):
        with pytest.raises(crnt_lib.CrntError) as ei:
            crnt_lib.decode_batch_static([dict(A=16, G=144, flags=flags)], llr, out)
        assert ei.value.code == crnt_lib.EINVAL
    # pageable host buffers: refused before anything is launched
    llr_h = np.zeros(132, dtype=np.int8)
    out_h = np.zeros(2, dtype=np.uint8)
    for a, b in ((llr_h, out), (llr, out_h)):
        with pytest.raises(crnt_lib.CrntError) as ei:
            crnt_lib.decode_batch_static([dict(A=16, G=132)], a, b)
        assert ei.value.code == crnt_lib.EINVAL
