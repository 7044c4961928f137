"""crnt_decode_batch_static -- the decode for callers that cannot allocate
device memory -- gives the same output as crnt_decode_batch, bit for bit, on
two calls in a row (the second call reuses the fixed workspace the first one
left behind).  Kept in a file that pytest collects last."""
import numpy as np
import pytest

import synth
from gpu_helpers import make_tb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _batch(orc, seed, n, amax):
    shapes = synth.tti_batch(seed=seed, n_tb=n, amax=amax)
    tbs, llrs = [], []
    for i, s in enumerate(shapes):
        tbs.append(dict(A=s["A"], G=s["G"], Qm=s["Qm"], max_iter=6, early_stop=i % 2))
        llrs.append(make_tb(orc, s["A"], s["G"], s["Qm"], seed * 100 + i, snr=s["snr_db"])[1])
    return tbs, np.concatenate(llrs)


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
    keys = ("status", "tb_crc_ok", "C", "Kp", "Km", "F", "cb_iters", "cb_crc_ok", "P_used")
    for a, b in zip(res_static, res_ref):
        assert {k: a[k] for k in keys} == {k: b[k] for k in keys}


def test_static_decode_matches_existing_entry_point_twice(orc, crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with crnt_lib.Context(0) as ctx:
        # first call: small and mid-size TBs; second call: includes the largest
        # TB sizes (13 code blocks) so it overwrites more of the workspace
        tbs1, llr1 = _batch(orc, 3, 12, 20000)
        _compare(crnt_lib, ctx, tbs1, llr1)
        tbs2, llr2 = _batch(orc, 4, 6, 75376)
        tbs2.append(dict(A=75376, G=86400, Qm=6, max_iter=6, early_stop=1))
        llr2 = np.concatenate([llr2, make_tb(orc, 75376, 86400, 6, 4242, snr=20.0)[1]])
        _compare(crnt_lib, ctx, tbs2, llr2)


def test_static_decode_rejects_beyond_its_limits(crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda")
    llr = torch.zeros(65 * 132, dtype=torch.int8, device=dev)
    out = torch.zeros(65 * 2, dtype=torch.uint8, device=dev)
    with pytest.raises(crnt_lib.CrntError) as ei:
        crnt_lib.decode_batch_static([dict(A=16, G=132)] * 65, llr, out)
    assert ei.value.code == crnt_lib.ENOMEM
    with pytest.raises(crnt_lib.CrntError) as ei:
        crnt_lib.decode_batch_static([dict(A=16, G=132, flags=crnt_lib.F_HARQ)], llr, out)
    assert ei.value.code == crnt_lib.EINVAL
