"""GPU parity of the downlink encoder + rate matcher (crnt_encode_batch)
against the oracle encoder: every coded bit equal (integer work,
tolerance 0).  Host and device buffers are both exercised."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = crnt_lib.Context(0)
    yield c
    c.close()


def shapes():
    out = [(6120, 18444, 2, 1, 0), (75376, 86400, 6, 1, 0), (16, 132, 2, 1, 0),
           (16, 1200, 2, 1, 1), (6128, 13000, 2, 1, 2), (40000, 60000, 4, 2, 3),
           (1000, 1004, 4, 1, 0)]
    for i, s in enumerate(synth.tti_batch(seed=21, n_tb=30)):
        out.append((s["A"], s["G"], s["Qm"], 1, i % 4))
    return out


def test_encode_matches_oracle(orc, crnt_lib, ctx):
    tbs, payloads, want = [], [], []
    for i, (A, G, Qm, NL, rv) in enumerate(shapes()):
        a = synth.bits(30 + i, 1, A)
        tbs.append(dict(A=A, G=G, Qm=Qm, NL=NL, rv=rv))
        payloads.append(np.packbits(a))
        want.append(orc.encode_tb(a, G, Qm=Qm, NL=NL, rv=rv))
    bits = np.concatenate(payloads)
    want = np.concatenate(want)
    # host buffers
    e = np.zeros(len(want), dtype=np.uint8)
    ctx.encode_batch(tbs, bits, e)
    bad = np.nonzero(e != want)[0]
    assert len(bad) == 0, (len(bad), bad[:5])
    # device buffers
    bd = torch.from_numpy(bits).cuda()
    ed = torch.zeros(len(want), dtype=torch.uint8, device="cuda")
    ctx.encode_batch(tbs, bd, ed)
    torch.cuda.synchronize()
    assert np.array_equal(ed.cpu().numpy(), want)
    # page-locked host buffers, read and written in place by the kernel
    bp = torch.from_numpy(bits).pin_memory()
    ep = torch.zeros(len(want), dtype=torch.uint8).pin_memory()
    ctx.encode_batch(tbs, bp, ep)
    assert np.array_equal(ep.numpy(), want)


def test_encode_decode_round_trip(crnt_lib, ctx):
    # product encoder -> noiseless LLRs -> product decoder recovers the bits
    specs = synth.tti_batch(seed=5, n_tb=20)
    tbs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"]) for s in specs]
    pay = [np.packbits(synth.bits(i, 2, t["A"])) for i, t in enumerate(tbs)]
    bits = np.concatenate(pay)
    e = np.zeros(sum(t["G"] for t in tbs), dtype=np.uint8)
    ctx.encode_batch(tbs, bits, e)
    llr = np.where(e == 0, 60, -60).astype(np.int8)
    out = np.zeros(len(bits), dtype=np.uint8)
    res = ctx.decode_batch([dict(t, max_iter=4) for t in tbs], llr, out)
    # (punctured high-rate blocks may need several iterations even without noise)
    assert all(r["tb_crc_ok"] for r in res)
    assert np.array_equal(out, bits)
