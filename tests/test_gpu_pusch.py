"""GPU parity of the PUSCH front stage (descrambling with the length-31 Gold
sequence, data-only channel de-interleaver; the demultiplexing ahead of the
decoder in Sec. IV-B) against the CPU oracle, through the C ABI: the
encoder's transmit direction bit by bit, and decoding from received PUSCH
order with the de-rate-matched streams, extrinsics, hard decisions,
iteration counts and payloads bit-exact."""
import numpy as np
import pytest

import synth
from gpu_helpers import check_batch, oracle_batch, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = crnt_lib.Context(0)
    yield c
    c.close()


def pusch_inputs(orc, crnt_lib, shapes, seed, noiseless=False, pusch=None):
    """TB parameters, received LLRs (transmitted order) and the e-sequence
    LLRs the oracle's receiver recovers from them."""
    tbs, rx, e_llr = [], [], []
    for i, s in enumerate(shapes):
        on = pusch is None or pusch[i]
        NL = s.get("NL", 1)
        tb = dict(A=s["A"], G=s["G"], Qm=s["Qm"], NL=NL, P=0, max_iter=6, early_stop=i % 2,
                  flags=crnt_lib.F_PUSCH if on else 0, c_init=s["c_init"],
                  n_symb=s.get("n_symb", 12))
        a = synth.bits(seed, 100 + i, s["A"])
        e = orc.encode_tb(a, s["G"], Qm=s["Qm"], NL=NL)
        ncol = tb["n_symb"] or 12
        tx = orc.pusch_tx(e, s["Qm"] * NL, s["c_init"], ncol) if on else e
        if noiseless:
            llr = np.where(tx == 0, 100, -100).astype(np.int8)
        else:
            llr = synth.channel_llrs(tx, s["Qm"], synth.sigma2_snr(s["snr_db"]), seed, 200 + i)
        tbs.append(tb)
        rx.append(llr)
        e_llr.append(orc.pusch_rx(llr, s["Qm"] * NL, s["c_init"], ncol) if on else llr)
    return tbs, rx, e_llr


def small_shapes():
    # several chunks of 4096 positions, every modulation, two layers, other
    # column counts, the largest G (100 PRBs x 6 bits x 2 layers)
    return [dict(A=6120, G=144 * 2 * 60, Qm=2, c_init=1639431, snr_db=4.0),
            dict(A=20000, G=144 * 4 * 50, Qm=4, c_init=(1 << 31) - 1, snr_db=9.0),
            dict(A=75376, G=144 * 6 * 100, Qm=6, c_init=12345, snr_db=20.0),
            dict(A=16, G=144 * 2, Qm=2, c_init=0, snr_db=3.0),
            dict(A=40000, G=144 * 6 * 100, Qm=6, NL=2, c_init=777777, snr_db=8.0),
            dict(A=1000, G=10 * 2 * 90, Qm=2, c_init=424242, n_symb=10, snr_db=5.0),
            dict(A=1000, G=2 * 2 * 600, Qm=2, c_init=99, n_symb=1, snr_db=5.0)]


def test_encoder_transmit_order_matches_oracle(orc, crnt_lib, ctx):
    shapes = small_shapes()
    tbs, rx, _ = pusch_inputs(orc, crnt_lib, shapes, 3, noiseless=True,
                              pusch=[True, True, True, True, True, True, False])
    pay = np.concatenate([np.packbits(synth.bits(3, 100 + i, s["A"]))
                          for i, s in enumerate(shapes)])
    out = np.zeros(sum(s["G"] for s in shapes), dtype=np.uint8)
    ctx.encode_batch(tbs, pay, out)
    want = np.concatenate([(r < 0).astype(np.uint8) for r in rx])
    assert np.array_equal(out, want)
    dev = torch.device("cuda")
    out_d = torch.zeros(len(out), dtype=torch.uint8, device=dev)
    ctx.encode_batch(tbs, torch.from_numpy(pay).to(dev), out_d)
    assert np.array_equal(out_d.cpu().numpy(), want)


def test_decode_from_pusch_order_matches_oracle(orc, crnt_lib, ctx):
    shapes = small_shapes()
    tbs, rx, e_llr = pusch_inputs(orc, crnt_lib, shapes, 5,
                                  pusch=[True, True, True, True, True, True, False])
    rx[0][::97] = -128  # -128 reads as -127 before the sign flip
    e_llr[0] = orc.pusch_rx(rx[0], 2, shapes[0]["c_init"])
    g = run_gpu(crnt_lib, ctx, tbs, np.concatenate(rx))
    check_batch(orc, crnt_lib, tbs, e_llr, g)
    assert sum(r["tb_crc_ok"] for r in g["res"]) >= 3


def test_pusch_tti_through_decode_batch(orc, crnt_lib, ctx):
    # a TTI in PUSCH order (40 cells x 8 UEs shapes rounded to PRBs) through
    # crnt_decode_batch from host buffers (three chunks): every TB against
    # the oracle's receiver + decoder
    shapes = synth.pusch_batch(11, n_tb=64, amax=40000)
    tbs, rx, e_llr = pusch_inputs(orc, crnt_lib, shapes, 11)
    nbytes = sum(t["A"] // 8 for t in tbs)
    out = np.zeros(nbytes, dtype=np.uint8)
    res = ctx.decode_batch(tbs, np.concatenate(rx), out)
    want = oracle_batch(orc, crnt_lib, tbs, e_llr, range(len(tbs)))
    off = np.cumsum([0] + [t["A"] // 8 for t in tbs])
    for t in range(len(tbs)):
        cbs, bits, ok, _ = want[t]
        assert res[t]["tb_crc_ok"] == ok, t
        assert res[t]["cb_iters"] == [c[3] for c in cbs], t
        assert np.array_equal(np.unpackbits(out[off[t]:off[t + 1]]), bits), t
