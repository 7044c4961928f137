"""The launch gate (crnt_plan_launch_gated): a decode enqueued before its
LLRs are ready waits, bounded on the GPU clock, for a ready word.  A word
that nothing sets makes the wait expire: every TB reports CRNT_ETIMEDOUT
and the context decodes the next launch normally.  A word the host sets
after the launch releases a decode identical to an ungated one."""
import time

import numpy as np
import pytest

import synth
from gpu_helpers import make_tb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup(orc, crnt_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = crnt_lib.Context(0)
    shapes = synth.tti_batch(seed=61, n_tb=24, amax=40000)
    tbs, llrs = [], []
    for i, s in enumerate(shapes):
        tbs.append(dict(A=s["A"], G=s["G"], Qm=s["Qm"], max_iter=6, early_stop=1))
        llrs.append(make_tb(orc, s["A"], s["G"], s["Qm"], 610 + i, snr=s["snr_db"])[1])
    dev = torch.device("cuda")
    llr = torch.from_numpy(np.concatenate(llrs)).to(dev)
    nbytes = sum(t["A"] // 8 for t in tbs)
    plan = crnt_lib.Plan(ctx, tbs)
    out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    plan.launch(llr, out)
    want = [r for r in plan.results()]
    want_bits = out.cpu().numpy().copy()
    yield ctx, plan, llr, nbytes, want, want_bits
    plan.close()
    ctx.close()


def test_gate_that_nobody_opens_expires(crnt_lib, setup):
    ctx, plan, llr, nbytes, want, want_bits = setup
    dev = torch.device("cuda")
    ready = torch.zeros(1, dtype=torch.int32, device=dev)  # never set
    out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t0 = time.time()
    plan.launch_gated(llr, out, ready, 20000)  # 20 ms
    res = plan.results()
    assert time.time() - t0 < 5.0
    assert all(r["status"] == crnt_lib.ETIMEDOUT for r in res)
    assert not out.any()  # nothing decoded
    # the context and the plan stay usable: the next launch decodes normally
    plan.launch(llr, out)
    res = plan.results()
    assert [r["status"] for r in res] == [0] * len(res)
    assert [(r["cb_iters"], r["tb_crc_ok"]) for r in res] == \
        [(r["cb_iters"], r["tb_crc_ok"]) for r in want]
    assert np.array_equal(out.cpu().numpy(), want_bits)


def test_gate_opened_by_the_host_releases_the_decode(crnt_lib, setup):
    ctx, plan, llr, nbytes, want, want_bits = setup
    dev = torch.device("cuda")
    ready = torch.zeros(1, dtype=torch.int32).pin_memory()  # page-locked host word
    out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    plan.launch_gated(llr, out, ready, 2_000_000)  # 2 s
    time.sleep(0.005)
    ready.fill_(1)  # the host's store; the decode starts on seeing it
    res = plan.results()
    assert [r["status"] for r in res] == [0] * len(res)
    assert [(r["cb_iters"], r["cb_iters_run"], r["tb_crc_ok"]) for r in res] == \
        [(r["cb_iters"], r["cb_iters_run"], r["tb_crc_ok"]) for r in want]
    assert np.array_equal(out.cpu().numpy(), want_bits)


def test_gate_arguments_checked(crnt_lib, setup):
    ctx, plan, llr, nbytes, _, _ = setup
    dev = torch.device("cuda")
    ready = torch.ones(1, dtype=torch.int32, device=dev)
    out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    for us in (0, 10_000_001):
        with pytest.raises(crnt_lib.CrntError) as ei:
            plan.launch_gated(llr, out, ready, us)
        assert ei.value.code == crnt_lib.EINVAL
    # a PUSCH-order batch cannot be gated (its front stage reads the LLRs first)
    t = dict(A=1000, G=2 * 2 * 600, Qm=2, flags=crnt_lib.F_PUSCH, c_init=5, n_symb=1)
    pp = crnt_lib.Plan(ctx, [t])
    with pytest.raises(crnt_lib.CrntError) as ei:
        pp.launch_gated(torch.zeros(2400, dtype=torch.int8, device=dev), out, ready, 1000)
    assert ei.value.code == crnt_lib.EINVAL
    pp.close()
