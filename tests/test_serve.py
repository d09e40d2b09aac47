"""Serving loop: admission by HBM footprint, residency, retirement (CPU, with
test doubles), and on the GPU: each request's SNR is the same alone and in a
mix of concurrently served requests."""
import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs, serve


class FakeBank:
    def __init__(self, req):
        self.req = req
        self.pushed = 0
        self.closed = False

    def push(self, x, **kw):
        self.pushed += 1

    def close(self):
        self.closed = True


def _req(rid, T, arrival, life):
    bank = inputs.single_rate_bank(T, 4, 10, seed=rid)
    return serve.Request(rid=rid, bank=bank, arrival_block=arrival, lifetime=life)


def test_admission_budget_order_and_retirement():
    fp = lambda r: 100 * r.bank.n_templates
    made = {}

    def make(r):
        made[r.rid] = FakeBank(r)
        return made[r.rid]

    s = serve.Server(hbm_budget=1000, n_streams=3, block_len=16, make_bank=make, footprint=fp,
                     use_cuda=False)
    assert s.submit(_req(0, 6, 0, 2))      # 600 bytes
    assert s.submit(_req(1, 5, 0, 3))      # 500: must wait for 0 to retire
    assert s.submit(_req(2, 1, 0, 1))      # 100: fits, but may not overtake 1
    assert not s.submit(_req(3, 11, 0, 1)) # above the whole budget: rejected
    assert s.rejected == [3]
    r = s.step(None)
    assert r["active"] == [0] and r["pending"] == 2
    r = s.step(None)
    assert r["active"] == [0]              # 0 runs its 2 blocks, then retires
    assert made[0].closed and made[0].pushed == 2
    r = s.step(None)
    assert r["active"] == [1, 2] and r["used_bytes"] == 600 and s.used == 500
    r = s.step(None)
    assert r["active"] == [1]              # 2 retired after one block
    assert made[2].pushed == 1
    s.step(None)
    assert made[1].pushed == 3 and s.active == [] and s.used == 0


def test_arrivals_wait_for_their_block():
    s = serve.Server(10**9, 1, 16, make_bank=FakeBank, footprint=lambda r: 1, use_cuda=False)
    s.submit(_req(0, 2, 3, 1))
    for b in range(3):
        assert s.step(None)["active"] == []
    assert s.step(None)["active"] == [0]


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["plain", "fp16"])
def test_request_alone_equals_request_in_mix(form):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    block = 2048
    x = torch.from_numpy(inputs.strain(3, 6 * block, seed=9)).cuda()
    if form == "plain":
        banks = [inputs.multi_rate_bank(5, 3, seed=40 + i) for i in range(3)]
    else:
        banks = [inputs.single_rate_bank(7 + 3 * i, 40, 300, seed=40 + i) for i in range(3)]
    spec = [(0, 5), (1, 3), (2, 4)]      # (arrival block, lifetime): overlapping

    def run(which):
        make, fp = serve.device_bank_factory(form, block_len=block, n_streams=3)
        s = serve.Server(10**11, 3, block, make, fp)
        for i in which:
            s.submit(serve.Request(i, banks[i], spec[i][0], spec[i][1], keep_snr=True))
        for b in range(6):
            s.step(x[:, b * block:(b + 1) * block].contiguous())
        s.drain()
        return {i: np.stack(s.finished[i].snr) for i in which if i in s.finished}

    mix = run([0, 1, 2])
    for i in range(3):
        alone = run([i])
        assert np.array_equal(mix[i], alone[i]), i
    # and each request's SNR is the oracle's for the strain it saw: its bank
    # starts from zero state at its first block
    from oracle import oracle
    from tests._util import TOL_PLAIN, TOL_TC, rel_rms
    xh = x.cpu().numpy()
    tol = TOL_PLAIN if form == "plain" else TOL_TC
    for i in range(3):
        first, life = spec[i]
        z = np.concatenate(list(mix[i]), axis=-1)          # [3, T, life * block]
        seg = xh[:, first * block:(first + life) * block]
        for s in range(3):
            if form == "plain":
                ref = oracle.spiir_multirate(banks[i], seg[s])
            else:
                ref = oracle.spiir_single(banks[i], seg[s])
            err = rel_rms(z[s], ref)
            assert err.max() <= tol, (i, s, float(err.max()))
