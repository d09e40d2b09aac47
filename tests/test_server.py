"""The batched server (spiir_server_t, serve.BatchedServer): many banks in one
push per block.

CPU: admission and retirement drive the engine's add/remove in arrival order.
GPU: a member that joins before the first push gives the oracle's SNR
(Eqs. iireq0, iireq1; Sec. 2.2 for multi-rate members); every member's SNR is
the same bit for bit alone and in a mix whose membership changes from block
to block (members join and leave, pools grow and reuse freed ranges); a
single-rate member that joins later gives the oracle's SNR for a filter state
that starts at zero at its first block while its delayed inputs read the
continuous strain history."""
import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs, serve
from tests._util import TOL_PLAIN, rel_rms


class FakeEngine:
    def __init__(self):
        self.members = {}
        self.next = 0
        self.calls = []

    def member_footprint(self, bank):
        return 100 * bank.n_templates

    def add(self, bank):
        mid = self.next
        self.next += 1
        self.members[mid] = bank
        self.calls.append(("add", mid))
        return mid

    def remove(self, mid):
        del self.members[mid]
        self.calls.append(("remove", mid))

    def push(self, x):
        self.calls.append(("push", sorted(self.members)))

    def read(self, mid, out=None):
        return mid


def _req(rid, T, arrival, life, **kw):
    return serve.Request(rid, inputs.single_rate_bank(T, 4, 10, seed=rid), arrival, life, **kw)


def test_batched_admission_and_retirement_drive_the_engine():
    eng = FakeEngine()
    s = serve.BatchedServer(1000, 3, 16, eng, use_cuda=False)
    assert s.submit(_req(0, 6, 0, 2))
    assert s.submit(_req(1, 5, 0, 3))          # must wait for 0 to retire
    assert s.submit(_req(2, 1, 1, 1))
    assert not s.submit(_req(3, 11, 0, 1))     # above the budget
    for _ in range(6):
        s.step(None)
    pushes = [c[1] for c in eng.calls if c[0] == "push"]
    assert pushes == [[0], [0], [1, 2], [1], [1]]
    assert ("remove", 0) in eng.calls and eng.members == {}
    assert s.used == 0


# --------------------------------------------------------------------------- GPU


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(banks, spec, x, block, n_levels, max_delay, **kw):
    """Serve banks[i] from block spec[i][0] for spec[i][1] blocks; return each
    member's SNR [n_streams, T, lifetime * block]."""
    from paper_1702_02256_gb300 import spiir
    S = x.shape[0]
    n_blocks = x.shape[1] // block
    srv = spiir.Server(S, n_levels, block, max_delay, **kw)
    ids, outs = {}, {i: [] for i in range(len(banks))}
    for b in range(n_blocks):
        for i, (first, life) in enumerate(spec):
            if b == first:
                ids[i] = srv.add(banks[i])
            if i in ids and b == first + life:
                srv.remove(ids.pop(i))
        srv.push(x[:, b * block:(b + 1) * block].contiguous())
        for i, mid in ids.items():
            outs[i].append(srv.read(mid).cpu().numpy())
    srv.sync_status()
    srv.close()
    return {i: np.concatenate(v, axis=-1) for i, v in outs.items() if v}


@pytest.mark.gpu
def test_members_from_the_first_block_match_the_oracle(torch_cuda, oracle_mod):
    """Three multi-rate members (7 rates) and two single-rate ones cannot share
    a server; each kind gets its own. Three streams, 3 blocks of 4096."""
    import torch
    block = 4096
    x = torch.from_numpy(inputs.strain(3, 3 * block, seed=61)).cuda()
    xh = x.cpu().numpy()
    multi = [inputs.multi_rate_bank(T, 7, seed=70 + T) for T in (3, 9, 5)]
    z = _run(multi, [(0, 3)] * 3, x, block, 7, 1023)
    for i, bank in enumerate(multi):
        for s in range(3):
            ref = oracle_mod.spiir_multirate(bank, xh[s])
            assert rel_rms(z[i][s], ref).max() <= TOL_PLAIN, (i, s)
    # single rate: a template of 1200 filters is split into parts (combine
    # pass), the others write their rows directly
    single = [inputs.single_rate_bank(4, [1200, 3, 0, 64], 1023, seed=81),
              inputs.single_rate_bank(6, 40, 500, seed=82)]
    z = _run(single, [(0, 3)] * 2, x, block, 1, 1023)
    for i, bank in enumerate(single):
        for s in range(3):
            ref = oracle_mod.spiir_single(bank, xh[s])
            got = z[i][s]
            assert rel_rms(got, ref).max() <= TOL_PLAIN, (i, s)
    assert np.all(z[0][:, 2] == 0)                      # template without filters


@pytest.mark.gpu
@pytest.mark.parametrize("n_levels", [1, 4])
def test_member_alone_equals_member_in_a_changing_mix(torch_cuda, n_levels):
    import torch
    block = 2048
    n_blocks = 8
    x = torch.from_numpy(inputs.strain(2, n_blocks * block, seed=63)).cuda()
    if n_levels == 1:
        banks = [inputs.single_rate_bank(T, M, 700, seed=90 + T) for T, M in
                 [(5, 64), (40, 300), (3, 1500), (17, 8), (60, 128)]]
    else:
        banks = [inputs.multi_rate_bank(T, 4, seed=90 + T, delay_max=700) for T in (5, 40, 3, 17, 60)]
    # joins and leaves at different blocks; member 4 joins after 1 leaves so
    # it can reuse (part of) 1's ranges, member 3 outgrows the pools
    spec = [(0, 8), (0, 3), (1, 5), (2, 6), (4, 4)]
    mix = _run(banks, spec, x, block, n_levels, 700)
    for i in range(len(banks)):
        only = [(spec[j] if j == i else (n_blocks + 1, 0)) for j in range(len(banks))]
        alone = _run(banks, only, x, block, n_levels, 700)
        assert np.array_equal(mix[i], alone[i]), i


@pytest.mark.gpu
def test_late_single_rate_member_against_the_oracle(torch_cuda, oracle_mod):
    """A member joining at block 2: y_k = 0 before its first sample n0, then
    y_k[n] = a_k y_k[n-1] + b_k x[n - d_k] with x the continuous strain."""
    import torch
    block = 4096
    x = torch.from_numpy(inputs.strain(1, 5 * block, seed=64)).cuda()
    xh = x.cpu().numpy()
    early = inputs.single_rate_bank(4, 100, 1023, seed=95)
    late = inputs.single_rate_bank(5, [3, 200, 64, 1, 700], 1023, seed=96)
    z = _run([early, late], [(0, 5), (2, 3)], x, block, 1, 1023)
    ref = oracle_mod.spiir_single_from(late, xh[0], start=2 * block)
    assert rel_rms(z[1][0], ref[:, 2 * block:]).max() <= TOL_PLAIN


@pytest.mark.gpu
@pytest.mark.parametrize("mode,tc_min", [("fp16", 1), ("fp16", 24), ("bf16", 24)])
def test_block_form_members_match_the_oracle(torch_cuda, oracle_mod, mode, tc_min):
    """Tensor-core server, 7 rates: at levels 0-4 (4096-256 samples per
    block) the templates with at least tc_min filters there run in the block
    form batched over all members, the others (and levels 5-6) in the plain
    form; members present from the first push against the FP64 oracle at the
    block form's tolerance (fp16; single-pass bf16 at its looser bound)."""
    import torch
    from paper_1702_02256_gb300 import spiir
    from tests._util import TOL_TC
    tol = TOL_TC if mode == "fp16" else 1e-2
    block = 4096
    x = torch.from_numpy(inputs.strain(3, 3 * block, seed=65)).cuda()
    xh = x.cpu().numpy()
    banks = [inputs.multi_rate_bank(T, 7, seed=170 + T) for T in (3, 70, 5)]
    srv = spiir.Server(3, 7, block, 1023, mode=mode, chunk_len=256, tc_min_filters=tc_min)
    ids = [srv.add(b) for b in banks]
    out = {i: [] for i in ids}
    for b in range(3):
        srv.push(x[:, b * block:(b + 1) * block].contiguous())
        for i in ids:
            out[i].append(srv.read(i).cpu().numpy())
    info = srv.info()
    srv.sync_status()
    srv.close()
    assert info["tc_levels"] == 5
    for i, bank in zip(ids, banks):
        z = np.concatenate(out[i], axis=-1)
        for s in range(3):
            ref = oracle_mod.spiir_multirate(bank, xh[s])
            assert rel_rms(z[s], ref).max() <= tol, (i, s)


@pytest.mark.gpu
def test_block_form_member_alone_equals_member_in_a_changing_mix(torch_cuda):
    import torch
    block = 2048
    n_blocks = 7
    x = torch.from_numpy(inputs.strain(3, n_blocks * block, seed=66)).cuda()
    banks = [inputs.multi_rate_bank(T, 4, seed=190 + T, delay_max=900) for T in (5, 80, 3, 17, 130)]
    spec = [(0, 7), (0, 3), (1, 5), (2, 5), (4, 3)]
    kw = dict(mode="fp16", chunk_len=256, tc_min_filters=40)
    mix = _run(banks, spec, x, block, 4, 900, **kw)
    for i in range(len(banks)):
        only = [(spec[j] if j == i else (n_blocks + 1, 0)) for j in range(len(banks))]
        alone = _run(banks, only, x, block, 4, 900, **kw)
        assert np.array_equal(mix[i], alone[i]), i


@pytest.mark.gpu
def test_server_rejects_bad_requests(torch_cuda):
    """Wrong rate count or a delay above max_delay: EINVAL at add; an unknown
    member: EINVAL; a member that has not taken part in a push yet: ESTATE;
    removing it before its first push leaves no trace; pushes without
    members keep the strain moving; split bf16 is a bank mode only."""
    import torch
    from paper_1702_02256_gb300 import spiir
    with pytest.raises(spiir.SpiirError) as e:
        spiir.Server(2, 3, 1024, 200, mode="bf16x2")
    assert e.value.status == spiir.EUNSUPPORTED
    srv = spiir.Server(2, 3, 1024, 200)
    with pytest.raises(spiir.SpiirError) as e:
        srv.add(inputs.multi_rate_bank(3, 4, seed=1, delay_max=100))
    assert e.value.status == spiir.EINVAL
    with pytest.raises(spiir.SpiirError) as e:
        srv.add(inputs.multi_rate_bank(3, 3, seed=1, delay_max=300))
    assert e.value.status == spiir.EINVAL and "max_delay" in str(e.value)
    x = torch.zeros((2, 1024), dtype=torch.float32, device="cuda")
    srv.push(x)
    mid = srv.add(inputs.multi_rate_bank(3, 3, seed=2, delay_max=200))
    with pytest.raises(spiir.SpiirError) as e:
        srv.read(mid)
    assert e.value.status == spiir.ESTATE
    srv.remove(mid)
    with pytest.raises(spiir.SpiirError) as e:
        srv.remove(mid)
    assert e.value.status == spiir.EINVAL
    mid = srv.add(inputs.multi_rate_bank(3, 3, seed=3, delay_max=200))
    srv.push(x)
    assert srv.read(mid).shape == (2, 3, 1024)
    assert srv.info()["n_members"] == 1
    srv.sync_status()
    srv.close()
