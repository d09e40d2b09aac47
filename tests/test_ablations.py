"""The paper's reduction alternatives (Sec. 3.1.3), rebuilt from the
committed compile-time switch of the recursion kernel: shuffle butterfly for
every group size, shared-memory column sums for every group, and cross-warp
direct atomics. Each build must still give the oracle's SNR (Eqs. iireq0,
iireq1; Sec. 2.2) on banks whose units take every reduction path: groups of
1-32 lanes and units spanning 2-4 warps, single and multi-rate. Each build
runs in a process of its own (a process loads one libspiir)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHECK = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_1702_02256_gb300 import inputs
from oracle import oracle
from tests._util import gpu_snr, rel_rms
out = {}
single = inputs.single_rate_bank(9, [1, 3, 8, 20, 40, 100, 300, 700, 1000], 900, seed=5)
x = inputs.strain(1, 2 * 4096, seed=6)
z = gpu_snr(single, x, push_blocks=1)[0]
out["single"] = float(rel_rms(z, oracle.spiir_single(single, x[0])).max())
multi = inputs.multi_rate_bank(12, 5, seed=7, count_range=(2.0, 700.0))
z = gpu_snr(multi, x, push_blocks=1)[0]
out["multi"] = float(rel_rms(z, oracle.spiir_multirate(multi, x[0])).max())
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def ablation_libs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_02256_gb300 import build
    return build.build_ablations(["shuffle", "smem", "atomics"])


@pytest.mark.parametrize("name", ["shuffle", "smem", "atomics"])
def test_reduction_ablation_matches_oracle(ablation_libs, oracle_mod, name):
    env = dict(os.environ, SPIIR_LIB=ablation_libs[name])
    r = subprocess.run([sys.executable, "-c", _CHECK.replace("ROOT", repr(ROOT))], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    err = json.loads(r.stdout.strip().splitlines()[-1])
    assert err["single"] <= 1e-5 and err["multi"] <= 1e-5, err
