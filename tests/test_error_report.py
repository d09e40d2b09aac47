"""Per-dtype SNR error of every form against the FP64 oracle (config-3-shaped
bank, 2 streams). Prints one line per form; asserts each form's bound."""
import numpy as np
import pytest

from paper_1702_02256_gb300 import inputs
from tests._util import TOL_PLAIN, TOL_TC, gpu_snr, rel_rms

pytestmark = pytest.mark.gpu


def test_error_per_dtype(oracle_mod, capsys):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = inputs.workload(3, scale_templates=64, n_samples=4 * 4096)
    refs = [oracle_mod.spiir_single(w["bank"], w["x"][s]) for s in range(2)]
    bounds = {"plain": TOL_PLAIN, "fp16": TOL_TC, "bf16": 1e-2, "bf16x2": TOL_TC}
    lines = []
    for mode, tol in bounds.items():
        kw = {} if mode == "plain" else dict(mode=mode, chunk_len=256)
        z = gpu_snr(w["bank"], w["x"], push_blocks=1, n_streams=2, **kw)
        err = np.concatenate([rel_rms(z[s], refs[s]) for s in range(2)])
        lines.append(f"SNR error vs FP64 oracle [{mode}]: max {err.max():.3e} "
                     f"median {np.median(err):.3e} over {err.size} template-streams")
        assert err.max() <= tol
    with capsys.disabled():
        print("\n" + "\n".join(lines))
