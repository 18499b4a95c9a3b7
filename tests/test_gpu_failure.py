"""Device-side failure detection without a GPU fault: a tensor-core pipeline
wait that never completes runs out after its bounded number of polls, the
kernel reports SCOUP_ERR_TIMEOUT through its status word, and the context
stays usable (a normal decode afterwards is correct)."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13600_gb300 import build
    build.build()
    import paper_2605_13600_gb300 as gb
    return gb


def test_gemm_wait_timeout_reported_and_context_survives(gb, oracle_lib):
    import torch
    from paper_2605_13600_gb300._lib import SCOUP_ERR_TIMEOUT
    t0 = time.perf_counter()
    rc, msg = gb.scoup_selftest_gemm_timeout()
    elapsed = time.perf_counter() - t0
    assert rc == SCOUP_ERR_TIMEOUT, (rc, msg)
    assert elapsed < 30.0
    # the context is still usable: a normal decode gives the right answer
    rng = np.random.default_rng(1)
    W = rng.random((300, 64)).astype(np.float32) / 64
    B = synth.unit_rows(rng, 64, 32)
    out = torch.empty((300, 32), dtype=torch.float32, device="cuda")
    ws = gb.scoup_decode(torch.from_numpy(W).cuda(), torch.from_numpy(B).cuda(), out)
    assert gb.scoup_read_stats(ws)["status"] == 0
    torch.cuda.synchronize()
    Wb = torch.from_numpy(W).to(torch.bfloat16).double().numpy()
    Bb = torch.from_numpy(B).to(torch.bfloat16).double().numpy()
    ref = oracle_lib.decode(Wb, Bb.astype(np.float32))
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5
