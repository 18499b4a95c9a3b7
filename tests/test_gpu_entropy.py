"""GPU entropy (fused into Top-K), entropy filter and relevancy score vs the
FP64 oracle.  Inputs come from the oracle or from seeded draws; integer
decisions (the filter's kept set) are compared on identical float32 inputs."""
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


def test_topk_entropy_on_oracle_accumulator(gb, oracle_lib, cfg1, cfg1_oracle):
    import torch
    acc32 = cfg1_oracle["acc"].astype(np.float32)
    n, C = acc32.shape
    K = cfg1.K
    dev = torch.device("cuda:0")
    a = torch.from_numpy(acc32).to(dev)
    idx = torch.empty((n, K), dtype=torch.int32, device=dev)
    val = torch.empty((n, K), dtype=torch.float32, device=dev)
    H = torch.full((n,), -1.0, dtype=torch.float32, device=dev)
    gb.scoup_topk_entropy(a, K, idx, val, H)
    idx0 = torch.empty_like(idx)
    val0 = torch.empty_like(val)
    gb.scoup_topk(a, K, idx0, val0)
    torch.cuda.synchronize()
    # the fused entropy leaves the Top-K untouched
    assert torch.equal(idx, idx0) and torch.equal(val, val0)
    H_ora = oracle_lib.entropy(acc32.astype(np.float64))
    err = np.abs(H.cpu().numpy() - H_ora)
    assert err.max() <= 2e-5 * np.maximum(1.0, H_ora).max(), err.max()
    # compensated form: entropy of sum + compensation
    comp = (np.random.default_rng(0).standard_normal(acc32.shape) * 1e-7 * acc32).astype(np.float32)
    gb.scoup_topk_entropy(a, K, idx, val, H, comp=torch.from_numpy(comp).to(dev))
    torch.cuda.synchronize()
    H_c = oracle_lib.entropy(acc32.astype(np.float64) + comp.astype(np.float64))
    assert np.abs(H.cpu().numpy() - H_c).max() <= 2e-5 * np.maximum(1.0, H_c).max()


def test_entropy_after_gpu_uplift(gb, oracle_lib, cfg1, cfg1_oracle):
    """End to end: GPU uplift -> fused Top-K + entropy vs the oracle's entropy of
    its own accumulator (rows whose stop decisions are clear)."""
    import torch
    up = gb.Uplift(cfg1)
    up.run(topk=False)
    n = cfg1.scene.n
    H = torch.empty((n,), dtype=torch.float32, device="cuda")
    gb.scoup_topk_entropy(up.accum, cfg1.K, up.topk_idx, up.topk_val, H)
    torch.cuda.synchronize()
    H_ora = oracle_lib.entropy(cfg1_oracle["acc"])
    clear = ~(cfg1_oracle["risk"] > 0).any(axis=1)
    # a 1e-4 relative accumulator error moves H by at most ~2e-4 (1 + max |log p|)
    assert np.abs(H.cpu().numpy() - H_ora)[clear].max() <= 5e-3


@pytest.mark.parametrize("n", [1, 37, 5000])
def test_entropy_filter_exact(gb, oracle_lib, n):
    import torch
    rng = np.random.default_rng(n)
    H32 = np.round(rng.random(n) * 4.0, 1).astype(np.float32)  # many ties
    dev = torch.device("cuda:0")
    Hd = torch.from_numpy(H32).to(dev)
    K = 3
    for keep in sorted({0, 1, n // 2, max(0, n - 1), n, n + 5}):
        idx = torch.arange(n * K, dtype=torch.int32, device=dev).reshape(n, K)
        val = torch.ones((n, K), dtype=torch.float32, device=dev)
        mask = torch.full((n,), 7, dtype=torch.uint8, device=dev)
        gb.scoup_entropy_filter(Hd, keep, idx, val, mask)
        want = oracle_lib.entropy_filter(H32.astype(np.float64), keep)
        got = mask.cpu().numpy()
        np.testing.assert_array_equal(got, want)
        kept = want.astype(bool)
        assert (idx.cpu().numpy()[~kept] == -1).all() and (val.cpu().numpy()[~kept] == 0).all()
        assert (idx.cpu().numpy()[kept] >= 0).all()


def test_entropy_filter_in_a_cuda_graph(gb, oracle_lib):
    """The filter runs without host round-trips: captured once in a CUDA graph
    and replayed on new entropies, it keeps exactly the oracle's Gaussians."""
    import torch
    n, K, keep = 70_000, 4, 31_337
    rng = np.random.default_rng(71)
    dev = torch.device("cuda:0")
    Hd = torch.empty(n, dtype=torch.float32, device=dev)
    idx = torch.empty((n, K), dtype=torch.int32, device=dev)
    val = torch.empty((n, K), dtype=torch.float32, device=dev)
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    ws = torch.empty(int(gb.scoup_entropy_filter_workspace_size()), dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside the capture
        gb.scoup_entropy_filter(Hd.fill_(1.0), keep, idx, val, mask, workspace=ws)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        gb.scoup_entropy_filter(Hd, keep, idx, val, mask, workspace=ws)
    for trial in range(2):
        H32 = np.round(rng.random(n) * 3.0, 2).astype(np.float32)  # many ties
        Hd.copy_(torch.from_numpy(H32))
        idx.copy_(torch.arange(n * K, dtype=torch.int32).reshape(n, K))
        val.fill_(1.0)
        g.replay()
        torch.cuda.synchronize()
        want = oracle_lib.entropy_filter(H32.astype(np.float64), keep)
        np.testing.assert_array_equal(mask.cpu().numpy(), want)
        kept = want.astype(bool)
        assert kept.sum() == keep
        assert (idx.cpu().numpy()[~kept] == -1).all() and (idx.cpu().numpy()[kept] >= 0).all()


def test_relevancy_matches_oracle(gb, oracle_lib):
    import torch
    rng = np.random.default_rng(9)
    P, n_canon, Q = 3000, 4, 28
    sim = rng.uniform(-1, 1, (P, n_canon + Q)).astype(np.float32)
    sim[5, :] = 0.25  # query equal to every canonical phrase: R = 1/2
    R = torch.empty((P, Q), dtype=torch.float32, device="cuda")
    gb.scoup_relevancy(torch.from_numpy(sim).cuda(), n_canon, R, alpha=10.0)
    torch.cuda.synchronize()
    s64 = sim.astype(np.float64)
    want = np.stack([oracle_lib.relevancy(s64[:, n_canon + q], s64[:, :n_canon], 10.0) for q in range(Q)], axis=1)
    assert np.abs(R.cpu().numpy() - want).max() <= 2e-6
    assert np.allclose(R.cpu().numpy()[5], 0.5)


def test_relevancy_pipeline_bf16(gb, oracle_lib):
    """codes -> bf16 decode -> cosine to 4 canonical + 28 query vectors -> relevancy."""
    import torch
    rng = np.random.default_rng(10)
    P, C, D = 1500, 256, 512
    W = np.zeros((P, C), np.float32)
    for p in range(P):
        j = rng.choice(C, size=8, replace=False)
        W[p, j] = rng.random(8).astype(np.float32)
    B = synth.unit_rows(rng, C, D)
    T = synth.unit_rows(rng, 32, D)
    dev = torch.device("cuda:0")
    feats = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    n2 = torch.empty((P,), dtype=torch.float32, device=dev)
    gb.scoup_decode(torch.from_numpy(W).to(dev), torch.from_numpy(B).to(dev), feats, n2)
    sim = torch.empty((P, 32), dtype=torch.float32, device=dev)
    gb.scoup_similarity(feats, torch.from_numpy(T).to(dev), sim, feat_norm2=n2)
    R = torch.empty((P, 28), dtype=torch.float32, device=dev)
    gb.scoup_relevancy(sim, 4, R)
    torch.cuda.synchronize()
    S = oracle_lib.similarity(oracle_lib.decode(W.astype(np.float64), B), T)
    want = np.stack([oracle_lib.relevancy(S[:, 4 + q], S[:, :4], 10.0) for q in range(28)], axis=1)
    err = np.abs(R.cpu().numpy() - want)
    # dR/ds <= alpha / 4 per similarity; two similarities per term, each within the bf16 bound
    assert err.max() <= 1e-2 and err.mean() <= 1e-3
    # the same relevancy computed in the similarity GEMM's epilogue
    Rf = torch.empty((P, 28), dtype=torch.float32, device=dev)
    gb.scoup_similarity_relevancy(feats, torch.from_numpy(T).to(dev), 4, Rf, feat_norm2=n2)
    torch.cuda.synchronize()
    assert torch.equal(Rf, R)


@pytest.mark.parametrize("P,Q,n_canon", [(5037, 32, 4), (300, 16, 4), (1, 32, 8), (2900, 16, 12)])
def test_similarity_relevancy_epilogue_equals_two_calls(gb, P, Q, n_canon):
    """The fused form (relevancy in the similarity GEMM's epilogue) equals
    scoup_similarity followed by scoup_relevancy bit for bit: ragged row
    counts, rows of zero norm (similarity 0, relevancy 1/2), 16 or 32 text
    vectors, several canonical phrases."""
    import torch
    rng = np.random.default_rng(P + Q)
    D = 512
    dev = torch.device("cuda:0")
    F = torch.from_numpy(rng.normal(size=(P, D)).astype(np.float32)).to(dev).to(torch.bfloat16)
    F[::97] = 0.0
    T = torch.from_numpy(synth.unit_rows(rng, Q, D)).to(dev)
    sim = torch.empty((P, Q), dtype=torch.float32, device=dev)
    gb.scoup_similarity(F, T, sim)
    R = torch.empty((P, Q - n_canon), dtype=torch.float32, device=dev)
    gb.scoup_relevancy(sim, n_canon, R, alpha=10.0)
    Rf = torch.full((P, Q - n_canon), -7.0, dtype=torch.float32, device=dev)
    gb.scoup_similarity_relevancy(F, T, n_canon, Rf, alpha=10.0)
    torch.cuda.synchronize()
    assert torch.equal(Rf, R)
    assert torch.all(Rf[::97] == 0.5)


@pytest.mark.parametrize("n_canon,nq", [(1, 31), (2, 43), (4, 28)])
def test_relevancy_row_widths(gb, oracle_lib, n_canon, nq):
    """Rows of at most 32 columns (read by shuffles) and wider rows (the
    general loop), one or several canonical phrases, a ragged row count."""
    import torch
    rng = np.random.default_rng(100 + nq)
    P = 1237
    sim = rng.uniform(-1, 1, (P, n_canon + nq)).astype(np.float32)
    R = torch.empty((P, nq), dtype=torch.float32, device="cuda")
    gb.scoup_relevancy(torch.from_numpy(sim).cuda(), n_canon, R, alpha=10.0)
    torch.cuda.synchronize()
    s64 = sim.astype(np.float64)
    want = np.stack([oracle_lib.relevancy(s64[:, n_canon + q], s64[:, :n_canon], 10.0) for q in range(nq)], axis=1)
    assert np.abs(R.cpu().numpy() - want).max() <= 2e-6
