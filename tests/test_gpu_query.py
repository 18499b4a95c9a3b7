"""GPU parity of the decode with the text query in the same GEMM
(scoup_decode_query: Eq. 8 and App. B, with the relevancy of Eq. 9) against
the FP64 oracle.

The similarity's numerator is <What_p, G_q> with G = C T^T (associativity of
<What_p C, t_q>): What and G are rounded to bf16 (G after FP32 sums over D),
the products accumulate in FP32; the denominator is the norm of the stored
(bf16-rounded) feature row and |t_q| in FP32.  The bound below carries each of
those roundings; the features themselves are the decode's, bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from synth.scenes import unit_rows

pytestmark = pytest.mark.gpu

U = 2.0 ** -8    # unit roundoff of bf16
E32 = 2.0 ** -24  # unit roundoff of FP32


def _codes(rng, P, C, nnz=8):
    W = np.zeros((P, C), np.float32)
    for p in range(P):
        k = int(rng.integers(0, nnz + 1))
        idx = rng.choice(C, size=k, replace=False)
        W[p, idx] = rng.random(k).astype(np.float32) * float(rng.random())
    return W


def _sim_bound(W, B, T, F, S):
    """|sim_gpu - S| for S the exact cosine of F = W B against T (FP64)."""
    W64, B64, T64 = (np.abs(x.astype(np.float64)) for x in (W, B, T))
    C, D = B.shape
    G = np.abs(T.astype(np.float64) @ B.astype(np.float64).T)  # |G|, Q x C
    eG = U * G + D * E32 * (T64 @ B64.T)  # bf16 rounding of G after FP32 sums
    M1 = W64 @ G.T
    M2 = W64 @ eG.T
    err_num = U * M1 + (1 + U) * M2 + C * 2 * E32 * (1 + U) * (M1 + M2)
    mag = W64 @ B64
    dF = np.linalg.norm((2 * U + U * U) * mag + U * (np.abs(F) + 2 * U * mag), axis=1)
    fn = np.linalg.norm(F, axis=1)
    tn = np.linalg.norm(T.astype(np.float64), axis=1)
    den = np.maximum(fn - dF, 1e-150)[:, None] * np.maximum(tn, 1e-150)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):  # rows of zero norm are not `live`
        bound = err_num / den + np.abs(S) * (dF / np.maximum(fn - dF, 1e-150))[:, None]
    return bound * 1.01 + 1e-5 * np.abs(S) + 1e-6, fn > 2 * dF


def _run(W, B, T, n_canon=0, alpha=10.0, store=True, codes_bf16=False):
    from paper_2605_13600_gb300 import scoup
    dev = torch.device("cuda:0")
    P, D, Q = W.shape[0], B.shape[1], T.shape[0]
    codes = torch.from_numpy(W).to(dev)
    if codes_bf16:
        codes = codes.to(torch.bfloat16)
    feats = torch.full((P, D), float("nan"), dtype=torch.bfloat16, device=dev) if store else None
    n2 = torch.full((P,), -1.0, dtype=torch.float32, device=dev)
    out = torch.full((P, Q - n_canon), float("nan"), dtype=torch.float32, device=dev)
    ws = scoup.scoup_decode_query(codes, torch.from_numpy(B).to(dev), torch.from_numpy(T).to(dev), out,
                                  n_canon=n_canon, alpha=alpha, features=feats, feat_norm2=n2)
    assert scoup.scoup_read_stats(ws)["status"] == 0
    torch.cuda.synchronize()
    return out.cpu().numpy(), (feats.float().cpu().numpy() if store else None), n2.cpu().numpy()


@pytest.mark.parametrize("P,C,D,Q", [(1, 64, 32, 16), (300, 256, 512, 32), (1000, 72, 272, 16),
                                     (257, 256, 48, 32), (2049, 256, 512, 16)])
def test_query_similarity_matches_oracle(P, C, D, Q):
    """Ragged row blocks, one or two column tiles (and a ragged one), 16 or 32
    text vectors; a zero code row and a zero text row give similarity 0."""
    from paper_2605_13600_gb300 import scoup
    rng = np.random.default_rng(P + C + D + Q)
    W = _codes(rng, P, C)
    W[0] = 0.0
    B = unit_rows(rng, C, D)
    T = unit_rows(rng, Q, D)
    T[-1] = 0.0
    got, feats, n2 = _run(W, B, T)
    F = oracle.decode(W.astype(np.float64), B)
    S = oracle.similarity(F, T)
    S[:, -1] = 0.0
    bound, live = _sim_bound(W, B, T, F, S)
    err = np.abs(got - S)
    assert (err[live] <= bound[live]).all(), float(np.max(err[live] - bound[live]))
    assert (got[0] == 0).all() and (got[:, -1] == 0).all()
    # the features are the decode's, bit for bit; the norms are those of the stored rows
    dev = torch.device("cuda:0")
    ref = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    scoup.scoup_decode(torch.from_numpy(W).to(dev), torch.from_numpy(B).to(dev), ref)
    torch.cuda.synchronize()
    assert np.array_equal(feats, ref.float().cpu().numpy())
    want_n2 = (feats.astype(np.float64) ** 2).sum(1)
    assert np.allclose(n2, want_n2, rtol=D * E32 * 2, atol=1e-30)


@pytest.mark.parametrize("Q,n_canon", [(32, 4), (16, 4), (32, 8), (16, 12)])
def test_query_relevancy_is_relevancy_of_the_similarity(Q, n_canon):
    """The relevancy form (Eq. 9 in the query unit's epilogue) equals
    scoup_relevancy applied to the similarity form's output bit for bit, and
    the oracle's relevancy of the exact similarities within alpha / 4 times
    the similarity bound (dR/ds <= alpha / 4 for each of the two terms)."""
    from paper_2605_13600_gb300 import scoup
    rng = np.random.default_rng(Q * 100 + n_canon)
    P, C, D = 1500, 256, 512
    W = _codes(rng, P, C)
    B = unit_rows(rng, C, D)
    T = unit_rows(rng, Q, D)
    sim, _, _ = _run(W, B, T)
    rel, _, _ = _run(W, B, T, n_canon=n_canon, alpha=10.0, store=False)
    dev = torch.device("cuda:0")
    R = torch.empty((P, Q - n_canon), dtype=torch.float32, device=dev)
    scoup.scoup_relevancy(torch.from_numpy(sim).to(dev), n_canon, R, alpha=10.0)
    torch.cuda.synchronize()
    assert np.array_equal(rel, R.cpu().numpy())
    F = oracle.decode(W.astype(np.float64), B)
    S = oracle.similarity(F, T)
    bound, live = _sim_bound(W, B, T, F, S)
    want = np.stack([oracle.relevancy(S[:, n_canon + q], S[:, :n_canon], 10.0) for q in range(Q - n_canon)], 1)
    bmax = bound.max(axis=1, keepdims=True)
    err = np.abs(rel - want)
    assert (err[live] <= (10.0 / 4.0 * 2.0 * bmax + 2e-6)[live]).all()


def test_query_without_features_and_bf16_codes():
    """features=None writes no features but the same similarities and norms;
    bf16 codes give the same result as f32 codes holding the same values."""
    rng = np.random.default_rng(77)
    P, C, D, Q = 777, 256, 512, 32
    W = torch.from_numpy(_codes(rng, P, C)).to(torch.bfloat16).float().numpy()
    B = unit_rows(rng, C, D)
    T = unit_rows(rng, Q, D)
    a, _, n_a = _run(W, B, T, store=True)
    b, _, n_b = _run(W, B, T, store=False)
    c, _, n_c = _run(W, B, T, store=False, codes_bf16=True)
    assert np.array_equal(a, b) and np.array_equal(n_a, n_b)
    assert np.array_equal(a, c) and np.array_equal(n_a, n_c)


def test_query_chunked_f32_codes_sampled_rows():
    """More rows than one f32 conversion chunk (262,144): every chunk writes its
    own rows; sampled rows on both sides of the chunk boundary against FP64."""
    rng = np.random.default_rng(91)
    P, C, D, Q = 262144 + 3001, 256, 512, 32
    W = np.zeros((P, C), np.float32)
    idx = rng.integers(0, C, size=(P, 8))
    np.put_along_axis(W, idx, rng.random((P, 8)).astype(np.float32) * 0.2, axis=1)
    B = unit_rows(rng, C, D)
    T = unit_rows(rng, Q, D)
    got, _, _ = _run(W, B, T, store=False)
    rows = np.unique(np.concatenate([np.arange(262144 - 40, 262144 + 40), rng.integers(0, P, 300), [P - 1]]))
    Ws = W[rows]
    F = oracle.decode(Ws.astype(np.float64), B)
    S = oracle.similarity(F, T)
    bound, live = _sim_bound(Ws, B, T, F, S)
    err = np.abs(got[rows] - S)
    assert (err[live] <= bound[live]).all()


def test_query_invalid_arguments():
    from paper_2605_13600_gb300 import scoup
    dev = torch.device("cuda:0")
    W = torch.zeros((10, 64), device=dev)
    B = torch.zeros((64, 32), device=dev)
    for Q, n_canon in ((48, 0), (32, 3), (16, 16)):
        T = torch.zeros((Q, 32), device=dev)
        out = torch.empty((10, Q - min(n_canon, Q - 1)), device=dev)
        with pytest.raises((scoup.ScoupError, ValueError)):
            scoup.scoup_decode_query(W, B, T, out, n_canon=n_canon)
