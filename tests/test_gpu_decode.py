"""GPU parity of the codebook decode (Sec. 4.3, Eq. 8) and the cosine
similarity to text vectors (App. B) against the FP64 oracle.

Two comparisons per case:
  * against the oracle on the bf16-rounded operands the kernel is specified to
    consume: only the FP32 accumulation order (and, for bf16 output, one final
    rounding) separates the two;
  * against the oracle on the unrounded FP32 inputs, with the bound the BF16
    operand rounding implies: each operand carries a relative error of at most
    u = 2^-8, so |F_gpu - F| <= (2u + u^2) sum_c |w_c||b_cd| (+ u |F| for bf16
    output) plus the accumulation term.
"""
import numpy as np
import pytest
import torch

import oracle
from synth.scenes import unit_rows

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8  # unit roundoff of bf16 (8 significant bits, round to nearest)


def _cos_shift(delta_norm, norm):
    """Bound on |cos(a + d, b) - cos(a, b)| for |d| <= delta_norm, |a| = norm
    (first order: the direction of a turns by at most |d| / |a|, twice that
    bounds the cosine change)."""
    return 2.0 * delta_norm / np.maximum(norm, 1e-30)


def _sparse_codes(rng, P, C, nnz=8):
    """Non-negative rows with a few non-zeros summing to at most 1 (what the
    sparse-code rendering produces)."""
    W = np.zeros((P, C), np.float32)
    for p in range(P):
        k = int(rng.integers(0, nnz + 1))
        idx = rng.choice(C, size=k, replace=False)
        v = rng.random(k).astype(np.float32)
        W[p, idx] = v / max(1.0, float(v.sum())) * float(rng.random())
    return W


def _bf16(x: np.ndarray) -> np.ndarray:
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def _run_decode(W, B, out_dtype, codes_bf16=False):
    from paper_2605_13600_gb300 import scoup
    dev = torch.device("cuda:0")
    codes = torch.from_numpy(W).to(dev)
    if codes_bf16:
        codes = codes.to(torch.bfloat16)
    cb = torch.from_numpy(B).to(dev)
    P, D = W.shape[0], B.shape[1]
    feats = torch.full((P, D), float("nan"), dtype=out_dtype, device=dev)
    n2 = torch.full((P,), -1.0, dtype=torch.float32, device=dev) if out_dtype == torch.bfloat16 else None
    ws = scoup.scoup_decode(codes, cb, feats, n2)
    st = scoup.scoup_read_stats(ws)
    assert st["status"] == 0, st
    torch.cuda.synchronize()
    return feats.float().cpu().numpy(), (n2.cpu().numpy() if n2 is not None else None)


SHAPES = [
    (1, 64, 32), (127, 64, 64), (300, 256, 48), (1000, 256, 512), (129, 72, 256), (513, 256, 272),
]


@pytest.mark.parametrize("P,C,D", SHAPES)
@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16])
def test_decode_matches_oracle(P, C, D, out_dtype):
    rng = np.random.default_rng(P * 7 + C * 3 + D)
    W = _sparse_codes(rng, P, C)
    B = unit_rows(rng, C, D)
    got, n2 = _run_decode(W, B, out_dtype)
    assert np.isfinite(got).all()
    # (1) oracle on the rounded operands
    ref_r = oracle.decode(_bf16(W).astype(np.float64), _bf16(B))
    mag = np.abs(_bf16(W)).astype(np.float64) @ np.abs(_bf16(B)).astype(np.float64)
    tol_acc = 2.0 ** -22 * C * mag + 1e-30
    if out_dtype == torch.bfloat16:
        tol_acc = tol_acc + U_BF16 * np.abs(ref_r)
    assert (np.abs(got - ref_r) <= tol_acc * 1.0001 + 1e-12).all(), np.max(np.abs(got - ref_r) - tol_acc)
    # (2) oracle on the unrounded inputs, bound from the operand rounding
    ref = oracle.decode(W.astype(np.float64), B)
    mag_u = np.abs(W).astype(np.float64) @ np.abs(B).astype(np.float64)
    bound = (2 * U_BF16 + U_BF16 ** 2) * mag_u + tol_acc
    assert (np.abs(got - ref) <= bound + 1e-12).all()
    if n2 is not None:
        np.testing.assert_allclose(n2, (got.astype(np.float64) ** 2).sum(1), rtol=1e-5, atol=1e-12)


def test_decode_bf16_codes_and_chunks():
    """bf16 codes are consumed as they are; P above one conversion chunk."""
    rng = np.random.default_rng(11)
    P, C, D = 262144 + 300, 64, 32
    W = _bf16(rng.random((P, C), dtype=np.float32) / C)
    B = unit_rows(rng, C, D)
    for codes_bf16 in (False, True):
        got, _ = _run_decode(W, B, torch.float32, codes_bf16=codes_bf16)
        rows = np.concatenate([np.arange(0, 200), np.arange(262000, P)])
        ref_r = oracle.decode(W[rows].astype(np.float64), _bf16(B))
        mag = np.abs(W[rows]).astype(np.float64) @ np.abs(_bf16(B)).astype(np.float64)
        assert (np.abs(got[rows] - ref_r) <= 2.0 ** -22 * C * mag + 1e-12).all()


def test_decode_empty_and_invalid():
    from paper_2605_13600_gb300 import scoup
    from paper_2605_13600_gb300._lib import ScoupError
    dev = torch.device("cuda:0")
    cb = torch.zeros((64, 32), dtype=torch.float32, device=dev)
    scoup.scoup_decode(torch.zeros((0, 64), device=dev), cb, torch.zeros((0, 32), device=dev))
    with pytest.raises(ScoupError):  # C not a multiple of 8
        scoup.scoup_decode(torch.zeros((4, 60), device=dev), torch.zeros((60, 32), device=dev),
                           torch.zeros((4, 32), device=dev))
    with pytest.raises(ScoupError):  # D not a multiple of 16
        scoup.scoup_decode(torch.zeros((4, 64), device=dev), torch.zeros((64, 40), device=dev),
                           torch.zeros((4, 40), device=dev))


@pytest.mark.parametrize("P,D,Q", [(1, 64, 16), (200, 512, 32), (1000, 256, 256), (131, 40, 48)])
def test_similarity_matches_oracle(P, D, Q):
    from paper_2605_13600_gb300 import scoup
    rng = np.random.default_rng(P + D + Q)
    dev = torch.device("cuda:0")
    F = rng.standard_normal((P, D)).astype(np.float32)
    F[0] = 0.0  # a zero feature row gives similarity 0
    T = unit_rows(rng, Q, D)
    T[-1] = 0.0  # a zero (padding) text row gives 0
    Fb = torch.from_numpy(F).to(torch.bfloat16)
    out = torch.full((P, Q), float("nan"), dtype=torch.float32, device=dev)
    for with_norms in (False, True):
        n2 = None
        if with_norms:
            n2 = (Fb.double() ** 2).sum(1).float().to(dev)
        scoup.scoup_similarity(Fb.to(dev), torch.from_numpy(T).to(dev), out, feat_norm2=n2)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # oracle on the rounded operands: accumulation order only
        ref_r = oracle.similarity(Fb.double().numpy(), _bf16(T))
        ref_r[:, -1] = 0.0
        assert np.abs(got - ref_r).max() <= 2e-5 * np.sqrt(D / 64.0) + 1e-6
        assert (got[0] == 0).all() and (got[:, -1] == 0).all()
        # unrounded text: each text vector moves by at most u |t| when rounded
        ref = oracle.similarity(Fb.double().numpy(), T)
        assert np.abs(got - ref).max() <= _cos_shift(U_BF16, 1.0) * 1.01 + 1e-4


def test_decode_then_similarity_pipeline():
    """Rendered codes -> bf16 features (+ norms) -> cosine, vs the oracle on FP32 inputs."""
    from paper_2605_13600_gb300 import scoup
    rng = np.random.default_rng(5)
    dev = torch.device("cuda:0")
    P, C, D, Q = 2000, 256, 512, 32
    W = _sparse_codes(rng, P, C)
    B = unit_rows(rng, C, D)
    T = unit_rows(rng, Q, D)
    feats = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    n2 = torch.empty((P,), dtype=torch.float32, device=dev)
    scoup.scoup_decode(torch.from_numpy(W).to(dev), torch.from_numpy(B).to(dev), feats, n2)
    out = torch.empty((P, Q), dtype=torch.float32, device=dev)
    scoup.scoup_similarity(feats, torch.from_numpy(T).to(dev), out, feat_norm2=n2)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    F = oracle.decode(W.astype(np.float64), B)
    ref = oracle.similarity(F, T)
    live = np.abs(W).sum(1) > 0
    # per row: codes and codebook rounded (2u + u^2 of sum |w||b|), features
    # rounded on output (u |F|), text rounded (u |t|)
    mag = np.abs(W).astype(np.float64) @ np.abs(B).astype(np.float64)
    fnorm = np.linalg.norm(F, axis=1)
    dF = np.linalg.norm((2 * U_BF16 + U_BF16 ** 2) * mag + U_BF16 * (np.abs(F) + 2 * U_BF16 * mag), axis=1)
    bound = (_cos_shift(dF, fnorm)[:, None] + _cos_shift(U_BF16, 1.0)) * 1.01 + 1e-4
    err = np.abs(got - ref)
    assert (err[live] <= bound[live]).all()
    assert err[live].mean() <= 2e-3
    assert (got[~live] == 0).all()


def test_decode_full_size_sampled_rows():
    """The decode at the benchmark's size (2,073,600 rows = one 1920 x 1080
    view, C = 256, D = 512, bf16 codes in, bf16 features out, one launch)
    on seeded 8-sparse code rows: 256 sampled rows against the oracle on the
    unrounded inputs with the operand-rounding bound of the module header."""
    import paper_2605_13600_gb300 as gb
    from paper_2605_13600_gb300 import build
    build.build()
    P, C, D, nnz = 1920 * 1080, 256, 512, 8
    rng = np.random.default_rng(402)
    idx = rng.integers(0, C, size=(P, nnz)).astype(np.int64)
    val = (rng.random((P, nnz), dtype=np.float32) / nnz).astype(np.float32)
    B = unit_rows(rng, C, D)
    dev = torch.device("cuda:0")
    W = torch.zeros((P, C), dtype=torch.float32, device=dev)
    W.scatter_add_(1, torch.from_numpy(idx).to(dev), torch.from_numpy(val).to(dev))  # repeated atoms add up
    Wb = W.to(torch.bfloat16)
    F = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    n2 = torch.zeros((P,), dtype=torch.float32, device=dev)
    gb.scoup_decode(Wb, torch.from_numpy(B).to(dev), F, n2)
    torch.cuda.synchronize()
    rows = np.concatenate([[0, 1, P - 2, P - 1], rng.integers(0, P, 252)])
    Wr = np.zeros((rows.size, C))
    for q, p in enumerate(rows):
        np.add.at(Wr[q], idx[p], val[p].astype(np.float64))
    ref = oracle.decode(Wr, B)
    got = F[torch.from_numpy(rows).to(dev)].float().cpu().numpy().astype(np.float64)
    mag = np.abs(Wr) @ np.abs(B.astype(np.float64))
    bound = (2 * U_BF16 + U_BF16 ** 2) * mag + 2.0 ** -22 * C * mag + U_BF16 * np.abs(ref) + 1e-12
    assert (np.abs(got - ref) <= bound).all(), float(np.max(np.abs(got - ref) - bound))
    np.testing.assert_allclose(n2[torch.from_numpy(rows).to(dev)].cpu().numpy(),
                               (got ** 2).sum(1), rtol=1e-5, atol=1e-12)
