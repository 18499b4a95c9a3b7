"""Comparison rules of the GPU-vs-oracle parity tests.

Tolerances (the target precision of the uplift):
  * raw accumulators: |gpu - oracle| <= RTOL * oracle + risk + ATOL_REL * max(row)
    (binary32 accumulation of positive terms; `risk` is the oracle's bound on
    contributions whose transmittance-stop decision lies within the margin of
    the 1e-4 threshold);
  * Top-K index sets: identical, except that an atom may be swapped with
    another whose oracle value lies within TIE_RTOL (relative) of the K-th
    value, or within the risk bound;
  * Top-K coefficients: within RTOL relative per kept atom.
"""
import numpy as np

RTOL = 1e-4
TIE_RTOL = 1e-5
ATOL_REL = 1e-6


def check_accum(gpu: np.ndarray, ora: np.ndarray, risk: np.ndarray, rtol=RTOL):
    gpu = gpu.astype(np.float64)
    rowmax = np.abs(ora).max(axis=1, keepdims=True)
    tol = rtol * np.abs(ora) + risk + ATOL_REL * rowmax + 1e-30
    err = np.abs(gpu - ora)
    bad = err > tol
    rel = err / np.maximum(np.abs(ora), 1e-30)
    nz = ora > 0
    info = {"max_rel_err": float(rel[nz & ~(risk > 0)].max()) if (nz & ~(risk > 0)).any() else 0.0,
            "mean_rel_err": float(rel[nz & ~(risk > 0)].mean()) if (nz & ~(risk > 0)).any() else 0.0,
            "n_bad": int(bad.sum())}
    if bad.any():
        i, j = np.argwhere(bad)[0]
        info["first_bad"] = (int(i), int(j), float(gpu[i, j]), float(ora[i, j]), float(risk[i, j]))
    return info


def check_topk(gidx: np.ndarray, gval: np.ndarray, ora_acc: np.ndarray, risk: np.ndarray,
               K: int, rtol=RTOL, tie_rtol=TIE_RTOL):
    """Validate GPU Top-K (idx, val) rows against the oracle accumulator."""
    import oracle
    oidx, oval = oracle.topk(ora_acc, K)
    n = ora_acc.shape[0]
    n_set_diff = n_tie_ok = 0
    worst_val = 0.0
    problems = []
    for i in range(n):
        gs = set(int(j) for j in gidx[i] if j >= 0)
        os_ = set(int(j) for j in oidx[i] if j >= 0)
        row = ora_acc[i]
        if gs != os_:
            n_set_diff += 1
            kept = oval[i] > 0
            kth = row[oidx[i][kept][-1]] if kept.any() else 0.0
            ok = True
            for j in gs ^ os_:
                slack = tie_rtol * kth + risk[i, j] + (risk[i, oidx[i][kept][-1]] if kept.any() else 0.0)
                if not (abs(row[j] - kth) <= slack):
                    ok = False
            if len(gs) != len(os_):
                ok = ok and abs(len(gs) - len(os_)) <= 1 and risk[i].max() > 0
            if ok:
                n_tie_ok += 1
            else:
                problems.append(("set", i, sorted(gs), sorted(os_)))
                continue
        # values of common atoms
        gmap = {int(j): float(v) for j, v in zip(gidx[i], gval[i]) if j >= 0}
        omap = {int(j): float(v) for j, v in zip(oidx[i], oval[i]) if j >= 0}
        if gs == os_:
            for j in gs:
                rel = abs(gmap[j] - omap[j]) / max(omap[j], 1e-30)
                worst_val = max(worst_val, rel if risk[i].max() == 0 else 0.0)
                slack = rtol * omap[j] + 2 * risk[i].sum() / max(row[list(os_)].sum(), 1e-30)
                if abs(gmap[j] - omap[j]) > slack:
                    problems.append(("val", i, j, gmap[j], omap[j]))
        # order: descending values, padding at the end
        g_valid = gidx[i] >= 0
        if g_valid.any():
            if not (np.diff(gval[i][g_valid]) <= 1e-7).all():
                problems.append(("order", i))
            if not (gidx[i][g_valid.sum():] == -1).all():
                problems.append(("pad", i))
    return {"n_set_diff": n_set_diff, "n_tie_ok": n_tie_ok, "max_val_rel_err": worst_val,
            "problems": problems[:10], "n_problems": len(problems)}
