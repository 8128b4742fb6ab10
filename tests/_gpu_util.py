"""Helpers shared by the GPU tests: run a workload through the C ABI and
compare with the oracle."""

import numpy as np
import torch

from paper_1511_05174_gb300.context import Context


def budgets(w, mode):
    levels = w.K_levels if mode == "cross_scale" else w.K_levels[:1]
    uniform = all(np.all(k == k[0]) for k in levels if len(k))
    if uniform:
        K = [int(k[0]) if len(k) else 1 for k in levels]
        return K, None, K[0]
    Kmax = int(max(int(k.max()) for k in levels))
    K_patch = [torch.from_numpy(k.astype(np.int8)).cuda() for k in levels]
    return [Kmax] * len(levels), K_patch, Kmax


def run_gpu(w, mode="cross_scale", precision="fp32", ctx=None):
    ctx = ctx or Context(0)
    ctx.load_workload(w)
    meas = torch.from_numpy(np.ascontiguousarray(w.meas)).cuda()
    # dense Phi: the measurements are per patch already ([B, M])
    Y = meas.contiguous() if w.sensing.kind == "dense" else ctx.extract(meas)
    K, K_patch, Kmax = budgets(w, mode)
    sup, coef, keff = ctx.solve(Y, mode, precision, K=K, K_patch=K_patch, Kmax=Kmax)
    img = ctx.aggregate(sup, coef, keff)
    torch.cuda.synchronize()
    return {"Y": Y.cpu().numpy(), "sup": sup.cpu().numpy(), "coef": coef.cpu().numpy(),
            "keff": keff.cpu().numpy().astype(np.int64), "img": img.cpu().numpy().astype(np.float64),
            "stats": ctx.stats(), "ctx": ctx}


def compare(D0, sup_g, coef_g, keff_g, om_o, al_o, k_o):
    """(support-set match rate, worst relative L2 of x_hat = D_|Omega alpha over
    matching patches, indices of mismatching patches)."""
    D = D0.astype(np.float64)
    B = len(k_o)
    match = np.zeros(B, bool)
    worst = 0.0
    for b in range(B):
        sg = sup_g[b, :keff_g[b]]
        so = om_o[b, :k_o[b]]
        if keff_g[b] != k_o[b] or set(sg.tolist()) != set(so.tolist()):
            continue
        match[b] = True
        xg = D[sg].T @ coef_g[b, :keff_g[b]].astype(np.float64) if keff_g[b] else np.zeros(D.shape[1])
        xo = D[so].T @ al_o[b, :k_o[b]] if k_o[b] else np.zeros(D.shape[1])
        den = max(np.linalg.norm(xo), 1e-30)
        worst = max(worst, float(np.linalg.norm(xg - xo) / den) if np.linalg.norm(xo) > 0 else float(np.linalg.norm(xg)))
    return float(match.mean()) if B else 1.0, worst, np.flatnonzero(~match)
