"""Training and evaluation of the learned warm start / block-preconditioner
correction (the model of ba_mlp_*; see include/sqrtba.h).

    samples = solver_samples(scene)          # per LM iteration of a plain solve
    model, log = train(samples_list)          # GPU training with the library's kernels
    result = compare(scene, model)            # learned vs plain block-Jacobi PCG

The data are generated by the solver itself: at every LM iteration of a
plain solve, the reduced camera system at that state and damping is solved
tightly (Nash-Sofer forcing 1e-4) and the per-camera tuples (damped
block-Jacobi block M_i, right-hand side g_i, solution block x*_i,
observation count) are recorded.  Training runs entirely in the library's
CUDA kernels (tcgen05 forward, FP32 backward, Adam); PyTorch only holds the
device buffers and draws the minibatch indices.
"""
from __future__ import annotations

import time

import numpy as np

from . import Mlp, Problem, mlp_params_flat


def init_params(seed=0, sizes=(19, 256, 256, 256, 54)):
    """He-normal hidden layers, zero output layer (the untrained model is
    plain block Jacobi from the block-Jacobi solution M^-1 g)."""
    rng = np.random.default_rng(seed)
    params = []
    for li in range(len(sizes) - 1):
        fi, fo = sizes[li], sizes[li + 1]
        W = np.zeros((fo, fi)) if li == len(sizes) - 2 else rng.standard_normal((fo, fi)) * np.sqrt(2.0 / fi)
        params.append((W, np.zeros(fo)))
    return mlp_params_flat(params)


def solver_samples(scene, tight_eta=1e-4, max_lm_iters=50, stream=None):
    """Per-camera (M, g, x*, count) at every LM iteration of a plain solve."""
    Ms, gs, xs, cs = [], [], [], []
    with Problem.from_scene(scene, max_lm_iters=max_lm_iters, stream=stream) as plain, \
            Problem.from_scene(scene, cg_eta=tight_eta, max_cg_iters=500, stream=stream) as tight:
        _, _, cam_off, _ = plain.export_order()
        count = np.diff(cam_off).astype(np.int32)
        while not plain.get_state()["stopped"]:
            lam = plain.get_state()["lambda"]
            c, x = plain.get_params()
            tight.set_params(c, x)
            tight.linearize()
            tight.marginalize_qr(lam)
            tight.pcg_solve()
            M, g = tight.export_rcs_diag()
            dp, _ = tight.export_step()
            Ms.append(M.reshape(-1, 81))
            gs.append(g)
            xs.append(dp)
            cs.append(count)
            plain.lm_step()
    return dict(M=np.concatenate(Ms), g=np.concatenate(gs), xstar=np.concatenate(xs), count=np.concatenate(cs))


def _merge(samples):
    return {k: np.concatenate([s[k] for s in samples]) for k in samples[0]}


def clean_samples(data, max_ratio=1e6, chunk=1 << 20):
    """Drops the samples the normalised loss cannot use; returns (data, counts).

    The loss of one sample is divided by ||L^T x*||^2 (L the Cholesky factor
    of its block M), so a sample is kept only if its entries are finite, M is
    positive definite (in FP64), x* is non-zero in the M-norm, and the
    block-Jacobi term ||L^-1 g||^2 is at most `max_ratio` times that norm (a
    sample beyond it would dominate a minibatch's mean loss by itself)."""
    n = data["g"].shape[0]
    keep = np.zeros(n, bool)
    counts = dict(total=int(n), non_finite=0, not_pd=0, zero_target=0, ratio=0)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        M = data["M"][a:b].reshape(-1, 9, 9).astype(np.float64)
        g = data["g"][a:b].astype(np.float64)
        x = data["xstar"][a:b].astype(np.float64)
        fin = np.isfinite(M).all(axis=(1, 2)) & np.isfinite(g).all(axis=1) & np.isfinite(x).all(axis=1)
        M = np.where(fin[:, None, None], M, np.eye(9))
        g = np.where(fin[:, None], g, 0.0)
        x = np.where(fin[:, None], x, 0.0)
        L = np.zeros_like(M)
        pd = np.ones(b - a, bool)
        for j in range(9):  # column-by-column Cholesky over the whole chunk
            d = M[:, j, j] - np.einsum("nk,nk->n", L[:, j, :j], L[:, j, :j])
            pd &= d > 0
            L[:, j, j] = np.sqrt(np.where(d > 0, d, 1.0))
            for i in range(j + 1, 9):
                L[:, i, j] = (M[:, i, j] - np.einsum("nk,nk->n", L[:, i, :j], L[:, j, :j])) / L[:, j, j]
        w = np.zeros_like(g)
        for i in range(9):
            w[:, i] = (g[:, i] - np.einsum("nk,nk->n", L[:, i, :i], w[:, :i])) / L[:, i, i]
        z2 = np.einsum("nij,ni->nj", L, x)
        z2 = np.einsum("nj,nj->n", z2, z2)
        w2 = np.einsum("ni,ni->n", w, w)
        ok_fin, ok_pd = fin, fin & pd
        ok_z = ok_pd & (z2 > 0)
        ok = ok_z & (w2 <= max_ratio * z2)
        counts["non_finite"] += int((~ok_fin).sum())
        counts["not_pd"] += int((ok_fin & ~ok_pd).sum())
        counts["zero_target"] += int((ok_pd & ~ok_z).sum())
        counts["ratio"] += int((ok_z & ~ok).sum())
        keep[a:b] = ok
    counts["kept"] = int(keep.sum())
    return {k: v[keep] for k, v in data.items()}, counts


def train(samples, params=None, steps=1500, batch=2048, lr=1e-3, seed=0, stream=None, stats=None):
    """Trains a model on solver samples (a dict or a list of dicts) on the
    GPU; returns (Mlp, list of losses).  The samples pass through
    clean_samples first; its counts go into `stats` (a dict) if given.
    Raises FloatingPointError at the first non-finite minibatch loss."""
    import torch
    data = _merge(samples) if isinstance(samples, (list, tuple)) else samples
    data, counts = clean_samples(data)
    if stats is not None:
        stats.update(counts)
    if counts["kept"] == 0:
        raise ValueError(f"no usable training sample: {counts}")
    dev = torch.device("cuda")
    n = data["g"].shape[0]
    model = Mlp(params if params is not None else init_params(seed), stream=stream)
    t = {k: torch.as_tensor(np.ascontiguousarray(v), device=dev,
                            dtype=torch.int32 if k == "count" else torch.float32) for k, v in data.items()}
    feats = torch.zeros((n, 19), dtype=torch.float32, device=dev)
    aux = torch.zeros((n, 72), dtype=torch.float32, device=dev)
    model.prepare(t["M"], t["g"], t["xstar"], t["count"], feats, aux)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    losses = []
    for _ in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device=dev, generator=gen)
        losses.append(model.train_step(feats[idx].contiguous(), aux[idx].contiguous(), lr))
        if not np.isfinite(losses[-1]):
            model.close()
            raise FloatingPointError(f"non-finite minibatch loss at step {len(losses) - 1}")
    return model, losses


def solve_to_tol(p, f_tau, max_iters=50):
    """LM iterations until an accepted cost <= f_tau; (iters, pcg iters, reached, final cost)."""
    iters = cg = 0
    cost = None
    while iters < max_iters:
        r = p.lm_step()
        iters += 1
        cg += r["cg_iters"]
        if r["accepted"]:
            cost = r["new_cost"]
            if cost <= f_tau:
                return iters, cg, True, cost
        if r["stop"]:
            break
    return iters, cg, False, cost


def compare(scene, model, tau=0.01, repeats=3, stream=None):
    """Plain block-Jacobi PCG from zero vs the learned warm start and
    corrected preconditioner on one scene: LM iterations, PCG iterations and
    device time to the 1% cost tolerance f_tau = f* + tau (f0 - f*), with f*
    the plain solver's converged cost, and the converged costs of both."""
    import torch
    out = {}
    with Problem.from_scene(scene, stream=stream) as p:
        reps = p.solve()
    f0 = reps[0]["cost"]
    f_star = min([r["new_cost"] for r in reps if r["accepted"]] + [f0])
    f_tau = f_star + tau * (f0 - f_star)
    for name, learned in (("plain", 0), ("learned", 1)):
        with Problem.from_scene(scene, use_learned=learned, stream=stream) as p:
            if learned:
                p.set_learned(model)
            times = []
            for _ in range(repeats):
                p.set_params(scene.cams, scene.pts)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                it, cg, ok, cost = solve_to_tol(p, f_tau)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            p.set_params(scene.cams, scene.pts)
            full = p.solve()
            final = [r["new_cost"] for r in full if r["accepted"]]
            out[name] = dict(lm_iters=it, pcg_iters=cg, reached=ok, seconds=float(np.median(times)),
                             final_cost=final[-1] if final else f0,
                             fallbacks=p.learned_fallbacks() if learned else 0)
    out["f_tau"] = f_tau
    out["f_star"] = f_star
    return out
