"""The mapping stream (Section 3.2 "Mapping") over a sequence of keyframes.

Per keyframe j: the first keyframe initialises the map from its points (Eq. 6);
every later one inserts its points through the opacity gate (Eq. 7 reading);
then `iters` mapping iterations (render, L1 + planar loss, adjoint, Adam) run
over the window of the last `window` keyframes, and the map is densified by
splitting (densification reading). Every step runs in the library's kernels;
this module only sequences the calls and keeps statistics.

Also: collection of (features, converged parameters) pairs of inserted
Gaussians, training of the learned initialiser on them, and the
time-to-PSNR comparison of learned against plain initialisation.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import torch

from .api import MLP, GaussianMap

PATCH_CENTRE = slice(36, 39)   # RGB of the centre pixel of the 5x5 patch in the MLP features


def run_stream(gm: GaussianMap, cams: Sequence, targets: torch.Tensor, points: Sequence[torch.Tensor],
               window: int = 8, iters: int = 100, insert: bool = True, densify: bool = True,
               collect: bool = False, track_psnr: str = "", mlp: Optional[MLP] = None,
               flush: Optional[torch.Tensor] = None, clarity: bool = False) -> dict:
    """Run the mapping stream. ``targets`` [F, 3, H, W] and each ``points[j]`` [k, 3] live on the
    device. With ``mlp`` the learned initialiser initialises inserted Gaussians.

    ``track_psnr``: "" (none), "final" (the newest keyframe's PSNR after its last iteration,
    computed outside the timed region) or "curve" (after every iteration). Mapping time is
    taken with CUDA events around every iteration (PSNR kernels and the optional L2 ``flush``
    write run between the brackets); insertion and densification are timed apart. With
    ``clarity`` the newest keyframe's dominated pixels are counted before each densification
    (the Eq. 9 split mask, active when the map's clarity_sigma > 0).

    Returns statistics: Gaussians after each keyframe, inserted per keyframe, per-keyframe
    mapping ms, insertion and densification ms, PSNR ("psnr": [F] or [F, iters]), and (with
    ``collect``) the features of the inserted Gaussians with their parameters after the
    keyframe's iterations (canonical form) as training pairs for the initialiser."""
    F = len(cams)
    H, W = targets.shape[2], targets.shape[3]
    dev = targets.device
    stream = torch.cuda.current_stream(dev)
    gm.set_initializer(mlp)
    loss = torch.empty(3, device=dev)
    n_gauss, n_inserted, xs, ys = [], [], [], []
    ev_map, ev_ins, ev_den, curves, finals = [], [], [], [], []
    launches0 = gm.launches

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e
    try:
        for j in range(F):
            feats = MLP.features(cams[j], targets[j], points[j]) if (collect or j == 0) else None
            n0 = gm.n
            e0 = ev()
            if j == 0:
                gm.init_map(points[j], feats[:, PATCH_CENTRE].contiguous())
                mask = torch.ones(points[j].shape[0], dtype=torch.bool, device=dev)
                k = gm.n - n0
            elif insert:
                k, mask = gm.insert(cams[j], targets[j], points[j], return_mask=True)
            else:
                k, mask = 0, None
            e1 = ev()
            ev_ins.append((e0, e1))
            n_inserted.append(int(k))
            views = list(range(max(0, j - window + 1), j + 1))
            wc = [cams[v] for v in views]
            wt = targets[views[0]:j + 1]
            rgb = torch.empty(len(views), 3, H, W, device=dev)
            curve = torch.empty(iters, device=dev) if track_psnr == "curve" else None
            its = []
            for it in range(iters):
                if flush is not None:
                    flush.zero_()
                a = ev()
                gm.iterate(wc, wt, loss, rgb)
                its.append((a, ev()))
                if curve is not None:
                    gm.psnr(rgb[-1], targets[j], curve[it])
            ev_map.append(its)
            if curve is not None:
                curves.append(curve)
            elif track_psnr == "final":
                finals.append(gm.psnr(rgb[-1], targets[j]))
            if collect and k > 0:
                xs.append(feats[mask])
                ys.append(gm.mlp_targets(n0, k))
            d0 = ev()
            if densify:
                if clarity:
                    gm.count_dominant([cams[j]])
                gm.densify()
            ev_den.append((d0, ev()))
            n_gauss.append(gm.n)
    finally:
        gm.set_initializer(None)
    torch.cuda.synchronize(dev)
    it_ms = [[x.elapsed_time(y) for x, y in its] for its in ev_map]
    kf_ms = [sum(m) for m in it_ms]
    t_map = sum(kf_ms) / 1000.0
    out = {"n_gauss": n_gauss, "n_inserted": n_inserted, "keyframe_ms": kf_ms, "iteration_ms": it_ms,
           "map_seconds": t_map,
           "insert_ms": sum(x.elapsed_time(y) for x, y in ev_ins),
           "densify_ms": sum(x.elapsed_time(y) for x, y in ev_den),
           "iterations": F * iters, "iters_per_s": F * iters / max(t_map, 1e-9),
           "launches": gm.launches - launches0}
    if track_psnr == "curve":
        out["psnr"] = torch.stack(curves).cpu()
    elif track_psnr == "final":
        out["psnr"] = torch.stack(finals).cpu()
    if collect:
        out["features"] = torch.cat(xs) if xs else torch.empty(0, 80, device=dev)
        out["targets"] = torch.cat(ys) if ys else torch.empty(0, 16, device=dev)
    return out


def train_mlp(mlp: MLP, X: torch.Tensor, Y: torch.Tensor, epochs: int = 200, batch: int = 4096, lr: float = 1e-3,
              seed: int = 0) -> List[float]:
    """Minibatch Adam on the MSE between predictions and converged parameters (all on the GPU
    in the library's kernels). Returns the loss of each epoch's last batch."""
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    n = X.shape[0]
    losses = []
    for _ in range(epochs):
        perm = torch.randperm(n, device=X.device, generator=g)
        last = None
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            if idx.numel() < 16:
                continue
            last = mlp.backward(X[idx].contiguous(), Y[idx].contiguous())
            mlp.step(lr)
        if last is not None:
            losses.append(float(last))
    return losses


def iterations_to_reach(curves: torch.Tensor, goals: torch.Tensor) -> torch.Tensor:
    """Per keyframe, the first iteration (1-based) whose PSNR reaches the goal (len + 1 if never)."""
    reached = curves >= goals[:, None]
    first = torch.where(reached.any(1), reached.float().argmax(1) + 1,
                        torch.full((curves.shape[0],), curves.shape[1] + 1))
    return first
