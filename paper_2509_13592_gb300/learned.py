"""Unrolled FISTA network: K layers of eq:fista with learned per-layer multipliers.

Layer k (k = 0..K-1), on every snapshot of a batch that shares one element mask:

    u_k = z_k - a_k mu (G z_k - b),   c_k = S_{t_k mu lam}(u_k),   z_{k+1} = c_k + beta_k (c_k - c_{k-1})

with z_0 = c_{-1} = 0, FISTA's momentum beta_k, mu = 1/max Lambda and lam the snapshot's LASSO weight.
a = t = 1 is plain FISTA with K iterations; training learns the 2K multipliers.  Forward and backward are
the library's kernels (bccb_unrolled_fwd / bccb_unrolled_bwd, through the binding); PyTorch only holds the
tensors, computes the loss and runs the optimizer on the 2K scalars.

The network's output is accepted when its FP64 relative KKT residual (bccb_batch_results) is at most
`kkt_tol`; otherwise plain FISTA, warm-started from the network's output with the momentum restarted, runs
on the failing snapshots (infer_with_fallback).
"""
from __future__ import annotations

import dataclasses
import os
from typing import Optional

import numpy as np
import torch

from . import binding as B


class UnrolledNet:
    """Device state for a batch of `batch` snapshots that share `mask` (M1 x M2) on an L1 x L2 grid."""

    def __init__(self, M1, M2, mask, L1, L2, batch, lam_frac, stream=None):
        self.M1, self.M2, self.L1, self.L2 = M1, M2, L1, L2
        self.mask = np.ascontiguousarray(mask, np.uint8).reshape(-1)
        self.N = int(self.mask.sum())
        self.L = L1 * L2
        self.batch = batch
        self.lam_frac = lam_frac
        inst = dict(M1=M1, M2=M2, L1=L1, L2=L2, mask=self.mask, y=np.zeros(self.N, np.complex64), lam=lam_frac,
                    lam_is_frac=True)
        self.solver = B.BatchSolver([inst] * batch, "fista", stream=stream)

    @property
    def handle(self):
        return self.solver.handle

    def close(self):
        self.solver.close()


class UnrolledFISTA(torch.autograd.Function):
    """c_{K-1} = Net(y; a, t).  y: packed complex64 (batch * N) on the GPU; scale = a, thresh = t:
    float32 (K,) on the GPU.  Returns the packed complex64 (batch * L1 * L2) output.  The backward
    gives dLoss/da, dLoss/dt and, when y requires a gradient, dLoss/dy (PyTorch's convention for
    complex tensors, dLoss/dRe + j dLoss/dIm, is the library's)."""

    @staticmethod
    def forward(ctx, y, scale, thresh, net):
        K = scale.numel()
        c = torch.empty(net.batch * net.L, dtype=torch.complex64, device=y.device)
        need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        saved = torch.empty(K * 2 * net.batch * net.L, dtype=torch.complex64, device=y.device) if need else None
        B.bccb_unrolled_fwd(net.handle, y, net.batch, K, scale.detach().contiguous(), thresh.detach().contiguous(),
                            c, saved)
        ctx.net = net
        ctx.saved = saved
        ctx.save_for_backward(scale.detach(), thresh.detach())
        return c

    @staticmethod
    def backward(ctx, grad_c):
        scale, thresh = ctx.saved_tensors
        K = scale.numel()
        g_s = torch.zeros(K, dtype=torch.float64, device=scale.device)
        g_t = torch.zeros(K, dtype=torch.float64, device=scale.device)
        g_y = torch.empty(ctx.net.batch * ctx.net.N, dtype=torch.complex64, device=scale.device) \
            if ctx.needs_input_grad[0] else None
        B.bccb_unrolled_bwd(ctx.net.handle, ctx.net.batch, K, scale.contiguous(), thresh.contiguous(), ctx.saved,
                            grad_c.contiguous().to(torch.complex64), g_s, g_t, g_y)
        return g_y, g_s.to(scale.dtype), g_t.to(thresh.dtype), None


def net_forward(net: UnrolledNet, y, scale, thresh):
    return UnrolledFISTA.apply(y, scale, thresh, net)


def relative_errors(c, ref, batch, L):
    """Per-snapshot ||c - ref|| / ||ref|| for packed outputs."""
    d = (c - ref).reshape(batch, L)
    r = ref.reshape(batch, L)
    return torch.linalg.vector_norm(d, dim=1) / torch.linalg.vector_norm(r, dim=1).clamp_min(1e-30)


def infer_with_fallback(net: UnrolledNet, y, scale, thresh, kkt_tol=1e-2, fallback_iters=1000):
    """Run the network with the FP64 KKT check; snapshots whose relative KKT residual exceeds kkt_tol
    get `fallback_iters` iterations of plain FISTA warm-started from the network's output.
    Returns (c, kkt_after_net, fallback_mask)."""
    c = torch.empty(net.batch * net.L, dtype=torch.complex64, device=y.device)
    B.bccb_unrolled_fwd(net.handle, y, net.batch, scale.numel(), scale, thresh, c, None, True)
    kkt = net.solver.results()["kkt"]
    B.bccb_set_kkt_tol(net.handle, kkt_tol)
    bad = np.flatnonzero(B.bccb_batch_status(net.handle, net.batch) == B.ERR_KKT)
    if bad.size:
        ys = y.reshape(net.batch, net.N)[torch.as_tensor(bad, device=y.device)].reshape(-1).contiguous()
        c0 = c.reshape(net.batch, net.L)[torch.as_tensor(bad, device=y.device)].reshape(-1).contiguous()
        inst = dict(M1=net.M1, M2=net.M2, L1=net.L1, L2=net.L2, mask=net.mask,
                    y=np.zeros(net.N, np.complex64), lam=net.lam_frac, lam_is_frac=True)
        fb = B.BatchSolver([inst] * bad.size, "fista")
        out = torch.empty_like(c0)
        torch.cuda.synchronize()
        fb.solve(ys, fallback_iters, out, c0=c0, check=False)
        torch.cuda.synchronize()
        c.reshape(net.batch, net.L)[torch.as_tensor(bad, device=y.device)] = out.reshape(bad.size, net.L)
        fb.close()
    mask = np.zeros(net.batch, bool)
    mask[bad] = True
    return c, kkt, mask


@dataclasses.dataclass
class TrainConfig:
    M1: int = 32
    M2: int = 32
    N: int = 256
    L1: int = 256
    L2: int = 256
    layers: int = 16
    batch: int = 64
    steps: int = 100
    target_iters: int = 1000
    lam_frac: float = 0.05
    lr: float = 0.05
    mask_seed: int = 5000
    first_snapshot: int = 0
    checkpoint: Optional[str] = None
    checkpoint_every: int = 20


def fixed_mask(cfg: TrainConfig):
    import synth

    return synth.make_mask(np.random.Generator(np.random.PCG64(cfg.mask_seed)), cfg.M1, cfg.M2, cfg.N)


def snapshot_batch(cfg: TrainConfig, mask, first, count):
    """Training / evaluation snapshots: the fixed mask, K ~ U{1..8} off-grid sources with CN(0,1)
    amplitudes, SNR ~ U[0, 30] dB (seeded by snapshot index)."""
    import synth

    ys = []
    for i in range(first, first + count):
        rng = np.random.Generator(np.random.PCG64(5001 + i))
        K = int(rng.integers(1, 9))
        snr = float(rng.uniform(0.0, 30.0))
        sub = int(rng.integers(0, 2**62))
        s = synth.make_snapshot(sub, cfg.M1, cfg.M2, cfg.N, cfg.L1, cfg.L2, K, snr, mask=mask)
        ys.append(s.y.astype(np.complex64))
    return torch.from_numpy(np.concatenate(ys)).cuda()


def plain_fista(cfg: TrainConfig, mask, y, iters, batch, solver=None):
    """Plain batched FISTA on `batch` snapshots of the fixed array (a solver of that batch may be
    passed in and is then reused)."""
    s = solver
    if s is None:
        inst = dict(M1=cfg.M1, M2=cfg.M2, L1=cfg.L1, L2=cfg.L2, mask=mask, y=np.zeros(cfg.N, np.complex64),
                    lam=cfg.lam_frac, lam_is_frac=True)
        s = B.BatchSolver([inst] * batch, "fista")
    out = torch.empty(batch * cfg.L1 * cfg.L2, dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    s.solve(y, iters, out, check=False)
    torch.cuda.synchronize()
    if solver is None:
        s.close()
    return out


def train(cfg: TrainConfig, resume: bool = False, log=print):
    """Trains the 2K multipliers (log-parametrised, Adam) on snapshot batches against the
    target_iters-iteration plain FISTA result.  Checkpoints {log_a, log_t, optimizer, step} to
    cfg.checkpoint every checkpoint_every steps and at the end; resume=True continues from it."""
    mask = fixed_mask(cfg)
    net = UnrolledNet(cfg.M1, cfg.M2, mask, cfg.L1, cfg.L2, cfg.batch, cfg.lam_frac)
    log_a = torch.zeros(cfg.layers, device="cuda", requires_grad=True)
    log_t = torch.zeros(cfg.layers, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([log_a, log_t], lr=cfg.lr)
    step0 = 0
    if resume and cfg.checkpoint and os.path.exists(cfg.checkpoint):
        ck = torch.load(cfg.checkpoint, map_location="cuda")
        with torch.no_grad():
            log_a.copy_(ck["log_a"])
            log_t.copy_(ck["log_t"])
        opt.load_state_dict(ck["opt"])
        step0 = int(ck["step"])
    history = []
    inst = dict(M1=cfg.M1, M2=cfg.M2, L1=cfg.L1, L2=cfg.L2, mask=mask, y=np.zeros(cfg.N, np.complex64),
                lam=cfg.lam_frac, lam_is_frac=True)
    target_solver = B.BatchSolver([inst] * cfg.batch, "fista")
    for step in range(step0, cfg.steps):
        first = cfg.first_snapshot + step * cfg.batch
        y = snapshot_batch(cfg, mask, first, cfg.batch)
        with torch.no_grad():
            target = plain_fista(cfg, mask, y, cfg.target_iters, cfg.batch, target_solver)
        c = net_forward(net, y, log_a.exp(), log_t.exp())
        loss = (relative_errors(c, target, cfg.batch, net.L) ** 2).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        history.append(float(loss.detach()))
        if log and (step % 10 == 0 or step == cfg.steps - 1):
            log(f"step {step} loss {history[-1]:.4e}")
        if cfg.checkpoint and ((step + 1) % cfg.checkpoint_every == 0 or step == cfg.steps - 1):
            torch.save({"log_a": log_a.detach(), "log_t": log_t.detach(), "opt": opt.state_dict(), "step": step + 1},
                       cfg.checkpoint)
    net.close()
    target_solver.close()
    return log_a.detach().exp(), log_t.detach().exp(), history


def evaluate(cfg: TrainConfig, scale, thresh, n_eval=8192, first=10**7, sweep=(16, 32, 64, 128, 256, 512),
             kkt_tol=1e-2):
    """Batched inference on n_eval held-out snapshots: the network's time and relative error against
    target_iters-iteration plain FISTA, plain FISTA's error and time at the iteration counts in `sweep`,
    and how many snapshots the KKT check sends to the fallback."""
    mask = fixed_mask(cfg)
    y = snapshot_batch(cfg, mask, first, n_eval)
    L = cfg.L1 * cfg.L2
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def timed(fn):
        torch.cuda.synchronize()
        ev[0].record()
        out = fn()
        ev[1].record()
        torch.cuda.synchronize()
        return out, ev[0].elapsed_time(ev[1])

    inst = dict(M1=cfg.M1, M2=cfg.M2, L1=cfg.L1, L2=cfg.L2, mask=mask, y=np.zeros(cfg.N, np.complex64),
                lam=cfg.lam_frac, lam_is_frac=True)
    solver = B.BatchSolver([inst] * n_eval, "fista")
    out = torch.empty(n_eval * L, dtype=torch.complex64, device="cuda")
    solver.solve(y, 10, out, check=False)  # warm-up (setup, momentum table)

    def plain(iters):
        o = torch.empty(n_eval * L, dtype=torch.complex64, device="cuda")
        solver.solve(y, iters, o, check=False)
        return o

    ref, t_ref = timed(lambda: plain(cfg.target_iters))
    net = UnrolledNet(cfg.M1, cfg.M2, mask, cfg.L1, cfg.L2, n_eval, cfg.lam_frac)
    with torch.no_grad():
        net_forward(net, y, scale, thresh)  # warm-up
        c_net, t_net = timed(lambda: net_forward(net, y, scale, thresh))
    res = {"n_eval": n_eval, "layers": int(scale.numel()), "target_iters": cfg.target_iters,
           "target_ms": t_ref, "net_ms": t_net,
           "net_rel_err_mean": relative_errors(c_net, ref, n_eval, L).mean().item(),
           "net_rel_err_median": relative_errors(c_net, ref, n_eval, L).median().item(), "plain": {}}
    for it in sweep:
        o, t = timed(lambda: plain(it))
        e = relative_errors(o, ref, n_eval, L)
        res["plain"][it] = {"ms": t, "rel_err_mean": e.mean().item(), "rel_err_median": e.median().item()}
    _, kkt, fb = infer_with_fallback(net, y, scale, thresh, kkt_tol=kkt_tol, fallback_iters=1)
    res["kkt_tol"] = kkt_tol
    res["kkt_fail_fraction"] = float(fb.mean())
    res["kkt_median"] = float(np.median(kkt))
    net.close()
    solver.close()
    return res


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="train and evaluate the unrolled FISTA network")
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--layers", type=int, default=16)
    ap.add_argument("--lr", type=float, default=0.05)
    ap.add_argument("--eval", type=int, default=8192)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--resume", action="store_true")
    ap.add_argument("--save", default=None, help="write the trained multipliers and the loss curve (JSON)")
    args = ap.parse_args()
    cfg = TrainConfig(layers=args.layers, batch=args.batch, steps=args.steps, lr=args.lr,
                      checkpoint=args.checkpoint)
    import time

    t0 = time.time()
    a, t, hist = train(cfg, resume=args.resume, log=lambda m: print(m, flush=True))
    train_s = time.time() - t0
    res = evaluate(cfg, a, t, n_eval=args.eval)
    res.update({"train_steps": args.steps, "train_batch": args.batch, "train_snapshots": args.steps * args.batch,
                "train_seconds": train_s, "loss_first": hist[0] if hist else None,
                "loss_last": hist[-1] if hist else None, "scale": a.tolist(), "thresh": t.tolist()})
    if args.save:
        with open(args.save, "w") as f:
            json.dump({"layers": args.layers, "scale": a.tolist(), "thresh": t.tolist(),
                       "train_snapshots": args.steps * args.batch, "train_batch": args.batch, "lr": args.lr,
                       "train_seconds": train_s,
                       "loss_curve": [[i, float(v)] for i, v in enumerate(hist) if i % 10 == 0 or i == len(hist) - 1],
                       "eval": {k: v for k, v in res.items() if k not in ("scale", "thresh")}}, f, indent=1)
    print(json.dumps(res), flush=True)
