"""Learned warm start for the 2D Rayleigh-Benard cell.

A 4-layer 3x3 convolutional network (32 channels, ReLU, BF16 weights on the
tensor cores with FP32 accumulation and FP32 Adam master weights) maps, at the
65 x 65 coarse nodes of a 513 x 513 cell, five input channels to the
time-averaged temperature and velocity (T, u/U, v/U) of the statistically
steady flow.  Two input forms:

    "coords": conductive temperature, x, y (unit square), (log10 Ra - 7) / 1.5,
              (Pr - 3.855) / 3.145
    "coarse": the time-averaged T, u/U, v/U of a cheap 65 x 65 run of the same
              cell at the same (Ra, Pr) (the form the warm-start configuration
              names), (log10 Ra - 7) / 1.5, (Pr - 3.855) / 3.145

the second paying for the coarse run, counted in fine-step equivalents (its
steps times 65^2 / 513^2).  The prediction is upsampled vertex-aligned (coarse node (i, j) =
fine node (8i, 8j)) and the solver starts from f = f_eq(1, u), g = g_eq(T, u)
(tlbm_init_fields) instead of the conductive state.

Training data are time averages of the batched solver's own runs.  The solver,
the convolutions and their gradients, the loss, the optimiser, the upsampling
and the initial state run in this project's CUDA kernels through the C ABI;
torch holds the tensors and does the light bookkeeping (slicing and averaging
snapshots, scaling the predicted velocity to lattice units).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import tlbm

COARSE = 65
FINE = 513
FACTOR = 8
CIN, WIDTH, COUT, LAYERS = 5, 32, 3, 4


# ------------------------------------------------------------------ features


def features(Ra: float, Pr: float, n: int = COARSE, fine: int = FINE) -> np.ndarray:
    """Input channels at the coarse nodes (vertex-aligned with the fine cell)."""
    f = (fine - 1) // (n - 1)
    idx = np.arange(n) * f  # fine node index of each coarse node
    yy, xx = np.meshgrid(idx, idx, indexing="ij")
    t_cond = 0.5 - (yy + 0.5) / fine
    x = np.zeros((CIN, n, n), dtype=np.float32)
    x[0] = t_cond
    x[1] = xx / (fine - 1)
    x[2] = yy / (fine - 1)
    x[3] = (math.log10(Ra) - 7.0) / 1.5
    x[4] = (Pr - 3.855) / 3.145
    return x


def features_coarse(Ra: float, Pr: float, fields: np.ndarray) -> np.ndarray:
    """Input channels of the "coarse" form: fields = (3, 65, 65) time-averaged
    T, u/U, v/U of the 65 x 65 run."""
    x = np.zeros((CIN,) + fields.shape[1:], dtype=np.float32)
    x[0:3] = fields
    x[3] = (math.log10(Ra) - 7.0) / 1.5
    x[4] = (Pr - 3.855) / 3.145
    return x


def coarse_fields(draw_list, warm_tf: float = 30.0, avg_tf: float = 10.0, samples: int = 40,
                  precision=tlbm.TLBM_FP32):
    """Time-averaged (T, u/U, v/U) of a 65 x 65 run of each draw (same Ra, Pr,
    seed), canonical roll sense; a run that diverged (the 65^2 cell is far too
    coarse at the highest Ra) gives the conductive profile at rest.  Returns the
    fields, the per-draw divergence flags and the steps of one run."""
    import torch

    n = COARSE
    tf = free_fall_steps(n)
    U = 0.1 / math.sqrt(3.0)
    inst = [(n, n, 1, Ra, Pr, 0.1, seed) for Ra, Pr, seed in draw_list]
    b = tlbm.Batch(inst, lattice=tlbm.TLBM_D2Q9_D2Q5, precision=precision)
    b.init(1e-3)
    b.step(int(warm_tf * tf))
    every = max(1, int(avg_tf * tf / samples))
    acc = torch.zeros((len(inst), 3, n, n), dtype=torch.float64, device="cuda")
    T = torch.empty((n, n), dtype=torch.float32, device="cuda")
    ux = torch.empty_like(T)
    uy = torch.empty_like(T)
    for _ in range(samples):
        b.step(every)
        for k in range(len(inst)):
            tlbm.tlbm_batch_macros(b.b, k, None, ux, uy, None, T, tlbm.TLBM_OUT_F32)
            acc[k, 0] += T
            acc[k, 1] += ux / U
            acc[k, 2] += uy / U
    status = b.status()
    b.close()
    out = (acc / samples).float().cpu().numpy()
    yy = np.arange(n)[:, None]
    for k in range(len(inst)):
        if status[k] or not np.isfinite(out[k]).all():
            out[k] = 0.0
            out[k, 0] = 0.5 - (yy + 0.5) / n
    steps = int(warm_tf * tf) + samples * every
    return canonical_roll(out), status, steps


def draws(n: int, seed: int, log_ra=(6.0, 8.0), prs=(0.71, 7.0)):
    r = np.random.default_rng(seed)
    return [(float(10.0 ** r.uniform(*log_ra)), float(r.choice(prs)), 5000 + seed * 1000 + i) for i in range(n)]


# ------------------------------------------------------------------ network


class ConvNet:
    """3x3 conv stack on the project's kernels; activations NCHW."""

    def __init__(self, seed: int = 0, device: str = "cuda"):
        import torch

        self.torch = torch
        rng = np.random.default_rng(seed)
        chans = [CIN] + [WIDTH] * (LAYERS - 1) + [COUT]
        self.shapes = list(zip(chans[1:], chans[:-1]))  # (cout, cin)
        self.w, self.b, self.a, self.mw, self.vw, self.mb, self.vb = [], [], [], [], [], [], []
        for cout, cin in self.shapes:
            std = math.sqrt(2.0 / (9 * cin))
            w = torch.tensor(rng.normal(0, std, (cout, cin, 3, 3)), dtype=torch.float32, device=device)
            if cout == COUT:
                w *= 0.1
            self.w.append(w)
            self.b.append(torch.zeros(cout, dtype=torch.float32, device=device))
            self.a.append(torch.empty(tlbm.tlbm_conv3x3_weight_elems(cin), dtype=torch.bfloat16, device=device))
            self.mw.append(torch.zeros_like(w))
            self.vw.append(torch.zeros_like(w))
            self.mb.append(torch.zeros(cout, dtype=torch.float32, device=device))
            self.vb.append(torch.zeros(cout, dtype=torch.float32, device=device))
        self.t = 0
        self.pack()

    def pack(self):
        for (cout, cin), w, a in zip(self.shapes, self.w, self.a):
            tlbm.tlbm_conv3x3_pack_weights(w, cout, cin, a, self.torch.cuda.current_stream())

    def forward(self, x16, B: int, H: int, W: int):
        """x16: BF16 [B][CIN][H][W].  Returns the FP32 output and keeps what the
        backward pass needs."""
        torch = self.torch
        s = torch.cuda.current_stream()
        self.cache = []
        a_in = x16
        for k, (cout, cin) in enumerate(self.shapes):
            y = torch.empty((B, cout, H, W), dtype=torch.float32, device=x16.device)
            last = k == len(self.shapes) - 1
            act = None if last else torch.empty((B, cout, H, W), dtype=torch.bfloat16, device=x16.device)
            tlbm.tlbm_conv3x3_forward(a_in, self.a[k], self.b[k], y, act, B, cin, cout, H, W, 0 if last else 1, s)
            self.cache.append((a_in, y))
            a_in = act
        return y

    def backward(self, g32, g16, B: int, H: int, W: int):
        torch = self.torch
        s = torch.cuda.current_stream()
        at = torch.empty(32 * 288, dtype=torch.bfloat16, device=g32.device)
        self.gw = [None] * len(self.shapes)
        self.gb = [None] * len(self.shapes)
        for k in range(len(self.shapes) - 1, -1, -1):
            cout, cin = self.shapes[k]
            x_in, _ = self.cache[k]
            ws = torch.empty(tlbm.tlbm_conv3x3_workspace_bytes(B, cin, cout, H, W), dtype=torch.uint8,
                             device=g32.device)
            dw = torch.empty((cout, cin, 3, 3), dtype=torch.float32, device=g32.device)
            db = torch.empty(cout, dtype=torch.float32, device=g32.device)
            tlbm.tlbm_conv3x3_backward_weight(x_in, g16, g32, dw, db, B, cin, cout, H, W, ws, s)
            self.gw[k], self.gb[k] = dw, db
            if k > 0:
                wb = self.a_plain_bf16(k)
                dx = torch.empty((B, cin, H, W), dtype=torch.float32, device=g32.device)
                tlbm.tlbm_conv3x3_backward_data(g16, wb, dx, B, cin, cout, H, W, at, s)
                _, y_prev = self.cache[k - 1]
                g32 = torch.empty_like(dx)
                g16 = torch.empty(dx.shape, dtype=torch.bfloat16, device=g32.device)
                tlbm.tlbm_relu_backward(dx, y_prev, dx.numel(), g32, g16, s)

    def a_plain_bf16(self, k):
        """BF16 copy of layer k's weights in [cout][cin][3][3] order."""
        torch = self.torch
        w16 = torch.empty(self.w[k].shape, dtype=torch.bfloat16, device=self.w[k].device)
        tlbm.tlbm_to_bf16(self.w[k], self.w[k].numel(), w16, torch.cuda.current_stream())
        return w16

    def adam(self, lr: float):
        s = self.torch.cuda.current_stream()
        self.t += 1
        for k in range(len(self.shapes)):
            tlbm.tlbm_adam_step(self.w[k], self.gw[k], self.mw[k], self.vw[k], self.w[k].numel(), lr, 0.9, 0.999,
                                1e-8, self.t, s)
            tlbm.tlbm_adam_step(self.b[k], self.gb[k], self.mb[k], self.vb[k], self.b[k].numel(), lr, 0.9, 0.999,
                                1e-8, self.t, s)
        self.pack()

    def state(self):
        return {"w": [w.cpu().numpy() for w in self.w], "b": [b.cpu().numpy() for b in self.b]}


def train(net: ConvNet, X: np.ndarray, Y: np.ndarray, iters: int = 2000, lr: float = 2e-3, log_every: int = 200):
    """Full-batch Adam on the mean squared error; returns the loss history."""
    import torch

    B, _, H, W = X.shape
    s = torch.cuda.current_stream()
    x32 = torch.tensor(X, dtype=torch.float32, device="cuda")
    x16 = torch.empty(x32.shape, dtype=torch.bfloat16, device="cuda")
    tlbm.tlbm_to_bf16(x32, x32.numel(), x16, s)
    tgt = torch.tensor(Y, dtype=torch.float32, device="cuda")
    g32 = torch.empty_like(tgt)
    g16 = torch.empty(tgt.shape, dtype=torch.bfloat16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    part = torch.zeros(1024, dtype=torch.float64, device="cuda")
    hist = []
    for it in range(1, iters + 1):
        y = net.forward(x16, B, H, W)
        tlbm.tlbm_mse_loss(y, tgt, y.numel(), g32, g16, loss, part, s)
        net.backward(g32, g16, B, H, W)
        net.adam(lr if it < 0.7 * iters else lr * 0.2)
        if it == 1 or it % log_every == 0 or it == iters:
            hist.append((it, float(loss.item())))
    return hist


def factor(fine: int) -> int:
    """Fine nodes per coarse interval; the cells are vertex-aligned (fine = 64 k + 1)."""
    if fine < COARSE or (fine - 1) % (COARSE - 1):
        raise ValueError(f"fine size {fine} is not 64 k + 1")
    return (fine - 1) // (COARSE - 1)


def predict(net: ConvNet, Ra: float, Pr: float, fine: int = FINE, x: np.ndarray | None = None):
    """Coarse (3, 65, 65) FP32 prediction on the device: T, u/U, v/U (x: the
    input channels; default the "coords" form)."""
    import torch

    s = torch.cuda.current_stream()
    x = features(Ra, Pr, fine=fine) if x is None else x
    x32 = torch.tensor(x[None], dtype=torch.float32, device="cuda")
    x16 = torch.empty(x32.shape, dtype=torch.bfloat16, device="cuda")
    tlbm.tlbm_to_bf16(x32, x32.numel(), x16, s)
    return net.forward(x16, 1, COARSE, COARSE)[0]


def warm_start(h, coarse, U: float, fine: int = FINE):
    """Upsample a coarse (T, u/U, v/U) prediction to the fine cell and start the
    solver from it."""
    import torch

    s = torch.cuda.current_stream()
    up = torch.empty((3, fine, fine), dtype=torch.float32, device="cuda")
    tlbm.tlbm_upsample_bilinear(coarse.contiguous(), 3, COARSE, COARSE, factor(fine), up, s)
    T = up[0].clamp(-0.5, 0.5).contiguous()
    ux = (up[1] * U).contiguous()
    uy = (up[2] * U).contiguous()
    tlbm.tlbm_init_fields(h, T, ux, uy, None)


# ------------------------------------------------------------------ data and evaluation


def free_fall_steps(n: int = FINE, Ma: float = 0.1) -> int:
    return int(math.ceil(n / (Ma / math.sqrt(3.0))))


def canonical_roll(Y: np.ndarray) -> np.ndarray:
    """Mirror (x -> 1 - x, u -> -u) every target whose mean circulation is
    clockwise-negative, so that all targets share one roll direction.

    The sense of the large-scale roll is picked by the initial noise (the cell is
    mirror-symmetric), so raw time averages of different seeds would cancel in
    the fit; both senses carry the same Nusselt number."""
    Y = np.array(Y, copy=True)
    n = Y.shape[-1]
    yc = (np.arange(n) - 0.5 * (n - 1))[:, None]
    for k in range(Y.shape[0]):
        circ = float((Y[k, 1] * yc).sum())  # u > 0 above the centre, u < 0 below: positive
        if circ < 0.0:
            Y[k] = Y[k][:, :, ::-1]
            Y[k, 1] *= -1.0
    return Y


def generate(draw_list, warm_tf: float, avg_tf: float, samples: int, precision=tlbm.TLBM_FP32, fine: int = FINE):
    """Time-averaged coarse (T, u/U, v/U) of each draw's statistically steady run."""
    import torch

    f = factor(fine)
    tf = free_fall_steps(fine)
    U = 0.1 / math.sqrt(3.0)
    inst = [(fine, fine, 1, Ra, Pr, 0.1, seed) for Ra, Pr, seed in draw_list]
    b = tlbm.Batch(inst, lattice=tlbm.TLBM_D2Q9_D2Q5, precision=precision)
    b.init(1e-3)
    b.step(int(warm_tf * tf))
    every = max(1, int(avg_tf * tf / samples))
    acc = torch.zeros((len(inst), 3, COARSE, COARSE), dtype=torch.float64, device="cuda")
    T = torch.empty((fine, fine), dtype=torch.float32, device="cuda")
    ux = torch.empty_like(T)
    uy = torch.empty_like(T)
    for _ in range(samples):
        b.step(every)
        for k in range(len(inst)):
            tlbm.tlbm_batch_macros(b.b, k, None, ux, uy, None, T, tlbm.TLBM_OUT_F32)
            acc[k, 0] += T[::f, ::f]
            acc[k, 1] += ux[::f, ::f] / U
            acc[k, 2] += uy[::f, ::f] / U
    status = b.status()
    b.close()
    return (acc / samples).float().cpu().numpy(), status


def steps_to_steady(nu: np.ndarray, dt: int, window: int, ref: float, tol: float = 0.01, hold: int = 2):
    """First step after which the trailing mean of Nu over `window` samples
    stays within tol of ref for hold * window samples (None if never).

    Meaningful for flows that settle to a steady state; a chaotic cell's Nu keeps
    fluctuating by far more than 1 % and never holds."""
    n = len(nu)
    if n < window:
        return None
    tm = np.convolve(nu, np.ones(window) / window, mode="valid")  # tm[k] = mean(nu[k : k+window])
    ok = np.abs(tm - ref) <= tol * abs(ref)
    need = hold * window
    for k in range(len(ok)):
        if ok[k:k + need].all() and len(ok[k:k + need]) == need:
            return (k + window) * dt
    return None


def steps_to_reach(nu: np.ndarray, dt: int, window: int, ref: float, tol: float = 0.01):
    """First step at which the trailing mean of Nu over `window` samples comes
    within tol of ref or crosses it (None if never): the end of the start-up
    transient, defined also for a statistically steady, fluctuating Nu."""
    if len(nu) < window:
        return None
    tm = np.convolve(nu, np.ones(window) / window, mode="valid")
    d = tm - ref
    for k in range(len(d)):
        if abs(d[k]) <= tol * abs(ref) or (k > 0 and np.sign(d[k]) != np.sign(d[k - 1])):
            return (k + window) * dt
    return None


def evaluate(net: ConvNet, draw_list, run_tf: float, ref_tf: float, samples_per_tf: int = 16,
             precision=tlbm.TLBM_FP32, fine: int = FINE):
    """Conductive start vs learned warm start on the same draws (one batch)."""
    import torch

    tf = free_fall_steps(fine)
    U = 0.1 / math.sqrt(3.0)
    n = len(draw_list)
    inst = [(fine, fine, 1, Ra, Pr, 0.1, seed) for Ra, Pr, seed in draw_list] * 2
    b = tlbm.Batch(inst, lattice=tlbm.TLBM_D2Q9_D2Q5, precision=precision)
    b.init(1e-3)
    for k, (Ra, Pr, _) in enumerate(draw_list):
        warm_start(b.instance(n + k), predict(net, Ra, Pr, fine), U, fine)
    torch.cuda.synchronize()
    dt = max(1, tf // samples_per_tf)
    total = int(run_tf * samples_per_tf)
    nus = np.zeros((2 * n, total))
    for s_ in range(total):
        b.step(dt)
        nus[:, s_] = b.nusselt(allow_diverged=True)  # the status is recorded below
    status = b.status()
    b.close()
    window = samples_per_tf // 2  # half a free-fall time
    series = {"dt": dt, "samples_per_tf": samples_per_tf, "nu": np.round(nus, 5).tolist()}
    out = []
    ref_samples = int(ref_tf * samples_per_tf)
    for k, (Ra, Pr, seed) in enumerate(draw_list):
        ref = float(nus[k, -ref_samples:].mean())
        tail = nus[k, -ref_samples:]
        out.append({"Ra": Ra, "Pr": Pr, "Nu_ref": ref, "Nu_ref_rel_std": float(tail.std() / abs(ref)),
                    "steps_conductive": steps_to_reach(nus[k], dt, window, ref),
                    "steps_warm": steps_to_reach(nus[n + k], dt, window, ref),
                    "held_conductive": steps_to_steady(nus[k], dt, window, ref),
                    "held_warm": steps_to_steady(nus[n + k], dt, window, ref),
                    "diverged": bool(status[k] or status[n + k])})
    return out, series


def evaluate_starts(draw_list, starts: dict, run_tf: float, ref_tf: float, samples_per_tf: int = 16,
                    precision=tlbm.TLBM_FP32, fine: int = FINE, extra_cost: dict | None = None):
    """The conductive start and every learned start of `starts` (name -> list
    of coarse (3, 65, 65) device predictions, one per draw) on the same draws,
    in one batch.  extra_cost[name]: fine-step equivalents spent before the
    start (a coarse run), added to its step counts.  Per draw: the reference Nu
    (the conductive run's mean over its last ref_tf free-fall times) and, per
    start, the steps to reach and to hold it (None if never)."""
    import torch

    tf = free_fall_steps(fine)
    U = 0.1 / math.sqrt(3.0)
    n = len(draw_list)
    names = list(starts)
    inst = [(fine, fine, 1, Ra, Pr, 0.1, seed) for Ra, Pr, seed in draw_list] * (1 + len(names))
    b = tlbm.Batch(inst, lattice=tlbm.TLBM_D2Q9_D2Q5, precision=precision)
    b.init(1e-3)
    for g, name in enumerate(names):
        for k in range(n):
            warm_start(b.instance((g + 1) * n + k), starts[name][k], U, fine)
    torch.cuda.synchronize()
    dt = max(1, tf // samples_per_tf)
    total = int(run_tf * samples_per_tf)
    nus = np.zeros((len(inst), total))
    for s_ in range(total):
        b.step(dt)
        nus[:, s_] = b.nusselt(allow_diverged=True)  # the status is recorded below
    status = b.status()
    b.close()
    window = samples_per_tf // 2  # half a free-fall time
    ref_samples = int(ref_tf * samples_per_tf)
    extra_cost = extra_cost or {}
    out = []
    for k, (Ra, Pr, seed) in enumerate(draw_list):
        ref = float(nus[k, -ref_samples:].mean())
        e = {"Ra": Ra, "Pr": Pr, "Nu_ref": ref, "Nu_ref_rel_std": float(nus[k, -ref_samples:].std() / abs(ref)),
             "steps_conductive": steps_to_reach(nus[k], dt, window, ref),
             "held_conductive": steps_to_steady(nus[k], dt, window, ref),
             "diverged": bool(status[k])}
        for g, name in enumerate(names):
            row = (g + 1) * n + k
            cost = int(extra_cost.get(name, [0] * n)[k])
            r, h = steps_to_reach(nus[row], dt, window, ref), steps_to_steady(nus[row], dt, window, ref)
            e[f"steps_{name}"] = None if r is None else r + cost
            e[f"held_{name}"] = None if h is None else h + cost
            e[f"cost_{name}"] = cost
            e["diverged"] = e["diverged"] or bool(status[row])
        out.append(e)
    return out, {"dt": dt, "samples_per_tf": samples_per_tf, "nu": np.round(nus, 5).tolist(), "starts": names}


def summarize_starts(ev, names) -> dict:
    """Per learned start: median step ratio conductive / learned for both
    criteria, over the draws where both runs met it."""
    res = {}
    for name in names:
        res[name] = {}
        for key, a, b in (("reach", "steps_conductive", f"steps_{name}"),
                          ("held", "held_conductive", f"held_{name}")):
            both = [e for e in ev if e[a] and e[b] and not e["diverged"]]
            res[name][key] = {"compared": len(both), "faster": sum(e[b] < e[a] for e in both),
                              "median_speedup": float(np.median([e[a] / e[b] for e in both])) if both else None,
                              "median_steps_conductive": float(np.median([e[a] for e in both])) if both else None,
                              "median_steps_learned": float(np.median([e[b] for e in both])) if both else None}
    return res


def summarize(ev) -> dict:
    """Median step ratio conductive / warm for both criteria, over the draws
    where both runs met it."""
    res = {}
    for key, a, b in (("reach", "steps_conductive", "steps_warm"), ("held", "held_conductive", "held_warm")):
        both = [e for e in ev if e[a] and e[b] and not e["diverged"]]
        res[key] = {"compared": len(both), "warm_faster": sum(e[b] < e[a] for e in both),
                    "median_speedup": float(np.median([e[a] / e[b] for e in both])) if both else None,
                    "median_steps_conductive": float(np.median([e[a] for e in both])) if both else None,
                    "median_steps_warm": float(np.median([e[b] for e in both])) if both else None}
    return res


def time_layers(batch: int = 48, n: int = COARSE, reps: int = 20, warmup: int = 3):
    """CUDA-event timings (ms per call, median over reps) of the 32 -> 32
    channel layer at the training batch: forward (tcgen05), data gradient
    (tcgen05) and weight gradient (tcgen05), each with the FLOPs of its GEMM
    (2 x pixels x 32 x 288) as TFLOP/s and its compulsory HBM bytes as GB/s."""
    import torch

    s = torch.cuda.current_stream()
    B, C, M = batch, WIDTH, WIDTH
    g = torch.Generator(device="cpu").manual_seed(0)
    x = (torch.rand((B, C, n, n), generator=g) * 2 - 1).to(torch.bfloat16).cuda()
    w = ((torch.rand((M, C, 3, 3), generator=g) * 2 - 1) * 0.1).cuda()
    bias = torch.zeros(M, dtype=torch.float32, device="cuda")
    a = torch.empty(tlbm.tlbm_conv3x3_weight_elems(C), dtype=torch.bfloat16, device="cuda")
    tlbm.tlbm_conv3x3_pack_weights(w, M, C, a, s)
    w16 = w.to(torch.bfloat16)
    y = torch.empty((B, M, n, n), dtype=torch.float32, device="cuda")
    act = torch.empty((B, M, n, n), dtype=torch.bfloat16, device="cuda")
    dy32 = torch.empty_like(y).uniform_(-1, 1)
    dy16 = dy32.to(torch.bfloat16)
    dx = torch.empty((B, C, n, n), dtype=torch.float32, device="cuda")
    at = torch.empty(32 * 288, dtype=torch.bfloat16, device="cuda")
    ws = torch.empty(tlbm.tlbm_conv3x3_workspace_bytes(B, C, M, n, n), dtype=torch.uint8, device="cuda")
    dw = torch.empty((M, C, 3, 3), dtype=torch.float32, device="cuda")
    db = torch.empty(M, dtype=torch.float32, device="cuda")
    ops = {
        "forward": (lambda: tlbm.tlbm_conv3x3_forward(x, a, bias, y, act, B, C, M, n, n, 1, s),
                    x.numel() * 2 + y.numel() * 6),
        "backward_data": (lambda: tlbm.tlbm_conv3x3_backward_data(dy16, w16, dx, B, C, M, n, n, at, s),
                          dy16.numel() * 2 + dx.numel() * 4),
        "backward_weight": (lambda: tlbm.tlbm_conv3x3_backward_weight(x, dy16, dy32, dw, db, B, C, M, n, n, ws, s),
                            x.numel() * 2 + dy16.numel() * 2 + dy32.numel() * 4),
    }
    flops = 2.0 * B * n * n * M * C * 9
    out = {"batch": B, "n": n, "cin": C, "cout": M, "gemm_flops": flops}
    for name, (fn, nbytes) in ops.items():
        for _ in range(warmup):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        out[name] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12, "gbs": nbytes / (ms * 1e-3) / 1e9}
    out["timeouts"] = tlbm.tlbm_conv3x3_status()
    return out


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser(description="train and evaluate the learned warm start")
    ap.add_argument("--train-draws", type=int, default=48)
    ap.add_argument("--eval-draws", type=int, default=16)
    ap.add_argument("--warm-tf", type=float, default=40.0)
    ap.add_argument("--avg-tf", type=float, default=20.0)
    ap.add_argument("--samples", type=int, default=80)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--run-tf", type=float, default=60.0)
    ap.add_argument("--ref-tf", type=float, default=20.0)
    ap.add_argument("--coarse-warm-tf", type=float, default=30.0, help="65^2 run: free-fall times before averaging")
    ap.add_argument("--coarse-avg-tf", type=float, default=10.0, help="65^2 run: free-fall times averaged")
    ap.add_argument("--fine", type=int, default=FINE, help="fine cell size, 64 k + 1")
    ap.add_argument("--log-ra", type=float, nargs=2, default=(6.0, 8.0), help="log10 Ra range of the draws")
    ap.add_argument("--input", default="both", choices=["coords", "coarse", "both"])
    ap.add_argument("--out", default="", help="write the full result (per-draw steps and Nu series), JSON")
    ap.add_argument("--out-compact", default="",
                    help="write the result without the Nu series, with the command and the device, JSON")
    ap.add_argument("--save-data", default="", help="write the generated training targets (.npz)")
    ap.add_argument("--load-data", default="", help="reuse training targets written by --save-data")
    ap.add_argument("--time-layers", action="store_true",
                    help="only time the 32-channel layer's forward and gradients at the training batch, JSON")
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    if args.time_layers:
        print(json.dumps(time_layers(batch=args.train_draws)))
        return 0
    t0 = time.time()
    tr = draws(args.train_draws, seed=1, log_ra=tuple(args.log_ra))
    ev_draws = draws(args.eval_draws, seed=2, log_ra=tuple(args.log_ra))
    if args.load_data:
        z = np.load(args.load_data)
        Y, st = z["Y"], list(z["status"])
    else:
        Y, st = generate(tr, args.warm_tf, args.avg_tf, args.samples, fine=args.fine)
    if args.save_data:
        np.savez(args.save_data, Y=Y, status=np.array(st))
    Y = canonical_roll(Y)
    keep = [k for k in range(len(tr)) if not st[k] and np.isfinite(Y[k]).all()]
    modes = ["coords", "coarse"] if args.input == "both" else [args.input]
    t1 = time.time()
    res = {"fine": args.fine, "log_ra": list(args.log_ra), "train_draws": len(tr), "train_kept": len(keep),
           "eval_draws": len(ev_draws), "run_tf": args.run_tf, "ref_tf": args.ref_tf, "inputs": {}}
    starts, costs = {}, {}
    for mode in modes:
        tm = time.time()
        if mode == "coords":
            X = np.stack([features(Ra, Pr, fine=args.fine) for Ra, Pr, _ in tr])
            Xe = [features(Ra, Pr, fine=args.fine) for Ra, Pr, _ in ev_draws]
            cost = [0] * len(ev_draws)
            info = {}
        else:
            ftr, sttr, steps_c = coarse_fields(tr, args.coarse_warm_tf, args.coarse_avg_tf)
            fev, stev, _ = coarse_fields(ev_draws, args.coarse_warm_tf, args.coarse_avg_tf)
            X = np.stack([features_coarse(Ra, Pr, f) for (Ra, Pr, _), f in zip(tr, ftr)])
            Xe = [features_coarse(Ra, Pr, f) for (Ra, Pr, _), f in zip(ev_draws, fev)]
            ratio = (COARSE * COARSE) / float(args.fine * args.fine)
            cost = [int(round(steps_c * ratio))] * len(ev_draws)
            info = {"coarse_steps": steps_c, "coarse_cost_fine_steps": cost[0],
                    "coarse_diverged_train": int(sum(bool(x) for x in sttr)),
                    "coarse_diverged_eval": int(sum(bool(x) for x in stev))}
        net = ConvNet(seed=0)
        hist = train(net, X[keep], Y[keep], iters=args.iters)
        starts[mode] = [predict(net, Ra, Pr, args.fine, x) for (Ra, Pr, _), x in zip(ev_draws, Xe)]
        costs[mode] = cost
        torch.cuda.synchronize()
        res["inputs"][mode] = dict(info, loss=hist, seconds=time.time() - tm)
    t2 = time.time()
    ev, series = evaluate_starts(ev_draws, starts, args.run_tf, args.ref_tf, fine=args.fine, extra_cost=costs)
    t3 = time.time()
    res.update({"summary": summarize_starts(ev, modes), "eval": ev, "series": series,
                "seconds": {"data": t1 - t0, "train": t2 - t1, "eval": t3 - t2}})
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(json.dumps(res))
    del res["series"]
    if args.out_compact:
        props = torch.cuda.get_device_properties(0)
        given = list(argv if argv is not None else sys.argv[1:])
        kept = []  # the command without the output paths
        while given:
            a = given.pop(0)
            if a in ("--out", "--out-compact", "--save-data", "--load-data"):
                if given:
                    given.pop(0)
                continue
            if a.split("=", 1)[0] in ("--out", "--out-compact", "--save-data", "--load-data"):
                continue
            kept.append(a)
        compact = dict(res, command=" ".join(["python -m paper_2211_03160_gb300.surrogate"] + kept),
                       hardware=f"{props.name} (sm_{props.major}{props.minor}), FP32 storage for every run")
        with open(args.out_compact, "w") as fh:
            fh.write(json.dumps(compact, indent=1))
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
