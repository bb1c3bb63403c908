"""Learned-DBP training loop (Sec. IV-B/IV-C) on the library's own kernels.

Per iteration, on the GPU: 16-QAM frames with a launch power drawn per frame
from the training set (Sec. IV-B), RRC pulse shaping (ldbp_tx), the channel
with ASE noise (ssm_forward), the LDBP forward pass with step checkpoints
(ldbp_apply), the receiver loss and its gradient (ldbp_rx), the hand-written
adjoint (ldbp_backward) and Adam (ldbp_adam_step).  The host only draws the
symbol indices and powers (seeded), and keeps the pruning schedule: at
predefined, front-loaded iterations the outermost tap pair of one filter is
removed (Sec. IV-C, Example 2), choosing the filter whose outermost tap has
the smallest magnitude among those above their target length.

Options: learnable nonlinear coefficients c_i (the scaling of Remark 1; their
gradients come from ldbp_backward_c and a host-side Adam updates the M
values), and the filter initialisations of Sec. V-E: least squares (default),
unit filters (h = (1, 0, ..., 0), link-agnostic) and random filters
(i.i.d. N(0, 1) real and imaginary parts, divided by sum_{k=-K}^{K} |h_k|^2).
"""
from __future__ import annotations

import dataclasses
import json
import math

import numpy as np
import torch

import synth
from . import api, init


@dataclasses.dataclass
class TrainConfig:
    batch: int = 64
    nsym: int = 16384
    sps: int = 2
    rolloff: float = 0.1
    baud: float = 10e9
    n_spans: int = 25
    span_km: float = 80.0
    channel_steps: int = 100
    ase: bool = True
    nf_db: float = 5.0
    powers_dbm: tuple = tuple(range(-4, 7))
    t_start: int = 31
    t_end: int = 3
    t_end_odd: int = 0             # > 0: filters at odd step indices are pruned to this length (alternating, Sec. V-B)
    iters: int = 1000
    lr: float = 1e-3
    lr_final: float = 0.0          # cosine decay from lr to lr_final over the run (0: constant lr)
    prune_frac: float = 0.6
    w_max: float = 0.0             # LS-fit half band (rad/sample); 0: the signal band
    seed: int = 3
    linear_only: bool = False
    learn_c: bool = False          # train the nonlinear coefficients too (Remark 1)
    kappa: int = 0                 # > 0: learned enhanced SSM, a (2 kappa + 1)-tap filter on |v|^2 per step
    init: str = "ls"               # "ls", "unit" or "random" filters (Sec. V-E)
    data_pool: int = 0             # > 0: make this many batches with the channel once and cycle through them

    @property
    def fs(self):
        return self.baud * self.sps

    @property
    def n(self):
        return self.nsym * self.sps


def iteration_record(step: int, loss: float, lr: float, T) -> dict:
    """One line of the training log.  The loss is the batch-mean ||s_hat - s||^2 / N_sym
    with E|s|^2 = 1, so 10 log10(1 / loss) is the batch's effective SNR (Eq. (14))
    up to the sample mean of |s|^2."""
    snr = 10.0 * math.log10(1.0 / loss) if loss > 0 else float("inf")
    return {"step": int(step), "loss": float(loss), "snr_db": snr, "lr": float(lr),
            "taps": int(sum(T)), "T": [int(t) for t in T]}


def prune_choice(taps, lengths, targets) -> int:
    """Which filter loses its outermost tap pair at a pruning step (Sec. IV-C):
    among the filters still longer than their target, the one whose outermost
    tap h_K (K = (T - 1) / 2) has the smallest magnitude; ties go to the
    lowest step index.  taps: [M, stride] half-tap vectors; targets: one
    length for all filters or one per filter; returns -1 when every filter is
    at its target."""
    tg = [int(targets)] * len(lengths) if np.isscalar(targets) else [int(t) for t in targets]
    best, mag = -1, np.inf
    for i, T in enumerate(lengths):
        if T > tg[i]:
            a = abs(taps[i][(T - 1) // 2])
            if a < mag:
                best, mag = i, a
    return best


def pruning_schedule(total_steps: int, iters: int, frac: float):
    """Front-loaded pruning iterations floor(frac iters (j/P)^2), j = 1..P."""
    return [int(math.floor(frac * iters * (j / total_steps) ** 2)) for j in range(1, total_steps + 1)]


class Trainer:
    def __init__(self, cfg: TrainConfig, fiber=None):
        self.cfg = cfg
        self.fiber = fiber or synth.Fiber()
        M = cfg.n_spans
        self.M = M
        self.T = [cfg.t_start] * M
        taps, c = init.ldbp_init(self.T, span_km=cfg.span_km, fs=cfg.fs, fiber=self.fiber, sps=cfg.sps,
                                 rolloff=cfg.rolloff, w_max=cfg.w_max or None)
        if cfg.init == "unit":
            taps = init.unit_filters(self.T)
        elif cfg.init == "random":
            taps = init.random_filters(self.T, cfg.seed)
        elif cfg.init != "ls":
            raise ValueError(f"unknown initialisation {cfg.init!r}")
        self.c = [0.0] * M if cfg.linear_only else [float(np.float32(ci)) for ci in c]
        self.mc = np.zeros(M)
        self.vc = np.zeros(M)
        if cfg.kappa > 0:  # filters on |v|^2, unit-initialised; stored with an even stride (complex view for Adam)
            if cfg.learn_c:
                raise ValueError("learn_c is not supported together with kappa > 0")
            self.eta = torch.zeros((M, 2 * cfg.kappa + 2), dtype=torch.float32, device="cuda")
            self.eta[:, cfg.kappa] = 1.0
            self.me = torch.zeros_like(self.eta)
            self.ve = torch.zeros_like(self.eta)
        self.stride = (cfg.t_start - 1) // 2 + 1
        arr = np.zeros((M, self.stride), np.complex64)
        for i, h in enumerate(taps):
            arr[i, : len(h)] = h
        self.taps = torch.from_numpy(arr).cuda()
        self.m = torch.zeros((M, self.stride, 2), dtype=torch.float32, device="cuda")
        self.v = torch.zeros_like(self.m)
        self.step_count = 0
        self.targets = [cfg.t_end_odd if (cfg.t_end_odd > 0 and i % 2 == 1) else cfg.t_end for i in range(M)]
        steps = sum((cfg.t_start - t) // 2 for t in self.targets)
        self.schedule = pruning_schedule(steps, cfg.iters, cfg.prune_frac) if steps else []
        B, n = cfg.batch, cfg.n
        self.ckpt = torch.empty((M, B, n), dtype=torch.complex64, device="cuda")
        self.out = torch.empty((B, n), dtype=torch.complex64, device="cuda")
        self.ws_rx = torch.empty((B, n), dtype=torch.complex64, device="cuda")
        self.ws_bwd = None
        self.history = []
        self.pool = [self._make_frames(it) for it in range(cfg.data_pool)]

    # ------------------------------------------------------------------ data
    def link(self, counter: int):
        cfg = self.cfg
        return synth.Link(cfg.n_spans, cfg.span_km, cfg.channel_steps, True, cfg.ase, cfg.nf_db, 1.946e14,
                          seed=cfg.seed * 1000003 + 17, counter=counter)

    def frames(self, it: int, batch=None, powers_dbm=None):
        """Symbols (device complex64 [B, nsym]), launch powers (device float32 [B]) and received waveforms;
        with a data pool, training iteration it reuses pool batch it mod data_pool."""
        if self.pool and batch is None and powers_dbm is None:
            return self.pool[it % len(self.pool)]
        return self._make_frames(it, batch, powers_dbm)

    def _make_frames(self, it: int, batch=None, powers_dbm=None):
        cfg = self.cfg
        B = batch or cfg.batch
        s = synth.qam16_symbols(B, cfg.nsym, cfg.seed * 7919 + it).astype(np.complex64)
        pd = synth.launch_powers_dbm(B, cfg.seed * 104729 + it, powers_dbm or cfg.powers_dbm)
        p = (1e-3 * 10.0 ** (pd / 10.0)).astype(np.float32)
        sd = torch.from_numpy(s).cuda()
        pw = torch.from_numpy(p).cuda()
        x = api.tx(sd, pw, sps=cfg.sps, rolloff=cfg.rolloff)
        y = api.ssm_forward(self.fiber, self.link(it), cfg.fs, x, out=x)
        return sd, pw, y

    # ------------------------------------------------------------------ training
    def train_step(self, it: int) -> float:
        cfg = self.cfg
        sd, pw, y = self.frames(it)
        if cfg.kappa > 0:
            return self._train_step_essm(it, sd, pw, y)
        api.ldbp_apply(self.taps, self.T, self.c, y, ckpt=self.ckpt, out=self.out)
        stats, _, g = api.rx(self.out, sd, pw, sps=cfg.sps, rolloff=cfg.rolloff, grad=True, workspace=self.ws_rx)
        need = api.ldbp_backward_workspace_bytes(cfg.n, cfg.batch, self.T)
        if self.ws_bwd is None or self.ws_bwd.numel() < need:
            self.ws_bwd = torch.empty(need, dtype=torch.uint8, device="cuda")
        res = api.ldbp_backward(self.taps, self.T, self.c, self.ckpt, g, want_gx=False, workspace=self.ws_bwd,
                                want_gc=cfg.learn_c)
        gt = res[1]
        self.step_count += 1
        api.adam_step(self.taps, gt, self.m, self.v, self.T, self.step_count, lr=self.lr_at(it))
        if cfg.learn_c:
            self.adam_c(res[2].cpu().numpy().astype(np.float64), self.lr_at(it))
        while self.schedule and self.schedule[0] <= it:
            self.schedule.pop(0)
            self.prune_one()
        loss = float(stats[:, 0].mean().item())
        self.history.append(loss)
        return loss

    def _train_step_essm(self, it, sd, pw, y):
        """One iteration of the learned enhanced SSM: taps and the |v|^2 filters by Adam."""
        cfg = self.cfg
        ks = [cfg.kappa] * self.M
        api.ldbp_essm_apply(self.taps, self.T, self.c, self.eta, ks, y, ckpt=self.ckpt, out=self.out)
        stats, _, g = api.rx(self.out, sd, pw, sps=cfg.sps, rolloff=cfg.rolloff, grad=True, workspace=self.ws_rx)
        _, gt, ge = api.ldbp_essm_backward(self.taps, self.T, self.c, self.eta, ks, self.ckpt, g, want_gx=False)
        self.step_count += 1
        lr = self.lr_at(it)
        api.adam_step(self.taps, gt, self.m, self.v, self.T, self.step_count, lr=lr)
        api.adam_step(torch.view_as_complex(self.eta.view(self.M, -1, 2)), torch.view_as_complex(ge.view(self.M, -1, 2)),
                      self.me.view(self.M, -1, 2), self.ve.view(self.M, -1, 2), [2 * cfg.kappa + 1] * self.M,
                      self.step_count, lr=lr)
        while self.schedule and self.schedule[0] <= it:
            self.schedule.pop(0)
            self.prune_one()
        loss = float(stats[:, 0].mean().item())
        self.history.append(loss)
        return loss

    def apply(self, y):
        """The trained model on received waveforms y (device complex64 [B, n])."""
        if self.cfg.kappa > 0:
            return api.ldbp_essm_apply(self.taps, self.T, self.c, self.eta, [self.cfg.kappa] * self.M, y)
        return api.ldbp_apply(self.taps, self.T, self.c, y)

    def adam_c(self, gc, lr, b1=0.9, b2=0.999, eps=1e-8):
        """Adam on the nonlinear coefficients (host side, M values; same step count as the taps)."""
        t = self.step_count
        self.mc = b1 * self.mc + (1 - b1) * gc
        self.vc = b2 * self.vc + (1 - b2) * gc * gc
        mh = self.mc / (1 - b1 ** t)
        vh = self.vc / (1 - b2 ** t)
        self.c = [float(np.float32(ci - lr * m / (np.sqrt(v) + eps))) for ci, m, v in zip(self.c, mh, vh)]

    def lr_at(self, it: int) -> float:
        cfg = self.cfg
        if cfg.lr_final <= 0.0:
            return cfg.lr
        f = min(1.0, it / max(1, cfg.iters - 1))
        return cfg.lr_final + 0.5 * (cfg.lr - cfg.lr_final) * (1.0 + math.cos(math.pi * f))

    def prune_one(self):
        """Remove the outermost tap pair of one filter (Sec. IV-C)."""
        best = prune_choice(self.taps.cpu().numpy(), self.T, self.targets)
        if best >= 0:
            self.T[best] -= 2

    def fit(self, iters=None, log_every=0, log_path=None):
        """Runs the iterations; with log_path, appends one JSON line per iteration
        (iteration, loss, effective SNR of the batch, learning rate, filter lengths)."""
        log = open(log_path, "a") if log_path else None
        try:
            for it in range(iters or self.cfg.iters):
                loss = self.train_step(it)
                rec = iteration_record(self.step_count, loss, self.lr_at(it), self.T)
                if log is not None:
                    log.write(json.dumps(rec) + "\n")
                if log_every and it % log_every == 0:
                    print(f"it {it:5d} loss {loss:.4e} snr {rec['snr_db']:.2f} dB taps {rec['taps']}")
        finally:
            if log is not None:
                log.close()
        return self.history

    # ------------------------------------------------------------------ evaluation
    def evaluate(self, frames: int = 4, power_dbm: float = 0.0, first_frame: int = 10_000_000):
        """Effective SNR (dB) of LDBP, of 1-StPS FD DBP and of no compensation at one power."""
        cfg = self.cfg
        acc = {"ldbp": [0.0, 0.0], "dbp": [0.0, 0.0]}
        for f in range(frames):
            sd, pw, y = self.frames(first_frame + f, powers_dbm=(power_dbm,))
            out = self.apply(y)
            st, _, _ = api.rx(out, sd, pw, sps=cfg.sps, rolloff=cfg.rolloff)
            z = api.dbp_apply(self.fiber, self.link(0), cfg.fs, y, steps_per_span=1, symmetric=False)
            sd2, _, _ = api.rx(z, sd, pw, sps=cfg.sps, rolloff=cfg.rolloff)
            for key, s in (("ldbp", st), ("dbp", sd2)):
                s = s.double().cpu()
                acc[key][0] += float(s[:, 1].sum())
                acc[key][1] += float(s[:, 0].sum())
        return {k: 10 * np.log10(a / b) for k, (a, b) in acc.items()}

    # ------------------------------------------------------------------ checkpoint / resume
    def state(self):
        return {"taps": self.taps.cpu().numpy(), "T": np.array(self.T), "c": np.array(self.c),
                "m": self.m.cpu().numpy(), "v": self.v.cpu().numpy(), "step": self.step_count,
                "schedule": np.array(self.schedule, dtype=np.int64), "mc": self.mc, "vc": self.vc,
                **({"eta": self.eta.cpu().numpy(), "me": self.me.cpu().numpy(), "ve": self.ve.cpu().numpy()}
                   if self.cfg.kappa > 0 else {})}

    def save(self, path):
        np.savez(path, **self.state())

    def load(self, path):
        d = np.load(path)
        self.taps.copy_(torch.from_numpy(d["taps"]))
        self.T = [int(t) for t in d["T"]]
        self.c = [float(x) for x in d["c"]]
        self.m.copy_(torch.from_numpy(d["m"]))
        self.v.copy_(torch.from_numpy(d["v"]))
        self.step_count = int(d["step"])
        self.schedule = [int(t) for t in d["schedule"]]
        if "mc" in d:
            self.mc, self.vc = np.array(d["mc"]), np.array(d["vc"])
        if self.cfg.kappa > 0:
            for name in ("eta", "me", "ve"):
                getattr(self, name).copy_(torch.from_numpy(d[name]))
