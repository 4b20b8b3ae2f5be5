"""Training and checked rollout of the learned window surrogate (host orchestration).

Every computation runs in librod: the training windows come from the plain GPU step
(``RodSystem.step``), features, targets, the four convolutions, their gradients and Adam run in
the surrogate's kernels (``Surrogate.train_step``), and a rollout is one library call
(``rod_surrogate_rollout``) that checks sampled rods against a shadow system following the
plain method and redoes a segment with the plain step when the sampled tip error exceeds the
bound.  This module only picks batches, learning rates and samples, and gathers statistics of
the unscaled features and targets (means and standard deviations) to set the scales.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

from .binding import RodSystem, Surrogate

POSITIONS = 51
ELEMENTS = 50

# The default recipe: noise level of the training perturbations (x the output scale of each
# group), bound of the sampled tip error in a checked rollout (below the 1e-3 L target, since
# only a sample of the rods is checked)
DEFAULT_NOISE = 0.05
DEFAULT_CHECK_BOUND = 8e-4
DEFAULT_SAMPLE = 16              # rods followed by the shadow systems
# launch shape of the shadows: three 50-element rods per 192-thread block.  A shadow's step is
# latency-bound, and an FP64 warp instruction holds a sub-partition's FP64 unit for 64 cycles
# however many lanes are active: two rods per block (one warp per sub-partition) took 4.86 ms
# for a check of 500 steps, three 5.38 ms (two sub-partitions then hold two warps) on 6 SMs
# instead of 8, five rods 7.85 ms.
SHADOW_SHAPE = (192, 192)
# the global check's single shadow runs the whole horizon with sequential plain steps: two rods
# per block, the shortest step
GLOBAL_SHADOW_SHAPE = (128, 128)
# shadow systems of a locally checked rollout: one check lasts about four segments of the
# network, so four checks are in flight; with three rods per block they take 24 SMs, and the
# network keeps 128, on which its 1024 groups of four windows take four rounds as on 152 (64 x 64
# carpet, 200 calls: 2 rods per block and three shadows 38 ms, 3 rods and four shadows 34 ms,
# five shadows 40 ms -- their 30 SMs cost the network a fifth round)
LOCAL_SHADOWS = 4


def couple_samples(problem, t: float, T: float) -> np.ndarray:
    """(3, R) base couple A sin(2 pi (t + k T / 2) / period + phi) for k = 0, 1, 2 (zero without
    actuation): the three couple features of a window starting at t."""
    R = len(problem.n_elem)
    if problem.act_amp is None:
        return np.zeros((3, R))
    A = np.asarray(problem.act_amp, dtype=np.float64)
    om = 2.0 * np.pi / np.asarray(problem.act_period, dtype=np.float64)
    ph = np.asarray(problem.act_phase, dtype=np.float64)
    return np.stack([A * np.sin(om * (t + 0.5 * k * T) + ph) for k in range(3)])


@dataclasses.dataclass
class Windows:
    """Snapshots of one trajectory of the plain step, ``window`` fine steps apart (device)."""
    problem: object
    states: list          # [(x, v, Q, w)] float64 CUDA tensors, len = n_windows + 1
    acts: list            # [(3, R)] float64 CUDA tensors, couple samples of window k
    window: int
    dt: float
    t0: float = 0.0       # simulated time of states[0]

    @property
    def n_windows(self) -> int:
        return len(self.states) - 1

    @property
    def n_rods(self) -> int:
        return len(self.problem.n_elem)


def generate(problem, n_windows: int, window: int = 50, dt: Optional[float] = None,
             skip_windows: int = 0, smooth: bool = False, sub: int = 5) -> Windows:
    """Run the plain GPU step on ``problem`` from its state and keep the state every ``window``
    steps (after ``skip_windows`` windows).  Every rod must have 50 elements.

    smooth=True keeps instead the window average of the state around every window boundary:
    samples every ``sub`` steps weighted by a triangle of half-width ``window`` steps (the state
    before the start counts as the initial state), directors re-orthonormalised.  This removes
    the oscillations a window of fine steps cannot resolve (the rotary-shear modes of the rods,
    near the window's own period) and keeps the slower bending motion."""
    import torch
    dt = float(problem.dt if dt is None else dt)
    if np.any(np.asarray(problem.n_elem) != ELEMENTS):
        raise ValueError("the surrogate is defined for rods of 50 elements")
    s = RodSystem(problem)
    s.set_state(*problem.state())
    if skip_windows:
        s.step(skip_windows * window, dt)
    T = window * dt
    t0 = s.time
    acts = [torch.tensor(couple_samples(problem, t0 + k * T, T), device="cuda") for k in range(n_windows)]
    if not smooth:
        states = []
        for k in range(n_windows + 1):
            states.append([a.clone() for a in s.get_state(device=True)])
            if k < n_windows:
                s.step(window, dt)
        torch.cuda.synchronize()
        s.close()
        return Windows(problem, states, acts, window, dt, t0)
    if window % sub:
        raise ValueError("window must be a multiple of sub")
    h = window // sub
    wts = {i: (h - abs(i)) / float(h * h) for i in range(-h + 1, h)}     # sums to 1
    first = [a.clone() for a in s.get_state(device=True)]
    acc = {}
    states = [None] * (n_windows + 1)

    def add(k, m, st):
        wt = wts[m - k * h]
        if k not in acc:
            acc[k] = [wt * a for a in st]
        else:
            for a, b in zip(acc[k], st):
                a.add_(b, alpha=wt)

    ortho = Surrogate(window, dt)   # its perturbation kernel at zero noise re-orthonormalises

    def finish(k):
        states[k] = ortho.perturb(acc.pop(k), None, np.ones(ortho.N_OUTPUTS), 0.0)

    # samples m = -h+1 .. 0 are the initial state
    for m in range(-h + 1, 1):
        for k in (0, 1):
            if abs(m - k * h) < h:
                add(k, m, first)
    last = n_windows * h + h - 1
    for m in range(1, last + 1):
        s.step(sub, dt)
        st = s.get_state(device=True)
        for k in (m // h, m // h + 1):
            if 0 <= k <= n_windows and abs(m - k * h) < h:
                add(k, m, st)
        k_done = (m - h + 1) // h
        if (m - h + 1) % h == 0 and 0 <= k_done <= n_windows and k_done in acc:
            finish(k_done)
    for k in sorted(acc):
        finish(k)
    torch.cuda.synchronize()
    s.close()
    return Windows(problem, states, acts, window, dt, t0)


def fit_scales(sur: Surrogate, data: Sequence[Windows], max_windows: int = 64, output_floor: float = 1e-3):
    """Feature shift = mean, scale = 1 / std (over the defined entries), output scale = std of
    the unscaled targets, from up to ``max_windows`` windows of every trajectory."""
    import torch
    fsum = torch.zeros(Surrogate.N_FEATURES, dtype=torch.float64, device="cuda")
    fsq = torch.zeros_like(fsum)
    fcnt = torch.zeros_like(fsum)
    tsq = torch.zeros(Surrogate.N_OUTPUTS, dtype=torch.float64, device="cuda")
    tcnt = 0
    for d in data:
        ks = np.linspace(0, d.n_windows - 1, min(max_windows, d.n_windows)).round().astype(int)
        for k in np.unique(ks):
            F, M = sur.raw_features(d.states[k], d.acts[k])
            Mf = M.to(torch.float64)
            fsum += (F * Mf).sum(dim=(0, 2))
            fsq += (F * F * Mf).sum(dim=(0, 2))
            fcnt += Mf.sum(dim=(0, 2))
            Tg = sur.raw_targets(d.states[k], d.states[k + 1])
            tsq += (Tg * Tg).sum(dim=(0, 2))
            tcnt += Tg.shape[0] * Tg.shape[2]
    mean = (fsum / fcnt.clamp(min=1)).cpu().numpy()
    var = (fsq / fcnt.clamp(min=1)).cpu().numpy() - mean ** 2
    std = np.sqrt(np.maximum(var, 0.0))
    rms = np.sqrt((tsq / max(tcnt, 1)).cpu().numpy())
    shift, scale, out = scales_from_moments(mean, std, rms, output_floor=output_floor)
    sur.set_scales(shift, scale, out)
    return shift, scale, out


FEATURE_GROUPS = [range(0, 3), range(3, 6), range(6, 12), range(12, 15), range(15, 18), range(18, 21), range(21, 24)]
OUTPUT_GROUPS = [range(0, 3), range(3, 6), range(6, 12), range(12, 15)]


def scales_from_moments(mean, std, rms, output_floor: float = 1e-3):
    """Shift = mean per feature; one scale per feature group (position, velocity, directors,
    angular velocity, relative rotation, edge, couple) = 1 / the largest spread in the group, so
    that a channel with little or no spread in the data (for example an out-of-plane component
    of a planar motion) is not blown up: noise there stays at the group's own scale.  Output
    scale = rms per target channel, floored at ``output_floor`` times the largest of its group."""
    mean, std, rms = (np.asarray(a, dtype=np.float64) for a in (mean, std, rms))
    scale = np.ones_like(std)
    for g in FEATURE_GROUPS:
        g = list(g)
        top = float(np.max(std[g]))
        scale[g] = 1.0 / top if top > 0 else 1.0
    out = rms.copy()
    for g in OUTPUT_GROUPS:
        g = list(g)
        top = float(np.max(rms[g]))
        out[g] = np.maximum(rms[g], output_floor * top) if top > 0 else 1.0
    return mean, scale, out


def _layer_shapes():
    return [(64, 32), (64, 64), (64, 64), (16, 64)]


def initial_params(seed: int = 0, last_gain: float = 0.1) -> np.ndarray:
    """He-style initial weights (std sqrt(2 / fan_in), fan_in = 5 C_in), zero biases; the last
    layer is scaled by ``last_gain`` so that the untrained network starts near the prior."""
    rng = np.random.default_rng(seed)
    parts = []
    shapes = _layer_shapes()
    for l, (co, ci) in enumerate(shapes):
        std = math.sqrt(2.0 / (5 * ci)) * (last_gain if l == len(shapes) - 1 else 1.0)
        parts.append(rng.normal(0.0, std, co * 5 * ci))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def train(sur: Surrogate, data: Sequence[Windows], steps: int, lr: float = 1e-3, lr_end: float = 1e-5,
          batch_rods: Optional[int] = None, seed: int = 0, log_every: int = 0, noise: float = 0.0,
          pushforward: float = 0.0, pushforward_start: float = 0.5) -> List[float]:
    """Adam on random windows: each step takes window k of trajectory d (random, every window of
    every trajectory equally likely) for
    ``batch_rods`` consecutive rods (all rods by default).  Cosine decay from lr to lr_end.

    noise > 0: the window start is perturbed by Gaussian noise of ``noise`` times the largest
    output scale of each group (the typical change over one window): positions, velocities,
    angular velocities and a small turn of the directors (clamped entries stay as they are),
    while the target stays the unperturbed window end, so that the network learns to pull a
    perturbed state back to the trajectory (and to damp what it cannot follow).
    pushforward > 0: after a fraction ``pushforward_start`` of the steps, with that probability
    the window start is the network's own prediction from the previous window's start (the
    network then learns to correct its own one-window error).
    Returns the loss of every step."""
    import torch
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    spread = None
    if noise > 0:
        if sur.scales is None:
            raise ValueError("set the scales (fit_scales) before training with noise")
        out = np.asarray(sur.scales[2], dtype=np.float64)
        # one noise level per group (positions, velocities, directors, angular velocities):
        # the largest output scale of the group
        spread = np.concatenate([np.full(len(g), out[list(g)].max()) for g in OUTPUT_GROUPS])
    scratch = {}
    losses = []
    weights = np.array([d.n_windows for d in data], dtype=np.float64)
    weights /= weights.sum()
    for it in range(steps):
        di = int(rng.choice(len(data), p=weights))   # every window equally likely
        d = data[di]
        use_pf = pushforward > 0 and it >= pushforward_start * steps and rng.random() < pushforward
        k = int(rng.integers(1 if use_pf else 0, d.n_windows))
        a, b, act = d.states[k], d.states[k + 1], d.acts[k]
        if use_pf:
            if di not in scratch:
                scratch[di] = RodSystem(d.problem)
                scratch[di].set_state(*[t.cpu().numpy() for t in d.states[0]])
            sysk = scratch[di]
            sysk.set_state(*d.states[k - 1])
            sysk.time = d.t0 + (k - 1) * d.window * d.dt
            sur.apply(sysk, 1)
            a = [t.clone() for t in sysk.get_state(device=True)]
            torch.cuda.synchronize()
        if noise > 0:
            a = _perturb(sur, a, d, spread, noise, gen)
        if batch_rods and batch_rods < d.n_rods:
            r0 = int(rng.integers(0, d.n_rods - batch_rods + 1))
            a = _rod_slice(a, r0, batch_rods)
            b = _rod_slice(b, r0, batch_rods)
            act = act[:, r0:r0 + batch_rods].contiguous()
        f = 0.5 * (1.0 + math.cos(math.pi * it / max(steps - 1, 1)))
        rate = lr_end + (lr - lr_end) * f
        loss = sur.train_step(a, b, act, rate)
        losses.append(loss)
        if log_every and (it % log_every == 0 or it == steps - 1):
            print(f"step {it:6d}  lr {rate:.2e}  loss {loss:.4e}", flush=True)
    for sysk in scratch.values():
        sysk.close()
    torch.cuda.synchronize()
    return losses


def _perturb(sur, state, d, spread, noise, gen):
    """Window start plus noise (rod_surrogate_perturb): positions, velocities and angular
    velocities by noise x the output scale of their channel; directors turned by angles of
    noise x the largest director scale (first-order turn, then Gram-Schmidt); clamped ends kept.
    The standard normal draws come from ``gen``."""
    import torch
    x, v, Q, w = state

    def rnd(a):
        return torch.randn(a.shape, generator=gen, device=a.device, dtype=a.dtype)

    draws = [rnd(x), rnd(v), rnd(w), rnd(w)]
    clamp = getattr(d.problem, "clamp_base", None)
    held = None
    if clamp is not None and np.any(np.asarray(clamp)):
        held = torch.tensor(np.asarray(clamp).astype(np.int8), device=x.device)
    return sur.perturb(state, draws, spread, noise, held)


def train_default(steps: int = 15000, side: int = 32, n_windows: int = 200, seed: int = 101,
                  window: int = 50, dt: float = 1e-5, log_every: int = 0,
                  later_starts=(0.2, 0.4, 0.7, 0.9), later_windows: int = 50):
    """The default surrogate: trained on windows of a carpet of 50-element rods with amplitudes
    0.2..0.8 EI/L, periods 0.5..2 s and random phases -- side^2 x n_windows windows from rest
    (2 x 10^5 by default) and side^2 x later_windows windows from each of the times
    ``later_starts`` (s) of the same run, so that the network sees the beating carpet after the
    start-up as well (none of them covers 0.5..0.6 s); group-shared output scales,
    noise-injected Adam with cosine decay 2e-3 -> 2e-5.  Returns the surrogate and a dict of
    training facts."""
    import time
    import rodgen
    t = time.time()
    p = rodgen.cilia_carpet(side=side, n=ELEMENTS, amp_range=(0.2, 0.8), period_range=(0.5, 2.0), seed=seed)
    data = [generate(p, n_windows=n_windows, window=window, dt=dt)]
    for ts in later_starts:
        data.append(generate(p, n_windows=later_windows, window=window, dt=dt,
                             skip_windows=int(round(ts / (window * dt)))))
    t_data = time.time() - t
    sur = Surrogate(window, dt)
    fit_scales(sur, data, output_floor=1.0)
    sur.set_params(initial_params(seed=0))
    t = time.time()
    losses = train(sur, data, steps=steps, lr=2e-3, lr_end=2e-5, seed=0, noise=DEFAULT_NOISE, log_every=log_every)
    info = {"windows": sum(d.n_windows * d.n_rods for d in data), "train_steps": steps, "data_s": t_data,
            "train_s": time.time() - t, "loss_first": float(losses[0]), "loss_last_200": float(np.mean(losses[-200:]))}
    del data
    return sur, info


def _rod_slice(state, r0: int, n: int):
    x, v, Q, w = state
    ns, ne = slice(r0 * POSITIONS, (r0 + n) * POSITIONS), slice(r0 * ELEMENTS, (r0 + n) * ELEMENTS)
    return [x[:, ns].contiguous(), v[:, ns].contiguous(), Q[:, ne].contiguous(), w[:, ne].contiguous()]


def subset_problem(problem, rods: Sequence[int]):
    """The rods ``rods`` of a problem as a problem of their own (same order)."""
    rods = np.asarray(rods, dtype=np.int64)
    node = np.concatenate([np.arange(r * POSITIONS, (r + 1) * POSITIONS) for r in rods])
    elem = np.concatenate([np.arange(r * ELEMENTS, (r + 1) * ELEMENTS) for r in rods])

    def pick(a, idx):
        return None if a is None else np.ascontiguousarray(np.asarray(a)[..., idx])

    return problem.replace(
        n_elem=np.asarray(problem.n_elem)[rods], rest_len=pick(problem.rest_len, elem),
        radius=pick(problem.radius, rods), youngs=pick(problem.youngs, rods),
        shear_mod=pick(problem.shear_mod, rods), density=pick(problem.density, rods),
        x=pick(problem.x, node), v=pick(problem.v, node), Q=pick(problem.Q, elem), w=pick(problem.w, elem),
        clamp_base=pick(problem.clamp_base, rods), act_amp=pick(problem.act_amp, rods),
        act_period=pick(problem.act_period, rods), act_phase=pick(problem.act_phase, rods),
        tip_force=None if problem.tip_force is None else pick(problem.tip_force, rods),
        rest_kappa=None if problem.rest_kappa is None else _vor_pick(problem.rest_kappa, rods),
        rest_sigma=pick(problem.rest_sigma, elem), elem_couple=pick(problem.elem_couple, elem))


def _vor_pick(a, rods):
    idx = np.concatenate([np.arange(r * (ELEMENTS - 1), (r + 1) * (ELEMENTS - 1)) for r in rods])
    return np.ascontiguousarray(np.asarray(a)[..., idx])


class CheckedRollout:
    """A system advanced by the surrogate with periodic checks of ``n_sample`` sampled rods
    against the plain step.

    mode "global": one shadow system follows the sampled rods with the plain step from the
    initial state (the check measures the accumulated error exactly, at the cost of running
    the plain step for the whole horizon on the side).
    mode "local": ``n_shadows`` shadow systems take turns; each segment's check restarts the
    plain step from the surrogate's own state of the sampled rods at the segment's start, so
    the checks of different segments run while the network goes on (the check measures the
    error the surrogate adds in one segment; ``stats["sum_err"]`` bounds the accumulated
    error if segment errors add up without growing).  ``t0``: the simulated time of the
    problem's state (the actuation phase)."""

    def __init__(self, sur: Surrogate, problem, n_sample: int = DEFAULT_SAMPLE, seed: int = 0,
                 shadow_shape=None, mode: str = "global", n_shadows: int = LOCAL_SHADOWS, t0: float = 0.0):
        if mode not in ("global", "local"):
            raise ValueError("mode is 'global' or 'local'")
        R = len(problem.n_elem)
        rng = np.random.default_rng(seed)
        self.sample = np.sort(rng.choice(R, size=min(n_sample, R), replace=False)).astype(np.int32)
        self.sur = sur
        self.mode = mode
        self.system = RodSystem(problem)
        self.system.set_state(*problem.state())
        self.system.time = t0
        sub = subset_problem(problem, self.sample)
        if shadow_shape is None:
            shadow_shape = GLOBAL_SHADOW_SHAPE if mode == "global" else SHADOW_SHAPE
        self.shadows = []
        for _ in range(1 if mode == "global" else n_shadows):
            sh = RodSystem(sub, use_torch_stream=False)
            sh.set_launch(*shadow_shape)   # few rods per block: the shadow's step is latency-bound
            sh.set_state(*sub.state())
            sh.time = t0
            self.shadows.append(sh)
        self.shadow = self.shadows[0]

    def run(self, n_calls: int, check_every: int = 10, bound: float = DEFAULT_CHECK_BOUND) -> dict:
        """``bound`` is the target for the accumulated sampled tip error; a local check gets its
        share per segment, bound x (the segment's calls) / n_calls (segments have check_every
        calls, fewer toward the end: see rod_surrogate_rollout_local)."""
        if self.mode == "global":
            return self.sur.rollout(self.system, self.shadow, self.sample, n_calls, check_every, bound)
        local = bound * min(1.0, check_every / max(n_calls, 1))
        return self.sur.rollout_local(self.system, self.shadows, self.sample, n_calls, check_every, local)

    def close(self):
        self.system.close()
        for sh in self.shadows:
            sh.close()


def tip_error(problem, xa, xb) -> np.ndarray:
    """Per-rod |x_tip(a) - x_tip(b)| / L for two position arrays (3, N) of rods of 50 elements."""
    tips = np.arange(len(problem.n_elem)) * POSITIONS + ELEMENTS
    L = np.asarray(problem.rest_len).reshape(-1, ELEMENTS).sum(axis=1)
    d = np.asarray(xa)[:, tips] - np.asarray(xb)[:, tips]
    return np.sqrt((d * d).sum(axis=0)) / L


def _main():
    """Time the surrogate on the 64 x 64 carpet: ``python -m paper_2605_13766_gb300.surrogate``
    applies ``--calls`` windows with seeded untrained weights (or trains first with
    ``--train-steps``) and prints the time per call."""
    import argparse
    import json
    import time

    import torch
    import rodgen
    ap = argparse.ArgumentParser()
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--side", type=int, default=64)
    ap.add_argument("--train-steps", type=int, default=0)
    args = ap.parse_args()
    if args.train_steps:
        sur, _ = train_default(steps=args.train_steps)
    else:
        sur = Surrogate(50, 1e-5)
        sur.set_params(initial_params(seed=3))
        rng = np.random.default_rng(0)
        sur.set_scales(rng.normal(0, 0.01, 24), np.exp(rng.normal(0, 1, 24)), np.full(15, 1e-7))
    p = rodgen.cilia_carpet(side=args.side, n=ELEMENTS)
    s = RodSystem(p)
    s.set_state(*p.state())
    sur.apply(s, 1)
    torch.cuda.synchronize()
    t = time.perf_counter()
    sur.apply(s, args.calls)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    print(json.dumps({"rods": p.n_rods, "calls": args.calls, "us_per_call": dt / args.calls * 1e6}))


if __name__ == "__main__":
    _main()
