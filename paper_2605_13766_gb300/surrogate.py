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

    @property
    def n_windows(self) -> int:
        return len(self.states) - 1

    @property
    def n_rods(self) -> int:
        return len(self.problem.n_elem)


def generate(problem, n_windows: int, window: int = 50, dt: Optional[float] = None,
             skip_windows: int = 0) -> Windows:
    """Run the plain GPU step on ``problem`` from its state and keep the state every ``window``
    steps (after ``skip_windows`` windows).  Every rod must have 50 elements."""
    import torch
    dt = float(problem.dt if dt is None else dt)
    if np.any(np.asarray(problem.n_elem) != ELEMENTS):
        raise ValueError("the surrogate is defined for rods of 50 elements")
    s = RodSystem(problem)
    s.set_state(*problem.state())
    if skip_windows:
        s.step(skip_windows * window, dt)
    states, acts = [], []
    T = window * dt
    for k in range(n_windows + 1):
        st = [a.clone() for a in s.get_state(device=True)]
        states.append(st)
        if k < n_windows:
            acts.append(torch.tensor(couple_samples(problem, s.time, T), device="cuda"))
            s.step(window, dt)
    torch.cuda.synchronize()
    s.close()
    return Windows(problem, states, acts, window, dt)


def fit_scales(sur: Surrogate, data: Sequence[Windows], max_windows: int = 64):
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
    shift, scale, out = scales_from_moments(mean, std, rms)
    sur.set_scales(shift, scale, out)
    return shift, scale, out


FEATURE_GROUPS = [range(0, 3), range(3, 6), range(6, 12), range(12, 15), range(15, 18), range(18, 21), range(21, 24)]
OUTPUT_GROUPS = [range(0, 3), range(3, 6), range(6, 12), range(12, 15)]


def scales_from_moments(mean, std, rms, feature_floor: float = 1e-6, output_floor: float = 1e-3):
    """Shift = mean and scale = 1 / std per feature, output scale = rms per target channel, with
    every spread floored at a fraction of the largest one of its group (position, velocity,
    directors, ... ): a channel that only carries rounding noise (for example the out-of-plane
    components of a planar motion) is then not blown up to order one."""
    mean, std, rms = (np.asarray(a, dtype=np.float64) for a in (mean, std, rms))
    std = std.copy()
    for g in FEATURE_GROUPS:
        g = list(g)
        top = float(np.max(std[g] + np.abs(mean[g])))
        std[g] = np.maximum(std[g], feature_floor * top) if top > 0 else 1.0
    out = rms.copy()
    for g in OUTPUT_GROUPS:
        g = list(g)
        top = float(np.max(rms[g]))
        out[g] = np.maximum(rms[g], output_floor * top) if top > 0 else 1.0
    return mean, 1.0 / std, out


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
          batch_rods: Optional[int] = None, seed: int = 0, log_every: int = 0) -> List[float]:
    """Adam on random windows: each step takes window k of trajectory d (random) for
    ``batch_rods`` consecutive rods (all rods by default).  Cosine decay from lr to lr_end.
    Returns the loss of every step."""
    import torch
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        d = data[rng.integers(len(data))]
        k = int(rng.integers(d.n_windows))
        a, b, act = d.states[k], d.states[k + 1], d.acts[k]
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
    torch.cuda.synchronize()
    return losses


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
    """A system advanced by the surrogate, checked every ``check_every`` calls on ``n_sample``
    sampled rods that a shadow system follows with the plain step."""

    def __init__(self, sur: Surrogate, problem, n_sample: int = 64, seed: int = 0):
        R = len(problem.n_elem)
        rng = np.random.default_rng(seed)
        self.sample = np.sort(rng.choice(R, size=min(n_sample, R), replace=False)).astype(np.int32)
        self.sur = sur
        self.system = RodSystem(problem)
        self.system.set_state(*problem.state())
        sub = subset_problem(problem, self.sample)
        self.shadow = RodSystem(sub, use_torch_stream=False)
        self.shadow.set_state(*sub.state())

    def run(self, n_calls: int, check_every: int = 10, bound: float = 5e-4) -> dict:
        return self.sur.rollout(self.system, self.shadow, self.sample, n_calls, check_every, bound)

    def close(self):
        self.system.close()
        self.shadow.close()


def tip_error(problem, xa, xb) -> np.ndarray:
    """Per-rod |x_tip(a) - x_tip(b)| / L for two position arrays (3, N) of rods of 50 elements."""
    tips = np.arange(len(problem.n_elem)) * POSITIONS + ELEMENTS
    L = np.asarray(problem.rest_len).reshape(-1, ELEMENTS).sum(axis=1)
    d = np.asarray(xa)[:, tips] - np.asarray(xb)[:, tips]
    return np.sqrt((d * d).sum(axis=0)) / L
