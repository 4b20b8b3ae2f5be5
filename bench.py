#!/usr/bin/env python3
"""Benchmark: FP64 element-steps/s of the Cosserat-rod step on GB300.

Default workload: the 10^4-rod random packing (element counts U{16..256}, seeded; rod-rod
contact through the uniform cell list; gravity; dt = 5e-6 s).  One bench "step" is one time
step of the whole ensemble (contact broad + narrow phase, strains, curvatures, internal and
external loads, Verlet update with the exponential-map director update).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload packing|carpet|cantilever]
                  [--impl ours|reference]

Multi-GPU: replicas only (no data-path collective): every rank advances its own independent
ensemble; value = all ranks' element-steps / max-over-ranks time (weak scaling).
--impl reference times the plain CPU oracle (test infrastructure) on a bounded sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import rodgen  # noqa: E402

METRIC = "element-steps/sec FP64 on 1 GB300 (% HBM roofline); surrogate speedup at <=1e-3 err"
UNIT = "element-steps/s"

# FP64 peak of the part: 2 FP64 FMA per clock per SM (an FMA-throughput probe measured 1.91 per
# clock at 2.07 GHz) x 152 SMs x 2.07 GHz max SM clock x 2 flop per FMA.
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12

# FP64 flops per unit of each kernel as the kernel evaluates them, counted by ncu on the active
# threads (add/sub/mul = 1 flop, fma = 2) and divided by the units of the launch.  pack_one_step:
# one launch of pack_kernel_plain<3> on the 10^4-rod packing near step 1000, 124.40M DFMA +
# 22.41M DADD + 91.46M DMUL on 1,366,295 element-steps.  pack_steps: one 20-step launch of
# pack_kernel<0> on the 64 x 64 carpet, 370.54M DFMA + 70.36M DADD + 284.39M DMUL on 4,096,000
# element-steps.
FLOPS_PER_UNIT = {
    "pack_one_step": 265.4,   # per element-step
    "pack_steps": 267.5,      # per element-step
}
# FP64-pipe instructions per unit (thread level, ncu smsp__sass_thread_inst_executed_op_fp64):
# a DMUL or DADD takes the FP64 unit as long as a DFMA, so the pipe is bound by instructions,
# not flops; peak 2 per clock per SM x 152 SMs x 2.07 GHz.
FP64_INSTR_PER_UNIT = {
    "pack_one_step": 176.40,
    "pack_steps": 179.15,
}
FP64_INSTR_PEAK = 2 * 152 * 2.07e9
FLOPS_SOURCE = "executed FP64 arithmetic of the kernel (ncu: DFMA x 2 + DADD + DMUL) per element-step"
# The method's FP64 work per element-step as the oracle states it: every addition, subtraction,
# multiplication and division of one step of the oracle's source evaluated over counting numbers
# (oracle/count_flops.py, general bent and spinning states of the packing's and the carpet's
# recipes); special-function calls (sqrt, sin, cos, atan2, floor) are counted apart.  The kernel
# executes fewer operations than the oracle states (reciprocals of constants stored once,
# rotation maps by series, products fused), so the roofline fraction uses the executed count,
# which never credits the kernel with work it does not do.
ORACLE_FLOPS_PER_UNIT = {
    "pack_one_step": 588.76,   # the step without contact (the step kernel's share)
    "pack_steps": 588.34,      # the carpet's step
}
ORACLE_SPECIAL_PER_UNIT = {
    "pack_one_step": 8.99,
    "pack_steps": 8.94,
}
# the oracle's contact evaluation (cell list, exact closest points of every candidate) on the
# packing's placement density, per element-step, on top of the step
ORACLE_CONTACT_FLOPS_PER_UNIT = 511.02
# Algorithmic HBM bytes per element-step: the state makes one round trip (6 node + 12 element
# doubles, read and written: 288 B), the rest length is read (8 B), and with contact each
# segment's cell key and sorted index are written and read (16 B).
BYTES_PER_UNIT = {"packing": 312.0, "carpet": 296.0, "cantilever": 296.0}


def _measured_bf16_tflops():
    """(dense BF16 TFLOP/s, where it comes from): the measured sustained cuBLAS figure when the pod's
    MEASURED_PEAKS.json is present, else an earlier measurement on a GB300 (1.7 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
    except Exception:
        return 1700.0, "1.7 PFLOP/s sustained, an earlier GB300 measurement (of fallback)"


def _measured_hbm_gbs():
    """(HBM copy bandwidth in GB/s, where it comes from): the measured figure when the pod's
    MEASURED_PEAKS.json is present, else an earlier measurement on a GB300 (6.8 TB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except Exception:
        return 6800.0, "6.8 TB/s, an earlier GB300 copy measurement (of fallback)"


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of one capture of the
# current kernel; reset to None whenever the kernel changes.  pack_one_step: launches of the
# packing's steps near step 1000 at the 256 x 256 shape (the force entries read only for
# segments with skin-list candidates).
# The carpet's state stays on chip between the steps of a launch: its traffic is one read of
# the state and constants per launch (the written state is still in L2 when the launch ends).
# CPU seconds the reference arm spends on its W + K samples (the whole run stays within minutes)
REF_BUDGET_S = 90.0
TRAFFIC_PER_LAUNCH = {
    "pack_one_step": 275.60e6 + 143.95e6,
    "pack_steps": 37.78e6,
}


def _workload(name: str, rank: int):
    seed = 1234
    if name == "packing":
        p = rodgen.random_packing_cached(seed=seed)
        desc = {"workload": "random packing, 10^4 rods, n~U{16..256} (seeded), contact k=1e4 c=10, gravity, dt=5e-6",
                "rods": p.n_rods, "elements": p.n_elems, "dt": 5e-6,
                "note": "timed steps sit inside the workload's 5000-step run, after an untimed pre-roll from "
                        "the placement to a contact-dense state (timed_window); the first steps after the "
                        "placement, which has no overlap, are reported as early_window"}
        return p, 5e-6, desc
    if name == "carpet":
        p = rodgen.cilia_carpet()
        return p, 1e-5, {"workload": "cilia carpet 64x64 rods x 50 elements, base couple, Stokes drag, dt=1e-5",
                         "rods": p.n_rods, "elements": p.n_elems, "dt": 1e-5}
    if name == "cantilever":
        p = rodgen.cantilever()
        return p, 1e-5, {"workload": "one clamped rod, 100 elements, tip force, damping, dt=1e-5",
                         "rods": 1, "elements": 100, "dt": 1e-5}
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _reference(args, world, rank):
    """CPU oracle as the reference arm, its OpenMP build on all host cores: W untimed and
    exactly K timed steps, each step a bounded sample of the same workload -- s time steps of
    its first m rods, sized during the warm-up so that all W + K samples take about
    REF_BUDGET_S seconds."""
    if rank != 0:
        return
    from oracle.oracle import build_oracle_omp, omp_threads, using_library
    omp = build_oracle_omp()
    cores = omp_threads(omp)
    with using_library(omp):
        _reference_run(args, world, omp, cores)


def _reference_run(args, world, omp, cores):
    from oracle.oracle import Oracle
    p, dt, desc = _workload(args.workload, 0)
    K, W = max(1, args.steps), max(args.warmup, 3)
    target = min(0.5, REF_BUDGET_S / (K + W))          # seconds per sample
    # calibration (the first warm-up sample): one time step of enough rods for ~2e4 elements
    eo = p.elem_offsets()
    m = int(min(p.n_rods, max(1, np.searchsorted(eo, 20000))))
    q = p.take_rods(0, m)
    o = Oracle(q)
    st = q.state()
    t0 = time.perf_counter()
    st = o.step(*st, dt=dt, n_steps=1)
    per_elem_step = (time.perf_counter() - t0) / q.n_elems
    # the sample: s steps of the first m rods
    if per_elem_step * p.n_elems <= target:
        m, s = p.n_rods, max(1, int(target / (per_elem_step * p.n_elems)))
    else:
        m, s = int(min(p.n_rods, max(1, np.searchsorted(eo, target / per_elem_step)))), 1
    q = p.take_rods(0, m)
    o = Oracle(q)
    st = q.state()
    for _ in range(W - 1):
        st = o.step(*st, dt=dt, n_steps=s)
    times = []
    for _ in range(K):
        t0 = time.perf_counter()
        st = o.step(*st, dt=dt, n_steps=s)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = q.n_elems * s * K / tot
    sample = (f"each step: {s} time step(s) of the first {m} of {p.n_rods} rods ({q.n_elems} of {p.n_elems} "
              f"elements) of the {desc['workload']}, the oracle's OpenMP build on {cores} host threads "
              f"(contact search serial)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": tot / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": dict(desc, l2="state larger than L2 (196 MB)" if args.workload == "packing" else "n/a"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _cpu_baseline(p, dt, desc, workload):
    """The oracle timed on the host cores on a bounded sample of the workload: its OpenMP build
    on every core (the per-rod right-hand side and the per-item updates in parallel, the contact
    search serial) and the plain build on one thread."""
    from oracle.oracle import Oracle, build_oracle, build_oracle_omp, omp_threads, using_library
    build_oracle()
    omp = build_oracle_omp()
    n = {"packing": 3, "carpet": 20, "cantilever": 2000}[workload]
    st = p.state()
    with using_library(omp):
        o = Oracle(p)
        t0 = time.perf_counter()
        o.step(*st, dt=dt, n_steps=n)
        el_all = time.perf_counter() - t0
    o = Oracle(p)
    t0 = time.perf_counter()
    o.step(*st, dt=dt, n_steps=n)
    el_one = time.perf_counter() - t0
    cores = omp_threads(omp)
    return {"value": p.n_elems * n / el_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} time steps of the full workload ({p.n_elems} elements), the oracle's OpenMP build on "
                      f"{cores} host threads (contact search serial)",
            "single_thread": {"value": p.n_elems * n / el_one, "unit": UNIT, "cores": 1,
                              "sample": f"the same {n} steps, plain oracle, one thread"}}


def _e2e(s, start_state, p, dt, K, world, dist, barrier):
    """Same metric through the public API from pinned host buffers: set_state (H2D) of the timed
    window's start state, K steps, get_state (D2H) inside the timed region."""
    import torch
    from paper_2605_13766_gb300.replicas import slowest, total
    x, v, Q, w = start_state
    pin = [torch.from_numpy(a).pin_memory() for a in (x, v, Q, w)]
    outs = [torch.empty(a.shape, dtype=torch.float64).pin_memory() for a in (x, v, Q, w)]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_state(*[a.numpy() for a in pin])
    s.step(K, dt)
    xs = s.get_state(out=[o.numpy() for o in outs])
    t_e2e = slowest(time.perf_counter() - t0)
    state_bytes = 8 * (6 * p.n_nodes + 12 * p.n_elems)
    e2e = {"value": total(p.n_elems * K) / t_e2e, "unit": UNIT, "h2d_bytes_per_step": state_bytes / K,
           "d2h_bytes_per_step": state_bytes / K,
           "note": f"set_state of the timed window's start state from pinned host + {K} steps + get_state to "
                   f"host per round trip (host wall clock; set_state rebuilds the contact grid and list)"}
    del outs, xs

    return e2e


def _adjoint_timing():
    """Gradient of a tip-target loss with respect to the rest curvature and the element couples
    over the adjoint workload (1024 rods x 64 elements, 2000 steps of 1e-5 s, checkpoint every
    100 steps): the checkpointed forward run and the reverse sweep (recompute of each segment and
    the hand-written adjoint kernels), each timed with CUDA events on the system's stream."""
    import torch
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300.autograd import tip_indices
    p = rodgen.adjoint_batch()
    n_steps, dt, every = 2000, 1e-5, 100
    s = RodSystem(p)
    k0 = torch.tensor(p.rest_kappa, device="cuda")
    c0 = torch.tensor(p.elem_couple, device="cuda")
    state0 = [torch.tensor(a, device="cuda") for a in p.state()]
    tips = tip_indices(p.node_offsets())
    targets = torch.tensor(p.extra["targets"], device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    times = []
    for rep in range(2):                      # the first pair warms up
        s.set_params(k0, c0)
        s.set_state(*state0)
        torch.cuda.synchronize()
        ev[0].record(s.torch_stream)
        s.forward_checkpointed(n_steps, dt, every)
        ev[1].record(s.torch_stream)
        x = s.get_state(device=True)[0]
        gx = torch.zeros_like(x)
        gx[:, tips] = 2.0 * (x[:, tips] - targets)
        z = torch.zeros
        s.torch_stream.wait_stream(torch.cuda.current_stream())
        e2 = torch.cuda.Event(enable_timing=True)
        e2.record(s.torch_stream)
        gk, gc = s.backward(gx, z((3, s.n_nodes), dtype=torch.float64, device="cuda"),
                            z((9, s.n_elems), dtype=torch.float64, device="cuda"),
                            z((3, s.n_elems), dtype=torch.float64, device="cuda"))
        ev[2].record(s.torch_stream)
        torch.cuda.synchronize()
        times.append((ev[0].elapsed_time(ev[1]) / 1e3, e2.elapsed_time(ev[2]) / 1e3))
    s.close()
    t_fwd, t_bwd = times[-1]
    units = p.n_elems * n_steps
    return {"workload": "1024 rods x 64 elements, 2000 steps of 1e-5 s, checkpoint every 100, tip-target loss",
            "forward_elem_steps_per_s": units / t_fwd, "backward_elem_steps_per_s": units / t_bwd,
            "gradient_elem_steps_per_s": units / (t_fwd + t_bwd), "forward_s": t_fwd, "backward_s": t_bwd,
            "grad_norm": {"rest_kappa": float(gk.norm()), "elem_couple": float(gc.norm())},
            "check": "gradients checked against Richardson-extrapolated central differences in the GPU tests"}


def _surrogate_speedup(train_steps: int):
    """Surrogate speed-up at the tip-error bound: the 64 x 64 carpet of 50-element rods from rest
    over 10^4 fine steps of 1e-5 s (200 calls of 50 steps), plain GPU step vs the checked
    rollout (sampled rods against a shadow system every 10 calls, plain-step redo above the
    bound); the network is first trained by the library's kernels (default recipe)."""
    import time

    import torch
    import rodgen
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300 import surrogate as S
    sur, info = S.train_default(steps=train_steps)
    p = rodgen.cilia_carpet(side=64, n=50)
    dt, W, n_calls = 1e-5, 50, 200
    s = RodSystem(p)
    s.set_state(*p.state())
    ref = {}
    for k in range(1, 11):
        s.step(20 * W, dt)
        ref[20 * k] = s.get_state()[0]
    s.set_state(*p.state())
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.torch_stream)
    s.step_async(n_calls * W, dt)
    e1.record(s.torch_stream)
    s.sync()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    s.close()
    net = RodSystem(p)
    net.set_state(*p.state())
    worst = 0.0
    t_net = 0.0
    for k in range(1, 11):
        n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0.record(net.torch_stream)
        sur.apply(net, 20)
        n1.record(net.torch_stream)
        torch.cuda.synchronize()
        t_net += n0.elapsed_time(n1) / 1e3
        worst = max(worst, float(S.tip_error(p, net.get_state()[0], ref[20 * k]).max()))
    net.close()
    # the network alone: 200 calls of the fused tcgen05 kernel, CUDA events around each 20;
    # executed BF16 work per call: 256 tile rows per four windows, 32 input and 16 output channels
    us_call = t_net / n_calls * 1e6
    flop_call = p.n_rods / 4 * 256 * 2 * 5 * (32 * 64 + 64 * 64 + 64 * 64 + 64 * 16)
    bf16_peak = _measured_bf16_tflops()
    el = p.n_elems * n_calls * W
    modes = {}
    for mode in ("local", "global"):
        warm = S.CheckedRollout(sur, p, seed=1, mode=mode)
        warm.run(2, check_every=1, bound=1.0)
        warm.close()
        ro = S.CheckedRollout(sur, p, seed=1, mode=mode)
        torch.cuda.synchronize()
        t = time.perf_counter()
        stats = ro.run(n_calls, check_every=10, bound=S.DEFAULT_CHECK_BOUND)
        torch.cuda.synchronize()
        t_sur = time.perf_counter() - t
        final = float(S.tip_error(p, ro.system.get_state()[0], ref[n_calls]).max())
        ro.close()
        modes[mode] = {"speedup": t_plain / t_sur, "surrogate_elem_steps_per_s": el / t_sur,
                       "final_tip_err": final, "rollout": stats}
    # out of the training window: t in [0.5, 0.6] s of the same carpet (training saw the first
    # 0.1 s of 32 x 32 carpets from rest), and a carpet whose amplitude and period both lie
    # outside the training ranges (0.2..0.8 EI/L, 0.5..2 s)
    later = _pre_rolled(p, dt, 50_000)
    beyond = rodgen.cilia_carpet(side=64, n=50, amp_factor=1.0, period=0.3)
    out = {"t_0.5_to_0.6_s": _rollout_case(sur, later, dt, W, n_calls, t0=0.5),
           "amp_1.0_EI_over_L_period_0.3_s": _rollout_case(sur, beyond, dt, W, n_calls)}
    head = modes["local"]
    return {"workload": "cilia carpet 64x64 rods x 50 elements, 10^4 steps of 1e-5 s (200 calls of 50 steps)",
            "out_of_window": out,
            "speedup": head["speedup"], "check": "local (pipelined per-segment checks); global below",
            "plain_elem_steps_per_s": el / t_plain, "surrogate_elem_steps_per_s": head["surrogate_elem_steps_per_s"],
            "max_tip_err_network_every_20_calls": worst, "final_tip_err_checked_rollout": head["final_tip_err"],
            "err_unit": "|x_tip - x_tip(plain)| / L, max over all rods", "bound": 1e-3,
            "check_bound_sampled": S.DEFAULT_CHECK_BOUND, "modes": modes,
            "timing": "plain: CUDA events on its stream; rollout: host wall clock around the whole checked rollout",
            "training": info, "dtype": "bf16 tensor cores (tcgen05, accumulators in tensor memory), FP32 accumulation, FP64 state",
            "network": {"us_per_call": us_call, "tensor_tflops_executed": flop_call / (us_call * 1e-6) / 1e12,
                        "bf16_peak_tflops": bf16_peak[0], "bf16_frac": flop_call / (us_call * 1e-6) / 1e12 / bf16_peak[0],
                        "peak_source": bf16_peak[1],
                        "note": "fused inference kernel alone (features, four convolutions, FP64 update) per call "
                                "of 50 fine steps on the 4096 rods, CUDA events; the FP64 features and update, "
                                "not the tensor cores, bound it"}}


def _pre_rolled(p, dt, n_steps):
    """The problem with its state advanced n_steps plain GPU steps from rest."""
    from paper_2605_13766_gb300 import RodSystem
    s = RodSystem(p)
    s.set_state(*p.state())
    s.step(n_steps, dt)
    x, v, Q, w = s.get_state()
    s.close()
    return p.replace(x=x, v=v, Q=Q, w=w)


def _rollout_case(sur, p, dt, W, n_calls, t0=0.0):
    """Checked rollout (local checks) of n_calls windows from the problem's state at time t0
    against the plain GPU step over the same interval: speed-up, tip errors, fallbacks."""
    import time

    import torch
    from paper_2605_13766_gb300 import RodSystem
    from paper_2605_13766_gb300 import surrogate as S
    s = RodSystem(p)
    s.set_state(*p.state())
    s.time = t0
    s.step(n_calls * W, dt)
    ref = s.get_state()[0]
    s.set_state(*p.state())
    s.time = t0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.torch_stream)
    s.step_async(n_calls * W, dt)
    e1.record(s.torch_stream)
    s.sync()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    s.close()
    ro = S.CheckedRollout(sur, p, seed=1, mode="local", t0=t0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    stats = ro.run(n_calls, check_every=10, bound=S.DEFAULT_CHECK_BOUND)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t
    err = S.tip_error(p, ro.system.get_state()[0], ref)
    ro.close()
    return {"t0": t0, "speedup": t_plain / t_sur, "final_tip_err": float(err.max()),
            "fallback_calls": int(stats["fallback_calls"]), "surrogate_calls": int(stats["surrogate_calls"]),
            "rollout": stats}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="packing", choices=["packing", "carpet", "cantilever"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch-shape", default=None,
                    help="elements,threads per block for the step kernels (skips the autotuner)")
    ap.add_argument("--skin", type=float, default=None,
                    help="contact skin list (m); default 0.5 mm for the packing, 0 = cell search every step")
    ap.add_argument("--surrogate-train-steps", type=int, default=15000)
    ap.add_argument("--preroll", type=int, default=None,
                    help="contact workloads: untimed steps of the same run before the timed window (default: "
                         "4000, less what keeps the timed and profiled steps inside the run's 5000); the early "
                         "window from the placement is reported beside it")
    ap.add_argument("--no-full-run", action="store_true",
                    help="skip the timing of the whole 5000-step contact run from the placement")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        _reference(args, world, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2605_13766_gb300 import RodSystem, build
    from paper_2605_13766_gb300.replicas import slowest, total
    build.build()
    p, dt, desc = _workload(args.workload, rank)
    s = RodSystem(p)
    skin = args.skin if args.skin is not None else (5e-4 if args.workload == "packing" else 0.0)
    if p.contact:
        s.contact_skin(skin)
    s.set_state(*p.state())
    W = max(args.warmup, 3)
    K = args.steps
    # launch shape (elements and threads per block) picked by the library's autotuner on the
    # live state, which it restores afterwards
    tuned = None
    if args.launch_shape:
        te, tt = (int(v) for v in args.launch_shape.split(","))
        s.set_launch(te, tt)
        tuned = {"elems_per_block": te, "threads_per_block": tt, "trial_ms_per_step": None}
    elif not args.no_autotune:
        te, tt, tms = s.autotune(dt, trial_steps=5)
        tuned = {"elems_per_block": te, "threads_per_block": tt, "trial_ms_per_step": tms}
    stream = s.torch_stream

    def timed(n):
        """n steps in one call, CUDA events on the library's stream; (seconds, launches, rebuilds)."""
        launches0 = s.launch_count
        builds0 = s.contact_list_builds()
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s.step_async(n, dt)
        ev1.record(stream)
        s.sync()
        torch.cuda.synchronize()
        barrier()
        return ev0.elapsed_time(ev1) / 1e3, s.launch_count - launches0, s.contact_list_builds() - builds0

    def pairs_now():
        """Segment pairs in contact at the current state (the cell-grid search; the skin list is
        rebuilt at the next step)."""
        return s.contact_pair_count()[0] if p.contact else None

    # ---- early window: W warm-up steps from the placement, then K timed steps (no contact yet
    # on the packing: it starts without overlap)
    early = None
    run_steps = 5000
    if not p.contact:
        preroll = 0
    elif args.preroll is not None:
        preroll = args.preroll
    else:
        preroll = max(W + K, min(4000, run_steps - (W + 2 * K + 1)))
    if preroll > 0:
        s.step(W, dt)
        t_e, l_e, b_e = timed(K)
        early = {"steps": f"{W + 1}..{W + K}", "value": total(p.n_elems * K) / slowest(t_e),
                 "ms_per_step": slowest(t_e) * 1e3 / K, "gpu_launches": l_e, "rebuilds": b_e,
                 "contact_pairs_at_end": pairs_now()}
        # ---- untimed pre-roll of the same run to a contact-dense state
        done = W + K
        while done < preroll:
            n = min(500, preroll - done)
            s.step(n, dt)
            done += n
    else:
        done = 0
    # the window's start state, kept on the host for the end-to-end measurement
    start_state = s.get_state()
    pairs0 = pairs_now()
    s.step(W, dt)
    torch.cuda.synchronize()
    diag0 = s.diagnostics(per_rod=False)[1]   # energy parts and orthonormality before the timed steps

    # ---- timed region (device time, CUDA events on the stream the library launches on)
    clocks = ClockSampler(local)
    clocks.start()
    t_local, launches, builds = timed(K)
    clk = clocks.stop()
    t_max = slowest(t_local)
    value = total(p.n_elems * K) / t_max
    pairs1 = pairs_now()
    window = {"first_timed_step": done + W + 1, "last_timed_step": done + W + K,
              "contact_pairs_at_start": pairs0, "contact_pairs_at_end": pairs1,
              "rebuilds_in_timed_steps": builds}
    diag1 = s.diagnostics(per_rod=False)[1]
    diag = {"energy_before": float(diag0[:5].sum()), "energy_after": float(diag1[:5].sum()),
            "energy_parts_after": [float(e) for e in diag1[:5]],
            "max_orthonormality_error_after": float(diag1[5]),
            "note": "energy of the timed steps' first and last states: kinetic, strain, work potential of "
                    "gravity and tip forces (the contact springs' stored energy is not in the sum and "
                    "moves energy into or out of it; damping, drag and the dashpot dissipate); parts: "
                    "translational, rotational, shear/stretch, bend/twist, potential"}

    # ---- per-kernel device times: the next K steps with CUDA events around every launch
    # (eager launches: the event pairs sit between kernels on the same stream)
    s.step(1, dt)   # takes the rebuild that the pair count above requested
    builds_p0 = s.contact_list_builds()
    s.profile(True)
    s.step_async(K, dt)
    s.sync()
    prof = s.profile_read()
    s.profile(False)
    builds_p = s.contact_list_builds() - builds_p0
    if p.contact and skin > 0:
        rebuild_ms = sum(prof.get(k, (0.0, 0))[0] for k in
                         ("contact_bin", "contact_scan", "contact_scatter", "contact_sort", "contact_list_build"))
        window["rebuild"] = {
            "rebuilds_in_profiled_steps": builds_p,
            "rebuild_kernels_ms_per_step": rebuild_ms / K,
            "ms_per_rebuild": (rebuild_ms / builds_p) if builds_p else None,
            "steps_per_rebuild": (K / builds_p) if builds_p else None,
            "note": "eager profiled steps launch the gated rebuild kernels every step (they return at once "
                    "when no rebuild is due); their time over K steps is the amortised rebuild cost"}

    # ---- end to end through the public API with pinned host buffers (from the window's start)
    e2e = None
    if not args.no_e2e:
        e2e = _e2e(s, start_state, p, dt, K, world, dist, barrier)

    # ---- the whole contact run from the placement (the workload's 5000 steps in one call,
    # graph-replayed), timed with CUDA events like the window
    full = None
    if p.contact and not args.no_full_run:
        s.set_state(*p.state())
        t_f, l_f, b_f = timed(run_steps)
        full = {"steps": run_steps, "value": total(p.n_elems * run_steps) / slowest(t_f),
                "ms_per_step": slowest(t_f) * 1e3 / run_steps, "gpu_launches": l_f, "rebuilds": b_f,
                "contact_pairs_at_end": pairs_now()}

    # ---- roofline of the dominant kernel
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dname, (dms, dn) = dom
    avg_ms = dms / max(dn, 1)
    fpu = FLOPS_PER_UNIT.get(dname)
    units = p.n_elems * (K if dname == "pack_steps" else 1)
    achieved = (fpu * units / (avg_ms * 1e-3) / 1e12) if fpu else None
    hbm_peak, hbm_src = _measured_hbm_gbs()
    bpu = BYTES_PER_UNIT.get(args.workload)
    hbm = None
    if bpu:
        k_gbs = bpu * units / (avg_ms * 1e-3) / 1e9
        step_gbs = bpu * value / 1e9
        hbm = {"bytes_per_unit": bpu, "peak_gbs": hbm_peak, "peak_source": hbm_src,
               "kernel_gbs": k_gbs, "kernel_frac": k_gbs / hbm_peak,
               "step_gbs": step_gbs, "step_frac": step_gbs / hbm_peak,
               "note": "algorithmic bytes (one HBM round trip of the state plus rest lengths and, with contact, "
                       "the cell key and sorted index) x units / time"}
    roof = {"bound": "alu", "kernel": dname, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
            "traffic": TRAFFIC_PER_LAUNCH.get(dname), "avg_launch_ms": avg_ms,
            "flops_per_unit": fpu, "flops_source": FLOPS_SOURCE,
            "flops_per_unit_oracle": ORACLE_FLOPS_PER_UNIT.get(dname),
            "special_calls_per_unit_oracle": ORACLE_SPECIAL_PER_UNIT.get(dname),
            "frac_uses": "flops_per_unit (executed by the kernel); flops_per_unit_oracle is the oracle's "
                         "statement of the same step, counted on its source",
            "peak_source": "FP64: 2 FMA/clk/SM x 152 SMs x 2.07 GHz (nominal unit count; an FMA probe measured 1.91/clk)",
            "hbm_frac": hbm["step_frac"] if hbm else None, "hbm": hbm,
            "fp64_pipe": ({"instr_per_unit": FP64_INSTR_PER_UNIT[dname],
                           "achieved_instr_per_s": FP64_INSTR_PER_UNIT[dname] * units / (avg_ms * 1e-3),
                           "peak_instr_per_s": FP64_INSTR_PEAK,
                           "frac": FP64_INSTR_PER_UNIT[dname] * units / (avg_ms * 1e-3) / FP64_INSTR_PEAK,
                           "note": "FP64-pipe instruction rate against 2 per clock per SM (DMUL and DADD cost "
                                   "a DFMA's slot, so the flop fraction understates the pipe's load)"}
                          if dname in FP64_INSTR_PER_UNIT else None),
            "kernel_share": {k: round(v[0] / max(sum(x[0] for x in prof.values()), 1e-12), 4)
                             for k, v in prof.items() if v[1]}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(p, dt, desc, args.workload)
    sur = None
    if rank == 0 and world == 1 and not args.no_surrogate:
        sur = _surrogate_speedup(args.surrogate_train_steps)
    adj = None
    if rank == 0 and world == 1 and not args.no_adjoint:
        adj = _adjoint_timing()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": t_max * 1e3 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic (seeded)",
                "config": dict(desc, parallelism=f"replicas x{world}" if world > 1 else "1 GPU", launch_shape=tuned,
                               contact_search=("none" if not p.contact else
                                               f"skin list, skin {skin:g} m, {builds} rebuilds in the timed steps"
                                               if skin > 0 else "cell grid searched every step"),
                               l2="state (196 MB) larger than L2, no flush needed" if args.workload == "packing"
                               else "state L2/smem resident",
                               timed_window=window),
                "clocks": clk, "gpu_launches": launches, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
                "early_window": early, "full_run": full, "surrogate": sur, "adjoint": adj, "diagnostics": diag}
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
