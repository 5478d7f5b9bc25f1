"""Benchmark of the GB300 relativistic lattice Boltzmann path.

Metric: MLUPS (million lattice-cell updates per second) and the fraction of
the HBM roofline, FP32 vs FP64, forward and adjoint step, on one GB300.

Workload (default): the periodic 512^3 box (eps = 1 + 0.2 phi with phi a
Gaussian random field filtered with sigma = 8 cells, n = eps^(3/4), a
divergence-free beta with max |beta| = 0.3, tau = 0.7; ``workloads.random_box``).
One bench step = one lattice time step (the fused stream-and-collide sweep
over every cell) of the headline variant, FP32 deviation storage; a state
(20.4 GB per FP32 buffer) is far larger than L2, so no flush is needed
between steps.  Legs measured in the same run: FP64 forward, FP32 / FP64
adjoint step (forward recompute + adjoint kernel), the general equation of
state, the 3D shock on a sphere (200 x 100 x 100, forward, adjoint step and a
whole 2000-step gradient), the launch-bound 1D shock tube, the accuracy of
the FP32 path, an end-to-end job through host buffers and the oracle on the
host cores.  MLUPS and bytes count the collided cells (not solid cells, not
ghost planes).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload box512|sphere]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the lattice is not sharded: replicas only); value = all ranks'
cell updates / max over ranks of the timed region.
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

METRIC = "MLUPS and % of HBM roofline, FP32 vs FP64, forward and adjoint step, 1 GB300"
FALLBACK_HBM_GBS = 6800.0
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (vector and tensor), nominal
# FP64 pipe instructions of one update of the all-FP64 step, counted by ncu
# (smsp__inst_executed_pipe_fp64 per 32-cell warp of k_step_f64: 57 moment
# additions, the recovery, the equilibria and BGK), and the FP64 instruction
# rate derived from the nominal FP64 peak (1.25 TFLOP/s = 625 G fused
# multiply-adds per second, one FP64 pipe instruction each).
FP64_OPS_PER_UPDATE = 203
FP64_PEAK_GOPS = FP64_NOMINAL_TFLOPS * 1e3 / 2

# Algorithmic bytes per lattice update (every population read once and written once).
BYTES_FWD = {"fp64": 38 * 8 * 2, "fp32": 38 * 4 * 2}
# Adjoint step: state read (gather), lambda_{t+1} read, lambda_t written.
BYTES_ADJ = {"fp64": 38 * 8 * 3, "fp32": 38 * 4 * 3}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist

    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(ws, device=None):
    if ws > 1:
        import torch.distributed as dist

        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity for one rank)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(cells_per_rank: int, steps: int, ms_max: float, ws: int) -> float:
    """Whole-job MLUPS: every rank's updates over the slowest rank's time."""
    return cells_per_rank * steps * ws / (ms_max * 1e-3) / 1e6


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle sampling in the background (200 ms)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return float("nan")

        sm = np.array([num(r[1]) for r in rows])
        smax = np.array([num(r[2]) for r in rows])
        pw = np.array([num(r[3]) for r in rows])
        load = pw > (np.nanmin(pw) + 0.25 * (np.nanmax(pw) - np.nanmin(pw))) if np.isfinite(pw).any() else sm > 0
        if load.sum() == 0:
            load = np.ones_like(sm, bool)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for k, nm in enumerate(names):
            if any(r[5 + k].lower().startswith("active") for r, l in zip(rows, load) if l):
                reasons.append(nm)
        return {"sm_mhz": float(np.nanmedian(sm[load])), "sm_max_mhz": float(np.nanmax(smax)), "reasons": reasons,
                "samples": int(load.sum()), "power_w_max": float(np.nanmax(pw))}


# ----------------------------------------------------------------------------- timing legs
def _events(torch, stream):
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    return a, b


def time_forward(sim, steps, warmup, ws, device):
    """K lattice steps of the context's own state; returns (ms_total, launches)."""
    import torch

    sim.step(warmup)
    torch.cuda.synchronize()
    barrier(ws, device)
    torch.cuda.synchronize()
    a, b = _events(torch, sim.stream)
    l0 = sim.launches
    a.record(sim.stream)
    sim.step(steps)
    b.record(sim.stream)
    torch.cuda.synchronize()
    barrier(ws, device)
    torch.cuda.synchronize()
    return a.elapsed_time(b), sim.launches - l0


def time_adjoint(sim, steps, warmup):
    """K adjoint steps, each = forward recompute of the state (step_into) plus
    the adjoint kernel, as the sqrt(T) checkpointed backward pass runs them."""
    import torch

    s0 = sim.state()  # read only below
    s1 = sim.new_state()
    l_in = torch.zeros_like(s0)
    l_out = torch.zeros_like(s0)
    l_in[:, :sim.N].normal_()
    acc = torch.zeros(4, dtype=torch.float64, device=sim.device)

    def one():
        sim.step_into(s0, s1)
        sim.adjoint_step(s0, l_in, l_out, acc[0:1], acc[1:4])

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    a, b = _events(torch, sim.stream)
    l0 = sim.launches
    a.record(sim.stream)
    for _ in range(steps):
        one()
    b.record(sim.stream)
    torch.cuda.synchronize()
    ms_all = a.elapsed_time(b)
    launches = sim.launches - l0
    # the adjoint kernel alone (its launch pair)
    a.record(sim.stream)
    for _ in range(steps):
        sim.adjoint_step(s0, l_in, l_out, acc[0:1], acc[1:4])
    b.record(sim.stream)
    torch.cuda.synchronize()
    return ms_all, a.elapsed_time(b), launches


def cpu_baseline(w, budget_s=12.0):
    """The FP64 oracle as it stands, on all host cores, on the full lattice of
    the workload for as many whole steps as fit in about budget_s seconds."""
    import oracle

    p = oracle.Params(**w.params())
    st = oracle.init(p, w.n, w.eps, w.beta, w.solid)
    oracle.run(p, st, 1, solid=w.solid)  # warm-up
    t0 = time.time()
    k = 0
    while True:
        oracle.run(p, st, 1, solid=w.solid)
        k += 1
        if time.time() - t0 > budget_s and k >= 2:
            break
    dt = time.time() - t0
    out = {"value": collided_cells(w) * k / dt / 1e6, "unit": "MLUPS", "cores": oracle.get_threads(), "kind": "oracle",
           "sample": f"{k} FP64 oracle steps of the full {w.nx}x{w.ny}x{w.nz} sphere lattice ({dt:.1f} s)"}
    out["detail"] = oracle_thread_scaling(w)
    return out


def cpu_baseline_slab(w, nz_slab, budget_s=4.0):
    """The oracle on a z slab of a large periodic box (the whole box would need
    two 40 GB host states and minutes per step): whole steps at all host
    cores and at one thread, MLUPS."""
    import oracle

    import workloads as W

    slab = W.Workload(w.name + "_slab", w.nx, w.ny, nz_slab, w.tau, w.c_l, w.xbc, w.steps,
                      np.ascontiguousarray(w.n[:nz_slab]), np.ascontiguousarray(w.eps[:nz_slab]),
                      np.ascontiguousarray(w.beta[:, :nz_slab]))
    p = oracle.Params(**slab.params())
    nthr = oracle.get_threads()
    res = {}
    for label, t in (("threads_all", nthr), ("threads_1", 1)):
        oracle.set_threads(t)
        st = oracle.init(p, slab.n, slab.eps, slab.beta)
        v, k = _oracle_mlups(p, st, None, slab.N, budget_s, 1)
        res[label] = {"mlups": v, "steps": k}
    oracle.set_threads(nthr)
    return {"value": res["threads_all"]["mlups"], "unit": "MLUPS", "cores": nthr, "kind": "oracle",
            "sample": f"whole FP64 oracle steps of a {w.nx}x{w.ny}x{nz_slab} periodic slab of the "
                      f"{w.nx}x{w.ny}x{w.nz} box (about {budget_s:.0f} s per thread count)",
            "detail": res}


def _oracle_mlups(p, st, solid, N, budget_s, min_steps):
    import oracle

    oracle.run(p, st, 1, solid=solid)
    t0 = time.time()
    k = 0
    while True:
        oracle.run(p, st, min_steps, solid=solid)
        k += min_steps
        if time.time() - t0 > budget_s:
            break
    return N * k / (time.time() - t0) / 1e6, k


def oracle_thread_scaling(w, budget_s=2.0):
    """The oracle at one thread and at all host cores on the 1D shock tube
    (1600 cells) and on the given 3D workload, MLUPS (bounded samples)."""
    import oracle

    import workloads as W

    nthr = oracle.get_threads()
    res = {"cores": nthr}
    tube = W.shock_tube_1d()
    for name, wl, ms in (("shock_tube_1600", tube, 50), (f"{w.name}_{w.nx}x{w.ny}x{w.nz}", w, 1)):
        p = oracle.Params(**wl.params())
        for label, t in (("threads_1", 1), ("threads_all", nthr)):
            oracle.set_threads(t)
            st = oracle.init(p, wl.n, wl.eps, wl.beta, wl.solid)
            v, k = _oracle_mlups(p, st, wl.solid, collided_cells(wl), budget_s, ms)
            res.setdefault(name, {})[label] = {"mlups": v, "steps": k}
    oracle.set_threads(nthr)
    return res


def accuracy_leg(w, steps, device):
    """Max relative error of the FP32 deviation path against the FP64 path on
    the benchmark workload after `steps` steps (n and eps relative per cell,
    beta over max(max|beta|, 1e-3); solid cells excluded).  The FP64 GPU path
    is held to the FP64 oracle within 1e-10 by the parity tests."""
    import torch

    from paper_0912_2913_gb300 import RLB

    out = {}
    for prec in ("fp64", "fp32"):
        sim = RLB.from_workload(w, prec, device=device).init_fields(w.n, w.eps, w.beta, w.solid)
        sim.step(steps)
        n, e, b, _ = sim.macro()
        out[prec] = (n, e, b, sim.stats()["n_unphysical"])
        sim.close()
    n0, e0, b0, u0 = out["fp64"]
    n1, e1, b1, u1 = out["fp32"]
    m = torch.isfinite(n0)
    en = float(((n1 - n0).abs() / n0.abs())[m].max())
    ee = float(((e1 - e0).abs() / e0.abs())[m].max())
    bs = max(float(b0[:, m].abs().max()), 1e-3)
    eb = float((b1 - b0)[:, m].abs().max()) / bs
    del out
    torch.cuda.empty_cache()
    return {"reference": "FP64 GPU path (held to the FP64 oracle at 1e-10 by the parity tests)", "steps": steps,
            "fp32_max_rel_err": {"n": en, "eps": ee, "beta": eb}, "unphysical": {"fp64": u0, "fp32": u1}}


def gamma_law_leg(w, steps, device, peak, ms_eps3p, cells):
    """The FP64 step with the general equation of state (an ideal gas with
    rest mass, Gamma = 1.2, m = 0.3: Newton recovery) on the same workload."""
    import torch

    from paper_0912_2913_gb300 import RLB

    sim = RLB.from_workload(w, "fp64", device=device, eos="gamma_law", eos_gamma=1.2, eos_mass=0.3)
    sim.init_fields(w.n, w.eps, w.beta, w.solid)
    ms, _ = time_forward(sim, steps, 3, 1, device)
    st = sim.stats()
    sim.close()
    torch.cuda.empty_cache()
    leg = _leg(cells, ms, steps, BYTES_FWD["fp64"], peak,
               {"eos": "P = (Gamma - 1)(eps - n m), Gamma = 1.2, m = 0.3", "bound": "alu",
                "ratio_to_eps3p_step": (ms / steps) / ms_eps3p, "n_unphysical": st["n_unphysical"]})
    return leg


def f64df_leg(w, steps, device, peak, ms_fp64, cells):
    """The FP64-storage step with its arithmetic in compensated binary32
    pairs (RLB_F64_ARITH=df, the measured ablation of the all-FP64 step)."""
    import torch

    from paper_0912_2913_gb300 import RLB

    os.environ["RLB_F64_ARITH"] = "df"
    try:
        sim = RLB.from_workload(w, "fp64", device=device).init_fields(w.n, w.eps, w.beta, w.solid)
    finally:
        os.environ.pop("RLB_F64_ARITH", None)
    ms, _ = time_forward(sim, steps, 3, 1, device)
    sim.close()
    torch.cuda.empty_cache()
    return _leg(cells, ms, steps, BYTES_FWD["fp64"], peak,
                {"arithmetic": "compensated binary32 pairs, binary64 storage and recovery root",
                 "ratio_to_fp64_step": (ms / steps) / ms_fp64})


def shock_tube_graph_leg(device, steps_per_graph=100, replays=20):
    """The launch-bound 1D shock tube (1600 cells, FP64): microseconds per step
    with one rlb_step call per 1000 steps, and with steps_per_graph steps
    captured once in a CUDA graph and replayed."""
    import torch

    import workloads as W
    from paper_0912_2913_gb300 import RLB

    w = W.shock_tube_1d()
    s = torch.cuda.Stream(device=device)
    sim = RLB.from_workload(w, "fp64", device=device, stream=s).init_fields(w.n, w.eps, w.beta)
    sim.step(10)
    torch.cuda.synchronize()
    a, b = _events(torch, s)
    a.record(s)
    sim.step(1000)
    b.record(s)
    torch.cuda.synchronize()
    us_plain = a.elapsed_time(b) * 1e3 / 1000
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sim.step(steps_per_graph)
    with torch.cuda.stream(s):  # replay() launches on the current stream
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        a.record(s)
        for _ in range(replays):
            g.replay()
        b.record(s)
    torch.cuda.synchronize()
    us_graph = a.elapsed_time(b) * 1e3 / (replays * steps_per_graph)
    sim.close()
    return {"workload": "shock tube 1600x1x1 FP64, outflow ghosts at both ends", "us_per_step_stream": us_plain,
            "us_per_step_graph": us_graph, "steps_per_graph": steps_per_graph,
            "mlups_graph": collided_cells(w) / us_graph}


def gradient_run_leg(w, T, device, ms_forward, budget_cap=200e9, reserve=40e9):
    """One whole gradient evaluation through rlb_run (FP32, T steps, loss =
    sum of P^2 = (eps/3)^2 over the plane x = 120, gradients for tau,
    beta_in and the initial fields): forward and backward pass times, with
    plain sqrt(T) checkpointing (K = 45) and with the last states of the run
    kept within a device-memory budget (min(budget_cap, free - reserve)) so
    fewer steps are recomputed.  ratio_to_forward = backward ms per step over
    the forward step of the headline leg."""
    import torch

    from paper_0912_2913_gb300 import RunSpec, rlb_run

    torch.cuda.empty_cache()
    budget = max(0.0, min(budget_cap, torch.cuda.mem_get_info(device)[0] - reserve))
    out = {"steps": T, "loss": "sum over the plane x = 120 of (eps/3)^2",
           "warmup": "one untimed 20-step gradient run of each kind first"}
    for name, K, b, TT in (("warmup", 5, None, 20), ("warmup", None, 1e30, 20), ("sqrt_t", 45, None, T),
                           ("stored_tail", None, budget, T)):
        spec = RunSpec.from_workload(w, "fp32", steps=TT, checkpoint_every=K, store_budget_bytes=b, device=device)
        f64 = dict(dtype=torch.float64, device=device)
        tau = torch.tensor(w.tau, **f64, requires_grad=True)
        bi = torch.tensor(w.beta_in, **f64, requires_grad=True)
        n0, e0, b0 = (torch.from_numpy(np.ascontiguousarray(a)).to(device).requires_grad_(True)
                      for a in (w.n, w.eps, w.beta))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record()
        try:
            n, e, bb = rlb_run(tau, bi, n0, e0, b0, spec)
        except ValueError as err:  # the budget does not hold even the plain checkpointed run
            out[name] = {"skipped": str(err)}
            continue
        ev[1].record()
        L = (e[:, :, 120] / 3.0).square().sum()
        ev[2].record()
        L.backward()
        ev[3].record()
        torch.cuda.synchronize()
        fwd, bwd = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
        plan = spec.last_plan
        if name == "warmup":
            spec.last_sim.close()
            continue
        out[name] = {"forward_ms": fwd, "backward_ms": bwd, "backward_ms_per_step": bwd / T,
                     "ratio_to_forward": (bwd / T) / ms_forward, "states_held": plan.states_held,
                     "state_gb": plan.states_held * spec.last_sim.state_bytes / 1e9, "stored_tail": plan.P,
                     "checkpoint_every": plan.K, "recomputed_steps": plan.recomputed_steps,
                     "grad_finite": bool(torch.isfinite(tau.grad) and torch.isfinite(bi.grad).all()
                                         and torch.isfinite(e0.grad).all())}
        spec.last_sim.close()
        del n, e, bb, L, tau, bi, n0, e0, b0, spec
        torch.cuda.empty_cache()
    return out


def e2e_run(w, job_steps, jobs, device, cells):
    """End to end through the public API: host fields -> rlb_init_fields
    (H2D) -> job_steps steps -> rlb_macro to host (D2H), FP32."""
    import torch

    from paper_0912_2913_gb300 import RLB

    sim = RLB.from_workload(w, "fp32", device=device)
    hn = torch.from_numpy(np.ascontiguousarray(w.n)).pin_memory().numpy()
    he = torch.from_numpy(np.ascontiguousarray(w.eps)).pin_memory().numpy()
    hb = torch.from_numpy(np.ascontiguousarray(w.beta)).pin_memory().numpy()
    hs = None if w.solid is None else torch.from_numpy(np.ascontiguousarray(w.solid)).pin_memory().numpy()
    sim.init_fields(hn, he, hb, hs).step(20)
    sim.macro(where="host")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(jobs):
        sim.init_fields(hn, he, hb, hs)
        sim.step(job_steps)
        out = sim.macro(where="host")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    sim.close()
    bi = hn.nbytes + he.nbytes + hb.nbytes + (0 if hs is None else hs.nbytes)
    bo = out[0].nbytes + out[1].nbytes + out[2].nbytes
    return {"value": cells * job_steps * jobs / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": bi / job_steps,
            "d2h_bytes_per_step": bo / job_steps,
            "job": f"{jobs} x (host fields -> init -> {job_steps} FP32 steps -> macro to host)"}


def traffic_from_profiles(kernel: str, digest: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current inputs of the kernel's translation unit."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(f"{kernel}/{workload}")
        if e and e.get("build") == digest:
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def collided_cells(w) -> int:
    """Cells a step collides: every cell but the solid ones and the x ghost
    planes of a non-periodic lattice."""
    n = w.N
    if w.solid is not None:
        n -= int(np.count_nonzero(w.solid))
    if w.xbc != 0:
        ghost = np.ones((w.nz, w.ny, 2), bool)
        if w.solid is not None:
            ghost &= w.solid[:, :, [0, -1]] == 0
        n -= int(ghost.sum())
    return n


def kernel_frac(w, ms, bytes_per_update, peak, cells=None):
    """Fraction of the HBM peak of one kernel launch over the lattice that
    moves bytes_per_update per collided cell in ms milliseconds."""
    cells = w.N if cells is None else cells
    return bytes_per_update * cells / (ms * 1e-3) / 1e9 / peak


def _leg(cells, ms_total, steps, bytes_per_update, peak, extra=None):
    ms = ms_total / steps
    gbs = bytes_per_update * cells / (ms * 1e-3) / 1e9
    d = {"mlups": cells / (ms * 1e-3) / 1e6, "ms_per_step": ms, "bytes_per_update": bytes_per_update,
         "achieved_gbs": gbs, "frac_hbm": gbs / peak}
    if extra:
        d.update(extra)
    return d


BOX_DESC = ("random_box 512^3 periodic, eps = 1 + 0.2 phi (Gaussian random field, sigma 8, max|phi| = 1), "
            "n = eps^(3/4), div-free beta, max|beta| = 0.3, tau = 0.7")
SPHERE_DESC = ("sphere_3d 200x100x100, inflow plane x = 0 at beta_x = 0.5, eps = n = 1; interior at rest with "
               "n = 0.3 and eps = 1 (the literal eps = 0.1 leaves the scheme's domain within 30 steps); solid "
               "sphere r = 15 at (60,50,50); outflow copy at x = 199; tau = 0.8")


def make_workload(name):
    """The named workload with its own step count (box 1000, sphere 5000)."""
    import workloads as W

    if name == "box512":
        return W.random_box(L=512), BOX_DESC
    return W.sphere_3d(), SPHERE_DESC


def time_noalloc(sim, steps):
    """ms per call of rlb_adjoint_step_noalloc (the persistent register
    kernel + finalize) on the context's state, after one set-up call."""
    import torch

    from paper_0912_2913_gb300 import _native as Nat

    s0 = sim.state()
    l_in = torch.zeros_like(s0)
    l_out = torch.zeros_like(s0)
    acc = torch.zeros(4, dtype=torch.float64, device=sim.device)
    Nat.rlb_adjoint_step_noalloc(sim.ctx, s0, l_in, l_out, acc[0:1], acc[1:4])
    torch.cuda.synchronize()
    a, b = _events(torch, sim.stream)
    a.record(sim.stream)
    for _ in range(steps):
        Nat.rlb_adjoint_step_noalloc(sim.ctx, s0, l_in, l_out, acc[0:1], acc[1:4])
    b.record(sim.stream)
    torch.cuda.synchronize()
    del l_in, l_out
    return a.elapsed_time(b) / steps


def precision_legs(w, prec, steps, peak, device, ms_fwd=None, adjoint=True):
    """Forward leg (unless ms_fwd is given) and adjoint-step leg of one
    precision on workload w; the adjoint step = forward recompute + adjoint
    kernel, as the sqrt(T) backward pass runs them."""
    import torch

    from paper_0912_2913_gb300 import RLB

    cells = collided_cells(w)
    legs = {}
    sim = RLB.from_workload(w, prec, device=device).init_fields(w.n, w.eps, w.beta, w.solid)
    if ms_fwd is None:
        ms, _ = time_forward(sim, steps, 3, 1, device)
        ms_fwd = ms / steps
        extra = None
        if prec == "fp64":
            extra = {"bound": "alu", "fp64_ops_per_update": FP64_OPS_PER_UPDATE,
                     "fp64_peak_gops": FP64_PEAK_GOPS, "fp64_peak": "nominal 1.25 TFLOP/s = 625 G FMA/s",
                     "fp64_alu_frac": FP64_OPS_PER_UPDATE * cells / (ms_fwd * 1e-3) / (FP64_PEAK_GOPS * 1e9)}
        legs[f"{prec}_forward"] = _leg(cells, ms, steps, BYTES_FWD[prec], peak, extra)
    else:
        sim.step(3)
    if adjoint:
        ka = max(1, steps // 2)
        ms_all, ms_k, _ = time_adjoint(sim, ka, 3)
        ms_na = time_noalloc(sim, ka)
        legs[f"{prec}_adjoint"] = _leg(cells, ms_all, ka, BYTES_ADJ[prec] + BYTES_FWD[prec], peak,
                                       {"adjoint_kernel_ms": ms_k / ka,
                                        "adjoint_kernel_frac_hbm": kernel_frac(w, ms_k / ka, BYTES_ADJ[prec], peak,
                                                                               cells),
                                        "noalloc_adjoint_ms": ms_na,
                                        "ratio_to_forward": (ms_all / ka) / ms_fwd})
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return legs


def slab_leg(w, steps, peak, device, ms_whole, nslabs=4):
    """The z-slab decomposition on one GPU: the workload cut into nslabs z
    slabs (one context each, two halo planes), every step = the slab steps
    + rlb_halo_exchange between neighbours.  MLUPS over the whole lattice's
    collided cells; the exchange's own time from a run of exchanges alone."""
    import torch

    from paper_0912_2913_gb300 import _native as Nat
    from paper_0912_2913_gb300.slabs import SlabLattice

    lat = SlabLattice.from_workload(w, "fp32", nslabs=nslabs, device=device)
    lat.init_fields(w.n, w.eps, w.beta, w.solid).step(3)
    torch.cuda.synchronize()
    st = lat.slabs[0].stream
    a, b = _events(torch, st)
    a.record(st)
    lat.step(steps)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    a.record(st)
    for _ in range(steps):
        lat.exchange()
    b.record(st)
    torch.cuda.synchronize()
    ms_x = a.elapsed_time(b) / steps
    lat.close()
    del lat
    torch.cuda.empty_cache()
    cells = collided_cells(w)
    return _leg(cells, ms, steps, BYTES_FWD["fp32"], peak,
                {"slabs": nslabs, "exchange_ms_per_step": ms_x, "ratio_to_whole_lattice_step": (ms / steps) / ms_whole,
                 "halo_bytes_per_step": 2 * 10 * w.nx * w.ny * 4 * nslabs})


def sphere_legs(steps, grad_steps, peak, device, adjoint=True):
    """The 3D shock on a sphere as a leg of the box benchmark: FP32 forward,
    FP32 adjoint step and a whole FP32 gradient run."""
    import torch

    from paper_0912_2913_gb300 import RLB

    w, desc = make_workload("sphere")
    cells = collided_cells(w)
    sim = RLB.from_workload(w, "fp32", device=device).init_fields(w.n, w.eps, w.beta, w.solid)
    ms, _ = time_forward(sim, steps, 20, 1, device)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    out = {"workload": desc, "cells": w.N, "collided_cells": cells,
           "fp32_forward": _leg(cells, ms, steps, BYTES_FWD["fp32"], peak)}
    if adjoint:
        out.update(precision_legs(w, "fp32", max(1, steps // 2), peak, device, ms_fwd=ms / steps))
        if grad_steps > 0:
            out["fp32_gradient_run"] = gradient_run_leg(w, grad_steps, device, ms / steps)
    return out


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    init_dist(ws, "nccl")
    from paper_0912_2913_gb300 import RLB
    from paper_0912_2913_gb300 import build as B

    w, wdesc = make_workload(args.workload)
    cells = collided_cells(w)
    peak, peak_kind = measured_peaks()
    legs = {}
    with ClockSampler(local) as clk:
        # headline leg: FP32 deviation storage, forward
        sim = RLB.from_workload(w, "fp32", device=device).init_fields(w.n, w.eps, w.beta, w.solid)
        ms, launches = time_forward(sim, args.steps, args.warmup, ws, device)
        ms_max = max_over_ranks(ms, ws, device)
        value = aggregate(cells, args.steps, ms_max, ws)
        stats32 = sim.stats()
        legs["fp32_forward"] = _leg(cells, ms, args.steps, BYTES_FWD["fp32"], peak)
        achieved = legs["fp32_forward"]["achieved_gbs"] * args.steps / max(launches, 1)
        sim.close()
        del sim
        torch.cuda.empty_cache()
        if not args.headline_only:
            k_side = max(1, args.steps // (10 if args.workload == "box512" else 4))
            if not args.no_adjoint:
                legs.update(precision_legs(w, "fp32", k_side * 2, peak, device, ms_fwd=ms / args.steps))
            legs.update(precision_legs(w, "fp64", k_side, peak, device, adjoint=not args.no_adjoint))
            legs["fp64_gamma_law_forward"] = gamma_law_leg(w, k_side, device, peak,
                                                           legs["fp64_forward"]["ms_per_step"], cells)
            legs["fp32_z_slabs"] = slab_leg(w, k_side * 2, peak, device, ms / args.steps)
            legs["fp64_df_arith_forward"] = f64df_leg(w, k_side, device, peak, legs["fp64_forward"]["ms_per_step"],
                                                      cells)
            if args.workload == "sphere":
                if not args.no_adjoint and args.grad_steps > 0:
                    legs["fp32_gradient_run"] = gradient_run_leg(w, args.grad_steps, device, ms / args.steps)
            else:
                legs["sphere"] = sphere_legs(1000, args.grad_steps, peak, device, adjoint=not args.no_adjoint)
            legs["shock_tube_fp64"] = shock_tube_graph_leg(device)
    clocks = clk.summary()
    accuracy = accuracy_leg(w, min(w.steps, 1000), device) if (rank == 0 and not args.headline_only) else None
    e2e = None
    if rank == 0 and not args.no_e2e:
        e2e = e2e_run(w, args.e2e_steps or w.steps, 1, device, cells)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_budget) if args.workload == "sphere" else cpu_baseline_slab(w, 32)
    if rank == 0:
        kern = "k_step_f32"
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wdesc + "; FP32 deviation storage, FP64 recovery root", "cells": w.N,
                       "collided_cells": cells,
                       "l2": "state larger than L2 (no flush needed)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic_from_profiles(kern, B.unit_digest("rlb_forward.cu"), args.workload),
                         "kernel": kern,
                         "bytes_per_launch": BYTES_FWD["fp32"] * cells},
            "legs": legs,
            "clocks": clocks,
            "e2e": e2e,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "stats_fp32": stats32,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_reference(args):
    """The FP64 CPU oracle (the reference arm) on the benchmark workload: each
    step is one oracle step of a bounded sample of it (a 10-plane z slab
    through the middle of the lattice: the sphere's centre plane for the
    sphere)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads as W

    w, wdesc = make_workload(args.workload)
    nz = 10
    z0 = w.nz // 2 - nz // 2
    sl = lambda a: None if a is None else np.ascontiguousarray(a[..., z0:z0 + nz, :, :])
    sub = W.Workload(w.name + "_slab", w.nx, w.ny, nz, w.tau, w.c_l, w.xbc, args.steps, sl(w.n), sl(w.eps),
                     sl(w.beta), sl(w.solid), w.n_in, w.eps_in, w.beta_in)
    p = oracle.Params(**sub.params())
    st = oracle.init(p, sub.n, sub.eps, sub.beta, sub.solid)
    oracle.run(p, st, args.warmup, solid=sub.solid)
    t0 = time.time()
    oracle.run(p, st, args.steps, solid=sub.solid)
    dt = time.time() - t0
    v = collided_cells(sub) * args.steps / dt / 1e6
    sample = f"{args.steps} FP64 oracle steps of a {w.nx}x{w.ny}x{nz} z slab (z = {z0}..{z0 + nz - 1}) of the lattice"
    line = {"metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wdesc, "cells": w.N, "sample_cells": sub.N},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Short runs of the benchmark workload for ncu captures: --profile step
    runs warm-up + --steps forward steps; --profile adjoint runs --steps
    (forward recompute + adjoint) steps; --profile box / adjoint_box run
    forward / adjoint steps on the periodic random box of side --box;
    --profile tube runs FP64 steps of the 1600-cell shock tube."""
    import torch

    import workloads as W
    from paper_0912_2913_gb300 import RLB

    on_box = args.profile in ("box", "adjoint_box")
    if args.profile == "tube":
        w = W.shock_tube_1d(steps=args.steps)
        args.precision = "fp64"
    else:
        w = W.random_box(L=args.box, steps=args.steps) if on_box else W.sphere_3d(steps=args.steps)
        if on_box:
            w.c_l = args.c_l
    sim = RLB.from_workload(w, args.precision, device="cuda:0").init_fields(w.n, w.eps, w.beta, w.solid)
    if args.profile in ("step", "box", "tube"):
        sim.step(args.steps)
    else:
        sim.step(5)
        time_adjoint(sim, args.steps, 1)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "precision": args.precision, "steps": args.steps,
                      "stats": sim.stats()}), flush=True)
    sim.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end job (0: the workload's own step count)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--grad-steps", type=int, default=2000,
                    help="steps of the whole-gradient leg (rlb_run forward + backward); 0 skips it")
    ap.add_argument("--workload", choices=["box512", "sphere"], default="box512")
    ap.add_argument("--profile", choices=["step", "adjoint", "box", "adjoint_box", "tube"], default=None,
                    help="short run of one kernel family for ncu captures (no JSON bench line)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--box", type=int, default=256)
    ap.add_argument("--c-l", dest="c_l", type=float, default=1.0, help="lattice speed of the --profile box runs")
    args = ap.parse_args(argv)
    if args.profile:
        run_profile(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
