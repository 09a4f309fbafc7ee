#!/usr/bin/env python3
"""Benchmark of the grid-side Hartree step on GB300 (one JSON line on stdout).

Workload: the 8x8x8 diamond supercell (4,096 Gaussian charges, sigma = 0.5 Bohr,
a = 53.92 Bohr) on a 512^3 FP32 grid.  One step is the whole per-iteration hot
path: density splat over the bisection-ordered atoms, the five-pass Poisson
solve with the fused Green multiply and E_H reduction, and the adjoint force
gather.  The atom reorder (modified recursive bisection) runs once per
geometry before timing and is reported as reorder_ms.

value: HBM yardstick bytes per step (40 N_tot, the five read+write sweeps of
the Poisson solve) x steps / time, summed over ranks ("GB/s", higher is
better).  ms_per_step, solve_ms and the per-kernel breakdown sit beside it.

--impl reference times the FP64 CPU oracle (the paper's method written out
plainly, the library's parity reference) on the host cores, on a bounded 256^3
sample of the same system.
Multi-GPU: one replica per GPU (the single grid does not shard without an
all-to-all; replicas run independent workloads), launched with torchrun.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Hartree solve ms & HBM GB/s at 512^3 fp32; batched/adjoint vs plain solve"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="diamond512",
                    choices=["diamond512", "diamond256", "ortho360", "paper420", "paper420cube", "paper840"],
                    help="diamond256: the 4x4x4 cell on 256^3 (same density and sigma), for small profiler captures; "
                         "ortho360: the 37.9 x 40.4 x 42.1 Bohr cell on 360 x 384 x 400 (diamond density); "
                         "paper420: 16,384 diamond atoms on the 420 x 420 x 210 grid of the paper's benchmarks; "
                         "paper420cube / paper840: 32,768 / 65,536 atoms on 420^3 / 840 x 420 x 420")
    ap.add_argument("--skip-side", action="store_true", help="skip the e2e, adjoint and batched measurements")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16split"],
                    help="bf16split: b passes on the tensor cores (N2 = 256: the diamond256 workload)")
    ap.add_argument("--tc-parts", default="fp16", choices=["fp16", "bf16"],
                    help="operand format of the tensor-core split: FP16 hi/lo pairs or BF16 in three parts")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle timing
def oracle_sample(threads):
    """One oracle step (splat, Poisson, E_H, forces) on the 256^3 diamond sample; seconds."""
    import oracle as O
    from paper_1209_4506_gb300 import synth

    O.set_threads(threads)
    S = synth.config5()  # 4x4x4 diamond cell, 512 atoms, sigma 0.5, 256^3: the 512^3 system's density and width
    t0 = time.perf_counter()
    rho = O.splat(S.n, S.cell, S.sigma, S.pos, S.q, 5.0)
    vh, eh, _, _ = O.poisson(S.cell, rho)
    O.forces(S.n, S.cell, S.sigma, S.pos, S.q, vh, 5.0)
    return time.perf_counter() - t0, S


SAMPLE_TEXT = ("oracle step (splat 5 sigma, FP64 Poisson, E_H, forces) on the 4x4x4 diamond cell, 512 atoms, "
               "256^3 grid (same density and sigma as the 512^3 workload); GB/s on its own 40 N_tot yardstick")


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (x itself on one rank): the job's time is its slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ybytes, steps, seconds, world):
    """Whole-job GB/s: every rank runs its own replica of the workload (weak scaling)."""
    return world * ybytes * steps / seconds / 1e9


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = len(os.sched_getaffinity(0))
    for _ in range(args.warmup):
        oracle_sample(threads)
    times = []
    for _ in range(args.steps):
        t, S = oracle_sample(threads)
        times.append(t)
    total = sum(times)
    ybytes = 40.0 * S.n_tot
    value = ybytes * args.steps / total / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "diamond 4x4x4 supercell, 512 Gaussian charges, 256^3 grid (bounded sample of the "
                               "512^3 diamond workload)", "grid": list(S.n), "atoms": S.n_atoms},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": SAMPLE_TEXT},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def kernel_traffic(name):
    """ncu DRAM bytes per launch for `name`, if the capture matches the current source."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        ent = d[name]
        src = os.path.join(ROOT, ent["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        return float(ent["bytes"]) if h == ent["sha256"] else None
    except Exception:
        return None


def time_events(fn, reps, stream, warm=3):
    """Average device milliseconds of fn() over reps calls (CUDA events on `stream`)."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def graph_of(fn, stream):
    """Capture fn() (after one eager call on a side stream) into a CUDA graph."""
    import torch

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        fn()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


def batched_section(dev, stream, reps):
    """64 uneven FP32 cells: one persistent launch vs 64 plan solves, both replayed from CUDA graphs."""
    import numpy as np
    import torch

    from paper_1209_4506_gb300 import synth
    from paper_1209_4506_gb300.hartree import HartreeBatch, HartreePlan

    cells = synth.config4()
    pts = sum(int(np.prod(S.n)) for S in cells)
    B = HartreeBatch([(S.n, S.cell, S.sigma, S.n_atoms) for S in cells])
    pos = torch.tensor(np.concatenate([S.pos for S in cells]).reshape(-1, 3), device=dev)
    q = torch.tensor(np.concatenate([S.q for S in cells]), device=dev)
    vh = torch.empty(int(B.grid_off[-1]), dtype=torch.float32, device=dev)
    eh = torch.empty(len(cells), dtype=torch.float64, device=dev)
    gB = graph_of(lambda: B.solve(pos, q, vh, eh), stream)
    t_b = time_events(gB.replay, reps, stream)
    B.device_status()
    eh_b = eh.clone()
    plans, args = [], []
    for S in cells:
        P = HartreePlan(S.n, S.cell, S.sigma, "fp32", max_atoms=max(S.n_atoms, 1))
        plans.append(P)
        args.append((torch.tensor(S.pos, device=dev), torch.tensor(S.q, device=dev),
                     torch.empty(S.n, dtype=torch.float32, device=dev), torch.empty((), dtype=torch.float64, device=dev)))

    def plain():
        for P, (p_, q_, v_, e_) in zip(plans, args):
            P.solve(p_, q_, vh=v_, eh=e_)

    t_p_eager = time_events(plain, max(3, reps // 4), stream)
    gP = graph_of(plain, stream)
    t_p = time_events(gP.replay, reps, stream)
    eh_p = torch.stack([a[3] for a in args])
    max_rel = float(((eh_b - eh_p).abs() / eh_p.abs()).max().item())
    y = 40.0 * pts
    out = {"cells": len(cells), "grid_points": pts, "atoms": int(B.atom_off[-1]), "launches_per_solve": 1,
           "batched_ms": t_b, "batched_gbs": y / (t_b * 1e-3) / 1e9,
           "plain_ms": t_p, "plain_gbs": y / (t_p * 1e-3) / 1e9, "plain_eager_ms": t_p_eager,
           "speedup_vs_plain_graph": t_p / t_b, "eh_max_rel_diff_vs_plain": max_rel,
           "form": "CUDA graph replay of hartree_solve_batched vs of 64 hartree_solve calls (splat + 5 passes + E_H)"}
    for P in plans:
        P.close()
    B.close()
    return out


def adjoint_section(plan, pos, q, rho, vh, stream, reps, plain_solve_ms):
    """Forward + backward through the autograd wrappers at the bench's grid, beside the plain solve."""
    import torch

    from paper_1209_4506_gb300.autograd import hartree_energy, hartree_energy_atoms

    pos_g = pos.clone().requires_grad_(True)
    q_g = q.clone().requires_grad_(True)

    def atoms(store):
        def f():
            pos_g.grad = None
            q_g.grad = None
            e = hartree_energy_atoms(pos_g, q_g, plan, store_potential=store)
            e.backward()
        return f

    plan.splat(pos, q, rho)
    rho_g = rho.clone().requires_grad_(True)

    def dens():
        rho_g.grad = None
        hartree_energy(rho_g, plan).backward()

    t_rec = time_events(atoms(False), reps, stream)
    t_sto = time_events(atoms(True), reps, stream)
    t_den = time_events(dens, reps, stream)
    return {"atoms_recompute_ms": t_rec, "atoms_stored_potential_ms": t_sto, "density_ms": t_den,
            "plain_solve_ms": plain_solve_ms,
            "form": "torch.autograd forward + backward: E_H(pos, q) -> (-F, phi), recomputing V_H in the backward "
                    "(or keeping it); E_H(rho) -> V_H dV (backward = one more solve)"}


def other_grids_section(dev, stream, reps):
    """The grids that are not powers of two: 360 x 384 x 400 (orthorhombic cell at diamond density) and the
    paper's memory-benchmark grids at 0.257 Bohr: 420 x 420 x 210, 420^3 and 840 x 420 x 420 (16,384, 32,768 and
    65,536 diamond atoms).  Per grid: the autotuned solve (five passes and the E_H
    reduction, CUDA events) with its fraction of the measured HBM peak on the 40 N_tot yardstick, and the whole
    step (setup, splat, solve, forces) over the bisection-ordered atoms."""
    import torch

    from paper_1209_4506_gb300 import synth
    from paper_1209_4506_gb300.hartree import HartreePlan, atoms_reorder

    pk, _ = peaks()
    out = {}
    for key, S in (("ortho360", synth.config3b()), ("paper420", synth.config_paper420()),
                   ("paper420cube", synth.config_paper420cube()), ("paper840", synth.config_paper840())):
        apl = 16
        perm, _ = atoms_reorder(S.pos, (S.n_atoms + apl - 1) // apl)
        plan = HartreePlan(S.n, S.cell, S.sigma, "fp32", atoms_per_leaf=apl, max_atoms=S.n_atoms)
        variants = plan.autotune()
        pos = torch.tensor(S.pos[perm], device=dev)
        q = torch.tensor(S.q[perm], device=dev)
        rho = plan.splat(pos, q)
        vh = torch.empty_like(rho)
        eh = torch.empty((), dtype=torch.float64, device=dev)
        f = torch.empty((S.n_atoms, 3), dtype=torch.float64, device=dev)
        t_solve = time_events(lambda: plan.solve_density(rho, vh, eh), reps, stream)
        t_step = time_events(lambda: plan.step(pos, q, vh=vh, eh=eh, f=f), reps, stream)
        plan.device_status()
        y = 40.0 * S.n_tot
        out[key] = {"grid": list(S.n), "atoms": S.n_atoms, "solve_ms": t_solve,
                    "solve_gbs": y / (t_solve * 1e-3) / 1e9,
                    "solve_frac": y / (t_solve * 1e-3) / 1e9 / pk["hbm_gbs"],
                    "step_ms": t_step, "variants": variants,
                    "note": "solve = five passes + E_H reduction; frac of the measured HBM peak, 40 N_tot bytes"}
        plan.close()
    return out


def side_sections(args, plan, pos_h, q_h, pos, q, rho, vh, stream, world, barrier, ybytes, plain_solve_ms, dev):
    """e2e through the C ABI with host buffers, the adjoint forms and the batched form."""
    import torch

    # end to end: pinned host buffers in, host results out, copies and read-back inside the timed region
    pos_pin = torch.tensor(pos_h).pin_memory()
    q_pin = torch.tensor(q_h).pin_memory()
    eh_pin = torch.empty(1, dtype=torch.float64).pin_memory().numpy()
    f_pin = torch.empty((len(q_h), 3), dtype=torch.float64).pin_memory().numpy()
    for _ in range(3):
        plan.step_host(pos_pin.numpy(), q_pin.numpy(), eh_out=eh_pin, f_out=f_pin)
    n_e2e = max(10, min(args.steps, 100))
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        plan.step_host(pos_pin.numpy(), q_pin.numpy(), eh_out=eh_pin, f_out=f_pin)
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = {"value": job_throughput(ybytes, n_e2e, t_e2e, world), "unit": "GB/s",
           "h2d_bytes_per_step": int(pos_h.nbytes + q_h.nbytes), "d2h_bytes_per_step": int(8 + pos_h.nbytes),
           "ms_per_step": 1e3 * t_e2e / n_e2e, "api": "hartree_step_host"}
    side_reps = max(5, min(args.steps, 50))
    adjoint = adjoint_section(plan, pos, q, rho, vh, stream, side_reps, plain_solve_ms)
    batched = batched_section(dev, stream, side_reps)
    other = other_grids_section(dev, stream, side_reps)
    return e2e, adjoint, batched, other


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1209_4506_gb300 import synth
    from paper_1209_4506_gb300.hartree import HartreePlan, atoms_reorder

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    if args.workload == "diamond512":
        S = synth.config3a()
        wl_text = "diamond 8x8x8 supercell, 4096 Gaussian charges (sigma 0.5 Bohr, cutoff 5 sigma), 512^3 grid"
    elif args.workload == "paper420":
        S = synth.config_paper420()
        wl_text = ("diamond 16x16x8 supercell, 16384 Gaussian charges (sigma 0.8 Bohr, cutoff 5 sigma), "
                   "420 x 420 x 210 grid (h = 0.257 Bohr)")
    elif args.workload == "paper420cube":
        S = synth.config_paper420cube()
        wl_text = ("diamond 16x16x16 supercell, 32768 Gaussian charges (sigma 0.8 Bohr, cutoff 5 sigma), "
                   "420^3 grid (h = 0.257 Bohr)")
    elif args.workload == "paper840":
        S = synth.config_paper840()
        wl_text = ("diamond 32x16x16 supercell, 65536 Gaussian charges (sigma 0.8 Bohr, cutoff 5 sigma), "
                   "840 x 420 x 420 grid (h = 0.257 Bohr)")
    elif args.workload == "ortho360":
        S = synth.config3b()
        wl_text = (f"orthorhombic 37.9 x 40.4 x 42.1 Bohr cell, {S.n_atoms} Gaussian charges at diamond density "
                   "(sigma 0.5 Bohr, cutoff 5 sigma), 360 x 384 x 400 grid")
    else:
        S = synth.config5()
        wl_text = "diamond 4x4x4 supercell, 512 Gaussian charges (sigma 0.5 Bohr, cutoff 5 sigma), 256^3 grid"
    apl = 16
    t0 = time.perf_counter()
    perm, _ = atoms_reorder(S.pos, (S.n_atoms + apl - 1) // apl)
    reorder_ms = 1e3 * (time.perf_counter() - t0)
    pos_h, q_h = S.pos[perm], S.q[perm]
    from paper_1209_4506_gb300 import capi

    flags = capi.HARTREE_FLAG_TC_BF16 if args.precision == "bf16split" and args.tc_parts == "bf16" else 0
    plan = HartreePlan(S.n, S.cell, S.sigma, args.precision, atoms_per_leaf=apl, max_atoms=S.n_atoms, flags=flags)
    variants = plan.autotune()
    pos = torch.tensor(pos_h, device=dev)
    q = torch.tensor(q_h, device=dev)
    # the same decomposition on the device (hartree_atoms_reorder_device), timed with CUDA events
    pos_raw = torch.tensor(S.pos, device=dev)
    perm_d = torch.empty(S.n_atoms, dtype=torch.int32, device=dev)
    ls_d = torch.empty((S.n_atoms + apl - 1) // apl + 1, dtype=torch.int32, device=dev)
    stream0 = torch.cuda.current_stream(dev)

    def reorder_device():
        capi.check(capi.hartree_atoms_reorder_device(plan.handle, pos_raw.data_ptr(), None, S.n_atoms,
                                                     (S.n_atoms + apl - 1) // apl, perm_d.data_ptr(),
                                                     ls_d.data_ptr(), stream0.cuda_stream))

    reorder_device_ms = time_events(reorder_device, 10, stream0)
    reorder_device_equal = bool(np.array_equal(perm_d.cpu().numpy(), perm))
    vh = torch.empty(S.n, dtype=torch.float32, device=dev)
    rho = torch.empty(S.n, dtype=torch.float32, device=dev)
    eh = torch.empty((), dtype=torch.float64, device=dev)
    f = torch.empty((S.n_atoms, 3), dtype=torch.float64, device=dev)
    ntot = S.n_tot
    ybytes = 40.0 * ntot
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.step(pos, q, vh=vh, eh=eh, f=f)

    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)  # let the sampler attach before the timed region
    launches0 = plan.launch_count
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = plan.launch_count - launches0
    t_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_per_step = t_ms / args.steps
    value = job_throughput(ybytes, args.steps, t_ms * 1e-3, world)

    # per-kernel durations from CUDA events on the launching stream (same kernels, split calls)
    names = ["splat", "pass0_c_r2c", "pass1_b_fwd", "pass2_a_green", "pass3_b_inv", "pass4_c_c2r", "forces"]
    acc = {k: 0.0 for k in names}
    reps = max(10, min(args.steps, 100))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
    for r in range(reps + 3):
        ev[0].record(stream)
        plan.splat(pos, q, rho)
        ev[1].record(stream)
        for p in range(5):
            plan.solve_pass(p, rho=rho, vh=vh)
            ev[2 + p].record(stream)
        plan.forces(pos, q, vh=vh, f=f, want_phi=False)
        ev[7].record(stream)
        torch.cuda.synchronize()
        if r >= 3:
            for i, k in enumerate(names):
                acc[k] += ev[i].elapsed_time(ev[i + 1])
    kernels_ms = {k: acc[k] / reps for k in names}
    solve_ms = sum(kernels_ms[k] for k in names[1:6])
    # the step's own kernels (a plan with HARTREE_FLAG_FUSED_SPLAT runs the splat inside pass 0)
    fused = plan.fused_splat
    if fused:
        kernels_ms["splat_r2c_fused"] = time_events(lambda: plan.splat_pass(pos, q), reps, stream)
    step_names = (["splat_r2c_fused"] if fused else ["splat", "pass0_c_r2c"]) + names[2:]
    # the opt-in fused splat on a plan of its own, against the two kernels it replaces
    fused_splat = None
    if not args.skip_side and args.precision == "fp32" and not fused:
        fplan = HartreePlan(S.n, S.cell, S.sigma, "fp32", atoms_per_leaf=apl, max_atoms=S.n_atoms,
                            flags=capi.HARTREE_FLAG_FUSED_SPLAT)
        if fplan.fused_splat:
            t_f = time_events(lambda: fplan.splat_pass(pos, q), reps, stream)
            fused_splat = {"fused_ms": t_f, "separate_ms": kernels_ms["splat"] + kernels_ms["pass0_c_r2c"],
                           "form": "HARTREE_FLAG_FUSED_SPLAT: atom setup + k_r2c_splat (density never in HBM) vs "
                                   "atom setup + k_splat_binned + the r2c pass"}
        fplan.close()
    # algorithmic bytes per launch (fp32): c passes read / write N real + N1 N2 (N3/2+1) complex, b / a read+write the
    # half spectrum; splat writes N; forces read V once
    half = 8.0 * S.n[0] * S.n[1] * (S.n[2] // 2 + 1)
    alg = {"splat": 4.0 * ntot, "pass0_c_r2c": 4.0 * ntot + half, "pass1_b_fwd": 2 * half,
           "pass2_a_green": 2 * half, "pass3_b_inv": 2 * half, "pass4_c_c2r": half + 4.0 * ntot,
           "forces": 4.0 * ntot, "splat_r2c_fused": half}
    kernel_names = {"splat": "k_leaf_setup + k_splat_binned", "pass0_c_r2c": "k_r2c_fast/k_r2c_stream",
                    "pass1_b_fwd": "k_col_fast/k_col_tma/k_col_pair MODE 0",
                    "pass2_a_green": "k_col_fast/k_col_tma/k_col_pair MODE 2",
                    "pass3_b_inv": "k_col_fast/k_col_tma/k_col_pair MODE 1",
                    "pass4_c_c2r": "k_c2r_fast/k_c2r_stream", "forces": "k_slab_order + k_forces<float>",
                    "splat_r2c_fused": "k_leaf_setup + k_r2c_splat"}
    # the roofline object: the longest kernel of the step as timed
    dom = max(step_names, key=lambda k: kernels_ms[k])
    pk, src = peaks()
    achieved = alg[dom] / (kernels_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": kernel_names[dom], "achieved": achieved, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": kernel_traffic(kernel_names[dom]),
                "algorithmic_bytes": alg[dom], "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"
                if src == "measured" else "fallback 6.8 TB/s"}
    solve_roofline = {"bound": "hbm", "achieved": ybytes / (solve_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                      "unit": "GB/s", "frac": ybytes / (solve_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                      "note": "five Poisson passes, 40 N_tot algorithmic bytes"}

    e2e = adjoint = batched = other = None
    if not args.skip_side:
        e2e, adjoint, batched, other = side_sections(args, plan, pos_h, q_h, pos, q, rho, vh, stream, world, barrier, ybytes,
                                              solve_ms + kernels_ms["splat"], dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = len(os.sched_getaffinity(0))
        t_list = [oracle_sample(threads)[0] for _ in range(3)]
        t_cpu = statistics.median(t_list)
        t_one = oracle_sample(1)[0]  # the same step on one core
        cpu = {"value": 40.0 * 256 ** 3 / t_cpu / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": SAMPLE_TEXT + f"; median of 3 steps, {t_cpu:.2f} s each",
               "single_core": {"value": 40.0 * 256 ** 3 / t_one / 1e9, "unit": "GB/s", "seconds": t_one}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else
                     ("f32, b passes f16 hi/lo split" if args.tc_parts == "fp16" else "f32, b passes bf16 3-part split"),
            "data": "synthetic",
            "config": {"workload": wl_text + (", FP32" if args.precision == "fp32" else
                                              ", FP32 with tensor-core split b passes") +
                                   ": splat + Poisson + E_H + forces",
                       "grid": list(S.n), "atoms": S.n_atoms, "yardstick_bytes_per_step": ybytes,
                       "l2": f"inputs larger than L2 (each grid array {4 * ntot / 1e9:.2f} GB)" if 4 * ntot > 129e6
                             else "working set larger than L2 (three 64 MB grid arrays); profiling case",
                       "parallelism": f"replicas x{world}", "variants": variants},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clocks, "solve_ms": solve_ms, "solve_gbs": ybytes / (solve_ms * 1e-3) / 1e9,
            "solve_points_per_s": ntot / (solve_ms * 1e-3), "solve_roofline": solve_roofline,
            "kernels_ms": kernels_ms, "step_kernels": step_names, "fused_splat": fused_splat,
            "step_path": "splat fused into the r2c pass (no density grid)" if fused
                         else "separate splat kernel and density grid",
            "batched": batched, "adjoint": adjoint, "other_grids": other,
            "solve_ms_ortho360": other["ortho360"]["solve_ms"] if other else None,
            "solve_ms_paper420": other["paper420"]["solve_ms"] if other else None,
            "reorder_ms": reorder_ms, "reorder_device_ms": reorder_device_ms,
            "reorder_device_equals_host": reorder_device_equal,
            "eh": float(eh.item()),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
