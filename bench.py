"""Benchmark of the polymer-flooding Newton step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c3|c2|c3s|c1|paper] [--precision fp64|mixed]
                    [--subs mixed,batch,serve|none] [--mode single|batch|serve]
                    [--profile-iters N]

A step is one full Newton iteration of the fully implicit water/oil/polymer
model (Alg. 1): property evaluation, residual and 3x3 block-Jacobian assembly
with upstream fluxes and wells, convergence test, forcing term (Sec. 3.3),
CPR preconditioner set-up and FGMRES solve (Alg. 2), update.  The timed
iterations run inside the time loop (begin-step work, convergence checks and
BHP-limit re-solves are inside the timed region).  The default workload is the
600x450x100 grid (27,000,000 cells, seeded channelised permeability, 40
injectors and 80 producers) in FP64; the metric is cells x Newton iterations
per second.

The default run (one GPU) prints one JSON line:
  * the headline: K timed Newton iterations, no instrumentation inside the
    timed region;
  * ``roofline``: the CPR-FP preconditioner apply (the largest share of the
    step) and the SpMV, per-launch times from a separate instrumented pass of
    the same workload (CUDA events around each launch);
  * ``e2e``: the same iterations through the C ABI with the state copied in
    from and out to pinned host memory every iteration (L2 flushed as in the
    device-timed loop);
  * ``mixed``, ``batch``, ``serve``: the mixed-precision form on the same
    grid (with its error against the FP64 path), the batched ensemble and the
    serving loop, each a shorter run whose size is stated in its entry;
  * ``cpu_baseline``: the FP64 oracle on all host cores (one process per
    core, each on a bounded sample of the workload) and on one core.

Multi-GPU: the path does not shard (one scenario per GPU), so N ranks run N
independent replicas; value is the total over ranks, time the max over ranks.

``--impl reference`` times the FP64 CPU oracle on the host cores (one process
per core) on a bounded sample of the same workload (rank 0 only).
``--profile-iters N`` runs N Newton iterations between cudaProfilerStart and
cudaProfilerStop after the warm-up and exits (for ncu --profile-from-start off).
"""

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from scenarios import generate as G  # noqa: E402

# GB300 FP64 (non-tensor) peak from unit counts and clocks: 152 SMs x 2070 MHz x
# 4 flop per clock per SM (2 FP64 FMA; 1.25 TFLOP/s nominal)
FP64_PEAK_TFLOPS = 152 * 2070e6 * 4 / 1e12
HBM_FALLBACK_GBS = 6800.0         # profiling recipe fallback when no measured peak exists
L2_BYTES = 129 * 1024 * 1024
# Algorithmic bytes and FP64 flops per cell of one CPR-FP preconditioner apply
# (Alg. 2): block-ILU(0) apply + stage-2 SpMV + pressure multigrid V-cycle, the
# per-cell figures of the survey's measurement table (FP64: 600 + 584 + 350 B;
# mixed, BF16/FP32 storage: 190 + 330 + 180 B; 126 + 126 + 60 flop).
PRECOND_BYTES_PER_CELL = {"fp64": 600 + 584 + 350, "mixed": 190 + 330 + 180}
PRECOND_FLOPS_PER_CELL = 126 + 126 + 60
# FP64 flops per cell the current apply kernels execute (interior cell): the
# ILU(0) sweeps 117 (black 6 x 9 multiply-adds through J_bj D_j^-1 and a 3x3
# product, red 6 x 8 and a 3x3 product, averaged over the colours), stage 2 on
# the black rows 24, the multigrid cycle about 37 (finest level 1+1 sweeps and
# the red-only restriction, the coarser levels 2+2 at 1/7 of the cells)
PRECOND_KERNEL_FLOPS_PER_CELL = 117 + 24 + 37
THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
STAGE1 = {"bjacobi": 0, "ilu0": 1}
SPMV_KERNEL = {False: "k_spmv_cells / k_spmv_rows (FP64, well border fused)",
               True: "k_spmv_cells_f32 (FP32 J and vector, well border fused)"}


def workload(name):
    if name == "c1":
        return G.scenario_c1(), "10x10x3 (300 cells), C1 physics, 30 daily steps"
    if name == "c3":
        return G.scenario_c3(), "600x450x100 (27,000,000 cells) channelised, 40 injectors / 80 producers"
    if name == "c3s":
        return (G.scenario_c3(nx=300, ny=225, nz=30),
                "300x225x30 (2,025,000 cells) channelised recipe, 40 injectors / 80 producers (profiling size)")
    if name == "paper":
        return (G.scenario_layered_table4(nx=951, ny=1920, refine_z=3, dt_days=1.0),
                "951x1920x15 (27,388,800 cells): the paper's high-resolution grid over the Table 4 layers "
                "(each split in three), 20x20x1.33 m cells, 4 corner injectors, horizontal producer, 1-day steps")
    return G.scenario_c2(), "100x100x10 (100,000 cells) layered lognormal, 5-spot, 0.3 PV slug"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return float(d.get("hbm_gbs", HBM_FALLBACK_GBS)), "measured"
        except Exception:
            pass
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the run."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per SpMV launch from
# the ncu captures summarised in profiles/; the 27M-cell figures are the 2M-cell
# captures scaled by the number of 3x3 blocks (traffic grows with them).
_BLOCKS_C3, _BLOCKS_C3S = 188_250_000, 14_008_500     # 3x3 blocks of 600x450x100 and 300x225x30
SPMV_TRAFFIC = {("c3s", "fp64"): 1000.17e6, ("c3s", "mixed"): 520.75e6,
                ("c3", "fp64"): 1000.17e6 * _BLOCKS_C3 / _BLOCKS_C3S,
                ("c3", "mixed"): 520.75e6 * _BLOCKS_C3 / _BLOCKS_C3S}
# DRAM traffic per CPR-FP preconditioner apply (summed over the apply's
# kernels) from the ncu captures summarised in profiles/ (300x225x30; the
# 600x450x100 figures scale its bytes per cell by the cells); None where no
# capture of the current kernels exists.
PRECOND_TRAFFIC = {("c3", "fp64"): 1091.9 * 27_000_000, ("c3", "mixed"): 441.9 * 27_000_000,
                   ("c3s", "fp64"): 2211.2e6, ("c3s", "mixed"): 894.8e6}


def max_over_ranks(values, dist, device="cpu"):
    """Element-wise maximum of per-rank timings (the slowest rank defines the
    job's time); identity without a process group."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


# Values of a 3x3 Jacobian block the SpMV needs: the oil row's polymer column is
# zero by the model's structure (no oil term depends on C), so 8 of the 9.
BLOCK_VALUES = 8


def spmv_bytes(blocks, ncell, npf, nw, jbytes, xbytes):
    """Algorithmic bytes of one SpMV launch: the 3x3 blocks of J (the 8 values
    that are not structurally zero, jbytes each), the vector read (xbytes per
    unknown) and the FP64 result written, the well border (B and C per
    perforation, D per well)."""
    return blocks * BLOCK_VALUES * jbytes + 3 * ncell * (xbytes + 8) + npf * 3 * 2 * jbytes + nw * jbytes


def spmv_flops(blocks, npf, nw):
    """Algorithmic flops of one SpMV launch: one multiply-add (2 flops) per
    nonzero block value, the well border's column (3 per perforation) and row
    (3 per perforation) and its diagonal."""
    return blocks * 2 * BLOCK_VALUES + npf * 12 + nw * 2


def assembly_bytes(ncell, jbytes):
    """Compulsory bytes of one assembly: x, phi_r, M^n, the three face
    transmissibilities and weights read (104 B per cell); R (24 B) and the 7
    Jacobian blocks (63 values of jbytes) written."""
    return ncell * (104 + 24 + 63 * jbytes)


def replica_throughput(world, cells, iters, seconds):
    """Whole-job cells x Newton iterations per second for ``world`` replicas
    that each ran ``iters`` iterations on ``cells`` cells in ``seconds``
    (max over ranks)."""
    return world * cells * iters / seconds


def spmv_algorithmic(sc, nwell_perf):
    """Bytes and FP64 flops of one SpMV launch (structured 3x3 blocks)."""
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    n = nx * ny * nz
    faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    blocks = n + 2 * faces
    return blocks, n, faces


def solver_opts(args, B, precision):
    prec = B.PF_PREC_MIXED if precision == "mixed" else B.PF_PREC_FP64
    pc = B.PF_PC_CPR if args.precond == "cpr" else B.PF_PC_BJACOBI
    return dict(precision=prec, precond=pc, use_forcing=1, newton_tol=args.newton_tol, gmres_restart=30,
                gmres_max_iter=300, autotune=args.autotune, amg_pre_sweeps=args.amg_pre,
                amg_post_sweeps=args.amg_post, amg_cycle=args.amg_cycle, forcing_form=args.forcing_form,
                stage1=STAGE1[args.stage1], amg_coarse_sweeps=args.amg_coarse, reorth_eta=args.reorth_eta,
                krylov_lookahead=args.lookahead, amg_coarse_size=args.amg_coarse_size)


class NewtonDriver:
    """Newton iterations inside the time loop (Sec. 3 step 4): a converged
    iteration ends the step (with the BHP-limit check; a switch re-solves the
    step), a diverged or capped step is cut in half; each ``iteration()``
    returns after one full assemble -> solve -> update."""

    def __init__(self, B, sim, dt):
        self.B, self.sim, self.dt0 = B, sim, dt
        self.dt = dt
        self.in_step = False
        self.its = 0

    def iteration(self):
        B, sim = self.B, self.sim
        while True:
            if not self.in_step:
                sim.begin_step(self.dt)
                self.in_step = True
                self.its = 0
            try:
                r = sim.newton_iteration()
            except B.PfError as e:        # diverged iterate: cut the step (Sec. 3, step 4(a))
                if e.status != B.PF_ENOT_CONVERGED:
                    raise
                sim.abort_step()
                self.in_step = False
                self.dt *= 0.5
                continue
            if r.converged:
                self.in_step = False
                if sim.end_step():
                    continue          # BHP-limit switch: re-solve the step
                self.dt = self.dt0
                continue
            self.its += 1
            if self.its >= 25:        # cut the step (Sec. 3, step 4(a))
                sim.abort_step()
                self.in_step = False
                self.dt *= 0.5
            return r


def timed_iterations(sim, drv, steps, stream, flush, dist):
    """``steps`` Newton iterations, each bracketed by CUDA events on the
    library's stream, L2 flushed before each; returns device seconds, host
    wall seconds, Krylov iterations and kernel launches of the region."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    krylov = 0
    launches0 = sim.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))                  # evict L2 between timed iterations (same stream)
        ev[k][0].record(stream)
        r = drv.iteration()
        ev[k][1].record(stream)
        krylov += r.krylov_iters
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    return dev_s, wall, krylov, sim.launch_count() - launches0


def instrumented_pass(B, sim, drv, steps):
    """Per-kernel-class launches and device time over ``steps`` further Newton
    iterations (CUDA events around every launch or graph launch); this pass
    is separate from the timed region."""
    import torch
    torch.cuda.synchronize()
    sim.kernel_timing_enable(True)
    for _ in range(steps):
        drv.iteration()
    torch.cuda.synchronize()
    kt = {name: sim.kernel_timing(name) for name in B.PF_KT}
    sim.kernel_timing_enable(False)
    return kt


def e2e_iterations(sim, drv, steps, stream, flush, dist):
    """The metric end to end through the C ABI with host buffers: each
    iteration takes the state from pinned host memory, runs one Newton
    iteration and returns the state to pinned host memory (two buffers
    alternate); L2 is flushed before each iteration as in the device loop."""
    import torch
    nunk = sim.nunk
    h_in = torch.empty(nunk, dtype=torch.float64, pin_memory=True)
    h_out = torch.empty(nunk, dtype=torch.float64, pin_memory=True)
    sim.get_x_ptr(h_in.data_ptr())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    bufs = (h_in, h_out)
    krylov = 0
    t0 = time.perf_counter()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        sim.set_x_ptr(bufs[k % 2].data_ptr())
        krylov += drv.iteration().krylov_iters
        sim.get_x_ptr(bufs[(k + 1) % 2].data_ptr())
    torch.cuda.synchronize()
    return time.perf_counter() - t0, nunk * 8, krylov


def precond_roofline(kt, ncell, precision, hbm_peak, hbm_kind, traffic=None):
    """Roofline of one CPR-FP preconditioner apply (a CUDA graph of the
    first-stage sweeps, stage 2 and the multigrid cycle) from its live
    per-apply time: algorithmic bytes and flops per cell times the cells.
    FP64 takes the binding one of the FP64 rate and HBM; the mixed form does
    FP32/BF16 arithmetic and is bound by HBM."""
    cnt, ms = kt["precond"]
    if cnt == 0:
        return None
    t = ms / cnt / 1000.0
    nbytes = PRECOND_BYTES_PER_CELL[precision] * ncell
    flops = PRECOND_FLOPS_PER_CELL * ncell
    gbs = nbytes / t / 1e9
    tfl = flops / t / 1e12
    out = {"kernel": "CPR-FP preconditioner apply (Alg. 2; one CUDA graph: ILU(0) sweeps, stage 2, multigrid)",
           "algorithmic_bytes": nbytes, "algorithmic_flops": flops, "avg_launch_us": round(t * 1e6, 2),
           "launches": cnt, "traffic": traffic, "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4),
           "hbm_peak": hbm_peak, "hbm_peak_kind": hbm_kind}
    t_alu = flops / (FP64_PEAK_TFLOPS * 1e12) if precision == "fp64" else 0.0
    if t_alu > nbytes / (hbm_peak * 1e9):
        out.update(bound="alu", achieved=round(tfl, 4), peak=round(FP64_PEAK_TFLOPS, 4), unit="TFLOP/s (FP64)",
                   frac=round(tfl / FP64_PEAK_TFLOPS, 4),
                   peak_kind="FP64 rate from unit counts and clocks: 152 SMs x 2070 MHz x 4 flop/clk")
        # the same time against the flops the kernels execute (fewer than the survey's count)
        kfl = PRECOND_KERNEL_FLOPS_PER_CELL * ncell
        out["kernel_count"] = {"flops_per_cell": PRECOND_KERNEL_FLOPS_PER_CELL, "flops": kfl,
                               "achieved": round(kfl / t / 1e12, 4),
                               "frac": round(kfl / t / 1e12 / FP64_PEAK_TFLOPS, 4),
                               "traffic_frac": round(traffic / t / 1e9 / hbm_peak, 4) if traffic else None}
    else:
        out.update(bound="hbm", achieved=round(gbs, 1), peak=hbm_peak, unit="GB/s", frac=round(gbs / hbm_peak, 4),
                   peak_kind=hbm_kind)
    return out


def spmv_roofline(kt, sc, sim, precision, hbm_peak, hbm_kind, workload):
    blocks, ncell, faces = spmv_algorithmic(sc, sim.npf)
    mixed = precision == "mixed"
    jbytes = 4 if mixed else 8
    xbytes = 4 if mixed else 8      # J x with the FP64 vector, or its FP32 copy in mixed precision
    nbytes = spmv_bytes(blocks, ncell, sim.npf, sim.nw, jbytes, xbytes)
    flops = spmv_flops(blocks, sim.npf, sim.nw)
    cnt, ms = kt["spmv"]
    if cnt == 0:
        return None
    t = ms / cnt / 1000.0
    gbs = nbytes / t / 1e9
    tfl = flops / t / 1e12
    out = {"kernel": SPMV_KERNEL[mixed], "algorithmic_bytes": nbytes, "algorithmic_flops": flops,
           "avg_launch_us": round(t * 1e6, 2), "launches": cnt,
           "traffic": SPMV_TRAFFIC.get((workload, precision)), "hbm_gbs": round(gbs, 1),
           "hbm_frac": round(gbs / hbm_peak, 4), "hbm_peak": hbm_peak, "hbm_peak_kind": hbm_kind}
    t_alu = flops / (FP64_PEAK_TFLOPS * 1e12) if not mixed else 0.0
    if t_alu > nbytes / (hbm_peak * 1e9):
        out.update(bound="alu", achieved=round(tfl, 4), peak=round(FP64_PEAK_TFLOPS, 4), unit="TFLOP/s (FP64)",
                   frac=round(tfl / FP64_PEAK_TFLOPS, 4),
                   peak_kind="FP64 rate from unit counts and clocks: 152 SMs x 2070 MHz x 4 flop/clk")
    else:
        out.update(bound="hbm", achieved=round(gbs, 1), peak=hbm_peak, unit="GB/s", frac=round(gbs / hbm_peak, 4),
                   peak_kind=hbm_kind)
    return out


def assembly_roofline(kt, ncell, precision, hbm_peak):
    asm_calls = kt["props"][0]
    if asm_calls == 0:
        return None
    nbytes = assembly_bytes(ncell, 4 if precision == "mixed" else 8)
    t = sum(kt[k][1] for k in ("props", "face", "gather", "wells")) / 1000.0 / asm_calls
    gbs = nbytes / t / 1e9
    return {"kernels": "k_cell_props + k_face_flux + k_gather + k_wells", "algorithmic_bytes": nbytes,
            "us_per_assembly": round(t * 1e6, 2), "achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4),
            "hbm_peak": hbm_peak, "bound": "FP64 ALU (the residual and flux values stay FP64)"}


def start_sim(args, B, sc, precision, stream):
    """Simulator of ``sc`` on ``stream``, past its start-up steps (untimed,
    the library's own step loop) and ``args.warmup`` warm-up iterations."""
    import torch
    with torch.cuda.stream(stream):
        sim = B.Simulator(sc, stream=B.current_stream_handle(), **solver_opts(args, B, precision))
    sim.run_schedule(n_steps=args.startup_steps)
    drv = NewtonDriver(B, sim, sc["schedule"][0]["dt"])
    for _ in range(args.warmup):
        drv.iteration()
    torch.cuda.synchronize()
    return sim, drv


def run_profile_window(args, B):
    """--profile-iters: after the start-up and warm-up, N Newton iterations
    between cudaProfilerStart and cudaProfilerStop (what an ncu run with
    --profile-from-start off captures), then exit."""
    import torch
    sc, desc = workload(args.workload)
    stream = torch.cuda.Stream()
    sim, drv = start_sim(args, B, sc, args.precision, stream)
    l0 = sim.launch_count()
    torch.cuda.profiler.start()
    krylov = 0
    for _ in range(args.profile_iters):
        krylov += drv.iteration().krylov_iters
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    out = {"profile_window": desc, "precision": args.precision, "newton_iters": args.profile_iters,
           "krylov_iters": krylov, "kernel_launches": sim.launch_count() - l0}
    sim.close()
    return out


def run_ours(args, rank, world, dist):
    import torch
    from paper_1807_05298_gb300 import binding as B

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    B.set_programmatic_launch(bool(args.pdl))
    if args.profile_iters:
        return run_profile_window(args, B)
    sc, desc = workload(args.workload)
    stream = torch.cuda.Stream()
    sim, drv = start_sim(args, B, sc, args.precision, stream)
    n = sim.n
    tuning = sim.tuning()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    # headline: no instrumentation inside the timed region
    clocks = ClockSampler(dev)
    if rank == 0:
        clocks.start()
    dev_s, wall, krylov, launches = timed_iterations(sim, drv, args.steps, stream, flush, dist)
    clk = clocks.stop() if rank == 0 else None
    # per-kernel-class times, in a separate pass
    kt = instrumented_pass(B, sim, drv, args.prof_steps)
    # end to end with host buffers
    e2e_steps = args.e2e_steps or max(3, args.steps // 2)
    e2e_wall, state_bytes, e2e_krylov = e2e_iterations(sim, drv, e2e_steps, stream, flush, dist)

    prec_check = None
    if args.precision == "mixed" and args.check_fp64 and rank == 0:
        with torch.cuda.stream(stream):
            prec_check = precision_check(B, sim, sc, solver_opts(args, B, "mixed"), drv.dt0, drv.in_step,
                                         B.current_stream_handle())
    nw, npf = sim.nw, sim.npf
    spmv_roof = spmv_roofline(kt, sc, sim, args.precision, *peaks(), args.workload)
    sim.close()

    t_dev, e2e_wall, wall = max_over_ranks([dev_s, e2e_wall, wall], dist, device="cuda")
    value = replica_throughput(world, n, args.steps, t_dev)
    e2e_value = replica_throughput(world, n, e2e_steps, e2e_wall)
    hbm_peak, hbm_kind = peaks()
    pre_roof = precond_roofline(kt, n, args.precision, hbm_peak, hbm_kind,
                                PRECOND_TRAFFIC.get((args.workload, args.precision)))
    roof = dict(pre_roof) if pre_roof else spmv_roof
    if pre_roof:
        roof["spmv"] = spmv_roof
    out = None
    if rank == 0:
        out = {
            "metric": "cells*Newton-iters/s",
            "value": round(value, 1),
            "unit": "cells*Newton-iters/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(1000.0 * t_dev / args.steps, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64-residual/f32-jacobian",
            "data": "synthetic (seeded SplitMix64/Box-Muller inputs shaped after the paper's workloads)",
            "config": {"workload": desc, "cells": n, "wells": nw, "perforations": npf, "precision": args.precision,
                       "autotune": args.autotune, "launch_shapes": tuning,
                       "amg": [args.amg_pre, args.amg_post, args.amg_cycle, args.amg_coarse],
                       "amg_coarse_size": args.amg_coarse_size,
                       "reorth_eta": args.reorth_eta, "precond": args.precond, "stage1": args.stage1,
                       "pdl": args.pdl, "krylov_lookahead": args.lookahead, "gmres_restart": 30,
                       "forcing_term": f"Sec. 3.3 form {args.forcing_form}", "newton_tol": args.newton_tol,
                       "startup_steps": args.startup_steps,
                       "l2": "flushed between timed iterations (256 MiB write); the working set also exceeds L2"
                             if n >= 1_000_000 else "flushed between timed iterations (256 MiB write)",
                       "timing": "CUDA events on the library's stream around each timed iteration, no "
                                 "per-kernel instrumentation; kernel shares and the roofline from a separate "
                                 "pass of %d iterations" % args.prof_steps,
                       "parallelism": "replicas"},
            "krylov_iters_per_newton": round(krylov / args.steps, 2),
            "wall_s": round(wall, 4),
            "e2e": {"value": round(e2e_value, 1), "unit": "cells*Newton-iters/s",
                    "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                    "steps": e2e_steps, "krylov_iters_per_newton": round(e2e_krylov / e2e_steps, 2),
                    "timing": "host wall clock over later Newton iterations of the same run (the Krylov count "
                              "per iteration differs from the timed region's)"},
            "gpu_launches": int(launches),
            "roofline": roof,
            "assembly": assembly_roofline(kt, n, args.precision, hbm_peak),
            "kernels_ms": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in kt.items()},
            "kernels_ms_iters": args.prof_steps,
            "clocks": clk,
        }
        if prec_check is not None:
            out["precision_check"] = prec_check
        if world == 1:
            subs = [x for x in args.subs.split(",") if x and x != "none"]
            if "mixed" in subs and args.precision == "fp64":
                out["mixed"] = sub_mixed(args, B, sc, desc, value)
            if "batch" in subs:
                out["batch"] = run_batch(args, headline=value)
            if "serve" in subs:
                out["serve"] = run_serve(args, headline=value)
            out["cpu_baseline"] = None if args.no_cpu_baseline else cpu_baseline(args)
    return out


def sub_mixed(args, B, sc, desc, fp64_value):
    """The mixed-precision form on the headline's grid: FP32 assembly
    derivatives and Jacobian, FP32/BF16 preconditioner, FP64 residual, norms
    and Krylov orthogonalisation; timed like the headline over fewer
    iterations, with its error against the FP64 path on one step."""
    import torch
    stream = torch.cuda.Stream()
    sim, drv = start_sim(args, B, sc, "mixed", stream)
    tuning = sim.tuning()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    dev_s, wall, krylov, launches = timed_iterations(sim, drv, args.sub_steps, stream, flush, None)
    kt = instrumented_pass(B, sim, drv, max(2, args.prof_steps // 2))
    hbm_peak, hbm_kind = peaks()
    with torch.cuda.stream(stream):
        chk = precision_check(B, sim, sc, solver_opts(args, B, "mixed"), drv.dt0, drv.in_step,
                              B.current_stream_handle()) if args.check_fp64 else None
    n = sim.n
    sim.close()
    value = n * args.sub_steps / dev_s
    return {"value": round(value, 1), "unit": "cells*Newton-iters/s", "steps": args.sub_steps,
            "ms_per_step": round(1000.0 * dev_s / args.sub_steps, 4), "workload": desc,
            "dtype": "f64-residual/f32-jacobian/bf16-f32-preconditioner",
            "krylov_iters_per_newton": round(krylov / args.sub_steps, 2), "gpu_launches": int(launches),
            "vs_fp64_headline": round(value / fp64_value, 4), "launch_shapes": tuning,
            "roofline": precond_roofline(kt, n, "mixed", hbm_peak, hbm_kind,
                                         PRECOND_TRAFFIC.get((args.workload, "mixed"))),
            "precision_check": chk}


def oracle_sample(args):
    """A bounded sample of the workload for the CPU oracle: the full grid's
    recipe on its top layers (same physics, wells and schedule)."""
    if args.workload == "c1":
        return G.scenario_c1(), "full 10x10x3 grid"
    if args.workload == "c3":
        sc = G.scenario_c3(nx=120, ny=90, nz=2)
        return sc, "120x90x2 sample of the channelised recipe"
    if args.workload == "paper":
        sc = G.scenario_layered_table4(nx=40, ny=48, refine_z=1, dz=4.0 / 3.0, dt_days=1.0)
        return sc, "40x48x5 sample of the 951x1920x15 recipe (same cell size, one cell per layer)"
    sc = G.scenario_c2(nz=1)
    return sc, "100x100x1 slab (top layer) of the 100x100x10 recipe, injectors on their 400 bar limit"


class OracleRunner:
    """The oracle's Newton iteration (Alg. 1: dual-number assembly, scaled
    residual test, direct sparse solve, update) inside its own fixed-step time
    loop on a sample scenario; a step that fails within 25 iterations is cut in
    half.  One ``iteration()`` is one assemble -> solve -> update; convergence
    checks and step starts that fall on the way are included."""

    def __init__(self, sc, tol=1e-8):
        from oracle import model as M
        self.M = M
        self.st = M.Setup(sc)
        self.x = M.initial_state(self.st)
        # rate wells with a BHP limit run on the limit, the regime the GPU
        # benchmark reaches after its start-up steps
        self.ctl = [dict(c, ctrl="bhp", target=c["limit"]) if c["ctrl"] != "bhp" and c.get("limit") else dict(c)
                    for c in sc["schedule"][0]["controls"]]
        self.dt0 = self.dt = sc["schedule"][0]["dt"]
        self.tol = tol
        self.n = self.st.n
        self._begin()

    def _begin(self):
        M, st = self.M, self.st
        self.M_old = M.masses(st, self.x)
        self.gam = M.well_gamma(st, self.x, self.ctl)
        self.x_old = self.x.copy()
        self.its = 0

    def iteration(self):
        M, st = self.M, self.st
        while True:
            R, J = M.assemble(st, self.x, self.M_old, self.dt, self.ctl, self.gam)
            ok = np.all(np.isfinite(R))
            if ok and M.scaled_residual(st, R, self.dt, self.ctl) <= self.tol:
                self.dt = self.dt0            # step converged: start the next one
                self._begin()
                continue
            if not ok or self.its >= 25:      # cut the step
                self.x = self.x_old
                self.dt *= 0.5
                self._begin()
                continue
            self.x = M.update(st, self.x, M.solve_linear(J, -R), 0.2)
            self.its += 1
            return


def time_oracle(sc, budget_s, max_iters):
    r = OracleRunner(sc)
    its = 0
    t0 = time.perf_counter()
    while its < max_iters and time.perf_counter() - t0 < budget_s:
        r.iteration()
        its += 1
    return its, time.perf_counter() - t0, r.n


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(conn, workload):
    """One host core's oracle: the workload's bounded sample in its own time
    loop; answers ("iter", k) with the seconds k Newton iterations took and
    ("budget", seconds, cap) with the iterations that fit and their seconds."""
    import types
    sc, _ = oracle_sample(types.SimpleNamespace(workload=workload))
    r = OracleRunner(sc)
    conn.send(r.n)
    while True:
        msg = conn.recv()
        if msg[0] == "iter":
            t0 = time.perf_counter()
            for _ in range(msg[1]):
                r.iteration()
            conn.send(time.perf_counter() - t0)
        elif msg[0] == "budget":
            its, t0 = 0, time.perf_counter()
            while its < msg[2] and time.perf_counter() - t0 < msg[1]:
                r.iteration()
                its += 1
            conn.send((its, time.perf_counter() - t0))
        else:
            return


class OraclePool:
    """One oracle process per host core (spawned, one BLAS thread each), each
    on its own copy of the workload's sample; no GPU work in any of them."""

    def __init__(self, workload, procs):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in THREAD_VARS}
        for k in THREAD_VARS:
            os.environ[k] = "1"
        self.conns, self.procs = [], []
        try:
            for _ in range(procs):
                a, b = ctx.Pipe()
                p = ctx.Process(target=_oracle_worker, args=(b, workload), daemon=True)
                p.start()
                self.conns.append(a)
                self.procs.append(p)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.cells = [c.recv() for c in self.conns]

    def iterate(self, k=1):
        for c in self.conns:
            c.send(("iter", k))
        return [c.recv() for c in self.conns]

    def budget(self, seconds, cap=1000):
        for c in self.conns:
            c.send(("budget", seconds, cap))
        return [c.recv() for c in self.conns]

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)


def precision_check(B, sim, sc, opts, dt, in_step, stream):
    """Error of the mixed-precision result against the FP64 path: both take
    one time step from the same state under the same controls (switched rate
    wells pinned on their BHP limit, no further switching), each to the same
    Newton tolerance on the FP64 residual; reports the max-norm differences of
    the fields relative to each field's max-norm.  The FP64 path is the one the
    parity tests pin to the oracle at 1e-6."""
    if in_step:
        sim.abort_step()
    ctl = [dict(c) for c in sc["schedule"][0]["controls"]]
    for w, sw in enumerate(sim.switched()):
        if sw:
            ctl[w] = dict(ctl[w], ctrl="bhp", target=ctl[w]["limit"])
    ctl = [dict(c, limit=None) for c in ctl]
    x0 = sim.get_x()
    o64 = dict(opts, precision=B.PF_PREC_FP64)
    s64 = B.Simulator(sc, stream=stream, **o64)
    s64.set_controls(ctl)
    sim.set_controls(ctl)
    res = None
    for _ in range(4):
        s64.set_x(x0)
        sim.set_x(x0)
        rc_m, rep_m = sim.step(dt, raise_on_failure=False)
        rc_d, rep_d = s64.step(dt, raise_on_failure=False)
        if rc_m == B.PF_OK and rc_d == B.PF_OK:
            xm, xd = sim.get_x(), s64.get_x()
            n = sim.n
            err = {}
            for name, a in (("P", 0), ("S", 1), ("C", 2)):
                ref = max(float(np.abs(xd[a:3 * n:3]).max()), 1e-300)
                err[name] = float(np.abs(xm[a:3 * n:3] - xd[a:3 * n:3]).max()) / ref
            if sim.nw:
                ref = float(np.abs(xd[3 * n:]).max())
                err["Pb"] = float(np.abs(xm[3 * n:] - xd[3 * n:]).max()) / ref
            res = {"vs": "FP64 GPU path (pinned to the FP64 oracle at 1e-6 by the parity tests), same start "
                         "state and controls, one time step", "dt_days": dt / G.DAY,
                   "max_rel_err": {k: float("%.3e" % v) for k, v in err.items()},
                   "newton_iters": {"mixed": rep_m.newton_iters, "fp64": rep_d.newton_iters},
                   "krylov_iters": {"mixed": rep_m.krylov_iters, "fp64": rep_d.krylov_iters},
                   "newton_tol": opts["newton_tol"]}
            break
        dt *= 0.5
    s64.close()
    return res or {"vs": "FP64 GPU path", "error": "step did not converge in either precision"}


def cpu_baseline(args):
    """The FP64 oracle as it stands on the host cores: one process per core,
    each on its own copy of the bounded sample, for about cpu_budget seconds;
    and the same sample on one core for comparison."""
    sc, sample = oracle_sample(args)
    procs = host_cores()
    pool = OraclePool(args.workload, procs)
    try:
        res = pool.budget(args.cpu_budget)
    finally:
        pool.close()
    work = sum(n * its for n, (its, _) in zip(pool.cells, res))
    secs = max(t for _, t in res)
    its1, secs1, n1 = time_oracle(sc, args.cpu_budget / 2.0, 1000)
    return {"value": round(work / secs, 1), "unit": "cells*Newton-iters/s", "cores": procs, "kind": "oracle",
            "sample": "%s, one copy per core in %d processes (numpy dual-number assembly + scipy sparse LU, one "
                      "thread each): %d Newton iterations in %.1f s" % (sample, procs, sum(i for i, _ in res), secs),
            "one_core": {"value": round(n1 * its1 / secs1, 1), "cores": 1,
                         "sample": "%s: %d Newton iterations in %.1f s" % (sample, its1, secs1)},
            "host_cpus": os.cpu_count()}


def run_reference(args, rank):
    """The reference arm: the FP64 oracle on every host core, one process
    per core on its own copy of the bounded sample; a step is one Newton
    iteration on every core."""
    if rank != 0:
        return None
    sc, sample = oracle_sample(args)
    procs = host_cores()
    pool = OraclePool(args.workload, procs)
    try:
        for _ in range(args.warmup):
            pool.iterate(1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.iterate(1)
        secs = time.perf_counter() - t0
    finally:
        pool.close()
    value = sum(pool.cells) * args.steps / secs
    desc = "%s, one copy per host core (%d processes)" % (sample, procs)
    return {"impl": "reference", "metric": "cells*Newton-iters/s", "value": round(value, 1),
            "unit": "cells*Newton-iters/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000.0 * secs / args.steps, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": desc},
            "cpu_baseline": {"kind": "oracle", "cores": procs, "sample": desc, "value": round(value, 1),
                             "unit": "cells*Newton-iters/s"},
            "e2e": {"value": round(value, 1), "unit": "cells*Newton-iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_batch(args, headline=None):
    """64 uneven scenarios (20k-400k cells, the C2 recipe with seeded slug
    concentration and RRF) resident at once, driven concurrently (pf_batch),
    against the same members run one after another on one host thread, in the
    batched form's precision and in plain FP64."""
    import torch
    from paper_1807_05298_gb300 import binding as B
    torch.cuda.set_device(0)
    members = [G.scenario_member(i) for i in range(args.members)]
    cells = [sc["nx"] * sc["ny"] * sc["nz"] for sc in members]
    steps = args.batch_steps

    def opts(precision):
        return dict(precision=B.PF_PREC_MIXED if precision == "mixed" else B.PF_PREC_FP64, precond=B.PF_PC_CPR,
                    use_forcing=1, newton_tol=args.newton_tol, autotune=args.autotune, stage1=STAGE1[args.stage1])

    # the stream form (each member its own launches on its own stream), the
    # packed form (the members' assemblies packed into shared launches), and
    # the same members one after another
    runs = [("batched", args.batch_precision, args.threads, False), ("batched_packed", args.batch_precision,
                                                                     args.threads, True),
            ("one_at_a_time", args.batch_precision, 1, False)]
    if args.batch_precision != "fp64":
        runs.append(("one_at_a_time_fp64", "fp64", 1, False))
    out = {}
    for label, precision, threads, packed in runs:
        batch = B.Batch(members, n_threads=threads, packed=packed, pack_window_us=args.pack_window_us,
                        **opts(precision))
        batch.run(n_steps=args.startup_steps, raise_on_failure=False)   # start-up + graph capture, untimed
        torch.cuda.synchronize()
        p0 = batch.packing_stats()
        t0 = time.perf_counter()
        reps = batch.run(n_steps=steps, raise_on_failure=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        p1 = batch.packing_stats()
        batch.close()
        newton = [r.newton_iters if r.status == 0 else 0 for r in reps]
        work = sum(n * k for n, k in zip(cells, newton))
        out[label] = {"value": round(work / wall, 1), "wall_s": round(wall, 3), "newton_iters": sum(newton),
                      "failed_members": sum(1 for r in reps if r.status != 0),
                      "krylov_iters": sum(r.krylov_iters for r in reps), "threads": threads, "precision": precision}
        if packed:
            packs = p1[0] - p0[0]
            out[label].update(packs=packs, window_us=args.pack_window_us,
                              mean_members_per_pack=round((p1[1] - p0[1]) / packs, 2) if packs else None)
    best = max(("batched", "batched_packed"), key=lambda k: out[k]["value"])
    res = {"metric": "cells*Newton-iters/s", "value": out[best]["value"], "form": best, "unit": "cells*Newton-iters/s",
           "n_gpus": 1, "steps": steps, "warmup": args.startup_steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.batch_precision, "data": "synthetic",
           "config": {"workload": "batched ensemble: %d scenarios of 20k-400k cells (100x100x10 recipe, seeds "
                                  "100+), %d steps each after %d start-up steps" % (args.members, steps,
                                                                                   args.startup_steps),
                      "total_cells": sum(cells), "precision": args.batch_precision, "precond": "cpr",
                      "timing": "host wall clock around pf_batch_run (all members resident)"},
           "speedup_vs_one_at_a_time": round(out[best]["value"] / out["one_at_a_time"]["value"], 3)}
    res.update(out)
    if "one_at_a_time_fp64" in out:
        res["speedup_vs_one_at_a_time_fp64"] = round(out[best]["value"] / out["one_at_a_time_fp64"]["value"], 3)
    if headline is not None:
        res["vs_fp64_headline"] = round(out[best]["value"] / headline, 4)
    return res


def run_serve(args, headline=None):
    """Poisson arrivals of scenarios of 10k-2M cells (mixed precision), admitted
    by device footprint into a continuous-batching server; latency p50/p99 and
    aggregate throughput."""
    import torch
    from paper_1807_05298_gb300 import binding as B
    from scenarios.generate import uniform01
    torch.cuda.set_device(0)
    prec = B.PF_PREC_MIXED if args.serve_precision == "mixed" else B.PF_PREC_FP64
    opt = dict(precision=prec, precond=B.PF_PC_CPR, use_forcing=1, newton_tol=args.newton_tol,
               autotune=args.autotune, stage1=STAGE1[args.stage1])
    u = uniform01(5, 9, 2 * args.requests)
    reqs = []
    for r in range(args.requests):
        n = math.exp(math.log(1e4) + (math.log(2e6) - math.log(1e4)) * u[r])
        nx, ny, nz = G.scenario_size(500 + r, n, 10)
        reqs.append(G.scenario_c2(seed=500 + r, nx=nx, ny=ny, nz=nz, n_steps=args.serve_steps,
                                  slug_steps=args.serve_steps, dt_days=args.dt_days))
    cells = [sc["nx"] * sc["ny"] * sc["nz"] for sc in reqs]
    budget = int(args.hbm_budget_gb * 2 ** 30)
    srv = B.Server(budget, n_workers=args.threads, **opt)
    # capacity: a calibration burst submitted at once
    calib = reqs[:args.calib]
    t0 = time.perf_counter()
    tk = [srv.submit(sc) for sc in calib]
    res = [srv.wait(t) for t in tk]
    cap_wall = time.perf_counter() - t0
    cap_cells_s = sum(c * args.serve_steps for c in cells[:args.calib]) / cap_wall   # cells*steps per second
    mean_work = float(np.mean([c * args.serve_steps for c in cells]))
    lam = args.load * cap_cells_s / mean_work                                 # requests per second
    gaps = -np.log(uniform01(6, 9, args.requests)) / lam
    arrivals = np.cumsum(gaps)
    t0 = time.perf_counter()
    tickets = []
    for sc, ta in zip(reqs, arrivals):
        d = t0 + ta - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tickets.append(srv.submit(sc))
    res = [srv.wait(t) for t in tickets]
    srv.close()
    lat = np.array([r.t_end - r.t_submit for r in res])
    ok = [r.state == B.PF_REQ_DONE for r in res]
    span = max(r.t_end for r in res) - min(r.t_submit for r in res)
    work = sum(c * r.report.newton_iters for c, r in zip(cells, res))
    res = {"metric": "scenario latency p50/p99 and cells*Newton-iters/s", "value": round(work / span, 1),
            "unit": "cells*Newton-iters/s", "n_gpus": 1, "steps": args.serve_steps, "warmup": args.calib,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.serve_precision,
            "data": "synthetic", "config": {"workload": "serving: %d Poisson arrivals, 10k-2M cells, %d steps of "
                                                      "%g d each" % (args.requests, args.serve_steps, args.dt_days),
                                            "load": args.load, "arrival_rate_per_s": round(lam, 4),
                                            "hbm_budget_gb": args.hbm_budget_gb, "workers": args.threads},
            "latency_s": {"p50": round(float(np.percentile(lat, 50)), 4),
                          "p99": round(float(np.percentile(lat, 99)), 4), "max": round(float(lat.max()), 4)},
            "completed": int(sum(ok)), "requests": args.requests, "total_cells": int(sum(cells)),
            "capacity_cells_steps_per_s": round(cap_cells_s, 1)}
    if headline is not None:
        res["vs_fp64_headline"] = round(res["value"] / headline, 4)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c3s", "paper"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--precond", default="cpr", choices=["cpr", "bjacobi"])
    ap.add_argument("--newton-tol", type=float, default=1e-8)
    ap.add_argument("--startup-steps", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serve"])
    ap.add_argument("--subs", default="mixed,batch,serve",
                    help="sub-results in the default line (one GPU): mixed, batch, serve or none")
    ap.add_argument("--sub-steps", type=int, default=10, help="timed Newton iterations of the mixed sub-run")
    ap.add_argument("--prof-steps", type=int, default=4,
                    help="Newton iterations of the instrumented pass (kernel shares, roofline)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="end-to-end iterations (0: max(3, steps / 2))")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="run this many Newton iterations between cudaProfilerStart/Stop and exit")
    ap.add_argument("--autotune", type=int, default=1, help="tune the per-cell kernels' block sizes at set-up")
    ap.add_argument("--amg-pre", type=int, default=1)
    ap.add_argument("--amg-post", type=int, default=1)
    ap.add_argument("--amg-cycle", type=int, default=1)
    ap.add_argument("--reorth-eta", type=float, default=0.2,
                    help="second Gram-Schmidt pass when the first leaves less than this fraction of |w|")
    ap.add_argument("--amg-coarse-size", type=int, default=32,
                    help="cells of the coarsest pressure level, solved by a dense inverse (at most 64)")
    ap.add_argument("--amg-coarse", type=int, default=2,
                    help="smoothing sweeps on the levels below the finest (-1: as on the finest)")
    ap.add_argument("--pdl", type=int, default=0, help="programmatic dependent launch of the kernels")
    ap.add_argument("--lookahead", type=int, default=1, choices=[0, 1],
                    help="enqueue Arnoldi step j+1 before the host reads step j (krylov_lookahead)")
    ap.add_argument("--stage1", default="ilu0", choices=["bjacobi", "ilu0"],
                    help="local solve of the preconditioner (CPR first stage)")
    ap.add_argument("--check-fp64", type=int, default=1,
                    help="mixed precision: state the error against the FP64 path on one step")
    ap.add_argument("--forcing-form", type=int, default=3, choices=[1, 2, 3],
                    help="which choice of the Sec. 3.3 forcing term; 3 is the paper's")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--batch-precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--threads", type=int, default=16)
    ap.add_argument("--pack-window-us", type=float, default=0.0,
                    help="batch: how long the first member at an assembly waits for the others (packed form)")
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--serve-steps", type=int, default=10)
    ap.add_argument("--serve-precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--calib", type=int, default=8)
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--dt-days", type=float, default=2.0)
    ap.add_argument("--hbm-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    if args.mode != "single":
        from paper_1807_05298_gb300 import build as bld
        bld.build()
        out = run_batch(args) if args.mode == "batch" else run_serve(args)
        print(json.dumps(out))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out is not None:
            print(json.dumps(out))
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    from paper_1807_05298_gb300 import build as bld
    if rank == 0 or world == 1:
        bld.build()
    if dist:
        dist.barrier()
    out = run_ours(args, rank, world, dist)
    if out is not None:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
