#!/usr/bin/env python
"""Benchmark of the fused lattice-Boltzmann step with the wall-link boundary
schemes (one JSON line on rank 0).

Default workload: 64 batched 2D Hartmann channels (widths U{64..512}, Ha
U[1,30], wall-to-node fraction q U[0,1), Shercliff c_w log-U[1e-3,1], seed
2506), FP16 offset storage with FP32 arithmetic, all cases advanced by one
kernel launch per time step, replayed as CUDA graphs; the FP64 invariant /
residual reduction runs every 100 steps inside the timed region.
``--workload pipe`` and ``--workload cd`` time the 3D MHD pipe and the
flow + concentration channel instead.

``--impl reference`` times the FP64 CPU oracle (the baseline this build is
checked against) on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline; time-to-steady-state at fixed error"
CHECK_EVERY = 100


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["hartmann_batch", "pipe", "pipe_fp32", "cd", "steady_pipe"],
                    default="hartmann_batch")
    # steady_pipe: time to steady state, warm-started FP16 batch vs cold FP32 one case at a time
    ap.add_argument("--steady-cases", type=int, default=4)
    ap.add_argument("--steady-tol", type=float, default=1e-8)
    ap.add_argument("--switch-tol", type=float, default=1e-5,
                    help="residual at which the FP16-storage phase hands over to FP32")
    ap.add_argument("--steady-max-steps", type=int, default=2000000)
    ap.add_argument("--train-cases", type=int, default=512)
    ap.add_argument("--train-R", type=float, default=62.0)
    ap.add_argument("--train-tol", type=float, default=1e-5)
    ap.add_argument("--train-epochs", type=int, default=100)
    ap.add_argument("--train-per-case", type=int, default=2048)
    ap.add_argument("--train-max-steps", type=int, default=200000)
    ap.add_argument("--reference-steps", type=int, default=0,
                    help="steady_pipe reference arm: steps to project the oracle's time over (0: the "
                         "plain form's step count is unknown to that arm; it reports seconds per 1000 steps)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch", default=None,
                    help="variant,block,blocks_per_sm,nodes_per_thread,stages,min_blocks (skips the autotuner)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-iters", type=int, default=5)
    return ap.parse_args()


# ----------------------------------------------------------------------------- workloads
def build_workload(name):
    """Returns dict(cases, geo=[(solid, links)], lattice, prec, physics, infos, desc)."""
    from paper_2506_00907_gb300 import cases as CS
    from paper_2506_00907_gb300 import inputs as IN
    from paper_2506_00907_gb300 import lbm
    if name == "hartmann_batch":
        cases, geo, infos = [], [], []
        for dr in IN.hartmann_batch(64):
            c, s, l, info = CS.hartmann_channel(dr["W"], dr["Ha"], dr["q"], dr["cw"], clamp_cw=True)
            cases.append(c)
            geo.append((s, l))
            infos.append(info)
        clamped = sum(1 for i in infos if i["cw_clamped"])
        return dict(cases=cases, geo=geo, infos=infos, lattice=lbm.LBM_D2Q9, prec=lbm.LBM_FP16S, cw_clamped=clamped,
                    physics=lbm.LBM_FLOW | lbm.LBM_MHD, planes=19, storage="fp16-offset", dim=2,
                    desc="64 batched 2D Hartmann channels, W~U{64..512} (W x (W+2) nodes), Ha~U[1,30], "
                         "q~U[0,1), c_w~logU[1e-3,1], seed 2506; D2Q9 + D2Q5 x 2 (B1, B2)")
    if name in ("pipe", "pipe_fp32"):
        dr = IN.pipe_draws(1, Ha=(5.0, 20.0), cw=(0.01, 1.0))[0]
        c, s, l, info = CS.pipe((32, 128, 128), 62.0, dr["Ha"], ("shercliff", dr["cw"]))
        prec = lbm.LBM_FP16S if name == "pipe" else lbm.LBM_FP32
        return dict(cases=[c], geo=[(s, l)], infos=[info], lattice=lbm.LBM_D3Q19, prec=prec,
                    physics=lbm.LBM_FLOW | lbm.LBM_MHD, planes=40, dim=3,
                    storage="fp16-offset" if name == "pipe" else "fp32",
                    desc="3D MHD pipe 32x128x128 (periodic axial), R = 62, Ha=%.2f, Shercliff c_w=%.3g; "
                         "D3Q19 + D3Q7 x 3" % (dr["Ha"], dr["cw"]))
    c, s, l, info = CS.reactive_channel(512, 256, 0.25, 0.05, 1e-2)
    return dict(cases=[c], geo=[(s, l)], infos=[info], lattice=lbm.LBM_D2Q9, prec=lbm.LBM_FP32,
                physics=lbm.LBM_FLOW | lbm.LBM_CD, planes=14, storage="fp32", dim=2,
                desc="D2Q9 flow + D2Q5 concentration 512x256, moving top wall U=0.05 with given C, "
                     "Robin reactive bottom wall k=1e-2, q=0.25")


# ----------------------------------------------------------------------------- helpers
STEP_SOURCES = ("lattice.cuh", "types.cuh", "kernels.cuh", "kernels_bulk.cuh", "kernels_ring.cuh")   # the step kernels


STEP_KERNEL = {
    0: "k_step (bulk nodes) + k_boundary (wall-link nodes)",
    1: "k_step_bulk (bulk-copy loads and stores, boundary nodes included)",
    2: "k_step_pair (x-adjacent node pairs, packed FP32) + k_boundary (wall-link nodes)",
    3: "k_step_ring (producer warp, bulk-copy ring of stages, consumer warps) + k_boundary (wall-link nodes)"}


def kernel_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2506_00907_gb300", "csrc")
    for f in STEP_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(workload):
    """DRAM bytes per step launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "step_traffic.json")
    try:
        rec = json.load(open(p)).get(workload)
    except Exception:
        return None
    if not rec or rec.get("kernel_hash") != kernel_hash():
        return None
    return rec.get("bytes_per_launch")


def peak_hbm():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device, self.lines, self.proc = device, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=lambda: self.lines.extend(iter(self.proc.stdout.readline, "")),
                                      daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, device=None):
    """The slowest rank's time (ms) through the initialised process group
    (any backend); the local value when there is no group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(units_per_rank, world, steps, ms_max):
    """Node updates of all ranks per second (weak scaling: every rank runs the
    same batch), in millions."""
    return world * units_per_rank * steps / (ms_max * 1e-3) / 1e6


# ----------------------------------------------------------------------------- oracle timing
def oracle_sample(wl, target_nodes):
    """OracleSim objects for the first cases of the workload up to target_nodes
    fluid nodes, with links from the oracle's own builder."""
    import oracle as O
    from oracle import links as LK
    sims, nodes = [], 0
    threads = os.cpu_count() or 1
    for (c, info) in zip(wl["cases"], wl["infos"]):
        shape = (c.nx, c.ny, c.nz)
        dim = wl["dim"]
        if "W" in info:
            d = 1.0 - info["q"]
            walls = LK.channel_y(2, c.nx, c.ny, 1, d, d)
            p = {(1, s, O.F): dict(kind=O.VELOCITY) for s in (0, 1)}
            p.update({(1, s, O.G0): dict(kind=O.FLUX, kappa1=info["kappa1"]) for s in (0, 1)})
            p.update({(1, s, O.G0 + 1): dict(kind=O.GIVEN, phi_wall=info["B0"]) for s in (0, 1)})
            solid = LK.box_solid(shape, walls)
            links = LK.box_links(2, shape, walls, p, has_g=True)
            has_h, has_g = False, True
        elif "R" in info:
            wall = info["wall"]
            g0 = dict(kind=O.GIVEN, phi_wall=0.0) if wall == "insulating" else \
                dict(kind=O.FLUX) if wall == "conducting" else dict(kind=O.FLUX, kappa1=-info["eta"] / (wall[1] * info["R"]))
            params = {O.F: dict(kind=O.VELOCITY), O.G0: g0, O.G0 + 1: dict(kind=O.GIVEN, phi_wall=info["B0"]),
                      O.G0 + 2: dict(kind=O.GIVEN, phi_wall=0.0)}
            solid = LK.pipe_solid(shape, info["R"])
            links, _ = LK.pipe_links(shape, info["R"], params)
            has_h, has_g = False, True
        else:
            d = 1.0 - info["q"]
            walls = LK.channel_y(2, c.nx, c.ny, 1, d, d)
            p = {(1, 0, O.F): dict(kind=O.VELOCITY), (1, 1, O.F): dict(kind=O.VELOCITY, u_wall=(info["U"], 0, 0)),
                 (1, 0, O.H): dict(kind=O.FLUX, kappa0=info["k"], kappa1=-info["k"]),
                 (1, 1, O.H): dict(kind=O.GIVEN, phi_wall=2.0, u_wall=(info["U"], 0, 0))}
            solid = LK.box_solid(shape, walls)
            links = LK.box_links(2, shape, walls, p, has_h=True)
            has_h, has_g = True, False
        s = O.OracleSim(dim, shape, solid, c.tau_nu, c.tau_D, c.tau_eta, tuple(c.accel), has_h, has_g, threads)
        s.set_links(links)
        s.init(rho0=c.rho0, C0=c.C0, B0=tuple(c.B0))
        sims.append((s, int(np.sum(np.asarray(solid) == 0))))
        nodes += sims[-1][1]
        if nodes >= target_nodes:
            break
    return sims, nodes, threads


def time_oracle(sims, budget_s=12.0, max_steps=None):
    """Steps the sample until the budget is used; returns (MLUPS, steps)."""
    for s, _ in sims:
        s.step(1)                       # warm
    nodes = sum(n for _, n in sims)
    t0 = time.perf_counter()
    steps = 0
    while True:
        for s, _ in sims:
            s.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s or (max_steps and steps >= max_steps):
            break
    return nodes * steps / el / 1e6, steps, el


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    if args.workload == "steady_pipe":
        return run_reference_steady(args)
    wl = build_workload(args.workload)
    sims, nodes, threads = oracle_sample(wl, 2.0e5)
    for _ in range(args.warmup):
        for s, _ in sims:
            s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s, _ in sims:
            s.step(1)
    el = time.perf_counter() - t0
    mlups = nodes * args.steps / el / 1e6
    sample = "first %d cases of the workload (%d fluid nodes), FP64 oracle, one time step per bench step" % (
        len(sims), nodes)
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["desc"], "sample": sample},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_steady(args):
    """The oracle on case 0 of the steady workload: seconds for --reference-steps
    time steps of all held-out cases, projected from the timed steps."""
    wl = steady_workload(args)
    sims, nodes, threads = oracle_sample(dict(wl, cases=wl["cases"][:1], infos=wl["infos"][:1]), 1.0)
    for _ in range(args.warmup):
        for s, _ in sims:
            s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s, _ in sims:
            s.step(1)
    el = time.perf_counter() - t0
    mlups = nodes * args.steps / el / 1e6
    fluid = sum(int(np.sum(np.asarray(s) == 0)) for s, _ in wl["geo"])
    steps = args.reference_steps or 1000
    value = fluid * steps / (mlups * 1e6)
    sample = "FP64 oracle on case 0 (%d fluid nodes), %d steps in %.1f s; value = %d steps of all %d cases at " \
             "that rate" % (nodes, args.steps, el, steps, len(wl["cases"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["desc"], "sample": sample},
            "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2506_00907_gb300 import build as B
    from paper_2506_00907_gb300 import lbm
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    wl = build_workload(args.workload)
    stream = torch.cuda.Stream()                 # the solver's stream; every event below is recorded on it
    torch.cuda.set_stream(stream)
    sol = lbm.Solver(wl["lattice"], wl["prec"], wl["physics"], wl["cases"], stream=stream.cuda_stream, device=local)
    for i, (s, l) in enumerate(wl["geo"]):
        sol.set_walls(i, s, l)
    fluid = sum(int(np.sum(np.asarray(s) == 0)) for s, _ in wl["geo"])
    tune = None
    if args.launch:
        sol.set_launch(*(int(x) for x in args.launch.split(",")))
        tune = sol.get_launch()
    elif not args.no_autotune:
        cache = os.path.join(ROOT, "paper_2506_00907_gb300", "_build", "autotune.txt")
        sol.autotune(cache, iters=20)
        tune = sol.get_launch()
    sol.set_graph(CHECK_EVERY)
    K = max(CHECK_EVERY, (args.steps // CHECK_EVERY) * CHECK_EVERY)
    W = max(3, args.warmup)

    kernel_ev = []                  # (start, end, steps) around each replay of the step graph

    def run(nsteps, timed=False, collect_last=True):
        # the check of each block of steps is collected only after the next
        # block has been enqueued, so the GPU never waits for the host
        done, pending = 0, False
        while done < nsteps:
            k = min(CHECK_EVERY, nsteps - done)
            if timed:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sol.step(k)
                b.record(stream)
                kernel_ev.append((a, b, k))
            else:
                sol.step(k)
            done += k
            if pending:
                sol.check_wait(raise_unstable=False)
                pending = False
            if done % CHECK_EVERY == 0:
                sol.check_async()
                pending = True
        if pending and collect_last:
            sol.check_wait(raise_unstable=False)
    run(W)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    run(K, timed=True, collect_last=False)
    e1.record(stream)
    sol.check_wait(raise_unstable=False)          # the last block's check (its kernels precede e1)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), device="cuda")
    if world > 1:
        dist.barrier()
    ms_step = ms / K
    value = whole_job_mlups(fluid, world, K, ms)

    elem = {lbm.LBM_FP64: 8, lbm.LBM_FP32: 4}.get(wl["prec"], 2)
    alg_bytes = 2.0 * wl["planes"] * elem * fluid                # one read + one write per population
    peak, peak_kind = peak_hbm()
    # the step kernels alone (bulk k_step + boundary k_boundary): replays of the
    # step graph hold only step launches
    per_step = lbm.lbm_launches_per_step(sol.ctx)
    launches = K * per_step + 2 * (K // CHECK_EVERY)
    ms_kernel = sum(a.elapsed_time(b) for a, b, _ in kernel_ev) / sum(k for _, _, k in kernel_ev)
    achieved = alg_bytes / (ms_kernel * 1e-3) / 1e9
    out = sol.check(raise_unstable=False)
    stable = bool(np.all(out[:, 5] == 0))

    # end to end through the C ABI: pinned host state in, 100 steps, reductions out
    blob_np = sol.get_state()
    pinned = torch.empty(blob_np.size, dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = blob_np
    red = np.zeros(8 * len(wl["cases"]))
    L = lbm.lib()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_iters):
        L.lbm_set_state(sol.ctx, pinned.data_ptr(), blob_np.size)
        sol.step(CHECK_EVERY)
        L.lbm_check(sol.ctx, red.ctypes.data_as(lbm.ctypes.POINTER(lbm.ctypes.c_double)))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * fluid * CHECK_EVERY * args.e2e_iters / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": int(blob_np.size) / CHECK_EVERY, "d2h_bytes_per_step": red.nbytes / CHECK_EVERY,
           "step": "host->device state copy from pinned memory, %d time steps, FP64 reductions read back; "
                   "bytes are per time step" % CHECK_EVERY}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sims, nodes, threads = oracle_sample(wl, 1.5e6)
        mlups, steps, el = time_oracle(sims, budget_s=12.0)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "FP64 oracle on the first %d cases (%d fluid nodes), %d steps in %.1f s" % (
                   len(sims), nodes, steps, el)}
    if rank == 0:
        traffic = measured_traffic(args.workload)
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl["desc"], "storage": wl["storage"], "cases": len(wl["cases"]),
                           "fluid_nodes": fluid, "launch": tune,
                           "graph_steps": CHECK_EVERY, "reduction_every": CHECK_EVERY,
                           "cw_raised_to_stability_limit": wl.get("cw_clamped", 0),
                           "l2": "state %.0f MB > 129 MB L2, no flush" % (2 * wl["planes"] * elem * fluid / 1e6),
                           "stable": stable},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "peak_kind": peak_kind,
                             "bytes_per_step": alg_bytes, "ms_per_step_kernels": ms_kernel,
                             "timing": "CUDA events on the solver stream around each replay of the %d-step "
                                       "graph inside the timed region (step launches only)" % CHECK_EVERY,
                             "kernel": STEP_KERNEL[tune["variant"] if tune else 0]
                                       + ": one time step, %d launches" % per_step},
                "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    sol.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- time to steady state
STEADY_SHAPE, STEADY_R = (32, 256, 256), 126.0


def steady_workload(args):
    """Held-out MHD pipes of the steady-state comparison (seed 2507)."""
    from paper_2506_00907_gb300 import cases as CS
    from paper_2506_00907_gb300 import inputs as IN
    from paper_2506_00907_gb300 import lbm
    from paper_2506_00907_gb300 import surrogate as SG
    held = IN.pipe_draws(args.steady_cases, seed=2507, Ha=SG.HA_RANGE, cw=SG.CW_RANGE)
    group = [CS.pipe(STEADY_SHAPE, STEADY_R, h["Ha"], ("shercliff", h["cw"])) for h in held]
    return dict(held=held, group=group, cases=[g[0] for g in group], geo=[(g[1], g[2]) for g in group],
                infos=[g[3] for g in group], dim=3, lattice=lbm.LBM_D3Q19, planes=40,
                desc="3D MHD pipe 32x256x256 (periodic axial), R = 126, %d held-out cases Ha~U[10,50], "
                     "Shercliff c_w~logU[1e-3,1] (seed 2507); D3Q19 + D3Q7 x 3" % len(held))


def run_steady(args):
    """Wall time to the steady-state residual: the plain form (FP32 storage,
    one case per context, cold start) against the combined form (network warm
    start, FP16 storage, all cases in one launch per step, then FP32 from
    the switch residual on)."""
    import torch
    from paper_2506_00907_gb300 import build as B
    from paper_2506_00907_gb300 import inputs as IN
    from paper_2506_00907_gb300 import lbm
    from paper_2506_00907_gb300 import surrogate as SG
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    if world > 1:
        raise SystemExit("steady_pipe runs on one GPU")
    torch.cuda.set_device(local)
    B.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    phys = lbm.LBM_FLOW | lbm.LBM_MHD
    wl = steady_workload(args)
    held, group = wl["held"], wl["group"]
    fluid = [int(np.sum(np.asarray(g[1]) == 0)) for g in group]

    # the network: steady fields that the batched solver produces at the training resolution
    t0 = time.perf_counter()
    draws = IN.pipe_draws(args.train_cases, seed=IN.SEED, Ha=SG.HA_RANGE, cw=SG.CW_RANGE)
    n_t = int(2 * args.train_R) + 4
    X, T, gstats = SG.generate(draws, n=n_t, R=args.train_R, tol=args.train_tol, max_steps=args.train_max_steps,
                               prec=lbm.LBM_FP32, batch=128, stream=stream.cuda_stream, per_case=args.train_per_case)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, hist = SG.train(X, T, epochs=args.train_epochs, batch=4096, lr=3e-3, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    sur = SG.Surrogate(net, SG.HA_RANGE, SG.CW_RANGE)

    def fields(sol, i, g):
        m = sol.moments(i)
        fl = np.asarray(group[g][1]).reshape(-1) == 0
        return m["u"][fl, 0], m["B"][fl, 0]

    # plain form
    plain = []
    for i, (c, solid, links, info) in enumerate(group):
        sol = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP32, phys, [c], stream=stream.cuda_stream)
        sol.set_walls(0, solid, links)
        sol.set_graph(CHECK_EVERY)
        torch.cuda.synchronize()
        t = time.perf_counter()
        k, r = sol.run_to_steady(args.steady_max_steps, CHECK_EVERY, args.steady_tol)
        dt = time.perf_counter() - t
        plain.append(dict(steps=int(k), residual=float(r), s=dt, fields=fields(sol, 0, i)))
        sol.close()
    plain_s = sum(p["s"] for p in plain)

    # combined form (contexts and walls are set up outside the timed region, as for the plain form)
    t_setup = time.perf_counter()
    s16 = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP16S, phys, wl["cases"], stream=stream.cuda_stream)
    s32 = lbm.Solver(lbm.LBM_D3Q19, lbm.LBM_FP32, phys, wl["cases"], stream=stream.cuda_stream)
    h2d = 0
    for i, (c, solid, links, info) in enumerate(group):
        s16.set_walls(i, solid, links)
        s32.set_walls(i, solid, links)
        h2d += np.asarray(solid).nbytes + np.asarray(links).nbytes
    s16.set_graph(CHECK_EVERY)
    s32.set_graph(CHECK_EVERY)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    t = time.perf_counter()
    warm = [SG.warm_start(s16, i, sur, g[3], STEADY_SHAPE, STEADY_R, held[i]["Ha"], held[i]["cw"])
            for i, g in enumerate(group)]
    k16, r16 = s16.run_to_steady(args.steady_max_steps, CHECK_EVERY, args.switch_tol)
    s32.convert_from(s16)
    k32, r32 = s32.run_to_steady(args.steady_max_steps, CHECK_EVERY, args.steady_tol)
    comb_s = time.perf_counter() - t
    t_rb = time.perf_counter()
    comb_fields = [fields(s32, i, i) for i in range(len(group))]
    readback_s = time.perf_counter() - t_rb
    s16.close()
    s32.close()

    def nrel(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    err_u = max(nrel(cf[0], p["fields"][0]) for cf, p in zip(comb_fields, plain))
    err_b = max(nrel(cf[1], p["fields"][1]) for cf, p in zip(comb_fields, plain))
    plain_steps = sum(p["steps"] for p in plain)
    alg = 2.0 * 40 * 4 * sum(f * p["steps"] for f, p in zip(fluid, plain))
    achieved = alg / plain_s / 1e9
    peak, peak_kind = peak_hbm()
    cpu = None
    if not args.no_cpu_baseline:
        sims, nodes, threads = oracle_sample(dict(wl, cases=wl["cases"][:1], infos=wl["infos"][:1]), 1.0)
        mlups, st, el = time_oracle(sims, budget_s=12.0)
        cpu_s = sum(f * p["steps"] for f, p in zip(fluid, plain)) / (mlups * 1e6)
        cpu = {"value": cpu_s, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": "FP64 oracle, case 0 of the workload (%d fluid nodes), %d steps in %.1f s = %.1f MLUPS; "
                         "value = the plain form's node updates to steady state at that rate" % (
                             nodes, st, el, mlups)}
    line = {"metric": METRIC, "value": comb_s, "unit": "s", "n_gpus": 1, "steps": int(k16 + k32),
            "warmup": 0, "ms_per_step": 1e3 * comb_s / max(1, k16 + k32), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "residual": args.steady_tol, "switch_residual": args.switch_tol,
                       "plain": "FP32 storage, one case per context, cold start, CUDA graphs of %d steps, "
                                "residual every %d steps" % (CHECK_EVERY, CHECK_EVERY),
                       "combined": "network warm start, FP16 offset storage with all cases in one launch per "
                                   "step until the switch residual, then FP32 storage (state converted on the GPU)",
                       "l2": "state > 129 MB L2, no flush"},
            "plain_s": plain_s, "speedup": plain_s / comb_s,
            "plain": [{k: v for k, v in p.items() if k != "fields"} for p in plain],
            "combined": {"fp16_steps": int(k16), "fp16_residual": float(r16), "fp32_steps": int(k32),
                         "fp32_residual": float(r32), "warm_started": warm},
            "error_vs_plain": {"u1": err_u, "b1": err_b},
            "surrogate": {"train_cases": args.train_cases, "train_R": args.train_R, "samples": int(len(X)),
                          "generate_s": gen_s, "train_s": train_s, "loss_first": float(hist[0]),
                          "loss_last": float(hist[-1]), "generate": gstats},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "plain form, k_step + k_boundary FP32 with the residual check every %d steps"
                                   % CHECK_EVERY},
            "e2e": {"value": setup_s + comb_s + readback_s, "unit": "s", "h2d_bytes_per_step": h2d / max(1, k16 + k32),
                    "d2h_bytes_per_step": sum(8 * 8 * f for f in fluid) / max(1, k16 + k32),
                    "step": "context creation and wall upload, the combined run, moments read back"},
            "gpu_launches": int(2 * (k16 + k32) + 3 * (k16 + k32) // CHECK_EVERY)}
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "steady_pipe":
        return run_steady(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
