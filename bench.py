#!/usr/bin/env python3
"""Throughput of the axisymmetric multiphase D2Q9 update on one GB300.

Workload (default): the FP32 propagating density wave on a 4096 (z) x 2048 (r)
lattice -- Carnahan-Starling EOS (a = 1, b = 4, R = 1) at T = 0.9 T_c on the
liquid branch (rho0 = coexistence liquid density), A = -0.152, tau = 0.6,
rho = rho0 (1 + 0.01 sin(2 pi z / nz)) + U(-1e-4, 1e-4) (PCG64 seed 20151201),
u = 0, free-slip top, specular axis, periodic z.  One step = one time step of
the whole lattice, which the fused kernel does in one launch (gather, moments,
psi, forces, EDM, axisymmetric source, collision).  Metric: MLUPS (million
lattice-node updates per second).

`python bench.py --gpus N --steps K --warmup W` prints one JSON line.  Under
torchrun each rank runs an independent replica (the solves share nothing), so
scaling is weak and value = all nodes updated / max rank time.
`--impl reference` times the FP64 CPU oracle on a bounded window of the same
workload instead.
"""
import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NZ, NR, TAU, A, T_OVER_TC = 4096, 2048, 0.6, -0.152, 0.9
# Algorithmic bytes per node and time step, FP32 (the roofline figure): the two-kernel form of the
# step reads 9 populations and writes rho, j_z, j_r, psi (52 B), then reads 9 populations and the 4
# fields and writes 9 populations (88 B): 140 B.  The fused kernel needs only the population floor,
# 9 reads + 9 writes = 72 B, which is reported beside it.
BYTES_STEP = 140
BYTES_FUSED = 72
BYTES_B = 88
WORKLOAD = "density wave 4096x2048, CS T=0.9Tc, tau=0.6, A=-0.152, FP32 deviation storage"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="wave", choices=["wave", "batched", "served"],
                    help="wave: the 4096x2048 density wave (headline); batched: 256 uneven droplets in one "
                         "launch per step vs one solve at a time; served: Poisson request stream with "
                         "continuous batching vs a one-at-a-time server")
    ap.add_argument("--requests", type=int, default=48, help="served: requests per arrival rate")
    ap.add_argument("--budget-mb", type=int, default=4096, help="served: HBM admission budget")
    ap.add_argument("--grid", default="%dx%d" % (NZ, NR),
                    help="wave: nz x nr of the wave (the default is the headline workload; other sizes are "
                         "for profiling)")
    ap.add_argument("--path", default="fused", choices=["fused", "split"],
                    help="wave: the single-pass kernel (default) or the two-kernel path")
    args = ap.parse_args()
    _set_grid(args.grid)
    return args


def _set_grid(spec):
    global NZ, NR, WORKLOAD
    nz, nr = (int(x) for x in spec.lower().split("x"))
    if (nz, nr) != (NZ, NR):
        NZ, NR = nz, nr
        WORKLOAD = "density wave %dx%d, CS T=0.9Tc, tau=0.6, A=-0.152, FP32 deviation storage" % (NZ, NR)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    """Measured HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            data = json.load(fh)

        def find(d):
            if isinstance(d, dict):
                for k, v in d.items():
                    if isinstance(v, (int, float)) and "hbm" in k.lower() and "gb" in k.lower():
                        return float(v)
                for v in d.values():
                    r = find(v)
                    if r:
                        return r
            return None

        v = find(data)
        if v:
            return v, "measured"
    except (OSError, ValueError):
        pass
    return 6800.0, "fallback"


def _source_hash():
    h = hashlib.sha256()
    for fn in sorted(glob.glob(os.path.join(ROOT, "paper_1512_01977_gb300", "csrc", "*"))):
        with open(fn, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic():
    """Per-launch DRAM bytes of the fused step kernel on this workload from the
    committed ncu summary, or None when the kernel sources changed since."""
    path = os.path.join(ROOT, "profiles", "k_step_batch_fp32_wave4096x2048.md")
    try:
        vals = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line and line.strip().startswith("- "):
                    k, v = line.strip()[2:].split(":", 1)
                    vals[k.strip()] = v.strip().strip("`")
        if vals.get("source_sha") == _source_hash():
            return int(float(vals["dram_bytes_per_launch"]))
    except (OSError, KeyError, ValueError):
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _wave_fields(nz, nr, rho0):
    from paper_1512_01977_gb300 import inputs as I

    return I.density_wave(nz, nr, rho0, amp=0.01, noise=1e-4, seed=20151201)


def _cpu_baseline(rho0, steps=4):
    """The FP64 oracle, as it stands, on the full grid for a few steps (1 core)."""
    import oracle as O

    p = O.make_params(NZ, NR, TAU, O.EOS_CS, T_OVER_TC, A=A, top=O.TOP_FREESLIP)
    o = O.Oracle(p).init(*_wave_fields(NZ, NR, rho0))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return {"value": NZ * NR * steps / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "%d steps of the full %dx%d grid, FP64, single thread (%.1f s)" % (steps, NZ, NR, dt)}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a 256 x 256 window of the workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle as O

    nz, nr = 256, 256
    p = O.make_params(nz, nr, TAU, O.EOS_CS, T_OVER_TC, A=A, top=O.TOP_FREESLIP)
    rho0 = O.eos.maxwell_densities(p)[1]
    o = O.Oracle(p).init(*_wave_fields(nz, nr, rho0))
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = nz * nr * args.steps / dt / 1e6
    sample = "%dx%d window of the workload (same EOS, tau, A, wave recipe), FP64, single thread" % (nz, nr)
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (oracle window %dx%d)" % (nz, nr), "nz": nz, "nr": nr},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import ctypes as C

    import numpy as np
    import torch

    import __graft_entry__
    from paper_1512_01977_gb300 import lbm

    from paper_1512_01977_gb300 import replicas

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    rep = replicas.Replicas(device=torch.device("cuda", local))
    __graft_entry__.build()

    eos = lbm.make_eos(lbm.EOS_CS, T_OVER_TC)
    rho0 = lbm.lbm_eos_coexistence(eos)[1]
    fields = _wave_fields(NZ, NR, rho0)
    n = NZ * NR
    # pinned host copies of the inputs and outputs (the e2e leg copies through them)
    pin = lambda: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    h_in = [pin() for _ in range(3)]
    for dst, src in zip(h_in, fields):
        dst[:] = src.reshape(-1)
    h_out = [pin() for _ in range(4)]

    stream = torch.cuda.Stream()
    s = lbm.Solver(NZ, NR, TAU, eos=eos, A=A, precision=32, rho_ref=rho0, stream=stream.cuda_stream)
    if args.path == "split":
        lbm.lbm_axi_set_tuning(s.h, lbm.PATH_SPLIT, 0)
    s.init(*h_in)
    lbm.lbm_axi_step(s.h, args.warmup)

    def barrier():
        rep.barrier()

    # ---- device-timed throughput: K steps, inputs resident in HBM
    props = torch.cuda.get_device_properties(local)
    smi_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if ws >= 1 else str(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(smi_index) as clk:
        e0.record(stream)
        lbm.lbm_axi_step_async(s.h, args.steps)
        e1.record(stream)
        e1.synchronize()
    lbm.lbm_axi_sync(s.h)
    barrier()
    ms = e0.elapsed_time(e1)
    ms_max = rep.max(ms)
    value = replicas.aggregate_rate(n * args.steps, ws, ms_max * 1e-3) / 1e6  # MLUPS

    # ---- per-kernel device time (CUDA events around each launch, same stream)
    path, rows_per_cta = lbm.lbm_axi_get_tuning(s.h)
    kr = max(20, min(args.steps, 1000))
    ms_a, ms_b = lbm.lbm_axi_time_kernels(s.h, kr)
    t_a, t_b = ms_a / kr * 1e-3, ms_b / kr * 1e-3
    t_iso = t_b  # one launch bracketed by its own events
    t_step = ms * 1e-3 / args.steps
    if path == lbm.PATH_FUSED:
        # the timed region ran this kernel alone, one launch per step: its average
        # launch duration over that region is the region's time per step
        t_a, t_b = 0.0, t_step
    peak, peak_kind = _peaks()
    # fused path: one launch does the whole step, so its algorithmic bytes are the step's 140 B/node
    bytes_main = BYTES_STEP if path == lbm.PATH_FUSED else BYTES_B
    ach_b = bytes_main * n / t_b / 1e9
    traffic = _ncu_traffic() if path == lbm.PATH_FUSED else None  # the committed counters are the fused kernel's

    # ---- end to end through the C ABI: pinned host -> init -> K steps -> moments -> pinned host
    barrier()
    w0 = time.perf_counter()
    lbm.lbm_axi_init(s.h, NZ, NR, *h_in)
    lbm.lbm_axi_step(s.h, args.steps)
    ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    rc = lbm.lib().lbm_axi_moments(s.h, *[ptr(a) for a in h_out])
    if rc != 0:
        raise lbm.LbmError(rc, "lbm_axi_moments")
    barrier()
    wall = time.perf_counter() - w0
    e2e = replicas.aggregate_rate(n * args.steps, ws, rep.max(wall)) / 1e6
    mass_rw, _ = s.mass()
    s.close()

    pop_mb = int(round(9 * n * 4 / 1e6))
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = _cpu_baseline(rho0)
        out = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nz": NZ, "nr": NR, "nodes": n, "replicas": ws,
                       "l2": ("no flush: inputs larger than L2 (2 x %d MB FP32 population buffers)" % pop_mb)
                       if 2 * pop_mb > 129 else "inputs smaller than L2 (%d MB): not an HBM measurement" % (2 * pop_mb),
                       "parallelism": "replicas only (independent solves per GPU)",
                       "device": props.name},
            "roofline": {"bound": "hbm",
                         "kernel": "k_step_batch (one-pass gather+psi+forces+EDM+source+collide; a batch of one)"
                         if path == lbm.PATH_FUSED else "k_update (forces+EDM+source+collide)",
                         "achieved": ach_b, "peak": peak, "unit": "GB/s", "frac": ach_b / peak,
                         "peak_source": peak_kind, "traffic": traffic,
                         "algorithmic_bytes_per_node": bytes_main, "avg_launch_us": t_b * 1e6,
                         "avg_launch_source": "timed region / launches" if path == lbm.PATH_FUSED
                         else "CUDA events around each launch",
                         "isolated_launch_us": t_iso * 1e6,
                         "launches_per_step": 1 if path == lbm.PATH_FUSED else 2,
                         "kernel_floor_bytes_per_node": BYTES_FUSED,
                         "kernel_floor_frac": BYTES_FUSED * n / t_step / 1e9 / peak,
                         "step_frac": BYTES_STEP * n / t_step / 1e9 / peak,
                         "rows_per_cta": rows_per_cta},
            "e2e": {"value": e2e, "unit": "MLUPS", "h2d_bytes_per_step": 3 * 8 * n / args.steps,
                    "d2h_bytes_per_step": 4 * 8 * n / args.steps,
                    "note": "one solve: init from pinned host fields, K steps, moments back to pinned host"},
            "gpu_launches": (1 if path == lbm.PATH_FUSED else 2) * args.steps,
            "clocks": clk.summary(),
            "mass_rweighted": mass_rw,
        }
        if cpu is not None:
            out["cpu_baseline"] = cpu
        print(json.dumps(out))
    rep.close()


def run_batched(args):
    """256 independent droplets (sizes log-uniform 64x32 .. 512x256, R = 0.25 of
    the shorter side, T/Tc ~ U[0.5, 0.85], tau ~ U[0.6, 1.0], CS, FP32 with
    deviations about rho_v, started at rest), `--steps` steps each: one batched launch per step
    (autotuned) against the same solves stepped one at a time."""
    import torch

    import __graft_entry__
    from paper_1512_01977_gb300 import inputs as I
    from paper_1512_01977_gb300 import lbm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    __graft_entry__.build()
    specs = I.batch_droplets(n=256, seed=4)
    steps = args.steps

    def make():
        out = []
        for sp in specs:
            eos = lbm.make_eos(lbm.EOS_CS, sp["T_over_Tc"])
            rv, rl = lbm.lbm_eos_coexistence(eos)
            s = lbm.Solver(sp["nz"], sp["nr"], sp["tau"], eos=eos, A=A, precision=32, rho_ref=rv)
            s.init(*I.droplet(sp["nz"], sp["nr"], sp["R"], rl, rv), physical=True)  # at rest
            out.append(s)
        return out

    nodes = sum(sp["nz"] * sp["nr"] for sp in specs)
    # one at a time: each solve's own CUDA-graph step loop
    solvers = make()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok_seq = []
    for s in solvers:
        try:
            s.step(steps)
            ok_seq.append(True)
        except lbm.LbmError:
            ok_seq.append(False)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    failed_seq = ok_seq.count(False)
    for s in solvers:
        s.close()
    # batched
    solvers = make()
    b = lbm.Batch(solvers)
    tuning = b.autotune(trials=3)
    b.step(args.warmup)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    b.step_async(steps)
    b.sync()
    t_batch = time.perf_counter() - w0
    status = b.status()
    b.close()
    for s in solvers:
        s.close()
    # only solves that finished every step are credited (a solve that went
    # unphysical is not counted in either arm)
    nodes_ok = sum(sp["nz"] * sp["nr"] for sp, st in zip(specs, status) if st == lbm.OK)
    nodes_ok_seq = sum(sp["nz"] * sp["nr"] for sp, ok in zip(specs, ok_seq) if ok)
    value = nodes_ok * steps / t_batch / 1e6
    print(json.dumps({
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": t_batch * 1e3 / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "256 droplets, log-uniform 64x32..512x256, one launch per step", "solves": 256,
                   "nodes": nodes, "nodes_completed": nodes_ok, "tuning_strip_grid": list(tuning),
                   "credit": "node-steps of solves that finished every step"},
        "one_at_a_time": {"value": nodes_ok_seq * steps / t_seq / 1e6, "unit": "MLUPS", "wall_s": t_seq,
                          "failed": failed_seq},
        "speedup_vs_one_at_a_time": (nodes_ok * steps / t_batch) / (nodes_ok_seq * steps / t_seq),
        "failed": sum(1 for x in status if x != lbm.OK),
        "gpu_launches": steps,
    }))


def run_served(args):
    """Poisson request streams (rates 10..1000/s): continuous batching vs one
    request at a time; p50 / p99 latency and MLUPS per rate."""
    import torch

    import __graft_entry__
    from paper_1512_01977_gb300 import inputs as I
    from paper_1512_01977_gb300 import serve

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    __graft_entry__.build()
    rows = []
    for rate in (10, 30, 100, 300, 1000):
        reqs = I.request_stream(rate, args.requests, seed=5)
        _, st = serve.serve(reqs, budget_bytes=args.budget_mb << 20)
        _, sq = serve.serve_sequential(reqs)
        rows.append({"rate_per_s": rate, "batched": st, "one_at_a_time": sq})
    best = max(r["batched"]["mlups"] for r in rows)
    print(json.dumps({
        "metric": "MLUPS", "value": best, "unit": "MLUPS", "n_gpus": 1, "steps": None, "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "served Poisson stream, droplets + waves, CS/vdW, T/Tc 0.5..0.9, "
                               "grids 32x32..1024x512, 1k..20k steps", "requests_per_rate": args.requests,
                   "budget_mb": args.budget_mb},
        "rates": rows,
    }))


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
