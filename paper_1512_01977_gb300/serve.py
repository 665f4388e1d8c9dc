"""Continuous-batching request loop over the batched engine.

Requests (droplet oscillations and density waves of uneven grids, EOS kinds,
temperatures and step counts) arrive on a schedule.  The server keeps every
admitted solve's populations resident on the GPU, admits waiting requests in
arrival order while the summed device footprint stays within a budget, and
advances all active solves together -- one launch of the batched fused kernel
per time step -- in ticks that end when the next solve completes (or after
`max_tick_steps`).  Finished solves are read back (rho, mass) and released,
which frees room for the next admissions.  A request whose state goes
unphysical is retired with an error status without disturbing the others.

The one-at-a-time baseline (`serve_sequential`) runs the same requests in
arrival order, each alone.
"""
import dataclasses
import time

import numpy as np

from . import inputs as I
from . import lbm

TAU = 1.0
A = -0.152
LAMBDA_VDW = 0.01


@dataclasses.dataclass
class Result:
    id: int
    status: int
    t_arrive: float
    t_start: float
    t_done: float
    steps: int
    nodes: int
    mass_rweighted: float = float("nan")
    rho: np.ndarray = None

    @property
    def latency(self):
        return self.t_done - self.t_arrive


def make_solver(req, precision=32, stream=None):
    """Solver and initial fields of one request.  Droplets: P2-perturbed (0.05)
    droplet of radius 0.25 of the shorter side on the axis; waves:
    rho0 (1 + 0.01 sin(2 pi z / nz)) + U(-1e-4, 1e-4) on the liquid branch.
    tau is the request's "tau" when given, else TAU."""
    kind = lbm.EOS_CS if req["eos"] == "cs" else lbm.EOS_VDW
    eos = lbm.make_eos(kind, req["T_over_Tc"], lam=LAMBDA_VDW)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    nz, nr = req["nz"], req["nr"]
    if req["kind"] == "droplet":
        fields = I.droplet(nz, nr, 0.25 * min(nz, nr), rl, rv, eps=0.05)
        rho_ref = rv
    else:
        fields = I.density_wave(nz, nr, rl, seed=1000 + req["id"])
        rho_ref = rl
    s = lbm.Solver(nz, nr, req.get("tau", TAU), eos=eos, A=A, precision=precision, rho_ref=rho_ref if precision == 32 else 0.0,
                   stream=stream)
    return s, fields


def start(s, fields):
    """Initialise a request's solve with the fluid at rest (the given u = 0 is
    the physical velocity), as the droplet tests of the method start."""
    s.init(*fields, physical=True)
    return s


def _finish(s, req, status, t_arrive, t_start, t_done, keep_rho):
    res = Result(id=req["id"], status=status, t_arrive=t_arrive, t_start=t_start, t_done=t_done,
                 steps=req["steps"], nodes=req["nz"] * req["nr"])
    if status == lbm.OK:
        res.mass_rweighted = s.mass()[0]
        if keep_rho:
            res.rho = lbm.lbm_axi_moments(s.h, req["nz"], req["nr"], want=("rho",))["rho"]
    s.close()
    return res


def serve(requests, budget_bytes=4 << 30, max_tick_steps=2000, precision=32, keep_rho=False, clock=None,
          autotune=False):
    """Serve `requests` (dicts with t_arrive in seconds) with continuous
    batching.  Returns (results, stats)."""
    clock = clock or time.perf_counter
    pending = sorted(requests, key=lambda r: r["t_arrive"])
    active = []  # dicts: req, solver, remaining, t_start, footprint
    results = []
    used = 0
    t0 = clock()
    qi = 0
    ticks = 0
    batch = None
    batch_members = None
    node_steps = 0
    while qi < len(pending) or active:
        now = clock() - t0
        # admit arrived requests in order while they fit
        while qi < len(pending) and pending[qi]["t_arrive"] <= now:
            req = pending[qi]
            fp = lbm.lbm_axi_footprint(req["nz"], req["nr"], precision)
            if active and used + fp > budget_bytes:
                break
            s, fields = make_solver(req, precision)
            qi += 1
            try:
                start(s, fields)
            except lbm.LbmError as e:  # unphysical initial state: retired at admission
                t = clock() - t0
                results.append(_finish(s, req, e.code, req["t_arrive"], t, t, keep_rho))
                continue
            active.append(dict(req=req, s=s, remaining=req["steps"], t_start=clock() - t0, fp=fp))
            used += fp
        if not active:
            if qi >= len(pending):
                break
            # idle until the next arrival
            wait = pending[qi]["t_arrive"] - (clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
            continue
        members = tuple(id(a["s"]) for a in active)
        if members != batch_members:
            if batch is not None:
                batch.close()
            batch = lbm.Batch([a["s"] for a in active])
            if autotune:
                batch.autotune(trials=3)
            batch_members = members
        k = min(max_tick_steps, min(a["remaining"] for a in active))
        batch.step_async(k)
        batch.sync()
        status = batch.status()
        ticks += 1
        node_steps += k * sum(a["req"]["nz"] * a["req"]["nr"] for a in active)
        now = clock() - t0
        keep = []
        for a, st in zip(active, status):
            a["remaining"] -= k
            if a["remaining"] <= 0 or st != lbm.OK:
                keep.append(None)
                results.append(_finish(a["s"], a["req"], st, a["req"]["t_arrive"], a["t_start"], now, keep_rho))
                used -= a["fp"]
            else:
                keep.append(a)
        if any(x is None for x in keep):
            batch.close()
            batch = None
            batch_members = None
            active = [a for a in keep if a is not None]
    if batch is not None:
        batch.close()
    makespan = clock() - t0
    return results, summarize(results, makespan, node_steps, ticks)


def serve_sequential(requests, precision=32, keep_rho=False, clock=None):
    """Baseline: one request at a time, in arrival order, each alone."""
    clock = clock or time.perf_counter
    pending = sorted(requests, key=lambda r: r["t_arrive"])
    results = []
    t0 = clock()
    node_steps = 0
    for req in pending:
        now = clock() - t0
        if req["t_arrive"] > now:
            time.sleep(req["t_arrive"] - now)
        t_start = clock() - t0
        s, fields = make_solver(req, precision)
        try:
            start(s, fields)
            s.step(req["steps"])
            st = lbm.OK
        except lbm.LbmError as e:
            st = e.code
        node_steps += req["steps"] * req["nz"] * req["nr"]
        results.append(_finish(s, req, st, req["t_arrive"], t_start, clock() - t0, keep_rho))
    makespan = clock() - t0
    return results, summarize(results, makespan, node_steps, len(pending))


def summarize(results, makespan, node_steps, ticks):
    lat = np.array([r.latency for r in results]) if results else np.array([np.nan])
    ok = sum(1 for r in results if r.status == lbm.OK)
    return dict(requests=len(results), completed=ok, failed=len(results) - ok,
                p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                mean_latency_s=float(lat.mean()), makespan_s=makespan,
                mlups=node_steps / makespan / 1e6 if makespan > 0 else float("nan"), ticks=ticks)
