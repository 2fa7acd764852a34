"""Benchmark of the immersed-boundary coupling step on GB300.

One step = the forward coupling (FE force + spreading + interpolation,
ib_forward) over the 256^3 workload: a Holzapfel-Ogden ventricle-like shell
(160x100x10 hexes) plus two fibre-reinforced leaflet-like sheets (80x40x2
each), 172,800 elements, 1,382,400 Gauss points, 16-mode velocity field.
Inputs are seeded and synthetic (inputs.py).  The adjoint (ib_backward: the
fused backward of the step for cotangents of f and U, with position, velocity
and material-parameter gradients) is timed the same way and reported as the
adjoint/forward ratio.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (bounded sample
of the same workload per step).  Under torchrun each rank runs an independent
replica (its own seed); value = Gauss points of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IB force+spread+interp Gauss-pts/s, % HBM roofline; adjoint/forward time ratio"
# The kernels of the spreading step as ib_spread runs them alone.
SPREAD_KERNELS = ("k_spread_zero<float>", "k_tile_info", "k_spread_push_fx", "k_spread_merge_fx")
# FE force: the algorithmic FP32 operations per Gauss point (fadd + fmul +
# 2 ffma, counted by ncu for the thread-per-element form of the force kernel,
# which does no redundant work, law set NH/Psi_2/Psi_4, on this workload; the
# eight-lane kernel k_fe8 executes 1,184, its shuffle reductions included);
# FP32 peak = 152 SMs x 128 lanes x 2 (fma) x the SM clock.
FE_FLOPS_PER_GP = 1024.5
FP32_LANES_PER_SM = 128
UNIT = "Gauss-pts/s"
# fluid of the explicit IB step (synthetic, unit periodic box): density,
# viscosity and time step
FLUID_RHO, FLUID_MU, FLUID_DT = 1.0, 0.01, 1e-4
WORKLOAD = ("shell256: 256^3 periodic MAC grid; HO ventricle-like shell 160x100x10 hex + two "
            "80x40x2 fibre-reinforced leaflet sheets; 172,800 trilinear hexes, 1,382,400 Gauss "
            "points; 16 divergence-free Fourier velocity modes")
L2_FLUSH_BYTES = 256 << 20


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(times, device="cpu"):
    """Per-step times reduced to their maximum over the ranks (replicas: the
    job ends when the slowest replica does).  No collective with one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(times), device=device, dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all replicas processed over the
    slowest replica's time."""
    return units_per_rank * world / (ms * 1e-3)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_sm_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def sum_traffic(kernels):
    """Sum of kernel_traffic over kernels (None if any is unknown)."""
    vals = [kernel_traffic(k) for k in kernels]
    return None if any(v is None for v in vals) else sum(vals)


def kernel_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's
    source is unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)[kernel]
        src = open(os.path.join(ROOT, d["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != d["sha"]:
            return None
        return float(d["bytes_per_launch"])
    except Exception:
        return None


def oracle_forward_rate(prob, min_seconds=10.0, max_reps=8):
    """The oracle (single-threaded FP64) on the whole workload, repeated."""
    import oracle
    from paper_2503_22695_gb300 import inputs as I
    m = oracle.Model(prob)
    x = I.from_split(prob.cell, prob.off, prob.grid)
    u = prob.u.astype("float64")
    reps, t0 = 0, time.perf_counter()
    while True:
        G, _ = m.fe_force(x)
        m.spread(x, G)
        m.interp(x, u)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds or reps >= max_reps:
            break
    support = m.support_count(x)
    return prob.n_gauss * reps / dt, reps, dt, support


# ---------------------------------------------------------------------------
# the oracle on every host core: the unchanged single-threaded oracle in one
# process per core, each on its own contiguous slice of the elements (the
# force, spreading and interpolation numerators are sums over elements, so
# the slices together are the whole forward)
# ---------------------------------------------------------------------------
def _sub_mesh(prob, e0, e1, x):
    """Elements [e0, e1) of a problem as a self-contained mesh (nodes renumbered)."""
    import numpy as np
    conn = prob.conn[:, e0:e1]
    used = np.unique(conn)
    remap = -np.ones(prob.n_nodes, dtype=np.int64)
    remap[used] = np.arange(len(used))
    return dict(grid=prob.grid, conn=remap[conn].astype(np.int32), X=prob.X[:, used],
                fibres=prob.fibres[:, e0:e1], mat_id=prob.mat_id[e0:e1],
                materials=prob.materials), np.ascontiguousarray(x[:, used])


def _oracle_worker(mesh, xs, shm_name, u_shape, min_s, steps, barrier, out):
    import numpy as np
    from multiprocessing import shared_memory
    import oracle
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        u = np.ndarray(u_shape, dtype=np.float64, buffer=shm.buf)
        m = oracle.Model(**mesh)
        q = 8 * m.E if m.conn.shape[0] == 8 else 4 * m.E
        barrier.wait()
        times = []
        for k in range(steps if steps else 1 << 30):
            t0 = time.perf_counter()
            G, _ = m.fe_force(xs)
            m.spread(xs, G)
            m.interp(xs, u)
            times.append(time.perf_counter() - t0)
            if steps:
                barrier.wait()          # steps end together (reference arm)
            elif sum(times) >= min_s:
                break
        out.put((q, times))
    finally:
        del u
        shm.close()


def oracle_pool_rate(prob, workers, min_s=3.0, steps=0, n_elems=None):
    """The oracle on `workers` host processes over the first n_elems elements
    (all by default).  steps = 0: every worker repeats the forward on its
    slice for at least min_s seconds; returns (Gauss points/s over the wall
    time, per-worker repetitions, wall seconds).  steps > 0: that many
    synchronised steps; returns (points per step, per-step wall seconds)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import numpy as np
    from paper_2503_22695_gb300 import inputs as I
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")           # never fork a CUDA process
    x = I.from_split(prob.cell, prob.off, prob.grid)
    E = prob.n_elems if n_elems is None else n_elems
    bounds = [E * i // workers for i in range(workers + 1)]
    shm = shared_memory.SharedMemory(create=True, size=prob.u.size * 8)
    try:
        np.ndarray(prob.u.shape, dtype=np.float64, buffer=shm.buf)[...] = prob.u
        barrier = ctx.Barrier(workers + 1)
        out = ctx.Queue()
        procs = []
        for i in range(workers):
            mesh, xs = _sub_mesh(prob, bounds[i], bounds[i + 1], x)
            pr = ctx.Process(target=_oracle_worker,
                             args=(mesh, xs, shm.name, prob.u.shape, min_s, steps, barrier, out))
            pr.start()
            procs.append(pr)
        barrier.wait()                      # every worker has built its slice
        t0 = time.perf_counter()
        step_t = []
        if steps:
            for _ in range(steps):
                barrier.wait()
                t1 = time.perf_counter()
                step_t.append(t1 - t0)
                t0 = t1
        res = [out.get() for _ in procs]
        wall = time.perf_counter() - t0
        for pr in procs:
            pr.join()
    finally:
        shm.close()
        shm.unlink()
    if steps:
        return sum(q for q, _ in res), step_t
    pts = sum(q * len(t) for q, t in res)
    return pts / wall, [len(t) for _, t in res], wall


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import oracle
    from paper_2503_22695_gb300 import inputs as I
    oracle.build()
    prob = I.shell_sheets_problem()
    workers = os.cpu_count() or 1
    E = prob.n_elems
    # per-step sample: the first k elements of the mesh (whole elements, the
    # full 256^3 grid), split over one oracle process per host core, sized
    # from a one-core probe so that W + K steps take about two minutes
    k0 = max(workers, E // 64)
    _, t_probe = oracle_pool_rate(prob, 1, steps=1, n_elems=k0)
    per_elem = t_probe[0] / k0
    budget = 120.0 / max(1, args.steps + args.warmup)
    k = int(min(E, max(workers, budget * workers / per_elem)))
    pts, step_t = oracle_pool_rate(prob, workers, steps=args.warmup + args.steps, n_elems=k)
    t = sum(step_t[args.warmup:]) / args.steps
    value = pts / t
    sample = (f"first {k} of {E} elements ({pts} Gauss points) of the shell256 workload per "
              f"step, full 256^3 grid (zero-fill and stencils included), split over "
              f"{workers} single-threaded oracle processes")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    from paper_2503_22695_gb300 import _build
    _build.build()
    from paper_2503_22695_gb300 import ibfe
    from paper_2503_22695_gb300 import inputs as I

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    if args.workload == "shell256":
        prob = I.shell_sheets_problem(seed=3000 + 17 * rank)
    else:   # smaller case for profiling captures: the 128^3 HO shell
        prob = I.shell_problem(seed=2000 + 17 * rank)
    Q, E, N = prob.n_gauss, prob.n_elems, prob.n_nodes
    n = prob.grid.n[0]
    conn = torch.from_numpy(prob.conn).to(dev)
    X = torch.from_numpy(prob.X).to(dev)
    fib = torch.from_numpy(prob.fibres).to(dev)
    mid = torch.from_numpy(prob.mat_id).to(dev)
    plan = ibfe.Plan(conn, X, prob.grid.n, prob.grid.h, fibres=fib, mat_id=mid)
    cell = torch.from_numpy(prob.cell).to(dev)
    off = torch.from_numpy(prob.off).to(dev)
    pos = ibfe.Pos(cell=cell, off=off)
    u = torch.from_numpy(prob.u).to(dev)
    tuning = fixed_or_autotuned(args, plan, [ibfe.Material(m.model, m.params)
                                             for m in prob.materials], pos, u)
    mats = [ibfe.Material(m.model, m.params) for m in prob.materials]
    G = torch.empty((3, N), device=dev)
    f = torch.empty(plan.grid_shape(), device=dev)
    U = torch.empty((3, N), device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(step_fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        for a, b in evs:
            flush.zero_()                      # L2 flush outside the timed interval
            a.record(stream)
            step_fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    fwd = lambda: ibfe.ib_forward(plan, mats, pos, u, G, f, U)
    # --- forward ---------------------------------------------------------
    for _ in range(args.warmup):
        fwd()
    barrier()
    # the timed steps sit inside a profiler range, so that a launch list taken
    # with `ncu --profile-from-start off` holds exactly their kernels
    torch.cuda.profiler.start()
    with ClockSampler(local) as clk:
        ms = timed(fwd, args.steps)
    torch.cuda.profiler.stop()
    t_fwd = sum(ms) / len(ms)
    barrier()
    # per-stage split from a separate pass with stage events on
    ibfe.ib_plan_profile(plan, reset=True)
    ibfe.ib_plan_set_profiling(plan, True)
    timed(fwd, args.steps)
    ibfe.ib_plan_set_profiling(plan, False)
    stages = ibfe.ib_plan_profile(plan, reset=True)
    # the spreading alone (ib_spread: its far-tile zeros, push and merge; in
    # ib_forward the zeros overlap the force) for its HBM roofline
    Gs = G.clone()
    for _ in range(args.warmup):
        ibfe.ib_spread(plan, pos, Gs, f)
    barrier()
    ibfe.ib_plan_set_profiling(plan, True)
    timed(lambda: ibfe.ib_spread(plan, pos, Gs, f), args.steps)
    ibfe.ib_plan_set_profiling(plan, False)
    spread_alone = ibfe.ib_plan_profile(plan, reset=True)["spread"]
    barrier()

    # --- the same forward with FP32 stability scalars (second plan) ---------
    plan32 = ibfe.Plan(conn, X, prob.grid.n, prob.grid.h, fibres=fib, mat_id=mid,
                       precision=ibfe.IB_FP32_SPLIT_F32STAB)
    fwd32 = lambda: ibfe.ib_forward(plan32, mats, pos, u, G, f, U)
    for _ in range(args.warmup):
        fwd32()
    barrier()
    ms32 = timed(fwd32, args.steps)
    t_fwd32 = sum(ms32) / len(ms32)
    del plan32
    barrier()

    # --- the same forward with the nodal quadrature rule (N coupling points) ---
    plann = ibfe.Plan(conn, X, prob.grid.n, prob.grid.h, fibres=fib, mat_id=mid,
                      quad=ibfe.IB_QUAD_NODAL)
    fwdn = lambda: ibfe.ib_forward(plann, mats, pos, u, G, f, U)
    for _ in range(args.warmup):
        fwdn()
    barrier()
    msn = timed(fwdn, args.steps)
    t_fwdn = sum(msn) / len(msn)
    del plann
    barrier()

    # --- the same structure as linear tetrahedra (six per hexahedron) -------
    tprob = I.tet_problem(prob)
    plant = ibfe.Plan(torch.from_numpy(tprob.conn).to(dev), X, prob.grid.n, prob.grid.h,
                      fibres=torch.from_numpy(tprob.fibres).to(dev),
                      mat_id=torch.from_numpy(tprob.mat_id).to(dev))
    ibfe.ib_plan_autotune(plant, mats, pos, u)
    fwdt = lambda: ibfe.ib_forward(plant, mats, pos, u, G, f, U)
    for _ in range(args.warmup):
        fwdt()
    barrier()
    mst = timed(fwdt, args.steps)
    t_fwdt = sum(mst) / len(mst)
    Et, Qt = tprob.n_elems, tprob.n_gauss
    del plant
    barrier()

    # --- quadratic (P2) tetrahedra: a node added at every edge's middle -----
    qprob = I.tet10_problem(prob)
    planq = ibfe.Plan(torch.from_numpy(qprob.conn).to(dev),
                      torch.from_numpy(qprob.X).to(dev), prob.grid.n, prob.grid.h,
                      fibres=torch.from_numpy(qprob.fibres).to(dev),
                      mat_id=torch.from_numpy(qprob.mat_id).to(dev))
    posq = ibfe.Pos(cell=torch.from_numpy(qprob.cell).to(dev),
                    off=torch.from_numpy(qprob.off).to(dev))
    ibfe.ib_plan_autotune(planq, mats, posq, u)
    Gq = torch.empty((3, qprob.n_nodes), device=dev)
    Uq = torch.empty((3, qprob.n_nodes), device=dev)
    fwdq = lambda: ibfe.ib_forward(planq, mats, posq, u, Gq, f, Uq)
    for _ in range(args.warmup):
        fwdq()
    barrier()
    msq = timed(fwdq, args.steps)
    t_fwdq = sum(msq) / len(msq)
    Eq, Nq, Qq = qprob.n_elems, qprob.n_nodes, qprob.n_gauss
    del planq, posq, Gq, Uq, qprob
    barrier()

    # --- adjoint ---------------------------------------------------------
    rng = np.random.default_rng(77 + rank)
    gU = torch.from_numpy(rng.normal(size=(3, N)).astype(np.float32)).to(dev)
    gf = torch.from_numpy((rng.normal(size=(3, n, n, n)) * 1e-3).astype(np.float32)).to(dev)
    gu = torch.empty_like(u)
    gx = torch.empty((3, N), device=dev)

    def adj():
        # the backward of the forward step for cotangents of f and U: position,
        # velocity and material-parameter gradients (one fused call)
        ibfe.ib_backward(plan, mats, pos, u, G, None, gf, gU, gx, gu)

    for _ in range(args.warmup):
        adj()
    barrier()
    ms_adj = timed(adj, args.steps)
    t_adj = sum(ms_adj) / len(ms_adj)
    barrier()

    # --- end to end through host buffers ---------------------------------
    # The step a user runs from host memory: positions and velocity up, G, f
    # and U down, every copy inside the timed interval.  The velocity upload
    # (201 MB) and the interpolation run on a second stream with a second
    # plan (a plan serves one call at a time) beside the force and the spread;
    # the field download overlaps the interpolation.  Outputs equal
    # ib_forward's bit for bit (checked once below).
    h_cell = cell.cpu().pin_memory()
    h_off = off.cpu().pin_memory()
    h_u = u.cpu().pin_memory()
    h_G = torch.empty((3, N), pin_memory=True)
    h_f = torch.empty(plan.grid_shape(), pin_memory=True)
    h_U = torch.empty((3, N), pin_memory=True)
    d_cell, d_off, d_u = torch.empty_like(cell), torch.empty_like(off), torch.empty_like(u)
    pos_e = ibfe.Pos(cell=d_cell, off=d_off)
    plan_i = ibfe.Plan(conn, X, prob.grid.n, prob.grid.h, fibres=fib, mat_id=mid)
    ibfe.ib_plan_set_tuning(plan_i, tuning)
    s_u = torch.cuda.Stream()
    ev_pos = torch.cuda.Event()
    Ge, fe, Ue = torch.empty_like(G), torch.empty_like(f), torch.empty_like(U)

    def e2e():
        d_cell.copy_(h_cell, non_blocking=True)
        d_off.copy_(h_off, non_blocking=True)
        ev_pos.record(stream)
        with torch.cuda.stream(s_u):
            s_u.wait_event(ev_pos)
            d_u.copy_(h_u, non_blocking=True)
            ibfe.ib_interp(plan_i, pos_e, d_u, Ue)
            h_U.copy_(Ue, non_blocking=True)
        ibfe.ib_fe_force(plan, mats, pos_e, Ge)
        h_G.copy_(Ge, non_blocking=True)
        ibfe.ib_spread(plan, pos_e, Ge, fe)
        h_f.copy_(fe, non_blocking=True)
        stream.wait_stream(s_u)

    for _ in range(args.warmup):
        e2e()
    barrier()
    fwd()
    torch.cuda.synchronize()
    if not (torch.equal(h_G, G.cpu()) and torch.equal(h_f, f.cpu()) and torch.equal(h_U, U.cpu())):
        raise RuntimeError("end-to-end outputs differ from ib_forward's")
    ms_e2e = timed(e2e, args.steps)
    t_e2e = sum(ms_e2e) / len(ms_e2e)
    # the link alone: the two large copies of the step (velocity up, field
    # down), each by itself and both at once on two streams
    up = lambda: d_u.copy_(h_u, non_blocking=True)
    down = lambda: h_f.copy_(fe, non_blocking=True)

    def both():
        with torch.cuda.stream(s_u):
            s_u.wait_stream(stream)
            up()
        down()
        stream.wait_stream(s_u)

    link = {}
    for key, fn in (("h2d_ms", up), ("d2h_ms", down), ("both_ms", both)):
        fn()
        ms_l = timed(fn, args.steps)
        link[key] = sum(ms_l) / len(ms_l)
    link["h2d_GBps"] = u.numel() * 4 / (link["h2d_ms"] * 1e-3) / 1e9
    link["d2h_GBps"] = f.numel() * 4 / (link["d2h_ms"] * 1e-3) / 1e9
    del plan_i
    barrier()
    h2d = (h_cell.numel() * 4 + h_off.numel() * 4 + h_u.numel() * 4)
    d2h = (h_G.numel() + h_f.numel() + h_U.numel()) * 4

    # --- fluid step and the explicit IB step (Section 4.2) at the same grid --
    fluid_line = None
    if not args.no_fluid:
        fl = ibfe.Fluid(prob.grid.n, prob.grid.h, FLUID_RHO, FLUID_MU, FLUID_DT)
        uf = torch.empty_like(u)
        pf = torch.empty(plan.grid_shape()[1:], device=dev)
        fstep = lambda: ibfe.ib_fluid_step(fl, u, f, uf, pf)
        for _ in range(args.warmup):
            fstep()
        barrier()
        ms_fl = timed(fstep, args.steps)
        _, _, res = ibfe.ib_fluid_step(fl, u, f, uf, pf, residuals=True)
        # the step advances x and u in place: both are restored from copies
        # outside the timed interval so every timed step starts from x^0, u^0
        cell0, off0, u0 = cell.clone(), off.clone(), u.clone()
        cs, os_, us = cell.clone(), off.clone(), u.clone()
        pos_s = ibfe.Pos(cell=cs, off=os_)

        def restore():
            cs.copy_(cell0)
            os_.copy_(off0)
            us.copy_(u0)

        def ibstep():
            ibfe.ib_step(plan, fl, mats, pos_s, us, G, f, U, pf)

        for _ in range(args.warmup):
            restore()
            ibstep()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for a, b in ev:
            restore()
            flush.zero_()
            a.record(stream)
            ibstep()
            b.record(stream)
        torch.cuda.synchronize()
        ms_st = [a.elapsed_time(b) for a, b in ev]
        cells = n ** 3
        t_fl, t_st = sum(ms_fl) / len(ms_fl), sum(ms_st) / len(ms_st)
        fluid_line = {
            "grid": [n, n, n], "rho": FLUID_RHO, "mu": FLUID_MU, "dt": FLUID_DT,
            "multigrid": {"levels": fl.levels(), "helmholtz_cycles": fl.cycles()[0],
                          "poisson_cycles": fl.cycles()[1],
                          "smoothing": "red-black Gauss-Seidel, 2 pre + 2 post sweeps",
                          "launch": "one CUDA graph per step"},
            "fluid_step_ms": t_fl, "cells_per_s": cells / (t_fl * 1e-3),
            "relative_residuals": {"helmholtz": res[0], "poisson": res[1]},
            "ib_step_ms": t_st,
            "ib_step_gauss_points_per_s": Q * world / (t_st * 1e-3),
            "note": "ib_step = nodal force + spread at x^n, fluid step, interpolation of "
                    "u^{n+1} at x^n, position update; x and u restored outside the timed "
                    "interval"}
        del fl, uf, cs, os_, us, cell0, off0, u0
        barrier()

    # --- batched workload: 48 HO shells on their own grids, one graph -----
    batch_line = None
    if not args.no_batch:
        bprobs = I.batch_problems(seed=5000 + 97 * rank)
        brng = np.random.default_rng(5 + rank)
        binst = []
        for bp in bprobs:
            N_i, sh = bp.n_nodes, (3,) + tuple(bp.u.shape[1:])
            binst.append(dict(
                conn=torch.from_numpy(bp.conn).to(dev), X=torch.from_numpy(bp.X).to(dev),
                fibres=torch.from_numpy(bp.fibres).to(dev),
                mat_id=torch.from_numpy(bp.mat_id).to(dev), n=bp.grid.n, h=bp.grid.h,
                mats=[ibfe.Material(m.model, m.params) for m in bp.materials],
                cell=torch.from_numpy(bp.cell).to(dev), off=torch.from_numpy(bp.off).to(dev),
                u=torch.from_numpy(bp.u).to(dev),
                G=torch.empty((3, N_i), device=dev), f=torch.empty(sh, device=dev),
                U=torch.empty((3, N_i), device=dev),
                gU=torch.from_numpy(brng.normal(size=(3, N_i)).astype(np.float32)).to(dev),
                gf=torch.from_numpy((brng.normal(size=sh) * 1e-3).astype(np.float32)).to(dev),
                gu=torch.empty(sh, device=dev), gx=torch.empty((3, N_i), device=dev)))
        batch = ibfe.Batch(binst)
        for _ in range(args.warmup):
            batch.forward()
            batch.adjoint()
        barrier()
        ms_bf = timed(batch.forward, args.steps)
        ms_ba = timed(batch.adjoint, args.steps)
        qb = sum(bp.n_gauss for bp in bprobs)
        tbf, tba = sum(ms_bf) / len(ms_bf), sum(ms_ba) / len(ms_ba)
        # the plain FP64 GPU form of the same instances: one FP64 plan each,
        # positions and data widened exactly, ib_forward called in turn
        f64 = []
        for bp, d in zip(bprobs, binst):
            g = bp.grid
            x64 = torch.from_numpy(I.from_split(bp.cell, bp.off, g)).to(dev)
            p64 = ibfe.Plan(d["conn"], d["X"].double(), g.n, g.h, g.origin,
                            fibres=d["fibres"].double(), mat_id=d["mat_id"],
                            precision=ibfe.IB_FP64)
            N_i, sh = bp.n_nodes, (3,) + tuple(bp.u.shape[1:])
            f64.append((p64, d["mats"], ibfe.Pos(x64=x64), d["u"].double(),
                        torch.empty((3, N_i), device=dev, dtype=torch.float64),
                        torch.empty(sh, device=dev, dtype=torch.float64),
                        torch.empty((3, N_i), device=dev, dtype=torch.float64)))

        def fwd64():
            for (p64, m64, x64, u64, G64, f64_, U64) in f64:
                ibfe.ib_forward(p64, m64, x64, u64, G64, f64_, U64)
        for _ in range(args.warmup):
            fwd64()
        ms_64 = timed(fwd64, args.steps)
        t64 = sum(ms_64) / len(ms_64)
        batch_line = {
            "workload": f"{len(bprobs)} HO ventricle-like shells, grids 32^3..128^3, "
                        f"{min(bp.n_elems for bp in bprobs)}..{max(bp.n_elems for bp in bprobs)} "
                        f"hexes each, {qb} Gauss points; one packed plan (one launch per "
                        f"stage over all instances), one CUDA-graph launch per pass",
            "gauss_points": qb, "forward_ms": tbf, "adjoint_ms": tba,
            "forward_value": qb / (tbf * 1e-3), "unit": UNIT,
            "adjoint_forward_ratio": tba / tbf, "tuning": batch.tuning(),
            "fp64_gpu_form": {"forward_ms": t64, "forward_value": qb / (t64 * 1e-3),
                              "note": "one FP64 plan per instance, ib_forward in turn; "
                                      "accuracy of both forms against the oracle in "
                                      "tests/test_gpu_batch.py"}}
        del batch, binst, f64
        barrier()

    # --- max over ranks ----------------------------------------------------
    t_fwd, t_adj, t_e2e = max_over_ranks([t_fwd, t_adj, t_e2e], dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # --- rooflines ----------------------------------------------------------
    # The headline roofline is the spreading step against HBM: its result is
    # the dense force field, 12 n^3 bytes written once (the spreading's
    # algorithmic bytes), over the step's own time when it runs alone
    # (ib_spread: far-tile zeros, accumulation and merge, timed by the
    # library's events on the stream its kernels are launched on).
    hbm_peak, peak_kind = measured_peaks()
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or measured_sm_mhz()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fwd_stages = {k: v for k, v in stages.items() if v[1] > 0}
    per_launch_ms = {k: v[0] / max(1, v[1]) for k, v in stages.items() if v[1] > 0}
    peak_src = ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s")
    spread_bytes = 12.0 * n ** 3            # the dense force field written once
    spread_ms = spread_alone[0] / max(1, spread_alone[1])
    spread_gbs = spread_bytes / (spread_ms * 1e-3) / 1e9
    roof = {"kernel": "spreading step (ib_spread alone: " + " + ".join(SPREAD_KERNELS) + ")",
            "bound": "hbm", "achieved": spread_gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": spread_gbs / hbm_peak,
            "traffic": sum_traffic(SPREAD_KERNELS),
            "traffic_unit": "DRAM bytes per step (ncu, sum over the step's kernels)",
            "bytes_per_launch": spread_bytes, "launch_ms": spread_ms,
            "peak_source": peak_src}
    force_ms = per_launch_ms["force"]
    fp32_peak = FP32_LANES_PER_SM * 2 * n_sm * sm_mhz * 1e6 / 1e12   # TFLOP/s
    fe_achieved = FE_FLOPS_PER_GP * Q / (force_ms * 1e-3) / 1e12
    force_roof = {"kernel": "k_fe8", "bound": "alu", "achieved": fe_achieved,
                  "peak": fp32_peak, "unit": "TFLOP/s (FP32)", "frac": fe_achieved / fp32_peak,
                  "traffic": kernel_traffic("k_fe8"), "traffic_unit": "DRAM bytes per launch",
                  "work_per_launch": FE_FLOPS_PER_GP * Q, "launch_ms": force_ms,
                  "peak_source": f"128 FP32 lanes x 2 x {n_sm} SMs x {sm_mhz:.0f} MHz (median "
                                 f"SM clock sampled during the timed steps)",
                  "note": "no FP64 instruction (J - 1 and I4f - 1 by compensated FP32 sums)"}

    # cpu baseline (the oracle on one core, then on every host core) and the
    # stencil-support count for the bytes model
    if args.no_cpu_baseline:
        cpu_rate, reps, cpu_t, support = None, 0, 0.0, 0
        pool_rate, pool_reps, pool_t, cores = None, [], 0.0, 0
    else:
        cpu_rate, reps, cpu_t, support = oracle_forward_rate(prob)
        cores = os.cpu_count() or 1
        pool_rate, pool_reps, pool_t = oracle_pool_rate(prob, cores)
    b_force = 56.0 * E + 52.0 * N
    b_interp = 4.0 * support + 12.0 * N
    b_fwd = b_force + spread_bytes + b_interp
    fwd_gbs = b_fwd / (t_fwd * 1e-3) / 1e9
    b_sup = b_force + 4.0 * support + b_interp
    sup_gbs = b_sup / (t_fwd * 1e-3) / 1e9
    # the interpolation kernel: velocity read on the stencil support (4|S|),
    # the points' split positions in (16 B) and w j0 U^IB out (12 B)
    interp_ms = per_launch_ms["interp"]
    b_ik = 4.0 * support + 28.0 * Q
    interp_roof = {"kernel": "k_interp_tma<0>", "bound": "hbm",
                   "achieved": b_ik / (interp_ms * 1e-3) / 1e9, "peak": hbm_peak,
                   "unit": "GB/s", "frac": b_ik / (interp_ms * 1e-3) / 1e9 / hbm_peak,
                   "traffic": kernel_traffic("k_interp_tma<0>"),
                   "traffic_unit": "DRAM bytes per launch", "bytes_per_launch": b_ik,
                   "launch_ms": interp_ms, "peak_source": peak_src,
                   "model": "4|S| (u on the stencil support) + 16 Q (positions) + 12 Q (values)"}
    launches = sum(v[2] for v in stages.values())
    workload = WORKLOAD if args.workload == "shell256" else (
        "shell128: 128^3 periodic MAC grid; HO ventricle-like shell 60x40x6 hex; 14,400 "
        "elements, 115,200 Gauss points (profiling case)")
    line = {
        "metric": METRIC,
        "value": job_rate(Q, world, t_fwd),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_fwd,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "precision": "FP32 arithmetic on split positions (int cell + FP32 offset); J-1 and the "
                     "fibre invariant I4f-1 as compensated FP32 pairs (twice-FP32 precision, "
                     "no FP64 instructions)",
        "data": "synthetic",
        "config": {"workload": workload, "grid": [n, n, n], "elements": E, "nodes": N,
                   "gauss_points": Q, "l2": "flushed before every timed step (256 MiB write)",
                   "tuning": dict(zip(("points_per_item", "force_ctas_per_sm",
                                       "spread_ctas_per_sm_cap", "interp_ctas_per_sm_cap"),
                                      tuning)),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "fp32_scalars": {"ms_per_step": t_fwd32, "value": Q * world / (t_fwd32 * 1e-3),
                         "note": "same forward with J-1 and I4f-1 as plain FP32 sums "
                                 "(IB_FP32_SPLIT_F32STAB; its Hessian-vector product misses the "
                                 "2e-5 adjoint tolerance at this size)"},
        "nodal_rule": {"ms_per_step": t_fwdn, "points": N,
                       "note": "the same forward with the nodal quadrature rule of Section 4.4 "
                               "(coupling points = the N nodes; the force keeps the Gauss rule)"},
        "tetrahedra": {"ms_per_step": t_fwdt, "elements": Et, "points": Qt,
                       "value": Qt * world / (t_fwdt * 1e-3), "unit": UNIT,
                       "note": "the same forward with every hexahedron split into six linear "
                               "tetrahedra (4-point coupling rule; force at the centroid)"},
        "tetrahedra_p2": {"ms_per_step": t_fwdq, "elements": Eq, "nodes": Nq, "points": Qq,
                          "value": Qq * world / (t_fwdq * 1e-3), "unit": UNIT,
                          "note": "the same forward on quadratic tetrahedra (the six tetrahedra "
                                  "per hexahedron with a node at every edge's middle; 4-point "
                                  "rule for force and coupling)"},
        "batched": batch_line,
        "fluid": fluid_line,
        "adjoint_ms_per_step": t_adj,
        "adjoint_forward_ratio": t_adj / t_fwd,
        "roofline": roof,
        "force_roofline": force_roof,
        "interp_roofline": interp_roof,
        "forward_roofline": {"bytes_per_step": b_fwd, "achieved_GBps": fwd_gbs,
                             "frac": fwd_gbs / hbm_peak, "peak": hbm_peak,
                             "support_faces": support,
                             "model": "56E + 52N (force) + 12 n^3 (spread) + 4|S| + 12N (interp)"},
        "support_roofline": {"bytes_per_step": b_sup, "achieved_GBps": sup_gbs,
                             "frac": sup_gbs / hbm_peak, "peak": hbm_peak,
                             "model": "the forward with the dense spread output 12 n^3 "
                                      "replaced by the stencil support 4|S|"},
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in fwd_stages.items()},
        "gpu_launches": launches,
        "e2e": {"value": job_rate(Q, world, t_e2e), "unit": UNIT, "ms_per_step": t_e2e,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipeline": "ib_fe_force + ib_spread on the caller's stream; velocity upload + "
                            "ib_interp on a second stream and plan; downloads as each output "
                            "is ready (outputs checked equal to ib_forward's)",
                "link": {k: round(v, 4) for k, v in link.items()},
                "link_note": "the 201 MB velocity upload and field download alone, each by "
                             "itself and both at once (pinned host buffers)"},
        "cpu_baseline": {"value": pool_rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"the full shell256 forward (force+spread+interp) split by "
                                   f"elements over {cores} single-threaded oracle processes, "
                                   f"{min(pool_reps) if pool_reps else 0}+ repetitions each in "
                                   f"{pool_t:.1f} s",
                         "single_core": {"value": cpu_rate, "unit": UNIT, "cores": 1,
                                         "sample": f"the full shell256 forward, {reps} "
                                                   f"repetitions in {cpu_t:.1f} s"}},
        "clocks": clocks,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def fixed_or_autotuned(args, plan, mats, pos, u):
    """The plan's launch tuning: --tuning if given, else the autotuner's choice.
    (A profiler slows the launches it does not capture, so a run under ncu
    that autotunes may choose differently from the bench; --tuning pins it.)"""
    from paper_2503_22695_gb300 import ibfe
    if args.tuning:
        t = [int(v) for v in args.tuning.split(",")]
        ibfe.ib_plan_set_tuning(plan, t)
        return t
    return ibfe.ib_plan_autotune(plan, mats, pos, u)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shell256", choices=["shell256", "shell128"],
                    help="shell128 (128^3 ventricle shell) is a small case for profiling")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-fluid", action="store_true",
                    help="skip the fluid step and the explicit IB step")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle timing (profiling runs)")
    ap.add_argument("--tuning", default=None,
                    help="points per item, force CTAs/SM, spread and interp caps, e.g. "
                         "1024,4,8,3 (default: the autotuner's choice)")
    ap.add_argument("--profile-once", choices=["forward", "backward", "fluid", "step"],
                    help="run one ib_forward (or ib_backward) between cudaProfilerStart/Stop "
                         "after warm-up, for ncu --profile-from-start off; prints no bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_once:
        return profile_once(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


def profile_once(args):
    """One forward or backward of the workload inside a profiler range."""
    import numpy as np
    import torch
    from paper_2503_22695_gb300 import ibfe
    from paper_2503_22695_gb300 import inputs as I
    p = I.named(args.workload)
    dev = "cuda"
    conn = torch.from_numpy(p.conn).to(dev)
    X = torch.from_numpy(p.X).to(dev)
    plan = ibfe.Plan(conn, X, p.grid.n, p.grid.h, p.grid.origin,
                     fibres=torch.from_numpy(p.fibres).to(dev),
                     mat_id=torch.from_numpy(p.mat_id).to(dev))
    pos = ibfe.Pos(cell=torch.from_numpy(p.cell).to(dev), off=torch.from_numpy(p.off).to(dev))
    mats = [ibfe.Material(m.model, m.params) for m in p.materials]
    u = torch.from_numpy(p.u).to(dev)
    rng = np.random.default_rng(77)
    gU = torch.from_numpy(rng.normal(size=(3, p.n_nodes)).astype(np.float32)).to(dev)
    gf = torch.from_numpy((rng.normal(size=p.u.shape) * 1e-3).astype(np.float32)).to(dev)

    fixed_or_autotuned(args, plan, mats, pos, u)   # the launch shapes the bench times
    if args.profile_once in ("fluid", "step"):
        fl = ibfe.Fluid(p.grid.n, p.grid.h, FLUID_RHO, FLUID_MU, FLUID_DT)
        f = torch.from_numpy((rng.normal(size=p.u.shape) * 50.0).astype(np.float32)).to(dev)
        if args.profile_once == "fluid":
            run = lambda: ibfe.ib_fluid_step(fl, u, f)
        else:
            run = lambda: ibfe.ib_step(plan, fl, mats, pos, u.clone())
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        run()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return 0
    for _ in range(2):
        G = ibfe.ib_forward(plan, mats, pos, u)[0]
        if args.profile_once == "backward":
            ibfe.ib_backward(plan, mats, pos, u, G, None, gf, gU)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    if args.profile_once == "forward":
        ibfe.ib_forward(plan, mats, pos, u)
    else:
        ibfe.ib_backward(plan, mats, pos, u, G, None, gf, gU)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    return 0


if __name__ == "__main__":
    sys.exit(main())
