#!/usr/bin/env python
"""Throughput benchmark of the MinxEnt-LBM time step on GB300.

Metric: lattice updates per second (GLUPS = 1e9 LU/s) of the fused
stream + MinxEnt4 collide + boundary step, with the achieved HBM fraction of
that kernel, for the mixed-precision batched form, beside the plain FP64
single-instance kernel and the error of the mixed form against FP64.

Default workload (one GPU): an ensemble of 64 D2Q9 lid-driven cavities of
uneven size (side 64 * U{1..16}), Reynolds number (log-uniform 100..1e4) and
lid speed (uniform 0.05..0.1), drawn with seed 0; FP32 collide arithmetic,
populations stored as FP16 deviations from W_a rho0; one persistent launch
per step over the per-instance tile table, step loop replayed from a CUDA
graph; per-instance FP64 mass / momentum totals every 100 steps.

One "step" = one time step of every instance.  With N GPUs (torchrun) the
ensemble has 64 N members, partitioned by cost across ranks with no
collective on the data path (weak scaling).

--impl reference times the FP64 CPU oracle (the paper's algorithm written
plainly, on the host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MinxEnt-LBM GLUPS & % HBM peak, mixed/batched vs plain FP64 at stated error"
MEMBERS_PER_GPU = 64
CONS_EVERY = 100
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=list(WORKLOADS), default="ensemble64")
    p.add_argument("--compute", choices=["f32", "f64"], default="f32")
    p.add_argument("--storage", choices=["f16", "bf16", "f32", "f64"], default=None,
                   help="default: the workload's own storage type")
    p.add_argument("--collision", choices=["minxent4", "minxent2", "mrt", "trt", "srt"],
                   default="minxent4",
                   help="srt: the SRT-BGK twin kernel (bandwidth reference); minxent2, mrt, "
                        "trt: the paper's other rules")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the FP64 comparison, e2e and CPU-baseline legs")
    return p.parse_args()


# ----------------------------------------------------------------------------
# Distributed plumbing (one process per GPU; barrier + max-over-ranks timing).
# ----------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if torch.cuda.is_available():
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def reduce(self, value: float, op: str) -> float:
        if not self.pg:
            return value
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------------------
# Workloads.  The default is the batched cavity ensemble; the others are the
# single-instance configurations, timed the same way (for profiling and for
# the per-config numbers).
# ----------------------------------------------------------------------------
WORKLOADS = {
    "ensemble64": "batched ensemble of 64 D2Q9 lid-driven cavities per GPU: side 64*U{1..16}, "
                  "Re log-uniform [100, 1e4], lid speed U[0.05, 0.1], seed 0",
    "cavity2048": "D2Q9 lid-driven cavity 2048x2048, lid speed 0.1, Re 5000, rho0 1 + U(-1e-6, 1e-6)",
    "tg512": "D2Q9 Taylor-Green vortex 512x512 periodic, u0 0.02, nu 1e-3",
    "tubes4096": "batched ensemble of 4096 D1Q3 shock tubes per GPU: N log-uniform [200, 20000], "
                 "density ratio U[1.5, 4], nu log-uniform [1e-5, 1e-2], seed 1",
    "tube800": "D1Q3 shock tube, 800 nodes, rho 1 | 0.5, nu 1e-3, zero-gradient ends",
}
DEFAULT_STORAGE = {"ensemble64": "f16", "cavity2048": "f16", "tg512": "f32", "tubes4096": "f32",
                   "tube800": "f32"}


class Workload:
    """Lattice parameters and initial fields of this rank's share."""

    def __init__(self, name: str, rank: int, world: int, members_per_gpu: int | None = None):
        from paper_1801_03863_gb300 import workloads as wl
        from paper_1801_03863_gb300.partition import partition
        self.name = name
        self.lattice, self.bc = "d2q9", "cavity"
        self.u_lid = None
        self.member_ids = [0]
        self.total_members = 1  # members over all ranks (single-instance runs: replicas)
        if name == "ensemble64":
            per = members_per_gpu or MEMBERS_PER_GPU
            self.total_members = per * world
            members = wl.cavity_ensemble(count=per * world, seed=0)
            mine = partition([m.side * m.side for m in members], world)[rank]
            self.member_ids = list(mine)
            self.members = [members[i] for i in mine]
            self.dims = [(m.side, m.side) for m in self.members]
            self.nu = [m.nu for m in self.members]
            self.u_lid = [m.u_lid for m in self.members]
            rho = [wl.cavity(members[i].side, noise=1e-6, seed=i)[0].ravel() for i in mine]
            self.rho = np.concatenate(rho)
            self.ux = np.zeros_like(self.rho)
            self.uy = np.zeros_like(self.rho)
        elif name == "cavity2048":
            side, u = 2048, 0.1
            self.dims, self.nu, self.u_lid = [(side, side)], [wl.nu_from_reynolds(5000, u, side)], [u]
            r, x, y = wl.cavity(side, noise=1e-6, seed=0)
            self.rho, self.ux, self.uy = r.ravel(), x.ravel(), y.ravel()
        elif name == "tg512":
            self.bc = "periodic"
            self.dims, self.nu = [(512, 512)], [1e-3]
            r, x, y = wl.taylor_green(512, u0=0.02)
            self.rho, self.ux, self.uy = r.ravel(), x.ravel(), y.ravel()
        elif name == "tubes4096":
            self.lattice, self.bc = "d1q3", "zero_gradient"
            self.total_members = (members_per_gpu or 4096) * world
            members = wl.tube_ensemble(count=self.total_members, seed=1)
            mine = partition([m.n for m in members], world)[rank]
            self.member_ids = list(mine)
            self.dims = [(members[i].n, 1) for i in mine]
            self.nu = [members[i].nu for i in mine]
            self.rho = np.concatenate([wl.tube_fields(members[i])[0].ravel() for i in mine])
            self.ux = np.zeros_like(self.rho)
            self.uy = None
        elif name == "tube800":
            self.lattice, self.bc = "d1q3", "zero_gradient"
            self.dims, self.nu = [(800, 1)], [1e-3]
            r, x = wl.shock_tube_1d(800)
            self.rho, self.ux, self.uy = r.ravel(), x.ravel(), None
        self.nodes = int(sum(a * b for a, b in self.dims))
        self.q = 9 if self.lattice == "d2q9" else 3

    def lattice_obj(self, compute: str, storage: str, collision: str = "minxent4"):
        from paper_1801_03863_gb300 import lbm
        return lbm.Lattice(self.lattice, self.dims, self.nu, self.bc, u_lid=self.u_lid,
                           compute=compute, storage=storage, collision=collision)

    def fields(self):
        return (self.rho, self.ux, self.uy) if self.q == 9 else (self.rho, self.ux)

    def bytes_per_lu(self, storage: str) -> int:
        return 2 * self.q * {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[storage]


# ----------------------------------------------------------------------------
# Measurement helpers.
# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        # samples under load: the top half of the clock distribution excludes idle edges
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d and d[k]:
                    return float(d[k]), "measured"
        except (OSError, ValueError):
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    """Hash of the sources the step kernels are compiled from."""
    h = hashlib.sha256()
    for f in ("lbm_common.cuh", "lbm_num.cuh", "lbm_collide.cuh", "lbm_step.cuh",
              "lbm_step_smem.cuh", "lbm_aux.h"):
        h.update(open(os.path.join(ROOT, "paper_1801_03863_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_node(storage: str, kind: str):
    """DRAM bytes per node of the step kernel from the committed ncu summary,
    or None when the kernel changed since the counters were taken or the
    counters were taken on another launch shape."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except ValueError:
        return None
    e = d.get(storage)
    if not e or e.get("source_hash") != kernel_source_hash() or e.get("kind") != kind:
        return None
    return float(e["dram_bytes_per_node"])


def _oracle_sim(wk: "Workload", i: int, nx: int | None = None, collision: str = "minxent4"):
    """An oracle lattice with instance i's parameters (optionally resized)."""
    import oracle
    from paper_1801_03863_gb300 import workloads as wl
    coll = {"minxent4": oracle.MINXENT4, "minxent2": oracle.MINXENT2, "mrt": oracle.MRT,
            "trt": oracle.TRT, "srt": oracle.SRT}[collision]
    nx0, ny0 = wk.dims[i]
    if wk.lattice == "d1q3":
        n = nx or nx0
        sim = oracle.Sim(oracle.D1Q3, n, 1, oracle.tau_from_nu(wk.nu[i]), oracle.BC_ZERO_GRADIENT,
                         collision=coll)
        r, x = wl.shock_tube_1d(n)
        sim.init(r, x)
        return sim, n
    side = nx or nx0
    bc = {"cavity": oracle.BC_CAVITY, "periodic": oracle.BC_PERIODIC}[wk.bc]
    nu = wk.nu[i]
    if wk.bc == "cavity" and nx:  # keep the Reynolds number when resizing
        nu = nu * side / nx0
    ulid = wk.u_lid[i] if wk.u_lid else 0.0
    sim = oracle.Sim(oracle.D2Q9, side, side if nx else ny0, oracle.tau_from_nu(nu), bc,
                     collision=coll, u_lid=ulid)
    if wk.bc == "cavity":
        sim.init(*wl.cavity(side, noise=1e-6, seed=0))
    else:
        sim.init(*wl.taylor_green(side, u0=0.02, ny=side if nx else ny0))
    return sim, side * (side if nx else ny0)


def cpu_oracle_sample(wk: "Workload", collision: str, budget_s: float = 12.0):
    """Time the FP64 oracle on instance 0 of the workload for ~budget_s seconds."""
    import oracle
    sim, nodes = _oracle_sim(wk, 0, collision=collision)
    t0 = time.perf_counter()
    sim.step(2)
    per = (time.perf_counter() - t0) / 2
    steps = max(2, int(budget_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    lu = nodes * steps
    return {"value": lu / dt / 1e9, "unit": "GLUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"instance 0 of the workload ({wk.dims[0][0]}x{wk.dims[0][1]}) x {steps} "
                      f"steps = {lu / 1e6:.1f} M LU in {dt:.1f} s, FP64 {collision.upper()}",
            "host_cpus": os.cpu_count()}


# ----------------------------------------------------------------------------
# The reference arm: the FP64 CPU oracle.
# ----------------------------------------------------------------------------
def run_reference(args, dist):
    if dist.rank != 0:
        return 0
    import oracle
    oracle.build()
    wk = Workload(args.workload, 0, 1)
    # per-step sample: instance 0's parameters on a lattice sized so that the
    # whole --steps/--warmup run takes about two minutes on the host cores
    probe, pn = _oracle_sim(wk, 0, nx=128 if wk.lattice == "d2q9" else 4096,
                            collision=args.collision)
    t0 = time.perf_counter()
    probe.step(3)
    rate = 3 * pn / (time.perf_counter() - t0)
    per_step_s = 120.0 / max(args.steps + args.warmup, 1)
    want = rate * per_step_s
    if wk.lattice == "d2q9":
        size = int(max(16, min(wk.dims[0][0], math.sqrt(want))))
    else:
        size = int(max(64, min(wk.dims[0][0], want)))
    sim, nodes = _oracle_sim(wk, 0, nx=size, collision=args.collision)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    value = nodes * args.steps / dt / 1e9
    sample = (f"instance 0's parameters on {nodes} nodes per step (bounded sample of the "
              f"{wk.nodes}-node workload), FP64 {args.collision.upper()} on {oracle.num_threads()} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_for(args, wk, None),
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_for(args, wk, lat):
    c = {
        "workload": WORKLOADS[wk.name] + f"; {args.collision.upper()}, {args.compute.upper()} collide, "
                    f"{args.storage.upper()} deviation storage, CUDA-graph step loop",
        "instances_per_gpu": len(wk.dims),
        "nodes_per_gpu": wk.nodes,
        "lattice": wk.lattice,
        "compute": args.compute,
        "storage": args.storage,
        "collision": args.collision,
        "conservation_every": CONS_EVERY,
        "l2": ("inputs larger than L2 (two population copies, no flush needed)"
               if 2 * wk.nodes * wk.bytes_per_lu(args.storage) // 2 > 129e6 else
               "L2-resident working set (not an HBM measurement)"),
    }
    if lat is not None:
        c["launch_shape"] = lat.launch_shape()
    return c


# ----------------------------------------------------------------------------
# Our arm.
# ----------------------------------------------------------------------------
def run_ours(args, dist):
    import torch

    import __graft_entry__
    __graft_entry__.build()

    torch.cuda.set_device(dist.local)
    wk = Workload(args.workload, dist.rank, dist.world)
    lat = wk.lattice_obj(args.compute, args.storage, args.collision)
    stream = lat.stream
    cons = torch.empty(3 * len(wk.dims), dtype=torch.float64, device="cuda")

    lat.init(*wk.fields())
    lat.step(max(args.warmup, 3))
    lat.conservation_device(cons)
    torch.cuda.synchronize()

    sampler = ClockSampler(dist.local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    chunks = []
    k = args.steps
    while k > 0:
        c = min(CONS_EVERY, k)
        chunks.append(c)
        k -= c
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in chunks]
    dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for c, (ea, eb) in zip(chunks, step_ev):
        ea.record(stream)
        lat.step(c)
        eb.record(stream)
        lat.conservation_device(cons)
    ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    dist.barrier()
    sampler.stop()
    t_ms = ev0.elapsed_time(ev1)
    step_ms = sum(a.elapsed_time(b) for a, b in step_ev)
    st = lat.status()

    t_max = dist.reduce(t_ms, "max")
    total_lu = dist.reduce(float(wk.nodes) * args.steps, "sum")
    value = total_lu / (t_max * 1e-3) / 1e9

    peak, peak_kind = measured_peaks()
    bpl = wk.bytes_per_lu(args.storage)
    launch_ms = step_ms / args.steps
    achieved = wk.nodes * bpl / (launch_ms * 1e-3) / 1e9
    shape = lat.launch_shape()
    tpn = traffic_per_node(f"{wk.name}:{args.collision}:{args.storage}", shape["kind"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": None if tpn is None else tpn * wk.nodes,
                "algorithmic_bytes_per_launch": wk.nodes * bpl,
                "kernel": f"lbm step kernel ({shape['kind']}) {wk.lattice.upper()} "
                          f"{args.storage} storage, {args.compute} compute, "
                          f"{args.collision.upper()}",
                "avg_launch_ms": launch_ms}

    # the sharded path's one collective: every rank gets every member's
    # conservation totals (ensembles; single-instance runs are replicas)
    totals = None
    if wk.total_members > 1 or dist.world == 1:
        from paper_1801_03863_gb300.partition import gather_totals
        table = gather_totals(cons.view(-1, 3).cpu().numpy(), wk.member_ids, wk.total_members,
                              dist.pg)
        totals = {"members": int(table.shape[0]), "sum_rho": float(table[:, 0].sum()),
                  "sum_rho_u": [float(table[:, 1].sum()), float(table[:, 2].sum())]}

    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.compute, "data": "synthetic", "config": config_for(args, wk, lat),
        "roofline": roofline,
        "gpu_launches": args.steps + 2 * len(chunks),
        "clocks": sampler.summary(),
        "status": st,
        "totals": totals,
    }

    if not args.no_extras and dist.rank == 0:
        line["e2e"] = e2e_leg(args, lat, wk)
        if wk.lattice == "d2q9":
            line["fp64_plain"] = fp64_plain_leg(args.collision)
        if args.compute == "f32":
            line["error_vs_fp64"] = error_leg(args, wk)
        if dist.world == 1:
            line["cpu_baseline"] = cpu_oracle_sample(wk, args.collision)
    lat.close()
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def e2e_leg(args, lat, wk):
    """Same K steps through the public C ABI with host buffers: upload of the
    initial fields from pinned memory, the step loop with the conservation
    totals read to the host every CONS_EVERY steps (as in the device-timed
    loop), read-back of rho and u."""
    import torch

    from paper_1801_03863_gb300 import lbm
    n = wk.nodes
    nf = 3 if wk.q == 9 else 2
    pin = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2 * nf)]
    for j, a in enumerate(wk.fields()):
        pin[j].numpy()[:] = a
    count = len(wk.dims)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_init(lat._h, *[pin[j].numpy() for j in range(nf)])
    k, chunks = args.steps, 0
    while k > 0:
        c = min(CONS_EVERY, k)
        lbm.lbm_step(lat._h, c)
        lbm.lbm_conservation(lat._h, count)
        k -= c
        chunks += 1
    code = lbm.load().lbm_moments(lat._h, pin[nf].data_ptr(), pin[nf + 1].data_ptr(),
                                  pin[nf + 2].data_ptr() if nf == 3 else None)
    dt = time.perf_counter() - t0
    lbm._check(code, "lbm_moments", allow_unstable=True)
    return {"value": n * args.steps / dt / 1e9, "unit": "GLUPS",
            "h2d_bytes_per_step": nf * 8 * n / args.steps,
            "d2h_bytes_per_step": (nf * 8 * n + chunks * 3 * 8 * count) / args.steps,
            "note": "lbm_init from pinned host arrays + lbm_step(K) with lbm_conservation to the "
                    "host every %d steps + lbm_moments to pinned host" % CONS_EVERY}


def fp64_plain_leg(collision: str, steps: int = 20):
    """The plain FP64 single-instance kernel: one 2048^2 cavity, Re 5000, U 0.1."""
    import torch
    wk = Workload("cavity2048", 0, 1)
    with wk.lattice_obj("f64", "f64", collision) as lat:
        lat.init(*wk.fields())
        lat.step(3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(lat.stream)
        lat.step(steps)
        e1.record(lat.stream)
        lat.stream.synchronize()
        ms = e0.elapsed_time(e1) / steps
        shape = lat.launch_shape()
    peak, _ = measured_peaks()
    glups = wk.nodes / (ms * 1e-3) / 1e9
    return {"workload": WORKLOADS["cavity2048"] + f"; {collision.upper()}, FP64 collide and storage",
            "value": glups, "unit": "GLUPS", "ms_per_step": ms,
            "hbm_frac": glups * 1e9 * wk.bytes_per_lu("f64") / (peak * 1e9), "launch_shape": shape}


def error_leg(args, wk, steps: int = 100):
    """rho/u error of the benchmarked precision against an FP64 run of the same
    workload after `steps` steps (relative L2 / Linf over all nodes)."""
    res = {}
    for comp, stor in (("f64", "f64"), (args.compute, args.storage)):
        lat = wk.lattice_obj(comp, stor, args.collision)
        lat.init(*wk.fields())
        lat.step(steps)
        r, x, y = lat.moments(allow_unstable=True)
        res[comp] = (r, x, np.zeros_like(x) if y is None else y, lat.status())
        lat.close()
    r0, x0, y0, st0 = res["f64"]
    r1, x1, y1, st = res[args.compute]
    u0 = np.sqrt(x0 * x0 + y0 * y0)
    du = np.sqrt((x1 - x0) ** 2 + (y1 - y0) ** 2)
    return {"steps": steps, "storage": args.storage,
            "rho_linf_rel": float(np.abs(r1 - r0).max() / np.abs(r0).max()),
            "rho_l2_rel": float(np.linalg.norm(r1 - r0) / np.linalg.norm(r0)),
            "u_linf_rel": float(du.max() / max(u0.max(), 1e-300)),
            "u_l2_rel": float(np.linalg.norm(du) / max(np.linalg.norm(u0), 1e-300)),
            "unstable_nodes": st["unstable"], "unstable_nodes_fp64": st0["unstable"]}


def main():
    args = parse()
    if args.storage is None:
        args.storage = "f64" if args.compute == "f64" else DEFAULT_STORAGE[args.workload]
    dist = Dist()
    try:
        if args.impl == "reference":
            return run_reference(args, dist)
        return run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
