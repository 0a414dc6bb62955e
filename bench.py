#!/usr/bin/env python
"""Benchmark of the nodal-density hot path on GB300.

One step = one pass of the path over one batch of nodes of the bulk
workload (1,024-atom hcp Mg-like cell, 96x96x160 grid, 8th-order FD,
Gaussian projectors, P = 16 poles, 33^3 regions, mixed precision): Fermi
poles on the spectral interval, the cost-sorted work list, every
(node, pole) COCG solve, and the pole-weighted density and band-energy
accumulation.  Successive steps take successive node batches of the
workload (4,096 nodes in all).

Prints one JSON line (rank 0):
  value    (node, pole) solves/s over the timed steps, device-resident
           inputs (Hamiltonian built before the timed region);
  e2e      the same metric through the C ABI from host buffers: every step
           builds the Hamiltonian from host arrays, solves, and copies rho
           and e back to the host;
  roofline HBM roofline of the solver kernel: algorithmic bytes (80 B per
           region point per COCG iteration in mixed mode, 160 B in FP64)
           / the kernel's CUDA-event time, against the measured copy
           bandwidth;
  cpu_baseline  the FP64 oracle (plain C, OpenMP) on a bounded sample.
--impl reference times the oracle itself as the reference arm.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(node,pole) solves/sec and density nodes/sec at rel err<=1e-6; matvec HBM GB/s"
BYTES_PER_POINT_ITER = {"mixed": 80.0, "fp64": 160.0}
# DRAM bytes (read + write) per region-point iteration of the solver kernel,
# from one ncu capture of a full bench launch (summary under profiles/:
# kernel k_cocg, bulk workload, one 256-node x 16-pole batch, 512 x 3),
# keyed by workload, precision and launch shape (threads per CTA, CTAs per
# SM), scaled to a launch by its region-point iterations.  Valid only for
# the kernel sources with the fingerprint below; any change to them makes
# the figure stale (null).
TRAFFIC_PER_POINT_ITER = {("bulk_mixed", "mixed", 512, 3): 130.0}
TRAFFIC_SOURCES = ("paper_1907_02604_gb300/csrc/md_solver.cu", "paper_1907_02604_gb300/csrc/md_solver.h",
                   "paper_1907_02604_gb300/csrc/md_device.cuh", "paper_1907_02604_gb300/csrc/md_internal.h",
                   "paper_1907_02604_gb300/csrc/md_operator.cuh")
TRAFFIC_FINGERPRINT = "53842885215939a9:0a35456717bedd0f:6685de8068da134b:6a946dc70a5a74c8:325f5235402aed53"
# FP64 operations (a multiply-add counted as two) per region point and COCG
# iteration of the FP64 form at 8th order with projectors: stencil 12 offset
# pairs x 6 = 72, diagonal 8, projector apply 24 and coefficients 12 (1.5
# atoms per point), p update 8, x and r updates 16, r^T r and ||r||^2 8, p^T Ap 8
FP64_FLOPS_PER_POINT_ITER = 156.0
L2_FLUSH_BYTES = 256 << 20   # written between timed steps: twice the 129 MB L2
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, vendor figure (context beside the measured copy peak)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bulk_mixed")
    ap.add_argument("--nodes-per-step", type=int, default=256)
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--kernel", default="auto", choices=["auto", "generic", "zmarch", "cluster"],
                    help="solver kernel (auto: the autotuner's choice)")
    ap.add_argument("--maxit", type=int, default=0, help="iteration cap (profiling runs)")
    ap.add_argument("--reliable-delta", type=float, default=0.0,
                    help="mixed precision: residual drop between FP64 residual refreshes (0 = library default)")
    ap.add_argument("--reliable-every", type=int, default=0,
                    help="mixed precision: most iterations between refreshes (0 = library default)")
    ap.add_argument("--method", default="cocg", choices=["cocg", "shifted"])
    ap.add_argument("--no-shifted", action="store_true", help="skip the shifted-COCG side measurement")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip the FP64-form side measurement")
    ap.add_argument("--no-lssgq", action="store_true", help="skip the Lanczos-quadrature side measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint side measurement")
    ap.add_argument("--no-screw", action="store_true", help="skip the batched uneven (screw) side measurement")
    ap.add_argument("--locality", default="", metavar="S1,S2,...",
                    help="print the locality report (rho_j against region half-width s) instead of timing")
    ap.add_argument("--locality-nodes", type=int, default=16)
    ap.add_argument("--large-pass", action="store_true",
                    help="report one full pass of the workload (every node, fused band-energy forces) instead of timing")
    return ap.parse_args()


def kernel_fingerprint():
    import hashlib
    parts = []
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            parts.append(hashlib.sha256(fh.read()).hexdigest()[:16])
    return ":".join(parts)


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def oracle_sample(w, timed, bar, target_s=20.0):
    """The oracle on a bounded sample of the timed batches' nodes (all poles
    of each): its solve rate on the host cores (the CPU baseline), and the
    error of the timed GPU densities and band energies against it on those
    nodes (max |d| / max |oracle| over the sample, and per node where
    rho_j > 1e-3 max rho).  `timed`: (node indices into the workload, GPU
    rho, GPU e) per distinct timed batch; chunks of nodes doubling up to 16 are
    taken from the batches in turn, starting at a quarter of the host threads
    (so that every thread has systems to take from the first chunk on)."""
    from oracle import density as od
    H = od.build(w)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t_used, solves, n_done = 0.0, 0, 0
    cursor = [0] * len(timed)
    k, b = max(1, min(16, threads // 4)), 0
    g_rho, g_e, o_rho, o_e = [], [], [], []
    while t_used < target_s and any(c < len(t[0]) for c, t in zip(cursor, timed)):
        j = b % len(timed)
        b += 1
        idx, rho_g, e_g = timed[j]
        c = cursor[j]
        if c >= len(idx):
            continue
        take = np.arange(c, min(c + k, len(idx)))
        cursor[j] = take[-1] + 1
        t0 = time.perf_counter()
        res = od.solve(w.subset(idx[take]), H, tol=w.tol)
        t_used += time.perf_counter() - t0
        n_done += len(take)
        solves += len(take) * w.n_poles
        g_rho.append(rho_g[take])
        g_e.append(e_g[take])
        o_rho.append(res.rho)
        o_e.append(res.e_node)
        k = min(2 * k, 16)
    cpu = {"value": solves / t_used, "unit": "solves/s", "cores": threads, "kind": "oracle",
           "sample": f"{n_done} nodes x {w.n_poles} poles of the timed batches of {w.name} "
                     f"(FP64 COCG, tol {w.tol:g}), {t_used:.1f} s"}
    gr, ge, orr, oe = (np.concatenate(a) for a in (g_rho, g_e, o_rho, o_e))
    keep = np.abs(orr) > 1e-3 * np.abs(orr).max()
    parity = {"nodes": int(len(orr)), "systems": int(len(orr) * w.n_poles),
              "max_rel_err_rho": float(np.abs(gr - orr).max() / np.abs(orr).max()),
              "max_rel_err_e": float(np.abs(ge - oe).max() / np.abs(oe).max()),
              "per_node_max_rel_err_rho": float((np.abs(gr - orr)[keep] / np.abs(orr)[keep]).max()),
              "bar": bar, "reference": "FP64 oracle (plain C COCG) on the same nodes of the timed batches"}
    parity["pass"] = bool(max(parity["max_rel_err_rho"], parity["max_rel_err_e"]) <= bar)
    return cpu, parity


def workload_config(w, bs, prec):
    """The workload part of the line's config, shared by both arms."""
    lo, hi = int(w.halfwidth.min()), int(w.halfwidth.max())
    region = f"{2 * lo + 1}^3" if lo == hi else f"{2 * lo + 1}^3..{2 * hi + 1}^3"
    return {"workload": w.name, "nodes_per_step": bs, "poles": w.n_poles, "region": region,
            "grid": list(w.shape), "atoms": len(w.atoms), "fd_order": w.fd_order, "precision": prec,
            "tol": w.tol}


def run_reference(args, world, rank):
    if rank != 0:
        return
    from synthetic import make_workload
    from oracle import _native
    _native.build()
    w = make_workload(args.workload)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # each step: a batch of nodes (all poles) of the same workload, as many as
    # keep the whole run near 200 s, but at least enough systems for every
    # host thread to take several (the oracle runs its systems in parallel)
    from oracle import density as od
    H = od.build(w)
    calib = max(1, threads // 4)
    t = time.perf_counter()
    od.solve(w.subset(np.arange(calib)), H, tol=w.tol)
    per_node = (time.perf_counter() - t) / calib
    per_step_nodes = int(200.0 / max(args.steps + args.warmup, 1) / max(per_node, 1e-3))
    per_step_nodes = max(max(1, threads // 4), min(per_step_nodes, 4 * threads))
    cursor = calib
    for _ in range(args.warmup):
        od.solve(w.subset(np.arange(cursor, cursor + per_step_nodes) % len(w.nodes)), H, tol=w.tol)
        cursor += per_step_nodes
    t0 = time.perf_counter()
    for _ in range(args.steps):
        od.solve(w.subset(np.arange(cursor, cursor + per_step_nodes) % len(w.nodes)), H, tol=w.tol)
        cursor += per_step_nodes
    el = time.perf_counter() - t0
    solves = args.steps * per_step_nodes * w.n_poles
    val = solves / el
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(w, min(args.nodes_per_step, len(w.nodes)), args.precision or w.precision),
           "cpu_baseline": {"value": val, "unit": "solves/s", "cores": threads, "kind": "oracle",
                            "sample": f"{per_step_nodes} nodes x {w.n_poles} poles per step of {w.name} "
                                      f"({per_step_nodes * w.n_poles} systems over {threads} threads)"},
           "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_locality(args, rank, local):
    """rho_j and e_j of the same nodes as the region half-width s grows (the
    analogue of the paper's convergence of the nodal fields with cluster
    size, Section 4), FP64 solves at tol 1e-10, each s reported against the
    largest: the truncation error of the local evaluation, not a parity
    figure.  Rank 0 only."""
    if rank != 0:
        return
    import torch
    torch.cuda.set_device(local)
    from synthetic import make_workload
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density, make_poles
    w = make_workload(args.workload)
    s_list = sorted({int(t) for t in args.locality.split(",")})
    c = w.node_coords()
    ok = np.ones(len(w.nodes), bool)
    for d in range(3):   # every region inside the open axes at the largest s
        if not w.periodic[d]:
            ok &= (c[:, d] - s_list[-1] >= 0) & (c[:, d] + s_list[-1] < w.shape[d])
    nodes = w.nodes[np.nonzero(ok)[0][:args.locality_nodes]]
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    res = {}
    for s in s_list:
        hw = np.full(len(nodes), s, np.int32)
        rho, e, st = density(ham, z, wt, nodes, hw, SolverOptions(tol=1e-10, precision="fp64"), energy=True)
        res[s] = (rho.cpu().numpy(), e.cpu().numpy(), st)
    r_ref, e_ref, _ = res[s_list[-1]]
    curve = []
    for s in s_list:
        rho, e, st = res[s]
        dims = [w.shape[d] if (w.periodic[d] and 2 * s + 1 >= w.shape[d]) else 2 * s + 1 for d in range(3)]
        curve.append({"s": s, "region": "x".join(map(str, dims)),
                      "rho_max_rel_diff": float(np.abs(rho - r_ref).max() / np.abs(r_ref).max()),
                      "e_max_rel_diff": float(np.abs(e - e_ref).max() / np.abs(e_ref).max()),
                      "iters_mean": float(st["iters_mean"]), "converged": int(st["n_converged"])})
    print(json.dumps({"report": "locality", "workload": w.name, "nodes": len(nodes), "poles": w.n_poles,
                      "precision": "fp64", "tol": 1e-10, "reference_s": s_list[-1], "curve": curve}), flush=True)


def run_large_pass(args, rank, local):
    """One full pass of the large configuration: every node (about 200,000)
    x 16 poles in mixed precision through the fused adjoint with the
    band-energy loss (L = E_band: a = 0, b = 1), streamed in batches of
    --nodes-per-step nodes; the band energy, the converged count and the
    Hellmann-Feynman forces summed over the batches (forces are linear in
    dL/dV), reported on the 2,000 sites nearest the loop line.  A report,
    not the benchmark line.  Rank 0 only."""
    if rank != 0:
        return
    import torch
    torch.cuda.set_device(local)
    from synthetic import make_workload
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density_fused_adjoint, make_poles
    w = make_workload(args.workload)
    t0 = time.perf_counter()
    ham = Hamiltonian.from_workload(w)
    lo, hi = ham.spectral_bounds()
    z, wt = make_poles(w.kT, w.mu, lo, hi, w.n_poles)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    opts = SolverOptions(tol=w.tol, maxit=w.maxit, precision="mixed")
    bs = args.nodes_per_step
    F = torch.zeros((len(w.atoms), 3), dtype=torch.float64, device="cuda")
    e_band = 0.0
    conv = systems = point_iters = iters = 0
    t1 = time.perf_counter()
    for b0 in range(0, len(w.nodes), bs):
        nd, hw = w.nodes[b0:b0 + bs], w.halfwidth[b0:b0 + bs]
        ones = torch.ones(len(nd), dtype=torch.float64, device="cuda")
        _, e, _, Fb, st = density_fused_adjoint(ham, z, wt, nd, hw, None, ones, opts, forces=True)
        F += Fb
        e_band += float(e.sum().item())
        conv += st["n_converged"]
        systems += st["n_systems"]
        point_iters += st["total_point_iters"]
        iters += st["total_iters"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t1
    sel = F[torch.as_tensor(w.meta["force_atoms"], device="cuda")].cpu().numpy()
    print(json.dumps({"report": "large_pass", "workload": w.name, "nodes": int(len(w.nodes)), "poles": w.n_poles,
                      "systems": systems, "converged": conv, "iters_mean": iters / max(systems, 1),
                      "grid": list(w.shape), "atoms": int(len(w.atoms)), "precision": "mixed", "tol": w.tol,
                      "batch_nodes": bs, "hamiltonian_build_s": t_build, "wall_s": wall,
                      "solves_per_s": systems / wall, "point_iters_per_s": point_iters / wall,
                      "e_band": e_band, "force_atoms": int(len(sel)),
                      "force_norm": float(np.linalg.norm(sel)), "force_max_abs": float(np.abs(sel).max()),
                      "loss": "band energy (fused adjoint, no checkpoint)"}), flush=True)


def main():
    args = parse()
    world, rank, local, dist = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.locality:
        run_locality(args, rank, local)
        return
    if args.large_pass:
        run_large_pass(args, rank, local)
        return
    import torch
    torch.cuda.set_device(local)
    from synthetic import make_workload
    from paper_1907_02604_gb300 import Hamiltonian, Plan, SolverOptions, density, make_poles
    from paper_1907_02604_gb300.sharding import (batch_slice, gather_nodes, node_cost, partition_nodes,
                                                 rank_batch)

    w = make_workload(args.workload)
    prec = args.precision or w.precision
    n_nodes = len(w.nodes)
    bs = min(args.nodes_per_step, n_nodes)
    n_batches = max(1, n_nodes // bs)
    opts = SolverOptions(tol=w.tol, maxit=args.maxit or w.maxit, precision=prec, block=args.block,
                         ctas_per_sm=args.ctas_per_sm, method=args.method, kernel=args.kernel,
                         reliable_delta=args.reliable_delta, reliable_every=args.reliable_every)
    stream = torch.cuda.current_stream()

    # one rank: consecutive batches of the node list; several ranks: each
    # takes its share of a cost-balanced partition (all poles of a node on
    # one rank), in batches of bs nodes
    parts, _ = partition_nodes(node_cost(w.halfwidth), world)

    def batch_idx(i, r=rank):
        if world == 1:
            return np.arange(n_nodes)[batch_slice(n_nodes, bs, 1, 0, i)]
        return rank_batch(parts[r], bs, i)

    def batch(i):
        idx = batch_idx(i)
        return w.nodes[idx], w.halfwidth[idx]

    # ---- device-resident inputs: Hamiltonian built and batches planned -----
    # before timing; a step replays one batch's CUDA graph (solver + pole
    # accumulation).
    ham = Hamiltonian.from_workload(w)
    lo, hi = ham.spectral_bounds()
    z, wt = make_poles(w.kT, w.mu, lo, hi, w.n_poles)
    # the expansion error r - f on the spectral interval: parity targets r
    # (both sides use the same poles); this is how far r is from the exact
    # Fermi-Dirac function at this P
    eg = np.linspace(lo, hi, 100001)
    r_eg = np.imag(wt[None, :] / (eg[:, None] - z[None, :])).sum(axis=1)
    f_eg = 0.5 * (1.0 - np.tanh(0.5 * (eg - w.mu) / w.kT))
    expansion = {"P": w.n_poles, "max_abs_r_minus_f": float(np.abs(r_eg - f_eg).max()),
                 "interval": [float(lo), float(hi)], "kT": w.kT, "mu": w.mu}
    n_plans = min(n_batches, args.warmup + args.steps)
    plans = []
    for i in range(n_plans):
        nd, hw = batch(i)
        plans.append(Plan(ham, z, wt, nd, hw, opts, energy=True, stream=stream))

    def plan_of(i):
        return plans[i % n_plans]

    for i in range(args.warmup):
        plan_of(i).launch(stream)
        plan_of(i).stats(stream, strict=False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(args.steps):
        if i:
            flush.zero_()   # no step starts with the previous step's data in L2
        plan_of(args.warmup + i).launch(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    el_ms = ev0.elapsed_time(ev1)
    # per-step statistics (a plan replayed in the timed region repeats the
    # same solves, so its last launch stands for each of its launches)
    stats = [plan_of(args.warmup + i).stats(stream, strict=False) for i in range(args.steps)]
    gathered = None
    if dist:
        t = torch.tensor([el_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el_ms = float(t.item())
        dist.barrier()
        # after the timed region: the densities of every rank's timed batches
        # gathered into one node vector (the only exchange the path has)
        timed_j = sorted({(args.warmup + i) % n_plans for i in range(args.steps)})
        tparts = [np.concatenate([batch_idx(j, r) for j in timed_j]) for r in range(world)]
        mine = torch.cat([plans[j].rho for j in timed_j])
        full = gather_nodes(mine, tparts, n_nodes)
        gathered = {"nodes": int(torch.isfinite(full).sum().item()), "expected": int(sum(len(p) for p in tparts)),
                    "collective": "all_gather of rho (NCCL), outside the timed region"}
    solves_rank = sum(s["n_systems"] for s in stats)
    total_solves = solves_rank * world
    value = total_solves / (el_ms / 1e3)
    kernel_ms = sum(s["kernel_ms"] for s in stats)
    point_iters = sum(s["total_point_iters"] for s in stats)
    conv = sum(s["n_converged"] for s in stats)
    B = BYTES_PER_POINT_ITER[prec]
    achieved = point_iters * B / (kernel_ms / 1e3) / 1e9
    shape = plans[0].launch_shape()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    per_sm = shape[1] // n_sm if shape[1] % n_sm == 0 else 0
    tkey = (w.name, prec, shape[0], per_sm)
    traffic = None
    if tkey in TRAFFIC_PER_POINT_ITER and kernel_fingerprint() == TRAFFIC_FINGERPRINT:
        traffic = TRAFFIC_PER_POINT_ITER[tkey] * point_iters / len(stats)   # bytes per launch
    peak, peak_kind = read_peaks()

    from dataclasses import replace as _replace

    def side(sopts, note):
        """The same steps with other solver options; density compared with
        the timed run's on the same batches."""
        splans = [Plan(ham, z, wt, *batch(i), sopts, energy=True, stream=stream) for i in range(n_plans)]
        for i in range(args.warmup):
            splans[i % n_plans].launch(stream)
            splans[i % n_plans].stats(stream, strict=False)
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for i in range(args.steps):
            splans[(args.warmup + i) % n_plans].launch(stream)
        s1.record(stream)
        torch.cuda.synchronize()
        sms = s0.elapsed_time(s1)
        sst = [splans[(args.warmup + i) % n_plans].stats(stream, strict=False) for i in range(args.steps)]
        diff = 0.0
        for i in range(args.steps):
            a = splans[(args.warmup + i) % n_plans].rho
            b = plan_of(args.warmup + i).rho
            diff = max(diff, float((a - b).abs().max() / b.abs().max()))
        out = {"value": sum(x["n_systems"] for x in sst) * world / (sms / 1e3), "unit": "solves/s",
               "ms_per_step": sms / args.steps,
               "converged": f"{sum(x['n_converged'] for x in sst)}/{sum(x['n_systems'] for x in sst)}",
               "point_iters_per_s": sum(x["total_point_iters"] for x in sst) * world / (sms / 1e3),
               "max_rel_diff_rho_vs_timed": diff, "note": note,
               "kernel_ms": sum(x["kernel_ms"] for x in sst),
               "point_iters": sum(x["total_point_iters"] for x in sst)}
        for sp in splans:
            sp.close()
        return out

    # ---- side measurements: shifted COCG, and the plain FP64 form ----------
    shifted = fp64_form = None
    if args.method == "cocg" and not args.no_shifted:
        shifted = side(_replace(opts, method="shifted", block=0, ctas_per_sm=0),
                       "method 1: per node one Krylov sequence serves all poles (density only)")
    if prec == "mixed" and not args.no_fp64_form:
        fp64_form = side(_replace(opts, precision="fp64", block=0, ctas_per_sm=0),
                         "per-pole COCG with FP64 vectors; speedup = value / this value")
        fp64_form["speedup_mixed_over_fp64"] = value / fp64_form["value"]
        # its roofline: FP64 operations per region-point iteration over the
        # solver kernel's time, against this GPU's FP64 FMA rate measured now
        # (md_fma_rate: bounded FMA chains on every SM)
        from paper_1907_02604_gb300 import fma_rate
        peak64 = fma_rate("fp64", stream)
        ach64 = FP64_FLOPS_PER_POINT_ITER * fp64_form["point_iters"] / (fp64_form["kernel_ms"] / 1e3) / 1e12
        fp64_form["roofline"] = {"bound": "fp64", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                                 "frac": ach64 / peak64, "flops_per_point_iter": FP64_FLOPS_PER_POINT_ITER,
                                 "peak_kind": "measured (md_fma_rate, FP64 FMA chains)"}

    # ---- side measurement: the batched uneven workload, all 1,250 nodes x
    # 16 poles (20,000 systems, regions 17^3..41^3) in one graph launch ----
    screw = None
    if not args.no_screw and w.name != "screw_batched":
        ws_ = make_workload("screw_batched")
        ham_s = Hamiltonian.from_workload(ws_, stream=stream)
        zs, wts_ = make_poles(ws_.kT, ws_.mu, *ham_s.spectral_bounds(stream=stream), ws_.n_poles)
        ps_ = Plan(ham_s, zs, wts_, ws_.nodes, ws_.halfwidth,
                   SolverOptions(tol=ws_.tol, maxit=ws_.maxit, precision="mixed"), energy=True, stream=stream)
        ps_.launch(stream)
        ps_.stats(stream, strict=False)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        ps_.launch(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        sst = ps_.stats(stream, strict=False)
        sms = t0.elapsed_time(t1)
        shp = ps_.launch_shape()
        screw = {"workload": ws_.name, "systems": sst["n_systems"], "value": sst["n_systems"] / (sms / 1e3),
                 "unit": "solves/s", "launch_ms": sms, "converged": f"{sst['n_converged']}/{sst['n_systems']}",
                 "iters_mean": sst["iters_mean"], "point_iters_per_s": sst["total_point_iters"] / (sms / 1e3),
                 "launch_shape": {"threads_per_cta": shp[0], "ctas": shp[1]},
                 "note": "one graph-captured persistent launch of every system, after one warm-up launch"}
        ps_.close()
        ham_s.close()

    # ---- side measurement: the paper's Lanczos quadrature (Eq. 9, K = 40) --
    # in FP64 and with FP32 vectors; the mixed densities are compared with
    # the FP64 ones on the same batches
    lssgq = None
    if not args.no_lssgq:
        from paper_1907_02604_gb300 import lssgq_rules
        K = 40

        def lssgq_run(precision):
            def step(i):
                nd, hw = batch(i)
                R = lssgq_rules(ham, nd, hw, K=K, precision=precision, stream=stream)
                rho, _, _ = R.fields(w.mu, w.kT, stream=stream)
                return R, rho

            for i in range(args.warmup):
                step(i)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = [step(args.warmup + i) for i in range(args.steps)]
            torch.cuda.synchronize()
            return out, time.perf_counter() - t0

        pts = sum(int(np.sum((2 * batch(args.warmup + i)[1].astype(np.int64) + 1) ** 3)) for i in range(args.steps))
        lssgq = {}
        ref = None
        for precision in ("fp64", "mixed"):
            out, el = lssgq_run(precision)
            entry = {"value": sum(R.n_nodes for R, _ in out) * world / el, "unit": "density nodes/s",
                     "K": K, "ms_per_step": 1e3 * el / args.steps,
                     "point_iters_per_s": pts * K * world / el,
                     "lanczos_steps": sum(int(R.k_used.sum()) for R, _ in out)}
            if ref is None:
                ref = [rho for _, rho in out]
            else:
                entry["max_rel_diff_rho_vs_fp64"] = max(float((rho - r).abs().max() / r.abs().max())
                                                        for (_, rho), r in zip(out, ref))
                entry["accuracy"] = ("FP32 Lanczos vectors: the rule nodes carry ~2^-24 max|lambda| absolute "
                                     "error, which the Fermi factor (slope 1/(4 kT)) turns into density errors "
                                     "of order 1e-5..1e-4 at kT = 0.01 Ha; this form does not meet the 1e-5 "
                                     "mixed-precision bar and is a speed figure only")
            lssgq[precision] = entry
        lssgq["note"] = ("Lanczos Gauss rules + fields at (mu, kT); host-timed, includes the per-call "
                         "work-list upload and status read-back")

    # ---- side measurement: the adjoint (dL/dV and forces) on the adjoint ---
    # workload in FP64: the forward solve keeping a checkpoint, the
    # checkpointed adjoint pass, and the fused one-pass form (host-timed
    # calls, like the LSSGQ figures)
    adjoint = None
    if not args.no_adjoint:
        from paper_1907_02604_gb300 import Workspace, density_adjoint, density_fused_adjoint
        wa = make_workload("adjoint_fp64")
        sl = batch_slice(len(wa.nodes), min(32, len(wa.nodes)), world, rank, 0)
        nd_a, hw_a = wa.nodes[sl], wa.halfwidth[sl]
        ham_a = Hamiltonian.from_workload(wa, stream=stream)
        za, wta = make_poles(wa.kT, wa.mu, *ham_a.spectral_bounds(stream=stream), wa.n_poles)
        opts_a = SolverOptions(tol=wa.tol, maxit=wa.maxit, precision="fp64")
        ones = torch.ones(len(nd_a), dtype=torch.float64, device="cuda")
        ws = Workspace(ham_a, nd_a, hw_a, wa.n_poles)

        def fwd():
            return density(ham_a, za, wta, nd_a, hw_a, opts_a, energy=True, checkpoint=ws, stream=stream)

        def adj():
            return density_adjoint(ham_a, za, wta, nd_a, hw_a, ones, ones, opts_a, checkpoint=ws, forces=True,
                                   stream=stream)

        def fused():
            return density_fused_adjoint(ham_a, za, wta, nd_a, hw_a, ones, ones, opts_a, forces=True, stream=stream)

        def timed(fn):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            return out, time.perf_counter() - t0

        fwd(), adj(), fused()   # warm-up
        _, t_fwd = timed(fwd)
        (g_c, F_c), t_adj = timed(adj)
        (_, _, g_f, F_f, _), t_fused = timed(fused)
        pts = int(np.sum((2 * hw_a.astype(np.int64) + 1) ** 3))
        adjoint = {"workload": wa.name, "systems": len(nd_a) * wa.n_poles, "precision": "fp64",
                   "forward_with_checkpoint_ms": 1e3 * t_fwd, "adjoint_pass_ms": 1e3 * t_adj,
                   "fused_forward_adjoint_ms": 1e3 * t_fused, "adjoint_over_forward": t_adj / t_fwd,
                   "adjoint_checkpoint_read_GB_s": pts * wa.n_poles * 16 / t_adj / 1e9,
                   "max_rel_diff_dLdV_fused_vs_checkpointed": float((g_f - g_c).abs().max() / g_c.abs().max()),
                   "max_rel_diff_forces_fused_vs_checkpointed": float((F_f - F_c).abs().max() / F_c.abs().max()),
                   "note": "dL/drho = dL/de = 1 on every node, forces on every atom; host-timed calls"}
        ws.close()
        ham_a.close()

    # ---- end to end through the C ABI from host buffers -------------------
    e2e = None
    if not args.no_e2e:
        h2d = d2h = 0

        # the step's inputs sit in pinned host memory (numpy views of pinned
        # tensors reach the C ABI unchanged), and results come back into
        # pinned tensors
        import copy

        def pinned(a):
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

        wp = copy.copy(w)
        wp.v_ext, wp.atoms, wp.depth, wp.sigma = (pinned(w.v_ext), pinned(w.atoms), pinned(w.depth),
                                                  pinned(w.sigma))
        nodes_p, hw_p = pinned(w.nodes.astype(np.int64)), pinned(w.halfwidth.astype(np.int32))
        rho_h = torch.empty(bs, dtype=torch.float64).pin_memory()
        e_h = torch.empty(bs, dtype=torch.float64).pin_memory()

        def e2e_step(i):
            nonlocal h2d, d2h
            idx = batch_idx(i)
            nd, hw = nodes_p[idx], hw_p[idx]
            hm = Hamiltonian.from_workload(wp, stream=stream)
            l2, h2 = hm.spectral_bounds(stream=stream)
            z, wt = make_poles(w.kT, w.mu, l2, h2, w.n_poles)
            rho, e, st = density(hm, z, wt, nd, hw, opts, energy=True, stream=stream, strict=False)
            rho_h[:len(nd)].copy_(rho)
            e_h[:len(nd)].copy_(e)
            hm.close()
            h2d = (w.v_ext.nbytes + w.atoms.nbytes + w.depth.nbytes + w.sigma.nbytes
                   + nd.nbytes + hw.nbytes + 32 * w.n_poles)
            d2h = 2 * len(nd) * 8 + st["n_systems"] * 20
            return st["n_systems"]

        for i in range(min(args.warmup, 3)):
            e2e_step(i)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        n_e2e = sum(e2e_step(args.warmup + i) for i in range(args.steps))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if dist:
            t = torch.tensor([el], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": n_e2e * world / el, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = parity = None
    if not args.no_cpu and world == 1:
        timed = []
        for j in sorted({(args.warmup + i) % n_plans for i in range(args.steps)}):
            timed.append((batch_idx(j), plans[j].rho.cpu().numpy(), plans[j].e.cpu().numpy()))
        cpu, parity = oracle_sample(w, timed, 1e-5 if prec == "mixed" else 1e-6)
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": el_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if prec == "mixed" else "f64",
        "data": "synthetic",
        "config": {**workload_config(w, bs, prec),
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB written)",
                   "pole_expansion": expansion,
                   "parallelism": (f"nodes sharded over {world} GPU(s), no collective in the timed region"
                                   + ("; cost-balanced node partition" if world > 1 else ""))},
        "nodes_per_s": value / w.n_poles,
        "converged": f"{conv}/{solves_rank}",
        "iters_mean": float(np.mean([s["iters_mean"] for s in stats])),
        "refreshes_per_system": float(sum(s["reliable_updates"] for s in stats) / max(solves_rank, 1)),
        "point_iters_per_s": point_iters * world / (el_ms / 1e3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                     "algorithmic_bytes_per_launch": point_iters * B / len(stats),
                     "kernel": "k_cocg<MixedMode>" if prec == "mixed" else "k_cocg<FP64Mode>",
                     "bytes_per_point_iter": B, "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "parity": parity,
        "gather": gathered,
        "e2e": e2e,
        "shifted_cocg": shifted,
        "fp64_form": fp64_form,
        "screw_batched": screw,
        "lssgq": lssgq,
        "adjoint": adjoint,
        "gpu_launches": 2 * args.steps,
        "launch_shape": {"threads_per_cta": shape[0], "ctas": shape[1]},
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
