#!/usr/bin/env python3
"""Preconditioned solves/s (+ p50/p99 latency) of the multilevel smoothed
Schwarz FGMRES solver on one GB300 per rank.

A step is one whole solve for one parameter vector mu: assembly of J(mu) on
every level, the subdomain and coarsest factorisations, and FGMRES(30) with the
V-cycle preconditioner to rtol 1e-8.  Ranks solve independent parameters
(replicas, weak scaling); there is no data-path collective.

python bench.py [--gpus N --steps K --warmup W] [--impl msp|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "preconditioned solves/s + p50/p99 latency at rtol 1e-8: mixed/batched vs FP64"
UNIT = "solves/s"
# FP64 on GB300 runs on the SIMT pipe: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 SIMT: 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
DESCR = {
    "cube64_3lvl": "64^3/32^3/16^3 independently jittered Kuhn tet meshes (274,625 fine nodes, "
                   "1.57M tets), k(x;mu)=exp(sum_j mu_j 0.5 cos(pi a_j.x)), 512 subdomains per "
                   "smoothed level, overlap 2, nu=2, coarsest direct, FGMRES(30) rtol 1e-8, "
                   "one mu per step (16 sequential)",
    "cube16_3lvl": "16^3/8^3/4^3 jittered Kuhn meshes, 64/8 subdomains, overlap 2",
    "cube8_2lvl": "8^3/4^3 jittered Kuhn meshes, k=1, 8 subdomains, overlap 1",
    "p2cube32_3lvl": "quadratic (P2) elements, DoFs on the vertices and edge midpoints (N = (1,1,0,0)), on "
                     "32^3/16^3/8^3 jittered Kuhn meshes: 274,625 fine DoFs, 512 + 64 subdomains, overlap 1, "
                     "nu=2, P2 interpolation between the non-nested levels, coarsest direct, FGMRES(30) rtol 1e-8",
    "p2p1cube32_3lvl": "a quadratic (P2) field u and a linear (P1) field p on one mesh, coupled by k (u - p) "
                       "(N = (2,1,0,0)), on 32^3/16^3/8^3 jittered Kuhn meshes: 310,562 fine DoFs, field-split "
                       "transfers (P2 interpolation for u, P1 for p), 512 + 64 subdomains, overlap 1, nu=2, "
                       "coarsest direct, FGMRES(30) rtol 1e-8",
    "elast32_3lvl": "linear elasticity (three P1 displacement fields per vertex, Poisson ratio 0.3, "
                    "Young's modulus k(x;mu), unit body force along -z) on 32^3/16^3/8^3 jittered "
                    "Kuhn meshes: 107,811 fine DoFs, 64 + 8 subdomains, overlap 1, nu=2, field-split "
                    "P, coarsest direct, FGMRES(30) rtol 1e-8",
}


# ------------------------------------------------------- replicas (N > 1)
def max_over_ranks(x: float) -> float:
    """The maximum of a per-rank scalar over all ranks (x itself with one rank).
    NCCL reduces on the rank's GPU, gloo on the host."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_request(rank: int, i: int) -> int:
    """Request number (the seed of mu) of the i-th solve of replica `rank`:
    disjoint between ranks for i < 100000."""
    return rank * 100000 + i


def whole_job_rate(units_per_rank: int, world: int, ms_slowest: float) -> float:
    """Units of all ranks per second of the slowest rank."""
    return units_per_rank * world / (ms_slowest / 1e3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="msp", choices=["msp", "reference"])
    ap.add_argument("--workload", default="cube64_3lvl")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32", "bf16", "f64tc"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-f64tc", action="store_true",
                    help="skip the FP64 run whose factor products use the tensor cores (digit slices)")
    ap.add_argument("--no-mls", action="store_true",
                    help="skip the MLS-transfer variant (Section 3.2) of the same workload")
    ap.add_argument("--no-hbm", action="store_true",
                    help="skip the per-launch HBM figures of the fine-level SpMV and transfers")
    ap.add_argument("--no-precision-study", action="store_true",
                    help="skip the 96^3 L-shaped precision study (FP64 / FP32 / BF16 factors)")
    ap.add_argument("--no-elastic", action="store_true",
                    help="skip the linear-elasticity (three fields per vertex) object")
    ap.add_argument("--no-p2", action="store_true",
                    help="skip the quadratic-element (DoFs on vertices and edges) object")
    ap.add_argument("--no-ilu", action="store_true",
                    help="skip the ILU(2)/ILU(0) subdomain-solver variant (Section 4.4)")
    ap.add_argument("--no-literal", action="store_true",
                    help="skip the paper-literal Algorithm 2 and one-level RAS iteration study")
    ap.add_argument("--batch", type=int, default=4,
                    help="concurrent instances of the batched FP32-factor measurement")
    ap.add_argument("--serve", type=int, default=400,
                    help="requests served from the start of the three-hierarchy trace (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrivals per second")
    ap.add_argument("--serve-precision", default="bf16", choices=["f32", "bf16"],
                    help="subdomain factors of the served solves (FP64 outer loop)")
    ap.add_argument("--serve-trace", action="store_true",
                    help="also serve the full trace: 2000 requests at 200/s over 32^3, 64^3 and 128^3 hierarchies "
                         "(probabilities 0.5/0.35/0.15), 120 GB budget")
    ap.add_argument("--profile-ops", default=None,
                    help="profiling mode: run each of the comma-separated operators of the finest level once "
                         "(J, P, PT, RAS, factor) inside an NVTX range of that name, for single-kernel ncu "
                         "captures (ncu --nvtx --nvtx-include NAME/), print their algorithmic bytes and exit")
    ap.add_argument("--cpu-sample", type=int, default=64,
                    help="fine subdomains factored/solved by the CPU baseline sample (512 / 64 = x8)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            self.f.close()
            os.unlink(self.f.name)
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        self.f.close()
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------- CPU baseline
def make_oracle(levels, w):
    import oracle
    import synthetic as syn
    return oracle.Oracle(levels, delta=w["delta"], nu_pre=w["nu"], nu_post=w["nu"], coef=w["coef"],
                         wave=syn.wave_vectors(), scale=w["scale"], load=w["load"])


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name, or on Arm the
    implementer and part numbers), with the machine type."""
    import platform
    name, impl, part = None, None, None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k, _, v = line.partition(":")
                k, v = k.strip(), v.strip()
                if k == "model name" and name is None:
                    name = v
                elif k == "CPU implementer" and impl is None:
                    impl = v
                elif k == "CPU part" and part is None:
                    part = v
    except OSError:
        pass
    if name:
        return f"{name} ({platform.machine()})"
    if impl or part:
        return f"{platform.machine()}, CPU implementer {impl}, part {part}"
    return platform.machine()


def cpu_baseline(o, levels, w, mu, iters, sample, slice_index=0):
    """The oracle, as it stands, on a bounded sample of one solve of the workload.

    Timed: assembly of every level (full); LU of one slice of `sample` fine
    subdomains, [slice_index * sample, ...) modulo their count, and of every
    coarser-level block and the coarsest block (full); one V-cycle whose
    fine-level RAS solves run for that slice only; and the rest of one FGMRES
    iteration (SpMVs, transfers, coarser levels, coarsest solve: full).  The
    fine-level factor and solve times are scaled by n_sub / sample; a solve
    costs assembly + factor + iters x (V-cycle + SpMV), with `iters` measured
    (the GPU's mean count of the same solves, or the oracle's own full solve).
    Consecutive slice indices walk through every fine subdomain once per
    n_sub / sample calls, so that averaged over such a cycle nothing is
    extrapolated from a subset.
    """
    L = len(levels)
    nsub0 = o.get("n_subs", 0)
    sample = max(1, min(sample, nsub0))
    nslices = max(1, nsub0 // sample)
    lo = (slice_index % nslices) * sample
    hi = min(nsub0, lo + sample)
    scale = nsub0 / (hi - lo)
    t0 = time.perf_counter()
    o.assemble(mu)
    t_asm = time.perf_counter() - t0
    # factor: the fine slice (scaled), coarser levels in full
    t0 = time.perf_counter()
    o.factor_range(0, lo, hi)
    t_f0 = (time.perf_counter() - t0) * scale
    t0 = time.perf_counter()
    for l in range(1, L - 1):
        o.factor_range(l, 0, o.get("n_subs", l))
    t_rest_f = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.factor_coarsest()
    t_fc = time.perf_counter() - t0
    t_factor = t_f0 + t_rest_f + t_fc
    # one iteration: fine RAS applications (the slice, scaled) + everything else
    n0 = levels[0].n_nodes
    r = np.random.default_rng(0).normal(size=n0)
    t0 = time.perf_counter()
    o.ras_apply_range(r, 0, lo, hi)
    t_ras0 = (time.perf_counter() - t0) * scale
    t0 = time.perf_counter()
    nu = w["nu"]
    # the remainder of a V-cycle: fine SpMVs and transfers, coarser levels
    for _ in range(2 * nu + 1):
        o.spmv(r, 0)
    if L > 1:
        rc = o.restrict(r, 0)
        o.interp(rc, 0)
        for l in range(1, L - 1):
            for _ in range(2 * nu):
                o.ras_apply(rc, l)
                o.spmv(rc, l)
            rc = o.restrict(rc, l)
        o.coarse_solve(rc)
    t_rest = time.perf_counter() - t0
    # the outer SpMV of one iteration (the oracle's Gram-Schmidt, a few vector
    # passes, is left out: well under 1% of an iteration here)
    t0 = time.perf_counter()
    o.spmv(r, 0)
    t_gs = time.perf_counter() - t0
    t_iter = 2 * nu * t_ras0 + t_rest + t_gs
    t_solve = t_asm + t_factor + iters * t_iter
    cores = os.cpu_count()
    omp = os.environ.get("OMP_NUM_THREADS")
    if omp:
        cores = int(omp)
    return {"value": 1.0 / t_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "seconds_per_solve": t_solve,
            "extrapolated": {"fine_subdomains_timed": hi - lo, "fine_subdomains": nsub0,
                             "scale": round(scale, 3), "slice": [lo, hi]},
            "sample": (f"one solve of the workload: assembly + coarser-level and coarsest LU in "
                       f"full; LU and RAS solves of fine subdomains {lo}..{hi - 1} of {nsub0} scaled "
                       f"x{scale:.1f}; {iters} iterations (measured) x (V-cycle + SpMV; Gram-Schmidt "
                       f"left out)"),
            "parts_s": {"assemble": t_asm, "factor": t_factor, "iteration": t_iter}}


# ------------------------------------------------------------- msp arm
def run_msp(args):
    import torch
    import torch.distributed as dist

    import synthetic as syn
    import paper_2412_08981_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P.load()
    levels, w = syn.workload(args.workload)
    kw = dict(delta=w["delta"], nu_pre=w["nu"], nu_post=w["nu"], restart=w["restart"],
              coef=w["coef"], wave=syn.wave_vectors(), scale=w["scale"], load=w["load"])
    stream = torch.cuda.Stream()

    def mu_of(i):
        return syn.mu_draw(replica_request(rank, i))

    def measure(precision, steps, warmup, transfer="bary", lv=None, opts=None, time_dominant=None, time_class=None):
        h = P.Hierarchy(levels if lv is None else lv, precision=precision,
                        **(dict(kw, transfer=transfer) if opts is None else opts))
        inst = h.assemble(mu_of(0), stream=stream)
        n = h.n_dofs(0)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        iters, relres = [], []

        def step(i):
            inst.reassemble(mu_of(i))
            inst.factor()
            st = inst.solve(x, rtol=args.rtol)
            iters.append(st["iterations"])
            relres.append(st["rel_residual"])
            return st

        # warm-up, with every kernel class timed to find the dominant one
        inst.profile_enable(P.msp.KERNEL_CLASSES)
        inst.profile_reset()
        for i in range(warmup):
            step(1000 + i)
        prof = inst.profile()
        # The coarsest block's tile steps run on forked streams beside the
        # persistent factorisation; their events also count the time they wait
        # behind it for SMs, so they are not candidates (the serialised ncu
        # launch list puts them at ~12 % of the solve).
        dominant = max((k for k in prof if k not in ("ldlt_diag", "ldlt_panel", "ldlt_trail")),
                       key=lambda k: prof[k]["ms"])
        kernel_ms = {k: round(v["ms"] / max(1, warmup), 3) for k, v in prof.items() if v["ms"] > 0}
        warm_launches = {k: v["launches"] for k, v in prof.items()}
        shares = {k: v["ms"] for k, v in prof.items()}
        tot = sum(shares.values()) or 1.0
        shares = {k: round(v / tot, 4) for k, v in shares.items() if v > 0}
        # The FP64 run times its dominant class live (the roofline); the other
        # runs time nothing inside the timed region, so that the factorisation
        # replays from its CUDA graph (captured by one more untimed step).
        if time_dominant is None:
            time_dominant = precision in ("f64", "f64tc")
        if time_class is not None:
            inst.profile_enable([time_class])
        elif time_dominant:
            inst.profile_enable([dominant])
        else:
            inst.profile_enable([])
            step(2000)
        inst.profile_reset()
        iters.clear()
        relres.clear()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        clk = Clocks(local)
        clk.start()
        evs[0].record(stream)
        for i in range(steps):
            step(i)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        if world > 1:
            dist.barrier()
        ms = evs[0].elapsed_time(evs[-1])
        lat = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
        prof = inst.profile()
        launches = int(sum(v["launches"] for v in prof.values()))
        grids = {"factor_ctas": [h.info(l)["fac_ctas"] for l in range(h.nlevels)],
                 "ras_ctas": [h.info(l)["ras_ctas"] for l in range(h.nlevels)],
                 "spmv_lanes_J_P_R": [h.info(l)["spmv_lanes"] for l in range(h.nlevels)]}
        out = dict(ms=ms, lat=lat, iters=list(iters), relres=list(relres), prof=prof, dominant=dominant, grids=grids,
                   shares=shares, kernel_ms=kernel_ms, warm_launches=warm_launches, launches=launches,
                   clocks=clocks,
                   x=x.cpu().numpy())
        # end to end through the host-buffer entry point
        xh = torch.zeros(n, dtype=torch.float64).pin_memory()
        xnp = xh.numpy()
        inst.solve_host(mu_of(0), xnp, rtol=args.rtol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(steps, 8))
        stages = []
        for i in range(e2e_steps):
            st = inst.solve_host(mu_of(i), xnp, rtol=args.rtol)
            stages.append((st["ms_assemble"], st["ms_factor"], st["ms_solve"]))
        e2e_s = time.perf_counter() - t0
        out["stage_ms"] = dict(zip(("assemble", "factor", "fgmres"),
                                   [round(float(v), 3) for v in np.mean(stages, axis=0)]))
        out["e2e"] = {"value": e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * 8,
                      "d2h_bytes_per_step": 8 * n}
        inst.close()
        h.close()
        return out

    def measure_batched(precision, steps, warmup, B):
        """B instances of the hierarchy solve different mu concurrently, each on
        its own stream and host thread (the C calls release the GIL)."""
        import threading
        h = P.Hierarchy(levels, precision=precision, **kw)
        streams = [torch.cuda.Stream() for _ in range(B)]
        insts = [h.assemble(mu_of(0), stream=streams[b]) for b in range(B)]
        n = levels[0].n_nodes
        xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(B)]
        lat, iters = [], []
        lock = threading.Lock()

        def worker(b, lo, hi, record):
            for i in range(lo + b, hi, B):
                t0 = time.perf_counter()
                insts[b].reassemble(mu_of(i))
                insts[b].factor()
                st = insts[b].solve(xs[b], rtol=args.rtol)
                dt = (time.perf_counter() - t0) * 1e3
                if record:
                    with lock:
                        lat.append(dt)
                        iters.append(st["iterations"])

        def run(lo, hi, record):
            th = [threading.Thread(target=worker, args=(b, lo, hi, record)) for b in range(B)]
            for t in th:
                t.start()
            for t in th:
                t.join()

        run(1000, 1000 + max(warmup, B), False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(0, steps, True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        for inst in insts:
            inst.close()
        h.close()
        return dict(value=steps / wall, lat=lat, iters=iters, wall_s=wall)

    def measure_hbm_kernels(reps=40, lv=None, opts=None):
        """The memory-bound operators of the finest level: J x (SpMV), P x_c
        (interpolation) and P^T x (restriction), each launch preceded by an L2
        eviction (a 256 MB read, which leaves clean lines).  The CUDA event
        clock ticks in microseconds, too coarse for one launch, so a sequence
        of `reps` (eviction, launch) pairs is timed against the same sequence
        without the launches, both queued behind a GPU sleep so that the host
        never starves the stream; the difference over reps is the launch.
        Algorithmic bytes: 12 per nonzero (value + column) + 4 per row pointer
        + 8 per vector entry read or written."""
        h = P.Hierarchy(levels if lv is None else lv, precision="f64", **(kw if opts is None else opts))
        inst = h.assemble(mu_of(0), stream=stream)
        i0, i1 = h.info(0), h.info(1)
        n0, n1 = i0["n_dofs"], i1["n_dofs"]
        flush = torch.zeros(32 << 20, dtype=torch.float64, device="cuda")  # 256 MB
        peak = measured_peak("hbm_gbs", 6755.1)
        ops = {"spmv_J0": (P.msp.MSP_OP_SPMV, n0, n0, 12 * i0["nnz"] + 4 * (n0 + 1) + 8 * n0 + 8 * n0),
               "interp_P0": (P.msp.MSP_OP_INTERP, n1, n0, 12 * i0["P_nnz"] + 4 * (n0 + 1) + 8 * n1 + 8 * n0),
               "restrict_PT0": (P.msp.MSP_OP_RESTRICT, n0, n1,
                                12 * i0["R_nnz"] + 4 * (n1 + 1) + 8 * n0 + 8 * n1)}
        out = {"l2": "evicted before every launch (256 MB read)", "peak_gbs": peak,
               "peak_source": "MEASURED_PEAKS hbm_gbs", "reps": reps, "rows_level0": n0,
               "nnz_level0": int(i0["nnz"])}

        def seq(fn):
            torch.cuda._sleep(4_000_000)  # ~2 ms: the host queues the whole sequence meanwhile
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                flush.sum()
                if fn:
                    fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        with torch.cuda.stream(stream):
            for name, (op, nin, nout, nbytes) in ops.items():
                x = torch.rand(nin, dtype=torch.float64, device="cuda")
                y = torch.zeros(nout, dtype=torch.float64, device="cuda")
                fn = lambda: inst.apply_op(op, 0, x, y)  # noqa: E731
                seq(fn)  # warm-up
                d = []
                for _ in range(3):
                    d.append(seq(fn) - seq(None))
                us = 1e3 * float(np.median(d)) / reps
                gbs = nbytes / (us * 1e-6) / 1e9
                out[name] = {"bytes_per_launch": int(nbytes), "us_per_launch": round(us, 2),
                             "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 3)}
        inst.close()
        h.close()
        return out

    def measure_batched_uneven(total=128, group=16, reps=3):
        """Batched uneven solves: `total` parameters, half on a 32^3 and half on a
        48^3 hierarchy (FP32 factors, FP64 outer loop), `group` instances
        resident at once (half of each).  Three ways, each warmed up and then
        timed `reps` times on the host wall clock over the same parameters
        (the median is reported):
          streams: every instance on its own stream and host thread, each
            re-assembling, factoring and solving its share in turn;
          batch: rounds of `group` parameters through one msp_batch: one
            msp_batch_assemble, one msp_batch_factor (the persistent-level
            blocks of all of them in one launch), one msp_solve_batch (FGMRES
            of all of them in lockstep, each V-cycle and Krylov step one
            launch per kernel for the whole round);
          batch_pipelined: the same as four msp_batch groups, each on its own
            stream and host thread."""
        import threading
        hs = []
        for name in ("cube32b_3lvl", "cube48_3lvl"):
            lv, wl = syn.workload(name)
            kk = dict(delta=wl["delta"], nu_pre=wl["nu"], nu_post=wl["nu"], restart=wl["restart"],
                      coef=wl["coef"], wave=syn.wave_vectors(), scale=wl["scale"], load=wl["load"])
            hs.append(P.Hierarchy(lv, precision="f32", **kk))
        streams = [torch.cuda.Stream() for _ in range(group)]
        insts = [hs[b % 2].assemble(mu_of(0), stream=streams[b]) for b in range(group)]
        xs = [torch.zeros(hs[b % 2].n_dofs(0), dtype=torch.float64, device="cuda") for b in range(group)]
        bstream = torch.cuda.Stream()
        out = {"hierarchies": ["cube32b_3lvl (35,937 nodes, 125 subdomains)", "cube48_3lvl (117,649 nodes, 343)"],
               "factor_precision": "f32", "solves": total, "resident_instances": group, "rtol": args.rtol}

        errs = []

        def run_threads(worker, count):
            th = [threading.Thread(target=worker, args=(b,)) for b in range(count)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            if errs:
                raise errs[0]

        def streams_way(lo, hi):
            def worker(b):
                try:
                    for i in range(lo + b, hi, group):
                        insts[b].reassemble(mu_of(i))
                        insts[b].factor()
                        insts[b].solve(xs[b], rtol=args.rtol)
                except Exception as e:
                    errs.append(e)
            run_threads(worker, group)

        batch = P.msp.Batch(insts, stream=bstream)
        batch_iters = []

        def batch_way(lo, hi):
            for r0 in range(lo, hi, group):
                assert hi - r0 >= group
                batch.assemble([mu_of(r0 + b) for b in range(group)])
                batch.factor()
                st = batch.solve(xs, rtol=args.rtol)
                batch_iters.extend(x["iterations"] for x in st)

        # the same batches pipelined: the resident instances as `npipe` msp_batch
        # groups, each on its own stream and host thread, so that one group's
        # factorisation overlaps another's solves
        npipe = 4
        per = group // npipe
        pstreams = [torch.cuda.Stream() for _ in range(npipe)]
        pbatches = None

        def pipelined_way(lo, hi):
            def worker(gi):
                try:
                    ids = list(range(gi * per, (gi + 1) * per))
                    for r0 in range(lo, hi, group):
                        pbatches[gi].assemble([mu_of(r0 + b) for b in ids])
                        pbatches[gi].factor()
                        pbatches[gi].solve([xs[b] for b in ids], rtol=args.rtol)
                except Exception as e:
                    errs.append(e)
            run_threads(worker, npipe)

        for name, fn in (("streams", streams_way), ("batch", batch_way), ("batch_pipelined", pipelined_way)):
            if name == "batch_pipelined":
                batch.close()
                pbatches = [P.msp.Batch(insts[g * per:(g + 1) * per], stream=pstreams[g]) for g in range(npipe)]
            fn(5000, 5000 + group)  # warm-up
            torch.cuda.synchronize()
            rates = []
            for _ in range(reps):  # each way timed `reps` times over the same parameters: the median
                t0 = time.perf_counter()
                fn(0, total)
                torch.cuda.synchronize()
                rates.append(total / (time.perf_counter() - t0))
            out[name] = {"value": float(np.median(rates)), "unit": UNIT, "reps": [round(v, 1) for v in rates]}
        out["batch"]["how"] = ("rounds of 16 parameters through one msp_batch: msp_batch_assemble, msp_batch_factor "
                               "(the persistent levels' blocks of all 16 in one launch, replayed from a CUDA graph), "
                               "msp_solve_batch (the 16 FGMRES solves in lockstep, every V-cycle and Krylov launch "
                               "shared)")
        out["batch"]["iterations_mean"] = float(np.mean(batch_iters)) if batch_iters else None
        out["batch_pipelined"]["how"] = (f"the 16 instances as {npipe} msp_batch groups of {per}, each on its own "
                                         "stream and host thread (one group's factorisation overlaps another's "
                                         "solves)")
        out["batch_vs_streams"] = out["batch"]["value"] / out["streams"]["value"]
        out["batch_pipelined_vs_streams"] = out["batch_pipelined"]["value"] / out["streams"]["value"]
        for bt in pbatches:
            bt.close()
        for inst in insts:
            inst.close()
        for h in hs:
            h.close()
        return out

    def measure_precision_study(steps):
        """The precision study: the 96^3 L-shaped domain, four levels, 2048
        subdomains, k spanning 1e-2 .. 1e2, FGMRES to rtol 1e-10, with FP64,
        FP32 and BF16 subdomain factors.  Per precision: solves/s over
        `steps` parameters (events on the instance stream), iterations, and
        the relative error of the parameter-0 solution against the FP64
        oracle's (a seeded sample of it, tests/golden/lshape96_4lvl_oracle.txt,
        written from the oracle alone by tests/golden/make_lshape96.py)."""
        lv, wl = syn.workload("lshape96_4lvl")
        kl = dict(delta=wl["delta"], nu_pre=wl["nu"], nu_post=wl["nu"], restart=wl["restart"],
                  coef=wl["coef"], wave=syn.wave_vectors(), scale=wl["scale"], load=wl["load"])
        gold = os.path.join(ROOT, "tests", "golden", "lshape96_4lvl_oracle.txt")
        gi, gv, gmeta = [], [], {}
        if os.path.exists(gold):
            with open(gold) as fh:
                for line in fh:
                    if line.startswith("#"):
                        continue
                    a, b = line.split()
                    if a.isdigit():
                        gi.append(int(a))
                        gv.append(float(b))
                    else:
                        gmeta[a] = float(b)
        gi, gv = np.array(gi, np.int64), np.array(gv)
        out = {"workload": "lshape96_4lvl", "dofs": lv[0].n_nodes, "subdomains_level0": None,
               "rtol": wl["rtol"], "oracle_iterations": int(gmeta["iterations"]) if gmeta else None}
        x64 = None
        for prec in ("f64", "f64tc", "f32", "bf16"):
            h = P.Hierarchy(lv, precision=prec, **kl)
            out["subdomains_level0"] = h.info(0)["n_sub"]
            inst = h.assemble(mu_of(0), stream=stream)
            x = torch.zeros(h.n_dofs(0), dtype=torch.float64, device="cuda")
            its = []
            for i in range(2):  # warm-up (the second factorisation is captured as a graph)
                inst.reassemble(mu_of(100 + i))
                inst.factor()
                inst.solve(x, rtol=wl["rtol"])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(steps):
                inst.reassemble(mu_of(i))
                inst.factor()
                its.append(inst.solve(x, rtol=wl["rtol"])["iterations"])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            inst.reassemble(mu_of(0))
            inst.factor()
            st = inst.solve(x, rtol=wl["rtol"])
            xv = x.cpu().numpy()
            e = {"value": steps / (ms / 1e3), "unit": UNIT, "steps": steps,
                 "iterations_mean": float(np.mean(its)), "iterations_param0": st["iterations"]}
            if gi.size:
                e["rel_err_vs_oracle_sample"] = float(np.linalg.norm(xv[gi] - gv) / np.linalg.norm(gv))
            if x64 is None:
                x64 = xv
            else:
                e["rel_diff_vs_f64_solution"] = float(np.linalg.norm(xv - x64) / np.linalg.norm(x64))
            out[prec] = e
            inst.close()
            h.close()
        return out

    SERVE_NAMES = ("cube32_3lvl", "cube64_3lvl", "cube128_4lvl")
    SERVE_PROBS = (0.5, 0.35, 0.15)

    def serve_hierarchies(precision, names=SERVE_NAMES):
        out = []
        for nm in names:
            lv, ww = syn.workload(nm)
            kk = dict(delta=ww["delta"], nu_pre=ww["nu"], nu_post=ww["nu"], restart=ww["restart"],
                      coef=ww["coef"], wave=syn.wave_vectors(), scale=ww["scale"], load=ww["load"])
            out.append(P.Hierarchy(lv, precision=precision, **kk))
        return out

    def serve_run(srv, ids, gaps, which, req0, keep_x=0):
        """Poisson arrivals (inter-arrival `gaps`, hierarchy `which`) of seeded mu
        (request numbers req0 + i), submitted on time by a host thread and
        polled in order.  Returns per-request latency, queueing delay and
        iterations, the wall time from the first arrival to the last
        completion, and the solutions of the first `keep_x` requests."""
        import threading
        nreq = len(gaps)
        rids = [None] * nreq
        t0 = time.perf_counter()

        def submitter():
            t = t0
            for i in range(nreq):
                t += gaps[i]
                dt = t - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                rids[i] = srv.submit(ids[which[i]], mu_of(req0 + i), rtol=args.rtol)

        th = threading.Thread(target=submitter)
        th.start()
        lat, queue, iters, xs = [], [], [], []
        for i in range(nreq):
            while rids[i] is None:
                time.sleep(0.0005)
            x = None
            if i < keep_x:
                x = np.zeros(hs_n[which[i]])
            rc, st = srv.poll(rids[i], x, -1)
            if rc != P.msp.MSP_OK:
                raise RuntimeError(f"request {i} failed with status {rc}")
            lat.append(st["ms_total"])
            queue.append(st["ms_queue"])
            iters.append(st["iterations"])
            if x is not None:
                xs.append(x)
        th.join()
        return dict(lat=np.array(lat), queue=np.array(queue), iters=np.array(iters),
                    wall=time.perf_counter() - t0, xs=xs)

    def queue_trend(q):
        """Mean queueing delay (ms) of the first and the last quarter of the requests."""
        k = max(1, len(q) // 4)
        return float(np.mean(q[:k])), float(np.mean(q[-k:]))

    hs_n = []

    def measure_serving(nreq, rate, cap_rates=(0.9, 0.75), cap_seconds=8.0, fp64_sample=40, full=False):
        """Serving the three-hierarchy trace: Poisson arrivals at `rate`/s of
        seeded mu on resident 32^3 / 64^3 / 128^3 hierarchies drawn with
        probabilities 0.5 / 0.35 / 0.15 (the first `nreq` requests of the
        2000-request trace), FP32 subdomain factors under the FP64 outer loop,
        4 slots per hierarchy, 120 GB budget, through msp_submit / msp_poll.
        Then a capacity search: arrivals at fractions of the measured
        throughput, each for `cap_seconds`, reporting whether the queue grew.
        And the plain FP64 path on the same mix: the first `fp64_sample`
        requests solved one after another with FP64 factors (no concurrency),
        whose solutions are compared with the served ones."""
        hs = serve_hierarchies(args.serve_precision)
        hs_n.clear()
        hs_n.extend(h.n_dofs(0) for h in hs)
        srv = P.Server(slots_per_hierarchy=4, budget_bytes=120 << 30)
        ids = [srv.add(h) for h in hs]
        rng = np.random.default_rng(99)
        gaps_all = rng.exponential(1.0 / rate, size=2000)
        which_all = rng.choice(len(SERVE_NAMES), size=2000, p=SERVE_PROBS)
        gaps, which = gaps_all[:nreq], which_all[:nreq]
        # warm every slot's instance first (not timed)
        warm = [srv.submit(ids[k], mu_of(900 + k)) for k in range(len(hs)) for _ in range(4)]
        for r in warm:
            srv.poll(r, None, -1)
        keep = min(fp64_sample, nreq)
        tr = serve_run(srv, ids, gaps, which, 5000, keep_x=keep)
        thr = nreq / tr["wall"]
        q0, q1 = queue_trend(tr["queue"])
        out = {"hierarchies": {nm: int((which == k).sum()) for k, nm in enumerate(SERVE_NAMES)},
               "dofs": {nm: hs_n[k] for k, nm in enumerate(SERVE_NAMES)},
               "requests": nreq, "of_trace": 2000, "arrival_rate_per_s": rate,
               "factor_precision": args.serve_precision + " (FP64 outer loop, SpMV, transfers, coarsest level)",
               "slots_per_hierarchy": 4, "mem_budget_bytes": 120 << 30,
               "value": thr, "unit": UNIT,
               "latency_ms": {"p50": float(np.percentile(tr["lat"], 50)),
                              "p99": float(np.percentile(tr["lat"], 99))},
               "queue_ms_first_last_quarter": [q0, q1],
               "iterations_mean": float(np.mean(tr["iters"])),
               "timing": "host wall clock from the first arrival to the last completion"}
        # capacity: the highest of these arrival rates whose queueing delay does not grow
        cap = []
        seed = 7000
        for frac in cap_rates:
            lam = frac * thr
            n = max(16, int(lam * cap_seconds))
            r2 = np.random.default_rng(seed)
            seed += 1
            g2 = r2.exponential(1.0 / lam, size=n)
            w2 = r2.choice(len(SERVE_NAMES), size=n, p=SERVE_PROBS)
            c = serve_run(srv, ids, g2, w2, 20000 + seed * 1000)
            a0, a1 = queue_trend(c["queue"])
            cap.append({"arrival_rate_per_s": lam, "fraction_of_saturated": frac, "requests": n,
                        "value": n / c["wall"], "unit": UNIT,
                        "latency_ms": {"p50": float(np.percentile(c["lat"], 50)),
                                       "p99": float(np.percentile(c["lat"], 99))},
                        "queue_ms_first_last_quarter": [a0, a1],
                        "queue_grows": bool(a1 > 2.0 * a0 + 50.0)})
        out["capacity_runs"] = cap
        ok = [c for c in cap if not c["queue_grows"]]
        out["capacity_per_s"] = max((c["arrival_rate_per_s"] for c in ok), default=None)
        srv.close()
        if keep == 0:
            for h in hs:
                h.close()
            return out
        # the plain FP64 path, sequentially, on the first requests of the same trace
        h64 = serve_hierarchies("f64")
        insts = [h.assemble(mu_of(0), stream=stream) for h in h64]
        xh = [np.zeros(h.n_dofs(0)) for h in h64]
        for k, inst in enumerate(insts):  # warm-up (not timed)
            inst.solve_host(mu_of(900 + k), xh[k], rtol=args.rtol)
        torch.cuda.synchronize()
        diffs = []
        t0 = time.perf_counter()
        for i in range(keep):
            k = int(which[i])
            insts[k].solve_host(mu_of(5000 + i), xh[k], rtol=args.rtol)
            diffs.append(float(np.linalg.norm(tr["xs"][i] - xh[k]) / np.linalg.norm(xh[k])))
        t64 = time.perf_counter() - t0
        v64 = keep / t64
        out["fp64_sequential"] = {
            "value": v64, "unit": UNIT, "requests": keep,
            "hierarchies": {nm: int((which[:keep] == k).sum()) for k, nm in enumerate(SERVE_NAMES)},
            "what": "the first requests of the same trace, one after another, FP64 factors, no concurrency, "
                    "through msp_solve_host (host wall clock)"}
        for inst in insts:
            inst.close()
        for h in h64:
            h.close()
        out["served_vs_fp64_solution_rel_diff_max"] = max(diffs) if diffs else None
        out["speedup_vs_fp64_sequential"] = thr / v64
        if out["capacity_per_s"]:
            out["capacity_vs_fp64_sequential"] = out["capacity_per_s"] / v64
        for h in hs:
            h.close()
        return out

    if args.profile_ops:
        profile_ops(P, torch, levels, kw, args)
        return
    res = measure(args.precision, args.steps, args.warmup)
    hbm = measure_hbm_kernels() if world == 1 and len(levels) > 1 and not args.no_hbm else None
    if hbm is not None and args.workload == "cube64_3lvl":
        # the same operators on the 96^3 L-shaped domain, whose level-0 matrix
        # (802,081 rows, ~12M nonzeros, ~160 MB) is larger than the L2 cache,
        # and on the 128^3 cube (2.15M rows, 31.8M nonzeros, ~430 MB)
        for big in ("lshape96_4lvl", "cube128_4lvl"):
            lvb, wb = syn.workload(big)
            hbm[big] = measure_hbm_kernels(
                lv=lvb, opts=dict(delta=wb["delta"], nu_pre=wb["nu"], nu_post=wb["nu"], restart=wb["restart"],
                                  coef=wb["coef"], wave=syn.wave_vectors(), scale=wb["scale"], load=wb["load"]))
    ms = max_over_ranks(res["ms"])
    value = whole_job_rate(args.steps, world, ms)
    mixed = None
    if not args.no_mixed and args.precision == "f64":
        mres = measure("f32", args.steps, args.warmup)
        mms = max_over_ranks(mres["ms"])
        mval = whole_job_rate(args.steps, world, mms)
        err = float(np.linalg.norm(mres["x"] - res["x"]) / np.linalg.norm(res["x"]))
        mixed = {"precision": "f32 subdomain factors, FP64 outer loop/SpMV/coarsest",
                 "value": mval, "unit": UNIT, "speedup_vs_f64": mval / value,
                 "latency_ms": {"p50": float(np.percentile(mres["lat"], 50)),
                                "p99": float(np.percentile(mres["lat"], 99))},
                 "iterations_mean": float(np.mean(mres["iters"])),
                 "rel_diff_vs_f64_solution": err, "e2e": mres["e2e"],
                 "final_rel_residual_max": float(np.max(mres["relres"])),
                 "stage_ms_host": mres["stage_ms"], "kernel_ms_per_solve": mres["kernel_ms"],
                 "grids": mres["grids"]}
        bres16 = measure("bf16", args.steps, args.warmup)
        b16 = args.steps / (bres16["ms"] / 1e3)
        mixed["bf16"] = {
            "precision": "BF16 subdomain factors (factored in FP32, rounded to nearest even), FP32 "
                         "accumulation in the solves, FP64 outer loop/SpMV/coarsest",
            "value": b16, "unit": UNIT, "speedup_vs_f64": b16 / value,
            "iterations_mean": float(np.mean(bres16["iters"])),
            "rel_diff_vs_f64_solution": float(np.linalg.norm(bres16["x"] - res["x"]) /
                                              np.linalg.norm(res["x"])),
            "final_rel_residual_max": float(np.max(bres16["relres"])),
            "stage_ms_host": bres16["stage_ms"], "kernel_ms_per_solve": bres16["kernel_ms"],
            "grids": bres16["grids"]}
        if args.batch > 1:
            bres = measure_batched("f32", max(args.steps, 2 * args.batch), args.warmup, args.batch)
            bval = bres["value"]
            if world > 1:
                bval = whole_job_rate(max(args.steps, 2 * args.batch), world,
                                      1e3 * max_over_ranks(bres["wall_s"]))
            mixed["batched"] = {
                "instances": args.batch, "value": bval, "unit": UNIT,
                "speedup_vs_f64": bval / value,
                "latency_ms": {"p50": float(np.percentile(bres["lat"], 50)),
                               "p99": float(np.percentile(bres["lat"], 99))},
                "iterations_mean": float(np.mean(bres["iters"])),
                "timing": "host wall clock over all instances, after a device synchronisation"}
    f64tc = None
    if not args.no_f64tc and args.precision == "f64":
        tres = measure("f64tc", args.steps, args.warmup, time_class="ldlt_blocks")
        tval = whole_job_rate(args.steps, world, max_over_ranks(tres["ms"]))
        tp = tres["prof"].get("ldlt_blocks", {})
        t_ms = tp.get("ms", 0.0) / max(1, tp.get("timed", 0))
        f64tc = {"precision": "FP64 factors, solves, outer loop; the panel and trailing products of the "
                              "persistent factorisation on the BF16 tensor cores, exact, by eight 7-bit digit "
                              "slices per operand (Ozaki scheme, FP64-class accuracy)",
                 "value": tval, "unit": UNIT, "speedup_vs_f64": tval / value,
                 "latency_ms": {"p50": float(np.percentile(tres["lat"], 50)),
                                "p99": float(np.percentile(tres["lat"], 99))},
                 "iterations_mean": float(np.mean(tres["iters"])),
                 "rel_diff_vs_f64_solution": float(np.linalg.norm(tres["x"] - res["x"]) / np.linalg.norm(res["x"])),
                 "final_rel_residual_max": float(np.max(tres["relres"])), "e2e": tres["e2e"],
                 "stage_ms_host": tres["stage_ms"], "kernel_ms_per_solve": tres["kernel_ms"],
                 "grids": tres["grids"], "dominant": tres["dominant"]}
        if t_ms > 0:
            eff = tp["flops"] / max(1, tp["launches"]) / (t_ms / 1e3) / 1e12
            f64tc["ldlt_blocks"] = {
                "avg_launch_ms": t_ms, "algorithmic_fp64_tflops": eff,
                "vs_fp64_pipe_peak": eff / FP64_PEAK_TFLOPS,
                "note": "the FP64 flops of the same factorisation over the launch time; the products run on "
                        "the tensor cores (36 BF16 digit-pair MMAs per 128 x 64 x 64 product), the diagonal "
                        "tiles on the FP64 pipe"}
    mls = None
    if not args.no_mls and args.precision == "f64":
        mls = {"transfer": "overlapping MLS both ways (Section 3.2), restriction of residual "
                           "densities scaled by nodal volumes"}
        for prec in ("f64", "f32"):
            k = args.steps  # same mu sequence as the barycentric runs
            r = measure(prec, k, args.warmup, transfer="mls")
            ref = res["x"] if prec == "f64" else (mres["x"] if mixed else res["x"])
            mls[prec] = {"value": k / (r["ms"] / 1e3), "unit": UNIT, "steps": k,
                         "iterations_mean": float(np.mean(r["iters"])),
                         "final_rel_residual_max": float(np.max(r["relres"])),
                         "rel_diff_vs_barycentric_solution":
                             float(np.linalg.norm(r["x"] - ref) / np.linalg.norm(ref)),
                         "stage_ms_host": r["stage_ms"],
                         "transfer_ms_per_solve": r["kernel_ms"].get("transfer", 0.0)}
    uneven = None
    if args.batch > 0 and args.precision == "f64" and world == 1:
        uneven = measure_batched_uneven()
    study = None
    if not args.no_precision_study and args.precision == "f64" and world == 1:
        study = measure_precision_study(max(2, min(args.steps, 4)))
    elastic = None
    if not args.no_elastic and args.precision == "f64":
        # the multi-field case: three displacement fields per vertex
        lv_e, w_e = syn.workload("elast32_3lvl")
        kw_e = dict(delta=w_e["delta"], nu_pre=w_e["nu"], nu_post=w_e["nu"], restart=w_e["restart"],
                    coef=w_e["coef"], wave=syn.wave_vectors(), scale=w_e["scale"], load=w_e["load"],
                    pde="elasticity", poisson=w_e["poisson"])
        k = max(2, min(args.steps, 8))
        elastic = {"workload": "elast32_3lvl", "description": DESCR["elast32_3lvl"],
                   "dofs": 3 * lv_e[0].n_nodes}
        x64 = None
        for prec in ("f64", "f32"):
            r = measure(prec, k, args.warmup, lv=lv_e, opts=kw_e, time_dominant=False)
            e = {"value": k / (r["ms"] / 1e3), "unit": UNIT, "steps": k,
                 "iterations_mean": float(np.mean(r["iters"])),
                 "final_rel_residual_max": float(np.max(r["relres"])),
                 "stage_ms_host": r["stage_ms"], "kernel_ms_per_solve": r["kernel_ms"]}
            if x64 is None:
                x64 = r["x"]
            else:
                e["rel_diff_vs_f64_solution"] = float(np.linalg.norm(r["x"] - x64) / np.linalg.norm(x64))
            elastic[prec] = e
    p2 = None
    if not args.no_p2 and args.precision == "f64":
        # DoFs on edges: quadratic elements, and a quadratic field coupled to a
        # linear one (different interpolations per field)
        p2 = {}
        for wl_name, key in (("p2cube32_3lvl", "p2"), ("p2p1cube32_3lvl", "p2p1")):
            lv_q, w_q = syn.workload(wl_name)
            kw_q = dict(delta=w_q["delta"], nu_pre=w_q["nu"], nu_post=w_q["nu"], restart=w_q["restart"],
                        coef=w_q["coef"], wave=syn.wave_vectors(), scale=w_q["scale"], load=w_q["load"],
                        pde=w_q["pde"], coupling=w_q.get("coupling", 1.0))
            k = max(2, min(args.steps, 8))
            obj = {"workload": wl_name, "description": DESCR[wl_name]}
            x64 = None
            for prec in ("f64", "f32"):
                r = measure(prec, k, args.warmup, lv=lv_q, opts=kw_q, time_dominant=False)
                e = {"value": k / (r["ms"] / 1e3), "unit": UNIT, "steps": k,
                     "iterations_mean": float(np.mean(r["iters"])),
                     "final_rel_residual_max": float(np.max(r["relres"])),
                     "stage_ms_host": r["stage_ms"], "kernel_ms_per_solve": r["kernel_ms"]}
                obj["dofs"] = int(r["x"].size)
                if x64 is None:
                    x64 = r["x"]
                else:
                    e["rel_diff_vs_f64_solution"] = float(np.linalg.norm(r["x"] - x64) / np.linalg.norm(x64))
                obj[prec] = e
            p2[key] = obj
    ilu = None
    if not args.no_ilu and args.precision == "f64":
        ilu = {"subdomain_solver": "ILU(2) on level 0, ILU(0) on level 1 (Section 4.4); coarsest direct (FP64)"}
        for prec in ("f64", "f32"):
            r = measure(prec, args.steps, args.warmup, opts=dict(kw, ilu=(2, 0)), time_dominant=False)
            ilu[prec] = {"value": args.steps / (r["ms"] / 1e3), "unit": UNIT, "steps": args.steps,
                         "iterations_mean": float(np.mean(r["iters"])),
                         "final_rel_residual_max": float(np.max(r["relres"])),
                         "rel_diff_vs_exact_lu_solution": float(np.linalg.norm(r["x"] - res["x"]) /
                                                                np.linalg.norm(res["x"])),
                         "stage_ms_host": r["stage_ms"], "kernel_ms_per_solve": r["kernel_ms"]}
    literal = None
    if not args.no_literal and args.precision == "f64":
        # Algorithm 2 as printed: every level RAS-smoothed (the coarsest too,
        # boxes of the same grid), its = 3, MLS both ways with the interpolated
        # residual, delta = 1; against one-level RAS with delta = 1
        lv_all = syn.hierarchy(w["ns"], tuple(w["parts"]) + (w["parts"][-1],))
        base = dict(coef=w["coef"], wave=syn.wave_vectors(), scale=w["scale"], load=w["load"],
                    restart=w["restart"], delta=1, coarse="ras")
        k = max(2, min(args.steps, 4))
        literal = {"note": "iteration study of Section 4's comparison; FP64; delta = 1"}
        for tag, lv, o in (
                ("algorithm2_literal", lv_all, dict(base, nu_pre=3, nu_post=3, transfer="mls",
                                                    restrict_scaling=False)),
                ("algorithm2_mls_scaled", lv_all, dict(base, nu_pre=3, nu_post=3, transfer="mls")),
                ("one_level_ras", lv_all[:1], dict(base, nu_pre=1, nu_post=0))):
            r = measure("f64", k, 1, lv=lv, opts=o)
            literal[tag] = {"levels": len(lv), "value": k / (r["ms"] / 1e3), "unit": UNIT,
                            "steps": k, "iterations_mean": float(np.mean(r["iters"])),
                            "final_rel_residual_max": float(np.max(r["relres"])),
                            "stage_ms_host": r["stage_ms"]}
    serving = None
    if args.serve > 0 and world == 1:
        serving = measure_serving(args.serve, args.serve_rate)
    if args.serve_trace and world == 1:
        serving = dict(serving or {}, trace=measure_serving(2000, 200.0, cap_rates=(), fp64_sample=0))
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    prof = res["prof"][res["dominant"]]
    is_flop = res["dominant"].startswith("ldlt")
    if prof["timed"] > 0:
        dom_ms = prof["ms"] / prof["timed"]
    else:  # reduced precisions replay the factorisation graph untimed: the warm-up's events per launch
        dom_ms = res["kernel_ms"][res["dominant"]] * args.warmup / max(1, res["warm_launches"][res["dominant"]])
    if is_flop:
        peak = FP64_PEAK_TFLOPS if args.precision in ("f64", "f64tc") else FP32_PEAK_TFLOPS  # f32, bf16: FP32 SIMT diag/panel
        achieved = prof["flops"] / max(1, prof["launches"]) / (dom_ms / 1e3) / 1e12
        roof = {"kernel": res["dominant"], "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": "derived: 152 SMs x FMA/clk x 2 x 2.07 GHz (FP64 SIMT, no fast "
                               "FP64 tensor path on GB300); probe measured 1.19 TFLOP/s FP64",
                "traffic": traffic_for(res["dominant"], args.workload, args.precision)}
    else:
        peak = measured_peak("hbm_gbs", 6755.1)
        achieved = prof["bytes"] / max(1, prof["launches"]) / (dom_ms / 1e3) / 1e9
        roof = {"kernel": res["dominant"], "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": "MEASURED_PEAKS hbm_gbs",
                "traffic": traffic_for(res["dominant"], args.workload, args.precision)}
    roof["avg_launch_ms"] = dom_ms
    roof["grids"] = res["grids"]
    roof["time_shares_warmup"] = res["shares"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": args.workload, "description": DESCR.get(args.workload, ""),
                   "parallelism": f"replicas x{world} (independent mu per rank)",
                   "factor_precision": args.precision, "rtol": args.rtol,
                   "l2": "inputs larger than L2 (subdomain factors of several GB)"},
        "latency_ms": {"p50": float(np.percentile(res["lat"], 50)),
                       "p99": float(np.percentile(res["lat"], 99))},
        "iterations_mean": float(np.mean(res["iters"])),
        "final_rel_residual_max": float(np.max(res["relres"])),
        "stage_ms_host": res["stage_ms"], "kernel_ms_per_solve": res["kernel_ms"],
        "clocks": res["clocks"], "e2e": res["e2e"], "gpu_launches": res["launches"],
        "roofline": roof,
    }
    if mixed:
        line["mixed"] = mixed
    if f64tc:
        line["f64_tc"] = f64tc
    if mls:
        line["mls"] = mls
    if ilu:
        line["ilu"] = ilu
    if p2:
        line["p2"] = p2
    if hbm:
        line["hbm_kernels"] = hbm
    if elastic:
        line["elasticity"] = elastic
    if study:
        line["precision_study"] = study
    if uneven:
        line["batched_uneven"] = uneven
    if literal:
        line["paper_literal"] = literal
    if serving:
        line["serving"] = serving
    if world == 1 and not args.no_cpu_baseline:
        levels_, w_ = syn.workload(args.workload)
        line["cpu_baseline"] = cpu_baseline(make_oracle(levels_, w_), levels_, w_, mu_of(0),
                                            int(round(np.mean(res["iters"]))), args.cpu_sample)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, KeyError, ValueError):
        return fallback


def kernel_source_hash(name):
    """Hash of the CUDA source file that holds a kernel class."""
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2412_08981_gb300", "csrc", name), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload, precision):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    this workload and factor precision and the source file of the kernel is
    unchanged since (else null)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    e = t.get(kernel)
    if not e or "kernel_file" not in e:
        return None
    if e.get("workload") != workload or e.get("precision") != precision:
        return None
    try:
        if e.get("source_hash") != kernel_source_hash(e["kernel_file"]):
            return None
    except OSError:
        return None
    return e.get("bytes_per_launch")


# ------------------------------------------------------- profiling mode
def profile_ops(P, torch, levels, kw, args):
    """Each requested operator of the finest level once, inside an NVTX range
    named after it, after an untimed warm-up call outside the ranges; for
    single-kernel ncu captures (ncu --nvtx --nvtx-include NAME/ -c 1).  Prints
    the algorithmic bytes of each (the same formulas as hbm_kernels; for the
    factorisation, the stored envelopes read and written once)."""
    import synthetic as syn
    ops = [o.strip() for o in args.profile_ops.split(",") if o.strip()]
    h = P.Hierarchy(levels, precision=args.precision, **kw)
    stream = torch.cuda.current_stream()
    inst = h.assemble(syn.mu_draw(0), stream=stream)
    i0, i1 = h.info(0), h.info(1)
    n0, n1 = i0["n_dofs"], i1["n_dofs"]
    es = {"f64": 8, "f64tc": 8, "f32": 4, "bf16": 2}[args.precision]
    m = P.msp
    table = {"J": (m.MSP_OP_SPMV, n0, n0, 12 * i0["nnz"] + 4 * (n0 + 1) + 16 * n0),
             "P": (m.MSP_OP_INTERP, n1, n0, 12 * i0["P_nnz"] + 4 * (n0 + 1) + 8 * n1 + 8 * n0),
             "PT": (m.MSP_OP_RESTRICT, n0, n1, 12 * i0["R_nnz"] + 4 * (n1 + 1) + 8 * n0 + 8 * n1),
             "RAS": (m.MSP_OP_RAS, n0, n0, 2 * i0["factor_elems"] * es + 13 * i0["sub_dofs"] + 8 * n0)}
    out = {"workload": args.workload, "precision": args.precision, "ops": {}}
    inst.factor()
    if "factor" in ops:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("factor")
        inst.factor()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        env = sum(h.info(l)["factor_elems"] for l in range(h.nlevels - 1) if h.info(l)["fac_ctas"] > 0)
        out["ops"]["factor"] = {"envelope_bytes_read_and_written": 2 * env * es,
                                "levels": [l for l in range(h.nlevels - 1) if h.info(l)["fac_ctas"] > 0]}
    for name in ops:
        if name not in table:
            continue
        op, nin, nout, nbytes = table[name]
        x = torch.rand(nin, dtype=torch.float64, device="cuda")
        y = torch.zeros(nout, dtype=torch.float64, device="cuda")
        inst.apply_op(op, 0, x, y)  # warm-up, outside the range
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(name)
        inst.apply_op(op, 0, x, y)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        out["ops"][name] = {"algorithmic_bytes": int(nbytes)}
    inst.close()
    h.close()
    print(json.dumps(out), flush=True)


# -------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle timed on the host cores, on this arm's workload and metric.

    The first warm-up step is one whole oracle solve of the first parameter
    (assembly, every factor, FGMRES to rtol): it measures the iteration count
    that the other steps use, and its wall time is reported beside the line.
    Every other step is the bounded sample of cpu_baseline, its fine slice
    advancing by one per step so that every fine subdomain is timed once per
    n_sub / sample steps.  ms_per_step is the wall time the timed steps took;
    value is the solves/s that their samples extrapolate to."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synthetic as syn
    levels, w = syn.workload(args.workload)
    o = make_oracle(levels, w)
    full = None
    iters = None
    t_all = time.perf_counter()
    if args.warmup >= 1:
        t0 = time.perf_counter()
        o.assemble(syn.mu_draw(0))
        o.factor()
        _, so = o.fgmres(rtol=args.rtol, restart=w["restart"])
        full = {"seconds": time.perf_counter() - t0, "iterations": so["iters"],
                "rel_residual": so["relres"], "what": "one whole oracle solve of parameter 0 (first warm-up step)"}
        iters = so["iters"]
    if iters is None:
        iters = 5  # no warm-up step to measure it: the count the oracle and the GPU give on this workload
    vals, walls = [], []
    for i in range(max(0, args.warmup - 1) + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(o, levels, w, syn.mu_draw(i), iters, args.cpu_sample, slice_index=i)
        if i >= max(0, args.warmup - 1):
            vals.append(cb["seconds_per_solve"])
            walls.append(time.perf_counter() - t0)
    s = float(np.sum(vals))
    value = len(vals) / s
    cb["value"] = value
    cb["extrapolated"]["steps_cover_every_fine_subdomain"] = bool(
        len(vals) >= cb["extrapolated"]["fine_subdomains"] // max(1, cb["extrapolated"]["fine_subdomains_timed"]))
    cb["sample"] = ("per step: " + cb["sample"] + "; the fine slice advances by one per step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "description": DESCR.get(args.workload, "")},
            "extrapolated_seconds_per_solve": s / len(vals),
            "full_solve": full, "iterations_used": iters,
            "wall_s_total": time.perf_counter() - t_all,
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_msp(args)


if __name__ == "__main__":
    main()
