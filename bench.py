"""Benchmark of the fused relativistic-LB stream-collide step on GB300.

Workload (default): 3-D MRT periodic box, D3Q19, 256^3 nodes, FP64, tau_v = 0.9,
tau_e = 0.55, tau_eps = 0.8 (tau_q = tau_f = tau_v), seeded smooth random fields
(e = e0 (1 + 0.1 modes), solenoidal u with max|u| = 0.3, n = n0 (1 + 0.05 modes)).
A "step" is one lattice time step: one pass of the fused pull-stream + moments +
recovery + equilibria + MRT collide over all 16.7 M nodes (one kernel launch).
Metric: MLUPS (million lattice-node updates per second), higher is better.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload box256|box512_fp32]

The metric has two halves, FP64 and FP32 population storage.  The default run
times the 256^3 FP64 box and then the 512^3 FP32-storage box of the same fields
and relaxation times, and nests the second in the same line as ``fp32_storage``
(its own timing, roofline, clocks, end-to-end figure and per-field error against
the FP64 path).  Each box is timed as repeated regions of exactly K steps (at
least --min-repeats of them and --min-seconds of device time); the median region
is reported, with the spread.

Prints one JSON line.  ``--impl reference`` times the CPU oracle (the plain FP64
statement of the scheme) on the host cores over a bounded sample of the same
workload.  Under torchrun every rank runs its own replica (the lattices are
independent; there is no data-path collective), the elapsed time is the max over
ranks and ``value`` counts all ranks' node updates.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

WORKLOADS = {
    "box256": dict(N=256, precision="fp64", dtype="f64 (FP64 storage; sums, recovery and links in 64-bit block fixed point)",
                   bytes_per_update=608,
                   desc="3-D MRT periodic box, D3Q19, 256^3 nodes, FP64, tau_v=0.9 tau_e=0.55 tau_eps=0.8, "
                        "seeded smooth fields (max|u|=0.3), 500 steps"),
    "box128": dict(N=128, precision="fp64", dtype="f64 (FP64 storage; sums, recovery and links in 64-bit block fixed point)",
                   bytes_per_update=608,
                   desc="3-D MRT periodic box, D3Q19, 128^3 nodes, FP64 (small profiling case of the 256^3 "
                        "workload, 1.3 GB of lattices)"),
    "box128_fp32": dict(N=128, precision="fp32", dtype="f32-storage/f64-recovery", bytes_per_update=304,
                        desc="3-D MRT periodic box, D3Q19, 128^3 nodes, FP32 storage (small profiling case)"),
    "tubes": dict(N=None, precision="fp32", dtype="f32-storage/f64-recovery", bytes_per_update=304,
                  desc="tau sweep: 1024 quasi-1D D3Q19 shock tubes, lengths uniform in [200, 3200], (tau_v, tau_e, "
                       "tau_eps) log-uniform in [0.51, 3] with tau_e <= tau_v, P ratio 5.43:2.22, FP32 populations / "
                       "FP64 recovery, 4000 steps in one persistent launch from a CUDA graph"),
    "adjoint": dict(N=None, precision="fp64", dtype="f64", bytes_per_update=608,
                    desc="adjoint: quasi-1D D3Q19 shock tube of 1600 nodes, FP64 MRT (0.9, 0.55, 0.8), 4000 steps "
                         "with sqrt(T) checkpoints; gradient of the P/u profile misfit w.r.t. tau_v, tau_e, "
                         "tau_eps and the 1600-value initial e field (forward + recompute + reverse)"),
    "tubes_small": dict(N=None, precision="fp32", dtype="f32-storage/f64-recovery", bytes_per_update=304,
                        desc="small profiling case of the tau sweep: 128 tubes of the same length / tau "
                             "distribution, FP32 storage"),
    "box512_fp32": dict(N=512, precision="fp32", dtype="f32-storage/f64-recovery", bytes_per_update=304,
                        desc="3-D MRT periodic box, D3Q19, 512^3 nodes, FP32 population storage with FP64 sums "
                             "and recovery, same fields and taus, 200 steps"),
}
TAUS = dict(tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8)
# step counts of the workloads as configured (256^3 box: 500, 512^3 FP32 box: 200, tau sweep
# and adjoint: 4000)
DEFAULT_STEPS = {"box256": 500, "box128": 500, "box128_fp32": 500, "box512_fp32": 200, "tubes": 4000,
                 "tubes_small": 200, "adjoint": 4000}

# DRAM bytes (read + write) per node update of the step kernel, from ncu captures of the
# 128^3 box with the same kernel (the 256^3 / 512^3 lattices exceed the capture size
# rule); traffic per launch = bytes per update x nodes.  profiles/k_step_ws_box128_f64.md:
# 639.1 MB read + 580.9 MB written / 2,097,152; profiles/k_step_box128_f32.md: 318.8 MB
# read + 268.0 MB written / 2,097,152.
NCU_BYTES_PER_UPDATE = {"fp64": (639101952 + 580899840) / 2097152, "fp32": (318842112 + 267988736) / 2097152}
# k_tubes on the 1024-tube sweep at 320 threads x 2 CTAs per SM
# (profiles/k_tubes_sweep1024_fp32.md): 49.65 GB over 1,719,757 nodes x 200 steps
NCU_BYTES_PER_UPDATE_TUBES = (12.790533e9 + 36.859571e9) / (1719757 * 200)

# FP64-pipe operations of one FP32-storage node update (the sums are exact on the
# FP32 and integer pipes and rounded to FP64 by integer bit assembly): recovery 15
# (|M|^2 3, quadratic residual 2, Newton step 1, reciprocal 2, u 3 and its 3
# conversions to FP32, P 1) + the three equilibrium constants 3.
FP64_OPS_PER_UPDATE_F32S = 18

# FP64-pipe operations (int64 -> FP64 conversion = 1) of one FP64 node update: the 38
# roundings of the relaxed links.  The sums, the recovery, the equilibria and the
# relaxation run in 64-bit fixed point on the integer pipes.
FP64_OPS_PER_UPDATE = 38


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def reduce_max(value: float, dist) -> float:
    """Max of a per-rank float over all ranks (the job's elapsed time)."""
    if dist is None:
        return value
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Whole-job throughput: units of all replicas over the slowest rank's time (MLUPS for node updates)."""
    return units_per_rank * world_size / seconds / 1e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
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
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(seconds_budget=15.0):
    """The oracle (plain FP64, torch CPU ops) on a bounded sample of the workload:
    a 48^3 box of the same generator and relaxation times, as many steps as fit the
    budget (at least 1).  Returns MLUPS and what was run."""
    import oracle.rlb_oracle as O
    from paper_1211_3286_gb300 import inputs as I
    n = 48
    affinity = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    torch.set_num_threads(affinity)
    e, ux, uy, uz, nn = I.periodic_box(None, shape=(n, n, n))
    prm = O.Params(collision="mrt", **TAUS)
    f, g = O.init_populations(e, torch.stack([ux, uy, uz]), nn)
    t0 = time.perf_counter()
    steps = 0
    while steps < 1 or time.perf_counter() - t0 < seconds_budget:
        f, g = O.step(f, g, prm)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": n ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": torch.get_num_threads(),
            "host_cpus": os.cpu_count(), "affinity_cpus": affinity,
            "cores_note": "cores = torch CPU threads the oracle ran on, set to the process's CPU affinity",
            "cpu_model": _cpu_model(), "kind": "oracle",
            "sample": "%d^3 MRT box, %d steps, same generator and taus, FP64 oracle" % (n, steps),
            "seconds": round(dt, 2)}


def _cpu_model():
    """Host CPU model as lscpu or /proc/cpuinfo name it (best effort)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def run_reference(args):
    dist, rank, ws = _dist()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    cb = cpu_baseline(args.ref_seconds)
    line = {"impl": "reference", "metric": "MLUPS", "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "reference_sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_tubes(args, dist, rank, ws, local):
    import numpy as np
    from paper_1211_3286_gb300 import inputs as I
    from paper_1211_3286_gb300.batch import TubeBatch
    wl = WORKLOADS[args.workload]
    lengths, taus = I.tube_sweep(128 if args.workload == "tubes_small" else 1024)
    nodes = int(lengths.sum())
    parts = [I.shock_tube(int(L)) for L in lengths]
    fields = [torch.from_numpy(np.concatenate([p[c].reshape(-1) for p in parts])) for c in range(5)]
    stream = torch.cuda.Stream()
    b = TubeBatch(lengths, taus, precision="fp32", stream=stream)
    b.set_fields(*[t.cuda() for t in fields])
    if args.tubes_shape:
        shape = tuple(int(v) for v in args.tubes_shape.split(","))
        b.set_shape(*shape)
    else:
        shape = b.autotune(16)
    b.run(args.warmup)
    b.check()
    b.set_fields(*[t.cuda() for t in fields])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as cs:
        ev0.record(stream)
        b.run(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    b.check()
    ms = reduce_max(ev0.elapsed_time(ev1), dist)
    clocks = cs.summary()
    mlups = whole_job_rate(nodes * args.steps, ws, ms / 1e3)
    e2e = None
    if not args.no_e2e:
        import ctypes
        from paper_1211_3286_gb300 import _lib as L
        hf = [t.pin_memory() for t in fields]
        outs = [torch.empty(nodes, dtype=torch.float64).pin_memory() for _ in range(6)]
        # one untimed host round trip (staging buffer allocated on first use)
        b.set_fields(*hf)
        L.rlb_batch_get_fields(b.handle, *[ctypes.c_void_p(o.data_ptr()) for o in outs], L.RLB_HOST)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.set_fields(*hf)
        b.run(args.steps)
        L.rlb_batch_get_fields(b.handle, *[ctypes.c_void_p(o.data_ptr()) for o in outs], L.RLB_HOST)
        dt = time.perf_counter() - t0
        e2e = {"value": nodes * args.steps * ws / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 5 * nodes * 8 / args.steps, "d2h_bytes_per_step": 6 * nodes * 8 / args.steps,
               "what": "rlb_batch_set_fields(host) + rlb_batch_run(K) + rlb_batch_get_fields(host), pinned"}
    b.close()
    # shock-tube profile error of the FP32-storage sweep against the FP64 path (same
    # tubes, taus and steps; outside the timed region)
    err = None
    if not args.no_error:
        out = {}
        for prec in ("fp32", "fp64"):
            bb = TubeBatch(lengths, taus, precision=prec, stream=stream)
            bb.set_fields(*[t.cuda() for t in fields])
            bb.run(args.steps)
            bb.check()
            out[prec] = bb.fields("cuda")
            offs = np.asarray(bb.offsets)
            bb.close()
        a, r = ({k: v.cpu() for k, v in out[p].items()} for p in ("fp32", "fp64"))
        per = []
        for t in range(len(lengths)):
            s0, s1 = int(offs[t]), int(offs[t + 1])
            ee = float((a["e"][s0:s1] - r["e"][s0:s1]).abs().max() / r["e"][s0:s1].abs().max())
            eu = float((a["ux"][s0:s1] - r["ux"][s0:s1]).abs().max() / max(float(r["ux"][s0:s1].abs().max()), 0.1))
            per.append(max(ee, eu))
        per = np.asarray(per)
        w = int(per.argmax())
        err = {"per_tube": {"median": float(np.median(per)), "p90": float(np.percentile(per, 90)),
                            "max": float(per.max()), "worst_tube": w, "worst_taus": [float(x) for x in taus[w]]},
               "steps": args.steps, "metric": "per tube: max over e and ux of max|fp32 - fp64| / max|fp64| "
               "(ux over max(max|ux|, 0.1)); FP64 path = oracle to 1e-12"}
    hbm_peak, peak_kind = _peaks()
    upd_s = nodes * args.steps / (ms / 1e3)
    gbs = 304 * upd_s / 1e9
    fp64_peak = 152 * 2 * 2.07
    traffic = (NCU_BYTES_PER_UPDATE_TUBES * nodes * args.steps
               if args.workload == "tubes" and NCU_BYTES_PER_UPDATE_TUBES is not None else None)
    alu = {"bound": "alu", "achieved": FP64_OPS_PER_UPDATE_F32S * upd_s / 1e9, "peak": fp64_peak,
           "unit": "G FP64 op/s", "traffic": traffic,
           "peak_kind": "derived: 152 SM x 2 FP64 op/clk x 2.07 GHz (measured 2.05 DFMA/clk/SM)"}
    alu["frac"] = alu["achieved"] / fp64_peak
    hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "traffic": traffic, "peak_kind": peak_kind, "note": "streaming-equivalent bytes (304 B/update); the tubes "
           "are re-read through L2"}
    roof = alu if alu["frac"] > hbm["frac"] else hbm
    if rank == 0:
        line = {"metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
                "config": {"workload": wl["desc"], "nodes": nodes, "launch_shape": {"threads": shape[0],
                           "ctas_per_sm": shape[1]}, "l2": "batch lattices %.0f MB; one launch covers all steps"
                           % (2 * 38 * nodes * 4 / 1e6)},
                "roofline": roof, "hbm_roofline": hbm, "clocks": clocks, "e2e": e2e, "gpu_launches": 1}
        if err is not None:
            line["error_vs_fp64"] = err
        print(json.dumps(line))


def run_adjoint(args, dist, rank, ws, local):
    from paper_1211_3286_gb300 import inputs as I
    from paper_1211_3286_gb300.adjoint import misfit_gradient
    from paper_1211_3286_gb300.lattice import Lattice
    wl = WORKLOADS["adjoint"]
    L, T = 1600, args.steps
    zg = ("zero_gradient", "periodic", "periodic")
    e, ux, uy, uz, n = (torch.from_numpy(a).cuda() for a in I.shock_tube(L))
    pert = torch.from_numpy(I.perturbation(L)).reshape(1, 1, L).cuda()
    stream = torch.cuda.Stream()
    tgt = Lattice((1, 1, L), collision="mrt", tau_f=0.9, tau_v=0.909, tau_e=0.5555, tau_eps=0.808, bc=zg,
                  stream=stream)
    tgt.set_fields(e * (1 + 1e-3 * pert), ux, uy, uz, n)
    tgt.step(T)
    tf = tgt.fields("cuda")
    tgt.close()
    lat = Lattice((1, 1, L), collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8, bc=zg, stream=stream)

    def one():
        lat.set_fields(e, ux, uy, uz, n)
        return misfit_gradient(lat, T, tf["P"], tf["ux"], tf["uy"], tf["uz"])
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    reps = 3
    with ClockSampler(local) as cs:
        t0 = time.perf_counter()
        for _ in range(reps):
            loss, dtau, de0 = one()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
    lat.close()
    if rank == 0:
        line = {"metric": "MLUPS", "value": L * T / dt / 1e6, "unit": "MLUPS", "n_gpus": ws, "steps": T,
                "warmup": args.warmup, "ms_per_step": dt * 1e3 / T, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["desc"], "ms_per_gradient": dt * 1e3, "loss": loss,
                           "dtau": dtau.tolist(), "value_counts": "forward node updates per second of a full "
                           "gradient (forward + recompute + reverse)"},
                "clocks": cs.summary(), "e2e": None, "gpu_launches": reps * adjoint_launches(T)}
        print(json.dumps(line))


def adjoint_launches(T):
    """librlb kernels of one gradient on the 1600-node tube: k_init (set_fields); T forward
    steps; k_adj_loss; k_adj_fwd; T - nseg recompute steps (segments of K = ceil(sqrt T)
    steps, each refilled from its checkpoint); T reverse steps; k_adj_e0; two k_rowsum."""
    K = max(1, math.ceil(math.sqrt(T)))
    nseg = (T + K - 1) // K
    return 1 + T + 1 + 1 + (T - nseg) + T + 1 + 2


def time_box(args, wl, steps, dist, ws, local, min_repeats=5, min_seconds=2.0, e2e=True):
    """Time one box workload: warm-up, then repeated timed regions of exactly
    ``steps`` launches each (at least ``min_repeats`` of them and at least
    ``min_seconds`` of device time in total), each bracketed by a barrier and a
    device synchronisation, with CUDA events on the library's stream.  Returns
    the median region, its spread, the clocks sampled over all regions and the
    end-to-end (host buffers) measurement."""
    from paper_1211_3286_gb300 import inputs as I
    from paper_1211_3286_gb300.lattice import Lattice
    N = wl["N"]
    nodes = N ** 3
    stream = torch.cuda.Stream()
    e, ux, uy, uz, n = I.periodic_box(N, device="cuda")
    with torch.cuda.stream(stream):
        lat = Lattice((N, N, N), collision="mrt", precision=wl["precision"], stream=stream, **TAUS)
    lat.set_fields(e, ux, uy, uz, n)
    del e, ux, uy, uz, n
    torch.cuda.synchronize()

    lat.step(args.warmup)
    lat.check()
    regions = []
    with ClockSampler(local) as cs:
        while len(regions) < min_repeats or sum(regions) < min_seconds * 1e3:
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            ev0.record(stream)
            lat.step(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            regions.append(reduce_max(ev0.elapsed_time(ev1), dist))
            if len(regions) >= 200:
                break
    if dist is not None:
        dist.barrier()
    lat.check()
    ms = statistics.median(regions)
    clocks = cs.summary()

    # end to end through the C ABI with pinned host buffers: upload the initial
    # fields, run the steps, read the final fields back
    out_e2e = None
    if e2e:
        from paper_1211_3286_gb300 import _lib as L
        import ctypes
        hf = [t.cpu().pin_memory() for t in I.periodic_box(N, device="cuda")]
        outs = [torch.empty((N, N, N), dtype=torch.float64).pin_memory() for _ in range(6)]
        # one untimed host round trip: the library allocates its host-I/O staging
        # buffer on first use (one-time setup, like the warm-up steps)
        lat.set_fields(*hf)
        L.rlb_get_fields(lat.handle, *[ctypes.c_void_p(o.data_ptr()) for o in outs], L.RLB_HOST)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        lat.set_fields(*hf)
        lat.step(steps)
        L.rlb_get_fields(lat.handle, *[ctypes.c_void_p(o.data_ptr()) for o in outs], L.RLB_HOST)
        dt = reduce_max(time.perf_counter() - t0, dist)
        out_e2e = {"value": whole_job_rate(nodes * steps, ws, dt), "unit": "MLUPS",
                   "h2d_bytes_per_step": 5 * nodes * 8 / steps, "d2h_bytes_per_step": 6 * nodes * 8 / steps,
                   "what": "rlb_set_fields(host) + rlb_step(K) + rlb_get_fields(host), pinned buffers"}
        del hf, outs
    lat.close()
    del lat
    torch.cuda.empty_cache()

    per_launch_s = ms / 1e3 / steps
    hbm_peak, peak_kind = _peaks()
    gbs = wl["bytes_per_update"] * nodes / per_launch_s / 1e9
    nb = NCU_BYTES_PER_UPDATE.get(wl["precision"])
    traffic = None if nb is None else nb * nodes
    hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "traffic": traffic, "peak_kind": peak_kind,
           "algorithmic_bytes": "%d B per node update x %d nodes per launch" % (wl["bytes_per_update"], nodes)}
    roof = hbm
    fp64_ops = FP64_OPS_PER_UPDATE if wl["precision"] == "fp64" else FP64_OPS_PER_UPDATE_F32S
    # The FP64 pipe (152 SMs x 2 instructions per clock x 2.07 GHz) carries the
    # int64 -> FP64 roundings (and, with FP32 storage, the recovery); the roofline
    # reported is the bound with the larger fraction.
    fp64_peak = 152 * 2 * 2.07
    gops = fp64_ops * nodes / per_launch_s / 1e9
    alu = {"bound": "alu", "achieved": gops, "peak": fp64_peak, "unit": "G FP64-pipe op/s",
           "frac": gops / fp64_peak, "traffic": traffic,
           "peak_kind": "derived: 152 SM x 2 FP64 op/clk x 2.07 GHz (measured 2.05 DFMA/clk/SM)",
           "hbm_frac": gbs / hbm_peak}
    if alu["frac"] > hbm["frac"]:
        roof = alu
    per_step = sorted(r / steps for r in regions)
    return {"value": whole_job_rate(nodes * steps, ws, ms / 1e3), "ms_per_step": ms / steps,
            "ms_per_step_spread": [per_step[0], per_step[-1]], "repeats": len(regions),
            "ms_per_step_x_sm_mhz": (ms / steps * clocks["sm_mhz"]) if clocks.get("sm_mhz") else None,
            "nodes": nodes, "roofline": roof, "hbm_roofline": hbm, "clocks": clocks, "e2e": out_e2e,
            "gpu_launches": steps * len(regions)}


def run_ours(args):
    dist, rank, ws = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (librlb has no CPU path)")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()

    if args.workload in ("tubes", "tubes_small"):
        return run_tubes(args, dist, rank, ws, local)
    if args.workload == "adjoint":
        return run_adjoint(args, dist, rank, ws, local)
    wl = WORKLOADS[args.workload]
    r = time_box(args, wl, args.steps, dist, ws, local, min_repeats=args.min_repeats,
                 min_seconds=args.min_seconds, e2e=not args.no_e2e)

    # FP32 storage: per-field error of the final fields against the FP64 path on the
    # same initial fields and step count (outside the timed region)
    err = None
    if wl["precision"] == "fp32" and not args.no_error:
        err = fp32_error_vs_fp64(wl["N"], args.steps, torch.cuda.Stream())

    # the metric's second half: the FP32-storage variant of the same box, 512^3,
    # timed the same way after the FP64 lattice is freed
    f32 = None
    if args.workload == "box256" and not args.no_fp32_storage:
        w32 = WORKLOADS["box512_fp32"]
        k32 = args.steps if args.steps_given else DEFAULT_STEPS["box512_fp32"]
        f32 = time_box(args, w32, k32, dist, ws, local, min_repeats=args.min_repeats,
                       min_seconds=args.min_seconds, e2e=not args.no_e2e)
        f32 = {"workload": w32["desc"], "metric": "MLUPS", "unit": "MLUPS", "steps": k32, "dtype": w32["dtype"],
               **f32, "speedup_vs_fp64": f32["value"] / r["value"]}
        if not args.no_error:
            f32["error_vs_fp64"] = fp32_error_vs_fp64(w32["N"], k32, torch.cuda.Stream())

    if rank == 0:
        line = {"metric": "MLUPS", "value": r["value"], "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
                "config": {"workload": wl["desc"], "nodes": r["nodes"], "l2": "lattice (%.1f GB) larger than L2"
                           % (2 * 38 * r["nodes"] * (8 if wl["precision"] == "fp64" else 4) / 1e9),
                           "parallelism": "replicas" if ws > 1 else "single",
                           "timing": "median of %d timed regions of %d steps each" % (r["repeats"], args.steps)},
                "ms_per_step_spread": r["ms_per_step_spread"], "repeats": r["repeats"],
                "ms_per_step_x_sm_mhz": r["ms_per_step_x_sm_mhz"],
                "roofline": r["roofline"], "hbm_roofline": r["hbm_roofline"], "clocks": r["clocks"],
                "e2e": r["e2e"], "gpu_launches": r["gpu_launches"]}
        if err is not None:
            line["error_vs_fp64"] = err
        if f32 is not None:
            line["fp32_storage"] = f32
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(args.ref_seconds)
        print(json.dumps(line))


def fp32_error_vs_fp64(N, steps, stream):
    """Final fields of the FP32-storage lattice against the FP64 lattice (which matches
    the FP64 oracle to 1e-12) after the same steps from the same initial fields:
    max|a - b| / max|b| per field, velocities over max(max|u|, 0.1)."""
    from paper_1211_3286_gb300 import inputs as I
    from paper_1211_3286_gb300.lattice import Lattice
    out = {}
    for prec in ("fp32", "fp64"):
        with torch.cuda.stream(stream):
            lat = Lattice((N, N, N), collision="mrt", precision=prec, stream=stream, **TAUS)
        lat.set_fields(*I.periodic_box(N, device="cuda"))
        lat.step(steps)
        lat.check()
        out[prec] = lat.fields("cuda")
        lat.close()
    a, b = out["fp32"], out["fp64"]
    umax = max(float(b[k].abs().max()) for k in ("ux", "uy", "uz"))
    err = {}
    for k in ("e", "P", "n", "ux", "uy", "uz"):
        scale = max(umax, 0.1) if k.startswith("u") else float(b[k].abs().max())
        err[k] = float((a[k] - b[k]).abs().max()) / scale
    del out, a, b
    torch.cuda.empty_cache()
    return {"per_field": err, "steps": steps, "metric": "max|fp32 - fp64| / max|fp64| per field, "
            "velocities over max(max|u|, 0.1); FP64 path = oracle to 1e-12"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's own step count)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="box256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the FP32-storage error run against the FP64 path")
    ap.add_argument("--min-repeats", type=int, default=5,
                    help="box workloads: at least this many timed regions of --steps steps (median reported)")
    ap.add_argument("--min-seconds", type=float, default=2.0,
                    help="box workloads: repeat timed regions until this much device time has passed")
    ap.add_argument("--tubes-shape", default=None,
                    help="threads,ctas_per_sm for the tube sweep instead of autotuning (for profiling)")
    ap.add_argument("--no-fp32-storage", action="store_true",
                    help="default workload only: skip the nested FP32-storage 512^3 box")
    ap.add_argument("--ref-seconds", type=float, default=20.0,
                    help="CPU budget of the oracle sample (reference arm and cpu_baseline)")
    args = ap.parse_args()
    args.steps_given = args.steps is not None
    if args.steps is None:
        args.steps = DEFAULT_STEPS.get(args.workload, 500)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
