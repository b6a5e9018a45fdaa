"""Throughput benchmark of the rigid-aggregate FSD time step on GB300.

Metric: bead-steps/sec (beads x timed steps / seconds) of the full step
(neighbour lists, lubrication blocks, per-aggregate LUs, preconditioned
saddle-point solve to a relative residual of 1e-6, outputs, rigid-body
update) on 32768 beads = 4096 rigid 8-bead random-attachment aggregates at
bead volume fraction 0.2 in simple shear (rate 1), lubrication cut-off 3a,
constant xi = 0.5.  `value` is the mixed-precision path (FP32 operator inside
FP64 iterative refinement, FP64 Arnoldi and LU); the plain FP64 path and the
mixed path with an FP32 inner Krylov basis are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload step|batch|rods|seeds|oracle-ladder|configs]

With N > 1 (torchrun) every rank steps its own replica of the suspension (the
single-suspension solve does not shard); value = beads x steps x ranks / the
slowest rank's time.  --impl reference times the FP64 CPU oracle on a bounded
32-bead sample of the same workload per step.

--profile-run only steps the mixed path with the host-driven loop (no graph,
no other passes, no JSON line): the command the ncu launch lists and kernel
captures under profiles/ are taken on.

--workload batch times the batched form instead: 64 independent suspensions
(bead counts log-uniform in [256, 8192], aggregate sizes uniform in 2..64,
volume fractions uniform in [0.05, 0.3]) advanced together by
fsd_step_batch (one graph per system and step, all in flight), next to the
same suspensions stepped one at a time; mixed precision, GMRES 1e-6,
autotuned splitting.

--workload rods runs the rod scaling study of Sec. 3.3: Brownian rigid rods
(8 and 27 beads) with Hertz contact at phi 0.01, 0.05, 0.10 and 8192 / 32768
beads, xi = 0.5 and xi = 25/L; it reports t_s (wall time per step per bead)
for every point.

--workload seeds times the step benchmark's mixed path on five independently
generated suspensions of the same workload (median and interquartile
range); --workload oracle-ladder times the CPU oracle on 32, 128 and 512
beads (no GPU); --workload configs runs the scaling study's two other
configurations: 4096 beads at phi 0.1 with xi = 25/L against xi = 0.5 (FP64
and mixed), and the Brownian size ladder of 16-bead aggregates at phi 0.24
(32 768 to 262 144 beads, mixed, both xi)."""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

# The batched form runs one stream per system: 32 hardware work queues (the
# CUDA default is 8) let the systems' graphs run side by side instead of
# sharing 8 queues.  It must be set before the CUDA context exists.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bead-steps/sec at 32k beads (GMRES 1e-6), mixed vs FP64 on GB300; % HBM peak"
UNIT = "bead-steps/s"

WORKLOAD = dict(n_agg=4096, n_b=8, phi=0.2, seed=1, shear=1.0, lub=3.0, xi=0.5, tol=1e-6, dt=1e-3,
                rp=2.0)
SAMPLE_AGG = 4  # oracle sample: 4 aggregates x 8 beads at the same phi / generator


def workload_name(w):
    """The workload, from its defining constants only (both arms print it)."""
    import synth

    L = synth.box_for_phi(w["n_agg"] * w["n_b"], w["phi"])
    return ("%d beads: %d rigid %d-bead random-attachment aggregates, phi %.2f, L %.2f, "
            "shear %g, lubrication %ga, xi %.2f, GMRES %g"
            % (w["n_agg"] * w["n_b"], w["n_agg"], w["n_b"], w["phi"], L, w["shear"], w["lub"],
               w["xi"], w["tol"]))


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of this GPU during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.device_id = device_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- work model
# Algorithmic work per launch of each kernel group.
# FP32 flops of one directed FTS pair (operator form, FMA = 2): geometry 21,
# moment expansion 10, radial table 75 (six coefficients: five Horner steps
# of two flops for seven functions, the interval index), free-space scalars
# 38, operator-form contraction 206
FLOP_PER_PAIR = 350


def group_work(group, s, prm, st, prec_bytes=4):
    """(bound, algorithmic amount per launch, unit) for a kernel group."""
    n = prm["grid"]
    G = n * n * (n + 2)
    Nt = s.n_beads
    w = prec_bytes
    if group == "realspace":
        return "alu", st["n_pairs"] * FLOP_PER_PAIR, "TFLOP/s"
    if group == "spread":
        # write the six density grids once (the grid-centric kernel needs no
        # zeroing pass), read bead moments and positions
        return "hbm", 6 * n ** 3 * w + Nt * (12 * 8 + 4 * w), "GB/s"
    if group == "fft_green":
        # one forward and one inverse 3D transform of six real grids, each
        # reading and writing every grid value once; in a Lees-Edwards box the
        # z pass also reads the three Green's factors of every half-spectrum
        # point (they depend on the wave vector, not only on |k|)
        le = 3 * n * (n // 2 + 1) * n * w if prm.get("flags", 0) & 16 else 0
        return "hbm", 4 * 6 * G * w + le, "GB/s"
    if group == "interp":
        return "hbm", 6 * G * w + Nt * (12 * 8 + 4 * w), "GB/s"
    return "hbm", None, "GB/s"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def traffic_for(group):
    """dram bytes per launch of the group's kernel from the committed ncu
    summary, if the kernel source has not changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(group)
    if not e:
        return None
    src = os.path.join(ROOT, e["source"])
    if not os.path.exists(src):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != e.get("source_sha256_16"):
        return None
    return e["bytes_per_launch"]


def group_roofline(group, ms_per_launch, s, prm, st, pk, pk_kind, alu32):
    """Achieved rate and fraction of the binding peak for one kernel group:
    HBM groups against the measured copy bandwidth, the real-space pair sum
    against the FP32 FMA rate measured in this run (fsd_fma_throughput)."""
    bound, work, unit = group_work(group, s, prm, st)
    r = {"bound": bound, "launch_ms": round(ms_per_launch, 5)}
    if work is None:
        return r
    if bound == "alu":
        achieved = work / (ms_per_launch / 1e3) / 1e12
        peak = alu32 / 1e12
        r.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                  "peak_source": "FP32 FMA rate measured in this run (fsd_fma_throughput)",
                  "flops_per_launch": work})
    else:
        achieved = work / (ms_per_launch / 1e3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        r.update({"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                  "peak_source": "hbm_gbs (%s)" % pk_kind, "bytes_per_launch": work})
    return r


def subbox_reference():
    """The stored oracle solution of the 384-bead accuracy sub-box (written
    by tests/golden/make_subbox_reference.py from the oracle alone)."""
    import importlib.util

    path = os.path.join(ROOT, "tests", "golden", "make_subbox_reference.py")
    spec = importlib.util.spec_from_file_location("make_subbox_reference", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.load()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def accuracy_subbox(pkg, stream):
    """Relative L2 error of U, Omega and S against the dense oracle on a
    384-bead sub-box of the benchmark's suspension (same generator, phi 0.2,
    8-bead aggregates), solved at the benchmark's settings: xi 0.5, default
    P and grid (x_err 1e-6), GMRES 1e-6, r_p 2a, lubrication 3a, graph loop."""
    w = WORKLOAD
    g = subbox_reference()
    out = {"workload": "384 beads: 48 x 8-bead aggregates, phi 0.2, L %.2f, shear 1 (and shear plus "
                       "random aggregate forces / torques)" % g["L"]}
    for name, prec, extra in (("mixed", pkg.FSD_MIXED, 0), ("fp64", pkg.FSD_FP64, 0),
                              ("mixed_fp32_krylov", pkg.FSD_MIXED, pkg.FSD_FLAG_FP32_KRYLOV)):
        s = pkg.Suspension(g["pos"], g["body"], g["L"], stream=stream, precision=prec, xi=w["xi"],
                           tol=w["tol"], lub_cutoff=w["lub"], precond_cutoff=w["rp"],
                           flags=pkg.FSD_FLAG_GRAPH | extra)
        prm = s.params
        errs = {}
        for case, ft in (("shear", None), ("shear+forces", np.ascontiguousarray(g["ft"]))):
            Uref, Sref = g["cases"][case]
            vel, S, st, _ = s.solve(ft, w["shear"])
            errs[case] = {"U": _rel(vel[:, :3], Uref[:, :3]), "Omega": _rel(vel[:, 3:], Uref[:, 3:]),
                          "S": _rel(S, Sref), "iters": st["iters"], "rel_residual": st["rel_residual"]}
        s.close()
        out[name] = errs
        out["grid_P"] = [prm["grid"], prm["P"]]
    out["gate"] = "1e-5 on each of U, Omega, S (tests/test_gpu_benchmark_settings.py)"
    return out


def fft_vs_library(n, xi, L, hand_ms):
    """cuFFT (through torch.fft) on the same six n^3 FP32 grids: forward R2C
    and inverse C2R alone, and with a Green's-function scaling pass between
    them, next to the library's hand-written fused chain (x + y, z with the
    Green's function, y + x; `hand_ms` from the library profiler).  A
    comparison only: the library does not call cuFFT."""
    import torch

    g = torch.randn(6, n, n, n, device="cuda", dtype=torch.float32)
    kk = 2.0 * np.pi / L * torch.fft.fftfreq(n, 1.0 / n, device="cuda", dtype=torch.float32)
    kr = 2.0 * np.pi / L * torch.fft.rfftfreq(n, 1.0 / n, device="cuda", dtype=torch.float32)
    k2 = kk[:, None, None] ** 2 + kk[None, :, None] ** 2 + kr[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    A = (1.0 + k2 / (4 * xi * xi)) * torch.exp(-k2 / (4 * xi * xi)) / k2
    A[0, 0, 0] = 0.0

    def transforms():
        return torch.fft.irfftn(torch.fft.rfftn(g, dim=(1, 2, 3)), s=(n, n, n), dim=(1, 2, 3))

    def with_green():
        sp = torch.fft.rfftn(g, dim=(1, 2, 3))
        sp.mul_(A)
        return torch.fft.irfftn(sp, s=(n, n, n), dim=(1, 2, 3))

    res = {}
    for name, fn in (("cufft_r2c_c2r_ms", transforms), ("cufft_with_green_scaling_ms", with_green)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / 10
    del g, A, k2
    torch.cuda.empty_cache()
    res.update({"hand_written_fused_ms": hand_ms, "grid": n, "fields": 6,
                "note": "same six FP32 real grids, forward and inverse 3D transforms; the hand-written "
                        "chain also applies the full Green's function (projection, Faxen factors, six "
                        "read-out fields), the cuFFT leg a scalar scaling only"})
    res["speedup_hand_written_vs_cufft_transforms"] = res["cufft_r2c_c2r_ms"] / hand_ms
    return res


# ------------------------------------------------------------ oracle arm
def oracle_sample_step(seed):
    import oracle as O
    import synth

    w = WORKLOAD
    pos, body, L = synth.suspension(SAMPLE_AGG, w["n_b"], w["phi"], seed)
    t = time.perf_counter()
    O.solve(pos, body, L, gamma=w["shear"], rlub=w["lub"])
    return len(pos), time.perf_counter() - t


def cpu_baseline(steps=3):
    beads, secs = 0, 0.0
    for k in range(steps):
        b, t = oracle_sample_step(100 + k)
        beads += b
        secs += t
    return {"value": beads / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d oracle solves of a %d-bead sub-box (%d x %d-bead aggregates, phi %.2f, "
                      "same generator, shear and lubrication), dense FP64 Ewald mobility + LAPACK; "
                      "numpy BLAS default threads; %.1f s"
                      % (steps, SAMPLE_AGG * WORKLOAD["n_b"], SAMPLE_AGG, WORKLOAD["n_b"],
                         WORKLOAD["phi"], secs)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    for k in range(args.warmup):
        oracle_sample_step(200 + k)
    beads, secs = 0, 0.0
    for k in range(args.steps):
        b, t = oracle_sample_step(300 + k)
        beads += b
        secs += t
    v = beads / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(WORKLOAD), "beads": WORKLOAD["n_agg"] * WORKLOAD["n_b"],
                       "aggregates": WORKLOAD["n_agg"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "each step one dense oracle solve of a %d-bead sub-box (%d x %d-bead "
                                       "aggregates, same phi, generator, shear and lubrication)"
                                       % (SAMPLE_AGG * WORKLOAD["n_b"], SAMPLE_AGG, WORKLOAD["n_b"])},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ multi-rank helpers
# One process per GPU; ranks step independent work (replicas of the
# suspension, or shards of the batched form) with no data-path collective:
# only the timing is reduced.
def reduce_max(x):
    """Max of x over the ranks of the default process group (x alone when
    there is none)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x):
    """Sum of x over the ranks of the default process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def weak_value(units_local, seconds_local):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return reduce_sum(units_local) / reduce_max(seconds_local)


def shard_by_cost(costs, world):
    """Independent systems assigned to ranks, most expensive first, each to
    the least loaded rank (longest processing time first); returns the
    sorted system indices of every rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


# ------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, local_rank):
    import multiprocessing as mp

    # the batched form's 64 suspensions are generated on host cores while
    # the GPU measurements run (spawned workers, started before CUDA is used)
    jobs = batch_jobs()
    mine = shard_by_cost([int(j[2]) for j in jobs], world)[rank]
    pool = mp.get_context("spawn").Pool(max(1, min(8, (os.cpu_count() or 2) // (2 * world))))
    batch_async = pool.map_async(_batch_system, [jobs[i] for i in mine])
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import synth
    import paper_2607_25161_gb300 as pkg
    from __graft_entry__ import build

    build()
    w = WORKLOAD
    pos, body, L = synth.suspension(w["n_agg"], w["n_b"], w["phi"], w["seed"])
    Nt = len(pos)
    stream = torch.cuda.Stream()
    common = dict(xi=w["xi"], lub_cutoff=w["lub"], tol=w["tol"],
                  flags=pkg.FSD_FLAG_LEES_EDWARDS | pkg.FSD_FLAG_GRAPH, precond_cutoff=w["rp"])

    def make(prec):
        return pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=prec, **common)

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x)

    def timed_steps(s, K, ft=None, vel=None):
        """K steps timed with CUDA events on the library stream."""
        launches, iters = 0, 0
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            st, _ = s.step(ft, w["shear"], w["dt"], vel=vel)
            launches += st["kernel_launches"]
            iters += st["iters"]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1), launches, iters

    # ---- mixed (headline)
    s = make(pkg.FSD_MIXED)
    prm = s.params
    for _ in range(args.warmup):
        s.step(None, w["shear"], w["dt"])
    dev_id = local_rank
    if os.environ.get("CUDA_VISIBLE_DEVICES"):
        ids = os.environ["CUDA_VISIBLE_DEVICES"].split(",")
        if local_rank < len(ids):
            dev_id = ids[local_rank]
    clk = ClockSampler(dev_id)
    clk.start()
    ms, launches, iters = timed_steps(s, args.steps)
    clocks = clk.stop()
    ms_max = max_over_ranks(ms)
    value = Nt * args.steps * world / (ms_max / 1e3)

    s.close()

    # ---- end to end: pinned host input and output every step (fresh context)
    s = make(pkg.FSD_MIXED)
    # its first solve, on the initial configuration, is compared with the
    # FP64 path's below (the 32768-bead system is too large for the oracle)
    v_mixed, S_mixed, _, _ = s.solve(None, w["shear"])
    for _ in range(args.warmup):
        s.step(None, w["shear"], w["dt"])
    ft_h = torch.zeros((w["n_agg"], 6), dtype=torch.float64).pin_memory()
    vel_h = torch.zeros((w["n_agg"], 6), dtype=torch.float64).pin_memory()
    K2 = max(3, args.steps // 2)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K2):
        s.step(ft_h, w["shear"], w["dt"], vel=vel_h)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": Nt * K2 * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(ft_h.numel() * 8), "d2h_bytes_per_step": int(vel_h.numel() * 8),
           "steps": K2, "api": "fsd_step with pinned host force/torque in and velocities out"}
    s.close()

    # ---- profile pass: per kernel group device time (fresh context, separate run)
    s = make(pkg.FSD_MIXED)
    for _ in range(min(args.warmup, 3)):
        s.step(None, w["shear"], w["dt"])
    s.profile(True)
    PS = 2
    stp = None
    prof_iters = 0
    for _ in range(PS):
        stp, _ = s.step(None, w["shear"], w["dt"])
        prof_iters += stp["iters"]
    prof = s.profile_read()
    s.profile(False)
    # FP32 operator applications alone (real space + wave space), for the
    # roofline: per-application group times, free of the step's one FP64
    # application and of the split of a group over several timed scopes
    KA = 10
    Fa = np.random.default_rng(5).normal(size=(Nt, 11))
    ua = np.zeros((Nt, 11))
    s.apply_mobility(Fa, part=3, precision=pkg.FSD_MIXED, out=ua)
    s.profile(True)
    for _ in range(KA):
        s.apply_mobility(Fa, part=3, precision=pkg.FSD_MIXED, out=ua)
    prof_op = s.profile_read()
    s.profile(False)
    s.close()

    # ---- warm start (initial guess = previous step's solution), reported beside
    s = pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=pkg.FSD_MIXED,
                       **dict(common, flags=common["flags"] | pkg.FSD_FLAG_WARM_START))
    for _ in range(args.warmup):
        s.step(None, w["shear"], w["dt"])
    msw, _, itw = timed_steps(s, args.steps)
    s.close()
    msw = max_over_ranks(msw)
    warm = {"value": Nt * args.steps * world / (msw / 1e3), "ms_per_step": msw / args.steps,
            "iters_per_step": itw / args.steps,
            "note": "same workload and tolerance; GMRES starts from the previous step's solution"}

    # ---- FP32 inner Krylov basis (FSD_FLAG_FP32_KRYLOV), reported beside
    s = pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=pkg.FSD_MIXED,
                       **dict(common, flags=common["flags"] | pkg.FSD_FLAG_FP32_KRYLOV))
    v_k32, S_k32, _, _ = s.solve(None, w["shear"])
    for _ in range(args.warmup):
        s.step(None, w["shear"], w["dt"])
    msk, _, itk = timed_steps(s, args.steps)
    s.close()
    msk = max_over_ranks(msk)
    fp32_krylov = {"value": Nt * args.steps * world / (msk / 1e3), "ms_per_step": msk / args.steps,
                   "iters_per_step": itk / args.steps,
                   "note": "same workload and tolerance with FSD_FLAG_FP32_KRYLOV: the inner GMRES "
                           "keeps its Krylov bases in FP32 and orthogonalises with FP32 products "
                           "(FP64 refinement residual, Hessenberg and LU); not the headline, whose "
                           "Arnoldi orthogonalisation is FP64"}

    # ---- Brownian step: fsd_brownian (PSE far-field slip: analytic wave
    #      part + Lanczos real-space square root; near-field force by the
    #      default pairwise sampler) before each step, kT = 1 (same workload)
    s = make(pkg.FSD_MIXED)
    for k in range(args.warmup):
        s.brownian(1.0, w["dt"], seed=11, step=k, outputs=False)
        s.step(None, w["shear"], w["dt"])
    barrier()
    torch.cuda.synchronize()
    eb0 = torch.cuda.Event(enable_timing=True)
    eb1 = torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    lz_r = lz_n = itb = 0
    lz_ch = 0.0
    for k in range(args.steps):
        _, _, stb = s.brownian(1.0, w["dt"], seed=11, step=1000 + k, outputs=False)
        lz_r += stb["iters"]
        lz_n += stb["outer_iters"]
        lz_ch = max(lz_ch, stb["rel_residual"])
        stb2, _ = s.step(None, w["shear"], w["dt"])
        itb += stb2["iters"]
    eb1.record(stream)
    torch.cuda.synchronize()
    s.close()
    msb = max_over_ranks(eb0.elapsed_time(eb1))
    brown = {"value": Nt * args.steps * world / (msb / 1e3), "ms_per_step": msb / args.steps,
             "kT": 1.0, "dt": w["dt"], "iters_per_step": itb / args.steps,
             "lanczos_real_per_step": lz_r / args.steps, "lanczos_real_last_change_max": lz_ch,
             "near_field_sampler": "pairwise (library default): sum_p K_p^T psi_p, K_p the pair model's "
                                   "dissipation-form factor; covariance exactly R_FU^nf, no iteration",
             "note": "each step: PSE far-field slip (analytic wave part + Lanczos real-space square root, "
                     "FP32 operator) and the near-field Brownian force, then the mixed solve with them; "
                     "drift not included (see brownian_drift)"}

    # ---- the same workload in the co-moving cube (FSD_FLAG_COMOVING: no
    #      sheared images, bodies move by their disturbance velocity only)
    s = pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=pkg.FSD_MIXED,
                       **dict(common, flags=pkg.FSD_FLAG_COMOVING | pkg.FSD_FLAG_GRAPH))
    for _ in range(min(args.warmup, 3)):
        s.step(None, w["shear"], w["dt"])
    barrier()
    torch.cuda.synchronize()
    el0 = torch.cuda.Event(enable_timing=True)
    el1 = torch.cuda.Event(enable_timing=True)
    el0.record(stream)
    its_le = []
    for _ in range(args.steps):
        stl, _ = s.step(None, w["shear"], w["dt"])
        its_le.append(stl["iters"])
    el1.record(stream)
    torch.cuda.synchronize()
    s.close()
    msl = max_over_ranks(el0.elapsed_time(el1))
    lees = {"value": Nt * args.steps * world / (msl / 1e3), "ms_per_step": msl / args.steps,
            "iters_first_last": [its_le[0], its_le[-1]],
            "note": "co-moving cube (no sheared images; disturbance velocity only), one graph per step"}

    # ---- the same Brownian step with the paper's near-field sampler
    #      (preconditioned Lanczos, Sec. 2.2)
    s = pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=pkg.FSD_MIXED,
                       **dict(common, nf_sampler=pkg.FSD_NF_LANCZOS))
    for k in range(min(args.warmup, 3)):
        s.brownian(1.0, w["dt"], seed=11, step=k, outputs=False)
        s.step(None, w["shear"], w["dt"])
    barrier()
    torch.cuda.synchronize()
    ep0 = torch.cuda.Event(enable_timing=True)
    ep1 = torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    lz_n = 0
    lz_ch = 0.0
    for k in range(args.steps):
        _, _, stl = s.brownian(1.0, w["dt"], seed=11, step=1000 + k, outputs=False)
        lz_n += stl["outer_iters"]
        lz_ch = max(lz_ch, stl["rel_residual"])
        s.step(None, w["shear"], w["dt"])
    ep1.record(stream)
    torch.cuda.synchronize()
    s.close()
    msp = max_over_ranks(ep0.elapsed_time(ep1))
    brown["lanczos_near_field"] = {
        "value": Nt * args.steps * world / (msp / 1e3), "ms_per_step": msp / args.steps,
        "lanczos_near_per_step": lz_n / args.steps, "lanczos_last_change_max": lz_ch,
        "note": "near-field force by the paper's preconditioned Lanczos (block-Cholesky "
                "preconditioner, stopping at lanczos_tol 1e-7 or 60 steps; the last relative change "
                "is reported)"}

    # ---- Brownian step with the drift (Sec. 2.4; appendix on the drift):
    #      fsd_brownian, fsd_drift (two solves at displaced configurations),
    #      then the step's solve: three solves per step either way
    drift_lines = {}
    for dname, meth in (("rfd", pkg.FSD_DRIFT_RFD), ("fixman", pkg.FSD_DRIFT_FIXMAN)):
        s = make(pkg.FSD_MIXED)

        def one(k):
            s.brownian(1.0, w["dt"], seed=11, step=k, outputs=False)
            _, _, _, std, _ = s.drift(meth, 1.0, dt=w["dt"], seed=11, step=k, outputs=False)
            st2, _ = s.step(None, w["shear"], w["dt"])
            return std["iters"] + st2["iters"]
        for k in range(min(args.warmup, 3)):
            one(k)
        KD = max(3, args.steps // 2)
        barrier()
        torch.cuda.synchronize()
        ed0 = torch.cuda.Event(enable_timing=True)
        ed1 = torch.cuda.Event(enable_timing=True)
        ed0.record(stream)
        itd = sum(one(2000 + k) for k in range(KD))
        ed1.record(stream)
        torch.cuda.synchronize()
        s.close()
        msd = max_over_ranks(ed0.elapsed_time(ed1))
        drift_lines[dname] = {"value": Nt * KD * world / (msd / 1e3), "ms_per_step": msd / KD,
                              "steps": KD, "iters_per_step": itd / KD, "solves_per_step": 3}
    drift_lines["note"] = ("kT = 1: Brownian terms, the drift by RFD (eps = tol^(1/3) a) or the modified "
                           "Fixman midpoint (m = 100), then the step's mixed solve and update")

    # ---- plain FP64 path on the same initial configuration
    s64 = make(pkg.FSD_FP64)
    v_64, S_64, _, _ = s64.solve(None, w["shear"])
    agree = {"U": _rel(v_mixed[:, :3], v_64[:, :3]), "Omega": _rel(v_mixed[:, 3:], v_64[:, 3:]),
             "S": _rel(S_mixed, S_64),
             "fp32_krylov": {"U": _rel(v_k32[:, :3], v_64[:, :3]),
                             "Omega": _rel(v_k32[:, 3:], v_64[:, 3:]), "S": _rel(S_k32, S_64)},
             "note": "mixed (and mixed with the FP32 inner Krylov basis) vs plain FP64 GPU solve of "
                     "the 32768-bead initial configuration, all at GMRES 1e-6 (relative L2)"}
    for _ in range(max(1, min(args.warmup, 2))):
        s64.step(None, w["shear"], w["dt"])
    K64 = max(2, min(args.steps, 5))
    ms64, _, iters64 = timed_steps(s64, K64)
    s64.profile(True)
    st64, _ = s64.step(None, w["shear"], w["dt"])
    prof64 = s64.profile_read()
    s64.close()
    ms64 = max_over_ranks(ms64)
    fp64 = {"value": Nt * K64 * world / (ms64 / 1e3), "ms_per_step": ms64 / K64, "steps": K64,
            "iters_per_step": iters64 / K64,
            "kernel_ms_per_step": {g: round(v[0], 4) for g, v in prof64.items()}}

    # ---- batched form: 64 independent suspensions advanced together, and
    #      the same contexts one at a time (no autotuning on either side)
    systems_mine = batch_async.get()
    pool.close()
    pool.join()
    Bt, _, batch = batch_measure(pkg, systems_mine, max(3, min(args.steps, 5)), 3, tuned=False,
                                 world=world)
    Bt.close()
    nj = [int(j[2]) for j in jobs]
    batch["workload"] = ("%d suspensions, %d beads (%d..%d per system, log-uniform), aggregate sizes "
                         "2..64, phi 0.05..0.3, shear 1, lubrication 3a, GMRES 1e-6, mixed, default xi"
                         % (len(jobs), sum(nj), min(nj), max(nj)))
    batch["execution"] = ("fsd_step_batch: one CUDA graph per system and step on its own stream, all "
                          "systems in flight, CUDA_DEVICE_MAX_CONNECTIONS=%s"
                          % os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8")
                          + ("; systems sharded over ranks" if world > 1 else ""))

    # ---- measured arithmetic peaks, accuracy against the oracle, cuFFT
    alu32 = pkg.fma_throughput(32, stream.cuda_stream)
    alu64 = pkg.fma_throughput(64, stream.cuda_stream)
    accuracy = accuracy_subbox(pkg, stream.cuda_stream)
    accuracy["agreement_32768_beads"] = agree
    fftcmp = fft_vs_library(prm["grid"], w["xi"], L, prof_op["fft_green"][0] / KA)

    if rank != 0:
        return

    # ---- roofline of every kernel group of an FP32 operator application
    #      (the work the Krylov iterations repeat); the dominant one leads
    pk, pk_kind = peaks()
    op_groups = ("realspace", "spread", "fft_green", "interp")
    dom = max(op_groups, key=lambda g: prof_op[g][0])
    groups = {g: group_roofline(g, prof_op[g][0] / KA, s, prm, stp, pk, pk_kind, alu32)
              for g in op_groups}
    for g in op_groups:
        groups[g]["traffic"] = traffic_for(g)
    roof = {"kernel_group": dom}
    roof.update(groups[dom])
    roof.update({"launch": "one FP32 operator application (the group's kernels), mean of %d" % KA,
                 "groups": groups,
                 "measured_fma": {"fp32_tflops": alu32 / 1e12, "fp64_tflops": alu64 / 1e12,
                                  "how": "fsd_fma_throughput: independent FMA chains on every SM, "
                                         "best of 3 launches, CUDA events"}})

    base = cpu_baseline(3) if world == 1 or rank == 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload_name(w), "beads": Nt, "aggregates": w["n_agg"],
                   "method": "grid %d^3, P %d (wave-space operator error ~7e-7), rc %.2f"
                             % (prm["grid"], prm["P"], prm["rc"]),
                   "precision": "mixed: FP32 operator in FP64 iterative refinement; FP64 Arnoldi, residual, LU",
                   "l2": "working set per step > L2 (grids, Krylov basis, neighbour lists ~0.5 GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "initial_guess": "zero each step",
                   "execution": "each step's solve and rigid-body update as one CUDA graph "
                                "(GMRES loops as conditional nodes); geometry prepared before it",
                   "precond_cutoff": "r_p = %ga: per-aggregate Schur blocks without near-field pairs "
                                     "(the paper's 2.1a lets GMRES iterations grow 59 -> 150 over 30 steps "
                                     "on this workload; same 1e-6 tolerance either way)" % w["rp"],
                   "integration": "Lees-Edwards box: bodies move by their full velocity, the periodic images "
                                  "across y by shear L dt per step (sheared images in every operator)"},
        "iters_per_step": iters / args.steps,
        "fp64": fp64,
        "kernel_ms_per_step": {g: round(v[0] / PS, 4) for g, v in prof.items()},
        "profile_iters_per_step": prof_iters / PS,
        "warm_start": warm,
        "fp32_krylov": fp32_krylov,
        "brownian": brown,
        "brownian_drift": drift_lines,
        "comoving_cube": lees,
        "accuracy": accuracy,
        "fft_vs_library": fftcmp,
        "batch": batch,
        "roofline": roof,
        "cpu_baseline": base,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------ ncu target
def run_profile(args, local_rank):
    """Mixed steps of the benchmark workload through the host-driven loop, so
    that every kernel is an ordinary launch an ncu capture can see."""
    import torch

    torch.cuda.set_device(local_rank)
    import synth
    import paper_2607_25161_gb300 as pkg
    from __graft_entry__ import build

    build()
    w = WORKLOAD
    pos, body, L = synth.suspension(w["n_agg"], w["n_b"], w["phi"], w["seed"])
    s = pkg.Suspension(pos, body, L, precision=pkg.FSD_MIXED, xi=w["xi"], lub_cutoff=w["lub"],
                       tol=w["tol"], flags=pkg.FSD_FLAG_LEES_EDWARDS, precond_cutoff=w["rp"])
    for _ in range(args.warmup):
        st, _ = s.step(None, w["shear"], w["dt"])
    torch.cuda.synchronize()
    # the timed steps inside one NVTX range (ncu --nvtx --nvtx-include "timed_steps/")
    torch.cuda.nvtx.range_push("timed_steps")
    launches = []
    for _ in range(args.steps):
        st, _ = s.step(None, w["shear"], w["dt"])
        launches.append(st["kernel_launches"])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    s.close()
    print("profile run: %d warm-up and %d timed steps, %d iterations and %s kernel launches in the "
          "timed steps" % (args.warmup, args.steps, st["iters"], launches))


# ---------------------------------------------------------- batched form
BATCH = dict(n_sys=64, seed=4, n_lo=256, n_hi=8192, phi_lo=0.05, phi_hi=0.3, size_lo=2, size_hi=64,
             shear=1.0, lub=3.0, tol=1e-6, dt=1e-3, rp=2.0)


def _batch_system(args_):
    import synth

    s, seed, n, phi = args_
    pos, body, L = synth.mixed_suspension(int(n), float(phi), seed * 1000 + s, BATCH["size_lo"],
                                          BATCH["size_hi"])
    return pos, body, L


def batch_systems():
    """The batched workload, generated in parallel (spawned workers: no
    process is forked after CUDA is initialised)."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        return pool.map(_batch_system, batch_jobs())


def batch_jobs():
    b = BATCH
    rng = np.random.default_rng(b["seed"])
    n = np.rint(np.exp(rng.uniform(np.log(b["n_lo"]), np.log(b["n_hi"]), size=b["n_sys"]))).astype(int)
    phi = rng.uniform(b["phi_lo"], b["phi_hi"], size=b["n_sys"])
    return [(s, b["seed"], n[s], phi[s]) for s in range(b["n_sys"])]


def batch_measure(pkg, systems, steps, warmup, tuned, world=1):
    """The batched form on `systems`: fsd_step_batch timed over `steps`
    steps (wall clock, device synchronised on both sides), end to end with
    pinned host forces in and velocities out, and the same contexts stepped
    one at a time.  tuned: FSD_FLAG_AUTOTUNE per system (both sides use the
    same contexts either way)."""
    import torch

    b = BATCH
    nb = sum(len(p) for p, _, _ in systems)
    flags = pkg.FSD_FLAG_COMOVING | (pkg.FSD_FLAG_AUTOTUNE if tuned else 0)
    prm = dict(precision=pkg.FSD_MIXED, tol=b["tol"], lub_cutoff=b["lub"], precond_cutoff=b["rp"],
               flags=flags)
    t_set = time.perf_counter()
    B = pkg.Batch(systems, prm)
    t_set = time.perf_counter() - t_set
    rates = np.full(B.n_sys, b["shear"])
    for _ in range(warmup):
        B.step(None, rates, b["dt"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters = launches = 0
    for _ in range(steps):
        st, _ = B.step(None, rates, b["dt"])
        iters += sum(x["iters"] for x in st)
        launches += sum(x["kernel_launches"] for x in st)
    torch.cuda.synchronize()
    dt_b = time.perf_counter() - t0
    value = weak_value(nb * steps, dt_b)
    dt_b = reduce_max(dt_b)
    ft_h = torch.zeros((B.n_agg, 6), dtype=torch.float64).pin_memory()
    vel_h = torch.zeros((B.n_agg, 6), dtype=torch.float64).pin_memory()
    K2 = max(2, steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K2):
        B.step(ft_h, rates, b["dt"], vel=vel_h)
    torch.cuda.synchronize()
    e2e_value = weak_value(nb * K2, time.perf_counter() - t0)
    views = [B.system(k) for k in range(B.n_sys)]
    for v in views:  # untimed: each view captures its own step graph first
        v.step(None, b["shear"], b["dt"])
    K1 = max(2, min(steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K1):
        for v in views:
            v.step(None, b["shear"], b["dt"])
    torch.cuda.synchronize()
    dt_1 = time.perf_counter() - t0
    one = weak_value(nb * K1, dt_1)
    out = {"value": value, "unit": UNIT, "ms_per_step": dt_b / steps * 1e3, "steps": steps,
           "beads": nb, "systems": len(systems), "iters_per_system_step": iters / (steps * len(systems)),
           "setup_s": round(t_set, 1), "autotuned": bool(tuned),
           "one_at_a_time": {"value": one, "ms_per_step": dt_1 / K1 * 1e3, "steps": K1,
                             "note": "the same contexts (same parameters) stepped sequentially with fsd_step"},
           "speedup_batched": value / one,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(ft_h.numel() * 8),
                   "d2h_bytes_per_step": int(vel_h.numel() * 8), "steps": K2,
                   "api": "fsd_step_batch with pinned host forces in and velocities out"},
           "gpu_launches": int(reduce_sum(launches))}
    return B, views, out


def run_batch(args, rank, world, local_rank):
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2607_25161_gb300 as pkg
    from __graft_entry__ import build

    t_gen = time.perf_counter()
    systems_all = batch_systems()
    t_gen = time.perf_counter() - t_gen
    # N > 1: each rank advances its share of the independent systems
    mine = shard_by_cost([len(p) for p, _, _ in systems_all], world)[rank]
    systems = [systems_all[i] for i in mine]
    build()
    b = BATCH
    clk = ClockSampler(local_rank)
    clk.start()
    if dist is not None:
        dist.barrier()
    B, views, meas = batch_measure(pkg, systems, args.steps, args.warmup, tuned=True, world=world)
    clocks = clk.stop()
    value = meas["value"]
    # dominant kernel group of the largest system, profiled alone
    big = int(np.argmax([len(p) for p, _, _ in systems]))
    sv = views[big]
    sv.profile(True)
    stp, _ = sv.step(None, b["shear"], b["dt"])
    prof = sv.profile_read()
    sv.profile(False)
    sprm = sv.params
    pk, pk_kind = peaks()
    dom = max((g for g in prof if prof[g][1] > 0), key=lambda g: prof[g][0])
    per_launch_ms = prof[dom][0] / prof[dom][1]
    bound, work, unit = group_work(dom, sv, sprm, stp)
    roof = {"kernel_group": dom, "bound": bound, "launch_ms": per_launch_ms,
            "system": "largest of the batch (%d beads, grid %d^3), profiled alone" % (len(systems[big][0]),
                                                                                   sprm["grid"])}
    if work is not None and bound != "alu":
        achieved = work / (per_launch_ms / 1e3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        roof.update({"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": "hbm_gbs (%s)" % pk_kind, "bytes_per_launch": work})
    elif work is not None:
        peak = pkg.fma_throughput(32) / 1e12
        achieved = work / (per_launch_ms / 1e3) / 1e12
        roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": "FP32 FMA rate measured in this run (fsd_fma_throughput)",
                     "flops_per_launch": work})
    roof["traffic"] = None
    xis = sorted(set(round(p["xi"], 3) for p in B.params))
    B.close()
    if rank != 0:
        return
    line = {
        "metric": "bead-steps/sec of 64 independent suspensions advanced together (GMRES 1e-6, mixed)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": meas["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batched form: %d suspensions, %d beads (%d..%d per system, log-uniform), "
                               "aggregate sizes 2..64, phi 0.05..0.3, shear 1, lubrication 3a, GMRES 1e-6"
                               % (len(systems_all), sum(len(p) for p, _, _ in systems_all),
                                  min(len(p) for p, _, _ in systems_all),
                                  max(len(p) for p, _, _ in systems_all)),
                   "parallelism": ("systems sharded over %d ranks by bead count (no collective; "
                                   "rank 0's roofline and statistics)" % world) if world > 1 else "single GPU",
                   "autotune": "xi per system by timing (chosen: %s), real-space tile per system" % xis,
                   "execution": "fsd_step_batch: one CUDA graph per system and step on its own stream, "
                                "all systems in flight; launch phase on 8 host threads; "
                                "CUDA_DEVICE_MAX_CONNECTIONS=%s" % os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8"),
                   "l2": "working set > L2 (64 grids and Krylov bases)",
                   "generation_s": round(t_gen, 1), "setup_s": meas["setup_s"]},
        "one_at_a_time": dict(meas["one_at_a_time"], speedup_batched=meas["speedup_batched"]),
        "iters_per_system_step": meas["iters_per_system_step"],
        "roofline": roof,
        "cpu_baseline": cpu_baseline(3),
        "e2e": meas["e2e"],
        "gpu_launches": meas["gpu_launches"],
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- oracle ladder
def run_oracle_ladder(args):
    """The CPU oracle (dense FP64 Ewald mobility + LAPACK) on 8-bead
    aggregate suspensions of 32, 128 and 512 beads at phi 0.1 (the
    512-aggregate workload's generator): seconds per solve, bead-steps/s,
    and the power law t ~ N^p fitted through the ladder.  CPU only."""
    import oracle as O
    import synth

    pts = []
    for n_agg in (4, 16, 64):
        pos, body, L = synth.suspension(n_agg, 8, 0.1, 1)
        t = time.perf_counter()
        O.solve(pos, body, L, gamma=1.0, rlub=3.0)
        dt = time.perf_counter() - t
        pts.append({"beads": len(pos), "seconds": round(dt, 3), "bead_steps_per_s": len(pos) / dt})
    x = np.log([q["beads"] for q in pts])
    y = np.log([q["seconds"] for q in pts])
    p = float(np.polyfit(x, y, 1)[0])
    print(json.dumps({"impl": "reference", "workload": "oracle ladder, 8-bead aggregates, phi 0.1",
                      "points": pts, "cost_exponent": p, "cores": os.cpu_count()}), flush=True)


# ------------------------------------------------------------ seed spread
SEEDS = (1, 2, 3, 4, 5)


def _seed_system(seed):
    import synth

    w = WORKLOAD
    return synth.suspension(w["n_agg"], w["n_b"], w["phi"], seed)


def run_seeds(args, local_rank):
    """The step benchmark (mixed, one graph per step) on independently
    generated suspensions of the same workload: median and interquartile
    range of bead-steps/s over the seeds."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(min(len(SEEDS), os.cpu_count() or 1)) as pool:
        systems = pool.map(_seed_system, SEEDS)
    import torch

    torch.cuda.set_device(local_rank)
    import paper_2607_25161_gb300 as pkg
    from __graft_entry__ import build

    build()
    w = WORKLOAD
    stream = torch.cuda.Stream()
    clk = ClockSampler(local_rank)
    clk.start()
    vals, its = [], []
    for seed, (pos, body, L) in zip(SEEDS, systems):
        s = pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=pkg.FSD_MIXED,
                           xi=w["xi"], lub_cutoff=w["lub"], tol=w["tol"], precond_cutoff=w["rp"],
                           flags=pkg.FSD_FLAG_COMOVING | pkg.FSD_FLAG_GRAPH)
        for _ in range(args.warmup):
            s.step(None, w["shear"], w["dt"])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it = 0
        for _ in range(args.steps):
            st, _ = s.step(None, w["shear"], w["dt"])
            it += st["iters"]
        e1.record(stream)
        torch.cuda.synchronize()
        s.close()
        vals.append(len(pos) * args.steps / (e0.elapsed_time(e1) / 1e3))
        its.append(it / args.steps)
    clocks = clk.stop()
    q1, med, q3 = (float(np.percentile(vals, q)) for q in (25, 50, 75))
    print(json.dumps({"metric": METRIC, "workload": workload_name(w), "seeds": list(SEEDS),
                      "values": vals, "iters_per_step": its, "median": med, "iqr": [q1, q3],
                      "unit": UNIT, "steps": args.steps, "warmup": args.warmup, "clocks": clocks}),
          flush=True)


# ------------------------------------------------------ rod scaling study
# Sec. 3.3: N Brownian rigid rods of n_b beads in a periodic cube with normal
# contact between rods; t_s = wall time per step per bead at phi in {0.01,
# 0.05, 0.10}, n_b in {8, 27}, xi = 0.5 and xi = 25/L.
RODS = dict(n_b=(8, 27), phi=(0.01, 0.05, 0.10), n_tot=(8192, 32768), kT=1.0, dt=1e-3, kn=1e4,
            lub=3.0, rp=2.0, tol=1e-6, seed=7)


def _rod_system(args_):
    import synth

    nb, phi, n_tot = args_
    return synth.rod_suspension(n_tot // nb, nb, phi, RODS["seed"])


def rod_points():
    import synth

    pts = []
    for nb in RODS["n_b"]:
        for phi in RODS["phi"]:
            for n in RODS["n_tot"]:
                L = synth.box_for_phi((n // nb) * nb, phi)
                if 2.0 * nb < 0.5 * L:  # a rod must be shorter than half the box
                    pts.append((nb, phi, n))
    return pts


def run_rods(args, local_rank):
    import multiprocessing as mp

    pts = rod_points()
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        systems = pool.map(_rod_system, pts)
    t_gen = time.perf_counter() - t0
    import torch

    torch.cuda.set_device(local_rank)
    import paper_2607_25161_gb300 as pkg
    from __graft_entry__ import build

    build()
    r = RODS
    stream = torch.cuda.Stream()
    dev_id = local_rank
    if os.environ.get("CUDA_VISIBLE_DEVICES"):
        ids = os.environ["CUDA_VISIBLE_DEVICES"].split(",")
        if local_rank < len(ids):
            dev_id = ids[local_rank]
    clk = ClockSampler(dev_id)
    clk.start()
    K = max(3, min(args.steps, 5))
    out = []
    launches = 0
    for (nb, phi, n), (pos, body, L) in zip(pts, systems):
        for xi_mode in ("0.5", "25/L"):
            xi = 0.5 if xi_mode == "0.5" else 25.0 / L
            s = pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=pkg.FSD_MIXED, xi=xi,
                               lub_cutoff=r["lub"], precond_cutoff=r["rp"], tol=r["tol"],
                               flags=pkg.FSD_FLAG_GRAPH)
            prm = s.params
            ft = torch.zeros((s.n_agg, 6), dtype=torch.float64, device="cuda")
            ok = (pkg.FSD_OK, pkg.FSD_EOVERLAP)

            def one(k):
                s.brownian(r["kT"], r["dt"], seed=r["seed"], step=k, outputs=False)
                s.contact(r["kn"], out=ft)
                st, _ = s.step(ft, 0.0, r["dt"], allow=ok)
                return st
            for k in range(min(args.warmup, 3)):
                one(k)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            its = 0
            for k in range(K):
                st = one(100 + k)
                its += st["iters"]
                launches += st["kernel_launches"]
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            s.close()
            out.append({"n_b": nb, "phi": phi, "beads": len(pos), "L": round(L, 2), "xi": xi_mode,
                        "xi_value": round(xi, 4), "rc": round(prm["rc"], 2), "grid": prm["grid"],
                        "ms_per_step": round(ms, 3), "t_s_us": round(1e3 * ms / len(pos), 4),
                        "bead_steps_per_s": round(len(pos) / (ms / 1e3), 1), "iters_per_step": its / K})
            print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    clocks = clk.stop()
    head = next(p for p in out if p["n_b"] == 8 and p["phi"] == 0.10 and p["beads"] == 32768
                and p["xi"] == "0.5")
    line = {
        "metric": "t_s: wall time per step per bead of Brownian rigid rods (Sec. 3.3 scaling study)",
        "value": head["bead_steps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "rods: n_b %s, phi %s, N_tot %s, xi 0.5 and 25/L; value = the 8-bead, "
                               "phi 0.10, 32768-bead, xi 0.5 point" % (r["n_b"], r["phi"], r["n_tot"]),
                   "step": "fsd_brownian (kT 1) + fsd_contact_forces (Hertz, kn 1e4 kT/a^1.5) + fsd_step "
                           "(mixed, GMRES 1e-6, lubrication 3a, one graph), dt 1e-3, no shear, no drift",
                   "generation_s": round(t_gen, 1)},
        "points": out,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------- configurations 2 and 5
# Config 2: 512 x 8-bead aggregates (4096 beads) at phi 0.1, shear 1,
# lubrication 3a, the plain FP64 method with xi = 25/L (the size rule) and
# xi = 0.5, 100 steps.  Config 5: 16-bead aggregates, lubrication 3a, shear
# 0.1, Brownian (kT 1, PSE), mixed, xi = 0.5 and 25/L, scaling in N at
# 32768, 65536, 131072 and 262144 beads.
CFG2 = dict(n_agg=512, n_b=8, phi=0.1, seed=2, shear=1.0, lub=3.0, tol=1e-6, dt=1e-3, rp=2.0)
CFG5 = dict(n_b=16, phi=0.24, seed=5, shear=0.1, lub=3.0, tol=1e-6, dt=1e-3, rp=2.0, kT=1.0,
            base_aggs=(256, 512, 1024, 2048))


def _cfg5_base(n_agg):
    import synth

    c = CFG5
    return synth.dense_suspension(n_agg, c["n_b"], c["phi"], c["seed"])


def _time_steps(pkg, s, stream, K, warm, shear, dt, brownian_kT=0.0):
    import torch

    def one(k):
        if brownian_kT > 0:
            s.brownian(brownian_kT, dt, seed=17, step=k, outputs=False)
        st, _ = s.step(None, shear, dt)
        return st
    for k in range(warm):
        one(k)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its = launches = 0
    for k in range(K):
        st = one(100 + k)
        its += st["iters"]
        launches += st["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / K, its / K, launches


def run_configs(args, local_rank):
    """Configurations 2 and 5: one JSON line with every point."""
    import multiprocessing as mp

    c5 = CFG5
    pool = mp.get_context("spawn").Pool(len(c5["base_aggs"]))
    bases = pool.imap(_cfg5_base, c5["base_aggs"])  # smallest first
    import torch

    torch.cuda.set_device(local_rank)
    import synth
    import paper_2607_25161_gb300 as pkg
    from __graft_entry__ import build

    build()
    stream = torch.cuda.Stream()
    clk = ClockSampler(local_rank)
    clk.start()
    launches = 0
    # ---- config 2
    c2 = CFG2
    pos, body, L = synth.suspension(c2["n_agg"], c2["n_b"], c2["phi"], c2["seed"])
    L2 = L
    K2 = args.steps
    cfg2 = []
    for prec, pname in ((pkg.FSD_FP64, "fp64"), (pkg.FSD_MIXED, "mixed")):
        for xi_mode in ("25/L", "0.5"):
            xi = 25.0 / L if xi_mode == "25/L" else 0.5
            s = pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=prec, xi=xi,
                               lub_cutoff=c2["lub"], tol=c2["tol"], precond_cutoff=c2["rp"],
                               flags=pkg.FSD_FLAG_COMOVING | pkg.FSD_FLAG_GRAPH)
            prm = s.params
            ms, its, nl = _time_steps(pkg, s, stream, K2, 3, c2["shear"], c2["dt"])
            launches += nl
            s.close()
            cfg2.append({"precision": pname, "xi": xi_mode, "xi_value": round(xi, 4),
                         "rc": round(prm["rc"], 3), "grid": prm["grid"], "ms_per_step": round(ms, 4),
                         "bead_steps_per_s": len(pos) * 1e3 / ms, "iters_per_step": its})
            print(json.dumps(dict(cfg2[-1], config=2)), file=sys.stderr, flush=True)
    # ---- config 5: each size is the 2 x 2 x 2 periodic replica of a base box
    cfg5 = []
    K5 = max(3, min(args.steps, 10))
    for n_agg, (bp, bb, bL) in zip(c5["base_aggs"], bases):
        pos, body, Ls = synth.replicate_box(bp, bb, bL, (2, 2, 2))
        L = Ls[0]
        phi = len(pos) * 4.0 / 3.0 * np.pi / L ** 3
        for xi_mode in ("0.5", "25/L"):
            xi = 25.0 / L if xi_mode == "25/L" else 0.5
            s = pkg.Suspension(pos, body, L, stream=stream.cuda_stream, precision=pkg.FSD_MIXED, xi=xi,
                               lub_cutoff=c5["lub"], tol=c5["tol"], precond_cutoff=c5["rp"],
                               flags=pkg.FSD_FLAG_COMOVING | pkg.FSD_FLAG_GRAPH)
            prm = s.params
            ms, its, nl = _time_steps(pkg, s, stream, K5, 3, c5["shear"], c5["dt"], c5["kT"])
            launches += nl
            s.close()
            cfg5.append({"beads": len(pos), "aggregates": int(body.max()) + 1, "L": round(L, 3),
                         "phi": round(phi, 4), "xi": xi_mode, "xi_value": round(xi, 4),
                         "rc": round(prm["rc"], 3), "grid": prm["grid"], "ms_per_step": round(ms, 3),
                         "bead_steps_per_s": len(pos) * 1e3 / ms, "t_s_us": 1e3 * ms / len(pos),
                         "iters_per_step": its})
            print(json.dumps(dict(cfg5[-1], config=5)), file=sys.stderr, flush=True)
    pool.close()
    pool.join()
    clocks = clk.stop()
    head = next(p for p in cfg5 if p["beads"] == 262144 and p["xi"] == "0.5")
    line = {
        "metric": "bead-steps/sec of configurations 2 (FP64, 4096 beads) and 5 (Brownian, 32k-262k beads)",
        "value": head["bead_steps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": K5, "warmup": 3,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "value = config 5 at 262144 beads, xi 0.5",
                   "config2": "512 x 8-bead aggregates, phi 0.1, L %.2f, shear 1, lubrication 3a, GMRES 1e-6, "
                              "%d timed steps after 3; FP64 (the config) and mixed" % (L2, K2),
                   "config5": "16-bead aggregates at phi %.2f (the densest reachable: see DESIGN), each size the "
                              "2x2x2 periodic replica of a generated box of 1/8 the beads; shear 0.1, lubrication "
                              "3a, Brownian kT 1 (PSE far field, pairwise near field), mixed, GMRES 1e-6, %d timed "
                              "steps after 3" % (c5["phi"], K5)},
        "config2": cfg2, "config5": cfg5, "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="step",
                    choices=("step", "batch", "rods", "seeds", "oracle-ladder", "configs"))
    ap.add_argument("--profile-run", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "oracle-ladder":
        if rank == 0:
            run_oracle_ladder(args)
        return
    if args.profile_run:
        run_profile(args, local_rank)
        return
    if args.workload == "batch":
        run_batch(args, rank, world, local_rank)
        return
    if args.workload == "rods":
        if rank == 0:
            run_rods(args, local_rank)
        return
    if args.workload == "seeds":
        if rank == 0:
            run_seeds(args, local_rank)
        return
    if args.workload == "configs":
        if rank == 0:
            run_configs(args, local_rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
