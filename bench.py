"""Benchmark of the clover-Wilson hot path on GB300.

One step = one pass of the whole hot path over one synthetic lattice of the
paper's 16^4 size (kappa 0.12, c_sw 1.0, eps 0.2, seed 2, 1 RHS):
  1. qcd_load_gauge  -- pack the canonical links (device) into the SoA copies
  2. qcd_clover_build -- clover term and its FP64 6x6 inverse
  3. qcd_cg_solve     -- mixed FP32/FP64-reliable CG on Mhat^dag Mhat to a true
                         FP64 relative residual 1e-8
  4. qcd_fermion_force -- dS/dU from that solution (clover derivative included)
value = device time per step (CUDA events on the library's stream, L2 flushed
between steps).  The JSON line also carries the plain FP64 GPU solve time, the
Dslash GFLOPS / GB/s of the kernels inside the solve, the roofline of the
dominant kernel, an end-to-end number with host buffers, and the FP64 numpy
oracle timed on a bounded sample on the host cores.  Beside the step it
measures the hopping-kernel bandwidth of Mhat^dag Mhat on 32^3 x 64 and
48^3 x 96 (FP32 / FP16, 1 and 8 / 4 RHS) and the batched FP16 8-RHS solve
against 8 sequential FP64 solves on 32^3 x 64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun) every rank solves its own replica of the workload (the
path has no exchange step on one lattice per GPU); value = N lattices / the
slowest rank's time.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

# the oracle timed as the CPU baseline runs on one host thread: no BLAS / OpenMP thread pools
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GFLOPS & HBM GB/s; time to 1e-8 CG solve, mixed vs FP64, 1 GB300"
# FP64 peak of GB300 derived from its unit counts and clock (2 FP64 FMA / clock / SM x 152 SMs x
# 2.07 GHz), reported beside the probe's measured figure, which the ALU rooflines divide by
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
WORKLOAD = "c1_16^4"
# DRAM bytes (read + write) per launch from one ncu capture of the current kernel, with the summary
# that holds the command; a kernel changed since its capture has no entry (traffic null)
NCU_TRAFFIC = {
    "cg_persistent_p32": (41.4e6, "profiles/cg_persistent_16x16x16x16.md"),
    # mean of the clover-inverse (63.3 MB) and xpay (70.2 MB) passes over a step's mix of the two
    "dslash_p64": (66.7e6, "profiles/dslash_pair64_16x16x16x16.md"),
}
# FP64 pipe activity (% of active cycles) from the same captures, for the kernels bound by it: the
# counted flops of a launch leave out that spin projection and reconstruction are additions, each
# taking an FMA slot of the pipe
NCU_FP64_PIPE = {
    "dslash_p64": (84.3, "profiles/dslash_pair64_16x16x16x16.md"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-hbm", action="store_true", help="skip the large-volume Dslash bandwidth measurement")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 32^3x64 8-RHS batched-mixed vs sequential-FP64 solve comparison")
    ap.add_argument("--no-md", action="store_true",
                    help="skip the clover-determinant, full-solve and R-algorithm sections")
    ap.add_argument("--no-slab", action="store_true", help="skip the two-slab time decomposition section")
    ap.add_argument("--only", default=None, choices=[None, "dslash", "peaks"],
                    help="dslash: only apply Mhat^dag Mhat (FP32 and FP64) a few times, for profiler captures; "
                         "peaks: only measure the FP64 / FP32 FMA and L2 copy denominators")
    ap.add_argument("--nrhs", type=int, default=None, help="right-hand sides for --only dslash")
    ap.add_argument("--precs", default="32,64", help="precisions for --only dslash")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_params(name):
    from paper_0910_0262_gb300 import synth
    w = dict(synth.WORKLOADS[name])
    w["kappa"], w["csw"], w["t_bc"] = synth.KAPPA, synth.CSW, synth.T_BC
    return w


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.device_id = device_id  # what nvidia-smi -i selects: the GPU's UUID, else its PCI bus id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device_id), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi needs a moment to start: let its first sample arrive before the timed region
        t0 = time.perf_counter()
        while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
            time.sleep(0.01)

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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "device": str(self.device_id)}


def smi_device_id(dev):
    """The nvidia-smi selector of torch device `dev`: its UUID ("GPU-..."), else its PCI bus id, so that
    the clocks sampled are this GPU's even when CUDA_VISIBLE_DEVICES renumbers the devices."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    if uuid is not None and str(uuid):
        u = str(uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    bus = getattr(props, "pci_bus_id", None)
    if bus is not None:
        return "%08X:%02X:%02X.0" % (getattr(props, "pci_domain_id", 0), bus, getattr(props, "pci_device_id", 0))
    return str(dev.index if hasattr(dev, "index") else dev)


def max_over_ranks(x, device=None):
    """Largest value of x over all ranks (the slowest replica sets the job's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(seed, rank):
    """Each rank solves its own lattice: same recipe, seed offset by the rank."""
    return seed + 1000 * rank


# ------------------------------------------------------------------- ours --
def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_0910_0262_gb300 import synth, build
    from paper_0910_0262_gb300 import qcd as Q

    build.build()
    # the oracle's full hot-path steps (the CPU-baseline leg) run in spawned processes on host cores of
    # their own while the GPU sections run; started before the first GPU call
    jobs = None
    if rank == 0 and world == 1 and not args.no_cpu:
        jobs = OracleJobs([(args.workload, True), ("c0_8x8x16x16", False)])
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload_params(args.workload)
    dims = w["dims"]
    U_np, b_np = synth.make_problem(dims, w["eps"], replica_seed(w["seed"], rank), w["nrhs"])
    U = torch.from_numpy(U_np).to(dev)
    b = torch.from_numpy(b_np).to(dev)
    stream = torch.cuda.current_stream(dev)
    op = Q.CloverWilson(dims, w["t_bc"], stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2
    X, Y, Z, T = dims
    F = torch.empty((T, Z, Y, X, 4, 3, 3), dtype=torch.complex128, device=dev)
    x = torch.zeros_like(b)
    mixed = dict(tol=1e-8, inner_prec=32, reliable_every=50, reliable_delta=0.1, max_iter=20000)
    prm = Q.solver_params(**mixed)
    nrhs = w["nrhs"]
    stats = (Q.SolverStats * nrhs)()

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        Q.qcd_load_gauge(op.ctx, Q._ptr(U), 1, Q.QCD_GAUGE_RECON12)
        if ev:
            ev[1].record(stream)
        Q.qcd_clover_build(op.ctx, w["kappa"], w["csw"])
        if ev:
            ev[2].record(stream)
        s = Q.qcd_cg_solve(op.ctx, Q._ptr(x), Q._ptr(b), nrhs, prm, stats)
        if s != Q.QCD_OK:
            raise RuntimeError("mixed solve did not converge")
        if ev:
            ev[3].record(stream)
        Q.qcd_fermion_force(op.ctx, Q._ptr(F), Q._ptr(x), nrhs, Q.QCD_FORCE_INPUT_IS_SOLUTION, None, None)
        if ev:
            ev[4].record(stream)

    # the warm-up runs with the per-kernel events on, so that the event-carrying CUDA graphs are
    # recorded before the timed steps; enabling again below clears the counters
    Q.qcd_profile(op.ctx, 1)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    sampler = ClockSampler(smi_device_id(dev))
    sampler.start()
    Q.qcd_profile(op.ctx, 1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t0
    prof = Q.qcd_profile_read(op.ctx)
    Q.qcd_profile(op.ctx, 0)
    clocks = sampler.stop()
    parts = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in evs])  # ms
    step_ms = parts.sum(axis=1)
    ms_per_step = float(np.mean(step_ms))
    iters = stats[0].iters
    resid = max(stats[r].true_rel_resid for r in range(nrhs))

    if world > 1:
        ms_per_step = max_over_ranks(ms_per_step, dev)
    x_mixed, F_step = x.clone(), F.clone()  # the last timed step's solution and force

    # plain FP64 GPU solve on the same lattice, for the mixed-vs-FP64 comparison
    fp64 = Q.solver_params(tol=1e-8, inner_prec=64, max_iter=20000)
    st64 = (Q.SolverStats * nrhs)()
    times64, prof64 = [float("nan")], []
    if not args.no_fp64:
        Q.qcd_profile(op.ctx, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times64 = []
        for _ in range(max(2, min(args.steps, 3))):
            flush.zero_()
            e0.record(stream)
            Q.qcd_cg_solve(op.ctx, Q._ptr(x), Q._ptr(b), nrhs, fp64, st64)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times64.append(e0.elapsed_time(e1))
        prof64 = Q.qcd_profile_read(op.ctx)
        Q.qcd_profile(op.ctx, 0)

    x_fp64 = x.clone()
    result = dict(metric=METRIC, value=ms_per_step * 1.0, unit=step_unit(w))
    solve_mixed = float(np.mean(parts[:, 2]))
    solve64 = None if args.no_fp64 else float(np.mean(times64))

    def kstats(prof_list, prefix):
        rows = [p for p in prof_list if p["name"].startswith(prefix)]
        ms = sum(p["total_ms"] for p in rows)
        n = sum(p["launches"] for p in rows)
        by = sum(p["bytes"] for p in rows)
        fl = sum(p["flops"] for p in rows)
        return dict(launches=n, avg_us=1e3 * ms / max(n, 1), gbs=by / (ms * 1e-3) / 1e9 if ms else 0.0,
                    gflops=fl / (ms * 1e-3) / 1e9 if ms else 0.0, bytes_per_launch=by / max(n, 1))

    d32 = kstats(prof, "dslash_p32")
    d64 = kstats(prof, "dslash_p64")
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    device_peaks = measure_device_peaks(Q)
    total_launches = next((p["launches"] for p in prof if p["name"] == "launches_total"), None)
    # per-step device time of each kernel class: sampled average duration x launches per step
    per_step_launches = {"dslash_p32": 4 * iters, "dslash_p64": 4 * max(stats[0].reliable_updates, 0),
                         "force_links": 1, "force_edges": 1, "force_clover_coeff": 1, "clover_build": 1,
                         "cg_update": iters,
                         "p_update": iters}
    classes = {}
    for key, n in per_step_launches.items():
        ks = kstats(prof, key)
        if ks["launches"]:
            classes[key] = dict(ks, launches_per_step=n, est_ms_per_step=ks["avg_us"] * n / 1e3)
    # the persistent single-RHS iteration kernel is timed on every launch (not sampled)
    for p in prof:
        if p["name"].startswith("cg_persistent") and p["launches"]:
            ks = kstats(prof, p["name"])
            classes[p["name"]] = dict(ks, launches_per_step=p["launches"] / args.steps,
                                      est_ms_per_step=p["total_ms"] / args.steps)
    dominant = max(classes, key=lambda k: classes[k]["est_ms_per_step"])
    result.update({
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 reliable",
        "data": "synthetic (seeded near-unit SU(3) links, Gaussian source)",
        "config": step_config(args.workload, w, world),
        "parts_ms": {"load_gauge": float(np.mean(parts[:, 0])), "clover_build": float(np.mean(parts[:, 1])),
                     "cg_solve_mixed": solve_mixed, "fermion_force": float(np.mean(parts[:, 3]))},
        "solve": {"mixed_ms": solve_mixed, "fp64_ms": solve64, "speedup_mixed_vs_fp64": None if solve64 is None else solve64 / solve_mixed,
                  "mixed_iters": iters, "fp64_iters": st64[0].iters, "reliable_updates": stats[0].reliable_updates,
                  "true_rel_resid_mixed": resid, "true_rel_resid_fp64": st64[0].true_rel_resid},
        # hopping launches of the solve by precision (FP32 only when its hops run as separate launches
        # rather than inside the persistent kernel)
        "dslash": {k: v for k, v in (("fp32_in_solve", d32), ("fp64_in_solve", d64)) if v["launches"]},
        "kernels_per_step": classes,
        "gpu_launches": total_launches,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    })
    result["device_peaks"] = device_peaks
    # roofline of the kernel with the largest device time per step
    dk = classes[dominant]
    tr = NCU_TRAFFIC.get(dominant)
    common = {"kernel": dominant, "traffic": None if tr is None else tr[0],
              "traffic_source": None if tr is None else tr[1],
              "algorithmic_bytes_per_launch": dk["bytes_per_launch"]}
    if dominant.startswith("cg_persistent") and dominant != "cg_persistent_p64" and V_HALF(w) <= L2_RESIDENT_VH:
        # the persistent iteration's working set (links, clover pair, six spinor fields) stays in the
        # 129 MB L2 at this size (ncu: DRAM traffic a few percent of the algorithmic bytes), so its
        # roofline is the measured L2-resident copy bandwidth; its fraction of HBM is given beside it
        result["roofline"] = dict(common, bound="l2", achieved=dk["gbs"], peak=device_peaks["l2_copy_gbs"],
                                  unit="GB/s", frac=dk["gbs"] / device_peaks["l2_copy_gbs"],
                                  peak_source="L2-resident copy measured in this run (of measured)",
                                  hbm_peak=hbm_peak, hbm_frac=dk["gbs"] / hbm_peak)
    elif dominant.startswith("dslash_p32") or dominant.startswith("cg_persistent"):
        result["roofline"] = dict(common, bound="hbm", achieved=dk["gbs"], peak=hbm_peak, unit="GB/s",
                                  frac=dk["gbs"] / hbm_peak, peak_source="MEASURED_PEAKS.json hbm_gbs (of measured)")
    else:
        p64 = device_peaks["fp64_tflops"]
        result["roofline"] = dict(common, bound="alu", achieved=dk["gflops"] / 1e3, peak=p64, unit="TFLOP/s",
                                  frac=dk["gflops"] / 1e3 / p64,
                                  peak_source="FP64 FMA probe measured in this run (of measured)")
        if dominant in NCU_FP64_PIPE:
            result["roofline"]["fp64_pipe_active_pct_ncu"] = NCU_FP64_PIPE[dominant][0]
            result["roofline"]["fp64_pipe_source"] = NCU_FP64_PIPE[dominant][1]
    if not args.no_md:
        result["clover_det_and_full_solve"] = clover_det_section(op, x, b, stream)
        result["r_algorithm_step"] = r_step_section(op, U, w, stream)
    if not args.no_slab and world == 1:
        result["slab_decomposition"] = slab_section(w)
    if not args.no_hbm or not args.no_batched:
        result.update(large_volume(dev, hbm_peak, not args.no_hbm, not args.no_batched, jobs is not None))
    if not args.no_hbm:
        result["dslash_largest_volume"] = largest_volume(dev, hbm_peak, jobs is not None)
    if not args.no_e2e:
        result["e2e"] = run_e2e(op, U_np, b_np, w, stream, dev)
    if jobs is not None:
        cn = lambda t: t.detach().cpu().numpy()
        gpu = {"mhat": {p: cn(op.dslash(b, Q.QCD_OP_MHAT, precision=p))[0] for p in (64, 32, 16)},
               "x_mixed": cn(x_mixed)[0], "x_fp64": cn(x_fp64)[0], "F_step": cn(F_step),
               "force_from": lambda xo: cn(op.fermion_force(torch.from_numpy(xo[None]).to(dev),
                                                            input_is_solution=True)[0])}
        result["cpu_baseline"], result["errors"] = cpu_baseline(jobs, args.workload, gpu)
        jobs.close()
    op.close()
    return result


def r_step_section(op, U, w, stream, warmup=2, reps=5, eps=0.02, beta=5.6):
    """One two-flavour R-algorithm step on the step's lattice (one pseudofermion, determinant term,
    mixed FP32 solve to 1e-8), as a step of a trajectory (the clover term of the new links is left to
    the next step): device time (CUDA events, median of `reps`) and its kernel classes from one
    profiled step; momenta and noise drawn on the host with numpy (seeded)."""
    import torch
    from paper_0910_0262_gb300 import synth
    rng = np.random.default_rng(71)
    Ut = U.clone()
    p = rng.standard_normal(tuple(Ut.shape[:5]) + (8,))
    P = torch.from_numpy(np.einsum('...a,aij->...ij', 1j * p, synth.T_GEN)).to(Ut.device)
    eta = torch.from_numpy(synth.gaussian_sources(w["dims"], 1, rng)).to(Ut.device)
    kw = dict(tol=1e-8, inner_prec=32, reliable_every=50, reliable_delta=0.1)
    ts, iters = [], []
    for k in range(warmup + reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if k == warmup:
            op.profile(True)
        e0.record(stream)
        st, ok = op.r_step(Ut, P, eta, eps, beta, clover_det=True, defer_clover=True, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        if k == warmup:
            prof = op.profile_read()
            op.profile(False)
        if not ok:
            raise RuntimeError("R step solve did not converge")
        if k >= warmup:
            ts.append(e0.elapsed_time(e1))
            iters.append(st[0]["iters"])
    classes = {}
    for q in prof:
        key = q["name"].split("_r")[0] if q["name"].startswith("dslash") else q["name"]
        c = classes.setdefault(key, {"launches": 0, "ms": 0.0})
        c["launches"] += q["launches"]
        c["ms"] += q["total_ms"]
    op.load_gauge(U, recon12=True)
    op.clover_build(w["kappa"], w["csw"])
    return {"ms": float(np.median(ts)), "eps": eps, "beta": beta, "pseudofermions": 1, "clover_det": True,
            "solve": "mixed fp32, tol 1e-8", "cg_iters": iters, "plaquette_after": op.plaquette(),
            "kernel_ms_one_step": {k: round(v["ms"], 4) for k, v in sorted(classes.items(), key=lambda kv: -kv[1]["ms"])},
            "timing": f"median of {reps} steps after {warmup}, CUDA events"}


def clover_det_section(op, x, b, stream, warmup=3, reps=10):
    """On the step's lattice: device times (CUDA events on the library's stream, median of `reps`
    after `warmup`) of the clover determinant term -- log det A per parity, its force alone, the
    pseudofermion force with and without it -- and of the full-lattice helpers (source preparation,
    odd-site reconstruction), with the determinant term's value."""
    import torch

    def timed(fn):
        for _ in range(warmup):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    le, lo = op.clover_logdet()
    res = {"logdet_even": le, "logdet_odd": lo, "S_det": -2.0 * lo,
           "logdet_ms": timed(op.clover_logdet),
           "det_force_alone_ms": timed(lambda: op.fermion_force(None, clover_det=True)),
           "pf_force_ms": timed(lambda: op.fermion_force(x, input_is_solution=True)),
           "pf_plus_det_force_ms": timed(lambda: op.fermion_force(x, input_is_solution=True, clover_det=True)),
           "prepare_source_ms": timed(lambda: op.prepare_source(b, b)),
           "reconstruct_odd_ms": timed(lambda: op.reconstruct_odd(x, b)),
           "timing": f"median of {reps} after {warmup} warm-up, CUDA events (calls that synchronise included)"}
    res["det_term_marginal_ms"] = res["pf_plus_det_force_ms"] - res["pf_force_ms"]
    return res


def dslash_bandwidth(op, b, hbm_peak, rhs_list, warmup=5, reps=20):
    """Mhat^dag Mhat (4 hopping launches with fused clover epilogues) in FP32 and FP16 for each RHS
    count: after `warmup` applications, `reps` applications each timed by the library's per-launch
    CUDA events (device time of the 4 launches); the median application gives the per-launch time,
    and the algorithmic bytes and flops the library counts per launch give GB/s and GFLOP/s."""
    import torch
    from paper_0910_0262_gb300 import qcd as Q
    out = {}
    for prec in (32, 16):
        for nrhs in rhs_list:
            v = b[:nrhs].contiguous()
            for _ in range(warmup):
                op.dslash(v, Q.QCD_OP_MDAGM, precision=prec)
            samples = []
            for _ in range(reps):
                op.profile(True)
                op.dslash(v, Q.QCD_OP_MDAGM, precision=prec)
                rows = [p for p in op.profile_read() if p["name"].startswith(f"dslash_p{prec}")]
                op.profile(False)
                samples.append((sum(p["total_ms"] for p in rows), sum(p["bytes"] for p in rows),
                                sum(p["flops"] for p in rows), sum(p["launches"] for p in rows)))
            ms = float(np.median([t[0] for t in samples]))
            by, fl, n = samples[0][1], samples[0][2], samples[0][3]
            gbs = by / (ms * 1e-3) / 1e9
            out[f"fp{prec}_rhs{nrhs}"] = {"launches": n, "avg_us": 1e3 * ms / n, "gbs": gbs, "frac_hbm": gbs / hbm_peak,
                                          "gflops": fl / (ms * 1e-3) / 1e9, "bytes_per_launch": by / n,
                                          "timing": f"median of {reps} applications after {warmup} warm-up"}
    return out


def sampled_mhat_errors(op, U_np, b, dims, kappa, csw, t_bc, nsites=32, seed=11):
    """Relative L2 error of the GPU's Mhat (FP64, FP32, FP16) on the first RHS against the oracle's
    single-site Mhat at nsites sampled even sites (the first and last half index among them)."""
    from paper_0910_0262_gb300 import qcd as Q
    vh = b.shape[1]
    sites = np.unique(np.concatenate([[0, vh - 1], np.random.default_rng(seed).choice(vh, nsites - 2)]))
    b0 = b[:1].contiguous()
    want = oracle_sampled_mhat(U_np, b0[0].cpu().numpy(), dims, sites, kappa, csw, t_bc)
    idx = torch_index(sites, b.device)
    return {f"mhat_fp{p}_vs_oracle_sampled": rel_l2(op.dslash(b0, Q.QCD_OP_MHAT, precision=p)[0][idx].cpu().numpy(),
                                                     want)
            for p in (64, 32, 16)} | {"sites": int(len(sites))}


def torch_index(a, device):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.int64), device=device)


def large_volume(dev, hbm_peak, do_hbm, do_batched, do_errors=False):
    """32^3 x 64 lattice (eps 0.15, seed 4, 8 RHS; working set far above the 129 MB L2).

    dslash_large_volume: Mhat^dag Mhat in FP32 and FP16 with 12-real links, 1 and 8 RHS
    (dslash_bandwidth), against the measured HBM bandwidth.
    batched_solve: one batched mixed solve of the 8 RHS (FP16 inner, FP64 reliable updates) against
    8 sequential plain FP64 solves, both to a true residual of 1e-8.
    """
    import torch
    from paper_0910_0262_gb300 import synth
    from paper_0910_0262_gb300 import qcd as Q
    w = synth.WORKLOADS["c3_32^3x64"]
    dims = w["dims"]
    U_np, b_np = synth.make_problem(dims, w["eps"], w["seed"], w["nrhs"])
    stream = torch.cuda.current_stream(dev)
    op = Q.CloverWilson(dims, -1.0, stream=stream)
    op.load_gauge(torch.from_numpy(U_np).to(dev), recon12=True)
    op.clover_build(0.12, 1.0)
    b = torch.from_numpy(b_np).to(dev)
    res = {}
    if do_hbm:
        res["dslash_large_volume"] = {"dims": list(dims), "op": "Mhat^dag Mhat (4 hopping launches with fused "
                                      "clover epilogues)", "peak_gbs": hbm_peak,
                                      "results": dslash_bandwidth(op, b, hbm_peak, (1, 8))}
        if do_errors:
            res["dslash_large_volume"]["errors"] = sampled_mhat_errors(op, U_np, b, dims, 0.12, 1.0, -1.0)
    if do_batched:
        kw = dict(tol=1e-8, reliable_every=50, reliable_delta=0.1)

        def timed(fn):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return out, e0.elapsed_time(e1)

        op.cg_solve(b[:1], inner_prec=16, **kw)  # warm up graph capture
        op.cg_solve(b, inner_prec=16, **kw)
        (xb, stb, okb), t_batched = timed(lambda: op.cg_solve(b, inner_prec=16, **kw))
        # where the batched solve's time goes: the library's per-launch events in one more (profiled) solve
        op.profile(True)
        _, t_prof = timed(lambda: op.cg_solve(b, inner_prec=16, **kw))
        prof = op.profile_read()
        op.profile(False)
        seq16, t_seq16 = timed(lambda: [op.cg_solve(b[r:r + 1].contiguous(), inner_prec=16, **kw)
                                        for r in range(b.shape[0])])
        seq, t_seq = timed(lambda: [op.cg_solve(b[r:r + 1].contiguous(), inner_prec=64, **kw)
                                    for r in range(b.shape[0])])
        n_it = max(s["iters"] for s in stb)

        def cls(prefix):
            rows = [p for p in prof if p["name"].startswith(prefix)]
            return sum(p["total_ms"] for p in rows), sum(p["launches"] for p in rows)

        hop_ms, hop_n = cls("dslash_p16")
        pu_ms, pu_n = cls("p_update")
        rel_ms, rel_n = cls("dslash_p64")
        parts = {"inner_hopping_fp16": hop_ms / max(hop_n, 1) * 4 * n_it,
                 "inner_p_update": pu_ms / max(pu_n, 1) * n_it,
                 "reliable_update_hopping_fp64": rel_ms}
        parts["rest"] = t_prof - sum(parts.values())
        res["batched_solve"] = {
            "dims": list(dims), "nrhs": int(b.shape[0]),
            "batched_mixed_fp16_ms": t_batched, "sequential_mixed_fp16_ms": t_seq16, "sequential_fp64_ms": t_seq,
            "speedup": t_seq / t_batched, "batching_gain_vs_sequential_mixed": t_seq16 / t_batched,
            "batched_iters": [s["iters"] for s in stb], "batched_reliable_updates": stb[0]["reliable_updates"],
            "batched_true_rel_resid": max(s["true_rel_resid"] for s in stb),
            "sequential_mixed_iters": [s[1][0]["iters"] for s in seq16],
            "sequential_mixed_true_rel_resid": max(s[1][0]["true_rel_resid"] for s in seq16),
            "sequential_iters": [s[1][0]["iters"] for s in seq],
            "sequential_true_rel_resid": max(s[1][0]["true_rel_resid"] for s in seq),
            "converged": bool(okb and all(s[2] for s in seq) and all(s[2] for s in seq16)),
            "breakdown_ms": {"profiled_solve_ms": t_prof, **parts,
                             "how": "per-launch CUDA events of the library (inner kernels sampled on the first "
                                    "iteration of each graph, times the iterations run; every reliable-update "
                                    "launch); rest = the profiled solve's time minus these: the reliable "
                                    "updates' BLAS, launch gaps and host looks at the solver state"}}
    op.close()
    return res


def largest_volume(dev, hbm_peak, do_errors=False):
    """48^3 x 96 lattice (eps 0.15, seed 5, 4 RHS; 10.6 M sites): the hopping-kernel bandwidth of
    Mhat^dag Mhat in FP32 and FP16 for 1 and 4 RHS (dslash_bandwidth)."""
    import torch
    from paper_0910_0262_gb300 import synth
    from paper_0910_0262_gb300 import qcd as Q
    w = synth.WORKLOADS["c4_48^3x96"]
    dims = w["dims"]
    U_np, b_np = synth.make_problem(dims, w["eps"], w["seed"], w["nrhs"])
    op = Q.CloverWilson(dims, -1.0, stream=torch.cuda.current_stream(dev))
    op.load_gauge(torch.from_numpy(U_np).to(dev), recon12=True)
    if not do_errors:
        del U_np
    op.clover_build(0.12, 1.0)
    b = torch.from_numpy(b_np).to(dev)
    res = {"dims": list(dims), "op": "Mhat^dag Mhat (4 hopping launches with fused clover epilogues)",
           "peak_gbs": hbm_peak, "results": dslash_bandwidth(op, b, hbm_peak, (1, 4))}
    if do_errors:
        res["errors"] = sampled_mhat_errors(op, U_np, b, dims, 0.12, 1.0, -1.0)
    op.close()
    return res


def slab_section(w, reps=5):
    """The time decomposition on one GPU: the step's lattice cut into two t-slabs, each a context of its
    own on a stream of its own, driven by a host thread.  The halos and sums go through the library's
    in-process group (NativeSlabGroup: native callbacks, CUDA events between the slabs' streams, one host
    barrier per exchange or sum only to publish them, halos read in place); the same solve through the
    Python group (LocalSlabGroup: torch
    copies after host synchronisation) is given beside it.  Times Mhat^dag Mhat in FP32 (four
    exchanges) and the mixed FP32 solve to 1e-8 against one context, with the halo bytes per exchange.
    Both slabs share one GPU, so this measures the halo path's cost, not a multi-GPU speed."""
    import torch
    from paper_0910_0262_gb300 import synth, slab
    from paper_0910_0262_gb300 import qcd as Q
    dims = w["dims"]
    U, b = synth.make_problem(dims, w["eps"], w["seed"], 1)
    bounds = [slab.slab_bounds(dims[3], 2, r) for r in range(2)]
    bd = torch.from_numpy(b).cuda()
    kw = dict(tol=1e-8, inner_prec=32, reliable_every=50, reliable_delta=0.1, max_iter=20000)

    def measure(grp, with_mdagm):
        ops = []
        for r, (t0, tl) in enumerate(bounds):
            st = torch.cuda.Stream()
            op = slab.SlabCloverWilson(dims, t0, tl, grp.member(r), w["t_bc"], stream=st)
            with torch.cuda.stream(st):
                op.load_gauge(torch.from_numpy(slab.extended_links(U, t0, tl)).cuda(), recon12=True)
            op.clover_build(w["kappa"], w["csw"])
            ops.append(op)

        def on_slabs(fn):
            def job(r):
                op = ops[r]
                a, c = slab.slab_rows(dims, op.t_offset, op.t_local)
                with torch.cuda.stream(op.stream):
                    out = fn(op, bd[:, a:c].contiguous())
                    op.stream.synchronize()
                return out
            t0 = time.perf_counter()
            res = grp.run([lambda r=r: job(r) for r in range(2)])
            return res, 1e3 * (time.perf_counter() - t0)

        t_mdagm, t_solve, iters, ok = [], [], None, True
        for k in range(reps + 1):
            if with_mdagm:
                _, t = on_slabs(lambda op, v: op.dslash(v, Q.QCD_OP_MDAGM, precision=32))
                if k:
                    t_mdagm.append(t)
            res, ts = on_slabs(lambda op, v: op.cg_solve(v, **kw))
            if k:
                t_solve.append(ts)
            iters = res[0][1][0]["iters"]
            ok = ok and all(r[2] for r in res)
        halo = Q.qcd_slab_halo_bytes(ops[0].ctx, 32, 1)
        for op in ops:
            op.close()
        if hasattr(grp, "close"):
            grp.close()
        return (float(np.median(t_mdagm)) if t_mdagm else None), float(np.median(t_solve)), iters, ok, halo

    mdagm_n, solve_n, iters, ok_n, halo = measure(slab.NativeSlabGroup(2), True)
    _, solve_p, _, ok_p, _ = measure(slab.LocalSlabGroup(2), False)
    one = Q.CloverWilson(dims, w["t_bc"])
    one.load_gauge(torch.from_numpy(U).cuda(), recon12=True)
    one.clover_build(w["kappa"], w["csw"])
    t1 = []
    for k in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st1, ok1 = one.cg_solve(bd, **kw)
        torch.cuda.synchronize()
        if k:
            t1.append(1e3 * (time.perf_counter() - t0))
    one.close()
    return {"dims": list(dims), "slabs": [list(s) for s in bounds], "gpus": 1,
            "mdagm_fp32_ms_two_slabs": mdagm_n, "mixed_solve_ms_two_slabs": solve_n,
            "mixed_solve_ms_two_slabs_python_exchange": solve_p, "mixed_solve_ms_one_context": float(np.median(t1)),
            "iters_two_slabs": iters, "iters_one_context": st1[0]["iters"], "converged": bool(ok_n and ok_p and ok1),
            "halo_bytes_per_exchange_fp32": halo, "exchanges_per_mdagm": 4,
            "exchange": "the library's in-process group (qcd_local_group_*); python_exchange: LocalSlabGroup",
            "timing": f"median of {reps} after one, host wall clock around both slabs' calls"}


def run_e2e(op, U_np, b_np, w, stream, dev):
    """The same step through the public API from pinned host buffers: links and source copied in,
    solution and force read back, all inside the timed region."""
    import torch
    from paper_0910_0262_gb300 import qcd as Q
    U_h = torch.from_numpy(U_np).pin_memory()
    b_h = torch.from_numpy(b_np).pin_memory()
    x_h = torch.empty_like(b_h).pin_memory()
    X, Y, Z, T = w["dims"]
    F_h = torch.empty((T, Z, Y, X, 4, 3, 3), dtype=torch.complex128).pin_memory()
    kw = dict(tol=1e-8, inner_prec=32, reliable_every=50, reliable_delta=0.1, max_iter=20000)
    times = []
    for k in range(4):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        op.load_gauge(U_h, recon12=True)           # host pointer: the library copies it in
        op.clover_build(w["kappa"], w["csw"])
        b = b_h.to(dev, non_blocking=True)
        x, st, ok = op.cg_solve(b, **kw)
        F, _ = op.fermion_force(x, input_is_solution=True)
        x_h.copy_(x)
        F_h.copy_(F)
        torch.cuda.synchronize(dev)
        if k:
            times.append((time.perf_counter() - t0) * 1e3)
    return {"value": float(np.mean(times)), "unit": "ms per hot-path step (16^4, solve to 1e-8)",
            "h2d_bytes_per_step": int(U_h.numel() * 16 + b_h.numel() * 16),
            "d2h_bytes_per_step": int(x_h.numel() * 16 + F_h.numel() * 16)}


# ------------------------------------------------------------ CPU oracle --
# The CPU-baseline leg and the reference arm: the numpy FP64 oracle as it stands (oracle/), timed on
# the host cores, one thread per job (the BLAS / OpenMP pools are pinned to one thread above).  No
# other part of this file imports oracle/.

def _host_cores():
    try:
        return sorted(os.sched_getaffinity(0))
    except AttributeError:
        return list(range(os.cpu_count() or 1))


def oracle_hot_path(name, out_dir=None, with_force=True, tick=None):
    """One hot-path step of the oracle on workload `name`, on the calling thread: the clover term and
    its inverse (SchurOperator), the CG of oracle.cg on Mhat^dag Mhat to a true relative residual of
    1e-8 with the oracle's own iteration count, and the force from that solution; each part timed by
    the wall clock.  tick() (optional) is called before each unit of work: the clover build, every
    Mhat^dag Mhat application of the CG, the force.  With out_dir the solution (x), the force (F) and
    Mhat b (Mb, timed separately as one operator application) are saved there as <name>_<key>.npy."""
    from paper_0910_0262_gb300 import synth
    from oracle import evenodd, cg as ocg, force as oforce
    w = workload_params(name)
    U, b = synth.make_problem(w["dims"], w["eps"], w["seed"], w["nrhs"])
    tick = tick or (lambda: None)
    tick()
    t0 = time.perf_counter()
    op = evenodd.SchurOperator(U, w["kappa"], w["csw"], w["t_bc"])
    t_clover = time.perf_counter() - t0
    applications = [0]

    def apply_A(v):
        tick()
        applications[0] += 1
        return op.MdagM(v)

    t0 = time.perf_counter()
    x, iters, true_res = ocg.cg(apply_A, b[0], tol=1e-8)
    t_solve = time.perf_counter() - t0
    res = {"workload": name, "dims": list(w["dims"]), "clover_s": t_clover, "solve_s": t_solve, "cg_iters": iters,
           "mdagm_applications": applications[0], "true_rel_resid": true_res}
    if with_force:
        tick()
        t0 = time.perf_counter()
        F = oforce.lie_force(U, oforce.gradient(op, x))
        res["force_s"] = time.perf_counter() - t0
    res["step_s"] = t_clover + t_solve + res.get("force_s", 0.0)
    if out_dir is not None:
        t0 = time.perf_counter()
        Mb = op.Mhat(b[0])
        res["mhat_apply_s"] = time.perf_counter() - t0
        np.save(os.path.join(out_dir, f"{name}_x.npy"), x)
        np.save(os.path.join(out_dir, f"{name}_Mb.npy"), Mb)
        if with_force:
            np.save(os.path.join(out_dir, f"{name}_F.npy"), F)
    return res


def _oracle_job(name, out_dir, core, with_force):
    """Body of one spawned oracle process: pinned to `core`, writes <name>.json (and the arrays)."""
    if core is not None:
        try:
            os.sched_setaffinity(0, {core})
        except (AttributeError, OSError):
            core = None
    try:
        res = oracle_hot_path(name, out_dir, with_force)
    except Exception as e:  # reported in the bench line instead of a number
        res = {"error": repr(e)}
    res["core"] = core
    with open(os.path.join(out_dir, f"{name}.json"), "w") as f:
        json.dump(res, f)


class OracleJobs:
    """Full hot-path steps of the oracle for the CPU baseline, each in a spawned process on a host
    core of its own (the last cores of this process's affinity set), started before the first GPU
    call and collected after the GPU sections."""

    def __init__(self, jobs):
        import multiprocessing as mp
        import tempfile
        self.dir = tempfile.mkdtemp(prefix="qcd_oracle_")
        ctx = mp.get_context("spawn")
        cores = _host_cores()
        self.procs = {}
        for k, (name, with_force) in enumerate(jobs):
            core = cores[-1 - k] if len(cores) > len(jobs) else None
            p = ctx.Process(target=_oracle_job, args=(name, self.dir, core, with_force), daemon=True)
            p.start()
            self.procs[name] = p

    def result(self, name, timeout=1200.0):
        p = self.procs[name]
        p.join(timeout)
        if p.is_alive():
            p.terminate()
            return {"error": f"oracle job {name} did not finish in {timeout:.0f} s"}
        try:
            with open(os.path.join(self.dir, f"{name}.json")) as f:
                return json.load(f)
        except OSError:
            return {"error": f"oracle job {name} exited with {p.exitcode} and no result"}

    def array(self, name, key):
        return np.load(os.path.join(self.dir, f"{name}_{key}.npy"))

    def close(self):
        import shutil
        for p in self.procs.values():
            if p.is_alive():
                p.terminate()
        shutil.rmtree(self.dir, ignore_errors=True)


def rel_l2(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_true_residual(name, x):
    """|b - Mhat^dag Mhat x| / |b| of a GPU solution x of workload `name`, recomputed by the oracle."""
    from paper_0910_0262_gb300 import synth
    from oracle import evenodd
    w = workload_params(name)
    U, b = synth.make_problem(w["dims"], w["eps"], w["seed"], w["nrhs"])
    op = evenodd.SchurOperator(U, w["kappa"], w["csw"], w["t_bc"])
    return rel_l2(op.MdagM(x), b[0])


def oracle_sampled_mhat(U, v, dims, sites, kappa, csw, t_bc):
    """Mhat v at the sampled even half indices `sites`, evaluated one site at a time by the oracle's
    single-site operator (lattices too large for the whole-lattice oracle)."""
    from oracle import local
    out = []
    for h in sites:
        i = next(i for i in (2 * int(h), 2 * int(h) + 1) if sum(local.coords(dims, i)) % 2 == 0)
        out.append(local.mhat_site(U, v, dims, local.coords(dims, i), kappa, csw, t_bc))
    return np.array(out)


def cpu_baseline(jobs, name, gpu):
    """The CPU-baseline leg of the GPU arm: the oracle's measured hot-path steps (jobs started by
    run_ours) and the error of every GPU result of the step's workload against the oracle's.

    gpu: numpy copies of the GPU results on workload `name` -- "mhat" {precision: Mhat b}, "x_mixed",
    "x_fp64", "F_step" (force from the mixed solution) -- and "force_from" (a function returning the
    GPU force for a given solution, evaluated here on the oracle's own solution)."""
    c1 = jobs.result(name)
    c0 = jobs.result("c0_8x8x16x16")
    cores = _host_cores()
    out = {"unit": step_unit(workload_params(name)), "kind": "oracle", "cores": 1,
           "cores_available": len(cores)}
    if "error" in c1:
        out.update(value=None, sample=c1["error"])
        return out, {}
    out.update({
        "value": c1["step_s"] * 1e3,
        "sample": f"one full hot-path step of the numpy FP64 oracle on {'x'.join(map(str, c1['dims']))}: clover "
                  f"term + inverse, CG to a true residual of 1e-8 ({c1['cg_iters']} iterations, "
                  f"{c1['mdagm_applications']} Mhat^dag Mhat applications, true residual "
                  f"{c1['true_rel_resid']:.2e}), force; one thread, measured (nothing scaled)",
        "parts_s": {k: c1[k] for k in ("clover_s", "solve_s", "force_s")},
        "s_per_cg_iteration": c1["solve_s"] / max(c1["mdagm_applications"], 1),
        "mhat_apply_ms": c1["mhat_apply_s"] * 1e3, "core": c1["core"],
        "c0_8x8x16x16_solve": c0 if "error" in c0 else {
            "solve_ms": c0["solve_s"] * 1e3, "clover_ms": c0["clover_s"] * 1e3, "cg_iters": c0["cg_iters"],
            "true_rel_resid": c0["true_rel_resid"], "core": c0["core"]},
    })
    x_or = jobs.array(name, "x")
    F_or = jobs.array(name, "F")
    Mb_or = jobs.array(name, "Mb")
    errors = {"reference": f"numpy FP64 oracle on {name}; relative L2 over the whole field"}
    for prec, y in sorted(gpu["mhat"].items()):
        errors[f"mhat_fp{prec}_vs_oracle"] = rel_l2(y, Mb_or)
    errors["solution_mixed_vs_oracle_solution"] = rel_l2(gpu["x_mixed"], x_or)
    errors["solution_fp64_vs_oracle_solution"] = rel_l2(gpu["x_fp64"], x_or)
    errors["true_rel_resid_mixed_by_oracle"] = oracle_true_residual(name, gpu["x_mixed"])
    errors["force_kernels_vs_oracle_same_solution"] = rel_l2(gpu["force_from"](x_or), F_or)
    errors["force_step_vs_oracle"] = rel_l2(gpu["F_step"], F_or)
    errors["note"] = ("two solutions to a residual of 1e-8 differ by up to the condition number times 1e-8, "
                      "so the step's force differs from the oracle's by as much; the force kernels on one "
                      "solution agree to rounding")
    return out, errors


def step_config(name, w, world):
    """The workload of one hot-path step (the same dict in both arms)."""
    return {"workload": name, "dims": list(w["dims"]), "nrhs": w["nrhs"], "kappa": w["kappa"],
            "csw": w["csw"], "eps": w["eps"], "seed": w["seed"], "tol": 1e-8,
            "inner": "fp32, 12-real links, reliable update every 50 its or 0.1 drop",
            "l2": "flushed (256 MiB write) before every step, outside the step's events",
            "parallelism": f"replicas x{world}"}


def step_unit(w):
    """The metric's unit for workload w (the same string in both arms)."""
    d = w["dims"]
    lat = f"{d[0]}^4" if len(set(d)) == 1 else "x".join(map(str, d))
    return f"ms per hot-path step ({lat}, solve to 1e-8)"


def V_HALF(w):
    return int(np.prod(w["dims"])) // 2


# half volume up to which a single-RHS iteration's working set (about 1.6 kB per even site at FP32
# with 12-real links) stays in the 129 MB L2
L2_RESIDENT_VH = 1 << 16


def measure_device_peaks(Q):
    """The rooflines' ALU and L2 denominators, measured here with the library's probes (CUDA events):
    FP64 and FP32 FMA throughput, and the bandwidth of a copy between two 24 MiB buffers (48 MiB in
    L2), beside the derived FP64 figure of the unit counts and the maximum clock."""
    return {"fp64_tflops": Q.qcd_probe_fma_peak(64), "fp32_tflops": Q.qcd_probe_fma_peak(32),
            "l2_copy_gbs": Q.qcd_probe_copy_bandwidth(24 << 20, 20),
            "fp64_tflops_derived": FP64_PEAK_TFLOPS,
            "how": "qcd_probe_fma_peak (8 FMA chains per thread, 8 x 256 threads per SM) and "
                   "qcd_probe_copy_bandwidth (24 MiB -> 24 MiB, 32 passes per launch, read + write bytes)"}


# -------------------------------------------------------------- reference --
class SliceRunner:
    """Runs fn(tick) on a worker thread in consecutive slices: each run_slice(n) lets the worker pass
    n more calls of tick() (None: run to the end) and returns the wall time the slice took."""

    def __init__(self, fn):
        self._go = threading.Semaphore(0)
        self._parked = threading.Semaphore(0)
        self._left = 0
        self.finished = False
        self.result = None
        self.error = None
        self._thread = threading.Thread(target=self._run, args=(fn,), daemon=True)
        self._thread.start()
        self._parked.acquire()  # the worker waits at its first tick

    def _tick(self):
        if self._left == 0:
            self._parked.release()
            self._go.acquire()
        self._left -= 1

    def _run(self, fn):
        try:
            self.result = fn(self._tick)
        except BaseException as e:  # re-raised by the caller
            self.error = e
        self.finished = True
        self._parked.release()

    def run_slice(self, n=None):
        if self.finished:
            return 0.0
        self._left = (1 << 60) if n is None else n
        t0 = time.perf_counter()
        self._go.release()
        self._parked.acquire()
        return time.perf_counter() - t0


def run_reference(args, world, rank):
    """The oracle arm: ONE full hot-path step of the numpy FP64 oracle on the workload (clover term and
    inverse, CG to a true relative residual of 1e-8 with the oracle's own iteration count, force), on
    one host thread, measured in `steps` consecutive timed slices: slice k < steps runs the next unit
    of work (the clover build, one Mhat^dag Mhat application of the CG, the force), the last slice the
    rest.  value = the sum of the slices = one measured hot-path step; ms_per_step = that sum / steps,
    the mean duration of a timed slice.  Each warm-up step applies the oracle's Mhat once."""
    from paper_0910_0262_gb300 import synth
    from oracle import evenodd
    w = workload_params(args.workload)
    U, b = synth.make_problem(w["dims"], w["eps"], w["seed"], w["nrhs"])
    if args.warmup:
        op = evenodd.SchurOperator(U, w["kappa"], w["csw"], w["t_bc"])
        for _ in range(args.warmup):
            op.Mhat(b[0])
        del op
    del U, b
    runner = SliceRunner(lambda tick: oracle_hot_path(args.workload, tick=tick))
    slices = [runner.run_slice(1 if k < args.steps - 1 else None) for k in range(args.steps)]
    if not runner.finished:
        slices[-1] += runner.run_slice(None)
    if runner.error is not None:
        raise runner.error
    r = runner.result
    total_ms = 1e3 * float(np.sum(slices))
    unit = step_unit(w)
    sample = (f"one full hot-path step of the numpy FP64 oracle, measured in {args.steps} timed slices: clover term "
              f"+ inverse, CG to a true residual of 1e-8 ({r['cg_iters']} iterations, {r['mdagm_applications']} "
              f"Mhat^dag Mhat applications, true residual {r['true_rel_resid']:.2e}), force; one thread")
    cores = 1
    return {"impl": "reference", "metric": METRIC, "value": total_ms, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": step_config(args.workload, w, world),
            "timed": {"hot_path_steps": 1, "slices": args.steps, "slice_ms": [1e3 * t for t in slices],
                      "parts_s": {k: r[k] for k in ("clover_s", "solve_s", "force_s")}},
            "cpu_baseline": {"value": total_ms, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": total_ms, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_dslash_only(args):
    """Load the workload's links, build the clover term, apply Mhat^dag Mhat in FP32 (12-real links)
    and FP64 `steps` times each; prints a one-line JSON summary (for profiler captures)."""
    import torch
    from paper_0910_0262_gb300 import synth, build
    from paper_0910_0262_gb300 import qcd as Q
    build.build()
    w = workload_params(args.workload)
    nrhs = args.nrhs or w["nrhs"]
    U_np, b_np = synth.make_problem(w["dims"], w["eps"], w["seed"], nrhs)
    op = Q.CloverWilson(w["dims"], w["t_bc"])
    op.load_gauge(torch.from_numpy(U_np).cuda(), recon12=True)
    op.clover_build(w["kappa"], w["csw"])
    b = torch.from_numpy(b_np).cuda()
    for prec in [int(p) for p in args.precs.split(",")]:
        for _ in range(args.steps):
            y = op.dslash(b, Q.QCD_OP_MDAGM, precision=prec)
    torch.cuda.synchronize()
    print(json.dumps({"only": "dslash", "workload": args.workload, "applications": args.steps,
                      "norm": float(torch.linalg.vector_norm(y).item())}))


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.only == "dslash":
        run_dslash_only(args)
        return
    if args.only == "peaks":
        from paper_0910_0262_gb300 import build
        from paper_0910_0262_gb300 import qcd as Q
        build.build()
        print(json.dumps({"only": "peaks", **measure_device_peaks(Q),
                          "hbm_copy_gbs_1GiB": Q.qcd_probe_copy_bandwidth(1 << 30, 10)}))
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, world, rank)))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = run_ours(args, world, rank, local)
    if world > 1:
        res["value"] = res["ms_per_step"]
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
