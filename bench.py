"""Benchmark of the Vegas + |M|^2 hot path (g g -> t tbar g g, 2^22 events/step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload gg_ttxgg_13tev] [--no-cpu-baseline]

A step is one Vegas iteration of the whole path: Philox uniforms, Vegas map,
luminosity map, RAMBO on diet + massive rescaling, cuts, |M|^2 (helicity and
colour sums), Vegas accumulation, deterministic reduction and grid refinement.
The headline arm (FP32 amplitudes) is timed with CUDA events per step, with an
L2 flush between steps outside the timed region; the FP64 arm, the FP32/FP64
cross-section error on an identical frozen grid, an end-to-end number through
the C ABI with host buffers, the FMA-pipe roofline of the |M|^2 kernel, the
derivative workload (mf_grad, 2^20 events), the mixed multi-process launch and
the oracle timed on the host cores are added to the one JSON line rank 0 prints.
An iteration runs in chunks of 2^20 events: a sampling kernel writes per-event
records and the list of events passing the cuts, the |M|^2 kernel (k_me_acc)
evaluates the listed events and accumulates the Vegas sums.

``--impl reference`` times the FP64 CPU oracle (there is no runnable reference
implementation: the paper ships no code), on the host cores, on a bounded
sample of the same workload.

Multi-GPU (torchrun): every rank processes its own 2^22 events (weak scaling,
disjoint Philox event ranges); the Vegas totals (2 + 50 d + 2 doubles) are
all-reduced once per step before the refinement.
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "gg→tt̄gg events/s on 1 GB300, FP32/TC vs FP64 fused at σ rel.err≤1e-5; % FMA peak"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP32_LANES_PER_SM = 128            # FP32 FMA lanes per Blackwell SM (4 sub-partitions x 32)
FP64_NOMINAL_TFLOPS = 1.25         # GB300's published FP64 rate (the measured DFMA rate is reported beside it)


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# --------------------------------------------------------------------------- oracle (CPU) legs
def _oracle_worker(args):
    """Oracle event weights of a block of events (runs in a spawned process)."""
    cfg, seed, it, start, count = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import integrate as oi, philox, vegas
    st = oi.Setup(cfg, amplitude="feynman")
    ev = np.arange(start, start + count, dtype=np.uint64)
    y = philox.uniforms(seed, it, ev, st.ndim)
    w, _ = st.weights(y, vegas.uniform_grid(st.ndim))
    return float(w.sum()), int(count)


def oracle_rate(cfg, seed, seconds, cores, block=64):
    """Events/s of the oracle on `cores` processes, running for ~`seconds`."""
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    done = 0
    nxt = 0
    with ctx.Pool(cores) as pool:
        # warm the workers (imports, colour matrices) outside the clock
        pool.map(_oracle_worker, [(cfg, seed, 99, 0, 2)] * cores)
        t0 = time.perf_counter()
        pending = []
        while True:
            while len(pending) < 2 * cores and time.perf_counter() - t0 < seconds:
                pending.append(pool.apply_async(_oracle_worker, ((cfg, seed, 0, nxt, block),)))
                nxt += block
            if not pending:
                break
            r = pending.pop(0).get()
            done += r[1]
        dt = time.perf_counter() - t0
    return done / dt, done, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return 0
    from paper_2211_14056_gb300.workloads import WORKLOADS, oracle_cfg
    w = WORKLOADS[args.workload]
    cores = host_cores()
    per_step = max(3.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    rates = []
    for i in range(args.warmup + args.steps):
        rate, n, dt = oracle_rate(oracle_cfg(w), w["seed"], per_step, cores)
        if i >= args.warmup:
            rates.append((rate, n, dt))
    value = statistics.mean(r[0] for r in rates)
    sample = (f"first {rates[0][1]} events of iteration 0 of {args.workload} per step "
              f"(~{per_step:.0f} s of CPU work on {cores} processes), FP64 Feynman-diagram oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(r[2] for r in rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "events_per_step": "time-bounded sample", "cpu": cpu_model()},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gg_ttxgg_13tev")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the derivative and mixed-launch legs")
    ap.add_argument("--adapt-events", type=int, default=2 ** 20)
    ap.add_argument("--profile-case", type=int, default=0, metavar="EVENTS",
                    help="only run 3 iterations of EVENTS events each (small case for ncu captures)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32tc", "fp64"],
                    help="arithmetic of --profile-case (fp32tc: FP32 with the tensor-core colour sum)")
    ap.add_argument("--launch-shapes", action="store_true",
                    help="only run the full launch-shape sweep of the |M|^2 kernel (10^6 g g -> t tbar g g events "
                         "per shape) and print it as one JSON line")
    ap.add_argument("--profile-kernel", default="iterate", choices=["iterate", "me", "grad", "pdf", "hel"],
                    help="--profile-case target: whole iterations, sampling + the |M|^2 kernel alone, "
                         "two reverse-mode derivative calls (mf_grad with every per-event output), the "
                         "parton-density kernel, or iterations with helicity sampling (hel)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import numpy as np
    import torch
    import paper_2211_14056_gb300 as mf
    from paper_2211_14056_gb300 import flops as mflops
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, oracle_cfg, process_kwargs

    torch.cuda.set_device(local)
    if args.launch_shapes:
        print(json.dumps({"launch_shapes": _launch_shape_leg(mf, torch, full=True)}), flush=True)
        return 0
    if args.profile_case:
        w = WORKLOADS[args.workload]
        prec = {"fp32": mf.MF_FP32, "fp32tc": mf.MF_FP32_TC, "fp64": mf.MF_FP64}[args.precision]
        p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, prec))
        g = p.grid()
        if args.profile_kernel == "me":
            ne = args.profile_case
            mom = torch.empty(p.n_ext * 4 * ne, dtype=torch.float64, device="cuda")
            me = torch.empty(ne, dtype=torch.float64, device="cuda")
            p.sample(g, w["seed"], 0, ne, momenta=mom)
            for it in range(3):
                p.matrix_element(ne, mom, me)
            torch.cuda.synchronize()
            print(json.dumps({"profile_case": args.workload, "kernel": "me", "events": ne,
                              "precision": args.precision, "mean_me2": float(me.mean())}))
            return 0
        if args.profile_kernel == "pdf":
            r = _pdf_leg(mf, torch, n=args.profile_case, reps=2)
            print(json.dumps({"profile_case": "pdf", "points": args.profile_case, "result": r}))
            return 0
        if args.profile_kernel == "grad":
            ne = args.profile_case
            th = torch.empty(3 * ne, dtype=torch.float64, device="cuda")
            dy = torch.empty(p.ndim * ne, dtype=torch.float64, device="cuda")
            for it in range(2):
                sigma, ds = p.grad(g, w["seed"], it, ne, th, dy)
            print(json.dumps({"profile_case": args.workload, "kernel": "grad", "events": ne,
                              "precision": args.precision, "sigma": sigma, "dsigma": ds}))
            return 0
        if args.profile_kernel == "hel":
            p.set_helicity_sampling(True)     # iterations with one drawn helicity configuration per event
        for it in range(3):
            r = p.vegas_iterate(g, w["seed"], it, args.profile_case, refine=True)
        print(json.dumps({"profile_case": args.workload, "events": args.profile_case, "precision": args.precision,
                          "I": r["I"], "sigma": r["sigma"]}))
        return 0
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = WORKLOADS[args.workload]
    n = w["events"]
    ng = {"gg_ttx": 2, "gg_ttxg": 3, "gg_ttxgg": 4}[w["process"]]
    pid = PROCESS_IDS[w["process"]]
    from paper_2211_14056_gb300.sharding import shard_range
    first, _ = shard_range(rank, world, n)             # this rank's Philox event range
    p32 = mf.Process(pid, **process_kwargs(w, mf.MF_FP32))
    ptc = mf.Process(pid, **process_kwargs(w, mf.MF_FP32_TC))
    p64 = mf.Process(pid, **process_kwargs(w, mf.MF_FP64))
    stream = torch.cuda.current_stream()

    # 1. adapt a grid in FP64 (5 iterations on a smaller event count), then freeze it
    g64 = p64.grid()
    adapt_n = min(args.adapt_events, n)
    for it in range(5):
        p64.vegas_accumulate(g64, w["seed"], it, first, adapt_n)
        if dist is not None:
            _allreduce_totals(dist, g64, torch)
        p64.vegas_finish(g64, adapt_n * world, refine=True)
    frozen = g64.get()
    g32 = p32.grid()
    gtc = ptc.grid()
    gtc.set(frozen)
    g32.set(frozen)
    g64.set(frozen)

    # 2. sigma error FP32 vs FP64 on identical events and the identical frozen grid
    w32 = torch.empty(n, dtype=torch.float64, device="cuda")
    w64 = torch.empty(n, dtype=torch.float64, device="cuda")
    r32 = _iter(p32, g32, 1000, False, w32, dist, torch, w, first, n, world)
    r64 = _iter(p64, g64, 1000, False, w64, dist, torch, w, first, n, world)
    sig_err = abs(r32["I_k"] / r64["I_k"] - 1)
    rtc = _iter(ptc, gtc, 1000, False, None, dist, torch, w, first, n, world)
    sig_err_tc = abs(rtc["I_k"] / r64["I_k"] - 1)
    both = (w64 != 0) & (w32 != 0)
    flips = int(((w64 != 0) ^ (w32 != 0)).sum())      # cut / threshold decisions taken differently
    relw = ((w32[both] - w64[both]).abs() / w64[both].abs()).double()
    w_max_fp32 = float(w32.max())                     # the unweighting's maximum weight (this frozen grid)
    ev_err = {"max": float(relw.max()), "median": float(relw.median()),
              "p999": float(torch.quantile(relw[: 2 ** 24].float(), 0.999)),
              "decision_flips": flips, "events_compared": int(both.sum())}
    del w32, w64

    # 3. FP64 arm timing (1 warm-up + 2 steps)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(proc, grid, steps, warm, base_it):
        for i in range(warm):
            _iter(proc, grid, base_it + i, True, None, dist, torch, w, first, n, world)
        grid.profile(True)
        times, acc_times, passes, me_times = [], [], [], []
        launches0 = mf.kernel_launches()
        for i in range(steps):
            flush.fill_(float(i))
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            proc.vegas_accumulate(grid, w["seed"], base_it + warm + i, first, n)
            e1.record(stream)
            if dist is not None:
                _allreduce_totals(dist, grid, torch)
            r = proc.vegas_finish(grid, n * world, refine=True)
            e2.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e2))
            acc_times.append(e0.elapsed_time(e1))
            passes.append(r["n_pass"])
            smp_ms, me_ms, chunks = grid.profile_read()
            me_times.append((me_ms, chunks, smp_ms))
        launches = mf.kernel_launches() - launches0
        grid.profile(False)
        return times, acc_times, passes, launches, me_times

    t64, a64, pass64, _, me64 = timed(p64, g64, 2, 1, 2000)
    ms64 = _max_over_ranks(statistics.mean(t64), dist, torch)

    # 4. headline FP32 arm: K timed steps (clocks sampled meanwhile)
    with ClockSampler(local) as clk:
        t32, a32, pass32, launches, me32 = timed(p32, g32, args.steps, args.warmup, 3000)
        ttc, _, _, _, metc = timed(ptc, gtc, args.steps, args.warmup, 3000)
    mstc = _max_over_ranks(sum(ttc) / args.steps, dist, torch)
    ms32 = _max_over_ranks(sum(t32) / args.steps, dist, torch)
    value = n * world / (ms32 * 1e-3)
    value64 = n * world / (ms64 * 1e-3)

    # 5. end to end through the C ABI with host buffers: grid edges in, result out
    e2e_steps = max(2, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        g32.set(frozen)                                    # H2D of the host-side grid
        r = p32.vegas_iterate(g32, w["seed"], 4000 + i, n, refine=True)   # D2H of the result
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = n / e2e_s

    # 6. roofline of the dominant kernel, k_me_acc (FMA pipes): algorithmic
    #    flops of the events it evaluates / its CUDA-event time on the stream
    fpe = mflops.me2_flops_per_event(ng)
    me_ms = statistics.mean(m[0] for m in me32)
    chunks = me32[0][1]
    achieved = fpe * statistics.mean(pass32) / (me_ms * 1e-3) / 1e12
    peak_meas = mf.fma_throughput(mf.MF_FP32)
    peak64_meas = mf.fma_throughput(mf.MF_FP64)
    achieved64 = fpe * statistics.mean(pass64) / (statistics.mean(m[0] for m in me64) * 1e-3) / 1e12
    traffic = _ncu_traffic("k_me_acc_gg_ttxgg_fp32")
    # the sampling kernel's HBM roofline: record bytes written per event over
    # its CUDA-event time (it is bound by the FP64 pipe, not by HBM)
    hbm_peak = _measured_peaks().get("hbm_gbs")
    spe = mflops.sampler_bytes_per_event(ng, p32.ndim, statistics.mean(pass32) / n, 4)
    smp_ms = statistics.mean(m[2] for m in me32)
    smp_gbs = spe * n / (smp_ms * 1e-3) / 1e9
    sm_max = _measured_peaks().get("sm_max_mhz", 2070.0)
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    peak_derived = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12

    # 7. the derivative and mixed-launch workloads (N = 1 only)
    grad = mixed = shapes = pp = pdfk = unw = hel = None
    if world == 1 and not args.no_extras:
        grad = _grad_leg(p32, p64, g32, g64, w, torch)
        mixed = _mixed_leg(mf, torch)
        shapes = _launch_shape_leg(mf, torch)
        pp = _pp_leg(mf, torch)
        pdfk = _pdf_leg(mf, torch)
        unw = _unweight_leg(p32, g32, w, torch, n, w_max_fp32)
        hel = _helicity_leg(mf, torch, w, frozen, n)

    # 8. CPU baseline: the oracle on the host cores (rank 0 only, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate, done, dt = oracle_rate(oracle_cfg(w), w["seed"], 20.0, cores)
        cpu = {"value": rate, "unit": "events/s", "cores": cores, "kind": "oracle",
               "sample": f"events 0..{done - 1} of iteration 0 on the uniform grid, {dt:.1f} s on {cores} "
                         f"processes ({cpu_model()}), FP64 Feynman-diagram oracle"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "process": "g g -> t tbar g g", "events_per_step": n,
                       "precision": "FP32 kinematics and amplitudes (FMA colour sum); FP64 Vegas map, Newton polish, "
                                    "weight and sums",
                       "l2": "flushed (512 MB write) between timed steps; inputs are generated in-kernel",
                       "grid": "adapted by 5 FP64 iterations of 2^20 events, then refined every step"},
            "fp64": {"value": value64, "unit": "events/s", "ms_per_step": ms64},
            "fp32_tc": {"value": n * world / (mstc * 1e-3), "unit": "events/s", "ms_per_step": mstc,
                        "me_ms_per_step": statistics.mean(m[0] for m in metc), "sigma_rel_err_vs_fp64": sig_err_tc,
                        "colour_sum": "integer D C on the tensor cores (mma.m16n8k8 TF32, J split hi + lo, FP32 "
                                      "accumulate); same steps, same frozen grid and events as the headline arm"},
            "speedup_fp32_vs_fp64": value / value64,
            "sigma_rel_err_fp32_vs_fp64": sig_err, "event_rel_err_fp32": ev_err,
            "pass_fraction": statistics.mean(pass32) / (n * world),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_derived, "unit": "TFLOP/s",
                         "frac": achieved / peak_derived, "traffic": traffic,
                         "kernel": "k_me_acc<4,float>", "flops_per_event": fpe,
                         "launch_ms": me_ms / chunks, "launches_per_step": chunks,
                         "sampling_ms_per_step": smp_ms,
                         "sampling": {"kernel": "k_sample_rec<float>", "bound": "FP64 pipe (Vegas map, Newton "
                                      "polish, weight), not HBM", "bytes_per_event": spe, "achieved": smp_gbs,
                                      "peak": hbm_peak, "unit": "GB/s",
                                      "frac": (smp_gbs / hbm_peak) if hbm_peak else None,
                                      "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
                         "peak_source": f"derived: {sm_count} SMs (device) x {FP32_LANES_PER_SM} FP32 FMA lanes x "
                                        f"2 flop x {sm_max:.0f} MHz",
                         "peak_measured_fma": peak_meas, "frac_of_measured_fma": achieved / peak_meas,
                         "fp64": {"kernel": "k_me_acc<4,double>", "achieved": achieved64, "peak": FP64_NOMINAL_TFLOPS,
                                  "frac": achieved64 / FP64_NOMINAL_TFLOPS, "peak_source": "nominal FP64 rate",
                                  "peak_measured_fma": peak64_meas, "frac_of_measured_fma": achieved64 / peak64_meas}},
            "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": int(frozen.nbytes),
                    "d2h_bytes_per_step": 48},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if grad is not None:
            line["grad"] = grad
        if mixed is not None:
            line["mixed"] = mixed
        if shapes is not None:
            line["launch_shape"] = shapes
        if pp is not None:
            line["pp_ttxgg"] = pp
        if pdfk is not None:
            line["pdf_interpolation"] = pdfk
        if unw is not None:
            line["unweighting"] = unw
        if hel is not None:
            line["helicity_sampling"] = hel
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _grad_leg(p32, p64, g32, g64, w, torch):
    """mf_grad (reverse mode) on the frozen grid: d sigma/d(g_s, m_t, Gamma_t)
    and the per-event derivatives with respect to every uniform; events/s."""
    out = {}
    for name, p, g, n, reps in (("fp32", p32, g32, 2 ** 20, 2), ("fp64", p64, g64, 2 ** 18, 1)):
        th = torch.empty(3 * n, dtype=torch.float64, device="cuda")
        dy = torch.empty(p.ndim * n, dtype=torch.float64, device="cuda")
        p.grad(g, w["seed"], 5000, 4096, th, dy)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(reps):
            sigma, ds = p.grad(g, w["seed"], 5001 + r, n, th, dy)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"events": n, "ms": ms, "events_per_s": n / (ms * 1e-3), "sigma_pb": sigma,
                     "dsigma_dgs_dmt_dwt": ds, "mode": "reverse: one adjoint sweep of |M|^2 per event",
                     "sampler_tangent_passes": 1 + p.ndim // 2,
                     "per_event_outputs": "dw/d(g_s, m_t, Gamma_t) [3, n], dw/dy [ndim, n]"}
        del th, dy
    return out


def _mixed_leg(mf, torch, iters=5):
    """The batched launch of several processes (own grids, FP32): the
    autotuner's candidates, then graph-replayed iterations; against the same
    processes iterated one after the other through mf_vegas_iterate."""
    from paper_2211_14056_gb300.workloads import MIXED, PROCESS_IDS, WORKLOADS, process_kwargs
    seed = MIXED["seed"]

    def make():
        procs, grids = [], []
        for name in MIXED["workloads"]:
            wk = WORKLOADS[name]
            p = mf.Process(PROCESS_IDS[wk["process"]], **process_kwargs(wk, mf.MF_FP32))
            procs.append(p)
            grids.append(p.grid())
        return procs, grids

    procs, grids = make()
    m = mf.Mixed(procs, grids, MIXED["events"])
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for it in range(3):
            m.run(seed, it, refine=True, stream=side)
        # tile 0: every process in its own specialised |M|^2 kernel within the iteration
        cands = [(c, t) for c in (1, 2, 0) for t in (8, 32, 128, 512)] + [(0, 0), (2, 0)]
        times, best = m.autotune(seed, cands, stream=side)
        m.use_graph(True)
        m.run(seed, 3, refine=True, stream=side)          # capture
        side.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for i in range(iters):
            res = m.run(seed, 4 + i, refine=True, stream=side)
        e1.record(side)
        side.synchronize()
    ms_mixed = e0.elapsed_time(e1) / iters
    sprocs, sgrids = make()
    for it in range(3):
        for p, g, n in zip(sprocs, sgrids, MIXED["events"]):
            p.vegas_iterate(g, seed, it, n, refine=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(iters):
        for p, g, n in zip(sprocs, sgrids, MIXED["events"]):
            p.vegas_iterate(g, seed, 3 + i, n, refine=True)
    e1.record()
    torch.cuda.synchronize()
    ms_sep = e0.elapsed_time(e1) / iters
    total = sum(MIXED["events"])
    return {"workloads": MIXED["workloads"], "events": MIXED["events"], "ms_per_iteration": ms_mixed,
            "events_per_s": total / (ms_mixed * 1e-3), "separate_ms_per_iteration": ms_sep,
            "speedup_vs_separate": ms_sep / ms_mixed,
            "autotune": {"candidates": cands, "ms": times, "best": cands[best]},
            "graph": True, "I_pb": [r["I"] for r in res]}


def _pp_leg(mf, torch, iters=5):
    """p p -> t tbar g g as the sum of its seven subprocess channels (gg, q q~,
    q~ q, q g, g q, q~ g, g q~; each its own grid, tabulated densities), in one
    mixed plan (FP32): three adaptation iterations, the autotuner's choice of
    launch form, then graph-replayed iterations.  sigma is the sum of the
    channels' estimates, its error their errors in quadrature."""
    from paper_2211_14056_gb300.pdfgrid import synthetic_set
    from paper_2211_14056_gb300.workloads import PP_CHANNELS, PROCESS_IDS, process_kwargs
    pdf = mf.PDFSet.from_dict(synthetic_set())
    names = list(PP_CHANNELS)
    procs = [mf.Process(PROCESS_IDS[PP_CHANNELS[k]["process"]], **process_kwargs(PP_CHANNELS[k], mf.MF_FP32, pdf=pdf))
             for k in names]
    grids = [p.grid() for p in procs]
    n = [PP_CHANNELS[k]["events"] for k in names]
    m = mf.Mixed(procs, grids, n)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for it in range(3):
            m.run(11, it, refine=True, stream=side)
        cands = [(0, 32), (0, 128), (0, 0)]
        times, best = m.autotune(11, cands, stream=side)
        m.use_graph(True)
        m.run(11, 3, refine=True, stream=side)
        side.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for i in range(iters):
            res = m.run(11, 4 + i, refine=True, stream=side)
        e1.record(side)
        side.synchronize()
    ms = e0.elapsed_time(e1) / iters
    total = sum(n)
    sig = sum(r["I_k"] for r in res)
    err = sum(r["sigma_k"] ** 2 for r in res) ** 0.5
    hel = _pp_helicity(mf, torch, names, n, [g.get() for g in grids], pdf)
    return {"channels": names, "events": n, "ms_per_iteration": ms, "events_per_s": total / (ms * 1e-3),
            "helicity_sampling": hel,
            "sigma_pb": sig, "sigma_err_pb": err,
            "channel_sigma_pb": {k: r["I_k"] for k, r in zip(names, res)},
            "autotune": {"candidates": cands, "ms": times, "best": cands[best]}, "precision": "FP32",
            "pdf": "synthetic tabulated set (9 flavours, 97 x 41 nodes), log-bicubic interpolation, "
                   "Q = sqrt(s_hat)/2"}


def _pp_helicity(mf, torch, names, n, edges, pdf, rounds=3):
    """The seven channels on their grids frozen after the mixed run, summed
    against the adapted helicity draw (three table-refining iterations per
    channel first): each round iterates every channel once (one channel
    after another, CUDA events around the round); sigma is the sum of the
    channels' estimates, its error their errors in quadrature, and the
    efficiency gain (time x error^2) summed over the same for the draw."""
    import statistics as stats
    from paper_2211_14056_gb300.workloads import PP_CHANNELS, PROCESS_IDS, process_kwargs
    out = {}
    for label in ("summed", "adapted"):
        procs = [mf.Process(PROCESS_IDS[PP_CHANNELS[k]["process"]], **process_kwargs(PP_CHANNELS[k], mf.MF_FP32, pdf=pdf))
                 for k in names]
        grids = [p.grid() for p in procs]
        for p, g, e, k in zip(procs, grids, edges, names):
            g.set(e)
            if label == "adapted":
                p.set_helicity_sampling("adaptive")
                for it in range(3):
                    p.vegas_iterate(g, 21, 100 + it, PP_CHANNELS[k]["events"], refine="helicities")
        ts, sig, err = [], [], []
        for r in range(rounds):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            res = [p.vegas_iterate(g, 22, 200 + r, m, refine=False) for p, g, m in zip(procs, grids, n)]
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            sig.append(sum(x["I_k"] for x in res))
            err.append(sum(x["sigma_k"] ** 2 for x in res) ** 0.5)
        out[label] = {"ms_per_round": stats.mean(ts), "events_per_s": sum(n) / (stats.mean(ts) * 1e-3),
                      "sigma_pb": stats.mean(sig), "sigma_err_pb": stats.mean(err)}
    u, a = out["summed"], out["adapted"]
    out["efficiency_gain"] = (u["ms_per_round"] * u["sigma_err_pb"] ** 2) / (a["ms_per_round"] * a["sigma_err_pb"] ** 2)
    return out


def _pdf_leg(mf, torch, n=2 ** 26, reps=5):
    """The interpolation kernel alone (mf_pdf_eval, FP32 arithmetic): x and Q^2
    read, x f written (24 bytes per point of HBM traffic, 1.5 GB per launch,
    inputs larger than L2); GB/s against the measured copy bandwidth."""
    import statistics as stats
    from paper_2211_14056_gb300 import pdfgrid
    pdf = mf.PDFSet.from_dict(pdfgrid.synthetic_set())
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    x = torch.exp(torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-9.0, 0.0, generator=g))
    q2 = torch.exp(torch.empty(n, dtype=torch.float64, device="cuda").uniform_(2.0, 18.0, generator=g))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    res = {}
    for name, prec in (("fp32", mf.MF_FP32), ("fp64", mf.MF_FP64)):
        pdf.eval(pdfgrid.GLUON, n, x, q2, out, precision=prec)
        ts = []
        for r in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            pdf.eval(pdfgrid.GLUON, n, x, q2, out, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = stats.mean(ts)
        gbs = 24.0 * n / (ms * 1e-3) / 1e9
        peak = _measured_peaks().get("hbm_gbs")
        res[name] = {"points": n, "ms": ms, "points_per_s": n / (ms * 1e-3), "achieved": gbs, "unit": "GB/s",
                     "peak": peak, "frac": gbs / peak if peak else None}
    res["kernel"] = "k_pdf_eval (flavour table staged in shared memory)"
    res["bytes_per_point"] = 24
    return res


def _unweight_leg(p, g, w, torch, n, w_max, reps=3):
    """Hit-or-miss unweighting (mf_unweight) of n FP32 g g -> t tbar g g events
    on the frozen grid with w_max = the largest weight of one iteration: the
    same kernels as an iteration plus the hit-or-miss pass; unweighted events
    per second and the unweighting efficiency."""
    import statistics as stats
    cap = n // 8
    mom = torch.empty(p.n_ext * 4 * cap, dtype=torch.float64, device="cuda")
    wt = torch.empty(cap, dtype=torch.float64, device="cuda")
    ev = torch.empty(cap, dtype=torch.int64, device="cuda")
    p.unweight(g, w["seed"], 6000, 0, n, w_max, cap, mom, wt, ev)
    ts, kept = [], []
    for r in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        k, o, st = p.unweight(g, w["seed"], 6001 + r, 0, n, w_max, cap, mom, wt, ev)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        kept.append(k)
    ms = stats.mean(ts)
    return {"events": n, "w_max": w_max, "ms": ms, "weighted_events_per_s": n / (ms * 1e-3),
            "kept_per_call": stats.mean(kept), "unweighted_events_per_s": stats.mean(kept) / (ms * 1e-3),
            "efficiency": stats.mean(kept) / n}


def _helicity_leg(mf, torch, w, edges, n, reps=4):
    """Helicity sampling against the helicity sum: FP32 g g -> t tbar g g on
    the frozen grid `edges`, `reps` iterations of n events each way (distinct
    iteration numbers, no refinement).  Per way: CUDA-event time per
    iteration, its |M|^2 kernel's share, the variance per event n sigma_k^2
    (mean over the iterations) and the estimate; the efficiency gain is
    (time x variance) summed over (time x variance) sampled: how much less
    device time the sampled form needs for the same statistical error."""
    import statistics as stats
    from paper_2211_14056_gb300 import flops as mflops
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, process_kwargs
    out = {}
    for label, on in (("summed", False), ("sampled", True), ("adapted", "adaptive")):
        p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, mf.MF_FP32))
        p.set_helicity_sampling(on)
        g = p.grid()
        g.set(edges)
        if on == "adaptive":
            # the helicity table adapts over five iterations (the edges stay frozen)
            for it in range(5):
                p.vegas_iterate(g, w["seed"], 6900 + it, n, refine="helicities")
        p.vegas_iterate(g, w["seed"], 7000, n, refine=False)
        g.profile(True)
        ts, me, var, Is, npass = [], [], [], [], []
        for r in range(reps):
            g.set(edges)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            res = p.vegas_iterate(g, w["seed"], 7001 + r, n, refine=False)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            me.append(g.profile_read()[1])
            var.append(res["sigma_k"] ** 2 * n)
            Is.append(res["I_k"])
            npass.append(res["n_pass"])
        g.profile(False)
        fpe = mflops.me2_flops_per_event_hel(4) if on else mflops.me2_flops_per_event(4)
        me_ms = stats.mean(me)
        out[label] = {"ms_per_iteration": stats.mean(ts), "me_ms": me_ms, "events_per_s": n / (stats.mean(ts) * 1e-3),
                      "var_per_event": stats.mean(var), "I_k": Is, "flops_per_event": fpe,
                      "me_tflops": fpe * stats.mean(npass) / (me_ms * 1e-3) / 1e12}
    u = out["summed"]
    out["kernel"] = "k_me_acc_hel<4,float> (sampled, adapted) vs k_me_acc<4,float> (summed)"
    out["events"] = n
    out["draw"] = ("sampled: uniform over the 32 configurations of the gluons and the antitop, top summed; "
                   "adapted: the same with the helicity table refined over five iterations")
    for k in ("sampled", "adapted"):
        s = out[k]
        s["variance_ratio"] = s["var_per_event"] / u["var_per_event"]
        s["time_ratio"] = u["ms_per_iteration"] / s["ms_per_iteration"]
        s["efficiency_gain"] = (u["ms_per_iteration"] * u["var_per_event"]) / (s["ms_per_iteration"] * s["var_per_event"])
    out["efficiency_gain"] = out["sampled"]["efficiency_gain"]
    out["efficiency_gain_adapted"] = out["adapted"]["efficiency_gain"]
    return out


def _launch_shape_leg(mf, torch, full=False, n=10 ** 6, reps=3):
    """The launch-shape study (arXiv:2211.14056 Sec. 3, Fig. 3: run time of
    10^6 g g -> t tbar g g events against threads per block): one Vegas
    accumulation of n FP32 events (sampling + |M|^2 + accumulation) per launch
    shape of the |M|^2 kernel, warps per CTA 1..7 (32..224 threads) at the
    most CTAs per SM that fit (``full``: every CTA count up to that), on the
    uniform grid.  Times are CUDA events on the stream, mean of `reps` calls
    after one warm-up call."""
    import statistics as stats
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS["gg_ttxgg_13tev"]
    p = mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, mf.MF_FP32))
    g = p.grid()
    pts = []
    for W in range(1, 8):
        cmax = p.set_launch_shape(W)
        cs = list(range(1, cmax + 1)) if full else sorted({cmax, 1} if W == 4 else {cmax})
        for c in cs:
            p.set_ctas_per_sm(c)
            p.vegas_accumulate(g, w["seed"], 0, 0, n)
            g.profile(True)
            tt, tm = [], []
            for r in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                p.vegas_accumulate(g, w["seed"], 1 + r, 0, n)
                e1.record()
                torch.cuda.synchronize()
                tt.append(e0.elapsed_time(e1))
                tm.append(g.profile_read()[1])
            g.profile(False)
            ms = stats.mean(tt)
            pts.append({"threads_per_block": 32 * W, "warps_per_cta": W, "ctas_per_sm": c, "warps_per_sm": W * c,
                        "ms": ms, "me_ms": stats.mean(tm), "events_per_s": n / (ms * 1e-3)})
    p.set_launch_shape(0)
    p.set_ctas_per_sm(0)
    best = min(pts, key=lambda x: x["ms"])
    default = [x for x in pts if x["warps_per_cta"] == 4 and x["ctas_per_sm"] == max(
        y["ctas_per_sm"] for y in pts if y["warps_per_cta"] == 4)][0]
    return {"workload": "gg_ttxgg_13tev (uniform grid), FP32", "events": n, "points": pts, "best": best,
            "default": default}


def _ncu_traffic(name):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None): the summary lists the source files
    the kernel is compiled from (`kernel_sources`) and their SHA-256."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        k, _, v = line.strip().partition(":")
        if k in ("dram_bytes_per_launch", "sources_sha256", "kernel_sources"):
            rec[k] = v.strip()
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2211_14056_gb300", "csrc")
    files = rec["kernel_sources"].split() if "kernel_sources" in rec else \
        sorted(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    if rec.get("sources_sha256") != h.hexdigest() or "dram_bytes_per_launch" not in rec:
        return None
    return int(rec["dram_bytes_per_launch"])


def _allreduce_totals(dist, grid, torch):
    """Sum the grid's device totals over ranks (NCCL), in place."""
    from paper_2211_14056_gb300.sharding import allreduce_totals, totals_tensor
    allreduce_totals(totals_tensor(grid))


def _iter(proc, grid, it, refine, weights, dist, torch, w, first, n, world):
    proc.vegas_accumulate(grid, w["seed"], it, first, n, weights=weights)
    if dist is not None:
        _allreduce_totals(dist, grid, torch)
    return proc.vegas_finish(grid, n * world, refine=refine)


def _max_over_ranks(x, dist, torch):
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


if __name__ == "__main__":
    sys.exit(main())
