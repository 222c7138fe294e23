"""Throughput of the TWA hot path on B300: spin-trajectory-steps per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: N = 10^4 spins, alpha = 1, w = N Gamma / 2, Gamma = 1, dt = 2e-5,
M = 1024 trajectories per GPU (weak scaling: rank r runs trajectories
[r M, (r+1) M) of one ensemble), W and L held as BF16 hi+lo images, FP32 state,
BF16X2 contractions on tcgen05 (W hi + lo and L hi + lo against the state and
the noise rounded once to BF16). One step = one stochastic-Heun step of all M
trajectories: noise, L.eta and W.s (predictor), W.s~ (corrector), moments.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
the host cores instead, on a bounded trajectory sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2608_10075_b300.configs import LARGE_N1E4 as CFG  # noqa: E402

METRIC = "spin-traj-steps/s at N=1e4 (mixed vs FP64 GPU, observables within 3 SE)"
UNIT = "spin-traj-steps/s"
WORKLOAD = ("TWA stochastic Heun, N=10000 alpha=1 w=5000 Gamma=1 dt=2e-5, M=1024 trajectories/GPU, "
            "BF16B tcgen05 contractions (W and L one BF16 product, hi+lo within 64 columns of the diagonal, "
            "against a BF16 operand), FP32 state")
REF_SAMPLE_M = 16


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# The tensor-core kernel and its device helpers occupy twa_tc.cu up to this line;
# the host code after it does not change the kernel.
KERNEL_SECTION_END = "// elementwise kernels of the mixed path"


def kernel_source_sha(kernel_file):
    """sha256 prefix of the kernel section of a source file (the whole file if
    it has no section marker)."""
    src = os.path.join(ROOT, "paper_2608_10075_b300", "csrc", kernel_file)
    text = open(src, "rb").read()
    cut = text.find(KERNEL_SECTION_END.encode())
    return hashlib.sha256(text[:cut] if cut >= 0 else text).hexdigest()[:16]


def recorded_traffic(kernel_file, summary):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (matching sha256 prefix of the kernel section);
    else None."""
    path = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_2608_10075_b300", "csrc", kernel_file)
    if not (os.path.exists(path) and os.path.exists(src)):
        return None
    sha = kernel_source_sha(kernel_file)
    txt = open(path).read()
    m_sha = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", txt)
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if m_sha and m_b and m_sha.group(1) == sha:
        return float(m_b.group(1))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms, from before
    the warm-up to the end of the run; mark() notes the sample index at a point
    of the run and stats(a, b) summarises the samples between two marks."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, device_index, interval_ms=50):
        self.idx = device_index
        self.interval = interval_ms
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def mark(self):
        # let the sampler catch up with the work just finished
        time.sleep(2.5 * self.interval / 1000.0)
        return len(self.lines)

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()

    def stats(self, a=0, b=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm, smax, power, reasons = [], [], [], set()
        for ln in self.lines[a:b]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(self.NAMES, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm),
                "interval_ms": self.interval}


def fft_length(N):
    """Circle length of the Toeplitz route: the smallest even 2^a 3^b 5^c >= max(2, 2N - 2)."""
    P = max(2, 2 * N - 2)
    while True:
        v = P
        for f in (2, 3, 5):
            while v % f == 0:
                v //= f
        if v == 1 and P % 2 == 0:
            return P
        P += 1


# FP32 peak of the FFT route's ALU work: 148 SMs x 128 FP32 lanes x 2 FLOP per
# FMA x 2032 MHz (the maximum SM clock)
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2032e6 / 1e12


def fft_roofline(N, M, kernel_ms):
    """FP32 roofline of the FFT route's dominant kernel (predictor or corrector:
    one forward and one inverse complex transform of length P per trajectory,
    5 P log2 P FLOP each)."""
    import math
    P = fft_length(N)
    flops = 2 * 5.0 * P * math.log2(P) * M
    k = max(("predict", "correct"), key=lambda x: kernel_ms.get(x, 0.0))
    achieved = flops / (kernel_ms[k] * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "k_fft_%s" % ("pred" if k == "predict" else "corr"), "P": P,
            "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
            "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 FLOP/FMA x 2032 MHz",
            "flops_per_launch": flops, "kernel_ms": kernel_ms[k]}


def host_threads():
    """Threads the oracle's BLAS uses (its matmuls are the only parallel part)."""
    try:
        from threadpoolctl import threadpool_info
        return max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except ImportError:
        # OpenBLAS defaults to one thread per available core
        return len(os.sched_getaffinity(0))


def cpu_oracle_rate(N, M_sample, steps, cfg, min_seconds=10.0):
    """Time the FP64 CPU oracle (as it stands) on a trajectory sample: at least
    `steps` steps and at least `min_seconds` of host work."""
    from oracle.twa_oracle import TWAOracle
    o = TWAOracle(N, cfg["alpha"], cfg["w"], cfg["Gamma"], cfg["dt"], 0, M_sample)
    o.run(1)   # warm-up step (first-touch of buffers)
    t0 = time.perf_counter()
    done = 0
    while done < steps or time.perf_counter() - t0 < min_seconds:
        o.run(1)
        done += 1
    el = time.perf_counter() - t0
    return N * M_sample * done / el, el, host_threads(), done


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    N = CFG["N"]
    K, Wm = args.steps, args.warmup
    from oracle.twa_oracle import TWAOracle
    t_setup = time.perf_counter()
    o = TWAOracle(N, CFG["alpha"], CFG["w"], CFG["Gamma"], CFG["dt"], 0, REF_SAMPLE_M)
    t_setup = time.perf_counter() - t_setup
    o.run(Wm)
    t0 = time.perf_counter()
    o.run(K)
    el = time.perf_counter() - t0
    threads = host_threads()
    v = N * REF_SAMPLE_M * K / el
    sample = "%d of the %d trajectories, all %d sites, %d timed steps (+%d warm-up); W, L set-up %.1f s untimed" % (
        REF_SAMPLE_M, CFG["M"], N, K, Wm, t_setup)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": 1e3 * el / max(K, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "TWA stochastic Heun, N=10000 alpha=1 w=5000 Gamma=1 dt=2e-5, "
                                   "%d-trajectory sample of the M=1024 ensemble, FP64 CPU oracle" % REF_SAMPLE_M,
                       "N": N, "M": REF_SAMPLE_M, "alpha": CFG["alpha"], "w": CFG["w"], "dt": CFG["dt"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def precision_check(twa, stream, rank, precisions, M_sub=128, steps=200):
    """The metric's qualifier on a subset of the ensemble: each mixed precision
    and the FP64 GPU path on the same trajectories and seeds, `steps` steps,
    window over the second half; unpaired differences in units of the combined
    standard error, and the paired per-trajectory difference with its
    standard error."""
    import math

    import numpy as np
    N = CFG["N"]
    t0 = (steps // 2) * CFG["dt"]
    obs, smp = {}, {}
    for prec in ("fp64",) + tuple(precisions):
        with twa.TWA(N, CFG["alpha"], CFG["w"], CFG["Gamma"], CFG["dt"], seed=0, precision=prec, stream=stream,
                     traj_offset=rank * CFG["M"], window_start=t0) as g:
            g.run(M_sub, steps)
            obs[prec] = g.observables()
            Sz, A, A2, ASz, Sz2 = g.moments().T
            smp[prec] = {"Sz": Sz, "SpSm": A + 0.5 * Sz, "G2num": A2 + 2 * ASz - Sz / 3 + 0.5 * Sz2 - 4.0 / 3.0 * A}
    out = {"trajectories": M_sub, "steps": steps, "window_steps": steps - steps // 2}
    b = obs["fp64"]
    for prec in precisions:
        a = obs[prec]
        res = {"observables": {}}
        worst = 0.0
        for k in ("Sz", "SpSm", "G2num", "g2"):
            se = math.hypot(a[k + "_se"], b[k + "_se"])
            r = {"mixed": a[k], "fp64": b[k], "diff_in_se": (a[k] - b[k]) / se}
            if k in smp["fp64"]:
                d = smp[prec][k] - smp["fp64"][k]
                r["paired_diff"] = float(np.mean(d))
                r["paired_se"] = float(np.std(d, ddof=1) / math.sqrt(M_sub))
            worst = max(worst, abs(r["diff_in_se"]))
            res["observables"][k] = r
        res["max_abs_diff_in_se"] = worst
        res["within_3se"] = worst <= 3.0
        out[prec] = res
    return out


def run_ours(args, rank, world, dist):
    import torch

    from paper_2608_10075_b300 import twa

    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    N, M = CFG["N"], CFG["M"]
    K, Wm = args.steps, args.warmup
    clocks = ClockSampler(local).start()
    ctx = twa.TWA(N, CFG["alpha"], CFG["w"], CFG["Gamma"], CFG["dt"], seed=0, precision=CFG["precision"],
                  window_start=0.0, stream=stream, traj_offset=rank * M)
    ctx.run(M, 0)
    ctx.run(M, Wm)
    ctx.sync()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- timed region: K steps, device-resident inputs ----
    barrier()
    torch.cuda.synchronize()
    c0 = clocks.mark()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.run(M, K)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    c1 = clocks.mark()
    ctx.sync()
    if dist is not None:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = N * M * world * K / (ms * 1e-3)

    # ---- per-kernel times on the launching stream (separate pass, same K) ----
    kp = max(K, 20)
    c2 = clocks.mark()
    ctx.profile(True)
    ctx.run(M, kp)
    prof = ctx.profile_read()
    ctx.profile(False)
    c3 = clocks.mark()
    step_kernel_ms = sum(v[0] for v in prof.values()) / max(kp, 1)
    # per launch class the library reports the tensor-core FLOPs it issued
    # (products per entry of the precision, the two-product band included) and
    # the algorithmic FLOPs of the contractions (2 N^2 per column for a W.s, 2
    # per nonzero of L for an L.eta, counted once); the predictor and corrector
    # launches of step t also carry the L.eta tiles of t + 1
    flops = {"predict": 2.0 * N * N * 2 * M, "correct": 2.0 * N * N * 2 * M,
             "noise_factor": 2.0 * (N * (N + 1) / 2.0) * 2 * M}
    alg_total = sum(prof[k][3] for k in flops)
    in_mixed = prof["predict"][3] + prof["correct"][3] - kp * (flops["predict"] + flops["correct"])
    assert min(abs(in_mixed), abs(in_mixed - kp * flops["noise_factor"])) <= 1e-6 * alg_total, in_mixed
    assert abs(prof["noise_factor"][3] - prof["noise_factor"][1] * flops["noise_factor"]) <= 1e-6 * alg_total
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    dominant = max((k for k in flops if prof[k][1]), key=lambda k: prof[k][0])
    n_dom = max(prof[dominant][1], 1)
    d_ms_prof = prof[dominant][0] / n_dom
    # the dominant kernel's time in the timed region: its share of the step in
    # the profiled pass applied to the timed step (launch gaps included, so the
    # per-step kernel times add up to ms_per_step). In the timed region the noise
    # draw of a later step runs on a second stream beside the contractions (the
    # profiled pass runs it alone, to time it): it is left out of the shares.
    noise_overlapped = os.environ.get("TWA_NOISE_OVERLAP", "1") != "0"
    serial_ms = step_kernel_ms - (prof["noise"][0] / kp if noise_overlapped and prof.get("noise") else 0.0)
    share = prof[dominant][0] / kp / serial_ms
    launches_per_step = prof[dominant][1] / kp
    # every launch of a step (the profiled pass counts them per kernel class):
    # predictor and corrector launches and the closing kernel, plus the noise
    # kernel where the draw does not ride in the two launches
    launches_per_step_all = int(round(sum(v[1] for v in prof.values()) / kp))
    d_ms = (ms / K) * share / launches_per_step
    d_exec = prof[dominant][2] / n_dom
    d_algo = prof[dominant][3] / n_dom
    achieved = d_algo / (d_ms * 1e-3) / 1e12
    executed_tflops = d_exec / (d_ms * 1e-3) / 1e12
    step_algo = (2 * 2.0 * N * N * 2 * M + 2.0 * N * (N + 1) / 2.0 * 2 * M)   # W.s twice + L.eta once
    traffic = recorded_traffic("twa_tc.cu", "tc_mix_%s_n10000.md" % dominant)
    kernel_name = {"predict": "k_tc<MIX> (W.s + Heun predictor, with L.eta tiles of step t+1)",
                   "correct": "k_tc<MIX> (W.s~ + Heun corrector, with L.eta tiles of step t+1)",
                   "noise_factor": "k_tc<LETA> (L.eta)"}[dominant]

    # ---- end to end through the C ABI with host buffers ----
    # the state arrives from pinned host memory as FP32 (twa_set_state_f32: the
    # mixed-precision state as it is), every step's moments and the observables
    # go back; the same with FP64 host buffers (twa_set_state) beside it
    mom_bytes = 5 * 8 * M

    def end_to_end(dtype):
        xs = [torch.empty((M, N), dtype=dtype, pin_memory=True) for _ in range(3)]
        host = tuple(x.numpy() for x in xs)
        if dtype == torch.float32:
            ctx.get_state_f32(out=host)
        else:
            ctx.get_state(out=host)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_state(*host)                              # host -> device, pinned
        ctx.run(M, K)
        ctx.moments()                                     # device -> host
        ob = ctx.observables()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if dist is not None:
            tt = torch.tensor([t], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        return N * M * world * K / t, 3 * xs[0].element_size() * M * N, ob

    e2e64, h2d64, _ = end_to_end(torch.float64)
    e2e, h2d, obs = end_to_end(torch.float32)
    d2h = mom_bytes + 160

    # ---- sustained: a seconds-long block of steps under the power limit ----
    sustained = None
    if not args.no_sustained:
        ks = args.sustained_steps
        c4 = clocks.mark()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ctx.run(M, ks)
        a1.record(stream)
        torch.cuda.synchronize()
        s_ms = a0.elapsed_time(a1)
        c5 = clocks.mark()
        sustained = {"value": N * M * world * ks / (s_ms * 1e-3), "ms_per_step": s_ms / ks, "steps": ks,
                     "seconds": s_ms * 1e-3, "clocks": clocks.stats(c4, c5),
                     "all_contractions_algorithmic_tflops": step_algo / (s_ms / ks * 1e-3) / 1e12}
    ctx.close()

    # ---- beside the dense route: the FFT route and the plain FP64 GPU path ----
    def side_run(precision, route, steps, warm, noise="cholesky", integrator="heun"):
        g = twa.TWA(N, CFG["alpha"], CFG["w"], CFG["Gamma"], CFG["dt"], seed=0, precision=precision,
                    stream=stream, traj_offset=rank * M, ws_route=route, noise_route=noise, integrator=integrator)
        g.run(M, warm)
        g.sync()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        g.run(M, steps)
        a1.record(stream)
        torch.cuda.synchronize()
        t_ms = a0.elapsed_time(a1) / steps
        g.profile(True)
        g.run(M, min(steps, 20))
        p = g.profile_read()
        g.close()
        return {"value": N * M * world / (t_ms * 1e-3), "ms_per_step": t_ms, "steps": steps,
                "kernel_ms_per_step": {k: v[0] / v[1] for k, v in p.items() if v[1]}}

    side = {}
    if not args.no_side:
        side["fft_route"] = side_run(CFG["precision"], "fft", min(K, 300), 3)
        side["fft_route"]["speedup_vs_dense"] = side["fft_route"]["value"] / value
        side["fft_route"]["roofline"] = fft_roofline(N, M, side["fft_route"]["kernel_ms_per_step"])
        # W.s by FFT and the pump noise from the same circulant embedding: no contraction left
        side["fft_route_circulant_noise"] = side_run(CFG["precision"], "fft", min(K, 300), 3, noise="circulant")
        side["fft_route_circulant_noise"]["speedup_vs_dense"] = side["fft_route_circulant_noise"]["value"] / value
        side["fft_route_circulant_noise"]["roofline"] = fft_roofline(
            N, M, side["fft_route_circulant_noise"]["kernel_ms_per_step"])
        # the dense route in the other tensor-core precisions (one-term BF16, TF32,
        # and the FP32-accurate TF32 split)
        for prec in ("bf16x3", "bf16", "tf32", "fp32", "bf16x2", "bf16l2", "bf16b"):
            if prec != CFG["precision"]:
                side["dense_" + prec] = side_run(prec, "dense", min(K, 300), 3)
                side["dense_" + prec]["speedup_vs_main"] = side["dense_" + prec]["value"] / value
        # the paper's semi-implicit midpoint integrator in place of Heun
        side["dense_midpoint"] = side_run(CFG["precision"], "dense", min(K, 300), 3, integrator="midpoint")
        side["dense_midpoint"]["speedup_vs_main"] = side["dense_midpoint"]["value"] / value
        side["fp64_gpu"] = side_run("fp64", "dense", 2, 1)
        side["fp64_gpu"]["mixed_speedup"] = value / side["fp64_gpu"]["value"]
    qualifier = None
    if not args.no_precision_check:
        others = tuple(p for p in ("bf16x3", "bf16x2", "bf16l2", "bf16b") if p != CFG["precision"])
        qualifier = precision_check(twa, stream, rank, (CFG["precision"],) + (() if args.no_side else others))
    clocks.stop()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, el, threads, steps_cpu = cpu_oracle_rate(N, REF_SAMPLE_M, 3, CFG)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d trajectories x %d sites x %d steps of the same workload (%.1f s); W, L set-up untimed"
                         % (REF_SAMPLE_M, N, steps_cpu, el)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if CFG["precision"].startswith("bf16") else CFG["precision"], "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "M_per_gpu": M, "alpha": CFG["alpha"], "w": CFG["w"],
                       "Gamma": CFG["Gamma"], "dt": CFG["dt"], "precision": CFG["precision"],
                       "parallelism": "trajectory shards, no data-path collective" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2: W and L BF16 hi+lo images 800 MB, state 0.9 GB"},
            "roofline": {"bound": "tensor", "kernel": kernel_name, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": "%s bf16_tflops_sustained" % peak_src,
                         "work": "algorithmic: 2 N^2 per column for W.s, 2 per nonzero of L for L.eta, "
                                 "counted once (no split-precision multiplier)",
                         "kernel_ms": d_ms, "kernel_ms_profile_pass": d_ms_prof,
                         "algorithmic_flops_per_launch": d_algo, "executed_flops_per_launch": d_exec,
                         "tensor_pipe_tflops": executed_tflops, "tensor_pipe_frac": executed_tflops / peak,
                         "frac_of_burst_peak": achieved / float(peaks.get("bf16_tflops", peak)),
                         "step_algorithmic_tflops": step_algo / (ms / K * 1e-3) / 1e12,
                         "step_algorithmic_frac": step_algo / (ms / K * 1e-3) / 1e12 / peak,
                         "kernel_ms_per_step_profile_pass": {k: v[0] / max(kp, 1) for k, v in prof.items() if v[1]},
                         "step_kernel_ms_profile_pass": step_kernel_ms,
                         "noise_overlapped": noise_overlapped,
                         "profile_pass_clocks": clocks.stats(c2, c3)},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
                    "note": "set_state_f32 from pinned host FP32 buffers (the mixed-precision state), K steps, "
                            "moments and observables to host",
                    "fp64_host_state": {"value": e2e64, "h2d_bytes_per_step": h2d64 / K}},
            "gpu_launches": launches_per_step_all * K,
            "clocks": clocks.stats(c0, c1),
            "sustained": sustained,
            "precision_check": qualifier,
            "observables": {k: obs[k] for k in ("sigma_z", "SpSm", "g2", "w_tilde", "stability", "nonfinite")},
        }
        line.update(side)
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the FFT-route, other-precision and FP64-GPU legs")
    ap.add_argument("--no-sustained", action="store_true", help="skip the seconds-long sustained leg")
    ap.add_argument("--no-precision-check", action="store_true",
                    help="skip the mixed-vs-FP64 comparison on a 128-trajectory subset")
    ap.add_argument("--sustained-steps", type=int, default=2500,
                    help="steps of the seconds-long sustained leg")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(env_int("LOCAL_RANK", 0))
            dist_mod.init_process_group("nccl")
        else:
            dist_mod.init_process_group("gloo")
        dist = dist_mod
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    else:
        rc = run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
