"""Precision and gradient studies on the GPU, through the C ABI.

    python -m paper_2608_10075_b300.studies precision [--M-ref 512] [--steps S]
    python -m paper_2608_10075_b300.studies gradients [--M 2048] [--steps S]
    python -m paper_2608_10075_b300.studies phase [--Ns 100] [--alphas 0.5 1 2] [--T 15]
    python -m paper_2608_10075_b300.studies linewidth [--N 500] [--alpha 1] [--wt 0.5]
    python -m paper_2608_10075_b300.studies scan [--T 1.0] [--small-route resident]
    python -m paper_2608_10075_b300.studies routes [--Ns 10000 20000 30000 60000] [--M 1024]
    python -m paper_2608_10075_b300.studies resident [--Ns 16 64 100 128] [--M 1024] [--steps 2000]

precision: N = 1024, alpha in {0.5, 1, 2}, w = N Gamma / 2, dt = 1e-4, T = 2,
window (1, 2]. The same trajectories (same seed and counters) run on the FP64
path and on the mixed paths (BF16, TF32, BF16X3, BF16X2, BF16L2, BF16B, FP32 from a TF32 split,
BF16X3 with the FFT pump field);
each observable is reported with its standard error and, per mixed path, the
paired difference to FP64 (mean over trajectories of the per-trajectory
difference, and its standard error), which isolates the arithmetic error from
the sampling noise.

phase: the phase-diagram workflow on the batched scan. For every (N, alpha) the
pump prefactor is set from a target w~ = w_max / (Gamma N) (main text, "Observables
and method"): one calibration batch at w = 1 gives each point's w_max, which is
linear in w, so w = w~ Gamma N / w_max(w = 1). By default the g2_min protocol of
the main text: ten equally spaced w~ in [1/10, 1] per (N, alpha), a preparation
time of 10 / Gamma and an average over the following 5 / Gamma, all points run as
one batch; each (N, alpha) reports g2(w~), <S+S->/N and the minimum of g2 with the
w~ where it falls (--spacing log and a wider range show the thermal side too).

gradients: N = 1024, alpha = 1, w = N Gamma / 4, dt = 1e-4, T = 2, window
(1, 2], checkpoints every 64 steps. twa_grad (BF16X3) gives d<S+S->/dw,
d<S+S->/dalpha and dg2/dalpha; central differences with common random numbers
(the same seed, delta = 1e-4) of the mixed forward run check them.

routes: the dense route and the Toeplitz/FFT route (Cholesky and circulant
noise draws) at N beyond the benchmark's 10^4, alpha = 1, w = N Gamma / 2,
dt = 2e-5, M trajectories: time per step (CUDA events around twa_run after a
warm-up) and spin-trajectory-steps per second, with the FFT route's circle
length and CTAs per trajectory (one CTA up to P = 28000, else a cluster).

resident: the small-N routes side by side -- the resident route on the tensor
cores (BF16X2, N <= 128), the resident route in FP32 SIMT, the dense route
(BF16X2) -- at alpha = 1, w = N Gamma / 2, dt = 0.05 / (Gamma N): time per step
of one call of `steps` steps (CUDA events) after a warm-up call.

Each study prints one JSON line per case.
"""
import argparse
import json
import math
import time

import numpy as np

from . import twa
from .configs import ADJOINT_N1024, MIXED_N1024

KEYS = ("Sz", "SpSm", "G2num", "g2")


def _linear_samples(means):
    """Per-trajectory samples of S^z, <S+S->, <S+S+S-S-> from window means."""
    Sz, A, A2, ASz, Sz2 = means.T
    return {"Sz": Sz, "SpSm": A + 0.5 * Sz, "G2num": A2 + 2 * ASz - Sz / 3 + 0.5 * Sz2 - 4.0 / 3.0 * A}


def _run(N, alpha, w, G, dt, steps, M, t0, precision, route="dense", noise="cholesky"):
    t = time.perf_counter()
    with twa.TWA(N, alpha, w, G, dt, seed=0, precision=precision, window_start=t0, ws_route=route,
                 noise_route=noise) as g:
        g.run(M, steps)
        obs = g.observables()
        means = g.moments()
    return obs, means, time.perf_counter() - t


def precision_study(args):
    c = MIXED_N1024
    N, w, G, dt = c["N"], c["w"], c["Gamma"], c["dt"]
    steps = args.steps or int(round(c["T"] / dt))
    t0 = steps * dt - c["window"]
    for alpha in (args.alphas or c["alphas"]):
        ref_obs, ref_means, ref_t = _run(N, alpha, w, G, dt, steps, args.M_ref, t0, "fp64")
        ref_s = _linear_samples(ref_means)
        line = {"study": "precision", "N": N, "alpha": alpha, "w": w, "dt": dt, "steps": steps,
                "M_ref": args.M_ref, "stability": ref_obs["stability"], "w_tilde": ref_obs["w_tilde"],
                "fp64": {k: [ref_obs[k], ref_obs[k + "_se"]] for k in KEYS}, "fp64_seconds": ref_t}
        # the circulant draw has the same noise law but other per-trajectory values,
        # so only its unpaired difference (diff_over_se) measures its error
        for name, prec, route, noise in [x for x in (("bf16", "bf16", "dense", "cholesky"),
                                         ("tf32", "tf32", "dense", "cholesky"),
                                         ("bf16x3", "bf16x3", "dense", "cholesky"),
                                         ("bf16x2", "bf16x2", "dense", "cholesky"),
                                         ("bf16l2", "bf16l2", "dense", "cholesky"),
                                         ("bf16b", "bf16b", "dense", "cholesky"),
                                         ("fp32", "fp32", "dense", "cholesky"),
                                         ("bf16x3_fft", "bf16x3", "fft", "cholesky"),
                                         ("fft_circulant_noise", "bf16x3", "fft", "circulant"))
                                         if not args.only or x[0] in args.only]:
            obs, means, secs = _run(N, alpha, w, G, dt, steps, args.M_ref, t0, prec, route, noise)
            s = _linear_samples(means)
            paired = {}
            for k in ("Sz", "SpSm", "G2num"):
                d = s[k] - ref_s[k]
                paired[k] = [float(d.mean()), float(d.std(ddof=1) / math.sqrt(len(d)))]
            line[name] = {"obs": {k: [obs[k], obs[k + "_se"]] for k in KEYS},
                          "diff_over_se": {k: abs(obs[k] - ref_obs[k]) / math.hypot(obs[k + "_se"], ref_obs[k + "_se"])
                                           for k in KEYS},
                          "paired_diff": paired, "seconds": secs}
        if args.M_full > args.M_ref:
            obs, _, secs = _run(N, alpha, w, G, dt, steps, args.M_full, t0, "bf16x3")
            line["bf16x3_full_M"] = {"M": args.M_full, "obs": {k: [obs[k], obs[k + "_se"]] for k in KEYS},
                                     "seconds": secs}
        print(json.dumps(line), flush=True)


def _observables(N, alpha, w, G, dt, steps, M, t0, precision="bf16x3"):
    with twa.TWA(N, alpha, w, G, dt, seed=0, precision=precision, window_start=t0) as g:
        g.run(M, steps)
        return g.observables()


def gradient_study(args):
    c = dict(ADJOINT_N1024)
    # other sizes (e.g. N = 10^4, w = N Gamma / 4, dt = 2e-5) on request
    for k in ("N", "w", "dt", "delta"):
        v = getattr(args, k, None)
        if v:
            c[k] = type(c[k])(v)
    N, alpha, w, G, dt = c["N"], c["alpha"], c["w"], c["Gamma"], c["dt"]
    steps = args.steps or int(round(c["T"] / dt))
    t0 = 0.5 * steps * dt            # window: the second half of the run
    M, d = args.M, c["delta"]
    prec = getattr(args, "precision", "bf16x3")
    out = {"study": "gradients", "N": N, "alpha": alpha, "w": w, "dt": dt, "steps": steps, "M": M,
           "checkpoint": c["checkpoint"], "delta": d, "precision": prec}
    for obj in ("SpSm", "g2"):
        t = time.perf_counter()
        with twa.TWA(N, alpha, w, G, dt, seed=0, precision=prec, window_start=t0) as g:
            r = g.grad(obj, M, steps, checkpoint=c["checkpoint"], want_alpha=True)
        out["adjoint_" + obj] = {**r, "seconds": time.perf_counter() - t}
    fd = {}
    t = time.perf_counter()
    for key, (a2, w2, h) in {"w": (alpha, None, w * d), "alpha": (None, w, d)}.items():
        vals = []
        for s in (+1, -1):
            aa = alpha + s * d if key == "alpha" else alpha
            ww = w * (1 + s * d) if key == "w" else w
            vals.append(_observables(N, aa, ww, G, dt, steps, M, t0, prec))
        for obj in ("SpSm", "g2"):
            fd["d%s_d%s" % (obj, key)] = (vals[0][obj] - vals[1][obj]) / (2 * h)
    out["crn_fd"] = fd
    out["crn_fd_seconds"] = time.perf_counter() - t
    # The same differences through twa_grad's own forward run (the run the adjoint
    # differentiates), from the forward means it returns. The tensor-core images
    # hold W / w and L / sqrt(w), so a step in w changes only two FP32 factors; a
    # step in alpha changes the images, whose BF16 hi/lo pairs represent w_ij to
    # ~2^-17 relative (rounding of that size enters the alpha quotient).
    for dd in (d, 10 * d):
        fdt = {}
        for key, h in (("w", w * dd), ("alpha", dd)):
            vals = []
            for s in (+1, -1):
                aa = alpha + s * dd if key == "alpha" else alpha
                ww = w * (1 + s * dd) if key == "w" else w
                with twa.TWA(N, aa, ww, G, dt, seed=0, precision=prec, window_start=t0) as g:
                    mu = g.grad("SpSm", M, steps, checkpoint=c["checkpoint"], want_alpha=False)["mu"]
                Sz, A, A2, ASz, Sz2 = mu
                spsm = A + 0.5 * Sz
                vals.append({"SpSm": spsm, "g2": (A2 + 2 * ASz - Sz / 3 + 0.5 * Sz2 - 4.0 / 3.0 * A) / spsm ** 2})
            for obj in ("SpSm", "g2"):
                fdt["d%s_d%s" % (obj, key)] = (vals[0][obj] - vals[1][obj]) / (2 * h)
        tag = "delta_%g" % dd
        out["crn_fd_same_forward_" + tag] = fdt
        out["rel_diff_same_forward_" + tag] = {
            "dSpSm_dw": abs(out["adjoint_SpSm"]["dJ_dw"] - fdt["dSpSm_dw"]) / abs(fdt["dSpSm_dw"]),
            "dSpSm_dalpha": abs(out["adjoint_SpSm"]["dJ_dalpha"] - fdt["dSpSm_dalpha"]) / abs(fdt["dSpSm_dalpha"]),
            "dg2_dalpha": abs(out["adjoint_g2"]["dJ_dalpha"] - fdt["dg2_dalpha"]) / abs(fdt["dg2_dalpha"]),
        }
    out["rel_diff"] = {
        "dSpSm_dw": abs(out["adjoint_SpSm"]["dJ_dw"] - fd["dSpSm_dw"]) / abs(fd["dSpSm_dw"]),
        "dSpSm_dalpha": abs(out["adjoint_SpSm"]["dJ_dalpha"] - fd["dSpSm_dalpha"]) / abs(fd["dSpSm_dalpha"]),
        "dg2_dalpha": abs(out["adjoint_g2"]["dJ_dalpha"] - fd["dg2_dalpha"]) / abs(fd["dg2_dalpha"]),
    }
    print(json.dumps(out), flush=True)


def scan_study(args):
    """The 96-point scan (N in {100, 300, 1000, 3000}, six alpha, four w, M = 512,
    dt = 0.02 / (N Gamma)) over the horizon T (the workload's is 1 / Gamma).
    Throughput counts N M steps per point. With --small-route resident the
    points with N <= --resident-max-n run as one resident batch (each CTA
    integrating its trajectories for all steps in one launch; on the tensor cores
    in the scan's precision when that is BF16X2 and N <= 128, else FP32) on a
    stream of their own, concurrently with the dense batch of the larger points."""
    import threading

    from .configs import SCAN_POINTS, scan_points
    pts = scan_points()
    for p in pts:
        p["steps"] = max(1, int(round(args.T / p["dt"])))
        p["window_start"] = 0.5 * p["steps"] * p["dt"]
    M = SCAN_POINTS["M"]
    units = sum(p["N"] * M * p["steps"] for p in pts)
    groups = [("dense", args.precision, "dense", pts)]
    if args.small_route == "resident":
        # the resident route is faster only where the dense one is launch-bound
        small = [p for p in pts if p["N"] <= args.resident_max_n]
        res_prec = args.precision if args.precision == "bf16x2" and args.resident_max_n <= 128 else "fp32"
        groups = [("dense", args.precision, "dense", [p for p in pts if p["N"] > args.resident_max_n]),
                  ("resident", res_prec, "resident", small)]
    results, times = {}, {}

    def run_group(name, prec, route, gp, stream):
        t0 = time.perf_counter()
        results[name] = twa.batch_run(gp, M, seed=0, precision=prec, ws_route=route, stream=stream)
        times[name] = time.perf_counter() - t0

    streams = [None] * len(groups)
    if len(groups) > 1:
        import torch
        streams = [torch.cuda.Stream() for _ in groups]
    t = time.perf_counter()
    th = [threading.Thread(target=run_group, args=(*g, s)) for g, s in zip(groups, streams)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    t_batch = time.perf_counter() - t
    res = []
    for name, _, _, gp in groups:
        res += results[name][0]
    line = {"study": "scan", "points": len(pts), "M": M, "T": args.T, "precision": args.precision,
            "small_route": args.small_route, "spin_traj_steps": units, "batched_seconds": t_batch,
            "batched_rate": units / t_batch,
            "groups": {name: {"points": len(gp), "precision": prec, "route": route, "seconds": times[name],
                              "spin_traj_steps": sum(p["N"] * M * p["steps"] for p in gp),
                              "tiles": list(results[name][1])} for name, prec, route, gp in groups},
            "nonfinite": sum(r["nonfinite"] for r in res)}
    if args.sequential:
        t = time.perf_counter()
        for p in pts:
            with twa.TWA(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed=0, precision=args.precision,
                         window_start=p["window_start"]) as g:
                g.run(M, p["steps"])
                g.sync()
        t_seq = time.perf_counter() - t
        line.update(sequential_seconds=t_seq, sequential_rate=units / t_seq, batch_speedup=t_seq / t_batch)
    order = [p for _, _, _, gp in groups for p in gp]
    line["sample"] = [{k: res[i][k] for k in ("sigma_z", "SpSm", "g2", "w_tilde")} | {"N": order[i]["N"],
                      "alpha": order[i]["alpha"], "w": order[i]["w"]} for i in range(0, len(order), 23)]
    print(json.dumps(line), flush=True)


def phase_grid(Ns, alphas, wts, T, window, dt_scale, w_max_unit):
    """Points of the phase scan: w = w~ Gamma N / w_max(w = 1) for each target w~,
    dt = dt_scale / (Gamma N), T / dt steps, averaging over the last `window`."""
    pts = []
    for N in Ns:
        dt = dt_scale / N
        steps = max(1, int(round(T / dt)))
        for a in alphas:
            for wt in wts:
                pts.append(dict(N=N, alpha=a, w=wt * N / w_max_unit[(N, a)], Gamma=1.0, dt=dt, steps=steps,
                                window_start=max(0.0, steps * dt - window), wt=wt))
    return pts


def phase_lines(pts, res):
    """One summary per (N, alpha): the g2 and <S+S->/N curves over w~ and the
    minimum of g2."""
    out = {}
    for p, r in zip(pts, res):
        d = out.setdefault((p["N"], p["alpha"]), {"study": "phase", "N": p["N"], "alpha": p["alpha"], "wt": [],
                                                  "wt_lib": [], "g2": [], "g2_se": [], "SpSm_over_N": [],
                                                  "sigma_z": [], "stability": []})
        d["wt"].append(p["wt"])
        d["wt_lib"].append(r["w_tilde"])
        d["g2"].append(r["g2"])
        d["g2_se"].append(r["g2_se"])
        d["SpSm_over_N"].append(r["SpSm"] / p["N"])
        d["sigma_z"].append(r["sigma_z"])
        d["stability"].append(r["stability"])
    for d in out.values():
        k = min(range(len(d["g2"])), key=lambda j: d["g2"][j])
        d["g2_min"], d["g2_min_se"], d["wt_at_min"] = d["g2"][k], d["g2_se"][k], d["wt"][k]
        # superradiant: <S+S-> above N, the independent-emitter value
        d["superradiant_wt"] = [wt for wt, x in zip(d["wt"], d["SpSm_over_N"]) if x > 1.0]
    return list(out.values())


def phase_study(args, runner=None):
    runner = runner or twa.batch_run
    Ns, alphas = args.Ns, args.alphas
    if args.spacing == "log":
        wts = list(np.logspace(math.log10(args.wt_min), math.log10(args.wt_max), args.n_wt))
    else:
        wts = list(np.linspace(args.wt_min, args.wt_max, args.n_wt))
    cal = [dict(N=N, alpha=a, w=1.0, Gamma=1.0, dt=args.dt_scale / N, steps=1, window_start=0.0)
           for N in Ns for a in alphas]
    route = getattr(args, "route", "dense")
    res, _ = runner(cal, 8, seed=0, precision=args.precision, ws_route=route)
    w_max_unit = {(p["N"], p["alpha"]): r["w_max"] for p, r in zip(cal, res)}
    pts = phase_grid(Ns, alphas, wts, args.T, args.window, args.dt_scale, w_max_unit)
    t = time.perf_counter()
    res, tiles = runner([{k: v for k, v in p.items() if k != "wt"} for p in pts], args.M, seed=0,
                        precision=args.precision, ws_route=route)
    secs = time.perf_counter() - t
    for d in phase_lines(pts, res):
        d.update(M=args.M, T=args.T, window=args.window, dt=args.dt_scale / d["N"], precision=args.precision,
                 route=route, batch_seconds=secs, points_in_batch=len(pts), tiles=list(tiles))
        print(json.dumps(d), flush=True)


def linewidth_study(args):
    """The linewidth of the main text ("Observables and method") at one phase point:
    w from the target w~ (one calibration context: w_max is linear in w), a
    preparation of T_prep, then the two-time correlation over T_meas from the
    three trajectory copies (twa_correlation), its spectrum and FWHM."""
    N, a, G = args.N, args.alpha, 1.0
    dt = args.dt_scale / (G * N)
    with twa.TWA(N, a, 1.0, G, dt, seed=0, precision=args.precision) as g:
        g.run(8, 1)
        wmax1 = g.observables()["w_max"]
    w = args.wt * G * N / wmax1
    prep = int(round(args.T_prep / dt))
    lags = int(round(args.T_meas / dt))
    stride = max(1, lags // args.n_lags)
    t = time.perf_counter()
    with twa.TWA(N, a, w, G, dt, seed=0, precision=args.precision, window_start=prep * dt) as g:
        r = g.correlation(args.M, prep, lags, stride, args.eps, args.n_omega, args.omega_max)
    secs = time.perf_counter() - t
    out = {"study": "linewidth", "N": N, "alpha": a, "w_tilde": args.wt, "w": w, "dt": dt, "M": args.M,
           "prep_steps": prep, "lag_steps": lags, "lag_stride": stride, "eps": args.eps, "precision": args.precision,
           "fwhm": r["fwhm"], "fwhm_se": r["fwhm_se"], "omega_peak": r["omega_peak"], "S_peak": r["S_peak"],
           "spsm_tau0": r["spsm_tau0"], "C_over_C0": [float(abs(c) / abs(r["C"][0])) for c in r["C"][::max(1, len(r["C"]) // 20)]],
           "seconds": secs}
    print(json.dumps(out), flush=True)


def routes_study(args):
    import torch
    for N in args.Ns:
        w, dt = N / 2.0, 2e-5
        for route, noise in (("dense", "cholesky"), ("fft", "cholesky"), ("fft", "circulant")):
            t = time.perf_counter()
            with twa.TWA(N, 1.0, w, 1.0, dt, seed=0, precision=args.precision, ws_route=route,
                         noise_route=noise) as g:
                setup = time.perf_counter() - t
                g.run(args.M, args.warmup)
                g.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.run(args.M, args.steps)
                e1.record()
                g.sync()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                ob = g.observables()
            print(json.dumps({"study": "routes", "N": N, "route": route, "noise": noise, "M": args.M,
                              "precision": args.precision, "ms_per_step": ms,
                              "spin_traj_steps_per_s": N * args.M / (ms * 1e-3), "setup_s": setup,
                              "fft_length": ob["fft_length"], "fft_ctas": ob["fft_ctas"],
                              "sigma_z": ob["sigma_z"], "nonfinite": ob["nonfinite"]}), flush=True)


def resident_study(args):
    import torch
    for N in args.Ns:
        for route, prec in (("resident", "bf16x2"), ("resident", "fp32"), ("dense", "bf16x2")):
            if route == "resident" and prec == "bf16x2" and N > 128:
                continue
            with twa.TWA(N, 1.0, N / 2.0, 1.0, 0.05 / N, seed=0, precision=prec, ws_route=route,
                         window_start=0.0) as g:
                g.run(args.M, 10)
                g.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.run(args.M, args.steps)
                e1.record()
                g.sync()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
            print(json.dumps({"study": "resident", "N": N, "route": route, "precision": prec, "M": args.M,
                              "steps": args.steps, "us_per_step": 1e3 * ms / args.steps,
                              "spin_traj_steps_per_s": N * args.M * args.steps / (ms * 1e-3)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    s = sub.add_parser("scan")
    s.add_argument("--T", type=float, default=0.02, help="horizon in 1/Gamma (the full scan is T = 1)")
    s.add_argument("--precision", default="bf16x3")
    s.add_argument("--sequential", action="store_true", help="also run the points one by one")
    s.add_argument("--small-route", choices=["dense", "resident"], default="dense",
                   help="route of the small points")
    s.add_argument("--resident-max-n", type=int, default=128,
                   help="largest N run on the resident route (<= 512)")
    p = sub.add_parser("precision")
    p.add_argument("--M-ref", type=int, default=512)
    p.add_argument("--M-full", type=int, default=MIXED_N1024["M"])
    p.add_argument("--steps", type=int, default=0)
    p.add_argument("--alphas", type=float, nargs="*", default=None, help="a subset of the study's exponents")
    p.add_argument("--only", nargs="*", default=None,
                   help="a subset of the mixed cases (bf16 tf32 bf16x3 bf16x2 bf16l2 bf16b fp32 bf16x3_fft fft_circulant_noise)")
    f = sub.add_parser("phase")
    f.add_argument("--Ns", type=int, nargs="+", default=[100])
    f.add_argument("--alphas", type=float, nargs="+", default=[0.5, 1.0, 2.0])
    f.add_argument("--n-wt", type=int, default=10)
    f.add_argument("--wt-min", type=float, default=0.1)
    f.add_argument("--wt-max", type=float, default=1.0)
    f.add_argument("--spacing", choices=["linear", "log"], default="linear")
    f.add_argument("--M", type=int, default=256)
    f.add_argument("--T", type=float, default=15.0, help="horizon in 1/Gamma")
    f.add_argument("--window", type=float, default=5.0, help="averaging window at the end of the run, 1/Gamma")
    f.add_argument("--dt-scale", type=float, default=0.02, help="dt = dt_scale / (Gamma N)")
    f.add_argument("--precision", default="bf16x3")
    f.add_argument("--route", choices=["dense", "resident"], default="dense",
                   help="resident: every point's run in one launch (FP32 for N <= 512, BF16X2 for N <= 128)")
    lw = sub.add_parser("linewidth")
    lw.add_argument("--N", type=int, default=500)
    lw.add_argument("--alpha", type=float, default=1.0)
    lw.add_argument("--wt", type=float, default=0.5, help="target w~ = w_max / (Gamma N)")
    lw.add_argument("--M", type=int, default=1024)
    lw.add_argument("--T-prep", type=float, default=10.0)
    lw.add_argument("--T-meas", type=float, default=5.0)
    lw.add_argument("--dt-scale", type=float, default=0.05)
    lw.add_argument("--n-lags", type=int, default=1000)
    lw.add_argument("--eps", type=float, default=1e-2)
    lw.add_argument("--n-omega", type=int, default=801)
    lw.add_argument("--omega-max", type=float, default=20.0)
    lw.add_argument("--precision", default="bf16x2")
    q = sub.add_parser("gradients")
    q.add_argument("--M", type=int, default=ADJOINT_N1024["M"])
    q.add_argument("--steps", type=int, default=0)
    q.add_argument("--N", type=int, default=0, help="sites (default: the adjoint workload's 1024)")
    q.add_argument("--w", type=float, default=0.0, help="pump prefactor (default N Gamma / 4 of the workload)")
    q.add_argument("--dt", type=float, default=0.0)
    q.add_argument("--delta", type=float, default=0.0, help="finite-difference step (default 1e-4)")
    q.add_argument("--precision", default="bf16x3", help="precision of the adjoint and of the differences")
    r = sub.add_parser("routes")
    r.add_argument("--Ns", type=int, nargs="+", default=[10000, 20000, 30000, 60000])
    r.add_argument("--M", type=int, default=1024)
    r.add_argument("--steps", type=int, default=20)
    r.add_argument("--warmup", type=int, default=3)
    r.add_argument("--precision", default="bf16x2")
    rs = sub.add_parser("resident")
    rs.add_argument("--Ns", type=int, nargs="+", default=[16, 64, 100, 128])
    rs.add_argument("--M", type=int, default=1024)
    rs.add_argument("--steps", type=int, default=2000)
    a = ap.parse_args()
    if a.cmd == "routes":
        routes_study(a)
    elif a.cmd == "resident":
        resident_study(a)
    elif a.cmd == "precision":
        precision_study(a)
    elif a.cmd == "phase":
        phase_study(a)
    elif a.cmd == "scan":
        scan_study(a)
    elif a.cmd == "linewidth":
        linewidth_study(a)
    else:
        gradient_study(a)


if __name__ == "__main__":
    main()
