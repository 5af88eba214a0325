#!/usr/bin/env python
"""Benchmark of the KP-sum + split Bregman deblurring hot path on GB300.

One step = one batch of independent deblur requests through the whole path:
kp_build (TSVD of R(A) by EGKB in FP32 with automatic rank, then Terms(A_k)) for every
request, then split Bregman (isotropic TV, 100 outer steps, CGLS <= 100 inner steps) for
all of them in one batched solve.  Workload: n = 128 images, 31 x 31 two-Gaussian
mixture PSFs, reflexive boundary, noise 1 % and 5 % (alternating), mu = 1, lambda = 0.1,
beta = lambda^2/2 (gamma = 2).  Seeded synthetic inputs (paper_2410_00233_gb300.inputs)
stand in for the paper's IR Tools images and PSFs.

value: deblurs/s of the mixed path (KP GEMMs in the selected precision, FP64 vectors),
inputs resident in HBM, L2 flushed between timed steps.  e2e: the same through the
host-pointer C ABI (PSFs and b uploaded from pinned memory, x read back, every step).
plain: FP32 EGKB + FP64 split Bregman, one request at a time (the paper's arithmetic).

--impl reference times the CPU oracle (test infrastructure) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_IMG = 128
PSF_S = 31
# DRAM bytes (read + write) per KP-apply launch with all 256 problems of the headline batch
# active, by (precision, apply variant), from ncu captures on this workload (one part, the
# first CGLS applies): profiles/tc_apply_dram_medium_batch256.txt.
DRAM_BYTES_256_ACTIVE = {(3, 3): 252.3e6, (3, 1): 257.1e6, (3, 2): 258.3e6, (3, 0): 316.2e6}
OUTER = 100
MU, LAM = 1.0, 0.1
WORKLOAD = ("n=128 images, 31x31 two-Gaussian-mixture PSF, reflexive boundary, EGKB(FP32) "
            "automatic rank (tau=1e-3, cap 30), isotropic split Bregman 100 outer, noise 1%/5%")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--prec", default="auto", choices=["auto", "fp64", "fp32", "tf32x3", "tf32x2", "bf16x3", "bf16x2"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--outer", type=int, default=OUTER, help="split Bregman outer steps (profiling runs only)")
    ap.add_argument("--serve", action="store_true",
                    help="serving run: Poisson arrivals into the continuous-batching server")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: arrivals per second")
    ap.add_argument("--count", type=int, default=64, help="serving: requests")
    ap.add_argument("--sizes", default="128,256", help="serving: image sizes drawn uniformly")
    ap.add_argument("--n", type=int, default=1024, help="single: image side")
    ap.add_argument("--workload", default="medium",
                    choices=["medium", "batched96", "sweep", "direct", "tsvd", "dense_tsvd", "single"],
                    help="medium: the headline batch; batched96: 96 uneven problems (n 64..384) in "
                         "one batched launch; sweep: 100 lambda values on one set of KP factors; "
                         "direct: split Bregman with the explicit A vs the KP sum on one request; "
                         "tsvd: the TSVD in single vs double precision, full vs one-sided reorthogonalisation; "
                         "dense_tsvd: the TSVD of a general explicit operator (kp_build_dense); "
                         "single: one serving-workload request of side --n alone (latency)")
    ap.add_argument("--profile", action="store_true",
                    help="profiling run: the timed steps only (no replay, e2e, plain or CPU legs), "
                         "with the library's host-driven loop (ncu cannot profile kernels inside "
                         "graphs with conditional nodes)")
    ap.add_argument("--sub-batches", type=int, default=0,
                    help="concurrent parts of the batched solve (0: the library's default)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving block of the default run")
    ap.add_argument("--no-large", action="store_true", help="skip the n = 512 block of the default run")
    ap.add_argument("--serve-count", type=int, default=12, help="serving block: requests per arrival rate")
    ap.add_argument("--cpu-worker", type=float, default=0.0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-samples", type=int, default=1, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm): a bounded sample in a single-threaded process
# ---------------------------------------------------------------------------------------

def cpu_worker(seconds: float, samples: int = 1) -> list:
    """`samples` bounded samples of one medium request on the CPU oracle: the full EGKB build,
    then as many of the 100 split Bregman outer steps as fit in `seconds` (at least one),
    extrapolated to the full solve.  One outer step is probed first to size the sample."""
    from oracle import kpsb_oracle as O
    from paper_2410_00233_gb300 import inputs as I

    pr = I.problem_medium(0)
    b_true = O.blur(pr.psf, pr.x_true, pr.bc)
    b = b_true + I.noise_vector(b_true, pr.eta, pr.zeta)
    probe = None
    out = []
    for _ in range(samples):
        t0 = time.perf_counter()
        Kop, ts = O.kp_build(pr.psf, pr.n, pr.bc, pr.k, pr.p, "egkb", tau=pr.tau, start=pr.start)
        t_build = time.perf_counter() - t0
        A = lambda X: O.kp_apply(Kop, X)  # noqa: E731
        AT = lambda Y: O.kp_apply_t(Kop, Y)  # noqa: E731
        if probe is None:
            t1 = time.perf_counter()
            O.split_bregman(A, AT, b, MU, LAM, LAM * LAM / 2, True, 1)
            probe = time.perf_counter() - t1
        done = int(min(OUTER, max(1, (seconds - t_build) / max(probe, 1e-3))))
        t1 = time.perf_counter()
        O.split_bregman(A, AT, b, MU, LAM, LAM * LAM / 2, True, done)
        t_outer = (time.perf_counter() - t1) / done
        total = t_build + t_outer * OUTER
        out.append(dict(value=1.0 / total, wall_s=t_build + t_outer * done, t_build=t_build, t_outer=t_outer,
                        outer_timed=done, k=ts.k,
                        sample=(f"1 request (n=128): full EGKB(FP64 oracle, k={ts.k}) + the first {done} of {OUTER} "
                                f"split Bregman outer steps (CGLS to RC<1e-4), extrapolated to the full solve")))
    return out


def host_cpu() -> dict:
    """The host's CPU model and logical core count (reported beside the CPU baseline)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    model = line.split(":", 1)[1].strip()
                    if low.startswith("model name"):
                        break
    except OSError:
        pass
    import platform

    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def run_cpu_baseline(seconds: float, samples: int = 1) -> list:
    """Runs cpu_worker in a fresh single-threaded process (no GPU visible)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", str(seconds),
                        "--cpu-samples", str(samples)],
                       capture_output=True, text=True, env=env, timeout=60 + 3 * seconds * samples + 120)
    if r.returncode != 0:
        raise RuntimeError("cpu worker failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    for d in out:
        d["cores"] = 1
    return out


def reference_arm(args):
    """The CPU oracle on the headline workload: each step is one bounded sample (the full
    EGKB build and the first outer steps that fit in about 6 s, extrapolated to the full
    solve); value = mean extrapolated deblurs/s over the timed steps, ms_per_step = mean
    measured wall time of a sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = run_cpu_baseline(6.0, args.warmup + args.steps)[args.warmup:]
    v = statistics.mean(d["value"] for d in res)
    wall = statistics.mean(d["wall_s"] for d in res)
    host = host_cpu()
    line = {
        "impl": "reference", "metric": "deblurs/sec + p50/p99 latency, mixed-precision vs plain path, equal ISNR",
        "value": v, "unit": "deblurs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": 1, "parallelism": "host, 1 thread",
                   "step": "one bounded sample: full EGKB build + the first outer steps within ~6 s, "
                           "extrapolated to 100 outer steps (value); ms_per_step is the sample's wall time"},
        "cpu_baseline": {"value": v, "unit": "deblurs/s", "cores": 1, "kind": "oracle", "sample": res[-1]["sample"],
                         **host},
        "e2e": {"value": v, "unit": "deblurs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        return parse_clocks(out)


def parse_clocks(out: str) -> dict:
    """Median SM clock, maximum SM clock and the throttle reasons seen in ClockSampler.Q's CSV
    rows (noheader, nounits); rows that do not parse are skipped."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
            "samples": len(sm)}


def make_inputs(K, I, torch, count: int, first: int, dev):
    """Requests first..first+count-1: PSF (host), x_true, b on the device (exact blur on the
    GPU, noise scaled on the host as in the paper's experiments)."""
    import numpy as np

    reqs = []
    for i in range(first, first + count):
        pr = I.problem_medium(i)
        psf_d = torch.from_numpy(np.asfortranarray(pr.psf).reshape(-1, order="F").copy()).to(dev)
        x_d = torch.from_numpy(pr.x_true.reshape(-1, order="F").copy()).to(dev)
        bt_d = torch.empty_like(x_d)
        K.kp_blur_dev(psf_d.data_ptr(), PSF_S, PSF_S, N_IMG, pr.bc, x_d.data_ptr(), bt_d.data_ptr())
        torch.cuda.synchronize()
        b_true = bt_d.cpu().numpy().reshape(N_IMG, N_IMG, order="F")
        b = b_true + I.noise_vector(b_true, pr.eta, pr.zeta)
        b_d = torch.from_numpy(b.reshape(-1, order="F").copy()).to(dev)
        reqs.append(dict(pr=pr, b=b, b_d=b_d, x_d=torch.zeros_like(b_d)))
    return reqs


def run_step(K, reqs, prec, outer=OUTER, sub_batches=0):
    """The whole hot path for one batch: kp_build for all, one batched split Bregman."""
    probs = [dict(psf=r["pr"].psf, n=N_IMG, bc=r["pr"].bc, rank_or_tol=r["pr"].tau, method=K.EGKB,
                  p=r["pr"].p, seed=r["pr"].seed) for r in reqs]
    kps = K.kp_build_batched(probs)
    jobs = [dict(kp=kp, b=r["b_d"].data_ptr(), x=r["x_d"].data_ptr(), mu=MU, lam=LAM, tv=K.ISO, iters=outer)
            for kp, r in zip(kps, reqs)]
    stats = K.sb_solve_batched(jobs, on_device=True, prec=prec, sub_batches=sub_batches)
    return kps, stats


# ---------------------------------------------------------------------------------------
# Serving (continuous batching): Poisson arrivals, 30 % PSF reuse, mixed sizes
# ---------------------------------------------------------------------------------------

def serve_main(args):
    import numpy as np
    import torch

    from paper_2410_00233_gb300 import inputs as I
    from paper_2410_00233_gb300 import kpsb as K

    torch.cuda.set_device(0)
    K.lib()
    precs = {"fp64": K.P_FP64, "fp32": K.P_FP32, "tf32x3": K.P_TF32X3, "tf32x2": K.P_TF32X2,
             "bf16x3": K.P_BF16X3, "bf16x2": K.P_BF16X2}
    prec = precs[args.prec if args.prec != "auto" else "tf32x2"]
    sizes = [int(x) for x in args.sizes.split(",")]
    g = I.rng(5000)
    pool = []  # (psf, key) of earlier requests
    reqs = []
    for i in range(args.count):
        n = sizes[int(g.integers(len(sizes)))]
        reuse = [p for p in pool if p[2] == n]
        if reuse and g.uniform() < 0.3:
            psf, key, _ = reuse[int(g.integers(len(reuse)))]
        else:
            psf = I.psf_turbulence(31, g) if g.uniform() < 0.5 else I.psf_gaussian_mixture(31, g)
            key = 90000 + i
            pool.append((psf, key, n))
        xt = I.image_piecewise_constant(n, g)
        eta = float(g.uniform(0.01, 0.05))
        reqs.append(dict(n=n, psf=psf, key=key, xt=xt, eta=eta, zeta=I.gaussian((n, n), g),
                         tv=K.ISO if g.uniform() < 0.5 else K.ANISO))
    # blurred data through the library's exact blur (outside the timed region)
    for r in reqs:
        n = r["n"]
        psf_d = torch.from_numpy(np.asfortranarray(r["psf"]).reshape(-1, order="F").copy()).cuda()
        x_d = torch.from_numpy(r["xt"].reshape(-1, order="F").copy()).cuda()
        bt_d = torch.empty_like(x_d)
        K.kp_blur_dev(psf_d.data_ptr(), 31, 31, n, K.BC_REFLEXIVE, x_d.data_ptr(), bt_d.data_ptr())
        torch.cuda.synchronize()
        bt = bt_d.cpu().numpy().reshape(n, n, order="F")
        r["b"] = bt + I.noise_vector(bt, r["eta"], r["zeta"])
    arrivals = np.cumsum(g.exponential(1.0 / args.rate, size=args.count))
    srv = K.Server(budget_bytes=64 << 30, max_active=256, round_steps=5)
    launches0 = K.kpsb_kernel_launches()
    t0 = time.perf_counter()
    ids = []
    for r, ta in zip(reqs, arrivals):
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(r["psf"], r["n"], K.BC_REFLEXIVE, 20, r["b"], MU, LAM, r["tv"], OUTER,
                              prec=prec, psf_key=r["key"]))
    lats, isnrs = [], []
    for r, rid in zip(reqs, ids):
        x, st, lat = srv.poll(rid, timeout_us=-1)
        lats.append(lat)
        isnrs.append(20 * math.log10(np.linalg.norm(r["b"] - r["xt"]) / np.linalg.norm(x - r["xt"])))
    t_all = time.perf_counter() - t0
    sst = srv.stats()
    srv.close()
    lat = sorted(lats)
    out = {"metric": "serving deblurs/sec + p50/p99 latency (continuous batching)", "value": args.count / t_all,
           "unit": "deblurs/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "config": {"workload": f"Poisson arrivals {args.rate}/s, {args.count} requests, n in {sizes}, "
                                  "31x31 turbulence/mixture PSFs, 30% PSF reuse, noise U[1%,5%], k=20, "
                                  "iso/aniso 50/50, 100 outer", "kp_gemm": args.prec},
           "p50_s": lat[len(lat) // 2], "p99_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
           "makespan_s": t_all, "isnr_db_mean": statistics.mean(isnrs), "server": sst,
           "gpu_launches": K.kpsb_kernel_launches() - launches0}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------------------
# Blocks of the default run: serving (Poisson arrivals, mixed sizes) and the n = 512 case
# ---------------------------------------------------------------------------------------

SERVE_SIZES = (128, 256, 512, 1024)
SERVE_RATES = (10.0, 50.0, 500.0)

# Arithmetic of a split mode's KP apply: bytes per element of a factor-table plane and of an
# iterate plane, table planes, tensor products per useful product.
SPLIT_MODES = {"tf32x2": (4, 1, 2), "tf32x3": (4, 2, 3), "bf16x3": (2, 2, 3), "bf16x2": (2, 1, 2)}


def apply_roofline(mode: str, n: int, problem_applies: float, sum_kn3: float, flops: float, seconds: float,
                   tensor_peak_tflops: float, hbm_peak_gbs: float) -> dict:
    """Which ceiling binds a batch of KP applies, and how close they came.  Per problem and
    apply the kernel must read the factor tables (two n x n tables per term, in `fpl` planes),
    the split iterate (two planes) and write the FP32 result; its useful work is 4 k n^3 flops
    (Sec. 4.2).  Below the ridge (the mode's useful tensor peak, the dtype's peak over its
    products per useful product, divided by HBM bandwidth) the apply is HBM-bound."""
    es, fpl, prods = SPLIT_MODES[mode]
    nn = float(n) * n
    sum_k = sum_kn3 / float(n) ** 3
    nbytes = sum_k * 2 * nn * es * fpl + problem_applies * (2 * nn * es + 4 * nn)
    intensity = flops / nbytes
    ridge = (tensor_peak_tflops / prods) * 1e12 / (hbm_peak_gbs * 1e9)
    return {"bytes": nbytes, "achieved_gbs": nbytes / seconds / 1e9, "intensity": intensity, "ridge": ridge,
            "bound": "hbm" if intensity < ridge else "tensor"}



def _isnr(x, b, xt):
    import numpy as np

    return 20 * math.log10(np.linalg.norm(b - xt) / np.linalg.norm(x - xt))


def _pct(vals, q):
    v = sorted(vals)
    return v[min(len(v) - 1, int(q * len(v)))]


def serving_trace(K, I, torch, seed: int, count: int, rate: float, sizes=SERVE_SIZES):
    """Requests of the serving workload: n uniform in `sizes`, a 31 x 31 turbulence-like or
    two-Gaussian-mixture PSF (30 % of requests reuse an earlier PSF of the same size, a KP
    cache hit), noise U[1 %, 5 %], iso/aniso 50/50, reflexive boundary; Poisson arrival times.
    Blurred data comes from the library's exact blur (outside any timed region)."""
    import numpy as np

    g = I.rng(seed)
    pool, reqs = [], []
    for i in range(count):
        n = sizes[int(g.integers(len(sizes)))]
        reuse = [p for p in pool if p[2] == n]
        if reuse and g.uniform() < 0.3:
            psf, key, _ = reuse[int(g.integers(len(reuse)))]
        else:
            psf = I.psf_turbulence(31, g) if g.uniform() < 0.5 else I.psf_gaussian_mixture(31, g)
            key = seed * 1000 + i + 1
            pool.append((psf, key, n))
        xt = I.image_piecewise_constant(n, g)
        eta = float(g.uniform(0.01, 0.05))
        reqs.append(dict(n=n, psf=psf, key=key, xt=xt, eta=eta, zeta=I.gaussian((n, n), g),
                         tv=K.ISO if g.uniform() < 0.5 else K.ANISO))
    for r in reqs:
        n = r["n"]
        psf_d = torch.from_numpy(np.asfortranarray(r["psf"]).reshape(-1, order="F").copy()).cuda()
        x_d = torch.from_numpy(r["xt"].reshape(-1, order="F").copy()).cuda()
        bt_d = torch.empty_like(x_d)
        K.kp_blur_dev(psf_d.data_ptr(), 31, 31, n, K.BC_REFLEXIVE, x_d.data_ptr(), bt_d.data_ptr())
        torch.cuda.synchronize()
        bt = bt_d.cpu().numpy().reshape(n, n, order="F")
        r["b"] = bt + I.noise_vector(bt, r["eta"], r["zeta"])
    arrivals = np.cumsum(g.exponential(1.0 / rate, size=count))
    return reqs, arrivals


def serve_trace_run(K, reqs, arrivals, prec, round_steps=5):
    """Feeds a trace to a fresh continuous-batching server at its arrival times; returns the
    per-request results, latencies (submit to result) and the makespan."""
    srv = K.Server(budget_bytes=64 << 30, max_active=256, round_steps=round_steps)
    launches0 = K.kpsb_kernel_launches()
    t0 = time.perf_counter()
    ids = []
    for r, ta in zip(reqs, arrivals):
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(r["psf"], r["n"], K.BC_REFLEXIVE, 20, r["b"], MU, LAM, r["tv"], OUTER,
                              prec=prec, psf_key=r["key"]))
    outs = [srv.poll(i, timeout_us=-1) for i in ids]
    t_all = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return dict(x=[o[0] for o in outs], stats=[o[1] for o in outs], lat=[o[2] for o in outs], makespan=t_all,
                server=st, launches=K.kpsb_kernel_launches() - launches0)


def plain_service_times(K, I, torch, seed: int):
    """Per-size service time of the plain path (FP32 EGKB build, FP64 split Bregman), one
    request per size alone: the build in full and the first m outer steps timed (m = 3 for
    n <= 256, 1 above), extrapolated to 100 outer steps by the CGLS iteration count of the
    same request on the mixed path (BF16X3: the CGLS iteration is the unit of work)."""
    out = {}
    for n in SERVE_SIZES:
        reqs, _ = serving_trace(K, I, torch, seed + n, 1, 1.0, sizes=(n,))
        r = reqs[0]
        m = 3 if n <= 256 else 1
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kp = K.kp_build(r["psf"], n, K.BC_REFLEXIVE, 20, K.EGKB, seed=r["key"])
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, st_m = K.sb_solve(kp, r["b"], MU, LAM, r["tv"], m, prec=K.P_FP64)
        t_m = time.perf_counter() - t0
        _, st_mix_m = K.sb_solve(kp, r["b"], MU, LAM, r["tv"], m, prec=K.P_BF16X3)
        _, st_mix = K.sb_solve(kp, r["b"], MU, LAM, r["tv"], OUTER, prec=K.P_BF16X3)
        kp.close()
        scale = st_mix.iota_total / max(1, st_mix_m.iota_total)
        out[n] = dict(build_s=t_build, sb_first_outer_s=t_m, outer_timed=m, iota_timed=st_m.iota_total,
                      iota_full_est=round(st_m.iota_total * scale), service_s=t_build + t_m * scale)
    return out


def fifo(arrivals, service):
    """Latencies and makespan of one server taking requests one at a time in arrival order."""
    t, lat = 0.0, []
    for a, sv in zip(arrivals, service):
        t = max(t, a) + sv
        lat.append(t - a)
    return lat, t


def serving_block(K, I, torch, count: int):
    """Configuration 5: Poisson arrivals at several rates, mixed sizes, the mixed path (BF16X3
    Kronecker GEMMs, FP64 split Bregman) through the continuous-batching server against the
    plain path one request at a time on the same traces."""
    import numpy as np

    prec = K.P_BF16X3
    # warm-up: every size once through the server (tables, tuner choices, graph paths)
    reqs, arr = serving_trace(K, I, torch, 6999, 4, 1000.0)
    serve_trace_run(K, reqs, arr * 0, prec)
    plain = plain_service_times(K, I, torch, 7100)
    rates = []
    isnr_pairs = []
    for ri, rate in enumerate(SERVE_RATES):
        reqs, arrivals = serving_trace(K, I, torch, 7000 + ri, count, rate)
        res = serve_trace_run(K, reqs, arrivals, prec)
        lat_plain, mk_plain = fifo(arrivals, [plain[r["n"]]["service_s"] for r in reqs])
        isnr = [_isnr(x, r["b"], r["xt"]) for x, r in zip(res["x"], reqs)]
        rates.append({"rate_per_s": rate, "requests": count, "sizes": [r["n"] for r in reqs],
                      "deblurs_per_s": count / res["makespan"], "p50_ms": 1e3 * _pct(res["lat"], 0.5),
                      "p99_ms": 1e3 * _pct(res["lat"], 0.99), "makespan_s": res["makespan"],
                      "isnr_db_mean": statistics.mean(isnr), "cache_hits": res["server"]["cache_hits"],
                      "peak_device_bytes": res["server"]["peak_bytes"], "gpu_launches": res["launches"],
                      "plain_fifo": {"deblurs_per_s": count / mk_plain, "p50_ms": 1e3 * _pct(lat_plain, 0.5),
                                     "p99_ms": 1e3 * _pct(lat_plain, 0.99)}})
        if ri == 0:  # equal ISNR: every n = 128 request of the first trace solved alone in FP64
            for x, r in zip(res["x"], reqs):
                if r["n"] == 128:
                    kp = K.kp_build(r["psf"], 128, K.BC_REFLEXIVE, 20, K.EGKB, seed=r["key"])
                    x64, _ = K.sb_solve(kp, r["b"], MU, LAM, r["tv"], OUTER, prec=K.P_FP64)
                    kp.close()
                    isnr_pairs.append((_isnr(x, r["b"], r["xt"]), _isnr(x64, r["b"], r["xt"])))
    # equal ISNR at every size: 5 outer steps, mixed vs FP64, one request per size
    short = []
    for n in SERVE_SIZES:
        reqs, _ = serving_trace(K, I, torch, 7200 + n, 1, 1.0, sizes=(n,))
        r = reqs[0]
        kp = K.kp_build(r["psf"], n, K.BC_REFLEXIVE, 20, K.EGKB, seed=r["key"])
        xm, _ = K.sb_solve(kp, r["b"], MU, LAM, r["tv"], 5, prec=prec)
        x64, _ = K.sb_solve(kp, r["b"], MU, LAM, r["tv"], 5, prec=K.P_FP64)
        kp.close()
        short.append({"n": n, "isnr_abs_diff_db": abs(_isnr(xm, r["b"], r["xt"]) - _isnr(x64, r["b"], r["xt"]))})
    head = rates[0]
    return {
        "workload": "configuration 5: Poisson arrivals at %s req/s, %d requests per rate, n uniform in %s, "
                    "31x31 turbulence/mixture PSFs with 30%% reuse (KP cache), noise U[1%%,5%%], iso/aniso 50/50, "
                    "k=20, 100 outer steps" % (list(SERVE_RATES), count, list(SERVE_SIZES)),
        "mixed_path": "continuous-batching server, BF16X3 Kronecker GEMMs + FP64 split Bregman, rounds of 5 "
                      "outer steps, size groups concurrent",
        "plain_path": "FP32 EGKB + FP64 split Bregman one request at a time (FIFO on the same arrival trace); "
                      "per-size service times measured with the first outer steps and extrapolated by CGLS count",
        "deblurs_per_s": head["deblurs_per_s"], "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
        "rates": rates, "plain_service_s": plain,
        "isnr_abs_diff_db_max_full_n128": max((abs(a - b) for a, b in isnr_pairs), default=None),
        "isnr_pairs_full_n128": len(isnr_pairs),
        "isnr_abs_diff_db_5_outer": short,
    }


def large_block(K, I, torch, peaks):
    """Configuration 3 (n = 512, 63 x 63 turbulence-like PSF, zero boundary, k = 20): the TSVD
    (EGKB with k_p = 40 and full reorthogonalisation; RSVD with p = 10, q = 1) with the
    achieved bandwidth of its R(A) products and CGS2 passes (CUDA events around every call,
    algorithmic bytes), the singular values against the FP64 TSVD on the GPU, then split
    Bregman iso and aniso for 100 outer steps in every Kronecker-GEMM precision, with ISNR
    against the FP64 path (10 outer steps for the comparison: FP64 GEMMs at this size are
    slow on GB300's FP64 pipe)."""
    import numpy as np

    pr = I.problem_large(0)
    n = pr.n
    b = _blur_data(K, torch, pr, 63, 63, n)
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {"workload": "configuration 3: n=512, 63x63 turbulence-like PSF, zero boundary, k=20, 1% noise"}
    tsvd = {}
    sig64 = None
    for name, method, p, fp64 in (("egkb_fp64", K.EGKB, 20, True), ("egkb", K.EGKB, 20, False),
                                  ("rsvd", K.RSVD, 10, False)):
        K.kp_build(pr.psf, n, pr.bc, 20, method, p=p, seed=pr.seed, fp64=fp64).close()  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kp = K.kp_build(pr.psf, n, pr.bc, 20, method, p=p, seed=pr.seed, fp64=fp64)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        sig = K.kp_info(kp)["sigma"]
        kp.close()
        if fp64:
            sig64 = sig
            tsvd[name] = {"build_ms": 1e3 * t_build, "k": len(sig)}
            continue
        K.kpsb_gemm_timing(True)
        K.kp_build(pr.psf, n, pr.bc, 20, method, p=p, seed=pr.seed).close()
        row = {"build_ms": 1e3 * t_build, "k": len(sig),
               "sigma_err_vs_fp64_over_sigma1": float(np.max(np.abs(sig - sig64[:len(sig)])) / sig64[0])}
        for tname, cat in K.TSVD_TIMERS.items():
            calls, ms, nbytes = K.kpsb_timer_stats(cat)
            if calls:
                row[tname] = {"calls": calls, "ms": ms, "algorithmic_bytes": nbytes,
                              "achieved_gbs": nbytes / (ms / 1e3) / 1e9,
                              "frac_of_hbm": nbytes / (ms / 1e3) / 1e9 / hbm}
        K.kpsb_gemm_timing(False)
        tsvd[name] = row
    out["tsvd"] = tsvd
    out["hbm_peak_gbs"] = hbm
    kp = K.kp_build(pr.psf, n, pr.bc, 20, K.EGKB, p=20, seed=pr.seed)
    k = K.kp_info(kp)["k"]
    precs = (("fp32", K.P_FP32), ("tf32x3", K.P_TF32X3), ("tf32x2", K.P_TF32X2), ("bf16x3", K.P_BF16X3),
             ("bf16x2", K.P_BF16X2))
    sb = {}
    for tvn, tv in (("iso", K.ISO), ("aniso", K.ANISO)):
        x64, _ = K.sb_solve(kp, b, MU, LAM, tv, 10, prec=K.P_FP64)
        ref10 = _isnr(x64, b, pr.x_true)
        rows = {}
        for pname, prec in precs:
            x10, _ = K.sb_solve(kp, b, MU, LAM, tv, 10, prec=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, st = K.sb_solve(kp, b, MU, LAM, tv, OUTER, prec=prec)
            t = time.perf_counter() - t0
            rows[pname] = {"sb_100_outer_s": t, "iota_total": st.iota_total, "isnr_db": _isnr(x, b, pr.x_true),
                           "isnr_abs_diff_db_vs_fp64_10_outer": abs(_isnr(x10, b, pr.x_true) - ref10)}
        sb[tvn] = {"fp64_isnr_db_10_outer": ref10, "precisions": rows}
    kp.close()
    out["k"] = k
    out["split_bregman"] = sb
    return out


# ---------------------------------------------------------------------------------------
# 96 uneven problems in one batched build + solve; lambda sweep on shared factors
# ---------------------------------------------------------------------------------------

def _blur_data(K, torch, pr, s0, s1, n):
    import numpy as np

    from paper_2410_00233_gb300 import inputs as I

    psf_d = torch.from_numpy(np.asfortranarray(pr.psf).reshape(-1, order="F").copy()).cuda()
    x_d = torch.from_numpy(pr.x_true.reshape(-1, order="F").copy()).cuda()
    bt_d = torch.empty_like(x_d)
    K.kp_blur_dev(psf_d.data_ptr(), s0, s1, n, pr.bc, x_d.data_ptr(), bt_d.data_ptr())
    torch.cuda.synchronize()
    bt = bt_d.cpu().numpy().reshape(n, n, order="F")
    return bt + I.noise_vector(bt, pr.eta, pr.zeta)


def batched96_main(args):
    import numpy as np
    import torch

    from paper_2410_00233_gb300 import inputs as I
    from paper_2410_00233_gb300 import kpsb as K

    torch.cuda.set_device(0)
    K.lib()
    precs = {"fp64": K.P_FP64, "fp32": K.P_FP32, "tf32x3": K.P_TF32X3, "tf32x2": K.P_TF32X2,
             "bf16x3": K.P_BF16X3, "bf16x2": K.P_BF16X2}
    prec = precs[args.prec if args.prec != "auto" else "tf32x2"]
    prs = [I.problem_batched(i) for i in range(96)]
    bs = [_blur_data(K, torch, pr, pr.psf.shape[0], pr.psf.shape[1], pr.n) for pr in prs]
    probs = [dict(psf=pr.psf, n=pr.n, bc=pr.bc, rank_or_tol=pr.k, method=K.EGKB, p=pr.p, seed=pr.seed)
             for pr in prs]

    def step():
        kps = K.kp_build_batched(probs)
        jobs = [dict(kp=kp, b=b, mu=MU, lam=LAM, tv=K.ISO if pr.iso else K.ANISO, iters=args.outer)
                for kp, b, pr in zip(kps, bs, prs)]
        return K.sb_solve_batched(jobs, prec=prec)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    times = []
    outs = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        outs, _ = step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    isnr = [20 * math.log10(np.linalg.norm(b - pr.x_true) / np.linalg.norm(x - pr.x_true))
            for x, b, pr in zip(outs, bs, prs)]
    t = sum(times)
    print(json.dumps({"metric": "batched deblurs/sec (96 uneven problems per launch)", "value": 96 * args.steps / t,
                      "unit": "deblurs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1000 * t / args.steps, "higher_is_better": True, "data": "synthetic",
                      "config": {"workload": "96 problems, n in {64,128,256,384} x 24, odd PSF sizes 15-63 "
                                             "(mixture / turbulence), k in [5,20], iso/aniso and zero/reflexive "
                                             "alternating independently of n, noise 1-5%, 100 outer; host arrays through the C ABI",
                                 "kp_gemm": args.prec if args.prec != "auto" else "tf32x2",
                                 "note": "every size on the tensor cores (n=64 on the masked two-stage kernel); "
                                         "size groups run concurrently; apply variants autotuned per group"},
                      "isnr_db_mean": statistics.mean(isnr), "isnr_db_min": min(isnr)}), flush=True)


def sweep_main(args):
    import numpy as np
    import torch

    from paper_2410_00233_gb300 import inputs as I
    from paper_2410_00233_gb300 import kpsb as K

    torch.cuda.set_device(0)
    K.lib()
    precs = {"fp64": K.P_FP64, "fp32": K.P_FP32, "tf32x3": K.P_TF32X3, "tf32x2": K.P_TF32X2,
             "bf16x3": K.P_BF16X3, "bf16x2": K.P_BF16X2}
    prec = precs[args.prec if args.prec != "auto" else "tf32x2"]
    pr = I.problem_medium(0)
    b = _blur_data(K, torch, pr, PSF_S, PSF_S, N_IMG)
    lams = np.logspace(-2, 1, 100)  # lambda in [1e-2, 10], beta = lambda^2 / gamma, gamma = 2
    kp = K.kp_build(pr.psf, N_IMG, pr.bc, pr.tau, K.EGKB, p=pr.p, seed=pr.seed)
    jobs = [dict(kp=kp, b=b, mu=MU, lam=float(l), tv=K.ISO, iters=args.outer) for l in lams]
    if not args.profile:
        K.sb_solve_batched(jobs[:4], prec=prec)  # warm-up
    torch.cuda.synchronize()
    if args.profile:
        K.kpsb_gemm_timing(True)  # host-driven loop: every kernel is a plain launch
    t0 = time.perf_counter()
    outs, stats = K.sb_solve_batched(jobs, prec=prec)
    t = time.perf_counter() - t0
    if args.profile:
        K.kpsb_gemm_timing(False)
        print(json.dumps({"profile_run": True, "workload": "sweep", "solves": len(lams), "outer": args.outer,
                          "seconds": t}), flush=True)
        return
    isnr = [20 * math.log10(np.linalg.norm(b - pr.x_true) / np.linalg.norm(x - pr.x_true)) for x in outs]
    best = int(np.argmax(isnr))
    print(json.dumps({"metric": "lambda sweep: split Bregman solves/sec on shared KP factors", "value": len(lams) / t,
                      "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
                      "config": {"workload": "n=128, 31x31 mixture PSF (reflexive), EGKB auto k, 100 log-spaced "
                                             "lambda in [1e-2, 10], beta = lambda^2/2, isotropic, 100 outer",
                                 "kp_gemm": args.prec},
                      "seconds": t, "best_lambda": float(lams[best]), "best_isnr_db": isnr[best],
                      "iota_total_mean": statistics.mean(s.iota_total for s in stats)}), flush=True)


def direct_main(args):
    """The paper's comparison (Sec. 4.3, Table 4): split Bregman with the explicit operator A
    (FP64 dense products) against the same solve with the KP sum (FP64 and TF32x2 products),
    on one medium request (n = 128, 31x31 PSF), with the predicted speed-up of eq. (4.4)."""
    import numpy as np
    import torch

    from paper_2410_00233_gb300 import costs as C
    from paper_2410_00233_gb300 import inputs as I
    from paper_2410_00233_gb300 import kpsb as K

    torch.cuda.set_device(0)
    K.lib()
    pr = I.problem_medium(0)
    b = _blur_data(K, torch, pr, PSF_S, PSF_S, N_IMG)
    n, N = N_IMG, N_IMG * N_IMG

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    def isnr(x):
        return 20 * math.log10(np.linalg.norm(b - pr.x_true) / np.linalg.norm(x - pr.x_true))

    A, t_form_a = timed(lambda: K.kp_dense_blur(pr.psf, n, pr.bc))
    (xa, sa), t_sb_a = timed(lambda: K.sb_solve(A, b, MU, LAM, K.ISO, args.outer))
    A.close()
    kp, t_build = timed(lambda: K.kp_build(pr.psf, n, pr.bc, pr.tau, K.EGKB, p=pr.p, seed=pr.seed))
    k = K.kp_info(kp)["k"]
    res = {}
    for name, prec in (("kp_fp64", K.P_FP64), ("kp_tf32x2", K.P_TF32X2)):
        (x, st), t = timed(lambda: K.sb_solve(kp, b, MU, LAM, K.ISO, args.outer, prec=prec))
        res[name] = {"sb_s": t, "total_s": t + t_build, "iota_total": st.iota_total, "isnr_db": isnr(x),
                     "sb_speedup_vs_direct": t_sb_a / t}
    print(json.dumps({
        "metric": "split Bregman with the explicit A vs the KP sum (Sec. 4.3, Table 4)", "unit": "s",
        "value": res["kp_tf32x2"]["sb_s"], "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
        "config": {"workload": "one request: n=128, 31x31 two-Gaussian mixture PSF (reflexive), EGKB auto k, "
                               "isotropic split Bregman, %d outer" % args.outer, "k": k},
        "direct_A": {"form_A_s": t_form_a, "sb_s": t_sb_a, "iota_total": sa.iota_total, "isnr_db": isnr(xa)},
        "kp_build_s": t_build, **res,
        "predicted_sb_speedup_eq_4_4": C.sb_speedup(N, N, k, n),
        "predicted_sb_speedup_this_implementation": C.sb_speedup_this_implementation(n, k),
        "note": "eq. (4.4) counts the augmented matrix as dense; here L is applied as a sparse difference, "
                "so one direct CGLS step costs 4 N^2 flops against 8 k n^3 with the KP sum"}), flush=True)


def tsvd_main(args):
    """The paper's SP/DP comparison of the TSVD (Sec. 1, Sec. 5: EGKB(SP), EGKB(DP), RSVD):
    build time per precision and reorthogonalisation, and how far the single-precision
    singular values sit from the double-precision ones, on the medium workload (n = 128, auto
    k) and the large one (n = 512, 63x63 turbulence-like PSF, k = 20)."""
    import numpy as np
    import torch

    from paper_2410_00233_gb300 import inputs as I
    from paper_2410_00233_gb300 import kpsb as K

    torch.cuda.set_device(0)
    K.lib()
    if args.profile:  # profiling run: two single-precision builds of each method at n = 512, nothing else
        pr = I.problem_large(0)
        for _ in range(2):
            K.kp_build(pr.psf, pr.n, pr.bc, 20, K.EGKB, p=pr.p, seed=pr.seed).close()
            K.kp_build(pr.psf, pr.n, pr.bc, 20, K.RSVD, p=10, seed=pr.seed).close()
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "workload": "tsvd n=512 (EGKB k_p=40, RSVD p=10), 2 builds each"}))
        return
    rows = []
    for name, pr, rank in (("medium n=128 auto-k", I.problem_medium(0), None),
                           ("large n=512 k=20", I.problem_large(0), 20)):
        rk = pr.tau if rank is None else rank
        variants = [("EGKB full", K.EGKB, False), ("EGKB one-sided", K.EGKB, True)]
        if rank is not None:
            variants.append(("RSVD", K.RSVD, False))
        for vname, method, one_sided in variants:
            res = {}
            for prec, fp64 in (("SP", False), ("DP", True)):
                opts = dict(p=pr.p if method == K.EGKB else 10, seed=pr.seed, one_sided=one_sided, fp64=fp64)
                K.kp_build(pr.psf, pr.n, pr.bc, rk, method, **opts).close()  # warm-up
                ts = []
                for _ in range(3):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    kp = K.kp_build(pr.psf, pr.n, pr.bc, rk, method, **opts)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
                    sig = K.kp_info(kp)["sigma"]
                    kp.close()
                res[prec] = (min(ts), sig)
            (t_sp, s_sp), (t_dp, s_dp) = res["SP"], res["DP"]
            k = min(len(s_sp), len(s_dp))
            rows.append({"config": name, "method": vname, "k_sp": len(s_sp), "k_dp": len(s_dp),
                         "sp_ms": 1000 * t_sp, "dp_ms": 1000 * t_dp, "dp_over_sp": t_dp / t_sp,
                         "max_sigma_diff_over_sigma1": float(np.max(np.abs(s_sp[:k] - s_dp[:k])) / s_dp[0])})
    print(json.dumps({"metric": "TSVD of R(A): single vs double precision (build time, sigma agreement)",
                      "unit": "ms", "n_gpus": 1, "data": "synthetic", "rows": rows}), flush=True)


def dense_tsvd_main(args):
    """The TSVD of R(A) for a general operator given as an explicit matrix (kp_build_dense,
    eq. (2.2) indexing read in place, n = 64 and 128): build time for EGKB and RSVD, the
    planted singular values recovered, and the effective bandwidth of the R(A) products
    (each pass over A streams its n^4 FP32 entries).  The operator is
    A = sum_i s_i Ax_i (x) Ay_i + eps G with Frobenius-orthonormal factors, so the singular
    values of R(A) are s_i up to eps ||R(G)||."""
    import numpy as np
    import torch

    from paper_2410_00233_gb300 import inputs as I
    from paper_2410_00233_gb300 import kpsb as K

    torch.cuda.set_device(0)
    K.lib()
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    s_true = np.array([1.0, 0.5, 0.25, 0.125])
    r = len(s_true)
    rows = []
    for n in (64, 128):
        g = I.rng(8000 + n)
        qx, _ = np.linalg.qr(g.standard_normal((n * n, r)))
        qy, _ = np.linalg.qr(g.standard_normal((n * n, r)))
        A = np.zeros((n * n, n * n))
        for i in range(r):
            A += s_true[i] * np.kron(qx[:, i].reshape(n, n, order="F"), qy[:, i].reshape(n, n, order="F"))
        eps = 1e-4 / n
        A += eps * g.standard_normal((n * n, n * n))
        A = np.asfortranarray(A)
        for mname, method, p in (("EGKB", K.EGKB, 4), ("RSVD", K.RSVD, 6)):
            K.kp_build_dense(A, n, r, method, p=p, seed=1).close()  # warm-up
            ts = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                kp = K.kp_build_dense(A, n, r, method, p=p, seed=1)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                inf = K.kp_info(kp)
                kp.close()
            # the passes over A timed on the device: CUDA events around every R(A) product,
            # algorithmic bytes 4 n^4 per pass (8 vectors per pass) counted by the library
            K.kpsb_gemm_timing(True)
            K.kp_build_dense(A, n, r, method, p=p, seed=1).close()
            calls, ra_ms, ra_bytes = K.kpsb_timer_stats(K.TSVD_TIMERS["ra_products"])
            K.kpsb_gemm_timing(False)
            t = min(ts)
            sig = inf["sigma"]
            k = min(len(sig), r)
            rows.append({"n": n, "method": mname, "k": len(sig), "k_p": inf["kp"], "build_ms": 1000 * t,
                         "max_sigma_err_over_s1": float(np.max(np.abs(sig[:k] - s_true[:k]))),
                         "ra_product_calls": calls, "ra_products_device_ms": ra_ms,
                         "ra_products_algorithmic_bytes": ra_bytes,
                         "ra_products_gbs": ra_bytes / (ra_ms / 1e3) / 1e9 if ra_ms else None,
                         "ra_products_frac_of_hbm": (ra_bytes / (ra_ms / 1e3) / 1e9 / hbm) if ra_ms else None,
                         "note": "build_ms is host wall time and includes the FP32 copy and upload of A; the "
                                 "R(A) product figures are device time of the passes over A alone"})
    print(json.dumps({"metric": "TSVD of R(A) for an explicit general operator (kp_build_dense)", "unit": "ms",
                      "n_gpus": 1, "data": "synthetic (planted KP sum + dense perturbation)", "rows": rows}),
          flush=True)


def single_main(args):
    """One request of the serving workload (side --n, k = 20, 31x31 PSF) alone: kp_build +
    split Bregman (--outer steps) in the selected precision, device-timed; with --profile the
    solve runs the host-driven loop (every kernel a plain launch) for ncu."""
    import torch

    from paper_2410_00233_gb300 import inputs as I
    from paper_2410_00233_gb300 import kpsb as K

    torch.cuda.set_device(0)
    K.lib()
    precs = {"fp64": K.P_FP64, "fp32": K.P_FP32, "tf32x3": K.P_TF32X3, "tf32x2": K.P_TF32X2,
             "bf16x3": K.P_BF16X3, "bf16x2": K.P_BF16X2}
    prec = precs[args.prec if args.prec != "auto" else "bf16x3"]
    reqs, _ = serving_trace(K, I, torch, 7300 + args.n, 1, 1.0, sizes=(args.n,))
    r = reqs[0]
    kp = K.kp_build(r["psf"], args.n, K.BC_REFLEXIVE, 20, K.EGKB, seed=r["key"])
    K.sb_solve(kp, r["b"], MU, LAM, r["tv"], 1, i_max=3, fixed_inner=True, prec=prec)  # warm-up
    if args.profile:
        K.kpsb_gemm_timing(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, st = K.sb_solve(kp, r["b"], MU, LAM, r["tv"], args.outer, prec=prec)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    if args.profile:
        K.kpsb_gemm_timing(False)
    print(json.dumps({"metric": "one request alone: split Bregman seconds", "value": t, "unit": "s",
                      "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
                      "config": {"workload": "serving request, n=%d, k=20, %d outer" % (args.n, args.outer),
                                 "kp_gemm": args.prec if args.prec != "auto" else "bf16x3"},
                      "iota_total": st.iota_total, "isnr_db": _isnr(x, r["b"], r["xt"])}), flush=True)


def main():
    args = parse()
    if args.cpu_worker > 0:
        print(json.dumps(cpu_worker(args.cpu_worker, args.cpu_samples)), flush=True)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.serve:
        serve_main(args)
        return
    if args.workload == "batched96":
        batched96_main(args)
        return
    if args.workload == "sweep":
        sweep_main(args)
        return
    if args.workload == "direct":
        direct_main(args)
        return
    if args.workload == "tsvd":
        tsvd_main(args)
        return
    if args.workload == "dense_tsvd":
        dense_tsvd_main(args)
        return
    if args.workload == "single":
        single_main(args)
        return

    import numpy as np
    import torch

    from paper_2410_00233_gb300 import inputs as I
    from paper_2410_00233_gb300 import kpsb as K

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if not os.path.exists(K.LIB_PATH):
        from paper_2410_00233_gb300 import build as B

        B.build()
    K.lib()
    precs = {"fp64": K.P_FP64, "fp32": K.P_FP32, "tf32x3": K.P_TF32X3, "tf32x2": K.P_TF32X2,
             "bf16x3": K.P_BF16X3, "bf16x2": K.P_BF16X2}
    prec_name = args.prec
    if prec_name == "auto":
        prec_name = os.environ.get("KPSB_BENCH_PREC", "tf32x2")
    prec = precs[prec_name]
    B = args.batch
    W, S = args.warmup, args.steps
    # inputs of every step, distinct requests per rank and step
    from paper_2410_00233_gb300 import shard

    steps_in = [make_inputs(K, I, torch, B, shard.request_ids(rank, s, B).start, dev) for s in range(W + S)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    # warm-up
    for s in range(W):
        run_step(K, steps_in[s], prec, args.outer, args.sub_batches)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    times = []
    launches0 = K.kpsb_kernel_launches()
    if args.profile:
        K.kpsb_gemm_timing(True)  # host-driven loop: every kernel is a plain launch
    clocks = ClockSampler(local)
    ks = []
    stats_first = None
    for s in range(W, W + S):
        flush.fill_(float(s))  # evict L2 between timed steps
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        kps, stats = run_step(K, steps_in[s], prec, args.outer, args.sub_batches)
        ev1.record()
        barrier()
        times.append(ev0.elapsed_time(ev1) / 1000.0)
        ks.extend(K.kp_info(kp)["k"] for kp in kps)
        if stats_first is None:
            stats_first = stats
        del kps
    clk = clocks.stop()
    launches = K.kpsb_kernel_launches() - launches0
    t_rank = sum(times)
    t_max = shard.job_seconds(t_rank, dist, dev)
    value = shard.throughput(B * S, world, t_max)
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "value": world * B * S / t_max, "unit": "deblurs/s",
                              "steps": S, "batch": B, "outer": args.outer, "gpu_launches": launches}), flush=True)
        return

    # roofline of the dominant kernel: one instrumented replay of the first timed step (the
    # library then drives the CGLS loop from the host and brackets every KP apply with CUDA
    # events on its stream); the timed steps above ran the production graph path
    flush.fill_(-1.0)
    torch.cuda.synchronize()
    K.kpsb_gemm_timing(True)
    t0 = time.perf_counter()
    reqs = steps_in[W]
    kps_i = K.kp_build_batched([dict(psf=r["pr"].psf, n=N_IMG, bc=r["pr"].bc, rank_or_tol=r["pr"].tau,
                                     method=K.EGKB, p=r["pr"].p, seed=r["pr"].seed) for r in reqs])
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    # the batch's TSVD (Alg. 1) ran as one-block EGKB launches: their algorithmic bytes (R(A)
    # products and CGS2 passes, counted on the device) over their CUDA-event time
    eb_calls, eb_ms, eb_bytes = K.kpsb_timer_stats(K.TSVD_TIMERS["egkb_block"])
    # one part (sub_batches=1): the applies run alone, so their events time the kernel itself
    st_i = K.sb_solve_batched([dict(kp=kp, b=r["b_d"].data_ptr(), x=r["x_d"].data_ptr(), mu=MU, lam=LAM,
                                    tv=K.ISO, iters=args.outer) for kp, r in zip(kps_i, reqs)],
                              on_device=True, prec=prec, sub_batches=1)
    torch.cuda.synchronize()
    t_instr = time.perf_counter() - t0
    del kps_i
    gl, gms, gflops = K.kpsb_gemm_stats()
    phases = {"build_s": t_build, "solve_s": t_instr - t_build}
    for cat, name in enumerate(K.TIMER_NAMES):
        cl, cms, _ = K.kpsb_timer_stats(cat)
        phases[name + "_ms"] = cms
        phases[name + "_launches"] = cl
    # every forward apply is followed by one ||z||^2 kernel, every transpose apply by one f kernel
    phases["cgls_iterations_batch"] = phases["cgls_zz_launches"]
    gapplies = phases["cgls_zz_launches"] + phases["cgls_f_launches"]
    pa, kn3 = K.kpsb_apply_counts()  # problem-applies actually performed (active problems), sum k n^3
    phases["active_problems_per_apply"] = pa / gapplies if gapplies else None
    # the apply variant the replay ran (the autotuner's choice for this batch, n = 128)
    replay_variant = None
    bucket = 1
    while bucket < B:
        bucket <<= 1
    for t in K.kpsb_tuned_variants():
        if t["n"] == N_IMG and t["prec"] == prec and t["bucket"] == bucket and not t["shared"]:
            replay_variant = t["variant"]
    # DRAM traffic per launch of that kernel: ncu captures (dram__bytes_read.sum +
    # dram__bytes_write.sum) of each variant on this workload (256 requests, one part, every
    # problem active: the first CGLS applies), forward and transpose alternating; inactive
    # problems read nothing, so the launch's traffic follows its active problems.
    traffic = None
    cap = DRAM_BYTES_256_ACTIVE.get((prec, replay_variant))
    if cap is not None and gapplies and pa:
        traffic = cap * (pa / gapplies) / 256.0
    K.kpsb_gemm_timing(False)
    # ISNR of the mixed path on the first timed step
    reqs = steps_in[W]
    isnr_mixed = []
    for r in reqs:
        x = r["x_d"].cpu().numpy().reshape(N_IMG, N_IMG, order="F")
        isnr_mixed.append(20 * math.log10(np.linalg.norm(r["b"] - r["pr"].x_true) /
                                          np.linalg.norm(x - r["pr"].x_true)))

    # equal ISNR over the timed step: the plain arithmetic (FP64 Kronecker GEMMs, same factors
    # builder, same split Bregman) on every 8th request of the first timed step, batched for
    # time, against the mixed path's result of the same request
    isnr_cmp = None
    if not args.no_plain:
        sample = list(range(0, len(reqs), 8))
        kps_p = K.kp_build_batched([dict(psf=reqs[i]["pr"].psf, n=N_IMG, bc=reqs[i]["pr"].bc,
                                         rank_or_tol=reqs[i]["pr"].tau, method=K.EGKB, p=reqs[i]["pr"].p,
                                         seed=reqs[i]["pr"].seed) for i in sample])
        xs = [torch.zeros_like(reqs[i]["b_d"]) for i in sample]
        K.sb_solve_batched([dict(kp=kp, b=reqs[i]["b_d"].data_ptr(), x=x.data_ptr(), mu=MU, lam=LAM, tv=K.ISO,
                                 iters=args.outer) for kp, i, x in zip(kps_p, sample, xs)],
                           on_device=True, prec=K.P_FP64)
        torch.cuda.synchronize()
        diffs = []
        for i, x in zip(sample, xs):
            r = reqs[i]
            xp = x.cpu().numpy().reshape(N_IMG, N_IMG, order="F")
            diffs.append(abs(_isnr(xp, r["b"], r["pr"].x_true) - isnr_mixed[i]))
        del kps_p
        isnr_cmp = {"isnr_abs_diff_db_max": max(diffs), "isnr_abs_diff_db_mean": statistics.mean(diffs),
                    "requests": len(sample),
                    "sample": "every 8th request of the first timed step, FP64 Kronecker GEMMs (the plain "
                              "arithmetic) batched, against the mixed result of the same request"}

    # end to end through the host-pointer C ABI (pinned host buffers), every step
    e2e = None
    if True:
        n_e2e = min(S, 3)
        pins = []
        for s in range(W, W + n_e2e):
            bufs = []
            for r in steps_in[s]:
                bp = torch.empty((N_IMG * N_IMG,), dtype=torch.float64).pin_memory()
                bp.numpy()[:] = r["b"].reshape(-1, order="F")
                xp = torch.empty((N_IMG * N_IMG,), dtype=torch.float64).pin_memory()
                bufs.append((bp, xp))
            pins.append(bufs)
        t_e2e = 0.0
        for j, s in enumerate(range(W, W + n_e2e)):
            flush.fill_(float(j))
            barrier()
            t0 = time.perf_counter()
            probs = [dict(psf=r["pr"].psf, n=N_IMG, bc=r["pr"].bc, rank_or_tol=r["pr"].tau, method=K.EGKB,
                          p=r["pr"].p, seed=r["pr"].seed) for r in steps_in[s]]
            kps = K.kp_build_batched(probs)
            import ctypes as C

            arr = (K.SBJob * B)()
            st_arr = (K.SBStats * B)()
            for i, (kp, (bp, xp)) in enumerate(zip(kps, pins[j])):
                arr[i].kp = kp.ptr
                arr[i].b, arr[i].x = bp.data_ptr(), xp.data_ptr()
                arr[i].mu, arr[i].lambda_, arr[i].beta = MU, LAM, 0.0
                arr[i].tv, arr[i].iters = K.ISO, args.outer
                arr[i].stats = C.pointer(st_arr[i])
            o = K._sb_opts(prec=prec)
            K._check("sb_solve_batched", K.lib().sb_solve_batched(B, arr, 0, C.byref(o)))
            t_e2e += time.perf_counter() - t0
            del kps
        t_e2e = shard.job_seconds(t_e2e, dist, dev)
        h2d = B * (N_IMG * N_IMG * 8 + PSF_S * PSF_S * 8)
        d2h = B * N_IMG * N_IMG * 8
        e2e = {"value": world * B * n_e2e / t_e2e, "unit": "deblurs/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    out = None
    if rank == 0:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except Exception:
            pass
        hbm_peak = peaks.get("hbm_gbs")
        tsvd_roof = None
        if eb_calls and eb_ms:
            ach = eb_bytes / (eb_ms / 1e3) / 1e9
            tsvd_roof = {"kernel": "egkb_block_kernel: Alg. 1 steps 3-15 of every request of the step, one "
                                   "thread block per request, %d launch(es)" % eb_calls,
                         "bound": "hbm", "achieved": ach, "unit": "GB/s",
                         "peak": hbm_peak or 6800.0,
                         "peak_note": "of measured" if hbm_peak else "of fallback",
                         "frac": ach / (hbm_peak or 6800.0), "algorithmic_bytes": eb_bytes, "ms": eb_ms,
                         "bytes_note": "R(A) products (vectors read and written, the PSF) and CGS2 passes "
                                       "(2 (2m + 3) N elements for m basis vectors) of every EGKB step; "
                                       "the bases of a request stay in L2/L1 between passes, so this can "
                                       "exceed what DRAM alone would allow"}
        # plain path: FP32 EGKB + FP64 split Bregman, one request at a time
        plain = None
        if not args.no_plain:
            r = steps_in[W][0]
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            xd = torch.zeros_like(r["b_d"])
            torch.cuda.synchronize()
            ev0.record()
            kp = K.kp_build(r["pr"].psf, N_IMG, r["pr"].bc, r["pr"].tau, K.EGKB, p=r["pr"].p, seed=r["pr"].seed)
            st = K.sb_solve_dev(kp, r["b_d"].data_ptr(), xd.data_ptr(), MU, LAM, K.ISO, args.outer, prec=K.P_FP64)
            ev1.record()
            torch.cuda.synchronize()
            tp = ev0.elapsed_time(ev1) / 1000.0
            x = xd.cpu().numpy().reshape(N_IMG, N_IMG, order="F")
            isnr_plain = 20 * math.log10(np.linalg.norm(r["b"] - r["pr"].x_true) /
                                         np.linalg.norm(x - r["pr"].x_true))
            plain = {"value": 1.0 / tp, "unit": "deblurs/s", "latency_ms": tp * 1000.0,
                     "isnr_db": isnr_plain, "isnr_mixed_db": isnr_mixed[0],
                     "isnr_abs_diff_db": abs(isnr_plain - isnr_mixed[0]),
                     "iota_total": st.iota_total, "iota_total_mixed": stats_first[0].iota_total}
        # roofline of the dominant kernel (KP GEMM)
        achieved = gflops / (gms / 1000.0) / 1e12 if gms > 0 else None
        src = "of measured" if "bf16_tflops_sustained" in peaks else "of fallback: 1700 TFLOP/s sustained bf16"
        if prec in (K.P_TF32X3, K.P_TF32X2):
            peak = peaks.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25)
            roof = {"bound": "tensor", "peak_note": "TF32 = sustained bf16 x 1.1/2.25 (%s)" % src}
        elif prec in (K.P_BF16X3, K.P_BF16X2):
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            roof = {"bound": "tensor", "peak_note": "sustained bf16 (%s)" % src}
        elif prec == K.P_FP32:
            peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            roof = {"bound": "alu", "peak_note": "FP32 FMA: 152 SM x 128 lanes x 2 x max SM clock"}
        else:
            peak = 152 * 2 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            roof = {"bound": "alu", "peak_note": "FP64 FMA: 152 SM x 2 lanes x 2 x max SM clock"}
        roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None})
        tc_prec = {K.P_TF32X2: "tf32x2", K.P_TF32X3: "tf32x3", K.P_BF16X3: "bf16x3", K.P_BF16X2: "bf16x2"}
        if prec in tc_prec and gl and gms > 0 and pa:
            hbm_peak = peaks.get("hbm_gbs", 6800.0)
            rl = apply_roofline(tc_prec[prec], N_IMG, pa, kn3, gflops, gms / 1000.0, peak, hbm_peak)
            alg_bytes, ach_gbs, oi, ridge = rl["bytes"], rl["achieved_gbs"], rl["intensity"], rl["ridge"]
            prods = SPLIT_MODES[tc_prec[prec]][2]
            tensor_view = {"achieved_tflops": achieved, "peak_tflops": peak, "frac": roof["frac"],
                           "peak_note": roof["peak_note"],
                           "useful_ceiling_note": "a split mode does %d products per useful one" % prods}
            hbm_view = {"achieved_gbs": ach_gbs, "peak_gbs": hbm_peak, "frac": ach_gbs / hbm_peak,
                        "algorithmic_bytes_per_launch": alg_bytes / gl,
                        "peak_note": "of measured" if "hbm_gbs" in peaks else "of fallback"}
            if rl["bound"] == "hbm":
                roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": ach_gbs / hbm_peak, "peak_note": hbm_view["peak_note"]}
            roof.update({"operational_intensity_flop_per_byte": oi, "ridge_flop_per_byte": ridge,
                         "tensor_view": tensor_view, "hbm_view": hbm_view})
        roof.update({"traffic": traffic,
                     "traffic_note": "bytes per launch (DRAM read + write): ncu capture of the same kernel on "
                                     "this workload with all 256 problems active, times the replay's mean "
                                     "active fraction" if traffic is not None else
                                     "no capture of this kernel variant on this workload",
                     "kernel": "KP apply, %s tensor-core kernel (autotuned for %d jobs), %d launch(es) per apply" % (
                         K.VARIANT_NAMES.get(replay_variant, "?"), B, round(gl / max(1, gapplies))),
                     "tuned_variants": K.kpsb_tuned_variants(),
                     "launches": gl, "kernel_ms": gms, "instrumented_step_s": t_instr,
                     "algorithmic_flops_per_launch": (gflops / gl) if gl else None,
                     "measured": "CUDA events around every KP apply in an instrumented replay of one timed step"})
        cpu = None
        if not args.no_cpu:
            try:
                d = run_cpu_baseline(20.0)[0]
                cpu = {"value": d["value"], "unit": "deblurs/s", "cores": d["cores"], "kind": "oracle",
                       "sample": d["sample"], **host_cpu()}
            except Exception as e:  # reported, not fatal
                cpu = {"value": None, "unit": "deblurs/s", "cores": 1, "kind": "oracle", "sample": str(e)[:200]}
        serving = None
        if not args.no_serve:
            try:
                serving = serving_block(K, I, torch, args.serve_count)
            except Exception as e:  # reported, not fatal
                serving = {"error": str(e)[:300]}
        large = None
        if not args.no_large:
            try:
                large = large_block(K, I, torch, peaks)
            except Exception as e:  # reported, not fatal
                large = {"error": str(e)[:300]}
        lat = sorted(times)
        out = {
            "metric": "deblurs/sec + p50/p99 latency, mixed-precision vs plain path, equal ISNR",
            "value": value, "unit": "deblurs/s", "n_gpus": world, "steps": S, "warmup": W,
            "ms_per_step": 1000.0 * t_max / S, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"{prec_name}+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch_per_gpu": B, "global_batch": B * world,
                       "n": N_IMG, "psf": PSF_S, "outer_iters": args.outer, "mean_k": statistics.mean(ks),
                       "kp_gemm": prec_name, "l2": "flushed (256 MB write) between timed steps",
                       "sub_batches": ("auto: %d concurrent parts of the batch" % max(1, min(4, B // 64))
                                       if args.sub_batches <= 0 else args.sub_batches),
                       "parallelism": f"dp{world} (independent requests per GPU)"},
            "p50_ms": 1000.0 * lat[len(lat) // 2], "p99_ms": 1000.0 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "latency_note": "p50/p99: per-request latency of the batched step (every request of a step completes "
                            "with the step); per-request latencies under arrivals are in serving",
            "isnr_db_mean": statistics.mean(isnr_mixed), "equal_isnr": isnr_cmp,
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
            "plain": plain, "clocks": clk,
            "phases_instrumented_step": phases, "tsvd_roofline": tsvd_roof,
            "serving": serving, "large_n512": large,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
