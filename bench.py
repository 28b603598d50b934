"""Benchmark: HBS build seconds + incident angles per second at N = 100 000.

Workload (default): the complicated obstacle, r0 = 0.3 with 60 seeded Fourier modes of
amplitude <= 0.05, omega = 60, d = 1, N = 100 000 boundary nodes, 1000 incident angles
in 100 groups of 10 that share a Bloch phase.  One step = the whole hot path:
hbs_build (HBS compression and inversion, neighbour factors, periodizer precompute)
followed by hbs_solve of all 1000 angles (Bragg amplitudes + flux errors).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` = angles solved per second of whole-step time (build
included) with the geometry resident on the device; `e2e` = the same through the C ABI
with host arrays (host-to-device copies and the read-back of the amplitudes inside the
timed region).  Under torchrun every rank solves its own copy of the workload on its GPU
(independent problems, no collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1301_1247_gb300 import inputs  # noqa: E402

METRIC = "HBS build s + incident angles/s at N=1e5, err <=1e-10 vs FP64 plain path"
UNIT = "angles/s"
# FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _measured_peaks():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {"bf16_tflops": 1900.0}  # fallback: one earlier GB300 measurement


MEASURED_PEAKS = _measured_peaks()
# FP32-pipe instruction issue: 152 SM x 128 lanes x 2.07 GHz (instructions / s)
FP32_INSTR_PEAK = 152 * 128 * 2.07e9


def kernel_peak(name, prec):
    """(bound, peak TFLOP/s, note) for a kernel's algorithmic FP64-equivalent rate, by the unit
    that executes its arithmetic in this precision mode."""
    if name == "k_oz_mma":
        return ("tensor", MEASURED_PEAKS["bf16_tflops"],
                "executed bf16 tensor flops (28 digit pairs x 4 real products x 2 m n k, padded tiles) "
                "against the measured cuBLAS bf16 burst rate in MEASURED_PEAKS.json")
    if name == "k_zgemm_batched_df" or (prec >= 1 and name in ("k_pqr", "k_cpqr")):
        per = {"k_zgemm_batched_df": 48.0 / 8.0, "k_pqr": 102.0 / 16.0, "k_cpqr": 102.0 / 16.0}[name]
        return ("alu", FP32_INSTR_PEAK / per / 1e12,
                "double-float arithmetic on the FP32 pipes: %.2f FP32-pipe instructions per FP64-equivalent flop "
                "(complex multiply-add = 4 error-free multiply-adds of 12 instructions) at 152 SM x 128 lanes x "
                "2.07 GHz" % per)
    return ("alu", FP64_PEAK_TFLOPS, "FP64 from unit counts x clock (152 SM x 2 DFMA/clk x 2.07 GHz); "
                                      "no FP64 figure in MEASURED_PEAKS.json")

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, averaged over the
# kernel's launches in one step of this bench's default workload) from one ncu capture,
# with the digest of the sources the kernel is built from at capture time.  The figure
# is reported only while those sources are unchanged.
NCU_TRAFFIC = {
    # profiles/launch_list_complicated_n100k.md: mean over the kernel's launches in one run
    "k_pqr": {"bytes_per_launch": 4.962e+09, "sources": ['paper_1301_1247_gb300/csrc/pqr.cu', 'paper_1301_1247_gb300/csrc/common.cuh', 'paper_1301_1247_gb300/csrc/gridsync.cuh', 'paper_1301_1247_gb300/csrc/dense_kernels.cuh', 'paper_1301_1247_gb300/csrc/dfloat.cuh', 'paper_1301_1247_gb300/csrc/dfcore.cuh', 'paper_1301_1247_gb300/csrc/hankel_table.h', 'paper_1301_1247_gb300/csrc/balance.hpp'],
              "digest": "a6d5580279ef7a21"},
    "k_zgemm_batched_df": {"bytes_per_launch": 3.087e+08, "sources": ['paper_1301_1247_gb300/csrc/zgemm.cuh', 'paper_1301_1247_gb300/csrc/common.cuh', 'paper_1301_1247_gb300/csrc/dfcore.cuh', 'paper_1301_1247_gb300/csrc/dfloat.cuh', 'paper_1301_1247_gb300/csrc/hankel_table.h'],
                           "digest": "982e0a980ec1bb5a"},
}


def _sources_digest(paths):
    import hashlib
    hsh = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()[:16]


def measured_traffic(kernel):
    rec = NCU_TRAFFIC.get(kernel)
    if rec is None:
        return None
    try:
        if _sources_digest(rec["sources"]) != rec["digest"]:
            return None
    except OSError:
        return None
    return rec["bytes_per_launch"]


def workload(name):
    if name == "complicated_n100k":
        w = inputs.workload_complicated_n100k()
    elif name == "wiggly_n10k":
        w = inputs.workload_wiggly_n10k()
    elif name == "star_n400":
        w = inputs.workload_star_n400()
    else:
        raise SystemExit(f"unknown workload {name}")
    w["name"] = name
    return w


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def _cuda():
    import torch
    return torch.cuda.is_available()


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(ws, units_per_step, steps, ms_max):
    """Units per second of the whole job: every rank processes units_per_step units per
    step (weak scaling), and the slowest rank's time (ms_max, max over ranks) counts."""
    return ws * units_per_step * steps / (ms_max / 1e3)


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def run_ours(args, ws, rank, local):
    import torch
    from paper_1301_1247_gb300 import hbs

    torch.cuda.set_device(local)
    w = workload(args.workload)
    obs, omega, d, n = w["obstacle"], w["omega"], w["d"], w["N"]
    thetas = np.asarray(w["thetas"], dtype=np.float64).ravel()
    x, y, dx, dy = obs.sample(n)
    gx, gy, gdx, gdy = (torch.from_numpy(a).cuda() for a in (x, y, dx, dy))
    hx, hy, hdx, hdy = (torch.from_numpy(a).pin_memory() for a in (x, y, dx, dy))
    hth = torch.from_numpy(thetas).pin_memory()
    stream = torch.cuda.current_stream()
    tol = 1e-12

    prec = {"fp64": 0, "df": 1, "tc": 2}[args.precision]
    opts = hbs.default_options(precision=prec)

    def step(device_inputs: bool):
        if device_inputs:
            h = hbs.Handle(gx, gy, gdx, gdy, d, omega, tol, opts, stream=stream)
        else:
            h = hbs.Handle(hx.numpy(), hy.numpy(), hdx.numpy(), hdy.numpy(), d, omega, tol, opts, stream=stream)
        r = h.solve(hth.numpy(), stream=stream)
        amps = [r.bragg(i) for i in range(len(thetas))]
        return h, r, amps

    info = None
    for _ in range(args.warmup):
        h, r, amps = step(True)
        info = h.info()
        del h, r
    torch.cuda.synchronize()

    # ---- device-resident inputs: value + roofline
    hbs.profile_reset()
    hbs.profile_enable(True)
    l0 = hbs.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            h, r, amps = step(True)
            if info is None:
                info = h.info()
            del h, r
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    launches = hbs.launch_count() - l0
    hbs.profile_enable(False)
    prof = hbs.profile_get()
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, ws)

    # ---- end to end: host inputs, copies and read-back inside the timed region
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        h, r, amps = step(False)
        del h, r
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(max(e2.elapsed_time(e3), 1e3 * (time.perf_counter() - t0)), ws)
    flux = [a[3] for a in amps]

    # accuracy check (outside the timed region): one Bloch group against the all-FP64 plain
    # per-phase path (q + 2M + 2l applies of an FP64-built compressed inverse)
    err = None
    if not args.no_check:
        th2 = np.asarray(w["thetas"])
        gsel = th2[0] if th2.ndim == 2 else thetas[: min(10, len(thetas))]
        idx = [int(np.flatnonzero(thetas == t)[0]) for t in gsel]
        h64 = hbs.Handle(x, y, dx, dy, d, omega, tol)
        ref = h64.solve_plain(gsel)
        errs = []
        for i, k in enumerate(idx):
            _, c1, d1, _ = amps[k]
            _, c2, d2, _ = ref.bragg(i)
            a, b = np.concatenate([c1, d1]), np.concatenate([c2, d2])
            errs.append(float(np.linalg.norm(a - b) / np.linalg.norm(b)))
        err = max(errs)
        del h64, ref

    n_ang = len(thetas)
    value = whole_job_rate(ws, n_ang, args.steps, ms_max)
    kern = {k: v for k, v in prof.items() if not k.startswith("phase:")}
    phases = {k[6:]: round(v["ms"] / args.steps, 2) for k, v in prof.items() if k.startswith("phase:")}
    top = max(kern.items(), key=lambda kv: kv[1]["ms"])
    tname, tv = top
    achieved = tv["flops"] / (tv["ms"] / 1e3) / 1e12 if tv["ms"] > 0 else 0.0
    kbound, kpeak, knote = kernel_peak(tname, prec)
    shares = {k: round(v["ms"] / sum(x["ms"] for x in kern.values()), 4) for k, v in
              sorted(kern.items(), key=lambda kv: -kv[1]["ms"])[:8]}
    # algorithmic FP64(-equivalent) rate of the top kernels that record flops
    rates = {k: round(v["flops"] / (v["ms"] / 1e3) / 1e12, 4) for k, v in
             sorted(kern.items(), key=lambda kv: -kv[1]["ms"])[:8] if v["flops"] > 0 and v["ms"] > 0}
    h2d = 4 * n * 8 + n_ang * 8
    n_orders = sum(len(a[1]) for a in amps)
    d2h = n_orders * 2 * 16 + n_ang * 8
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f64 (complex128)",
                  1: "f64 (complex128) data; double-float (2xFP32) arithmetic for the dense products, the QR and "
                     "Gauss-Jordan updates, the Hankel series and the Schur LU (refined once in FP64)",
                  2: "f64 (complex128) data; double-float (2xFP32) arithmetic for the dense products, the QR and "
                     "Gauss-Jordan updates, the Hankel series and the Schur LU (refined once in FP64); products with "
                     "k >= 96 on tcgen05 tensor cores from exact bf16 digit planes"}[prec],
        "data": "synthetic", "err_vs_fp64_plain_path": err,
        "config": {"workload": w["name"], "N": n, "omega": omega, "d": d, "angles": n_ang,
                   "bloch_groups": int(np.asarray(w["thetas"]).shape[0]) if np.asarray(w["thetas"]).ndim == 2 else None,
                   "tol": tol, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (factor + precompute %.1f GB resident)" % (info["device_bytes"] / 1e9),
                   "build_s": round(info["build_seconds"], 3), "max_rank": info["max_rank"],
                   "nb_rank": info["nb_rank"], "M": info["m"], "levels": info["levels"],
                   "nb_id_residual": info["nb_residual"], "periodizer_id_residual": info["pid_residual"],
                   "periodizer_ranks": [info["pid_col_rank"], info["pid_row_rank"]],
                   "phases_ms_per_step": phases, "max_flux_error": float(max(flux)),
                   "solve_angles_per_s": round(n_ang / (phases.get("solve:projections", 0) / 1e3 +
                                                       phases.get("solve:schur", 0) / 1e3 +
                                                       phases.get("solve:bragg", 0) / 1e3 + 1e-9), 1)},
        "e2e": {"value": round(whole_job_rate(ws, n_ang, args.steps, e2e_ms), 3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"bound": kbound, "kernel": tname, "achieved": round(achieved, 4), "peak": round(kpeak, 4),
                     "unit": "TFLOP/s", "frac": round(achieved / kpeak, 4),
                     "traffic": measured_traffic(tname),
                     "peak_note": knote + " (of measured)" if kbound == "tensor" else knote,
                     "kernel_time_shares": shares, "kernel_tflops": rates,
                     "kernel_frac": {k: round(r / kernel_peak(k, prec)[1], 4) for k, r in rates.items()}},
        "clocks": clocks,
    }
    return out


def oracle_sample(w, n_sample):
    """Dense oracle on the same obstacle family at a bounded N; returns (fill+solve seconds, parts)."""
    from oracle import qp_dense as qd
    obs, omega, d = w["obstacle"], w["omega"], w["d"]
    th = float(np.asarray(w["thetas"]).ravel()[0])
    x, y, dx, dy = obs.sample(n_sample)
    t0 = time.perf_counter()
    qd.dense_solve(x, y, dx, dy, omega, d, th, qd.Options(m=120, h=0.4, c=2.0, w=2.0))
    return time.perf_counter() - t0


def cpu_baseline(w, n_sample):
    secs = oracle_sample(w, n_sample)
    n = w["N"]
    scale = (n / n_sample) ** 3
    per_angle = secs * scale
    cores = os.cpu_count()
    return {"value": 1.0 / per_angle, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"dense FP64 fill + LAPACK solve of one angle at N={n_sample} (same obstacle, omega="
                      f"{w['omega']}, M=120) took {secs:.2f} s; extrapolated to N={n} by (N/{n_sample})^3 "
                      f"(LU-dominated), i.e. {per_angle:.3g} s per angle"}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    w = workload(args.workload)
    n_sample = 1500 if w["N"] > 1500 else w["N"]
    for _ in range(args.warmup):
        oracle_sample(w, n_sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample(w, n_sample)
    secs = (time.perf_counter() - t0) / args.steps
    n = w["N"]
    value = 1.0 / (secs * (n / n_sample) ** 3)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (complex128)", "data": "synthetic",
            "config": {"workload": w["name"], "N": n, "omega": w["omega"], "sample_N": n_sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"one angle, dense oracle at N={n_sample}, extrapolated by (N/{n_sample})^3"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_gemm(args):
    """Kernel benchmark of hbs_zgemm (C = A B, device complex128, m x n x k) in the chosen
    arithmetic; one JSON line with the FP64-equivalent rate (8 m n k flops per product).  The
    dense products of the precompute (Z = V [P | Y_sel]: 690 x 180 x N at the bench workload)
    have this shape."""
    import torch
    from paper_1301_1247_gb300 import hbs
    m, n, k = args.gemm
    prec = {"fp64": 0, "df": 1, "tc": 2}[args.precision]
    torch.manual_seed(0)
    a = torch.randn(m * k, dtype=torch.complex128, device="cuda")
    b = torch.randn(k * n, dtype=torch.complex128, device="cuda")
    c = torch.zeros(m * n, dtype=torch.complex128, device="cuda")
    for _ in range(max(args.warmup, 1)):
        hbs.zgemm(m, n, k, 1.0, a, m, 0, b, k, 0.0, c, m, prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        hbs.zgemm(m, n, k, 1.0, a, m, 0, b, k, 0.0, c, m, prec)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    return {"metric": "complex GEMM FP64-equivalent rate (hbs_zgemm)", "value": round(8.0 * m * n * k / (ms / 1e3) / 1e12, 3),
            "unit": "TFLOP/s", "ms_per_call": round(ms, 3), "steps": args.steps, "warmup": args.warmup,
            "config": {"m": m, "n": n, "k": k, "precision": args.precision}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="complicated_n100k")
    ap.add_argument("--cpu-sample-n", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true", help="skip the FP64 plain-path accuracy check")
    ap.add_argument("--precision", choices=["fp64", "df", "tc"], default="tc")
    ap.add_argument("--gemm", type=int, nargs=3, metavar=("M", "N", "K"),
                    help="time hbs_zgemm alone at this shape instead of the solver step")
    args = ap.parse_args()
    if args.gemm:
        print(json.dumps(run_gemm(args)))
        return
    ws, rank, local = dist_init()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out))
        return
    out = run_ours(args, ws, rank, local)
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(workload(args.workload), args.cpu_sample_n)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
