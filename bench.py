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
    # kernels whose updates run in double-float on double-float and tensor-precision handles:
    # FP32-pipe instructions per FP64-equivalent flop (a complex multiply-add is 4 error-free
    # multiply-adds of 12 instructions, 48 per 8 flops; the pivoted QR's update, 102 per 16)
    df_per = {"k_zgemm_batched_df": 48.0 / 8.0, "k_pqr": 102.0 / 16.0, "k_cpqr": 102.0 / 16.0,
              "k_schur_solve": 48.0 / 8.0, "k_pgj": 48.0 / 8.0, "k_gj_inverse": 48.0 / 8.0,
              "k_bgj_panel": 48.0 / 8.0}
    if name == "k_zgemm_batched_df" or (prec >= 1 and name in df_per):
        per = df_per[name]
        return ("alu", FP32_INSTR_PEAK / per / 1e12,
                "double-float arithmetic on the FP32 pipes: %.2f FP32-pipe instructions per FP64-equivalent flop "
                "(complex multiply-add = 4 error-free multiply-adds of 12 instructions) at 152 SM x 128 lanes x "
                "2.07 GHz" % per)
    return ("alu", FP64_PEAK_TFLOPS, "FP64 from unit counts x clock (152 SM x 2 DFMA/clk x 2.07 GHz); "
                                      "no FP64 figure in MEASURED_PEAKS.json")

# The algorithmic flop count each kernel's record uses (the survey's per-unit figures).
FLOP_COUNT_NOTE = {
    "k_pqr": "8 m n k per m x n block of rank k (interpolative decomposition; Householder executes ~2x)",
    "k_cpqr": "8 m n k per m x n block of rank k (interpolative decomposition; Householder executes ~2x)",
    "k_pgj": "8 n^3 per n x n block (Gauss-Jordan inverse)",
    "k_zgemm_batched_df": "8 m n k per product",
    "k_zgemm_batched": "8 m n k per product",
    "k_oz_mma": "executed bf16 digit-plane flops on padded tiles",
}

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum averaged over the
# kernel's launches in one step) from ncu captures, per workload, with the digest of the
# sources the kernel is built from at capture time; reported only while they are unchanged.
# A record is either a capture of that workload ("bytes_per_launch") or a capture of a smaller
# one scaled to this workload's launches by their algorithmic bytes ("ratio_to_algorithmic",
# DRAM bytes over algorithmic bytes in the capture), for kernels whose traffic grows with
# their operands (the batched GEMMs).  k_pqr's traffic does not grow in proportion to its
# work (one launch, the periodizer families, dominates it by writing back its trailing
# matrix when the matrices outgrow L2), so its N = 1e4 capture is not scaled.
NCU_TRAFFIC = {
    # profiles/k_pqr_wiggly_n10k.md: all 8 launches of a step at N = 1e4 (24 over 3 steps)
    ("wiggly_n10k", "k_pqr"): {"bytes_per_launch": 4.024e+08, "note": "ncu capture of this workload",
                                "sources": ['paper_1301_1247_gb300/csrc/pqr.cu', 'paper_1301_1247_gb300/csrc/common.cuh', 'paper_1301_1247_gb300/csrc/gridsync.cuh', 'paper_1301_1247_gb300/csrc/dense_kernels.cuh', 'paper_1301_1247_gb300/csrc/dfloat.cuh', 'paper_1301_1247_gb300/csrc/dfcore.cuh', 'paper_1301_1247_gb300/csrc/hankel_table.h', 'paper_1301_1247_gb300/csrc/balance.hpp', 'paper_1301_1247_gb300/csrc/devbuf.hpp'],
                                "digest": "d697f4a8d32a5b40"},
    # profiles/k_zgemm_batched_df_wiggly_n10k.md: all 141 launches of 3 steps at N = 1e4 moved
    # 25.40 MB of DRAM per launch against 37.38 MB of algorithmic bytes per launch (the same
    # command's profiled pass); scaled to the N = 1e5 launches by their algorithmic bytes
    ("complicated_n100k", "k_zgemm_batched_df"): {
        "ratio_to_algorithmic": 0.6795, "scaled_from": "wiggly_n10k",
        "note": "scaled: an ncu capture at N = 1e4 (wiggly_n10k) gave 0.6795 DRAM bytes per algorithmic byte; "
                "times this workload's algorithmic bytes per launch",
        "sources": ['paper_1301_1247_gb300/csrc/zgemm.cuh', 'paper_1301_1247_gb300/csrc/common.cuh', 'paper_1301_1247_gb300/csrc/dfcore.cuh', 'paper_1301_1247_gb300/csrc/dfloat.cuh', 'paper_1301_1247_gb300/csrc/hankel_table.h'],
        "digest": "a70804a592ca9be0"},
}


def _sources_digest(paths):
    import hashlib
    hsh = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()[:16]


def measured_traffic(workload_name, kernel, alg_bytes_per_launch=None):
    """(DRAM bytes per launch, how they were obtained), or (None, why not)."""
    rec = NCU_TRAFFIC.get((workload_name, kernel))
    if rec is None:
        return None, (f"no ncu capture of {kernel} for this workload (profiles/ holds the kernel captures at "
                      "N = 1e4)")
    try:
        if _sources_digest(rec["sources"]) != rec["digest"]:
            return None, f"the ncu capture of {kernel} predates its current sources"
    except OSError:
        return None, "sources of the capture not found"
    if "bytes_per_launch" in rec:
        return rec["bytes_per_launch"], rec["note"]
    if not alg_bytes_per_launch:
        return None, "no algorithmic bytes to scale the capture by"
    return rec["ratio_to_algorithmic"] * alg_bytes_per_launch, rec["note"]


def split_profile(prof, steps):
    """Split hbs.profile_get() records: the per-kernel records, each phase's host wall time
    (ms per step; "phase:<name>") and, per phase, each kernel's device time (ms per step) and
    launches per step ("in:<phase>:<kernel>", phase names themselves hold colons)."""
    kern = {k: v for k, v in prof.items() if not k.startswith(("phase:", "in:"))}
    phases = {k[6:]: round(v["ms"] / steps, 2) for k, v in prof.items() if k.startswith("phase:")}
    by_phase = {}
    for k, v in prof.items():
        if k.startswith("in:"):
            ph, kn = k[3:].rsplit(":", 1)
            by_phase.setdefault(ph, {})[kn] = {"ms": round(v["ms"] / steps, 3), "launches": v["launches"] / steps}
    return kern, phases, by_phase


def workload(name):
    if name == "complicated_n100k":
        w = inputs.workload_complicated_n100k()
    elif name == "wiggly_n10k":
        w = inputs.workload_wiggly_n10k()
    elif name == "star_n400":
        w = inputs.workload_star_n400()
    elif name == "transmission_n10k":
        w = inputs.workload_transmission_n10k()
    else:
        raise SystemExit(f"unknown workload {name}")
    w["name"] = name
    return w


def workload_config(w, ws):
    """The `config` object of both arms: the workload by name and size."""
    th = np.asarray(w["thetas"])
    extra = {"problem": "transmission", "index": w["index"]} if w.get("index") else {}
    return {"workload": w["name"], **extra, "N": w["N"], "omega": w["omega"], "d": w["d"], "angles": int(th.size),
            "bloch_groups": int(th.shape[0]) if th.ndim == 2 else None, "tol": 1e-12,
            "parallelism": f"replicas x{ws}",
            "l2": "inputs larger than L2 (the resident factor and precompute are several GB)"}


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
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region.
    `gpu` is the nvidia-smi id (UUID preferred) of the GPU being timed."""

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


def _gpu_id_for_smi(local):
    """The nvidia-smi id of CUDA device `local`: its UUID, which does not depend on
    CUDA_VISIBLE_DEVICES (nvidia-smi numbers all GPUs of the host); the ordinal otherwise."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:  # noqa: BLE001 - older torch without .uuid
        pass
    return str(local)


def wood_group_angles(omega, d, q, order=3):
    """q angles sharing the Bloch phase of an exact Rayleigh-Wood anomaly (Sec. 2.4):
    cos(theta_j) = 1 - 2 pi (order + j) / (omega d), all of them anomalies of that phase."""
    c = 1.0 - 2.0 * math.pi * (order + np.arange(q)) / (omega * d)
    return -np.arccos(c[c > -1.0])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def tuned_shapes():
    """The autotuner's choices (key -> [variant, ms]) from its file, if any."""
    path = os.environ.get("HBS_TUNE_FILE")
    out = {}
    if path and os.path.exists(path):
        for line in open(path):
            f = line.split()
            if len(f) == 3:
                out[f[0]] = [int(f[1]), float(f[2])]
    return out


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
    index = float(w.get("index", 0.0))  # > 0: the transmission problem (Sec. 5)
    opts = hbs.default_options(precision=prec, index=index)

    def step(device_inputs: bool):
        if device_inputs:
            h = hbs.Handle(gx, gy, gdx, gdy, d, omega, tol, opts, stream=stream)
        else:
            h = hbs.Handle(hx.numpy(), hy.numpy(), hdx.numpy(), hdy.numpy(), d, omega, tol, opts, stream=stream)
        r = h.solve(hth.numpy(), stream=stream)
        amps = [r.bragg(i) for i in range(len(thetas))]
        return h, r, amps

    def timed(fn, steps):
        """Device time (ms) of `steps` calls of fn on the launching stream, synchronized on both sides."""
        barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = None
        for _ in range(steps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        return e0.elapsed_time(e1), out

    info = None
    for _ in range(args.warmup):
        h, r, amps = step(True)
        info = h.info()
        del h, r
    torch.cuda.synchronize()

    # ---- the headline: device-resident inputs, no per-kernel profiling in the timed region
    hbs.profile_enable(False)
    l0 = hbs.launch_count()
    with ClockSampler(_gpu_id_for_smi(local)) as clk:
        ms, (h, r, amps) = timed(lambda: step(True), args.steps)
    if info is None:
        info = h.info()
    del h, r
    launches = hbs.launch_count() - l0
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, ws)

    # ---- end to end: host inputs, copies and read-back inside the timed region
    t0 = time.perf_counter()
    e2e_dev_ms, _ = timed(lambda: step(False), args.steps)
    e2e_ms = max_over_ranks(max(e2e_dev_ms, 1e3 * (time.perf_counter() - t0)), ws)
    flux = [a[3] for a in amps]

    # ---- a separate profiled pass of the same steps: per-kernel event pairs on the launching
    # stream give the kernel shares and the dominant kernel's rate (the library's phase
    # timers synchronize, so this pass runs slower than the headline and is not it)
    hbs.profile_reset()
    hbs.profile_enable(True)
    prof_ms, _ = timed(lambda: step(True)[0], args.steps)
    hbs.profile_enable(False)
    prof = hbs.profile_get()

    n_ang = len(thetas)
    th2 = np.asarray(w["thetas"])
    n_groups = th2.shape[0] if th2.ndim == 2 else 1
    fp64 = None
    err = None
    if not args.no_check and th2.ndim == 2:
        # ---- the all-FP64 baselines on this GPU (outside the timed regions):
        #  * plain path: the paper's per-phase count of q + 2M + 2l applies of an FP64-built
        #    compressed inverse (Remarks 3.1, 3.2), timed on four groups, extrapolated to all;
        #  * FP64 precomputed path: the same library path as the headline, every step in FP64.
        torch.cuda.synchronize()
        t_b = time.perf_counter()
        h64 = hbs.Handle(gx, gy, gdx, gdy, d, omega, tol, hbs.default_options(precision=0, index=index),
                         stream=stream)
        torch.cuda.synchronize()
        build64_s = time.perf_counter() - t_b
        gflux = [max(flux[g * th2.shape[1]:(g + 1) * th2.shape[1]]) for g in range(n_groups)]
        picks = [0, n_groups // 2, n_groups - 1]
        for g in np.argsort(gflux)[::-1]:
            if int(g) not in picks:
                picks.append(int(g))
                break
        sel = np.concatenate([th2[g] for g in picks])
        plain_ms, ref = timed(lambda: h64.solve_plain(sel, stream=stream), 1)
        per_group_s = plain_ms / 1e3 / len(picks)
        pre64_ms, _ = timed(lambda: [h64.solve(thetas, stream=stream)], 1)
        per_group = {}
        for gi, g in enumerate(picks):
            e = 0.0
            for j in range(th2.shape[1]):
                k = g * th2.shape[1] + j
                _, c1, d1, _ = amps[k]
                _, c2, d2, _ = ref.bragg(gi * th2.shape[1] + j)
                e = max(e, _rel(np.concatenate([c1, d1]), np.concatenate([c2, d2])))
            per_group[f"group_{g}"] = e
        # a group at an exact Wood's anomaly, solved by the benchmarked handle and the plain path
        wth = wood_group_angles(omega, d, th2.shape[1])
        hb = hbs.Handle(gx, gy, gdx, gdy, d, omega, tol, opts, stream=stream)
        ra, rb = hb.solve(wth, stream=stream), h64.solve_plain(wth, stream=stream)
        e = 0.0
        for j in range(len(wth)):
            _, c1, d1, _ = ra.bragg(j)
            _, c2, d2, _ = rb.bragg(j)
            e = max(e, _rel(np.concatenate([c1, d1]), np.concatenate([c2, d2])))
        per_group["wood_anomaly_group"] = e
        err = {"max": max(per_group.values()), "per_group": per_group,
               "groups": "first, middle, last, worst-flux group of the workload, and one group of "
                         f"{len(wth)} angles at an exact Wood's anomaly (nw={ra.angle_info(0)[0]})"}
        plain_rate = n_ang / (build64_s + n_groups * per_group_s)
        pre64_rate = n_ang / (build64_s + pre64_ms / 1e3)
        value_now = whole_job_rate(1, n_ang, args.steps, ms)
        fp64 = {
            "plain_path_angles_per_s": round(plain_rate, 3),
            "plain_path": f"FP64 build {build64_s:.3f} s + {per_group_s:.3f} s per Bloch group of the paper's "
                          f"q + 2M + 2l applies (timed on {len(picks)} of {n_groups} groups, extrapolated to all)",
            "speedup_vs_fp64_plain": round(value_now / plain_rate, 2),
            "precomputed_path_angles_per_s": round(pre64_rate, 3),
            "precomputed_path": f"FP64 build {build64_s:.3f} s + {pre64_ms / 1e3:.3f} s to solve all {n_ang} angles "
                                "(the headline's path with every step in FP64; one step)",
            "speedup_vs_fp64_precomputed": round(value_now / pre64_rate, 2),
        }
        del h64, ref, hb, ra, rb

    value = whole_job_rate(ws, n_ang, args.steps, ms_max)
    kern, phases, by_phase = split_profile(prof, args.steps)
    if args.phase_kernels:
        with open(args.phase_kernels, "w") as f:
            json.dump({"phases_ms_per_step": phases, "kernels_by_phase": by_phase}, f, indent=1, sort_keys=True)
    top = max(kern.items(), key=lambda kv: kv[1]["ms"])
    tname, tv = top
    achieved = tv["flops"] / (tv["ms"] / 1e3) / 1e12 if tv["ms"] > 0 else 0.0
    kbound, kpeak, knote = kernel_peak(tname, prec)
    shares = {k: round(v["ms"] / sum(x["ms"] for x in kern.values()), 4) for k, v in
              sorted(kern.items(), key=lambda kv: -kv[1]["ms"])[:8]}
    # algorithmic FP64(-equivalent) rate of the top kernels that record flops
    rates = {k: round(v["flops"] / (v["ms"] / 1e3) / 1e12, 4) for k, v in
             sorted(kern.items(), key=lambda kv: -kv[1]["ms"])[:8] if v["flops"] > 0 and v["ms"] > 0}
    peaks_hbm = MEASURED_PEAKS.get("hbm_gbs", 6800.0)
    # HBM: a lower bound on the DRAM bytes of a step (every byte of the resident factor and
    # precompute written once and read once, plus the inputs and outputs) against its time
    hbm_bytes = 2.0 * info["device_bytes"] + 4 * n * 8 + n_ang * (8 + 64 * 16)
    hbm_gbs = hbm_bytes / (ms / args.steps / 1e3) / 1e9
    h2d = 4 * n * 8 + n_ang * 8
    n_orders = sum(len(a[1]) for a in amps)
    d2h = n_orders * 2 * 16 + n_ang * 8
    alg_b = tv["bytes"] / max(tv["launches"], 1)
    traffic_b, traffic_note = measured_traffic(w["name"], tname, alg_b)
    if traffic_b is not None:
        traffic_b = round(traffic_b, -3)
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
        "data": "synthetic", "err_vs_fp64_plain_path": err["max"] if err else None,
        "err_vs_fp64_plain_path_detail": err,
        "fp64_baselines": fp64,
        "config": workload_config(w, ws),
        "details": {"resident_gb": round(info["device_bytes"] / 1e9, 2),
                   "build_s": round(info["build_seconds"], 3), "max_rank": info["max_rank"],
                   "nb_rank": info["nb_rank"], "M": info["m"], "levels": info["levels"],
                   "nb_id_residual": info["nb_residual"], "periodizer_id_residual": info["pid_residual"],
                   "periodizer_ranks": [info["pid_col_rank"], info["pid_row_rank"]],
                   "profiled_pass_ms_per_step": round(prof_ms / args.steps, 2),
                   "autotuned_shapes": tuned_shapes(),
                   "phases_ms_per_step": phases, "max_flux_error": float(max(flux))},
        "e2e": {"value": round(whole_job_rate(ws, n_ang, args.steps, e2e_ms), 3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"bound": kbound, "kernel": tname, "achieved": round(achieved, 4), "peak": round(kpeak, 4),
                     "unit": "TFLOP/s", "frac": round(achieved / kpeak, 4),
                     "traffic": traffic_b,
                     "traffic_note": traffic_note,
                     "algorithmic_bytes_per_launch": round(tv["bytes"] / max(tv["launches"], 1), 1) or None,
                     "flop_count": FLOP_COUNT_NOTE.get(tname, "as recorded by the library"),
                     "peak_note": knote + " (of measured)" if kbound == "tensor" else knote,
                     "timed_in": "separate profiled pass of the same steps (per-launch CUDA events on the launching "
                                 "stream)",
                     "kernel_time_shares": shares, "kernel_tflops": rates,
                     "kernel_algorithmic_bytes_per_launch": {
                         k: round(v["bytes"] / max(v["launches"], 1), 1) for k, v in
                         sorted(kern.items(), key=lambda kv: -kv[1]["ms"])[:8] if v["bytes"] > 0},
                     "kernel_frac": {k: round(r / kernel_peak(k, prec)[1], 4) for k, r in rates.items()},
                     "hbm": {"bytes_per_step_lower_bound": hbm_bytes, "achieved_gbs": round(hbm_gbs, 2),
                             "peak_gbs": peaks_hbm, "frac": round(hbm_gbs / peaks_hbm, 5),
                             "note": "every resident byte (factor + precompute) written once and read once per "
                                     "step, plus inputs and outputs; of measured"}},
        "clocks": clocks,
    }
    return out


def oracle_sample(w, n_sample):
    """One dense oracle solve (one angle) on the workload's obstacle at a bounded N, with the
    oracle's own discretization readings (contour, Bragg sampling).  Returns (seconds to fill
    A and its images, seconds for the rest of the angle: periodizer blocks, LAPACK solve,
    Bragg extraction, size of the dense system)."""
    from oracle import qp_dense as qd
    from oracle import readings as rd
    obs, omega, d = w["obstacle"], w["omega"], w["d"]
    th = float(np.asarray(w["thetas"]).ravel()[0])
    x, y, dx, dy = obs.sample(n_sample)
    opts = rd.options(x, y, omega, d, th)
    index = w.get("index", 0.0)
    t0 = time.perf_counter()
    if index:  # the transmission oracle (Sec. 5): 2 N unknowns
        from oracle import transmission as tr
        blocks = tr.obstacle_blocks(x, y, dx, dy, omega, index, d)
        t1 = time.perf_counter()
        tr.dense_solve(x, y, dx, dy, omega, index, d, th, opts, blocks)
    else:
        blocks = qd.obstacle_blocks(x, y, dx, dy, omega, d)
        t1 = time.perf_counter()
        qd.dense_solve(x, y, dx, dy, omega, d, th, opts, blocks)
    t2 = time.perf_counter()
    size = (2 if index else 1) * n_sample + 2 * opts.m
    # the LAPACK factorization inside that solve, timed alone on a matrix of the same size, so
    # that the extrapolation scales it (size^3) apart from the rest of the angle (linear in N)
    import scipy.linalg
    rng = np.random.default_rng(0)
    a = rng.standard_normal((size, size)) + 1j * rng.standard_normal((size, size))
    t3 = time.perf_counter()
    scipy.linalg.lu_factor(a, overwrite_a=True, check_finite=False)
    lu_s = time.perf_counter() - t3
    return t1 - t0, t2 - t1, min(lu_s, t2 - t1), size


def oracle_step_seconds(w, n_sample, fill_s, solve_s, lu_s, size):
    """The oracle's time for one bench step (build + every angle) at the workload's N,
    extrapolated from a sample: the fill of A and its images grows as N^2 and is done once;
    each angle refills the periodizer blocks and samples (linear in N) and factors the dense
    system (LU, size^3)."""
    n, n_ang = w["N"], int(np.asarray(w["thetas"]).size)
    u = 2 if w.get("index") else 1  # unknowns per node
    m2 = size - u * n_sample
    fill = fill_s * (n / n_sample) ** 2
    per_angle = (solve_s - lu_s) * (n / n_sample) + lu_s * ((u * n + m2) / size) ** 3
    return fill + n_ang * per_angle, fill, per_angle


def cpu_baseline(w, sizes):
    rows = []
    for ns in sizes:
        f, s, lu, sz = oracle_sample(w, ns)
        rows.append({"N": ns, "system": sz, "fill_s": round(f, 3), "solve_s": round(s, 3), "lu_s": round(lu, 3)})
    last = rows[-1]
    step_s, fill, per_angle = oracle_step_seconds(w, last["N"], last["fill_s"], last["solve_s"], last["lu_s"],
                                                  last["system"])
    n_ang = int(np.asarray(w["thetas"]).size)
    return {"value": n_ang / step_s, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"dense FP64 oracle (fill of A and images, then per angle the periodizer blocks, LAPACK "
                      f"solve and Bragg extraction; M from the oracle's contour reading) timed at N in "
                      f"{[r['N'] for r in rows]}: {rows} (lu_s: the LAPACK factorization of that size timed "
                      f"alone); extrapolated to N={w['N']} from the largest: fill x N^2 = {fill:.3g} s once, "
                      f"per angle (solve - lu) x N + lu x system^3 = {per_angle:.3g} s, {n_ang} angles. Fill is "
                      f"single-threaded (SciPy Hankel), the factorization uses all cores (OpenBLAS)."}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    w = workload(args.workload)
    n_sample = 1500 if w["N"] > 1500 else w["N"]
    for _ in range(args.warmup):
        oracle_sample(w, n_sample)
    tt = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        f, s, lu, sz = oracle_sample(w, n_sample)
        tt.append((time.perf_counter() - t0, f, s, lu, sz))
    f = sum(t[1] for t in tt) / len(tt)
    s = sum(t[2] for t in tt) / len(tt)
    lu = sum(t[3] for t in tt) / len(tt)
    step_s, _, _ = oracle_step_seconds(w, n_sample, f, s, lu, tt[0][4])
    n_ang = int(np.asarray(w["thetas"]).size)
    value = n_ang / step_s
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (complex128)", "data": "synthetic",
            "config": workload_config(w, ws),
            "details": {"sample_N": n_sample, "sample_s_per_step": sum(t[0] for t in tt) / len(tt)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: one angle of the dense oracle at N={n_sample} (fill {f:.2f} s, "
                                       f"solve {s:.2f} s of which LAPACK factorization {lu:.2f} s); the step at "
                                       f"N={w['N']} extrapolated (fill x N^2 once; per angle (solve - lu) x N + "
                                       f"lu x system^3; {n_ang} angles)"},
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


def run_batch(args, ws, local):
    """Many gratings (config 3): one step = hbs_build_batch of all gratings (every tree level
    of every solver in the same launches) + hbs_solve of each grating's angles.  value =
    angles per second of step time."""
    import torch
    from paper_1301_1247_gb300 import hbs
    torch.cuda.set_device(local)
    w = inputs.workload_batch()
    geoms = [x["obstacle"].sample(x["N"]) for x in w]
    omegas = [x["omega"] for x in w]
    thetas = [np.asarray(x["thetas"], dtype=np.float64) for x in w]
    n_ang = int(sum(len(t) for t in thetas))
    stream = torch.cuda.current_stream()
    opts = hbs.default_options(precision={"fp64": 0, "df": 1, "tc": 2}[args.precision])

    def step():
        hs = hbs.build_batch(geoms, omegas, 1.0, 1e-12, opts, stream=stream)
        t_b = time.perf_counter()
        rs = [h.solve(t, stream=stream) for h, t in zip(hs, thetas)]
        flux = max(r.bragg(i)[3] for r, t in zip(rs, thetas) for i in range(len(t)))
        return hs, rs, t_b, flux

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    l0 = hbs.launch_count()
    with ClockSampler(_gpu_id_for_smi(local)) as clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        build_s = 0.0
        flux = 0.0
        for _ in range(args.steps):
            tb0 = time.perf_counter()
            hs, rs, t_b, f = step()
            build_s += t_b - tb0
            flux = max(flux, f)
            del hs, rs
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(ws)
    ms = max_over_ranks(max(e0.elapsed_time(e1), 1e3 * wall), ws)
    ns = np.array([x["N"] for x in w])
    return {"metric": "many gratings: build s + incident angles/s (256 gratings, N log-uniform in [400, 2e4])",
            "value": round(whole_job_rate(ws, n_ang, args.steps, ms), 2), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "dtype": args.precision,
            "config": {"workload": "batch_256", "gratings": len(w), "N_range": [int(ns.min()), int(ns.max())],
                       "N_total": int(ns.sum()), "omega_range": [5.0, 40.0], "angles": n_ang,
                       "parallelism": f"replicas x{ws}"},
            "details": {"build_s_per_step": round(build_s / args.steps, 4), "max_flux_error": float(flux)},
            "gpu_launches": int(hbs.launch_count() - l0), "clocks": clk.summary()}


def run_serving(args, local):
    """Serving (config 5): 32 resident solvers (N log-uniform in [2e3, 1e5], omega in [10, 60]);
    a Poisson stream of single-angle requests, 10 % exactly at Wood's anomalies, submitted by a
    client thread at their arrival times and batched by the library's request loop (batches
    form per geometry while others run; each batch is solved by Bloch phase).  value = solves
    per second from the first arrival to the last completion; p50/p99 latency from submission
    to completion."""
    import threading

    import torch
    from paper_1301_1247_gb300 import hbs
    torch.cuda.set_device(local)
    w = inputs.workload_serving()
    geoms = [x["obstacle"].sample(x["N"]) for x in w]
    omegas = [x["omega"] for x in w]
    opts = hbs.default_options(precision={"fp64": 0, "df": 1, "tc": 2}[args.precision])
    t0 = time.perf_counter()
    handles = [hbs.Handle(*g, 1.0, om, 1e-12, opts) for g, om in zip(geoms, omegas)]
    build_s = time.perf_counter() - t0
    resident = sum(h.info()["device_bytes"] for h in handles)
    sv = hbs.Server(hbm_budget_bytes=int(resident * 1.05), slots=args.slots, max_batch=256)
    gids = [sv.add(h) for h in handles]
    # warm-up requests (not counted): one per geometry
    for rid in [sv.submit(g, -1.0) for g in gids]:
        sv.wait(rid, 600.0)
    sv.close()  # the server does not own the solvers; a fresh one starts the measured stream
    times, gi, th = inputs.request_stream(5, args.requests, args.rate, omegas)
    sv2 = hbs.Server(hbm_budget_bytes=int(resident * 1.05), slots=args.slots, max_batch=256)
    gids = [sv2.add(h) for h in handles]
    rids = []

    def client():
        start = time.perf_counter()
        for t, g, a in zip(times, gi, th):
            dt = start + t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            rids.append(sv2.submit(gids[int(g)], float(a)))

    l0 = hbs.launch_count()
    with ClockSampler(_gpu_id_for_smi(local)) as clk:
        t_start = time.perf_counter()
        c = threading.Thread(target=client)
        c.start()
        c.join()
        worst_flux = 0.0
        for r in rids:
            worst_flux = max(worst_flux, sv2.wait(r, 600.0)[3])
        span = time.perf_counter() - t_start
    st = sv2.stats()
    return {"metric": "serving: solves/s with p50/p99 latency over 32 resident geometries (N 2e3-1e5, omega 10-60)",
            "value": round(len(rids) / span, 2), "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "dtype": args.precision,
            "p50_latency_ms": round(1e3 * st["p50_latency_s"], 3), "p99_latency_ms": round(1e3 * st["p99_latency_s"], 3),
            "max_latency_ms": round(1e3 * st["max_latency_s"], 3),
            "config": {"workload": "serving_32", "geometries": len(w), "N_range": [min(x["N"] for x in w),
                                                                                   max(x["N"] for x in w)],
                       "omega_range": [10.0, 60.0], "requests": len(rids), "arrival_rate_per_s": args.rate,
                       "wood_fraction": 0.1, "slots": args.slots},
            "details": {"build_s_all": round(build_s, 3), "resident_gb": round(resident / 1e9, 2),
                        "batches": st["batches"], "mean_batch": round(st["mean_batch"], 2),
                        "library_solves_per_s": round(st["solves_per_s"], 2), "max_flux_error": float(worst_flux)},
            "gpu_launches": int(hbs.launch_count() - l0), "clocks": clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="complicated_n100k",
                    help="complicated_n100k (the headline), wiggly_n10k, star_n400, or transmission_n10k "
                         "(dielectric obstacles, Sec. 6.3)")
    ap.add_argument("--cpu-sample-n", type=int, nargs="+", default=[400, 1000, 2000])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true", help="skip the FP64 plain-path accuracy check")
    ap.add_argument("--phase-kernels", metavar="PATH",
                    help="write the profiled pass's device time per phase and kernel (ms per step) as JSON")
    ap.add_argument("--precision", choices=["fp64", "df", "tc"], default="tc")
    ap.add_argument("--mode", choices=["solver", "batch", "serving"], default="solver",
                    help="solver: the headline step; batch: many gratings built at once; serving: request loop")
    ap.add_argument("--requests", type=int, default=6000, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=3000.0, help="serving: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=4, help="serving: concurrent batches")
    ap.add_argument("--gemm", type=int, nargs=3, metavar=("M", "N", "K"),
                    help="time hbs_zgemm alone at this shape instead of the solver step")
    args = ap.parse_args()
    if not args.no_autotune:
        # the launch-shape autotuner times the candidate shapes during the warm-up steps
        os.environ["HBS_AUTOTUNE"] = "1"
        if not os.environ.get("HBS_TUNE_FILE"):
            os.environ["HBS_TUNE_FILE"] = os.path.join(tempfile.gettempdir(),
                                                       f"hbsqp_tune_{os.getpid()}_{os.environ.get('RANK', '0')}.txt")
    if args.gemm:
        print(json.dumps(run_gemm(args)))
        return
    ws, rank, local = dist_init()
    if args.impl == "ours" and args.mode == "batch":
        out = run_batch(args, ws, local)
        if rank == 0:
            print(json.dumps(out))
        return
    if args.impl == "ours" and args.mode == "serving":
        print(json.dumps(run_serving(args, local)))
        return
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
