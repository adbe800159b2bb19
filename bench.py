#!/usr/bin/env python
"""Benchmark of the Laguerre-transform acoustic solver (one JSON line on stdout, rank 0).

Workload (default): the 2048 x 1024 random layered acoustic model (5 m spacing, 20 layers with
+-5 % node perturbation, Gardner density, Ricker 25 Hz source at (1024, 16), h = 200, alpha = 9,
512 harmonics), FP64 path, one shot.  A step is one Laguerre harmonic of the shot: right-hand side
of Eq. 9, the preconditioned CG solve to 1e-10 (stencil matvec, vector updates, preconditioner =
DST-I along x, partitioned tridiagonal solves along z, DST-I back), the history update and the
receiver gather.  The metric is harmonic-solves/s.  Extra keys report the same workload on the
mixed-precision path and the standalone preconditioner (1024 modes x nz 1024 x 512 RHS).

--impl reference times the CPU oracle (numpy/scipy float64) on the same workload and metric.
With --gpus N > 1 (torchrun) every rank runs its own replica shot (source shifted along the
surface line): scaling is weak, there is no data-path collective.
"""
import argparse
import ctypes as C
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

METRIC = "Laguerre-harmonic solves/s at 1e-8 rel err vs plain FP64 GPU; p50/p99 latency"
UNIT = "harmonic-solves/s"
WORKLOAD = ("random_layered_2048x1024 acoustic FP64 single shot: 5 m, 20 layers c~U(1500,4500)x(1+eps), "
            "rho=310c^0.25, Ricker 25 Hz at (1024,16), h=200, alpha=9, 512 harmonics, PCG tol 1e-10; "
            "step = one harmonic")

# dram__bytes_read.sum + dram__bytes_write.sum per launch from ncu captures, with the sha1 of the
# kernel source file at capture time (null when the kernel changed since).  See profiles/.
NCU_TRAFFIC = {
    # oz_pack_a_kernel<8, 7> (16.83 MB) + oz_gemm_kernel<8, 7> (58.85 MB), one 2048-mode x 1024-row
    # launch each (bench.py --capture-kernels; profiles/launches_dst_f64_random_layered_2048x1024.md)
    "dst_f64_oz": {"bytes": 75.68e6, "sha1": "78396d00351a",
                   "section": "// ============================================================================ exact-slice FP64 DST"},
}


def sha1_of(path):
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def section_sha1(path, marker):
    """sha1 of the source from the line holding `marker` to the end of the file (the kernels the
    counters were taken on; edits elsewhere in the file do not void them)."""
    with open(path, "rb") as f:
        data = f.read()
    i = data.find(marker.encode())
    return hashlib.sha1(data[i:] if i >= 0 else data).hexdigest()[:12]


def traffic_for(kernel_file, key):
    rec = NCU_TRAFFIC.get(key)
    if not rec:
        return None
    path = os.path.join(ROOT, "paper_1005_0542_gb300", "csrc", kernel_file)
    digest = section_sha1(path, rec["section"]) if "section" in rec else sha1_of(path)
    if digest != rec["sha1"]:
        return None
    return rec["bytes"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# The metric's accuracy gate: the first ACC_HARM harmonics of every leg (fields at every node)
# against the oracle's fields, the oracle solving to ACC_TOL (two solutions that each meet
# ||r|| <= tol ||b|| differ by up to cond(A) tol, so the reference is solved well below the legs'
# 1e-10); relative L2 at most GATE (the float64 legs are flagged against 1e-10 as well).
ACC_HARM = 2
ACC_TOL = 1e-13
GATE = 1e-8
GATE64 = 1e-10


def shot_fields(ctx, sh, nsrc, ncomp, shape, picks):
    """Host copies of the current harmonic's fields of the sources `picks` of a shot."""
    import torch
    from paper_1005_0542_gb300 import lagwave as L
    buf = torch.empty((nsrc, ncomp) + tuple(shape), dtype=torch.float64, device="cuda")
    L.check(L.lag_shot_copy_field(sh, C.c_void_p(buf.data_ptr())), ctx)
    torch.cuda.synchronize()
    out = [buf[i].cpu().numpy().copy() for i in picks]
    del buf
    return [o[0] if ncomp == 1 else o for o in out]


class OracleRefs:
    """Oracle solutions of the benchmark's problems, computed on demand (CPU, float64)."""

    def __init__(self, s):
        self.s = s
        self.cache = {}
        self.seconds = 0.0

    def _fm(self, s, wavelet="ricker"):
        from oracle import laguerre
        if wavelet == "paper":
            fun, t_end = laguerre.paper_wavelet(s.f0, s.t0, 4.0), s.t0 + 8.0 / s.f0
        else:
            fun, t_end = laguerre.ricker(s.f0, s.t0), s.t0 + 4.0 / s.f0
        # the coefficients of the whole series, as the shot computes them, then the first few
        return laguerre.forward_coeffs(fun, s.n_harm, s.h, s.alpha, t_end)[:ACC_HARM]

    def cartesian(self, src=None, free_surface=False):
        from oracle import solve
        s = self.s
        src = tuple(src or s.sources[0])
        key = ("cart", src, free_surface)
        if key not in self.cache:
            t0 = time.perf_counter()
            out = solve.acoustic_shot(s.c, s.rho, s.hx, s.hz, s.h, s.alpha, ACC_HARM, src, s.receivers[:1],
                                      s.t_out[:2], s.f0, s.t0, tol=ACC_TOL, keep_fields=True, fm=self._fm(s),
                                      free_surface=free_surface)
            self.seconds += time.perf_counter() - t0
            self.cache[key] = out["fields"]
        return self.cache[key]

    def cylindrical(self, s):
        from oracle import cyl
        key = ("cyl", s.name)
        if key not in self.cache:
            t0 = time.perf_counter()
            out = cyl.acoustic_shot(s.c, s.rho, s.hx, s.hz, s.h, s.alpha, ACC_HARM, s.sources[0], s.receivers[:1],
                                    s.t_out[:2], s.f0, s.t0, tol=ACC_TOL, keep_fields=True,
                                    fm=self._fm(s, "paper"), wavelet="paper")
            self.seconds += time.perf_counter() - t0
            self.cache[key] = out["fields"]
        return self.cache[key]

    def elastic_residual(self, s, fields, srcs):
        """||b - C R_0|| / ||b|| with the oracle's plane-strain operator for harmonic 0 (no history)."""
        from oracle import fd, solve
        t0 = time.perf_counter()
        lam, mu = solve.elastic_lame(s.c, s.vs, s.rho)
        f0m = self._fm(s)[0]
        res = []
        for R, (ix, iz) in zip(fields, srcs):
            cu, cw = fd.apply_C(R[0], R[1], lam, mu, s.rho, s.h, s.hx, s.hz)
            bz = f0m / (s.hx * s.hz)
            cw[iz, ix] -= bz
            res.append(float(np.sqrt(np.sum(cu * cu) + np.sum(cw * cw)) / abs(bz)))
        self.seconds += time.perf_counter() - t0
        return res

    def cyl_elastic_residual(self, s, R):
        """The same for the axisymmetric elastic operator (vertical force on the axis)."""
        from oracle import cyl_elastic, solve
        t0 = time.perf_counter()
        lam, mu = solve.elastic_lame(s.c, s.vs, s.rho)
        co = cyl_elastic.coefficients(lam, mu, s.hx, s.hz)
        cq, cu = cyl_elastic.apply_C(R[0], R[1], co, s.rho, s.h, s.hx, s.hz)
        ir, iz = s.sources[0]
        b = self._fm(s, "paper")[0] / (2.0 * np.pi * s.hx * s.hz)
        cu[ir, iz] -= b
        self.seconds += time.perf_counter() - t0
        return float(np.sqrt(np.sum(cq * cq) + np.sum(cu * cu)) / abs(b))


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def accuracy_report(acc, refs):
    """Every leg's first harmonics against the oracle: relative L2 over every node."""
    rep = {"gate": GATE, "harmonics": list(range(ACC_HARM)), "oracle_tol": ACC_TOL,
           "measure": ("relative L2 error over every node of each harmonic's field R_m, the leg's own shot "
                       "(its warm-up harmonics, solved at the leg's tolerance 1e-10) against the oracle's "
                       "field (PCG to 1e-13); elastic legs: the oracle operator's relative residual "
                       "||b - C R_0|| / ||b|| of harmonic 0 (the 4096 x 2048 elastic oracle solve does not fit "
                       "the bench's time)")}
    ok = True
    for leg, item in acc.items():
        kind, fields = item[0], item[1]
        try:
            if kind in ("cart", "cart_fs", "cart_src", "cyl"):
                if kind == "cyl":
                    ref = refs.cylindrical(item[2])
                elif kind == "cart_src":
                    ref = refs.cartesian(src=item[2])
                else:
                    ref = refs.cartesian(free_surface=(kind == "cart_fs"))
                errs = [_rel_l2(f, r) for f, r in zip(fields, ref)]
                e = {"rel_l2": errs, "max": max(errs), "pass": max(errs) <= GATE}
                if leg in ("headline_fp64", "layered", "free_surface") or leg.endswith("_fp64"):
                    e["pass_1e-10"] = max(errs) <= GATE64
            elif kind == "cart_elastic":
                res = refs.elastic_residual(item[2], fields, item[3])
                e = {"oracle_operator_residual": res, "max": max(res), "pass": max(res) <= 2e-10,
                     "solver_tol": 1e-10}
            elif kind == "cyl_elastic":
                res = refs.cyl_elastic_residual(item[2], fields[0])
                e = {"oracle_operator_residual": [res], "max": res, "pass": res <= 2e-10, "solver_tol": 1e-10}
            else:
                raise ValueError(f"unknown accuracy entry kind {kind!r}")
        except Exception as exc:  # a failed reference is reported, not hidden
            e = {"error": f"{type(exc).__name__}: {exc}", "pass": False}
        ok = ok and e["pass"]
        rep[leg] = e
    rep["all_pass"] = ok
    rep["oracle_seconds"] = refs.seconds
    return rep


# FP64 ALU peak derived from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz
# (1.25 TFLOP/s nominal; the DFMA probe measured 1.20 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.path is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------- GPU arm
def gpu_arm(args, rank, world, local_rank):
    import torch
    from paper_1005_0542_gb300 import inputs
    from paper_1005_0542_gb300 import lagwave as L
    from paper_1005_0542_gb300.replicas import replica_source, whole_job_rate

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    ctx = L.create(local_rank, stream=torch.cuda.current_stream().cuda_stream)
    s = inputs.random_layered()
    if world > 1:  # replica r: its own source on the same row
        s.sources = [replica_source(s.sources[0], rank, s.nx)]
    peaks, peak_src = load_peaks()

    def make_shot(prec, n_harm=None, tune=0, free_surface=False, layered=0):
        g = L.grid(s.nx, s.nz, s.hx, s.hz, free_surface)
        lag = L.laguerre(s.h, s.alpha, n_harm or s.n_harm)
        sv = L.solver(tol=s.tol, prec=prec, tune=tune, layered=layered)
        w = L.wavelet(s.f0, s.t0)
        c_, pc = L.f64(s.c)
        r_, pr = L.f64(s.rho)
        t_, pt = L.f64(s.t_out)
        sh = C.c_void_p()
        L.check(L.lag_shot_create(ctx, C.byref(g), pc, None, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                                  L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                                  C.byref(sh)), ctx)
        return sh

    def timed_steps(sh, W, K, keep=None):
        """W warm-up harmonics, then the timed region: K harmonics in the production configuration
        (each harmonic's PCG solve is one graph launch).  Then the kernel-class times: the next K
        harmonics of the same shot with a CUDA event pair per launch on the shot's stream (a graph
        cannot bracket its kernels with events, so this pass launches eagerly; it is not timed).
        keep (a list): the fields of the first ACC_HARM warm-up harmonics are appended to it."""
        for m in range(W):
            L.check(L.lag_shot_step(sh, 1), ctx, ok=(L.LAG_OK,))
            if keep is not None and m < ACC_HARM:
                keep.append(shot_fields(ctx, sh, 1, 1, s.c.shape, [0])[0])
        stream = torch.cuda.ExternalStream(L.lag_shot_stream(sh))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = L.lag_kernel_launches(ctx)
        e0.record(stream)
        for _ in range(K):
            L.check(L.lag_shot_step(sh, 1), ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        launches = L.lag_kernel_launches(ctx) - l0
        ms = e0.elapsed_time(e1)
        L.lag_profile_enable(ctx, 1)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(K):
            L.check(L.lag_shot_step(sh, 1), ctx)
        p1.record(stream)
        torch.cuda.synchronize()
        nk = L.lag_profile_num_classes()
        cnt = (C.c_longlong * nk)()
        kms = (C.c_double * nk)()
        L.check(L.lag_profile_read(ctx, nk, cnt, kms), ctx)
        L.lag_profile_enable(ctx, 0)
        prof = {L.lag_profile_class_name(i).decode(): (cnt[i], kms[i]) for i in range(nk) if cnt[i]}
        return ms, launches, prof, p0.elapsed_time(p1)

    def iters_of(sh, m0, m1):
        its = np.zeros((1, s.n_harm), dtype=np.int32)
        st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
        L.lag_shot_stats(sh, C.byref(st))
        return its[0, m0:m1]

    def traces_of(sh):
        tr = np.zeros((len(s.receivers), s.t_out.size))
        L.check(L.lag_shot_traces(sh, tr.ctypes.data_as(L.PD)), ctx)
        return tr

    W, K = args.warmup, args.steps
    acc = {}  # leg -> fields of harmonics 0 .. ACC_HARM-1 (the oracle check after the timed legs)
    # ---- headline: FP64 path
    sh = make_shot(L.LAG_FP64)
    acc["headline_fp64"] = []
    with ClockSampler(local_rank) as clk:
        ms, launches, prof, ms_prof = timed_steps(sh, W, K, keep=acc["headline_fp64"])
    clocks = clk.summary()
    its = iters_of(sh, W, W + K)
    its_prof = iters_of(sh, W + K, W + 2 * K)                          # the profiled harmonics
    tr64 = traces_of(sh)
    L.lag_shot_destroy(sh)
    value, t_sec = whole_job_rate(ms / 1e3, K, world, dist=dist, device="cuda")

    # roofline of the dominant kernel (the float64 DST: two launches per preconditioner apply, one
    # apply per PCG iteration): algorithmic flops of the real launches over the measured DST time
    ku, kv = (s.nx + 1) // 2, s.nx // 2
    flops_launch = 2.0 * s.nz * (ku * ku + kv * kv)          # float64 multiply-adds x 2
    n_dst, ms_dst = prof.get("dst_f64", (0, 0.0))
    real = 2 * int(its_prof.sum())
    probe = C.c_void_p()
    L.check(L.lag_precond_create_sep(ctx, C.byref(L.grid(s.nx, 2, s.hx, s.hz)), 1.0, 1.0, 1.0, L.LAG_FP64, 0,
                                     C.byref(probe)), ctx)
    on_tc = L.lag_precond_uses_tensor_cores(probe) == 1
    L.lag_precond_destroy(probe)
    fp64_equiv = (real * flops_launch) / (ms_dst / 1e3) / 1e12 if ms_dst > 0 else None
    if on_tc:
        # exact-slice DST on the bf16 tensor cores: 36 bf16 slice products per float64 product at
        # this length (45 above 2048); timed inside a long step -> the sustained bf16 peak
        npair = L.lag_dst_f64_slice_products(s.nx)
        achieved = fp64_equiv * npair if fp64_equiv else None
        peak = peaks["bf16_tflops_sustained"]
        roofline = {"bound": "tensor",
                    "kernel": "oz_gemm_kernel + oz_pack_a_kernel (float64 DST as exact bf16 slice products, tcgen05)",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": (achieved / peak) if achieved else None,
                    "traffic": traffic_for("k_dst_tc.cu", "dst_f64_oz"),
                    "flops_per_launch": flops_launch * npair, "slice_products": npair,
                    "fp64_equivalent_tflops": fp64_equiv, "fp64_alu_peak_tflops": FP64_PEAK_TFLOPS,
                    "launches_timed": n_dst, "launches_real": real,
                    "ms_share": ms_dst / ms_prof if ms_prof > 0 else None,
                    "peak_note": f"bf16 dense, sustained, {peak_src} (MEASURED_PEAKS.json bf16_tflops_sustained)"}
    else:
        roofline = {"bound": "alu", "kernel": "dst_simt_kernel<double> (folded FP64 DST GEMM)",
                    "achieved": fp64_equiv, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": (fp64_equiv / FP64_PEAK_TFLOPS) if fp64_equiv else None,
                    "traffic": traffic_for("k_dst.cu", "dst_f64"),
                    "flops_per_launch": flops_launch, "launches_timed": n_dst, "launches_real": real,
                    "ms_share": ms_dst / ms_prof if ms_prof > 0 else None,
                    "peak_note": "derived: 152 SM x 2 FP64 FMA/clk x 2 x 2.07 GHz"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic (seeded layered medium; no dataset)",
           "config": {"workload": WORKLOAD, "grid": [s.nx, s.nz], "harmonics_timed": [W, W + K],
                      "l2": "inputs larger than L2: ~250 MB of vectors/coefficients touched per step",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "gpu_launches": int(launches), "pcg_iters_per_step": float(np.mean(its)),
           "roofline": roofline,
           "kernel_ms": {k: {"launches": c, "ms": round(v, 3)} for k, (c, v) in sorted(prof.items())},
           "kernel_ms_region": (f"harmonics {W + K}..{W + 2 * K - 1} of the same shot right after the timed region, "
                                "a CUDA event pair per launch on the shot's stream (eager launches; the timed "
                                "region replays its PCG chunks as CUDA graphs)"),
           "clocks": clocks}
    if rank != 0:
        return None
    refs = OracleRefs(s)
    if args.no_extras:
        if not args.no_accuracy:
            out["accuracy"] = accuracy_report({"headline_fp64": ("cart", acc["headline_fp64"])}, refs)
        return out

    # ---- mixed-precision path, same workload, same harmonics
    shm = make_shot(L.LAG_MIXED)
    acc["mixed"] = []
    msm, launches_m, profm, _ = timed_steps(shm, W, K, keep=acc["mixed"])
    itsm = iters_of(shm, W, W + K)
    trm = traces_of(shm)
    L.lag_shot_destroy(shm)
    rel = float(np.linalg.norm(trm - tr64) / np.linalg.norm(tr64))
    out["mixed"] = {"value": K / (msm / 1e3), "ms_per_step": msm / K, "speedup_vs_fp64_gpu": (K / (msm / 1e3)) / value,
                    "pcg_iters_per_step": float(np.mean(itsm)), "traces_rel_l2_vs_fp64_gpu": rel,
                    "gpu_launches": int(launches_m),
                    "kernel_ms": {k: {"launches": c, "ms": round(v, 3)} for k, (c, v) in sorted(profm.items())}}

    # ---- the same with the autotuned plan (partition count, bf16 product count)
    sht = make_shot(L.LAG_MIXED, tune=1)
    acc["mixed_tuned"] = []
    mst, _, proft, _ = timed_steps(sht, W, K, keep=acc["mixed_tuned"])
    trt = traces_of(sht)
    L.lag_shot_destroy(sht)
    out["mixed_tuned"] = {"value": K / (mst / 1e3), "ms_per_step": mst / K,
                          "traces_rel_l2_vs_fp64_gpu": float(np.linalg.norm(trt - tr64) / np.linalg.norm(tr64)),
                          "kernel_ms": {k: {"launches": c, "ms": round(v, 3)} for k, (c, v) in sorted(proft.items())}}

    # ---- the same shot with a free surface on top (Sec. 2.1, Eq. 3), float64 path
    shf = make_shot(L.LAG_FP64, free_surface=True)
    Kf = min(K, 16)
    acc["free_surface"] = []
    msf, _, proff, _ = timed_steps(shf, W, Kf, keep=acc["free_surface"])
    itsf = iters_of(shf, W, W + Kf)
    L.lag_shot_destroy(shf)
    out["free_surface"] = {"config": "the 2048x1024 shot with a free surface at z = 0 (zero-flux top face), FP64",
                           "value": Kf / (msf / 1e3), "unit": UNIT, "steps": Kf, "ms_per_step": msf / Kf,
                           "pcg_iters_per_step": float(np.mean(itsf))}

    # ---- the same shot with the layered preconditioner (per-row midranges), both paths
    for key, prec in (("layered", L.LAG_FP64), ("layered_mixed", L.LAG_MIXED)):
        shl = make_shot(prec, layered=1)
        acc[key] = []
        msl, launches_l, profl, _ = timed_steps(shl, W, K, keep=acc[key])
        itsl = iters_of(shl, W, W + K)
        trl = traces_of(shl)
        L.lag_shot_destroy(shl)
        out[key] = {"config": "the 2048x1024 shot preconditioned with per-row midranges kappa~(z), rho~(z) "
                              f"({'FP64' if prec == L.LAG_FP64 else 'mixed'} path)",
                    "value": K / (msl / 1e3), "unit": UNIT, "ms_per_step": msl / K,
                    "speedup_vs_fp64_gpu": (K / (msl / 1e3)) / value,
                    "pcg_iters_per_step": float(np.mean(itsl)),
                    "traces_rel_l2_vs_fp64_gpu": float(np.linalg.norm(trl - tr64) / np.linalg.norm(tr64)),
                    "gpu_launches": int(launches_l),
                    "kernel_ms": {k: {"launches": c, "ms": round(v, 3)} for k, (c, v) in sorted(profl.items())}}

    # ---- batched mixed path: 64 sources on the surface line share one shot (one launch set per step)
    out["batched"] = batched_leg(ctx, args, acc)
    # ---- elastic 4096 x 2048, 16 sources, FGMRES(20), float32 vector preconditioner
    if args.elastic_sources > 0:
        out["elastic"] = elastic_leg(ctx, args, acc=acc)
        out["elastic_layered"] = elastic_leg(ctx, args, layered=1, acc=acc)

    # ---- the paper's own 2.5D axisymmetric (r, z) acoustic problem
    if args.cyl_steps > 0:
        out["cylindrical"] = cylindrical_leg(ctx, args, acc)

    # ---- every leg's first harmonics against the oracle (the metric's "at 1e-8 rel err")
    if not args.no_accuracy:
        kinds = {"headline_fp64": "cart", "mixed": "cart", "mixed_tuned": "cart", "free_surface": "cart_fs",
                 "layered": "cart", "layered_mixed": "cart"}
        out["accuracy"] = accuracy_report({k: (v if isinstance(v, tuple) else (kinds[k], v)) for k, v in acc.items()},
                                          refs)

    # ---- served stream: Poisson arrivals of acoustic / elastic shots, continuous batching
    out["serving"] = serving_leg(ctx, args)

    # ---- standalone preconditioner: 1024 modes x nz 1024 x 512 rhs
    out["precond_bench"] = precond_bench(ctx, s, peaks, peak_src)

    # ---- end to end through the public API from pinned host buffers
    out["e2e"] = e2e(ctx, s, args.e2e_harmonics)

    # ---- CPU oracle on a bounded sample of the same workload
    out["cpu_baseline"] = cpu_baseline(s, args.cpu_seconds)
    L.lag_destroy(ctx)
    return out


def batched_leg(ctx, args, acc=None):
    """64 sources at ix = round((s + 1/2) 2048 / 64), iz = 2 on the 2048 x 1024 model, mixed path.
    The fields of the middle source in the first two (warm-up) harmonics go to acc["batched"]."""
    import torch
    from paper_1005_0542_gb300 import inputs
    from paper_1005_0542_gb300 import lagwave as L
    nsrc = args.batch_sources
    s = inputs.random_layered(sources=inputs.surface_line_sources(2048, nsrc, iz=2))
    g = L.grid(s.nx, s.nz, s.hx, s.hz)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=s.tol, prec=L.LAG_MIXED, tune=1)
    w = L.wavelet(s.f0, s.t0)
    c_, pc = L.f64(s.c)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    sh = C.c_void_p()
    L.check(L.lag_shot_create(ctx, C.byref(g), pc, None, pr, C.byref(lag), C.byref(sv), C.byref(w), nsrc,
                              L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                              C.byref(sh)), ctx)
    pick = nsrc // 2
    kept = []
    for _ in range(ACC_HARM):  # warm-up harmonics
        L.check(L.lag_shot_step(sh, 1), ctx)
        kept.append(shot_fields(ctx, sh, nsrc, 1, s.c.shape, [pick])[0])
    if acc is not None:
        acc["batched"] = ("cart_src", kept, s.sources[pick])
    stream = torch.cuda.ExternalStream(L.lag_shot_stream(sh))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    K = args.batch_steps
    for _ in range(K):
        L.check(L.lag_shot_step(sh, 1), ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # kernel classes: the next K harmonics with an event pair per launch (eager, not timed)
    L.lag_profile_enable(ctx, 1)
    for _ in range(K):
        L.check(L.lag_shot_step(sh, 1), ctx)
    torch.cuda.synchronize()
    nk = L.lag_profile_num_classes()
    cnt = (C.c_longlong * nk)()
    kms = (C.c_double * nk)()
    L.check(L.lag_profile_read(ctx, nk, cnt, kms), ctx)
    L.lag_profile_enable(ctx, 0)
    prof = {L.lag_profile_class_name(i).decode(): (cnt[i], kms[i]) for i in range(nk) if cnt[i]}
    its = np.zeros((nsrc, s.n_harm), dtype=np.int32)
    st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
    L.lag_shot_stats(sh, C.byref(st))
    L.lag_shot_destroy(sh)
    out = {"config": f"2048x1024 model, {nsrc} sources on row 2, mixed path, autotuned plan, one shot; "
                     f"step = one harmonic of every source", "value": nsrc * K / (ms / 1e3), "unit": UNIT, "steps": K,
           "ms_per_step": ms / K, "pcg_iters_per_solve": float(its[:, ACC_HARM:ACC_HARM + K].mean()),
           "kernel_ms": {k: {"launches": c, "ms": round(v, 3)} for k, (c, v) in sorted(prof.items())},
           "kernel_ms_region": "the K harmonics after the timed ones, a CUDA event pair per launch (eager)"}
    tri = prof.get("tri_f32")
    if tri and tri[0] > 0:
        # every launch solves all running sources' spectra: 8 B per point (float32 read + write);
        # launches late in a harmonic skip the sources that have converged, so this is a lower bound
        pts_per_launch = nsrc * s.nx * s.nz
        gbs = 8.0 * pts_per_launch * tri[0] / (tri[1] / 1e3) / 1e9
        out["tri_roofline"] = {"bound": "hbm", "achieved_at_most": gbs, "peak": load_peaks()[0]["hbm_gbs"],
                               "unit": "GB/s", "frac_at_most": gbs / load_peaks()[0]["hbm_gbs"],
                               "bytes_per_point": 8, "launches": tri[0], "avg_ms": tri[1] / tri[0]}
    return out


def cylindrical_leg(ctx, args, acc=None):
    """The paper's own 2.5D axisymmetric acoustic problem (Sec. 2.1, the r-weighted scheme of
    Sec. 2.3, the cylindrical preconditioner: DCT-II along z + general tridiagonal systems along r).
    Sec. 3.2's experiment: homogeneous half space, a point source on the axis at the surface, the
    wavelet of Eq. 23 (30 Hz, t0 = 0.2 s, gamma = 4), alpha = 9, h = 400, mesh step lambda/40, on
    2^k x 2^k nodes; here 2048 x 2048 (the paper's smallest mesh is 4096^2), FP64 path, where A == B
    and PCG takes one iteration; plus a random layered half space (layers along z) at 2048 x 1024
    for the iterative case, and the same model as an elastic half space (Sec. 2.2: Vs = Vp / 1.73,
    a vertical force on the axis, FGMRES(20) with K = diag(B1, B2), B1 with its hoop term).
    step = one harmonic."""
    import torch
    from paper_1005_0542_gb300 import inputs
    from paper_1005_0542_gb300 import lagwave as L
    out = {}
    for key, nr, nz, layered, prec, elastic in (("homogeneous_fp64", 2048, 2048, False, L.LAG_FP64, False),
                                                ("layered_fp64", 2048, 1024, True, L.LAG_FP64, False),
                                                ("layered_mixed", 2048, 1024, True, L.LAG_MIXED, False),
                                                ("elastic_layered_mixed", 2048, 1024, True, L.LAG_MIXED, True)):
        s = inputs.cylindrical(nr=nr, nz=nz, n_harm=64, layered=layered, elastic=elastic)
        g = L.grid(s.nx, s.nz, s.hx, s.hz, cylindrical=True)
        lag = L.laguerre(s.h, s.alpha, s.n_harm)
        sv = L.solver(tol=1e-10, prec=prec, restart_k=s.restart)
        w = L.wavelet(s.f0, s.t0, 4.0, L.LAG_WAVELET_PAPER)
        c_, pc = L.f64(s.c)
        r_, pr = L.f64(s.rho)
        t_, pt = L.f64(s.t_out)
        v_, pv = L.f64(s.vs) if elastic else (None, None)
        sh = C.c_void_p()
        L.check(L.lag_shot_create(ctx, C.byref(g), pc, pv, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                                  L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                                  C.byref(sh)), ctx)
        W, K = 3, args.cyl_steps
        kept = []
        for m in range(W):
            L.check(L.lag_shot_step(sh, 1), ctx)
            if m < (1 if elastic else ACC_HARM):
                kept.append(shot_fields(ctx, sh, 1, 2 if elastic else 1, s.c.shape, [0])[0])
        if acc is not None:
            acc["cylindrical_" + key] = ("cyl_elastic" if elastic else "cyl", kept, s)
        stream = torch.cuda.ExternalStream(L.lag_shot_stream(sh))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            L.check(L.lag_shot_step(sh, 1), ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        L.lag_profile_enable(ctx, 1)  # kernel classes: the next K harmonics, eager launches
        for _ in range(K):
            L.check(L.lag_shot_step(sh, 1), ctx)
        torch.cuda.synchronize()
        nk = L.lag_profile_num_classes()
        cnt = (C.c_longlong * nk)()
        kms = (C.c_double * nk)()
        L.check(L.lag_profile_read(ctx, nk, cnt, kms), ctx)
        L.lag_profile_enable(ctx, 0)
        its = np.zeros((1, s.n_harm), dtype=np.int32)
        st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
        L.lag_shot_stats(sh, C.byref(st))
        L.lag_shot_destroy(sh)
        out[key] = {"grid_r_z": [nr, nz], "h_m": s.hx, "value": K / (ms / 1e3), "unit": UNIT, "steps": K,
                    "ms_per_step": ms / K,
                    ("fgmres_iters_per_step" if elastic else "pcg_iters_per_step"): float(its[0, W:W + K].mean()),
                    "kernel_ms": {L.lag_profile_class_name(i).decode(): {"launches": cnt[i], "ms": round(kms[i], 3)}
                                  for i in range(nk) if cnt[i]}}
    out["config"] = ("2.5D axisymmetric half space (r, z), source on the axis, Eq. 23 wavelet 30 Hz, "
                     "mesh lambda/40; acoustic: homogeneous (Sec. 3.2) and random layered media; elastic "
                     "(Sec. 2.2): the layered medium as Vp, Vs = Vp / 1.73, vertical force, FGMRES(20) with "
                     "K = diag(B1, B2) of Eq. 22")
    return out


def elastic_leg(ctx, args, layered=0, acc=None):
    """The elastic workload: 4096 x 2048 at 2.5 m, layered Vp / Vs / rho with a dipping interface,
    vertical-force Ricker 20 Hz, sources on the surface line batched in one shot, FGMRES(20) to
    1e-10 with the float32 vector preconditioner (tensor-core DST) and float64 Krylov vectors;
    step = one harmonic of every source.  layered=1: K = diag(B1, B2) with per-row midranges."""
    import torch
    from paper_1005_0542_gb300 import inputs
    from paper_1005_0542_gb300 import lagwave as L
    nsrc = args.elastic_sources
    s = inputs.elastic_layered(nsrc=nsrc)
    g = L.grid(s.nx, s.nz, s.hx, s.hz)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=1e-10, prec=L.LAG_MIXED, restart_k=s.restart, layered=layered)
    w = L.wavelet(s.f0, s.t0)
    c_, pc = L.f64(s.c)
    v_, pv = L.f64(s.vs)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    sh = C.c_void_p()
    L.check(L.lag_shot_create(ctx, C.byref(g), pc, pv, pr, C.byref(lag), C.byref(sv), C.byref(w), nsrc,
                              L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                              C.byref(sh)), ctx)
    held = L.lag_bytes_in_use(ctx)
    L.check(L.lag_shot_step(sh, 1), ctx)  # warm-up harmonic
    if acc is not None:  # harmonic 0 of two sources, for the oracle operator's residual
        picks = [0, nsrc // 2]
        acc["elastic_layered" if layered else "elastic"] = (
            "cart_elastic", shot_fields(ctx, sh, nsrc, 2, s.c.shape, picks), s, [s.sources[i] for i in picks])
    stream = torch.cuda.ExternalStream(L.lag_shot_stream(sh))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    K = args.elastic_steps
    for _ in range(K):
        L.check(L.lag_shot_step(sh, 1), ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    its = np.zeros((nsrc, s.n_harm), dtype=np.int32)
    st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
    L.lag_shot_stats(sh, C.byref(st))
    L.lag_shot_destroy(sh)
    kind = "per-row midranges (layered K)" if layered else "Eq. 22's whole-medium midranges"
    return {"config": f"{s.nx}x{s.nz} elastic, 2.5 m, {nsrc} sources on row 2, FGMRES({s.restart}) to 1e-10, "
                      f"float32 preconditioner, {kind}; step = one harmonic of every source",
            "value": nsrc * K / (ms / 1e3), "unit": UNIT, "steps": K, "ms_per_step": ms / K,
            "gmres_iters_per_solve": float(its[:, 1:1 + K].mean()), "device_gb": held / 1e9}


def _serve_trace(ctx, trace, active, budget_s):
    """Submit `trace` on its Poisson schedule to the continuous-batching server, serve until every
    request is done or `budget_s` seconds have passed since the first arrival, cancel what is left.
    Media are generated once per (kind, mesh) and shared by the requests that draw that pair (the
    solve's cost depends on the mesh, the kind and the harmonic count, not on the draw)."""
    from paper_1005_0542_gb300 import inputs
    from paper_1005_0542_gb300 import lagwave as L
    media, reqs, keep = {}, [], []
    for q in trace:
        key = (q["kind"], q["nx"], q["nz"])
        if key not in media:
            if q["kind"] == "acoustic":
                m = inputs.random_layered(nx=q["nx"], nz=q["nz"], hx=5.0, n_harm=8, seed=q["seed"],
                                          sources=[(q["nx"] // 2, min(16, q["nz"] - 1))])
            else:
                m = inputs.elastic_layered(nx=q["nx"], nz=q["nz"], hx=2.5, n_harm=8, seed=q["seed"], nsrc=1)
            m.receivers = m.receivers[:16]
            m.t_out = m.t_out[:100]
            arrs = [L.f64(m.c), L.f64(m.rho), L.f64(m.t_out), L.points(m.sources), L.points(m.receivers)]
            if m.vs is not None:
                arrs.append(L.f64(m.vs))
            media[key] = (m, arrs)
        m, arrs = media[key]
        rq = L.lag_request()
        rq.kind = 1 if m.vs is not None else 0
        rq.grid = L.grid(m.nx, m.nz, m.hx, m.hz)
        rq.c_host, rq.rho_host = arrs[0][1], arrs[1][1]
        if m.vs is not None:
            rq.vs_host = arrs[5][1]
        rq.lag = L.laguerre(m.h, m.alpha, q["n_harm"])
        rq.solver = L.solver(tol=m.tol, prec=L.LAG_MIXED, restart_k=m.restart)
        rq.wavelet = L.wavelet(m.f0, m.t0)
        rq.nsrc, rq.src = len(m.sources), C.cast(arrs[3], C.POINTER(L.lag_point))
        rq.nrcv, rq.rcv = len(m.receivers), C.cast(arrs[4], C.POINTER(L.lag_point))
        rq.nt, rq.t_out_host = m.t_out.size, arrs[2][1]
        ncomp = 2 if m.vs is not None else 1
        reqs.append((q, rq, np.zeros(len(m.sources) * ncomp * len(m.receivers) * m.t_out.size)))
    L.check(L.lag_serve_start(ctx, active), ctx)
    t0 = time.perf_counter()
    tickets = []
    for q, rq, buf in reqs:  # submit on the Poisson schedule (the request arrays are copied)
        while time.perf_counter() - t0 < q["arrival"] - trace[0]["arrival"]:
            time.sleep(0.0005)
        t = C.c_uint64()
        L.check(L.lag_serve_submit(ctx, C.byref(rq), C.byref(t)), ctx)
        tickets.append(t.value)
    results = [None] * len(reqs)
    cancelled = False
    while True:
        pending = 0
        for i, ((q, rq, buf), t) in enumerate(zip(reqs, tickets)):
            if results[i] is not None:
                continue
            res = L.lag_result()
            res.traces_host = buf.ctypes.data_as(L.PD)
            if L.lag_serve_poll(ctx, t, C.byref(res)) == L.LAG_OK:
                results[i] = (res.status, res.t_submit, res.t_admit, res.t_done, res.harmonics_done)
            else:
                pending += 1
        if pending == 0:
            break
        if not cancelled and time.perf_counter() - t0 > budget_s:
            for i, t in enumerate(tickets):
                if results[i] is None:
                    L.lag_serve_cancel(ctx, t)
            cancelled = True
        time.sleep(0.005)
    makespan = time.perf_counter() - t0
    L.check(L.lag_serve_stop(ctx), ctx)
    done = [(q, r) for (q, rq, buf), r in zip(reqs, results) if r[0] == L.LAG_OK]
    lat = np.array([r[3] - r[1] for _, r in done]) if done else np.zeros(1)
    queue = np.array([r[2] - r[1] for _, r in done]) if done else np.zeros(1)
    service = np.array([r[3] - r[2] for _, r in done]) if done else np.zeros(1)
    solves = sum(r[4] for r in results)  # every harmonic solved, the cancelled requests' included
    return {"requests": len(reqs), "completed": len(done),
            "admitted": sum(1 for r in results if r[2] > 0), "harmonic_solves": int(solves),
            "cancelled_at_budget": sum(1 for r in results if r[0] == L.LAG_ECANCELED),
            "failed": sum(1 for r in results if r[0] not in (L.LAG_OK, L.LAG_ECANCELED)),
            "value": solves / makespan, "unit": UNIT, "makespan_s": makespan, "budget_s": budget_s,
            "offered_rps": len(reqs) / max(trace[-1]["arrival"] - trace[0]["arrival"], 1e-9),
            "achieved_rps": len(done) / makespan,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queue_s": float(np.mean(queue)), "mean_service_s": float(np.mean(service)),
            "p50_service_s": float(np.percentile(service, 50)), "p99_service_s": float(np.percentile(service, 99))}


def serving_leg(ctx, args):
    """The served stream of the workload: Poisson arrivals at 50 requests/s of acoustic / elastic
    shots (half each) on meshes drawn from {256^2, 512x1024, 1024x2048, 2048x1024, 4096x2048},
    128-1024 harmonics each, one source, mixed path, continuous batching in `serve_active` slots.
    The offered load is far above one GPU's capacity: the trace's requests (all arriving within a
    few seconds) are served for a wall budget, then the rest are cancelled; the report gives offered
    against achieved load, the latency of the completed requests split into queueing and service,
    and a second, sub-capacity run (the two smallest meshes, 128-256 harmonics, 1 request/s) whose
    latency is the service time alone."""
    from paper_1005_0542_gb300 import inputs
    trace = inputs.request_trace(count=args.serve_requests, rate=50.0, n_lo=128, n_hi=1024)
    over = _serve_trace(ctx, trace, args.serve_active, args.serve_seconds)
    over["config"] = (f"{len(trace)} Poisson requests at 50/s, acoustic/elastic, meshes from "
                      "{256^2, 512x1024, 1024x2048, 2048x1024, 4096x2048}, 128-1024 harmonics each, mixed path, "
                      f"{args.serve_active} concurrent slots, served for {args.serve_seconds:.0f} s")
    small = inputs.request_trace(count=10, rate=1.0, seed=inputs.SEED_BASE + 6, n_lo=128, n_hi=256,
                                 meshes=inputs.SERVE_MESHES[:2])
    sub = _serve_trace(ctx, small, args.serve_active, 300.0)
    sub["config"] = "10 Poisson requests at 1/s, meshes 256^2 and 512x1024, 128-256 harmonics, mixed path"
    over["sub_capacity"] = sub
    return over


def precond_bench(ctx, s, peaks, peak_src):
    import torch
    from paper_1005_0542_gb300 import lagwave as L
    nx, nz, nrhs = 1024, 1024, 512
    kap = s.rho * s.c ** 2
    kt = 0.5 * (kap.min() + kap.max())
    rt = 0.5 * (s.rho.min() + s.rho.max())
    res = {"config": "1024 modes x nz 1024 x 512 RHS, midrange coefficients of the 2048x1024 model at 5 m"}
    gen = torch.Generator(device="cuda").manual_seed(7)
    r = torch.randn((nrhs, nz, nx), dtype=torch.float64, device="cuda", generator=gen)
    z = torch.empty_like(r)
    for prec, name in ((L.LAG_FP64, "fp64"), (L.LAG_MIXED, "mixed")):
        p = C.c_void_p()
        L.check(L.lag_precond_create(ctx, C.byref(L.grid(nx, nz, 5.0, 5.0)), kt, rt, s.h, prec, C.byref(p)), ctx)
        for _ in range(2):
            L.check(L.lag_precond_apply(p, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), nrhs), ctx)
        L.lag_synchronize(ctx)
        L.lag_profile_enable(ctx, 1)
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            L.check(L.lag_precond_apply(p, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), nrhs), ctx)
        L.lag_synchronize(ctx)
        wall = (time.perf_counter() - t0) / reps
        nk = L.lag_profile_num_classes()
        cnt = (C.c_longlong * nk)()
        ms = (C.c_double * nk)()
        L.check(L.lag_profile_read(ctx, nk, cnt, ms), ctx)
        L.lag_profile_enable(ctx, 0)
        prof = {L.lag_profile_class_name(i).decode(): (cnt[i], ms[i] / max(cnt[i], 1)) for i in range(nk) if cnt[i]}
        pts = nrhs * nx * nz
        entry = {"apply_ms": wall * 1e3, "ps_per_point": wall * 1e12 / pts,
                 "kernels": {k: {"avg_ms": v} for k, (c, v) in prof.items()}}
        tri = prof.get("tri_f64" if prec == L.LAG_FP64 else "tri_f32")
        if tri:
            eb = 16 if prec == L.LAG_FP64 else 8
            gbs = eb * pts / (tri[1] / 1e3) / 1e9
            if prec == L.LAG_FP64:
                # float64 is 1/64 of float32 on this part: 9 FP64 flops per point (forward sweep
                # FMA + multiply, back substitution FMA, spike correction two FMAs) bound the kernel
                tf = 9.0 * pts / (tri[1] / 1e3) / 1e12
                entry["tri_roofline"] = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                         "frac": tf / FP64_PEAK_TFLOPS, "flops_per_point": 9,
                                         "hbm_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"],
                                         "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 x 2.07 GHz"}
            else:
                entry["tri_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                         "frac": gbs / peaks["hbm_gbs"], "bytes_per_point": eb,
                                         "peak_source": peak_src}
        L.lag_precond_destroy(p)
        res[name] = entry
    del r, z
    torch.cuda.empty_cache()
    return res


def e2e(ctx, s, nh):
    import torch
    from paper_1005_0542_gb300 import lagwave as L

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t

    c, rho, tout = pinned(s.c), pinned(s.rho), pinned(s.t_out)
    tr = torch.empty((1, len(s.receivers), s.t_out.size), dtype=torch.float64, pin_memory=True)
    g = L.grid(s.nx, s.nz, s.hx, s.hz)
    lag = L.laguerre(s.h, s.alpha, nh)
    sv = L.solver(tol=s.tol)
    w = L.wavelet(s.f0, s.t0)
    P = lambda t: C.cast(t.data_ptr(), L.PD)  # noqa: E731
    t0 = time.perf_counter()
    L.check(L.lag_solve_acoustic(ctx, C.byref(g), P(c), P(rho), C.byref(lag), C.byref(sv), C.byref(w), 1,
                                 L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, P(tout),
                                 P(tr), None), ctx)
    dt = time.perf_counter() - t0
    h2d = (c.numel() + rho.numel() + tout.numel()) * 8 + 8 * (1 + len(s.receivers))
    d2h = tr.numel() * 8
    return {"value": nh / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / nh, "d2h_bytes_per_step": d2h / nh,
            "harmonics": nh, "seconds": dt,
            "api": "lag_solve_acoustic (host medium in, host traces out; includes medium/plan setup)"}


def oracle_harmonics(s, budget_s, max_harm, min_harm=1):
    """Time the oracle on harmonics 0, 1, ... of the shot until the budget is spent."""
    from oracle import fd, krylov, laguerre, precond
    kap = fd.kappa_from_velocity(s.c, s.rho)
    pr = precond.acoustic_params(kap, s.rho, s.h)
    nz, nx = s.nz, s.nx
    fm = laguerre.forward_coeffs(laguerre.ricker(s.f0, s.t0), max_harm, s.h, s.alpha, s.t0 + 4.0 / s.f0)
    R, times, iters = [], [], []
    src = s.sources[0]
    for m in range(max_harm):
        t0 = time.perf_counter()
        b = np.zeros((nz, nx))
        if m:
            b -= s.rho * s.h ** 2 * float(laguerre.c_m(m, s.alpha)) * laguerre.history_direct(R, m, s.alpha)
        b[src[1], src[0]] += fm[m] / (s.hx * s.hz)
        x, it, _ = krylov.pcg(lambda v: fd.apply_A(v.reshape(nz, nx), kap, s.rho, s.h, s.hx, s.hz).ravel(),
                              lambda v: precond.apply_inverse(v.reshape(nz, nx), s.hx, s.hz, *pr).ravel(),
                              b.ravel(), s.tol)
        R.append(x.reshape(nz, nx))
        times.append(time.perf_counter() - t0)
        iters.append(it)
        if sum(times) >= budget_s and m + 1 >= min_harm:
            break
    return times, iters


def oracle_iteration_seconds(budget):
    """Seconds per oracle PCG iteration on the benchmark shot's first harmonic (run in a child
    process pinned to one thread for the single-core figure)."""
    from oracle import fd, krylov, laguerre, precond
    from paper_1005_0542_gb300 import inputs
    s = inputs.random_layered()
    kap = fd.kappa_from_velocity(s.c, s.rho)
    pr = precond.acoustic_params(kap, s.rho, s.h)
    nz, nx = s.nz, s.nx
    fm = laguerre.forward_coeffs(laguerre.ricker(s.f0, s.t0), 1, s.h, s.alpha, s.t0 + 4.0 / s.f0)
    b = np.zeros((nz, nx))
    b[s.sources[0][1], s.sources[0][0]] = fm[0] / (s.hx * s.hz)
    A = lambda v: fd.apply_A(v.reshape(nz, nx), kap, s.rho, s.h, s.hx, s.hz).ravel()  # noqa: E731
    M = lambda v: precond.apply_inverse(v.reshape(nz, nx), s.hx, s.hz, *pr).ravel()  # noqa: E731
    k, t = 1, 0.0
    while True:
        t0 = time.perf_counter()
        krylov.pcg(A, M, b.ravel(), 1e-30, max_iter=k)   # exactly k iterations
        t = time.perf_counter() - t0
        if t >= budget or k >= 64:
            return t / k, k
        k *= 2


def cpu_baseline(s, budget):
    times, iters = oracle_harmonics(s, budget, 64)
    out = {"value": len(times) / sum(times), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"first {len(times)} harmonics of the same shot (oracle PCG, direct DST, Thomas; "
                     f"{sum(times):.1f} s, {np.mean(iters):.0f} PCG iterations/harmonic)"}
    # one core: a child process with single-threaded BLAS times PCG iterations of the first harmonic;
    # the rate is one harmonic per (seconds per iteration x the iterations per harmonic above)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               GOTO_NUM_THREADS="1", PYTHONPATH=ROOT)
    code = ("import json, bench; t, k = bench.oracle_iteration_seconds(%r); print(json.dumps([t, k]))"
            % (budget / 2,))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                           timeout=max(120.0, 8 * budget))
        t_it, k = json.loads(r.stdout.strip().splitlines()[-1])
        out["one_core"] = {"value": 1.0 / (t_it * float(np.mean(iters))), "unit": UNIT, "cores": 1,
                           "sample": f"{k} PCG iterations of harmonic 0 on one thread ({t_it:.2f} s each), "
                                     f"x {np.mean(iters):.0f} iterations per harmonic"}
    except (subprocess.SubprocessError, ValueError, IndexError, OSError) as exc:
        out["one_core"] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


# ---------------------------------------------------------------------------------- ncu capture
def capture_kernels(args):
    """One launch of each hot kernel through the C ABI on inputs larger than L2 (1024 modes x
    nz 1024 x 16 RHS, float64 arrays of 134 MB), for `ncu -k ... -c N` captures."""
    import torch
    from paper_1005_0542_gb300 import lagwave as L
    ctx = L.create(0, stream=torch.cuda.current_stream().cuda_stream)
    nx = nz = 1024
    nrhs = 16
    gen = torch.Generator(device="cuda").manual_seed(1)
    r = torch.randn((nrhs, nz, nx), dtype=torch.float64, device="cuda", generator=gen)
    z = torch.empty_like(r)
    rf = torch.randn((2 * nrhs, nz, nx), dtype=torch.float32, device="cuda", generator=gen)
    zf = torch.empty_like(rf)
    P = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731

    def plan(prec):
        p = C.c_void_p()
        L.check(L.lag_precond_create_sep(ctx, C.byref(L.grid(nx, nz, 5.0, 5.0)), 3e10, 3e10, 2.2e7, prec, 0,
                                         C.byref(p)), ctx)
        return p
    p64, pmx = plan(L.LAG_FP64), plan(L.LAG_MIXED)
    c = np.full((nz, nx), 3000.0)
    rho = np.full((nz, nx), 2000.0)
    m = C.c_void_p()
    c_, pc = L.f64(c)
    r_, pr = L.f64(rho)
    L.check(L.lag_medium_create_acoustic(ctx, C.byref(L.grid(nx, nz, 5.0, 5.0)), pc, pr, 200.0, C.byref(m)), ctx)
    torch.cuda.synchronize()
    L.check(L.lag_precond_dst(p64, P(r), P(z), nrhs), ctx)             # exact-slice FP64 DST (pack + tcgen05)
    L.check(L.lag_precond_tridiag(p64, P(r), P(z), nrhs), ctx)         # FP64 tridiagonal solve
    L.check(L.lag_precond_dst(pmx, P(r), P(z), nrhs), ctx)             # pack + tcgen05 DST GEMM
    L.check(L.lag_precond_tridiag_f32(pmx, P(rf), P(zf), 2 * nrhs), ctx)  # FP32 tridiagonal solve
    L.check(L.lag_apply_operator(m, P(r), P(z), nrhs), ctx)            # acoustic stencil
    # the shot's shape: one 2048 x 1024 field through the exact-slice FP64 DST
    ph = C.c_void_p()
    L.check(L.lag_precond_create_sep(ctx, C.byref(L.grid(2048, 1024, 5.0, 5.0)), 3e10, 3e10, 2.2e7, L.LAG_FP64, 0,
                                     C.byref(ph)), ctx)
    rh = torch.randn((1, 1024, 2048), dtype=torch.float64, device="cuda", generator=gen)
    zh = torch.empty_like(rh)
    L.check(L.lag_precond_dst(ph, P(rh), P(zh), 1), ctx)
    torch.cuda.synchronize()
    L.lag_destroy(ctx)
    print(json.dumps({"capture": "ok"}))


def capture_extensions(args):
    """One launch of the kernels of the layered and cylindrical plans through the C ABI, 1024 x 1024
    x 16 RHS float64 (134 MB > L2): the general tridiagonal solve (one factor set per partition)
    of a layered plan, then the forward and the inverse DCT-II of a cylindrical float64 plan
    (exact slices; the inverse gathers even / odd modes and ends in the E/O butterfly); then a
    two-harmonic cylindrical elastic shot of 1024 x 512 (the axisymmetric elastic stencil and the
    FGMRES kernels), for `ncu -k ... -c N` captures."""
    import torch
    from paper_1005_0542_gb300 import lagwave as L
    ctx = L.create(0, stream=torch.cuda.current_stream().cuda_stream)
    n, nrhs = 1024, 16
    gen = torch.Generator(device="cuda").manual_seed(2)
    r = torch.randn((nrhs, n, n), dtype=torch.float64, device="cuda", generator=gen)
    z = torch.empty_like(r)
    P = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    rng = np.random.default_rng(3)
    ax = 3e10 * rng.uniform(0.3, 1.0, n)
    d = 2.2e7 * rng.uniform(0.5, 1.0, n)
    a_, pa = L.f64(ax)
    d_, pd = L.f64(d)
    pl = C.c_void_p()
    L.check(L.lag_precond_create_layered(ctx, C.byref(L.grid(n, n, 5.0, 5.0)), pa, pa, pd, L.LAG_FP64, 0,
                                         C.byref(pl)), ctx)
    pc = C.c_void_p()
    L.check(L.lag_precond_create_sep(ctx, C.byref(L.grid(n, n, 5.0, 5.0, cylindrical=True)), 3e10, 3e10, 2.2e7,
                                     L.LAG_FP64, 0, C.byref(pc)), ctx)
    torch.cuda.synchronize()
    L.check(L.lag_precond_tridiag(pl, P(r), P(z), nrhs), ctx)        # general tridiagonal solve (layered)
    L.check(L.lag_precond_dst(pc, P(r), P(z), nrhs), ctx)            # forward DCT-II (fold + exact slices)
    L.check(L.lag_precond_dst_inverse(pc, P(z), P(r), nrhs), ctx)    # inverse DCT-II (gather + GEMM + E/O)
    L.check(L.lag_precond_tridiag(pc, P(r), P(z), nrhs), ctx)        # systems along r (cylindrical)
    torch.cuda.synchronize()
    # a cylindrical elastic shot, 1024 x 512 (r x z), 2 harmonics, mixed path: the axisymmetric
    # elastic stencil and the FGMRES Gram-Schmidt kernels (basis vectors 8.4 MB each, 176 MB > L2)
    from paper_1005_0542_gb300 import inputs
    se = inputs.cylindrical(nr=1024, nz=512, n_harm=2, layered=True, elastic=True)
    ge = L.grid(se.nx, se.nz, se.hx, se.hz, cylindrical=True)
    lag = L.laguerre(se.h, se.alpha, se.n_harm)
    sv = L.solver(tol=1e-10, prec=L.LAG_MIXED, restart_k=se.restart)
    w = L.wavelet(se.f0, se.t0, 4.0, L.LAG_WAVELET_PAPER)
    c_, pcv = L.f64(se.c)
    v_, pvs = L.f64(se.vs)
    r_, prh = L.f64(se.rho)
    t_, pt = L.f64(se.t_out)
    tr = np.zeros((1, 2, len(se.receivers), se.t_out.size))
    L.check(L.lag_solve_elastic(ctx, C.byref(ge), pcv, pvs, prh, C.byref(lag), C.byref(sv), C.byref(w), 1,
                                L.points(se.sources), len(se.receivers), L.points(se.receivers), se.t_out.size, pt,
                                tr.ctypes.data_as(L.PD), None), ctx)
    L.lag_destroy(ctx)
    print(json.dumps({"capture": "ok"}))


def capture_shot(args):
    """Three harmonics of the 2048 x 1024 shot (--capture-shot fp64 or mixed) with every kernel
    launched eagerly (no graphs), for `ncu -k ... -s N -c M` captures at the shot's shape: the
    exact-slice pack and GEMM, the float64 tridiagonal solve (fp64); the split-bf16 DST kernels
    (forward pack + GEMM, inverse pack + GEMM + butterfly with the CG dots), the float32
    tridiagonal solve (mixed); the PCG kernels (both)."""
    import torch
    from paper_1005_0542_gb300 import inputs
    from paper_1005_0542_gb300 import lagwave as L
    os.environ["LAGWAVE_GRAPHS"] = "0"
    ctx = L.create(0, stream=torch.cuda.current_stream().cuda_stream)
    s = inputs.random_layered()
    g = L.grid(s.nx, s.nz, s.hx, s.hz)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=s.tol, prec=L.LAG_MIXED if args.capture_shot == "mixed" else L.LAG_FP64)
    w = L.wavelet(s.f0, s.t0)
    c_, pc = L.f64(s.c)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    sh = C.c_void_p()
    L.check(L.lag_shot_create(ctx, C.byref(g), pc, None, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                              L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                              C.byref(sh)), ctx)
    L.check(L.lag_shot_step(sh, 3), ctx)
    torch.cuda.synchronize()
    L.lag_shot_destroy(sh)
    L.lag_destroy(ctx)
    print(json.dumps({"capture": "ok"}))


# ---------------------------------------------------------------------------------- reference arm
def reference_arm(args):
    from paper_1005_0542_gb300 import inputs
    s = inputs.random_layered()
    # the oracle's harmonics are sequential: W untimed warm-up harmonics, then K timed ones;
    # each step is one harmonic of the oracle on the full 2048 x 1024 model (about 4 s on 16 Arm
    # cores), so at most 3 + 12 of them run: the whole arm stays near a minute
    W, K = min(args.warmup, 3), min(args.steps, 12)
    times, iters = oracle_harmonics(s, float("inf"), W + K, min_harm=W + K)
    tk = times[W:W + K]
    v = len(tk) / sum(tk)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": K,
            "warmup": W, "ms_per_step": 1e3 * sum(tk) / len(tk), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded layered medium; no dataset)",
            "config": {"workload": WORKLOAD, "grid": [s.nx, s.nz], "harmonics_timed": [W, W + K]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"harmonics {W}..{W + K - 1} of the shot on the host cores"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=48)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lagwave", choices=["lagwave", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="headline only (for launch-list captures)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the oracle check of the legs' first harmonics")
    ap.add_argument("--e2e-harmonics", type=int, default=4)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batch-sources", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--elastic-sources", type=int, default=16, help="0 skips the elastic leg")
    ap.add_argument("--elastic-steps", type=int, default=2)
    ap.add_argument("--cyl-steps", type=int, default=8, help="harmonics timed per cylindrical case; 0 skips the leg")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-active", type=int, default=8)
    ap.add_argument("--serve-seconds", type=float, default=90.0,
                    help="wall budget of the served stream; requests still running or queued then are cancelled")
    ap.add_argument("--capture-extensions", action="store_true",
                    help="launch the layered / cylindrical plan kernels once (1024 x 1024 x 16 RHS) for ncu, then exit")
    ap.add_argument("--capture-shot", choices=["fp64", "mixed"],
                    help="three eager harmonics of the 2048 x 1024 shot on the given path for ncu, then exit")
    ap.add_argument("--capture-kernels", action="store_true",
                    help="launch each hot kernel once (1024 x 1024 x 16 RHS) for ncu captures, then exit")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.capture_kernels:
        capture_kernels(args)
        return
    if args.capture_extensions:
        capture_extensions(args)
        return
    if args.capture_shot:
        capture_shot(args)
        return
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(args)), flush=True)
        return
    out = gpu_arm(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
