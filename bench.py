"""Benchmark of the ACCORD-FBS hot path on one GB300 (or N replicas).

A step is one accord_fit to KKT residual <= 1e-4 on the hub-and-block
workload p = 40000, n = 1000, lambda = 0.1 (mixed BF16x3 GEMMs, FP64 line
search / KKT reductions), X resident in HBM.  The headline value is prox-grad
iterations per second over the timed fits; ms_per_step is the time to KKT.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded
row-block sample of the same workload on this host's cores.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "prox-grad iters/s to KKT 1e-4 (hub-and-block p=40000, n=1000, lambda=0.1)"
UNIT = "iters/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 3; 2000 for --workload diff, whose step is ~1 ms, so that the "
                         "clock sampler sees the timed region)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--p", type=int, default=40000)
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--kkt-tol", type=float, default=1e-4)
    ap.add_argument("--coarse-kkt", type=float, default=5e-3,
                    help="one-product gradients while the KKT residual is above this (0: three products throughout)")
    ap.add_argument("--fp64-iters", type=int, default=2, help="FP64 iterations timed for the comparison (0: skip)")
    ap.add_argument("--tf32-fits", type=int, default=1, help="TF32x3 fits timed for the comparison (0: skip)")
    ap.add_argument("--refresh-cost-fits", type=int, default=3,
                    help="fits each with and without the refresh of Y, to report what the refresh costs (0: skip)")
    ap.add_argument("--fp64-full", action="store_true",
                    help="also run one whole FP64 fit to the same KKT tolerance (several minutes at p=40000), "
                         "timed, and grade the mixed estimate against it (rel. Frobenius, support, FP64 KKT)")
    ap.add_argument("--no-sequential", action="store_true",
                    help="path: skip the baseline of the same fits made one accord_fit call at a time")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile-run", action="store_true",
                    help="instead of timing: the fixed call sequence the ncu summaries were captured from "
                         "(path: one accord_path with per-launch events; diff: a fit, three derivative and "
                         "X-gradient calls, and three post-processing calls at p=16000)")
    ap.add_argument("--workload", choices=["fit", "path", "diff", "refit"], default="fit",
                    help="fit: one fit at p=40000 (default); path: lambda path x bootstrap subsamples at p=4000; "
                         "diff: held-out derivative in log(lambda) at p=2000; refit: Eq. 3.8 refit at p=40000")
    args = ap.parse_args(argv)
    if args.steps is None:
        args.steps = 2000 if args.workload == "diff" else 3
    return args


def make_workload(p, n):
    from synth import workload
    return workload("hubblock", p=p, n=n)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# --------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[1]) for r in rows])
        mx = np.array([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(np.nanmax(mx)), "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ CPU oracle ----
def oracle_sample(X64, lam, rows, row0=0, lam_d=None):
    """One accepted FBS iteration of the oracle (Algorithm 1 trial + the next
    gradient) on rows [row0, row0+rows) of Omega^0 = I; returns seconds.  lam
    may be a (rows x p) weight matrix (the refit of Eq. 3.8), lam_d then the
    diagonal weight."""
    from oracle import accord_ref as R
    n, p = X64.shape
    lam_d = lam if lam_d is None else lam_d
    Om = np.zeros((rows, p))
    Om[np.arange(rows), row0 + np.arange(rows)] = 1.0
    Y = Om @ X64.T
    G = Y @ X64 / n
    t0 = time.perf_counter()
    R.kkt_residual(Om, G, lam, lam_d, row0=row0)
    Op, Yp, d2, dy2, gp, dG = R.fbs_trial(Om, Y, G, X64, 1.0, lam, lam_d, row0=row0)
    G = Yp @ X64 / n
    return time.perf_counter() - t0


def cpu_rows_for(X64, lam, seconds):
    """Rows per sample so that one sample takes about `seconds`."""
    m0 = 128
    t = oracle_sample(X64, lam, m0)
    return int(max(16, min(X64.shape[1], m0 * seconds / max(t, 1e-3)))), t


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except Exception:
        pass
    return os.cpu_count() or 1


# ---------------------------------------------------------------- ours -----
def _code_only(src):
    """Source text without comments and blank space, so that a change to a
    comment does not count as a change to the kernel (string literals in
    these files hold no comment markers)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_digest():
    """Digest of the prox kernel's code (its translation unit and the two
    headers it inlines), comments excluded."""
    h = hashlib.sha256()
    for name in ("gemm_tc.cu", "tc_ptx.cuh", "common.cuh"):
        h.update(_code_only(open(os.path.join(ROOT, "paper_2412_11554_gb300", "csrc", name)).read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, digest):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the summary is missing or predates the kernel's source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(kernel)
    if not e or e.get("source_digest") != digest:
        return None
    return e.get("dram_bytes_per_launch")


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2412_11554_gb300 import build as B
    B.build()
    import paper_2412_11554_gb300 as A

    w = make_workload(args.p, args.n)
    n, p = w.n, w.p
    X = torch.as_tensor(w.X, device="cuda")
    ws = torch.empty(A.accord_workspace_bytes(n, p, precision="mixed", max_iter=500), dtype=torch.uint8,
                     device="cuda")
    Om = torch.empty((p, p), dtype=torch.float32, device="cuda")
    fit_kw = dict(precision="mixed", kkt_tol=args.kkt_tol, max_iter=500, workspace=ws, Omega=Om,
                  coarse_kkt=args.coarse_kkt)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        A.accord_fit(X, w.lam, **fit_kw)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    stats = []
    stream = torch.cuda.current_stream()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    # one event per fit boundary: the whole region is e[0] .. e[K], and the
    # per-fit times give the median and best fit beside the aggregate
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        _, st = A.accord_fit(X, w.lam, profile=1, **fit_kw)
        stats.append(st)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[-1])
    fit_ms = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps))
    iters = sum(s.iters for s in stats)
    t_max = ms
    it_all = iters
    if world > 1:
        tt = torch.tensor([ms, float(iters)], device="cuda", dtype=torch.float64)
        mx = tt.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        t_max, it_all = float(mx[0]), float(tt[1])
    value = it_all / (t_max / 1e3)

    # ----- roofline of the dominant kernel (live CUDA-event timing) -----
    tp = sum(s.t_prox_gemm_ms for s in stats)
    ty = sum(s.t_y_gemm_ms for s in stats)
    npx = sum(s.n_prox_gemm for s in stats)
    ny = sum(s.n_y_gemm for s in stats)
    nco = sum(s.coarse_prox for s in stats)
    flops = 2.0 * n * p * p
    pk, pk_src = peaks()
    peak = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")))
    dominant = "tc_gemm_prox" if tp >= ty else "tc_gemm_y"
    avg_ms = (tp / max(npx, 1)) if dominant == "tc_gemm_prox" else (ty / max(ny, 1))
    achieved = flops / (avg_ms / 1e3) / 1e12
    digest = kernel_digest()
    roofline = {"bound": "tensor", "kernel": dominant, "achieved": round(achieved, 2), "peak": peak,
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "peak_source": f"bf16_tflops_sustained ({pk_src})",
                "traffic": profiled_traffic(dominant, digest),
                "algorithmic_flops_per_launch": flops,
                # executed: three split products a launch, one in the coarse launches
                "executed_frac": round((3 * (npx - nco) + nco) / max(npx, 1) * achieved / peak, 4),
                "coarse_launches_per_fit": nco / max(len(stats), 1),
                "avg_launch_ms": {"tc_gemm_prox": round(tp / max(npx, 1), 3), "y_update": round(ty / max(ny, 1), 3)},
                "gemm_share_of_step": round((tp + ty) / ms, 3)}

    # ----- the Y update, the second kernel: Y+ = Y + Delta X^T from the buckets -----
    # algorithmic bytes per launch: Y in, Y+ out and its two BF16 planes
    # (12 pn), X^T read once (4 pn) and the bucket entries (8 bytes each).
    # The kernel itself gathers one X^T row (4n bytes) per entry, most of
    # them from L2; that volume is reported beside it.
    ent = sum(s.delta_entries for s in stats) / max(ny, 1)
    if ent > 0 and ty > 0:
        hbm = float(pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
        t_y = ty / max(ny, 1) / 1e3
        by = 16.0 * p * n + 8.0 * ent
        moved = 12.0 * p * n + 8.0 * ent + 4.0 * n * ent
        roofline["y_update"] = {"bound": "hbm", "kernel": "sparse_y_kernel", "achieved": round(by / t_y / 1e9, 1),
                                "peak": hbm, "unit": "GB/s", "frac": round(by / t_y / 1e9 / hbm, 4),
                                "algorithmic_bytes_per_launch": round(by), "delta_entries_per_launch": round(ent),
                                "gathered_bytes_per_launch": round(moved),
                                "gathered_gbs": round(moved / t_y / 1e9, 1),
                                "note": "gathered: one X^T row per applied Delta entry, mostly served by L2"}

    # ----- end to end through the public API with host buffers -----
    # Each step: X from pinned host memory, the fit, and the estimate back to
    # pinned host memory as compressed sparse rows (accord_to_csr: the exact
    # nonzero entries of Omega-hat).  The same loop with the dense p x p
    # download is reported beside it (e2e_dense_omega).
    e2e = e2e_dense = None
    if not args.no_e2e:
        Xh = torch.as_tensor(w.X).pin_memory()
        Xd = torch.empty_like(X)
        nnz0 = stats[-1].nnz_offdiag + p if stats else p
        hrp = torch.empty(p + 1, dtype=torch.int64).pin_memory()
        hci = torch.empty(max(nnz0, 1), dtype=torch.int32).pin_memory()
        hva = torch.empty(max(nnz0, 1), dtype=torch.float32).pin_memory()

        def e2e_loop(dense):
            Oh = torch.empty((p, p), dtype=torch.float32).pin_memory() if dense else None
            barrier()
            torch.cuda.synchronize()
            e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e2[0].record(stream)
            it2, d2h = 0, 0
            for _ in range(args.steps):
                Xd.copy_(Xh, non_blocking=True)
                _, st = A.accord_fit(Xd, w.lam, **fit_kw)
                if dense:
                    Oh.copy_(Om, non_blocking=True)
                    d2h = Oh.numel() * 4
                else:
                    rp, ci, va = A.accord_to_csr(Om, nnz_hint=st.nnz_offdiag + p)
                    k = ci.numel()
                    if k > hci.numel():
                        raise RuntimeError("estimate has more nonzeros than the warm-up fits")
                    hrp.copy_(rp, non_blocking=True)
                    hci[:k].copy_(ci, non_blocking=True)
                    hva[:k].copy_(va, non_blocking=True)
                    d2h = (p + 1) * 8 + k * 8
                it2 += st.iters
            e2[1].record(stream)
            torch.cuda.synchronize()
            barrier()
            ms2 = e2[0].elapsed_time(e2[1])
            if world > 1:  # whole job: iterations of all ranks over the slowest rank's time
                tt2 = torch.tensor([ms2, float(it2)], device="cuda", dtype=torch.float64)
                mx2 = tt2.clone()
                dist.all_reduce(mx2, op=dist.ReduceOp.MAX)
                dist.all_reduce(tt2, op=dist.ReduceOp.SUM)
                ms2, it2 = float(mx2[0]), float(tt2[1])
            return {"value": round(it2 / (ms2 / 1e3), 3), "unit": UNIT,
                    "h2d_bytes_per_step": int(Xh.numel() * 4), "d2h_bytes_per_step": int(d2h)}

        e2e = e2e_loop(False)
        e2e["result"] = "Omega-hat as compressed sparse rows (accord_to_csr), exact"
        if world == 1:  # informational; it pins p^2 floats of host memory per rank
            e2e_dense = e2e_loop(True)
            e2e_dense["result"] = "Omega-hat dense, p x p FP32"

    # ----- FP64 GPU path on the same workload: per-launch GEMM times from a short fit -----
    # (the measured time to KKT of a whole FP64 fit is the opt-in --fp64-full leg)
    fp64 = None
    if args.fp64_iters > 0:
        O64 = torch.empty((p, p), dtype=torch.float64, device="cuda")
        _, s64 = A.accord_fit(X, w.lam, precision="fp64", kkt_tol=0.0, max_iter=args.fp64_iters, Omega=O64,
                              check=False, profile=1)
        del O64
        t_px = s64.t_prox_gemm_ms / max(s64.n_prox_gemm, 1)
        t_yg = s64.t_y_gemm_ms / max(s64.n_y_gemm, 1)
        fp64 = {"iters_timed": s64.iters, "prox_gemm_ms": round(t_px, 1), "y_gemm_ms": round(t_yg, 1),
                "prox_gemm_fp64_tflops": round(flops / (t_px / 1e3) / 1e12, 3),
                "y_gemm_fp64_tflops": round(flops / (t_yg / 1e3) / 1e12, 3),
                "setup_ms": round(s64.t_setup_ms, 1),
                "note": "FP64 SIMT GEMMs, one prox and one dense Y GEMM per trial; time to KKT of a whole FP64 "
                        "fit: --fp64-full"}

    # ----- TF32x3 mode on the same workload (whole fits to the same KKT) -----
    tf32 = None
    if args.tf32_fits > 0:
        Ot = torch.empty((p, p), dtype=torch.float32, device="cuda")
        st32 = []
        torch.cuda.synchronize()
        e3 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e3[0].record(stream)
        for _ in range(args.tf32_fits):
            _, s32 = A.accord_fit(X, w.lam, precision="tf32x3", kkt_tol=args.kkt_tol, max_iter=500, Omega=Ot,
                                  profile=1)
            st32.append(s32)
        e3[1].record(stream)
        torch.cuda.synchronize()
        del Ot
        ms3 = e3[0].elapsed_time(e3[1])
        it3 = sum(s.iters for s in st32)
        np3 = max(sum(s.n_prox_gemm for s in st32), 1)
        nc3 = sum(s.coarse_prox for s in st32)
        tp3 = sum(s.t_prox_gemm_ms for s in st32) / np3
        # TF32 dense peak: the measured BF16 peak times the nominal TF32 / BF16 ratio (1.1 / 2.25)
        peak32 = peak * 1.1 / 2.25
        ach32 = flops / (tp3 / 1e3) / 1e12
        tf32 = {"fits": len(st32), "iters_per_s": round(it3 / (ms3 / 1e3), 3),
                "time_to_kkt_s": round(ms3 / len(st32) / 1e3, 3), "iters_per_fit": it3 / len(st32),
                "final_kkt": st32[-1].kkt, "status": st32[-1].status,
                "prox_gemm_ms": round(tp3, 3), "prox_achieved_tflops": round(ach32, 2),
                # executed: three split products a launch, one in the coarse launches
                "prox_executed_frac_of_tf32_peak": round((3 * (np3 - nc3) + nc3) / np3 * ach32 / peak32, 4),
                "coarse_launches_per_fit": nc3 / len(st32),
                "tf32_peak_tflops": round(peak32, 1),
                "peak_note": "measured sustained BF16 peak x nominal TF32/BF16 ratio 1.1/2.25"}

    # ----- what the refresh of Y costs a fit: the same fits without it -----
    refresh_cost = None
    if args.refresh_cost_fits > 0:
        def time_fit(fn):
            e4 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            e4[0].record(stream)
            res = fn()
            e4[1].record(stream)
            torch.cuda.synchronize()
            return e4[0].elapsed_time(e4[1]), res

        try:
            refresh_cost = refresh_cost_leg(A, X, w.lam, fit_kw, args.refresh_cost_fits, time_fit)
        except Exception as exc:  # an informational leg: it never takes the bench line down with it
            refresh_cost = {"error": f"{type(exc).__name__}: {exc}"}

    fp64_full = None
    if args.fp64_full and rank == 0:
        fp64_full = fp64_full_leg(A, X, w, Om, stats[-1], args.kkt_tol)

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        X64 = w.X.astype(np.float64)
        rows, _ = cpu_rows_for(X64, w.lam, args.cpu_seconds)
        t = oracle_sample(X64, w.lam, rows)
        cpu = {"value": round((rows / p) / t, 6), "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"one accepted FBS iteration of the FP64 oracle on {rows} of {p} rows of Omega "
                         f"(rows are independent), scaled to all rows; {t:.1f} s"}

    if rank == 0:
        mean_iters = iters / max(len(stats), 1)
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / max(args.steps, 1), 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 (fp32 accumulate, fp64 reductions)",
            "data": "synthetic (seeded hub-and-block precision, Gaussian X)",
            "config": {"workload": w.name, "p": p, "n": n, "lambda": w.lam, "kkt_tol": args.kkt_tol,
                       "precision": "mixed_bf16x3", "coarse_kkt": args.coarse_kkt, "y_refresh": 32, "tau0": 1.0,
                       "beta": 0.5,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": f"inputs larger than L2 (Omega {4 * p * p / 1e9:.1f} GB per buffer)"},
            "time_to_kkt_s": round(ms / max(args.steps, 1) / 1e3, 3),
            "fit_ms": {"median": round(fit_ms[len(fit_ms) // 2], 2), "best": round(fit_ms[0], 2)} if fit_ms else None,
            "iters_per_fit": mean_iters, "trials_per_fit": sum(s.trials for s in stats) / max(len(stats), 1),
            "prox_launches_per_fit": sum(s.n_prox_gemm for s in stats) / max(len(stats), 1),
            "solve_iters_per_s": round(iters / (sum(s.t_solve_ms for s in stats) / 1e3), 3),
            "setup_ms": round(sum(s.t_setup_ms for s in stats) / max(len(stats), 1), 2),
            "final_kkt": stats[-1].kkt if stats else None, "status": stats[-1].status if stats else None,
            "gpu_launches": int(sum(s.n_launches for s in stats)),
            "y_refresh": {"refreshes_per_fit": sum(s.y_refreshes for s in stats) / max(len(stats), 1),
                          "max_drift": max((s.y_drift for s in stats), default=0.0), "cost": refresh_cost},
            "roofline": roofline, "e2e": e2e, "e2e_dense_omega": e2e_dense, "fp64_gpu": fp64, "tf32x3_gpu": tf32,
            "fp64_full": fp64_full,
            "cpu_baseline": cpu,
            "clocks": clk,
            "kernel_source_digest": digest,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def refresh_cost_leg(A, X, lam, fit_kw, k, time_fit):
    """What the refresh of Y costs a fit. The default refreshes every 32
    accepted steps, before a predicted passing KKT test, and before a stop;
    y_refresh = 0 carries Y through the whole fit instead. The two run in
    alternation, k fits each, timed by time_fit(fn) -> (ms, fn()). Reports the
    median times, their difference, and each fit's iterations and prox
    launches: a refresh can repeat a passing KKT test on the fresh Y."""
    times = {32: [], 0: []}
    last = {}
    for _ in range(k):
        for yr in (0, 32):  # the default last: the caller's Omega buffer ends with its estimate
            ms, (_, st) = time_fit(lambda yr=yr: A.accord_fit(X, lam, y_refresh=yr, **fit_kw))
            times[yr].append(ms)
            last[yr] = st
    med = {yr: sorted(t)[len(t) // 2] for yr, t in times.items()}
    with_, without = last[32], last[0]
    return {"fits_each": k, "fit_ms_with": round(med[32], 2), "fit_ms_without": round(med[0], 2),
            "cost_ms_per_fit": round(med[32] - med[0], 2), "refreshes_per_fit": with_.y_refreshes,
            "iters_with": with_.iters, "iters_without": without.iters,
            "prox_launches_with": with_.n_prox_gemm, "prox_launches_without": without.n_prox_gemm,
            "final_kkt_without": without.kkt}


def _kkt_and_support(O32, O64, Gm64, G64, lam, s_diag, band, rows=2000):
    """Row block by row block on the device, in FP64: the KKT residual of Eq.
    3.3 of the mixed estimate O32 (gradient Gm64 = O32 S), and the off-diagonal
    support of O32 against O64 (gradient G64 = O64 S).  A support mismatch is
    borderline when its slack is within `band`: lambda - |G_ij| for a zero
    entry of O64, |omega_ij| S_jj for a nonzero one (gradient units)."""
    import torch
    p = O64.shape[0]
    kkt, tp, n32, n64, mism, unexpl = 0.0, 0, 0, 0, 0, 0
    largest = []
    for r0 in range(0, p, rows):
        r1 = min(p, r0 + rows)
        a, b = O32[r0:r1].double(), O64[r0:r1]
        g32, g64 = Gm64[r0:r1], G64[r0:r1]
        idx = torch.arange(r1 - r0, device=a.device)
        diag = torch.zeros_like(a, dtype=torch.bool)
        diag[idx, r0 + idx] = True
        res = torch.where(a != 0, (g32 + lam * torch.sign(a)).abs(), (g32.abs() - lam).clamp_min(0.0))
        d = a[idx, r0 + idx]
        res[idx, r0 + idx] = (g32[idx, r0 + idx] - 1.0 / d + lam).abs()
        kkt = max(kkt, float(res.max()))
        pa, pb = (a != 0) & ~diag, (b != 0) & ~diag
        tp += int((pa & pb).sum())
        n32 += int(pa.sum())
        n64 += int(pb.sum())
        diff = pa != pb
        slack = torch.where(pb, b.abs() * s_diag[None, :], lam - g64.abs())
        mism += int(diff.sum())
        unexpl += int((diff & (slack > band)).sum())
        if bool(diff.any()):
            largest.append(slack[diff].max().item())
    return {"fp64_kkt_of_mixed": kkt, "support_f1": 2.0 * tp / max(n32 + n64, 1), "nnz_offdiag_mixed": n32,
            "nnz_offdiag_fp64": n64, "support_mismatches": mism, "unexplained_mismatches": unexpl,
            "largest_mismatch_slack": max(largest) if largest else 0.0}


def fp64_full_leg(A, X, w, O32, st32, kkt_tol):
    """One whole FP64 fit to the same KKT tolerance on the same workload
    (time to KKT measured from the call, as for the mixed fits), and the mixed
    estimate graded against it."""
    import torch
    p = w.p
    O64 = torch.empty((p, p), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    _, s64 = A.accord_fit(X, w.lam, precision="fp64", kkt_tol=kkt_tol, max_iter=500, Omega=O64, check=False)
    e[1].record()
    torch.cuda.synchronize()
    t = e[0].elapsed_time(e[1]) / 1e3
    out = {"status": s64.status, "iters": s64.iters, "trials": s64.trials, "time_to_kkt_s": round(t, 2),
           "setup_ms": round(s64.t_setup_ms, 1), "iters_per_s": round(s64.iters / t, 4), "final_kkt": s64.kkt}
    # accuracy of the mixed estimate against the FP64 one
    rel = float(torch.linalg.vector_norm(O32.double() - O64) / torch.linalg.vector_norm(O64))
    Gm64 = A.accord_grad(X, O32.double())      # FP64 product at the mixed estimate
    Gm = A.accord_grad(X, O32)                 # the mixed product at the same point
    err_g = float((Gm.double() - Gm64).abs().max())
    del Gm
    G64 = A.accord_grad(X, O64)                # FP64 gradient at the FP64 estimate
    Xd = X.double()
    s_diag = (Xd * Xd).sum(dim=0) / X.shape[0]
    del Xd
    band = 10.0 * err_g + st32.kkt + s64.kkt
    out.update({"mixed_iters": st32.iters, "mixed_rel_fro_to_fp64": rel, "mixed_grad_err_max": err_g,
                "support_band": band,
                "support_rule": "a mismatch is borderline when its slack (lambda - |G| at a zero, |omega| S_jj at a "
                                "nonzero of the FP64 estimate) is within 10 x the mixed gradient error plus both "
                                "fits' stopping KKT"})
    out.update(_kkt_and_support(O32, O64, Gm64, G64, w.lam, s_diag, band))
    del Gm64, G64, O64
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.p, args.n)
    X64 = w.X.astype(np.float64)
    p = w.p
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(args.steps + args.warmup, 1)))
    rows, _ = cpu_rows_for(X64, w.lam, per_step)
    for _ in range(max(args.warmup, 0)):
        oracle_sample(X64, w.lam, rows)
    ts = [oracle_sample(X64, w.lam, rows, row0=(k * rows) % max(p - rows, 1)) for k in range(args.steps)]
    t = float(sum(ts))
    value = args.steps * (rows / p) / t
    cores = cpu_threads()
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": 0, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * t / max(args.steps, 1), 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": w.name, "p": p, "n": w.n, "lambda": w.lam, "kkt_tol": args.kkt_tol,
                      "precision": "fp64_oracle", "tau0": 1.0, "beta": 0.5,
                      "parallelism": f"host cores ({cores})", "l2": "not applicable (CPU)"},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"per step one accepted FBS iteration on {rows} of {p} rows, scaled"},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------ lambda path ---
PATH_METRIC = "lambda-path estimates/s (scale-free p=4000, 32 lambdas x 16 bootstrap subsamples, KKT 1e-4)"
PATH_UNIT = "estimates/s"


def path_evaluations(res):
    """Prox evaluations per chain: every trial, plus the evaluation whose KKT
    check ended each estimate (status OK or NOT_CONVERGED)."""
    ended = ((res.entry_status == 0) | (res.entry_status == 1)).astype(np.int64)
    return (res.trials.astype(np.int64) + ended).sum(axis=0)


def oracle_trial_seconds(Xs, lam, rows):
    """One FBS trial of the oracle (prox, Y+, next gradient) on `rows` rows of
    Omega^0 = I for the data matrix Xs; returns seconds."""
    return oracle_sample(np.asarray(Xs, dtype=np.float64), lam, rows)


def sequential_fits(A, X, pw, kw, stream):
    """The path's 512 problems solved one accord_fit call at a time: along
    each subsample's chain, every penalty warm-started from the previous
    estimate, on the same data matrix the path uses (the distinct rows, row j
    scaled by sqrt(K c_j / n_s): the subsample's S), one workspace for all."""
    import torch
    p = X.shape[1]
    mats = []
    for s in pw.subsamples:
        u, c = np.unique(np.asarray(s), return_counts=True)
        scale = np.sqrt(len(u) * c / float(len(s)))
        idx = torch.as_tensor(u, device="cuda")
        mats.append((X.index_select(0, idx) * torch.as_tensor(scale, dtype=torch.float32, device="cuda")[:, None])
                    .contiguous())
    kmax = max(m.shape[0] for m in mats)
    ws = torch.empty(A.accord_workspace_bytes(kmax, p, **kw), dtype=torch.uint8, device="cuda")
    O = torch.empty((p, p), dtype=torch.float32, device="cuda")
    iters = trials = 0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for m in mats:
        for k, lam in enumerate(pw.lambdas):
            _, st = A.accord_fit(m, float(lam), Omega=O, init_from_omega=k > 0, workspace=ws, **kw)
            iters += st.iters
            trials += st.trials
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nfit = len(mats) * len(pw.lambdas)
    return {"value": round(nfit / (ms / 1e3), 3), "unit": PATH_UNIT, "ms": round(ms, 1), "fits": nfit,
            "iters_total": iters, "trials_total": trials,
            "note": "one pass, the same problems and warm starts, one accord_fit call each"}


def run_path(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2412_11554_gb300 import build as B
    B.build()
    import paper_2412_11554_gb300 as A
    from synth import path_workload

    pw = path_workload()
    n_total, p = pw.X.shape
    nl, ns = len(pw.lambdas), len(pw.subsamples)
    X = torch.as_tensor(pw.X, device="cuda")
    kw = dict(precision="mixed", kkt_tol=pw.kkt_tol, max_iter=2000)
    ws = torch.empty(A.accord_path_workspace_bytes(n_total, p, pw.subsamples, nl, **kw), dtype=torch.uint8,
                     device="cuda")
    for _ in range(max(args.warmup, 0)):
        A.accord_path(X, pw.subsamples, pw.lambdas, workspace=ws, **kw)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = []
    for _ in range(args.steps):
        res.append(A.accord_path(X, pw.subsamples, pw.lambdas, workspace=ws, **kw))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    value = nl * ns * args.steps / (ms / 1e3)
    r0 = res[-1]

    # roofline of the batched prox GEMM: one more run with CUDA events around
    # every launch (direct launches instead of the graph)
    rp = A.accord_path(X, pw.subsamples, pw.lambdas, workspace=ws, profile=1, **kw)
    evals = path_evaluations(rp)
    K = np.array([len(np.unique(s)) for s in pw.subsamples], dtype=np.float64)
    # algorithmic bytes of one chain evaluation: Omega read + Omega+ written
    # (FP32) plus the BF16 hi/lo planes of Y and X^T (K columns each)
    bytes_alg = float(np.sum(evals * (8.0 * p * p + 8.0 * p * K)))
    flops_alg = float(np.sum(evals * 2.0 * K * p * p))
    pk, pk_src = peaks()
    peak = float(pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    prox_s = rp.stats.t_prox_gemm_ms / 1e3
    achieved = bytes_alg / prox_s / 1e9
    roofline = {"bound": "hbm", "kernel": "tc_gemm_prox (batched over chains)", "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": f"hbm_gbs ({pk_src})",
                "traffic": None, "algorithmic_bytes_total": bytes_alg, "prox_launches": rp.stats.n_prox_gemm,
                "prox_ms_total": round(rp.stats.t_prox_gemm_ms, 2),
                "tensor_tflops_algorithmic": round(flops_alg / prox_s / 1e12, 1),
                "prox_share_of_path": round(rp.stats.t_prox_gemm_ms / max(rp.stats.t_solve_ms, 1e-9), 3)}

    # launch cost of the captured trial graph: one replay after every chain
    # has finished (each kernel returns at once), times the replays of a path
    replays = int(r0.stats.n_prox_gemm) // 8
    graph = {"idle_replay_ms": round(r0.stats.t_graph_idle_ms, 4), "replays": replays,
             "launch_share_of_path": round(r0.stats.t_graph_idle_ms * replays / max(r0.stats.t_solve_ms, 1e-9), 4)}

    seq = None
    if not args.no_sequential and rank == 0:
        seq = sequential_fits(A, X, pw, kw, stream)

    e2e = None
    if not args.no_e2e:
        Xh = torch.as_tensor(pw.X).pin_memory()
        Bh = torch.empty((ns, p, p), dtype=torch.float32).pin_memory()
        Xd = torch.empty_like(X)
        torch.cuda.synchronize()
        e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e2[0].record(stream)
        for _ in range(args.steps):
            Xd.copy_(Xh, non_blocking=True)
            r = A.accord_path(Xd, pw.subsamples, pw.lambdas, workspace=ws, **kw)
            Bh.copy_(r.omega_best, non_blocking=True)
        e2[1].record(stream)
        torch.cuda.synchronize()
        ms2 = e2[0].elapsed_time(e2[1])
        e2e = {"value": round(nl * ns * args.steps / (ms2 / 1e3), 3), "unit": PATH_UNIT,
               "h2d_bytes_per_step": int(Xh.numel() * 4), "d2h_bytes_per_step": int(Bh.numel() * 4)}

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        Xs = pw.X[pw.subsamples[0]]
        rows = 128
        t = oracle_trial_seconds(Xs, float(pw.lambdas[0]), rows)
        rows = int(max(16, min(p, rows * args.cpu_seconds / max(t, 1e-3))))
        t = oracle_trial_seconds(Xs, float(pw.lambdas[0]), rows)
        trials_per_est = float(evals.sum()) / (nl * ns)
        cpu = {"value": round(1.0 / (t * (p / rows) * trials_per_est), 6), "unit": PATH_UNIT,
               "cores": cpu_threads(), "kind": "oracle",
               "sample": f"one FBS trial of the FP64 oracle on {rows} of {p} rows of subsample 0 ({t:.1f} s), "
                         f"scaled to all rows and to the GPU run's {trials_per_est:.1f} prox evaluations per estimate"}

    if rank == 0:
        out = {"metric": PATH_METRIC, "value": round(value, 3), "unit": PATH_UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / max(args.steps, 1), 2),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "bf16x3 (fp32 accumulate, fp64 reductions)",
               "data": "synthetic (seeded scale-free precision, Gaussian X, bootstrap subsamples)",
               "config": {"workload": pw.name, "p": p, "n_total": n_total, "n_lambda": nl, "n_sub": ns,
                          "subsample_rows": [len(s) for s in pw.subsamples], "distinct_rows": K.astype(int).tolist(),
                          "lambda_range": [float(pw.lambdas[0]), float(pw.lambdas[-1])], "kkt_tol": pw.kkt_tol,
                          "precision": "mixed_bf16x3", "parallelism": "batched chains, CUDA graph",
                          "autotuned_prox_tiles": {"tile": "256x256 per CTA pair", "group_m": int(r0.stats.tile_group_m),
                                                   "pairs": int(r0.stats.tile_pairs)},
                          "l2": "inputs larger than L2 (16 chains x 64 MB Omega per buffer)"},
               "status": int(r0.status), "estimates_not_converged": int(np.sum(r0.entry_status == 1)),
               "prox_evaluations": int(evals.sum()), "iters_total": int(r0.stats.iters),
               "setup_ms": round(r0.stats.t_setup_ms, 2), "solve_ms": round(r0.stats.t_solve_ms, 2),
               "gpu_launches": int(r0.stats.n_launches), "best_index": r0.best_index.tolist(),
               "y_refresh": {"refreshes": int(r0.stats.y_refreshes), "max_drift": r0.stats.y_drift},
               "graph": graph, "sequential_fits": seq,
               "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk}
        print(json.dumps(out))


# ------------------------------------------------------- differentiation ---
DIFF_METRIC = "held-out derivative d L_val / d log(lambda) evaluations/s (AR(1)+random p=2000, n=300+100, lambda=0.2)"


def run_diff(args):
    import torch
    from paper_2412_11554_gb300 import build as B
    B.build()
    import paper_2412_11554_gb300 as A
    from synth import diff_workload
    w = diff_workload()
    n, p = w.X_train.shape
    nv = w.X_val.shape[0]
    Xt, Xv = torch.as_tensor(w.X_train, device="cuda"), torch.as_tensor(w.X_val, device="cuda")
    O, st = A.accord_fit(Xt, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=20000)
    for _ in range(max(args.warmup, 0)):
        A.accord_dloss_dloglam(Xt, Xv, O, w.lam)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        d, lv, _ = A.accord_dloss_dloglam(Xt, Xv, O, w.lam)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    value = args.steps / (ms / 1e3)
    # one call reads X_train, X_val and the estimate once at minimum; at this
    # size it is bound by launch and row-solve latency, not by bandwidth
    bytes_alg = 4.0 * (n + nv) * p + 4.0 * p * p
    achieved = bytes_alg / (ms / args.steps / 1e3) / 1e9
    pk, pk_src = peaks()
    peak = float(pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    roofline = {"bound": "hbm", "kernel": "whole accord_dloss_dloglam call (12 launches)",
                "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 5),
                "peak_source": f"hbm_gbs ({pk_src})", "traffic": None, "algorithmic_bytes_per_call": bytes_alg,
                "note": "latency-bound at p=2000: 12 launches and 2000 small row systems per call"}
    e2e = None
    if not args.no_e2e:
        Xth, Xvh = torch.as_tensor(w.X_train).pin_memory(), torch.as_tensor(w.X_val).pin_memory()
        Oh = O.cpu().pin_memory()
        Xtd, Xvd, Od = torch.empty_like(Xt), torch.empty_like(Xv), torch.empty_like(O)
        torch.cuda.synchronize()
        e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e2[0].record(stream)
        for _ in range(args.steps):
            Xtd.copy_(Xth, non_blocking=True)
            Xvd.copy_(Xvh, non_blocking=True)
            Od.copy_(Oh, non_blocking=True)
            A.accord_dloss_dloglam(Xtd, Xvd, Od, w.lam)
        e2[1].record(stream)
        torch.cuda.synchronize()
        ms2 = e2[0].elapsed_time(e2[1])
        e2e = {"value": round(args.steps / (ms2 / 1e3), 3), "unit": "evaluations/s",
               "h2d_bytes_per_step": int((Xth.numel() + Xvh.numel() + Oh.numel()) * 4), "d2h_bytes_per_step": 16}
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import accord_ref as R
        O64 = O.double().cpu().numpy()
        t0 = time.perf_counter()
        R.implicit_dloglam(O64, w.X_train, w.X_val, w.lam)
        t = time.perf_counter() - t0
        cpu = {"value": round(1.0 / t, 4), "unit": "evaluations/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"one full oracle evaluation ({t:.2f} s)"}
    out = {"metric": DIFF_METRIC, "value": round(value, 3), "unit": "evaluations/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / max(args.steps, 1), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16x3 products (fp32 accumulate, S in f64), f64 row systems and reductions",
           "data": "synthetic (seeded AR(1) + random-edge precision, Gaussian X)",
           "config": {"workload": w.name, "p": p, "n": n, "n_val": nv, "lambda": w.lam,
                      "active_offdiag": int(st.nnz_offdiag), "l2": "working set (32 MB S, 16 MB Omega) within L2"},
           "dloss_dloglam": d, "loss_val": lv, "gpu_launches": 12 * args.steps, "roofline": roofline, "e2e": e2e,
           "cpu_baseline": cpu, "clocks": clk}
    print(json.dumps(out))


# ----------------------------------------------------------------- refit ---
REFIT_METRIC = "Eq. 3.8 refit prox-grad iters/s to KKT 1e-4 (hub-and-block p=40000, n=1000, lambda=0.1, phi=0.5)"


def run_refit(args):
    import torch
    from paper_2412_11554_gb300 import build as B
    B.build()
    import paper_2412_11554_gb300 as A
    w = make_workload(args.p, args.n)
    n, p = w.n, w.p
    X = torch.as_tensor(w.X, device="cuda")
    ws = torch.empty(A.accord_workspace_bytes(n, p, precision="mixed", max_iter=500), dtype=torch.uint8,
                     device="cuda")
    Oh, st0 = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=args.kkt_tol, max_iter=500, workspace=ws)
    Om = torch.empty((p, p), dtype=torch.float32, device="cuda")
    kw = dict(precision="mixed", kkt_tol=args.kkt_tol, max_iter=500, workspace=ws, Omega=Om)
    for _ in range(max(args.warmup, 0)):
        A.accord_refit(X, w.lam, 0.5, Oh, **kw)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        _, s = A.accord_refit(X, w.lam, 0.5, Oh, profile=1, **kw)
        stats.append(s)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    iters = sum(s.iters for s in stats)
    tp = sum(s.t_prox_gemm_ms for s in stats)
    npx = sum(s.n_prox_gemm for s in stats)
    pk, pk_src = peaks()
    peak = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")))
    achieved = 2.0 * n * p * p / (tp / max(npx, 1) / 1e3) / 1e12

    # end to end: X and the estimate to refit from pinned host memory, the
    # refit, and its result back as compressed sparse rows
    e2e = None
    if not args.no_e2e:
        Xh, Ohh = torch.as_tensor(w.X).pin_memory(), Oh.cpu().pin_memory()
        Xd, Ohd = torch.empty_like(X), torch.empty_like(Oh)
        torch.cuda.synchronize()
        e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e2[0].record(stream)
        it2, d2h = 0, 0
        for _ in range(args.steps):
            Xd.copy_(Xh, non_blocking=True)
            Ohd.copy_(Ohh, non_blocking=True)
            _, s2 = A.accord_refit(Xd, w.lam, 0.5, Ohd, **kw)
            rp, ci, va = A.accord_to_csr(Om, nnz_hint=s2.nnz_offdiag + p)
            hrp, hci, hva = rp.cpu(), ci.cpu(), va.cpu()
            d2h = (p + 1) * 8 + ci.numel() * 8
            it2 += s2.iters
        e2[1].record(stream)
        torch.cuda.synchronize()
        ms2 = e2[0].elapsed_time(e2[1])
        e2e = {"value": round(it2 / (ms2 / 1e3), 3), "unit": "iters/s",
               "h2d_bytes_per_step": int((Xh.numel() + Ohh.numel()) * 4), "d2h_bytes_per_step": int(d2h),
               "result": "refit estimate as compressed sparse rows (accord_to_csr), exact"}

    # the oracle's refit iteration on a block of rows: weights phi * lambda on
    # the support of the estimate, infinite off it (Eq. 3.8)
    cpu = None
    if not args.no_cpu_baseline:
        X64 = w.X.astype(np.float64)
        rows, _ = cpu_rows_for(X64, w.lam, args.cpu_seconds)
        sup = Oh[:rows].cpu().numpy() != 0
        sup[np.arange(rows), np.arange(rows)] = True
        Wt = np.where(sup, 0.5 * w.lam, np.inf)
        t = oracle_sample(X64, Wt, rows, lam_d=0.5 * w.lam)
        cpu = {"value": round((rows / p) / t, 6), "unit": "iters/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"one accepted FBS iteration of the FP64 oracle refit on {rows} of {p} rows of Omega "
                         f"(rows are independent), scaled to all rows; {t:.1f} s"}
    out = {"metric": REFIT_METRIC, "value": round(iters / (ms / 1e3), 3), "unit": "iters/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / max(args.steps, 1), 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16x3 (fp32 accumulate, fp64 reductions)",
           "data": "synthetic (seeded hub-and-block precision, Gaussian X)",
           "config": {"workload": w.name, "p": p, "n": n, "lambda": w.lam, "phi": 0.5, "kkt_tol": args.kkt_tol,
                      "support_nnz_offdiag": int(st0.nnz_offdiag)},
           "iters_per_refit": iters / max(len(stats), 1), "status": stats[-1].status if stats else None,
           "gpu_launches": int(sum(s.n_launches for s in stats)),
           "roofline": {"bound": "tensor", "kernel": "tc_gemm_prox (refit mask)", "achieved": round(achieved, 2),
                        "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                        "peak_source": f"bf16_tflops_sustained ({pk_src})", "traffic": None,
                        "avg_launch_ms": round(tp / max(npx, 1), 3)},
           "e2e": e2e, "cpu_baseline": cpu, "clocks": clk}
    print(json.dumps(out))


def run_profile_sequence(args):
    """Fixed call sequences for ncu to capture (the lambda path with
    per-launch events; the derivative, X-gradient and post-processing calls):
    no timing, a few statistics."""
    import torch
    from paper_2412_11554_gb300 import build as B
    B.build()
    import paper_2412_11554_gb300 as A
    if args.workload == "path":
        from synth import path_workload
        pw = path_workload()
        X = torch.as_tensor(pw.X, device="cuda")
        r = A.accord_path(X, pw.subsamples, pw.lambdas, profile=1, omega_best=False, tau_warm=0, precision="mixed",
                          kkt_tol=pw.kkt_tol, max_iter=2000)
        torch.cuda.synchronize()
        print(json.dumps({"solve_ms": r.stats.t_solve_ms, "prox_ms": r.stats.t_prox_gemm_ms,
                          "prox_launches": r.stats.n_prox_gemm, "iters": r.stats.iters, "trials": r.stats.trials,
                          "status": r.status}))
    elif args.workload == "diff":
        from synth import diff_workload
        w = diff_workload()
        Xt, Xv = torch.as_tensor(w.X_train, device="cuda"), torch.as_tensor(w.X_val, device="cuda")
        O, st = A.accord_fit(Xt, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=20000)
        for _ in range(3):
            d, lv, _ = A.accord_dloss_dloglam(Xt, Xv, O, w.lam)
            A.accord_grad_x(Xt, O)
        p = 16000
        gen = torch.Generator(device="cuda").manual_seed(1)
        Om = torch.eye(p, device="cuda") + 0.01 * (torch.rand(p, p, device="cuda", generator=gen) < 0.01).float()
        for _ in range(3):
            A.accord_postprocess(Om)
        torch.cuda.synchronize()
        print(json.dumps({"dloss": d, "status": st.status, "nnz_offdiag": st.nnz_offdiag}))
    else:
        raise SystemExit("--profile-run applies to --workload path or diff")


def main():
    args = parse()
    if args.profile_run:
        run_profile_sequence(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "path":
        run_path(args)
    elif args.workload == "diff":
        run_diff(args)
    elif args.workload == "refit":
        run_refit(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
