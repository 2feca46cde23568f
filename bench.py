#!/usr/bin/env python3
"""H_eff*psi benchmark on GB300: FP64-equivalent TFLOP/s of the two-site DMRG
effective-Hamiltonian product and Davidson time-to-eigenvalue, one JSON line.

A step is one H_eff*psi over nvec vectors of the named synthetic workload with
operators resident in HBM, run the way the library runs it by default (each apply
replayed as a CUDA graph).  `value` = algorithmic flops (min-order plan count, the
same for every precision) x steps / device time of the split-precision path.  The
line also carries the plain FP64 path on the same workload (rate, fraction of the
FP64 tensor peak), the relative difference of the two results and of both from the
oracle on sampled entries, and the Davidson time to the eigenvalue, split vs FP64.
Per-kernel CUDA-event timing (for the roofline) runs in a separate pass of the same
steps, launched directly.  Under torchrun every rank runs an independent replica (the
product does not shard); value sums the ranks' work over the slowest rank's time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config precision]
                    [--precision split|fp64] [--nvec 1] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hψ FP64-equiv TFLOP/s; Davidson time-to-E, split vs FP64 (|ΔE/E|≤1e-10)"
UNIT = "TFLOP/s"
SPLIT_PAIRS = 21   # BF16 slice-pair products per FP64-equivalent product (6 slices, i+j<=5)
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SPLIT_ARITH = ("FP64-equivalent: every FP64 operand cut into 6 BF16 digit slices, 21 slice-pair "
               "products on tcgen05 with exactly representable FP32 partial sums for levels 0-3, "
               "recombined in int64 fixed point, FP64 output")
# DRAM bytes per launch of the dominant kernel from one ncu capture, keyed by the sha256
# of the kernel source it was taken on and the workload it was taken on.  "alg" is the
# algorithmic bytes per launch of the captured case: a capture of a smaller case of the
# same workload (fewer terms) is scaled to a full launch by the ratio of algorithmic
# bytes.  A changed kernel, or a workload without a capture, reports null.
NCU_TRAFFIC = {
    # k_umma, mid workload: (507.8 + 594.0 + 507.5 + 594.4) / 4 MB per launch
    # (profiles/split_umma_mid.md)
    ("f62b783283bb5466dde7e40be8d46d080ad38ae0a71c9bcc1cab68db999bd095", "mid"): dict(traffic=550.9e6),
    # k_fp64_tiles, mid workload: (280.7 + 363.6) / 2 MB per launch (profiles/fp64_tiles_mid.md)
    ("650a109e74edab18a3dc989256a122e4e1942d7c6ca9fc79c7845bd665ff2377", "mid"): dict(traffic=322.2e6),
    # spin-adapted su2_mid (profiles/su2_mid.md): k_umma (1339.9 + 1309.7 + 1336.5 +
    # 1309.7) / 4 MB, k_fp64_tiles (708.3 + 992.7) / 2 MB per launch
    ("f62b783283bb5466dde7e40be8d46d080ad38ae0a71c9bcc1cab68db999bd095", "su2_mid"): dict(traffic=1323.9e6),
    ("650a109e74edab18a3dc989256a122e4e1942d7c6ca9fc79c7845bd665ff2377", "su2_mid"): dict(traffic=850.5e6),
    # k_umma, precision workload, captured on its first 200 terms: (2651.0 + 2655.3) / 2 MB
    # per launch against 2580.4 MB of algorithmic bytes per launch (profiles/split_umma_precision.md)
    ("f62b783283bb5466dde7e40be8d46d080ad38ae0a71c9bcc1cab68db999bd095", "precision"):
        dict(traffic=2653.2e6, alg=2580436912),
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="precision")
    ap.add_argument("--precision", default="split", help="split (Ozaki BF16 slices, default) or fp64")
    ap.add_argument("--nvec", type=int, default=1)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--terms", type=int, default=None, help="fewer terms than the workload (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample length")
    ap.add_argument("--oracle-entries", type=int, default=200,
                    help="output entries the oracle checks on the bench workload (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-davidson", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 path on the bench workload")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedule")
    ap.add_argument("--no-per-gemm", action="store_true", help="skip the one-launch-per-GEMM comparison")
    ap.add_argument("--no-su2", action="store_true", help="skip the spin-adapted (SU(2)) measurement")
    ap.add_argument("--no-update-steps", action="store_true",
                    help="skip timing the truncation and renormalisation steps of the update")
    return ap.parse_args(argv)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(vals, dist, device):
    """Element-wise maximum of a list of floats over all ranks (identity without dist)."""
    if dist is None:
        return list(vals)
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_tflops(flops_per_step, steps, world, t_max_ms):
    """Aggregate rate of `world` replicas that each ran `steps` steps within t_max_ms."""
    return flops_per_step * steps * world / (t_max_ms * 1e-3) / 1e12


def load_workload(name, seed, n_terms=None):
    """The named workload: U(1) (dmrg_synth) or spin-adapted (names su2_*)."""
    if name.startswith("su2_"):
        from dmrg_synth import su2 as G
        return G.generate(name, seed=seed, n_terms=n_terms)
    import dmrg_synth as S
    return S.generate(name, seed=seed, n_terms=n_terms)


def term_subset(p, n_terms):
    """The first n_terms terms of a U(1) workload (the same operator data): a bounded
    sample of the workload for the oracle."""
    if hasattr(p, "rank2") or n_terms >= p.n_terms:
        return p
    return dataclasses.replace(p, coef=p.coef[:n_terms], delta=p.delta[:n_terms], parity=p.parity[:n_terms],
                               a_off=p.a_off[:n_terms], b_off=p.b_off[:n_terms])


def oracle_for(p):
    """The oracle module of the problem's symmetry (apply, plan)."""
    if hasattr(p, "rank2"):
        from oracle import su2 as o
    else:
        from oracle import heff as o
    return o


def workload_config(p, args, precision):
    sub = '' if args.terms is None else f' (first {args.terms} terms)'
    common = {"sectors": int(len(p.left)), "terms": int(p.n_terms), "psi_dim": int(p.dim),
              "operator_GB": round(p.op_data.size * 8 / 1e9, 3), "nvec": args.nvec, "precision": precision,
              "l2": "inputs larger than L2 (all operator blocks are read every step)",
              "parallelism": "replicas"}
    if hasattr(p, "rank2"):
        from dmrg_synth import su2 as G
        cfg = G.CONFIGS[args.config]
        return {"workload": f"{args.config}{sub}: spin-adapted two-site H_eff, {cfg['D']} multiplets per block over "
                            f"{len(p.left)} (n,2S) sectors, T={p.n_terms} terms, target (n,2S)={tuple(p.target)}, "
                            f"|psi|={p.dim}, seed {args.seed}", "D": cfg["D"], **common}
    import dmrg_synth as S
    cfg = S.CONFIGS[args.config]
    return {"workload": f"{args.config}{sub}: two-site H_eff, D={cfg['D']} per block over {len(p.left)} (n,2Sz) "
                        f"sectors, T={p.n_terms} terms, |psi|={p.dim}, seed {args.seed}", "D": cfg["D"], **common}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except (OSError, ValueError):
        return {}


def kernel_sha(name: str) -> str:
    return hashlib.sha256(open(os.path.join(ROOT, "paper_2407_07411_gb300", "csrc", name), "rb").read()).hexdigest()


def ncu_traffic(src_name, config, alg_bytes_per_launch):
    """DRAM bytes per launch from the ncu capture table, scaled to this launch's
    algorithmic bytes when the capture was taken on a smaller case; None without one."""
    e = NCU_TRAFFIC.get((kernel_sha(src_name), config))
    if e is None:
        return None
    if "alg" in e:
        return round(e["traffic"] * alg_bytes_per_launch / e["alg"])
    return e["traffic"]


def split_peak(timed_long):
    """FP64-equivalent ceiling of the split path: the BF16 tensor peak / 21 slice pairs."""
    pk = peaks()
    key = "bf16_tflops_sustained" if timed_long else "bf16_tflops"
    bf16 = pk.get(key)
    if bf16 is None:
        bf16 = 1700.0 if timed_long else 1900.0
        return bf16 / SPLIT_PAIRS, f"profiling recipe fallback {bf16} TFLOP/s bf16 / {SPLIT_PAIRS} slice pairs"
    return bf16 / SPLIT_PAIRS, f"of measured: MEASURED_PEAKS.json {key} ({bf16} TFLOP/s bf16) / {SPLIT_PAIRS} slice pairs"


def roofline(stats, fp64_peak, timed_long, config):
    """Dominant kernel (largest summed event time) against its tensor peak."""
    by_kernel = {}
    for s in stats:
        k = s["name"].split("/")[0]
        d = by_kernel.setdefault(k, dict(ms=0.0, flops=0.0, bytes=0.0, launches=0))
        d["ms"] += s["ms_total"]; d["flops"] += s["flops_total"]; d["bytes"] += s["bytes_total"]
        d["launches"] += s["launches"]
    if not by_kernel:
        return None
    name, d = max(by_kernel.items(), key=lambda kv: kv[1]["ms"])
    if d["ms"] <= 0:
        return None
    achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
    if name.startswith("fp64"):
        peak, src, src_name = fp64_peak, "measured live: DMMA m16n8k16 probe (dmrg_probe_fp64_peak)", "k_fp64.cu"
    else:
        peak, src = split_peak(timed_long)
        src_name = "k_split.cu"
    alg = d["bytes"] / max(d["launches"], 1)
    return {"kernel": name, "bound": "tensor", "achieved": round(achieved, 4), "peak": round(peak, 4),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4) if peak else None,
            "traffic": ncu_traffic(src_name, config, alg) if config else None,
            "algorithmic_bytes_per_launch": round(alg), "launches": d["launches"],
            "avg_launch_ms": round(d["ms"] / max(d["launches"], 1), 5), "peak_source": src,
            "timing": "per-kernel CUDA events on the launching stream, in a pass of the same steps launched "
                      "directly (graph replay carries no per-kernel events)"}


def time_applies(h, X, Y, nvec, steps, st, barrier):
    """Device time (ms) of `steps` applies on stream st, CUDA events, barrier on both sides."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(st)
    for _ in range(steps):
        h.apply(X, Y, nvec=nvec)
    e1.record(st)
    barrier()
    return e0.elapsed_time(e1)


def update_steps(lib, h, p, fp64_peak, reps=5):
    """The steps after the eigensolver on this workload, CUDA events around each call:
    decomposition/truncation of a wave function to D = |psi| / 4 states, and
    renormalisation of every A_t block into random orthonormal bases keeping 60 % of each
    sector (FP64 flops 2 d_p d_q d'_q + 2 d'_p d_p d'_q per block)."""
    import numpy as np
    import torch
    out = {}
    psi = torch.from_numpy(p.random_vectors(1)[0]).cuda()
    D = max(1, p.dim // 4)
    h.svd_truncate(psi, D)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        h.svd_truncate(psi, D)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    out["svd_truncate"] = {"D": D, "ms": round(float(np.median(ts)), 4), "blocks": int(len(h.psi_blocks()))}
    rng = np.random.default_rng(0)
    dims = p.left[:, 2].astype(np.int32)
    new = np.maximum(1, np.ceil(0.6 * dims)).astype(np.int32)
    U = np.concatenate([np.linalg.qr(rng.standard_normal((d, d)))[0][:, :k].ravel() for d, k in zip(dims, new)])
    idx = {(int(n), int(s)): i for i, (n, s, _) in enumerate(p.left)}
    blocks, flops = [], 0
    for t in range(p.n_terms):
        for q in range(len(dims)):
            if p.a_off[t, q] >= 0:
                o = idx[(int(p.left[q][0]) + int(p.delta[t][0]), int(p.left[q][1]) + int(p.delta[t][1]))]
                blocks.append((q, o, int(p.a_off[t, q])))
                flops += 2 * int(dims[o]) * int(dims[q]) * int(new[q]) + 2 * int(new[o]) * int(dims[o]) * int(new[q])
    blocks = np.array(blocks, np.int64)
    n_out = int(sum(int(new[a]) * int(new[b]) for a, b, _ in blocks))
    Ud = torch.from_numpy(U).cuda()
    opd = torch.from_numpy(p.op_data).cuda()
    outd = torch.empty(n_out, dtype=torch.float64, device="cuda")
    lib.renormalise(dims, new, Ud, blocks, opd, outd)

    def timed(fn):
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))
    one_shot = timed(lambda: lib.renormalise(dims, new, Ud, blocks, opd, outd))
    plan = lib.Renorm(dims, new, blocks, opd.numel(), n_out)   # set-up once, outside the timing
    plan.run(Ud, opd, outd)
    ms = timed(lambda: plan.run(Ud, opd, outd))
    plan.close()
    tf = flops / (ms * 1e-3) / 1e12
    out["renormalise"] = {"blocks": int(len(blocks)), "ms": round(ms, 4), "fp64_tflops": round(tf, 4),
                          "frac_of_fp64_peak": round(tf / fp64_peak, 4) if fp64_peak else None,
                          "one_shot_ms": round(one_shot, 4),
                          "note": "dmrg_renorm_run of a plan built once (basis copy and transposition included); "
                                  "one_shot_ms: dmrg_renormalise, which also builds the plan and allocates"}
    del opd, outd, Ud
    return out


def davidson_run(h, x0, tol, warm_iters):
    """One timed dmrg_davidson solve from x0 (after an untimed warm-up of warm_iters
    steps that captures the apply graph of every basis size)."""
    import torch
    if warm_iters:
        h.davidson(torch.from_numpy(x0).cuda(), tol=1e-9, max_iter=warm_iters)
    return h.davidson(torch.from_numpy(x0).cuda(), tol=tol, max_iter=800)


def time_to_e(ev, info, e_ref):
    """First Rayleigh-Ritz step whose lowest Ritz value is within 1e-10 (relative) of e_ref."""
    import numpy as np
    th, tm = info["theta"], info["time"]
    hit = np.nonzero(np.abs(th - e_ref) <= 1e-10 * abs(e_ref))[0]
    return {"time_to_E_s": round(float(tm[hit[0]]), 5) if hit.size else None,
            "iters_to_E": int(hit[0]) + 1 if hit.size else None, "E": float(ev[0]),
            "rel_err_E": abs(float(ev[0]) - e_ref) / abs(e_ref), "iters": info["iters"],
            "converged": info["converged"], "resid_max": info["resid_max"], "seconds": round(info["seconds"], 5)}


def davidson_time_to_e(lib, p, args, h64=None, hsplit=None):
    """Davidson time-to-eigenvalue for the split and the FP64 path: wall time from the
    dmrg_davidson call to the first Rayleigh-Ritz step whose lowest Ritz value is within
    1e-10 (relative) of E_ref, the lowest eigenvalue of a GPU FP64 solve to a residual
    of 1e-10 (validated against the oracle's E0 by the test suite on this workload).
    On workloads other than tiny/mid the FP64 reference solve (same start vector) is
    the timed FP64 run."""
    import numpy as np
    import torch
    x0 = p.random_vectors(1)
    out = {"criterion": "|theta - E_ref| <= 1e-10 |E_ref|", "block": 1, "tol": 1e-9}
    own64 = h64 is None
    h64 = h64 or lib.HEff.from_problem(p, precision="fp64")
    small = args.config in ("tiny", "mid", "su2_tiny", "su2_mid")
    ref_ev, ref_info = davidson_run(h64, x0, 1e-10, 0 if small else 30)
    e_ref = float(ref_ev[0])
    out["E_ref"] = e_ref
    out["E_ref_source"] = f"GPU FP64 Davidson, residual {ref_info['resid_max']:.1e}, {ref_info['iters']} steps"
    own_split = hsplit is None
    hs = hsplit or lib.HEff.from_problem(p, precision="split_bf16")
    for prec, h in (("split", hs), ("fp64", h64)):
        if prec == "fp64" and not small:
            ev, info = ref_ev, ref_info
        else:
            ev, info = davidson_run(h, x0, 1e-9, 50)
        out[prec] = time_to_e(ev, info, e_ref)
    if out["split"]["time_to_E_s"] and out["fp64"]["time_to_E_s"]:
        out["fp64_over_split"] = round(out["fp64"]["time_to_E_s"] / out["split"]["time_to_E_s"], 3)
    # the same criterion for restarted Lanczos (small workloads only)
    if small:
        lz = {}
        for prec, h in (("split", hs), ("fp64", h64)):
            h.lanczos(torch.from_numpy(x0[0]).cuda(), tol=1e-9, max_iter=200)    # warm-up
            ev, info = h.lanczos(torch.from_numpy(x0[0]).cuda(), tol=1e-9, max_iter=3000)
            hit = np.nonzero(np.abs(info["theta"] - e_ref) <= 1e-10 * abs(e_ref))[0]
            lz[prec] = {"time_to_E_s": round(float(info["time"][hit[0]]), 5) if hit.size else None,
                        "iters_to_E": int(hit[0]) + 1 if hit.size else None, "E": ev,
                        "rel_err_E": abs(ev - e_ref) / abs(e_ref), "iters": info["iters"],
                        "converged": info["converged"], "seconds": round(info["seconds"], 5)}
        out["lanczos"] = lz
    if own64:
        h64.close()
    if own_split:
        hs.close()
    return out


def su2_section(lib, args, fp64_peak, steps=200):
    """Spin-adapted (SU(2)) H_eff*psi on the 1024-multiplet mid workload (600 terms,
    singlet target): FP64-equivalent TFLOP/s of both paths (graph replays after an
    autotune, CUDA events) with their fraction of the FP64 and BF16-per-pair peaks, the
    relative difference of the split result from the FP64 one, and Davidson (and
    Lanczos) time-to-eigenvalue split vs FP64."""
    import numpy as np
    import torch
    from dmrg_synth import su2 as G
    p = G.generate("su2_mid", seed=args.seed)
    X = torch.from_numpy(p.random_vectors(1)).cuda()
    st = torch.cuda.current_stream()
    out = {"workload": f"su2_mid: {int(p.left[:, 2].sum())} multiplets per block over {len(p.left)} (n,2S) sectors, "
                       f"T={p.n_terms} terms, singlet target (20,0), |psi|={p.dim}, seed {args.seed}",
           "operator_GB": round(p.op_data.size * 8 / 1e9, 3)}
    ys = {}
    for prec in ("fp64", "split"):
        h = lib.HEff.from_problem(p, precision="fp64" if prec == "fp64" else "split_bf16")
        h.autotune(nvec=1, reps=2)
        Y = torch.empty_like(X)
        for _ in range(3):
            h.apply(X, Y)
        ms = time_applies(h, X, Y, 1, steps, st, torch.cuda.synchronize) / steps
        tf = h.flops / (ms * 1e-3) / 1e12
        if prec == "fp64":
            pk, src = fp64_peak, "DMMA probe (dmrg_probe_fp64_peak)"
        else:
            pk, src = split_peak(False)
        out[prec] = {"ms_per_apply": round(ms, 5), "value": round(tf, 4), "unit": UNIT, "steps": steps,
                     "frac_of_peak": round(tf / pk, 4) if pk else None, "peak": round(pk, 4) if pk else None,
                     "peak_source": src}
        out["flops_per_apply"] = h.flops
        ys[prec] = Y.cpu().numpy()
        h.close()
    out["split_rel_fro_vs_fp64"] = float(np.linalg.norm(ys["split"] - ys["fp64"]) / np.linalg.norm(ys["fp64"]))
    a = argparse.Namespace(**{**vars(args), "config": "su2_mid"})
    out["davidson"] = davidson_time_to_e(lib, p, a)
    return out


def calibrate_terms(oheff, p, x, seconds_per_call):
    """Terms of a bounded oracle sample whose one call takes about seconds_per_call."""
    n0 = max(1, min(p.n_terms, 20))
    t0 = time.perf_counter()
    oheff.apply(term_subset(p, n0), x)
    per_term = (time.perf_counter() - t0) / n0
    return max(1, min(p.n_terms, int(seconds_per_call / max(per_term, 1e-9))))


def cpu_baseline(p, seconds):
    """The oracle as it stands, timed on the host cores on a bounded sample: full
    oracle H_eff*psi calls over the first T' terms of the bench workload (T' chosen
    so that one call takes about a quarter of the sample)."""
    import numpy as np
    oheff = oracle_for(p)
    x = p.random_vectors(1)[0]
    T = calibrate_terms(oheff, p, x, seconds / 4) if not hasattr(p, "rank2") else p.n_terms
    q = term_subset(p, T)
    flops = int(oheff.plan(q)[:, 4].sum())
    calls, t0, c0 = 0, time.perf_counter(), time.process_time()
    while True:
        oheff.apply(q, x)
        calls += 1
        wall = time.perf_counter() - t0
        if wall >= seconds:
            break
    cpu = time.process_time() - c0
    return {"value": round(flops * calls / wall / 1e12, 6), "unit": UNIT,
            "cores": round(cpu / wall, 2), "kind": "oracle",
            "sample": f"{calls} oracle H_eff*psi calls (numpy block loop) over the first {T} of {p.n_terms} terms "
                      f"of the bench workload ({flops / 1e9:.2f} GFLOP each), {wall:.1f} s wall; cores = process "
                      f"CPU time / wall time", "host_cores_available": os.cpu_count(), "_np": np.__version__}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    p = load_workload(args.config, args.seed)
    oheff = oracle_for(p)
    x = p.random_vectors(1)[0]
    # bounded sample: the first T' terms, so that warm-up + steps take about 150 s
    T = calibrate_terms(oheff, p, x, 150.0 / max(args.steps + args.warmup, 1)) if not hasattr(p, "rank2") \
        else p.n_terms
    q = term_subset(p, T)
    flops = int(oheff.plan(q)[:, 4].sum())
    for _ in range(args.warmup):
        oheff.apply(q, x)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        oheff.apply(q, x)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    value = flops * args.steps / wall / 1e12
    sample = (f"each step = one oracle H_eff*psi over {'all' if T >= p.n_terms else f'the first {T}'} of the "
              f"{p.n_terms} terms of the {args.config} workload")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded sector structure, random operator blocks)",
            "config": workload_config(p, args, "fp64 (oracle)"),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "kind": "oracle", "cores": round(cpu / wall, 2),
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_section(lib, p, X, nvec, steps_budget_ms, st, barrier, fp64_peak):
    """The plain FP64 path on the bench workload: FP64 TFLOP/s (graph replays, CUDA
    events) and its fraction of the FP64 tensor peak; returns (dict, handle, Y)."""
    import torch
    h = lib.HEff.from_problem(p, precision="fp64", max_nvec=nvec)
    Y = torch.empty_like(X)
    t0 = time.perf_counter()
    h.apply(X, Y, nvec=nvec)     # warm-up (captures the graph)
    torch.cuda.synchronize()
    one = (time.perf_counter() - t0) * 1e3
    steps = max(3, min(50, int(steps_budget_ms / max(one, 1e-3))))
    ms = time_applies(h, X, Y, nvec, steps, st, barrier) / steps
    tf = h.flops * nvec / (ms * 1e-3) / 1e12
    return ({"ms_per_apply": round(ms, 5), "value": round(tf, 4), "unit": UNIT, "steps": steps,
             "frac_of_fp64_peak": round(tf / fp64_peak, 4) if fp64_peak else None,
             "peak": round(fp64_peak, 4) if fp64_peak else None,
             "peak_source": "measured live: DMMA m16n8k16 probe (dmrg_probe_fp64_peak); MEASURED_PEAKS.json "
                            "has no FP64 entry"}, h, Y)


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2407_07411_gb300 as lib

    precision = {"fp64": "fp64", "split": "split_bf16", "split_bf16": "split_bf16"}[args.precision]
    p = load_workload(args.config, args.seed, n_terms=args.terms)
    h = lib.HEff.from_problem(p, precision=precision, max_nvec=args.nvec)
    flops_vec = h.flops
    fp64_peak = lib.probe_fp64_peak()
    tune = None
    if not args.no_autotune:   # untimed: the schedule the timed steps run with
        t0 = time.perf_counter()
        tune = h.autotune(nvec=args.nvec, reps=3)
        tune["seconds"] = round(time.perf_counter() - t0, 3)
        tune["default_ms"], tune["best_ms"] = round(tune["default_ms"], 5), round(tune["best_ms"], 5)
    X = torch.from_numpy(p.random_vectors(args.nvec)).cuda()
    Y = torch.empty_like(X)
    st = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        h.apply(X, Y, nvec=args.nvec)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # timed steps: the product's default path (every apply a CUDA graph replay)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].isdigit() else local
    h.profile(False)            # resets the launch counters; graph replays keep counting
    with ClockSampler(gpu_index) as clk:
        ms = time_applies(h, X, Y, args.nvec, args.steps, st, barrier)
    launches = sum(s["launches"] for s in h.profile_read())
    t_max = max_over_ranks([ms], dist, "cuda")[0]
    value = whole_job_tflops(flops_vec * args.nvec, args.steps, ws, t_max)
    y_main = Y.cpu().numpy()

    # per-kernel CUDA events (direct launches) over the same number of steps: roofline
    h.profile(True)
    p_ms = time_applies(h, X, Y, args.nvec, args.steps, st, barrier)
    stats = h.profile_read()
    h.profile(False)
    profiled = {"ms_per_step": round(p_ms / args.steps, 5),
                "value": round(whole_job_tflops(flops_vec * args.nvec, args.steps, ws, p_ms), 6),
                "note": "the same steps launched directly with per-kernel CUDA events (feeds roofline)"}

    # end to end through the public host API: pinned H2D of x, apply, D2H of y
    xh = torch.from_numpy(p.random_vectors(args.nvec)).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    for _ in range(2):
        h.apply_host_ptr(xh.data_ptr(), yh.data_ptr(), args.nvec)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h.apply_host_ptr(xh.data_ptr(), yh.data_ptr(), args.nvec)
    e2e_s = max_over_ranks([time.perf_counter() - t0], dist, "cuda")[0]
    nbytes = args.nvec * p.dim * 8
    e2e = {"value": round(whole_job_tflops(flops_vec * args.nvec, e2e_steps, ws, e2e_s * 1e3), 6), "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
           "api": "dmrg_heff_apply_host (pinned host buffers, synchronous)"}

    # the same apply with one launch per grouped GEMM (each stage's persistent launch split
    # into a launch per GEMM), everything else unchanged
    per_gemm = None
    if not args.no_per_gemm:
        sched = h.schedule
        h.schedule = dict(sched, per_gemm=1)
        pg_steps = max(3, min(args.steps, int(3000.0 / max(t_max / args.steps, 1e-3))))
        h.apply(X, Y, nvec=args.nvec)
        pg_ms = max_over_ranks([time_applies(h, X, Y, args.nvec, pg_steps, st, barrier)], dist, "cuda")[0]
        h.schedule = sched
        per_gemm = {"steps": pg_steps, "ms_per_step": round(pg_ms / pg_steps, 5),
                    "value": round(whole_job_tflops(flops_vec * args.nvec, pg_steps, ws, pg_ms), 6),
                    "gemm_launches_per_step": sum(h.gemm_count(args.nvec)),
                    "batched_speedup": round((pg_ms / pg_steps) / (t_max / args.steps), 3)}

    split = precision != "fp64"
    cfg_key = args.config if args.terms is None and args.nvec == 1 else None
    line = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64-equivalent (6 bf16 slices)" if split else "f64",
            "arith": SPLIT_ARITH if split else "FP64 DMMA tensor cores (mma.sync m16n8k16), FP64 accumulation",
            "data": "synthetic (seeded sector structure, random operator blocks)",
            "config": workload_config(p, args, precision),
            "timing": "CUDA events on the launching stream around K graph-replayed applies, barrier + synchronize "
                      "on both sides; operators larger than L2 are read every step",
            "roofline": roofline(stats, fp64_peak, timed_long=p_ms > 2000, config=cfg_key),
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches, "profiled": profiled,
            "autotune": tune, "per_gemm": per_gemm,
            "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in s.items()} for s in stats],
            "flops_per_step": flops_vec * args.nvec}

    line["memory_GB"] = {k: round(v / 1e9, 3) for k, v in h.memory().items()}
    # a workload whose split and FP64 handles do not fit the device together (large):
    # the split Davidson solve runs first, its handle is closed, then the FP64 path
    h64 = None
    seq = False
    if rank == 0 and split and not args.no_fp64:
        free, _ = torch.cuda.mem_get_info()
        hp = lib.HEff.from_problem(p, precision="fp64", plan_only=True, max_nvec=args.nvec)
        seq = hp.memory()["total"] > free - (4 << 30)
        hp.close()
    x0 = p.random_vectors(1)
    dav_split = None
    if seq:
        if not args.no_davidson:
            dav_split = davidson_run(h, x0, 1e-8, 20)
        h.close()
        h = None
        torch.cuda.empty_cache()
    if rank == 0 and split and not args.no_fp64:
        fp, h64, Y64 = fp64_section(lib, p, X, args.nvec, 6000.0, st, barrier, fp64_peak)
        y64 = Y64.cpu().numpy()
        fp["split_over_fp64_speed"] = round(value / ws / fp["value"], 3) if fp["value"] else None
        line["fp64"] = fp
        line["split_rel_fro_vs_fp64"] = float(np.linalg.norm(y_main - y64) / np.linalg.norm(y64))
        del Y64
    if rank == 0 and args.oracle_entries > 0 and not hasattr(p, "rank2"):
        # both results against the oracle on sampled output entries (vector 0)
        from oracle import heff as oheff
        idx = np.sort(np.random.default_rng(4).choice(p.dim, min(args.oracle_entries, p.dim), replace=False))
        t0 = time.perf_counter()
        ref = oheff.apply_entries(p, X[0].cpu().numpy(), idx)
        nr = np.linalg.norm(ref)
        chk = {"entries": int(len(idx)), "seconds": round(time.perf_counter() - t0, 2),
               f"{'split' if split else 'fp64'}_rel_fro": float(np.linalg.norm(y_main[0][idx] - ref) / nr)}
        if "fp64" in line:
            chk["fp64_rel_fro"] = float(np.linalg.norm(y64[0][idx] - ref) / nr)
        chk["tolerance"] = {"split": 1e-11, "fp64": 1e-12}
        line["oracle_check"] = chk
    if rank == 0 and not args.no_davidson and seq:
        ev64, info64 = davidson_run(h64, x0, 1e-8, 0)
        e_ref = float(ev64[0])
        dav = {"criterion": "|theta - E_ref| <= 1e-10 |E_ref|", "block": 1, "tol": 1e-8, "E_ref": e_ref,
               "E_ref_source": f"GPU FP64 Davidson, residual {info64['resid_max']:.1e}, {info64['iters']} steps",
               "split": time_to_e(*dav_split, e_ref), "fp64": time_to_e(ev64, info64, e_ref),
               "note": "both solves to residual 1e-8 from the same start vector, one after the other (the two "
                       "handles do not fit the device together); the FP64 solve is the reference"}
        dav["split_minus_fp64_E"] = float(dav_split[0][0]) - e_ref
        if dav["split"]["time_to_E_s"] and dav["fp64"]["time_to_E_s"]:
            dav["fp64_over_split"] = round(dav["fp64"]["time_to_E_s"] / dav["split"]["time_to_E_s"], 3)
        line["davidson"] = dav
    elif rank == 0 and not args.no_davidson:
        line["davidson"] = davidson_time_to_e(lib, p, args, h64=h64, hsplit=h if split and args.nvec == 1 else None)
    if h64 is not None:
        h64.close()
    if rank == 0 and not args.no_su2 and args.config == "mid":
        line["su2"] = su2_section(lib, args, fp64_peak)
    if rank == 0 and h is not None and not args.no_update_steps and args.config in ("tiny", "mid", "precision"):
        line["update_steps"] = update_steps(lib, h, p, fp64_peak)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
        line["cpu_baseline"].pop("_np", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if h is not None:
        h.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
