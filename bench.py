"""Benchmark of the columnwise W, V setup (direct approximate factoring of the
inverse) on one GB300, printing one JSON line.

Workload (default): 2D upwind convection-diffusion on a 256 x 256 grid
(n = 65,536), W pattern = pattern(A^2) (<= 13 indices per column), V = the
optimal upper-triangular pattern chosen by the leverage rule with the
Gauss-Seidel budget, DIAF-S (unit w_j), b = A ones.

One step = one pass of the whole hot path over the workload: the setup
(symbolic pass, gather, QR, V rule, DIAF solve, scatter into CSC W and V)
plus one application of W V^-1 (row-oriented copies and the triangular
solve).  value = columns per second of that step with the inputs resident in
HBM; L2 is flushed (a 256 MiB write) before every timed step.  e2e = the same
through the public API from pinned host buffers, with the inputs copied in
and W, V, the residuals copied out inside the timed region (the copy out on
a second stream, beside the apply: they are final once diaf_factor is done).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl diaf|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import make_workload  # noqa: E402

UNIT = "columns/s"
# the workloads in words, for the metric string
WORKLOAD_TEXT = {
    "convdiff32": "32x32 convection-diffusion, W = pattern(A)",
    "convdiff256_A2": "256x256 convection-diffusion, W = pattern(A^2)",
    "powerlaw200k": "power-law random n = 200,000, W = pattern(A)",
    "helmholtz512": "512x512 complex shifted Helmholtz, W = pattern(A)",
    "lognormal64": "64^3 lognormal diffusion-convection, W = pattern(A^2)",
}


def metric_name(workload: str, alg: str) -> str:
    return (f"W,V setup columns/s (DIAF-{alg}, {WORKLOAD_TEXT.get(workload, workload)}); "
            "vs plain FP64 GPU form")


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant numeric kernel, from one ncu capture of the current kernel per
# (workload, algorithm, precision) (profiles/); None elsewhere.
TRAFFIC = {
    ("convdiff2d_256x256_Wp2", "S", "mixed32"): 27_404_544 + 25_064_704,   # column_thread_kernel<16>
    ("convdiff2d_256x256_Wp2", "S", "fp64"): 24_367_104 + 768,             # column_warp_kernel<double,16,32,S>
    ("helmholtz2d_512x512", "S", "mixed32"): 133_269_248 + 48_194_304,     # column_mixed_kernel<Cx<float>,16,32,S>
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ALU peaks of the GB300 (the peaks file measures only copy bandwidth and
# bf16 GEMM): FP32 = 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
# = 80.5 TFLOP/s; FP64 = 1.25 TFLOP/s nominal.
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_NOMINAL_TFLOPS = 1.25


JACOBI_SWEEPS = 5  # mean sweeps of the FP32 Jacobi on the headline workload (phase-timer build)


def dominant_kernel(bucket: int, prec: str, alg: str, cplx: bool) -> str:
    """Name of the numeric kernel that runs size bucket `bucket` (0: tiles up
    to 32 x 16, 1: up to 64 x 32, 2: larger) for this precision and form."""
    if prec == "fp64":
        return "column_cta_kernel" if bucket == 2 else "column_warp_kernel"
    if bucket == 2:
        return "column_cta_mixed_kernel" if (alg == "S" and not cplx) else "column_cta_kernel (FP64)"
    if bucket == 0 and alg == "S" and not cplx:
        return "column_thread_kernel (four lanes per column)"
    return "column_mixed_kernel"


def algorithmic_flops(m: np.ndarray, k: np.ndarray, l: np.ndarray, alg: str, cplx: bool,
                      sweeps: float = JACOBI_SWEEPS) -> tuple[float, float]:
    """(all flops, FP64 flops) the method does per factorisation, summed over
    the columns: QR of the m x k tile 2k^2(m - k/3), leverage keys m k^2,
    then DIAF-S: QR of the tile without the I_j rows, one-sided Jacobi on its
    k x k R -- `sweeps` sweeps of k(k-1)/2 rotations, each a 2k-flop inner
    product and two 6k-flop column-pair updates (R and V) --, the FP64
    correction (H x = A-hat^T A-hat x: 4 m k) and v, residual (2 m k);
    DIAF-Q: Jacobi on the l x k Q_I, the FP64 correction and solves
    (4 m k + 2 k^2), v, residual.  Complex arithmetic counts 4x."""
    m = m.astype(np.float64); k = k.astype(np.float64); l = l.astype(np.float64)
    f32 = 2 * k**2 * (m - k / 3) + m * k**2
    if alg == "S":
        f32 += 2 * k**2 * (np.maximum(m - l, k) - k / 3) + sweeps * k * (k - 1) / 2 * 14 * k
        f64 = 4 * m * k + 2 * m * k
    else:
        f32 += sweeps * k * (k - 1) / 2 * (8 * l + 6 * k)
        f64 = 4 * m * k + 2 * k**2 + 2 * m * k
    c = 4 if cplx else 1
    return float((f32 + f64).sum() * c), float(f64.sum() * c)


def gathered_bytes(w) -> float:
    """Bytes the gather of every tile reads: each J_j column's entries of A
    (value and row index) once per column j that uses it."""
    nnz = np.diff(w.A.colptr).astype(np.float64)
    per = 16.0 + 4.0 if w.A.is_complex else 8.0 + 4.0
    return float(nnz[w.PW.rowidx].sum() * per)


def tile_sizes(w):
    """m_j = |R_j| and k_j of the workload (structure only)."""
    import scipy.sparse as sp
    A, PW = w.A, w.PW
    B = sp.csc_matrix((np.ones(A.nnz), A.rowidx, A.colptr), shape=(A.n, A.n))
    P = sp.csc_matrix((np.ones(PW.nnz), PW.rowidx, PW.colptr), shape=(A.n, A.n))
    m = np.diff((B @ P).tocsc().indptr)
    return m, PW.counts()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        # returns once the sampler has printed its first line, so that it is
        # live when the timed region starts; that line (taken before the
        # region) is kept only as a fallback for regions shorter than a period
        self.first = ""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            import select
            if select.select([self.proc.stdout], [], [], 10.0)[0]:
                self.first = self.proc.stdout.readline()
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [r.split(", ") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        during = len(rows)
        if not rows:
            rows = [r.split(", ") for r in (self.first or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": during,
                **({} if during else {"note": "timed region shorter than the 100 ms sampling period: "
                                              "the sample taken just before it"})}


def cpu_baseline(w, alg, seconds=12.0):
    """The oracle as it stands, on this host's cores, on whole passes over the
    workload's columns until about `seconds` of CPU work."""
    import oracle as O
    cores = os.cpu_count() or 1
    O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, cols=np.arange(64, dtype=np.int32))  # build + warm
    t0 = time.perf_counter()
    cols = 0
    passes = 0
    while time.perf_counter() - t0 < seconds:
        O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol, nthreads=cores)
        cols += w.n
        passes += 1
    dt = time.perf_counter() - t0
    return {"value": cols / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{passes} full pass(es) over all {w.n} columns ({dt:.1f} s, OpenMP over columns)"}


def run_reference(args):
    """--impl reference: the CPU oracle, timed on the host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.workload, alg=args.alg)
    import oracle as O
    cores = os.cpu_count() or 1
    O.factor(w.A, w.PW, w.vrule, w.budget, alg=args.alg, cols=np.arange(64, dtype=np.int32))
    for _ in range(args.warmup):
        O.factor(w.A, w.PW, w.vrule, w.budget, alg=args.alg, tie_tol=w.tie_tol, nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.factor(w.A, w.PW, w.vrule, w.budget, alg=args.alg, tie_tol=w.tie_tol, nthreads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    val = w.n / (ms / 1e3)
    line = {"impl": "reference", "metric": metric_name(args.workload, args.alg), "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "alg": args.alg, "columns_per_step": w.n},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full pass(es) over all {w.n} columns"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def learned_report(dev, keep=12, train_N=40, train_seeds=(11, 12), eval_N=64, epochs=20, powers=(2, 3)):
    """The learned J_j proposal against the fixed sparsified-powers rule at
    equal nnz(W), on the eval_N^3 lognormal operator: one network per
    candidate set pattern(A^p), trained from scratch on the GPU (targets from
    FP64 solves with a diagonal V on train_N^3 instances of other seeds), and
    every rule evaluated with a diagonal V and with the configuration's own
    upper-triangular V: ||A W V^-1 - I||_F^2 (diagonal V), median scaled
    column residual, setup time, BiCGSTAB to 1e-8 (iterations counted as
    differing only when they differ by more than 2)."""
    import torch
    from paper_1208_3573_gb300 import diaf
    from paper_1208_3573_gb300.learned import Proposer, fixed_rule, host_pattern, toggle_targets, scaled_residuals
    from workloads import patterns as pats
    from workloads.configs import lognormal

    def events(fn, reps=5):
        out, ts = None, []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(); out = fn(); e1.record(); e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return out, statistics.median(ts)

    w = lognormal(eval_N, 0)
    Ad = diaf.DeviceCSC.from_host(w.A, dev)
    b = torch.from_numpy(w.b).to(dev)
    S = diaf.Solver(Ad)
    FR, fixed_ms = events(lambda: fixed_rule(Ad, keep))
    rules = {"fixed_sparsified_powers": FR}
    out = {"workload": w.name, "keep": keep, "fixed_rule_ms": fixed_ms, "train": {}}
    for p in powers:
        t0 = time.perf_counter()
        feats, targs = [], []
        for seed in train_seeds:
            wt = lognormal(train_N, seed)
            ones = torch.ones(wt.n, dtype=torch.int32, device=dev)
            CAND = pats.pattern_power(wt.A, p)
            At = diaf.DeviceCSC.from_host(wt.A, dev)
            T = toggle_targets(At, CAND, host_pattern(fixed_rule(At, keep)), ones, wt.vrule, wt.tie_tol)
            feats.append(diaf.propose_features(At, diaf.DeviceCSC.from_host(CAND, dev)))
            targs.append(T.value)
        torch.cuda.synchronize()
        t_targets = time.perf_counter() - t0
        net = Proposer(seed=0, device=dev)
        t0 = time.perf_counter()
        hist = net.fit(feats, targs, epochs=epochs, batch=4096, lr=3e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        CANDe = diaf.DeviceCSC.from_host(pats.pattern_power(w.A, p), dev)
        J, propose_ms = events(lambda: net.propose(Ad, CANDe, keep))
        name = f"learned_A{p}"
        rules[name] = J
        out["train"][name] = {"candidates": f"pattern(A^{p}) (at most {int(torch.diff(CANDe.colptr).max())} "
                                            f"per column)", "instances": f"{train_N}^3 seeds {list(train_seeds)}",
                              "targets_s": t_targets, "train_s": t_train,
                              "rows": int(sum(torch.isfinite(t).sum().item() for t in targs)),
                              "loss_first": hist[0], "loss_last": hist[-1], "propose_ms": propose_ms}
    for vname, budget in (("V_diagonal", np.ones(w.n, dtype=np.int32)), ("V_upper_config", w.budget)):
        bud = torch.from_numpy(budget).to(dev)
        res = {}
        for name, P in rules.items():
            r = {"nnz_W": P.nnz}
            _, r["factor_ms_mixed32"] = events(lambda: diaf.factor(Ad, P, w.vrule, bud, alg="S", prec="mixed32",
                                                                   tie_tol=w.tie_tol), 3)
            F, r["factor_ms_fp64"] = events(lambda: diaf.factor(Ad, P, w.vrule, bud, alg="S", prec="fp64",
                                                                tie_tol=w.tie_tol), 3)
            sr = scaled_residuals(F)
            if vname == "V_diagonal":
                r["fro2_AWVinv_minus_I"] = float(np.sum(sr ** 2))
            r["colres_median"] = float(np.median(sr))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                _, info = S.bicgstab(b, F, tol=1e-8, maxit=2000)
                torch.cuda.synchronize()
                r.update(bicgstab_its=info.iterations, converged=bool(info.converged),
                         breakdown=bool(info.breakdown), relres=float(info.relres),
                         solve_ms=1e3 * (time.perf_counter() - t0))
            except diaf.DiafError as e:  # e.g. a zero diagonal entry of V
                r.update(bicgstab_its=None, converged=False, error=str(e)[:160])
            F.close()
            res[name] = r
        f = res["fixed_sparsified_powers"]
        for name in rules:
            if name.startswith("learned") and f.get("converged") and res[name].get("converged"):
                d = f["bicgstab_its"] - res[name]["bicgstab_its"]
                res[name]["its_gain_vs_fixed"] = d
                res[name]["gain_beyond_jitter"] = abs(d) > 2
        out[vname] = res
    return out


def kv_sweep(w, A, PW, alg, prec, dev, budgets=(1, 2, 3, 4, 6, 8, 13)):
    """The k_V sweep of Sec. 5 on this workload: at most k_V entries per
    column of V (upper rule): ||A W - V||_F, setup time, BiCGSTAB to 1e-8 --
    for the configured algorithm and for the stabilised DIAF-Q of Sec. 3.2
    (trigger |v_jj| < 1e-2, v_jj imposed as 2: the paper's Table 6 setting),
    with the number of stabilised columns."""
    import torch
    from paper_1208_3573_gb300 import diaf
    S = diaf.Solver(A)
    b = torch.from_numpy(w.b).to(dev)

    def run(bud, a, stab):
        F = diaf.factor(A, PW, w.vrule, bud, alg=a, prec=prec, tie_tol=w.tie_tol, stab_tol=stab, stab_r=2.0)
        res = F.res.cpu().numpy()
        fl = F.flags.cpu().numpy()
        row = {"nnz_V": int(F.V.nnz), "nrm_AW_minus_V": float(np.sqrt(np.sum(res ** 2))),
               "setup_ms": F.timings()["total_ms"], "vjj_zero_columns": int(np.count_nonzero(fl & 4))}
        if stab > 0:
            row["stabilised_columns"] = int(np.count_nonzero(fl & 128))
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = S.bicgstab(b, F, tol=1e-8, maxit=1000)
            torch.cuda.synchronize()
            row.update(bicgstab_its=info.iterations, converged=bool(info.converged),
                       breakdown=bool(info.breakdown), relres=float(info.relres),
                       solve_ms=1e3 * (time.perf_counter() - t0))
        except diaf.DiafError as e:  # no solve: V has a zero or missing diagonal entry
            row.update(converged=False, solve=str(e)[:80])
        F.close()
        return row

    out = []
    for kv in budgets:
        bud = torch.full((w.n,), kv, dtype=torch.int32, device=dev)
        out.append({"k_V": kv, f"DIAF-{alg}": run(bud, alg, 0.0), "DIAF-Q stabilised": run(bud, "Q", 1e-2)})
    return out


def block_v_report(w, A, PW, alg, prec, dev, bsize=64, budgets=(4, 8, 16)):
    """Block-diagonal V (the V structure of the paper's experiments, Sec. 5)
    on this workload: contiguous blocks of `bsize` rows, at most k_V entries
    per column chosen by the leverage rule inside the block."""
    import torch
    from paper_1208_3573_gb300 import diaf
    S = diaf.Solver(A)
    b = torch.from_numpy(w.b).to(dev)
    blk = diaf.contiguous_blocks(w.n, bsize, device=dev)
    x = torch.ones(w.n, dtype=b.dtype, device=dev)
    y = torch.empty_like(x)
    out = []
    for kv in budgets:
        bud = torch.full((w.n,), kv, dtype=torch.int32, device=dev)
        F = diaf.factor(A, PW, diaf.RULE_BLOCK, bud, alg=alg, prec=prec, tie_tol=w.tie_tol, blocks=blk)
        row = {"block_rows": bsize, "k_V": kv, "setup_ms": F.timings()["total_ms"], "nnz_V": int(F.V.nnz),
               "nrm_AW_minus_V": float(np.sqrt(np.sum(F.res.cpu().numpy() ** 2)))}
        try:
            F.apply(x, y)  # prepares the block LU
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(); F.apply(x, y); e1.record(); e1.synchronize()
            row["apply_ms"] = e0.elapsed_time(e1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = S.bicgstab(b, F, tol=1e-8, maxit=1000)
            torch.cuda.synchronize()
            row.update(bicgstab_its=info.iterations, converged=bool(info.converged),
                       solve_ms=1e3 * (time.perf_counter() - t0))
        except diaf.DiafError as e:
            row["solve"] = str(e)[:80]
        F.close()
        out.append(row)
    return out


def rank_max(x: float, world: int) -> float:
    """The largest value of x over the ranks (the slowest rank's time); the
    process group's backend decides where the reduction tensor lives."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ms_local: float, world: int) -> tuple[float, float]:
    """(units/s of the whole job, step ms): every rank processes units_per_rank
    in ms_local; the job takes as long as its slowest rank."""
    ms = rank_max(ms_local, world)
    return world * units_per_rank / (ms / 1e3), ms


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="diaf", choices=["diaf", "reference"])
    ap.add_argument("--workload", default="convdiff256_A2")
    ap.add_argument("--alg", default="S", choices=["S", "Q"])
    ap.add_argument("--prec", default="mixed32", choices=["fp64", "mixed32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the solve / other-form side measurements")
    ap.add_argument("--no-autotune", action="store_true", help="default launch tuning instead of diaf_autotune")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned J_j proposal report")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1208_3573_gb300 import diaf

    w = make_workload(args.workload, alg=args.alg)
    cplx = w.A.is_complex
    A = diaf.DeviceCSC.from_host(w.A)
    PW = diaf.DeviceCSC.from_host(w.PW)
    bud = torch.from_numpy(w.budget).to(dev)
    x1 = torch.ones(w.n, dtype=torch.complex128 if cplx else torch.float64, device=dev)
    y1 = torch.empty_like(x1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    do_apply = w.meta.get("apply", True)
    tuning, tune_ms = None, None
    if not args.no_autotune:  # once, before the warm-up (not timed)
        tuning, tune_ms = diaf.autotune(A, PW, w.vrule, bud, alg=args.alg, prec=args.prec, tie_tol=w.tie_tol)

    def step(Ad, PWd, budd):
        F = diaf.factor(Ad, PWd, w.vrule, budd, alg=args.alg, prec=args.prec, tie_tol=w.tie_tol, stream=stream,
                        tuning=tuning)
        if do_apply:
            F.apply(x1, y1, stream=stream)
        return F

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    lcount = None
    for _ in range(args.warmup):
        F = step(A, PW, bud)
        if lcount is None:
            lcount = np.diff(F.V.colptr.cpu().numpy())
        F.close()
    barrier()

    # ---- timed region (device-resident inputs)
    launches0 = diaf.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms, numeric_ms, total_ms, bucket_cols = [], [], [], None
    with ClockSampler(local) as clk:
        barrier()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            F = step(A, PW, bud)
            ev[i][1].record(stream)
            t = F.timings()
            kern_ms.append(t["bucket_ms"])
            numeric_ms.append(t["numeric_ms"])
            total_ms.append(t["total_ms"])
            if lcount is None:
                lcount = np.diff(F.V.colptr.cpu().numpy())
            bucket_cols = t["bucket_cols"]
            F.close()
        barrier()
    launches = diaf.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, ms = whole_job_rate(w.n, float(np.mean(step_ms)), world)

    # ---- e2e through the public API from pinned host buffers
    def pin(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()

    hA = [pin(w.A.colptr), pin(w.A.rowidx), pin(w.A.vals)]
    hP = [pin(w.PW.colptr), pin(w.PW.rowidx)]
    hB = pin(w.budget)
    h2d = sum(t.numel() * t.element_size() for t in hA + hP + [hB])
    e2e_ms = []
    d2h = 0
    host = None  # pinned output buffers, allocated in the untimed first pass and reused
    # W, V and the residuals are final once diaf_factor's numeric pass is done:
    # their copy back runs on a second stream while the apply runs
    copy_stream = torch.cuda.Stream(device=dev)
    for i in range(max(1, args.steps // 2) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        Ad = diaf.DeviceCSC(w.n, *(t.to(dev, non_blocking=True) for t in hA))
        PWd = diaf.DeviceCSC(w.n, *(t.to(dev, non_blocking=True) for t in hP))
        budd = hB.to(dev, non_blocking=True)
        F = diaf.factor(Ad, PWd, w.vrule, budd, alg=args.alg, prec=args.prec, tie_tol=w.tie_tol, stream=stream,
                        tuning=tuning)
        outs = [F.W.vals, F.V.colptr, F.V.rowidx, F.V.vals, F.res]
        if host is None or any(h.shape != o.shape or h.dtype != o.dtype for h, o in zip(host, outs)):
            host = [torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs]
        factored = torch.cuda.Event()
        factored.record(stream)
        copy_stream.wait_event(factored)
        with torch.cuda.stream(copy_stream):
            for h, o in zip(host, outs):
                h.copy_(o, non_blocking=True)
        if do_apply:
            F.apply(x1, y1, stream=stream)
        stream.wait_stream(copy_stream)
        s1.record(stream)
        torch.cuda.synchronize()
        d2h = sum(h.numel() * h.element_size() for h in host)
        F.close()
        if i > 0:
            e2e_ms.append(s0.elapsed_time(s1))
    e2e_val, _ = whole_job_rate(w.n, float(np.mean(e2e_ms)), world)

    # ---- roofline of the dominant kernel (the numeric column kernel)
    peaks, peak_src = _peaks()
    m, k = tile_sizes(w)
    flops, flops64 = algorithmic_flops(m, k, lcount, args.alg, cplx)
    kern = float(np.mean([sum(x) for x in kern_ms]))
    achieved = flops / (kern / 1e3)
    # the kernel of the bucket that took the most time
    bucket_mean = np.mean(np.array(kern_ms, dtype=np.float64), axis=0)
    dom = int(np.argmax(bucket_mean))
    kname = dominant_kernel(dom, args.prec, args.alg, cplx)
    if args.prec == "fp64":
        peak, src = FP64_NOMINAL_TFLOPS * 1e12, "FP64 nominal 1.25 TFLOP/s"
    else:
        peak, src = FP32_TFLOPS * 1e12, "FP32 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
    # DRAM bytes (read + write) of one launch of the dominant kernel, from one ncu
    # capture of the current kernel on this workload; None where none was taken
    traffic = TRAFFIC.get((w.name, args.alg, args.prec))
    gbytes = gathered_bytes(w)
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": f"{kname} (size bucket {dom}, {bucket_mean[dom] / kern:.0%} of the numeric pass; "
                                                        "the figures cover the whole pass)",
            "kernel_ms": kern, "algorithmic_flops": flops, "jacobi_sweeps_assumed": JACOBI_SWEEPS,
            "peak_source": src,
            "fp64": {"flops": flops64, "achieved": flops64 / (kern / 1e3) / 1e12, "peak": FP64_NOMINAL_TFLOPS,
                     "unit": "TFLOP/s", "frac": flops64 / (kern / 1e3) / (FP64_NOMINAL_TFLOPS * 1e12)},
            "gather": {"bytes": gbytes, "achieved": gbytes / (kern / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                       "unit": "GB/s", "frac": gbytes / (kern / 1e3) / 1e9 / peaks["hbm_gbs"],
                       "note": "gathered entries (value + row index) per launch over the numeric pass time, "
                               "against the measured HBM copy bandwidth"}}

    extras = {}
    if not args.no_extras and rank == 0 and do_apply:
        # BiCGSTAB with the preconditioner (not part of the setup metric)
        F = diaf.factor(A, PW, w.vrule, bud, alg=args.alg, prec=args.prec, tie_tol=w.tie_tol)
        S = diaf.Solver(A)
        b = torch.from_numpy(w.b).to(dev)
        S.bicgstab(b, F, tol=1e-8, maxit=1000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, info = S.bicgstab(b, F, tol=1e-8, maxit=1000)
        torch.cuda.synchronize()
        solve_ms = 1e3 * (time.perf_counter() - t0)
        x0, info0 = S.bicgstab(b, None, tol=1e-8, maxit=1000)
        extras["bicgstab"] = {"its": info.iterations, "converged": bool(info.converged), "relres": info.relres,
                              "solve_ms": solve_ms, "its_unpreconditioned": info0.iterations,
                              "err_inf": float((x - 1).abs().max().item())}
        # GMRES(50) to 1e-6 (the paper's solver for the complex problems)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xg, ig = S.gmres(b, F, tol=1e-6, restart=50, maxit=2000)
        torch.cuda.synchronize()
        extras["gmres50"] = {"its": ig.iterations, "converged": bool(ig.converged), "relres": ig.relres,
                             "solve_ms": 1e3 * (time.perf_counter() - t0)}
        F.close()
        # the stabilised DIAF-Q of Sec. 3.2 (trigger |v_jj| < 1e-2, r = 2, the
        # paper's experiments) on the same V pattern rule
        Fs = diaf.factor(A, PW, w.vrule, bud, alg="Q", prec=args.prec, tie_tol=w.tie_tol, stab_tol=1e-2, stab_r=2.0)
        stab = int(np.count_nonzero(Fs.flags.cpu().numpy() & 128))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xs, isb = S.bicgstab(b, Fs, tol=1e-8, maxit=1000)
        torch.cuda.synchronize()
        extras["bicgstab_stabilised_q"] = {"its": isb.iterations, "converged": bool(isb.converged),
                                           "relres": isb.relres, "solve_ms": 1e3 * (time.perf_counter() - t0),
                                           "stabilised_columns": stab, "setup_ms": Fs.timings()["total_ms"]}
        Fs.close()
    if not args.no_extras and rank == 0:
        # the plain FP64 form on the same workload: columns/s and residual agreement
        if args.prec != "fp64":
            tt = []
            for _ in range(3):
                flush.zero_()
                torch.cuda.synchronize()
                Fd = diaf.factor(A, PW, w.vrule, bud, alg=args.alg, prec="fp64", tie_tol=w.tie_tol)
                tt.append(Fd.timings()["total_ms"])
                res64 = Fd.res.cpu().numpy()
                Fd.close()
            Fm = diaf.factor(A, PW, w.vrule, bud, alg=args.alg, prec=args.prec, tie_tol=w.tie_tol)
            resm = Fm.res.cpu().numpy()
            fb = Fm.fallbacks()
            Fm.close()
            # relative difference where the residual is above the rounding floor of the column
            # (1e-10 of max |a_ij|: below it both are zero to the rounding of w)
            floor = 1e-10 * float(np.abs(w.A.vals).max())
            rel = np.abs(resm - res64) / np.maximum(np.abs(res64), floor)
            c64 = w.n / (statistics.median(tt) / 1e3)
            extras["fp64_plain"] = {"factor_columns_per_s": c64, "factor_ms": statistics.median(tt),
                                    "speedup_of_mixed": (w.n / (float(np.mean(total_ms)) / 1e3)) / c64,
                                    "res_rel_diff_max": float(rel.max()), "res_rel_diff_median": float(np.median(rel)),
                                    "mixed_fp64_fallback_columns": int(sum(fb))}
        # numeric refactorization on a fixed structure: the CUDA-graph plan replayed
        P = diaf.Plan(A, PW, w.vrule, bud, alg=args.alg, prec=args.prec, tie_tol=w.tie_tol, tuning=tuning)
        P.execute()
        torch.cuda.synchronize()
        tr = []
        for _ in range(5):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.execute(stream)
            e1.record(stream)
            e1.synchronize()
            tr.append(e0.elapsed_time(e1))
        extras["graph_replay"] = {"numeric_columns_per_s": w.n / (statistics.median(tr) / 1e3),
                                  "ms": statistics.median(tr)}
        del P
        # the other algorithm, same workload (factor only, median of 3)
        other = "Q" if args.alg == "S" else "S"
        tt = []
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            Fo = diaf.factor(A, PW, w.vrule, bud, alg=other, prec=args.prec, tie_tol=w.tie_tol)
            tt.append(Fo.timings()["total_ms"])
            Fo.close()
        extras[f"alg_{other}_factor_columns_per_s"] = w.n / (statistics.median(tt) / 1e3)
    if not args.no_extras and rank == 0 and do_apply:
        try:
            extras["kv_sweep"] = kv_sweep(w, A, PW, args.alg, args.prec, dev)
        except Exception as e:
            extras["kv_sweep"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    if not args.no_extras and rank == 0 and do_apply:
        try:
            extras["block_v"] = block_v_report(w, A, PW, args.alg, args.prec, dev)
        except Exception as e:
            extras["block_v"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    if not args.no_extras and not args.no_learned and rank == 0:
        try:
            extras["learned_proposal"] = learned_report(dev)
        except Exception as e:  # reported, not fatal: the setup metric above stands on its own
            extras["learned_proposal"] = {"error": f"{type(e).__name__}: {e}"[:300]}

    if rank == 0:
        line = {"metric": metric_name(args.workload, args.alg), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": ("c64+c128" if cplx else "f32+f64") if args.prec == "mixed32" else ("c128" if cplx else "f64"),
                "data": "synthetic",
                "config": {"workload": w.name, "n": w.n, "alg": args.alg, "prec": args.prec,
                           "nnz_A": w.A.nnz, "nnz_W": w.PW.nnz, "columns_per_step": w.n,
                           "l2": "flushed (256 MiB write) before every timed step",
                           "step": "diaf_factor + one diaf_apply" if do_apply else "diaf_factor",
                           "bucket_cols": bucket_cols, "tie_tol": w.tie_tol,
                           "tuning": tuning if tuning is not None else "default", "autotune_numeric_ms": tune_ms,
                           "parallelism": f"replicas x{world}"},
                "setup_ms": float(np.mean(total_ms)), "numeric_pass_ms": float(np.mean(numeric_ms)),
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(launches), "roofline": roof, "peaks_source": peak_src}
        line.update(extras)
        line["clocks"] = clk.summary()
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(w, args.alg)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
