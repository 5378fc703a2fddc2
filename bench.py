#!/usr/bin/env python
"""Benchmark of the GB300 Golub-Kahan partial SVD (arXiv 2104.10785).

Metric: converged top-k singular triplets per second at <= 1e-8 relative residual.
Default workload: dense 100000 x 40000 operator stored in bf16, A = U diag(i^-1.5) V^T
with seeded orthonormal factors, top-100 triplets, tol 1e-8, in the precision form with
the learned Krylov dimension: one step = the sketch of A and the network's prediction of
K, then one full gk_psvd call (start vector, bidiagonalization sweeps with
reorthogonalization, small SVDs, restarts if the prediction was short, Ritz vectors) on
inputs resident in HBM.  Beside it: the same bf16 operator at the fixed Krylov dimension
200, and the plain path (the f32-stored copy at K = 200).  The end-to-end figure times
the same steps from host buffers (host-to-device copy of the operator and device-to-host
copy of U, S, V inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gk|reference] [--workload NAME]

The line also carries "batched": the 512-problem batched workload (dense f32, uneven sizes,
ranks 5..64 + 1e-6 noise) solved by the plain pipeline (batched Algorithm 3 for the rank,
then the batched top-r partial SVD) and by the learned one (sketch + network -> rank and
Krylov dimension, one batched partial SVD judged by its own spectrum), converged triplets/s
of each.  `--workload batched_f32_512_rank5to64` makes that the headline line.

With N > 1 (torchrun) every rank solves its own replica (the method has no exchange
step at this size); value = triplets of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
F64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64 (CUDA cores); measured f64 FMA here: 1.19


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.lines = []
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": float(np.median(power)) if power else None}


# ---------------------------------------------------------------------------
# replicas: the slowest rank's time and the whole job's rate
# ---------------------------------------------------------------------------
def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over the ranks of the default process group (x itself without one).
    NCCL reduces a device tensor, gloo a host one."""
    import torch
    import torch.distributed as tdist

    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    dev = device if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed (each the same share: weak scaling) per second of the slowest rank."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------------------
# host buffers next to the GPU
# ---------------------------------------------------------------------------
def gpu_local_cpus(gpu_index):
    """CPUs of the NUMA node the GPU hangs off (sysfs local_cpulist of its PCI function), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", str(gpu_index)],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        dom, rest = out.split(":", 1)
        bus = "%04x:%s" % (int(dom, 16), rest.lower())
        txt = open(f"/sys/bus/pci/devices/{bus}/local_cpulist").read().strip()
        cpus = set()
        for part in txt.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        avail = os.sched_getaffinity(0)
        cpus &= avail
        return cpus or None
    except Exception:
        return None


def host_page_report():
    """Transparent huge page mode and this process's huge-page-backed anonymous memory (kB), for
    reading an end-to-end figure: copies from 64 KB pages run slower after long kernel runs."""
    rep = {}
    try:
        rep["thp"] = open("/sys/kernel/mm/transparent_hugepage/enabled").read().strip()
    except OSError:
        rep["thp"] = None
    try:
        for line in open("/proc/self/smaps_rollup"):
            if line.startswith("AnonHugePages:"):
                rep["anon_huge_kb"] = int(line.split()[1])
    except OSError:
        pass
    return rep


def link_rate(host, dev):
    """H2D copy rate (GB/s) of one host buffer into a device buffer of the same size, after one
    untimed copy: the state of the host link when the end-to-end figure was taken."""
    import torch

    dev.copy_(host, non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dev.copy_(host, non_blocking=True)
    torch.cuda.synchronize()
    return host.numel() * host.element_size() / (time.perf_counter() - t0) / 1e9


class near_gpu:
    """Run the block (pinned host allocations) on the GPU's local CPUs, so that the pages land on
    its NUMA node; restores the previous affinity."""

    def __init__(self, gpu_index):
        self.cpus = gpu_local_cpus(gpu_index)
        self.old = None

    def __enter__(self):
        if self.cpus:
            self.old = os.sched_getaffinity(0)
            os.sched_setaffinity(0, self.cpus)
        return self

    def __exit__(self, *exc):
        if self.old is not None:
            os.sched_setaffinity(0, self.old)
        return False


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def make_workload(name, device, want_plain=True, seed=None):
    import torch

    import synth

    w = dict(synth.WORKLOADS[name])
    w["name"] = name
    if seed is not None:  # another draw of the same recipe (operator, start vector)
        w["seed"] = int(seed)
    t0 = time.time()
    if w["kind"] == "spectrum_pow":
        sig = synth.sigma_power(w["n"], w["e"])
        A32, Ut, Vt = synth.torch_prescribed_spectrum(w["m"], w["n"], sig, w["seed"], device=device, keep_top=w["k"])
        w["sigma_true"] = sig[: w["k"]]
        w["A"] = A32.to(torch.bfloat16)
        w["A_plain"] = A32 if want_plain else None
        if not want_plain:
            del A32
    elif w["kind"] == "spectrum":
        sig = synth.sigma_geometric(w["n"], w["q"])
        A, U0, V0 = synth.prescribed_spectrum(w["m"], w["n"], sig, w["seed"])
        w["sigma_true"] = sig[: w["k"]]
        w["A"] = torch.from_numpy(A).to(device)
        w["A_plain"] = None
    elif w["kind"] == "product":
        w["A"] = synth.torch_gaussian_product(w["m"], w["n"], w["r"], w["noise"], w["seed"], device=device)
        w["A_plain"] = None
    elif w["kind"] == "sparse":
        import paper_2104_10785_gb300 as gk

        sigp = 100.0 * 0.95 ** np.arange(1, w["k"] + 1)
        d = synth.sparse_planted(w["m"], w["n"], w["per_row"], sigp, w["seed"])
        c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        w["A"] = gk.CSR(w["m"], w["n"], c(d["rowptr"]), c(d["colind"]), c(d["vals"]), c(d["t_rowptr"]),
                        c(d["t_colind"]), c(d["t_vals"]))
        w["csr_host"] = d
        w["A_plain"] = None
    else:
        raise SystemExit(f"workload {name} is not benchmarked by this script")
    torch.cuda.synchronize()
    w["gen_seconds"] = time.time() - t0
    return w


def profiled_traffic(kernel, workload, source="gk_matvec.cu", field="bytes_per_launch"):
    """A figure recorded from an ncu capture in profiles/*.md (DRAM bytes per full-size launch, or
    with field="ratio" DRAM bytes over algorithmic bytes), used only while the kernel's source
    file is unchanged since the capture (else None)."""
    import glob
    import hashlib
    import re

    src = os.path.join(ROOT, "paper_2104_10785_gb300", "csrc", source)
    h = hashlib.md5(open(src, "rb").read()).hexdigest()
    pat = re.compile(r"roofline-traffic:\s*kernel=(\S+)\s+workload=(\S+)\s+" + field +
                     r"=([0-9.]+)\s+source_md5=(\w+)")
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(f):
            mm = pat.search(line)
            if mm and mm.group(1) == kernel and mm.group(2) == workload and mm.group(4) == h:
                return float(mm.group(3)) if field == "ratio" else int(mm.group(3))
    return None


def err_rel_paper(r_atu, S):
    """The paper's err_rel (Section 5): ||A^T U - V Sigma||_F / ||Sigma||_F, from the per-triplet
    residuals r_atu[i] = ||A^T u_i - s_i v_i|| (column norms of A^T U - V Sigma)."""
    import torch

    r = torch.as_tensor(r_atu, dtype=torch.float64)
    return float(torch.linalg.vector_norm(r)) / float(torch.linalg.vector_norm(torch.as_tensor(S, dtype=torch.float64)))


def operator_dtype(A):
    return A.vals.dtype if hasattr(A, "t_vals") else A.dtype


def operator_bytes(A):
    """Bytes of the stored operator (a CSR counts A and its transpose)."""
    if hasattr(A, "t_vals"):
        return sum(t.numel() * t.element_size() for t in (A.vals, A.colind, A.rowptr, A.t_vals, A.t_colind, A.t_rowptr))
    return A.numel() * A.element_size()


def algorithmic_bytes(w, which):
    """Bytes one launch of the product kernel must move: the stored operator once (a CSR: its
    values, column indices and row pointers), the input vector (f32, gathered once for a CSR:
    f64), the f64 output and the f64 vector it subtracts."""
    m, n = w["m"], w["n"]
    A = w["A"]
    if hasattr(A, "t_vals"):
        es = A.vals.element_size()
        nnz = A.vals.numel()
        rows, cols = (m, n) if which == "matvec" else (n, m)
        return nnz * (es + 4) + 4 * (rows + 1) + 8 * cols + 16 * rows
    es = A.element_size()
    if which == "matvec":
        return es * m * n + 4 * n + 8 * m + 8 * m
    return es * m * n + 4 * m + 8 * n + 8 * n


def orth_work(m, n, K, keep, cycles, passes=1):
    """f64 flops and bytes of the classical Gram-Schmidt of one solve: step j of a cycle
    orthogonalizes the m-vector against j columns and the n-vector against j + 1; each pass reads
    the columns twice (coefficients, update) and the vector twice, writes it once.  The library's
    default rule runs one pass and a second only where the first cancels, so passes = 1 counts the
    least work the solve did (an achieved rate from it is a lower bound)."""
    fl = by = 0
    for c in range(cycles):
        for j in range(0 if c == 0 else keep, K):
            for length, cols in ((m, j), (n, j + 1)):
                fl += passes * 4 * length * cols
                by += passes * (16 * length * cols + 24 * length)
    return fl, by


# ---------------------------------------------------------------------------
# CPU oracle samples
# ---------------------------------------------------------------------------
def oracle_operator(w):
    import torch

    import oracle

    A = w["A"]
    if "csr_host" in w:
        d = w["csr_host"]
        return oracle.Operator.csr(w["m"], w["n"], d["rowptr"], d["colind"], d["vals"], "f32")
    if A.dtype == torch.bfloat16:
        bits = A.view(torch.int16).cpu().numpy().view(np.uint16)
        return oracle.Operator.dense(None, dtype="bf16", bits=bits)
    return oracle.Operator.dense(A.cpu().numpy())


def oracle_complete_solves(op, w, q1, K, budget_s=20.0):
    """The oracle, as it stands, solving the workload completely (the partial SVD at the
    workload's k, tol and the Krylov dimension K the GPU used; Algorithm 3 for the rank
    workload), repeated while the time spent stays under budget_s (at least once).
    Returns (units per second, solves, seconds, oracle info of the last solve)."""
    import oracle

    reps, t0, info = 0, time.perf_counter(), None
    while reps == 0 or time.perf_counter() - t0 < budget_s:
        if w["kind"] == "product":
            r, kp, _ = oracle.numrank(op, q1, eps=w["eps"], kmax=512)
            info = {"rank": r, "kprime": kp}
        else:
            _, _, _, info = oracle.psvd(op, w["k"], K, q1, tol=w["tol"], max_restarts=400)
        reps += 1
    dt = time.perf_counter() - t0
    units = reps * (1 if w["kind"] == "product" else w["k"])
    return units / dt, reps, dt, info


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# batched workload: plain vs learned pipelines
# ---------------------------------------------------------------------------
def batched_leg(device, steps, warmup, keep_mats=False):
    import torch

    import paper_2104_10785_gb300 as gk
    from paper_2104_10785_gb300 import predictor
    import synth

    w = synth.WORKLOADS["batched_f32_512_rank5to64"]
    t0 = time.time()
    shapes = synth.batched_shapes(w["count"], w["seed"])
    mats = synth.torch_batched_products(shapes, 1e-6, w["seed"], device=device)
    torch.cuda.synchronize()
    gen = time.time() - t0
    params = predictor.load(device=device)
    if params is None:
        raise SystemExit("trained predictor weights are missing")
    truth = [s[2] for s in shapes]
    stream = torch.cuda.current_stream(device)
    res = {}
    for name, fn in (("plain", lambda: predictor.plain_batched(mats, w["eps"], w["tol"])),
                     ("learned", lambda: predictor.learned_batched(mats, params, w["eps"], w["tol"]))):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        launches0 = gk.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ranks, out, info = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # bytes of A the pipeline must stream: each product (and the sketch) reads its operator once
        a_bytes = sum(mv * A.shape[0] * A.shape[1] * 4 for mv, A in zip(info["matvecs_per_problem"], mats))
        trip = int(sum(ranks))
        res[name] = {"value": trip / (ms / 1e3), "unit": "triplets/s", "ms_per_step": ms, "triplets": trip,
                     "matvecs": int(info["matvecs"]), "ranks_equal_truth": ranks == truth,
                     "status": int(info["status"]), "operator_GB_per_s": a_bytes / (ms / 1e3) / 1e9,
                     "launches_per_step": (gk.launch_count() - launches0) / steps}
        if name == "learned":
            res[name]["fallbacks"] = info["fallbacks"]
    res["learned_speedup"] = res["plain"]["ms_per_step"] / res["learned"]["ms_per_step"]
    # dominant kernel: the persistent solver of the learned pipeline (one launch per call), timed
    # with CUDA events around the call; algorithmic bytes = every product streams its operator once
    pred = predictor.predict(mats, params)
    probs = [dict(A=A, k=r, krylov_dim=K, tol=w["tol"], rank_cut=w["eps"]) for A, (r, K) in zip(mats, pred)]
    gk.gk_psvd_batched(probs, autotune=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = max(1, steps)
    e0.record(stream)
    for _ in range(reps):
        out, st, info = gk.gk_psvd_batched(probs, autotune=True)
    e1.record(stream)
    torch.cuda.synchronize()
    kms = e0.elapsed_time(e1) / reps
    kbytes = sum(o[3]["matvecs"] * A.shape[0] * A.shape[1] * 4 for o, A in zip(out, mats))
    hbm, peak_kind = peaks()
    # DRAM bytes over algorithmic bytes from a capture of the first 64 problems, scaled to this
    # launch by the bytes it streams (each product reads its operator once at either size)
    ratio = profiled_traffic("k_batched<float>", "batched_f32_512_rank5to64", "gk_batched_kernel.cuh", "ratio")
    res["roofline"] = {"bound": "hbm", "achieved": kbytes / (kms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                       "frac": kbytes / (kms / 1e3) / 1e9 / hbm,
                       "traffic": int(ratio * kbytes) if ratio is not None else None, "kernel": "k_batched<float>",
                       "bytes_per_launch": int(kbytes), "avg_launch_ms": kms, "launches": reps,
                       "cluster_size": info["reserved"], "clusters": info["kprime"], "peak_source": peak_kind}
    if keep_mats:
        res["_mats"], res["_shapes"] = mats, shapes
    res["config"] = {"workload": "batched_f32_512_rank5to64", "count": w["count"], "eps": w["eps"], "tol": w["tol"],
                     "bytes": int(sum(A.numel() * 4 for A in mats)), "gen_seconds": gen,
                     "l2": "inputs larger than L2 (%.1f GB in total)" % (sum(A.numel() * 4 for A in mats) / 1e9)}
    return res


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The CPU oracle, as it stands, on the host cores: complete solves of the workload (no
    extrapolation), as many as fit in about 20 s and at least one; for the batched workload
    the oracle's complete pipeline (Algorithm 3, then the top-r partial SVD) on every second
    problem of the batch.  Work is never extrapolated; `steps` is the number of complete solves
    timed (the --steps request is recorded beside it)."""
    import torch

    import oracle
    import synth

    if rank != 0:
        return None
    device = torch.device("cuda", 0) if torch.cuda.is_available() else None
    if device is None:
        return {"impl": "reference", "unavailable": "the synthetic operator is generated on the GPU and no GPU is visible"}
    common = {"impl": "reference", "n_gpus": world, "warmup": 0, "requested_steps": args.steps,
              "requested_warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "f64", "data": "synthetic"}
    if args.workload == "batched_f32_512_rank5to64":
        w = synth.WORKLOADS[args.workload]
        shapes = synth.batched_shapes(w["count"], w["seed"])
        mats = synth.torch_batched_products(shapes, 1e-6, w["seed"], device=device)
        idx = tuple(range(0, 512, 2))
        value, cores, desc = oracle_batched_sample(mats, shapes, w, idx)
        return dict(common, **{
            "metric": "converged top-k triplets/sec at <=1e-8 rel. residual", "value": value, "unit": "triplets/s",
            "steps": 1, "ms_per_step": sum(shapes[i][2] for i in idx) / value * 1e3,
            "config": {"workload": args.workload, "count": w["count"], "eps": w["eps"], "tol": w["tol"]},
            "cpu_baseline": {"value": value, "unit": "triplets/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "triplets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        })
    if args.workload == "rsgd_f64_64x784x256_rank5":
        # the oracle's Algorithm 4 on a bounded sample of the same seeded data (no GPU work)
        w = dict(synth.WORKLOADS[args.workload], name=args.workload)
        X, Vd, y, W0, batches, q1, _ = synth.rsgd_data(w["P"], w["N"], w["d1"], w["d2"], w["r"], 3, w["b"],
                                                       seed=w["seed"])
        cpu = rsgd_oracle_sample(w, X, Vd, y, W0, batches, q1)
        return dict(common, **{
            "metric": "Algorithm 4 problem-steps/sec (two rank-5 inner SVDs per problem-step)", "value": cpu["value"],
            "unit": "problem-steps/s", "steps": 1, "ms_per_step": 1e3 / cpu["value"],
            "config": {"workload": args.workload, "problems": w["P"], "d1": w["d1"], "d2": w["d2"], "r": w["r"],
                       "batch": w["b"], "k_inner": w["k_inner"]},
            "cpu_baseline": cpu,
            "e2e": {"value": cpu["value"], "unit": "problem-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        })
    w = make_workload(args.workload, device, want_plain=False, seed=args.seed)
    K = w.get("K", 0)
    if w["name"] == "dense_bf16_100000x40000_top100":
        # the Krylov dimension of the measured arm's configuration: the committed network's choice
        # for this operator (a configuration value; the timed work below is the oracle alone)
        from paper_2104_10785_gb300 import predictor

        kparams = predictor.load(device=device, path=predictor.KRYLOV_PARAMS_FILE)
        if kparams is not None:
            K = predictor.predict_krylov(w["A"], kparams, w["k"])
    op = oracle_operator(w)
    del w["A"]
    torch.cuda.empty_cache()
    cores = cpu_threads()
    oracle.set_threads(cores)
    q1 = oracle.start_vector(w["seed"], w["m"])
    value, reps, dt, oinfo = oracle_complete_solves(op, w, q1, K)
    numrank = w["kind"] == "product"
    unit = "rank estimations/s" if numrank else "triplets/s"
    sample = (f"{reps} complete oracle {'rank estimate' if numrank else 'solve'}{'s' if reps > 1 else ''} of the "
              f"{w['m']}x{w['n']} {w['dtype']} operator" + ("" if numrank else f" (k={w['k']}, K={K}, tol={w['tol']})")
              + f", {dt:.1f} s")
    line = dict(common, **{"value": value, "unit": unit, "steps": reps, "ms_per_step": dt / reps * 1e3,
                           "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                                            "sample": sample},
                           "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    if numrank:
        line.update({"metric": "numerical rank estimations/sec (Algorithm 3, eps 1e-5 relative)",
                     "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "true_rank": w["r"], "eps": w["eps"],
                                "rank": oinfo["rank"]}})
    else:
        line.update({"metric": "converged top-k triplets/sec at <=1e-8 rel. residual",
                     "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "k": w["k"], "krylov_dim": K,
                                "tol": w["tol"], "storage": w["dtype"]}})
    return line


def run_gk(args, rank, world):
    import torch

    import paper_2104_10785_gb300 as gk
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
    gk.lib()
    if args.workload == "batched_f32_512_rank5to64":
        return run_batched_headline(args, rank, world, device)
    if args.workload == "dense_f32_50000x20000_rank200":
        return run_numrank_headline(args, rank, world, device)
    if args.workload == "rsgd_f64_64x784x256_rank5":
        return run_rsgd_headline(args, rank, world, device)
    w = make_workload(args.workload, device, want_plain=not args.no_plain, seed=args.seed)
    k, K, tol = w["k"], (args.krylov if args.krylov else w["K"]), w["tol"]
    A = w["A"]
    stream = torch.cuda.current_stream(device)
    kw = dict(krylov_dim=K, seed=w["seed"])
    # experimental kernels, off unless asked for: the bidiagonal SVD of a restart-free cycle, the
    # predictor's sketch on the tcgen05 tensor cores, the Ritz vectors in double-f32
    exp = {}
    if args.bdsvd:
        exp["bdsvd"] = True
    if args.sketch_tc:
        exp["sketch_tc"] = True
    if args.ritz_df:
        exp["ritz_df"] = True
    kw.update(exp)
    # the bf16 precision form takes its Krylov dimension from the learned predictor (sketch +
    # network, inside every timed step); --fixed-krylov times the workload's fixed K instead
    from paper_2104_10785_gb300 import predictor

    kparams = None
    if w["name"] == "dense_bf16_100000x40000_top100" and not args.fixed_krylov:
        kparams = predictor.load(device=device, path=predictor.KRYLOV_PARAMS_FILE)
        if kparams is None:
            raise SystemExit("trained Krylov-dimension weights are missing")

    def solve(Aop, **extra):
        if kparams is not None:
            return predictor.learned_psvd(Aop, kparams, k, tol, seed=w["seed"], **exp, **extra)
        return gk.gk_psvd(Aop, k, tol, **kw, **extra)

    def barrier():
        if dist:
            tdist.barrier()

    # warm-up
    for _ in range(args.warmup):
        U, S, V, st, info = solve(A)
    torch.cuda.synchronize()

    # timed region: inputs resident in HBM (8 GB operator > 129 MB L2)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    # an operator that fits in L2 (129 MB) is flushed from it before every timed step (a 512 MB
    # write between the events of consecutive steps)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device) if operator_bytes(A) < (256 << 20) else None
    clocks = ClockSampler(gpu_index)
    barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos, statuses = [], []
    launches0 = gk.launch_count()
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        U, S, V, st, info = solve(A, profile=True)
        evs[i][1].record(stream)
        infos.append(info)
        statuses.append(st)
    torch.cuda.synchronize()
    launches_timed = gk.launch_count() - launches0
    barrier()
    clk = clocks.stop()
    Kused = infos[-1].get("krylov_dim", K)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), device)
    value = whole_job_rate(k * args.steps, world, ms / 1e3)

    # accuracy of the returned triplets on the stored operator (FP64-grade residual kernels: f64
    # products, or double-f32 products of all k triplets per pass over a reduced-precision A)
    torch.cuda.synchronize()
    t_res = time.perf_counter()
    r_av, r_atu = gk.gk_residuals(A, U, S, V)
    torch.cuda.synchronize()
    resid_check_ms = (time.perf_counter() - t_res) * 1e3
    s1 = float(S[0])
    resid_rel = float(torch.maximum(r_av, r_atu).max()) / s1
    err_rel = err_rel_paper(r_atu, S)
    sig_err = float(np.max(np.abs(S.cpu().numpy() - w["sigma_true"]) / w["sigma_true"])) if "sigma_true" in w else None

    # dominant kernel group (CUDA events recorded by the library around every launch group)
    tot = {key: sum(i[key] for i in infos) for key in ("ms_matvec", "ms_matvec_t", "ms_orth", "ms_small",
                                                        "ms_restart", "n_matvec", "n_matvec_t")}
    hbm, peak_kind = peaks()
    f64_op = operator_dtype(A) == torch.float64
    is_csr = hasattr(A, "t_vals")
    names = {"matvec": "k_spmv (A x)" if is_csr else ("k_gemv_f64" if f64_op else "k_gemv_bulk+k_gemv_reduce"),
             "matvec_t": "k_spmv (A^T x)" if is_csr else ("k_gemvt_f64" if f64_op else "k_gemvt_lp+k_gemvt_reduce")}
    groups = {}
    for which in ("matvec", "matvec_t"):
        nl = tot["n_" + which]
        if nl <= 0:
            continue
        avg_ms = tot["ms_" + which] / nl
        bpl = algorithmic_bytes(w, which)
        g = {"kernel": names[which], "avg_launch_ms": avg_ms, "launches": nl, "bytes_per_launch": bpl,
             "GBs": bpl / (avg_ms / 1e3) / 1e9, "total_ms": tot["ms_" + which]}
        if f64_op and not is_csr:
            g["flops_per_launch"] = 2 * w["m"] * w["n"]
            g["TFLOPs"] = g["flops_per_launch"] / (avg_ms / 1e3) / 1e12
        groups[which] = g
    keep = k + (Kused - k) // 2
    ofl, oby = orth_work(w["m"], w["n"], Kused, keep, infos[-1]["cycles"])
    oms = tot["ms_orth"] / len(infos)
    # vectors past 8192 entries: one cooperative launch per Gram-Schmidt on the bases' double-f32
    # copies (FP32 pipes); shorter ones: the one-CTA f64 kernel
    groups["orth"] = {"kernel": "k_orth_coop (double-f32 Gram-Schmidt, per solve)", "total_ms": tot["ms_orth"],
                      "ms_per_solve": oms, "flops_per_solve": ofl, "bytes_per_solve": oby,
                      "TFLOPs": ofl / (oms / 1e3) / 1e12 if oms > 0 else None,
                      "GBs": oby / (oms / 1e3) / 1e9 if oms > 0 else None,
                      "passes_counted": 1}
    dom = max(groups, key=lambda g: groups[g]["total_ms"])
    G = groups[dom]
    if dom == "orth":
        # the basis products run in double-f32 arithmetic on the FP32 pipes: bound by HBM
        roof = {"bound": "hbm", "achieved": G["GBs"], "peak": hbm, "unit": "GB/s", "frac": G["GBs"] / hbm,
                "traffic": None, "kernel": G["kernel"], "bytes_per_solve": G["bytes_per_solve"],
                "ms_per_solve": G["ms_per_solve"], "peak_source": peak_kind}
    elif f64_op and not is_csr:
        achieved = G["TFLOPs"]
        roof = {"bound": "alu", "achieved": achieved, "peak": F64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / F64_PEAK_TFLOPS, "traffic": None, "kernel": G["kernel"],
                "peak_source": "nominal FP64 rate of the GB300 (f64 FMA on CUDA cores)"}
    else:
        kname = G["kernel"]
        traffic = args.traffic if args.traffic is not None else profiled_traffic(kname, w["name"])
        roof = {"bound": "hbm", "achieved": G["GBs"], "peak": hbm, "unit": "GB/s", "frac": G["GBs"] / hbm,
                "traffic": traffic, "kernel": kname, "bytes_per_launch": G["bytes_per_launch"],
                "avg_launch_ms": G["avg_launch_ms"], "launches": G["launches"], "peak_source": peak_kind}
    roof["groups"] = groups
    step_ms = ms / args.steps
    breakdown = {key: tot[key] / args.steps for key in ("ms_matvec", "ms_matvec_t", "ms_orth", "ms_small",
                                                          "ms_restart")}

    # with the learned Krylov dimension: the same operator at the workload's fixed K beside it
    fixed = None
    if kparams is not None:
        gk.gk_psvd(A, k, tol, **kw)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(reps):
            Uf, Sf, Vf, stf, infof = gk.gk_psvd(A, k, tol, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        fms = e0.elapsed_time(e1) / reps
        fixed = {"value": k / (fms / 1e3), "unit": "triplets/s", "ms_per_step": fms, "krylov_dim": K,
                 "matvecs": infof["matvecs"], "restarts": infof["restarts"], "status": stf,
                 "learned_speedup": (k / (step_ms / 1e3)) / (k / (fms / 1e3))}

    # Algorithm 2 as printed on the same operator: K^ steps of Algorithm 1, the SVD of B, no
    # restart (same Krylov space as the learned solve's single cycle)
    fsvd = None
    if kparams is not None:
        try:
            kf = int(Kused)
            gk.gk_fsvd(A, kf, k, route=1, bdsvd=args.bdsvd)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = max(1, min(args.steps, 3))
            e0.record(stream)
            for _ in range(reps):
                Uq, Sq, Vq, stq, infq = gk.gk_fsvd(A, kf, k, route=1, bdsvd=args.bdsvd)
            e1.record(stream)
            torch.cuda.synchronize()
            qms = e0.elapsed_time(e1) / reps
            ra, rb = gk.gk_residuals(A, Uq, Sq, Vq)
            fsvd = {"value": k / (qms / 1e3), "unit": "triplets/s", "ms_per_step": qms, "krylov_steps": kf,
                    "route": 1, "status": stq, "matvecs": infq["matvecs"],
                    "resid_max_rel": float(torch.maximum(ra, rb).max()) / float(Sq[0])}
        except Exception as exc:  # an auxiliary leg: the headline stands without it
            fsvd = {"error": repr(exc)[:300]}

    # the block form of Algorithm 2 on the same operator (experimental, --block-leg S,STEPS): one
    # cycle of STEPS blocks of S start vectors, the k largest triplets, their FP64-grade residuals
    block = None
    if args.block_leg:
        try:
            bs, bsteps = (int(v) for v in args.block_leg.split(","))
            bkw = dict(seed=w["seed"], f32_products=args.block_f32, ritz_df=args.ritz_df, block_gs=args.block_gs)
            gk.gk_block_fsvd(A, bs, bsteps, k, **bkw)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = max(1, min(args.steps, 3))
            e0.record(stream)
            for _ in range(reps):
                Ub, Sb, Vb, rb_est, stb, infb = gk.gk_block_fsvd(A, bs, bsteps, k, **bkw)
            e1.record(stream)
            torch.cuda.synchronize()
            bms = e0.elapsed_time(e1) / reps
            ra, rb = gk.gk_residuals(A, Ub, Sb, Vb)
            infp = gk.gk_block_fsvd(A, bs, bsteps, k, profile=True, **bkw)[5]  # phase times, untimed
            passes = infb["matvecs"] / bs  # one pass over a dense reduced-precision A per block product
            block = {"value": k / (bms / 1e3), "unit": "triplets/s", "ms_per_step": bms, "s": bs, "block_steps": bsteps,
                     "operator_passes": passes,
                     # the operator's bytes over the whole solve's time: a lower bound on the block
                     # products' achieved rate (the solve also spends time outside them)
                     "operator_gbs_whole_solve": passes * operator_bytes(A) / (bms / 1e3) / 1e9,
                     "f32_products": bool(args.block_f32), "ritz_df": bool(args.ritz_df),
                     "block_gs": bool(args.block_gs), "status": stb, "matvecs": infb["matvecs"],
                     "breakdowns": infb["breakdowns"], "launches": infb["launches"],
                     "resid_est_max_rel": float(rb_est.max()) / float(Sb[0]),
                     "resid_max_rel": float(torch.maximum(ra, rb).max()) / float(Sb[0]),
                     "ms_phases": {"A_P": infp["ms_matvec"], "At_Q": infp["ms_matvec_t"], "gram_schmidt": infp["ms_orth"],
                                   "small_kernels_and_svd": infp["ms_small"], "ritz_vectors": infp["ms_restart"]}}
        except Exception as exc:  # an auxiliary leg: the headline stands without it
            block = {"error": repr(exc)[:300]}

    # the same solve with two classical Gram-Schmidt passes per vector (the rule the paper's
    # reorthogonalization is run with when cancellation is not tested), and with the fused sweep
    # (one pass over A per step); same operator, K and start vector
    legs = {}
    for name, extra in (("two_pass_cgs", dict(reorth_passes=2)), ("fused_sweep", dict(fused=True))):
        try:
            kk = dict(krylov_dim=int(Kused), seed=w["seed"], **extra)
            gk.gk_psvd(A, k, tol, **kk)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = max(1, min(args.steps, 3))
            e0.record(stream)
            for _ in range(reps):
                Ul, Sl, Vl, stl, infl = gk.gk_psvd(A, k, tol, **kk)
            e1.record(stream)
            torch.cuda.synchronize()
            lms = e0.elapsed_time(e1) / reps
            Ul, Sl, Vl, stl, infl = gk.gk_psvd(A, k, tol, profile=True, **kk)
            ra, rb = gk.gk_residuals(A, Ul, Sl, Vl)
            legs[name] = {"value": k / (lms / 1e3), "unit": "triplets/s", "ms_per_step": lms, "krylov_dim": int(Kused),
                          "status": stl, "matvecs": infl["matvecs"], "restarts": infl["restarts"],
                          "ms_orth_per_solve": infl["ms_orth"], "ms_matvec_per_solve": infl["ms_matvec"],
                          "ms_matvec_t_per_solve": infl["ms_matvec_t"], "fused_cluster": infl["reserved"],
                          "resid_max_rel": float(torch.maximum(ra, rb).max()) / float(Sl[0])}
        except Exception as exc:  # auxiliary legs: the headline stands without them
            legs[name] = {"error": repr(exc)[:300]}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        # host buffers from the library's allocator (huge-page backed, registered), on the GPU's
        # local CPUs
        with near_gpu(gpu_index) as ng:
            if is_csr:
                parts = [gk.host_empty(t.shape, t.dtype) for t in
                         (A.rowptr, A.colind, A.vals, A.t_rowptr, A.t_colind, A.t_vals)]
                for hp_, t in zip(parts, (A.rowptr, A.colind, A.vals, A.t_rowptr, A.t_colind, A.t_vals)):
                    hp_.copy_(t)
                Ah = gk.CSR(w["m"], w["n"], *parts)
                host_list = parts
                big = A.vals
                big_h = parts[2]
            else:
                Ah = gk.host_empty(A.shape, A.dtype)
                Ah.copy_(A)
                host_list = [Ah]
                big, big_h = A, Ah
            outs = (gk.host_empty((k, w["m"]), torch.float64), gk.host_empty((k,), torch.float64),
                    gk.host_empty((k, w["n"]), torch.float64))
        solve(Ah, out=outs)
        # the host link's bandwidth at this moment, for reading the figure
        Bd = torch.empty_like(big)
        h2d_gbs = link_rate(big_h, Bd)
        pages = host_page_report()
        del Bd
        barrier()
        reps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(reps):
            Uh, Sh, Vh, sth, infoh = solve(Ah, out=outs)
            float(Sh[0])  # the result is read on the host
        te = (time.perf_counter() - t0) / reps
        # one more call (untimed) with the library's event timing, to split copies from kernels
        infop = solve(Ah, out=outs, profile=True)[4]
        te = max_over_ranks(te, device)
        e2e = {"value": whole_job_rate(k, world, te), "unit": "triplets/s", "library_ms": infoh["seconds"] * 1e3,
               "profiled_call_ms": {key: infop[key] for key in ("seconds", "ms_copy", "ms_matvec", "ms_matvec_t",
                                                                "ms_orth", "ms_small", "ms_restart")},
               "h2d_bytes_per_step": int(operator_bytes(Ah)),
               "d2h_bytes_per_step": int(8 * k * (w["m"] + w["n"] + 1)), "ms_per_step": te * 1e3,
               "h2d_GBs_torch_copy": h2d_gbs, "host_pages": pages,
               "host_buffers": "gk_host_alloc (huge-page backed, registered), allocated on the GPU's local CPUs %s" % (
                   sorted(ng.cpus) if ng.cpus else "(local CPU list unavailable: default placement)")}
        for t in list(host_list) + list(outs):
            gk.host_free(t)
        del Ah, outs, host_list

    # plain path: the same solve on the f32-stored copy
    plain = None
    if w.get("A_plain") is not None and not args.no_plain:
        Ap = w["A_plain"]
        gk.gk_psvd(Ap, k, tol, **kw)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = max(1, min(args.steps, 3))
        for _ in range(reps):
            Up, Sp, Vp, stp, infop = gk.gk_psvd(Ap, k, tol, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / reps
        ra, rb = gk.gk_residuals(Ap, Up, Sp, Vp)
        plain = {"value": k / (pms / 1e3), "unit": "triplets/s", "ms_per_step": pms, "storage": "f32",
                 "status": stp, "matvecs": infop["matvecs"], "restarts": infop["restarts"],
                 "resid_max_rel": float(torch.maximum(ra, rb).max()) / float(Sp[0]),
                 "bf16_speedup": (k / (step_ms / 1e3)) / (k / (pms / 1e3))}
        del Ap, w["A_plain"]
        torch.cuda.empty_cache()

    # CPU oracle baseline (rank 0, N = 1 only): the oracle's complete solve of the same operator
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        op = oracle_operator(w)
        cores = cpu_threads()
        oracle.set_threads(cores)
        q1 = oracle.start_vector(w["seed"], w["m"])
        v, reps, dt, oinfo = oracle_complete_solves(op, w, q1, int(Kused))
        cpu = {"value": v, "unit": "triplets/s", "cores": cores, "kind": "oracle",
               "sample": (f"{reps} complete oracle solve{'s' if reps > 1 else ''} (k={k}, K={int(Kused)}, tol={tol}) "
                          f"of the same {w['m']}x{w['n']} {w['dtype']} operator, {dt:.1f} s "
                          f"({oinfo['matvecs']} products, {oinfo['restarts']} restarts in the last)")}
        del op

    a_dtype, a_bytes = operator_dtype(A), operator_bytes(A)
    batched = None
    if not args.no_batched and args.workload == "dense_bf16_100000x40000_top100":
        del A
        w.pop("A", None)
        torch.cuda.empty_cache()
        batched = batched_leg(device, steps=2, warmup=1)

    last = infos[-1]
    out = {
        "metric": "converged top-k triplets/sec at <=1e-8 rel. residual",
        "value": value, "unit": "triplets/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if a_dtype == torch.bfloat16 else ("f64" if a_dtype == torch.float64 else "f32"),
        "data": "synthetic",
        "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "k": k, "krylov_dim": Kused, "tol": tol,
                   "seed": w["seed"], **({"experimental": sorted(exp)} if exp else {}), "krylov": "learned (sketch + network in every step)" if kparams is not None else "fixed",
                   "storage": w["dtype"], "accumulate": "f32 runs combined in f64; f64 basis, small SVD, residuals",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": ("inputs larger than L2 (operator %.2f GB)" % (a_bytes / 1e9)) if flush is None else
                   "L2 flushed before every timed step (operator %.1f MB)" % (a_bytes / 1e6)},
        "status": statuses[-1], "resid_max_rel": resid_rel, "err_rel_paper": err_rel, "resid_check_ms": resid_check_ms,
        "sigma_rel_err_vs_prescribed": sig_err,
        "restarts": last["restarts"], "matvecs": last["matvecs"], "steps_per_solve": last["steps"],
        "breakdown_ms_per_step": breakdown,
        "roofline": roof, "clocks": clk, "gpu_launches": None,
        "e2e": e2e, "cpu_baseline": cpu, "plain_f32": plain, "fixed_krylov": fixed, "fsvd": fsvd,
        **({"block_fsvd": block} if args.block_leg else {}),
        "two_pass_cgs": legs.get("two_pass_cgs"), "fused_sweep": legs.get("fused_sweep"),
        "gen_seconds": w["gen_seconds"],
        "batched": batched,
    }
    out["gpu_launches"] = int(launches_timed)
    return out


def run_numrank_headline(args, rank, world, device):
    """Numerical rank (Algorithm 3 on Algorithm 1) of the dense f32 rank-200 product: one step =
    one gk_numrank call; value = rank estimations per second; the rank must equal the true 200."""
    import torch

    import paper_2104_10785_gb300 as gk
    import synth

    w = make_workload(args.workload, device, want_plain=False, seed=args.seed)
    A = w["A"]
    stream = torch.cuda.current_stream(device)
    eps, kmax = w["eps"], 512
    for _ in range(args.warmup):
        r, _, st, info = gk.gk_numrank(A, eps, kmax, seed=w["seed"])
    torch.cuda.synchronize()
    clocks = ClockSampler(device.index or 0)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos, ranks = [], []
    for i in range(args.steps):
        evs[i][0].record(stream)
        r, _, st, info = gk.gk_numrank(A, eps, kmax, seed=w["seed"], profile=True)
        evs[i][1].record(stream)
        infos.append(info)
        ranks.append(r)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms = max_over_ranks(ms, device)
    value = whole_job_rate(args.steps, world, ms / 1e3)
    tot = {key: sum(i[key] for i in infos) for key in ("ms_matvec", "ms_matvec_t", "ms_orth", "n_matvec",
                                                        "n_matvec_t")}
    hbm, peak_kind = peaks()
    groups = {}
    for which, kname in (("matvec", "k_gemv_bulk+k_gemv_reduce"), ("matvec_t", "k_gemvt_lp+k_gemvt_reduce")):
        nl = tot["n_" + which]
        if nl > 0:
            avg = tot["ms_" + which] / nl
            bpl = algorithmic_bytes(w, which)
            groups[which] = {"kernel": kname, "avg_launch_ms": avg, "launches": nl, "bytes_per_launch": bpl,
                             "GBs": bpl / (avg / 1e3) / 1e9, "total_ms": tot["ms_" + which]}
    kp = infos[-1]["kprime"]
    ofl, oby = orth_work(w["m"], w["n"], kp, 0, 1)
    oms = tot["ms_orth"] / len(infos)
    groups["orth"] = {"kernel": "k_orth_coop (double-f32 Gram-Schmidt, per call)", "total_ms": tot["ms_orth"],
                      "ms_per_call": oms, "bytes_per_call": oby,
                      "TFLOPs": ofl / (oms / 1e3) / 1e12 if oms > 0 else None,
                      "GBs": oby / (oms / 1e3) / 1e9 if oms > 0 else None}
    G = groups["matvec"] if groups["matvec"]["total_ms"] >= groups["matvec_t"]["total_ms"] else groups["matvec_t"]
    roof = {"bound": "hbm", "achieved": G["GBs"], "peak": hbm, "unit": "GB/s", "frac": G["GBs"] / hbm,
            "traffic": None, "kernel": G["kernel"], "bytes_per_launch": G["bytes_per_launch"],
            "avg_launch_ms": G["avg_launch_ms"], "launches": G["launches"], "peak_source": peak_kind,
            "groups": groups}
    # end to end from library host memory (4 GB H2D per call, the rank read back)
    Ah = gk.host_empty(A.shape, A.dtype)
    Ah.copy_(A)
    gk.gk_numrank(Ah, eps, kmax, seed=w["seed"])
    t0 = time.perf_counter()
    reps = max(1, min(args.steps, 3))
    for _ in range(reps):
        rh, _, sth, infoh = gk.gk_numrank(Ah, eps, kmax, seed=w["seed"])
    te = (time.perf_counter() - t0) / reps
    e2e = {"value": world / te, "unit": "rank estimations/s", "ms_per_step": te * 1e3,
           "h2d_bytes_per_step": int(Ah.numel() * Ah.element_size()), "d2h_bytes_per_step": 4, "rank": rh}
    gk.host_free(Ah)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        op = oracle_operator(w)
        cores = cpu_threads()
        oracle.set_threads(cores)
        q1 = oracle.start_vector(w["seed"], w["m"])
        v, reps, dt, oinfo = oracle_complete_solves(op, w, q1, 0)
        cpu = {"value": v, "unit": "rank estimations/s", "cores": cores, "kind": "oracle",
               "sample": (f"{reps} complete oracle rank estimate{'s' if reps > 1 else ''} (Algorithm 3) of the same "
                          f"{w['m']}x{w['n']} f32 operator, {dt:.1f} s (rank {oinfo['rank']}, k' {oinfo['kprime']})")}
    return {
        "metric": "numerical rank estimations/sec (Algorithm 3, eps 1e-5 relative)",
        "value": value, "unit": "rank estimations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "true_rank": w["r"], "eps": eps, "kmax": kmax,
                   "l2": "inputs larger than L2 (operator %.1f GB)" % (A.numel() * A.element_size() / 1e9)},
        "ranks": sorted(set(ranks)), "rank_equals_truth": all(r == w["r"] for r in ranks), "steps_per_call": kp,
        "roofline": roof, "clocks": clk, "gpu_launches": int(sum(i["launches"] for i in infos)),
        "e2e": e2e, "cpu_baseline": cpu,
    }


def rsgd_flops(w, matvecs):
    """FP64 flops of one Algorithm 4 call: the inner solves' products (2 per entry of a d1 x d2
    matrix), the mini-batch gradients, the projection (GV, UG, U C) and the update and
    retraction passes."""
    P, d1, d2, r, b = w["P"], w["d1"], w["d2"], w["r"], w["b"]
    per_step = P * (2 * b * d1 * d2 + 2 * 2 * d1 * d2 * r + 2 * d1 * r * r + 2 * d1 * d2 * 2 * r + 2 * d1 * d2 * r)
    return 2.0 * d1 * d2 * matvecs, per_step


def run_rsgd_headline(args, rank, world, device):
    """Algorithm 4 for 64 problems at the paper's 784 x 256 shape: one step = one RSGD iteration of
    every problem (two batched rank-5 inner SVDs); value = problem-steps per second."""
    import numpy as np
    import torch

    import paper_2104_10785_gb300 as gk
    import synth

    w = dict(synth.WORKLOADS[args.workload], name=args.workload)
    P, N, d1, d2, r, b, kin = w["P"], w["N"], w["d1"], w["d2"], w["r"], w["b"], w["k_inner"]
    total = args.warmup + args.steps
    t0 = time.perf_counter()
    X, Vd, y, W0, batches, q1, Ws = synth.rsgd_data(P, N, d1, d2, r, total, b, seed=w["seed"] + rank)
    gen_s = time.perf_counter() - t0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    Xd, Vdd, yd, Wd, Bd, qd = dev(X), dev(Vd), dev(y), dev(W0), dev(batches), dev(q1)
    stream = torch.cuda.current_stream(device)
    for t in range(args.warmup):
        gk.gk_rsgd_batched(Xd, Vdd, yd, Wd, Bd[t:t + 1], qd, w["eta"], w["lam"], r, kin)
    torch.cuda.synchronize()
    clocks = ClockSampler(device.index or 0)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    launches0 = gk.launch_count()
    for i in range(args.steps):
        t = args.warmup + i
        evs[i][0].record(stream)
        st, info = gk.gk_rsgd_batched(Xd, Vdd, yd, Wd, Bd[t:t + 1], qd, w["eta"], w["lam"], r, kin)
        evs[i][1].record(stream)
        infos.append(info)
    torch.cuda.synchronize()
    launches = gk.launch_count() - launches0
    clk = clocks.stop()
    ms = sum(a.elapsed_time(bb) for a, bb in evs)
    ms = max_over_ranks(ms, device)
    value = whole_job_rate(P * args.steps, world, ms / 1e3)
    mv = sum(i["matvecs"] for i in infos)
    f_inner, f_step = rsgd_flops(w, mv)
    flops = f_inner + f_step * args.steps
    achieved = flops / (ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": F64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / F64_PEAK_TFLOPS, "traffic": None,
            "kernel": "k_batched<double> (inner SVDs) + k_rsgd_* (gradient, projection, retraction)",
            "flops_per_step": flops / args.steps, "inner_matvecs_per_step": mv / args.steps,
            "peak_source": "nominal FP64 rate of the GB300 (f64 FMA on CUDA cores); the 64 matrices (103 MB) "
                           "stay in L2 across an inner solve's products"}
    Wh = Wd.cpu().numpy()
    agree = float(np.mean([np.mean(np.sign(np.sum((X[p] @ Wh[p]) * Vd[p], axis=1)) ==
                                   np.sign(np.sum((X[p] @ Ws[p]) * Vd[p], axis=1))) for p in range(min(P, 8))]))
    # end to end: every step's mini-batches (P x b pairs and labels) copied in from pinned host
    # memory as a compact data set, the step, and the P iterates W copied back
    e2e = None
    if not args.no_e2e:
        Xb = torch.empty((P, b, d1), dtype=torch.float64).pin_memory()
        Vb = torch.empty((P, b, d2), dtype=torch.float64).pin_memory()
        yb = torch.empty((P, b), dtype=torch.float64).pin_memory()
        Wout = torch.empty((P, d1, d2), dtype=torch.float64).pin_memory()
        t = total - 1
        for p in range(P):
            Xb[p] = torch.from_numpy(X[p][batches[t, p]])
            Vb[p] = torch.from_numpy(Vd[p][batches[t, p]])
            yb[p] = torch.from_numpy(y[p][batches[t, p]])
        Xbd = torch.empty_like(Xb, device=device)
        Vbd = torch.empty_like(Vb, device=device)
        ybd = torch.empty_like(yb, device=device)
        ident = torch.arange(b, dtype=torch.int32, device=device).repeat(P).view(1, P, b).contiguous()

        def e2e_step():
            Xbd.copy_(Xb, non_blocking=True)
            Vbd.copy_(Vb, non_blocking=True)
            ybd.copy_(yb, non_blocking=True)
            gk.gk_rsgd_batched(Xbd, Vbd, ybd, Wd, ident, qd, w["eta"], w["lam"], r, kin)
            Wout.copy_(Wd, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 3))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        te = e0.elapsed_time(e1) / reps
        e2e = {"value": world * P / (te / 1e3), "unit": "problem-steps/s", "ms_per_step": te,
               "h2d_bytes_per_step": int((Xb.numel() + Vb.numel() + yb.numel()) * 8),
               "d2h_bytes_per_step": int(Wout.numel() * 8)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = rsgd_oracle_sample(w, X, Vd, y, W0, batches, q1)
    return {
        "metric": "Algorithm 4 problem-steps/sec (two rank-5 inner SVDs per problem-step)",
        "value": value, "unit": "problem-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "problems": P, "samples": N, "d1": d1, "d2": d2, "r": r, "batch": b,
                   "eta": w["eta"], "lam": w["lam"], "k_inner": kin,
                   "l2": "working set per step larger than L2 (batches 0.14 GB, W 0.10 GB, Gr and W - eta Z "
                         "0.21 GB; data set 1.09 GB)"},
        "status": 0, "sign_agreement_with_planted": agree, "gen_seconds": gen_s,
        "roofline": roof, "clocks": clk, "gpu_launches": int(launches), "e2e": e2e, "cpu_baseline": cpu,
    }


def rsgd_oracle_sample(w, X, Vd, y, W0, batches, q1, problems=32, steps=3):
    """The oracle (oracle/rsgd.py) as it stands on a bounded sample of the workload: the first
    `problems` problems for `steps` steps; returns the cpu_baseline entry in problem-steps/s."""
    import oracle
    from oracle import rsgd as ors

    cores = cpu_threads()
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    for p in range(problems):
        Wp = W0[p]
        for t in range(steps):
            Wp = ors.rsgd_step(X[p], Vd[p], y[p], batches[t, p], Wp, w["eta"], w["lam"], w["r"], w["k_inner"], q1[p])
    dt = time.perf_counter() - t0
    return {"value": problems * steps / dt, "unit": "problem-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{problems} of the {w['P']} problems for {steps} steps each ({problems * steps} problem-steps, "
                      f"{dt:.1f} s)"}


def oracle_batched_sample(mats, shapes, w, idx=tuple(range(0, 512, 2))):
    """The oracle, as it stands, on a bounded sample of the batch: for each sampled problem
    Algorithm 3 for the rank, then the top-r partial SVD (K = max(2r, r+16)), on the stored
    f32 bytes; returns (triplets per second, cores, description)."""
    import oracle
    import synth

    cores = cpu_threads()
    oracle.set_threads(cores)
    trip = 0
    t = time.perf_counter()
    for i in idx:
        A = mats[i].cpu().numpy()
        op = oracle.Operator.dense(A)
        q1 = synth.start_vector(A.shape[0], w["seed"] + i)
        r, kp, _ = oracle.numrank(op, q1, eps=w["eps"], kmax=min(min(A.shape), 160))
        r = max(1, r)
        K = min(max(2 * r, r + 16), min(A.shape))
        oracle.psvd(op, r, K, q1, tol=w["tol"], max_restarts=400)
        trip += r
    dt = time.perf_counter() - t
    desc = (f"{len(idx)} problems of the batch (every {idx[1] - idx[0] if len(idx) > 1 else 1}th from {idx[0]}): "
            f"the oracle's Algorithm 3 then its top-r partial SVD, {trip} triplets in {dt:.1f} s")
    return trip / dt, cores, desc


def run_batched_headline(args, rank, world, device):
    """The batched workload as the headline: value = converged triplets/s of the learned pipeline
    (sketch, network, one batched partial SVD judged by its own spectrum, plain fallback); the plain
    pipeline beside it.  Timed with CUDA events around whole pipeline calls (each synchronizes)."""
    import torch

    clocks = ClockSampler(device.index or 0)
    res = batched_leg(device, args.steps, args.warmup, keep_mats=True)
    clk = clocks.stop()
    mats, shapes = res.pop("_mats"), res.pop("_shapes")
    import paper_2104_10785_gb300 as gk
    from paper_2104_10785_gb300 import predictor
    import synth

    wb = synth.WORKLOADS["batched_f32_512_rank5to64"]
    # end to end: the 512 operators in library host memory, copied in, the learned pipeline, the
    # triplets copied out, every step
    e2e = None
    if not args.no_e2e:
        params = predictor.load(device=device)
        # the batch in one library host buffer (huge-page granularity) with the device layout: each
        # operator's rows padded to 16 bytes (the solver's vector path), operators at 16-byte
        # offsets; one H2D copy moves the batch into one device buffer of the same layout
        offs, tot = [], 0
        lds = [int(A.stride(0)) for A in mats]
        for A, ld in zip(mats, lds):
            offs.append(tot)
            tot += (A.shape[0] * ld + 3) // 4 * 4
        with near_gpu(device.index or 0):
            pool = gk.host_empty((tot,), torch.float32)
            # room for up to 80 triplets per problem (U^T, S, V^T regions) in a second buffer
            rcap = 80
            su, sn = sum(A.shape[0] for A in mats), sum(A.shape[1] for A in mats)
            opool = gk.host_empty((rcap * (su + sn + len(mats)),), torch.float64)
        dbuf = torch.empty(tot, dtype=torch.float32, device=device)
        hosts = [pool[o:o + A.shape[0] * ld].view(A.shape[0], ld)[:, :A.shape[1]] for o, A, ld in zip(offs, mats, lds)]
        devs = [dbuf[o:o + A.shape[0] * ld].view(A.shape[0], ld)[:, :A.shape[1]] for o, A, ld in zip(offs, mats, lds)]
        for h, A in zip(hosts, mats):
            h.copy_(A)
        oregions = (opool[:rcap * su], opool[rcap * su:rcap * su + len(mats) * rcap], opool[rcap * (su + len(mats)):])

        def e2e_step():
            dbuf.copy_(pool, non_blocking=True)
            ranks, out, info = predictor.learned_batched(devs, params, wb["eps"], wb["tol"])
            bufs = info["outputs"]
            if bufs is not None and all(b.numel() <= h.numel() for b, h in zip(bufs, oregions)):
                # three copies: every problem's r^ columns of U^T, the values, the columns of V^T
                for b, h in zip(bufs, oregions):
                    h[:b.numel()].copy_(b, non_blocking=True)
                nbytes = sum(b.numel() * 8 for b in bufs)
            else:
                nbytes, o = 0, 0
                for (U, S, V, _), A, r in zip(out, mats, ranks):
                    m, n = A.shape
                    for src in (U[:, :r].T, V[:, :r].T, S[:r]):
                        opool[o:o + src.numel()].view(src.shape).copy_(src, non_blocking=True)
                        o += src.numel()
                    nbytes += 8 * r * (m + n + 1)
            torch.cuda.synchronize()
            return ranks, nbytes

        e2e_step()
        torch.cuda.synchronize()
        h2d_gbs = link_rate(pool, dbuf)
        pages = host_page_report()
        reps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(reps):
            ranks, d2h = e2e_step()
        te = (time.perf_counter() - t0) / reps
        trip = int(sum(ranks))
        e2e = {"value": trip * world / te, "unit": "triplets/s", "ms_per_step": te * 1e3,
               "h2d_bytes_per_step": int(pool.numel() * 4), "d2h_bytes_per_step": int(d2h),
               "h2d_GBs_torch_copy": h2d_gbs, "host_pages": pages,
               "layout": "rows padded to 16 bytes, one host buffer and one device buffer for the batch"}
        del hosts, devs, dbuf, oregions
        gk.host_free(pool)
        gk.host_free(opool)
        del pool, opool
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, desc = oracle_batched_sample(mats, shapes, wb)
        cpu = {"value": v, "unit": "triplets/s", "cores": cores, "kind": "oracle", "sample": desc}
    del mats
    ms = res["learned"]["ms_per_step"]
    ms = max_over_ranks(ms, device)
    value = whole_job_rate(res["learned"]["triplets"], world, ms / 1e3)
    return {
        "metric": "converged top-k triplets/sec at <=1e-8 rel. residual",
        "value": value, "unit": "triplets/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": res.pop("config"), "clocks": clk,
        "gpu_launches": int(res["learned"]["launches_per_step"] * args.steps),
        "roofline": res.pop("roofline"), "e2e": e2e, "cpu_baseline": cpu, "batched": res,
    }


# ---------------------------------------------------------------------------
# one kernel family on seeded inputs, for ncu captures (nothing is timed or printed as a result)
# ---------------------------------------------------------------------------
def profile_case(args):
    """--case products: A (m x n, N(0,1) drawn by torch's CUDA generator, stored in --dtype) and
    `reps` calls of gk_matvec(A, x) and gk_matvec(A, y, trans=True).
    --case psvd: `reps` calls of gk_psvd (k = 16, K = 48, tol 1e-8) on the same kind of operator
    (--fused: with the fused sweep).
    --case batched: the first --count problems of the 512-problem batched recipe; `reps` rounds
    of the learned pipeline's sketch and its batched partial SVD with the committed network's
    (rank, K); prints the operator bytes the last solve streamed.
    --case sketch: `reps` calls of gk_sketch_batched on the same kind of operator (one problem;
    --tcgen05: the tensor-core form).
    --case block: `reps` calls of gk_block_numrank (block size --s, --kmax block steps, eps 1e-8)
    on the same kind of operator (--block-f32: its f32 block products; --fsvd R: gk_block_fsvd for R
    triplets after --kmax block steps instead)."""
    import torch

    import paper_2104_10785_gb300 as gk
    import synth

    torch.cuda.set_device(0)
    if args.case in ("products", "psvd", "sketch", "block"):
        dt = {"bf16": torch.bfloat16, "f16": torch.float16, "f32": torch.float32, "f64": torch.float64}[args.dtype]
        g = torch.Generator(device="cuda").manual_seed(1)
        A = torch.randn(args.m, args.n, generator=g, device="cuda", dtype=torch.float32).to(dt)
        x = torch.randn(args.n, generator=g, device="cuda", dtype=torch.float64)
        y = torch.randn(args.m, generator=g, device="cuda", dtype=torch.float64)
        for _ in range(args.reps):
            if args.case == "products":
                gk.gk_matvec(A, x)
                gk.gk_matvec(A, y, trans=True)
            elif args.case == "sketch":
                gk.gk_sketch_batched([A], seed=1, tcgen05=args.tcgen05)
            elif args.case == "block" and args.fsvd > 0:
                gk.gk_block_fsvd(A, args.s, args.kmax, args.fsvd, f32_products=args.block_f32, block_gs=args.block_gs)
            elif args.case == "block":
                gk.gk_block_numrank(A, args.s, 1e-8, args.kmax, f32_products=args.block_f32, block_gs=args.block_gs)
            else:
                gk.gk_psvd(A, 16, 1e-8, krylov_dim=48, max_restarts=0, fused=args.fused)
    elif args.case == "batched":
        from paper_2104_10785_gb300 import predictor

        w = synth.WORKLOADS["batched_f32_512_rank5to64"]
        shapes = synth.batched_shapes(512, w["seed"])[: args.count]
        mats = synth.torch_batched_products(shapes, 1e-6, w["seed"])
        params = predictor.load()
        if params is None:
            raise SystemExit("trained predictor weights are missing")
        for _ in range(args.reps):
            pred = predictor.predict(mats, params)
            out, _, _ = gk.gk_psvd_batched([dict(A=A, k=r, krylov_dim=K, tol=w["tol"], rank_cut=w["eps"])
                                            for A, (r, K) in zip(mats, pred)])
        alg = sum(o[3]["matvecs"] * A.shape[0] * A.shape[1] * 4 for o, A in zip(out, mats))
        print("algorithmic_bytes_per_launch", alg)
    torch.cuda.synchronize()
    print("ok")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gk", choices=["gk", "reference"])
    ap.add_argument("--workload", default="dense_bf16_100000x40000_top100")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--seed", type=int, default=None,
                    help="draw the workload (operator and start vector) with this seed instead of its recipe's")
    ap.add_argument("--krylov", type=int, default=0,
                    help="with --fixed-krylov: this Krylov dimension instead of the workload's")
    ap.add_argument("--fixed-krylov", action="store_true",
                    help="time the default workload at its fixed Krylov dimension instead of the learned one")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture of this kernel")
    ap.add_argument("--case", default=None, choices=["products", "psvd", "batched", "sketch", "block"],
                    help="run one kernel family on seeded inputs for an ncu capture, then exit")
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f16", "f32", "f64"])
    ap.add_argument("--m", type=int, default=40000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--fused", action="store_true", help="--case psvd: run the fused sweep (GK_FLAG_FUSED)")
    ap.add_argument("--tcgen05", action="store_true", help="--case sketch: the tensor-core form (GK_FLAG_SKETCH_TC)")
    ap.add_argument("--bdsvd", action="store_true",
                    help="headline solve: the bidiagonal SVD kernel for restart-free cycles (GK_FLAG_BDSVD)")
    ap.add_argument("--ritz-df", action="store_true",
                    help="headline solve: Ritz vectors from the double-f32 basis copies (GK_FLAG_RITZ_DF)")
    ap.add_argument("--sketch-tc", action="store_true",
                    help="headline solve: the predictor's sketch on the tcgen05 tensor cores (GK_FLAG_SKETCH_TC)")
    ap.add_argument("--block-leg", default=None, metavar="S,STEPS",
                    help="headline: also time gk_block_fsvd (S start vectors, STEPS block steps, the workload's k "
                         "triplets; --block-f32 for its f32 products) on the same operator (experimental)")
    ap.add_argument("--block-gs", action="store_true",
                    help="--block-leg and --case block: the block Gram-Schmidt (GK_FLAG_BLOCK_GS)")
    ap.add_argument("--s", type=int, default=8, help="--case block: start vectors per block")
    ap.add_argument("--kmax", type=int, default=16, help="--case block: block steps")
    ap.add_argument("--block-f32", action="store_true", help="--case block: f32 block products (GK_FLAG_BLOCK_F32)")
    ap.add_argument("--fsvd", type=int, default=0,
                    help="--case block: the block form of Algorithm 2 for this many triplets instead of the rank")
    args = ap.parse_args()
    if args.case is not None:
        profile_case(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and args.impl == "gk":
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_gk(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1 and args.impl == "gk":
        import torch.distributed as tdist

        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
