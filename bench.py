#!/usr/bin/env python3
"""Density matrices per second of the GB300 Chebyshev Fermi-operator solver.

One step = one density matrix for each tight-binding Hamiltonian N in {1000, 2000, 5000}
(4 orbitals per atom, 0.1 atoms / A^3, 400 Chebyshev terms, kT = 0.1 eV, N_e = N/2, mu by
float64 bisection on exact moments), with the matrix products in BF16x3 split precision on
the tensor cores, the three instances computed by one batched call (one grouped launch per
stage). Inputs are resident in HBM; the L2 is flushed (256 MiB write) before every timed
step. Also reported: the 512-instance batch (N log-uniform in [64, 1024], kT ~ U(0.05, 0.2)
eV, 300 terms) replayed as one CUDA graph per batch. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle on the host cores on a bounded sample of the same
workload (rank 0 only). Under torchrun every rank runs the same workload on its own GPU
(independent replicas, weak scaling); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NS = (1000, 2000, 5000)
N_TERMS = 400
KT = 0.1
METRIC = "density matrices/s & % tensor peak, N=1k-5k, mixed vs FP64 at ||dP||/sqrt(N)<=1e-6"
WORKLOAD = ("tight-binding H (N/4 atoms, 0.1/A^3, 4 orbitals, hopping -2exp(-r/1.5A) cut at 6A), "
            "one DM per N in {1000,2000,5000} per step, 400 terms, kT=0.1 eV, N_e=N/2, "
            "mu by FP64 bisection on exact moments")
SPLIT = {"bf16x3": 6, "fp16x2": 3, "bf16x1": 1, "fp64": 1}
# The paper's own timings (float64 throughout, its own model Hamiltonians, one GPU): context
# for the numbers above, not a target; the paper prints them in its prose and plots only.
PAPER_CONTEXT = {
    "hardware": "NVIDIA V100 (Summit, 7.8 TFLOP/s FP64) and AMD MI250X (Crusher); MAGMA 2.6.1 dgemm",
    "time_per_dm": "close to or below 1 s up to N = 4000 with L = 1024 terms (Sec. Results, Fig. 3 "
                   "bottom); about 62 dgemm of N = 4000, ~7.9e12 flop",
    "stream_speedup": "about 1.6x at N = 700 (> 1000 terms) and 1.2x at N = 1000 (1024 terms) on V100 "
                      "from concurrent streams",
    "accuracy": "relative Frobenius error about 1e-7 at about 500 terms, N = 800 metallic model, "
                "kT = 0.1 eV (Sec. Accuracy, Fig. 6)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", default="bf16x3", choices=("bf16x3", "fp16x2", "bf16x1", "fp64"))
    ap.add_argument("--ns", default=",".join(str(n) for n in NS))
    ap.add_argument("--n-terms", type=int, default=N_TERMS, help="Chebyshev terms (profiling cases)")
    ap.add_argument("--no-fp64-check", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-instance batch measurement")
    ap.add_argument("--batch-count", type=int, default=512, help="instances of the batch measurement")
    ap.add_argument("--tile", default="",
                    help="force the product kernel's tile as NxCTASxDRAIN[xSTORE] (e.g. 256x1x16, or "
                         "256x1x8x2 for upper-block plane storage) instead of autotuning it; profiling "
                         "runs use this so the captured kernel is the timed one")
    ap.add_argument("--chain", type=int, default=0, choices=(0, 1, 2),
                    help="product launches: 0 library default, 1 one per product, 2 one per chain")
    ap.add_argument("--chain-window", type=int, default=0,
                    help="chain launches: tiles per step of an instance window (0: one window)")
    ap.add_argument("--no-order", action="store_true",
                    help="skip the learned-order measurement on the batch family")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-mu measurement on the metallic model")
    ap.add_argument("--learned-pairs", type=int, default=20000,
                    help="method-generated training pairs of the learned-mu measurement")
    ap.add_argument("--learned-only", action="store_true",
                    help="run only the learned-mu measurement and print it")
    ap.add_argument("--batch-only", action="store_true",
                    help="measure only the batch (profiling runs); the JSON line then describes the batch")
    return ap.parse_args()


def tile_args(spec: str, chain: int = 0, chain_window: int = 0) -> dict:
    out = {"chain": chain, "chain_window": chain_window}
    if not spec:
        return out
    parts = [int(x) for x in spec.lower().split("x")]
    out.update({"tile_n": parts[0], "tile_ctas": parts[1], "tile_drain": parts[2]})
    if len(parts) > 3:
        out["tile_store"] = parts[3]
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_index)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        # start timing only once sampling has begun (nvidia-smi takes a moment to start)
        t0 = time.monotonic()
        while self.proc is not None and time.monotonic() - t0 < 1.5:
            if os.path.getsize(self.path) > 0 or self.proc.poll() is not None:
                break
            time.sleep(0.02)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[3:7]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------- CPU baseline
# The oracle's work for one density matrix of size N: the mu search (eigenvalues of H, their
# Chebyshev moments and the bisection on the polynomial trace) and the plain three-term
# recursion sum_n c_n T_n(X) on the full N x N matrices (n_terms - 1 products, each term
# costing the same N^3 product and N^2 updates). At N = 2000 and 5000 the recursion is timed
# on its first terms and scaled by (n_terms - 1) / (terms - 1); the mu search is timed whole.
CPU_TERMS = {1000: N_TERMS, 2000: 48, 5000: 7}


def cpu_pieces(ns):
    """The timed pieces of the oracle's work for the N mix: (label, N, kind, terms)."""
    out = []
    for n in ns:
        terms = min(N_TERMS, CPU_TERMS.get(n, max(3, int(N_TERMS * (1000.0 / n) ** 3))))
        out.append((f"N={n} mu search", n, "mu", N_TERMS))
        out.append((f"N={n} recursion, {terms} of {N_TERMS} terms", n, "rec", terms))
    return out


def run_cpu_piece(piece, cache):
    """Runs one piece of the oracle on the workload's own Hamiltonian; returns seconds."""
    import numpy as np
    import oracle as O
    import synth
    _, n, kind, terms = piece
    if n not in cache:
        h = synth.tight_binding(n, 2000 + n)
        ea, eb = O.gershgorin_bounds(h)
        cache[n] = {"h": h, "ea": ea, "eb": eb}
    c = cache[n]
    t0 = time.perf_counter()
    if kind == "mu":
        taus = O.moments_eig(O.spectrum_scaled(np.linalg.eigvalsh(c["h"]), c["ea"], c["eb"]), N_TERMS)
        br = O.bisect_mu(lambda mu: O.poly_trace(mu, taus, KT, c["ea"], c["eb"], N_TERMS), n / 2,
                         c["ea"], c["eb"], KT)
        c["mu"] = br.mu
    else:
        mu = c.get("mu", -6.0)
        coef = O.chebyshev_coeffs(KT, mu, c["ea"], c["eb"], N_TERMS)
        x = O.scale_hamiltonian(c["h"], c["ea"], c["eb"])
        O.chebyshev_naive(x, coef[:terms])
    return time.perf_counter() - t0


def mix_seconds(ns, times):
    """Oracle seconds per step of the N mix from the per-piece times (the recursion scaled by
    (n_terms - 1) / (terms - 1) products)."""
    total = 0.0
    for label, n, kind, terms in cpu_pieces(ns):
        total += times[label] * ((N_TERMS - 1) / max(1, terms - 1) if kind == "rec" else 1.0)
    return total


def cpu_baseline(ns) -> dict:
    """The oracle timed once on every piece of the step's N mix (about 15-25 s on the host
    cores), converted to density matrices per second of the mix."""
    cache, times = {}, {}
    for piece in cpu_pieces(ns):
        times[piece[0]] = run_cpu_piece(piece, cache)
    t = mix_seconds(ns, times)
    return {"value": len(ns) / t, "unit": "density matrices/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "oracle (numpy/LAPACK float64) on the step's own H at every N: the mu search "
                      "(eigvalsh, moments, bisection) whole, the N x N three-term recursion on its first "
                      "terms scaled to all terms; " + "; ".join(f"{k} {v:.2f} s" for k, v in times.items()),
            "seconds_sampled": sum(times.values()), "seconds_per_step_estimated": t,
            "pieces_s": times}


def traffic_record(kernel: str, source: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the
    kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(kernel)
    if not rec:
        return None
    with open(os.path.join(ROOT, source), "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != digest:
        return None
    return rec


# --------------------------------------------------------------- float64 GEMM peak
def fp64_gemm_peak(n: int = 8192, reps: int = 4) -> dict:
    """Measured float64 matrix-product rate of this GPU: torch.matmul (cuBLAS DGEMM) of two
    n x n float64 matrices, 2 n^3 flops, best of `reps` timed with CUDA events after one
    warm-up. The denominator of the float64 path's roofline fraction."""
    import torch
    a = torch.rand((n, n), dtype=torch.float64, device="cuda")
    b = torch.rand((n, n), dtype=torch.float64, device="cuda")
    c = a @ b
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b, c
    torch.cuda.empty_cache()
    return {"tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12, "n": n, "ms": best,
            "how": f"torch.matmul float64 {n}^3 (cuBLAS DGEMM), best of {reps}, CUDA events"}


# ------------------------------------------------- the paper's comparison, re-timed
def eigh_baseline(hs: dict, results: dict, kT: float, reps: int = 2) -> dict:
    """Density matrices by diagonalisation, the comparison the paper times against its
    expansion (cuSolver / MAGMA dsyevd): torch.linalg.eigh in float64 (cuSolver syevd) and
    P = U f(Lambda) U^T (cuBLAS), at the mu the solver found. Library calls; context only."""
    import torch
    out = {}
    for n, h in hs.items():
        mu = results[n]["mu"]
        times = []
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            lam, u = torch.linalg.eigh(h)
            occ = 0.5 - 0.5 * torch.tanh((lam - mu) / (2.0 * kT))
            p = (u * occ) @ u.T
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            del lam, u, p
        out[str(n)] = {"ms": statistics.median(times[1:])}
    return out


# ------------------------------------------------------------- 512-instance batch
def bench_batch(solver, stream, flush, steps, precision, count=512, n_terms=300, rank=0, world=1,
                tile=None):
    """Density matrices per second of the batch of `count` tight-binding instances with N
    log-uniform in [64, 1024] and kT ~ U(0.05, 0.2) eV, replayed as one CUDA graph per batch
    (L2 flushed before each), plus one profiled eager pass for the product roofline. With
    several ranks the instances are sharded by cost (no collective on the data path) and the
    batch time is the maximum over ranks."""
    import torch
    import synth
    from paper_2306_12616_gb300 import FO_FLAG_GRAPH
    from paper_2306_12616_gb300.dist import rank_share, reduce_max
    ns_all = [int(n) for n in synth.batch_sizes(count, 4000)]
    kts_all = [float(t) for t in synth.batch_temperatures(count, 4000)]
    mine = rank_share(ns_all, rank, world)
    ns, kts = [ns_all[i] for i in mine], [kts_all[i] for i in mine]
    hs = [torch.from_numpy(synth.tight_binding(ns_all[i], 4000 + i)).to(flush.device) for i in mine]
    ps = [torch.empty_like(h) for h in hs]
    ne = [n / 2 for n in ns]
    prm = solver.params(n_terms, 0.1, precision=precision, mu_mode="bisect", flags=FO_FLAG_GRAPH,
                        **(tile or {}))
    _, res = solver.density_matrix_batched(hs, ne, prm, kT=kts, outs=ps)   # plan, autotune, capture
    ok = all(r["status"] == 0 for r in res)
    worst_tr = max(abs(r["trace"] - n / 2) / n for r, n in zip(res, ns))
    for _ in range(3):
        solver.density_matrix_batched(hs, ne, prm, kT=kts, outs=ps, sync=False)
    times = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.density_matrix_batched(hs, ne, prm, kT=kts, outs=ps, sync=False)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = reduce_max(statistics.median(times))
    # profiled eager pass: stage times and the product kernel's achieved rate
    prm_e = solver.params(n_terms, 0.1, precision=precision, mu_mode="bisect", **(tile or {}))
    solver.density_matrix_batched(hs, ne, prm_e, kT=kts, outs=ps, sync=False)
    torch.cuda.synchronize()
    solver.profile_enable(True)
    flush.fill_(1.0)
    solver.density_matrix_batched(hs, ne, prm_e, kT=kts, outs=ps, sync=False)
    prof = solver.profile_read(reset=True)
    solver.profile_enable(False)
    pr = prof["products"]
    del hs, ps
    torch.cuda.empty_cache()
    return {"workload": f"{count} tight-binding H, N log-uniform in [64, 1024] (multiples of 4), "
                        f"kT ~ U(0.05, 0.2) eV, N_e = N/2, {n_terms} terms, {precision}, mu by bisection",
            "dm_per_s": count / (ms * 1e-3), "ms_per_batch": ms, "steps": steps, "graph": True,
            "ranks": world, "instances_this_rank": len(ns),
            "scaling": "strong" if world > 1 else None,
            "sum_n3": float(sum(float(n) ** 3 for n in ns_all)), "all_status_ok": ok,
            "worst_trace_err_over_N": worst_tr, "tile_n": res[0]["tile_n"],
            "tile_ctas": res[0]["tile_ctas"], "tile_drain": res[0]["tile_drain"],
            "tile_store": res[0]["tile_store"],
            "eager_ms_per_batch": prof["call"]["ms"],
            "products_achieved_tflops": pr["flops"] / (pr["ms"] * 1e-3) / 1e12 if pr["ms"] > 0 else None,
            "products_share": pr["ms"] / max(1e-9, prof["call"]["ms"]),
            "stages_ms": {k: v["ms"] for k, v in prof.items() if isinstance(v, dict)}}


# ----------------------------- learned expansion order on the 512-instance batch family
def bench_learned_order(solver, stream, flush, steps, count=512, n_terms=300, pairs=2048, lanczos=40,
                        epochs=150):
    """The learned expansion order (FO_MU_ORDER) on the batch family with Lanczos bounds: the
    network is trained on `pairs` method-generated pairs of the family (matrices drawn on the
    device, sizes log-uniform in [64, 1024]), then the 512-instance batch (the batch_512
    matrices) is solved with mu by bisection at the configured 300 terms and with the
    learned order (mu by bisection at that order), each replayed as one CUDA graph, the L2
    flushed before each replay. Reported per form: density matrices/s, products per DM; for
    the learned order the coefficients used, the extra truncation against the 300-term P
    and the trace errors."""
    import numpy as np
    import torch
    import synth
    from synth.device import tight_binding_batch
    from paper_2306_12616_gb300 import FO_FLAG_GRAPH
    dev = flush.device
    t0 = time.perf_counter()
    ns_tr = [int(n) for n in synth.batch_sizes(pairs, 9100)]
    kts_tr = [float(t) for t in synth.batch_temperatures(pairs, 9100)]
    groups = {}
    for i, n in enumerate(ns_tr):
        groups.setdefault(n, []).append(i)
    hs_tr = [None] * pairs
    for n, idx in groups.items():
        hb = tight_binding_batch(len(idx), n, 9200 + n, dev)
        for j, i in enumerate(idx):
            hs_tr[i] = hb[j]
    prm_f = solver.params(n_terms, 0.1, precision="bf16x3", lanczos_steps=lanczos)
    feats, tgts = [], []
    for b0 in range(0, pairs, 512):
        f, t, r = solver.learned_features(hs_tr[b0:b0 + 512], [n / 2 for n in ns_tr[b0:b0 + 512]], prm_f,
                                          kT=kts_tr[b0:b0 + 512])
        if any(x["status"] != 0 for x in r):
            raise RuntimeError("training pair generation failed")
        feats.append(f)
        tgts.append(t)
    del hs_tr, groups
    feat, tgt = torch.cat(feats), torch.cat(tgts)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    solver.mlp_init(91)
    losses = solver.mlp_train(feat, tgt, epochs=epochs, batch=256, lr=1e-3, seed=91)
    train_s = time.perf_counter() - t0
    del feat, tgt, feats, tgts
    torch.cuda.empty_cache()
    ns = [int(n) for n in synth.batch_sizes(count, 4000)]
    kts = [float(t) for t in synth.batch_temperatures(count, 4000)]
    hs = [torch.from_numpy(synth.tight_binding(ns[i], 4000 + i)).to(dev) for i in range(count)]
    ne = [n / 2 for n in ns]
    out = {}
    results = {}
    for label, mode in (("bisection", "bisect"), ("learned_order", "order")):
        ps = [torch.empty_like(h) for h in hs]
        prm = solver.params(n_terms, 0.1, precision="bf16x3", mu_mode=mode, lanczos_steps=lanczos,
                            flags=FO_FLAG_GRAPH)
        _, res = solver.density_matrix_batched(hs, ne, prm, kT=kts, outs=ps)
        for _ in range(3):
            solver.density_matrix_batched(hs, ne, prm, kT=kts, outs=ps, sync=False)
        times = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.density_matrix_batched(hs, ne, prm, kT=kts, outs=ps, sync=False)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        results[label] = (ps, res)
        out[label] = {"dm_per_s": count / (ms * 1e-3), "ms_per_batch": ms,
                      "products_per_dm": float(np.mean([r["n_gemm"] for r in res])),
                      "all_status_ok": all(r["status"] == 0 for r in res),
                      "worst_trace_err": max(abs(r["trace"] - x) for r, x in zip(res, ne))}
    po, ro = results["learned_order"]
    pb, _ = results["bisection"]
    extra = [float(torch.linalg.norm(a - b)) / math.sqrt(n) for a, b, n in zip(po, pb, ns)]
    used = [r["order"] for r in ro]
    out["learned_order"].update({
        "coefficients_used": {"min": min(used), "median": float(np.median(used)), "max": max(used),
                              "of": n_terms},
        "extra_truncation_vs_full_order": {"median": float(np.median(extra)), "max": max(extra),
                                           "metric": "||P_order - P_300||_F / sqrt(N)"}})
    del hs, results, po, pb
    torch.cuda.empty_cache()
    return {"workload": f"{count} tight-binding H (the batch_512 matrices), N log-uniform in [64, 1024], "
                        f"kT ~ U(0.05, 0.2) eV, N_e = N/2, {n_terms} terms, bf16x3, Lanczos bounds "
                        f"({lanczos} steps), one CUDA graph per batch",
            "training": {"pairs": pairs, "epochs": epochs, "pair_generation_s": gen_s, "train_s": train_s,
                         "loss_first": losses[0], "loss_last": losses[-1]},
            "forms": out}


# ------------------------------------------- learned mu on the metallic model (N = 1024)
def bench_learned_metallic(solver, stream, pairs=20000, held_out=64, n=1024, n_terms=1000, kT=0.01,
                           epochs=150, chunk=64, reps=3, tr_tols=(None, 0.5)):
    """The learned chemical potential on a high density of states at the Fermi level:
    metallic Hamiltonians (N = 1024, 25 % of the onsite energies ~ N(0, 0.02 eV)), kT =
    0.01 eV, 1000 terms, N_e = 0.775 N (Fermi level at 0 eV), BF16x3. The network is trained
    on `pairs` (H, mu) pairs that the exact method generates (matrices drawn on the device,
    N_e ~ U(0.74, 0.81) N), then a held-out batch of `held_out` matrices is solved with mu
    by bisection (the judge) and with the learned proposal, at the default trace tolerance
    (1e-7 N, the split form's rounding band, then the trace correction to 1e-8) and at half an
    electron; reported per form: density matrices/s (CUDA events,
    eager calls), products per density matrix, evaluations of P, acceptance, and the
    proposal error against the exact mu."""
    import numpy as np
    import torch
    import synth
    from synth.device import metallic_batch
    dev = torch.device("cuda", torch.cuda.current_device())
    prm = solver.params(n_terms, kT, precision="bf16x3")
    rng = np.random.default_rng(5500)
    t0 = time.perf_counter()
    feats, tgts = [], []
    for b in range((pairs + chunk - 1) // chunk):
        hb = metallic_batch(chunk, n, 6000 + b, dev)
        ne = rng.uniform(0.74, 0.81, chunk) * n
        f, t, res = solver.learned_features([hb[i] for i in range(chunk)], ne, prm)
        if any(r["status"] != 0 for r in res):
            raise RuntimeError("training pair generation failed")
        feats.append(f)
        tgts.append(t)
        del hb
    feat, tgt = torch.cat(feats)[:pairs], torch.cat(tgts)[:pairs]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    solver.mlp_init(55)
    losses = solver.mlp_train(feat, tgt, epochs=epochs, batch=256, lr=1e-3, seed=55)
    train_s = time.perf_counter() - t0
    del feat, tgt, feats, tgts
    hs = [torch.from_numpy(synth.metallic(n, 5000 + i)).to(dev) for i in range(held_out)]
    ne = [synth.metallic_electrons(n)] * held_out
    outs = [torch.empty_like(h) for h in hs]

    def timed(p):
        _, res = solver.density_matrix_batched(hs, ne, p, outs=outs)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.density_matrix_batched(hs, ne, p, outs=outs)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        return res, {"dm_per_s": held_out / (ms * 1e-3), "ms_per_batch": ms,
                     "products_per_dm": float(np.mean([r["n_gemm"] for r in res])),
                     "all_status_ok": all(r["status"] == 0 for r in res),
                     "worst_trace_err": max(abs(r["trace"] - x) for r, x in zip(res, ne)),
                     "worst_trace_raw_err": max(abs(r["trace_raw"] - x) for r, x in zip(res, ne)),
                     "trace_corrected": float(np.mean([r["trace_gamma"] != 0.0 for r in res]))}

    rb, bis = timed(solver.params(n_terms, kT, precision="bf16x3", mu_mode="bisect"))
    # proposal error of the trained network on the held-out batch, against the exact mu
    f_h, _, _ = solver.learned_features(hs, ne, prm)
    _, norm = solver.mlp_get_params()
    y = solver.mlp_forward((f_h - torch.tensor(norm[:68], device=dev)) / torch.tensor(norm[68:136], device=dev))
    mux = y[:, 0].double().cpu().numpy() * norm[138] + norm[136]
    mu0 = np.array([0.5 * (r["emin"] + r["emax"]) + 0.5 * (r["emax"] - r["emin"]) * x for r, x in zip(rb, mux)])
    err = np.abs(mu0 - np.array([r["mu"] for r in rb]))
    forms = {"bisection": bis}
    for tol in tr_tols:
        kw = {"tr_tol": tol} if tol is not None else {}
        rl, st = timed(solver.params(n_terms, kT, precision="bf16x3", mu_mode="learned", max_newton=3, **kw))
        st["accepted"] = float(np.mean([r["learned_accepted"] for r in rl]))
        st["evaluations"] = float(np.mean([r["evals"] for r in rl]))
        st["tr_tol"] = tol if tol is not None else f"1e-7 N = {1e-7 * n:g}"
        forms["learned_tol_" + ("default" if tol is None else f"{tol:g}")] = st
    del hs, outs
    torch.cuda.empty_cache()
    return {"workload": f"{held_out} metallic H (tight-binding hopping, 25% of onsite energies ~ N(0, 0.02 eV)), "
                        f"N={n}, N_e={ne[0]:g}, kT={kT} eV, {n_terms} terms, bf16x3",
            "training": {"pairs": pairs, "epochs": epochs, "pair_generation_s": gen_s, "train_s": train_s,
                         "loss_first": losses[0], "loss_last": losses[-1]},
            "proposal_err_eV": {"median": float(np.median(err)), "max": float(err.max())},
            "forms": forms}


# --------------------------------------------------------------------------- main
def run_reference(args, rank, world):
    """The oracle on the host cores. Each step (warm-up or timed) runs the next piece of the
    oracle's work for the N mix in turn (a mu search or a column block of the recursion, on
    the workload's own H); pieces the timed steps did not reach are timed after them, so that
    every piece is measured. value = DMs of the mix per second estimated from the median time
    of each piece; ms_per_step = the measured mean time of the timed steps."""
    if rank != 0:
        return
    ns = [int(x) for x in args.ns.split(",")]
    pieces = cpu_pieces(ns)
    cache, seen = {}, {}
    for w in range(args.warmup):
        run_cpu_piece(pieces[w % len(pieces)], cache)
    step_s = []
    for j in range(args.steps):
        piece = pieces[(args.warmup + j) % len(pieces)]
        t = run_cpu_piece(piece, cache)
        step_s.append(t)
        seen.setdefault(piece[0], []).append(t)
    for piece in pieces:
        if piece[0] not in seen:
            seen[piece[0]] = [run_cpu_piece(piece, cache)]
    times = {k: statistics.median(v) for k, v in seen.items()}
    value = len(ns) / mix_seconds(ns, times)
    sample = ("oracle (numpy/LAPACK float64) on the workload's own H, one piece per step in turn: "
              + "; ".join(f"{k} {v:.2f} s" for k, v in times.items())
              + "; recursion scaled by its number of products")
    out = {"metric": METRIC, "value": value, "unit": "density matrices/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": statistics.mean(step_s) * 1e3 if step_s else None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n": ns, "n_terms": args.n_terms, "kT_eV": KT,
                      "precision": "fp64 (numpy/LAPACK oracle)"},
           "cpu_baseline": {"value": value, "unit": "density matrices/s", "cores": os.cpu_count(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "density matrices/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import synth
    from paper_2306_12616_gb300 import Solver
    from paper_2306_12616_gb300.dist import reduce_max

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.batch_only:
        solver = Solver(local)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        b = bench_batch(solver, torch.cuda.current_stream(), flush, max(1, args.steps), args.precision,
                        count=args.batch_count, rank=rank, world=world, tile=tile_args(args.tile, args.chain, args.chain_window))
        if rank == 0:
            print(json.dumps({"metric": "density matrices/s (batch)", "value": b["dm_per_s"],
                              "unit": "density matrices/s", "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": b["ms_per_batch"], "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                              "config": {"workload": b["workload"]}, "batch": b}), flush=True)
        solver.close()
        return
    if args.learned_only:
        solver = Solver(local)
        out = bench_learned_metallic(solver, torch.cuda.current_stream(), pairs=args.learned_pairs)
        if rank == 0:
            print(json.dumps({"learned_mu_metallic": out}), flush=True)
        solver.close()
        return
    ns = [int(x) for x in args.ns.split(",")]
    solver = Solver(local)
    stream = torch.cuda.current_stream()
    prm = solver.params(args.n_terms, KT, precision=args.precision, mu_mode="bisect", **tile_args(args.tile, args.chain, args.chain_window))

    # inputs resident in HBM (a different replica per rank)
    hs, ps, hcpu = {}, {}, {}
    for n in ns:
        h = synth.tight_binding(n, 2000 + n + 100003 * rank)
        hcpu[n] = torch.from_numpy(h).pin_memory()
        hs[n] = hcpu[n].to(dev)
        ps[n] = torch.empty((n, n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    hl, pl, nel = [hs[n] for n in ns], [ps[n] for n in ns], [n / 2 for n in ns]

    # validation pass: status, trace, and every split form against the FP64 GPU path
    accuracy, fp64_ms, results, fp64_gemms = {}, {}, {}, {}
    _, res_b = solver.density_matrix_batched(hl, nel, prm, outs=pl)
    others = [x for x in ("bf16x3", "fp16x2", "bf16x1") if x != args.precision]
    for n, res in zip(ns, res_b):
        results[n] = res
        accuracy[n] = {"trace_minus_Ne": res["trace"] - n / 2, "trace_raw_minus_Ne": res["trace_raw"] - n / 2,
                       "trace_gamma": res["trace_gamma"]}
        if not args.no_fp64_check and args.precision != "fp64":
            p64 = torch.empty_like(ps[n])
            prm64 = solver.params(args.n_terms, KT, precision="fp64", mu_mode="bisect")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, r64 = solver.density_matrix(hs[n], n / 2, prm64, out=p64)
            fp64_ms[n] = (time.perf_counter() - t0) * 1e3
            fp64_gemms[n] = r64["n_gemm"]
            accuracy[n].update({"dP_frob_over_sqrtN": float(torch.linalg.norm(ps[n] - p64) / math.sqrt(n)),
                                "dmu": res["mu"] - r64["mu"], "fp64_trace_minus_Ne": r64["trace"] - n / 2})
            # the other split forms on the same H, against the same float64 P
            forms = {}
            for prec2 in others:
                q = torch.empty_like(ps[n])
                _, r2 = solver.density_matrix(hs[n], n / 2, solver.params(args.n_terms, KT, precision=prec2,
                                                                          mu_mode="bisect"), out=q)
                forms[prec2] = {"dP_frob_over_sqrtN": float(torch.linalg.norm(q - p64) / math.sqrt(n)),
                                "trace_minus_Ne": r2["trace"] - n / 2,
                                "trace_raw_minus_Ne": r2["trace_raw"] - n / 2,
                                "trace_gamma": r2["trace_gamma"], "status": r2["status"]}
                del q
            accuracy[n]["other_split_forms"] = forms
            del p64

    def step():
        solver.density_matrix_batched(hl, nel, prm, outs=pl, sync=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, events on the launching stream, L2 flushed before each step
    def timed_region():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        solver.profile_enable(True)
        per_step = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            per_step.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        prof = solver.profile_read(reset=True)
        solver.profile_enable(False)
        return per_step, prof, clocks.stop()

    # a region that saw a hardware or thermal slowdown on any rank is measured once more by
    # every rank (sw_power_cap is the normal state of a dense tensor-core load and is only
    # reported); the decision is reduced over the ranks so that their barriers stay paired
    throttled = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    per_step, prof, clk = timed_region()
    first = sorted(throttled & set(clk.get("reasons", [])))
    if reduce_max(1.0 if first else 0.0) > 0.0:
        per_step, prof, clk = timed_region()
        clk["remeasured_after"] = first or ["another rank"]
    total_ms = reduce_max(sum(per_step))
    ms_per_step = total_ms / args.steps
    value = world * len(ns) / (ms_per_step * 1e-3)

    # end to end through the host-buffer C ABI call (H2D + solve + D2H inside the region):
    # one batched host call per step from pinned buffers, enqueued without waiting
    # (FO_FLAG_NO_RESULT_SYNC), so that the library overlaps a step's input copy and the
    # previous step's output copy with a solve; the region ends when every output is on the
    # host (fo_host_wait)
    from paper_2306_12616_gb300 import FO_FLAG_NO_RESULT_SYNC, FoParams
    hout = [torch.empty((n, n), dtype=torch.float64).pin_memory() for n in ns]
    hin = [hcpu[n] for n in ns]
    solver.density_matrix_batched_host(hin, nel, prm, hout)
    prm_async = FoParams.from_buffer_copy(prm)
    prm_async.flags |= FO_FLAG_NO_RESULT_SYNC
    e2e_steps = max(2, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.density_matrix_batched_host(hin, nel, prm_async, hout)
    solver.host_wait()
    e2e_ms = reduce_max((time.perf_counter() - t0) * 1e3 / e2e_steps)
    e2e_bytes = sum(8 * n * n for n in ns)
    # the host copies of the last step equal the device-resident results of the timed steps
    e2e_dev = max(float((hout[j] - pl[j].cpu()).abs().max()) for j in range(len(ns)))

    # what the trace correction costs: the same steps without it (FO_FLAG_NO_TRACE_FIX)
    fix_cost = None
    if args.precision != "fp64":
        from paper_2306_12616_gb300 import FO_FLAG_NO_TRACE_FIX
        prm_nf = solver.params(args.n_terms, KT, precision=args.precision, mu_mode="bisect",
                               flags=FO_FLAG_NO_TRACE_FIX, **tile_args(args.tile, args.chain, args.chain_window))
        solver.density_matrix_batched(hl, nel, prm_nf, outs=pl)
        nf = []
        for _ in range(max(3, args.steps // 4)):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.density_matrix_batched(hl, nel, prm_nf, outs=pl, sync=False)
            e1.record(stream)
            e1.synchronize()
            nf.append(e0.elapsed_time(e1))
        nf_ms = statistics.median(nf)
        fix_cost = {"ms_per_step_without": nf_ms, "dm_per_s_without": len(ns) / (nf_ms * 1e-3),
                    "ms_per_step_with": statistics.median(per_step),
                    "extra_products_per_dm": 1, "extra_share": statistics.median(per_step) / nf_ms - 1.0}
        solver.density_matrix_batched(hl, nel, prm, outs=pl)   # leave the corrected P in place

    pk, pk_kind = peaks()
    prod = prof["products"]
    achieved = prod["flops"] / (prod["ms"] * 1e-3) / 1e12 if prod["ms"] > 0 else None
    f64pk = fp64_gemm_peak() if (rank == 0 and (args.precision == "fp64" or fp64_ms)) else None
    if args.precision == "fp64":
        peak = f64pk["tflops"] if f64pk else None
        unit_peak = "TFLOP/s"
    else:
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        if args.precision == "fp16x2":
            peak = peak  # fp16 and bf16 share the dense tensor rate
        unit_peak = "TFLOP/s"
    kernel_name = "k_tc_gemm" if args.precision != "fp64" else "k_gemm_f64"
    trec = traffic_record(kernel_name, "paper_2306_12616_gb300/csrc/gemm_tc.cu"
                          if args.precision != "fp64" else "paper_2306_12616_gb300/csrc/gemm_f64.cu")
    launches_per_step = prof["call"]["launches"] / max(1, args.steps)
    roof = {"bound": "tensor", "kernel": kernel_name, "achieved": achieved, "peak": peak,
            "unit": unit_peak, "frac": (achieved / peak) if (achieved and peak) else None,
            "peak_kind": (f"{pk_kind} bf16 sustained" if args.precision != "fp64"
                          else "measured fp64 DGEMM (fp64_gemm_peak)") if peak else None,
            "avg_launch_ms": prod["ms"] / max(1, prod["launches"]),
            "launches_timed": prod["launches"],
            "share_of_step": prod["ms"] / max(1e-9, prof["call"]["ms"]),
            "traffic": (trec["bytes_per_launch"] if trec else None),
            "traffic_note": (trec["note"] if trec else "no ncu capture of the current kernel source")}
    batch = None if args.no_batch else bench_batch(solver, stream, flush, max(3, args.steps // 2),
                                                    args.precision, count=args.batch_count,
                                                    rank=rank, world=world, tile=tile_args(args.tile, args.chain, args.chain_window))
    eigh = None if args.no_fp64_check else eigh_baseline(hs, results, KT)
    learned = None
    if not args.no_learned and rank == 0:
        try:
            learned = bench_learned_metallic(solver, stream, pairs=args.learned_pairs)
        except Exception as exc:   # reported, never fatal to the headline measurement
            learned = {"error": f"{type(exc).__name__}: {exc}"}
    order = None
    if not args.no_order and not args.no_batch and rank == 0 and args.precision == "bf16x3":
        try:
            order = bench_learned_order(solver, stream, flush, max(3, args.steps // 2), count=args.batch_count)
        except Exception as exc:   # reported, never fatal to the headline measurement
            order = {"error": f"{type(exc).__name__}: {exc}"}
    cb = cpu_baseline(ns) if (rank == 0 and world == 1) else None
    per_n = {}
    for n in ns:
        per_n[str(n)] = {"n_gemm": results[n]["n_gemm"], "k": results[n]["k"], "m": results[n]["m"],
                         "bisect_iters": results[n]["bisect_iters"], "mu_eV": results[n]["mu"],
                         "status": results[n]["status"], "tile_n": results[n]["tile_n"],
                         "tile_ctas": results[n]["tile_ctas"], "tile_drain": results[n]["tile_drain"],
                         "tile_store": results[n]["tile_store"]}
        if n in accuracy:
            per_n[str(n)].update(accuracy[n])
        if n in fp64_ms:
            per_n[str(n)]["fp64_gpu_ms"] = fp64_ms[n]
    # the float64 path (one call per N, wall time around a synchronised call) against the
    # measured float64 GEMM rate: n_gemm symmetric products of n^2 (n + 1) flops each
    fp64_roof = None
    if fp64_ms and f64pk:
        fl = sum(fp64_gemms[n] * n * n * (n + 1.0) for n in fp64_ms)
        tt = sum(fp64_ms.values()) * 1e-3
        fp64_roof = {"bound": "fp64", "achieved": fl / tt / 1e12, "peak": f64pk["tflops"], "unit": "TFLOP/s",
                     "frac": fl / tt / 1e12 / f64pk["tflops"], "peak_how": f64pk["how"],
                     "note": "whole float64 calls (products, moments, contraction, mu) over the product flops"}
    stages = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps}
              for k, v in prof.items() if isinstance(v, dict)}
    if args.precision != "fp64":
        # algorithmic bytes per step of the HBM-bound stages (float32 masters kept on and above
        # the diagonal, 16-bit planes in full; n_pad = N rounded up to 128) and the rate reached
        hbm = pk.get("hbm_gbs")
        # (tr P and ||P||_F^2 are summed in the epilogue of the product that writes P: the trace
        # stage only adds the per-tile partials and touches the diagonal, so it is not listed)
        byts = {"bounds": 0.0, "moments": 0.0, "contract": 0.0}
        for n in ns:
            kk, mm = results[n]["k"], results[n]["m"]
            npad = -(-n // 128) * 128
            sp = {"bf16x3": 3, "fp16x2": 2, "bf16x1": 1}[args.precision]   # 16-bit planes
            byts["bounds"] += 8 * n * n + 8 * n * (n + 1) / 2 + (4 + 2 * sp) * npad * npad
            byts["moments"] += (kk - 1 + mm - 1) * 4 * npad * (npad + 128) / 2
            byts["contract"] += (kk - 1 + mm) * 4 * npad * (npad + 4) / 2 + 3 * sp * npad * npad
        for name, b in byts.items():
            t = stages[name]["ms_per_step"] * 1e-3
            stages[name]["algorithmic_bytes"] = b
            stages[name]["achieved_gbs"] = b / t / 1e9 if t > 0 else None
            stages[name]["frac_of_hbm"] = (b / t / 1e9) / hbm if (t > 0 and hbm) else None
    out = {
        "metric": METRIC, "value": value, "unit": "density matrices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if args.precision != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": ns, "n_terms": args.n_terms, "kT_eV": KT,
                   "precision": f"{args.precision} split products, fp32 accumulation; fp64 bounds, "
                                f"coefficients, moments, traces and mu" if args.precision != "fp64"
                   else "fp64 throughout",
                   "parallelism": f"replicas x{world}", "l2": "flushed before every timed step "
                   "(256 MiB write); per-step working set several GB > L2"},
        "e2e": {"value": world * len(ns) / (e2e_ms * 1e-3), "unit": "density matrices/s",
                "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes, "steps": e2e_steps,
                "pipelined": "host-buffer calls enqueued back to back, input and output copies on "
                             "copy streams overlapping the neighbouring steps' solves",
                "max_abs_diff_vs_device": e2e_dev},
        "gpu_launches": int(round(launches_per_step)) * args.steps,
        "roofline": roof,
        "cpu_baseline": cb,
        "clocks": clk,
        "per_n": per_n,
        "stages": stages,
        "fp64_gpu_dm_per_s": (len(fp64_ms) / (sum(fp64_ms.values()) * 1e-3)) if fp64_ms else None,
        "fp64_gpu_roofline": fp64_roof,
        "trace_correction": fix_cost,
        "batch_512": batch,
        "eigh_fp64_cusolver": eigh,
        "learned_mu_metallic": learned,
        "learned_order_batch": order,
        "paper_context": PAPER_CONTEXT,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
