"""Benchmark of the block Wiedemann rank path on GB300.

Default workload (one GPU): the K-theory-scale matrix sized after GL7d19
(Table tab:res): 1,900,000 x 1,950,000, ~40.7M nnz (Poisson 19.5 per row,
uniform columns), planted rank 1,805,000, block m = n = 32, p = 2147483629,
L = 118,752 terms.

A timed step is the next stretch of that sequence: TERMS_PER_STEP = 256 terms
S_0 .. S_255 with the symmetric projection of Section 2.3 (X = Y^T; the
paper's own choice), i.e. 128 applications of the preconditioned black box to
the block D1 Y (width 32) with both SpMM passes and the two Gram projections
of each application (S_2k = V_k^T V_k after pass 2, S_2k+1 from pass 1's
output; the captured 64-application graphs of the sequence loop), plus the
sequence set-up (D1, D2, Y, T_0, S_0).  Inputs are resident in HBM (the matrix
loaded once).  value = SpMM nnz*vec per second over the timed steps (2 passes
x nnz x 32 block columns per application; --projection generic: the paired
block [D1 X | D1 Y] of width 64).  In the same run: the whole time to rank of
the workload (ingest from pinned host CSR, all L terms, sigma-basis trailing
the sequence, readout; e2e), the same with the generic
projection (an independent X, Section 2.5), the secondary 200,000 x 180,000
block-8 workload's time to rank, the roofline of k_spmm and the CPU oracle on
a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wr|reference]
                    [--matrix c2|c1] [--projection symmetric|generic] [--pipeline 0|1|2|3]
                    [--no-time-to-rank] [--no-generic-time-to-rank]
                    [--chain-reduction] [--locality-order] [--early-termination ORDERS]
                    [--workload single|batch|serve] [--only-blackbox | --only-sigma | --probe-mma]

With N > 1 (torchrun, one rank per GPU) every rank computes its column slab of
Y (Section 3.1: column block j of S_i depends on Y_j only; wr_sequence_slab_device)
for the same step terms, with no exchange while iterating, and the slabs are
all-gathered once per step over NCCL (strong scaling: the step's terms are the
same for every N).
--impl reference times the CPU oracle on the host cores on a bounded sample of
the same workload (one application per step).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mod-p SpMM nnz·vec/s, %HBM peak; batched/served vs plain time-to-rank (exact)"
UNIT = "nnz*vec/s"
TERMS_PER_STEP = 256


def workload(rank: int = 0, matrix: str = "c2"):
    """The bench matrix and its parameters (seeded; rank > 0 only for the
    independent-matrix mode)."""
    from paper_0704_2351_gb300 import synth
    if matrix == "c1":
        seed = synth.SEED_BASE + 1 + 1000 * rank
        A = synth.config1(seed=seed)
        return A, dict(p=synth.PRIME_C1, m=8, n=8, seed=seed, key="c1", name=(
            "power-law sparse matrix 200000x180000, %d nnz (20/row base, alpha 2.1 column degrees), planted rank "
            "170000; block Wiedemann m=n=8 mod p=1073741789, L=45002" % A.nnz))
    seed = synth.SEED_BASE + 2 + 1000 * rank
    A = synth.config2(seed=seed)
    return A, dict(p=synth.PRIME_C2, m=32, n=32, seed=seed, key="c2", name=(
        "K-theory-scale sparse matrix 1900000x1950000 (after GL7d19), %d nnz (Poisson 19.5/row, uniform "
        "columns), planted rank 1805000; block Wiedemann m=n=32 mod p=2147483629, L=118752" % A.nnz))


def spmm_traffic(width, kernel_file="paper_0704_2351_gb300/csrc/wr_spmm_kernel.cuh",
                 summary="profiles/spmm_traffic_config2.md"):
    """DRAM bytes (read + write) per k_spmm launch on the bench workload at
    the given block width, from the committed ncu summary's line
    `traffic_bytes_per_launch: X source_sha256: Y width: W`; None when the
    SpMM source has changed since that capture (Y differs from the current
    file's hash) or there is no line for that width."""
    try:
        text = open(os.path.join(ROOT, summary)).read()
        src = hashlib.sha256(open(os.path.join(ROOT, kernel_file), "rb").read()).hexdigest()
    except OSError:
        return None, "no summary"
    stale = False
    for line in text.splitlines():
        if line.strip().startswith("traffic_bytes_per_launch:"):
            f = line.split()
            try:
                val, sha, w = float(f[1]), f[3], int(f[5])
            except (IndexError, ValueError):
                continue
            if w != width:
                continue
            if sha != src:
                stale = True
                continue
            return val, summary
    return None, ("k_spmm source changed since the capture" if stale else "no traffic line for width %d" % width)


def apply_options(wr, ctx, args):
    """Read-time passes and early termination, when asked for (all off by
    default), and the column-slab size of the SpMM passes (0: the library's
    default)."""
    wr.wr_set_chain_reduction(ctx, bool(getattr(args, "chain_reduction", False)))
    wr.wr_set_locality_order(ctx, bool(getattr(args, "locality_order", False)))
    wr.wr_set_early_termination(ctx, int(getattr(args, "early_termination", 0)))
    wr.wr_set_pipeline(ctx, int(getattr(args, "pipeline", 1)))
    wr.wr_set_projection_overlap(ctx, bool(getattr(args, "projection_overlap", False)))
    if int(getattr(args, "lane_width", 0)):
        wr.wr_set_lane_width(ctx, int(args.lane_width))
    wr.wr_set_tensor_projection(ctx, int(getattr(args, "tensor_projection", -1)))
    wr.wr_set_column_slabs(ctx, int(getattr(args, "slab_bytes", 0)))


def options_config(args):
    out = {"chain_reduction": bool(getattr(args, "chain_reduction", False)),
           "locality_order": bool(getattr(args, "locality_order", False)),
           "early_termination_orders": int(getattr(args, "early_termination", 0))}
    if int(getattr(args, "slab_bytes", 0)) != 0:
        out["column_slab_bytes"] = int(args.slab_bytes)
    out["pipeline"] = {0: "off", 1: "automatic", 2: "sigma-basis first",
                       3: "sequence first"}[int(getattr(args, "pipeline", 1))]
    if bool(getattr(args, "projection_overlap", False)):
        out["projection_overlap"] = True
    if int(getattr(args, "lane_width", 0)):
        out["lane_width"] = int(args.lane_width)
    if int(getattr(args, "tensor_projection", -1)) != -1:
        out["tensor_projection"] = int(args.tensor_projection)
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def start_clock_sampler(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        return subprocess.Popen(cmd, stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def stop_clock_sampler(proc, path, device):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or f[0] != str(device):
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


def cpu_baseline(A, cfg, budget_s=15.0, terms_cap=400):
    """The oracle as it stands, on the host's cores, over the first terms of
    the same sequence (each term after S_0 = one black-box application = 2
    sparse passes over Y alone), bounded to about budget_s seconds; the CPU
    time of the whole L-term sequence is extrapolated from it (labelled)."""
    import oracle
    st = oracle.Setup(A, cfg["p"], cfg["m"], cfg["n"], cfg["seed"], symmetric=cfg.get("symmetric", False))
    t = time.perf_counter()
    oracle.sequence(A, st, L=2)
    per = max(time.perf_counter() - t, 1e-4)
    terms = int(min(terms_cap, max(2, budget_s / per)))
    if terms == 2:  # one application already takes the budget: that run is the sample
        el = per
    else:
        t = time.perf_counter()
        oracle.sequence(A, st, L=terms)
        el = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0))
    v = 2.0 * A.nnz * cfg["n"] * (terms - 1) / el
    L = oracle.seq_length(st.N, cfg["m"], cfg["n"])
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d terms of the same sequence (%d black-box applications to Y, 2 sparse passes "
                      "each, %.1f s)" % (terms, terms - 1, el),
            "sequence_s_extrapolated": el / (terms - 1) * (L - 1),
            "extrapolation": "x (L - 1) / %d applications, L = %d" % (terms - 1, L)}


def run_blackbox_only(args):
    """Black-box applications only (matrix ingest, then W + K applications):
    for profiler captures of the SpMM passes and for the SpMM rate on a
    matrix whose working set exceeds L2.  --matrix c1: the bench workload
    (block 8); --matrix c2: the 1,900,000 x 1,950,000 Poisson-row matrix of
    ~37M nnz with block 32 (p = 2147483629), where the gathered block alone
    (1.9M x 128 bytes) is twice the L2.  Prints per-pass times from the
    library's CUDA-event samples and the algorithmic GB/s against the HBM
    peak."""
    import torch
    from paper_0704_2351_gb300 import wr
    A, cfg = workload(0, args.matrix)
    p, n, seed, name = cfg["p"], cfg["n"], cfg["seed"], cfg["name"]
    ctx = wr.wr_create(0)
    apply_options(wr, ctx, args)
    mat = wr.wr_matrix_load_csr(ctx, A.rows, A.cols, A.rowptr, A.colidx, A.vals)
    N = min(A.rows, A.cols)
    g = torch.Generator().manual_seed(seed)
    v = torch.randint(0, p, (N, n), generator=g, dtype=torch.int64).to(torch.int32).cuda()
    out = torch.empty_like(v)
    prm = wr.make_params(p, 1, n, seed)
    for _ in range(args.warmup):
        wr.wr_blackbox_apply_device(ctx, mat, prm, v, out, n)
    wr.wr_set_profiling(ctx, True)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        wr.wr_blackbox_apply_device(ctx, mat, prm, v, out, n)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t) / max(args.steps, 1)
    # per-pass algorithmic bytes, as the library counts them for the loop
    nv = 1 << max(0, (n - 1).bit_length())
    per_pass = [4.0 * A.nnz + 4.0 * nv * (A.rows + A.cols) + 4.0 * r for r in (A.rows, A.cols)]
    peak = measured_peaks().get("hbm_gbs")
    line = {"only": "blackbox", "workload": name, "steps": args.steps, "ms_per_application_wall": ms,
            "algorithmic_bytes_per_pass": per_pass,
            "gbs_per_pass_at_wall_time": 1e-6 * sum(per_pass) / ms, "hbm_peak_gbs": peak,
            "options": options_config(args)}
    print(json.dumps(line), flush=True)
    wr.wr_matrix_free(mat)
    wr.wr_destroy(ctx)
    return 0


def run_batch(args):
    """Batched workload: chain-complex pairs (d_n, d_{n+1}, d_n d_{n+1} = 0)
    with row counts log-uniform in [5,000, 300,000], each matrix solved
    modulo 4 primes below 2^30 (rank over Q = the maximum).  Plain = every job
    through wr_rank one at a time; batched = one wr_rank_batch call.  Both
    are timed end to end (host clock, results copied back); every batched
    rank must equal the plain one and the planted rank."""
    import torch
    from paper_0704_2351_gb300 import synth, wr
    pairs = synth.config3_pairs(npairs=args.pairs)
    mats = [A for pr in pairs for A in pr]
    primes = []
    c = (1 << 30) - 1
    while len(primes) < 4:
        if all(c % d for d in range(2, int(c ** 0.5) + 1)):
            primes.append(c)
        c -= 2
    ctx = wr.wr_create(0)
    apply_options(wr, ctx, args)
    wr.wr_set_batch_slots(ctx, args.slots)
    wr.wr_set_batch_fusion(ctx, not args.no_batch_fusion)
    handles = [wr.wr_matrix_load_csr(ctx, A.rows, A.cols, A.rowptr, A.colidx, A.vals) for A in mats]
    b = args.block
    jobs = [(i, p) for i in range(len(mats)) for p in primes]
    params = [wr.make_params(p, b, b, synth.SEED_BASE + 3 + 7 * i) for (i, p) in jobs]
    # warm-up (module load, first graph instantiation)
    small = min(range(len(mats)), key=lambda i: mats[i].nnz)
    wr.wr_result_free(wr.wr_rank(ctx, handles[small], params[small * 4]))
    torch.cuda.synchronize()
    t = time.perf_counter()
    plain = []
    phases = {"sequence_ms": 0.0, "sigma_ms": 0.0, "sigma_tail_ms": 0.0, "readout_ms": 0.0}
    for h, (i, p), prm in zip([handles[i] for i, _ in jobs], jobs, params):
        res = wr.wr_rank(ctx, h, prm)
        plain.append(wr.wr_result_rank(res))
        wr.wr_result_free(res)
        tm = wr.wr_last_timings(ctx)
        for k in phases:
            phases[k] += tm[k]
    t_plain = time.perf_counter() - t
    t = time.perf_counter()
    outs = wr.wr_rank_batch(ctx, [handles[i] for i, _ in jobs], params)
    t_batch = time.perf_counter() - t
    batched = [wr.wr_result_rank(o) for o in outs]
    for o in outs:
        wr.wr_result_free(o)
    assert batched == plain, "batched ranks differ from the plain ones"
    for k, (i, p) in enumerate(jobs):
        assert batched[k] == mats[i].rank, "job %d: rank %d != planted %d" % (k, batched[k], mats[i].rank)
    rank_q = [max(batched[4 * i: 4 * i + 4]) for i in range(len(mats))]
    chain_ok = all(rank_q[2 * k] + rank_q[2 * k + 1] <= pairs[k][0].cols for k in range(len(pairs)))
    work = sum(2.0 * mats[i].nnz * b * ((-(-min(mats[i].rows, mats[i].cols) // b)) * 2 + 1) for i, _ in jobs)
    line = {"metric": METRIC, "workload": "batched", "value": work / t_batch, "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "int64", "data": "synthetic",
            "config": {"pairs": args.pairs, "matrices": len(mats), "primes": primes, "jobs": len(jobs),
                       "block": [b, b], "slots": args.slots, "options": options_config(args),
                       "fusion": "jobs on one matrix share one sequence loop (up to 4 primes per block)"
                                 if not args.no_batch_fusion else "off",
                       "rows": [int(min(A.rows for A in mats)), int(max(A.rows for A in mats))],
                       "nnz_total": int(sum(A.nnz for A in mats))},
            "plain_s": t_plain, "batched_s": t_batch, "speedup": t_plain / t_batch,
            "plain_phases_ms_summed": {k: round(v, 1) for k, v in phases.items()},
            "ranks_equal_planted": True, "chain_rank_sum_ok": chain_ok,
            "gpu_launches_batched": wr.wr_last_timings(ctx)["kernel_launches"]}
    print(json.dumps(line), flush=True)
    for h in handles:
        wr.wr_matrix_free(h)
    wr.wr_destroy(ctx)
    return 0


def _latency_stats(lat):
    lat = sorted(lat)
    pick = lambda q: lat[min(len(lat) - 1, max(0, int(math.ceil(q * len(lat))) - 1))]
    return {"p50_ms": pick(0.5), "p99_ms": pick(0.99), "mean_ms": sum(lat) / len(lat)}


def run_serve(args):
    """Served workload: a Poisson trace of rank queries (rows log-uniform in
    [1,000, rows_hi], 10-20 nnz/row, planted rank 0.95 min(R, C), 4 primes
    below 2^30, m = n = 16).  Plain = one request at a time in arrival order
    (latency = queueing behind earlier requests + own time, from the measured
    service times).  Served = the continuous-batching server fed at the
    trace's arrival times, at the trace rate and at 0.7x the plain capacity."""
    import torch
    from paper_0704_2351_gb300 import synth, wr
    trace = synth.config4_trace(nreq=args.requests, rate=args.rate, hi=args.rows_hi)
    primes = [1073741789, 1073741783, 1073741741, 1073741723]
    mats = [synth.config4_matrix(r) for r in trace]
    ctx = wr.wr_create(0)
    apply_options(wr, ctx, args)
    handles = [wr.wr_matrix_load_csr(ctx, A.rows, A.cols, A.rowptr, A.colidx, A.vals) for A in mats]
    b = args.block
    params = [wr.make_params(primes[r["prime_slot"]], b, b, r["seed"]) for r in trace]
    wr.wr_result_free(wr.wr_rank(ctx, handles[0], params[0]))
    torch.cuda.synchronize()
    service = []
    ranks = []
    for h, prm in zip(handles, params):
        t = time.perf_counter()
        res = wr.wr_rank(ctx, h, prm)
        service.append(time.perf_counter() - t)
        ranks.append(wr.wr_result_rank(res))
        wr.wr_result_free(res)
    assert ranks == [r["rank"] for r in trace], "plain ranks differ from the planted ones"
    cap_plain = len(trace) / sum(service)

    def plain_latency(arrivals):
        """One request at a time in arrival order: (latencies in ms, completions/s)."""
        free, lat = 0.0, []
        for a, s in zip(arrivals, service):
            start = max(a, free)
            free = start + s
            lat.append(1e3 * (free - a))
        return lat, len(arrivals) / (free - arrivals[0])

    def served(arrivals):
        srv = wr.wr_server_start(ctx, max_slots=args.slots, hbm_budget=args.hbm_budget, queue_cap=1 << 20)
        t0 = time.perf_counter()
        tickets = []
        for a, h, prm in zip(arrivals, handles[:len(arrivals)], params[:len(arrivals)]):
            d = a - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            tickets.append(wr.wr_submit(srv, h, prm))
        got = []
        for tk in tickets:
            res = wr.wr_wait(srv, tk, 3600 * 1000)
            got.append(wr.wr_result_rank(res))
            wr.wr_result_free(res)
        st = wr.wr_server_stats(srv)
        wr.wr_server_stop(srv)
        assert got == ranks[:len(arrivals)], "served ranks differ from the plain ones"
        return st

    arr = [r["t"] for r in trace]
    out = {}
    for name, scale in [("trace_rate", 1.0), ("rate_0.7x_plain_capacity", None)]:
        if scale is None:
            # the first quarter of the trace, arrivals stretched to 0.7x the
            # plain capacity (the whole trace would take n / (0.7 capacity))
            k = max(20, len(arr) // 4)
            lam = 0.7 * cap_plain
            a = [x * args.rate / lam for x in arr[:k]]
        else:
            lam = args.rate
            a = arr
        st = served(a)
        lat, thr = plain_latency(a)
        out[name] = {"arrival_rate_rps": lam, "requests": len(a),
                     "served": {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                                "throughput_rps": st["throughput_rps"], "max_resident": st["max_resident"]},
                     "plain": dict(_latency_stats(lat), throughput_rps=thr)}
    line = {"metric": METRIC, "workload": "served", "unit": "requests/s", "n_gpus": 1,
            "value": out["trace_rate"]["served"]["throughput_rps"], "higher_is_better": True,
            "dtype": "int64", "data": "synthetic",
            "config": {"requests": len(trace), "rate": args.rate, "rows": [1000, args.rows_hi],
                       "block": [b, b], "slots": args.slots, "hbm_budget": args.hbm_budget,
                       "options": options_config(args),
                       "nnz_total": int(sum(A.nnz for A in mats))},
            "plain_capacity_rps": cap_plain, "results": out, "ranks_equal_planted": True}
    print(json.dumps(line), flush=True)
    for h in handles:
        wr.wr_matrix_free(h)
    wr.wr_destroy(ctx)
    return 0


def run_sigma_only(args):
    """The sigma-basis alone on a random sequence (default: L = 45,002 terms
    of 8 x 8 residues mod 1073741789, the 200,000 x 180,000 workload's shape;
    --sigma-block 32 --sigma-L 118752: the default workload's shape); a
    random sequence has the generic degree profile of a full-rank one.  W + K
    times, for profiler captures and timing of the sigma-basis kernels."""
    import torch
    from paper_0704_2351_gb300 import wr
    p, m, n, L = 1073741789, 8, 8, 45002
    if args.sigma_block:
        m = n = args.sigma_block
        p = 2147483629
    if args.sigma_L:
        L = args.sigma_L
    g = torch.Generator().manual_seed(7)
    S = torch.randint(0, p, (L, m, n), generator=g, dtype=torch.int64).to(torch.int32).cuda()
    q = m + n
    P = torch.empty((L + 2, n, q), dtype=torch.int32, device="cuda")
    deg = torch.empty(q, dtype=torch.int32, device="cuda")
    ctx = wr.wr_create(0)
    wr.wr_set_sigma_chunk(ctx, args.sigma_chunk)
    wr.wr_set_sigma_leaf(ctx, args.sigma_leaf)
    for _ in range(args.warmup):
        wr.wr_sigma_basis_device(ctx, S, L, m, n, p, P, deg, L + 1)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        wr.wr_sigma_basis_device(ctx, S, L, m, n, p, P, deg, L + 1)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t) / max(args.steps, 1)
    # one more run with the phase timers on (their events synchronise the
    # stream, so that run is not the timed one)
    wr.wr_set_profiling(ctx, True)
    wr.wr_sigma_basis_device(ctx, S, L, m, n, p, P, deg, L + 1)
    tm = wr.wr_last_timings(ctx)
    print(json.dumps({"only": "sigma", "L": L, "block": [m, n], "chunk": args.sigma_chunk, "leaf": args.sigma_leaf,
                      "ms_per_sigma_basis": ms,
                      "window_ms": tm["sigma_window_ms"], "local_ms": tm["sigma_local_ms"],
                      "apply_ms": tm["sigma_apply_ms"], "product_ms": tm["sigma_product_ms"]}), flush=True)
    wr.wr_destroy(ctx)
    return 0


def run_gram_only(args):
    """The projection's Gram product alone on rows shaped as the default
    workload's block (N = 1,900,000 rows of 32 residues, L = R = the row,
    p = 2147483629; --gram-width 64: the paired generic block, X half and Y
    half of 32): wr_gram_device with the tensor-core path and with the
    integer path, W + K calls each (for profiler captures of k_gram_tc and
    its time per Gram)."""
    import torch
    from paper_0704_2351_gb300 import wr
    p, m, n, N = 2147483629, 32, 32, args.gram_rows
    g = torch.Generator().manual_seed(1)
    rw = args.gram_width
    yoff = 0 if rw == 32 else 32
    t = torch.randint(0, p, (N, rw), generator=g, dtype=torch.int64).to(torch.int32).cuda()
    w = torch.randint(1, p, (N,), generator=g, dtype=torch.int64).to(torch.int32).cuda()
    G = torch.empty((m, n), dtype=torch.int32, device="cuda")
    ctx = wr.wr_create(0)
    out = {"only": "gram", "rows": N, "block": [m, n], "row_residues": rw}
    for mode, name in [(1, "tensor_cores_ms"), (0, "integer_ms")]:
        wr.wr_set_tensor_projection(ctx, mode)
        for _ in range(args.warmup):
            wr.wr_gram_device(ctx, p, N, m, n, t, rw, yoff, w, G)
        torch.cuda.synchronize()
        tt = time.perf_counter()
        for _ in range(args.steps):
            wr.wr_gram_device(ctx, p, N, m, n, t, rw, yoff, w, G)
        torch.cuda.synchronize()
        out[name] = 1e3 * (time.perf_counter() - tt) / max(args.steps, 1)
    print(json.dumps(out), flush=True)
    wr.wr_destroy(ctx)
    return 0


def run_probe_mma(args):
    """Tensor-core rate on this GPU: one block per SM issuing chains of bf16
    tcgen05 MMAs (M = 128, N = 256, K = 16) on shared-memory tiles, fp32
    accumulators in tensor memory (wr_probe_mma).  Prints dense bf16 TFLOP/s
    and the measured cuBLAS peak beside it.  (The int8 kind of tcgen05.mma
    does not exist for sm_103a: ptxas rejects it, so there is no int8 line.)"""
    from paper_0704_2351_gb300 import wr
    import torch
    ctx = wr.wr_create(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    iters = 20000
    wr.wr_probe_mma(ctx, 100, sms)
    ms = min(wr.wr_probe_mma(ctx, iters, sms) for _ in range(5))
    flops = 2.0 * 128 * 256 * 64 * iters * sms
    peaks = measured_peaks()
    print(json.dumps({"probe": "tcgen05 kind::f16 bf16 -> fp32, M=128 N=256 K=16, one block per SM",
                      "blocks": sms, "iters": iters, "ms": ms, "tflops": flops / ms / 1e9,
                      "cublas_bf16_tflops_measured": peaks.get("bf16_tflops")}), flush=True)
    wr.wr_destroy(ctx)
    return 0


def run_reference(args):
    """The CPU oracle as it stands on the host's cores, on the bench's
    workload.  A step is one of the oracle's exact sparse passes mod p (the
    product of a slice of an eighth of the matrix's rows with the workload's
    32-column block, the slices taken in turn), so that the whole --steps K
    --warmup W run stays within minutes; value = nnz*vec per second as for
    the GPU."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    A, cfg = workload(0, args.matrix)
    import oracle
    from paper_0704_2351_gb300 import synth
    oracle.load()
    st = oracle.Setup(A, cfg["p"], cfg["m"], cfg["n"], cfg["seed"])
    x = np.ascontiguousarray(st.Y if A.cols == st.N else oracle.derive_block(cfg["seed"], oracle.TAG_Y, A.cols,
                                                                            cfg["n"], cfg["p"]))
    slices = []
    k = 8
    for i in range(k):
        r0, r1 = A.rows * i // k, A.rows * (i + 1) // k
        rp = A.rowptr[r0:r1 + 1] - A.rowptr[r0]
        slices.append(synth.CSR(r1 - r0, A.cols, rp, A.colidx[A.rowptr[r0]:A.rowptr[r1]],
                                A.vals[A.rowptr[r0]:A.rowptr[r1]]))
    for i in range(args.warmup):
        oracle.csr_mul(slices[i % k], x, cfg["p"])
    t = time.perf_counter()
    work = 0.0
    for i in range(args.steps):
        S = slices[i % k]
        oracle.csr_mul(S, x, cfg["p"])
        work += float(S.nnz) * cfg["n"]
    el = time.perf_counter() - t
    v = work / el
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": cfg["name"], "projection": args.projection,
                                            "step": "one sparse pass mod p of the CPU "
                                            "oracle: an eighth of the rows times the %d-column block" % cfg["n"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d row slices of one eighth of the matrix, one pass each" % args.steps},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_to_rank_host(wr, ctx, A, params):
    """wr_matrix_load_csr from pinned host arrays + wr_rank + the rank read
    back: the whole job through the public API.  Returns (rank, seconds,
    phase timings, host-to-device bytes)."""
    import ctypes
    import torch
    from paper_0704_2351_gb300.wr import _lib, vp, _check
    h_rp = torch.from_numpy(A.rowptr.astype(np.int64)).pin_memory()
    h_ci = torch.from_numpy(A.colidx.astype(np.int32)).pin_memory()
    h_va = torch.from_numpy(A.vals.astype(np.int32)).pin_memory()
    torch.cuda.synchronize()
    t = time.perf_counter()
    h = vp()
    _check(_lib.wr_matrix_load_csr(vp(ctx), A.rows, A.cols, vp(h_rp.data_ptr()), vp(h_ci.data_ptr()),
                                   vp(h_va.data_ptr()), ctypes.byref(h)))
    res = wr.wr_rank(ctx, h.value, params)
    r = wr.wr_result_rank(res)
    el = time.perf_counter() - t
    tm = wr.wr_last_timings(ctx)
    wr.wr_result_free(res)
    wr.wr_matrix_free(h.value)
    h2d = 8 * (A.rows + 1) + 8 * A.nnz
    return r, el, tm, h2d


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="wr", choices=["wr", "reference"])
    ap.add_argument("--matrix", default="c2", choices=["c2", "c1"],
                    help="c2: the 1.9M x 1.95M block-32 matrix (default); c1: the 200,000 x 180,000 block-8 one")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-rank", action="store_true",
                    help="skip the whole time-to-rank runs (timed steps only)")
    ap.add_argument("--no-generic-time-to-rank", action="store_true",
                    help="skip the second time to rank with the generic projection")
    ap.add_argument("--projection", default="symmetric", choices=["generic", "symmetric"],
                    help="symmetric: X = Y^T (Section 2.3), two terms per application of the width-n block "
                         "(default); generic: independent X, paired with Y in one width-2n block when m = n")
    ap.add_argument("--multi", default="slab", choices=["slab", "independent"],
                    help="N > 1: column slabs of one sequence (default) or an independent matrix per rank")
    ap.add_argument("--only-blackbox", action="store_true",
                    help="only ingest + black-box applications (for profiler captures)")
    ap.add_argument("--only-sigma", action="store_true",
                    help="only the sigma-basis on a random sequence of the workload's shape")
    ap.add_argument("--probe-mma", action="store_true", help="the tensor-core rate probe")
    ap.add_argument("--only-gram", action="store_true", help="only the projection's Gram product (profiler captures)")
    ap.add_argument("--gram-rows", type=int, default=1900000, help="--only-gram: rows of the block")
    ap.add_argument("--gram-width", type=int, default=32, choices=[32, 64],
                    help="--only-gram: residues per row (32: symmetric block; 64: paired generic block)")
    ap.add_argument("--sigma-chunk", type=int, default=0, help="orders per sigma-basis chunk (0: automatic)")
    ap.add_argument("--sigma-leaf", type=int, default=0, help="orders per PM-Basis leaf (0: automatic)")
    ap.add_argument("--sigma-block", type=int, default=0,
                    help="--only-sigma: block m = n (with p = 2147483629; 0: 8 x 8 mod 1073741789)")
    ap.add_argument("--sigma-L", type=int, default=0, help="--only-sigma: sequence length (0: 45,002)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve"],
                    help="single: the one-matrix line (default); batch / serve: batched or "
                         "served against plain time-to-rank")
    ap.add_argument("--pairs", type=int, default=64, help="batch: chain-complex pairs")
    ap.add_argument("--requests", type=int, default=1000, help="serve: requests in the trace")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: trace arrival rate (1/s)")
    ap.add_argument("--rows-hi", type=int, default=500000, help="serve: largest row count")
    ap.add_argument("--block", type=int, default=0, help="batch / serve: block width m = n")
    ap.add_argument("--slots", type=int, default=8, help="batch / serve: concurrent slots")
    ap.add_argument("--no-batch-fusion", action="store_true",
                    help="batch: every job its own sequence loop (no sharing of the matrix passes)")
    ap.add_argument("--hbm-budget", type=int, default=0, help="serve: admission budget in bytes (0: none)")
    ap.add_argument("--chain-reduction", action="store_true",
                    help="remove unit singleton rows/columns at load (rank = pivots + rank of the rest)")
    ap.add_argument("--locality-order", action="store_true",
                    help="renumber rows and columns by decreasing entry count at load (same results)")
    ap.add_argument("--pipeline", type=int, default=1, choices=[0, 1, 2, 3],
                    help="time to rank: sigma-basis after the sequence (0), trailing it with automatic stream "
                         "priorities (1), with its own stream first (2) or with the sequence's first (3)")
    ap.add_argument("--tensor-projection", type=int, default=-1, choices=[-1, 0, 1],
                    help="Gram products on the tensor cores: 1 on, 0 off, -1 automatic (blocks of 16 and more)")
    ap.add_argument("--lane-width", type=int, default=0,
                    help="SpMM residues per lane, + 16 for streaming cache hints (0: tuned per matrix)")
    ap.add_argument("--projection-overlap", action="store_true",
                    help="the Gram projections beside the passes on a side stream (measured slower)")
    ap.add_argument("--slab-bytes", type=int, default=0,
                    help="gathered block bytes per column slab of the SpMM passes (0: no slabs, the default)")
    ap.add_argument("--early-termination", type=int, default=0,
                    help="quiet orders after which the sequence stops (0: all L terms)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.probe_mma:
        return run_probe_mma(args)
    if args.only_gram:
        return run_gram_only(args)
    if args.only_blackbox:
        return run_blackbox_only(args)
    if args.only_sigma:
        return run_sigma_only(args)
    if args.workload == "batch":
        args.block = args.block or 8
        return run_batch(args)
    if args.workload == "serve":
        args.block = args.block or 16
        return run_serve(args)
    return run_single(args)


def run_single(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_0704_2351_gb300 import shard, wr

    slab = world > 1 and args.multi == "slab"
    A, cfg = workload(0 if slab else rank, args.matrix)
    p, m, n = cfg["p"], cfg["m"], cfg["n"]
    sym = args.projection == "symmetric"
    cfg["symmetric"] = sym
    N = min(A.rows, A.cols)
    L_full = -(-N // m) + -(-N // n) + 2
    T = TERMS_PER_STEP
    stream = torch.cuda.Stream()
    ctx = wr.wr_create(local, stream.cuda_stream)
    apply_options(wr, ctx, args)
    proj = wr.WR_PROJ_SYMMETRIC if sym else wr.WR_PROJ_GENERIC
    params = wr.make_params(p, m, n, cfg["seed"], projection=proj)
    d_rp = torch.from_numpy(A.rowptr.astype(np.int64)).to("cuda")
    d_ci = torch.from_numpy(A.colidx.astype(np.int32)).to("cuda")
    d_va = torch.from_numpy(A.vals.astype(np.int32)).to("cuda")
    mat = wr.wr_matrix_load_csr_device(ctx, A.rows, A.cols, A.nnz, d_rp, d_ci, d_va)
    del d_rp, d_ci, d_va
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    if slab:
        c0, w = shard.column_slab(n, rank, world)
        dS = torch.empty((T, m, max(w, 1)), dtype=torch.int32, device="cuda")
        apps = T - 1                      # one term per application of the slab
        width = w
    else:
        dS = torch.empty((T, m, n), dtype=torch.int32, device="cuda")
        paired = (not sym) and m == n
        apps = (T - 1 + 1) // 2 if (paired or sym) else T - 1
        width = 2 * n if paired else n
    work_rank = 2.0 * A.nnz * width * apps  # nnz*vec of this rank per step
    torch.cuda.synchronize()

    def step():
        if slab:
            if w > 0:
                wr.wr_sequence_slab_device(ctx, mat, params, c0, w, dS, T)
        else:
            wr.wr_sequence_device(ctx, mat, params, dS, T)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    wr.wr_set_profiling(ctx, True)
    clk_path = os.path.join(tempfile.gettempdir(), "wr_bench_clocks_%d_%d.csv" % (os.getpid(), rank))
    sampler = start_clock_sampler(clk_path)
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = spmm_ms = spmm_bytes = 0.0
    spmm_launches = 0
    launches0 = wr.wr_last_timings(ctx)["kernel_launches"]
    gathered = None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        if slab:
            with torch.cuda.stream(stream):
                gathered = shard.gather_columns(dS, n, world)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        tm = wr.wr_last_timings(ctx)
        spmm_ms += tm["spmm_ms"]
        spmm_bytes += tm["spmm_bytes"]
        spmm_launches += tm["spmm_launches"]
    torch.cuda.synchronize()
    launches = wr.wr_last_timings(ctx)["kernel_launches"] - launches0
    clocks = stop_clock_sampler(sampler, clk_path, local)
    try:
        os.remove(clk_path)
    except OSError:
        pass
    wr.wr_set_profiling(ctx, False)
    t_max = total_ms
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        wt = torch.tensor([work_rank], device="cuda", dtype=torch.float64)
        dist.all_reduce(wt)
        work_all = float(wt.item())
    else:
        work_all = work_rank
    value = work_all * args.steps / (t_max * 1e-3)

    # roofline of the dominant kernel (k_spmm), from the sampled launches of the timed steps
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    roof = None
    if spmm_launches:
        avg_s = spmm_ms / spmm_launches * 1e-3
        per_launch = spmm_bytes / spmm_launches
        ach = per_launch / avg_s / 1e9
        traffic, tsrc = spmm_traffic(width)
        roof = {"bound": "hbm", "achieved": ach, "peak": peak if peak else 6800.0, "unit": "GB/s",
                "frac": ach / (peak if peak else 6800.0), "traffic": traffic, "traffic_source": tsrc,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak else "fallback",
                "kernel": "k_spmm (both passes of the black box)", "avg_launch_us": avg_s * 1e6,
                "bytes_per_launch": per_launch, "sampled_launches": spmm_launches,
                "bytes_definition": "4 B per stored entry + 4 B x block width per gathered and per written row "
                                    "+ 4 B scale per written row (compulsory bytes of one pass)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if slab else "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": cfg["name"], "block": [m, n], "prime": p, "seq_len": L_full,
                       "projection": args.projection,
                       "step": ("terms S_0..S_%d of the sequence: %d applications of the black box to a block of "
                                "width %d with both SpMM passes and the projections, plus the sequence set-up"
                                % (T - 1, apps, width)) + (
                                    "; this rank's column slab [%d, %d) of Y, slabs all-gathered (NCCL) once per "
                                    "step" % (c0, c0 + w) if slab else ""),
                       "parallelism": ("column slabs of Y over %d GPUs" % world) if slab else (
                           "independent matrix per rank" if world > 1 else "one GPU"),
                       "l2": "inputs larger than L2 (block 1.9M x 256 B); a 256 MB buffer is also written between "
                             "timed steps",
                       "options": options_config(args)},
            "roofline": roof, "gpu_launches": launches, "clocks": clocks}

    # the whole job: time to rank through the public API from pinned host buffers
    if rank == 0 and world == 1 and not args.no_time_to_rank:
        r, el, tm, h2d = _time_to_rank_host(wr, ctx, A, params)
        assert r == A.rank, "rank %d != planted %d" % (r, A.rank)
        L = tm["sequence_terms"] or L_full
        # the passes the sequence ran: two per application, of the block's width
        seq_apps = (L - 1 + 1) // 2 if (sym or (m == n)) else L - 1
        seq_work = 2.0 * A.nnz * (n if sym or m != n else 2 * n) * seq_apps
        line["time_to_rank_ms"] = 1e3 * el
        line["time_to_rank_phases_ms"] = {k: round(tm[k], 1) for k in
                                          ["setup_ms", "sequence_ms", "sigma_ms", "sigma_tail_ms", "readout_ms"]}
        line["rank"] = r
        line["e2e"] = {"value": seq_work / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": 8, "ms_per_step": 1e3 * el,
                       "step": "one whole rank computation: CSR ingest from pinned host memory, all %d terms, "
                               "sigma-basis, readout; value = the sequence's nnz*vec (2 passes x nnz x block "
                               "width per application) / wall time" % L}
        if args.matrix == "c2" and sym and not args.no_generic_time_to_rank:
            # the other projection on the same matrix (the independent X of
            # Section 2.5, paired with Y in one width-64 block)
            prm_g = wr.make_params(p, m, n, cfg["seed"], projection=wr.WR_PROJ_GENERIC)
            rg, elg, tmg, _ = _time_to_rank_host(wr, ctx, A, prm_g)
            assert rg == A.rank, "rank %d != planted %d" % (rg, A.rank)
            line["time_to_rank_generic_ms"] = 1e3 * elg
            line["time_to_rank_generic_phases_ms"] = {k: round(tmg[k], 1) for k in
                                                      ["setup_ms", "sequence_ms", "sigma_ms", "sigma_tail_ms",
                                                       "readout_ms"]}
        if args.matrix == "c2":
            A1, cfg1 = workload(0, "c1")
            prm1 = wr.make_params(cfg1["p"], cfg1["m"], cfg1["n"], cfg1["seed"])
            _time_to_rank_host(wr, ctx, A1, prm1)  # first use of this matrix shape (tuner)
            r1, el1, tm1, _ = _time_to_rank_host(wr, ctx, A1, prm1)
            assert r1 == A1.rank
            line["time_to_rank_config1_ms"] = 1e3 * el1
            line["time_to_rank_config1_workload"] = cfg1["name"]
    elif rank == 0:
        line["e2e"] = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A, cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    wr.wr_matrix_free(mat)
    wr.wr_destroy(ctx)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
