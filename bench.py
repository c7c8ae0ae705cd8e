#!/usr/bin/env python
"""Benchmark of the SP2 hot path on GB300.

Workload (default): the ELLPACK X^2 SpGEMM case -- a 3D tight-binding Hamiltonian
(sites uniform in a periodic cube at 0.1 per cubic Angstrom, hopping -exp(-r/1.5) for
r < 4 Angstrom, onsite ~N(0, 0.5), Morton-ordered, seed 0), N = 262144, FP64 values and
int32 indices, drop tolerance 1e-6; X = one SP2 step of H (built untimed, on the GPU).
One step = one SP2 iteration on X through the C ABI (sp2_step): branch from tr X and
||X||_F^2, the thresholded product with the fused update (X^2 or 2X - X^2), the FP64
traces of the result and the host read of that 56-byte result.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SP2 iters/s & ELLPACK X² SpGEMM HBM GB/s; mixed vs FP64 at ‖ΔD‖_F/√N≤1e-5"
UNIT = "iter/s"
# FP64 FMA units: 2 per SM per clock (1.25 TFLOP/s nominal = 152 SMs x 2 x 2 flop x 2.07 GHz)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=None,
                   help="matrix size (default: 262144 for spgemm, 131072 for sp2, 1048576 for sizing)")
    p.add_argument("--tau", type=float, default=1e-6)
    p.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--workload", default="spgemm",
                   choices=["spgemm", "sp2", "batched", "sizing", "model", "schedule", "rowblock"],
                   help="spgemm: one SP2 iteration at N=262144 (default); sp2: whole purifications, FP64 vs "
                        "mixed at N=131072; batched: 256 clusters in one graph launch vs one by one; sizing: "
                        "heuristic vs structural vs MLP output widths for mixed SP2 at N=1048576; model: the paper's "
                        "model Hamiltonians at N=32000; schedule: stall-rule and precision-schedule variants; "
                        "rowblock: the row-block split of one SP2 run with its ranks as threads on one GPU")
    p.add_argument("--count", type=int, default=256)
    p.add_argument("--path", type=int, default=0,
                   help="SpGEMM first pass: 0 automatic (for symmetric products the cascade of tight, loose "
                        "and full-row passes), 1/2/4 column blocks with 1/2/4 warps per row, 3 two-step, "
                        "7/8 compact forms of 2/3, 9 row tiles, 10-12 hash, -1 tuned")
    p.add_argument("--full-rows", dest="symmetric", action="store_false",
                   help="SP2 steps compute full product rows instead of the upper triangle of the "
                        "symmetric product mirrored (the default)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-f32-view", action="store_true",
                   help="skip the FP32 step of the same product (the first pass of mixed precision)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-literal-m", action="store_true",
                   help="skip the product of X truncated to the 128 largest entries per row")
    p.add_argument("--no-tts", action="store_true",
                   help="skip the time-to-solution block (whole SP2 runs of the C1, C3, C4 and C5 workloads)")
    return p.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "fallback": True}


def workload_config(a, extra=None):
    c = {"workload": "SP2 iteration on ELLPACK X^2 SpGEMM: 3D tight-binding N=%d, %s values, int32 indices, "
                     "tau=%g, X = one SP2 step of H" % (a.n, a.dtype.upper(), a.tau),
         "n": a.n, "tau": a.tau, "seed": a.seed,
         "hamiltonian": "periodic cube, density 0.1/A^3, -exp(-r/1.5) for r<4 A, onsite N(0,0.5), Morton order"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------ host-side helpers
def fma_count(idx, nnz):
    """sum over rows i of sum_{k in row i} nnz[k] (products of X*X)."""
    n, w = idx.shape
    mask = np.arange(w)[None, :] < nnz[:, None]
    return int(np.where(mask, nnz[idx], 0).sum())


def fma_count_upper(idx, nnz):
    """Products of the upper triangle of X*X: sum over the entries (i, k) of X of the
    number of entries of row k with a column >= i (what the symmetric product computes)."""
    n, w = idx.shape
    mask = np.arange(w)[None, :] < nnz[:, None]
    rows = np.repeat(np.arange(n, dtype=np.int64), nnz)
    cols = idx[mask].astype(np.int64)
    keys = rows * n + cols  # sorted: rows ascending, columns ascending within a row
    start = np.concatenate([[0], np.cumsum(nnz, dtype=np.int64)])
    pos = np.searchsorted(keys, cols * n + rows)  # first entry of row k = cols with column >= i = rows
    return int((start[cols + 1] - pos).sum())


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id, enabled=True):
        self.proc = None
        self.dev_id = dev_id
        if not enabled:
            return
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(dev_id)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clocks not sampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out = self.proc.communicate(timeout=5)[0]
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_traffic(dtype):
    """Per-launch DRAM bytes of the SpGEMM kernel from the committed ncu summary, or None
    if the kernel's source file changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "spgemm_traffic.json")
    try:
        rec = json.load(open(path))
        ent = rec.get(dtype)
        if not ent:
            return None
        src = os.path.join(ROOT, "paper_2102_08505_gb300", "csrc", ent.get("source", "spgemm.cu"))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if ent.get("source_sha256", ent.get("spgemm_cu_sha256")) == sha:
            return ent.get("dram_bytes_per_launch_full_size")
    except Exception:
        pass
    return None


# ------------------------------------------------------------------ oracle timing (CPU)
def oracle_prepare(a, threads):
    """Oracle-side input of the timed iteration: X = one SP2 step of H, built by the oracle."""
    from oracle import oracle as O
    from paper_2102_08505_gb300 import inputs as I
    O.set_threads(threads)
    H = O.Ell(*I.tight_binding(a.n, seed=a.seed))
    lo, hi = O.gershgorin(H)
    X0 = O.x0(H, lo, hi, a.tau)
    nocc = a.n / 2

    def traces(X):
        live = np.arange(X.w)[None, :] < X.nnz[:, None]
        return O.trace(X), float(np.where(live, X.val, 0.0).__pow__(2).sum())

    t0, t02 = traces(X0)
    up = abs(2 * t0 - t02 - nocc) < abs(t02 - nocc)
    X1 = O.spgemm(X0, X0, X0 if up else None, -1.0 if up else 1.0, 2.0 if up else 0.0, a.tau)
    t1, t12 = traces(X1)
    up = abs(2 * t1 - t12 - nocc) < abs(t12 - nocc)
    O.set_threads(1)
    return X1, up


def oracle_iteration_rate(a, X1, up, sample_rows, threads, reps=1):
    """Times the oracle's SP2 iteration (product with the update, then the trace) on a
    row sample of X; returns (iterations/s scaled to all rows, median s, rows, times)."""
    from oracle import oracle as O
    O.set_threads(threads)
    rng = np.random.default_rng(1234)
    rows = np.sort(rng.choice(a.n, size=min(sample_rows, a.n), replace=False)).astype(np.int32)
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        out = O.spgemm(X1, X1, X1 if up else None, -1.0 if up else 1.0, 2.0 if up else 0.0, a.tau, rows=rows)
        _ = O.trace(out)
        times.append(time.perf_counter() - t)
    O.set_threads(1)
    sec = float(np.median(times))
    return 1.0 / (sec * a.n / len(rows)), sec, len(rows), times


def cpu_baseline(a):
    from oracle import oracle as O
    threads = O.max_threads()
    X1, up = oracle_prepare(a, threads)
    # bounded sample: about 10 s of CPU work
    _, sec0, rows0, _ = oracle_iteration_rate(a, X1, up, 4096, threads)
    target = int(min(a.n, max(4096, rows0 * 10.0 / max(sec0, 1e-3))))
    rate, sec, rows, _ = oracle_iteration_rate(a, X1, up, target, threads)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of %d product rows of one SP2 iteration (oracle SpGEMM + update + trace, %.1f s on %d "
                      "threads), scaled to the whole iteration" % (rows, a.n, sec, threads)}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    threads = O.max_threads()
    X1, up = oracle_prepare(a, threads)
    # each step: one whole SP2 iteration of the oracle (every product row, the update and
    # the trace), about 1.7 s on 16 Grace cores at N = 262144
    sample = a.n
    oracle_iteration_rate(a, X1, up, sample, threads, reps=max(1, a.warmup))
    rate, sec, rows, times = oracle_iteration_rate(a, X1, up, sample, threads, reps=max(1, a.steps))
    per_step_ms = 1000.0 * float(np.mean(times)) * a.n / rows
    rate = 1000.0 / per_step_ms
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": per_step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(a),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d of %d product rows per step: whole SP2 iterations (oracle SpGEMM + "
                                   "update + trace), %d timed" % (rows, a.n, len(times))},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def spgemm_kernel_name(a):
    """The first-pass SpGEMM kernel that the chosen path launches."""
    p = a.path
    if p == 0:
        p = (7 if a.dtype == "f64" else 8) if a.symmetric else (4 if a.dtype == "f64" else 3)
    casc = " then the loose and full-row passes over the rows passed on" if a.path == 0 and a.symmetric else ""
    if p in (1, 2, 4, 7):
        w = 2 if p == 7 else p
        return "spgemm_block_kernel (%d warp%s per row%s)%s" % (w, "s" if w > 1 else "", ", compact" if p == 7 else "",
                                                              casc)
    if p == 8:
        return "spgemm_super_kernel (one warp per row, two k steps per pass, compact)" + casc
    if p == 9:
        return "spgemm_tile_kernel (8-row tiles sharing one column index, one warp per row)"
    if p == -1:
        return "tuned first pass"
    if p == 3:
        return "spgemm_super_kernel (one warp per row, two k steps per pass)"
    return "spgemm_hash_kernel (2^%d slots per warp)" % p


# ------------------------------------------------------------------ our arm
def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_2102_08505_gb300 import shard
    rank, local, world = shard.rank_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2102_08505_gb300 import inputs as I
    from paper_2102_08505_gb300 import sp2ell as S

    DT = S.SP2_F64 if a.dtype == "f64" else S.SP2_F32
    esz = 8 if a.dtype == "f64" else 4
    stream = torch.cuda.current_stream()
    nocc = a.n / 2

    # ---------------- setup (untimed): H -> X0 -> X (one SP2 step), all on the GPU
    idx, val, nnz = I.tight_binding(a.n, seed=a.seed + rank)
    H = S.Ellpack.from_numpy(idx, val, nnz)
    X0 = S.Ellpack.empty(a.n, H.width + 32)
    S.sp2_x0(H, X0, a.tau)
    if DT == S.SP2_F32:
        X0f = S.Ellpack.empty(a.n, X0.width, S.SP2_F32)
        S.ellpack_copy(X0, X0f)
        X0 = X0f
    w1 = 4 * X0.width
    while True:
        X1 = S.Ellpack.empty(a.n, w1, DT)
        rc, info = S.sp2_step(X0, X1, nocc, a.tau, raise_on_overflow=False, symmetric=a.symmetric)
        if rc == 0:
            break
        w1 = ((info.required_width + 31) // 32) * 32
    w1 = ((int(info.max_row_nnz) + 31) // 32) * 32
    Xs = S.Ellpack.empty(a.n, w1, DT)
    S.ellpack_copy(X1, Xs)
    X1 = Xs
    traces = (info.trXn, info.trXn2)
    del X0, H
    X2 = S.Ellpack.empty(a.n, 32, DT)
    rc, info = S.sp2_step(X1, X2, nocc, a.tau, traces=traces, raise_on_overflow=False, symmetric=a.symmetric)
    w2 = ((info.required_width + 31) // 32) * 32
    X2 = S.Ellpack.empty(a.n, w2, DT)
    info = S.sp2_step(X1, X2, nocc, a.tau, traces=traces, spgemm_path=a.path, symmetric=a.symmetric)
    torch.cuda.synchronize()
    h_idx, h_val, h_nnz = [t.cpu().numpy() for t in (X1.idx, X1.val, X1.nnz)]
    nnz_in = int(h_nnz.sum())
    fmas = fma_count(h_idx, h_nnz)
    # products executed: the upper triangle only when the symmetric product is used
    fmas_exec = fma_count_upper(h_idx, h_nnz) if a.symmetric else fmas
    nnz_out = int(info.nnz_total)
    alg_bytes = (4 + esz) * (2 * nnz_in + nnz_out) + 12 * a.n  # A, B, C read/written once + 3 nnz arrays
    in_bytes = X1.idx.numel() * 4 + X1.val.numel() * esz + a.n * 4

    # ---------------- device-timed steps
    for _ in range(a.warmup):
        S.sp2_step(X1, X2, nocc, a.tau, traces=traces, spgemm_path=a.path, symmetric=a.symmetric)
    torch.cuda.synchronize()
    clocks = Clocks(local, enabled=not a.no_clocks)
    shard.barrier()
    torch.cuda.synchronize()
    S.sp2_profile_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        S.sp2_step(X1, X2, nocc, a.tau, traces=traces, spgemm_path=a.path, symmetric=a.symmetric)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = S.sp2_profile_stop()
    shard.barrier()
    clk = clocks.stop()
    ms = shard.max_over_ranks(e0.elapsed_time(e1) / a.steps, dev)
    value = world * 1000.0 / ms

    # the first pass of one product: the pass over every row plus, for the automatic path of
    # a symmetric product, the later passes of its cascade over the rows passed on
    cnt, tot = prof["spgemm"]
    ccnt, ctot = prof["cascade"]
    k_ms = (tot + ctot) / max(a.steps, 1)
    tflops = 2.0 * fmas_exec / (k_ms * 1e-3) / 1e12
    eff_tflops = 2.0 * fmas / (k_ms * 1e-3) / 1e12
    gbs = alg_bytes / (k_ms * 1e-3) / 1e9
    pk = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    derived_peak = FP64_PEAK_TFLOPS if a.dtype == "f64" else FP32_PEAK_TFLOPS
    # the FMA rate of this GPU measured now (dependent-free FMA chains, 8 CTAs per SM)
    alu_peak = S.sp2_fma_peak(DT, 5)
    traffic = kernel_traffic(a.dtype)
    # the bound is the roof the kernel's arithmetic intensity meets first: FP64 products hit
    # the FP64 FMA rate long before HBM; FP32 products would reach HBM first
    alu_view = {"achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak,
                "peak_source": "of measured: sp2_fma_peak, %s FMA chains timed in this run (derived %.4g)" % (
                    "DFMA" if a.dtype == "f64" else "FFMA", derived_peak),
                "flops_per_launch": 2.0 * fmas_exec,
                "flops": "2 x the products executed" + (" (upper triangle of the symmetric product)" if a.symmetric else "")}
    hbm_view = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "peak_source": "of measured" if "fallback" not in pk else "of fallback",
                "algorithmic_bytes_per_launch": alg_bytes}
    alu_bound = (2.0 * fmas_exec / (alu_peak * 1e12)) > (alg_bytes / (hbm_peak * 1e9))
    main, other = (alu_view, hbm_view) if alu_bound else (hbm_view, alu_view)
    roofline = {"bound": "alu" if alu_bound else "hbm", **{k: main[k] for k in ("achieved", "peak", "unit", "frac")},
                "traffic": traffic, "peak_source": main["peak_source"],
                "kernel": spgemm_kernel_name(a), "kernel_ms": k_ms, "launches_timed": cnt + ccnt,
                "kernel_ms_split": {"every_row_pass": tot / max(a.steps, 1), "cascade_passes": ctot / max(a.steps, 1),
                                    "cascade_launches_per_step": ccnt / max(a.steps, 1)},
                ("hbm_view" if alu_bound else "alu_view"): other,
                **({"alu_detail": alu_view} if alu_bound else {"hbm_detail": hbm_view})}

    # ---------------- end to end through the C ABI with host buffers
    # Every step uploads its input from pinned host memory, runs the SP2 step and downloads
    # the result.  Two buffer sets on two streams overlap step t+1's upload and step t-1's
    # download with step t's product (the copy engines run beside the SMs).
    e2e = None
    if not a.no_e2e:
        import torch as _t
        hi = _t.from_numpy(h_idx).pin_memory()
        hv = _t.from_numpy(h_val).pin_memory()
        hn = _t.from_numpy(h_nnz).pin_memory()
        vdt = _t.float64 if DT == S.SP2_F64 else _t.float32
        outs = [(_t.empty((a.n, w2), dtype=_t.int32).pin_memory(), _t.empty((a.n, w2), dtype=vdt).pin_memory(),
                 _t.empty(a.n, dtype=_t.int32).pin_memory()) for _ in range(2)]
        Xins = [S.Ellpack.empty(a.n, w1, DT) for _ in range(2)]
        Xouts = [X2, S.Ellpack.empty(a.n, w2, DT)]
        streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]  # not the legacy stream

        def upload(t):
            b = t % 2
            S._check(S.lib.ellpack_upload(S._d(Xins[b]), hi.data_ptr(), hv.data_ptr(), hn.data_ptr(),
                                          S._stream(streams[b])))

        def step_and_download(t):
            b = t % 2
            S.sp2_step(Xins[b], Xouts[b], nocc, a.tau, traces=traces, spgemm_path=a.path, symmetric=a.symmetric,
                       stream=streams[b])
            oi, ov, on = outs[b]
            S._check(S.lib.ellpack_download_async(S._d(Xouts[b]), oi.data_ptr(), ov.data_ptr(), on.data_ptr(),
                                                  S._stream(streams[b])))

        def run(k):
            upload(0)
            for t in range(k):
                if t + 1 < k:
                    upload(t + 1)
                step_and_download(t)

        run(max(2, a.warmup))
        ksteps = max(2, min(a.steps, 20))
        shard.barrier()
        torch.cuda.synchronize()
        e0.record(streams[0])
        run(ksteps)
        tail = torch.cuda.Event()
        tail.record(streams[1])
        streams[0].wait_event(tail)
        e1.record(streams[0])
        torch.cuda.synchronize()
        ems = shard.max_over_ranks(e0.elapsed_time(e1) / ksteps, dev)
        out_bytes = a.n * w2 * (4 + esz) + 4 * a.n
        e2e = {"value": world * 1000.0 / ems, "unit": UNIT, "h2d_bytes_per_step": in_bytes,
               "d2h_bytes_per_step": out_bytes, "ms_per_step": ems, "steps": ksteps,
               "api": "ellpack_upload + sp2_step + ellpack_download_async (pinned host buffers, two streams: "
                      "step t+1's upload and step t-1's download overlap step t)"}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a)
    tts = None
    if rank == 0 and world == 1 and not a.no_tts and a.dtype == "f64":
        tts = time_to_solution(a, local)
    literal_m = None
    if rank == 0 and world == 1 and not a.no_literal_m:
        literal_m = literal_m_product(a, S, X1, DT, esz, nocc, stream)
    f32 = None
    if rank == 0 and world == 1 and a.dtype == "f64" and not a.no_f32_view:
        f32 = f32_step(a, S, X1, nocc, stream, traces, fmas_exec, nnz_in, hbm_peak)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": a.dtype, "data": "synthetic",
            "config": workload_config(a, {
                "width_in": w1, "width_out": w2, "nnz_per_row_in": nnz_in / a.n, "nnz_per_row_out": nnz_out / a.n,
                "fma_per_row": fmas / a.n, "fma_per_row_executed": fmas_exec / a.n,
                "symmetric_product": "upper triangle computed and mirrored" if a.symmetric else "full rows",
                "branch": "2X-X^2" if info.branch == 2 else "X^2",
                "l2": "no flush: inputs %.2f GB > 129 MB L2" % (in_bytes / 1e9),
                "parallelism": "replicas" if world > 1 else "single GPU"}),
            "spgemm_path": a.path,
            "spgemm_gflops": tflops * 1e3, "spgemm_effective_gflops": eff_tflops * 1e3, "spgemm_hbm_gbs": gbs,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(prof["launches"]),
            "kernels_timed": {k: prof[k] for k in ("spgemm", "cascade", "large_rows", "reduce", "other", "symmetry")},
            "clocks": clk,
        }
        if tts is not None:
            line["time_to_solution"] = tts
        if literal_m is not None:
            line["literal_m128"] = literal_m
        if f32 is not None:
            line["f32_step"] = f32
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def literal_m_product(a, S, X1, DT, esz, nocc, stream, width=128):
    """The same SP2 step with X cut to the configuration's width as written: each row keeps
    its `width` largest |x_ij| (then in column order).  The cut X is no longer symmetric,
    so the product runs on full rows.  Timed with CUDA events after a warm-up."""
    import torch
    idx, val, nnz = X1.idx, X1.val.double(), X1.nnz
    live = torch.arange(idx.shape[1], device=idx.device)[None, :] < nnz[:, None]
    mag = torch.where(live, val.abs(), torch.full_like(val, -1.0))
    top = torch.topk(mag, k=min(width, idx.shape[1]), dim=1).indices
    ci = torch.gather(idx, 1, top)
    cv = torch.gather(val, 1, top)
    keep = torch.gather(live, 1, top)
    ci = torch.where(keep, ci, torch.full_like(ci, 2 ** 30))
    order = torch.argsort(ci, dim=1)
    ci, cv = torch.gather(ci, 1, order), torch.gather(cv, 1, order)
    cn = keep.sum(dim=1).to(torch.int32)
    ci = torch.where(ci == 2 ** 30, torch.zeros_like(ci), ci).to(torch.int32).contiguous()
    Xm = S.Ellpack(ci, cv.to(X1.val.dtype).contiguous(), cn.contiguous())
    rows_cut = int((nnz > width).sum().item())
    probe = S.Ellpack.empty(a.n, 32, DT)
    rc, info = S.sp2_step(Xm, probe, nocc, a.tau, raise_on_overflow=False, symmetric=False)
    Y = S.Ellpack.empty(a.n, ((info.required_width + 31) // 32) * 32, DT)
    for _ in range(max(3, a.warmup)):
        S.sp2_step(Xm, Y, nocc, a.tau, symmetric=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(a.steps, 10))
    e0.record(stream)
    for _ in range(reps):
        info = S.sp2_step(Xm, Y, nocc, a.tau, symmetric=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    h_idx, h_nnz = ci.cpu().numpy(), cn.cpu().numpy()
    fmas = fma_count(h_idx, h_nnz)
    return {"ms_per_step": ms, "iters_per_s": 1000.0 / ms, "rows_cut": rows_cut,
            "nnz_per_row_in": float(h_nnz.mean()), "nnz_per_row_out": float(info.nnz_total) / a.n,
            "fma_per_row": fmas / a.n, "gflops": 2.0 * fmas / (ms * 1e-3) / 1e9,
            "product": "full rows (the cut X is not symmetric)"}


def f32_step(a, S, X1, nocc, stream, traces, fmas_exec, nnz_in, hbm_peak):
    """The same SP2 step with X rounded to FP32 (the products of mixed precision): step time
    and the first pass (every-row pass plus cascade passes, CUDA events of the library's
    profiler) against the measured FFMA rate and the HBM copy rate."""
    import torch
    Xf = S.Ellpack.empty(a.n, X1.width, S.SP2_F32)
    S.ellpack_copy(X1, Xf)
    probe = S.Ellpack.empty(a.n, 32, S.SP2_F32)
    rc, info = S.sp2_step(Xf, probe, nocc, a.tau, traces=traces, raise_on_overflow=False, symmetric=a.symmetric)
    Y = S.Ellpack.empty(a.n, ((info.required_width + 31) // 32) * 32, S.SP2_F32)
    for _ in range(max(3, a.warmup)):
        S.sp2_step(Xf, Y, nocc, a.tau, traces=traces, symmetric=a.symmetric)
    torch.cuda.synchronize()
    reps = max(3, min(a.steps, 20))
    S.sp2_profile_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        info = S.sp2_step(Xf, Y, nocc, a.tau, traces=traces, symmetric=a.symmetric)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = S.sp2_profile_stop()
    ms = e0.elapsed_time(e1) / reps
    k_ms = (prof["spgemm"][1] + prof["cascade"][1]) / reps
    bytes_ = 8 * (2 * nnz_in + int(info.nnz_total)) + 12 * a.n  # int32 index + FP32 value per entry
    peak = S.sp2_fma_peak(S.SP2_F32, 5)
    tfl = 2.0 * fmas_exec / (k_ms * 1e-3) / 1e12
    gbs = bytes_ / (k_ms * 1e-3) / 1e9
    return {"ms_per_step": ms, "iters_per_s": 1000.0 / ms, "first_pass_ms": k_ms,
            "alu_view": {"achieved": tfl, "peak": peak, "unit": "TFLOP/s", "frac": tfl / peak,
                         "peak_source": "of measured: sp2_fma_peak, FFMA chains timed in this run"},
            "hbm_view": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                         "algorithmic_bytes_per_launch": bytes_, "peak_source": "of measured"},
            "product": "X rounded to FP32, symmetric" if a.symmetric else "X rounded to FP32, full rows"}


def diff_fro(S, D1, D2):
    """||D1 - D2||_F through the library (ellpack_add on a copy, then the norm)."""
    A = D1.to_torch()
    w = A.width + D2.width
    Aw = S.Ellpack.empty(A.n, w, S.SP2_F64)
    S.ellpack_copy(A, Aw)
    S.ellpack_add(Aw, D2.to_torch(), 1.0, -1.0, 0.0)
    return float(np.sqrt(S.ellpack_frobenius2(Aw)))


# ------------------------------------------------------------------ time to solution
def _median_runs(fn, reps, warm=1):
    """Runs fn() warm times untimed, then reps times; returns (median seconds, last result)."""
    import torch
    out = None
    for _ in range(warm):
        out = fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    return float(np.median(times)), out, times


def time_to_solution(a, dev_id, reps=3):
    """Whole SP2 purifications on one GPU, each entry the median of `reps` runs after a
    warm-up, with the SM clocks sampled around it and the distance of every result to the
    FP64 GPU run of the same input (||D - D_FP64||_F / sqrt(N), same tau):
      C1: banded N = 1024, band 16 (the gapped variant: A/B onsite splitting 10), FP64,
          iterations per second with the whole loop in one cooperative launch (sp2_purify),
          host-stepped (small_path = 0) and as one captured graph (sp2_purify_batched of one
          matrix); the literal gapless configuration beside it;
      C3: gapped 3D tight-binding N = 131072, FP64 against mixed precision;
      C4: 256 gapped open clusters, N log-uniform in [512, 8192]: one graph launch in mixed
          precision and in FP64, against FP64 purified one by one;
      C5: gapped 3D tight-binding N = 1048576, input width 128: mixed precision with the
          row-length MLP (trained here on about 50k rows of SP2 products of 4096 .. 16384
          site Hamiltonians), mixed precision with the heuristic widths, and plain FP64."""
    import torch
    from paper_2102_08505_gb300 import inputs as I
    from paper_2102_08505_gb300 import learned
    from paper_2102_08505_gb300 import sp2ell as S
    out = {}
    tol = 1e-10

    def clocked(fn):
        c = Clocks(dev_id, enabled=not a.no_clocks)
        r = fn()
        r["clocks"] = c.stop()
        return r

    def dD(Dx, Dy, n):
        return diff_fro(S, Dx, Dy) / np.sqrt(n)

    # C1 ---------------------------------------------------------------------------
    def c1():
        r = {}
        n, tau = 1024, 1e-5
        Hg = S.Ellpack.from_numpy(*I.banded(n, band=16, seed=1, delta=10.0, width=64))
        opt = S.sp2_options_default(tau=tau)  # n <= 2048: the whole loop in one cooperative launch
        t_one, (D, st), _ = _median_runs(lambda: S.sp2_purify(Hg, n / 2, tol, opt), reps * 3)
        opth = S.sp2_options_default(tau=tau, small_path=0)
        t_host, (Dh, sh), _ = _median_runs(lambda: S.sp2_purify(Hg, n / 2, tol, opth), reps * 3)
        optg = S.sp2_options_default(tau=tau, graph=1)
        t_graph, (Dg, sg), _ = _median_runs(lambda: S.sp2_purify_batched([Hg], [n // 2], tol, optg), reps * 3)
        r["gapped_delta10"] = {
            "iterations": st["iterations"], "status": st["status"], "final_err": float(st["err"][-1]),
            "one_launch": {"time_s": t_one, "iters_per_s": st["iterations"] / t_one,
                           "api": "sp2_purify (the loop as one cooperative kernel)"},
            "host_stepped": {"time_s": t_host, "iters_per_s": sh["iterations"] / t_host,
                             "iterations": sh["iterations"], "dD_vs_one_launch": dD(Dh, D, n)},
            "graph": {"time_s": t_graph, "iters_per_s": sg[0]["iterations"] / t_graph,
                      "iterations": sg[0]["iterations"], "dD_vs_one_launch": dD(Dg[0], D, n)},
            "max_row_nnz": int(max(st["max_row_nnz"]))}
        H = S.Ellpack.from_numpy(*I.banded(n, band=16, seed=1, width=64))
        t_lit, (Dl, sl), _ = _median_runs(lambda: S.sp2_purify(H, n / 2, tol, opt, allow_notconv=True), reps)
        r["literal_gapless"] = {"time_s": t_lit, "iterations": sl["iterations"], "status": sl["status"],
                                "final_err": float(sl["err"][-1]), "max_row_nnz": int(max(sl["max_row_nnz"])),
                                "iters_per_s": sl["iterations"] / t_lit}
        r["workload"] = "banded N=1024 band 16, nocc 512, tau 1e-5, tol 1e-10, input width 64"
        return r
    out["C1"] = clocked(c1)

    # C3 ---------------------------------------------------------------------------
    def c3():
        n, tau = 131072, 1e-5
        H = S.Ellpack.from_numpy(*I.tight_binding(n, seed=0, delta=10.0))
        r, Ds = {}, {}
        for name, prec in (("f64", S.SP2_PREC_F64), ("mixed", S.SP2_PREC_MIXED)):
            opt = S.sp2_options_default(tau=tau, precision=prec)
            t, (D, st), times = _median_runs(lambda: S.sp2_purify(H, n / 2, tol, opt), reps)
            Ds[name] = D
            r[name] = {"time_s": t, "times_s": times, "iterations": st["iterations"],
                       "fp32_iterations": st["fp32_iterations"], "status": st["status"],
                       "iters_per_s": st["iterations"] / t, "final_err": float(st["err"][-1])}
        r["mixed"]["dD_vs_f64"] = dD(Ds["mixed"], Ds["f64"], n)
        r["speedup_mixed_vs_f64"] = r["f64"]["time_s"] / r["mixed"]["time_s"]
        r["workload"] = "3D tight-binding gapped (delta 10) N=131072, nocc N/2, tau 1e-5, tol 1e-10"
        return r
    out["C3"] = clocked(c3)

    # C4 ---------------------------------------------------------------------------
    def c4():
        tau = 1e-5
        sizes = I.cluster_sizes(256, 512, 8192, seed=0)
        Hs = [S.Ellpack.from_numpy(*I.tight_binding(int(m), seed=k, delta=10.0, periodic=False))
              for k, m in enumerate(sizes)]
        noccs = [(h.n + 1) // 2 for h in Hs]  # the A sublattice's states: the gap stays at nocc
        r, Dsets = {}, {}
        for name, prec in (("batched_mixed_graph", S.SP2_PREC_MIXED), ("batched_f64_graph", S.SP2_PREC_F64)):
            opt = S.sp2_options_default(tau=tau, precision=prec, graph=1)
            t, (Ds, sts), times = _median_runs(lambda: S.sp2_purify_batched(Hs, noccs, tol, opt), reps)
            Dsets[name] = Ds
            r[name] = {"time_s": t, "times_s": times, "iterations_total": int(sum(x["iterations"] for x in sts)),
                       "max_iterations": int(max(x["iterations"] for x in sts))}
        opt = S.sp2_options_default(tau=tau, precision=S.SP2_PREC_F64)

        def one_by_one():
            return [S.sp2_purify(H, m, tol, opt) for H, m in zip(Hs, noccs)]
        t, res1, times = _median_runs(one_by_one, reps)
        r["one_by_one_f64"] = {"time_s": t, "times_s": times, "iterations_total": int(sum(x[1]["iterations"] for x in res1))}
        ref = [x[0] for x in res1]
        for name in Dsets:
            d = [dD(Dx, Dy, h.n) for Dx, Dy, h in zip(Dsets[name], ref, Hs)]
            r[name]["dD_vs_one_by_one_f64_max"] = float(max(d))
        r["speedup_batched_mixed_vs_one_by_one_f64"] = t / r["batched_mixed_graph"]["time_s"]
        r["speedup_batched_mixed_vs_batched_f64"] = r["batched_f64_graph"]["time_s"] / r["batched_mixed_graph"]["time_s"]
        r["workload"] = "256 gapped open 3D clusters, N log-uniform [512, 8192], sum N = %d, tau 1e-5" % int(sizes.sum())
        return r
    out["C4"] = clocked(c4)

    # C5 ---------------------------------------------------------------------------
    def c5():
        n, tau = 1048576, 1e-5
        t0 = time.perf_counter()
        feat, counts = learned.default_training_set(seed=100, rows=50000, tau=tau, dtype=S.SP2_F32)
        pred, loss = learned.train(feat, counts, seed=0, steps=1500, batch=2048, lr=2e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        idx, val, nnz = I.tight_binding(n, seed=0, delta=10.0, width=128)
        H = S.Ellpack.from_numpy(idx, val, nnz)
        r, Ds = {"training": {"rows": int(counts.shape[0]), "collect_and_train_s": t_train, "final_batch_loss": loss}}, {}
        for name, prec, sizing in (("plain_f64", S.SP2_PREC_F64, 0), ("mixed_heuristic", S.SP2_PREC_MIXED, 0),
                                   ("mixed_mlp", S.SP2_PREC_MIXED, 2)):
            kw = dict(tau=tau, precision=prec, sizing=sizing)
            if sizing == 2:
                kw["predictor"] = pred
            opt = S.sp2_options_default(**kw)
            t, (D, st), times = _median_runs(lambda: S.sp2_purify(H, n / 2, tol, opt), reps)
            Ds[name] = D
            r[name] = {"time_s": t, "times_s": times, "iterations": st["iterations"],
                       "fp32_iterations": st["fp32_iterations"], "status": st["status"],
                       "width_max": st["width_max"], "regrows": st["regrows"],
                       "peak_product_bytes": int(st["width_max"]) * n * (12 if prec == S.SP2_PREC_F64 else 8)}
            if sizing == 2:
                r[name].update({"pred_log_mae": st["pred_log_mae"], "pred_under_frac": st["pred_under_frac"]})
            del D
        for name in ("mixed_heuristic", "mixed_mlp"):
            r[name]["dD_vs_f64"] = dD(Ds[name], Ds["plain_f64"], n)
        r["dD_mlp_vs_heuristic"] = dD(Ds["mixed_mlp"], Ds["mixed_heuristic"], n)
        r["speedup_mixed_mlp_vs_plain_f64"] = r["plain_f64"]["time_s"] / r["mixed_mlp"]["time_s"]
        r["speedup_mixed_mlp_vs_mixed_heuristic"] = r["mixed_heuristic"]["time_s"] / r["mixed_mlp"]["time_s"]
        r["workload"] = "3D tight-binding gapped (delta 10) N=1048576, input width 128, tau 1e-5, tol 1e-10"
        return r
    out["C5"] = clocked(c5)
    tgt = out["C5"]
    out["target_met"] = bool(tgt["mixed_mlp"]["dD_vs_f64"] <= 1e-5 and tgt["speedup_mixed_mlp_vs_plain_f64"] > 1.0 and
                             out["C3"]["mixed"]["dD_vs_f64"] <= 1e-5 and out["C3"]["speedup_mixed_vs_f64"] > 1.0 and
                             out["C4"]["batched_mixed_graph"]["dD_vs_one_by_one_f64_max"] <= 1e-5 and
                             out["C4"]["speedup_batched_mixed_vs_one_by_one_f64"] > 1.0)
    return out


def run_rowblock(a):
    """The row-block split of one SP2 run (shard.row_block_sp2) with its ranks run as threads
    of one process on one GPU (exchanges through host memory): the same 3D gapped
    Hamiltonian as the sp2 workload, against the whole run (sp2_purify, FP64).  It shows
    what the split itself costs (halo requests, exchanges, block products); it is not a
    multi-GPU scaling figure."""
    import threading
    import torch
    from paper_2102_08505_gb300 import inputs as I
    from paper_2102_08505_gb300 import shard
    from paper_2102_08505_gb300 import sp2ell as S
    n = a.n
    tau = a.tau if a.tau != 1e-6 else 1e-5
    idx, val, nnz = I.tight_binding(n, seed=a.seed, delta=10.0)
    H = S.Ellpack.from_numpy(idx, val, nnz)
    t_whole, (Dw, sw), _ = _median_runs(lambda: S.sp2_purify(H, n / 2, 1e-10, S.sp2_options_default(tau=tau)), 3)
    out = {"whole": {"time_s": t_whole, "iterations": sw["iterations"]}}
    for world in (2, 4):
        bounds = shard.block_bounds(n, world)
        blocks = [S.Ellpack.from_numpy(idx[bounds[r]:bounds[r + 1]], val[bounds[r]:bounds[r + 1]],
                                       nnz[bounds[r]:bounds[r + 1]]) for r in range(world)]

        def run_once():
            hub = shard.LocalComm.Hub(world)
            res, errs = {}, []

            def rank(r):
                try:
                    torch.cuda.set_device(0)
                    res[r] = shard.row_block_sp2(shard.LocalComm(hub, r), bounds, blocks[r], n / 2, 1e-10, tau,
                                                 shard.GPUBlockOps())
                except Exception as e:
                    errs.append(e)
            ts = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
            for t in ts:
                t.start()
            for t in ts:
                t.join()
            if errs:
                raise errs[0]
            return res
        t, res, _ = _median_runs(run_once, 1, warm=0)
        st = res[0][1]
        out["ranks_%d" % world] = {"time_s": t, "iterations": st["iterations"], "branches_match": st["branch"] == sw["branch"],
                                   "halo_rows_per_iteration_rank0": float(np.mean(st["halo_rows"]))}
    print(json.dumps({"workload": "row-block split of SP2, ranks as threads on one GPU, 3D tight-binding gapped "
                                  "N=%d tau=%g tol=1e-10" % (n, tau), **out}), flush=True)


def run_sp2(a):
    """Whole SP2 purifications of a gapped 3D tight-binding H (A/B onsite splitting 10):
    FP64 against mixed precision, time to solution and distance between the results."""
    import torch
    from paper_2102_08505_gb300 import inputs as I
    from paper_2102_08505_gb300 import sp2ell as S
    n = a.n
    tau = a.tau if a.tau != 1e-6 else 1e-5
    idx, val, nnz = I.tight_binding(n, seed=a.seed, delta=10.0)
    H = S.Ellpack.from_numpy(idx, val, nnz)
    out = {}
    Ds = {}
    for name, prec in (("f64", S.SP2_PREC_F64), ("mixed", S.SP2_PREC_MIXED)):
        opt = S.sp2_options_default(tau=tau, precision=prec, spgemm_path=a.path)
        for _ in range(max(1, a.warmup)):
            S.sp2_purify(H, n / 2, 1e-10, opt)
        torch.cuda.synchronize()
        times = []
        for _ in range(max(1, a.steps)):
            t0 = time.perf_counter()
            D, st = S.sp2_purify(H, n / 2, 1e-10, opt)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        Ds[name] = D
        out[name] = {"time_s": float(np.median(times)), "iterations": st["iterations"],
                     "fp32_iterations": st["fp32_iterations"], "status": st["status"],
                     "iters_per_s": st["iterations"] / float(np.median(times)),
                     "final_err": float(st["err"][-1]), "nnz_per_row": float(st["nnz_total"][-1]) / n}
    dD = diff_fro(S, Ds["mixed"], Ds["f64"]) / np.sqrt(n)
    tr = S.ellpack_trace(Ds["mixed"].to_torch())
    line = {"workload": "sp2 time to solution, 3D tight-binding gapped N=%d tau=%g tol=1e-10" % (n, tau),
            "f64": out["f64"], "mixed": out["mixed"], "speedup_mixed_vs_f64": out["f64"]["time_s"] / out["mixed"]["time_s"],
            "dD_fro_over_sqrtN": dD, "mixed_trace_error": abs(tr - n / 2)}
    print(json.dumps(line), flush=True)


def run_batched(a):
    """256 gapped open 3D clusters with N log-uniform in [512, 8192]: one graph-captured
    batched launch (mixed and FP64) against the same matrices purified one by one.  Under
    torchrun the matrices are dealt to ranks by size (no collective on the data path);
    times are the maximum over ranks."""
    import torch
    import torch.distributed as dist
    from paper_2102_08505_gb300 import inputs as I
    from paper_2102_08505_gb300 import shard
    from paper_2102_08505_gb300 import sp2ell as S
    rank, local, world = shard.rank_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sizes = I.cluster_sizes(a.count, 512, 8192, seed=a.seed)
    mine = shard.deal(sizes, world)[rank]
    tau = 1e-5
    Hs = []
    for m in mine:
        idx, val, nnz = I.tight_binding(int(sizes[m]), seed=a.seed + m, delta=10.0, periodic=False)
        Hs.append(S.Ellpack.from_numpy(idx, val, nnz))
    noccs = [(h.n + 1) // 2 for h in Hs]  # the A sublattice's states: the gap stays at nocc
    res = {}
    for name, prec, graph in (("batched_mixed_graph", S.SP2_PREC_MIXED, 1), ("batched_f64_graph", S.SP2_PREC_F64, 1),
                              ("batched_mixed_host", S.SP2_PREC_MIXED, 0)):
        opt = S.sp2_options_default(tau=tau, precision=prec, graph=graph, spgemm_path=a.path)
        S.sp2_purify_batched(Hs, noccs, 1e-10, opt)
        torch.cuda.synchronize()
        shard.barrier()
        t0 = time.perf_counter()
        Ds, sts = S.sp2_purify_batched(Hs, noccs, 1e-10, opt)
        torch.cuda.synchronize()
        dt = shard.max_over_ranks(time.perf_counter() - t0, dev)
        res[name] = {"time_s": dt, "iterations_total": int(shard.sum_over_ranks(sum(s["iterations"] for s in sts), dev)),
                     "max_iterations": int(shard.max_over_ranks(max(s["iterations"] for s in sts), dev))}
    opt = S.sp2_options_default(tau=tau, precision=S.SP2_PREC_F64, spgemm_path=a.path)
    torch.cuda.synchronize()
    shard.barrier()
    t0 = time.perf_counter()
    its = 0
    for H, nocc in zip(Hs, noccs):
        D, st = S.sp2_purify(H, nocc, 1e-10, opt)
        its += st["iterations"]
    torch.cuda.synchronize()
    res["one_by_one_f64"] = {"time_s": shard.max_over_ranks(time.perf_counter() - t0, dev),
                             "iterations_total": int(shard.sum_over_ranks(its, dev))}
    if rank == 0:
        line = {"workload": "batched SP2: %d gapped open 3D clusters, N log-uniform [512, 8192], sum N = %d" % (
            len(sizes), int(sizes.sum())), "n_gpus": world, "parallelism": "matrices dealt to ranks" if world > 1
            else "single GPU", **res,
            "speedup_batched_mixed_vs_one_by_one_f64":
                res["one_by_one_f64"]["time_s"] / res["batched_mixed_graph"]["time_s"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


MODEL_SETS = {  # the paper's parameter sets of the two-level chain model Hamiltonians
    "metals": dict(d_aa=-1.0, d_bb=-1.0, k=-0.01),
    "semiconductor": dict(d_bb=-1.0, d_ab=-2.0, k=-0.01),
    "soft_matter": dict(d_bb=-1.0, d_ab=-1.0, eps_a=-10.0, k=-0.1, r=1.0),
}


def run_model(a):
    """The paper's own workload: ELLPACK X^2 of the model Hamiltonians (metals,
    semiconductor, soft matter) at N = 32000, FP64, tau = 1e-5 (one product each, timed
    with CUDA events after a warm-up), and SP2 on the semiconductor set (gapped at half
    filling) at N = 4000."""
    import torch
    from paper_2102_08505_gb300 import inputs as I
    from paper_2102_08505_gb300 import sp2ell as S
    n = a.n
    tau = a.tau if a.tau != 1e-6 else 1e-5
    out = {}
    for name, p in MODEL_SETS.items():
        idx, val, nnz = I.model_chain(n, seed=a.seed, **p)
        H = S.Ellpack.from_numpy(idx, val, nnz)
        fmas = fma_count(idx, nnz)
        w = 32
        while True:
            C = S.Ellpack.empty(n, w)
            rc, req = S.ellpack_multiply(H, H, C, 1.0, 0.0, tau, raise_on_overflow=False)
            if rc == 0:
                break
            w = ((req + 31) // 32) * 32
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = max(1, min(a.steps, 3))
        e0.record()
        for _ in range(reps):
            S.ellpack_multiply(H, H, C, 1.0, 0.0, tau)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"nnz_per_row": float(nnz.mean()), "product_nnz_per_row": float(C.nnz.double().mean()),
                     "fma": fmas, "x2_ms": ms, "gflops": 2.0 * fmas / (ms * 1e-3) / 1e9}
        del C, H
    # SP2 on the semiconductor set, the one gapped at half filling (FP64 and mixed), at
    # N = 4000 (its density matrix keeps ~3100 entries per row).  Its error settles on the
    # floor tau sets, above tol: the stall rule stops it, as written (ratio 1) and with
    # ratio 0.9, which also ends a slow monotone drift on that floor.
    ns = min(n, 4000)
    idx, val, nnz = I.model_chain(ns, seed=a.seed, **MODEL_SETS["semiconductor"])
    H = S.Ellpack.from_numpy(idx, val, nnz)
    for prec_name, prec, ratio in (("f64", S.SP2_PREC_F64, 1.0), ("mixed", S.SP2_PREC_MIXED, 1.0),
                                   ("f64_stall_ratio0.9", S.SP2_PREC_F64, 0.9),
                                   ("mixed_stall_ratio0.9", S.SP2_PREC_MIXED, 0.9)):
        opt = S.sp2_options_default(tau=tau, precision=prec, stall_ratio=ratio)
        S.sp2_purify(H, ns / 2, 1e-10, opt, allow_notconv=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D, st = S.sp2_purify(H, ns / 2, 1e-10, opt, allow_notconv=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["sp2_semiconductor_n%d_%s" % (ns, prec_name)] = {
            "time_s": dt, "iterations": st["iterations"], "status": st["status"], "iters_per_s": st["iterations"] / dt,
            "final_err": float(st["err"][-1]), "nnz_per_row_D": float(st["nnz_total"][-1]) / ns}
    print(json.dumps({"workload": "model Hamiltonians (two-level A/B chain), N=%d, FP64 X^2 and SP2, tau=%g" % (n, tau),
                      **out}), flush=True)


def run_schedule(a):
    """Stopping-rule and precision-schedule variants of SP2 on the gapped 3D tight-binding H
    (N=131072, tau=1e-5, tol=1e-10): the stall rule's arming threshold for FP64, and the
    FP32 -> FP64 switch point and tail length for mixed precision; time to solution and
    distance to the FP64 result."""
    import torch
    from paper_2102_08505_gb300 import inputs as I
    from paper_2102_08505_gb300 import sp2ell as S
    n = a.n
    tau = a.tau if a.tau != 1e-6 else 1e-5
    idx, val, nnz = I.tight_binding(n, seed=a.seed, delta=10.0)
    H = S.Ellpack.from_numpy(idx, val, nnz)

    def timed(opt):
        S.sp2_purify(H, n / 2, 1e-10, opt, allow_notconv=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D, st = S.sp2_purify(H, n / 2, 1e-10, opt, allow_notconv=True)
        torch.cuda.synchronize()
        return D, st, time.perf_counter() - t0

    out = {}
    ref = None
    for arm in (0.1, 0.01, 1.0):
        D, st, dt = timed(S.sp2_options_default(tau=tau, stall_arm=arm))
        if arm == 0.1:
            ref = D
        out["f64_stall_arm_%g" % arm] = {"time_s": dt, "iterations": st["iterations"], "status": st["status"],
                                          "final_err": float(st["err"][-1])}
    for name, sw, tail in (("switch_1e-6_tail_2", 1e-6, 2), ("switch_1e-4_tail_2", 1e-4, 2),
                           ("switch_1e-8_tail_2", 1e-8, 2), ("switch_at_fp32_stall_tail_2", 1e-300, 2),
                           ("switch_1e-6_tail_1", 1e-6, 1), ("switch_1e-6_tail_4", 1e-6, 4)):
        D, st, dt = timed(S.sp2_options_default(tau=tau, precision=S.SP2_PREC_MIXED, switch_tol=sw, n_fp64_tail=tail))
        out["mixed_" + name] = {"time_s": dt, "iterations": st["iterations"], "fp32_iterations": st["fp32_iterations"],
                                "status": st["status"], "dD_vs_f64": diff_fro(S, D, ref) / np.sqrt(n)}
    print(json.dumps({"workload": "SP2 schedule variants, 3D tight-binding gapped N=%d tau=%g tol=1e-10" % (n, tau),
                      **out}), flush=True)


def run_sizing(a):
    """Output sizing of the SP2 products: heuristic widths with regrow, exact structural
    counts before every multiply, and the row-length MLP (trained on about 50k rows of
    SP2 products of gapped 3D Hamiltonians of 4096 .. 16384 sites), each used for a mixed
    precision SP2 run on a gapped 3D tight-binding H of N=1048576 sites (input width 128);
    beside them plain FP64 SP2 with heuristic widths, the form the others are measured
    against."""
    import torch
    from paper_2102_08505_gb300 import inputs as I
    from paper_2102_08505_gb300 import learned
    from paper_2102_08505_gb300 import sp2ell as S
    n = a.n
    tau = a.tau if a.tau != 1e-6 else 1e-5
    t0 = time.perf_counter()
    feat, counts = learned.default_training_set(seed=100 + a.seed, rows=50000, tau=tau, dtype=S.SP2_F32)
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    pred, loss = learned.train(feat, counts, seed=a.seed, steps=1500, batch=2048, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    idx, val, nnz = I.tight_binding(n, seed=a.seed, delta=10.0)
    w0 = max(128, ((int(nnz.max()) + 31) // 32) * 32)
    pad_i = np.zeros((n, w0), np.int32)
    pad_v = np.full((n, w0), np.nan)
    pad_i[:, :idx.shape[1]] = idx
    pad_v[:, :idx.shape[1]] = val
    H = S.Ellpack.from_numpy(pad_i, pad_v, nnz)
    res, Ds = {}, {}
    for mode, name, prec in ((2, "mlp", S.SP2_PREC_MIXED), (1, "structural", S.SP2_PREC_MIXED),
                             (0, "heuristic", S.SP2_PREC_MIXED), (0, "plain_f64", S.SP2_PREC_F64)):
        kw = dict(tau=tau, precision=prec, sizing=mode, spgemm_path=a.path)
        if mode == 2:
            kw["predictor"] = pred
        opt = S.sp2_options_default(**kw)
        times = []
        try:
            for _ in range(max(1, min(a.warmup, 2))):
                S.sp2_purify(H, n / 2, 1e-10, opt)
            torch.cuda.synchronize()
            for _ in range(max(1, min(a.steps, 3))):
                t0 = time.perf_counter()
                D, st = S.sp2_purify(H, n / 2, 1e-10, opt)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
        except S.Sp2Error as e:
            st = getattr(e, "stats", {})
            res[name] = {"error": str(e), "iterations": st.get("iterations"),
                         "max_row_nnz": [int(x) for x in st.get("max_row_nnz", [])],
                         "err": [float(x) for x in st.get("err", [])], "width_max": st.get("width_max")}
            continue
        Ds[name] = D
        res[name] = {"time_s": float(np.median(times)), "iterations": st["iterations"], "status": st["status"],
                     "width_max": st["width_max"], "regrows": st["regrows"], "struct_passes": st["struct_passes"],
                     "peak_product_bytes": int(st["width_max"]) * n * 12}
        if mode == 2:
            res[name].update({"pred_log_mae": st["pred_log_mae"], "pred_under_frac": st["pred_under_frac"]})
    line = {"workload": "SP2 output sizing, 3D tight-binding gapped N=%d tau=%g mixed precision" % (n, tau),
            "training": {"rows": int(counts.shape[0]), "collect_s": t_collect, "train_s": t_train,
                         "final_batch_loss": loss},
            **res,
            **{"dD_%s_vs_mlp" % k: diff_fro(S, Ds[k], Ds["mlp"]) / np.sqrt(n) for k in Ds if k != "mlp" and "mlp" in Ds},
            **({"speedup_mixed_mlp_vs_plain_f64": res["plain_f64"]["time_s"] / res["mlp"]["time_s"]}
               if "time_s" in res.get("plain_f64", {}) and "time_s" in res.get("mlp", {}) else {})}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.n is None:
        a.n = {"sp2": 131072, "sizing": 1048576, "model": 32000, "schedule": 131072,
               "rowblock": 131072}.get(a.workload, 262144)
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "sp2":
        run_sp2(a)
    elif a.workload == "batched":
        run_batched(a)
    elif a.workload == "sizing":
        run_sizing(a)
    elif a.workload == "model":
        run_model(a)
    elif a.workload == "schedule":
        run_schedule(a)
    elif a.workload == "rowblock":
        run_rowblock(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
