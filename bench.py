#!/usr/bin/env python3
"""Benchmark of partial modular polynomial evaluation on GB300.

One step = one poly_eval_run over the whole hot path (power tables, Step A,
Step B) for the large workload: n=9, a 62-bit prime, 1e6 terms in 5,041
(x1,x2) groups with Zipf(1.1) sizes, x3..x9 exponents in 0..20, T=1024 points.
The metric is term-point evaluations per second (s*T per step).

  value    device time of K steps with the terms resident in HBM (CUDA events
           on the launch stream; L2 flushed by a 256 MB write between steps)
  e2e      the same metric through the C ABI with host buffers: create from
           host arrays (upload), run into pinned host memory (download), destroy
  roofline Step B, timed live with events on its stream, against the integer
           multiply issue rate of the SMs at the sampled SM clock
  cpu_baseline  the oracle's matrix method (single thread) over the workload; also
           the oracle's plain definition on 1/64 of the groups, and both on
           every host core over the whole workload

--impl reference times the oracle instead (the method's plain CPU statement).
Under torchrun each rank evaluates its own block of T points (weak scaling,
no data-path collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

# 32-bit integer operations per term-point of each modular product, by kind.
# Lazy Barrett: quotient x1*w1 (wide) + hi(x1*w0) + hi(x0*w1); the low halves of
# x*w and q*p, each one wide and two low multiplies.  Montgomery: the 128-bit
# x*y and hi(q*p) (each one high and three wide), q = lo*p' (one wide, two low).
# 32-bit Barrett: hi(x*wq) and two low multiplies.  The roofline weights each
# kind by the measured issue rate of mad.lo relative to its own
# (poly_eval_int_pipe_rates), so `peak` is the mad.lo rate of all SMs at the
# sampled clock and `achieved` is Step B's term-points/s times the weighted count.
OPS_PER_TP = {"barrett64": {"wide": 3, "hi": 2, "lo": 4}, "mont64": {"wide": 8, "hi": 2, "lo": 4},
              "barrett32": {"wide": 0, "hi": 1, "lo": 2}}
# FP64-pipe operations per term-point of the FP64 path, counted in the source:
# Algorithm 2's product (mul, fma, mul, floor, fma, add, and two compare-and-
# correct pairs: 10) and Algorithm 3's sum (add, compare, correct: 3).
FP64_OPS_PER_TP = 13
GOLDEN = os.path.join(ROOT, "tests", "golden", "fullsize_images.json")
_GOLD = None


def golden() -> dict:
    """Stored SHA-256 digests of the oracle's images of the full-size workloads
    (written by tests/golden/make_fullsize_digests.py; read here as data)."""
    global _GOLD
    if _GOLD is None:
        try:
            with open(GOLDEN) as f:
                _GOLD = json.load(f)
        except Exception:
            _GOLD = {}
    return _GOLD


def oracle_match(rec, w, out):
    """True / False when a stored oracle digest exists for exactly these inputs,
    None otherwise.  `out` is a (T, G) tensor or array of the images."""
    if not rec or rec.get("inputs") != wl.inputs_digest(w):
        return None
    if hasattr(out, "cpu"):
        out = out.cpu().numpy()
    return wl.images_digest(out) == rec["images"]


# DRAM bytes (read + write) of one Step B launch on the large workload, from
# ncu captures of the current kernel with the item shapes the tuner picks for
# it (the mean of the two timed launches of each capture); reported only when
# the timed plan has one of these shapes (None for other workloads).
STEPB_TRAFFIC_LARGE = [
    {"bytes": (102_800_128 + 103_015_936) // 2,
     "shape": {"K": 12, "slabs": 1, "tchunk": 224, "warps_per_block": 4, "tail_points": 128}},
    {"bytes": (89_652_992 + 89_678_080) // 2,
     "shape": {"K": 16, "slabs": 1, "tchunk": 224, "warps_per_block": 4, "tail_points": 128}},
]


def stepb_traffic(config, vkey, plan):
    """The captured DRAM bytes of Step B if the timed plan is a captured one."""
    if config != "large" or vkey != "barrett64":
        return None
    for ref in STEPB_TRAFFIC_LARGE:
        if all(plan.get(k) == v for k, v in ref["shape"].items()):
            return ref["bytes"]
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large",
                    choices=["large", "large30", "tiny", "width62", "width62ntt", "width50", "batched", "served",
                             "interp"])
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--tiles", default="",
                    help="force Step B tiles K,slabs,tchunk,warps_per_block,tail (no tuning), e.g. 16,1,224,4,128")
    ap.add_argument("--method", default="auto", choices=["auto", "matrix", "fast"],
                    help="auto: what poly_eval_run picks (the tuner's choice); fast: poly_eval_run_fast")
    ap.add_argument("--serve-seconds", type=float, default=15.0)
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="Poisson request rate; 0 = 0.7x the burst capacity measured in the same run")
    ap.add_argument("--serve-burst", type=int, default=3000)
    ap.add_argument("--serve-streams", type=int, default=4, help="epochs in flight at once (at most 4)")
    ap.add_argument("--serve-epoch-jobs", type=int, default=64, help="requests per epoch at most")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and served sections")
    ap.add_argument("--no-tune", action="store_true", help="skip poly_eval_tune before timing")
    ap.add_argument("--variant", default="auto")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-stride", type=int, default=1)
    ap.add_argument("--split", default="weak", choices=["weak", "strong", "group"],
                    help="N > 1: weak = each rank its own block of T points; strong = the T points split into "
                         "contiguous blocks; group = contiguous ranges of (x1,x2) groups (whole output columns)")
    ap.add_argument("--terms", type=int, default=0,
                    help="a smaller case of the same generator (profiling): terms instead of the config's")
    ap.add_argument("--points", type=int, default=0, help="likewise, points T instead of the config's")
    return ap.parse_args()


def make_workload(name, terms=0, points=0):
    kw = {}
    if terms:
        kw["s"] = terms
    if points:
        kw["T"] = points
    if name == "large":
        return wl.config_large(**kw)
    if name == "large30":
        return wl.config_large(bits=30, **kw)
    if name == "tiny":
        return wl.config_tiny()
    if name == "width62":
        return wl.config_width(62, **kw)
    if name == "width62ntt":
        return wl.config_width(62, ntt=True, **kw)
    return wl.config_width(50, **kw)


def workload_config(w, name):
    """The workload as both arms name it (the same dict for the GPU arm and the
    oracle's reference arm); how an arm ran it goes under its own keys."""
    key = w.exps[:, 0].astype(np.int64) * (1 << 32) + w.exps[:, 1].astype(np.int64)
    return {"workload": w.name, "terms": w.s, "n": w.n, "T": int(w.T), "prime_bits": int(w.p).bit_length(),
            "groups": int(np.unique(key).shape[0]), "config": name,
            "l2": "GPU arm: flushed between timed steps by a 256 MB device write"}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_share(w, split, rank, world):
    """The part of workload `w` that rank `rank` of `world` evaluates, as
    (workload, first point, points, scaling).  No exchange is needed in any
    split (the images of different points and of different groups are
    independent): weak gives every rank T points of its own, strong splits the
    T points into contiguous blocks, group gives each rank the sub-polynomial
    of a contiguous range of (x1,x2) groups with about equal terms."""
    from paper_2004_11571_gb300 import sharding
    if world == 1 or split == "weak":
        t0, T = sharding.weak_block(int(w.T), w.t0, rank)
        return w, t0, T, "weak"
    if split == "strong":
        t0, T = sharding.strong_block(int(w.T), w.t0, rank, world)
        return w, t0, T, "strong"
    key = w.exps[:, 0].astype(np.int64) * (1 << 32) + w.exps[:, 1].astype(np.int64)
    if np.any(key[1:] > key[:-1]):
        w = wl.sort_by_group(w)
        key = w.exps[:, 0].astype(np.int64) * (1 << 32) + w.exps[:, 1].astype(np.int64)
    starts = np.flatnonzero(np.concatenate([[True], key[1:] != key[:-1]])) if w.s else np.zeros(0, np.int64)
    off = np.concatenate([starts, [w.s]])
    g0, g1 = sharding.group_split(off, world)[rank]
    a, b = int(off[g0]), int(off[g1])
    sub = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs[a:b], exps=w.exps[a:b], beta=w.beta, T=w.T, t0=w.t0,
                      name=w.name)
    return sub, w.t0, int(w.T), "strong"


def reduce_over_ranks(values, dist, device, op="max"):
    """Element-wise max (or sum) of a list of floats over all ranks (identity
    without a process group)."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()]


_HOST_CPU = None


def host_cpu():
    """The host CPU's model name and logical core count (lscpu, else /proc/cpuinfo)."""
    global _HOST_CPU
    if _HOST_CPU is None:
        model = ""
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            model = next((l.split(":", 1)[1].strip() for l in out.splitlines() if l.startswith("Model name")), "")
        except Exception:
            pass
        if not model:
            try:
                with open("/proc/cpuinfo") as f:
                    model = next((l.split(":", 1)[1].strip() for l in f if l.lower().startswith("model name")), "")
            except Exception:
                pass
        _HOST_CPU = {"model": model or "unknown", "logical_cores": os.cpu_count() or 0}
    return _HOST_CPU


def cpu_baseline(w, stride):
    """The oracle's matrix method (one thread) on every `stride`-th group, all T points."""
    import oracle
    keys, tg = oracle.group_keys(w.exps)
    sel = (tg % stride) == 0
    sub = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs[sel], exps=w.exps[sel], beta=w.beta, T=w.T, t0=w.t0)
    t = time.perf_counter()
    oracle.eval_matrix(sub)
    dt = time.perf_counter() - t
    return {"value": sub.term_points / dt, "unit": "term-points/s", "cores": 1, "kind": "oracle",
            "sample": f"the oracle's matrix method (gcc -O2, unsigned __int128) on every {stride}-th group: "
                      f"{sub.s} terms x {w.T} points = {sub.term_points:.3e} term-points in {dt:.1f} s",
            "seconds": dt, "host": host_cpu()}


def cpu_baseline_direct(w, stride=64):
    """The oracle's plain definition (one thread: every point's powers of beta,
    then each term's product of them) on every `stride`-th group, all T points."""
    import oracle
    keys, tg = oracle.group_keys(w.exps)
    sel = (tg % stride) == 0
    sub = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs[sel], exps=w.exps[sel], beta=w.beta, T=w.T, t0=w.t0)
    t = time.perf_counter()
    oracle.eval_direct(sub)
    dt = time.perf_counter() - t
    return {"value": sub.term_points / dt, "unit": "term-points/s", "cores": 1, "kind": "oracle (definition)",
            "sample": f"the definition in the oracle (gcc -O2, unsigned __int128) on every {stride}-th group: "
                      f"{sub.s} terms x {w.T} points = {sub.term_points:.3e} term-points in {dt:.1f} s",
            "seconds": dt, "host": host_cpu()}


def _oracle_share(config, rank, nproc, barrier, queue, definition=False):
    """Child of cpu_baseline_all_cores: the oracle's matrix method (or its plain
    definition) on the groups g with g % nproc == rank, all T points, timed
    after a common barrier."""
    import oracle
    w = make_workload(config)
    _, tg = oracle.group_keys(w.exps)
    sel = (tg % nproc) == rank
    sub = wl.Workload(p=w.p, n=w.n, coeffs=w.coeffs[sel], exps=w.exps[sel], beta=w.beta, T=w.T, t0=w.t0)
    oracle.build()
    barrier.wait()
    t = time.perf_counter()
    (oracle.eval_direct if definition else oracle.eval_matrix)(sub)
    queue.put((sub.term_points, time.perf_counter() - t))


def cpu_baseline_all_cores(config, nproc=None, definition=False):
    """The same oracle (matrix method, or the plain definition) as independent
    processes over disjoint group subsets of the full workload, one per host
    core (spawned, not forked)."""
    import multiprocessing as mp
    nproc = nproc or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(nproc), ctx.Queue()
    procs = [ctx.Process(target=_oracle_share, args=(config, r, nproc, barrier, queue, definition))
             for r in range(nproc)]
    for pr in procs:
        pr.start()
    try:
        res = [queue.get(timeout=600) for _ in procs]
    except Exception as ex:  # a child failed: report it instead of waiting
        for pr in procs:
            pr.terminate()
        return {"error": f"oracle processes did not finish: {ex!r}"}
    for pr in procs:
        pr.join()
    tp = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    what = "the definition in the oracle" if definition else "the oracle's matrix method"
    return {"value": tp / dt, "unit": "term-points/s", "cores": nproc,
            "kind": "oracle (definition)" if definition else "oracle",
            "sample": f"{what} (gcc -O2) as {nproc} processes over disjoint group subsets "
                      f"(g mod {nproc}) of the full workload: {tp:.3e} term-points, slowest process {dt:.2f} s",
            "seconds": dt, "host": host_cpu()}


def hbm_peak_gbs():
    """Measured copy bandwidth of this machine's GPUs, else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bench_compact(pe, dense, torch, reps=20):
    """Sparse images of the benchmark's output (poly_eval_compact): one read of
    the dense images to count, one to write, 12 bytes per kept coefficient."""
    T, G = dense.shape
    for _ in range(3):
        pe.compact(dense)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        row_ptr, cols, vals = pe.compact(dense)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / reps
    nnz = int(cols.shape[0])
    algo = 2 * T * G * 8 + 12 * nnz + 8 * (T + 1)
    peak, src = hbm_peak_gbs()
    return {"nnz": nnz, "ms": dt * 1e3, "bound": "hbm", "achieved_gbs": algo / dt / 1e9, "peak_gbs": peak,
            "frac": algo / dt / 1e9 / peak, "peak_source": src,
            "note": "host-timed, includes one stream synchronization per call"}


def bench_multiprime(pe, torch, w, nprimes=4, reps=5):
    """The benchmark's term list modulo several 62-bit primes (Chinese
    remaindering): one full create, then poly_eval_create_like per extra prime
    (coefficients only), and all primes evaluated in one batch."""
    primes = [int(w.p)] + [wl.random_prime(62, 7000 + k) for k in range(1, nprimes)]
    ints = np.random.default_rng(7).integers(0, 1 << 63, size=w.s, dtype=np.uint64)
    coeffs = [(ints % np.uint64(p)).astype(np.uint64) for p in primes]
    torch.cuda.synchronize()
    t = time.perf_counter()
    layout = pe.Poly(primes[0], coeffs[0], w.exps, sorted_hint=True)
    create_ms = (time.perf_counter() - t) * 1e3
    t = time.perf_counter()
    polys = [layout] + [layout.like(p, c) for p, c in zip(primes[1:], coeffs[1:])]
    like_ms = (time.perf_counter() - t) * 1e3 / (nprimes - 1)
    outs = [torch.empty((w.T, layout.G), dtype=torch.int64, device="cuda") for _ in primes]
    betas = [np.random.default_rng(100 + k).integers(2, p, size=w.n - 2, dtype=np.uint64)
             for k, p in enumerate(primes)]
    batch = pe.Batch([(q, b, w.T, 1, o) for q, b, o in zip(polys, betas, outs)])
    for _ in range(2):
        batch.launch()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        batch.launch()
    ev[1].record()
    torch.cuda.synchronize()
    batch_ms = ev[0].elapsed_time(ev[1]) / reps
    for q, b, o in zip(polys, betas, outs):
        q.run(b, w.T, out=o)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        for q, b, o in zip(polys, betas, outs):
            q.run(b, w.T, out=o)
    ev[1].record()
    torch.cuda.synchronize()
    loop_ms = ev[0].elapsed_time(ev[1]) / reps
    batch.close()
    for q in polys:
        q.close()
    tp = nprimes * w.s * w.T
    return {"primes": nprimes, "create_ms": create_ms, "create_like_ms": like_ms,
            "shared_exponent_bytes": int(w.s * (w.n - 2)), "batch_ms": batch_ms,
            "batch_term_points_per_s": tp / (batch_ms * 1e-3), "loop_ms": loop_ms,
            "loop_term_points_per_s": tp / (loop_ms * 1e-3),
            "note": "create/create_like host-timed; batch and loop timed with CUDA events, inputs resident"}


def _fast_counts(off, T):
    """Shoup products (NTT butterflies and scalings) and Montgomery products
    (pointwise) of the fast method's product trees and series for column
    offsets `off` and T points, following the library's block structure."""
    Tp = 64
    while Tp < T:
        Tp *= 2
    lg = lambda x: x.bit_length() - 1
    ntt = lambda N: (N // 2) * lg(N)
    shoup = mont = 0
    # Newton step k: five NTTs of size 2k (one transform of h serves both products), two scalings, two
    # pointwise products; then N h with three NTTs of size 2Tp.
    series_shoup = sum(5 * ntt(2 << k) + 2 * (2 << k) for k in range(lg(Tp)))
    series_shoup += 3 * ntt(2 * Tp) + 2 * Tp
    series_mont = sum(2 * (2 << k) for k in range(lg(Tp))) + 2 * Tp
    for g in range(len(off) - 1):
        n = int(off[g + 1] - off[g])
        for a in range(0, n, Tp):
            d = min(Tp, n - a)
            L = 32
            while L < d:
                for ps in range(0, d, 2 * L):
                    la = min(L, d - ps)
                    if min(L, d - ps - la):
                        shoup += 6 * ntt(2 * L) + 2 * 2 * L
                        mont += 3 * 2 * L
                L *= 2
            shoup += series_shoup
            mont += series_mont
    return shoup, mont


def _fast_launches(off, T):
    """Kernel launches of one fast-method run: power tables, Step A, leaves, the
    merge levels some block reaches, series, sum."""
    Tp = 64
    while Tp < T:
        Tp *= 2
    dmax = max(min(Tp, int(off[g + 1] - off[g])) for g in range(len(off) - 1))
    levels, L = 0, 32
    while L < dmax:
        levels += 1
        L *= 2
    return 5 + levels


def bench_fast(pe, torch, mhz, reps=3):
    """The fast method (Sect. 2.3.1) beside the matrix method on NTT-friendly
    62-bit primes: the width workload (81 groups of ~49,000 terms) at T = 4096
    and 1024, and the large workload's shape (5,041 Zipf groups) at T = 1024."""
    rates = pe.int_pipe_rates()
    wide, hi = rates["mad_lo"] / rates["mad_wide"], rates["mad_lo"] / rates["mad_hi"]
    shoup_slots, mont_slots = 3 * wide + 2 * hi + 4, 8 * wide + 2 * hi + 4   # lazy Shoup product; Montgomery
    peak = pe.num_sms() * rates["mad_lo"] * mhz * 1e6
    res = []
    cases = [wl.config_width(62, ntt=True), wl.config_width(62, ntt=True, T=1024),
             wl.make_zipf(n=9, s=1_000_000, p=wl.random_ntt_prime(62, 20, 5), deg12=70, deg_rest=20, T=1024,
                          seed=wl.SEED_LARGE + 1, a=1.1, name="large shape n=9 s=1e6 G=5041 T=1024 p62 ntt")]
    for w in cases:
        poly = pe.Poly.from_workload(w)
        out_m = torch.empty((w.T, poly.G), dtype=torch.int64, device="cuda")
        out_f = torch.empty_like(out_m)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        poly.run(w.beta, w.T, out=out_m)
        poly.run_fast(w.beta, w.T, out=out_f)
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            poly.run(w.beta, w.T, out=out_m)
        ev[1].record()
        for _ in range(reps):
            poly.run_fast(w.beta, w.T, out=out_f)
        ev[2].record()
        torch.cuda.synchronize()
        m_ms, f_ms = ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps
        identical = bool(torch.equal(out_m, out_f))
        _, off = poly.monomials(w.beta)
        sh, mo = _fast_counts(off, w.T)
        slots = sh * shoup_slots + mo * mont_slots
        res.append({"workload": w.name, "matrix_ms": m_ms, "fast_ms": f_ms, "fast_over_matrix": m_ms / f_ms,
                    "identical": identical, "fast_term_points_per_s": w.s * w.T / (f_ms * 1e-3),
                    "shoup_products": sh, "montgomery_products": mo,
                    "products_per_term_point": (sh + mo) / (w.s * w.T),
                    "roofline": {"bound": "alu", "achieved": slots / (f_ms * 1e-3) / 1e9, "peak": peak / 1e9,
                                 "unit": "Gslot/s", "frac": slots / (f_ms * 1e-3) / peak,
                                 "algorithmic": f"Shoup products {shoup_slots:.1f} mad.lo slots, Montgomery "
                                                f"{mont_slots:.1f}; counted from the block structure"}})
        poly.close()
        del out_m, out_f
    return res


def _vdm_counts(off):
    """Algorithmic multiplies of the solver: exact 64x64-bit products of the
    product tree and of the correlation, fixed-multiplier products of Horner."""
    tree = corr = horner = n2 = 0
    for g in range(len(off) - 1):
        n = int(off[g + 1] - off[g])
        L = 1
        while L < n:
            for base in range(0, n, 2 * L):
                la = min(L, n - base)
                tree += la * min(L, n - base - la)
            L *= 2
        corr += n * (n - 1) // 2
        horner += 2 * n * n
        n2 += n * n
    return tree, corr, horner, n2


def bench_interp(pe, torch, mhz, reps=10):
    """Interpolation from images (Sect. 1) after an evaluation at T = u points:
    a factor of the m = 14 symmetric Toeplitz determinant by size (34,937
    terms, largest coefficient 9,705 terms) and the gcd benchmark's g by size
    (10^4 terms, largest coefficient 122 terms)."""
    rates = pe.int_pipe_rates()
    wide = rates["mad_lo"] / rates["mad_wide"]
    slots_exact = 4 * wide
    slots_b = sum(n * c for n, c in zip(OPS_PER_TP["barrett64"].values(),
                                        (wide, rates["mad_lo"] / rates["mad_hi"], 1.0)))
    peak = pe.num_sms() * rates["mad_lo"] * mhz * 1e6 / 1e9
    res = []
    for w in (wl.config_interp(), wl.config_interp(seed=wl.SEED_INTERP + 1, s=10_000, u=122, n=9)):
        poly = pe.Poly.from_workload(w)
        images = poly.run(w.beta, w.T, t0=1)
        torch.cuda.synchronize()
        t = time.perf_counter()
        images = poly.run(w.beta, w.T, t0=1)
        torch.cuda.synchronize()
        eval_ms = (time.perf_counter() - t) * 1e3
        z, off = poly.monomials(w.beta)
        for _ in range(3):
            c = pe.vandermonde_solve(w.p, off, z, images, t0=1)
        pe.vandermonde_timing(True)
        kms = {"leaves": 0.0, "tree": 0.0, "correlation": 0.0, "horner": 0.0}
        t = time.perf_counter()
        for _ in range(reps):
            c = pe.vandermonde_solve(w.p, off, z, images, t0=1)
            for k, v in pe.vandermonde_timing().items():
                kms[k] += v / reps
        dt = (time.perf_counter() - t) / reps
        pe.vandermonde_timing(False)
        exact = pe.to_u64(c).tolist() == w.coeffs.tolist()
        tree, corr, horner, n2 = _vdm_counts(off)
        ach = horner * slots_b / (kms["horner"] * 1e-3) / 1e9 if kms["horner"] > 0 else None
        res.append({"workload": w.name, "terms": w.s, "columns": int(poly.G), "max_terms": int(w.T),
                    "sum_n2": n2, "exact": exact, "ms": dt * 1e3, "terms_per_s": w.s / dt, "n2_per_s": n2 / dt,
                    "kernel_ms": kms, "eval_images_ms": eval_ms,
                    "multiplies": {"tree_exact": tree, "correlation_exact": corr, "horner_fixed": horner},
                    "roofline": {"kernel": "pe::k_vdm_solve", "bound": "alu", "unit": "Gslot/s",
                                 "achieved": ach, "peak": peak, "frac": ach / peak if ach else None,
                                 "algorithmic": f"2 n^2 lazy Barrett products per column ({slots_b:.2f} mad.lo "
                                                f"slots each) = {horner} products",
                                 "tree_frac": (tree * slots_exact / (kms["tree"] * 1e-3) / 1e9 / peak
                                               if kms["tree"] > 0 else None),
                                 "correlation_frac": (corr * slots_exact / (kms["correlation"] * 1e-3) / 1e9 / peak
                                                      if kms["correlation"] > 0 else None)},
                    "note": "ms is host-timed per call (tile upload, five or more launches, one synchronization)"})
        poly.close()
        del images, z, c
    return res


def stepb_roofline(pe, vkey, p, s, T, tps_b, stepb_ms, mhz, traffic=None):
    """Step B against the issue rate of its pipe at the sampled SM clock: the
    integer multiply pipe (mad.lo slots) for the integer products, the FP64
    pipe (fma.rn.f64 rate) for Algorithm 2; plus the register-only loop of the
    same product (poly_eval_modmul_peak) as a second denominator."""
    sms = pe.num_sms()
    if vkey == "fp64":
        rates = pe.fp64_pipe_rates()
        slots = FP64_OPS_PER_TP
        peak = sms * rates["fma"] * mhz * 1e6 / 1e9
        roof = {"bound": "alu", "achieved": tps_b * slots / 1e9, "peak": peak, "unit": "G FP64 op/s",
                "peak_source": f"{sms} SMs x {rates['fma']:.2f} fma.rn.f64 per SM-clock (measured) x "
                               f"{mhz:.0f} MHz (median sampled SM clock)",
                "algorithmic": f"{FP64_OPS_PER_TP} FP64 operations per term-point (Algorithm 2 product 10, "
                               f"Algorithm 3 sum 3) x {s}x{T} term-points"}
    else:
        rates = pe.int_pipe_rates()
        cost = {"lo": 1.0, "hi": rates["mad_lo"] / rates["mad_hi"], "wide": rates["mad_lo"] / rates["mad_wide"]}
        slots = sum(n * cost[k] for k, n in OPS_PER_TP[vkey].items())
        peak = sms * rates["mad_lo"] * mhz * 1e6 / 1e9
        roof = {"bound": "alu", "achieved": tps_b * slots / 1e9, "peak": peak, "unit": "Gslot/s",
                "peak_source": f"{sms} SMs x {rates['mad_lo']:.1f} mad.lo.u32 per SM-clock (measured) x "
                               f"{mhz:.0f} MHz (median sampled SM clock)",
                "algorithmic": f"{OPS_PER_TP[vkey]} 32-bit multiplies per term-point = {slots:.2f} mad.lo slots "
                               f"x {s}x{T} term-points"}
    roof.update({"frac": roof["achieved"] / peak, "traffic": traffic, "kernel": "pe::k_stepB",
                 "variant": vkey, "sms": sms, "sm_mhz": mhz, "ops_per_term_point": slots,
                 "peak_term_points_per_s": peak * 1e9 / slots, "stepB_ms": stepb_ms,
                 "stepB_term_points_per_s": tps_b})
    try:
        cal, cal_mhz = pe.modmul_peak(vkey, p)
        roof.update({"register_only_term_points_per_s": cal, "frac_of_register_only": tps_b / cal,
                     "register_only_frac_of_peak": cal * slots / (peak * 1e9), "register_only_sm_mhz": cal_mhz})
    except Exception as ex:  # pragma: no cover
        roof["register_only_error"] = str(ex)
    return roof


def bench_config(pe, torch, name, w, variant, steps=4, warmup=2, method="matrix", tune=False):
    """One full-size workload on one product: device time per run (terms
    resident, L2 flushed between runs), Step B's roofline, and whether the
    output equals the oracle's stored images."""
    poly = pe.Poly.from_workload(w, variant=variant)
    T = int(w.T)
    if tune and variant == "auto":
        pe.tune(poly, T)
    out = torch.empty((T, poly.G), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    run = poly.run_fast if method == "fast" else poly.run
    for _ in range(warmup):
        run(w.beta, T, w.t0, out=out, stream=stream)
    torch.cuda.synchronize()
    identical = oracle_match(golden().get("single", {}).get(name), w, out)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    poly.set_timing(True)
    poly.kernel_times()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        run(w.beta, T, w.t0, out=out, stream=stream)
        b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    poly.set_timing(False)
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    _, t_a, t_b, runs = poly.kernel_times()
    plan = poly.plan_info(T)
    vkey = variant if variant in OPS_PER_TP or variant == "fp64" else (
        "barrett32" if int(w.p) < (1 << 30) else "barrett64")
    res = {"workload": w.name, "variant": vkey if method == "matrix" else "fast method", "ms_per_run": ms,
           "term_points_per_s": w.s * T / (ms * 1e-3), "identical_to_oracle": identical,
           "tiles": {k: plan[k] for k in ("K", "slabs", "tchunk", "warps_per_block", "tail_points", "method")},
           "clocks": clk}
    if method == "matrix" and runs and t_b > 0:
        res["stepA_ms"] = t_a / runs
        res["roofline"] = stepb_roofline(pe, vkey, int(w.p), w.s, T, w.s * T / (t_b / runs * 1e-3), t_b / runs,
                                         clk["sm_mhz"] or 1920.0)
    poly.close()
    del out, flush
    return res


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    w = make_workload(args.config, args.terms, args.points)
    stride = max(args.cpu_sample_stride, 1) * 8
    for _ in range(args.warmup):
        cpu_baseline(w, stride * 8)       # untimed warm-up on a smaller sample
    vals, secs = [], []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(w, stride)
        vals.append(cb["value"])
        secs.append(cb["seconds"])
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": "term-point evaluations/s", "value": value, "unit": "term-points/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(w, args.config),
            "plan": {"implementation": "the oracle's matrix method (gcc -O2), one host core"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": cb["sample"], "value": value,
                             "unit": "term-points/s", "host": host_cpu()},
            "e2e": {"value": value, "unit": "term-points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2004_11571_gb300 as pe

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = make_workload(args.config, args.terms, args.points)
    variant = args.variant
    if variant == "auto" and args.config == "width50":
        variant = "fp64"
    if variant == "auto" and args.method == "matrix":    # an explicit product keeps poly_eval_run on the matrix method
        variant = "barrett32" if int(w.p) < (1 << 30) else "barrett64"
    w_full = w
    w, t0, T, scaling = rank_share(w_full, args.split, rank, world)
    poly = pe.Poly.from_workload(w, variant=variant)
    G, s = poly.G, w.s
    tuned = None
    if args.tiles:
        K, slabs, tchunk, wpb, tail = (int(x) for x in args.tiles.split(","))
        poly.set_tiles(K=K, slabs=slabs, tchunk=tchunk, warps_per_block=wpb, tail=tail)
    elif not args.no_tune and variant in ("auto",):
        tiles, tuned_ms = pe.tune(poly, T)          # measures tile shapes and products for this shape
        tuned = {"tiles": tiles, "ms": tuned_ms}
    out = torch.empty((T, G), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    run = poly.run_fast if args.method == "fast" else poly.run
    for _ in range(max(args.warmup, 0)):
        run(w.beta, T, t0, out=out, stream=stream)
        flush.zero_()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    poly.set_timing(True)
    poly.kernel_times()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        run(w.beta, T, t0, out=out, stream=stream)
        b.record(stream)
    barrier()
    clk = clocks.stop()
    poly.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    t_pt, t_a, t_b, runs = poly.kernel_times()
    # Whole-job throughput: the term-points of every rank over the slowest rank's time.
    max_total_ms, = reduce_over_ranks([total_ms], dist, "cuda", "max")
    job_tp, = reduce_over_ranks([float(s) * T * args.steps], dist, "cuda", "sum")
    value = job_tp / (max_total_ms * 1e-3)
    plan = poly.plan_info(T)
    launches = poly.launches_per_run(T) * args.steps
    fast_off = None
    if args.method == "fast" or (args.method == "auto" and plan["method"] == "fast"):
        _, fast_off = poly.monomials(w.beta)
        launches = _fast_launches(fast_off, T) * args.steps

    # End to end through the C ABI with host buffers: the terms in page-locked
    # host memory (uploaded inside the timed region), the images downloaded into
    # page-locked host memory.
    host_out = torch.empty((T, G), dtype=torch.int64, pin_memory=True).numpy()
    h_coeffs = torch.from_numpy(w.coeffs.view(np.int64)).pin_memory().numpy().view(np.uint64)
    h_exps = torch.from_numpy(np.ascontiguousarray(w.exps)).pin_memory().numpy()
    e2e_t = []
    h2d = s * 8 + s * (w.n - 2) * (1 if int(w.exps[:, 2:].max(initial=0)) <= 255 else 2)
    for k in range(max(args.e2e_steps, 1) + 1):      # the first step is an untimed warm-up
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        p2 = pe.Poly(w.p, h_coeffs, h_exps, variant=variant, sorted_hint=True)
        (p2.run_fast if args.method == "fast" else p2.run)(w.beta, T, t0, out=host_out)
        p2.close()
        if k:
            e2e_t.append(time.perf_counter() - t_start)
    e2e_slowest, = reduce_over_ranks([statistics.median(e2e_t)], dist, "cuda", "max")
    e2e_val = job_tp / args.steps / e2e_slowest

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # Roofline of Step B: integer-multiply (or FP64) issue rate at the sampled SM clock.
    vkey = variant if variant in OPS_PER_TP or variant == "fp64" else (
        "barrett32" if int(w.p) < (1 << 30) else "barrett64")
    tps_b = s * T / (t_b / runs * 1e-3) if runs and t_b > 0 else None
    mhz = clk["sm_mhz"] or 1920.0
    sms = pe.num_sms()
    roof = None
    if fast_off is not None:
        rates = pe.int_pipe_rates()
        wide, hi = rates["mad_lo"] / rates["mad_wide"], rates["mad_lo"] / rates["mad_hi"]
        sh, mo = _fast_counts(fast_off, T)
        slots = sh * (3 * wide + 2 * hi + 4) + mo * (8 * wide + 2 * hi + 4)
        step_s = statistics.mean(step_ms) * 1e-3
        peak = sms * rates["mad_lo"] * mhz * 1e6 / 1e9
        roof = {"bound": "alu", "achieved": slots / step_s / 1e9, "peak": peak, "unit": "Gslot/s",
                "frac": slots / step_s / 1e9 / peak, "traffic": None, "kernel": "fast method (all kernels)",
                "algorithmic": f"{sh} Shoup and {mo} Montgomery products per run (NTT butterflies, scalings, "
                               f"pointwise products), counted from the block structure",
                "peak_source": f"{sms} SMs x {rates['mad_lo']:.1f} mad.lo.u32 per SM-clock (measured) x "
                               f"{mhz:.0f} MHz (median sampled SM clock)"}
    elif tps_b:
        roof = stepb_roofline(pe, vkey, int(w.p), s, T, tps_b, t_b / runs, mhz,
                              stepb_traffic(args.config, vkey, plan))
    line = {"metric": "term-point evaluations/s", "value": value, "unit": "term-points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": True, "scaling": scaling, "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": workload_config(w_full, args.config),
            "plan": {"variant": variant, "tiles": plan, "tuned": tuned is not None, "split": args.split,
                     "rank0_points": f"{t0}..{t0 + T - 1}", "rank0_terms": s, "rank0_groups": G},
            "clocks": clk,
            "e2e": {"value": e2e_val, "unit": "term-points/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(T * G * 8), "median_s": statistics.median(e2e_t)},
            "gpu_launches": launches,
            "kernel_ms_per_step": {"power_tables": t_pt / max(runs, 1), "stepA": t_a / max(runs, 1),
                                   "stepB": t_b / max(runs, 1)},
            "roofline": roof,
            "identical_to_oracle": oracle_match(golden().get("single", {}).get(args.config), w, out)
            if t0 == w.t0 and args.method != "fast" else None}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_sample_stride)
        line["cpu_baseline_definition"] = cpu_baseline_direct(w)
        if args.config in ("large", "large30", "tiny"):
            line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.config)
            line["cpu_baseline_definition_all_cores"] = cpu_baseline_all_cores(args.config, definition=True)
    if world == 1 and not args.no_extras:
        line["sparse_images"] = bench_compact(pe, out, torch)
        line["interpolation"] = bench_interp(pe, torch, mhz)
        if args.config == "large":
            line["multi_prime"] = bench_multiprime(pe, torch, w)
            line["fast_method"] = bench_fast(pe, torch, mhz)
    poly.close()
    if world == 1 and not args.no_extras and args.config == "large":
        # The large workload on the Montgomery product, and the width pair
        # (4e6 terms, 81 groups, T = 4096): 62-bit on the integer products,
        # 50-bit on Algorithm 2's FP64 product.
        line["large_montgomery"] = bench_config(pe, torch, "large", w, "mont64", steps=5, warmup=2)
        w62, w50 = wl.config_width(62), wl.config_width(50)
        line["width"] = [bench_config(pe, torch, "width62", w62, "auto", steps=4, warmup=2, tune=True),
                         bench_config(pe, torch, "width62", w62, "mont64", steps=3, warmup=1),
                         bench_config(pe, torch, "width50", w50, "fp64", steps=3, warmup=1)]
        del w62, w50
    if world == 1 and not args.no_extras:
        del out, flush
        torch.cuda.empty_cache()
        bargs = argparse.Namespace(**vars(args))
        bargs.steps, bargs.warmup = 4, 2
        line["batched"] = run_batched(bargs, print_line=False)
        line["served"] = served_in_child(args)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batched(args, print_line=True):
    """Config of 512 independent polynomials: one CUDA-graph launch of the
    persistent kernel vs a loop of per-polynomial poly_eval_run calls; the same
    for the jobs below 2^28 term-points alone (the ones the queue kernel runs:
    larger jobs leave the graph as plain runs); both outputs checked against the
    oracle's stored images."""
    import torch
    import paper_2004_11571_gb300 as pe

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    t_gen = time.perf_counter()
    ws = wl.config_batched(count=args.batch_count)
    t_gen = time.perf_counter() - t_gen
    t_create = time.perf_counter()
    polys = [pe.Poly.from_workload(w) for w in ws]
    t_create = time.perf_counter() - t_create
    outs = [torch.empty((w.T, p.G), dtype=torch.int64, device="cuda") for w, p in zip(ws, polys)]
    from paper_2004_11571_gb300 import sharding
    t0s = [sharding.weak_block(int(w.T), 1, rank)[0] for w in ws]
    tp = sum(w.s * w.T for w in ws)
    small = [k for k, w in enumerate(ws) if w.s * w.T < (1 << 28)]
    tp_small = sum(ws[k].s * ws[k].T for k in small)
    t_plan = time.perf_counter()
    batch = pe.Batch([(p, w.beta, w.T, t0, o) for p, w, t0, o in zip(polys, ws, t0s, outs)])
    t_plan = time.perf_counter() - t_plan
    batch_small = pe.Batch([(polys[k], ws[k].beta, ws[k].T, t0s[k], outs[k]) for k in small])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for a, b2 in evs:
            flush.zero_()
            a.record(stream)
            fn()
            b2.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b2) for a, b2 in evs]

    def loop(jobs):
        for k in jobs:
            polys[k].run(ws[k].beta, ws[k].T, t0s[k], out=outs[k], stream=stream)

    records = golden().get("batched", {}).get("jobs", [])

    def check():
        """Jobs whose output equals the oracle's stored images (None: no record for these inputs)."""
        if rank != 0 or len(records) != len(ws) or any(t0 != w.t0 for t0, w in zip(t0s, ws)):
            return None
        torch.cuda.synchronize()
        res = [oracle_match(r, w, o) for r, w, o in zip(records, ws, outs)]
        if any(x is None for x in res):
            return {"identical": None, "jobs_without_record": sum(x is None for x in res)}
        return {"identical": all(res), "jobs_checked": len(res), "jobs_differing": sum(not x for x in res)}

    every = list(range(len(ws)))
    for _ in range(max(args.warmup, 0)):
        batch.launch(stream)
        loop(every)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms_batch = timed(lambda: batch.launch(stream), args.steps)
    clk = clocks.stop()
    check_batch = check()
    for o in outs:
        o.fill_(-1)
    ms_loop = timed(lambda: loop(every), max(1, args.steps // 2))
    check_loop = check()
    for _ in range(2):
        batch_small.launch(stream)
        loop(small)
    ms_small_batch = timed(lambda: batch_small.launch(stream), args.steps)
    ms_small_loop = timed(lambda: loop(small), args.steps)
    v_batch = tp / (statistics.mean(ms_batch) * 1e-3)
    v_loop = tp / (statistics.mean(ms_loop) * 1e-3)
    v_sb = tp_small / (statistics.mean(ms_small_batch) * 1e-3)
    v_sl = tp_small / (statistics.mean(ms_small_loop) * 1e-3)
    launches_loop = sum(p.launches_per_run(w.T) for p, w in zip(polys, ws))
    bl = batch.launches()
    bls = batch_small.launches()
    batch.close()
    batch_small.close()
    for p in polys:
        p.close()
    if rank != 0:
        return None
    summary = {"workload": f"{len(ws)} polynomials: n 6..12, s log-uniform 1e3..1e6, D 5..60, "
                           "T in {64,256,1024,2048}, 50/62-bit primes",
               "term_points": tp, "batched_term_points_per_s": v_batch, "ms_per_launch": statistics.mean(ms_batch),
               "plain_loop_term_points_per_s": v_loop, "plain_loop_ms": statistics.mean(ms_loop),
               "ms_per_step": {"batched": [round(x, 3) for x in ms_batch], "plain_loop": [round(x, 3) for x in ms_loop]},
               "batched_over_plain_loop": v_batch / v_loop, "launches_batched": bl["kernels"],
               "plain_run_jobs": bl["plain_jobs"], "launches_plain_loop": launches_loop,
               "oracle_check_batched": check_batch, "oracle_check_plain_loop": check_loop,
               "queue_jobs": {"jobs": len(small), "term_points": tp_small,
                              "batched_term_points_per_s": v_sb, "ms_per_launch": statistics.mean(ms_small_batch),
                              "plain_loop_term_points_per_s": v_sl, "plain_loop_ms": statistics.mean(ms_small_loop),
                              "batched_over_plain_loop": v_sb / v_sl, "launches_batched": bls["kernels"],
                              "note": "the jobs below 2^28 term-points, which the queue kernel runs"},
               "clocks": clk}
    if not print_line:
        return summary
    line = {"metric": "term-point evaluations/s (batched)", "value": v_batch * world, "unit": "term-points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms_batch),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"batched {len(ws)} polynomials, n 6..12, s log-uniform 1e3..1e6, "
                                   "D 5..60, T in {64,256,1024,2048}, 50/62-bit primes",
                       "term_points": tp, "terms": sum(w.s for w in ws), "jobs": len(ws),
                       "l2": "flushed between timed steps by a 256 MB device write"},
            "clocks": clk, "plain_loop": {"value": v_loop, "ms_per_step": statistics.mean(ms_loop),
                                          "launches": launches_loop},
            "batched_over_plain_loop": v_batch / v_loop, "gpu_launches": bl["kernels"] * args.steps,
            "queue_jobs": summary["queue_jobs"], "oracle_check_batched": check_batch,
            "oracle_check_plain_loop": check_loop,
            "host_seconds": {"generate": t_gen, "create": t_create, "plan_and_capture": t_plan}}
    print(json.dumps(line), flush=True)
    return summary


class PinnedRing:
    """Page-locked host output buffers handed out in FIFO order.

    Regions are kept in allocation order.  The ring is wrapped when the newest
    region starts below the oldest: the free space is then the gap between the
    newest region's end and the oldest region's start; otherwise it is the
    space after the newest region plus the space before the oldest."""

    def __init__(self, nbytes):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True).numpy()
        self.cap = nbytes
        self.regions = []   # (start, end, tag) in allocation order

    def alloc(self, size, wait_oldest):
        size = (size + 255) // 256 * 256
        if size > self.cap:
            raise ValueError("output larger than the ring")
        while True:
            if not self.regions:
                return 0
            tail, head = self.regions[0][0], self.regions[-1][1]
            if self.regions[-1][0] < tail:           # wrapped: free is [head, tail)
                if tail - head >= size:
                    return head
            elif self.cap - head >= size:            # not wrapped: after the newest ...
                return head
            elif tail >= size:                       # ... or before the oldest
                return 0
            wait_oldest()

    def commit(self, start, size, tag):
        size = (size + 255) // 256 * 256
        self.regions.append((start, start + size, tag))

    def view(self, start, shape):
        n = shape[0] * shape[1] * 8
        return self.buf[start:start + n].view(np.uint64).reshape(shape)


def served_child_argv(args):
    """Command line of `bench.py --config served` with this run's serving options."""
    return [sys.executable, os.path.join(ROOT, "bench.py"), "--config", "served",
            "--batch-count", str(args.batch_count), "--serve-seconds", str(args.serve_seconds),
            "--serve-rate", str(args.serve_rate), "--serve-burst", str(args.serve_burst),
            "--serve-streams", str(args.serve_streams), "--serve-epoch-jobs", str(args.serve_epoch_jobs)]


def served_in_child(args):
    """The served section in a process of its own, as a server runs: inside
    this process, after the other sections, the same bursts measured 1.3-3x
    slower with the SM clocks at their maximum.  Falls back to this process
    if the child fails."""
    try:
        r = subprocess.run(served_child_argv(args), capture_output=True, text=True, timeout=900)
        lines = [ln for ln in r.stdout.strip().splitlines() if ln.startswith("{")]
        if r.returncode == 0 and lines:
            res = json.loads(lines[-1])
            res.pop("metric", None)
            res["process"] = "child (bench.py --config served)"
            return res
        why = f"child exited {r.returncode}: {r.stderr.strip().splitlines()[-1:] }"
    except Exception as e:  # noqa: BLE001 - any failure of the child falls back to this process
        why = f"child failed: {e!r}"
    res = run_served(args)
    res["process"] = f"this process ({why})"
    return res


def run_served(args, pool=None):
    """Served workload: requests drawn from the batched mixture (30% reuse a
    resident polynomial at a new beta).  Three measurements: a burst submitted
    back to back (throughput at saturation; the median of three), the same requests through the plain
    path one by one (create, run into host memory, destroy), and a Poisson
    stream at 0.7x the burst's request rate (or --serve-rate) for latency below
    saturation.  Requests in the stored seeded sample (~1%) are copied out as
    they complete and compared with the oracle's images once the timed region
    has ended (hashing their inputs and outputs inside it cost the client
    thread tens of milliseconds per burst)."""
    import torch
    import paper_2004_11571_gb300 as pe

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if pool is None:
        pool = wl.config_batched(seed=wl.SEED_SERVE, count=args.batch_count)
    G = [int(len(np.unique(w.exps[:, 0].astype(np.int64) * 65536 + w.exps[:, 1]))) for w in pool]
    ring = PinnedRing(6 << 30)
    sample = {r["index"]: r for r in golden().get("served", {}).get("sample", [])}
    if args.batch_count != 512:
        sample = {}

    submit_s = [0.0]

    def drive(reqs, srv, paced):
        ids = {}
        start = time.perf_counter()
        tp = 0.0
        checks = {"checked": 0, "matched": 0, "without_record": 0}
        kept = []                      # sampled outputs, compared with the oracle after the timed region

        def wait_oldest():
            s0, e0, (t, i, shape) = ring.regions.pop(0)
            srv.poll(t)
            if i in sample:
                kept.append((i, ring.view(s0, shape).copy()))

        for i, (ts, k, beta) in enumerate(reqs):
            w = pool[k]
            if paced:
                delay = start + ts - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            shape = (w.T, G[k])
            off = ring.alloc(shape[0] * shape[1] * 8, wait_oldest)
            out = ring.view(off, shape)
            ticket = None
            ts0 = time.perf_counter()
            if beta is not None and k in ids:
                try:
                    ticket, _ = srv.submit(beta, w.T, out, resident_id=ids[k])
                except pe.PolyEvalError:
                    ticket = None
            while ticket is None:
                try:
                    ticket, nid = srv.submit(w.beta if beta is None else beta, w.T, out,
                                             poly=(w.p, w.coeffs, w.exps), borrow=True)
                    ids[k] = nid
                except pe.PolyEvalError as e:
                    if e.status != pe.PE_ERR_ADMISSION:
                        raise
                    if ring.regions:
                        wait_oldest()
                    else:
                        time.sleep(0.001)
            submit_s[0] += time.perf_counter() - ts0
            ring.commit(off, shape[0] * shape[1] * 8, (ticket, i, shape))
            tp += w.s * w.T
        while ring.regions:
            wait_oldest()
        elapsed = time.perf_counter() - start
        for i, out in kept:
            ok = oracle_match(sample[i], wl.served_workload(pool, reqs[i]), out)
            if ok is None:
                checks["without_record"] += 1
            else:
                checks["checked"] += 1
                checks["matched"] += int(ok)
        checks["identical"] = (checks["matched"] == checks["checked"]) if checks["checked"] else None
        return elapsed, tp, checks

    burst = wl.served_requests(seed=wl.SEED_SERVE, rate=2000.0, duration=1.0 + args.serve_burst / 2000.0,
                               pool=pool)[:args.serve_burst]
    # (1) burst: throughput at saturation
    srv = pe.Server(mem_cap_bytes=40 << 30, streams=args.serve_streams, max_epoch_jobs=args.serve_epoch_jobs)
    drive(burst[:50], srv, False)                      # warm-up
    srv.close()
    # three bursts, each on a fresh server; the median one is reported (a burst
    # lasts well under a second and single bursts spread widely)
    runs = []
    for _ in range(3):
        srv = pe.Server(mem_cap_bytes=40 << 30, streams=args.serve_streams, max_epoch_jobs=args.serve_epoch_jobs)
        t_b, tp_b, chk_b = drive(burst, srv, False)
        runs.append((t_b, tp_b, chk_b, srv.stats()))
        srv.close()
    runs.sort(key=lambda r: r[0])
    t_burst, tp_burst, _, st_burst = runs[1]
    burst_rates = [len(burst) / r[0] for r in runs]
    # the sampled requests of all three bursts are checked
    chk_burst = {k: sum(r[2][k] for r in runs) for k in ("checked", "matched", "without_record")}
    chk_burst["identical"] = (chk_burst["matched"] == chk_burst["checked"]) if chk_burst["checked"] else None
    # (2) the plain path, one request at a time
    polys = {}
    t0 = time.perf_counter()
    tp_plain = 0.0
    for (ts, k, beta) in burst:
        w = pool[k]
        out = ring.view(0, (w.T, G[k]))
        if beta is None or k not in polys:
            if k in polys:
                polys[k].close()
            polys[k] = pe.Poly.from_workload(w)
        polys[k].run(w.beta if beta is None else beta, w.T, 1, out=out)
        tp_plain += w.s * w.T
    t_plain = time.perf_counter() - t0
    for p in polys.values():
        p.close()
    # (3) Poisson stream below saturation: 0.7x the burst's request rate unless a rate is given
    capacity = len(burst) / t_burst
    rate = args.serve_rate if args.serve_rate > 0 else 0.7 * capacity
    reqs = wl.served_requests(seed=wl.SEED_SERVE, rate=rate, duration=args.serve_seconds, pool=pool)
    srv = pe.Server(mem_cap_bytes=40 << 30, streams=args.serve_streams, max_epoch_jobs=args.serve_epoch_jobs)
    submit_s[0] = 0.0
    t_pois, tp_pois, chk_pois = drive(reqs, srv, True)
    st_pois = srv.stats()
    srv.close()
    return {
        "workload": f"requests from the {len(pool)}-polynomial batched mixture, 30% reuse a resident "
                    "polynomial at a new beta, 40 GB resident cap",
        "burst": {"requests": len(burst), "seconds": t_burst, "term_points_per_s": tp_burst / t_burst,
                  "requests_per_s": capacity, "p50_ms": st_burst["p50_ms"],
                  "p99_ms": st_burst["p99_ms"], "epochs": st_burst["epochs"], "rejected": st_burst["rejected"],
                  "requests_per_s_of_three_bursts": burst_rates, "oracle_check": chk_burst},
        "plain_per_request": {"requests": len(burst), "seconds": t_plain, "term_points_per_s": tp_plain / t_plain,
                              "requests_per_s": len(burst) / t_plain},
        "served_over_plain": (tp_burst / t_burst) / (tp_plain / t_plain),
        "poisson": {"rate_per_s": rate, "rate_over_burst_capacity": rate / capacity,
                    "seconds": args.serve_seconds, "requests": len(reqs),
                    "completed": st_pois["completed"], "achieved_requests_per_s": len(reqs) / t_pois,
                    "goodput_term_points_per_s": tp_pois / t_pois, "p50_ms": st_pois["p50_ms"],
                    "p99_ms": st_pois["p99_ms"], "max_ms": st_pois["max_ms"], "rejected": st_pois["rejected"],
                    "evictions": st_pois["evictions"], "epochs": st_pois["epochs"], "oracle_check": chk_pois,
                    "host_seconds": {"client_submit": submit_s[0], "worker_upload": st_pois["upload_s"],
                                     "worker_plan": st_pois["plan_s"], "worker_launch": st_pois["launch_s"],
                                     "worker_finish": st_pois["finish_s"], "gpu_busy": st_pois["busy_s"]}},
    }


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batched":
        run_batched(args)
    elif args.config == "served":
        print(json.dumps({"metric": "served", **run_served(args)}), flush=True)
    elif args.config == "interp":
        import torch
        import paper_2004_11571_gb300 as pe
        torch.cuda.set_device(0)
        clocks = ClockSampler(0)
        clocks.start()
        res = bench_interp(pe, torch, 2070.0, reps=max(args.steps, 1))
        clk = clocks.stop()
        mhz = clk["sm_mhz"] or 2070.0
        for c in res:                      # peaks at the sampled clock instead of the nominal one
            r = c["roofline"]
            r["peak"] *= mhz / 2070.0
            for k in ("frac", "tree_frac", "correlation_frac"):
                if r.get(k) is not None:
                    r[k] *= 2070.0 / mhz
        print(json.dumps({"metric": "interpolation from images (transposed Vandermonde solves)",
                          "value": res[0]["terms_per_s"], "unit": "terms recovered/s", "clocks": clk,
                          "cases": res}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
