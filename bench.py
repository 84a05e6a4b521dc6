"""Benchmark: Wang-Landau move attempts per second on the micromagnetic lines
of the 64x64 periodic square Ising lattice (arXiv:1302.2320), one GB300.

A step is one pass of the whole path over one fresh batch: walker
initialisation for every line l = 0..N/2 (new seed per step), the walk of every
line for a fixed move budget (spin-exchange proposals, Eq. 3 acceptance, ln g
and histogram updates, flatness checks every C moves, stage steps ln f -> ln f
/ 4), and the FP64 assembly of ln g_kl (Eq. 4).  Deterministic mode: the timed
launch shape is the one whose trajectories the GPU tests compare bit for bit
with the CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank walks its own
surface (seed offset by rank): per-GPU work is fixed, scaling is weak, and the
only cross-rank traffic is the barrier and the max-over-ranks of the timings.

Other modes, each printing its own JSON line: --converge L (time to ln f_min
of a whole surface; for square L with stored exact values also the surface
summed over l against the exact zero-field g_k, as in Fig. 5), --serve N
(Poisson request stream through the serving loop), --accuracy (12x12 against
the exact surface), --L (the benchmark on another square lattice).
"""
from __future__ import annotations

import argparse
import math
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LATTICE, L = "square", 64
LN_F_MIN = 1e-6
FLATNESS = 0.8
CHECK_INTERVAL = 16384
MOVES_PER_LINE = 1 << 22
# Algorithmic work of one move attempt on the square lattice (the method's own
# arithmetic, not the instructions a kernel happens to issue):
#   Philox4x32-10: 10 rounds x (2 32x32->64 products + 2 three-input xors)
#   list picks: 2 products;  Eq. 3 threshold: 1 product + ~6 ops
#   change of k: 8 neighbour sites (~2 ops each), 8 spin bits (2 ops each), 8 sums, 4 compares
#   bookkeeping: ~4 ops
MUL_OPS_PER_MOVE = 23       # 32x32->64 products
ALU_OPS_PER_MOVE = 113      # logic / add / shift / compare
INT_OPS_PER_MOVE = MUL_OPS_PER_MOVE + ALU_OPS_PER_MOVE
# random shared-memory accesses per move: 2 list entries, 2z = 8 neighbour spin
# words, 1 ln g; per accepted move 2 list writes, 2 spin updates, 1 ln g write
SMEM_ACCESSES_PER_MOVE, SMEM_ACCESSES_PER_ACCEPT = 11, 5


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


KERNEL_SOURCES = ["paper_1302_2320_gb300/csrc/wl_walk.cuh", "paper_1302_2320_gb300/csrc/wl_device.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "walk_kernel_L64_traffic.txt")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def walker_traffic(moves_per_line: int, mapping: int):
    """DRAM bytes of one benchmark walk launch from the committed ncu summary,
    or None when it was taken on another launch shape or an older kernel."""
    try:
        fields = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if (fields.get("kernel_source_sha256") == kernel_source_hash()
                and int(fields.get("moves_per_line", -1)) == moves_per_line
                and int(fields.get("mapping", -1)) == mapping):
            return int(fields["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def sum_over_lines(lines, N: int, kstep: int = 2):
    """ln g_k = ln sum_l g_kl from the assembled lines l = 0..N/2 (ln g_kl over
    k = 0, kstep, ...; -inf where unvisited), lines l > N/2 by the l <-> N - l
    mirror: the sum the paper compares with the exact zero-field g_k (Sec. 4,
    Fig. 5)."""
    import numpy as np
    width = max(len(v) for v in lines)
    mat = np.full((N + 1, width), -np.inf)
    for ell, v in enumerate(lines):
        mat[ell, :len(v)] = v
        mat[N - ell, :len(v)] = v
    top = mat.max(axis=0)
    out = np.full(width, -np.inf)
    fin = np.isfinite(top)
    out[fin] = top[fin] + np.log(np.exp(mat[:, fin] - top[fin]).sum(axis=0))
    full = np.full((width - 1) * kstep + 1, -np.inf)
    full[::kstep] = out
    return full


def exact_gk_comparison(lng_k, path: str, NB: int):
    """Differences between a summed surface and the stored exact zero-field
    ln g_k (columns k, ln g_k): |d ln g_k| and |dS_k| with S_k = ln g_k / N_B
    (the quantity of Fig. 5), over every k with g_k > 0 and over the inner k
    (without the two lowest and two highest energies of the spectrum)."""
    import numpy as np
    ex = np.full(NB + 1, -np.inf)
    for k, v in np.loadtxt(path, ndmin=2):
        ex[int(k)] = v
    got = np.full(NB + 1, -np.inf)
    got[:min(len(lng_k), NB + 1)] = lng_k[:NB + 1]
    ks = np.nonzero(np.isfinite(ex))[0]
    missing = int((~np.isfinite(got[ks])).sum())
    ks = ks[np.isfinite(got[ks])]
    d = np.abs(got[ks] - ex[ks])
    inner = d[2:-2] if d.size > 4 else d
    return {"exact": os.path.relpath(path, ROOT), "k_compared": int(ks.size), "k_missing": missing,
            "max_abs_dlng": float(d.max()), "mean_abs_dlng": float(d.mean()),
            "max_abs_dS": float(d.max() / NB), "mean_abs_dS": float(d.mean() / NB),
            "inner_max_abs_dS": float(inner.max() / NB),
            "worst_k": int(ks[int(np.argmax(d))])}


def line_moves_summary(moves, N: int):
    """Moves each line took to reach ln f_min (its move counter t), lines
    l = 0..N/2: quantiles, a log2 histogram and the four lines the paper walks
    individually (l = N/8, N/4, 3N/8, N/2)."""
    import numpy as np
    t = np.asarray(moves, dtype=np.int64)
    walked = t[t > 0]
    q = np.quantile(walked, [0.5, 0.9, 0.99, 1.0]) if walked.size else [0, 0, 0, 0]
    hist = {}
    for v in walked:
        b = int(v).bit_length() - 1
        hist[f"2^{b}"] = hist.get(f"2^{b}", 0) + 1
    return {"lines_walked": int(walked.size),
            "p50": int(q[0]), "p90": int(q[1]), "p99": int(q[2]), "max": int(q[3]),
            "argmax_l": int(np.argmax(t)) if t.size else 0,
            "log2_histogram": dict(sorted(hist.items(), key=lambda kv: int(kv[0][2:]))),
            "paper_lines": {str(l): int(t[l]) for l in (N // 8, N // 4, 3 * N // 8, N // 2)
                            if l < t.size}}


def parse_line(text: str, N: int) -> int:
    """A line given as an integer or as [a*]N[//b] (e.g. N//8, 3*N//8, N//2)."""
    m = re.fullmatch(r"\s*(?:(\d+)\s*\*\s*)?N\s*(?://\s*(\d+))?\s*", text)
    if m:
        return int(m.group(1) or 1) * N // int(m.group(2) or 1)
    return int(text)


def converge_on_cpu(lat, Lc, ells, args, gpu_moves, to_gpu_moves=False):
    """The same surface walked to ln f_min by the oracle (deterministic, as it
    stands) on every host core, one line per thread, largest lines first; the
    chain is the GPU's, so each line's move count must match.  With
    to_gpu_moves each line is walked only as far as the GPU got (a run that hit
    its time limit): the time the host cores need for the same progress."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    code = oracle.LATTICE_NAMES[lat]
    threads = os.cpu_count() or 1
    ells = sorted(ells, key=lambda l: -oracle.line_nbins(code, Lc, l))

    def one(ell):
        st = oracle.run_line(code, Lc, ell, 1, args.ln_f_min, args.check_interval,
                             int(FLATNESS * 1000), gpu_moves[ell] if to_gpu_moves else 2**62, 0,
                             same_f_resets=args.same_f_resets)
        return ell, st.t

    def one_c(ell):
        Cl = max(args.check_interval, args.check_per_bin * oracle.line_nbins(code, Lc, ell))
        st = oracle.run_line(code, Lc, ell, 1, args.ln_f_min, Cl,
                             int(FLATNESS * 1000), gpu_moves[ell] if to_gpu_moves else 2**62, 0,
                             same_f_resets=args.same_f_resets)
        return ell, st.t
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        res = dict(ex.map(one_c if args.check_per_bin else one, ells))
    sec = time.perf_counter() - t0
    same = all(res[l] == gpu_moves[l] for l in ells)
    return {"seconds": sec, "cores": threads, "kind": "oracle", "moves": int(sum(res.values())),
            "same_moves_per_line_as_gpu": bool(same),
            "sample": ("every walked line to the GPU's move count (same chain), one thread per line"
                       if to_gpu_moves else "every walked line to ln f_min, one thread per line")}


def run_converge(args):
    """Time to ln f_min: one whole surface walked until every line converged
    (or the time limit), reported as its own JSON line.  Under torchrun the
    surface is split by lines (LPT on bins^2, paper_1302_2320_gb300.shard):
    each rank walks its share on its GPU, the assembled lines are gathered on
    rank 0, and the time is the maximum over ranks."""
    import paper_1302_2320_gb300 as wl
    from paper_1302_2320_gb300 import shard
    world, rank, local = _dist()
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
        torch.cuda.set_device(local)
    wl.build()
    lat, Lc = args.lattice, args.converge
    h = wl.Handle(lat, Lc, deterministic=1, check_interval=args.check_interval, seed=1,
                  mapping=args.mapping, timeout_ms=int(args.time_limit * 1000),
                  same_f_resets=args.same_f_resets, form=args.form)
    if args.check_per_bin:
        h.set_option("check_per_bin", args.check_per_bin)
    if args.move_budget:
        h.set_option("move_budget", args.move_budget)
    if args.slice_ms > 0 and args.form == 0:
        # slices end by device time: no line waits for a slower one at a slice end
        h.set_option("slice_ms", args.slice_ms)
        h.set_option("slice_moves", 1 << 40)
    lo, hi = 0, h.N // 2
    if args.lines:
        lo, hi = (int(x) for x in args.lines.split(":"))
    ells = list(range(lo, hi + 1))
    if args.line_set:
        N = h.N
        ells = sorted({parse_line(x, N) for x in args.line_set.split(",")})
        lo, hi = ells[0], ells[-1]
    ells_all = list(ells)
    if world > 1:
        costs = {l: c for l, c in shard.handle_costs(h).items() if l in set(ells_all)}
        ells = shard.lpt_partition(costs, world)[rank]
    h.select_lines(ells)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    rc = h.run(args.ln_f_min, FLATNESS, allow=(wl.WL_OK, wl.WL_ETIMEOUT, wl.WL_ENOTCONVERGED))
    sec = time.perf_counter() - t0
    st = h.stats()
    moves = [0] * (h.N // 2 + 1)
    stages = {}
    for ell in ells:
        sc = h.line_state(ell)["sc"]
        moves[ell] = int(sc[1])
        stages[ell] = int(sc[3])
    lines = None
    if rc == wl.WL_OK or world == 1:
        h.assemble()
        lines = {ell: h.get_lng(ell) for ell in ells}
    if dist:
        import torch
        agg = torch.tensor([sec, st["moves"], st["lines_converged"], st["lines"], st["accepts"],
                            int(rc != wl.WL_OK)], dtype=torch.float64)
        mx = agg.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(agg, op=dist.ReduceOp.SUM)
        mv = torch.tensor(moves, dtype=torch.int64)
        dist.all_reduce(mv, op=dist.ReduceOp.SUM)
        moves = mv.tolist()
        sec = float(mx[0])
        st = dict(st, moves=int(agg[1]), lines_converged=int(agg[2]), lines=int(agg[3]),
                  accepts=int(agg[4]))
        failed = int(mx[5])
        rc = wl.WL_OK if not failed else wl.WL_ETIMEOUT
        lines = shard.gather_lines(dist, lines or {}) if not failed else None
        if rank != 0:
            h.close()
            dist.destroy_process_group()
            return 0
    line = {"mode": "time_to_ln_f_min", "lattice": lat, "L": Lc, "N": h.N, "lines": st["lines"],
            "ln_f_min": args.ln_f_min, "check_interval": args.check_interval,
            "check_per_bin": args.check_per_bin,
            "same_f_resets": args.same_f_resets, "n_gpus": world,
            "status": {wl.WL_OK: "converged", wl.WL_ETIMEOUT: "time limit"}.get(rc, "move budget"),
            "walk_ms": st["walk_ms"],
            "seconds": sec, "lines_converged": st["lines_converged"],
            "min_stage": st["min_stage"], "max_stage": st["max_stage"], "moves": st["moves"],
            "moves_per_s": st["moves"] / sec, "mapping": st["mapping"],
            "accept_rate": st["accepts"] / max(st["moves"], 1)}
    if world > 1:
        line["parallelism"] = f"lines sharded over {world} ranks (LPT on bins^2), gathered on rank 0"
    line["lines_walked"] = [lo, hi] if not args.line_set else ells
    line["form"] = "persistent" if args.form == 0 else "one launch per line"
    line["slices"] = (f"{args.slice_ms} ms of device time" if args.slice_ms > 0 and args.form == 0
                      else f"{h.get_option('slice_moves')} moves per line")
    if len(ells) <= 16:
        line["per_line"] = {str(l): {"moves": moves[l], "stage": stages.get(l)} for l in ells}
    line["moves_to_converge"] = line_moves_summary(moves, h.N)
    if args.cpu_converge and (rc == wl.WL_OK or len(ells_all) <= (os.cpu_count() or 1)):
        line["cpu_oracle"] = converge_on_cpu(lat, Lc, ells_all, args, moves, to_gpu_moves=rc != wl.WL_OK)
        line["gpu_speedup_over_cpu"] = line["cpu_oracle"]["seconds"] / sec
    exact = os.path.join(ROOT, "tests", "golden", f"square_L{Lc}_gk_exact.txt")
    if (lat == "square" and os.path.exists(exact) and (lo, hi) == (0, h.N // 2)
            and rc == wl.WL_OK and lines is not None):
        surface = [lines[ell] for ell in range(h.N // 2 + 1)]
        line["sum_over_lines_vs_exact_gk"] = exact_gk_comparison(
            sum_over_lines(surface, h.N), exact, 2 * h.N)
    print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()
    return 0


SERVE_MIX = [("square", 16), ("square", 24), ("square", 32), ("square", 48),
             ("triangular", 16), ("triangular", 32), ("cubic", 6), ("cubic", 8)]
SERVE_MIX_SMALL = [("square", 16), ("triangular", 16), ("cubic", 6)]


def run_serve(args):
    """Serving: a Poisson stream of DOS requests through the continuous-batching
    loop; p50/p99 time-to-DOS (submit -> assembled surface in host memory) and
    aggregate moves/s."""
    import numpy as np
    import paper_1302_2320_gb300 as wl
    wl.build()
    rng = np.random.default_rng(2024)
    n = args.serve
    mix = SERVE_MIX if args.serve_mix == "full" else SERVE_MIX_SMALL
    u_choices = [float(x) for x in args.serve_u.split(",")]
    kinds = [mix[i] for i in rng.integers(0, len(mix), n)]
    us = rng.choice(u_choices, n)
    budget = args.serve_moves if args.serve_moves > 0 else 2**62      # 0: walk to ln f_min
    # calibrate: each lattice alone (all at once, each on its own stream) at the
    # mix's mean ln f_min -> mean service time
    srv = wl.Server(hbm_budget=args.hbm_budget, max_active=args.max_active)
    solo = {}
    cal = {}
    for lat, L in mix:
        cal[(lat, L)] = (time.perf_counter(), srv.submit(lat, L, seed=7, ln_f_min=u_choices[0],
                                                         check_interval=args.check_interval,
                                                         move_budget=budget))
    for key, (t0, rid) in cal.items():
        srv.wait(rid)
        info = srv.info(rid)
        solo[key] = info["finish_s"] - info["start_s"]
        srv.release(rid)
    # service time of a finer ln f_min, for the arrival rate only: sqrt of the ratio
    slow = {u: math.sqrt(u_choices[0] / u) for u in u_choices}
    mean_solo = float(np.mean([solo[k] * slow[float(u)] for k, u in zip(kinds, us)]))
    lam = args.load * args.max_active / mean_solo          # requests per second
    gaps = rng.exponential(1.0 / lam, n)
    ids, t_start = [], time.perf_counter()
    t_next = t_start
    for x in range(n):
        t_next += gaps[x]
        while time.perf_counter() < t_next:
            time.sleep(min(0.002, max(0.0, t_next - time.perf_counter())))
        lat, L = kinds[x]
        ids.append(srv.submit(lat, L, seed=100 + x, ln_f_min=float(us[x]),
                              check_interval=args.check_interval, move_budget=budget))
    lat_s, moves, fails, rcs = [], 0, 0, []
    for rid in ids:
        rc = srv.wait(rid)
        rcs.append(rc)
        info = srv.info(rid)
        fails += info["state"] != 2
        lat_s.append(info["finish_s"] - info["submit_s"])
        moves += info["moves"]
        srv.release(rid)
    span = time.perf_counter() - t_start
    srv.close()
    lat_s = np.array(lat_s)
    line = {"mode": "serving", "requests": n, "failed": int(fails),
            "p50_time_to_dos_s": float(np.percentile(lat_s, 50)),
            "p99_time_to_dos_s": float(np.percentile(lat_s, 99)),
            "mean_time_to_dos_s": float(lat_s.mean()), "makespan_s": span,
            "aggregate_moves_per_s": moves / span, "offered_load": args.load,
            "arrival_rate_per_s": lam, "max_active": args.max_active, "hbm_budget": args.hbm_budget,
            "move_budget_per_line": budget if args.serve_moves > 0 else None,
            "converged_requests": int(sum(1 for r in rcs if r == wl.WL_OK)),
            "check_interval": args.check_interval,
            "mix": [f"{lat} L={L}" for lat, L in mix], "ln_f_min": u_choices,
            "p50_by_lattice_s": {f"{lat} L={L}": float(np.percentile(
                [t for t, k in zip(lat_s, kinds) if k == (lat, L)] or [0.0], 50)) for lat, L in mix},
            "solo_seconds": {f"{lat} L={L}": v for (lat, L), v in solo.items()}}
    print(json.dumps(line), flush=True)
    return 0


def run_accuracy(args):
    """Accuracy of a whole surface against the exact transfer-matrix values
    (tests/golden/square_L{L}_exact.txt, L = 6, 8 or 12): seeds walked
    concurrently, production mode, to ln f_min; mean and max |d ln g_kl| over
    the inner bins and over the two ends of each line's spectrum (the lowest and
    highest k, where the paper also sees the largest deviations)."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    import paper_1302_2320_gb300 as wl
    wl.build()
    La = args.accuracy_L
    N = La * La
    exact = {}
    for ell, k, lg in np.loadtxt(os.path.join(ROOT, "tests", "golden", f"square_L{La}_exact.txt")):
        exact.setdefault(int(ell), {})[int(k)] = float(lg)

    def one(seed):
        h = wl.Handle("square", La, seed=seed, deterministic=0, check_interval=args.check_interval,
                      timeout_ms=int(args.time_limit * 1000), same_f_resets=args.same_f_resets)
        t0 = time.perf_counter()
        rc = h.run(args.ln_f_min, FLATNESS, allow=(wl.WL_OK, wl.WL_ETIMEOUT))
        sec = time.perf_counter() - t0
        h.assemble()
        out = rc, sec, h.stats()["moves"], [h.get_lng(ell) for ell in range(N // 2 + 1)]
        h.close()
        return out

    t0 = time.perf_counter()
    with ThreadPoolExecutor(args.seeds) as ex:
        res = list(ex.map(one, range(1, args.seeds + 1)))
    inner, ends = [], []
    for rc, _, _, lines in res:
        for ell in range(N // 2 + 1):
            ks = sorted(exact[ell])
            for k in ks:
                d = abs(lines[ell][k // 2] - exact[ell][k])
                (ends if k in (ks[0], ks[-1]) and len(ks) > 2 else inner).append(d)
    inner, ends = np.array(inner), np.array(ends)
    print(json.dumps({"mode": f"accuracy_square_L{La}", "ln_f_min": args.ln_f_min, "seeds": args.seeds,
                      "check_interval": args.check_interval, "production": True,
                      "same_f_resets": args.same_f_resets,
                      "converged_seeds": sum(r[0] == wl.WL_OK for r in res),
                      "seconds_per_seed": [r[1] for r in res], "wall_s": time.perf_counter() - t0,
                      "moves_per_seed": [r[2] for r in res],
                      "inner_mean": float(inner.mean()), "inner_max": float(inner.max()),
                      "ends_mean": float(ends.mean()), "ends_max": float(ends.max()),
                      "all_mean": float(np.concatenate([inner, ends]).mean()),
                      "tolerance": {"mean": 0.02, "max": 0.1},
                      "inner_within_tolerance": bool(inner.mean() <= 0.02 and inner.max() <= 0.1)}),
          flush=True)
    return 0


def rank_seed(rank: int) -> int:
    """Each rank walks its own surface replica: seeds never overlap across ranks."""
    return 1000 * (rank + 1)


def combine_ranks(dist, total_ms, e2e_sec, moves, e2e_moves, device=None):
    """Max over ranks of the timings, sum over ranks of the work (moves)."""
    import torch
    if not dist:
        return float(total_ms), float(e2e_sec), float(moves), float(e2e_moves)
    mx = torch.tensor([total_ms, e2e_sec], dtype=torch.float64, device=device)
    sm = torch.tensor([moves, e2e_moves], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(mx[1]), float(sm[0]), float(sm[1])


def _cpu_sample(ells, budget, seed, threads, Lc=L):
    """Oracle (deterministic mode, as it stands) on a bounded sample of lines."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    def one(ell):
        st = oracle.run_line(oracle.SQUARE, Lc, ell, seed, LN_F_MIN, CHECK_INTERVAL,
                             int(FLATNESS * 1000), budget, 0)
        return st.t
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        moves = sum(ex.map(one, ells))
    return moves, time.perf_counter() - t0


def run_reference(args):
    """Reference arm: the CPU oracle on this host's cores, walking every line of
    the benchmark surface.  The walks persist across steps (initialised in the
    first warm-up step), and each step advances every line by the same number
    of moves, so a step times the walk itself, bounded in size."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    N = L * L
    ells = list(range(1, N // 2 + 1))          # every walking line of the surface
    per_step = 1 << 17                          # moves per line per step (bounded sample)
    states = {}

    def advance(ell):
        st = states.get(ell)
        t0 = st.t if st is not None else 0
        st = oracle.run_line(oracle.SQUARE, L, ell, 1, LN_F_MIN, CHECK_INTERVAL,
                             int(FLATNESS * 1000), t0 + per_step, 0, state=st)
        states[ell] = st
        return st.t - t0

    tot_moves, tot_sec = 0, 0.0
    with ThreadPoolExecutor(threads) as ex:
        for s in range(max(args.warmup, 1) + args.steps):
            t0 = time.perf_counter()
            moves = sum(ex.map(advance, ells))
            sec = time.perf_counter() - t0
            if s >= max(args.warmup, 1):
                tot_moves += moves
                tot_sec += sec
    value = tot_moves / tot_sec
    line = {"impl": "reference", "metric": "WL move attempts/sec", "value": value,
            "unit": "moves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot_sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"square L={L} periodic, {N // 2 + 1} lines, ln_f_min={LN_F_MIN}, "
                       f"C={CHECK_INTERVAL}, deterministic; every line walked on by {per_step} "
                       f"moves per step (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": "moves/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} moves x {len(ells)} lines per step, walks "
                                       f"continued across steps"},
            "e2e": {"value": value, "unit": "moves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_1302_2320_gb300 as wl

    world, rank, local = _dist()
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    torch.cuda.set_device(local)
    wl.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    L = args.L
    N = L * L

    h = wl.Handle(LATTICE, L, deterministic=1, check_interval=CHECK_INTERVAL,
                  move_budget=args.moves_per_line, slice_moves=args.moves_per_line,
                  mapping=args.mapping, form=args.form, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def step(seed):
        h.reset()
        h.set_option("seed", seed)
        h.run(LN_F_MIN, FLATNESS)
        h.assemble()

    seed0 = rank_seed(rank)
    for w in range(max(args.warmup, 1)):
        step(seed0 + w)
    mapping = args.mapping
    if mapping == 0:
        # the lane-count tuner times one candidate per step: finish it, then fix its choice
        extra = 0
        while h.get_option("tuned_mapping") == 0 and extra < 3:
            step(seed0 + 50 + extra)
            extra += 1
        mapping = h.get_option("tuned_mapping") or h.stats()["mapping"]
    h.set_option("mapping", mapping)            # fixed for the timed steps

    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    moves = launches = accepts = batches = 0
    walk_ms = 0.0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.fill_(s)                           # evict the previous step's state from L2
        ev[s][0].record(stream)
        step(seed0 + 100 + s)
        ev[s][1].record(stream)
        st = h.stats()
        moves += st["moves"]
        accepts += st["accepts"]
        batches += st["batches"]
        walk_ms += st["walk_ms"]
        launches += st["launches"] + 1           # + the assembly kernel
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)

    # end to end through the C ABI with host buffers: one pass per step including
    # the device->host copy of the assembled surface into pinned host memory
    surf_n = h.get_option("bins")
    host = torch.empty(surf_n, dtype=torch.float64, pin_memory=True).numpy()
    e2e_moves, e2e_sec = 0, 0.0
    for s in range(args.steps):
        flush.fill_(s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(seed0 + 200 + s)
        h.get_surface(host)
        e2e_sec += time.perf_counter() - t0
        e2e_moves += h.stats()["moves"]
    clk = clocks.stop() if rank == 0 else None

    total_ms, e2e_sec, moves, e2e_moves = combine_ranks(dist, total_ms, e2e_sec, moves, e2e_moves, dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    value = moves / (total_ms / 1000.0)
    per_rank_moves = moves / world
    walk_s = walk_ms / 1000.0
    walk_rate = per_rank_moves / walk_s                  # moves/s of the walker kernel alone
    rates = wl.wl_measure_peaks()                        # this GPU's integer and random-access rates
    # integer issue: the mix's time per move at the measured per-class rates
    t_move = MUL_OPS_PER_MOVE / rates["mulwide_ops_per_s"] + ALU_OPS_PER_MOVE / rates["iadd3_ops_per_s"]
    alu_peak = INT_OPS_PER_MOVE / t_move / 1e12                              # Tops/s
    achieved = walk_rate * INT_OPS_PER_MOVE / 1e12
    acc_rate = accepts / max(moves, 1)
    smem_per_move = SMEM_ACCESSES_PER_MOVE + SMEM_ACCESSES_PER_ACCEPT * acc_rate
    traffic = walker_traffic(args.moves_per_line, mapping) if L == 64 else None

    cpu = None
    if not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        ells = [N // 8, N // 4, 3 * N // 8, N // 2]
        ells = (ells * ((threads + 3) // 4))[:max(threads, 4)]
        m, sec = _cpu_sample(ells, args.cpu_moves, 1, threads, L)
        cpu = {"value": m / sec, "unit": "moves/s", "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_moves} moves on each of {len(ells)} walks of lines "
                         f"N/8, N/4, 3N/8, N/2 (deterministic, C={CHECK_INTERVAL}), {sec:.1f} s"}

    bytes_d2h = surf_n * 8 + 64
    bytes_h2d = 4 * (N // 2 + 1) + 4096 * 4
    line = {
        "metric": "WL move attempts/sec", "value": value, "unit": "moves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"square L={L} periodic, {N // 2 + 1} lines (l<=N/2), "
                               f"ln_f_min={LN_F_MIN}, C={CHECK_INTERVAL}, "
                               f"{args.moves_per_line} moves/line/step, deterministic",
                   "lattice": LATTICE, "L": L, "lines": N // 2 + 1, "ln_f_min": LN_F_MIN,
                   "check_interval": CHECK_INTERVAL, "moves_per_line": args.moves_per_line,
                   "form": "persistent" if args.form == 0 else "one launch per line", "mapping": mapping,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "kernel": "walk_kernel", "ops_per_move": INT_OPS_PER_MOVE,
                     "peak_basis": (f"measured on this GPU by wl_measure_peaks: {MUL_OPS_PER_MOVE} "
                                    f"32x32->64 products at {rates['mulwide_ops_per_s']:.3g}/s plus "
                                    f"{ALU_OPS_PER_MOVE} add/logic ops at {rates['iadd3_ops_per_s']:.3g}/s "
                                    f"per move"),
                     "random_access": {"level": "shared memory (lists, spins, ln g window)",
                                       "accesses_per_move": smem_per_move,
                                       "achieved": walk_rate * smem_per_move,
                                       "peak": rates["smem_words_per_s"], "unit": "accesses/s",
                                       "frac": walk_rate * smem_per_move / rates["smem_words_per_s"],
                                       "peak_basis": "random 4-byte shared-memory reads, all SMs (wl_measure_peaks)"},
                     "measured_rates": rates},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_moves / e2e_sec, "unit": "moves/s", "h2d_bytes_per_step": bytes_h2d,
                "d2h_bytes_per_step": bytes_d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "walk_ms_per_step": walk_ms / args.steps,
        "accept_rate": acc_rate, "moves_per_batch": moves / max(batches, 1),
    }
    print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--moves-per-line", type=int, default=MOVES_PER_LINE)
    ap.add_argument("--L", type=int, default=L, help="square lattice size (default 64)")
    ap.add_argument("--mapping", type=int, default=0)
    ap.add_argument("--cpu-moves", type=int, default=150_000_000)
    ap.add_argument("--form", type=int, default=0, help="0 persistent batched, 1 one launch per line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--converge", type=int, default=0,
                    help="walk a whole LxL surface to ln f_min and report the time instead")
    ap.add_argument("--lattice", default="square")
    ap.add_argument("--ln-f-min", type=float, default=LN_F_MIN)
    ap.add_argument("--check-interval", type=int, default=CHECK_INTERVAL)
    ap.add_argument("--time-limit", type=float, default=600.0, help="seconds, --converge only")
    ap.add_argument("--lines", default="", help="A:B, walk only lines A..B (--converge only)")
    ap.add_argument("--line-set", default="",
                    help="--converge: comma-separated lines, expressions of N allowed (e.g. N//8,N//2)")
    ap.add_argument("--same-f-resets", type=int, default=0, help="extra same-f resets per stage")
    ap.add_argument("--slice-ms", type=int, default=100,
                    help="--converge: slices end after this much device time (0: by moves)")
    ap.add_argument("--move-budget", type=int, default=0, help="--converge: per-line move cap (0: none)")
    ap.add_argument("--check-per-bin", type=int, default=0,
                    help="--converge: a line of n bins checks flatness every max(C, c n) moves")
    ap.add_argument("--cpu-converge", action="store_true",
                    help="--converge: also walk the surface with the oracle on every host core")
    ap.add_argument("--serve", type=int, default=0, help="run the serving benchmark with N requests")
    ap.add_argument("--serve-moves", type=int, default=1 << 22,
                    help="per-line move budget of a request (0: walk to ln f_min)")
    ap.add_argument("--serve-mix", choices=["full", "small"], default="full")
    ap.add_argument("--serve-u", default="1e-6,1e-7", help="ln f_min values drawn per request")
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--hbm-budget", type=int, default=32 << 30)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--accuracy", action="store_true", help="accuracy against the exact surface")
    ap.add_argument("--accuracy-L", type=int, default=12, choices=[6, 8, 12])
    ap.add_argument("--seeds", type=int, default=8)
    args = ap.parse_args()
    if args.accuracy:
        return run_accuracy(args)
    if args.serve:
        return run_serve(args)
    if args.converge:
        return run_converge(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
