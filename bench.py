"""Benchmark: batch-dynamic SpGEMM on one GB300 (and N replicas).

Workload (the stencil configuration): 7-point stencil matrix on a 128^3 grid
(n = 2,097,152, nnz(A) = 14,581,760), C = A A in (+,.) on double
(nnz(C) = 51,742,208); each step applies one batch of 10^4 mixed updates
(inserts / deletes / value changes within two grid hops, 0.07% of nnz(A))
through the C ABI and brings C up to date.  Inputs are resident in HBM when
a timed step starts; L2 is flushed (256 MiB write) before every timed step.

Printed JSON line (rank 0): value = batches/s over all ranks (each rank a
replica on its own GPU: "replicas only", no data-path collective), the
per-batch latency, the full static GPU recompute and the speedup over it,
the recompute kernels' HBM roofline, an end-to-end number through the
public API with host buffers, the oracle's CPU baseline, and clocks.

--impl reference runs the CPU oracle (the deliberately slow reference) on
the same workload and metric.
"""

from __future__ import annotations

import argparse
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

METRIC = "dynamic batch latency & speedup vs static GPU recompute; recompute HBM GB/s"
GRID = 128
BATCH = 10000


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes (read + write) of the numeric stage's kernels in one step of a
# workload, from the ncu capture summarised in
# profiles/numeric_stage_dram_stencil128.md (valid while those kernels are
# unchanged); None where no capture exists.
NUMERIC_TRAFFIC = {"stencil": 82590208}


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def slowest_rank_ms(dist, local_ms, device):
    """The largest of the ranks' timed totals (every rank timed the same
    number of steps); the job's rate is all ranks' units over this time."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_units(count, rank, world):
    """Independent units (instances) of rank `rank` out of `world`: every
    world-th unit, so uneven sizes spread evenly; no unit is shared."""
    return list(range(rank, count, world))


class StencilWorkload:
    """128^3 7-point stencil, C = A A in (+,.) f64, mixed batches within two
    grid hops (inserts / deletes / value changes, a third each)."""
    name = "stencil"
    batch = BATCH
    sweep = (1, 100, 1000, 10000, 100000, 1000000)
    vsize, dtype = 8, "f64"

    def __init__(self):
        self.describe = "stencil 128^3 7-point, C = A A (+,.) f64, batches of 10^4 mixed updates"
        self.unit = "batches/s (10^4-update batches)"

    def operands(self):
        from workloads import stencil7
        return stencil7(GRID, GRID, GRID, seed=1), None

    def batches(self, count, seed0, nupd=None):
        from workloads import stencil_batch
        return [stencil_batch(GRID, GRID, GRID, nupd or self.batch, seed=seed0 + i) for i in range(count)]


class Rmat20Workload:
    """R-MAT scale 20, edge factor 16, Graph500 parameters, symmetrised,
    int32 weights U[1,100]; B is n x 256 with 1% density, int32 U[1,100];
    C = A B in (min,+) (multi-source path relaxation); batches of undirected
    edge insertions (held-out edges) and deletions of A, half each."""
    name = "rmat20"
    batch = 1000
    sweep = (100, 1000, 10000, 100000)
    vsize, dtype = 4, "i32"

    def __init__(self):
        self.describe = ("R-MAT scale 20 ef 16 (0.57,0.19,0.19,0.05) symmetrised, C = A B (min,+) i32 with B n x 256 "
                         "at 1%, batches of 10^3 undirected edge insertions/deletions of A")
        self.unit = "batches/s (10^3-edge batches)"
        self._A = self._held = None
        self._streams = {}

    def operands(self):
        from workloads import MIN_PLUS_I32, bernoulli_sparse, rmat_symmetric
        self._A, self._held = rmat_symmetric(20, 16, (0.57, 0.19, 0.19, 0.05), seed=3, kind=MIN_PLUS_I32,
                                             holdout=400000)
        B = bernoulli_sparse(1 << 20, 256, 0.01, seed=3, kind=MIN_PLUS_I32)
        return self._A, B

    def batches(self, count, seed0, nupd=None):
        from workloads import EdgeStream
        es = self._streams.get(seed0)
        if es is None:
            es = self._streams[seed0] = EdgeStream(self._A, self._held, seed0)
        return [es.batch(nupd or self.batch) for _ in range(count)]


class Rmat21Workload(Rmat20Workload):
    """R-MAT scale 21, edge factor 8, (0.45, 0.15, 0.15, 0.25), symmetrised,
    (+,.) f64 U(0,1), C = A A (nnz(C) about 1.2e9); batches of undirected
    edge insertions (held-out edges) and deletions, half each."""
    name = "rmat21"
    batch = 1000
    cpu_rows_only = True  # the oracle's full C (1.2e9 entries) does not fit a bounded CPU sample
    sweep = (10, 100, 1000, 10000)
    vsize, dtype = 8, "f64"

    def __init__(self, scale=21):
        super().__init__()
        self.scale = scale
        self.describe = (f"R-MAT scale {scale} ef 8 (0.45,0.15,0.15,0.25) symmetrised, C = A A (+,.) f64, "
                         "batches of 10^3 undirected edge insertions/deletions")
        self.unit = "batches/s (10^3-edge batches)"

    def operands(self):
        from workloads import PLUS_TIMES_F64, rmat_symmetric
        self._A, self._held = rmat_symmetric(self.scale, 8, R21, seed=5, kind=PLUS_TIMES_F64,
                                             holdout=400000 >> max(0, 21 - self.scale))
        return self._A, None


WORKLOADS = {"stencil": StencilWorkload, "rmat20": Rmat20Workload, "rmat21": Rmat21Workload}


# --------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (median SM clock, reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        self.proc.wait()
        with open(self.path) as f:
            out = self.parse(f)
        os.unlink(self.path)
        return out

    @staticmethod
    def parse(lines):
        """Samples in FIELDS order (csv, no header, no units): the median SM
        clock, the maximum, and every throttle reason seen Active."""
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ GPU arm

def gpu_arm(args):
    import torch
    import paper_2202_08808_gb300 as pkg
    W = WORKLOADS[args.workload]()

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    A, B = W.operands()
    g = pkg.DynamicSpGEMM(A, B)
    info = g.info()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    vsize = W.vsize
    s_entry = 4 + vsize  # column + value bytes per entry

    # device-resident batches: warm-up, timed steps, then instrumented steps
    n_prof = min(args.steps, 10)
    nb = args.warmup + args.steps + 2 + n_prof
    host_batches = W.batches(nb, 1000 * (rank + 1))
    dev_batches = []
    for b in host_batches:
        dev_batches.append(type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(),
                                   torch.from_numpy(b.val).cuda(), torch.from_numpy(b.op).cuda()))
    torch.cuda.synchronize()

    # the clock sampler starts first: its start-up pause (an idle host) comes
    # before the warm-up steps, which then run right before the timed ones
    clocks = ClockSampler(local)
    clocks.start()
    tuned = None
    if args.autotune > 0:
        # bins chosen by measurement on calibration batches of the same workload
        cal = [type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(), torch.from_numpy(b.val).cuda(),
                       torch.from_numpy(b.op).cuda()) for b in W.batches(args.autotune, 3000 * (rank + 1))]
        best, cand_ms = g.autotune(cal)
        tuned = {"chosen": best, "candidate_ms": [round(x, 4) for x in cand_ms], "batches": args.autotune}
    for k in range(args.warmup):  # eager, captured, replayed; like the timed steps
        flush.zero_()
        g.apply_batch(dev_batches[k])
    barrier()

    # timed steps: no instrumentation inside the step
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = pkg.kernel_launches()
    runs0 = g.run_counts()
    barrier()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        g.apply_batch(dev_batches[args.warmup + k])
        ev1[k].record(stream)
    launches = pkg.kernel_launches() - launches0
    runs1 = g.run_counts()
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    lat = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = slowest_rank_ms(dist, sum(lat), "cuda")

    # instrumented steps (events between the stages) for the stage times and
    # the recompute roofline, on further batches of the same workload
    g.set_profiling(True)
    base = args.warmup + args.steps
    for k in range(2):
        g.apply_batch(dev_batches[base + k])
    stage_acc = {s: 0.0 for s in pkg.STAGES}
    stats_acc = []
    for k in range(n_prof):
        flush.zero_()
        stats_acc.append(g.apply_batch(dev_batches[base + 2 + k]))
        for s, v in g.stage_times().items():
            stage_acc[s] += v
    g.set_profiling(False)

    # recompute roofline: algorithmic bytes of the numeric stage (gather model)
    R = sum(s["affected_rows"] for s in stats_acc)
    a_ent = sum(s["a_entries"] for s in stats_acc)
    prods = sum(s["products"] for s in stats_acc)
    nnzw = sum(s["nnz_written"] for s in stats_acc)
    # gather model: an 8 B row header per row of R and per B row read (the
    # row's place and length), the A' entries, every product's B entry, and
    # the entries of C written
    alg_bytes = 8 * R + (s_entry + 8) * a_ent + s_entry * prods + s_entry * nnzw
    numeric_ms = stage_acc["numeric"]
    peak, peak_kind = peaks()
    achieved = alg_bytes / (numeric_ms * 1e-3) / 1e9 if numeric_ms > 0 else 0.0

    # static comparator: full recompute of C from the same A', B' on the device,
    # under every built-in tuning of the row bins; the fastest counts
    def time_static():
        ts = []
        for k in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.recompute_all()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)
    static_runs = {"handle_bins": time_static()}
    keep_tuning = g.get_tuning()
    for ci, cand in enumerate(pkg.tuning_candidates()):
        g.set_tuning(cand)
        static_runs[f"candidate_{ci}"] = time_static()
    g.set_tuning(keep_tuning)
    static_med = min(static_runs.values())
    cusparse = cusparse_static(A, B, flush, stream) if (W.name == "stencil" and not args.no_cusparse) else None
    for b in W.batches(2, 7000 * (rank + 1)):  # re-capture the pipeline under the restored bins
        g.apply_batch(type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(),
                              torch.from_numpy(b.val).cuda(), torch.from_numpy(b.op).cuda()))

    # end to end through the public API with pinned host buffers: upload of
    # the batch, apply, read back the affected row set and its rows of C
    e2e_ms, h2d, d2h = [], 0, 0
    pinned = []
    # (the first W, untimed, are the warm-up: they also fill the pinned host
    # allocator that the read-back arrays come from)
    n_warm = max(3, args.warmup)
    for b in W.batches(max(3, min(args.steps, 10)) + n_warm, 5000 * (rank + 1)):
        pinned.append(type(b)(torch.from_numpy(b.row).pin_memory(), torch.from_numpy(b.col).pin_memory(),
                              torch.from_numpy(b.val).pin_memory(), torch.from_numpy(b.op).pin_memory()))
    out = None  # one set of page-locked result arrays, reused by every read (as a serving loop keeps them)
    for k, b in enumerate(pinned):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the batch and then R with its rows of C', one call and (with the
        # page-locked result arrays) one synchronisation
        _, (rows, rp, col, val) = g.apply_read_affected(b, out=out)
        t1 = time.perf_counter()
        if out is None:  # sized after the first (untimed) read, with room for the next batches
            nr, ne = 2 * rows.shape[0] + 1024, 2 * col.shape[0] + 4096
            out = tuple(torch.empty(m, dtype=dt, pin_memory=True).numpy() for m, dt in
                        ((nr, torch.int32), (nr + 1, torch.int64), (ne, torch.int32),
                         (ne, torch.float64 if val.dtype == np.float64 else torch.int32)))
        if k >= n_warm:
            e2e_ms.append((t1 - t0) * 1e3)
        h2d = len(b.row) * (4 + 4 + vsize + 1)
        d2h = rows.nbytes + rp.nbytes + col.nbytes + val.nbytes + 13 * 8
    e2e_mean = statistics.mean(e2e_ms)

    # batch-size sweep (latency and speedup from one update to 10^6)
    sweep = []
    if not args.no_sweep:
        for nupd in W.sweep:
            # a new launch size runs eagerly once and is captured on its
            # second batch: the median is over the replays after those (ten
            # up to 10^4 updates, where a step is well under a millisecond)
            bs = W.batches(12 if nupd <= 10000 else 5, 9000 + nupd, nupd)
            dbs = [type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(),
                           torch.from_numpy(b.val).cuda(), torch.from_numpy(b.op).cuda()) for b in bs]
            torch.cuda.synchronize()
            ts = []
            for kb, db in enumerate(dbs):
                # as in the timed steps: the flush is enqueued before the
                # start event, without a host synchronisation in between
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = g.apply_batch(db)
                e1.record(stream)
                torch.cuda.synchronize()
                if kb >= 2:
                    ts.append(e0.elapsed_time(e1))
            med = statistics.median(ts)
            sweep.append({"batch": nupd, "entries": len(bs[0]), "frac_nnz_a": len(bs[0]) / A.nnz,
                          "latency_ms": round(med, 4),
                          "speedup_vs_static": round(static_med / med, 2), "affected_rows": st["affected_rows"]})

    # the delta path of Eq. 1 beside the row path, on insert-only batches of
    # the same sizes (positions two grid hops away, never inserted before),
    # the two paths alternating on the same handle
    delta = []
    if not args.no_sweep and W.name == "stencil":
        from workloads import stencil_insert_batch
        taken: set = set()
        Ag = g.read_A()  # positions present now (earlier batches inserted some two hops away)
        present = np.repeat(np.arange(Ag.nrows, dtype=np.int64), np.diff(Ag.rowptr)) * Ag.ncols + Ag.col

        def timed(b, algebraic):
            db = type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(),
                         torch.from_numpy(b.val).cuda(), torch.from_numpy(b.op).cuda())
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = g.apply_batch(db, algebraic=algebraic)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), st

        for nupd in (1000, 10000, 100000):
            t_alg, t_row, alg_ok, rows_alg, rows_row = [], [], True, 0, 0
            for r in range(5):
                ta, sa = timed(stencil_insert_batch(GRID, GRID, GRID, nupd, 8000 + 10 * r + nupd, taken, present), True)
                tr, sr_ = timed(stencil_insert_batch(GRID, GRID, GRID, nupd, 8005 + 10 * r + nupd, taken, present),
                                False)
                if r < 2:
                    continue  # the first two of each size warm the paths (buffers; the row path's graph capture)
                t_alg.append(ta)
                t_row.append(tr)
                alg_ok &= sa["algebraic"] == 1
                rows_alg, rows_row = sa["affected_rows"], sr_["affected_rows"]
            ma, mr = statistics.median(t_alg), statistics.median(t_row)
            delta.append({"batch": nupd, "delta_path_ms": round(ma, 4), "row_path_ms": round(mr, 4),
                          "delta_speedup_vs_row": round(mr / ma, 2), "delta_speedup_vs_static": round(static_med / ma, 2),
                          "rows_touched_delta": rows_alg, "rows_recomputed_row": rows_row, "all_delta": bool(alg_ok)})

    masked = masked_leg(args, flush, stream) if (not args.no_masked and W.name == "stencil") else None

    out = None
    if rank == 0:
        cpu = None if args.no_cpu else cpu_baseline(args, W, budget_s=args.cpu_budget)
        ms_per_step = total_ms / args.steps
        out = {
            "metric": METRIC,
            "value": round(world * args.steps / (total_ms * 1e-3), 3),
            "unit": W.unit,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": W.dtype,
            "data": "synthetic",
            "config": {"workload": W.describe,
                       "n": info["n"], "nnz_a": info["nnz_a"], "nnz_c": info["nnz_c"], "batch": W.batch,
                       "batch_entries": len(host_batches[0]),
                       "l2": "flushed before every timed step (256 MiB write)", "parallelism": f"replicas x{world}"},
            "latency_ms": {"mean": round(statistics.mean(lat), 4), "p50": round(statistics.median(lat), 4),
                           "p99": round(float(np.percentile(lat, 99)), 4), "max": round(max(lat), 4)},
            "graph_runs_timed": {k: runs1[k] - runs0[k] for k in runs0},
            "static_recompute_ms": round(static_med, 3),
            "static_runs_ms": {k: round(v, 3) for k, v in static_runs.items()},
            "static_best": min(static_runs, key=static_runs.get),
            "cusparse_static": cusparse,
            "tuning": tuned,
            "speedup_vs_static": round(static_med / statistics.median(lat), 2),
            "stages_ms": {s: round(v / max(n_prof, 1), 4) for s, v in stage_acc.items()},
            "stages_note": f"device time per stage, mean of {n_prof} further steps run with stage events",
            "roofline": {"bound": "hbm", "kernel": "numeric recompute (all bins) of the affected rows",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "alg_bytes_per_step": int(alg_bytes / max(n_prof, 1)),
                         "traffic": NUMERIC_TRAFFIC.get(W.name),
                         "traffic_note": ("DRAM bytes of the numeric kernels in one step (ncu, "
                                          "profiles/numeric_stage_dram_stencil128.md)"
                                          if W.name in NUMERIC_TRAFFIC else None)},
            "e2e": {"value": round(1e3 / e2e_mean, 3), "unit": W.unit,
                    "latency_ms": round(e2e_mean, 4), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "gpu_launches_per_step": round(launches / args.steps, 1),
            "clocks": clk,
            "wall_s_timed": round(wall, 3),
            "batch_sweep": sweep,
            "delta_path_insert_only": delta,
            "masked_general_updates": masked,
            "cpu_baseline": cpu,
        }
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


def cusparse_static(A, B, flush, stream):
    """An external sanity reference for the static (+,.) product: cuSPARSE's
    SpGEMM (torch's CSR x CSR product on the device) on the same A', timed
    like the static recompute (median of three, L2 flushed before each);
    not on the library's path."""
    import torch
    try:
        def dev(M):
            return torch.sparse_csr_tensor(torch.from_numpy(np.asarray(M.rowptr, np.int64)).cuda(),
                                           torch.from_numpy(np.asarray(M.col, np.int64)).cuda(),
                                           torch.from_numpy(np.asarray(M.val, np.float64)).cuda(),
                                           size=(M.nrows, M.ncols))
        a = dev(A)
        b = a if B is None else dev(B)
        ts, nnz = [], None
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c = a @ b
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            nnz = int(c._nnz())
            del c
        return {"ms": round(statistics.median(ts), 3), "nnz_c": nnz,
                "what": "torch CSR @ CSR on the device (cuSPARSE SpGEMM), f64, the build's A"}
    except Exception as e:  # a comparator only: report why it did not run
        return {"unavailable": str(e).splitlines()[0][:200]}


def masked_leg(args, flush, stream, scale=20):
    """The entry-level masked recompute (Algorithm 2) beside the row path,
    on R-MAT scale 20 (edge factor 8, (0.45,0.15,0.15,0.25), symmetrised,
    C = A A in (+,.) f64): the same edge batches (half insertions of
    held-out edges, half deletions) applied to a row-path handle and to a
    handle with the Bloom filter, each apply timed on the device with L2
    flushed before it; then sampled rows of the two C's compared."""
    import torch
    import paper_2202_08808_gb300 as pkg
    W = Rmat21Workload(scale)
    A, _ = W.operands()
    g_row = pkg.DynamicSpGEMM(A)
    g_msk = pkg.DynamicSpGEMM(A, bloom=True)
    res = []

    def timed(g, db):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = g.apply_batch(db)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st

    for n_edges in (100, 1000, 10000):
        bs = W.batches(6, 600 + n_edges, n_edges)
        t_row, t_msk, s_row, s_msk = [], [], None, None
        for k, b in enumerate(bs):
            db = type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(), torch.from_numpy(b.val).cuda(),
                         torch.from_numpy(b.op).cuda())
            tr, s_row = timed(g_row, db)
            tm, s_msk = timed(g_msk, db)
            if k >= 2:  # the first two of each size warm the paths (buffers; the row path's graph capture)
                t_row.append(tr)
                t_msk.append(tm)
        mr, mm = statistics.median(t_row), statistics.median(t_msk)
        res.append({"edges": n_edges, "row_path_ms": round(mr, 4), "masked_path_ms": round(mm, 4),
                    "masked_speedup_vs_row": round(mr / mm, 2),
                    "row_path": {"affected_rows": s_row["affected_rows"], "products": s_row["products"],
                                 "nnz_written": s_row["nnz_written"]},
                    "masked_path": {"rows_of_c_star": s_msk["affected_rows"], "c_star_entries": s_msk["masked_entries"],
                                    "kept_a_entries": s_msk["a_entries"], "products": s_msk["products"],
                                    "nnz_written": s_msk["nnz_written"]}})
    rows = np.unique(g_row.last_affected())[:2000]
    ra, rb = g_row.read_rows_C(rows), g_msk.read_rows_C(rows)
    same = bool(np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1]))
    scale_v = np.maximum(np.abs(ra[2]), 1e-300) if same else None
    rel = float(np.max(np.abs(ra[2] - rb[2]) / scale_v)) if same and ra[2].size else None
    info = g_row.info()
    out = {"workload": f"R-MAT scale {scale} ef 8 (0.45,0.15,0.15,0.25) symmetrised, C = A A (+,.) f64",
           "n": info["n"], "nnz_a": info["nnz_a"], "nnz_c": info["nnz_c"],
           "l2": "flushed before every timed apply", "batches": res,
           "same_rows_sampled": int(rows.shape[0]), "same_pattern": same, "max_rel_diff": rel}
    g_row.close()
    g_msk.close()
    return out


# ------------------------------------------------- batched instances (group)

G500 = (0.57, 0.19, 0.19, 0.05)


def batched_instances(count, seed=4):
    """The batched workload: `count` independent R-MAT instances (scale 10..16
    uniform, edge factor 8, Graph500 parameters), (+,.) f64 U(0,1) for even t
    and (min,+) int32 U[1,100] for odd t, C = A A; one batch size per
    instance, log-uniform in 10..10^4 undirected-edge changes (insertions of
    held-out edges, drawn with replacement when the batch wants more than the
    pool holds, and deletions of present edges)."""
    from workloads import MIN_PLUS_I32, PLUS_TIMES_F64, rmat_symmetric
    rng = np.random.default_rng(seed)
    scales = rng.integers(10, 17, size=count)
    sizes = np.floor(10 ** rng.uniform(1, 4, size=count)).astype(np.int64)
    out = []
    for t in range(count):
        sr = PLUS_TIMES_F64 if t % 2 == 0 else MIN_PLUS_I32
        pool = int(min(max(16, sizes[t]), (8 << int(scales[t])) // 20))  # at most ~5% of the edges held out
        A, held = rmat_symmetric(int(scales[t]), 8, G500, seed=1000 * seed + t, kind=sr, holdout=pool)
        out.append({"A": A, "held": held, "size": int(sizes[t]), "scale": int(scales[t]), "sr": sr})
    return out


def batched_batches(insts, step, device=True, uneven=False):
    """One batch per instance: of the instance's own size, or (uneven) of a
    size drawn afresh for every step, log-uniform in 10..10^4 edges."""
    import torch
    from workloads import rmat_edge_batch
    bs = []
    rng = np.random.default_rng(31 * step + 7) if uneven else None
    for t, it in enumerate(insts):
        size = int(10 ** rng.uniform(1, 4)) if uneven else it["size"]
        b = rmat_edge_batch(it["A"], it["held"], size, seed=7919 * (step + 1) + t)
        if device:
            b = type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(), torch.from_numpy(b.val).cuda(),
                        torch.from_numpy(b.op).cuda())
        bs.append(b)
    return bs


def batched_arm(args):
    import torch
    import paper_2202_08808_gb300 as pkg
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:  # the instances are independent: each rank takes its share, no data-path collective
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    t0 = time.perf_counter()
    mine = shard_units(args.instances, rank, world)
    insts = [batched_instances(args.instances, seed=4)[t] for t in mine] if world > 1 else \
        batched_instances(args.instances, seed=4)
    count = len(insts)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    hs = [pkg.DynamicSpGEMM(it["A"], exact_static=1) for it in insts]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    nnz_c = sum(h.info()["nnz_c"] for h in hs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    step_no = [0]

    def next_batches(device=True, uneven=False):
        step_no[0] += 1
        return batched_batches(insts, step_no[0], device, uneven)

    def time_group(grp, steps, warmup, collect=None, uneven=False):
        for _ in range(warmup):
            grp.apply(next_batches(uneven=uneven))
        torch.cuda.synchronize()
        pre = [next_batches(uneven=uneven) for _ in range(steps)]
        ms = []
        k0 = pkg.kernel_launches()
        for k in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats, _ = grp.apply(pre[k])
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            if collect is not None:
                collect.append(stats)
        return ms, pkg.kernel_launches() - k0

    grp = pkg.Group(hs)
    default_ms, _ = time_group(grp, args.steps, args.warmup)

    # autotune every instance on two calibration batches of its own size
    t0 = time.perf_counter()
    chosen = {}
    for t, h in enumerate(hs):
        cal = [batched_batches([insts[t]], 100000 + 2 * t + j)[0] for j in range(2)]
        best, _ = h.autotune(cal)
        key = tuple(best.values())
        chosen[key] = chosen.get(key, 0) + 1
    tune_s = time.perf_counter() - t0
    cands = [tuple(c.values()) for c in pkg.tuning_candidates()]

    stats_acc = []
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.perf_counter()
    tuned_ms, launches = time_group(grp, args.steps, args.warmup, stats_acc)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()

    # the same instances as separate apply_batch calls, one after another
    for _ in range(args.warmup):
        for h, b in zip(hs, next_batches()):
            h.apply_batch(b)
    torch.cuda.synchronize()
    sep_ms = []
    for k in range(args.steps):
        bs = next_batches()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for h, b in zip(hs, bs):
            h.apply_batch(b)
        e1.record(stream)
        torch.cuda.synchronize()
        sep_ms.append(e0.elapsed_time(e1))

    # fresh uneven sizes every step (log-uniform 10..10^4 edges per instance):
    # with every member's launch sizes reserved for the largest batch, the
    # group replays one captured pipeline whatever the sizes; separate calls
    # take the same batches
    def runs():
        c = [h.run_counts() for h in hs]
        return {k: sum(x[k] for x in c) for k in ("replayed", "captured", "eager")}
    for h in hs:  # launch sizes for the largest batch of the distribution: 10^4 edges, both directions
        h.reserve(2 * 10 ** 4)
    for _ in range(2):  # eager, captured
        grp.apply(next_batches(uneven=True))
    r0 = runs()
    uneven_ms, _ = time_group(grp, args.steps, 0, uneven=True)
    r1 = runs()
    uneven_sep = []
    for k in range(args.steps):
        bs = next_batches(uneven=True)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for h, b in zip(hs, bs):
            h.apply_batch(b)
        e1.record(stream)
        torch.cuda.synchronize()
        uneven_sep.append(e0.elapsed_time(e1))
    member_runs = sum(r1[k] - r0[k] for k in r1)
    uneven = {"group_ms": round(statistics.median(uneven_ms), 4),
              "separate_calls_ms": round(statistics.median(uneven_sep), 4),
              "speedup_group_vs_separate": round(statistics.median(uneven_sep) / statistics.median(uneven_ms), 2),
              "member_runs_replayed": round((r1["replayed"] - r0["replayed"]) / max(member_runs, 1), 3),
              "member_runs": int(member_runs)}

    # end to end with pinned host batches through the group call
    e2e_ms, h2d = [], 0
    for k in range(max(3, min(args.steps, 5))):
        hb = [type(b)(torch.from_numpy(b.row).pin_memory(), torch.from_numpy(b.col).pin_memory(),
                      torch.from_numpy(b.val).pin_memory(), torch.from_numpy(b.op).pin_memory())
              for b in next_batches(device=False)]
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats, _ = grp.apply(hb)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        h2d = sum(len(b.row) * (4 + 4 + b.val.element_size() + 1) for b in hb)
    d2h = count * 13 * 8  # per-member statistics read back

    med = statistics.median(tuned_ms)
    job_ms = slowest_rank_ms(dist, sum(tuned_ms), "cuda")
    R = sum(st["affected_rows"] for ss in stats_acc for st in ss) / len(stats_acc)
    alg = 0.0
    for ss in stats_acc:
        for t, st in enumerate(ss):
            se = 12 if insts[t]["sr"] == 0 else 8
            alg += 12 * st["affected_rows"] + (se + 12) * st["a_entries"] + se * st["products"] + se * st["nnz_written"]
    alg /= len(stats_acc)
    peak, peak_kind = peaks()
    achieved = alg / (statistics.mean(tuned_ms) * 1e-3) / 1e9
    if dist is not None:
        dist.barrier()
    if rank != 0:
        grp.close()
        dist.destroy_process_group()
        return
    cpu = None if args.no_cpu else batched_cpu_baseline(insts, args.cpu_budget)
    out = {
        "metric": METRIC,
        "value": round(args.instances * args.steps / (job_ms * 1e-3), 1),
        "unit": f"instance batches/s ({args.instances} instances per step)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(statistics.mean(tuned_ms), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+i32", "data": "synthetic",
        "config": {"workload": f"batched: {args.instances} R-MAT instances, scales 10-16, edge factor 8, C = A A, half "
                               "(+,.) f64 half (min,+) i32, one batch each of 10..10^4 edge changes (log-uniform)",
                   "nnz_c_total": int(nnz_c), "batch_entries_per_step": int(2 * sum(it["size"] for it in insts)),
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"instances sharded over {world} GPU(s), rank 0's share in the per-rank keys"},
        "latency_ms": {"p50": round(med, 4), "p99": round(float(np.percentile(tuned_ms, 99)), 4)},
        "group_default_tuning_ms": round(statistics.median(default_ms), 4),
        "group_tuned_ms": round(med, 4),
        "separate_calls_ms": round(statistics.median(sep_ms), 4),
        "speedup_group_vs_separate": round(statistics.median(sep_ms) / med, 2),
        "uneven_sizes_every_step": uneven,
        "autotune": {"seconds": round(tune_s, 2), "chosen": {str(cands.index(k)): v for k, v in chosen.items()}},
        "affected_rows_per_step": int(R),
        "roofline": {"bound": "hbm", "kernel": "whole group step (every stage of every instance)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_kind": peak_kind, "alg_bytes_per_step": int(alg), "traffic": None},
        "e2e": {"value": round(1e3 * count / statistics.mean(e2e_ms), 1), "unit": "instance batches/s",
                "latency_ms": round(statistics.mean(e2e_ms), 4), "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches), "gpu_launches_per_step": round(launches / args.steps, 1),
        "clocks": clk, "wall_s_timed": round(wall, 3),
        "setup_s": {"generate": round(gen_s, 1), "build": round(build_s, 1)},
        "cpu_baseline": cpu,
    }
    grp.close()
    if dist is not None:
        dist.destroy_process_group()
    print(json.dumps(out), flush=True)


def batched_cpu_baseline(insts, budget_s):
    """The oracle's row-dynamic route on the instances of scale <= 12 of the
    batched workload, one batch each, until the budget (set-up included) is
    used; single-threaded C."""
    import oracle
    from oracle import OMat
    times, k, start = [], 0, time.perf_counter()
    for t, it in enumerate(insts):
        if it["scale"] > 12:
            continue
        Ao = OMat.from_csr(it["A"])
        Co = Ao.multiply(Ao)
        b = batched_batches([it], 500000 + t, device=False)[0]
        t0 = time.perf_counter()
        oracle.row_dynamic(Ao, Co, b)
        times.append(time.perf_counter() - t0)
        k += 1
        if time.perf_counter() - start > budget_s:
            break
    mean = statistics.mean(times)
    return {"value": round(1.0 / mean, 3), "unit": "instance batches/s", "cores": 1, "kind": "oracle",
            "sample": f"one batch on each of {k} instances of scale <= 12 (apply + affected rows + row recompute)"}


# ------------------------------------------- learned sizing + serving

R21 = (0.45, 0.15, 0.15, 0.25)


def _dev_batch(b):
    import torch
    return type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(), torch.from_numpy(b.val).cuda(),
                   torch.from_numpy(b.op).cuda())


def train_estimator(pkg, seeds, steps, log):
    """Features and exact row sizes of R-MAT scale-18 instances (all rows
    after the build, and the affected rows after two random batches), then
    SGD on the GPU."""
    import torch
    from workloads import PLUS_TIMES_F64, EdgeStream, mlp_init_params, rmat_symmetric
    Xs, ys = [], []
    t0 = time.perf_counter()
    for sd in seeds:
        A, held = rmat_symmetric(18, 8, R21, seed=sd, kind=PLUS_TIMES_F64, holdout=20000)
        g = pkg.DynamicSpGEMM(A)
        X, y = g.row_features()
        Xs.append(X)
        ys.append(y)
        es = EdgeStream(A, held, sd)
        for ne in (300, 3000):
            g.apply_batch(_dev_batch(es.batch(ne)))
            X, y = g.row_features(torch.from_numpy(g.last_affected()).cuda())
            Xs.append(X)
            ys.append(y)
        g.close()
    X, y = torch.cat(Xs), torch.cat(ys)
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(1)).cuda()
    X, y = X[perm].contiguous(), y[perm].contiguous()
    data_s = time.perf_counter() - t0
    est = pkg.Estimator(mlp_init_params(seeds[0]))
    loss0, _ = est.grad(X, y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss1 = est.train(X, y, batch=4096, steps=steps, lr=5e-4)
    train_s = time.perf_counter() - t0
    log(f"estimator: {X.shape[0]} rows, loss {loss0:.3f} -> {loss1:.4f} in {steps} steps ({train_s:.2f} s)")
    return est, {"rows": int(X.shape[0]), "graphs": len(seeds), "loss_initial": round(loss0, 4),
                 "loss_final": round(loss1, 5), "steps": steps, "batch": 4096, "train_s": round(train_s, 3),
                 "data_s": round(data_s, 2)}


def learned_arm(args):
    import torch
    import paper_2202_08808_gb300 as pkg
    from paper_2202_08808_gb300.serving import Request, Server, latency_summary
    from workloads import PLUS_TIMES_F64, EdgeStream, rmat_symmetric
    torch.cuda.set_device(0)

    def log(msg):
        print(msg, file=sys.stderr, flush=True)

    est, est_info = train_estimator(pkg, list(range(50, 50 + args.train_graphs)), args.train_steps, log)
    t0 = time.perf_counter()
    A, held = rmat_symmetric(args.scale, 8, R21, seed=5, kind=PLUS_TIMES_F64, holdout=400000)
    gen_s = time.perf_counter() - t0
    modes = {"bound": pkg.SIZE_BOUND, "exact": pkg.SIZE_EXACT, "learned": pkg.SIZE_LEARNED}
    hs = {}
    t0 = time.perf_counter()
    for name, mode in modes.items():
        hs[name] = pkg.DynamicSpGEMM(A)
        hs[name].set_sizing(mode, est if mode == pkg.SIZE_LEARNED else None, est_min=args.est_min,
                            margin=args.est_margin)
    torch.cuda.synchronize()
    build_s = (time.perf_counter() - t0) / len(modes)
    info = hs["bound"].info()
    log(f"scale {args.scale}: nnz(A) {info['nnz_a']}, nnz(C) {info['nnz_c']}, build {build_s:.2f} s per handle")
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    # the same batches, in the same order, on the three handles
    rng = np.random.default_rng(500)
    es = EdgeStream(A, held, 501)
    sizes = np.floor(10 ** rng.uniform(1, 5, size=args.compare_batches)).astype(int)
    warm = [_dev_batch(es.batch(int(x))) for x in (100, 1000, 10000)]
    for h in hs.values():
        for b in warm:
            h.apply_batch(b)
    times = {k: [] for k in modes}
    stats = {k: [] for k in modes}
    worst_rel = 0.0
    for x in sizes:
        b = _dev_batch(es.batch(int(x)))
        for name, h in hs.items():
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = h.apply_batch(b)
            e1.record(stream)
            torch.cuda.synchronize()
            times[name].append(e0.elapsed_time(e1))
            stats[name].append(st)
        # identical outputs: same affected rows, same patterns, values equal to rounding
        R = hs["bound"].last_affected()
        samp = R if R.shape[0] <= 20000 else np.sort(np.random.default_rng(int(x)).choice(R, 20000, replace=False))
        ref = hs["bound"].read_rows_C(samp)
        for name in ("exact", "learned"):
            assert np.array_equal(hs[name].last_affected(), R), f"{name}: affected rows differ"
            got = hs[name].read_rows_C(samp)
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), f"{name}: patterns differ"
            nz = ref[2] != 0
            if nz.any():
                worst_rel = max(worst_rel, float(np.max(np.abs(got[2][nz] - ref[2][nz]) / np.abs(ref[2][nz]))))
    assert worst_rel <= 2e-12, worst_rel
    per_mode = {}
    for name in modes:
        t = np.array(times[name])
        per_mode[name] = {"mean_ms": round(float(t.mean()), 4), "p50_ms": round(float(np.median(t)), 4),
                          "p99_ms": round(float(np.percentile(t, 99)), 4),
                          "batches_per_s": round(len(t) / (t.sum() * 1e-3), 2),
                          "est_rows": int(sum(s["est_rows"] for s in stats[name])),
                          "est_overflows": int(sum(s["est_overflows"] for s in stats[name]))}
    by_decade = {}
    for d in range(1, 5):
        sel = [k for k, x in enumerate(sizes) if 10 ** d <= x < 10 ** (d + 1)]
        if sel:
            by_decade[f"1e{d}"] = {name: round(float(np.mean([times[name][k] for k in sel])), 4) for name in modes}
    log(f"sizing: {per_mode}")

    # serving on the learned handle: service rate with every request queued,
    # then Poisson arrivals at 0.5x, 1x and 2x that rate
    srv_h = hs["learned"]
    for name in ("bound", "exact"):
        hs[name].close()
    qrng = np.random.default_rng(502)

    def requests(count, rate):
        out = []
        t = 0.0
        for k in range(count):
            if rate is not None:
                t += float(qrng.exponential(1.0 / rate))
            out.append(Request(k, t, es.batch(int(10 ** qrng.uniform(1, 5)))))
        return out

    srv = Server(srv_h, max_wave=args.max_wave, read_results=False)
    cal = requests(args.requests, None)
    t0 = time.perf_counter()
    res = srv.serve(cal)
    wall = time.perf_counter() - t0
    mu = len(res) / wall
    serving = {"service_rate_req_s": round(mu, 2), "saturated": latency_summary(res, wall)}
    clocks = ClockSampler(0)
    clocks.start()
    for f in (0.5, 1.0, 2.0):
        srv = Server(srv_h, max_wave=args.max_wave, read_results=False)
        reqs = requests(args.requests, f * mu)
        t0 = time.perf_counter()
        res = srv.serve(reqs)
        wall = time.perf_counter() - t0
        serving[f"rate_{f}x"] = dict(latency_summary(res, wall), offered_req_s=round(f * mu, 2), waves=srv.waves,
                                     conflicts=srv.conflicts)
    clk = clocks.stop()
    log(f"serving: {serving}")
    srv_h.close()
    serving_stencil = serving_on_stencil(args, log)

    cpu = None if args.no_cpu else learned_cpu_baseline(A, held, args.cpu_budget)
    lm = per_mode["learned"]
    out = {
        "metric": METRIC,
        "value": lm["batches_per_s"],
        "unit": "batches/s (learned sizing, batches of 10..10^5 edge changes)",
        "n_gpus": 1, "steps": int(len(sizes)), "warmup": 3, "ms_per_step": lm["mean_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"learned sizing + serving: R-MAT scale {args.scale}, edge factor 8, (0.45,0.15,0.15,0.25), "
                               "symmetrised, C = A A (+,.) f64; estimator trained on scale-18 instances",
                   "nnz_a": info["nnz_a"], "nnz_c": info["nnz_c"], "batch_sizes": [int(x) for x in sizes],
                   "l2": "flushed before every timed batch (256 MiB write)"},
        "sizing": per_mode,
        "sizing_by_decade_ms": by_decade,
        "speedup_learned_vs_exact": round(per_mode["exact"]["mean_ms"] / lm["mean_ms"], 3),
        "speedup_learned_vs_bound": round(per_mode["bound"]["mean_ms"] / lm["mean_ms"], 3),
        "max_rel_diff_between_sizings": worst_rel,
        "estimator": est_info,
        "serving": serving,
        "serving_stencil": serving_stencil,
        "clocks": clk,
        "setup_s": {"generate": round(gen_s, 1), "build_per_handle": round(build_s, 2)},
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)


def serving_on_stencil(args, log):
    """Continuous batching where footprints are small: the 128^3 stencil with
    requests of 10..10^3 updates (log-uniform).  The same queued stream is
    served with waves of one request (a plain queue) and with waves of up to
    max_wave requests, then Poisson streams at 0.5x, 1x and 2x the batched
    service rate."""
    import paper_2202_08808_gb300 as pkg
    from paper_2202_08808_gb300.serving import Request, Server, latency_summary
    from workloads import stencil7, stencil_batch
    A = stencil7(GRID, GRID, GRID, seed=1)
    g = pkg.DynamicSpGEMM(A)
    rng = np.random.default_rng(504)

    def requests(count, rate, seed0):
        out, t = [], 0.0
        for k in range(count):
            if rate is not None:
                t += float(rng.exponential(1.0 / rate))
            out.append(Request(k, t, stencil_batch(GRID, GRID, GRID, int(10 ** rng.uniform(1, 3)), seed=seed0 + k)))
        return out

    res = {}
    # a plain queue (one request at a time, nothing overlapped), waves one
    # after another, and pipelined waves (the next wave runs on the GPU while
    # the previous one's rows are read back)
    for name, mw, pipe in (("queue", 1, False), ("waves", args.max_wave, False),
                           ("pipelined", args.max_wave, True)):
        Server(g, max_wave=mw, read_results=True, pipelined=pipe).serve(requests(20, None, 600000 + mw))  # warm graphs
        srv = Server(g, max_wave=mw, read_results=True, pipelined=pipe)
        reqs = requests(args.requests, None, 700000 + 1000 * mw)
        t0 = time.perf_counter()
        out = srv.serve(reqs)
        wall = time.perf_counter() - t0
        res[f"saturated_{name}"] = dict(latency_summary(out, wall), waves=srv.waves, conflicts=srv.conflicts,
                                        overlapped_reads=srv.overlaps() if pipe else 0)
    mu = res["saturated_pipelined"]["throughput_req_s"]
    for f in (0.5, 1.0, 2.0):
        srv = Server(g, max_wave=args.max_wave, read_results=True, pipelined=True)
        reqs = requests(args.requests, f * mu, 800000 + int(10 * f))
        t0 = time.perf_counter()
        out = srv.serve(reqs)
        wall = time.perf_counter() - t0
        res[f"rate_{f}x"] = dict(latency_summary(out, wall), offered_req_s=round(f * mu, 2), waves=srv.waves,
                                 conflicts=srv.conflicts)
    g.close()
    log(f"serving on the stencil: {res}")
    return res


def learned_cpu_baseline(A, held, budget_s, n_batches=None, edges=100, unit="batches/s (100-edge batches)"):
    """The oracle on a bounded sample of the same workload: apply a batch,
    find its affected rows, recompute them (the row-dynamic route without the
    write into a stored C, which is too large for the sample); single-threaded C."""
    from oracle import OMat, affected_rows
    from workloads import EdgeStream
    start = time.perf_counter()
    Ao = OMat.from_csr(A)
    es = EdgeStream(A, held, 503)
    times, rows = [], 0
    while time.perf_counter() - start < budget_s and len(times) < (n_batches or 20):
        b = es.batch(edges)
        t0 = time.perf_counter()
        pre = Ao.presence(b)
        Ao.apply(b)
        post = Ao.presence(b)
        R = affected_rows(Ao, b, pre, post, b_nrows=A.nrows, b_is_a=True)
        Ao.multiply_rows(Ao, R)
        times.append(time.perf_counter() - t0)
        rows += len(R)
    mean = statistics.mean(times)
    return {"value": round(1.0 / mean, 4), "unit": unit, "cores": 1, "kind": "oracle", "latency_ms": round(mean * 1e3, 3),
            "sample": f"{len(times)} batches of {edges} edge changes on the same graph ({rows} affected rows "
                      "recomputed, without the write into a stored C)"}


# ------------------------------------------------------------ CPU oracle

def cpu_baseline(args, W, budget_s=20.0, steps=None, warmup=0, single=True):
    """The oracle's row-dynamic route (apply, affected rows, recompute of R)
    on a bounded sample of the same workload: consecutive batches until the
    time budget is used, first single-threaded, then with its row loops on
    all host cores (os.cpu_count() threads; the same results).  value and
    cores are the all-cores figures; single_core holds the other."""
    import oracle
    from oracle import OMat
    A, B = W.operands()
    if getattr(W, "cpu_rows_only", False):
        return learned_cpu_baseline(A, W._held, budget_s if steps is None else 1e9, n_batches=steps,
                                    edges=W.batch, unit=W.unit)
    Ao = OMat.from_csr(A)
    Bo = OMat.from_csr(B) if B is not None else None
    Co = Ao.multiply(Bo if Bo is not None else Ao)
    for w in range(warmup):  # untimed
        oracle.row_dynamic(Ao, Co, W.batches(1, 60000 + w)[0], Bo)
    ncores = os.cpu_count() or 1
    k = 0

    def run(threads, budget):
        nonlocal k
        oracle.set_threads(threads)
        times = []
        try:
            while True:
                b = W.batches(1, 70000 + k)[0]
                t0 = time.perf_counter()
                oracle.row_dynamic(Ao, Co, b, Bo)
                times.append(time.perf_counter() - t0)
                k += 1
                if steps is not None and len(times) >= steps:
                    break
                if steps is None and (sum(times) > budget or len(times) >= 200):
                    break
        finally:
            oracle.set_threads(1)
        return times

    one = run(1, budget_s / 2) if single else None
    many = run(ncores, budget_s / 2)
    mean = statistics.mean(many)
    out = {"value": round(1.0 / mean, 4), "unit": W.unit, "cores": ncores,
           "kind": "oracle", "latency_ms": round(mean * 1e3, 3),
           "sample": f"{len(many)} consecutive batches of the workload ({W.describe}): apply + affected rows + "
                     f"row recompute, the row loops on {ncores} threads",
           "times_ms": [round(t * 1e3, 2) for t in many[:20]]}
    if one is not None:
        m1 = statistics.mean(one)
        out["single_core"] = {"value": round(1.0 / m1, 4), "cores": 1, "latency_ms": round(m1 * 1e3, 3),
                              "sample": f"{len(one)} consecutive batches, single-threaded"}
    return out


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    W = WORKLOADS[args.workload if args.workload in WORKLOADS else "stencil"]()
    res = cpu_baseline(args, W, steps=args.steps, warmup=args.warmup, single=False)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": res["unit"], "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["latency_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": W.dtype, "data": "synthetic",
        "config": {"workload": W.describe, "batch": W.batch},
        "cpu_baseline": {"kind": "oracle", "cores": res["cores"], "sample": res["sample"], "value": res["value"]},
        "e2e": {"value": res["value"], "unit": res["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def profile_arm(args):
    """One warmed-up dynamic step (NVTX range "step") or one static recompute
    (NVTX range "static") of the stencil, R-MAT scale-20 or R-MAT A A
    workload (scale --scale), for ncu captures filtered with --nvtx-include."""
    import torch
    import paper_2202_08808_gb300 as pkg
    torch.cuda.set_device(0)
    name = args.workload if args.workload in WORKLOADS else "stencil"
    # rmat21 at a smaller --scale: the same kernels on a case small enough for full ncu captures
    W = WORKLOADS[name](args.scale) if name == "rmat21" else WORKLOADS[name]()
    A, B = W.operands()
    g = pkg.DynamicSpGEMM(A, B)
    if args.profile == "static":
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("static")
        g.recompute_all()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print("static profiled")
        return
    nupd = args.batch if args.workload == "stencil" else W.batch
    bs = W.batches(4, 100, nupd)
    dev = [type(b)(torch.from_numpy(b.row).cuda(), torch.from_numpy(b.col).cuda(), torch.from_numpy(b.val).cuda(),
                   torch.from_numpy(b.op).cuda()) for b in bs]
    for b in dev[:3]:
        g.apply_batch(b)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("step")
    st = g.apply_batch(dev[3])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print("step profiled", st)
    if args.profile == "read":  # R and its rows of C' into page-locked arrays (sized by a first read)
        rows, rp, col, val = g.read_affected()
        out = tuple(torch.empty(x.shape[0], dtype=dt, pin_memory=True).numpy() for x, dt in
                    ((rows, torch.int32), (rp, torch.int64), (col, torch.int32),
                     (val, torch.float64 if val.dtype == np.float64 else torch.int32)))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("read")
        g.read_affected(out=out)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print("read profiled", rows.shape[0], col.shape[0])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cusparse", action="store_true", help="skip the cuSPARSE static-product comparator")
    ap.add_argument("--no-masked", action="store_true",
                    help="skip the masked-path leg (Algorithm 2 beside the row path on R-MAT scale 20)")
    ap.add_argument("--profile", choices=["step", "static", "read"], default=None,
                    help="run one NVTX-marked step, static recompute or read of a step's affected rows for ncu, "
                         "then exit")
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--workload", choices=["stencil", "rmat20", "rmat21", "batched", "learned"], default="stencil",
                    help="stencil: the 128^3 stencil with 10^4-update batches; rmat20: R-MAT scale 20 (min,+) "
                         "A B with 10^3-edge batches; rmat21: R-MAT scale 21 (+,.) A A with 10^3-edge batches; "
                         "batched: 256 R-MAT instances; learned: learned vs exact vs bound sizing and the serving "
                         "loop on R-MAT scale 21")
    ap.add_argument("--autotune", type=int, default=0,
                    help="stencil/rmat20: choose the row bins on this many calibration batches before timing")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--scale", type=int, default=21)
    ap.add_argument("--train-graphs", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--est-min", type=int, default=128)
    ap.add_argument("--est-margin", type=float, default=0.25)
    ap.add_argument("--compare-batches", type=int, default=16)
    ap.add_argument("--requests", type=int, default=300)
    ap.add_argument("--max-wave", type=int, default=32)
    args = ap.parse_args()
    if args.profile:
        profile_arm(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batched":
        batched_arm(args)
    elif args.workload == "learned":
        learned_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
