"""Serving loop: a stream of update batches against one device-resident
handle, with continuous batching.

Requests (update batches of A) arrive over time.  Each turn of the loop
takes the requests that have arrived and not yet run, in arrival order, and
admits as many as it can into one *wave*, applied as a single batch (the
requests concatenated in arrival order, so the last write of an entry wins
exactly as if they ran one by one):

- a request joins only if its footprint (the rows of C it can touch, and
  the rows its entries could connect) shares no row with the footprints
  already in the wave, nor with the wave still being read back (below); by
  default the first request that conflicts ends the wave.  With
  ``overtake`` a conflicting request is passed over instead and its
  footprint still counts, so a later request joins only if it meets none of
  the footprints examined before it: it overtakes only requests it commutes
  with, and conflicting requests stay in arrival order;
- at most ``max_wave`` requests and ``max_wave_entries`` update entries per
  wave (the slots);
- and only while the wave's estimated device memory (its batch and working
  buffers, and the C rows it will read back) fits in the free HBM reported
  by the driver, minus ``hbm_reserve`` bytes.

Waves are pipelined on the GPU (``pipelined``, the default with a GPU): a
turn admits the next wave from everything that has arrived by then -- while
the previous wave's rows have not been read back yet -- with one batched
footprint call (``dspg_footprint_batch``), starts it without waiting
(``dspg_apply_batch_async``), reads the previous wave's rows on a second
stream while it runs, and only then waits for it.  The previous wave's rows
lie outside the running wave's footprint, so reading them meanwhile is
exact.  A request that conflicts with the wave being read waits until that
read is done.  The result of a request is its affected rows of C (the rows
of its wave's affected set inside its footprint) right after its wave
commits, which, by the disjointness, is the result it would have had alone
in arrival order: see ``tests/test_gpu_serving.py``.  All computation is in
the library's kernels; this module schedules, moves data, and sorts each
wave's affected rows to its requests.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class UpdateBatch:
    """Host arrays of an update batch: row, col, val, op (include/dspg.h)."""
    row: np.ndarray
    col: np.ndarray
    val: np.ndarray
    op: np.ndarray

    def __len__(self) -> int:
        return int(self.row.shape[0])


def concat(batches) -> UpdateBatch:
    """Batches concatenated in order (the last write of an entry wins)."""
    return UpdateBatch(np.concatenate([b.row for b in batches]), np.concatenate([b.col for b in batches]),
                       np.concatenate([b.val for b in batches]), np.concatenate([b.op for b in batches]))


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start of the stream
    batch: object   # host (numpy) arrays row, col, val, op, as UpdateBatch


@dataclass
class Result:
    rid: int
    arrival: float
    start: float     # wave launch, seconds after the start
    done: float      # results read back
    wave: int
    wave_size: int
    rows: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    rowptr: np.ndarray | None = None
    col: np.ndarray | None = None
    val: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    """Continuous-batching server over one DynamicSpGEMM handle (C = A B with
    updates of A; C = A A in the intended use)."""

    def __init__(self, g, max_wave: int = 32, max_wave_entries: int = 1 << 21, hbm_reserve: int = 4 << 30,
                 read_results: bool = True, hbm_free=None, overtake: bool = False, scan: int | None = None,
                 bitmap_device: str = "cuda", pipelined: bool | None = None):
        """bitmap_device: where the footprint bitmaps live.  The library
        writes them on the GPU ("cuda"); "cpu" is for driving the scheduling
        alone with a stand-in for the handle (the host-logic tests)."""
        import torch
        self.g = g
        self.bitmap_device = bitmap_device
        self.max_wave = max_wave
        self.overtake = overtake  # pass over a conflicting request instead of ending the wave
        self.scan = scan if scan is not None else 4 * max_wave  # queued requests examined per wave
        self.max_wave_entries = max_wave_entries
        self.hbm_reserve = hbm_reserve
        self.read_results = read_results
        self._free = hbm_free or (lambda: torch.cuda.mem_get_info()[0])
        info = g.info()
        self.n = info["n"]
        self.c_row_bytes = (info["nnz_c"] / max(self.n, 1)) * (4 + (8 if g.sr == 0 else 4))
        self.words = (self.n + 31) // 32
        self._union = torch.zeros(self.words, dtype=torch.int32, device=bitmap_device)
        self._fp = [torch.zeros(self.words, dtype=torch.int32, device=bitmap_device) for _ in range(max_wave)]
        self._pin = None
        self.waves = 0
        self.conflicts = 0
        self.memory_stops = 0
        self.pipelined = (bitmap_device != "cpu") if pipelined is None else pipelined
        self.trace = []  # pipelined: (wave, "apply" or "read", start event, end event)
        self._base = None
        if self.pipelined:
            self._fstack = torch.zeros((self.scan, self.words), dtype=torch.int32, device=bitmap_device)
            self._wave_union = torch.zeros(self.words, dtype=torch.int32, device=bitmap_device)

    def _stage(self, b: UpdateBatch) -> UpdateBatch:
        """The wave's batch in pinned host memory (buffers kept and grown), so
        its upload is a plain asynchronous copy."""
        import torch
        n = len(b)
        if self._pin is None or self._pin[0].shape[0] < n:
            cap = max(n, 1024) * 2
            pin = self.bitmap_device != "cpu"

            def buf(dt):
                t = torch.empty(cap, dtype=dt)
                return t.pin_memory() if pin else t

            self._pin = (buf(torch.int32), buf(torch.int32), buf(torch.from_numpy(b.val[:0]).dtype), buf(torch.uint8))
        r, c, v, o = self._pin
        r[:n].numpy()[:] = b.row
        c[:n].numpy()[:] = b.col
        v[:n].numpy()[:] = b.val
        o[:n].numpy()[:] = b.op
        return UpdateBatch(r[:n], c[:n], v[:n], o[:n])

    def _wave_bytes(self, entries: int, fp_rows: int) -> float:
        # device copy of the batch + sort/merge buffers (~64 B per entry) and
        # the rows of C read back for the wave
        return 64.0 * entries + 2.0 * fp_rows * self.c_row_bytes

    def serve(self, requests: list[Request], clock=time.perf_counter) -> list[Result]:
        """Serve the requests; pipelined waves unless ``pipelined`` is off."""
        if self.pipelined:
            return self._serve_pipelined(requests, clock)
        return self._serve_waves(requests, clock)

    def _admit(self, queue, stream, limit):
        """The next wave: at most `limit` candidates from the head of the
        queue (slots and entries), footprints and admission in one call
        against the union already in self._union, then the memory budget.
        Returns (wave as (request, footprint row) pairs, queue positions
        taken)."""
        cands, entries = [], 0
        for req in queue[: min(self.scan, limit)]:
            if len(cands) >= self.max_wave:
                break
            if cands and entries + len(req.batch) > self.max_wave_entries:
                break
            cands.append(req)
            entries += len(req.batch)
        if self.max_wave == 1 and not cands:
            return [], []
        admitted, rows = self.g.footprint_batch([r.batch for r in cands], self._fstack[: len(cands)], self._union,
                                                or_anyway=self.overtake, stream=stream)
        budget = self._free() - self.hbm_reserve
        wave, taken, fp_rows, entries = [], [], 0, 0
        for j, (req, ok) in enumerate(zip(cands, admitted)):
            if not ok:
                self.conflicts += 1
                if self.overtake:
                    continue
                break
            if wave and self._wave_bytes(entries + len(req.batch), fp_rows + rows[j]) > budget:
                self.memory_stops += 1
                break
            wave.append((req, j))
            taken.append(j)
            fp_rows += rows[j]
            entries += len(req.batch)
        return wave, taken

    def _finish(self, w, results, clock, t0, stream):
        """Read a committed wave's rows (on `stream`) and hand each request
        the rows of the wave's affected set inside its own footprint."""
        import torch
        R, labels = w["R"], w["labels"]
        if self.read_results:
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            rp, col, val = self.g.read_rows_C(R, stream=stream)
            ev1.record(stream)
            self.trace.append((w["wave"], "read", ev0, ev1))
        done = clock() - t0
        for slot, req in enumerate(w["reqs"]):
            pos = np.nonzero(labels == slot)[0] if len(w["reqs"]) > 1 else np.arange(R.shape[0])
            res = Result(req.rid, req.arrival, w["start"], done, w["wave"], len(w["reqs"]), R[pos])
            if self.read_results:
                lens = rp[pos + 1] - rp[pos]
                res.rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
                idx = np.repeat(rp[pos], lens) + (np.arange(int(lens.sum())) - np.repeat(res.rowptr[:-1], lens))
                res.col, res.val = col[idx], val[idx]
            results.append(res)

    def _serve_pipelined(self, requests: list[Request], clock=time.perf_counter) -> list[Result]:
        import torch
        order = sorted(requests, key=lambda r: (r.arrival, r.rid))
        results: list[Result] = []
        queue: list[Request] = []
        nxt = 0
        run_stream = torch.cuda.Stream()
        read_stream = torch.cuda.Stream()
        self._base = torch.cuda.Event(enable_timing=True)
        self._base.record(run_stream)
        inflight = None  # the committed wave whose rows are still to be read
        # running averages: requests per wave (how many candidates a turn
        # examines) and how often the wave being read blocked the next one
        # (then the loop reads first and admits after, instead of admitting
        # twice)
        avg_wave, blocked = 1.0, 0.0
        turn = 0
        t0 = clock()
        while nxt < len(order) or queue or inflight is not None:
            now = clock() - t0
            while nxt < len(order) and order[nxt].arrival <= now:
                queue.append(order[nxt])
                nxt += 1
            if not queue and inflight is None:
                time.sleep(max(0.0, min(order[nxt].arrival - now, 0.01)))
                continue
            wave, taken = [], []
            if queue and inflight is not None and blocked > 0.5:
                self._finish(inflight, results, clock, t0, read_stream)
                inflight = None
            if queue:
                # the wave being read back keeps its rows: admissions avoid them
                if inflight is not None:
                    self._union.copy_(self._wave_union)
                else:
                    self._union.zero_()
                # a footprint costs about a detection pass, and the ones of
                # candidates left in the queue are computed again next turn
                # (A changes in between): while waves hold one request, a turn
                # examines the head only, and every fourth turn a few more,
                # so that waves can grow again
                turn += 1
                limit = 1 if (avg_wave < 1.2 and turn % 4) else max(2, int(2 * avg_wave + 1))
                wave, taken = self._admit(queue, run_stream, limit)
                if inflight is not None:
                    blocked = 0.8 * blocked + 0.2 * (0.0 if wave else 1.0)
                if not wave and inflight is None and queue:
                    raise RuntimeError("no request admitted against an empty wave")
                if wave:
                    avg_wave = 0.8 * avg_wave + 0.2 * len(wave)
            if wave:
                keep = set(taken)
                cand = queue[: max(taken) + 1]
                queue = [r for k, r in enumerate(cand) if k not in keep] + queue[len(cand):]
                start = clock() - t0
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(run_stream)
                self.g.apply_batch_async(self._stage(concat([r.batch for r, _ in wave])), stream=run_stream)
                ev1.record(run_stream)
                self.trace.append((self.waves, "apply", ev0, ev1))
            if inflight is not None:  # meanwhile: the previous wave's rows
                self._finish(inflight, results, clock, t0, read_stream)
                inflight = None
            if wave:
                self.g.apply_batch_wait(stream=run_stream)
                R = self.g.last_affected(stream=run_stream)
                labels = None
                if len(wave) > 1 and R.shape[0]:
                    Rt = torch.from_numpy(R.astype(np.int64)).to(self._fstack.device)
                    word, bit = Rt >> 5, (Rt & 31).to(torch.int32)
                    lab = torch.full((R.shape[0],), -1, dtype=torch.int32, device=Rt.device)
                    for slot, (_, j) in enumerate(wave):
                        hit = ((self._fstack[j][word] >> bit) & 1).bool()
                        lab[hit] = slot
                    labels = lab.cpu().numpy()
                self._wave_union.zero_()
                for _, j in wave:
                    self._wave_union |= self._fstack[j]
                inflight = {"reqs": [r for r, _ in wave], "R": R, "labels": labels, "start": start,
                            "wave": self.waves}
                self.waves += 1
        torch.cuda.synchronize()
        return results

    def overlaps(self) -> int:
        """Pipelined runs: how many wave reads ran while the next wave's
        apply was on the GPU (their event intervals intersect)."""
        if self._base is None:
            return 0
        span = {}
        for w, kind, e0, e1 in self.trace:
            span[(w, kind)] = (self._base.elapsed_time(e0), self._base.elapsed_time(e1))
        n = 0
        for (w, kind), (r0, r1) in span.items():
            if kind != "read" or (w + 1, "apply") not in span:
                continue
            a0, a1 = span[(w + 1, "apply")]
            n += max(r0, a0) < min(r1, a1)
        return n

    def _serve_waves(self, requests: list[Request], clock=time.perf_counter) -> list[Result]:
        import torch

        order = sorted(requests, key=lambda r: (r.arrival, r.rid))
        results: list[Result] = []
        queue: list[Request] = []
        nxt = 0
        t0 = clock()
        while nxt < len(order) or queue:
            now = clock() - t0
            while nxt < len(order) and order[nxt].arrival <= now:
                queue.append(order[nxt])
                nxt += 1
            if not queue:
                time.sleep(max(0.0, min(order[nxt].arrival - now, 0.01)))
                continue
            # admit a wave: scan the queue in arrival order; a request joins if
            # its footprint is disjoint from everything scanned before it (the
            # wave, and with overtake the requests passed over), so a request
            # only ever overtakes earlier ones it commutes with
            self._union.zero_()
            wave, fps, fp_rows, entries = [], [], 0, 0
            budget = self._free() - self.hbm_reserve
            taken = []  # queue positions admitted
            for qi, req in enumerate(queue[: self.scan]):
                if len(wave) >= self.max_wave:
                    break
                if self.max_wave == 1:  # a plain queue: one request per wave, no footprint needed
                    wave.append(req)
                    fps.append(None)
                    taken.append(qi)
                    break
                f = self._fp[len(wave)]
                # the footprint and the admission test against the wave's rows
                # in one call (a wave that closes below drops its bitmap anyway)
                rows_f, disjoint = self.g.footprint(req.batch, f, self._union, or_anyway=self.overtake)
                fits = not wave or (entries + len(req.batch) <= self.max_wave_entries and
                                    self._wave_bytes(entries + len(req.batch), fp_rows + rows_f) <= budget)
                if not fits:
                    self.memory_stops += 1
                    break
                if not disjoint:
                    self.conflicts += 1
                    if self.overtake:
                        continue
                    break
                wave.append(req)
                fps.append(f)
                taken.append(qi)
                fp_rows += rows_f
                entries += len(req.batch)
            keep = set(taken)
            queue = [r for qi, r in enumerate(queue) if qi not in keep]
            start = clock() - t0
            self.g.apply_batch(self._stage(concat([r.batch for r in wave])))
            R = self.g.last_affected()
            if len(wave) > 1:  # each request's rows: the wave's affected rows inside its footprint
                fps = [f.cpu().numpy().view(np.uint32) for f in fps]
            for req, fbits in zip(wave, fps):
                if fbits is None or len(wave) == 1:
                    rows = R
                else:
                    rows = R[((fbits[R >> 5] >> (R & 31).astype(np.uint32)) & 1) != 0] if R.shape[0] else R
                res = Result(req.rid, req.arrival, start, 0.0, self.waves, len(wave), rows)
                if self.read_results:
                    res.rowptr, res.col, res.val = self.g.read_rows_C(rows)
                res.done = clock() - t0
                results.append(res)
            self.waves += 1
        return results


def latency_summary(results: list[Result], wall: float | None = None) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    span = wall if wall is not None else (max(r.done for r in results) - min(r.arrival for r in results))
    sizes = np.array([r.wave_size for r in results])
    return {"requests": len(results), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "throughput_req_s": round(len(results) / span, 2), "mean_wave_size": round(float(sizes.mean()), 2)}
