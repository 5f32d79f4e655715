"""Serving loop: a stream of update batches against one device-resident
handle, with continuous batching.

Requests (update batches of A) arrive over time.  Each turn of the loop
takes the requests that have arrived and not yet run, in arrival order, and
admits as many as it can into one *wave*, applied as a single batch (the
requests concatenated in arrival order, so the last write of an entry wins
exactly as if they ran one by one):

- a request joins only if its footprint (``dspg_footprint``: the rows of C
  it can touch, and the rows its entries could connect) shares no row with
  the footprints already in the wave; by default the first request that
  conflicts ends the wave.  With ``overtake`` a conflicting request is passed
  over instead and its footprint still counts, so a later request joins only
  if it meets none of the footprints examined before it: it overtakes only
  requests it commutes with, and conflicting requests stay in arrival order;
- at most ``max_wave`` requests and ``max_wave_entries`` update entries per
  wave (the slots);
- and only while the wave's estimated device memory (its batch and working
  buffers, and the C rows it will read back) fits in the free HBM reported
  by the driver, minus ``hbm_reserve`` bytes.

Requests that arrive while a wave runs on the GPU wait for the next turn.
The result of a request is its affected rows of C (the rows of the wave's
affected set inside its footprint) right after its wave commits, which, by
the disjointness, is the result it would have had alone in arrival order:
see ``tests/test_gpu_serving.py``.  All computation is in the library's
kernels; this module only schedules and moves data.
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
                 bitmap_device: str = "cuda"):
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
