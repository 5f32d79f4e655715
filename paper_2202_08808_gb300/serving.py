"""Serving loop: a stream of update batches against one device-resident
handle, with continuous batching.

Requests (update batches of A) arrive over time.  Each turn of the loop
takes the requests that have arrived and not yet run, in arrival order, and
admits as many as it can into one *wave*, applied as a single batch (the
requests concatenated in arrival order, so the last write of an entry wins
exactly as if they ran one by one):

- a request joins only if its footprint (``dspg_footprint``: the rows of C
  it can touch, and the rows its entries could connect) shares no row with
  the footprints already in the wave; the first one that conflicts ends the
  wave, so no request ever overtakes an earlier one;
- at most ``max_wave`` requests and ``max_wave_entries`` update entries per
  wave (the slots);
- and only while the wave's estimated device memory (its batch and working
  buffers, and the C rows it will read back) fits in the free HBM reported
  by the driver, minus ``hbm_reserve`` bytes.

Requests that arrive while a wave runs on the GPU wait for the next turn.
The result of a request is its affected rows of C (the rows of the wave's
affected set inside its footprint) right after its wave commits, which, by
the disjointness, is the result it would have had alone: see
``tests/test_gpu_serving.py``.  All computation is in the library's
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
                 read_results: bool = True, hbm_free=None):
        import torch
        self.g = g
        self.max_wave = max_wave
        self.max_wave_entries = max_wave_entries
        self.hbm_reserve = hbm_reserve
        self.read_results = read_results
        self._free = hbm_free or (lambda: torch.cuda.mem_get_info()[0])
        info = g.info()
        self.n = info["n"]
        self.c_row_bytes = (info["nnz_c"] / max(self.n, 1)) * (4 + (8 if g.sr == 0 else 4))
        self.words = (self.n + 31) // 32
        self._union = torch.zeros(self.words, dtype=torch.int32, device="cuda")
        self._fp = [torch.zeros(self.words, dtype=torch.int32, device="cuda") for _ in range(max_wave)]
        self.waves = 0
        self.conflicts = 0
        self.memory_stops = 0

    def _wave_bytes(self, entries: int, fp_rows: int) -> float:
        # device copy of the batch + sort/merge buffers (~64 B per entry) and
        # the rows of C read back for the wave
        return 64.0 * entries + 2.0 * fp_rows * self.c_row_bytes

    def serve(self, requests: list[Request], clock=time.perf_counter) -> list[Result]:
        import torch

        from .dspg import bitmap_admit

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
            # admit a wave
            self._union.zero_()
            wave, fps, fp_rows, entries = [], [], 0, 0
            budget = self._free() - self.hbm_reserve
            for req in queue:
                if len(wave) >= self.max_wave or (wave and entries + len(req.batch) > self.max_wave_entries):
                    break
                f = self._fp[len(wave)]
                f.zero_()
                self.g.footprint(req.batch, f)
                fbits = f.cpu().numpy().view(np.uint32)
                rows_f = _popcount(fbits)
                if wave and self._wave_bytes(entries + len(req.batch), fp_rows + rows_f) > budget:
                    self.memory_stops += 1
                    break
                if not bitmap_admit(f, self._union):
                    self.conflicts += 1
                    break
                wave.append(req)
                fps.append(fbits)
                fp_rows += rows_f
                entries += len(req.batch)
            queue = queue[len(wave):]
            start = clock() - t0
            cat = concat([r.batch for r in wave])
            pinned = UpdateBatch(torch.from_numpy(cat.row).pin_memory(), torch.from_numpy(cat.col).pin_memory(),
                                 torch.from_numpy(cat.val).pin_memory(), torch.from_numpy(cat.op).pin_memory())
            self.g.apply_batch(pinned)
            R = self.g.last_affected()
            for req, fbits in zip(wave, fps):
                rows = R[((fbits[R >> 5] >> (R & 31).astype(np.uint32)) & 1) != 0] if R.shape[0] else R
                res = Result(req.rid, req.arrival, start, 0.0, self.waves, len(wave), rows)
                if self.read_results:
                    res.rowptr, res.col, res.val = self.g.read_rows_C(rows)
                res.done = clock() - t0
                results.append(res)
            self.waves += 1
        return results


def _popcount(words: np.ndarray) -> int:
    if hasattr(np, "bitwise_count"):
        return int(np.bitwise_count(words).sum())
    return int(np.unpackbits(words.view(np.uint8)).sum())


def latency_summary(results: list[Result], wall: float | None = None) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    span = wall if wall is not None else (max(r.done for r in results) - min(r.arrival for r in results))
    sizes = np.array([r.wave_size for r in results])
    return {"requests": len(results), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "throughput_req_s": round(len(results) / span, 2), "mean_wave_size": round(float(sizes.mean()), 2)}
