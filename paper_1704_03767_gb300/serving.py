"""Continuous-batching query server over a database kept resident in HBM (query-based
co-expression search, Sec. 1 of the paper).

The database is ranked once and its tensor-core operands are built once; they stay on the GPU.
Clients submit batches of query profiles (b x n) at any time. One worker thread per stream slot
takes pending batches in arrival order whenever a slot is free and the batch's device memory fits
the budget still unreserved (the worker that wakes first admits the head of the queue and runs
it on the slot's own CUDA stream):

    host->device copy of the profiles, ktau_rank_prepare_async, ktau_query (exact tau-b against every
    database row + exact top-k by |tau|), device->host copy of the top-k

so batches that arrive while others are on the GPU overlap with them. When several batches are
pending, consecutive ones (in arrival order, up to max_batch profiles and within the memory budget)
are merged into one launch and their rows split back afterwards: under load this amortises the
per-launch host work. The result of a batch does not depend on what else is in flight or merged
with it: every query row is scored against the database on its own (exact integer counts formed
into tau by one fixed epilogue, top-k per row).

All computation is in libktau.so; this module is host-side scheduling only.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np
import torch

from . import binding as kb


@dataclasses.dataclass
class Request:
    rid: int
    queries: np.ndarray           # [b, n] float32 (host)
    arrival: float                # time.perf_counter() at submission (or the scheduled time)
    admitted: float = 0.0
    finished: float = 0.0
    topk_idx: np.ndarray | None = None
    topk_tau: np.ndarray | None = None
    tau: torch.Tensor | None = None   # [b, m_db] FP64 on the device when keep_tau
    error: str | None = None
    reserved: int = 0
    slot: int = -1
    done: threading.Event = dataclasses.field(default_factory=threading.Event)

    cancelled: bool = False

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Admission:
    """Admission by device memory: a batch enters when its estimated footprint fits the budget
    that in-flight batches have not reserved, and a stream slot is free. Batches are admitted in
    arrival order (no overtaking)."""

    def __init__(self, budget_bytes: int, slots: int):
        self.budget = int(budget_bytes)
        self.reserved = 0
        self.free_slots = list(range(slots))

    def try_admit(self, need: int):
        if not self.free_slots:
            return None
        if need > self.budget:
            raise ValueError(f"batch needs {need} bytes, more than the whole budget {self.budget}")
        if self.reserved + need > self.budget:
            return None
        self.reserved += need
        return self.free_slots.pop(0)

    def release(self, slot: int, need: int):
        self.reserved -= need
        self.free_slots.append(slot)
        self.free_slots.sort()


class QueryServer:
    def __init__(self, db: np.ndarray | torch.Tensor, k: int = 100, slots: int = 4,
                 mem_budget: int | None = None, keep_tau: bool = False, options=None,
                 device: int = 0, max_batch: int = 512, merge: bool = True):
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        dbt = torch.as_tensor(db).to(self.dev, dtype=torch.float32).contiguous()
        self.db = kb.ktau_rank_prepare(dbt)
        self.m_db, self.n = dbt.shape
        self.k = min(k, self.m_db)
        self.options = options
        self.keep_tau = keep_tau
        if kb.ktau_allpairs_path(self.db) == kb.KTAU_PATH_SIGNGEMM:
            kb.ktau_prepare_signs(self.db)  # resident tensor-core operands of the database
        torch.cuda.synchronize(self.dev)
        del dbt
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            mem_budget = int(free * 0.6)
        self.admission = Admission(mem_budget, slots)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        # Per-slot buffers for batches of up to max_batch profiles, allocated once: the request
        # path then allocates nothing but the batch's ranked handle (from the library's cache).
        self.max_batch = max_batch
        self.merge = merge
        self.slot_buf = []
        for _ in range(slots):
            self.slot_buf.append({
                "qh": torch.empty((max_batch, self.n), dtype=torch.float32).pin_memory(),
                "qd": torch.empty((max_batch, self.n), dtype=torch.float32, device=self.dev),
                "S": torch.empty((max_batch, self.m_db), dtype=torch.int32, device=self.dev),
                "idx": torch.empty((max_batch, self.k), dtype=torch.int32, device=self.dev),
                "tk": torch.empty((max_batch, self.k), dtype=torch.float64, device=self.dev),
                "idx_h": torch.empty((max_batch, self.k), dtype=torch.int32).pin_memory(),
                "tk_h": torch.empty((max_batch, self.k), dtype=torch.float64).pin_memory()})
        self.cv = threading.Condition()
        self.pending = collections.deque()
        self.running = True
        self.next_id = 0
        self.timeline = []  # (rid, slot, admitted, finished)
        self.threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(slots)]
        for t in self.threads:
            t.start()

    # -- memory estimate of one batch (outputs + query ranks + library scratch)
    def footprint(self, b: int) -> int:
        ld = (self.n + 15) // 16 * 16
        ranked = b * ld * 6 + b * 64 + 4096
        outs = b * self.m_db * 4 + b * self.k * 12
        if self.keep_tau:
            outs += b * self.m_db * 8
        return ranked + outs + kb.ktau_query_scratch_bytes(self.db, b, self.k)

    def submit(self, queries, arrival: float | None = None) -> Request:
        q = np.ascontiguousarray(np.asarray(queries, dtype=np.float32))
        if q.ndim != 2 or q.shape[1] != self.n:
            raise ValueError(f"queries must be [b, {self.n}]")
        with self.cv:
            r = Request(self.next_id, q, time.perf_counter() if arrival is None else arrival)
            self.next_id += 1
            self.pending.append(r)
            self.cv.notify_all()
        return r

    def cancel(self, r: Request) -> bool:
        """Withdraws a request that has not been admitted yet; True when it was withdrawn (its
        `error` says so and `done` is set). Admitted requests run to completion."""
        with self.cv:
            try:
                self.pending.remove(r)
            except ValueError:
                return False
            r.cancelled = True
            r.error = "cancelled"
            r.finished = time.perf_counter()
            r.done.set()
            self.cv.notify_all()
            return True

    def _take(self):
        """Under the lock: the next group to run and its slot, or None to wait. The head of the
        queue, plus the consecutive requests behind it that fit in one launch; admitted when a
        slot is free and its memory fits (no overtaking)."""
        group = [self.pending[0]]
        rows = group[0].queries.shape[0]
        if self.merge and rows <= self.max_batch:
            for r in list(self.pending)[1:]:
                b = r.queries.shape[0]
                if rows + b > self.max_batch:
                    break
                group.append(r)
                rows += b
        need = self.footprint(rows)
        if need > self.admission.budget and len(group) > 1:
            group, rows = group[:1], group[0].queries.shape[0]
            need = self.footprint(rows)
        try:
            slot = self.admission.try_admit(need)
        except ValueError as e:  # larger than the whole budget: rejected
            r = self.pending.popleft()
            r.error = str(e)
            r.finished = time.perf_counter()
            r.done.set()
            return "rejected"
        if slot is None:
            return None
        now = time.perf_counter()
        for r in group:
            self.pending.popleft()
            r.slot, r.admitted = slot, now
        group[0].reserved = need
        return group, slot

    def _worker(self):
        torch.cuda.set_device(self.dev)
        while True:
            with self.cv:
                while True:
                    if not self.pending:
                        if not self.running:
                            return
                        self.cv.wait()
                        continue
                    got = self._take()
                    if got == "rejected":
                        continue
                    if got is None:
                        self.cv.wait()  # a slot or memory frees up when a batch finishes
                        continue
                    group, slot = got
                    break
            try:
                self._run(group, self.streams[slot], slot)
            except Exception as e:  # reported on the requests; the server keeps running
                for r in group:
                    r.error = repr(e)
            now = time.perf_counter()
            with self.cv:
                self.admission.release(slot, group[0].reserved)
                for r in group:
                    r.finished = now
                    self.timeline.append((r.rid, r.slot, r.admitted, r.finished))
                self.cv.notify_all()
            for r in group:
                r.done.set()

    def _run(self, group, st: torch.cuda.Stream, slot: int):
        sizes = [r.queries.shape[0] for r in group]
        b = sum(sizes)
        with torch.cuda.stream(st):
            if b <= self.max_batch:
                buf = self.slot_buf[slot]
                qh = buf["qh"][:b].numpy()
                o = 0
                for r, sz in zip(group, sizes):
                    qh[o:o + sz] = r.queries
                    o += sz
                qd = buf["qd"][:b]
                qd.copy_(buf["qh"][:b], non_blocking=True)
                S, idx, tk = buf["S"][:b], buf["idx"][:b], buf["tk"][:b]
                idx_h, tk_h = buf["idx_h"][:b], buf["tk_h"][:b]
            else:  # one request larger than the slot buffers: buffers of its own
                qd = torch.from_numpy(group[0].queries).pin_memory().to(self.dev,
                                                                         non_blocking=True)
                S = torch.empty((b, self.m_db), dtype=torch.int32, device=self.dev)
                idx = torch.empty((b, self.k), dtype=torch.int32, device=self.dev)
                tk = torch.empty((b, self.k), dtype=torch.float64, device=self.dev)
                idx_h = torch.empty((b, self.k), dtype=torch.int32).pin_memory()
                tk_h = torch.empty((b, self.k), dtype=torch.float64).pin_memory()
            # No host round trip between the rank transform and the query: the statistics copy is
            # read when ktau_query needs it.
            R = kb.ktau_rank_prepare_async(qd, st)
            tau = torch.empty((b, self.m_db), dtype=torch.float64, device=self.dev) \
                if self.keep_tau else None
            kb.ktau_query(self.db, R, tau, S, None, 32, self.k, idx, tk, self.options, st)
            idx_h.copy_(idx, non_blocking=True)
            tk_h.copy_(tk, non_blocking=True)
            R.free_on(st)  # waits for this slot's stream only
        # copies: the slot's pinned buffers are reused by its next launch
        o = 0
        for r, sz in zip(group, sizes):
            r.topk_idx = idx_h[o:o + sz].numpy().copy()
            r.topk_tau = tk_h[o:o + sz].numpy().copy()
            r.tau = tau[o:o + sz] if tau is not None else None
            o += sz

    def stop(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        for t in self.threads:
            t.join(timeout=30)
        self.db.free()


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    i = min(len(xs) - 1, max(0, int(round(p / 100.0 * (len(xs) - 1)))))
    return xs[i]


def run_open_loop(server: QueryServer, batches, rate_per_s: float, arrivals=None):
    """Submits `batches` as a Poisson stream of the given rate (arrival times from
    synthetic.poisson_arrivals when not given) and waits for all. Returns the requests."""
    from synthetic import poisson_arrivals

    arr = poisson_arrivals(len(batches), rate_per_s) if arrivals is None else arrivals
    t0 = time.perf_counter()
    reqs = []
    for a, q in zip(arr, batches):
        now = time.perf_counter() - t0
        if a > now:
            time.sleep(a - now)
        reqs.append(server.submit(q, arrival=t0 + a))
    for r in reqs:
        r.done.wait()
    return reqs
