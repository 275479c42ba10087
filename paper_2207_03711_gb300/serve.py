"""Continuous-batching request loop for VQE energy and gradient requests.

Requests of different sizes (qubits, bond dimension, precision) are admitted while
device memory allows. Each admitted request owns an MPS handle on its own CUDA stream,
so the gate chains of all requests in flight run side by side on the device (one thread
block, i.e. one SM, per evaluation slot); a request that finishes releases its memory and
the loop admits the next ones that fit (first fit in arrival order). Every result is
computed by the same deterministic kernels as a lone call, so it does not depend on what
else is in flight. A request can be cancelled (Future.cancel) until it starts running.
Latencies (submit to result) give p50/p99 beside the throughput.

First fit lets small requests pass a large one that does not fit yet; so that a steady
stream of small requests cannot starve it, once the oldest queued request has waited
longer than max_wait_s nothing behind it is admitted until it fits (head-of-line
reservation). Handles take and return device memory stream-ordered on their own stream,
so a request that finishes does not wait for the launches of the others.

The host objects of a request (Jordan-Wigner Hamiltonian with its prefix trie, compiled
circuit) are built at submission, because the device-memory estimate needs their sizes.
"""
import collections
import concurrent.futures
import threading
import time

import numpy as np

from . import (MPS_MIXED, circ_create, circ_get_rotations, circ_set_reference, circ_uccsd,
               ham_jw_from_integrals, mps_create, mps_estimate_bytes, vqe_energy, vqe_gradient)


def uccsd_circuit(n_qubits, n_electrons, n_doubles=None):
    """The UCCSD circuit, or (n_doubles given) its singles plus the first n_doubles
    doubles in canonical order, on the Hartree-Fock reference."""
    full = circ_uccsd(n_qubits, n_electrons)
    if n_doubles is None:
        return full
    n_singles = 2 * (n_electrons // 2) * ((n_qubits - n_electrons) // 2)
    paulis, pidx, scale = circ_get_rotations(full)
    keep = pidx < n_singles + n_doubles
    c = circ_create(paulis[keep], pidx[keep], scale[keep])
    circ_set_reference(c, np.array([1] * n_electrons + [0] * (n_qubits - n_electrons), dtype=np.uint8))
    return c


class Request:
    """kind: "energy" or "gradient"; h, eri: spatial-orbital integrals (chemist order);
    theta: UCCSD amplitudes; sel: parameter indices of a gradient request; n_slots:
    slots of the gradient's handle (shared-prefix forks run (n_slots - 1) / 2 rotations
    per pass); n_doubles: keep the singles and the first n_doubles doubles only."""

    def __init__(self, kind, h, eri, n_electrons, chi, theta, precision=MPS_MIXED, sel=None, n_slots=None,
                 tag=None, n_doubles=None):
        if kind not in ("energy", "gradient"):
            raise ValueError(f"unknown request kind {kind!r}")
        self.kind, self.h, self.eri = kind, np.asarray(h), np.asarray(eri)
        self.n_electrons, self.chi, self.precision = int(n_electrons), int(chi), precision
        self.theta = np.asarray(theta, dtype=np.float64)
        self.sel = None if sel is None else np.asarray(sel, dtype=np.int32)
        self.n_slots = n_slots if n_slots is not None else (1 if kind == "energy" else 9)
        self.tag = tag
        self.n_doubles = n_doubles
        self.n_qubits = 2 * self.h.shape[0]


class _Item:
    __slots__ = ("req", "ham", "circ", "need", "future", "t_submit", "t_start", "t_done")


class Server:
    """budget_bytes: device bytes the loop may hand out (default: 80 % of the free device
    memory at construction); max_inflight: requests running at once; max_wait_s: queue
    age after which the oldest request reserves the head of the line. run_fn replaces
    the device execution (host-logic tests); it receives the request and returns its
    value."""

    def __init__(self, budget_bytes=None, max_inflight=16, device=0, run_fn=None, max_wait_s=30.0):
        self._run_fn = run_fn
        self.max_wait_s = float(max_wait_s)
        self._device = device
        if budget_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            budget_bytes = int(0.8 * free)
        self.budget = int(budget_bytes)
        self.max_inflight = int(max_inflight)
        self.used = 0
        self.peak_used = 0
        self.inflight = 0
        self.peak_inflight = 0
        self._queue = collections.deque()
        self._cv = threading.Condition()
        self._closed = False
        self._records = []
        self._t0 = time.perf_counter()
        self._admitter = threading.Thread(target=self._admit_loop, daemon=True)
        self._admitter.start()

    # ------------------------------------------------------------------ submission
    def submit(self, req, need_bytes=None):
        it = _Item()
        it.req = req
        it.future = concurrent.futures.Future()
        it.t_submit = time.perf_counter()
        it.t_start = it.t_done = None
        it.ham = it.circ = None
        if need_bytes is None:
            it.ham = ham_jw_from_integrals(req.h, req.eri)
            it.circ = uccsd_circuit(req.n_qubits, req.n_electrons, req.n_doubles)
            need_bytes = mps_estimate_bytes(req.n_qubits, req.chi, req.precision, req.n_slots, it.circ, it.ham)
        it.need = int(need_bytes)
        if it.need > self.budget:
            it.future.set_exception(MemoryError(f"request needs {it.need} B, budget is {self.budget} B"))
            return it.future
        with self._cv:
            if self._closed:
                raise RuntimeError("server is closed")
            self._queue.append(it)
            self._cv.notify_all()
        return it.future

    # ------------------------------------------------------------------ scheduling
    def _admit_loop(self):
        while True:
            with self._cv:
                while True:
                    if self._closed and not self._queue:
                        return
                    picked = []
                    for it in [q for q in self._queue if q.future.cancelled()]:
                        self._queue.remove(it)          # cancelled while queued
                    if self.inflight < self.max_inflight:
                        room = self.budget - self.used
                        now = time.perf_counter()
                        for i, it in enumerate(list(self._queue)):
                            if self.inflight + len(picked) >= self.max_inflight:
                                break
                            if it.need <= room:
                                picked.append(it)
                                room -= it.need
                            elif i == 0 and now - it.t_submit > self.max_wait_s:
                                break       # the starving head keeps the room it waits for
                    if picked:
                        break
                    # wake up again when the head of the queue reaches its age limit
                    timeout = None
                    if self._queue:
                        timeout = max(0.001, self._queue[0].t_submit + self.max_wait_s - time.perf_counter()
                                      + 0.001)
                    self._cv.wait(timeout)
                for it in picked:
                    self._queue.remove(it)
                    self.used += it.need
                    self.inflight += 1
                self.peak_used = max(self.peak_used, self.used)
                self.peak_inflight = max(self.peak_inflight, self.inflight)
            for it in picked:
                threading.Thread(target=self._run, args=(it,), daemon=True).start()

    def _execute(self, it):
        if self._run_fn is not None:
            return self._run_fn(it.req)
        import torch
        req = it.req
        torch.cuda.set_device(self._device)
        stream = torch.cuda.Stream(device=self._device)
        M = mps_create(req.n_qubits, req.chi, req.precision, n_slots=req.n_slots, cuda_stream=stream.cuda_stream)
        try:
            if req.kind == "energy":
                return float(vqe_energy(M, it.circ, it.ham, req.theta))
            sel = req.sel if req.sel is not None else np.arange(req.theta.size, dtype=np.int32)
            return vqe_gradient(M, it.circ, it.ham, req.theta, sel)
        finally:
            M.close()

    def _run(self, it):
        it.t_start = time.perf_counter()
        if not it.future.set_running_or_notify_cancel():   # cancelled after admission
            with self._cv:
                self.used -= it.need
                self.inflight -= 1
                self._cv.notify_all()
            return
        try:
            value = self._execute(it)
            err = None
        except Exception as e:  # noqa: BLE001 - delivered through the future
            value, err = None, e
        it.t_done = time.perf_counter()
        with self._cv:
            self.used -= it.need
            self.inflight -= 1
            self._records.append((it.t_submit, it.t_start, it.t_done, it.req.kind))
            self._cv.notify_all()
        if err is None:
            it.future.set_result(value)
        else:
            it.future.set_exception(err)

    # ------------------------------------------------------------------ reporting
    def records(self):
        """(t_submit, t_start, t_done, kind) of every completed request."""
        with self._cv:
            return list(self._records)

    def stats(self):
        with self._cv:
            rec = list(self._records)
        if not rec:
            return {"completed": 0}
        lat = np.array([d - s for s, _, d, _ in rec])
        wait = np.array([b - s for s, b, _, _ in rec])
        span = max(d for _, _, d, _ in rec) - min(s for s, _, _, _ in rec)
        return {"completed": len(rec), "throughput_per_s": len(rec) / span if span > 0 else float("inf"),
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "queue_wait_p50_s": float(np.percentile(wait, 50)), "peak_inflight": self.peak_inflight,
                "peak_used_bytes": self.peak_used, "budget_bytes": self.budget}

    def close(self, wait=True):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        if wait:
            self._admitter.join()
            while True:
                with self._cv:
                    if self.inflight == 0:
                        break
                    self._cv.wait(0.05)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
