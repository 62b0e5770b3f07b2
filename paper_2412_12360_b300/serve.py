"""Continuous-batching server for forward + time-reversal-gradient solves of mixed sizes.

Requests (a scene: grid, sources, detectors, design box and densities, step count) arrive at any
time. A scheduler thread admits them in arrival order whenever a slot is free and the request's
device footprint (fdtd_footprint_bytes: fields, CPML memories, adjoint state and the boundary-face
history) fits in the memory budget still free. An admitted request's handle is created and its
inputs uploaded on a private stream, then it joins the running requests, which are advanced in
chunks of steps by fdtd_group_step: it launches each kernel of a time step (the forward, or the
reverse pair) once for the blocks of every request of a group, so small requests that run at the
same time share the GPU's SMs rather than queueing behind each other's launches. The running requests
form groups whose per-step bytes fit in about half of the L2, stepped one group after another. A request moves from its forward
to its reverse sweep, and leaves the group, at the step where it finishes; finished requests return
their detector outputs and dL/deps and free their memory (stream-ordered), which admits the next
ones.

The numerical work of every request is the library's, and a request's arithmetic does not depend on
which others share its launches, so its result is bitwise the same alone and in the mix.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Deque, List, Optional

import numpy as np


def one_shot(solver):
    """Configure a handle that solves once: time loops launched directly rather than captured into
    CUDA graphs, face copies in line rather than on a second stream. Building the graphs of a single
    solve costs more host time than replaying them saves; on one B300 the sequential stream of served
    requests ran at 13.8 Gcell-steps/s with the library defaults, 14.7 with in-line face copies and
    15.9 with direct launches as well (results bitwise the same)."""
    solver.fdtd_set_graphs(False)
    solver.fdtd_set_face_overlap(False)


def admit_count(queue_footprints, inflight: int, used: int, budget: int, max_inflight: int) -> int:
    """How many requests at the head of the queue can be admitted now: first-come first-served, while a
    slot is free and the next request's footprint fits in the memory still free (the head blocks the
    ones behind it, so no request starves)."""
    n = 0
    for fp in queue_footprints:
        if inflight + n >= max_inflight or used + fp > budget:
            break
        used += fp
        n += 1
    return n


def step_bytes(scene) -> int:
    """The bytes one time step of a request reads and writes at least: its fields (or its primal and
    adjoint fields) and inverse permittivity, 52 B per cell. Requests stepped together keep the GPU's
    L2 to themselves only while these sum to less than it holds."""
    nx, ny, nz = scene.n
    return 52 * nx * ny * nz


def partition(sizes, budget: int, max_group: int):
    """Split requests (in order) into consecutive groups whose sizes sum to at most `budget` (a request
    larger than the budget forms a group of its own), each of at most max_group; budget <= 0: groups of
    max_group regardless of size. Returns lists of indices."""
    groups, cur, used = [], [], 0
    for i, b in enumerate(sizes):
        if cur and (len(cur) >= max_group or (budget > 0 and used + b > budget)):
            groups.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += b
    if cur:
        groups.append(cur)
    return groups


@dataclass
class Result:
    detectors: np.ndarray
    dL_deps: np.ndarray
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Job:
    scene: object
    dL_ddet: Optional[np.ndarray]
    future: Future
    arrival: float
    footprint: int
    admitted: float = 0.0
    solver: object = None
    done: object = None
    det: object = None
    grad: object = None
    gvec: object = None
    finishing: bool = False


class Server:
    """Continuous-batching solver service on one GPU.

    budget_bytes: device memory the server may give to requests (default: 85 % of the free memory).
    max_inflight: requests running at once (at most the library's group size, 8).
    chunk_steps: time steps per grouped call between scheduling decisions (admission, phase changes).
    ahead: grouped calls enqueued ahead of the GPU at most (enough to cover a request's set-up on the
    host, few enough that a request that arrives meanwhile joins soon).
    group_bytes: the running requests are stepped in groups whose step bytes (step_bytes) sum to at
    most this, one group after another for chunk_steps each (0: all in one group). Small requests fill
    the GPU only side by side; larger ones run fastest in few at a time, each group's state staying in
    L2 across its chunk of steps. The default, 64 MiB (about half of a B300's 126 MB L2), served a
    stream of 64^3 and 96^3 requests at 12.1 Gcell-steps/s on one B300, against 11.6 with all running
    requests in one group and 11.7 / 12.0 with 100 / 128 MiB.
    """

    def __init__(self, budget_bytes: Optional[int] = None, max_inflight: int = 4, device: int = 0,
                 footprint=None, chunk_steps: int = 32, ahead: int = 4, group_bytes: int = 64 << 20):
        import torch
        from . import fdtd

        self._torch = torch
        self._fdtd = fdtd
        self.device = torch.device("cuda", device)
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(0.85 * free)
        self.budget = int(budget_bytes)
        self.max_inflight = max(1, min(int(max_inflight), fdtd.MAX_GROUP))
        self.chunk_steps = int(chunk_steps)
        self.ahead = max(1, int(ahead))
        self.group_bytes = int(group_bytes)
        self._footprint = footprint or (lambda sc: fdtd.footprint_bytes(sc, sc.nsteps, record_faces=True))
        self._queue: Deque[_Job] = collections.deque()
        self._inflight: List[_Job] = []
        self._used = 0
        self._lock = threading.Condition()
        self._stop = False
        self.stream = torch.cuda.Stream(device=self.device)   # the group's stream
        self._setup = torch.cuda.Stream(device=self.device)   # where admitted handles are prepared
        self._ticks: Deque[object] = collections.deque()
        self.peak_inflight = 0
        self.cancelled = 0  # requests cancelled by their client before admission
        self.group_calls = 0
        self._thread = threading.Thread(target=self._loop, name="fdtd-server", daemon=True)
        self._thread.start()

    # ---- client side ---------------------------------------------------------------------------
    def submit(self, scene, dL_ddet: Optional[np.ndarray] = None) -> Future:
        fp = int(self._footprint(scene))
        if fp > self.budget:
            raise ValueError("request needs %d bytes, more than the server's budget of %d" % (fp, self.budget))
        fut: Future = Future()
        with self._lock:
            self._queue.append(_Job(scene, dL_ddet, fut, time.perf_counter(), fp))
            self._lock.notify()
        return fut

    def close(self):
        with self._lock:
            self._stop = True
            self._lock.notify()
        self._thread.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- scheduler ----------------------------------------------------------------------------
    def _admit(self, job: _Job):
        torch, fdtd = self._torch, self._fdtd
        sc = job.scene
        job.admitted = time.perf_counter()
        with torch.cuda.stream(self.stream):
            ndet_total = None
            job.solver = fdtd.Solver(sc, stream=self._setup)
            one_shot(job.solver)
            job.solver.fdtd_begin(sc.nsteps, record_faces=True)
            ndet_total = job.solver.fdtd_detector_total()
            g = job.dL_ddet if job.dL_ddet is not None else np.ones(ndet_total)
            job.gvec = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float64)).pin_memory().to(
                self.device, non_blocking=True)
            job.det = torch.empty(ndet_total, dtype=torch.float64, device=self.device)
            job.grad = torch.empty(sc.design_shape(), dtype=torch.float32, device=self.device)
        job.solver.fdtd_set_stream(self.stream)  # waits for the set-up; the request joins the group

    def _retire(self, job: _Job):
        """A finished request (its event has fired): report, copy its results out and free it, without
        waiting for the group's stream (the other requests keep running)."""
        try:
            job.solver.fdtd_poll_status()  # raises on a timeout or non-finite fields (the client gets it)
            det = job.det.cpu().numpy()
            grad = job.grad.cpu().numpy()
        finally:  # the request's memory goes back whatever happened (freed in stream order)
            job.solver.close()
        job.future.set_result(Result(det, grad, job.arrival, job.admitted, time.perf_counter()))

    def _advance(self):
        """Phase changes of the running requests, then one grouped chunk of steps for those still
        stepping (enqueued only; no synchronisation)."""
        fdtd = self._fdtd
        stepping = []
        for job in self._inflight:
            if job.finishing:
                continue
            try:
                ph, _ = job.solver.fdtd_phase()
                if ph == fdtd.PHASE_FORWARD_DONE:
                    job.solver.fdtd_read_detectors(job.det)
                    job.solver.fdtd_begin_backward(job.gvec)
                    ph = fdtd.PHASE_BACKWARD
                if ph == fdtd.PHASE_DONE:
                    job.solver.fdtd_finish_backward(job.grad)
                    job.done = self._torch.cuda.Event()
                    job.done.record(self.stream)
                    job.finishing = True
                    continue
            except Exception as e:  # noqa: BLE001 - report to the client
                job.done = self._torch.cuda.Event()
                job.done.record(self.stream)
                job.finishing = True
                job.error = e
                continue
            stepping.append(job)
        for grp in partition([step_bytes(j.scene) for j in stepping], self.group_bytes, fdtd.MAX_GROUP):
            fdtd.group_step([stepping[i].solver for i in grp], self.chunk_steps)
            self.group_calls += 1
            ev = self._torch.cuda.Event()
            ev.record(self.stream)
            self._ticks.append(ev)
        while len(self._ticks) > self.ahead:  # at most `ahead` chunks enqueued ahead of the GPU
            self._ticks.popleft().synchronize()
        return bool(stepping)

    def _loop(self):
        torch = self._torch
        torch.cuda.set_device(self.device)
        while True:
            with self._lock:
                if self._stop and not self._queue and not self._inflight:
                    return
                if not self._queue and not self._inflight:
                    self._lock.wait(timeout=0.05)
                    continue
            progressed = False
            for job in list(self._inflight):
                if job.finishing and job.done.query():
                    self._inflight.remove(job)
                    self._used -= job.footprint
                    try:
                        if getattr(job, "error", None) is not None:
                            job.solver.close()
                            raise job.error
                        self._retire(job)
                    except Exception as e:  # noqa: BLE001 - report to the client
                        job.future.set_exception(e)
                    progressed = True
            while True:
                with self._lock:
                    while self._queue and self._queue[0].future.cancelled():  # Future.cancel() by the client
                        self._queue.popleft()
                        self.cancelled += 1
                    if not self._queue or admit_count([self._queue[0].footprint], len(self._inflight), self._used,
                                                      self.budget, self.max_inflight) == 0:
                        break
                    job = self._queue.popleft()
                    if not job.future.set_running_or_notify_cancel():  # cancelled in between
                        self.cancelled += 1
                        continue
                self._used += job.footprint
                try:
                    self._admit(job)
                    self._inflight.append(job)
                    self.peak_inflight = max(self.peak_inflight, len(self._inflight))
                except Exception as e:  # noqa: BLE001 - report to the client
                    self._used -= job.footprint
                    if job.solver is not None:
                        job.solver.close()
                    job.future.set_exception(e)
                progressed = True
            if self._inflight:
                progressed |= self._advance()
            if not progressed:
                time.sleep(0.0002)


def run_sequential(scenes, device: int = 0):
    """The same requests solved one after another on the default stream (the comparison baseline)."""
    import torch
    from . import fdtd

    out = []
    for sc in scenes:
        with fdtd.Solver(sc) as s:
            one_shot(s)  # one solve per handle, as in the server
            s.fdtd_forward(sc.nsteps, record_faces=True)
            det = s.detectors()
            grad = s.gradient(np.ones(s.fdtd_detector_total()))
        out.append((det, grad))
    torch.cuda.synchronize()
    return out


def latency_stats(results) -> dict:
    lat = np.array([r.latency for r in results])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "n": int(lat.size)}
