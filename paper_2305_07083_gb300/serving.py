"""Continuous-batching compositing server on one GPU.

In-situ clients submit compositing jobs: a data-parallel *blend* job
composites one frame of brick fragment tiles (Sec. 4.2), an image-parallel
*accumulate* job refines one frame progressively from one fragment tile per
image tile over many passes (Sec. 4.1, progressive refinement).  The server

* admits queued jobs in arrival order while their HBM footprint fits the
  budget and a slot is free, giving each job its own resident framebuffer
  (a handle of libdfb.so);
* on every step composites the next frame of *every* active job in one
  batched launch (dfb_run_frames: each job's frame is a prepared tile set,
  validated once; one bucketing pass and one persistent composite launch
  over all their work items), so jobs that arrive while others are on the
  GPU join the next launch;
* retires jobs whose last frame has been composited: their RGBA8 frame is
  read back, the latency (arrival to result on the host) is recorded and
  the footprint is released for the next queued job.

Work items of different jobs never interact, so a job's result is the same
alone and in any mix.  This module only schedules: every step of the
compositing runs in the library's kernels.
"""

from __future__ import annotations

import time
import weakref
from dataclasses import dataclass, field

import numpy as np

from . import dfb as D


@dataclass
class FrameData:
    """One frame's fragment tiles, resident in device memory (16-byte
    aligned pools of T*T-pixel tiles)."""
    tile_ids: np.ndarray
    keys: np.ndarray
    rgba: object          # device tensor, tiles back to back, storage dtype
    depth: object         # device tensor, tiles back to back, FP32
    fragment_pixels: int
    rgba_ptrs: np.ndarray = None
    depth_ptrs: np.ndarray = None
    tileset: object = None

    def pointers(self, T, dtype):
        if self.rgba_ptrs is None:
            n, P = len(self.tile_ids), T * T
            self.rgba_ptrs = D.pool_pointers(self.rgba, n, P * 4 * D.ELEMENT_BYTES[dtype])
            self.depth_ptrs = D.pool_pointers(self.depth, n, P * 4)
        return self.rgba_ptrs, self.depth_ptrs

    def prepared(self, handle, T, dtype):
        """The frame as a prepared tile set for handles shaped like
        `handle` (made once; every job on this frame shares it)."""
        if self.tileset is None:
            rp, dp = self.pointers(T, dtype)
            self.tileset = D.dfb_tileset_create(handle, self.tile_ids, self.keys, rp, dp)
            weakref.finalize(self, D.dfb_tileset_destroy, self.tileset)
        return self.tileset


@dataclass
class Job:
    job_id: int
    client: int
    arrival: float        # seconds after the server's start
    kind: str             # "blend" or "accumulate"
    W: int
    H: int
    T: int
    frames: list          # FrameData per pass (cycled if shorter than n_frames)
    n_frames: int
    mode: int = D.DFB_BLEND_DEPTH
    # filled in by the server
    handle: object = None
    done_frames: int = 0
    admitted: float = -1.0
    finished: float = -1.0
    result: np.ndarray = None
    fragment_pixels: int = 0

    def footprint(self, dtype) -> int:
        """Bytes this job holds in HBM while active: its framebuffers
        (colour 16 B, sum/M2/compensation 48 B, RGBA8 4 B per pixel) and the
        fragment tiles of the frames it references."""
        px = self.W * self.H
        fb = px * (16 + 48 + 4)
        eb = D.ELEMENT_BYTES[dtype]
        frag = sum(len(f.tile_ids) * self.T * self.T * (4 * eb + 4) for f in self.frames)
        return fb + frag


@dataclass
class ServerStats:
    jobs: int = 0
    steps: int = 0
    launches_frames: int = 0
    fragment_pixels: int = 0
    wall_s: float = 0.0
    latencies_ms: list = field(default_factory=list)
    latencies_by_kind: dict = field(default_factory=dict)  # kind -> latencies (ms)
    batch_sizes: list = field(default_factory=list)
    peak_active: int = 0
    peak_footprint: int = 0
    host_ms: dict = field(default_factory=dict)   # host time per phase of the loop
    gpu_ms: float = 0.0                          # device time of the batched launches

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"jobs": self.jobs, "steps": self.steps,
                "frames_composited": self.launches_frames,
                "fragment_pixels": self.fragment_pixels, "wall_s": self.wall_s,
                "fragment_pixels_per_s": self.fragment_pixels / max(self.wall_s, 1e-9),
                "latency_ms_p50": float(np.percentile(lat, 50)),
                "latency_ms_p99": float(np.percentile(lat, 99)),
                "latency_ms_max": float(lat.max()),
                "latency_ms_by_kind": {
                    k: {"jobs": len(v), "p50": float(np.percentile(v, 50)),
                        "p99": float(np.percentile(v, 99))}
                    for k, v in sorted(self.latencies_by_kind.items()) if v},
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "max_batch": int(max(self.batch_sizes)) if self.batch_sizes else 0,
                "peak_active_jobs": self.peak_active,
                "peak_footprint_bytes": self.peak_footprint,
                "host_ms": {k: round(v, 3) for k, v in self.host_ms.items()},
                "gpu_busy_ms": round(self.gpu_ms, 3)}


def admit(queue, n_active: int, used: int, budget: int, max_slots: int, footprint) -> list:
    """Jobs to admit now, taken from the front of `queue` (arrival order,
    removed from it): while a slot is free and the job's footprint fits the
    budget.  A job that does not fit stops the admission (no overtaking);
    when nothing is active the head job is admitted whatever its size, so a
    job larger than the budget cannot block the server."""
    out = []
    while queue and n_active + len(out) < max_slots:
        fp = footprint(queue[0])
        if (n_active or out) and used + fp > budget:
            break
        out.append(queue.pop(0))
        used += fp
    return out


class Server:
    def __init__(self, budget_bytes: int, max_slots: int = 64, dtype: int = D.DFB_F16,
                 stream=None, keep_results: bool = True):
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.dtype = dtype
        self.stream = stream
        self.keep_results = keep_results
        self.pool = {}  # resident framebuffers by shape, reused across jobs
        self.out_pool = {}

    # -- one job's frame ---------------------------------------------------
    def _submit(self, job: Job):
        fr = job.frames[job.done_frames % len(job.frames)]
        rp, dp = fr.pointers(job.T, self.dtype)
        D.dfb_begin_frame(job.handle, job.done_frames > 0)
        D.dfb_submit_tiles(job.handle, fr.tile_ids, fr.keys, rp, dp, None, D.DFB_PTR_DEVICE)
        return fr.fragment_pixels

    def _open(self, job: Job):
        key = (job.W, job.H, job.T, job.mode)
        free = self.pool.get(key)
        if free:
            job.handle = free.pop()   # a resident framebuffer; its first frame resets it
            return
        flags = D.DFB_FLAG_ACCUMULATE | D.DFB_FLAG_PACK_RGBA8
        job.handle = D.dfb_create_ex(job.W, job.H, job.T, job.mode, self.dtype, flags, 0,
                                     max(4096, max(len(f.tile_ids) for f in job.frames)))

    def close(self):
        """Free the pooled framebuffers."""
        for hs in self.pool.values():
            for h in hs:
                D.dfb_destroy(h)
        self.pool = {}
        self.out_pool = {}

    # -- the loop -------------------------------------------------------------
    def run(self, jobs, time_limit_s: float = 1e9, trace: bool = False) -> ServerStats:
        """Serve `jobs` (any order; admitted by arrival time) until all have
        finished or the time limit has passed.

        The host never waits for a step: a finished job's RGBA8 frame is
        copied out on the stream (device copy, then into pinned host memory)
        behind its last frame, its framebuffer goes back to the pool at once
        (later work on the stream is ordered after the copy), and its
        completion is observed by polling an event.  The library bounds how
        far the host runs ahead (a batch waits for the previous batch before
        reusing its staging buffers).

        With `keep_results`, a finished job's frame is copied out of the
        pooled pinned buffer into its own array (`job.result`); otherwise the
        client takes it in place and the buffer goes back to the pool.

        With `trace`, the stats also split the host time by phase (admit,
        deliver, prepare, launch, retire) and sum the device time of every
        batched launch (CUDA events around each step on the stream).
        """
        import torch
        stream = self.stream if self.stream is not None else torch.cuda.current_stream()
        pending = sorted(jobs, key=lambda j: (j.arrival, j.job_id))
        queue, active, inflight = [], [], []
        used = 0
        st = ServerStats()
        phase = {"admit": 0.0, "deliver": 0.0, "prepare": 0.0, "launch": 0.0, "retire": 0.0}
        step_events = []
        t0 = time.perf_counter()

        def observe(block):
            nonlocal inflight
            keep = []
            for i, (job, ev, dev, host) in enumerate(inflight):
                if (block and i == 0) or ev.query():
                    if block and i == 0:
                        ev.synchronize()
                    job.finished = time.perf_counter() - t0
                    st.latencies_ms.append(1e3 * (job.finished - job.arrival))
                    st.latencies_by_kind.setdefault(job.kind, []).append(st.latencies_ms[-1])
                    st.jobs += 1
                    if self.keep_results:
                        job.result = host.numpy().view(np.uint32).copy()
                    self._release_out(job, dev, host)
                else:
                    keep.append((job, ev, dev, host))
            inflight = keep

        while pending or queue or active or inflight:
            ta = time.perf_counter()
            now = ta - t0
            if now > time_limit_s:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            for job in admit(queue, len(active), used, self.budget, self.max_slots,
                             lambda j: j.footprint(self.dtype)):
                self._open(job)
                job.admitted = time.perf_counter() - t0
                used += job.footprint(self.dtype)
                active.append(job)
            st.peak_active = max(st.peak_active, len(active))
            st.peak_footprint = max(st.peak_footprint, used)
            tm = time.perf_counter()
            observe(False)
            tb = time.perf_counter()
            phase["admit"] += tm - ta
            phase["deliver"] += tb - tm
            if not active:
                if inflight:
                    observe(True)
                elif pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.001)))
                continue
            # one step: the next frame of every active job in one launch
            fpx = 0
            sets, acc = [], []
            for job in active:
                fr = job.frames[job.done_frames % len(job.frames)]
                sets.append(fr.prepared(job.handle, job.T, self.dtype))
                acc.append(1 if job.done_frames > 0 else 0)
                fpx += fr.fragment_pixels
            tc = time.perf_counter()
            if trace:
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            D.dfb_run_frames([j.handle for j in active], sets, acc, stream)
            if trace:
                e1 = torch.cuda.Event(enable_timing=True)
                e1.record(stream)
                step_events.append((e0, e1))
            td = time.perf_counter()
            phase["prepare"] += tc - tb
            phase["launch"] += td - tc
            st.steps += 1
            st.batch_sizes.append(len(active))
            st.launches_frames += len(active)
            st.fragment_pixels += fpx
            still = []
            for job in active:
                job.fragment_pixels += job.frames[job.done_frames % len(job.frames)].fragment_pixels
                job.done_frames += 1
                if job.done_frames >= job.n_frames:
                    dev, host = self._take_out(job)
                    D.dfb_read_rgba8(job.handle, dev)          # ordered after its frame
                    host.copy_(dev, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                    inflight.append((job, ev, dev, host))
                    self.pool.setdefault((job.W, job.H, job.T, job.mode), []).append(job.handle)
                    job.handle = None
                    used -= job.footprint(self.dtype)
                else:
                    still.append(job)
            active = still
            phase["retire"] += time.perf_counter() - td
        while inflight and time.perf_counter() - t0 <= time_limit_s:
            observe(True)
        st.wall_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        st.host_ms = {k: 1e3 * v for k, v in phase.items()}
        st.gpu_ms = sum(a.elapsed_time(b) for a, b in step_events)
        for job in active:       # time limit: release what is still open
            self.pool.setdefault((job.W, job.H, job.T, job.mode), []).append(job.handle)
            job.handle = None
        return st

    # output buffers for finished frames, pooled by shape
    def _take_out(self, job):
        import torch
        free = self.out_pool.setdefault((job.W, job.H), [])
        if free:
            return free.pop()
        dev = torch.empty((job.H, job.W), dtype=torch.int32, device="cuda")
        host = torch.empty((job.H, job.W), dtype=torch.int32).pin_memory()
        return dev, host

    def _release_out(self, job, dev, host):
        self.out_pool.setdefault((job.W, job.H), []).append((dev, host))


def make_jobs(templates, arrivals, seed=0, accumulate_frames=64, T=64):
    """Jobs for (time, client) arrivals: half blend jobs on a random blend
    template, half accumulate jobs of `accumulate_frames` passes.  Jobs on
    the same template share its FrameData (and so its prepared tile sets)."""
    rng = np.random.default_rng([seed, 6])
    shared = {}

    def frame(kind, i, j, d):
        key = (kind, i, j)
        if key not in shared:
            shared[key] = FrameData(d["tile_ids"], d["keys"], d["rgba"], d["depth"],
                                    d["fragment_pixels"])
        return shared[key]

    jobs = []
    for i, (t, c) in enumerate(arrivals):
        if rng.random() < 0.5:
            k = int(rng.integers(len(templates["blend"])))
            W, H, _, fd = templates["blend"][k]
            jobs.append(Job(i, c, t, "blend", W, H, T, [frame("blend", k, 0, fd)], 1))
        else:
            k = int(rng.integers(len(templates["accumulate"])))
            W, H, passes = templates["accumulate"][k]
            frames = [frame("accumulate", k, j, p) for j, p in enumerate(passes)]
            jobs.append(Job(i, c, t, "accumulate", W, H, T, frames, accumulate_frames))
    return jobs


def run_alone(job: Job, dtype: int = D.DFB_F16, stream=None) -> np.ndarray:
    """The job on its own: each frame through dfb_end_frame; returns RGBA8."""
    srv = Server(budget_bytes=1 << 62, max_slots=1, dtype=dtype, stream=stream)
    srv._open(job)
    for f in range(job.n_frames):
        job.done_frames = f
        srv._submit(job)
        D.dfb_end_frame(job.handle, stream)
    job.done_frames = job.n_frames
    out = np.empty((job.H, job.W), np.uint32)
    D.dfb_read_rgba8(job.handle, out)
    D.dfb_destroy(job.handle)
    job.handle = None
    return out


def poisson_arrivals(n_clients: int, mean_gap_s: float, duration_s: float, seed: int):
    """Per client, exponential gaps of mean `mean_gap_s` up to `duration_s`:
    returns sorted (time, client) pairs."""
    rng = np.random.default_rng([seed, 5])
    out = []
    for c in range(n_clients):
        t = rng.exponential(mean_gap_s)
        while t < duration_s:
            out.append((t, c))
            t += rng.exponential(mean_gap_s)
    out.sort()
    return out
