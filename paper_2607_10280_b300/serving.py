"""Continuous-batching server for single-image feature-extraction requests.

Requests of mixed size p, depth L and bond cap chi arrive at any time.  The
server keeps `slots` execution slots, each with its own CUDA stream, a reusable
MPS batch (``Batch.reshape`` reuses its device memory; ``Batch.reserve`` sizes
every lazily allocated buffer up front, so no wave allocates) and pinned staging
buffers.  Whenever a slot is free and requests are waiting, it forms a wave from
the waiting requests in arrival order, admitting each while the wave's device
footprint (site tensors, environments and, for a truncating circuit under the
mixed precision, its complex128 chain) fits the slot's share of the memory
budget, and launches the wave: pixels host->device, circuit, Pauli cache, ANO
features and linear layer for images that have an epilogue registered for their
size, results device->host.  Waves on different slots overlap on the GPU; a
request that arrives while others run is admitted as soon as a slot frees,
without waiting for the rest.

A request whose circuit truncates lossily runs a long sequential chain on a
complex128 state (its latency grows with p^2 L); `long_slots` of the slots serve
only such requests, the others only the rest, so a short request never waits
behind a truncating chain.

Each image's arithmetic is independent of the other images in its wave, so a
request's result does not depend on the mix it was served in.

The scheduler is a Python thread, and Python's cyclic garbage collector stops every
thread while it walks the heap: a full collection over a process that holds torch,
the server and a few thousand requests took about 100 ms, during which no wave was
launched or retired.  With ``freeze_gc`` (the default) ``start()`` moves every object
that exists at that moment into the collector's permanent generation
(``gc.freeze``), and the scheduler does the same again every ``freeze_every`` retired
waves, so the collections that run while serving walk only the objects created since
the last freeze; ``stop()`` hands them back (``gc.unfreeze``).  Frozen objects are
not searched for reference cycles until then; a request and its results form none.

Two settings belong to the process, before CUDA starts: ``CUDA_DEVICE_MAX_CONNECTIONS=32``
gives every slot's stream a hardware queue of its own (with the default 8, streams share
queues, and work on a short-lane slot's idle stream waited behind a long-lane chain on
the same queue: up to 75 ms of host time per launch with six slots), and
``CUDA_MODULE_LOADING=EAGER`` loads every kernel at start-up instead of at its first
launch.
"""
from __future__ import annotations

import collections
import gc
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .api import Batch, ano_features, pair_count
from .flops import lossy, operator_product_path, padding


def image_footprint(p: int, chi: int, precision: str = "mixed", L: int = None) -> int:
    """Device bytes one image holds in a batch: site tensors (2 ld^2 complex values per
    qubit) and right environments (ld^2).  With its depth L known, also the left
    environments of an image built as an operator product (ld^2 per qubit) and, under
    the mixed precisions, the complex128 sites of a truncating chain (2 ld^2 at 16 B)."""
    n = p * p
    ld = padding(p, chi)
    elem = 16 if precision == "fp64" else 8
    b = n * 3 * ld * ld * elem
    if L is not None:
        if operator_product_path(p, L, chi):
            b += n * ld * ld * elem
        if precision in ("mixed", "mixed_orth64") and lossy(p, L, chi):
            b += n * 2 * ld * ld * 16
    return b


def request_class(r) -> str:
    """Latency class of a request: its (p, L, chi)."""
    return f"p{r.p}_L{r.L}_chi{r.chi}"


def form_wave(pending, max_images: int, room: int, footprint) -> tuple:
    """Admission policy: take requests from the front of `pending` (arrival order)
    while the wave has fewer than max_images images and its summed footprint stays
    within `room` bytes.  Returns (wave, bytes); pending keeps the rest."""
    wave, foot = [], 0
    while pending and len(wave) < max_images:
        f = footprint(pending[0])
        if foot + f > room:
            break
        wave.append(pending.popleft())
        foot += f
    return wave, foot


@dataclass
class Request:
    p: int
    L: int
    chi: int
    pixels: np.ndarray
    id: int = 0
    t_submit: float = 0.0
    t_launch: float = 0.0   # when its wave was handed to the GPU (queueing = t_launch - t_submit)
    t_done: float = 0.0
    pauli: np.ndarray = None
    features: np.ndarray = None
    output: np.ndarray = None
    lane: str = ""          # "long" (truncating chain) or "short": the slots that served it
    event: threading.Event = field(default_factory=threading.Event)

    @property
    def latency_s(self) -> float:
        return self.t_done - self.t_submit


class _Slot:
    def __init__(self, idx, precision, max_images, max_p, max_chi, max_pairs, epi_m, epi_out, launch_shape,
                 max_L, long_lane=False):
        self.idx = idx
        self.long_lane = long_lane          # serves only requests that run a truncating chain
        self.stream = torch.cuda.Stream()
        self.precision = precision
        # sized once for the largest wave, every lazily allocated buffer included, then
        # re-laid-out per wave without allocation
        self.batch = Batch(np.full(max_images, max_p, np.int32), max_chi, precision, self.stream)
        self.batch.reserve(max_L)
        if launch_shape:
            self.batch.set_launch_shape(*launch_shape)
        max_pixels = max_images * max_p * max_p
        max_epi_images = max_images
        dt = torch.float64 if precision == "fp64" else torch.float32
        self.px_host = torch.empty(max_pixels, dtype=torch.float64).pin_memory()
        self.px_dev = torch.empty(max_pixels, dtype=torch.float64, device="cuda")
        self.pauli_dev = torch.empty((max_pairs, 16), dtype=dt, device="cuda")
        self.pauli_host = torch.empty((max_pairs, 16), dtype=dt).pin_memory()
        self.epi_m = max(1, epi_m)
        self.feat_host = torch.empty(max_epi_images * self.epi_m, dtype=torch.float32).pin_memory()
        self.out_host = torch.empty(max_epi_images * max(1, epi_out), dtype=torch.float32).pin_memory()
        self.started = torch.cuda.Event(enable_timing=True)
        self.done = torch.cuda.Event(enable_timing=True)
        self.wave = None
        self.host_ms = 0.0
        self.phase_ms = ()
        self.footprint = 0


class Server:
    """Continuous-batching server (see module docstring).

    params:    float64 device tensor [L_max][n_max][2] of rotation angles (ladder ansatz)
    epilogue:  {p: (abd [m][16] f32, W [out][m] f32, bias [out] f32)} device tensors for
               the sizes that get ANO features and a linear layer
    """

    def __init__(self, params: torch.Tensor, epilogue: dict = None, slots: int = 4,
                 max_images_per_wave: int = 64, budget_bytes: int = 2 << 30, precision: str = "mixed",
                 launch_shape=None, max_p: int = 16, max_chi: int = 32, long_slots: int = None,
                 long_launch_shape=(0, 128, 0), freeze_gc: bool = True, freeze_every: int = 256):
        self.params = params
        self.freeze_gc = freeze_gc
        self.freeze_every = max(1, freeze_every)
        self._retired_since_freeze = 0
        self._frozen = False
        self.epilogue = epilogue or {}
        self.precision = precision
        self.max_images = max_images_per_wave
        self.budget = budget_bytes
        self.slot_budget = budget_bytes // slots
        self.launch_shape = launch_shape
        self.max_p, self.max_chi = max_p, max_chi
        epi_out = max((W.shape[0] for (_, W, _) in self.epilogue.values()), default=1)
        epi_m = max((pair_count(p) for p in self.epilogue), default=1)
        # slots reserved for truncating chains (only the mixed precisions route them
        # differently; one slot serves everything)
        if long_slots is None:
            long_slots = 1 if slots >= 2 else 0
        self.long_slots = max(0, min(long_slots, slots - 1))
        # the long lane's truncation chains run on 128-thread teams (shorter chains when
        # a wave holds few images)
        self.slots = [_Slot(i, precision, max_images_per_wave, max_p, max_chi,
                            max_images_per_wave * pair_count(max_p), epi_m, epi_out,
                            long_launch_shape if i >= slots - self.long_slots else launch_shape,
                            params.shape[0], long_lane=i >= slots - self.long_slots)
                      for i in range(slots)]
        self.pending = collections.deque()        # requests for the short lane
        self.pending_long = collections.deque()   # requests that run a truncating chain
        # (slot, images, long lane, device ms, host ms spent launching, host ms per launch
        # phase: reshape, pixel staging, circuit, Pauli cache, epilogue) per wave
        self.wave_log = []
        self.lock = threading.Lock()
        self.inflight_bytes = 0
        self.completed = []
        self._next_id = 0
        self._stop = False
        self._thread = None
        self.waves = 0
        self.max_wave = 0
        self.max_inflight_bytes = 0

    # -------------------------------------------------------------- client side
    def submit(self, req: Request) -> Request:
        if req.p * req.p > self.params.shape[1] or req.L > self.params.shape[0]:
            raise ValueError("request exceeds the server's parameter table")
        if req.p > self.max_p or req.chi > self.max_chi:
            raise ValueError("request exceeds the server's largest image size or bond cap")
        if image_footprint(req.p, req.chi, self.precision, req.L) > self.slot_budget:
            raise ValueError("request does not fit a slot's memory budget")
        with self.lock:
            req.id = self._next_id
            self._next_id += 1
            req.t_submit = time.perf_counter()
            self._queue_of(req).append(req)
        return req

    def _is_long(self, req) -> bool:
        return self.long_slots > 0 and self.precision in ("mixed", "mixed_orth64") and lossy(req.p, req.L, req.chi)

    def _queue_of(self, req):
        return self.pending_long if self._is_long(req) else self.pending

    def start(self):
        if self.freeze_gc and not self._frozen:
            gc.collect()
            gc.freeze()
            self._frozen = True
        self._stop = False
        self._thread = threading.Thread(target=self._loop, daemon=True)
        self._thread.start()

    def stop(self, drain: bool = True):
        if drain:
            while True:
                with self.lock:
                    busy = self.pending or self.pending_long or any(s.wave for s in self.slots)
                if not busy:
                    break
                time.sleep(0.0005)
        self._stop = True
        if self._thread:
            self._thread.join()
        if self._frozen:
            gc.unfreeze()
            self._frozen = False

    # -------------------------------------------------------------- server loop
    def _loop(self):
        torch.cuda.set_device(self.params.device)
        while not self._stop:
            progressed = self.poll()
            if not progressed:
                time.sleep(0.0002)

    def poll(self) -> bool:
        """One scheduling round: retire finished waves, then admit and launch new ones."""
        progressed = False
        for s in self.slots:
            if s.wave is not None and s.done.query():
                self._retire(s)
                progressed = True
        for s in self.slots:
            if s.wave is None:
                wave = self._admit(self.pending_long if s.long_lane else self.pending)
                if not wave:
                    continue
                self._launch(s, wave)
                progressed = True
        return progressed

    def _admit(self, queue):
        with self.lock:
            room = min(self.slot_budget, self.budget - self.inflight_bytes)
            wave, foot = form_wave(queue, self.max_images, room,
                                   lambda r: image_footprint(r.p, r.chi, self.precision, r.L))
            if wave:
                self.inflight_bytes += foot
                self.max_inflight_bytes = max(self.max_inflight_bytes, self.inflight_bytes)
            return (wave, foot) if wave else None

    def _launch(self, s: _Slot, admitted):
        wave, foot = admitted
        t_launch = time.perf_counter()
        # images with an epilogue first, grouped by size, so that each group's Pauli
        # blocks are contiguous
        wave.sort(key=lambda r: (0 if r.p in self.epilogue else 1, r.p))
        for r in wave:
            r.lane = "long" if s.long_lane else "short"
            r.t_launch = t_launch
        ps = np.array([r.p for r in wave], np.int32)
        chis = np.array([r.chi for r in wave], np.int32)
        Ls = np.array([r.L for r in wave], np.int32)
        with torch.cuda.stream(s.stream):
            s.started.record(s.stream)
            s.batch.reshape(ps, chis)
            t_reshape = time.perf_counter()
            offs = s.batch.pixel_offsets
            for i, r in enumerate(wave):
                s.px_host[offs[i]:offs[i + 1]] = torch.from_numpy(r.pixels)
            n_px = int(offs[-1])
            s.px_dev[:n_px].copy_(s.px_host[:n_px], non_blocking=True)
            t_pixels = time.perf_counter()
            s.batch.apply_circuit(s.px_dev[:n_px], Ls, "ladder", self.params)
            t_circuit = time.perf_counter()
            n_pairs = int(s.batch.pair_offsets[-1])
            s.batch.pauli_cache(s.pauli_dev[:n_pairs])
            t_pauli = time.perf_counter()
            s.pauli_host[:n_pairs].copy_(s.pauli_dev[:n_pairs], non_blocking=True)
            epi = []
            i = 0
            while i < len(wave) and wave[i].p in self.epilogue:
                j = i
                while j < len(wave) and wave[j].p == wave[i].p:
                    j += 1
                abd, W, bias = self.epilogue[wave[i].p]
                m = pair_count(wave[i].p)
                a0, a1 = int(s.batch.pair_offsets[i]), int(s.batch.pair_offsets[j])
                feats, out = ano_features(s.pauli_dev[a0:a1], m, abd, W, bias, s.stream)
                f0 = i * s.epi_m
                s.feat_host[f0:f0 + feats.numel()].copy_(feats.reshape(-1), non_blocking=True)
                o0 = i * W.shape[0]
                s.out_host[o0:o0 + out.numel()].copy_(out.reshape(-1), non_blocking=True)
                epi.append((i, j, m, W.shape[0], feats, out))   # keep device results alive
                i = j
            s.done.record(s.stream)
        s.wave = (wave, epi)
        t_end = time.perf_counter()
        s.host_ms = (t_end - t_launch) * 1e3
        # host ms of each launch phase: reshape, pixel staging, circuit, Pauli cache, epilogue
        s.phase_ms = tuple(1e3 * (b - a) for a, b in ((t_launch, t_reshape), (t_reshape, t_pixels),
                                                       (t_pixels, t_circuit), (t_circuit, t_pauli),
                                                       (t_pauli, t_end)))
        s.footprint = foot
        self.waves += 1
        self.max_wave = max(self.max_wave, len(wave))

    def _retire(self, s: _Slot):
        wave, epi = s.wave
        offs = s.batch.pair_offsets
        now = time.perf_counter()
        for i, r in enumerate(wave):
            r.pauli = s.pauli_host[offs[i]:offs[i + 1]].numpy().copy()
        for (i, j, m, od, _, _) in epi:
            for k in range(i, j):
                wave[k].features = s.feat_host[k * s.epi_m:k * s.epi_m + m].numpy().copy()
                wave[k].output = s.out_host[k * od:(k + 1) * od].numpy().copy()
        for r in wave:
            r.t_done = now
            r.event.set()
        if self._frozen:
            self._retired_since_freeze += 1
            if self._retired_since_freeze >= self.freeze_every:
                gc.freeze()
                self._retired_since_freeze = 0
        self.wave_log.append((s.idx, len(wave), s.long_lane, s.started.elapsed_time(s.done), s.host_ms,
                              s.phase_ms))
        with self.lock:
            self.inflight_bytes -= s.footprint
            self.completed.extend(wave)
        s.wave = None
        s.footprint = 0


def latency_report(reqs) -> dict:
    lat = np.array([r.latency_s for r in reqs]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "requests": len(reqs)}


def latency_by(reqs, key) -> dict:
    """latency_report of the requests grouped by key(request)."""
    groups = collections.defaultdict(list)
    for r in reqs:
        groups[key(r)].append(r)
    return {k: latency_report(v) for k, v in sorted(groups.items())}
