"""Python API over the C ABI.  PyTorch provides device memory and streams; every
step of the path runs in the CUDA library (``_lib``).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import ANSATZ, PAIR_SET, PAULI_KERNEL, PRECISION, check, lib, mps_circuit


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def pair_count(p: int, pair_set: str = "hv") -> int:
    return int(lib().mps_pair_count(int(p), PAIR_SET[pair_set]))


def _pair_offsets(p: np.ndarray, pair_set: str = "hv") -> np.ndarray:
    """Prefix sums of the images' pair counts (the library's count, once per distinct side)."""
    sides, inv = np.unique(p, return_inverse=True)
    counts = np.array([pair_count(int(q), pair_set) for q in sides], dtype=np.int64)
    return np.concatenate([[0], np.cumsum(counts[inv.reshape(-1)])])


ROUTES = ("operator_product", "layer_pipelined", "sequential", "sequential_complex128")


def plan_image(p: int, L: int, chi: int, ansatz: str = "ladder", precision: str = "mixed",
               layer_pipeline: bool = True) -> dict:
    """How the library would run one image (host-side, no GPU needed): kernel route,
    largest bond, whether a step truncates lossily, and the site padding."""
    out = (ctypes.c_int32 * 4)()
    st = lib().mps_plan_image(int(p), int(L), int(chi), ANSATZ[ansatz], PRECISION[precision],
                              1 if layer_pipeline else 0, out)
    if st not in (0, 5):
        check(st)
    return {"route": ROUTES[out[0]], "bond": int(out[1]), "lossy": bool(out[2]), "padding": int(out[3]),
            "supported": st == 0}


def launch_count() -> int:
    return int(lib().mps_launch_count())


class Batch:
    """A batch of images, one MPS each (Sec. II.B, Eq. 3), on one CUDA stream."""

    # Pauli-cache kernel of new batches (set_pauli_sweep): None = the library default
    pauli_kernel_default = None

    def __init__(self, p, chi, precision: str = "mixed", stream=None):
        p = np.atleast_1d(np.asarray(p, dtype=np.int32))
        self.n_images = len(p)
        self.p = p
        self.n = p.astype(np.int64) ** 2
        chi_arr = np.broadcast_to(np.asarray(chi, dtype=np.int32), p.shape).copy()
        self.chi = chi_arr
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        handle = ctypes.c_void_p()
        check(lib().mps_create_batch(
            self.n_images, p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            chi_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0, PRECISION[precision],
            _stream_handle(self.stream), ctypes.byref(handle)))
        self._h = handle
        self.pixel_offsets = np.concatenate([[0], np.cumsum(self.n)])
        self._pair_offs = {"hv": _pair_offsets(p, "hv")}
        self.pair_offsets = self._pair_offs["hv"]
        if Batch.pauli_kernel_default is not None:
            self.set_pauli_sweep(Batch.pauli_kernel_default)

    def reshape(self, p, chi):
        """New image list for this batch, reusing its device memory when it fits."""
        p = np.atleast_1d(np.asarray(p, dtype=np.int32))
        chi_arr = np.broadcast_to(np.asarray(chi, dtype=np.int32), p.shape).copy()
        check(lib().mps_reshape_batch(self._h, len(p), p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      chi_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0))
        self.n_images, self.p, self.chi = len(p), p, chi_arr
        self.n = p.astype(np.int64) ** 2
        self.pixel_offsets = np.concatenate([[0], np.cumsum(self.n)])
        self._pair_offs = {"hv": _pair_offsets(p, "hv")}
        self.pair_offsets = self._pair_offs["hv"]

    def reserve(self, L_max: int):
        """Allocate every buffer a circuit of up to L_max layers may need on this layout
        (or a smaller one), so that later calls allocate nothing."""
        check(lib().mps_reserve(self._h, int(L_max)))

    # -- lifetime ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(lib().mps_destroy_batch(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the path ------------------------------------------------------------------
    def apply_circuit(self, pixels: torch.Tensor, L, ansatz: str = "ladder", params: torch.Tensor = None):
        """pixels: float64 device tensor, packed [sum n_i]; params: float64 device [L][n][2]."""
        assert pixels.is_cuda and pixels.dtype == torch.float64 and pixels.is_contiguous()
        if pixels.numel() != int(self.pixel_offsets[-1]):
            raise ValueError(f"pixels must hold {int(self.pixel_offsets[-1])} values, got {pixels.numel()}")
        c = mps_circuit()
        c.ansatz = ANSATZ[ansatz]
        L_arr = np.broadcast_to(np.asarray(L, dtype=np.int32), self.p.shape).copy()
        self._L = L_arr
        c.L = int(L_arr.max()) if len(L_arr) else 0
        c.L_per_image = L_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if params is not None:
            assert params.is_cuda and params.dtype == torch.float64 and params.is_contiguous()
            if params.dim() != 3 or params.shape[2] != 2 or params.shape[0] < c.L or params.shape[1] < int(self.n.max()):
                raise ValueError(f"params must be [>= {c.L}][>= {int(self.n.max())}][2], got {tuple(params.shape)}")
            c.params = params.data_ptr()
            c.params_n = params.shape[1]
        else:
            c.params = None
            c.params_n = 0
        self._pixels_ref, self._params_ref = pixels, params   # keep alive while queued
        check(lib().mps_apply_circuit(self._h, _ptr(pixels), ctypes.byref(c)))

    def pair_offsets_for(self, pair_set: str = "hv") -> np.ndarray:
        if pair_set not in self._pair_offs:
            self._pair_offs[pair_set] = _pair_offsets(self.p, pair_set)
        return self._pair_offs[pair_set]

    def pauli_cache(self, out: torch.Tensor = None, pair_set: str = "hv") -> torch.Tensor:
        """Pauli cache [sum m_i][16] (Sec. II.C, Eq. 5), float64 (fp64) or float32.
        pair_set "hv": horizontal + vertical neighbours; "hvd": also both diagonals."""
        dtype = torch.float64 if self.precision == "fp64" else torch.float32
        total = int(self.pair_offsets_for(pair_set)[-1])
        if out is None:
            out = torch.empty((total, 16), dtype=dtype, device="cuda")
        assert out.dtype == dtype and out.shape == (total, 16) and out.is_contiguous()
        check(lib().mps_pauli_cache(self._h, PAIR_SET[pair_set], _ptr(out), None))
        return out

    def set_launch_shape(self, images_per_cta: int = 0, circuit_threads: int = 0, pauli_threads: int = 0):
        check(lib().mps_set_launch_shape(self._h, int(images_per_cta), int(circuit_threads), int(pauli_threads)))

    # -- diagnostics -----------------------------------------------------------------
    def sync(self):
        check(lib().mps_sync(self._h))

    def bond_dims(self) -> list:
        buf = np.zeros(int((self.n + 1).sum()), dtype=np.int32)
        check(lib().mps_bond_dims(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        out, o = [], 0
        for n in self.n:
            out.append(buf[o:o + n + 1].tolist())
            o += n + 1
        return out

    def set_layer_pipeline(self, enable: bool = True):
        """Layer-pipelined circuit kernel where it applies (ladder, no truncation, L <= 4)."""
        check(lib().mps_set_layer_pipeline(self._h, 1 if enable else 0))

    def set_half_structure(self, enable: bool = True):
        """Contractions over half of the right bond at half-structured sites (ladder
        circuits built as operator products); results are bit-identical either way."""
        check(lib().mps_set_half_structure(self._h, 1 if enable else 0))

    def set_block_truncation(self, enable: bool = True):
        """FP64 truncations may decouple only the kept from the dropped directions when
        the cut lies in a clear gap (the default); False runs the full FP64
        eigen-decomposition every time.  The truncated states agree to rounding."""
        check(lib().mps_set_block_truncation(self._h, 1 if enable else 0))

    def set_real_arithmetic(self, enable: bool = True):
        """Real-element environment and Pauli kernels for a real state (paper ansatz,
        mixed precisions); results agree with the complex kernels to rounding."""
        check(lib().mps_set_real_arithmetic(self._h, 1 if enable else 0))

    def set_pauli_sweep(self, mode="auto"):
        """Pauli-cache kernel at bonds up to 16 under the mixed precisions: "sweep" (one
        sweep per image), "column" (the column walk) or "auto" (the default: the sweep for
        equal-size half-structured batches); True / False stand for "sweep" / "column".
        The kernels give bit-identical caches."""
        if mode is True:
            mode = "sweep"
        elif mode is False:
            mode = "column"
        check(lib().mps_set_pauli_sweep(self._h, PAULI_KERNEL[mode]))

    def set_timing(self, enable: bool = True):
        check(lib().mps_set_timing(self._h, 1 if enable else 0))

    def kernel_times(self) -> dict:
        """{kind: (total ms, launches)} since the last call, from the library's events."""
        ms = (ctypes.c_double * len(_lib.KERNEL_KINDS))()
        cnt = (ctypes.c_int64 * len(_lib.KERNEL_KINDS))()
        check(lib().mps_kernel_times(self._h, ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(_lib.KERNEL_KINDS)}

    def discarded_weight(self) -> np.ndarray:
        buf = np.zeros(self.n_images, dtype=np.float64)
        check(lib().mps_discarded_weight(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return buf


def ano_features(pauli: torch.Tensor, m: int, abd: torch.Tensor, W: torch.Tensor = None,
                 bias: torch.Tensor = None, stream=None, feats: torch.Tensor = None, out: torch.Tensor = None):
    """Features q (Eq. 5) and, if W is given, y = W q + b (Eq. 6).

    pauli: [n_images * m, 16] float32/float64; abd: float32 [m][16]; W: float32 [out][m].
    feats / out: optional preallocated float32 [n_images][m] / [n_images][out] outputs.
    """
    n_images = pauli.shape[0] // m
    if feats is None:
        feats = torch.empty((n_images, m), dtype=torch.float32, device=pauli.device)
    out_dim = 0
    if W is not None:
        out_dim = W.shape[0]
        if out is None:
            out = torch.empty((n_images, out_dim), dtype=torch.float32, device=pauli.device)
    else:
        out = None
    check(lib().ano_features(_ptr(pauli), 1 if pauli.dtype == torch.float64 else 0, n_images, m,
                             _ptr(abd), _ptr(W) if W is not None else None,
                             _ptr(bias) if bias is not None else None, out_dim, _ptr(feats),
                             _ptr(out) if out is not None else None, _stream_handle(stream)))
    return feats, out


def extract(pixels, p, L: int, chi: int, precision: str = "mixed", ansatz: str = "ladder",
            params=None, stream=None) -> torch.Tensor:
    """One-call Pauli cache for a batch of equal-size images.

    pixels: [B][p*p] (host numpy/torch or device tensor, float64); params: [L][p*p][2].
    Returns a device tensor [B][m][16].
    """
    px = torch.as_tensor(pixels, dtype=torch.float64)
    B = px.shape[0]
    px = px.reshape(-1).contiguous().cuda()
    pr = None
    if params is not None:
        pr = torch.as_tensor(params, dtype=torch.float64).contiguous().cuda()
    batch = Batch(np.full(B, p, dtype=np.int32), chi, precision, stream)
    batch.apply_circuit(px, L, ansatz, pr)
    out = batch.pauli_cache()
    batch.sync()
    batch.close()
    return out.reshape(B, -1, 16)


class Pipeline:
    """End-to-end path for a fixed batch layout: host pixels in, host results out.

    Every step copies the pixels from (pinned) host memory to the device, runs the
    circuit, the Pauli cache, the ANO features and the linear layer, and copies the
    Pauli cache, the features and the reconstruction back to pinned host buffers.
    Uploads and downloads run on two copy streams of their own, with `depth` sets of
    device and host buffers, so that the copies of one step overlap the kernels of the
    next (one copy stream for both would queue the next step's upload behind this
    step's download, which waits for this step's kernels, and stall the kernels).
    With overlap (the default) every buffer set also has its own batch and compute
    stream, so the kernels of consecutive steps overlap too: the next step's circuit
    and environment chains (latency-bound, few resources) and its first Pauli CTAs run
    on the SMs that the last wave of this step's Pauli kernel leaves idle.  That takes
    `depth` batches of device memory; overlap=False keeps one batch and one compute
    stream (the stream argument).  Every step is ordered after the work queued on the
    stream argument when it is submitted.  submit() enqueues a step and returns its
    slot, result(slot) waits for that step's results.  A slot's host buffers stay valid
    until the slot is submitted again (`depth` submits later).  run() is submit() then
    result().
    """

    def __init__(self, p, chi, L, precision, params, abd, W=None, bias=None, ansatz="ladder", stream=None,
                 depth: int = 2, overlap: bool = True):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.L, self.ansatz = L, ansatz
        self.params, self.abd, self.W, self.bias = params, abd, W, bias
        p = np.atleast_1d(np.asarray(p))
        if len(set(p.tolist())) != 1:
            raise ValueError("Pipeline needs images of one size (one pair layout for the ANO layer)")
        self.m = pair_count(int(p[0]))
        dev = torch.device("cuda", torch.cuda.current_device())
        depth = max(1, depth)
        if overlap:
            streams = [torch.cuda.Stream(device=dev) for _ in range(depth)]
            batches = [Batch(p, chi, precision, s) for s in streams]
        else:
            streams = [self.stream] * depth
            batches = [Batch(p, chi, precision, self.stream)] * depth
        self.batch = batches[0]
        self.batches = batches if overlap else batches[:1]
        n_px = int(self.batch.pixel_offsets[-1])
        self.copy_stream = torch.cuda.Stream(device=dev)       # host -> device
        self.d2h_stream = torch.cuda.Stream(device=dev)        # device -> host
        dt = torch.float64 if precision == "fp64" else torch.float32
        B = self.batch.n_images
        n_pairs = int(self.batch.pair_offsets[-1])
        self.slots = []
        for i in range(depth):
            sl = {"px": torch.empty(n_px, dtype=torch.float64, device=dev),
                  "pauli": torch.empty((n_pairs, 16), dtype=dt, device=dev),
                  "feats": torch.empty((B, self.m), dtype=torch.float32, device=dev),
                  "out": None if W is None else torch.empty((B, W.shape[0]), dtype=torch.float32, device=dev),
                  "pauli_h": torch.empty((n_pairs, 16), dtype=dt).pin_memory(),
                  "feats_h": torch.empty((B, self.m), dtype=torch.float32).pin_memory(),
                  "out_h": None if W is None else torch.empty((B, W.shape[0]), dtype=torch.float32).pin_memory(),
                  "batch": batches[i], "stream": streams[i],
                  "ev_in": torch.cuda.Event(), "ev_comp": torch.cuda.Event(), "ev_out": torch.cuda.Event(),
                  "ev_user": torch.cuda.Event()}
            self.slots.append(sl)
        self._next = 0
        self.h2d_bytes = n_px * 8
        sl = self.slots[0]
        self.d2h_bytes = (sl["pauli_h"].numel() * sl["pauli_h"].element_size() + sl["feats_h"].numel() * 4
                          + (0 if sl["out_h"] is None else sl["out_h"].numel() * 4))

    def set_launch_shape(self, images_per_cta: int = 0, circuit_threads: int = 0, pauli_threads: int = 0):
        for b in self.batches:
            b.set_launch_shape(images_per_cta, circuit_threads, pauli_threads)

    def sync(self):
        """Wait for every submitted step; raises if a kernel reported an error."""
        for b in self.batches:
            b.sync()

    def submit(self, host_pixels: torch.Tensor) -> int:
        k = self._next
        self._next = (k + 1) % len(self.slots)
        sl = self.slots[k]
        sl["ev_out"].synchronize()          # the previous results of this slot have been read back
        cs, st, b = self.copy_stream, sl["stream"], sl["batch"]
        with torch.cuda.stream(cs):
            cs.wait_event(sl["ev_comp"])     # the previous step of this slot no longer reads its pixels
            sl["px"].copy_(host_pixels, non_blocking=True)
            sl["ev_in"].record(cs)
        with torch.cuda.stream(st):
            if st is not self.stream:
                sl["ev_user"].record(self.stream)
                st.wait_event(sl["ev_user"])
            st.wait_event(sl["ev_in"])
            b.apply_circuit(sl["px"], self.L, self.ansatz, self.params)
            b.pauli_cache(sl["pauli"])
            ano_features(sl["pauli"], self.m, self.abd, self.W, self.bias, st, feats=sl["feats"], out=sl["out"])
            sl["ev_comp"].record(st)
        ds = self.d2h_stream
        with torch.cuda.stream(ds):
            ds.wait_event(sl["ev_comp"])
            sl["pauli_h"].copy_(sl["pauli"], non_blocking=True)
            sl["feats_h"].copy_(sl["feats"], non_blocking=True)
            if sl["out"] is not None:
                sl["out_h"].copy_(sl["out"], non_blocking=True)
            sl["ev_out"].record(ds)
        return k

    def result(self, k: int):
        sl = self.slots[k]
        sl["ev_out"].synchronize()
        return sl["pauli_h"], sl["feats_h"], sl["out_h"]

    def run(self, host_pixels: torch.Tensor):
        return self.result(self.submit(host_pixels))


def save_pauli_cache(path: str, cache: torch.Tensor, meta: dict = None) -> None:
    """Write a Pauli cache (any device, [M][16]) and its description to an .npz file.
    The cache depends on the images only, so training can reload it instead of
    simulating the circuits again (Sec. II.C)."""
    meta = dict(meta or {})
    np.savez(path, cache=cache.detach().cpu().numpy(), meta=np.array(repr(sorted(meta.items()))))


def load_pauli_cache(path: str, device=None) -> torch.Tensor:
    with np.load(path if str(path).endswith(".npz") else str(path) + ".npz") as z:
        t = torch.from_numpy(z["cache"].copy())
    return t.to(device) if device is not None else t


class Trainer:
    """Full-batch training of (A, B, D) and (W, b) on a cached Pauli cache
    (Sec. II.C-D, MSE term of Eq. 7, two Adam optimizers), through ano_train_step.

    pauli: device [n_images * m][16] (float32 or float64); abd [m][16], W [out][m] and
    bias [out] are device float32 tensors trained in place.  step(targets) enqueues
    one step on the stream and returns the device loss (float64 scalar tensor) at
    the parameters before the update.
    """

    def __init__(self, pauli: torch.Tensor, m: int, abd: torch.Tensor, W: torch.Tensor, bias: torch.Tensor,
                 lr_abd: float = 1e-2, lr_linear: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8, mse_weight: float = 1.0, stream=None):
        for name, t in (("abd", abd), ("W", W), ("bias", bias)):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        self.pauli, self.m = pauli, m
        self.n_images = pauli.shape[0] // m
        self.abd, self.W, self.bias = abd, W, bias
        self.out_dim = W.shape[0]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.hp = _lib.ano_adam(lr_abd, lr_linear, beta1, beta2, eps, mse_weight)
        n_par = m * 16 + self.out_dim * m + self.out_dim
        self.moments = torch.zeros(2 * n_par, dtype=torch.float32, device=pauli.device)
        n_ws = lib().ano_train_workspace_floats(self.n_images, m, self.out_dim)
        if n_ws < 0:
            raise ValueError("bad training sizes")
        self.workspace = torch.zeros(int(n_ws), dtype=torch.float32, device=pauli.device)
        self.loss = torch.zeros((), dtype=torch.float64, device=pauli.device)
        self.t = 0

    def step(self, targets: torch.Tensor) -> torch.Tensor:
        assert targets.is_cuda and targets.dtype == torch.float32 and targets.is_contiguous()
        assert targets.shape == (self.n_images, self.out_dim)
        self.t += 1
        check(lib().ano_train_step(_ptr(self.pauli), 1 if self.pauli.dtype == torch.float64 else 0,
                                   self.n_images, self.m, _ptr(self.abd), _ptr(self.W), _ptr(self.bias),
                                   self.out_dim, _ptr(targets), _ptr(self.moments), self.t,
                                   ctypes.byref(self.hp), _ptr(self.workspace), _ptr(self.loss),
                                   _stream_handle(self.stream)))
        return self.loss

    def gradients(self):
        """Views of the last step's gradients (g_abd [m][16], g_W [out][m], g_b [out])."""
        B, m, O = self.n_images, self.m, self.out_dim
        g0 = 2 * B * m + B * O
        g = self.workspace[g0:g0 + m * 16 + O * m + O]
        return g[:m * 16].view(m, 16), g[m * 16:m * 16 + O * m].view(O, m), g[m * 16 + O * m:]

    def state_dict(self) -> dict:
        return {"abd": self.abd.clone(), "W": self.W.clone(), "bias": self.bias.clone(),
                "moments": self.moments.clone(), "t": self.t}

    def load_state_dict(self, sd: dict) -> None:
        self.abd.copy_(sd["abd"])
        self.W.copy_(sd["W"])
        self.bias.copy_(sd["bias"])
        self.moments.copy_(sd["moments"])
        self.t = int(sd["t"])
