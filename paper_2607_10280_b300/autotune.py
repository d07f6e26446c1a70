"""Launch-shape autotuner for the CUDA kernels.

The circuit kernel runs one team of `circuit_threads` threads per image (several
one-warp images per CTA when the team is a single warp: `images_per_cta`); the
Pauli kernel runs one team of `pauli_threads` threads per (image, grid column)
unit.  The best shape depends on the image mix, the bond dimension and the GPU,
so it is measured: every candidate runs the real workload a few times and the
library's per-kernel CUDA events (``Batch.set_timing``) give each kernel's time.
The two kernels do not interact, so each knob set is tuned on its own kernel's
time.  Choices are cached in a JSON file keyed by GPU name and a workload
signature.
"""
from __future__ import annotations

import json
import os

CIRCUIT_SHAPES = [(1, 32), (2, 32), (4, 32), (1, 64)]   # (images_per_cta, circuit_threads)
PAULI_THREADS = [32, 64, 128]


def _cache_path() -> str:
    return os.environ.get("MPSANO_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mpsano_autotune.json"))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(path, data):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except Exception:
        pass


def signature(batch, L, ansatz="ladder") -> str:
    """Workload key: image sizes, bond caps, layers, precision, ansatz."""
    import numpy as np
    ps, counts = np.unique(batch.p, return_counts=True)
    mix = ",".join(f"{int(p)}x{int(c)}" for p, c in zip(ps, counts))
    chis = ",".join(str(int(c)) for c in sorted(set(batch.chi.tolist())))
    Ls = ",".join(str(int(v)) for v in sorted(set(np_atleast(L))))
    return f"p[{mix}]chi[{chis}]L[{Ls}]{batch.precision}/{ansatz}"


def np_atleast(v):
    import numpy as np
    return np.atleast_1d(np.asarray(v)).tolist()


def tune(batch, run_step, key: str, reps: int = 3, use_cache: bool = True, verbose: bool = False) -> dict:
    """Pick the launch shape of `batch` for the workload that `run_step()` enqueues.

    run_step must enqueue one full pass (circuit + Pauli cache) on the batch's
    stream.  Returns {'images_per_cta', 'circuit_threads', 'pauli_threads',
    'circuit_ms', 'pauli_ms', 'source'} and leaves the batch set to that shape.
    """
    import torch
    dev = torch.cuda.get_device_name()
    full_key = f"{dev}|{key}"
    path = _cache_path()
    cache = _load(path) if use_cache else {}
    if full_key in cache:
        c = cache[full_key]
        batch.set_launch_shape(c["images_per_cta"], c["circuit_threads"], c["pauli_threads"])
        return dict(c, source="cache")

    def measure(kind):
        batch.set_timing(True)
        batch.kernel_times()
        run_step()                     # warm
        batch.kernel_times()
        for _ in range(reps):
            run_step()
        t = batch.kernel_times()
        batch.set_timing(False)
        return t[kind][0] / max(1, t[kind][1])

    best_c = None
    for ipc, ct in CIRCUIT_SHAPES:
        batch.set_launch_shape(ipc, ct, 0)
        ms = measure("circuit")
        if verbose:
            print(f"circuit images_per_cta={ipc} threads={ct}: {ms:.3f} ms")
        if best_c is None or ms < best_c[0]:
            best_c = (ms, ipc, ct)
    batch.set_launch_shape(best_c[1], best_c[2], 0)
    best_p = None
    for pt in PAULI_THREADS:
        batch.set_launch_shape(0, 0, pt)
        ms = measure("pauli")
        if verbose:
            print(f"pauli threads={pt}: {ms:.3f} ms")
        if best_p is None or ms < best_p[0]:
            best_p = (ms, pt)
    batch.set_launch_shape(best_c[1], best_c[2], best_p[1])
    choice = {"images_per_cta": best_c[1], "circuit_threads": best_c[2], "pauli_threads": best_p[1],
              "circuit_ms": best_c[0], "pauli_ms": best_p[0]}
    if use_cache:
        cache = _load(path)
        cache[full_key] = choice
        _store(path, cache)
    return dict(choice, source="measured")
