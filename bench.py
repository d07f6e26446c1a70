"""Benchmark of the MPS-ANO-VQC feature-extraction hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (one step): 1024 synthetic garment-like 7x7 images (49 qubits each),
ladder ansatz with L = 4 layers, bond dimension chi = 16, mixed precision
(complex64 state, FP64 inside truncations): circuit -> MPS -> Pauli cache of the
84 horizontal/vertical pairs x 16 Paulis -> ANO features -> linear layer 84 ->
784.  Metric: images/s.  Under torchrun every rank runs its own batch of 1024
images (weak scaling; no collective on the data path).

Prints one JSON line (rank 0).  Beside the headline it reports the same images
through the plain per-image FP64 GPU path, the error of the mixed path against
the FP64 oracle on sampled images, the roofline of the dominant kernel, clocks
sampled during the timed region, and the oracle timed on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))

# The committed ncu summary of each timed kernel and the sources that build it: the
# DRAM traffic a capture recorded is reported only while these files are unchanged
# (the summary carries their hash).
PROFILED = {
    "pauli": ("profiles/pauli_sweep_kernel_7x7_L4_chi16_b1024.md",
              ("pauli_sweep.cuh", "pauli_launch_sweep.cu", "pauli.cuh", "linalg.cuh", "common.cuh")),
    "circuit": ("profiles/ladder_mpo_direct_kernel_7x7_L4_chi16_b1024.md",
                ("ladder_mpo.cu", "circuit.cuh", "common.cuh")),
    "renv": ("profiles/lenv_kernel_7x7_L4_chi16_b1024.md",
             ("pauli_sweep.cuh", "pauli_launch_sweep.cu", "pauli.cuh", "linalg.cuh", "common.cuh")),
    "chain": ("profiles/circuit_kernel_fp64_chain_7x7_L4_chi8_b1024.md",
              ("circuit.cuh", "circuit_launch.cuh", "linalg.cuh", "common.cuh")),
}


def source_hash(files) -> str:
    """sha256 over the named files of the package's csrc/ (name, then bytes)."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2607_10280_b300", "csrc", f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel: str):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed ncu
    summary of `kernel` (a capture of this benchmark's own launch), or None when there
    is none or the kernel's sources changed after it was taken."""
    import re
    spec = PROFILED.get(kernel)
    if spec is None:
        return None
    path, files = spec
    try:
        with open(os.path.join(ROOT, path)) as fh:
            text = fh.read()
    except OSError:
        return None
    m = re.search(r"Source hash \(sha256\): ([0-9a-f]{64})", text)
    if not m or m.group(1) != source_hash(files):
        return None
    total = 0.0
    for name in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        m = re.search(r"\| " + re.escape(name) + r" \| ([0-9.]+) \| (\w+) \|", text)
        scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(m.group(2)) if m else None
        if scale is None:
            return None
        total += float(m.group(1)) * scale
    return total
sys.path.insert(0, ROOT)

P, L, CHI, BATCH = 7, 4, 16, 1024
OUT_DIM = 784
METRIC = "images/s @49q L=4 chi=16 batched mixed (c64 + FP64 truncation) vs plain FP64"
WORKLOAD = {"workload": "7x7 garment-like images (49 qubits), ladder ansatz L=4, chi=16, "
                        "84 H+V pairs x 16 Paulis, ANO + linear 84->784",
            "images_per_gpu": BATCH, "p": P, "L": L, "chi": CHI, "pairs": 84,
            "precision": "mixed", "data": "synthetic garment-like pixels, seed 0"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600, help="timed steps (600 headline steps take about 1.1 s)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-sample", type=int, default=8, help="images timed through the per-image FP64 path")
    ap.add_argument("--batch", type=int, default=BATCH, help="images per GPU (profiling of smaller cases)")
    ap.add_argument("--config", default="headline", choices=["headline", "sweep", "trunc", "large_chi", "paper",
                                                            "uneven", "large", "serve", "train", "diag"],
                    help="headline (default): 7x7 L=4 chi=16; the others are the chi x L sweep, the uneven "
                         "batch, the 16x16 batch, the serving run, training on cached Paulis and the "
                         "156-pair layout with diagonals")
    ap.add_argument("--requests", type=int, default=20000, help="serving run: number of requests (10 s at 2000/s)")
    ap.add_argument("--serve-slots", type=int, default=6, help="serving run: execution slots")
    ap.add_argument("--serve-long-slots", type=int, default=4,
                    help="serving run: slots reserved for requests that run a truncating chain")
    ap.add_argument("--pauli-kernel", default="default", choices=["default", "sweep", "column"],
                    help="Pauli-cache kernel at bonds up to 16 (mps_set_pauli_sweep); default: the library's")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------ oracle on CPU
def oracle_sample(n_images: int, processes: int):
    """Time the CPU oracle on a bounded sample of the workload; returns (images/s, cores, sample)."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"   # inherited by the spawned oracle workers
    from oracle import pipeline
    from paper_2607_10280_b300 import synth
    X = synth.garment_pixels(n_images, P)
    params = synth.circuit_params(L, P * P)
    t0 = time.perf_counter()
    pipeline.pauli_cache_batch(X, P, L, CHI, "ladder", params, processes=processes)
    dt = time.perf_counter() - t0
    return n_images / dt, processes, f"{n_images} of the 7x7 L=4 chi=16 images, oracle MPS (numpy FP64), " \
                                     f"{processes} spawn processes x 1 BLAS thread, Pauli cache only"


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, gpu_index=0):
        try:
            rows = [r.split(", ") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = [r for r in rows if len(r) >= 9 and r[0].strip() == str(gpu_index)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        load = [s for s in sm if s > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = cpu_cores()
    procs = min(cores, 16)
    per_step = max(procs, 8)
    times = []
    for i in range(args.warmup + args.steps):
        v, c, sample = oracle_sample(per_step, procs)
        if i >= args.warmup:
            times.append(per_step / v)
    value = per_step * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, precision="fp64 oracle", images_per_step=per_step),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "images/s", "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    global BATCH
    BATCH = args.batch
    WORKLOAD["images_per_gpu"] = BATCH
    rank, world, local = dist_env()
    cores = cpu_cores()
    # the oracle baseline is timed first, before any CUDA context exists on this process
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        procs = min(cores, 16)
        v, c, sample = oracle_sample(2 * procs, procs)
        cpu = {"value": v, "unit": "images/s", "cores": c, "kind": "oracle", "sample": sample}

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from oracle import pipeline as opipe
    from paper_2607_10280_b300 import api, flops, synth
    from paper_2607_10280_b300.build import build
    build()
    if PAULI_KERNEL != "default":
        api.Batch.pauli_kernel_default = PAULI_KERNEL

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    m = api.pair_count(P)
    X = synth.garment_pixels(BATCH, P, seed=synth.SEED_PIXELS + 7919 * rank)
    params_np = synth.circuit_params(L, P * P)
    abd_np = synth.observable_params(m)
    W_np, b_np = synth.linear_params(OUT_DIM, m)
    pixels = torch.tensor(X.reshape(-1), dtype=torch.float64, device=dev)
    params = torch.tensor(params_np, dtype=torch.float64, device=dev)
    abd = torch.tensor(abd_np, dtype=torch.float32, device=dev)
    W = torch.tensor(W_np, dtype=torch.float32, device=dev)
    bias = torch.tensor(b_np, dtype=torch.float32, device=dev)
    batch = api.Batch(np.full(BATCH, P, np.int32), CHI, "mixed", stream)
    pauli = torch.empty((BATCH * m, 16), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)   # > 126 MB L2

    def step():
        batch.apply_circuit(pixels, L, "ladder", params)
        batch.pauli_cache(pauli)
        return api.ano_features(pauli, m, abd, W, bias)

    def path_only():
        batch.apply_circuit(pixels, L, "ladder", params)
        batch.pauli_cache(pauli)

    # launch shapes measured on this workload (untimed; part of the warm-up)
    from paper_2607_10280_b300 import autotune
    shape = autotune.tune(batch, path_only, autotune.signature(batch, L), use_cache=False)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # correctness guard on sampled images against the FP64 oracle (before timing)
    feats, out = step()
    torch.cuda.synchronize()
    got = pauli.double().cpu().numpy().reshape(BATCH, m, 16)
    err_idx = [0, BATCH // 2, BATCH - 1]
    errs = [np.abs(got[i] - opipe.pauli_cache(X[i], P, L, CHI, "ladder", params_np)) for i in err_idx]
    err = {"max_abs": float(max(e.max() for e in errs)), "mae": float(np.mean([e.mean() for e in errs])),
           "images": len(err_idx), "reference": "CPU FP64 oracle at chi=16 (exact: chi = 2^L)", "tolerance": 1e-5}

    # ---------------- timed region (device events per step; L2 flushed between steps)
    batch.set_timing(True)
    batch.kernel_times()
    n0 = api.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # raw clock samples (the JSON line carries their summary)
    import tempfile
    clock_path = os.path.join(os.environ.get("BENCH_OUT_DIR", tempfile.gettempdir()), f"bench_clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clock_path), exist_ok=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(clock_path) as clk:
        t_wall = time.perf_counter()
        kt = {"circuit": [0.0, 0], "renv": [0.0, 0], "pauli": [0.0, 0]}
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    launches = (api.launch_count() - n0) / args.steps
    for k, (ms, cnt) in batch.kernel_times().items():
        kt[k] = [ms, cnt]
    batch.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * BATCH * args.steps / (total_ms / 1e3)

    # ---------------- sustained: the same step for at least 1 s with clocks sampled, when
    # the K timed steps are shorter than that (the clock record needs samples)
    sustained = None
    step_s = total_ms / args.steps / 1e3
    if t_wall < 1.0:
        n_sus = int(np.ceil(1.0 / max(step_s, 1e-6)))
        with ClockSampler(clock_path.replace(".csv", "_sustained.csv")) as clk_sus:
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            for _ in range(n_sus):
                step()
            e_b.record(stream)
            torch.cuda.synchronize()
        sus_ms = e_a.elapsed_time(e_b)
        sustained = {"steps": n_sus, "value": world * BATCH * n_sus / (sus_ms / 1e3), "unit": "images/s",
                     "ms_per_step": sus_ms / n_sus, "l2": "not flushed between these steps",
                     "clocks": clk_sus.summary(local)}

    # ---------------- roofline of the dominant kernel (ALU bound, FP32 pipe)
    fk = "column" if PAULI_KERNEL == "column" else "sweep"
    f = flops.image_flops(P, L, CHI, kernel=fk)
    # the same contraction without exploiting the half-structured sites (context only)
    f_dense = flops.image_flops(P, L, CHI, dense=True, kernel=fk)
    dom = max(("circuit", "renv", "pauli"), key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / max(1, kt[dom][1])
    achieved = BATCH * f[dom] / (dom_ms / 1e3) / 1e12
    peak = 148 * 128 * 2 * 2.032e9 / 1e12   # FP32 lanes x FMA x max SM clock
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": profiled_traffic(dom), "traffic_unit": "bytes per launch (ncu capture of this launch)",
                "kernel": dom, "pipe": "fp32",
                "peak_note": "148 SMs x 128 FP32 lanes x 2 flops x 2032 MHz (nominal); the FMA probe measured 65.6",
                "kernel_ms": {k: kt[k][0] / max(1, kt[k][1]) for k in kt},
                "flops_per_image": f,
                "dense_form": {"flops_per_image": f_dense[dom],
                               "tflops_equivalent": BATCH * f_dense[dom] / (dom_ms / 1e3) / 1e12,
                               "note": "the same contraction without skipping the structural zeros of "
                                       "half-structured sites; achieved counts only the work done"}}

    # ---------------- end to end through the public API with host buffers
    pipe = api.Pipeline(np.full(BATCH, P, np.int32), CHI, L, "mixed", params, abd, W, bias, stream=stream)
    pipe.set_launch_shape(shape["images_per_cta"], shape["circuit_threads"], shape["pauli_threads"])
    host_px = torch.tensor(X.reshape(-1), dtype=torch.float64).pin_memory()
    # untimed warm-up of every buffer slot of the pipeline (W steps, at least two rounds
    # of the slots), as for the device-timed loop
    for _ in range(max(args.warmup, 2 * len(pipe.slots))):
        pipe.run(host_px)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps, int(np.ceil(1.0 / max(step_s, 1e-6))))   # at least about 1 s
    # every step: pinned host pixels -> device, the whole path, results -> pinned host
    # memory, read on the host; a step's copies and kernels overlap the next step's (a
    # batch and a compute stream per buffer slot)
    with ClockSampler(clock_path.replace(".csv", "_e2e.csv")) as clk_e2e:
        t0 = time.perf_counter()
        prev = None
        for _ in range(e2e_steps):
            k = pipe.submit(host_px)
            if prev is not None:
                res = pipe.result(prev)
            prev = k
        res = pipe.result(prev)
        torch.cuda.synchronize()
        e2e_dt = time.perf_counter() - t0
    e2e = {"value": world * BATCH * e2e_steps / e2e_dt, "unit": "images/s",
           "h2d_bytes_per_step": pipe.h2d_bytes, "d2h_bytes_per_step": pipe.d2h_bytes,
           "steps": e2e_steps, "overlap": "consecutive steps on two compute streams (one batch each)",
           "clocks": clk_e2e.summary(local)}

    # ---------------- the plain per-image FP64 GPU path on a sample of the same images
    ns = args.fp64_sample
    single = [api.Batch(np.array([P], np.int32), CHI, "fp64", stream) for _ in range(1)]
    px1 = [torch.tensor(X[i], dtype=torch.float64, device=dev) for i in range(ns)]
    out64 = torch.empty((m, 16), dtype=torch.float64, device=dev)
    single[0].apply_circuit(px1[0], L, "ladder", params)
    single[0].pauli_cache(out64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(ns):
        single[0].apply_circuit(px1[i], L, "ladder", params)
        single[0].pauli_cache(out64)
        api.ano_features(out64, m, abd, W, bias)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_per_image = ns / (e0.elapsed_time(e1) / 1e3)
    # ---------------- the batched FP64 path on the same 1024 images (same kernels, complex128)
    b64 = api.Batch(np.full(BATCH, P, np.int32), CHI, "fp64", stream)
    pauli64 = torch.empty((BATCH * m, 16), dtype=torch.float64, device=dev)

    def step64():
        b64.apply_circuit(pixels, L, "ladder", params)
        b64.pauli_cache(pauli64)
        return api.ano_features(pauli64, m, abd, W, bias)
    step64()
    torch.cuda.synchronize()
    n64 = 5
    ms64 = _time_events(torch, step64, n64, stream)
    b64.close()
    fp64_batched = {"value": BATCH / (ms64 / 1e3), "unit": "images/s", "ms_per_step": ms64, "steps": n64,
                    "speedup_of_mixed_batched": value / world / (BATCH / (ms64 / 1e3))}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
                "config": dict(WORKLOAD, l2="flushed between timed steps (256 MB write outside the step events)",
                               parallelism=f"replicas x{world}",
                               launch_shape={k: shape[k] for k in ("images_per_cta", "circuit_threads",
                                                                   "pauli_threads")}),
                "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
                "clocks": clk.summary(local),
                "fp64_per_image_gpu": {"value": fp64_per_image, "unit": "images/s", "sample": ns,
                                       "speedup_of_mixed_batched": value / world / fp64_per_image},
                "fp64_batched_gpu": fp64_batched, "sustained": sustained,
                "error_vs_fp64_oracle": err, "wall_s_timed": t_wall}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ other configurations
def run_diag(args):
    """The paper's full 7x7 pair layout: horizontal, vertical and both diagonal
    neighbours (156 pairs), 1024 images, L = 4, chi = 16, mixed precision, then ANO
    (156 x 16) and a linear layer 156 -> 784; beside it the same batch with the 84
    H+V pairs.  The site tensors (205 MB) exceed L2, so timed steps read HBM."""
    torch = _setup_torch()
    from oracle import pipeline as opipe
    from paper_2607_10280_b300 import api, synth
    p, B, L, chi = 7, 1024, 4, 16
    X = synth.garment_pixels(B, p)
    params_np = synth.circuit_params(L, p * p)
    params = torch.tensor(params_np, dtype=torch.float64, device="cuda")
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    sample = [0, B // 2, B - 1]
    rows = {}
    for pair_set, diagonals in (("hvd", True), ("hv", False)):
        m = api.pair_count(p, pair_set)
        abd = torch.tensor(synth.observable_params(m), dtype=torch.float32, device="cuda")
        W = torch.tensor(np.random.default_rng(3).standard_normal((p * p * 16, m)) / np.sqrt(m),
                         dtype=torch.float32, device="cuda")
        bias = torch.zeros(p * p * 16, dtype=torch.float32, device="cuda")
        b = api.Batch(np.full(B, p, np.int32), chi, "mixed")
        pauli = torch.empty((B * m, 16), dtype=torch.float32, device="cuda")

        def step():
            b.apply_circuit(px, L, "ladder", params)
            b.pauli_cache(pauli, pair_set)
            return api.ano_features(pauli, m, abd, W, bias)
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        ms = _time_events(torch, step, max(10, args.steps))
        got = pauli.double().cpu().numpy().reshape(B, m, 16)
        err = max(float(np.max(np.abs(got[i] - opipe.pauli_cache(X[i], p, L, chi, "ladder", params_np,
                                                                   diagonals=diagonals))))
                  for i in sample)
        rows[pair_set] = {"pairs": m, "ms_per_step": ms, "images_per_s": B / (ms / 1e3),
                          "max_err_vs_oracle_sampled": err}
        b.close()
        print(json.dumps({pair_set: rows[pair_set]}), file=sys.stderr, flush=True)
    line = {"metric": "images/s, 7x7 L=4 chi=16 batch 1024, 156 H+V+diagonal pairs + ANO + linear 156->784",
            "value": rows["hvd"]["images_per_s"], "unit": "images/s", "n_gpus": 1,
            "config": {"workload": "7x7 garment-like, ladder ansatz, L=4, chi=16, mixed; pair sets hvd (156) and hv (84)",
                       "images": B, "l2": "site tensors 205 MB > L2"},
            "table": rows}
    print(json.dumps(line), flush=True)


PAULI_KERNEL = "default"


def _setup_torch():
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2607_10280_b300.build import build
    build()
    if PAULI_KERNEL != "default":
        from paper_2607_10280_b300 import api
        api.Batch.pauli_kernel_default = PAULI_KERNEL
    return torch


def _time_events(torch, fn, steps, stream=None):
    stream = stream or torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_sweep(args):
    """chi x L sweep at 7x7 (Sec. III, Fig. 3): per (L, chi), chi = 2 .. 2048, the mixed and
    FP64 batched paths, their MAE (Eq. 7) and max error vs the FP64 oracle at chi = 64,
    whether the FP64 path is near-exact (MAE <= 1e-12, Sec. III), and images/s.  Bonds
    never exceed 2^L, so every chi >= 2^L gives the exact state at the cost of chi = 2^L.
    At a truncated point (chi < 2^L) every image's circuit truncates lossily, so the mixed
    path runs all of them on its complex128 chain; the complex64-state chain
    (mixed_fast) is timed beside it with its error, which is what the FP64 state buys."""
    torch = _setup_torch()
    from oracle import pipeline as opipe
    from paper_2607_10280_b300 import api, flops, synth
    B = min(args.batch, 1024)
    m = api.pair_count(P)
    X = synth.garment_pixels(B, P)
    sample = [0, B // 2, B - 1]
    rows = []
    for Lr in (1, 2, 3, 4):
        params_np = synth.circuit_params(Lr, P * P)
        params = torch.tensor(params_np, dtype=torch.float64, device="cuda")
        px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
        refs = [opipe.pauli_cache(X[i], P, Lr, 64, "ladder", params_np) for i in sample]
        for chi in (2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048):
            res = {}
            lossy = flops.lossy(P, Lr, chi)
            for prec in ("mixed", "fp64") + (("mixed_fast",) if lossy else ()):
                b = api.Batch(np.full(B, P, np.int32), chi, prec)
                pauli = torch.empty((B * m, 16), dtype=torch.float64 if prec == "fp64" else torch.float32,
                                    device="cuda")

                def step():
                    b.apply_circuit(px, Lr, "ladder", params)
                    b.pauli_cache(pauli)
                step()
                torch.cuda.synchronize()
                ms = _time_events(torch, step, 3 if prec == "fp64" else 10)
                got = pauli.double().cpu().numpy().reshape(B, m, 16)
                res[prec] = (ms, got, b.discarded_weight())
                b.close()
            errs = [np.abs(res["mixed"][1][i] - refs[k]) for k, i in enumerate(sample)]
            errs64 = [np.abs(res["fp64"][1][i] - refs[k]) for k, i in enumerate(sample)]
            row = {"L": Lr, "chi": chi,
                   "mae_mixed_vs_exact": float(np.mean([e.mean() for e in errs])),
                   "max_mixed_vs_exact": float(max(e.max() for e in errs)),
                   "mae_fp64_vs_exact": float(np.mean([e.mean() for e in errs64])),
                   "near_exact_fp64": bool(np.mean([e.mean() for e in errs64]) <= 1e-12),
                   "max_mixed_vs_fp64_gpu_all_images": float(np.max(np.abs(res["mixed"][1] - res["fp64"][1]))),
                   "images_on_complex128_chain": B if lossy else 0,
                   "discarded_weight_mean": float(np.mean(res["fp64"][2])),
                   "images_per_s_mixed": B / (res["mixed"][0] / 1e3),
                   "images_per_s_fp64": B / (res["fp64"][0] / 1e3)}
            if lossy:
                e_fast = np.abs(res["mixed_fast"][1] - res["fp64"][1]).reshape(B, -1).max(1)
                row.update({"images_per_s_mixed_fast": B / (res["mixed_fast"][0] / 1e3),
                            "max_mixed_fast_vs_fp64_gpu_all_images": float(e_fast.max()),
                            "mixed_fast_images_over_1e-5": int((e_fast > 1e-5).sum())})
            rows.append(row)
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    line = {"metric": "chi x L sweep at 7x7: MAE vs exact (chi=64 FP64 oracle) and images/s", "value":
            rows[-1]["images_per_s_mixed"], "unit": "images/s", "n_gpus": 1, "config":
            {"workload": "7x7 garment-like, ladder ansatz, L in 1..4, chi in {2,4,...,2048}", "images": B,
             "exact_reference": "oracle MPS chi=64 on 3 sampled images"},
            "max_mixed_vs_fp64_gpu_all_points": max(r["max_mixed_vs_fp64_gpu_all_images"] for r in rows),
            "table": rows}
    print(json.dumps(line), flush=True)


def run_trunc(args):
    """The chi x L sweep's truncated point that costs most: 1024 garment-like 7x7 images,
    L = 4, chi = 8 (the exact bond 16 is cut to 8 at the middle cuts of every layer).
    MPS_MIXED runs these chains on a complex128 state (its truncating circuit kernel is
    the FP64 one), so the roofline is the circuit kernel's FP64 pipe; beside it the
    plain FP64 path and the complex64-state chain (MPS_MIXED_FAST, which misses 1e-5)."""
    torch = _setup_torch()
    from oracle import pipeline as opipe
    from paper_2607_10280_b300 import api, flops, synth
    p, B, Lr, chi = 7, min(args.batch, 1024), 4, 8
    m = api.pair_count(p)
    X = synth.garment_pixels(B, p)
    params_np = synth.circuit_params(Lr, p * p)
    params = torch.tensor(params_np, dtype=torch.float64, device="cuda")
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    res = {}
    steps = max(5, min(args.steps, 40))
    for prec in ("mixed", "fp64", "mixed_fast"):
        b = api.Batch(np.full(B, p, np.int32), chi, prec)
        pauli = torch.empty((B * m, 16), dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")

        def step():
            b.apply_circuit(px, Lr, "ladder", params)
            b.pauli_cache(pauli)
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        b.set_timing(True)
        b.kernel_times()
        ms = _time_events(torch, step, steps)
        kt = {k: v[0] / steps for k, v in b.kernel_times().items()}   # ms per step and kind
        b.set_timing(False)
        res[prec] = {"ms_per_step": ms, "images_per_s": B / (ms / 1e3), "kernel_ms_per_step": kt,
                     "pauli": pauli.double().cpu().numpy().reshape(B, m, 16)}
        b.close()
    err_fp64 = np.abs(res["mixed"]["pauli"] - res["fp64"]["pauli"]).reshape(B, -1).max(1)
    err_fast = np.abs(res["mixed_fast"]["pauli"] - res["fp64"]["pauli"]).reshape(B, -1).max(1)
    sample = [0, B // 2, B - 1]
    oerr = []
    for i in sample:
        ref, st = opipe.pauli_cache(X[i], p, Lr, chi, "ladder", params_np, return_state=True)
        if st.min_gap >= 1e-6:
            oerr.append(float(np.max(np.abs(res["mixed"]["pauli"][i] - ref))))
    f = flops.circuit_flops_by_pipe(p * p, Lr, chi, "ladder", "fp64")
    circ_ms = res["mixed"]["kernel_ms_per_step"]["circuit"]
    peak64, peak32 = 1.25, 148 * 128 * 2 * 2.032e9 / 1e12
    achieved = B * f["fp64"] / (circ_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                "frac": achieved / peak64, "traffic": profiled_traffic("chain"),
                "kernel": "circuit (FP64 chain + rounding)",
                "peak_note": "nominal FP64 rate of B300 (1.25 TFLOP/s, about 2 DFMA per SM and clock at 2032 MHz)",
                "fp32_side": {"achieved": B * f["fp32"] / (circ_ms / 1e3) / 1e12, "peak": peak32,
                              "note": "FP32 Jacobi that starts each eigen-decomposition"},
                "flops_per_image": f, "kernel_ms": circ_ms}
    for r in res.values():
        del r["pauli"]
    line = {"metric": "images/s, 7x7 L=4 chi=8 batch 1024 (truncated regime), mixed at <=1e-5",
            "value": res["mixed"]["images_per_s"], "unit": "images/s", "n_gpus": 1, "higher_is_better": True,
            "config": {"workload": "7x7 garment-like images, ladder ansatz L=4, chi=8, 84 H+V pairs x 16 Paulis "
                                   "(circuit + Pauli cache)", "images": B, "steps": steps},
            "table": res, "roofline": roofline,
            "max_err_mixed_vs_fp64_gpu_all_images": float(err_fp64.max()),
            "max_err_mixed_fast_vs_fp64_gpu_all_images": float(err_fast.max()),
            "images_over_1e-5_mixed_fast": int((err_fast > 1e-5).sum()),
            "max_err_mixed_vs_oracle_sampled": max(oerr) if oerr else None}
    print(json.dumps(line), flush=True)


def run_large_chi(args):
    """The large-chi end of the paper's sweep (Sec. III): 64 garment-like 7x7 images at
    L = 5, 6, 7 with chi in {16, 32, 64, 128}.  Bonds above 32 run the kernels with their
    workspaces in global memory; at L = 7, chi = 64 the cut from 128 to 64 binds.  Per row:
    images/s (mixed and FP64), the discarded weight, and the MAE and max error (Eq. 7) of
    the mixed path against the FP64 path at chi = 2^L (exact)."""
    torch = _setup_torch()
    from paper_2607_10280_b300 import api, synth
    p, B = 7, min(args.batch, 64)
    m = api.pair_count(p)
    X = synth.garment_pixels(B, p)
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    rows = []
    for Lr in (5, 6, 7):
        params = torch.tensor(synth.circuit_params(Lr, p * p), dtype=torch.float64, device="cuda")
        exact = None
        res = {}
        for chi in (128, 64, 32, 16):
            r = {"L": Lr, "chi": chi}
            for prec in ("fp64", "mixed"):
                b = api.Batch(np.full(B, p, np.int32), chi, prec)
                out = torch.empty((B * m, 16), dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")

                def step():
                    b.apply_circuit(px, Lr, "ladder", params)
                    b.pauli_cache(out)
                step()
                torch.cuda.synchronize()
                ms = _time_events(torch, step, 2)
                r[f"images_per_s_{prec}"] = B / (ms / 1e3)
                got = out.double().cpu().numpy().reshape(B, m, 16)
                if prec == "fp64":
                    r["discarded_weight_mean"] = float(np.mean(b.discarded_weight()))
                    r["max_bond"] = int(max(max(x) for x in b.bond_dims()))
                    if chi == 128:
                        exact = got
                res[prec] = got
                b.close()
            e = np.abs(res["mixed"] - exact)
            r["mae_mixed_vs_exact"] = float(e.mean())
            r["max_mixed_vs_exact"] = float(e.max())
            r["max_mixed_vs_fp64_same_chi"] = float(np.max(np.abs(res["mixed"] - res["fp64"])))
            rows.append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
    line = {"metric": "large-chi sweep at 7x7: images/s and error vs exact (chi = 2^L), L = 5..7, chi = 16..128",
            "value": rows[-1]["images_per_s_mixed"], "unit": "images/s", "n_gpus": 1,
            "config": {"workload": "7x7 garment-like, ladder ansatz, L in 5..7, chi in {16,32,64,128}", "images": B,
                       "exact_reference": "the FP64 path at chi = 128 (= 2^L for L = 7, exact below)"},
            "table": rows}
    print(json.dumps(line), flush=True)


def run_paper(args):
    """The paper's own circuit (Sec. II.B, Eq. 2: H, R_Y(2 pi x - pi), staggered CNOTs, L
    encoding-entangling layers) on 1024 garment-like 7x7 images at chi = 2^L (its first
    near-exact point, Sec. III), circuit + Pauli cache for the 84 H+V pairs and the
    paper's 156-pair layout with diagonals.  Its state is real: the mixed path runs the
    real-element environment and Pauli kernels, shown beside the complex ones and the
    FP64 path, with the max error against FP64 over all images."""
    torch = _setup_torch()
    from paper_2607_10280_b300 import api, synth
    p, B = 7, min(args.batch, 1024)
    X = synth.garment_pixels(B, p)
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    rows = []
    for pair_set in ("hv", "hvd"):
        m = api.pair_count(p, pair_set)
        for Lr in (1, 2, 3, 4):
            chi = 1 << Lr
            r = {"pairs": pair_set, "L": Lr, "chi": chi}
            outs = {}
            for name, prec, real in (("mixed_real", "mixed", True), ("mixed_complex", "mixed", False),
                                     ("fp64", "fp64", False)):
                b = api.Batch(np.full(B, p, np.int32), chi, prec)
                b.set_real_arithmetic(real)
                out = torch.empty((B * m, 16), dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")

                def step():
                    b.apply_circuit(px, Lr, "paper")
                    b.pauli_cache(out, pair_set)
                step()
                torch.cuda.synchronize()
                b.set_timing(True)
                b.kernel_times()
                steps = 10 if prec != "fp64" else 3
                ms = _time_events(torch, step, steps)
                kt = {k: v[0] / steps for k, v in b.kernel_times().items()}
                b.close()
                r[f"images_per_s_{name}"] = B / (ms / 1e3)
                r[f"kernel_ms_{name}"] = kt
                outs[name] = out.double().cpu().numpy()
            r["max_err_mixed_real_vs_fp64"] = float(np.max(np.abs(outs["mixed_real"] - outs["fp64"])))
            r["max_err_mixed_complex_vs_fp64"] = float(np.max(np.abs(outs["mixed_complex"] - outs["fp64"])))
            rows.append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
    line = {"metric": "images/s, paper ansatz 7x7 batch 1024 at chi = 2^L (circuit + Pauli cache), real vs complex kernels",
            "value": rows[3]["images_per_s_mixed_real"], "unit": "images/s", "n_gpus": 1,
            "config": {"workload": "7x7 garment-like images, paper ansatz (H, R_Y(2 pi x - pi), staggered CNOTs), "
                                   "L = 1..4, chi = 2^L; pair sets H+V (84) and H+V+diagonals (156)", "images": B},
            "table": rows}
    print(json.dumps(line), flush=True)


def run_uneven(args):
    """512 images with p ~ U{4..16}, chi = 16, L in {1, 2}: the batched pipeline (persistent,
    cost-ordered circuit kernel; autotuned launch shape) replayed as one CUDA graph, vs a
    per-image launch loop."""
    torch = _setup_torch()
    from paper_2607_10280_b300 import api, autotune, synth
    B = 512
    sizes = synth.uneven_sizes(B)
    X = synth.uneven_pixels(sizes)
    chi = 16
    out_rows = []
    for Lr in (1, 2):
        params = torch.tensor(synth.circuit_params(Lr, 256), dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            b = api.Batch(sizes, chi, "mixed", s)
            px = torch.tensor(np.concatenate(X), dtype=torch.float64, device="cuda")
            pauli = torch.empty((int(b.pair_offsets[-1]), 16), dtype=torch.float32, device="cuda")

            def step():
                b.apply_circuit(px, Lr, "ladder", params)
                b.pauli_cache(pauli)
            shape = autotune.tune(b, step, autotune.signature(b, Lr), use_cache=False)
            step()
            s.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                step()
            g.replay()
            s.synchronize()
            ms_graph = _time_events(torch, g.replay, 20, s)
            # per-image launch loop: one batch per image, launched one after another
            singles = [api.Batch(np.array([p], np.int32), chi, "mixed", s) for p in sizes]
            pxs = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in X]
            outs = [torch.empty((api.pair_count(int(p)), 16), dtype=torch.float32, device="cuda") for p in sizes]

            def loop():
                for i in range(B):
                    singles[i].apply_circuit(pxs[i], Lr, "ladder", params)
                    singles[i].pauli_cache(outs[i])
            loop()
            s.synchronize()
            ms_loop = _time_events(torch, loop, 2, s)
            got = pauli.cpu().numpy()
            same = all(np.array_equal(got[b.pair_offsets[i]:b.pair_offsets[i + 1]], outs[i].cpu().numpy())
                       for i in range(0, B, 37))
            qubit_layers = float(np.sum(sizes.astype(np.int64) ** 2) * Lr)
            out_rows.append({"L": Lr, "graph_images_per_s": B / (ms_graph / 1e3),
                             "loop_images_per_s": B / (ms_loop / 1e3),
                             "graph_qubit_layers_per_s": qubit_layers / (ms_graph / 1e3),
                             "speedup": ms_loop / ms_graph, "launch_shape": {k: shape[k] for k in (
                                 "images_per_cta", "circuit_threads", "pauli_threads")},
                             "graph_equals_loop_on_sampled_images": bool(same)})
            for x in singles:
                x.close()
            b.close()
    line = {"metric": "images/s, 512 uneven images p~U{4..16} chi=16, graph-replayed batch vs per-image loop",
            "value": out_rows[-1]["graph_images_per_s"], "unit": "images/s", "n_gpus": 1,
            "config": {"workload": "uneven sizes p ~ U{4..16} (16-256 qubits), ladder, chi=16, L in {1,2}",
                       "images": B}, "table": out_rows}
    print(json.dumps(line), flush=True)


def run_large(args):
    """16x16 images (256 qubits), 256 per batch, L in {1,2}, chi in {16,32}, mixed vs FP64,
    then ANO (480 pairs x 16 N(0,1) coefficients) and a linear layer 480 -> 4096 (64x64)."""
    torch = _setup_torch()
    from oracle import pipeline as opipe
    from paper_2607_10280_b300 import api, synth
    p, B = 16, 256
    m = api.pair_count(p)
    X = synth.garment_pixels(B, p)
    abd = torch.tensor(synth.observable_params(m), dtype=torch.float32, device="cuda")
    W = torch.tensor(np.random.default_rng(3).standard_normal((4096, m)) / np.sqrt(m), dtype=torch.float32,
                     device="cuda")
    bias = torch.zeros(4096, dtype=torch.float32, device="cuda")
    rows = []
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    for Lr in (1, 2):
        params_np = synth.circuit_params(Lr, p * p)
        params = torch.tensor(params_np, dtype=torch.float64, device="cuda")
        ref = opipe.pauli_cache(X[0], p, Lr, 64, "ladder", params_np)
        for chi in (16, 32):
            r = {"L": Lr, "chi": chi}
            for prec in ("mixed", "fp64"):
                b = api.Batch(np.full(B, p, np.int32), chi, prec)
                pauli = torch.empty((B * m, 16), dtype=torch.float64 if prec == "fp64" else torch.float32,
                                    device="cuda")

                def step():
                    b.apply_circuit(px, Lr, "ladder", params)
                    b.pauli_cache(pauli)
                    return api.ano_features(pauli, m, abd, W, bias)
                step()
                torch.cuda.synchronize()
                ms = _time_events(torch, step, 5 if prec == "mixed" else 2)
                r[f"images_per_s_{prec}"] = B / (ms / 1e3)
                r[f"max_err_{prec}_vs_exact_image0"] = float(np.max(np.abs(
                    pauli[:m].double().cpu().numpy() - ref)))
                b.close()
            rows.append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
    line = {"metric": "images/s, 16x16 (256 qubits) batch 256 + ANO 480x16 + linear 480->4096",
            "value": rows[0]["images_per_s_mixed"], "unit": "images/s", "n_gpus": 1,
            "config": {"workload": "16x16 garment-like, ladder ansatz, L in {1,2}, chi in {16,32}", "images": B},
            "table": rows}
    print(json.dumps(line), flush=True)


def _oracle_serve_job(job):
    """One sampled serving request through the CPU oracle (spawn-pool worker)."""
    from oracle import pipeline as opipe
    idx, x, p, L, chi, params_np = job
    ref, st = opipe.pauli_cache(x, p, L, chi, "ladder", params_np, return_state=True)
    return idx, ref, st.min_gap


def run_serve(args):
    """Poisson arrivals at 2000 requests/s of single images with p in 6..16, L in 1..4,
    chi in {4,8,16,32}; p = 7 requests also get ANO (84 x 16) and a linear layer 84 -> 784.
    Six slots (--serve-slots), four of them (--serve-long-slots) reserved for requests whose
    circuit truncates (they run a complex128 chain, on 128-thread teams).  Latency per (L, chi), per p and per lane, device time per wave;
    every result against the batched FP64 path afterwards, and a stratified sample (one
    request of every (p, L, chi) class that occurred, and more of the truncating and the
    16x16 ones) against the CPU oracle."""
    # a serving process loads every kernel when CUDA starts: a kernel loaded lazily at its
    # first launch stalls the launching thread until the device's running work allows it
    os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")
    # every slot's stream on a hardware queue of its own: with the default of 8 queues
    # streams share them, and an event on a short-lane slot's idle stream then waited
    # behind a long-lane chain on the same queue (up to 75 ms, measured with 6 slots)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    torch = _setup_torch()
    from paper_2607_10280_b300 import api, synth
    from paper_2607_10280_b300.flops import lossy
    from paper_2607_10280_b300.serving import Request, Server, latency_by, latency_report
    reqs = synth.serving_requests(args.requests)
    params_np = synth.circuit_params(4, 256)
    params = torch.tensor(params_np, dtype=torch.float64, device="cuda")
    m7 = api.pair_count(7)
    W, b = synth.linear_params(784, m7)
    epi = {7: (torch.tensor(synth.observable_params(m7), dtype=torch.float32, device="cuda"),
               torch.tensor(W, dtype=torch.float32, device="cuda"), torch.tensor(b, dtype=torch.float32,
                                                                                device="cuda"))}
    srv = Server(params, epi, slots=args.serve_slots, max_images_per_wave=64, budget_bytes=4 << 30,
                 long_slots=args.serve_long_slots)
    # warm the slots (kernel attributes, first launches)
    warm = [srv.submit(Request(r["p"], r["L"], r["chi"], r["pixels"])) for r in reqs[:64]]
    srv.start()
    for w in warm:
        w.event.wait()
    srv.stop()
    srv.completed.clear()
    srv.wave_log.clear()
    srv.waves = 0
    # Python's collector pauses every thread, the scheduler's included: record each pause
    import gc
    gc_pauses = []
    gc_t = {}

    def _gc_cb(phase, info):
        if phase == "start":
            gc_t["t"] = time.perf_counter()
        elif "t" in gc_t:
            t_end = time.perf_counter()
            gc_pauses.append((info.get("generation", -1), (t_end - gc_t.pop("t")) * 1e3, t_end))
    gc.callbacks.append(_gc_cb)
    srv.start()
    t0 = time.perf_counter()
    submitted = []
    for r in reqs:
        delay = r["t"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        submitted.append(srv.submit(Request(r["p"], r["L"], r["chi"], r["pixels"])))
    for q in submitted:
        q.event.wait()
    t1 = max(q.t_done for q in submitted)
    srv.stop()
    gc.callbacks.remove(_gc_cb)
    rep = latency_report(submitted)
    waves = np.array([w[3] for w in srv.wave_log])
    lanes = {}
    for name, flag in (("short", False), ("long", True)):
        ws = np.array([w[3] for w in srv.wave_log if w[2] == flag])
        sz = np.array([w[1] for w in srv.wave_log if w[2] == flag])
        hs = np.array([w[4] for w in srv.wave_log if w[2] == flag])
        if len(ws):
            lanes[name] = {"waves": int(len(ws)), "device_ms_p50": float(np.percentile(ws, 50)),
                           "device_ms_p99": float(np.percentile(ws, 99)), "device_ms_max": float(ws.max()),
                           "host_launch_ms_p50": float(np.percentile(hs, 50)),
                           "host_launch_ms_p99": float(np.percentile(hs, 99)), "host_launch_ms_max": float(hs.max()),
                           "host_phase_ms_max": dict(zip(("reshape", "pixels", "circuit", "pauli", "epilogue"),
                                                         np.max([w[5] for w in srv.wave_log if w[2] == flag],
                                                                axis=0).round(2).tolist())),
                           "images_per_wave_mean": float(sz.mean())}
    # latency = queueing (arrival -> wave launch) + service (launch -> result on the host)
    split = {}
    for name in ("short", "long"):
        rs = [q for q in submitted if q.lane == name]
        if rs:
            qw = np.array([q.t_launch - q.t_submit for q in rs]) * 1e3
            sv = np.array([q.t_done - q.t_launch for q in rs]) * 1e3
            split[name] = {"queue_ms_p50": float(np.percentile(qw, 50)), "queue_ms_p99": float(np.percentile(qw, 99)),
                           "service_ms_p50": float(np.percentile(sv, 50)),
                           "service_ms_p99": float(np.percentile(sv, 99))}
    # pauses while requests were in flight (t0 .. t1; start() itself runs one full
    # collection before t0) and after
    run_p = [g for g in gc_pauses if t0 <= g[2] <= t1]
    gcp = np.array([g[1] for g in run_p]) if run_p else np.zeros(1)

    # every result against the batched FP64 path, by (p, L, chi) group
    groups = {}
    for i, r in enumerate(reqs):
        groups.setdefault((r["p"], r["L"], r["chi"]), []).append(i)
    err = np.zeros(len(reqs))
    for (p, Lr, chi), idx in groups.items():
        bt = api.Batch(np.full(len(idx), p, np.int32), chi, "fp64")
        px = torch.tensor(np.concatenate([reqs[i]["pixels"] for i in idx]), dtype=torch.float64, device="cuda")
        bt.apply_circuit(px, Lr, "ladder", params)
        ref = bt.pauli_cache().cpu().numpy().reshape(len(idx), -1, 16)
        bt.close()
        for k, i in enumerate(idx):
            err[i] = float(np.max(np.abs(submitted[i].pauli - ref[k])))

    # stratified oracle sample: one per (p, L, chi) class, then more truncating and 16x16
    rng = np.random.default_rng(5)
    sample = [int(rng.choice(idx)) for idx in groups.values()]
    extra = [i for i, r in enumerate(reqs) if lossy(r["p"], r["L"], r["chi"]) or r["p"] == 16]
    rng.shuffle(extra)
    for i in extra:
        if len(sample) >= max(200, len(groups) + 40):
            break
        if i not in sample:
            sample.append(i)
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    jobs = [(i, reqs[i]["pixels"], reqs[i]["p"], reqs[i]["L"], reqs[i]["chi"], params_np) for i in sample]
    with mp.get_context("spawn").Pool(min(cpu_cores(), 32)) as pool:
        outs = pool.map(_oracle_serve_job, jobs, chunksize=1)
    oerr, ties = [], 0
    for i, ref, gap in outs:
        if gap < 1e-6:
            ties += 1          # near-tie at a truncation cut: no unique answer
            continue
        oerr.append(float(np.max(np.abs(submitted[i].pauli - ref))))
    by_lc = latency_by(submitted, lambda r: f"L{r.L}_chi{r.chi}")
    by_p = latency_by(submitted, lambda r: f"p{r.p}")
    by_lane = latency_by(submitted, lambda r: "long" if lossy(r.p, r.L, r.chi) else "short")
    line = {"metric": "serving: images/s and p50/p99 latency, Poisson 2000 req/s, mixed p/L/chi",
            "value": len(submitted) / (t1 - t0), "unit": "images/s", "n_gpus": 1,
            "latency": rep, "latency_by_lane": by_lane, "latency_by_L_chi": by_lc, "latency_by_p": by_p,
            "arrival_rate_hz": 2000.0, "waves": srv.waves, "max_wave": srv.max_wave,
            "device_ms_per_wave": {"p50": float(np.percentile(waves, 50)), "p99": float(np.percentile(waves, 99)),
                                   "max": float(waves.max()), "lanes": lanes},
            "latency_split_by_lane": split,
            "gc_pauses": {"count": len(run_p), "max_ms": float(gcp.max()), "total_ms": float(gcp.sum()),
                          "gen2": sum(1 for g in run_p if g[0] == 2),
                          "after_last_result": [round(g[1], 2) for g in gc_pauses if g[2] > t1]},
            "max_inflight_bytes": srv.max_inflight_bytes, "budget_bytes": srv.budget,
            "check_all_vs_fp64_gpu": {"requests": len(reqs), "max_abs": float(err.max()),
                                      "over_1e-5": int((err > 1e-5).sum())},
            "check_sample_vs_oracle": {"requests": len(sample), "classes": len(groups),
                                       "max_abs": max(oerr) if oerr else None, "over_1e-5": int(sum(e > 1e-5 for e in oerr)),
                                       "skipped_ties": ties},
            "config": {"workload": "single images p~U{6..16}, L~U{1..4}, chi~U{4,8,16,32}, p=7 with ANO + "
                                   "linear 84->784", "requests": len(submitted), "slots": len(srv.slots),
                       "long_slots": srv.long_slots}}
    print(json.dumps(line), flush=True)
    assert err.max() <= 1e-5 and (not oerr or max(oerr) <= 1e-5), "serving results exceed 1e-5"


def run_train(args):
    """Training on cached Paulis (Sec. II.C-D): the Pauli cache of 1024 7x7 images
    (L = 4, chi = 16) is computed once; then full-batch steps of the MSE term of Eq. 7
    with two Adam optimizers train (A, B, D) and the linear layer 84 -> 784 towards
    synthetic 28 x 28 targets.  Reports training steps/s, the step time against one
    recomputation of the cache, and the loss curve."""
    torch = _setup_torch()
    from paper_2607_10280_b300 import api, synth
    p, B, L, chi, O = 7, 1024, 4, 16, 784
    m = api.pair_count(p)
    X = synth.garment_pixels(B, p)
    Y = torch.tensor(synth.garment_pixels(B, 28, seed=5), dtype=torch.float32, device="cuda")
    params = torch.tensor(synth.circuit_params(L, p * p), dtype=torch.float64, device="cuda")
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    b = api.Batch(np.full(B, p, np.int32), chi, "mixed")
    pauli = torch.empty((B * m, 16), dtype=torch.float32, device="cuda")

    def cache():
        b.apply_circuit(px, L, "ladder", params)
        b.pauli_cache(pauli)
    cache()
    torch.cuda.synchronize()
    cache_ms = _time_events(torch, cache, 5)
    abd = torch.tensor(synth.observable_params(m), dtype=torch.float32, device="cuda")
    Wn, bn = synth.linear_params(O, m)
    W = torch.tensor(Wn, dtype=torch.float32, device="cuda")
    bias = torch.tensor(bn, dtype=torch.float32, device="cuda")
    tr = api.Trainer(pauli, m, abd, W, bias, lr_abd=1e-2, lr_linear=1e-3)
    first = tr.step(Y).item()
    steps = max(10, args.steps)
    losses = []
    step_ms = _time_events(torch, lambda: losses.append(tr.step(Y)), steps)
    losses = [first] + [x.item() for x in losses]
    line = {"metric": "training steps/s on cached Paulis, 1024 7x7 images, ANO 84x16 + linear 84->784, "
                      "MSE + two Adam optimizers",
            "value": 1e3 / step_ms, "unit": "steps/s", "n_gpus": 1, "higher_is_better": True,
            "images_per_s": B * 1e3 / step_ms, "ms_per_step": step_ms,
            "pauli_cache_ms": cache_ms, "cache_over_step": cache_ms / step_ms,
            "loss_first": losses[0], "loss_last": losses[-1], "steps_timed": steps,
            "config": {"workload": "7x7 garment-like images, ladder L=4 chi=16 Pauli cache (once); "
                                   "targets 28x28 garment-like (synthetic)", "images": B, "pairs": m,
                       "out_dim": O}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    PAULI_KERNEL = a.pauli_kernel
    if a.impl == "reference":
        run_reference(a)
    elif a.config == "headline":
        run_ours(a)
    else:
        {"sweep": run_sweep, "trunc": run_trunc, "large_chi": run_large_chi, "paper": run_paper, "uneven": run_uneven, "large": run_large, "serve": run_serve,
         "train": run_train, "diag": run_diag}[a.config](a)
