#!/usr/bin/env python
"""Throughput of the 1 mm MPM JTV-MAP fit on GB300, in Mvoxel.GN-iter/s.

Workload: a 176 x 240 x 256 volume at 1 mm, PDw / T1w / MTw SPGR contrasts
(6 / 21 / 6 degrees, TR 25 ms, 8 / 8 / 6 echoes 2.3 ms apart) of a seeded
piecewise-smooth phantom with smooth B1+ / B1- fields and Rician noise at
first-echo SNR 20, float32 throughout, JTV lambda = 10; one step is one whole
mpm_fit call: constant initial maps, 20 Newton updates with 30 PCG iterations
each, and the posterior variance at the final maps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank fits its own subject
(independent replicas, weak scaling); the step time is the maximum over ranks.
``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
slab of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mvoxel·GN-iter/s, 1mm MPM JTV fit"
UNIT = "Mvoxel·GN-iter/s"
SHAPE = (176, 240, 256)
VX = (1.0, 1.0, 1.0)
GN_ITERS = 20
CG_ITERS = 30
LAMBDA = 10.0
EPS = 1e-3
SNR = 20.0
L2_BYTES = 129 * 2 ** 20
CPU_SAMPLE_Z = 32        # cpu_baseline: a 176 x 240 x 32 slab, one update
REF_SAMPLE_Z = 32        # reference arm: a 176 x 240 x 32 slab per step, one update
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shape", default=None,
                    help="override the volume (nx,ny,nz) for profiling runs on a smaller case")
    ap.add_argument("--echo-dtype", choices=["f32", "bf16"], default="f32",
                    help="storage of the echo images (computation stays float32)")
    ap.add_argument("--config", choices=["1mm", "0.8mm"], default="1mm",
                    help="1mm: 176x240x256 at 1 mm; 0.8mm: 208x300x320 at 0.8 mm")
    ap.add_argument("--write-traffic", nargs="+", metavar="CSV", default=None,
                    help="write profiles/dram_traffic.json from the per-kernel ncu captures "
                         "of TRAFFIC_COMMANDS; runs no GPU work")
    ap.add_argument("--print-hashes", action="store_true",
                    help="print the source hash of every kernel kind (stderr) before running")
    ap.add_argument("--launch-table", metavar="CSV", default=None,
                    help="print the per-kernel launch table of an ncu --csv capture; runs no GPU work")
    ap.add_argument("--workload", choices=["plain", "batched", "served", "moved"], default="plain",
                    help="plain: one subject per fit; batched: 16 uneven subjects per "
                         "mpm_fit_batch call, compared with plain fits of the same subjects; "
                         "served: Poisson arrivals through mpm_server_* vs FIFO plain fits")
    ap.add_argument("--solver", choices=["pcg", "mg"], default="pcg",
                    help="mg: time to |r| <= 1e-3 |r_0| of the fit's Newton systems, block-Jacobi "
                         "PCG against multigrid-preconditioned CG (instead of the fit)")
    ap.add_argument("--batch-mix", choices=["uneven", "small"], default="uneven",
                    help="batched: 16 subjects of uneven sizes (64^3 .. 176x240x256), or 16 x 64^3")
    ap.add_argument("--requests", type=int, default=24, help="served: number of requests")
    ap.add_argument("--rate", type=float, default=3.0, help="served: arrivals per second")
    args = ap.parse_args(argv)
    global SHAPE, VX
    if args.config == "0.8mm":
        SHAPE, VX = (208, 300, 320), (0.8, 0.8, 0.8)
    if args.shape:
        SHAPE = tuple(int(v) for v in args.shape.split(","))
        assert len(SHAPE) == 3
    return args


# ------------------------------------------------------------ distributed

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(seconds: float, units: float, world: int, backend_device=None):
    """Whole-job value over replicas: total units / max seconds over ranks."""
    if world <= 1:
        return units / seconds, seconds
    import torch
    import torch.distributed as dist
    dev = backend_device if backend_device is not None else torch.device("cpu")
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return u.item() / t.item(), t.item()


# --------------------------------------------------------------- inputs

def workload_inputs(seed: int, device, echo_dtype: str = "f32"):
    """Phantom maps and B1 fields on the host, noise-free images from the
    library's own forward model on the GPU, Rician noise drawn on the GPU."""
    import torch

    import paper_2102_01604_gb300 as mpm
    from paper_2102_01604_gb300 import phantom

    prot = phantom.protocol()
    ph = phantom.phantom(SHAPE, seed=seed)
    y_true = torch.from_numpy(ph["y"].astype(np.float32)).to(device)
    b1p = torch.from_numpy(ph["b1p"].astype(np.float32)).to(device)
    b1m = torch.from_numpy(ph["b1m"].astype(np.float32)).to(device)
    p0 = mpm.make_problem(prot, SHAPE)
    s = mpm.mpm_forward(p0, y_true, b1p, b1m)
    sig2, i = [], 0
    for ne in prot["n_echoes"]:
        m = s[i].double().mean().item() / SNR
        sig2.append(m * m)
        i += ne
    prot["sigma2"] = sig2
    x = phantom.rician_torch(s, prot, seed + 1)
    del s
    if echo_dtype == "bf16":
        x = x.to(torch.bfloat16)
    torch.cuda.synchronize()
    return prot, ph, x, b1p, b1m


# ------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ roofline

def step_bytes(j: int, K: int, cg_iters: int = None) -> int:
    """Bytes PCG iteration j moves per voxel (pcg_step.cuh): j = 0 reads z_0, w,
    H and writes p_0, v_0; later iterations read z, v, p, w, H and write z, v,
    p; even j >= 2 also read p_{j-2} and write x, and read x when j > 2."""
    T = K * (K + 1) // 2
    f = 4
    if j == 0:
        return K * f + f + T * f + 2 * K * f
    b = 3 * K * f + f + T * f + 3 * K * f
    if j >= 2 and j % 2 == 0:
        b += 2 * K * f + (K * f if j > 2 else 0)
    return b


def algorithmic_bytes(K: int, C: int, I: int, echo_bytes: int = 4, cg_iters: int = None):
    """Bytes each kernel must move per voxel (reads + writes of its operands,
    float32, every array touched once).  pcg_step_per_solve sums step_bytes
    over the iterations of one solve; pcg_step is its mean per launch."""
    cg = cg_iters or CG_ITERS
    T = K * (K + 1) // 2
    f = 4
    per_solve = sum(step_bytes(j, K) for j in range(cg))
    xcount = max((j for j in range(2, cg, 2)), default=0)
    pend = cg - xcount                                  # directions folded by the final pass
    final = (K * f if xcount else 0) + pend * K * f + 2 * K * f
    return {
        "grad_hess": I * echo_bytes + K * f + f + C * f + K * f + T * f,
        "jtv": K * f + f,
        "pcg_init": f + 2 * K * f + T * f + K * f,
        "pcg_step_per_solve": per_solve,
        "pcg_step": per_solve / cg,
        "pcg_final": final,
        "uncertainty": T * f + f + K * f,
    }


def kernel_roofline(prof: dict, n_vox: int, steps: int, K: int, C: int, I: int, peak_gbs: float,
                    echo_bytes: int = 4):
    ab = algorithmic_bytes(K, C, I, echo_bytes)
    solves = steps * GN_ITERS
    per_kernel = {}
    for kind, v in prof.items():
        if not v["launches"]:
            continue
        if kind == "pcg_step" and v["launches"] % CG_ITERS == 0:
            total_bytes = ab["pcg_step_per_solve"] * n_vox * (v["launches"] // CG_ITERS)
        elif kind in ab:
            total_bytes = ab[kind] * n_vox * v["launches"]
        else:
            total_bytes = None
        entry = {"ms_total": round(v["ms"], 3), "launches": v["launches"],
                 "us_per_launch": round(1000.0 * v["ms"] / v["launches"], 2)}
        if total_bytes is not None and v["ms"] > 0:
            gbs = total_bytes / (v["ms"] * 1e-3) / 1e9
            entry["bytes_per_launch"] = int(total_bytes / v["launches"])
            entry["achieved_gbs"] = round(gbs, 1)
            entry["frac_of_measured_hbm"] = round(gbs / peak_gbs, 4)
        per_kernel[kind] = entry
    return per_kernel


def measured_peak():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Source files that define each kernel kind (besides device_common.cuh,
# which every kernel includes).
KIND_SOURCES = {
    "grad_hess": ["voxel_kernels.cu", "voxel_tma.cu", "voxel_model.cuh", "tma_common.cuh"],
    "uncertainty": ["voxel_kernels.cu"],
    "jtv": ["stencil_kernels.cu"],
    "pcg_init": ["stencil_kernels.cu", "pcg_step.cuh"],
    "pcg_step": ["stencil_kernels.cu", "stencil_tma.cu", "pcg_step.cuh", "tma_common.cuh"],
    "pcg_final": ["stencil_kernels.cu", "pcg_step.cuh"],
    "grad_hess_proj": ["projection.cu", "voxel_model.cuh"],
    "reslice": ["projection.cu"],
}


def kernel_source_hash(kind: str):
    """Hash of the sources of one kernel kind, or None for an unknown kind."""
    if kind not in KIND_SOURCES:
        return None
    h = hashlib.sha256()
    for name in ["device_common.cuh"] + KIND_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2102_01604_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kind: str, n_vox: int):
    """DRAM bytes per launch from the committed ncu capture of this kernel kind
    (on a smaller volume), scaled to n_vox voxels; None when the kernel's
    sources changed since the capture."""
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
    except (OSError, ValueError):
        return None
    k = tr.get("kernels", {}).get(kind)
    if not k or k.get("source_hash") != kernel_source_hash(kind):
        return None
    return int(k["dram_bytes_per_voxel"] * n_vox)


# Kernel kind of each kernel function (the name before its template arguments).
KERNEL_KIND = {
    "k_pcg_step_tma": "pcg_step", "k_pcg_step": "pcg_step", "k_pcg_init": "pcg_init",
    "k_jtv": "jtv", "k_pcg_final": "pcg_final", "k_grad_hess": "grad_hess",
    "k_grad_hess_tma": "grad_hess", "k_uncertainty": "uncertainty",
    "k_grad_hess_proj": "grad_hess_proj", "k_push_all": "reslice",
    # the phase-batched forms (mpm_fit_batch with opts.graph = 2)
    "k_pcg_step_tma_batch": "pcg_step", "k_pcg_init_batch": "pcg_init", "k_jtv_batch": "jtv",
    "k_pcg_final_batch": "pcg_final", "k_grad_hess_batch": "grad_hess",
    "k_grad_hess_tma_batch": "grad_hess", "k_uncertainty_batch": "uncertainty",
}


def read_ncu_csv(path: str):
    """Launches of an `ncu --csv` metrics log in launch order: for each, the
    kernel function name and its metric values."""
    import csv
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    launches = {}
    for r in csv.DictReader(lines):
        d = launches.setdefault(int(r["ID"]), {"name": r["Kernel Name"], "metrics": {}})
        d["metrics"][r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
    out = []
    for i in sorted(launches):
        name = launches[i]["name"]
        name = name[5:] if name.startswith("void ") else name
        name = name.replace("<unnamed>", "unnamed").split("(")[0].split("<")[0].strip()
        out.append((name.split("::")[-1], launches[i]["metrics"]))
    return out


def read_log_json(path: str, key: str):
    """The first JSON object with `key` that the program printed into an ncu
    log (None if there is none)."""
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("{") and key in line:
                try:
                    d = json.loads(line)
                except ValueError:
                    continue
                if key in d:
                    return d
    return None


def launch_table(launches) -> str:
    """Per kernel function: launches, total ncu time, share of the total and
    DRAM bytes per launch, largest total first."""
    agg = {}
    for name, m in launches:
        a = agg.setdefault(name, [0, 0.0, 0.0])
        a[0] += 1
        a[1] += m.get("gpu__time_duration.sum", 0.0)
        a[2] += m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
    total = sum(a[1] for a in agg.values()) or 1.0
    rows = [f"{len(launches)} launches, {total / 1e6:.1f} ms"]
    for name, (n, t, b) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        rows.append(f"{name:24s} {n:5d} {t / 1e6:9.2f} ms {100 * t / total:5.1f}% "
                    f"{b / n / 1e6:9.1f} MB/launch")
    return "\n".join(rows)


# DRAM traffic captures: one ncu run per kernel kind, on a 176 x 240 x 128
# volume (images 476 MB and every solver vector 86 MB, so the operands do not
# fit the 129 MB L2), one kernel (-k), the launches after -s of it only.  The
# metrics (DRAM bytes read and written, duration) take one pass.  Each run
# writes ncu's CSV and the bench's own output (its voxel count and the source
# hash of every kernel kind) into one file, which --write-traffic reads.
TRAFFIC_SHAPE = (176, 240, 128)
TRAFFIC_CAPTURES = {
    # kind: (kernel name regex, launches skipped, launches captured, workload)
    "pcg_step": ("k_pcg_step", 48, 30, "plain"),     # after the autotuner's 18 and one solve
    "pcg_init": ("k_pcg_init", 1, 2, "plain"),
    "pcg_final": ("k_pcg_final", 1, 2, "plain"),
    "jtv": ("k_jtv", 1, 2, "plain"),
    "grad_hess": ("k_grad_hess", 1, 2, "plain"),
    "uncertainty": ("k_uncertainty", 0, 1, "plain"),
    "grad_hess_proj": ("k_grad_hess_proj", 3, 3, "moved"),
    "reslice": ("k_push_all", 1, 2, "moved"),
}


def traffic_command(kind: str) -> str:
    rx, skip, count, workload = TRAFFIC_CAPTURES[kind]
    shape = ",".join(str(v) for v in TRAFFIC_SHAPE)
    return (f"ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
            f"--clock-control none -k regex:{rx} -s {skip} -c {count} --csv "
            f"python bench.py --workload {workload} --shape {shape} --steps 1 --warmup 0 "
            f"--no-cpu-baseline --no-e2e --print-hashes > traffic_{kind}.csv 2>&1")


TRAFFIC_COMMANDS = [traffic_command(k) for k in TRAFFIC_CAPTURES] + [
    "python bench.py --write-traffic " + " ".join(f"traffic_{k}.csv" for k in TRAFFIC_CAPTURES)]


def write_traffic(paths, out: str = TRAFFIC_FILE, commands=()):
    """Per kernel kind, the mean DRAM bytes per launch and per voxel
    (`dram__bytes_read.sum + dram__bytes_write.sum` of the captured launches,
    divided by the capture's voxel count) into `out`, with the source hash of
    the kind that the captured program printed; kinds of `out` that these
    logs do not cover are kept.  Refuses (ValueError) when a
    log lacks the program's hashes or voxel count, or when a captured kind's
    sources have changed since the capture."""
    doc = {"workload": f"{'x'.join(str(v) for v in TRAFFIC_SHAPE)} volume, one capture per "
                       "kernel kind; per-voxel bytes are scaled to other volumes by the voxel count",
           "capture": list(commands),
           "per_voxel_of": "reconstruction voxels (k_grad_hess_proj: acquisition voxels of one "
                           "contrast, here the same count)",
           "kernels": {}}
    try:
        with open(out) as f:
            old = json.load(f).get("kernels", {})
    except (OSError, ValueError):
        old = {}
    # kinds not recaptured keep their entry (their source hash still guards them)
    doc["kernels"].update({k: v for k, v in old.items() if "voxels" in v})
    for path in paths:
        hashes = read_log_json(path, "kernel_source_hashes")
        line = read_log_json(path, "config")
        if not hashes or not line or "voxels" not in line["config"]:
            raise ValueError(f"{path}: no source hashes or voxel count from the captured program")
        n_vox = int(line["config"]["voxels"])
        agg = {}
        for name, m in read_ncu_csv(path):
            kind = KERNEL_KIND.get(name)
            if kind is None:
                continue
            a = agg.setdefault(kind, [0, 0.0])
            a[0] += 1
            a[1] += m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        for kind, (n, b) in agg.items():
            captured = hashes["kernel_source_hashes"].get(kind)
            if captured != kernel_source_hash(kind):
                raise ValueError(f"{path}: {kind} was captured from sources {captured}, "
                                 f"now {kernel_source_hash(kind)}")
            doc["kernels"][kind] = {"launches": n, "voxels": n_vox,
                                    "dram_bytes_per_launch": int(b / n),
                                    "dram_bytes_per_voxel": round(b / n / n_vox, 3),
                                    "source_hash": captured}
    doc["kernels"] = dict(sorted(doc["kernels"].items()))
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    return doc


def print_source_hashes():
    """One JSON line on stderr naming the source hash of every kernel kind
    (read back from ncu logs by --write-traffic)."""
    print(json.dumps({"kernel_source_hashes": {k: kernel_source_hash(k) for k in KIND_SOURCES}}),
          file=sys.stderr, flush=True)


# ---------------------------------------------------------- CPU oracle

def oracle_sample(z_planes: int, seed: int):
    """The oracle's inputs for a 176 x 240 x z slab of the bench phantom."""
    import oracle as orc
    from paper_2102_01604_gb300 import phantom

    shape = (SHAPE[0], SHAPE[1], z_planes)
    ph = phantom.phantom(SHAPE, seed=seed)
    n = shape[0] * shape[1] * shape[2]
    y, b1p, b1m = ph["y"][:, :n], ph["b1p"][:n], ph["b1m"][:, :n]
    prot = phantom.protocol()
    s = orc.forward(orc.make_problem(prot, shape), y, b1p, b1m)
    prot["sigma2"] = phantom.noise_sigma2(s, prot, SNR)
    x = phantom.rician(s, prot, seed + 1).astype(np.float32)
    return orc.make_problem(prot, shape, lam=LAMBDA, eps=EPS), shape, x, b1p, b1m


def time_oracle(z_planes: int, seed: int, reps: int = 1, threads: int = 1):
    """Seconds of one oracle update (30 PCG, objective at both ends) on a
    176 x 240 x z slab, on `threads` host threads (0: all cores; the threaded
    build rounds exactly like the serial one).  Returns (voxels, times, threads)."""
    import oracle as orc
    p, shape, x, b1p, b1m = oracle_sample(z_planes, seed)
    n = shape[0] * shape[1] * shape[2]
    used = orc.use_threads(threads)
    times = []
    try:
        for _ in range(reps):
            t0 = time.perf_counter()
            r = orc.fit(p, x, None, b1p, b1m, gn_iters=1, cg_iters=CG_ITERS)
            times.append(time.perf_counter() - t0)
            assert r["iters"] == 1
    finally:
        orc.use_threads(1)
    return n, times, used


def time_small_fit():
    """Seconds of the oracle's whole fit of the small configuration (32 x 32 x
    16 voxels, 10 updates x 30 PCG), single-threaded."""
    import oracle as orc
    from paper_2102_01604_gb300 import phantom
    shape = (32, 32, 16)
    ph = phantom.phantom(shape, seed=0, with_b1m=False)
    prot = phantom.protocol()
    s = orc.forward(orc.make_problem(prot, shape), ph["y"], ph["b1p"], None)
    prot["sigma2"] = phantom.noise_sigma2(s, prot, SNR)
    x = phantom.rician(s, prot, 1).astype(np.float32)
    p = orc.make_problem(prot, shape, lam=LAMBDA, eps=EPS)
    t0 = time.perf_counter()
    r = orc.fit(p, x, None, ph["b1p"], None, gn_iters=10, cg_iters=CG_ITERS)
    t = time.perf_counter() - t0
    assert r["iters"] == 10
    return int(np.prod(shape)), t


def cpu_baseline(seed: int):
    """The FP64 oracle on the host: all cores (the reported value) and one
    core on the same 176 x 240 x 32 slab, plus the small configuration's whole
    fit on one core."""
    n, times, used = time_oracle(CPU_SAMPLE_Z, seed, threads=0)
    t = times[0]
    n1, times1, _ = time_oracle(CPU_SAMPLE_Z, seed, threads=1)
    t1 = times1[0]
    ns, ts = time_small_fit()
    return {"value": round(n / t / 1e6, 5), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"176x240x{CPU_SAMPLE_Z} slab of the same phantom, 1 update (30 PCG) "
                      f"with objective at both ends, FP64 C on {used} OpenMP threads; {t:.2f} s; "
                      f"host has {os.cpu_count()} cores",
            "single_core": {"value": round(n1 / t1 / 1e6, 5), "cores": 1, "seconds": round(t1, 2)},
            "small_config_fit": {"value": round(ns * 10 / ts / 1e6, 5), "cores": 1,
                                 "seconds": round(ts, 3),
                                 "sample": "32x32x16, 10 updates x 30 PCG, whole fit"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        time_oracle(REF_SAMPLE_Z, args.seed, threads=0)
    total_t, total_units, used = 0.0, 0, 1
    for _ in range(args.steps):
        n, times, used = time_oracle(REF_SAMPLE_Z, args.seed, threads=0)
        total_t += times[0]
        total_units += n * 1
    value = total_units / total_t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * total_t / args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"176x240x{REF_SAMPLE_Z} slab of the 1 mm MPM JTV-MAP "
                               f"workload, 1 update x {CG_ITERS} PCG per step",
                   "runs_on": f"host CPU (FP64 oracle, {used} OpenMP threads)"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"176x240x{REF_SAMPLE_Z} slab, 1 update per step"},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- our arm

def run_ours(args):
    import torch

    import paper_2102_01604_gb300 as mpm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = args.seed + 1000 * rank

    prot, ph, x, b1p, b1m = workload_inputs(seed, dev, args.echo_dtype)
    problem = mpm.make_problem(prot, SHAPE, vx=VX, lam=LAMBDA, eps=EPS,
                               echo_dtype=1 if args.echo_dtype == "bf16" else 0)
    opts = mpm.make_opts(gn_iters=GN_ITERS, cg_iters=CG_ITERS, newton_per_irls=1, init=True)
    K, C = problem.n_maps, problem.n_contrasts
    I = sum(prot["n_echoes"])
    N = int(np.prod(SHAPE))
    y = torch.empty((K, N), dtype=torch.float32, device=dev)
    var = torch.empty((K, N), dtype=torch.float32, device=dev)
    ws = mpm.workspace(problem, opts, device=dev)

    # stencil tile shape for this volume, chosen by timing (outside the timed region)
    tile, tile_ms = mpm.mpm_autotune(problem, opts, ws=ws)

    def step():
        st, rep = mpm.mpm_fit(problem, opts, x, y, b1p, b1m, var=var, ws=ws)
        return rep

    for _ in range(args.warmup):
        rep = step()
    torch.cuda.synchronize()

    # ---- timed region: device time of K whole fits
    mpm.mpm_profile_enable(True)
    mpm.mpm_profile_read()
    launches0 = mpm.mpm_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        rep = step()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = mpm.mpm_kernel_launches() - launches0
    prof = mpm.mpm_profile_read()
    mpm.mpm_profile_enable(False)
    seconds = e0.elapsed_time(e1) / 1000.0
    units = float(N) * GN_ITERS * args.steps
    value, t_max = aggregate(seconds, units, world, dev)
    final_F = rep.F[rep.iters]

    # ---- end to end: pinned host inputs in, maps and variances out.  Every
    # step uploads its images and B1 fields and reads back its maps and
    # variances; a copy stream overlaps step i + 1's upload and step i's read
    # back with the fits (two device buffer sets, used in turn).
    e2e = None
    if not args.no_e2e:
        xh = x.cpu().pin_memory()
        bph = b1p.cpu().pin_memory()
        bmh = b1m.cpu().pin_memory()
        yh = torch.empty((K, N), dtype=torch.float32).pin_memory()
        vh = torch.empty((K, N), dtype=torch.float32).pin_memory()
        comp = torch.cuda.current_stream()
        copy_s = torch.cuda.Stream()
        sets = [{"x": torch.empty_like(x), "bp": torch.empty_like(b1p), "bm": torch.empty_like(b1m),
                 "y": torch.empty_like(y), "v": torch.empty_like(var),
                 "ready": torch.cuda.Event()} for _ in range(2)]

        def upload(b):
            with torch.cuda.stream(copy_s):
                b["x"].copy_(xh, non_blocking=True)
                b["bp"].copy_(bph, non_blocking=True)
                b["bm"].copy_(bmh, non_blocking=True)
                b["ready"].record(copy_s)

        def e2e_run(steps):
            upload(sets[0])
            for i in range(steps):
                b = sets[i % 2]
                if i + 1 < steps:
                    upload(sets[(i + 1) % 2])      # the set's previous fit has returned
                comp.wait_event(b["ready"])
                mpm.mpm_fit(problem, opts, b["x"], b["y"], b["bp"], b["bm"], var=b["v"], ws=ws)
                copy_s.wait_stream(comp)
                with torch.cuda.stream(copy_s):
                    yh.copy_(b["y"], non_blocking=True)
                    vh.copy_(b["v"], non_blocking=True)
            comp.wait_stream(copy_s)

        e2e_run(2)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(comp)
        copy_s.wait_stream(comp)
        e2e_run(args.steps)
        f1.record(comp)
        torch.cuda.synchronize()
        e2e_val, _ = aggregate(f0.elapsed_time(f1) / 1000.0, units, world, dev)
        h2d = xh.numel() * xh.element_size() + bph.numel() * 4 + bmh.numel() * 4
        d2h = 2 * K * N * 4
        e2e = {"value": round(e2e_val / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "overlap": "copy stream: step i+1 upload and step i read-back run beside the fits"}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    peak, peak_src = measured_peak()
    kern = kernel_roofline(prof, N, args.steps, K, C, I, peak,
                           echo_bytes=2 if args.echo_dtype == "bf16" else 4)
    dominant = max(kern, key=lambda k: kern[k]["ms_total"])
    dk = kern[dominant]
    traffic = measured_traffic(dominant, N)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": dk.get("achieved_gbs"),
                "peak": peak, "unit": "GB/s",
                "frac": dk.get("frac_of_measured_hbm"), "traffic": traffic,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                else "fallback 6.8 TB/s",
                "share_of_step": round(dk["ms_total"] / (1000 * seconds), 3),
                "traffic_source": "ncu DRAM bytes of the kernel at "
                                  f"{'x'.join(str(v) for v in TRAFFIC_SHAPE)} (profiles/dram_traffic.json), "
                                  "scaled by the voxel count" if traffic is not None else
                                  "no capture of the current kernel sources"}
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(args.seed)
    line = {
        "metric": METRIC, "value": round(value / 1e6, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * t_max / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{VX[0]:g} mm MPM JTV-MAP fit, {SHAPE[0]}x{SHAPE[1]}x{SHAPE[2]} "
                               "voxels, PDw/T1w/MTw 8/8/6 echoes, Rician SNR 20, 20 updates x 30 "
                               "PCG + posterior variance"
                               + (", echoes stored bf16" if args.echo_dtype == "bf16" else ""),
                   "echo_storage": args.echo_dtype,
                   "stencil_tile": ["16x16", "32x8", "32x16"][tile] if tile >= 0 else "plain kernel",
                   "tile_autotune_us": [round(1000 * t, 1) for t in tile_ms],
                   "voxels": N, "gn_iters": GN_ITERS, "cg_iters": CG_ITERS, "lambda": LAMBDA,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2 (images {x.numel() * x.element_size() / 1e6:.0f} MB, L2 129 MB); "
                         "no flush",
                   "final_objective": final_F},
        "roofline": roofline,
        "kernels": kern,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------------- solver arm

MG_OPTS = dict(mg_levels=8, mg_nu=1, mg_omega=0.7, mg_coarse_sweeps=20)
SOLVER_TOL = 1e-3        # the paper's CG tolerance (Sec. 2.7)
SOLVER_UPDATES = (0, 1, 5)


def run_solvers(args):
    """Time to |r| <= 1e-3 |r_0| of the Newton systems of the 1 mm fit (after
    0, 1 and 5 updates), block-Jacobi PCG (the paper's preconditioner) against
    the multigrid-preconditioned CG; device time of whole mpm_solve calls,
    CUDA events, after warm-up."""
    import torch

    import paper_2102_01604_gb300 as mpm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = args.seed + 1000 * rank
    prot, ph, x, b1p, b1m = workload_inputs(seed, dev, args.echo_dtype)
    problem = mpm.make_problem(prot, SHAPE, vx=VX, lam=LAMBDA, eps=EPS,
                               echo_dtype=1 if args.echo_dtype == "bf16" else 0)
    K = problem.n_maps
    N = int(np.prod(SHAPE))
    fit_opts = mpm.make_opts(gn_iters=GN_ITERS, cg_iters=CG_ITERS)
    ws = mpm.workspace(problem, fit_opts, device=dev)
    mpm.mpm_autotune(problem, fit_opts, ws=ws)
    y = torch.empty((K, N), dtype=torch.float32, device=dev)
    systems = []
    for k in SOLVER_UPDATES:
        mpm.mpm_fit(problem, mpm.make_opts(gn_iters=k, cg_iters=CG_ITERS), x, y, b1p, b1m, ws=ws)
        w, _ = mpm.mpm_jtv_weights(problem, y)
        g, h, _ = mpm.mpm_grad_hess(problem, x, y, b1p, b1m)
        systems.append((k, h, w, g, y.clone()))
    del ws
    torch.cuda.synchronize()
    max_it = 400
    delta = torch.empty((K, N), dtype=torch.float32, device=dev)
    resid = torch.empty(max_it + 1, dtype=torch.float64, device=dev)
    results = []
    for k, h, w, g, yk in systems:
        row = {"update": k}
        for name, extra in (("block_jacobi", {}), ("multigrid", MG_OPTS)):
            # the iterations the tolerance needs, then the solve capped there: a
            # solve enqueues all cg_iters iterations (those after the stop return
            # at once), so a loose cap would time empty launches
            opts = mpm.make_opts(cg_iters=max_it, tol_cg=SOLVER_TOL, **extra)
            sws = mpm.workspace(problem, opts, mpm._lib.CALL_SOLVE, device=dev)
            resid.fill_(float("nan"))
            mpm.mpm_solve(problem, opts, h, w, g, yk, delta=delta, resid=resid, ws=sws)
            need = int(np.sum(np.isfinite(resid.cpu().numpy()))) - 1
            opts = mpm.make_opts(cg_iters=max(need, 1), tol_cg=SOLVER_TOL, **extra)
            for _ in range(max(args.warmup, 1)):
                resid.fill_(float("nan"))
                mpm.mpm_solve(problem, opts, h, w, g, yk, delta=delta, resid=resid, ws=sws)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                mpm.mpm_solve(problem, opts, h, w, g, yk, delta=delta, resid=resid, ws=sws)
            e1.record()
            torch.cuda.synchronize()
            r = resid.cpu().numpy()
            iters = int(np.sum(np.isfinite(r))) - 1
            row[name] = {"iters": iters, "rel_resid": float(r[iters] / r[0]),
                         "ms": round(e0.elapsed_time(e1) / args.steps, 3)}
            del sws
        row["speedup"] = round(row["block_jacobi"]["ms"] / row["multigrid"]["ms"], 3)
        results.append(row)
    if rank == 0:
        line = {"metric": f"ms to |r| <= {SOLVER_TOL:g} |r_0| per Newton system, 1 mm MPM JTV fit",
                "value": results[0]["multigrid"]["ms"], "unit": "ms", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"Newton systems of the {VX[0]:g} mm fit "
                                       f"({SHAPE[0]}x{SHAPE[1]}x{SHAPE[2]}) after "
                                       f"{', '.join(str(k) for k in SOLVER_UPDATES)} updates",
                           "multigrid": MG_OPTS, "max_iters": max_it},
                "systems": results}
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------- batched arm

BATCH_SUBJECTS = 16


def batch_specs(seed: int, mix: str = "uneven"):
    """16 subjects: sizes between 64^3 and 176x240x256 (multiples of 4; all
    64^3 for the small mix), 2-3 contrasts (PDw, T1w[, MTw]), 4-8 echoes per
    contrast, seeded."""
    rng = np.random.default_rng(seed + 4242)
    specs = []
    for i in range(BATCH_SUBJECTS):
        t = rng.uniform(0.0, 1.0) if mix == "uneven" else 0.0
        dims = tuple(int(round((64 + t * (m - 64)) / 4)) * 4 for m in (176, 240, 256))
        nc = int(rng.integers(2, 4))
        contrasts = ("PDw", "T1w", "MTw")[:nc]
        echoes = tuple(int(v) for v in rng.integers(4, 9, size=nc))
        specs.append((dims, contrasts, echoes))
    return specs


def run_batched(args):
    import torch

    import paper_2102_01604_gb300 as mpm
    from paper_2102_01604_gb300 import phantom

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    subjects = []
    for i, (dims, contrasts, echoes) in enumerate(batch_specs(args.seed + 1000 * rank, args.batch_mix)):
        prot = phantom.protocol(contrasts, echoes)
        with_mt = "MTw" in contrasts
        ph = phantom.phantom(dims, seed=args.seed + 17 * i + 1000 * rank, n_contrasts=len(contrasts),
                             with_mt=with_mt)
        yt = torch.from_numpy(ph["y"].astype(np.float32)).to(dev)
        b1p = torch.from_numpy(ph["b1p"].astype(np.float32)).to(dev)
        b1m = torch.from_numpy(ph["b1m"].astype(np.float32)).to(dev)
        s = mpm.mpm_forward(mpm.make_problem(prot, dims), yt, b1p, b1m)
        sig2, j = [], 0
        for ne in prot["n_echoes"]:
            m = s[j].double().mean().item() / SNR
            sig2.append(m * m)
            j += ne
        prot["sigma2"] = sig2
        x = phantom.rician_torch(s, prot, args.seed + 31 * i + 1).to(torch.bfloat16)
        del s, yt
        problem = mpm.make_problem(prot, dims, lam=LAMBDA, eps=EPS, echo_dtype=1)
        N = int(np.prod(dims))
        subjects.append({"problem": problem, "x": x, "b1p": b1p, "b1m": b1m, "N": N,
                         "y": torch.empty((problem.n_maps, N), device=dev),
                         "var": torch.empty((problem.n_maps, N), device=dev)})
    plain_opts = mpm.make_opts(gn_iters=GN_ITERS, cg_iters=CG_ITERS, graph=False)
    lanes_opts = mpm.make_opts(gn_iters=GN_ITERS, cg_iters=CG_ITERS, graph=True)
    phased_opts = mpm.make_opts(gn_iters=GN_ITERS, cg_iters=CG_ITERS, graph="phased")
    for sj in subjects:
        sj["ws"] = mpm.workspace(sj["problem"], plain_opts, device=dev)
        mpm.mpm_autotune(sj["problem"], plain_opts, ws=sj["ws"])
    torch.cuda.synchronize()
    total_vox = sum(sj["N"] for sj in subjects)

    def plain_step():
        for sj in subjects:
            mpm.mpm_fit(sj["problem"], plain_opts, sj["x"], sj["y"], sj["b1p"], sj["b1m"],
                        var=sj["var"], ws=sj["ws"])

    def batch_step(opts):
        mpm.mpm_fit_batch([sj["problem"] for sj in subjects], opts,
                          [sj["x"] for sj in subjects], [sj["y"] for sj in subjects],
                          b1ps=[sj["b1p"] for sj in subjects], b1ms=[sj["b1m"] for sj in subjects],
                          vars=[sj["var"] for sj in subjects], wss=[sj["ws"] for sj in subjects])

    def phased_step():
        batch_step(phased_opts)

    def lanes_step():
        batch_step(lanes_opts)

    counted = {}

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        counted["l0"] = mpm.mpm_kernel_launches()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        counted["n"] = mpm.mpm_kernel_launches() - counted["l0"]
        return a.elapsed_time(b) / 1000.0

    clocks = ClockSampler(local)
    clocks.start()
    t_batch = timed(phased_step)
    clk = clocks.stop()
    launches = counted["n"]
    t_lanes = timed(lanes_step)
    launches_lanes = counted["n"]
    t_plain = timed(plain_step)
    launches_plain = counted["n"]
    units = float(total_vox) * GN_ITERS * args.steps
    v_batch, tb = aggregate(t_batch, units, world, dev)
    v_lanes, tl = aggregate(t_lanes, units, world, dev)
    v_plain, tp = aggregate(t_plain, units, world, dev)
    if rank == 0:
        sizes = "64^3..176x240x256" if args.batch_mix == "uneven" else "all 64^3"
        line = {
            "metric": f"Mvoxel·GN-iter/s, batched MPM JTV fits (16 subjects, {sizes})",
            "value": round(v_batch / 1e6, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * tb / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"16 subjects, sizes {sizes}, 2-3 contrasts, 4-8 echoes "
                                   "per contrast, echoes stored bf16, 20 updates x 30 PCG + "
                                   "posterior variance each; one mpm_fit_batch call per step, "
                                   "phase-batched (opts.graph = 2: one launch per phase for "
                                   "each class of subjects)",
                       "subjects": [[sj["problem"].nx, sj["problem"].ny, sj["problem"].nz,
                                     sj["problem"].n_contrasts] for sj in subjects],
                       "voxels": total_vox,
                       "lanes_value": round(v_lanes / 1e6, 3),
                       "plain_value": round(v_plain / 1e6, 3),
                       "batched_over_plain": round(v_batch / v_plain, 3),
                       "lanes_over_plain": round(v_lanes / v_plain, 3),
                       "launches_per_step": {"phased": launches // args.steps,
                                             "lanes": launches_lanes // args.steps,
                                             "plain": launches_plain // args.steps},
                       "l2": "inputs larger than L2; no flush"},
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------- spatial projection arm

def moved_affines(shape):
    """Acquisition -> reconstruction voxel maps of the three scans: PDw in
    place, T1w turned 2 degrees about z and shifted (1.5, -1, 0.5) voxels, MTw
    turned 3 degrees about x and shifted (-0.75, 2, 1), turns about the
    volume centre."""
    ctr = (np.array(shape, dtype=np.float64) - 1) / 2

    def turn(ax, deg, t):
        a = np.deg2rad(deg)
        R = np.eye(3)
        i, j = [(1, 2), (0, 2), (0, 1)][ax]
        R[i, i], R[i, j], R[j, i], R[j, j] = np.cos(a), -np.sin(a), np.sin(a), np.cos(a)
        A = np.eye(4)
        A[:3, :3] = R
        A[:3, 3] = ctr - R @ ctr + np.asarray(t, dtype=np.float64)
        return A
    return [np.eye(4), turn(2, 2.0, [1.5, -1.0, 0.5]), turn(0, 3.0, [-0.75, 2.0, 1.0])]


def run_moved(args):
    import torch

    import paper_2102_01604_gb300 as mpm
    from paper_2102_01604_gb300 import phantom

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = args.seed + 1000 * rank
    contrasts, echoes = ("PDw", "T1w", "MTw"), (8, 8, 6)
    prot = phantom.protocol(contrasts, echoes)
    ph = phantom.phantom(SHAPE, seed=seed)
    yt = torch.from_numpy(ph["y"].astype(np.float32)).to(dev)
    grids = [SHAPE] * 3
    affs = moved_affines(SHAPE)
    proj = mpm.make_projection(grids, affs)
    N = int(np.prod(SHAPE))
    p_full = mpm.make_problem(prot, SHAPE, vx=VX)
    # each scan: the truth pulled to its grid, the library's forward model, Rician noise
    xs, bps, bms, sig2 = [], [], [], []
    i0 = 0
    for c in range(3):
        sub = {k: (v[c:c + 1] if isinstance(v, list) else v) for k, v in prot.items()}
        sub["te"] = prot["te"][i0:i0 + echoes[c]]
        i0 += echoes[c]
        fc = phantom.phantom(grids[c], seed=seed + 101 + c, n_contrasts=1)
        bp = torch.from_numpy(fc["b1p"].astype(np.float32)).to(dev)
        bm = torch.from_numpy(fc["b1m"].astype(np.float32)).to(dev)
        yc = mpm.mpm_pull(p_full, proj, c, yt)
        ps = mpm.make_problem(sub, grids[c], vx=VX)
        s = mpm.mpm_forward(ps, yc[:ps.n_maps].contiguous(), bp, bm)
        m = s[0].double().mean().item() / SNR
        sub["sigma2"] = [m * m]
        sig2.append(m * m)
        xs.append(phantom.rician_torch(s, sub, seed + 31 * c + 1).contiguous())
        bps.append(bp)
        bms.append(bm[0].contiguous())
        del s, yc
    prot["sigma2"] = sig2
    problem = mpm.make_problem(prot, SHAPE, vx=VX, lam=LAMBDA, eps=EPS)
    opts = mpm.make_opts(gn_iters=GN_ITERS, cg_iters=CG_ITERS)
    K = problem.n_maps
    y = torch.empty((K, N), dtype=torch.float32, device=dev)
    var = torch.empty((K, N), dtype=torch.float32, device=dev)
    ws = mpm.workspace_proj(problem, proj, opts, device=dev)
    mpm.mpm_autotune(problem, opts, ws=ws)
    # the same images fitted as if the scans were aligned (plain path)
    x_cat = torch.cat(xs, 0).contiguous()
    b1m_cat = torch.stack(bms, 0).contiguous()
    ws_plain = mpm.workspace(problem, opts, device=dev)

    def step():
        return mpm.mpm_fit_proj(problem, proj, opts, xs, y, bps, bms, var=var, ws=ws)[1]

    def plain_step():
        return mpm.mpm_fit(problem, opts, x_cat, y, bps[0], b1m_cat, var=var, ws=ws_plain)[1]

    def timed(fn, profile):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        if profile:
            mpm.mpm_profile_enable(True)
            mpm.mpm_profile_read()
        l0 = mpm.mpm_kernel_launches()
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            rep = fn()
        e1.record()
        torch.cuda.synchronize()
        prof = mpm.mpm_profile_read() if profile else None
        if profile:
            mpm.mpm_profile_enable(False)
        return e0.elapsed_time(e1) / 1000.0, rep, mpm.mpm_kernel_launches() - l0, prof

    clocks = ClockSampler(local)
    clocks.start()
    seconds, rep, launches, prof = timed(step, True)
    clk = clocks.stop()
    t_plain, _, _, _ = timed(plain_step, False)
    units = float(N) * GN_ITERS * args.steps
    value, t_max = aggregate(seconds, units, world, dev)
    v_plain, _ = aggregate(t_plain, units, world, dev)
    err = (y - yt).abs().mean(dim=1).tolist()
    if rank == 0:
        peak, peak_src = measured_peak()
        I = sum(echoes)
        kern = kernel_roofline(prof, N, args.steps, K, 3, I, peak)
        T = K * (K + 1) // 2
        evals = args.steps * (GN_ITERS + 1)
        gh_bytes = sum(N * (e * 4 + K * 4 + 8 + (K + T) * 4) for e in echoes) * evals
        rs_bytes = (3 * N * (K + T) * 4 + N * (K + T) * 4) * evals
        for kind, b in (("grad_hess_proj", gh_bytes), ("reslice", rs_bytes)):
            if kind in kern and prof[kind]["ms"] > 0:
                gbs = b / (prof[kind]["ms"] * 1e-3) / 1e9
                kern[kind]["bytes_per_launch"] = int(b / kern[kind]["launches"])
                kern[kind]["achieved_gbs"] = round(gbs, 1)
                kern[kind]["frac_of_measured_hbm"] = round(gbs / peak, 4)
        line = {
            "metric": "Mvoxel·GN-iter/s, 1 mm MPM JTV fit with spatial projection (moved scans)",
            "value": round(value / 1e6, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * t_max / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{SHAPE[0]}x{SHAPE[1]}x{SHAPE[2]} reconstruction grid, PDw/T1w/MTw "
                                   "8/8/6 echoes on their own grids: T1w turned 2 deg about z and "
                                   "shifted (1.5, -1, 0.5) voxels, MTw turned 3 deg about x and "
                                   "shifted (-0.75, 2, 1); Rician SNR 20; 20 updates x 30 PCG + "
                                   "posterior variance (mpm_fit_proj)",
                       "voxels": N,
                       "plain_value": round(v_plain / 1e6, 3),
                       "projection_cost": round(v_plain / value - 1.0, 4),
                       "map_error_vs_truth": [round(v, 4) for v in err],
                       "final_objective": rep.F[rep.iters],
                       "l2": "inputs larger than L2; no flush"},
            "kernels": kern, "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------- served arm

SERVED_SIZES = [((64, 64, 64), (1.0, 1.0, 1.0)), ((128, 128, 128), (1.0, 1.0, 1.0)),
                ((176, 240, 256), (1.0, 1.0, 1.0)), ((208, 300, 320), (0.8, 0.8, 0.8))]


def served_requests(n: int, rate: float, seed: int):
    """Seeded Poisson arrivals; each request draws one of the four volumes,
    3 or 4 contrasts (PDw, T1w, MTw[, VFA15]) and 4-8 echoes per contrast."""
    rng = np.random.default_rng(seed + 777)
    t, out = 0.0, []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        dims, vx = SERVED_SIZES[int(rng.integers(0, len(SERVED_SIZES)))]
        nc = int(rng.integers(3, 5))
        contrasts = ("PDw", "T1w", "MTw", "VFA15")[:nc]
        echoes = tuple(int(v) for v in rng.integers(4, 9, size=nc))
        out.append({"arrival": t, "dims": dims, "vx": vx, "contrasts": contrasts, "echoes": echoes})
    return out


def run_served(args):
    import time as _time

    import torch

    import paper_2102_01604_gb300 as mpm
    from paper_2102_01604_gb300 import phantom

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    opts = mpm.make_opts(gn_iters=50, cg_iters=CG_ITERS, tol_gn=1e-4)
    reqs = served_requests(args.requests, args.rate, args.seed + 1000 * rank)
    for i, r in enumerate(reqs):           # inputs resident before the clock starts
        prot = phantom.protocol(r["contrasts"], r["echoes"])
        ph = phantom.phantom(r["dims"], seed=args.seed + 13 * i, n_contrasts=len(r["contrasts"]))
        yt = torch.from_numpy(ph["y"].astype(np.float32)).to(dev)
        bp = torch.from_numpy(ph["b1p"].astype(np.float32)).to(dev)
        bm = torch.from_numpy(ph["b1m"].astype(np.float32)).to(dev)
        s = mpm.mpm_forward(mpm.make_problem(prot, r["dims"], vx=r["vx"]), yt, bp, bm)
        sig2, j = [], 0
        for ne in prot["n_echoes"]:
            m = s[j].double().mean().item() / SNR
            sig2.append(m * m)
            j += ne
        prot["sigma2"] = sig2
        r["x"] = phantom.rician_torch(s, prot, args.seed + 29 * i + 1)
        del s, yt
        r["problem"] = mpm.make_problem(prot, r["dims"], vx=r["vx"], lam=LAMBDA, eps=EPS)
        r["b1p"], r["b1m"] = bp, bm
        r["N"] = int(np.prod(r["dims"]))
        K = r["problem"].n_maps
        r["y"] = torch.empty((K, r["N"]), device=dev)
        r["var"] = torch.empty((K, r["N"]), device=dev)
        r["ws_bytes"] = mpm.mpm_workspace_size(r["problem"], opts)
    torch.cuda.synchronize()
    # one workspace as large as the biggest request for the plain arm; the
    # served arm gets an arena of 24 GB (or what is free) and 8 slots
    free, _ = torch.cuda.mem_get_info()
    arena_bytes = int(min(24 << 30, free * 0.7))
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device=dev)
    for r in reqs:                         # warm-up: tile shapes and first launches
        mpm.mpm_autotune(r["problem"], opts, ws=arena[:max(r["ws_bytes"], 1)])
    warm = reqs[0]
    mpm.mpm_fit(warm["problem"], opts, warm["x"], warm["y"], warm["b1p"], warm["b1m"],
                var=warm["var"], ws=arena[:warm["ws_bytes"]])
    torch.cuda.synchronize()

    def clock():
        return _time.perf_counter()

    # plain: one fit at a time, first come first served
    t0 = clock()
    lat_plain, units_plain = [], 0.0
    for r in reqs:
        now = clock() - t0
        if now < r["arrival"]:
            _time.sleep(r["arrival"] - now)
        st, rep = mpm.mpm_fit(r["problem"], opts, r["x"], r["y"], r["b1p"], r["b1m"], var=r["var"],
                              ws=arena[:r["ws_bytes"]])
        lat_plain.append(clock() - t0 - r["arrival"])
        units_plain += r["N"] * rep.iters
    span_plain = clock() - t0

    # served: continuous batching
    launches0 = mpm.mpm_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    srv = mpm.Server(arena, max_slots=8)
    t0 = clock()
    nxt, live, lat_srv, units_srv = 0, {}, [None] * len(reqs), 0.0
    while nxt < len(reqs) or live:
        now = clock() - t0
        while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
            r = reqs[nxt]
            live[srv.submit(r["problem"], opts, r["x"], r["y"], r["b1p"], r["b1m"], r["var"])] = nxt
            nxt += 1
        if not live:
            _time.sleep(max(0.0, reqs[nxt]["arrival"] - (clock() - t0)))
            continue
        srv.step()
        for t in list(live):
            state, status, rep = srv.poll(t)
            if state >= 2:
                i = live.pop(t)
                lat_srv[i] = clock() - t0 - reqs[i]["arrival"]
                units_srv += reqs[i]["N"] * rep.iters
    span_srv = clock() - t0
    clk = clocks.stop()
    srv.close()
    launches = mpm.mpm_kernel_launches() - launches0
    pct = lambda a, q: float(np.percentile(np.array(a), q))
    if rank == 0:
        line = {
            "metric": "Mvoxel·GN-iter/s, served MPM JTV fits (continuous batching); p50/p99 latency",
            "value": round(units_srv / span_srv / 1e6, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.requests, "warmup": 1, "ms_per_step": round(1000 * span_srv / args.requests, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "latency_s": {"mean": round(float(np.mean(lat_srv)), 3), "p50": round(pct(lat_srv, 50), 3),
                          "p99": round(pct(lat_srv, 99), 3)},
            "plain": {"value": round(units_plain / span_plain / 1e6, 3),
                      "latency_s": {"mean": round(float(np.mean(lat_plain)), 3),
                                    "p50": round(pct(lat_plain, 50), 3),
                                    "p99": round(pct(lat_plain, 99), 3)}},
            "config": {"workload": f"{args.requests} requests, Poisson arrivals at {args.rate}/s, "
                                   "volumes 64^3 / 128^3 / 176x240x256 (1 mm) / 208x300x320 (0.8 mm), "
                                   "3-4 contrasts, 4-8 echoes, stop at |dF|/F < 1e-4 (<= 50 updates), "
                                   "30 PCG, posterior variance; served: 8 slots, arena "
                                   f"{arena_bytes / 2**30:.1f} GiB; plain: FIFO one fit at a time",
                       "mix": [[*r["dims"], len(r["contrasts"])] for r in reqs],
                       "steps_meaning": "requests"},
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.write_traffic:
        doc = write_traffic(args.write_traffic, commands=TRAFFIC_COMMANDS)
        for kind, k in doc["kernels"].items():
            print(f"{kind:16s} {k['launches']:5d} launches {k['dram_bytes_per_voxel']:9.3f} B/voxel")
        return 0
    if args.launch_table:
        print(launch_table(read_ncu_csv(args.launch_table)))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.print_hashes:
        print_source_hashes()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "moved":
        return run_moved(args)
    if args.solver == "mg":
        return run_solvers(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
