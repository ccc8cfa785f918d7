#!/usr/bin/env python
"""Benchmark of the voxel-driven cone-beam backprojection on GB300.

Workload (the paper's RabbitCT case, Sect. 3.1): a 512^3 float32 volume
(256 mm cube, 0.5 mm voxels) reconstructed from 496 projections of
1248 x 960 pixels over a 200-degree C-arm short scan.  Data: the seeded
uniform [0, 1) timing stack (synthetic; the RabbitCT data set is not
available).  One step = one full reconstruction: reset the volume,
backproject all 496 projections, read the volume out.

Metric: GUP/s = L^3 * N / t (SI giga voxel updates per second with the
nominal count, Sect. 3.2), for FP32 projections (the headline `value`) and
the FP16 / BF16 projection-storage forms, plus the fraction of the
gather/FP32 roofline of the backprojection kernel.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank reconstructs its own volume (independent problems,
weak scaling, no collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import contextlib
import gc
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GUP/s at 512³×496 proj: FP32 vs FP16-projection form, % of roofline"
UNIT = "GUP/s"

# Roofline of the backprojection kernels (one update = one voxel x one
# projection), from the METHOD's work per update, per SM per clock, times the
# SMs and the SM clock sampled under load.  Every bound below is derivable
# from the per-update operation counts of Sect. 3.1-3.2 and the unit counts of
# the GPU; nothing in them comes from a profile of the kernel, so overhead the
# kernel adds cannot raise its peak.
#   fp32_pipe: 128 FP32 lanes per SM over the 20.5 FP32-pipe operations an
#     update needs with FMA and incremental stepping: 3 FFMA geometry + 1.5
#     FFMA of the y/z terms per 4 voxels, 2 FMUL u/v, 2 floor, 2 FADD/FFMA
#     gather coordinate, 2 FADD fractions, 3 FADD + 3 FFMA bilinear
#     interpolation, 1 FMUL + 1 FFMA weight and accumulate (the paper's 31
#     flop, Sect. 3.2, with the multiply-adds fused);
#   mufu: 16 reciprocals per SM per clock, one per update;
#   smem (TMA path): 128 B per SM per clock of shared-memory bandwidth over
#     the 4 projection texels an update reads: 16 B for float32 storage, 8 B
#     for 16-bit storage;
#   gather (texture path): the texture unit's 2x2-gather rate for the storage
#     type, MEASURED on this GPU by bp_probe_gather (one gather per update).
FP32_PER_SM_CLK = 128.0
FP32_INSTR_PER_UPDATE = 20.5
MUFU_PER_SM_CLK = 16.0
SMEM_BYTES_PER_SM_CLK = 128.0
TEXELS_PER_UPDATE = 4
# Diagnostics only (they explain where a kernel loses time; they are not its
# roofline): instruction issue at the instructions per computed update that
# ncu counts for the kernel (smsp__inst_executed x 32 / computed updates;
# profiles/<kernel>_<form>_512x64.md), and shared-memory bandwidth including
# the TMA fill of each brick's box.
ISSUE_PER_SM_CLK = 128.0
INSTR_PER_UPDATE = {("texture", "f32"): 29.8, ("texture", "f16"): 26.0, ("tma", "f32"): 24.4, ("tma", "f16"): 23.3}
# Adjoint (B^T, the same arithmetic per update as B, with the four corner
# terms scattered instead of gathered):
#   fp32_pipe: the forward's 20.5 FP32-pipe operations (geometry, floor,
#     fractions, four bilinear weights, 1/w^2);
#   smem_atomics: four shared-memory atomics per update, conflict-free (one
#     wavefront per warp instruction, one wavefront per SM per clock);
#   mufu: one reciprocal per update.
# Diagnostics: ncu's instructions per nominal update and wavefronts per
# atomic instruction (profiles/bp_adjoint_smem_kernel_256.md).
ADJ_ATOMICS_PER_UPDATE = 4
ADJ_INSTR_PER_UPDATE = 53.1
ADJ_ATOMIC_WAVEFRONTS = 3.67


def adjoint_roofline_gups(sm_mhz: float, sms: int) -> dict:
    f = sm_mhz * 1e6
    bounds = {"fp32_pipe": sms * FP32_PER_SM_CLK / FP32_INSTR_PER_UPDATE * f / 1e9,
              "smem_atomics": sms * 32.0 / ADJ_ATOMICS_PER_UPDATE * f / 1e9,
              "mufu": sms * MUFU_PER_SM_CLK * f / 1e9}
    bounds["min"] = min(bounds.values())
    return bounds


def adjoint_diagnostics_gups(sm_mhz: float, sms: int) -> dict:
    """Rates the adjoint kernel as built could reach if issue or its bank
    conflicts alone bound it (from its ncu profile; not the roofline)."""
    f = sm_mhz * 1e6
    return {"issue_at_measured_instr": sms * ISSUE_PER_SM_CLK / ADJ_INSTR_PER_UPDATE * f / 1e9,
            "smem_atomics_at_measured_wavefronts":
                sms / (ADJ_ATOMICS_PER_UPDATE * ADJ_ATOMIC_WAVEFRONTS / 32) * f / 1e9,
            "instr_per_update": ADJ_INSTR_PER_UPDATE, "wavefronts_per_atomic": ADJ_ATOMIC_WAVEFRONTS}


def texel_bytes_per_update(form: str) -> float:
    """Projection bytes an update reads: four texels of the storage type."""
    return TEXELS_PER_UPDATE * (4 if form == "f32" else 2)


def tma_smem_bytes_per_update(form: str, depth: int = 16) -> float:
    """Shared-memory bytes per update of the TMA kernel as built: the staged
    8-byte elements an update loads (two for float32 pairs, one for 16-bit
    column quads) plus the box fill (120 element columns by the box rows of
    the brick depth) per 32 x 16 x depth brick; a diagnostic."""
    rows = {8: 36, 12: 48, 16: 58}[depth] - (0 if form == "f32" else 1)
    loads = 2 if form == "f32" else 1
    return 8.0 * loads + 120 * rows * 8 / (32 * 16 * depth)


def roofline_peak_gups(path: str, form: str, sm_mhz: float, sms: int, gather_per_sm_clk: float) -> dict:
    f = sm_mhz * 1e6
    bounds = {
        "fp32_pipe": sms * FP32_PER_SM_CLK / FP32_INSTR_PER_UPDATE * f / 1e9,
        "mufu": sms * MUFU_PER_SM_CLK * f / 1e9,
    }
    if path == "tma":
        bounds["smem"] = sms * SMEM_BYTES_PER_SM_CLK / texel_bytes_per_update(form) * f / 1e9
    else:
        bounds["gather"] = sms * gather_per_sm_clk * f / 1e9
    bounds["min"] = min(bounds.values())
    return bounds


def roofline_diagnostics_gups(path: str, form: str, sm_mhz: float, sms: int, depth: int = 16) -> dict:
    """What the kernel as built is limited by (from its ncu profile): issue at
    its measured instructions per update, and for the TMA path shared-memory
    bandwidth including the box fill.  Explains a fraction; not the peak."""
    f = sm_mhz * 1e6
    d = {}
    instr = INSTR_PER_UPDATE.get((path, form))
    if instr is not None:
        d["issue_at_measured_instr"] = sms * ISSUE_PER_SM_CLK / instr * f / 1e9
        d["instr_per_update"] = instr
    if path == "tma":
        d["smem_with_box_fill"] = sms * SMEM_BYTES_PER_SM_CLK / tma_smem_bytes_per_update(form, depth) * f / 1e9
    return d


def algorithmic_bytes(L: int, n: int, isx: int, isy: int, form: str, path: str, computed_fraction: float,
                       Lz: int | None = None, depth: int = 16) -> int:
    """Bytes one mid-step launch of the backprojection kernel must move: the
    L x L x Lz volume (Lz = L for the whole cube) read and written once, each
    of the n projections read once (the TMA path reads staged images of
    8-byte elements, isx + 1 columns padded to an even count: float32 pairs,
    isy rows; 16-bit column quads, isy + 1 rows), and for the FP32 form the
    per-block centring records (3 x 16 B) of the (block, projection) pairs it
    computes (texture blocks of 32 x 8 x 4 voxels, TMA bricks of 32 x 16 x
    depth)."""
    px = 4 if form == "f32" else 2
    Lz = L if Lz is None else Lz
    if path == "tma":
        pitch = -(-(isx + 1) // 2) * 2
        rows = isy if form == "f32" else isy + 1
        total = 8 * L * L * Lz + n * pitch * rows * 8
        tile = (32, 16, depth)
    else:
        total = 8 * L * L * Lz + n * isx * isy * px
        tile = (32, 8, 4)
    if form == "f32":
        blocks = -(-L // tile[0]) * -(-L // tile[1]) * -(-Lz // tile[2])
        total += int(48 * n * blocks * computed_fraction)
    return int(total)


def ncu_fields(kernel_file: str, profile: str, names) -> dict | None:
    """Numbers from a committed ncu summary (its "- name: value" list items),
    or None when the summary is missing, lacks one of them, or the kernel
    source changed since it was captured (the summary records the source's
    sha256)."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        src = open(os.path.join(ROOT, "paper_1104_5243_gb300", "csrc", kernel_file), "rb").read()
    except OSError:
        return None
    fields = {}
    for ln in text.splitlines():
        item = ln.strip().lstrip("-* ").strip()
        if ":" in item and item.startswith(tuple(names) + ("source_sha256",)):
            k, v = item.split(":", 1)
            fields[k.strip("` ")] = v.strip().strip("`")
    if fields.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    try:
        return {k: float(fields[k]) for k in names}
    except (KeyError, ValueError):
        return None


def hbm_peak_gbs() -> tuple[float, str]:
    """HBM bandwidth peak: the measured copy figure of MEASURED_PEAKS.json
    when present, else 6800 GB/s (one earlier measurement on a GB300)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "fallback"


def ncu_traffic(kernel_file: str, profile: str):
    """DRAM bytes per launch from a committed ncu summary (None as ncu_fields)."""
    f = ncu_fields(kernel_file, profile, ["traffic_bytes_per_launch"])
    return None if f is None else f["traffic_bytes_per_launch"]


# Utilisation of the FP32 (FMA) pipe, of shared memory and of DRAM, and the
# issue rate, each in % of its peak, from the committed full ncu capture of
# the dominant kernel on the 512^3 x 64 case.
NCU_FRACTIONS = ["fma_pipe_pct", "smem_wavefronts_pct", "dram_pct", "issue_active_pct"]


@contextlib.contextmanager
def gc_paused():
    """Python's cyclic garbage collector off inside a timed region (collected
    just before), as timeit does: a collection of the bench's heap inside a
    step stalls the host thread that issues the copies and launches."""
    gc.collect()
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.err = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:  # nvidia-smi missing
            self.err = str(e)
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        if self.err or not getattr(self, "lines", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": self.err or "no samples"}
        sm, smax, pw, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": "unparsable samples"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "power_w_max": max(pw),
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_id_for_smi(torch, dev: int) -> str | None:
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id
        dom = torch.cuda.get_device_properties(dev).pci_domain_id
        devid = torch.cuda.get_device_properties(dev).pci_device_id
        return f"{dom:08x}:{bus:02x}:{devid:02x}.0"
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis and "," not in vis:
            return vis
        return None


# ---------------------------------------------------------------------------
# Multi-rank bookkeeping (one process per GPU, no data-path collective): the
# slowest rank's time decides, and the value is the work of all ranks over
# that time.  By default every rank reconstructs its own volume (weak
# scaling); with --split z the ranks share one volume, each the z-slab
# slab_of_rank gives it, from the whole projection stack (strong scaling).
def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gups(updates_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """GUP/s of the whole job: every rank's updates over the slowest rank's time."""
    return updates_per_rank * steps * world / (max_ms / 1e3) / 1e9


def slab_of_rank(L: int, world: int, rank: int, granule: int = 8) -> tuple[int, int]:
    """(z0, nz) of this rank's slab when the z extent of an L^3 volume is
    split over world ranks, as the paper splits the z loop between threads
    (Sect. 6): contiguous slabs of whole granules (8 slices, the depth of
    the shallowest TMA brick, so no rank computes a partial brick except at
    the top of the volume), in rank order, sizes differing by at most one
    granule.  A rank left without a granule gets nz = 0."""
    if L < 1 or world < 1 or not 0 <= rank < world or granule < 1:
        raise ValueError("slab_of_rank: need L >= 1, world >= 1, 0 <= rank < world, granule >= 1")
    units = -(-L // granule)
    q, r = divmod(units, world)
    u0 = rank * q + min(rank, r)
    u1 = u0 + q + (1 if rank < r else 0)
    z0, z1 = min(L, u0 * granule), min(L, u1 * granule)
    return z0, z1 - z0


def reciprocal_modes(bp, step, out, stream, args, updates: int, gups_fast: float) -> dict:
    """The paper's reciprocal comparison (Sect. 7.2): the same float32 step
    with the IEEE reciprocal (BP_OPT_IEEE_RCP 1) against the approximate one
    (the default), GUP/s of each and the PSNR of the approximate volume
    against the IEEE one (M = max - min of the IEEE volume).  Runs after the
    timed region."""
    import math

    import torch
    from paper_1104_5243_gb300 import _native as N
    step()
    fast = out.clone()
    bp.set_option(N.BP_OPT_IEEE_RCP, 1)
    for _ in range(args.warmup):
        step()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    ieee = out.clone()
    bp.set_option(N.BP_OPT_IEEE_RCP, 0)
    span = float(ieee.max() - ieee.min())
    mse = float(((fast.double() - ieee.double()) ** 2).mean())
    psnr = 10.0 * math.log10(span * span / mse) if mse > 0 else float("inf")
    return {"approx_gups": round(gups_fast, 2), "ieee_gups": round(updates / (ms / 1e3) / 1e9, 2),
            "psnr_approx_vs_ieee_db": round(psnr, 1),
            "note": "f32, same workload and path; uniform [0,1) stack"}


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def cpu_baseline(L: int, n_sample: int):
    """The FP64 oracle (as it stands) on a bounded sample of the workload: the
    full L^3 volume backprojected from the first n_sample projections, with
    OpenMP schedule(static,1) over z (the paper's Sect. 6 scheme)."""
    import numpy as np

    import oracle
    from paper_1104_5243_gb300 import synth
    scan, vol = synth.SCANS["full"], synth.Volume(L)
    oracle.build()
    A = oracle.carm_matrices(scan)[:n_sample]
    stack = synth.uniform_stack(n_sample, scan.isy, scan.isx, seed=synth.TIMING_SEED)
    out = np.zeros((L, L, L), dtype=np.float64)
    t0 = time.perf_counter()
    oracle.backproject(L, vol.R, vol.O, stack, A, vol=out)
    dt = time.perf_counter() - t0
    gups = L ** 3 * n_sample / dt / 1e9
    return {"value": round(gups, 4), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "cpu_model": cpu_model(), "affinity_cpus": len(os.sched_getaffinity(0)),
            "sample": f"{L}^3 volume x first {n_sample} of 496 projections (1248x960), FP64, "
                      f"{dt:.1f} s", "seconds": round(dt, 2)}


def cpu_baseline_one_core(L: int, n_sample: int):
    """The same oracle on one host core (OMP_NUM_THREADS=1, read when the
    oracle library loads), in a child process started by fork+exec, so the
    parent's CUDA context is not inherited."""
    import subprocess
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_baseline(%d, %d)))" % (ROOT, L, n_sample))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": UNIT, "cores": d["cores"], "sample": d["sample"]}


def run_reference(args, rank: int):
    """Reference arm: the FP64 oracle (there is no reference implementation
    of the paper's code) on the host cores, each step a bounded sample of the
    512^3 x 496 workload: the full volume from --ref-proj projections."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(args.L, max(1, args.ref_proj // 8))
    samples = [cpu_baseline(args.L, args.ref_proj) for _ in range(args.steps)]
    value = statistics.median(c["value"] for c in samples)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"FDK backprojection {args.L}^3 x 496 x 1248x960, uniform [0,1) stack seed "
                               "20110426, 200-degree C-arm (bounded sample per step)",
                   "L": args.L, "n_proj": 496, "detector": [1248, 960]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": samples[0]["cores"], "kind": "oracle",
                         "sample": samples[0]["sample"], "cpu_model": samples[0]["cpu_model"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def link_rates(host_src, dev_dst, host_dst, dev_src, stream) -> dict:
    """Host-to-device and device-to-host copy rates (GB/s) on the end-to-end
    step's own pinned buffers, in the same run: the projection stack up, the
    volume down, two copies each, CUDA events on the stream."""
    import torch
    out = {}
    for name, dst, src in (("h2d_gbs", dev_dst, host_src), ("d2h_gbs", host_dst, dev_src)):
        n = min(dst.numel(), src.numel())
        d, s_ = dst.view(-1)[:n], src.view(-1)[:n]
        d.copy_(s_, non_blocking=True)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(2):
            d.copy_(s_, non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        out[name] = round(2 * n * 4 / (t0.elapsed_time(t1) / 1e3) / 1e9, 1)
    return out


def time_volume(api, N, L: int, scan, stack, A, form: str, warmup: int, steps: int, stream) -> dict:
    """GUP/s of the device-resident step at another volume size: nominal
    updates over the step time, and over the backprojection kernels' event
    time (nominal and computed updates), with the path and brick depth the
    library chose (and, on the texture path, its warp layout)."""
    import torch
    from paper_1104_5243_gb300 import synth
    vol = synth.Volume(L)
    out = torch.empty((L, L, L), dtype=torch.float32, device="cuda")
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=form)

    def step():
        bp.reset()
        bp.add_projections(stack, A)
        bp.finalize(out)

    for _ in range(warmup):
        step()
    bp.set_option(N.BP_OPT_TIMING, 1)
    bp.kernel_stats()
    c0 = bp.query(N.BP_QUERY_UPDATES_COMPUTED)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    launches, kms = bp.kernel_stats()
    computed = (bp.query(N.BP_QUERY_UPDATES_COMPUTED) - c0) / steps
    nominal = L ** 3 * scan.n
    res = {"gups": round(nominal / (ms / 1e3) / 1e9, 2), "ms_per_step": round(ms, 3),
           "kernel_gups": round(nominal / (kms / steps / 1e3) / 1e9, 2),
           "kernel_gups_computed": round(computed / (kms / steps / 1e3) / 1e9, 2),
           "computed_fraction": round(computed / nominal, 4), "path": bp.last_path,
           "brick_depth": bp.query(N.BP_QUERY_LAST_BRICK_DEPTH) if bp.last_path == "tma" else None,
           "lanes_x": bp.query(N.BP_QUERY_LAST_LANES_X) if bp.last_path == "texture" else None,
           "steps": steps}
    bp.close()
    del out
    torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=512)
    ap.add_argument("--forms", default="f32,f16,bf16")
    ap.add_argument("--path", default="auto", choices=["auto", "texture", "tma"],
                    help="data path of the backprojection (profiling runs; default: the library's choice)")
    ap.add_argument("--n-proj", type=int, default=496, help="projections per step (profiling runs)")
    ap.add_argument("--split", default="replica", choices=["replica", "z"],
                    help="replica: each rank reconstructs its own volume (weak scaling); z: the ranks "
                         "share one volume, one z-slab each (strong scaling)")
    ap.add_argument("--cpu-proj", type=int, default=160, help="projections in the oracle sample")
    ap.add_argument("--ref-proj", type=int, default=48, help="projections per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the adjoint and learned-filter timings")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.split == "z" and world > -(-args.L // 8):      # every rank sees the same sizes and stops here
        ap.error(f"--split z: {world} ranks but only {-(-args.L // 8)} slabs of 8 slices")

    import numpy as np
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from paper_1104_5243_gb300 import build as native_build
    native_build.build()
    from paper_1104_5243_gb300 import _native as N
    from paper_1104_5243_gb300 import api, synth

    full = synth.SCANS["full"]
    scan = synth.Scan(n=args.n_proj, isx=full.isx, isy=full.isy, pitch=full.pitch,
                      scan_deg=full.scan_deg * (args.n_proj - 1) / (full.n - 1))
    vol = synth.Volume(args.L)
    A = api.carm_matrices(scan)                         # FP64 on the GPU
    stack_host = torch.from_numpy(synth.uniform_stack(scan.n, scan.isy, scan.isx)).pin_memory()
    stack = stack_host.cuda()
    z0, nz = (0, args.L) if args.split == "replica" else slab_of_rank(args.L, world, rank)
    updates = args.L * args.L * nz * scan.n           # this rank's updates per step
    job_updates = updates * world if args.split == "replica" else args.L ** 3 * scan.n
    out = torch.empty((nz, args.L, args.L), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def rank_max(x: float) -> float:
        return max_over_ranks(x, dist, "cuda")

    smi_id = gpu_id_for_smi(torch, local_rank)
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    gather_rate = {f: N.bp_probe_gather({"f32": N.BP_F32, "f16": N.BP_F16, "bf16": N.BP_BF16}[f])
                   for f in args.forms.split(",")}
    forms = {}
    kernel = {}
    path_taken = {}
    depth_taken = {}
    clocks = None
    rcp_modes = None
    # End to end through the public API: pinned host projections in, the
    # finished volume out to pinned host memory, every step, in the one call
    # that does both (the last launch stores the volume into the host buffer).
    # Measured before the device-resident forms: after the clock sampler's
    # nvidia-smi had run and been stopped, steps of this region took up to
    # 54-99 ms against 45 ms with unchanged kernel times (host copies held up).
    e2e = None
    if not args.no_e2e:
        vol_host = torch.empty((nz, args.L, args.L), dtype=torch.float32).pin_memory()
        bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype="f32", nz=nz, z0=z0)

        def step_e2e():
            bp.reset()
            bp.add_projections_finalize(stack_host, A, vol_host)

        for _ in range(max(args.warmup, 5)):   # host-copy warm-up: the first pinned transfers run slower
            step_e2e()
        barrier()
        with gc_paused():
            t0 = time.perf_counter()
            walls = []
            for _ in range(args.steps):
                ts = time.perf_counter()
                step_e2e()     # returns after the finished volume is in host memory
                walls.append((time.perf_counter() - ts) * 1e3)
            torch.cuda.synchronize()
            t_end = time.perf_counter()
        wall = rank_max(t_end - t0)
        bp.close()
        link = link_rates(stack_host, stack, vol_host, out, stream)
        e2e = {"value": round(whole_job_gups(job_updates, args.steps, 1, wall * 1e3), 2), "unit": UNIT,
               "link": link,
               "step_ms": {"mean": round(wall * 1e3 / args.steps, 2), "median": round(statistics.median(walls), 2),
                           "min": round(min(walls), 2), "max": round(max(walls), 2),
                           "each": [round(w, 2) for w in walls]},
               "device_resident_ms_per_step": None,   # filled in after the forms below
               "h2d_bytes_per_step": int(stack_host.numel() * 4),
               "d2h_bytes_per_step": int(vol_host.numel() * 4),
               "step": "reset + bp_add_projections_finalize (pinned host images in, finished volume into "
                       "pinned host memory)"}

    for form in args.forms.split(","):
        bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=form, nz=nz, z0=z0)
        bp.set_option(N.BP_OPT_PATH, {"auto": 0, "texture": 1, "tma": 2}[args.path])

        def step():
            bp.reset()
            bp.add_projections(stack, A)
            bp.finalize(out)

        for _ in range(args.warmup):
            step()
        bp.set_option(N.BP_OPT_TIMING, 1)
        bp.kernel_stats()
        computed0 = bp.query(N.BP_QUERY_UPDATES_COMPUTED)
        barrier()
        with ClockSampler(smi_id) as cs, gc_paused():
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(args.steps):
                step()
            t1.record(stream)
            torch.cuda.synchronize()
        ms = rank_max(t0.elapsed_time(t1))
        launches, kms = bp.kernel_stats()
        computed = bp.query(N.BP_QUERY_UPDATES_COMPUTED) - computed0
        path_taken[form] = bp.last_path
        depth_taken[form] = bp.query(N.BP_QUERY_LAST_BRICK_DEPTH)
        bp.set_option(N.BP_OPT_TIMING, 0)
        gups = whole_job_gups(job_updates, args.steps, 1, ms)
        forms[form] = {"value": round(gups, 2), "ms_per_step": round(ms / args.steps, 3)}
        kernel[form] = {"launches": launches, "kernel_ms": kms,
                        "kernel_gups": updates * args.steps / (kms / 1e3) / 1e9 if kms > 0 else None,
                        "computed_fraction": computed / (updates * args.steps),
                        "kernel_gups_computed": computed / (kms / 1e3) / 1e9 if kms > 0 else None}
        if form == "f32":
            clocks = cs.summary()
            if not args.no_extra:
                rcp_modes = reciprocal_modes(bp, step, out, stream, args, updates,
                                             updates * args.steps / (ms / 1e3) / 1e9)
        bp.close()

    if e2e is not None:
        e2e["device_resident_ms_per_step"] = forms.get("f32", {}).get("ms_per_step")

    # The other volume sizes of the full-scale and precision workloads
    # (256^3: 1 mm voxels, and 1024^3: 0.25 mm, from the same 496
    # projections of 1248x960), f32 and f16 storage, device-resident,
    # timed like the headline (kernel events on the context's stream).
    sizes = {}
    if not args.no_extra and args.split == "replica" and args.n_proj == 496:
        for L2 in (256, 1024):
            if L2 == args.L:
                continue
            sizes[str(L2)] = {f: time_volume(api, N, L2, scan, stack, A, f, 3, 2 if L2 > 512 else args.steps,
                                             stream)
                              for f in ("f32", "f16")}

    # The other two timed paths of the method: the adjoint (B^T, the autograd
    # backward) on the differentiation workload, 256^3 -> 248 x 624x480, and
    # one training step of the learned filter (8 phantoms at 128^3 x 120 x
    # 312x240: row filter, backprojection, adjoint, filter gradient).
    extra = {}
    if not args.no_extra:
        half = synth.SCANS["half"]
        vh = synth.Volume(256)
        Ah = api.carm_matrices(half)
        fvol = torch.from_numpy(synth.uniform_volume(256, seed=5)).cuda()
        gproj = torch.empty((half.n, half.isy, half.isx), dtype=torch.float32, device="cuda")
        bp = api.Backprojector(vh.L, vh.R, vh.O, half.isx, half.isy)
        for _ in range(args.warmup):
            bp.adjoint(fvol, Ah, out=gproj)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            bp.adjoint(fvol, Ah, out=gproj)
        t1.record(stream)
        torch.cuda.synchronize()
        ams = t0.elapsed_time(t1) / args.steps
        bp.close()
        agups = 256 ** 3 * half.n / (ams / 1e3) / 1e9
        abounds = adjoint_roofline_gups((clocks or {}).get("sm_mhz") or 2070.0, sms)
        abind = min((k for k in abounds if k != "min"), key=lambda k: abounds[k])
        extra["adjoint"] = {"workload": "B^T 256^3 -> 248 x 624x480", "ms_per_call": round(ams, 3),
                            "gups": round(agups, 2),
                            "roofline": {"bound": abind, "achieved": round(agups, 2),
                                         "peak": round(abounds["min"], 1), "unit": UNIT,
                                         "frac": round(agups / abounds["min"], 4),
                                         "bounds_gups": {k: round(v, 1) for k, v in abounds.items()},
                                         "peak_basis": "min(FP32 pipe at 20.5 FP32 operations per update, "
                                                       "4 conflict-free shared-memory atomics per update, MUFU) "
                                                       "x SMs x sampled SM clock",
                                         "note": "achieved is per call (4 launches, the output zeroing "
                                                 "and the centring pre-pass included)"},
                            "diagnostics": {k: round(v, 1) for k, v in
                                            adjoint_diagnostics_gups((clocks or {}).get("sm_mhz") or 2070.0,
                                                                     sms).items()}}
        from paper_1104_5243_gb300 import learned as lm
        torch.manual_seed(0)
        lm.train(steps=args.warmup, batch=8)
        torch.cuda.synchronize()
        t = time.perf_counter()
        lm.train(steps=args.steps, batch=8)
        torch.cuda.synchronize()
        extra["learned_filter_train_step"] = {
            "workload": "8 phantoms, 128^3 x 120 x 312x240, forward + backward + Adam",
            "ms_per_step": round((time.perf_counter() - t) / args.steps * 1e3, 2),
            "note": "includes generating the phantom batch on the GPU once per call"}
        # CGLS on the adjoint's workload: per iteration one forward model
        # (B^T) and one transpose (B) through the library, plus the vector
        # updates; (K + 1 iterations - 1 iteration) / K removes the initial
        # transpose
        from paper_1104_5243_gb300 import iterative
        bp = api.Backprojector(vh.L, vh.R, vh.O, half.isx, half.isy)
        ops = iterative.Operators(bp, Ah, iterative.model_scale(vh.R, api.iso_pitch(half)))
        pdata = ops.forward(fvol)
        iterative.cgls(ops, pdata, 1)
        torch.cuda.synchronize()
        t = time.perf_counter()
        iterative.cgls(ops, pdata, 1)
        torch.cuda.synchronize()
        t1 = time.perf_counter() - t
        t = time.perf_counter()
        iterative.cgls(ops, pdata, args.steps + 1)
        torch.cuda.synchronize()
        cg_ms = (time.perf_counter() - t - t1) / args.steps * 1e3
        bp.close()
        extra["cgls_iteration"] = {"workload": "256^3 x 248 x 624x480, one B^T and one B per iteration",
                                   "ms_per_iteration": round(cg_ms, 3),
                                   "gups": round(2 * 256 ** 3 * half.n / (cg_ms / 1e3) / 1e9, 1)}
        # A 512^3 volume reconstructed slab by slab (4 slabs of 128 slices)
        # into pinned host memory, from the device stack: two slab contexts
        # moved over the volume, each on its own stream and host thread
        big = torch.empty((args.L,) * 3, dtype=torch.float32).pin_memory()
        slab = max(8, args.L // 4)
        api.backproject_slabs(args.L, vol.R, vol.O, stack, A, slab=slab, out=big)
        torch.cuda.synchronize()
        t = time.perf_counter()
        api.backproject_slabs(args.L, vol.R, vol.O, stack, A, slab=slab, out=big)
        torch.cuda.synchronize()
        sl_s = time.perf_counter() - t
        # the same with the two slab contexts kept across reconstructions
        # (their allocations made once), as a series of volumes uses them
        pool = api.slab_contexts(args.L, vol.R, vol.O, scan.isx, scan.isy, slab, count=2)
        api.backproject_slabs(args.L, vol.R, vol.O, stack, A, slab=slab, out=big, pool=pool)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            api.backproject_slabs(args.L, vol.R, vol.O, stack, A, slab=slab, out=big, pool=pool)
        torch.cuda.synchronize()
        pool_s = (time.perf_counter() - t) / args.steps
        for bp in pool:
            bp.close()
        extra["slab_reconstruction"] = {
            "workload": f"{args.L}^3 x {scan.n} x {scan.isx}x{scan.isy} in slabs of {slab} slices into pinned "
                        "host memory, two slab contexts on their own streams and host threads",
            "ms": round(sl_s * 1e3, 2), "gups": round(args.L ** 3 * scan.n / sl_s / 1e9, 1),
            "note": "ms / gups: one call that creates its two contexts",
            "reused_contexts_ms": round(pool_s * 1e3, 2),
            "reused_contexts_gups": round(args.L ** 3 * scan.n / pool_s / 1e9, 1)}
        del big

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    head = "f32" if "f32" in forms else next(iter(forms))
    f32 = forms[head]
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peaks = {f: roofline_peak_gups(path_taken.get(f, "texture"), f, sm_mhz, sms, gather_rate[f]) for f in forms}
    peak = peaks[head]
    k = kernel[head]
    achieved = k["kernel_gups_computed"]
    head_path = path_taken.get(head, "texture")
    kname, ksrc = ("bp_tma_kernel", "bp_tma.cu") if head_path == "tma" else ("bp_fwd_kernel", "bp_fwd.cu")
    traffic = ncu_traffic(ksrc, f"{kname}_{head}_{args.L}.md") if args.n_proj == 496 and nz == args.L else None
    ncu_pct = ncu_fields(ksrc, f"{kname}_{head}_{args.L}x64.md", NCU_FRACTIONS)
    basis = ("shared-memory bandwidth" if head_path == "tma" else "the measured texture gather rate")
    head_depth = depth_taken.get(head) or 16
    alg_bytes = algorithmic_bytes(vol.L, min(scan.n, 64), scan.isx, scan.isy, head, head_path,
                                  k["computed_fraction"], nz, head_depth)
    avg_ms = k["kernel_ms"] / max(k["launches"], 1)
    hbm_peak, hbm_src = hbm_peak_gbs()
    bind = min((kk for kk in peak if kk != "min"), key=lambda kk: peak[kk])
    roofline = {
        "bound": "alu", "unit": UNIT, "kernel": f"{kname} ({head} projections, {head_path} path)",
        "achieved": round(achieved, 2) if achieved else None,
        "peak": round(peak["min"], 1),
        "frac": round(achieved / peak["min"], 4) if achieved else None,
        "binding": bind,
        "peak_basis": f"min(FP32 pipe at {FP32_INSTR_PER_UPDATE} FP32 operations per update, "
                      f"{basis} at the 4 texels an update reads, MUFU) x SMs x sampled SM clock "
                      "(derived from unit counts and clocks; no profile of the kernel enters it); "
                      "achieved counts the updates computed (culled bricks excluded)",
        "achieved_nominal": round(k["kernel_gups"], 2),
        "computed_fraction": round(k["computed_fraction"], 4),
        "peak_at_sm_mhz": sm_mhz,
        "gather_per_sm_clk_measured": {f: round(v, 3) for f, v in gather_rate.items()},
        "bounds_gups": {kk: round(v, 1) for kk, v in peak.items()},
        "diagnostics": {kk: round(v, 1) for kk, v in
                        roofline_diagnostics_gups(head_path, head, sm_mhz, sms, head_depth).items()},
        "avg_launch_ms": round(k["kernel_ms"] / max(k["launches"], 1), 4),
        "launches": k["launches"],
        "traffic": traffic,
        "ncu_pct_of_peak": (dict(ncu_pct, profile=f"profiles/{kname}_{head}_{args.L}x64.md")
                            if ncu_pct else None),
        "algorithmic_bytes_per_launch": alg_bytes,
        # DRAM side (not the bound): bytes per launch over the average launch
        # time, against the HBM peak
        "hbm": ({"algorithmic_gbs": round(alg_bytes / (avg_ms / 1e3) / 1e9, 1),
                 "traffic_gbs": round(traffic / (avg_ms / 1e3) / 1e9, 1) if traffic else None,
                 "peak_gbs": hbm_peak, "peak_source": hbm_src,
                 "frac_algorithmic": round(alg_bytes / (avg_ms / 1e3) / 1e9 / hbm_peak, 4),
                 "frac_traffic": round(traffic / (avg_ms / 1e3) / 1e9 / hbm_peak, 4) if traffic else None}
                if avg_ms > 0 else None),
    }
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(args.L, args.cpu_proj)
        cpu["one_core"] = cpu_baseline_one_core(args.L, max(1, args.cpu_proj // 16))
    line = {
        "metric": METRIC, "value": f32["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": f32["ms_per_step"], "higher_is_better": True,
        "scaling": "weak" if args.split == "replica" else "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"FDK backprojection {args.L}^3 x {scan.n} x {scan.isx}x{scan.isy}, "
                               f"uniform [0,1) stack seed 20110426, {scan.scan_deg:.0f}-degree C-arm",
                   "L": args.L, "n_proj": scan.n, "detector": [scan.isx, scan.isy],
                   "l2": "inputs larger than L2 (2.38 GB projections + 0.54 GB volume per step)",
                   "step": "reset + bp_add_projections(496, device-resident) + finalize",
                   "parallelism": (f"replicas x{world}" if args.split == "replica"
                                   else f"z-slabs x{world} (rank 0: z {z0}..{z0 + nz - 1})")},
        "forms": {kk: {**v, "kernel_gups": round(kernel[kk]["kernel_gups"], 2),
                       "kernel_gups_computed": round(kernel[kk]["kernel_gups_computed"], 2),
                       "frac_of_roofline": round(kernel[kk]["kernel_gups_computed"] / peaks[kk]["min"], 4),
                       "roofline_gups": round(peaks[kk]["min"], 1)}
                  for kk, v in forms.items()},
        "fp16_vs_fp32": (round(forms["f16"]["value"] / forms["f32"]["value"], 3)
                         if "f16" in forms and "f32" in forms else None),
        "kernel_events": {kk: {"launches": v["launches"], "kernel_ms": round(v["kernel_ms"], 3)}
                          for kk, v in kernel.items()},
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
        # per batch of 64 projections: the copy/conversion kernel into the
        # projection arrays, the block pre-pass (culling masks; centring
        # records for FP32) and the backprojection kernel; `value`'s timed
        # region is the head form's
        "gpu_launches": kernel[head]["launches"] * 3,
        "gpu_launches_by_form": {kk: v["launches"] * 3 for kk, v in kernel.items()},
        "cpu_baseline": cpu,
        "paths": {kk: path_taken.get(kk) for kk in forms},
        "brick_depth": {kk: depth_taken.get(kk) for kk in forms},
        "sizes": sizes or None,
        "reciprocal_modes": rcp_modes,
        **extra,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
