"""Benchmark: stray-field + LLG cell-updates/s of spring-pulled PMA film pairs.

Workload: two PMA films of 1024 x 256 x 2 cells (4 nm), gap 5 cells,
Ms = 1.1e6 A/m, Aex = 1.5e-11 J/m, Ku = 1e6 J/m^3 along z, alpha = 0.5, seeded
~20-cell up/down domains, slider on a spring k = 1e-3 N/m pulled at 1 m/s,
adaptive Dormand-Prince 5(4) with the displacement updated every stage.
One bench step = one accepted RK45 step of the whole path (both demag fields,
both stray fields with prefilter and tricubic gather, forces, LLG stages, slider).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torch.distributed.run: independent replicas, one per GPU
(a single film pair does not shard), timing = max over ranks.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stray-field+LLG cell-updates/s, FP32 vs mixed-prec at <=1e-4 rel L2; % HBM roof"
UNIT = "cell-updates/s"
WORKLOAD = "stick-slip PMA film pair 1024x256x2 (4 nm), gap 5, spring-pulled, adaptive DP45"
# name -> (description, builder); the thick ones plan z by FFT
WORKLOADS = {
    "stick_slip": (WORKLOAD, lambda seed: __import__("workloads").film_pair_stick_slip(seed=seed)),
    "cubes64": ("vortex cube pair 64x64x64 (2 nm), gap 3 along x, spring-pulled, adaptive DP45",
                lambda seed: __import__("workloads").cube_pair((64, 64, 64), 3, seed)),
    "films512x512x8": ("random-unit film pair 512x512x8 (4 nm), gap 1, adaptive DP45",
                       lambda seed: __import__("workloads").film_pair_plain((512, 512, 8), 1, seed)),
    "friction_pbc": ("friction films of Sec. IV.B: CoCrPt 256x256x5 (4 nm), gap 5, periodic in-plane "
                     "(2 images each side), 20-cell stripes, spring 0.005 N/m at 2 m/s, adaptive DP45",
                     lambda seed: __import__("workloads").film_pair_friction(seed=seed)),
}
TIMING_CLASSES = ["fft_x_forward", "fft_y_pass_mix_prefilter", "fft_x_inverse_prefilter",
                  "spline_gather_force", "llg_stage", "slider_reduce", "combine_normalise",
                  "fft_y_forward_thick", "fft_z_pass_thick", "fft_y_inverse_thick"]
# the same classes in the reduced-precision form (every source through the separate passes)
MIXED_CLASSES = dict(enumerate(TIMING_CLASSES))
MIXED_CLASSES.update({7: "ydft_forward_tensor", 8: "z_plane_mix", 9: "ydft_inverse_prefilter_tensor"})


BATCH_LANES = 16


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--precision", default="fp32", choices=["fp32", "mixed"],
                   help="precision of the timed context; the fp32 line also reports the mixed form beside it")
    p.add_argument("--no-mixed", action="store_true", help="fp32 line without the mixed-precision comparison")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--lanes", type=int, default=BATCH_LANES, help="streams of the batch256 workload")
    p.add_argument("--no-autotune", action="store_true",
                   help="batch256: keep the planner's model FFT plans instead of timing candidates per length")
    p.add_argument("--workload", default="stick_slip",
                   choices=sorted(WORKLOADS) + ["plain64_sweep", "cubes64_gradients", "batch256", "divcurl_sweep",
                                                "eddy_cube64"],
                   help="stick_slip (the headline workload), a thick-source workload, or the "
                        "plain 64x64x1 film pair swept over 16 sub-cell offsets (stray field only)")
    return p.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device):
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, seconds, world):
    """Units processed by all ranks per second of the slowest rank (weak scaling)."""
    return units_per_rank * steps * world / seconds


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ algorithmic bytes
def algorithmic_bytes(mm, fp, mixed=False):
    """Bytes each kernel class must move per launch (both magnets): the FP32
    classes, and with mixed=True those of the reduced-precision form that are
    not tensor-core products (whose measure is flops, dft_flops)."""
    n = [fp.n_base, fp.n_slider]
    N = [int(np.prod(x)) for x in n]
    info = [mm.plan_info(0), mm.plan_info(1)]
    # thick route (either magnet above 4 layers, and every source of the
    # reduced-precision form): y forward, z pass (direct sum up to 8 source
    # layers, else z FFT), y inverse as passes of their own
    thick = mixed or max(n[0][2], n[1][2]) > 4
    xf = yp = xi = ga = yf3 = z3 = yi3 = 0
    for s in (0, 1):
        nx, ny, nz = n[s]
        Qx, Qy = info[s]["fft"]
        kxh, kyq = Qx // 2 + 1, Qy // 2 + 1
        rx, ry, rz = info[s]["coef"]
        t = 1 - s
        x1 = 3 * nz * kxh * ny * 8
        yc = rz * kxh * ry * 8
        coef = rz * ry * rx * 4
        xf += 3 * N[s] * 4 + x1
        yp += x1 + 6 * nz * kxh * kyq * 4 + rz * nz * 3 * kxh * kyq * 4 + x1 + yc
        xi += x1 + yc + 3 * N[s] * 4 + coef
        ga += coef + 3 * N[t] * 4 + 3 * N[t] * 4
        yf3 += 24 * nz * kxh * (ny + Qy)
        Qz = info[s]["Qz"]
        if Qz == 0:  # direct z sum: Y in, N and per-box-plane S spectra, H and C spectra out
            z3 += 8 * 3 * nz * kxh * Qy + 4 * (6 * nz + 3 * nz * rz) * kxh * kyq + 8 * (3 * nz + rz) * kxh * Qy
        else:        # z FFT: Y in, H spectra out, C spectra out, N and S quarter spectra
            z3 += 2 * 24 * nz * kxh * Qy + 8 * rz * kxh * Qy + 36 * kxh * kyq * (Qz // 2 + 1)
        yi3 += 24 * nz * kxh * (Qy + ny) + 8 * rz * kxh * (Qy + ry)
    # LLG stage i reads ys, y, Hself, Hstray and k_1..k_{i-1}, writes k_i and
    # (i < 7) the next stage input; stage 7 reads k_1..k_6 for the error norm
    per_stage = []
    for i in range(1, 8):
        arrays = 4 + (i - 1) + 1 + (1 if i < 7 else 0)
        if i == 7:
            arrays = 3 + 6 + 1
        per_stage.append(arrays)
    st = sum(3 * x * 4 for x in N) * float(np.mean(per_stage[1:]))
    if mixed:
        return {0: xf, 2: xi, 3: ga, 4: st, 8: z3}
    if thick:
        return {0: xf, 2: xi, 3: ga, 4: st, 7: yf3, 8: z3, 9: yi3}
    return {0: xf, 1: yp, 2: xi, 3: ga, 4: st}


KERNEL_OF_CLASS = {0: ("k_xfwd", ["fft_passes.cu", "fft.cuh", "prefilter.cuh", "umma.cuh", "mm_internal.h"]),
                   1: ("k_ypass", ["fft_passes.cu", "fft.cuh", "prefilter.cuh", "umma.cuh", "mm_internal.h"]),
                   2: ("k_xinv", ["fft_passes.cu", "fft.cuh", "prefilter.cuh", "umma.cuh", "mm_internal.h"]),
                   3: ("k_gather", ["gather.cu", "dfloat.cuh", "spline_w.cuh", "mm_internal.h"]),
                   4: ("k_stage", ["llg.cu", "mm_internal.h"])}


def profiled_traffic(cls):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged since."""
    import hashlib
    import re
    if cls not in KERNEL_OF_CLASS:
        return None, None
    name, files = KERNEL_OF_CLASS[cls]
    path = os.path.join(ROOT, "profiles", "%s_stick_slip_1024x256x2.md" % name)
    try:
        text = open(path).read()
    except OSError:
        return None, None
    t = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    s = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    if not t or not s:
        return None, None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1801_04181_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != s.group(1):
        return None, os.path.relpath(path, ROOT) + " (stale: kernel changed since the capture)"
    return int(t.group(1)), os.path.relpath(path, ROOT)


def dft_flops(mm, fp):
    """Flops of the tensor-core y DFT classes per launch (both magnets): three
    BF16 products x 2 flops x rows x (2 Nc) x (2 Kc) of the real-form product,
    unpadded.  Forward: rows (plane, kx) = 3 nz kxh, Kc = ny, Nc = Qy; inverse:
    the demag rows (Kc = Qy, Nc = ny) and the coefficient rows (r_z kxh rows,
    Nc = r_y)."""
    fwd = inv = 0
    for s, n in enumerate((fp.n_base, fp.n_slider)):
        nz, ny = n[2], n[1]
        info = mm.plan_info(s)
        Qx, Qy = info["fft"]
        kxh = Qx // 2 + 1
        _, ry, rz = info["coef"]
        fwd += 3 * 2 * (3 * nz * kxh) * (2 * Qy) * (2 * ny)
        inv += 3 * 2 * (3 * nz * kxh) * (2 * ny) * (2 * Qy) + 3 * 2 * (rz * kxh) * (2 * ry) * (2 * Qy)
    return {7: fwd, 9: inv}


def measured_tensor_peak():
    """Dense BF16 TFLOP/s of the GB300s: the sustained figure (a kernel
    timed inside a long step), else the burst one, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            P = json.load(f)
        if "bf16_tflops_sustained" in P:
            return float(P["bf16_tflops_sustained"]), "measured (sustained)"
        return float(P["bf16_tflops"]), "measured (burst)"
    except Exception:
        return 1700.0, "fallback (sustained)"


def field_set(mm):
    """Stray fields both ways and both demag fields at the current state (host, FP64)."""
    return [mm.compute_stray_field(0).double().cpu(), mm.compute_stray_field(1).double().cpu(),
            mm.compute_demag(0).double().cpu(), mm.compute_demag(1).double().cpu()]


def run_mixed_compare(fp, m0, m1, ref_fields, steps, warmup, fp32_value):
    """The reduced-precision form on the same workload: throughput, its field
    error against the FP32 path at the same initial state, and the tensor
    roofline of its DFT kernel classes."""
    import torch
    from paper_1801_04181_gb300 import MMError
    from paper_1801_04181_gb300 import pair_context as gpu_pair

    if max(fp.n_base[2], fp.n_slider[2]) > 8:
        return {"unavailable": "the reduced-precision form takes sources of at most 8 layers"}
    try:
        mm = gpu_pair(fp, m0, m1, adaptive=True, rtol=1e-5, precision="mixed")
        got = field_set(mm)
    except MMError as e:
        return {"unavailable": str(e)}
    names = ["H_stray_base_to_slider", "H_stray_slider_to_base", "H_demag_base", "H_demag_slider"]
    err = {k: float((a - b).norm() / b.norm()) for k, a, b in zip(names, got, ref_fields)}
    dt = 1e-13
    for _ in range(max(warmup, 3)):
        _, dt = mm.step(1, dt)
    mm.set_timing(False)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        _, dt = mm.step(1, dt)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    mm.reset_timing()
    mm.set_timing(True)
    for _ in range(max(1, min(steps, 20))):
        _, dt = mm.step(1, dt)
    torch.cuda.synchronize()
    mm.set_timing(False)
    kt = {c: mm.timing(c) for c in range(len(TIMING_CLASSES))}
    flops = dft_flops(mm, fp)
    peak, src = measured_tensor_peak()
    tensor = {}
    for c, f in flops.items():
        tot, nl = kt[c]
        if nl:
            avg = tot / nl / 1e3
            tensor[MIXED_CLASSES[c]] = {"achieved": round(f / avg / 1e12, 1), "peak": peak, "peak_source": src,
                                         "unit": "TFLOP/s", "frac": round(f / avg / 1e12 / peak, 4),
                                         "flops_per_launch": int(f), "avg_launch_ms": round(avg * 1e3, 5)}
    value = fp.cells() * steps / (ms / 1e3)
    mm.close()
    return {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "vs_fp32": round(value / fp32_value, 4),
            "dtype": "split-bf16 (hi.hi + hi.lo + lo.hi) tensor-core y DFTs, f32 accumulation; rest f32",
            "rel_l2_vs_fp32": err,
            "roofline": {"bound": "tensor", "kernels": tensor},
            "kernel_times": {MIXED_CLASSES[c]: {"ms": round(kt[c][0], 3), "launches": kt[c][1]}
                             for c in kt if kt[c][1]}}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            P = json.load(f)
        return float(P["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle sample
# A bounded sample of one Dormand-Prince step of the oracle: one stray-field
# direction (potential on the box by linear convolution, banded prefilter,
# 64-term evaluation, force) plus one self-demag field, i.e. half of one field
# evaluation; a step makes six evaluations, so the sample is 1/12 of a step.
# The kernel windows are set-up, computed beforehand by the process pool and
# handed to the workers through shared memory.
SAMPLE_SHARE = 12


def _oracle_sample(fp, m0, m1, S, N):
    from oracle import fields as OF
    from oracle.interaction import stray_interaction

    box_lo, box_dims = OF.box_for_target(fp.n_slider, fp.offsets[1], fp.offsets[0], fp.u0, True)
    key = ("S", (3,) + tuple(reversed(fp.n_base)), tuple(fp.cell), tuple(box_lo), tuple(box_dims))
    t0 = time.perf_counter()
    stray_interaction(fp.mat_base.Ms * m0, fp.mat_slider.Ms * m1, fp.cell, fp.offsets[0], fp.offsets[1],
                      fp.u0, True, kernel_cache={key: S})
    OF.demag_conv(fp.mat_base.Ms * m0, fp.cell, kernel=N)
    return time.perf_counter() - t0


def _oracle_sample_task(job):
    """One oracle sample in a pool worker, its windows attached from shared memory."""
    from multiprocessing import shared_memory

    fp, m0, m1, (s_name, s_shape), (n_name, n_shape) = job
    blocks = [shared_memory.SharedMemory(name=s_name), shared_memory.SharedMemory(name=n_name)]
    try:
        S = np.ndarray(s_shape, dtype=np.float64, buffer=blocks[0].buf)
        N = np.ndarray(n_shape, dtype=np.float64, buffer=blocks[1].buf)
        t = _oracle_sample(fp, m0, m1, S, N)
        del S, N
        return t
    finally:
        for b in blocks:
            b.close()


class OracleSampler:
    """Times the oracle on the bounded sample: in this process (one thread) and
    as one concurrent sample per worker of a spawn pool (all host cores)."""

    def __init__(self, fp, m0, m1, pool, workers):
        from multiprocessing import shared_memory

        from oracle import fields as OF
        from oracle.fields import kernel_windows_pooled

        self.fp, self.m0, self.m1, self.pool, self.workers = fp, m0, m1, pool, workers
        box_lo, box_dims = OF.box_for_target(fp.n_slider, fp.offsets[1], fp.offsets[0], fp.u0, True)
        S, N = kernel_windows_pooled(fp.n_base, fp.cell, box_lo, box_dims, pool)
        self.blocks, self.views = [], []
        for a in (S, N):
            b = shared_memory.SharedMemory(create=True, size=a.nbytes)
            v = np.ndarray(a.shape, dtype=np.float64, buffer=b.buf)
            v[...] = a
            self.blocks.append(b)
            self.views.append(v)
        self.job = (fp, m0, m1, (self.blocks[0].name, S.shape), (self.blocks[1].name, N.shape))

    def single(self):
        """Seconds of one sample on one thread."""
        return _oracle_sample(self.fp, self.m0, self.m1, *self.views)

    def concurrent(self):
        """Wall seconds of `workers` samples run at once, one per worker."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_sample_task, [self.job] * self.workers, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.views = []
        for b in self.blocks:
            b.close()
            b.unlink()
        self.blocks = []

    def describe(self):
        return "one stray-field direction + one self-demag of the %dx%dx%d pair (1/%d of a DP45 step: " \
               "6 field evaluations x 2 halves); kernel windows precomputed as set-up" % \
               (tuple(self.fp.n_base) + (SAMPLE_SHARE,))


def oracle_pool_size():
    return max(1, min(64, os.cpu_count() or 1))


def cpu_oracle_sample(fp, m0, m1, pool, workers):
    """cpu_baseline entry: the oracle on all `workers` host cores (concurrent
    samples, one per core) and on one thread, scaled to cell-updates/s."""
    smp = OracleSampler(fp, m0, m1, pool, workers)
    try:
        t1 = smp.single()
        tw = smp.concurrent()
    finally:
        smp.close()
    cells = fp.cells()
    return {"value": workers * cells / (SAMPLE_SHARE * tw), "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": smp.describe() + "; %d concurrent samples (one per core) in %.1f s" % (workers, tw),
            "sample_seconds": tw,
            "single_thread": {"value": cells / (SAMPLE_SHARE * t1), "cores": 1, "sample_seconds": t1}}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import workloads
    from paper_1801_04181_gb300 import pair_context as gpu_pair

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    cpu_base = None
    pool = None
    # the CPU sample times the open-boundary oracle: periodic workloads report none
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload != "friction_pbc":
        # start the oracle's process pool before the first GPU call
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(oracle_pool_size())

    wl_name, wl_make = WORKLOADS[args.workload]
    fp, m0, m1 = wl_make(args.seed + 101 * rank)
    mm = gpu_pair(fp, m0, m1, adaptive=True, rtol=1e-5, precision=args.precision)
    cells = fp.cells()
    # fields at the initial state, for the mixed form's error beside this line
    want_mixed = args.precision == "fp32" and not args.no_mixed and rank == 0 and world == 1
    ref_fields = field_set(mm) if want_mixed else None
    stream = torch.cuda.current_stream()
    dt = 1e-13
    for _ in range(max(args.warmup, 3)):
        _, dt = mm.step(1, dt)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    # the timed region runs without the per-launch event pairs (they cost ~5%
    # of a step in host overhead); kernel times come from a separate run below
    mm.set_timing(False)
    launches0 = mm.launch_count()
    acc0, rej0 = mm.step_stats()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        _, dt = mm.step(1, dt)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = mm.launch_count() - launches0
    acc1, rej1 = mm.step_stats()
    clk = clocks.stop()
    # per-kernel times: CUDA events around every launch, on the library stream
    mm.reset_timing()
    mm.set_timing(True)
    for _ in range(max(1, min(args.steps, 50))):
        _, dt = mm.step(1, dt)
    torch.cuda.synchronize()
    mm.set_timing(False)
    kt = {c: mm.timing(c) for c in range(len(TIMING_CLASSES))}
    ms = max_over_ranks(ms, world, "cuda")
    value = whole_job_rate(cells, args.steps, ms / 1e3, world)

    # end to end through the public API with host buffers: upload m, step, read m + force
    pin = [torch.empty(mm.shapes[g], dtype=torch.float32).pin_memory() for g in (0, 1)]
    out = [torch.empty(mm.shapes[g], dtype=torch.float32).pin_memory() for g in (0, 1)]
    for g in (0, 1):
        mm.download_magnetization(g, pin[g])
    k_e2e = max(1, min(args.steps, 50))
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        for g in (0, 1):
            mm.upload_magnetization(g, pin[g])
        _, dt = mm.step(1, dt)
        for g in (0, 1):
            mm.download_magnetization(g, out[g])
        mm.get_force(1)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e = whole_job_rate(cells, k_e2e, e2e_s, world)
    h2d = sum(int(np.prod(mm.shapes[g])) * 4 for g in (0, 1))

    # power bookkeeping at the final state (one field evaluation, the torque
    # with H_eff and the |m x H_eff|^2 sums), host-timed around the call
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pw = mm.power()
    power = {"P_in_W": pw["P_in"], "P_diss_W": pw["P_diss"], "P_visc_W": pw["P_visc"],
             "ms": round((time.perf_counter() - t0) * 1e3, 3),
             "what": "mm_get_power at the final state: P_in = -F.v_s, Gilbert dissipation per magnet, "
                     "viscous drive loss"}

    # roofline of the dominant kernel class
    ab = algorithmic_bytes(mm, fp, mixed=args.precision == "mixed")
    dom = max(ab.keys(), key=lambda c: kt[c][0])
    tot_ms, nl = kt[dom]
    avg_s = tot_ms / max(nl, 1) / 1e3
    peak, src = measured_peaks()
    achieved = ab[dom] / avg_s / 1e9
    traffic, traffic_src = profiled_traffic(dom) if args.workload == "stick_slip" else (None, None)
    roof = {"bound": "hbm", "kernel": TIMING_CLASSES[dom], "achieved": round(achieved, 1),
            "peak": peak, "peak_source": src, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "algorithmic_bytes_per_launch": int(ab[dom]), "avg_launch_ms": round(avg_s * 1e3, 5),
            "traffic": traffic, "traffic_source": traffic_src}
    if args.precision == "mixed":
        # the dominant tensor-core DFT class against the BF16 tensor peak
        fl = dft_flops(mm, fp)
        dom = max(fl.keys(), key=lambda c: kt[c][0])
        tot_ms, nl = kt[dom]
        avg_s = tot_ms / max(nl, 1) / 1e3
        tpk, tsrc = measured_tensor_peak()
        roof = {"bound": "tensor", "kernel": MIXED_CLASSES[dom], "achieved": round(fl[dom] / avg_s / 1e12, 1),
                "peak": tpk, "peak_source": tsrc, "unit": "TFLOP/s",
                "frac": round(fl[dom] / avg_s / 1e12 / tpk, 4), "flops_per_launch": int(fl[dom]),
                "avg_launch_ms": round(avg_s * 1e3, 5), "traffic": None}
    names = MIXED_CLASSES if args.precision == "mixed" else dict(enumerate(TIMING_CLASSES))
    ktab = {}
    for c in kt:
        if not kt[c][1]:
            continue
        e = {"ms": round(kt[c][0], 3), "launches": kt[c][1]}
        if c in ab:  # the FP32 classes with a byte model: per-launch HBM roofline
            avg = kt[c][0] / kt[c][1] / 1e3
            e.update({"algorithmic_bytes_per_launch": int(ab[c]), "achieved_GBs": round(ab[c] / avg / 1e9, 1),
                      "frac": round(ab[c] / avg / 1e9 / peak, 4)})
        ktab[names[c]] = e
    fft_cmp = cufft_compare(mm, fp, kt) if args.workload == "stick_slip" and args.precision == "fp32" else None
    mixed = None
    if want_mixed:
        mixed = run_mixed_compare(fp, m0, m1, ref_fields, max(1, min(args.steps, 50)), args.warmup, value)
    if pool is not None:
        try:
            cpu_base = cpu_oracle_sample(fp, m0, m1, pool, oracle_pool_size())
        finally:
            pool.close()
            pool.join()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "split-bf16 tensor-core y DFTs + f32",
            "data": "synthetic",
            "config": {"workload": wl_name, "cells": cells, "precision": args.precision,
                       "fft": [list(mm.plan_info(0)["fft"]) + [mm.plan_info(0)["Qz"]]],
                       "adaptive_rtol": 1e-5, "accepted": acc1 - acc0, "rejected": rej1 - rej0,
                       "dt_final_s": dt, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "no flush: per-step working set (~0.4 GB of spectra, kernels and RK "
                             "arrays) exceeds the 129 MB L2"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d + 32,
                    "steps": k_e2e},
            "gpu_launches": int(launches),
            "roofline": roof,
            "kernel_times": ktab,
            "cufft_compare": fft_cmp,
            "mixed": mixed,
            "power": power,
            "clocks": clk,
            "cpu_baseline": cpu_base,
        }
        print(json.dumps(line))
    mm.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cufft_compare(mm, fp, kt, reps=20):
    """cuFFT (through torch.fft) on the same grid, as a timed comparison only.

    R2C of the source planes of both magnets and C2R of their output planes on
    the zero-padded Qx x Qy grid: the bare transforms, with neither the
    spectral products nor the prefilters that our three FFT passes also do.
    """
    import torch
    info = [mm.plan_info(0), mm.plan_info(1)]
    Qx, Qy = info[0]["fft"]
    if info[0]["Qz"] or info[1]["Qz"]:
        return None
    nx, ny, nz = fp.n_base
    n_in = 2 * 3 * nz
    n_out = 2 * 3 * nz + info[0]["coef"][2] + info[1]["coef"][2]
    x = torch.zeros((n_in, Qy, Qx), device="cuda")
    x[:, :ny, :nx] = torch.randn((n_in, ny, nx), device="cuda")
    Xo = torch.randn((n_out, Qy, Qx // 2 + 1), device="cuda", dtype=torch.complex64)
    for _ in range(3):
        torch.fft.rfft2(x)
        torch.fft.irfft2(Xo, s=(Qy, Qx))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        torch.fft.rfft2(x)
        torch.fft.irfft2(Xo, s=(Qy, Qx))
    e1.record()
    torch.cuda.synchronize()
    ours = sum(kt[c][0] / max(kt[c][1], 1) for c in (0, 1, 2))
    return {"cufft_ms_per_evaluation": round(e0.elapsed_time(e1) / reps, 4),
            "ours_ms_per_evaluation": round(ours, 4),
            "what": "cuFFT R2C of %d planes + C2R of %d planes on %dx%d (bare transforms) vs "
                    "our x-forward, y and x-inverse passes (transforms + spectral products + "
                    "prefilters)" % (n_in, n_out, Qx, Qy)}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores.

    One reference step = one round of concurrent bounded samples, one per
    core (each 1/12 of a DP45 step of the stick-slip pair); the steps are
    capped so the run ends within a few minutes, and the line reports the
    steps actually timed with their measured time per step."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import multiprocessing as mp

    import workloads

    fp, m0, m1 = workloads.film_pair_stick_slip(seed=args.seed)
    nw = min(args.warmup, 1)
    ns = max(1, min(args.steps, 3))
    workers = oracle_pool_size()
    pool = mp.get_context("spawn").Pool(workers)
    try:
        smp = OracleSampler(fp, m0, m1, pool, workers)
        try:
            for _ in range(nw):
                smp.concurrent()
            t0 = time.perf_counter()
            for _ in range(ns):
                smp.concurrent()
            wall = time.perf_counter() - t0
            desc = smp.describe()
        finally:
            smp.close()
    finally:
        pool.close()
        pool.join()
    step_s = wall / ns
    v = workers * fp.cells() / SAMPLE_SHARE / step_s
    sample = desc + "; one step = %d concurrent samples (one per core)" % workers
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": ns, "warmup": nw, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": fp.cells(),
                       "step": "%d/%d of a DP45 step of the pair (one bounded sample per core)"
                               % (workers, SAMPLE_SHARE)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_sweep(args):
    """Plain film pair 64x64x1 (4 nm, gap 1, random unit m), the slider displaced
    along x by 16 evenly spaced offsets in [0, 1) cell: both stray-field
    directions with their forces per offset.  Metric: stray-field
    cell-evaluations/s = 2 N offsets / time (no LLG in this workload)."""
    import torch
    import workloads
    from paper_1801_04181_gb300 import pair_context as gpu_pair

    fp, m0, m1 = workloads.film_pair_plain((64, 64, 1), 1, args.seed)
    mm = gpu_pair(fp, m0, m1, mech=False)
    offs = [k / 16.0 for k in range(16)]

    def sweep():
        for u in offs:
            mm.set_displacement((u * fp.cell[0], 0.0, 0.0))
            mm.compute_stray_field(0)
            mm.compute_stray_field(1)

    for _ in range(max(args.warmup, 3)):
        sweep()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = mm.launch_count()
    e0.record()
    for _ in range(args.steps):
        sweep()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cells = fp.cells()
    line = {"metric": "stray-field cell-evaluations/s (plain 64x64x1 pair, 16 offsets)",
            "value": cells * len(offs) * args.steps / (ms / 1e3), "unit": "cell-evaluations/s",
            "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "plain film pair 64x64x1 (4 nm), gap 1, 16 x-offsets in [0, 1)",
                       "cells": cells, "fft": [mm.plan_info(0)["fft"]],
                       "step": "one sweep: 16 offsets x both stray-field directions",
                       "l2": "L2-resident: a launch- and latency-bound workload"},
            "gpu_launches": int(mm.launch_count() - launches0)}
    print(json.dumps(line))
    mm.close()


def run_divcurl(args):
    """Sec. IV.A: a frozen random base film 64x64x4 (4 nm), the slider film
    above it (gap 1) moved along x by 16 partial offsets in [0, 1) cell; per
    offset the base's stray field inside the slider (potential, prefilter,
    gather) and its divergence and curl means D(x), C(x) by central
    differences.  Reported: D(x)/D(0) - 1 and C(x)/C(0) - 1, the paper's
    measure of what the interpolation does to div and curl; timed: offsets
    per second (field + diagnostics, one synchronisation per offset)."""
    import torch
    import workloads
    from paper_1801_04181_gb300 import pair_context as gpu_pair

    fp, m0, m1 = workloads.film_pair_plain((64, 64, 4), 1, args.seed)
    mm = gpu_pair(fp, m0, m1, mech=False)
    offs = [k / 16.0 for k in range(16)]

    def sweep():
        out = []
        for u in offs:
            mm.set_displacement((u * fp.cell[0], 0.0, 0.0))
            H = mm.compute_stray_field(0)
            out.append(mm.div_curl(H, fp.cell))
        return out

    for _ in range(max(args.warmup, 3)):
        sweep()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dc = sweep()
    torch.cuda.synchronize()
    s = time.perf_counter() - t0
    D0, C0 = dc[0]
    # the paper's reference comparison (Sec. IV.A), outside the timed sweep:
    # linear interpolation of the field vectors between the two whole-cell
    # positions, (1 - x) H(0) + x H(1), blended by torch from two library
    # evaluations and judged by the same D, C
    mm.set_displacement((0.0, 0.0, 0.0))
    H0 = mm.compute_stray_field(0)
    mm.set_displacement((fp.cell[0], 0.0, 0.0))
    H1 = mm.compute_stray_field(0)
    lin = [mm.div_curl(((1.0 - u) * H0 + u * H1).contiguous(), fp.cell) for u in offs]
    # the four-point difference variant of the gradient, judged against its own x = 0
    fd4 = []
    for u in offs:
        mm.set_displacement((u * fp.cell[0], 0.0, 0.0))
        fd4.append(mm.div_curl(mm.compute_stray_field_fd4(0), fp.cell))
    # the paper's second method, direct componentwise interpolation of the
    # tensor field, judged against its own stationary (x = 0, node) field
    cw = []
    for u in offs:
        mm.set_displacement((u * fp.cell[0], 0.0, 0.0))
        cw.append(mm.div_curl(mm.compute_stray_field_componentwise(0), fp.cell))
    line = {"metric": "div/curl diagnostic offsets/s (frozen random base 64x64x4, 16 partial moves)",
            "value": len(offs) * args.steps / s, "unit": "offsets/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "random-unit film pair 64x64x4 (4 nm), gap 1, slider moved by x in [0, 1)",
                       "step": "one sweep: 16 offsets x (stray field of the base in the slider + D, C)"},
            "div_curl": {"x": offs, "D0": D0, "C0": C0,
                         "D_rel": [d / D0 - 1.0 for d, _ in dc], "C_rel": [c / C0 - 1.0 for _, c in dc],
                         "linear_D_rel": [d / D0 - 1.0 for d, _ in lin],
                         "linear_C_rel": [c / C0 - 1.0 for _, c in lin],
                         "fd4_D0": fd4[0][0], "fd4_C0": fd4[0][1],
                         "fd4_D_rel": [d / fd4[0][0] - 1.0 for d, _ in fd4],
                         "fd4_C_rel": [c / fd4[0][1] - 1.0 for _, c in fd4],
                         "componentwise_D0": cw[0][0], "componentwise_C0": cw[0][1],
                         "componentwise_D_rel": [d / cw[0][0] - 1.0 for d, _ in cw],
                         "componentwise_C_rel": [c / cw[0][1] - 1.0 for _, c in cw]}}
    print(json.dumps(line))
    mm.close()


def run_gradients(args):
    """Two 64^3 vortex cubes (2 nm, gap 3 along x, slider at 1.7 cells): one
    step is mm_backward_energy of the slider's energy in the base's field --
    the forward stray field and force plus the transposed path giving
    dE/dm of both cubes and dE/du.  Metric: cells of both cubes / time."""
    import torch
    import workloads
    from paper_1801_04181_gb300 import pair_context as gpu_pair

    fp, m0, m1 = workloads.cube_pair((64, 64, 64), 3, args.seed)
    fp.u0 = (1.7, 0.0, 0.0)
    mm = gpu_pair(fp, m0, m1, mech=False)
    for _ in range(max(args.warmup, 3)):
        mm.backward_energy(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mm.backward_energy(0)
    torch.cuda.synchronize()
    s = time.perf_counter() - t0
    cells = fp.cells()
    line = {"metric": "energy-gradient cell-evaluations/s (forward + adjoint, 64^3 cube pair)",
            "value": cells * args.steps / s, "unit": "cell-evaluations/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "vortex cube pair 64x64x64 (2 nm), gap 3 along x, u = 1.7 cells",
                       "cells": cells, "fft": [list(mm.plan_info(0)["fft"]) + [mm.plan_info(0)["Qz"]]],
                       "step": "mm_backward_energy(src=0): stray field, force, dE/dm (both), dE/du; "
                               "host-timed, one synchronisation per step"}}
    print(json.dumps(line))
    mm.close()


def run_eddy(args):
    """Eddy currents of a conducting 64^3 vortex cube (2 nm, Sec. III.B): one
    step is mm_eddy_field -- E_sol and H_eddy by cross products with S
    through the potential path, the electric potential by FP64 SOR to 1e-9 of
    its source, the current.  Drive: dB/dt = mu0 Ms dm/dt of the cube's own
    LLG motion at the seeded state (the rate of its demag field left out),
    sigma = 1e6 S/m.  Metric: cells / time (host-timed, one synchronisation
    per call, the SOR convergence checks included)."""
    import torch
    import workloads
    from paper_1801_04181_gb300 import pair_context as gpu_pair

    fp, m0, m1 = workloads.cube_pair((64, 64, 64), 3, args.seed)
    mm = gpu_pair(fp, m0, m1, mech=False)
    dm, _ = mm.compute_torque(0)
    mu0 = 4e-7 * np.pi
    dB = (mu0 * fp.mat_base.Ms * dm).contiguous()
    sigma = 1e6
    sweeps = 0
    for _ in range(max(args.warmup, 3)):
        _, _, sweeps = mm.eddy_field(0, dB, sigma)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, _, sweeps = mm.eddy_field(0, dB, sigma)
    torch.cuda.synchronize()
    s = time.perf_counter() - t0
    N = int(np.prod(fp.n_base))
    line = {"metric": "eddy-field cell-evaluations/s (64^3 conducting vortex cube)",
            "value": N * args.steps / s, "unit": "cell-evaluations/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (electric potential f64)", "data": "synthetic",
            "config": {"workload": "vortex cube 64x64x64 (2 nm), dB/dt = mu0 Ms dm/dt, sigma = 1e6 S/m",
                       "cells": N, "sor_sweeps": sweeps,
                       "step": "mm_eddy_field: 6 potential-path passes, SOR, current; host-timed"}}
    print(json.dumps(line))
    mm.close()


def batch_cost(fp):
    """Cost model for spreading pairs: grid area x (source layers + box layers)."""
    return fp.n_base[0] * fp.n_base[1] * (fp.n_base[2] + 4)


def batch_shard(specs, world, rank, lanes):
    """This rank's pairs (longest processing time first over the ranks) and
    their lane streams (the same rule over the rank's lanes)."""
    from paper_1801_04181_gb300 import assign_lanes

    cost = [batch_cost(fp) for fp in specs]
    mine = [i for i, r in enumerate(assign_lanes(cost, world)) if r == rank]
    return mine, assign_lanes([cost[i] for i in mine], lanes)


def run_batch(args):
    """256 independent spring-pulled PMA film pairs of uneven sizes (nx in
    64..512, ny in 64..256, nz in 1..4, slider displaced by U[0, 50) cells,
    pulled at U[0.1, 10] m/s), spread over --lanes streams (16) by longest
    processing time first; one bench step = one mm_step_batch call in which
    every pair takes one accepted adaptive DP45 step.  Metric: cells of all
    pairs x steps / time.  Under torchrun the pairs are spread over the ranks
    the same way (strong scaling: the batch is fixed)."""
    import torch
    import workloads
    from paper_1801_04181_gb300 import step_batch
    from paper_1801_04181_gb300 import pair_context as gpu_pair

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(oracle_pool_size())
    specs = workloads.batch_pairs(256, seed=args.seed)
    mine, lanes = batch_shard(specs, world, rank, args.lanes)
    streams = [torch.cuda.Stream() for _ in range(args.lanes)]
    t_setup = time.perf_counter()
    batch = []
    for i, l in zip(mine, lanes):
        m0, m1 = workloads.batch_patterns(specs[i])
        batch.append(gpu_pair(specs[i], m0, m1, adaptive=True, rtol=1e-5, stream=streams[l],
                              precision=args.precision))
    cells = sum(specs[i].cells() for i in mine)
    # the project's autotuner: candidate radix orders per transform length,
    # timed on the pairs themselves (a length is timed once, then shared)
    tune = {"enabled": not args.no_autotune, "lengths_timed": 0, "seconds": 0.0}
    if not args.no_autotune:
        t_tune = time.perf_counter()
        for mm in batch:
            tune["lengths_timed"] += mm.autotune(candidates=4, reps=2)
        torch.cuda.synchronize()
        tune["seconds"] = round(time.perf_counter() - t_tune, 2)
    dts = [1e-13] * len(batch)
    for _ in range(max(args.warmup, 3)):
        _, dts = step_batch(batch, 1, dts)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for mm in batch:
        mm.set_timing(False)
    cur = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = sum(mm.launch_count() for mm in batch)
    st0 = [mm.step_stats() for mm in batch]
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(cur)
    for s in streams:
        s.wait_event(ev0)
    for _ in range(args.steps):
        _, dts = step_batch(batch, 1, dts)
    for s in streams:
        cur.wait_stream(s)
    ev1.record(cur)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = sum(mm.launch_count() for mm in batch) - launches0
    st1 = [mm.step_stats() for mm in batch]
    acc = sum(b[0] - a[0] for a, b in zip(st0, st1))
    rej = sum(b[1] - a[1] for a, b in zip(st0, st1))
    # modelled bytes per batched step: each pair's per-launch bytes x its launches per step
    k_t = max(1, min(args.steps, 10))
    for mm in batch:
        mm.reset_timing()
        mm.set_timing(True)
    for _ in range(k_t):
        _, dts = step_batch(batch, 1, dts)
    torch.cuda.synchronize()
    bytes_step = 0.0
    flops_step = 0.0  # reduced precision: split-product flops of the tensor-core DFTs
    for i, mm in zip(mine, batch):
        ab = algorithmic_bytes(mm, specs[i], mixed=args.precision == "mixed")
        for c, b in ab.items():
            bytes_step += b * mm.timing(c)[1] / k_t
        if args.precision == "mixed":
            for c, f in dft_flops(mm, specs[i]).items():
                flops_step += f * mm.timing(c)[1] / k_t
        mm.set_timing(False)
    ms = max_over_ranks(ms, world, "cuda")
    total_cells = sum(fp.cells() for fp in specs)  # every rank's pairs together
    value = total_cells * args.steps / (ms / 1e3)
    # end to end through the public API: upload m of every pair from pinned
    # host memory, step the batch, download m and read the slider force
    pin = [[torch.empty(mm.shapes[g], dtype=torch.float32).pin_memory() for g in (0, 1)] for mm in batch]
    for mm, p in zip(batch, pin):
        for g in (0, 1):
            mm.download_magnetization(g, p[g])
    k_e2e = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        for mm, p in zip(batch, pin):
            for g in (0, 1):
                mm.upload_magnetization(g, p[g])
        _, dts = step_batch(batch, 1, dts)
        for mm, p in zip(batch, pin):
            for g in (0, 1):
                mm.download_magnetization(g, p[g])
            mm.get_force(1)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e = total_cells * k_e2e / e2e_s
    h2d = sum(int(np.prod(mm.shapes[g])) * 4 for mm in batch for g in (0, 1))
    peak, src = measured_peaks()
    achieved = bytes_step / (ms / args.steps / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": "whole batched step (all kernel classes of all pairs, concurrent)",
            "achieved": round(achieved, 1), "peak": peak, "peak_source": src, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "algorithmic_bytes_per_step": int(bytes_step),
            "traffic": None,
            "traffic_source": "not captured: a batched step is thousands of concurrent launches"}
    if args.precision == "mixed":
        tpk, tsrc = measured_tensor_peak()
        rate = flops_step / (ms / args.steps / 1e3) / 1e12
        roof["tensor"] = {"what": "split-product flops of the tensor-core y DFTs of all pairs per batched step "
                                  "/ step time", "achieved": round(rate, 1), "peak": tpk, "peak_source": tsrc,
                          "unit": "TFLOP/s", "frac": round(rate / tpk, 4), "flops_per_step": int(flops_step)}
        roof["algorithmic_bytes_note"] = "FP32 classes only (the tensor-core DFT and split passes not counted)"
    cpu_base = None
    if pool is not None:
        try:
            mid = int(np.argsort([fp.cells() for fp in specs])[len(specs) // 2])
            m0, m1 = workloads.batch_patterns(specs[mid])
            cpu_base = cpu_oracle_sample(specs[mid], m0, m1, pool, oracle_pool_size())
            cpu_base["sample"] += "; the median-size pair of the batch"
        finally:
            pool.close()
            pool.join()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "split-bf16 tensor-core y DFTs + f32",
            "data": "synthetic",
            "config": {"precision": args.precision,
                       "workload": "batch of 256 PMA film pairs, sizes U{64..512}xU{64..256}xU{1..4} "
                                   "(4 nm), slider at U[0, 50) cells, pulled at U[0.1, 10] m/s, "
                                   "adaptive DP45 per pair",
                       "pairs": len(batch), "cells": cells, "lanes": args.lanes,
                       "accepted": acc, "rejected": rej, "setup_s": round(t_setup, 1), "autotune": tune,
                       "parallelism": "pairs over ranks" if world > 1 else "single",
                       "l2": "no flush: the batch's working set (tens of GB) exceeds the 129 MB L2"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": h2d + 32 * len(batch), "steps": k_e2e},
            "gpu_launches": int(launches),
            "roofline": roof,
            "clocks": clk,
            "cpu_baseline": cpu_base,
        }
        print(json.dumps(line))
    for mm in batch:
        mm.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "plain64_sweep":
        run_sweep(args)
    elif args.workload == "cubes64_gradients":
        run_gradients(args)
    elif args.workload == "batch256":
        run_batch(args)
    elif args.workload == "divcurl_sweep":
        run_divcurl(args)
    elif args.workload == "eddy_cube64":
        run_eddy(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
