"""Benchmark: block orthogonalization (TreeTSPQR, locally orthogonal basis) on GB300.

Default workload (the headline): one restart cycle of block GMRes with the
2D 5-point Dirichlet Laplacian on a 1024 x 1024 grid (n = 1,048,576), s = 8
right-hand sides U(-1, 1), restart m = 30 blocks: 31 orthogonalizations
(k = 0, 8, ..., 240 prior columns), then the correction Y = V C through
apply_Q.  The stencil and the small host least-squares solve sit outside the
timed region; the orthogonalization and apply_Q kernels are timed with CUDA
events on the basis stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lo|reference]

One JSON line on rank 0.  A "step" is one restart cycle.  `value` is
algorithmic GB/s of the hot path: per orthogonalization
8nK + 8nK + 8ns + 8ns + 4pk^2 + 8pKs bytes (K = k + s, p chunks), per apply_Q
8nk + 8nm + 4pk^2.  Multi-GPU runs are independent replicas (the method has
no exchange step on one GPU per problem): value = bytes of all ranks / max time.
"""

import os

# The CPU baseline (the oracle) is timed single-threaded: fix BLAS threads
# before numpy is imported anywhere.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "block-orth GB/s vs HBM peak; mixed vs FP64 speedup at ‖QᵀQ−I‖≤1e-12"
NX = NY = 1024
S = 8
M_RESTART = 30
CHUNK = 8192   # chunk rows of the cycle's basis: lo_tune_chunk_rows' choice on GB300 (4096: 1.5 % slower)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz
# The translation unit (with the headers it includes) of each kernel whose DRAM
# traffic was captured: a change to any of these files invalidates the capture.
KERNEL_TU = {
    "tc_step": ["paper_2204_13393_gb300/csrc/lo_umma.cu", "paper_2204_13393_gb300/csrc/lo_ozaki.cu",
                "paper_2204_13393_gb300/csrc/lo_oz_common.cuh", "paper_2204_13393_gb300/csrc/lo_recombine.h",
                "paper_2204_13393_gb300/csrc/lo_internal.h", "include/lo.h"],
}
# DRAM bytes of one step's launches of each kernel group from one ncu capture
# (bench.py --case profile: n = 2^20, s = 8, k = 120, 8192-row chunks, two local
# passes), with that group's algorithmic bytes in the same step, keyed by
# (kernel group, precision); "src" is the sha256 prefix of the translation
# units (comments stripped) when the counters were taken.  The reported
# traffic scales the measured ratio to the average launch group of the cycle;
# a code change in those units invalidates the entry (traffic: null).
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
#       --clock-control none --profile-from-start off python bench.py --case profile
TRAFFIC = {
    # k_oz_coef<8,1,1> + k_umma_update<8,1> (the iterate) + k_umma_gram<8,7> (its Gram), and the
    # pass-3 launches that exit at once; algorithmic 16nK + 8ns
    ("refine", "fp64_tc"): {"kernel": "tc_step", "src": "16fbce56b5ce6596",
                            "dram_bytes": 3781129728 + 92645376, "algorithmic_bytes": 2214592512},
    # k_oz_coef<8,2,1> + k_umma_update<8,2>; algorithmic 8nK + 16ns + 8pKs
    ("update", "fp64_tc"): {"kernel": "tc_step", "src": "16fbce56b5ce6596",
                            "dram_bytes": 1952426752 + 122739456, "algorithmic_bytes": 1209008128},
    # k_umma_srcexp<8> + k_umma_gram<8,7> (pass 1); algorithmic 8nK
    ("gram", "fp64_tc"): {"kernel": "tc_step", "src": "16fbce56b5ce6596",
                          "dram_bytes": 1897126912 + 30527488, "algorithmic_bytes": 1073741824},
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def peaks_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def orth_bytes(n, s, k, p):
    K = k + s
    return 16 * n * K + 16 * n * s + 4 * p * k * k + 8 * p * K * s


def apply_bytes(n, k, m, p):
    return 8 * n * k + 8 * n * m + 4 * p * k * k


def update_bytes_flops(n, s, k, p):
    """Algorithmic bytes and float64 flops of one stage-2 (assembly) launch."""
    K = k + s
    return 8 * n * K + 16 * n * s + 8 * p * K * s, n * (4 * k * s + 2 * s * s)


def gram_bytes_flops(n, s, k):
    return 8 * n * (k + s), 2 * n * (k + s) * s


def refine_bytes_flops(n, s, k, passes):
    """Bytes and float64 flops the reiteration passes of one step must move and
    do (BCGS-PIP+, Alg. 8): per pass >= 2 the iterate Y = (A - Q P) N^{-1} reads
    [Q A] and writes Y (8nK + 8ns), and its Gram [Q Y]^T Y reads [Q Y] (8nK)."""
    K = k + s
    extra = max(0, int(passes) - 1)
    return extra * (16 * n * K + 8 * n * s), extra * (4 * n * K * s)


def strip_comments(text):
    """C/C++ source without its comments, with every run of whitespace outside
    string and character literals as one space (the literals kept as they
    are), so that a comment- or layout-only edit does not invalidate a capture."""
    out, i, n = [], 0, len(text)
    space = False
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            if space:
                out.append(" ")
                space = False
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
            space = True
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            space = True
        elif c.isspace():
            space = True
            i += 1
        else:
            if space:
                out.append(" ")
                space = False
            out.append(c)
            i += 1
    return "".join(out).strip()


def src_hash(kernel):
    """sha256 prefix of the kernel's translation unit, comments stripped."""
    h = hashlib.sha256()
    for rel in KERNEL_TU[kernel]:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def traffic_capture(group, precision):
    """The ncu capture of this kernel group's dominant kernel, if its sources are unchanged."""
    cap = TRAFFIC.get((group, precision))
    return cap if cap and cap["src"] == src_hash(cap["kernel"]) else None


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- GPU arm

def replica_reduce(ms_local, bytes_local, dist=None, device=None):
    """Independent replicas (one problem per rank, no exchange in the method):
    the job time is the slowest rank's, the work is the sum over ranks."""
    if dist is None:
        return float(ms_local), int(bytes_local)
    import torch

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    b = torch.tensor([float(bytes_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), int(b.item())


def gmres_cycle(lo, torch, basis, B, stream, Hbuf, Rbuf, events, record=None, passes=None):
    """One restart cycle on the device.  events: list receiving (start, end)
    CUDA event pairs around each hot-path call; passes (untimed cycles only):
    list receiving the local Gram passes each step ran.  Returns the apply_Q
    result."""
    n, s = B.shape
    m = M_RESTART
    basis.reset()
    X = torch.empty_like(B)
    U = torch.empty_like(B)
    V_last = U

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        events.append((e0, e1))
        return r

    # V_0 H_0 = R0 (x0 = 0, so R0 = B)
    timed(lambda: basis.orthogonalize(B, U=U, H=None, R=Rbuf[0]))
    if passes is not None:
        passes.append(basis.last_step_info()[0])
    if record is not None:
        record.append(B.clone())
    for j in range(m):
        lo.laplace5_apply(NX, NY, U, X, stream=stream)
        if record is not None:
            record.append(X.clone())
        k = (j + 1) * s
        timed(lambda: basis.orthogonalize(X, U=U, H=Hbuf[j][:k], R=Rbuf[j + 1]))
        if passes is not None:
            passes.append(basis.last_step_info()[0])
    # small least-squares on the host (harness; untimed)
    torch.cuda.current_stream().synchronize()
    basis.sync()
    Hm = np.zeros(((m + 1) * s, m * s))
    Hh = [h.cpu().numpy() for h in Hbuf]
    Rh = [r.cpu().numpy() for r in Rbuf]
    for j in range(m):
        k = (j + 1) * s
        Hm[:k, j * s:(j + 1) * s] = Hh[j][:k]
        Hm[k:k + s, j * s:(j + 1) * s] = Rh[j + 1]
    rhs = np.zeros(((m + 1) * s, s))
    rhs[:s] = Rh[0]
    y = np.linalg.lstsq(Hm, rhs, rcond=None)[0]
    Yc = torch.from_numpy(np.ascontiguousarray(y)).to(B.device)
    # The correction uses the first m blocks (m*s columns) of the basis: apply_Q over
    # all m+1 blocks with a zero last block row.
    C = torch.zeros(((m + 1) * s, s), dtype=torch.float64, device=B.device)
    C[:m * s] = Yc
    return timed(lambda: basis.apply_Q(C))


def run_gpu(args):
    import torch

    from paper_2204_13393_gb300 import inputs as I
    from paper_2204_13393_gb300 import lo

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lo.library()
    n, s, m = NX * NY, S, M_RESTART
    stream = torch.cuda.current_stream()
    chunk = args.chunk_rows or lo.tune_chunk_rows(n, s, m + 1, precision=args.precision, stream=stream)
    basis = lo.Basis(n, s, m + 1, chunk, sync=False, stream=stream, precision=args.precision)
    p = basis.num_chunks
    B = torch.from_numpy(I.uniform(n, s, I.seed_for(2, rank))).to(dev)
    Hbuf = [torch.empty(((j + 1) * s, s), dtype=torch.float64, device=dev) for j in range(m)]
    Rbuf = [torch.empty((s, s), dtype=torch.float64, device=dev) for _ in range(m + 1)]
    bytes_cycle = sum(orth_bytes(n, s, j * s, p) for j in range(m + 1)) + apply_bytes(n, (m + 1) * s, s, p)

    for _ in range(args.warmup):
        ev = []
        gmres_cycle(lo, torch, basis, B, stream, Hbuf, Rbuf, ev)
    # the local passes of every step (the steps are bit for bit the same every cycle)
    step_passes = []
    gmres_cycle(lo, torch, basis, B, stream, Hbuf, Rbuf, [], passes=step_passes)
    torch.cuda.synchronize()
    basis.profile_read()
    basis.set_profiling(True)
    launches0 = lo.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    events = []
    # the timed cycles are the profiler window (ncu --profile-from-start off)
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            gmres_cycle(lo, torch, basis, B, stream, Hbuf, Rbuf, events)
        torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    launches = lo.launch_count() - launches0
    basis.set_profiling(False)
    prof = basis.profile_read()
    dev_ms = sum(e0.elapsed_time(e1) for e0, e1 in events)
    # replicas: max time over ranks, bytes of all ranks
    t_local, total_bytes = replica_reduce(dev_ms, bytes_cycle * args.steps, dist, dev)
    gbs = total_bytes / (t_local * 1e-3) / 1e9

    # correctness of the last cycle (properties at full size)
    Q = basis.apply_Q(torch.eye((m + 1) * s, dtype=torch.float64, device=dev))
    G = Q.T @ Q
    e_perp = float(torch.linalg.norm(G - torch.eye(G.shape[0], dtype=torch.float64, device=dev)))
    del Q, G

    # dominant kernel group (pass-1 Gram, stage-2 assembly or the reiteration
    # passes) and its roofline
    hbm_peak, hbm_src = peaks()
    tc = args.precision in ("fp64_tc", "mixed_tc")
    kinds = {g: v for g, v in prof.items() if v[1] > 0}
    dom = max((g for g in ("gram", "update", "refine") if g in kinds), key=lambda g: kinds[g][0])
    bsum = fsum = 0
    for j in range(m + 1):
        if dom == "update":
            b_, f_ = update_bytes_flops(n, s, j * s, p)
        elif dom == "gram":
            b_, f_ = gram_bytes_flops(n, s, j * s)
        else:
            b_, f_ = refine_bytes_flops(n, s, j * s, step_passes[j])
        bsum += b_ * args.steps
        fsum += f_ * args.steps
    t_dom = kinds[dom][0] * 1e-3
    ach_gbs = bsum / t_dom / 1e9
    ach_tf = fsum / t_dom / 1e12
    cap = traffic_capture(dom, args.precision)
    launches_dom = kinds[dom][1]
    traffic = (round(cap["dram_bytes"] / cap["algorithmic_bytes"] * bsum / launches_dom)
               if cap else None)
    if tc:
        # s = 8, 16, 32 keep digit planes of the prior panels: tcgen05 kernels
        kernel_name = ({"update": "k_umma_update", "gram": "k_umma_gram",
                        "refine": "k_umma_update<S,1> + k_umma_gram (passes >= 2)"} if s in (8, 16, 32)
                       else {"update": "k_oz_update", "gram": "k_oz_gram",
                             "refine": "k_oz_update + k_oz_gram (passes >= 2)"})[dom]
        # tensor work: 28 fp16 digit-pair products per float64 product, 2 flops each
        tens_tf = 28 * fsum / t_dom / 1e12
        tens_peak = peaks_bf16()
        bound = "hbm" if bsum / (hbm_peak * 1e9) >= 28 * fsum / (tens_peak * 1e12) else "tensor"
        if bound == "hbm":
            roof = {"bound": "hbm", "achieved": round(ach_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(ach_gbs / hbm_peak, 4), "traffic": traffic, "kernel": kernel_name,
                    "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)",
                    "tensor_tflops_fp16": round(tens_tf, 1), "launches": kinds[dom][1]}
        else:
            roof = {"bound": "tensor", "achieved": round(tens_tf, 1), "peak": tens_peak, "unit": "TFLOP/s",
                    "frac": round(tens_tf / tens_peak, 4), "traffic": traffic, "kernel": kernel_name,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops (fp16 mma at the same rate)",
                    "hbm_achieved_gbs": round(ach_gbs, 1), "launches": kinds[dom][1]}
    else:
        kernel_name = {"update": "k_update", "gram": "k_gram1", "refine": "k_gram (passes >= 2)"}[dom]
        roof = {"bound": "alu", "achieved": round(ach_tf, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(ach_tf / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                "kernel": kernel_name, "peak_source": "float64 pipe: 152 SMs x 2 DFMA/clk x 2070 MHz",
                "hbm_achieved_gbs": round(ach_gbs, 1), "hbm_frac_of_measured": round(ach_gbs / hbm_peak, 4),
                "launches": kinds[dom][1]}

    out = None
    if rank == 0:
        e2e = run_e2e(lo, torch, dev, basis, B, stream, n, s, m, p, args.precision, chunk)
        cpu = cpu_baseline(args.cpu_budget) if world == 1 or rank == 0 else None
        clocks = clk.summary()
        targets = None
        if not args.no_targets and world == 1:
            targets = {"cycle_mixed": mixed_cycle(lo, torch, dev, B, stream, n, s, m, chunk, max(3, args.steps),
                                                  args.warmup, t_local / args.steps, bytes_cycle)}
            basis.close()
            torch.cuda.empty_cache()
            targets.update(target_points(lo, torch, dev, args))
        out = {
            "metric": METRIC, "value": round(gbs, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_local / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "block-GMRes restart cycle, 2D 5-point Laplacian 1024x1024 (n=1048576), "
                                   "s=8 RHS U(-1,1), m=30: 31 orthogonalizations (k=0..240) + apply_Q; "
                                   "stencil and host least-squares untimed",
                       "n": n, "s": s, "restart_blocks": m, "chunk_rows": chunk,
                       "chunk_rows_from": "fixed" if args.chunk_rows else "lo_tune_chunk_rows (measured)", "chunks": p,
                       "precision": args.precision, "leaf": "pip2", "reduction": "auto",
                       "arithmetic": ("float64-accurate products on fp16 tensor cores (exact 8-bit digit "
                                      "splitting, exact float32 sums, integer recombination); float64 "
                                      "small factors") if args.precision == "fp64_tc" else args.precision,
                       "l2": "inputs larger than L2 (basis 2.1 GB, 8 MB per block)",
                       "parallelism": f"replicas{world}"},
            "block_steps_per_s": round((m + 1) * args.steps * world / (t_local * 1e-3), 2),
            "hbm_frac_of_step": round(gbs / world / hbm_peak, 4),
            "wall_s": round(wall, 3),
            "kernel_ms": {g: round(v[0], 3) for g, v in prof.items()},
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "cpu_baseline": cpu,
            "e_perp_final": e_perp,
            "step_passes": step_passes,
        }
        if targets is not None:
            out.update(targets)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def mixed_cycle(lo, torch, dev, B, stream, n, s, m, chunk, steps, warmup, fp64_ms, bytes_cycle):
    """The same cycle on a basis of the mixed tensor-core form (first Gram pass
    on the leading 4 digit planes, float64 reiteration): ms per cycle, its
    speedup over the float64 form measured above, and the final basis's
    orthogonality (the speedup is stated at e_perp <= 1e-12)."""
    Hbuf = [torch.empty(((j + 1) * s, s), dtype=torch.float64, device=dev) for j in range(m)]
    Rbuf = [torch.empty((s, s), dtype=torch.float64, device=dev) for _ in range(m + 1)]
    b = lo.Basis(n, s, m + 1, chunk, sync=False, stream=stream, precision="mixed_tc")
    for _ in range(warmup):
        gmres_cycle(lo, torch, b, B, stream, Hbuf, Rbuf, [])
    torch.cuda.synchronize()
    events = []
    for _ in range(steps):
        gmres_cycle(lo, torch, b, B, stream, Hbuf, Rbuf, events)
    torch.cuda.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in events) / steps
    Q = b.apply_Q(torch.eye((m + 1) * s, dtype=torch.float64, device=dev))
    ep = float(torch.linalg.norm(Q.T @ Q - torch.eye((m + 1) * s, dtype=torch.float64, device=dev)))
    del Q
    b.close()
    return {"precision": "mixed_tc", "ms_per_cycle": round(ms, 4), "gbs": round(bytes_cycle / (ms * 1e-3) / 1e9, 2),
            "speedup_vs_fp64_tc": round(fp64_ms / ms, 4), "e_perp_final": ep, "stated": ep <= 1e-12,
            "cycles": steps}


def run_e2e(lo, torch, dev, basis, B, stream, n, s, m, p, basis_precision, chunk):
    """The same cycle's orthogonalizations through the public API with pinned
    host buffers: each call copies W in, U/H/R out and waits (wall clock)."""
    rec = []
    ev = []
    Hbuf = [torch.empty(((j + 1) * s, s), dtype=torch.float64, device=dev) for j in range(m)]
    Rbuf = [torch.empty((s, s), dtype=torch.float64, device=dev) for _ in range(m + 1)]
    gmres_cycle(lo, torch, basis, B, stream, Hbuf, Rbuf, ev, record=rec)
    Wh = [x.cpu().pin_memory() for x in rec]
    Uh = torch.empty((n, s), dtype=torch.float64).pin_memory()
    Hh = torch.empty(((m + 1) * s, s), dtype=torch.float64).pin_memory()
    Rh = torch.empty((s, s), dtype=torch.float64).pin_memory()
    hb = lo.Basis(n, s, m + 1, chunk, sync=True, stream=stream, precision=basis_precision)
    t = 0.0
    h2d = d2h = 0
    tot_bytes = 0
    for rep in range(2):  # one untimed warm-up cycle (first-call set-up per depth), one timed
        hb.truncate(0)
        torch.cuda.synchronize()
        for j, W in enumerate(Wh):
            k = j * s
            t0 = time.perf_counter()
            hb.orthogonalize(W, U=Uh, H=Hh[:k] if k else None, R=Rh)
            if rep:
                t += time.perf_counter() - t0
                h2d += n * s * 8
                d2h += n * s * 8 + (k * s + s * s) * 8
                tot_bytes += orth_bytes(n, s, k, p)
    hb.close()
    return {"value": round(tot_bytes / t / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "calls_per_step": len(Wh),
            "note": "31 lo_orthogonalize calls of one cycle with pinned host W/U/H/R, after one untimed "
                    "warm-up cycle; wall clock incl. copies"}


# --------------------------------------------------------------------------- CPU oracle

# The cycle's 31 orthogonalization depths k = 8 j, j = 0..30, in bisection
# order, so that any prefix of the sample spreads over the whole k range.
SPREAD = [0, 30, 15, 7, 23, 3, 11, 19, 27, 1, 5, 9, 13, 17, 21, 25, 29,
          2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 22, 24, 26, 28]


def oracle_basis_at_depth(O, n, s, cr, k):
    """An oracle basis holding k columns, built without running k / s steps:
    local factors Q_i = the first k unit vectors of the chunk (orthonormal) and
    tree factors T_i = I / sqrt(p) (upper triangular, sum_i T_i^T T_i = I), a
    valid locally orthogonal representation (Sec. 4.1) with the shapes of the
    cycle's basis at that depth; the oracle's work per step depends on those
    shapes only."""
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    p = len(ora.bounds)
    for i, (b, e) in enumerate(ora.bounds):
        Qi = np.zeros((e - b, k))
        Qi[np.arange(k), np.arange(k)] = 1.0
        ora.Qloc[i] = Qi
        ora.T[i] = np.eye(k) / np.sqrt(p)
    return ora


def oracle_sample(budget_s, depths=None):
    """Time the oracle (TreeTSPQR, BCGS-PIP+ local and reduction solvers, as
    the GPU arm runs) on orthogonalization steps of the cycle at full n, at the
    cycle's own depths (``depths``: indices j of k = 8 j; default: bisection
    order until the budget is spent).  Returns (bytes, seconds, depths done)."""
    from oracle import lo_oracle as O
    from paper_2204_13393_gb300 import inputs as I

    n, s = NX * NY, S
    order = list(depths) if depths is not None else SPREAD
    t = 0.0
    nbytes = 0
    done = []
    for j in order:
        k = j * s
        ora = oracle_basis_at_depth(O, n, s, CHUNK, k)
        p = len(ora.bounds)
        W = I.uniform(n, s, I.seed_for(2, 100 + j))
        t0 = time.perf_counter()
        ora.orthogonalize(W, "pip2", "pip2")
        t += time.perf_counter() - t0
        nbytes += orth_bytes(n, s, k, p)
        done.append(j)
        del ora
        if depths is None and t >= budget_s:
            break
    return nbytes, t, done


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _depth_text(done):
    ks = sorted(8 * j for j in done)
    return f"{len(done)} of the cycle's 31 depths (k = {', '.join(map(str, ks))})"


def cpu_baseline(budget_s):
    """The oracle on this host's cores: single-threaded in this process, and
    with every core's BLAS threads in a child process (the same sample)."""
    nbytes, t, done = oracle_sample(budget_s)
    out = {"value": round(nbytes / t / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"one orthogonalization step at each of {_depth_text(done)}, n=1048576, from a "
                     f"locally orthogonal basis of that depth; numpy oracle TreeTSPQR with BCGS-PIP+ local "
                     f"and reduction, single-threaded BLAS; {t:.1f} s"}
    cores = _cores()
    if cores > 1:
        env = dict(os.environ)
        for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(cores)
        try:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample",
                                ",".join(map(str, done))], env=env, capture_output=True, text=True,
                               timeout=max(60.0, 4 * budget_s))
            d = json.loads(r.stdout.strip().splitlines()[-1])
            out["all_cores"] = {"value": round(d["bytes"] / d["seconds"] / 1e9, 4), "unit": "GB/s",
                                "cores": cores, "seconds": round(d["seconds"], 2),
                                "sample": "the same steps, BLAS with one thread per core"}
        except Exception as exc:  # report, never fail the GPU line for the baseline
            out["all_cores"] = {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}
    return out


def run_cpu_sample(arg):
    depths = [int(x) for x in arg.split(",") if x]
    b, t, done = oracle_sample(0.0, depths)
    print(json.dumps({"bytes": b, "seconds": t, "depths": done}), flush=True)


def run_reference(args):
    """The reference arm: the oracle as it stands on this host's cores, on the
    cycle's metric; each step times two orthogonalizations of the cycle at
    full n, the depths following the bisection order, so the steps together
    sample the same k mix as the GPU arm's cycle."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    pos = 0

    def step():
        nonlocal pos
        ds = [SPREAD[pos % len(SPREAD)], SPREAD[(pos + 1) % len(SPREAD)]]
        pos += 2
        return oracle_sample(0.0, ds)

    for _ in range(args.warmup):
        step()
    tot_b = tot_t = 0.0
    depths = []
    for _ in range(args.steps):
        b, t, d = step()
        tot_b += b
        tot_t += t
        depths += d
    gbs = tot_b / tot_t / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_t / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "block-GMRes restart cycle, 2D 5-point Laplacian 1024x1024 (n=1048576), "
                                   "s=8 RHS U(-1,1), m=30: 31 orthogonalizations (k=0..240) + apply_Q; "
                                   "stencil and host least-squares untimed",
                       "n": NX * NY, "s": S, "restart_blocks": M_RESTART, "chunk_rows": CHUNK},
            "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: two orthogonalization steps of the cycle at full n "
                                       f"(numpy oracle, single-threaded BLAS); timed steps covered "
                                       f"{_depth_text(sorted(set(depths)))}"},
            "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """A single mid-cycle orthogonalization (n = 2^20, s = 8, k = 120 prior
    columns from Gaussian blocks by default, --profile-blocks sets k / 8;
    8192-row chunks) for ncu captures: the basis is larger than L2.  The last
    step runs between cudaProfilerStart and cudaProfilerStop (ncu
    --profile-from-start off captures only it)."""
    import torch

    from paper_2204_13393_gb300 import inputs as I
    from paper_2204_13393_gb300 import lo

    n, s, kb = 2 ** 20, 8, args.profile_blocks
    dev = torch.device("cuda", 0)
    lo.library()
    b = lo.Basis(n, s, kb + 1, CHUNK, sync=True, precision=args.precision)
    for j in range(kb):
        b.orthogonalize(torch.from_numpy(I.gaussian(n, s, I.seed_for(9, j))).to(dev))
    W = torch.from_numpy(I.gaussian(n, s, I.seed_for(9, kb))).to(dev)
    torch.cuda.synchronize()
    b.set_profiling(True)
    torch.cuda.profiler.start()
    b.orthogonalize(W)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    prof = b.profile_read()
    print(json.dumps({"case": "profile", "precision": args.precision, "n": n, "s": s, "k": kb * s,
                      "chunks": b.num_chunks,
                      "kernel_ms": {g: round(v[0], 4) for g, v in prof.items()},
                      "passes_tree": b.last_step_info()}), flush=True)


def run_batched_case(args):
    """Batched uneven instances: 64 independent problems (n log-uniform in
    [1e4, 2^20], s from {4, 8, 16}, 1..30 prior blocks built untimed, new block
    N(0,1)); chunk rows from the autotuner; one lo_orthogonalize_batched call
    (a cached CUDA graph) against 64 sequential lo_orthogonalize calls."""
    import torch

    from paper_2204_13393_gb300 import inputs as I
    from paper_2204_13393_gb300 import lo

    dev = torch.device("cuda", 0)
    lo.library()
    if args.batch_recipe == "small":
        # 64 copies of the small block-Arnoldi step's shape (n = 4096, s = 4, 8 prior blocks, 512-row chunks)
        specs = [(4096, 4, 8)] * 64
    else:
        specs = I.batch_instances(64, I.seed_for(5))
    bases, Ws, Us, Hs, Rs, kbs, nbytes, tuned = [], [], [], [], [], [], 0, {}
    t_tune = time.perf_counter()
    for i, (n, s, kb) in enumerate(specs):
        M = kb + 1
        key = (n, s, M)
        if key not in tuned:
            tuned[key] = 512 if args.batch_recipe == "small" else lo.tune_chunk_rows(n, s, M, precision=args.precision)
        cr = tuned[key]
        b = lo.Basis(n, s, M, cr, precision=args.precision, sync=False)
        g = torch.Generator(device=dev)
        g.manual_seed(I.seed_for(5, i))
        for j in range(kb):
            b.orthogonalize(torch.randn(n, s, dtype=torch.float64, device=dev, generator=g))
        b.sync()
        bases.append(b)
        Ws.append(torch.randn(n, s, dtype=torch.float64, device=dev, generator=g))
        Us.append(torch.empty(n, s, dtype=torch.float64, device=dev))
        Hs.append(torch.empty(kb * s, s, dtype=torch.float64, device=dev))
        Rs.append(torch.empty(s, s, dtype=torch.float64, device=dev))
        kbs.append(kb)
        nbytes += orth_bytes(n, s, kb * s, b.num_chunks)
    t_tune = time.perf_counter() - t_tune
    stream = torch.cuda.current_stream()

    def sequential():
        for b, kb in zip(bases, kbs):
            b.truncate(kb)
        for b, W, U, H, R in zip(bases, Ws, Us, Hs, Rs):
            b.orthogonalize(W, U=U, H=H, R=R)
        for b in bases:
            b.sync()

    def batched():
        for b, kb in zip(bases, kbs):
            b.truncate(kb)
        lo.orthogonalize_batched(bases, Ws, Us, Hs, Rs)

    def routed(mode):
        def fn():
            lo.set_batched_route(mode)
            batched()
        return fn

    res = {}
    routes = {}
    for name, fn in (("sequential", sequential), ("batched", routed("auto")), ("graph", routed("graph")),
                     ("persistent", routed("persistent"))):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / args.steps
        if name != "sequential":
            routes[name] = lo.batched_persistent_count()
    lo.set_batched_route("auto")
    print(json.dumps({"case": "batched", "recipe": args.batch_recipe, "precision": args.precision,
                      "instances": len(specs),
                      "persistent_instances": routes,
                      "ms_graph_only": round(res["graph"], 3), "ms_persistent_where_possible": round(res["persistent"], 3),
                      "bytes_per_step": nbytes, "ms_batched": round(res["batched"], 3),
                      "ms_sequential": round(res["sequential"], 3),
                      "gbs_batched": round(nbytes / res["batched"] / 1e6, 1),
                      "gbs_sequential": round(nbytes / res["sequential"] / 1e6, 1),
                      "speedup": round(res["sequential"] / res["batched"], 3),
                      "tuned_chunk_rows": sorted(set(tuned.values())), "setup_s": round(t_tune, 1)}),
          flush=True)


def mixed_measure(lo, torch, dev, n, cr, kappas, reps, check_n=8192):
    """Mixed-precision workload: n rows, s = 16, 30 prior blocks (480 columns,
    Gaussian, built untimed; regenerated from one seed for each form, so only
    one basis is resident at a time), new block a Stewart-type matrix
    U diag(sigma) V^T with kappa from ``kappas`` (orthonormal factors by
    CholeskyQR2 of Gaussians) plus a component along the last prior block.
    Each step is timed with CUDA events for the float64 tensor-core form and
    the mixed tensor-core form.  Per result: the step's orthogonality
    sqrt(|U^T U - I|^2 + 2 |Q^T U|^2) (Q^T U measured by one more projection
    of U: the H output of a PQR step of U) and its residual
    |W - Q H - U R| / |W|; and, on a sampled run of the same shape at
    n = check_n rows (the oracle at full n would take hours), the U, H, R
    error of each form against the CPU oracle (BCGS-PIP+ TreeTSPQR)."""
    s, kb = 16, 30
    out = {"n": n, "s": s, "k": kb * s, "chunk_rows": cr, "results": []}
    Ws = {}
    for kappa in kappas:
        g = torch.Generator(device=dev)
        g.manual_seed(2204133930 + 4100 + int(round(np.log10(kappa))))
        Uh = orthonormal_columns(torch, torch.randn(n, s, dtype=torch.float64, device=dev, generator=g))
        Vh = orthonormal_columns(torch, torch.randn(s, s, dtype=torch.float64, device=dev, generator=g))
        sig = torch.tensor([kappa ** (-j / (s - 1.0)) for j in range(s)], dtype=torch.float64, device=dev)
        Ws[kappa] = ((Uh * sig) @ Vh.T).cpu()
        del Uh
    rows = {kappa: {"kappa": kappa} for kappa in kappas}
    nbytes = orth_bytes(n, s, kb * s, max(1, n // cr))
    for prec in ("fp64_tc", "mixed_tc"):
        b = lo.Basis(n, s, kb + 2, cr, precision=prec, sync=True)
        g = torch.Generator(device=dev)
        g.manual_seed(2204133930 + 4000)
        last = None
        for _ in range(kb):
            last = torch.randn(n, s, dtype=torch.float64, device=dev, generator=g)
            b.orthogonalize(last)
        for kappa in kappas:
            # the block also has components along the basis, like a Krylov block
            W = Ws[kappa].to(dev) + 0.5 * last / float(n) ** 0.5
            times = []
            for rep in range(max(2, reps)):
                b.truncate(kb)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                U, H, R = b.orthogonalize(W)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            passes = b.last_step_info()
            C = torch.zeros(((kb + 1) * s, s), dtype=torch.float64, device=dev)
            C[:kb * s] = H
            res = float(torch.linalg.norm(W - b.apply_Q(C) - U @ R) / torch.linalg.norm(W))
            UtU = U.T @ U
            b.truncate(kb)
            _, QtU, _ = b.orthogonalize(U.clone())   # H = Q^T U against the kb prior blocks
            eye = torch.eye(s, dtype=torch.float64, device=dev)
            eperp = float(torch.sqrt(torch.linalg.norm(UtU - eye) ** 2 + 2 * torch.linalg.norm(QtU) ** 2))
            ms = min(times[1:])
            rows[kappa][prec] = {"ms": round(ms, 3), "gbs": round(nbytes / ms / 1e6, 1), "e_perp": eperp,
                                 "residual": res, "passes": passes[0], "tree_iterations": passes[1]}
            del U, H, R, W, C
        b.close()
        del last
        torch.cuda.empty_cache()
    # the sampled run against the oracle
    if check_n:
        chk = mixed_oracle_check(lo, torch, dev, check_n, kappas)
        for kappa in kappas:
            for prec in ("fp64_tc", "mixed_tc"):
                rows[kappa][prec]["oracle_sample"] = chk[kappa][prec]
    for kappa in kappas:
        r = rows[kappa]
        r["speedup_mixed_vs_fp64"] = round(r["fp64_tc"]["ms"] / r["mixed_tc"]["ms"], 3)
        r["speedup_stated"] = r["mixed_tc"]["e_perp"] <= 1e-12
        out["results"].append(r)
    return out


def mixed_oracle_check(lo, torch, dev, n, kappas):
    """U, H, R of both forms against the CPU oracle at n rows (s = 16, 30 prior
    Gaussian blocks, 1024-row chunks, the same block recipe as mixed_measure)."""
    from oracle import lo_oracle as O
    from paper_2204_13393_gb300 import inputs as I

    s, kb, cr = 16, 30, 1024
    prior = [I.gaussian(n, s, I.seed_for(4, j)) for j in range(kb)]
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    for P in prior:
        ora.orthogonalize(P, "pip2", "pip2")
    out = {}
    for kappa in kappas:
        W = I.stewart(n, s, kappa, I.seed_for(4, 100 + int(round(np.log10(kappa))))) + 0.5 * prior[-1] / np.sqrt(n)
        import copy
        o = copy.deepcopy(ora)
        Uo, Po, No = o.orthogonalize(W, "pip2", "pip2")
        out[kappa] = {}
        for prec in ("fp64_tc", "mixed_tc"):
            b = lo.Basis(n, s, kb + 1, cr, precision=prec, sync=True)
            for P in prior:
                b.orthogonalize(torch.from_numpy(P).to(dev))
            U, H, R = (x.cpu().numpy() for x in b.orthogonalize(torch.from_numpy(W).to(dev)))
            b.close()

            def rel(a, c):
                return float(np.linalg.norm(a - c) / np.linalg.norm(c))
            out[kappa][prec] = {"n": n, "U_rel": rel(U, Uo), "H_rel": rel(H, Po), "R_rel": rel(R, No)}
    return out


def run_mixed_case(args):
    import torch

    from paper_2204_13393_gb300 import lo

    dev = torch.device("cuda", 0)
    lo.library()
    cr = args.mixed_cr or lo.tune_chunk_rows(args.mixed_n, 16, 32, precision="fp64_tc")
    out = mixed_measure(lo, torch, dev, args.mixed_n, cr, [float(x) for x in args.mixed_kappas.split(",")],
                        args.steps)
    out["case"] = "mixed"
    out["chunk_rows_from"] = "option" if args.mixed_cr else "lo_tune_chunk_rows (measured)"
    print(json.dumps(out), flush=True)


def orthonormal_columns(torch, X):
    """Q of X = QR by CholeskyQR2: two passes of X <- X L^-T with L the
    Cholesky factor of X^T X (the s x s factor on the host), so only matrix
    products run on the device.  For a Gaussian X (condition ~1) the result
    is orthonormal to rounding."""
    for _ in range(2):
        G = (X.T @ X).cpu().numpy()
        Linv_t = np.linalg.inv(np.linalg.cholesky(G)).T
        X = X @ torch.from_numpy(np.ascontiguousarray(Linv_t)).to(X.device)
    return X


def run_step_case(args):
    """The small block-Arnoldi step (n = 4096, s = 4, 8 prior blocks built by
    orthogonalizing seeded N(0,1) blocks, 512-row chunks, new block N(0,1)):
    launch-bound, so one step is captured once in a CUDA graph on the basis
    stream and replayed 1000 times; reported as the median replay time (CUDA
    events) and steps/s, with e_perp of the 9-block basis and the H, R of the
    replays against an eager step."""
    import torch

    from paper_2204_13393_gb300 import inputs as I
    from paper_2204_13393_gb300 import lo

    n, s, kb, cr = 4096, 4, 8, 512
    dev = torch.device("cuda", 0)
    lo.library()
    out = {"case": "step", "n": n, "s": s, "k": kb * s, "chunk_rows": cr, "results": {}}
    for prec in args.step_precisions.split(","):
        st = torch.cuda.Stream()
        b = lo.Basis(n, s, kb + 1, cr, sync=False, stream=st, precision=prec)
        with torch.cuda.stream(st):
            for j in range(kb):
                b.orthogonalize(torch.from_numpy(I.gaussian(n, s, I.seed_for(1, j))).to(dev))
            W = torch.from_numpy(I.gaussian(n, s, I.seed_for(1, kb))).to(dev)
            U = torch.empty(n, s, dtype=torch.float64, device=dev)
            H = torch.empty(kb * s, s, dtype=torch.float64, device=dev)
            R = torch.empty(s, s, dtype=torch.float64, device=dev)
            l0 = lo.launch_count()
            st.synchronize()
            torch.cuda.profiler.start()              # the eager step is the profiler window
            b.orthogonalize(W, U=U, H=H, R=R)       # eager step (also the warm-up)
            st.synchronize()
            torch.cuda.profiler.stop()
            launches = lo.launch_count() - l0
        st.synchronize()
        H0, R0 = H.clone(), R.clone()
        b.truncate(kb)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            b.orthogonalize(W, U=U, H=H, R=R)   # the basis holds 9 blocks; each replay rewrites the 9th
        times = []
        with torch.cuda.stream(st):
            for _ in range(20):
                g.replay()
            for _ in range(1000):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                g.replay()
                e1.record(st)
                times.append((e0, e1))
        st.synchronize()
        us = sorted(e0.elapsed_time(e1) * 1e3 for e0, e1 in times)
        med = us[len(us) // 2]
        # the same step as one persistent launch (lo_orthogonalize_batched with
        # one instance, route 'persistent': init kernel + the persistent kernel)
        lo.set_batched_route("persistent")
        ptimes = []
        with torch.cuda.stream(st):
            for rep in range(220):
                b.truncate(kb)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                lo.orthogonalize_batched([b], [W], [U], [H], [R])
                e1.record(st)
                if rep >= 20:
                    ptimes.append((e0, e1))
        st.synchronize()
        lo.set_batched_route("auto")
        pus = sorted(e0.elapsed_time(e1) * 1e3 for e0, e1 in ptimes)
        pmed = pus[len(pus) // 2]
        Hp, Rp = H.clone(), R.clone()
        Q = b.apply_Q(torch.eye((kb + 1) * s, dtype=torch.float64, device=dev))
        st.synchronize()
        eperp = float(torch.linalg.norm(Q.T @ Q - torch.eye((kb + 1) * s, dtype=torch.float64, device=dev)))
        nbytes = orth_bytes(n, s, kb * s, n // cr)
        out["results"][prec] = {
            "us_median": round(med, 2), "us_p10": round(us[len(us) // 10], 2), "us_p90": round(us[9 * len(us) // 10], 2),
            "steps_per_s": round(1e6 / med, 1), "gbs": round(nbytes / (med * 1e-6) / 1e9, 2),
            "e_perp": eperp, "H_replay_vs_eager": float((H - H0).abs().max()),
            "R_replay_vs_eager": float((R - R0).abs().max()), "launches_per_step": launches,
            "persistent_launch": {"us_median": round(pmed, 2), "us_p10": round(pus[len(pus) // 10], 2),
                                  "steps_per_s": round(1e6 / pmed, 1), "launches_per_step": 2,
                                  "H_vs_eager": float((Hp - H0).abs().max() / H0.abs().max()),
                                  "R_vs_eager": float((Rp - R0).abs().max() / R0.abs().max()),
                                  "note": "device time between events around one lo_orthogonalize_batched "
                                          "call (a cached graph: init + persistent kernel; float64 on the "
                                          "CUDA cores)"}}
        b.close()
    print(json.dumps(out), flush=True)


def tsqr_measure(lo, torch, dev, ns, ss, kappas, forms, reps, cr_fixed=0, verbose=False):
    """Tall-skinny QR (k = 0 step): A = U diag(sigma) V^T with Haar U, V (QR of
    Gaussians on the device) and sigma log-spaced from 1 to 1/kappa.  Each form
    ("precision" or "precision:leaf") gets the autotuned chunk size (or
    cr_fixed); one step is timed with CUDA events (min over ``reps``
    repetitions after one warm-up).  Algorithmic bytes 32ns: read A twice,
    write the local panel and U.  Reported with e_perp = |U^T U - I|_F and
    |A - UR|_F / |A|_F.  The profiled step of each form runs between
    cudaProfilerStart and cudaProfilerStop (for ncu --profile-from-start off)."""
    hbm, _src = peaks()
    rows = []
    g = torch.Generator(device=dev)
    g.manual_seed(2204133930 + 3000)
    for n in ns:
        for s in ss:
            nbytes = 32 * n * s
            for kappa in kappas:
                Uh = orthonormal_columns(torch, torch.randn(n, s, dtype=torch.float64, device=dev, generator=g))
                Vh = orthonormal_columns(torch, torch.randn(s, s, dtype=torch.float64, device=dev, generator=g))
                sig = torch.tensor([kappa ** (-j / max(s - 1.0, 1.0)) for j in range(s)], dtype=torch.float64,
                                   device=dev)
                A = (Uh * sig) @ Vh.T
                del Uh
                row = {"n": n, "s": s, "kappa": kappa}
                for form in forms:
                    prec, _, leaf = form.partition(":")
                    leaf = leaf or "pip2"
                    cr = cr_fixed or lo.tune_chunk_rows(n, s, 1, precision=prec, leaf=leaf)
                    b = lo.Basis(n, s, 1, cr, precision=prec, leaf=leaf, sync=True)
                    U = torch.empty_like(A)
                    times = []
                    for rep in range(1 + max(1, reps)):
                        b.truncate(0)
                        torch.cuda.synchronize()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        _, _, R = b.orthogonalize(A, U=U)
                        e1.record()
                        torch.cuda.synchronize()
                        times.append(e0.elapsed_time(e1))
                    ms = min(times[1:])
                    b.truncate(0)
                    b.set_profiling(True)
                    torch.cuda.profiler.start()
                    b.orthogonalize(A, U=U)
                    torch.cuda.synchronize()
                    torch.cuda.profiler.stop()
                    prof = {k_: round(v[0], 4) for k_, v in b.profile_read().items() if v[0] > 0}
                    b.set_profiling(False)
                    eye = torch.eye(s, dtype=torch.float64, device=dev)
                    eperp = float(torch.linalg.norm(U.T @ U - eye))
                    res = float(torch.linalg.norm(A - U @ R) / torch.linalg.norm(A))
                    row[form] = {"ms": round(ms, 4), "gbs": round(nbytes / ms / 1e6, 1),
                                 "frac_hbm": round(nbytes / ms / 1e6 / hbm, 3), "chunk_rows": cr,
                                 "e_perp": eperp, "residual": res, "passes": b.last_step_info()[0],
                                 "kernel_ms": prof}
                    b.close()
                    del U
                rows.append(row)
                if verbose:
                    print(json.dumps(row), flush=True)
                del A
    return rows


def run_tsqr_case(args):
    """--case tsqr: the tall-skinny QR sweep (--tsqr-n, --tsqr-s, --tsqr-kappas,
    --tsqr-precisions)."""
    import torch

    from paper_2204_13393_gb300 import lo

    dev = torch.device("cuda", 0)
    lo.library()
    rows = tsqr_measure(lo, torch, dev, [int(a) for a in args.tsqr_n.split(",")],
                        [int(b) for b in args.tsqr_s.split(",")],
                        [float(x) for x in args.tsqr_kappas.split(",")], args.tsqr_precisions.split(","),
                        args.steps, args.tsqr_cr, verbose=True)
    print(json.dumps({"case": "tsqr", "n": args.tsqr_n, "results": rows}), flush=True)


def target_points(lo, torch, dev, args):
    """The two measurements reported beside the cycle, on the current GPU: the
    tall-skinny QR at n = 2^24, s = 8 (FP64 target: >= 70 % of the HBM
    roofline, e_perp <= 1e-12) and the mixed form's speedup over the float64
    form at n = 2^24, s = 16, k = 480, kappa <= 1e6."""
    hbm, _ = peaks()
    out = {}
    t0 = time.perf_counter()
    rows = tsqr_measure(lo, torch, dev, [2 ** 24], [8], [1e2, 1e6, 1e10], args.target_forms.split(","), 3)
    out["tsqr_2p24_s8"] = {
        "roofline_time_ms_at_70pct": round(32 * 2 ** 24 * 8 / (0.7 * hbm * 1e9) * 1e3, 4),
        "results": rows, "seconds": round(time.perf_counter() - t0, 1)}
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    mx = mixed_measure(lo, torch, dev, 2 ** 24, args.mixed_cr or 131072, [1e2, 1e4, 1e6], 3)
    mx["chunk_rows_from"] = "option" if args.mixed_cr else "fixed (131072: the tuner's choice for the float64 form)"
    mx["seconds"] = round(time.perf_counter() - t0, 1)
    out["mixed_speedup"] = mx
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lo", choices=["lo", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for the CPU baseline")
    ap.add_argument("--precision", default="fp64_tc", choices=["fp64", "fp64_tc", "mixed_fp32", "mixed_tc"],
                    help="fp64_tc (default): float64-accurate products on the tensor cores; fp64: native float64")
    ap.add_argument("--case", default="cycle", choices=["cycle", "profile", "batched", "mixed", "tsqr", "step"],
                    help="profile: one mid-cycle step for ncu captures; batched: 64 uneven instances; "
                         "mixed: float64 vs mixed tensor-core forms at n = 2^24, s = 16, k = 480; "
                         "tsqr: k = 0 steps at n = 2^24; step: the small step (n = 4096, s = 4, k = 32), "
                         "graph-replayed")
    ap.add_argument("--batch-recipe", default="uneven", choices=["uneven", "small"],
                    help="--case batched: the uneven 64-instance batch, or 64 copies of the small step")
    ap.add_argument("--mixed-n", type=int, default=2 ** 24)
    ap.add_argument("--mixed-cr", type=int, default=0, help="chunk rows for --case mixed (0: lo_tune_chunk_rows)")
    ap.add_argument("--mixed-kappas", default="1e2,1e4,1e6", help="condition numbers for --case mixed")
    ap.add_argument("--step-precisions", default="fp64,fp64_tc", help="forms for --case step")
    ap.add_argument("--profile-blocks", type=int, default=15,
                    help="--case profile: prior blocks of the profiled step (k = 8 x this)")
    ap.add_argument("--chunk-rows", type=int, default=CHUNK,
                    help="chunk rows of the cycle's basis (0: lo_tune_chunk_rows, measured on this GPU)")
    ap.add_argument("--tsqr-n", default=str(2 ** 24), help="comma-separated row counts for --case tsqr")
    ap.add_argument("--tsqr-s", default="8", help="comma-separated block widths for --case tsqr")
    ap.add_argument("--tsqr-cr", type=int, default=0, help="chunk rows for --case tsqr (0: autotuned)")
    ap.add_argument("--tsqr-kappas", default="1e2,1e6,1e10", help="condition numbers for --case tsqr")
    ap.add_argument("--tsqr-precisions", default="fp64,fp64_tc,fp64:hh",
                    help="forms (precision[:leaf]) for --case tsqr")
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-targets", action="store_true",
                    help="skip the tall-skinny target point and the mixed speedup in the default line")
    ap.add_argument("--target-forms", default="fp64_tc,fp64:hh",
                    help="forms of the tall-skinny target point in the default line")
    args = ap.parse_args()
    if args.cpu_sample is not None:
        run_cpu_sample(args.cpu_sample)
        return
    if args.case == "profile":
        run_profile_case(args)
        return
    if args.case == "batched":
        run_batched_case(args)
        return
    if args.case == "mixed":
        run_mixed_case(args)
        return
    if args.case == "tsqr":
        run_tsqr_case(args)
        return
    if args.case == "step":
        run_step_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
