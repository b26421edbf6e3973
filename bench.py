#!/usr/bin/env python3
"""Throughput of the GPU reduction path: compress + decompress of a 513^3 FP32
Gaussian random field (power spectrum ~|k|^-11/3, unit variance; stands in for
the paper's NYX 512^3 FP32 fields, which are not available) at a relative
L-infinity bound of 1e-3, on one GB300.

One step = hpdr_compress_async (device field -> device container) followed by
hpdr_decompress_async (container -> device field, header parsed on the
device): the step queues without host waits.  value = 2 x field bytes per
step / step time (each direction moves the field's original bytes once; the
paper's throughput unit is original bytes per second).

Run:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torchrun: every rank compresses its own field (replicas,
no data exchange); value = bytes of all ranks / max time over ranks.
"""
import argparse
import ctypes as C
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress/decompress GB/s on 1 GB300 at rel L∞ 1e-3; % of HBM roofline"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--shape", default="513,513,513")
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32",
                    help="element type of the timed field (f64 for profiling the FP64 path)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-to-host leg")
    ap.add_argument("--cpu-planes", type=int, default=257,
                    help="planes of the field in the CPU-baseline sample")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the 257^3 adjoint leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-field batched leg")
    ap.add_argument("--batch-dict", type=int, default=8192, help="dictionary size of the batched leg")
    ap.add_argument("--no-stream", action="store_true", help="skip the 1025^3 host-streamed leg")
    ap.add_argument("--no-lossless", action="store_true", help="skip the lossless (Huffman-only) leg")
    ap.add_argument("--no-l2s", action="store_true", help="skip the statistical L2 mode leg")
    ap.add_argument("--no-zfp", action="store_true", help="skip the fixed-rate ZFP leg")
    ap.add_argument("--no-coords", action="store_true", help="skip the non-uniform grid leg")
    ap.add_argument("--no-bounds", action="store_true",
                    help="skip the legs at the other bounds (1e-2, 1e-4) and the 500x500x100 FP64 field")
    return ap.parse_args()


def workload_name(shape, tol, dtype="f32"):
    return "%s %s power-law field (|k|^-11/3), rel Linf %g, compress+decompress" % (
        "x".join(str(s) for s in shape), "FP64" if dtype == "f64" else "FP32", tol)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows),
                "window": "warmup+timed region (200 ms sampling)"}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


LEVEL_GROUPS = ("c_restrict_quant_L", "d_restrict_sym_L", "d_expand_L", "c_solves_L", "d_solves_L")


def source_hash(group="c_restrict_quant_L"):
    """SHA-256 prefix of the sources of a kernel group's translation unit: the
    plane-streaming level kernels (decomp.cu, levels_dev.cuh, levels.cuh,
    internal.cuh), the solves (levels.cu, levels_dev.cuh, levels.cuh,
    internal.cuh) or the Huffman kernels (huffman.cu, huffman.cuh,
    internal.cuh)."""
    if group in ("c_solves_L", "d_solves_L"):
        files = ("levels.cu", "levels_dev.cuh", "levels.cuh", "internal.cuh")
    elif group in LEVEL_GROUPS:
        files = ("decomp.cu", "levels_dev.cuh", "levels.cuh", "internal.cuh")
    else:
        files = ("huffman.cu", "huffman.cuh", "internal.cuh")
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2503_06322_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_group):
    """DRAM bytes per launch of a kernel group from the committed ncu summary,
    only if it was captured from the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    cur = source_hash(kernel_group)
    for ln in lines:
        parts = [p.strip() for p in ln.strip().strip("|").split("|")]
        if len(parts) >= 4 and parts[0] == kernel_group and parts[1] == cur:
            try:
                return float(parts[3])
            except ValueError:
                return None
    return None


# ---------------------------------------------------------------------------
def algorithmic_bytes(group, S, NL, NL1, bits, nch):
    """Bytes each kernel group must move per launch (the roofline numerator)."""
    new = NL - NL1
    if group == "c_restrict_quant_L":      # read v_L, write symbols, b and coarse copy
        return S * NL + 2 * new + 2 * S * NL1
    if group == "d_expand_L":              # read symbols and corrected coarse grid, write field
        return 2 * new + S * NL1 + S * NL
    if group == "d_restrict_sym_L":        # read symbols, write b
        return 2 * new + S * NL1
    if group == "d_decode":                # read bitstream + chunk table, write symbols
        return bits / 8.0 + 8 * nch + 2 * NL
    if group == "norm":
        return S * NL
    return None


def run_ours(args, rank, world, local):
    import torch
    from paper_2503_06322_gb300 import fields, hpdr

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    shape = tuple(int(x) for x in args.shape.split(","))
    u = fields.powerlaw_field_torch(shape, seed=args.seed + rank, device=dev,
                                    dtype=torch.float64 if args.dtype == "f64" else torch.float32)
    nbytes = u.numel() * u.element_size()
    L = hpdr.lib()
    ctx = hpdr.context(local)
    stream = torch.cuda.current_stream()
    cap = hpdr.hpdr_compress_bound(shape, u.dtype)
    cbuf = torch.empty(cap, dtype=torch.uint8, device=dev)
    rec = torch.empty_like(u)

    # the timed step queues hpdr_compress_async and hpdr_decompress_async (the
    # header is parsed on the device), so steps follow each other without host
    # waits; their device results are checked after the timed region
    nres = 64
    res_c = torch.zeros((nres, 2), dtype=torch.int64, device=dev)
    res_d = torch.zeros((nres, 1), dtype=torch.int64, device=dev)

    def step(i=0):
        hpdr.hpdr_compress_async(u, args.tol, cbuf, res_c[i % nres])
        hpdr.hpdr_decompress_async(cbuf, rec, res_d[i % nres])

    def check_results():
        torch.cuda.synchronize()
        bad_c = int((res_c[:, 1] != 0).sum())
        bad_d = int((res_d[:, 0] != 0).sum())
        if bad_c or bad_d:
            raise RuntimeError("device status: compress %s decompress %s"
                               % (res_c[:, 1].tolist(), res_d[:, 0].tolist()))
        return int(res_c[0, 0])

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for i in range(max(args.warmup, 3)):
        step(i)
    # the waiting API gives the same container (checked here, outside the timing)
    comp_bytes = check_results()
    ref = hpdr.hpdr_compress(u, args.tol)
    if ref.numel() != comp_bytes or not torch.equal(ref, cbuf[:comp_bytes]):
        raise RuntimeError("asynchronous and waiting compression disagree")
    del ref
    # ---- per-direction throughput (separate, untimed for `value`) ----
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    nsep = min(20, args.steps)
    tc = td = 0.0
    for i in range(nsep):
        e0.record(stream)
        hpdr.hpdr_compress_async(u, args.tol, cbuf, res_c[i % nres])
        e1.record(stream)
        hpdr.hpdr_decompress_async(cbuf, rec, res_d[i % nres])
        e2.record(stream)
        torch.cuda.synchronize()
        tc += e0.elapsed_time(e1)
        td += e1.elapsed_time(e2)
    check_results()
    b = cbuf[:comp_bytes]

    # ---- timed region ----
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.6)
    L.hpdr_profile_enable.argtypes = [C.c_void_p, C.c_int]
    L.hpdr_profile_enable(ctx, 1)
    nprof_read = (C.c_char_p * 64)()
    ms_arr = (C.c_double * 64)()
    cnt_arr = (C.c_longlong * 64)()
    L.hpdr_profile_read.argtypes = [C.c_void_p, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                    C.POINTER(C.c_longlong), C.c_int]
    L.hpdr_launch_count.restype = C.c_ulonglong
    L.hpdr_profile_read(ctx, nprof_read, ms_arr, cnt_arr, 64)   # clear
    barrier()
    launches0 = L.hpdr_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        if i == 500:   # the diagnostics' event pool covers the first 500 steps
            L.hpdr_profile_enable(ctx, 0)
        step(i)
    t_stop.record(stream)
    barrier()
    check_results()
    launches = L.hpdr_launch_count() - launches0
    L.hpdr_profile_enable(ctx, 0)
    ng = L.hpdr_profile_read(ctx, nprof_read, ms_arr, cnt_arr, 64)
    groups = {nprof_read[i].decode(): (ms_arr[i], cnt_arr[i]) for i in range(ng)}
    ms_total = t_start.elapsed_time(t_stop)
    clk = clocks.stop()
    ms_total = max_over_ranks(ms_total, dev)
    ms_step = ms_total / args.steps
    value = job_gbs(world, 2.0 * nbytes, ms_step)

    # ---- correctness of the timed output ----
    tau = args.tol * u.abs().max().item()
    err = (rec - u).abs().max().item()

    # ---- roofline of the dominant single kernel ----
    NL = u.numel()
    NL1 = level_nodes(shape, 1)
    bits = _parse_bits(b)
    kchunk = int.from_bytes(b[56:60].cpu().numpy().tobytes(), "little")
    nch = (NL + kchunk - 1) // kchunk
    single = ["c_restrict_quant_L", "d_expand_L", "d_restrict_sym_L", "d_decode", "norm"]
    best = max((g for g in single if g in groups), key=lambda g: groups[g][0])
    ms_b, cnt_b = groups[best]
    avg_s = ms_b / cnt_b * 1e-3
    alg = algorithmic_bytes(best, u.element_size(), NL, NL1, bits, nch)
    peak, peak_kind = measured_peak()
    achieved = alg / avg_s / 1e9
    traffic = ncu_traffic(best)
    prof_steps = max(1, groups.get("norm", (0, 1))[1])
    breakdown = {g: round(v[0] / prof_steps, 4) for g, v in sorted(groups.items(), key=lambda x: -x[1][0])}
    roofline = {"bound": "hbm", "kernel": best, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": int(alg),
                "avg_launch_ms": round(avg_s * 1e3, 4)}

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic (seeded power-law Gaussian random field generated on the device)",
        "config": {"workload": workload_name(shape, args.tol, args.dtype), "shape": list(shape),
                   "tol": args.tol, "tol_kind": "rel", "mode": "Linf", "dict_size": 8192,
                   "chunk": kchunk, "l2": "inputs larger than L2 (%d MB field, 129 MB L2)" % (nbytes // 10**6),
                   "parallelism": "replicas x%d" % world},
        "compress_gbs": round(nbytes / (tc / nsep * 1e-3) / 1e9, 2),
        "decompress_gbs": round(nbytes / (td / nsep * 1e-3) / 1e9, 2),
        "compression_ratio": round(nbytes / comp_bytes, 4),
        "max_err_over_tau": round(err / tau, 4),
        "roofline": roofline, "breakdown_ms_per_step": breakdown,
        "gpu_launches": int(launches), "clocks": clk,
    }
    return out, u, cbuf, comp_bytes


def max_over_ranks(x, device):
    """The largest per-rank value over the process group (the slowest rank's
    time); the value itself when there is no group or a single rank."""
    import torch
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(world, bytes_per_rank_step, ms_per_step):
    """Whole-job throughput: bytes all ranks moved per step / the step time."""
    return world * bytes_per_rank_step / (ms_per_step * 1e-3) / 1e9


def level_nodes(shape, down):
    """Node count of the level `down` coarsenings below the finest grid."""
    n = 1
    for s in shape:
        for _ in range(down):
            s = (s + 1) // 2 if s % 2 else s // 2 + 1
        n *= s
    return n


def _parse_bits(buf):
    h = buf[:128].cpu().numpy().tobytes()
    return int.from_bytes(h[112:120], "little")


E2E_C_INIT = 128 << 20      # Alg. 4: first chunk
E2E_C_LIMIT = 256 << 20     # Alg. 4: largest chunk, the fixed pipeline's slab size
PROFILE_MB = (8, 16, 32, 64, 128, 256, 512, 1024, 2048)


def profile_model(h, tol):
    """Model of the adaptive pipeline (Sec. V-C) profiled on the field itself:
    chunk sizes from 8 MiB up to the whole field, f = 0.1."""
    from paper_2503_06322_gb300 import hpdr
    fb = h.numel() * h.element_size()
    sizes = [m << 20 for m in PROFILE_MB if (m << 20) < fb] + [fb]
    return hpdr.pipeline_profile(h, tol, sizes, reps=2, f=0.1)


def run_e2e(args, u, out):
    """Host to host through the public API: a pinned host field is compressed
    by the adaptive pipeline of Alg. 4 (chunks copied in, compressed,
    containers copied out, overlapped on three streams; chunk sizes from the
    model profiled on this field before the timed region) and the container
    decompressed back to host memory.  The same with fixed 256 MiB slabs is
    reported beside it."""
    import torch
    from paper_2503_06322_gb300 import hpdr
    h_in = torch.empty(u.shape, dtype=u.dtype, pin_memory=True)
    h_in.copy_(u.cpu())
    h_out = torch.empty_like(h_in).pin_memory()
    model = profile_model(h_in, args.tol)
    plane = h_in.element_size() * h_in[0].numel()
    planes = hpdr.pipeline_plan(model, h_in.shape[0], plane, E2E_C_INIT, E2E_C_LIMIT)
    cap = max(hpdr.streamed_bound_plan(u.shape, u.dtype, planes), hpdr.streamed_bound(u.shape, u.dtype))
    h_c = torch.empty(cap, dtype=torch.uint8, pin_memory=True)

    def adaptive():
        b = hpdr.hpdr_compress_host_adaptive(h_in, args.tol, model, c_init=E2E_C_INIT, c_limit=E2E_C_LIMIT,
                                             out=h_c)
        hpdr.hpdr_decompress_host_streamed(b, out=h_out)
        return b.numel()

    def fixed():
        b = hpdr.hpdr_compress_host_streamed(h_in, args.tol, out=h_c)
        hpdr.hpdr_decompress_host_streamed(b, out=h_out)
        return b.numel()

    fb = u.numel() * u.element_size()
    k = max(3, min(args.steps, 10))
    # the two pipelines alternate step by step, so that both see the same
    # host and link conditions; each reports the median of its k steps
    for _ in range(2):
        fixed()
        adaptive()
    times = {"fixed": [], "adaptive": []}
    for _ in range(k):
        for name, step in (("fixed", fixed), ("adaptive", adaptive)):
            t0 = time.perf_counter()
            step()
            times[name].append((time.perf_counter() - t0) * 1e3)
    ms = sorted(times["adaptive"])[k // 2]
    fms = sorted(times["fixed"])[k // 2]
    tau = args.tol * h_in.abs().max().item()
    fixed()
    ferr = (h_out.double() - h_in.double()).abs().max().item() / tau
    nb = adaptive()
    err = (h_out.double() - h_in.double()).abs().max().item() / tau
    return {"value": round(2.0 * fb / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": fb + nb, "d2h_bytes_per_step": nb + fb,
            "ms_per_step": round(ms, 3), "steps": k, "max_err_over_tau": round(err, 4),
            "path": "pinned host field -> hpdr_compress_host_adaptive (Alg. 4 chunks, C_init 128 MiB, "
                    "C_limit 256 MiB) -> hpdr_decompress_host_streamed -> pinned host field (wall clock, "
                    "median of the steps)",
            "chunks_planes": planes,
            "model": {k2: float("%.4g" % v) for k2, v in model.as_dict().items()},
            "fixed_256MiB": {"value": round(2.0 * fb / (fms * 1e-3) / 1e9, 2), "ms_per_step": round(fms, 3),
                             "max_err_over_tau": round(ferr, 4)}}


def run_adjoint(args, dev):
    """257^3 FP32 coefficient set; loss = mean((R(c) - t)^2) through the
    autograd wrapper (forward hpdr_recompose, backward hpdr_recompose_adjoint)."""
    import torch
    from paper_2503_06322_gb300 import autograd, fields, hpdr
    shape = (257, 257, 257)
    u0 = fields.powerlaw_field_torch(shape, seed=4, device=dev)
    t = fields.powerlaw_field_torch(shape, seed=5, device=dev)
    c0 = hpdr.hpdr_decompose(u0)

    def step():
        c = c0.detach().requires_grad_(True)
        loss = ((autograd.recompose(c, shape) - t) ** 2).mean()
        loss.backward()
        return c.grad

    for _ in range(3):
        step()
    k = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(k):
        g = step()
    e1.record()
    torch.cuda.synchronize()
    fwd_bwd = e0.elapsed_time(e1) / k
    e0.record()
    for _ in range(k):
        hpdr.hpdr_recompose(c0, shape)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / k
    return {"workload": "257^3 FP32 coefficients, loss = mean((recompose(c) - t)^2)",
            "fwd_bwd_ms_per_step": round(fwd_bwd, 3), "recompose_ms": round(fwd, 3),
            "grad_norm": round(float(g.norm().item()), 6)}


def run_batched(args, dev):
    """256 FP32 fields, 2-D or 3-D, dims log-uniform in [17, 513], own bounds in
    {1e-2, 1e-3, 1e-4}: one graph replay vs one hpdr_compress call per field."""
    import torch
    from paper_2503_06322_gb300 import fields, hpdr
    shapes = fields.batch_shapes(count=256, seed=3)
    us = [fields.powerlaw_field_torch(sh, seed=1000 + i, device=dev) for i, (sh, _) in enumerate(shapes)]
    tols = [t for _, t in shapes]
    total = sum(u.numel() * u.element_size() for u in us)
    D = args.batch_dict
    out, offs, sizes = hpdr.hpdr_compress_batched(us, tols, dict_size=D)   # captures + tunes
    for _ in range(2):
        hpdr.hpdr_compress_batched(us, tols, out=out, dict_size=D)
    torch.cuda.synchronize()
    k = 5
    t0 = time.perf_counter()
    for _ in range(k):
        hpdr.hpdr_compress_batched(us, tols, out=out, dict_size=D)
    bt = (time.perf_counter() - t0) / k
    bufs = [torch.empty(hpdr.hpdr_compress_bound(u.shape, u.dtype, D), dtype=torch.uint8, device=dev)
            for u in us]
    for u, t, b in zip(us, tols, bufs):
        hpdr.hpdr_compress(u, t, out=b, dict_size=D)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        for u, t, b in zip(us, tols, bufs):
            hpdr.hpdr_compress(u, t, out=b, dict_size=D)
    st = (time.perf_counter() - t0) / k
    return {"workload": "256 FP32 fields (2-D/3-D, dims log-uniform in [17,513]), rel Linf bound each "
                        "from {1e-2,1e-3,1e-4}, D = %d" % D,
            "total_bytes": total, "graph_gbs": round(total / bt / 1e9, 2),
            "sequential_gbs": round(total / st / 1e9, 2), "speedup": round(st / bt, 3),
            "streams_chosen": int(hpdr.lib().hpdr_batched_streams(hpdr.context())),
            "compression_ratio": round(total / sum(sizes), 4)}


def run_stream(args, dev):
    """1025^3 FP32 (4.3 GB) power-law field plus a tanh front, in pinned host
    memory, compressed at rel Linf 1e-3 and decompressed back: fixed 256 MiB
    slabs and the adaptive chunks of Alg. 4 (model profiled on the field)."""
    import ctypes as C
    import torch
    from paper_2503_06322_gb300 import fields, hpdr
    shape = (1025, 1025, 1025)
    ud = fields.front_field_torch(shape, seed=7, device=dev)
    h = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    h.copy_(ud)
    del ud
    torch.cuda.empty_cache()
    model = profile_model(h, args.tol)
    plane = 4 * 1025 * 1025
    planes = hpdr.pipeline_plan(model, shape[0], plane, E2E_C_INIT, E2E_C_LIMIT)
    cap = max(hpdr.streamed_bound(shape, torch.float32), hpdr.streamed_bound_plan(shape, torch.float32, planes))
    hc = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
    out = torch.empty_like(h).pin_memory()
    L = hpdr.lib()
    ctx = hpdr.context(dev.index)
    names = (C.c_char_p * 64)()
    ms = (C.c_double * 64)()
    cnt = (C.c_longlong * 64)()
    fb = h.numel() * 4

    def one(compress):
        # two warm-up calls (the first use of the pinned buffers is slow),
        # then the median of three timed calls; the middle one is profiled
        for _ in range(2):
            b = compress()
        tcs, g = [], {}
        for r in range(3):
            L.hpdr_profile_read(ctx, names, ms, cnt, 64)
            L.hpdr_profile_enable(ctx, 1 if r == 1 else 0)
            t0 = time.perf_counter()
            b = compress()
            tcs.append(time.perf_counter() - t0)
            L.hpdr_profile_enable(ctx, 0)
            n = L.hpdr_profile_read(ctx, names, ms, cnt, 64)
            if r == 1:
                g = {names[i].decode(): ms[i] for i in range(n)}
                tprof = tcs[-1]
        tc = sorted(tcs)[1]
        comp = g.get("s_compute", 0.0)
        xfer = g.get("s_h2d", 0.0) + g.get("s_d2h", 0.0)
        exposed = max(0.0, tprof * 1e3 - comp) / xfer if xfer > 0 else None
        tds = []
        hpdr.hpdr_decompress_host_streamed(b, out=out)                  # warm
        for _ in range(3):
            t0 = time.perf_counter()
            hpdr.hpdr_decompress_host_streamed(b, out=out)
            tds.append(time.perf_counter() - t0)
        td = sorted(tds)[1]
        err = (out - h).abs().max().item() / (args.tol * h.abs().max().item())
        return {"compress_host_to_host_gbs": round(fb / tc / 1e9, 2),
                "decompress_host_to_host_gbs": round(fb / td / 1e9, 2),
                "exposed_transfer_fraction": None if exposed is None else round(min(1.0, exposed), 4),
                "compute_ms": round(comp, 2), "transfer_ms": round(xfer, 2), "wall_ms": round(tc * 1e3, 2),
                "compression_ratio": round(fb / b.numel(), 4), "max_err_over_tau": round(err, 4)}

    fixed = one(lambda: hpdr.hpdr_compress_host_streamed(h, args.tol, out=hc))
    adaptive = one(lambda: hpdr.hpdr_compress_host_adaptive(h, args.tol, model, c_init=E2E_C_INIT,
                                                            c_limit=E2E_C_LIMIT, out=hc))
    adaptive["chunks_planes"] = planes
    adaptive["model"] = {k: float("%.4g" % v) for k, v in model.as_dict().items()}
    whole = hpdr.hpdr_compress(h.cuda(), args.tol).numel()
    return {"workload": "1025^3 FP32 power-law field + tanh front, pinned host, rel Linf 1e-3",
            "fixed_256MiB": fixed, "adaptive_alg4": adaptive, "whole_field_ratio": round(fb / whole, 4)}


def run_bounds(args, u):
    """The scale workload's other measured points: the timed field at relative
    Linf 1e-2 and 1e-4, and a 500 x 500 x 100 FP64 power-law field (seed 2) at
    1e-3; compress + decompress through the asynchronous calls."""
    import numpy as np
    import torch
    from paper_2503_06322_gb300 import fields, hpdr
    dev = u.device

    def leg(x, tol, steps=10):
        cap = hpdr.hpdr_compress_bound(tuple(x.shape), x.dtype)
        cbuf = torch.empty(cap, dtype=torch.uint8, device=dev)
        rec = torch.empty_like(x)
        rc = torch.zeros((steps + 3, 2), dtype=torch.int64, device=dev)
        rd = torch.zeros((steps + 3, 1), dtype=torch.int64, device=dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for i in range(3):
            hpdr.hpdr_compress_async(x, tol, cbuf, rc[i])
            hpdr.hpdr_decompress_async(cbuf, rec, rd[i])
        tc = td = 0.0
        for i in range(steps):
            e[0].record()
            hpdr.hpdr_compress_async(x, tol, cbuf, rc[3 + i])
            e[1].record()
            hpdr.hpdr_decompress_async(cbuf, rec, rd[3 + i])
            e[2].record()
            torch.cuda.synchronize()
            tc += e[0].elapsed_time(e[1])
            td += e[1].elapsed_time(e[2])
        if int((rc[:, 1] != 0).sum()) or int((rd[:, 0] != 0).sum()):
            return {"error": "device status"}
        nb = x.numel() * x.element_size()
        tau = tol * x.abs().max().item()
        return {"compress_gbs": round(nb / (tc / steps * 1e-3) / 1e9, 2),
                "decompress_gbs": round(nb / (td / steps * 1e-3) / 1e9, 2),
                "gbs": round(2 * nb / ((tc + td) / steps * 1e-3) / 1e9, 2),
                "compression_ratio": round(nb / int(rc[3, 0]), 4),
                "max_err_over_tau": round((rec - x).abs().max().item() / tau, 4)}

    res = {"workload": "the timed field at relative Linf 1e-2 and 1e-4; 500x500x100 FP64 power-law field (seed 2) "
                       "at 1e-3; compress + decompress, device-resident"}
    for tol in (1e-2, 1e-4):
        res["tol_%g" % tol] = leg(u, tol)
    f64 = torch.from_numpy(fields.powerlaw_field((500, 500, 100), seed=2, dtype=np.float64)).to(dev)
    res["fp64_500x500x100"] = leg(f64, 1e-3)
    del f64
    torch.cuda.empty_cache()
    return res


def run_l2s(args, u):
    """The timed workload in statistical L2 mode (bins bounding the expected
    RMS error by tau = tol * rms(u)) beside the max-norm bins of the headline:
    compress + decompress throughput (CUDA events over ten steps after three
    warm-ups), compression ratio and the RMS error over tau."""
    import torch
    from paper_2503_06322_gb300 import hpdr
    cap = hpdr.hpdr_compress_bound(tuple(u.shape), u.dtype)
    cbuf = torch.empty(cap, dtype=torch.uint8, device=u.device)
    rec = torch.empty_like(u)

    def step():
        b = hpdr.hpdr_compress(u, args.tol, mode=hpdr.L2_STAT, out=cbuf)
        hpdr.hpdr_decompress(b, out=rec)
        return b

    for _ in range(3):
        b = step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 10
    e0.record()
    for _ in range(n):
        b = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    fb = u.numel() * u.element_size()
    tau = args.tol * u.double().pow(2).mean().sqrt().item()
    e_rms = (rec.double() - u.double()).pow(2).mean().sqrt().item()
    return {"workload": "the timed field, statistical L2 bins, tau = tol * rms(u)",
            "gbs": round(2.0 * fb / (ms * 1e-3) / 1e9, 2), "ms_per_step": round(ms, 3),
            "compression_ratio": round(fb / b.numel(), 4), "rms_err_over_tau": round(e_rms / tau, 4),
            "max_err_over_tau": round((rec - u).abs().max().item() / tau, 4)}


def run_coords(args, u):
    """The timed field on a non-uniform grid: node coordinates clustered
    towards both ends of every dimension (a boundary-layer mesh), compressed
    and decompressed through hpdr_compress(coords=...) / hpdr_decompress at
    the headline bound; throughput over ten steps after three warm-ups
    (CUDA events), ratio and max error over tau."""
    import torch
    from paper_2503_06322_gb300 import fields, hpdr
    co = fields.node_coords(tuple(u.shape), 0, kind="stretched")
    cap = hpdr.hpdr_compress_bound(tuple(u.shape), u.dtype)
    cbuf = torch.empty(cap, dtype=torch.uint8, device=u.device)
    rec = torch.empty_like(u)

    def step():
        b = hpdr.hpdr_compress(u, args.tol, out=cbuf, coords=co)
        hpdr.hpdr_decompress(b, out=rec)
        return b

    for _ in range(3):
        b = step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 10
    e0.record()
    for _ in range(n):
        b = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    fb = u.numel() * u.element_size()
    tau = args.tol * u.abs().max().item()
    return {"workload": "the timed field on a stretched grid (x = sinh(4 (t - 1/2)) per dimension)",
            "gbs": round(2.0 * fb / (ms * 1e-3) / 1e9, 2), "ms_per_step": round(ms, 3),
            "compression_ratio": round(fb / b.numel(), 4),
            "max_err_over_tau": round((rec - u).abs().max().item() / tau, 4)}


def run_zfp(args, u):
    """Fixed-rate ZFP (Alg. 3) on the timed field at 8 and 16 bits per value:
    compress and decompress throughput (field bytes / time, CUDA events over
    ten calls after three warm-ups each), ratio and RMS error over the
    field's standard deviation."""
    import torch
    from paper_2503_06322_gb300 import hpdr
    fb = u.numel() * u.element_size()
    res = {"workload": "the timed field, fixed rate, one thread per 4^3 block"}
    std = u.double().std().item()
    for rate in (8, 16):
        cap = hpdr.zfp_bound(tuple(u.shape), rate, u.dtype)
        cbuf = torch.empty(cap, dtype=torch.uint8, device=u.device)
        rec = torch.empty_like(u)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        for _ in range(3):
            b = hpdr.hpdr_zfp_compress(u, rate, out=cbuf)
            hpdr.hpdr_zfp_decompress(b, out=rec)
        n = 10
        e0.record()
        for _ in range(n):
            b = hpdr.hpdr_zfp_compress(u, rate, out=cbuf)
        e1.record()
        for _ in range(n):
            hpdr.hpdr_zfp_decompress(b, out=rec)
        e2.record()
        torch.cuda.synchronize()
        tc, td = e0.elapsed_time(e1) / n, e1.elapsed_time(e2) / n
        err = (rec.double() - u.double()).pow(2).mean().sqrt().item() / std
        res["rate_%d" % rate] = {"compress_gbs": round(fb / (tc * 1e-3) / 1e9, 2),
                                 "decompress_gbs": round(fb / (td * 1e-3) / 1e9, 2),
                                 "compression_ratio": round(fb / b.numel(), 4), "rms_err_over_std": float("%.4g" % err)}
        del cbuf, rec
    return res


def run_lossless(args, dev):
    """The Huffman stage on its own (Alg. 2) through hpdr_lossless_compress /
    hpdr_lossless_decompress, device-resident: 1 GiB of byte keys (rounded
    Laplacian of scale 6 around 128, about 4.4 bits of entropy) and 256 Mi
    16-bit keys (rounded Laplacian of scale 40, about 7.7 bits).  Throughput =
    key bytes / time, CUDA events around five calls after one warm-up."""
    import torch
    from paper_2503_06322_gb300 import hpdr
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    res = {"workload": "1 GiB byte keys (Laplacian, scale 6) and 256 Mi 16-bit keys (Laplacian, scale 40), "
                       "synthetic, device-resident; key bytes / time"}
    for name, n, kb, scale in (("byte_keys", 1 << 30, 1, 6.0), ("keys16", 1 << 28, 2, 40.0)):
        x = torch.empty(n, device=dev).exponential_(generator=g)
        x.sub_(torch.empty(n, device=dev).exponential_(generator=g)).mul_(scale).round_()
        keys = (x + 128).clamp_(0, 255).to(torch.uint8) if kb == 1 else x.clamp_(-32768, 32767).to(torch.int16)
        del x
        buf = torch.empty(hpdr.lossless_bound(n, kb), dtype=torch.uint8, device=dev)
        out = torch.empty_like(keys)
        b = hpdr.hpdr_lossless_compress(keys, out=buf)
        hpdr.hpdr_lossless_decompress(b, out=out)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        reps = 5
        e0.record()
        for _ in range(reps):
            b = hpdr.hpdr_lossless_compress(keys, out=buf)
        e1.record()
        for _ in range(reps):
            hpdr.hpdr_lossless_decompress(b, out=out)
        e2.record()
        torch.cuda.synchronize()
        tc, td = e0.elapsed_time(e1) / reps, e1.elapsed_time(e2) / reps
        nbytes = n * kb
        res[name] = {"compress_gbs": round(nbytes / (tc * 1e-3) / 1e9, 2),
                     "decompress_gbs": round(nbytes / (td * 1e-3) / 1e9, 2),
                     "compression_ratio": round(nbytes / b.numel(), 4),
                     "bits_per_key": round(8.0 * b.numel() / n, 4),
                     "round_trip_exact": bool(torch.equal(out, keys))}
        del keys, buf, out, b
        torch.cuda.empty_cache()
    return res


def cpu_sample(args, u_host_planes, steps=1):
    """The oracle (single-threaded C, FP64) on the first planes of the field."""
    import numpy as np
    import oracle
    x = np.ascontiguousarray(u_host_planes)
    t = 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        b = oracle.compress(x, args.tol)
        oracle.decompress(b)
        t += time.perf_counter() - t0
    gbs = 2.0 * x.nbytes * steps / t / 1e9
    return gbs, t / steps, x.shape


# ---- the oracle on every host core: one unmodified single-threaded oracle
# process per core, each on its own slab of planes (spawned processes; the
# field reaches them through shared memory)
_CPU_X = None
_CPU_SHM = None


def _cpu_worker_init(shm_name, shape, dtype):
    global _CPU_X, _CPU_SHM
    import numpy as np
    from multiprocessing import shared_memory
    import oracle
    _CPU_SHM = shared_memory.SharedMemory(name=shm_name)
    _CPU_X = np.ndarray(shape, dtype=dtype, buffer=_CPU_SHM.buf)
    oracle.api._L()


def _cpu_worker_ready(_):
    return os.getpid()


def _cpu_worker(task):
    import numpy as np
    import oracle
    lo, hi, tol = task
    x = np.ascontiguousarray(_CPU_X[lo:hi])
    t0 = time.perf_counter()
    b = oracle.compress(x, tol)
    oracle.decompress(b)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample_all_cores(args, u_host_planes, steps=1, planes_per_core=32):
    """The oracle as it stands, one process per host core, each compressing
    and decompressing its own slab of `planes_per_core` planes; returns GB/s
    of the whole pool (2 x bytes / wall time of the timed map), the seconds
    per step, the number of processes and the sample's shape."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import numpy as np
    ncores = host_cores()
    n = min(u_host_planes.shape[0], ncores * planes_per_core)
    x = np.ascontiguousarray(u_host_planes[:n])
    nproc = max(1, min(ncores, n // 2))
    cuts = [round(i * n / nproc) for i in range(nproc + 1)]
    tasks = [(cuts[i], cuts[i + 1], args.tol) for i in range(nproc)]
    shm = shared_memory.SharedMemory(create=True, size=x.nbytes)
    try:
        np.ndarray(x.shape, dtype=x.dtype, buffer=shm.buf)[...] = x
        ctx = mp.get_context("spawn")
        with ctx.Pool(nproc, initializer=_cpu_worker_init, initargs=(shm.name, x.shape, x.dtype)) as pool:
            pool.map(_cpu_worker_ready, range(nproc), chunksize=1)
            t = 0.0
            for _ in range(steps):
                t0 = time.perf_counter()
                pool.map(_cpu_worker, tasks, chunksize=1)
                t += time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()
    return 2.0 * x.nbytes * steps / t / 1e9, t / steps, nproc, x.shape


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    shape = tuple(int(x) for x in args.shape.split(","))

    if args.impl == "reference":
        # the reference arm is the CPU oracle, timed as it stands on the host cores
        if rank != 0:
            return 0
        from paper_2503_06322_gb300 import fields
        import numpy as np
        per_core = 9
        planes = min(shape[0], host_cores() * per_core)
        sample = fields.powerlaw_field((planes,) + shape[1:], seed=args.seed)
        gbs, sec, ncores, shp = cpu_sample_all_cores(args, sample, steps=args.warmup + args.steps,
                                                     planes_per_core=per_core)
        desc = ("oracle compress+decompress of a %s sample of the %s workload per step, one "
                "single-threaded oracle process per host core on its own slab of %d planes" % (
                    "x".join(map(str, shp)), "x".join(map(str, shape)), per_core))
        out = {"impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(sec * 1e3, 2), "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": workload_name(shape, args.tol), "shape": list(shape)},
               "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": ncores,
                                "kind": "oracle", "sample": desc},
               "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return 0

    import torch
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    out, u, cbuf, nb = run_ours(args, rank, world, local)
    if not args.no_e2e:
        e2e = run_e2e(args, u, out)
        if world > 1:
            ms = max_over_ranks(e2e["ms_per_step"], u.device)
            e2e["value"] = round(job_gbs(world, 2.0 * u.numel() * u.element_size(), ms), 2)
        out["e2e"] = e2e
    del cbuf
    if rank == 0 and not args.no_adjoint:
        out["adjoint"] = run_adjoint(args, u.device)
    if rank == 0 and not args.no_bounds:
        try:
            out["bounds"] = run_bounds(args, u)
        except Exception as exc:       # a side leg never stops the headline line
            out["bounds"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if rank == 0 and not args.no_l2s:
        out["l2_stat"] = run_l2s(args, u)
    if rank == 0 and not args.no_zfp:
        out["zfp"] = run_zfp(args, u)
    if rank == 0 and not args.no_coords:
        try:
            out["coords"] = run_coords(args, u)
        except Exception as exc:       # a side leg never stops the headline line
            out["coords"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if rank == 0 and not args.no_batched:
        out["batched"] = run_batched(args, u.device)
    if rank == 0 and not args.no_stream:
        out["host_streamed"] = run_stream(args, u.device)
    if rank == 0 and not args.no_lossless:
        out["lossless"] = run_lossless(args, u.device)
    if rank == 0 and world == 1 and not args.no_cpu:
        planes = min(args.cpu_planes, shape[0])
        host = u[:planes].cpu().numpy()
        gbs1, sec1, shp1 = cpu_sample(args, host)
        gbsn, secn, ncores, shpn = cpu_sample_all_cores(args, host)
        out["cpu_baseline"] = {
            "value": round(gbsn, 4), "unit": "GB/s", "cores": ncores, "kind": "oracle",
            "sample": "oracle compress+decompress, one single-threaded oracle process per host core, "
                      "each on its own slab of the first %d planes (%s) of the timed field, %.1f s"
                      % (shpn[0], "x".join(map(str, shpn)), secn),
            "single_core": {"value": round(gbs1, 4), "unit": "GB/s", "cores": 1,
                            "sample": "the first %d planes (%s) in one process, %.1f s"
                                      % (planes, "x".join(map(str, shp1)), sec1)}}
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
