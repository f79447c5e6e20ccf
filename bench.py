"""Benchmark: GF(p^k) matmul field Gop/s (coefficient-plane tensor-core form
vs FP64 q-adic form) and REDQ residues/s, on one GB300 (or N replicas).

One step = one pass of the whole hot path over one batch of synthetic input:
  plane   GF(101^2), n = 4096: DQT pack of A and B (int8 centred planes ->
          bf16 operand planes) + tensor-core plane GEMM with the fused
          mod-p / mod-P epilogue.                           [headline]
Measured beside it (each a full path of its own, reported as extra keys):
  fp64    the FP64 q-adic form on the same inputs (pack -> FP64 GEMM with
          REDQ after every n_q = 6 products)
  redq    standalone REDQ over 2^28 packed words (p = 7, q = 2^10, 5 digits)
  polymul 65,536 degree-3 products over Z/7 (Alg. 1 + Alg. 2)
  large   GF(251^2), n = 16384 plane form
  batched 4096 uneven products over GF(2^8), GF(7^4), GF(31^2), one launch
  fqt     16,384 degree-500 polynomial products over Z/3 by the d-FQT (Sec. 6),
          every valid d with binary64 and 64-bit integer words (d = 0: the
          classical delayed reduction); REDQ with q = 1176, a multiple of p

`--workload NAME` runs NAME alone as the headline (same JSON contract).
`--impl reference` times the oracle (plain CPU schoolbook arithmetic) on a
bounded sample of the same workload.
Inputs are seeded synthetic data shaped like the paper's workloads.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLUSH_NOTE = "inputs larger than L2 (129 MB)"
METRIC = "GF(p^k) matmul field Gop/s, INT8-plane vs FP64 q-adic; REDQ residues/s"


def headline_config(n):
    """The headline workload's config, shared by both arms."""
    return {"workload": f"GF(101^2) n={n}: pack A,B in one launch (int8 centred planes -> bf16 "
                        f"operands) + tcgen05 plane GEMM + fused mod-p/mod-P epilogue",
            "p": 101, "k": 2, "n": n, "l2": FLUSH_NOTE}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# headline GEMM from one ncu capture of the same workload, valid only while
# the kernel's source file, "//" comments and blank lines aside, is the one
# captured (its hash below); otherwise the line reports null.
PLANE_KERNEL = "gemm_planes_pair_kernel<2,128,false>"
MEASURED_TRAFFIC = {
    PLANE_KERNEL: {
        "file": "paper_0710_0510_gb300/csrc/k_gemm_tc.cu",
        "code_sha256": "a7b0456e9cf491ed560a2a76356ba13dfd97780ae7206f98b3cbd1498f7f999e",
        "bytes": 460768256 + 30390528, "n": 4096},
    "gemm_planes_pair_kernel<2,128,true>": {
        "file": "paper_0710_0510_gb300/csrc/k_gemm_tc.cu",
        "code_sha256": "a7b0456e9cf491ed560a2a76356ba13dfd97780ae7206f98b3cbd1498f7f999e",
        "bytes": 68392448 + 12731392, "n": 4096},
}

def plane_kernel(p, n):
    """Name of the kernel the k = 2 plane GEMM dispatches to for an n x n x n
    product over GF(p^2): CTA pairs when there are two tile rows or more and
    K fits one exact FP32 chunk of 64-wide K-blocks, one CTA per tile
    otherwise (the same rule as the launcher in k_gemm_tc.cu)."""
    h = (p - 1) // 2
    chunk_kb = ((1 << 24) - 2 * p) // (h * h) // 64
    if n > 128 and (n + 63) // 64 <= chunk_kb:
        return PLANE_KERNEL
    return "gemm_planes_tc_kernel<2,128,false>"


def source_hash(path):
    """sha256 of a source file with "//" comments and blank lines removed."""
    import hashlib
    code = []
    with open(os.path.join(ROOT, path)) as fh:
        for line in fh:
            line = line.split("//", 1)[0].rstrip()
            if line:
                code.append(line)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()


def measured_traffic(kernel, n):
    """(bytes per launch, where they come from) for `kernel` at size n, or
    (None, reason) when no capture of the current source exists."""
    rec = MEASURED_TRAFFIC.get(kernel)
    if not rec or rec["bytes"] is None or rec["n"] != n:
        return None, "no ncu capture of this kernel at this size"
    if source_hash(rec["file"]) != rec["code_sha256"]:
        return None, "the kernel changed since its ncu capture"
    return rec["bytes"], (f"ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, one launch) "
                          f"of {rec['file']} with source hash {rec['code_sha256'][:16]}")


# ---------------------------------------------------------- device status --

class LegWithheld(RuntimeError):
    """A bounded wait in one of the kernels ran out during a timed leg: its
    results and its time are not valid, so the leg reports no value."""


# Returns None while no kernel has recorded a device timeout since the last
# call, else the error text; set by main() to read the library's status word.
STATUS_READER = None


def device_error():
    return STATUS_READER() if STATUS_READER is not None else None


def library_status_reader(q):
    def read():
        try:
            q.sync_status()
        except q.QadicError as exc:
            if exc.status == q.E_DEVICE_TIMEOUT:
                return str(exc)
            raise
        return None
    return read


def guarded(fn, *a, **kw):
    """fn(*a, **kw), or a withheld-leg record when a device wait expired."""
    try:
        return fn(*a, **kw)
    except LegWithheld as exc:
        return {"status": "device_timeout", "value": None, "error": str(exc)}
PQ_Q = 1176


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plane",
                    choices=["plane", "fp64", "redq", "polymul", "large", "batched", "fqt", "fold",
                             "karatsuba", "e4m3"])
    ap.add_argument("--n", type=int, default=None, help="override the matrix size")
    ap.add_argument("--words", type=int, default=1 << 28, help="REDQ sweep size (words)")
    ap.add_argument("--extras", default="all", choices=["all", "none"],
                    help="none: only the selected workload's timed step (for profiling)")
    return ap.parse_args()


# ------------------------------------------------------------ distributed --

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), dist


def reduce_max(x: float, dist) -> float:
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------- clocks --

class Clocks:
    """nvidia-smi sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs),
                "reasons": sorted(reasons), "samples": len(sms)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "bf16": d["bf16_tflops"],
                "bf16_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


def apply_clock_regime(obj, clocks, pk):
    """Every tensor roofline in `obj` is compared against the cuBLAS bf16 peak
    (times `peak_scale` for another operand type) measured in the clock
    regime this run saw: the burst figure when the SM
    clock stayed at its maximum with no power cap (the sustained cuBLAS loop
    ran power-capped at a lower clock, so it would flatter a kernel running
    at full clock), else the sustained one.  Both fractions are kept."""
    sm, smax = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    full_clock = (sm is not None and smax and sm >= 0.97 * smax
                  and "sw_power_cap" not in clocks.get("reasons", []))
    peak = pk["bf16"] if full_clock else pk["bf16_sustained"]
    regime = (f"{pk['source']} bf16 {'burst' if full_clock else 'sustained'} (cuBLAS): "
              f"SM clock {sm} of {smax} MHz during the timed region, reasons {clocks.get('reasons')}")

    def walk(x):
        if isinstance(x, dict):
            r = x.get("roofline")
            if isinstance(r, dict) and r.get("bound") == "tensor" and r.get("unit") == "TFLOP/s":
                a, sc = r["achieved"], r.get("peak_scale", 1.0)
                r.update({"peak": sc * peak, "frac": a / (sc * peak),
                          "frac_of_burst": a / (sc * pk["bf16"]),
                          "frac_of_sustained": a / (sc * pk["bf16_sustained"]),
                          "peak_source": regime if sc == 1.0 else
                          f"{regime}; x {sc} (nominal ratio of this operand type to bf16)"})
            for v in x.values():
                walk(v)

    walk(obj)


# -------------------------------------------------------------- timing --

def time_steps(torch, step, steps, warmup, dist, kernel_events=None):
    """Run `warmup` untimed steps then `steps` timed steps bracketed by a
    barrier and a synchronize; returns (total ms max over ranks, kernel ms
    per launch or None)."""
    for _ in range(warmup):
        step(None)
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    kev = [] if kernel_events else None
    start.record(stream)
    for _ in range(steps):
        step(kev)
    end.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    # the status word is sticky: an expiry in a warm-up or a timed step shows
    # here; every rank learns whether any rank saw one
    err = device_error()
    if reduce_max(1.0 if err else 0.0, dist) > 0:
        raise LegWithheld(err or "a device wait expired on another rank")
    total = reduce_max(start.elapsed_time(end), dist)
    kms = None
    if kev:
        kms = sum(a.elapsed_time(b) for a, b in kev) / len(kev)
    return total, kms


def ev_pair(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# ------------------------------------------------------------ workloads --

def make_plane_workload(torch, q, W, p, n, salt=0):
    k = 2
    h = (p - 1) // 2
    f = q.Field(p, k)
    A = W.centred_planes(k, n, n, h, index=2, salt=salt)
    B = W.centred_planes(k, n, n, h, index=2, salt=salt + 1)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    opA = torch.empty((k, n, n), dtype=torch.bfloat16, device="cuda")
    opB = torch.empty((k, n, n), dtype=torch.bfloat16, device="cuda")
    C = torch.empty((k, n, n), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    pack_events = []

    def step(kev):
        # both operands packed by one launch, then the plane GEMM
        if kev is not None:
            a, b = ev_pair(torch)
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        f.pack_operands(q.FMT_INT8_PLANES, dA, dB, n, n, n, opA, opB)
        if kev is not None:
            a.record(stream)
        f.gemm(q.PATH_PLANES, opA, opB, n, n, n, C=C)
        if kev is not None:
            b.record(stream)
            kev.append((a, b))
            pack_events.append((e0, a))

    step.pack_events = pack_events
    return f, A, B, C, step


def bench_plane(args, torch, q, W, dist, p=101, n=4096, name="plane"):
    if args.n:
        n = args.n
    f, A, B, C, step = make_plane_workload(torch, q, W, p, n)
    total, kms = time_steps(torch, step, args.steps, args.warmup, dist, kernel_events=True)
    ms = total / args.steps
    pev = step.pack_events[-args.steps:]
    pack_ms = sum(e0.elapsed_time(e1) for e0, e1 in pev) / len(pev)
    field_ops = 2.0 * n ** 3
    flops = 4 * 2.0 * n ** 3          # k^2 plane products
    pk = peaks()
    achieved = flops / (kms * 1e-3) / 1e12
    kernel = plane_kernel(p, n)
    traffic, traffic_source = measured_traffic(kernel, n)
    res = {
        "ms_per_step": ms, "value": field_ops / (ms * 1e-3) / 1e9, "n": n, "p": p,
        "kernel_ms": kms,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_sustained"],
                     "unit": "TFLOP/s", "frac": achieved / pk["bf16_sustained"],
                     "traffic": traffic, "traffic_source": traffic_source,
                     "traffic_unit": "bytes per launch (DRAM read + write)",
                     "algorithmic_bytes": 2 * 2 * n * n * 2 + 2 * n * n,
                     "kernel": kernel,
                     "peak_source": pk["source"] + " bf16 sustained (cuBLAS)"},
        "gpu_launches": 2 * args.steps,
    }
    # the pack launch on its own: k int8 planes of A and B read, k bf16
    # planes of each written
    pack_bytes = 2 * (2 * n * n * 1 + 2 * n * n * 2)
    res["pack"] = {"kernel": "pack_vec_ab", "ms": pack_ms, "algorithmic_bytes": pack_bytes,
                   "achieved_gbs": pack_bytes / (pack_ms * 1e-3) / 1e9,
                   "frac_of_hbm": pack_bytes / (pack_ms * 1e-3) / 1e9 / pk["hbm_gbs"]}
    return f, A, B, C, res


def bench_fold(args, torch, q, W, f, A, B, n, C_plane, steps=20):
    """Fold-before form on the same inputs: pack A (OPERAND_A) and B into its
    multiplication matrices (OPERAND_B_FOLD), one prime-field tensor-core
    GEMM over k K with k accumulators; bit-exact against the plane form."""
    k = f.k
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    opA = torch.empty((k, n, n), dtype=torch.bfloat16, device="cuda")
    opB = torch.empty((k, k * q.fold_n_pad(n), n), dtype=torch.bfloat16, device="cuda")
    C = torch.empty((k, n, n), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(kev):
        f.pack(q.FMT_INT8_PLANES, dA, n, n, q.FMT_OPERAND_A, out=opA)
        f.pack(q.FMT_INT8_PLANES, dB, n, n, q.FMT_OPERAND_B_FOLD, out=opB, ld_out=n)
        if kev is not None:
            a, b = ev_pair(torch)
            a.record(stream)
        f.gemm(q.PATH_FOLD, opA, opB, n, n, n, C=C, ldb=n)
        if kev is not None:
            b.record(stream)
            kev.append((a, b))

    total, kms = time_steps(torch, step, steps, 3, None, kernel_events=True)
    ms = total / steps
    pk = peaks()
    achieved = 2.0 * k * k * n ** 3 / (kms * 1e-3) / 1e12
    return {"value": 2.0 * n ** 3 / (ms * 1e-3) / 1e9, "unit": "field Gop/s", "ms_per_step": ms,
            "kernel_ms": kms, "bitexact_vs_plane": bool(torch.equal(C, C_plane)),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_sustained"],
                         "unit": "TFLOP/s", "frac": achieved / pk["bf16_sustained"],
                         "traffic": None, "kernel": "gemm_fold_tc_kernel<2,256,fold>"}}


def bench_karatsuba(args, torch, q, W, f, A, B, n, C_plane, steps=20):
    """Karatsuba form (k = 2) on the same inputs: three bf16 planes per
    operand (c_0, c_1, c_0 + c_1), three plane products on the tensor cores;
    bit-exact against the plane form."""
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    opA = torch.empty((3, n, n), dtype=torch.bfloat16, device="cuda")
    opB = torch.empty((3, n, n), dtype=torch.bfloat16, device="cuda")
    C = torch.empty((2, n, n), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(kev):
        f.pack(q.FMT_INT8_PLANES, dA, n, n, q.FMT_OPERAND_A_KARA, out=opA)
        f.pack(q.FMT_INT8_PLANES, dB, n, n, q.FMT_OPERAND_B_KARA, out=opB)
        if kev is not None:
            a, b = ev_pair(torch)
            a.record(stream)
        f.gemm(q.PATH_KARATSUBA, opA, opB, n, n, n, C=C)
        if kev is not None:
            b.record(stream)
            kev.append((a, b))

    total, kms = time_steps(torch, step, steps, 3, None, kernel_events=True)
    ms = total / steps
    pk = peaks()
    achieved = 2.0 * 3 * n ** 3 / (kms * 1e-3) / 1e12   # three plane products
    return {"value": 2.0 * n ** 3 / (ms * 1e-3) / 1e9, "unit": "field Gop/s", "ms_per_step": ms,
            "kernel_ms": kms, "bitexact_vs_plane": bool(torch.equal(C, C_plane)),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_sustained"],
                         "unit": "TFLOP/s", "frac": achieved / pk["bf16_sustained"],
                         "traffic": None, "kernel": "gemm_fold_tc_kernel<3,128,karatsuba>",
                         "flop_count": "3 plane products (2 * 3 * n^3)"}}


def make_e4m3_inputs(q, W, p=31, n=4096):
    """GF(p^2) field and the two n x n operands (int8 centred planes) of the
    e4m3 comparison."""
    k, h = 2, (p - 1) // 2
    return (q.Field(p, k), W.centred_planes(k, n, n, h, index=2, salt=31),
            W.centred_planes(k, n, n, h, index=2, salt=32))


def bench_e4m3(args, torch, q, W, p=31, n=4096, steps=20):
    """GF(p^2) with p <= 31 on both plane paths, same inputs: the bf16 plane
    path (one-launch pack + kind::f16 GEMM) and the e4m3 one (one-launch pack
    + kind::f8f6f4 GEMM, half the operand bytes, twice the tensor rate);
    bit-exact against each other."""
    k = 2
    f, A, B = make_e4m3_inputs(q, W, p, n)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    stream = torch.cuda.current_stream()
    out = {}
    Cs = {}
    pk = peaks()
    for name, dt in (("bf16", torch.bfloat16), ("e4m3", torch.uint8)):
        opA = torch.empty((k, n, n), dtype=dt, device="cuda")
        opB = torch.empty((k, n, n), dtype=dt, device="cuda")
        C = torch.empty((k, n, n), dtype=torch.uint8, device="cuda")

        def step(kev, name=name, opA=opA, opB=opB, C=C):
            # both operands packed by one launch
            f.pack_operands(q.FMT_INT8_PLANES, dA, dB, n, n, n, opA, opB, e4m3=name == "e4m3")
            if kev is not None:
                a, b = ev_pair(torch)
                a.record(stream)
            f.gemm(q.PATH_PLANES if name == "bf16" else q.PATH_PLANES_E4M3, opA, opB, n, n, n, C=C)
            if kev is not None:
                b.record(stream)
                kev.append((a, b))

        total, kms = time_steps(torch, step, steps, 3, None, kernel_events=True)
        ms = total / steps
        achieved = 4 * 2.0 * n ** 3 / (kms * 1e-3) / 1e12
        kernel = ("gemm_planes_pair_kernel<2,128,false>" if name == "bf16"
                  else "gemm_planes_pair_kernel<2,128,true>")
        traffic, traffic_source = measured_traffic(kernel, n)
        scale = 2.0 if name == "e4m3" else 1.0
        peak = pk["bf16_sustained"] * scale
        out[name] = {"value": 2.0 * n ** 3 / (ms * 1e-3) / 1e9, "unit": "field Gop/s",
                     "ms_per_step": ms, "kernel_ms": kms,
                     "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                                  "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                                  "traffic_source": traffic_source,
                                  "algorithmic_bytes": 2 * 2 * n * n * (2 if name == "bf16" else 1)
                                  + 2 * n * n,
                                  "peak_scale": scale, "kernel": kernel,
                                  "peak_source": pk["source"] + " bf16 sustained (cuBLAS)" +
                                  (" x 2, the nominal fp8/bf16 dense ratio" if name == "e4m3"
                                   else "")}}
        Cs[name] = C
    out["bitexact_e4m3_vs_bf16"] = bool(torch.equal(Cs["bf16"], Cs["e4m3"]))
    out["kernel_speedup_e4m3"] = out["bf16"]["kernel_ms"] / out["e4m3"]["kernel_ms"]
    out["workload"] = f"GF({p}^2) n={n}, int8 centred planes resident"
    return out


def bench_fp64(args, torch, q, W, f, A, B, n, reps=2):
    """FP64 q-adic form on the same inputs (pack + FP64 GEMM with REDQ)."""
    k = f.k
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    a64 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    b64 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    C = torch.empty((k, n, n), dtype=torch.uint8, device="cuda")

    def step(kev):
        f.pack(q.FMT_INT8_PLANES, dA, n, n, q.FMT_QADIC_F64, out=a64)
        f.pack(q.FMT_INT8_PLANES, dB, n, n, q.FMT_QADIC_F64, out=b64)
        f.gemm(q.PATH_FP64_QADIC, a64, b64, n, n, n, C=C)

    total, _ = time_steps(torch, step, reps, 1, None)
    ms = total / reps
    fl = 2.0 * n ** 3
    return C, {"value": fl / (ms * 1e-3) / 1e9, "unit": "field Gop/s", "ms_per_step": ms,
               "fp64_tflops": fl / (ms * 1e-3) / 1e12, "n_q": f.n_q, "log2_q": f.log2_q}


def bench_redq(args, torch, q, W, count=None, steps=10):
    count = count or args.words
    w = W.redq_words(count, 5, 10)
    d = torch.from_numpy(w).cuda()
    out = torch.empty_like(d)
    res = {}
    best = None
    for mode in (3, 1, 0, 2):
        for int_floor in (False, True):
            def step(kev):
                q.redq(7, 10, 5, d, out=out, table_mode=mode, int_floor=int_floor)
            total, _ = time_steps(torch, step, steps, 3, None)
            ms = total / steps
            gbs = 16.0 * count / (ms * 1e-3) / 1e9
            key = f"mode{mode}{'_int' if int_floor else '_lemma1'}"
            res[key] = {"ms": ms, "GB/s": gbs}
            if best is None or ms < best[1]:
                best = (key, ms)
    key, ms = best
    pk = peaks()
    gbs = 16.0 * count / (ms * 1e-3) / 1e9
    # q a multiple of p: q = 1176 = 7 * 168, the largest with q^5 <= 2^51
    # (no correction tables; Lemma 1 floors by q^j instead of shifts)
    del d
    dq = torch.from_numpy(W.redq_words_q(count, 5, PQ_Q)).cuda()
    pq = {}
    for form in ("lemma1", "int", "f32_digits"):
        def step(kev):
            q.redq_pq(7, PQ_Q, 5, dq, out=out, int_floor=form == "int",
                      f32_digits=form == "f32_digits")
        total, _ = time_steps(torch, step, steps, 3, None)
        pms = total / steps
        pgbs = 16.0 * count / (pms * 1e-3) / 1e9
        pq[form] = {
            "value": 5.0 * count / (pms * 1e-3), "unit": "residues/s", "ms": pms,
            "roofline": {"bound": "hbm", "achieved": pgbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": pgbs / pk["hbm_gbs"], "traffic": None}}
        if form == "lemma1":
            # the Lemma 1 form takes one round-up multiply a word (the floor
            # by q^2 = 1,382,976 < 2^32; the floors below 2^32 are 32-bit
            # integer ones): far from the FP64 pipe's limit, which the
            # chain of four multiplies a word reached
            pq["lemma1"]["fp64_pipe"] = fp64_pipe(1.0 * count, pms)
    del dq
    return None, out, {"value": 5.0 * count / (ms * 1e-3), "unit": "residues/s", "best": key,
                       "ms": ms, "words": count,
                       "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"],
                                    "unit": "GB/s", "frac": gbs / pk["hbm_gbs"], "traffic": None},
                       "variants": res,
                       "q_multiple_of_p": {"p": 7, "q": PQ_Q, "digits": 5, **pq}}


# FP64 multiplies (or FMAs) per second measured on this GPU: DFMA 1.01
# TFLOP/s counts two flops per instruction.
FP64_OPS_PEAK = 0.505e12


def fp64_pipe(ops, ms):
    """Second roofline for a kernel whose FP64 instructions are the limit."""
    rate = ops / (ms * 1e-3)
    return {"bound": "alu (FP64 pipe)", "ops_per_launch": ops, "achieved_Tops": rate / 1e12,
            "peak_Tops": FP64_OPS_PEAK / 1e12, "frac": rate / FP64_OPS_PEAK,
            "peak_source": "measured DFMA rate 1.01 TFLOP/s / 2 flops per instruction"}


def bench_polymul(args, torch, q, W, count=65536, steps=50):
    a, b = W.polymul_pairs(count, 7, 4)
    da = torch.from_numpy(a).cuda()
    db = torch.from_numpy(b).cuda()
    out = torch.empty((count, 7), dtype=torch.uint8, device="cuda")

    def step(kev):
        q.polymul_batched(7, 4, da, db, out=out)

    total, _ = time_steps(torch, step, steps, 3, None)
    ms = total / steps
    # the same launches replayed from a CUDA graph: the GPU time of a batch
    # without the host's per-call work (the API figure above includes it)
    graph_us = None
    try:
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step(None)   # warm-up on the capture stream
        torch.cuda.current_stream().wait_stream(side)
        with torch.cuda.graph(g):
            for _ in range(50):
                step(None)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = ev_pair(torch)
        e0.record()
        for _ in range(5):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_us = e0.elapsed_time(e1) * 1e3 / (5 * 50)
    except Exception as exc:   # capture is an extra figure only
        print(f"polymul graph capture: {exc}", file=sys.stderr)
    # labelled scaling run: 2^24 pairs (252 MB moved) for the HBM fraction
    big = 1 << 24
    ba, bb = W.polymul_pairs(big, 7, 4, salt=1)
    dba, dbb = torch.from_numpy(ba).cuda(), torch.from_numpy(bb).cuda()
    bout = torch.empty((big, 7), dtype=torch.uint8, device="cuda")

    def step_big(kev):
        q.polymul_batched(7, 4, dba, dbb, out=bout)

    tb, _ = time_steps(torch, step_big, 10, 3, None)
    msb = tb / 10
    gbs = 15.0 * big / (msb * 1e-3) / 1e9
    pk = peaks()

    def step_big_int(kev):
        q.polymul_batched(7, 4, dba, dbb, out=bout, int_words=True)

    ti, _ = time_steps(torch, step_big_int, 10, 3, None)
    msi = ti / 10
    gbi = 15.0 * big / (msi * 1e-3) / 1e9
    del dba, dbb, bout
    return a, b, out, {"value": count / (ms * 1e-3), "unit": "products/s", "us_per_batch": ms * 1e3,
                       "graph_replayed_us_per_batch": graph_us,
                       "residues_per_s": 7 * count / (ms * 1e-3),
                       "scaling_2_24_pairs": {
                           "value": big / (msb * 1e-3), "unit": "products/s", "ms": msb,
                           "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"],
                                        "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
                                        "traffic": None, "bytes_per_pair": 15},
                           "fp64_pipe": fp64_pipe(2.0 * big, msb),
                           "int64_words": {"value": big / (msi * 1e-3), "ms": msi,
                                           "GB/s": gbi, "frac": gbi / pk["hbm_gbs"]}}}


FQT_P, FQT_N, FQT_COUNT = 3, 500, 16384


def bench_fqt(args, torch, q, W, steps=20):
    """Long polynomial products (Sec. 6): 16384 pairs of degree 500 over Z/3
    (the paper's example p and N), every valid FQT degree d with binary64
    and 64-bit integer words; d = 0 is the classical delayed reduction."""
    a, b = W.polylong_pairs(FQT_COUNT, FQT_N, FQT_P)
    da = torch.from_numpy(a).cuda()
    db = torch.from_numpy(b).cuda()
    out = torch.empty((FQT_COUNT, 2 * FQT_N + 1), dtype=torch.uint8, device="cuda")
    variants = {}
    best = None
    for int_words in (False, True):
        for d in range(0, 8):
            try:
                info = q.polymul_fqt_info(FQT_P, FQT_N, d, int_words)
            except q.QadicError:
                continue

            def step(kev):
                q.polymul_fqt(FQT_P, d, da, db, out=out, int_words=int_words)

            total, _ = time_steps(torch, step, steps, 3, None)
            ms = total / steps
            key = f"{'int64' if int_words else 'f64'}_d{d}"
            wmac = info.word_products * FQT_COUNT / (ms * 1e-3)
            variants[key] = {"ms": ms, "products_per_s": FQT_COUNT / (ms * 1e-3),
                             "word_products_per_s": wmac, "log2_q": info.log2_q,
                             "n_q": info.n_q, "D_q": info.D_q}
            if not int_words:
                variants[key]["fp64_tflops"] = 2 * wmac / 1e12
            if best is None or ms < best[1]:
                best = (key, ms)
    f64 = {k: v for k, v in variants.items() if k.startswith("f64")}
    bf = min(f64, key=lambda k: f64[k]["ms"])
    return {"value": FQT_COUNT / (best[1] * 1e-3), "unit": "products/s", "best": best[0],
            "ms": best[1], "variants": variants,
            "fqt_over_classical_f64": f64["f64_d0"]["ms"] / f64[bf]["ms"],
            "fqt_over_classical_int64": variants["int64_d0"]["ms"] /
            min(v["ms"] for k, v in variants.items() if k.startswith("int64")),
            "roofline_f64": {"bound": "alu", "kernel": f"polymul_fqt_kernel<f64> ({bf})",
                             "achieved": f64[bf]["fp64_tflops"], "peak": 1.05, "unit": "TFLOP/s",
                             "frac": f64[bf]["fp64_tflops"] / 1.05, "traffic": None,
                             "peak_source": "FP64 FMA rate measured on this GPU"}}


def make_batched(torch, q, W, count=4096, salt=0):
    """4096 products, m, n, K log-uniform in [16, 256], fields GF(2^8),
    GF(7^4), GF(31^2), coefficients uniform per field."""
    import numpy as np
    fields = [q.Field(2, 8), q.Field(7, 4), q.Field(31, 2)]
    dims, fidx = W.batched_shapes(count, index=3, salt=salt)
    g = W.rng(3, salt + 17)
    sa = sb = sc = 0
    offs = []
    for (m, n, K), fi in zip(dims, fidx):
        m, n, K, k = int(m), int(n), int(K), fields[fi].k
        offs.append((sa, sb, sc))
        sa += k * m * K
        sb += k * K * n
        sc += k * m * n
    hA = np.empty(sa, np.uint8)
    hB = np.empty(sb, np.uint8)
    for (m, n, K), fi, (a, b, c) in zip(dims, fidx, offs):
        f = fields[fi]
        hA[a:a + f.k * m * K] = g.integers(0, f.p, f.k * m * K, dtype=np.uint8)
        hB[b:b + f.k * K * n] = g.integers(0, f.p, f.k * K * n, dtype=np.uint8)
    dA = torch.from_numpy(hA).cuda()
    dB = torch.from_numpy(hB).cuda()
    dC = torch.zeros(sc, dtype=torch.uint8, device="cuda")
    descs = []
    for (m, n, K), fi, (a, b, c) in zip(dims, fidx, offs):
        descs.append(q.GemmDesc(int(fi), int(m), int(n), int(K), dA.data_ptr() + a,
                                dB.data_ptr() + b, dC.data_ptr() + c, int(K), int(n), int(n), 0))
    # room for the converted operands: the tensor-core path
    ws = torch.empty(q.batched_workspace_size(descs, fields), dtype=torch.uint8, device="cuda")
    return fields, dims, fidx, offs, hA, hB, dC, descs, ws


def bench_batched(args, torch, q, W):
    fields, dims, fidx, offs, hA, hB, dC, descs, ws = make_batched(torch, q, W)
    darr = q.desc_array(descs)   # built once: the host stays ahead of the GPU

    def step(kev):
        q.batched_gemm(fields, darr, ws, graph=True)

    # the tensor-core path (the workspace holds the converted operands)
    total, _ = time_steps(torch, step, args.steps, args.warmup, None)
    ms = total / args.steps
    ops = float(sum(2 * int(m) * int(n) * int(K) for m, n, K in dims))
    flops = float(sum(2 * fields[fi].k ** 2 * int(m) * int(n) * int(K)
                      for (m, n, K), fi in zip(dims, fidx)))
    pk = peaks()
    achieved = flops / (ms * 1e-3) / 1e12
    # all three fields have p <= 31: the products run on fp8 e4m3 operands,
    # so the peak is the bf16 one times the nominal fp8 / bf16 ratio (4.5 /
    # 2.25 PFLOP/s dense)
    roofline = {"bound": "tensor", "achieved": achieved,
                "peak": 2.0 * pk["bf16_sustained"], "unit": "TFLOP/s",
                "frac": achieved / (2.0 * pk["bf16_sustained"]), "traffic": None,
                "operand_dtype": "fp8 e4m3", "peak_scale": 2.0,
                "kernel": "tc_convert_kernel + tc_products_kernel (tcgen05 kind::f8f6f4, "
                          "FP32 accumulators in tensor memory)",
                "note": "plane flops 2 k^2 m n K of the products over the time of both "
                        "launches (the conversion included)"}
    out = {"value": ops / (ms * 1e-3) / 1e9, "unit": "field Gop/s", "ms_per_step": ms,
           "products": len(descs), "field_ops": ops, "plane_flops": flops, "roofline": roofline}
    if args.extras == "none":
        return out
    # the register-staged path (work-list-only workspace): default tiles,
    # then the autotuner's choice on this batch (tuning is setup, outside
    # the timed region)
    ws_list = torch.empty(q.batched_workspace_size(descs), dtype=torch.uint8, device="cuda")

    def step_reg(kev):
        q.batched_gemm(fields, darr, ws_list, graph=True)

    for k in range(1, 9):
        q.batched_select_tiles(k, -1)
    tot_r, _ = time_steps(torch, step_reg, args.steps, args.warmup, None)
    ms_register = tot_r / args.steps
    chosen = q.batched_autotune(fields, descs, ws_list, reps=3)
    tot_rt, _ = time_steps(torch, step_reg, args.steps, args.warmup, None)
    ms_register_tuned = tot_rt / args.steps
    del ws_list
    # one launch per product through the same entry point (no graph)
    single_ws = torch.empty(max(q.batched_workspace_size([d], fields) for d in descs),
                            dtype=torch.uint8, device="cuda")

    def step_each(kev):
        for d in descs:
            q.batched_gemm(fields, [d], single_ws)

    tot1, _ = time_steps(torch, step_each, 2, 1, None)
    ms1 = tot1 / 2
    # the same launches with an event pair around each: the summed GPU time
    # of the per-product kernels, without the host's work-list building
    stream = torch.cuda.current_stream()
    evs = [ev_pair(torch) for _ in descs]
    for (e0, e1), d in zip(evs, descs):
        e0.record(stream)
        q.batched_gemm(fields, [d], single_ws)
        e1.record(stream)
    torch.cuda.synchronize()
    ms1_gpu = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    out.update({
            "one_launch_per_product": {"value": ops / (ms1 * 1e-3) / 1e9, "ms": ms1,
                                       "ms_gpu_only": ms1_gpu,
                                       "note": "ms: wall time of 4096 API calls (host builds a "
                                               "work list per call); ms_gpu_only: summed event "
                                               "time of the 4096 launches"},
            "speedup_vs_per_product_gpu_only": ms1_gpu / ms,
            "speedup_vs_per_product": ms1 / ms,
            "register_staged": {"ms_default_tiles": ms_register,
                                "ms_autotuned": ms_register_tuned,
                                "autotuned_tiles": {str(k): dict(zip(("bm", "bn", "bk"),
                                                                     q.batched_tile_configs(k)[c][:3]))
                                                    for k, c in chosen.items()},
                                "note": "work-list-only workspace (and the allocation-free "
                                        "call): operands staged through registers, mma.sync"}})
    return out


def bench_fp64_gf27(args, torch, q, W, n=1024):
    """GF(3^3), n = 1024, log-coded inputs: pack (log -> q-adic FP64 word by
    table lookup) + FP64 q-adic GEMM with REDQ every n_q = 85 products."""
    f, A, B, C, step = make_fp64_gf27(torch, q, W, n)
    total, _ = time_steps(torch, step, args.steps, args.warmup, None)
    ms = total / args.steps
    fl = 2.0 * n ** 3
    return {"value": fl / (ms * 1e-3) / 1e9, "unit": "field Gop/s", "ms_per_step": ms,
            "n_q": f.n_q, "log2_q": f.log2_q,
            "roofline": {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": 1.05,
                         "unit": "TFLOP/s", "frac": fl / (ms * 1e-3) / 1e12 / 1.05,
                         "traffic": None, "kernel": "gemm_f64_kernel<3>",
                         "peak_source": "FP64 FMA rate measured on this GPU (DMMA 1.05, DFMA 1.01, "
                                        "cuBLAS 1.10 TFLOP/s)"}}


def make_fp64_gf27(torch, q, W, n=1024):
    f = q.Field(3, 3)
    A = W.log_matrix(n, n, 27, index=1, salt=0)
    B = W.log_matrix(n, n, 27, index=1, salt=1)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    a64 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    b64 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    C = torch.empty((3, n, n), dtype=torch.uint8, device="cuda")

    def step(kev):
        f.pack(q.FMT_LOG, dA, n, n, q.FMT_QADIC_F64, out=a64)
        f.pack(q.FMT_LOG, dB, n, n, q.FMT_QADIC_F64, out=b64)
        f.gemm(q.PATH_FP64_QADIC, a64, b64, n, n, n, C=C)

    return f, A, B, C, step


def e2e_plane(args, torch, q, W, f, A, B, n):
    """Same metric through qadic_matmul_host: pinned host inputs, H2D copies,
    pack, GEMM, D2H of C, all inside the timed region."""
    k = f.k
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.empty((k, n, n), dtype=torch.uint8).pin_memory()
    ws = torch.empty(f.matmul_workspace_size(q.PATH_PLANES, q.FMT_INT8_PLANES, n, n, n),
                     dtype=torch.uint8, device="cuda")

    def step(kev):
        f.matmul_host(q.PATH_PLANES, q.FMT_INT8_PLANES, hA, hB, hC, n, n, n, ws)

    total, _ = time_steps(torch, step, max(3, args.steps // 2), 2, None)
    ms = total / max(3, args.steps // 2)
    return hC, {"value": 2.0 * n ** 3 / (ms * 1e-3) / 1e9, "unit": "field Gop/s",
                "h2d_bytes_per_step": int(A.nbytes + B.nbytes), "d2h_bytes_per_step": int(hC.numel()),
                "ms_per_step": ms}


# ------------------------------------------------------------ CPU oracle --

def cpu_baseline_plane(p, n, target_s=12.0):
    """Oracle (plain C schoolbook, OpenMP) on a bounded sample of the n x n
    workload: whole output rows, field Gop/s scaled by the ops done."""
    import numpy as np
    import oracle
    from paper_0710_0510_gb300 import workloads as W
    oracle.build()
    k = 2
    h = (p - 1) // 2
    poly = oracle.smallest_irreducible(p, k)
    B = W.centred_planes(k, n, n, h, index=2, salt=1)
    Bt = np.ascontiguousarray(np.transpose(B, (1, 2, 0)))          # (K, n, k)
    rows = 2
    spent = 0.0
    done = 0
    while True:
        A = W.centred_planes(k, rows, n, h, index=2, salt=0)        # rows of the same law
        Ar = np.ascontiguousarray(np.transpose(A, (1, 2, 0)))
        t0 = time.perf_counter()
        oracle.gemm(p, poly, Ar, Bt)
        dt = time.perf_counter() - t0
        spent, done = dt, rows
        if dt > target_s / 4 or rows >= n:
            break
        rows = min(n, max(rows * 2, int(rows * target_s / 4 / max(dt, 1e-3))))
    ops = 2.0 * done * n * n
    return {"value": ops / spent / 1e9, "unit": "field Gop/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{done} of {n} output rows of the n={n} GF({p}^2) product "
                                        f"({spent:.1f} s)"}


def cpu_baselines_all():
    """The oracle as it stands, on bounded samples of every workload, on all
    host cores (and on one core for the polynomial and GF(3^3) workloads).
    Rates are scaled to each workload's unit by the work the sample did."""
    import numpy as np
    import oracle
    from paper_0710_0510_gb300 import workloads as W
    oracle.build()
    cores = oracle.num_threads()
    out = {"cores": cores, "kind": "oracle"}

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    a, b = W.polymul_pairs(65536, 7, 4)
    for th, tag in ((cores, "all_cores"), (1, "one_core")):
        oracle.set_threads(th)
        dt = timed(lambda: oracle.polymul(7, a, b))
        out[f"polymul_65536_z7_{tag}"] = {"value": 65536 / dt, "unit": "products/s",
                                          "sample": "all 65,536 pairs", "s": dt}
    oracle.set_threads(cores)
    poly27 = oracle.smallest_irreducible(3, 3)
    T = oracle.antilog(3, poly27)
    A = T[W.log_matrix(1024, 1024, 27, index=1, salt=0).astype(np.int64)]
    B = T[W.log_matrix(1024, 1024, 27, index=1, salt=1).astype(np.int64)]
    for th, tag, rows in ((cores, "all_cores", 1024), (1, "one_core", 64)):
        oracle.set_threads(th)
        dt = timed(lambda: oracle.gemm(3, poly27, A[:rows], B))
        out[f"gf27_n1024_{tag}"] = {"value": 2.0 * rows * 1024 * 1024 / dt / 1e9,
                                    "unit": "field Gop/s", "s": dt,
                                    "sample": f"{rows} of 1024 output rows"}
    oracle.set_threads(cores)
    # batched: a sample of the 4096 products (same generator as the GPU run)
    dims, fidx = W.batched_shapes(4096, index=3, salt=0)
    fields = [(2, oracle.smallest_irreducible(2, 8)), (7, oracle.smallest_irreducible(7, 4)),
              (31, oracle.smallest_irreducible(31, 2))]
    rng = np.random.default_rng(1)
    ops, spent = 0.0, 0.0
    for i in range(0, 4096, 32):
        m, n, K = (int(x) for x in dims[i])
        p, poly = fields[int(fidx[i])]
        k = len(poly) - 1
        Ai = rng.integers(0, p, (m, K, k))
        Bi = rng.integers(0, p, (K, n, k))
        spent += timed(lambda: oracle.gemm(p, poly, Ai, Bi))
        ops += 2.0 * m * n * K
    out["batched_4096"] = {"value": ops / spent / 1e9, "unit": "field Gop/s", "s": spent,
                           "sample": "128 of the 4096 products (every 32nd)"}
    # GF(251^2) n = 16384: 8 output rows, extrapolated by the op count
    h = 125
    poly251 = oracle.smallest_irreducible(251, 2)
    B = np.ascontiguousarray(np.transpose(W.centred_planes(2, 16384, 16384, h, index=2, salt=1),
                                          (1, 2, 0)))
    A = np.ascontiguousarray(np.transpose(W.centred_planes(2, 8, 16384, h, index=2, salt=0),
                                          (1, 2, 0)))
    dt = timed(lambda: oracle.gemm(251, poly251, A, B))
    out["gf251_2_n16384"] = {"value": 2.0 * 8 * 16384 * 16384 / dt / 1e9, "unit": "field Gop/s",
                             "s": dt, "sample": "8 of 16384 output rows (extrapolated)"}
    del A, B
    w = W.redq_words(1 << 24, 5, 10)
    dt = timed(lambda: oracle.redq(7, 1024, 4, w))
    out["redq_2_24_words"] = {"value": 5.0 * (1 << 24) / dt, "unit": "residues/s", "s": dt,
                              "sample": "2^24 of the 2^28 words"}
    pa, pb = W.polylong_pairs(1024, FQT_N, FQT_P)
    dt = timed(lambda: oracle.polymul_long(FQT_P, pa, pb))
    out["polymul_long_p3_n500"] = {"value": 1024 / dt, "unit": "products/s", "s": dt,
                                   "sample": "1024 of the 16384 pairs"}
    return out


def run_reference(args):
    rank, world, dist = 0, 1, None
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
    p, n = (101, args.n or 4096)
    vals = []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline_plane(p, n, target_s=2.0)
    for _ in range(args.steps):
        cb = cpu_baseline_plane(p, n, target_s=5.0)
        vals.append(cb["value"])
    value = statistics.median(vals)
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "field Gop/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": headline_config(n),
            "runs": "the oracle (plain C schoolbook arithmetic, OpenMP) on bounded row samples "
                    "of the same product",
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "field Gop/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ main --

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, dist = dist_setup()
    import torch
    import paper_0710_0510_gb300 as q
    from paper_0710_0510_gb300 import workloads as W
    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    dev_index = torch.cuda.current_device()
    uuid = getattr(torch.cuda.get_device_properties(dev_index), "uuid", None)
    smi_id = f"GPU-{uuid}" if uuid else str(dev_index)
    q.lib()
    global STATUS_READER
    STATUS_READER = library_status_reader(q)
    STATUS_READER()   # start from a clear status word

    line = {"metric": METRIC,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic (seeded, shaped like the paper's workloads)"}
    extras = {}
    try:
        with Clocks(smi_id) as clk:
            run_workload(args, torch, q, W, dist, rank, world, line, extras)
    except LegWithheld as exc:
        # the headline leg itself saw a device timeout: no value is reported
        line.update({"value": None, "status": "device_timeout", "error": str(exc),
                     "unit": line.get("unit")})
        line.setdefault("config", {"workload": args.workload})
    line["clocks"] = clk.summary()
    if args.workload == "plane" and rank == 0 and args.extras == "all" and "status" not in line:
        run_plane_extras(args, torch, q, W, extras)
    if rank == 0:
        if args.workload == "plane" and args.extras == "all":
            line["cpu_baseline"] = cpu_baseline_plane(101, line["config"]["n"])
            line["cpu_baselines_all"] = cpu_baselines_all()
        line.update(extras)
        apply_clock_regime(line, line.get("clocks", {}), peaks())
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_workload(args, torch, q, W, dist, rank, world, line, extras):
    """The selected workload's timed leg (fills `line`), with the plane
    workload's same-input comparisons in `extras`."""
    if args.workload == "plane":
        f, A, B, C, res = bench_plane(args, torch, q, W, dist)
        n = res["n"]
        line.update({"value": res["value"] * world, "unit": "field Gop/s",
                     "ms_per_step": res["ms_per_step"], "dtype": "bf16 (exact small integers), "
                     "f32 accumulate", "roofline": res["roofline"],
                     "gpu_launches": res["gpu_launches"]})
        line["config"] = headline_config(n)
        extras["pack"] = res["pack"]
        if rank == 0 and args.extras == "all":
            def fp64_leg():
                C64, fp = bench_fp64(args, torch, q, W, f, A, B, n)
                fp["bitexact_vs_plane"] = bool(torch.equal(C64, C))
                return fp
            fp = guarded(fp64_leg)
            extras["fp64_qadic"] = fp
            if fp.get("value"):
                extras["plane_over_fp64"] = res["value"] / fp["value"]
            extras["fold_before"] = guarded(bench_fold, args, torch, q, W, f, A, B, n, C)
            extras["karatsuba"] = guarded(bench_karatsuba, args, torch, q, W, f, A, B, n, C)

            def e2e_leg():
                hC, e2e = e2e_plane(args, torch, q, W, f, A, B, n)
                e2e["bitexact"] = bool(torch.equal(hC, C.cpu()))
                return e2e
            line["e2e"] = guarded(e2e_leg)
    elif args.workload == "redq":
        d, out, r = bench_redq(args, torch, q, W)
        line.update({"value": r["value"] * world, "unit": "residues/s", "ms_per_step": r["ms"],
                     "dtype": "f64 words, integer REDQ", "roofline": r["roofline"],
                     "gpu_launches": args.steps})
        line["config"] = {"workload": f"REDQ sweep: {args.words} FP64 words, 5 digits, p=7, "
                          "q=2^10", "l2": FLUSH_NOTE}
        extras["redq_variants"] = r["variants"]
        extras["q_multiple_of_p"] = r["q_multiple_of_p"]
    elif args.workload == "polymul":
        a, b, out, r = bench_polymul(args, torch, q, W)
        line.update({"value": r["value"] * world, "unit": "products/s",
                     "ms_per_step": r["us_per_batch"] / 1e3, "dtype": "f64 product, u64 REDQ",
                     "gpu_launches": 50})
        line["config"] = {"workload": "65,536 pairs of degree-3 polynomials over Z/7, q=2^8"}
        extras["scaling_2_24_pairs"] = r["scaling_2_24_pairs"]
        extras["graph_replayed_us_per_batch"] = r["graph_replayed_us_per_batch"]
    elif args.workload in ("fold", "karatsuba"):
        f, A, B, C, step = make_plane_workload(torch, q, W, 101, args.n or 4096)
        step(None)
        n = args.n or 4096
        fn = bench_fold if args.workload == "fold" else bench_karatsuba
        r = fn(args, torch, q, W, f, A, B, n, C, steps=args.steps)
        line.update({"value": r["value"] * world, "unit": "field Gop/s",
                     "ms_per_step": r["ms_per_step"], "dtype": "bf16 exact, f32 accumulate",
                     "roofline": r["roofline"], "gpu_launches": 3 * args.steps})
        line["config"] = {"workload": f"GF(101^2) n={n}, {args.workload} form", "p": 101,
                          "k": 2, "n": n, "l2": FLUSH_NOTE}
        extras["bitexact_vs_plane"] = r["bitexact_vs_plane"]
    elif args.workload == "e4m3":
        n = args.n or 4096
        r = bench_e4m3(args, torch, q, W, n=n, steps=args.steps)
        e = r["e4m3"]
        line.update({"value": e["value"] * world, "unit": "field Gop/s",
                     "ms_per_step": e["ms_per_step"], "dtype": "fp8 e4m3 exact, f32 accumulate",
                     "roofline": e["roofline"], "gpu_launches": 2 * args.steps})
        line["config"] = {"workload": f"GF(31^2) n={n}: pack A, B in one launch to e4m3 planes + "
                          "tcgen05 kind::f8f6f4 plane GEMM + fused epilogue", "p": 31, "k": 2, "n": n,
                          "l2": "each step writes and reads more than L2 (129 MB)"}
        extras.update({k_: r[k_] for k_ in ("bf16", "bitexact_e4m3_vs_bf16", "kernel_speedup_e4m3")})
    elif args.workload == "fqt":
        r = bench_fqt(args, torch, q, W)
        line.update({"value": r["value"] * world, "unit": "products/s", "ms_per_step": r["ms"],
                     "dtype": "f64 or int64 q-adic words", "roofline": r["roofline_f64"],
                     "gpu_launches": 1})
        line["config"] = {"workload": f"{FQT_COUNT} pairs of degree-{FQT_N} polynomials over "
                          f"Z/{FQT_P}, d-FQT (d = 0: classical delayed reduction)"}
        extras.update({k: r[k] for k in ("best", "variants", "fqt_over_classical_f64",
                                         "fqt_over_classical_int64")})
    elif args.workload == "large":
        f, A, B, C, res = bench_plane(args, torch, q, W, dist, p=251, n=args.n or 16384)
        line.update({"value": res["value"] * world, "unit": "field Gop/s",
                     "ms_per_step": res["ms_per_step"], "dtype": "bf16 exact, f32 accumulate",
                     "roofline": res["roofline"], "gpu_launches": res["gpu_launches"]})
        line["config"] = {"workload": f"GF(251^2) n={res['n']} plane form", "p": 251, "k": 2,
                          "n": res["n"], "l2": FLUSH_NOTE}
    elif args.workload == "batched":
        r = bench_batched(args, torch, q, W)
        line.update({"value": r["value"] * world, "unit": "field Gop/s",
                     "ms_per_step": r["ms_per_step"], "dtype": "fp8 e4m3 exact, f32 accumulate",
                     "roofline": r["roofline"], "gpu_launches": 2 * args.steps})
        line["config"] = {"workload": "4096 products, m,n,K log-uniform in [16,256], fields "
                          "GF(2^8), GF(7^4), GF(31^2); conversion + one persistent tcgen05 "
                          "launch, graph-replayed"}
        extras.update({k: r[k] for k in ("one_launch_per_product", "speedup_vs_per_product",
                                         "speedup_vs_per_product_gpu_only",
                                         "products", "register_staged") if k in r})
    elif args.workload == "fp64":
        r = bench_fp64_gf27(args, torch, q, W)
        line.update({"value": r["value"] * world, "unit": "field Gop/s",
                     "ms_per_step": r["ms_per_step"], "dtype": "f64",
                     "roofline": r["roofline"], "gpu_launches": 3 * args.steps})
        line["config"] = {"workload": "GF(3^3) n=1024 log-coded: pack (log->q-adic table) + "
                          "FP64 q-adic GEMM, REDQ every n_q=85 products"}
    else:
        raise SystemExit(f"workload {args.workload} not available")


def run_plane_extras(args, torch, q, W, extras):
    """Every other workload, each its own guarded leg, beside the headline."""
    def pick(keys):
        return lambda r: {k: r[k] for k in keys} if "status" not in r else r

    r2 = guarded(lambda: bench_redq(args, torch, q, W)[2])
    extras["redq"] = pick(("value", "unit", "best", "ms", "roofline", "q_multiple_of_p"))(r2)
    extras["polymul"] = guarded(lambda: bench_polymul(args, torch, q, W)[3])
    bb = guarded(bench_batched, args, torch, q, W)
    extras["batched"] = pick(("value", "unit", "ms_per_step", "one_launch_per_product",
                              "speedup_vs_per_product_gpu_only", "speedup_vs_per_product",
                              "roofline", "register_staged"))(bb)
    g27 = guarded(bench_fp64_gf27, args, torch, q, W)
    extras["polymul_fqt_p3_n500"] = guarded(bench_fqt, args, torch, q, W)
    extras["fp64_gf27_n1024"] = g27
    del bb
    torch.cuda.empty_cache()

    def large_leg():
        lf, lA, lB, lC, lres = bench_plane(argparse.Namespace(n=None, steps=5, warmup=2), torch, q,
                                           W, None, p=251, n=16384)
        return {"value": lres["value"], "unit": "field Gop/s", "ms_per_step": lres["ms_per_step"],
                "kernel_ms": lres["kernel_ms"], "roofline": lres["roofline"]}
    extras["large_gf251_2_n16384"] = guarded(large_leg)
    torch.cuda.empty_cache()
    extras["e4m3_gf31_2_n4096"] = guarded(bench_e4m3, args, torch, q, W)
    torch.cuda.empty_cache()


if __name__ == "__main__":
    sys.exit(main())
