"""Throughput of the per-token CDF step on one GB300 (or N replicas).

Workload (default): the full-size model (30 layers, hidden 576, 9/3 heads,
FFN 1536, vocabulary 49,152), BF16 weights random-init seed 1, FP32 mix /
bias, one 8,192-token seeded Zipf/Markov stream, 2,048-token KV window
sliding by 512, confidence skip off.  One "step" compresses the whole stream:
every token runs the model, the biased softmax, the N-gram, the mix, the CDF
quantiser and the head / mixer / N-gram updates (the GPU half ends at the
coder's interval per token; the end-to-end number includes the host coder).

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "tokens/s compressed on 1 GB300 (batched vs plain) at bpb within 0.5% of FP64 oracle"

# prefill_rows: the encoder runs the model over up to this many (stream,
# position) rows per forward pass (0: one position per step).  It changes no
# coded bit; the decoder always steps one position at a time.
WORKLOADS = {
    # one stream, the full-size model in BF16 weights (the headline
    # configuration): tensor-core path, encoder prefill of 512 positions
    "full_bf16_single": dict(shape=S.FULL, fmt="bf16", seed=1, n_streams=1, length=8192, path="tc",
                             prefill_rows=4096),
    # the same, one position per model step (what its decoder runs)
    "full_bf16_single_tc_stepwise": dict(shape=S.FULL, fmt="bf16", seed=1, n_streams=1, length=8192, path="tc",
                                         prefill_rows=0),
    # the CUDA-core GEMV path (FP32 activations), with and without prefill
    "full_bf16_single_gemv": dict(shape=S.FULL, fmt="bf16", seed=1, n_streams=1, length=8192, path="gemv",
                                  prefill_rows=4096),
    "full_bf16_single_stepwise": dict(shape=S.FULL, fmt="bf16", seed=1, n_streams=1, length=8192, path="gemv",
                                      prefill_rows=0),
    # the plain single-stream FP32 path (the denominator of "batched vs plain")
    "full_fp32_single": dict(shape=S.FULL, fmt="fp32", seed=1, n_streams=1, length=8192, path="gemv",
                             prefill_rows=0),
    "small_fp32_single": dict(shape=S.SMALL, fmt="fp32", seed=0, n_streams=1, length=1024, path="gemv",
                              prefill_rows=0),
    # 256 streams with log-uniform lengths 512..16,384 on the tensor-core path
    "batched_bf16_tc": dict(shape=S.FULL, fmt="bf16", seed=2, n_streams=256, lengths=(512, 16384), path="tc",
                            prefill_rows=4096),
    # the same 256 streams cut to their first 512 tokens: the batch stays full
    "batched_bf16_tc_512": dict(shape=S.FULL, fmt="bf16", seed=2, n_streams=256, lengths=(512, 16384),
                                cap=512, path="tc", prefill_rows=4096),
    "batched_bf16_tc_512_stepwise": dict(shape=S.FULL, fmt="bf16", seed=2, n_streams=256, lengths=(512, 16384),
                                         cap=512, path="tc", prefill_rows=0),
    # a small case of the batched prefill for profiling: 32 streams x 256
    # tokens, 4,096 forward rows (128 positions per stream), 1.5 GB of KV
    "prof_tc_32x256": dict(shape=S.FULL, fmt="bf16", seed=2, n_streams=32, length=256, path="tc",
                           prefill_rows=4096),
    # a small case of the single-stream prefill for profiling: the headline's
    # stream and kernels with 512 forward rows (about 1 GB on the device)
    "prof_single_p512": dict(shape=S.FULL, fmt="bf16", seed=1, n_streams=1, length=8192, path="tc",
                             prefill_rows=512),
    # FP8 E4M3 weights, 1,024 streams x 4,096 tokens (first 256 tokens per stream)
    "fp8_tc_1024_256": dict(shape=S.FULL, fmt="fp8", seed=4, n_streams=1024, length=4096, cap=256, path="tc",
                            prefill_rows=4096),
    # the same 1,024 FP8 streams cut to their first 1,024 tokens: the batch
    # stays full and the windows grow to half the context
    "fp8_tc_1024x1024": dict(shape=S.FULL, fmt="fp8", seed=4, n_streams=1024, length=4096, cap=1024, path="tc",
                             prefill_rows=4096),
    # the precision workload as stated: 1,024 FP8 streams x 4,096 tokens
    "fp8_tc_1024x4096": dict(shape=S.FULL, fmt="fp8", seed=4, n_streams=1024, length=4096, path="tc",
                             prefill_rows=4096),
    # differentiation: 64 BF16 streams x 4,096 tokens, the head and mixer
    # updated by the mixed-NLL gradient (hand-written backward in the loop)
    "diff_bf16_tc_64x4096": dict(shape=S.FULL, fmt="bf16", seed=3, n_streams=64, length=4096, path="tc",
                                 prefill_rows=4096, rule="mixed_nll"),
}

# The headline metric's denominator and numerators: batched BF16 / FP8
# throughput as a multiple of the plain single-stream FP32 path.
PLAIN = "full_fp32_single"
BATCHED = ("batched_bf16_tc", "fp8_tc_1024x1024")


# Kernels of one decode step on the tensor-core path with BF16 weights: the
# embedding; per layer the RMSNorm operand, QKV, attention (with the append),
# O, RMSNorm operand, gate/up and down; the final RMSNorm operand, the LM
# head; the vocabulary step and the coder's device search.
DECODE_STEP_LAUNCHES = 1 + 7 * 30 + 2 + 2


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_lengths(wl, world: int = 1):
    """Lengths of the whole job: world x n_streams streams (weak scaling)."""
    n = wl["n_streams"] * world
    if "lengths" in wl:
        lo, hi = wl["lengths"]
        lens = S.stream_lengths(wl["seed"], n, lo, hi)
    else:
        lens = np.full(n, wl["length"], dtype=np.int64)
    if "cap" in wl:
        lens = np.minimum(lens, wl["cap"])
    return lens


def _stream_job(args):
    seed, j, n, vocab = args
    return S.token_stream(seed, j, n, vocab)


def workload_streams(wl, world: int = 1, rank: int = 0):
    """This rank's share of the job's streams (longest-first bin packing).
    Large workloads are drawn by a pool of spawned worker processes (the
    generator is a per-token Python loop)."""
    from paper_2602_19626_gb300.partition import partition_streams
    shape = wl["shape"]
    lens = workload_lengths(wl, world)
    mine = sorted(partition_streams(lens, world)[rank])
    jobs = [(wl["seed"], j, int(lens[j]), shape.vocab) for j in mine]
    if sum(int(lens[j]) for j in mine) < 200_000:
        return [_stream_job(a) for a in jobs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_stream_job, jobs, chunksize=8))


# ------------------------------------------------------------- oracle (CPU)

def oracle_rate(wl, budget_s: float, first_tokens: int | None = None):
    """FP64 oracle on the host cores: tokens/s over the first tokens of the
    workload's first stream, sized to take about budget_s seconds.  Returns
    (tokens, seconds, interval bits): the last is sum -log2((hi - lo) / T)
    over the coded intervals, the code length the coder's intervals give."""
    from oracle.compress import StepConfig, StreamState
    from oracle.model import Model
    shape = wl["shape"]
    toks = S.token_stream(wl["seed"], 0, int(workload_lengths(wl)[0]), shape.vocab)
    model = Model(shape, S.weights(shape, wl["seed"]), wl["fmt"])
    cfg = StepConfig(rule=wl.get("rule", "paper"))
    st = StreamState.new(model, cfg)
    t0 = time.perf_counter()
    n = 0
    bits = 0.0
    for t in toks:
        _, _, cdf = st.predict()
        st.update(int(t))
        bits += -np.log2((int(cdf[int(t) + 1]) - int(cdf[int(t)])) / cfg.T)
        n += 1
        el = time.perf_counter() - t0
        if first_tokens is not None:
            if n >= first_tokens:
                break
        elif el >= budget_s:
            break
    el = time.perf_counter() - t0
    return n, el, bits


def interval_bits(iv_row, n: int, log2_total: int = 24) -> float:
    """sum -log2((hi - lo) / T) over the first n coded intervals of one stream."""
    lo = iv_row[:n, 0].astype(np.float64)
    hi = iv_row[:n, 1].astype(np.float64)
    return float(np.sum(log2_total - np.log2(hi - lo)))


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def blas_threads() -> int:
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count() or 1


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    budget = 8.0
    S.weights(wl["shape"], wl["seed"])          # generate outside the timed steps
    for _ in range(args.warmup):
        oracle_rate(wl, 0.0, first_tokens=2)
    n_tot, t_tot = 0, 0.0
    for _ in range(args.steps):
        n, el, _ = oracle_rate(wl, budget)
        n_tot += n
        t_tot += el
    v = n_tot / t_tot
    sample = (f"first {n_tot // max(args.steps, 1)} tokens of the first stream per step "
              f"(about {budget:.0f} s each), FP64 oracle on {wl['fmt']}-dequantised weights")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "tokens/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_tot / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "model": "smollm2-135m-shape random-init",
                   "streams": wl["n_streams"], "tokens": int(workload_lengths(wl).sum())},
        "cpu_baseline": {"value": v, "unit": "tokens/s", "cores": blas_threads(), "cpu": cpu_model(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "tokens/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    """(HBM GB/s, dense BF16 tensor TFLOP/s burst, source)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


# CUDA-core FP32 peak: SMs x 128 FP32 lanes x 2 flops per fused multiply-add
# x SM clock (the maximum SM clock of the part, 2,070 MHz)
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(n_sm: int, sm_mhz: float) -> float:
    return n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


TC_KINDS = {"gemv_qkv", "gemv_o", "gemv_gate_up", "gemv_down", "lm_head"}


def roofline_of(kind: dict, path: str, fmt: str, n_sm: int, sm_max_mhz: float) -> dict:
    """The bound of one traced kernel kind from its arithmetic intensity:
    HBM below the ridge, else the tensor pipe (projections on the
    tensor-core path) or the CUDA-core FP32 pipe (everything else)."""
    hbm, bf16, src = measured_peaks()
    per_ms = kind["ms"] / max(kind["launches"], 1)
    per_bytes = kind["bytes"] / max(kind["launches"], 1)
    per_flops = kind.get("flops", 0.0) / max(kind["launches"], 1)
    ai = per_flops / per_bytes if per_bytes else 0.0
    # projections on the tensor-core path, and the attention over a BF16 KV
    # cache (BF16 / FP8 weights), run on the tensor pipe
    if (path == "tc" and kind["name"] in TC_KINDS) or (kind["name"] == "attn" and fmt != "fp32"):
        # FP8 peak = measured BF16 x the nominal 2x ratio of the FP8 rate
        fp8_gemm = fmt == "fp8" and kind["name"] != "attn"
        peak_c, unit_peak = (bf16 * 2 if fp8_gemm else bf16), "tensor"
        peak_src = f"{src} bf16{' x2 (fp8 nominal ratio)' if fp8_gemm else ''}"
    else:
        peak_c, unit_peak = fp32_peak_tflops(n_sm, sm_max_mhz), "alu"
        peak_src = f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x {sm_max_mhz:.0f} MHz"
    ridge = peak_c * 1e12 / (hbm * 1e9)
    out = {"kernel": kind["name"], "ms_per_launch": per_ms, "bytes_per_launch": per_bytes,
           "flops_per_launch": per_flops, "intensity": ai}
    if ai > ridge:
        achieved = per_flops / (per_ms / 1000.0) / 1e12
        out.update({"bound": unit_peak, "achieved": achieved, "peak": peak_c, "unit": "TFLOP/s",
                    "frac": achieved / peak_c, "peak_source": peak_src})
    else:
        achieved = per_bytes / (per_ms / 1000.0) / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "peak_source": src})
    return out


def ncu_traffic(kind: str, workload: str):
    """DRAM bytes per launch of `kind` from the committed ncu summary, or None
    when there is none or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    h = kernel_sources_hash(kind)
    with open(path) as fh:
        for line in fh:
            f = line.split()
            if len(f) >= 4 and not line.startswith("#") and f[0] == kind and f[2] == workload and f[3] == h:
                return float(f[1])
    return None


# The device sources each traced kernel kind is built from; a kind not listed
# is keyed by every device source.
KIND_SOURCES = {
    "attn": ("k_attn_t5.cu", "model_dev.cuh", "tc5.cuh", "internal.h"),
    "vocab": ("k_vocab.cu", "internal.h"),
    "ngram_update": ("k_vocab.cu", "internal.h"),
}


def kernel_sources_hash(kind: str = "") -> str:
    """Hash of the device code a kernel kind is built from (its kernel file
    and the headers it includes; every kernel file and header for other
    kinds); host-only orchestration and the host coder are left out."""
    d = os.path.join(ROOT, "paper_2602_19626_gb300", "csrc")
    names = KIND_SOURCES.get(kind)
    if names is None:
        names = [n for n in os.listdir(d)
                 if (n.startswith("k_") and n.endswith(".cu")) or n.endswith(".cuh") or n == "internal.h"]
    m = hashlib.sha256()
    for name in sorted(names):
        with open(os.path.join(d, name), "rb") as fh:
            m.update(fh.read())
    return m.hexdigest()[:12]


def prefill_positions(wl, n_streams: int, max_len: int) -> int:
    """Positions per model forward: the library's rule (largest power of two m
    with n m <= prefill_rows dividing the window and the slide, doubling only
    while m is below the longest stream), or 1."""
    shape, rows = wl["shape"], wl.get("prefill_rows", 0)
    if rows < 2:
        return 1
    m = 1
    while 2 * m * n_streams <= rows and shape.slide % (2 * m) == 0 and shape.ctx_len % (2 * m) == 0 and m < max_len:
        m *= 2
    return m if m >= 2 else 1


def dominant_kind(trace, wl, n_streams: int, max_len: int):
    """The traced kernel kind the roofline reports, and the kinds that run
    beside it.  The dominant kind is the one with the largest share of the
    trace.  With the prefill, a chunk's N-gram pass runs beside its forward,
    and its vocabulary loop beside the next two chunks' forwards: when the
    loop dominates, it is the chain that paces the timed run and the forward
    kinds and the N-gram pass run beside it; when a forward kind dominates,
    the loop and the N-gram pass run beside the forwards."""
    dom = max(trace, key=lambda k: k["ms"])
    if prefill_positions(wl, n_streams, max_len) < 2:
        return dom, []
    loop = {"ngram_update", "vocab"}
    if dom["name"] in loop:
        beside = [k["name"] for k in trace if k["name"] != dom["name"] and k["launches"]]
    else:
        beside = sorted(loop)
    return dom, beside


def run_gpu(args, wl):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2602_19626_gb300 import nc24

    shape = wl["shape"]
    streams = workload_streams(wl, ws, rank)
    lens = np.array([len(s) for s in streams], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    flat = np.concatenate(streams).astype(np.int32)
    n_tok = int(lens.sum())
    stride = int(lens.max())
    cstream = torch.cuda.Stream()
    cfg = nc24.make_config(shape, fmt=wl["fmt"], max_streams=len(streams), device=dev, stream=cstream,
                           path=wl.get("path", "gemv"), prefill_rows=wl.get("prefill_rows", 0),
                           rule=wl.get("rule", "paper"))
    ctx = nc24.Context(cfg, S.flat_weights(shape, wl["seed"]))
    tok_dev = torch.from_numpy(flat).to(f"cuda:{dev}")
    iv = torch.empty((len(streams), stride, 2), dtype=torch.int32, device=f"cuda:{dev}")
    torch.cuda.synchronize()

    def step():
        ctx.encode_intervals(tok_dev, offs, lens, iv, stride)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = ClockSampler(dev)
    with torch.cuda.stream(cstream):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(cstream)
        for _ in range(args.steps):
            step()
        e1.record(cstream)
        torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([ms], device=f"cuda:{dev}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    if ws > 1:
        t = torch.tensor([n_tok], device=f"cuda:{dev}", dtype=torch.float64)
        torch.distributed.all_reduce(t)
        job_tokens = float(t.item())
    else:
        job_tokens = float(n_tok)
    total_tokens = job_tokens * args.steps
    value = total_tokens / (ms / 1000.0)
    print(f"[bench] timed {args.steps} steps: {ms:.1f} ms, {value:.1f} tokens/s", file=sys.stderr, flush=True)

    # correctness guard on the timed output: intervals are non-empty, in range
    ivh = iv.cpu().numpy().view(np.uint32)
    lo, hi = ivh[..., 0], ivh[..., 1]
    ok = bool(np.all(hi[:, : lens.min()] > lo[:, : lens.min()]) and np.all(hi <= (1 << 24)))

    # per-kernel trace (one more pass, every kernel between CUDA events on the
    # context's stream): the dominant kernel's bytes and average duration
    roofline, kernels, launches_per_step = None, None, 155 * n_tok
    try:
        trace = ctx.encode_intervals(tok_dev, offs, lens, iv, stride, trace=True)
        tot_ms = sum(k["ms"] for k in trace) or 1.0
        dom, beside = dominant_kind(trace, wl, len(streams), int(lens.max()))
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        roofline = roofline_of(dom, wl.get("path", "gemv"), wl["fmt"], n_sm, 2070.0)
        roofline["share"] = dom["ms"] / tot_ms
        roofline["beside_critical_path"] = beside
        roofline["traffic"] = ncu_traffic(dom["name"], args.workload)
        # the largest kernel of the model forward, beside the loop that paces the run
        fwd = [k for k in trace if k["name"] not in ("vocab", "ngram_update", "prepare") and k["launches"]]
        if dom["name"] in ("vocab", "ngram_update") and fwd:
            fk = max(fwd, key=lambda k: k["ms"])
            roofline["forward"] = roofline_of(fk, wl.get("path", "gemv"), wl["fmt"], n_sm, 2070.0)
            roofline["forward"]["share"] = fk["ms"] / tot_ms
        kernels = {k["name"]: {"launches": k["launches"], "ms": round(k["ms"], 3),
                               "share": round(k["ms"] / tot_ms, 4),
                               "GBps": round(k["bytes"] / (k["ms"] / 1000.0) / 1e9, 1) if k["ms"] > 0 else None,
                               "TFLOPs": round(k["flops"] / (k["ms"] / 1000.0) / 1e12, 2) if k["ms"] > 0 else None}
                   for k in trace if k["launches"]}
        launches_per_step = sum(k["launches"] for k in trace)
        roofline["graphed"] = bool(trace[0]["graphed"])
    except Exception as exc:  # keep the measured line even if tracing fails
        print(f"[bench] trace failed: {exc}", file=sys.stderr, flush=True)

    # end to end through the public API: host tokens in, container bytes out
    host_streams = [np.ascontiguousarray(s) for s in streams]
    ctx.encode(host_streams)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    nbytes = 0
    blob = b""
    for _ in range(e2e_steps):
        blob = ctx.encode(host_streams)
        nbytes = len(blob)
    e2e_s = time.perf_counter() - t0
    # the decoder (one position per step: it learns each token from the
    # coder) on the same container, through nc_decode
    decode = None
    if rank == 0 and not args.no_decode:
        t0 = time.perf_counter()
        back = ctx.decode(blob)
        dec_s = time.perf_counter() - t0
        decode = {"value": n_tok / dec_s, "unit": "tokens/s", "s": dec_s,
                  "lossless": bool(all(np.array_equal(a, b) for a, b in zip(back, host_streams)))}
        # the floor of the decode step's chain of dependent launches: a
        # captured graph of empty kernels, one per kernel of a step
        links = DECODE_STEP_LAUNCHES
        us = nc24.nc_launch_chain_floor(dev, links, 152, 256, 20)
        decode["launch_chain_floor"] = {"links": links, "us_per_link": us, "us_per_step": us * links,
                                        "blocks": 152, "threads": 256}
    if ws > 1:
        t = torch.tensor([e2e_s], device=f"cuda:{dev}", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": job_tokens * e2e_steps / e2e_s, "unit": "tokens/s",
           "h2d_bytes_per_step": int(flat.nbytes + 16 * len(streams)),
           "d2h_bytes_per_step": int(8 * n_tok), "container_bytes": nbytes,
           "bits_per_token": 8.0 * nbytes / n_tok}

    ctx.close()
    extras = {}
    for name in args.extra:
        try:
            extras[name] = extra_throughput(name, dev)
        except Exception as exc:
            extras[name] = {"error": str(exc)[:200]}
    cpu = None
    bpb = None
    if rank == 0 and not args.no_cpu_baseline:
        n, el, obits = oracle_rate(wl, args.cpu_budget)
        cpu = {"value": n / el, "unit": "tokens/s", "cores": blas_threads(), "cpu": cpu_model(), "kind": "oracle",
               "sample": f"first {n} tokens of the workload's first stream, FP64 oracle on "
                         f"{wl['fmt']}-dequantised weights, {el:.1f} s"}
        # the timed run's coded intervals on the same prefix against the
        # oracle's: the "bpb within 0.5% of the FP64 oracle" of the metric
        gbits = interval_bits(ivh[0], n)
        nbyt = S.n_bytes(streams[0][:n])
        rel = (gbits - obits) / obits
        bpb = {"tokens": n, "gpu_bits": gbits, "oracle_bits": obits, "gpu_bpb": gbits / nbyt,
               "oracle_bpb": obits / nbyt, "rel": rel, "within_0.5pct": bool(abs(rel) <= 5e-3),
               "what": "sum -log2((hi - lo) / 2^24) of the timed run's intervals and the oracle's over the "
                       "cpu_baseline's prefix of the first stream"}
    ratios = {}
    if PLAIN in extras and "value" in extras[PLAIN]:
        for name in BATCHED:
            if name in extras and "value" in extras[name]:
                ratios[name] = extras[name]["value"] / extras[PLAIN]["value"]
        ratios["headline"] = value / extras[PLAIN]["value"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "tokens/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if wl.get("path", "gemv") == "tc" else "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "model": "smollm2-135m-shape random-init",
                       "weights": wl["fmt"], "streams_per_gpu": wl["n_streams"],
                       "tokens_per_gpu": n_tok, "ctx_len": shape.ctx_len, "slide": shape.slide,
                       "path": wl.get("path", "gemv"), "parallelism": f"replicas{ws}",
                       "prefill_rows": wl.get("prefill_rows", 0),
                       "positions_per_forward": prefill_positions(wl, len(streams), int(lens.max())),
                       "l2": "inputs larger than L2: weights (BF16 269 MB) are re-read every model "
                             "forward, and each timed step codes the whole workload"},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline, "kernels": kernels, "clocks": clocks, "e2e": e2e,
            "cpu_baseline": cpu, "bpb_vs_oracle": bpb, "intervals_valid": ok,
            "decode": decode,
            "batched_over_plain": ratios or None,
        }
        if extras:
            line["extra"] = extras
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def extra_throughput(name, dev):
    """Device-resident throughput of another workload (one warm-up, one timed
    pass), reported beside the headline line."""
    import torch
    from paper_2602_19626_gb300 import nc24
    wl = WORKLOADS[name]
    shape = wl["shape"]
    streams = workload_streams(wl)
    lens = np.array([len(s) for s in streams], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    flat = np.concatenate(streams).astype(np.int32)
    stride = int(lens.max())
    cstream = torch.cuda.Stream()
    cfg = nc24.make_config(shape, fmt=wl["fmt"], max_streams=wl["n_streams"], device=dev, stream=cstream,
                           path=wl.get("path", "gemv"), prefill_rows=wl.get("prefill_rows", 0),
                           rule=wl.get("rule", "paper"))
    ctx = nc24.Context(cfg, S.flat_weights(shape, wl["seed"]))
    tok_dev = torch.from_numpy(flat).to(f"cuda:{dev}")
    iv = torch.empty((wl["n_streams"], stride, 2), dtype=torch.int32, device=f"cuda:{dev}")
    torch.cuda.synchronize()
    ctx.encode_intervals(tok_dev, offs, lens, iv, stride)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(cstream)
    ctx.encode_intervals(tok_dev, offs, lens, iv, stride)
    e1.record(cstream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    ivh = iv.cpu().numpy().view(np.uint32)
    bits = sum(interval_bits(ivh[j], int(lens[j])) for j in range(len(lens)))
    return {"value": float(lens.sum()) / (ms / 1000.0), "unit": "tokens/s", "ms": ms,
            "streams": wl["n_streams"], "tokens": int(lens.sum()), "weights": wl["fmt"],
            "path": wl.get("path", "gemv"), "rule": wl.get("rule", "paper"),
            "positions_per_forward": prefill_positions(wl, len(lens), int(lens.max())),
            "bits_per_token": bits / float(lens.sum())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full_bf16_single", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tokens", type=int, default=0,
                    help="cut every stream to this many tokens (short runs for profiling)")
    ap.add_argument("--extra", nargs="*",
                    default=[PLAIN, *BATCHED, "diff_bf16_tc_64x4096", "full_bf16_single_tc_stepwise"],
                    help="further workloads timed once each and reported under 'extra'")
    ap.add_argument("--no-decode", action="store_true", help="skip timing nc_decode on the headline container")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.tokens > 0:
        wl = dict(wl, cap=min(wl.get("cap", args.tokens), args.tokens))
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_gpu(args, wl)


if __name__ == "__main__":
    main()
