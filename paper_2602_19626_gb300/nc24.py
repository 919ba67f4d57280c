"""ctypes binding of libnc24.so (include/nc24.h), argument marshalling only.

Every function of the C ABI is exposed under its own name with the same
arguments; ``Context`` wraps a context handle for convenience.  All compute
runs in the library's CUDA kernels: there is no Python or CPU fallback, and
importing this module fails loudly when the library has not been built.

Device buffers are passed as torch CUDA tensors (their data_ptr()); host
buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libnc24.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libnc24.so is not built ({_LIB_PATH}); run paper_2602_19626_gb300/build.py "
                      "or __graft_entry__.build() first")
lib = C.CDLL(_LIB_PATH)

NC_OK, NC_EINVAL, NC_ENOMEM, NC_ECUDA, NC_ETIMEOUT, NC_ECORRUPT, NC_ESTATE, NC_ENUMERIC = range(8)
NC_FP32, NC_BF16, NC_FP8E4M3 = 0, 1, 2
NC_RULE_PAPER, NC_RULE_MIXED_NLL = 0, 1
NC_PATH_GEMV, NC_PATH_TC = 0, 1
NC_CODER_ARITH, NC_CODER_RANS = 0, 1
CODER = {"arith": NC_CODER_ARITH, "rans": NC_CODER_RANS}
FMT = {"fp32": NC_FP32, "bf16": NC_BF16, "fp8": NC_FP8E4M3}
RULE = {"paper": NC_RULE_PAPER, "mixed_nll": NC_RULE_MIXED_NLL}


class nc_config(C.Structure):
    _fields_ = [
        ("n_layers", C.c_int), ("d_model", C.c_int), ("n_heads", C.c_int), ("n_kv_heads", C.c_int),
        ("d_ffn", C.c_int), ("vocab", C.c_int),
        ("rope_theta", C.c_float), ("rms_eps", C.c_float),
        ("ctx_len", C.c_int), ("slide", C.c_int),
        ("ngram_order", C.c_int), ("use_head", C.c_int),
        ("cdf_log2_total", C.c_int), ("floor", C.c_uint32),
        ("bias_lr", C.c_float), ("mix_eta", C.c_float), ("w_llm_init", C.c_float),
        ("temperature", C.c_float),
        ("warmup", C.c_int), ("weight_fmt", C.c_int), ("update_rule", C.c_int), ("path", C.c_int),
        ("max_streams", C.c_int), ("device", C.c_int), ("cuda_stream", C.c_void_p),
        ("prefill_rows", C.c_int), ("skip", C.c_int), ("coder", C.c_int),
    ]


NC_TRACE_KINDS = 16


class nc_trace(C.Structure):
    _fields_ = [("n_kinds", C.c_int), ("graphed", C.c_int), ("name", (C.c_char * 32) * NC_TRACE_KINDS),
                ("launches", C.c_int64 * NC_TRACE_KINDS), ("ms", C.c_double * NC_TRACE_KINDS),
                ("bytes", C.c_double * NC_TRACE_KINDS), ("flops", C.c_double * NC_TRACE_KINDS)]


_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)
_I64P = C.POINTER(C.c_int64)
_U32P = C.POINTER(C.c_uint32)
_F32P = C.POINTER(C.c_float)
_U8P = C.POINTER(C.c_uint8)
_SZP = C.POINTER(C.c_size_t)

_SIGS = {
    "nc_config_default": (None, [C.POINTER(nc_config)]),
    "nc_ctx_create": (C.c_int, [C.POINTER(nc_config), _P, C.c_size_t, C.POINTER(_P)]),
    "nc_ctx_destroy": (None, [_P]),
    "nc_stream_open": (C.c_int, [_P, C.c_int32, C.c_int64]),
    "nc_stream_close": (C.c_int, [_P, C.c_int32]),
    "nc_step_cdf": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "nc_update_bias": (C.c_int, [_P, C.c_int, _P, _P]),
    "nc_encode": (C.c_int, [_P, C.c_int, _P, _P, _P, _SZP]),
    "nc_decode": (C.c_int, [_P, _P, C.c_size_t, _P, _P]),
    "nc_encode_intervals": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.c_int64, C.POINTER(nc_trace)]),
    "nc_encode_probe": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.c_int64, C.c_int64, _P, _P, _P, _P]),
    "nc_container_streams": (C.c_int, [_P, C.c_size_t, C.POINTER(C.c_int)]),
    "nc_status_str": (C.c_char_p, [C.c_int]),
    "nc_last_error": (C.c_char_p, [_P]),
    "nc_probs_to_cdf": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_uint32, _P, _P]),
    "nc_probs_to_cdf_noalloc": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_uint32, _P, _P]),
    "nc_floor_counts": (C.c_int, [_P, C.c_int64, C.c_uint32, C.c_uint32, _P, _P]),
    "nc_step_probe": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P]),
    "nc_stream_state": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "nc_gemm_tc": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "nc_ac_encode": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, _SZP, C.POINTER(C.c_uint64)]),
    "nc_ac_decode": (C.c_int, [_P, C.c_uint64, _P, C.c_int, C.c_int64, C.c_int, _P]),
    "nc_ans_encode": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, _SZP]),
    "nc_split_chunks": (C.c_int, [_P, C.c_int64, _P, C.c_int, C.c_int, _P, C.POINTER(C.c_int)]),
    "nc_hybrid_segments": (C.c_int, [_P, C.c_int64, _P, _P, C.c_int64, _I64P]),
    "nc_hybrid_pack": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, C.c_size_t, _P, C.c_size_t, _P, _SZP]),
    "nc_hybrid_parse": (C.c_int, [_P, C.c_size_t, _P, _P, C.c_int64, _I64P, C.POINTER(C.c_int), _SZP, _SZP,
                                  _SZP]),
    "nc_ans_decode": (C.c_int, [_P, C.c_size_t, _P, C.c_int, C.c_int64, C.c_int, _P]),
    "nc_selftest_wait": (C.c_int, [_P, C.c_uint32]),
    "nc_launch_chain_floor": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _F32P]),
    "nc_mix_nll_fwd": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int, C.c_int, C.c_float, _P, _P]),
    "nc_mix_nll_bwd": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.c_int, C.c_int, C.c_float, _P, _P, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class NcError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{lib.nc_status_str(status).decode()}: {msg}")


def _ptr(x):
    """Address of a numpy array, a torch tensor or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(type(x))


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


# ------------------------------------------------------------- same names

def nc_config_default() -> nc_config:
    c = nc_config()
    lib.nc_config_default(C.byref(c))
    return c


def nc_status_str(status: int) -> str:
    return lib.nc_status_str(status).decode()


def nc_probs_to_cdf(p, cdf, log2_total=24, floor=1, stream=None) -> int:
    """p: CUDA float32 [n, V]; cdf: CUDA int32/uint32 [n, V + 1]."""
    n, V = p.shape
    return lib.nc_probs_to_cdf(_ptr(p), n, V, log2_total, floor, _ptr(cdf), _stream_ptr(stream))


NC_NOALLOC_MAX_ROWS = 4096


def nc_probs_to_cdf_noalloc(p, cdf, log2_total=24, floor=1, stream=None) -> int:
    """As nc_probs_to_cdf, without allocating device memory (at most
    NC_NOALLOC_MAX_ROWS rows per call; calls must not overlap on the GPU)."""
    n, V = p.shape
    return lib.nc_probs_to_cdf_noalloc(_ptr(p), n, V, log2_total, floor, _ptr(cdf), _stream_ptr(stream))


def nc_floor_counts(p, K, floor, c, stream=None) -> int:
    return lib.nc_floor_counts(_ptr(p), p.numel(), K, floor, _ptr(c), _stream_ptr(stream))


def nc_gemm_tc(W, X, Y, bn=128, w_scale=None, x_scale=None, fp8=False, stream=None) -> int:
    """W CUDA [M, K], X CUDA [N, K] (bf16, or uint8 E4M3 bytes with fp8); Y CUDA float32 [N, M]."""
    M, K = W.shape
    N = X.shape[0]
    return lib.nc_gemm_tc(_ptr(W), _ptr(X), _ptr(w_scale), _ptr(x_scale), int(fp8), M, N, K, bn, _ptr(Y),
                          _stream_ptr(stream))


def nc_ac_encode(lo: np.ndarray, hi: np.ndarray, log2_total: int):
    """Encode intervals on the host; returns (bytes, nbits)."""
    lo = np.ascontiguousarray(lo, dtype=np.uint32)
    hi = np.ascontiguousarray(hi, dtype=np.uint32)
    nb = C.c_size_t(0)
    bits = C.c_uint64(0)
    st = lib.nc_ac_encode(_ptr(lo), _ptr(hi), lo.size, log2_total, None, C.byref(nb), C.byref(bits))
    if st:
        raise NcError(st, "nc_ac_encode")
    out = np.zeros(max(nb.value, 1), dtype=np.uint8)
    st = lib.nc_ac_encode(_ptr(lo), _ptr(hi), lo.size, log2_total, _ptr(out), C.byref(nb), C.byref(bits))
    if st:
        raise NcError(st, "nc_ac_encode")
    return out[: nb.value].tobytes(), bits.value


def nc_ac_decode(data: bytes, nbits: int, cdfs: np.ndarray, log2_total: int) -> np.ndarray:
    cdfs = np.ascontiguousarray(cdfs, dtype=np.uint32)
    n, V1 = cdfs.shape
    buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    sym = np.zeros(n, dtype=np.int32)
    st = lib.nc_ac_decode(_ptr(buf), nbits, _ptr(cdfs), V1 - 1, n, log2_total, _ptr(sym))
    if st:
        raise NcError(st, "nc_ac_decode")
    return sym


def nc_split_chunks(tokens: np.ndarray, is_boundary: np.ndarray, n_chunks: int) -> np.ndarray:
    """Cut positions 0 = c_0 < ... < c_m = n of a file's tokens (Sec. 3.11)."""
    tokens = np.ascontiguousarray(tokens, dtype=np.int32)
    bnd = np.ascontiguousarray(is_boundary, dtype=np.uint8)
    cuts = np.zeros(n_chunks + 1, dtype=np.int64)
    m = C.c_int(0)
    st = lib.nc_split_chunks(_ptr(tokens), tokens.size, _ptr(bnd), bnd.size, n_chunks, _ptr(cuts), C.byref(m))
    if st:
        raise NcError(st, "nc_split_chunks")
    return cuts[: m.value + 1] if m.value else cuts[:1]


def nc_launch_chain_floor(device: int, n_links: int, blocks: int = 152, threads: int = 256,
                          reps: int = 20) -> float:
    """Microseconds per link of a graph-captured chain of empty dependent launches."""
    us = C.c_float(0.0)
    st = lib.nc_launch_chain_floor(device, n_links, blocks, threads, reps, C.byref(us))
    if st:
        raise NcError(st, "nc_launch_chain_floor")
    return us.value


def _host_bytes(data: bytes) -> np.ndarray:
    return np.frombuffer(data, dtype=np.uint8).copy() if len(data) else np.zeros(1, np.uint8)


def nc_hybrid_segments(data: bytes):
    """The text (0) / binary (1) runs of a byte string (Sec. 3.10): kinds uint8, lengths int64."""
    buf = _host_bytes(data)
    n = C.c_int64(0)
    st = lib.nc_hybrid_segments(_ptr(buf), len(data), None, None, 0, C.byref(n))
    if st:
        raise NcError(st, "nc_hybrid_segments")
    kinds = np.zeros(max(n.value, 1), dtype=np.uint8)
    lens = np.zeros(max(n.value, 1), dtype=np.int64)
    st = lib.nc_hybrid_segments(_ptr(buf), len(data), _ptr(kinds), _ptr(lens), kinds.size, C.byref(n))
    if st:
        raise NcError(st, "nc_hybrid_segments")
    return kinds[: n.value], lens[: n.value]


def nc_hybrid_pack(kinds, lens, method: int, stored: bytes, text: bytes) -> bytes:
    """An NC06 container from its runs, the stored blob and the text runs' NC05 container."""
    kinds = np.ascontiguousarray(kinds, dtype=np.uint8)
    lens = np.ascontiguousarray(lens, dtype=np.int64)
    sb, tb = _host_bytes(stored), _host_bytes(text)
    nb = C.c_size_t(0)
    st = lib.nc_hybrid_pack(_ptr(kinds), _ptr(lens), kinds.size, method, _ptr(sb), len(stored), _ptr(tb),
                            len(text), None, C.byref(nb))
    if st:
        raise NcError(st, "nc_hybrid_pack(size)")
    out = np.zeros(nb.value, dtype=np.uint8)
    st = lib.nc_hybrid_pack(_ptr(kinds), _ptr(lens), kinds.size, method, _ptr(sb), len(stored), _ptr(tb),
                            len(text), _ptr(out), C.byref(nb))
    if st:
        raise NcError(st, "nc_hybrid_pack")
    return out[: nb.value].tobytes()


def nc_hybrid_parse(data: bytes):
    """(kinds, lens, method, stored_off, stored_len, text_off) of an NC06 container."""
    buf = _host_bytes(data)
    n, m = C.c_int64(0), C.c_int(0)
    so, sl, to = C.c_size_t(0), C.c_size_t(0), C.c_size_t(0)
    args = (C.byref(n), C.byref(m), C.byref(so), C.byref(sl), C.byref(to))
    st = lib.nc_hybrid_parse(_ptr(buf), len(data), None, None, 0, *args)
    if st:
        raise NcError(st, "nc_hybrid_parse")
    kinds = np.zeros(max(n.value, 1), dtype=np.uint8)
    lens = np.zeros(max(n.value, 1), dtype=np.int64)
    st = lib.nc_hybrid_parse(_ptr(buf), len(data), _ptr(kinds), _ptr(lens), kinds.size, *args)
    if st:
        raise NcError(st, "nc_hybrid_parse")
    return kinds[: n.value], lens[: n.value], m.value, so.value, sl.value, to.value


# The binary blob of an NC06 container (Sec. 3.10): LZMA from 4 KB up, gzip
# below, stored raw when the compressed form is not shorter.
_BLOB_RAW, _BLOB_GZIP, _BLOB_LZMA = 0, 1, 2


def _blob_pack(blob: bytes):
    import gzip
    import lzma
    if not blob:
        return _BLOB_RAW, b""
    m, s = (_BLOB_LZMA, lzma.compress(blob)) if len(blob) >= 4096 else (_BLOB_GZIP, gzip.compress(blob, mtime=0))
    return (m, s) if len(s) < len(blob) else (_BLOB_RAW, blob)


def _blob_unpack(method: int, stored: bytes) -> bytes:
    import gzip
    import lzma
    import zlib
    try:
        return {_BLOB_RAW: lambda b: b, _BLOB_GZIP: gzip.decompress, _BLOB_LZMA: lzma.decompress}[method](stored)
    except (OSError, EOFError, lzma.LZMAError, zlib.error) as exc:
        raise NcError(NC_ECORRUPT, f"NC06 binary section: {exc}") from exc


def nc_ans_encode(lo: np.ndarray, hi: np.ndarray, log2_total: int) -> bytes:
    """rANS-code intervals on the host; returns the bytes."""
    lo = np.ascontiguousarray(lo, dtype=np.uint32)
    hi = np.ascontiguousarray(hi, dtype=np.uint32)
    nb = C.c_size_t(0)
    st = lib.nc_ans_encode(_ptr(lo), _ptr(hi), lo.size, log2_total, None, C.byref(nb))
    if st:
        raise NcError(st, "nc_ans_encode")
    out = np.zeros(max(nb.value, 1), dtype=np.uint8)
    st = lib.nc_ans_encode(_ptr(lo), _ptr(hi), lo.size, log2_total, _ptr(out), C.byref(nb))
    if st:
        raise NcError(st, "nc_ans_encode")
    return out[: nb.value].tobytes()


def nc_ans_decode(data: bytes, cdfs: np.ndarray, log2_total: int) -> np.ndarray:
    cdfs = np.ascontiguousarray(cdfs, dtype=np.uint32)
    n, V1 = cdfs.shape
    buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    sym = np.zeros(n, dtype=np.int32)
    st = lib.nc_ans_decode(_ptr(buf), len(data), _ptr(cdfs), V1 - 1, n, log2_total, _ptr(sym))
    if st:
        raise NcError(st, "nc_ans_decode")
    return sym


def nc_mix_nll_fwd(z, b, p_ng, theta, target, warm, tau, loss, stream=None) -> int:
    n, V = z.shape
    return lib.nc_mix_nll_fwd(_ptr(z), _ptr(b), _ptr(p_ng), _ptr(theta), _ptr(target), _ptr(warm),
                              n, V, tau, _ptr(loss), _stream_ptr(stream))


def nc_mix_nll_bwd(z, b, p_ng, theta, target, warm, gout, tau, db, dtheta, stream=None) -> int:
    n, V = z.shape
    return lib.nc_mix_nll_bwd(_ptr(z), _ptr(b), _ptr(p_ng), _ptr(theta), _ptr(target), _ptr(warm),
                              _ptr(gout), n, V, tau, _ptr(db), _ptr(dtheta), _stream_ptr(stream))


# ------------------------------------------------------------- context

def make_config(shape, fmt="bf16", rule="paper", max_streams=1, ngram_order=3, use_head=True,
                warmup=100, log2_total=24, floor=1, alpha=1e-3, eta=1.0, w_llm=0.85, tau=1.0,
                device=0, stream=None, path="gemv", prefill_rows=0, skip=False, coder="arith") -> nc_config:
    """nc_config from a shape with the fields of synthetic.ModelShape."""
    c = nc_config_default()
    c.n_layers, c.d_model, c.n_heads = shape.n_layers, shape.d_model, shape.n_heads
    c.n_kv_heads, c.d_ffn, c.vocab = shape.n_kv_heads, shape.d_ffn, shape.vocab
    c.rope_theta, c.rms_eps = shape.rope_theta, shape.rms_eps
    c.ctx_len, c.slide = shape.ctx_len, shape.slide
    c.ngram_order, c.use_head = ngram_order, int(bool(use_head))
    c.cdf_log2_total, c.floor = log2_total, floor
    c.bias_lr, c.mix_eta, c.w_llm_init, c.temperature = alpha, eta, w_llm, tau
    c.warmup = warmup
    c.weight_fmt = FMT[fmt] if isinstance(fmt, str) else fmt
    c.update_rule = RULE[rule] if isinstance(rule, str) else rule
    c.path = NC_PATH_GEMV if path == "gemv" else NC_PATH_TC
    c.max_streams, c.device = max_streams, device
    c.cuda_stream = _stream_ptr(stream) if stream is not None else None
    c.prefill_rows = prefill_rows
    c.skip = int(bool(skip))
    c.coder = CODER[coder] if isinstance(coder, str) else coder
    return c


class Context:
    """Owns one nc_ctx.  weights: the flat FP32 numpy buffer (host)."""

    def __init__(self, cfg: nc_config, weights: np.ndarray):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        h = C.c_void_p()
        st = lib.nc_ctx_create(C.byref(cfg), _ptr(w), w.nbytes, C.byref(h))
        if st:
            raise NcError(st, "nc_ctx_create")
        self.h = h
        self.cfg = cfg
        self.V = cfg.vocab

    def close(self):
        if self.h:
            lib.nc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st:
            raise NcError(st, f"{what}: {lib.nc_last_error(self.h).decode()}")

    def stream_open(self, sid: int, expected_len: int):
        self._check(lib.nc_stream_open(self.h, sid, expected_len), "nc_stream_open")

    def stream_close(self, sid: int):
        self._check(lib.nc_stream_close(self.h, sid), "nc_stream_close")

    def step_cdf(self, ids, prev=None, cdf_out=None):
        """Returns cdf_out (numpy uint32 [n, V+1] when not given)."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        if cdf_out is None:
            cdf_out = np.zeros((ids.size, self.V + 1), dtype=np.uint32)
        prev_a = None if prev is None else np.ascontiguousarray(prev, dtype=np.int32)
        self._check(lib.nc_step_cdf(self.h, ids.size, _ptr(ids), _ptr(prev_a), _ptr(cdf_out)), "nc_step_cdf")
        return cdf_out

    def step_probe(self, ids, z=None, p_tilde=None, p_ng=None, p=None, cdf_out=None):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        self._check(lib.nc_step_probe(self.h, ids.size, _ptr(ids), _ptr(z), _ptr(p_tilde), _ptr(p_ng),
                                      _ptr(p), _ptr(cdf_out)), "nc_step_probe")

    def update_bias(self, ids, observed):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        obs = np.ascontiguousarray(observed, dtype=np.int32)
        self._check(lib.nc_update_bias(self.h, ids.size, _ptr(ids), _ptr(obs)), "nc_update_bias")

    def stream_state(self, sid: int):
        b = np.zeros(self.V, dtype=np.float32)
        th = np.zeros(2, dtype=np.float32)
        n = C.c_int64(0)
        self._check(lib.nc_stream_state(self.h, sid, _ptr(b), _ptr(th), C.byref(n)), "nc_stream_state")
        return b, th, n.value

    def encode(self, streams) -> bytes:
        arrs = [np.ascontiguousarray(s, dtype=np.int32) for s in streams]
        ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        lens = np.array([a.size for a in arrs], dtype=np.int64)
        nb = C.c_size_t(0)
        self._check(lib.nc_encode(self.h, len(arrs), ptrs, _ptr(lens), None, C.byref(nb)), "nc_encode(size)")
        out = np.zeros(nb.value, dtype=np.uint8)
        self._check(lib.nc_encode(self.h, len(arrs), ptrs, _ptr(lens), _ptr(out), C.byref(nb)), "nc_encode")
        return out[: nb.value].tobytes()

    def encode_file(self, tokens, is_boundary, n_chunks: int = 8) -> bytes:
        """One file's tokens as up to n_chunks streams of one container, cut
        at line-ending tokens (Sec. 3.11; nc_split_chunks)."""
        toks = np.ascontiguousarray(tokens, dtype=np.int32)
        c = nc_split_chunks(toks, is_boundary, n_chunks)
        parts = [toks[c[i]:c[i + 1]] for i in range(len(c) - 1)] or [toks[:0]]
        return self.encode(parts)

    def decode_file(self, data: bytes) -> np.ndarray:
        """Inverse of encode_file: the chunks in order, concatenated."""
        parts = self.decode(data)
        return np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)

    def encode_hybrid(self, data: bytes) -> bytes:
        """An arbitrary byte string as one NC06 container (Sec. 3.10): its
        text runs coded as the streams of one NC05 container (one batch), its
        binary runs as one blob.  Without the tokenizer, a text byte enters
        the model as the token id equal to its value.  The context's
        max_streams bounds the number of text runs of one file."""
        kinds, lens = nc_hybrid_segments(data)
        buf = np.frombuffer(data, dtype=np.uint8)
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        texts = [buf[offs[i]:offs[i + 1]].astype(np.int32) for i in range(kinds.size) if kinds[i] == 0]
        blob = b"".join(data[offs[i]:offs[i + 1]] for i in range(kinds.size) if kinds[i] == 1)
        method, stored = _blob_pack(blob)
        return nc_hybrid_pack(kinds, lens, method, stored, self.encode(texts) if texts else b"")

    def decode_hybrid(self, data: bytes) -> bytes:
        """Inverse of encode_hybrid."""
        kinds, lens, method, so, sl, to = nc_hybrid_parse(data)
        blob = _blob_unpack(method, data[so:so + sl])
        n_text = int((kinds == 0).sum())
        texts = self.decode(data[to:]) if n_text else []
        if len(texts) != n_text or len(blob) != int(lens[kinds == 1].sum()):
            raise NcError(NC_ECORRUPT, "NC06 sections disagree with the run table")
        out, ti, bo = [], 0, 0
        for k, n in zip(kinds, lens):
            if k == 0:
                t = texts[ti]
                ti += 1
                if t.size != n:
                    raise NcError(NC_ECORRUPT, "NC06 text run length")
                out.append(t.astype(np.uint8).tobytes())
            else:
                out.append(blob[bo:bo + int(n)])
                bo += int(n)
        return b"".join(out)

    def encode_intervals(self, tokens_dev, offsets, lens, intervals_dev, stride: int, trace: bool = False):
        """Device half of encode: tokens_dev CUDA int32 (flat), offsets/lens
        host int64, intervals_dev CUDA int32/uint32 [n, stride, 2].  Returns
        the per-kernel trace as a list of dicts when trace is set."""
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        ln = np.ascontiguousarray(lens, dtype=np.int64)
        tr = nc_trace() if trace else None
        self._check(lib.nc_encode_intervals(self.h, ln.size, _ptr(tokens_dev), _ptr(offs), _ptr(ln),
                                            _ptr(intervals_dev), stride, C.byref(tr) if tr else None),
                    "nc_encode_intervals")
        if not tr:
            return None
        return [dict(name=tr.name[k].value.decode(), launches=tr.launches[k], ms=tr.ms[k], bytes=tr.bytes[k],
                     flops=tr.flops[k], graphed=bool(tr.graphed)) for k in range(tr.n_kinds)]

    def encode_probe(self, tokens_dev, offsets, lens, intervals_dev, stride: int, probe_pos: int,
                     z=None, p_tilde=None, p_ng=None, p=None):
        """encode_intervals that also writes each stream's z, p_tilde, p_ng
        and p at token index probe_pos (CUDA float32 [n, V] each, or None)."""
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        ln = np.ascontiguousarray(lens, dtype=np.int64)
        self._check(lib.nc_encode_probe(self.h, ln.size, _ptr(tokens_dev), _ptr(offs), _ptr(ln),
                                        _ptr(intervals_dev), stride, probe_pos, _ptr(z), _ptr(p_tilde),
                                        _ptr(p_ng), _ptr(p)), "nc_encode_probe")

    def selftest_wait(self, polls: int):
        """One bounded device wait that gives up (nc_selftest_wait): raises
        NcError(NC_ETIMEOUT) and leaves the context poisoned."""
        self._check(lib.nc_selftest_wait(self.h, polls), "nc_selftest_wait")

    def decode(self, data: bytes):
        buf = np.frombuffer(data, dtype=np.uint8).copy()
        n = C.c_int(0)
        st = lib.nc_container_streams(_ptr(buf), buf.size, C.byref(n))
        if st:
            raise NcError(st, "nc_container_streams")
        lens = np.zeros(max(n.value, 1), dtype=np.int64)
        self._check(lib.nc_decode(self.h, _ptr(buf), buf.size, None, _ptr(lens)), "nc_decode(query)")
        outs = [np.zeros(max(int(l), 1), dtype=np.int32) for l in lens[: n.value]]
        ptrs = (C.c_void_p * max(len(outs), 1))(*[o.ctypes.data for o in outs])
        self._check(lib.nc_decode(self.h, _ptr(buf), buf.size, ptrs, _ptr(lens)), "nc_decode")
        return [o[: int(l)] for o, l in zip(outs, lens[: n.value])]
