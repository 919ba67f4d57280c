"""Oracle runs that GPU tests start in spawned worker processes.

Each job builds the FP64 oracle model from the seeded synthetic weights in
the worker (the model is too large to pickle cheaply) and returns plain
numpy results, so several long oracle runs proceed side by side on the host
cores while the GPU side of a test runs.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

import synthetic as S
from oracle.coder import Encoder
from oracle.compress import StepConfig, StreamState
from oracle.model import Model


def compress_recorded(shape, seed: int, fmt: str, tokens, record_at, cfg: StepConfig | None = None):
    """Compress `tokens` on the oracle (Algorithm 1); returns the coded bit
    count, the ideal bits and, at each token index of record_at, the
    intermediate distributions (z, p_tilde, p_ng, p) and the CDF."""
    cfg = cfg or StepConfig()
    st = StreamState.new(Model(shape, S.weights(shape, seed), fmt), cfg)
    enc = Encoder(cfg.T)
    want = set(int(i) for i in record_at)
    rec = {}
    for k, t in enumerate(np.asarray(tokens)):
        _, _, cdf = st.predict()
        if k in want:
            z, pt, png, p = st._cur
            rec[k] = dict(z=z.copy(), p_tilde=pt.copy(), p_ng=None if png is None else png.copy(), p=p.copy(),
                          cdf=np.asarray(cdf, dtype=np.int64).copy())
        enc.encode(cdf, int(t))
        st.update(int(t))
    _, nbits = enc.finish()
    return dict(nbits=nbits, ideal_bits=st.ideal_bits, slides=st.cache.slides, records=rec)


def logits_recorded(shape, seed: int, fmt: str, tokens, record_at):
    """The oracle model alone over `tokens` (BOS first): logits z at each
    token index of record_at."""
    m = Model(shape, S.weights(shape, seed), fmt)
    cache = m.new_cache()
    want = set(int(i) for i in record_at)
    last = Model.BOS
    out = {}
    for k, t in enumerate(np.asarray(tokens)):
        if k > max(want):
            break
        z = m.step(cache, last)
        if k in want:
            out[k] = z.copy()
        last = int(t)
    return out


_BLAS_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


class OraclePool:
    """A pool of `workers` spawned processes whose BLAS libraries each use
    cores / workers threads (oversubscribed BLAS threads spin and slow every
    worker down many times over).  The thread limits sit in the environment
    from construction to close(), so every worker the pool starts inherits
    them; the calling process keeps the threads it already has."""

    def __init__(self, workers: int):
        per = str(max(1, (os.cpu_count() or 1) // workers))
        self._saved = {k: os.environ.get(k) for k in _BLAS_VARS}
        for k in _BLAS_VARS:
            os.environ[k] = per
        self.pool = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))

    def submit(self, fn, *args):
        return self.pool.submit(fn, *args)

    def close(self):
        self.pool.shutdown(wait=True, cancel_futures=True)
        for k, v in self._saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
