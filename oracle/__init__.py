"""FP64 CPU oracle of the per-token CDF step (test infrastructure only).

This package is the correctness reference for the CUDA path.  It is plain,
slow and written to be checked against the paper by eye:

* ``model``     - decoder-only transformer decode step with the sliding KV
                  window (Sec. 3.2, Eq. lm; Sec. 3.9), FP64.
* ``head``      - adaptive log-space bias head (Sec. 3.6).
* ``ngram``     - interpolated token N-gram with capped continuation lists
                  (Sec. 3.4).
* ``mixer``     - linear mixture with exponential-weights update (Sec. 3.5),
                  and the mixed-distribution NLL gradient used by the
                  differentiable update rule.
* ``cdf``       - CDF quantisation with per-symbol floors (Sec. 3.3).
* ``coder``     - 32-bit arithmetic coder (Sec. 3.8), pure-Python integers.
* ``ans``       - rANS coder on the same integer CDFs (the ANS coder named as
                  future work in Sec. 6), pure-Python integers.
* ``container`` - NC05-style container (Sec. 3.12).
* ``chunking``  - file-level split into chunks at line ends (Sec. 3.11), on
                  token ids.
* ``hybrid``    - NC06 hybrid binary format (Sec. 3.10): text / binary
                  segmentation, the binary blob and the container layout.
* ``compress``  - the compression / decompression loop (Algorithm 1).
* ``numerics``  - bf16 / fp8-e4m3 rounding used to derive the dequantised
                  weight variants from the FP32 canonical weights.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import anything from this package.  The CUDA path never does, and the
two share no code: the only common module is ``synthetic`` (seeded inputs).
"""
