"""NC05-style container (Sec. 3.12), little-endian.

Header, 9 bytes: magic 'NC05', 1-byte feature flags, 2-byte temperature tau,
2-byte stream (chunk) count.  Then one 12-byte record per stream (token
count, bit count, stream byte length), then the concatenated coded streams.

Readings where the paper is silent: byte order little-endian; tau is IEEE
binary16; flag bits: bit0 N-gram, bit1 adaptive head, bit2 confidence skip,
bit3 mixed-NLL update rule, bit4 the rANS coder (ans.py) in place of the
arithmetic coder.  One extension byte follows the 9-byte header and
records the numeric path (weight format in the low nibble, kernel path in the
high nibble), because a decoder must replay the encoder's exact arithmetic.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"NC05"
FLAG_NGRAM, FLAG_HEAD, FLAG_SKIP, FLAG_MIXED_NLL, FLAG_RANS = 1, 2, 4, 8, 16
HEADER = 9
RECORD = 12


class ContainerError(ValueError):
    pass


def pack(flags: int, tau: float, path_byte: int, records, payloads) -> bytes:
    tau16 = np.array([tau], dtype=np.float16).view(np.uint16)[0]
    out = bytearray(MAGIC)
    out += struct.pack("<BHH", flags, int(tau16), len(records))
    out += struct.pack("<B", path_byte)
    for (ntok, nbits, nbytes) in records:
        out += struct.pack("<III", ntok, nbits, nbytes)
    for p in payloads:
        out += p
    return bytes(out)


def unpack(buf: bytes):
    if len(buf) < HEADER + 1 or buf[:4] != MAGIC:
        raise ContainerError("bad magic or truncated header")
    flags, tau16, n = struct.unpack_from("<BHH", buf, 4)
    path_byte = buf[9]
    tau = float(np.array([tau16], dtype=np.uint16).view(np.float16)[0])
    off = HEADER + 1
    if len(buf) < off + RECORD * n:
        raise ContainerError("truncated stream table")
    recs = [struct.unpack_from("<III", buf, off + RECORD * j) for j in range(n)]
    off += RECORD * n
    payloads = []
    for (_, nbits, nbytes) in recs:
        if nbytes != (nbits + 7) // 8 or off + nbytes > len(buf):
            raise ContainerError("inconsistent stream record")
        payloads.append(buf[off:off + nbytes])
        off += nbytes
    if off != len(buf):
        raise ContainerError("trailing bytes")
    return flags, tau, path_byte, recs, payloads
