"""NC06 hybrid binary format (Sec. 3.10, Sec. 3.12): test infrastructure only.

Segmentation of an arbitrary byte string into alternating text and binary
runs, by the four rules of Sec. 3.10, applied in the order listed:
  1. a byte is text-like when it is printable ASCII (32..126), tab, LF or CR;
  2. a text run shorter than 64 bytes becomes binary;
  3. a binary gap of at most 8 bytes between two text runs becomes text;
  4. a binary run shorter than 64 bytes next to a text run becomes text.
Adjacent runs of one kind merge after each rule.  In this order every gap
rule 3 bridges is also a binary run under 64 bytes next to text, which rule
4 absorbs, so rule 3 changes nothing; it is kept as written.  Bridging
before the demotion would read uniformly random bytes as text (their short
text-like runs are mostly separated by gaps of at most 8 bytes).

The binary runs are concatenated into one blob, stored LZMA-compressed when
the blob holds at least 4 KB, gzip-compressed when smaller, or raw when the
compressed form is not shorter.  The text runs are coded as the streams of
one NC05 container (the caller supplies its bytes).

Container (little-endian):
    "NC06", version 1 (u8), flags (u8), tau (binary16), entry count E (u32),
    (the flags and tau of the text runs' NC05 container; 0 and 1.0 without text)
    E entries of kind (u8: 0 text, 1 binary) and length (u32),
    blob method (u8: 0 raw, 1 gzip, 2 LZMA), blob length (u32), blob,
    the text runs' NC05 container (empty when there is no text run).
"""
from __future__ import annotations

import gzip
import lzma
import struct

TEXT, BINARY = 0, 1
MIN_TEXT = 64          # rule 2: shorter text runs become binary
MAX_GAP = 8            # rule 3: binary gaps up to this length between text runs become text
MIN_BINARY = 64        # rule 4: shorter binary runs next to text become text
LZMA_MIN = 4096        # blobs of at least 4 KB try LZMA, smaller ones gzip
RAW, GZIP, LZMA = 0, 1, 2


def is_text_byte(b: int) -> bool:
    """Rule 1."""
    return 32 <= b <= 126 or b in (9, 10, 13)


def _merge(runs):
    out = []
    for kind, length in runs:
        if length == 0:
            continue
        if out and out[-1][0] == kind:
            out[-1] = (kind, out[-1][1] + length)
        else:
            out.append((kind, length))
    return out


def segment(data: bytes):
    """The runs [(kind, length), ...] covering data in order, kinds alternating."""
    # rule 1: every byte classified, maximal runs of one kind
    runs = []
    for b in data:
        kind = TEXT if is_text_byte(b) else BINARY
        if runs and runs[-1][0] == kind:
            runs[-1] = (kind, runs[-1][1] + 1)
        else:
            runs.append((kind, 1))
    # rule 2: short text runs
    runs = _merge([(BINARY if (k == TEXT and n < MIN_TEXT) else k, n) for k, n in runs])
    # rule 3: short gaps between two text runs
    runs = _merge([(TEXT if (k == BINARY and 0 < i < len(runs) - 1 and n <= MAX_GAP) else k, n)
                   for i, (k, n) in enumerate(runs)])
    # rule 4: short binary runs next to a text run
    has_text_neighbour = lambda i: (i > 0 and runs[i - 1][0] == TEXT) or (i + 1 < len(runs) and runs[i + 1][0] == TEXT)
    runs = _merge([(TEXT if (k == BINARY and n < MIN_BINARY and has_text_neighbour(i)) else k, n)
                   for i, (k, n) in enumerate(runs)])
    return runs


def split(data: bytes, runs):
    """The text runs' bytes and the binary blob (the binary runs concatenated)."""
    texts, blob, off = [], bytearray(), 0
    for kind, n in runs:
        if kind == TEXT:
            texts.append(bytes(data[off:off + n]))
        else:
            blob += data[off:off + n]
        off += n
    return texts, bytes(blob)


def pack_blob(blob: bytes):
    """(method, stored bytes) by the size rule, raw when compression does not help."""
    if not blob:
        return RAW, b""
    packed = (LZMA, lzma.compress(blob)) if len(blob) >= LZMA_MIN else (GZIP, gzip.compress(blob, mtime=0))
    return packed if len(packed[1]) < len(blob) else (RAW, blob)


def unpack_blob(method: int, stored: bytes) -> bytes:
    if method == RAW:
        return stored
    if method == GZIP:
        return gzip.decompress(stored)
    if method == LZMA:
        return lzma.decompress(stored)
    raise ValueError(f"unknown blob method {method}")


def pack(runs, method: int, stored: bytes, text_container: bytes) -> bytes:
    """The container; its flags byte and temperature are those of the text
    runs' NC05 container (bytes 4 and 5..6), or 0 and 1.0 without text."""
    if text_container:
        if text_container[:4] != b"NC05" or len(text_container) < 9:
            raise ValueError("the text section is not an NC05 container")
        flags, tau_half = text_container[4], struct.unpack_from("<H", text_container, 5)[0]
    else:
        flags, tau_half = 0, 0x3C00                      # 1.0 in binary16
    out = bytearray(b"NC06")
    out += struct.pack("<BBHI", 1, flags, tau_half, len(runs))
    for kind, n in runs:
        out += struct.pack("<BI", kind, n)
    out += struct.pack("<BI", method, len(stored))
    out += stored
    out += text_container
    return bytes(out)


def unpack(buf: bytes):
    """(flags, tau_half, runs, method, stored, text_container)."""
    if len(buf) < 12 or buf[:4] != b"NC06":
        raise ValueError("not an NC06 container")
    version, flags, tau_half, n = struct.unpack_from("<BBHI", buf, 4)
    if version != 1:
        raise ValueError(f"NC06 version {version}")
    off = 12
    runs = []
    for _ in range(n):
        kind, length = struct.unpack_from("<BI", buf, off)
        runs.append((kind, length))
        off += 5
    method, size = struct.unpack_from("<BI", buf, off)
    off += 5
    stored = bytes(buf[off:off + size])
    if len(stored) != size:
        raise ValueError("truncated NC06 binary section")
    return flags, tau_half, runs, method, stored, bytes(buf[off + size:])


def join(runs, texts, blob: bytes) -> bytes:
    """Inverse of split."""
    out, ti, bo = bytearray(), 0, 0
    for kind, n in runs:
        if kind == TEXT:
            out += texts[ti]
            ti += 1
        else:
            out += blob[bo:bo + n]
            bo += n
    return bytes(out)
