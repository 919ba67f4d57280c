"""Range asymmetric numeral systems (rANS) coder over integer CDFs, pure-Python
integers (test infrastructure only).

The paper names ANS as a future replacement of its arithmetic coder (Sec. 6,
Future Work); this is the range variant of Duda's asymmetric numeral systems,
on the same integer CDFs of total M = 2^n the quantiser produces (Sec. 3.3).

A symbol s has start c_s = cdf[s] and frequency f_s = cdf[s + 1] - cdf[s] >= 1.
The coder's state is one integer x, and the two maps are

    C(s, x) = floor(x / f_s) * M + (x mod f_s) + c_s        (encode)
    D(x)    = (s, f_s * floor(x / M) + (x mod M) - c_s)      (decode)

where s in D is the symbol with c_s <= x mod M < c_s + f_s.  D(C(s, x)) =
(s, x) exactly, and C grows x by a factor of about M / f_s, so the final state
carries the information -log2(f_s / M) per symbol.

Streaming: the state stays in I = [L, 2^32 L) with L = 2^31 (a multiple of M
for n <= 31).  The encoder takes the symbols in reverse order, starting from
x = L; before C(s, .) it moves the low 32 bits of x out while
x >= x_max(s) = (L / M) * 2^32 * f_s, which keeps C(s, x) inside I.  The
decoder takes the symbols in order and refills from the words after D while
x < L, so it reads the words in the reverse order of their writing; after the
last symbol its state is L again.

Byte layout: the encoder's final state as 8 little-endian bytes, then the
moved-out words in reverse order of writing, 4 little-endian bytes each.
"""
from __future__ import annotations

WORD_BITS = 32
WORD_MASK = (1 << WORD_BITS) - 1
L = 1 << 31


class AnsError(ValueError):
    pass


def encode(intervals, log2M: int) -> bytes:
    """Code the symbols given as (lo, hi) = (c_s, c_s + f_s) intervals, in order."""
    if not 1 <= log2M <= 31:
        raise AnsError("total out of range")
    M = 1 << log2M
    x = L
    words = []
    for lo, hi in reversed(list(intervals)):
        lo, hi = int(lo), int(hi)
        if not 0 <= lo < hi <= M:
            raise AnsError("empty or out-of-range interval")
        f = hi - lo
        x_max = ((L >> log2M) << WORD_BITS) * f
        while x >= x_max:
            words.append(x & WORD_MASK)
            x >>= WORD_BITS
        x = (x // f) * M + (x % f) + lo
    out = bytearray(x.to_bytes(8, "little"))
    for w in reversed(words):
        out += w.to_bytes(4, "little")
    return bytes(out)


class Decoder:
    def __init__(self, data: bytes, log2M: int):
        if not 1 <= log2M <= 31:
            raise AnsError("total out of range")
        if len(data) < 8 or (len(data) - 8) % 4:
            raise AnsError("truncated stream")
        self.data, self.log2M = data, log2M
        self.x = int.from_bytes(data[:8], "little")
        self.pos = 8

    def target(self) -> int:
        """The count value in [0, M) that selects the next symbol."""
        return self.x & ((1 << self.log2M) - 1)

    def consume(self, lo: int, hi: int):
        f = hi - lo
        self.x = f * (self.x >> self.log2M) + self.target() - lo
        # a valid stream leaves x >= f >= 1 here, so one refill reaches L;
        # the bound keeps a corrupt one (x = 0, zero words) from looping
        for _ in range(2):
            if self.x >= L:
                break
            w = 0
            if self.pos + 4 <= len(self.data):
                w = int.from_bytes(self.data[self.pos:self.pos + 4], "little")
            self.pos += 4
            self.x = (self.x << WORD_BITS) | w

    def decode(self, cdf) -> int:
        t = self.target()
        lo, hi = 0, len(cdf) - 2             # largest s with cdf[s] <= t
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if int(cdf[mid]) <= t:
                lo = mid
            else:
                hi = mid - 1
        self.consume(int(cdf[lo]), int(cdf[lo + 1]))
        return lo

    def finished(self) -> bool:
        """Every word read and the state back at L."""
        return self.x == L and self.pos == len(self.data)
