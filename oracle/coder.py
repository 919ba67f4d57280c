"""32-bit arithmetic coder (Sec. 3.8), after Witten, Neal and Cleary (1987).

State: low, high in [0, 2^32), high inclusive.  With R = high - low + 1 and a
symbol interval [cdf[s], cdf[s+1]) of a CDF totalling T:
    high = low + floor(R * cdf[s+1] / T) - 1
    low  = low + floor(R * cdf[s]   / T)
then renormalise: while both ends are in the lower half emit 0, in the upper
half emit 1 (each followed by the pending opposite bits), and while they
straddle the middle half (low >= Q, high < 3Q) count a pending bit; each case
doubles the range.  HALF = 2^31, Q = 2^30.  finish() counts one more pending
bit and emits 0 if low < Q else 1.  The decoder mirrors the narrowing with a
32-bit value register (bits past the end read as 0) and finds s by binary
search over the CDF.

After renormalisation low < HALF <= high and not (Q <= low and high < 3Q),
so R > Q = 2^30: every symbol of count >= 1 keeps a width of at least
R / T > 2^30 / T (64 at T = 2^24), so the coder never loses a symbol.  (The
paper states R >= 2^31 and a width of 128; with the pending-bit case the
guaranteed bound is R > 2^30.)
"""
from __future__ import annotations

TOP = (1 << 32) - 1
HALF = 1 << 31
QTR = 1 << 30


class BitWriter:
    def __init__(self):
        self.bits: list[int] = []

    def put(self, b: int):
        self.bits.append(b)

    def to_bytes(self) -> bytes:
        out = bytearray((len(self.bits) + 7) // 8)
        for i, b in enumerate(self.bits):
            if b:
                out[i >> 3] |= 0x80 >> (i & 7)
        return bytes(out)


class Encoder:
    def __init__(self, T: int):
        self.T = T
        self.low, self.high, self.pending = 0, TOP, 0
        self.w = BitWriter()
        self.min_range = TOP + 1

    def _emit(self, b):
        self.w.put(b)
        for _ in range(self.pending):
            self.w.put(1 - b)
        self.pending = 0

    def encode_interval(self, lo: int, hi: int):
        assert 0 <= lo < hi <= self.T
        R = self.high - self.low + 1
        self.high = self.low + (R * hi) // self.T - 1
        self.low = self.low + (R * lo) // self.T
        while True:
            if self.high < HALF:
                self._emit(0)
            elif self.low >= HALF:
                self._emit(1)
                self.low -= HALF
                self.high -= HALF
            elif self.low >= QTR and self.high < 3 * QTR:
                self.pending += 1
                self.low -= QTR
                self.high -= QTR
            else:
                break
            self.low = 2 * self.low
            self.high = 2 * self.high + 1
        self.min_range = min(self.min_range, self.high - self.low + 1)

    def encode(self, cdf, s: int):
        self.encode_interval(int(cdf[s]), int(cdf[s + 1]))

    def finish(self):
        self.pending += 1
        self._emit(0 if self.low < QTR else 1)
        return self.w.to_bytes(), len(self.w.bits)


class Decoder:
    def __init__(self, data: bytes, nbits: int, T: int):
        self.data, self.nbits, self.T = data, nbits, T
        self.pos = 0
        self.low, self.high = 0, TOP
        self.value = 0
        for _ in range(32):
            self.value = (self.value << 1) | self._bit()

    def _bit(self) -> int:
        i = self.pos
        self.pos += 1
        if i >= self.nbits:
            return 0
        return (self.data[i >> 3] >> (7 - (i & 7))) & 1

    def target(self) -> int:
        """The count value in [0, T) that selects the next symbol."""
        R = self.high - self.low + 1
        return ((self.value - self.low + 1) * self.T - 1) // R

    def decode(self, cdf) -> int:
        t = self.target()
        lo, hi = 0, len(cdf) - 2            # largest s with cdf[s] <= t
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if int(cdf[mid]) <= t:
                lo = mid
            else:
                hi = mid - 1
        s = lo
        self.consume(int(cdf[s]), int(cdf[s + 1]))
        return s

    def consume(self, lo: int, hi: int):
        R = self.high - self.low + 1
        self.high = self.low + (R * hi) // self.T - 1
        self.low = self.low + (R * lo) // self.T
        while True:
            if self.high < HALF:
                pass
            elif self.low >= HALF:
                self.low -= HALF
                self.high -= HALF
                self.value -= HALF
            elif self.low >= QTR and self.high < 3 * QTR:
                self.low -= QTR
                self.high -= QTR
                self.value -= QTR
            else:
                break
            self.low = 2 * self.low
            self.high = 2 * self.high + 1
            self.value = 2 * self.value + self._bit()
