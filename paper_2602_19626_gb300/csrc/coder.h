// Host 32-bit arithmetic coder (Sec. 3.8, after Witten, Neal and Cleary 1987)
// and the NC05-style container (Sec. 3.12).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace nc {

// Encoder state: low, high in [0, 2^32) with high inclusive.  For an interval
// [lo, hi) of a total T = 2^log2T the range R = high - low + 1 narrows to
// high = low + floor(R hi / T) - 1, low += floor(R lo / T); renormalisation
// emits equal leading bits (plus pending opposite bits) and counts a pending
// bit while the range straddles the middle half.  After renormalisation
// R > 2^30, so every count >= 1 keeps a non-empty sub-interval.
class AcEncoder {
 public:
  explicit AcEncoder(int log2T) : log2T_(log2T) {}
  // false for an empty or out-of-range interval
  bool encode(uint32_t lo, uint32_t hi);
  void finish();
  const std::vector<uint8_t>& bytes() const { return out_; }
  uint64_t nbits() const { return nbits_; }

 private:
  void put(int b) {
    if ((nbits_ & 7) == 0) out_.push_back(0);
    if (b) out_.back() |= (uint8_t)(0x80u >> (nbits_ & 7));
    ++nbits_;
  }
  void emit(int b) {
    put(b);
    for (; pending_; --pending_) put(!b);
  }
  int log2T_;
  uint64_t low_ = 0, high_ = 0xFFFFFFFFull, pending_ = 0, nbits_ = 0;
  std::vector<uint8_t> out_;
};

class AcDecoder {
 public:
  AcDecoder(const uint8_t* bits, uint64_t nbits, int log2T);
  // the count in [0, T) that selects the next symbol
  uint32_t target() const;
  // consume the decoded symbol's interval [lo, hi)
  void consume(uint32_t lo, uint32_t hi);

 private:
  int bit() {
    const uint64_t i = pos_++;
    if (i >= nbits_) return 0;
    return (bits_[i >> 3] >> (7 - (i & 7))) & 1;
  }
  const uint8_t* bits_;
  uint64_t nbits_, pos_ = 0;
  int log2T_;
  uint64_t low_ = 0, high_ = 0xFFFFFFFFull, value_ = 0;
};

// rANS coder on the same integer CDFs (the ANS coder named as future work in
// Sec. 6): state x in [L, 2^32 L), L = 2^31, total M = 2^log2T (log2T <= 31).
// A symbol [lo, hi) with f = hi - lo encodes as x -> floor(x / f) M +
// (x mod f) + lo after moving the low 32 bits of x out while
// x >= (L / M) 2^32 f; it decodes as x -> f floor(x / M) + (x mod M) - lo,
// refilling 32 bits while x < L.  The encoder runs the symbols in reverse
// from x = L; its output is the final state (8 bytes, little-endian) and then
// the moved-out words in reverse order of writing (4 bytes each), which is
// the order the decoder reads them in.
// false for an empty or out-of-range interval
bool rans_encode(const uint32_t* lo, const uint32_t* hi, int64_t n, int log2T, std::vector<uint8_t>* out);

class RansDecoder {
 public:
  RansDecoder(const uint8_t* data, size_t nbytes, int log2T);
  // false for a length that is not 8 + 4 k bytes
  bool valid() const { return nbytes_ >= 8 && (nbytes_ - 8) % 4 == 0; }
  // the count in [0, M) that selects the next symbol
  uint32_t target() const { return (uint32_t)(x_ & mask_); }
  // consume the decoded symbol's interval [lo, hi)
  void consume(uint32_t lo, uint32_t hi);
  // every word read and the state back at L
  bool finished() const;

 private:
  const uint8_t* data_;
  size_t nbytes_, pos_ = 8;
  int log2T_;
  uint64_t mask_, x_ = 0;
};

// File-level chunking (Sec. 3.11) on token ids: cut k of n_chunks - 1 falls
// just after the first line-ending token (is_boundary[id] != 0) at or after
// position ceil(k n / n_chunks) - 1; cuts without a line end after them, at
// or before the previous cut, or at n are dropped.  cuts receives
// 0 = c_0 < ... < c_m = n (m <= n_chunks chunks; m = 0 for n = 0).
// false for out-of-range ids or n_chunks < 1.
bool split_points(const int32_t* tokens, int64_t n, const uint8_t* is_boundary, int V, int n_chunks,
                  std::vector<int64_t>* cuts);

// Container: "NC05", flags, tau (binary16), stream count, extension byte
// (weight format | path << 4), then per stream (tokens, bits, bytes) as
// little-endian uint32, then the payloads.
constexpr size_t kHeaderBytes = 9;
constexpr size_t kRecordBytes = 12;

struct StreamRecord {
  uint32_t ntok, nbits, nbytes;
};

uint16_t float_to_half_bits(float f);
float half_bits_to_float(uint16_t h);

size_t container_size(const std::vector<StreamRecord>& recs);
void container_write(uint8_t* out, uint8_t flags, float tau, uint8_t path_byte,
                     const std::vector<StreamRecord>& recs,
                     const std::vector<const std::vector<uint8_t>*>& payloads);
// false on malformed input
bool container_read(const uint8_t* in, size_t n, uint8_t* flags, float* tau, uint8_t* path_byte,
                    std::vector<StreamRecord>* recs, std::vector<const uint8_t*>* payloads);

// NC06 hybrid format (Sec. 3.10).  The runs of text (kind 0) and binary
// (kind 1) bytes of a byte string, alternating, by the four rules applied
// in the order listed: bytes classed text-like when printable ASCII
// (32..126), tab, LF or CR; text runs under 64 bytes become binary; binary
// gaps of at most 8 bytes between two text runs become text; binary runs
// under 64 bytes next to a text run become text.  Adjacent runs of one kind
// merge after each rule.
constexpr uint8_t kRunText = 0, kRunBinary = 1;
struct HybridRun {
  uint8_t kind;
  int64_t len;
};
void hybrid_segments(const uint8_t* data, int64_t n, std::vector<HybridRun>* runs);

// NC06 container: "NC06", version 1, flags, tau (binary16), run count (u32),
// per run kind (u8) and length (u32), the binary blob's method (u8: 0 raw,
// 1 gzip, 2 LZMA) and stored length (u32), the stored blob, then the text
// runs' NC05 container to the end.  Little-endian.
constexpr size_t kHybridHeaderBytes = 12, kHybridRunBytes = 5, kHybridBlobBytes = 5;
size_t hybrid_size(size_t n_runs, size_t n_stored, size_t n_text);
void hybrid_write(uint8_t* out, uint8_t flags, uint16_t tau_half, const std::vector<HybridRun>& runs, uint8_t method,
                  const uint8_t* stored, size_t n_stored, const uint8_t* text, size_t n_text);
// false on malformed input; offsets are into `in`
bool hybrid_read(const uint8_t* in, size_t n, uint8_t* flags, uint16_t* tau_half, std::vector<HybridRun>* runs,
                 uint8_t* method, size_t* stored_off, size_t* stored_len, size_t* text_off);

}  // namespace nc
