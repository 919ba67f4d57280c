// Host arithmetic coder and container (Sec. 3.8, Sec. 3.12).
#include "coder.h"

#include <cmath>
#include <cstring>

namespace nc {

namespace {
constexpr uint64_t kHalf = 1ull << 31;
constexpr uint64_t kQtr = 1ull << 30;
}  // namespace

bool AcEncoder::encode(uint32_t lo, uint32_t hi) {
  const uint64_t T = 1ull << log2T_;
  if (lo >= hi || hi > T) return false;
  const uint64_t R = high_ - low_ + 1;
  high_ = low_ + ((R * hi) >> log2T_) - 1;
  low_ = low_ + ((R * lo) >> log2T_);
  for (;;) {
    if (high_ < kHalf) {
      emit(0);
    } else if (low_ >= kHalf) {
      emit(1);
      low_ -= kHalf;
      high_ -= kHalf;
    } else if (low_ >= kQtr && high_ < 3 * kQtr) {
      ++pending_;
      low_ -= kQtr;
      high_ -= kQtr;
    } else {
      break;
    }
    low_ <<= 1;
    high_ = (high_ << 1) | 1;
  }
  return true;
}

void AcEncoder::finish() {
  ++pending_;
  emit(low_ < kQtr ? 0 : 1);
}

AcDecoder::AcDecoder(const uint8_t* bits, uint64_t nbits, int log2T)
    : bits_(bits), nbits_(nbits), log2T_(log2T) {
  for (int i = 0; i < 32; ++i) value_ = (value_ << 1) | (uint64_t)bit();
}

uint32_t AcDecoder::target() const {
  const uint64_t R = high_ - low_ + 1;
  return (uint32_t)((((value_ - low_ + 1) << log2T_) - 1) / R);
}

void AcDecoder::consume(uint32_t lo, uint32_t hi) {
  const uint64_t R = high_ - low_ + 1;
  high_ = low_ + ((R * hi) >> log2T_) - 1;
  low_ = low_ + ((R * lo) >> log2T_);
  for (;;) {
    if (high_ < kHalf) {
    } else if (low_ >= kHalf) {
      low_ -= kHalf;
      high_ -= kHalf;
      value_ -= kHalf;
    } else if (low_ >= kQtr && high_ < 3 * kQtr) {
      low_ -= kQtr;
      high_ -= kQtr;
      value_ -= kQtr;
    } else {
      break;
    }
    low_ <<= 1;
    high_ = (high_ << 1) | 1;
    value_ = (value_ << 1) | (uint64_t)bit();
  }
}

// ------------------------------------------------------------------ rANS
namespace {
constexpr uint64_t kRansL = 1ull << 31;
constexpr int kWordBits = 32;

uint64_t load_le(const uint8_t* p, int nbytes) {
  uint64_t v = 0;
  for (int i = nbytes - 1; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
void store_le(uint8_t* p, uint64_t v, int nbytes) {
  for (int i = 0; i < nbytes; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
}  // namespace

bool rans_encode(const uint32_t* lo, const uint32_t* hi, int64_t n, int log2T, std::vector<uint8_t>* out) {
  if (log2T < 1 || log2T > 31) return false;
  const uint64_t M = 1ull << log2T;
  uint64_t x = kRansL;
  std::vector<uint32_t> words;
  for (int64_t i = n - 1; i >= 0; --i) {
    if (lo[i] >= hi[i] || hi[i] > M) return false;
    const uint64_t f = hi[i] - lo[i];
    const uint64_t x_max = ((kRansL >> log2T) << kWordBits) * f;   // <= 2^63
    while (x >= x_max) {
      words.push_back((uint32_t)x);
      x >>= kWordBits;
    }
    x = (x / f) * M + (x % f) + lo[i];
  }
  out->assign(8 + 4 * words.size(), 0);
  store_le(out->data(), x, 8);
  uint8_t* p = out->data() + 8;
  for (size_t k = words.size(); k-- > 0; p += 4) store_le(p, words[k], 4);
  return true;
}

RansDecoder::RansDecoder(const uint8_t* data, size_t nbytes, int log2T)
    : data_(data), nbytes_(nbytes), log2T_(log2T), mask_((1ull << log2T) - 1) {
  if (valid()) x_ = load_le(data_, 8);
}

void RansDecoder::consume(uint32_t lo, uint32_t hi) {
  const uint64_t f = hi - lo;
  x_ = f * (x_ >> log2T_) + (x_ & mask_) - lo;
  // a valid stream leaves x >= f >= 1 here, so one refill reaches L; the
  // bound keeps a corrupt one (x = 0, zero words) from looping
  for (int k = 0; k < 2 && x_ < kRansL; ++k) {
    const uint64_t w = pos_ + 4 <= nbytes_ ? load_le(data_ + pos_, 4) : 0;
    pos_ += 4;
    x_ = (x_ << kWordBits) | w;
  }
}

bool RansDecoder::finished() const { return x_ == kRansL && pos_ == nbytes_; }

// ------------------------------------------------------- file-level chunks
bool split_points(const int32_t* tokens, int64_t n, const uint8_t* is_boundary, int V, int n_chunks,
                  std::vector<int64_t>* cuts) {
  cuts->assign(1, 0);
  if (n_chunks < 1) return false;
  for (int64_t i = 0; i < n; ++i)
    if (tokens[i] < 0 || tokens[i] >= V) return false;
  if (n == 0) return true;
  for (int k = 1; k < n_chunks; ++k) {
    const int64_t target = (k * n + n_chunks - 1) / n_chunks;      // ceil(k n / N)
    int64_t p = target > 0 ? target - 1 : 0;
    while (p < n && !is_boundary[tokens[p]]) ++p;
    if (p >= n) break;                                               // no line end after the target
    const int64_t c = p + 1;
    if (c > cuts->back() && c < n) cuts->push_back(c);
  }
  cuts->push_back(n);
  return true;
}

// IEEE binary16 conversion, round to nearest even (for the 2-byte tau field).
uint16_t float_to_half_bits(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint32_t sign = (x >> 16) & 0x8000u;
  const int32_t exp = (int32_t)((x >> 23) & 0xFF) - 127 + 15;
  uint32_t mant = x & 0x7FFFFFu;
  if (((x >> 23) & 0xFF) == 0xFF) return (uint16_t)(sign | 0x7C00u | (mant ? 0x200u : 0));
  if (exp >= 31) return (uint16_t)(sign | 0x7C00u);
  if (exp <= 0) {
    if (exp < -10) return (uint16_t)sign;
    mant |= 0x800000u;
    const int shift = 14 - exp;
    uint32_t hm = mant >> shift;
    const uint32_t rem = mant & ((1u << shift) - 1), halfway = 1u << (shift - 1);
    if (rem > halfway || (rem == halfway && (hm & 1))) ++hm;
    return (uint16_t)(sign | hm);
  }
  uint32_t h = sign | ((uint32_t)exp << 10) | (mant >> 13);
  const uint32_t rem = mant & 0x1FFFu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1))) ++h;
  return (uint16_t)h;
}

float half_bits_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
  const int exp = (h >> 10) & 0x1F;
  const uint32_t mant = h & 0x3FFu;
  float f;
  if (exp == 0) {
    f = std::ldexp((float)mant, -24);
    if (sign) f = -f;
    return f;
  }
  uint32_t x;
  if (exp == 31)
    x = sign | 0x7F800000u | (mant << 13);
  else
    x = sign | ((uint32_t)(exp - 15 + 127) << 23) | (mant << 13);
  std::memcpy(&f, &x, 4);
  return f;
}

static void put_u16(uint8_t* p, uint16_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
}
static void put_u32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static uint16_t get_u16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t get_u32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

size_t container_size(const std::vector<StreamRecord>& recs) {
  size_t n = kHeaderBytes + 1 + kRecordBytes * recs.size();
  for (const auto& r : recs) n += r.nbytes;
  return n;
}

void container_write(uint8_t* out, uint8_t flags, float tau, uint8_t path_byte,
                     const std::vector<StreamRecord>& recs,
                     const std::vector<const std::vector<uint8_t>*>& payloads) {
  std::memcpy(out, "NC05", 4);
  out[4] = flags;
  put_u16(out + 5, float_to_half_bits(tau));
  put_u16(out + 7, (uint16_t)recs.size());
  out[9] = path_byte;
  uint8_t* p = out + kHeaderBytes + 1;
  for (const auto& r : recs) {
    put_u32(p, r.ntok);
    put_u32(p + 4, r.nbits);
    put_u32(p + 8, r.nbytes);
    p += kRecordBytes;
  }
  for (size_t i = 0; i < recs.size(); ++i) {
    if (recs[i].nbytes) std::memcpy(p, payloads[i]->data(), recs[i].nbytes);
    p += recs[i].nbytes;
  }
}

namespace {
bool text_like(uint8_t b) { return (b >= 32 && b <= 126) || b == 9 || b == 10 || b == 13; }
void merge_runs(std::vector<HybridRun>* r) {
  std::vector<HybridRun> out;
  for (const HybridRun& x : *r) {
    if (x.len == 0) continue;
    if (!out.empty() && out.back().kind == x.kind) out.back().len += x.len;
    else out.push_back(x);
  }
  r->swap(out);
}
}  // namespace

void hybrid_segments(const uint8_t* data, int64_t n, std::vector<HybridRun>* runs) {
  std::vector<HybridRun>& r = *runs;
  r.clear();
  for (int64_t i = 0; i < n; ++i) {                      // rule 1: maximal runs of one class
    const uint8_t k = text_like(data[i]) ? kRunText : kRunBinary;
    if (!r.empty() && r.back().kind == k) ++r.back().len;
    else r.push_back({k, 1});
  }
  for (HybridRun& x : r)                                 // rule 2
    if (x.kind == kRunText && x.len < 64) x.kind = kRunBinary;
  merge_runs(runs);
  // rule 3: runs alternate, so a binary run with a run on both sides lies
  // between two text runs
  for (size_t i = 1; i + 1 < r.size(); ++i)
    if (r[i].kind == kRunBinary && r[i].len <= 8) r[i].kind = kRunText;
  merge_runs(runs);
  // rule 4: a binary run has a text neighbour unless it is the only run
  if (r.size() > 1)
    for (HybridRun& x : r)
      if (x.kind == kRunBinary && x.len < 64) x.kind = kRunText;
  merge_runs(runs);
}

size_t hybrid_size(size_t n_runs, size_t n_stored, size_t n_text) {
  return kHybridHeaderBytes + kHybridRunBytes * n_runs + kHybridBlobBytes + n_stored + n_text;
}

void hybrid_write(uint8_t* out, uint8_t flags, uint16_t tau_half, const std::vector<HybridRun>& runs, uint8_t method,
                  const uint8_t* stored, size_t n_stored, const uint8_t* text, size_t n_text) {
  std::memcpy(out, "NC06", 4);
  out[4] = 1;
  out[5] = flags;
  put_u16(out + 6, tau_half);
  put_u32(out + 8, (uint32_t)runs.size());
  size_t off = kHybridHeaderBytes;
  for (const HybridRun& x : runs) {
    out[off] = x.kind;
    put_u32(out + off + 1, (uint32_t)x.len);
    off += kHybridRunBytes;
  }
  out[off] = method;
  put_u32(out + off + 1, (uint32_t)n_stored);
  off += kHybridBlobBytes;
  if (n_stored) std::memcpy(out + off, stored, n_stored);
  off += n_stored;
  if (n_text) std::memcpy(out + off, text, n_text);
}

bool hybrid_read(const uint8_t* in, size_t n, uint8_t* flags, uint16_t* tau_half, std::vector<HybridRun>* runs,
                 uint8_t* method, size_t* stored_off, size_t* stored_len, size_t* text_off) {
  if (!in || n < kHybridHeaderBytes + kHybridBlobBytes || std::memcmp(in, "NC06", 4) != 0 || in[4] != 1) return false;
  *flags = in[5];
  *tau_half = get_u16(in + 6);
  const size_t nr = get_u32(in + 8);
  if ((n - kHybridHeaderBytes - kHybridBlobBytes) / kHybridRunBytes < nr) return false;
  size_t off = kHybridHeaderBytes;
  runs->resize(nr);
  for (size_t j = 0; j < nr; ++j) {
    const uint8_t k = in[off];
    const uint32_t len = get_u32(in + off + 1);
    if (k > kRunBinary || len == 0) return false;
    (*runs)[j] = {k, (int64_t)len};
    off += kHybridRunBytes;
  }
  *method = in[off];
  *stored_len = get_u32(in + off + 1);
  off += kHybridBlobBytes;
  if (*method > 2 || *stored_len > n - off) return false;
  *stored_off = off;
  *text_off = off + *stored_len;
  return true;
}

bool container_read(const uint8_t* in, size_t n, uint8_t* flags, float* tau, uint8_t* path_byte,
                    std::vector<StreamRecord>* recs, std::vector<const uint8_t*>* payloads) {
  if (!in || n < kHeaderBytes + 1 || std::memcmp(in, "NC05", 4) != 0) return false;
  *flags = in[4];
  *tau = half_bits_to_float(get_u16(in + 5));
  const size_t ns = get_u16(in + 7);
  *path_byte = in[9];
  size_t off = kHeaderBytes + 1;
  if (n < off + kRecordBytes * ns) return false;
  recs->resize(ns);
  for (size_t j = 0; j < ns; ++j) {
    (*recs)[j].ntok = get_u32(in + off);
    (*recs)[j].nbits = get_u32(in + off + 4);
    (*recs)[j].nbytes = get_u32(in + off + 8);
    off += kRecordBytes;
  }
  payloads->resize(ns);
  for (size_t j = 0; j < ns; ++j) {
    const auto& r = (*recs)[j];
    if ((uint64_t)r.nbytes != ((uint64_t)r.nbits + 7) / 8 || off + r.nbytes > n) return false;
    (*payloads)[j] = in + off;
    off += r.nbytes;
  }
  return off == n;
}

}  // namespace nc
