// Host harness for tests/test_codec_block_host.py: the GPU codec's embedded
// coder (emit_mem, compiled as plain C++) on plane masks chosen to reach the
// edges of its 128-bit group-coded assembly (all 64 coefficients significant
// in the top plane, coefficient 63 alone, runs ending at 63), checked against
// a direct bit-by-bit restatement of the group coding, against the exact bit
// count, and by decoding the bits back.  Prints "ok <cases>" or the first
// failing case.
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "../../paper_2009_12623_gb300/csrc/codec_block.cuh"

using namespace fwi::zblock;

namespace {

struct Writer {  // LSB-first bit writer
  std::vector<uint64_t> w;
  uint64_t acc = 0;
  int fill = 0;
  long bits = 0;
  void put(uint64_t v, int k) {
    bits += k;
    if (k == 0) return;
    acc |= v << fill;
    int nf = fill + k;
    if (nf >= 64) {
      w.push_back(acc);
      acc = fill ? (v >> (64 - fill)) : 0ull;
      nf -= 64;
    }
    fill = nf;
  }
  void flush() {
    if (fill) w.push_back(acc);
  }
};

struct BitList {  // reference: one bit per call
  std::vector<int> b;
  void bit(int v) { b.push_back(v & 1); }
};

// The group coding restated bit by bit: for each plane from the top, the
// bits of the already significant coefficients; then, while not all 64 are
// significant, a group bit saying whether any of the rest is set in this
// plane, and if so the run of zeros up to the next set one and that one.
void reference(const uint64_t* plane, int emax, int planes, BitList& out) {
  out.bit(1);
  for (int i = 0; i < 8; ++i) out.bit((emax + 127) >> i);
  int n = 0;
  for (int b = 31; b >= 32 - planes; --b) {
    const uint64_t m = plane[b];
    for (int i = 0; i < n; ++i) out.bit((int)(m >> i));
    while (n < 64) {
      bool any = false;
      for (int i = n; i < 64; ++i) any |= ((m >> i) & 1) != 0;
      out.bit(any);
      if (!any) break;
      while (!((m >> n) & 1)) {
        out.bit(0);
        ++n;
      }
      out.bit(1);
      ++n;
    }
  }
}

struct Planes {
  const uint64_t* p;
  uint64_t operator()(int b) const { return p[b]; }
};

struct Reader {
  const uint64_t* buf;
  long pos, end, nw;
  uint64_t peek() const {
    const long i = pos >> 6;
    const int o = (int)(pos & 63);
    uint64_t v = i < nw ? buf[i] : 0ull;
    v >>= o;
    if (o && i + 1 < nw) v |= buf[i + 1] << (64 - o);
    return v;
  }
};

struct Sink {
  uint64_t* p;
  void operator()(int b, uint64_t m) const { p[b] = m; }
};

bool check(const uint64_t* plane, int planes, int emax, int minexp, int id) {
  BitList ref;
  reference(plane, emax, planes, ref);
  Writer wr;
  emit_mem(wr, Planes{plane}, emax, planes);
  wr.flush();
  if (wr.bits != (long)ref.b.size() || count_bits_mem(Planes{plane}, planes) != (int)ref.b.size()) {
    printf("case %d: %ld bits emitted, %zu expected\n", id, wr.bits, ref.b.size());
    return false;
  }
  for (size_t i = 0; i < ref.b.size(); ++i)
    if ((int)((wr.w[i >> 6] >> (i & 63)) & 1) != ref.b[i]) {
      printf("case %d: bit %zu differs\n", id, i);
      return false;
    }
  uint64_t back[32] = {0};
  Reader rd{wr.w.data(), 0, (long)ref.b.size(), (long)wr.w.size()};
  Sink sk{back};
  int de = 0, dp = 0;
  if (!decode_planes_mem(rd, minexp, sk, de, dp) || rd.pos != rd.end || de != emax || dp != planes) {
    printf("case %d: decoding failed\n", id);
    return false;
  }
  for (int b = 31; b >= 32 - planes; --b)
    if (back[b] != plane[b]) {
      printf("case %d: plane %d decodes differently\n", id, b);
      return false;
    }
  return true;
}

}  // namespace

int main() {
  const int emax = 0, minexp = -21;  // planes_for(0, -21) = 32
  const int planes = planes_for(emax, minexp);
  std::vector<std::vector<uint64_t>> cases;
  auto add = [&](std::vector<uint64_t> top) {  // given top planes, the rest random
    std::vector<uint64_t> p(32, 0);
    for (size_t i = 0; i < top.size(); ++i) p[31 - i] = top[i];
    cases.push_back(p);
  };
  add({~0ull});                                 // every coefficient in the top plane
  add({1ull << 63});                            // coefficient 63 alone
  add({3ull << 62});                            // 62 and 63
  add({1ull, 1ull << 63});                      // 0, then 63 in the next plane
  add({0ull, ~0ull});                           // an empty top plane, then all
  add({0x8000000000000001ull, ~0ull});          // both ends, then all
  add({0x5555555555555555ull});                 // every other coefficient
  add({0xaaaaaaaaaaaaaaaaull});                 // every other, from 1 (ends at 63)
  add({0x7fffffffffffffffull, 1ull << 63});     // 0..62, then 63
  std::mt19937_64 rng(7);
  for (int k = 0; k < 2000; ++k) {              // random planes, dense to sparse
    std::vector<uint64_t> p(32);
    for (int b = 0; b < 32; ++b) {
      uint64_t v = rng();
      for (int r = 0; r < (int)(rng() % 4); ++r) v &= rng();
      p[b] = v;
    }
    cases.push_back(p);
  }
  int id = 0;
  for (auto& p : cases)
    if (!check(p.data(), planes, emax, minexp, id++)) return 1;
  printf("ok %d\n", id);
  return 0;
}
