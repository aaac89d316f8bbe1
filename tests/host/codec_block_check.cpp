// Host harness for tests/test_codec_block_host.py: runs the GPU codec's
// per-block code (paper_2009_12623_gb300/csrc/codec_block.cuh, compiled as
// plain C++) on blocks read from stdin, with the same plane-mask functors the
// kernels use, and writes what it codes and decodes to stdout.
//   stdin : int32 minexp, int32 n, then n blocks of 64 uint32 (FP32 bits, x fastest)
//   stdout: per block int32 nbits, int32 nwords, nwords uint64, 64 uint32 decoded bits,
//           int32 ok (decoder accepted the block and consumed exactly nbits),
//           int32 cut_ok, int32 long_ok (the same block declared one bit shorter or one bit
//           longer than it is was accepted: both must be 0)
#include <math.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../paper_2009_12623_gb300/csrc/codec_block.cuh"

using namespace fwi::zblock;

namespace {

struct Writer {  // LSB-first bit writer, as the kernels' shared-memory writer
  std::vector<uint64_t> w;
  uint64_t acc = 0;
  int fill = 0;
  void put(uint64_t v, int k) {
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

struct Reader {  // the kernels' bounded reader: peek() returns the next 64 bits
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

struct Planes {  // plane b from the [plane] arrays of low and high halves
  const uint32_t* lo;
  const uint32_t* hi;
  uint64_t operator()(int b) const { return (uint64_t)lo[b] | ((uint64_t)hi[b] << 32); }
};

struct Sink {
  uint32_t* lo;
  uint32_t* hi;
  void operator()(int b, uint64_t m) const {
    lo[b] = (uint32_t)m;
    hi[b] = (uint32_t)(m >> 32);
  }
};

}  // namespace

int main() {
  int32_t minexp = 0, n = 0;
  if (fread(&minexp, 4, 1, stdin) != 1 || fread(&n, 4, 1, stdin) != 1 || n < 0) return 2;
  for (int blk = 0; blk < n; ++blk) {
    uint32_t u[64];
    if (fread(u, 4, 64, stdin) != 64) return 2;
    // encoder: coefficients, the two plane transposes, exact count, emission
    int emax = 0, planes = 0;
    quantise_coeffs(u, minexp, emax, planes);
    uint32_t lo[32] = {0}, hi[32] = {0};
    if (planes) {
      transpose32(u);
      transpose32(u + 32);
      for (int b = 0; b < 32; ++b)
        if (b >= 32 - planes) {
          lo[b] = u[b];
          hi[b] = u[32 + b];
        }
    }
    const Planes pl{lo, hi};
    const int32_t nbits = count_bits_mem(pl, planes);
    Writer wr;
    emit_mem(wr, pl, emax, planes);
    wr.flush();
    const int32_t nwords = (int32_t)wr.w.size();
    // decoder: plane masks from the bits, then values
    uint32_t dlo[32] = {0}, dhi[32] = {0};
    Reader rd{wr.w.data(), 0, nbits, nwords};
    int demax = 0, dplanes = 0;
    Sink sink{dlo, dhi};
    int32_t ok = decode_planes_mem(rd, minexp, sink, demax, dplanes) && rd.pos == nbits ? 1 : 0;
    int32_t wrong_len_ok[2];
    for (int w = 0; w < 2; ++w) {
      const long end = w ? nbits + 1 : nbits - 1;
      uint32_t xlo[32] = {0}, xhi[32] = {0};
      Reader rx{wr.w.data(), 0, end, nwords};
      Sink sx{xlo, xhi};
      int xe = 0, xp = 0;
      wrong_len_ok[w] = decode_planes_mem(rx, minexp, sx, xe, xp) && rx.pos == end ? 1 : 0;
    }
    uint32_t q[64];
    for (int b = 0; b < 32; ++b) {
      const bool coded = b >= 32 - dplanes;
      q[b] = coded ? dlo[b] : 0u;
      q[32 + b] = coded ? dhi[b] : 0u;
    }
    float v[64];
    dequantise(q, demax, dplanes, v);
    fwrite(&nbits, 4, 1, stdout);
    fwrite(&nwords, 4, 1, stdout);
    fwrite(wr.w.data(), 8, wr.w.size(), stdout);
    fwrite(v, 4, 64, stdout);
    fwrite(&ok, 4, 1, stdout);
    fwrite(wrong_len_ok, 4, 2, stdout);
  }
  return 0;
}
