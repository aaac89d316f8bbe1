// Per-block arithmetic of the fixed-accuracy codec (one 4x4x4 block held in
// 64 registers).  Written as __host__ __device__ functions so the CUDA kernels
// in codec.cu and any host-side harness compile the very same code.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FZ_HD __host__ __device__ __forceinline__
#else
#define FZ_HD inline
#endif

namespace fwi {
namespace zblock {

constexpr int kS = 25;  // block-floating-point fraction bits
constexpr int kG = 11;  // guard planes
constexpr uint32_t kNB = 0xAAAAAAAAu;

FZ_HD int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}
FZ_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}
FZ_HD int popc64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __popcll(x);
#else
  return __builtin_popcountll(x);
#endif
}
// index of the lowest set bit (x != 0)
FZ_HD int ctz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}
FZ_HD float as_float(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
// x rounded toward zero to an integer (|x| < 2^31)
FZ_HD int trunc_to_int(float x) {
#ifdef __CUDA_ARCH__
  return __float2int_rz(x);
#else
  return (int)x;
#endif
}

// ---- coefficient order (ascending total sequency, ties x-fastest) ----------
struct PermTable {
  int v[64];
};
FZ_HD constexpr PermTable make_perm() {
  PermTable t{};
  int n = 0;
  for (int s = 0; s <= 9; ++s)
    for (int idx = 0; idx < 64; ++idx)
      if ((idx & 3) + ((idx >> 2) & 3) + (idx >> 4) == s) t.v[n++] = idx;
  return t;
}
FZ_HD constexpr int perm_at(int p) { return make_perm().v[p]; }

// ---- lifting transform on four values ---------------------------------------
// (x0..x3) -> (S, D, d0, d1): pair differences and floor means, the same on
// the two means, then the linear trend D/2 removed from both differences.
FZ_HD void lift_fwd(int& x0, int& x1, int& x2, int& x3) {
  int d0 = x1 - x0;
  int s0 = x0 + (d0 >> 1);
  int d1 = x3 - x2;
  int s1 = x2 + (d1 >> 1);
  int D = s1 - s0;
  int S = s0 + (D >> 1);
  int h = D >> 1;
  x0 = S;
  x1 = D;
  x2 = d0 - h;
  x3 = d1 - h;
}
FZ_HD void lift_inv(int& x0, int& x1, int& x2, int& x3) {
  int h = x1 >> 1;
  int d1 = x3 + h;
  int d0 = x2 + h;
  int s0 = x0 - h;
  int s1 = x1 + s0;
  int a2 = s1 - (d1 >> 1);
  int a3 = d1 + a2;
  int a0 = s0 - (d0 >> 1);
  int a1 = d0 + a0;
  x0 = a0;
  x1 = a1;
  x2 = a2;
  x3 = a3;
}
// The block lives in 64 uint32 registers throughout; the transform reads and
// writes them as two's-complement int32 (same bits, no extra registers).
FZ_HD void lift_fwd_u(uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t& a3) {
  int x0 = (int)a0, x1 = (int)a1, x2 = (int)a2, x3 = (int)a3;
  lift_fwd(x0, x1, x2, x3);
  a0 = (uint32_t)x0;
  a1 = (uint32_t)x1;
  a2 = (uint32_t)x2;
  a3 = (uint32_t)x3;
}
FZ_HD void lift_inv_u(uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t& a3) {
  int x0 = (int)a0, x1 = (int)a1, x2 = (int)a2, x3 = (int)a3;
  lift_inv(x0, x1, x2, x3);
  a0 = (uint32_t)x0;
  a1 = (uint32_t)x1;
  a2 = (uint32_t)x2;
  a3 = (uint32_t)x3;
}
FZ_HD void xform_fwd(uint32_t* q) {
#pragma unroll
  for (int l = 0; l < 16; ++l) lift_fwd_u(q[4 * l], q[4 * l + 1], q[4 * l + 2], q[4 * l + 3]);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i) lift_fwd_u(q[i + 16 * k], q[i + 16 * k + 4], q[i + 16 * k + 8], q[i + 16 * k + 12]);
#pragma unroll
  for (int l = 0; l < 16; ++l) lift_fwd_u(q[l], q[l + 16], q[l + 32], q[l + 48]);
}
FZ_HD void xform_inv(uint32_t* q) {
#pragma unroll
  for (int l = 0; l < 16; ++l) lift_inv_u(q[l], q[l + 16], q[l + 32], q[l + 48]);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i) lift_inv_u(q[i + 16 * k], q[i + 16 * k + 4], q[i + 16 * k + 8], q[i + 16 * k + 12]);
#pragma unroll
  for (int l = 0; l < 16; ++l) lift_inv_u(q[4 * l], q[4 * l + 1], q[4 * l + 2], q[4 * l + 3]);
}

// Byte permute: byte i of the result is byte ((s >> 4i) & 7) of the 8 bytes
// of (x, y), x first.
FZ_HD uint32_t byte_perm(uint32_t x, uint32_t y, uint32_t s) {
#ifdef __CUDA_ARCH__
  return __byte_perm(x, y, s);
#else
  const uint64_t v = (uint64_t)x | ((uint64_t)y << 32);
  uint32_t r = 0;
  for (int i = 0; i < 4; ++i) r |= (uint32_t)((v >> (8 * ((s >> (4 * i)) & 7u))) & 0xffu) << (8 * i);
  return r;
#endif
}

// 32x32 bit-matrix transpose in registers: afterwards bit i of a[b] is what
// was bit b of a[i] (recursive exchange of the off-diagonal blocks).  The
// 16-bit and 8-bit exchanges are byte permutes (two per word pair).
FZ_HD void transpose32(uint32_t* a) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {  // halves: a[k].hi <-> a[k+16].lo
    const uint32_t x = a[k], y = a[k + 16];
    a[k] = byte_perm(x, y, 0x5410u);
    a[k + 16] = byte_perm(x, y, 0x7632u);
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {  // bytes: bytes 1, 3 of a[k] <-> bytes 0, 2 of a[k+8]
    if (k & 8) continue;
    const uint32_t x = a[k], y = a[k + 8];
    a[k] = byte_perm(x, y, 0x6240u);
    a[k + 8] = byte_perm(x, y, 0x7351u);
  }
#pragma unroll
  for (int lv = 2; lv < 5; ++lv) {
    const int j = 16 >> lv;
    const uint32_t m = lv == 0 ? 0x0000FFFFu : lv == 1 ? 0x00FF00FFu : lv == 2 ? 0x0F0F0F0Fu
                     : lv == 3 ? 0x33333333u : 0x55555555u;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & j) continue;
      const uint32_t t = ((a[k] >> j) ^ a[k + j]) & m;
      a[k + j] ^= t;
      a[k] ^= t << j;
    }
  }
}

FZ_HD int planes_for(int emax, int minexp) {
  int p = emax - minexp + kG;
  p = p < 0 ? 0 : (p > 32 ? 32 : p);
  if (p == 30 || p == 31) p = 32;
  return p;
}

FZ_HD uint64_t plane(const uint32_t* u, int b) {
  return (uint64_t)u[b] | ((uint64_t)u[32 + b] << 32);
}

// FP32 bit patterns of a block -> 32 plane masks (u[b] | u[32+b] << 32 is
// plane b), block exponent and coded-plane count.  Returns false (and codes
// the block as zero) when the block holds NaN or Inf.
FZ_HD bool quantise_coeffs(uint32_t* u, int minexp, int& emax, int& planes);
FZ_HD bool quantise(uint32_t* u, int minexp, int& emax, int& planes) {
  const bool finite = quantise_coeffs(u, minexp, emax, planes);
  transpose32(u);
  transpose32(u + 32);
  return finite;
}

// The same up to the negabinary coefficients in sequency order (u[p] is
// coefficient p); the caller transposes the two halves into plane masks.
FZ_HD bool quantise_coeffs(uint32_t* u, int minexp, int& emax, int& planes) {
  uint32_t maxbits = 0;
#pragma unroll
  for (int i = 0; i < 64; ++i) maxbits = maxbits > (u[i] & 0x7fffffffu) ? maxbits : (u[i] & 0x7fffffffu);
  const bool finite = maxbits < 0x7f800000u;
  if (!finite) maxbits = 0;
  emax = 0;
  planes = 0;
  if (maxbits) {
    const int E = (int)(maxbits >> 23);
    const int e = E ? E - 126 : (32 - clz32(maxbits)) - 149;  // frexp exponent of max |x|
    emax = e > -127 ? e : -127;
    planes = planes_for(emax, minexp);
  }
  if (!planes) {  // nothing to code: skip the transform
#pragma unroll
    for (int i = 0; i < 64; ++i) u[i] = 0u;
    return finite;
  }
  // q = trunc(x 2^(S - emax)) (in place).  |x| < 2^emax, so |q| < 2^S.
  // Scaling by a power of two is exact whenever the product is a normal
  // number; a product that is not (subnormal or flushed to zero) is below 1
  // in magnitude and truncates to 0 either way.  2^(S - emax) is applied as
  // two normal factors because S - emax can exceed 127.
  const int k = kS - emax;  // -103 .. 152
  const int k1 = k < 127 ? k : 127;
  const float s1 = as_float((uint32_t)(k1 + 127) << 23), s2 = as_float((uint32_t)(k - k1 + 127) << 23);
#pragma unroll
  for (int i = 0; i < 64; ++i) u[i] = (uint32_t)trunc_to_int((as_float(u[i]) * s1) * s2);
  xform_fwd(u);
  // sequency order and negabinary, through a register permutation
  uint32_t c[64];
#pragma unroll
  for (int p = 0; p < 64; ++p) c[p] = (u[perm_at(p)] + kNB) ^ kNB;
#pragma unroll
  for (int p = 0; p < 64; ++p) u[p] = c[p];
  return finite;
}

// Exact number of bits the block codes to.
FZ_HD int count_bits(const uint32_t* u, int planes) {
  if (planes == 0) return 1;
  int nbits = 9, n = 0;
#pragma unroll
  for (int b = 31; b >= 0; --b) {
    if (b >= 32 - planes) {
      const uint64_t m = plane(u, b);
      const uint64_t r = n < 64 ? (m >> n) : 0ull;
      const int nend = r ? 64 - clz64(m) : n;
      nbits += nend + popc64(r) + (nend < 64 ? 1 : 0);
      n = nend;
    }
  }
  return nbits;
}

// The same count with the plane masks in memory: P(b) returns plane b (a
// rolled loop: small code for the instruction cache).
template <class P>
FZ_HD int count_bits_mem(const P& pl, int planes) {
  if (planes == 0) return 1;
  int nbits = 9, n = 0;
  for (int b = 31; b >= 32 - planes; --b) {
    const uint64_t m = pl(b);
    const uint64_t r = n < 64 ? (m >> n) : 0ull;
    const int nend = r ? 64 - clz64(m) : n;
    nbits += nend + popc64(r) + (nend < 64 ? 1 : 0);
    n = nend;
  }
  return nbits;
}

// Embedded bit-plane coding: per plane, the bits of the coefficients already
// significant, then group tests each followed by the run up to the next
// newly significant coefficient.  W provides put(value, nbits), 1..64 bits.
template <class W>
FZ_HD void emit(W& w, const uint32_t* u, int emax, int planes) {
  if (planes == 0) {
    w.put(0ull, 1);
    return;
  }
  w.put(1ull | ((uint64_t)(emax + 127) << 1), 9);
  int n = 0;
#pragma unroll
  for (int b = 31; b >= 0; --b) {
    if (b >= 32 - planes) {
      const uint64_t m = plane(u, b);
      if (n > 0) w.put(n < 64 ? (m & ((1ull << n) - 1ull)) : m, n);
      uint64_t r = n < 64 ? (m >> n) : 0ull;
      while (n < 64) {
        if (!r) {
          w.put(0ull, 1);
          break;
        }
        const int j = ctz64(r);
        if (j < 63) {
          w.put(1ull | (1ull << (j + 1)), j + 2);  // group bit, then the run up to the 1
        } else {
          w.put(1ull, 1);
          w.put(1ull << j, j + 1);
        }
        n += j + 1;
        r = (j + 1 < 64) ? (r >> (j + 1)) : 0ull;
      }
    }
  }
}

// emit with the plane masks in memory (P(b) returns plane b).  A plane's
// group-coded part is assembled in a 128-bit register pair (lo, hi) and
// written with one or two puts: its first group bit 1, then the bits of
// r = m >> n up to r's highest set bit, each set bit followed by a group bit
// (1 while another set bit follows, else the final 0, which is left out when
// the last set bit is coefficient 63).  A set bit of r at position p with i
// set bits below it lands at s = 1 + p + i, its group bit at s + 1; at most
// 128 bits (64 set bits from n = 0).
template <class W, class P>
FZ_HD void emit_mem(W& w, const P& pl, int emax, int planes) {
  if (planes == 0) {
    w.put(0ull, 1);
    return;
  }
  w.put(1ull | ((uint64_t)(emax + 127) << 1), 9);
  int n = 0;
  for (int b = 31; b >= 32 - planes; --b) {
    const uint64_t m = pl(b);
    if (n > 0) w.put(n < 64 ? (m & ((1ull << n) - 1ull)) : m, n);
    if (n >= 64) continue;
    uint64_t t = m >> n;
    if (!t) {
      w.put(0ull, 1);  // no newly significant coefficient
      continue;
    }
    uint64_t lo = 1ull, hi = 0ull;
    int i = 0, s = 0;
    do {
      const int p = ctz64(t);
      t &= t - 1ull;
      s = 1 + p + i;
      if (s < 63) {
        lo |= 3ull << s;
      } else if (s == 63) {
        lo |= 1ull << 63;
        hi |= 1ull;
      } else {
        hi |= 3ull << (s - 64);
      }
      ++i;
    } while (t);
    // the last set bit's group bit is the final 0 (or absent)
    if (s + 1 < 64)
      lo &= ~(1ull << (s + 1));
    else if (s + 1 < 128)
      hi &= ~(1ull << (s + 1 - 64));
    const int nend = n + (s - i) + 1;  // coefficients significant after this plane
    const int len = s + 1 + (nend < 64 ? 1 : 0);
    if (len <= 64) {
      w.put(lo, len);
    } else {
      w.put(lo, 64);
      w.put(hi, len - 64);
    }
    n = nend;
  }
}

// Inverse of emit: plane b goes to sink(b, mask) for every coded plane
// (uncoded planes are left to the caller).  R provides pos/end (bit
// positions) and peek() (the next 64 bits, zero past the words it holds).
// The next bits are held in a 64-bit window w (wa of them valid), refilled
// from the reader only when a field runs past it.  One loop pass reads one
// group test and its run, or finishes a plane and takes the next plane's
// verbatim bits, so a lane's passes follow its own block's runs rather than
// the warp's largest run count in every plane.  Whatever the bits, the loop
// stops after at most 64 runs and one pass per plane; the bounds are checked
// once, by the caller, which rejects the block unless the reader stops
// exactly at end.  Returns false on a malformed header or run.
template <class R, class K>
FZ_HD bool decode_planes_mem(R& rd, int minexp, K& sink, int& emax, int& planes) {
  emax = 0;
  planes = 0;
  if (rd.pos + 1 > rd.end) return false;
  uint64_t w = rd.peek();
  int wa = 64;
  if (!(w & 1ull)) {
    rd.pos += 1;
    return true;
  }
  if (rd.pos + 9 > rd.end) return false;
  emax = (int)((w >> 1) & 0xffull) - 127;
  rd.pos += 9;
  w >>= 9;
  wa -= 9;
  planes = planes_for(emax, minexp);
  if (planes == 0) return false;
  const int blast = 32 - planes;
  int b = 31, n = 0;  // the top plane has no verbatim bits
  uint64_t m = 0ull;
  for (;;) {
    if (n < 64) {  // a group test
      if (wa < 1) {
        w = rd.peek();
        wa = 64;
      }
      const bool group = (w & 1ull) != 0ull;
      rd.pos += 1;
      w >>= 1;
      wa -= 1;
      if (group) {  // the run: j zero bits, then the newly significant coefficient's 1
        int j = w ? ctz64(w) : 64;
        if (j >= wa) {
          w = rd.peek();
          wa = 64;
          j = w ? ctz64(w) : 64;
        }
        if (j >= 64 - n) return false;
        rd.pos += j + 1;
        if (j < 63) {
          w >>= j + 1;
          wa -= j + 1;
        } else {
          w = 0ull;
          wa = 0;
        }
        m |= 1ull << (n + j);
        n += j + 1;
        continue;
      }
    }
    sink(b, m);  // plane b is complete
    if (--b < blast) break;
    m = 0ull;
    if (n > 0) {  // the bits of the coefficients already significant, verbatim
      if (wa < n) {
        w = rd.peek();
        wa = 64;
      }
      rd.pos += n;
      if (n < 64) {
        m = w & ((1ull << n) - 1ull);
        w >>= n;
        wa -= n;
      } else {
        m = w;
        w = 0ull;
        wa = 0;
      }
    }
  }
  return true;
}

// Plane masks -> FP32 values: one rounding of q 2^(emax - S).
FZ_HD void dequantise(uint32_t* u, int emax, int planes, float* v) {
  if (planes == 0) {
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = 0.0f;
    return;
  }
  transpose32(u);
  transpose32(u + 32);
  uint32_t c[64];
#pragma unroll
  for (int p = 0; p < 64; ++p) c[perm_at(p)] = (u[p] ^ kNB) - kNB;
  xform_inv(c);
  const int* q = reinterpret_cast<const int*>(c);
  const int k = emax - kS;
  if (k >= -126) {
    const float scale = as_float((uint32_t)(k + 127) << 23);
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = (float)q[i] * scale;
  } else {
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = (float)((double)q[i] * exp2((double)k));
  }
}

}  // namespace zblock
}  // namespace fwi
