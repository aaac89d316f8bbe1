// Fixed-accuracy block codec for FP32 wavefields on sm_103a (Sec. 1.3 of
// Kukreja et al.: every checkpoint is compressed with an absolute error
// tolerance atol; the format is this project's ZFP-style design).
//
// Per 4x4x4 block: block exponent -> 25-bit block-floating-point integers ->
// integer lifting transform along x, y, z -> sequency order -> negabinary ->
// embedded bit planes (planes = emax - minexp + 11, raised to 32 when fewer
// than 3 planes would be dropped).
//
// GPU organisation: one thread per block, one CTA (128 threads) per chunk of
// 128 consecutive blocks.  The 64 coefficients of a block live in registers;
// two 32x32 bit-matrix transposes turn them into 64-bit plane masks, from
// which the exact bit count of every plane is computed with popc/clz.  A CTA
// scan of the counts and a decoupled look-back across chunks (chunk order is
// the CTA's ticket order, so every predecessor is already resident) give each
// chunk its word offset in one pass; the chunk's bits are then assembled in
// shared memory and written with coalesced 64-bit stores.  Decoding reverses
// this with one CTA per chunk: the chunk's words are staged in shared memory,
// block offsets come from a scan of the u16 length table, and each thread
// rebuilds its plane masks (ctz finds every newly significant coefficient).
#include <cuda_runtime.h>
#include <stdint.h>

#include "codec_block.cuh"
#include "common.cuh"

namespace fwi {
namespace {

using namespace zblock;

constexpr int kWordsMax = (ZC_CHUNK * ZC_MAXBITS + 63) / 64;  // 4242 words
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr long kSpinLimit = 1L << 24;

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Shared-memory bit writer (words assembled with atomicOr, so neighbouring
// threads may share a boundary word).
struct SWriter {
  unsigned long long* buf;
  unsigned long long acc;
  int fill;
  int word;
  __device__ __forceinline__ void put(unsigned long long v, int k) {  // 1 <= k <= 64
    acc |= v << fill;
    int nf = fill + k;
    if (nf >= 64) {
      atomicOr(&buf[word], acc);
      ++word;
      acc = fill ? (v >> (64 - fill)) : 0ull;
      nf -= 64;
    }
    fill = nf;
  }
  __device__ __forceinline__ void flush() {
    if (fill) atomicOr(&buf[word], acc);
  }
};

struct EncArgs {
  const float* in;
  int nx, ny, nz;
  long pitch;
  long nbx, nby, nblocks, nchunks;
  int minexp;
  uint8_t* out;
  const unsigned long long* base;
  unsigned long long limit;
  unsigned long long chunk_table, length_table, payload;
  unsigned long long* size_out;
  int* status;
  unsigned long long* desc;
  unsigned int* ticket;
};

__device__ __forceinline__ void put_u32(uint8_t* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }
__device__ __forceinline__ void put_u64(uint8_t* p, unsigned long long v) {
  *reinterpret_cast<unsigned long long*>(p) = v;
}

__global__ void __launch_bounds__(ZC_CHUNK) k_encode(EncArgs a) {
  __shared__ unsigned long long sbuf[kWordsMax + 1];
  __shared__ int s_chunk;
  __shared__ unsigned s_warp[ZC_CHUNK / 32];
  __shared__ unsigned long long s_prefix;
  const int tid = threadIdx.x;
  if (tid == 0) s_chunk = (int)atomicAdd(a.ticket, 1u);
  __syncthreads();
  const long chunk = s_chunk;
  const long blk = chunk * ZC_CHUNK + tid;
  const bool valid = blk < a.nblocks;
  const unsigned long long base = a.base ? *a.base : 0ull;
  const unsigned long long avail = a.limit > base ? a.limit - base : 0ull;
  uint8_t* out = a.out + base;

  // ---- gather the block (edge blocks replicate the last plane) ------------
  uint32_t u[64];
  int planes = 0, emax = 0, nbits = 0;
  if (valid) {
    const long bx = blk % a.nbx, by = (blk / a.nbx) % a.nby, bz = blk / (a.nbx * a.nby);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long z = min(4 * bz + k, (long)a.nz - 1);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long y = min(4 * by + j, (long)a.ny - 1);
        const float* row = a.in + a.pitch * (y + (long)a.ny * z);
#pragma unroll
        for (int i = 0; i < 4; ++i) u[i + 4 * j + 16 * k] = __float_as_uint(__ldg(row + min(4 * bx + i, (long)a.nx - 1)));
      }
    }
    if (!quantise(u, a.minexp, emax, planes)) atomicOr(a.status, ST_NONFINITE);
    nbits = count_bits(u, planes);
  }

  // ---- CTA exclusive scan of bit counts ------------------------------------
  const int lane = tid & 31, warp = tid >> 5;
  unsigned incl = (unsigned)nbits;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  unsigned warp_off = 0, total = 0;
#pragma unroll
  for (int w = 0; w < ZC_CHUNK / 32; ++w) {
    if (w < warp) warp_off += s_warp[w];
    total += s_warp[w];
  }
  const unsigned my_off = warp_off + incl - (unsigned)nbits;
  const unsigned W = (total + 63u) / 64u;

  // ---- decoupled look-back over chunks --------------------------------------
  if (tid == 0) {
    unsigned long long prefix = 0;
    if (chunk == 0) {
      st_release(&a.desc[0], kFlagPre | W);
    } else {
      st_release(&a.desc[chunk], kFlagAgg | W);
      long p = chunk - 1;
      while (p >= 0) {
        unsigned long long d;
        long spins = 0;
        while (((d = ld_acquire(&a.desc[p])) >> 62) == 0ull) {
          if (++spins > kSpinLimit) {
            atomicOr(a.status, ST_TIMEOUT);
            d = kFlagPre;
            break;
          }
          __nanosleep(32);
        }
        prefix += d & kValMask;
        if ((d >> 62) == 2ull) break;
        --p;
      }
      st_release(&a.desc[chunk], kFlagPre | (prefix + W));
    }
    s_prefix = prefix;
  }
  for (unsigned w = tid; w < W; w += ZC_CHUNK) sbuf[w] = 0ull;
  __syncthreads();
  const unsigned long long prefix = s_prefix;

  // ---- emit the bits into shared memory -----------------------------------
  if (valid) {
    SWriter wr{sbuf, 0ull, (int)(my_off & 63u), (int)(my_off >> 6)};
    emit(wr, u, emax, planes);
    wr.flush();
  }
  __syncthreads();

  // ---- write payload, tables and (last chunk) the header -------------------
  const unsigned long long pay = a.payload + 8ull * prefix;
  for (unsigned w = tid; w < W; w += ZC_CHUNK) {
    const unsigned long long off = pay + 8ull * w;
    if (off + 8 <= avail) put_u64(out + off, sbuf[w]);
  }
  if (valid) {
    const unsigned long long off = a.length_table + 2ull * blk;
    if (off + 2 <= avail) *reinterpret_cast<uint16_t*>(out + off) = (uint16_t)nbits;
  }
  if (tid == 0) {
    const unsigned long long off = a.chunk_table + 8ull * chunk;
    if (off + 8 <= avail) put_u64(out + off, prefix);
  }
  if (chunk == a.nchunks - 1) {
    // zero padding of the length table after the last block
    const unsigned long long lt_end = a.length_table + 2ull * a.nblocks;
    for (unsigned long long off = lt_end + 2ull * tid; off < a.payload; off += 2ull * ZC_CHUNK)
      if (off + 2 <= avail) *reinterpret_cast<uint16_t*>(out + off) = 0;
    if (tid == 0) {
      const unsigned long long words = prefix + W;
      const unsigned long long bytes = a.payload + 8ull * words;
      if (64 <= avail) {
        put_u32(out + 0, ZC_MAGIC);
        put_u32(out + 4, ZC_VERSION);
        put_u32(out + 8, (uint32_t)a.nx);
        put_u32(out + 12, (uint32_t)a.ny);
        put_u32(out + 16, (uint32_t)a.nz);
        put_u32(out + 20, (uint32_t)a.minexp);
        put_u64(out + 24, (unsigned long long)a.nblocks);
        put_u32(out + 32, (uint32_t)ZC_CHUNK);
        put_u32(out + 36, (uint32_t)a.nchunks);
        put_u64(out + 40, words);
        put_u64(out + 48, bytes);
        put_u32(out + 56, (uint32_t)(ZC_S | (ZC_G << 8)));
        put_u32(out + 60, 0u);
      }
      if (bytes > avail) atomicOr(a.status, ST_CAPACITY);
      *a.size_out = bytes;
    }
  }
}

// ---- decoder ------------------------------------------------------------------

struct DecArgs {
  const uint8_t* in;
  const unsigned long long* base;
  unsigned long long avail;  // bytes readable from the stream start (when base == NULL)
  unsigned long long limit;  // bytes readable from `in` (when base != NULL)
  float* out;
  int nx, ny, nz;
  long pitch;
  long nbx, nby, nblocks, nchunks;
  unsigned long long chunk_table, length_table, payload;
  int* status;
};

struct SReader {
  const unsigned long long* buf;
  long pos;
  long end;
  __device__ __forceinline__ unsigned long long peek() const {
    const long w = pos >> 6;
    const int o = (int)(pos & 63);
    unsigned long long v = buf[w] >> o;
    if (o) v |= buf[w + 1] << (64 - o);
    return v;
  }
};

__device__ __forceinline__ uint32_t get_u32(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ unsigned long long get_u64(const uint8_t* p) {
  return *reinterpret_cast<const unsigned long long*>(p);
}

__global__ void __launch_bounds__(ZC_CHUNK) k_decode(DecArgs a) {
  __shared__ unsigned long long sbuf[kWordsMax + 2];
  __shared__ unsigned s_warp[ZC_CHUNK / 32];
  __shared__ unsigned long long s_first, s_words;
  __shared__ int s_minexp, s_bad;
  const int tid = threadIdx.x;
  const long chunk = blockIdx.x;
  const unsigned long long base = a.base ? *a.base : 0ull;
  const unsigned long long avail = a.base ? (a.limit > base ? a.limit - base : 0ull) : a.avail;
  const uint8_t* in = a.in + base;
  if (tid == 0) {
    int bad = 0;
    unsigned long long first = 0, words = 0;
    int minexp = 0;
    if (a.payload > avail || get_u32(in) != ZC_MAGIC || get_u32(in + 4) != ZC_VERSION ||
        (int)get_u32(in + 8) != a.nx || (int)get_u32(in + 12) != a.ny ||
        (int)get_u32(in + 16) != a.nz || get_u64(in + 24) != (unsigned long long)a.nblocks ||
        get_u32(in + 32) != (uint32_t)ZC_CHUNK || get_u32(in + 36) != (uint32_t)a.nchunks ||
        get_u32(in + 56) != (uint32_t)(ZC_S | (ZC_G << 8))) {
      bad = 1;
    } else {
      minexp = (int)get_u32(in + 20);
      const unsigned long long total = get_u64(in + 40);
      first = get_u64(in + a.chunk_table + 8ull * chunk);
      const unsigned long long next =
          chunk + 1 < a.nchunks ? get_u64(in + a.chunk_table + 8ull * (chunk + 1)) : total;
      if (total > (avail - a.payload) / 8 || first > next || next > total ||
          next - first > (unsigned long long)kWordsMax)
        bad = 1;
      words = next - first;
    }
    s_first = first;
    s_words = words;
    s_minexp = minexp;
    s_bad = bad;
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) atomicOr(a.status, ST_CORRUPT);
    return;
  }
  const long blk = chunk * ZC_CHUNK + tid;
  const bool valid = blk < a.nblocks;
  const int len = valid ? (int)*reinterpret_cast<const uint16_t*>(in + a.length_table + 2ull * blk) : 0;
  // CTA exclusive scan of block lengths
  const int lane = tid & 31, warp = tid >> 5;
  unsigned incl = (unsigned)len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  const unsigned long long W = s_words;
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(in + a.payload) + s_first;
  for (unsigned long long w = tid; w < W; w += ZC_CHUNK) sbuf[w] = __ldg(src + w);
  if (tid < 2) sbuf[W + tid] = 0ull;
  __syncthreads();
  unsigned warp_off = 0, total = 0;
#pragma unroll
  for (int w = 0; w < ZC_CHUNK / 32; ++w) {
    if (w < warp) warp_off += s_warp[w];
    total += s_warp[w];
  }
  if ((unsigned long long)total > 64ull * W) {
    if (tid == 0) atomicOr(a.status, ST_CORRUPT);
    return;
  }
  if (!valid) return;
  const long start = (long)(warp_off + incl - (unsigned)len);
  SReader rd{sbuf, start, start + len};
  uint32_t u[64];
  int emax = 0, planes = 0;
  if (!decode_planes(rd, s_minexp, u, emax, planes) || rd.pos != rd.end) {
    atomicOr(a.status, ST_CORRUPT);
    return;
  }
  float v[64];
  dequantise(u, emax, planes, v);
  const long bx = blk % a.nbx, by = (blk / a.nbx) % a.nby, bz = blk / (a.nbx * a.nby);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long z = 4 * bz + k;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long y = 4 * by + j;
      if (z < a.nz && y < a.ny) {
        float* row = a.out + a.pitch * (y + (long)a.ny * z);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const long x = 4 * bx + i;
          if (x < a.nx) row[x] = v[i + 4 * j + 16 * k];
        }
      }
    }
  }
}

}  // namespace

ZLayout zlayout(int nx, int ny, int nz) {
  ZLayout L{};
  L.nbx = (nx + 3) / 4;
  L.nby = (ny + 3) / 4;
  L.nbz = (nz + 3) / 4;
  L.nblocks = L.nbx * L.nby * L.nbz;
  L.nchunks = (L.nblocks + ZC_CHUNK - 1) / ZC_CHUNK;
  L.chunk_table = 64;
  L.length_table = L.chunk_table + 8 * (size_t)L.nchunks;
  L.payload = L.length_table + (size_t)((2 * L.nblocks + 7) / 8) * 8;
  size_t words = 0;
  for (long c = 0; c < L.nchunks; ++c) {
    long nb = L.nblocks - c * ZC_CHUNK;
    if (nb > ZC_CHUNK) nb = ZC_CHUNK;
    words += (size_t)((nb * ZC_MAXBITS + 63) / 64);
  }
  L.max_bytes = L.payload + 8 * words;
  return L;
}

size_t zfp_encode_scratch_words(int nx, int ny, int nz) {
  return (size_t)zlayout(nx, ny, nz).nchunks + 1;
}

static cudaError_t encode_common(const float* in, Grid g, int minexp, uint8_t* out,
                                 const unsigned long long* d_base, size_t capacity,
                                 unsigned long long* d_size, int* d_status,
                                 unsigned long long* scratch, cudaStream_t s) {
  ZLayout L = zlayout(g.nx, g.ny, g.nz);
  EncArgs a;
  a.in = in;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.pitch = g.pitch;
  a.nbx = L.nbx;
  a.nby = L.nby;
  a.nblocks = L.nblocks;
  a.nchunks = L.nchunks;
  a.minexp = minexp;
  a.out = out;
  a.base = d_base;
  a.limit = capacity;
  a.chunk_table = L.chunk_table;
  a.length_table = L.length_table;
  a.payload = L.payload;
  a.size_out = d_size;
  a.status = d_status;
  a.desc = scratch;
  a.ticket = reinterpret_cast<unsigned int*>(scratch + L.nchunks);
  const int ps = prof_begin(KC_ZFP_ENCODE, s);
  k_encode<<<(unsigned)L.nchunks, ZC_CHUNK, 0, s>>>(a);
  prof_end(ps, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t zfp_encode_launch(const float* in, Grid g, int minexp, uint8_t* out,
                              const unsigned long long* d_base, size_t capacity,
                              unsigned long long* d_size, int* d_status,
                              unsigned long long* scratch, cudaStream_t s) {
  size_t words = zfp_encode_scratch_words(g.nx, g.ny, g.nz);
  cudaError_t e = cudaMemsetAsync(scratch, 0, words * 8, s);
  if (e != cudaSuccess) return e;
  return encode_common(in, g, minexp, out, d_base, capacity, d_size, d_status, scratch, s);
}

cudaError_t zfp_decode_launch(const uint8_t* in, const unsigned long long* d_base, size_t avail,
                              float* out, Grid g, int* d_status, cudaStream_t s) {
  ZLayout L = zlayout(g.nx, g.ny, g.nz);
  DecArgs a;
  a.in = in;
  a.base = d_base;
  a.avail = avail;
  a.limit = avail;
  a.out = out;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.pitch = g.pitch;
  a.nbx = L.nbx;
  a.nby = L.nby;
  a.nblocks = L.nblocks;
  a.nchunks = L.nchunks;
  a.chunk_table = L.chunk_table;
  a.length_table = L.length_table;
  a.payload = L.payload;
  a.status = d_status;
  const int ps = prof_begin(KC_ZFP_DECODE, s);
  k_decode<<<(unsigned)L.nchunks, ZC_CHUNK, 0, s>>>(a);
  prof_end(ps, s);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fwi
