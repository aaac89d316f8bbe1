// Fixed-accuracy block codec for FP32 wavefields on sm_103a (Sec. 1.4 of
// Kukreja et al.: every checkpoint is compressed with an absolute error
// tolerance atol; the format is this project's ZFP-style design).
//
// Per 4x4x4 block: block exponent -> 25-bit block-floating-point integers ->
// integer lifting transform along x, y, z -> sequency order -> negabinary ->
// embedded bit planes (planes = emax - minexp + 11, raised to 32 when fewer
// than 3 planes would be dropped).
//
// GPU organisation: one thread per block, one warp per chunk of 32
// consecutive blocks (4 independent warps per CTA, never synchronised with
// each other).  The 64 coefficients of a block live in registers; two 32x32
// bit-matrix transposes turn them into 64-bit plane masks, from which the
// exact bit count of every plane is computed with popc/clz, and a warp scan
// of the counts places each block's bits in its chunk.  Chunk offsets: the
// staged encoder (k_encode_stage / _compact / _place, used by the sweeps and
// zfp_compress_fixed_accuracy) codes every chunk into a fixed staging slot,
// scans the word counts and copies the words into place; the single-pass
// encoder of the allocation-free entry point (k_encode_chained) finds them by
// a warp-parallel decoupled look-back across chunks (chunk order is the
// warp's ticket order, so every predecessor is already resident).  Either way
// a chunk's bits are assembled in the warp's shared-memory buffer and written
// with coalesced 64-bit stores.  Decoding reverses this with one warp
// per chunk: the chunk's words are staged in shared memory, block offsets come
// from a warp scan of the u16 length table, and each thread rebuilds its plane
// masks (ctz finds every newly significant coefficient).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "codec_block.cuh"
#include "common.cuh"

namespace fwi {
namespace {

using namespace zblock;

constexpr int kWordsMax = (ZC_CHUNK * ZC_MAXBITS + 63) / 64;  // 1061 words
constexpr int kWarps = 4;                                       // chunks per CTA
#ifndef FWI_ENC_MIN_CTAS
#define FWI_ENC_MIN_CTAS 6  // resident CTAs per SM the staged encoder is compiled for
#endif
#ifndef FWI_DEC_MIN_CTAS
#define FWI_DEC_MIN_CTAS 6  // the same for the decoder
#endif
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr long kSpinLimit = 1L << 24;

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Shared-memory bit writer over a zeroed buffer.  Neighbouring threads share
// at most a boundary word: a thread's first word (which may hold the previous
// thread's last bits) and its last, partial word are merged with atomicOr;
// the words in between are the thread's alone and are stored.
struct SWriter {
  unsigned long long* buf;
  unsigned long long acc;
  int fill;
  int word;
  int first;  // the thread's first word
  __device__ __forceinline__ void put(unsigned long long v, int k) {  // 1 <= k <= 64
    acc |= v << fill;
    int nf = fill + k;
    if (nf >= 64) {
      if (word == first)
        atomicOr(&buf[word], acc);
      else
        buf[word] = acc;
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

// Coordinates of block blk (x fastest) in a grid of nbx x nby x . blocks.
// 32-bit division whenever the block count allows it: 64-bit integer division
// is a long software sequence on the GPU.
__device__ __forceinline__ void block_xyz(long blk, long nbx, long nby, long nblocks, long& bx, long& by,
                                          long& bz) {
  if (nblocks <= 0xffffffffL) {
    const unsigned b = (unsigned)blk, nx = (unsigned)nbx, ny = (unsigned)nby;
    const unsigned q = b / nx;
    bx = b - q * nx;
    by = q % ny;
    bz = q / ny;
  } else {
    const long q = blk / nbx;
    bx = blk - q * nbx;
    by = q % nby;
    bz = q / nby;
  }
}

struct EncArgs {
  const float* in;
  bool vec_ok;  // rows 16-byte aligned (pitch % 4 == 0 and aligned base)
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
  const uint16_t* live;  // liveness map of the field (NULL = read every block)
  int live_ntx;
};

__device__ __forceinline__ void put_u32(uint8_t* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }
__device__ __forceinline__ void put_u64(uint8_t* p, unsigned long long v) {
  *reinterpret_cast<unsigned long long*>(p) = v;
}

__global__ void __launch_bounds__(ZC_CHUNK * kWarps, 4) k_encode_chained(EncArgs a) {
  __shared__ unsigned long long sbuf_all[kWarps][kWordsMax + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long* sbuf = sbuf_all[wid];
  long chunk = 0;
  if (lane == 0) chunk = (long)atomicAdd(a.ticket, 1u);
  chunk = __shfl_sync(0xffffffffu, chunk, 0);
  if (chunk >= a.nchunks) return;  // whole warp (grid is rounded up to whole CTAs)
  const long blk = chunk * ZC_CHUNK + lane;
  const bool valid = blk < a.nblocks;
  const unsigned long long base = a.base ? *a.base : 0ull;
  const unsigned long long avail = a.limit > base ? a.limit - base : 0ull;
  uint8_t* out = a.out + base;

  // ---- gather the block (edge blocks replicate the last plane) ------------
  uint32_t u[64];
  int planes = 0, emax = 0, nbits = 0;
  if (valid) {
    long bx, by, bz;
    block_xyz(blk, a.nbx, a.nby, a.nblocks, bx, by, bz);
    const long xb = 4 * bx;
    // 16-byte row loads when the 4 x values are in range and aligned
    const bool vec = a.vec_ok && xb + 3 < a.nx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long z = min(4 * bz + k, (long)a.nz - 1);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long y = min(4 * by + j, (long)a.ny - 1);
        const float* row = a.in + a.pitch * (y + (long)a.ny * z);
        const int o = 4 * j + 16 * k;
        if (vec) {
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + xb));
          u[o] = v.x;
          u[o + 1] = v.y;
          u[o + 2] = v.z;
          u[o + 3] = v.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) u[o + i] = __float_as_uint(__ldg(row + min(xb + i, (long)a.nx - 1)));
        }
      }
    }
    if (!quantise(u, a.minexp, emax, planes)) atomicOr(a.status, ST_NONFINITE);
    nbits = count_bits(u, planes);
  }

  // ---- warp exclusive scan of bit counts -------------------------------------
  unsigned incl = (unsigned)nbits;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
  const unsigned my_off = incl - (unsigned)nbits;
  const unsigned W = (total + 63u) / 64u;

  // ---- decoupled look-back over chunks (32 predecessors per step) ------------
  // The chunk's word count is published first and its inclusive prefix as
  // soon as it is known, so the prefix frontier keeps pace with the warps in
  // flight.  A descriptor packs flag (aggregate / inclusive prefix) and value
  // in one 64-bit word, so relaxed loads and stores suffice.
  if (lane == 0) st_relaxed(&a.desc[chunk], (chunk == 0 ? kFlagPre : kFlagAgg) | W);
  unsigned long long prefix = 0;
  if (chunk > 0) {
    long top = chunk - 1;
    while (true) {
      const long idx = top - lane;
      unsigned long long d = kFlagPre;  // before chunk 0: an inclusive prefix of 0
      if (idx >= 0) {
        long spins = 0;
        while (((d = ld_relaxed(&a.desc[idx])) >> 62) == 0ull) {
          if (++spins > kSpinLimit) {
            atomicOr(a.status, ST_TIMEOUT);
            d = kFlagPre;
            break;
          }
          __nanosleep(32);
        }
      }
      const unsigned pre = __ballot_sync(0xffffffffu, (d >> 62) == 2ull);
      const int stop = pre ? __ffs(pre) - 1 : 31;  // nearest inclusive prefix
      unsigned long long v = lane <= stop ? (d & kValMask) : 0ull;
#pragma unroll
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      prefix += v;
      if (pre) break;
      top -= 32;
    }
    if (lane == 0) st_relaxed(&a.desc[chunk], kFlagPre | (prefix + W));
  }

  // ---- assemble the chunk's bits in the warp's shared-memory buffer ----------
  for (unsigned w = lane; w < W; w += 32) sbuf[w] = 0ull;
  __syncwarp();
  if (valid) {
    SWriter wr{sbuf, 0ull, (int)(my_off & 63u), (int)(my_off >> 6), (int)(my_off >> 6)};
    emit(wr, u, emax, planes);
    wr.flush();
  }
  __syncwarp();

  // ---- write payload, tables and (last chunk) the header -------------------
  const unsigned long long pay = a.payload + 8ull * prefix;
  for (unsigned w = lane; w < W; w += 32) {
    const unsigned long long off = pay + 8ull * w;
    if (off + 8 <= avail) put_u64(out + off, sbuf[w]);
  }
  if (valid) {
    const unsigned long long off = a.length_table + 2ull * blk;
    if (off + 2 <= avail) *reinterpret_cast<uint16_t*>(out + off) = (uint16_t)nbits;
  }
  if (lane == 0) {
    const unsigned long long off = a.chunk_table + 8ull * chunk;
    if (off + 8 <= avail) put_u64(out + off, prefix);
  }
  if (chunk == a.nchunks - 1) {
    // zero padding of the length table after the last block
    const unsigned long long lt_end = a.length_table + 2ull * a.nblocks;
    for (unsigned long long off = lt_end + 2ull * lane; off < a.payload; off += 64ull)
      if (off + 2 <= avail) *reinterpret_cast<uint16_t*>(out + off) = 0;
    if (lane == 0) {
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

// ---- staged encoder (no inter-chunk dependency) --------------------------------
// Pass 1: every warp codes its chunk into its own fixed staging slot
// (kWordsMax words) and records the word count; pass 2: one CTA per tile of
// kTile chunks adds the counts of all earlier tiles and of its own earlier
// chunks, then copies the words into place (2x the compressed bytes of extra
// traffic, no waiting between chunks).
constexpr int kTile = 1024;  // chunks per compaction CTA

struct StageArgs {
  unsigned long long* stage;     // nchunks x kWordsMax words
  unsigned* words;               // per-chunk word count
  unsigned long long* tile_sum;  // per-tile word totals (zeroed before pass 1)
  unsigned long long* offset;    // per-chunk word offset in the payload
};

__device__ __forceinline__ void gather_block(const EncArgs& a, long bx, long by, long bz, uint32_t* u) {
  const long xb = 4 * bx;
  const bool vec = a.vec_ok && xb + 3 < a.nx;  // 16-byte row loads when aligned and in range
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long z = min(4 * bz + k, (long)a.nz - 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long y = min(4 * by + j, (long)a.ny - 1);
      const float* row = a.in + a.pitch * (y + (long)a.ny * z);
      const int o = 4 * j + 16 * k;
      if (vec) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + xb));
        u[o] = v.x;
        u[o + 1] = v.y;
        u[o + 2] = v.z;
        u[o + 3] = v.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) u[o + i] = __float_as_uint(__ldg(row + min(xb + i, (long)a.nx - 1)));
      }
    }
  }
}

// Shared memory of the staged encoder, per warp: the low and high halves of
// the 32 plane masks of each lane's block ([plane][lane] u32 arrays,
// conflict-free), and a buffer in which the chunk's words are assembled when
// they fit (always for real wavefields; a larger chunk is assembled directly
// in its global staging slot instead).
constexpr int kAsmWords = 128;  // 9 KB of shared memory per warp: six encoder CTAs fit an SM
constexpr int kEncSmemPerWarp = 2 * 32 * 32 * 4 + (kAsmWords + 1) * 8;
constexpr int kEncSmem = kWarps * kEncSmemPerWarp;

struct SmemPlanes {  // plane b of one lane's block
  const uint32_t* lo;
  const uint32_t* hi;
  __device__ __forceinline__ uint64_t operator()(int b) const {
    return (uint64_t)lo[b * 32] | ((uint64_t)hi[b * 32] << 32);
  }
};

__global__ void __launch_bounds__(ZC_CHUNK * kWarps, FWI_ENC_MIN_CTAS) k_encode_stage(EncArgs a, StageArgs st) {
  extern __shared__ unsigned long long enc_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* base = reinterpret_cast<unsigned char*>(enc_smem) + (size_t)wid * kEncSmemPerWarp;
  uint32_t* lo = reinterpret_cast<uint32_t*>(base);  // [32][32]
  uint32_t* hi = lo + 32 * 32;
  unsigned long long* sbuf = reinterpret_cast<unsigned long long*>(hi + 32 * 32);
  const long chunk = (long)blockIdx.x * kWarps + wid;
  if (chunk >= a.nchunks) return;  // whole warp
  const long blk = chunk * ZC_CHUNK + lane;
  const bool valid = blk < a.nblocks;
  int planes = 0, emax = 0, nbits = 0;
  long bx = 0, by = 0, bz = 0;
  if (valid) block_xyz(blk, a.nbx, a.nby, a.nblocks, bx, by, bz);
  // a block the forward step found below the threshold of this tolerance
  // codes as zero (no coded plane): it is not read
  const bool read = valid && (!a.live || ((a.live[(bz * a.nby + by) * a.live_ntx + (bx >> 4)] >> (bx & 15)) & 1));
  if (read) {
    uint32_t u[64];
    gather_block(a, bx, by, bz, u);
    if (!quantise_coeffs(u, a.minexp, emax, planes)) atomicOr(a.status, ST_NONFINITE);
    if (planes) {  // a block with no coded plane is the single bit 0: nothing to transpose
      transpose32(u);
#pragma unroll
      for (int b = 0; b < 32; ++b)
        if (b >= 32 - planes) lo[b * 32 + lane] = u[b];
      transpose32(u + 32);
#pragma unroll
      for (int b = 0; b < 32; ++b)
        if (b >= 32 - planes) hi[b * 32 + lane] = u[32 + b];
    }
  }
  const SmemPlanes mine{lo + lane, hi + lane};
  if (valid) nbits = count_bits_mem(mine, planes);
  unsigned incl = (unsigned)nbits;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
  const unsigned my_off = incl - (unsigned)nbits;
  const unsigned W = (total + 63u) / 64u;
  unsigned long long* dst = st.stage + chunk * (long)kWordsMax;
  unsigned long long* buf = W <= (unsigned)kAsmWords ? sbuf : dst;  // warp-uniform
  for (unsigned w = lane; w < W; w += 32) buf[w] = 0ull;
  __syncwarp();
  if (valid) {
    SWriter wr{buf, 0ull, (int)(my_off & 63u), (int)(my_off >> 6), (int)(my_off >> 6)};
    emit_mem(wr, mine, emax, planes);
    wr.flush();
  }
  __syncwarp();
  if (buf == sbuf)
    for (unsigned w = lane; w < W; w += 32) dst[w] = sbuf[w];
  if (valid) {
    const unsigned long long base = a.base ? *a.base : 0ull;
    const unsigned long long avail = a.limit > base ? a.limit - base : 0ull;
    const unsigned long long off = a.length_table + 2ull * blk;
    if (off + 2 <= avail) *reinterpret_cast<uint16_t*>(a.out + base + off) = (uint16_t)nbits;
  }
  if (lane == 0) {
    st.words[chunk] = W;
    atomicAdd(&st.tile_sum[chunk / kTile], (unsigned long long)W);
  }
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  unsigned long long t = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// Chunk offsets: one CTA (256 threads, 4 chunks per thread) per tile of kTile
// chunks adds the totals of the earlier tiles to a scan of its own chunks.
__global__ void __launch_bounds__(256) k_encode_compact(EncArgs a, StageArgs st) {
  __shared__ unsigned long long red[8];
  __shared__ unsigned long long wsum[8];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long tile = blockIdx.x;
  const long c0 = tile * kTile;
  const unsigned long long base = a.base ? *a.base : 0ull;
  const unsigned long long avail = a.limit > base ? a.limit - base : 0ull;
  uint8_t* out = a.out + base;
  // words of all earlier tiles
  unsigned long long pre = 0;
  for (long t = tid; t < tile; t += blockDim.x) pre += st.tile_sum[t];
  pre = block_sum_u64(pre, red);
  // exclusive scan of this tile's chunk word counts (4 consecutive per thread)
  unsigned cw[4];
  unsigned mine = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long c = c0 + 4 * tid + i;
    cw[i] = c < a.nchunks ? st.words[c] : 0u;
    mine += cw[i];
  }
  unsigned long long incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  unsigned long long woff = 0, tile_total = 0;
  for (int i = 0; i < 8; ++i) {
    if (i < w) woff += wsum[i];
    tile_total += wsum[i];
  }
  unsigned long long off = pre + woff + incl - mine;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long c = c0 + 4 * tid + i;
    if (c < a.nchunks) {
      st.offset[c] = off;
      const unsigned long long t = a.chunk_table + 8ull * c;
      if (t + 8 <= avail) put_u64(out + t, off);
    }
    off += cw[i];
  }
  if (tile == (a.nchunks - 1) / kTile) {
    // zero padding of the length table after the last block, header, size
    const unsigned long long lt_end = a.length_table + 2ull * a.nblocks;
    for (unsigned long long o = lt_end + 2ull * tid; o < a.payload; o += 2ull * blockDim.x)
      if (o + 2 <= avail) *reinterpret_cast<uint16_t*>(out + o) = 0;
    if (tid == 0) {
      const unsigned long long words = pre + tile_total;
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

// Placement: one warp per chunk moves its staged words to their offset.
__global__ void __launch_bounds__(256) k_encode_place(EncArgs a, StageArgs st) {
  const int lane = threadIdx.x & 31;
  const long chunk = (long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (chunk >= a.nchunks) return;
  const unsigned long long base = a.base ? *a.base : 0ull;
  const unsigned long long avail = a.limit > base ? a.limit - base : 0ull;
  uint8_t* out = a.out + base;
  const unsigned n = st.words[chunk];
  const unsigned long long pay = a.payload + 8ull * st.offset[chunk];
  const unsigned long long* from = st.stage + chunk * (long)kWordsMax;
  for (unsigned k = lane; k < n; k += 32) {
    const unsigned long long dst = pay + 8ull * k;
    if (dst + 8 <= avail) put_u64(out + dst, from[k]);
  }
}

// ---- decoder ------------------------------------------------------------------

struct DecArgs {
  const uint8_t* in;
  bool vec_ok;
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

// Bit reader over a chunk's words (staged in shared memory, or in global
// memory for a chunk larger than the staging buffer); words at index >= nw
// read as zero, so a peek at the end never leaves the chunk.  Positions are
// bits from the chunk's first word (at most 64 kWordsMax, checked by the
// caller), so 32-bit arithmetic holds them.
struct SReader {
  const unsigned long long* buf;
  int pos;
  int end;
  int nw;
  __device__ __forceinline__ unsigned long long peek() const {
    const int w = pos >> 6;
    const int o = (int)(pos & 63);
    unsigned long long v = w < nw ? buf[w] : 0ull;
    v >>= o;
    if (o && w + 1 < nw) v |= buf[w + 1] << (64 - o);
    return v;
  }
};

__device__ __forceinline__ uint32_t get_u32(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ unsigned long long get_u64(const uint8_t* p) {
  return *reinterpret_cast<const unsigned long long*>(p);
}

// Shared memory of the decoder, per warp: the plane masks of each lane's
// block ([plane][lane] low / high halves) and the chunk's words when they fit.
// The decoder stages up to dec_words() words of a chunk (larger chunks are
// read from global memory by the bounded reader): 9 KB of shared memory per
// warp, so that six decoder CTAs fit an SM.
constexpr int dec_words(bool) { return 128; }
constexpr int dec_smem_per_warp(bool image) { return 2 * 32 * 32 * 4 + (dec_words(image) + 2) * 8; }
constexpr int dec_smem(bool image) { return kWarps * dec_smem_per_warp(image); }

struct SmemSink {  // plane b of one lane's block
  uint32_t* lo;
  uint32_t* hi;
  __device__ __forceinline__ void operator()(int b, uint64_t m) const {
    lo[b * 32] = (uint32_t)m;
    hi[b * 32] = (uint32_t)(m >> 32);
  }
};

// Tail of the decoder (one lane per block).  Every lane of the warp reaches
// the warp barrier; then each lane's decoded block moves to the warp's shared
// memory (the plane masks and staged words are dead by then), freeing its 64
// registers, so the decoder fits six CTAs per SM and several rows' loads and
// stores can be in flight at once.  IMAGE: image the block (ImageArgs) and
// write it only where im.rec_block flags it, skipping blocks coded as zero;
// else write it.
constexpr int kVStride = 68;  // floats per lane: 16-byte rows, conflict-free per quarter warp
static_assert(32 * kVStride * 4 <= dec_smem_per_warp(true) && 32 * kVStride * 4 <= dec_smem_per_warp(false),
              "decoded blocks fit the warp's area");

template <bool IMAGE>
__device__ __forceinline__ void finish_blocks(const DecArgs& a, const ImageArgs& im, long blk, bool valid,
                                              int minexp, uint32_t* lo, uint32_t* hi,
                                              const unsigned long long* words_src, long start, int len,
                                              long nwords, float* warp_area) {
  const int lane = threadIdx.x & 31;
  bool work = valid;
  int emax = 0, planes = 0;
  if (work) {
    SReader rd{words_src, (int)start, (int)(start + len), (int)nwords};
    SmemSink sink{lo + lane, hi + lane};
    if (!decode_planes_mem(rd, minexp, sink, emax, planes) || rd.pos != rd.end) {
      atomicOr(a.status, ST_CORRUPT);
      work = false;
    } else if (planes == 0 && IMAGE) {
      work = false;  // a zero block images nothing
    }
  }
  const bool coded = work && planes > 0;  // otherwise a zero block to be written (plain decoder)
  float v[64];
  if (coded) {
    uint32_t u[64];
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      const bool in = b >= 32 - planes;
      u[b] = in ? lo[b * 32 + lane] : 0u;
      u[32 + b] = in ? hi[b * 32 + lane] : 0u;
    }
    dequantise(u, emax, planes, v);
  }
  __syncwarp();  // every lane is done with the warp's plane masks and words
  float* vs = warp_area + lane * kVStride;
  if (coded) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      *reinterpret_cast<float4*>(vs + 4 * i) = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else if (work) {
#pragma unroll
    for (int i = 0; i < 16; ++i) *reinterpret_cast<float4*>(vs + 4 * i) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  asm volatile("" ::: "memory");  // the rows below read the block back from shared memory
  if (!work) return;
  long bx, by, bz;
  block_xyz(blk, a.nbx, a.nby, a.nblocks, bx, by, bz);
  const long xb = 4 * bx;
  const bool vec = a.vec_ok && xb + 3 < a.nx;
  const bool store = !IMAGE || im.rec_block[blk] != 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long z = 4 * bz + k;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long y = 4 * by + j;
      if (z < a.nz && y < a.ny) {
        const long c = a.pitch * (y + (long)a.ny * z) + xb;
        const float4 u4 = *reinterpret_cast<const float4*>(vs + 4 * j + 16 * k);
        const float uv[4] = {u4.x, u4.y, u4.z, u4.w};
        if (vec) {
          if (IMAGE) {
            const float4 lp = __ldg(reinterpret_cast<const float4*>(im.lp + c));
            const float4 lc = __ldg(reinterpret_cast<const float4*>(im.lc + c));
            const float4 ln = __ldg(reinterpret_cast<const float4*>(im.ln + c));
            float4 g = *reinterpret_cast<const float4*>(im.g + c);
            g.x = image_update(g.x, uv[0], lp.x, lc.x, ln.x, im.idt2);
            g.y = image_update(g.y, uv[1], lp.y, lc.y, ln.y, im.idt2);
            g.z = image_update(g.z, uv[2], lp.z, lc.z, ln.z, im.idt2);
            g.w = image_update(g.w, uv[3], lp.w, lc.w, ln.w, im.idt2);
            *reinterpret_cast<float4*>(im.g + c) = g;
          }
          if (store) *reinterpret_cast<float4*>(a.out + c) = u4;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (xb + i < a.nx) {
              if (IMAGE)
                im.g[c + i] = image_update(im.g[c + i], uv[i], __ldg(im.lp + c + i), __ldg(im.lc + c + i),
                                           __ldg(im.ln + c + i), im.idt2);
              if (store) a.out[c + i] = uv[i];
            }
        }
      }
    }
  }
}

// IMAGE: instead of writing the decoded block, image it (finish_blocks).
template <bool IMAGE>
__global__ void __launch_bounds__(ZC_CHUNK * kWarps, FWI_DEC_MIN_CTAS) k_decode(DecArgs a, ImageArgs im) {
  extern __shared__ unsigned long long dec_smem_buf[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* wbase = reinterpret_cast<unsigned char*>(dec_smem_buf) + (size_t)wid * dec_smem_per_warp(IMAGE);
  uint32_t* lo = reinterpret_cast<uint32_t*>(wbase);  // [32][32]
  uint32_t* hi = lo + 32 * 32;
  unsigned long long* sbuf = reinterpret_cast<unsigned long long*>(hi + 32 * 32);
  const long chunk = (long)blockIdx.x * kWarps + wid;
  if (chunk >= a.nchunks) return;  // whole warp
  const unsigned long long base = a.base ? *a.base : 0ull;
  const unsigned long long avail = a.base ? (a.limit > base ? a.limit - base : 0ull) : a.avail;
  const uint8_t* in = a.in + base;
  if (a.payload > avail) {  // the tables do not fit (warp-uniform)
    if (lane == 0) atomicOr(a.status, ST_CORRUPT);
    return;
  }
  // One round trip: lanes 0-7 load the eight header words, lanes 8-9 this
  // chunk's and the next chunk's payload offsets, every lane its block's
  // coded length (all inside the tables).
  const long blk = chunk * ZC_CHUNK + lane;
  const bool valid = blk < a.nblocks;
  unsigned long long hw = 0;
  if (lane < 8)
    hw = get_u64(in + 8 * lane);
  else if (lane == 8 || (lane == 9 && chunk + 1 < a.nchunks))
    hw = get_u64(in + a.chunk_table + 8ull * (chunk + lane - 8));
  const int len = valid ? (int)*reinterpret_cast<const uint16_t*>(in + a.length_table + 2ull * blk) : 0;
  const unsigned long long h0 = __shfl_sync(0xffffffffu, hw, 0), h1 = __shfl_sync(0xffffffffu, hw, 1);
  const unsigned long long h2 = __shfl_sync(0xffffffffu, hw, 2), h3 = __shfl_sync(0xffffffffu, hw, 3);
  const unsigned long long h4 = __shfl_sync(0xffffffffu, hw, 4), h5 = __shfl_sync(0xffffffffu, hw, 5);
  const unsigned long long h7 = __shfl_sync(0xffffffffu, hw, 7);
  const unsigned long long first = __shfl_sync(0xffffffffu, hw, 8);
  unsigned long long next = __shfl_sync(0xffffffffu, hw, 9);
  const unsigned long long pay_words = h5;  // payload words (bytes 40..47)
  if (chunk + 1 >= a.nchunks) next = pay_words;
  const bool bad = (uint32_t)h0 != ZC_MAGIC || (uint32_t)(h0 >> 32) != ZC_VERSION ||
                   (int)(uint32_t)h1 != a.nx || (int)(uint32_t)(h1 >> 32) != a.ny ||
                   (int)(uint32_t)h2 != a.nz || h3 != (unsigned long long)a.nblocks ||
                   (uint32_t)h4 != (uint32_t)ZC_CHUNK || (uint32_t)(h4 >> 32) != (uint32_t)a.nchunks ||
                   (uint32_t)h7 != (uint32_t)(ZC_S | (ZC_G << 8)) || pay_words > (avail - a.payload) / 8 ||
                   first > next || next > pay_words || next - first > (unsigned long long)kWordsMax;
  if (bad) {  // warp-uniform
    if (lane == 0) atomicOr(a.status, ST_CORRUPT);
    return;
  }
  const int minexp = (int)(uint32_t)(h2 >> 32);  // bytes 20..23
  const unsigned long long words = next - first;
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(in + a.payload) + first;
  // A chunk of blocks that are all the single bit 0 (one payload word, zero)
  // has nothing to image.
  if (IMAGE && words == 1 && __all_sync(0xffffffffu, !valid || len == 1)) {
    unsigned long long w0 = 0;
    if (lane == 0) w0 = __ldg(src);
    if (__shfl_sync(0xffffffffu, w0, 0) == 0ull) return;  // else the blocks below report the corruption
  }
  // stage the chunk's words (when they fit) and scan the block lengths
  const bool staged = words <= (unsigned long long)dec_words(IMAGE);  // warp-uniform
  if (staged) {
    for (unsigned long long w = lane; w < words; w += 32) sbuf[w] = __ldg(src + w);
  }
  unsigned incl = (unsigned)len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  if ((unsigned long long)total > 64ull * words) {
    if (lane == 0) atomicOr(a.status, ST_CORRUPT);
    return;
  }
  finish_blocks<IMAGE>(a, im, blk, valid, minexp, lo, hi, staged ? sbuf : src, (long)(incl - (unsigned)len), len,
                       (long)words, reinterpret_cast<float*>(wbase));
}

// Blocks coded as zero (length one bit) per slot: grid (ctas per slot, slots).
__global__ void __launch_bounds__(256) k_count_zero_blocks(const uint8_t* arena, const unsigned long long* offs,
                                                           unsigned long long capacity,
                                                           unsigned long long length_table,
                                                           unsigned long long payload, long nblocks,
                                                           unsigned long long* counts) {
  const int slot = blockIdx.y;
  const unsigned long long base = offs[slot];
  if (base > capacity || payload > capacity - base) {
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[slot] = ~0ull;
    return;
  }
  const uint16_t* len = reinterpret_cast<const uint16_t*>(arena + base + length_table);
  unsigned long long n = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nblocks; i += (long)gridDim.x * blockDim.x)
    n += len[i] == 1;
#pragma unroll
  for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&counts[slot], n);
}

}  // namespace

cudaError_t zfp_count_zero_blocks_launch(const uint8_t* arena, const unsigned long long* offs, int nslots,
                                         size_t capacity, Grid g, unsigned long long* counts, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const ZLayout L = zlayout(g.nx, g.ny, g.nz);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)nslots, s);
  if (e != cudaSuccess) return e;
  const long per = std::min<long>(64, (L.nblocks + 255) / 256);
  for (int j0 = 0; j0 < nslots; j0 += 65535) {
    const int n = std::min(65535, nslots - j0);
    k_count_zero_blocks<<<dim3((unsigned)per, (unsigned)n), 256, 0, s>>>(
        arena, offs + j0, capacity, L.length_table, L.payload, L.nblocks, counts + j0);
    count_launch();
  }
  return cudaGetLastError();
}

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


// The codec kernels' dynamic shared-memory limit: a kernel attribute takes
// effect in the context of the device current when it is set, so it is set
// once per device, on that device's first launch.
constexpr int kMaxDevices = 64;
static std::mutex g_attr_mu;
static bool g_attr_done[kMaxDevices];

static cudaError_t ensure_codec_attributes() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(k_encode_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, kEncSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_decode<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dec_smem(false));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_decode<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dec_smem(true));
  if (e != cudaSuccess) return e;
  g_attr_done[dev] = true;
  return cudaSuccess;
}

static EncArgs encode_args(const float* in, Grid g, int minexp, uint8_t* out,
                           const unsigned long long* d_base, size_t capacity,
                           unsigned long long* d_size, int* d_status) {
  ZLayout L = zlayout(g.nx, g.ny, g.nz);
  EncArgs a;
  a.in = in;
  a.vec_ok = (g.pitch % 4 == 0) && (((uintptr_t)in & 15) == 0);
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
  a.desc = nullptr;
  a.ticket = nullptr;
  a.live = nullptr;
  a.live_ntx = 0;
  return a;
}

size_t zfp_encode_scratch_bytes(int nx, int ny, int nz) {
  ZLayout L = zlayout(nx, ny, nz);
  const size_t ntiles = (size_t)((L.nchunks + kTile - 1) / kTile);
  return (size_t)L.nchunks * kWordsMax * 8 + (size_t)L.nchunks * 12 + ntiles * 8 + 256;
}

cudaError_t zfp_encode_launch(const float* in, Grid g, int minexp, uint8_t* out,
                              const unsigned long long* d_base, size_t capacity,
                              unsigned long long* d_size, int* d_status, void* scratch,
                              cudaStream_t s, const LiveMap* live) {
  if (!scratch) return cudaErrorInvalidValue;
  EncArgs a = encode_args(in, g, minexp, out, d_base, capacity, d_size, d_status);
  if (live && live->words) {
    // the map must have been written at exactly this tolerance's threshold
    if (live->threshold != live_threshold(minexp) || !(live->threshold > 0.0f) ||
        live->ntx != (g.pitch + 63) / 64 || live->nby != (int)a.nby)
      return cudaErrorInvalidValue;
    a.live = live->words;
    a.live_ntx = live->ntx;
  }
  const long ntiles = (a.nchunks + kTile - 1) / kTile;
  StageArgs st;
  st.stage = static_cast<unsigned long long*>(scratch);
  st.tile_sum = st.stage + (size_t)a.nchunks * kWordsMax;
  st.offset = st.tile_sum + ntiles;
  st.words = reinterpret_cast<unsigned*>(st.offset + a.nchunks);
  cudaError_t e = cudaMemsetAsync(st.tile_sum, 0, ntiles * 8, s);
  if (e != cudaSuccess) return e;
  if ((e = ensure_codec_attributes()) != cudaSuccess) return e;
  const int ps = prof_begin(KC_ZFP_ENCODE, s);
  k_encode_stage<<<(unsigned)((a.nchunks + kWarps - 1) / kWarps), ZC_CHUNK * kWarps, kEncSmem, s>>>(a, st);
  k_encode_compact<<<(unsigned)ntiles, 256, 0, s>>>(a, st);
  k_encode_place<<<(unsigned)((a.nchunks + 7) / 8), 256, 0, s>>>(a, st);
  prof_end(ps, s);
  count_launch();
  count_launch();
  count_launch();
  return cudaGetLastError();
}

size_t zfp_encode_chained_scratch_words(int nx, int ny, int nz) {
  return (size_t)zlayout(nx, ny, nz).nchunks + 1;
}

cudaError_t zfp_encode_chained_launch(const float* in, Grid g, int minexp, uint8_t* out,
                                      const unsigned long long* d_base, size_t capacity,
                                      unsigned long long* d_size, int* d_status,
                                      unsigned long long* scratch, cudaStream_t s) {
  if (!scratch) return cudaErrorInvalidValue;
  EncArgs a = encode_args(in, g, minexp, out, d_base, capacity, d_size, d_status);
  cudaError_t e = cudaMemsetAsync(scratch, 0, (size_t)(a.nchunks + 1) * 8, s);
  if (e != cudaSuccess) return e;
  a.desc = scratch;
  a.ticket = reinterpret_cast<unsigned int*>(scratch + a.nchunks);
  const int ps = prof_begin(KC_ZFP_ENCODE, s);
  k_encode_chained<<<(unsigned)((a.nchunks + kWarps - 1) / kWarps), ZC_CHUNK * kWarps, 0, s>>>(a);
  prof_end(ps, s);
  count_launch();
  return cudaGetLastError();
}

ZeroBlocks zero_blocks(const uint8_t* arena, const unsigned long long* base, size_t capacity, Grid g) {
  const ZLayout L = zlayout(g.nx, g.ny, g.nz);
  ZeroBlocks z;
  z.arena = arena;
  z.base = base;
  z.length_table = L.length_table;
  z.payload = L.payload;
  z.capacity = capacity;
  z.nbx = (int)L.nbx;
  z.nby = (int)L.nby;
  return z;
}

static DecArgs decode_args(const uint8_t* in, const unsigned long long* d_base, size_t avail, float* out, Grid g,
                           int* d_status) {
  ZLayout L = zlayout(g.nx, g.ny, g.nz);
  DecArgs a;
  a.in = in;
  a.vec_ok = (g.pitch % 4 == 0) && (((uintptr_t)out & 15) == 0);
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
  return a;
}

cudaError_t zfp_decode_launch(const uint8_t* in, const unsigned long long* d_base, size_t avail,
                              float* out, Grid g, int* d_status, cudaStream_t s) {
  const DecArgs a = decode_args(in, d_base, avail, out, g, d_status);
  const cudaError_t e = ensure_codec_attributes();
  if (e != cudaSuccess) return e;
  const int ps = prof_begin(KC_ZFP_DECODE, s);
  k_decode<false><<<(unsigned)((a.nchunks + kWarps - 1) / kWarps), ZC_CHUNK * kWarps, dec_smem(false), s>>>(
      a, ImageArgs{});
  prof_end(ps, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t zfp_decode_image_launch(const uint8_t* in, const unsigned long long* d_base, size_t avail,
                                    float* uk_out, Grid g, int* d_status, const ImageArgs& im, cudaStream_t s) {
  if (!im.lp || !im.lc || !im.ln || !im.g || !im.rec_block) return cudaErrorInvalidValue;
  const DecArgs a = decode_args(in, d_base, avail, uk_out, g, d_status);
  if (a.vec_ok && ((((uintptr_t)im.lp | (uintptr_t)im.lc | (uintptr_t)im.ln | (uintptr_t)im.g) & 15) != 0))
    return cudaErrorInvalidValue;
  const cudaError_t e = ensure_codec_attributes();
  if (e != cudaSuccess) return e;
  const int ps = prof_begin(KC_ZFP_DECODE, s);
  k_decode<true><<<(unsigned)((a.nchunks + kWarps - 1) / kWarps), ZC_CHUNK * kWarps, dec_smem(true), s>>>(a, im);
  prof_end(ps, s);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fwi
