// Allocation-free variant of zfp_compress_fixed_accuracy.
//
// Why it exists: the regular entry point takes its scratch (a staging slot
// per chunk, about the size of the field, plus size and status words) from
// the device's stream-ordered memory pool on every call.  Some callers cannot allocate device memory mid-run -- for example a
// solver that has already handed nearly all free HBM to its checkpoint arena,
// or an application whose memory policy forbids allocations after start-up.
// This variant runs the single-pass encoder (chunks find their offsets by a
// decoupled look-back, so its scratch is one descriptor per chunk) with that
// scratch in a fixed block inside the library's own device image, so it
// calls no cudaMalloc, cudaMallocAsync, cudaFree or allocating library
// routine.
//
// Limits and behaviour:
//   - The scratch holds kMaxChunks descriptors: fields of up to
//     kMaxChunks * 32 blocks of 4x4x4 values (4,194,304 blocks, about
//     2.7e8 values, e.g. 881 x 881 x 287).  Larger fields are rejected with FWI_ERR_ARG before any
//     device work.
//   - The block occupies about 1 MiB on every GPU that loads the library,
//     until the process exits.
//   - All calls share the block and it keeps the previous call's contents;
//     each call clears the words that must start at zero.  Calls that overlap
//     on the GPU (other streams, other host threads) race on it.
//   - The first call on a device looks up the block's device address with
//     cudaGetSymbolAddress (with that device current); make that first call
//     before any stream capture.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr long kMaxChunks = 131072;
// Word layout of the block for a field of nchunks chunks: words [0, nchunks)
// hold the chunks' look-back descriptors and word nchunks the chunk ticket
// (both cleared by the encoder launch); the stream size and the status word
// sit at fixed offsets after the largest descriptor area.
constexpr long kSizeWord = kMaxChunks + 2;
constexpr long kStatusWord = kMaxChunks + 3;
constexpr long kScratchWords = kMaxChunks + 8;
static_assert(kStatusWord < kScratchWords, "scratch layout");

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned long long* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch block for the current device (set up once).
cudaError_t scratch_address(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int zfp_compress_fixed_accuracy_noalloc(const float* d_in, int nx, int ny, int nz,
                                                   double atol, void* d_out, size_t out_capacity,
                                                   size_t* h_out_bytes, void* stream) {
  using namespace fwi;
  if (!d_in || !d_out || !h_out_bytes || nx <= 0 || ny <= 0 || nz <= 0 || !(atol > 0.0) ||
      !isfinite(atol) || ((uintptr_t)d_out & 7) || ((uintptr_t)d_in & 3))
    return FWI_ERR_ARG;
  // size guard in 64-bit arithmetic, before any layout work: each block
  // count is at most 2^29, so no product below can overflow
  const long nbx = ((long)nx + 3) / 4, nby = ((long)ny + 3) / 4, nbz = ((long)nz + 3) / 4;
  const long max_blocks = kMaxChunks * ZC_CHUNK;
  if (nbx > max_blocks || nby > max_blocks || nbz > max_blocks || nbx * nby > max_blocks ||
      nbx * nby * nbz > max_blocks)
    return FWI_ERR_ARG;  // beyond the fixed scratch
  unsigned long long* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return FWI_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* d_size = scratch + kSizeWord;
  int* d_status = reinterpret_cast<int*>(scratch + kStatusWord);
  int e_frexp;
  frexp(atol, &e_frexp);
  const int minexp = e_frexp - 1;
  // the encoder clears its descriptors and ticket itself; clear the status here
  if (cudaMemsetAsync(d_status, 0, sizeof(int), s) != cudaSuccess ||
      zfp_encode_chained_launch(d_in, Grid{nx, ny, nz, nx}, minexp, (uint8_t*)d_out, nullptr,
                                out_capacity, d_size, d_status, scratch, s) != cudaSuccess) {
    cudaGetLastError();
    return FWI_ERR_CUDA;
  }
  unsigned long long size = 0;
  int flags = 0;
  if (cudaMemcpyAsync(&size, d_size, sizeof(size), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&flags, d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FWI_ERR_CUDA;
  }
  *h_out_bytes = (size_t)size;
  return status_from_flags(flags);
}
