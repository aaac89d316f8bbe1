// Host-side helpers shared by the entry-point translation units: stream-
// ordered scratch allocations, the codec side stream, argument checks and the
// device slot-table bookkeeping of the checkpoint store.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "common.cuh"

namespace fwi {
namespace {

// 8th-order central second-difference weights (times h^2).
const double kC[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

// Stream-ordered allocations released when the scope ends.
struct Pool {
  cudaStream_t s;
  std::vector<void*> ptrs;
  bool failed = false;
  explicit Pool(cudaStream_t st) : s(st) {}
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMallocAsync(&p, n * sizeof(T), s) != cudaSuccess) {
      failed = true;
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Pool() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

// A second stream for codec work with a few events.  `main` is the stream
// the sweep itself runs on (the caller's).  On destruction the codec stream
// is joined into it, so stream-ordered frees on the caller's stream stay
// safe on every return path.
struct CodecStream {
  cudaStream_t owner;
  cudaStream_t main;
  cudaStream_t s = nullptr;
  cudaEvent_t ev[8] = {nullptr};
  cudaEvent_t done = nullptr;
  bool ok = false;
  explicit CodecStream(cudaStream_t o) : owner(o), main(o) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s = nullptr;
      return;
    }
    for (auto& e : ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    // codec work may only start after everything the owner issued so far
    ok = cudaEventRecord(done, owner) == cudaSuccess && cudaStreamWaitEvent(s, done, 0) == cudaSuccess;
  }
  // main waits for all codec work issued so far
  cudaError_t join() {
    cudaError_t e = cudaEventRecord(done, s);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(main, done, 0);
  }
  ~CodecStream() {
    if (s) {
      if (done) join();
      cudaStreamDestroy(s);
    }
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (done) cudaEventDestroy(done);
    cudaGetLastError();
  }
};

// NVTX range of the sweep phase being enqueued ("fwi forward sweep",
// "fwi reverse sweep", ...), for profilers: nsys shows it on the host
// timeline, and `ncu --nvtx --nvtx-include "fwi reverse sweep/"` profiles
// only that phase's kernels.  Costs nothing when no tool is attached.
struct PhaseRange {
  const char* name = nullptr;
  void enter(const char* n) {
    if (n == name) return;
    if (name) nvtxRangePop();
    nvtxRangePushA(n);
    name = n;
  }
  ~PhaseRange() {
    if (name) nvtxRangePop();
  }
};
constexpr const char* kPhaseForward = "fwi forward sweep";
constexpr const char* kPhaseReverse = "fwi reverse sweep";

bool geometry_ok(const fwi_geometry* g) {
  return g && g->nx > 0 && g->ny > 0 && g->nz > 0 && g->nt >= 0 && g->h > 0 && g->dt > 0 &&
         g->nbl >= 0 && (g->nbl == 0 || (g->sponge_R > 0 && g->sponge_R < 1 && g->vmax > 0)) &&
         (long)g->nx * g->ny * g->nz < (1L << 40);
}

int minexp_of(double atol) {
  int e;
  frexp(atol, &e);
  return e - 1;
}

// Where the reverse sweeps decode u^{k-1}: beside adjoint step k on the
// codec stream (1), or in order on the sweep's own stream before it (0).  In
// order is faster on GB300 (881x881x287, full history at atol 1e-4: reverse
// phase 3.80 s against 4.15 s overlapped, where the adjoint stencil ran
// 1.37-1.71 ms per step instead of 1.08 ms): the memory-bound stencil and
// the decoder, which writes a whole field per step, contend for HBM and L2
// rather than filling each other's idle cycles.  Encoding keeps its overlap
// with the next forward step (forward phase 3.06 s against 3.13 s in order).
#ifndef FWI_DECODE_OVERLAP
#define FWI_DECODE_OVERLAP 0
#endif
constexpr bool kDecodeOverlap = FWI_DECODE_OVERLAP != 0;

#define CK(x)                          \
  do {                                 \
    if ((x) != cudaSuccess) {          \
      cudaGetLastError();              \
      return FWI_ERR_CUDA;             \
    }                                  \
  } while (0)

}  // namespace

// Offset bookkeeping for compressed slots: slot j starts where slot j-1 ended
// (256-byte aligned); the largest end so far is kept in *peak.  Run on the
// device so that no host synchronisation is needed between checkpoints.
cudaError_t slot_offset_launch(unsigned long long* off, const unsigned long long* size, int j,
                               cudaStream_t s);
cudaError_t track_peak_launch(const unsigned long long* off, const unsigned long long* size, int j,
                              unsigned long long* peak, cudaStream_t s);

}  // namespace fwi

// The checkpoint store behind the opaque handle of include/fwi.h.
struct fwi_ckpt_store {
  uint8_t* arena = nullptr;
  size_t capacity = 0;
  fwi_store_stats stats{};
  // slot table of the last forward sweep (device), kept for a later reverse sweep
  unsigned long long* d_offs = nullptr;
  unsigned long long* d_sizes = nullptr;
  int slot_cap = 0;
  bool filled = false;  // a forward sweep completed and its checkpoints are in the arena
  int nslots = 0;       // slots the last forward sweep used
  bool lossy = false;   // whether they hold compressed streams
  float* carry = nullptr;  // binomial: final forward state pair kept between the two halves
  size_t carry_bytes = 0;
  fwi_geometry geom{};
  fwi_ckpt_policy pol{};
};
