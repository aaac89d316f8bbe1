// Internal definitions shared by the libfwi translation units (not part of
// the C ABI; the public interface is include/fwi.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "fwi.h"

namespace fwi {

// ---- launch accounting and optional per-kernel timing ------------------------
void count_launch();
// Kernel classes timed by fwi_profile_* (CUDA events on the launching stream).
enum KernelClass : int {
  KC_STENCIL_FWD = 0,
  KC_STENCIL_ADJ = 1,
  KC_ZFP_ENCODE = 2,
  KC_ZFP_DECODE = 3,
  KC_OTHER = 4,
  KC_COUNT = 5,
};
// Returns a slot (or -1 when profiling is off); pair with prof_end.
int prof_begin(int cls, cudaStream_t s);
void prof_end(int slot, cudaStream_t s);

// ---- device status word -----------------------------------------------------
// One int per call, OR-ed bit flags written by kernels; translated to a status
// code on the host.
enum : int {
  ST_NONFINITE = 1,
  ST_CORRUPT = 2,
  ST_CAPACITY = 4,
  ST_TIMEOUT = 8,
};
int status_from_flags(int flags);

// ---- pitched wavefield layout ----------------------------------------------
// Working fields are [nz][ny][pitch], pitch = nx rounded up to a multiple of 4
// (16-byte rows); the padding columns hold zeros.
struct Grid {
  int nx, ny, nz;
  int pitch;
  size_t cells() const { return (size_t)pitch * ny * nz; }
};
inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// ---- codec layout -----------------------------------------------------------
constexpr int ZC_S = 25;        // block-floating-point fraction bits
constexpr int ZC_G = 11;        // guard planes
constexpr int ZC_CHUNK = 32;    // blocks per chunk (one warp)
constexpr int ZC_MAXBITS = 9 + 32 * 64 + 64;
constexpr uint32_t ZC_MAGIC = 0x315A4346u;  // "FCZ1"
constexpr uint32_t ZC_VERSION = 1u;

struct ZLayout {
  long nbx, nby, nbz, nblocks, nchunks;
  size_t chunk_table, length_table, payload;  // byte offsets in the stream
  size_t max_bytes;
};
ZLayout zlayout(int nx, int ny, int nz);

// Compress one pitched field into out (device), which has `capacity` bytes
// counted from the device offset *d_base (bytes; NULL = 0).  The stream size
// is written to *d_size (device); flags go to *d_status.  Two passes with no
// dependency between chunks: code every chunk into a fixed staging slot, then
// one CTA per tile of chunks places the words.  `scratch` must hold
// zfp_encode_scratch_bytes() bytes.  Asynchronous.
size_t zfp_encode_scratch_bytes(int nx, int ny, int nz);
cudaError_t zfp_encode_launch(const float* in, Grid g, int minexp, uint8_t* out,
                              const unsigned long long* d_base, size_t capacity,
                              unsigned long long* d_size, int* d_status, void* scratch,
                              cudaStream_t s);
// Single-pass variant whose scratch is only nchunks+1 words (per-chunk
// look-back descriptors and a ticket), zeroed here: chunks find their offset
// by a decoupled look-back over their predecessors.  Same stream.
size_t zfp_encode_chained_scratch_words(int nx, int ny, int nz);
cudaError_t zfp_encode_chained_launch(const float* in, Grid g, int minexp, uint8_t* out,
                                      const unsigned long long* d_base, size_t capacity,
                                      unsigned long long* d_size, int* d_status,
                                      unsigned long long* scratch, cudaStream_t s);

// Decompress a stream located at in + *d_base (d_base NULL = 0) of at most
// `avail` bytes into a pitched field.  Asynchronous; errors go to *d_status.
cudaError_t zfp_decode_launch(const uint8_t* in, const unsigned long long* d_base,
                              size_t avail, float* out, Grid g, int* d_status,
                              cudaStream_t s);

// ---- stencil ----------------------------------------------------------------
struct StencilParams {
  Grid g;
  float c[5];      // 8th-order coefficients / h^2
  float dt;
  const float* b;  // dt^2 / m, pitched
  const float* sx; // damping profile s(x) * dt / 2 per axis
  const float* sy;
  const float* sz;
  int* status;     // device status word (bounded waits report timeouts here)
};

// out = step(cur, prev) with one point injection (cell index in the pitched
// layout, or -1) of value q * b / (1 + s dt/2).  out may alias prev.
cudaError_t stencil_step_launch(const StencilParams& p, const float* cur, const float* prev,
                                float* out, long src_cell, const float* d_wavelet, int n,
                                cudaStream_t s);
// Adjoint step with fused imaging:
//   out = step(cur, prev);  grad -= weight * uk * (out - 2 cur + prev) / dt^2
// (receiver injection is added afterwards by inject_adjoint_launch).
cudaError_t stencil_adjoint_launch(const StencilParams& p, const float* cur, const float* prev,
                                   float* out, const float* uk, float* grad, float weight,
                                   cudaStream_t s);
// out[rec] += r * fac; if uk: grad[rec] -= weight * uk[rec] * r * fac / dt^2.
cudaError_t inject_adjoint_launch(const StencilParams& p, const long* rec_cell, const float* rec_fac,
                                  int nrec, const float* resid_row, float* out, const float* uk,
                                  float* grad, float weight, cudaStream_t s);
// fac[r] = b / (1 + s dt/2) at receiver r (injection weight).
cudaError_t rec_fac_launch(const StencilParams& p, const long* rec_cell, int nrec, float* fac,
                           cudaStream_t s);
// d_row[r] = field[rec_cell[r]]
cudaError_t gather_launch(const float* field, const long* rec_cell, int nrec, float* d_row,
                          cudaStream_t s);
// rec_cell[r] = pitched cell of (i,j,k); flags ST_CORRUPT (as "bad index") on out-of-range.
cudaError_t rec_cells_launch(const int* rec_ijk, int nrec, Grid g, long* rec_cell, int* d_status,
                             cudaStream_t s);
// Setup: b = dt^2/m (pitched, zero in padding), damping profiles.
cudaError_t setup_model_launch(const float* m, Grid g, float dt, float* b, int* d_status,
                               cudaStream_t s);
cudaError_t setup_profiles_launch(Grid g, int nbl, double h, double vmax, double R, double dt,
                                  float* sx, float* sy, float* sz, cudaStream_t s);
// Pitched <-> packed copies.
cudaError_t pack_launch(const float* pitched, Grid g, float* packed, cudaStream_t s);
cudaError_t unpack_launch(const float* packed, Grid g, float* pitched, cudaStream_t s);
cudaError_t unpack_add_launch(const float* pitched, Grid g, float* packed, cudaStream_t s);
// Residual r = a - b, FP64 half-sum-of-squares added to *d_acc; dot product
// likewise.  `part` holds reduce_scratch_doubles() doubles; the summation
// order is fixed, so results are bitwise reproducible.
size_t reduce_scratch_doubles();
cudaError_t misfit_launch(const float* a, const float* b, size_t n, float* r, double* d_acc,
                          double* part, cudaStream_t s);
cudaError_t dot_launch(const float* a, const float* b, size_t n, double* d_acc, double* part,
                       cudaStream_t s);

}  // namespace fwi
