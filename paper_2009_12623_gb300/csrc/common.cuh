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
void count_launches(unsigned long long n);  // kernels of a replayed CUDA graph
unsigned long long launches_so_far();
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

// Per 4x4x4 block of a field, whether any value reaches `threshold` (or is
// NaN/Inf): bit bx % 16 of words[(bz * nby + by) * ntx + bx / 16], ntx =
// ceil(pitch / 64) (one 16-bit word per 64-cell tile row segment).  Written
// by a forward step for the field it produces; with threshold =
// 2^(minexp - 11) a block without its bit codes as zero (no coded plane), so
// the encoder need not read it.
struct LiveMap {
  uint16_t* words;
  float threshold;
  int ntx, nby;
};
size_t live_map_words(Grid g);
// The threshold for tolerance exponent minexp, or 0 when no map can stand in
// for the encoder's own test at that tolerance (below 2^-126 a block of
// subnormals can still code planes).
float live_threshold(int minexp);

// Compress one pitched field into out (device), which has `capacity` bytes
// counted from the device offset *d_base (bytes; NULL = 0).  The stream size
// is written to *d_size (device); flags go to *d_status.  Two passes with no
// dependency between chunks: code every chunk into a fixed staging slot, then
// one CTA per tile of chunks places the words.  `scratch` must hold
// zfp_encode_scratch_bytes() bytes.  Asynchronous.
size_t zfp_encode_scratch_bytes(int nx, int ny, int nz);
// With live (nullable, written for this field at this tolerance's
// threshold), blocks without their live bit are coded as zero unread.
cudaError_t zfp_encode_launch(const float* in, Grid g, int minexp, uint8_t* out,
                              const unsigned long long* d_base, size_t capacity,
                              unsigned long long* d_size, int* d_status, void* scratch,
                              cudaStream_t s, const LiveMap* live = nullptr);
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

// Where a compressed field's block-length table lies, for kernels that
// consume its decoded values only where the imaging decoder wrote them: a
// block whose coded length is one bit decodes to exactly 0, so its cells are
// neither written nor needed.  The stream starts at arena + *base (a device
// word); arena == NULL means "no table: every block is live".
struct ZeroBlocks {
  const uint8_t* arena;
  const unsigned long long* base;
  unsigned long long length_table;  // byte offsets within the stream
  unsigned long long payload;
  unsigned long long capacity;      // bytes readable from arena
  int nbx, nby;                     // blocks per row and per column of a layer
};
ZeroBlocks zero_blocks(const uint8_t* arena, const unsigned long long* base, size_t capacity, Grid g);
// counts[j] = blocks coded as zero in the stream at arena + offs[j], j < nslots
// (UINT64_MAX where the stream does not fit the capacity).  Asynchronous.
cudaError_t zfp_count_zero_blocks_launch(const uint8_t* arena, const unsigned long long* offs, int nslots,
                                         size_t capacity, Grid g, unsigned long long* counts, cudaStream_t s);

#ifdef __CUDACC__
// The length table, or NULL when there is none or the stream does not fit
// the arena (then every block counts as live).
__device__ __forceinline__ const uint16_t* zero_table(const ZeroBlocks& z) {
  if (!z.arena) return nullptr;
  const unsigned long long b = *z.base;
  if (b > z.capacity || z.payload > z.capacity - b) return nullptr;
  return reinterpret_cast<const uint16_t*>(z.arena + b + z.length_table);
}
// Whether cell (x, y, z) lies in a block that is not coded as zero.
__device__ __forceinline__ bool block_live(const uint16_t* tab, const ZeroBlocks& z, int x, int y, int zz) {
  return !tab || tab[((long)(zz >> 2) * z.nby + (y >> 2)) * z.nbx + (x >> 2)] != 1;
}
// One cell of the imaging sum (Eq. 4): g - u (l_prev - 2 l_cur + l_next) idt2
// with l_prev = lambda_{k-1}, l_cur = lambda_k, l_next = lambda_{k+1} and
// idt2 = weight / dt^2, in one fixed rounding sequence (no contraction), so
// that every kernel that images a cell produces the same bits.
__device__ __forceinline__ float image_update(float g, float u, float lp, float lc, float ln, float idt2) {
  const float d = __fadd_rn(__fsub_rn(lp, __fmul_rn(2.0f, lc)), ln);
  return __fsub_rn(g, __fmul_rn(__fmul_rn(u, d), idt2));
}
#endif

// Imaging from a compressed state (full-history reverse sweep): the decoder
// of u^k, run after the adjoint step that produced lambda_{k-1}, images the
// blocks u^k does not code as zero straight from its registers,
//   g -= u^k (lp - 2 lc + ln) idt2,
// and writes decoded values only for blocks flagged in rec_block (those with
// receivers, whose imaging correction the receiver injection adds).
struct ImageArgs {
  const float* lp;   // lambda_{k-1}
  const float* lc;   // lambda_k
  const float* ln;   // lambda_{k+1}
  float* g;
  float idt2;
  const uint8_t* rec_block;  // per block (codec block order): 1 = holds a receiver
};
cudaError_t zfp_decode_image_launch(const uint8_t* in, const unsigned long long* d_base, size_t avail,
                                    float* uk_out, Grid g, int* d_status, const ImageArgs& im,
                                    cudaStream_t s);
// rec_block[b] = 1 for every 4x4x4 block b (codec order) holding a receiver cell
// (pitched cell indices), 0 elsewhere.
cudaError_t receiver_blocks_launch(const long* rec_cell, int nrec, Grid g, uint8_t* rec_block, cudaStream_t s);

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

// The adjoint recurrence's step without imaging (the same step, no source),
// timed as an adjoint-stencil launch; out may alias prev.
cudaError_t stencil_adjoint_step_launch(const StencilParams& p, const float* cur, const float* prev,
                                        float* out, cudaStream_t s);
// out = step(cur, prev) with one point injection (cell index in the pitched
// layout, or -1) of value q * b / (1 + s dt/2).  out may alias prev.
// With live (nullable), also writes the liveness map of out (every word).
cudaError_t stencil_step_launch(const StencilParams& p, const float* cur, const float* prev,
                                float* out, long src_cell, const float* d_wavelet, int n,
                                cudaStream_t s, const LiveMap* live = nullptr);
// Adjoint step with fused imaging:
//   out = step(cur, prev);  grad -= weight * uk * (out - 2 cur + prev) / dt^2
// (receiver injection is added afterwards by inject_adjoint_launch).
cudaError_t stencil_adjoint_launch(const StencilParams& p, const float* cur, const float* prev,
                                   float* out, const float* uk, float* grad, float weight,
                                   cudaStream_t s);
// out[rec] += r * fac; if uk: grad[rec] -= weight * uk[rec] * r * fac / dt^2
// (skipped where zb, nullable, marks the block of uk as zero).
cudaError_t inject_adjoint_launch(const StencilParams& p, const long* rec_cell, const float* rec_fac,
                                  int nrec, const float* resid_row, float* out, const float* uk,
                                  float* grad, float weight, cudaStream_t s, const ZeroBlocks* zb = nullptr);
// fac[r] = b / (1 + s dt/2) at receiver r (injection weight).
cudaError_t rec_fac_launch(const StencilParams& p, const long* rec_cell, int nrec, float* fac,
                           cudaStream_t s);
// d_row[r] = field[rec_cell[r]]
cudaError_t gather_launch(const float* field, const long* rec_cell, int nrec, float* d_row,
                          cudaStream_t s);
// rec_cell[r] = pitched cell of (i,j,k) - (ox,oy,oz); flags ST_CORRUPT (as
// "bad index") when that lies outside the grid.
cudaError_t rec_cells_launch(const int* rec_ijk, int nrec, Grid g, long* rec_cell, int* d_status,
                             cudaStream_t s, int ox = 0, int oy = 0, int oz = 0);
// Setup: b = dt^2/m (pitched, zero in padding), damping profiles.  The model
// may be a larger packed array (rows of mnx, mny rows per plane; 0 = the
// grid's own) of which the window at (ox, oy, oz) is used.
cudaError_t setup_model_launch(const float* m, Grid g, float dt, float* b, int* d_status,
                               cudaStream_t s, int mnx = 0, int mny = 0, int ox = 0, int oy = 0,
                               int oz = 0);
cudaError_t setup_profiles_launch(Grid g, int nbl, double h, double vmax, double R, double dt,
                                  float* sx, float* sy, float* sz, cudaStream_t s);
// Pitched <-> packed copies.
cudaError_t pack_launch(const float* pitched, Grid g, float* packed, cudaStream_t s);
cudaError_t unpack_launch(const float* packed, Grid g, float* pitched, cudaStream_t s);
cudaError_t unpack_add_launch(const float* pitched, Grid g, float* packed, cudaStream_t s);
// dst (packed, gnx x gny per plane) at window (ox, oy, oz) += pitched field.
cudaError_t stack_add_launch(const float* pitched, Grid g, float* dst, int gnx, int gny, int ox, int oy,
                             int oz, cudaStream_t s);

// ---- many fields per launch (batched shots) ---------------------------------
constexpr int kStencilMaxFields = 32;
// One field of a multi-field stencil launch: the step (forward, with its
// point source) or the adjoint step with imaging, as in the single-field calls.
struct StencilField {
  const float* cur;
  const float* prev;
  float* out;
  long src_cell;          // forward: injection cell or -1
  const float* wavelet;   // forward: source samples (device)
  int n;                  // forward: time index of the sample
  const float* uk;        // adjoint: forward state for the imaging condition
  float* grad;            // adjoint: gradient accumulator
  int zc;                 // z-chunk of the tiles (0: automatic)
};
// Resident CTAs of the multi-field forward or adjoint kernel on the whole GPU
// (0 on failure).
int stencil_multi_capacity(bool adjoint);
// One persistent launch over the tiles of all fields; ctas <= 0 = resident capacity.
cudaError_t stencil_multi_launch(bool adjoint, int nfields, const StencilParams* const* p,
                                 const StencilField* f, float weight, int ctas, cudaStream_t s);
struct RecTask {
  const float* field;   // gather: sampled field
  float* row_out;       // gather: output row
  const long* cell;
  const float* fac;     // inject: weights
  const float* row_in;  // inject: residual row
  float* out;           // inject: adjoint field
  const float* uk;      // inject: forward state (NULL: no imaging term)
  float* grad;
};
struct MultiRec {
  RecTask t[kStencilMaxFields];
  int first[kStencilMaxFields + 1];
  int nfields;
  float idt2;
};
cudaError_t gather_multi_launch(int nfields, const RecTask* t, const int* nrec, cudaStream_t s);
cudaError_t inject_multi_launch(int nfields, const RecTask* t, const int* nrec, float dt, float weight,
                                cudaStream_t s);

// Bounded-wait self-test: one CTA waits `polls` polls on an mbarrier that
// never completes and flags ST_TIMEOUT in *d_status.
cudaError_t wait_selftest_launch(int* d_status, long polls, cudaStream_t s);
cudaError_t quotient_selftest_launch(const float* num, const float* den, float* out, long n, cudaStream_t s);

// Residual r = a - b, FP64 half-sum-of-squares added to *d_acc; dot product
// likewise.  `part` holds reduce_scratch_doubles() doubles; the summation
// order is fixed, so results are bitwise reproducible.
size_t reduce_scratch_doubles();
cudaError_t misfit_launch(const float* a, const float* b, size_t n, float* r, double* d_acc,
                          double* part, cudaStream_t s);
cudaError_t dot_launch(const float* a, const float* b, size_t n, double* d_acc, double* part,
                       cudaStream_t s);

}  // namespace fwi
