/*
 * libfwi -- GB300 (sm_103a) checkpointed full-waveform-inversion gradient with
 * lossy, error-bounded checkpoint compression.
 *
 * Method: Kukreja et al., "Lossy Checkpoint Compression in Full Waveform
 * Inversion".  The library computes, for one shot, the simulated data
 * d_sim = P_r A(m)^-1 P_s^T q_s (Sec. 2, Eq. (2)), the misfit
 * Phi = 1/2 ||d_sim - d_obs||^2 (Eq. (3)) and its gradient with respect to
 * the squared slowness m (Eq. (4)), keeping the forward wavefield as
 * checkpoints (Sec. 1.3) that are compressed with a fixed-accuracy block codec
 * (Sec. 1.4, Fig. 1).
 *
 * Conventions shared by every call:
 *   - Fields are FP32, C order [nz][ny][nx] (x fastest), unpadded, on the
 *     device unless the name starts with h_.
 *   - Pointers named d_* are caller-owned device memory; h_* are host memory.
 *     The library allocates device memory only inside fwi_ckpt_store_create
 *     (the checkpoint arena, freed by fwi_ckpt_store_destroy) and for the
 *     per-call working set (wavefields, scan scratch), which it takes from the
 *     device's stream-ordered memory pool and returns before the call ends.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *     their kernels on it; a call that returns a host scalar (h_out_bytes,
 *     h_misfit, h_out) synchronises that stream before returning.
 *   - Every call returns FWI_OK (0) or a negative status; nothing aborts or
 *     throws across this interface.  fwi_status_string names the codes.
 */
#ifndef FWI_H
#define FWI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define FWI_OK 0
#define FWI_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, ...) */
#define FWI_ERR_CAPACITY (-2)  /* output or checkpoint arena too small */
#define FWI_ERR_CORRUPT (-3)   /* malformed compressed stream */
#define FWI_ERR_NONFINITE (-4) /* NaN or Inf in a field given to the codec */
#define FWI_ERR_CUDA (-5)      /* a CUDA runtime call failed */
#define FWI_ERR_TIMEOUT (-6)   /* a bounded device-side wait gave up */
#define FWI_ERR_NOMEM (-7)     /* device allocation failed */

/* ---- geometry ------------------------------------------------------------- */
/* Grid, time axis and absorbing layer (Sec. 3, "Reference Problem": grid with
 * an absorbing layer on every face, fixed step dt, nt steps).  The nbl-cell
 * layer is part of the nx*ny*nz grid.  Its damping rate at depth d (m) into
 * the layer is (3 vmax / 2W) ln(1/sponge_R) (d/W)^2, W = nbl*h, summed over
 * the three axes, and it multiplies the model given to the call. */
typedef struct {
  int nx, ny, nz;
  double h;        /* grid spacing, m */
  double dt;       /* time step, s */
  int nt;          /* number of time steps N */
  int nbl;         /* absorbing-layer width, cells (0 = none) */
  double sponge_R; /* target reflection coefficient of the layer, (0,1) */
  double vmax;     /* reference velocity of the damping profile, m/s */
} fwi_geometry;

/* ---- checkpoint policy and schedule (Sec. 1.3) ---------------------------- */
#define FWI_CKPT_FULL 1    /* keep every forward state u^1..u^N */
#define FWI_CKPT_EVERY_K 2 /* keep the pair (u^{c-1}, u^c) at c = 0, K, 2K, ...;
                              recompute the states in between during the
                              reverse sweep */
#define FWI_CKPT_BINOMIAL 3 /* at most k_or_snaps state pairs at a time, placed by
                               recursive splitting so that the forward steps
                               recomputed are the fewest possible (the
                               Revolve family of schedules, Sec. 1.3); the
                               pairs are used last-in first-out */
#define FWI_CKPT_SUBSAMPLE 4 /* the subsampling baseline of Sec. 4.7: keep u^k only for
                                k = f, 2f, ... (f = k_or_snaps) and apply the imaging
                                condition only at those steps, weighted by f */
typedef struct {
  int mode;       /* FWI_CKPT_* */
  int k_or_snaps; /* K for FWI_CKPT_EVERY_K, snapshot pairs for FWI_CKPT_BINOMIAL,
                     the factor f for FWI_CKPT_SUBSAMPLE */
  double atol;    /* > 0: compress every checkpoint with this absolute error
                     tolerance (Sec. 1.4); <= 0: raw FP32 copies */
} fwi_ckpt_policy;

/* Actions of a schedule: the "forward, store, backward, load and recompute
 * events" of Sec. 1.3. */
#define FWI_ACT_ADVANCE 1   /* forward step: u^step -> u^{step+1}, record data d^step */
#define FWI_ACT_STORE 2     /* store the state at `step` (arg = 1: u^step; 2: u^{step-1}, u^step) */
#define FWI_ACT_RESTORE 3   /* make the stored state at `step` current (arg as for STORE) */
#define FWI_ACT_RECOMPUTE 4 /* forward step without recording: u^step -> u^{step+1} */
#define FWI_ACT_ADJOINT 5   /* adjoint step k = step (lambda_{k-1}) and imaging with u^k
                               weighted by arg (0 means 1; -1: no imaging) */
#define FWI_ACT_FREE 6      /* drop the most recently stored state pair (binomial) */
typedef struct {
  int kind;
  int step;
  int arg;
} fwi_action;

/* Fill out[0..cap) with the schedule fwi_gradient executes for nt steps under
 * pol; *n_out = total number of actions.  Returns FWI_ERR_CAPACITY (with
 * *n_out set) when cap is smaller; out may be NULL with cap = 0 to query. */
int fwi_ckpt_schedule(int nt, const fwi_ckpt_policy* pol, fwi_action* out, size_t cap,
                      size_t* n_out);

/* ---- compressed checkpoint store (Fig. 1: the compressed states handed from
 * the forward to the reverse sweep) -------------------------------------- */
typedef struct fwi_ckpt_store fwi_ckpt_store;

/* One device arena of capacity_bytes (cudaMalloc).  Checkpoints are appended
 * by a device-side cursor, so no host synchronisation happens per checkpoint.
 * FWI_ERR_NOMEM if the arena cannot be allocated. */
int fwi_ckpt_store_create(size_t capacity_bytes, fwi_ckpt_store** out);
int fwi_ckpt_store_destroy(fwi_ckpt_store* st);

typedef struct {
  size_t capacity_bytes;
  size_t used_bytes;     /* bytes the last gradient stored (or needed, if it overflowed) */
  size_t raw_bytes;      /* FP32 bytes of the same checkpoints uncompressed */
  int n_checkpoints;     /* fields stored by the last gradient */
  int overflowed;        /* 1 if the last gradient ran out of arena */
} fwi_store_stats;
int fwi_ckpt_store_stats(const fwi_ckpt_store* st, fwi_store_stats* out);

/* Bytes of each checkpoint slot the last forward sweep filled, in slot order
 * (full history: slot j holds u^{j+1}; every-K: the pairs in schedule order,
 * u^k before u^{k-1}; binomial: the last state held by each slot), written to
 * h_bytes[0 .. min(cap, n) - 1] with n, the slot count, in *n_out (0 while
 * the store holds no forward sweep).  Compressed stores report each stream's size, raw
 * stores the field size.  This is how the compressibility of the wavefield
 * over the simulation (Sec. 4.1) is read.  Synchronous (device-to-host copy).
 * FWI_ERR_ARG for a null store or n_out, a negative cap, or a null h_bytes
 * with cap > 0. */
int fwi_ckpt_store_slot_bytes(const fwi_ckpt_store* st, unsigned long long* h_bytes, int cap, int* n_out);

/* Blocks of 4x4x4 values that each compressed slot of the last forward sweep
 * codes as zero (the single bit 0: every value of the block lies below the
 * tolerance's last coded bit plane, Sec. 1.4), same slot order and argument
 * rules as fwi_ckpt_store_slot_bytes; raw stores report 0.  Such blocks
 * decode to exactly 0, and the full-history reverse sweep neither writes nor
 * images them, so this is how much of each state that sweep skips.  Counted
 * on the device from the streams' length tables; synchronous.  A slot whose
 * stream does not fit the arena reports UINT64_MAX. */
int fwi_ckpt_store_slot_zero_blocks(const fwi_ckpt_store* st, unsigned long long* h_counts, int cap,
                                    int* n_out);

/* ---- forward modelling (Sec. 2, Eq. (1)-(2)) ------------------------------ */
/* Runs u^{n+1} for n = 0..nt-1 from the zero state (or from the given pair
 * d_u_prev_init = u^{-1}, d_u_cur_init = u^0) and records
 * d_rec_out[n*nrec + r] = u^{n+1} at receiver r.
 *   d_m        squared slowness 1/c^2 (s^2/m^2), nx*ny*nz
 *   h_wavelet  source samples q^0..q^{nt-1} (host), added at (src_i, src_j, src_k)
 *   d_rec_ijk  nrec (i,j,k) int triples (device), grid nodes
 *   d_u_prev_out / d_u_last_out   optional: u^{nt-1} and u^{nt}
 * Scheme: 8th-order Laplacian, 2nd-order leapfrog in time, absorbing layer
 * (see fwi_geometry). */
int fwi_forward(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i,
                int src_j, int src_k, const int* d_rec_ijk, int nrec, float* d_rec_out,
                const float* d_u_prev_init, const float* d_u_cur_init, float* d_u_prev_out,
                float* d_u_last_out, void* stream);

/* ---- gradient (Sec. 2, Eq. (3)-(4); Sec. 1.3-1.4, Fig. 1) ---------------- */
/* Forward sweep storing checkpoints into st per pol, misfit, adjoint sweep
 * decompressing them, imaging condition accumulated as
 *   d_grad += dPhi/dm = -sum_{k=1}^{N} u^k (l_{k-1} - 2 l_k + l_{k+1}) / dt^2
 * (the damping is held fixed).  *h_misfit = Phi (FP64).  Synchronises.
 * FWI_ERR_CAPACITY if the arena is too small for the policy (the store's
 * stats then give the bytes needed); d_grad is left unchanged in that case.
 * d_obs is nt*nrec, time-major. */
int fwi_gradient(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i,
                 int src_j, int src_k, const int* d_rec_ijk, int nrec, const float* d_obs,
                 float* d_grad, double* h_misfit, fwi_ckpt_store* st,
                 const fwi_ckpt_policy* pol, void* stream);

/* The two halves of fwi_gradient, for callers that form the adjoint source
 * themselves (automatic differentiation: the forward pass keeps the
 * checkpoints, the backward pass receives dL/dd for any loss L).
 * fwi_forward_store runs the forward sweep, writes the records
 * (d_rec_out[n*nrec + r] = u^{n+1}) and stores the checkpoints per pol in st
 * (FWI_ERR_CAPACITY as for fwi_gradient).  fwi_adjoint_store then runs the
 * reverse sweep from those checkpoints with the adjoint source d_resid
 * (nt*nrec) injected at the receivers and accumulates
 *   d_grad += -sum_k u^k (l_{k-1} - 2 l_k + l_{k+1}) / dt^2 = J^T d_resid
 * (Eq. (4), J = dd/dm).  It needs the same geometry, policy, model,
 * wavelet and acquisition as the forward call (FWI_ERR_ARG if the store holds
 * no checkpoints from a matching forward call).  Both synchronise. */
int fwi_forward_store(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i,
                      int src_j, int src_k, const int* d_rec_ijk, int nrec, float* d_rec_out,
                      fwi_ckpt_store* st, const fwi_ckpt_policy* pol, void* stream);
int fwi_adjoint_store(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i,
                      int src_j, int src_k, const int* d_rec_ijk, int nrec, const float* d_resid,
                      float* d_grad, fwi_ckpt_store* st, const fwi_ckpt_policy* pol, void* stream);

/* The same gradient with every array in host memory (h_m, h_rec_ijk, h_obs,
 * h_grad: same layouts as above; pinned memory gives the fastest copies).
 * Copies the model and receivers, runs the forward sweep while h_obs and
 * h_grad travel to the device on a second stream, then the misfit and the
 * reverse sweep (the same kernels as fwi_gradient, bitwise the same result),
 * and copies h_grad back (h_grad += ...).  h_misfit is required.
 * Synchronises. */
int fwi_gradient_host(const fwi_geometry* g, const float* h_m, const float* h_wavelet,
                      int src_i, int src_j, int src_k, const int* h_rec_ijk, int nrec,
                      const float* h_obs, float* h_grad, double* h_misfit, fwi_ckpt_store* st,
                      const fwi_ckpt_policy* pol, void* stream);

/* ---- batched shots (Sec. 2: the misfit and its gradient are sums over
 * shots; Sec. 3: every shot images only its own part of the model) -------- */
/* One shot of a batch.  The shot is modelled on its aperture: the sub-grid
 * nx*ny*nz at (x0, y0, z0) of the model grid, with the absorbing layer of
 * fwi_geometry (nbl, sponge_R, vmax) inside the aperture on all six faces, as
 * if fwi_gradient were called on that window of the model.  Source and
 * receivers are in model-grid coordinates and must lie in the aperture. */
typedef struct {
  int x0, y0, z0;          /* aperture origin in the model grid (cells) */
  int nx, ny, nz;          /* aperture extent (cells) */
  int nt;                  /* record length of this shot (steps, >= 1) */
  int src_i, src_j, src_k; /* source cell */
  int rec_first, nrec;     /* its receivers: rows rec_first .. rec_first+nrec-1 of d_rec_ijk */
  long long wavelet_first; /* its nt source samples start at h_wavelets[wavelet_first] */
  long long obs_first;     /* its nt*nrec samples (time-major) start at d_obs[obs_first]
                              (likewise in d_rec_out and d_resid) */
} fwi_shot;

/* A batch plan owns everything the shots need on the device: per-shot
 * wavefields and model windows, the checkpoint arena (arena_bytes), the
 * launch configuration and, with FWI_BATCH_GRAPH, the CUDA graph of a whole
 * call, captured on first use and replayed while the call's device pointers
 * stay the same.  All shots advance together, one launch per time step
 * covering the tiles of every active shot; checkpoints follow pol (modes
 * FWI_CKPT_FULL and FWI_CKPT_EVERY_K) for each shot independently, and the
 * result of every shot equals that of a single-shot call on its aperture.
 *   g          model grid (nx, ny, nz), h, dt and absorbing layer; g->nt is unused
 *   h_shots    nshots shot descriptions (host, copied)
 *   d_rec_ijk  receiver cells (i,j,k) in model-grid coordinates, int32, used
 *              during this call only
 *   flags      FWI_BATCH_GRAPH and/or FWI_BATCH_TUNE (pick the tile depth and
 *              the persistent grid size by timing candidates on the plan's
 *              own fields, at the first call)
 * FWI_ERR_CAPACITY when pol stores raw fields that cannot fit in arena_bytes;
 * FWI_ERR_NOMEM when the working set does not fit on the device. */
#define FWI_BATCH_GRAPH 1
#define FWI_BATCH_TUNE 2
typedef struct fwi_batch fwi_batch;
int fwi_batch_create(const fwi_geometry* g, int nshots, const fwi_shot* h_shots, const int* d_rec_ijk,
                     const fwi_ckpt_policy* pol, size_t arena_bytes, int flags, fwi_batch** out);
int fwi_batch_destroy(fwi_batch* b);

/* Stacked gradient of all shots: d_grad (model grid) += sum over shots of
 * the shot's dPhi_s/dm placed at its aperture, in shot order;
 * h_misfit[s] = Phi_s (FP64).  d_m is the model (model grid), h_wavelets the
 * source samples, d_obs the observed records.  Synchronises.
 * FWI_ERR_CAPACITY if the compressed checkpoints overflow the arena. */
int fwi_batch_gradient(fwi_batch* b, const float* d_m, const float* h_wavelets, const float* d_obs,
                       float* d_grad, double* h_misfit, void* stream);
/* The two halves, as fwi_forward_store / fwi_adjoint_store for each shot:
 * the forward records (d_rec_out, laid out like d_obs) with the checkpoints
 * kept in the plan, then d_grad += sum_s J_s^T d_resid_s.  The adjoint call
 * needs a completed forward call on the same plan (FWI_ERR_ARG otherwise). */
int fwi_batch_forward(fwi_batch* b, const float* d_m, const float* h_wavelets, float* d_rec_out,
                      void* stream);
int fwi_batch_adjoint(fwi_batch* b, const float* d_m, const float* h_wavelets, const float* d_resid,
                      float* d_grad, void* stream);

/* Configuration and counters of a plan. */
typedef struct {
  int nshots;
  int max_nt;             /* longest record (steps) */
  int zc;                 /* tile depth (z planes per tile) of the forward kernel, 0 = per-shot automatic */
  int ctas;               /* CTAs of each persistent forward-stencil launch */
  int zc_adjoint;         /* the same for the adjoint kernel */
  int ctas_adjoint;
  int tuned;              /* 1 once the autotuner has run */
  int graph_nodes;        /* nodes of the last captured graph (0: none) */
  uint64_t launches_per_call; /* kernels one gradient call launches */
  size_t arena_bytes;
  size_t used_bytes;      /* checkpoint bytes of the last forward sweep */
  size_t raw_bytes;       /* the same checkpoints uncompressed */
  size_t device_bytes;    /* device memory the plan holds */
} fwi_batch_stats;
int fwi_batch_get_stats(const fwi_batch* b, fwi_batch_stats* out);

/* ---- failure detection ---------------------------------------------------- */
/* Every device-side wait of the library (TMA-completion barriers of the
 * stencil pipeline, look-back spins of the single-pass encoder) is bounded:
 * when it gives up, the kernel flags a timeout, waits (bounded) for its own
 * copies in flight and returns, and the call returns FWI_ERR_TIMEOUT with the
 * context still usable.  This self-test runs that path on purpose: one CTA
 * waits `polls` polls (1 .. 2^20) on a barrier nothing ever completes.  It
 * returns FWI_ERR_TIMEOUT when the bounded wait works (FWI_ERR_ARG for a bad
 * count).  Synchronises. */
int fwi_selftest_bounded_wait(long long polls, void* stream);

/* Self-test of the damping quotient of the leapfrog kernels (Sec. 2, Eq. (1)
 * with the absorbing layer: the update is divided by 1 + eta, eta >= 0):
 * d_out[i] = d_num[i] / d_den[i] computed exactly as the stencil kernels
 * compute it (reciprocal estimate, one Newton-Raphson step, remainder
 * correction), so that tests can compare it with IEEE division.  Device
 * arrays of n floats; d_den[i] must lie in [1, 2^126) and d_num[i] be
 * finite.  Returns FWI_ERR_ARG for n < 0 or a null pointer with n > 0.
 * Synchronises. */
int fwi_selftest_damped_quotient(const float* d_num, const float* d_den, float* d_out, long long n,
                                 void* stream);

/* ---- fixed-accuracy codec (Sec. 1.4) -------------------------------------- */
/* Stream format (shared bit-for-bit with the CPU oracle):
 *   64-byte header (magic "FCZ1", version, nx, ny, nz, minexp, nblocks,
 *   chunk size 32, nchunks, payload words, total bytes, format params),
 *   nchunks u64 chunk word offsets, nblocks u16 block bit lengths (padded to
 *   8 bytes), then the payload of u64 words.  Each 4x4x4 block (x fastest,
 *   blocks ordered x, y, z; edge blocks replicate the last plane) carries:
 *   1 flag bit, 8 bits of block exponent, then embedded bit planes of its 64
 *   negabinary transform coefficients.  With minexp = floor(log2 atol), every
 *   decoded value satisfies |x - x'| <= 2^minexp <= atol whenever the block's
 *   largest exponent is within 24 of minexp (tolerances coarser than FP32's
 *   own resolution of the block); otherwise |x - x'| < 2^(emax-24). */

/* Worst-case stream size (bytes) for an nx*ny*nz field; 0 on bad sizes. */
size_t zfp_max_compressed_bytes(int nx, int ny, int nz);

/* Compress d_in with tolerance atol > 0 into d_out (device, out_capacity
 * bytes, 8-byte aligned).  *h_out_bytes = stream size.  FWI_ERR_CAPACITY (with *h_out_bytes =
 * the size needed) if out_capacity is too small; FWI_ERR_NONFINITE if d_in
 * holds NaN or Inf.  Synchronises. */
int zfp_compress_fixed_accuracy(const float* d_in, int nx, int ny, int nz, double atol,
                                void* d_out, size_t out_capacity, size_t* h_out_bytes,
                                void* stream);

/* Decompress a stream of in_bytes bytes (d_in 8-byte aligned) into d_out.  FWI_ERR_CORRUPT for a
 * malformed stream (reads stay inside [d_in, d_in + in_bytes)), FWI_ERR_ARG
 * if its dimensions differ from nx, ny, nz.  Synchronises. */
int zfp_decompress(const void* d_in, size_t in_bytes, float* d_out, int nx, int ny, int nz,
                   void* stream);

/* Allocation-free variant of zfp_compress_fixed_accuracy, same arguments,
 * results and stream.  The paper has no counterpart: this exists for callers
 * that cannot allocate device memory mid-run (a solver that has given nearly
 * all free HBM to its checkpoint arena, or an application whose memory policy
 * forbids allocations after start-up).  The regular call takes its encoder
 * scratch from the stream-ordered pool; this one uses a fixed block of about
 * 1 MiB inside the library's device image, held on every GPU that loads the
 * library until exit, and calls no cudaMalloc, cudaMallocAsync, cudaFree or
 * allocating library routine.
 *   - Fields of more than 4,194,304 blocks of 4x4x4 (131,072 chunks of 32) are
 *     rejected with FWI_ERR_ARG before any device work.
 *   - All calls share the block and it keeps the last call's contents; each
 *     call clears what must start at zero.  Calls that overlap on the GPU
 *     (other streams or host threads) race on it.
 *   - The first call on a device looks up the block's address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.
 * Synchronises. */
int zfp_compress_fixed_accuracy_noalloc(const float* d_in, int nx, int ny, int nz, double atol,
                                        void* d_out, size_t out_capacity, size_t* h_out_bytes,
                                        void* stream);

/* ---- FP64 reductions ------------------------------------------------------ */
/* d_resid = d_sim - d_obs (may alias d_sim); *h_misfit = 1/2 sum resid^2 in
 * FP64 (Eq. (3)).  Synchronises. */
int fwi_misfit(const float* d_sim, const float* d_obs, size_t n, float* d_resid,
               double* h_misfit, void* stream);

/* *h_out = sum_i a_i b_i accumulated in FP64 (inner products of the adjoint
 * and Taylor tests and of the angle metric, Sec. 3.1).  Synchronises. */
int fwi_dot_f64(const float* d_a, const float* d_b, size_t n, double* h_out, void* stream);

/* ---- misc ----------------------------------------------------------------- */
const char* fwi_status_string(int status);
/* Number of kernels this library has launched since load (for accounting). */
uint64_t fwi_kernel_launch_count(void);

/* Per-kernel timing for roofline accounting.  While enabled, the library
 * records a CUDA event pair on the launching stream around every launch of
 * the timed classes (0 forward stencil, 1 adjoint stencil (imaging fused or not),
 * 2 codec encode, 3 codec decode, 4 everything else); read returns, per
 * class, the summed device milliseconds and launch count since the last
 * reset (it waits for recorded events).  n must be >= 5. */
int fwi_profile_enable(int on);
int fwi_profile_reset(void);
int fwi_profile_read(double* ms_out, uint64_t* launches_out, int n);

#ifdef __cplusplus
}
#endif
#endif
