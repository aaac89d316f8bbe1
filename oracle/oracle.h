/*
 * Reference ("oracle") implementation of the checkpointed FWI gradient of
 * Kukreja et al., "Lossy Checkpoint Compression in Full Waveform Inversion".
 *
 * TEST INFRASTRUCTURE ONLY.  This library is a plain, slow, obviously correct
 * CPU restatement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path (the CUDA library and its Python binding) never does.  It shares no
 * code, header, table or constant generator with the CUDA sources.
 *
 * Precision: every wave-field, adjoint and gradient quantity is FP64.  The
 * codec takes FP32 input (the GPU stores FP32 wavefields) so that both sides
 * make every quantisation decision on identical bits.
 *
 * Sections of the paper this follows:
 *   Sec. 2, Eq. (1)  isotropic acoustic wave equation  m u_tt - lap(u) = q_s
 *   Sec. 2, Eq. (2)  d_sim = P_r A(m)^-1 P_s^T q_s
 *   Sec. 2, Eq. (3)  Phi_s(m) = 1/2 || d_sim - d_obs ||^2
 *   Sec. 2, Eq. (4)  grad Phi_s = sum_t u[t] v_tt[t]  (adjoint run backwards)
 *   Sec. 1.3         checkpointing (store / restore / recompute); exact
 *   Sec. 1.4, Fig. 1 lossy compression of every checkpoint (ZFP, fixed accuracy)
 *   Sec. 3           reference problem: 8 Hz Ricker, absorbing layer, dt
 *
 * Parity status of each function is stated beside it ("pinned by ..." names
 * the tests that tie it to something other than itself).
 */
#ifndef FWI_ORACLE_H
#define FWI_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (0 = success). */
#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_CAPACITY (-2)
#define ORACLE_ERR_CORRUPT (-3)
#define ORACLE_ERR_NONFINITE (-4)
#define ORACLE_ERR_NOMEM (-7)

/* Grid and time axis.  Fields are [nz][ny][nx], x fastest.  The nbl-cell
 * absorbing layer is part of the grid on all six faces. */
typedef struct {
  int nx, ny, nz;
  double h;        /* grid spacing, m */
  double dt;       /* time step, s */
  int nt;          /* number of time steps N */
  int nbl;         /* absorbing-layer width, cells */
  double sponge_R; /* target reflection coefficient of the layer */
  double vmax;     /* reference velocity of the damping profile, m/s */
} oracle_geometry;

/* Checkpoint policies (Sec. 1.3).  atol <= 0 stores raw copies; atol > 0
 * stores fixed-accuracy compressed FP32 copies (Sec. 1.4). */
#define ORACLE_CKPT_FULL 1    /* keep u^k for every k = 1..N */
#define ORACLE_CKPT_EVERY_K 2 /* keep (u^{c-1}, u^c) for c = 0, K, 2K, ... */
#define ORACLE_CKPT_BINOMIAL 3 /* at most k state pairs at a time, placed to minimise recomputation */
#define ORACLE_CKPT_SUBSAMPLE 4 /* keep u^k only for k = f, 2f, ...; image only there, weight f */
typedef struct {
  int mode;
  int k;
  double atol;
} oracle_policy;

/* Checkpoint-schedule actions (Sec. 1.3: forward, store, backward, load and
 * recompute events). */
#define ORACLE_ACT_ADVANCE 1 /* forward step: u^{step} -> u^{step+1}, recording data */
#define ORACLE_ACT_STORE 2   /* store checkpoint at step (arg = levels: 1 or 2) */
#define ORACLE_ACT_RESTORE 3 /* restore checkpoint at step */
#define ORACLE_ACT_RECOMPUTE 4 /* forward step without recording: u^{step} -> u^{step+1} */
#define ORACLE_ACT_ADJOINT 5 /* adjoint step k = step: lambda_{k-1}; imaging with u^k weighted by
                                arg (0 means 1; -1: no imaging) */
#define ORACLE_ACT_FREE 6    /* drop the most recent stored state (binomial schedules) */
typedef struct {
  int kind;
  int step;
  int arg;
} oracle_action;

/* ---- stencil and sweeps (FP64) ------------------------------------------ */

/* 1D damping-rate profile s(i), i = 0..n-1, in 1/s.  Zero outside the layer;
 * inside, (3 vmax / 2W) ln(1/R) (d/W)^2 with d the depth into the layer (m)
 * and W = nbl h.  Sec. 3 ("absorbing boundary layer"); the formula is this
 * library's reading (the paper gives none).  Pinned: tests check the profile's
 * closed-form values and that a wave leaving the grid is absorbed. */
void oracle_sponge_profile(int n, int nbl, double h, double vmax, double R, double* s);

/* Lu = 8th-order central Laplacian of u (homogeneous Dirichlet outside the
 * grid).  Discretises lap(u) of Eq. (1).  Pinned: exact on polynomials of
 * degree <= 9 per axis; h^8 convergence on smooth fields. */
void oracle_laplacian(const oracle_geometry* g, const double* u, double* Lu);

/* Forward sweep of Eq. (1)-(2): u^{n+1} for n = 0..N-1 from u^0 = u^-1 = 0
 * (or from the given initial pair), source q^n added at one cell, records
 * d^n = P_r u^{n+1}.  m0 is the model that weights the damping (NULL: m).
 * u_prev_init/u_cur_init (NULL: zero) start the sweep from a stored state.
 * u_last (optional) receives u^N, u_before_last (optional) u^{N-1}.
 * Pinned: homogeneous Green's function; dot-product test with the adjoint. */
int oracle_forward(const oracle_geometry* g, const double* m, const double* m0,
                   const double* wavelet, int si, int sj, int sk,
                   const int* rec_ijk, int nrec, double* rec_out,
                   const double* u_prev_init, const double* u_cur_init,
                   double* u_before_last, double* u_last);

/* Adjoint sweep (Sec. 2, "solving an adjoint equation backwards in time"):
 * lambda_{k-1} for k = N..1 with lambda_N = lambda_{N+1} = 0 and the data
 * residual injected at the receivers; returns lambda_n sampled at the
 * source cell, n = 0..N-1 (the transpose of the forward map q -> d).
 * Pinned: dot-product test <F q, d> = <q, F^T d>. */
int oracle_adjoint_trace(const oracle_geometry* g, const double* m, const double* m0,
                         const double* resid, const int* rec_ijk, int nrec,
                         int si, int sj, int sk, double* src_trace);

/* Checkpointed gradient, Eq. (3)-(4): misfit Phi = 1/2 sum (d_sim-d_obs)^2 and
 * grad += dPhi/dm (damping held fixed), with checkpoints stored per policy
 * (raw or compressed) and the forward state recomputed where the policy
 * requires.  d_sim_out (optional, N*nrec) receives the simulated data.
 * Pinned: Taylor test (second-order remainder), finite differences, every-K
 * raw store bit-identical to full history. */
int oracle_gradient(const oracle_geometry* g, const double* m, const double* m0,
                    const double* wavelet, int si, int sj, int sk,
                    const int* rec_ijk, int nrec, const double* d_obs,
                    const oracle_policy* pol, double* grad, double* misfit,
                    double* d_sim_out, double* ckpt_bytes_out);

/* One shot of a survey, modelled on its aperture: the nx*ny*nz window at
 * (x0, y0, z0) of the model grid, with the absorbing layer inside the
 * window.  Source and receivers are in model-grid coordinates; the shot's
 * nt source samples start at wavelets[wavelet_first], its nt*nrec observed
 * samples (time-major) at d_obs[obs_first], its receivers at row rec_first
 * of rec_ijk. */
typedef struct {
  int x0, y0, z0, nx, ny, nz;
  int nt;
  int src_i, src_j, src_k;
  int rec_first, nrec;
  long long wavelet_first, obs_first;
} oracle_shot;

/* Stacked gradient of a survey (Sec. 2: Phi = sum over shots of Eq. (3), so
 * its gradient is the sum of the shots' Eq. (4)): for every shot, the
 * gradient of oracle_gradient on the shot's window of m (damping weighted
 * by that window) is added into grad (the model grid) at the window, in shot
 * order; misfit[s] = Phi_s.  Pinned: one full-grid shot equals
 * oracle_gradient; translating a shot in a homogeneous model translates its
 * gradient; a finite-difference derivative of sum_s Phi_s on windows cut by
 * the test itself; shot order changes nothing beyond rounding. */
int oracle_gradient_batch(const oracle_geometry* g, const double* m, int nshots,
                          const oracle_shot* shots, const double* wavelets,
                          const int* rec_ijk, const double* d_obs,
                          const oracle_policy* pol, double* grad, double* misfit);

/* Checkpoint schedule for the policy: the ordered list of actions that
 * oracle_gradient executes.  Binomial: with the state at a stored and s more
 * snapshot slots, serving adjoint steps a+n .. a+1 costs
 *   cost(n, 0) = n(n+1)/2 (restart from a for every step),
 *   cost(n, s) = min(cost(n, 0), min_{0<m<n} m + cost(n-m, s-1) + cost(m, s)),
 * the recursive splitting of Sec. 1.3's Revolve-family schedules; the
 * smallest minimising m is taken.  Pinned: the table equals Griewank's
 * closed-form minimum and the schedule's raw result equals full history. */
long long oracle_binomial_cost(int n, int s);
/* Returns ORACLE_ERR_CAPACITY (and the needed count in *n_out) when cap is
 * too small. */
int oracle_ckpt_schedule(int nt, const oracle_policy* pol, oracle_action* out,
                         size_t cap, size_t* n_out);

/* ---- fixed-accuracy block codec (Sec. 1.4; format defined by this project) */

/* Worst-case stream size in bytes for an nx*ny*nz field. */
size_t oracle_zfp_max_bytes(int nx, int ny, int nz);

/* Compress an FP32 field [nz][ny][nx] with absolute tolerance atol > 0.
 * Returns ORACLE_ERR_CAPACITY with *out_bytes = required size if cap is too
 * small, ORACLE_ERR_NONFINITE on NaN/Inf input. */
int oracle_zfp_compress(const float* in, int nx, int ny, int nz, double atol,
                        uint8_t* out, size_t cap, size_t* out_bytes);

/* Decompress a stream made by oracle_zfp_compress (or by the GPU encoder,
 * which writes the identical format).  ORACLE_ERR_CORRUPT on malformed input
 * (never reads outside [in, in+in_bytes)). */
int oracle_zfp_decompress(const uint8_t* in, size_t in_bytes, float* out,
                          int nx, int ny, int nz);

/* Single-block building blocks, exported for the pins. */
int oracle_zfp_minexp(double atol);
/* Encode one 4x4x4 block (x fastest) into bits[] (LSB-first 64-bit words);
 * returns the bit count or a negative status. */
int oracle_zfp_encode_block(const float v[64], int minexp, uint64_t* bits, int nwords);
/* Decode one block from bits[]; returns bits consumed or a negative status. */
int oracle_zfp_decode_block(const uint64_t* bits, int nbits, int minexp, float v[64]);
/* Forward / inverse integer lifting transform of a block (in place, int32). */
void oracle_zfp_fwd_xform(int32_t q[64]);
void oracle_zfp_inv_xform(int32_t q[64]);
/* 1D 4-point lifting pair, for the exhaustive invertibility pin. */
void oracle_zfp_fwd_lift4(int32_t* p, int stride);
void oracle_zfp_inv_lift4(int32_t* p, int stride);
/* Coefficient order: perm[p] = block index of the p-th coded coefficient. */
void oracle_zfp_perm(int perm[64]);
/* Block-floating-point integers of a block and its coded-plane count. */
int oracle_zfp_block_quantise(const float v[64], int minexp, int32_t q[64], int* emax, int* planes);

/* Number of OpenMP threads the oracle uses. */
int oracle_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
