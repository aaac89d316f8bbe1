/*
 * Oracle wave propagation, adjoint and checkpointed gradient -- TEST
 * INFRASTRUCTURE ONLY (see oracle.h).  FP64 throughout, plain loops.
 *
 * Discretisation (the paper fixes the PDE, Sec. 2 Eq. (1), but not its
 * discretisation; these are the readings this project takes):
 *   L u      8th-order central second differences per axis, zero outside
 *            the grid, so L is symmetric.
 *   damping  sigma(x) = m0(x) s(x) with s the absorbing-layer profile and
 *            m0 the model the layer was set up with (held fixed, i.e. not
 *            differentiated).
 *   time     m u_tt + sigma u_t - L u = P_s^T q, centred differences:
 *            a+ u^{n+1} = (2m/dt^2) u^n + L u^n - a- u^{n-1} + P_s^T q^n,
 *            a+- = m/dt^2 +- sigma/(2 dt),  n = 0..N-1,  u^0 = u^-1 = 0.
 *   data     d^n = P_r u^{n+1} (Eq. (2)).
 *   misfit   Phi = 1/2 sum_n |d^n - d_obs^n|^2 (Eq. (3)).
 *   adjoint  a+ l_{k-1} = (2m/dt^2) l_k + L l_k - a- l_{k+1} + P_r^T r^{k-1},
 *            k = N..1, l_N = l_{N+1} = 0: the exact transpose of the forward
 *            recurrence (the self-adjointness noted in Sec. 2).
 *   gradient dPhi/dm = -sum_{k=1}^{N} u^k (l_{k-1} - 2 l_k + l_{k+1}) / dt^2,
 *            the zero-lag correlation of u with the adjoint's second time
 *            difference (Eq. (4)), with the sign and dt factors that make it
 *            the exact derivative of the discrete Phi.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* 8th-order central coefficients of d^2/dx^2 (times h^2). */
static const double OC[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

void oracle_sponge_profile(int n, int nbl, double h, double vmax, double R, double* s) {
  double W = nbl * h;
  for (int i = 0; i < n; i++) {
    double d = 0.0;
    if (i < nbl) d = (nbl - i) * h;
    if (i > n - 1 - nbl) {
      double d2 = (i - (n - 1 - nbl)) * h;
      if (d2 > d) d = d2;
    }
    s[i] = (nbl > 0 && d > 0.0) ? (3.0 * vmax / (2.0 * W)) * log(1.0 / R) * (d / W) * (d / W) : 0.0;
  }
}

static double oc_at(const double* u, const oracle_geometry* g, long x, long y, long z) {
  if (x < 0 || y < 0 || z < 0 || x >= g->nx || y >= g->ny || z >= g->nz) return 0.0;
  return u[x + (long)g->nx * (y + (long)g->ny * z)];
}

void oracle_laplacian(const oracle_geometry* g, const double* u, double* Lu) {
  double ih2 = 1.0 / (g->h * g->h);
#pragma omp parallel for schedule(static)
  for (long z = 0; z < g->nz; z++)
    for (long y = 0; y < g->ny; y++)
      for (long x = 0; x < g->nx; x++) {
        double c = oc_at(u, g, x, y, z);
        double acc = 3.0 * OC[0] * c;
        for (int r = 1; r <= 4; r++) {
          acc += OC[r] * (oc_at(u, g, x + r, y, z) + oc_at(u, g, x - r, y, z));
          acc += OC[r] * (oc_at(u, g, x, y + r, z) + oc_at(u, g, x, y - r, z));
          acc += OC[r] * (oc_at(u, g, x, y, z + r) + oc_at(u, g, x, y, z - r));
        }
        Lu[x + (long)g->nx * (y + (long)g->ny * z)] = acc * ih2;
      }
}

/* sigma = m0 * (s_x + s_y + s_z) */
static void oc_sigma(const oracle_geometry* g, const double* m0, double* sig) {
  double* sx = (double*)malloc(sizeof(double) * g->nx);
  double* sy = (double*)malloc(sizeof(double) * g->ny);
  double* sz = (double*)malloc(sizeof(double) * g->nz);
  oracle_sponge_profile(g->nx, g->nbl, g->h, g->vmax, g->sponge_R, sx);
  oracle_sponge_profile(g->ny, g->nbl, g->h, g->vmax, g->sponge_R, sy);
  oracle_sponge_profile(g->nz, g->nbl, g->h, g->vmax, g->sponge_R, sz);
  for (long z = 0; z < g->nz; z++)
    for (long y = 0; y < g->ny; y++)
      for (long x = 0; x < g->nx; x++) {
        long i = x + (long)g->nx * (y + (long)g->ny * z);
        sig[i] = m0[i] * (sx[x] + sy[y] + sz[z]);
      }
  free(sx);
  free(sy);
  free(sz);
}

/* One step of the leapfrog recurrence:
 *   out = ((2m/dt^2) cur + L cur - a- prev + inj) / a+
 * where inj adds val[i] at cell[i].  out may alias prev. */
static void oc_step(const oracle_geometry* g, const double* m, const double* sig,
                    const double* cur, const double* prev, double* out, double* Lbuf,
                    const long* cell, const double* val, int ninj) {
  long C = (long)g->nx * g->ny * g->nz;
  double idt2 = 1.0 / (g->dt * g->dt);
  oracle_laplacian(g, cur, Lbuf);
  for (int i = 0; i < ninj; i++) Lbuf[cell[i]] += val[i];
#pragma omp parallel for schedule(static)
  for (long i = 0; i < C; i++) {
    double ap = m[i] * idt2 + sig[i] / (2.0 * g->dt);
    double am = m[i] * idt2 - sig[i] / (2.0 * g->dt);
    out[i] = (2.0 * m[i] * idt2 * cur[i] + Lbuf[i] - am * prev[i]) / ap;
  }
}

static int oc_check(const oracle_geometry* g) {
  if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->nt < 0 || !(g->h > 0) || !(g->dt > 0))
    return ORACLE_ERR_ARG;
  return 0;
}

static long oc_cell(const oracle_geometry* g, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) return -1;
  return i + (long)g->nx * (j + (long)g->ny * k);
}

int oracle_forward(const oracle_geometry* g, const double* m, const double* m0,
                   const double* wavelet, int si, int sj, int sk,
                   const int* rec_ijk, int nrec, double* rec_out,
                   const double* u_prev_init, const double* u_cur_init,
                   double* u_before_last, double* u_last) {
  if (oc_check(g)) return ORACLE_ERR_ARG;
  long C = (long)g->nx * g->ny * g->nz;
  long src = oc_cell(g, si, sj, sk);
  if (src < 0 || (nrec > 0 && (!rec_ijk || !rec_out))) return ORACLE_ERR_ARG;
  long* rc = (long*)malloc(sizeof(long) * (nrec > 0 ? nrec : 1));
  for (int r = 0; r < nrec; r++) {
    rc[r] = oc_cell(g, rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2]);
    if (rc[r] < 0) { free(rc); return ORACLE_ERR_ARG; }
  }
  double* sig = (double*)malloc(sizeof(double) * C);
  double* prev = (double*)calloc(C, sizeof(double));
  double* cur = (double*)calloc(C, sizeof(double));
  double* Lb = (double*)malloc(sizeof(double) * C);
  oc_sigma(g, m0 ? m0 : m, sig);
  if (u_prev_init) memcpy(prev, u_prev_init, sizeof(double) * C);
  if (u_cur_init) memcpy(cur, u_cur_init, sizeof(double) * C);
  for (int n = 0; n < g->nt; n++) {
    double q = wavelet[n];
    oc_step(g, m, sig, cur, prev, prev, Lb, &src, &q, 1); /* prev <- u^{n+1} */
    double* t = prev; prev = cur; cur = t;               /* cur = u^{n+1} */
    for (int r = 0; r < nrec; r++) rec_out[(long)n * nrec + r] = cur[rc[r]];
  }
  if (u_before_last) memcpy(u_before_last, prev, sizeof(double) * C);
  if (u_last) memcpy(u_last, cur, sizeof(double) * C);
  free(rc); free(sig); free(prev); free(cur); free(Lb);
  return 0;
}

int oracle_adjoint_trace(const oracle_geometry* g, const double* m, const double* m0,
                         const double* resid, const int* rec_ijk, int nrec,
                         int si, int sj, int sk, double* src_trace) {
  if (oc_check(g)) return ORACLE_ERR_ARG;
  long C = (long)g->nx * g->ny * g->nz;
  long src = oc_cell(g, si, sj, sk);
  if (src < 0) return ORACLE_ERR_ARG;
  long* rc = (long*)malloc(sizeof(long) * (nrec > 0 ? nrec : 1));
  for (int r = 0; r < nrec; r++) {
    rc[r] = oc_cell(g, rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2]);
    if (rc[r] < 0) { free(rc); return ORACLE_ERR_ARG; }
  }
  double* sig = (double*)malloc(sizeof(double) * C);
  double* lnext = (double*)calloc(C, sizeof(double)); /* l_{k+1} */
  double* lcur = (double*)calloc(C, sizeof(double));  /* l_k */
  double* Lb = (double*)malloc(sizeof(double) * C);
  oc_sigma(g, m0 ? m0 : m, sig);
  for (int k = g->nt; k >= 1; k--) {
    oc_step(g, m, sig, lcur, lnext, lnext, Lb, rc, resid + (long)(k - 1) * nrec, nrec);
    double* t = lnext; lnext = lcur; lcur = t; /* lcur = l_{k-1} */
    src_trace[k - 1] = lcur[src];
  }
  free(rc); free(sig); free(lnext); free(lcur); free(Lb);
  return 0;
}

/* ---- checkpoint schedule ------------------------------------------------ */

static void oc_emit(oracle_action* out, size_t cap, size_t* n, int kind, int step, int arg) {
  if (*n < cap && out) {
    out[*n].kind = kind;
    out[*n].step = step;
    out[*n].arg = arg;
  }
  (*n)++;
}

/* Binomial cost table cost[n][s], n = 0..N, s = 0..S (plain dynamic
 * programming over the split point). */
static long long* oc_binomial_table(int N, int S) {
  long long* c = (long long*)malloc(sizeof(long long) * (size_t)(N + 1) * (S + 1));
  for (int n = 0; n <= N; n++)
    for (int s = 0; s <= S; s++) {
      long long best = (long long)n * (n + 1) / 2;
      if (s > 0)
        for (int m = 1; m < n; m++) {
          long long v = m + c[(size_t)(n - m) * (S + 1) + (s - 1)] + c[(size_t)m * (S + 1) + s];
          if (v < best) best = v;
        }
      c[(size_t)n * (S + 1) + s] = best;
    }
  return c;
}

long long oracle_binomial_cost(int n, int s) {
  if (n < 0 || s < 0) return -1;
  long long* c = oc_binomial_table(n, s);
  long long v = c[(size_t)n * (s + 1) + s];
  free(c);
  return v;
}

typedef struct {
  oracle_action* out;
  size_t cap, n;
  const long long* cost;
  int S;
  int state;    /* step of the current forward state */
  int advanced; /* steps 0 .. advanced-1 have been run once (recorded) */
} oc_binom;

static void oc_advance_to(oc_binom* b, int target) {
  while (b->state < target) {
    int kind = b->state >= b->advanced ? ORACLE_ACT_ADVANCE : ORACLE_ACT_RECOMPUTE;
    oc_emit(b->out, b->cap, &b->n, kind, b->state, 0);
    b->state++;
    if (b->state > b->advanced) b->advanced = b->state;
  }
}

/* serve adjoint steps a+n .. a+1, the state at a being stored, s spare slots */
static void oc_binom_gen(oc_binom* b, int a, int n, int s) {
  if (n <= 0) return;
  long long base = (long long)n * (n + 1) / 2;
  int m_best = 0;
  if (s > 0) {
    long long best = base;
    for (int m = 1; m < n; m++) {
      long long v = m + b->cost[(size_t)(n - m) * (b->S + 1) + (s - 1)] + b->cost[(size_t)m * (b->S + 1) + s];
      if (v < best) {
        best = v;
        m_best = m;
      }
    }
  }
  if (m_best == 0) {
    for (int k = a + n; k > a; k--) {
      if (b->state != a) {
        oc_emit(b->out, b->cap, &b->n, ORACLE_ACT_RESTORE, a, 2);
        b->state = a;
      }
      oc_advance_to(b, k);
      oc_emit(b->out, b->cap, &b->n, ORACLE_ACT_ADJOINT, k, 0);
    }
    return;
  }
  if (b->state != a) {
    oc_emit(b->out, b->cap, &b->n, ORACLE_ACT_RESTORE, a, 2);
    b->state = a;
  }
  oc_advance_to(b, a + m_best);
  oc_emit(b->out, b->cap, &b->n, ORACLE_ACT_STORE, a + m_best, 2);
  oc_binom_gen(b, a + m_best, n - m_best, s - 1);
  oc_emit(b->out, b->cap, &b->n, ORACLE_ACT_FREE, a + m_best, 2);
  oc_binom_gen(b, a, m_best, s);
}

int oracle_ckpt_schedule(int nt, const oracle_policy* pol, oracle_action* out, size_t cap,
                         size_t* n_out) {
  if (!pol || nt < 0 || !n_out) return ORACLE_ERR_ARG;
  size_t n = 0;
  if (pol->mode == ORACLE_CKPT_FULL) {
    /* forward: advance and keep every state u^1..u^N */
    for (int s = 0; s < nt; s++) {
      oc_emit(out, cap, &n, ORACLE_ACT_ADVANCE, s, 0);
      oc_emit(out, cap, &n, ORACLE_ACT_STORE, s + 1, 1);
    }
    /* reverse: load u^k, adjoint step k */
    for (int k = nt; k >= 1; k--) {
      oc_emit(out, cap, &n, ORACLE_ACT_RESTORE, k, 1);
      oc_emit(out, cap, &n, ORACLE_ACT_ADJOINT, k, 0);
    }
  } else if (pol->mode == ORACLE_CKPT_EVERY_K) {
    int K = pol->k;
    if (K < 1) return ORACLE_ERR_ARG;
    /* forward: keep the state pair (u^{c-1}, u^c) at c = 0, K, 2K, ... <= N */
    oc_emit(out, cap, &n, ORACLE_ACT_STORE, 0, 2);
    for (int s = 0; s < nt; s++) {
      oc_emit(out, cap, &n, ORACLE_ACT_ADVANCE, s, 0);
      if ((s + 1) % K == 0) oc_emit(out, cap, &n, ORACLE_ACT_STORE, s + 1, 2);
    }
    /* reverse, one segment per checkpoint: restore, recompute the segment,
     * then the adjoint steps that need it */
    for (int c = (nt / K) * K; c >= 0; c -= K) {
      int e = c + K - 1 < nt ? c + K - 1 : nt;
      int lo = c > 1 ? c : 1;
      if (e < lo) continue;
      oc_emit(out, cap, &n, ORACLE_ACT_RESTORE, c, 2);
      for (int s = c; s < e; s++) oc_emit(out, cap, &n, ORACLE_ACT_RECOMPUTE, s, 0);
      for (int k = e; k >= lo; k--) oc_emit(out, cap, &n, ORACLE_ACT_ADJOINT, k, 0);
    }
  } else if (pol->mode == ORACLE_CKPT_SUBSAMPLE) {
    /* subsampled imaging (Sec. 4.7): states kept only at multiples of f */
    int f = pol->k;
    if (f < 1) return ORACLE_ERR_ARG;
    for (int s = 0; s < nt; s++) {
      oc_emit(out, cap, &n, ORACLE_ACT_ADVANCE, s, 0);
      if ((s + 1) % f == 0) oc_emit(out, cap, &n, ORACLE_ACT_STORE, s + 1, 1);
    }
    for (int k = nt; k >= 1; k--) {
      if (k % f == 0) {
        oc_emit(out, cap, &n, ORACLE_ACT_RESTORE, k, 1);
        oc_emit(out, cap, &n, ORACLE_ACT_ADJOINT, k, f);
      } else {
        oc_emit(out, cap, &n, ORACLE_ACT_ADJOINT, k, -1);
      }
    }
  } else if (pol->mode == ORACLE_CKPT_BINOMIAL) {
    if (pol->k < 0) return ORACLE_ERR_ARG;
    /* the zero state before the first step is the bottom snapshot */
    oc_emit(out, cap, &n, ORACLE_ACT_STORE, 0, 2);
    long long* cost = oc_binomial_table(nt, pol->k);
    oc_binom b = {out, cap, n, cost, pol->k, 0, 0};
    oc_binom_gen(&b, 0, nt, pol->k);
    n = b.n;
    free(cost);
  } else {
    return ORACLE_ERR_ARG;
  }
  *n_out = n;
  return (n > cap || !out) ? ORACLE_ERR_CAPACITY : 0;
}

/* ---- checkpointed gradient ---------------------------------------------- */

/* A stored field: raw FP64 copy, or a compressed FP32 copy. */
typedef struct {
  double* raw;
  uint8_t* z;
  size_t zbytes;
} oc_saved;

static int oc_save(const oracle_geometry* g, const double* f, double atol, oc_saved* s,
                   double* bytes) {
  long C = (long)g->nx * g->ny * g->nz;
  memset(s, 0, sizeof(*s));
  if (atol <= 0.0) {
    s->raw = (double*)malloc(sizeof(double) * C);
    memcpy(s->raw, f, sizeof(double) * C);
    *bytes += 4.0 * C; /* the GPU keeps raw checkpoints in FP32 */
    return 0;
  }
  float* tmp = (float*)malloc(sizeof(float) * C);
  for (long i = 0; i < C; i++) tmp[i] = (float)f[i];
  size_t cap = oracle_zfp_max_bytes(g->nx, g->ny, g->nz);
  uint8_t* buf = (uint8_t*)malloc(cap);
  size_t used = 0;
  int st = oracle_zfp_compress(tmp, g->nx, g->ny, g->nz, atol, buf, cap, &used);
  free(tmp);
  if (st) { free(buf); return st; }
  s->z = (uint8_t*)realloc(buf, used);
  s->zbytes = used;
  *bytes += (double)used;
  return 0;
}

static int oc_load(const oracle_geometry* g, const oc_saved* s, double* f) {
  long C = (long)g->nx * g->ny * g->nz;
  if (s->raw) {
    memcpy(f, s->raw, sizeof(double) * C);
    return 0;
  }
  if (!s->z) { /* never stored: the zero state before the first step */
    memset(f, 0, sizeof(double) * C);
    return 0;
  }
  float* tmp = (float*)malloc(sizeof(float) * C);
  int st = oracle_zfp_decompress(s->z, s->zbytes, tmp, g->nx, g->ny, g->nz);
  for (long i = 0; i < C && !st; i++) f[i] = (double)tmp[i];
  free(tmp);
  return st;
}

static void oc_free_saved(oc_saved* s) {
  free(s->raw);
  free(s->z);
  memset(s, 0, sizeof(*s));
}

int oracle_gradient(const oracle_geometry* g, const double* m, const double* m0,
                    const double* wavelet, int si, int sj, int sk,
                    const int* rec_ijk, int nrec, const double* d_obs,
                    const oracle_policy* pol, double* grad, double* misfit,
                    double* d_sim_out, double* ckpt_bytes_out) {
  if (oc_check(g) || !pol || !grad || !misfit) return ORACLE_ERR_ARG;
  int N = g->nt;
  long C = (long)g->nx * g->ny * g->nz;
  long src = oc_cell(g, si, sj, sk);
  if (src < 0 || nrec < 0) return ORACLE_ERR_ARG;
  long* rc = (long*)malloc(sizeof(long) * (nrec > 0 ? nrec : 1));
  for (int r = 0; r < nrec; r++) {
    rc[r] = oc_cell(g, rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2]);
    if (rc[r] < 0) { free(rc); return ORACLE_ERR_ARG; }
  }
  size_t nact = 0;
  int st = oracle_ckpt_schedule(N, pol, NULL, 0, &nact);
  if (st != ORACLE_ERR_CAPACITY && st != 0) { free(rc); return st; }
  oracle_action* act = (oracle_action*)malloc(sizeof(oracle_action) * (nact ? nact : 1));
  st = oracle_ckpt_schedule(N, pol, act, nact, &nact);

  double* sig = (double*)malloc(sizeof(double) * C);
  oc_sigma(g, m0 ? m0 : m, sig);
  double* Lb = (double*)malloc(sizeof(double) * C);
  double* prev = (double*)calloc(C, sizeof(double)); /* forward state u^{s-1} */
  double* cur = (double*)calloc(C, sizeof(double));  /* forward state u^s */
  int state_step = 0;
  double* dsim = (double*)calloc((size_t)N * (nrec > 0 ? nrec : 1), sizeof(double));
  double* resid = (double*)calloc((size_t)N * (nrec > 0 ? nrec : 1), sizeof(double));
  oc_saved* saved_cur = (oc_saved*)calloc((size_t)N + 1, sizeof(oc_saved));
  oc_saved* saved_prev = (oc_saved*)calloc((size_t)N + 1, sizeof(oc_saved));
  double** avail = (double**)calloc((size_t)N + 1, sizeof(double*)); /* u^k ready for imaging */
  double* lnext = (double*)calloc(C, sizeof(double)); /* l_{k+1} */
  double* lcur = (double*)calloc(C, sizeof(double));  /* l_k */
  double* lnew = (double*)malloc(sizeof(double) * C); /* l_{k-1} */
  double bytes = 0.0;
  int residual_ready = 0;
  double idt2 = 1.0 / (g->dt * g->dt);

  for (size_t a = 0; a < nact && !st; a++) {
    int kind = act[a].kind, s = act[a].step;
    if (kind == ORACLE_ACT_ADVANCE || kind == ORACLE_ACT_RECOMPUTE) {
      if (state_step != s) { st = ORACLE_ERR_ARG; break; }
      double q = wavelet[s];
      oc_step(g, m, sig, cur, prev, prev, Lb, &src, &q, 1);
      double* t = prev; prev = cur; cur = t;
      state_step = s + 1;
      if (kind == ORACLE_ACT_ADVANCE) {
        for (int r = 0; r < nrec; r++) dsim[(long)s * nrec + r] = cur[rc[r]];
      } else if (pol->mode != ORACLE_CKPT_BINOMIAL) {
        avail[s + 1] = (double*)malloc(sizeof(double) * C);
        memcpy(avail[s + 1], cur, sizeof(double) * C);
      }
    } else if (kind == ORACLE_ACT_STORE) {
      if (state_step != s) { st = ORACLE_ERR_ARG; break; }
      if (s > 0) {
        st = oc_save(g, cur, pol->atol, &saved_cur[s], &bytes);
        if (!st && act[a].arg == 2) st = oc_save(g, prev, pol->atol, &saved_prev[s], &bytes);
      }
    } else if (kind == ORACLE_ACT_RESTORE) {
      if (act[a].arg == 2) {
        st = oc_load(g, &saved_prev[s], prev);
        if (!st) st = oc_load(g, &saved_cur[s], cur);
        state_step = s;
      }
      if (!st && s >= 1 && pol->mode != ORACLE_CKPT_BINOMIAL) {
        avail[s] = (double*)malloc(sizeof(double) * C);
        st = oc_load(g, &saved_cur[s], avail[s]);
      }
    } else if (kind == ORACLE_ACT_FREE) {
      oc_free_saved(&saved_cur[s]);
      oc_free_saved(&saved_prev[s]);
    } else if (kind == ORACLE_ACT_ADJOINT) {
      int k = s;
      if (!residual_ready) {
        /* all data recorded: residual and misfit, Eq. (3) */
        double phi = 0.0;
        for (long i = 0; i < (long)N * nrec; i++) {
          resid[i] = dsim[i] - d_obs[i];
          phi += 0.5 * resid[i] * resid[i];
        }
        *misfit = phi;
        residual_ready = 1;
      }
      /* binomial schedules image with the current forward state; the
       * action's weight scales the imaging term (-1: none) */
      const int weight = act[a].arg == 0 ? 1 : act[a].arg;
      const double* uk = avail[k];
      if (pol->mode == ORACLE_CKPT_BINOMIAL) uk = state_step == k ? cur : NULL;
      if (!uk && weight > 0) { st = ORACLE_ERR_ARG; break; }
      oc_step(g, m, sig, lcur, lnext, lnew, Lb, rc, resid + (long)(k - 1) * nrec, nrec);
      if (weight > 0) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < C; i++) grad[i] -= weight * uk[i] * (lnew[i] - 2.0 * lcur[i] + lnext[i]) * idt2;
      }
      double* t = lnext; lnext = lcur; lcur = lnew; lnew = t;
      if (pol->mode != ORACLE_CKPT_BINOMIAL) {
        free(avail[k]);
        avail[k] = NULL;
      }
    }
  }
  if (!residual_ready && !st) { /* N = 0 */
    *misfit = 0.0;
  }
  if (d_sim_out && !st) memcpy(d_sim_out, dsim, sizeof(double) * (size_t)N * nrec);
  if (ckpt_bytes_out) *ckpt_bytes_out = bytes;
  for (int k = 0; k <= N; k++) {
    free(avail[k]);
    oc_free_saved(&saved_cur[k]);
    oc_free_saved(&saved_prev[k]);
  }
  free(avail); free(saved_cur); free(saved_prev);
  free(act); free(rc); free(sig); free(Lb); free(prev); free(cur);
  free(dsim); free(resid); free(lnext); free(lcur); free(lnew);
  return st;
}

int oracle_gradient_batch(const oracle_geometry* g, const double* m, int nshots,
                          const oracle_shot* shots, const double* wavelets,
                          const int* rec_ijk, const double* d_obs,
                          const oracle_policy* pol, double* grad, double* misfit) {
  if (oc_check(g) || !m || nshots < 0 || (nshots > 0 && (!shots || !wavelets)) || !pol || !grad ||
      !misfit)
    return ORACLE_ERR_ARG;
  for (int s = 0; s < nshots; s++) {
    const oracle_shot* sh = &shots[s];
    if (sh->nx < 1 || sh->ny < 1 || sh->nz < 1 || sh->x0 < 0 || sh->y0 < 0 || sh->z0 < 0 ||
        sh->x0 + sh->nx > g->nx || sh->y0 + sh->ny > g->ny || sh->z0 + sh->nz > g->nz ||
        sh->nt < 0 || sh->nrec < 0 || (sh->nrec > 0 && (!rec_ijk || !d_obs)))
      return ORACLE_ERR_ARG;
    /* the shot's own problem: its window of the model and local coordinates */
    oracle_geometry lg = *g;
    lg.nx = sh->nx;
    lg.ny = sh->ny;
    lg.nz = sh->nz;
    lg.nt = sh->nt;
    long C = (long)sh->nx * sh->ny * sh->nz;
    double* mw = (double*)malloc(sizeof(double) * C);
    double* gw = (double*)calloc(C, sizeof(double));
    int* rl = (int*)malloc(sizeof(int) * 3 * (sh->nrec > 0 ? sh->nrec : 1));
    for (int k = 0; k < sh->nz; k++)
      for (int j = 0; j < sh->ny; j++)
        for (int i = 0; i < sh->nx; i++)
          mw[i + (long)sh->nx * (j + (long)sh->ny * k)] =
              m[(sh->x0 + i) + (long)g->nx * ((sh->y0 + j) + (long)g->ny * (sh->z0 + k))];
    const int* rg = rec_ijk ? rec_ijk + 3L * sh->rec_first : NULL;
    for (int r = 0; r < sh->nrec; r++) {
      rl[3 * r] = rg[3 * r] - sh->x0;
      rl[3 * r + 1] = rg[3 * r + 1] - sh->y0;
      rl[3 * r + 2] = rg[3 * r + 2] - sh->z0;
    }
    int st = oracle_gradient(&lg, mw, NULL, wavelets + sh->wavelet_first, sh->src_i - sh->x0,
                             sh->src_j - sh->y0, sh->src_k - sh->z0, rl, sh->nrec,
                             d_obs ? d_obs + sh->obs_first : NULL, pol, gw, &misfit[s], NULL, NULL);
    if (!st)
      for (int k = 0; k < sh->nz; k++)
        for (int j = 0; j < sh->ny; j++)
          for (int i = 0; i < sh->nx; i++)
            grad[(sh->x0 + i) + (long)g->nx * ((sh->y0 + j) + (long)g->ny * (sh->z0 + k))] +=
                gw[i + (long)sh->nx * (j + (long)sh->ny * k)];
    free(mw);
    free(gw);
    free(rl);
    if (st) return st;
  }
  return ORACLE_OK;
}
