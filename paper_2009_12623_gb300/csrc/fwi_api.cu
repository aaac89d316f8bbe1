// C-ABI entry points of libfwi (declared in include/fwi.h): checkpoint store,
// checkpoint schedule, forward modelling, the checkpointed gradient of
// Kukreja et al. (Sec. 2 Eq. (2)-(4), Sec. 1.3-1.4, Fig. 1), the codec calls
// and the FP64 reductions.  Host code here only validates arguments, owns
// memory and sequences the kernels of stencil.cu and codec.cu on the caller's
// stream; every arithmetic step of the path runs on the GPU.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "runtime.cuh"

namespace fwi {

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// ---- per-kernel timing: event pairs recorded around launches ---------------
namespace {
struct ProfSlot {
  int cls;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfSlot> g_prof_slots;   // recorded, not yet read
std::vector<cudaEvent_t> g_prof_free;  // reusable events
double g_prof_ms[KC_COUNT] = {0};
unsigned long long g_prof_n[KC_COUNT] = {0};

cudaEvent_t prof_event() {
  if (!g_prof_free.empty()) {
    cudaEvent_t e = g_prof_free.back();
    g_prof_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Fold completed slots into the totals (caller holds the lock).
void prof_drain(bool wait) {
  size_t keep = 0;
  for (size_t i = 0; i < g_prof_slots.size(); ++i) {
    ProfSlot& p = g_prof_slots[i];
    if (wait) cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_prof_ms[p.cls] += ms;
      g_prof_n[p.cls] += 1;
      g_prof_free.push_back(p.a);
      g_prof_free.push_back(p.b);
    } else {
      cudaGetLastError();
      g_prof_slots[keep++] = p;
    }
  }
  g_prof_slots.resize(keep);
}
}  // namespace

int prof_begin(int cls, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return -1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return -1;  // launches inside a CUDA graph are not timed one by one
  }
  if (g_prof_slots.size() > 4096) prof_drain(false);
  cudaEvent_t a = prof_event(), b = prof_event();
  if (!a || !b) return -1;
  cudaEventRecord(a, s);
  g_prof_slots.push_back(ProfSlot{cls, a, b});
  return (int)g_prof_slots.size() - 1;
}

void prof_end(int slot, cudaStream_t s) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < (int)g_prof_slots.size()) cudaEventRecord(g_prof_slots[slot].b, s);
}

int status_from_flags(int f) {
  if (f & ST_CAPACITY) return FWI_ERR_CAPACITY;
  if (f & ST_NONFINITE) return FWI_ERR_NONFINITE;
  if (f & ST_CORRUPT) return FWI_ERR_CORRUPT;
  if (f & ST_TIMEOUT) return FWI_ERR_TIMEOUT;
  return FWI_OK;
}

namespace {

// Everything the sweeps need on the device.
struct Sweep {
  Grid G;
  StencilParams sp;
  float* d_wavelet = nullptr;
  long src = -1;
  long* rec_cell = nullptr;
  float* rec_fac = nullptr;
  int* d_status = nullptr;
};

int setup_sweep(Pool& pool, const fwi_geometry* g, const float* d_m, const float* h_wavelet,
                int si, int sj, int sk, const int* d_rec_ijk, int nrec, Sweep& sw) {
  cudaStream_t s = pool.s;
  sw.G = Grid{g->nx, g->ny, g->nz, round_up(g->nx, 4)};
  sw.sp.g = sw.G;
  for (int r = 0; r < 5; ++r) sw.sp.c[r] = (float)(kC[r] / (g->h * g->h));
  sw.sp.dt = (float)g->dt;
  float* b = pool.get<float>(sw.G.cells());
  float* sx = pool.get<float>(g->nx);
  float* sy = pool.get<float>(g->ny);
  float* sz = pool.get<float>(g->nz);
  sw.d_wavelet = pool.get<float>(g->nt > 0 ? g->nt : 1);
  sw.rec_cell = pool.get<long>(nrec > 0 ? nrec : 1);
  sw.rec_fac = pool.get<float>(nrec > 0 ? nrec : 1);
  sw.d_status = pool.get<int>(1);
  if (pool.failed) return FWI_ERR_NOMEM;
  sw.sp.b = b;
  sw.sp.sx = sx;
  sw.sp.sy = sy;
  sw.sp.sz = sz;
  sw.sp.status = sw.d_status;
  CK(cudaMemsetAsync(sw.d_status, 0, sizeof(int), s));
  if (g->nt > 0) CK(cudaMemcpyAsync(sw.d_wavelet, h_wavelet, sizeof(float) * g->nt, cudaMemcpyHostToDevice, s));
  CK(setup_model_launch(d_m, sw.G, (float)g->dt, b, sw.d_status, s));
  CK(setup_profiles_launch(sw.G, g->nbl, g->h, g->vmax, g->sponge_R, g->dt, sx, sy, sz, s));
  CK(rec_cells_launch(d_rec_ijk, nrec, sw.G, sw.rec_cell, sw.d_status, s));
  CK(rec_fac_launch(sw.sp, sw.rec_cell, nrec, sw.rec_fac, s));
  sw.src = (long)si + (long)sw.G.pitch * ((long)sj + (long)g->ny * sk);
  return FWI_OK;
}

bool in_grid(const fwi_geometry* g, int i, int j, int k) {
  return i >= 0 && j >= 0 && k >= 0 && i < g->nx && j < g->ny && k < g->nz;
}

// Schedule generator: the event list of Sec. 1.3 for the two policies.
struct Sched {
  std::vector<fwi_action> a;
  void add(int kind, int step, int arg) { a.push_back(fwi_action{kind, step, arg}); }
};

// Binomial checkpointing.  With the state at step a stored and s further
// snapshot slots, serving adjoint steps a+n .. a+1 needs at least
//   cost(n, s) = n + t(n, s+1)
// forward steps, t(l, S) = r l - C(S+r, S+1) being Griewank's minimum for l
// steps and S snapshots (r: the smallest r with C(S+r, S) >= l).  A split at
// m costs m + cost(n-m, s-1) + cost(m, s); the smallest optimal m is used,
// and with no spare slot every adjoint step restarts from a.  A stored state
// is restored only when the current forward state is not already at a, so
// data are always recorded from the exact first pass.
struct Binomial {
  Sched& out;
  int state = 0;     // step of the current forward state
  int advanced = 0;  // steps 0 .. advanced-1 ran once (recorded)
  Binomial(Sched& o, int) : out(o) {}

  static long long choose_capped(int n, int k, long long cap) {  // C(n, k), capped at cap + 1
    if (k < 0 || k > n) return 0;
    long long c = 1;
    for (int i = 1; i <= k; ++i) {
      c = c * (n - k + i) / i;
      if (c > cap) return cap + 1;
    }
    return c;
  }
  static long long cost(int n, int s) {
    if (n <= 0) return 0;
    const int S = s + 1;
    int r = 0;
    while (choose_capped(S + r, S, n) < n) ++r;
    // C(S+r, S+1) = C(S+r, r-1), a product of r-1 terms (exact at each step)
    long long c = r >= 1 ? 1 : 0;
    for (int i = 1; i <= r - 1; ++i) c = c * (S + 1 + i) / i;
    return (long long)n + (long long)r * n - c;
  }
  void advance_to(int target) {
    while (state < target) {
      out.add(state >= advanced ? FWI_ACT_ADVANCE : FWI_ACT_RECOMPUTE, state, 0);
      ++state;
      if (state > advanced) advanced = state;
    }
  }
  void restore(int a) {
    if (state != a) {
      out.add(FWI_ACT_RESTORE, a, 2);
      state = a;
    }
  }
  void reverse(int a, int n, int s) {
    if (n <= 0) return;
    int m_best = 0;
    if (s > 0) {
      long long best = (long long)n * (n + 1) / 2;
      for (int m = 1; m < n; ++m) {
        const long long v = m + cost(n - m, s - 1) + cost(m, s);
        if (v < best) {
          best = v;
          m_best = m;
        }
      }
    }
    if (m_best == 0) {
      for (int k = a + n; k > a; --k) {
        restore(a);
        advance_to(k);
        out.add(FWI_ACT_ADJOINT, k, 0);
      }
      return;
    }
    restore(a);
    advance_to(a + m_best);
    out.add(FWI_ACT_STORE, a + m_best, 2);
    reverse(a + m_best, n - m_best, s - 1);
    out.add(FWI_ACT_FREE, a + m_best, 2);
    reverse(a, m_best, s);
  }
};

int make_schedule(int nt, const fwi_ckpt_policy* pol, Sched& out) {
  if (!pol || nt < 0) return FWI_ERR_ARG;
  if (pol->mode == FWI_CKPT_FULL) {
    for (int s = 0; s < nt; ++s) {
      out.add(FWI_ACT_ADVANCE, s, 0);
      out.add(FWI_ACT_STORE, s + 1, 1);
    }
    for (int k = nt; k > 0; --k) {
      out.add(FWI_ACT_RESTORE, k, 1);
      out.add(FWI_ACT_ADJOINT, k, 0);
    }
    return FWI_OK;
  }
  if (pol->mode == FWI_CKPT_EVERY_K) {
    const int K = pol->k_or_snaps;
    if (K < 1) return FWI_ERR_ARG;
    out.add(FWI_ACT_STORE, 0, 2);
    for (int s = 1; s <= nt; ++s) {
      out.add(FWI_ACT_ADVANCE, s - 1, 0);
      if (s % K == 0) out.add(FWI_ACT_STORE, s, 2);
    }
    // segments [c, min(c+K-1, nt)] from the last checkpoint back to 0
    for (int c = nt - nt % K; c >= 0; c -= K) {
      const int last = std::min(c + K - 1, nt);
      const int first = std::max(c, 1);
      if (last < first) continue;
      out.add(FWI_ACT_RESTORE, c, 2);
      for (int s = c; s < last; ++s) out.add(FWI_ACT_RECOMPUTE, s, 0);
      for (int k = last; k >= first; --k) out.add(FWI_ACT_ADJOINT, k, 0);
    }
    return FWI_OK;
  }
  if (pol->mode == FWI_CKPT_SUBSAMPLE) {  // imaging every f-th step only (Sec. 4.7)
    const int f = pol->k_or_snaps;
    if (f < 1) return FWI_ERR_ARG;
    for (int s = 0; s < nt; ++s) {
      out.add(FWI_ACT_ADVANCE, s, 0);
      if ((s + 1) % f == 0) out.add(FWI_ACT_STORE, s + 1, 1);
    }
    for (int k = nt; k > 0; --k) {
      if (k % f == 0) {
        out.add(FWI_ACT_RESTORE, k, 1);
        out.add(FWI_ACT_ADJOINT, k, f);
      } else {
        out.add(FWI_ACT_ADJOINT, k, -1);
      }
    }
    return FWI_OK;
  }
  if (pol->mode == FWI_CKPT_BINOMIAL) {
    if (pol->k_or_snaps < 0) return FWI_ERR_ARG;
    out.add(FWI_ACT_STORE, 0, 2);  // the zero state before the first step
    Binomial b(out, pol->k_or_snaps);
    b.reverse(0, nt, pol->k_or_snaps);
    return FWI_OK;
  }
  return FWI_ERR_ARG;
}

}  // namespace

__global__ void k_slot_offset(unsigned long long* off, const unsigned long long* size, int j) {
  off[j] = j == 0 ? 0ull : off[j - 1] + ((size[j - 1] + 255ull) & ~255ull);
}
__global__ void k_track_peak(const unsigned long long* off, const unsigned long long* size, int j,
                             unsigned long long* peak) {
  const unsigned long long e = off[j] + ((size[j] + 255ull) & ~255ull);
  if (e > *peak) *peak = e;
}
cudaError_t slot_offset_launch(unsigned long long* off, const unsigned long long* size, int j,
                               cudaStream_t s) {
  k_slot_offset<<<1, 1, 0, s>>>(off, size, j);
  count_launch();
  return cudaGetLastError();
}
cudaError_t track_peak_launch(const unsigned long long* off, const unsigned long long* size, int j,
                              unsigned long long* peak, cudaStream_t s) {
  k_track_peak<<<1, 1, 0, s>>>(off, size, j, peak);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fwi

using namespace fwi;


extern "C" {

const char* fwi_status_string(int st) {
  switch (st) {
    case FWI_OK: return "ok";
    case FWI_ERR_ARG: return "invalid argument";
    case FWI_ERR_CAPACITY: return "capacity exceeded";
    case FWI_ERR_CORRUPT: return "corrupt compressed stream";
    case FWI_ERR_NONFINITE: return "non-finite value";
    case FWI_ERR_CUDA: return "CUDA runtime error";
    case FWI_ERR_TIMEOUT: return "device wait timed out";
    case FWI_ERR_NOMEM: return "device allocation failed";
    default: return "unknown status";
  }
}

uint64_t fwi_kernel_launch_count(void) { return g_launches.load(); }

int fwi_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return FWI_OK;
}

int fwi_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain(true);
  for (int i = 0; i < KC_COUNT; ++i) {
    g_prof_ms[i] = 0.0;
    g_prof_n[i] = 0;
  }
  return FWI_OK;
}

int fwi_profile_read(double* ms_out, uint64_t* launches_out, int n) {
  if (!ms_out || !launches_out || n < KC_COUNT) return FWI_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain(true);
  for (int i = 0; i < KC_COUNT; ++i) {
    ms_out[i] = g_prof_ms[i];
    launches_out[i] = g_prof_n[i];
  }
  return FWI_OK;
}

int fwi_ckpt_schedule(int nt, const fwi_ckpt_policy* pol, fwi_action* out, size_t cap,
                      size_t* n_out) {
  if (!n_out) return FWI_ERR_ARG;
  Sched sc;
  int st = make_schedule(nt, pol, sc);
  if (st) return st;
  *n_out = sc.a.size();
  if (!out || cap < sc.a.size()) return FWI_ERR_CAPACITY;
  memcpy(out, sc.a.data(), sizeof(fwi_action) * sc.a.size());
  return FWI_OK;
}

int fwi_ckpt_store_create(size_t capacity_bytes, fwi_ckpt_store** out) {
  if (!out || capacity_bytes == 0) return FWI_ERR_ARG;
  fwi_ckpt_store* st = new fwi_ckpt_store();
  if (cudaMalloc(&st->arena, capacity_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete st;
    return FWI_ERR_NOMEM;
  }
  st->capacity = capacity_bytes;
  st->stats.capacity_bytes = capacity_bytes;
  *out = st;
  return FWI_OK;
}

int fwi_ckpt_store_destroy(fwi_ckpt_store* st) {
  if (!st) return FWI_ERR_ARG;
  if (st->arena) cudaFree(st->arena);
  if (st->d_offs) cudaFree(st->d_offs);
  if (st->carry) cudaFree(st->carry);
  delete st;
  return FWI_OK;
}

int fwi_ckpt_store_stats(const fwi_ckpt_store* st, fwi_store_stats* out) {
  if (!st || !out) return FWI_ERR_ARG;
  *out = st->stats;
  return FWI_OK;
}

int fwi_ckpt_store_slot_bytes(const fwi_ckpt_store* st, unsigned long long* h_bytes, int cap, int* n_out) {
  if (!st || !n_out || cap < 0 || (cap > 0 && !h_bytes)) return FWI_ERR_ARG;
  const int n = st->filled ? st->nslots : 0;
  *n_out = n;
  const int k = std::min(n, cap);
  if (k == 0) return FWI_OK;
  if (!st->lossy) {
    const unsigned long long field = (unsigned long long)st->geom.nx * st->geom.ny * st->geom.nz * 4ull;
    for (int i = 0; i < k; ++i) h_bytes[i] = field;
    return FWI_OK;
  }
  if (!st->d_offs || st->slot_cap < n ||
      cudaMemcpy(h_bytes, st->d_offs + st->slot_cap, sizeof(unsigned long long) * (size_t)k,
                 cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return FWI_ERR_CUDA;
  }
  return FWI_OK;
}

int fwi_ckpt_store_slot_zero_blocks(const fwi_ckpt_store* st, unsigned long long* h_counts, int cap,
                                    int* n_out) {
  if (!st || !n_out || cap < 0 || (cap > 0 && !h_counts)) return FWI_ERR_ARG;
  const int n = st->filled ? st->nslots : 0;
  *n_out = n;
  const int k = std::min(n, cap);
  if (k == 0) return FWI_OK;
  if (!st->lossy) {
    for (int i = 0; i < k; ++i) h_counts[i] = 0;
    return FWI_OK;
  }
  if (!st->d_offs || st->slot_cap < n) return FWI_ERR_CUDA;
  const Grid G{st->geom.nx, st->geom.ny, st->geom.nz, round_up(st->geom.nx, 4)};
  unsigned long long* d_counts = nullptr;
  const size_t bytes = sizeof(unsigned long long) * (size_t)k;
  if (cudaMalloc(&d_counts, bytes) != cudaSuccess) {
    cudaGetLastError();
    return FWI_ERR_NOMEM;
  }
  const bool ok = zfp_count_zero_blocks_launch(st->arena, st->d_offs, k, st->capacity, G, d_counts, 0) ==
                      cudaSuccess &&
                  cudaMemcpy(h_counts, d_counts, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d_counts);
  if (!ok) {
    cudaGetLastError();
    return FWI_ERR_CUDA;
  }
  return FWI_OK;
}

int fwi_forward(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i,
                int src_j, int src_k, const int* d_rec_ijk, int nrec, float* d_rec_out,
                const float* d_u_prev_init, const float* d_u_cur_init, float* d_u_prev_out,
                float* d_u_last_out, void* stream) {
  if (!geometry_ok(g) || !d_m || (g->nt > 0 && !h_wavelet) || nrec < 0 ||
      (nrec > 0 && (!d_rec_ijk || !d_rec_out)) || !in_grid(g, src_i, src_j, src_k))
    return FWI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Pool pool(s);
  Sweep sw;
  int st = setup_sweep(pool, g, d_m, h_wavelet, src_i, src_j, src_k, d_rec_ijk, nrec, sw);
  if (st) return st;
  float* prev = pool.get<float>(sw.G.cells());
  float* cur = pool.get<float>(sw.G.cells());
  if (pool.failed) return FWI_ERR_NOMEM;
  CK(cudaMemsetAsync(prev, 0, sw.G.cells() * 4, s));
  CK(cudaMemsetAsync(cur, 0, sw.G.cells() * 4, s));
  if (d_u_prev_init) CK(unpack_launch(d_u_prev_init, sw.G, prev, s));
  if (d_u_cur_init) CK(unpack_launch(d_u_cur_init, sw.G, cur, s));
  for (int n = 0; n < g->nt; ++n) {
    CK(stencil_step_launch(sw.sp, cur, prev, prev, sw.src, sw.d_wavelet, n, s));
    std::swap(prev, cur);
    CK(gather_launch(cur, sw.rec_cell, nrec, d_rec_out + (size_t)n * nrec, s));
  }
  if (d_u_prev_out) CK(pack_launch(prev, sw.G, d_u_prev_out, s));
  if (d_u_last_out) CK(pack_launch(cur, sw.G, d_u_last_out, s));
  int flags = 0;
  CK(cudaMemcpyAsync(&flags, sw.d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flags & ST_CORRUPT) return FWI_ERR_ARG;  // receiver outside the grid
  return status_from_flags(flags);
}

}  // extern "C"

namespace {

enum { PH_FWD = 1, PH_REV = 2 };

bool same_run(const fwi_geometry& a, const fwi_geometry& b, const fwi_ckpt_policy& p,
              const fwi_ckpt_policy& q) {
  return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.h == b.h && a.dt == b.dt && a.nt == b.nt &&
         a.nbl == b.nbl && a.sponge_R == b.sponge_R && a.vmax == b.vmax && p.mode == q.mode &&
         p.k_or_snaps == q.k_or_snaps && p.atol == q.atol;
}

// The checkpointed sweeps.  PH_FWD: forward sweep recording data (into
// d_rec_out, or an internal buffer) and storing checkpoints per the policy.
// PH_REV: reverse sweep from the store's checkpoints with the adjoint source
// d_resid (or, when both phases run, the residual d_sim - d_obs, whose misfit
// goes to *h_misfit), accumulating d_grad += dPhi/dm.
int run_sweeps(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i, int src_j,
               int src_k, const int* d_rec_ijk, int nrec, float* d_rec_out, const float* d_obs,
               const float* d_resid, float* d_grad, double* h_misfit, fwi_ckpt_store* store,
               const fwi_ckpt_policy* pol, void* stream, int phases) {
  const bool do_fwd = phases & PH_FWD, do_rev = phases & PH_REV;
  if (!geometry_ok(g) || !d_m || (g->nt > 0 && !h_wavelet) || nrec < 0 ||
      (nrec > 0 && !d_rec_ijk) || !store || !pol || !in_grid(g, src_i, src_j, src_k))
    return FWI_ERR_ARG;
  if (do_rev && !d_grad) return FWI_ERR_ARG;
  if (do_fwd && do_rev && nrec > 0 && (!d_obs || !h_misfit)) return FWI_ERR_ARG;
  if (!do_fwd && do_rev && nrec > 0 && !d_resid) return FWI_ERR_ARG;
  if (do_fwd && !do_rev && nrec > 0 && !d_rec_out) return FWI_ERR_ARG;
  if (!do_fwd && (!store->filled || !same_run(store->geom, *g, store->pol, *pol))) return FWI_ERR_ARG;
  Sched sc;
  int st = make_schedule(g->nt, pol, sc);
  if (st) return st;
  const bool lossy = pol->atol > 0.0;
  if (lossy && !isfinite(pol->atol)) return FWI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Pool pool(s);
  Sweep sw;
  st = setup_sweep(pool, g, d_m, h_wavelet, src_i, src_j, src_k, d_rec_ijk, nrec, sw);
  if (st) return st;
  const Grid G = sw.G;
  const size_t fbytes = G.cells() * sizeof(float);
  const int N = g->nt;

  // slot numbering: (step, level) -> slot; level 1 = u^step, 0 = u^{step-1}
  std::map<std::pair<int, int>, int> slot;
  for (const fwi_action& a : sc.a)
    if (a.kind == FWI_ACT_STORE && a.step > 0) {
      const int j = (int)slot.size();
      slot[{a.step, 1}] = j;
      if (a.arg == 2) slot[{a.step, 0}] = j + 1;
    }
  const bool binom = pol->mode == FWI_CKPT_BINOMIAL;
  const int nslots = binom ? 2 * pol->k_or_snaps : (int)slot.size();
  const size_t raw_slot = (fbytes + 255) / 256 * 256;
  // forward phase: the actions before the first one that is neither ADVANCE nor STORE
  size_t first_rev = sc.a.size();
  for (size_t i = 0; i < sc.a.size(); ++i)
    if (sc.a[i].kind != FWI_ACT_ADVANCE && sc.a[i].kind != FWI_ACT_STORE) {
      first_rev = i;
      break;
    }
  if (do_fwd) {
    store->filled = false;
    store->stats = fwi_store_stats{store->capacity, 0, (size_t)nslots * (size_t)G.nx * G.ny * G.nz * 4,
                                   nslots, 0};
  }
  if (!lossy && (size_t)nslots * raw_slot > store->capacity) {
    store->stats.used_bytes = (size_t)nslots * raw_slot;
    store->stats.overflowed = 1;
    return FWI_ERR_CAPACITY;
  }

  float* fprev = pool.get<float>(G.cells());
  float* fcur = pool.get<float>(G.cells());
  float* lnext = pool.get<float>(G.cells());
  float* lcur = pool.get<float>(G.cells());
  float* gacc = pool.get<float>(G.cells());
  float* dsim = (do_fwd && do_rev) || !d_rec_out ? pool.get<float>((size_t)N * (nrec > 0 ? nrec : 1)) : d_rec_out;
  double* d_phi = pool.get<double>(1);
  double* d_part = pool.get<double>(reduce_scratch_doubles());
  if (store->slot_cap < nslots + 1) {
    if (store->d_offs) cudaFree(store->d_offs);
    store->d_offs = nullptr;
    store->slot_cap = 0;
    if (cudaMalloc(&store->d_offs, sizeof(unsigned long long) * (2 * (nslots + 1) + 1)) != cudaSuccess) {
      cudaGetLastError();
      return FWI_ERR_NOMEM;
    }
    store->slot_cap = nslots + 1;
  }
  unsigned long long* offs = store->d_offs;
  unsigned long long* sizes = store->d_offs + store->slot_cap;
  unsigned long long* d_peak = store->d_offs + 2 * store->slot_cap;  // largest arena end so far
  // binomial schedules also store snapshots during the reverse sweep
  const bool encodes = lossy && (do_fwd || binom);
  void* scratch = encodes ? (void*)pool.get<unsigned char>(zfp_encode_scratch_bytes(G.nx, G.ny, G.nz)) : nullptr;
  const int K = pol->mode == FWI_CKPT_EVERY_K ? pol->k_or_snaps : 1;
  std::vector<float*> ring(K, nullptr);
  for (int i = 0; i < K; ++i) ring[i] = pool.get<float>(G.cells());
  float* rprev = pool.get<float>(G.cells());
  if (pool.failed) return FWI_ERR_NOMEM;
  for (float* f : {fprev, fcur, lnext, lcur, gacc, rprev}) CK(cudaMemsetAsync(f, 0, fbytes, s));
  CK(cudaMemsetAsync(d_phi, 0, sizeof(double), s));
  if (do_fwd) CK(cudaMemsetAsync(sizes, 0, sizeof(unsigned long long) * (store->slot_cap + 1), s));
  if (do_fwd) CK(cudaMemsetAsync(d_peak, 0, sizeof(unsigned long long), s));
  const int minexp = lossy ? minexp_of(pol->atol) : 0;

  // Encoding runs on a second stream so that compressing u^{n+1} overlaps
  // the next stencil step (which only reads that buffer); decoding u^{k-1}
  // runs in order before adjoint step k (kDecodeOverlap).  Per-buffer events
  // order every overwrite after the codec reads or writes that buffer.
  CodecStream cs(s);
  if (!cs.ok) return FWI_ERR_CUDA;
  s = cs.main;  // the sweep's own stream from here on
  const cudaStream_t enc_s = cs.s;
  const cudaStream_t dec_s = kDecodeOverlap ? cs.s : s;
  auto store_field = [&](const float* f, int j, const LiveMap* live = nullptr) -> int {
    if (lossy) {
      CK(slot_offset_launch(offs, sizes, j, enc_s));
      CK(zfp_encode_launch(f, G, minexp, store->arena, offs + j, store->capacity, sizes + j,
                           sw.d_status, scratch, enc_s, live));
      CK(track_peak_launch(offs, sizes, j, d_peak, enc_s));
    } else {
      CK(cudaMemcpyAsync(store->arena + (size_t)j * raw_slot, f, fbytes, cudaMemcpyDeviceToDevice, enc_s));
    }
    return FWI_OK;
  };
  auto load_field = [&](int j, float* f, cudaStream_t st) -> int {
    if (lossy) {
      CK(zfp_decode_launch(store->arena, offs + j, store->capacity, f, G, sw.d_status, st));
    } else {
      CK(cudaMemcpyAsync(f, store->arena + (size_t)j * raw_slot, fbytes, cudaMemcpyDeviceToDevice, st));
    }
    return FWI_OK;
  };
  // forward-state buffers: "encoded" events guard their reuse
  float* fbuf[2] = {fprev, fcur};
  cudaEvent_t f_read[2] = {cs.ev[0], cs.ev[1]};
  bool f_pending[2] = {false, false};
  auto fidx = [&](const float* p) { return p == fbuf[0] ? 0 : 1; };
  // Full-history compressed sweeps: each forward step also records which
  // blocks of the state it writes reach the tolerance's last coded plane
  // (one liveness map per state buffer, reused with it), and the encoder
  // codes the other blocks as zero without reading them.  Every stored state
  // of these schedules comes from a forward step of the same sweep.
  const bool live_maps = lossy && do_fwd && (pol->mode == FWI_CKPT_FULL || pol->mode == FWI_CKPT_SUBSAMPLE) &&
                         live_threshold(minexp) > 0.0f;
  LiveMap lmap[2] = {};
  if (live_maps) {
    for (int i = 0; i < 2; ++i) {
      lmap[i].words = pool.get<uint16_t>(live_map_words(G));
      lmap[i].threshold = live_threshold(minexp);
      lmap[i].ntx = (G.pitch + 63) / 64;
      lmap[i].nby = (G.ny + 3) / 4;
    }
    if (pool.failed) return FWI_ERR_NOMEM;
  }
  auto live_of = [&](const float* f) -> const LiveMap* { return live_maps ? &lmap[fidx(f)] : nullptr; };
  // full-history decode double buffer
  float* dbuf[2] = {rprev, ring[0]};
  cudaEvent_t d_ready[2] = {cs.ev[2], cs.ev[3]}, d_used[2] = {cs.ev[4], cs.ev[5]};
  bool d_issued[2] = {false, false}, d_inuse[2] = {false, false};
  int d_step[2] = {-1, -1};
  const bool full = pol->mode == FWI_CKPT_FULL || pol->mode == FWI_CKPT_SUBSAMPLE;
  // Full-history compressed reverse sweeps image in the decoder: the adjoint
  // step becomes a plain step into a third lambda buffer (lambda_{k+1} stays
  // readable), then the decoder of u^k images its blocks that are not coded
  // as zero (one-bit blocks decode to exactly 0, so their imaging term is
  // exactly zero); the receiver injection skips those blocks too.
  const bool image_in_decoder = full && lossy && do_rev;
  float* lthird = nullptr;
  uint8_t* rec_block = nullptr;
  if (image_in_decoder) {
    const ZLayout ZL = zlayout(G.nx, G.ny, G.nz);
    lthird = pool.get<float>(G.cells());
    rec_block = pool.get<uint8_t>((size_t)ZL.nblocks);
    if (pool.failed) return FWI_ERR_NOMEM;
    CK(cudaMemsetAsync(lthird, 0, fbytes, s));
    CK(receiver_blocks_launch(sw.rec_cell, nrec, G, rec_block, s));
  }
  const float idt2 = 1.0f / (sw.sp.dt * sw.sp.dt);  // as the adjoint stencil forms it
  int next_buf = 0;
  auto issue_decode = [&](int k) -> int {  // u^k into the next decode buffer, on dec_s
    const int b = next_buf;
    next_buf ^= 1;
    // in order on the sweep's stream: first wait for every encode issued so
    // far (the state may have been stored moments ago)
    if (!kDecodeOverlap) CK(cs.join());
    if (d_inuse[b]) CK(cudaStreamWaitEvent(dec_s, d_used[b], 0));
    if ((st = load_field(slot[{k, 1}], dbuf[b], dec_s))) return st;
    CK(cudaEventRecord(d_ready[b], dec_s));
    d_issued[b] = true;
    d_step[b] = k;
    return FWI_OK;
  };
  cudaEvent_t ev_adv = cs.ev[6];

  std::vector<float*> avail(N + 2, nullptr);
  int seg_c = 0;
  bool resid_ready = false;
  int state_step = 0;          // step of the forward state held in (fprev, fcur)
  std::vector<int> bstack;     // binomial: steps of the stored pairs, bottom first
  auto bslot = [&](int depth, int level) { return 2 * depth + (level ? 0 : 1); };
  if (binom && !do_fwd) {
    // the reverse half starts where the forward half stopped: rebuild the
    // snapshot stack and bring back the final state pair
    for (size_t i = 0; i < first_rev; ++i)
      if (sc.a[i].kind == FWI_ACT_STORE && sc.a[i].step > 0) bstack.push_back(sc.a[i].step);
    if (!store->carry || store->carry_bytes < 2 * fbytes) return FWI_ERR_ARG;
    CK(cudaMemcpyAsync(fprev, store->carry, fbytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(fcur, (uint8_t*)store->carry + fbytes, fbytes, cudaMemcpyDeviceToDevice, s));
    state_step = N;
  }
  PhaseRange phase;
  for (size_t ai = 0; ai < sc.a.size(); ++ai) {
    const fwi_action& a = sc.a[ai];
    if ((ai < first_rev && !do_fwd) || (ai >= first_rev && !do_rev)) continue;
    if (ai == first_rev && do_fwd && !do_rev && binom) break;
    phase.enter(ai < first_rev ? kPhaseForward : kPhaseReverse);
    switch (a.kind) {
      case FWI_ACT_ADVANCE:
      case FWI_ACT_RECOMPUTE: {
        if (a.kind == FWI_ACT_RECOMPUTE && !binom) {  // every-K: segment ring
          const int i = a.step - seg_c;
          const float* prev = i == 0 ? rprev : ring[i - 1];
          CK(stencil_step_launch(sw.sp, ring[i], prev, ring[i + 1], sw.src, sw.d_wavelet, a.step, s));
          avail[a.step + 1] = ring[i + 1];
          break;
        }
        if (state_step != a.step) return FWI_ERR_ARG;
        const int w = fidx(fprev);  // the step overwrites fprev (and its liveness map)
        if (f_pending[w]) CK(cudaStreamWaitEvent(s, f_read[w], 0));
        f_pending[w] = false;
        CK(stencil_step_launch(sw.sp, fcur, fprev, fprev, sw.src, sw.d_wavelet, a.step, s, live_of(fprev)));
        std::swap(fprev, fcur);
        state_step = a.step + 1;
        if (a.kind == FWI_ACT_ADVANCE)
          CK(gather_launch(fcur, sw.rec_cell, nrec, dsim + (size_t)a.step * nrec, s));
        break;
      }
      case FWI_ACT_STORE:
        if (a.step > 0) {
          if (state_step != a.step) return FWI_ERR_ARG;
          CK(cudaEventRecord(ev_adv, s));
          CK(cudaStreamWaitEvent(enc_s, ev_adv, 0));
          const int j1 = binom ? bslot((int)bstack.size(), 1) : slot[{a.step, 1}];
          const int j0 = binom ? bslot((int)bstack.size(), 0) : (a.arg == 2 ? slot[{a.step, 0}] : -1);
          if ((st = store_field(fcur, j1, live_of(fcur)))) return st;
          if (a.arg == 2 && (st = store_field(fprev, j0))) return st;
          CK(cudaEventRecord(f_read[fidx(fcur)], enc_s));
          f_pending[fidx(fcur)] = true;
          if (a.arg == 2) {
            CK(cudaEventRecord(f_read[fidx(fprev)], enc_s));
            f_pending[fidx(fprev)] = true;
          }
          if (binom) bstack.push_back(a.step);
        }
        break;
      case FWI_ACT_FREE:
        if (!binom || bstack.empty() || bstack.back() != a.step) return FWI_ERR_ARG;
        CK(cs.join());  // the slot's next user must not overtake the encode
        bstack.pop_back();
        break;
      case FWI_ACT_RESTORE:
        if (a.arg == 1 && image_in_decoder) break;  // decoded (and imaged) by its adjoint step
        if (a.arg == 1) {  // single state u^k (decoded ahead on the codec stream)
          if (!(d_issued[0] && d_step[0] == a.step) && !(d_issued[1] && d_step[1] == a.step)) {
            if ((st = issue_decode(a.step))) return st;
          }
        } else if (binom) {  // the top snapshot pair becomes the forward state
          CK(cs.join());
          f_pending[0] = f_pending[1] = false;
          if (a.step == 0) {
            if (!bstack.empty()) return FWI_ERR_ARG;
            CK(cudaMemsetAsync(fprev, 0, fbytes, s));
            CK(cudaMemsetAsync(fcur, 0, fbytes, s));
          } else {
            if (bstack.empty() || bstack.back() != a.step) return FWI_ERR_ARG;
            const int d = (int)bstack.size() - 1;
            if ((st = load_field(bslot(d, 0), fprev, s))) return st;
            if ((st = load_field(bslot(d, 1), fcur, s))) return st;
          }
          state_step = a.step;
        } else {           // every-K: state pair at the segment start (on the main stream)
          CK(cs.join());
          seg_c = a.step;
          if (a.step == 0) {
            CK(cudaMemsetAsync(rprev, 0, fbytes, s));
            CK(cudaMemsetAsync(ring[0], 0, fbytes, s));
          } else {
            if ((st = load_field(slot[{a.step, 0}], rprev, s))) return st;
            if ((st = load_field(slot[{a.step, 1}], ring[0], s))) return st;
          }
          avail[a.step] = ring[0];
        }
        break;
      case FWI_ACT_ADJOINT: {
        const int k = a.step;
        const int weight = a.arg == 0 ? 1 : a.arg;
        if (!resid_ready) {
          CK(cs.join());  // every checkpoint of the first pass is stored
          if (do_fwd) CK(misfit_launch(dsim, d_obs, (size_t)N * nrec, dsim, d_phi, d_part, s));
          resid_ready = true;
        }
        const float* resid = do_fwd ? dsim : d_resid;
        if (weight < 0) {  // adjoint step without imaging (subsampled schedules)
          CK(stencil_step_launch(sw.sp, lcur, lnext, lnext, -1, sw.d_wavelet, 0, s));
          CK(inject_adjoint_launch(sw.sp, sw.rec_cell, sw.rec_fac, nrec, resid + (size_t)(k - 1) * nrec,
                                   lnext, nullptr, gacc, 0.f, s));
          std::swap(lcur, lnext);
          break;
        }
        if (image_in_decoder) {
          const int j = slot[{k, 1}];
          const ZeroBlocks zb = zero_blocks(store->arena, offs + j, store->capacity, G);
          CK(stencil_adjoint_step_launch(sw.sp, lcur, lnext, lthird, s));  // lambda_{k-1}
          ImageArgs im;
          im.lp = lthird;
          im.lc = lcur;
          im.ln = lnext;
          im.g = gacc;
          im.idt2 = idt2 * (float)weight;
          im.rec_block = rec_block;
          CK(zfp_decode_image_launch(store->arena, offs + j, store->capacity, dbuf[0], G, sw.d_status, im, s));
          CK(inject_adjoint_launch(sw.sp, sw.rec_cell, sw.rec_fac, nrec, resid + (size_t)(k - 1) * nrec,
                                   lthird, dbuf[0], gacc, (float)weight, s, &zb));
          float* t = lnext;  // lambda_{k+1} <- lambda_k <- lambda_{k-1}
          lnext = lcur;
          lcur = lthird;
          lthird = t;
          avail[k] = nullptr;
          break;
        }
        const float* uk = avail[k];
        int b = -1;
        if (full) {
          b = (d_issued[0] && d_step[0] == k) ? 0 : ((d_issued[1] && d_step[1] == k) ? 1 : -1);
          if (b < 0) return FWI_ERR_ARG;
          CK(cudaStreamWaitEvent(s, d_ready[b], 0));
          uk = dbuf[b];
          // decode the next stored state while this step runs
          for (size_t nx = ai + 1; nx < sc.a.size(); ++nx)
            if (sc.a[nx].kind == FWI_ACT_RESTORE) {
              if ((st = issue_decode(sc.a[nx].step))) return st;
              break;
            }
        } else if (binom) {
          uk = state_step == k ? fcur : nullptr;
        }
        if (!uk) return FWI_ERR_ARG;
        CK(stencil_adjoint_launch(sw.sp, lcur, lnext, lnext, uk, gacc, (float)weight, s));
        CK(inject_adjoint_launch(sw.sp, sw.rec_cell, sw.rec_fac, nrec, resid + (size_t)(k - 1) * nrec,
                                 lnext, uk, gacc, (float)weight, s));
        if (full) {
          CK(cudaEventRecord(d_used[b], s));
          d_inuse[b] = true;
        }
        std::swap(lcur, lnext);  // lcur = l_{k-1}, lnext = l_k
        avail[k] = nullptr;
        break;
      }
      default:
        return FWI_ERR_ARG;
    }
  }
  if (binom && do_fwd && !do_rev) {
    // keep the final forward state pair for the reverse half
    if (store->carry_bytes < 2 * fbytes) {
      if (store->carry) cudaFree(store->carry);
      store->carry = nullptr;
      store->carry_bytes = 0;
      if (cudaMalloc(&store->carry, 2 * fbytes) != cudaSuccess) {
        cudaGetLastError();
        return FWI_ERR_NOMEM;
      }
      store->carry_bytes = 2 * fbytes;
    }
    CK(cudaMemcpyAsync(store->carry, fprev, fbytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync((uint8_t*)store->carry + fbytes, fcur, fbytes, cudaMemcpyDeviceToDevice, s));
  }
  CK(cs.join());
  unsigned long long* d_end = d_peak;
  int flags = 0;
  double phi = 0.0;
  unsigned long long used = lossy ? 0ull : (unsigned long long)nslots * raw_slot;
  CK(cudaMemcpyAsync(&flags, sw.d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&phi, d_phi, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (lossy && do_fwd) CK(cudaMemcpyAsync(&used, d_end, sizeof(used), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (do_fwd) {
    store->stats.used_bytes = (size_t)used;
    store->stats.overflowed = (flags & ST_CAPACITY) ? 1 : 0;
  }
  if (flags) {
    if ((flags & ST_CORRUPT) && !(flags & ST_CAPACITY) && !(flags & ST_NONFINITE)) {
      // an out-of-range receiver also raises this flag during setup
      return FWI_ERR_ARG;
    }
    return status_from_flags(flags);
  }
  if (do_fwd) {
    store->filled = true;
    store->geom = *g;
    store->pol = *pol;
    store->nslots = nslots;
    store->lossy = lossy;
  }
  // a binomial reverse half reuses the snapshot slots of the forward half,
  // so the store no longer holds that forward sweep
  if (binom && do_rev && !do_fwd) store->filled = false;
  if (do_rev) {
    CK(unpack_add_launch(gacc, G, d_grad, s));
    CK(cudaStreamSynchronize(s));
  }
  if (do_fwd && do_rev && h_misfit) *h_misfit = phi;
  return FWI_OK;
}

}  // namespace

extern "C" {

int fwi_gradient(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i,
                 int src_j, int src_k, const int* d_rec_ijk, int nrec, const float* d_obs,
                 float* d_grad, double* h_misfit, fwi_ckpt_store* store,
                 const fwi_ckpt_policy* pol, void* stream) {
  if (!h_misfit || !d_grad) return FWI_ERR_ARG;
  return run_sweeps(g, d_m, h_wavelet, src_i, src_j, src_k, d_rec_ijk, nrec, nullptr, d_obs, nullptr,
                    d_grad, h_misfit, store, pol, stream, PH_FWD | PH_REV);
}

int fwi_forward_store(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i,
                      int src_j, int src_k, const int* d_rec_ijk, int nrec, float* d_rec_out,
                      fwi_ckpt_store* store, const fwi_ckpt_policy* pol, void* stream) {
  return run_sweeps(g, d_m, h_wavelet, src_i, src_j, src_k, d_rec_ijk, nrec, d_rec_out, nullptr, nullptr,
                    nullptr, nullptr, store, pol, stream, PH_FWD);
}

int fwi_adjoint_store(const fwi_geometry* g, const float* d_m, const float* h_wavelet, int src_i,
                      int src_j, int src_k, const int* d_rec_ijk, int nrec, const float* d_resid,
                      float* d_grad, fwi_ckpt_store* store, const fwi_ckpt_policy* pol, void* stream) {
  return run_sweeps(g, d_m, h_wavelet, src_i, src_j, src_k, d_rec_ijk, nrec, nullptr, nullptr, d_resid,
                    d_grad, nullptr, store, pol, stream, PH_REV);
}

int fwi_gradient_host(const fwi_geometry* g, const float* h_m, const float* h_wavelet, int src_i,
                      int src_j, int src_k, const int* h_rec_ijk, int nrec, const float* h_obs,
                      float* h_grad, double* h_misfit, fwi_ckpt_store* st,
                      const fwi_ckpt_policy* pol, void* stream) {
  if (!geometry_ok(g) || !h_m || !h_grad || !h_misfit || nrec < 0 || (nrec > 0 && (!h_rec_ijk || !h_obs)))
    return FWI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t C = (size_t)g->nx * g->ny * g->nz;
  const size_t nobs = (size_t)g->nt * nrec;
  float *dm = nullptr, *dobs = nullptr, *dgrad = nullptr, *drecs = nullptr;
  int* drec = nullptr;
  double* dphi = nullptr;
  double* dpart = nullptr;
  cudaStream_t cp = nullptr;
  cudaEvent_t ready = nullptr;
  int rc = FWI_OK;
  if (cudaMallocAsync(&dm, C * 4, s) != cudaSuccess || cudaMallocAsync(&dgrad, C * 4, s) != cudaSuccess ||
      cudaMallocAsync(&dobs, (nobs ? nobs : 1) * 4, s) != cudaSuccess ||
      cudaMallocAsync(&drecs, (nobs ? nobs : 1) * 4, s) != cudaSuccess ||
      cudaMallocAsync(&drec, (nrec ? nrec : 1) * 12, s) != cudaSuccess ||
      cudaMallocAsync(&dphi, sizeof(double), s) != cudaSuccess ||
      cudaMallocAsync(&dpart, reduce_scratch_doubles() * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    rc = FWI_ERR_NOMEM;
  }
  // the model and receivers are needed first; the observed data and the
  // incoming gradient only after the forward sweep, so they travel on a
  // copy stream while it runs
  if (!rc && (cudaStreamCreateWithFlags(&cp, cudaStreamNonBlocking) != cudaSuccess ||
              cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
              cudaEventRecord(ready, s) != cudaSuccess || cudaStreamWaitEvent(cp, ready, 0) != cudaSuccess))
    rc = FWI_ERR_CUDA;
  if (!rc && (cudaMemcpyAsync(dm, h_m, C * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
              (nrec && cudaMemcpyAsync(drec, h_rec_ijk, (size_t)nrec * 12, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
              cudaMemsetAsync(dphi, 0, sizeof(double), s) != cudaSuccess ||
              cudaMemcpyAsync(dgrad, h_grad, C * 4, cudaMemcpyHostToDevice, cp) != cudaSuccess ||
              (nobs && cudaMemcpyAsync(dobs, h_obs, nobs * 4, cudaMemcpyHostToDevice, cp) != cudaSuccess) ||
              cudaEventRecord(ready, cp) != cudaSuccess))
    rc = FWI_ERR_CUDA;
  if (!rc) rc = fwi_forward_store(g, dm, h_wavelet, src_i, src_j, src_k, drec, nrec, drecs, st, pol, stream);
  double phi = 0.0;
  if (!rc && (cudaStreamWaitEvent(s, ready, 0) != cudaSuccess ||
              misfit_launch(drecs, dobs, nobs, drecs, dphi, dpart, s) != cudaSuccess ||
              cudaMemcpyAsync(&phi, dphi, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess))
    rc = FWI_ERR_CUDA;
  if (!rc) rc = fwi_adjoint_store(g, dm, h_wavelet, src_i, src_j, src_k, drec, nrec, drecs, dgrad, st, pol,
                                  stream);
  if (!rc && (cudaMemcpyAsync(h_grad, dgrad, C * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
    rc = FWI_ERR_CUDA;
  if (!rc) *h_misfit = phi;
  if (cp) {
    cudaStreamSynchronize(cp);
    cudaStreamDestroy(cp);
  }
  if (ready) cudaEventDestroy(ready);
  for (void* p : {(void*)dm, (void*)dobs, (void*)dgrad, (void*)drec, (void*)drecs, (void*)dphi, (void*)dpart})
    if (p) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  cudaGetLastError();
  return rc;
}

int fwi_selftest_bounded_wait(long long polls, void* stream) {
  if (polls < 1 || polls > (1LL << 20)) return FWI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int* d_status = nullptr;
  if (cudaMallocAsync(&d_status, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return FWI_ERR_NOMEM;
  }
  int flags = 0;
  int rc = FWI_OK;
  if (cudaMemsetAsync(d_status, 0, sizeof(int), s) != cudaSuccess ||
      wait_selftest_launch(d_status, (long)polls, s) != cudaSuccess ||
      cudaMemcpyAsync(&flags, d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    rc = FWI_ERR_CUDA;
  cudaFreeAsync(d_status, s);
  cudaStreamSynchronize(s);
  cudaGetLastError();
  return rc ? rc : status_from_flags(flags);
}

int fwi_selftest_damped_quotient(const float* d_num, const float* d_den, float* d_out, long long n,
                                 void* stream) {
  if (n < 0 || (n > 0 && (!d_num || !d_den || !d_out))) return FWI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (quotient_selftest_launch(d_num, d_den, d_out, (long)n, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FWI_ERR_CUDA;
  }
  return FWI_OK;
}

size_t zfp_max_compressed_bytes(int nx, int ny, int nz) {
  if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
  return zlayout(nx, ny, nz).max_bytes;
}

int zfp_compress_fixed_accuracy(const float* d_in, int nx, int ny, int nz, double atol, void* d_out,
                                size_t out_capacity, size_t* h_out_bytes, void* stream) {
  if (!d_in || !d_out || !h_out_bytes || nx <= 0 || ny <= 0 || nz <= 0 || !(atol > 0.0) ||
      !isfinite(atol) || ((uintptr_t)d_out & 7) || ((uintptr_t)d_in & 3))
    return FWI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Pool pool(s);
  void* scratch = pool.get<unsigned char>(zfp_encode_scratch_bytes(nx, ny, nz));
  unsigned long long* d_size = pool.get<unsigned long long>(1);
  int* d_status = pool.get<int>(1);
  if (pool.failed) return FWI_ERR_NOMEM;
  CK(cudaMemsetAsync(d_status, 0, sizeof(int), s));
  CK(zfp_encode_launch(d_in, Grid{nx, ny, nz, nx}, minexp_of(atol), (uint8_t*)d_out, nullptr,
                       out_capacity, d_size, d_status, scratch, s));
  unsigned long long size = 0;
  int flags = 0;
  CK(cudaMemcpyAsync(&size, d_size, sizeof(size), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&flags, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *h_out_bytes = (size_t)size;
  return status_from_flags(flags);
}

int zfp_decompress(const void* d_in, size_t in_bytes, float* d_out, int nx, int ny, int nz,
                   void* stream) {
  if (!d_in || !d_out || nx <= 0 || ny <= 0 || nz <= 0 || ((uintptr_t)d_in & 7) ||
      ((uintptr_t)d_out & 3))
    return FWI_ERR_ARG;
  if (in_bytes < 64) return FWI_ERR_CORRUPT;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t hdr[16];
  CK(cudaMemcpyAsync(hdr, d_in, 64, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hdr[0] != ZC_MAGIC || hdr[1] != ZC_VERSION) return FWI_ERR_CORRUPT;
  if ((int)hdr[2] != nx || (int)hdr[3] != ny || (int)hdr[4] != nz) return FWI_ERR_ARG;
  Pool pool(s);
  int* d_status = pool.get<int>(1);
  if (pool.failed) return FWI_ERR_NOMEM;
  CK(cudaMemsetAsync(d_status, 0, sizeof(int), s));
  CK(zfp_decode_launch((const uint8_t*)d_in, nullptr, in_bytes, d_out, Grid{nx, ny, nz, nx}, d_status, s));
  int flags = 0;
  CK(cudaMemcpyAsync(&flags, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return status_from_flags(flags);
}

int fwi_misfit(const float* d_sim, const float* d_obs, size_t n, float* d_resid, double* h_misfit,
               void* stream) {
  if (!h_misfit || (n > 0 && (!d_sim || !d_obs || !d_resid))) return FWI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Pool pool(s);
  double* acc = pool.get<double>(1);
  double* part = pool.get<double>(reduce_scratch_doubles());
  if (pool.failed) return FWI_ERR_NOMEM;
  CK(cudaMemsetAsync(acc, 0, sizeof(double), s));
  CK(misfit_launch(d_sim, d_obs, n, d_resid, acc, part, s));
  CK(cudaMemcpyAsync(h_misfit, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return FWI_OK;
}

int fwi_dot_f64(const float* d_a, const float* d_b, size_t n, double* h_out, void* stream) {
  if (!h_out || (n > 0 && (!d_a || !d_b))) return FWI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Pool pool(s);
  double* acc = pool.get<double>(1);
  double* part = pool.get<double>(reduce_scratch_doubles());
  if (pool.failed) return FWI_ERR_NOMEM;
  CK(cudaMemsetAsync(acc, 0, sizeof(double), s));
  CK(dot_launch(d_a, d_b, n, acc, part, s));
  CK(cudaMemcpyAsync(h_out, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return FWI_OK;
}

}  // extern "C"
