// Batched shots (declared in include/fwi.h): the misfit of a survey and its
// gradient are sums over shots (Kukreja et al., Sec. 2, Eq. (3)-(4)), and
// every shot is modelled on its own aperture of the model (Sec. 3).  A plan
// holds the working set of all shots on the device and advances them
// together: one persistent stencil launch per time step covers the tiles of
// every active shot, one launch samples (or injects at) the receivers of all
// of them, and the checkpoints of each shot follow the policy exactly as a
// single-shot call on the aperture would, so the stacked result equals the
// sum of single-shot gradients bit for bit.
//
// Alignment of shots with different record lengths: the forward sweeps all
// start at step 0 (shorter shots drop out early); the reverse sweeps all end
// at k = 1 (longer shots start first), so the every-K segments [c, c+K-1] of
// all shots coincide and each segment is restored, recomputed and reversed
// for all shots at once.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "runtime.cuh"

using namespace fwi;

namespace {

enum { PH_FWD = 1, PH_REV = 2 };

struct BShot {
  fwi_shot sp{};
  Grid G{};
  StencilParams p{};
  long src = -1;
  long* rec_cell = nullptr;
  float* rec_fac = nullptr;
  float* dsim = nullptr;  // records, then the residual (fused call)
  float* f[2] = {nullptr, nullptr};  // forward pair; reverse: decode buffers / segment start pair
  float* l[2] = {nullptr, nullptr};  // adjoint pair
  float* gacc = nullptr;
  std::vector<float*> ring;  // every-K recompute ring, ring[0] = f[1]
  float* b = nullptr;
};

struct Graph {
  cudaGraphExec_t exec = nullptr;
  int phases = 0;
  const void* key[5] = {};
  size_t nodes = 0;
  unsigned long long launches = 0;
};

}  // namespace

struct fwi_batch {
  fwi_geometry g{};
  fwi_ckpt_policy pol{};
  int flags = 0;
  std::vector<BShot> shots;
  int nmax = 0;
  int K = 1;
  bool lossy = false;
  int minexp = 0;
  std::vector<void*> allocs;
  size_t device_bytes = 0;
  bool alloc_failed = false;
  int* d_status = nullptr;
  double* d_phi = nullptr;
  double* d_part = nullptr;
  float* d_wav = nullptr;
  size_t nwav = 0;
  uint8_t* arena = nullptr;
  size_t capacity = 0;
  unsigned long long* d_offs = nullptr;  // offsets [nslots], sizes [nslots], peak [1]
  int nslots = 0;
  std::vector<size_t> raw_off;
  std::map<std::tuple<int, int, int>, int> slot;  // (shot, step, level) -> slot, in issue order
  void* enc_scratch = nullptr;
  cudaStream_t cs = nullptr;   // codec side stream
  cudaStream_t own = nullptr;  // graph launches when the caller passes the legacy stream
  cudaEvent_t ev[8] = {};
  int* h_flags = nullptr;  // pinned results of the last call
  double* h_phi = nullptr;
  unsigned long long* h_used = nullptr;
  int zc = 0, ctas = 0, zc_adj = 0, ctas_adj = 0;
  bool tuned = false;
  bool filled = false;
  std::vector<Graph> graphs;
  unsigned long long launches_per_call = 0;
  size_t graph_nodes = 0;
  size_t used = 0, raw_total = 0, raw_padded = 0;

  template <class T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      alloc_failed = true;
      return nullptr;
    }
    allocs.push_back(p);
    device_bytes += n * sizeof(T);
    return static_cast<T*>(p);
  }
  ~fwi_batch() {
    for (Graph& gr : graphs)
      if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (cs) cudaStreamSynchronize(cs);
    if (own) cudaStreamSynchronize(own);
    for (void* p : allocs) cudaFree(p);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
    if (own) cudaStreamDestroy(own);
    if (h_flags) cudaFreeHost(h_flags);
    if (h_phi) cudaFreeHost(h_phi);
    if (h_used) cudaFreeHost(h_used);
    cudaGetLastError();
  }
};

namespace {

// The launch groups of one multi-field call: at most kStencilMaxFields
// fields per launch.
int stencil_groups(bool adjoint, const std::vector<const StencilParams*>& P,
                   const std::vector<StencilField>& F, float weight, int ctas, cudaStream_t s) {
  for (size_t i = 0; i < F.size(); i += kStencilMaxFields) {
    const int n = (int)std::min<size_t>(kStencilMaxFields, F.size() - i);
    CK(stencil_multi_launch(adjoint, n, P.data() + i, F.data() + i, weight, ctas, s));
  }
  return FWI_OK;
}

int rec_groups(bool inject, const std::vector<RecTask>& T, const std::vector<int>& N, float dt,
               cudaStream_t s) {
  for (size_t i = 0; i < T.size(); i += kStencilMaxFields) {
    const int n = (int)std::min<size_t>(kStencilMaxFields, T.size() - i);
    if (inject)
      CK(inject_multi_launch(n, T.data() + i, N.data() + i, dt, 1.0f, s));
    else
      CK(gather_multi_launch(n, T.data() + i, N.data() + i, s));
  }
  return FWI_OK;
}

int setup_models(fwi_batch* B, const float* d_m, cudaStream_t s) {
  for (BShot& sh : B->shots) {
    CK(setup_model_launch(d_m, sh.G, (float)B->g.dt, sh.b, B->d_status, s, B->g.nx, B->g.ny, sh.sp.x0,
                          sh.sp.y0, sh.sp.z0));
    CK(rec_fac_launch(sh.p, sh.rec_cell, sh.sp.nrec, sh.rec_fac, s));
  }
  return FWI_OK;
}

// Everything one call enqueues, with no host synchronisation (so that it
// can be captured as one CUDA graph).  Results land in the pinned buffers.
int run(fwi_batch* B, int phases, const float* d_m, const float* d_obs, const float* d_resid,
        float* d_rec_out, float* d_grad, cudaStream_t s) {
  const bool fwd = phases & PH_FWD, rev = phases & PH_REV;
  const int S = (int)B->shots.size();
  const float dtf = (float)B->g.dt;
  unsigned long long* offs = B->d_offs;
  unsigned long long* sizes = B->d_offs + B->nslots;
  unsigned long long* peak = B->d_offs + 2 * B->nslots;
  cudaStream_t cs = B->cs;
  cudaEvent_t* ev = B->ev;
  int st = FWI_OK;

  auto fork = [&]() -> int {  // codec stream continues after everything issued on s so far
    CK(cudaEventRecord(ev[6], s));
    CK(cudaStreamWaitEvent(cs, ev[6], 0));
    return FWI_OK;
  };
  auto join = [&]() -> int {  // s continues after everything issued on the codec stream
    CK(cudaEventRecord(ev[7], cs));
    CK(cudaStreamWaitEvent(s, ev[7], 0));
    return FWI_OK;
  };
  auto store_field = [&](const BShot& sh, const float* f, int j) -> int {
    if (j < 0 || j >= B->nslots) return FWI_ERR_ARG;
    if (B->lossy) {
      CK(slot_offset_launch(offs, sizes, j, cs));
      CK(zfp_encode_launch(f, sh.G, B->minexp, B->arena, offs + j, B->capacity, sizes + j, B->d_status,
                           B->enc_scratch, cs));
      CK(track_peak_launch(offs, sizes, j, peak, cs));
    } else {
      CK(cudaMemcpyAsync(B->arena + B->raw_off[j], f, sh.G.cells() * 4, cudaMemcpyDeviceToDevice, cs));
    }
    return FWI_OK;
  };
  auto load_field = [&](const BShot& sh, int j, float* f, cudaStream_t on) -> int {
    if (j < 0 || j >= B->nslots) return FWI_ERR_ARG;
    if (B->lossy)
      CK(zfp_decode_launch(B->arena, offs + j, B->capacity, f, sh.G, B->d_status, on));
    else
      CK(cudaMemcpyAsync(f, B->arena + B->raw_off[j], sh.G.cells() * 4, cudaMemcpyDeviceToDevice, on));
    return FWI_OK;
  };
  auto slot_of = [&](int sh, int step, int level) {
    auto it = B->slot.find(std::make_tuple(sh, step, level));
    return it == B->slot.end() ? -1 : it->second;
  };

  CK(cudaMemsetAsync(B->d_status, 0, sizeof(int), s));
  if (fwd) CK(cudaMemsetAsync(B->d_phi, 0, sizeof(double) * S, s));
  if ((st = setup_models(B, d_m, s))) return st;
  if ((st = fork())) return st;

  std::vector<const StencilParams*> P;
  std::vector<StencilField> F;
  std::vector<RecTask> T;
  std::vector<int> NR;
  auto clear = [&]() {
    P.clear();
    F.clear();
    T.clear();
    NR.clear();
  };

  PhaseRange phase;
  // ---- forward sweep: u^{n+1} for all shots with n < nt, records, checkpoints
  if (fwd) {
    phase.enter(kPhaseForward);
    if (B->lossy) CK(cudaMemsetAsync(B->d_offs, 0, sizeof(unsigned long long) * (2 * B->nslots + 1), s));
    for (BShot& sh : B->shots) {
      CK(cudaMemsetAsync(sh.f[0], 0, sh.G.cells() * 4, s));
      CK(cudaMemsetAsync(sh.f[1], 0, sh.G.cells() * 4, s));
    }
    bool pend[2] = {false, false};
    for (int n = 0; n < B->nmax; ++n) {
      const int w = n & 1;  // the step writes u^{n+1} over u^{n-1} in f[w]
      if (pend[w]) CK(cudaStreamWaitEvent(s, ev[w], 0));
      pend[w] = false;
      clear();
      for (int i = 0; i < S; ++i) {
        BShot& sh = B->shots[i];
        if (n >= sh.sp.nt) continue;
        StencilField fl{};
        fl.cur = sh.f[w ^ 1];
        fl.prev = sh.f[w];
        fl.out = sh.f[w];
        fl.src_cell = sh.src;
        fl.wavelet = B->d_wav + sh.sp.wavelet_first;
        fl.n = n;
        fl.zc = B->zc;
        P.push_back(&sh.p);
        F.push_back(fl);
        RecTask t{};
        t.field = sh.f[w];
        t.row_out = (d_rec_out ? d_rec_out + sh.sp.obs_first : sh.dsim) + (size_t)n * sh.sp.nrec;
        t.cell = sh.rec_cell;
        T.push_back(t);
        NR.push_back(sh.sp.nrec);
      }
      if ((st = stencil_groups(false, P, F, 1.0f, B->ctas, s))) return st;
      if ((st = rec_groups(false, T, NR, dtf, s))) return st;
      // checkpoints of this step
      const bool pair = B->pol.mode == FWI_CKPT_EVERY_K;
      if (pair && (n + 1) % B->K != 0) continue;
      bool any = false;
      for (int i = 0; i < S; ++i) {
        BShot& sh = B->shots[i];
        if (n >= sh.sp.nt) continue;
        if (!any && (st = fork())) return st;
        any = true;
        if ((st = store_field(sh, sh.f[w], slot_of(i, n + 1, 1)))) return st;
        if (pair && (st = store_field(sh, sh.f[w ^ 1], slot_of(i, n + 1, 0)))) return st;
      }
      if (any) {
        CK(cudaEventRecord(ev[w], cs));
        pend[w] = true;
        if (pair) {
          CK(cudaEventRecord(ev[w ^ 1], cs));
          pend[w ^ 1] = true;
        }
      }
    }
  }

  // ---- reverse sweep -------------------------------------------------------
  if (rev) {
    phase.enter(kPhaseReverse);
    if ((st = join())) return st;  // every checkpoint is stored
    std::vector<const float*> resid(S);
    std::vector<float*> lc(S), ln(S);
    for (int i = 0; i < S; ++i) {
      BShot& sh = B->shots[i];
      const size_t nd = (size_t)sh.sp.nt * sh.sp.nrec;
      if (fwd) CK(misfit_launch(sh.dsim, d_obs + sh.sp.obs_first, nd, sh.dsim, B->d_phi + i, B->d_part, s));
      resid[i] = fwd ? sh.dsim : d_resid + sh.sp.obs_first;
      CK(cudaMemsetAsync(sh.l[0], 0, sh.G.cells() * 4, s));
      CK(cudaMemsetAsync(sh.l[1], 0, sh.G.cells() * 4, s));
      CK(cudaMemsetAsync(sh.gacc, 0, sh.G.cells() * 4, s));
      lc[i] = sh.l[0];
      ln[i] = sh.l[1];
    }
    // adjoint step k for the shots with first <= k <= last(shot), imaging with uk(shot)
    auto adjoint = [&](int k, auto active, auto ukof) -> int {
      clear();
      for (int i = 0; i < S; ++i) {
        if (!active(i)) continue;
        BShot& sh = B->shots[i];
        StencilField fl{};
        fl.cur = lc[i];
        fl.prev = ln[i];
        fl.out = ln[i];
        fl.src_cell = -1;
        fl.uk = ukof(i);
        fl.grad = sh.gacc;
        fl.zc = B->zc_adj;
        P.push_back(&sh.p);
        F.push_back(fl);
        RecTask t{};
        t.cell = sh.rec_cell;
        t.fac = sh.rec_fac;
        t.row_in = resid[i] + (size_t)(k - 1) * sh.sp.nrec;
        t.out = ln[i];
        t.uk = fl.uk;
        t.grad = sh.gacc;
        T.push_back(t);
        NR.push_back(sh.sp.nrec);
      }
      int r = stencil_groups(true, P, F, 1.0f, B->ctas_adj, s);
      if (r) return r;
      if ((r = rec_groups(true, T, NR, dtf, s))) return r;
      for (int i = 0; i < S; ++i)
        if (active(i)) std::swap(lc[i], ln[i]);
      return FWI_OK;
    };

    if (B->pol.mode == FWI_CKPT_FULL) {
      // u^k decoded into f[k & 1] one step ahead (on the codec stream when
      // kDecodeOverlap, else in order on s)
      const cudaStream_t dq = kDecodeOverlap ? cs : s;
      bool used[2] = {false, false};
      auto prefetch = [&](int k) -> int {
        const int q = k & 1;
        if (used[q]) CK(cudaStreamWaitEvent(dq, ev[4 + q], 0));
        for (int i = 0; i < S; ++i)
          if (k <= B->shots[i].sp.nt) {
            int r = load_field(B->shots[i], slot_of(i, k, 1), B->shots[i].f[q], dq);
            if (r) return r;
          }
        CK(cudaEventRecord(ev[2 + q], dq));
        return FWI_OK;
      };
      if ((st = fork())) return st;
      if (B->nmax > 0 && (st = prefetch(B->nmax))) return st;
      for (int k = B->nmax; k >= 1; --k) {
        const int q = k & 1;
        CK(cudaStreamWaitEvent(s, ev[2 + q], 0));
        if (k > 1 && (st = prefetch(k - 1))) return st;
        st = adjoint(
            k, [&](int i) { return k <= B->shots[i].sp.nt; },
            [&](int i) { return (const float*)B->shots[i].f[q]; });
        if (st) return st;
        CK(cudaEventRecord(ev[4 + q], s));
        used[q] = true;
      }
    } else {  // every-K: segments from the last checkpoint back to 0
      const int K = B->K;
      int cmax = 0;
      for (const BShot& sh : B->shots) cmax = std::max(cmax, sh.sp.nt - sh.sp.nt % K);
      for (int c = cmax; c >= 0; c -= K) {
        const int first = std::max(c, 1);
        std::vector<int> last(S, -1);
        int maxlast = -1;
        for (int i = 0; i < S; ++i) {
          const int nt = B->shots[i].sp.nt;
          if (c > nt) continue;
          const int l = std::min(c + K - 1, nt);
          if (l < first) continue;
          last[i] = l;
          maxlast = std::max(maxlast, l);
        }
        if (maxlast < 0) continue;
        // restore the pair (u^{c-1}, u^c) into (f[0], ring[0] = f[1])
        for (int i = 0; i < S; ++i) {
          if (last[i] < 0) continue;
          BShot& sh = B->shots[i];
          if (c == 0) {
            CK(cudaMemsetAsync(sh.f[0], 0, sh.G.cells() * 4, s));
            CK(cudaMemsetAsync(sh.f[1], 0, sh.G.cells() * 4, s));
          } else {
            if ((st = load_field(sh, slot_of(i, c, 0), sh.f[0], s))) return st;
            if ((st = load_field(sh, slot_of(i, c, 1), sh.f[1], s))) return st;
          }
        }
        // recompute u^{c+1} .. u^{last} into the ring
        for (int stp = c; stp < maxlast; ++stp) {
          clear();
          for (int i = 0; i < S; ++i) {
            if (stp >= last[i]) continue;
            BShot& sh = B->shots[i];
            const int r = stp - c;
            StencilField fl{};
            fl.cur = sh.ring[r];
            fl.prev = r == 0 ? sh.f[0] : sh.ring[r - 1];
            fl.out = sh.ring[r + 1];
            fl.src_cell = sh.src;
            fl.wavelet = B->d_wav + sh.sp.wavelet_first;
            fl.n = stp;
            fl.zc = B->zc;
            P.push_back(&sh.p);
            F.push_back(fl);
          }
          if ((st = stencil_groups(false, P, F, 1.0f, B->ctas, s))) return st;
        }
        for (int k = maxlast; k >= first; --k) {
          st = adjoint(
              k, [&](int i) { return last[i] >= k; },
              [&](int i) { return (const float*)B->shots[i].ring[k - c]; });
          if (st) return st;
        }
      }
    }
    // stacking: the shots' gradients into the model grid, in shot order
    for (BShot& sh : B->shots)
      CK(stack_add_launch(sh.gacc, sh.G, d_grad, B->g.nx, B->g.ny, sh.sp.x0, sh.sp.y0, sh.sp.z0, s));
  }
  if ((st = join())) return st;
  CK(cudaMemcpyAsync(B->h_flags, B->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(B->h_phi, B->d_phi, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
  if (B->lossy && fwd) CK(cudaMemcpyAsync(B->h_used, peak, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  return FWI_OK;
}

// Autotuner: time each candidate (tile depth, persistent grid size) on the
// plan's own fields for a few steps of the forward and of the adjoint
// kernel, and keep the fastest of each.
int tune(fwi_batch* B, cudaStream_t s) {
  if (stencil_multi_capacity(false) <= 0) return FWI_ERR_CUDA;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  int nz = 1;
  for (const BShot& sh : B->shots) nz = std::max(nz, sh.G.nz);
  std::vector<int> zcs = {0, nz, (nz + 1) / 2, (nz + 2) / 3, (nz + 3) / 4, 64, 48, 32, 24, 16};
  std::sort(zcs.begin(), zcs.end());
  zcs.erase(std::unique(zcs.begin(), zcs.end()), zcs.end());
  cudaEvent_t ta, tb;
  CK(cudaEventCreate(&ta));
  if (cudaEventCreate(&tb) != cudaSuccess) {
    cudaEventDestroy(ta);
    return FWI_ERR_CUDA;
  }
  const int reps = 3;
  int rc = FWI_OK;
  for (int adj = 0; adj < 2 && rc == FWI_OK; ++adj) {
    const int cap = stencil_multi_capacity(adj != 0);
    std::vector<int> grids;
    for (int m = 1; m * sms <= cap; ++m) grids.push_back(m * sms);
    if (grids.empty()) grids.push_back(cap);
    float best = 1e30f;
    int bz = 0, bg = cap;
    for (int zc : zcs) {
      if (zc != 0 && (zc < 8 || zc > nz)) continue;
      for (int grid : grids) {
        std::vector<const StencilParams*> P;
        std::vector<StencilField> F;
        for (BShot& sh : B->shots) {
          StencilField fl{};
          fl.zc = zc;
          if (adj) {
            fl.cur = sh.l[0];
            fl.prev = sh.l[1];
            fl.out = sh.l[1];
            fl.uk = sh.f[0];
            fl.grad = sh.gacc;
          } else {
            fl.cur = sh.f[1];
            fl.prev = sh.f[0];
            fl.out = sh.f[0];
          }
          fl.src_cell = -1;
          P.push_back(&sh.p);
          F.push_back(fl);
        }
        int r = stencil_groups(adj, P, F, 1.0f, grid, s);  // warm-up
        if (r == FWI_OK && cudaEventRecord(ta, s) != cudaSuccess) r = FWI_ERR_CUDA;
        for (int i = 0; i < reps && r == FWI_OK; ++i) r = stencil_groups(adj, P, F, 1.0f, grid, s);
        float ms = 0.f;
        if (r == FWI_OK && (cudaEventRecord(tb, s) != cudaSuccess || cudaEventSynchronize(tb) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, ta, tb) != cudaSuccess))
          r = FWI_ERR_CUDA;
        if (r) {
          rc = r;
          break;
        }
        if (ms < best) {
          best = ms;
          bz = zc;
          bg = grid;
        }
      }
      if (rc) break;
    }
    if (adj) {
      B->zc_adj = bz;
      B->ctas_adj = bg;
    } else {
      B->zc = bz;
      B->ctas = bg;
    }
  }
  cudaEventDestroy(ta);
  cudaEventDestroy(tb);
  cudaGetLastError();
  if (rc == FWI_OK) B->tuned = true;
  return rc;
}

bool shot_ok(const fwi_geometry* g, const fwi_shot& s) {
  return s.nx > 0 && s.ny > 0 && s.nz > 0 && s.x0 >= 0 && s.y0 >= 0 && s.z0 >= 0 && s.x0 + s.nx <= g->nx &&
         s.y0 + s.ny <= g->ny && s.z0 + s.nz <= g->nz && s.nt >= 1 && s.nrec >= 0 && s.rec_first >= 0 &&
         s.wavelet_first >= 0 && s.obs_first >= 0 && s.src_i >= s.x0 && s.src_i < s.x0 + s.nx &&
         s.src_j >= s.y0 && s.src_j < s.y0 + s.ny && s.src_k >= s.z0 && s.src_k < s.z0 + s.nz;
}

int call(fwi_batch* B, int phases, const float* d_m, const float* h_wavelets, const float* d_obs,
         const float* d_resid, float* d_rec_out, float* d_grad, double* h_misfit, void* stream) {
  const bool fwd = phases & PH_FWD, rev = phases & PH_REV;
  if (!B || !d_m || !h_wavelets) return FWI_ERR_ARG;
  if (rev && !d_grad) return FWI_ERR_ARG;
  if (fwd && rev && (!d_obs || !h_misfit)) return FWI_ERR_ARG;
  if (!fwd && rev && !d_resid) return FWI_ERR_ARG;
  if (fwd && !rev && !d_rec_out) return FWI_ERR_ARG;
  if (!fwd && !B->filled) return FWI_ERR_ARG;
  cudaStream_t user = (cudaStream_t)stream;
  const bool graph = B->flags & FWI_BATCH_GRAPH;
  cudaStream_t s = user;
  if (graph && user == nullptr) {
    // stream capture needs a stream of its own; order it after the caller's work
    s = B->own;
    CK(cudaStreamSynchronize(user));
  }
  CK(cudaMemcpyAsync(B->d_wav, h_wavelets, sizeof(float) * B->nwav, cudaMemcpyHostToDevice, s));
  int st = FWI_OK;
  if ((B->flags & FWI_BATCH_TUNE) && !B->tuned && fwd) {
    CK(cudaMemsetAsync(B->d_status, 0, sizeof(int), s));
    if ((st = setup_models(B, d_m, s))) return st;
    if ((st = tune(B, s))) return st;
  }
  if (fwd) B->filled = false;
  if (graph) {
    const void* key[5] = {d_m, d_obs, d_resid, d_rec_out, d_grad};
    Graph* gr = nullptr;
    for (Graph& x : B->graphs)
      if (x.phases == phases && std::equal(key, key + 5, x.key)) gr = &x;
    if (!gr) {
      const unsigned long long l0 = launches_so_far();
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      st = run(B, phases, d_m, d_obs, d_resid, d_rec_out, d_grad, s);
      cudaGraph_t G = nullptr;
      const cudaError_t e = cudaStreamEndCapture(s, &G);
      if (st || e != cudaSuccess || !G) {
        if (G) cudaGraphDestroy(G);
        cudaGetLastError();
        return st ? st : FWI_ERR_CUDA;
      }
      Graph x;
      x.phases = phases;
      std::copy(key, key + 5, x.key);
      x.launches = launches_so_far() - l0;
      cudaGraphGetNodes(G, nullptr, &x.nodes);
      const cudaError_t ei = cudaGraphInstantiate(&x.exec, G, 0);
      cudaGraphDestroy(G);
      if (ei != cudaSuccess) {
        cudaGetLastError();
        return FWI_ERR_CUDA;
      }
      B->graphs.push_back(x);
      gr = &B->graphs.back();
      count_launches(0);
    } else {
      count_launches(gr->launches);
    }
    B->graph_nodes = gr->nodes;
    B->launches_per_call = gr->launches;
    CK(cudaGraphLaunch(gr->exec, s));
  } else {
    const unsigned long long l0 = launches_so_far();
    if ((st = run(B, phases, d_m, d_obs, d_resid, d_rec_out, d_grad, s))) {
      cudaStreamSynchronize(s);
      cudaGetLastError();
      return st;
    }
    B->launches_per_call = launches_so_far() - l0;
  }
  CK(cudaStreamSynchronize(s));
  const int flags = *B->h_flags;
  if (fwd && B->lossy) B->used = (size_t)*B->h_used;
  if (flags) {
    if ((flags & ST_CORRUPT) && !(flags & (ST_CAPACITY | ST_NONFINITE))) return FWI_ERR_CORRUPT;
    return status_from_flags(flags);
  }
  if (fwd) B->filled = true;
  if (fwd && rev)
    for (size_t i = 0; i < B->shots.size(); ++i) h_misfit[i] = B->h_phi[i];
  return FWI_OK;
}

}  // namespace

extern "C" {

int fwi_batch_create(const fwi_geometry* g, int nshots, const fwi_shot* h_shots, const int* d_rec_ijk,
                     const fwi_ckpt_policy* pol, size_t arena_bytes, int flags, fwi_batch** out) {
  if (!out || !geometry_ok(g) || nshots <= 0 || !h_shots || !pol) return FWI_ERR_ARG;
  if (pol->mode != FWI_CKPT_FULL && pol->mode != FWI_CKPT_EVERY_K) return FWI_ERR_ARG;
  if (pol->mode == FWI_CKPT_EVERY_K && pol->k_or_snaps < 1) return FWI_ERR_ARG;
  if (pol->atol > 0.0 && !isfinite(pol->atol)) return FWI_ERR_ARG;
  if (flags & ~(FWI_BATCH_GRAPH | FWI_BATCH_TUNE)) return FWI_ERR_ARG;
  for (int i = 0; i < nshots; ++i) {
    if (!shot_ok(g, h_shots[i])) return FWI_ERR_ARG;
    if (h_shots[i].nrec > 0 && !d_rec_ijk) return FWI_ERR_ARG;
  }
  if (stencil_multi_capacity(false) <= 0) return FWI_ERR_CUDA;
  fwi_batch* B = new fwi_batch();
  B->g = *g;
  B->pol = *pol;
  B->flags = flags;
  B->K = pol->mode == FWI_CKPT_EVERY_K ? pol->k_or_snaps : 1;
  B->lossy = pol->atol > 0.0;
  if (B->lossy) {
    int e;
    frexp(pol->atol, &e);
    B->minexp = e - 1;
  }
  auto fail = [&](int code) {
    delete B;
    return code;
  };
  if (cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&B->own, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return fail(FWI_ERR_CUDA);
  }
  for (cudaEvent_t& e : B->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(FWI_ERR_CUDA);
    }
  if (cudaMallocHost(&B->h_flags, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&B->h_phi, sizeof(double) * nshots) != cudaSuccess ||
      cudaMallocHost(&B->h_used, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail(FWI_ERR_NOMEM);
  }
  cudaStream_t s = B->own;
  B->shots.resize(nshots);
  size_t nwav = 1, scratch = 0;
  for (int i = 0; i < nshots; ++i) {
    BShot& sh = B->shots[i];
    sh.sp = h_shots[i];
    const fwi_shot& sp = sh.sp;
    B->nmax = std::max(B->nmax, sp.nt);
    nwav = std::max(nwav, (size_t)sp.wavelet_first + sp.nt);
    sh.G = Grid{sp.nx, sp.ny, sp.nz, round_up(sp.nx, 4)};
    const size_t C = sh.G.cells();
    sh.p.g = sh.G;
    for (int r = 0; r < 5; ++r) sh.p.c[r] = (float)(kC[r] / (g->h * g->h));
    sh.p.dt = (float)g->dt;
    sh.b = B->alloc<float>(C);
    float* sx = B->alloc<float>(sp.nx);
    float* sy = B->alloc<float>(sp.ny);
    float* sz = B->alloc<float>(sp.nz);
    sh.p.b = sh.b;
    sh.p.sx = sx;
    sh.p.sy = sy;
    sh.p.sz = sz;
    sh.rec_cell = B->alloc<long>(sp.nrec);
    sh.rec_fac = B->alloc<float>(sp.nrec);
    sh.dsim = B->alloc<float>((size_t)sp.nt * (sp.nrec > 0 ? sp.nrec : 1));
    sh.f[0] = B->alloc<float>(C);
    sh.f[1] = B->alloc<float>(C);
    sh.l[0] = B->alloc<float>(C);
    sh.l[1] = B->alloc<float>(C);
    sh.gacc = B->alloc<float>(C);
    if (pol->mode == FWI_CKPT_EVERY_K) {
      sh.ring.push_back(sh.f[1]);
      for (int r = 1; r < B->K; ++r) sh.ring.push_back(B->alloc<float>(C));
    }
    if (B->alloc_failed) return fail(FWI_ERR_NOMEM);
    sh.src = (long)(sp.src_i - sp.x0) +
             (long)sh.G.pitch * ((long)(sp.src_j - sp.y0) + (long)sp.ny * (sp.src_k - sp.z0));
    if (B->lossy) scratch = std::max(scratch, zfp_encode_scratch_bytes(sp.nx, sp.ny, sp.nz));
  }
  B->nwav = nwav;
  B->d_wav = B->alloc<float>(nwav);
  B->d_status = B->alloc<int>(1);
  B->d_phi = B->alloc<double>(nshots);
  B->d_part = B->alloc<double>(reduce_scratch_doubles());
  if (B->lossy) B->enc_scratch = B->alloc<unsigned char>(scratch);
  // checkpoint slots in the order the forward sweep issues them
  for (int n = 0; n < B->nmax; ++n) {
    if (pol->mode == FWI_CKPT_EVERY_K && (n + 1) % B->K != 0) continue;
    for (int i = 0; i < nshots; ++i) {
      if (n >= B->shots[i].sp.nt) continue;
      const size_t raw = (B->shots[i].G.cells() * 4 + 255) / 256 * 256;
      const size_t packed = (size_t)B->shots[i].sp.nx * B->shots[i].sp.ny * B->shots[i].sp.nz * 4;
      for (int level = 1; level >= (pol->mode == FWI_CKPT_EVERY_K ? 0 : 1); --level) {
        B->slot[std::make_tuple(i, n + 1, level)] = B->nslots++;
        B->raw_off.push_back(B->raw_padded);
        B->raw_total += packed;
        B->raw_padded += raw;
      }
    }
  }
  if (!B->lossy && B->raw_padded > arena_bytes) return fail(FWI_ERR_CAPACITY);
  B->d_offs = B->alloc<unsigned long long>(2 * (size_t)B->nslots + 1);
  B->capacity = arena_bytes;
  B->arena = B->alloc<uint8_t>(arena_bytes);
  if (B->alloc_failed) return fail(FWI_ERR_NOMEM);
  // fixed per-shot setup: damping profiles and receiver cells
  if (cudaMemsetAsync(B->d_status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return fail(FWI_ERR_CUDA);
  }
  for (BShot& sh : B->shots) {
    if (setup_profiles_launch(sh.G, g->nbl, g->h, g->vmax, g->sponge_R, g->dt, const_cast<float*>(sh.p.sx),
                              const_cast<float*>(sh.p.sy), const_cast<float*>(sh.p.sz), s) != cudaSuccess ||
        rec_cells_launch(d_rec_ijk ? d_rec_ijk + 3 * (size_t)sh.sp.rec_first : nullptr, sh.sp.nrec, sh.G,
                         sh.rec_cell, B->d_status, s, sh.sp.x0, sh.sp.y0, sh.sp.z0) != cudaSuccess) {
      cudaGetLastError();
      return fail(FWI_ERR_CUDA);
    }
    sh.p.status = B->d_status;
  }
  int flags_h = 0;
  if (cudaMemcpyAsync(&flags_h, B->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return fail(FWI_ERR_CUDA);
  }
  if (flags_h) return fail(FWI_ERR_ARG);  // a receiver outside its shot's aperture
  // default launch shape: deep tiles while the tile list still fills the GPU
  B->ctas = stencil_multi_capacity(false);
  B->ctas_adj = stencil_multi_capacity(true);
  int nz = 1;
  long cols = 0;
  for (const BShot& sh : B->shots) {
    nz = std::max(nz, sh.G.nz);
    cols += (long)((sh.G.pitch + 63) / 64) * ((sh.G.ny + 15) / 16);
  }
  int zc = nz;
  while (zc > 16 && cols * ((nz + zc - 1) / zc) < 2L * B->ctas) zc = (zc + 1) / 2;
  B->zc = B->zc_adj = zc;
  *out = B;
  return FWI_OK;
}

int fwi_batch_destroy(fwi_batch* b) {
  if (!b) return FWI_ERR_ARG;
  delete b;
  return FWI_OK;
}

int fwi_batch_gradient(fwi_batch* b, const float* d_m, const float* h_wavelets, const float* d_obs,
                       float* d_grad, double* h_misfit, void* stream) {
  return call(b, PH_FWD | PH_REV, d_m, h_wavelets, d_obs, nullptr, nullptr, d_grad, h_misfit, stream);
}

int fwi_batch_forward(fwi_batch* b, const float* d_m, const float* h_wavelets, float* d_rec_out,
                      void* stream) {
  return call(b, PH_FWD, d_m, h_wavelets, nullptr, nullptr, d_rec_out, nullptr, nullptr, stream);
}

int fwi_batch_adjoint(fwi_batch* b, const float* d_m, const float* h_wavelets, const float* d_resid,
                      float* d_grad, void* stream) {
  return call(b, PH_REV, d_m, h_wavelets, nullptr, d_resid, nullptr, d_grad, nullptr, stream);
}

int fwi_batch_get_stats(const fwi_batch* b, fwi_batch_stats* out) {
  if (!b || !out) return FWI_ERR_ARG;
  fwi_batch_stats st{};
  st.nshots = (int)b->shots.size();
  st.max_nt = b->nmax;
  st.zc = b->zc;
  st.ctas = b->ctas;
  st.zc_adjoint = b->zc_adj;
  st.ctas_adjoint = b->ctas_adj;
  st.tuned = b->tuned ? 1 : 0;
  st.graph_nodes = (int)b->graph_nodes;
  st.launches_per_call = b->launches_per_call;
  st.arena_bytes = b->capacity;
  st.used_bytes = b->lossy ? b->used : b->raw_padded;
  st.raw_bytes = b->raw_total;
  st.device_bytes = b->device_bytes;
  *out = st;
  return FWI_OK;
}

}  // extern "C"
