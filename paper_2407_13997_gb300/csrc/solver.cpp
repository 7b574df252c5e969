// Host control plane of libwrmg: the level hierarchy, the V(2,2) cycle
// (Algorithm Vcycle), Chebyshev(2) relaxation weights with the 10-step Arnoldi
// eigen-estimate (Sec. 3), the coarse direct solve, FGMRES (restart 30, MGS,
// Givens) and inexact Newton with Eisenstat-Walker forcing terms (Sec. 5).
// Every vector operation runs in this library's kernels on the context stream;
// only Krylov scalars (dot products, Hessenberg entries) come to the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <atomic>
#include <functional>
#include <map>
#include <memory>
#include <mutex>

#include "wrmg_internal.h"

void launch_patch_slots(const LevelGeom& g, const BlockSet& bs, int blk, int* out_sp, cudaStream_t s);

namespace {
std::atomic<int64_t> g_launches{0};
}  // namespace
void wr_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void wr_count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void wr_uncount_launches(int64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

// host-side fault injection: the n-th device allocation from now on fails (0 = off)
std::atomic<int64_t> g_fail_alloc{0};

// Autotuner of the smoother-apply tile: every variant is timed on the level's own
// stored factors (one warm-up and two timed launches, CUDA events on the stream)
// and the fastest is kept.  The choice is cached for the process per key, so every
// context and batch of one shape and precision uses the same tile (and therefore
// the same summation order) from then on.
namespace {
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;
}  // namespace

int tune_apply_variant(const TuneKey& key, cudaStream_t s, const std::function<void(int)>& launch) {
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  cudaEvent_t e0, e1;
  WR_CUDA(cudaEventCreate(&e0));
  WR_CUDA(cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 0.f;
  for (int v = 0; v < kApplyTileVariants; ++v) {
    if (v == 4 && !(key.k == 1 && key.q == 0)) continue;  // tile 4 exists for Q2/Q1 DG(0) only (else it is tile 3)
    // FP64 DG(1): A10 is stored by segments and the warp tiles run as tile 2
    if (v >= 3 && key.q == 1 && key.precision == WR_FP64) continue;
    launch(v);
    WR_CUDA(cudaEventRecord(e0, s));
    launch(v);
    launch(v);
    WR_CUDA(cudaEventRecord(e1, s));
    WR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    WR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (best < 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return g_tuned.emplace(key, best).first->second;  // a concurrent tuner may have won: keep its choice
}

namespace {

struct Level {
  LevelGeom g;
  BlockSet bs;
  double* W = nullptr;
  double* Wq = nullptr;     // W and grad W at the Gauss points (launch_wq)
  void* factors = nullptr;  // stored factors (null when the level recomputes them per apply)
  bool recompute = false;   // factors recomputed in windows of `nw` slabs at every smoother apply
  int nw = 0;
  int variant = -1;         // apply tile chosen by the autotuner (-1: not yet, the default of k)
  // time-parallel patch solve: nchunk chunks of Lc slabs, chunk transfer matrices Tm,
  // chunk-boundary states carry (nchunk = 1: the plain sweep over all slabs)
  int nchunk = 1, Lc = 0;
  double *Tm = nullptr, *carry = nullptr;
  double *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr, *z = nullptr, *t = nullptr;
  double lam = 0.0;
  bool lam_set = false;
};

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct wr_ctx {
  std::string err;
  cudaStream_t s = nullptr;
  wr_options opt;
  PhysParams ph;
  FeTables tab;
  int k = 0, q = 0, N = 0;
  double T = 1.0;
  std::vector<Level> L;  // 0 = coarsest
  BlockSet cbs;
  double* cfactors = nullptr;
  double *Ce = nullptr, *ye = nullptr, *Yp = nullptr;
  std::vector<double*> V, Z;
  double *F = nullptr, *w = nullptr, *hb = nullptr, *hx = nullptr;
  double *partials = nullptr, *dres = nullptr, *hres = nullptr;
  // device-resident Krylov scalars: FGMRES Hessenberg, rotations, right-hand side and
  // least-squares solution, the Arnoldi Hessenberg of the eigen-estimate, and scalars
  double* kd = nullptr;
  unsigned* kcnt = nullptr;  // zeroed block counter of the one-launch reductions
  double* hk = nullptr;  // pinned host copy of the eigen-estimate Hessenberg
  double* kH() { return kd; }
  double* kcs() { return kd + (opt.gmres_restart + 1) * opt.gmres_restart; }
  double* ksn() { return kcs() + opt.gmres_restart; }
  double* kg() { return ksn() + opt.gmres_restart; }
  double* ky() { return kg() + opt.gmres_restart + 1; }
  double* keH() { return ky() + opt.gmres_restart; }
  double* kscal() { return keH() + (opt.eig_steps + 1) * opt.eig_steps; }
  static int64_t krylov_doubles(const wr_options& o) {
    return (int64_t)(o.gmres_restart + 1) * o.gmres_restart + 4 * o.gmres_restart + 1 +
           (int64_t)(o.eig_steps + 1) * o.eig_steps + 8;
  }
  int* herr = nullptr;
  int* slots = nullptr;
  int* derr = nullptr;   // device error flag of the bounded waits
  int* fstat = nullptr;  // device zero-pivot flag of the factorisation
  bool heat = false;     // the heat equation (one scalar field) instead of Navier-Stokes
  double t0 = 0.0;       // the problem's start time
  double* u0 = nullptr;  // slab-0 initial state set by wr_set_initial_state (a finest-level spatial block)
  double* htmp = nullptr;  // heat equation: scratch of the tensor-product operator passes
  std::vector<void*> allocs;
  int64_t bytes = 0;
  bool linearised = false;
  int vcycles = 0;
  // CUDA-event timing of the smoother-apply kernel (per level), enabled by wr_profile
  bool prof = false;
  std::vector<std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> prof_jac;  // J(W)x element kernel, per level
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;

  cudaEvent_t next_event() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e;
      WR_CUDA(cudaEventCreate(&e));
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }

  bool dry = false;  // count the allocations of wr_create without making them
  // levels (from the finest down) that recompute their factors; -1 = decide from the options
  int forced_recompute = -1;
  void* fwin = nullptr;  // factor window of the recomputing levels
  // allocate from the stream-ordered pool on s (no device-wide synchronisation
  // in cudaMalloc/cudaFree while other streams run; used by the server)
  bool stream_ordered = false;
  const std::atomic<int>* cancel = nullptr;  // set by the server: stop the solve at the next check

  void check_cancel() const {
    if (cancel && cancel->load()) throw WrError(WR_ERR_CANCELLED, "the request was cancelled");
  }

  template <typename Tp>
  Tp* alloc(size_t count) {
    void* p = nullptr;
    const size_t nb = std::max<size_t>(count * sizeof(Tp), 16);
    if (dry) {
      bytes += nb;
      return reinterpret_cast<Tp*>(uintptr_t(256));
    }
    if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1)
      throw WrError(WR_ERR_NOMEM, "injected allocation failure (wr_inject_alloc_failure)");
    cudaError_t e = stream_ordered ? cudaMallocAsync(&p, nb, s) : cudaMalloc(&p, nb);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw WrError(WR_ERR_NOMEM, "cudaMalloc of " + std::to_string(nb) + " bytes failed (" + cudaGetErrorString(e) +
                                      "); " + std::to_string(bytes) + " bytes already held");
    }
    allocs.push_back(p);
    bytes += nb;
    return static_cast<Tp*>(p);
  }
  ~wr_ctx() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    if (stream_ordered) {
      for (void* p : allocs) cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    } else {
      for (void* p : allocs) cudaFree(p);
    }
    if (hres) cudaFreeHost(hres);
    if (hk) cudaFreeHost(hk);
    if (herr) cudaFreeHost(herr);
  }

  Level& fine() { return L.back(); }
  int top() const { return (int)L.size() - 1; }

  double dot(int64_t n, const double* x, const double* y) {
    krylov_axpy_dot(n, nullptr, nullptr, const_cast<double*>(x), y, partials, kcnt, dres, s);
    WR_CUDA(cudaMemcpyAsync(hres, dres, sizeof(double), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    if (*herr) throw WrError(WR_ERR_TIMEOUT, "a bounded wait in the smoother kernel gave up");
    return *hres;
  }
  void check_device() {
    WR_CUDA(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    if (*herr) throw WrError(WR_ERR_TIMEOUT, "a bounded wait in the smoother kernel gave up");
  }
  double norm(int64_t n, const double* x) { return std::sqrt(dot(n, x, x)); }
  // ||x|| to the host; also leaves ||x|| in kscal()[0] and 1 / ||x|| in kscal()[1] on the device
  double norm_dev(int64_t n, double* x) {
    krylov_axpy_norm(n, nullptr, nullptr, x, partials, kcnt, kscal(), kscal() + 1, nullptr, 0.0, 0.0, s);
    return read_scalar(kscal());
  }
  double read_scalar(const double* d) {
    WR_CUDA(cudaMemcpyAsync(hres, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    if (*herr) throw WrError(WR_ERR_TIMEOUT, "a bounded wait in the smoother kernel gave up");
    return *hres;
  }
  // Modified Gram-Schmidt of V[j+1] against V[0..j] on the device: H[i][j] (row
  // stride m) = <w, V[i]> after w -= H[i-1][j] V[i-1]; then H[j+1][j] = ||w|| and
  // w /= H[j+1][j] (skipped if 0; with breakdown = true, w = 0 where H[j+1][j] <=
  // 1e-14 |H[j][j]| + 1e-300).
  void mgs_dev(int64_t n, double* H, int m, int j, bool breakdown) {
    double* w = V[j + 1];
    if (n <= mgs_small_limit()) {  // short vectors: the whole column in one launch
      KrylovBasis vb{};
      for (int i = 0; i <= j; ++i) vb.p[i] = V[i];
      krylov_mgs_small(n, vb, j, w, H, m, j, breakdown, s);
      return;
    }
    for (int i = 0; i <= j; ++i)
      krylov_axpy_dot(n, i ? H + (i - 1) * m + j : nullptr, i ? V[i - 1] : nullptr, w, V[i], partials, kcnt,
                      H + i * m + j, s);
    krylov_axpy_norm(n, H + j * m + j, V[j], w, partials, kcnt, H + (j + 1) * m + j, kscal() + 2,
                     breakdown ? H + j * m + j : nullptr, 1e-14, 1e-300, s);
    vec_scale_dev(n, kscal() + 2, w, w, s);
  }

  void jac(int l, const double* x, double* y) {
    if (heat) heat_jacobian(L[l].g, tab, ph, x, y, htmp, s);
    else if (prof && l < (int)prof_jac.size()) {
      cudaEvent_t e0 = next_event(), e1 = next_event();
      launch_jacobian_wq(L[l].g, tab, ph, L[l].Wq, x, y, ye, s, e0, e1);
      prof_jac[l].push_back({e0, e1});
    } else {
      launch_jacobian_wq(L[l].g, tab, ph, L[l].Wq, x, y, ye, s);
    }
  }
  // J inside the preconditioner (smoother residuals, the residual restricted to the
  // next level, eigen-estimates): single-precision element arithmetic in the
  // reduced-precision forms; the Newton residual and the outer FGMRES use jac().
  void jac_inner(int l, const double* x, double* y) {
    if (!heat && opt.precision != WR_FP64) launch_jacobian_f32(L[l].g, tab, ph, L[l].W, x, y, ye, s);
    else jac(l, x, y);
  }
  void restrict_to(int l, const double* xf, double* xc) {
    if (heat) heat_restrict(L[l].g, L[l - 1].g, tab, xf, xc, s);
    else launch_restrict(L[l].g, L[l - 1].g, tab, xf, xc, s);
  }
  void prolong_add(int l, const double* xc, double* xf) {
    if (heat) heat_prolong_add(L[l].g, L[l - 1].g, tab, xc, xf, s);
    else launch_prolong_add(L[l].g, L[l - 1].g, tab, xc, xf, s);
  }
  void project(const LevelGeom& g, double* x) {
    if (!heat) launch_project_pressure(g, tab, x, s);  // the heat operator has no null space
  }
  void residual(const double* U, double* Fo) {
    if (heat) heat_residual(fine().g, tab, ph, U, Fo, htmp, s);
    else launch_residual(fine().g, tab, ph, U, Fo, ye, s);
  }

  // Recomputing levels: per window of slabs, the convection element matrices and
  // the slab factors are rebuilt into the window buffer and applied at once; the
  // forward substitution carries the jump state across windows through the
  // previous slab's patch outputs.
  void factor_window(int l, int s0, int nwc, bool check) {
    Level& lv = L[l];
    LevelGeom gw = lv.g;
    gw.N = nwc;
    gw.ndofs = (int64_t)nwc * gw.nt * gw.S;
    if (ph.conv != 0.0) launch_conv_elements(gw, tab, lv.W + (int64_t)s0 * gw.nt * gw.S, Ce, opt.precision, s);
    launch_block_factor(gw, tab, ph, lv.bs, Ce, fwin, opt.precision, fstat, s, check);
  }

  void patch_apply_windows(int l, const double* r, double* y) {
    Level& lv = L[l];
    const LevelGeom& g = lv.g;
    const int64_t slab_out = (int64_t)g.npatch() * g.nt * lv.bs.ms;
    for (int s0 = 0; s0 < g.N; s0 += lv.nw) {
      const int nwc = std::min(lv.nw, g.N - s0);
      factor_window(l, s0, nwc, false);
      LevelGeom gw = g;
      gw.N = nwc;
      gw.ndofs = (int64_t)nwc * gw.nt * gw.S;
      const double* prev = s0 > 0 ? Yp + (s0 - 1) * slab_out : nullptr;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (prof) {
        e0 = next_event();
        e1 = next_event();
        WR_CUDA(cudaEventRecord(e0, s));
      }
      launch_block_apply(gw, tab, lv.bs, fwin, opt.precision, r + (int64_t)s0 * g.nt * g.S, Yp + s0 * slab_out, derr,
                         s, prev);
      if (prof) {
        WR_CUDA(cudaEventRecord(e1, s));
        prof_ev[l].push_back({e0, e1});
      }
    }
    launch_scatter(g, lv.bs, Yp, y, s);
  }

  // (A) every chunk from a zero state, (B) chain the chunk-end states, (C) every chunk
  // but the first again from its incoming state; then the scatter
  void patch_apply_time_parallel(int l, const double* r, double* y) {
    Level& lv = L[l];
    ChunkPlan a;
    a.nchunk = lv.nchunk;
    a.Lc = lv.Lc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      e0 = next_event();
      e1 = next_event();
      WR_CUDA(cudaEventRecord(e0, s));
    }
    launch_block_apply(lv.g, tab, lv.bs, lv.factors, opt.precision, r, Yp, derr, s, nullptr, lv.variant, &a);
    cr_carry(lv.g, lv.bs, lv.nchunk, lv.Lc, lv.Tm, Yp, lv.carry, s);
    ChunkPlan c = a;
    c.c_first = 1;
    c.prev_mode = 1;
    c.prev = lv.carry;
    launch_block_apply(lv.g, tab, lv.bs, lv.factors, opt.precision, r, Yp, derr, s, nullptr, lv.variant, &c);
    if (prof) {
      WR_CUDA(cudaEventRecord(e1, s));
      prof_ev[l].push_back({e0, e1});
    }
    launch_scatter(lv.g, lv.bs, Yp, y, s);
  }

  // Chunk transfer matrices: column j of every T_c is the chunk-end state of a sweep
  // with a zero right-hand side from the unit incoming state j.
  void build_transfer_matrices(int l) {
    Level& lv = L[l];
    const int mv = 2 * lv.bs.nvg * lv.bs.nvg;
    vec_zero(lv.g.ndofs, lv.x, s);
    ChunkPlan u;
    u.nchunk = lv.nchunk;
    u.Lc = lv.Lc;
    u.prev_mode = 2;
    u.prev = lv.carry;  // the unit state lives in the first carry slab during set-up
    for (int j = 0; j < mv; ++j) {
      cr_unit_state(lv.g, lv.bs, j, lv.carry, s);
      launch_block_apply(lv.g, tab, lv.bs, lv.factors, opt.precision, lv.x, Yp, derr, s, nullptr, lv.variant, &u);
      cr_gather_column(lv.g, lv.bs, lv.nchunk, lv.Lc, j, Yp, lv.Tm, s);
    }
  }

  void patch_apply(int l, const double* r, double* y) {
    if (!linearised) throw WrError(WR_ERR_STATE, "wr_linearise must be called first");
    if (heat) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (prof) {
        e0 = next_event();
        e1 = next_event();
        WR_CUDA(cudaEventRecord(e0, s));
      }
      heat_patch_apply(L[l].g, tab, static_cast<const double*>(L[l].factors), r, Yp, y, s);
      if (prof) {
        WR_CUDA(cudaEventRecord(e1, s));
        prof_ev[l].push_back({e0, e1});
      }
      return;
    }
    if (L[l].recompute) {
      patch_apply_windows(l, r, y);
      return;
    }
    if (L[l].nchunk > 1) {
      patch_apply_time_parallel(l, r, y);
      return;
    }
    if (prof) {
      cudaEvent_t e0 = next_event(), e1 = next_event();
      WR_CUDA(cudaEventRecord(e0, s));
      launch_block_apply(L[l].g, tab, L[l].bs, L[l].factors, opt.precision, r, Yp, derr, s, nullptr, L[l].variant);
      WR_CUDA(cudaEventRecord(e1, s));
      prof_ev[l].push_back({e0, e1});
    } else {
      launch_block_apply(L[l].g, tab, L[l].bs, L[l].factors, opt.precision, r, Yp, derr, s, nullptr, L[l].variant);
    }
    launch_scatter(L[l].g, L[l].bs, Yp, y, s);
  }

  void coarse_solve(const double* b, double* x) {
    if (!linearised) throw WrError(WR_ERR_STATE, "wr_linearise must be called first");
    const LevelGeom& g = L[0].g;
    vec_zero(g.ndofs, x, s);
    if (heat) {
      heat_coarse_apply(g, tab, cfactors, b, x, s);
      return;
    }
    launch_block_apply(g, tab, cbs, cfactors, WR_FP64, b, x, derr, s);
    launch_project_pressure(g, tab, x, s);
  }

  // opt.cheb_steps steps of preconditioned Chebyshev iteration (Saad, Alg. 12.1)
  void smooth(int l, const double* b, double* x, bool zero_guess) {
    Level& lv = L[l];
    const int64_t n = lv.g.ndofs;
    if (!lv.lam_set) throw WrError(WR_ERR_STATE, "no eigen-estimate on this level");
    const double a = opt.cheb_lo * lv.lam, bb = opt.cheb_hi * lv.lam;
    const double theta = 0.5 * (bb + a), delta = 0.5 * (bb - a), sigma = theta / delta;
    if (zero_guess) {
      vec_zero(n, x, s);
      vec_copy(n, b, lv.r, s);
    } else {
      jac_inner(l, x, lv.t);
      vec_copy(n, b, lv.r, s);
      vec_axpby(n, -1.0, lv.t, 1.0, lv.r, s);
    }
    double rho = 1.0 / sigma;
    patch_apply(l, lv.r, lv.d);
    vec_scale(n, 1.0 / theta, lv.d, s);
    for (int step = 0; step < opt.cheb_steps; ++step) {
      vec_axpby(n, 1.0, lv.d, 1.0, x, s);
      if (step == opt.cheb_steps - 1) break;
      jac_inner(l, x, lv.t);
      vec_copy(n, b, lv.r, s);
      vec_axpby(n, -1.0, lv.t, 1.0, lv.r, s);
      patch_apply(l, lv.r, lv.z);
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      vec_axpby(n, 2.0 * rho_new / delta, lv.z, rho_new * rho, lv.d, s);
      rho = rho_new;
    }
  }

  void vcycle(const double* b, double* x) {
    const int T_ = top();
    std::vector<const double*> bl(T_ + 1);
    std::vector<double*> xl(T_ + 1);
    for (int l = 0; l <= T_; ++l) {
      bl[l] = L[l].b;
      xl[l] = L[l].x;
    }
    bl[T_] = b;
    xl[T_] = x;
    for (int l = T_; l >= 1; --l) {
      smooth(l, bl[l], xl[l], true);
      jac_inner(l, xl[l], L[l].t);
      vec_copy(L[l].g.ndofs, bl[l], L[l].r, s);
      vec_axpby(L[l].g.ndofs, -1.0, L[l].t, 1.0, L[l].r, s);
      restrict_to(l, L[l].r, L[l - 1].b);
    }
    coarse_solve(L[0].b, xl[0]);
    for (int l = 1; l <= T_; ++l) {
      prolong_add(l, xl[l - 1], xl[l]);
      smooth(l, bl[l], xl[l], false);
    }
    ++vcycles;
  }

  void linearise(const double* W, bool eig) {
    const int T_ = top();
    if (heat) {  // linear: the blocks do not depend on W
      for (int l = 1; l <= T_; ++l) heat_factor(L[l].g, tab, ph, false, static_cast<double*>(L[l].factors), fstat, s);
      heat_factor(L[0].g, tab, ph, true, cfactors, fstat, s);
      linearised = true;
      if (eig)
        for (int l = 1; l <= T_; ++l) eigen_estimate(l);
      return;
    }
    vec_copy(L[T_].g.ndofs, W, L[T_].W, s);
    for (int l = T_; l >= 1; --l) launch_inject(L[l].g, L[l - 1].g, L[l].W, L[l - 1].W, s);
    for (int l = 0; l <= T_; ++l) launch_wq(L[l].g, tab, L[l].W, L[l].Wq, s);
    for (int l = 1; l <= T_; ++l) {
      if (L[l].recompute) {  // one pass over the windows checks every block for a zero pivot
        for (int s0 = 0; s0 < L[l].g.N; s0 += L[l].nw) factor_window(l, s0, std::min(L[l].nw, L[l].g.N - s0), true);
        continue;
      }
      if (ph.conv != 0.0) launch_conv_elements(L[l].g, tab, L[l].W, Ce, opt.precision, s);
      launch_block_factor(L[l].g, tab, ph, L[l].bs, Ce, L[l].factors, opt.precision, fstat, s);
    }
    if (ph.conv != 0.0) launch_conv_elements(L[0].g, tab, L[0].W, Ce, WR_FP64, s);
    launch_block_factor(L[0].g, tab, ph, cbs, Ce, cfactors, WR_FP64, fstat, s);
    linearised = true;
    if (opt.autotune && q <= 1)  // DG(2), DG(3) have the one CTA tile
      for (int l = 1; l <= T_; ++l)
        if (!L[l].recompute && L[l].variant < 0 && L[l].nchunk == 1) {
          Level& lv = L[l];
          vec_zero(lv.g.ndofs, lv.x, s);
          const TuneKey key{0, k, q, opt.precision, (int64_t)lv.g.npatch(), lv.g.N};
          lv.variant = tune_apply_variant(key, s, [&](int v) {
            launch_block_apply(lv.g, tab, lv.bs, lv.factors, opt.precision, lv.x, Yp, derr, s, nullptr, v);
          });
        }
    for (int l = 1; l <= T_; ++l)
      if (L[l].nchunk > 1) build_transfer_matrices(l);
    if (eig)
      for (int l = 1; l <= T_; ++l) eigen_estimate(l);
  }

  // Largest real part of the Ritz values of opt.eig_steps Arnoldi (MGS) steps on M^{-1} J.
  void eigen_estimate(int l) {
    Level& lv = L[l];
    const int64_t n = lv.g.ndofs;
    const int m = opt.eig_steps;
    double* H = keH();
    if (heat) heat_splitmix(lv.g.ndofs, (uint64_t)l, V[0], s);
    else launch_splitmix_free(lv.g, (uint64_t)l, V[0], s);
    krylov_axpy_norm(n, nullptr, nullptr, V[0], partials, kcnt, kscal(), kscal() + 1, nullptr, 0.0, 0.0, s);
    vec_scale_dev(n, kscal() + 1, V[0], V[0], s);
    // all m steps run on the device; after a breakdown the basis vectors are zero
    for (int j = 0; j < m; ++j) {
      jac_inner(l, V[j], lv.t);
      patch_apply(l, lv.t, V[j + 1]);
      mgs_dev(n, H, m, j, true);
    }
    WR_CUDA(cudaMemcpyAsync(hk, H, sizeof(double) * (m + 1) * m, cudaMemcpyDeviceToHost, s));
    check_device();
    std::vector<double> Hh(hk, hk + (m + 1) * m);
    int mm = m;
    for (int j = 0; j < m; ++j)
      if (Hh[(j + 1) * m + j] <= 1e-14 * std::fabs(Hh[j * m + j]) + 1e-300) {
        mm = j + 1;
        break;
      }
    lv.lam = max_real_eigenvalue(Hh, mm, m);
    lv.lam_set = true;
  }

  // Eigenvalues of the leading mm x mm block of the upper Hessenberg H (row
  // stride ld) by the complex shifted QR algorithm with Wilkinson shifts and
  // deflation (Golub & Van Loan, Sec. 7.5); returns the largest real part.
  static double max_real_eigenvalue(const std::vector<double>& H, int mm, int ld) {
    using cd = std::complex<double>;
    std::vector<cd> A(mm * mm);
    for (int i = 0; i < mm; ++i)
      for (int j = 0; j < mm; ++j) A[i * mm + j] = H[i * ld + j];
    auto at = [&](int i, int j) -> cd& { return A[i * mm + j]; };
    int hi = mm - 1, its = 0;
    std::vector<double> cs(mm);
    std::vector<cd> sn(mm);
    while (hi > 0 && its < 200 * mm) {
      int lo = hi;
      while (lo > 0 && std::abs(at(lo, lo - 1)) > 1e-15 * (std::abs(at(lo, lo)) + std::abs(at(lo - 1, lo - 1)))) --lo;
      if (lo == hi) {
        --hi;
        its = 0;
        continue;
      }
      const cd a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
      const cd tr = a + d, det = a * d - b * c;
      const cd disc = std::sqrt(tr * tr / 4.0 - det);
      cd mu = (std::abs(tr / 2.0 + disc - d) < std::abs(tr / 2.0 - disc - d)) ? tr / 2.0 + disc : tr / 2.0 - disc;
      if (its > 0 && its % 11 == 0) mu = d + cd(std::abs(at(hi, hi - 1)), 0.0);  // exceptional shift
      for (int i = lo; i <= hi; ++i) at(i, i) -= mu;
      for (int i = lo; i < hi; ++i) {
        const cd x = at(i, i), y = at(i + 1, i);
        const double r = std::sqrt(std::norm(x) + std::norm(y));
        if (r == 0.0) { cs[i] = 1.0; sn[i] = 0.0; continue; }
        if (std::abs(x) == 0.0) {
          cs[i] = 0.0;
          sn[i] = 1.0;
        } else {
          cs[i] = std::abs(x) / r;
          sn[i] = (x / std::abs(x)) * std::conj(y) / r;
        }
        for (int j = i; j <= hi; ++j) {
          const cd u = at(i, j), v = at(i + 1, j);
          at(i, j) = cs[i] * u + sn[i] * v;
          at(i + 1, j) = -std::conj(sn[i]) * u + cs[i] * v;
        }
      }
      for (int i = lo; i < hi; ++i)
        for (int kk = lo; kk <= std::min(i + 1, hi); ++kk) {
          const cd u = at(kk, i), v = at(kk, i + 1);
          at(kk, i) = u * cs[i] + v * std::conj(sn[i]);
          at(kk, i + 1) = -u * sn[i] + v * cs[i];
        }
      for (int i = lo; i <= hi; ++i) at(i, i) += mu;
      ++its;
    }
    double best = -1e300;
    for (int i = 0; i < mm; ++i) best = std::max(best, at(i, i).real());
    return best;
  }

  // Right-preconditioned FGMRES with zero initial guess; returns iterations.  The
  // Arnoldi (MGS) coefficients, Givens rotations, least-squares solve and solution
  // update stay on the device; the host reads the residual estimate once per
  // iteration (the convergence test) and the true residual norm once per restart.
  int fgmres(const double* b, double* x, double tol) {
    Level& fl = fine();
    const int64_t n = fl.g.ndofs;
    const int m = opt.gmres_restart;
    double *H = kH(), *cs = kcs(), *sn = ksn(), *gg = kg();
    KrylovBasis zb{};
    for (int i = 0; i < m; ++i) zb.p[i] = Z[i];
    vec_zero(n, x, s);
    vec_copy(n, b, w, s);
    double beta = norm_dev(n, w);
    int its = 0;
    while (beta > tol && its < opt.gmres_maxit) {
      vec_scale_dev(n, kscal() + 1, w, V[0], s);  // V[0] = w / beta
      WR_CUDA(cudaMemcpyAsync(gg, kscal(), sizeof(double), cudaMemcpyDeviceToDevice, s));  // g = beta e_1
      int jend = 0;
      for (int j = 0; j < m; ++j) {
        check_cancel();
        vcycle(V[j], Z[j]);
        project(fl.g, Z[j]);
        jac(top(), Z[j], V[j + 1]);
        mgs_dev(n, H, m, j, false);
        krylov_givens(H, cs, sn, gg, j, m, kscal() + 3, s);
        const double res = read_scalar(kscal() + 3);
        ++its;
        jend = j + 1;
        if (!std::isfinite(res)) throw WrError(WR_ERR_NAN, "FGMRES residual is not finite");
        if (std::fabs(res) <= tol || its >= opt.gmres_maxit) break;
      }
      krylov_update(n, H, gg, ky(), jend, m, zb, x, s);
      jac(top(), x, w);
      vec_axpby(n, 1.0, b, -1.0, w, s);  // w = b - J x
      beta = norm_dev(n, w);
    }
    return its;
  }

  // Newton gives up early (WR_ERR_NOT_CONVERGED) once ||F|| exceeds newton_divtol ||F_0||
  // (divergence) or FGMRES has exhausted gmres_maxit in newton_stall consecutive steps.
  bool newton_gave_up(double fnorm, double f0, int stalls) const {
    if (opt.newton_divtol > 0.0 && fnorm > opt.newton_divtol * f0) return true;
    return opt.newton_stall > 0 && stalls >= opt.newton_stall;
  }

  int solve(double* U, wr_stats* st) {
    Level& fl = fine();
    const int64_t n = fl.g.ndofs;
    wr_stats loc;
    std::memset(&loc, 0, sizeof(loc));
    residual(U, F);
    double fnorm = norm(n, F);
    const double f0 = fnorm;
    double eta = opt.ew ? 0.5 : opt.eta_fixed;
    loc.residual_norms[0] = fnorm;
    int status = WR_ERR_NOT_CONVERGED;
    const int v0 = vcycles;
    int stalls = 0;  // consecutive Newton steps whose FGMRES ran out of iterations
    for (int it = 0; it < opt.newton_maxit && it < 64; ++it) {
      check_cancel();
      if (!std::isfinite(fnorm)) {
        status = WR_ERR_NAN;
        break;
      }
      if (fnorm <= opt.newton_rtol * f0) {
        status = WR_OK;
        break;
      }
      if (newton_gave_up(fnorm, f0, stalls)) break;  // diverged or stagnated
      double t0 = now_ms();
      linearise(U, true);
      WR_CUDA(cudaStreamSynchronize(s));
      double t1 = now_ms();
      loc.setup_ms += t1 - t0;
      vec_scale(n, -1.0, F, s);
      // FGMRES writes the Newton step into Z-independent scratch: reuse hx as the step
      const int its = fgmres(F, hx, eta * fnorm);
      WR_CUDA(cudaStreamSynchronize(s));
      loc.krylov_ms += now_ms() - t1;
      stalls = its >= opt.gmres_maxit ? stalls + 1 : 0;
      vec_axpby(n, 1.0, hx, 1.0, U, s);
      residual(U, F);
      const double fnew = norm(n, F);
      loc.gmres_its[loc.newton_its] = its;
      loc.newton_its++;
      loc.residual_norms[loc.newton_its] = fnew;
      if (opt.ew) {
        const double gamma = 0.9, alpha = 2.0;
        double en = gamma * std::pow(fnew / fnorm, alpha);
        const double safe = gamma * std::pow(eta, alpha);
        if (safe > 0.1) en = std::max(en, safe);
        eta = std::min(0.9, std::max(en, 0.5 * opt.newton_rtol * f0 / fnew));
      }
      fnorm = fnew;
    }
    if (status == WR_ERR_NOT_CONVERGED && std::isfinite(fnorm) && fnorm <= opt.newton_rtol * f0) status = WR_OK;
    loc.vcycles = vcycles - v0;
    if (st) *st = loc;
    return status;
  }
};

double hessenberg_max_real_eig(const std::vector<double>& H, int mm, int ld) {
  return wr_ctx::max_real_eigenvalue(H, mm, ld);
}

namespace {
thread_local std::string g_context_free_error;
}  // namespace

void wr_set_context_free_error(const std::string& msg) { g_context_free_error = msg; }

namespace {

int fail(wr_ctx* c, const WrError& e) {
  if (c) c->err = e.what();
  return e.code;
}

template <typename Fn>
int guarded(wr_ctx* c, Fn&& fn) {
  try {
    return fn();
  } catch (const WrError& e) {
    return fail(c, e);
  } catch (const std::exception& e) {
    if (c) c->err = e.what();
    return WR_ERR_CUDA;
  }
}

void need(bool cond, const char* msg) {
  if (!cond) throw WrError(WR_ERR_ARG, msg);
}

void check_level(const wr_ctx* c, int level, int lo) {
  need(level >= lo && level < (int)c->L.size(), "level out of range");
}

}  // namespace

extern "C" {

void wr_default_options(wr_options* o) {
  if (!o) return;
  o->precision = WR_FP64;
  o->cheb_steps = 2;
  o->cheb_lo = 0.25;
  o->cheb_hi = 1.05;
  o->eig_steps = 10;
  o->newton_rtol = 1e-8;
  o->newton_maxit = 20;
  o->ew = 1;
  o->eta_fixed = 1e-4;
  o->gmres_restart = 30;
  o->gmres_maxit = 200;
  o->patch_assembly = WR_PATCH_SUBMATRIX;
  o->scatter_weight = WR_WEIGHT_ONE;
  o->store_factors = WR_STORE;
  o->autotune = 1;
  o->apply_tile = -1;
  o->time_parallel = 0;
  o->newton_divtol = 1e6;
  o->newton_stall = 3;
  o->recompute_slabs = 0;
  o->memory_budget_mb = 0;
}

static int create_impl(wr_ctx* cptr, const wr_problem* p, const wr_options* o, void* stream);

int wr_create(wr_ctx** out, const wr_problem* p, const wr_options* o, void* stream) {
  if (!out || !p) return WR_ERR_ARG;
  *out = nullptr;
  auto c = std::make_unique<wr_ctx>();
  const int rc = create_impl(c.get(), p, o, stream);
  *out = c.release();
  return rc;
}

int wr_estimate_bytes(const wr_problem* p, const wr_options* o, int64_t* out) {
  if (!p || !out) return WR_ERR_ARG;
  wr_ctx c;
  c.dry = true;
  const int rc = create_impl(&c, p, o, nullptr);
  *out = c.bytes;
  return rc;
}

// The heat equation's hierarchy: FP64 stored inverses of every (patch, slab) block,
// the whole-mesh coarse block, and the same Krylov workspace as Navier-Stokes.
static int create_heat(wr_ctx* c, const wr_problem* p) {
  c->heat = true;
  c->opt.precision = WR_FP64;
  c->opt.store_factors = WR_STORE;
  c->opt.autotune = 0;
  c->tab = build_tables(p->k - 1, p->q);  // the degree-k tables are the Navier-Stokes velocity ones of k - 1
  const int m = heat_block_size(p->k, p->q, 0), mc = heat_block_size(p->k, p->q, p->n_coarse);
  size_t max_yp = 1;
  for (int n = p->n_coarse; n <= p->n_fine; n *= 2) {
    Level lv;
    lv.g = make_heat_geom(n, p->k, p->q, p->n_slabs, p->T);
    lv.bs.kind = 0;
    lv.bs.nvg = lv.bs.npg = 0;
    lv.bs.ms = m;
    const int64_t nd = lv.g.ndofs;
    lv.W = c->alloc<double>(1);
    lv.b = c->alloc<double>(nd);
    lv.x = c->alloc<double>(nd);
    lv.r = c->alloc<double>(nd);
    lv.d = c->alloc<double>(nd);
    lv.z = c->alloc<double>(nd);
    lv.t = c->alloc<double>(nd);
    if (n > p->n_coarse) {
      lv.factors = c->alloc<double>((size_t)lv.g.npatch() * p->n_slabs * m * m);
      max_yp = std::max(max_yp, (size_t)lv.g.npatch() * p->n_slabs * m);
    }
    lv.nw = p->n_slabs;
    c->L.push_back(lv);
  }
  c->cbs.kind = 1;
  c->cbs.ms = mc;
  c->cfactors = c->alloc<double>((size_t)p->n_slabs * mc * mc);
  c->Ce = c->alloc<double>(1);
  c->ye = c->alloc<double>(1);
  c->Yp = c->alloc<double>(max_yp);
  const int64_t nfine = c->fine().g.ndofs;
  const int nvec = std::max(c->opt.gmres_restart, c->opt.eig_steps) + 1;
  for (int i = 0; i < nvec; ++i) c->V.push_back(c->alloc<double>(nfine));
  for (int i = 0; i < c->opt.gmres_restart; ++i) c->Z.push_back(c->alloc<double>(nfine));
  c->F = c->alloc<double>(nfine);
  c->w = c->alloc<double>(nfine);
  c->hb = c->alloc<double>(nfine);
  c->hx = c->alloc<double>(nfine);
  c->partials = c->alloc<double>(dot_partials_size());
  c->dres = c->alloc<double>(1);
  c->kd = c->alloc<double>(wr_ctx::krylov_doubles(c->opt));
  c->kcnt = c->alloc<unsigned>(1);
  c->derr = c->alloc<int>(1);
  c->fstat = c->alloc<int>(1);
  c->u0 = c->alloc<double>(c->fine().g.S);
  c->htmp = c->alloc<double>(heat_op_scratch(c->fine().g));
  c->slots = c->alloc<int>(32);
  if (c->dry) return WR_OK;
  WR_CUDA(cudaMemsetAsync(c->derr, 0, sizeof(int), c->s));
  // zero Hessenbergs: the entries below the subdiagonal are never written
  WR_CUDA(cudaMemsetAsync(c->kd, 0, sizeof(double) * wr_ctx::krylov_doubles(c->opt), c->s));
  WR_CUDA(cudaMemsetAsync(c->kcnt, 0, sizeof(unsigned), c->s));
  WR_CUDA(cudaStreamSynchronize(c->s));
  WR_CUDA(cudaMallocHost(&c->hres, sizeof(double)));
  WR_CUDA(cudaMallocHost(&c->herr, sizeof(int)));
  WR_CUDA(cudaMallocHost(&c->hk, sizeof(double) * (c->opt.eig_steps + 1) * c->opt.eig_steps));
  *c->herr = 0;
  return WR_OK;
}

static int create_impl(wr_ctx* cptr, const wr_problem* p, const wr_options* o, void* stream) {
  wr_ctx* c = cptr;
  int rc = guarded(c, [&]() -> int {
    const bool heat = p->kind == WR_HEAT || p->kind == WR_HEAT_EIGEN;
    need(p->k == 1 || p->k == 2 || (heat && p->k == 3), "k must be 1 or 2 (1, 2 or 3 for the heat equation)");
    need(p->q >= 0 && p->q <= 3, "q must be 0..3");
    if (heat) {
      need(p->n_coarse == 1 || p->n_coarse == 2, "the heat equation coarsens to 1x1 or 2x2");
      need(heat_block_fits(p->k, p->q, p->n_coarse),
           "the coarse heat block does not fit in shared memory: coarsen to 1x1");
    } else {
      need(p->n_coarse == 2 || (p->n_coarse == 3 && p->k == 1), "n_coarse must be 2 (or 3 for k = 1)");
    }
    need(p->n_fine >= 4 && p->n_fine <= 4096, "n_fine out of range");
    need(p->n_slabs >= 1 && p->T > 0.0, "need n_slabs >= 1 and T > 0");
    int nf = p->n_fine;
    while (nf > p->n_coarse && nf % 2 == 0) nf /= 2;
    need(nf == p->n_coarse, "n_fine must be n_coarse times a power of two");
    need(p->kind >= WR_TAYLOR_GREEN && p->kind <= WR_HEAT_EIGEN, "unknown problem kind");
    need(p->n_modes >= 0 && p->n_modes <= 8, "at most 8 Fourier modes");
    need(p->n_modes == 0 || (p->mx && p->my && p->amp), "Fourier mode arrays missing");
    if (o) c->opt = *o;
    else wr_default_options(&c->opt);
    need(c->opt.precision == WR_FP64 || c->opt.precision == WR_FP32 || c->opt.precision == WR_BF16,
         "precision must be WR_FP64, WR_FP32 or WR_BF16");
    need(c->opt.cheb_steps >= 1 && c->opt.eig_steps >= 1 && c->opt.eig_steps <= c->opt.gmres_restart,
         "bad Chebyshev / eigen-estimate steps");
    need(c->opt.gmres_restart >= 1 && c->opt.gmres_restart <= kMaxKrylovBasis, "bad restart");
    need(c->opt.patch_assembly == WR_PATCH_SUBMATRIX || c->opt.patch_assembly == WR_PATCH_LOCAL,
         "patch_assembly must be WR_PATCH_SUBMATRIX or WR_PATCH_LOCAL");
    need(c->opt.scatter_weight == WR_WEIGHT_ONE || c->opt.scatter_weight == WR_WEIGHT_MULTIPLICITY,
         "scatter_weight must be WR_WEIGHT_ONE or WR_WEIGHT_MULTIPLICITY");
    if (!heat && p->q >= 2) {
      need(c->opt.precision == WR_FP64, "DG(2) and DG(3) run with FP64 factors");
      need(p->n_coarse == 2, "DG(2) and DG(3) coarsen to 2x2");
      need(c->opt.time_parallel == 0, "the parallel-in-time patch solve is built for DG(0) and DG(1)");
    }
    need(c->opt.store_factors == WR_STORE || c->opt.store_factors == WR_RECOMPUTE ||
             c->opt.store_factors == WR_STORE_AUTO,
         "store_factors must be WR_STORE, WR_RECOMPUTE or WR_STORE_AUTO");
    need(c->opt.recompute_slabs >= 0 && c->opt.memory_budget_mb >= 0, "bad recompute_slabs / memory_budget_mb");
    need(c->opt.apply_tile >= -1 && c->opt.apply_tile < kApplyTileVariants, "apply_tile must be -1 .. 4");
    c->s = static_cast<cudaStream_t>(stream);
    c->k = p->k; c->q = p->q; c->N = p->n_slabs; c->T = p->T;
    c->ph.kind = p->kind; c->ph.steady = p->steady; c->ph.nu = p->nu; c->ph.conv = p->conv; c->ph.T = p->T;
    c->ph.n_modes = p->n_modes;
    c->ph.t0 = p->t0;
    c->t0 = p->t0;
    for (int m = 0; m < p->n_modes; ++m) { c->ph.mx[m] = p->mx[m]; c->ph.my[m] = p->my[m]; c->ph.amp[m] = p->amp[m]; }
    if (heat) return create_heat(c, p);
    c->tab = build_tables(p->k, p->q);
    std::vector<int> ns;
    for (int n = p->n_coarse; n <= p->n_fine; n *= 2) ns.push_back(n);
    const int ms = patch_ms(p->k), nt = p->q + 1;
    const size_t fsz = factor_elem_bytes(c->opt.precision);
    const int nsmooth = (int)ns.size() - 1;
    const int nw = c->opt.recompute_slabs > 0 ? std::min(c->opt.recompute_slabs, p->n_slabs)
                                              : std::max(1, (p->n_slabs + 15) / 16);
    // how many of the finest smoothed levels recompute their factors
    int nrec = 0;
    if (c->forced_recompute >= 0) {
      nrec = c->forced_recompute;
    } else if (c->opt.store_factors == WR_RECOMPUTE) {
      nrec = nsmooth;
    } else if (c->opt.store_factors == WR_STORE_AUTO) {
      // the fewest recomputing levels whose allocations fit the budget (store all
      // when no budget is given and no device may be queried, as in a dry run)
      int64_t budget = (int64_t)c->opt.memory_budget_mb << 20;
      if (budget == 0 && !c->dry) {
        size_t fr = 0, tot = 0;
        WR_CUDA(cudaMemGetInfo(&fr, &tot));
        budget = (int64_t)(0.92 * (double)fr);
      }
      nrec = 0;
      if (budget > 0) {
        nrec = nsmooth;
        for (int r = 0; r <= nsmooth; ++r) {
          wr_ctx t;
          t.dry = true;
          t.forced_recompute = r;
          if (create_impl(&t, p, &c->opt, nullptr) == WR_OK && t.bytes <= budget) {
            nrec = r;
            break;
          }
        }
      }
    }
    size_t max_ce = 0, max_ye = 0, max_yp = 0, max_fw = 0;
    for (size_t l = 0; l < ns.size(); ++l) {
      Level lv;
      lv.g = make_geom(ns[l], p->k, p->q, p->n_slabs, p->T);
      lv.bs.kind = 0;
      lv.bs.nvg = patch_nvg(p->k);
      lv.bs.npg = patch_npg(p->k);
      lv.bs.ms = ms;
      lv.bs.local = c->opt.patch_assembly == WR_PATCH_LOCAL;
      lv.bs.weighted = c->opt.scatter_weight == WR_WEIGHT_MULTIPLICITY;
      const int64_t nd = lv.g.ndofs;
      lv.W = c->alloc<double>(nd);
      lv.Wq = c->alloc<double>(wq_doubles(lv.g));
      lv.b = c->alloc<double>(nd);
      lv.x = c->alloc<double>(nd);
      lv.r = c->alloc<double>(nd);
      lv.d = c->alloc<double>(nd);
      lv.z = c->alloc<double>(nd);
      lv.t = c->alloc<double>(nd);
      const size_t nvl = p->k + 2, nvle = nvl * nvl, elem = nt * (2 * nvle + (p->k + 1) * (p->k + 1));
      lv.recompute = l >= 1 && (int)l > nsmooth - nrec;
      lv.nw = lv.recompute ? nw : p->n_slabs;
      max_ce = std::max(max_ce, (size_t)lv.nw * lv.g.ncells() * nt * 4 * nvle * nvle);
      max_ye = std::max(max_ye, (size_t)p->n_slabs * lv.g.ncells() * elem);
      if (l >= 1) {
        const size_t per_slab = (size_t)lv.g.npatch() * nt * nt * factor_block_elems(p->k, c->opt.precision);
        if (lv.recompute) {
          max_fw = std::max(max_fw, per_slab * nw);
        } else {
          void* f = nullptr;
          if (fsz == 2) f = c->alloc<uint16_t>(per_slab * p->n_slabs);
          else if (fsz == 4) f = c->alloc<float>(per_slab * p->n_slabs);
          else f = c->alloc<double>(per_slab * p->n_slabs);
          lv.factors = f;
        }
        max_yp = std::max(max_yp, (size_t)lv.g.npatch() * p->n_slabs * nt * ms);
      }
      c->L.push_back(lv);
    }
    if (c->opt.apply_tile >= 0)
      for (auto& lv : c->L) lv.variant = c->opt.apply_tile;
    // time-parallel patch solve on the smoothed levels with too few patches to fill the
    // GPU: about one chunk per free CTA slot, at least 2 and at most N / 2 chunks
    int cap = 152 * (p->k == 1 ? 3 : 1);
    if (!c->dry) {
      int dev = 0, sms = 0;
      WR_CUDA(cudaGetDevice(&dev));
      WR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      cap = sms * (p->k == 1 ? 3 : 1);
    }
    for (size_t l = 1; l < c->L.size(); ++l) {
      Level& lv = c->L[l];
      if (lv.recompute || c->opt.time_parallel == 0 || p->n_slabs < 4) continue;
      const int np_ = lv.g.npatch();
      int C = 1;
      if (c->opt.time_parallel == 2) C = std::min(4, p->n_slabs / 2);
      else if (2 * np_ <= cap) C = std::min(cap / np_, p->n_slabs / 2);
      if (C < 2) continue;
      lv.Lc = (p->n_slabs + C - 1) / C;
      lv.nchunk = (p->n_slabs + lv.Lc - 1) / lv.Lc;
      if (lv.nchunk < 2) {
        lv.nchunk = 1;
        continue;
      }
      const int mv = 2 * lv.bs.nvg * lv.bs.nvg;
      lv.Tm = c->alloc<double>((size_t)np_ * lv.nchunk * mv * mv);
      lv.carry = c->alloc<double>((size_t)lv.nchunk * np_ * nt * ms);
    }
    c->cbs.kind = 1;
    c->cbs.nvg = c->L[0].g.nv - 2;
    c->cbs.npg = c->L[0].g.np;
    c->cbs.ms = coarse_ms(p->k, p->n_coarse);
    need(2 * c->cbs.nvg * c->cbs.nvg + c->cbs.npg * c->cbs.npg <= c->cbs.ms, "coarse block exceeds the slot layout");
    c->cfactors = c->alloc<double>((size_t)p->n_slabs * nt * nt * block_elems(c->cbs.ms, WR_FP64));
    if (max_fw > 0) {
      if (fsz == 2) c->fwin = c->alloc<uint16_t>(max_fw);
      else if (fsz == 4) c->fwin = c->alloc<float>(max_fw);
      else c->fwin = c->alloc<double>(max_fw);
    }
    c->Ce = c->alloc<double>(p->conv != 0.0 ? max_ce : 1);
    c->ye = c->alloc<double>(max_ye);
    c->Yp = c->alloc<double>(max_yp);
    const int64_t nfine = c->fine().g.ndofs;
    const int nvec = std::max(c->opt.gmres_restart, c->opt.eig_steps) + 1;
    for (int i = 0; i < nvec; ++i) c->V.push_back(c->alloc<double>(nfine));
    for (int i = 0; i < c->opt.gmres_restart; ++i) c->Z.push_back(c->alloc<double>(nfine));
    c->F = c->alloc<double>(nfine);
    c->w = c->alloc<double>(nfine);
    c->hb = c->alloc<double>(nfine);
    c->hx = c->alloc<double>(nfine);
    c->partials = c->alloc<double>(dot_partials_size());
    c->dres = c->alloc<double>(1);
    c->kd = c->alloc<double>(wr_ctx::krylov_doubles(c->opt));
    c->kcnt = c->alloc<unsigned>(1);
    c->slots = c->alloc<int>(2 * ms);
    c->derr = c->alloc<int>(1);
    c->fstat = c->alloc<int>(1);
    c->u0 = c->alloc<double>(c->fine().g.S);
    if (c->dry) return WR_OK;
    // on the context's stream: its memory may come from the stream-ordered pool
    WR_CUDA(cudaMemsetAsync(c->derr, 0, sizeof(int), c->s));
    // zero Hessenbergs: the entries below the subdiagonal are never written
    WR_CUDA(cudaMemsetAsync(c->kd, 0, sizeof(double) * wr_ctx::krylov_doubles(c->opt), c->s));
    WR_CUDA(cudaMemsetAsync(c->kcnt, 0, sizeof(unsigned), c->s));
    WR_CUDA(cudaStreamSynchronize(c->s));
    WR_CUDA(cudaMallocHost(&c->hres, sizeof(double)));
    WR_CUDA(cudaMallocHost(&c->herr, sizeof(int)));
    WR_CUDA(cudaMallocHost(&c->hk, sizeof(double) * (c->opt.eig_steps + 1) * c->opt.eig_steps));
    *c->herr = 0;
    return WR_OK;
  });
  return rc;  // on failure the context is still returned, so wr_last_error works
}

int wr_destroy(wr_ctx* c) {
  delete c;
  return WR_OK;
}

const char* wr_last_error(const wr_ctx* c) {
  if (c) return c->err.c_str();
  return g_context_free_error.empty() ? "null context" : g_context_free_error.c_str();
}

int wr_num_levels(const wr_ctx* c, int* out) {
  if (!c || !out) return WR_ERR_ARG;
  *out = (int)c->L.size();
  return WR_OK;
}

int wr_ndofs(const wr_ctx* c, int level, int64_t* out) {
  if (!c || !out || level < 0 || level >= (int)c->L.size()) return WR_ERR_ARG;
  *out = c->L[level].g.ndofs;
  return WR_OK;
}

int wr_apply_tile(const wr_ctx* c, int level, int* variant) {
  if (!c || !variant || level < 1 || level >= (int)c->L.size()) return WR_ERR_ARG;
  *variant = c->L[level].variant;
  return WR_OK;
}

int wr_factor_storage(const wr_ctx* c, int level, int* stored, int* window_slabs) {
  if (!c || level < 1 || level >= (int)c->L.size()) return WR_ERR_ARG;
  if (stored) *stored = c->L[level].recompute ? 0 : 1;
  if (window_slabs) *window_slabs = c->L[level].nw;
  return WR_OK;
}

int wr_device_bytes(const wr_ctx* c, int64_t* out) {
  if (!c || !out) return WR_ERR_ARG;
  *out = c->bytes;
  return WR_OK;
}

int wr_patch_dofs(const wr_ctx* cc, int level, int64_t patch, int slab, int64_t* idx, int* len) {
  wr_ctx* c = const_cast<wr_ctx*>(cc);
  return guarded(c, [&]() -> int {
    need(c != nullptr && idx != nullptr && len != nullptr, "null argument");
    check_level(c, level, 0);
    const Level& lv = c->L[level];
    need(patch >= 0 && patch < lv.g.npatch() && slab >= 0 && slab < lv.g.N, "patch or slab out of range");
    if (c->heat) {
      need(level >= 1, "the heat equation's coarsest level has no patches");
      const int np = heat_patch_slots(lv.g, (int)patch, c->slots, c->s);
      std::vector<int> sp(np);
      WR_CUDA(cudaMemcpyAsync(sp.data(), c->slots, sizeof(int) * np, cudaMemcpyDeviceToHost, c->s));
      WR_CUDA(cudaStreamSynchronize(c->s));
      int cnt = 0;
      for (int a = 0; a < lv.g.nt; ++a)
        for (int s = 0; s < np; ++s)
          if (sp[s] >= 0) idx[cnt++] = ((int64_t)slab * lv.g.nt + a) * lv.g.S + sp[s];
      *len = cnt;
      return WR_OK;
    }
    const int ms = lv.bs.ms;
    launch_patch_slots(lv.g, lv.bs, (int)patch, c->slots, c->s);
    std::vector<int> sp(ms);
    WR_CUDA(cudaMemcpyAsync(sp.data(), c->slots, sizeof(int) * ms, cudaMemcpyDeviceToHost, c->s));
    WR_CUDA(cudaStreamSynchronize(c->s));
    int cnt = 0;
    for (int a = 0; a < lv.g.nt; ++a)
      for (int s = 0; s < ms; ++s)
        if (sp[s] >= 0) idx[cnt++] = ((int64_t)slab * lv.g.nt + a) * lv.g.S + sp[s];
    *len = cnt;
    return WR_OK;
  });
}

int wr_initial_guess(wr_ctx* c, double* U) {
  return guarded(c, [&]() -> int {
    need(c && U, "null argument");
    if (c->heat) vec_zero(c->fine().g.ndofs, U, c->s);  // natural boundary conditions: start from zero
    else launch_boundary_values(c->fine().g, c->tab, c->ph, U, c->s);
    return WR_OK;
  });
}

int wr_residual(wr_ctx* c, const double* U, double* F) {
  return guarded(c, [&]() -> int {
    need(c && U && F && U != F, "null or aliased argument");
    c->residual(U, F);
    return WR_OK;
  });
}

int wr_linearise(wr_ctx* c, const double* W) {
  return guarded(c, [&]() -> int {
    need(c && W, "null argument");
    c->linearise(W, true);
    return WR_OK;
  });
}

int wr_linearise_no_eig(wr_ctx* c, const double* W) {
  return guarded(c, [&]() -> int {
    need(c && W, "null argument");
    c->linearise(W, false);
    return WR_OK;
  });
}

int wr_get_lambda(const wr_ctx* c, int level, double* lam) {
  if (!c || !lam || level < 1 || level >= (int)c->L.size()) return WR_ERR_ARG;
  if (!c->L[level].lam_set) return WR_ERR_STATE;
  *lam = c->L[level].lam;
  return WR_OK;
}

int wr_set_lambda(wr_ctx* c, int level, double lam) {
  if (!c || level < 1 || level >= (int)c->L.size() || !(lam > 0.0)) return WR_ERR_ARG;
  c->L[level].lam = lam;
  c->L[level].lam_set = true;
  return WR_OK;
}

int wr_apply_jacobian(wr_ctx* c, int level, const double* x, double* y) {
  return guarded(c, [&]() -> int {
    need(c && x && y && x != y, "null or aliased argument");
    check_level(c, level, 0);
    c->jac(level, x, y);
    return WR_OK;
  });
}

int wr_patch_apply(wr_ctx* c, int level, const double* r, double* y) {
  return guarded(c, [&]() -> int {
    need(c && r && y && r != y, "null or aliased argument");
    check_level(c, level, 1);
    c->patch_apply(level, r, y);
    return WR_OK;
  });
}

int wr_smooth(wr_ctx* c, int level, const double* b, double* x, int zero_guess) {
  return guarded(c, [&]() -> int {
    need(c && b && x && b != x, "null or aliased argument");
    check_level(c, level, 1);
    c->smooth(level, b, x, zero_guess != 0);
    return WR_OK;
  });
}

int wr_restrict(wr_ctx* c, int fine_level, const double* xf, double* xc) {
  return guarded(c, [&]() -> int {
    need(c && xf && xc, "null argument");
    check_level(c, fine_level, 1);
    c->restrict_to(fine_level, xf, xc);
    return WR_OK;
  });
}

int wr_prolong_add(wr_ctx* c, int fine_level, const double* xc, double* xf) {
  return guarded(c, [&]() -> int {
    need(c && xf && xc, "null argument");
    check_level(c, fine_level, 1);
    c->prolong_add(fine_level, xc, xf);
    return WR_OK;
  });
}

int wr_coarse_solve(wr_ctx* c, const double* b, double* x) {
  return guarded(c, [&]() -> int {
    need(c && b && x && b != x, "null or aliased argument");
    c->coarse_solve(b, x);
    return WR_OK;
  });
}

int wr_vcycle(wr_ctx* c, const double* b, double* x) {
  return guarded(c, [&]() -> int {
    need(c && b && x && b != x, "null or aliased argument");
    c->vcycle(b, x);
    return WR_OK;
  });
}

int wr_vcycle_host(wr_ctx* c, const double* b_host, double* x_host) {
  return guarded(c, [&]() -> int {
    need(c && b_host && x_host, "null argument");
    const int64_t n = c->fine().g.ndofs;
    WR_CUDA(cudaMemcpyAsync(c->hb, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
    c->vcycle(c->hb, c->hx);
    WR_CUDA(cudaMemcpyAsync(x_host, c->hx, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
    c->check_device();
    return WR_OK;
  });
}

int wr_project_pressure(wr_ctx* c, double* x) {
  return guarded(c, [&]() -> int {
    need(c && x, "null argument");
    c->project(c->fine().g, x);
    return WR_OK;
  });
}

int wr_solve(wr_ctx* c, double* U, wr_stats* st) {
  return guarded(c, [&]() -> int {
    need(c && U, "null argument");
    const int rc = c->solve(U, st);
    if (rc == WR_ERR_NOT_CONVERGED) c->err = "Newton iteration limit reached";
    if (rc == WR_ERR_NAN) c->err = "residual norm is not finite";
    return rc;
  });
}

int wr_set_initial_state(wr_ctx* c, const double* u0) {
  return guarded(c, [&]() -> int {
    need(c != nullptr, "null context");
    if (!u0) {
      c->ph.u0 = nullptr;
      return WR_OK;
    }
    WR_CUDA(cudaMemcpyAsync(c->u0, u0, sizeof(double) * c->fine().g.S, cudaMemcpyDeviceToDevice, c->s));
    c->ph.u0 = c->u0;
    return WR_OK;
  });
}

int wr_solve_timestepping(wr_ctx* c, int n_steps, double* U, wr_stats* st) {
  return guarded(c, [&]() -> int {
    need(c && U && n_steps >= 1, "null argument or n_steps < 1");
    need(c->N == 1, "the timestepping comparator needs a one-slab context");
    const LevelGeom& g = c->fine().g;
    const int64_t step = g.ndofs, last = (int64_t)(g.nt - 1) * g.S;
    wr_stats tot;
    std::memset(&tot, 0, sizeof(tot));
    int status = WR_OK;
    for (int i = 0; i < n_steps; ++i) {
      double* Ui = U + i * step;
      c->ph.t0 = c->t0 + i * c->T;
      if (i > 0) {  // the previous step's end state, held in the context's own buffer
        WR_CUDA(cudaMemcpyAsync(c->u0, Ui - step + last, sizeof(double) * g.S, cudaMemcpyDeviceToDevice, c->s));
        c->ph.u0 = c->u0;
      }
      if (c->heat) vec_zero(g.ndofs, Ui, c->s);
      else launch_boundary_values(g, c->tab, c->ph, Ui, c->s);
      wr_stats si;
      const int rc = c->solve(Ui, &si);
      tot.newton_its += si.newton_its;
      tot.vcycles += si.vcycles;
      tot.setup_ms += si.setup_ms;
      tot.krylov_ms += si.krylov_ms;
      if (i < 64) {
        for (int j = 0; j < si.newton_its && j < 64; ++j) tot.gmres_its[i] += si.gmres_its[j];
        tot.residual_norms[i] = si.residual_norms[si.newton_its < 64 ? si.newton_its : 64];
      }
      if (rc != WR_OK && status == WR_OK) status = rc;
    }
    c->ph.t0 = c->t0;
    if (st) *st = tot;
    if (status == WR_ERR_NOT_CONVERGED) c->err = "Newton iteration limit reached in a time step";
    return status;
  });
}

int wr_solve_host(wr_ctx* c, double* U_host, wr_stats* st) {
  return guarded(c, [&]() -> int {
    need(c && U_host, "null argument");
    const int64_t n = c->fine().g.ndofs;
    WR_CUDA(cudaMemcpyAsync(c->hb, U_host, sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
    const int rc = c->solve(c->hb, st);
    WR_CUDA(cudaMemcpyAsync(U_host, c->hb, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
    WR_CUDA(cudaStreamSynchronize(c->s));
    if (rc == WR_ERR_NOT_CONVERGED) c->err = "Newton iteration limit reached";
    return rc;
  });
}

int wr_launch_count(int64_t* out) {
  if (!out) return WR_ERR_ARG;
  *out = g_launches.load();
  return WR_OK;
}

int wr_profile(wr_ctx* c, int enable) {
  return guarded(c, [&]() -> int {
    need(c != nullptr, "null context");
    WR_CUDA(cudaStreamSynchronize(c->s));
    c->prof = enable != 0;
    c->prof_ev.assign(c->L.size(), {});
    c->prof_jac.assign(c->L.size(), {});
    c->ev_used = 0;
    // create the events now so that none is created inside a timed region
    while (c->prof && c->ev_pool.size() < 4096) {
      cudaEvent_t e;
      WR_CUDA(cudaEventCreate(&e));
      c->ev_pool.push_back(e);
    }
    return WR_OK;
  });
}

int wr_profile_smoother(wr_ctx* c, int level, double* total_ms, int* launches) {
  return guarded(c, [&]() -> int {
    need(c && total_ms && launches, "null argument");
    check_level(c, level, 1);
    need(level < (int)c->prof_ev.size(), "profiling not enabled");
    WR_CUDA(cudaStreamSynchronize(c->s));
    double tot = 0.0;
    for (auto& pr : c->prof_ev[level]) {
      float ms = 0.f;
      WR_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
      tot += ms;
    }
    *total_ms = tot;
    *launches = (int)c->prof_ev[level].size();
    return WR_OK;
  });
}

int wr_profile_jacobian(wr_ctx* c, int level, double* total_ms, int* launches, double* flops_per_launch) {
  return guarded(c, [&]() -> int {
    need(c && total_ms && launches, "null argument");
    check_level(c, level, 0);
    need(!c->heat, "the heat equation has no element kernel");
    need(level < (int)c->prof_jac.size(), "profiling not enabled");
    WR_CUDA(cudaStreamSynchronize(c->s));
    double tot = 0.0;
    for (auto& pr : c->prof_jac[level]) {
      float ms = 0.f;
      WR_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
      tot += ms;
    }
    *total_ms = tot;
    *launches = (int)c->prof_jac[level].size();
    const LevelGeom& g = c->L[level].g;
    if (flops_per_launch) *flops_per_launch = jac_flops_per_cell_slab(g.k, g.q) * g.ncells() * g.N;
    return WR_OK;
  });
}

int wr_measure_fp64_tflops(void* stream, double* out) {
  if (!out) return WR_ERR_ARG;
  try {
    *out = measure_fp64_tflops(static_cast<cudaStream_t>(stream));
    return WR_OK;
  } catch (const WrError& e) {
    return e.code;
  }
}

}  // extern "C"

int create_context(wr_ctx** out, const wr_problem* p, const wr_options* o, void* stream, bool stream_ordered) {
  if (!out || !p) return WR_ERR_ARG;
  *out = nullptr;
  auto c = std::make_unique<wr_ctx>();
  c->stream_ordered = stream_ordered;
  const int rc = create_impl(c.get(), p, o, stream);
  *out = c.release();
  return rc;
}

void set_cancel_flag(wr_ctx* c, const std::atomic<int>* flag) { c->cancel = flag; }

extern "C" {

int wr_inject_alloc_failure(int64_t nth) {
  if (nth < 0) return WR_ERR_ARG;
  g_fail_alloc.store(nth);
  return WR_OK;
}

int wr_selftest_bounded_wait(void* stream, int* timed_out, double* waited_ms) {
  if (!timed_out || !waited_ms) return WR_ERR_ARG;
  try {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* d = nullptr;
    WR_CUDA(cudaMalloc(&d, 16));
    std::unique_ptr<void, void (*)(void*)> hold(d, [](void* q) { cudaFree(q); });
    int* flag = static_cast<int*>(d);
    unsigned long long* ns = reinterpret_cast<unsigned long long*>(static_cast<char*>(d) + 8);
    launch_bounded_wait_selftest(flag, ns, s);
    int h = 0;
    unsigned long long hn = 0;
    WR_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaMemcpyAsync(&hn, ns, sizeof(hn), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    *timed_out = h;
    *waited_ms = hn * 1e-6;
    return WR_OK;
  } catch (const WrError& e) {
    return e.code;
  }
}

}  // extern "C"
