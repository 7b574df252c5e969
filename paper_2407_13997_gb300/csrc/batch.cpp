// Batching form: many independent space-time solves (uneven meshes, slab counts,
// viscosities and forcings; one Taylor-Hood order and DG order per batch)
// advanced in lock step, with one launch per stage for all members.
//
// Layout.  Member m has levels 0 (coarsest) .. L_m; "depth" d = L_m - level
// counts from every member's finest level.  For each depth the vectors of all
// members that have a level there are concatenated in one arena per role
// (b, x, r, d, z, t), so every stage of the V-cycle (Algorithm Vcycle) is one
// batched launch over a device table of BatchSeg entries, and the smoother is a
// single persistent launch over every member's patches.  Coarse solves of all
// members run in one launch per coarse-block shape.  Newton, FGMRES and the
// Chebyshev/Arnoldi scalars are per member on the host; members that converge
// leave the active set and the tables are rebuilt without them.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>

#include "wrmg_internal.h"

namespace {

struct Member {
  PhysParams ph;
  int nc = 2, L = 0;
  std::vector<LevelGeom> g;  // 0 .. L
  std::vector<double*> W;
  std::vector<void*> factors;  // per level (index 0 unused)
  double* cf = nullptr;
  BlockSet cbs;
  std::vector<double> lam;
};

struct Arena {
  double *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr, *z = nullptr, *t = nullptr;
};

struct Table {
  std::vector<BatchSeg> h;
  std::vector<int> members;
  BatchSeg* d = nullptr;  // device copy, capacity B
  int n = 0;
  int64_t units = 0, dofs = 0, dofsc = 0, items = 0, tblks = 0;
  double* coef = nullptr;  // device: per-segment coefficient rows (Chebyshev), kCoefRows x B
};

constexpr int kCoefRows = 16;

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct wr_batch {
  std::string err;
  cudaStream_t s = nullptr;
  wr_options opt;
  int k = 1, q = 0, nt = 1;
  FeTables tab;
  std::vector<Member> mem;
  int B = 0, D = 0;
  std::vector<std::vector<int64_t>> off, off_ye, off_yp;  // [depth][member], -1 = absent
  std::vector<int64_t> arena_size;
  std::vector<Arena> ar;
  double *ye = nullptr, *yp = nullptr, *Ce = nullptr;
  std::vector<double*> V, Z;
  double *F = nullptr, *w = nullptr, *step = nullptr, *U = nullptr, *vb = nullptr, *vx = nullptr;
  double *partials = nullptr, *dres = nullptr, *hres = nullptr, *hcoef = nullptr, *dcoef = nullptr;
  int64_t* dseeds = nullptr;
  // device-resident Krylov scalars, member-indexed: FGMRES Hessenberg ((R+1) x R),
  // rotations (R), right-hand side (R+1) and least-squares solution (R); the Arnoldi
  // Hessenberg of the eigen-estimate ((e+1) x e); norms, reciprocals and statuses
  double *kH = nullptr, *kcs = nullptr, *ksn = nullptr, *kg = nullptr, *ky = nullptr, *keH = nullptr;
  double *kbeta = nullptr, *kinv = nullptr, *kstat = nullptr;
  double* hkH = nullptr;  // pinned host copy of keH
  // set for one solve by batch_solve_hooked: a member's result is copied to Uout[m]
  // and on_done(m, status) runs as soon as it leaves the lock-step set; a member whose
  // cancel flag is set leaves with WR_ERR_CANCELLED
  double* const* Uout = nullptr;
  const std::atomic<int>* const* member_cancel = nullptr;
  std::function<void(int, int)> on_done;
  int *derr = nullptr, *herr = nullptr, *fstat = nullptr;
  std::vector<char> active;
  std::vector<Table> smooth;  // per depth: members with a smoothing level there
  Table coarse2, coarse3, fine;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  bool linearised = false;

  template <typename Tp>
  Tp* alloc(size_t count) {
    void* p = nullptr;
    const size_t nb = std::max<size_t>(count * sizeof(Tp), 16);
    if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1)
      throw WrError(WR_ERR_NOMEM, "injected allocation failure (wr_inject_alloc_failure)");
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw WrError(WR_ERR_NOMEM, "cudaMalloc of " + std::to_string(nb) + " bytes failed; " +
                                      std::to_string(bytes) + " bytes already held by the batch");
    }
    allocs.push_back(p);
    bytes += nb;
    return static_cast<Tp*>(p);
  }
  ~wr_batch() {
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* p : allocs) cudaFree(p);
    if (hres) cudaFreeHost(hres);
    if (hcoef) cudaFreeHost(hcoef);
    if (hkH) cudaFreeHost(hkH);
    if (herr) cudaFreeHost(herr);
  }

  BlockSet patch_set() const {
    BlockSet bs;
    bs.kind = 0;
    bs.nvg = patch_nvg(k);
    bs.npg = patch_npg(k);
    bs.ms = patch_ms(k);
    bs.local = opt.patch_assembly == WR_PATCH_LOCAL;
    bs.weighted = opt.scatter_weight == WR_WEIGHT_MULTIPLICITY;
    return bs;
  }
  int64_t elem_size() const { return (int64_t)nt * (2 * (k + 2) * (k + 2) + (k + 1) * (k + 1)); }

  // ---------------------------------------------------------------- tables
  void upload(Table& t) {
    t.n = (int)t.h.size();
    if (!t.d) {
      t.d = alloc<BatchSeg>(B);
      t.coef = alloc<double>((size_t)kCoefRows * B);
    }
    if (t.n) WR_CUDA(cudaMemcpyAsync(t.d, t.h.data(), sizeof(BatchSeg) * t.n, cudaMemcpyHostToDevice, s));
  }

  void add_seg(Table& t, int m, int d, bool coarse_block) {
    const Member& M = mem[m];
    const int l = M.L - d;
    BatchSeg sg;
    std::memset(&sg, 0, sizeof(sg));
    sg.g = M.g[l];
    sg.gc = l >= 1 ? M.g[l - 1] : M.g[l];
    sg.ph = M.ph;
    sg.member = m;
    sg.off = off[d][m];
    sg.offc = (l >= 1 && d + 1 < D) ? off[d + 1][m] : 0;
    sg.off_ye = off_ye[d][m] >= 0 ? off_ye[d][m] : 0;
    sg.off_yp = off_yp[d][m] >= 0 ? off_yp[d][m] : 0;
    sg.W = M.W[l];
    if (coarse_block) {
      sg.bs = M.cbs;
      sg.factors = M.cf;
      sg.xa = ar[d].b + off[d][m];
      sg.ya = ar[d].x + off[d][m];
    } else {
      sg.bs = patch_set();
      sg.factors = l >= 1 ? M.factors[l] : nullptr;
    }
    sg.u_elem = t.units;
    sg.u_dof = t.dofs;
    sg.u_dofc = t.dofsc;
    sg.u_patch = t.items;
    sg.u_tblk = t.tblks;
    t.units += elem_units(sg.g);
    t.dofs += sg.g.ndofs;
    t.dofsc += l >= 1 ? sg.gc.ndofs : 0;
    t.items += coarse_block ? 1 : sg.g.npatch();
    t.tblks += (int64_t)sg.g.N * sg.g.nt;
    t.h.push_back(sg);
    t.members.push_back(m);
  }

  void reset(Table& t) {
    t.h.clear();
    t.members.clear();
    t.units = t.dofs = t.dofsc = t.items = t.tblks = 0;
  }

  void build_tables() {
    ++table_ver;
    smooth.resize(D);
    for (int d = 0; d < D; ++d) {
      reset(smooth[d]);
      for (int m = 0; m < B; ++m)
        if (active[m] && mem[m].L - d >= 1) add_seg(smooth[d], m, d, false);
      upload(smooth[d]);
    }
    reset(coarse2);
    reset(coarse3);
    reset(fine);
    for (int m = 0; m < B; ++m) {
      if (!active[m]) continue;
      add_seg(mem[m].nc == 3 ? coarse3 : coarse2, m, mem[m].L, true);
      add_seg(fine, m, 0, false);
    }
    upload(coarse2);
    upload(coarse3);
    upload(fine);
    if (linearised) upload_chebyshev();
  }

  // per-segment Chebyshev coefficients of every smoothing table (rows: 1/theta, then (c1, c2) per step)
  void upload_chebyshev() {
    ++table_ver;  // the graph reads the coefficient arrays; re-capture after a change
    const int steps = opt.cheb_steps;
    for (int d = 0; d < D; ++d) {
      Table& t = smooth[d];
      if (!t.n) continue;
      std::vector<double> rows((size_t)kCoefRows * B, 0.0);
      for (int i = 0; i < t.n; ++i) {
        const Member& M = mem[t.members[i]];
        const double lam = M.lam[M.L - d];
        const double a = opt.cheb_lo * lam, bb = opt.cheb_hi * lam;
        const double theta = 0.5 * (bb + a), delta = 0.5 * (bb - a), sigma = theta / delta;
        rows[0 * B + i] = 1.0 / theta;
        double rho = 1.0 / sigma;
        for (int st = 1; st < steps && 2 * st < kCoefRows; ++st) {
          const double rho_new = 1.0 / (2.0 * sigma - rho);
          rows[(size_t)(2 * st - 1) * B + i] = rho_new * rho;
          rows[(size_t)(2 * st) * B + i] = 2.0 * rho_new / delta;
          rho = rho_new;
        }
      }
      WR_CUDA(cudaMemcpyAsync(t.coef, rows.data(), sizeof(double) * rows.size(), cudaMemcpyHostToDevice, s));
    }
  }

  // ---------------------------------------------------------------- batched stages
  std::vector<double> dots(const Table& t, const double* x, const double* y) {
    std::vector<double> out(t.n);
    if (!t.n) return out;
    bt_dot(t.d, t.n, x, y, partials, dres, s);
    WR_CUDA(cudaMemcpyAsync(hres, dres, sizeof(double) * t.n, cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    if (*herr) throw WrError(WR_ERR_TIMEOUT, "a bounded wait in the smoother kernel gave up");
    std::copy(hres, hres + t.n, out.begin());
    return out;
  }
  // per-segment coefficients to the device; the stream is drained first so that the
  // pinned staging row is not overwritten while an earlier copy from it is pending
  const double* coefs(const std::vector<double>& c) {
    WR_CUDA(cudaStreamSynchronize(s));
    std::copy(c.begin(), c.end(), hcoef);
    WR_CUDA(cudaMemcpyAsync(dcoef, hcoef, sizeof(double) * c.size(), cudaMemcpyHostToDevice, s));
    return dcoef;
  }

  void jac(const Table& t, const double* x, double* y) {
    if (t.n) bt_jacobian(k, q, t.d, t.n, t.units, t.dofs, tab, x, y, ye, s);
  }  // inside the preconditioner: single-precision element arithmetic in the reduced-precision forms
  void jac_inner(const Table& t, const double* x, double* y) {
    if (opt.precision == WR_FP64) jac(t, x, y);
    else if (t.n) bt_jacobian_f32(k, q, t.d, t.n, t.units, t.dofs, tab, x, y, ye, s);
  }

  void papply(const Table& t, int d, const double* r, double* y) {
    if (t.n) bt_block_apply(k, q, opt.precision, t.d, t.n, t.items, t.dofs, tab, r, y, yp, derr, 0, s, depth_variant[d]);
  }
  void residual_b_minus(const Table& t, const double* b, double* x, double* tmp, double* r) {
    jac_inner(t, x, tmp);
    bt_copy(t.d, t.n, t.dofs, b, r, s);
    bt_axpby(t.d, t.n, t.dofs, nullptr, -1.0, tmp, nullptr, 1.0, r, s);
  }

  void smooth_depth(int d, const double* b, double* x, bool zero_guess) {
    Table& t = smooth[d];
    if (!t.n) return;
    Arena& a = ar[d];
    if (zero_guess) {
      bt_axpby(t.d, t.n, t.dofs, nullptr, 0.0, x, nullptr, 0.0, x, s);
      bt_copy(t.d, t.n, t.dofs, b, a.r, s);
    } else {
      residual_b_minus(t, b, x, a.t, a.r);
    }
    papply(t, d, a.r, a.d);
    bt_axpby(t.d, t.n, t.dofs, nullptr, 0.0, a.d, t.coef, 0.0, a.d, s);  // d = M^{-1} r / theta
    for (int st = 0; st < opt.cheb_steps; ++st) {
      bt_axpby(t.d, t.n, t.dofs, nullptr, 1.0, a.d, nullptr, 1.0, x, s);
      if (st == opt.cheb_steps - 1) break;
      residual_b_minus(t, b, x, a.t, a.r);
      papply(t, d, a.r, a.z);
      const int row = 2 * (st + 1);
      bt_axpby(t.d, t.n, t.dofs, t.coef + (size_t)row * B, 0.0, a.z, t.coef + (size_t)(row - 1) * B, 0.0, a.d, s);
    }
  }

  void coarse_solves() {
    for (Table* t : {&coarse2, &coarse3}) {
      if (!t->n) continue;
      bt_fill_abs(t->d, t->n, t->dofs, 0.0, s);
      bt_block_apply(k, q, WR_FP64, t->d, t->n, t->items, 0, tab, nullptr, nullptr, nullptr, derr,
                     t == &coarse3 ? 3 : 2, s);
      bt_project_pressure(t->d, t->n, t->tblks, tab, nullptr, true, s);
    }
  }

  // The V-cycle of the current tables as one CUDA graph: it reads vb and writes vx
  // (depth-0 arenas), is captured after the tables or the Chebyshev coefficients
  // change (an eager cycle runs first, so every kernel's one-time set-up is done),
  // and replays as one launch.
  std::vector<int> depth_variant = std::vector<int>(16, -1);  // tuned apply tile per depth
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap_stream = nullptr;
  int64_t table_ver = 0, graph_ver = -1, graph_kernels = 0;
  bool use_graphs = true;

  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    graph_ver = -1;
  }

  void vcycle_graph() {
    if (!use_graphs) {
      vcycle(vb, vx);
      return;
    }
    if (graph_ver != table_ver) {
      drop_graph();
      vcycle(vb, vx);  // eager: one-time kernel attributes, and this call's result
      // capture on a private stream (the caller's may be the legacy default stream,
      // which cannot capture); the graph is launched on the caller's stream
      if (!cap_stream) WR_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
      cudaGraph_t graph = nullptr;
      int64_t before = 0;
      wr_launch_count(&before);
      WR_CUDA(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
      std::swap(s, cap_stream);
      try {
        vcycle(vb, vx);
      } catch (...) {
        std::swap(s, cap_stream);
        cudaStreamEndCapture(cap_stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      std::swap(s, cap_stream);
      const cudaError_t ce = cudaStreamEndCapture(cap_stream, &graph);
      int64_t after = 0;
      wr_launch_count(&after);
      wr_uncount_launches(after - before);  // captured, not launched
      if (ce != cudaSuccess || !graph) throw WrError(WR_ERR_CUDA, "V-cycle graph capture failed");
      const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) throw WrError(WR_ERR_CUDA, "V-cycle graph instantiation failed");
      graph_kernels = after - before;
      graph_ver = table_ver;
      return;
    }
    WR_CUDA(cudaGraphLaunch(gexec, s));
    wr_count_launches(graph_kernels);
  }

  // one V(2,2) cycle of every active member through the graph: x0 = V-cycle(b0)
  void vcycle_via_graph(const double* b0, double* x0) {
    bt_copy(fine.d, fine.n, fine.dofs, b0, vb, s);
    vcycle_graph();
    bt_copy(fine.d, fine.n, fine.dofs, vx, x0, s);
  }

  // one V(2,2) cycle of every active member: b0, x0 are depth-0 arena vectors
  void vcycle(const double* b0, double* x0) {
    for (int d = 0; d < D; ++d) {
      Table& t = smooth[d];
      if (!t.n) continue;
      const double* b = d == 0 ? b0 : ar[d].b;
      double* x = d == 0 ? x0 : ar[d].x;
      smooth_depth(d, b, x, true);
      residual_b_minus(t, b, x, ar[d].t, ar[d].r);
      bt_restrict(t.d, t.n, t.dofsc, tab, ar[d].r, ar[d + 1].b, s);
    }
    coarse_solves();
    for (int d = D - 1; d >= 0; --d) {
      Table& t = smooth[d];
      if (!t.n) continue;
      const double* b = d == 0 ? b0 : ar[d].b;
      double* x = d == 0 ? x0 : ar[d].x;
      bt_prolong_add(t.d, t.n, t.dofs, tab, ar[d + 1].x, x, s);
      smooth_depth(d, b, x, false);
    }
  }

  // ---------------------------------------------------------------- setup
  void linearise_members(const double* Warena) {
    for (int m = 0; m < B; ++m) {
      if (!active[m]) continue;
      Member& M = mem[m];
      WR_CUDA(cudaMemcpyAsync(M.W[M.L], Warena + off[0][m], sizeof(double) * M.g[M.L].ndofs,
                              cudaMemcpyDeviceToDevice, s));
      for (int l = M.L; l >= 1; --l) launch_inject(M.g[l], M.g[l - 1], M.W[l], M.W[l - 1], s);
      for (int l = 1; l <= M.L; ++l) {
        if (M.ph.conv != 0.0) launch_conv_elements(M.g[l], tab, M.W[l], Ce, opt.precision, s);
        launch_block_factor(M.g[l], tab, M.ph, patch_set(), Ce, M.factors[l], opt.precision, fstat, s);
      }
      if (M.ph.conv != 0.0) launch_conv_elements(M.g[0], tab, M.W[0], Ce, WR_FP64, s);
      launch_block_factor(M.g[0], tab, M.ph, M.cbs, Ce, M.cf, WR_FP64, fstat, s);
    }
    build_tables();
    if (opt.autotune)
      for (int d = 0; d < D; ++d) {
        Table& t = smooth[d];
        if (!t.n || depth_variant[d] >= 0) continue;
        bt_axpby(t.d, t.n, t.dofs, nullptr, 0.0, ar[d].x, nullptr, 0.0, ar[d].x, s);
        const TuneKey key{1, k, q, opt.precision, t.items, 0};
        depth_variant[d] = tune_apply_variant(key, s, [&](int v) {
          bt_block_apply(k, q, opt.precision, t.d, t.n, t.items, t.dofs, tab, ar[d].x, ar[d].d, yp, derr, 0, s, v);
        });
      }
    for (int d = 0; d < D; ++d) eigen_depth(d);
    linearised = true;
    upload_chebyshev();
  }

  // 10-step Arnoldi (MGS) on M^{-1} J for every member with a smoothing level at depth
  // d, all on the device (after a member's breakdown its basis vectors are zero); the
  // host reads the Hessenbergs once at the end
  void eigen_depth(int d) {
    Table& t = smooth[d];
    if (!t.n) return;
    const int ne = opt.eig_steps;
    const int64_t es = (int64_t)(ne + 1) * ne;
    std::vector<int64_t> seeds(t.n);
    for (int i = 0; i < t.n; ++i) seeds[i] = mem[t.members[i]].L - d;  // seed = level index
    WR_CUDA(cudaMemcpyAsync(dseeds, seeds.data(), sizeof(int64_t) * t.n, cudaMemcpyHostToDevice, s));
    bt_splitmix(t.d, t.n, t.dofs, dseeds, V[0], s);
    bt_axpy_norm(t.d, t.n, nullptr, 0, -1, nullptr, V[0], partials, kbeta, 1, 0, kinv, -1, nullptr, 0, s);
    bt_scale_dev(t.d, t.n, t.dofs, kinv, V[0], V[0], s);
    for (int j = 0; j < ne; ++j) {
      jac_inner(t, V[j], ar[d].t);
      papply(t, d, ar[d].t, V[j + 1]);
      for (int i = 0; i <= j; ++i)
        bt_axpy_dot(t.d, t.n, keH, es, i ? (i - 1) * ne + j : -1, i ? V[i - 1] : nullptr, V[j + 1], V[i], partials,
                    keH, es, i * ne + j, s);
      bt_axpy_norm(t.d, t.n, keH, es, j * ne + j, V[j], V[j + 1], partials, keH, es, (j + 1) * ne + j, kinv,
                   j * ne + j, nullptr, 0, s);
      bt_scale_dev(t.d, t.n, t.dofs, kinv, V[j + 1], V[j + 1], s);
    }
    WR_CUDA(cudaMemcpyAsync(hkH, keH, sizeof(double) * es * B, cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    if (*herr) throw WrError(WR_ERR_TIMEOUT, "a bounded wait in the smoother kernel gave up");
    for (int e = 0; e < t.n; ++e) {
      Member& M = mem[t.members[e]];
      std::vector<double> H(hkH + t.members[e] * es, hkH + (t.members[e] + 1) * es);
      int mm = ne;
      for (int j = 0; j < ne; ++j)
        if (H[(j + 1) * ne + j] <= 1e-14 * std::fabs(H[j * ne + j]) + 1e-300) {
          mm = j + 1;
          break;
        }
      M.lam[M.L - d] = hessenberg_max_real_eig(H, mm, ne);
    }
  }

  // ---------------------------------------------------------------- FGMRES and Newton in lock step
  // ||w|| of the members of table t to beta[member] (and to the device: kbeta, 1 / ||w||
  // in kinv, the FGMRES right-hand side g_b[0]); one synchronisation
  void member_norms(Table& t, std::vector<double>& beta) {
    if (!t.n) return;
    bt_axpy_norm(t.d, t.n, nullptr, 0, -1, nullptr, w, partials, kbeta, 1, 0, kinv, -1, kg, opt.gmres_restart + 1, s);
    WR_CUDA(cudaMemcpyAsync(hres, kbeta, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WR_CUDA(cudaStreamSynchronize(s));
    if (*herr) throw WrError(WR_ERR_TIMEOUT, "a bounded wait in the smoother kernel gave up");
    for (int m : t.members) beta[m] = hres[m];
  }

  // x = step for J x = b on the fine table's members; tol per member (indexed by member
  // id).  Every member's Arnoldi (MGS) coefficients, Givens rotations, least-squares
  // solve and solution update stay on the device; the host reads the members' residual
  // estimates once per iteration and their true residual norms once per restart.
  std::vector<int> fgmres(const double* b, double* x, const std::vector<double>& tol) {
    const int R = opt.gmres_restart;
    const int64_t hs = (int64_t)(R + 1) * R;
    std::vector<int> its(B, 0);
    std::vector<char> saved(active);
    Table& f = fine;
    bt_axpby(f.d, f.n, f.dofs, nullptr, 0.0, x, nullptr, 0.0, x, s);
    bt_copy(f.d, f.n, f.dofs, b, w, s);
    std::vector<double> beta(B, 0.0);
    member_norms(f, beta);
    for (int m = 0; m < B; ++m)
      if (active[m] && !(beta[m] > tol[m])) active[m] = 0;
    build_tables();
    std::vector<int> jend(B, 0);
    while (fine.n > 0) {
      Table& t = fine;
      bt_scale_dev(t.d, t.n, t.dofs, kinv, w, V[0], s);  // V[0] = w / beta
      for (int m : t.members) jend[m] = 0;
      int j = 0;
      for (; j < R; ++j) {
        Table& ta = fine;
        if (!ta.n) break;
        vcycle_via_graph(V[j], Z[j]);
        bt_project_pressure(ta.d, ta.n, ta.tblks, tab, Z[j], false, s);
        jac(ta, Z[j], V[j + 1]);
        for (int i = 0; i <= j; ++i)
          bt_axpy_dot(ta.d, ta.n, kH, hs, i ? (i - 1) * R + j : -1, i ? V[i - 1] : nullptr, V[j + 1], V[i], partials,
                      kH, hs, i * R + j, s);
        bt_axpy_norm(ta.d, ta.n, kH, hs, j * R + j, V[j], V[j + 1], partials, kH, hs, (j + 1) * R + j, kinv, -1,
                     nullptr, 0, s);
        bt_givens(ta.d, ta.n, kH, kcs, ksn, kg, R, j, kstat, s);
        bt_scale_dev(ta.d, ta.n, ta.dofs, kinv, V[j + 1], V[j + 1], s);
        WR_CUDA(cudaMemcpyAsync(hres, kstat, sizeof(double) * ta.n, cudaMemcpyDeviceToHost, s));
        WR_CUDA(cudaMemcpyAsync(herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
        WR_CUDA(cudaStreamSynchronize(s));
        if (*herr) throw WrError(WR_ERR_TIMEOUT, "a bounded wait in the smoother kernel gave up");
        std::vector<int> finished;
        for (int e = 0; e < ta.n; ++e) {
          const int m = ta.members[e];
          its[m]++;
          jend[m] = j + 1;
          if (!std::isfinite(hres[e])) throw WrError(WR_ERR_NAN, "FGMRES residual is not finite");
          if (std::fabs(hres[e]) <= tol[m] || its[m] >= opt.gmres_maxit) finished.push_back(m);
        }
        if (!finished.empty()) {
          for (int m : finished) active[m] = 0;
          // solution update of the members that leave now (the tables now hold the rest)
          update_solution(x, finished, jend);
        }
      }
      // restart: the members still active update their solution and residual
      std::vector<int> rest(fine.members.begin(), fine.members.end());
      if (rest.empty()) break;
      update_solution(x, rest, jend);
      Table& tr = fine;
      jac(tr, x, w);
      bt_axpby(tr.d, tr.n, tr.dofs, nullptr, 1.0, b, nullptr, -1.0, w, s);
      member_norms(tr, beta);
      bool change = false;
      for (int m : rest)
        if (!(beta[m] > tol[m]) || its[m] >= opt.gmres_maxit) {
          active[m] = 0;
          change = true;
        }
      if (change) build_tables();
    }
    active = saved;
    build_tables();
    return its;
  }

  // x_m += sum_i y_i Z_i for the listed members (y from the triangular solve of their
  // Hessenberg, on the device); the listed members advanced in lock step, so they share
  // one basis length.  Leaves the active set and the tables as they were.
  void update_solution(double* x, const std::vector<int>& who, const std::vector<int>& jend) {
    std::vector<char> saved(active);
    std::fill(active.begin(), active.end(), 0);
    const int je = jend[who.front()];
    for (int m : who) {
      if (jend[m] != je) throw WrError(WR_ERR_ARG, "FGMRES members out of lock step");
      active[m] = 1;
    }
    build_tables();
    Table& t = fine;
    KrylovBasis zb{};
    for (int i = 0; i < je; ++i) zb.p[i] = Z[i];
    bt_krylov_update(t.d, t.n, t.dofs, kH, kg, ky, opt.gmres_restart, je, zb, x, s);
    active = saved;
    build_tables();
  }

  int solve(std::vector<wr_stats>& st) {
    std::fill(active.begin(), active.end(), 1);
    build_tables();
    std::vector<double> fnorm(B), f0(B), eta(B, opt.ew ? 0.5 : opt.eta_fixed);
    for (auto& x : st) std::memset(&x, 0, sizeof(x));
    bt_residual(k, q, fine.d, fine.n, fine.units, fine.dofs, tab, U, F, ye, s);
    {
      std::vector<double> r2 = dots(fine, F, F);
      for (int e = 0; e < fine.n; ++e) {
        const int m = fine.members[e];
        f0[m] = fnorm[m] = std::sqrt(r2[e]);
        st[m].residual_norms[0] = fnorm[m];
      }
    }
    int status = WR_OK;
    std::vector<int> stalls(B, 0);  // consecutive Newton steps whose FGMRES ran out of iterations
    std::vector<char> finished(B, 0);
    auto member_status = [&](int m) {
      if (!std::isfinite(fnorm[m])) return (int)WR_ERR_NAN;
      return fnorm[m] <= opt.newton_rtol * f0[m] ? (int)WR_OK : (int)WR_ERR_NOT_CONVERGED;
    };
    auto finish = [&](int m, int rc) {  // member m leaves: hand out its result now
      finished[m] = 1;
      if (Uout)
        WR_CUDA(cudaMemcpyAsync(Uout[m], U + off[0][m], sizeof(double) * mem[m].g[mem[m].L].ndofs,
                                cudaMemcpyDeviceToDevice, s));
      if (on_done) on_done(m, rc);
    };
    for (int it = 0; it < opt.newton_maxit && it < 64; ++it) {
      for (int m = 0; m < B; ++m) {
        if (!active[m]) continue;
        const bool done = !(fnorm[m] > opt.newton_rtol * f0[m]) || !std::isfinite(fnorm[m]);
        // a member that diverges or whose FGMRES stagnates leaves the batch early
        const bool gave_up = (opt.newton_divtol > 0.0 && fnorm[m] > opt.newton_divtol * f0[m]) ||
                             (opt.newton_stall > 0 && stalls[m] >= opt.newton_stall);
        const bool cancelled = member_cancel && member_cancel[m] && member_cancel[m]->load();
        if (done || gave_up || cancelled) {
          active[m] = 0;
          if (Uout || on_done) finish(m, cancelled ? (int)WR_ERR_CANCELLED : member_status(m));
        }
      }
      build_tables();
      if (!fine.n) break;
      const double t0 = now_ms();
      linearise_members(U);
      WR_CUDA(cudaStreamSynchronize(s));
      const double t1 = now_ms();
      bt_axpby(fine.d, fine.n, fine.dofs, nullptr, 0.0, F, nullptr, -1.0, F, s);
      std::vector<double> tol(B, 0.0);
      for (int m : fine.members) tol[m] = eta[m] * fnorm[m];
      std::vector<int> its = fgmres(F, step, tol);
      WR_CUDA(cudaStreamSynchronize(s));
      const double t2 = now_ms();
      bt_axpby(fine.d, fine.n, fine.dofs, nullptr, 1.0, step, nullptr, 1.0, U, s);
      bt_residual(k, q, fine.d, fine.n, fine.units, fine.dofs, tab, U, F, ye, s);
      std::vector<double> r2 = dots(fine, F, F);
      for (int e = 0; e < fine.n; ++e) {
        const int m = fine.members[e];
        const double fnew = std::sqrt(r2[e]);
        wr_stats& S = st[m];
        S.gmres_its[S.newton_its] = its[m];
        S.newton_its++;
        S.residual_norms[S.newton_its] = fnew;
        S.setup_ms += t1 - t0;
        S.krylov_ms += t2 - t1;
        S.vcycles += its[m];
        stalls[m] = its[m] >= opt.gmres_maxit ? stalls[m] + 1 : 0;
        if (opt.ew) {
          const double gamma = 0.9, alpha = 2.0;
          double en = gamma * std::pow(fnew / fnorm[m], alpha);
          const double safe = gamma * std::pow(eta[m], alpha);
          if (safe > 0.1) en = std::max(en, safe);
          eta[m] = std::min(0.9, std::max(en, 0.5 * opt.newton_rtol * f0[m] / fnew));
        }
        fnorm[m] = fnew;
      }
    }
    for (int m = 0; m < B; ++m)
      if (!(fnorm[m] <= opt.newton_rtol * f0[m])) status = std::isfinite(fnorm[m]) ? WR_ERR_NOT_CONVERGED : WR_ERR_NAN;
    if (Uout || on_done)
      for (int m = 0; m < B; ++m)
        if (!finished[m]) finish(m, member_status(m));
    std::fill(active.begin(), active.end(), 1);
    build_tables();
    return status;
  }
};

namespace {

template <typename Fn>
int bguard(wr_batch* b, Fn&& fn) {
  try {
    return fn();
  } catch (const WrError& e) {
    if (b) b->err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    if (b) b->err = e.what();
    return WR_ERR_CUDA;
  }
}

void bneed(bool c, const char* msg) {
  if (!c) throw WrError(WR_ERR_ARG, msg);
}

}  // namespace

extern "C" {

int wr_batch_create(wr_batch** out, int n, const wr_problem* ps, const wr_options* o, void* stream) {
  if (!out || !ps || n < 1) return WR_ERR_ARG;
  *out = nullptr;
  auto b = std::make_unique<wr_batch>();
  const int rc = bguard(b.get(), [&]() -> int {
    if (o) b->opt = *o;
    else wr_default_options(&b->opt);
    bneed(b->opt.precision >= WR_FP64 && b->opt.precision <= WR_BF16, "bad precision");
    bneed(b->opt.apply_tile >= -1 && b->opt.apply_tile < kApplyTileVariants, "bad apply_tile");
    bneed(b->opt.patch_assembly == WR_PATCH_SUBMATRIX || b->opt.patch_assembly == WR_PATCH_LOCAL,
          "bad patch_assembly");
    bneed(b->opt.scatter_weight == WR_WEIGHT_ONE || b->opt.scatter_weight == WR_WEIGHT_MULTIPLICITY,
          "bad scatter_weight");
    bneed(b->opt.cheb_steps >= 1 && 2 * b->opt.cheb_steps <= kCoefRows, "bad Chebyshev steps");
    bneed(b->opt.eig_steps >= 1 && b->opt.eig_steps <= b->opt.gmres_restart, "bad eigen-estimate steps");
    bneed(b->opt.gmres_restart >= 1 && b->opt.gmres_restart <= kMaxKrylovBasis, "bad restart");
    b->s = static_cast<cudaStream_t>(stream);
    b->B = n;
    b->k = ps[0].k;
    b->q = ps[0].q;
    b->nt = b->q + 1;
    bneed(b->k == 1 || b->k == 2, "k must be 1 or 2");
    bneed(b->q == 0 || b->q == 1, "q must be 0 or 1");
    b->tab = build_tables(b->k, b->q);
    b->mem.resize(n);
    int D = 0;
    for (int m = 0; m < n; ++m) {
      const wr_problem& p = ps[m];
      bneed(p.k == b->k && p.q == b->q, "every member of a batch must use the same k and q");
      bneed(p.n_coarse == 2 || (p.n_coarse == 3 && p.k == 1), "n_coarse must be 2 (or 3 for k = 1)");
      int nf = p.n_fine, L = 0;
      while (nf > p.n_coarse && nf % 2 == 0) { nf /= 2; ++L; }
      bneed(nf == p.n_coarse && L >= 1, "n_fine must be n_coarse times a power of two (at least 2 n_coarse)");
      bneed(p.n_slabs >= 1 && p.T > 0.0 && p.n_modes >= 0 && p.n_modes <= 8, "bad problem");
      bneed(p.n_modes == 0 || (p.mx && p.my && p.amp), "Fourier mode arrays missing");
      Member& M = b->mem[m];
      M.nc = p.n_coarse;
      M.L = L;
      M.ph.kind = p.kind; M.ph.steady = p.steady; M.ph.nu = p.nu; M.ph.conv = p.conv; M.ph.T = p.T;
      M.ph.n_modes = p.n_modes;
      M.ph.t0 = p.t0;
      for (int i = 0; i < p.n_modes; ++i) { M.ph.mx[i] = p.mx[i]; M.ph.my[i] = p.my[i]; M.ph.amp[i] = p.amp[i]; }
      for (int l = 0, nn = p.n_coarse; l <= L; ++l, nn *= 2) M.g.push_back(make_geom(nn, p.k, p.q, p.n_slabs, p.T));
      M.lam.assign(L + 1, 0.0);
      M.cbs.kind = 1;
      M.cbs.nvg = M.g[0].nv - 2;
      M.cbs.npg = M.g[0].np;
      M.cbs.ms = coarse_ms(p.k, p.n_coarse);
      D = std::max(D, L + 1);
    }
    b->D = D;
    b->depth_variant.assign(D, b->opt.apply_tile);
    b->off.assign(D, std::vector<int64_t>(n, -1));
    b->off_ye.assign(D, std::vector<int64_t>(n, -1));
    b->off_yp.assign(D, std::vector<int64_t>(n, -1));
    b->arena_size.assign(D, 0);
    std::vector<int64_t> ye_size(D, 0), yp_size(D, 0);
    size_t max_ce = 1;
    const int ms = patch_ms(b->k);
    for (int d = 0; d < D; ++d)
      for (int m = 0; m < n; ++m) {
        const Member& M = b->mem[m];
        const int l = M.L - d;
        if (l < 0) continue;
        b->off[d][m] = b->arena_size[d];
        b->arena_size[d] += M.g[l].ndofs;
        if (l >= 1) {
          b->off_ye[d][m] = ye_size[d];
          ye_size[d] += (int64_t)M.g[l].N * M.g[l].ncells() * b->elem_size();
          b->off_yp[d][m] = yp_size[d];
          yp_size[d] += (int64_t)M.g[l].npatch() * M.g[l].N * b->nt * ms;
        }
      }
    for (int m = 0; m < n; ++m) {
      const Member& M = b->mem[m];
      const size_t nvle = (size_t)(b->k + 2) * (b->k + 2);
      max_ce = std::max(max_ce, (size_t)M.g[M.L].N * M.g[M.L].ncells() * b->nt * 4 * nvle * nvle);
    }
    // per-member level data
    for (int m = 0; m < n; ++m) {
      Member& M = b->mem[m];
      M.W.resize(M.L + 1);
      M.factors.assign(M.L + 1, nullptr);
      for (int l = 0; l <= M.L; ++l) {
        M.W[l] = b->alloc<double>(M.g[l].ndofs);
        if (l >= 1) {
          const size_t nf = (size_t)M.g[l].npatch() * M.g[l].N * b->nt * b->nt * factor_block_elems(b->k, b->opt.precision);
          const int eb = factor_elem_bytes(b->opt.precision);
          if (eb == 2) M.factors[l] = b->alloc<uint16_t>(nf);
          else if (eb == 4) M.factors[l] = b->alloc<float>(nf);
          else M.factors[l] = b->alloc<double>(nf);
        }
      }
      M.cf = b->alloc<double>((size_t)M.g[0].N * b->nt * b->nt * block_elems(M.cbs.ms, WR_FP64));
    }
    b->ar.resize(D);
    for (int d = 0; d < D; ++d) {
      Arena& a = b->ar[d];
      const int64_t sz = std::max<int64_t>(b->arena_size[d], 1);
      a.b = b->alloc<double>(sz); a.x = b->alloc<double>(sz); a.r = b->alloc<double>(sz);
      a.d = b->alloc<double>(sz); a.z = b->alloc<double>(sz); a.t = b->alloc<double>(sz);
      for (double* v : {a.b, a.x, a.r, a.d, a.z, a.t}) WR_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * sz, b->s));
    }
    b->ye = b->alloc<double>(std::max<int64_t>(*std::max_element(ye_size.begin(), ye_size.end()), 1));
    b->yp = b->alloc<double>(std::max<int64_t>(*std::max_element(yp_size.begin(), yp_size.end()), 1));
    b->Ce = b->alloc<double>(max_ce);
    const int64_t n0 = b->arena_size[0];
    const int nvec = std::max(b->opt.gmres_restart, b->opt.eig_steps) + 1;
    for (int i = 0; i < nvec; ++i) {
      b->V.push_back(b->alloc<double>(n0));
      WR_CUDA(cudaMemsetAsync(b->V.back(), 0, sizeof(double) * n0, b->s));
    }
    for (int i = 0; i < b->opt.gmres_restart; ++i) {
      b->Z.push_back(b->alloc<double>(n0));
      WR_CUDA(cudaMemsetAsync(b->Z.back(), 0, sizeof(double) * n0, b->s));
    }
    for (double** v : {&b->F, &b->w, &b->step, &b->U, &b->vb, &b->vx}) {
      *v = b->alloc<double>(n0);
      WR_CUDA(cudaMemsetAsync(*v, 0, sizeof(double) * n0, b->s));
    }
    b->partials = b->alloc<double>((size_t)bt_dot_blocks() * n);
    b->dres = b->alloc<double>(n);
    b->dcoef = b->alloc<double>(2 * (size_t)n);
    b->dseeds = b->alloc<int64_t>(n);
    {
      const int R = b->opt.gmres_restart, ne = b->opt.eig_steps;
      b->kH = b->alloc<double>((size_t)n * (R + 1) * R);
      b->kcs = b->alloc<double>((size_t)n * R);
      b->ksn = b->alloc<double>((size_t)n * R);
      b->kg = b->alloc<double>((size_t)n * (R + 1));
      b->ky = b->alloc<double>((size_t)n * R);
      b->keH = b->alloc<double>((size_t)n * (ne + 1) * ne);
      b->kbeta = b->alloc<double>(n);
      b->kinv = b->alloc<double>(n);
      b->kstat = b->alloc<double>(n);
      WR_CUDA(cudaMemsetAsync(b->keH, 0, sizeof(double) * n * (ne + 1) * ne, b->s));
      WR_CUDA(cudaMallocHost(&b->hkH, sizeof(double) * n * (ne + 1) * ne));
    }
    b->derr = b->alloc<int>(1);
    b->fstat = b->alloc<int>(1);
    WR_CUDA(cudaMemsetAsync(b->derr, 0, sizeof(int), b->s));
    WR_CUDA(cudaMallocHost(&b->hres, sizeof(double) * n));
    WR_CUDA(cudaMallocHost(&b->hcoef, sizeof(double) * 2 * n));
    WR_CUDA(cudaMallocHost(&b->herr, sizeof(int)));
    *b->herr = 0;
    b->active.assign(n, 1);
    b->build_tables();
    WR_CUDA(cudaStreamSynchronize(b->s));
    return WR_OK;
  });
  *out = b.release();
  return rc;
}

int wr_batch_destroy(wr_batch* b) {
  delete b;
  return WR_OK;
}

const char* wr_batch_last_error(const wr_batch* b) { return b ? b->err.c_str() : "null batch"; }

int wr_batch_ndofs(const wr_batch* b, int member, int64_t* out) {
  if (!b || !out || member < 0 || member >= b->B) return WR_ERR_ARG;
  const Member& M = b->mem[member];
  *out = M.g[M.L].ndofs;
  return WR_OK;
}

int wr_batch_device_bytes(const wr_batch* b, int64_t* out) {
  if (!b || !out) return WR_ERR_ARG;
  *out = b->bytes;
  return WR_OK;
}

int wr_batch_linearise(wr_batch* b, double* const* W) {
  return bguard(b, [&]() -> int {
    bneed(b && W, "null argument");
    for (int m = 0; m < b->B; ++m) {
      bneed(W[m] != nullptr, "null member vector");
      WR_CUDA(cudaMemcpyAsync(b->U + b->off[0][m], W[m], sizeof(double) * b->mem[m].g[b->mem[m].L].ndofs,
                              cudaMemcpyDeviceToDevice, b->s));
    }
    std::fill(b->active.begin(), b->active.end(), 1);
    b->linearise_members(b->U);
    WR_CUDA(cudaStreamSynchronize(b->s));
    return WR_OK;
  });
}

int wr_batch_get_lambda(const wr_batch* b, int member, int level, double* lam) {
  if (!b || !lam || member < 0 || member >= b->B) return WR_ERR_ARG;
  const Member& M = b->mem[member];
  if (level < 1 || level > M.L || !b->linearised) return WR_ERR_ARG;
  *lam = M.lam[level];
  return WR_OK;
}

int wr_batch_vcycle(wr_batch* b, double* const* bin, double* const* xout) {
  return bguard(b, [&]() -> int {
    bneed(b && bin && xout, "null argument");
    if (!b->linearised) throw WrError(WR_ERR_STATE, "wr_batch_linearise must be called first");
    for (int m = 0; m < b->B; ++m)
      WR_CUDA(cudaMemcpyAsync(b->vb + b->off[0][m], bin[m], sizeof(double) * b->mem[m].g[b->mem[m].L].ndofs,
                              cudaMemcpyDeviceToDevice, b->s));
    b->vcycle_graph();
    for (int m = 0; m < b->B; ++m)
      WR_CUDA(cudaMemcpyAsync(xout[m], b->vx + b->off[0][m], sizeof(double) * b->mem[m].g[b->mem[m].L].ndofs,
                              cudaMemcpyDeviceToDevice, b->s));
    return WR_OK;
  });
}

// One V-cycle on the batch's own right-hand side arena (for throughput measurements).
int wr_batch_vcycle_resident(wr_batch* b) {
  return bguard(b, [&]() -> int {
    bneed(b != nullptr, "null argument");
    if (!b->linearised) throw WrError(WR_ERR_STATE, "wr_batch_linearise must be called first");
    b->vcycle_graph();
    return WR_OK;
  });
}

int wr_batch_initial_guess(wr_batch* b, double* const* U) {
  return bguard(b, [&]() -> int {
    bneed(b && U, "null argument");
    std::fill(b->active.begin(), b->active.end(), 1);
    b->build_tables();
    bt_boundary(b->fine.d, b->fine.n, b->fine.dofs, b->tab, b->U, b->s);
    for (int m = 0; m < b->B; ++m)
      WR_CUDA(cudaMemcpyAsync(U[m], b->U + b->off[0][m], sizeof(double) * b->mem[m].g[b->mem[m].L].ndofs,
                              cudaMemcpyDeviceToDevice, b->s));
    return WR_OK;
  });
}

int wr_batch_solve(wr_batch* b, double* const* U, wr_stats* st) {
  return bguard(b, [&]() -> int {
    bneed(b && U, "null argument");
    for (int m = 0; m < b->B; ++m)
      WR_CUDA(cudaMemcpyAsync(b->U + b->off[0][m], U[m], sizeof(double) * b->mem[m].g[b->mem[m].L].ndofs,
                              cudaMemcpyDeviceToDevice, b->s));
    std::vector<wr_stats> loc(b->B);
    const int rc = b->solve(loc);
    for (int m = 0; m < b->B; ++m)
      WR_CUDA(cudaMemcpyAsync(U[m], b->U + b->off[0][m], sizeof(double) * b->mem[m].g[b->mem[m].L].ndofs,
                              cudaMemcpyDeviceToDevice, b->s));
    WR_CUDA(cudaStreamSynchronize(b->s));
    if (st)
      for (int m = 0; m < b->B; ++m) st[m] = loc[m];
    if (rc == WR_ERR_NOT_CONVERGED) b->err = "Newton iteration limit reached for at least one member";
    return rc;
  });
}

}  // extern "C"

int batch_solve_hooked(wr_batch* b, double* const* U, wr_stats* st, const std::atomic<int>* const* cancel,
                       const std::function<void(int, int)>& on_done) {
  return bguard(b, [&]() -> int {
    bneed(b && U && st, "null argument");
    for (int m = 0; m < b->B; ++m)
      WR_CUDA(cudaMemcpyAsync(b->U + b->off[0][m], U[m], sizeof(double) * b->mem[m].g[b->mem[m].L].ndofs,
                              cudaMemcpyDeviceToDevice, b->s));
    std::vector<wr_stats> loc(b->B);
    struct Reset {  // the hooks belong to this call only
      wr_batch* b;
      ~Reset() {
        b->Uout = nullptr;
        b->member_cancel = nullptr;
        b->on_done = nullptr;
      }
    } reset{b};
    b->Uout = U;
    b->member_cancel = cancel;
    b->on_done = [&](int m, int rc) {
      st[m] = loc[m];
      on_done(m, rc);
    };
    const int rc = b->solve(loc);
    WR_CUDA(cudaStreamSynchronize(b->s));
    return rc;
  });
}

extern "C" int wr_batch_set_graphs(wr_batch* b, int enable) {
  if (!b) return WR_ERR_ARG;
  b->use_graphs = enable != 0;
  b->drop_graph();
  return WR_OK;
}
