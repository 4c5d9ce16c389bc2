// C ABI (include/helm.h): setup of the operators and the coarse factor, the
// V-cycle and FGMRES iteration as a captured CUDA graph, the host loop that
// launches iterations and reads the device's convergence state, batched
// solves over several streams, and the single-step entry points.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "runtime.h"

using namespace helm;

namespace {

struct Profile {
  bool on = false;
  static constexpr int kPhases = 6;
  double ms[kPhases] = {0};
  int calls[kPhases] = {0};
  std::vector<cudaEvent_t> ev;   // kPhases + 1 per iteration
};
const char* kPhaseNames[Profile::kPhases] = {"vcycle_pre_restrict", "coarse_solve", "vcycle_prolong_post",
                                             "apply_A0", "arnoldi_dots_givens", "arnoldi_update"};

template <typename T> struct Prec {
  using value_type = T;
  c2<T>* coefAe = nullptr;   // fine A_eps
  c2<T>* wdinv = nullptr;    // fine omega/diag(A_eps)
  c2<T>* hrow = nullptr;     // heterogeneous k: per-DoF rows of -M_k - i B_k (fine), N x noff
  c2<T>* hwd = nullptr;      // heterogeneous k: per-DoF omega / diag(A_eps)
  c2<T>* coefAc = nullptr;   // coarse A_eps
  T* pw = nullptr;           // prolongation weights
  c2<T>* Dinv = nullptr;     // coarse factor: inverses of the Schur blocks
  c2<T>* Lm = nullptr;       // Dinv[J] A_J,J-1 (couplings folded into the inverses)
  c2<T>* Up = nullptr;       // Dinv[J] A_J,J+1
  CoarsePlan plan{};
  // V-cycle workspaces
  c2<T>* ua = nullptr;
  c2<T>* ub = nullptr;
  c2<T>* r = nullptr;
  c2<T>* fT = nullptr;
  c2<T>* rc = nullptr;
  c2<T>* uc = nullptr;
  unsigned* gbar = nullptr;   // grid barrier of the whole-grid coarse solve
  SegBufs<T> seg{};           // segmented solve workspaces (plan.seg)
  const SegBufs<T>* segp() const { return plan.seg ? &seg : nullptr; }
};

}  // namespace

struct helm_ctx {
  int dim = 2, order = 1, n = 0;
  bool op_only = false;        // fine-level operators only (helm_operator_setup)
  int elements = HELM_SIMPLICES;   // HELM_TENSOR: Q_order on squares / cubes (helm_setup_q)
  double k = 0, h = 0, shift = 0;
  bool het = false;                // one wavenumber per element (helm_setup_het)
  std::vector<double> kf, kc;      // ... of the fine and of the coarse elements
  double2* hrowA0 = nullptr;       // per-DoF rows of the fine operators' k-dependent part (complex128)
  double2* hrowC = nullptr;        // the same on the coarse level (read by the factorisation)
  helm_opts opts{};
  cudaStream_t s = nullptr;
  int dev = 0;                 // device the handle was set up on
  int nsm = 0;
  HostTables tab;
  GridDesc gf{}, gc{};
  CoarseLayout L{};
  int ncls_f = 0, ncls_c = 0;
  double2* coefA0 = nullptr;   // fine A0 (FP64)
  Prec<double> p64;
  Prec<float> p32;
  // Krylov
  KrylovBufs kb{};
  KState* st_h = nullptr;   // pinned mirror
  int* err_h = nullptr;     // pinned mirror of the error word (read without blocking)
  int* err = nullptr;
  double2* rres = nullptr;  // true residual buffer
  double2* Fdev = nullptr;  // staging for host solves
  double2* xdev = nullptr;
  cudaGraphExec_t iter = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float setup_ms = 0.f;
  int setup_kernels = 0;
  int reused_blocks = 0;       // coarse blocks whose inverse was copied from a converged chain
  int iter_nodes = 0;          // kernel nodes in the captured iteration graph
  Profile prof;
  std::vector<void*> allocs;
  size_t bytes = 0;            // device bytes held by the handle

  template <typename P> cudaError_t alloc(P** p, size_t nbytes) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(nbytes, 16));
    if (e == cudaSuccess) {
      allocs.push_back(*p);
      bytes += std::max<size_t>(nbytes, 16);
    }
    return e;
  }
  template <typename T> Prec<T>& prec();
};
template <> Prec<double>& helm_ctx::prec<double>() { return p64; }
template <> Prec<float>& helm_ctx::prec<float>() { return p32; }

namespace {

thread_local const char* g_last_cuda_error = "none";

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorName(e);
  return e == cudaErrorMemoryAllocation ? HELM_ENOMEM : HELM_ECUDA;
}

#define CK(x)                                 \
  do {                                        \
    cudaError_t e_ = (x);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

template <typename T>
StencilView<T> make_view(const GridDesc& g, const c2<T>* coef, const c2<T>* wdinv, const c2<T>* hrow = nullptr,
                         const c2<T>* hwd = nullptr) {
  StencilView<T> v{};
  v.coef = coef;
  v.wdinv = wdinv;
  v.hrow = hrow;
  v.hwd = hwd;
  v.g = g;
  int side = 2 * g.R + 1;
  for (int o = 0; o < g.noff; ++o) {
    int t = o, lin = 0, mul = 1;
    for (int ax = 0; ax < 3; ++ax) {
      int d = 0;
      if (ax < g.dim) {
        d = t % side - g.R;
        t /= side;
      }
      v.dx[o][ax] = d;
      if (ax < g.dim) {
        lin += d * mul;
        mul *= g.W;
      }
    }
    v.off[o] = lin;
  }
  return v;
}

template <typename T>
TransferView<T> make_transfer(const helm_ctx* h, const T* w) {
  TransferView<T> P{};
  P.w = w;
  P.fine = h->gf;
  P.coarse = h->gc;
  P.pf = h->tab.pf;
  P.npc = h->tab.npc;
  P.npo = h->tab.npo;
  int q = h->order;
  for (int o = 0; o < P.npo; ++o) {
    int t = o;
    for (int ax = 0; ax < 3; ++ax) {
      P.po[o][ax] = ax < h->dim ? t % (q + 1) : 0;
      if (ax < h->dim) t /= (q + 1);
    }
  }
  return P;
}

// complex coefficient table K - lam M - i k B for one level
std::vector<double2> complex_table(const std::vector<double>& K, const std::vector<double>& M,
                                   const std::vector<double>& B, double k, double eps) {
  std::vector<double2> c(K.size());
  for (size_t i = 0; i < K.size(); ++i) {
    // (K - k^2 M) + i (-eps M - k B)
    c[i] = make_double2(K[i] - k * k * M[i], -eps * M[i] - k * B[i]);
  }
  return c;
}

std::vector<double2> wdinv_table(const std::vector<double2>& coef, int ncls, int noff, double omega) {
  std::vector<double2> d(ncls);
  int center = noff / 2;   // box centre (all offsets zero)
  for (int c = 0; c < ncls; ++c) {
    double2 a = coef[(size_t)c * noff + center];
    double m2 = a.x * a.x + a.y * a.y;
    d[c] = m2 > 0 ? make_double2(omega * a.x / m2, -omega * a.y / m2) : make_double2(0, 0);
  }
  return d;
}

template <typename T>
int upload(helm_ctx* h, c2<T>** dst, const std::vector<double2>& src) {
  std::vector<c2<T>> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = mk((T)src[i].x, (T)src[i].y);
  CK(h->alloc(dst, sizeof(c2<T>) * tmp.size()));
  CK(cudaMemcpy(*dst, tmp.data(), sizeof(c2<T>) * tmp.size(), cudaMemcpyHostToDevice));
  return HELM_OK;
}
template <typename T>
int upload_real(helm_ctx* h, T** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.begin(), src.end());
  CK(h->alloc(dst, sizeof(T) * tmp.size()));
  CK(cudaMemcpy(*dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice));
  return HELM_OK;
}

template <typename T>
int setup_prec(helm_ctx* h, const std::vector<double2>& Ae, const std::vector<double2>& wd,
               const std::vector<double2>& Ac, bool solves) {
  Prec<T>& p = h->prec<T>();
  int rc;
  if ((rc = upload<T>(h, &p.coefAe, Ae))) return rc;
  if ((rc = upload<T>(h, &p.wdinv, wd))) return rc;
  if ((rc = upload<T>(h, &p.coefAc, Ac))) return rc;
  if ((rc = upload_real<T>(h, &p.pw, h->tab.pw))) return rc;
  if (!solves) return HELM_OK;   // tables only (the FP64 coarse table feeds the factorisation)
  size_t Nf = (size_t)h->gf.N, Nc = (size_t)h->L.nb * h->L.ldb;
  CK(h->alloc(&p.ua, sizeof(c2<T>) * Nf));
  CK(h->alloc(&p.ub, sizeof(c2<T>) * Nf));
  CK(h->alloc(&p.r, sizeof(c2<T>) * Nf));
  CK(h->alloc(&p.fT, sizeof(c2<T>) * Nf));
  CK(h->alloc(&p.rc, sizeof(c2<T>) * Nc));
  CK(h->alloc(&p.uc, sizeof(c2<T>) * Nc));
  CK(h->alloc(&p.gbar, sizeof(unsigned) * kBarWords));
  if ((rc = plan_coarse_solve<T>(h->L, &p.plan))) return rc;
  // the elimination order (one chain, or two chains meeting in the middle) is fixed
  // here, before the factorisation, and used by both the factor and the solve
  h->L.mid = p.plan.ncl == 2 ? h->L.nb / 2 : h->L.nb - 1;
  return HELM_OK;
}

// One V(nu,nu)-cycle on A_eps (Algorithm 1, two levels): z = Vcycle(f), u^0 = 0.
// f: complex128, or (complex64 form) a double-float Krylov slot read through its high
// parts; z: complex128, or complex64 (the complex64 form's preconditioned vectors).
template <typename T, typename Vf, typename Vz>
void enqueue_vcycle(helm_ctx* h, VecSel<const Vf> f, VecSel<Vz> z, const int* active,
                    cudaStream_t s, Profile* prof, int ev0) {
  using V = c2<T>;
  Prec<T>& p = h->prec<T>();
  StencilView<T> Ae = make_view<T>(h->gf, p.coefAe, p.wdinv, p.hrow, p.hwd);
  TransferView<T> P = make_transfer<T>(h, p.pw);
  const int nu = h->opts.nu;
  V* cur = p.ua;
  V* oth = p.ub;
  // 2D: presmoothing and the residual in one tiled kernel, the prolongation and the
  // postsmoothing in another (smooth.cu)
  if (launch_smooth_tile<T, Vf, V>(Ae, f, nullptr, nullptr, nullptr, nullptr, nu, vsel<V>(cur), p.r, active, s)) {
    launch_restrict<T>(P, h->L, p.r, p.rc, active, s);
    if (prof) cudaEventRecord(prof->ev[ev0 + 1], s);
    launch_coarse_solve<T>(p.plan, p.Dinv, p.Lm, p.Up, h->L, p.rc, p.uc, p.gbar, h->err, active, h->nsm, s,
                           p.segp());
    if (prof) cudaEventRecord(prof->ev[ev0 + 2], s);
    if (launch_smooth_tile<T, Vf, Vz>(Ae, f, cur, &P, &h->L, p.uc, nu, z, nullptr, active, s)) return;
    launch_prolong_add<T>(P, h->L, p.uc, cur, active, s);   // (not reached: both tiles fit alike)
    return;
  }
  VecSel<const V> fT;
  if constexpr (sizeof(V) == sizeof(double2)) {
    launch_jacobi_from_zero<T, double2>(Ae, f, cur, nullptr, nu >= 2, active, s);
    fT = VecSel<const V>{reinterpret_cast<const V*>(f.base), f.stride, f.jsel, f.jadd};
  } else {
    // complex64: u^1 = w D^-1 f with f converted once (the fused two-sweep kernel would
    // convert f at every neighbour on the slow double-to-float path), then one sweep
    launch_jacobi_from_zero<T, Vf>(Ae, f, nu >= 2 ? oth : cur, p.fT, false, active, s);
    fT = vsel<const V>(p.fT);
    if (nu >= 2) launch_jacobi<T, V, V>(Ae, fT, oth, vsel<V>(cur), active, s);
  }
  for (int it = 2; it < nu; ++it) {   // presmoothing steps 3..nu
    launch_jacobi<T, V, V>(Ae, fT, cur, vsel<V>(oth), active, s);
    std::swap(cur, oth);
  }
  launch_residual<T, V, V>(Ae, fT, cur, p.r, active, s);
  launch_restrict<T>(P, h->L, p.r, p.rc, active, s);
  if (prof) cudaEventRecord(prof->ev[ev0 + 1], s);
  launch_coarse_solve<T>(p.plan, p.Dinv, p.Lm, p.Up, h->L, p.rc, p.uc, p.gbar, h->err, active,
                         h->nsm, s, p.segp());
  if (prof) cudaEventRecord(prof->ev[ev0 + 2], s);
  launch_prolong_add<T>(P, h->L, p.uc, cur, active, s);
  for (int it = 0; it < nu; ++it) {   // postsmoothing
    if (it == nu - 1) {
      launch_jacobi<T, V, Vz>(Ae, fT, cur, z, active, s);
    } else {
      launch_jacobi<T, V, V>(Ae, fT, cur, vsel<V>(oth), active, s);
      std::swap(cur, oth);
    }
  }
}

void enqueue_vcycle_any(helm_ctx* h, VecSel<const double2> f, VecSel<double2> z, const int* active,
                        cudaStream_t s, Profile* prof = nullptr, int ev0 = 0) {
  if (h->opts.precision == HELM_MIXED)
    enqueue_vcycle<float, double2, double2>(h, f, z, active, s, prof, ev0);
  else
    enqueue_vcycle<double, double2, double2>(h, f, z, active, s, prof, ev0);
}

// One FGMRES/Arnoldi step j (device index): z_j = Vcycle(u_j), w = A0 z_j, then the
// lagged Gram-Schmidt step (finishes v_j and column j-1 with its Givens rotation and
// convergence test, orthogonalises w, u_{j+1} = w/||w||). A step with pre == 0 skips the
// preconditioner and A0 and only finishes the last column of the cycle.
void enqueue_iteration(helm_ctx* h, cudaStream_t s, Profile* prof = nullptr, int ev0 = 0) {
  const KrylovBufs& kb = h->kb;
  const int* act = &kb.st->pre;
  const int* jsel = &kb.st->j;
  if (prof) cudaEventRecord(prof->ev[ev0 + 0], s);
  StencilView<double> A0 = make_view<double>(h->gf, h->coefA0, nullptr, h->hrowA0);
  if (h->opts.precision == HELM_MIXED) {
    // complex64 form: the preconditioner reads slot j of the basis (high parts), z_j is
    // complex64, and w = A0 z_j is formed in double-float from it (exact products of the
    // complex64 z_j with the split complex128 coefficients)
    enqueue_vcycle<float, float4, float2>(h, VecSel<const float4>{kb.Vs, kb.ldN, jsel, 0},
                                          VecSel<float2>{kb.Z32, kb.ldN, jsel, 0}, act, s, prof, ev0);
    if (prof) cudaEventRecord(prof->ev[ev0 + 3], s);
    launch_apply_df(A0, VecSel<const float2>{kb.Z32, kb.ldN, jsel, 0}, kb.Ws, act, s);
  } else {
    enqueue_vcycle<double, double2, double2>(h, VecSel<const double2>{kb.W, 0, nullptr, 0},
                                             VecSel<double2>{kb.Z, kb.ldN, jsel, 0}, act, s, prof, ev0);
    if (prof) cudaEventRecord(prof->ev[ev0 + 3], s);
    launch_apply<double, double2, double2>(A0, VecSel<const double2>{kb.Z, kb.ldN, jsel, 0},
                                           VecSel<double2>{nullptr, 0, nullptr, 0}, act, s, kb.Ws);
  }
  if (prof) cudaEventRecord(prof->ev[ev0 + 4], s);
  launch_arnoldi(kb, s, prof ? prof->ev[ev0 + 5] : nullptr);
  if (prof) cudaEventRecord(prof->ev[ev0 + 6], s);
}

int capture_iteration(helm_ctx* h) {
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_iteration(h, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    h->iter_nodes = (int)nn;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->iter, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e == cudaSuccess) e = cudaGetLastError();   // nothing may be left pending from the capture
  return e == cudaSuccess ? HELM_OK : cuda_fail(e);
}

int check_err(helm_ctx* h) {
  int e = 0;
  cudaError_t ce = cudaMemcpy(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return HELM_ECUDA;
  return e;
}

// ---- solve driver: one FGMRES solve as a resumable state machine ----------
struct SolveTask {
  helm_ctx* h;
  const double2* F;
  double2* x;
  helm_result* res;
  enum Phase { ITER, WAIT_ITER, WAIT_END, DONE } phase = ITER;
  int launched_in_cycle = 0;
  int launched_total = 0;
  int cycles = 0;
  int kernels = 0;
  int rc = HELM_OK;
  cudaEvent_t ready = nullptr;
};

int solve_begin(SolveTask& t) {
  helm_ctx* h = t.h;
  cudaStream_t s = h->s;
  const KrylovBufs& kb = h->kb;
  KState st{};
  st.m = h->opts.restart;
  st.maxit = h->opts.maxit;
  st.tol = h->opts.tol;
  CK(cudaMemcpyAsync(kb.st, &st, sizeof(KState), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));
  CK(cudaMemsetAsync(t.x, 0, sizeof(double2) * kb.N, s));
  CK(cudaEventRecord(h->e0, s));
  launch_norm(kb, t.F, 0, s);          // ||F||, beta = ||F||  (x0 = 0: r0 = F)
  launch_cycle_start(kb, t.F, s);      // v1 = F / beta
  t.kernels = 3;
  CK(cudaEventCreateWithFlags(&t.ready, cudaEventDisableTiming));
  t.phase = SolveTask::ITER;
  return HELM_OK;
}

// Advance the task without blocking when possible. Returns true when done.
bool solve_step(SolveTask& t, bool blocking) {
  helm_ctx* h = t.h;
  cudaStream_t s = h->s;
  const KrylovBufs& kb = h->kb;
  const int m = h->opts.restart, maxit = h->opts.maxit;
  switch (t.phase) {
    case SolveTask::ITER: {
      // a cycle takes up to m + 1 steps: the last one only finishes column m - 1
      int chunk = std::min(4, m + 1 - t.launched_in_cycle);
      if (chunk < 1) chunk = 1;
      for (int c = 0; c < chunk; ++c) {
        if (h->prof.on) {
          KState cur;
          cudaMemcpyAsync(&cur, kb.st, sizeof(KState), cudaMemcpyDeviceToHost, s);
          cudaStreamSynchronize(s);
          if (!cur.active) break;
          int need = (Profile::kPhases + 1);
          if ((int)h->prof.ev.size() < need) {
            h->prof.ev.resize(need);
            for (auto& e : h->prof.ev) cudaEventCreate(&e);
          }
          enqueue_iteration(h, s, &h->prof, 0);
          cudaEventSynchronize(h->prof.ev[Profile::kPhases]);
          for (int ph = 0; ph < Profile::kPhases; ++ph) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, h->prof.ev[ph], h->prof.ev[ph + 1]);
            h->prof.ms[ph] += ms;
            h->prof.calls[ph] += 1;
          }
        } else {
          cudaGraphLaunch(h->iter, s);
        }
        t.kernels += h->iter_nodes;
      }
      t.launched_in_cycle += chunk;
      t.launched_total += chunk;
      cudaMemcpyAsync(h->st_h, kb.st, sizeof(KState), cudaMemcpyDeviceToHost, s);
      // the error word too: a bounded device wait that timed out ends the solve at the next
      // chunk boundary (every later launch would otherwise wait out its own limit again)
      cudaMemcpyAsync(h->err_h, h->err, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaEventRecord(t.ready, s);
      t.phase = SolveTask::WAIT_ITER;
      return false;
    }
    case SolveTask::WAIT_ITER: {
      if (blocking) cudaEventSynchronize(t.ready);
      else if (cudaEventQuery(t.ready) == cudaErrorNotReady) return false;
      if (h->st_h->active && *h->err_h == 0 && t.launched_in_cycle < m + 1) {
        t.phase = SolveTask::ITER;
        return false;
      }
      // cycle end: y = R^{-1} g, x += Z y, true residual
      launch_backsolve(kb, s);
      launch_update_x(kb, t.x, s);
      StencilView<double> A0 = make_view<double>(h->gf, h->coefA0, nullptr, h->hrowA0);
      launch_residual<double, double2, double2>(A0, vsel<const double2>(t.F), t.x, h->rres, nullptr, s);
      launch_norm(kb, h->rres, 1, s);
      t.kernels += 5;
      cudaMemcpyAsync(h->st_h, kb.st, sizeof(KState), cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(h->err_h, h->err, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaEventRecord(h->e1, s);
      cudaEventRecord(t.ready, s);
      t.cycles += 1;
      t.phase = SolveTask::WAIT_END;
      return false;
    }
    case SolveTask::WAIT_END: {
      if (blocking) cudaEventSynchronize(t.ready);
      else if (cudaEventQuery(t.ready) == cudaErrorNotReady) return false;
      KState* st = h->st_h;
      // (the state, the error word and e1 were recorded before `ready`, which has completed)
      const int e = *h->err_h;
      bool done = st->relres <= h->opts.tol || st->total >= maxit || st->breakdown || st->nonfinite ||
                  !(st->relres == st->relres) || e != 0;
      if (!done) {
        launch_cycle_start(kb, h->rres, s);   // restart from r = F - A0 x
        t.kernels += 1;
        t.launched_in_cycle = 0;
        t.phase = SolveTask::ITER;
        return false;
      }
      cudaError_t ce = cudaGetLastError();
      if (ce != cudaSuccess) t.rc = cuda_fail(ce);
      else if (e != 0) t.rc = e;
      if (t.res) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->e0, h->e1);
        t.res->iters = st->total;
        t.res->cycles = t.cycles;
        t.res->relres_true = st->relres;
        t.res->relres_est = st->est;
        t.res->solve_ms = ms;
        t.res->kernels = t.kernels;
        t.res->status = st->nonfinite || !(st->relres == st->relres) ? HELM_NONFINITE
                        : st->relres <= h->opts.tol                  ? HELM_CONVERGED
                        : st->breakdown                             ? HELM_BREAKDOWN
                                                                    : HELM_MAXIT;
      }
      cudaEventDestroy(t.ready);
      t.ready = nullptr;
      t.phase = SolveTask::DONE;
      return true;
    }
    case SolveTask::DONE:
      return true;
  }
  return true;
}

}  // namespace

// ---- resumable solves and memory accounting for the request server (serve.cu) ----
namespace helm {
struct Task {
  SolveTask t;
  helm_result res{};
};
int task_create(helm_t h, const double2* F, double2* x, Task** out) {
  Task* k = new (std::nothrow) Task();
  if (!k) return HELM_ENOMEM;
  k->t = SolveTask{h, F, x, &k->res};
  int rc = solve_begin(k->t);
  if (rc) {
    delete k;
    return rc;
  }
  *out = k;
  return HELM_OK;
}
bool task_step(Task* k, bool blocking, helm_result* res, int* rc) {
  if (!solve_step(k->t, blocking)) return false;
  if (res) *res = k->res;
  if (rc) *rc = k->t.rc;
  return true;
}
void task_destroy(Task* k) {
  if (k && k->t.ready) cudaEventDestroy(k->t.ready);
  delete k;
}
size_t handle_bytes(helm_t h) { return h ? h->bytes : 0; }

// Peak device bytes of helm_setup + helm_solve for one problem (mirrors the
// allocations of setup_impl / setup_prec; the coefficient tables are bounded by
// a fixed 1 MiB). Includes the FP64 factor workspace that setup frees again.
size_t estimate_bytes(int dim, int order, int n, int precision, int restart) {
  auto ipow = [](int64_t b, int d) {
    int64_t r = 1;
    for (int i = 0; i < d; ++i) r *= b;
    return r;
  };
  const int64_t N = ipow((int64_t)order * n + 1, dim);
  const int64_t Wc = (int64_t)order * (n / 2) + 1;
  const int64_t rows = order, plane = ipow(Wc, dim - 1);
  const int64_t nb = (Wc + rows - 1) / rows, B = rows * plane, ldb = (B + 1) & ~int64_t(1);
  const int64_t blk = B * ldb;
  const int64_t v = precision == HELM_MIXED ? 8 : 16;
  const int64_t m = restart, ldN = (N + 31) & ~int64_t(31), nblk = std::max<int64_t>(1, (N + 255) / 256);
  // (+ the coarse block maps and the group lists of the grouped block products)
  const int64_t prec = v * (4 * N + 2 * nb * ldb) + 64 + 3 * 4 * nb + 3 * 4 * kGroupInts * nb;
  // Dinv, Lm, Up; the mixed form's segmented solve adds two product sets and one vector
  const int64_t factor = v * 3 * blk * nb + (precision == HELM_MIXED ? 8 * (2 * blk * nb + nb * ldb) : 0);
  // basis (double-float), w split, Z (complex64 in the mixed form), W (FP64 form), residual
  const int64_t krylov = 16 * ldN * (m + 1) + 16 * ldN + v * ldN * m + (precision == HELM_MIXED ? 0 : 16 * ldN) +
                         16 * ldN +
                         16 * std::max<int64_t>(nblk, (N + 255) / 256) * kb_rows((int)m) + 16 * (m + 2) * (m + 6);
  const int64_t tables = 1 << 20;
  const int64_t transient = (precision == HELM_MIXED ? 16 * blk * nb : 0) + 16 * 2 * blk +
                            16 * 2 * (16 * ldb + 16 * B) + 64;
  return (size_t)(prec + factor + krylov + tables + transient);
}
}  // namespace helm

// ============================================================================
namespace {
template <typename T>
void enqueue_smooth(helm_ctx* h, const double2* f, double2* u, int nu, cudaStream_t s) {
  using V = c2<T>;
  Prec<T>& p = h->prec<T>();
  StencilView<T> Ae = make_view<T>(h->gf, p.coefAe, p.wdinv, p.hrow, p.hwd);
  if (launch_smooth_tile<T, double2, double2>(Ae, vsel<const double2>(f), nullptr, nullptr, nullptr, nullptr, nu,
                                              vsel<double2>(u), nullptr, nullptr, s))
    return;   // 2D: all nu sweeps in one tiled kernel
  V* cur = p.ua;
  V* oth = p.ub;
  const bool two = nu >= 3;   // the first two sweeps fused when two or more precede the last one
  VecSel<const V> fT;
  if constexpr (sizeof(V) == sizeof(double2)) {
    launch_jacobi_from_zero<T, double2>(Ae, vsel<const double2>(f), cur, nullptr, two, nullptr, s);
    fT = VecSel<const V>{reinterpret_cast<const V*>(f), 0, nullptr, 0};
  } else {
    launch_jacobi_from_zero<T, double2>(Ae, vsel<const double2>(f), two ? oth : cur, p.fT, false, nullptr, s);
    fT = vsel<const V>(p.fT);
    if (two) launch_jacobi<T, V, V>(Ae, fT, oth, vsel<V>(cur), nullptr, s);
  }
  for (int done = two ? 2 : 1; done < nu - 1; ++done) {
    launch_jacobi<T, V, V>(Ae, fT, cur, vsel<V>(oth), nullptr, s);
    std::swap(cur, oth);
  }
  launch_jacobi<T, V, double2>(Ae, fT, cur, vsel<double2>(u), nullptr, s);   // last sweep writes complex128
}
}  // namespace

extern "C" {

void helm_default_opts(helm_opts* o) {
  if (!o) return;
  o->dim = 2;
  o->omega = 0.6;
  o->nu = 2;
  o->restart = 50;
  o->maxit = 500;
  o->tol = 1e-8;
  o->precision = HELM_FP64;
  o->stream = nullptr;
}

const char* helm_last_cuda_error(void) { return g_last_cuda_error; }

const char* helm_strerror(int code) {
  switch (code) {
    case HELM_OK: return "ok";
    case HELM_EINVAL: return "invalid argument";
    case HELM_ENOMEM: return "device out of memory";
    case HELM_ECUDA: return "CUDA runtime error";
    case HELM_EZEROPIVOT: return "zero or non-finite pivot in the coarse factorisation";
    case HELM_ETIMEOUT: return "bounded device wait timed out";
    case HELM_ENOTSUP: return "configuration not supported on this device";
    case HELM_ESCRATCH: return "problem too large for the 4 MiB scratch of helm_coarse_solve_noalloc";
    default: return "unknown error";
  }
}

void helm_destroy(helm_t h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->iter) cudaGraphExecDestroy(h->iter);
  for (void* p : h->allocs) cudaFree(p);
  if (h->st_h) cudaFreeHost(h->st_h);
  if (h->err_h) cudaFreeHost(h->err_h);
  if (h->e0) cudaEventDestroy(h->e0);
  if (h->e1) cudaEventDestroy(h->e1);
  for (auto& e : h->prof.ev) cudaEventDestroy(e);
  delete h;
}

static int setup_impl(helm_ctx* h) {
  const helm_opts& o = h->opts;
  int rc = build_tables(o.dim, h->order, h->n, &h->tab, h->elements);
  if (rc) return rc;
  h->gf = h->tab.fine;
  h->gc = h->tab.coarse;
  h->ncls_f = h->tab.ncls_f;
  h->ncls_c = h->tab.ncls_c;
  if (h->gf.N >= (1ll << 31) / 2) return HELM_ENOTSUP;
  CK(cudaGetDevice(&h->dev));
  CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev));
  smooth_tile_prepare<float>();
  smooth_tile_prepare<double>();
  stencil_prepare();
  CK(cudaEventCreate(&h->e0));
  CK(cudaEventCreate(&h->e1));
  cudaStream_t s = h->s;

  // coefficient tables (Sec. 2, eq. sys_matrix): A0 = A(k, 0), A_eps = A(k, eps). With one
  // wavenumber per element the class tables hold K - i eps M and the k-dependent part
  // -M_k - i B_k comes as per-DoF rows (eq. sys_matrix with k in L^inf, Sec. 6).
  const double kt = h->het ? 0.0 : h->k;
  auto A0 = complex_table(h->tab.Kf, h->tab.Mf, h->tab.Bf, kt, 0.0);
  auto Ae = complex_table(h->tab.Kf, h->tab.Mf, h->tab.Bf, kt, h->shift);
  auto Ac = complex_table(h->tab.Kc, h->tab.Mc, h->tab.Bc, kt, h->shift);
  auto wd = wdinv_table(Ae, h->ncls_f, h->gf.noff, o.omega);
  if ((rc = upload<double>(h, &h->coefA0, A0))) return rc;
  std::vector<double2> hrf, hwdf;   // fine per-DoF rows and omega / diag(A_eps)
  if (h->het) {
    HetRows hf, hc;
    if ((rc = build_het_rows(o.dim, h->order, h->n, h->elements, h->kf.data(), &hf))) return rc;
    if ((rc = build_het_rows(o.dim, h->order, h->n / 2, h->elements, h->kc.data(), &hc))) return rc;
    auto rows = [](const HetRows& r) {
      std::vector<double2> v(r.Mk.size());
      for (size_t i = 0; i < v.size(); ++i) v[i] = make_double2(-r.Mk[i], -r.Bk[i]);
      return v;
    };
    hrf = rows(hf);
    const std::vector<double2> hrc = rows(hc);
    if ((rc = upload<double>(h, &h->hrowA0, hrf))) return rc;
    if ((rc = upload<double>(h, &h->hrowC, hrc))) return rc;
    // omega / diag: the class table's centre plus the DoF's own centre coefficient
    const int noff = h->gf.noff, ctr = noff / 2;
    hwdf.resize((size_t)h->gf.N);
    for (int64_t pdof = 0; pdof < h->gf.N; ++pdof) {
      int64_t t = pdof;
      int cls = 0, mul = 1;
      for (int ax = 0; ax < o.dim; ++ax) {
        const int a = (int)(t % h->gf.W);
        t /= h->gf.W;
        cls += axis_class(a, h->gf.W, h->gf.R, h->gf.q) * mul;
        mul *= h->gf.C1;
      }
      const double2 c = Ae[(size_t)cls * noff + ctr], e = hrf[(size_t)pdof * noff + ctr];
      const double dr = c.x + e.x, di = c.y + e.y, m2 = dr * dr + di * di;
      hwdf[pdof] = m2 > 0 ? make_double2(o.omega * dr / m2, -o.omega * di / m2) : make_double2(0, 0);
    }
  }
  auto upload_het = [&](auto& p) -> int {
    using TT = typename std::remove_reference_t<decltype(p)>::value_type;
    if (!h->het) return HELM_OK;
    int r2;
    if ((r2 = upload<TT>(h, &p.hrow, hrf))) return r2;
    return upload<TT>(h, &p.hwd, hwdf);
  };

  if (h->op_only) {
    // fine-level operators and the smoother's workspaces only
    CK(h->alloc(&h->err, sizeof(int)));
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));
    const size_t Nf = (size_t)h->gf.N;
    if (o.precision == HELM_MIXED) {
      if ((rc = setup_prec<float>(h, Ae, wd, Ac, false))) return rc;
      CK(h->alloc(&h->p32.ua, sizeof(float2) * Nf));
      CK(h->alloc(&h->p32.ub, sizeof(float2) * Nf));
      CK(h->alloc(&h->p32.fT, sizeof(float2) * Nf));
    }
    if ((rc = setup_prec<double>(h, Ae, wd, Ac, false))) return rc;
    if (o.precision == HELM_FP64) {
      CK(h->alloc(&h->p64.ua, sizeof(double2) * Nf));
      CK(h->alloc(&h->p64.ub, sizeof(double2) * Nf));
    }
    CK(cudaStreamSynchronize(s));
    return HELM_OK;
  }

  // coarse block layout
  CoarseLayout& L = h->L;
  L.rows = h->order;
  L.plane = 1;
  for (int ax = 0; ax < o.dim - 1; ++ax) L.plane *= h->gc.W;
  L.nb = (h->gc.W + L.rows - 1) / L.rows;
  L.B = L.rows * L.plane;
  L.ldb = (L.B + 1) & ~1;
  L.mid = L.nb - 1;   // single chain unless the solve plan runs two clusters (set below)
  if (o.precision == HELM_MIXED) {
    if ((rc = setup_prec<float>(h, Ae, wd, Ac, true))) return rc;
    if ((rc = upload_het(h->p32))) return rc;
  }
  if ((rc = setup_prec<double>(h, Ae, wd, Ac, o.precision == HELM_FP64))) return rc;
  if ((rc = upload_het(h->p64))) return rc;

  // coarse factorisation (Sec. 6: factor once, reuse): complex128 for the FP64 form,
  // complex double-float (16-byte float4 entries) for the mixed form, whose factor is
  // rounded to complex64 for the V-cycle
  const bool df = o.precision == HELM_MIXED;
  size_t blk = (size_t)L.B * L.ldb;
  // scratch of the factorisation, freed on every early return; the work buffers are released
  // before the Krylov storage is allocated, and D64 is either kept by the handle or freed
  struct FactorScratch {
    double2 *D64 = nullptr, *tmp = nullptr, *piv = nullptr;
    unsigned* bar = nullptr;
    int* reuse = nullptr;
    void free_work() {
      cudaFree(tmp);
      cudaFree(piv);
      cudaFree(bar);
      cudaFree(reuse);
      tmp = piv = nullptr;
      bar = nullptr;
      reuse = nullptr;
    }
    ~FactorScratch() {
      free_work();
      cudaFree(D64);
    }
  } fs;
  double2*& D64 = fs.D64;   // 16 bytes per entry: double2 (FP64) or float4 (double-float)
  double2*& tmp = fs.tmp;
  double2*& piv = fs.piv;
  unsigned*& bar = fs.bar;
  CK(cudaMalloc(&D64, sizeof(double2) * blk * L.nb));
  CK(cudaMalloc(&tmp, sizeof(double2) * 2 * blk));
  CK(cudaMalloc(&piv, sizeof(double2) * 2 * factor_workspace(L)));
  CK(cudaMalloc(&bar, 2 * kBarWords * sizeof(unsigned)));
  CK(cudaMalloc(&fs.reuse, kReuseStateInts * sizeof(int)));
  CK(h->alloc(&h->err, sizeof(int)));
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));
  CK(cudaEventRecord(h->e0, s));
  StencilView<double> Acv = make_view<double>(h->gc, h->p64.coefAc, nullptr, h->hrowC);
  // (blocks of a heterogeneous operator differ from line to line: no reuse of inverses)
  int* reuse = h->het ? nullptr : fs.reuse;
  if (h->het) CK(cudaMemsetAsync(fs.reuse, 0, kReuseStateInts * sizeof(int), s));
  rc = df ? coarse_factor_df(reinterpret_cast<float4*>(D64), reinterpret_cast<float4*>(tmp),
                             reinterpret_cast<float4*>(piv), bar, h->err, Acv, L, h->nsm, s, reuse)
          : coarse_factor_fp64(D64, tmp, piv, bar, h->err, Acv, L, h->nsm, s, reuse);
  h->setup_kernels = std::max(L.mid, L.nb - 1 - L.mid) + 1 + 1 + (o.precision == HELM_MIXED ? 1 : 0);
  // which chains converged: the repeated blocks are mapped to the converged one (CoarseLayout)
  std::vector<int> cmap, pmapf, pmapb;
  if (rc == HELM_OK) {
    int st[kReuseStateInts];
    cudaError_t e = cudaMemcpyAsync(st, fs.reuse, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e);
    } else {
      h->reused_blocks = coarse_reused_blocks(st, L);
      const CoarsePlan* plan = o.precision == HELM_MIXED ? &h->p32.plan : &h->p64.plan;
      coarse_block_maps(L, plan, st, &cmap, &pmapf, &pmapb);
      auto put = [&](const std::vector<int>& v, const int** dst) -> int {
        if (v.empty() || h->reused_blocks == 0) return HELM_OK;   // identity
        int* d = nullptr;
        CK(h->alloc(&d, sizeof(int) * v.size()));
        CK(cudaMemcpyAsync(d, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s));
        *dst = d;
        return HELM_OK;
      };
      if (!rc) rc = put(cmap, &L.cmap);
      if (!rc) rc = put(pmapf, &L.pmapf);
      if (!rc) rc = put(pmapb, &L.pmapb);
      if (h->reused_blocks == 0) cmap.clear();
      // grouped block products: every use of one (mapped) block in one group of up to gcap
      std::vector<int> gg, gf, gb;
      L.gcap = coarse_group_lists(L, plan, o.precision == HELM_MIXED ? sizeof(float2) : sizeof(double2), cmap,
                                  pmapf, pmapb, &gg, &gf, &gb, &L.grows);
      auto put_groups = [&](const std::vector<int>& v, const int** dst, int* n) -> int {
        *n = (int)(v.size() / kGroupInts);
        if (v.empty()) return HELM_OK;
        int* d = nullptr;
        CK(h->alloc(&d, sizeof(int) * v.size()));
        CK(cudaMemcpyAsync(d, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s));
        *dst = d;
        return HELM_OK;
      };
      if (!rc) rc = put_groups(gg, &L.ggemv, &L.ngemv);
      if (!rc) rc = put_groups(gf, &L.gfixf, &L.nfixf);
      if (!rc) rc = put_groups(gb, &L.gfixb, &L.nfixb);
    }
  }
  // couplings folded into the inverses: Lm[J] = Dinv[J] A_J,J-1, Up[J] = Dinv[J] A_J,J+1
  if (rc == HELM_OK && o.precision == HELM_MIXED) {
    Prec<float>& p = h->p32;
    if (h->alloc(&p.Dinv, sizeof(float2) * blk * L.nb) != cudaSuccess ||
        h->alloc(&p.Lm, sizeof(float2) * blk * L.nb) != cudaSuccess ||
        h->alloc(&p.Up, sizeof(float2) * blk * L.nb) != cudaSuccess) {
      rc = HELM_ENOMEM;
    } else {
      convert_factor_df(reinterpret_cast<const float4*>(D64), p.Dinv, blk * L.nb, s);
      coarse_couple_df(reinterpret_cast<const float4*>(D64), p.Lm, p.Up, Acv, L, h->nsm, s);
      if (p.plan.seg) {
        float2 *yb = nullptr, *Pf = nullptr, *Pb = nullptr;
        if (h->alloc(&yb, sizeof(float2) * (size_t)L.nb * L.ldb) != cudaSuccess ||
            h->alloc(&Pf, sizeof(float2) * blk * L.nb) != cudaSuccess ||
            h->alloc(&Pb, sizeof(float2) * blk * L.nb) != cudaSuccess) {
          rc = HELM_ENOMEM;
        } else {
          p.seg = SegBufs<float>{yb, Pf, Pb};
          coarse_seg_products(p.Lm, p.Up, Pf, Pb, L, p.plan, s, cmap);
          h->setup_kernels += coarse_seg_launches(L, p.plan);
        }
      }
    }
  } else if (rc == HELM_OK) {
    Prec<double>& p = h->p64;
    if (h->alloc(&p.Lm, sizeof(double2) * blk * L.nb) != cudaSuccess ||
        h->alloc(&p.Up, sizeof(double2) * blk * L.nb) != cudaSuccess) {
      rc = HELM_ENOMEM;
    } else {
      coarse_couple_fp64(D64, p.Lm, p.Up, Acv, L, h->nsm, s);
    }
  }
  cudaEventRecord(h->e1, s);
  cudaEventSynchronize(h->e1);
  cudaEventElapsedTime(&h->setup_ms, h->e0, h->e1);
  fs.free_work();
  if (rc == HELM_OK) {
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) rc = cuda_fail(le);
  }
  if (rc == HELM_OK) {
    int e = check_err(h);
    if (e) rc = e;
  }
  if (rc != HELM_OK) return rc;   // (fs frees D64)
  if (o.precision == HELM_MIXED) {
    cudaFree(D64);
    D64 = nullptr;
  } else {
    h->p64.Dinv = D64;
    h->allocs.push_back(D64);
    h->bytes += sizeof(double2) * blk * L.nb;
    D64 = nullptr;   // owned by the handle now
  }

  // Krylov storage
  KrylovBufs& kb = h->kb;
  const int m = o.restart;
  kb.N = h->gf.N;
  kb.ldN = (kb.N + 31) & ~int64_t(31);
  // element-wise Krylov kernels: one entry per thread
  kb.nblk = (int)std::max<int64_t>(1, (kb.N + 255) / 256);
  kb.exact_gs = o.precision == HELM_MIXED ? 0 : 1;
  kb.nblk_dots = dots_blocks(kb.N, h->nsm, kb.exact_gs);
  kb.m = m;
  kb.nblk_upd = update_blocks(kb.N, h->nsm, kb.exact_gs, sizeof(float4) * 2 * m);
  kb.pstride = std::max(kb.nblk, std::max(kb.nblk_upd, kb.nblk_dots));
  CK(h->alloc(&kb.Vs, sizeof(float4) * kb.ldN * (m + 1)));
  CK(h->alloc(&kb.Ws, sizeof(float4) * kb.ldN));
  if (o.precision == HELM_MIXED) {
    kb.W = nullptr;
    kb.Z = nullptr;
    CK(h->alloc(&kb.Z32, sizeof(float2) * kb.ldN * m));
    CK(cudaMemsetAsync(kb.Z32, 0, sizeof(float2) * kb.ldN * m, s));
  } else {
    kb.Z32 = nullptr;
    CK(h->alloc(&kb.W, sizeof(double2) * kb.ldN));
    CK(h->alloc(&kb.Z, sizeof(double2) * kb.ldN * m));
    CK(cudaMemsetAsync(kb.W, 0, sizeof(double2) * kb.ldN, s));
    CK(cudaMemsetAsync(kb.Z, 0, sizeof(double2) * kb.ldN * m, s));
  }
  CK(h->alloc(&kb.H, sizeof(double2) * (m + 1) * m));
  CK(h->alloc(&kb.cs, sizeof(double) * m));
  CK(h->alloc(&kb.sn, sizeof(double2) * m));
  CK(h->alloc(&kb.g, sizeof(double2) * (m + 1)));
  CK(h->alloc(&kb.y, sizeof(double2) * m));
  CK(h->alloc(&kb.zs, sizeof(double) * m));
  CK(h->alloc(&kb.cdf, sizeof(double2) * (2 * m + 2)));
  CK(h->alloc(&kb.hcol, sizeof(double2) * (m + 2)));
  CK(h->alloc(&kb.hp, sizeof(double2) * (m + 2)));
  CK(h->alloc(&kb.tp, sizeof(double2) * (m + 2)));
  CK(h->alloc(&kb.part, sizeof(double2) * (size_t)kb.pstride * kb_rows(m)));
  CK(h->alloc(&kb.st, sizeof(KState)));
  CK(h->alloc(&h->rres, sizeof(double2) * kb.ldN));
  CK(cudaMallocHost(&h->st_h, sizeof(KState)));
  CK(cudaMallocHost(&h->err_h, sizeof(int)));
  CK(cudaMemsetAsync(kb.Vs, 0, sizeof(float4) * kb.ldN * (m + 1), s));
  CK(cudaStreamSynchronize(s));
  return capture_iteration(h);
}

static int setup_any(double k, double h, int order, double shift, const helm_opts* opts, helm_t* out,
                     bool op_only, int elements = HELM_SIMPLICES, const double* k_fine = nullptr,
                     const double* k_coarse = nullptr) {
  if (!out) return HELM_EINVAL;
  *out = nullptr;
  helm_opts o;
  helm_default_opts(&o);
  if (opts) o = *opts;
  if (!(h > 0) || !(k > 0) || !(shift >= 0) || !std::isfinite(k) || !std::isfinite(shift)) return HELM_EINVAL;
  double nn = 1.0 / h;
  int n = (int)std::lround(nn);
  if (std::fabs(nn - n) > 1e-9 * nn || n < 4 || n % 2) return HELM_EINVAL;
  const bool q3 = elements == HELM_TENSOR && o.dim == 2 && order == 3;   // Q3 (2D, Gauss-Lobatto nodes)
  if (!(o.dim == 2 || o.dim == 3) || !(order == 1 || order == 2 || q3) || (o.dim == 3 && order != 1))
    return HELM_EINVAL;
  if (o.nu < 1 || o.nu > 8 || o.restart < 1 || o.restart > 512 || o.maxit < 1 || !(o.tol > 0) ||
      !(o.omega > 0) || !(o.precision == HELM_FP64 || o.precision == HELM_MIXED))
    return HELM_EINVAL;
  helm_ctx* c = new (std::nothrow) helm_ctx();
  if (!c) return HELM_ENOMEM;
  c->dim = o.dim;
  c->order = order;
  c->n = n;
  c->k = k;
  c->h = h;
  c->shift = shift;
  c->opts = o;
  c->s = (cudaStream_t)o.stream;
  c->op_only = op_only;
  c->elements = elements;
  if (k_fine) {
    // one wavenumber per element of each level (copied; k is their maximum, for reference)
    const int64_t nf = num_elements(o.dim, n, elements), nc = num_elements(o.dim, n / 2, elements);
    c->het = true;
    c->kf.assign(k_fine, k_fine + nf);
    c->kc.assign(k_coarse, k_coarse + nc);
    bool ok = true;
    for (double v : c->kf) ok = ok && std::isfinite(v) && v >= 0;
    for (double v : c->kc) ok = ok && std::isfinite(v) && v >= 0;
    if (!ok) {
      delete c;
      return HELM_EINVAL;
    }
  }
  int rc = setup_impl(c);
  if (rc != HELM_OK) {
    helm_destroy(c);
    return rc;
  }
  *out = c;
  return HELM_OK;
}

int helm_setup(double k, double h, int order, double shift, const helm_opts* opts, helm_t* out) {
  return setup_any(k, h, order, shift, opts, out, false);
}

int helm_setup_het(int elements, const double* k_fine, const double* k_coarse, double h, int order, double shift,
                   const helm_opts* opts, helm_t* out) {
  if (!k_fine || !k_coarse || !(elements == HELM_SIMPLICES || elements == HELM_TENSOR) || !out) return HELM_EINVAL;
  double kmax = 0;
  helm_opts o;
  helm_default_opts(&o);
  if (opts) o = *opts;
  const double nn = 1.0 / h;
  if (!(h > 0) || !(nn < 1e6) || !(o.dim == 2 || o.dim == 3)) return HELM_EINVAL;
  const int n = (int)std::lround(nn);
  if (n < 4 || n % 2) return HELM_EINVAL;
  const int64_t nf = num_elements(o.dim, n, elements);
  for (int64_t i = 0; i < nf; ++i) kmax = std::max(kmax, std::isfinite(k_fine[i]) ? k_fine[i] : -1.0);
  if (!(kmax > 0)) return HELM_EINVAL;
  return setup_any(kmax, h, order, shift, opts, out, false, elements, k_fine, k_coarse);
}

int helm_operator_setup(double k, double h, int order, double shift, const helm_opts* opts, helm_t* out) {
  return setup_any(k, h, order, shift, opts, out, true);
}

int helm_setup_q(double k, double h, int order, double shift, const helm_opts* opts, helm_t* out) {
  return setup_any(k, h, order, shift, opts, out, false, HELM_TENSOR);
}

int helm_num_dofs(helm_t h, int64_t* n) {
  if (!h || !n) return HELM_EINVAL;
  *n = h->gf.N;
  return HELM_OK;
}

int helm_num_coarse_dofs(helm_t h, int64_t* n) {
  if (!h || !n) return HELM_EINVAL;
  *n = h->gc.N;
  return HELM_OK;
}

int helm_factor_info(helm_t h, int* factored, int* reused) {
  if (!h || h->op_only) return HELM_EINVAL;
  if (factored) *factored = h->L.nb - h->reused_blocks;
  if (reused) *reused = h->reused_blocks;
  return HELM_OK;
}

int helm_setup_info(helm_t h, float* ms, int* kernels) {
  if (!h) return HELM_EINVAL;
  if (ms) *ms = h->setup_ms;
  if (kernels) *kernels = h->setup_kernels;
  return HELM_OK;
}

int helm_solve(helm_t h, const void* F, void* x, helm_result* res) {
  if (!h || !F || !x || h->op_only) return HELM_EINVAL;
  SolveTask t{h, (const double2*)F, (double2*)x, res};
  int rc = solve_begin(t);
  if (rc) return rc;
  while (!solve_step(t, true)) {
  }
  return t.rc;
}

int helm_solve_host(helm_t h, const void* F_host, void* x_host, helm_result* res) {
  if (!h || !F_host || !x_host || h->op_only) return HELM_EINVAL;
  size_t bytes = sizeof(double2) * h->gf.N;
  if (!h->Fdev) {
    CK(h->alloc(&h->Fdev, bytes));
    CK(h->alloc(&h->xdev, bytes));
  }
  CK(cudaMemcpyAsync(h->Fdev, F_host, bytes, cudaMemcpyHostToDevice, h->s));
  int rc = helm_solve(h, h->Fdev, h->xdev, res);
  if (rc) return rc;
  CK(cudaMemcpyAsync(x_host, h->xdev, bytes, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  return HELM_OK;
}

int helm_batch_solve(int count, const helm_t* hs, const void* const* F, void* const* x, helm_result* res) {
  if (count < 0 || (count > 0 && (!hs || !F || !x))) return HELM_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !F[i] || !x[i] || hs[i]->op_only) return HELM_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return HELM_EINVAL;
  }
  std::vector<SolveTask> tasks(count);
  int rc = HELM_OK;
  for (int i = 0; i < count; ++i) {
    tasks[i] = SolveTask{hs[i], (const double2*)F[i], (double2*)x[i], res ? &res[i] : nullptr};
    int r = solve_begin(tasks[i]);
    if (r) return r;
  }
  int left = count;
  while (left > 0) {
    left = 0;
    for (auto& t : tasks) {
      if (t.phase == SolveTask::DONE) continue;
      if (!solve_step(t, false)) ++left;
    }
  }
  for (auto& t : tasks)
    if (t.rc && !rc) rc = t.rc;
  return rc;
}

int helm_rhs_planewave(helm_t h, double theta, void* F_host) {
  if (!h || !F_host || h->het) return HELM_EINVAL;   // (the plane wave needs one wavenumber)
  rhs_planewave(h->dim, h->order, h->n, h->k, theta, (double2*)F_host, h->elements);
  return HELM_OK;
}

int helm_rhs_source(helm_t h, double sx, double sy, double sz, void* F_host) {
  if (!h || !F_host) return HELM_EINVAL;
  // f = 2 exp(-1000 |x - s|^2) = 2 exp(-|x - s|^2 / (2 sigma^2)) with sigma^2 = 1 / 2000, g = 0
  double c[3] = {sx, sy, sz};
  rhs_gaussian(h->dim, h->order, h->n, std::sqrt(1.0 / 2000.0), c, (double2*)F_host, h->elements);
  double2* F = (double2*)F_host;
  for (int64_t i = 0; i < h->gf.N; ++i) F[i] = make_double2(2.0 * F[i].x, 2.0 * F[i].y);
  return HELM_OK;
}

int helm_rhs_gaussian(helm_t h, double sigma, double cx, double cy, double cz, void* F_host) {
  if (!h || !F_host || !(sigma > 0)) return HELM_EINVAL;
  double c[3] = {cx, cy, cz};
  rhs_gaussian(h->dim, h->order, h->n, sigma, c, (double2*)F_host, h->elements);
  return HELM_OK;
}

static int mesh_n(int dim, int order, double h, bool q3_ok = false) {
  const bool q3 = q3_ok && dim == 2 && order == 3;
  if (!(h > 0) || !(dim == 2 || dim == 3) || !(order == 1 || order == 2 || q3) || (dim == 3 && order != 1))
    return -1;
  const double nn = 1.0 / h;
  if (!(nn < 1e6)) return -1;   // beyond any mesh whose DoF count fits the cap below
  const int n = (int)std::lround(nn);
  if (std::fabs(nn - n) > 1e-9 * nn || n < 4 || n % 2) return -1;
  int64_t N = 1;
  for (int d = 0; d < dim; ++d) N *= (int64_t)order * n + 1;
  if (N >= (1ll << 31) / 2) return -1;   // the solver's DoF cap
  return n;
}

int helm_load_planewave(int dim, int order, double h, double k, double theta, void* F_host) {
  const int n = mesh_n(dim, order, h);
  if (n < 0 || !F_host || !(k > 0)) return HELM_EINVAL;
  rhs_planewave(dim, order, n, k, theta, (double2*)F_host);
  return HELM_OK;
}

int helm_load_planewave_e(int dim, int order, int elements, double h, double k, double theta, void* F_host) {
  const int n = mesh_n(dim, order, h, elements == HELM_TENSOR);
  if (n < 0 || !(elements == HELM_SIMPLICES || elements == HELM_TENSOR) || !F_host || !(k > 0)) return HELM_EINVAL;
  rhs_planewave(dim, order, n, k, theta, (double2*)F_host, elements);
  return HELM_OK;
}

int helm_load_gaussian_e(int dim, int order, int elements, double h, double sigma, double cx, double cy, double cz,
                         void* F_host) {
  const int n = mesh_n(dim, order, h, elements == HELM_TENSOR);
  if (n < 0 || !(elements == HELM_SIMPLICES || elements == HELM_TENSOR) || !F_host || !(sigma > 0))
    return HELM_EINVAL;
  double c[3] = {cx, cy, cz};
  rhs_gaussian(dim, order, n, sigma, c, (double2*)F_host, elements);
  return HELM_OK;
}

int helm_host_stencil_row(int dim, int order, int elements, double h, int level, int64_t dof, double* K,
                          double* M, double* B) {
  const int n = mesh_n(dim, order, h, elements == HELM_TENSOR);
  if (n < 0 || !(elements == HELM_SIMPLICES || elements == HELM_TENSOR) || !(level == 0 || level == 1) || !K ||
      !M || !B)
    return HELM_EINVAL;
  HostTables t;
  const int rc = build_tables(dim, order, n, &t, elements);
  return rc != HELM_OK ? rc : host_stencil_row(t, level, dof, K, M, B);
}

int helm_host_het_row(int dim, int order, int elements, double h, int level, const double* k_elem, int64_t dof,
                      double* K, double* Mk, double* M, double* Bk) {
  const int n = mesh_n(dim, order, h, elements == HELM_TENSOR);
  if (n < 0 || !(level == 0 || level == 1) || !k_elem || !K || !Mk || !M || !Bk) return HELM_EINVAL;
  HetRows r;
  const int rc = build_het_rows(dim, order, level == 0 ? n : n / 2, elements, k_elem, &r);
  if (rc != HELM_OK) return rc;
  if (dof < 0 || dof >= r.g.N) return HELM_EINVAL;
  for (int o = 0; o < r.g.noff; ++o) {
    const size_t i = (size_t)dof * r.g.noff + o;
    K[o] = r.K[i];
    Mk[o] = r.Mk[i];
    M[o] = r.M[i];
    Bk[o] = r.Bk[i];
  }
  return HELM_OK;
}

int helm_host_prolongation_row(int dim, int order, int elements, double h, int64_t fine_dof, int64_t* cols,
                               double* w, int* count) {
  const int n = mesh_n(dim, order, h, elements == HELM_TENSOR);
  if (n < 0 || !(elements == HELM_SIMPLICES || elements == HELM_TENSOR) || !cols || !w || !count)
    return HELM_EINVAL;
  HostTables t;
  const int rc = build_tables(dim, order, n, &t, elements);
  return rc != HELM_OK ? rc : host_prolongation_row(t, fine_dof, cols, w, count);
}

int helm_load_gaussian(int dim, int order, double h, double sigma, double cx, double cy, double cz, void* F_host) {
  const int n = mesh_n(dim, order, h);
  if (n < 0 || !F_host || !(sigma > 0)) return HELM_EINVAL;
  double c[3] = {cx, cy, cz};
  rhs_gaussian(dim, order, n, sigma, c, (double2*)F_host);
  return HELM_OK;
}

int helm_apply(helm_t h, int which, const void* x, void* y) {
  if (!h || !x || !y || (which != 0 && which != 1)) return HELM_EINVAL;
  StencilView<double> A = which == 0 ? make_view<double>(h->gf, h->coefA0, nullptr, h->hrowA0)
                                     : make_view<double>(h->gf, h->p64.coefAe, nullptr, h->hrowA0);
  launch_apply<double, double2, double2>(A, vsel<const double2>((const double2*)x), vsel<double2>((double2*)y),
                                         nullptr, h->s);
  CK(cudaGetLastError());
  return HELM_OK;
}


int helm_smooth(helm_t h, const void* f, void* u, int nu) {
  if (!h || !f || !u || nu < 2 || nu > 8) return HELM_EINVAL;
  if (h->opts.precision == HELM_MIXED)
    enqueue_smooth<float>(h, (const double2*)f, (double2*)u, nu, h->s);
  else
    enqueue_smooth<double>(h, (const double2*)f, (double2*)u, nu, h->s);
  CK(cudaGetLastError());
  return HELM_OK;
}

int helm_vcycle(helm_t h, const void* f, void* u) {
  if (!h || !f || !u || h->op_only) return HELM_EINVAL;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));
  enqueue_vcycle_any(h, vsel<const double2>((const double2*)f), vsel<double2>((double2*)u), nullptr, h->s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->s));
  return check_err(h);
}

int helm_coarse_solve(helm_t h, const void* rc_nat, void* uc_nat) {
  if (!h || !rc_nat || !uc_nat || h->op_only) return HELM_EINVAL;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));
  if (h->opts.precision == HELM_MIXED) {
    Prec<float>& p = h->p32;
    launch_coarse_pack<double2, float2>(h->gc, h->L, (const double2*)rc_nat, p.rc, h->s);
    launch_coarse_solve<float>(p.plan, p.Dinv, p.Lm, p.Up, h->L, p.rc, p.uc, p.gbar, h->err,
                               nullptr, h->nsm, h->s, p.segp());
    launch_coarse_unpack<float2, double2>(h->gc, h->L, p.uc, (double2*)uc_nat, h->s);
  } else {
    Prec<double>& p = h->p64;
    launch_coarse_pack<double2, double2>(h->gc, h->L, (const double2*)rc_nat, p.rc, h->s);
    launch_coarse_solve<double>(p.plan, p.Dinv, p.Lm, p.Up, h->L, p.rc, p.uc, p.gbar, h->err,
                                nullptr, h->nsm, h->s);
    launch_coarse_unpack<double2, double2>(h->gc, h->L, p.uc, (double2*)uc_nat, h->s);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->s));
  return check_err(h);
}

int helm_set_profiling(helm_t h, int on) {
  if (!h) return HELM_EINVAL;
  h->prof.on = on != 0;
  for (int i = 0; i < Profile::kPhases; ++i) {
    h->prof.ms[i] = 0;
    h->prof.calls[i] = 0;
  }
  return HELM_OK;
}

int helm_last_profile(helm_t h, int cap, const char** names, double* ms, int* calls, int* n) {
  if (!h || !n) return HELM_EINVAL;
  int k = std::min(cap, Profile::kPhases);
  for (int i = 0; i < k; ++i) {
    if (names) names[i] = kPhaseNames[i];
    if (ms) ms[i] = h->prof.ms[i];
    if (calls) calls[i] = h->prof.calls[i];
  }
  *n = Profile::kPhases;
  return HELM_OK;
}

}  // extern "C"

// ============================================================================
// Coarse solve without device allocation (helm_coarse_solve_noalloc).
//
// The two block-padded coarse vectors that helm_coarse_solve keeps in the
// handle live here in one file-scope device array instead. In host code the
// symbol g_noalloc_scratch only names a host-side stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and cached; the kernels receive that address.
// ============================================================================
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
// Device address of the scratch array on device `dev`, which must be the current device
// (first call on that device: lookup).
int noalloc_scratch(int dev, void** out) {
  int cur = -1;
  CK(cudaGetDevice(&cur));
  if (cur != dev) return HELM_EINVAL;
  if (dev < 0 || dev >= kMaxDevices) return HELM_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return HELM_OK;
}

template <typename T>
int coarse_solve_noalloc(helm_t h, const double2* rc_nat, double2* uc_nat) {
  using V = c2<T>;
  Prec<T>& p = h->prec<T>();
  const size_t nvec = (size_t)h->L.nb * h->L.ldb;
  if (2 * nvec * sizeof(V) > kNoAllocScratchBytes) return HELM_ESCRATCH;
  void* base = nullptr;
  int rc = noalloc_scratch(h->dev, &base);
  if (rc) return rc;
  V* pad_rc = static_cast<V*>(base);
  V* pad_uc = pad_rc + nvec;   // 16-byte aligned: nvec * sizeof(V) is a multiple of 16 (ldb even)
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->s));   // the error word must start at zero
  launch_coarse_pack<double2, V>(h->gc, h->L, rc_nat, pad_rc, h->s);   // writes every padded entry
  launch_coarse_solve<T>(p.plan, p.Dinv, p.Lm, p.Up, h->L, pad_rc, pad_uc, p.gbar, h->err,
                         nullptr, h->nsm, h->s, p.segp());
  launch_coarse_unpack<V, double2>(h->gc, h->L, pad_uc, uc_nat, h->s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->s));
  return check_err(h);
}
}  // namespace

extern "C" int helm_coarse_solve_noalloc(helm_t h, const void* rc, void* uc) {
  if (!h || !rc || !uc || h->op_only) return HELM_EINVAL;
  if (h->opts.precision == HELM_MIXED)
    return coarse_solve_noalloc<float>(h, (const double2*)rc, (double2*)uc);
  return coarse_solve_noalloc<double>(h, (const double2*)rc, (double2*)uc);
}
