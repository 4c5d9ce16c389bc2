// Launchers of the hot-path kernels (internal to the library).
#pragma once

#include <vector>

#include "common.cuh"

namespace helm {

// Index selection from device state: a pointer into a strided array of vectors,
// base + (*jsel + jadd) * stride, so that a captured graph can address the
// current Krylov column without being re-captured.
template <typename V> struct VecSel {
  V* base;
  int64_t stride;
  const int* jsel;   // null -> index jadd
  int jadd;
  __device__ __forceinline__ V* ptr() const {
    return base + (int64_t)((jsel ? *jsel : 0) + jadd) * stride;
  }
};
template <typename V> inline VecSel<V> vsel(V* p) { return VecSel<V>{p, 0, nullptr, 0}; }

// ---- fine level (stencil.cu) -----------------------------------------------
// y = A x
template <typename T, typename Vin, typename Vout>
void launch_apply(const StencilView<T>& A, VecSel<const Vin> x, VecSel<Vout> y, const int* active,
                  cudaStream_t s, float4* ws = nullptr);   // ws: optional double-float split of y
                                                          // (y.base null: ws only)
// ws = A x in double-float from complex64 x and the complex128 table A (products exact to
// the double-float rounding of the coefficients)
void launch_apply_df(const StencilView<double>& A, VecSel<const float2> x, float4* ws, const int* active,
                     cudaStream_t s);
// r = f - A u
template <typename T, typename Vf, typename Vr>
void launch_residual(const StencilView<T>& A, VecSel<const Vf> f, const c2<T>* u, Vr* r,
                     const int* active, cudaStream_t s);
// u_out = omega D^-1 f (+ one more sweep if two_steps): the first nu <= 2 sweeps from u = 0.
// If fcopy != null, f is also stored in precision T there.
template <typename T, typename Vf>
void launch_jacobi_from_zero(const StencilView<T>& A, VecSel<const Vf> f, c2<T>* u_out,
                             c2<T>* fcopy, bool two_steps, const int* active, cudaStream_t s);
// out = u + omega D^-1 (f - A u)
template <typename T, typename Vf, typename Vout>
void launch_jacobi(const StencilView<T>& A, VecSel<const Vf> f, const c2<T>* u, VecSel<Vout> out,
                   const int* active, cudaStream_t s);
// u += P uc  (uc in block-padded coarse layout)
template <typename T>
void launch_prolong_add(const TransferView<T>& P, const CoarseLayout& L, const c2<T>* uc, c2<T>* u,
                        const int* active, cudaStream_t s);
// rc = P^T r (rc in block-padded coarse layout, padding zeroed)
template <typename T>
void launch_restrict(const TransferView<T>& P, const CoarseLayout& L, const c2<T>* r, c2<T>* rc,
                     const int* active, cudaStream_t s);
// padded <-> natural coarse ordering (with precision conversion)
// nu damped-Jacobi sweeps fused on 2D tiles (smooth.cu): from u^0 = 0 (u0 null) or from
// u^0 = u0 + P uc (post-smoothing; uc null: u0 alone); writes u^nu to out and, when r is
// given, the residual f - A u^nu. Returns false (nothing launched) where it does not apply
// (3D, or a tile that does not fit shared memory): the caller then runs the per-sweep kernels.
template <typename T>
void smooth_tile_prepare();
void stencil_prepare();   // (the same for the per-sweep and apply kernels' 49-point tables)   // raises the kernels' shared-memory limit (outside stream capture)
template <typename T, typename Vf, typename Vout>
bool launch_smooth_tile(const StencilView<T>& A, VecSel<const Vf> f, const c2<T>* u0, const TransferView<T>* P,
                        const CoarseLayout* L, const c2<T>* uc, int nu, VecSel<Vout> out, c2<T>* r,
                        const int* active, cudaStream_t s);
template <typename Vin, typename Vout>
void launch_coarse_pack(const GridDesc& gc, const CoarseLayout& L, const Vin* nat, Vout* pad,
                        cudaStream_t s);
template <typename Vin, typename Vout>
void launch_coarse_unpack(const GridDesc& gc, const CoarseLayout& L, const Vin* pad, Vout* nat,
                          cudaStream_t s);

// ---- coarse level (coarse.cu) ----------------------------------------------
struct CoarsePlan {
  int grid;     // 1: whole-grid chain (blocks too large for a cluster), 0: cluster kernel
  int ncl;      // clusters: 2 = twisted (top and bottom chains), 1 = single chain
  int CS;       // cluster size
  int R;        // rows per CTA
  int CW;       // columns per pipeline chunk (even)
  int nchunk;   // chunks per step
  int S;        // pipeline stages
  int nblk;     // CTAs of the grid kernel
  size_t smem;  // dynamic shared memory bytes
  int threads;
  int seg;      // 1: segmented triangular solves (complex64, twisted factorisation)
  int K;        // phase-A clusters (segments) per half-sweep path
  // phase B of the segmented solve (two clusters): its own cluster geometry
  int CSb, Rb, CWb, nchunkb, Sb, threadsb;
  size_t smemb;
};
// Workspaces of the segmented solve: yb one block-padded coarse vector; Pf, Pb the
// segment products of the forward and backward sweeps, nb x B x ldb each, by block.
template <typename T> struct SegBufs {
  c2<T>* yb;
  const c2<T>* Pf;
  const c2<T>* Pb;
};
template <typename T>
int plan_coarse_solve(const CoarseLayout& L, CoarsePlan* plan);
// uc = A^{-1} rc for the block-padded coarse vectors (uc also holds the block-diagonal
// pre-pass p = Dinv r). plan.seg with seg given: the segmented half-sweeps of the twisted
// form (seg->yb holds the forward sweep). Otherwise L.mid < L.nb - 1 runs the twisted form
// as three launches (forward chains, middle block, backward chains); bar: kBarWords unsigned
// for the grid kernel's barrier.
template <typename T>
void launch_coarse_solve(const CoarsePlan& plan, const c2<T>* Dinv, const c2<T>* Lm, const c2<T>* Up,
                         const CoarseLayout& L, const c2<T>* rc, c2<T>* uc, unsigned* bar, int* err,
                         const int* active, int nsm, cudaStream_t s, const SegBufs<T>* seg = nullptr);
// Segment products of both sweeps (plan.seg, complex64), and the number of launches it takes;
// segments that only repeat an earlier one (cmap_host: the host copy of L.cmap, may be empty)
// are not computed
void coarse_seg_products(const float2* Lm, const float2* Up, float2* Pf, float2* Pb, const CoarseLayout& L,
                         const CoarsePlan& plan, cudaStream_t s, const std::vector<int>& cmap_host);
// Host block maps (see CoarseLayout) from the factorisation's reuse state (host copy): cmap for
// the inverses and couplings, pmapf / pmapb for the segment products (left empty without plan.seg)
void coarse_block_maps(const CoarseLayout& L, const CoarsePlan* plan, const int* reuse_host, std::vector<int>* cmap,
                       std::vector<int>* pmapf, std::vector<int>* pmapb);
// Host group lists of the grouped block products (see CoarseLayout) from the block maps (empty
// map = identity): gemv for the pre-pass, fixf / fixb for the segmented sweeps' fix-ups (left
// empty without plan.seg), and the rows per slab (grows). Returns the group capacity (1, 2 or 4
// vectors: as many blocks of elem-byte values as 48 KB of shared memory holds; 0 = none fits,
// lists left empty).
int coarse_group_lists(const CoarseLayout& L, const CoarsePlan* plan, size_t elem, const std::vector<int>& cmap,
                       const std::vector<int>& pmapf, const std::vector<int>& pmapb, std::vector<int>* gemv,
                       std::vector<int>* fixf, std::vector<int>* fixb, int* grows);
int coarse_seg_launches(const CoarseLayout& L, const CoarsePlan& plan);
// Block-Thomas factorisation: Dinv[J] = (A_JJ - A_J,J-1 Dinv[J-1] A_J-1,J)^{-1} (two chains
// meeting at L.mid), in complex128 (8-pivot Gauss-Jordan panels) or in complex double-float
// (float4 hi/lo pairs, 16-pivot panels). tmp: 2 x B x ldb; piv: 2 x factor_workspace(L)
// elements; bar: 2 x kBarWords unsigned (two halves of the grid factor the two chains concurrently).
__host__ __device__ inline size_t factor_workspace(const CoarseLayout& L) {
  return 2 * 16 * (size_t)L.ldb + 2 * 16 * (size_t)L.B + 2 * 16 * 16;
}
// reuse (may be null): 2 x 8 ints of device state; when given, a chain whose inverse stopped
// changing (relative change below the precision's tolerance twice in a row) copies it to the
// rest of the chain instead of factoring; coarse_reused_blocks counts the copied blocks from a
// host copy of that state.
int coarse_factor_fp64(double2* Dinv, double2* tmp, double2* piv, unsigned* bar, int* err,
                       const StencilView<double>& Ac, const CoarseLayout& L, int nsm, cudaStream_t s, int* reuse);
int coarse_factor_df(float4* Dinv, float4* tmp, float4* piv, unsigned* bar, int* err,
                     const StencilView<double>& Ac, const CoarseLayout& L, int nsm, cudaStream_t s, int* reuse);
constexpr int kReuseStateInts = 16;
int coarse_reused_blocks(const int* reuse_host, const CoarseLayout& L);
// Lm[J] = Dinv[J] A_J,J-1 and Up[J] = Dinv[J] A_J,J+1 from the inverses (nb x B x ldb each)
void coarse_couple_fp64(const double2* D, double2* Lm, double2* Up, const StencilView<double>& Ac,
                        const CoarseLayout& L, int nsm, cudaStream_t s);
void coarse_couple_df(const float4* D, float2* Lm, float2* Up, const StencilView<double>& Ac, const CoarseLayout& L,
                      int nsm, cudaStream_t s);
// complex64 nearest to each double-float entry
void convert_factor_df(const float4* src, float2* dst, size_t n, cudaStream_t s);

// ---- Krylov (krylov.cu) ----------------------------------------------------
struct KState {
  int j;           // Arnoldi step of this cycle (slot j holds the vector u_j being finished);
                   // when the cycle stops: the number of finished columns
  int active;      // 1 while the cycle runs
  int total;       // finished Arnoldi columns over all cycles
  int converged;   // Givens estimate <= tol
  int breakdown;   // h_{j+1,j} == 0
  int pre;         // this step applies the preconditioner and A0 (else it only finishes column j-1)
  int ju;          // step whose correction sweep runs (j is already the next step by then)
  int m, maxit;
  int nonfinite;
  double nF;       // ||F||
  double beta;     // cycle's initial residual norm
  double tol;
  double est;      // |g_{j+1}| / ||F||
  double gabs;     // |g| of the last rotated column (|g_{c+1}| = |s_c| |g_c|)
  double inv_nF;   // 1 / ||F||
  double relres;   // true relative residual at cycle end
};

// Rows of the partials buffer (entry-major, kb.pstride apart): the inner products
// s_i = <v_i, u_j> (rows 0..m), t_i = <v_i, w> (rows m+1..2m+1) and one row of norms.
__host__ __device__ inline int64_t kb_row_s(int i) { return i; }
__host__ __device__ inline int64_t kb_row_t(int m, int i) { return (int64_t)m + 1 + i; }
__host__ __device__ inline int64_t kb_row_norm(int m) { return 2 * (int64_t)m + 2; }
__host__ __device__ inline int64_t kb_rows(int m) { return 2 * (int64_t)m + 3; }

struct KrylovBufs {
  // Krylov basis V in double-float form: each complex128 entry as a pair of
  // complex64 (hi + lo), 16 bytes like complex128, used by the Gram-Schmidt
  // kernels at FP32 throughput with ~48-bit accurate inner products.
  float4* Vs;      // (m+1) x ldN: (hi.re, hi.im, lo.re, lo.im) per entry
  double2* W;      // FP64 form: u_{j+1} in complex128, the next step's preconditioner input
                   // (null in the complex64 form, whose preconditioner reads slot j + 1)
  float4* Ws;      // w = A0 z_j as a double-float pair per entry (written by the apply)
  double2* Z;      // m x ldN preconditioned vectors, complex128 (FP64 form), or
  float2* Z32;     // the same in complex64 (complex64 form, where z_j is complex64 exactly)
  int64_t ldN;
  int64_t N;
  double2* H;      // (m+1) x m column-major, rotated (upper triangular R)
  double* cs;      // m
  double2* sn;     // m
  double2* g;      // m+1
  double2* y;      // m
  double* zs;      // m : scale of each preconditioned vector (1 / rho of its step)
  double2* cdf;    // 2m + 2 (as float4): the correction sweep's coefficients in double-float
  double2* hcol;   // m+2 : the column started by the previous step (finished by this one)
  double2* hp;     // m+1 : s_i = <v_i, u_j>
  double2* tp;     // m+1 : t_i = <v_i, w>
  double2* part;   // pstride x kb_rows(m) partial sums (inner products: double-float as float4)
  int nblk;        // blocks of the element-wise Krylov kernels (256 threads, one entry per thread)
  int nblk_dots;   // blocks of the inner-product kernel (dots_blocks(N, SMs))
  int m;           // restart length (host copy of KState::m, sizes launches)
  int nblk_upd;    // blocks of the update kernel (update_blocks)
  int pstride;     // row stride of the partials buffer: max over the kernels that write it
  int exact_gs;    // 1: both Gram-Schmidt passes in double-float (FP64 form); 0: the first
                   // pass's projections and the second pass's small correction sum in float
  KState* st;
};

// One Arnoldi step after w = A0 z_j: inner products, coefficients (finishing column j-1 with
// its Givens step), the joint correction sweep and u_{j+1} = w / ||w||. `mid` (may be null)
// is recorded between the coefficient kernel and the correction sweep.
void launch_arnoldi(const KrylovBufs& kb, cudaStream_t s, cudaEvent_t mid);
// blocks of the inner-product kernel for N entries: one wave on nsm SMs (exact: FP64 form)
int dots_blocks(int64_t N, int nsm, bool exact);
// blocks of the correction sweep (smem: its dynamic shared memory, 2 m float4)
int update_blocks(int64_t N, int nsm, bool exact, size_t smem);
void launch_cycle_start(const KrylovBufs& kb, const double2* r, cudaStream_t s);   // V0 = r / ||r||
void launch_backsolve(const KrylovBufs& kb, cudaStream_t s);
void launch_update_x(const KrylovBufs& kb, double2* x, cudaStream_t s);
// ||v||^2 into st field (which: 0 = nF (and beta), 1 = relres using nF)
void launch_norm(const KrylovBufs& kb, const double2* v, int which, cudaStream_t s);

}  // namespace helm
