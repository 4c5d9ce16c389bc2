// Shared device/host definitions of the GB300 Helmholtz twogrid-FGMRES library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <vector>

#include "helm.h"

namespace helm {

// ----------------------------------------------------------------------------
// Complex arithmetic on float2 / double2 (interleaved re, im).
// ----------------------------------------------------------------------------
template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <typename T> using c2 = typename C2<T>::type;

__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }

template <typename V> __host__ __device__ inline V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V> __host__ __device__ inline V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
template <typename V> __host__ __device__ inline V cmul(V a, V b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
template <typename V> __host__ __device__ inline V cfma(V a, V b, V acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc += conj(a) * b
template <typename V> __host__ __device__ inline V cfma_conj(V a, V b, V acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
template <typename V> __host__ __device__ inline V cinv(V a) {
  auto d = a.x * a.x + a.y * a.y;
  return mk(a.x / d, -a.y / d);
}

#if defined(__CUDACC__)
// conversions between precisions
__device__ inline float2 cvt(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
__device__ inline double2 cvt(float2 v, double2*) { return make_double2(v.x, v.y); }
__device__ inline float2 cvt(float2 v, float2*) { return v; }
__device__ inline double2 cvt(double2 v, double2*) { return v; }
// a double-float pair (hi.re, hi.im, lo.re, lo.im) read as complex64: its high parts, the
// nearest complex64 value of a normalised pair
__device__ inline float2 cvt(float4 v, float2*) { return make_float2(v.x, v.y); }
template <typename To, typename From> __device__ inline To to(From v) { return cvt(v, (To*)nullptr); }
#endif

// ----------------------------------------------------------------------------
// DoF grids and per-class stencils.
//
// A level's DoFs form a W^dim lattice (W = order*n + 1). Along each axis an
// index a belongs to one of C1 = 2R + q classes: the R positions nearest each
// boundary are their own classes, interior positions are classed by a mod q
// (R = reach of the stencil in lattice units = order, q = lattice period =
// order). The d-dimensional class is the mixed-radix number of the per-axis
// classes. Every DoF of a class has the same stencil (constant k, uniform
// mesh), with noff = (2R+1)^dim offsets in lexicographic box order.
// ----------------------------------------------------------------------------
constexpr int kMaxOff = 49;   // (2*1+1)^3 = 27, (2*2+1)^2 = 25, (2*3+1)^2 = 49 (Q3)
constexpr int kMaxCls = 81;   // (2*2+2)^2 = 36, (2+1)^3 = 27, (2*3+3)^2 = 81 (Q3)
constexpr int kMaxPW = 36;    // prolongation classes: (2q)^dim <= 36
constexpr int kMaxPO = 16;    // prolongation offsets: (q+1)^dim <= 16

struct GridDesc {
  int dim;      // 2 or 3
  int W;        // lattice points per side
  int R;        // stencil reach (lattice units)
  int q;        // lattice period
  int C1;       // per-axis classes = 2R + q
  int noff;     // (2R+1)^dim
  int64_t N;    // W^dim
};

// division and remainder by a small lattice period or transfer period (1, 2 and 4 are the
// periods of P1 and P2; they take shifts instead of an integer division)
__host__ __device__ inline int div_period(int a, int d) { return d == 1 ? a : d == 2 ? a >> 1 : d == 4 ? a >> 2 : a / d; }
__host__ __device__ inline int mod_period(int a, int d) { return d == 1 ? 0 : d == 2 ? a & 1 : d == 4 ? a & 3 : a % d; }

__host__ __device__ inline int axis_class(int a, int W, int R, int q) {
  if (a < R) return a;
  if (a >= W - R) return R + q + (a - (W - R));
  return R + mod_period(a, q);
}

// Device view of one operator's stencil table: coef[cls * noff + o].
template <typename T> struct StencilView {
  const c2<T>* coef;   // [ncls * noff]
  const c2<T>* wdinv;  // [ncls] omega / diag (only for smoothing operators), may be null
  GridDesc g;
  int off[kMaxOff];    // linear index offset of box point o
  int dx[kMaxOff][3];  // per-axis offset of box point o
  // Heterogeneous wavenumber (k per element): the operator is the class stencil plus a per-DoF
  // row, hrow[p * noff + o], in the same box layout (the k-dependent part -M_k - i B_k; null for
  // constant k). hwd[p] then replaces the class table's omega / diag.
  const c2<T>* hrow;
  const c2<T>* hwd;
};

// Prolongation (canonical interpolation V_2h -> V_h) as per-class weights.
// Fine index a on an axis: class a mod pf (pf = 2q), coarse anchor (a / pf) * q;
// weights w[cls][o] to coarse points anchor + box offset o in {0..q}^dim.
template <typename T> struct TransferView {
  const T* w;          // [npc * npo]
  GridDesc fine, coarse;
  int pf;              // 2q
  int npc, npo;        // (2q)^dim classes, (q+1)^dim offsets
  int po[kMaxPO][3];   // per-axis offsets of box point o
};

// Coarse vectors are stored block-padded: block J (grid line / line pair /
// plane) occupies [J*ldb, J*ldb + B), in-block index = lexicographic within
// the block. nb blocks; fake padding rows of the last block are identity rows.
struct CoarseLayout {
  int nb;       // number of blocks
  int B;        // DoFs per block (rows per block * W^(dim-1))
  int ldb;      // padded row length / block stride of vectors (even, >= B)
  int rows;     // lattice rows (or planes) per block = q
  int plane;    // W^(dim-1)
  int mid;      // middle block: top chain 0..mid-1 and bottom chain nb-1..mid+1 meet here
                // (twisted elimination); mid = nb-1 means a single top-down chain
  // Block maps of the coarse factor (device arrays of nb ints; null = identity). Where a
  // chain's Schur inverse converged during the factorisation, every later block of that chain
  // has the same inverse and the same couplings, and the segment products of whole segments
  // inside that range repeat: cmap[J] names the block whose Dinv, Lm and Up block J uses,
  // pmapf[J] / pmapb[J] the block whose forward / backward segment product it uses. The
  // repeated blocks are then read from one place (L2) and computed once.
  const int* cmap = nullptr;
  const int* pmapf = nullptr;
  const int* pmapb = nullptr;
  // Grouped block products (device arrays of kGroupInts ints per group: matrix block, count g,
  // kGroup source blocks, kGroup destination blocks). Vectors that use the same matrix block
  // (under the maps above) share a group of at most gcap, so the block is read once for all
  // of them. ggemv: the pre-pass p_J = Dinv[J] r_J; gfixf / gfixb: the fix-up products of the
  // forward / backward segmented sweeps. gcap = 0: no groups (blocks too wide to stage).
  const int* ggemv = nullptr;
  const int* gfixf = nullptr;
  const int* gfixb = nullptr;
  int ngemv = 0, nfixf = 0, nfixb = 0;
  int gcap = 0;
  int grows = 0;   // matrix rows per CTA (slab) of the grouped products
};
constexpr int kGroup = 4;
constexpr int kGroupInts = 2 + 2 * kGroup;
__host__ __device__ inline int map_block(const int* map, int J) {
#if defined(__CUDA_ARCH__)
  return map ? __ldg(map + J) : J;
#else
  return map ? map[J] : J;
#endif
}

#if defined(__CUDACC__)
// Index of coarse lattice point A (per-axis coordinates) in the block-padded coarse vector.
__device__ __forceinline__ int coarse_pad_index(const GridDesc& gc, const CoarseLayout& L, const int* A) {
  int last = gc.dim - 1;
  int J = A[last] / L.rows;
  int i = (A[last] - J * L.rows) * L.plane;
  int mul = 1;
  for (int ax = 0; ax < last; ++ax) {
    i += A[ax] * mul;
    mul *= gc.W;
  }
  return J * L.ldb + i;
}

// ----------------------------------------------------------------------------
// Bounded software grid barrier for cooperative launches.
// state[0] = arrival counter, state[kBarGen] = generation, on separate 128-byte
// lines (a barrier instance owns kBarWords words). Thread 0 of each CTA arrives
// after the CTA barrier that closes the phase and polls the generation (with a
// short back-off); the closing CTA barrier releases the other threads. On timeout
// the kernel's error word gets HELM_ETIMEOUT and the barrier returns false.
// ----------------------------------------------------------------------------
constexpr int kBarGen = 32;     // words: the generation sits 128 bytes after the counter
constexpr int kBarWords = 64;   // words per barrier instance
__device__ inline bool grid_barrier(unsigned* state, int* err, unsigned nblocks) {
  __shared__ int bar_ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = state + kBarGen;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(state, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(state, 0u);
      __threadfence();
      atomicAdd(state + kBarGen, 1u);
    } else {
      for (long long spins = 0; *vgen == gen;) {
        if (++spins > (1ll << 22)) {
          atomicCAS(err, 0, HELM_ETIMEOUT);
          ok = 0;
          break;
        }
        if (*(volatile int*)err != 0) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    bar_ok_s = ok;
  }
  __syncthreads();
  return bar_ok_s != 0;
}
#endif

// ----------------------------------------------------------------------------
// Host-side tables (computed in tables.cpp from element matrices).
// ----------------------------------------------------------------------------
struct HostTables {
  GridDesc fine, coarse;
  int ncls_f, ncls_c;
  // real stencils (K, M, B) per class, unit coefficients, for the fine and coarse level
  std::vector<double> Kf, Mf, Bf, Kc, Mc, Bc;   // [ncls * noff]
  // prolongation weights
  int pf, npc, npo;
  std::vector<double> pw;                         // [npc * npo]
};

// elements: HELM_SIMPLICES (P_order on triangles / Kuhn tetrahedra) or HELM_TENSOR (Q_order)
int build_tables(int dim, int order, int n, HostTables* t, int elements = HELM_SIMPLICES);
int host_stencil_row(const HostTables& t, int level, int64_t dof, double* K, double* M, double* B);

// Heterogeneous wavenumber (Sec. 2 with k in L^inf; Sec. 6, k(x) = k_max mu(x)): per-DoF rows
// (box offsets, as in the class tables) of K, M_k = sum_e k_e^2 M_e, M and B_k = sum_F k_F B_F
// on the full lattice of one level, from one wavenumber per element in the element order of the
// setup's iteration (cells x fastest, then the simplices of a cell); a boundary facet takes its
// element's value.
struct HetRows {
  GridDesc g;
  std::vector<double> K, Mk, M, Bk;   // [N * noff]
};
int64_t num_elements(int dim, int n, int elements);
int build_het_rows(int dim, int order, int n, int elements, const double* k_elem, HetRows* out);
int host_prolongation_row(const HostTables& t, int64_t fine_dof, int64_t* cols, double* w, int* count);
void rhs_planewave(int dim, int order, int n, double k, double theta, double2* F, int elements = HELM_SIMPLICES);
void rhs_gaussian(int dim, int order, int n, double sigma, const double* c, double2* F,
                  int elements = HELM_SIMPLICES);

}  // namespace helm
