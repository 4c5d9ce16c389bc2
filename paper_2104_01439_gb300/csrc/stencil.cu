// Fine-level matrix-free kernels of the twogrid V-cycle (Sec. 4, Algorithm 1;
// Sec. 6: K and M applied on the fly, "semi matrix-free").
//
// Every DoF reads its class (from its lattice position) and applies the
// class's (2R+1)^dim-point complex stencil. Neighbour indices are clamped into
// the vector, which is safe because a class's coefficient is exactly zero for
// every box point outside the domain. One thread per DoF, grid-stride, with
// the class tables staged in shared memory; the box size is a template
// parameter so the offset loop is fully unrolled.
#include <algorithm>

#include "dfloat.cuh"
#include "kernels.cuh"

namespace helm {
namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n, int per_block = kThreads) {
  int64_t b = (n + per_block - 1) / per_block;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16);
}

// lattice coordinates and class of DoF p (the last coordinate is what remains after the
// divisions of the others: no division for it)
__device__ __forceinline__ int decode(const GridDesc& g, int p, int* a) {
  int cls = 0, mul = 1, t = p;
  for (int ax = 0; ax < g.dim; ++ax) {
    if (ax == g.dim - 1) {
      a[ax] = t;
    } else {
      const int q = t / g.W;
      a[ax] = t - q * g.W;
      t = q;
    }
    cls += axis_class(a[ax], g.W, g.R, g.q) * mul;
    mul *= g.C1;
  }
  return cls;
}

__device__ __forceinline__ int class_of(const GridDesc& g, const int* a) {
  int cls = 0, mul = 1;
  for (int ax = 0; ax < g.dim; ++ax) {
    cls += axis_class(a[ax], g.W, g.R, g.q) * mul;
    mul *= g.C1;
  }
  return cls;
}

template <typename T>
__device__ __forceinline__ void stage_tables(const StencilView<T>& s, c2<T>* coef_s, c2<T>* dinv_s,
                                             int ncls) {
  int nc = ncls * s.g.noff;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) coef_s[i] = s.coef[i];
  if (dinv_s)
    for (int i = threadIdx.x; i < ncls; i += blockDim.x) dinv_s[i] = s.wdinv[i];
  __syncthreads();
}

__device__ __forceinline__ int ncls_of(const GridDesc& g) {
  int n = 1;
  for (int ax = 0; ax < g.dim; ++ax) n *= g.C1;
  return n;
}

// (A x)(p) with x read through conversion to precision T. In complex128 (FP64 issues at
// 1/58 of the FP32 rate on this GPU) a class whose coefficients are all real (every
// interior class of A0 = K - k^2 M; `real` is a per-class flag formed when the table is
// staged) takes real-by-complex products: 2 instead of 4 FP64 multiply-adds per offset.
template <int NOFF, typename T, typename Vin>
__device__ __forceinline__ c2<T> row_apply(const StencilView<T>& s, const c2<T>* c, int p, int N,
                                           const Vin* __restrict__ x, bool real = false) {
  c2<T> acc = mk(T(0), T(0));
  if (real) {
    c2<T> xv[NOFF];
#pragma unroll
    for (int o = 0; o < NOFF; ++o) xv[o] = to<c2<T>>(x[min(max(p + s.off[o], 0), N - 1)]);
#pragma unroll
    for (int o = 0; o < NOFF; ++o) {
      acc.x = fma(c[o].x, xv[o].x, acc.x);
      acc.y = fma(c[o].x, xv[o].y, acc.y);
    }
    return acc;
  }
#pragma unroll
  for (int o = 0; o < NOFF; ++o) {
    int q = min(max(p + s.off[o], 0), N - 1);
    acc = cfma(c[o], to<c2<T>>(x[q]), acc);
  }
  return acc;
}
// the per-DoF part of a heterogeneous-wavenumber operator, added to a class-stencil row
template <int NOFF, typename T, typename Vin>
__device__ __forceinline__ c2<T> het_apply(const StencilView<T>& s, int p, int N, const Vin* __restrict__ x,
                                           c2<T> acc) {
  const c2<T>* h = s.hrow + (int64_t)p * NOFF;
#pragma unroll
  for (int o = 0; o < NOFF; ++o) acc = cfma(h[o], to<c2<T>>(x[min(max(p + s.off[o], 0), N - 1)]), acc);
  return acc;
}

// the product's double-float split (hi + lo), read by the Gram-Schmidt inner products
__device__ __forceinline__ void store_split(float4* ws, int p, double2 v) { ws[p] = dfc_from(v); }
__device__ __forceinline__ void store_split(float4*, int, float2) {}

template <int NOFF, typename T, typename Vin, typename Vout>
__global__ void __launch_bounds__(kThreads) k_apply(StencilView<T> s, VecSel<const Vin> xs,
                                                     VecSel<Vout> ys, float4* __restrict__ ws,
                                                     const int* active) {
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char sm[];
  c2<T>* coef = reinterpret_cast<c2<T>*>(sm);
  __shared__ int real_cls[kMaxCls];
  int ncls = ncls_of(s.g);
  if (sizeof(T) == sizeof(double) && threadIdx.x < ncls) {
    bool r = true;
    for (int o = 0; o < NOFF; ++o) r = r && s.coef[threadIdx.x * NOFF + o].y == T(0);
    real_cls[threadIdx.x] = r ? 1 : 0;
  }
  stage_tables(s, coef, (c2<T>*)nullptr, ncls);   // (ends with a block barrier)
  const Vin* x = xs.ptr();
  Vout* y = ys.base ? ys.ptr() : nullptr;
  const int N = (int)s.g.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    int a[3];
    int cls = decode(s.g, p, a);
    const bool real = sizeof(T) == sizeof(double) && real_cls[cls] != 0;
    c2<T> v = row_apply<NOFF>(s, coef + cls * NOFF, p, N, x, real);
    if (s.hrow) v = het_apply<NOFF>(s, p, N, x, v);
    if (y) y[p] = to<Vout>(v);
    if (ws) store_split(ws, p, v);
  }
}

// ws = A x in double-float: complex64 x (exact), complex128 coefficients split into
// double-float pairs once per CTA; a real class takes two products per offset.
template <int NOFF>
__global__ void __launch_bounds__(kThreads) k_apply_df(StencilView<double> s, VecSel<const float2> xs,
                                                        float4* __restrict__ ws, const int* active) {
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char sm[];
  float4* coef = reinterpret_cast<float4*>(sm);
  __shared__ int real_cls[kMaxCls];
  const int ncls = ncls_of(s.g);
  for (int i = threadIdx.x; i < ncls * NOFF; i += blockDim.x) coef[i] = dfc_from(s.coef[i]);
  if (threadIdx.x < ncls) {
    bool r = true;
    for (int o = 0; o < NOFF; ++o) r = r && s.coef[threadIdx.x * NOFF + o].y == 0.0;
    real_cls[threadIdx.x] = r ? 1 : 0;
  }
  __syncthreads();
  const float2* x = xs.ptr();
  const int N = (int)s.g.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    int a[3];
    const int cls = decode(s.g, p, a);
    const float4* c = coef + cls * NOFF;
    float2 xv[NOFF];
#pragma unroll
    for (int o = 0; o < NOFF; ++o) xv[o] = x[min(max(p + s.off[o], 0), N - 1)];
    DFC_ACC acc{DF{0.f, 0.f}, DF{0.f, 0.f}};
    if (real_cls[cls]) {
#pragma unroll
      for (int o = 0; o < NOFF; ++o) {
        df_mac(c[o].x, c[o].z, xv[o].x, 0.f, acc.re);
        df_mac(c[o].x, c[o].z, xv[o].y, 0.f, acc.im);
      }
    } else {
#pragma unroll
      for (int o = 0; o < NOFF; ++o) {
        // c x = (cr xr - ci xi) + i (cr xi + ci xr)
        df_mac(c[o].x, c[o].z, xv[o].x, 0.f, acc.re);
        df_mac(-c[o].y, -c[o].w, xv[o].y, 0.f, acc.re);
        df_mac(c[o].x, c[o].z, xv[o].y, 0.f, acc.im);
        df_mac(c[o].y, c[o].w, xv[o].x, 0.f, acc.im);
      }
    }
    if (s.hrow) {   // heterogeneous wavenumber: the DoF's own row, split into double-float pairs
      const double2* hr = s.hrow + (int64_t)p * NOFF;
#pragma unroll
      for (int o = 0; o < NOFF; ++o) {
        const float4 h = dfc_from(hr[o]);
        df_mac(h.x, h.z, xv[o].x, 0.f, acc.re);
        df_mac(-h.y, -h.w, xv[o].y, 0.f, acc.re);
        df_mac(h.x, h.z, xv[o].y, 0.f, acc.im);
        df_mac(h.y, h.w, xv[o].x, 0.f, acc.im);
      }
    }
    ws[p] = dfc_fin(acc);
  }
}

template <int NOFF, typename T, typename Vf, typename Vr>
__global__ void __launch_bounds__(kThreads) k_residual(StencilView<T> s, VecSel<const Vf> fs,
                                                        const c2<T>* __restrict__ u,
                                                        Vr* __restrict__ r, const int* active) {
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char sm[];
  c2<T>* coef = reinterpret_cast<c2<T>*>(sm);
  int ncls = ncls_of(s.g);
  stage_tables(s, coef, (c2<T>*)nullptr, ncls);
  const Vf* f = fs.ptr();
  const int N = (int)s.g.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    int a[3];
    int cls = decode(s.g, p, a);
    c2<T> Au = row_apply<NOFF>(s, coef + cls * NOFF, p, N, u);
    if (s.hrow) Au = het_apply<NOFF>(s, p, N, u, Au);
    r[p] = to<Vr>(csub(to<c2<T>>(f[p]), Au));
  }
}

// First smoothing steps from u^0 = 0: u^1 = w D^-1 f, u^2 = u^1 + w D^-1 (f - A u^1),
// with u^1 at the neighbours recomputed from f (no u^1 pass through memory).
template <int NOFF, typename T, typename Vf>
__global__ void __launch_bounds__(kThreads) k_jacobi0(StencilView<T> s, VecSel<const Vf> fs,
                                                       c2<T>* __restrict__ uout,
                                                       c2<T>* __restrict__ fcopy, int two,
                                                       const int* active) {
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char sm[];
  c2<T>* coef = reinterpret_cast<c2<T>*>(sm);
  int ncls = ncls_of(s.g);
  c2<T>* dinv = coef + ncls * NOFF;
  stage_tables(s, coef, dinv, ncls);
  const Vf* f = fs.ptr();
  const int N = (int)s.g.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    int a[3];
    int cls = decode(s.g, p, a);
    c2<T> fp = to<c2<T>>(f[p]);
    if (fcopy) fcopy[p] = fp;
    const c2<T> dp = s.hwd ? s.hwd[p] : dinv[cls];
    c2<T> u1 = cmul(dp, fp);
    if (!two) {
      uout[p] = u1;
      continue;
    }
    c2<T> Au = mk(T(0), T(0));
    const c2<T>* c = coef + cls * NOFF;
#pragma unroll
    for (int o = 0; o < NOFF; ++o) {
      int na[3];
      for (int ax = 0; ax < 3; ++ax) na[ax] = ax < s.g.dim ? min(max(a[ax] + s.dx[o][ax], 0), s.g.W - 1) : 0;
      int q = min(max(p + s.off[o], 0), N - 1);
      c2<T> uq = cmul(s.hwd ? s.hwd[q] : dinv[class_of(s.g, na)], to<c2<T>>(f[q]));
      Au = cfma(c[o], uq, Au);
      if (s.hrow) Au = cfma(s.hrow[(int64_t)p * NOFF + o], uq, Au);
    }
    uout[p] = cfma(dp, csub(fp, Au), u1);
  }
}

template <int NOFF, typename T, typename Vf, typename Vout>
__global__ void __launch_bounds__(kThreads) k_jacobi(StencilView<T> s, VecSel<const Vf> fs,
                                                      const c2<T>* __restrict__ u,
                                                      VecSel<Vout> outs, const int* active) {
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char sm[];
  c2<T>* coef = reinterpret_cast<c2<T>*>(sm);
  int ncls = ncls_of(s.g);
  c2<T>* dinv = coef + ncls * NOFF;
  stage_tables(s, coef, dinv, ncls);
  const Vf* f = fs.ptr();
  Vout* out = outs.ptr();
  const int N = (int)s.g.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    int a[3];
    int cls = decode(s.g, p, a);
    c2<T> Au = row_apply<NOFF>(s, coef + cls * NOFF, p, N, u);
    if (s.hrow) Au = het_apply<NOFF>(s, p, N, u, Au);
    out[p] = to<Vout>(cfma(s.hwd ? s.hwd[p] : dinv[cls], csub(to<c2<T>>(f[p]), Au), u[p]));
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_prolong_add(TransferView<T> P, CoarseLayout L,
                                                           const c2<T>* __restrict__ uc,
                                                           c2<T>* __restrict__ u, const int* active) {
  if (active && *active == 0) return;
  const int N = (int)P.fine.N;
  const int q = P.coarse.q;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    int a[3];
    decode(P.fine, p, a);
    int cls = 0, mul = 1, anc[3];
    for (int ax = 0; ax < P.fine.dim; ++ax) {
      cls += mod_period(a[ax], P.pf) * mul;
      mul *= P.pf;
      anc[ax] = div_period(a[ax], P.pf) * q;
    }
    c2<T> acc = mk(T(0), T(0));
    for (int o = 0; o < P.npo; ++o) {
      T w = P.w[cls * P.npo + o];
      if (w == T(0)) continue;
      int A[3];
      for (int ax = 0; ax < P.fine.dim; ++ax) A[ax] = anc[ax] + P.po[o][ax];
      c2<T> v = uc[coarse_pad_index(P.coarse, L, A)];
      acc.x = fma(w, v.x, acc.x);
      acc.y = fma(w, v.y, acc.y);
    }
    u[p] = cadd(u[p], acc);
  }
}

// rc(A) = sum over fine DoFs a of P[a][A] r(a)  (the transpose of the interpolation)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_restrict(TransferView<T> P, CoarseLayout L,
                                                        const c2<T>* __restrict__ r,
                                                        c2<T>* __restrict__ rc, const int* active) {
  if (active && *active == 0) return;
  const int total = L.nb * L.ldb;
  const int q = P.coarse.q, pf = P.pf, d = P.fine.dim, Wf = P.fine.W;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int J = idx / L.ldb, i = idx - J * L.ldb;
    int A[3] = {0, 0, 0};
    bool valid = i < L.B;
    if (valid) {
      int t = i % L.plane, row = i / L.plane;
      for (int ax = 0; ax < d - 1; ++ax) {
        A[ax] = t % P.coarse.W;
        t /= P.coarse.W;
      }
      A[d - 1] = J * L.rows + row;
      valid = A[d - 1] < P.coarse.W;
    }
    c2<T> acc = mk(T(0), T(0));
    if (valid) {
      int lo[3], hi[3];
      for (int ax = 0; ax < 3; ++ax) {
        if (ax < d) {
          int cmin = div_period(A[ax] + q - 1, q) - 1;   // ceil((A-q)/q) for A >= 0
          lo[ax] = max(0, pf * cmin);
          hi[ax] = min(Wf - 1, pf * div_period(A[ax], q) + pf - 1);
        } else {
          lo[ax] = hi[ax] = 0;
        }
      }
      for (int a2 = lo[2]; a2 <= hi[2]; ++a2)
        for (int a1 = lo[1]; a1 <= hi[1]; ++a1)
          for (int a0 = lo[0]; a0 <= hi[0]; ++a0) {
            int a[3] = {a0, a1, a2};
            int cls = 0, mul = 1, o = 0, omul = 1;
            bool ok = true;
            for (int ax = 0; ax < d; ++ax) {
              cls += mod_period(a[ax], pf) * mul;
              mul *= pf;
              int oo = A[ax] - div_period(a[ax], pf) * q;
              ok &= (oo >= 0 && oo <= q);
              o += oo * omul;
              omul *= q + 1;
            }
            if (!ok) continue;
            T w = P.w[cls * P.npo + o];
            if (w == T(0)) continue;
            int fp = a0 + Wf * (a1 + Wf * a2);
            c2<T> v = r[fp];
            acc.x = fma(w, v.x, acc.x);
            acc.y = fma(w, v.y, acc.y);
          }
    }
    rc[idx] = acc;
  }
}

template <typename Vin, typename Vout>
__global__ void k_coarse_pack(GridDesc gc, CoarseLayout L, const Vin* nat, Vout* pad) {
  const int total = L.nb * L.ldb;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int J = idx / L.ldb, i = idx - J * L.ldb;
    Vout v = to<Vout>(mk(0.0, 0.0));
    if (i < L.B) {
      int row = J * L.rows + i / L.plane;
      if (row < gc.W) v = to<Vout>(nat[(int64_t)row * L.plane + i % L.plane]);
    }
    pad[idx] = v;
  }
}

template <typename Vin, typename Vout>
__global__ void k_coarse_unpack(GridDesc gc, CoarseLayout L, const Vin* pad, Vout* nat) {
  const int N = (int)gc.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    int row = p / L.plane, in = p % L.plane;
    int J = row / L.rows;
    nat[p] = to<Vout>(pad[J * L.ldb + (row - J * L.rows) * L.plane + in]);
  }
}

template <typename T>
size_t table_smem(const GridDesc& g, bool with_dinv) {
  int ncls = 1;
  for (int ax = 0; ax < g.dim; ++ax) ncls *= g.C1;
  return sizeof(c2<T>) * (size_t)(ncls * g.noff + (with_dinv ? ncls : 0));
}

}  // namespace

#define HELM_SWITCH_NOFF(noff, CALL9, CALL25, CALL27, CALL49) \
  switch (noff) {                                              \
    case 9: CALL9; break;                                      \
    case 25: CALL25; break;                                    \
    case 27: CALL27; break;                                    \
    case 49: CALL49; break;                                    \
    default: break;                                            \
  }

template <typename T, typename Vin, typename Vout>
void launch_apply(const StencilView<T>& A, VecSel<const Vin> x, VecSel<Vout> y, const int* active,
                  cudaStream_t s, float4* ws) {
  int g = grid_for(A.g.N);
  size_t sm = table_smem<T>(A.g, false);
  HELM_SWITCH_NOFF(A.g.noff, (k_apply<9, T, Vin, Vout><<<g, kThreads, sm, s>>>(A, x, y, ws, active)),
                   (k_apply<25, T, Vin, Vout><<<g, kThreads, sm, s>>>(A, x, y, ws, active)),
                   (k_apply<27, T, Vin, Vout><<<g, kThreads, sm, s>>>(A, x, y, ws, active)),
                   (k_apply<49, T, Vin, Vout><<<g, kThreads, sm, s>>>(A, x, y, ws, active)));
}

void launch_apply_df(const StencilView<double>& A, VecSel<const float2> x, float4* ws, const int* active,
                     cudaStream_t s) {
  int g = grid_for(A.g.N);
  size_t sm = table_smem<double>(A.g, false);   // 16 bytes per coefficient either way
  HELM_SWITCH_NOFF(A.g.noff, (k_apply_df<9><<<g, kThreads, sm, s>>>(A, x, ws, active)),
                   (k_apply_df<25><<<g, kThreads, sm, s>>>(A, x, ws, active)),
                   (k_apply_df<27><<<g, kThreads, sm, s>>>(A, x, ws, active)),
                   (k_apply_df<49><<<g, kThreads, sm, s>>>(A, x, ws, active)));
}

template <typename T, typename Vf, typename Vr>
void launch_residual(const StencilView<T>& A, VecSel<const Vf> f, const c2<T>* u, Vr* r,
                     const int* active, cudaStream_t s) {
  int g = grid_for(A.g.N);
  size_t sm = table_smem<T>(A.g, false);
  HELM_SWITCH_NOFF(A.g.noff, (k_residual<9, T, Vf, Vr><<<g, kThreads, sm, s>>>(A, f, u, r, active)),
                   (k_residual<25, T, Vf, Vr><<<g, kThreads, sm, s>>>(A, f, u, r, active)),
                   (k_residual<27, T, Vf, Vr><<<g, kThreads, sm, s>>>(A, f, u, r, active)),
                   (k_residual<49, T, Vf, Vr><<<g, kThreads, sm, s>>>(A, f, u, r, active)));
}

template <typename T, typename Vf>
void launch_jacobi_from_zero(const StencilView<T>& A, VecSel<const Vf> f, c2<T>* u_out, c2<T>* fcopy,
                             bool two_steps, const int* active, cudaStream_t s) {
  int g = grid_for(A.g.N);
  size_t sm = table_smem<T>(A.g, true);
  int two = two_steps ? 1 : 0;
  HELM_SWITCH_NOFF(A.g.noff, (k_jacobi0<9, T, Vf><<<g, kThreads, sm, s>>>(A, f, u_out, fcopy, two, active)),
                   (k_jacobi0<25, T, Vf><<<g, kThreads, sm, s>>>(A, f, u_out, fcopy, two, active)),
                   (k_jacobi0<27, T, Vf><<<g, kThreads, sm, s>>>(A, f, u_out, fcopy, two, active)),
                   (k_jacobi0<49, T, Vf><<<g, kThreads, sm, s>>>(A, f, u_out, fcopy, two, active)));
}

template <typename T, typename Vf, typename Vout>
void launch_jacobi(const StencilView<T>& A, VecSel<const Vf> f, const c2<T>* u, VecSel<Vout> out,
                   const int* active, cudaStream_t s) {
  int g = grid_for(A.g.N);
  size_t sm = table_smem<T>(A.g, true);
  HELM_SWITCH_NOFF(A.g.noff, (k_jacobi<9, T, Vf, Vout><<<g, kThreads, sm, s>>>(A, f, u, out, active)),
                   (k_jacobi<25, T, Vf, Vout><<<g, kThreads, sm, s>>>(A, f, u, out, active)),
                   (k_jacobi<27, T, Vf, Vout><<<g, kThreads, sm, s>>>(A, f, u, out, active)),
                   (k_jacobi<49, T, Vf, Vout><<<g, kThreads, sm, s>>>(A, f, u, out, active)));
}

template <typename T>
void launch_prolong_add(const TransferView<T>& P, const CoarseLayout& L, const c2<T>* uc, c2<T>* u,
                        const int* active, cudaStream_t s) {
  k_prolong_add<T><<<grid_for(P.fine.N), kThreads, 0, s>>>(P, L, uc, u, active);
}

template <typename T>
void launch_restrict(const TransferView<T>& P, const CoarseLayout& L, const c2<T>* r, c2<T>* rc,
                     const int* active, cudaStream_t s) {
  k_restrict<T><<<grid_for((int64_t)L.nb * L.ldb), kThreads, 0, s>>>(P, L, r, rc, active);
}

template <typename Vin, typename Vout>
void launch_coarse_pack(const GridDesc& gc, const CoarseLayout& L, const Vin* nat, Vout* pad,
                        cudaStream_t s) {
  k_coarse_pack<Vin, Vout><<<grid_for((int64_t)L.nb * L.ldb), kThreads, 0, s>>>(gc, L, nat, pad);
}
template <typename Vin, typename Vout>
void launch_coarse_unpack(const GridDesc& gc, const CoarseLayout& L, const Vin* pad, Vout* nat,
                          cudaStream_t s) {
  k_coarse_unpack<Vin, Vout><<<grid_for(gc.N), kThreads, 0, s>>>(gc, L, pad, nat);
}

// The 49-point (Q3) class tables exceed the default 48 KB of dynamic shared memory in
// complex128 (81 classes x 49 offsets x 16 B): raise the limit once, at setup (outside
// stream capture), for every instantiation that stages them.
void stencil_prepare() {
  const int lim = 100 * 1024;
  cudaFuncSetAttribute(k_apply<49, float, float2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_apply<49, double, double2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_apply_df<49>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_residual<49, float, float2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_residual<49, double, double2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi0<49, float, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi0<49, float, float4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi0<49, double, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi<49, float, float2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi<49, float, float2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi<49, double, double2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaGetLastError();
}

// ---- explicit instantiations -------------------------------------------------
// complex64 V-cycle (mixed precision): f = v_j (complex128) is read once and
// kept as complex64; the last post-smoothing sweep writes z_j in complex128.
template void launch_jacobi_from_zero<float, double2>(const StencilView<float>&, VecSel<const double2>,
                                                      float2*, float2*, bool, const int*, cudaStream_t);
template void launch_jacobi_from_zero<float, float4>(const StencilView<float>&, VecSel<const float4>,
                                                     float2*, float2*, bool, const int*, cudaStream_t);
template void launch_residual<float, float2, float2>(const StencilView<float>&, VecSel<const float2>,
                                                     const float2*, float2*, const int*, cudaStream_t);
template void launch_jacobi<float, float2, float2>(const StencilView<float>&, VecSel<const float2>,
                                                   const float2*, VecSel<float2>, const int*, cudaStream_t);
template void launch_jacobi<float, float2, double2>(const StencilView<float>&, VecSel<const float2>,
                                                    const float2*, VecSel<double2>, const int*, cudaStream_t);
template void launch_prolong_add<float>(const TransferView<float>&, const CoarseLayout&, const float2*,
                                        float2*, const int*, cudaStream_t);
template void launch_restrict<float>(const TransferView<float>&, const CoarseLayout&, const float2*,
                                     float2*, const int*, cudaStream_t);
template void launch_coarse_pack<double2, float2>(const GridDesc&, const CoarseLayout&, const double2*,
                                                  float2*, cudaStream_t);
template void launch_coarse_unpack<float2, double2>(const GridDesc&, const CoarseLayout&, const float2*,
                                                    double2*, cudaStream_t);
template void launch_apply<float, float2, float2>(const StencilView<float>&, VecSel<const float2>,
                                                  VecSel<float2>, const int*, cudaStream_t, float4*);
// complex128 everywhere
template void launch_jacobi_from_zero<double, double2>(const StencilView<double>&, VecSel<const double2>,
                                                       double2*, double2*, bool, const int*, cudaStream_t);
template void launch_residual<double, double2, double2>(const StencilView<double>&, VecSel<const double2>,
                                                        const double2*, double2*, const int*, cudaStream_t);
template void launch_jacobi<double, double2, double2>(const StencilView<double>&, VecSel<const double2>,
                                                      const double2*, VecSel<double2>, const int*,
                                                      cudaStream_t);
template void launch_prolong_add<double>(const TransferView<double>&, const CoarseLayout&, const double2*,
                                         double2*, const int*, cudaStream_t);
template void launch_restrict<double>(const TransferView<double>&, const CoarseLayout&, const double2*,
                                      double2*, const int*, cudaStream_t);
template void launch_coarse_pack<double2, double2>(const GridDesc&, const CoarseLayout&, const double2*,
                                                   double2*, cudaStream_t);
template void launch_coarse_unpack<double2, double2>(const GridDesc&, const CoarseLayout&, const double2*,
                                                     double2*, cudaStream_t);
template void launch_apply<double, double2, double2>(const StencilView<double>&, VecSel<const double2>,
                                                     VecSel<double2>, const int*, cudaStream_t, float4*);

}  // namespace helm
