// Fused damped-Jacobi smoothing on 2D tiles (Algorithm 1: the pre-smoothing, residual and
// post-smoothing lines of the twogrid cycle; Sec. 3 for the smoother).
//
// One CTA owns a TX x TY tile of the DoF lattice (TX = 64 - 2H) and stages the right-hand
// side f on the tile plus a halo of H points (64 columns) in shared memory. It then runs every sweep
//   u <- u + omega D^-1 (f - A u)
// in shared memory, each on a region one stencil reach R smaller than the previous one, so
// the tile's values after nu sweeps only depend on data the CTA loaded. Global memory sees
// f once, the start vector once (post-smoothing) and the results once, instead of every
// sweep's input and output. Work in the halo is repeated by the neighbouring tiles.
//   pre-smoothing, u^0 = 0:  u^1 = omega D^-1 f pointwise, then nu - 1 sweeps; optionally the
//                             residual f - A u^nu on the tile (for the restriction);
//   post-smoothing:          u^0 = u_pre + P u_c, gathered from the coarse correction at the
//                             staged points, then nu sweeps.
// Every point of the staged region takes its class (boundary position and lattice parity
// along each axis) from two per-axis arrays; points outside the domain hold zero, which is
// what the class stencils assume (their coefficients towards outside points are zero).
#include <algorithm>
#include <type_traits>

#include "kernels.cuh"

namespace helm {
namespace {

constexpr int kTileThreads = 256;

// Packed FP32 pairs (f32x2 instructions: one instruction for the two lanes of a float2).
__device__ __forceinline__ unsigned long long u64(float2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ float2 f2(unsigned long long a) { return *reinterpret_cast<float2*>(&a); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {   // a * b + c, per lane
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(u64(a)), "l"(u64(b)), "l"(u64(c)));
  return f2(d);
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u64(a)), "l"(u64(b)));
  return f2(d);
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u64(a)), "l"(u64(b)));
  return f2(d);
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u64(a)), "l"(u64(b)));
  return f2(d);
}
// complex128 <-> complex64 on the integer pipes. This GPU runs conversions between double and
// float on its FP64 unit (1/64 of the FP32 rate), which would bound the complex128 entry points;
// these take the IEEE bit fields apart instead. double -> float rounds to nearest (ties away
// from zero, which differs from the hardware's ties-to-even only on exact ties); zeros and
// values outside float's normal range take the hardware conversion.
__device__ __forceinline__ float d2f_bits(double d) {
  const int hi = __double2hiint(d), lo = __double2loint(d);
  const int e = (hi >> 20) & 0x7ff;
  if (e < 1023 - 126 || e > 1023 + 127) return (float)d;   // zero, subnormal or outside float's range
  unsigned f = (unsigned)(hi & 0x80000000) | ((unsigned)(e - 1023 + 127) << 23) | ((unsigned)(hi & 0xfffff) << 3) |
               ((unsigned)lo >> 29);
  f += ((unsigned)lo >> 28) & 1u;   // round: a carry out of the mantissa moves into the exponent
  return __uint_as_float(f);
}
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xff;
  if (e == 0 || e == 0xff) return (double)x;   // zero, subnormal, inf, NaN
  const unsigned m = b & 0x7fffff;
  return __hiloint2double((int)((b & 0x80000000u) | ((e - 127 + 1023) << 20) | (m >> 3)), (int)(m << 29));
}
__device__ __forceinline__ float2 stage_in(double2 v) { return make_float2(d2f_bits(v.x), d2f_bits(v.y)); }
__device__ __forceinline__ float2 stage_in(float4 v) { return make_float2(v.x, v.y); }   // a double-float's high parts
__device__ __forceinline__ float2 stage_in(float2 v) { return v; }
template <typename V, typename Vf> __device__ __forceinline__ V stage(Vf v) {
  if constexpr (sizeof(V) == sizeof(float2)) return stage_in(v);
  else return to<V>(v);
}
template <typename Vout, typename V> __device__ __forceinline__ Vout unstage(V v) {
  if constexpr (sizeof(Vout) == sizeof(double2) && sizeof(V) == sizeof(float2))
    return make_double2(f2d_bits(v.x), f2d_bits(v.y));
  else return to<Vout>(v);
}

// u + d (f - Au), the damped-Jacobi update of one point (d = omega / diag)
__device__ __forceinline__ float2 jacobi_step(float2 d, float2 f, float2 Au, float2 u) {
  const float2 t = fsub2(f, Au);
  const float2 a = ffma2(make_float2(d.x, d.x), t, u), b = fmul2(make_float2(d.y, d.y), t);
  return make_float2(a.x - b.y, a.y + b.x);
}
__device__ __forceinline__ double2 jacobi_step(double2 d, double2 f, double2 Au, double2 u) {
  return cfma(d, csub(f, Au), u);
}
// Interior 9-point stencil of a complex-symmetric operator, c(o) = c(-o): the centre and four
// offset pairs (x, y, diagonal, antidiagonal), each coefficient as (re, re) and (im, im) pairs
// so that sum c_o u_o = sum (re ⊙ s) + i sum (im ⊙ s) takes two packed FMAs per pair sum s.
struct Sym9 {
  float2 rr[5], ii[5];
};
// box index of the first offset of each pair (dx, dy in -1..1, o = (dx + 1) + 3 (dy + 1))
__host__ __device__ constexpr int sym9_first(int k) { return k == 0 ? 4 : k == 1 ? 5 : k == 2 ? 7 : k == 3 ? 8 : 2; }
// (A u) at the centre of a 3 x 3 window w[dy][dx]
__device__ __forceinline__ float2 sym9_apply(const Sym9& c, const float2 (&w)[3][3]) {
  const float2 sx = fadd2(w[1][2], w[1][0]), sy = fadd2(w[2][1], w[0][1]);
  const float2 sd = fadd2(w[2][2], w[0][0]), sa = fadd2(w[0][2], w[2][0]);
  float2 a = fmul2(c.rr[0], w[1][1]), b = fmul2(c.ii[0], w[1][1]);
  a = ffma2(c.rr[1], sx, a);
  b = ffma2(c.ii[1], sx, b);
  a = ffma2(c.rr[2], sy, a);
  b = ffma2(c.ii[2], sy, b);
  a = ffma2(c.rr[3], sd, a);
  b = ffma2(c.ii[3], sd, b);
  a = ffma2(c.rr[4], sa, a);
  b = ffma2(c.ii[4], sa, b);
  return make_float2(a.x - b.y, a.y + b.x);
}
constexpr int kRegionX = 64;   // staged columns per tile: two warp widths (the tile is 64 - 2H wide)
constexpr int kLoadRows = 10;  // staged rows per warp: RY = TY + 2H <= 8 * kLoadRows (TY <= 32, H <= 24)

// rows of the vertical strip one thread computes in a sweep (register blocking)
template <int R, typename T> struct Strip {
  static constexpr int VS = R >= 3 ? 1 : sizeof(T) == 8 ? (R == 1 ? 2 : 1) : (R == 1 ? 4 : 2);
};

// One sweep region of the tile: rows [m, RY - m), columns [m, kRegionX - m) of the staged
// region; lane l takes columns l and l + 32, warps take strips of VS rows. For every point:
// (A u)(p) from the (VS + 2R) x (2R + 1) window of u around the strip, then emit(p, Au).
// FAST: every staged point has the same class (interior of a period-1 lattice), whose
// coefficients the caller holds in registers (creg, indexed by compile-time offsets only);
// otherwise each point's class comes from the per-axis arrays and its stencil from shared
// memory, and points outside the domain are emitted with class -1.
template <int R, typename T, bool FAST, bool HET, typename Emit>
__device__ __forceinline__ void sweep_region(const c2<T>* __restrict__ u, int RY, int m, const int* cx, const int* cy,
                                             const c2<T>* coef, const c2<T> (&creg)[(2 * R + 1) * (2 * R + 1)],
                                             const Sym9& sym, const c2<T>* __restrict__ hrow, int gx0, int gy0,
                                             int W, Emit emit) {
  using V = c2<T>;
  constexpr int SIDE = 2 * R + 1, NO = SIDE * SIDE, VS = Strip<R, T>::VS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rows = RY - 2 * m;
  const int nstrips = (rows + VS - 1) / VS;
  for (int st = warp; st < nstrips; st += nw) {
    const int ly0 = m + st * VS;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int lx = lane + 32 * half;
      if (lx < m || lx >= kRegionX - m) continue;
      const int cxv = FAST ? 0 : cx[lx];
      // the window: rows ly0 - R .. ly0 + VS - 1 + R (clipped to the region), columns lx - R .. lx + R
      if constexpr (FAST && R == 1 && sizeof(T) == 4) {
        float2 w[VS + 2][3];
#pragma unroll
        for (int r = 0; r < VS + 2; ++r) {
          const int ly = min(ly0 - 1 + r, RY - 1);
#pragma unroll
          for (int c = 0; c < 3; ++c) w[r][c] = u[ly * kRegionX + lx - 1 + c];
        }
#pragma unroll
        for (int v = 0; v < VS; ++v) {
          const int ly = ly0 + v;
          if (ly >= RY - m) break;
          const float2 (&wv)[3][3] = *reinterpret_cast<const float2(*)[3][3]>(&w[v][0]);
          emit(ly, lx, 0, sym9_apply(sym, wv), w[v + 1][1]);
        }
        continue;
      }
      V win[VS + 2 * R][SIDE];
#pragma unroll
      for (int r = 0; r < VS + 2 * R; ++r) {
        const int ly = min(ly0 - R + r, RY - 1);
#pragma unroll
        for (int c = 0; c < SIDE; ++c) win[r][c] = u[ly * kRegionX + lx - R + c];
      }
#pragma unroll
      for (int v = 0; v < VS; ++v) {
        const int ly = ly0 + v;
        if (ly >= RY - m) break;
        V acc = mk(T(0), T(0));
        if (FAST) {
#pragma unroll
          for (int dy = 0; dy < SIDE; ++dy)
#pragma unroll
            for (int dx = 0; dx < SIDE; ++dx) acc = cfma(creg[dy * SIDE + dx], win[v + dy][dx], acc);
          emit(ly, lx, 0, acc, win[v + R][R]);
        } else {
          const int cyv = cy[ly];
          if (cxv < 0 || cyv < 0) {
            emit(ly, lx, -1, acc, acc);
            continue;
          }
          const V* c = coef + (cxv + cyv) * NO;
#pragma unroll
          for (int dy = 0; dy < SIDE; ++dy)
#pragma unroll
            for (int dx = 0; dx < SIDE; ++dx) acc = cfma(c[dy * SIDE + dx], win[v + dy][dx], acc);
          if constexpr (HET) {   // heterogeneous wavenumber: the point's own row
            const V* hr = hrow + ((int64_t)(gy0 + ly) * W + gx0 + lx) * NO;
#pragma unroll
            for (int dy = 0; dy < SIDE; ++dy)
#pragma unroll
              for (int dx = 0; dx < SIDE; ++dx) acc = cfma(hr[dy * SIDE + dx], win[v + dy][dx], acc);
          }
          emit(ly, lx, cxv + cyv, acc, win[v + R][R]);
        }
      }
    }
  }
}

template <int R, typename T, typename Vf, typename Vout, bool HET>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? (R == 1 ? 4 : R == 2 ? 3 : 2) : (R == 3 ? 1 : 2))
    k_smooth_tile(StencilView<T> s, VecSel<const Vf> fs,
                                                               const c2<T>* __restrict__ u0, TransferView<T> P,
                                                               CoarseLayout L, const c2<T>* __restrict__ uc, int nu,
                                                               int TY, int H, VecSel<Vout> outs,
                                                               c2<T>* __restrict__ rout, const int* active) {
  constexpr int SIDE = 2 * R + 1, NO = SIDE * SIDE;
  using V = c2<T>;
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char sm[];
  const GridDesc g = s.g;
  const int W = g.W, C1 = g.C1, ncls = C1 * C1;
  const int RX = kRegionX, RY = TY + 2 * H, TX = RX - 2 * H;
  V* coef = reinterpret_cast<V*>(sm);
  V* dinv = coef + ncls * NO;
  V* fsm = dinv + ncls;
  V* ua = fsm + RX * RY;
  V* ub = ua + RX * RY;
  int* cx = reinterpret_cast<int*>(ub + RX * RY);
  int* cy = cx + RX;
  const int gx0 = blockIdx.x * TX - H, gy0 = blockIdx.y * TY - H;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const V zero = mk(T(0), T(0));

  for (int i = tid; i < ncls * NO; i += blockDim.x) coef[i] = s.coef[i];
  for (int i = tid; i < ncls && s.wdinv; i += blockDim.x) dinv[i] = s.wdinv[i];
  for (int i = tid; i < RX; i += blockDim.x) {
    const int gx = gx0 + i;
    cx[i] = gx >= 0 && gx < W ? axis_class(gx, W, R, g.q) : -1;
  }
  for (int i = tid; i < RY; i += blockDim.x) {
    const int gy = gy0 + i;
    cy[i] = gy >= 0 && gy < W ? axis_class(gy, W, R, g.q) * C1 : -1;
  }
  // one class for the whole staged region: a period-1 lattice whose region lies inside the
  // interior band [R, W - R) on both axes
  // (reach 1 only: a reach-2 stencil belongs to a period-2 lattice, whose classes alternate)
  // (HET: a heterogeneous wavenumber, whose per-DoF rows and diagonal the kernel reads; the
  // constant-k instantiations carry none of that code)
  const V* hrow = HET ? s.hrow : nullptr;
  bool fast = !HET && R == 1 && g.q == 1 && gx0 >= R && gx0 + RX <= W - R && gy0 >= R && gy0 + RY <= W - R;
  // omega / diag of a staged point: per DoF for a heterogeneous wavenumber, else per class
  auto dg = [&](int cls, int ly, int lx) -> V {
    if constexpr (HET) return s.hwd[(int64_t)(gy0 + ly) * W + gx0 + lx];
    else return dinv[cls];
  };
  // f on the whole region, zero outside the domain: every load of the thread is issued
  // before the first store (rows warp + 8 i, i < kLoadRows)
  const Vf* f = fs.ptr();
#pragma unroll
  for (int b0 = 0; b0 < kLoadRows; b0 += kLoadRows / 2) {   // two batches (registers)
    Vf fv[kLoadRows / 2][2];
#pragma unroll
    for (int i = 0; i < kLoadRows / 2; ++i) {
      const int ly = warp + nw * (b0 + i), gy = gy0 + ly;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int gx = gx0 + lane + 32 * half;
        const bool in = ly < RY && gx >= 0 && gx < W && gy >= 0 && gy < W;
        fv[i][half] = in ? f[(int64_t)gy * W + gx] : Vf{};
      }
    }
#pragma unroll
    for (int i = 0; i < kLoadRows / 2; ++i) {
      const int ly = warp + nw * (b0 + i);
      if (ly < RY)
#pragma unroll
        for (int half = 0; half < 2; ++half) fsm[ly * RX + lane + 32 * half] = stage<V>(fv[i][half]);
    }
  }
  // the start vector (post-smoothing)
  for (int ly = warp; u0 && ly < RY; ly += nw) {
    const int gy = gy0 + ly;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int lx = lane + 32 * half;
      const int gx = gx0 + lx;
      const bool in = gx >= 0 && gx < W && gy >= 0 && gy < W;
      const int64_t p = (int64_t)gy * W + gx;
      {
        V v = in ? u0[p] : zero;
        if (in && uc) {
          // + (P u_c)(p): the canonical interpolation's weights of the fine point's class
          const int a[2] = {gx, gy};
          int pc = 0, mul = 1, anc[2];
          for (int ax = 0; ax < 2; ++ax) {
            pc += mod_period(a[ax], P.pf) * mul;
            mul *= P.pf;
            anc[ax] = div_period(a[ax], P.pf) * P.coarse.q;
          }
          for (int o = 0; o < P.npo; ++o) {
            const T w = P.w[pc * P.npo + o];
            if (w == T(0)) continue;
            const int A[3] = {anc[0] + P.po[o][0], anc[1] + P.po[o][1], 0};
            const V c = uc[coarse_pad_index(P.coarse, L, A)];
            v.x = fma(w, c.x, v.x);
            v.y = fma(w, c.y, v.y);
          }
        }
        ua[ly * RX + lx] = v;
      }
    }
  }
  __syncthreads();
  // the interior class's coefficients and diagonal scaling, in registers on the fast path
  V creg[NO], dreg = zero;
  Sym9 sym{};
  if (fast) {
    const int ic = cx[0] + cy[0];
#pragma unroll
    for (int o = 0; o < NO; ++o) creg[o] = coef[ic * NO + o];
    dreg = dinv[ic];
    if constexpr (R == 1 && sizeof(T) == 4) {
      // the packed form relies on c(o) = c(-o) (A complex symmetric, one class): checked here
#pragma unroll
      for (int o = 0; o < NO; ++o) fast = fast && creg[o].x == creg[NO - 1 - o].x && creg[o].y == creg[NO - 1 - o].y;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const V c = creg[sym9_first(k)];
        sym.rr[k] = make_float2(c.x, c.x);
        sym.ii[k] = make_float2(c.y, c.y);
      }
    }
  }

  V* cur = ua;
  V* nxt = ub;
  int done = 0;   // sweeps done
  if (!u0) {
    // first sweep from zero: u^1 = omega D^-1 f, pointwise on the whole region
    for (int ly = warp; ly < RY; ly += nw) {
      const int cyv = cy[ly];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int lx = lane + 32 * half, cxv = cx[lx];
        cur[ly * RX + lx] = (cxv >= 0 && cyv >= 0) ? cmul(fast ? dreg : dg(cxv + cyv, ly, lx), fsm[ly * RX + lx]) : zero;
      }
    }
    done = 1;
    __syncthreads();
  }
  // full sweeps, each on a region R smaller on every side (its inputs are valid to margin m - R)
  for (int k = 1; done < nu; ++k, ++done) {
    V* out = nxt;
    const V* in = cur;
    if (fast)
      sweep_region<R, T, true, HET>(in, RY, k * R, cx, cy, coef, creg, sym, hrow, gx0, gy0, W,
                               [&](int ly, int lx, int, V Au, V uc) {
                                 const int i = ly * RX + lx;
                                 out[i] = jacobi_step(dreg, fsm[i], Au, uc);
                               });
    else
      sweep_region<R, T, false, HET>(in, RY, k * R, cx, cy, coef, creg, sym, hrow, gx0, gy0, W,
                                [&](int ly, int lx, int cls, V Au, V uc) {
                                  const int i = ly * RX + lx;
                                  out[i] = cls < 0 ? zero : jacobi_step(dg(cls, ly, lx), fsm[i], Au, uc);
                                });
    V* t = cur;
    cur = nxt;
    nxt = t;
    __syncthreads();
  }
  // the tile: u^nu and the residual f - A u^nu
  Vout* out = outs.ptr();
  if (rout) {
    auto emit = [&](int ly, int lx, int cls, V Au, V) {
      if (cls < 0) return;
      const int64_t p = (int64_t)(gy0 + ly) * W + gx0 + lx;
      const int i = ly * RX + lx;
      out[p] = unstage<Vout>(cur[i]);
      rout[p] = csub(fsm[i], Au);
    };
    if (fast)
      sweep_region<R, T, true, HET>(cur, RY, H, cx, cy, coef, creg, sym, hrow, gx0, gy0, W, emit);
    else
      sweep_region<R, T, false, HET>(cur, RY, H, cx, cy, coef, creg, sym, hrow, gx0, gy0, W, emit);
  } else {
    for (int ly = H + warp; ly < H + TY; ly += nw) {
      if (cy[ly] < 0) continue;
      const int lx = H + lane;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int x = lx + 32 * half;
        if (x >= H + TX || cx[x] < 0) continue;
        out[(int64_t)(gy0 + ly) * W + gx0 + x] = unstage<Vout>(cur[ly * RX + x]);
      }
    }
  }
}

// shared memory of one tile (see the kernel's layout)
template <typename T>
size_t tile_smem(const GridDesc& g, int TY, int H) {
  const size_t ncls = (size_t)g.C1 * g.C1;
  const size_t RX = kRegionX, RY = TY + 2 * H;
  return sizeof(c2<T>) * (ncls * g.noff + ncls + 3 * RX * RY) + sizeof(int) * (RX + RY);
}

int g_smem_optin = 0;

}  // namespace

template <typename T>
void smooth_tile_prepare() {
  if (!g_smem_optin) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  const int lim = std::max(0, g_smem_optin - 1024);
  auto set = [&](auto kern) { cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); };
  auto all_r = [&](auto vf, auto vout, auto het) {
    using VF = decltype(vf);
    using VO = decltype(vout);
    constexpr bool HT = decltype(het)::value;
    set(k_smooth_tile<1, T, VF, VO, HT>);
    set(k_smooth_tile<2, T, VF, VO, HT>);
    set(k_smooth_tile<3, T, VF, VO, HT>);
  };
  for (int het = 0; het < 2; ++het) {
    auto with = [&](auto h) {
      all_r(double2{}, double2{}, h);
      all_r(double2{}, c2<T>{}, h);
      if constexpr (sizeof(T) == sizeof(float)) all_r(float4{}, c2<T>{}, h);   // the complex64 V-cycle's f
    };
    if (het)
      with(std::true_type{});
    else
      with(std::false_type{});
  }
  cudaGetLastError();
}

template <typename T, typename Vf, typename Vout>
bool launch_smooth_tile(const StencilView<T>& A, VecSel<const Vf> f, const c2<T>* u0, const TransferView<T>* P,
                        const CoarseLayout* L, const c2<T>* uc, int nu, VecSel<Vout> out, c2<T>* r,
                        const int* active, cudaStream_t s) {
  const GridDesc& g = A.g;
  if (g.dim != 2 || g.R < 1 || g.R > 3 || nu < 1 || (!A.wdinv && !A.hwd) || (uc && (!u0 || !P || !L)))
    return false;
  // sweeps with neighbours: all of them from a start vector, all but the first from zero
  const int full = u0 ? nu : nu - 1;
  const int H = full * g.R + (r ? g.R : 0);
  const int TX = kRegionX - 2 * H;
  if (TX < 16) return false;   // (nu R beyond 24: the per-sweep kernels)
  const size_t lim = (size_t)std::max(0, g_smem_optin - 1024);
  // the tallest tile (32, 16 or 8 rows) that fits two CTAs per SM and still gives the grid
  // about four CTAs per SM (small lattices take short tiles)
  const int64_t want = 4 * 152;
  int TY = 0;
  for (int ty : {32, 24, 16, 8}) {
    // four CTAs per SM for the complex64 reach-1 kernel (its register budget), else two
    const size_t cap = (sizeof(T) == 4 && g.R == 1) ? 56 * 1024 : 113 * 1024;
    if (tile_smem<T>(g, ty, H) > cap) continue;
    const int64_t tiles = (int64_t)((g.W + TX - 1) / TX) * ((g.W + ty - 1) / ty);
    TY = ty;
    if (tiles >= want) break;
  }
  if (!TY)
    for (int ty : {16, 8})
      if (tile_smem<T>(g, ty, H) <= lim) {
        TY = ty;
        break;
      }
  if (!TY) return false;
  const size_t smem = tile_smem<T>(g, TY, H);
  const dim3 grid((g.W + TX - 1) / TX, (g.W + TY - 1) / TY);
  TransferView<T> pv = P ? *P : TransferView<T>{};
  CoarseLayout lv = L ? *L : CoarseLayout{};
  auto go = [&](auto het) {
    constexpr bool HT = decltype(het)::value;
    if (g.R == 1)
      k_smooth_tile<1, T, Vf, Vout, HT><<<grid, kTileThreads, smem, s>>>(A, f, u0, pv, lv, uc, nu, TY, H, out, r, active);
    else if (g.R == 2)
      k_smooth_tile<2, T, Vf, Vout, HT><<<grid, kTileThreads, smem, s>>>(A, f, u0, pv, lv, uc, nu, TY, H, out, r, active);
    else
      k_smooth_tile<3, T, Vf, Vout, HT><<<grid, kTileThreads, smem, s>>>(A, f, u0, pv, lv, uc, nu, TY, H, out, r, active);
  };
  if (A.hrow)
    go(std::true_type{});
  else
    go(std::false_type{});
  return true;
}

template void smooth_tile_prepare<float>();
template void smooth_tile_prepare<double>();
// helm_smooth: f and u complex128
template bool launch_smooth_tile<float, double2, double2>(const StencilView<float>&, VecSel<const double2>,
                                                          const float2*, const TransferView<float>*,
                                                          const CoarseLayout*, const float2*, int,
                                                          VecSel<double2>, float2*, const int*, cudaStream_t);
template bool launch_smooth_tile<double, double2, double2>(const StencilView<double>&, VecSel<const double2>,
                                                           const double2*, const TransferView<double>*,
                                                           const CoarseLayout*, const double2*, int,
                                                           VecSel<double2>, double2*, const int*, cudaStream_t);
// V-cycle, complex64 form: f = a double-float basis slot, u and z complex64
template bool launch_smooth_tile<float, float4, float2>(const StencilView<float>&, VecSel<const float4>,
                                                        const float2*, const TransferView<float>*,
                                                        const CoarseLayout*, const float2*, int, VecSel<float2>,
                                                        float2*, const int*, cudaStream_t);
// V-cycle, FP64 form: f, u and z complex128
// (the double2 -> double2 instantiation above)
// V-cycle of helm_vcycle in the complex64 form: f complex128, u complex64, z complex128
template bool launch_smooth_tile<float, double2, float2>(const StencilView<float>&, VecSel<const double2>,
                                                         const float2*, const TransferView<float>*,
                                                         const CoarseLayout*, const float2*, int, VecSel<float2>,
                                                         float2*, const int*, cudaStream_t);

}  // namespace helm
