// Flexible GMRES (Saad 1993; Sec. 4: A0 P^{-1} (P u) = F) in complex128.
//
// Arnoldi orthogonalisation is classical Gram-Schmidt with one conditional
// second pass (DGKS criterion ||w_after|| < ||w_before|| / sqrt(2)); inner
// products are Hermitian, <a, b> = sum conj(a_i) b_i. Each pass is a
// grid-wide dot-product kernel (8 basis vectors per sweep over w), a one-block
// deterministic reduction, and an update kernel that also accumulates ||w||^2.
//
// GB300 issues FP64 at 1/58 of its FP32 rate, so the Gram-Schmidt arithmetic
// is done in double-float: every basis entry is stored as hi + lo float pairs,
// every product is formed exactly with an FMA (TwoProduct) and accumulated with
// Knuth's TwoSum; warp reductions stay in double-float and only the per-block
// partials are converted to double. Inner products carry ~48 significant bits
// (relative error ~1e-15 of sum |a_i b_i|), the vector w itself stays complex128.
// Complex Givens rotations (c real, s complex), the residual estimate
// |g_{j+1}| and the convergence test run on the device in one thread, so a
// captured iteration never returns to the host. All kernels read the Arnoldi
// index j and the 'active' flag from device state.
#include "dfloat.cuh"
#include "kernels.cuh"

namespace helm {
namespace {

constexpr int kT = 256;
constexpr int kG = 8;   // basis vectors per sweep

__device__ __forceinline__ double2 wsum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- double-float helpers (dfloat.cuh): warp reduction --------------------------
__device__ __forceinline__ DF df_wsum(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    v = df_add(v, w);
  }
  return v;
}

constexpr int kE = 4;    // basis entries per thread in the inner-product kernel
constexpr int kGD = 4;   // basis vectors per sweep of the inner-product kernel

// w -> (hi, lo) once per pass, so the inner products run on FP32 pipes only
__global__ void __launch_bounds__(kT) k_split_w(KrylovBufs kb) {
  KState* st = kb.st;
  if (!st->active) return;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < kb.N; n += (int64_t)gridDim.x * blockDim.x) {
    double2 v = kb.W[n];
    DF r = df_split(v.x), q = df_split(v.y);
    kb.Ws[n] = make_float4(r.h, q.h, r.l, q.l);
  }
}

// partial dots of w against the double-float basis V[0..j] (and ||w||^2 in the first pass).
// Grid: x over chunks of w (kE entries per thread), y over groups of kGD basis vectors, so
// that every (chunk, group) pair is its own block and many loads are in flight.
__global__ void __launch_bounds__(kT) k_dots(KrylovBufs kb, int second) {
  KState* st = kb.st;
  if (!st->active || (second && !st->reorth)) return;
  const int j = st->j, m = st->m;
  const int i0 = blockIdx.y * kGD;
  if (i0 > j) return;
  const int ng = min(kGD, j + 1 - i0);
  const int64_t N = kb.N, ld = kb.ldN;
  __shared__ float4 red[kT / 32][kGD];
  __shared__ double rn[kT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // partials are entry-major, part[i * pstride + block], so the reductions read them contiguously
  const int64_t PS = kb.pstride;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (!second && blockIdx.y == 0) {
    double s2 = 0.0;
#pragma unroll
    for (int k = 0; k < kE; ++k) {
      const int64_t n = base + k * stride;
      if (n < N) {
        double2 v = kb.W[n];
        s2 = fma(v.x, v.x, fma(v.y, v.y, s2));
      }
    }
    s2 = wsum(s2);
    if (lane == 0) rn[warp] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < kT / 32; ++i) t += rn[i];
      kb.part[(int64_t)(m + 1) * PS + blockIdx.x] = make_double2(t, 0.0);
    }
  }
  float4* part4 = reinterpret_cast<float4*>(kb.part);
  DF ar[kGD], ai[kGD];
#pragma unroll
  for (int t = 0; t < kGD; ++t) ar[t] = ai[t] = DF{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kE; ++k) {
    const int64_t n = base + k * stride;
    if (n >= N) break;
    const float4 w = kb.Ws[n];   // (hr, hi, lr, li)
#pragma unroll
    for (int t = 0; t < kGD; ++t) {
      if (t < ng) {
        const float4 v = kb.Vs[(int64_t)(i0 + t) * ld + n];
        // conj(v) w = (vr wr + vi wi) + i (vr wi - vi wr)
        df_mac(v.x, v.z, w.x, w.z, ar[t]);
        df_mac(v.y, v.w, w.y, w.w, ar[t]);
        df_mac(v.x, v.z, w.y, w.w, ai[t]);
        df_mac(-v.y, -v.w, w.x, w.z, ai[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < kGD; ++t) {
    DF r = df_wsum(ar[t]), q = df_wsum(ai[t]);
    if (lane == 0) red[warp][t] = make_float4(r.h, r.l, q.h, q.l);
  }
  __syncthreads();
  if (threadIdx.x < ng) {   // block partial, still double-float (converted by k_reduce_h)
    DF r{0.f, 0.f}, q{0.f, 0.f};
    for (int wi2 = 0; wi2 < kT / 32; ++wi2) {
      const float4 x = red[wi2][threadIdx.x];
      r = df_add(r, DF{x.x, x.y});
      q = df_add(q, DF{x.z, x.w});
    }
    part4[(int64_t)(i0 + threadIdx.x) * PS + blockIdx.x] = make_float4(r.h, r.l, q.h, q.l);
  }
}

// Deterministic reduction of the per-block partials of entry i by one warp (lanes
// stride over the blocks, then a fixed shuffle tree).
__device__ __forceinline__ double2 sum_partials(const KrylovBufs& kb, int i, int lane, int nrows) {
  double2 s = make_double2(0.0, 0.0);
  const double2* row = kb.part + (int64_t)i * kb.pstride;
  for (int b = lane; b < nrows; b += 32) s = cadd(s, row[b]);
  return wsum(s);
}

// h = sum of the inner-product partials (double-float, reduced in double-float and
// converted once); hp = this pass's h, hcol accumulates over the passes.
__global__ void __launch_bounds__(kT) k_reduce_h(KrylovBufs kb, double2* hp, int second) {
  KState* st = kb.st;
  if (!st->active || (second && !st->reorth)) return;
  const int j = st->j, m = st->m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float4* p4 = reinterpret_cast<const float4*>(kb.part);
  for (int i = blockIdx.x * nw + warp; i <= j; i += gridDim.x * nw) {
    DF r{0.f, 0.f}, q{0.f, 0.f};
    const float4* row = p4 + (int64_t)i * kb.pstride;
    for (int b = lane; b < kb.nblk_dots; b += 32) {
      const float4 x = row[b];
      r = df_add(r, DF{x.x, x.y});
      q = df_add(q, DF{x.z, x.w});
    }
    r = df_wsum(r);
    q = df_wsum(q);
    if (lane == 0) {
      double2 s2 = make_double2(df_val(r), df_val(q));
      hp[i] = s2;
      kb.hcol[i] = second ? cadd(kb.hcol[i], s2) : s2;
    }
  }
  if (!second && blockIdx.x == 0 && warp == 0) {
    double2 s2 = sum_partials(kb, m + 1, lane, kb.nblk_dots);   // ||w||^2 (FP64)
    if (lane == 0) st->wn0 = sqrt(s2.x);
  }
}

// w -= sum_i hp[i] V[i] (sum in double-float, subtraction in FP64);  partial ||w||^2.
// A warp takes 32 entries: its two half-warps sum over the two halves of the basis for two
// entries per lane (four loads in flight per basis vector and lane pair), meet with one
// shuffle, and then every lane finishes one entry (the FP64 tail uses all 32 lanes).
__global__ void __launch_bounds__(kT) k_update(KrylovBufs kb, const double2* hp, int second) {
  KState* st = kb.st;
  if (!st->active || (second && !st->reorth)) return;
  const int j = st->j, m = st->m;
  const int64_t N = kb.N, ld = kb.ldN;
  extern __shared__ float4 hs4[];   // per coefficient: (re.h, re.l, im.h, im.l)
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    DF r = df_split(hp[i].x), q = df_split(hp[i].y);
    hs4[i] = make_float4(r.h, r.l, q.h, q.l);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, half = lane >> 4;
  const int split = (j + 2) / 2;   // vectors [0, split) and [split, j]
  const int ib = half ? split : 0, ie = half ? j + 1 : split;
  double s2 = 0.0;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;   // warps in the grid
  for (int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wg * 32 < N; wg += nw) {
    const int64_t na = wg * 32 + (lane & 15), nb2 = na + 16;   // this lane's two entries
    DF ar{0.f, 0.f}, ai{0.f, 0.f}, br{0.f, 0.f}, bi{0.f, 0.f};
    const bool va = na < N, vb = nb2 < N;
    const float4* pa = kb.Vs + (va ? na : 0);
    const float4* pb = kb.Vs + (vb ? nb2 : 0);
#pragma unroll 4
    for (int i = ib; i < ie; ++i) {
      const float4 h = hs4[i];                          // (re.h, re.l, im.h, im.l)
      const float4 v = pa[(int64_t)i * ld], u = pb[(int64_t)i * ld];   // (hr, hi, lr, li)
      // h v = (hr vr - hi vi) + i (hr vi + hi vr)
      df_mac(h.x, h.y, v.x, v.z, ar);
      df_mac(-h.z, -h.w, v.y, v.w, ar);
      df_mac(h.x, h.y, v.y, v.w, ai);
      df_mac(h.z, h.w, v.x, v.z, ai);
      df_mac(h.x, h.y, u.x, u.z, br);
      df_mac(-h.z, -h.w, u.y, u.w, br);
      df_mac(h.x, h.y, u.y, u.w, bi);
      df_mac(h.z, h.w, u.x, u.z, bi);
    }
    auto xsum = [](DF v) {
      return df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.h, 16), __shfl_xor_sync(0xffffffffu, v.l, 16)});
    };
    ar = xsum(ar);
    ai = xsum(ai);
    br = xsum(br);
    bi = xsum(bi);
    // lanes 0-15 finish entry na, lanes 16-31 entry nb2 (= wg * 32 + lane in both cases)
    const int64_t n = wg * 32 + lane;
    const DF cr = half ? br : ar, ci = half ? bi : ai;
    if (n < N) {
      double2 w = kb.W[n];
      w.x -= df_val(cr);
      w.y -= df_val(ci);
      kb.W[n] = w;
      DF r = df_split(w.x), q = df_split(w.y);
      kb.Ws[n] = make_float4(r.h, q.h, r.l, q.l);
      s2 = fma(w.x, w.x, fma(w.y, w.y, s2));
    }
  }
  __shared__ double rn[kT / 32];
  s2 = wsum(s2);
  if ((threadIdx.x & 31) == 0) rn[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kT / 32; ++i) t += rn[i];
    kb.part[(int64_t)(m + 1) * kb.pstride + blockIdx.x] = make_double2(t, 0.0);
  }
}

__global__ void k_reduce_norm(KrylovBufs kb, int second) {
  KState* st = kb.st;
  if (!st->active || (second && !st->reorth)) return;
  const int m = st->m;
  double2 s2 = sum_partials(kb, m + 1, threadIdx.x & 31, kb.nblk_upd);
  if (threadIdx.x != 0) return;
  double wn = sqrt(s2.x);
  st->wn = wn;
  if (!second) st->reorth = (wn < 0.70710678118654752 * st->wn0) ? 1 : 0;
}

// v_{j+1} = w / ||w||: stored split (hi + lo) in the basis and in complex128 for the preconditioner
__device__ __forceinline__ void store_basis(const KrylovBufs& kb, int col, int64_t n, double2 v) {
  DF r = df_split(v.x), q = df_split(v.y);
  kb.Vs[(int64_t)col * kb.ldN + n] = make_float4(r.h, q.h, r.l, q.l);
  kb.vj[n] = v;
}

__global__ void __launch_bounds__(kT) k_normalize(KrylovBufs kb) {
  KState* st = kb.st;
  if (!st->active) return;
  const double wn = st->wn;
  if (!(wn > 1e-14 * st->beta) || !isfinite(wn)) return;   // breakdown: handled by k_givens
  const double inv = 1.0 / wn;
  const int col = st->j + 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < kb.N; n += stride) {
    double2 a = kb.W[n];
    store_basis(kb, col, n, make_double2(a.x * inv, a.y * inv));
  }
}

__device__ __forceinline__ double2 shfl_up2(double2 v, int d) {
  return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Givens step for column j (one warp). The previous rotations turn the new column
// h = (h_0..h_j, h_{j+1} = ||w||) into  col_i = c_i u_i + s_i h_{i+1}  with the carried
// value  u_0 = h_0,  u_{i+1} = -conj(s_i) u_i + c_i h_{i+1}  -- an affine recurrence in u.
// Each lane composes the maps of a contiguous chunk of rotations, a warp scan composes
// the chunks ((a2, b2) o (a1, b1) = (a2 a1, a2 b1 + b2)), and each lane then replays its
// chunk from its exclusive prefix. The new rotation [c s; -conj(s) c] zeroes h_{j+1}
// against u_j; the residual estimate is |g_{j+1}| / ||F||.
__global__ void __launch_bounds__(32) k_givens(KrylovBufs kb) {
  KState* st = kb.st;
  if (!st->active) return;
  const int j = st->j, m = st->m, lane = threadIdx.x;
  const double wn = st->wn;
  double2* Hc = kb.H + (int64_t)j * (m + 1);
  const int per = (j + 31) / 32;
  const int i0 = min(j, lane * per), i1 = min(j, i0 + per);
  double2 A = make_double2(1.0, 0.0), Bm = make_double2(0.0, 0.0);
  for (int i = i0; i < i1; ++i) {
    const double2 al = make_double2(-kb.sn[i].x, kb.sn[i].y);   // -conj(s_i)
    const double c = kb.cs[i];
    const double2 hn = kb.hcol[i + 1];
    Bm = cfma(al, Bm, make_double2(c * hn.x, c * hn.y));
    A = cmul(al, A);
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double2 Ap = shfl_up2(A, d), Bp = shfl_up2(Bm, d);
    if (lane >= d) {
      Bm = cfma(A, Bp, Bm);
      A = cmul(A, Ap);
    }
  }
  double2 Ae = shfl_up2(A, 1), Be = shfl_up2(Bm, 1);
  if (lane == 0) {
    Ae = make_double2(1.0, 0.0);
    Be = make_double2(0.0, 0.0);
  }
  double2 u = cfma(Ae, kb.hcol[0], Be);   // u at the start of this lane's chunk
  for (int i = i0; i < i1; ++i) {
    const double2 sv = kb.sn[i];
    const double c = kb.cs[i];
    const double2 hn = kb.hcol[i + 1];
    Hc[i] = cfma(sv, hn, make_double2(c * u.x, c * u.y));
    u = cfma(make_double2(-sv.x, sv.y), u, make_double2(c * hn.x, c * hn.y));
  }
  // u_j sits with the lane that replayed rotation j-1 (lane 0 when j == 0)
  const int owner = j == 0 ? 0 : (j - 1) / per;
  u = shfl2(u, owner);
  if (lane != 0) return;
  // new rotation zeroing (u_j, wn): [c s; -conj(s) c] [a; b] = [r; 0]
  const double2 a = u, b = make_double2(wn, 0.0);
  const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
  double c;
  double2 sv, r;
  if (bb == 0.0) {
    c = 1.0; sv = make_double2(0.0, 0.0); r = a;
  } else if (aa == 0.0) {
    c = 0.0; sv = make_double2(1.0, 0.0); r = b;
  } else {
    const double nu = hypot(aa, bb);
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    c = aa / nu;
    sv = cmul(ph, make_double2(b.x / nu, -b.y / nu));
    r = make_double2(ph.x * nu, ph.y * nu);
  }
  kb.cs[j] = c;
  kb.sn[j] = sv;
  Hc[j] = r;
  Hc[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = kb.g[j];
  const double2 gj1 = cmul(make_double2(-sv.x, sv.y), gj);
  kb.g[j + 1] = gj1;
  kb.g[j] = make_double2(c * gj.x, c * gj.y);
  const double est = hypot(gj1.x, gj1.y) / st->nF;
  st->est = est;
  st->j = j + 1;
  st->total += 1;
  if (!isfinite(est) || !isfinite(wn)) st->nonfinite = 1;
  if (!(wn > 1e-14 * st->beta)) st->breakdown = 1;
  if (est <= st->tol) st->converged = 1;
  if (st->converged || st->breakdown || st->nonfinite || st->j >= m || st->total >= st->maxit) st->active = 0;
}

// ||v||^2 partials / final
__global__ void __launch_bounds__(kT) k_norm_part(KrylovBufs kb, const double2* v) {
  double s = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < kb.N; n += stride) {
    double2 a = v[n];
    s = fma(a.x, a.x, fma(a.y, a.y, s));
  }
  __shared__ double rn[kT / 32];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) rn[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kT / 32; ++i) t += rn[i];
    kb.part[(int64_t)(kb.st->m + 1) * kb.pstride + blockIdx.x] = make_double2(t, 0.0);
  }
}
__global__ void k_norm_fin(KrylovBufs kb, int which) {
  KState* st = kb.st;
  const int m = st->m;
  double2 s2 = sum_partials(kb, m + 1, threadIdx.x & 31, kb.nblk);
  if (threadIdx.x != 0) return;
  double nrm = sqrt(s2.x);
  if (which == 0) {
    st->nF = nrm;
    st->beta = nrm;
  } else {
    st->beta = nrm;
    st->relres = st->nF > 0.0 ? nrm / st->nF : 0.0;
    if (!isfinite(nrm)) st->nonfinite = 1;
  }
}

// V0 = r / beta, g = (beta, 0, ...), new cycle
__global__ void __launch_bounds__(kT) k_cycle_start(KrylovBufs kb, const double2* r) {
  KState* st = kb.st;
  const double beta = st->beta;
  const bool ok = beta > 0.0 && isfinite(beta);
  const double inv = ok ? 1.0 / beta : 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < kb.N; n += stride) {
    double2 a = r[n];
    store_basis(kb, 0, n, make_double2(a.x * inv, a.y * inv));
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i <= st->m; i += blockDim.x) kb.g[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
    if (threadIdx.x == 0) {
      st->j = 0;
      st->active = ok ? 1 : 0;
      st->converged = 0;
      st->breakdown = 0;
      st->reorth = 0;
      if (!isfinite(beta)) st->nonfinite = 1;
    }
  }
}

// y = R^{-1} g over the cycle's j columns (R = rotated H, upper triangular),
// column-oriented: after y_i is known, every thread updates the rows above it.
__global__ void __launch_bounds__(kT) k_backsolve(KrylovBufs kb) {
  KState* st = kb.st;
  const int jj = st->j, m = st->m;
  __shared__ double2 rhs[512];
  __shared__ double2 yi_s;
  for (int i = threadIdx.x; i < jj; i += blockDim.x) rhs[i] = kb.g[i];
  __syncthreads();
  for (int i = jj - 1; i >= 0; --i) {
    const double2* Ri = kb.H + (int64_t)i * (m + 1);   // column i
    if (threadIdx.x == 0) {
      double2 yi = cmul(rhs[i], cinv(Ri[i]));
      kb.y[i] = yi;
      yi_s = yi;
    }
    __syncthreads();
    double2 yi = yi_s;
    for (int l = threadIdx.x; l < i; l += blockDim.x) rhs[l] = csub(rhs[l], cmul(Ri[l], yi));
    __syncthreads();
  }
}

// x += sum_i y_i Z[i]
__global__ void __launch_bounds__(kT) k_update_x(KrylovBufs kb, double2* x) {
  KState* st = kb.st;
  const int jj = st->j;
  extern __shared__ double2 ys[];
  for (int i = threadIdx.x; i < jj; i += blockDim.x) ys[i] = kb.y[i];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < kb.N; n += stride) {
    double2 a = x[n];
    for (int i = 0; i < jj; ++i) a = cfma(ys[i], kb.Z[(int64_t)i * kb.ldN + n], a);
    x[n] = a;
  }
}

}  // namespace

void launch_cgs_pass(const KrylovBufs& kb, bool second, cudaStream_t s) {
  int sec = second ? 1 : 0;
  if (!second) k_split_w<<<kb.nblk, kT, 0, s>>>(kb);
  k_dots<<<dim3(kb.nblk_dots, (kb.m + 1 + kGD - 1) / kGD), kT, 0, s>>>(kb, sec);
  k_reduce_h<<<(kb.m + 1 + kT / 32 - 1) / (kT / 32), kT, 0, s>>>(kb, kb.hp, sec);
  k_update<<<kb.nblk_upd, kT, sizeof(float4) * 513, s>>>(kb, kb.hp, sec);
  k_reduce_norm<<<1, 32, 0, s>>>(kb, sec);
}

void launch_normalize(const KrylovBufs& kb, cudaStream_t s) { k_normalize<<<kb.nblk, kT, 0, s>>>(kb); }

void launch_givens(const KrylovBufs& kb, cudaStream_t s) { k_givens<<<1, 32, 0, s>>>(kb); }

void launch_cycle_start(const KrylovBufs& kb, const double2* r, cudaStream_t s) {
  k_cycle_start<<<kb.nblk, kT, 0, s>>>(kb, r);
}

void launch_backsolve(const KrylovBufs& kb, cudaStream_t s) { k_backsolve<<<1, kT, 0, s>>>(kb); }

void launch_update_x(const KrylovBufs& kb, double2* x, cudaStream_t s) {
  k_update_x<<<kb.nblk, kT, sizeof(double2) * 512, s>>>(kb, x);
}

void launch_norm(const KrylovBufs& kb, const double2* v, int which, cudaStream_t s) {
  k_norm_part<<<kb.nblk, kT, 0, s>>>(kb, v);
  k_norm_fin<<<1, 32, 0, s>>>(kb, which);
}

}  // namespace helm
