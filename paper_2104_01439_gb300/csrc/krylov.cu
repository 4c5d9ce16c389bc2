// Flexible GMRES (Saad 1993; Sec. 4: A0 P^{-1} (P u) = F) in complex128.
//
// Arnoldi orthogonalisation is classical Gram-Schmidt with reorthogonalisation,
// in the lagged one-sweep form DCGS2 (Swirydowicz, Langou, Ananthan, Yang, Thomas,
// "Low synchronization Gram-Schmidt and GMRES algorithms", 2020): step j holds the
// vector u_j orthogonalised once; one sweep over the basis forms the inner products
// of both u_j (its second pass) and w = A0 z_j (its first pass), and one sweep applies
// both corrections. Column j-1 of the Hessenberg matrix is therefore finished one step
// late, and each cycle of m columns ends with a step that only finishes column m-1.
// The preconditioner sees u_j; FGMRES allows any z_j, and A0 z_j is expanded in the
// final orthonormal basis, so the Arnoldi relation A0 Z_m = V_{m+1} H_m holds exactly
// in exact arithmetic. Inner products are Hermitian, <a, b> = sum conj(a_i) b_i.
//
// GB300 issues FP64 at 1/58 of its FP32 rate, so the Gram-Schmidt arithmetic
// is done in double-float: every basis entry is stored as hi + lo float pairs,
// every product is formed exactly with an FMA (TwoProduct) and accumulated with
// Knuth's TwoSum; warp reductions stay in double-float and only the per-block
// partials are converted to double. Inner products carry ~48 significant bits
// (relative error ~1e-15 of sum |a_i b_i|), the vector w itself stays complex128.
// Complex Givens rotations (c real, s complex), the residual estimate
// |g_{j+1}| and the convergence test run on the device in one warp, so a
// captured iteration never returns to the host. All kernels read the Arnoldi
// index j and the 'active' / 'pre' flags from device state.
#include "dfloat.cuh"
#include "kernels.cuh"

namespace helm {
namespace {

constexpr int kT = 256;
constexpr int kMaxRestart = 512;   // helm_opts.restart <= 512

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

constexpr int kE = 8;    // basis entries per thread in the inner-product kernel
constexpr int kGD = 2;   // basis vectors per sweep of the inner-product kernel

// Inner products of the basis slots 0..j against two vectors in one sweep over V:
//   s_i = <v_i, u_j>  (u_j = the once-orthogonalised vector in slot j; s_j = ||u_j||^2)
//   t_i = <v_i, w>    (w = A0 z_j; only when this step applies the preconditioner)
// Grid: x over chunks of the vectors (kE entries per thread), y over groups of kGD basis
// slots, so every (chunk, group) pair is its own block. Block partials stay double-float.
__global__ void __launch_bounds__(kT, 5) k_dots2(KrylovBufs kb) {
  KState* st = kb.st;
  if (!st->active) return;
  const int j = st->j, m = st->m;
  const bool pre = st->pre != 0;
  const int i0 = blockIdx.y * kGD;
  if (i0 > j) return;
  const int ng = min(kGD, j + 1 - i0);
  const int64_t N = kb.N, ld = kb.ldN;
  __shared__ float4 red[kT / 32][2 * kGD];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t PS = kb.pstride;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float4* part4 = reinterpret_cast<float4*>(kb.part);
  const float4* uj = kb.Vs + (int64_t)j * ld;
  DF sr[kGD], si[kGD], tr[kGD], ti[kGD];
#pragma unroll
  for (int t = 0; t < kGD; ++t) sr[t] = si[t] = tr[t] = ti[t] = DF{0.f, 0.f};
  // entries base + k * stride, k < kE, in batches of two: the next batch's loads are issued
  // before the current batch's arithmetic. Out-of-range entries load entry 0 and are weighted 0.
  float4 u[2], w[2], v[2][kGD];
  auto load = [&](int k, int b) {
    const int64_t n = base + k * stride;
    const int64_t nn = n < N ? n : 0;
    const float4 z = dfc_zero();
    u[b] = n < N ? uj[nn] : z;
    w[b] = (pre && n < N) ? kb.Ws[nn] : z;
#pragma unroll
    for (int t = 0; t < kGD; ++t) v[b][t] = t < ng ? kb.Vs[(int64_t)(i0 + t) * ld + nn] : z;
  };
  load(0, 0);
#pragma unroll
  for (int k = 0; k < kE; ++k) {
    const int b = k & 1;
    if (k + 1 < kE) load(k + 1, b ^ 1);
#pragma unroll
    for (int t = 0; t < kGD; ++t) {
      const float4 vv = v[b][t], uu = u[b], ww = w[b];
      // conj(v) x = (vr xr + vi xi) + i (vr xi - vi xr)
      df_mac(vv.x, vv.z, uu.x, uu.z, sr[t]);
      df_mac(vv.y, vv.w, uu.y, uu.w, sr[t]);
      df_mac(vv.x, vv.z, uu.y, uu.w, si[t]);
      df_mac(-vv.y, -vv.w, uu.x, uu.z, si[t]);
      if (pre) {
        df_mac(vv.x, vv.z, ww.x, ww.z, tr[t]);
        df_mac(vv.y, vv.w, ww.y, ww.w, tr[t]);
        df_mac(vv.x, vv.z, ww.y, ww.w, ti[t]);
        df_mac(-vv.y, -vv.w, ww.x, ww.z, ti[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < kGD; ++t) {
    DF r = df_wsum(sr[t]), q = df_wsum(si[t]);
    if (lane == 0) red[warp][t] = make_float4(r.h, r.l, q.h, q.l);
    if (pre) {
      r = df_wsum(tr[t]);
      q = df_wsum(ti[t]);
      if (lane == 0) red[warp][kGD + t] = make_float4(r.h, r.l, q.h, q.l);
    }
  }
  __syncthreads();
  const int nout = pre ? 2 * kGD : kGD;
  if (threadIdx.x < nout && (threadIdx.x % kGD) < ng) {
    DF r{0.f, 0.f}, q{0.f, 0.f};
    for (int wi2 = 0; wi2 < kT / 32; ++wi2) {
      const float4 x = red[wi2][threadIdx.x];
      r = df_add(r, DF{x.x, x.y});
      q = df_add(q, DF{x.z, x.w});
    }
    const int t = threadIdx.x % kGD;
    const int64_t row = threadIdx.x < kGD ? kb_row_s(i0 + t) : kb_row_t(m, i0 + t);
    part4[row * PS + blockIdx.x] = make_float4(r.h, r.l, q.h, q.l);
  }
}

// Deterministic reduction of the per-block partials of row r by one warp (lanes
// stride over the blocks, then a fixed shuffle tree).
__device__ __forceinline__ double2 sum_partials(const KrylovBufs& kb, int64_t r, int lane, int nrows) {
  double2 s = make_double2(0.0, 0.0);
  const double2* row = kb.part + r * kb.pstride;
  for (int b = lane; b < nrows; b += 32) s = cadd(s, row[b]);
  return wsum(s);
}

// s_i, t_i = sums of the double-float block partials (reduced in double-float, converted once).
// One warp per row; rows 0..j are s, then (when the step applied the preconditioner) t.
__global__ void __launch_bounds__(kT) k_reduce2(KrylovBufs kb) {
  KState* st = kb.st;
  if (!st->active) return;
  const int j = st->j, m = st->m;
  const int nrow = st->pre ? 2 * (j + 1) : j + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float4* p4 = reinterpret_cast<const float4*>(kb.part);
  for (int q = blockIdx.x * nw + warp; q < nrow; q += gridDim.x * nw) {
    const bool is_t = q > j;
    const int i = is_t ? q - (j + 1) : q;
    DF r{0.f, 0.f}, c{0.f, 0.f};
    const float4* row = p4 + (is_t ? kb_row_t(m, i) : kb_row_s(i)) * kb.pstride;
    for (int b = lane; b < kb.nblk_dots; b += 32) {
      const float4 x = row[b];
      r = df_add(r, DF{x.x, x.y});
      c = df_add(c, DF{x.z, x.w});
    }
    r = df_wsum(r);
    c = df_wsum(c);
    if (lane == 0) (is_t ? kb.tp : kb.hp)[i] = make_double2(df_val(r), df_val(c));
  }
}

__device__ __forceinline__ double2 shfl_up2(double2 v, int d) {
  return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Coefficients of the step (one warp), lagged classical Gram-Schmidt with
// reorthogonalisation (Swirydowicz, Langou, Ananthan, Yang, Thomas 2020, DCGS2): the
// vector u_j in slot j was orthogonalised once; here it is corrected,
//   v_j = (u_j - sum_{i<j} s_i v_i) / rho,  rho^2 = ||u_j||^2 - sum_{i<j} |s_i|^2,
// which finishes column c = j-1 of the Hessenberg matrix (the previous step wrote
// A z_{j-1} = sum h_i v_i + u_j, u_j unnormalised):  h_i += s_i (i < j), h_{j,j-1} = rho.
// Its Givens step: the previous rotations turn the column h into
// col_i = c_i w_i + s_i h_{i+1} with the carried value w_0 = h_0,
// w_{i+1} = -conj(s_i) w_i + c_i h_{i+1} -- an affine recurrence in w. Each lane composes
// the maps of a contiguous chunk of rotations, a warp scan composes the chunks
// ((a2, b2) o (a1, b1) = (a2 a1, a2 b1 + b2)), and each lane replays its chunk from its
// exclusive prefix. The new rotation [c s; -conj(s) c] zeroes h_{c+1} against w_c; the
// residual estimate is |g_{c+1}| / ||F|| with |g_{c+1}| = |s| |g_c|. The new column j
// starts as  h_i = t_i (i < j),  h_jj = <v_j, w> = (t_j - sum_{i<j} conj(s_i) t_i) / rho,
// both divided by rho once more (the step's vector is z_j / rho).
// All operands are fetched into shared memory in one round before the arithmetic.
constexpr int kCoefMax = 520;   // restart length + 2 (helm_opts.restart <= 512)
__global__ void __launch_bounds__(32) k_coef(KrylovBufs kb) {
  KState* st = kb.st;
  if (!st->active) return;
  __shared__ double2 s_s[kCoefMax], s_t[kCoefMax], s_h[kCoefMax], s_sn[kCoefMax];
  __shared__ double s_cs[kCoefMax];
  const int j = st->j, m = st->m, lane = threadIdx.x;
  const bool pre = st->pre != 0;
  const double beta = st->beta;
  for (int i = lane; i <= j; i += 32) {
    s_s[i] = kb.hp[i];
    if (pre) s_t[i] = kb.tp[i];
    if (i < j) s_h[i] = kb.hcol[i];
    if (i + 1 < j) {
      s_sn[i] = kb.sn[i];
      s_cs[i] = kb.cs[i];
    }
  }
  const double2 gc = j >= 1 ? kb.g[j - 1] : make_double2(0.0, 0.0);
  __syncwarp();
  double a = 0.0;
  for (int i = lane; i < j; i += 32) a = fma(s_s[i].x, s_s[i].x, fma(s_s[i].y, s_s[i].y, a));
  a = wsum(a);
  const double rho2 = s_s[j].x - a;
  const double irho = rho2 > 0.0 ? rsqrt(rho2) : 0.0;
  const double rho = rho2 > 0.0 ? rho2 * irho : 0.0;
  int stop = 0;
  if (j == 0) {
    // r = beta u_0 = beta rho v_0
    if (lane == 0) {
      kb.g[0] = make_double2(beta * rho, 0.0);
      st->gabs = beta * rho;
    }
  } else {
    // finished column c = j - 1 (h_0..h_c), in place in s_h
    const int c = j - 1;
    for (int i = lane; i < j; i += 32) s_h[i] = cadd(s_h[i], s_s[i]);
    __syncwarp();
    const double hsub = rho;
    double2* Hc = kb.H + (int64_t)c * (m + 1);
    const int per = (c + 31) / 32;
    const int i0 = min(c, lane * per), i1 = min(c, i0 + per);
    double2 A = make_double2(1.0, 0.0), Bm = make_double2(0.0, 0.0);
    for (int i = i0; i < i1; ++i) {
      const double2 al = make_double2(-s_sn[i].x, s_sn[i].y);   // -conj(s_i)
      const double2 hn = s_h[i + 1];
      Bm = cfma(al, Bm, make_double2(s_cs[i] * hn.x, s_cs[i] * hn.y));
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
    double2 w = cfma(Ae, s_h[0], Be);   // w at the start of this lane's chunk
    for (int i = i0; i < i1; ++i) {
      const double2 sv = s_sn[i];
      const double cc = s_cs[i];
      const double2 hn = s_h[i + 1];
      Hc[i] = cfma(sv, hn, make_double2(cc * w.x, cc * w.y));
      w = cfma(make_double2(-sv.x, sv.y), w, make_double2(cc * hn.x, cc * hn.y));
    }
    // w_c sits with the lane that replayed rotation c-1 (lane 0 when c == 0)
    w = shfl2(w, c == 0 ? 0 : (c - 1) / per);
    if (lane == 0) {
      // new rotation zeroing (w_c, hsub): c = |w|/nu, s = (w/|w|) hsub/nu, r = (w/|w|) nu
      const double aa2 = w.x * w.x + w.y * w.y;
      double cr, sabs;
      double2 sv, r;
      if (!(hsub != 0.0)) {
        cr = 1.0; sv = make_double2(0.0, 0.0); r = w; sabs = 0.0;
      } else if (aa2 == 0.0) {
        cr = 0.0; sv = make_double2(1.0, 0.0); r = make_double2(hsub, 0.0); sabs = 1.0;
      } else {
        const double nu2 = fma(hsub, hsub, aa2);
        const double inu = rsqrt(nu2), iaa = rsqrt(aa2);
        const double nu = nu2 * inu, aa = aa2 * iaa;
        cr = aa * inu;
        sabs = hsub * inu;
        const double fs = sabs * iaa, fr = nu * iaa;
        sv = make_double2(w.x * fs, w.y * fs);
        r = make_double2(w.x * fr, w.y * fr);
      }
      kb.cs[c] = cr;
      kb.sn[c] = sv;
      Hc[c] = r;
      Hc[c + 1] = make_double2(0.0, 0.0);
      kb.g[c + 1] = cmul(make_double2(-sv.x, sv.y), gc);
      kb.g[c] = make_double2(cr * gc.x, cr * gc.y);
      const double gabs = sabs * st->gabs;
      st->gabs = gabs;
      const double est = gabs * st->inv_nF;
      st->est = est;
      st->total += 1;
      if (!isfinite(est) || !isfinite(hsub)) st->nonfinite = 1;
      if (!(hsub > 1e-14 * beta)) st->breakdown = 1;
      if (est <= st->tol) st->converged = 1;
      stop = st->converged || st->breakdown || st->nonfinite;
    }
    stop = __shfl_sync(0xffffffffu, stop, 0);
  }
  if (!pre || !(rho > 0.0)) stop = 1;
  if (stop) {
    if (lane == 0) {
      if (pre && !(rho > 0.0)) st->breakdown = 1;
      st->active = 0;
      st->pre = 0;
    }
    return;   // j columns are finished
  }
  // z_j is used scaled, zhat_j = z_j / rho (u_j is unnormalised): A0 zhat_j = w / rho, so the
  // new column and w carry a factor 1 / rho and the solution update takes y_j / rho
  double2 d = make_double2(0.0, 0.0);
  for (int i = lane; i < j; i += 32) d = cfma(make_double2(s_s[i].x, -s_s[i].y), s_t[i], d);
  d = wsum(d);
  const double i2 = irho * irho;
  const double2 hjj = make_double2((s_t[j].x - d.x) * i2, (s_t[j].y - d.y) * i2);
  // the correction sweep's coefficients as double-float pairs (re.h, re.l, im.h, im.l):
  // [0, j) s_i, [j, 2j) t_i / rho, then h_jj and 1 / rho
  float4* cdf = reinterpret_cast<float4*>(kb.cdf);
  for (int i = lane; i < j; i += 32) {
    const double2 tn = make_double2(s_t[i].x * irho, s_t[i].y * irho);
    kb.hcol[i] = tn;
    DF a = df_split(s_s[i].x), b = df_split(s_s[i].y);
    cdf[i] = make_float4(a.h, a.l, b.h, b.l);
    a = df_split(tn.x);
    b = df_split(tn.y);
    cdf[j + i] = make_float4(a.h, a.l, b.h, b.l);
  }
  if (lane == 0) {
    DF a = df_split(hjj.x), b = df_split(hjj.y);
    cdf[2 * j] = make_float4(a.h, a.l, b.h, b.l);
    a = df_split(irho);
    cdf[2 * j + 1] = make_float4(a.h, a.l, 0.f, 0.f);
    kb.zs[j] = irho;
    kb.hcol[j] = hjj;
    // the correction sweep of this step reads ju; the next step (its preconditioner and A0
    // included) runs at j + 1 and builds column total + 2 if it applies the preconditioner
    st->ju = j;
    st->j = j + 1;
    st->pre = (j + 1 < m && st->total + 2 <= st->maxit) ? 1 : 0;
  }
}

// One sweep over V[0..j-1] for both corrections of the step, all in double-float:
//   v_j = (u_j - sum s_i v_i) / rho          (written into slot j)
//   w  <- w / rho - sum t'_i v_i - h_jj v_j   (t'_i = t_i / rho)
// and w, unnormalised, becomes u_{j+1}: slot j+1 of the basis, the next step's
// preconditioner input (the FP64 form also gets it in complex128, W). Normalisation is
// lagged into rho.
// A warp takes 32 entries: its two half-warps sum over the two halves of the basis for two
// entries per lane, meet with one shuffle, and then every lane finishes one entry.
__global__ void __launch_bounds__(kT, 5) k_update2(KrylovBufs kb) {
  KState* st = kb.st;
  if (!st->active) return;
  const int j = st->ju;
  const int64_t N = kb.N, ld = kb.ldN;
  extern __shared__ float4 hs4[];   // [0, j): s_i, [j, 2j): t_i as (re.h, re.l, im.h, im.l)
  // s_i, t_i / rho, h_jj, 1 / rho as double-float pairs, prepared by the coefficient kernel
  const float4* cdf = reinterpret_cast<const float4*>(kb.cdf);
  for (int i = threadIdx.x; i < 2 * j; i += blockDim.x) hs4[i] = cdf[i];
  const float4 hq = cdf[2 * j], iq = cdf[2 * j + 1];
  const DF irho{iq.x, iq.y};
  const float4 hjj = make_float4(hq.x, hq.z, hq.y, hq.w);   // (hr, hi, lr, li) layout
  __syncthreads();
  const int lane = threadIdx.x & 31, half = lane >> 4;
  const int split = (j + 1) / 2;   // slots [0, split) and [split, j)
  const int ib = half ? split : 0, ie = half ? j : split;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wg * 32 < N; wg += nw) {
    const int64_t na = wg * 32 + (lane & 15), nb2 = na + 16;
    const bool va = na < N, vb = nb2 < N;
    const float4* pa = kb.Vs + (va ? na : 0);
    const float4* pb = kb.Vs + (vb ? nb2 : 0);
    DFC_ACC ua{}, ub{}, wa{}, wb{};
#pragma unroll 2
    for (int i = ib; i < ie; ++i) {
      const float4 hs = hs4[i], ht = hs4[j + i];   // (re.h, re.l, im.h, im.l)
      const float4 v = pa[(int64_t)i * ld], u = pb[(int64_t)i * ld];
      // c x = (cr xr - ci xi) + i (cr xi + ci xr), x in (hr, hi, lr, li) layout
      df_mac(hs.x, hs.y, v.x, v.z, ua.re);
      df_mac(-hs.z, -hs.w, v.y, v.w, ua.re);
      df_mac(hs.x, hs.y, v.y, v.w, ua.im);
      df_mac(hs.z, hs.w, v.x, v.z, ua.im);
      df_mac(hs.x, hs.y, u.x, u.z, ub.re);
      df_mac(-hs.z, -hs.w, u.y, u.w, ub.re);
      df_mac(hs.x, hs.y, u.y, u.w, ub.im);
      df_mac(hs.z, hs.w, u.x, u.z, ub.im);
      df_mac(ht.x, ht.y, v.x, v.z, wa.re);
      df_mac(-ht.z, -ht.w, v.y, v.w, wa.re);
      df_mac(ht.x, ht.y, v.y, v.w, wa.im);
      df_mac(ht.z, ht.w, v.x, v.z, wa.im);
      df_mac(ht.x, ht.y, u.x, u.z, wb.re);
      df_mac(-ht.z, -ht.w, u.y, u.w, wb.re);
      df_mac(ht.x, ht.y, u.y, u.w, wb.im);
      df_mac(ht.z, ht.w, u.x, u.z, wb.im);
    }
    auto xsum = [](DF v) {
      return df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.h, 16), __shfl_xor_sync(0xffffffffu, v.l, 16)});
    };
    ua.re = xsum(ua.re); ua.im = xsum(ua.im); ub.re = xsum(ub.re); ub.im = xsum(ub.im);
    wa.re = xsum(wa.re); wa.im = xsum(wa.im); wb.re = xsum(wb.re); wb.im = xsum(wb.im);
    // lanes 0-15 finish entry na, lanes 16-31 entry nb2 (= wg * 32 + lane in both cases)
    const int64_t n = wg * 32 + lane;
    if (n < N) {
      const DFC_ACC cu = half ? ub : ua;
      DFC_ACC cw = half ? wb : wa;
      float4* slot = kb.Vs + (int64_t)j * ld + n;
      const float4 d = dfc_sub(*slot, dfc_fin(cu));
      const float4 v = dfc_make(df_mul(dfc_re(d), irho), df_mul(dfc_im(d), irho));
      *slot = v;
      dfc_mac(hjj, v, cw);
      const float4 c = dfc_fin(cw);
      const float4 wd = kb.Ws[n];
      const float4 w = dfc_sub(dfc_make(df_mul(dfc_re(wd), irho), df_mul(dfc_im(wd), irho)), c);
      slot[ld] = w;
      if (kb.W) kb.W[n] = dfc_to_double(w);   // FP64 form: the next preconditioner input
    }
  }
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
    kb.part[kb_row_norm(kb.st->m) * kb.pstride + blockIdx.x] = make_double2(t, 0.0);
  }
}
__global__ void k_norm_fin(KrylovBufs kb, int which) {
  KState* st = kb.st;
  const int m = st->m;
  double2 s2 = sum_partials(kb, kb_row_norm(m), threadIdx.x & 31, kb.nblk);
  if (threadIdx.x != 0) return;
  double nrm = sqrt(s2.x);
  if (which == 0) {
    st->nF = nrm;
    st->inv_nF = nrm > 0.0 ? 1.0 / nrm : 0.0;
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
    const double2 v = make_double2(a.x * inv, a.y * inv);
    kb.Vs[n] = dfc_from(v);   // slot 0: the first step's preconditioner input
    if (kb.W) kb.W[n] = v;    // (in complex128 for the FP64 form)
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i <= st->m; i += blockDim.x) kb.g[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
    if (threadIdx.x == 0) {
      st->j = 0;
      st->active = ok ? 1 : 0;
      st->pre = ok && st->m >= 1 && st->total + 1 <= st->maxit ? 1 : 0;
      st->gabs = beta;
      st->converged = 0;
      st->breakdown = 0;
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
      kb.y[i] = make_double2(yi.x * kb.zs[i], yi.y * kb.zs[i]);   // the step used z_i / rho_i
      yi_s = yi;
    }
    __syncthreads();
    double2 yi = yi_s;
    for (int l = threadIdx.x; l < i; l += blockDim.x) rhs[l] = csub(rhs[l], cmul(Ri[l], yi));
    __syncthreads();
  }
}

// x += sum_i y_i Z[i]; complex64 Z: the sum in double-float (y_i split once per block,
// exact products with the complex64 entries), converted to complex128 once per entry
__global__ void __launch_bounds__(kT) k_update_x(KrylovBufs kb, double2* x) {
  KState* st = kb.st;
  const int jj = st->j;
  extern __shared__ double2 ys[];
  float4* yd = reinterpret_cast<float4*>(ys + kMaxRestart);
  for (int i = threadIdx.x; i < jj; i += blockDim.x) {
    ys[i] = kb.y[i];
    yd[i] = dfc_from(kb.y[i]);
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < kb.N; n += stride) {
    double2 a = x[n];
    if (kb.Z32) {
      DFC_ACC acc{DF{0.f, 0.f}, DF{0.f, 0.f}};
      for (int i = 0; i < jj; ++i) {
        const float2 z = kb.Z32[(int64_t)i * kb.ldN + n];
        dfc_mac(yd[i], make_float4(z.x, z.y, 0.f, 0.f), acc);
      }
      const double2 d = dfc_to_double(dfc_fin(acc));
      a.x += d.x;
      a.y += d.y;
    } else {
      for (int i = 0; i < jj; ++i) a = cfma(ys[i], kb.Z[(int64_t)i * kb.ldN + n], a);
    }
    x[n] = a;
  }
}

}  // namespace

void launch_arnoldi(const KrylovBufs& kb, cudaStream_t s, cudaEvent_t mid) {
  k_dots2<<<dim3(kb.nblk_dots, (kb.m + 1 + kGD - 1) / kGD), kT, 0, s>>>(kb);
  k_reduce2<<<(2 * (kb.m + 1) + kT / 32 - 1) / (kT / 32), kT, 0, s>>>(kb);
  k_coef<<<1, 32, 0, s>>>(kb);
  if (mid) cudaEventRecord(mid, s);
  k_update2<<<kb.nblk_upd, kT, sizeof(float4) * 2 * kb.m, s>>>(kb);
}

void launch_cycle_start(const KrylovBufs& kb, const double2* r, cudaStream_t s) {
  k_cycle_start<<<kb.nblk, kT, 0, s>>>(kb, r);
}

void launch_backsolve(const KrylovBufs& kb, cudaStream_t s) { k_backsolve<<<1, kT, 0, s>>>(kb); }

void launch_update_x(const KrylovBufs& kb, double2* x, cudaStream_t s) {
  k_update_x<<<kb.nblk, kT, (sizeof(double2) + sizeof(float4)) * kMaxRestart, s>>>(kb, x);
}

void launch_norm(const KrylovBufs& kb, const double2* v, int which, cudaStream_t s) {
  k_norm_part<<<kb.nblk, kT, 0, s>>>(kb, v);
  k_norm_fin<<<1, 32, 0, s>>>(kb, which);
}

}  // namespace helm
