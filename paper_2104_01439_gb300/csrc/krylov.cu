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
// In the complex64 form the first pass's projections, and the second pass's small
// correction sum, are formed in float (k_dots2, k_update2): the second pass, which
// stays double-float, completes them.
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

constexpr int kDT = 128;      // threads of the inner-product kernel
constexpr int kDS = 3;        // cp.async stages per thread of the inner-product kernel
constexpr int kDPerSM = 6;    // its resident blocks per SM aimed at (register bound)
// basis vectors per group of the inner-product kernel: 4 with float first-pass sums, 2 when
// both passes are double-float (register budget)
template <bool kExact> constexpr int kGDOf = kExact ? 2 : 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The inner-product kernel's work split: the (group, entry) space of ngr groups x N entries,
// flattened group-major, is cut into G equal contiguous ranges, one per block; block b holds
// [b T / G, (b + 1) T / G) with T = ngr N. dots_block_of(f) is the block whose range holds f.
__host__ __device__ inline int64_t dots_range_begin(int64_t b, int64_t T, int64_t G) { return b * T / G; }
__host__ __device__ inline int64_t dots_block_of(int64_t f, int64_t T, int64_t G) { return ((f + 1) * G - 1) / T; }

// Reduce-scatter across the warp of NV per-lane values (NV a power of two, 2..32): on return
// lane l holds the warp's total of value l / (32 / NV). NV - 1 exchanges (plus log2(32 / NV)
// full ones) instead of 5 NV.
template <int NV>
__device__ __forceinline__ DF df_reduce_scatter(DF (&v)[NV], int lane) {
#pragma unroll
  for (int n = NV, o = 16; n > 1; n >>= 1, o >>= 1) {
    const bool up = lane & o;   // this lane keeps the upper half of the live values
#pragma unroll
    for (int q = 0; q < n / 2; ++q) {
      const DF send = up ? v[q] : v[q + n / 2];
      const DF keep = up ? v[q + n / 2] : v[q];
      v[q] = df_add(keep, DF{__shfl_xor_sync(0xffffffffu, send.h, o), __shfl_xor_sync(0xffffffffu, send.l, o)});
    }
  }
  DF r = v[0];
#pragma unroll
  for (int o = 16 / NV; o > 0; o >>= 1)
    r = df_add(r, DF{__shfl_xor_sync(0xffffffffu, r.h, o), __shfl_xor_sync(0xffffffffu, r.l, o)});
  return r;
}
template <int NV>
__device__ __forceinline__ float f_reduce_scatter(float (&v)[NV], int lane) {
#pragma unroll
  for (int n = NV, o = 16; n > 1; n >>= 1, o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int q = 0; q < n / 2; ++q) {
      const float send = up ? v[q] : v[q + n / 2];
      v[q] = (up ? v[q + n / 2] : v[q]) + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float r = v[0];
#pragma unroll
  for (int o = 16 / NV; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// Accumulators of the first-pass products t_i = <v_i, w>: double-float (kExact) or float.
template <bool kExact> struct TAcc;
template <> struct TAcc<true> {
  DF r, i;
  __device__ __forceinline__ void mac(float4 v, float4 x) {
    df_mac(v.x, v.z, x.x, x.z, r);
    df_mac(v.y, v.w, x.y, x.w, r);
    df_mac(v.x, v.z, x.y, x.w, i);
    df_mac(-v.y, -v.w, x.x, x.z, i);
  }
};
template <> struct TAcc<false> {
  float r, i;
  __device__ __forceinline__ void mac(float4 v, float4 x) {   // the high parts of x only
    r = fmaf(v.x, x.x, fmaf(v.y, x.y, r));
    i = fmaf(v.x, x.y, fmaf(-v.y, x.x, i));
  }
};

// Inner products of the basis slots 0..j against two vectors in one sweep over V:
//   s_i = <v_i, u_j>  (u_j = the once-orthogonalised vector in slot j; s_j = ||u_j||^2)
//   t_i = <v_i, w>    (w = A0 z_j; only when this step applies the preconditioner)
// The slots are taken in groups of kGD (u_j and w are read once per group). A persistent
// grid of G blocks splits the (group, entry) space evenly (dots_range_begin), whatever j is;
// each block accumulates every group its range touches and writes one partial per row and
// block. Each thread streams its entries through shared memory with cp.async, kDS - 1
// entries ahead of the arithmetic.
// The s_i, the second pass that makes the basis orthogonal, are double-float (exact
// products, TwoSum accumulation). The t_i only choose the first correction, which the exact
// double-float update applies as given and the next step's second pass completes, so the
// complex64 form (kExact = false) forms them from the high parts in float (absolute error
// ~1e-7 |v_i| |w|, removed with the rest by that pass); the FP64 form keeps them double-float.
// Block partials are double-float.
template <bool kExact>
__global__ void __launch_bounds__(kDT, kDPerSM) k_dots2(KrylovBufs kb) {
  constexpr int kGD = kGDOf<kExact>, kQ = 2 + kGD;   // staged per entry: u_j, w, the group's slots
  constexpr int NV = 2 * kGD;                          // re, im of each slot
  __shared__ __align__(16) float4 stg[kDS][kQ][kDT];
  __shared__ float4 red[kDT / 32][2 * NV];            // [warp][value]: s as (h, l, 0, 0), then t
  KState* st = kb.st;
  if (!st->active) return;
  const int j = st->j, m = st->m;
  const bool pre = st->pre != 0;
  const int64_t N = kb.N, ld = kb.ldN;
  const int64_t T = (int64_t)((j + kGD) / kGD) * N, G = gridDim.x;
  const int64_t fe = dots_range_begin(blockIdx.x + 1, T, G);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t f = dots_range_begin(blockIdx.x, T, G); f < fe;) {
    const int g = (int)(f / N);
    const int64_t nbeg = f - (int64_t)g * N, nend = min(N, fe - (int64_t)g * N);
    f = (int64_t)g * N + nend;
    const int i0 = g * kGD, ng = min(kGD, j + 1 - i0);
    const float4* uj = kb.Vs + (int64_t)j * ld;
    const float4* vb = kb.Vs + (int64_t)i0 * ld;
    int vo[kGD];   // entry offsets of the slots; slots past ng repeat the last one (not written)
#pragma unroll
    for (int t = 0; t < kGD; ++t) vo[t] = min(t, ng - 1) * (int)ld;
    DF sr[kGD], si[kGD];
    TAcc<kExact> ta[kGD];
#pragma unroll
    for (int t = 0; t < kGD; ++t) {
      sr[t] = si[t] = DF{0.f, 0.f};
      ta[t] = TAcc<kExact>{};
    }
    // entry n of this thread's sequence nbeg + tid + k kDT into stage slot (empty groups past the end)
    auto issue = [&](int64_t n, int slot) {
      if (n < nend) {
        cp_async16(&stg[slot][0][tid], uj + n);
        if (pre) cp_async16(&stg[slot][1][tid], kb.Ws + n);
#pragma unroll
        for (int t = 0; t < kGD; ++t) cp_async16(&stg[slot][2 + t][tid], vb + vo[t] + n);
      }
      cp_async_commit();
    };
    int64_t n = nbeg + tid;
#pragma unroll
    for (int p = 0; p < kDS - 1; ++p) issue(n + (int64_t)p * kDT, p);
    for (int k = 0; n < nend; ++k, n += kDT) {
      issue(n + (int64_t)(kDS - 1) * kDT, (k + kDS - 1) % kDS);
      cp_async_wait<kDS - 1>();   // this entry's copies (issued by this thread) have landed
      const int slot = k % kDS;
      const float4 uu = stg[slot][0][tid];
      const float4 ww = stg[slot][1][tid];
#pragma unroll
      for (int t = 0; t < kGD; ++t) {
        const float4 vv = stg[slot][2 + t][tid];
        // conj(v) x = (vr xr + vi xi) + i (vr xi - vi xr)
        df_mac(vv.x, vv.z, uu.x, uu.z, sr[t]);
        df_mac(vv.y, vv.w, uu.y, uu.w, sr[t]);
        df_mac(vv.x, vv.z, uu.y, uu.w, si[t]);
        df_mac(-vv.y, -vv.w, uu.x, uu.z, si[t]);
        if (pre) ta[t].mac(vv, ww);
      }
    }
    cp_async_wait<0>();
    // warp sums: value 2t + 0/1 = re/im of slot i0 + t; lane l ends with value l / (32 / NV)
    DF sv[NV];
#pragma unroll
    for (int t = 0; t < kGD; ++t) {
      sv[2 * t] = sr[t];
      sv[2 * t + 1] = si[t];
    }
    const DF s_out = df_reduce_scatter<NV>(sv, lane);
    DF t_out{0.f, 0.f};
    if (pre) {
      if constexpr (kExact) {
        DF tv[NV];
#pragma unroll
        for (int t = 0; t < kGD; ++t) {
          tv[2 * t] = ta[t].r;
          tv[2 * t + 1] = ta[t].i;
        }
        t_out = df_reduce_scatter<NV>(tv, lane);
      } else {
        float tv[NV];
#pragma unroll
        for (int t = 0; t < kGD; ++t) {
          tv[2 * t] = ta[t].r;
          tv[2 * t + 1] = ta[t].i;
        }
        t_out = DF{f_reduce_scatter<NV>(tv, lane), 0.f};
      }
    }
    if ((lane & (32 / NV - 1)) == 0) {
      const int q = lane / (32 / NV);
      red[warp][q] = make_float4(s_out.h, s_out.l, 0.f, 0.f);
      red[warp][NV + q] = make_float4(t_out.h, t_out.l, 0.f, 0.f);
    }
    __syncthreads();
    // thread c < 2 kGD: slot i0 + c % kGD of s (c < kGD) or t (c >= kGD), re and im over the warps
    const int c = tid;
    if (c < (pre ? 2 * kGD : kGD) && c % kGD < ng) {
      const int t = c % kGD, base = (c < kGD ? 0 : NV) + 2 * t;
      DF r{0.f, 0.f}, q{0.f, 0.f};
#pragma unroll
      for (int wi2 = 0; wi2 < kDT / 32; ++wi2) {
        const float4 x = red[wi2][base], y = red[wi2][base + 1];
        r = df_add(r, DF{x.x, x.y});
        q = df_add(q, DF{y.x, y.y});
      }
      const int64_t row = c < kGD ? kb_row_s(i0 + t) : kb_row_t(m, i0 + t);
      reinterpret_cast<float4*>(kb.part)[row * kb.pstride + blockIdx.x] = make_float4(r.h, r.l, q.h, q.l);
    }
    __syncthreads();   // red is reused by the next group of the range
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

// s_i, t_i = sums of the double-float block partials (reduced in double-float, converted once)
// over the inner-product blocks whose ranges touched the slot's group.
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
    // the blocks whose ranges touched slot i's group (dots_range_begin)
    const int gd = kb.exact_gs ? kGDOf<true> : kGDOf<false>, g = i / gd;
    const int64_t T = (int64_t)((j + gd) / gd) * kb.N, G = kb.nblk_dots;
    const int blo = (int)dots_block_of((int64_t)g * kb.N, T, G);
    const int bhi = (int)dots_block_of((int64_t)(g + 1) * kb.N - 1, T, G);
    for (int b = blo + lane; b <= bhi; b += 32) {
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

// One sweep over V[0..j-1] for both corrections of the step:
//   v_j = (u_j - sum s_i v_i) / rho          (written into slot j)
//   w  <- w / rho - sum t'_i v_i - h_jj v_j   (t'_i = t_i / rho)
// and w, unnormalised, becomes u_{j+1}: slot j+1 of the basis, the next step's
// preconditioner input (the FP64 form also gets it in complex128, W). Normalisation is
// lagged into rho. The w correction is double-float throughout. The s_i are the second
// pass's coefficients, small against |w| (first-pass error, about 1e-7 |w| with float t_i),
// so in the complex64 form (kExact = false) sum s_i v_i is formed in float from the high
// parts (error ~1e-7 of that sum, ~1e-13 |w|) and subtracted from u_j in double-float;
// the FP64 form forms it in double-float.
// A warp takes 16 entries at a time: its two half-warps sum over the two halves of the basis,
// one entry per lane, and meet with one shuffle; the grid is one wave of resident blocks
// striding over the entries.
template <bool kExact> struct UAcc;
template <> struct UAcc<true> {
  DFC_ACC a;
  __device__ __forceinline__ void mac(float4 hs, float4 v) {   // hs: (re.h, re.l, im.h, im.l)
    df_mac(hs.x, hs.y, v.x, v.z, a.re);
    df_mac(-hs.z, -hs.w, v.y, v.w, a.re);
    df_mac(hs.x, hs.y, v.y, v.w, a.im);
    df_mac(hs.z, hs.w, v.x, v.z, a.im);
  }
  __device__ __forceinline__ void xsum() {
    auto x = [](DF v) {
      return df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.h, 16), __shfl_xor_sync(0xffffffffu, v.l, 16)});
    };
    a.re = x(a.re);
    a.im = x(a.im);
  }
  __device__ __forceinline__ float4 fin() const { return dfc_fin(a); }
};
template <> struct UAcc<false> {
  float re, im;
  __device__ __forceinline__ void mac(float4 hs, float4 v) {
    re = fmaf(hs.x, v.x, fmaf(-hs.z, v.y, re));
    im = fmaf(hs.x, v.y, fmaf(hs.z, v.x, im));
  }
  __device__ __forceinline__ void xsum() {
    re += __shfl_xor_sync(0xffffffffu, re, 16);
    im += __shfl_xor_sync(0xffffffffu, im, 16);
  }
  __device__ __forceinline__ float4 fin() const { return make_float4(re, im, 0.f, 0.f); }
};

template <bool kExact>
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
  for (int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wg * 16 < N; wg += nw) {
    const int64_t n = wg * 16 + (lane & 15);
    const bool valid = n < N;
    const float4* pv = kb.Vs + (valid ? n : 0);
    UAcc<kExact> ua{};
    DFC_ACC wa{};
#pragma unroll 4
    for (int i = ib; i < ie; ++i) {
      const float4 hs = hs4[i], ht = hs4[j + i];   // (re.h, re.l, im.h, im.l)
      const float4 v = pv[(int64_t)i * ld];
      // c x = (cr xr - ci xi) + i (cr xi + ci xr), x in (hr, hi, lr, li) layout
      ua.mac(hs, v);
      df_mac(ht.x, ht.y, v.x, v.z, wa.re);
      df_mac(-ht.z, -ht.w, v.y, v.w, wa.re);
      df_mac(ht.x, ht.y, v.y, v.w, wa.im);
      df_mac(ht.z, ht.w, v.x, v.z, wa.im);
    }
    ua.xsum();
    auto xsum = [](DF v) {
      return df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.h, 16), __shfl_xor_sync(0xffffffffu, v.l, 16)});
    };
    wa.re = xsum(wa.re);
    wa.im = xsum(wa.im);
    // lanes 0-15 finish the warp's 16 entries
    if (half == 0 && valid) {
      DFC_ACC cw = wa;
      float4* slot = kb.Vs + (int64_t)j * ld + n;
      const float4 d = dfc_sub(*slot, ua.fin());
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

}  // namespace

// Blocks of the correction sweep: one wave of resident blocks (at most one per 16 entries).
int update_blocks(int64_t N, int nsm, bool exact, size_t smem) {
  int per_sm = 0;
  const cudaError_t e = exact ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update2<true>, kT, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update2<false>, kT, smem);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * per_sm, (N + kT / 2 - 1) / (kT / 2)));
}

namespace {

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
  if (kb.exact_gs)
    k_dots2<true><<<kb.nblk_dots, kDT, 0, s>>>(kb);
  else
    k_dots2<false><<<kb.nblk_dots, kDT, 0, s>>>(kb);
  k_reduce2<<<(2 * (kb.m + 1) + kT / 32 - 1) / (kT / 32), kT, 0, s>>>(kb);
  k_coef<<<1, 32, 0, s>>>(kb);
  if (mid) cudaEventRecord(mid, s);
  if (kb.exact_gs)
    k_update2<true><<<kb.nblk_upd, kT, sizeof(float4) * 2 * kb.m, s>>>(kb);
  else
    k_update2<false><<<kb.nblk_upd, kT, sizeof(float4) * 2 * kb.m, s>>>(kb);
}

// One wave of resident blocks, and at least 64 entries per block (every range non-empty).
int dots_blocks(int64_t N, int nsm, bool exact) {
  int per_sm = 0;
  const cudaError_t e = exact ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dots2<true>, kDT, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dots2<false>, kDT, 0);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * per_sm, N / 64));
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
