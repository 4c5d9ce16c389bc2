// Coarse-grid direct solve of the twogrid cycle (Algorithm 1, coarse line;
// Sec. 6: LU factorisation computed once, reused by every FGMRES iteration).
//
// The coarse matrix A = A_eps^(2h) is block tridiagonal over blocks of grid
// lines (2D P1: one line; 2D P2: two lattice lines; 3D: one plane). Block LU
// ("block Thomas"):
//   S_0 = A_00,  S_J = A_JJ - A_J,J-1 S_{J-1}^{-1} A_J-1,J,   Dinv[J] = S_J^{-1}
// Forward:  w_J = Dinv[J] z_J,  z_{J+1} = r_{J+1} - A_J+1,J w_J   (z_0 = r_0)
// Backward: x_{nb-1} = w_{nb-1},  x_J = w_J - Dinv[J] (A_J,J+1 x_{J+1})
// Storing the inverses turns every sequential step of the triangular solves
// into a dense GEMV that many threads share. No pivoting: for eps > 0,
// Im(x^H A x) < 0 for every leading block, so all Schur complements are
// invertible (an ADR-style argument); a zero/non-finite pivot is reported.
//
// Factorisation: one cooperative grid per block; the Schur update uses the
// sparse couplings straight from the coarse stencil; the inverse is formed by
// in-place Gauss-Jordan with one grid barrier per pivot (pivot row double
// buffered in global memory). FP64 on GB300 is ALU-bound, so all SMs work on
// each block.
//
// Solve: one thread-block cluster (16 CTAs where the device allows, else 8).
// CTA c owns rows [cR, cR+R) of every Dinv[J]; those rows are streamed through
// a multi-stage shared-memory ring by bulk TMA copies (cp.async.bulk +
// mbarrier complete_tx), so a step's GEMV reads shared memory only. After the
// GEMV each CTA broadcasts its R results into every CTA's shared memory
// (st.shared::cluster), one cluster barrier ends the step, and each CTA then
// applies the sparse coupling for the next block locally.
#include <algorithm>

#include "kernels.cuh"

namespace helm {
namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after 2^20 polls, flags HELM_ETIMEOUT in the CTA's
// shared error word and in global memory; once flagged, later waits return at
// once so that a failed solve ends quickly instead of waiting out every step.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned parity, int* s_err, int* err) {
  if (*(volatile int*)s_err) return;
  for (int i = 0; i < (1 << 20); ++i)
    if (mbar_try_wait(bar, parity)) return;
  *(volatile int*)s_err = 1;
  atomicExch(err, HELM_ETIMEOUT);
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// Cluster-wide barrier. The non-.aligned forms are used on purpose: the
// .aligned forms require every thread of a warp to execute them convergently,
// which is not guaranteed right after the divergent single-thread producer code.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void st_cluster(const void* local, unsigned rank, float2 v) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(ra), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(const void* local, unsigned rank, double2 v) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(ra), "d"(v.x), "d"(v.y) : "memory");
}

template <typename V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Lattice coordinates of in-block index i of block J; returns false for padding rows.
__device__ __forceinline__ bool block_coords(const GridDesc& g, const CoarseLayout& L, int J, int i,
                                             int* a) {
  int row = i / L.plane, t = i - row * L.plane;
  for (int ax = 0; ax < g.dim - 1; ++ax) {
    a[ax] = t % g.W;
    t /= g.W;
  }
  a[g.dim - 1] = J * L.rows + row;
  return a[g.dim - 1] < g.W;
}
__device__ __forceinline__ int class_at(const GridDesc& g, const int* a) {
  int cls = 0, mul = 1;
  for (int ax = 0; ax < g.dim; ++ax) {
    cls += axis_class(a[ax], g.W, g.R, g.q) * mul;
    mul *= g.C1;
  }
  return cls;
}
// Neighbour of lattice point a along box offset o: returns its block and in-block index.
__device__ __forceinline__ bool neighbour(const GridDesc& g, const CoarseLayout& L,
                                          const int (*dx)[3], int o, const int* a, int* Jn, int* in) {
  int b[3];
  for (int ax = 0; ax < g.dim; ++ax) {
    b[ax] = a[ax] + dx[o][ax];
    if (b[ax] < 0 || b[ax] >= g.W) return false;
  }
  int last = g.dim - 1;
  *Jn = b[last] / L.rows;
  int idx = (b[last] - *Jn * L.rows) * L.plane, mul = 1;
  for (int ax = 0; ax < last; ++ax) {
    idx += b[ax] * mul;
    mul *= g.W;
  }
  *in = idx;
  return true;
}

// ---------------------------------------------------------------------------
// Factorisation kernel: Schur update + in-place Gauss-Jordan of block J.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_factor_block(c2<T>* D, c2<T>* Tmp, c2<T>* piv,
                                                      unsigned* bar, int* err, StencilView<T> Ac,
                                                      CoarseLayout L, int J) {
  using V = c2<T>;
  extern __shared__ __align__(128) unsigned char sm[];
  const GridDesc g = Ac.g;
  int ncls = 1;
  for (int ax = 0; ax < g.dim; ++ax) ncls *= g.C1;
  V* coef = reinterpret_cast<V*>(sm);
  for (int i = threadIdx.x; i < ncls * g.noff; i += blockDim.x) coef[i] = Ac.coef[i];
  __syncthreads();
  const int B = L.B, ldb = L.ldb;
  const int64_t blk = (int64_t)B * ldb;
  V* S = D + J * blk;
  const V* X = J > 0 ? D + (J - 1) * blk : nullptr;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const V zero = mk(T(0), T(0));

  // Tmp[a][l] = sum_{o: l+o in block J-1} A[l][l+o] X[a][l+o]   (= X A_{J-1,J})
  if (J > 0) {
    for (int64_t idx = gt; idx < (int64_t)B * B; idx += gs) {
      int aa = (int)(idx / B), l = (int)(idx - (int64_t)aa * B);
      int c[3];
      V acc = zero;
      if (block_coords(g, L, J, l, c)) {
        const V* cl = coef + class_at(g, c) * g.noff;
        for (int o = 0; o < g.noff; ++o) {
          int Jn, in;
          if (!neighbour(g, L, Ac.dx, o, c, &Jn, &in) || Jn != J - 1) continue;
          acc = cfma(cl[o], X[(int64_t)aa * ldb + in], acc);
        }
      }
      Tmp[(int64_t)aa * ldb + l] = acc;
    }
    if (!grid_barrier(bar, err, gridDim.x)) return;
  }
  // S[i][l] = A_JJ[i][l] - sum_{o: i+o in block J-1} A[i][i+o] Tmp[i+o][l]; zero padding columns
  for (int64_t idx = gt; idx < (int64_t)B * ldb; idx += gs) {
    int i = (int)(idx / ldb), l = (int)(idx - (int64_t)i * ldb);
    V v = zero;
    if (l < B) {
      int ci[3], cl[3];
      bool ri = block_coords(g, L, J, i, ci);
      bool rl = block_coords(g, L, J, l, cl);
      if (!ri) {
        v = i == l ? mk(T(1), T(0)) : zero;
      } else if (rl) {
        const V* c = coef + class_at(g, ci) * g.noff;
        int o = 0, mul = 1;
        bool in = true;
        for (int ax = 0; ax < g.dim; ++ax) {
          int d = cl[ax] - ci[ax];
          in &= (d >= -g.R && d <= g.R);
          o += (d + g.R) * mul;
          mul *= 2 * g.R + 1;
        }
        if (in) v = c[o];
        if (J > 0) {
          for (int oo = 0; oo < g.noff; ++oo) {
            int Jn, inb;
            if (!neighbour(g, L, Ac.dx, oo, ci, &Jn, &inb) || Jn != J - 1) continue;
            V t = Tmp[(int64_t)inb * ldb + l];
            v = csub(v, cmul(c[oo], t));
          }
        }
      }
    }
    S[idx] = v;
  }
  if (!grid_barrier(bar, err, gridDim.x)) return;

  // In-place Gauss-Jordan inversion of S (no pivoting).
  const int rpb = (B + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rpb, r1 = min(B, r0 + rpb), nr = max(0, r1 - r0);
  V* fs = coef + ncls * g.noff;   // per-row multipliers, rpb entries
  if (r0 <= 0 && 0 < r1)
    for (int j = threadIdx.x; j < B; j += blockDim.x) piv[j] = S[j];
  if (!grid_barrier(bar, err, gridDim.x)) return;
  for (int k = 0; k < B; ++k) {
    const V* pk = piv + (k & 1) * ldb;
    V pkk = pk[k];
    T mag = pkk.x * pkk.x + pkk.y * pkk.y;
    if (!(mag > T(0)) || !isfinite(mag)) {
      if (threadIdx.x == 0) atomicCAS(err, 0, HELM_EZEROPIVOT);
      return;
    }
    V p = cinv(pkk);
    for (int r = threadIdx.x; r < nr; r += blockDim.x) fs[r] = cmul(S[(int64_t)(r0 + r) * ldb + k], p);
    __syncthreads();
    for (int t = threadIdx.x; t < nr * B; t += blockDim.x) {
      int r = t / B, j = t - r * B, i = r0 + r;
      int64_t at = (int64_t)i * ldb + j;
      if (i == k) {
        S[at] = j == k ? p : cmul(p, pk[j]);
      } else if (j == k) {
        S[at] = mk(-fs[r].x, -fs[r].y);
      } else {
        V s = S[at];
        V f = fs[r];
        V pj = pk[j];
        s.x = fma(-f.x, pj.x, s.x);
        s.x = fma(f.y, pj.y, s.x);
        s.y = fma(-f.x, pj.y, s.y);
        s.y = fma(-f.y, pj.x, s.y);
        S[at] = s;
      }
    }
    __syncthreads();
    if (k + 1 < B && r0 <= k + 1 && k + 1 < r1) {
      V* nxt = piv + ((k + 1) & 1) * ldb;
      for (int j = threadIdx.x; j < B; j += blockDim.x) nxt[j] = S[(int64_t)(k + 1) * ldb + j];
    }
    if (!grid_barrier(bar, err, gridDim.x)) return;
  }
}

__global__ void k_convert(const double2* __restrict__ s, float2* __restrict__ d, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = make_float2((float)s[i].x, (float)s[i].y);
}

// ---------------------------------------------------------------------------
// Cluster solve kernel.
// ---------------------------------------------------------------------------
struct SolveGeom {
  int R, CW, nchunk, S;
  int maxc;   // max couplings of one DoF into an adjacent block: R (2R+1)^(dim-1)
  size_t off_mbar, off_rbar, off_coef, off_z, off_gath, off_rbuf, off_acc, off_w, off_stage;
  size_t off_clo, off_dn, off_up;
  size_t total;
};

template <typename T>
SolveGeom solve_geometry(const CoarseLayout& L, const GridDesc& gc, int CS, int CW, int S) {
  int ncls = 1;
  for (int ax = 0; ax < gc.dim; ++ax) ncls *= gc.C1;
  const int noff = gc.noff;
  using V = c2<T>;
  SolveGeom G;
  G.R = (L.B + CS - 1) / CS;
  G.CW = CW;
  G.nchunk = (L.ldb + CW - 1) / CW;
  G.S = S;
  auto al = [](size_t x) { return (x + 127) & ~size_t(127); };
  size_t o = 0;
  G.off_mbar = o; o = al(o + 8 * S);
  G.off_rbar = o; o = al(o + 16 + 16);   // two mbarriers, then the CTA's error word
  G.off_coef = o; o = al(o + sizeof(V) * ncls * noff);
  G.off_z = o; o = al(o + sizeof(V) * L.ldb);
  G.off_gath = o; o = al(o + sizeof(V) * 2 * L.ldb);
  G.off_rbuf = o; o = al(o + sizeof(V) * 2 * L.ldb);
  G.off_acc = o; o = al(o + sizeof(V) * G.R);
  G.off_w = o; o = al(o + sizeof(V) * (size_t)L.nb * G.R);
  G.off_stage = o; o = al(o + sizeof(V) * (size_t)S * G.R * CW);
  G.maxc = coupling_max(gc);
  // coupling lists, contiguous: clo [B], row [B], dn [B*maxc], up [B*maxc]
  G.off_clo = o;
  G.off_dn = o + sizeof(int) * 2 * (size_t)L.B;
  G.off_up = G.off_dn + sizeof(int) * (size_t)L.B * G.maxc;
  o = al(G.off_up + sizeof(int) * (size_t)L.B * G.maxc);
  G.total = o;
  return G;
}

template <typename T>
__global__ void __launch_bounds__(512, 1) k_coarse_solve(const c2<T>* __restrict__ Dinv, StencilView<T> Ac,
                                                        CoarseLayout L, SolveGeom G,
                                                        const int* __restrict__ cpl,
                                                        const c2<T>* __restrict__ rc, c2<T>* __restrict__ uc,
                                                        int* err, const int* active) {
  using V = c2<T>;
  if (active && *active == 0) return;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + G.off_mbar);
  uint64_t* rbar = reinterpret_cast<uint64_t*>(sm + G.off_rbar);
  V* coef = reinterpret_cast<V*>(sm + G.off_coef);
  V* zbuf = reinterpret_cast<V*>(sm + G.off_z);
  V* gath = reinterpret_cast<V*>(sm + G.off_gath);
  V* rbuf = reinterpret_cast<V*>(sm + G.off_rbuf);
  V* acc = reinterpret_cast<V*>(sm + G.off_acc);
  V* wrows = reinterpret_cast<V*>(sm + G.off_w);
  V* stage = reinterpret_cast<V*>(sm + G.off_stage);
  int* clo = reinterpret_cast<int*>(sm + G.off_clo);   // [B] in-plane class part, [B] row in block
  int* dn = reinterpret_cast<int*>(sm + G.off_dn);     // [B][maxc] (o | in << 8), -1 terminated
  int* up = reinterpret_cast<int*>(sm + G.off_up);
  int* s_err = reinterpret_cast<int*>(sm + G.off_rbar + 16);

  const GridDesc g = Ac.g;
  const unsigned rank = cluster_rank(), CS = cluster_size();
  const int B = L.B, ldb = L.ldb, nb = L.nb, R = G.R, CW = G.CW, nchunk = G.nchunk, S = G.S;
  const int r0 = (int)rank * R, r1 = min(B, r0 + R), nr = max(0, r1 - r0);
  const int nsteps = 2 * nb - 1, U = nsteps * nchunk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int maxc = G.maxc;
  const V zero = mk(T(0), T(0));
  int ncls = 1, cmul_last = 1;
  for (int ax = 0; ax < g.dim; ++ax) ncls *= g.C1;
  for (int ax = 0; ax < g.dim - 1; ++ax) cmul_last *= g.C1;
  if (tid == 0) *s_err = 0;
  for (int i = tid; i < ncls * g.noff; i += blockDim.x) coef[i] = Ac.coef[i];
  // coupling lists (built on the host by coupling_lists): plain copy
  for (int i = tid; i < 2 * B + 2 * B * maxc; i += blockDim.x) clo[i] = cpl[i];
  for (int i = tid; i < ldb; i += blockDim.x) {
    zbuf[i] = rc[i];   // z_0 = r_0
    gath[i] = zero;
    gath[ldb + i] = zero;
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&mbar[s], 1);
    mbar_init(&rbar[0], 1);
    mbar_init(&rbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // producer: unit u = (step s, chunk c) -> stage slot u % S
  auto issue = [&](int u) {
    int s = u / nchunk, c = u - s * nchunk;
    int blk = s < nb ? s : 2 * nb - 2 - s;
    int slot = u % S;
    V* dst = stage + (size_t)slot * R * CW;
    const V* src = Dinv + ((size_t)blk * B + r0) * ldb;
    if (nr == 0) {
      mbar_expect_tx(&mbar[slot], 0);
      return;
    }
    if (nchunk == 1) {
      unsigned bytes = (unsigned)(sizeof(V) * (size_t)nr * ldb);
      mbar_expect_tx(&mbar[slot], bytes);
      bulk_g2s(dst, src, bytes, &mbar[slot]);
    } else {
      int c0 = c * CW, nc = min(CW, ldb - c0);
      unsigned bytes = (unsigned)(sizeof(V) * nc);
      mbar_expect_tx(&mbar[slot], bytes * nr);
      for (int r = 0; r < nr; ++r) bulk_g2s(dst + (size_t)r * CW, src + (size_t)r * ldb + c0, bytes, &mbar[slot]);
    }
  };
  auto issue_r = [&](int b) {   // rc block b into rbuf[b & 1]
    unsigned bytes = (unsigned)(sizeof(V) * ldb);
    mbar_expect_tx(&rbar[b & 1], bytes);
    bulk_g2s(rbuf + (size_t)(b & 1) * ldb, rc + (size_t)b * ldb, bytes, &rbar[b & 1]);
  };
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int u = 0; u < min(S, U); ++u) issue(u);
    if (nb > 1) issue_r(1);
  }
  cluster_sync();   // every CTA initialised before any remote store

  int u = 0;
  for (int s = 0; s < nsteps; ++s) {
    const bool fwd = s < nb;
    const int blk = fwd ? s : 2 * nb - 2 - s;
    if (fwd && tid == 0 && blk + 2 < nb) issue_r(blk + 2);
    // ---- GEMV over the CTA's rows: acc[r] = Dinv[blk][r0+r][:] . zbuf
    for (int c = 0; c < nchunk; ++c, ++u) {
      int slot = u % S;
      mbar_wait(&mbar[slot], (unsigned)((u / S) & 1), s_err, err);
      const V* st = stage + (size_t)slot * R * CW;
      int c0 = c * CW, nc = min(CW, B - c0);
      for (int r = warp; r < nr; r += nwarps) {
        V sacc = zero;
        for (int col = lane; col < nc; col += 32) sacc = cfma(st[(size_t)r * CW + col], zbuf[c0 + col], sacc);
        sacc = warp_sum(sacc);
        if (lane == 0) acc[r] = c == 0 ? sacc : cadd(acc[r], sacc);
      }
      __syncthreads();
      if (tid == 0 && u + S < U) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(u + S);
      }
    }
    // ---- results of my rows, broadcast to every CTA
    V* gdst = gath + (size_t)(s & 1) * ldb;
    for (int t = tid; t < nr * (int)CS; t += blockDim.x) {
      int r = t / CS, dst_rank = t - r * CS;
      V val;
      if (fwd) {
        val = acc[r];
      } else {
        val = csub(wrows[(size_t)blk * R + r], acc[r]);
      }
      if (dst_rank == 0) {
        if (fwd) wrows[(size_t)blk * R + r] = val;
        if (!fwd || blk == nb - 1) uc[(size_t)blk * ldb + r0 + r] = val;
      }
      st_cluster(gdst + r0 + r, (unsigned)dst_rank, val);
    }
    cluster_sync();
    // ---- next GEMV input, computed locally from the gathered block
    if (s + 1 < nsteps) {
      const bool down = fwd && blk + 1 < nb;   // z_{blk+1} = r_{blk+1} - A_{blk+1,blk} w_blk
      const int Jd = down ? blk + 1 : blk - 1; // else q_{blk-1} = A_{blk-1,blk} x_blk
      const int* lst = down ? dn : up;
      const V* rb = rbuf + (size_t)(Jd & 1) * ldb;
      if (down) mbar_wait(&rbar[Jd & 1], (unsigned)(((Jd - 1) >> 1) & 1), s_err, err);
      for (int i = tid; i < B; i += blockDim.x) {
        const int lastc = Jd * L.rows + clo[B + i];
        V a = zero;
        if (lastc < g.W) {
          const V* c = coef + (clo[i] + axis_class(lastc, g.W, g.R, g.q) * cmul_last) * g.noff;
          for (int k = 0; k < maxc; ++k) {
            const int e = lst[i * maxc + k];
            if (e < 0) break;
            a = cfma(c[e & 255], gdst[e >> 8], a);
          }
          if (down) a = csub(rb[i], a);
        }
        zbuf[i] = a;
      }
      __syncthreads();
    }
  }
  cluster_sync();
}

}  // namespace

template <typename T>
int plan_coarse_solve(const CoarseLayout& L, const GridDesc& gc, CoarsePlan* plan) {
  using V = c2<T>;
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  size_t budget = (size_t)optin - 1024;
  cudaFuncSetAttribute(k_coarse_solve<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int CS : {16, 8, 4, 2, 1}) {
    // widest chunk (even, <= ldb) that leaves room for >= 2 stages
    for (int CW = L.ldb; CW >= 2; CW = ((CW / 2) + 1) & ~1) {
      for (int S = 4; S >= 2; --S) {
        SolveGeom G = solve_geometry<T>(L, gc, CS, CW, S);
        if (G.total > budget) continue;
        cudaFuncSetAttribute(k_coarse_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CS);
        cfg.blockDim = dim3(512);
        cfg.dynamicSmemBytes = G.total;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, (void*)k_coarse_solve<T>, &cfg) != cudaSuccess || ncl < 1) {
          cudaGetLastError();
          continue;
        }
        plan->CS = CS;
        plan->R = G.R;
        plan->CW = CW;
        plan->nchunk = G.nchunk;
        plan->S = S;
        plan->smem = G.total;
        plan->threads = 512;
        return HELM_OK;
      }
      if (CW == 2) break;
    }
  }
  return HELM_ENOTSUP;
}

template <typename T>
void launch_coarse_solve(const CoarsePlan& plan, const c2<T>* Dinv, const StencilView<T>& Ac,
                         const CoarseLayout& L, const int* cpl, const c2<T>* rc, c2<T>* uc, int* err,
                         const int* active, cudaStream_t s) {
  SolveGeom G = solve_geometry<T>(L, Ac.g, plan.CS, plan.CW, plan.S);
  // (the function's dynamic shared-memory cap was raised to the device limit by
  // plan_coarse_solve, outside any stream capture)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan.CS);
  cfg.blockDim = dim3(plan.threads);
  cfg.dynamicSmemBytes = G.total;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = plan.CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_coarse_solve<T>, Dinv, Ac, L, G, cpl, rc, uc, err, active);
}

template <typename T>
int launch_coarse_factor(c2<T>* Dinv, c2<T>* tmp, c2<T>* piv, unsigned* bar, int* err,
                         const StencilView<T>& Ac, const CoarseLayout& L, int nsm, cudaStream_t s) {
  int ncls = 1;
  for (int ax = 0; ax < Ac.g.dim; ++ax) ncls *= Ac.g.C1;
  int nblk = nsm;
  int rpb = (L.B + nblk - 1) / nblk;
  // +256: the grid barrier's static shared flag precedes the 128-byte aligned dynamic window
  size_t smem = sizeof(c2<T>) * ((size_t)ncls * Ac.g.noff + rpb) + 256;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_factor_block<T>, 256, smem);
  if (per_sm < 1) return HELM_ENOTSUP;
  nblk = std::min(nsm * std::min(per_sm, 2), std::max(1, L.B));
  rpb = (L.B + nblk - 1) / nblk;
  smem = sizeof(c2<T>) * ((size_t)ncls * Ac.g.noff + rpb) + 256;
  for (int J = 0; J < L.nb; ++J) {
    cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    StencilView<T> acv = Ac;
    CoarseLayout lv = L;
    int Jv = J;
    void* args[] = {&Dinv, &tmp, &piv, &bar, &err, &acv, &lv, &Jv};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_factor_block<T>, dim3(nblk), dim3(256), args, smem, s);
    if (e != cudaSuccess) return HELM_ECUDA;
  }
  return HELM_OK;
}

int coupling_max(const GridDesc& g) {
  int m = g.R;
  for (int ax = 0; ax < g.dim - 1; ++ax) m *= 2 * g.R + 1;
  return m;
}

// Coupling lists of the block-tridiagonal coarse matrix, per in-block index i:
// the in-plane part of its class, its row in the block, and the box offsets o
// whose neighbour lies in the previous (dn) / next (up) block, packed as
// o | (neighbour's in-block index << 8), -1 terminated. They do not depend on
// the block: only the class along the last axis does, and the kernel adds it.
void coupling_lists(const GridDesc& g, const CoarseLayout& L, std::vector<int>& out) {
  const int B = L.B, maxc = coupling_max(g);
  out.assign(2 * (size_t)B + 2 * (size_t)B * maxc, -1);
  int* clo = out.data();
  int* dn = clo + 2 * B;
  int* up = dn + (size_t)B * maxc;
  const int side = 2 * g.R + 1;
  for (int i = 0; i < B; ++i) {
    int row = i / L.plane, t = i - row * L.plane, a[3] = {0, 0, 0}, lo = 0, mul = 1;
    for (int ax = 0; ax < g.dim - 1; ++ax) {
      a[ax] = t % g.W;
      t /= g.W;
      lo += axis_class(a[ax], g.W, g.R, g.q) * mul;
      mul *= g.C1;
    }
    clo[i] = lo;
    clo[B + i] = row;
    int nd = 0, nu = 0;
    for (int o = 0; o < g.noff; ++o) {
      int d[3] = {0, 0, 0}, oo = o;
      for (int ax = 0; ax < g.dim; ++ax) {
        d[ax] = oo % side - g.R;
        oo /= side;
      }
      int inpl = 0, m2 = 1;
      bool ok = true;
      for (int ax = 0; ax < g.dim - 1; ++ax) {
        int b = a[ax] + d[ax];
        ok &= (b >= 0 && b < g.W);
        inpl += b * m2;
        m2 *= g.W;
      }
      if (!ok) continue;
      int rr = row + d[g.dim - 1];
      if (rr < 0 && nd < maxc) dn[(size_t)i * maxc + nd++] = o | (((rr + L.rows) * L.plane + inpl) << 8);
      if (rr >= L.rows && nu < maxc) up[(size_t)i * maxc + nu++] = o | (((rr - L.rows) * L.plane + inpl) << 8);
    }
  }
}

void launch_convert_factor(const double2* src, float2* dst, size_t n, cudaStream_t s) {
  k_convert<<<152 * 8, 256, 0, s>>>(src, dst, n);
}

template int plan_coarse_solve<float>(const CoarseLayout&, const GridDesc&, CoarsePlan*);
template int plan_coarse_solve<double>(const CoarseLayout&, const GridDesc&, CoarsePlan*);
template void launch_coarse_solve<float>(const CoarsePlan&, const float2*, const StencilView<float>&,
                                         const CoarseLayout&, const int*, const float2*, float2*, int*,
                                         const int*, cudaStream_t);
template void launch_coarse_solve<double>(const CoarsePlan&, const double2*, const StencilView<double>&,
                                          const CoarseLayout&, const int*, const double2*, double2*, int*,
                                          const int*, cudaStream_t);
template int launch_coarse_factor<double>(double2*, double2*, double2*, unsigned*, int*,
                                          const StencilView<double>&, const CoarseLayout&, int, cudaStream_t);
template int launch_coarse_factor<float>(float2*, float2*, float2*, unsigned*, int*,
                                         const StencilView<float>&, const CoarseLayout&, int, cudaStream_t);

}  // namespace helm
