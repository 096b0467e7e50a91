// fd_qr_df.cuh -- the QR re-orthogonalisation of Section 7 (pre-pivoted Householder QR of the
// block product, new log D, T update, Q formation) with its O(n^3) parts -- the Householder
// factorisation, the T update and the formation of Q -- in double-float arithmetic (fd_df.cuh:
// hi + lo FP32 pairs, about 46 significant bits) on the FP32 pipes, which this GPU issues about
// 64 times faster than FP64.  The pivot keys, the reflector scalars (reflector_math), log D and
// the T-update coefficients stay FP64; inputs and outputs (Xc, Tc -> Xn, Tn, log D) are FP64 as
// for cta_reortho.  Used by the mixed-precision chains, whose slice products are TF32.
//
// Working storage: the factorisation runs in place in Xn read as n x n complex df numbers
// (float4: Re hi, Re lo, Im hi, Im lo; 16 bytes like a complex128), and Xc, which is free after
// the columns are gathered, holds the permuted Tc in df for the T update.  Both may be shared or
// global memory.  All threads of the CTA call it; it ends with __syncthreads().
#pragma once

#include "fd_df.cuh"
#include "fd_fp64.cuh"

namespace fd {

__device__ __forceinline__ df::c4 ld4(const float4* p) {
  const float4 v = *p;
  return df::c4{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ void st4(float4* p, df::c4 v) { *p = make_float4(v.x, v.y, v.z, v.w); }
__device__ __forceinline__ df::c4 c4neg(df::c4 a) { return df::c4{-a.x, -a.y, -a.z, -a.w}; }
// a * b for complex df numbers
__device__ __forceinline__ df::c4 c4mul(df::c4 a, df::c4 b) {
  return c4neg(df::cms(df::c4{0.f, 0.f, 0.f, 0.f}, a, b));
}
__device__ __forceinline__ cplx c4join(df::c4 a) {
  return cx(df::join(a.x, a.y), df::join(a.z, a.w));
}

// Compensated accumulation (Ogita-Rump-Oishi Dot2 with df factors): s + c, the products exact
// to ~2^-46 and every rounding error of the running sum carried in c.
struct DAcc {
  float rs, rc, is, ic;
};
__device__ __forceinline__ void acc_prod(float& s, float& c, float ah, float al, float bh,
                                         float bl) {
  float p, e, s2, t;
  df::prod(ah, al, bh, bl, p, e);
  df::two_sum(s, p, s2, t);
  s = s2;
  c = df::add(c, df::add(t, e));
}
// A += conj(v) a
__device__ __forceinline__ void acc_conj(DAcc& A, df::c4 v, df::c4 a) {
  acc_prod(A.rs, A.rc, v.x, v.y, a.x, a.y);
  acc_prod(A.rs, A.rc, v.z, v.w, a.z, a.w);
  acc_prod(A.is, A.ic, v.x, v.y, a.z, a.w);
  acc_prod(A.is, A.ic, -v.z, -v.w, a.x, a.y);
}
// A += a b
__device__ __forceinline__ void acc_mul(DAcc& A, df::c4 a, df::c4 b) {
  acc_prod(A.rs, A.rc, a.x, a.y, b.x, b.y);
  acc_prod(A.rs, A.rc, -a.z, -a.w, b.z, b.w);
  acc_prod(A.is, A.ic, a.x, a.y, b.z, b.w);
  acc_prod(A.is, A.ic, a.z, a.w, b.x, b.y);
}
// xor-reduction of an accumulator inside aligned groups of W lanes (all 32 lanes call it)
__device__ __forceinline__ void acc_seg_sum(DAcc& A, int W) {
  for (int o = 1; o < W; o <<= 1) {
    const float rs = __shfl_xor_sync(0xffffffffu, A.rs, o);
    const float rc = __shfl_xor_sync(0xffffffffu, A.rc, o);
    const float is = __shfl_xor_sync(0xffffffffu, A.is, o);
    const float ic = __shfl_xor_sync(0xffffffffu, A.ic, o);
    float s, t;
    df::two_sum(A.rs, rs, s, t);
    A.rs = s;
    A.rc = df::add(df::add(A.rc, rc), t);
    df::two_sum(A.is, is, s, t);
    A.is = s;
    A.ic = df::add(df::add(A.ic, ic), t);
  }
}
__device__ __forceinline__ df::c4 acc_value(const DAcc& A) {
  df::c4 r;
  df::renorm(A.rs, A.rc, r.x, r.y);
  df::renorm(A.is, A.ic, r.z, r.w);
  return r;
}

__device__ __forceinline__ df::c4 df_of(double2 v) { return df::csplit(v.x, v.y); }
__device__ __forceinline__ df::c4 df_conj(df::c4 a) { return df::c4{a.x, a.y, -a.z, -a.w}; }

// C (m x p) = A (m x K) B (K x p) in df with the operands staged through shared memory: BM x BN
// output tiles (64 x 64, or 16 x 256 for a short-and-wide product), K in chunks of 16; 256
// threads, each a 4 x 4 block of outputs with compensated accumulators.  The threads run along
// the rows first (rows ty + TY a, columns tx + TX b): the epilogue's loads and stores of a
// column-major output are contiguous across neighbouring threads.  A(i, k) = aload(i, k) is
// staged with i fastest and B(k, j) = bload(k, j) with k fastest, so column-major operands in
// global memory are read contiguously; each thread issues its loads of a chunk together before
// storing them to shared memory (one memory latency per chunk, not one per element), and the B
// tile's rows are padded by one df number so that those stores avoid bank conflicts.  Both
// loaders are called once per element per tile, inside the bounds.
//   df_gemm_tiled: epi(i, j, c4) stores an output element.
//   df_gemm_sub_tiled: C(i, j) -= (A B)(i, j) in place at caddr(i, j) (a df number), the old
//   values of a thread's block loaded together before the update.
// sm: shared memory for DF_TILE_ELEMS(BM, BN) df numbers.  upper_a: A is upper triangular (its K
// chunks below a tile's rows are skipped).  All threads of the CTA call it (blockDim.x == 256).
#define DF_TILE_ELEMS(BM, BN) (16 * ((BM) + (BN) + 1))
template <int BM, int BN, bool SUB, class ALoad, class BLoad, class Epi>
__device__ inline void df_gemm_core(int m, int p, int K, const ALoad& aload, const BLoad& bload,
                                    const Epi& epi, float4* sm, bool upper_a) {
  static_assert(BM * BN == 4096, "256 threads of 4 x 4 outputs");
  constexpr int TY = BM / 4, TX = BN / 4, BS = BN + 1;
  constexpr int NA = 16 * BM / 256, NB = 16 * BN / 256, GB = NB < 8 ? NB : 8;
  float4* As = sm;            // [16][BM]: As[k * BM + i]
  float4* Bs = sm + 16 * BM;  // [16][BS]: Bs[k * BS + j]
  const int t = tid();
  const int ty = t % TY, tx = t / TY;
  const df::c4 zero{0.f, 0.f, 0.f, 0.f};
  for (int i0 = 0; i0 < m; i0 += BM)
    for (int j0 = 0; j0 < p; j0 += BN) {
      DAcc acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = DAcc{0.f, 0.f, 0.f, 0.f};
      // an upper triangular A (A(i, k) = 0 for k < i) contributes nothing below the tile's rows
      for (int k0 = upper_a ? (i0 / 16) * 16 : 0; k0 < K; k0 += 16) {
        __syncthreads();
        {
          df::c4 ra[NA];
#pragma unroll
          for (int u = 0; u < NA; ++u) {
            const int e = t + 256 * u, kk = e / BM, r = e % BM;
            const int i = i0 + r, k = k0 + kk;
            ra[u] = (i < m && k < K) ? aload(i, k) : zero;
          }
#pragma unroll
          for (int u = 0; u < NA; ++u) st4(As + t + 256 * u, ra[u]);
        }
#pragma unroll
        for (int g = 0; g < NB; g += GB) {
          df::c4 rb[GB];
#pragma unroll
          for (int u = 0; u < GB; ++u) {
            const int e = t + 256 * (g + u), kk = e % 16, r = e / 16;
            const int j = j0 + r, k = k0 + kk;
            rb[u] = (j < p && k < K) ? bload(k, j) : zero;
          }
#pragma unroll
          for (int u = 0; u < GB; ++u) {
            const int e = t + 256 * (g + u), kk = e % 16, r = e / 16;
            st4(Bs + kk * BS + r, rb[u]);
          }
        }
        __syncthreads();
        const int kn = min(16, K - k0);
        for (int kk = 0; kk < kn; ++kk) {
          df::c4 av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = ld4(As + kk * BM + ty + TY * a);
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = ld4(Bs + kk * BS + tx + TX * b);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc_mul(acc[a][b], av[a], bv[b]);
        }
      }
      if constexpr (SUB) {
        const df::c4 one{1.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int b0 = 0; b0 < 4; b0 += 2) {
          df::c4 old[2][4];
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              const int i = i0 + ty + TY * a, j = j0 + tx + TX * (b0 + b);
              old[b][a] = (i < m && j < p) ? ld4(epi(i, j)) : zero;
            }
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              const int i = i0 + ty + TY * a, j = j0 + tx + TX * (b0 + b);
              if (i < m && j < p) st4(epi(i, j), df::cms(old[b][a], acc_value(acc[a][b0 + b]), one));
            }
        }
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = i0 + ty + TY * a, j = j0 + tx + TX * b;
            if (i < m && j < p) epi(i, j, acc_value(acc[a][b]));
          }
      }
    }
  __syncthreads();
}
template <int BM = 64, int BN = 64, class ALoad, class BLoad, class Epi>
__device__ __forceinline__ void df_gemm_tiled(int m, int p, int K, const ALoad& aload,
                                              const BLoad& bload, const Epi& epi, float4* sm,
                                              bool upper_a = false) {
  df_gemm_core<BM, BN, false>(m, p, K, aload, bload, epi, sm, upper_a);
}
template <int BM = 64, int BN = 64, class ALoad, class BLoad, class CAddr>
__device__ __forceinline__ void df_gemm_sub_tiled(int m, int p, int K, const ALoad& aload,
                                                  const BLoad& bload, const CAddr& caddr,
                                                  float4* sm) {
  df_gemm_core<BM, BN, true>(m, p, K, aload, bload, caddr, sm, false);
}

// ---------------------------------------------------------------- register-resident columns
// A warp owns one column: lane l holds rows r0 + l + 32 u, u < DF_RMAX (n <= 32 DF_RMAX).
#define DF_RMAX 9
#define DF_PANEL 16

struct Col {
  df::c4 q[DF_RMAX];
};
__device__ __forceinline__ void col_load(Col& c, const float4* colp, int r0, int n) {
  const int l = lane_id();
#pragma unroll
  for (int u = 0; u < DF_RMAX; ++u) {
    const int i = r0 + l + 32 * u;
    c.q[u] = i < n ? ld4(colp + i) : df::c4{0.f, 0.f, 0.f, 0.f};
  }
}
__device__ __forceinline__ void col_store(const Col& c, float4* colp, int r0, int n) {
  const int l = lane_id();
#pragma unroll
  for (int u = 0; u < DF_RMAX; ++u) {
    const int i = r0 + l + 32 * u;
    if (i < n) st4(colp + i, c.q[u]);
  }
}
// Apply H = I - tau v v^H to the column (rows >= r0); v (rows r0.., zero above its own row,
// 1 on it) in shared memory.
__device__ __forceinline__ void acc_merge(DAcc& a, const DAcc& b) {
  float s, t;
  df::two_sum(a.rs, b.rs, s, t);
  a.rs = s;
  a.rc = df::add(df::add(a.rc, b.rc), t);
  df::two_sum(a.is, b.is, s, t);
  a.is = s;
  a.ic = df::add(df::add(a.ic, b.ic), t);
}
__device__ __forceinline__ void col_apply(Col& c, const float4* v, int r0, int n, float th,
                                          float tl) {
  const int l = lane_id();
  // three independent accumulators: the compensated sums are serial chains of dependent FP32
  // operations, so interleaving them keeps the pipes busier
  DAcc acc[3] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
  for (int u = 0; u < DF_RMAX; ++u) {
    const int i = r0 + l + 32 * u;
    if (i < n) acc_conj(acc[u % 3], ld4(v + i), c.q[u]);
  }
  acc_merge(acc[0], acc[1]);
  acc_merge(acc[0], acc[2]);
  DAcc& a0 = acc[0];
  acc_seg_sum(a0, 32);
  DAcc acc1 = a0;
  const df::c4 f = df::scale(acc_value(acc1), th, tl);
#pragma unroll
  for (int u = 0; u < DF_RMAX; ++u) {
    const int i = r0 + l + 32 * u;
    if (i < n) c.q[u] = df::cms(c.q[u], f, ld4(v + i));
  }
}

// Reflector of column k held in registers (rows r0..n-1, k >= r0): FP64 scalars from
// reflector_math; the column's rows > k become v (a_i / c), row k becomes 1, rows < k stay.
// Writes v (rows r0..n-1: 0 above k, 1 at k) to vs, and tau, alpha = R_kk to s.
__device__ __forceinline__ void col_reflector(Col& c, int k, int r0, int n, float4* vs,
                                              Small& s) {
  const int l = lane_id();
  float sh = 0.f, sl = 0.f;
  df::c4 x{0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int u = 0; u < DF_RMAX; ++u) {
    const int i = r0 + l + 32 * u;
    if (i > k && i < n) {
      float th, tl, t, s2;
      df::abs2(c.q[u], th, tl);
      df::two_sum(sh, th, s2, t);
      sh = s2;
      sl = df::add(sl, df::add(t, tl));
    }
    if (i == k) x = c.q[u];
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
    const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
    float s2, t;
    df::two_sum(sh, oh, s2, t);
    sh = s2;
    sl = df::add(df::add(sl, ol), t);
    x.x += __shfl_xor_sync(0xffffffffu, x.x, o);  // exactly one lane holds row k
    x.y += __shfl_xor_sync(0xffffffffu, x.y, o);
    x.z += __shfl_xor_sync(0xffffffffu, x.z, o);
    x.w += __shfl_xor_sync(0xffffffffu, x.w, o);
  }
  const Refl r = k == n - 1 ? Refl{c4join(x), cx(0, 0), 0.0, false}
                            : reflector_math(c4join(x), df::join(sh, sl));
  if (l == 0) {
    s.tau[k] = k == n - 1 || r.zero ? 0.0 : r.tau;
    st(s.rdiag + k, k == n - 1 ? c4join(x) : (r.zero ? cx(0, 0) : r.alpha));
    if (r.zero) atomicOr(&s.misc[0], 1);
  }
  const df::c4 ci = df::csplit(r.cinv.re, r.cinv.im);
#pragma unroll
  for (int u = 0; u < DF_RMAX; ++u) {
    const int i = r0 + l + 32 * u;
    if (i >= n) continue;
    df::c4 v;
    if (i < k) v = df::c4{0.f, 0.f, 0.f, 0.f};
    else if (i == k) v = df::c4{1.f, 0.f, 0.f, 0.f};
    else v = (k == n - 1 || r.zero) ? df::c4{0.f, 0.f, 0.f, 0.f} : c4mul(c.q[u], ci);
    st4(vs + i, v);
    if (i > k) c.q[u] = v;  // rows below k keep v; rows <= k keep R (and x on the diagonal)
  }
}

// T of the block reflector H_0 H_1 ... H_{np-1} = I - V T V^H of np consecutive reflectors
// (forward, column-wise: T upper triangular, T_jj = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j)
// (V(:, 0:j)^H v_j)).  V(r, j) = vs[j * n + r] for rows r0..n-1 (zero above row r0 + j, 1 on it).
// Tw, Sg: shared memory, DF_PANEL^2 df numbers each (column-major, leading dimension DF_PANEL).
__device__ inline void df_block_t(int np, int r0, int n, const float4* vs, const double* tau,
                                  float4* Tw, float4* Sg) {
  const int lane = lane_id(), w = warp_id(), NW = nwarps();
  // Gram entries S(i, j) = v_i^H v_j, i < j
  for (int pr = w; pr < np * np; pr += NW) {
    const int i = pr % np, j = pr / np;
    if (i >= j) continue;
    DAcc acc{0.f, 0.f, 0.f, 0.f};
    for (int r = r0 + j + lane; r < n; r += 32)  // v_j is zero above row r0 + j
      acc_conj(acc, ld4(vs + (size_t)i * n + r), ld4(vs + (size_t)j * n + r));
    acc_seg_sum(acc, 32);
    if (lane == 0) st4(Sg + i + j * DF_PANEL, acc_value(acc));
  }
  __syncthreads();
  if (w == 0) {
    for (int j = 0; j < np; ++j) {
      float th, tl;
      df::split(tau[j], th, tl);
      if (lane < j) {  // T(i, j) = -tau_j sum_{k=i}^{j-1} T(i, k) S(k, j)
        DAcc acc{0.f, 0.f, 0.f, 0.f};
        for (int k = lane; k < j; ++k)
          acc_mul(acc, ld4(Tw + lane + k * DF_PANEL), ld4(Sg + k + j * DF_PANEL));
        st4(Tw + lane + j * DF_PANEL, c4neg(df::scale(acc_value(acc), th, tl)));
      }
      if (lane == 0) st4(Tw + j + j * DF_PANEL, df::c4{th, tl, 0.f, 0.f});
      if (lane > j && lane < DF_PANEL) st4(Tw + lane + j * DF_PANEL, df::c4{0.f, 0.f, 0.f, 0.f});
      __syncwarp();
    }
  }
  __syncthreads();
}

// Apply the block reflector of np reflectors (vs, Tw as for df_block_t, rows r0..n-1) to columns
// c0..n-1 of the df matrix A (rows r0..n-1): A <- (I - V Tw' V^H) A with Tw' = Tw^H (adjoint:
// the factorisation's H_{np-1}...H_0) or Tw (the formation of Q's H_0...H_{np-1}).  Wg: global
// scratch for DF_PANEL x (n - c0) df numbers; gsm: shared memory for the GEMM tiles.
__device__ inline void df_apply_block(int np, int r0, int c0, int n, const float4* vs,
                                      const float4* Tw, bool adjoint, float4* A, float4* Wg,
                                      float4* gsm) {
  const int m = n - r0, p = n - c0;
  if (p <= 0) return;
  // W = V^H A(r0:, c0:)   (np x p)
  df_gemm_tiled<16, 256>(
      np, p, m, [&](int i, int k) { return df_conj(ld4(vs + (size_t)i * n + r0 + k)); },
      [&](int k, int j) { return ld4(A + r0 + k + (size_t)(c0 + j) * n); },
      [&](int i, int j, df::c4 v) { st4(Wg + i + (size_t)j * DF_PANEL, v); }, gsm);
  // W <- Tw' W, a thread per column
  for (int j = tid(); j < p; j += nthr()) {
    df::c4 wv[DF_PANEL];
#pragma unroll
    for (int k = 0; k < DF_PANEL; ++k)
      wv[k] = k < np ? ld4(Wg + k + (size_t)j * DF_PANEL) : df::c4{0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < DF_PANEL; ++i) {
      if (i >= np) break;
      DAcc acc{0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < DF_PANEL; ++k) {
        if (k >= np) break;
        if (adjoint ? (k <= i) : (k >= i)) {  // T^H lower, T upper triangular
          const df::c4 tk = adjoint ? df_conj(ld4(Tw + k + i * DF_PANEL)) : ld4(Tw + i + k * DF_PANEL);
          acc_mul(acc, tk, wv[k]);
        }
      }
      st4(Wg + i + (size_t)j * DF_PANEL, acc_value(acc));
    }
  }
  __syncthreads();
  // A(r0:, c0:) -= V W
  df_gemm_sub_tiled<64, 64>(
      m, p, np, [&](int i, int k) { return ld4(vs + (size_t)k * n + r0 + i); },
      [&](int k, int j) { return ld4(Wg + k + (size_t)j * DF_PANEL); },
      [&](int i, int j) { return A + r0 + i + (size_t)(c0 + j) * n; }, gsm);
}

// The QR of Section 7 (see cta_reortho) with the factorisation, the T update and the formation
// of Q in double-float, the O(n^3) work in shared-memory tiled df GEMMs on block reflectors
// (compact WY form) of DF_PANEL reflectors.  vsm: shared memory for vcap >= DF_PANEL (n + 2
// DF_PANEL) + DF_TILE_ELEMS(16, 256) df numbers (the panel's reflectors, its T and Gram
// matrices, the GEMM tiles).
// Tc is consumed: after its rows are gathered in df into Xc, its memory holds the block
// reflectors' DF_PANEL x n intermediate products.  n <= 32 * DF_RMAX.
__device__ inline void cta_reortho_df(int n, double2* Xc, double2* Xn, double2* Tc,
                                      double2* Tn, double* logD, Small& s, float4* vsm,
                                      int vcap) {
  const int lane = lane_id(), w = warp_id(), NW = nwarps();
  float4* A = reinterpret_cast<float4*>(Xn);
  float4* Td = reinterpret_cast<float4*>(Xc);
  float* keyf = (float*)s.key;
  // 1. pivot keys e^{logD_j} ||xc_j|| as FP32 logs (the order only has to be roughly sorted)
  for (int j = w; j < n; j += NW) {
    double a = 0.0;
    for (int i = lane; i < n; i += 32) a += abs2(ld(Xc + i + (size_t)j * n));
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) {
      float kk = (float)logD[j] + 0.5f * log_key(a);
      if (!(a == a) || !(kk == kk)) {
        kk = -INFINITY;
        atomicOr(&s.misc[0], 1);
      }
      keyf[j] = kk;
    }
  }
  __syncthreads();
  // 2. rank sort, descending key, ties by index
  for (int j = tid(); j < n; j += nthr()) {
    const float kj = keyf[j];
    int r = 0;
    for (int i = 0; i < n; ++i) {
      const float ki = keyf[i];
      r += (ki > kj) || (ki == kj && i < j);
    }
    s.perm[r] = j;
  }
  __syncthreads();
  // 3. gather the columns into the df working matrix; the column scaling is never formed
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n, k = e / n;
    const double2 x = Xc[i + (size_t)s.perm[k] * n];
    st4(A + e, df::csplit(x.x, x.y));
  }
  for (int k = tid(); k < n; k += nthr()) s.logw[k] = logD[s.perm[k]];
  if (w == 0) {
    double lo = INFINITY, hi = -INFINITY;
    for (int k = lane; k < n; k += 32) {
      lo = fmin(lo, logD[k]);
      hi = fmax(hi, logD[k]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      s.red[8] = 0.5 * (lo + hi);
      s.misc[4] = (hi - lo) < 1200.0 ? 1 : 0;
    }
  }
  __syncthreads();
  // Tc with its rows permuted, in df (Xc is free now)
  for (int e = tid(); e < n * n; e += nthr()) {
    const int k = e % n, c = e / n;
    const double2 t = Tc[s.perm[k] + (size_t)c * n];
    st4(Td + e, df::csplit(t.x, t.y));
  }
  const bool scaled = s.misc[4] != 0;
  // 4. blocked Householder factorisation: warp 0 factors a panel of DF_PANEL columns (each
  //    column first brought up to date with the panel's earlier reflectors, in registers), then
  //    the panel's block reflector I - V T V^H updates the trailing columns by two tiled GEMMs
  float4* Vs = vsm;                                  // DF_PANEL x n
  float4* Tw = vsm + (size_t)DF_PANEL * n;           // DF_PANEL^2
  float4* Sg = Tw + DF_PANEL * DF_PANEL;             // DF_PANEL^2
  float4* gsm = Sg + DF_PANEL * DF_PANEL;            // GEMM tiles
  float4* Wg = reinterpret_cast<float4*>(Tc);        // DF_PANEL x n, global
  for (int kb = 0; kb < n; kb += DF_PANEL) {
    const int pe = min(n, kb + DF_PANEL);  // panel columns kb..pe-1 (column n-1: no reflector)
    if (w == 0) {
      for (int c = kb; c < pe; ++c) {
        Col col;
        col_load(col, A + (size_t)c * n, kb, n);
        for (int r = kb; r < c; ++r) {
          float th, tl;
          df::split(s.tau[r], th, tl);
          col_apply(col, Vs + (size_t)(r - kb) * n, kb, n, th, tl);
        }
        col_reflector(col, c, kb, n, Vs + (size_t)(c - kb) * n, s);
        col_store(col, A + (size_t)c * n, kb, n);
        __syncwarp();
      }
    }
    __syncthreads();
    if (pe < n) {
      df_block_t(pe - kb, kb, n, Vs, s.tau + kb, Tw, Sg);
      df_apply_block(pe - kb, kb, pe, n, Vs, Tw, true, A, Wg, gsm);
    }
  }
  // 5. new log D, the row factors q_k = 1 / (sc_k |R_kk|), and the T-update coefficients
  //    C_kj = R'_kj sc_j q_k (j > k), C_kk = R_kk / |R_kk|, FP64, stored back in df
  for (int k = tid(); k < n; k += nthr()) {
    const double r2 = abs2(ld(s.rdiag + k));
    if (!(r2 > 0.0)) atomicOr(&s.misc[0], 1);
    const double ir = rsqrt64(r2);
    logD[k] = -log(ir) + s.logw[k];
    const double sc = scaled ? exp(s.logw[k] - s.red[8]) : 1.0;
    s.sa[k] = sc;
    s.sb[k] = scaled ? ir * rcp64(sc) : ir;
  }
  __syncthreads();
  for (int e = tid(); e < n * n; e += nthr()) {
    const int k = e % n, j = e / n;
    if (j < k) continue;
    cplx c;
    if (j == k) {
      c = s.sb[k] * ld(s.rdiag + k);
      if (scaled) c = s.sa[k] * c;
    } else {
      const cplx rkj = c4join(ld4(A + e));
      if (scaled) {
        c = s.sb[k] * (s.sa[j] * rkj);
      } else {
        const double ex = s.logw[j] - s.logw[k];
        const double m = sqrt64(abs2(rkj));
        c = m == 0.0 ? cx(0, 0) : (exp(log(m) + ex) * s.sb[k] * rcp64(m)) * rkj;
      }
    }
    if (!(abs2(c) < 1e72)) atomicOr(&s.misc[0], 1);  // beyond the df range
    st4(A + e, df::csplit(c.re, c.im));
  }
  __syncthreads();
  // 6. Tn = C (Pi^T Tc), C upper triangular, one tiled df GEMM
  df_gemm_tiled<64, 64>(
      n, n, n,
      [&](int i, int k) { return i <= k ? ld4(A + i + (size_t)k * n) : df::c4{0.f, 0.f, 0.f, 0.f}; },
      [&](int k, int j) { return ld4(Td + k + (size_t)j * n); },
      [&](int i, int j, df::c4 v) { st(Tn + i + (size_t)j * n, c4join(v)); }, gsm, true);
  // 7. form Q in place, Q = H_0 H_1 ... H_{n-2}, by groups of DF_PANEL reflectors from the last
  //    one down: a group's reflectors go to shared memory, its own columns become e_j, and its
  //    block reflector I - V T V^H is applied to columns k0..n-1 (rows k0..n-1)
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n, j = e / n;
    if (i < j) st4(A + e, df::c4{0.f, 0.f, 0.f, 0.f});
    if (i == n - 1 && j == n - 1) st4(A + e, df::c4{1.f, 0.f, 0.f, 0.f});  // e_{n-1}
  }
  __syncthreads();
  const int nref = n - 1;  // reflectors 0..n-2 (tau of column n-1 is 0)
  for (int k0 = ((nref - 1) / DF_PANEL) * DF_PANEL; nref > 0 && k0 >= 0; k0 -= DF_PANEL) {
    const int k1 = min(nref - 1, k0 + DF_PANEL - 1), np = k1 - k0 + 1;
    for (int e = tid(); e < np * n; e += nthr()) {
      const int r = k0 + e / n, i = e % n;
      df::c4 v{0.f, 0.f, 0.f, 0.f};
      if (i == r) v = df::c4{1.f, 0.f, 0.f, 0.f};
      else if (i > r) v = ld4(A + i + (size_t)r * n);
      st4(Vs + (size_t)(r - k0) * n + i, v);
    }
    __syncthreads();
    for (int e = tid(); e < np * (n - k0); e += nthr()) {
      const int j = k0 + e / (n - k0), i = k0 + e % (n - k0);
      st4(A + i + (size_t)j * n, i == j ? df::c4{1.f, 0.f, 0.f, 0.f} : df::c4{0.f, 0.f, 0.f, 0.f});
    }
    __syncthreads();
    df_block_t(np, k0, n, Vs, s.tau + k0, Tw, Sg);
    df_apply_block(np, k0, k0, n, Vs, Tw, false, A, Wg, gsm);
  }
  // 8. Q back to FP64, in place (each thread converts its own elements)
  for (int e = tid(); e < n * n; e += nthr()) {
    const df::c4 q = ld4(A + e);
    Xn[e] = make_double2(df::join(q.x, q.y), df::join(q.z, q.w));
  }
  __syncthreads();
}

// The stabilised product of two factored matrices (cta_merge) with its O(n^3) work in
// double-float: Xs Ds Ts (acting later) times Xa Da Ta = Xs [Ds Ts Xa] Da Ta, the bracket
// Xc = e^{-c} Ds (Ts Xa) as a tiled df GEMM (c = the mid-range of log Ds, so that Xc's rows lie
// within e^{+-span/2}), re-factored by the pre-pivoted QR of cta_reortho_df (the column scaling
// Da never formed), then X = Xs Q by a second GEMM and log D += c.  The df numbers carry FP32's
// exponent range and the QR squares its entries, so a left factor whose log D spans more than
// DF_MERGE_SPAN marks the configuration (misc[0]) instead of losing its small rows.  FP64 inputs
// and outputs; Ta is copied to Tw (the QR consumes its T input).  Scratch: Xc, Xn (Q), Tw; the
// result in X, Tn, logD.  sm: the QR's shared memory (vcap df numbers).
#define DF_MERGE_SPAN 76.0
__device__ inline void cta_merge_df(int n, const double2* Xs, const double2* Ts, const double* lDs,
                                    const double2* Xa, const double2* Ta, const double* lDa,
                                    double2* Xc, double2* Xn, double2* Tw, double2* Tn, double2* X,
                                    double* logD, Small& s, float4* sm, int vcap) {
  if (warp_id() == 0) {
    double lo = INFINITY, hi = -INFINITY;
    for (int k = lane_id(); k < n; k += 32) {
      lo = fmin(lo, lDs[k]);
      hi = fmax(hi, lDs[k]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane_id() == 0) {
      s.red[9] = 0.5 * (lo + hi);
      if (!(hi - lo <= DF_MERGE_SPAN)) atomicOr(&s.misc[0], 1);
    }
  }
  __syncthreads();
  const double c = s.red[9];
  for (int k = tid(); k < n; k += nthr()) {
    s.sa[k] = exp(lDs[k] - c);
    logD[k] = lDa[k];
  }
  for (int e = tid(); e < n * n; e += nthr()) Tw[e] = Ta[e];
  __syncthreads();
  df_gemm_tiled(
      n, n, n, [&](int i, int k) { return df_of(Ts[i + (size_t)k * n]); },
      [&](int k, int j) { return df_of(Xa[k + (size_t)j * n]); },
      [&](int i, int j, df::c4 v) {
        const double a = s.sa[i];
        Xc[i + (size_t)j * n] = make_double2(a * df::join(v.x, v.y), a * df::join(v.z, v.w));
      },
      sm);
  cta_reortho_df(n, Xc, Xn, Tw, Tn, logD, s, sm, vcap);
  for (int k = tid(); k < n; k += nthr()) logD[k] += c;
  df_gemm_tiled(
      n, n, n, [&](int i, int k) { return df_of(Xs[i + (size_t)k * n]); },
      [&](int k, int j) { return df_of(Xn[k + (size_t)j * n]); },
      [&](int i, int j, df::c4 v) {
        X[i + (size_t)j * n] = make_double2(df::join(v.x, v.y), df::join(v.z, v.w));
      },
      sm);
}

}  // namespace fd
