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

// ---------------------------------------------------------------- register-resident columns
// A warp owns one column: lane l holds rows r0 + l + 32 u, u < DF_RMAX (n <= 32 DF_RMAX).
#define DF_RMAX 9
#define DF_PANEL 8

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

// The QR of Section 7 (see cta_reortho) with the factorisation, the T update and the formation
// of Q in double-float.  vsm: shared memory for vcap df numbers, at least DF_PANEL n (the
// panel's reflectors; the T update stages blocks of columns of C in it).  n <= 32 * DF_RMAX.
__device__ inline void cta_reortho_df(int n, double2* Xc, double2* Xn, const double2* Tc,
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
  //    column first brought up to date with the panel's earlier reflectors), then every warp
  //    applies the panel's reflectors to its trailing columns in registers: one load and one
  //    store of a trailing column per panel.
  for (int kb = 0; kb < n; kb += DF_PANEL) {
    const int pe = min(n, kb + DF_PANEL);  // panel columns kb..pe-1 (column n-1: no reflector)
    if (w == 0) {
      for (int c = kb; c < pe; ++c) {
        Col col;
        col_load(col, A + (size_t)c * n, kb, n);
        for (int r = kb; r < c; ++r) {
          float th, tl;
          df::split(s.tau[r], th, tl);
          col_apply(col, vsm + (size_t)(r - kb) * n, kb, n, th, tl);
        }
        col_reflector(col, c, kb, n, vsm + (size_t)(c - kb) * n, s);
        col_store(col, A + (size_t)c * n, kb, n);
        __syncwarp();
      }
    }
    __syncthreads();
    float th[DF_PANEL], tl[DF_PANEL];
#pragma unroll
    for (int r = 0; r < DF_PANEL; ++r) df::split(kb + r < pe ? s.tau[kb + r] : 0.0, th[r], tl[r]);
    for (int j = pe + w; j < n; j += NW) {
      Col col;
      col_load(col, A + (size_t)j * n, kb, n);
      for (int r = kb; r < pe; ++r) col_apply(col, vsm + (size_t)(r - kb) * n, kb, n, th[r - kb], tl[r - kb]);
      col_store(col, A + (size_t)j * n, kb, n);
    }
    __syncthreads();
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
  // 6. Tn = C (Pi^T Tc), C upper triangular: in rounds, each warp owns a pair of output columns
  //    with its rows in registers (Tn[:, j] = sum_k C[:, k] T'[k][j]); the columns of C pass
  //    through shared memory in blocks of kbs, staged by the whole CTA once per round
  {
    const int kbs = max(1, min(32, vcap / n));
    for (int r0 = 0; r0 < n; r0 += 2 * NW) {
      const int j0 = r0 + 2 * w;
      const bool one = j0 < n, two = j0 + 1 < n;
      DAcc a0[DF_RMAX], a1[DF_RMAX];
#pragma unroll
      for (int u = 0; u < DF_RMAX; ++u) {
        a0[u] = DAcc{0.f, 0.f, 0.f, 0.f};
        a1[u] = a0[u];
      }
      for (int k0 = 0; k0 < n; k0 += kbs) {
        const int kn = min(kbs, n - k0);
        for (int e = tid(); e < kn * n; e += nthr()) {
          const int k = k0 + e / n, i = e % n;
          vsm[e] = i <= k ? A[i + (size_t)k * n] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        if (one)
          for (int k = k0; k < k0 + kn; ++k) {
            const df::c4 t0 = ld4(Td + k + (size_t)j0 * n);
            const df::c4 t1 = two ? ld4(Td + k + (size_t)(j0 + 1) * n)
                                  : df::c4{0.f, 0.f, 0.f, 0.f};
            const float4* ck = vsm + (size_t)(k - k0) * n;
#pragma unroll
            for (int u = 0; u < DF_RMAX; ++u) {
              if (32 * u > k) break;  // rows > k of column k of C are zero
              const int i = lane + 32 * u;
              if (i <= k && i < n) {
                const df::c4 c = ld4(ck + i);
                acc_mul(a0[u], c, t0);
                acc_mul(a1[u], c, t1);
              }
            }
          }
        __syncthreads();
      }
      if (one)
#pragma unroll
        for (int u = 0; u < DF_RMAX; ++u) {
          const int i = lane + 32 * u;
          if (i < n) {
            st(Tn + i + (size_t)j0 * n, c4join(acc_value(a0[u])));
            if (two) st(Tn + i + (size_t)(j0 + 1) * n, c4join(acc_value(a1[u])));
          }
        }
    }
  }
  __syncthreads();
  // 7. form Q in place, Q = H_0 H_1 ... H_{n-2}, by groups of DF_PANEL reflectors from the last
  //    one down: each group's reflectors go to shared memory, then a warp per column j >= k0
  //    applies them (from the highest) in registers; the group's own columns start as e_j.
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n, j = e / n;
    if (i < j) st4(A + e, df::c4{0.f, 0.f, 0.f, 0.f});
    if (i == n - 1 && j == n - 1) st4(A + e, df::c4{1.f, 0.f, 0.f, 0.f});  // e_{n-1}
  }
  __syncthreads();
  const int nref = n - 1;  // reflectors 0..n-2 (tau of column n-1 is 0)
  for (int k0 = ((nref - 1) / DF_PANEL) * DF_PANEL; nref > 0 && k0 >= 0; k0 -= DF_PANEL) {
    const int k1 = min(nref - 1, k0 + DF_PANEL - 1);
    for (int e = tid(); e < (k1 - k0 + 1) * n; e += nthr()) {
      const int r = k0 + e / n, i = e % n;
      df::c4 v{0.f, 0.f, 0.f, 0.f};
      if (i == r) v = df::c4{1.f, 0.f, 0.f, 0.f};
      else if (i > r) v = ld4(A + i + (size_t)r * n);
      st4(vsm + (size_t)(r - k0) * n + i, v);
    }
    __syncthreads();
    float th[DF_PANEL], tl[DF_PANEL];
#pragma unroll
    for (int r = 0; r < DF_PANEL; ++r) df::split(k0 + r <= k1 ? s.tau[k0 + r] : 0.0, th[r], tl[r]);
    for (int j = k0 + w; j < n; j += NW) {
      Col col;
      if (j <= k1) {  // e_j
#pragma unroll
        for (int u = 0; u < DF_RMAX; ++u) {
          const int i = k0 + lane + 32 * u;
          col.q[u] = i == j ? df::c4{1.f, 0.f, 0.f, 0.f} : df::c4{0.f, 0.f, 0.f, 0.f};
        }
      } else {
        col_load(col, A + (size_t)j * n, k0, n);
      }
      for (int r = min(j, k1); r >= k0; --r)
        col_apply(col, vsm + (size_t)(r - k0) * n, k0, n, th[r - k0], tl[r - k0]);
      col_store(col, A + (size_t)j * n, k0, n);
    }
    __syncthreads();
  }
  // 8. Q back to FP64, in place (each thread converts its own elements)
  for (int e = tid(); e < n * n; e += nthr()) {
    const df::c4 q = ld4(A + e);
    Xn[e] = make_double2(df::join(q.x, q.y), df::join(q.z, q.w));
  }
  __syncthreads();
}

}  // namespace fd
