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

// Lanes per column for a column reduction over `rows` rows: about 16-32 rows per lane.
__device__ __forceinline__ int df_seg_width(int rows) {
  int W = 1;
  while (W < 32 && rows > 32 * W) W <<= 1;
  return W;
}

// Reflector of column k (rows k..n-1) of the df matrix A, by one warp: FP64 scalars from
// reflector_math, v_i = a_i / c stored below the diagonal, tau and alpha = R_kk in s.
__device__ __forceinline__ void df_reflector(int n, int k, float4* A, Small& s) {
  const int lane = lane_id();
  if (k == n - 1) {
    if (lane == 0) {
      s.tau[k] = 0.0;
      st(s.rdiag + k, c4join(ld4(A + k + (size_t)k * n)));
    }
    return;
  }
  float sh = 0.f, sl = 0.f;
  for (int i = k + 1 + lane; i < n; i += 32) {
    float th, tl, t;
    df::abs2(ld4(A + i + (size_t)k * n), th, tl);
    float s2;
    df::two_sum(sh, th, s2, t);
    sh = s2;
    sl = df::add(sl, df::add(t, tl));
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
    const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
    float s2, t;
    df::two_sum(sh, oh, s2, t);
    sh = s2;
    sl = df::add(df::add(sl, ol), t);
  }
  const double sig = df::join(sh, sl);
  const cplx x = c4join(ld4(A + k + (size_t)k * n));
  const Refl r = reflector_math(x, sig);
  if (r.zero) {
    if (lane == 0) {
      s.tau[k] = 0.0;
      st(s.rdiag + k, cx(0, 0));
      atomicOr(&s.misc[0], 1);
    }
    return;
  }
  const df::c4 ci = df::csplit(r.cinv.re, r.cinv.im);
  for (int i = k + 1 + lane; i < n; i += 32)
    st4(A + i + (size_t)k * n, c4mul(ld4(A + i + (size_t)k * n), ci));
  if (lane == 0) {
    s.tau[k] = r.tau;
    st(s.rdiag + k, r.alpha);
  }
}

// Apply H_k = I - tau v v^H (v_k = 1, v_i = A(i,k) below the diagonal) to columns k+1..n-1.
__device__ __forceinline__ void df_householder_update(int n, int k, float4* A, Small& s) {
  const int lane = lane_id(), w = warp_id(), NW = nwarps();
  const int rows = n - k;
  const int W = df_seg_width(rows), spw = 32 / W, sl = lane % W;
  float th, tl;
  df::split(s.tau[k], th, tl);
  const float4* vcol = A + (size_t)k * n;
  for (int base = k + 1 + w * spw; base < n; base += NW * spw) {
    const int j = base + lane / W;
    const bool act = j < n;
    DAcc acc{0.f, 0.f, 0.f, 0.f};
    if (act)
      for (int i = k + sl; i < n; i += W) {
        const df::c4 v = i == k ? df::c4{1.f, 0.f, 0.f, 0.f} : ld4(vcol + i);
        acc_conj(acc, v, ld4(A + i + (size_t)j * n));
      }
    acc_seg_sum(acc, W);
    if (act) {
      const df::c4 f = df::scale(acc_value(acc), th, tl);
      for (int i = k + sl; i < n; i += W) {
        const df::c4 v = i == k ? df::c4{1.f, 0.f, 0.f, 0.f} : ld4(vcol + i);
        float4* p = A + i + (size_t)j * n;
        st4(p, df::cms(ld4(p), f, v));
      }
    }
  }
}

__device__ inline void cta_reortho_df(int n, double2* Xc, double2* Xn, const double2* Tc,
                                      double2* Tn, double* logD, Small& s) {
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
  // 4. Householder factorisation
  if (w == 0) df_reflector(n, 0, A, s);
  __syncthreads();
  for (int k = 0; k < n - 1; ++k) {
    df_householder_update(n, k, A, s);
    __syncthreads();
    if (w == (k + 1) % NW) df_reflector(n, k + 1, A, s);
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
  // 6. Tn = C (Pi^T Tc), C upper triangular: each thread a 2 x 2 tile of Tn
  {
    const int tiles_i = (n + 1) / 2;
    for (int t = tid(); t < tiles_i * tiles_i; t += nthr()) {
      const int i0 = 2 * (t % tiles_i), j0 = 2 * (t / tiles_i);
      DAcc a00{0.f, 0.f, 0.f, 0.f}, a01 = a00, a10 = a00, a11 = a00;
      const bool i1 = i0 + 1 < n, j1 = j0 + 1 < n;
      for (int k = i0; k < n; ++k) {
        const df::c4 c0 = ld4(A + i0 + (size_t)k * n);
        const df::c4 c1 = (i1 && k >= i0 + 1) ? ld4(A + i0 + 1 + (size_t)k * n)
                                              : df::c4{0.f, 0.f, 0.f, 0.f};
        const df::c4 t0 = ld4(Td + k + (size_t)j0 * n);
        const df::c4 t1 = j1 ? ld4(Td + k + (size_t)(j0 + 1) * n) : df::c4{0.f, 0.f, 0.f, 0.f};
        acc_mul(a00, c0, t0);
        acc_mul(a01, c0, t1);
        acc_mul(a10, c1, t0);
        acc_mul(a11, c1, t1);
      }
      st(Tn + i0 + (size_t)j0 * n, c4join(acc_value(a00)));
      if (j1) st(Tn + i0 + (size_t)(j0 + 1) * n, c4join(acc_value(a01)));
      if (i1) st(Tn + i0 + 1 + (size_t)j0 * n, c4join(acc_value(a10)));
      if (i1 && j1) st(Tn + i0 + 1 + (size_t)(j0 + 1) * n, c4join(acc_value(a11)));
    }
  }
  __syncthreads();
  // 7. form Q in place: Q = H_0 H_1 ... H_{n-2}, accumulated backwards; v_k is copied to the
  //    shared buffer vb before column k is overwritten
  float4* vb = reinterpret_cast<float4*>(s.vbuf);  // 2n df numbers
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n, j = e / n;
    if (i < j) st4(A + e, df::c4{0.f, 0.f, 0.f, 0.f});
    if (i == n - 1 && j == n - 1) st4(A + e, df::c4{1.f, 0.f, 0.f, 0.f});
  }
  if (n >= 2)
    for (int i = n - 1 + tid(); i < n; i += nthr()) vb[((n - 2) & 1) * n + i] = A[i + (size_t)(n - 2) * n];
  __syncthreads();
  for (int k = n - 2; k >= 0; --k) {
    const int rows = n - k - 1;
    const int W = df_seg_width(rows), spw = 32 / W, sl = lane % W;
    float th, tl;
    df::split(s.tau[k], th, tl);
    const float4* vk = vb + (k & 1) * n;
    for (int base = k + w * spw; base < n; base += NW * spw) {
      const int j = base + lane / W;
      const bool act = j < n && j > k;
      DAcc acc{0.f, 0.f, 0.f, 0.f};
      if (act)
        for (int i = k + 1 + sl; i < n; i += W) acc_conj(acc, ld4(vk + i), ld4(A + i + (size_t)j * n));
      acc_seg_sum(acc, W);
      if (act) {
        const df::c4 f = df::scale(acc_value(acc), th, tl);
        if (sl == 0) st4(A + k + (size_t)j * n, c4neg(f));
        for (int i = k + 1 + sl; i < n; i += W) {
          float4* p = A + i + (size_t)j * n;
          st4(p, df::cms(ld4(p), f, ld4(vk + i)));
        }
      }
      if (j == k) {  // this segment sets column k and copies v_{k-1}
        if (sl == 0) {
          float h, l;
          df::two_sum(1.f, -th, h, l);
          df::renorm(h, df::sub(l, tl), h, l);
          st4(A + k + (size_t)k * n, df::c4{h, l, 0.f, 0.f});
        }
        for (int i = k + 1 + sl; i < n; i += W) {
          const df::c4 v = ld4(vk + i);
          st4(A + i + (size_t)k * n, c4neg(df::scale(v, th, tl)));
        }
        if (k >= 1)
          for (int i = k + sl; i < n; i += W) vb[((k - 1) & 1) * n + i] = A[i + (size_t)(k - 1) * n];
      }
    }
    __syncthreads();
  }
  if (n == 1 && tid() == 0) st4(A, df::c4{1.f, 0.f, 0.f, 0.f});
  __syncthreads();
  // 8. Q back to FP64, in place (each thread converts its own elements)
  for (int e = tid(); e < n * n; e += nthr()) {
    const df::c4 q = ld4(A + e);
    Xn[e] = make_double2(df::join(q.x, q.y), df::join(q.z, q.w));
  }
  __syncthreads();
}

}  // namespace fd
