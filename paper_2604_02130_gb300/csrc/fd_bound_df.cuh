// fd_bound_df.cuh -- the block-boundary Green's function of the force sweep (Section 7 steps 7-9
// with t1 = t2, Section 5.3) in double-float arithmetic (fd_df.cuh) on the FP32 pipes, for the
// mixed-precision force of the streamed size classes:
//   L = X_L D_L T_L (left checkpoint), R^H = X_R D_R T_R (right checkpoint),
//   M = D_Lb^{-1} X_L^H X_R D_Rb^{-1} + D_Ls T_L T_R^H D_Rs,   G_t = X_R D_Rb^{-1} M^{-1} D_Lb^{-1} X_L^H.
// The scale factors (e^{-max(log D, 0)}, e^{min(log D, 0)}) are FP64; the three products, the LU
// factorisation of M with partial pivoting and the solve are df; inputs and output are FP64
// (column-major).  Working storage in global memory: three n x n df matrices.
#pragma once

#include "fd_qr_df.cuh"

namespace fd {

// Blocked LU with partial pivoting of the df matrix A (n x n, column-major), applied to the nr
// columns of B, then B <- U^{-1} B: on return B = A^{-1} B_in.  Panels of DF_LU_P columns are
// factored column by column (pivot search on FP32 magnitudes, full-row swaps of A and B); the
// block row of U and of B follow by forward substitution with the panel's unit L, and the
// trailing matrix and the remaining rows of B by df_gemm_tiled.  The back substitution runs by
// blocks too.  Reciprocal pivots (df) in s.vbuf; sm: shared memory for df_gemm_tiled.
#define DF_LU_P 16
__device__ inline void cta_lu_solve_blocked_df(int n, float4* A, float4* B, int nr, Small& s,
                                               float4* sm) {
  const int lane = lane_id(), w = warp_id();
  float4* piv = reinterpret_cast<float4*>(s.vbuf);
  const df::c4 one{1.f, 0.f, 0.f, 0.f};
  for (int kb = 0; kb < n; kb += DF_LU_P) {
    const int pe = min(n, kb + DF_LU_P);
    // (1) panel: columns kb..pe-1, rows kb..n-1
    for (int k = kb; k < pe; ++k) {
      if (w == 0) {
        float best = -1.f;
        int bi = k;
        for (int i = k + lane; i < n; i += 32) {
          const float4 v = A[i + (size_t)k * n];
          const float m = v.x * v.x + v.z * v.z;
          if (m > best) {
            best = m;
            bi = i;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
          }
        }
        if (lane == 0) s.piv[k] = bi;
      }
      __syncthreads();
      const int bi = s.piv[k];
      if (bi != k) {
        for (int j = tid(); j < n + nr; j += nthr()) {
          float4* a = j < n ? A + k + (size_t)j * n : B + k + (size_t)(j - n) * n;
          float4* b = j < n ? A + bi + (size_t)j * n : B + bi + (size_t)(j - n) * n;
          const float4 t = *a;
          *a = *b;
          *b = t;
        }
        __syncthreads();
      }
      if (w == 0) {
        df::c4 p = ld4(A + k + (size_t)k * n);
        float th, tl;
        df::abs2(p, th, tl);
        if (!(th > 0.f)) {
          if (lane == 0) atomicOr(&s.misc[0], 1);
          p = one;
          th = 1.f;
          tl = 0.f;
        }
        float yh, yl;
        df::recip(th, tl, yh, yl);
        const df::c4 pinv = df::scale(df_conj(p), yh, yl);
        if (lane == 0) st4(piv + k, pinv);
        for (int i = k + 1 + lane; i < n; i += 32)
          st4(A + i + (size_t)k * n, c4mul(ld4(A + i + (size_t)k * n), pinv));
      }
      __syncthreads();
      // rank-1 update inside the panel: columns k+1..pe-1, rows k+1..n-1
      const int m = n - k - 1, cols = pe - k - 1;
      for (int e = tid(); e < m * cols; e += nthr()) {
        const int i = k + 1 + e % m, j = k + 1 + e / m;
        float4* q = A + i + (size_t)j * n;
        st4(q, df::cms(ld4(q), ld4(A + i + (size_t)k * n), ld4(A + k + (size_t)j * n)));
      }
      __syncthreads();
    }
    // (2) block row: rows kb..pe-1 of A (columns pe..n-1) and of B <- L11^{-1} (.), a thread per
    //     column, the column's panel rows in registers
    for (int c = tid(); c < (n - pe) + nr; c += nthr()) {
      float4* col = c < n - pe ? A + (size_t)(pe + c) * n : B + (size_t)(c - (n - pe)) * n;
      df::c4 x[DF_LU_P];
#pragma unroll
      for (int r = 0; r < DF_LU_P; ++r) x[r] = kb + r < pe ? ld4(col + kb + r) : one;
#pragma unroll
      for (int r = 1; r < DF_LU_P; ++r)
#pragma unroll
        for (int q = 0; q < r; ++q)
          if (kb + r < pe) x[r] = df::cms(x[r], ld4(A + kb + r + (size_t)(kb + q) * n), x[q]);
#pragma unroll
      for (int r = 0; r < DF_LU_P; ++r)
        if (kb + r < pe) st4(col + kb + r, x[r]);
    }
    __syncthreads();
    // (3) trailing update: A22 -= L21 U12, B2 -= L21 B1
    if (pe < n) {
      const int m = n - pe;
      auto l21 = [&](int i, int k) { return ld4(A + pe + i + (size_t)(kb + k) * n); };
      df_gemm_sub_tiled(
          m, m, pe - kb, l21, [&](int k, int j) { return ld4(A + kb + k + (size_t)(pe + j) * n); },
          [&](int i, int j) { return A + pe + i + (size_t)(pe + j) * n; }, sm);
      df_gemm_sub_tiled(
          m, nr, pe - kb, l21, [&](int k, int j) { return ld4(B + kb + k + (size_t)j * n); },
          [&](int i, int j) { return B + pe + i + (size_t)j * n; }, sm);
    }
  }
  // back substitution: B <- U^{-1} B by blocks from the last one
  const int nblk = (n + DF_LU_P - 1) / DF_LU_P;
  for (int blk = nblk - 1; blk >= 0; --blk) {
    const int kb = blk * DF_LU_P, pe = min(n, kb + DF_LU_P);
    for (int c = tid(); c < nr; c += nthr()) {
      float4* col = B + (size_t)c * n;
      df::c4 x[DF_LU_P];
#pragma unroll
      for (int r = 0; r < DF_LU_P; ++r) x[r] = kb + r < pe ? ld4(col + kb + r) : one;
#pragma unroll
      for (int r = DF_LU_P - 1; r >= 0; --r) {
        if (kb + r >= pe) continue;
#pragma unroll
        for (int q = r + 1; q < DF_LU_P; ++q)
          if (kb + q < pe) x[r] = df::cms(x[r], ld4(A + kb + r + (size_t)(kb + q) * n), x[q]);
        x[r] = c4mul(x[r], ld4(piv + kb + r));
      }
#pragma unroll
      for (int r = 0; r < DF_LU_P; ++r)
        if (kb + r < pe) st4(col + kb + r, x[r]);
    }
    __syncthreads();
    if (kb > 0)
      df_gemm_sub_tiled(
          kb, nr, pe - kb, [&](int i, int k) { return ld4(A + i + (size_t)(kb + k) * n); },
          [&](int k, int j) { return ld4(B + kb + k + (size_t)j * n); },
          [&](int i, int j) { return B + i + (size_t)j * n; }, sm);
  }
  __syncthreads();
}

// G_t at a block boundary from the left checkpoint (XL, TL, logDL) and the right one (XR, TR,
// logDR), FP64 column-major, in df.  H, Mb, Wb: n x n df scratch.  Gout: FP64 column-major.
// sm: shared memory for df_gemm_tiled.
__device__ inline void boundary_green_df(int n, const double2* XL, const double2* TL,
                                         const double* logDL, const double2* XR,
                                         const double2* TR, const double* logDR, float4* H,
                                         float4* Mb, float4* Wb, double2* Gout, Small& s,
                                         float4* sm) {
  for (int k = tid(); k < n; k += nthr()) {
    s.sa[k] = exp(-fmax(logDL[k], 0.0));
    s.sc[k] = exp(fmin(logDL[k], 0.0));
    s.sb[k] = exp(-fmax(logDR[k], 0.0));
    s.sd[k] = exp(fmin(logDR[k], 0.0));
  }
  // H = X_L^H in df (column k of H is row k of X_L, conjugated); the right-hand side
  // W = D_Lb^{-1} X_L^H
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n, k = e / n;
    st4(H + e, df_conj(df_of(XL[k + (size_t)i * n])));
  }
  __syncthreads();
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n;
    float sh, sl;
    df::split(s.sa[i], sh, sl);
    st4(Wb + e, df::scale(ld4(H + e), sh, sl));
  }
  // M = diag(a) X_L^H X_R diag(b)
  df_gemm_tiled(
      n, n, n, [&](int i, int k) { return ld4(H + i + (size_t)k * n); },
      [&](int k, int j) { return df_of(XR[k + (size_t)j * n]); },
      [&](int i, int j, df::c4 v) {
        float sh, sl;
        df::split(s.sa[i] * s.sb[j], sh, sl);
        st4(Mb + i + (size_t)j * n, df::scale(v, sh, sl));
      },
      sm);
  // M += diag(c) T_L T_R^H diag(d), as M -= (-diag(c) T_L) (T_R^H diag(d))
  df_gemm_sub_tiled(
      n, n, n,
      [&](int i, int k) {
        float sh, sl;
        df::split(-s.sc[i], sh, sl);
        return df::scale(df_of(TL[i + (size_t)k * n]), sh, sl);
      },
      [&](int k, int j) {
        float sh, sl;
        df::split(s.sd[j], sh, sl);
        return df::scale(df_conj(df_of(TR[j + (size_t)k * n])), sh, sl);
      },
      [&](int i, int j) { return Mb + i + (size_t)j * n; }, sm);
  // W <- M^{-1} W
  cta_lu_solve_blocked_df(n, Mb, Wb, n, s, sm);
  // G = X_R diag(b) W
  df_gemm_tiled(
      n, n, n, [&](int i, int k) { return df_of(XR[i + (size_t)k * n]); },
      [&](int k, int j) {
        float sh, sl;
        df::split(s.sb[k], sh, sl);
        return df::scale(ld4(Wb + k + (size_t)j * n), sh, sl);
      },
      [&](int i, int j, df::c4 v) {
        Gout[i + (size_t)j * n] = make_double2(df::join(v.x, v.y), df::join(v.z, v.w));
      },
      sm);
}


}  // namespace fd
