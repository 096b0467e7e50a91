// fd_fp64.cuh -- CTA-level FP64 building blocks of the stabilised method (Section 7).
//
// Every routine is executed by all threads of one CTA on one configuration.  Matrices are
// complex128 (double2), column-major with leading dimension n, addressed through generic
// pointers so that the same code runs on shared-memory or global (L2-resident) buffers.
// Contract: inputs are visible to every thread on entry (the caller synchronised), and each
// routine ends with __syncthreads() so that its outputs are visible on return.
#pragma once

#include "fd_common.cuh"

namespace fd {

__device__ __forceinline__ int nthr() { return blockDim.x; }
__device__ __forceinline__ int tid() { return threadIdx.x; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int nwarps() { return blockDim.x >> 5; }

__device__ __forceinline__ int seg_width(int rows) {
  int w = 1;
  while (w < rows && w < 32) w <<= 1;
  return w;
}

// xor-reduction inside aligned groups of W lanes (all 32 lanes must call it)
__device__ __forceinline__ double seg_sum(double v, int W) {
  for (int o = W >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- operand views
struct RealMat {  // element (i,k) = p[i*rs + k*cs]
  const double* p;
  int rs, cs;
  __device__ __forceinline__ double operator()(int i, int k) const { return p[i * rs + k * cs]; }
};
struct CMat {  // element (i,k) = p[i*rs + k*cs]
  const double2* p;
  int rs, cs;
  __device__ __forceinline__ cplx operator()(int i, int k) const { return ld(p + i * rs + k * cs); }
};
struct CMatH {  // element (i,k) = conj(p[k*rs + i*cs]) : conjugate transpose of a stored matrix
  const double2* p;
  int rs, cs;
  __device__ __forceinline__ cplx operator()(int i, int k) const {
    return conj(ld(p + k * rs + i * cs));
  }
};

__device__ __forceinline__ void mac(cplx& acc, double a, cplx b) {
  acc.re = fma(a, b.re, acc.re);
  acc.im = fma(a, b.im, acc.im);
}
__device__ __forceinline__ void mac(cplx& acc, cplx a, double b) {
  acc.re = fma(a.re, b, acc.re);
  acc.im = fma(a.im, b, acc.im);
}
__device__ __forceinline__ void mac(cplx& acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}

// Out(i,j) <- epi(i, j, sum_k A(i,k) B(k,j)), i,j in [0,n), with TM x TN register tiles;
// consecutive threads take consecutive row tiles.  If TRI, A is upper triangular (A(i,k) = 0 for
// k < i; its first TM - 1 columns are masked explicitly).  Out must not alias A or B.
template <int TM, int TN, bool TRI, class AOp, class BOp, class Epi>
__device__ __forceinline__ void gemm_tiles(int n, const AOp& A, const BOp& B, const Epi& epi) {
  const int tm = (n + TM - 1) / TM, tn = (n + TN - 1) / TN;
  const int ntiles = tm * tn;
  for (int tile = tid(); tile < ntiles; tile += nthr()) {
    // TRI: row-major tile order, so that the lanes of a warp span one or two tile rows and the
    // triangular k-loop (from i0) saves work for the whole warp; else column-major
    const int i0 = TRI ? (tile / tn) * TM : (tile % tm) * TM;
    const int j0 = TRI ? (tile % tn) * TN : (tile / tm) * TN;
    int ii[TM], jj[TN];
#pragma unroll
    for (int a = 0; a < TM; ++a) ii[a] = min(i0 + a, n - 1);
#pragma unroll
    for (int b = 0; b < TN; ++b) jj[b] = min(j0 + b, n - 1);
    cplx acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] = cx(0, 0);
    int k = TRI ? i0 : 0;
#pragma unroll 2
    for (; k < n; ++k) {
      decltype(A(0, 0)) av[TM];
      decltype(B(0, 0)) bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = A(ii[a], k);
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = B(k, jj[b]);
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) mac(acc[a][b], av[a], bv[b]);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b)
        if (i0 + a < n && j0 + b < n) epi(i0 + a, j0 + b, acc[a][b]);
  }
}

// CTA GEMM: picks the largest register tile that still gives every thread at least one tile
// (small matrices use 1x1 tiles so that all warps -- and all four FP64 pipes of the SM -- work).
template <bool TRI, class AOp, class BOp, class Epi>
__device__ void cta_gemm(int n, const AOp& A, const BOp& B, const Epi& epi) {
  const int t2 = ((n + 1) >> 1) * ((n + 1) >> 1);
  if (t2 >= nthr())
    gemm_tiles<2, 2, TRI>(n, A, B, epi);
  else if (((n + 1) >> 1) * n >= nthr())
    gemm_tiles<1, 2, TRI>(n, A, B, epi);
  else
    gemm_tiles<1, 1, TRI>(n, A, B, epi);
  __syncthreads();
}

// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ void cta_copy(int count, double2* dst, const double2* src) {
  for (int e = tid(); e < count; e += nthr()) dst[e] = src[e];
}
__device__ __forceinline__ void cta_identity(int n, double2* A) {
  for (int e = tid(); e < n * n; e += nthr()) {
    int i = e % n, j = e / n;
    A[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}
__device__ __forceinline__ void cta_load_real(int count, double* dst, const double* src) {
  for (int e = tid(); e < count; e += nthr()) dst[e] = src[e];
}
// phase vector e^{i s phi} of one slice (s = +1 or -1)
__device__ __forceinline__ void cta_phase(int n, double2* ph, const double* phi_row, double s) {
  for (int x = tid(); x < n; x += nthr()) {
    double sn, cs;
    sincos(phi_row[x], &sn, &cs);
    ph[x] = make_double2(cs, s * sn);
  }
}
// rows of A scaled by ph:  A(i,j) *= ph[i]
__device__ __forceinline__ void cta_scale_rows(int n, double2* A, const double2* ph) {
  for (int e = tid(); e < n * n; e += nthr()) {
    int i = e % n;
    st(A + e, ld(ph + i) * ld(A + e));
  }
}

// Per-CTA small vectors (shared memory)
struct Small {
  double2* ph;     // 2n  phase of the current / next slice
  double2* rdiag;  // n   diag R of the last QR
  double2* vbuf;   // 2n  reflector copies (Q formation)
  double* logD;    // n   log D of the left / forward product
  double* logDR;   // n   log D of the right product (force)
  double* logw;    // n   permuted weights during a QR
  double* tau;     // n
  double* key;     // n   pivot keys / row scales
  double* sa;      // n   scale vectors
  double* sb;      // n
  double* sc;      // n
  double* sd;      // n
  int* perm;       // n
  int* piv;        // n
  int* misc;       // 32 ints: [0] status bits, [1] swap parity, [2] pivot index, [4] scaled QR,
                   // [5] leader-warp offset, [6] throughput mode (several CTAs per SM)
  double* red;     // 64 doubles: cross-warp reductions
};

__device__ __forceinline__ Small carve_small(char* base, int n) {
  Small s;
  char* p = base;
  s.ph = (double2*)p;    p += 32 * n;
  s.rdiag = (double2*)p; p += 16 * n;
  s.vbuf = (double2*)p;  p += 32 * n;
  s.logD = (double*)p;   p += 8 * n;
  s.logDR = (double*)p;  p += 8 * n;
  s.logw = (double*)p;   p += 8 * n;
  s.tau = (double*)p;    p += 8 * n;
  s.key = (double*)p;    p += 8 * n;
  s.sa = (double*)p;     p += 8 * n;
  s.sb = (double*)p;     p += 8 * n;
  s.sc = (double*)p;     p += 8 * n;
  s.sd = (double*)p;     p += 8 * n;
  p += 8 * n;  // spare
  s.red = (double*)p;    p += 8 * 64;
  s.perm = (int*)p;      p += 4 * n;
  s.piv = (int*)p;       p += 4 * n;
  s.misc = (int*)p;
  return s;
}

// ---------------------------------------------------------------- fast FP64 reciprocal / rsqrt
// The FP64 pipe of this GPU runs at 1/64 of the FP32 rate, so the serial steps of the QR and LU
// use short sequences: an FP32 hardware estimate refined by two Newton-Raphson steps (quadratic
// convergence: ~23 -> ~46 -> full 53 bits).  Arguments outside the FP32 normal range take the
// plain IEEE operation.
__device__ __forceinline__ double rcp64(double x) {
  const float xf = (float)x;
  const float af = fabsf(xf);
  if (!(af > 1e-36f && af < 1e36f)) return 1.0 / x;
  double r = (double)__frcp_rn(xf);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ double rsqrt64(double x) {
  const float xf = (float)x;
  if (!(xf > 1e-36f && xf < 1e36f)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf(xf);
  const double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}
__device__ __forceinline__ double sqrt64(double x) { return x > 0.0 ? x * rsqrt64(x) : 0.0; }

// Natural log of a positive double as an FP32 ordering key: exponent from the bit pattern,
// FP32 log of the mantissa in [1, 2).
__device__ __forceinline__ float log_key(double a) {
  const int hi = __double2hiint(a), lo = __double2loint(a);
  const int ex = ((hi >> 20) & 0x7ff) - 1023;
  const double m = __hiloint2double((hi & 0x800fffff) | 0x3ff00000, lo);
  return logf((float)m) + 0.69314718f * (float)ex;
}

// Serial steps (a reflector, a pivot search) run on a "leader" warp that rotates with the step,
// offset per CTA (s.misc[5]), so that the serial work of consecutive steps -- and of CTAs that
// share an SM -- lands on different SM sub-partitions and their FP64 pipes.
struct Small;
__device__ __forceinline__ int leader_warp(int step, const int* misc) {
  const int nw = nwarps();
  return ((step + misc[5]) % nw + nw) % nw;
}

// Segment width W for `cols` independent column reductions over `rows` rows.  The SM's FP64 unit
// takes one warp-instruction per ~19 cycles whatever the number of active lanes, with 64 cycles
// of latency.  With one CTA on the SM (latency mode, tput = false) W minimises the FP64
// instructions of the busiest warp slot, (column groups per sub-partition) x (8 per
// row-iteration + 2 per reduction level + 2); with several CTAs sharing the unit (throughput
// mode) it minimises the total, (column groups) x (the same per-group count).  `slots`: warps
// that share the columns (at most one per sub-partition counts).
__device__ __forceinline__ int seg_width_cols(int rows, int cols, bool tput, int slots = 4) {
  slots = max(1, min(4, slots));
  int best_w = 32, best_c = 1 << 30;
  for (int W = 1, lg = 0; W <= 32; W <<= 1, ++lg) {
    const int S = 32 / W;
    const int warps = (cols + S - 1) / S;
    const int per_sp = tput ? warps : (warps + slots - 1) / slots;
    const int cost = per_sp * (8 * ((rows + W - 1) / W) + 2 * lg + 2);
    if (cost < best_c || (cost == best_c && W > best_w)) {
      best_c = cost;
      best_w = W;
    }
  }
  return best_w;
}

// Segment width for a reduction over `rows` rows: about four rows per lane, at most a warp.
__device__ __forceinline__ int seg_width4(int rows) {
  int w = 1;
  while (w * 4 < rows && w < 32) w <<= 1;
  return w;
}

// ---------------------------------------------------------------- Householder helpers
// Reflector of a column with leading entry x and sig = sum of |a_i|^2 below it:
// H = I - tau v v^H with v_k = 1, v_i = a_i / c (i > k), H a = alpha e_k,
//   alpha = -(x/|x|) nrm,  c = x - alpha = x (|x| + nrm) / |x|,  nrm = sqrt(|x|^2 + sig),
//   tau = 2 / (v^H v) = 1 + |x| / nrm,   1 / c = conj(x) / (|x| (|x| + nrm)).
// The dependent chain is kept short for the FP64 pipe (64-cycle latency per dependent
// operation on this GPU): 1/|x|, 1/nrm and 1/(|x| + nrm) are seeded in FP32 from one FP64->FP32
// conversion each and refined in FP64 by one third-order step of Householder's iteration
// (Householder, "The Numerical Treatment of a Single Nonlinear Equation", 1970):
//   1/sqrt(a): e = 1 - a y^2,  y <- y (1 + e/2 + 3e^2/8);   1/s: e = 1 - s y,  y <- y (1 + e + e^2),
// which takes the ~2^-22 FP32 seeds past FP64 precision.  Arguments outside the FP32 range take
// the plain IEEE operations.
struct Refl {
  cplx alpha, cinv;
  double tau;
  bool zero;  // the column is exactly zero (singular product)
};
__device__ __forceinline__ double rsqrt_step3(double a, double y) {
  const double t = a * y;
  const double e = fma(-t, y, 1.0);
  return fma(y, e * fma(e, 0.375, 0.5), y);
}
__device__ __forceinline__ Refl reflector_math(cplx x, double sig) {
  const double x2 = abs2(x);
  const double n2 = x2 + sig;
  const float x2f = (float)x2, n2f = (float)n2;
  Refl r;
  r.zero = false;
  if (x2f > 1e-36f && n2f < 1e36f) {
    const float rxf = rsqrtf(x2f), rnf = rsqrtf(n2f);
    const float icf = __frcp_rn(fmaf(x2f, rxf, n2f * rnf));
    const double rx = rsqrt_step3(x2, (double)rxf), rn = rsqrt_step3(n2, (double)rnf);
    const double ax = x2 * rx, nrm = n2 * rn;
    double ic = (double)icf;
    const double e = fma(-(ax + nrm), ic, 1.0);
    ic = fma(ic, fma(e, e, e), ic);
    const double cf = rx * ic, g = nrm * rx;
    r.cinv = cx(x.re * cf, -x.im * cf);
    r.alpha = cx(-x.re * g, -x.im * g);
    r.tau = fma(ax, rn, 1.0);
    return r;
  }
  if (!(n2 > 0.0)) {
    r.zero = true;
    r.alpha = cx(0, 0);
    r.cinv = cx(0, 0);
    r.tau = 0.0;
    return r;
  }
  const double nrm = sqrt(n2);
  if (x2 > 0.0) {
    const double ax = sqrt(x2);
    const double cf = 1.0 / (ax * (ax + nrm)), g = nrm / ax;
    r.cinv = cx(x.re * cf, -x.im * cf);
    r.alpha = cx(-x.re * g, -x.im * g);
    r.tau = 1.0 + ax / nrm;
  } else {
    r.cinv = cx(1.0 / nrm, 0.0);
    r.alpha = cx(-nrm, 0.0);
    r.tau = 1.0;
  }
  return r;
}

// Finish the reflector of column k inside one segment of W lanes (sl = lane in segment) given
// its sig and leading entry x (known to every lane of the segment): scale the rows below the
// diagonal by 1/c, store tau and R_kk = alpha.
__device__ __forceinline__ void seg_reflector_finish(int n, int k, double2* A, int W, int sl,
                                                     cplx x, double sig, Small& s) {
  if (k == n - 1) {
    if (sl == 0) {
      s.tau[k] = 0.0;
      st(s.rdiag + k, x);
    }
    return;
  }
  const Refl r = reflector_math(x, sig);
  if (r.zero) {
    if (sl == 0) {
      s.tau[k] = 0.0;
      st(s.rdiag + k, cx(0, 0));
      atomicOr(&s.misc[0], 1);
    }
    return;
  }
  for (int i = k + 1 + sl; i < n; i += W) st(A + i + k * n, ld(A + i + k * n) * r.cinv);
  if (sl == 0) {
    s.tau[k] = r.tau;
    st(s.rdiag + k, r.alpha);
  }
}

// Reflector for column k of A (rows k..n-1), computed by one segment of W lanes (all 32 lanes of
// the warp call this; only the owning segment's results are stored).  v (rows > k) overwrites A;
// rdiag[k] = alpha.
__device__ __forceinline__ void seg_reflector(int n, int k, double2* A, int W, int sl, bool owner,
                                              Small& s) {
  double sa = 0.0, sb = 0.0;
  if (owner)
    for (int i = k + 1 + sl; i < n; i += W) {
      const cplx a = ld(A + i + k * n);
      sa = fma(a.re, a.re, sa);
      sb = fma(a.im, a.im, sb);
    }
  const double sig = seg_sum(sa + sb, W);
  if (!owner) return;
  seg_reflector_finish(n, k, A, W, sl, ld(A + k + k * n), sig, s);
}

// One warp's share of a Householder step: apply H_k = I - tau v v^H (v_k = 1, v_i = A(i,k) below
// the diagonal, rows k..n-1) to the columns j = base + lane/W, base = b0, b0 + bstep, ... < n,
// segments of W lanes per column.  If build_next, the segment that owns column k+1 (base b0 =
// k+1, first segment) accumulates that column's norm below row k+1 while it updates it and then
// builds the reflector of column k+1 without another pass.
__device__ __forceinline__ void hh_columns(int n, int k, double2* A, Small& s, int W, int b0,
                                           int bstep, bool build_next, bool tput) {
  const int lane = lane_id();
  const int sl = lane % W;
  const double tk = s.tau[k];
  for (int base = b0; base < n; base += bstep) {
    const int j = base + lane / W;
    const bool act = j < n;
    // two accumulators per component in latency mode (half the dependent chain), one in
    // throughput mode (two FP64 instructions fewer per column group)
    double sr0 = 0.0, sr1 = 0.0, si0 = 0.0, si1 = 0.0;
    if (act) {
      if (tput) {
        for (int i = k + sl; i < n; i += W) {
          const cplx v = (i == k) ? cx(1.0, 0.0) : ld(A + i + k * n);
          const cplx a = ld(A + i + j * n);
          sr0 = fma(v.re, a.re, sr0);
          sr0 = fma(v.im, a.im, sr0);
          si0 = fma(v.re, a.im, si0);
          si0 = fma(-v.im, a.re, si0);
        }
      } else {
        for (int i = k + sl; i < n; i += W) {
          const cplx v = (i == k) ? cx(1.0, 0.0) : ld(A + i + k * n);
          const cplx a = ld(A + i + j * n);
          sr0 = fma(v.re, a.re, sr0);
          sr1 = fma(v.im, a.im, sr1);
          si0 = fma(v.re, a.im, si0);
          si1 = fma(-v.im, a.re, si1);
        }
      }
    }
    const double sr = seg_sum(tput ? sr0 : sr0 + sr1, W);
    const double si = seg_sum(tput ? si0 : si0 + si1, W);
    const bool first = build_next && base == b0;  // warp-uniform
    const bool mine = first && j == k + 1;        // this segment builds the next reflector
    double sg0 = 0.0, sg1 = 0.0;
    cplx xn = cx(0.0, 0.0);
    if (act) {
      const cplx f = cx(tk * sr, tk * si);
      for (int i = k + sl; i < n; i += W) {
        const cplx v = (i == k) ? cx(1.0, 0.0) : ld(A + i + k * n);
        const cplx a = cfms(ld(A + i + j * n), f, v);
        st(A + i + j * n, a);
        if (mine) {
          if (i > k + 1) {
            sg0 = fma(a.re, a.re, sg0);
            sg1 = fma(a.im, a.im, sg1);
          } else if (i == k + 1) {
            xn = a;
          }
        }
      }
    }
    if (first) {
      const double sig = seg_sum(sg0 + sg1, W);
      // x = new A(k+1, k+1), held by the lane of the segment that owns row k+1
      const int src = (lane & ~(W - 1)) + (1 % W);
      xn.re = __shfl_sync(0xffffffffu, xn.re, src);
      xn.im = __shfl_sync(0xffffffffu, xn.im, src);
      __syncwarp();
      if (lane < W) seg_reflector_finish(n, k + 1, A, W, sl, xn, sig, s);
    }
  }
}

// Householder step k on the CTA.  The serial reflector of column k+1 is the critical path of
// the factorisation, so the warp that builds it (the step's leader) only updates the first few
// columns, with wide segments (short dependent chains); the other warps share the remaining
// columns with the segment width of seg_width_cols.
__device__ __forceinline__ void householder_step(int n, int k, double2* A, Small& s,
                                                 bool next_reflector) {
  const int w = warp_id(), NW = nwarps();
  const bool tput = s.misc[6] != 0;
  const int rows = n - k, cols = n - k - 1;
  const int lead = leader_warp(k + 1, s.misc);
  if (NW == 1) {
    const int W = seg_width_cols(rows, cols, tput);
    hh_columns(n, k, A, s, W, k + 1, 32 / W, next_reflector, tput);
    return;
  }
  int W1 = 32;  // smallest power of two with at most two rows per lane
  while (W1 > 1 && 2 * (W1 / 2) >= rows) W1 >>= 1;
  const int S1 = 32 / W1;
  if (w == lead) {
    hh_columns(n, k, A, s, W1, k + 1, n, next_reflector, tput);  // one round: k+1 .. k+S1
    return;
  }
  const int rest = cols - S1;
  if (rest <= 0) return;
  const int others = NW - 1;
  const int slot = (w - lead - 1 + NW) % NW;  // 0 .. others-1
  const int W = seg_width_cols(rows, rest, tput, others);
  const int spw = 32 / W;
  hh_columns(n, k, A, s, W, k + 1 + S1 + slot * spw, others * spw, false, tput);
}

// ---------------------------------------------------------------- QR re-orthogonalisation
// One stabilisation step (Eqs. prod_2_mat_stab .. res_2_mat_stab with the QR every n_stab
// slices of Section 9):  the current product is Xc diag(e^{logD}) Tc where Xc already carries
// the latest slices.  Householder QR of Z = Xc diag(D) with the columns pre-sorted by
// ||z_j|| = e^{logD_j} ||xc_j|| (pre-pivoting; the column scaling itself is never formed, since
// a Householder QR is invariant under it: QR(Y D Pi) = Q R_Y (Pi^T D Pi)).
// Result: Xn = Q, logD_k = log|R_kk| + logD_{pi(k)},
//         Tn = diag(D')^{-1} R Pi^T Tc  with coefficients R'_kj e^{logw_j - logw_k} / |R'_kk|.
__device__ inline void cta_reortho(int n, const double2* Xc, double2* Xn, const double2* Tc,
                                   double2* Tn, double* logD, Small& s) {
  const int lane = lane_id(), w = warp_id(), NW = nwarps();
  float* keyf = (float*)s.key;
  // 1. pivot keys (FP32 ordering keys: the pre-pivot order only has to be approximately sorted)
  {
    const int W0 = seg_width_cols(n, n, s.misc[6] != 0, NW);
    const int spw0 = 32 / W0;
    for (int base = w * spw0; base < n; base += NW * spw0) {
      const int j = base + lane / W0;
      const int sl = lane % W0;
      double a = 0.0;
      if (j < n)
        for (int i = sl; i < n; i += W0) a += abs2(ld(Xc + i + j * n));
      a = seg_sum(a, W0);
      if (j < n && sl == 0) {
        float kk = (float)logD[j] + 0.5f * log_key(a);
        if (!(a == a) || !(kk == kk)) {  // NaN
          kk = -INFINITY;
          atomicOr(&s.misc[0], 1);
        }
        keyf[j] = kk;
      }
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
  // 3. gather columns; column-scale factors sc_k = e^{logw_k - m} (m = mid-range) when the
  //    range of log D fits FP64 (|logw - m| < 600), else the per-element form below
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n, k = e / n;
    Xn[e] = Xc[i + s.perm[k] * n];
  }
  for (int k = tid(); k < n; k += nthr()) s.logw[k] = logD[s.perm[k]];
  if (w == 0) {
    double lo = INFINITY, hi = -INFINITY;
    for (int k = lane; k < n; k += 32) {
      const double v = logD[k];
      lo = fmin(lo, v);
      hi = fmax(hi, v);
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
  const bool scaled = s.misc[4] != 0;
  // 4. Householder factorisation, one barrier per column
  if (w == leader_warp(0, s.misc))
    seg_reflector(n, 0, Xn, seg_width4(n), lane % seg_width4(n), lane < seg_width4(n), s);
  __syncthreads();
  for (int k = 0; k < n - 1; ++k) {
    householder_step(n, k, Xn, s, true);
    __syncthreads();
  }
  // 5. new log D, the row factors q_k = 1 / (sc_k |R_kk|), and the T-update coefficients
  //    C_kj = R'_kj sc_j q_k (j > k), C_kk = R_kk / |R_kk| (in place in the upper triangle)
  for (int k = tid(); k < n; k += nthr()) {
    const double r2 = abs2(ld(s.rdiag + k));
    if (!(r2 > 0.0)) atomicOr(&s.misc[0], 1);
    const double ir = rsqrt64(r2);  // 1 / |R_kk|
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
    } else if (scaled) {
      c = s.sb[k] * (s.sa[j] * ld(Xn + e));
    } else {
      const cplx rkj = ld(Xn + e);
      const double ex = s.logw[j] - s.logw[k];
      const double m = sqrt64(abs2(rkj));
      c = m == 0.0 ? cx(0, 0) : (exp(log(m) + ex) * s.sb[k] * rcp64(m)) * rkj;
    }
    st(Xn + e, c);
  }
  __syncthreads();
  // 6. Tn = C (Pi^T Tc), C upper triangular
  {
    const int* perm = s.perm;
    struct CUp {
      const double2* p;
      int n;
      __device__ __forceinline__ cplx operator()(int i, int k) const {
        return k >= i ? ld(p + i + k * n) : cx(0, 0);
      }
    } Cop{Xn, n};
    struct TP {
      const double2* p;
      const int* perm;
      int n;
      __device__ __forceinline__ cplx operator()(int k, int c) const {
        return ld(p + perm[k] + c * n);
      }
    } Top{Tc, perm, n};
    cta_gemm<true>(n, Cop, Top, [&](int i, int j, cplx v) { st(Tn + i + j * n, v); });
  }
  // 7. form Q in place: Q = H_0 H_1 ... H_{n-2}, accumulated backwards
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n, j = e / n;
    if (i < j) Xn[e] = make_double2(0.0, 0.0);
    if (i == n - 1 && j == n - 1) Xn[e] = make_double2(1.0, 0.0);
  }
  if (n >= 2)  // copy v_{n-2} (rows > n-2) to vbuf[(n-2)&1]
    for (int i = n - 1 + tid(); i < n; i += nthr())
      s.vbuf[((n - 2) & 1) * n + i] = Xn[i + (n - 2) * n];
  __syncthreads();
  for (int k = n - 2; k >= 0; --k) {
    const int W = seg_width_cols(n - k, n - k, s.misc[6] != 0, NW);
    const int spw = 32 / W;
    const int sl = lane % W;
    const double tk = s.tau[k];
    const double2* vk = s.vbuf + (k & 1) * n;
    const int slot0 = (w - leader_warp(k, s.misc) + NW) % NW;
    for (int base = k + slot0 * spw; base < n; base += NW * spw) {
      const int j = base + lane / W;
      const bool act = j < n && j > k;
      double sr = 0.0, si = 0.0;
      if (act)
        for (int i = k + 1 + sl; i < n; i += W) {
          const cplx v = ld(vk + i), a = ld(Xn + i + j * n);
          sr = fma(v.re, a.re, sr);
          sr = fma(v.im, a.im, sr);
          si = fma(v.re, a.im, si);
          si = fma(-v.im, a.re, si);
        }
      sr = seg_sum(sr, W);
      si = seg_sum(si, W);
      if (act) {
        const cplx f = cx(tk * sr, tk * si);
        if (sl == 0) st(Xn + k + j * n, cx(-f.re, -f.im));
        for (int i = k + 1 + sl; i < n; i += W) st(Xn + i + j * n, cfms(ld(Xn + i + j * n), f, ld(vk + i)));
      }
      if (j == k) {  // this segment sets column k and copies v_{k-1}
        if (sl == 0) Xn[k + k * n] = make_double2(1.0 - tk, 0.0);
        for (int i = k + 1 + sl; i < n; i += W) st(Xn + i + k * n, cx(-tk, 0.0) * ld(vk + i));
        if (k >= 1)
          for (int i = k + sl; i < n; i += W) s.vbuf[((k - 1) & 1) * n + i] = Xn[i + (k - 1) * n];
      }
    }
    __syncthreads();
  }
  if (n == 1) {
    if (tid() == 0) Xn[0] = make_double2(1.0, 0.0);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- LU with partial pivoting
// Factor A in place (A = P^T L U, unit L), applying the same row operations to the n columns of
// Bm (so that Bm <- L^{-1} P Bm), then back-substitute Bm <- U^{-1} Bm.  On return Bm holds
// A^{-1} Bm_in and *logdet_out = log det A (principal logs of the pivots + i pi * swaps).
// Pivot search on FP32 magnitudes (partial pivoting only needs an approximately largest pivot);
// one complex reciprocal per pivot; back substitution with the columns of U pre-scaled by the
// reciprocal pivots, one barrier per step, rows scaled at the end.
__device__ inline void cta_lu_solve(int n, double2* A, double2* Bm, Small& s, double* logdet_re,
                                    double* logdet_im, int ncols = -1) {
  if (ncols < 0) ncols = n;  // right-hand sides: Bm is n x ncols, leading dimension n
  const int lane = lane_id(), w = warp_id();
  if (tid() == 0) s.misc[1] = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (w == leader_warp(k, s.misc)) {
      float best = -1.f;
      int bi = k;
      for (int i = k + lane; i < n; i += 32) {
        const float m = (float)abs2(ld(A + i + k * n));
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
      const int p = bi;
      if (p != k) {
        for (int j = lane; j < n; j += 32) {
          double2 t = A[k + j * n];
          A[k + j * n] = A[p + j * n];
          A[p + j * n] = t;
        }
        for (int j = lane; j < ncols; j += 32) {
          double2 t = Bm[k + j * n];
          Bm[k + j * n] = Bm[p + j * n];
          Bm[p + j * n] = t;
        }
        if (lane == 0) s.misc[1] ^= 1;
      }
      __syncwarp();
      cplx piv = ld(A + k + k * n);
      double p2 = abs2(piv);
      if (!(p2 > 0.0)) {  // singular: flagged; continue with a unit pivot
        if (lane == 0) atomicOr(&s.misc[0], 1);
        piv = cx(1.0, 0.0);
        p2 = 1.0;
      }
      const double ip2 = rcp64(p2);
      const cplx pinv = cx(piv.re * ip2, -piv.im * ip2);
      if (lane == 0) st(s.rdiag + k, pinv);
      for (int i = k + 1 + lane; i < n; i += 32) st(A + i + k * n, ld(A + i + k * n) * pinv);
    }
    __syncthreads();
    // trailing update of A (columns k+1..n-1) and of all columns of Bm, rows k+1..n-1
    const int m = n - k - 1;
    const int cols = m + ncols;
    for (int e = tid(); e < m * cols; e += nthr()) {
      const int i = k + 1 + e % m;
      const int c = e / m;
      const cplx l = ld(A + i + k * n);
      if (c < m) {
        const int j = k + 1 + c;
        st(A + i + j * n, cfms(ld(A + i + j * n), l, ld(A + k + j * n)));
      } else {
        const int j = c - m;
        st(Bm + i + j * n, cfms(ld(Bm + i + j * n), l, ld(Bm + k + j * n)));
      }
    }
    __syncthreads();
  }
  // log det A, and U's strict upper part pre-scaled by the pivot reciprocals: W(i,k) = U(i,k)/U(k,k)
  if (w == 0) {
    double lr = 0.0, li = 0.0;
    for (int k = lane; k < n; k += 32) {
      const cplx u = ld(A + k + k * n);
      lr += 0.5 * log(abs2(u));
      li += atan2(u.im, u.re);
    }
    lr = seg_sum(lr, 32);
    li = seg_sum(li, 32);
    if (lane == 0) {
      *logdet_re = lr;
      *logdet_im = li + (s.misc[1] ? 3.14159265358979323846 : 0.0);
    }
  }
  for (int e = tid(); e < n * n; e += nthr()) {
    const int i = e % n, k = e / n;
    if (i < k) st(A + e, ld(A + e) * ld(s.rdiag + k));
  }
  __syncthreads();
  // back substitution, unscaled rows: B(i,:) -= W(i,k) B(k,:) for i < k, then B(k,:) /= U(k,k)
  for (int k = n - 1; k >= 1; --k) {
    for (int e = tid(); e < k * ncols; e += nthr()) {
      const int i = e % k, j = e / k;
      st(Bm + i + j * n, cfms(ld(Bm + i + j * n), ld(A + i + k * n), ld(Bm + k + j * n)));
    }
    __syncthreads();
  }
  for (int e = tid(); e < n * ncols; e += nthr()) {
    const int i = e % n;
    st(Bm + e, ld(Bm + e) * ld(s.rdiag + i));
  }
  __syncthreads();
}

// ---------------------------------------------------------------- assembly (Section 7)
// With D = D_b D_s, D_b = max(D,1), D_s = min(D,1):
//   1 + X D T = X D_b C,  C = D_b^{-1} X^H + D_s T,
//   log det(1 + X D T) = log det X + sum log D_b + log det C,  G = C^{-1} D_b^{-1} X^H.
// X is the Q of the last QR (product of n-1 reflections): det X = (-1)^{n-1}.
// Cbuf and Gbuf are scratch; on return Gbuf holds G (column-major).
__device__ inline void cta_assemble(int n, const double2* X, const double2* T, const double* logD,
                             double2* Cbuf, double2* Gbuf, Small& s, double* ld_re,
                             double* ld_im) {
  for (int e = tid(); e < n * n; e += nthr()) {
    int i = e % n, j = e / n;
    double lb = fmax(logD[i], 0.0);
    double ls = fmin(logD[i], 0.0);
    double ib = exp(-lb), ds = exp(ls);
    cplx xh = conj(ld(X + j + i * n));
    cplx r = ib * xh;
    st(Gbuf + e, r);
    st(Cbuf + e, r + ds * ld(T + e));
  }
  __syncthreads();
  double cre = 0.0, cim = 0.0;
  cta_lu_solve(n, Cbuf, Gbuf, s, s.red + 0, s.red + 1);
  if (warp_id() == 0) {
    double sb = 0.0;
    for (int k = lane_id(); k < n; k += 32) sb += fmax(logD[k], 0.0);
    sb = seg_sum(sb, 32);
    if (lane_id() == 0) {
      cre = s.red[0] + sb;
      cim = s.red[1] + ((n - 1) & 1 ? 3.14159265358979323846 : 0.0);
      *ld_re = cre;
      *ld_im = cim;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- force building blocks
// Equal-time Green's function at a block boundary (Section 7 steps 7-9 with t1 = t2, combined
// with the stabilised pre-/suffix products of Section 5.3):
//   L = X_L diag(D_L) T_L = B_t...B_1,   R = (X_R diag(D_R) T_R)^H = B_Nt...B_{t+1},
//   1 + L R = X_L D_Lb [ D_Lb^{-1} X_L^H X_R D_Rb^{-1} + D_Ls T_L T_R^H D_Rs ] D_Rb X_R^H,
//   G_t = X_R D_Rb^{-1} M^{-1} D_Lb^{-1} X_L^H.
// identity_left: L = 1 (t = 0).  Scratch: Mb, Wb.  Result in Gout.
// With Gt_out (and a Wb of 2n columns) it also gives the unequal-time Green's function
// G(t, 0) = (L^{-1} + R)^{-1} (Section 4.2) from the same factored M:
//   L^{-1} + R = T_L^{-1} D_Ls^{-1} M D_Rb X_R^H  =>  G(t, 0) = X_R D_Rb^{-1} M^{-1} D_Ls T_L.
// Gout or Gt_out may be null (not wanted).
__device__ inline void boundary_green(int n, bool identity_left, const double2* XL, const double2* TL,
                               const double* logDL, const double2* XR, const double2* TR,
                               const double* logDR, double2* Mb, double2* Wb, double2* Gout,
                               Small& s, double2* Gt_out = nullptr) {
  for (int k = tid(); k < n; k += nthr()) {
    double lL = identity_left ? 0.0 : logDL[k];
    double lR = logDR[k];
    s.sa[k] = exp(-fmax(lL, 0.0));
    s.sc[k] = exp(fmin(lL, 0.0));
    s.sb[k] = exp(-fmax(lR, 0.0));
    s.sd[k] = exp(fmin(lR, 0.0));
  }
  __syncthreads();
  const double *a = s.sa, *b = s.sb, *c = s.sc, *dd = s.sd;
  if (identity_left) {
    // M = X_R D_Rb^{-1} + T_R^H D_Rs ;  RHS = 1
    for (int e = tid(); e < n * n; e += nthr()) {
      int i = e % n, j = e / n;
      cplx m = b[j] * ld(XR + e) + dd[j] * conj(ld(TR + j + i * n));
      st(Mb + e, m);
      if (Gout) Wb[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      if (Gt_out) Wb[(Gout ? n * n : 0) + e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
  } else {
    cta_gemm<false>(n, CMatH{XL, 1, n}, CMat{XR, 1, n},
                    [&](int i, int j, cplx v) { st(Mb + i + j * n, (a[i] * b[j]) * v); });
    cta_gemm<false>(n, CMat{TL, 1, n}, CMatH{TR, 1, n}, [&](int i, int j, cplx v) {
      st(Mb + i + j * n, ld(Mb + i + j * n) + (c[i] * dd[j]) * v);
    });
    for (int e = tid(); e < n * n; e += nthr()) {
      int i = e % n, j = e / n;
      if (Gout) st(Wb + e, a[i] * conj(ld(XL + j + i * n)));
      if (Gt_out) st(Wb + (Gout ? n * n : 0) + e, c[i] * ld(TL + e));
    }
    __syncthreads();
  }
  const int nr = (Gout ? n : 0) + (Gt_out ? n : 0);
  cta_lu_solve(n, Mb, Wb, s, s.red + 4, s.red + 5, nr);
  // Gout = X_R diag(b) W
  struct BW {
    const double2* p;
    const double* b;
    int n;
    __device__ __forceinline__ cplx operator()(int k, int j) const { return b[k] * ld(p + k + j * n); }
  };
  if (Gout) {
    BW Bop{Wb, b, n};
    cta_gemm<false>(n, CMat{XR, 1, n}, Bop, [&](int i, int j, cplx v) { st(Gout + i + j * n, v); });
  }
  if (Gt_out) {
    BW Bop{Wb + (Gout ? n * n : 0), b, n};
    cta_gemm<false>(n, CMat{XR, 1, n}, Bop,
                    [&](int i, int j, cplx v) { st(Gt_out + i + j * n, v); });
  }
}

// tr(O G) for O row-major and G column-major: both store (x, y) of O and (y, x) of G at x n + y,
// so the trace is the element-wise product summed.  red: 2 doubles per warp of scratch.
__device__ inline void cta_trace(int n, const double* O, const double2* G, double2* out,
                                 double* red) {
  double re = 0.0, im = 0.0;
  for (int e = tid(); e < n * n; e += nthr()) {
    const double o = O[e];
    const double2 g = G[e];
    re = fma(o, g.x, re);
    im = fma(o, g.y, im);
  }
  re = seg_sum(re, 32);
  im = seg_sum(im, 32);
  if (lane_id() == 0) {
    red[2 * warp_id()] = re;
    red[2 * warp_id() + 1] = im;
  }
  __syncthreads();
  if (tid() == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nwarps(); ++w) {
      a += red[2 * w];
      b += red[2 * w + 1];
    }
    *out = make_double2(a, b);
  }
  __syncthreads();
}

// Fermion number n = 1 - tr G / nx (Section 4.1, Eq. fermion_number); G column-major.
__device__ inline void cta_fermion_number(int n, const double2* G, double* out) {
  if (warp_id() == 0) {
    double re = 0.0, im = 0.0;
    for (int x = lane_id(); x < n; x += 32) {
      re += G[x + x * n].x;
      im += G[x + x * n].y;
    }
    re = seg_sum(re, 32);
    im = seg_sum(im, 32);
    if (lane_id() == 0) {
      out[0] = 1.0 - re / n;
      out[1] = -im / n;
    }
  }
}

__device__ __forceinline__ void emit_force_row(int n, const double2* G, double2* Frow) {
  // F[t,x] = i (1 - G_xx) = (Im G_xx, 1 - Re G_xx)
  for (int x = tid(); x < n; x += nthr()) {
    double2 g = G[x + x * n];
    Frow[x] = make_double2(g.y, 1.0 - g.x);
  }
}

__device__ __forceinline__ double wrap_pi(double x) {
  const double pi = 3.14159265358979323846;
  double y = remainder(x, 2.0 * pi);  // (-pi, pi]
  if (y <= -pi) y += 2.0 * pi;
  return y;
}

// ---------------------------------------------------------------- product of two UDV factors
// Section 7's stabilised product of two factored matrices, Xs Ds Ts (acting later) times
// Xa Da Ta:  Xs Ds Ts Xa Da Ta = Xs [Ds Ts Xa] Da Ta  with  Xc = e^{-m} Ds (Ts Xa),
// m = max log Ds, re-factored by the pre-pivoted QR (Xc Da Ta = Q D' T'), so that
// X = Xs Q, log D = log D' + m, T = T'.  The row scaling e^{log Ds - m} is formed: a factor whose
// log D spans more than 700 marks the configuration (misc[0]) instead of losing rows silently.
// X = Xs Q is a product of two Householder products (det X = +1).  Scratch: Xc, Q (n^2 each);
// X, T, logD receive the result (X may alias Xa, logD may alias lDa; T may not alias Ta).
__device__ inline void cta_merge(int n, const double2* Xs, const double2* Ts, const double* lDs,
                                 const double2* Xa, const double2* Ta, const double* lDa,
                                 double2* Xc, double2* Q, double2* X, double2* T, double* logD,
                                 Small& s) {
  if (warp_id() == 0) {
    double mx = -INFINITY;
    for (int k = lane_id(); k < n; k += 32) mx = fmax(mx, lDs[k]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane_id() == 0) s.red[9] = mx;
  }
  __syncthreads();
  const double m = s.red[9];
  for (int k = tid(); k < n; k += nthr()) {
    const double e = lDs[k] - m;
    if (e < -700.0) atomicOr(&s.misc[0], 1);  // the row scaling would underflow
    s.sa[k] = exp(e);
    logD[k] = lDa[k];
  }
  __syncthreads();
  const double* sa = s.sa;
  cta_gemm<false>(n, CMat{Ts, 1, n}, CMat{Xa, 1, n},
                  [&](int i, int j, cplx v) { st(Xc + i + j * n, sa[i] * v); });
  cta_reortho(n, Xc, Q, Ta, T, logD, s);
  for (int k = tid(); k < n; k += nthr()) logD[k] += m;
  cta_gemm<false>(n, CMat{Xs, 1, n}, CMat{Q, 1, n},
                  [&](int i, int j, cplx v) { st(X + i + j * n, v); });
  __syncthreads();
}

}  // namespace fd
