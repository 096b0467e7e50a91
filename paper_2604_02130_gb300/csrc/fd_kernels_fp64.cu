// fd_kernels_fp64.cu -- persistent per-configuration kernels of the FP64 path.
//
// One CTA owns one configuration at a time and pulls the next one from a cost-sorted queue
// (longest first).  The working matrices live in shared memory when the layout planner found
// room, else in the configuration's global scratch (L2-resident); see Layout.
#include "fd_fp64.cuh"
#include "fd_kernels.h"

namespace fd {

struct Bufs {
  double* E;
  double* Einv;
  double2* X[2];
  double2* T[2];
  double2 *Glo, *Ghi, *Ga, *Gb;
};

__device__ __forceinline__ void* place(char* smem, char* slot, const Layout& L, int b) {
  return L.in_smem[b] ? (void*)(smem + L.off[b]) : (void*)(slot + L.off[b]);
}

__device__ Bufs setup_bufs(char* smem, char* slot, const Desc& d, const Layout& L, bool force) {
  Bufs B;
  const int n = d.nx;
  B.E = L.in_smem[B_E] ? (double*)(smem + L.off[B_E]) : (double*)d.E;
  B.Einv = (force && L.in_smem[B_EINV]) ? (double*)(smem + L.off[B_EINV]) : (double*)d.Einv;
  if (L.in_smem[B_E]) cta_load_real(n * n, B.E, d.E);
  if (force && L.in_smem[B_EINV]) cta_load_real(n * n, B.Einv, d.Einv);
  B.X[0] = (double2*)place(smem, slot, L, B_X0);
  B.X[1] = (double2*)place(smem, slot, L, B_X1);
  B.T[0] = (double2*)place(smem, slot, L, B_T0);
  B.T[1] = (double2*)place(smem, slot, L, B_T1);
  if (force) {
    B.Glo = (double2*)place(smem, slot, L, B_GLO);
    B.Ghi = (double2*)place(smem, slot, L, B_GHI);
    B.Ga = (double2*)place(smem, slot, L, B_GA);
    B.Gb = (double2*)place(smem, slot, L, B_GB);
  } else {
    B.Glo = B.Ghi = B.Ga = B.Gb = nullptr;
  }
  return B;
}

// Apply slices s_begin..s_end-1 (0-based rows of phi) of the forward product to X:
// X <- B_s X = E diag(e^{i phi_s}) X.  The phase of the next slice is fused into the epilogue.
__device__ void fwd_slices(int n, const double* E, const double* phi, int s_begin, int s_end,
                           double2*& X, double2*& Xo, Small& s) {
  cta_phase(n, s.ph, phi + (size_t)s_begin * n, 1.0);
  __syncthreads();
  cta_scale_rows(n, X, s.ph);
  __syncthreads();
  for (int t = s_begin; t < s_end; ++t) {
    const bool has_next = t + 1 < s_end;
    double2* phn = s.ph + ((t - s_begin + 1) & 1) * n;
    if (has_next) cta_phase(n, phn, phi + (size_t)(t + 1) * n, 1.0);
    __syncthreads();
    double2* out = Xo;
    if (has_next)
      cta_gemm<false>(n, RealMat{E, 1, n}, CMat{X, 1, n},
                      [&](int i, int j, cplx v) { st(out + i + j * n, ld(phn + i) * v); });
    else
      cta_gemm<false>(n, RealMat{E, 1, n}, CMat{X, 1, n},
                      [&](int i, int j, cplx v) { st(out + i + j * n, v); });
    double2* tmp = X;
    X = Xo;
    Xo = tmp;
  }
}

// Intermediate-volume variant (Sections 8-9): slices s_begin..s_end-1 applied as
// X <- prod_k (1 + gamma_k K) diag(e^{i phi_s}) X, one pass over X per factor (the field phase is
// folded into the first pass), K applied matrix-free from its q entries per row: O(n q nx^2)
// per slice instead of the dense 4 nx^3.  A column index outside [0, nx) marks the
// configuration FD_ERR_NUMERIC and is skipped.
__device__ void fwd_slices_sparse(int n, const SparseHop* hop, const double* phi, int s_begin,
                                  int s_end, double2*& X, double2*& Xo, Small& s) {
  const int q = hop->q, nfac = hop->nfac;
  const int* __restrict__ col = hop->col;
  const double* __restrict__ val = hop->val;
  for (int t = s_begin; t < s_end; ++t) {
    cta_phase(n, s.ph, phi + (size_t)t * n, 1.0);
    __syncthreads();
    for (int k = 0; k < nfac; ++k) {
      const double2 g = hop->gamma[k];
      const bool first = k == 0;
      for (int e = tid(); e < n * n; e += nthr()) {
        const int i = e % n, base = e - i;  // column-major: element (i, j) at i + j n
        double ar = 0.0, ai = 0.0;
        for (int m = 0; m < q; ++m) {
          const int c = __ldg(col + i * q + m);
          const double v = __ldg(val + i * q + m);
          if ((unsigned)c >= (unsigned)n) {  // a column outside the matrix: flag, skip
            s.misc[0] = 1;
            continue;
          }
          cplx x = ld(X + base + c);
          if (first) x = ld(s.ph + c) * x;
          ar = fma(v, x.re, ar);
          ai = fma(v, x.im, ai);
        }
        cplx y = ld(X + e);
        if (first) y = ld(s.ph + i) * y;
        Xo[e] = make_double2(fma(g.x, ar, fma(-g.y, ai, y.re)), fma(g.x, ai, fma(g.y, ar, y.im)));
      }
      __syncthreads();
      double2* tmp = X;
      X = Xo;
      Xo = tmp;
    }
  }
}

// Right (backward) product as its adjoint: X <- B_s^H X = diag(e^{-i phi_s}) E X for
// s = s_hi-1 down to s_lo (0-based rows of phi).
__device__ void bwd_slices(int n, const double* E, const double* phi, int s_lo, int s_hi,
                           double2*& X, double2*& Xo, Small& s) {
  for (int t = s_hi - 1; t >= s_lo; --t) {
    cta_phase(n, s.ph, phi + (size_t)t * n, -1.0);
    __syncthreads();
    double2* out = Xo;
    const double2* ph = s.ph;
    cta_gemm<false>(n, RealMat{E, 1, n}, CMat{X, 1, n},
                    [&](int i, int j, cplx v) { st(out + i + j * n, ld(ph + i) * v); });
    double2* tmp = X;
    X = Xo;
    Xo = tmp;
  }
}

__device__ __forceinline__ int grab(int* queue, int* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = atomicAdd(queue, 1);
  __syncthreads();
  return *slot;
}

__device__ void write_green(int n, const double2* Gcol, double2* out) {
  for (int e = tid(); e < n * n; e += nthr()) {
    int i = e / n, j = e % n;  // row-major output
    out[e] = Gcol[i + j * n];
  }
}

__device__ void finish_status(const Desc& d, Small& s, int* status, double re, double im) {
  if (tid() == 0) {
    status[d.user_index] = (s.misc[0] || !isfinite(re) || !isfinite(im)) ? ST_NUMERIC : ST_OK;
  }
}

// ------------------------------------------------------------------ log det and G
__global__ void __launch_bounds__(256) k_fwd_fp64(const Desc* __restrict__ descs, int ndesc,
                                                   int* queue, int* status, char* scratch,
                                                   Layout L, const SparseHop* __restrict__ hops) {
  extern __shared__ __align__(16) char smem[];
  char* slotp = scratch + (size_t)blockIdx.x * L.slot_bytes;
  for (;;) {
    int* slot = (int*)(smem + L.smem_bytes - 16);
    int c = grab(queue, slot);
    if (c >= ndesc) return;
    const Desc d = descs[c];
    const int n = d.nx;
    Small s = carve_small(smem + L.small_off, n);
    if (tid() == 0) {
      s.misc[0] = 0;
      s.misc[5] = (int)((blockIdx.x / max(1, L.num_sms)) * 2);
      s.misc[6] = gridDim.x > (unsigned)L.num_sms;  // several CTAs per SM: throughput mode
    }
    Bufs B = setup_bufs(smem, slotp, d, L, false);
    double2* X = B.X[0];
    double2* Xo = B.X[1];
    double2* T = B.T[0];
    double2* To = B.T[1];
    cta_identity(n, X);
    cta_identity(n, T);
    for (int k = tid(); k < n; k += nthr()) s.logD[k] = 0.0;
    __syncthreads();
    const SparseHop* hop = hops ? hops + d.user_index : nullptr;
    for (int b = 0; b < d.nt; b += d.nstab) {
      if (hop)
        fwd_slices_sparse(n, hop, d.phi, b, b + d.nstab, X, Xo, s);
      else
        fwd_slices(n, B.E, d.phi, b, b + d.nstab, X, Xo, s);
      cta_reortho(n, X, Xo, T, To, s.logD, s);
      double2* t1 = X; X = Xo; Xo = t1;
      double2* t2 = T; T = To; To = t2;
    }
    cta_assemble(n, X, T, s.logD, Xo, To, s, s.red + 2, s.red + 3);
    double re = s.red[2], im = wrap_pi(s.red[3]);
    if (tid() == 0) {
      d.logdet[0] = re;
      d.logdet[1] = im;
    }
    if (d.G) write_green(n, To, d.G);
    if (d.nf) cta_fermion_number(n, To, d.nf);
    finish_status(d, s, status, re, im);
  }
}

// ------------------------------------------------------------------ force
// G <- B_s G B_s^{-1} = E diag(ph) G diag(ph*) E^{-1}; src may equal Ga; result in Ga.
__device__ void wrap_forward(int n, const double* E, const double* Einv, const double* phi_row,
                             const double2* src, double2* Ga, double2* Gb, Small& s) {
  cta_phase(n, s.ph, phi_row, 1.0);
  __syncthreads();
  for (int e = tid(); e < n * n; e += nthr()) {
    int i = e % n, j = e / n;
    st(Ga + e, ld(s.ph + i) * ld(src + e) * conj(ld(s.ph + j)));
  }
  __syncthreads();
  cta_gemm<false>(n, RealMat{E, 1, n}, CMat{Ga, 1, n},
                  [&](int i, int j, cplx v) { st(Gb + i + j * n, v); });
  cta_gemm<false>(n, CMat{Gb, 1, n}, RealMat{Einv, 1, n},
                  [&](int i, int j, cplx v) { st(Ga + i + j * n, v); });
}

// G <- B_s^{-1} G B_s = diag(ph*) E^{-1} G E diag(ph); src may equal Ga; result in Ga.
__device__ void wrap_backward(int n, const double* E, const double* Einv, const double* phi_row,
                              const double2* src, double2* Ga, double2* Gb, Small& s) {
  cta_phase(n, s.ph, phi_row, 1.0);
  cta_gemm<false>(n, RealMat{Einv, 1, n}, CMat{src, 1, n},
                  [&](int i, int j, cplx v) { st(Gb + i + j * n, v); });
  const double2* ph = s.ph;
  cta_gemm<false>(n, CMat{Gb, 1, n}, RealMat{E, 1, n}, [&](int i, int j, cplx v) {
    st(Ga + i + j * n, conj(ld(ph + i)) * v * ld(ph + j));
  });
}

// ------------------------------------------------------------------ force, phase A
// Two independent chains per configuration, four when they are split (ChainSpan):
//   forward : X D T <- B_t ... B_1 with a QR every n_stab slices; left checkpoints after blocks
//             1..nb-1; at the end log det and G_0 = G (also the boundary G of block 1).
//   backward: the right products as adjoints, X_R D_R T_R <- B_{t+1}^H ... B_Nt^H, a QR every
//             n_stab slices; right checkpoints at t = (b-1) n_stab for blocks b = nb..2.
__global__ void __launch_bounds__(256, 3) k_chain_fp64(const Desc* __restrict__ descs,
                                                     const Task* __restrict__ tasks, int ntasks,
                                                     int* queue, int* status, char* scratch,
                                                     Layout L) {
  extern __shared__ __align__(16) char smem[];
  char* slotp = scratch + (size_t)blockIdx.x * L.slot_bytes;
  allow_dependents();
  for (;;) {
    int* slot = (int*)(smem + L.smem_bytes - 16);
    const int q = grab(queue, slot);
    if (q >= ntasks) return;
    const Task tk = tasks[q];
    const Desc d = descs[tk.desc];
    // Task.b: a ChainCode (forward/backward chain, its second half, or a log det/G segment)
    const int ns = d.nstab, nb = d.nt / d.nstab;
    const int sg = (tk.b >= CT_SEG && tk.b < CT_FWD2) ? tk.b - CT_SEG : -1;
    const ChainSpan sp = chain_span(tk.b, nb, d.fsplit);
    const int n = d.nx;
    const FWork W{d.fws, n, nb};
    Small s = carve_small(smem + L.small_off, n);
    if (tid() == 0) {
      s.misc[0] = 0;
      s.misc[5] = (int)((blockIdx.x / max(1, L.num_sms)) * 2);
      s.misc[6] = gridDim.x > (unsigned)L.num_sms;  // several CTAs per SM: throughput mode
    }
    Bufs B = setup_bufs(smem, slotp, d, L, false);
    double2* X = B.X[0];
    double2* Xo = B.X[1];
    double2* T = B.T[0];
    double2* To = B.T[1];
    cta_identity(n, X);
    cta_identity(n, T);
    for (int k = tid(); k < n; k += nthr()) s.logD[k] = 0.0;
    __syncthreads();
    if (sg >= 0) {
      // one segment of the chain from the identity: blocks sg*kb+1 .. (sg+1)*kb, result in
      // the checkpoint storage of block sg+1 (merged by k_merge_fp64)
      const int kb = nb / d.nseg, b_first = sg * kb + 1;
      for (int b = b_first; b < b_first + kb; ++b) {
        fwd_slices(n, B.E, d.phi, (b - 1) * ns, b * ns, X, Xo, s);
        cta_reortho(n, X, Xo, T, To, s.logD, s);
        double2* t1 = X; X = Xo; Xo = t1;
        double2* t2 = T; T = To; To = t2;
      }
      cta_copy(n * n, W.LX(sg + 1), X);
      cta_copy(n * n, W.LT(sg + 1), T);
      for (int k = tid(); k < n; k += nthr()) W.LD(sg + 1)[k] = s.logD[k];
      if (tid() == 0 && s.misc[0]) atomicMax(status + d.user_index, ST_NUMERIC);
    } else if (sp.fwd) {
      for (int b = sp.first; b <= sp.last; ++b) {
        fwd_slices(n, B.E, d.phi, (b - 1) * ns, b * ns, X, Xo, s);
        cta_reortho(n, X, Xo, T, To, s.logD, s);
        double2* t1 = X; X = Xo; Xo = t1;
        double2* t2 = T; T = To; To = t2;
        if (b < nb || !sp.assemble) {  // left checkpoint b (the split half's full product: SX)
          cta_copy(n * n, b < nb ? W.LX(b) : W.SX(), X);
          cta_copy(n * n, b < nb ? W.LT(b) : W.ST(), T);
          double* ldst = b < nb ? W.LD(b) : W.SD();
          for (int k = tid(); k < n; k += nthr()) ldst[k] = s.logD[k];
          __syncthreads();
          if (tid() == 0 && d.sync) flag_store(d.sync + sp.flag, sp.count(b));
        }
      }
      if (sp.assemble) {
        cta_assemble(n, X, T, s.logD, Xo, To, s, s.red + 2, s.red + 3);
        const double re = s.red[2], im = wrap_pi(s.red[3]);
        if (tid() == 0) {
          d.logdet[0] = re;
          d.logdet[1] = im;
        }
        cta_copy(n * n, W.Gb(1), To);
        if (d.G) write_green(n, To, d.G);
        if (d.Gt) write_green(n, To, d.Gt);  // G(0, 0) = G
        if (d.nf) cta_fermion_number(n, To, d.nf);
        if (d.O) {  // FP32 copy of the response operator for the tensor-core wraps
          float* of = W.OF(d.Gt != nullptr);
          for (int e = tid(); e < n * n; e += nthr()) of[e] = (float)d.O[e];
        }
        __syncthreads();
        if (tid() == 0 && d.sync) flag_store(d.sync + SF_FWD, nb);  // G_0 written
        if (tid() == 0)
          atomicMax(status + d.user_index,
                    (s.misc[0] || !isfinite(re) || !isfinite(im)) ? ST_NUMERIC : ST_OK);
      } else if (tid() == 0 && s.misc[0]) {
        atomicMax(status + d.user_index, ST_NUMERIC);
      }
    } else {
      for (int b = sp.first; b >= sp.last; --b) {
        bwd_slices(n, B.E, d.phi, (b - 1) * ns, b * ns, X, Xo, s);
        cta_reortho(n, X, Xo, T, To, s.logD, s);
        double2* t1 = X; X = Xo; Xo = t1;
        double2* t2 = T; T = To; To = t2;
        cta_copy(n * n, W.RX(b), X);
        cta_copy(n * n, W.RT(b), T);
        for (int k = tid(); k < n; k += nthr()) W.RD(b)[k] = s.logD[k];
        __syncthreads();
        if (tid() == 0 && d.sync) flag_store(d.sync + sp.flag, sp.count(b));
      }
      if (tid() == 0 && s.misc[0]) atomicMax(status + d.user_index, ST_NUMERIC);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ force, phase B
// Boundary Green's function of block b (b = 2..nb): G_{(b-1)ns} from the left checkpoint b-1
// and the right checkpoint b (Section 7 steps 7-9 with t1 = t2; Section 5.3).  With the chains
// split at block h (ChainSpan) a left checkpoint beyond h is first merged with L_h and a right
// one below h+1 with R_{h+1} (cta_merge), and task b = 1 forms the full product L'_nb L_h, the
// assembly (log det, G_0) and the outputs of the forward chain.  Segmented chains (SegPlan) leave
// final checkpoints: only the waits differ.
// MERGE: the variant for calls with split or segmented chains (the plain one keeps its register
// budget).
template <bool MERGE>
__global__ void __launch_bounds__(256) k_boundary_fp64(const Desc* __restrict__ descs,
                                                        const Task* __restrict__ tasks,
                                                        int ntasks, int* queue, int* status,
                                                        char* scratch, Layout L) {
  extern __shared__ __align__(16) char smem[];
  char* slotp = scratch + (size_t)blockIdx.x * L.slot_bytes;
  allow_dependents();
  for (;;) {
    int* slot = (int*)(smem + L.smem_bytes - 16);
    const int q = grab(queue, slot);
    if (q >= ntasks) return;
    const Task tk = tasks[q];
    const Desc d = descs[tk.desc];
    const int n = d.nx, nb = d.nt / d.nstab, b = tk.b, h = MERGE ? d.fsplit : 0;
    const FWork W{d.fws, n, nb};
    // inputs: left checkpoint b-1 (merged when beyond h), right checkpoint b (merged below h+1)
    const bool ml = h > 0 && b - 1 > h, mr = h > 0 && b >= 2 && b <= h;
    const int wf = b == 1 ? h : (ml ? h : b - 1), wf2 = b == 1 ? nb - h : (ml ? b - 1 - h : 0);
    const int wb = b == 1 ? 0 : (mr ? nb - h : nb - b + 1), wb2 = mr ? h - b + 1 : 0;
    bool waited = true;
    if (MERGE && d.sync && d.fseg) {  // segmented chains: their two checkpoints' segment flags
      const int mb = nb / d.fseg;
      int i0, t0, i1, t1;
      seg_left_ready(b - 1, mb, i0, t0);
      seg_right_ready(b, nb, mb, i1, t1);
      waited = cta_wait_pairs(d.sync, i0, t0, i1, t1, slot + 1);
    } else if (d.sync) {
      waited = cta_wait_flags(d.sync, wf, wb, 0, slot + 1, wf2, wb2);
    }
    if (!waited && tid() == 0) atomicMax(status + d.user_index, ST_TIMEOUT);
    Small s = carve_small(smem + L.small_off, n);
    if (tid() == 0) {
      s.misc[0] = 0;
      s.misc[5] = (int)((blockIdx.x / max(1, L.num_sms)) * 2 + b);
      s.misc[6] = gridDim.x > (unsigned)L.num_sms;  // several CTAs per SM: throughput mode
    }
    double2* Ma = (double2*)place(smem, slotp, L, B_GA);
    double2* Mb = (double2*)place(smem, slotp, L, B_GB);
    __syncthreads();
    if (MERGE && b == 1) {  // split chains: G_0 and log det from the full product L'_nb L_h
      double2* X = (double2*)place(smem, slotp, L, B_X0);
      double2* T = (double2*)place(smem, slotp, L, B_T0);
      cta_merge(n, W.SX(), W.ST(), W.SD(), W.LX(h), W.LT(h), W.LD(h), Ma, Mb, X, T, s.logD, s);
      cta_assemble(n, X, T, s.logD, Ma, Mb, s, s.red + 2, s.red + 3);
      const double pi = 3.14159265358979323846;  // det X = +1 after the merge
      const double re = s.red[2], im = wrap_pi(s.red[3] - ((n - 1) & 1 ? pi : 0.0));
      if (tid() == 0) {
        d.logdet[0] = re;
        d.logdet[1] = im;
      }
      cta_copy(n * n, W.Gb(1), Mb);
      if (d.G) write_green(n, Mb, d.G);
      if (d.nf) cta_fermion_number(n, Mb, d.nf);
      __syncthreads();
      if (tid() == 0) {
        atomicMax(status + d.user_index,
                  (s.misc[0] || !isfinite(re) || !isfinite(im)) ? ST_NUMERIC : ST_OK);
        if (d.sync) flag_store(d.sync + SF_FWD, nb);  // G_0 written
      }
      __syncthreads();
      continue;
    }
    const double2 *XL = W.LX(b - 1), *TL = W.LT(b - 1), *XR = W.RX(b), *TR = W.RT(b);
    const double *DL = W.LD(b - 1), *DR = W.RD(b);
    if (MERGE && (ml || mr)) {
      double2* X = (double2*)place(smem, slotp, L, B_X0);
      double2* T = (double2*)place(smem, slotp, L, B_T0);
      if (ml) {
        cta_merge(n, XL, TL, DL, W.LX(h), W.LT(h), W.LD(h), Ma, Mb, X, T, s.logD, s);
        XL = X; TL = T; DL = s.logD;
      } else {
        cta_merge(n, XR, TR, DR, W.RX(h + 1), W.RT(h + 1), W.RD(h + 1), Ma, Mb, X, T, s.logD, s);
        XR = X; TR = T; DR = s.logD;
      }
    }
    boundary_green(n, false, XL, TL, DL, XR, TR, DR, Ma, Mb, (d.F || d.R) ? W.Gb(b) : nullptr, s,
                   d.Gt ? W.GT(b) : nullptr);
    if (d.Gt) write_green(n, W.GT(b), d.Gt + (size_t)(b - 1) * d.nstab * n * n);
    if (tid() == 0 && s.misc[0]) atomicMax(status + d.user_index, ST_NUMERIC);
    __syncthreads();
    if (tid() == 0 && d.sync) flag_add(d.sync + SF_BND, 1);
  }
}

// ------------------------------------------------------------------ force, phase C
// Block b: F row (b-1)ns from G_{(b-1)ns}; forward wraps from it for the first (n_stab-1)/2
// slices, backward wraps from G_{b ns} (the next block's boundary, G_0 for the last block).
__global__ void __launch_bounds__(256) k_wrap_fp64(const Desc* __restrict__ descs,
                                                    const Task* __restrict__ tasks, int ntasks,
                                                    int* queue, int* status, char* scratch,
                                                    Layout L) {
  extern __shared__ __align__(16) char smem[];
  char* slotp = scratch + (size_t)blockIdx.x * L.slot_bytes;
  for (;;) {
    int* slot = (int*)(smem + L.smem_bytes - 16);
    const int q = grab(queue, slot);
    if (q >= ntasks) return;
    const Task tk = tasks[q];
    const Desc d = descs[tk.desc];
    const int n = d.nx, ns = d.nstab, nb = d.nt / d.nstab, b = tk.b;
    const FWork W{d.fws, n, nb};
    // G_0 and every boundary Green's function of the configuration
    if (d.sync && !cta_wait_flags(d.sync, nb, 0, nb - 1, slot + 1) && tid() == 0)
      atomicMax(status + d.user_index, ST_TIMEOUT);
    Small s = carve_small(smem + L.small_off, n);
    if (tid() == 0) s.misc[0] = 0;
    const double* E = L.in_smem[B_E] ? (double*)(smem + L.off[B_E]) : d.E;
    const double* Einv = L.in_smem[B_EINV] ? (double*)(smem + L.off[B_EINV]) : d.Einv;
    if (L.in_smem[B_E]) cta_load_real(n * n, (double*)E, d.E);
    if (L.in_smem[B_EINV]) cta_load_real(n * n, (double*)Einv, d.Einv);
    double2* Ga = (double2*)place(smem, slotp, L, B_GA);
    double2* Gb = (double2*)place(smem, slotp, L, B_GB);
    __syncthreads();
    const int t0 = (b - 1) * ns, h = (ns - 1) / 2;
    if (d.F || d.R) {
      // G_r for every r of the block: force rows and/or response traces
      auto emit = [&](const double2* G, int r) {
        if (d.F) emit_force_row(n, G, d.F + (size_t)r * n);
        if (d.R) cta_trace(n, d.O, G, d.R + r, s.red + 32);
      };
      const double2* Glo = W.Gb(b);
      emit(Glo, t0);
      const double2* src = Glo;
      for (int j = 1; j <= h; ++j) {
        wrap_forward(n, E, Einv, d.phi + (size_t)(t0 + j - 1) * n, src, Ga, Gb, s);
        emit(Ga, t0 + j);
        src = Ga;
      }
      __syncthreads();
      src = W.Gb(b + 1);
      for (int qq = b * ns; qq >= t0 + h + 2; --qq) {
        wrap_backward(n, E, Einv, d.phi + (size_t)(qq - 1) * n, src, Ga, Gb, s);
        emit(Ga, qq - 1);
        src = Ga;
      }
      __syncthreads();
    }
    if (d.Gt) {
      // G(tau, 0) inside the block: forward G(t+1, 0) = E diag(ph_{t+1}) G(t, 0) from the lower
      // boundary, backward G(q-1, 0) = diag(ph_q^*) E^{-1} G(q, 0) from the upper one
      // (G(Nt, 0) = B_Nt...B_1 G = 1 - G for the last block).
      const size_t nn = (size_t)n * n;
      const double2* src = W.GT(b);
      for (int j = 1; j <= h; ++j) {
        cta_phase(n, s.ph, d.phi + (size_t)(t0 + j - 1) * n, 1.0);
        __syncthreads();
        for (int e = tid(); e < n * n; e += nthr()) st(Gb + e, ld(s.ph + e % n) * ld(src + e));
        __syncthreads();
        cta_gemm<false>(n, RealMat{E, 1, n}, CMat{Gb, 1, n},
                        [&](int i, int jj, cplx v) { st(Ga + i + jj * n, v); });
        write_green(n, Ga, d.Gt + (size_t)(t0 + j) * nn);
        src = Ga;
      }
      __syncthreads();
      double2* cur = Ga;
      if (b == nb) {  // 1 - G
        const double2* G0 = W.Gb(1);
        for (int e = tid(); e < n * n; e += nthr())
          st(Gb + e, cx((e % n == e / n) ? 1.0 : 0.0, 0.0) - ld(G0 + e));
        __syncthreads();
        src = Gb;
        cur = Ga;
      } else {
        src = W.GT(b + 1);
      }
      for (int qq = b * ns; qq >= t0 + h + 2; --qq) {
        cta_phase(n, s.ph, d.phi + (size_t)(qq - 1) * n, -1.0);
        __syncthreads();
        const double2* ph = s.ph;
        cta_gemm<false>(n, RealMat{Einv, 1, n}, CMat{src, 1, n},
                        [&](int i, int jj, cplx v) { st(cur + i + jj * n, ld(ph + i) * v); });
        write_green(n, cur, d.Gt + (size_t)(qq - 1) * nn);
        __syncthreads();
        src = cur;
        cur = (cur == Ga) ? Gb : Ga;
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ time-parallel log det/G
// Merge of the nseg segment products of one configuration (cta_merge: Section 7's stabilised
// product of two UDV factors, applied segment by segment, the accumulated product Xa Da Ta
// acting first) and the assembly.  A segment's log D must span less than 700 (else
// FD_ERR_NUMERIC) -- beta per segment up to ~100 at kappa = 1 on this lattice.  After a merge
// X = Xs Q is a product of two Householder products: det X = +1 (the assembly assumes
// (-1)^{n-1}, right for S = 1).
__global__ void __launch_bounds__(256) k_merge_fp64(const Desc* __restrict__ descs, int ndesc,
                                                     int* queue, int* status, char* scratch,
                                                     Layout L) {
  extern __shared__ __align__(16) char smem[];
  char* slotp = scratch + (size_t)blockIdx.x * L.slot_bytes;
  for (;;) {
    int* slot = (int*)(smem + L.smem_bytes - 16);
    const int c = grab(queue, slot);
    if (c >= ndesc) return;
    const Desc d = descs[c];
    const int n = d.nx, nb = d.nt / d.nstab, S = d.nseg;
    const FWork W{d.fws, n, nb};
    Small s = carve_small(smem + L.small_off, n);
    if (tid() == 0) {
      s.misc[0] = 0;
      s.misc[5] = (int)((blockIdx.x / max(1, L.num_sms)) * 2);
      s.misc[6] = gridDim.x > (unsigned)L.num_sms;
    }
    double2* Xa = (double2*)place(smem, slotp, L, B_X0);
    double2* Xc = (double2*)place(smem, slotp, L, B_X1);
    double2* Ta = (double2*)place(smem, slotp, L, B_T0);
    double2* Tn = (double2*)place(smem, slotp, L, B_T1);
    double2* Xn = (double2*)place(smem, slotp, L, B_GA);
    cta_copy(n * n, Xa, W.LX(1));
    cta_copy(n * n, Ta, W.LT(1));
    for (int k = tid(); k < n; k += nthr()) s.logD[k] = W.LD(1)[k];
    __syncthreads();
    for (int sg = 1; sg < S; ++sg) {
      cta_merge(n, W.LX(sg + 1), W.LT(sg + 1), W.LD(sg + 1), Xa, Ta, s.logD, Xc, Xn, Xa, Tn,
                s.logD, s);
      double2* t = Ta; Ta = Tn; Tn = t;
    }
    cta_assemble(n, Xa, Ta, s.logD, Xc, Xn, s, s.red + 2, s.red + 3);
    const double pi = 3.14159265358979323846;
    const double re = s.red[2], im = wrap_pi(s.red[3] - (S > 1 && ((n - 1) & 1) ? pi : 0.0));
    if (tid() == 0) {
      d.logdet[0] = re;
      d.logdet[1] = im;
    }
    if (d.G) write_green(n, Xn, d.G);
    if (d.nf) cta_fermion_number(n, Xn, d.nf);
    if (tid() == 0)
      atomicMax(status + d.user_index,
                (s.misc[0] || !isfinite(re) || !isfinite(im)) ? ST_NUMERIC : ST_OK);
    __syncthreads();
  }
}

void launch_fwd_fp64(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                     const Layout& L, int grid, cudaStream_t stream, const SparseHop* hops) {
  k_fwd_fp64<<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, ndesc, queue, status, scratch, L,
                                                         hops);
}
void launch_chain_fp64(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                       char* scratch, const Layout& L, int grid, cudaStream_t stream) {
  k_chain_fp64<<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, tasks, ntasks, queue, status,
                                                            scratch, L);
}
void launch_boundary_fp64(const Desc* descs, const Task* tasks, int ntasks, int* queue,
                          int* status, char* scratch, const Layout& L, int grid,
                          cudaStream_t stream, bool pdl, bool merge) {
  if (merge)
    launch_maybe_pdl(k_boundary_fp64<true>, grid, L.nthreads, L.smem_bytes, stream, pdl, descs,
                     tasks, ntasks, queue, status, scratch, L);
  else
    launch_maybe_pdl(k_boundary_fp64<false>, grid, L.nthreads, L.smem_bytes, stream, pdl, descs,
                     tasks, ntasks, queue, status, scratch, L);
}
void launch_wrap_fp64(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                      char* scratch, const Layout& L, int grid, cudaStream_t stream, bool pdl) {
  launch_maybe_pdl(k_wrap_fp64, grid, L.nthreads, L.smem_bytes, stream, pdl, descs, tasks, ntasks,
                   queue, status, scratch, L);
}
void launch_merge_fp64(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                       const Layout& L, int grid, cudaStream_t stream) {
  k_merge_fp64<<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, ndesc, queue, status, scratch,
                                                            L);
}
static const void* fp64_kernel(int which) {
  switch (which) {
    case 1: return (const void*)k_chain_fp64;
    case 2: return (const void*)k_boundary_fp64<false>;
    case 9: return (const void*)k_boundary_fp64<true>;
    case 3: return (const void*)k_wrap_fp64;
    case 8: return (const void*)k_merge_fp64;
    default: return (const void*)k_fwd_fp64;
  }
}
int occupancy_fp64(int which, int nthreads, int smem_bytes) {
  int nb = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fp64_kernel(which), nthreads, smem_bytes);
  return e == cudaSuccess ? nb : -1;
}
cudaError_t set_smem_fp64(int bytes) {
  for (const void* k : {(const void*)k_fwd_fp64, (const void*)k_chain_fp64,
                        (const void*)k_boundary_fp64<false>, (const void*)k_boundary_fp64<true>,
                        (const void*)k_wrap_fp64, (const void*)k_merge_fp64}) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t attrs_fp64(int which, cudaFuncAttributes* a) {
  return cudaFuncGetAttributes(a, fp64_kernel(which));
}

}  // namespace fd
