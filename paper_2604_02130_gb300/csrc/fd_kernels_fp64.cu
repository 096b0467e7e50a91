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
                                                   Layout L) {
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
    for (int b = 0; b < d.nt; b += d.nstab) {
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

__global__ void __launch_bounds__(256) k_force_fp64(const Desc* __restrict__ descs, int ndesc,
                                                     int* queue, int* status, char* scratch,
                                                     Layout L) {
  extern __shared__ __align__(16) char smem[];
  char* slotp = scratch + (size_t)blockIdx.x * L.slot_bytes;
  double2* ckbase = (double2*)(slotp + L.ws_bytes);
  for (;;) {
    int* slot = (int*)(smem + L.smem_bytes - 16);
    int c = grab(queue, slot);
    if (c >= ndesc) return;
    const Desc d = descs[c];
    const int n = d.nx, ns = d.nstab, nb = d.nt / d.nstab;
    Small s = carve_small(smem + L.small_off, n);
    if (tid() == 0) {
      s.misc[0] = 0;
      s.misc[5] = (int)((blockIdx.x / max(1, L.num_sms)) * 2);
    }
    Bufs B = setup_bufs(smem, slotp, d, L, true);
    // checkpoint b (1..nb-1): X (n*n), T (n*n), logD (n doubles, padded to n/2+1 complex)
    const size_t ck_stride = (size_t)2 * n * n + (n + 1) / 2;
    auto ckX = [&](int b) { return ckbase + (size_t)(b - 1) * ck_stride; };
    auto ckT = [&](int b) { return ckbase + (size_t)(b - 1) * ck_stride + (size_t)n * n; };
    auto ckD = [&](int b) { return (double*)(ckbase + (size_t)(b - 1) * ck_stride + (size_t)2 * n * n); };

    // ---- forward pass with checkpoints
    double2* X = B.X[0];
    double2* Xo = B.X[1];
    double2* T = B.T[0];
    double2* To = B.T[1];
    cta_identity(n, X);
    cta_identity(n, T);
    for (int k = tid(); k < n; k += nthr()) s.logD[k] = 0.0;
    __syncthreads();
    for (int b = 1; b <= nb; ++b) {
      fwd_slices(n, B.E, d.phi, (b - 1) * ns, b * ns, X, Xo, s);
      cta_reortho(n, X, Xo, T, To, s.logD, s);
      double2* t1 = X; X = Xo; Xo = t1;
      double2* t2 = T; T = To; To = t2;
      if (b < nb) {
        cta_copy(n * n, ckX(b), X);
        cta_copy(n * n, ckT(b), T);
        for (int k = tid(); k < n; k += nthr()) ckD(b)[k] = s.logD[k];
        __syncthreads();
      }
    }
    cta_assemble(n, X, T, s.logD, B.Ga, B.Ghi, s, s.red + 2, s.red + 3);
    double re = s.red[2], im = wrap_pi(s.red[3]);
    if (tid() == 0) {
      d.logdet[0] = re;
      d.logdet[1] = im;
    }
    if (d.G) write_green(n, B.Ghi, d.G);
    __syncthreads();

    // ---- backward (adjoint) sweep
    double2* Glo = B.Glo;
    double2* Ghi = B.Ghi;  // G_{b*ns}; starts as G_Nt = G_0
    cta_identity(n, X);
    cta_identity(n, T);
    for (int k = tid(); k < n; k += nthr()) s.logDR[k] = 0.0;
    __syncthreads();
    const int h = (ns - 1) / 2;  // forward wraps per block; ns-1-h backward wraps
    for (int b = nb; b >= 1; --b) {
      const int t0 = (b - 1) * ns;  // boundary time of this block
      bwd_slices(n, B.E, d.phi, t0, b * ns, X, Xo, s);
      cta_reortho(n, X, Xo, T, To, s.logDR, s);
      double2* t1 = X; X = Xo; Xo = t1;
      double2* t2 = T; T = To; To = t2;
      // G_{t0} at the boundary: left = checkpoint b-1 (identity for b = 1)
      if (b == 1)
        boundary_green(n, true, nullptr, nullptr, nullptr, X, T, s.logDR, B.Ga, B.Gb, Glo, s);
      else
        boundary_green(n, false, ckX(b - 1), ckT(b - 1), ckD(b - 1), X, T, s.logDR, B.Ga, B.Gb,
                       Glo, s);
      // F row t0 (slice t0+1) uses G_{t0}
      emit_force_row(n, Glo, d.F + (size_t)t0 * n);
      // forward wraps: G_{t0+j} = B_{t0+j} G_{t0+j-1} B_{t0+j}^{-1}, j = 1..h  (phi row t0+j-1)
      const double2* src = Glo;
      for (int j = 1; j <= h; ++j) {
        wrap_forward(n, B.E, B.Einv, d.phi + (size_t)(t0 + j - 1) * n, src, B.Ga, B.Gb, s);
        emit_force_row(n, B.Ga, d.F + (size_t)(t0 + j) * n);
        src = B.Ga;
      }
      __syncthreads();
      // backward wraps from G_{b*ns}: G_{q-1} = B_q^{-1} G_q B_q, q = b*ns .. t0+h+2 (phi row q-1)
      src = Ghi;
      for (int q = b * ns; q >= t0 + h + 2; --q) {
        wrap_backward(n, B.E, B.Einv, d.phi + (size_t)(q - 1) * n, src, B.Ga, B.Gb, s);
        emit_force_row(n, B.Ga, d.F + (size_t)(q - 1) * n);
        src = B.Ga;
      }
      __syncthreads();
      double2* tg = Ghi; Ghi = Glo; Glo = tg;
    }
    finish_status(d, s, status, re, im);
  }
}

void launch_fwd_fp64(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                     const Layout& L, int grid, cudaStream_t stream) {
  k_fwd_fp64<<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, ndesc, queue, status, scratch, L);
}
void launch_force_fp64(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                       const Layout& L, int grid, cudaStream_t stream) {
  k_force_fp64<<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, ndesc, queue, status, scratch,
                                                            L);
}
int occupancy_fp64(bool force, int nthreads, int smem_bytes) {
  int nb = 0;
  cudaError_t e;
  if (force)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_fp64, nthreads, smem_bytes);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_fp64, nthreads, smem_bytes);
  return e == cudaSuccess ? nb : -1;
}
cudaError_t set_smem_fp64(int bytes) {
  for (const void* k : {(const void*)k_fwd_fp64, (const void*)k_force_fp64}) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t attrs_fp64(bool force, cudaFuncAttributes* a) {
  return cudaFuncGetAttributes(a, force ? (const void*)k_force_fp64 : (const void*)k_fwd_fp64);
}

}  // namespace fd
