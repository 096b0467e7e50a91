// fd_noalloc.cu -- log det (and optionally G) for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs while another component owns every
// allocation (an embedding framework with its own memory pool, a real-time loop with a fixed
// memory budget set at start-up), or code that must not trigger the implicit device
// synchronisation of cudaMalloc/cudaFree in the middle of a pipelined step.  fd_logdet_noalloc
// serves them: it needs no fd_ctx and allocates nothing.  Its working memory is the file-scope
// array g_noalloc_scratch below, a fixed 12 MiB that every GPU loading this library holds until
// the process exits.  The caller passes inputs and outputs as usual.
//
// The array's name, used in host code, is only a host-side stand-in for the device object; the
// device address is obtained once per device with cudaGetSymbolAddress (see device_setup) and
// that address is what the kernel receives.
#include <mutex>

#include "fd_fp64.cuh"

#define FD_NOALLOC_SCRATCH_BYTES (12u << 20)
#define FD_NOALLOC_THREADS 256
#define FD_NOALLOC_MAX_DEVICES 64

namespace fd {
namespace {

static __device__ __align__(256) char g_noalloc_scratch[FD_NOALLOC_SCRATCH_BYTES];

struct NDesc {  // 48 bytes: FD_NOALLOC_MAX_BATCH of them travel as a kernel parameter
  int nx, nt, nstab, pad;
  const double* E;
  const double* phi;
  double* logdet;
  double2* G;
};
struct NPack {
  NDesc d[FD_NOALLOC_MAX_BATCH];
  int* status;
  long long slot_bytes;
};

// shared memory: E (8n^2) | X0 (16n^2) | X1 (16n^2) | small vectors; T0, T1 in the scratch slot
__host__ __device__ inline long long na_smem_bytes(int n) {
  long long o = 8LL * n * n + 32LL * n * n;
  return ((o + 15) & ~15LL) + ((small_bytes(n) + 15) & ~15) + 16;
}
__host__ __device__ inline long long na_slot_bytes(int n) {
  return ((32LL * n * n) + 255) & ~255LL;
}

__device__ void na_fwd_slices(int n, const double* E, const double* phi, int s_begin, int s_end,
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

// One CTA per configuration; CTA c uses slot c of the scratch array (passed in as `scratch`).
__global__ void __launch_bounds__(FD_NOALLOC_THREADS) k_fwd_fp64_noalloc(NPack pk, int batch,
                                                                          char* scratch) {
  extern __shared__ __align__(16) char smem[];
  const int c = blockIdx.x;
  if (c >= batch) return;
  const NDesc d = pk.d[c];
  const int n = d.nx;
  char* slot = scratch + (size_t)c * pk.slot_bytes;
  double* Es = (double*)smem;
  double2* X = (double2*)(smem + 8LL * n * n);
  double2* Xo = X + (size_t)n * n;
  long long so = (8LL * n * n + 32LL * n * n + 15) & ~15LL;
  Small s = carve_small(smem + so, n);
  double2* T = (double2*)slot;  // every buffer is fully written before it is read
  double2* To = T + (size_t)n * n;
  if (tid() == 0) {
    s.misc[0] = 0;
    s.misc[5] = 0;  // leader-warp offset of the shared CTA routines
    s.misc[6] = 0;  // latency-mode segment widths
  }
  cta_load_real(n * n, Es, d.E);
  cta_identity(n, X);
  cta_identity(n, T);
  for (int k = tid(); k < n; k += nthr()) s.logD[k] = 0.0;
  __syncthreads();
  for (int b = 0; b < d.nt; b += d.nstab) {
    na_fwd_slices(n, Es, d.phi, b, b + d.nstab, X, Xo, s);
    cta_reortho(n, X, Xo, T, To, s.logD, s);
    double2* t1 = X; X = Xo; Xo = t1;
    double2* t2 = T; T = To; To = t2;
  }
  cta_assemble(n, X, T, s.logD, Xo, To, s, s.red + 2, s.red + 3);
  const double re = s.red[2], im = wrap_pi(s.red[3]);
  if (tid() == 0) {
    d.logdet[0] = re;
    d.logdet[1] = im;
  }
  if (d.G)
    for (int e = tid(); e < n * n; e += nthr()) d.G[e] = To[(e / n) + (e % n) * n];
  if (tid() == 0 && pk.status)
    pk.status[c] = (s.misc[0] || !isfinite(re) || !isfinite(im)) ? ST_NUMERIC : ST_OK;
}

std::mutex g_setup_mu;
void* g_scratch_dev[FD_NOALLOC_MAX_DEVICES];
bool g_ready[FD_NOALLOC_MAX_DEVICES];

// Once per device, with that device current: the device address of the scratch array and the
// kernel's shared-memory limit.  Neither allocates.
int device_setup(int dev, char** scratch) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_ready[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FD_ERR_CUDA;
    if (cudaFuncSetAttribute(k_fwd_fp64_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)na_smem_bytes(FD_NOALLOC_MAX_NX)) != cudaSuccess)
      return FD_ERR_CUDA;
    g_scratch_dev[dev] = p;
    g_ready[dev] = true;
  }
  *scratch = (char*)g_scratch_dev[dev];
  return FD_OK;
}

}  // namespace
}  // namespace fd

extern "C" int fd_logdet_noalloc(int batch, const fd_problem* probs, double* logdet,
                                 double* const* G, int* status, void* stream) {
  using namespace fd;
  if (batch < 0 || (batch > 0 && (!probs || !logdet))) return FD_ERR_INVALID;
  if (batch > FD_NOALLOC_MAX_BATCH) return FD_ERR_TOO_LARGE;
  NPack pk;
  int nmax = 1;
  for (int c = 0; c < batch; ++c) {
    const fd_problem& p = probs[c];
    if (p.nx < 1 || p.nt < 1 || p.n_stab < 1 || p.n_stab > p.nt || p.nt % p.n_stab != 0 ||
        p.reserved != 0 || !p.expA || !p.phi || (G && !G[c]))
      return FD_ERR_INVALID;
    if (p.nx > FD_NOALLOC_MAX_NX) return FD_ERR_TOO_LARGE;
    nmax = p.nx > nmax ? p.nx : nmax;
    pk.d[c] = NDesc{p.nx, p.nt, p.n_stab, 0, p.expA, p.phi, logdet + 2 * (size_t)c,
                    G ? (double2*)G[c] : nullptr};
  }
  if (batch == 0) return FD_OK;
  pk.status = status;
  pk.slot_bytes = na_slot_bytes(nmax);
  if ((unsigned long long)pk.slot_bytes * (unsigned long long)batch > FD_NOALLOC_SCRATCH_BYTES)
    return FD_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FD_ERR_CUDA;
  if (dev < 0 || dev >= FD_NOALLOC_MAX_DEVICES) return FD_ERR_UNSUPPORTED;
  char* scratch = nullptr;
  int rc = device_setup(dev, &scratch);
  if (rc != FD_OK) return rc;
  k_fwd_fp64_noalloc<<<batch, FD_NOALLOC_THREADS, (size_t)na_smem_bytes(nmax),
                       (cudaStream_t)stream>>>(pk, batch, scratch);
  return cudaGetLastError() == cudaSuccess ? FD_OK : FD_ERR_CUDA;
}
