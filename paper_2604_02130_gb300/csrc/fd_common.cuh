// fd_common.cuh -- shared device-side definitions: complex helpers, the per-configuration
// descriptor, buffer placement and status codes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fd.h"

namespace fd {

// ---------------------------------------------------------------- complex FP64 helpers
struct cplx {
  double re, im;
};

__device__ __forceinline__ cplx cx(double r, double i) { return cplx{r, i}; }
__device__ __forceinline__ cplx operator+(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return cplx{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cplx operator*(double s, cplx a) { return cplx{s * a.re, s * a.im}; }
__device__ __forceinline__ cplx conj(cplx a) { return cplx{a.re, -a.im}; }
__device__ __forceinline__ double abs2(cplx a) { return fma(a.re, a.re, a.im * a.im); }
// conj(a) * b
__device__ __forceinline__ cplx cmulc(cplx a, cplx b) {
  return cplx{fma(a.re, b.re, a.im * b.im), fma(a.re, b.im, -a.im * b.re)};
}
// a - b c with four fused multiply-adds
__device__ __forceinline__ cplx cfms(cplx a, cplx b, cplx c) {
  return cplx{fma(-b.re, c.re, fma(b.im, c.im, a.re)), fma(-b.re, c.im, fma(-b.im, c.re, a.im))};
}
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  // scaled division (Smith-free but overflow-safe enough for O(1)..1e150 magnitudes)
  double s = fmax(fabs(b.re), fabs(b.im));
  double br = b.re / s, bi = b.im / s;
  double d = fma(br, br, bi * bi);
  return cplx{fma(a.re, br, a.im * bi) / (d * s), fma(a.im, br, -a.re * bi) / (d * s)};
}
__device__ __forceinline__ cplx ld(const double2* p) {
  double2 v = *p;
  return cplx{v.x, v.y};
}
__device__ __forceinline__ void st(double2* p, cplx v) { *p = make_double2(v.re, v.im); }

// ---------------------------------------------------------------- descriptors
// One configuration as the kernels see it (built on the host from fd_problem + outputs).
struct Desc {
  int nx, nt, nstab, user_index;
  const double* E;     // nx*nx (symmetric)
  const double* Einv;  // nx*nx or null
  const double* phi;   // nt*nx
  double* logdet;      // 2 doubles
  double2* G;          // nx*nx row-major or null
  double2* F;          // nt*nx row-major or null
  double2* Gt;         // unequal-time G(tau, 0): nt*nx*nx row-major [tau][i][j], or null
  double2* fws;        // force / G(tau, 0): per-configuration workspace (FWork), else null
  double* nf;          // fermion number 1 - tr G / nx (re, im), or null
  const double* O;     // response operator, nx*nx row-major, or null
  double2* R;          // response traces tr(O G_r), r = 0..nt-1, or null
  int* sync;           // phased path: this configuration's progress flags (SyncFlag), else null
  int nseg;            // time-parallel log det/G: number of segments of the chain (0: not split)
  int fsplit;          // force: chains split at block h = fsplit (0: not split; see ChainSpan)
  int fseg;            // force, streamed kernels: S segments per chain (0: not segmented; SegPlan)
  // streamed tensor-core kernels (nx above one tile): E and E^{-1} as chunked TF32 operands
  // (hi at the pointer, lo after it; see BLayout), prepared once per call; else null
  const float* Ec;
  const float* Eic;
};

// ---------------------------------------------------------------- overlapped phases
// The three launches of the phased path (chains, boundary Green's functions, wraps) overlap:
// the later ones are launched as programmatic dependents (they may start while the earlier grid
// still runs) and each task waits only for the data it reads, through per-configuration progress
// flags written with release and read with acquire semantics at GPU scope.
enum SyncFlag {
  SF_FWD = 0,   // forward chain: left checkpoints 1..v written; nb once G_0 (= G) is written
  SF_BWD = 1,   // backward chain: v right checkpoints written (blocks nb, nb-1, ...)
  SF_BND = 2,   // boundary Green's functions written (count)
  SF_FWD2 = 3,  // split chains: v local left products of the second forward half written
  SF_BWD2 = 4,  // split chains: v local right products of the second backward half written
  // segmented chains (SegPlan), + k for segment k < FD_SEG_MAX:
  SF_SEGF = 8,   // final left checkpoints written inside forward segment k (count)
  SF_SEGB = 16,  // final right checkpoints written inside backward segment k (count)
  SF_PREF = 24,  // prefix L_{k m} (the first checkpoint of forward segment k) formed by a merge
  SF_PREB = 32,  // suffix R_{nb - k m + 1} formed by a merge
  SF_LSF = 40,   // local product of forward segment k (from the identity) written
  SF_LSB = 48,   // local product of backward segment k written
  SF_NUM = 56    // ints per configuration
};
#define FD_SEG_MAX 8
// A wait gives up after this many cycles without any change of the configuration's flags
// (~4 s at 2 GHz; one checkpoint interval of the largest supported size takes well under that).
#define FD_SYNC_WAIT_CYCLES (8LL * 1000 * 1000 * 1000)

// Launch `kern` on `stream`, as a programmatic dependent of the previous kernel in the stream
// when `pdl` (it may then start before that kernel has finished; its tasks wait on the flags).
template <class... KArgs, class... Args>
inline cudaError_t launch_maybe_pdl(void (*kern)(KArgs...), int grid, int threads, int smem,
                                    cudaStream_t stream, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Let the dependent grid launch (issued by every CTA at its start).
__device__ __forceinline__ void allow_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// One thread, after a __syncthreads that follows the CTA's data writes.
__device__ __forceinline__ void flag_store(int* f, int v) {
  __threadfence();
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}
__device__ __forceinline__ void flag_add(int* f, int v) {
  __threadfence();
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}
__device__ __forceinline__ int flag_load(const int* f) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
  return v;
}
// CTA-wide wait until flags[i0] >= t0 and (i1 < 0 or) flags[i1] >= t1; as cta_wait_flags.
__device__ __forceinline__ bool cta_wait_pairs(const int* flags, int i0, int t0, int i1, int t1,
                                               volatile int* bcast) {
  if (threadIdx.x == 0) {
    long long c0 = clock64();
    int ok = 1, last = -1;
    for (;;) {
      const int f0 = flag_load(flags + i0), f1 = i1 >= 0 ? flag_load(flags + i1) : 0;
      if (f0 >= t0 && (i1 < 0 || f1 >= t1)) break;
      const int sum = f0 + f1;
      const long long now = clock64();
      if (sum != last) {
        last = sum;
        c0 = now;
      } else if (now - c0 > FD_SYNC_WAIT_CYCLES) {
        ok = 0;
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
    *bcast = ok;
  }
  __syncthreads();
  const bool ok = *bcast != 0;
  __syncthreads();
  return ok;
}

// CTA-wide wait until flags[SF_FWD] >= fwd, flags[SF_BWD] >= bwd, flags[SF_BND] >= bnd,
// flags[SF_FWD2] >= fwd2 and flags[SF_BWD2] >= bwd2.  Thread 0 polls; it gives up (false) after
// FD_SYNC_WAIT_CYCLES without progress of the flags.  `bcast` is a shared int.
__device__ __forceinline__ bool cta_wait_flags(const int* flags, int fwd, int bwd, int bnd,
                                               volatile int* bcast, int fwd2 = 0, int bwd2 = 0) {
  if (threadIdx.x == 0) {
    long long t0 = clock64();
    int ok = 1, last = -1;
    for (;;) {
      const int f0 = flag_load(flags + SF_FWD), f1 = flag_load(flags + SF_BWD),
                f2 = flag_load(flags + SF_BND);
      const int f3 = fwd2 > 0 ? flag_load(flags + SF_FWD2) : 0,
                f4 = bwd2 > 0 ? flag_load(flags + SF_BWD2) : 0;
      if (f0 >= fwd && f1 >= bwd && f2 >= bnd && f3 >= fwd2 && f4 >= bwd2) break;
      const int sum = f0 + f1 + f2 + f3 + f4;
      const long long now = clock64();
      if (sum != last) {
        last = sum;
        t0 = now;
      } else if (now - t0 > FD_SYNC_WAIT_CYCLES) {
        ok = 0;
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
    *bcast = ok;
  }
  __syncthreads();
  const bool ok = *bcast != 0;
  __syncthreads();
  return ok;
}

// Per-configuration force workspace in global memory (the force is split into phases that run
// on different CTAs):  left checkpoints L_b = B_{b ns}...B_1 as (X, T, log D) for b = 1..nb-1,
// right checkpoints (B_Nt...B_{(b-1)ns+1})^H as (X, T, log D) for b = 2..nb, and the
// block-boundary Green's functions G_{(b-1) ns} (column-major) for b = 1..nb, and, when the
// unequal-time Green's function is wanted, its boundary values G((b-1) ns, 0) for b = 2..nb,
// then (response traces) the operator O in FP32 for the tensor-core wraps.
struct FWork {
  double2* base;
  int n, nb;
  __host__ __device__ static size_t stride(int n) { return (size_t)2 * n * n + (n + 1) / 2; }
  // gt: room for the boundary values G((b-1) ns, 0) of the unequal-time Green's function
  // extra: room for that many more (X, T, log D) factors after the boundary Green's functions
  // (force only: the split chains' second forward half, the segmented chains' local products)
  __host__ __device__ static size_t elems(int n, int nb, bool gt, bool op = false,
                                          int extra = 0) {
    return (size_t)2 * (nb - 1) * stride(n) + (size_t)(gt ? 2 : 1) * nb * n * n +
           (op ? ((size_t)n * n + 3) / 4 : 0) + (size_t)extra * stride(n);
  }
  __device__ double2* LX(int b) const { return base + (size_t)(b - 1) * stride(n); }
  __device__ double2* LT(int b) const { return LX(b) + (size_t)n * n; }
  __device__ double* LD(int b) const { return (double*)(LX(b) + (size_t)2 * n * n); }
  __device__ double2* RX(int b) const { return base + (size_t)(nb - 1 + b - 2) * stride(n); }
  __device__ double2* RT(int b) const { return RX(b) + (size_t)n * n; }
  __device__ double* RD(int b) const { return (double*)(RX(b) + (size_t)2 * n * n); }
  // G_{(b-1) ns}; b = nb + 1 wraps to b = 1 (G_Nt = G_0)
  __device__ double2* Gb(int b) const {
    return base + (size_t)2 * (nb - 1) * stride(n) + (size_t)((b - 1) % nb) * n * n;
  }
  // G((b-1) ns, 0), b = 2..nb (column-major); G(0, 0) = G_0 = Gb(1)
  __device__ double2* GT(int b) const {
    return b == 1 ? Gb(1)
                  : base + (size_t)2 * (nb - 1) * stride(n) + (size_t)(nb + b - 1) * n * n;
  }
  // extra factors of the force (no G(tau, 0), no O): i = 0 the split chains' product of blocks
  // h+1..nb; the segmented chains' local products
  __device__ double2* XX(int i) const {
    return base + (size_t)2 * (nb - 1) * stride(n) + (size_t)nb * n * n + (size_t)i * stride(n);
  }
  __device__ double2* XT(int i) const { return XX(i) + (size_t)n * n; }
  __device__ double* XD(int i) const { return (double*)(XX(i) + (size_t)2 * n * n); }
  __device__ double2* SX() const { return XX(0); }
  __device__ double2* ST() const { return XT(0); }
  __device__ double* SD() const { return XD(0); }
  // O (row-major) in FP32, after the G(tau, 0) values when those are kept (gt)
  __device__ float* OF(bool gt) const {
    return (float*)(base + (size_t)2 * (nb - 1) * stride(n) + (size_t)(gt ? 2 : 1) * nb * n * n);
  }
};

// A (configuration, block) work item of the boundary and wrap phases of the force.
struct Task {
  int desc;  // index into the launch's descriptor array
  int b;     // block, 1-based
};

// Chain tasks (Task.b of the chain launch): 0 forward chain, 1 backward chain, 2 + s segment s
// of a time-parallel log det/G split, and the second halves of force chains split at block h.
enum ChainCode { CT_FWD = 0, CT_BWD = 1, CT_SEG = 2, CT_FWD2 = 64, CT_BWD2 = 65 };

// Blocks of a force chain task, forward ascending from `first` to `last`, backward descending.
// Unsplit (h = 0): forward 1..nb with the assembly at the end (log det, G_0), backward nb..2.
// Split at h (Desc.fsplit): forward 1..h, its second half h+1..nb from the identity (local
// products L'_b = B_{b ns}...B_{h ns+1}, the full one in FWork::SX), backward nb..h+1, its second
// half h..2 from the identity (local right products).  The boundary phase merges a local product
// with the first half's last checkpoint (L_b = L'_b L_h, R_b = R'_b R_{h+1}) and forms G_0 and
// log det from L'_nb L_h.  The progress flag counts the checkpoints written, in chain order.
struct ChainSpan {
  bool fwd;
  int first, last;
  int flag;       // SyncFlag index
  bool assemble;  // unsplit forward chain: log det and G_0 at the end
  __device__ int count(int b) const { return fwd ? b - first + 1 : first - b + 1; }
};
__device__ __forceinline__ ChainSpan chain_span(int code, int nb, int h) {
  switch (code) {
    case CT_FWD2: return ChainSpan{true, h + 1, nb, SF_FWD2, false};
    case CT_BWD2: return ChainSpan{false, h, 2, SF_BWD2, false};
    case CT_BWD: return ChainSpan{false, nb, h > 0 ? h + 1 : 2, SF_BWD, false};
    default: return ChainSpan{true, 1, h > 0 ? h : nb, SF_FWD, h == 0};
  }
}

// Segmented chains (Desc.fseg = S, the streamed kernels): forward segment k covers blocks
// k m + 1 .. (k+1) m (m = nb / S), backward segment k blocks nb - k m down to nb - (k+1) m + 1.
// Pass 1 runs segments from the identity in parallel: segment 0 writes its final checkpoints,
// segments 1..S-2 only their local product (FWork::XX).  A prefix task then forms the prefixes
// L_{k m} = (local product of segment k-1) L_{(k-1) m}, k = 2..S-1, in order (a short
// sequential chain of merges whose left factor spans only m blocks) and writes each as that
// checkpoint.  Pass 2 re-runs segments 1..S-1 from their exact prefix, writing their final
// checkpoints (all but the last, which the next prefix forms); the last forward segment ends
// with the assembly.  Backward in mirror image, with suffixes R_{nb - k m + 1} (the last
// backward segment stops at block 2 and writes R_2).  Chain task codes:
// pass 1 (CT_SFA/CT_SBA + k, k = 0..S-2), pass 2 (CT_SFB/CT_SBB + k, k = 1..S-1), and one
// prefix task per direction (CT_SFP/CT_SBP) that forms L_{2m}, ..., L_{(S-1)m} in order.
enum SegCode { CT_SFA = 96, CT_SFB = 112, CT_SBA = 128, CT_SBB = 144, CT_SFP = 160, CT_SBP = 161 };
// Which flag shows a final left checkpoint L_c (c = 1..nb-1) or right checkpoint R_c
// (c = 2..nb), and the value it must reach.
__device__ __forceinline__ void seg_left_ready(int c, int m, int& idx, int& thr) {
  const int k = (c - 1) / m, j = c - k * m;
  if (k == 0) { idx = SF_SEGF; thr = j; }
  else if (j < m) { idx = SF_SEGF + k; thr = j; }
  else { idx = SF_PREF + k + 1; thr = 1; }
}
__device__ __forceinline__ void seg_right_ready(int c, int nb, int m, int& idx, int& thr) {
  const int k = (nb - c) / m, j = nb - c + 1 - k * m;
  if (k == 0) { idx = SF_SEGB; thr = j; }
  else if (j < m) { idx = SF_SEGB + k; thr = j; }
  else { idx = SF_PREB + k + 1; thr = 1; }
}

// Where each working matrix lives: shared memory (offset in bytes from the dynamic smem base)
// or the CTA's global scratch slot (offset in bytes from the slot base).  Each persistent CTA
// owns one slot of `slot_bytes` and reuses it for every configuration it processes; the force
// checkpoints follow the working buffers inside the slot.  Generic pointers let the same code
// run on either memory.
enum Buf {
  B_E = 0,   // real nx*nx
  B_EINV,    // real nx*nx
  B_X0,      // complex nx*nx (column-major)
  B_X1,
  B_T0,
  B_T1,
  B_GLO,     // force only
  B_GHI,
  B_GA,
  B_GB,
  B_NBUF
};

struct Layout {
  int nthreads;
  int num_sms;                 // SMs of the device (CTA wave index -> leader-warp offset)
  int smem_bytes;              // dynamic shared memory per CTA
  int small_off;               // offset (bytes, in smem) of the small-vector area
  int in_smem[B_NBUF];         // 1 = shared memory
  long long off[B_NBUF];       // byte offsets
  long long ws_bytes;          // working buffers kept in global memory (bytes per slot)
  long long slot_bytes;        // ws_bytes + checkpoints (bytes per slot)
};

__host__ __device__ __forceinline__ int small_bytes(int n) {
  // ph 2n, rdiag n, vbuf 2n complex; 10 n doubles; red 64 doubles; perm, piv n ints; misc 32 ints
  return 16 * 5 * n + 8 * 10 * n + 8 * 64 + 4 * 2 * n + 4 * 32;
}

// Layout of the mixed-precision kernels (slice GEMMs on tcgen05).  Byte offsets into dynamic
// shared memory unless stated otherwise.  Operands use the K-major no-swizzle layout of
// fd_tc.cuh: A = E (Np rows x Kp, TF32), B = the current product (2*Np rows: Re then Im, x Kp).
struct MLayout {
  int nthreads;
  int num_sms;
  int smem_bytes;
  int n, Np, Kp, N;      // N = 2*Np MMA columns; Kp = Np
  int tmem_cols;
  int three;             // 1 = split TF32 (hi + lo, 3 MMAs per K step)
  int perm;              // 1 = matrix row i sits in accumulator lane 32*(i%4) + i/4 (spreads
                         //     small matrices over all four TMEM lane quarters / warps)
  int a_hi, a_lo;        // A operand(s): E
  int a2_hi, a2_lo;      // force only: E^{-1}
  int b_hi, b_lo;        // B operand(s); the region also hosts the FP64 block result Xc
  int xc_smem, xn_smem;  // 1 = shared memory, 0 = CTA scratch slot
  long long xc_off, xn_off;
  int t_smem, g_smem;        // 1 = T pair / force G buffers in shared memory
  long long t0_off, t1_off;  // T buffers (shared memory or scratch slot)
  int small_off;
  int bar_off;           // mbarrier (8 B), TMEM address (4 B), queue slot (4 B)
  long long slot_bytes;
  // force only
  long long g_off[4];    // G_lo, G_hi, G_a, G_b (complex128 n*n each)
  long long ws_bytes;    // slot bytes before the checkpoints
};

// Layout of the streamed tensor-core kernels (matrices larger than one tensor-core tile).  Every
// operand lives in global memory in a chunked K-major layout -- K in chunks of 16, then 8-row
// groups, then the four core matrices (8 rows x 4 TF32) along K -- so that the rows of one
// chunk form one contiguous slab that a single bulk copy moves into a shared-memory stage.
//   chains (slice products):  (E Y)^T = Y^T E,  A = Y^T (Mc rows: column j of Y as rows 2j (Re)
//                             and 2j+1 (Im)), B = E (Ne rows), accumulator 128 x Ne per M-tile
//   wraps:  W = M1 Z (A = M1, rows of E padded to Ma; B = Z as rows 2j+part, K = rows of Z), then
//           G = W M2 as C[c, 2r+part] = sum_k M2[c, k] W_part[r, k] (A = M2, B = W by rows),
//           the B rows split into npass passes of Nw rows (TMEM columns)
// Byte offsets into dynamic shared memory unless stated otherwise.
struct BLayout {
  int nthreads, num_sms, smem_bytes;
  int n;
  int Kp;          // K padded to a multiple of 16 (= Ne)
  int Ne;          // rows of E as the chains' B operand (n padded to 16)
  int Ma;          // rows of E / E^{-1} as the wraps' A operand (n padded to 128) = rows of the
                   // prepared chunked copies
  int Mc;          // rows of the chains' A operand (2n padded to 128)
  int Nw, npass;   // wraps: B rows per pass (a multiple of 16, at most 288) and passes
  int Nb;          // wraps: B rows allocated (npass * Nw >= 2n)
  int three;       // split TF32 (hi + lo, 3 MMAs per product)
  int nstages, stage_bytes;
  int a_lo, b_hi, b_lo;  // offsets inside a stage
  int small_off, ph_off, dg_off, bar_off;
  int tmem_cols;
  // CTA scratch slot (bytes from the slot base)
  long long a_off;                       // chains: A operand, hi then lo (Mc * Kp floats each)
  long long xc_off, xn_off, t0_off, t1_off;  // chains: FP64 n x n complex
  long long b1_off, b2_off;              // wraps: B operands, hi then lo (Nb * Kp floats each)
  long long slot_bytes;
};

// status codes written per configuration (device side); the host pre-fills ST_PENDING and the
// phases of a configuration combine theirs with atomicMax (any failure wins over OK)
enum { ST_OK = 0, ST_NUMERIC = 1, ST_TIMEOUT = 2, ST_PENDING = -1 };

}  // namespace fd
