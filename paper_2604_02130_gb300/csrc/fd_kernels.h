// fd_kernels.h -- launchers shared between the host runtime and the kernel translation units.
#pragma once

#include "fd_common.cuh"

namespace fd {

// Intermediate-volume variant (Sections 8-9): the hopping factor of a slice applied as
// prod_k (1 + gamma_k K) with the sparse K (q entries per row, row i at [i*q, i*q + q)); one
// entry per configuration, indexed by the user index of the descriptor.
#define FD_SPARSE_NFAC_MAX 8
struct SparseHop {
  const int* col;
  const double* val;
  int q, nfac;
  double2 gamma[FD_SPARSE_NFAC_MAX];
};

// One configuration of a local (BSS) slice update (the public fd_bss_slice, device view).
struct BssSlice {
  int nx, reserved;
  double2* G;          // nx*nx row-major, in/out
  double* phi;         // nx, in/out: the field of the slice
  const double* dphi;  // nx proposals
  const double* u;     // nx uniform random numbers
  const double* w;     // nx other-weight ratios
  int* acc;            // nx out: accepted
};

// FP64 path.  hops: null, or the product-form tables of the configurations (log det/G only).
void launch_fwd_fp64(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                     const Layout& L, int grid, cudaStream_t stream,
                     const SparseHop* hops = nullptr);
// force phases: A chains (2 tasks per configuration: Task.b = 0 forward, 1 backward),
// B boundary Green's functions, C wraps
void launch_chain_fp64(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                       char* scratch, const Layout& L, int grid, cudaStream_t stream);
// pdl: launch as a programmatic dependent of the previous kernel (tasks wait on the flags)
// merge: the variant that merges split chains' checkpoints first (attrs/occupancy: which 9)
void launch_boundary_fp64(const Desc* descs, const Task* tasks, int ntasks, int* queue,
                          int* status, char* scratch, const Layout& L, int grid,
                          cudaStream_t stream, bool pdl, bool merge);
void launch_wrap_fp64(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                      char* scratch, const Layout& L, int grid, cudaStream_t stream, bool pdl);
// time-parallel log det/G: merge of the segment products and assembly (kernel id 8)
void launch_merge_fp64(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                       const Layout& L, int grid, cudaStream_t stream);
cudaError_t set_smem_fp64(int bytes);
// kernel ids: 0 log det/G, 1 force chains, 2 boundary, 3 wraps
int occupancy_fp64(int which, int nthreads, int smem_bytes);  // -1 on error
cudaError_t attrs_fp64(int which, cudaFuncAttributes* a);

// mixed path (tcgen05 slice GEMMs)
void launch_fwd_mixed(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                      const MLayout& L, int grid, cudaStream_t stream);
// seg: the variant with the segmented chains' tasks (attrs/occupancy: which 9)
void launch_chain_mixed(const Desc* descs, const Task* tasks, int ntasks, int* queue,
                        int* status, char* scratch, const MLayout& L, int grid,
                        cudaStream_t stream, bool seg);
void launch_wrap_mixed(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                       char* scratch, const MLayout& L, int grid, cudaStream_t stream, bool pdl);
cudaError_t set_smem_mixed(int bytes);
// kernel ids as for the FP64 kernels: 0 log det/G, 1 force chains, 3 wraps
int occupancy_mixed(int which, int nthreads, int smem_bytes);  // -1 on error
cudaError_t attrs_mixed(int which, cudaFuncAttributes* a);

// streamed tensor-core path (matrices larger than one shared-memory tile): chunked TF32
// copies of the call's distinct E / E^{-1} (rows padded to Ma), then the chains and wraps
#define FD_BIG_PREP_MAX 16
struct BigPrepItem {
  const double* src;  // n x n row-major FP64
  float* dst;         // hi (Ma * Kp floats), then lo
};
struct BigPrep {
  BigPrepItem item[FD_BIG_PREP_MAX];
  int count, n, Ma, Kp, three;
};
cudaError_t launch_prep_big(const BigPrep& P, cudaStream_t stream);
void launch_chain_big(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                      char* scratch, const BLayout& L, int grid, cudaStream_t stream);
void launch_wrap_big(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                     char* scratch, const BLayout& L, int grid, cudaStream_t stream, bool pdl);
// mixed force, streamed classes: boundary Green's functions in double-float
void launch_boundary_big(const Desc* descs, const Task* tasks, int ntasks, int* queue,
                         int* status, char* scratch, const BLayout& L, int grid,
                         cudaStream_t stream, bool pdl);
cudaError_t set_smem_big(int bytes);
// kernel ids: 1 chains, 2 boundary Green's functions, 3 wraps
cudaError_t attrs_big(int which, cudaFuncAttributes* a);
// df numbers of shared memory: the streamed chains' df QR at size n, the boundary Green's
// function's GEMM tiles
int big_qr_vcap(int n);
int big_bound_tiles();

// local (BSS) slice updates (one CTA per configuration; G in shared memory as double-float
// pairs when maxn is small enough, else FP64 in place)
cudaError_t launch_bss(const BssSlice* slices, int batch, int maxn, double* dlogdet, int grid,
                       cudaStream_t stream);

// FP64 throughput probe
cudaError_t run_fp64_probe(int grid, int threads, int iters, double* out, cudaStream_t stream);
cudaError_t run_fp64_issue(double* out3);
// self-check of the FP64 refinements beside CUDA's IEEE operations (16 values per argument)
cudaError_t run_refine_check(const double* x, const double* y, const double* z, int n,
                             double* out, cudaStream_t stream);

}  // namespace fd
