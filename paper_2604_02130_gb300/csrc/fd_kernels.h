// fd_kernels.h -- launchers shared between the host runtime and the kernel translation units.
#pragma once

#include "fd_common.cuh"

namespace fd {

// FP64 path
void launch_fwd_fp64(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                     const Layout& L, int grid, cudaStream_t stream);
void launch_force_fp64(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                       const Layout& L, int grid, cudaStream_t stream);
cudaError_t set_smem_fp64(int bytes);
int occupancy_fp64(bool force, int nthreads, int smem_bytes);  // -1 on error
cudaError_t attrs_fp64(bool force, cudaFuncAttributes* a);

// mixed path (tcgen05 slice GEMMs)
void launch_fwd_mixed(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                      const MLayout& L, int grid, cudaStream_t stream);
void launch_force_mixed(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                        const MLayout& L, int grid, cudaStream_t stream);
cudaError_t set_smem_mixed(int bytes);
int occupancy_mixed(bool force, int nthreads, int smem_bytes);  // -1 on error
cudaError_t attrs_mixed(bool force, cudaFuncAttributes* a);

// FP64 throughput probe
cudaError_t run_fp64_probe(int grid, int threads, int iters, double* out, cudaStream_t stream);

}  // namespace fd
