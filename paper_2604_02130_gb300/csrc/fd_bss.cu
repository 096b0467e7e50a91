// fd_bss.cu -- local (BSS) updates of the auxiliary field at one time slice (Section 3).
//
// The sites of the slice are visited in order.  With G = G_{t-1} (slice t acting first) and the
// proposal phi_x -> phi_x + dphi_x, B_t becomes B_t (1 + delta e_x e_x^T), delta = e^{i dphi_x} - 1,
// and the matrix determinant lemma gives the ratio of determinants
//   r = det(1 + P') / det(1 + P) = 1 + delta (1 - G_xx),
// while Sherman-Morrison updates the Green's function of an accepted proposal:
//   G'_ij = G_ij - (delta / r) (delta_ix - G_ix) G_xj.
// Accepted iff u_x < |r| w_x.  A rejected proposal costs O(1), an accepted one O(nx^2) -- the
// complexity the paper states for BSS updates.  One CTA per configuration, FP64.
#include "fd_common.cuh"
#include "fd_kernels.h"

namespace fd {

__global__ void __launch_bounds__(256) k_bss_fp64(const BssSlice* __restrict__ slices, int batch,
                                                   double* dlogdet) {
  extern __shared__ __align__(16) double2 sh[];
  __shared__ double2 fact;
  __shared__ int accept;
  for (int c = blockIdx.x; c < batch; c += gridDim.x) {
    const BssSlice q = slices[c];
    const int n = q.nx;
    double2* col = sh;      // delta_ix - G_ix
    double2* row = sh + n;  // G_xj
    double lre = 0.0, lim = 0.0;
    for (int x = 0; x < n; ++x) {
      if (threadIdx.x == 0) {
        const double2 g = q.G[(size_t)x * n + x];
        double sn, cs;
        sincos(q.dphi[x], &sn, &cs);
        const cplx delta = cx(cs - 1.0, sn);
        const cplx r = cx(1.0, 0.0) + delta * cx(1.0 - g.x, -g.y);
        const double ar = hypot(r.re, r.im);
        const int acc = q.u[x] < ar * q.w[x];
        if (acc) {
          const cplx f = cdiv(delta, r);
          fact = make_double2(f.re, f.im);
          lre += log(ar);
          lim += atan2(r.im, r.re);
          q.phi[x] += q.dphi[x];
        }
        q.acc[x] = acc;
        accept = acc;
      }
      __syncthreads();
      if (accept) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          const double2 gi = q.G[(size_t)i * n + x];
          col[i] = make_double2((i == x ? 1.0 : 0.0) - gi.x, -gi.y);
          row[i] = q.G[(size_t)x * n + i];
        }
        __syncthreads();
        const cplx f = cx(fact.x, fact.y);
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
          const int i = e / n, j = e % n;
          const cplx a = f * cx(col[i].x, col[i].y);
          const cplx upd = a * cx(row[j].x, row[j].y);
          q.G[e] = make_double2(q.G[e].x - upd.re, q.G[e].y - upd.im);
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double pi = 3.14159265358979323846;
      double y = remainder(lim, 2.0 * pi);  // (-pi, pi]
      if (y <= -pi) y += 2.0 * pi;
      dlogdet[2 * c] = lre;
      dlogdet[2 * c + 1] = y;
    }
    __syncthreads();
  }
}

void launch_bss_fp64(const BssSlice* slices, int batch, int maxn, double* dlogdet, int grid,
                     cudaStream_t stream) {
  k_bss_fp64<<<grid, 256, (size_t)2 * maxn * sizeof(double2), stream>>>(slices, batch, dlogdet);
}

}  // namespace fd
