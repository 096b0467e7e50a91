// fd_bss.cu -- local (BSS) updates of the auxiliary field at one time slice (Section 3).
//
// The sites of the slice are visited in order.  With G = G_{t-1} (slice t acting first) and the
// proposal phi_x -> phi_x + dphi_x, B_t becomes B_t (1 + delta e_x e_x^T), delta = e^{i dphi_x} - 1,
// and the matrix determinant lemma gives the ratio of determinants
//   r = det(1 + P') / det(1 + P) = 1 + delta (1 - G_xx),
// while Sherman-Morrison updates the Green's function of an accepted proposal:
//   G'_ij = G_ij - a_i b_j,  a_i = (delta / r) (delta_ix - G_ix),  b_j = G_xj.
// Accepted iff u_x < |r| w_x.  A rejected proposal costs O(1), an accepted one O(nx^2) -- the
// complexity the paper states for BSS updates.  One CTA per configuration.
//
// Precision.  The nx^2 rank-1 updates are the bulk of the work, and on this GPU an SM retires
// FP64 instructions some seventy times slower than FP32 ones, so for nx <= kBssDfMax the slice
// keeps G in shared memory as double-float pairs (fd_df.cuh, ~46 significant bits) and updates
// it with FP32 instructions, converting from and back to FP64 once per call; the ratios,
// decisions and delta / r use the same pair arithmetic (FP64 where |r|^2 or (u/w)^2 leaves
// [2^-100, 2^100]).  Larger nx (or a G with entries beyond 2^100, outside the FP32 exponent
// range the pairs need) runs every step in FP64 on G in place in global memory.  The change of
// log det is summed in FP64.
#include "fd_common.cuh"
#include "fd_df.cuh"
#include "fd_kernels.h"

namespace fd {

namespace {

constexpr int kBssDfMax = 110;  // 16 nx^2 + 100 nx bytes of shared memory <= 205 KB

// Per-CTA shared memory (dynamic), sized for the largest nx of the launch.
struct BssSmem {
  df::c4* Gs;     // nx*nx df G (only when the df path is available)
  df::c4* Dg;     // the diagonal of Gs, kept by the deciding warp
  double2* a;     // staged a_i (df c4 or FP64 double2, 16 bytes each)
  double2* b;     // staged b_j
  double2* dl;    // delta_x
  double2* rs;    // r_x of accepted proposals
  double* v;      // u_x / w_x, then log|r_x|
  double* vv;     // (u_x / w_x)^2 or -1 when out of the range where squaring is safe, then arg r_x
  int* acc;       // decisions
};

__device__ __forceinline__ BssSmem bss_smem(char* base, int maxn, bool df_path) {
  BssSmem s;
  size_t off = 0;
  s.Gs = (df::c4*)base;
  if (df_path) off += (size_t)maxn * maxn * sizeof(df::c4);
  s.Dg = (df::c4*)(base + off);
  off += (size_t)maxn * 16;
  s.a = (double2*)(base + off);
  off += (size_t)maxn * 16;
  s.b = (double2*)(base + off);
  off += (size_t)maxn * 16;
  s.dl = (double2*)(base + off);
  off += (size_t)maxn * 16;
  s.rs = (double2*)(base + off);
  off += (size_t)maxn * 16;
  s.v = (double*)(base + off);
  off += (size_t)maxn * 8;
  s.vv = (double*)(base + off);
  off += (size_t)maxn * 8;
  s.acc = (int*)(base + off);
  return s;
}

// FP64 path: the Metropolis decision and delta / r for site x from G_xx (one thread).
__device__ __forceinline__ bool bss_decide(const BssSmem& s, int x, double gre, double gim,
                                           cplx& f) {
  const double2 d = s.dl[x];
  const double ore = 1.0 - gre, oim = -gim;
  const double rre = fma(d.x, ore, fma(-d.y, oim, 1.0));
  const double rim = fma(d.x, oim, d.y * ore);
  const double t = fma(rre, rre, rim * rim);  // |r|^2
  const double vv = s.vv[x];
  const bool normal = t > 1e-280 && t < 1e280;
  // u < |r| w  <=>  (u / w)^2 < |r|^2, squared where nothing under- or overflows
  const bool acc = (vv >= 0.0 && normal) ? vv < t : s.v[x] < sqrt(t);
  if (acc) {
    if (normal) {
      const double inv = 1.0 / t;  // delta conj(r) / |r|^2
      f = cx(fma(d.x, rre, d.y * rim) * inv, fma(d.y, rre, -d.x * rim) * inv);
    } else {
      f = cdiv(cx(d.x, d.y), cx(rre, rim));
    }
    s.rs[x] = make_double2(rre, rim);
  }
  s.acc[x] = acc;
  return acc;
}

// df path: the same decision in double-float arithmetic on the FP32 pipes (the FP64 unit would
// make this serial chain the longest part of a site), from the deciding warp's diagonal.  Where
// |r|^2 or (u / w)^2 leaves [2^-100, 2^100] it falls back to FP64 on the joined values.
__device__ __forceinline__ bool bss_decide_df(const BssSmem& s, int x, df::c4& f) {
  const df::c4 d = ((const df::c4*)s.dl)[x];
  const df::c4 one = {1.f, 0.f, 0.f, 0.f};
  const df::c4 r = df::cms(one, d, df::add_re(s.Dg[x], -1.f));  // 1 + delta (1 - G_xx)
  float th, tl;
  df::abs2(r, th, tl);
  const float2 vv = ((const float2*)s.vv)[x];
  bool acc;
  if (vv.x >= 0.f && th > 0x1p-100f && th < 0x1p100f) {
    acc = df::greater(th, tl, vv.x, vv.y);  // (u / w)^2 < |r|^2
    if (acc) {
      float yh, yl;
      df::recip(th, tl, yh, yl);
      const df::c4 mconj = {-r.x, -r.y, r.z, r.w};
      const df::c4 zero = {0.f, 0.f, 0.f, 0.f};
      f = df::scale(df::cms(zero, d, mconj), yh, yl);  // delta conj(r) / |r|^2
    }
  } else {
    const double rre = df::join(r.x, r.y), rim = df::join(r.z, r.w);
    acc = s.v[x] < sqrt(fma(rre, rre, rim * rim));
    if (acc) {
      const cplx fz = cdiv(cx(df::join(d.x, d.y), df::join(d.z, d.w)), cx(rre, rim));
      f = df::csplit(fz.re, fz.im);
    }
  }
  if (acc) ((df::c4*)s.rs)[x] = r;
  s.acc[x] = acc;
  return acc;
}

// df path: decide sites y, y+1, ... until one is accepted (its delta / r goes to *f); returns
// that site or n.  Rejected sites change nothing, so they need no barrier.
__device__ __forceinline__ int bss_next_df(const BssSmem& s, int y, int n, df::c4* f) {
  for (; y < n; ++y) {
    df::c4 fz;
    if (bss_decide_df(s, y, fz)) {
      *f = fz;
      return y;
    }
  }
  return n;
}

}  // namespace

// One CTA per configuration (grid-stride over the batch).  In the df path warp 0 decides while
// warps 1.. update: after the staging of accepted site x, warp 0 applies the same rank-1 update
// to its own copy of the diagonal (bitwise the values the other warps write into Gs) and decides
// x+1, x+2, ... until the next acceptance, overlapped with the nx^2 update.
__global__ void __launch_bounds__(544) k_bss(const BssSlice* __restrict__ slices, int batch,
                                              int maxn, int df_path, double* dlogdet) {
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ df::c4 fdf;
  __shared__ double2 f64;
  __shared__ int accept[2];  // FP64 path, double-buffered: site x uses accept[x & 1]
  __shared__ int next;       // df path: the next accepted site (n: none)
  const BssSmem s = bss_smem(smem_raw, maxn, df_path != 0);
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int c = blockIdx.x; c < batch; c += gridDim.x) {
    const BssSlice q = slices[c];
    const int n = q.nx;
    // df path: G -> shared memory as df pairs, unless an entry is beyond 2^100 (or not finite)
    int big = 0;
    if (df_path) {
      for (int e = tid; e < n * n; e += bd) {
        const double2 g = q.G[e];
        const uint64_t mx = df::dbits(g.x) & 0x7ff0000000000000ull;
        const uint64_t my = df::dbits(g.y) & 0x7ff0000000000000ull;
        big |= (mx >= (uint64_t)(1023 + 100) << 52) | (my >= (uint64_t)(1023 + 100) << 52);
        s.Gs[e] = df::csplit(g.x, g.y);
      }
    }
    const bool use_df = df_path && !__syncthreads_or(big);
    for (int x = tid; x < n; x += bd) {
      double sn, cs;
      sincos(q.dphi[x], &sn, &cs);
      const double v = q.u[x] / q.w[x];
      const double vv = v * v;
      s.v[x] = v;
      s.acc[x] = 0;
      if (use_df) {
        ((df::c4*)s.dl)[x] = df::csplit(cs - 1.0, sn);
        float2 p = make_float2(-1.f, 0.f);
        if (vv >= 0x1p-100 && vv <= 0x1p100) df::split(vv, p.x, p.y);
        ((float2*)s.vv)[x] = p;
        s.Dg[x] = s.Gs[x * n + x];
      } else {
        s.dl[x] = make_double2(cs - 1.0, sn);
        s.vv[x] = (vv >= 1e-280 && vv <= 1e280) ? vv : -1.0;
      }
    }
    __syncthreads();
    if (use_df) {
      // updaters: threads 32.. ; thread layout column j, rows i0, i0 + rpp, ...
      const int u = tid - 32, rpp = (bd - 32) / n;
      const int j = u >= 0 ? u % n : 0, i0 = u >= 0 ? u / n : rpp;
      if (tid == 0) next = bss_next_df(s, 0, n, &fdf);
      __syncthreads();
      df::c4* A = (df::c4*)s.a;
      df::c4* B = (df::c4*)s.b;
      const df::c4 zero = {0.f, 0.f, 0.f, 0.f};
      for (;;) {
        const int x = next;
        if (x >= n) break;
        if (u >= 0) {  // staging on the updating warps (the deciding warp's sub-partition is
                       // the busiest)
          const df::c4 f = fdf;
          for (int i = u; i < n; i += bd - 32) {
            df::c4 g = s.Gs[i * n + x];  // G_ix - delta_ix; a_i = -(delta / r)(G_ix - delta_ix)
            if (i == x) g = df::add_re(g, -1.f);
            A[i] = df::cms(zero, f, g);
            B[i] = s.Gs[x * n + i];
          }
        }
        __syncthreads();
        if (tid < 32) {
          // only the sites still to be decided need their diagonal entry
          for (int i = x + 1 + tid; i < n; i += 32) s.Dg[i] = df::cms(s.Dg[i], A[i], B[i]);
          __syncwarp();
          if (tid == 0) next = bss_next_df(s, x + 1, n, &fdf);
        } else if (i0 < rpp) {
          const df::c4 bj = B[j];
          int i = i0;
          for (; i + rpp < n; i += 2 * rpp) {  // two rows per trip, loads first
            const int e0 = i * n + j, e1 = e0 + rpp * n;
            const df::c4 g0 = s.Gs[e0], a0 = A[i], g1 = s.Gs[e1], a1 = A[i + rpp];
            s.Gs[e0] = df::cms(g0, a0, bj);
            s.Gs[e1] = df::cms(g1, a1, bj);
          }
          if (i < n) s.Gs[i * n + j] = df::cms(s.Gs[i * n + j], A[i], bj);
        }
        __syncthreads();
      }
    } else {
      for (int x = 0; x < n; ++x) {
        if (tid == 0) {
          const double2 g = q.G[(size_t)x * n + x];
          cplx f;
          const bool a = bss_decide(s, x, g.x, g.y, f);
          if (a) f64 = make_double2(f.re, f.im);
          accept[x & 1] = a;
        }
        __syncthreads();
        if (!accept[x & 1]) continue;  // uniform: every thread reads the same flag
        const cplx f = cx(f64.x, f64.y);
        for (int i = tid; i < n; i += bd) {
          const double2 g = q.G[(size_t)i * n + x];
          const cplx col = cx((i == x ? 1.0 : 0.0) - g.x, -g.y);
          const cplx a = f * col;
          s.a[i] = make_double2(a.re, a.im);
          s.b[i] = q.G[(size_t)x * n + i];
        }
        __syncthreads();
        for (int e = tid; e < n * n; e += bd) {
          const int i = e / n, jj = e - i * n;
          const double2 a = s.a[i], b = s.b[jj];
          const double2 g = q.G[e];
          q.G[e] = make_double2(fma(-a.x, b.x, fma(a.y, b.y, g.x)),
                                fma(-a.x, b.y, fma(-a.y, b.x, g.y)));
        }
        __syncthreads();
      }
    }
    // outputs: field row, decisions, G back to FP64; log|r_x| (k < n) and arg r_x (k >= n) of
    // the accepted sites on separate threads
    for (int k = tid; k < 2 * n; k += bd) {
      const int x = k < n ? k : k - n;
      const int a = s.acc[x];
      double val = 0.0;
      if (a) {
        double rre, rim;
        if (use_df) {
          const df::c4 r = ((const df::c4*)s.rs)[x];
          rre = df::join(r.x, r.y);
          rim = df::join(r.z, r.w);
        } else {
          rre = s.rs[x].x;
          rim = s.rs[x].y;
        }
        if (k < n) {
          const double t = fma(rre, rre, rim * rim);
          val = (t > 1e-280 && t < 1e280) ? 0.5 * log(t) : log(hypot(rre, rim));
        } else {
          val = atan2(rim, rre);
        }
      }
      if (k < n) {
        q.acc[x] = a;
        if (a) q.phi[x] += q.dphi[x];
        s.v[x] = val;
      } else {
        s.vv[x] = val;
      }
    }
    if (use_df) {
      for (int e = tid; e < n * n; e += bd) {
        const df::c4 g = s.Gs[e];
        q.G[e] = make_double2(df::join(g.x, g.y), df::join(g.z, g.w));
      }
    }
    __syncthreads();
    if (tid < 32) {
      double lr = 0.0, la = 0.0;
      for (int x = tid; x < n; x += 32) {
        lr += s.v[x];
        la += s.vv[x];
      }
      for (int o = 16; o > 0; o >>= 1) {
        lr += __shfl_down_sync(0xffffffffu, lr, o);
        la += __shfl_down_sync(0xffffffffu, la, o);
      }
      if (tid == 0) {
        const double pi = 3.14159265358979323846;
        double y = remainder(la, 2.0 * pi);  // (-pi, pi]
        if (y <= -pi) y += 2.0 * pi;
        dlogdet[2 * c] = lr;
        dlogdet[2 * c + 1] = y;
      }
    }
    __syncthreads();
  }
}

size_t bss_smem_bytes(int maxn, bool df_path) {
  return (df_path ? (size_t)maxn * maxn * sizeof(df::c4) : 0) + (size_t)maxn * 100;
}

// df path: 4, 8 or 16 updating warps (a multiple of the SM's four sub-partitions) and the
// deciding warp; the FP64 path uses them all alike.
int bss_threads(int maxn) { return 32 + (maxn <= 24 ? 128 : maxn <= 48 ? 256 : 512); }

cudaError_t launch_bss(const BssSlice* slices, int batch, int maxn, double* dlogdet, int grid,
                       cudaStream_t stream) {
  const bool df_path = maxn <= kBssDfMax;
  const size_t smem = bss_smem_bytes(maxn, df_path);
  cudaError_t e = cudaFuncSetAttribute(k_bss, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_bss<<<grid, bss_threads(maxn), smem, stream>>>(slices, batch, maxn, df_path ? 1 : 0, dlogdet);
  return cudaGetLastError();
}

}  // namespace fd
