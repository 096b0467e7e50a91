// fd_kernels_mixed.cu -- mixed-precision path: the slice products X <- E diag(e^{i phi_t}) X run
// on the tcgen05 tensor cores (TF32 operands, FP32 accumulation in TMEM), the QR
// re-orthogonalisation every n_stab slices, the scale separation and the assembly stay FP64
// (the same CTA routines as the FP64 path).
//
// Per slice one CTA issues, from a single thread, ceil(Nx/8) MMAs of shape 128 x 2Np x 8
// (x3 for split TF32):  D[i, j] = sum_k E[i, k] Y[k, j], with A = E (rows i, K-major) and
// B = Y stored as 2Np rows (Re Y[:, j], then Im Y[:, j]) with K = the row index of Y, so the
// accumulator holds row i of Re and Im of the product in TMEM lane i.  The epilogue reads each
// lane's row, multiplies it by the next slice's phase e^{i phi_{t+1, i}} (the diagonal factor of
// the next slice, fused here) and writes it back as the next B operand.  After the last slice of
// a block the FP32 result is widened to FP64 for the QR.
#include "fd_fp64.cuh"
#include "fd_kernels.h"
#include "fd_tc.cuh"

namespace fd {

// mbarrier waits give up after about one second at ~2 GHz
#define FD_WAIT_CYCLES (2LL * 1000 * 1000 * 1000)

struct MixedSmem {
  float* a_hi;
  float* a_lo;
  float* b_hi;
  float* b_lo;
  double2* Xc;
  double2* Xn;
  uint64_t* mbar;
  uint32_t* taddr;
  int* qslot;
};

__device__ __forceinline__ MixedSmem mixed_smem(char* smem, char* slot, const MLayout& L) {
  MixedSmem m;
  m.a_hi = (float*)(smem + L.a_hi);
  m.a_lo = L.three ? (float*)(smem + L.a_lo) : nullptr;
  m.b_hi = (float*)(smem + L.b_hi);
  m.b_lo = L.three ? (float*)(smem + L.b_lo) : nullptr;
  m.Xc = L.xc_smem ? (double2*)(smem + L.xc_off) : (double2*)(slot + L.xc_off);
  m.Xn = L.xn_smem ? (double2*)(smem + L.xn_off) : (double2*)(slot + L.xn_off);
  m.mbar = (uint64_t*)(smem + L.bar_off);
  m.taddr = (uint32_t*)(smem + L.bar_off + 8);
  m.qslot = (int*)(smem + L.bar_off + 12);
  return m;
}

// A operand: E (n x n FP64, symmetric) -> TF32 (hi, and lo = E - hi for the split mode), zero
// padded to Np x Kp.
// Accumulator lane of matrix row i, and back.
__device__ __forceinline__ int lane_of_row(const MLayout& L, int i) {
  return L.perm ? 32 * (i & 3) + (i >> 2) : i;
}
__device__ __forceinline__ int row_of_lane(const MLayout& L, int l) {
  return L.perm ? 4 * (l & 31) + (l >> 5) : l;
}

// A operand from E: the n matrix rows (at their permuted lanes), K padded with zeros.  Rows
// that hold no matrix row are not written: with the lane permutation they belong to other
// operands that share the 128-row footprint (their accumulator lanes are never read).
__device__ void fill_a(const MLayout& L, float* a_hi, float* a_lo, const double* E) {
  const int n = L.n, Kp = L.Kp;
  const int rows = L.perm ? n : L.Np;
  for (int e = tid(); e < rows * Kp; e += nthr()) {
    const int i = e / Kp, k = e % Kp;
    const int r = lane_of_row(L, i);
    double v = (i < n && k < n) ? E[i * n + k] : 0.0;
    float f = (float)v;
    float hi = tc::to_tf32(f);
    uint32_t o = tc::kmaj_off(r, k, Kp) >> 2;
    a_hi[o] = hi;
    if (L.three) a_lo[o] = tc::to_tf32(f - hi);
  }
}

// One slice GEMM on the tensor core: issue (single thread), commit, bounded wait.
// Returns false on a timeout (uniform across the CTA).
__device__ bool mma_ab(const MLayout& L, const MixedSmem& m, const float* a_hi, const float* a_lo,
                       uint32_t tbase, uint32_t& phase) {
  tc::fence_proxy_async();
  __syncthreads();
  if (tid() == 0) {
    tc::fence_after();
    const uint32_t idesc = tc::idesc_tf32(128, L.N);
    const uint32_t sbo = (uint32_t)(L.Kp / 4) * 128u;
    const uint32_t ah = tc::smem_u32(a_hi), bh = tc::smem_u32(m.b_hi);
    const uint32_t al = L.three ? tc::smem_u32(a_lo) : 0u, bl = L.three ? tc::smem_u32(m.b_lo) : 0u;
    for (int s = 0; s < L.Kp / 8; ++s) {
      const uint32_t o = 256u * s;
      tc::mma_tf32(tbase, tc::make_desc(ah + o, 128, sbo), tc::make_desc(bh + o, 128, sbo), idesc,
                   s > 0);
      if (L.three) {
        tc::mma_tf32(tbase, tc::make_desc(ah + o, 128, sbo), tc::make_desc(bl + o, 128, sbo),
                     idesc, 1);
        tc::mma_tf32(tbase, tc::make_desc(al + o, 128, sbo), tc::make_desc(bh + o, 128, sbo),
                     idesc, 1);
      }
    }
    tc::mma_commit(m.mbar);
  }
  bool ok = tc::mbar_wait(m.mbar, phase, FD_WAIT_CYCLES);
  phase ^= 1u;
  int bad = __syncthreads_or(!ok);
  tc::fence_after();
  return bad == 0;
}
__device__ __forceinline__ bool slice_mma(const MLayout& L, const MixedSmem& m, uint32_t tbase,
                                          uint32_t& phase) {
  return mma_ab(L, m, m.a_hi, m.a_lo, tbase, phase);
}

// Scale factor per row or column: p[x] (or its conjugate), or 1 when p == nullptr.  FP32: the
// epilogue and the operand fills work at the precision of the TF32 operands they produce (the
// FP64 pipe of this GPU is 1/64 of the FP32 rate).
struct Scale {
  const float2* p;
  bool cj;
  __device__ __forceinline__ float2 at(int x) const {
    if (!p) return make_float2(1.f, 0.f);
    float2 v = p[x];
    return cj ? make_float2(v.x, -v.y) : v;
  }
};
__device__ __forceinline__ float2 cmul32(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// phase vector e^{i s phi} of one slice in FP32
__device__ __forceinline__ void cta_phase32(int n, float2* ph, const double* phi_row, float s) {
  for (int x = tid(); x < n; x += nthr()) {
    float sn, cs;
    sincosf((float)phi_row[x], &sn, &cs);
    ph[x] = make_float2(cs, s * sn);
  }
}

enum EpiMode { TO_B_K = 0, TO_B_N = 1, TO_F32 = 2, NONE = 3 };

__device__ __forceinline__ void put_b(const MLayout& L, const MixedSmem& m, int row, int k,
                                      float v) {
  float hi = tc::to_tf32(v);
  uint32_t o = tc::kmaj_off(row, k, L.Kp) >> 2;
  m.b_hi[o] = hi;
  if (L.three) m.b_lo[o] = tc::to_tf32(v - hi);
}

// Response trace of a wrapped Green's function held in TMEM as G[c, l] = trs(l) v(l, c) tcs(c):
// *out = sum_{l,c} O[l n + c] G[c, l] = tr(O G), O row-major FP32; slot: one float2 per warp.
struct Trace {
  const float* O;  // null: no trace
  Scale rs, cs;
  float2* slot;
  double2* out;
};

// Epilogue of one MMA.  TMEM lane l (< n) holds v(l, c) = D[l, c] + i D[l, Np + c], c < n.
//   TO_B_K : B(n = c, k = l) = rs(l) v cs(c)   (the lane indexes K: slices, right products)
//   TO_B_N : B(n = l, k = c) = rs(l) v cs(c)   (the lane indexes N: wraps)
//   TO_F32 : out[l + c n]    = rs(l) v cs(c)   (column-major FP32 staging, out read as float2;
//            stage_to_fp64 converts it with full warps afterwards)
// diag (optional): diag[l] = v(l,l) in FP32 (shared memory), the diagonal of a wrapped G for a
// force row F = i (1 - G_ll); emit_force_row32 converts it after the epilogue's barrier (the
// FP64 conversions then run on full warps instead of one lane per instruction).
// tr (optional): the response trace above.
template <int MODE>
__device__ void epilogue(const MLayout& L, const MixedSmem& m, uint32_t tbase, Scale rs,
                         Scale cs, double2* out, float2* diag,
                         const Trace& tr = Trace{nullptr, {nullptr, false}, {nullptr, false},
                                                 nullptr, nullptr}) {
  const int n = L.n, Np = L.Np;
  const int w = warp_id(), nw = nwarps();
  const int quad = w & 3;
  const int half = w >> 2;
  const int nhalf = nw > 4 ? 2 : 1;
  const int l = row_of_lane(L, quad * 32 + lane_id());  // matrix row held by this thread
  const int first_row = row_of_lane(L, quad * 32);
  float2 acc = make_float2(0.f, 0.f);
  if (first_row < n) {
    const uint32_t lane_base = tbase + ((uint32_t)(quad * 32) << 16);
    const int nchunk = (Np + 15) / 16;
    const float2 r = l < n ? rs.at(l) : make_float2(1.f, 0.f);
    const float2 tr_r = (tr.O && l < n) ? tr.rs.at(l) : make_float2(1.f, 0.f);
    for (int c = half; c < nchunk; c += nhalf) {
      float re[16], im[16];
      tc::tmem_ld16(lane_base + (uint32_t)(c * 16), re);
      tc::tmem_ld16(lane_base + (uint32_t)(Np + c * 16), im);
      if (l < n) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int j = c * 16 + u;
          if (j < n) {
            const float2 v = make_float2(re[u], im[u]);
            if (diag && j == l) diag[l] = v;
            if (tr.O) {
              const float o = tr.O[l * n + j];
              const float2 g = cmul32(cmul32(tr_r, v), tr.cs.at(j));
              acc.x = fmaf(o, g.x, acc.x);
              acc.y = fmaf(o, g.y, acc.y);
            }
            if (MODE == NONE) continue;
            const float2 y = cmul32(cmul32(r, v), cs.at(j));
            if (MODE == TO_B_K) {
              put_b(L, m, j, l, y.x);
              put_b(L, m, Np + j, l, y.y);
            } else if (MODE == TO_B_N) {
              put_b(L, m, l, j, y.x);
              put_b(L, m, Np + l, j, y.y);
            } else {
              ((float2*)out)[l + j * n] = y;
            }
          }
        }
      }
    }
  }
  if (tr.O) {
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane_id() == 0) tr.slot[w] = acc;
  }
  tc::fence_before();
  __syncthreads();
  if (tr.O) {
    if (tid() == 0) {
      float2 t = make_float2(0.f, 0.f);
      for (int k = 0; k < nw; ++k) {
        t.x += tr.slot[k].x;
        t.y += tr.slot[k].y;
      }
      *tr.out = make_double2((double)t.x, (double)t.y);
    }
    __syncthreads();
  }
}

// B operand from an FP64 column-major matrix G (identity if G == nullptr):
// B(n = j, k = i) = rs(i) G[i, j] cs(j).  The padding (j >= n or k >= n) is zeroed in a separate
// pass so that the FP64 -> FP32 conversions run once per element of G on full warps.
__device__ void fill_b2(const MLayout& L, const MixedSmem& m, const double2* G, Scale rs,
                        Scale cs) {
  const int n = L.n, Np = L.Np, Kp = L.Kp;
  for (int e = tid(); e < 2 * Np * Kp; e += nthr()) {
    const int k = e % Kp, row = e / Kp;
    const int j = row < Np ? row : row - Np;
    if (j >= n || k >= n) put_b(L, m, row, k, 0.f);
  }
  for (int e = tid(); e < n * n; e += nthr()) {
    const int k = e % n, j = e / n;  // element (k, j) of G
    float2 x;
    if (G) {
      const double2 g = G[k + j * n];
      x = make_float2((float)g.x, (float)g.y);
    } else {
      x = make_float2(k == j ? 1.f : 0.f, 0.f);
    }
    const float2 y = cmul32(cmul32(rs.at(k), x), cs.at(j));
    put_b(L, m, j, k, y.x);
    put_b(L, m, Np + j, k, y.y);
  }
}

// Force row F[x] = i (1 - G_xx) = (Im G_xx, 1 - Re G_xx) from an FP32 diagonal.
__device__ __forceinline__ void emit_force_row32(int n, const float2* dg, double2* Frow) {
  for (int x = tid(); x < n; x += nthr())
    Frow[x] = make_double2((double)dg[x].y, 1.0 - (double)dg[x].x);
}

// FP32 staging (column-major n x n) -> FP64 block result, one element per thread-iteration.
__device__ __forceinline__ void stage_to_fp64(int n, const float2* stage, double2* X) {
  for (int e = tid(); e < n * n; e += nthr())
    X[e] = make_double2((double)stage[e].x, (double)stage[e].y);
  __syncthreads();
}

// After a slice MMA: the next B operand (with the next slice's phase), or, for the last slice
// of a block, the FP64 block result Xc by way of the FP32 staging buffer `stage`.
__device__ __forceinline__ void slice_epilogue(const MLayout& L, const MixedSmem& m,
                                               uint32_t tbase, const float2* ph, bool to_b,
                                               double2* stage) {
  if (to_b) {
    epilogue<TO_B_K>(L, m, tbase, Scale{ph, false}, Scale{nullptr, false}, nullptr, nullptr);
  } else {
    epilogue<TO_F32>(L, m, tbase, Scale{nullptr, false}, Scale{nullptr, false}, stage, nullptr);
    stage_to_fp64(L.n, (const float2*)stage, m.Xc);
  }
}

__device__ __forceinline__ int grab_m(int* queue, int* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = atomicAdd(queue, 1);
  __syncthreads();
  return *slot;
}

// ------------------------------------------------------------------ log det and G
__global__ void __launch_bounds__(256) k_fwd_mixed(const Desc* __restrict__ descs, int ndesc,
                                                    int* queue, int* status, char* scratch,
                                                    MLayout L) {
  extern __shared__ __align__(128) char smem[];
  char* slot = scratch + (size_t)blockIdx.x * L.slot_bytes;
  MixedSmem m = mixed_smem(smem, slot, L);
  if (warp_id() == 0) tc::tmem_alloc(m.taddr, (uint32_t)L.tmem_cols);
  if (tid() == 0) tc::mbar_init(m.mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *m.taddr;
  uint32_t phase = 0;
  const int n = L.n;
  double2* T = (double2*)((L.t_smem ? smem : slot) + L.t0_off);
  double2* To = (double2*)((L.t_smem ? smem : slot) + L.t1_off);
  for (;;) {
    int c = grab_m(queue, m.qslot);
    if (c >= ndesc) break;
    const Desc d = descs[c];
    Small s = carve_small(smem + L.small_off, n);
    float2* pf = (float2*)s.ph;  // FP32 phases: two halves of n
    if (tid() == 0) {
      s.misc[0] = 0;
      s.misc[5] = (int)((blockIdx.x / max(1, L.num_sms)) * 2);
      s.misc[6] = gridDim.x > (unsigned)L.num_sms;  // several CTAs per SM: throughput mode
    }
    fill_a(L, m.a_hi, m.a_lo, d.E);
    cta_identity(n, T);
    for (int k = tid(); k < n; k += nthr()) s.logD[k] = 0.0;
    bool ok = true;
    for (int b = 0; b < d.nt && ok; b += d.nstab) {
      cta_phase32(n, pf, d.phi + (size_t)b * n, 1.f);
      __syncthreads();
      fill_b2(L, m, b == 0 ? nullptr : m.Xn, Scale{pf, false}, Scale{nullptr, false});
      for (int t = b; t < b + d.nstab; ++t) {
        const bool last = t + 1 == b + d.nstab;
        float2* phn = pf + ((t - b + 1) & 1) * n;
        if (!last) cta_phase32(n, phn, d.phi + (size_t)(t + 1) * n, 1.f);
        if (!slice_mma(L, m, tbase, phase)) {
          ok = false;
          break;
        }
        slice_epilogue(L, m, tbase, phn, !last, To);  // To is free until the QR
      }
      if (!ok) break;
      cta_reortho(n, m.Xc, m.Xn, T, To, s.logD, s);
      double2* t2 = T; T = To; To = t2;
    }
    if (!ok) {
      if (tid() == 0) status[d.user_index] = ST_TIMEOUT;
      break;
    }
    cta_assemble(n, m.Xn, T, s.logD, m.Xc, To, s, s.red + 2, s.red + 3);
    const double re = s.red[2], im = wrap_pi(s.red[3]);
    if (tid() == 0) {
      d.logdet[0] = re;
      d.logdet[1] = im;
      status[d.user_index] = (s.misc[0] || !isfinite(re) || !isfinite(im)) ? ST_NUMERIC : ST_OK;
    }
    if (d.G)
      for (int e = tid(); e < n * n; e += nthr()) d.G[e] = To[(e / n) + (e % n) * n];
    if (d.nf) cta_fermion_number(n, To, d.nf);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp_id() == 0) tc::tmem_dealloc(tbase, (uint32_t)L.tmem_cols);
}

// ------------------------------------------------------------------ force (mixed)
// Phase A: the forward and backward chains of the force as separate tasks (a ChainCode: whole
// chains, halves, log det/G segments; or a SegCode: the segmented chains of SegPlan, joined by
// FP64 merges); slices on the tensor core, QR in FP64; checkpoints and G_0 go to the
// configuration's global workspace (FWork).  The backward chain multiplies the right products as
// adjoints, X_R <- diag(e^{-i phi_s}) E X_R, the conjugate phase applied in the epilogue.  The
// chain state between blocks is (m.Xn = Q of the last QR, T, log D).  SEG: the variant with the
// segmented chains' tasks (its FP64 merges need more registers; the plain one keeps 2 CTAs/SM).
template <bool SEG>
__global__ void __launch_bounds__(256, SEG ? 1 : 2) k_chain_mixed(const Desc* __restrict__ descs,
                                                      const Task* __restrict__ tasks, int ntasks,
                                                      int* queue, int* status, char* scratch,
                                                      MLayout L) {
  extern __shared__ __align__(128) char smem[];
  char* slot = scratch + (size_t)blockIdx.x * L.slot_bytes;
  MixedSmem m = mixed_smem(smem, slot, L);
  if (warp_id() == 0) tc::tmem_alloc(m.taddr, (uint32_t)L.tmem_cols);
  if (tid() == 0) tc::mbar_init(m.mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *m.taddr;
  uint32_t phase = 0;
  const int n = L.n;
  double2* T = (double2*)((L.t_smem ? smem : slot) + L.t0_off);
  double2* To = (double2*)((L.t_smem ? smem : slot) + L.t1_off);
  const Scale one{nullptr, false};
  allow_dependents();
  for (;;) {
    const int q = grab_m(queue, m.qslot);
    if (q >= ntasks) break;
    const Task tk = tasks[q];
    const Desc d = descs[tk.desc];
    const int ns = d.nstab, nb = d.nt / d.nstab;
    const FWork W{d.fws, n, nb};
    Small s = carve_small(smem + L.small_off, n);
    float2* pf = (float2*)s.ph;  // FP32 phases: two halves of n
    if (tid() == 0) {
      s.misc[0] = 0;
      s.misc[5] = (int)((blockIdx.x / max(1, L.num_sms)) * 2);
      s.misc[6] = gridDim.x > (unsigned)L.num_sms;  // several CTAs per SM: throughput mode
    }
    fill_a(L, m.a_hi, m.a_lo, d.E);
    cta_identity(n, T);
    for (int k = tid(); k < n; k += nthr()) s.logD[k] = 0.0;
    bool ok = true;
    // one forward block b: its slices on the tensor core, then the QR (the state advances)
    auto fwd_block = [&](int b, bool from_id) -> bool {
      const int t0 = (b - 1) * ns;
      cta_phase32(n, pf, d.phi + (size_t)t0 * n, 1.f);
      __syncthreads();
      fill_b2(L, m, from_id ? nullptr : m.Xn, Scale{pf, false}, one);
      for (int t = t0; t < t0 + ns; ++t) {
        const bool last = t + 1 == t0 + ns;
        float2* phn = pf + ((t - t0 + 1) & 1) * n;
        if (!last) cta_phase32(n, phn, d.phi + (size_t)(t + 1) * n, 1.f);
        if (!slice_mma(L, m, tbase, phase)) return false;
        slice_epilogue(L, m, tbase, phn, !last, To);  // To is free until the QR
      }
      cta_reortho(n, m.Xc, m.Xn, T, To, s.logD, s);
      double2* t2 = T; T = To; To = t2;
      return true;
    };
    // one backward block b (right products as adjoints)
    auto bwd_block = [&](int b, bool from_id) -> bool {
      const int t0 = (b - 1) * ns;
      fill_b2(L, m, from_id ? nullptr : m.Xn, one, one);
      for (int t = b * ns - 1; t >= t0; --t) {
        const bool last = t == t0;
        cta_phase32(n, pf, d.phi + (size_t)t * n, -1.f);
        if (!slice_mma(L, m, tbase, phase)) return false;
        if (last) {
          epilogue<TO_F32>(L, m, tbase, Scale{pf, false}, one, To, nullptr);
          stage_to_fp64(n, (const float2*)To, m.Xc);
        } else {
          epilogue<TO_B_K>(L, m, tbase, Scale{pf, false}, one, nullptr, nullptr);
        }
      }
      cta_reortho(n, m.Xc, m.Xn, T, To, s.logD, s);
      double2* t2 = T; T = To; To = t2;
      return true;
    };
    auto store_state = [&](double2* x, double2* t, double* dl) {
      cta_copy(n * n, x, m.Xn);
      cta_copy(n * n, t, T);
      for (int k = tid(); k < n; k += nthr()) dl[k] = s.logD[k];
      __syncthreads();
    };
    auto load_state = [&](const double2* x, const double2* t, const double* dl) {
      cta_copy(n * n, m.Xn, x);
      cta_copy(n * n, T, t);
      for (int k = tid(); k < n; k += nthr()) s.logD[k] = dl[k];
      __syncthreads();
    };
    // the end of the forward chain: log det, G_0 and the outputs
    auto assemble_out = [&]() {
      double2* G0 = W.Gb(1);
      cta_assemble(n, m.Xn, T, s.logD, m.Xc, G0, s, s.red + 2, s.red + 3);
      const double re = s.red[2], im = wrap_pi(s.red[3]);
      if (tid() == 0) {
        d.logdet[0] = re;
        d.logdet[1] = im;
        atomicMax(status + d.user_index,
                  (s.misc[0] || !isfinite(re) || !isfinite(im)) ? ST_NUMERIC : ST_OK);
      }
      if (d.G)
        for (int e = tid(); e < n * n; e += nthr()) d.G[e] = G0[(e / n) + (e % n) * n];
      if (d.Gt)  // G(0, 0) = G
        for (int e = tid(); e < n * n; e += nthr()) d.Gt[e] = G0[(e / n) + (e % n) * n];
      if (d.nf) cta_fermion_number(n, G0, d.nf);
      if (d.O) {  // FP32 copy of the response operator for the wrap epilogues
        float* of = W.OF(d.Gt != nullptr);
        for (int e = tid(); e < n * n; e += nthr()) of[e] = (float)d.O[e];
      }
      __syncthreads();
      if (tid() == 0 && d.sync) flag_store(d.sync + SF_FWD, nb);  // G_0 written
    };
    auto numeric_status = [&]() {
      if (tid() == 0 && s.misc[0]) atomicMax(status + d.user_index, ST_NUMERIC);
    };
    int fail_flag[3] = {-1, -1, -1};  // flags a failed task releases (set to nb)
    if (SEG && tk.b >= CT_SFA) {
      // ---- segmented chains (SegPlan), joined by FP64 merges
      const int S = d.fseg, mb = nb / S;
      const bool pre = tk.b >= CT_SFP;
      const int code = pre ? tk.b : (tk.b & ~15), k = pre ? 0 : (tk.b & 15);
      const bool fw = pre ? tk.b == CT_SFP : (code == CT_SFA || code == CT_SFB);
      const int FSEG = fw ? SF_SEGF : SF_SEGB, FPRE = fw ? SF_PREF : SF_PREB;
      const int FLS = fw ? SF_LSF : SF_LSB;
      // checkpoint c of this direction, the prefix checkpoint of segment kk, local product kk
      auto ckx = [&](int c) { return fw ? W.LX(c) : W.RX(c); };
      auto ckt = [&](int c) { return fw ? W.LT(c) : W.RT(c); };
      auto ckd = [&](int c) { return fw ? W.LD(c) : W.RD(c); };
      auto pre_c = [&](int kk) { return fw ? kk * mb : nb - kk * mb + 1; };
      auto loc = [&](int kk) { return (fw ? 0 : S - 2) + kk - 1; };
      __syncthreads();
      if (pre) {
        fail_flag[0] = FPRE + S - 1;
        for (int kk = 2; kk < S; ++kk) {
          if (!cta_wait_pairs(d.sync, FLS + kk - 1, 1, kk == 2 ? FSEG : FPRE + kk - 1,
                              kk == 2 ? mb : 1, m.qslot + 1) && tid() == 0)
            atomicMax(status + d.user_index, ST_TIMEOUT);
          const int a = pre_c(kk - 1), c = pre_c(kk), li = loc(kk - 1);
          cta_merge(n, W.XX(li), W.XT(li), W.XD(li), ckx(a), ckt(a), ckd(a), m.Xc, m.Xn, ckx(c),
                    To, s.logD, s);
          cta_copy(n * n, ckt(c), To);
          for (int e = tid(); e < n; e += nthr()) ckd(c)[e] = s.logD[e];
          __syncthreads();
          if (tid() == 0) flag_store(d.sync + FPRE + kk, 1);
        }
        numeric_status();
      } else {
        const bool pass2 = code == CT_SFB || code == CT_SBB;
        const int first = fw ? k * mb + 1 : nb - k * mb;
        const int last = fw ? (k + 1) * mb : max(2, nb - (k + 1) * mb + 1);
        fail_flag[0] = FSEG + k;
        fail_flag[1] = pass2 ? (fw && k == S - 1 ? SF_FWD : -1) : FLS + k;
        if (pass2) {
          if (!cta_wait_pairs(d.sync, k == 1 ? FSEG : FPRE + k, k == 1 ? mb : 1, -1, 0,
                              m.qslot + 1) && tid() == 0)
            atomicMax(status + d.user_index, ST_TIMEOUT);
          const int c = pre_c(k);
          load_state(ckx(c), ckt(c), ckd(c));
        }
        const int step = fw ? 1 : -1;
        for (int b = first; ok; b += step) {
          ok = fw ? fwd_block(b, !pass2 && b == first) : bwd_block(b, !pass2 && b == first);
          if (!ok) break;
          const bool lastb = b == last;
          // final checkpoints: pass 1 of segment 0, and pass 2 but for a segment's last block
          // (formed by the next prefix) and the forward chain's end (the assembly)
          if ((!pass2 && k == 0) || (pass2 && !(lastb && k < S - 1) && !(fw && b == nb))) {
            store_state(ckx(b), ckt(b), ckd(b));
            if (tid() == 0) flag_store(d.sync + FSEG + k, fw ? b - first + 1 : first - b + 1);
          }
          if (lastb) break;
        }
        if (ok && !pass2 && k > 0) {  // pass 1: the segment's local product
          const int li = loc(k);
          store_state(W.XX(li), W.XT(li), W.XD(li));
          if (tid() == 0) flag_store(d.sync + FLS + k, 1);
        }
        if (ok && fw && pass2 && k == S - 1) assemble_out();
        else if (ok) numeric_status();
      }
    } else {
      // ---- whole chains, split halves, or log det/G segments
      const int sg = (tk.b >= CT_SEG && tk.b < CT_FWD2) ? tk.b - CT_SEG : -1;
      const ChainSpan sp = chain_span(tk.b, nb, d.fsplit);
      const bool fwd = sg >= 0 || sp.fwd;
      fail_flag[0] = sg >= 0 ? SF_FWD : sp.flag;
      if (fwd) {
        // a segment of a time-parallel log det/G split runs blocks sg*kb+1 .. (sg+1)*kb
        const int kb = sg >= 0 ? nb / d.nseg : sp.last - sp.first + 1;
        const int b_first = sg >= 0 ? sg * kb + 1 : sp.first;
        for (int b = b_first; b < b_first + kb && ok; ++b) {
          ok = fwd_block(b, b == b_first);
          if (!ok) break;
          if (sg < 0 && (b < nb || !sp.assemble)) {  // checkpoint (a split half's product: SX)
            if (b < nb) store_state(W.LX(b), W.LT(b), W.LD(b));
            else store_state(W.SX(), W.ST(), W.SD());
            if (tid() == 0 && d.sync) flag_store(d.sync + sp.flag, sp.count(b));
          }
        }
        if (ok && sg >= 0) {  // segment result in the checkpoint storage of block sg+1
          store_state(W.LX(sg + 1), W.LT(sg + 1), W.LD(sg + 1));
          numeric_status();
        } else if (ok && !sp.assemble) {
          numeric_status();
        } else if (ok) {
          assemble_out();
        }
      } else {
        for (int b = sp.first; b >= sp.last && ok; --b) {
          ok = bwd_block(b, b == sp.first);
          if (!ok) break;
          store_state(W.RX(b), W.RT(b), W.RD(b));
          if (tid() == 0 && d.sync) flag_store(d.sync + sp.flag, sp.count(b));
        }
        if (ok) numeric_status();
      }
    }
    if (!ok) {
      if (tid() == 0) {
        atomicMax(status + d.user_index, ST_TIMEOUT);
        // release the dependent tasks (their inputs are invalid; the status says so)
        if (d.sync)
          for (int i = 0; i < 3; ++i)
            if (fail_flag[i] >= 0) flag_store(d.sync + fail_flag[i], nb);
      }
      break;
    }
    __syncthreads();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp_id() == 0) tc::tmem_dealloc(tbase, (uint32_t)L.tmem_cols);
}

// Phase C on the tensor core: block b's force rows.  Row (b-1)ns from the boundary G_{(b-1)ns};
// the wraps inside the block as two MMAs each (both TMEM layouts alternate, so no transposes):
//   forward  G_s     = E [D_s G_{s-1} D_s^*] E^{-1}:  MMA(A = E, B = D G D^*) gives
//            W = E (D G D^*) with lane = row; written lane-as-N it is the B operand of
//            MMA(A = E^{-1}), whose result E^{-1} W^T = G_s^T leaves column m of G_s in lane m.
//   backward G_{q-1} = D_q^* [E^{-1} G_q E] D_q: MMA(A = E^{-1}, B = G_q), then MMA(A = E,
//            B = (E^{-1} G_q)^T) leaves column m of E^{-1} G_q E in lane m.
// The diagonal (the force row) is read straight out of the second accumulator; the phases of
// the next wrap are applied while writing the next B operand.
__global__ void __launch_bounds__(256) k_wrap_mixed(const Desc* __restrict__ descs,
                                                     const Task* __restrict__ tasks, int ntasks,
                                                     int* queue, int* status, char* scratch,
                                                     MLayout L) {
  extern __shared__ __align__(128) char smem[];
  char* slot = scratch + (size_t)blockIdx.x * L.slot_bytes;
  MixedSmem m = mixed_smem(smem, slot, L);
  float* e2_hi = (float*)(smem + L.a2_hi);
  float* e2_lo = L.three ? (float*)(smem + L.a2_lo) : nullptr;
  if (warp_id() == 0) tc::tmem_alloc(m.taddr, (uint32_t)L.tmem_cols);
  if (tid() == 0) tc::mbar_init(m.mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *m.taddr;
  uint32_t phase = 0;
  const int n = L.n;
  const Scale one{nullptr, false};
  int last_desc = -1;
  for (;;) {
    const int q = grab_m(queue, m.qslot);
    if (q >= ntasks) break;
    const Task tk = tasks[q];
    const Desc d = descs[tk.desc];
    const int ns = d.nstab, nb = d.nt / d.nstab, b = tk.b;
    const FWork W{d.fws, n, nb};
    // G_0 and every boundary Green's function of the configuration
    if (d.sync && !cta_wait_flags(d.sync, nb, 0, nb - 1, m.qslot + 1) && tid() == 0)
      atomicMax(status + d.user_index, ST_TIMEOUT);
    Small s = carve_small(smem + L.small_off, n);
    float2* pf = (float2*)s.ph;
    if (tk.desc != last_desc) {  // tasks of one configuration are contiguous: reload E only then
      fill_a(L, m.a_hi, m.a_lo, d.E);
      fill_a(L, e2_hi, e2_lo, d.Einv);
      last_desc = tk.desc;
    }
    bool ok = true;
    const int t0 = (b - 1) * ns, h = (ns - 1) / 2;
    const double2* Glo = W.Gb(b);
    // force rows and/or response traces tr(O G_r) of every G_r of the block
    auto frow = [&](int r) { return d.F ? d.F + (size_t)r * n : nullptr; };
    float2* dstage = d.F ? (float2*)s.rdiag : nullptr;  // FP32 diagonal of the wrapped G
    const float* Of = d.R ? W.OF(d.Gt != nullptr) : nullptr;
    float2* tslot = (float2*)(s.red + 48);
    if (d.F) emit_force_row(n, Glo, frow(t0));
    if (d.R) cta_trace(n, d.O, Glo, d.R + t0, s.red + 32);
    // forward wraps from G_{t0}: G_{t0+j}, j = 1..h; slice t0+j uses phi row t0+j-1
    for (int j = 1; j <= h && ok; ++j) {
      float2* ph = pf + ((j & 1) ? n : 0);
      cta_phase32(n, ph, d.phi + (size_t)(t0 + j - 1) * n, 1.f);
      if (j == 1) {
        __syncthreads();
        fill_b2(L, m, Glo, Scale{ph, false}, Scale{ph, true});
      }
      if (!mma_ab(L, m, m.a_hi, m.a_lo, tbase, phase)) { ok = false; break; }
      epilogue<TO_B_N>(L, m, tbase, one, one, nullptr, nullptr);
      float2* phn = pf + ((j & 1) ? 0 : n);
      const bool more = j < h;
      if (more) cta_phase32(n, phn, d.phi + (size_t)(t0 + j) * n, 1.f);
      if (!mma_ab(L, m, e2_hi, e2_lo, tbase, phase)) { ok = false; break; }
      // lane l holds column l of G_{t0+j} itself
      const Trace trf{Of, one, one, tslot, d.R ? d.R + t0 + j : nullptr};
      if (more)
        epilogue<TO_B_N>(L, m, tbase, Scale{phn, true}, Scale{phn, false}, nullptr, dstage, trf);
      else
        epilogue<NONE>(L, m, tbase, one, one, nullptr, dstage, trf);
      if (d.F) emit_force_row32(n, dstage, frow(t0 + j));
    }
    // backward wraps from G_{b*ns}: G_{q-1}, q = b*ns .. t0+h+2; slice q uses phi row q-1
    bool first = true;
    for (int qq = b * ns; qq >= t0 + h + 2 && ok; --qq) {
      float2* ph = pf + ((qq & 1) ? n : 0);
      cta_phase32(n, ph, d.phi + (size_t)(qq - 1) * n, 1.f);
      if (first) {
        __syncthreads();
        fill_b2(L, m, W.Gb(b + 1), one, one);
        first = false;
      }
      if (!mma_ab(L, m, e2_hi, e2_lo, tbase, phase)) { ok = false; break; }
      epilogue<TO_B_N>(L, m, tbase, one, one, nullptr, nullptr);
      if (!mma_ab(L, m, m.a_hi, m.a_lo, tbase, phase)) { ok = false; break; }
      // lane m holds column m of E^{-1} G_q E; G_{q-1} = D^* (.) D has the same diagonal.
      // Next B: B(n = m, k = i) = G_{q-1}[i, m] = conj(ph_i) X[i, m] ph_m
      const bool more = qq - 1 >= t0 + h + 2;
      const Trace trb{Of, Scale{ph, false}, Scale{ph, true}, tslot,
                      d.R ? d.R + (qq - 1) : nullptr};
      if (more)
        epilogue<TO_B_N>(L, m, tbase, Scale{ph, false}, Scale{ph, true}, nullptr, dstage, trb);
      else
        epilogue<NONE>(L, m, tbase, one, one, nullptr, dstage, trb);
      if (d.F) emit_force_row32(n, dstage, frow(qq - 1));
    }
    if (!ok) {
      if (tid() == 0) atomicMax(status + d.user_index, ST_TIMEOUT);
      break;
    }
    __syncthreads();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp_id() == 0) tc::tmem_dealloc(tbase, (uint32_t)L.tmem_cols);
}

void launch_chain_mixed(const Desc* descs, const Task* tasks, int ntasks, int* queue,
                        int* status, char* scratch, const MLayout& L, int grid,
                        cudaStream_t stream, bool seg) {
  if (seg)
    k_chain_mixed<true><<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, tasks, ntasks, queue,
                                                                    status, scratch, L);
  else
    k_chain_mixed<false><<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, tasks, ntasks, queue,
                                                                     status, scratch, L);
}
void launch_wrap_mixed(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                       char* scratch, const MLayout& L, int grid, cudaStream_t stream, bool pdl) {
  launch_maybe_pdl(k_wrap_mixed, grid, L.nthreads, L.smem_bytes, stream, pdl, descs, tasks, ntasks,
                   queue, status, scratch, L);
}

void launch_fwd_mixed(const Desc* descs, int ndesc, int* queue, int* status, char* scratch,
                      const MLayout& L, int grid, cudaStream_t stream) {
  k_fwd_mixed<<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, ndesc, queue, status, scratch,
                                                           L);
}
cudaError_t set_smem_mixed(int bytes) {
  for (const void* k :
       {(const void*)k_fwd_mixed, (const void*)k_chain_mixed<false>,
        (const void*)k_chain_mixed<true>, (const void*)k_wrap_mixed}) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
static const void* mixed_kernel(int which) {
  switch (which) {
    case 1: return (const void*)k_chain_mixed<false>;
    case 9: return (const void*)k_chain_mixed<true>;
    case 3: return (const void*)k_wrap_mixed;
    default: return (const void*)k_fwd_mixed;
  }
}
cudaError_t attrs_mixed(int which, cudaFuncAttributes* a) {
  return cudaFuncGetAttributes(a, mixed_kernel(which));
}
int occupancy_mixed(int which, int nthreads, int smem_bytes) {
  int nb = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mixed_kernel(which), nthreads, smem_bytes);
  return e == cudaSuccess ? nb : -1;
}

}  // namespace fd
