// fd_kernels_big.cu -- mixed-precision kernels for matrices larger than one shared-memory tensor
// tile (the size classes whose TF32 operands do not fit next to each other in shared memory,
// up to Nx = 288).  The slice products (Section 7 products, Section 9 blocking) and the wraps of
// the force sweep run on the tcgen05 tensor cores with FP32 accumulators in TMEM; their operands
// live in global memory (L2) in the chunked K-major layout of BLayout and stream through a
// shared-memory pipeline: one thread issues the bulk copies of a chunk's slabs (completing on a
// "full" mbarrier) and the MMAs that read them (committed to an "empty" mbarrier that frees the
// stage).  Every wait is bounded (FD_BIG_WAIT_CYCLES): a timeout marks the configuration
// FD_ERR_TIMEOUT, drains the copies in flight, frees TMEM and ends the kernel.  The QR
// re-orthogonalisation keeps FP64 inputs, outputs and scalars with its O(n^3) parts in
// double-float arithmetic on the FP32 pipes (fd_qr_df.cuh); the scale separation and the
// assembly are the FP64 CTA routines of the other kernels.
//
// Chains (one task = one configuration's forward or backward chain, or one segment):
//   Y <- E D_t Y as (E Y)^T = Y^T E: A = Y^T (row 2j + part = part of column j of Y, part 0 Re,
//   1 Im), B = E; TMEM lane = row of A, TMEM column i = row i of the product.  The epilogue
//   multiplies row i by the next slice's phase (the real and imaginary part of an element sit in
//   neighbouring lanes and meet by a shuffle) and writes the next A in place, or, after the last
//   slice of a block, the FP64 product for the QR.
// Wraps (one task = one block of one configuration):
//   W = M1 Z: A = M1 (E or E^{-1}), B rows 2j + part = column j of Z, K = rows of Z; lane = row a
//   of W.  The epilogue writes W by rows as the next B (rows 2a + part, K = columns of W).
//   G = W M2 as C[c, 2r + part] = sum_k M2[c, k] W_part[r, k]: lane = column c of G, TMEM
//   columns 2r + part = row r.  The epilogue reads the force row's diagonal and writes the next
//   wrap's Z = D G D^* (or D^* G D) by columns.  No product needs a transposed write.
#include <algorithm>

#include "fd_bound_df.cuh"
#include "fd_fp64.cuh"
#include "fd_kernels.h"
#include "fd_qr_df.cuh"
#include "fd_tc.cuh"

namespace fd {

#define FD_BIG_WAIT_CYCLES (2LL * 1000 * 1000 * 1000)

// Element (r, k) of a chunked operand with Rp rows (floats from the base).
__host__ __device__ __forceinline__ size_t ck_off(int r, int k, int Rp) {
  return ((size_t)(k >> 4) * (Rp >> 3) + (r >> 3)) * 128 + ((k & 15) >> 2) * 32 + (r & 7) * 4 +
         (k & 3);
}
// First float of the slab of chunk kc that starts at row r0 (a multiple of 8).
__host__ __device__ __forceinline__ size_t ck_slab(int kc, int r0, int Rp) {
  return ((size_t)kc * (Rp >> 3) + (r0 >> 3)) * 128;
}

struct BigSmem {
  char* stages;
  uint64_t* full;
  uint64_t* empty;
  uint64_t* done;
  uint32_t* taddr;
  int* qslot;
};

__device__ __forceinline__ BigSmem big_smem(char* smem, const BLayout& L) {
  BigSmem m;
  m.stages = smem;
  uint64_t* bar = (uint64_t*)(smem + L.bar_off);
  m.full = bar;
  m.empty = bar + L.nstages;
  m.done = bar + 2 * L.nstages;
  m.taddr = (uint32_t*)(bar + 2 * L.nstages + 1);
  m.qslot = (int*)(m.taddr + 1);
  return m;
}

// Pipeline state of the issuing thread: chunks handed to the pipeline so far (g) and the parity
// of the `done` barrier (every thread keeps its own copy of dphase).
struct BigPipe {
  uint32_t g;
  uint32_t dphase;
};

__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
  hi = tc::to_tf32(v);
  lo = tc::to_tf32(v - hi);
}
__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// One 128-row tile on the tensor core: TMEM columns [0, NB) <- sum over the K chunks of
// A rows [a0, a0 + 128) (chunked, RpA rows) times B rows [b0, b0 + NB) (chunked, RpB rows).
// lo planes at +a_lo / +b_lo floats (split TF32).  Returns false (on every thread) after a
// bounded wait ran out; the copies in flight have then been waited for.
__device__ bool big_tile(const BLayout& L, const BigSmem& m, BigPipe& P, const float* A,
                         size_t a_lo, int RpA, int a0, const float* B, size_t b_lo, int RpB,
                         int b0, int NB, uint32_t tbase) {
  const int nK = L.Kp >> 4;
  const uint32_t S = (uint32_t)L.nstages;
  int ok = 1;
  if (tid() == 0) {
    const uint32_t a_bytes = 128u * 64u, b_bytes = (uint32_t)NB * 64u;
    const uint32_t tx = (L.three ? 2u : 1u) * (a_bytes + b_bytes);
    const uint32_t g0 = P.g;
    uint32_t issued = 0;  // chunks of this tile whose copies were issued
    auto issue = [&](int kc) -> bool {
      const uint32_t gg = g0 + (uint32_t)kc, s = gg % S;
      if (gg >= S && !tc::mbar_wait(m.empty + s, ((gg / S) - 1u) & 1u, FD_BIG_WAIT_CYCLES))
        return false;
      char* st = m.stages + (size_t)s * L.stage_bytes;
      tc::mbar_arrive_expect_tx(m.full + s, tx);
      tc::bulk_g2s(st, A + ck_slab(kc, a0, RpA), a_bytes, m.full + s);
      tc::bulk_g2s(st + L.b_hi, B + ck_slab(kc, b0, RpB), b_bytes, m.full + s);
      if (L.three) {
        tc::bulk_g2s(st + L.a_lo, A + a_lo + ck_slab(kc, a0, RpA), a_bytes, m.full + s);
        tc::bulk_g2s(st + L.b_lo, B + b_lo + ck_slab(kc, b0, RpB), b_bytes, m.full + s);
      }
      ++issued;
      return true;
    };
    // N pieces of at most 256 columns, multiples of 16
    const int npc = (NB + 255) / 256;
    const int pw = ((NB + npc - 1) / npc + 15) & ~15;
    const int pre = min((int)S, nK);
    for (int kc = 0; kc < pre && ok; ++kc) ok = issue(kc);
    int consumed = 0;
    for (int kc = 0; kc < nK && ok; ++kc) {
      const uint32_t gg = g0 + (uint32_t)kc, s = gg % S;
      if (!tc::mbar_wait(m.full + s, (gg / S) & 1u, FD_BIG_WAIT_CYCLES)) {
        ok = 0;
        break;
      }
      ++consumed;
      tc::fence_after();
      char* st = m.stages + (size_t)s * L.stage_bytes;
      const uint32_t ah = tc::smem_u32(st), bh = tc::smem_u32(st + L.b_hi);
      const uint32_t al = L.three ? tc::smem_u32(st + L.a_lo) : 0u;
      const uint32_t bl = L.three ? tc::smem_u32(st + L.b_lo) : 0u;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        for (int nb0 = 0; nb0 < NB; nb0 += pw) {
          const int nw = min(pw, NB - nb0);
          const uint32_t idesc = tc::idesc_tf32(128, nw);
          const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
          const uint32_t ko = 256u * ks, no = (uint32_t)(nb0 >> 3) * 512u;
          const uint64_t ad = tc::make_desc(ah + ko, 128, 512);
          const uint64_t bd = tc::make_desc(bh + no + ko, 128, 512);
          tc::mma_tf32(tbase + (uint32_t)nb0, ad, bd, idesc, acc);
          if (L.three) {
            tc::mma_tf32(tbase + (uint32_t)nb0, ad, tc::make_desc(bl + no + ko, 128, 512), idesc,
                         1u);
            tc::mma_tf32(tbase + (uint32_t)nb0, tc::make_desc(al + ko, 128, 512), bd, idesc, 1u);
          }
        }
      }
      tc::mma_commit(m.empty + s);
      // refill the stage the previous chunk used (its MMAs are queued ahead of this chunk's)
      if (kc >= 1 && kc - 1 + (int)S < nK) ok = issue(kc - 1 + (int)S);
    }
    if (ok) {
      tc::mma_commit(m.done);
    } else {
      // wait (bounded) for the copies still in flight before the CTA gives up
      for (uint32_t c = (uint32_t)consumed; c < issued; ++c) {
        const uint32_t gg = g0 + c;
        tc::mbar_wait(m.full + gg % S, (gg / S) & 1u, FD_BIG_WAIT_CYCLES);
      }
    }
    P.g = g0 + (uint32_t)nK;
  }
  if (__syncthreads_or(!ok)) return false;
  const bool fin = tc::mbar_wait(m.done, P.dphase, FD_BIG_WAIT_CYCLES);
  P.dphase ^= 1u;
  const int bad = __syncthreads_or(!fin);
  tc::fence_after();
  return bad == 0;
}

// ------------------------------------------------------------------ operand fills (generic proxy)
// Chunked copy of a real n x n matrix M (row-major; symmetric) with Rp rows: element (r, k) =
// M[r][k], zero outside n x n.  Consecutive threads write consecutive 16-byte groups.
__device__ void fill_real(int n, int Rp, int Kp, const double* M, float* hi, float* lo,
                          bool three) {
  const int groups = Rp * Kp / 4;
  for (int e = tid(); e < groups; e += nthr()) {
    const int r8 = e & 7, cm = (e >> 3) & 3, rg = (e >> 5) % (Rp >> 3), kc = (e >> 5) / (Rp >> 3);
    const int r = rg * 8 + r8, k0 = kc * 16 + cm * 4;
    float4 h, l;
    float* hp = &h.x;
    float* lp = &l.x;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + u;
      const float v = (r < n && k < n) ? (float)M[(size_t)r * n + k] : 0.f;
      split_tf32(v, hp[u], lp[u]);
    }
    reinterpret_cast<float4*>(hi)[e] = h;
    if (three) reinterpret_cast<float4*>(lo)[e] = l;
  }
}

// Chunked operand with rows 2j + part = part of column j of Z, K = row i of Z, where
// Z[i][j] = rs(i) X[i + j n] cs(j) (X column-major FP64; X == null: the identity), zero outside
// the matrix.  Used for the chains' A (= Y^T) and the wraps' first B.
struct PhaseVec {
  const float2* p;
  bool cj;
  __device__ __forceinline__ float2 at(int x) const {
    if (!p) return make_float2(1.f, 0.f);
    const float2 v = p[x];
    return cj ? make_float2(v.x, -v.y) : v;
  }
};
__device__ void fill_cols(int n, int Rp, int Kp, const double2* X, PhaseVec rs, PhaseVec cs,
                          float* hi, float* lo, bool three) {
  const int groups = Rp * Kp / 4;
  for (int e = tid(); e < groups; e += nthr()) {
    const int r8 = e & 7, cm = (e >> 3) & 3, rg = (e >> 5) % (Rp >> 3), kc = (e >> 5) / (Rp >> 3);
    const int row = rg * 8 + r8, k0 = kc * 16 + cm * 4;
    const int j = row >> 1, part = row & 1;
    float4 h, l;
    float* hp = &h.x;
    float* lp = &l.x;
    const float2 cj = j < n ? cs.at(j) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = k0 + u;
      float v = 0.f;
      if (j < n && i < n) {
        float2 x;
        if (X) {
          const double2 g = X[(size_t)i + (size_t)j * n];
          x = make_float2((float)g.x, (float)g.y);
        } else {
          x = make_float2(i == j ? 1.f : 0.f, 0.f);
        }
        const float2 y = cmul2(cmul2(rs.at(i), x), cj);
        v = part ? y.y : y.x;
      }
      split_tf32(v, hp[u], lp[u]);
    }
    reinterpret_cast<float4*>(hi)[e] = h;
    if (three) reinterpret_cast<float4*>(lo)[e] = l;
  }
}

// Store four consecutive K values of one row (k0 a multiple of 4) of a chunked operand.
__device__ __forceinline__ void put4(float* hi, float* lo, bool three, int row, int k0, int Rp,
                                     const float (&v)[4]) {
  float4 h, l;
  split_tf32(v[0], h.x, l.x);
  split_tf32(v[1], h.y, l.y);
  split_tf32(v[2], h.z, l.z);
  split_tf32(v[3], h.w, l.w);
  const size_t o = ck_off(row, k0, Rp);
  *reinterpret_cast<float4*>(hi + o) = h;
  if (three) *reinterpret_cast<float4*>(lo + o) = l;
}

// FP32 phases e^{i s phi} of one slice.
__device__ __forceinline__ void phase32(int n, float2* ph, const double* phi_row, float sgn) {
  for (int x = tid(); x < n; x += nthr()) {
    float sn, cs;
    sincosf((float)phi_row[x], &sn, &cs);
    ph[x] = make_float2(cs, sgn * sn);
  }
}

// ------------------------------------------------------------------ chain epilogue
// After the products of M-tile mt of a chain slice: TMEM lane q holds row m = 128 mt + q of
// (E Y)^T, i.e. part (m & 1) of column j = m / 2 of E Y, with TMEM column i = row i.
//   to_fp64 == false: next A (in place) = rows of D' E Y with D' = diag(rs) (rs null: none)
//   to_fp64 == true : X[i + j n] = (D' E Y)[i][j] in FP64 (column-major), the block's product
__device__ void epi_chain(const BLayout& L, uint32_t tbase, int mt, PhaseVec rs, bool to_fp64,
                          float* Ahi, float* Alo, double2* X) {
  const int n = L.n;
  const int w = warp_id(), quad = w & 3, half = w >> 2, nhalf = nwarps() > 4 ? 2 : 1;
  const int m = 128 * mt + quad * 32 + lane_id();
  const int j = m >> 1, part = m & 1;
  const uint32_t lane_base = tbase + ((uint32_t)(quad * 32) << 16);
  const int nchunk = L.Ne >> 4;
  for (int c = half; c < nchunk; c += nhalf) {
    float v[16];
    tc::tmem_ld16(lane_base + (uint32_t)(c * 16), v);
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      float o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float mine = v[4 * q4 + u];
        const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
        const float re = part ? other : mine, im = part ? mine : other;
        const int i = c * 16 + 4 * q4 + u;
        const float2 y = i < n ? cmul2(rs.at(i), make_float2(re, im)) : make_float2(0.f, 0.f);
        o[u] = part ? y.y : y.x;
        // FP64 output: lane part 0 writes even i, part 1 odd i
        if (to_fp64 && j < n && i < n && (i & 1) == part)
          X[(size_t)i + (size_t)j * n] = make_double2((double)y.x, (double)y.y);
      }
      if (!to_fp64 && m < L.Mc) put4(Ahi, Alo, L.three != 0, m, c * 16 + 4 * q4, L.Mc, o);
    }
  }
  tc::fence_before();
  __syncthreads();
}

// ------------------------------------------------------------------ wrap epilogues
// L1 (W = M1 Z) of pass p, M-tile mt: TMEM lane q = row a = 128 mt + q of W, TMEM column
// 2 cl + part = column c = p Nw / 2 + cl.  Writes B2 rows 2a + part (K = c).
__device__ void epi_w1(const BLayout& L, uint32_t tbase, int mt, int p, float* Bhi, float* Blo) {
  const int n = L.n;
  const int w = warp_id(), quad = w & 3, half = w >> 2, nhalf = nwarps() > 4 ? 2 : 1;
  const int a = 128 * mt + quad * 32 + lane_id();
  const uint32_t lane_base = tbase + ((uint32_t)(quad * 32) << 16);
  const int nchunk = L.Nw >> 4;
  const int c_base = p * (L.Nw >> 1);
  for (int c = half; c < nchunk; c += nhalf) {
    float v[16];
    tc::tmem_ld16(lane_base + (uint32_t)(c * 16), v);
    if (a < n) {
#pragma unroll
      for (int q4 = 0; q4 < 2; ++q4) {
        float re[4], im[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          re[u] = v[8 * q4 + 2 * u];
          im[u] = v[8 * q4 + 2 * u + 1];
        }
        const int k0 = c_base + c * 8 + 4 * q4;
        if (k0 < L.Kp) {
          put4(Bhi, Blo, L.three != 0, 2 * a, k0, L.Nb, re);
          put4(Bhi, Blo, L.three != 0, 2 * a + 1, k0, L.Nb, im);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
}

// R2 (G = W M2) of pass p, M-tile mt: TMEM lane q = column c = 128 mt + q of G, TMEM column
// 2 rl + part = row r = p Nw / 2 + rl.  dg (optional): dg[c] = G[c][c] (FP32, shared memory).
// With `next`: B1 rows 2c + part (K = r) of the next wrap's Z[r][c] = rs(r) G[r][c] cs(c).
__device__ void epi_w2(const BLayout& L, uint32_t tbase, int mt, int p, float2* dg, bool next,
                       PhaseVec rs, PhaseVec cs, float* Bhi, float* Blo) {
  const int n = L.n;
  const int w = warp_id(), quad = w & 3, half = w >> 2, nhalf = nwarps() > 4 ? 2 : 1;
  const int c = 128 * mt + quad * 32 + lane_id();
  const uint32_t lane_base = tbase + ((uint32_t)(quad * 32) << 16);
  const int nchunk = L.Nw >> 4;
  const int r_base = p * (L.Nw >> 1);
  const float2 cc = c < n ? cs.at(c) : make_float2(0.f, 0.f);
  for (int ch = half; ch < nchunk; ch += nhalf) {
    float v[16];
    tc::tmem_ld16(lane_base + (uint32_t)(ch * 16), v);
    if (c < n) {
#pragma unroll
      for (int q4 = 0; q4 < 2; ++q4) {
        float re[4], im[4];
        const int r0 = r_base + ch * 8 + 4 * q4;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = r0 + u;
          const float2 g = make_float2(v[8 * q4 + 2 * u], v[8 * q4 + 2 * u + 1]);
          if (dg && r == c) dg[c] = g;
          const float2 y = r < n ? cmul2(cmul2(rs.at(r), g), cc) : make_float2(0.f, 0.f);
          re[u] = y.x;
          im[u] = y.y;
        }
        if (next && r0 < L.Kp) {
          put4(Bhi, Blo, L.three != 0, 2 * c, r0, L.Nb, re);
          put4(Bhi, Blo, L.three != 0, 2 * c + 1, r0, L.Nb, im);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
}

// Make this CTA's generic-proxy global writes visible to its later bulk copies.
__device__ __forceinline__ void publish_for_copies() {
  tc::fence_proxy_async_global();
  __syncthreads();
}

__device__ __forceinline__ int grab_b(int* queue, int* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = atomicAdd(queue, 1);
  __syncthreads();
  return *slot;
}

// One chain slice: the Mc/128 M-tiles of (E Y)^T and their epilogues.
__device__ bool chain_slice(const BLayout& L, const BigSmem& m, BigPipe& P, const Desc& d,
                            float* Ahi, float* Alo, uint32_t tbase, PhaseVec rs, bool to_fp64,
                            double2* X) {
  const size_t a_lo = (size_t)L.Mc * L.Kp, e_lo = (size_t)L.Ma * L.Kp;
  for (int mt = 0; mt < (L.Mc >> 7); ++mt) {
    if (!big_tile(L, m, P, Ahi, a_lo, L.Mc, 128 * mt, d.Ec, e_lo, L.Ma, 0, L.Ne, tbase))
      return false;
    epi_chain(L, tbase, mt, rs, to_fp64, Ahi, Alo, X);
  }
  publish_for_copies();
  return true;
}

// ------------------------------------------------------------------ chains
// Task.b: a ChainCode (forward chain, backward chain, a log det/G segment) or a SegCode (the
// segmented chains of SegPlan).  Forward: slices with QR every n_stab, left checkpoints (when the
// configuration has a force workspace), assembly -> log det, G (and G(0,0), the fermion number,
// O in FP32 as asked).  Backward: the right products as adjoints X_R <- D_s^* E X_R, QR, right
// checkpoints.  The chain state between blocks is (Xn = Q of the last QR, T, log D).
__global__ void __launch_bounds__(256, 1) k_chain_big(const Desc* __restrict__ descs,
                                                      const Task* __restrict__ tasks, int ntasks,
                                                      int* queue, int* status, char* scratch,
                                                      BLayout L) {
  extern __shared__ __align__(1024) char smem[];
  char* slot = scratch + (size_t)blockIdx.x * L.slot_bytes;
  BigSmem m = big_smem(smem, L);
  if (warp_id() == 0) tc::tmem_alloc(m.taddr, (uint32_t)L.tmem_cols);
  if (tid() == 0) {
    for (int s = 0; s < 2 * L.nstages + 1; ++s) tc::mbar_init(m.full + s, 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *m.taddr;
  BigPipe P{0u, 0u};
  const int n = L.n;
  float* Ahi = (float*)(slot + L.a_off);
  float* Alo = Ahi + (size_t)L.Mc * L.Kp;
  double2* Xc = (double2*)(slot + L.xc_off);
  double2* Xn = (double2*)(slot + L.xn_off);
  double2* T = (double2*)(slot + L.t0_off);
  double2* To = (double2*)(slot + L.t1_off);
  float2* pf = (float2*)(smem + L.ph_off);  // FP32 phases, two halves of n
  float4* qsm = (float4*)m.stages;          // the df QR's shared memory (the idle stages)
  const int qcap = L.nstages * L.stage_bytes / 16;
  const PhaseVec none{nullptr, false};
  allow_dependents();
  bool ok = true;
  for (;;) {
    const int q = grab_b(queue, m.qslot);
    if (q >= ntasks) break;
    const Task tk = tasks[q];
    const Desc d = descs[tk.desc];
    const int ns = d.nstab, nb = d.nt / d.nstab;
    const FWork W{d.fws, n, nb};
    const bool keep = d.fws != nullptr;
    Small s = carve_small(smem + L.small_off, n);
    if (tid() == 0) {
      s.misc[0] = 0;
      s.misc[5] = (int)((blockIdx.x / max(1, L.num_sms)) * 2);
      s.misc[6] = 0;  // one CTA per SM: latency mode
    }
    cta_identity(n, T);
    for (int k = tid(); k < n; k += nthr()) s.logD[k] = 0.0;
    __syncthreads();
    // one forward block b: its slices on the tensor cores, then the QR (the state advances)
    auto fwd_block = [&](int b, bool from_id) -> bool {
      const int t0 = (b - 1) * ns;
      phase32(n, pf, d.phi + (size_t)t0 * n, 1.f);
      __syncthreads();
      fill_cols(n, L.Mc, L.Kp, from_id ? nullptr : Xn, PhaseVec{pf, false}, none, Ahi, Alo,
                L.three != 0);
      publish_for_copies();
      for (int t = t0; t < t0 + ns; ++t) {
        const bool last = t + 1 == t0 + ns;
        float2* phn = pf + ((t - t0 + 1) & 1) * n;
        if (!last) phase32(n, phn, d.phi + (size_t)(t + 1) * n, 1.f);
        __syncthreads();
        if (!chain_slice(L, m, P, d, Ahi, Alo, tbase, last ? none : PhaseVec{phn, false}, last,
                         Xc))
          return false;
      }
      cta_reortho_df(n, Xc, Xn, T, To, s.logD, s, qsm, qcap);
      double2* t2 = T; T = To; To = t2;
      return true;
    };
    // one backward block b (right products as adjoints)
    auto bwd_block = [&](int b, bool from_id) -> bool {
      const int t0 = (b - 1) * ns;
      fill_cols(n, L.Mc, L.Kp, from_id ? nullptr : Xn, none, none, Ahi, Alo, L.three != 0);
      publish_for_copies();
      for (int t = b * ns - 1; t >= t0; --t) {
        phase32(n, pf, d.phi + (size_t)t * n, -1.f);
        __syncthreads();
        // the block's last product goes out in FP64 (with its phase) for the QR
        if (!chain_slice(L, m, P, d, Ahi, Alo, tbase, PhaseVec{pf, false}, t == t0, Xc))
          return false;
      }
      cta_reortho_df(n, Xc, Xn, T, To, s.logD, s, qsm, qcap);
      double2* t2 = T; T = To; To = t2;
      return true;
    };
    auto store_state = [&](double2* x, double2* t, double* dl) {
      cta_copy(n * n, x, Xn);
      cta_copy(n * n, t, T);
      for (int k = tid(); k < n; k += nthr()) dl[k] = s.logD[k];
      __syncthreads();
    };
    auto load_state = [&](const double2* x, const double2* t, const double* dl) {
      cta_copy(n * n, Xn, x);
      cta_copy(n * n, T, t);
      for (int k = tid(); k < n; k += nthr()) s.logD[k] = dl[k];
      __syncthreads();
    };
    // the end of the forward chain: log det, G_0 and the outputs
    auto assemble_out = [&]() {
      double2* G0 = keep ? W.Gb(1) : To;  // To is free after the last swap
      cta_assemble(n, Xn, T, s.logD, Xc, G0, s, s.red + 2, s.red + 3);
      const double re = s.red[2], im = wrap_pi(s.red[3]);
      if (tid() == 0) {
        d.logdet[0] = re;
        d.logdet[1] = im;
        atomicMax(status + d.user_index,
                  (s.misc[0] || !isfinite(re) || !isfinite(im)) ? ST_NUMERIC : ST_OK);
      }
      if (d.G)
        for (int e = tid(); e < n * n; e += nthr()) d.G[e] = G0[(e / n) + (e % n) * n];
      if (d.Gt)
        for (int e = tid(); e < n * n; e += nthr()) d.Gt[e] = G0[(e / n) + (e % n) * n];
      if (d.nf) cta_fermion_number(n, G0, d.nf);
      if (keep && d.O) {
        float* of = W.OF(d.Gt != nullptr);
        for (int e = tid(); e < n * n; e += nthr()) of[e] = (float)d.O[e];
      }
      __syncthreads();
      if (tid() == 0 && d.sync) flag_store(d.sync + SF_FWD, nb);
    };
    auto numeric_status = [&]() {
      if (tid() == 0 && s.misc[0]) atomicMax(status + d.user_index, ST_NUMERIC);
    };
    int fail_flag[3] = {-1, -1, -1};  // flags a failed task releases (set to nb)
    if (tk.b >= CT_SFA) {
      // ---- segmented chains (SegPlan)
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
      if (pre) {
        fail_flag[0] = FPRE + S - 1;
        for (int kk = 2; kk < S; ++kk) {
          if (!cta_wait_pairs(d.sync, FLS + kk - 1, 1, kk == 2 ? FSEG : FPRE + kk - 1,
                              kk == 2 ? mb : 1, m.qslot + 1) && tid() == 0)
            atomicMax(status + d.user_index, ST_TIMEOUT);
          const int a = pre_c(kk - 1), c = pre_c(kk), li = loc(kk - 1);
          cta_merge_df(n, W.XX(li), W.XT(li), W.XD(li), ckx(a), ckt(a), ckd(a), Xc, Xn, T, To,
                       ckx(c), s.logD, s, qsm, qcap);
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
        const int kb = sg >= 0 ? nb / d.nseg : sp.last - sp.first + 1;
        const int b_first = sg >= 0 ? sg * kb + 1 : sp.first;
        for (int b = b_first; b < b_first + kb && ok; ++b) {
          ok = fwd_block(b, b == b_first);
          if (!ok) break;
          if (keep && sg < 0 && (b < nb || !sp.assemble)) {  // a split half's product: SX
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

// ------------------------------------------------------------------ wraps
// Phase C of the force on the tensor cores: block b's force rows.  Row (b-1)ns from the FP64
// boundary G_{(b-1)ns}; forward wraps G_s = E [D_s G_{s-1} D_s^*] E^{-1} from the lower boundary
// for (n_stab-1)/2 slices, backward wraps G_{q-1} = D_q^* [E^{-1} G_q E] D_q from the upper one.
// Each wrap is W = M1 Z (L1) then G = W M2 (R2); the diagonal of G is the force row.
__device__ bool wrap_products(const BLayout& L, const BigSmem& m, BigPipe& P, const float* M1,
                              const float* M2, float* B1h, float* B1l, float* B2h, float* B2l,
                              uint32_t tbase, float2* dg, bool next, PhaseVec rs, PhaseVec cs) {
  const size_t e_lo = (size_t)L.Ma * L.Kp, b_lo = (size_t)L.Nb * L.Kp;
  for (int p = 0; p < L.npass; ++p)
    for (int mt = 0; mt < (L.Ma >> 7); ++mt) {
      if (!big_tile(L, m, P, M1, e_lo, L.Ma, 128 * mt, B1h, b_lo, L.Nb, p * L.Nw, L.Nw, tbase))
        return false;
      epi_w1(L, tbase, mt, p, B2h, B2l);
    }
  publish_for_copies();
  for (int p = 0; p < L.npass; ++p)
    for (int mt = 0; mt < (L.Ma >> 7); ++mt) {
      if (!big_tile(L, m, P, M2, e_lo, L.Ma, 128 * mt, B2h, b_lo, L.Nb, p * L.Nw, L.Nw, tbase))
        return false;
      epi_w2(L, tbase, mt, p, dg, next, rs, cs, B1h, B1l);
    }
  publish_for_copies();
  return true;
}

__device__ __forceinline__ void force_row_from(int n, const float2* dg, double2* Frow) {
  for (int x = tid(); x < n; x += nthr())
    Frow[x] = make_double2((double)dg[x].y, 1.0 - (double)dg[x].x);
}

__global__ void __launch_bounds__(256, 1) k_wrap_big(const Desc* __restrict__ descs,
                                                     const Task* __restrict__ tasks, int ntasks,
                                                     int* queue, int* status, char* scratch,
                                                     BLayout L) {
  extern __shared__ __align__(1024) char smem[];
  char* slot = scratch + (size_t)blockIdx.x * L.slot_bytes;
  BigSmem m = big_smem(smem, L);
  if (warp_id() == 0) tc::tmem_alloc(m.taddr, (uint32_t)L.tmem_cols);
  if (tid() == 0) {
    for (int s = 0; s < 2 * L.nstages + 1; ++s) tc::mbar_init(m.full + s, 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *m.taddr;
  BigPipe P{0u, 0u};
  const int n = L.n;
  const size_t bsz = (size_t)L.Nb * L.Kp;
  float* B1h = (float*)(slot + L.b1_off);
  float* B1l = B1h + bsz;
  float* B2h = (float*)(slot + L.b2_off);
  float* B2l = B2h + bsz;
  // the padding rows and columns of both B operands stay zero
  for (size_t e = tid(); e < 2 * bsz / 4; e += nthr()) {  // hi and lo planes of B1 and B2
    reinterpret_cast<float4*>(B1h)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    reinterpret_cast<float4*>(B2h)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  publish_for_copies();
  float2* pf = (float2*)(smem + L.ph_off);
  float2* dg = (float2*)(smem + L.dg_off);
  const PhaseVec none{nullptr, false};
  bool ok = true;
  for (;;) {
    const int q = grab_b(queue, m.qslot);
    if (q >= ntasks) break;
    const Task tk = tasks[q];
    const Desc d = descs[tk.desc];
    const int ns = d.nstab, nb = d.nt / d.nstab, b = tk.b;
    const FWork W{d.fws, n, nb};
    // G_0 and every boundary Green's function of the configuration
    if (d.sync && !cta_wait_flags(d.sync, nb, 0, nb - 1, m.qslot + 1) && tid() == 0)
      atomicMax(status + d.user_index, ST_TIMEOUT);
    const int t0 = (b - 1) * ns, h = (ns - 1) / 2;
    const double2* Glo = W.Gb(b);
    auto frow = [&](int r) { return d.F + (size_t)r * n; };
    if (d.F) emit_force_row(n, Glo, frow(t0));
    for (int j = 1; j <= h && ok; ++j) {
      float2* ph = pf + ((j & 1) ? n : 0);
      float2* phn = pf + ((j & 1) ? 0 : n);
      phase32(n, ph, d.phi + (size_t)(t0 + j - 1) * n, 1.f);
      __syncthreads();
      if (j == 1) {
        fill_cols(n, L.Nb, L.Kp, Glo, PhaseVec{ph, false}, PhaseVec{ph, true}, B1h, B1l,
                  L.three != 0);
        publish_for_copies();
      }
      const bool more = j < h;
      if (more) phase32(n, phn, d.phi + (size_t)(t0 + j) * n, 1.f);
      __syncthreads();
      ok = wrap_products(L, m, P, d.Ec, d.Eic, B1h, B1l, B2h, B2l, tbase, dg, more,
                         PhaseVec{phn, false}, PhaseVec{phn, true});
      if (ok && d.F) force_row_from(n, dg, frow(t0 + j));
    }
    bool first = true;
    for (int qq = b * ns; qq >= t0 + h + 2 && ok; --qq) {
      float2* ph = pf + ((qq & 1) ? n : 0);
      phase32(n, ph, d.phi + (size_t)(qq - 1) * n, 1.f);
      __syncthreads();
      if (first) {
        fill_cols(n, L.Nb, L.Kp, W.Gb(b + 1), none, none, B1h, B1l, L.three != 0);
        publish_for_copies();
        first = false;
      }
      const bool more = qq - 1 >= t0 + h + 2;
      ok = wrap_products(L, m, P, d.Eic, d.Ec, B1h, B1l, B2h, B2l, tbase, dg, more,
                         PhaseVec{ph, true}, PhaseVec{ph, false});
      if (ok && d.F) force_row_from(n, dg, frow(qq - 1));
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

// ------------------------------------------------------------------ boundary Green's functions
// Phase B of the mixed force for the streamed size classes: G_{(b-1) ns} of block b from the left
// checkpoint b-1 and the right checkpoint b, in double-float (fd_bound_df.cuh); three n x n df
// work matrices in the CTA's slot.  Every checkpoint it reads is final (whole or segmented
// chains; the split chains of ChainSpan, which leave merges to this phase, are not planned for
// these classes: merging a second half's checkpoint forms a row scaling that spans beta/2 times
// the hopping bandwidth, beyond the FP32 exponent range of double-float numbers at low
// temperature).
__global__ void __launch_bounds__(256, 2) k_boundary_big(const Desc* __restrict__ descs,
                                                         const Task* __restrict__ tasks,
                                                         int ntasks, int* queue, int* status,
                                                         char* scratch, BLayout L) {
  extern __shared__ __align__(1024) char smem[];
  char* slot = scratch + (size_t)blockIdx.x * L.slot_bytes;
  int* qs = (int*)(smem + L.bar_off);
  const int n = L.n;
  float4* H = (float4*)(slot + L.b1_off);
  float4* Mb = H + (size_t)n * n;
  float4* Wb = Mb + (size_t)n * n;
  allow_dependents();
  for (;;) {
    const int q = grab_b(queue, qs);
    if (q >= ntasks) break;
    const Task tk = tasks[q];
    const Desc d = descs[tk.desc];
    const int nb = d.nt / d.nstab, b = tk.b;
    const FWork W{d.fws, n, nb};
    bool waited = true;
    if (d.sync && d.fseg) {  // segmented chains: the flags of the two checkpoints' segments
      const int mb = nb / d.fseg;
      int i0, t0, i1, t1;
      seg_left_ready(b - 1, mb, i0, t0);
      seg_right_ready(b, nb, mb, i1, t1);
      waited = cta_wait_pairs(d.sync, i0, t0, i1, t1, qs + 1);
    } else if (d.sync) {
      waited = cta_wait_flags(d.sync, b - 1, nb - b + 1, 0, qs + 1);
    }
    if (!waited && tid() == 0) atomicMax(status + d.user_index, ST_TIMEOUT);
    Small s = carve_small(smem + L.small_off, n);
    if (tid() == 0) s.misc[0] = 0;
    __syncthreads();
    boundary_green_df(n, W.LX(b - 1), W.LT(b - 1), W.LD(b - 1), W.RX(b), W.RT(b), W.RD(b), H, Mb,
                      Wb, W.Gb(b), s, (float4*)(smem + L.ph_off));
    if (tid() == 0 && s.misc[0]) atomicMax(status + d.user_index, ST_NUMERIC);
    __syncthreads();
    if (tid() == 0 && d.sync) flag_add(d.sync + SF_BND, 1);
  }
}

// Shared memory (df numbers): the df QR (its panel, T and Gram matrices and GEMM tiles) and the
// boundary Green's function (64 x 64 GEMM tiles).
int big_qr_vcap(int n) { return DF_PANEL * (n + 2 * DF_PANEL) + DF_TILE_ELEMS(16, 256); }
int big_bound_tiles() { return DF_TILE_ELEMS(64, 64); }

// ------------------------------------------------------------------ operand preparation
// Chunked TF32 copies (hi, then lo) of the distinct E and E^{-1} matrices of a call, rows padded
// to Ma (one item per blockIdx.y).
__global__ void k_prep_big(BigPrep P) {
  const BigPrepItem it = P.item[blockIdx.y];
  const int Rp = P.Ma, Kp = P.Kp, n = P.n;
  const int groups = Rp * Kp / 4;
  float* hi = it.dst;
  float* lo = it.dst + (size_t)Rp * Kp;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < groups; e += gridDim.x * blockDim.x) {
    const int r8 = e & 7, cm = (e >> 3) & 3, rg = (e >> 5) % (Rp >> 3), kc = (e >> 5) / (Rp >> 3);
    const int r = rg * 8 + r8, k0 = kc * 16 + cm * 4;
    float4 h, l;
    float* hp = &h.x;
    float* lp = &l.x;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + u;
      const float v = (r < n && k < n) ? (float)it.src[(size_t)r * n + k] : 0.f;
      split_tf32(v, hp[u], lp[u]);
    }
    reinterpret_cast<float4*>(hi)[e] = h;
    if (P.three) reinterpret_cast<float4*>(lo)[e] = l;
  }
}

cudaError_t launch_prep_big(const BigPrep& P, cudaStream_t stream) {
  if (P.count <= 0) return cudaSuccess;
  const int groups = P.Ma * P.Kp / 4;
  dim3 grid((unsigned)std::min(64, (groups + 255) / 256), (unsigned)P.count);
  k_prep_big<<<grid, 256, 0, stream>>>(P);
  return cudaGetLastError();
}
void launch_chain_big(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                      char* scratch, const BLayout& L, int grid, cudaStream_t stream) {
  k_chain_big<<<grid, L.nthreads, L.smem_bytes, stream>>>(descs, tasks, ntasks, queue, status,
                                                           scratch, L);
}
void launch_boundary_big(const Desc* descs, const Task* tasks, int ntasks, int* queue,
                         int* status, char* scratch, const BLayout& L, int grid,
                         cudaStream_t stream, bool pdl) {
  launch_maybe_pdl(k_boundary_big, grid, L.nthreads, L.smem_bytes, stream, pdl, descs, tasks,
                   ntasks, queue, status, scratch, L);
}
void launch_wrap_big(const Desc* descs, const Task* tasks, int ntasks, int* queue, int* status,
                     char* scratch, const BLayout& L, int grid, cudaStream_t stream, bool pdl) {
  launch_maybe_pdl(k_wrap_big, grid, L.nthreads, L.smem_bytes, stream, pdl, descs, tasks, ntasks,
                   queue, status, scratch, L);
}
cudaError_t set_smem_big(int bytes) {
  for (const void* k : {(const void*)k_chain_big, (const void*)k_wrap_big,
                        (const void*)k_boundary_big}) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t attrs_big(int which, cudaFuncAttributes* a) {
  return cudaFuncGetAttributes(a, which == 3   ? (const void*)k_wrap_big
                                  : which == 2 ? (const void*)k_boundary_big
                                               : (const void*)k_chain_big);
}

}  // namespace fd
