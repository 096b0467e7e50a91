// fd_api.cu -- host runtime behind the C ABI of include/fd.h: context, validation, planning
// (size classes, shared-memory placement, cost-sorted persistent queues), workspace and launches.
#include <algorithm>
#include <complex>
#include <map>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fd_kernels.h"

struct fd_ctx {
  int device = 0;
  int num_sms = 0;
  int max_smem_optin = 0;
  int smem_per_sm = 0;
  std::string err;
  char* scratch = nullptr;
  size_t scratch_cap = 0;
  fd::Desc* d_desc = nullptr;
  size_t desc_cap = 0;
  fd::Desc* h_desc = nullptr;  // pinned staging for the descriptor table
  size_t h_desc_cap = 0;
  int* d_queue = nullptr;
  int queue_cap = 0;
  fd::Task* d_tasks = nullptr;  // force boundary/wrap task table
  size_t tasks_cap = 0;
  fd::Task* h_tasks = nullptr;  // pinned staging
  size_t h_tasks_cap = 0;
  int* d_status = nullptr;
  int status_cap = 0;
  cudaEvent_t staging_done = nullptr;
  bool staging_pending = false;
  int last_batch = 0;
  int last_launches = 0;
  int smem_attr = 0;
  // side streams and events for concurrent size classes
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  int* last_status = nullptr;  // status array of the last graph launch (null: ctx's own)
  // autotuner plan cache: (kind, mixed, three, nx) -> threads per CTA
  std::map<long long, int> tuned;
  // optional per-launch timing (events around every kernel launch of a call)
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // pairs (start, stop)
  int ev_used = 0;
  // local (BSS) slice updates: device copy of the slice table
  fd::BssSlice* d_bss = nullptr;
  size_t bss_cap = 0;
  // intermediate-volume variant: device copy of the per-configuration sparse hopping tables
  fd::SparseHop* d_hop = nullptr;
  size_t hop_cap = 0;
  // failure-detection test hook: phased calls skip their chain launch (fd_debug_skip_chains)
  bool debug_skip_chains = false;
  // force chains split at the middle block: -1 when one chain outlasts an SM's share, 0 never,
  // 1 every configuration with at least 4 blocks (fd_set_force_split)
  int force_split = -1;
};

namespace {

using fd::Desc;
using fd::Layout;

int fail(fd_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int cuda_fail(fd_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, FD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define FD_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// What a call computes: log det/G (one persistent kernel), or the phased path (chains, boundary
// Green's functions, wraps) for the force F, the unequal-time G(tau, 0) and/or the response
// traces tr(O G_r) (bit mask).
enum Kind { K_FWD = 0, K_FORCE = 1, K_GTAU = 2, K_FORCE_GTAU = 3, K_RESP = 4 };
int kind_of(int what) {
  return ((what & FD_WANT_FORCE) ? K_FORCE : 0) | ((what & FD_WANT_GTAU) ? K_GTAU : 0) |
         ((what & FD_WANT_RESPONSE) ? K_RESP : 0);
}

// The output pointers of one call (host arrays of device pointers, or null when not wanted).
struct Outs {
  double* logdet = nullptr;
  double* const* G = nullptr;
  double* const* F = nullptr;
  double* const* Gt = nullptr;
  double* nf = nullptr;
  const double* const* O = nullptr;
  double* const* R = nullptr;
};

// One launch of a size class.  which: 0 log det/G, 1 force chains, 2 boundary G, 3 wraps.
struct Phase {
  int which;
  int mixed;  // 1: tcgen05 kernel (ML, or BL when big), 0: FP64 kernel (L)
  int big = 0;  // 1: streamed tcgen05 kernel (operands in global memory, BL)
  int merge = 0;  // boundary phase: the variant that merges split chains' checkpoints
  int seg = 0;    // shared-memory mixed chain phase: the variant with segmented-chain tasks
  Layout L;
  fd::MLayout ML;
  fd::BLayout BL{};
  int nthreads, smem, grid, occ;
  long long slot_bytes;
  size_t slot_off;  // byte offset of this launch's CTA slots in the group's scratch
  int ntasks;
};

struct Group {
  int kind;
  int nx;
  int mixed;              // any phase on the tensor cores
  std::vector<int> idx;   // user indices, cost-sorted (descending)
  std::vector<Phase> ph;  // launches, in order (one for log det/G, three for the force)
  size_t desc_off;        // first descriptor of this group in the table
  size_t scratch_off;     // byte offset of this group's scratch (slots, then FWork)
  size_t slots_bytes;     // CTA slots: one region per launch (the phases overlap)
  std::vector<fd::Task> tB, tC;  // force: boundary and wrap tasks
  std::vector<fd::Task> tA;      // force: chain tasks (b = 0 forward, 1 backward), LPT order
  size_t tA_off, tB_off, tC_off;  // their offsets in the task table
  std::vector<size_t> fws_off;   // force: per configuration, bytes from the group's FWork base
  size_t fws_bytes;
  std::vector<int> nseg;         // time-parallel log det/G: segments per configuration (or empty)
  std::vector<int> fsplit;       // force: block at which each configuration's chains split (0: not)
  std::vector<int> fseg;         // force, streamed classes: segments per chain (0: whole chains)
  // streamed tensor-core phases: chunked TF32 copies of the distinct E (and E^{-1}) matrices
  std::vector<const double*> prep_src;
  size_t prep_off = 0;   // byte offset from the group's scratch base
  size_t prep_each = 0;  // bytes per prepared matrix (hi and lo planes)
  int prep_Ma = 0, prep_Kp = 0, prep_three = 0;
  int qbase;                     // first queue counter of the group
  int grid;                      // largest grid of the phases (reported)
  int occ;
};

// Threads per CTA.  The FP64 pipe of this GPU (about 2 DFMA/clk/SM, spread over the four SM
// sub-partitions) is only kept busy when every sub-partition has warps issuing FP64 work, so even
// small matrices get 4-8 warps; the CTA routines spread their element loops over all of them.
int threads_for(int n) {
  if (n <= 12) return 128;
  return 256;
}

long long round16(long long x) { return (x + 15) & ~15LL; }

// Resident CTAs per SM for a kernel: the runtime's occupancy calculator, cross-checked by a
// direct count from the kernel's registers and shared memory (the smaller wins; 1 at least).
int resident_ctas(fd_ctx* ctx, bool mixed, int which, int nthreads, int smem_bytes) {
  int api = mixed ? fd::occupancy_mixed(which, nthreads, smem_bytes)
                  : fd::occupancy_fp64(which, nthreads, smem_bytes);
  cudaFuncAttributes fa;
  cudaError_t e = mixed ? fd::attrs_mixed(which, &fa) : fd::attrs_fp64(which, &fa);
  int manual = 1;
  if (e == cudaSuccess) {
    const int warps = (nthreads + 31) / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_warp > 0 ? 65536 / (regs_warp * warps) : 32;
    const int per_cta = smem_bytes + (int)fa.sharedSizeBytes + 1024;
    const int by_smem = per_cta > 0 ? (ctx->smem_per_sm + 1024) / per_cta : 32;
    const int by_thr = 2048 / (warps * 32);
    manual = std::max(1, std::min(std::min(by_regs, by_smem), std::min(by_thr, 32)));
  }
  // The runtime calculator reports 1 resident CTA for the tcgen05 kernels even where registers,
  // shared memory and threads allow more (ncu's launch statistics agree with the direct count);
  // those kernels use the direct count, bounded by the TMEM columns by the caller.
  if (api <= 0 || mixed) return manual;
  return std::max(1, std::min(api, manual));
}

long long tune_key(int kind, int mixed, int three, int nx) {
  return ((long long)kind << 40) | ((long long)mixed << 36) | ((long long)three << 32) | nx;
}

// Buffer sets of the kernels ("roles"): log det/G and the force chains (R_FWD), the boundary
// Green's functions (R_BOUND; R_BOUND2 with the second right-hand side of G(t, 0) beside G_t)
// and the wraps (R_WRAP); the merge of a time-parallel split (R_MERGE); boundary Green's
// functions that first merge a split chain's checkpoints (R_BOUNDM).
// R_FWD_SPARSE: log det/G with the product-form slices (no dense E).
enum Role {
  R_FWD = 0,
  R_BOUND = 2,
  R_WRAP = 3,
  R_BOUND2 = 4,
  R_MERGE = 5,
  R_FWD_SPARSE = 6,
  R_BOUNDM = 7
};

// Greedy placement: the buffers touched every slice first, then the per-block ones.
Layout plan_layout(int n, int role, int budget, int nthreads) {
  Layout L;
  memset(&L, 0, sizeof(L));
  L.nthreads = nthreads;
  const long long cm = 16LL * n * n, rm = 8LL * n * n;
  std::vector<std::pair<int, long long>> order;
  if (role == R_FWD)
    order = {{fd::B_E, rm}, {fd::B_X0, cm}, {fd::B_X1, cm}, {fd::B_T0, cm}, {fd::B_T1, cm}};
  else if (role == R_FWD_SPARSE)
    order = {{fd::B_X0, cm}, {fd::B_X1, cm}, {fd::B_T0, cm}, {fd::B_T1, cm}};
  else if (role == R_BOUND)
    order = {{fd::B_GA, cm}, {fd::B_GB, cm}};
  else if (role == R_BOUND2)
    order = {{fd::B_GA, cm}, {fd::B_GB, 2 * cm}};
  else if (role == R_MERGE)
    order = {{fd::B_X0, cm}, {fd::B_X1, cm}, {fd::B_T0, cm}, {fd::B_T1, cm}, {fd::B_GA, cm}};
  else if (role == R_BOUNDM)
    order = {{fd::B_GA, cm}, {fd::B_GB, cm}, {fd::B_X0, cm}, {fd::B_T0, cm}};
  else
    order = {{fd::B_E, rm}, {fd::B_EINV, rm}, {fd::B_GA, cm}, {fd::B_GB, cm}};
  long long used = round16(fd::small_bytes(n)) + 16;  // small vectors + queue slot
  long long gbytes = 0;
  std::vector<std::pair<int, long long>> placed;
  for (auto& b : order) {
    if (used + b.second <= budget) {
      L.in_smem[b.first] = 1;
      placed.push_back({b.first, b.second});
      used += round16(b.second);
    } else {
      L.in_smem[b.first] = 0;
      if (b.first == fd::B_E || b.first == fd::B_EINV) {
        L.off[b.first] = 0;  // read in place from the caller's input
      } else {
        L.off[b.first] = gbytes;
        gbytes += round16(b.second);
      }
    }
  }
  long long o = 0;
  for (auto& b : placed) {
    L.off[b.first] = o;
    o += round16(b.second);
  }
  L.small_off = (int)o;
  L.smem_bytes = (int)(o + round16(fd::small_bytes(n)) + 16);
  L.ws_bytes = round16(gbytes);
  L.slot_bytes = std::max(16LL, L.ws_bytes);
  return L;
}

// Mixed path: A = E (and, for the wraps, A2 = E^{-1}) and B = the product in shared memory
// (K-major TF32); for R_FWD then the FP64 block result Xc (aliasing B when it fits), the QR
// output Xn and the T pair, each in shared memory when it fits, else in the CTA's scratch slot.
// Returns smem_bytes = 0 if the tensor-core operands alone do not fit (or nx > 128).
fd::MLayout plan_mixed(int n, int role, bool three, int budget, int smem_per_sm) {
  fd::MLayout M;
  memset(&M, 0, sizeof(M));
  M.n = n;
  M.Np = (n + 7) & ~7;
  M.Kp = M.Np;
  M.N = 2 * M.Np;
  M.three = three ? 1 : 0;
  int need = M.Np + ((M.Np + 15) & ~15);
  M.tmem_cols = 32;
  while (M.tmem_cols < need) M.tmem_cols <<= 1;
  M.nthreads = n <= 12 ? 128 : 256;
  M.perm = n <= 64 ? 1 : 0;
  const long long a_bytes = (long long)(M.perm ? 128 : M.Np) * M.Kp * 4;
  const long long b_one = (long long)M.N * M.Kp * 4;
  const long long b_bytes = b_one * (three ? 2 : 1);
  const long long cm = 16LL * n * n;
  // A operands (E hi/lo, and E^{-1} hi/lo for the wraps).  With the lane permutation the
  // matrix rows sit in the first ceil(n/32) eight-row groups of each 32-lane quarter of the
  // 128-row operand; the MMA reads all 128 rows but only those lanes of the accumulator are
  // used, so up to 4 / ceil(n/32) operands share one 128-row footprint, each shifted by
  // ceil(n/32) row groups (fill_a writes only the used rows).
  const int nops = (three ? 2 : 1) * (role == R_WRAP ? 2 : 1);
  int op_off[4] = {0, 0, 0, 0};
  long long o = 0;
  if (M.perm) {
    const long long rg = (long long)(M.Kp / 4) * 128;  // one eight-row group (the SBO)
    const long long foot = (128LL * M.Kp * 4 + 127) & ~127LL;
    const int g = (n + 31) / 32, per = 4 / g;
    for (int k = 0; k < nops; ++k) {
      op_off[k] = (int)((k / per) * ((foot + 3 * rg + 127) & ~127LL) + (k % per) * g * rg);
      o = std::max(o, (long long)op_off[k] + foot);
    }
  } else {
    for (int k = 0; k < nops; ++k) {
      op_off[k] = (int)o;
      o += round16(a_bytes);
    }
  }
  int next = 0;
  M.a_hi = op_off[next++];
  M.a_lo = three ? op_off[next++] : -1;
  M.a2_hi = M.a2_lo = -1;
  if (role == R_WRAP) {
    M.a2_hi = op_off[next++];
    if (three) M.a2_lo = op_off[next++];
  }
  long long last_a = 0;
  for (int k = 0; k < nops; ++k) last_a = std::max(last_a, (long long)op_off[k]);
  o = (o + 127) & ~127LL;
  M.b_hi = (int)o;
  M.b_lo = three ? (int)(o + round16(b_one)) : -1;
  long long breg = round16(b_bytes);
  const long long fixed = round16(fd::small_bytes(n)) + 64;
  long long g = 0;  // scratch-slot bytes
  if (role == R_FWD) {
    // Xn first (the QR works in place on it), then Xc
    const bool xn_fits = o + breg + cm + fixed <= budget;
    const bool xc_alias = cm <= breg || (xn_fits ? o + std::max(breg, cm) + cm + fixed <= budget
                                                 : o + std::max(breg, cm) + fixed <= budget);
    if (xc_alias) {
      breg = std::max(breg, round16(cm));
      M.xc_smem = 1;
      M.xc_off = M.b_hi;
    } else {
      M.xc_smem = 0;
      M.xc_off = g;
      g += round16(cm);
    }
    o += breg;
    if (o + cm + fixed <= budget) {
      M.xn_smem = 1;
      M.xn_off = o;
      o += round16(cm);
    } else {
      M.xn_smem = 0;
      M.xn_off = g;
      g += round16(cm);
    }
    M.t_smem = o + 2 * round16(cm) + fixed <= budget ? 1 : 0;
    if (M.t_smem) {
      M.t0_off = o;
      o += round16(cm);
      M.t1_off = o;
      o += round16(cm);
    } else {
      M.t0_off = g;
      g += round16(cm);
      M.t1_off = g;
      g += round16(cm);
    }
  } else {  // wraps: no FP64 working matrices (Xc/Xn point at B, unused)
    o += breg;
    M.xc_smem = M.xn_smem = 1;
    M.xc_off = M.xn_off = M.b_hi;
    M.t_smem = 1;
    M.t0_off = M.t1_off = M.b_hi;
  }
  M.small_off = (int)o;
  o += round16(fd::small_bytes(n));
  M.bar_off = (int)o;
  o += 64;
  // the MMA reads 128 rows of A: keep that footprint inside the allocation
  long long foot = last_a + 128LL * M.Kp * 4;
  if (o < foot) o = foot;
  M.smem_bytes = (int)((o + 127) & ~127LL);
  // co-resident CTAs must fit the SM's 512 TMEM columns: size the request so that the
  // shared-memory occupancy limit enforces that
  const int max_ctas = 512 / M.tmem_cols;
  const int floor_bytes = smem_per_sm / (max_ctas + 1) + 1024;
  if (M.smem_bytes < floor_bytes) M.smem_bytes = (floor_bytes + 127) & ~127;
  if (M.smem_bytes > budget || M.Np > 128) {
    M.smem_bytes = 0;
    return M;
  }
  M.ws_bytes = round16(g);
  M.slot_bytes = std::max(16LL, M.ws_bytes);
  return M;
}

int validate(fd_ctx* ctx, int batch, const fd_problem* probs, const void* logdet, int prec,
             bool need_einv, bool need_e = true) {
  if (!ctx) return FD_ERR_INVALID;
  if (batch < 0) return fail(ctx, FD_ERR_INVALID, "batch < 0");
  if (batch > 0 && (!probs || !logdet)) return fail(ctx, FD_ERR_INVALID, "null probs or logdet");
  if (prec != FD_PREC_FP64 && prec != FD_PREC_MIXED_TF32 && prec != FD_PREC_MIXED_3XTF32)
    return fail(ctx, FD_ERR_INVALID, "unknown precision %d", prec);
  for (int c = 0; c < batch; ++c) {
    const fd_problem& p = probs[c];
    if (p.nx < 1 || p.nx > FD_NX_MAX)
      return fail(ctx, FD_ERR_INVALID, "config %d: nx=%d outside [1,%d]", c, p.nx, FD_NX_MAX);
    if (p.nt < 1) return fail(ctx, FD_ERR_INVALID, "config %d: nt=%d < 1", c, p.nt);
    if (p.n_stab < 1 || p.n_stab > p.nt)
      return fail(ctx, FD_ERR_INVALID, "config %d: n_stab=%d outside [1,nt]", c, p.n_stab);
    if (p.nt % p.n_stab != 0)
      return fail(ctx, FD_ERR_INVALID, "config %d: nt=%d not a multiple of n_stab=%d", c, p.nt,
                  p.n_stab);
    if (p.reserved != 0) return fail(ctx, FD_ERR_INVALID, "config %d: reserved != 0", c);
    if ((need_e && !p.expA) || !p.phi)
      return fail(ctx, FD_ERR_INVALID, "config %d: null expA or phi", c);
    if (need_einv && !p.expA_inv)
      return fail(ctx, FD_ERR_INVALID, "config %d: the force path (F, G(tau, 0), R) needs expA_inv", c);
  }
  return FD_OK;
}

// Waves a launch of `ntasks` tasks needs at `occ` resident CTAs per SM.
int waves(fd_ctx* ctx, int ntasks, int occ) {
  const int slots = std::max(1, ctx->num_sms * occ);
  return (ntasks + slots - 1) / slots;
}

Phase fp64_phase(fd_ctx* ctx, int n, int role, int which, int ntasks) {
  Phase P;
  memset(&P.ML, 0, sizeof(P.ML));
  P.which = which;
  P.mixed = 0;
  int nth = threads_for(n);
  auto it = ctx->tuned.find(tune_key(which, 0, 0, n));
  if (it != ctx->tuned.end()) {
    nth = it->second;
  } else if (nth == 256) {
    // with more tasks than resident 8-warp CTAs, 4-warp CTAs may take them all in one wave
    Layout l8 = plan_layout(n, role, ctx->max_smem_optin, 256);
    Layout l4 = plan_layout(n, role, ctx->max_smem_optin, 128);
    const int w8 = waves(ctx, ntasks, resident_ctas(ctx, false, which, 256, l8.smem_bytes));
    const int w4 = waves(ctx, ntasks, resident_ctas(ctx, false, which, 128, l4.smem_bytes));
    if (w4 < w8) nth = 128;
  }
  // a budget that keeps several CTAs per SM when everything fits, else the full opt-in budget;
  // with more tasks than SMs, a smaller budget (buffers in L1/L2-cached scratch) when that
  // needs fewer waves
  Layout full = plan_layout(n, role, 1 << 30, nth);
  int budget =
      full.smem_bytes <= ctx->smem_per_sm / 2 - 1024 ? full.smem_bytes : ctx->max_smem_optin;
  if (ntasks > ctx->num_sms && budget == ctx->max_smem_optin) {
    int best_w = waves(ctx, ntasks, resident_ctas(ctx, false, which, nth, plan_layout(n, role, budget, nth).smem_bytes));
    for (int div : {2, 3, 4}) {
      const int b2 = ctx->smem_per_sm / div - 2048;
      const int w2 = waves(ctx, ntasks, resident_ctas(ctx, false, which, nth, plan_layout(n, role, b2, nth).smem_bytes));
      if (w2 < best_w) {
        best_w = w2;
        budget = b2;
      }
    }
  }
  P.L = plan_layout(n, role, budget, nth);
  P.L.num_sms = ctx->num_sms;
  P.nthreads = nth;
  P.smem = P.L.smem_bytes;
  P.occ = resident_ctas(ctx, false, which, nth, P.smem);
  P.grid = std::max(1, std::min(ntasks, ctx->num_sms * P.occ));
  P.slot_bytes = P.L.slot_bytes;
  P.ntasks = ntasks;
  return P;
}

bool mixed_phase(fd_ctx* ctx, int n, int role, int which, bool three, int ntasks, Phase& P) {
  fd::MLayout M = plan_mixed(n, role, three, ctx->max_smem_optin, ctx->smem_per_sm);
  if (M.smem_bytes == 0) return false;
  auto it = ctx->tuned.find(tune_key(which, 1, three ? 1 : 0, n));
  if (it != ctx->tuned.end()) {
    M.nthreads = it->second;
  } else if (M.nthreads == 256) {
    const int cap = 512 / M.tmem_cols;
    const int w8 = waves(ctx, ntasks, std::min(cap, resident_ctas(ctx, true, which, 256, M.smem_bytes)));
    const int w4 = waves(ctx, ntasks, std::min(cap, resident_ctas(ctx, true, which, 128, M.smem_bytes)));
    if (w4 < w8) M.nthreads = 128;
  }
  M.num_sms = ctx->num_sms;
  memset(&P.L, 0, sizeof(P.L));
  P.which = which;
  P.mixed = 1;
  P.ML = M;
  P.nthreads = M.nthreads;
  P.smem = M.smem_bytes;
  P.occ = std::max(1, std::min(resident_ctas(ctx, true, which, M.nthreads, M.smem_bytes),
                               512 / M.tmem_cols));
  P.grid = std::max(1, std::min(ntasks, ctx->num_sms * P.occ));
  P.slot_bytes = M.slot_bytes;
  P.ntasks = ntasks;
  return true;
}

// Streamed tensor-core kernels (size classes whose operands do not fit the shared-memory tensor
// tiles): chunked operands in global memory, a shared-memory pipeline of as many stages as fit
// (at least two), TMEM for one 128-row tile of the product.  Returns smem_bytes = 0 if not even
// two stages fit.
fd::BLayout plan_big(fd_ctx* ctx, int n, bool three, bool wrap) {
  fd::BLayout B;
  memset(&B, 0, sizeof(B));
  B.n = n;
  B.three = three ? 1 : 0;
  B.Kp = (n + 15) & ~15;
  B.Ne = B.Kp;
  B.Ma = (n + 127) & ~127;
  B.Mc = (2 * n + 127) & ~127;
  const int nb16 = (2 * n + 15) & ~15;
  B.npass = (nb16 + 287) / 288;
  B.Nw = ((nb16 + B.npass - 1) / B.npass + 15) & ~15;
  B.Nb = B.npass * B.Nw;
  B.nthreads = 256;
  B.num_sms = ctx->num_sms;
  const int nbmax = wrap ? B.Nw : B.Ne;
  const int a_slab = 128 * 64, b_slab = nbmax * 64;
  B.a_lo = a_slab;
  B.b_hi = 2 * a_slab;
  B.b_lo = B.b_hi + b_slab;
  B.stage_bytes = (int)(((long long)2 * (a_slab + b_slab) + 1023) & ~1023LL);
  const long long small = wrap ? 0 : round16(fd::small_bytes(n));
  const long long rest = small + round16(16LL * n) + round16(8LL * n) + 256;
  const long long room = (long long)ctx->max_smem_optin - rest;
  const int S = (int)std::min<long long>(4, room / B.stage_bytes);
  if (S < 2) return B;  // smem_bytes = 0: does not fit
  // the chains' double-float QR works in the stages: a panel of 16 reflectors, its T and Gram
  // matrices and the GEMM tiles (df numbers of 16 bytes)
  if (!wrap && (long long)S * B.stage_bytes < 16LL * fd::big_qr_vcap(n)) return B;
  B.nstages = S;
  long long o = (long long)S * B.stage_bytes;
  B.small_off = (int)o;
  o += small;
  B.ph_off = (int)o;
  o += round16(16LL * n);
  B.dg_off = (int)o;
  o += round16(8LL * n);
  B.bar_off = (int)o;
  o += 8LL * (2 * S + 1) + 4 + 16;
  B.smem_bytes = (int)((o + 127) & ~127LL);
  B.tmem_cols = 32;
  while (B.tmem_cols < nbmax) B.tmem_cols <<= 1;
  const long long cm = 16LL * n * n;
  long long g = 0;
  if (wrap) {
    const long long bsz = 2LL * B.Nb * B.Kp * 4;  // hi and lo planes
    B.b1_off = g;
    g += (bsz + 255) & ~255LL;
    B.b2_off = g;
    g += (bsz + 255) & ~255LL;
  } else {
    B.a_off = g;
    g += (2LL * B.Mc * B.Kp * 4 + 255) & ~255LL;
    B.xc_off = g;
    g += (cm + 255) & ~255LL;
    B.xn_off = g;
    g += (cm + 255) & ~255LL;
    B.t0_off = g;
    g += (cm + 255) & ~255LL;
    B.t1_off = g;
    g += (cm + 255) & ~255LL;
  }
  B.slot_bytes = std::max(256LL, g);
  return B;
}

// Boundary Green's functions of the mixed force for the streamed size classes (double-float):
// the small-vector area and the queue slot in shared memory, three n x n df matrices per slot.
bool big_boundary_phase(fd_ctx* ctx, int n, int ntasks, Phase& P) {
  fd::BLayout B;
  memset(&B, 0, sizeof(B));
  B.n = n;
  B.nthreads = 256;
  B.num_sms = ctx->num_sms;
  B.small_off = 0;
  B.ph_off = (int)round16(fd::small_bytes(n));  // the df GEMM tiles
  B.bar_off = B.ph_off + fd::big_bound_tiles() * 16;
  B.smem_bytes = (int)((B.bar_off + 16 + 127) & ~127LL);
  B.b1_off = 0;
  B.slot_bytes = (3LL * n * n * 16 + 255) & ~255LL;
  memset(&P.L, 0, sizeof(P.L));
  memset(&P.ML, 0, sizeof(P.ML));
  P.which = 2;
  P.mixed = 0;
  P.big = 1;
  P.BL = B;
  P.nthreads = 256;
  P.smem = B.smem_bytes;
  cudaFuncAttributes fa;
  int by_regs = 1;
  if (fd::attrs_big(2, &fa) == cudaSuccess && fa.numRegs > 0)
    by_regs = std::max(1, 65536 / (((fa.numRegs * 32 + 255) / 256) * 256 * 8));
  const int by_smem = std::max(1, (ctx->smem_per_sm + 1024) / (B.smem_bytes + 1024));
  P.occ = std::max(1, std::min(by_regs, by_smem));
  P.grid = std::max(1, std::min(ntasks, ctx->num_sms * P.occ));
  P.slot_bytes = B.slot_bytes;
  P.ntasks = ntasks;
  return true;
}

bool big_phase(fd_ctx* ctx, int n, bool wrap, bool three, int ntasks, Phase& P) {
  fd::BLayout B = plan_big(ctx, n, three, wrap);
  if (B.smem_bytes == 0) return false;
  memset(&P.L, 0, sizeof(P.L));
  memset(&P.ML, 0, sizeof(P.ML));
  P.which = wrap ? 3 : 1;
  P.mixed = 1;
  P.big = 1;
  P.BL = B;
  P.nthreads = B.nthreads;
  P.smem = B.smem_bytes;
  const int by_smem = std::max(1, (ctx->smem_per_sm + 1024) / (B.smem_bytes + 1024));
  P.occ = std::max(1, std::min(by_smem, 512 / B.tmem_cols));
  P.grid = std::max(1, std::min(ntasks, ctx->num_sms * P.occ));
  P.slot_bytes = B.slot_bytes;
  P.ntasks = ntasks;
  return true;
}

// The chain phase of a size class on the tensor cores (the shared-memory tile, else the
// streamed kernel), or false.
bool tensor_chain(fd_ctx* ctx, int n, int which, bool three, int ntasks, Phase& P) {
  if (mixed_phase(ctx, n, R_FWD, which, three, ntasks, P)) {
    P.big = 0;
    return true;
  }
  return big_phase(ctx, n, false, three, ntasks, P);
}

std::vector<Group> plan(fd_ctx* ctx, int batch, const fd_problem* probs, int kind, int prec,
                        bool sparse = false) {
  std::vector<Group> groups;
  std::vector<int> order(batch);
  for (int c = 0; c < batch; ++c) order[c] = c;
  // size classes by nx, longest chains first inside a class
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (probs[a].nx != probs[b].nx) return probs[a].nx > probs[b].nx;
    const int na = probs[a].nt / probs[a].n_stab, nb = probs[b].nt / probs[b].n_stab;
    if (probs[a].nt != probs[b].nt) return probs[a].nt > probs[b].nt;
    if (na != nb) return na > nb;
    return a < b;
  });
  const bool mixed = prec != FD_PREC_FP64 && !sparse;
  const bool three = prec == FD_PREC_MIXED_3XTF32;
  // Force chains split at the middle block (ChainSpan): the halves run in parallel and the
  // boundary phase pays one merge (a product and a QR) per checkpoint of a second half, about a
  // chain's worth of QRs in all.  That pays where the chains alone would leave SMs idle: in
  // FP64 (QR-bound chains) when all the halves fit in one wave (4 batch <= SMs); measured on
  // 32 configurations of Nx = 72, beta = 32: 118 -> 95 ms, while 64 configurations at beta = 64
  // and the mixed path (tensor-core slices, FP64 merges) lose.  Classes whose boundary kernel
  // is the double-float one (streamed mixed classes) are never split (fd_kernels_big.cu).
  std::vector<char> split_c(batch, 0);
  if (kind == K_FORCE && !sparse && ctx->force_split != 0) {
    const bool auto_ok = prec == FD_PREC_FP64 && 4 * batch <= ctx->num_sms;
    for (int c = 0; c < batch; ++c) {
      const int nb = probs[c].nt / probs[c].n_stab;
      split_c[c] = nb >= 4 && (ctx->force_split > 0 || auto_ok);
    }
  }
  // Segmented chains (SegPlan) for the mixed path: S = nb / 8 segments (a power of two,
  // 4..FD_SEG_MAX, dividing nb) where one chain would outlast 1.5 times an SM's share of all the
  // call's chains -- a chain of nt slices costs ~nx^3 (nt + 150 nt / n_stab), a QR about as much
  // as 150 slice products, and re-running the segments adds up to half a chain of work.  The
  // critical path becomes 2 nb / S blocks and S - 2 merges (double-float in the streamed
  // classes, FP64 in the shared-memory ones); the boundary phase reads final checkpoints.
  std::vector<int> seg_c(batch, 0);
  if (kind == K_FORCE && !sparse && prec != FD_PREC_FP64 && ctx->force_split != 0) {
    auto ccost = [&](const fd_problem& p) {
      const double n3 = (double)p.nx * p.nx * p.nx;
      return n3 * ((double)p.nt + 150.0 * p.nt / p.n_stab);
    };
    double tot = 0.0;
    for (int c = 0; c < batch; ++c) tot += 2.0 * ccost(probs[c]);
    const double share = tot / std::max(1, ctx->num_sms);
    for (int c = 0; c < batch; ++c) {
      const int nb = probs[c].nt / probs[c].n_stab;
      // forced: segments of at least 4 blocks; automatic: of about 8
      int S = 1;
      const int mmin = ctx->force_split > 0 ? 4 : 8;
      while (2 * S <= FD_SEG_MAX && nb % (2 * S) == 0 && nb / (2 * S) >= mmin) S *= 2;
      if (S >= 4 && (ctx->force_split > 0 || ccost(probs[c]) > 1.5 * share)) seg_c[c] = S;
    }
  }
  int qnext = 0;
  size_t i = 0;
  while (i < order.size()) {
    Group g;
    g.kind = kind;
    g.nx = probs[order[i]].nx;
    while (i < order.size() && probs[order[i]].nx == g.nx) g.idx.push_back(order[i++]);
    const int n = g.nx, nd = (int)g.idx.size();
    g.mixed = 0;
    g.fws_bytes = 0;
    // Time-parallel log det/G when the class has fewer configurations than SMs (each chain
    // would be one CTA's serial work while most of the GPU idles): every chain is cut into
    // S segments (a power of two dividing its block count, at most half of it, S * configs at
    // most one wave of the chain kernel), computed from the identity in parallel and merged by a
    // stabilised product.
    int target = 1;
    if (kind == K_FWD && nd < ctx->num_sms && !sparse) {
      // as many segments as one wave of the chain kernel holds
      Phase P0;
      if (!(mixed && tensor_chain(ctx, n, 1, three, nd, P0)))
        P0 = fp64_phase(ctx, n, R_FWD, 1, nd);
      const int slots = ctx->num_sms * std::max(1, P0.occ);
      while (target < 16 && 2 * target * nd <= slots) target *= 2;
    }
    if (kind == K_FWD && target >= 2) {
      for (int k = 0; k < nd; ++k) {
        const int c = g.idx[k];
        const int nb = probs[c].nt / probs[c].n_stab;
        int S = 1;
        while (2 * S <= target && 2 * S <= nb / 2 && nb % (2 * S) == 0) S *= 2;
        g.nseg.push_back(S);
        for (int sg = 0; sg < S; ++sg) g.tA.push_back(fd::Task{k, 2 + sg});
        g.fws_off.push_back(g.fws_bytes);
        g.fws_bytes += (fd::FWork::elems(n, nb + 1, false) * 16 + 255) & ~(size_t)255;
      }
      Phase A;
      if (!(mixed && tensor_chain(ctx, n, 1, three, (int)g.tA.size(), A)))
        A = fp64_phase(ctx, n, R_FWD, 1, (int)g.tA.size());
      g.ph.push_back(A);
      g.ph.push_back(fp64_phase(ctx, n, R_MERGE, 8, nd));
    } else if (kind == K_FWD) {
      Phase P;
      if (mixed && mixed_phase(ctx, n, R_FWD, 0, three, nd, P)) {
        P.big = 0;
      } else if (mixed && big_phase(ctx, n, false, three, nd, P)) {
        // the streamed chain kernel runs the forward chains (no checkpoints)
        for (int k = 0; k < nd; ++k) g.tA.push_back(fd::Task{k, 0});
      } else {
        P = fp64_phase(ctx, n, sparse ? R_FWD_SPARSE : R_FWD, 0, nd);
      }
      g.ph.push_back(P);
    } else {
      // streamed mixed classes (double-float boundary kernel): no halves
      Phase A0;
      const bool streamed = mixed && !mixed_phase(ctx, n, R_FWD, 1, three, 2 * nd, A0) &&
                            big_phase(ctx, n, false, three, 2 * nd, A0);
      bool any_split = false;
      std::vector<fd::Task> seg_p1, seg_pre, seg_p2, seg_B, seg_C;
      for (int k = 0; k < nd; ++k) {
        const int c = g.idx[k];
        const int nb = probs[c].nt / probs[c].n_stab;
        // segments where planned, else halves (FP64 joins: not for the streamed classes)
        const int S = mixed ? seg_c[c] : 0;
        const int h = split_c[c] && !streamed && S == 0 ? nb / 2 : 0;
        g.fsplit.push_back(h);
        g.fseg.push_back(S);
        any_split |= h > 0;
        if (S) {
          // pass 1, the two prefix tasks, pass 2 (queued in that order across configurations)
          for (int sg = 0; sg <= S - 2; ++sg) {
            seg_p1.push_back(fd::Task{k, fd::CT_SFA + sg});
            seg_p1.push_back(fd::Task{k, fd::CT_SBA + sg});
          }
          seg_pre.push_back(fd::Task{k, fd::CT_SFP});
          seg_pre.push_back(fd::Task{k, fd::CT_SBP});
          for (int sg = 1; sg <= S - 1; ++sg) {
            seg_p2.push_back(fd::Task{k, fd::CT_SFB + sg});
            seg_p2.push_back(fd::Task{k, fd::CT_SBB + sg});
          }
        } else {
          g.tA.push_back(fd::Task{k, fd::CT_FWD});
          g.tA.push_back(fd::Task{k, fd::CT_BWD});
        }
        if (h) {
          g.tA.push_back(fd::Task{k, fd::CT_FWD2});
          g.tA.push_back(fd::Task{k, fd::CT_BWD2});
        }
        // a segmented configuration's checkpoints come last: its boundary and wrap tasks go to
        // the end of their queues (a wait that sees no progress for ~4 s gives up)
        std::vector<fd::Task>& tb = S ? seg_B : g.tB;
        std::vector<fd::Task>& tc = S ? seg_C : g.tC;
        for (int b = 2; b <= nb; ++b) tb.push_back(fd::Task{k, b});
        if (h) tb.push_back(fd::Task{k, 1});  // G_0 and log det from the halves
        for (int b = 1; b <= nb; ++b) tc.push_back(fd::Task{k, b});
        const int extra = h > 0 ? 1 : S > 0 ? 2 * (S - 2) : 0;
        g.fws_off.push_back(g.fws_bytes);
        g.fws_bytes += (fd::FWork::elems(n, nb, (kind & K_GTAU) != 0, (kind & K_RESP) != 0,
                                         extra) * 16 + 255) & ~(size_t)255;
      }
      // chains longest first (LPT): a forward chain carries one more QR and the assembly, so for
      // equal configurations all forward chains go out before the backward ones and the SMs that
      // receive an extra chain get a short one
      auto chain_cost = [&](const fd::Task& t) {
        const fd_problem& p = probs[g.idx[t.desc]];
        const long long nb = p.nt / p.n_stab, h = g.fsplit[t.desc];
        if (h) {
          const long long blocks = t.b == fd::CT_FWD ? h
                                   : t.b == fd::CT_BWD2 ? h - 1 : nb - h;
          return blocks * p.n_stab + 16 * blocks;
        }
        return t.b == 0 ? (long long)p.nt + 16 * (nb + 1)
                        : (long long)(p.nt - p.n_stab) + 16 * (nb - 1);
      };
      std::stable_sort(g.tA.begin(), g.tA.end(), [&](const fd::Task& a, const fd::Task& b) {
        return chain_cost(a) > chain_cost(b);
      });
      // segmented chains: every task waits only for tasks queued before it (pass 1, then the
      // prefixes, then the whole chains, then pass 2 by segment)
      std::stable_sort(seg_p2.begin(), seg_p2.end(), [](const fd::Task& a, const fd::Task& b) {
        return (a.b & 15) < (b.b & 15);
      });
      if (!seg_p1.empty()) {
        std::vector<fd::Task> all = seg_p1;
        all.insert(all.end(), seg_pre.begin(), seg_pre.end());
        all.insert(all.end(), g.tA.begin(), g.tA.end());
        all.insert(all.end(), seg_p2.begin(), seg_p2.end());
        g.tA.swap(all);
        g.tB.insert(g.tB.end(), seg_B.begin(), seg_B.end());
        g.tC.insert(g.tC.end(), seg_C.begin(), seg_C.end());
      }
      Phase A, C;
      const int ntA = (int)g.tA.size();
      bool any_seg = false;
      for (int S : g.fseg) any_seg |= S > 0;
      // the shared-memory mixed kernel has a variant with the segmented chains' tasks (which 9)
      const int whichA = any_seg && !streamed ? 9 : 1;
      if (!(mixed && tensor_chain(ctx, n, whichA, three, ntA, A)))
        A = fp64_phase(ctx, n, R_FWD, 1, ntA);
      if (A.mixed && !A.big && whichA == 9) {
        A.which = 1;
        A.seg = 1;
      }
      const bool two_rhs = (kind & K_GTAU) && (kind & (K_FORCE | K_RESP));
      // halves or segments: the boundary variant that merges / waits on segment flags
      const bool bvar = any_split || (any_seg && !streamed);
      Phase B = bvar ? fp64_phase(ctx, n, R_BOUNDM, 9, std::max(1, (int)g.tB.size()))
                     : fp64_phase(ctx, n, two_rhs ? R_BOUND2 : R_BOUND, 2,
                                  std::max(1, (int)g.tB.size()));
      B.which = 2;
      B.merge = bvar ? 1 : 0;
      // the tensor-core wrap kernels cover the force rows (the shared-memory one also the
      // response traces); G(tau, 0) wraps run in FP64
      const bool mixed_wrap = mixed && !(kind & K_GTAU);
      const int ntC = (int)g.tC.size();
      if (mixed_wrap && mixed_phase(ctx, n, R_WRAP, 3, three, ntC, C))
        C.big = 0;
      else if (!(mixed_wrap && !(kind & K_RESP) && big_phase(ctx, n, true, three, ntC, C)))
        C = fp64_phase(ctx, n, R_WRAP, 3, ntC);
      // the mixed force of a streamed class: boundary Green's functions in double-float
      if (C.big && A.big && kind == K_FORCE)
        big_boundary_phase(ctx, n, std::max(1, (int)g.tB.size()), B);
      g.ph.push_back(A);
      g.ph.push_back(B);
      g.ph.push_back(C);
    }
    // streamed tensor-core phases read chunked TF32 copies of the class's distinct matrices
    bool big_chain = false, big_wrap = false;
    for (auto& P : g.ph) {
      if (P.big && P.which == 3) big_wrap = true;
      else if (P.big) big_chain = true;
    }
    if (big_chain || big_wrap) {
      const fd::BLayout& BL = g.ph[0].big ? g.ph[0].BL : g.ph.back().BL;
      g.prep_Ma = BL.Ma;
      g.prep_Kp = BL.Kp;
      g.prep_three = BL.three;
      g.prep_each = ((size_t)2 * BL.Ma * BL.Kp * 4 + 255) & ~(size_t)255;
      for (int c : g.idx) {
        const double* mats[2] = {probs[c].expA, big_wrap ? probs[c].expA_inv : nullptr};
        for (const double* mtx : mats)
          if (mtx && std::find(g.prep_src.begin(), g.prep_src.end(), mtx) == g.prep_src.end())
            g.prep_src.push_back(mtx);
      }
    }
    g.slots_bytes = 0;
    g.grid = 0;
    g.occ = 0;
    for (auto& P : g.ph) {
      g.mixed |= P.mixed;
      // the launches of the phased path run concurrently: each gets its own slots
      P.slot_off = g.slots_bytes;
      g.slots_bytes += ((size_t)P.grid * (size_t)P.slot_bytes + 255) & ~(size_t)255;
      g.grid = std::max(g.grid, P.grid);
      g.occ = std::max(g.occ, P.occ);
    }
    g.qbase = qnext;
    qnext += (int)g.ph.size();
    groups.push_back(g);
  }
  return groups;
}

int ensure(fd_ctx* ctx, size_t ndesc, size_t nstatus, size_t nqueue, size_t scratch_bytes,
           size_t ntasks) {
  if (ntasks > ctx->tasks_cap) {
    if (ctx->d_tasks) cudaFree(ctx->d_tasks);
    ctx->d_tasks = nullptr;
    size_t cap = std::max<size_t>(ntasks, 1024);
    FD_CUDA(ctx, cudaMalloc(&ctx->d_tasks, cap * sizeof(fd::Task)));
    ctx->tasks_cap = cap;
  }
  if (ntasks > ctx->h_tasks_cap) {
    if (ctx->staging_pending) cudaEventSynchronize(ctx->staging_done);
    ctx->staging_pending = false;
    if (ctx->h_tasks) cudaFreeHost(ctx->h_tasks);
    ctx->h_tasks = nullptr;
    size_t cap = std::max<size_t>(ntasks, 1024);
    FD_CUDA(ctx, cudaMallocHost(&ctx->h_tasks, cap * sizeof(fd::Task)));
    ctx->h_tasks_cap = cap;
  }
  if (ndesc > ctx->desc_cap) {
    if (ctx->d_desc) cudaFree(ctx->d_desc);
    ctx->d_desc = nullptr;
    size_t cap = std::max<size_t>(ndesc, 256);
    FD_CUDA(ctx, cudaMalloc(&ctx->d_desc, cap * sizeof(Desc)));
    ctx->desc_cap = cap;
  }
  if (ndesc > ctx->h_desc_cap) {
    if (ctx->staging_pending) cudaEventSynchronize(ctx->staging_done);
    ctx->staging_pending = false;
    if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
    ctx->h_desc = nullptr;
    size_t cap = std::max<size_t>(ndesc, 256);
    FD_CUDA(ctx, cudaMallocHost(&ctx->h_desc, cap * sizeof(Desc)));
    ctx->h_desc_cap = cap;
  }
  if ((int)nstatus > ctx->status_cap) {
    if (ctx->d_status) cudaFree(ctx->d_status);
    ctx->d_status = nullptr;
    int cap = std::max<int>((int)nstatus, 256);
    FD_CUDA(ctx, cudaMalloc(&ctx->d_status, cap * sizeof(int)));
    ctx->status_cap = cap;
  }
  if ((int)nqueue > ctx->queue_cap) {
    if (ctx->d_queue) cudaFree(ctx->d_queue);
    ctx->d_queue = nullptr;
    int cap = std::max<int>((int)nqueue, 64);
    FD_CUDA(ctx, cudaMalloc(&ctx->d_queue, cap * sizeof(int)));
    ctx->queue_cap = cap;
  }
  if (scratch_bytes > ctx->scratch_cap) {
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    FD_CUDA(ctx, cudaMalloc(&ctx->scratch, scratch_bytes));
    ctx->scratch_cap = scratch_bytes;
  }
  return FD_OK;
}

size_t scratch_need(std::vector<Group>& groups) {
  size_t off = 0;
  for (auto& g : groups) {
    g.scratch_off = off;
    off += g.slots_bytes + g.fws_bytes;
    off = (off + 255) & ~(size_t)255;
    g.prep_off = off - g.scratch_off;
    off += g.prep_src.size() * g.prep_each;
  }
  return off;
}

size_t task_count(const std::vector<Group>& groups) {
  size_t t = 0;
  for (auto& g : groups) t += g.tA.size() + g.tB.size() + g.tC.size();
  return t;
}

int queue_count(const std::vector<Group>& groups) {
  int q = 0;
  for (auto& g : groups) q += (int)g.ph.size();
  return q;
}

// Host descriptor and task tables of a call.  `scratch` is the device scratch base (the force
// workspace of each configuration lives inside it).
void build_tables(std::vector<Group>& groups, const fd_problem* probs, const Outs& o,
                  char* scratch, int* sync, Desc* out, fd::Task* tasks) {
  size_t k = 0, t = 0;
  for (auto& g : groups) {
    g.desc_off = k;
    for (size_t q = 0; q < g.idx.size(); ++q) {
      const int c = g.idx[q];
      const fd_problem& p = probs[c];
      Desc d;
      d.nx = p.nx;
      d.nt = p.nt;
      d.nstab = p.n_stab;
      d.user_index = c;
      d.E = p.expA;
      d.Einv = p.expA_inv;
      d.phi = p.phi;
      d.logdet = o.logdet + 2 * (size_t)c;
      d.G = o.G ? (double2*)o.G[c] : nullptr;
      d.F = o.F ? (double2*)o.F[c] : nullptr;
      d.Gt = o.Gt ? (double2*)o.Gt[c] : nullptr;
      d.nf = o.nf ? o.nf + 2 * (size_t)c : nullptr;
      d.O = o.O ? o.O[c] : nullptr;
      d.R = o.R ? (double2*)o.R[c] : nullptr;
      d.sync = g.kind != K_FWD ? sync + fd::SF_NUM * (size_t)c : nullptr;
      d.fws = (g.kind != K_FWD || !g.nseg.empty())
                  ? (double2*)(scratch + g.scratch_off + g.slots_bytes + g.fws_off[q])
                  : nullptr;
      d.nseg = g.nseg.empty() ? 0 : g.nseg[q];
      d.fsplit = g.fsplit.empty() ? 0 : g.fsplit[q];
      d.fseg = g.fseg.empty() ? 0 : g.fseg[q];
      d.Ec = d.Eic = nullptr;
      for (size_t i = 0; i < g.prep_src.size(); ++i) {
        const float* dst = (const float*)(scratch + g.scratch_off + g.prep_off + i * g.prep_each);
        if (g.prep_src[i] == p.expA) d.Ec = dst;
        if (g.prep_src[i] == p.expA_inv) d.Eic = dst;
      }
      out[k++] = d;
    }
    g.tA_off = t;
    for (auto& x : g.tA) tasks[t++] = x;
    g.tB_off = t;
    for (auto& x : g.tB) tasks[t++] = x;
    g.tC_off = t;
    for (auto& x : g.tC) tasks[t++] = x;
  }
}

// Side streams for running several size classes concurrently (fork/join with events; the same
// pattern is recorded into CUDA graphs as parallel branches).
int ensure_side(fd_ctx* ctx, size_t n) {
  while (ctx->side.size() < n) {
    cudaStream_t s;
    cudaEvent_t e;
    FD_CUDA(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    FD_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->side.push_back(s);
    ctx->join.push_back(e);
  }
  if (!ctx->fork) FD_CUDA(ctx, cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming));
  return FD_OK;
}

// Enqueue one call: reset the queues and the status words, then each size class's launches in
// order (one persistent kernel for log det/G; chains, boundary and wrap kernels for the force) --
// on `stream` itself for a single class, else forked onto side streams and joined back.
int enqueue(fd_ctx* ctx, std::vector<Group>& groups, Desc* d_desc, fd::Task* d_tasks,
            int* d_queue, int* d_status, char* scratch, int batch, cudaStream_t stream,
            bool timing, const fd::SparseHop* hops = nullptr) {
  const int nq = queue_count(groups);
  FD_CUDA(ctx, cudaMemsetAsync(d_queue, 0, sizeof(int) * nq, stream));
  FD_CUDA(ctx, cudaMemsetAsync(d_status, 0xFF, sizeof(int) * batch, stream));  // pending
  // progress flags of the phased path (after the status words)
  FD_CUDA(ctx, cudaMemsetAsync(d_status + batch, 0, sizeof(int) * fd::SF_NUM * batch, stream));
  if (timing) {
    while ((int)ctx->ev.size() < 2 * nq) {
      cudaEvent_t e;
      FD_CUDA(ctx, cudaEventCreate(&e));
      ctx->ev.push_back(e);
    }
    ctx->ev_used = 2 * nq;
  }
  // with per-launch timing the size classes run one after another on the call's stream, so each
  // duration is that kernel's alone (as a profiler's serialised launch list sees it)
  const bool fork = groups.size() > 1 && !timing;
  const size_t nside = std::min<size_t>(groups.size(), 8);
  if (fork) {
    int rc = ensure_side(ctx, nside);
    if (rc != FD_OK) return rc;
    FD_CUDA(ctx, cudaEventRecord(ctx->fork, stream));
    for (size_t i = 0; i < nside; ++i) FD_CUDA(ctx, cudaStreamWaitEvent(ctx->side[i], ctx->fork, 0));
  }
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    Group& g = groups[gi];
    cudaStream_t s = fork ? ctx->side[gi % nside] : stream;
    const Desc* dd = d_desc + g.desc_off;
    const int nd = (int)g.idx.size();
    for (size_t i0 = 0; i0 < g.prep_src.size(); i0 += FD_BIG_PREP_MAX) {
      fd::BigPrep bp;
      memset(&bp, 0, sizeof(bp));
      bp.n = g.nx;
      bp.Ma = g.prep_Ma;
      bp.Kp = g.prep_Kp;
      bp.three = g.prep_three;
      bp.count = (int)std::min<size_t>(FD_BIG_PREP_MAX, g.prep_src.size() - i0);
      for (int i = 0; i < bp.count; ++i) {
        bp.item[i].src = g.prep_src[i0 + i];
        bp.item[i].dst = (float*)(scratch + g.scratch_off + g.prep_off + (i0 + i) * g.prep_each);
      }
      FD_CUDA(ctx, fd::launch_prep_big(bp, s));
      ctx->last_launches++;
    }
    for (size_t pi = 0; pi < g.ph.size(); ++pi) {
      const Phase& P = g.ph[pi];
      char* scr = scratch + g.scratch_off + P.slot_off;
      const int qi = g.qbase + (int)pi;
      if (timing) FD_CUDA(ctx, cudaEventRecord(ctx->ev[2 * qi], s));
      if ((P.which == 2 && g.tB.empty()) ||  // single-block configurations: no boundary phase
          (P.which == 1 && g.kind != K_FWD && ctx->debug_skip_chains)) {
        if (timing) FD_CUDA(ctx, cudaEventRecord(ctx->ev[2 * qi + 1], s));
        continue;
      }
      switch (P.big ? -P.which : P.which) {
        case 0:
          if (P.mixed)
            fd::launch_fwd_mixed(dd, nd, d_queue + qi, d_status, scr, P.ML, P.grid, s);
          else
            fd::launch_fwd_fp64(dd, nd, d_queue + qi, d_status, scr, P.L, P.grid, s, hops);
          break;
        case 1:
          if (P.mixed)
            fd::launch_chain_mixed(dd, d_tasks + g.tA_off, (int)g.tA.size(), d_queue + qi,
                                   d_status, scr, P.ML, P.grid, s, P.seg != 0);
          else
            fd::launch_chain_fp64(dd, d_tasks + g.tA_off, (int)g.tA.size(), d_queue + qi,
                                  d_status, scr, P.L, P.grid, s);
          break;
        case 8:
          fd::launch_merge_fp64(dd, nd, d_queue + qi, d_status, scr, P.L, P.grid, s);
          break;
        case -1:  // streamed tensor-core chains (force, segments, or log det/G)
          fd::launch_chain_big(dd, d_tasks + g.tA_off, (int)g.tA.size(), d_queue + qi, d_status,
                               scr, P.BL, P.grid, s);
          break;
        case -2:
          fd::launch_boundary_big(dd, d_tasks + g.tB_off, (int)g.tB.size(), d_queue + qi,
                                  d_status, scr, P.BL, P.grid, s, !timing);
          break;
        case -3:
          fd::launch_wrap_big(dd, d_tasks + g.tC_off, (int)g.tC.size(), d_queue + qi, d_status,
                              scr, P.BL, P.grid, s, !timing);
          break;
        case 2:
          fd::launch_boundary_fp64(dd, d_tasks + g.tB_off, (int)g.tB.size(), d_queue + qi,
                                   d_status, scr, P.L, P.grid, s, !timing, P.merge != 0);
          break;
        default:
          if (P.mixed)
            fd::launch_wrap_mixed(dd, d_tasks + g.tC_off, (int)g.tC.size(), d_queue + qi,
                                  d_status, scr, P.ML, P.grid, s, !timing);
          else
            fd::launch_wrap_fp64(dd, d_tasks + g.tC_off, (int)g.tC.size(), d_queue + qi,
                                 d_status, scr, P.L, P.grid, s, !timing);
      }
      ctx->last_launches++;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
      if (timing) FD_CUDA(ctx, cudaEventRecord(ctx->ev[2 * qi + 1], s));
    }
  }
  if (fork) {
    for (size_t i = 0; i < nside; ++i) {
      FD_CUDA(ctx, cudaEventRecord(ctx->join[i], ctx->side[i]));
      FD_CUDA(ctx, cudaStreamWaitEvent(stream, ctx->join[i], 0));
    }
  }
  return FD_OK;
}

int run(fd_ctx* ctx, int batch, const fd_problem* probs, const Outs& o, int prec, void* stream_,
        int kind, const fd::SparseHop* d_hop = nullptr) {
  cudaStream_t stream = (cudaStream_t)stream_;
  ctx->last_launches = 0;
  ctx->last_batch = batch;
  ctx->last_status = nullptr;
  if (batch == 0) return FD_OK;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  // Mixed precision: size classes whose operands fit in shared memory run the tensor-core
  // kernels of fd_kernels_mixed.cu, larger ones the streamed kernels of fd_kernels_big.cu
  // (fd_plan_query says which).
  std::vector<Group> groups = plan(ctx, batch, probs, kind, prec, d_hop != nullptr);
  size_t need = scratch_need(groups);
  const size_t ntasks = task_count(groups);
  int rc = ensure(ctx, (size_t)batch, (size_t)batch * (1 + fd::SF_NUM), queue_count(groups), need,
                  ntasks);
  if (rc != FD_OK) return rc;
  if (ctx->staging_pending) {
    FD_CUDA(ctx, cudaEventSynchronize(ctx->staging_done));
    ctx->staging_pending = false;
  }
  build_tables(groups, probs, o, ctx->scratch, ctx->d_status + batch, ctx->h_desc, ctx->h_tasks);
  FD_CUDA(ctx, cudaMemcpyAsync(ctx->d_desc, ctx->h_desc, sizeof(Desc) * batch,
                               cudaMemcpyHostToDevice, stream));
  if (ntasks)
    FD_CUDA(ctx, cudaMemcpyAsync(ctx->d_tasks, ctx->h_tasks, sizeof(fd::Task) * ntasks,
                                 cudaMemcpyHostToDevice, stream));
  FD_CUDA(ctx, cudaEventRecord(ctx->staging_done, stream));
  ctx->staging_pending = true;
  return enqueue(ctx, groups, ctx->d_desc, ctx->d_tasks, ctx->d_queue, ctx->d_status,
                 ctx->scratch, batch, stream, ctx->timing, d_hop);
}

// A captured call: its own descriptor table, queues, status words and scratch (so later calls
// on the context cannot move memory the graph uses), replayed with one cudaGraphLaunch.
struct GraphObj {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  Desc* d_desc = nullptr;
  fd::Task* d_tasks = nullptr;
  int* d_queue = nullptr;
  int* d_status = nullptr;
  char* scratch = nullptr;
  int batch = 0;
  int launches = 0;
};

void graph_free(GraphObj* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->d_desc) cudaFree(g->d_desc);
  if (g->d_tasks) cudaFree(g->d_tasks);
  if (g->d_queue) cudaFree(g->d_queue);
  if (g->d_status) cudaFree(g->d_status);
  if (g->scratch) cudaFree(g->scratch);
  delete g;
}

// Factors of the product form (Section 8): prod_k (1 + gamma_k x) equals the truncated
// exponential series s_n(x) = sum_{j<=n} x^j / j!, so gamma_k = -1 / x_k over the roots x_k of
// s_n.  The roots come from the Weierstrass (Durand-Kerner) simultaneous iteration on the monic
// polynomial n! s_n(x) = sum_j (n!/j!) x^j, then one Newton step each; the factors are accepted
// only if multiplying them out reproduces 1/j! to 1e-12.  Sorted by (re, im).
int taylor_factors(int n, std::complex<double>* gamma) {
  typedef std::complex<double> cd;
  if (n < 1 || n > FD_SPARSE_NFAC_MAX) return FD_ERR_INVALID;
  std::vector<double> a(n + 1);  // a[j] = n! / j!
  for (int j = 0; j <= n; ++j) {
    double v = 1.0;
    for (int k = j + 1; k <= n; ++k) v *= k;
    a[j] = v;
  }
  auto poly = [&](cd z) {
    cd s = a[n];
    for (int j = n - 1; j >= 0; --j) s = s * z + a[j];
    return s;
  };
  auto dpoly = [&](cd z) {
    cd s = (double)n * a[n];
    for (int j = n - 1; j >= 1; --j) s = s * z + (double)j * a[j];
    return s;
  };
  std::vector<cd> z(n);
  const cd seed(0.4, 0.9);
  cd w = 1.0;
  for (int k = 0; k < n; ++k) {
    z[k] = (0.5 + 0.5 * n) * w;
    w *= seed;
  }
  for (int it = 0; it < 1000; ++it) {
    double step = 0.0;
    for (int k = 0; k < n; ++k) {
      cd den = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != k) den *= z[k] - z[j];
      const cd d = poly(z[k]) / den;
      z[k] -= d;
      step = std::max(step, std::abs(d) / std::max(1.0, std::abs(z[k])));
    }
    if (step < 1e-15) break;
  }
  for (int k = 0; k < n; ++k) z[k] -= poly(z[k]) / dpoly(z[k]);
  std::vector<cd> g(n);
  for (int k = 0; k < n; ++k) g[k] = -1.0 / z[k];
  std::sort(g.begin(), g.end(), [](const cd& x, const cd& y) {
    return x.real() != y.real() ? x.real() < y.real() : x.imag() < y.imag();
  });
  // check: prod_k (1 + g_k x) = sum_j x^j / j!
  std::vector<cd> c(n + 1, 0.0);
  c[0] = 1.0;
  for (int k = 0; k < n; ++k)
    for (int j = k + 1; j >= 1; --j) c[j] += g[k] * c[j - 1];
  double inv_fact = 1.0;
  for (int j = 0; j <= n; ++j) {
    if (j > 0) inv_fact /= j;
    if (std::abs(c[j] - inv_fact) > 1e-12) return FD_ERR_NUMERIC;
  }
  for (int k = 0; k < n; ++k) gamma[k] = g[k];
  return FD_OK;
}

}  // namespace

extern "C" {

int fd_ctx_create(fd_ctx** out, int device) {
  if (!out) return FD_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return FD_ERR_CUDA;
  if (device < 0 || device >= ndev) return FD_ERR_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return FD_ERR_CUDA;
  fd_ctx* ctx = new fd_ctx();
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  cudaDeviceGetAttribute(&ctx->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  if (cudaEventCreateWithFlags(&ctx->staging_done, cudaEventDisableTiming) != cudaSuccess ||
      fd::set_smem_fp64(ctx->max_smem_optin) != cudaSuccess ||
      fd::set_smem_mixed(ctx->max_smem_optin) != cudaSuccess ||
      fd::set_smem_big(ctx->max_smem_optin) != cudaSuccess) {
    delete ctx;
    return FD_ERR_CUDA;
  }
  ctx->smem_attr = ctx->max_smem_optin;
  *out = ctx;
  return FD_OK;
}

void fd_ctx_destroy(fd_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->staging_pending) cudaEventSynchronize(ctx->staging_done);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->d_desc) cudaFree(ctx->d_desc);
  if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
  if (ctx->d_queue) cudaFree(ctx->d_queue);
  if (ctx->d_tasks) cudaFree(ctx->d_tasks);
  if (ctx->h_tasks) cudaFreeHost(ctx->h_tasks);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_bss) cudaFree(ctx->d_bss);
  if (ctx->d_hop) cudaFree(ctx->d_hop);
  if (ctx->staging_done) cudaEventDestroy(ctx->staging_done);
  for (auto e : ctx->ev) cudaEventDestroy(e);
  for (auto s : ctx->side) cudaStreamDestroy(s);
  for (auto e : ctx->join) cudaEventDestroy(e);
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  delete ctx;
}

const char* fd_last_error(const fd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int fd_reserve(fd_ctx* ctx, int batch, const fd_problem* probs, int what, int prec) {
  double dummy;
  int rc = validate(ctx, batch, probs, &dummy, prec, kind_of(what) != K_FWD);
  if (rc != FD_OK) return rc;
  if (batch == 0) return FD_OK;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  std::vector<Group> groups = plan(ctx, batch, probs, kind_of(what), prec);
  size_t need = scratch_need(groups);
  rc = ensure(ctx, (size_t)batch, (size_t)batch * (1 + fd::SF_NUM), queue_count(groups), need,
              task_count(groups));
  if (rc != FD_OK) return rc;
  if (ctx->max_smem_optin > ctx->smem_attr) {
    FD_CUDA(ctx, fd::set_smem_fp64(ctx->max_smem_optin));
    ctx->smem_attr = ctx->max_smem_optin;
  }
  return FD_OK;
}

int fd_logdet(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet, int prec,
              void* stream) {
  int rc = validate(ctx, batch, probs, logdet, prec, false);
  if (rc != FD_OK) return rc;
  Outs o;
  o.logdet = logdet;
  return run(ctx, batch, probs, o, prec, stream, K_FWD);
}

int fd_green(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet, double* const* G,
             int prec, void* stream) {
  int rc = validate(ctx, batch, probs, logdet, prec, false);
  if (rc != FD_OK) return rc;
  if (batch > 0 && !G) return fail(ctx, FD_ERR_INVALID, "null G array");
  for (int c = 0; c < batch; ++c)
    if (!G[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null G", c);
  Outs o;
  o.logdet = logdet;
  o.G = G;
  return run(ctx, batch, probs, o, prec, stream, K_FWD);
}

int fd_force(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet, double* const* G,
             double* const* F, int prec, void* stream) {
  int rc = validate(ctx, batch, probs, logdet, prec, true);
  if (rc != FD_OK) return rc;
  if (batch > 0 && !F) return fail(ctx, FD_ERR_INVALID, "null F array");
  for (int c = 0; c < batch; ++c) {
    if (!F[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null F", c);
    if (G && !G[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null G", c);
  }
  Outs o;
  o.logdet = logdet;
  o.G = G;
  o.F = F;
  return run(ctx, batch, probs, o, prec, stream, K_FORCE);
}

int fd_green_tau(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet,
                 double* const* G, double* const* Gtau, double* const* F, int prec, void* stream) {
  int rc = validate(ctx, batch, probs, logdet, prec, true);
  if (rc != FD_OK) return rc;
  if (batch > 0 && !Gtau) return fail(ctx, FD_ERR_INVALID, "null Gtau array");
  for (int c = 0; c < batch; ++c) {
    if (!Gtau[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null Gtau", c);
    if (G && !G[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null G", c);
    if (F && !F[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null F", c);
  }
  Outs o;
  o.logdet = logdet;
  o.G = G;
  o.F = F;
  o.Gt = Gtau;
  return run(ctx, batch, probs, o, prec, stream, F ? K_FORCE_GTAU : K_GTAU);
}

int fd_observables(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet,
                   double* const* G, double* const* F, double* nferm, const double* const* O,
                   double* const* R, int prec, void* stream) {
  if (!ctx) return FD_ERR_INVALID;
  if ((O == nullptr) != (R == nullptr))
    return fail(ctx, FD_ERR_INVALID, "O and R must both be given or both be NULL");
  const int kind = (F ? K_FORCE : 0) | (R ? K_RESP : 0);
  int rc = validate(ctx, batch, probs, logdet, prec, kind != K_FWD);
  if (rc != FD_OK) return rc;
  for (int c = 0; c < batch; ++c) {
    if (G && !G[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null G", c);
    if (F && !F[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null F", c);
    if (R && (!R[c] || !O[c])) return fail(ctx, FD_ERR_INVALID, "config %d: null O or R", c);
  }
  Outs o;
  o.logdet = logdet;
  o.G = G;
  o.F = F;
  o.nf = nferm;
  o.O = O;
  o.R = R;
  return run(ctx, batch, probs, o, prec, stream, kind);
}

int fd_bss_update(fd_ctx* ctx, int batch, const fd_bss_slice* slices, double* dlogdet,
                  void* stream_) {
  if (!ctx) return FD_ERR_INVALID;
  if (batch < 0) return fail(ctx, FD_ERR_INVALID, "batch < 0");
  if (batch == 0) return FD_OK;
  if (!slices || !dlogdet) return fail(ctx, FD_ERR_INVALID, "null slices or dlogdet");
  std::vector<fd::BssSlice> h(batch);
  int maxn = 1;
  for (int c = 0; c < batch; ++c) {
    const fd_bss_slice& s = slices[c];
    if (s.nx < 1 || s.nx > FD_NX_MAX)
      return fail(ctx, FD_ERR_INVALID, "slice %d: nx=%d outside [1,%d]", c, s.nx, FD_NX_MAX);
    if (s.reserved != 0) return fail(ctx, FD_ERR_INVALID, "slice %d: reserved != 0", c);
    if (!s.G || !s.phi_row || !s.dphi || !s.u || !s.w || !s.accepted)
      return fail(ctx, FD_ERR_INVALID, "slice %d: null pointer", c);
    h[c] = fd::BssSlice{s.nx, 0, (double2*)s.G, s.phi_row, s.dphi, s.u, s.w, s.accepted};
    maxn = std::max(maxn, s.nx);
  }
  cudaStream_t stream = (cudaStream_t)stream_;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  if ((size_t)batch > ctx->bss_cap) {
    if (ctx->d_bss) {
      FD_CUDA(ctx, cudaStreamSynchronize(stream));
      cudaFree(ctx->d_bss);
    }
    ctx->d_bss = nullptr;
    const size_t cap = std::max<size_t>(batch, 256);
    FD_CUDA(ctx, cudaMalloc(&ctx->d_bss, cap * sizeof(fd::BssSlice)));
    ctx->bss_cap = cap;
  }
  // pageable source: the copy is staged before the call returns
  FD_CUDA(ctx, cudaMemcpyAsync(ctx->d_bss, h.data(), sizeof(fd::BssSlice) * batch,
                               cudaMemcpyHostToDevice, stream));
  const int grid = std::min(batch, ctx->num_sms * 8);
  if (ctx->timing) {
    while (ctx->ev.size() < 2) {
      cudaEvent_t ev;
      FD_CUDA(ctx, cudaEventCreate(&ev));
      ctx->ev.push_back(ev);
    }
    ctx->ev_used = 2;
    FD_CUDA(ctx, cudaEventRecord(ctx->ev[0], stream));
  }
  cudaError_t e = fd::launch_bss(ctx->d_bss, batch, maxn, dlogdet, grid, stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
  if (ctx->timing) FD_CUDA(ctx, cudaEventRecord(ctx->ev[1], stream));
  ctx->last_launches = 1;
  return FD_OK;
}

int fd_debug_skip_chains(fd_ctx* ctx, int on) {
  if (!ctx) return FD_ERR_INVALID;
  ctx->debug_skip_chains = on != 0;
  return FD_OK;
}

int fd_set_force_split(fd_ctx* ctx, int mode) {
  if (!ctx || mode < -1 || mode > 1) return FD_ERR_INVALID;
  ctx->force_split = mode;
  return FD_OK;
}

int fd_taylor_factors(int n, double* gamma) {
  if (!gamma) return FD_ERR_INVALID;
  std::complex<double> g[FD_SPARSE_NFAC_MAX];
  const int rc = taylor_factors(n, g);
  if (rc != FD_OK) return rc;
  for (int k = 0; k < n; ++k) {
    gamma[2 * k] = g[k].real();
    gamma[2 * k + 1] = g[k].imag();
  }
  return FD_OK;
}

int fd_green_sparse(fd_ctx* ctx, int batch, const fd_problem* probs, const fd_sparse_hop* hop,
                    double* logdet, double* const* G, void* stream) {
  int rc = validate(ctx, batch, probs, logdet, FD_PREC_FP64, false, false);
  if (rc != FD_OK) return rc;
  if (batch == 0) return FD_OK;
  if (!hop) return fail(ctx, FD_ERR_INVALID, "null hop array");
  std::vector<fd::SparseHop> h(batch);
  for (int c = 0; c < batch; ++c) {
    const fd_sparse_hop& s = hop[c];
    if (s.q < 1 || s.q > 32)
      return fail(ctx, FD_ERR_INVALID, "config %d: q=%d outside [1,32]", c, s.q);
    if (s.nfac < 1 || s.nfac > FD_SPARSE_NFAC_MAX)
      return fail(ctx, FD_ERR_INVALID, "config %d: nfac=%d outside [1,%d]", c, s.nfac,
                  FD_SPARSE_NFAC_MAX);
    if (!s.col || !s.val) return fail(ctx, FD_ERR_INVALID, "config %d: null col or val", c);
    if (G && !G[c]) return fail(ctx, FD_ERR_INVALID, "config %d: null G", c);
    std::complex<double> g[FD_SPARSE_NFAC_MAX];
    if (taylor_factors(s.nfac, g) != FD_OK)
      return fail(ctx, FD_ERR_NUMERIC, "config %d: product-form factors for n=%d", c, s.nfac);
    fd::SparseHop& d = h[c];
    memset(&d, 0, sizeof(d));
    d.col = s.col;
    d.val = s.val;
    d.q = s.q;
    d.nfac = s.nfac;
    for (int k = 0; k < s.nfac; ++k) d.gamma[k] = make_double2(g[k].real(), g[k].imag());
  }
  cudaStream_t st = (cudaStream_t)stream;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  if ((size_t)batch > ctx->hop_cap) {
    if (ctx->d_hop) {
      FD_CUDA(ctx, cudaStreamSynchronize(st));
      cudaFree(ctx->d_hop);
    }
    ctx->d_hop = nullptr;
    const size_t cap = std::max<size_t>(batch, 64);
    FD_CUDA(ctx, cudaMalloc(&ctx->d_hop, cap * sizeof(fd::SparseHop)));
    ctx->hop_cap = cap;
  }
  // pageable source: the copy is staged before the call returns
  FD_CUDA(ctx, cudaMemcpyAsync(ctx->d_hop, h.data(), sizeof(fd::SparseHop) * batch,
                               cudaMemcpyHostToDevice, st));
  Outs o;
  o.logdet = logdet;
  o.G = G;
  return run(ctx, batch, probs, o, FD_PREC_FP64, stream, K_FWD, ctx->d_hop);
}

int fd_status(fd_ctx* ctx, void* stream, int* per_config_status, int batch) {
  if (!ctx) return FD_ERR_INVALID;
  if (batch < 0 || batch > ctx->last_batch)
    return fail(ctx, FD_ERR_INVALID, "batch %d exceeds last call's %d", batch, ctx->last_batch);
  if (batch > 0 && !per_config_status) return fail(ctx, FD_ERR_INVALID, "null status array");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  if (batch == 0) return FD_OK;
  std::vector<int> st(batch);
  FD_CUDA(ctx, cudaMemcpy(st.data(), ctx->last_status ? ctx->last_status : ctx->d_status,
                          sizeof(int) * batch, cudaMemcpyDeviceToHost));
  int worst = FD_OK;
  for (int c = 0; c < batch; ++c) {
    int code = st[c] == fd::ST_OK ? FD_OK
               : (st[c] == fd::ST_TIMEOUT || st[c] == fd::ST_PENDING) ? FD_ERR_TIMEOUT
                                                                      : FD_ERR_NUMERIC;
    per_config_status[c] = code;
    if (code < worst) worst = code;
  }
  return worst;
}

int fd_last_launch_count(const fd_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

int fd_graph_create(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet,
                    double* const* G, double* const* F, int prec, void** graph) {
  if (!graph) return fail(ctx, FD_ERR_INVALID, "null graph handle");
  *graph = nullptr;
  const bool force = F != nullptr;
  int rc = validate(ctx, batch, probs, logdet, prec, force);
  if (rc != FD_OK) return rc;
  if (batch < 1) return fail(ctx, FD_ERR_INVALID, "a graph needs batch >= 1");
  for (int c = 0; c < batch; ++c)
    if ((G && !G[c]) || (F && !F[c])) return fail(ctx, FD_ERR_INVALID, "config %d: null output", c);
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  const int kind = force ? K_FORCE : K_FWD;
  std::vector<Group> groups = plan(ctx, batch, probs, kind, prec);
  GraphObj* g = new GraphObj();
  g->batch = batch;
  std::vector<Desc> h(batch);
  size_t need = scratch_need(groups);
  const size_t ntasks = task_count(groups);
  std::vector<fd::Task> ht(std::max<size_t>(ntasks, 1));
  cudaStream_t cs = nullptr;
  int saved_launches = ctx->last_launches;
  auto bail = [&](int code) {
    if (cs) cudaStreamDestroy(cs);
    graph_free(g);
    ctx->last_launches = saved_launches;
    return code;
  };
#define FD_G(call)                                                do {                                                              cudaError_t e_ = (call);                                        if (e_ != cudaSuccess) return bail(cuda_fail(ctx, e_, #call));   } while (0)
  FD_G(cudaMalloc(&g->d_desc, sizeof(Desc) * batch));
  FD_G(cudaMalloc(&g->d_tasks, sizeof(fd::Task) * ht.size()));
  FD_G(cudaMalloc(&g->d_queue, sizeof(int) * std::max(1, queue_count(groups))));
  FD_G(cudaMalloc(&g->d_status, sizeof(int) * batch * (1 + fd::SF_NUM)));
  FD_G(cudaMalloc(&g->scratch, std::max<size_t>(need, 256)));
  Outs o;
  o.logdet = logdet;
  o.G = G;
  o.F = F;
  build_tables(groups, probs, o, g->scratch, g->d_status + batch, h.data(), ht.data());
  FD_G(cudaMemcpy(g->d_desc, h.data(), sizeof(Desc) * batch, cudaMemcpyHostToDevice));
  FD_G(cudaMemcpy(g->d_tasks, ht.data(), sizeof(fd::Task) * ht.size(), cudaMemcpyHostToDevice));
  FD_G(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  rc = ensure_side(ctx, std::min<size_t>(groups.size(), 8));
  if (rc != FD_OK) return bail(rc);
  FD_G(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  ctx->last_launches = 0;
  rc = enqueue(ctx, groups, g->d_desc, g->d_tasks, g->d_queue, g->d_status, g->scratch, batch, cs,
               false);
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(cs, &captured);
  g->graph = captured;
  if (rc != FD_OK) return bail(rc);
  if (ce != cudaSuccess) return bail(cuda_fail(ctx, ce, "cudaStreamEndCapture"));
  g->launches = ctx->last_launches;
  FD_G(cudaGraphInstantiate(&g->exec, g->graph, 0));
  cudaStreamDestroy(cs);
  cs = nullptr;
#undef FD_G
  ctx->last_launches = saved_launches;
  *graph = g;
  return FD_OK;
}

int fd_graph_launch(fd_ctx* ctx, void* graph, void* stream) {
  if (!ctx || !graph) return FD_ERR_INVALID;
  GraphObj* g = (GraphObj*)graph;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_CUDA(ctx, cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  ctx->last_batch = g->batch;
  ctx->last_launches = g->launches;
  ctx->last_status = g->d_status;
  return FD_OK;
}

int fd_graph_destroy(fd_ctx* ctx, void* graph) {
  if (!ctx) return FD_ERR_INVALID;
  if (!graph) return FD_OK;
  GraphObj* g = (GraphObj*)graph;
  if (ctx->last_status == g->d_status) ctx->last_status = nullptr;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_CUDA(ctx, cudaDeviceSynchronize());
  graph_free(g);
  return FD_OK;
}

// ---------------------------------------------------------------- autotuner
int fd_tune(fd_ctx* ctx, int batch, const fd_problem* probs, int what, int prec, int reps) {
  double dummy;
  const bool force = (what & FD_WANT_FORCE) != 0;
  int rc = validate(ctx, batch, probs, &dummy, prec, force);
  if (rc != FD_OK) return rc;
  if (batch == 0) return FD_OK;
  if (reps < 1) reps = 2;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  const int kind = force ? K_FORCE : K_FWD;
  // outputs for the trial runs
  size_t g_elems = 0, f_elems = 0;
  for (int c = 0; c < batch; ++c) {
    g_elems += (size_t)probs[c].nx * probs[c].nx;
    f_elems += (size_t)probs[c].nt * probs[c].nx;
  }
  double *d_ld = nullptr, *d_g = nullptr, *d_f = nullptr;
  FD_CUDA(ctx, cudaMalloc(&d_ld, sizeof(double) * 2 * batch));
  FD_CUDA(ctx, cudaMalloc(&d_g, sizeof(double) * 2 * g_elems));
  if (force) FD_CUDA(ctx, cudaMalloc(&d_f, sizeof(double) * 2 * f_elems));
  std::vector<double*> Gp(batch), Fp(batch);
  size_t og = 0, of = 0;
  for (int c = 0; c < batch; ++c) {
    Gp[c] = d_g + 2 * og;
    og += (size_t)probs[c].nx * probs[c].nx;
    Fp[c] = force ? d_f + 2 * of : nullptr;
    of += (size_t)probs[c].nt * probs[c].nx;
  }
  std::vector<Group> groups = plan(ctx, batch, probs, kind, prec);
  int result = FD_OK;
  for (auto& g : groups) {
    std::vector<fd_problem> sub;
    std::vector<double*> sg, sf;
    for (int c : g.idx) {
      sub.push_back(probs[c]);
      sg.push_back(Gp[c]);
      sf.push_back(Fp[c]);
    }
    const int three = prec == FD_PREC_MIXED_3XTF32 ? 1 : 0;
    // one launch at a time (coordinate search): each phase's threads per CTA is chosen on that
    // phase's own CUDA-event time, the other phases keeping their current choice
    for (size_t pi = 0; pi < g.ph.size() && result == FD_OK; ++pi) {
      const Phase& P = g.ph[pi];
      const long long key = tune_key(P.which, P.mixed, P.mixed ? three : 0, g.nx);
      float best = 1e30f;
      int best_t = 0;
      for (int nth : {128, 256}) {
        ctx->tuned[key] = nth;
        float tot = 0.f;
        for (int r = 0; r <= reps; ++r) {  // first run is a warm-up
          Outs o;
          o.logdet = d_ld;
          o.G = sg.data();
          o.F = force ? sf.data() : nullptr;
          const bool saved = ctx->timing;
          ctx->timing = true;
          int rr = run(ctx, (int)sub.size(), sub.data(), o, prec, nullptr, kind);
          ctx->timing = saved;
          if (rr != FD_OK) {
            result = rr;
            break;
          }
          cudaDeviceSynchronize();
          float ms = 0.f;
          if ((int)ctx->ev.size() > 2 * (int)pi + 1)
            cudaEventElapsedTime(&ms, ctx->ev[2 * pi], ctx->ev[2 * pi + 1]);
          if (r > 0) tot += ms;
        }
        if (result != FD_OK) break;
        if (tot < best) {
          best = tot;
          best_t = nth;
        }
      }
      if (result == FD_OK) ctx->tuned[key] = best_t;
    }
    if (result != FD_OK) break;
  }
  cudaDeviceSynchronize();
  cudaFree(d_ld);
  cudaFree(d_g);
  if (d_f) cudaFree(d_f);
  return result;
}

int fd_tune_nstab_stats(fd_ctx* ctx, const fd_problem* prob, const int* candidates, int ncand,
                        double rel_budget, int prec, int* best, double* err, double* ms) {
  if (!ctx || !prob || !candidates || ncand < 1 || !best) return FD_ERR_INVALID;
  *best = 0;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  int nmin = 1 << 30;
  for (int i = 0; i < ncand; ++i) {
    if (candidates[i] < 1 || prob->nt % candidates[i] != 0)
      return fail(ctx, FD_ERR_INVALID, "candidate n_stab=%d does not divide nt=%d",
                  candidates[i], prob->nt);
    nmin = std::min(nmin, candidates[i]);
  }
  const int n = prob->nx;
  const size_t gn = (size_t)n * n;
  double* d_ld = nullptr;
  double* d_g = nullptr;
  FD_CUDA(ctx, cudaMalloc(&d_ld, sizeof(double) * 2));
  FD_CUDA(ctx, cudaMalloc(&d_g, sizeof(double) * 2 * gn));
  std::vector<double> gref(2 * gn), got(2 * gn);
  double* gp[1] = {d_g};
  Outs o;
  o.logdet = d_ld;
  o.G = gp;
  // reference: FP64 with the smallest candidate interval
  fd_problem p = *prob;
  p.n_stab = nmin;
  int rc = run(ctx, 1, &p, o, FD_PREC_FP64, nullptr, K_FWD);
  double ref[2] = {0, 0};
  if (rc == FD_OK) {
    cudaDeviceSynchronize();
    cudaMemcpy(ref, d_ld, sizeof(ref), cudaMemcpyDeviceToHost);
    cudaMemcpy(gref.data(), d_g, sizeof(double) * 2 * gn, cudaMemcpyDeviceToHost);
  }
  double gmax = 1.0;
  for (size_t e = 0; e < gn; ++e) gmax = std::max(gmax, hypot(gref[2 * e], gref[2 * e + 1]));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int chosen = 0;
  float best_ms = 0.f;
  for (int i = 0; i < ncand && rc == FD_OK; ++i) {
    p.n_stab = candidates[i];
    rc = run(ctx, 1, &p, o, prec, nullptr, K_FWD);  // warm-up (plans and sizes the workspace)
    if (rc != FD_OK) break;
    cudaEventRecord(e0, 0);
    rc = run(ctx, 1, &p, o, prec, nullptr, K_FWD);
    cudaEventRecord(e1, 0);
    if (rc != FD_OK) break;
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    double g2[2];
    cudaMemcpy(g2, d_ld, sizeof(g2), cudaMemcpyDeviceToHost);
    cudaMemcpy(got.data(), d_g, sizeof(double) * 2 * gn, cudaMemcpyDeviceToHost);
    const double dre = fabs(g2[0] - ref[0]);
    const double dim = fabs(remainder(g2[1] - ref[1], 2.0 * 3.14159265358979323846));
    double e_ld = std::max(dre, dim) / std::max(1.0, hypot(ref[0], ref[1]));
    double e_g = 0.0;
    for (size_t e = 0; e < gn; ++e)
      e_g = std::max(e_g, hypot(got[2 * e] - gref[2 * e], got[2 * e + 1] - gref[2 * e + 1]));
    e_g /= gmax * gmax;
    const double e_all = std::max(e_ld, e_g);
    if (err) err[i] = e_all;
    if (ms) ms[i] = t;
    if (e_all <= rel_budget &&
        (chosen == 0 || t < best_ms || (t == best_ms && candidates[i] > chosen))) {
      chosen = candidates[i];
      best_ms = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_ld);
  cudaFree(d_g);
  if (rc != FD_OK) return rc;
  *best = chosen;
  return FD_OK;
}

int fd_tune_nstab(fd_ctx* ctx, const fd_problem* prob, const int* candidates, int ncand,
                  double rel_budget, int prec, int* best) {
  return fd_tune_nstab_stats(ctx, prob, candidates, ncand, rel_budget, prec, best, nullptr,
                             nullptr);
}

int fd_tune_save(fd_ctx* ctx, const char* path) {
  if (!ctx || !path) return FD_ERR_INVALID;
  FILE* f = fopen(path, "w");
  if (!f) return fail(ctx, FD_ERR_INVALID, "cannot write %s", path);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, ctx->device);
  fprintf(f, "[\n");
  size_t i = 0;
  for (auto& kv : ctx->tuned) {
    long long k = kv.first;
    fprintf(f, "  {\"gpu\": \"%s\", \"kind\": %lld, \"mixed\": %lld, \"three\": %lld, "
               "\"nx\": %lld, \"threads\": %d}%s\n",
            prop.name, (k >> 40) & 0xff, (k >> 36) & 0xf, (k >> 32) & 0xf, k & 0xffffffffLL,
            kv.second, ++i < ctx->tuned.size() ? "," : "");
  }
  fprintf(f, "]\n");
  fclose(f);
  return FD_OK;
}

int fd_tune_load(fd_ctx* ctx, const char* path) {
  if (!ctx || !path) return FD_ERR_INVALID;
  FILE* f = fopen(path, "r");
  if (!f) return fail(ctx, FD_ERR_INVALID, "cannot read %s", path);
  char line[512];
  int loaded = 0;
  while (fgets(line, sizeof(line), f)) {
    long long kind, mixed, three, nx;
    int threads;
    const char* q = strstr(line, "\"kind\"");
    if (!q) continue;
    if (sscanf(q, "\"kind\": %lld, \"mixed\": %lld, \"three\": %lld, \"nx\": %lld, "
                  "\"threads\": %d", &kind, &mixed, &three, &nx, &threads) == 5 &&
        (threads == 128 || threads == 256)) {
      ctx->tuned[tune_key((int)kind, (int)mixed, (int)three, (int)nx)] = threads;
      ++loaded;
    }
  }
  fclose(f);
  return loaded;
}

int fd_plan_query(fd_ctx* ctx, int batch, const fd_problem* probs, int what, int prec, int* info,
                  int max_groups) {
  double dummy;
  int rc = validate(ctx, batch, probs, &dummy, prec, kind_of(what) != K_FWD);
  if (rc != FD_OK) return rc;
  if (max_groups > 0 && !info) return fail(ctx, FD_ERR_INVALID, "null info");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  const int kind = kind_of(what);
  std::vector<Group> groups = plan(ctx, batch, probs, kind, prec);
  int k = 0, total = 0;
  for (auto& g : groups) {
    for (auto& P : g.ph) {
      ++total;
      if (k >= max_groups) continue;
      int* o = info + 8 * k++;
      o[0] = g.nx;
      o[1] = P.which + (P.mixed ? 4 : 0) + (P.big ? 16 : 0);
      o[2] = P.nthreads;
      o[3] = P.smem;
      o[4] = P.grid;
      o[5] = P.occ;
      o[6] = (int)(P.slot_bytes >> 10);
      o[7] = P.ntasks;
    }
  }
  return total;
}

int fd_set_timing(fd_ctx* ctx, int on) {
  if (!ctx) return FD_ERR_INVALID;
  ctx->timing = on != 0;
  ctx->ev_used = 0;
  return FD_OK;
}

int fd_last_kernel_ms(fd_ctx* ctx, double* ms, int max) {
  if (!ctx || (max > 0 && !ms)) return FD_ERR_INVALID;
  if (!ctx->timing) return fail(ctx, FD_ERR_INVALID, "timing is off (fd_set_timing)");
  int n = std::min(max, ctx->ev_used / 2);
  for (int i = 0; i < n; ++i) {
    FD_CUDA(ctx, cudaEventSynchronize(ctx->ev[2 * i + 1]));
    float t = 0.f;
    FD_CUDA(ctx, cudaEventElapsedTime(&t, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
    ms[i] = t;
  }
  return n;
}

int fd_measure_fp64_issue(fd_ctx* ctx, double* cycles) {
  if (!ctx || !cycles) return FD_ERR_INVALID;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_CUDA(ctx, fd::run_fp64_issue(cycles));
  return FD_OK;
}

int fd_check_fp64_refinements(const double* x, const double* y, const double* z, int n,
                              double* out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y || !z || !out))) return FD_ERR_INVALID;
  return fd::run_refine_check(x, y, z, n, out, (cudaStream_t)stream) == cudaSuccess
             ? FD_OK
             : FD_ERR_CUDA;
}

int fd_measure_fp64_peak(fd_ctx* ctx, double* gflops) {
  if (!ctx || !gflops) return FD_ERR_INVALID;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_CUDA(ctx, fd::run_fp64_probe(ctx->num_sms * 8, 256, 4096, gflops, 0));
  return FD_OK;
}

}  // extern "C"
