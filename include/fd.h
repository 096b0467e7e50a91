/*
 * fd.h -- C ABI of the batched, stabilised fermion-determinant library for NVIDIA GB300 (sm_103a).
 *
 * What it computes (arXiv 2604.02130, "Stable and Efficient Algorithms for the Fermion
 * Determinant"):
 *   time slices   B_t = E diag(exp(i phi_t)),   E = exp(delta*kappa*A)          (Section 2)
 *   product       P = B_Nt ... B_2 B_1  (slice 1 acts first; the order of the block fermion
 *                 matrix of Section 2, whose top-right block is +M_{Nt-1})
 *   log det       logdet = log det(1 + P)                        (Section 2, Eq. hamiltonian_alg)
 *   Green's fn    G = (1 + P)^{-1}                                (Section 2, "sausage" inverse)
 *   HMC force     F[t,x] = d logdet / d phi[t,x] = i (1 - [G_{t-1}]_{xx}),
 *                 G_{t-1} = (1 + B_{t-1}...B_1 B_Nt...B_t)^{-1}  (Section 4, Eq. response_result)
 * by the stabilised dense method of Section 7 (X D T representation, QR re-orthogonalisation
 * every n_stab slices as proposed in Section 9, scale-separated assembly).
 *
 * Conventions shared by every entry point:
 *   - All matrix/vector arguments inside fd_problem and all outputs are DEVICE pointers on the
 *     context's device, owned by the caller, and must stay valid until the stream reaches the
 *     end of the call.  Arrays of problems / of output pointers are HOST arrays, read during the
 *     call only.
 *   - Real matrices are float64 row-major (E and E^{-1} are symmetric, so row- and column-major
 *     coincide).  Complex outputs are complex128 interleaved (re, im), row-major.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 *     stream).  The return code covers host-side validation and launch errors only.  Device-side
 *     failures (non-finite values, zero pivots, a bounded wait that ran out) are recorded per
 *     configuration and read back with fd_status().
 *   - The library owns its workspace (checkpoints, per-configuration scratch, descriptor tables)
 *     inside the context.  A call may grow it with cudaMalloc, which synchronises the device;
 *     fd_reserve() sizes it ahead of time (required before stream capture).
 *   - Every function returns FD_OK (0) or a negative FD_ERR_* code; fd_last_error() gives text.
 *   - A context is not thread-safe; use one per host thread.  Its device tables (descriptors,
 *     queues, status words, scratch, the BSS and sparse-hopping tables) are reused by every call,
 *     so calls on one context issued to different streams must be ordered with events (or issued
 *     to one stream); CUDA graphs (fd_graph_create) own separate tables.
 */
#ifndef FD_H_
#define FD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest spatial size handled (honeycomb L = 12 gives Nx = 288). */
#define FD_NX_MAX 288

enum {
  FD_OK = 0,
  FD_ERR_INVALID = -1,     /* bad argument: null pointer, size out of range, nt % n_stab != 0 */
  FD_ERR_UNSUPPORTED = -2, /* valid request that this library does not implement */
  FD_ERR_CUDA = -3,        /* a CUDA runtime call failed (text in fd_last_error) */
  FD_ERR_NUMERIC = -4,     /* device: non-finite value or zero pivot in a configuration */
  FD_ERR_TIMEOUT = -5,     /* device: a bounded wait gave up (kernel returned early) */
  FD_ERR_TOO_LARGE = -6    /* request exceeds a fixed capacity (fd_logdet_noalloc limits) */
};

/* Arithmetic of the slice products.  QR re-orthogonalisation, scale separation, assembly,
 * boundary Green's functions and all outputs are FP64 in every mode (in the mixed modes, the
 * size classes whose tensor-core operands do not fit in shared memory -- nx 98..288 in split
 * TF32 -- stream their operands from global memory and run the O(nx^3) parts of the QR and of
 * the force's boundary Green's functions in double-float arithmetic, hi + lo FP32 pairs with
 * about 46 significant bits, keeping FP64 scalars, inputs and outputs; see fd_plan_query). */
enum {
  FD_PREC_FP64 = 0,        /* everything in FP64 (DFMA) */
  FD_PREC_MIXED_TF32 = 1,  /* slice GEMMs on tcgen05 tensor cores, TF32 operands, FP32 accumulate */
  FD_PREC_MIXED_3XTF32 = 2 /* as above with split (hi + lo) TF32 operands, 3 MMAs per product */
};

typedef struct fd_ctx fd_ctx;

/* One configuration.  All pointers are device pointers.
 *   nx        spatial sites, 1 <= nx <= FD_NX_MAX
 *   nt        time slices, nt >= 1
 *   n_stab    slices between QR re-orthogonalisations, 1 <= n_stab <= nt, nt % n_stab == 0
 *   expA      E = exp(delta*kappa*A), nx*nx float64 (symmetric)
 *   expA_inv  E^{-1}, nx*nx float64 (symmetric); needed for F, G(tau, 0) and R, may be
 *             NULL otherwise
 *   phi       nt*nx float64 row-major; row t-1 is the field of slice t */
typedef struct {
  int32_t nx;
  int32_t nt;
  int32_t n_stab;
  int32_t reserved; /* must be 0 */
  const double* expA;
  const double* expA_inv;
  const double* phi;
} fd_problem;

/* Create a context on CUDA device `device` (makes it current on the calling thread). */
int fd_ctx_create(fd_ctx** out, int device);
void fd_ctx_destroy(fd_ctx* ctx);
const char* fd_last_error(const fd_ctx* ctx);

/* Pre-size the workspace for up to `batch` configurations like `probs` with the given outputs
 * (`what` = bitmask of FD_WANT_*), so that later calls of that shape allocate nothing. */
enum {
  FD_WANT_LOGDET = 1,
  FD_WANT_GREEN = 2,
  FD_WANT_FORCE = 4,
  FD_WANT_GTAU = 8,
  FD_WANT_RESPONSE = 16
};
int fd_reserve(fd_ctx* ctx, int batch, const fd_problem* probs, int what, int prec);

/* log det(1 + B_Nt...B_1) for `batch` configurations.
 *   logdet  device, 2*batch float64: (re, im) per configuration; im wrapped to (-pi, pi].
 * A size class with fewer configurations than SMs runs time-parallel: each chain is cut into
 * segments computed concurrently and merged by the stabilised product of two UDV factors
 * (Section 7); a segment's log D must then span less than 700 (else FD_ERR_NUMERIC in fd_status),
 * which holds for beta per segment up to ~100 at kappa = 1 on the honeycomb lattice.  The same
 * holds for fd_green and fd_observables without F and R. */
int fd_logdet(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet, int prec,
              void* stream);

/* log det and the Green's function G = (1 + B_Nt...B_1)^{-1}.
 *   G  host array of `batch` device pointers; G[c] receives nx*nx complex128, row-major. */
int fd_green(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet, double* const* G,
             int prec, void* stream);

/* log det, (optionally) G, and the force F[t,x] = d logdet / d phi[t,x] (complex; for real
 * fields Im F = 1/2 exactly on a bipartite lattice).  Forward pass with checkpoints of
 * (X, D, T) every n_stab slices, then an adjoint backward sweep that recomputes the right
 * products, forms the equal-time Green's function stably at each block boundary and wraps it
 * through the block (Section 4, Eq. response_result; Section 7 steps 7-9 with t1 = t2).  The
 * forward and backward chains run as independent tasks; the boundary and wrap launches start
 * while the chains run (programmatic dependent launch) and each of their tasks waits only for
 * its own checkpoints; a task that sees no progress of its inputs for ~4 s gives up with
 * FD_ERR_TIMEOUT in fd_status.  Workspace per configuration:
 * (2 (nb-1) (2 nx^2 + ceil(nx/2)) + nb nx^2) * 16 bytes, nb = nt / n_stab.
 *   G  host array of device pointers or NULL (G not wanted)
 *   F  host array of `batch` device pointers; F[c] receives nt*nx complex128, row-major
 *      (row t-1 is slice t, like phi). */
int fd_force(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet, double* const* G,
             double* const* F, int prec, void* stream);

/* log det, (optionally) G and F, and the unequal-time Green's function
 * G(tau, 0) = (M^{-1})_{tau,0} = B_tau...B_1 (1 + B_Nt...B_1)^{-1}, tau = 0..nt-1 (Section 4.2,
 * Eq. sausage_all_in_denominator with t0 = 0).  At the block boundaries tau = (b-1) n_stab it is
 * formed stably from the left and right (X, D, T) checkpoints (Section 7 steps 7-9:
 * G(tau, 0) = X_R D_Rb^{-1} M^{-1} D_Ls T_L, M the boundary matrix of G_tau); inside a block it
 * is propagated one slice at a time, forward G(t+1, 0) = B_{t+1} G(t, 0) from the lower boundary
 * for (n_stab-1)/2 slices and backward G(t-1, 0) = B_t^{-1} G(t, 0) from the upper one
 * (G(nt, 0) = 1 - G for the last block), so no propagation runs over more than n_stab/2 slices.
 *   Gtau  host array of `batch` device pointers; Gtau[c] receives nt*nx*nx complex128, block
 *         tau row-major at offset tau*nx*nx (Gtau[c] block 0 = G)
 *   G, F  host arrays of device pointers, or NULL (not wanted); as for fd_force
 * With a mixed precision the chains run on the tensor cores and the G(tau, 0) wraps in FP64.
 * Not available through fd_graph_create. */
int fd_green_tau(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet,
                 double* const* G, double* const* Gtau, double* const* F, int prec, void* stream);

/* Local (BSS) updates of the auxiliary field at one time slice t (Section 3, the BSS algorithm).
 * One entry per configuration; all pointers are device pointers owned by the caller:
 *   nx        sites (1 <= nx <= FD_NX_MAX); reserved must be 0
 *   G         nx*nx complex128 row-major, in/out: on entry G_{t-1} = (1 + B_{t-1}...B_1
 *             B_Nt...B_t)^{-1} of the current field (slice t acting first; for t = 1 this is the
 *             G of fd_green), on return the same Green's function of the updated field
 *   phi_row   nx float64, in/out: the field of slice t (row t-1 of phi)
 *   dphi      nx float64: the proposals phi_x -> phi_x + dphi_x, visited for x = 0..nx-1 in order
 *   u, w      nx float64: uniform random numbers and the ratio of every other weight factor; the
 *             proposal at x is accepted iff u_x < |r_x| w_x with r_x = det(1+P')/det(1+P)
 *   accepted  nx int32 out: 1 where accepted
 * The ratio comes from the matrix determinant lemma, r_x = 1 + (e^{i dphi_x} - 1)(1 - G_xx), and
 * an accepted proposal updates G by Sherman-Morrison (O(nx^2); a rejected one costs O(1)).
 * dlogdet: device, 2*batch float64: sum of log r_x over the accepted sites (re, im wrapped to
 * (-pi, pi]), i.e. the change of log det.  A launch whose largest nx is <= 110 holds G in
 * shared memory as pairs of FP32 values (about 46 significant bits, relative error ~1e-14 per
 * update) and takes the ratios and decisions in the same pair arithmetic (FP64 where |r|^2 or
 * (u/w)^2 leaves [2^-100, 2^100]), converting G back to FP64 on return; larger nx, or a G with an
 * entry of magnitude >= 2^100, runs every step in FP64 with G updated in place.  dlogdet is
 * summed in FP64.  Asynchronous on `stream`; not available through fd_graph_create.  Wrapping G to the
 * next slice and re-stabilising it every n_stab slices (fd_green / fd_force) are the caller's
 * part of a sweep. */
typedef struct {
  int32_t nx;
  int32_t reserved; /* must be 0 */
  double* G;
  double* phi_row;
  const double* dphi;
  const double* u;
  const double* w;
  int32_t* accepted;
} fd_bss_slice;
int fd_bss_update(fd_ctx* ctx, int batch, const fd_bss_slice* slices, double* dlogdet,
                  void* stream);

/* Intermediate-volume variant (Sections 8-9): log det and optionally G with every slice's
 * hopping factor replaced by the degree-n Taylor polynomial of exp written as a product of
 * linear factors, B_t = prod_{k=1}^{n} (1 + gamma_k K) diag(e^{i phi_t}), applied matrix-free
 * with the sparse K -- O(n q nx) per column and slice instead of the dense O(nx^2) -- with the QR
 * re-orthogonalisation every n_stab slices (the sporadic stabilisation of Section 9) and the
 * assembly of fd_green.  The factors satisfy prod_k (1 + gamma_k x) = sum_{j<=n} x^j / j!
 * (fd_taylor_factors), so the result equals fd_green's with E = sum_{j<=n} K^j / j! and differs
 * from the one with E = exp(K) by O(nt delta^{n+1}) = O(beta delta^n).
 *   probs  as for fd_green; expA and expA_inv are not read (may be NULL)
 *   hop    host array of `batch` entries:
 *            q     entries per row of K, 1 <= q <= 32 (pad short rows with val = 0)
 *            nfac  n, 1 <= n <= 8 (the paper suggests 4)
 *            col   device, nx*q int32: the columns of row i's entries at [i*q, i*q + q)
 *            val   device, nx*q float64: their values K_{i,col} (delta*kappa on the honeycomb
 *                  lattice)
 *   G      host array of device pointers, or NULL for log det only
 * FP64 (DFMA) throughout, one persistent kernel, no time-parallel split; the caller's tables
 * must stay valid until the call has run.  Not available through fd_graph_create. */
typedef struct {
  int32_t q;
  int32_t nfac;
  const int32_t* col;
  const double* val;
} fd_sparse_hop;
int fd_green_sparse(fd_ctx* ctx, int batch, const fd_problem* probs, const fd_sparse_hop* hop,
                    double* logdet, double* const* G, void* stream);

/* The product-form factors of fd_green_sparse for n = 1..8: gamma[2k], gamma[2k+1] = (re, im) of
 * gamma_k, k = 0..n-1, sorted by (re, im) -- gamma_k = -1/x_k over the roots x_k of
 * sum_{j<=n} x^j / j! (Weierstrass / Durand-Kerner iteration, then checked by multiplying the
 * factors out).  Host only; returns FD_ERR_INVALID for n outside [1, 8]. */
int fd_taylor_factors(int n, double* gamma);

/* Failure-detection test hook.  With `on`, the phased calls (fd_force, fd_green_tau, and
 * fd_observables with F or R) skip their chain launch, so the boundary and wrap tasks wait for
 * checkpoints that never come: each bounded wait gives up after ~4 s without progress, the
 * kernels return, and every configuration reports FD_ERR_TIMEOUT in fd_status (outputs are then
 * undefined).  The context stays usable; switch the hook off for normal calls. */
int fd_debug_skip_chains(fd_ctx* ctx, int on);

/* Time-parallel force chains.  A force call (fd_force, or fd_observables with F only) runs two
 * chains per configuration, the forward one (left checkpoints, then log det and G_0) and the
 * backward one (right checkpoints), so a long chain is serial work on one SM.  Two decompositions
 * (Section 7's stabilised product of two factored matrices joins the pieces):
 *  - halves (the FP64 path, and the mixed path's shared-memory classes when forced): each chain
 *    runs as two halves in parallel, the second from the identity; the boundary phase merges a
 *    second half's checkpoint with the first half's last one (FP64) and forms log det and G_0
 *    from the forward halves.  A merge whose left factor spans more than e^700 marks the
 *    configuration FD_ERR_NUMERIC.
 *  - segments (the mixed path): S segments of about 8 blocks (4..8 segments, a power of two
 *    dividing the block count) run from the identity in parallel, their prefixes are formed in
 *    order by merges (double-float in the streamed classes, Nx above the shared-memory tile;
 *    FP64 in the others), and the segments are re-run from their exact prefixes, so every
 *    checkpoint is final.  In the streamed classes a segment whose log D spans more than e^76
 *    (beyond the double-float exponent range once squared) marks the configuration
 *    FD_ERR_NUMERIC.
 * mode -1 (default): halves in FP64 when 4 * batch <= the SM count; segments in the mixed path for
 * a configuration whose chain would outlast 1.5 times an SM's share of all the call's chains
 * (cost nx^3 (nt + 150 nt / n_stab)).  0: never.  1: segments of at least 4 blocks (S >= 4) in
 * the mixed path where the configuration has them, else halves (not in the streamed classes)
 * for every configuration with at least 4 blocks.  Results agree with the whole chains to
 * rounding.  Returns FD_ERR_INVALID for another mode. */
int fd_set_force_split(fd_ctx* ctx, int mode);

/* Wait for `stream` and copy the per-configuration device status of the LAST call on this
 * context into per_config_status[0..batch-1] (host): FD_OK, FD_ERR_NUMERIC or FD_ERR_TIMEOUT.
 * Returns the worst code seen (FD_OK if all succeeded). */
int fd_status(fd_ctx* ctx, void* stream, int* per_config_status, int batch);

/* Single-time observables (Section 4.1), with log det and optionally G and F in the same call:
 *   nferm  device, 2*batch float64 or NULL: the fermion number n = 1 - tr G / nx (re, im),
 *          Eq. fermion_number (the response to the chemical potential)
 *   O, R   both NULL, or host arrays of `batch` device pointers: O[c] an nx*nx float64 operator
 *          (row-major, read only), R[c] receives nt complex128, the response traces
 *          R[c][r] = tr(O G_r), G_r = (1 + B_r...B_1 B_Nt...B_{r+1})^{-1}, r = 0..nt-1 (G_0 = G;
 *          the thermal trace of the operator with the Green's function at every time slice).
 *          With O = A (the hopping matrix), -delta sum_r R[r] = d logdet / d kappa exactly.
 *   G, F   as for fd_force, each optional.
 * nferm alone (or with G) runs the single log det/G kernel; F or R run the phased force path
 * (chains, boundary Green's functions, wraps), so expA_inv is then required.  In the mixed
 * precisions the traces of the wrapped G_r accumulate in FP32 in the tensor-core epilogue.
 * Not available through fd_graph_create. */
int fd_observables(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet,
                   double* const* G, double* const* F, double* nferm, const double* const* O,
                   double* const* R, int prec, void* stream);

/* Number of kernel launches the last fd_logdet/fd_green/fd_force/fd_green_tau/fd_observables
 * call issued. */
int fd_last_launch_count(const fd_ctx* ctx);

/* Autotuner.  fd_tune times every launch (phase) of every size class of this batch with 128 and
 * 256 threads per CTA, one launch at a time on its own CUDA-event time (`reps` timed runs each
 * after a warm-up, FP64 or mixed as `prec` says), and keeps the faster choice per launch in the
 * context's plan cache, which later plans (calls, graphs, fd_plan_query) use.
 * Synchronous; allocates and frees its own trial outputs.
 * fd_tune_nstab picks, for one configuration, the QR interval among `candidates` (each must
 * divide nt) whose log det + G call at precision `prec` is fastest (CUDA-event time of the call
 * after a warm-up; ties to the larger interval) among those whose error stays within
 * `rel_budget` of an FP64 run with the smallest candidate -- the error being the larger of the
 * log det error (|d Re|, |d Im mod 2pi| over max(1, |logdet|)) and the G error (max |dG_ij| over
 * max(1, max|G|)^2); *best = 0 if none does.  Section 9's proposal of stabilising every
 * beta_0/delta slices with beta_0 ~ 10 is the regime this explores: fewer QRs cost accuracy in
 * the mixed path (its block products lose the small singular directions in proportion to the
 * block's condition number).  fd_tune_nstab_stats also writes each candidate's error and time
 * (err, ms: ncand doubles each, host, may be NULL).  Synchronous; allocates its trial outputs.
 * fd_tune_save / fd_tune_load write / read the plan cache as a JSON list (one object per size
 * class: gpu, kind, mixed, three, nx, threads); load returns the number of entries read. */
int fd_tune(fd_ctx* ctx, int batch, const fd_problem* probs, int what, int prec, int reps);
int fd_tune_nstab(fd_ctx* ctx, const fd_problem* prob, const int* candidates, int ncand,
                  double rel_budget, int prec, int* best);
int fd_tune_nstab_stats(fd_ctx* ctx, const fd_problem* prob, const int* candidates, int ncand,
                        double rel_budget, int prec, int* best, double* err, double* ms);
int fd_tune_save(fd_ctx* ctx, const char* path);
int fd_tune_load(fd_ctx* ctx, const char* path);

/* CUDA-graph batching.  fd_graph_create plans the call fd_force (F != NULL) or fd_green /
 * fd_logdet (F == NULL; G may be NULL) would make for this batch, gives it its own descriptor
 * table, queues, status words and scratch, and captures it -- the queue/status resets and one
 * persistent kernel per size class, the classes as parallel branches -- into an executable
 * graph.  fd_graph_launch replays it on `stream`: one cudaGraphLaunch, no host work.  Every
 * replay reads the inputs and writes the outputs through the pointers given at creation, so
 * callers update phi (and E) in place between replays.  fd_status after a replay reports that
 * replay.  fd_graph_destroy synchronises the device and frees the graph's memory.
 * The graph owns its memory; it stays valid across other calls on the context. */
int fd_graph_create(fd_ctx* ctx, int batch, const fd_problem* probs, double* logdet,
                    double* const* G, double* const* F, int prec, void** graph);
int fd_graph_launch(fd_ctx* ctx, void* graph, void* stream);
int fd_graph_destroy(fd_ctx* ctx, void* graph);

/* The launch plan a call with these arguments would use, without launching anything: one
 * record of 8 ints per kernel launch in info[8*g .. 8*g+7]:
 *   nx, kernel (+4 when it runs on the tensor cores, +16 for the kernels that stream their
 *   operands from global memory and use double-float QRs and boundary Green's functions):
 *   0 log det/G, 1 chains (force: forward and backward products, two tasks per configuration;
 *   time-parallel log det/G: segment products; streamed log det/G: one forward chain per
 *   configuration), 2 block-boundary Green's functions, 3 wraps and force rows, 8 merge of the
 *   segment products and assembly (FP64);  threads per CTA, dynamic shared memory bytes, grid (persistent CTAs),
 *   resident CTAs per SM, scratch KiB per CTA, tasks of the launch.
 * Returns the number of launches (>= 0, records beyond max_groups are not written) or a
 * negative FD_ERR_* code.  Synchronous, host only (queries the device's occupancy limits). */
int fd_plan_query(fd_ctx* ctx, int batch, const fd_problem* probs, int what, int prec, int* info,
                  int max_groups);

/* Per-launch timing.  With timing on, every kernel launch of a call is bracketed by CUDA events
 * recorded on the call's stream, and the launches run one after another (size classes are not
 * forked onto side streams and later phases do not start early), so each duration is that
 * kernel's alone.  fd_last_kernel_ms waits for them and writes the durations (ms) of the last
 * call's launches, in launch order, to ms[0..max-1]; it returns how many it wrote (>= 0) or a
 * negative FD_ERR_* code. */
int fd_set_timing(fd_ctx* ctx, int on);
int fd_last_kernel_ms(fd_ctx* ctx, double* ms, int max);

/* Measured FP64 FMA throughput of this device in GFLOP/s (a DFMA-bound loop over all SMs);
 * used to state roofline fractions.  Synchronous. */
int fd_measure_fp64_peak(fd_ctx* ctx, double* gflops);

/* Issue cost of FP64 instructions on this device (clock cycles per dependent DFMA), which decides
 * how the latency-bound QR and LU steps are laid out: cycles[0] one warp with 1 active lane,
 * cycles[1] one warp with 32 active lanes, cycles[2] seen by one of 8 warps of a CTA that all
 * issue independent DFMAs (the SM's shared FP64 pipe).  Synchronous. */
int fd_measure_fp64_issue(fd_ctx* ctx, double* cycles);

/* Self-check of the hand-written FP64 refinements that the serial QR and LU steps use in place
 * of IEEE division and square root (an FP32 hardware estimate refined by Newton or by
 * Householder's third-order iteration; Section 7's QR re-orthogonalisation is where they run).
 * For each argument i (x, y, z: device, n float64 each) writes 16 float64 to out[16 i ..]
 * (device): 0 rcp64(x), 1 CUDA's correctly rounded 1/x, 2 rsqrt64(x), 3 CUDA's 1/sqrt(x) as
 * two correctly rounded operations, 4 sqrt64(x), 5 CUDA's correctly rounded sqrt(x); then the
 * Householder reflector of a column with leading entry x + i y and squared norm z below it:
 * 6, 7 alpha = -(x/|x|) sqrt(|x|^2 + z), 8, 9 1/c = conj(x) / (|x| (|x| + sqrt(|x|^2 + z))),
 * 10 tau = 1 + |x| / sqrt(|x|^2 + z), 11 1 if the column is zero; 12..15 zero.  Runs on the
 * current device, asynchronously on `stream`.  Returns FD_OK, FD_ERR_INVALID or FD_ERR_CUDA. */
int fd_check_fp64_refinements(const double* x, const double* y, const double* z, int n,
                              double* out, void* stream);

/* ---------------------------------------------------------------------------------------
 * fd_logdet_noalloc: log det (and optionally G) without any memory allocation.
 * The paper has no counterpart; this entry point exists for callers that cannot allocate
 * device memory -- e.g. a host framework that owns every device allocation through its own
 * pool, a real-time loop whose memory budget is fixed at start-up, or a pipeline step that must
 * not suffer the implicit device-wide synchronisation of cudaMalloc/cudaFree.  It needs no
 * fd_ctx and never calls cudaMalloc, cudaFree or any allocating library routine.
 *
 * Working memory: one file-scope device array of 12 MiB inside libfd.so, held on every GPU that
 * loads the library until the process exits and shared by every call on that GPU.  Nothing in
 * it has to start at zero (each call writes every scratch entry before reading it), but it keeps
 * the last call's contents, so calls whose kernels overlap on the GPU race with each other:
 * issue them on one stream, or order them with events.
 *
 * Limits: batch <= FD_NOALLOC_MAX_BATCH, nx <= FD_NOALLOC_MAX_NX; larger requests return
 * FD_ERR_TOO_LARGE and launch nothing.  FP64 arithmetic only (the FD_PREC_FP64 path).
 * The first call on a device performs a one-time set-up on the current device (it looks up
 * the device address of the array and sets the kernel's shared-memory limit); make that first
 * call before any stream capture.  With CUDA's default lazy module loading, that first call is
 * also when the device loads this library's code and with it reserves the 12 MiB array, so a
 * caller whose memory pool later takes the whole device should make the first call at start-up,
 * before the pool does (a failed reservation returns FD_ERR_CUDA).  The looked-up address is
 * kept for the life of the process: resetting the device (cudaDeviceReset) after the first call
 * is not supported.
 *   probs   host array of `batch` problems (device pointers inside, as for fd_logdet)
 *   logdet  device, 2*batch float64 (re, im); G: NULL or host array of device pointers
 *           (nx*nx complex128, row-major); status: NULL or device int[batch] receiving 0 (ok)
 *           or 1 (non-finite value / zero pivot) per configuration.
 * Runs on the current device, asynchronously on `stream`.  Returns FD_OK, FD_ERR_INVALID,
 * FD_ERR_TOO_LARGE, FD_ERR_UNSUPPORTED (device index >= 64) or FD_ERR_CUDA. */
#define FD_NOALLOC_MAX_BATCH 64
#define FD_NOALLOC_MAX_NX 72
int fd_logdet_noalloc(int batch, const fd_problem* probs, double* logdet, double* const* G,
                      int* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FD_H_ */
