/*
 * mg.h — C ABI of the GB300 messenger Gibbs sampler.
 *
 * The library samples the joint posterior Pi(s, P(k) | d) of a Gaussian signal
 * s on a periodic 3D grid and its isotropic power spectrum P(k), for linear
 * data d = R s + eps with diagonal response R and diagonal noise covariance N
 * (Jasche & Lavaux 2014, "Matrix-free large scale Bayesian inference in
 * cosmology", Sec. 2).  One sweep is:
 *   t | s, d       messenger draw voxel by voxel (Sec. 3.1, Alg. 1 first loop)
 *   t_hat          forward orthonormal transform (Alg. 1, "ONT")
 *   s_hat | t_hat  signal draw mode by mode (Sec. 3.1, Alg. 1 second loop)
 *   s              inverse transform (Alg. 1)
 *   P | s          inverse-gamma draw per k-shell (Sec. 3.2, Alg. 2 on shells)
 * with T = tau 1, tau = tau_scale * min over observed voxels of N_i / R_i^2 and
 * N~ = N - R T R (Sec. 2).  All random draws are Philox4x32-10 keyed by the
 * seed with counter (index, sweep, chain, stream); see mg_philox().
 *
 * Conventions shared by every call:
 *   - Grids are cubic: nx = ny = nz = n with n in {8, 12, 16, 24, 32, 48, 64,
 *     96, 128, 192, 256} and equal box sides L[0] = L[1] = L[2].  Voxel index
 *     i = (ix*n + iy)*n + iz (z fastest); voxel i sits at ((i.)+1/2) L/n.
 *   - The transform is unitary: s_hat = DFT(s)/sqrt(M), M = n^3, V = L^3, and
 *     S_hat(k) = (M/V) P(shell(k)), S_hat(0) = 0.
 *   - Shells: with k_edges == NULL, n_bins linear shells of width k_Nyq/n_bins
 *     on [0, k_Nyq) (shell b holds b^2 (n/2)^2 <= n_bins^2 |m|^2 < (b+1)^2 (n/2)^2,
 *     m the integer wavenumber); otherwise n_bins+1 strictly increasing edges
 *     (in units of 2 pi / L * |m|).  Modes outside the edges form one extra
 *     overflow shell with index n_bins.  1 <= n_bins <= 254.
 *   - Ownership: every pointer argument is borrowed for the duration of the
 *     call only; input arrays are copied, output buffers belong to the caller.
 *     The context owns all device memory it allocates.
 *   - Errors: every call returns an mg_status and never throws.  A device-side
 *     fault (numeric, timeout) or a CUDA error becomes sticky on the context:
 *     later calls return it until mg_destroy.  mg_last_error() explains it.
 *   - Streams: work is enqueued on mg_options.cuda_stream (a cudaStream_t; NULL
 *     = the library's own stream).  Calls that return host data synchronise it.
 */
#ifndef MG_H_
#define MG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,       /* invalid argument or input data                      */
  MG_ENOMEM = 2,       /* device or host allocation failed                    */
  MG_ECUDA = 3,        /* a CUDA runtime call failed                          */
  MG_ETIMEOUT = 4,     /* a device-side wait ran out of its budget            */
  MG_ENUMERIC = 5,     /* a shell draw met sigma_b <= 0, X_b <= 0 or non-finite
                          values; that shell kept its previous P              */
  MG_ESTATE = 6,       /* call not valid in the context's current state       */
  MG_EUNSUPPORTED = 7, /* valid request the library does not implement        */
  MG_EBOUNDS = 8       /* bounds-checked build only (mg_build_flags): a kernel
                          met an index outside its buffer; the access was
                          skipped                                             */
} mg_status;

typedef struct mg_ctx mg_ctx;

/* Grid shape and box side lengths (cubic, see above). */
typedef struct {
  int32_t nx, ny, nz;
  double L[3];
} mg_grid;

typedef struct {
  int32_t precision;      /* 64: FP64 everywhere.  32: FFTs and per-voxel /
                             per-mode draws in FP32; shell sums and the
                             inverse-gamma parameters in FP64.  Default 64.   */
  int32_t n_chains;       /* chains per data set (group), >= 1.  Default 1.  */
  int32_t chain_id0;      /* chain id of a group's first chain (Philox counter
                             word 2); chain c uses chain_id0 + c.  Default 0. */
  double tau_scale;       /* in (0, 1]: tau = tau_scale * min N_i/R_i^2.     */
  const double* P0;       /* n_bins+1 starting powers shared by all chains, or
                             NULL for flat S_hat = 1 (P = V/M).               */
  int32_t record_every;   /* >0: the state after every record_every-th sweep
                             of mg_sweep is a sample: its s goes into per-voxel
                             FP64 sums of s and s^2 (mean/var of
                             mg_read_stats; added inside the next sweep, or
                             when read or replaced first) and its P(k) into
                             the trace (mg_read_pk_trace, mg_pk_acf,
                             mg_pk_quantiles); 0 = off.  mg_sweep_timed
                             records nothing.                                 */
  int32_t fix_P;          /* nonzero: hold P fixed (signal sampler only).     */
  int64_t timeout_cycles; /* budget of device-side waits in clock cycles;
                             0 = library default.                            */
  void* cuda_stream;      /* cudaStream_t the context enqueues on, or NULL.   */
  int32_t yz_cluster;     /* CTAs per x-plane in the y/z pass (1, 2, 4 or 8)
                             for every grid size; 0 = the default.  Sizes the
                             build does not provide give MG_EUNSUPPORTED.    */
  int32_t persistent;     /* nonzero: advance all chains of a batch in ONE
                             persistent kernel launch per sweep (grid sizes
                             16..128, at most 6 sizes and 64 chains per size);
                             MG_EUNSUPPORTED otherwise.  Default 0.          */
  int32_t autotune;       /* nonzero: at init, time the schedules the build
                             provides (y/z cluster size per grid size, the
                             persistent launch) on the context's own chains
                             and keep the fastest (see mg_tune).  Default 0. */
  int32_t mixing;         /* 1: every sweep is the messenger draw followed
                             by the mixing sampler of Sec. 3.3 (Alg. 3) on
                             the shells instead of Alg. 1's signal draw and
                             Alg. 2: x = s_hat/sqrt(S) drawn given S and t,
                             then one Metropolis-Hastings update of sqrt(S_b)
                             per shell with a truncated normal proposal
                             (Philox stream 4), then s_hat = sqrt(S) x.
                             2: sweeps alternate, those with an odd sweep
                             count (the Philox counter word 1) mixing, the
                             others plain.  0: plain sweeps.  Not with
                             persistent (MG_EUNSUPPORTED) or fix_P
                             (MG_EINVAL).  Default 0.                        */
  double start_dispersion; /* >= 0.  > 0: over-dispersed starts (Sec. 3.4 runs
                             independent chains from over-dispersed initial
                             conditions): chain c starts at
                             P_b = P0_b exp(start_dispersion z_b) with z_b the
                             first Box-Muller normal of Philox call
                             (b, 0, chain id, 2).  0: every chain starts at
                             P0.  Default 0.                                 */
} mg_options;

/* Chain statistics (mg_read_stats). Arrays are caller-owned with the sizes
 * given; pass NULL to skip one. */
typedef struct {
  int64_t sweeps;         /* sweeps completed by the context                 */
  int64_t records;        /* sweeps folded into mean/var and the P trace     */
  double tau;             /* tau of the chain's group                        */
  int32_t n_bins;         /* shells of the chain's group (excluding overflow)*/
  int64_t* n_b;           /* [n_bins+1] full-grid modes per shell (out)       */
  double* sigma_b;        /* [n_bins+1] last sweep's sum_k w_k |s_hat_k|^2    */
  double* chi_b;          /* [n_bins+1] last sweep's chi-square draw X_b; with
                             mixing sweeps: 1 where the shell's proposal was
                             accepted, else 0                                 */
  double* mean;           /* [M] per-voxel posterior mean of s over the
                             recorded samples, S1/n (out)                    */
  double* var;            /* [M] their variance (S2 - S1 mean)/(n-1), 0 for
                             n < 2 (out)                                     */
} mg_stats;

/* Fill *opt with the defaults listed in mg_options. */
void mg_options_init(mg_options* opt);

/* Create a context for one data set (Sec. 2 problem statement: grid, noise
 * covariance N, response R, data d, k-shells, seed).  N, R, d: host arrays of
 * M doubles.  R >= 0 (R = 0 marks an unobserved voxel); N > 0 wherever R > 0
 * (ignored where R = 0); at least one voxel observed.  k_edges: NULL or
 * n_bins+1 doubles.  The chains start at s = 0 and P = opt->P0.
 * Errors: MG_EINVAL for invalid arguments or data, MG_EUNSUPPORTED for grids
 * the library does not cover, MG_ENOMEM / MG_ECUDA.  *out is NULL on error. */
mg_status mg_init(mg_ctx** out, const mg_grid* grid, const double* N, const double* R,
                  const double* d, const double* k_edges, int32_t n_bins, uint64_t seed,
                  const mg_options* opt);

/* Create one context holding n_groups independent data sets of possibly
 * different grid sizes, each with opt->n_chains chains; every sweep advances
 * all chains (Sec. 3.4: independent chains need no communication).  Arrays
 * are indexed by group; k_edges[g] may be NULL.  Chains are numbered group by
 * group: chain = g * n_chains + c.  Errors as mg_init. */
mg_status mg_init_batch(mg_ctx** out, int32_t n_groups, const mg_grid* grids,
                        const double* const* N, const double* const* R, const double* const* d,
                        const double* const* k_edges, const int32_t* n_bins,
                        const uint64_t* seeds, const mg_options* opt);

/* Run n_sweeps Gibbs sweeps (Sec. 3.2: Alg. 1 then Alg. 2) on every chain,
 * asynchronously on the context's stream. n_sweeps >= 0. */
mg_status mg_sweep(mg_ctx* ctx, int64_t n_sweeps);

/* Like mg_sweep, but launches the passes one by one (no CUDA graph) with
 * CUDA events around each, and adds the elapsed milliseconds of all sweeps to
 * ms_out[0] (pass YZ: inverse y/z transforms, messenger draw, forward z/y),
 * ms_out[1] (pass X: forward x transform, signal draw, shell sums, inverse x)
 * and ms_out[2] (shell draw of P).  Synchronises. */
mg_status mg_sweep_timed(mg_ctx* ctx, int64_t n_sweeps, double* ms_out);

/* Current signal s of one chain in real space: M values of the context's
 * precision (double for 64, float for 32), written to out — device memory if
 * out_is_device, else host memory (the call then synchronises). */
mg_status mg_read_s(mg_ctx* ctx, int32_t chain, void* out, int32_t out_is_device);

/* Current P of one chain: n_bins+1 doubles to host memory, the last one the
 * overflow shell.  Synchronises. */
mg_status mg_read_pk(mg_ctx* ctx, int32_t chain, double* out);

/* Current P of every chain in one transfer: out (host, ideally pinned) gets
 * n_chains rows of B_max+1 doubles, B_max the largest n_bins in the context;
 * row c holds chain c's n_bins+1 values, the rest of the row is 0.  One copy
 * and one synchronisation for the whole batch (a per-sweep read of all chains
 * costs about as much as one mg_read_pk).  Synchronises. */
mg_status mg_read_pk_all(mg_ctx* ctx, double* out);

/* Statistics of one chain (see mg_stats). Synchronises. */
mg_status mg_read_stats(mg_ctx* ctx, int32_t chain, mg_stats* out);

/* Replace one chain's signal (M values of the context's precision, host or
 * device) — for over-dispersed starts and checkpoint resume. */
mg_status mg_set_s(mg_ctx* ctx, int32_t chain, const void* s, int32_t s_is_device);

/* Replace one chain's P (n_bins+1 host doubles, all > 0). */
mg_status mg_set_pk(mg_ctx* ctx, int32_t chain, const double* P);

/* Replace the data d of one data set (group) — M host doubles, finite — keeping
 * N and R: the messenger constants c = gamma d are recomputed, with
 * gamma = tau R / (tau R^2 + N~) (Sec. 3.1, t-conditional).  Chains keep
 * their state. */
mg_status mg_set_data(mg_ctx* ctx, int32_t group, const double* d);

/* Differentiation of K sweeps (K >= 1) of one chain with P = exp(logP) held
 * fixed and the Philox noise of the chain's next K sweeps held fixed, from the
 * chain's current state s_0.  Loss L = sum_j w_j |s_hat_K,j|^2 over the stored
 * modes of the K-th sample, w in the stored-mode layout [kx][ky][kz] with
 * kz in [0, n/2] (n*n*(n/2+1) host doubles).  Writes L to *loss, dL/dlogP to
 * dlogP (n_bins+1 host doubles) and dL/dd to dd (M host doubles).  The
 * gradients come from a hand-written adjoint of the sweep (transposed FFTs and
 * transposed per-voxel / per-mode affine maps) with the state checkpointed
 * after every forward sweep.  The chain's state, P and the sweep counter are
 * restored before returning.  Synchronises. */
mg_status mg_adjoint(mg_ctx* ctx, int32_t chain, int32_t K, const double* logP, const double* w, double* loss,
                     double* dlogP, double* dd);

/* The recorded P(k) trace of one chain (record_every > 0: P after every
 * record_every-th sweep of mg_sweep, kept on the device).  out: host array of
 * max_records * (n_bins+1) doubles, record-major; the first
 * min(records, max_records) rows are written.  *n_records (may be NULL)
 * receives the number of records.  Synchronises. */
mg_status mg_read_pk_trace(mg_ctx* ctx, int32_t chain, double* out, int64_t max_records, int64_t* n_records);

/* Statistical efficiency of a chain's recorded P(k) (the correlation-length
 * analysis of the paper's results section), computed on the device from the
 * trace: per shell b the autocorrelation
 *   C_n = [1/(R-n) sum_{i<R-n} (P_i - <P>)(P_{i+n} - <P>)] / Var(P),
 * n = 0 .. max_lag (R records, Var with 1/R), into acf[b * (max_lag+1) + n]
 * (host, (n_bins+1)*(max_lag+1) doubles), and the correlation length n_c[b] =
 * the first lag n >= 1 with C_n < 0.1, or -1 if none up to max_lag (host,
 * n_bins+1 int32).  A constant trace (a held empty shell) gives C_n = 1 and
 * n_c = -1.  MG_EINVAL unless 0 <= max_lag < R.  Synchronises. */
mg_status mg_pk_acf(mg_ctx* ctx, int32_t chain, int32_t max_lag, double* acf, int32_t* n_c);

/* Posterior quantiles of each shell's P from the recorded trace, computed on
 * the device (credible bands of the power spectrum): for q[i] in [0, 1],
 * h = (R-1) q, k = floor(h), out[b * n_q + i] = x_(k) + (h - k)(x_(k+1) - x_(k))
 * with x_(j) the j-th smallest of shell b's R recorded values.  q: host, n_q
 * doubles; out: host, (n_bins+1)*n_q doubles.  MG_EINVAL without records.
 * Cost O(R^2) per shell and quantile on the device.  Synchronises. */
mg_status mg_pk_quantiles(mg_ctx* ctx, int32_t chain, int32_t n_q, const double* q, double* out);

/* Gelman-Rubin convergence diagnostic of P(k) across chains (the use the
 * independent chains of Sec. 3.4 are put to), on the device from the recorded
 * traces of chains first_chain .. first_chain+n_chains-1 (2 <= n_chains <= 256,
 * all with the same shells), using records burn .. R-1 (at least 2): per
 * shell, with chain means m_j and unbiased variances v_j over those n
 * records, W = mean_j v_j, B = n/(n_chains-1) sum_j (m_j - mean m)^2 and
 * var+ = (n-1)/n W + B/n, rhat[b] = sqrt(var+ / W) (host, n_bins+1 doubles;
 * 1 where every chain is constant and equal, +inf where they are constant
 * and differ).  Synchronises. */
mg_status mg_pk_rhat(mg_ctx* ctx, int32_t first_chain, int32_t n_chains, int64_t burn, double* rhat);

/* Sweep counter (Philox counter word 1 of the next sweep); mg_set_sweep_count
 * restores it when resuming from a checkpoint. */
mg_status mg_get_sweep_count(mg_ctx* ctx, int64_t* out);
mg_status mg_set_sweep_count(mg_ctx* ctx, int64_t sweeps);

/* Shape queries: total chains, grid size n and shell count of one chain. */
mg_status mg_chain_info(mg_ctx* ctx, int32_t chain, int32_t* n, int32_t* n_bins, int32_t* n_chains);

/* Wait for all enqueued work and report any sticky device status. */
mg_status mg_sync(mg_ctx* ctx);

/* Human-readable description of the last error on ctx (never NULL); with
 * ctx == NULL, why the calling thread's last mg_init / mg_init_batch failed. */
const char* mg_last_error(const mg_ctx* ctx);

/* Free everything the context owns; ctx may be NULL. */
void mg_destroy(mg_ctx* ctx);

/* Autotuner: time every schedule the build provides for this context — the
 * y/z pass's cluster size per grid size and, where eligible, the persistent
 * one-launch sweep against one launch per pass — with `reps` sweeps each on
 * the context's own chains (their state, P and the sweep counter are saved
 * and restored, so the chains are unaffected), then keep the fastest.  The
 * choice is cached per GPU model and batch shape for later contexts in this
 * process.  Synchronises. */
mg_status mg_tune(mg_ctx* ctx, int32_t reps);

/* The schedule in use: number of grid sizes, and per size its n, y/z cluster
 * size; *persistent is 1 if the sweep is one persistent launch.  Arrays hold
 * at least 8 entries; any pointer may be NULL. */
mg_status mg_schedule(mg_ctx* ctx, int32_t* n_sizes, int32_t* n, int32_t* yz_cluster, int32_t* persistent);

/* The unit normals the sweep kernels make from Philox words (Box & Muller
 * 1958 with U(w) = (2w + 1) 2^-33): for i in [0, n_pairs), the words
 * wa = words_device[2i], wb = words_device[2i+1] give
 *   out_device[3i]   = sqrt(-2 ln U(wa)) cos(2 pi U(wb)),
 *   out_device[3i+1] = sqrt(-2 ln U(wa)) sin(2 pi U(wb)),
 *   out_device[3i+2] = -2 ln U(wa)  (the pair's squared radius: the shell
 *                                     sums' chi-square draw with 2 dof).
 * precision 64: out_device holds doubles, made as the FP64 path makes them
 * (table-driven logarithm, sine and cosine); precision 32: floats, as the
 * FP32 path makes them (the special-function unit).  words_device: device
 * memory of 2*n_pairs uint32; out_device: device memory of 3*n_pairs values.
 * stream: cudaStream_t or NULL.  MG_EINVAL for another precision, a negative
 * count or a NULL pointer with n_pairs > 0.  Synchronises. */
mg_status mg_normals(int32_t precision, const uint32_t* words_device, int64_t n_pairs, void* out_device,
                     void* stream);

/* Raw Philox4x32-10 words on the device (Salmon et al. 2011; the per-core
 * generators of Sec. 3.4): for i in [0, n_calls), call i uses counter
 * (ctr0 + i, ctr1, ctr2, ctr3) and key (seed & 0xffffffff, seed >> 32) and
 * writes its 4 words to out_device[4i .. 4i+3].  out_device: device memory of
 * 4*n_calls uint32.  stream: cudaStream_t or NULL.  Synchronises. */
mg_status mg_philox(uint64_t seed, uint32_t ctr0, uint32_t ctr1, uint32_t ctr2, uint32_t ctr3,
                    int64_t n_calls, uint32_t* out_device, void* stream);

/* Shell sums of a given half-complex spectrum without allocating anything on
 * the device.  The paper has no counterpart: this exists for callers that
 * cannot allocate device memory when they need the shell power of a sample —
 * code under an exhausted memory-pool budget, real-time pipelines that forbid
 * allocation (and the synchronisation it implies) after start-up, or host code
 * between kernels it does not own.
 *   s_hat: device array of n*n*(n/2+1) complex values (interleaved re, im;
 *          double if precision == 64, float if 32) in the layout [kx][ky][kz],
 *          kz in [0, n/2] — the unitary convention s_hat = DFT(s)/sqrt(n^3).
 *   n: even, 4 <= n <= 4096;  n_bins: linear shells on [0, k_Nyq) as in
 *          mg_init with k_edges == NULL, plus the overflow shell n_bins.
 *   sigma_out: device, n_bins+1 doubles: sum over the shell of w |s_hat|^2
 *          (w = 2 for 0 < kz < n/2, 1 on the kz = 0 and n/2 planes; DC excluded).
 *   nmodes_out: device, n_bins+1 doubles (sum of w), or NULL.
 *   stream: cudaStream_t or NULL; the call is asynchronous on it.
 * Every sum is formed in a fixed order, so repeated calls on the same input
 * return the same bits.
 * Scratch: a fixed file-scope device array of 256 x 255 x 2 doubles (1 MiB)
 * that every GPU loading the library holds until exit; n_bins > 254 does not
 * fit and returns MG_EINVAL.  The first call in a CUDA context (per device,
 * and again after cudaDeviceReset) looks up the array's device address
 * (cudaGetSymbolAddress) — make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other threads) race.  Errors: MG_EINVAL for bad arguments; MG_ECUDA if a
 * CUDA error from earlier work is already pending (nothing is launched), if
 * the address lookup fails (a later call retries it) or if a launch fails.
 * mg_last_error(NULL) gives the reason on this thread. */
mg_status mg_shell_sums_noalloc(const void* s_hat, int32_t precision, int32_t n, int32_t n_bins,
                                double* sigma_out, double* nmodes_out, void* stream);

/* Failure-detection hook, for tests of the error paths without a GPU fault
 * (the paper has no counterpart).  The after_calls-th checked CUDA runtime
 * call that context c makes from now on (1 = the next) is not made: it
 * reports cudaErrorUnknown, as a failing call would, so the library call that
 * made it returns MG_ECUDA, which is then sticky on c (mg_last_error says the
 * failure was injected).  0 disarms.  Nothing runs on the device because of
 * it.  MG_EINVAL for a null context or after_calls < 0. */
mg_status mg_inject_cuda_error(mg_ctx* c, int32_t after_calls);

/* FP64 fused multiply-add throughput of the current device in GFLOP/s
 * (2 flops per FMA), measured with CUDA events over three launches of a
 * kernel of independent FMA chains (best of three): the roofline denominator
 * of the FP64 sweep, which is bound by the FP64 pipe.  stream: cudaStream_t
 * or NULL.  Allocates and frees a small buffer; synchronises.  MG_EINVAL for
 * a null output, MG_ECUDA if a CUDA call fails. */
mg_status mg_fp64_fma_peak(double* gflops, void* stream);

/* How the library was built: MG_BUILD_CHECKED is set in the bounds-checked
 * build (every device index taken from a host table is checked before use; a
 * violation is skipped and reported as MG_EBOUNDS; grid sizes n <= 32 only). */
#define MG_BUILD_CHECKED 1
int32_t mg_build_flags(void);

#ifdef __cplusplus
}
#endif

#endif /* MG_H_ */
