/*
 * hawkes_gb300.h — C ABI of the GB300 (sm_103a) library for the exact
 * log-likelihood of a multivariate linear exponential Hawkes process and its
 * gradient.
 *
 * Problem statement (paper "Massively Parallel Exact Inference for Hawkes
 * Processes", Section 2):
 *   events   H = {(t_k, c_k)}, k = 0..N-1, t non-decreasing on [0, T], c_k in [0, M)
 *   intensity lambda_i(t) = mu_i + sum_{l before t} alpha[i][c_l] beta_{c_l} exp(-beta_{c_l} (t - t_l))
 *            (Eq. hawkes_excitation with one decay per source mark; a shared decay is the
 *             special case of Eq. hawkes_excitation with K = 1)
 *   L        = sum_k log lambda_{c_k}(t_k) - sum_i int_0^T lambda_i(t) dt
 *            (Eq. general_hawkes_likelihood, with the closed-form compensator
 *             T sum_i mu_i + sum_l colsum_{c_l} (1 - exp(-beta_{c_l} (T - t_l))))
 *   grads    dL/dmu, dL/dalpha, dL/dbeta (Appendix B, Eqs. grad_mu, grad_alpha, grad_gamma)
 *
 * Conventions
 *   - Marks are 0-based (the paper counts 1..M).
 *   - alpha is row-major M x M with row = TARGET mark, column = SOURCE mark, as the
 *     formula of Eq. hawkes_excitation indexes it.
 *   - beta: opts->beta_shared = 1 -> one decay beta[0] shared by every source (the
 *     gradient d_beta is then ONE float); 0 -> beta[M], one decay per source (d_beta[M]).
 *   - Gradients are of L itself, not of the per-event NLL -L/N.
 *   - Ties (equal times) count the earlier-indexed event at full weight, as the
 *     state recurrence of Eq. intensity_state_recurrence does with dt = 0.
 *   - N = 0 is legal: L = -T sum mu and the gradients reduce to the compensator terms.
 *   - Several decay kernels (opts->kernels = K > 1; paper, Eq. hawkes_excitation with its
 *     sum over kernels k = 1..K): kernel q has its own matrix and one decay shared by all
 *     sources,
 *         lambda_i(t) = mu_i + sum_q sum_{l before t} alpha_q[i][c_l] beta_q exp(-beta_q (t - t_l)).
 *     alpha is then [K][M][M] (kernel-major), beta [K], d_alpha [K][M][M] and d_beta [K];
 *     K > 1 needs beta_shared = 1 and the single-sequence entry points (hawkes_loglik,
 *     hawkes_loglik_grad, hawkes_workspace_size with B = 1), and runs the chunk-GEMM path.
 *
 * Memory and ownership
 *   - Every array argument of the device entry points is a DEVICE pointer owned by
 *     the caller; the library never frees or keeps them.  Times are FP64, marks int32,
 *     parameters FP32, the log-likelihood FP64, gradients FP32.
 *   - The library allocates no memory: the caller passes a device workspace of at least
 *     hawkes_workspace_size(...) bytes, 256-byte aligned.  Its contents on entry do not
 *     matter; it holds the device status word afterwards.  One workspace must not be
 *     used by two calls that run concurrently.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy default
 *     stream).  Nothing is read back to the host except by the *_host entry points and
 *     hawkes_last_device_status.
 *
 * Errors
 *   - Errors found on the host (null pointers, sizes, a too-small workspace, an
 *     unsupported configuration, a failed launch) are returned at once and nothing is
 *     launched.
 *   - Errors found on the device (unsorted times, a mark outside [0, M), a time outside
 *     [0, T], mu <= 0, alpha < 0, beta <= 0, a non-finite parameter, an intensity <= 0)
 *     are written to the status word in the workspace; the outputs of that call are then
 *     NaN.  hawkes_last_device_status synchronises the stream and returns that word.
 */
#ifndef HAWKES_GB300_H
#define HAWKES_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HAWKES_OK = 0,
    HAWKES_ERR_INVALID_ARG = 1,       /* null pointer, negative size, bad offsets, T < 0      */
    HAWKES_ERR_UNSORTED = 2,          /* t[k] < t[k-1] inside one sequence                     */
    HAWKES_ERR_MARK_RANGE = 3,        /* c[k] outside [0, M)                                   */
    HAWKES_ERR_TIME_RANGE = 4,        /* t[k] outside [0, T] (or not finite)                   */
    HAWKES_ERR_PARAM_DOMAIN = 5,      /* mu <= 0, alpha < 0, beta <= 0, or a non-finite value  */
    HAWKES_ERR_NONPOS_INTENSITY = 6,  /* some lambda_k <= 0 (impossible inside the domain)     */
    HAWKES_ERR_WORKSPACE = 7,         /* workspace null, too small or not 256-byte aligned     */
    HAWKES_ERR_UNSUPPORTED = 8,       /* a configuration the library does not implement          */
    HAWKES_ERR_CUDA = 9               /* a CUDA runtime call failed                            */
} hawkes_status;

typedef struct {
    int32_t beta_shared;  /* 1: beta[0] is one decay shared by all sources; 0: beta[M]        */
    int32_t chunk;        /* events per scan chunk; 0 = library default                        */
    int32_t validate;     /* 1: run the device input checks (default); 0: trust the inputs      */
    int32_t path;         /* 0: automatic; 1: state-walk kernels (M <= 64 with the gradient,
                             256 without); 2: chunk-GEMM kernels (shared decay, one sequence);
                             3: mark-major walk (one sequence, one kernel; reads alpha through
                             its support, see `support`).  Automatic: M <= 64 (256) -> 1, else
                             shared decay -> 2, per-source decays -> 3.  Every path gives the
                             same result within rounding.                                      */
    int32_t kernels;      /* decay kernels K: 0 or 1 = one kernel; 2..4 = several (see above)   */
    int32_t support;      /* 1: the gradient with respect to alpha is taken on alpha's support,
                             the entries alpha[i][j] != 0 (the interactions the model has): the
                             other entries of d_alpha are 0, every other output is unchanged.
                             0 (default): d_alpha in every entry.  Path 3 needs it for M > 128
                             (its rows of up to 128 support entries are checked on the device:
                             a longer row sets HAWKES_ERR_UNSUPPORTED in the status word).      */
    int32_t reduce;       /* how the chunk-GEMM path (path 2, one kernel) sums the N terms
                             log lambda_k: 0 (default) FP64 partial sums (per thread the running
                             product of its FP32 intensities as an FP32 mantissa and an integer
                             exponent, one FP64 log, FP64 sums across threads); 1 Kahan-
                             compensated FP32 sums of FP32 logs (per thread, then across threads
                             and blocks); 2 plain FP32 sums of FP32 logs.  Other paths: 0 only. */
    int32_t fp32_times;   /* precision ablation only (path 2): 1 forms every time difference
                             from the two times first rounded to FP32, instead of rounding
                             their FP64 difference.  0 (default) for any real use.             */
    int32_t walk_lanes;   /* path 1: lanes of one walker (the threads that share one chunk's
                             state; a warp walks 32 / lanes chunks at once): 8 or 16 (one mark
                             per lane: M <= lanes) or 32 (M <= 64); 0 = chosen from M (8 for
                             M <= 8, 16 for M <= 16, else 32).  Other paths ignore it.          */
} hawkes_opts;

/* Default options: per-source decay, default chunk, validation on, automatic path, one
 * decay kernel, dense alpha gradient.  On path 3 `chunk` is the segment length in events
 * (rounded up to whole tiles of 16,384 events; 0 = chosen by the library). */
hawkes_opts hawkes_default_opts(void);

/* Bytes of device workspace needed by a call on N events (all sequences together),
 * M marks and B sequences (B = 1 for the single-sequence entry points).  `grad` = 1
 * for the *_grad entry points.  Returns 0 if the configuration is unsupported. */
size_t hawkes_workspace_size(int64_t N, int32_t M, int32_t B, int32_t grad,
                             const hawkes_opts* opts);

/* Log-likelihood of one sequence (paper, Eq. general_hawkes_likelihood).
 *   t [N] FP64, c [N] int32, mu [M], alpha [M*M], beta [1 or M] FP32: device inputs.
 *   T: the observation end (host scalar), T >= t[N-1].
 *   out_ll: device pointer to ONE double, written with L. */
hawkes_status hawkes_loglik(const double* t, const int32_t* c, int64_t N, double T,
                            int32_t M, const float* mu, const float* alpha, const float* beta,
                            const hawkes_opts* opts, void* workspace, size_t workspace_bytes,
                            double* out_ll, void* stream);

/* Log-likelihood and gradient of one sequence (paper, Eq. general_hawkes_likelihood and
 * Appendix B, Eqs. grad_mu, grad_alpha, grad_gamma).  Inputs as hawkes_loglik.
 *   out_ll [1] FP64, d_mu [M], d_alpha [M*M], d_beta [1 if shared else M] FP32: device outputs. */
hawkes_status hawkes_loglik_grad(const double* t, const int32_t* c, int64_t N, double T,
                                 int32_t M, const float* mu, const float* alpha,
                                 const float* beta, const hawkes_opts* opts, void* workspace,
                                 size_t workspace_bytes, double* out_ll, float* d_mu,
                                 float* d_alpha, float* d_beta, void* stream);

/* Batched forms over B independent sequences of uneven length (the paper fits one
 * sequence at a time; the batch shares one launch sequence).  Sequence s owns events
 * [offsets[s], offsets[s+1]) of t and c; offsets [B+1] int64 with offsets[0] = 0 and
 * offsets[B] = N; T [B] FP64; mu [B*M]; alpha [B*M*M]; beta [B] if shared else [B*M].
 * All device pointers.  out_ll [B] FP64; d_mu [B*M]; d_alpha [B*M*M]; d_beta [B or B*M]. */
hawkes_status hawkes_loglik_varlen(const double* t, const int32_t* c, const int64_t* offsets,
                                   int32_t B, int64_t N, const double* T, int32_t M,
                                   const float* mu, const float* alpha, const float* beta,
                                   const hawkes_opts* opts, void* workspace,
                                   size_t workspace_bytes, double* out_ll, void* stream);

hawkes_status hawkes_loglik_grad_varlen(const double* t, const int32_t* c,
                                        const int64_t* offsets, int32_t B, int64_t N,
                                        const double* T, int32_t M, const float* mu,
                                        const float* alpha, const float* beta,
                                        const hawkes_opts* opts, void* workspace,
                                        size_t workspace_bytes, double* out_ll, float* d_mu,
                                        float* d_alpha, float* d_beta, void* stream);

/* Slices of one long sequence, for splitting its events over several devices (paper,
 * Section 3.3: a batch of events depends on the previous ones only through one carried
 * state, so the contributions of consecutive slices add up exactly).
 *
 * hawkes_slice_aggregate: the state that the slice's events [t, c] (device, N events) leave
 * at time t_next >= t[N-1] (the first event time of the next slice), from a zero start:
 *     agg_S[j] = sum_{l: c_l = j} exp(-beta_j (t_next - t_l)),
 *     agg_G[j] = sum_{l: c_l = j} (t_next - t_l) exp(-beta_j (t_next - t_l))
 * (device outputs [M]).  The carried state of slice r+1 is then
 *     S_{r+1} = d_r S_r + agg_S_r,  G_{r+1} = d_r (G_r + D_r S_r) + agg_G_r,
 * D_r = t_next - (first event time of slice r), d_r = exp(-beta D_r) (host-side exchange).
 * The workspace only needs its 256-byte header.  The inputs are not validated here.
 *
 * hawkes_loglik_grad_slice: hawkes_loglik_grad for a slice whose first event sees the
 * carried state carry_S, carry_G (device [M] each; both NULL = zero state, i.e. the first
 * slice).  T is the observation end of the whole sequence.  base_term = 1 adds the
 * -T sum(mu) term to L and -T to dL/dmu; set it in exactly one slice.  L and the gradients
 * of all slices sum to those of the whole sequence. */
hawkes_status hawkes_slice_aggregate(const double* t, const int32_t* c, int64_t N, int32_t M,
                                     const float* beta, const hawkes_opts* opts, double t_next,
                                     void* workspace, size_t workspace_bytes, float* agg_S,
                                     float* agg_G, void* stream);
hawkes_status hawkes_loglik_grad_slice(const double* t, const int32_t* c, int64_t N, double T,
                                       int32_t M, const float* mu, const float* alpha,
                                       const float* beta, const hawkes_opts* opts,
                                       const float* carry_S, const float* carry_G,
                                       int32_t base_term, void* workspace,
                                       size_t workspace_bytes, double* out_ll, float* d_mu,
                                       float* d_alpha, float* d_beta, void* stream);

/* End-to-end form of hawkes_loglik_grad with HOST buffers: copies t, c and the
 * parameters from host memory (pinned memory makes the copies asynchronous) into the
 * device workspace, runs the same kernels, copies L and the gradients back into host
 * memory and synchronises `stream` before returning.  The workspace (device) must hold
 * hawkes_workspace_size_host(N, M, opts) bytes.  Device-detected errors are returned
 * directly (the call synchronises anyway). */
size_t hawkes_workspace_size_host(int64_t N, int32_t M, const hawkes_opts* opts);
hawkes_status hawkes_loglik_grad_host(const double* t, const int32_t* c, int64_t N, double T,
                                      int32_t M, const float* mu, const float* alpha,
                                      const float* beta, const hawkes_opts* opts,
                                      void* workspace, size_t workspace_bytes, double* out_ll,
                                      float* d_mu, float* d_alpha, float* d_beta, void* stream);

/* hawkes_loglik_grad for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment convenience).  Some callers own no device allocator
 * (a plain C host, a plug-in whose device memory belongs to another runtime) or must not
 * make the blocking, device-synchronising cudaMalloc call; this entry point takes no
 * workspace and allocates nothing.  It runs the same kernels as hawkes_loglik_grad on a
 * fixed scratch array compiled into the library: hawkes_static_scratch_bytes() bytes
 * (16 MiB) of device memory that every GPU loading the library holds until exit.
 *   - Problems whose hawkes_workspace_size(N, M, 1, 1, opts) exceeds that size are
 *     rejected with HAWKES_ERR_WORKSPACE before anything is launched.
 *   - The first call on a device looks up the scratch address (cudaGetSymbolAddress)
 *     with that device current and caches it; make that first call before any stream
 *     capture.
 *   - All calls share the one array: calls that overlap on the GPU (from several streams
 *     or threads) race on it and must be serialised by the caller.  Each call writes or
 *     zeroes everything it reads, so leftovers of an earlier call do not matter.
 *   - Inputs and outputs are device pointers as in hawkes_loglik_grad; the device status
 *     word is in the scratch array and is not readable through hawkes_last_device_status;
 *     on a device-detected error the outputs are NaN. */
size_t hawkes_static_scratch_bytes(void);
hawkes_status hawkes_loglik_grad_static(const double* t, const int32_t* c, int64_t N, double T,
                                        int32_t M, const float* mu, const float* alpha,
                                        const float* beta, const hawkes_opts* opts,
                                        double* out_ll, float* d_mu, float* d_alpha,
                                        float* d_beta, void* stream);

/* Synchronises `stream` and returns the device status word of the last call that used
 * `workspace` (HAWKES_OK if the device found nothing wrong). */
hawkes_status hawkes_last_device_status(void* workspace, void* stream);

/* Per-mark event counts of the last validated call on `workspace` (int64 [B*M], device),
 * or NULL if that call did not validate.  The pointer is into the workspace. */
const int64_t* hawkes_mark_counts(void* workspace);

/* Integer tables of the last call on `workspace`, as device pointers into the workspace,
 * for checking the library's integer work bit by bit (no counterpart in the paper; the
 * chunks are the contiguous batches of Section 3.3).  N, M, B, grad and opts must be those
 * of that call; the pointers of tables that its path does not build are NULL.  Nothing is
 * launched or read back; read the tables after that call has completed.
 *   mark_counts   [B*M] int64: events of each (sequence, mark); meaningful only when the
 *                 call validated its inputs (opts->validate = 1)
 *   chunk_base    [B+1] int64: chunks of the sequences before each sequence; [B] = all chunks
 *   chunk_seq     [chunks] int32: the sequence that owns each chunk (chunk q of a sequence
 *                 covers its events [q C, min((q + 1) C, len)))
 *   bucket_start  [chunks][P+1] int32 (chunk-GEMM path): per chunk, the number of its events
 *                 whose mark block (mark mod P) is below q, q = 0..P
 *   bucket_slots  [N][4] uint32 (chunk-GEMM path): the chunk's events ordered by (mark mod P,
 *                 mark / P, index in the chunk); word 3 of slot r of a chunk starting at event
 *                 s0 (slot s0 + r) is (index in the chunk << 16) | (mark / P)
 *   chunk         C, events per chunk;  mark_blocks  P (chunk-GEMM path), else 0.
 *   support_row_ptr [M+1] int32, support_col [entries] int32 (mark-major path): the support
 *                 of alpha (every entry unless opts->support), row by row in column order
 *   mark_start    [segments*M+1] int32 (mark-major path): first sorted slot of each
 *                 (segment, mark); segment s covers events [s L, min((s+1) L, N)),
 *                 L = segment_events
 *   mark_slots    [N][4] uint32 (mark-major path): the events in (segment, mark, index)
 *                 order; words 0 and 1 are the FP32 bit patterns of hi = fp32(d) and
 *                 lo = fp32(d - hi), d = t - (time of the segment's first event) in FP64;
 *                 word 2 the event index, word 3 its mark.
 * Returns HAWKES_ERR_INVALID_ARG for a null workspace or output, or the status that
 * hawkes_workspace_size's configuration check gives. */
typedef struct {
    const int64_t* mark_counts;
    const int64_t* chunk_base;
    const int32_t* chunk_seq;
    const int32_t* bucket_start;
    const uint32_t* bucket_slots;
    int32_t chunk;
    int32_t mark_blocks;
    const int32_t* support_row_ptr;
    const int32_t* support_col;
    const int32_t* mark_start;
    const uint32_t* mark_slots;
    int64_t segment_events;
    int32_t segments;
    int32_t reserved;
} hawkes_tables;
hawkes_status hawkes_integer_tables(void* workspace, int64_t N, int32_t M, int32_t B,
                                    int32_t grad, const hawkes_opts* opts, hawkes_tables* out);

/* Static description of a status code. */
const char* hawkes_status_str(hawkes_status s);

/* Number of kernel launches made by the last call on this thread (for accounting). */
int32_t hawkes_last_launch_count(void);

/* Per-kernel timing for measurement (no counterpart in the paper).  After
 * hawkes_profile_enable(1), each call on this thread records a CUDA event on its stream
 * after every kernel it launches.  hawkes_profile_read synchronises on the last event and
 * writes up to `cap` (milliseconds, static kernel name) pairs of the most recent call, in
 * launch order; it returns how many it wrote (negative hawkes_status on a CUDA error).
 * Events are created once, at the first enable; nothing is allocated on the device. */
int32_t hawkes_profile_enable(int32_t on);
int32_t hawkes_profile_read(float* ms, const char** names, int32_t cap);

#ifdef __cplusplus
}
#endif
#endif /* HAWKES_GB300_H */
