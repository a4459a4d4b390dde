// Internal definitions shared by the kernels of libhawkes_gb300 (not part of
// the public C ABI, which is include/hawkes_gb300.h).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "hawkes_gb300.h"

#define HK_FULL 0xffffffffu

namespace hk {

// Workspace header: the first 256 bytes of every workspace.
constexpr int kCarrySegments = 64;   // at most this many segments in the carry pass

struct WsHeader {
    int32_t status;      // device status word (0 = ok, else a hawkes_status)
    int32_t validated;   // 1 if the last call ran the device checks
    int64_t nb;          // number of chunks of the last call (device-computed)
    int64_t pad[30];
};
static_assert(sizeof(WsHeader) == 256, "header must be 256 bytes");

// Everything one launch sequence needs.  Pointers are device pointers.
struct Problem {
    // events
    const double* t;
    const int32_t* c;
    const int64_t* off;      // [B+1]
    const double* Tarr;      // [B]
    int64_t N;
    int32_t B;
    int32_t M;
    // parameters (per sequence when B > 1)
    const float* mu;         // [B*M]
    const float* alpha;      // [B*M*M]
    const float* beta;       // [B] if shared else [B*M]
    int32_t shared;
    int32_t grad;
    int32_t single;          // 1: one sequence; off/Tarr point at header words set by k_init
    int32_t validated;       // 1: the device checks (and mark counts) run in this call
    const float* init_S;     // [M] state just before the first event (NULL = zero state)
    const float* init_G;     // [M] derivative state at the same time (NULL = zero)
    int32_t base_term;       // 1: include -T sum(mu) in L and -T in dL/dmu
    double T_single;
    // chunking
    int32_t C;               // events per chunk
    int32_t P;               // mark blocks of the pair kernels (chunk-GEMM path)
    int32_t Gc;              // chunks per scan group
    int64_t nb_max;          // upper bound on the number of chunks
    int64_t ng_max;          // upper bound on the number of groups
    // workspace regions
    WsHeader* hdr;
    int64_t* counts;         // [B*M]
    int64_t* chunk_base;     // [B+1]
    int32_t* chunk_seq;      // [nb_max]
    float* Shat;             // [nb_max*M] chunk-start states
    float* Ghat;             // [nb_max*M] chunk-start G states (grad only)
    float* grp_v;            // [ng_max*M]
    float* grp_g;            // [ng_max*M]
    double* grp_dt;          // [ng_max] time span of the composite after its last reset
    int32_t* grp_reset;      // [ng_max]
    float* carry_S;          // [ng_max*M]
    float* seg_comp;         // [5][kCarrySegments][M] segment composites of the carry pass
    float* carry_G;          // [ng_max*M]
    double* ll_acc;          // [B]   sum of log lambda
    double* dmu_acc;         // [B*M] sum of w over events of each mark
    double* dal_acc;         // [B*M*M]
    float* dal_part;         // [pair_slots][R][M] partial dalpha rows of the backward pair blocks
    int32_t* pair_redo;      // [pair_slots] blocks of the backward pairs to redo in FP32
    float* scratch;          // [M + 2] outputs of a slice that the caller does not see
    double* dbe_acc;         // [B*M] excitation part of dbeta
    double* E_acc;           // [B*M] sum (1 - exp(-beta (T - t))) per source
    double* F_acc;           // [B*M] sum (T - t) exp(-beta (T - t)) per source
    double* colsum;          // [B*M] sum_i alpha[s][i][j]
    // chunk-GEMM path
    float* Y;                // [nb_max*M]  alpha . Shat_b
    float* Z;                // [nb_max*M]  alpha . (Shat_b - beta Ghat_b)
    float* W;                // [M][nbp]  per-chunk weights of the dalpha GEMM, transposed:
                             // W[i * nbp + b] = sum of w_k e_k over the events k of mark i in chunk b
    float* dal_gemm;         // [M*M]
    // fp16 hi/lo operands of the tensor-core GEMMs (rows scaled by powers of two), as
    // paired rows: per group of 32 elements their 32 high parts, then their 32 low parts
    __half* al_p;            // [M][ldk]       alpha
    __half* S_p;             // [nb_max][ldk]  chunk-start states
    __half* G_p;             // [nb_max][ldk]  Shat - beta Ghat
    __half* Wt_p;            // [M][ldt]       W transposed (chunks contiguous)
    __half* St_p;            // [M][ldt]       S^ transposed
    float *isc_al, *isc_S, *isc_G, *isc_Wt, *isc_St;   // inverse row scales of the operands
    uint32_t* colmax;        // [M] column maxima scratch of the transposed operands
    // intra-chunk pair kernels
    float4* recs;            // [N]  events bucketed by mark block inside each chunk
    float2* src;             // [N]  (ep, mark) of every event in index order (backward sources)
    int4* kprep;             // [N]  backward row-group data of every bucket slot
    float* at;               // [P*P*128*128] alpha in tile-major order (forward pairs)
    int32_t* bstart;         // [nb_max * (P+1)] bucket offsets inside each chunk
    // row blocks of the backward pairs: R (a power of two) positions of one mark block, i.e.
    // marks I + P pos for pos in [q R, q R + R), row block I * nrb + q
    int32_t lgR;             // log2 R
    int32_t nrb;             // row blocks per mark block, ceil(ceil(M / P) / R)
    int32_t n_rb;            // P * nrb
    int32_t pair_slots;      // blocks the pair plan can hand out (target blocks + n_rb)
    int32_t* bsub;           // [nb_max * (n_rb + 1)] first bucket slot of every row block, then n
    int32_t* pwork;          // [n_rb * nb_max] backward work of every (row block, chunk)
    int64_t* pcum;           // [n_rb * (nb_max + 1)] its prefix over the chunks
    int64_t* ptot;           // [n_rb] its total
    int32_t* plan_b;         // backward pair plan: [0] blocks used, [1 + rb] blocks of row
                             //   block rb, [1 + n_rb + rb] its first block, then
                             //   [1 + 2 n_rb + x] = rb << 16 | k for block x
    uint8_t* wide;           // [nb_max] chunk spans too wide for the factorised weights
    float* Aint;             // [N]  sum_{l<k in chunk} P_kl alpha[c_k][c_l]
    float* Bint;             // [N]  same, weighted by (t_k - t_l)
    float* wbuf;             // [N]  w_k = 1 / lambda_k
    float* delta;            // [N]  t_k - t of the first event of k's chunk (chunk-GEMM path,
                             //      written by the scan; null on the state-walk path)
    float* Dspan;            // [nb_max] t of the next chunk's first event - t of its first (same)
    float* Tmt;              // [nb_max] T - t of the chunk's first event (same)
    // centering of the GEMM operands (the tensor-core accumulation error is one-signed
    // for same-signed operands; centred operands make it unbiased): column means of the
    // operands over a sample of chunks, added back exactly through the biases
    float* cen_S;            // [M] mean of S^_b[j] over the sampled chunks
    float* bias_Y;           // [M] alpha . cen_S  (FP64-accumulated)
    float* cen_Z;            // [M] mean of (S^_b - beta G^_b)[j] over the sampled chunks
    float* bias_Z;           // [M] alpha . cen_Z  (FP64-accumulated)
    float* cen_acc;          // [32][2M] column sums of the sampled rows per row slice, then
                             // the number of sampled rows
    double* wsum_acc;        // [M] sum_b W[b][i]
    uint32_t* wmax;          // [M] largest W[b][i] over b (bits of a non-negative float)
    int32_t w_rowstats;      // 1: the epilogue takes wsum_acc and wmax while it writes W
    int64_t ldk;             // 64 ceil(M / 32): halves per paired row of K = M elements
    int64_t ldt;             // 64 ceil(nbp / 32): halves per paired row of K = nbp elements
    int64_t nbp;             // nb_max rounded up to 8
    // mark-major walk (one decay per source, large M)
    int32_t support;         // 1: dalpha on alpha's support only (entries alpha == 0 get 0)
    int32_t* row_ptr;        // [M+1] support rows of alpha
    int32_t* sup_col;        // [nnz] column of each support entry, by row
    float* sup_val;          // [nnz] its value
    int32_t* tile_cnt;       // [ntiles][M] events per mark of each tile, then prefix in segment
    int32_t* seg_off;        // [nseg*M + 1] first sorted slot of every (segment, mark)
    double* seg_time;        // [3 nseg] first time, span to the next segment, T - first time
    float* seg_f;            // [4 nseg] the span and T - first time as FP32 (hi, lo) pairs
    int32_t nseg;            // segments
    int32_t ntiles;          // tiles of the sort
    int32_t seg_tiles;       // tiles per segment
    int32_t tile_warps;      // tiles (warps) per block of the sort kernels
    // precision options of the chunk-GEMM path
    int32_t reduce;          // 0: FP64 log-sum; 1: Kahan FP32; 2: plain FP32
    int32_t fp32_times;      // ablation: time differences of FP32-rounded times
    float* ll_part;          // [2 * kLogSumBlocks] per-block (sum, error) of the FP32 log-sums
    int32_t bucket_done;     // 1: the chunks were bucketed piece by piece as the events arrived
    int32_t walk_lanes;      // state walk: lanes per walker (0 = from M)
    // outputs
    double* out_ll;          // [B]
    float* d_mu;
    float* d_alpha;
    float* d_beta;
};

__device__ __forceinline__ void set_status(WsHeader* h, int code) {
    atomicCAS(&h->status, 0, code);
}

__device__ __forceinline__ bool failed(const WsHeader* h) {
    return *((volatile const int32_t*)&h->status) != 0;
}

// exp(x) in FP32 arithmetic whose rounding error has no systematic sign.  The decay
// factors exp(-beta dt) are multiplied along the chain of chunk (and event) steps, so a
// one-signed error of a fraction of an ulp per factor grows with the chain length, and
// the decay gradient (a small difference of state sums) amplifies it; an error of
// either sign at random does neither.  Method: Cody-Waite reduction x = k ln2 + r with
// ln2 split as 355/512 + c2 (k * 355/512 is exact for |k| < 2^15) and |r| <= ln2 / 2
// (k = 0 for |x| < ln2 / 2), the Taylor series e^r - 1 = r + r^2 (1/2! + r/3! + ... +
// r^6/8!) (truncation below 2.2e-10), one rounding of 1 + (e^r - 1), and the exact
// scaling by 2^k.  Exact 1 at x = 0, 0 below -104, +inf above 88.8.
__device__ __forceinline__ float exp_unbiased(float x) {
    float k = 0.f, r = x;
    if (!(fabsf(x) < 0.34657359f)) {
        if (x < -104.f) return 0.f;
        if (x > 88.8f) return __int_as_float(0x7f800000);
        k = rintf(x * 1.44269504f);
        r = fmaf(-k, 0.693359375f, x);
        r = fmaf(-k, -2.12194440e-4f, r);
    }
    float q = fmaf(r, 1.f / 40320.f, 1.f / 5040.f);
    q = fmaf(q, r, 1.f / 720.f);
    q = fmaf(q, r, 1.f / 120.f);
    q = fmaf(q, r, 1.f / 24.f);
    q = fmaf(q, r, 1.f / 6.f);
    q = fmaf(q, r, 0.5f);
    const float y = 1.f + fmaf(r * r, q, r);
    int ki = (int)k;
    if (ki == 0) return y;
    if (ki < -126) return (y * 0x1p-64f) * __int_as_float((ki + 64 + 127) << 23);
    if (ki > 127) return (y * 2.f) * __int_as_float((ki - 1 + 127) << 23);
    return y * __int_as_float((ki + 127) << 23);
}

// t_a - t_b as the kernels form a time difference: in FP64 (then rounded to FP32 by the
// caller), or, for the precision ablation, from the two times rounded to FP32 first.
__device__ __forceinline__ double tdiff(const Problem& p, double a, double b) {
    return p.fp32_times ? (double)((float)a - (float)b) : a - b;
}

// Compensated FP32 sum (Neumaier's variant of Kahan summation): the value is s + e.
struct SumF32 {
    float s = 0.f, e = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        e += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ void add(const SumF32& o) {
        add(o.s);
        e += o.e;
    }
};
constexpr int kLogSumBlocks = 4096;   // capacity of the per-block log-sum partials

__device__ __forceinline__ float beta_of(const Problem& p, int32_t seq, int32_t j) {
    return p.shared ? p.beta[seq] : p.beta[(int64_t)seq * p.M + j];
}

// chunk b of sequence seq covers events [s0, s1)
__device__ __forceinline__ void chunk_range(const Problem& p, int64_t b, int32_t seq,
                                            int64_t& s0, int64_t& s1) {
    int64_t q = b - p.chunk_base[seq];
    s0 = p.off[seq] + q * p.C;
    int64_t e = p.off[seq + 1];
    s1 = s0 + p.C < e ? s0 + p.C : e;
}

__device__ __forceinline__ int64_t num_chunks(const Problem& p) { return p.chunk_base[p.B]; }

// Sum of log lambda without per-event log rounding.  Running product of positive FP32 factors as an FP32 mantissa in [1, 2) and an integer
// binary exponent (no FP64 arithmetic per factor: this part's FP64 rate is 1/64 of its
// FP32 rate); one FP64 log per thread at the end.  Each factor adds one FP32 rounding
// (relative 2^-24, either sign) to the product.
struct LogProd {
    float m = 1.f;
    int e = 0;
    __device__ __forceinline__ void mul(float x) {
        uint32_t bx = __float_as_uint(x);
        const uint32_t ex = (bx >> 23) & 0xffu;
        if (ex - 1u < 254u) {                  // positive normal: mantissa and exponent by bits
            e += (int)ex - 127;
            m *= __uint_as_float((bx & 0x007fffffu) | 0x3f800000u);
        } else {                               // zero, subnormal, inf, NaN: propagate
            int k;
            const float f = frexpf(x, &k);
            e += k;
            m *= f;
        }
        const uint32_t bm = __float_as_uint(m);
        const uint32_t em = (bm >> 23) & 0xffu;
        if (em - 1u < 254u) {
            e += (int)em - 127;
            m = __uint_as_float((bm & 0x807fffffu) | 0x3f800000u);
        }
    }
    __device__ __forceinline__ double log_value() const {
        return log((double)m) + (double)e * 0.69314718055994530942;
    }
};

}  // namespace hk

// launch helpers implemented in the .cu files
namespace hk {
cudaError_t launch_prepare(const Problem& p, cudaStream_t s, int validate, int* nlaunch);
cudaError_t launch_prepare_head(const Problem& p, cudaStream_t s, int validate, int* nlaunch);
cudaError_t launch_validate_chunks(const Problem& p, cudaStream_t s, int64_t b_begin,
                                   int64_t b_end, int* nlaunch);
cudaError_t launch_scan(const Problem& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_scan_reduce(const Problem& p, cudaStream_t s, int64_t g_begin, int64_t g_end,
                               int* nlaunch);
cudaError_t launch_scan_rest(const Problem& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_walk(const Problem& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_gemm_path(const Problem& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_gemm_forward(const Problem& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_gemm_epilogue(const Problem& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_bucket_range(const Problem& p, cudaStream_t s, int64_t b_begin, int64_t b_end,
                                int* nlaunch);
cudaError_t launch_gemm_backward(const Problem& p, cudaStream_t s, int* nlaunch);

// ---------------------------------------------------------------------------
// Intra-chunk pairs of the chunk-GEMM path (pairs.cu, with the bucketing in gemm_path.cu).
// A bucketed record is (delta, em, ep, index << 16 | position): delta = t - t of the chunk's
// first event, em = exp(-beta delta), ep = exp(+beta delta) (0 in a wide chunk), the
// event's index in its chunk and the position c / P of its mark c in mark block c mod P.
// ---------------------------------------------------------------------------
constexpr float kWideLimit = 64.f;      // beta * span above which sums of exp(+beta delta) may overflow
constexpr int kPairTileFloats = 32768;  // shared-memory rows of one backward pair block: R M <= this
constexpr int kPairBlocksMax = 1024;    // thread blocks the backward pair plan aims at, at most
__device__ __forceinline__ int rec_idx(float4 r) { return __float_as_int(r.w) >> 16; }
__device__ __forceinline__ int rec_pos(float4 r) { return __float_as_int(r.w) & 0xffff; }
// Row blocks of the backward pairs: R = 2^lgR positions of one mark block (the largest power of two with R M
// words in kPairTileFloats, and no larger than the block's ceil(M / P) positions need),
// nrb of them per mark block, n_rb = P nrb in all.
struct PairRows {
    int lgR, nrb, n_rb, slots;
};
__host__ __device__ inline PairRows pair_rows(int M, int P) {
    const int TR = (M + P - 1) / P;
    int lg = 0;
    while ((int64_t)(2 << lg) * M <= kPairTileFloats && (1 << lg) < TR) ++lg;
    PairRows r;
    r.lgR = lg;
    r.nrb = (TR + (1 << lg) - 1) >> lg;
    r.n_rb = P * r.nrb;
    r.slots = kPairBlocksMax + r.n_rb;
    return r;
}
cudaError_t launch_pairs_forward(const Problem& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_pairs_backward(const Problem& p, cudaStream_t s, int* nlaunch);

// Several decay kernels: one workspace slice per kernel, each a complete single-kernel
// problem; the epilogue and the last step of the finalisation combine the slices.
constexpr int kMaxKernels = 4;
struct KernelSlice {
    const float* Y;
    const float* Z;
    const float* A;          // intra-chunk pair sums A_k, B_k of this kernel
    const float* B;
    float* W;                // rows of this kernel's dalpha GEMM
    double* E_acc;
    double* F_acc;
    double* dbe_acc;
    double* wsum_acc;
    const float* beta;       // this kernel's decay (one value)
    WsHeader* hdr;
    double* out_ll;          // this slice's partial log-likelihood
};
struct MultiSlices {
    int32_t K;
    KernelSlice k[kMaxKernels];
};
cudaError_t launch_epilogue_multi(const Problem& p0, const MultiSlices& ms, cudaStream_t s,
                                  int* nlaunch);
cudaError_t launch_finalize_multi(const Problem& p0, const MultiSlices& ms, cudaStream_t s,
                                  int* nlaunch);
cudaError_t launch_finalize(const Problem& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_finalize_mode(const Problem& p, cudaStream_t s, int mode, int* nlaunch);
// the mark-major walk (marks.cu): segment length L events
cudaError_t launch_marks(const Problem& p, int64_t L, cudaStream_t s, int* nlaunch);
int marks_row_max();
int marks_tile_events();
cudaError_t launch_slice_aggregate(const Problem& p, double t_next, float* agg_S, float* agg_G,
                                   cudaStream_t s, int* nlaunch);
int walk_max_m(int grad);
// Host-side argument checks of a single-sequence call (api.cu): 0 or the status that
// hawkes_loglik(_grad) returns before anything is launched.
int check_single_args(const double* t, const int32_t* c, int64_t N, double T, int32_t M,
                      const float* mu, const float* alpha, const float* beta,
                      const hawkes_opts* opts, const double* out_ll, const float* d_mu,
                      const float* d_alpha, const float* d_beta, int grad);
// Optional per-kernel timing: when enabled, records a CUDA event on the launch
// stream after each kernel (names are static strings).
void prof_mark(cudaStream_t s, const char* name);
}  // namespace hk
