// Chunk-GEMM path for one shared decay beta (any M).
//
// With chunk b starting at event s_b (time tau_b) and S^_b, G^_b the chunk-start
// states of the scan, every event k of the chunk splits into an inter-chunk part
// that depends on S^_b only through alpha . S^_b, and an intra-chunk part over the
// earlier events l of the same chunk (paper, Section 3.3: a batch depends on the
// previous one only through one carried state):
//   S_k = e_k S^_b + sum_{l<k in b} exp(-beta (t_k - t_l)) e_{c_l},   e_k = exp(-beta (t_k - tau_b))
//   G_k = e_k (delta_k S^_b + G^_b) + sum_{l<k in b} (t_k - t_l) exp(-beta (t_k - t_l)) e_{c_l}
// so with Y_b = alpha S^_b and Z_b = alpha G^_b (dense GEMMs over all chunks),
//   (alpha S_k)_{c_k} = e_k Y_b[c_k] + A_k,   A_k = sum_{l<k in b} exp(-beta(t_k-t_l)) alpha[c_k][c_l]
//   (alpha G_k)_{c_k} = e_k (delta_k Y_b[c_k] + Z_b[c_k]) + B_k   (B_k likewise, times (t_k - t_l))
//   lambda_k = mu_{c_k} + beta (alpha S_k)_{c_k}                  (Eq. hawkes_excitation, K = 1)
//   dL/dbeta (excitation part) = sum_k w_k [(alpha S_k)_{c_k} - beta (alpha G_k)_{c_k}]
//   dL/dalpha_ij (excitation part) = beta [ sum_b W[b][i] S^_b[j]
//                                          + sum_{pairs l<k in one chunk, c_k=i, c_l=j} w_k exp(-beta(t_k-t_l)) ]
// with W[b][i] = sum_{k in b, c_k = i} w_k e_k, the second dense GEMM.
#include <type_traits>

#include "common.cuh"

namespace hk {

// Tensor-core GEMM and fp16 hi/lo splitting of row-scaled operands into paired rows
// (tc_gemm.cu).
cudaError_t tc_gemm_f16x3(const __half* A, int64_t lda, const __half* B, int64_t ldb, float* D,
                          int64_t ldd, int Mdim, int Ndim, int64_t Kdim, int splits,
                          bool accumulate, WsHeader* hdr, cudaStream_t s, const float* bias,
                          const float* inv_sa, const float* inv_sb);
cudaError_t split_f16_rows(const float* src, int64_t lds, __half* dst, int64_t ldd,
                           int64_t rows, int64_t cols, cudaStream_t s, const float* centre,
                           const int64_t* rows_valid, float* inv_scale, const float* sub,
                           const float* coef);
cudaError_t split_f16_long_rows(const float* src, int64_t lds, __half* dst, int64_t ldd,
                                int64_t rows, int64_t cols, cudaStream_t s, float* inv_scale,
                                double* row_sum, const uint32_t* row_max = nullptr);
cudaError_t split_f16_rows_pair(const float* src, const float* sub, int64_t lds,
                                const float* centre, const float* centre2, const float* coef,
                                __half* out1,
                                float* isc1, __half* out2, float* isc2, int64_t ldd,
                                int64_t rows, int64_t cols, const int64_t* rows_valid,
                                uint32_t* colmax, cudaStream_t s);
cudaError_t transpose_split_f16(const float* src, int64_t cols, const int64_t* rows_valid,
                                int64_t rows_pad, __half* dst, int64_t ldd, cudaStream_t s,
                                const float* centre, uint32_t* amax_bits, float* inv_scale,
                                bool have_max);

// Centres of the GEMM operands.  The tensor cores accumulate the products of one k-group
// with a rounding toward zero, so when a row's products share one sign the error of every
// product adds up with that sign (Section 3's products of the states with alpha >= 0 are
// such rows: most marks fire rarely, and S^ - beta G^ of a rarely fired mark is mostly
// negative).  Each operand column is therefore centred on its mean over a sample of the
// chunks (every step-th chunk, at most kCentreRows of them) before the split, and the
// exact products alpha . centre (FP64-accumulated) are added back as the GEMM's bias.
// Any centre gives the same product up to rounding; a centre near the column mean makes
// the products of each row mixed in sign, so that the accumulation error has mean zero.
constexpr int kCentreRows = 1024;
constexpr int kCentreSlices = 32;     // row slices of the column sums, one block row each

// Column sums of S^ and S^ - beta G^ over the sampled chunks: block (x, y) takes 256
// columns and every kCentreSlices-th sampled row from slice y, and writes its sums to
// acc[y][2 M] (no atomics: the centres, and so the rounding of the GEMMs, are the same in
// every call); the number of sampled rows goes to acc_n.
__global__ void k_col_sums(Problem p, int want_z, float* acc, int* acc_n) {
    const int M = p.M;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nb = num_chunks(p);
    const int64_t step = nb > kCentreRows ? (nb + kCentreRows - 1) / kCentreRows : 1;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *acc_n = (int)((nb + step - 1) / step);
    if (j >= M) return;
    const float beta = p.beta[0];
    float s = 0.f, z = 0.f;
    for (int64_t b = (int64_t)blockIdx.y * step; b < nb; b += (int64_t)kCentreSlices * step) {
        const float v = p.Shat[b * M + j];
        s += v;
        if (want_z) z += v - beta * p.Ghat[b * M + j];
    }
    acc[(int64_t)blockIdx.y * 2 * M + j] = s;
    acc[(int64_t)blockIdx.y * 2 * M + M + j] = z;
}

// The centres cen_S, cen_Z: the column means over the sampled rows (the slices' sums added
// in slice order), one thread per column.
__global__ void k_centre_means(Problem p, int want_z, const float* acc, const int* acc_n) {
    const int M = p.M;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const float inv = *acc_n > 0 ? 1.f / (float)*acc_n : 0.f;
    float s = 0.f, z = 0.f;
    for (int y = 0; y < kCentreSlices; ++y) {
        s += acc[(int64_t)y * 2 * M + j];
        z += acc[(int64_t)y * 2 * M + M + j];
    }
    p.cen_S[j] = s * inv;
    if (want_z) p.cen_Z[j] = z * inv;
}

// bias_Y = alpha . cen_S and bias_Z = alpha . cen_Z in FP64, one warp per row of alpha.
__global__ void k_centres(Problem p, int want_z) {
    const int M = p.M;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < M; i += nwarps) {
        double y = 0.0, z = 0.0;
        for (int j = lane; j < M; j += 32) {
            const double a = (double)p.alpha[(int64_t)i * M + j];
            y += a * (double)p.cen_S[j];
            if (want_z) z += a * (double)p.cen_Z[j];
        }
        for (int o = 16; o >= 1; o >>= 1) {
            y += __shfl_xor_sync(HK_FULL, y, o);
            z += __shfl_xor_sync(HK_FULL, z, o);
        }
        if (lane == 0) {
            p.bias_Y[i] = (float)y;
            if (want_z) p.bias_Z[i] = (float)z;
        }
    }
}

// ---------------------------------------------------------------------------
// Bucketing of every chunk's events for the intra-chunk pairs (pairs.cu).
//
// The marks are dealt round-robin into P mark blocks (block of mark c = c mod P, position
// c / P; dealing spreads the few very frequent marks of a skewed mark distribution over all
// blocks) and every chunk's events are bucketed by block, each bucket sorted by (position,
// index), so that the targets of one row block (R consecutive positions of one block) are a
// contiguous run of slots.  Pair weights are exp(-beta (t_k - t_l)) = em_k * ep_l with
// em = exp(-beta delta), ep = exp(+beta delta), delta = t - tau_b; a chunk whose span would
// overflow ep is flagged "wide" and uses one exp per pair instead.
// ---------------------------------------------------------------------------
// One warp per chunk (up to eight chunks per block at a time, no block-wide barrier after
// the mark table): bucket the chunk's events by mark block, each bucket sorted by (position
// of the mark in its block, index in the chunk) in recs, with the first slot of every row
// block of the backward pairs in bsub, and every event's (ep, mark) in index order in src
// (the backward pairs' sources).  The sorted order comes from counts: per (block,
// position) - one mark - the number of the chunk's events, an exclusive scan of those counts
// in (block, position) order (the first slot of every mark), and the events taking their
// slots in index order (the lanes of one mark in one 32-event step ordered by lane).
// The per-mark counts are stored with one padding word after every 32, so that the
// lanes' contiguous runs of the scan fall in distinct banks.
__host__ __device__ inline int bucket_pad(int e) { return e + (e >> 5); }
__host__ __device__ inline int bucket_ints_per_warp(int P, int C, int M) {
    const int TR = (M + P - 1) / P;
    return 2 * P + 1 + bucket_pad(P * TR) + 1;
}
// shared memory of k_bucket: each warp's scratch, then the mark -> (block, position) table
__host__ __device__ inline size_t bucket_smem_bytes(int P, int C, int M, int warps) {
    return sizeof(int32_t) * ((size_t)warps * bucket_ints_per_warp(P, C, M) + (size_t)M);
}

__global__ void __launch_bounds__(256) k_bucket(Problem p, float4* recs, float2* src,
                                                int32_t* bstart, uint8_t* wide,
                                                int64_t b_begin, int64_t b_end) {
    extern __shared__ int32_t sm_i[];
    const int P = p.P, C = p.C;
    const int TR = (p.M + P - 1) / P, PT = P * TR;
    const int n_rb = p.n_rb, nrb = p.nrb, lgR = p.lgR;
    const int lane = threadIdx.x & 31;
    int32_t* cnt = sm_i + (threadIdx.x >> 5) * bucket_ints_per_warp(P, C, p.M);   // [P]
    int32_t* base = cnt + P;              // [P+1]
    int32_t* slot = base + P + 1;         // [P * TR] per (block, position), padded: count, then next slot
    const int PTP = bucket_pad(PT) + 1;
    // mark c -> (position c / P) << 16 | (block c mod P), so that no event divides by P
    int32_t* qtab = sm_i + (blockDim.x >> 5) * bucket_ints_per_warp(P, C, p.M);
    if (failed(p.hdr)) return;
    for (int c = threadIdx.x; c < p.M; c += blockDim.x) qtab[c] = ((c / P) << 16) | (c % P);
    __syncthreads();
    const float beta = p.beta[0];
    const int64_t nb = num_chunks(p) < b_end ? num_chunks(p) : b_end;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = b_begin + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); b < nb;
         b += nw) {
        int64_t s0, s1;
        chunk_range(p, b, 0, s0, s1);
        const int n = (int)(s1 - s0);
        for (int q = lane; q < P; q += 32) cnt[q] = 0;
        for (int e = lane; e < PTP; e += 32) slot[e] = 0;
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const int qp = qtab[__ldg(p.c + s0 + i)];
            const int q = qp & 0xffff;
            atomicAdd(&cnt[q], 1);
            atomicAdd(&slot[bucket_pad(q * TR + (qp >> 16))], 1);
        }
        __syncwarp();
        if (lane == 0) {
            int acc = 0;
            for (int q = 0; q < P; ++q) {
                base[q] = acc;
                bstart[b * (P + 1) + q] = acc;
                acc += cnt[q];
            }
            base[P] = acc;
            bstart[b * (P + 1) + P] = acc;
        }
        {
            // exclusive scan of the per-mark counts in (block, position) order: each lane sums
            // a contiguous run, the warp scans the run sums, each lane writes its run's prefixes
            const int per = (PT + 31) >> 5;
            const int e0 = min(lane * per, PT), e1 = min(e0 + per, PT);
            int sum = 0;
            for (int e = e0; e < e1; ++e) sum += slot[bucket_pad(e)];
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(HK_FULL, incl, o);
                if (lane >= o) incl += x;
            }
            int run = incl - sum;
            for (int e = e0; e < e1; ++e) {
                const int v = slot[bucket_pad(e)];
                slot[bucket_pad(e)] = run;
                run += v;
            }
        }
        __syncwarp();
        // first slot of every row block (block e / nrb, first position (e mod nrb) R)
        int32_t* bs = p.bsub + b * (n_rb + 1);
        for (int e = lane; e < n_rb; e += 32) {
            const int q = e / nrb;
            bs[e] = slot[bucket_pad(q * TR + ((e - q * nrb) << lgR))];
        }
        if (lane == 0) bs[n_rb] = n;
        __syncwarp();
        const bool isw = n > 0 && beta * (float)tdiff(p, p.t[s1 - 1], p.t[s0]) > kWideLimit;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const bool have = i < n;
            const int ci = have ? __ldg(p.c + s0 + i) : 0;
            const int qp = have ? qtab[ci] : 0;
            const int q = qp & 0xffff, pos = qp >> 16;
            // the lanes of one mark take consecutive slots in lane (= index) order
            const int key = have ? q * TR + pos : -1 - lane;
            const uint32_t peers = __match_any_sync(HK_FULL, key);
            const int leader = __ffs(peers) - 1;
            int first = 0;
            if (have && lane == leader) first = atomicAdd(&slot[bucket_pad(key)], __popc(peers));
            first = __shfl_sync(HK_FULL, first, leader);
            if (have) {
                const int at = first + __popc(peers & ((1u << lane) - 1u));   // from the chunk's start
                const float d = p.delta[s0 + i];
                const float em = exp_unbiased(-beta * d);
                const float ep = isw ? 0.f : exp_unbiased(beta * d);
                recs[s0 + at] = make_float4(d, em, ep, __int_as_float((i << 16) | pos));
                src[s0 + i] = make_float2(ep, __int_as_float(ci));
            }
        }
        if (lane == 0) wide[b] = isw ? 1 : 0;
        __syncwarp();
    }
}

// Row groups of the backward pairs, once per (chunk, bucket): for every 32-lane group of a
// bucket (sorted by (position, index)), u_k = w_k em_k, U_k = sum of u over the lane's row
// group (the events of its mark in the group) from k on, and the index of the previous
// event of the same mark in the group (-1 if none): kprep[slot] = (position, U_k, index,
// previous).  The target k then owes U_k ep_l to (c_k, c_l) for the sources l with index in
// [previous, k) (from 0 without a previous one): every (mark, source) pair of the group gets
// one add.  Also the backward pairs' work of every (row block, chunk) in pwork: per target its
// 32-source steps plus one.  Chunks too wide for the factorised weights get only the work
// (their pairs take one exp each, over all earlier sources).
__global__ void __launch_bounds__(256, 4) k_bwd_prep(Problem p, const float4* __restrict__ recs,
                                                  const int32_t* __restrict__ bstart,
                                                  const uint8_t* __restrict__ wide,
                                                  const float* __restrict__ wbuf, int4* kprep) {
    // A warp takes a chunk and its buckets kPrepBatch at a time: the bounds, first 32
    // records and weights of the batch's buckets are loaded together (three dependent loads
    // per batch instead of per bucket), then each bucket is processed in turn.
    constexpr int kPrepBatch = 8;
    __shared__ int32_t wsh[8][128];      // per warp: work of the bucket's row blocks
    if (failed(p.hdr)) return;
    const int P = p.P, C = p.C, lane = threadIdx.x & 31;
    const int nrb = p.nrb, lgR = p.lgR;
    int32_t* work = wsh[threadIdx.x >> 5];
    const int64_t nb = num_chunks(p);
    const int64_t wpb = blockDim.x >> 5;
    // one 32-event step of bucket I: the row groups' U and previous indices, and the work
    auto step = [&](int64_t s0, bool isw, int kk, int k1, float4 rk, float wk) {
        const bool have = kk < k1;
        const int ik = have ? rec_idx(rk) : -1;
        const int row = have ? rec_pos(rk) : -1 - lane;   // distinct for idle lanes
        int n = ik;                                        // sources of a wide chunk's target
        if (!isw) {
            float U = wk * rk.y;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float up = __shfl_down_sync(HK_FULL, U, o);
                const int rowo = __shfl_down_sync(HK_FULL, row, o);
                if (lane + o < 32 && rowo == row) U += up;
            }
            const int prow = __shfl_up_sync(HK_FULL, row, 1);
            const int pidx = __shfl_up_sync(HK_FULL, ik, 1);
            const int lo = (lane > 0 && prow == row) ? pidx : -1;
            if (have) kprep[s0 + kk] = make_int4(row, __float_as_int(U), ik, lo);
            n = ik - (lo > 0 ? lo : 0);
        }
        if (have) atomicAdd(&work[row >> lgR], ((n + 31) >> 5) + 1);
    };
    for (int64_t b = blockIdx.x * wpb + (threadIdx.x >> 5); b < nb; b += (int64_t)gridDim.x * wpb) {
        const bool isw = wide[b] != 0;
        const int64_t s0 = b * C;
        const int32_t* bs = bstart + b * (P + 1);
        for (int I0 = 0; I0 < P; I0 += kPrepBatch) {
            int k0v[kPrepBatch], k1v[kPrepBatch];
            float4 rkv[kPrepBatch];
            float wkv[kPrepBatch];
#pragma unroll
            for (int q = 0; q < kPrepBatch; ++q) {
                const bool in = I0 + q < P;
                k0v[q] = in ? __ldg(bs + I0 + q) : 0;
                k1v[q] = in ? __ldg(bs + I0 + q + 1) : 0;
            }
#pragma unroll
            for (int q = 0; q < kPrepBatch; ++q) {
                const int kk = k0v[q] + lane;
                rkv[q] = kk < k1v[q] ? __ldg(recs + s0 + kk) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < kPrepBatch; ++q) {
                const int kk = k0v[q] + lane;
                wkv[q] = (!isw && kk < k1v[q]) ? __ldg(wbuf + s0 + rec_idx(rkv[q])) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < kPrepBatch; ++q) {
                const int I = I0 + q;
                if (I >= P) break;
                for (int e = lane; e < nrb; e += 32) work[e] = 0;
                __syncwarp();
                step(s0, isw, k0v[q] + lane, k1v[q], rkv[q], wkv[q]);
                for (int kb = k0v[q] + 32; kb < k1v[q]; kb += 32) {
                    const int kk = kb + lane;
                    const float4 rk = kk < k1v[q] ? __ldg(recs + s0 + kk) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float wk = (!isw && kk < k1v[q]) ? __ldg(wbuf + s0 + rec_idx(rk)) : 0.f;
                    step(s0, isw, kk, k1v[q], rk, wk);
                }
                __syncwarp();
                for (int e = lane; e < nrb; e += 32) p.pwork[(int64_t)(I * nrb + e) * p.nb_max + b] = work[e];
                __syncwarp();
            }
        }
    }
}

// Per-event epilogue: lambda, log, w, the W entries of the dalpha GEMM, the dbeta sum and
// per-mark sums in shared-memory histograms flushed once per block.  One sequence: event k
// lies in chunk k / C, which starts at event C (k / C).  W is transposed ([M][nbp]) and its
// row sums are taken where it is split for the GEMM.  The compensator sums
// E_j = sum_{c_l = j} (1 - exp(-beta (T - t_l))) = n_j - sum exp(-beta (T - t_l)) and
// F_j = sum (T - t_l) exp(-beta (T - t_l)) only need the events with beta (T - t) < 104
// (below that exp underflows to 0 in FP32); n_j comes from the validation's mark counts
// or, without validation, from an integer histogram here.
constexpr float kTailLimit = 104.f;

__device__ __forceinline__ int64_t chunk_of(int64_t k, int C, int64_t N) {
    return N < (int64_t(1) << 31) ? (int64_t)((uint32_t)k / (uint32_t)C) : k / C;
}

// Per-thread sums of the epilogue.
struct EpiSums {
    LogProd lp;      // reduce mode 0: running product of the intensities
    SumF32 ls;       // modes 1, 2: FP32 log-sum
    double db = 0.0; // dbeta terms: FP32 terms summed in FP64, so that the near-cancelling sum
                     // does not depend on which thread took which event
};

// Event k (chunk b, mark ck, delta = t_k - chunk start) given y = Y[b][ck], z = Z[b][ck]
// (with the gradient) and its pair sums ak, bk: the log-intensity term, the compensator tail and, with the gradient, w, the
// dbeta term and the per-mark sum of w; returns w e_k, the event's W entry (0 without the
// gradient).
template <bool GRAD>
__device__ __forceinline__ float epi_event(const Problem& p, int64_t k, int64_t b, int ck,
                                           float delta, float y, float z, float ak, float bk,
                                           float beta, double T,
                                           int mode, bool counted, EpiSums& acc, float* hEt,
                                           float* hF, float* hmu, uint32_t* hcnt, float* wbuf) {
    const float ek = exp_unbiased(-beta * delta);
    const float aS = ek * y + ak;
    const float lam = __ldg(p.mu + ck) + beta * aS;
    if (!(lam > 0.f)) set_status(p.hdr, HAWKES_ERR_NONPOS_INTENSITY);
    if (mode == 0) acc.lp.mul(lam);
    else if (mode == 1) acc.ls.add(logf(lam));
    else acc.ls.s += logf(lam);
    if (!counted) atomicAdd(&hcnt[ck], 1u);
    if (beta * (__ldg(p.Tmt + b) - delta) < kTailLimit + 1.f) {   // T - t_k, to within rounding
        const float xT = (float)tdiff(p, T, p.t[k]);
        if (beta * xT < kTailLimit) {
            const float eT = exp_unbiased(-beta * xT);
            atomicAdd(&hEt[ck], eT);
            if (GRAD) atomicAdd(&hF[ck], xT * eT);
        }
    }
    if (!GRAD) return 0.f;
    const float w = 1.f / lam;
    acc.db += (double)(w * (ek * (z - beta * delta * y) + (ak - beta * bk)));
    wbuf[k] = w;
    atomicAdd(&hmu[ck], w);
    return w * ek;
}

// The block's sums into the accumulators: the log-likelihood (atomic FP64, or the block's
// FP32 partial for k_logsum_combine), dbeta, and the per-mark histograms.
template <bool GRAD>
__device__ __forceinline__ void epi_flush(const Problem& p, EpiSums& acc, int mode, bool counted,
                                          const float* hEt, const float* hF, const float* hmu,
                                          const uint32_t* hcnt, double* red_ll, double* red_db,
                                          SumF32* red_ls) {
    const int M = p.M;
    double ll = mode == 0 ? acc.lp.log_value() : 0.0;
    double dbd = acc.db;
    SumF32& ls = acc.ls;
    for (int o = 16; o >= 1; o >>= 1) {
        ll += __shfl_xor_sync(HK_FULL, ll, o);
        dbd += __shfl_xor_sync(HK_FULL, dbd, o);
        if (mode != 0) {
            SumF32 other;
            other.s = __shfl_xor_sync(HK_FULL, ls.s, o);
            other.e = __shfl_xor_sync(HK_FULL, ls.e, o);
            if (mode == 1) ls.add(other);
            else ls.s += other.s;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        red_ll[threadIdx.x >> 5] = ll;
        red_db[threadIdx.x >> 5] = dbd;
        red_ls[threadIdx.x >> 5] = ls;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, d = 0.0;
        SumF32 bl;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red_ll[w];
            d += red_db[w];
            if (mode == 1) bl.add(red_ls[w]);
            else bl.s += red_ls[w].s;
        }
        if (mode == 0) atomicAdd(&p.ll_acc[0], a);
        else if (blockIdx.x < kLogSumBlocks) {       // combined in block order by k_logsum_combine
            p.ll_part[2 * blockIdx.x] = bl.s;
            p.ll_part[2 * blockIdx.x + 1] = mode == 1 ? bl.e : 0.f;
        }
        if (GRAD) atomicAdd(&p.dbe_acc[0], d);
    }
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const double n = counted ? (blockIdx.x == 0 ? (double)p.counts[j] : 0.0) : (double)hcnt[j];
        const double e = n - (double)hEt[j];
        if (e != 0.0) atomicAdd(&p.E_acc[j], e);
        if (GRAD) {
            if (hF[j] != 0.f) atomicAdd(&p.F_acc[j], (double)hF[j]);
            if (hmu[j] != 0.f) atomicAdd(&p.dmu_acc[j], (double)hmu[j]);
        }
    }
}

// Event by event (for marks too many for the group kernel's shared memory): Y and Z gathered
// from global memory, W (transposed, zeroed before) accumulated by global reductions.
template <bool GRAD>
__global__ void __launch_bounds__(512, 3) k_epilogue(Problem p, const float* __restrict__ Aint,
                                                     const float* __restrict__ Bint, float* wbuf) {
    extern __shared__ float sh[];
    const int M = p.M, C = p.C;
    float* hEt = sh;                          // [M] sum of exp(-beta (T - t)) (tail events)
    float* hF = hEt + M;                      // [M]
    float* hmu = hF + M;                      // [M]
    uint32_t* hcnt = (uint32_t*)(hmu + M);    // [M] events per mark (without validation)
    __shared__ double red_ll[16];
    __shared__ double red_db[16];
    __shared__ SumF32 red_ls[16];
    if (failed(p.hdr)) return;
    const int64_t N = p.N, ldw = p.nbp;
    const int mode = p.reduce;                // 0: FP64 log of running products; 1, 2: FP32 logs
    const float beta = p.beta[0];
    const double T = p.Tarr[0];
    const bool counted = p.validated != 0;
    for (int j = threadIdx.x; j < 4 * M; j += blockDim.x) sh[j] = 0.f;
    __syncthreads();
    EpiSums acc;
#pragma unroll 4
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = chunk_of(k, C, N);
        const int ck = __ldg(p.c + k);
        const float y = __ldg(p.Y + b * M + ck);
        const float z = GRAD ? __ldg(p.Z + b * M + ck) : 0.f;
        const float bk = GRAD ? __ldg(Bint + k) : 0.f;
        const float wv = epi_event<GRAD>(p, k, b, ck, __ldg(p.delta + k), y, z, __ldg(Aint + k), bk,
                                         beta, T, mode, counted, acc, hEt, hF, hmu, hcnt, wbuf);
        if (GRAD) atomicAdd(&p.W[(int64_t)ck * ldw + b], wv);
    }
    epi_flush<GRAD>(p, acc, mode, counted, hEt, hF, hmu, hcnt, red_ll, red_db, red_ls);
}

// By groups of kEpiGroup consecutive chunks: a block takes a group at a time, accumulates
// its W entries in shared memory and writes them out as one 32-byte piece per mark (W is
// transposed, [M][nbp] with nbp a multiple of kEpiGroup, so the groups cover every column and
// W needs no zeroing).  The thread that writes a mark's piece also keeps the mark's largest
// entry and, in FP64, the sum of its entries, flushed once per block (wmax, wsum_acc), so
// that the split of W for the dalpha GEMM needs one pass over it instead of two.
constexpr int kEpiGroup = 8;

template <bool GRAD>
__global__ void __launch_bounds__(512, 3) k_epilogue_groups(Problem p, const float* __restrict__ Aint,
                                                         const float* __restrict__ Bint,
                                                         float* wbuf) {
    extern __shared__ double shd[];
    const int M = p.M, C = p.C;
    double* wsum = shd;                       // [M] this block's sums of W entries (GRAD)
    float* sh = (float*)(shd + (GRAD ? M : 0));
    float* hEt = sh;                          // [M] sum of exp(-beta (T - t)) (tail events)
    float* hF = hEt + M;                      // [M]
    float* hmu = hF + M;                      // [M]
    uint32_t* hcnt = (uint32_t*)(hmu + M);    // [M] events per mark (without validation)
    uint32_t* wmx = hcnt + M;                 // [M] this block's largest W entries (GRAD)
    float* Wg = (float*)(wmx + (GRAD ? M : 0));   // [kEpiGroup][M] the group's W entries (GRAD)
    __shared__ double red_ll[16];
    __shared__ double red_db[16];
    __shared__ SumF32 red_ls[16];
    if (failed(p.hdr)) return;
    const int64_t N = p.N, nb = p.nb_max, ldw = p.nbp;
    const int64_t ngroups = (nb + kEpiGroup - 1) / kEpiGroup;
    const int mode = p.reduce;
    const float beta = p.beta[0];
    const double T = p.Tarr[0];
    const bool counted = p.validated != 0;
    const int nt = blockDim.x;
    for (int j = threadIdx.x; j < (GRAD ? 5 : 4) * M; j += nt) sh[j] = 0.f;
    if (GRAD)
        for (int j = threadIdx.x; j < M; j += nt) wsum[j] = 0.0;
    __syncthreads();
    EpiSums acc;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int64_t b0 = g * kEpiGroup;
        const int nbg = (int)(nb - b0 < kEpiGroup ? nb - b0 : kEpiGroup);
        if (GRAD) {
            __syncthreads();                  // the previous group's entries are written out
            for (int j = threadIdx.x; j < kEpiGroup * M; j += nt) Wg[j] = 0.f;
            __syncthreads();
        }
        const int64_t k0 = b0 * C;
        const int64_t k1 = (b0 + nbg) * C < N ? (b0 + nbg) * C : N;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += nt) {
            const int64_t b = chunk_of(k, C, N);
            const int ck = __ldg(p.c + k);
            const float y = __ldg(p.Y + b * M + ck);
            const float z = GRAD ? __ldg(p.Z + b * M + ck) : 0.f;
            const float bk = GRAD ? __ldg(Bint + k) : 0.f;
            const float wv = epi_event<GRAD>(p, k, b, ck, __ldg(p.delta + k), y, z, __ldg(Aint + k),
                                             bk, beta, T, mode, counted, acc, hEt, hF, hmu, hcnt,
                                             wbuf);
            if (GRAD) atomicAdd(&Wg[(int)(b - b0) * M + ck], wv);
        }
        if (GRAD) {
            __syncthreads();
            for (int m = threadIdx.x; m < M; m += nt) {
                const float4 lo = make_float4(Wg[m], Wg[M + m], Wg[2 * M + m], Wg[3 * M + m]);
                const float4 hi = make_float4(Wg[4 * M + m], Wg[5 * M + m], Wg[6 * M + m], Wg[7 * M + m]);
                float4* dst = (float4*)(p.W + (int64_t)m * ldw + b0);
                dst[0] = lo;
                dst[1] = hi;
                const float mx = fmaxf(fmaxf(fmaxf(lo.x, lo.y), fmaxf(lo.z, lo.w)),
                                       fmaxf(fmaxf(hi.x, hi.y), fmaxf(hi.z, hi.w)));
                wmx[m] = max(wmx[m], __float_as_uint(mx));     // entries are >= 0
                wsum[m] += (double)((lo.x + lo.y) + (lo.z + lo.w)) +
                           (double)((hi.x + hi.y) + (hi.z + hi.w));
            }
        }
    }
    __syncthreads();
    if (GRAD)
        for (int m = threadIdx.x; m < M; m += nt) {
            if (wmx[m]) atomicMax(&p.wmax[m], wmx[m]);
            if (wsum[m] != 0.0) atomicAdd(&p.wsum_acc[m], wsum[m]);
        }
    epi_flush<GRAD>(p, acc, mode, counted, hEt, hF, hmu, hcnt, red_ll, red_db, red_ls);
}

// Shared memory of the group epilogue, and whether it fits.
static size_t epi_group_smem(int64_t M, bool grad) {
    return sizeof(float) * (size_t)M * (4 + (grad ? 1 + kEpiGroup : 0)) +
           (grad ? sizeof(double) * (size_t)M : 0);
}
static bool epi_groups(const Problem& p) {
    return epi_group_smem(p.M, p.grad) <= 227 * 1024 - 512;
}

// The FP32 log-sums of the epilogue's blocks, in block order (mode 1 compensated, mode 2
// plain), into ll_acc[0].
__global__ void k_logsum_combine(Problem p, int blocks) {
    if (threadIdx.x != 0 || failed(p.hdr)) return;
    SumF32 s;
    for (int b = 0; b < blocks; ++b) {
        SumF32 x;
        x.s = p.ll_part[2 * b];
        x.e = p.ll_part[2 * b + 1];
        if (p.reduce == 1) s.add(x);
        else s.s += x.s;
    }
    p.ll_acc[0] = (double)(p.reduce == 1 ? s.s + s.e : s.s);
}

// Blocks of the epilogue kernels: three per SM (512 threads, each ~20 events at N = 1e7).
int epilogue_blocks(int64_t N) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (int64_t)sms * 3;
    const int64_t need = (N + 511) / 512;
    if (need < blocks) blocks = need;
    return (int)(blocks > 0 ? blocks : 1);
}

// Bucketing of chunks [b_begin, b_end) (clipped to the chunks of the call); it needs only
// the chunks' offsets from the scan's reduce pass and their marks.
cudaError_t launch_bucket_range(const Problem& p, cudaStream_t s, int64_t b_begin, int64_t b_end,
                                int* nl) {
    cudaError_t err;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int P = p.P;
    if (b_end > p.nb_max) b_end = p.nb_max;
    int warps = 8;
    while (warps > 1 && bucket_smem_bytes(P, p.C, p.M, warps) > 227 * 1024) --warps;
    const size_t smem = bucket_smem_bytes(P, p.C, p.M, warps);
    if (smem > 48 * 1024) {
        err = cudaFuncSetAttribute(k_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    int64_t grid = (b_end - b_begin + warps - 1) / warps;
    if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
    k_bucket<<<(unsigned)(grid > 0 ? grid : 1), 32 * warps, smem, s>>>(p, p.recs, p.src, p.bstart,
                                                                    p.wide, b_begin, b_end);
    ++*nl;
    prof_mark(s, "bucket");
    return cudaGetLastError();
}

// Everything of the chunk-GEMM path before the per-event epilogue: operand centres and
// splits, Y and Z on the tensor cores, bucketing (unless done piece by piece) and the
// forward pairs.
cudaError_t launch_gemm_forward(const Problem& p, cudaStream_t s, int* nl) {
    cudaError_t err;
    const int64_t M = p.M, nb = p.nb_max;
    // Y = S^ alpha^T and Z = (S^ - beta G^) alpha^T on the tensor cores (rows = chunks)
    cudaMemsetAsync(p.wsum_acc, 0, sizeof(double) * (size_t)M, s);
    int* acc_n = (int*)(p.cen_acc + 2 * (size_t)kCentreSlices * M);
    k_col_sums<<<dim3((unsigned)((M + 255) / 256), kCentreSlices), 256, 0, s>>>(p, p.grad,
                                                                              p.cen_acc, acc_n);
    k_centre_means<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(p, p.grad, p.cen_acc, acc_n);
    k_centres<<<(unsigned)((M + 7) / 8), 256, 0, s>>>(p, p.grad);
    *nl += 3;
    prof_mark(s, "centres");
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int64_t* nb_dev = p.chunk_base + p.B;   // number of chunks, on the device
    if ((err = split_f16_rows(p.alpha, M, p.al_p, p.ldk, M, M, s, nullptr, nullptr,
                              p.isc_al, nullptr, nullptr)) != cudaSuccess)
        return err;
    ++*nl;
    prof_mark(s, "split_alpha");
    // S^ - m for Y and, with the gradient, S^ - beta G^ for Z (see below) in one pass over S^
    if (p.grad) {
        // (and the column maxima of S^ - m for the transposed split of the dalpha GEMM)
        if ((err = split_f16_rows_pair(p.Shat, p.Ghat, M, p.cen_S, p.cen_Z, p.beta, p.S_p,
                                       p.isc_S, p.G_p, p.isc_G, p.ldk, nb, M, nb_dev, p.colmax,
                                       s)) !=
            cudaSuccess)
            return err;
        ++*nl;
        prof_mark(s, "split_S_G");
    } else {
        if ((err = split_f16_rows(p.Shat, M, p.S_p, p.ldk, nb, M, s, p.cen_S, nb_dev,
                                  p.isc_S, nullptr, nullptr)) != cudaSuccess)
            return err;
        ++*nl;
        prof_mark(s, "split_S");
    }
    if ((err = tc_gemm_f16x3(p.S_p, p.ldk, p.al_p, p.ldk, p.Y, M, (int)nb,
                             (int)M, M, 1, false, p.hdr, s, p.bias_Y, p.isc_S, p.isc_al)) !=
        cudaSuccess)
        return err;
    ++*nl;
    prof_mark(s, "gemm_Y");
    if (p.grad) {
        // Z = (S^ - beta G^) alpha^T: the decay-gradient term of an event is
        // e (Z - beta delta Y) + (A - beta B), so the near-cancelling difference of the
        // forward state and its beta-derivative is formed once per chunk and element from
        // the scan's states (split above), before any rounding of the tensor-core product
        if ((err = tc_gemm_f16x3(p.G_p, p.ldk, p.al_p, p.ldk, p.Z, M, (int)nb,
                                 (int)M, M, 1, false, p.hdr, s, p.bias_Z, p.isc_G, p.isc_al)) !=
            cudaSuccess)
            return err;
        ++*nl;
        prof_mark(s, "gemm_Z");
    }
    // the events of every chunk bucketed by mark block (unless done piece by piece), then
    // the forward pairs
    if (!p.bucket_done) {
        err = launch_bucket_range(p, s, 0, nb, nl);
        if (err != cudaSuccess) return err;
    }
    return launch_pairs_forward(p, s, nl);
}

// The per-event epilogue of one kernel.
cudaError_t launch_gemm_epilogue(const Problem& p, cudaStream_t s, int* nl) {
    cudaError_t err;
    const int64_t M = p.M;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool groups = epi_groups(p);
    int blocks;
    if (groups) {
        if (p.grad && p.w_rowstats) cudaMemsetAsync(p.wmax, 0, sizeof(uint32_t) * (size_t)M, s);
        const size_t smem = epi_group_smem(M, p.grad);
        auto kern = p.grad ? k_epilogue_groups<true> : k_epilogue_groups<false>;
        if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem)) != cudaSuccess)
            return err;
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem);
        const int64_t ngroups = (p.nb_max + kEpiGroup - 1) / kEpiGroup;
        int64_t b = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
        if (b > ngroups) b = ngroups;
        if (p.reduce != 0 && b > kLogSumBlocks) b = kLogSumBlocks;
        blocks = (int)(b > 0 ? b : 1);
        kern<<<(unsigned)blocks, 512, smem, s>>>(p, p.Aint, p.Bint, p.wbuf);
    } else {
        if (p.grad) cudaMemsetAsync(p.W, 0, sizeof(float) * (size_t)M * (size_t)p.nbp, s);
        const size_t smem = sizeof(float) * 4 * (size_t)M;
        auto kern = p.grad ? k_epilogue<true> : k_epilogue<false>;
        if (smem > 48 * 1024) {
            err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
        }
        blocks = epilogue_blocks(p.N);
        if (p.reduce != 0 && blocks > kLogSumBlocks) blocks = kLogSumBlocks;
        kern<<<(unsigned)blocks, 512, smem, s>>>(p, p.Aint, p.Bint, p.wbuf);
    }
    ++*nl;
    if (p.reduce != 0) {
        k_logsum_combine<<<1, 32, 0, s>>>(p, blocks);
        ++*nl;
    }
    prof_mark(s, "epilogue");
    return cudaGetLastError();
}

// Everything after the epilogue: row groups and backward pairs, the dalpha GEMM and the
// finalisation (mode 1).
cudaError_t launch_gemm_backward(const Problem& p, cudaStream_t s, int* nl) {
    cudaError_t err;
    const int64_t M = p.M, nb = p.nb_max;
    const int64_t* nb_dev = p.chunk_base + p.B;   // number of chunks, on the device
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int P = p.P;
    if (p.grad) {
        int64_t blocks = (nb + 7) / 8;
        if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
        k_bwd_prep<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(p, p.recs, p.bstart, p.wide,
                                                                        p.wbuf, p.kprep);
        ++*nl;
        prof_mark(s, "bwd_prep");
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (p.grad) {
        err = launch_pairs_backward(p, s, nl);
        if (err != cudaSuccess) return err;
    }
    if (p.grad) {
        // dalpha_gemm[i][j] = sum_b W[b][i] S^[b][j] with the chunk index as the contiguous
        // K dimension: W is already transposed (columns past the chunk count are 0), S^ is
        // transposed here
        // (row maxima and sums from the group epilogue when it took them: one pass over W)
        if ((err = split_f16_long_rows(p.W, p.nbp, p.Wt_p, p.ldt, M, p.nbp, s, p.isc_Wt,
                                       p.w_rowstats ? nullptr : p.wsum_acc,
                                       p.w_rowstats ? p.wmax : nullptr)) != cudaSuccess)
            return err;
        ++*nl;
        prof_mark(s, "split_W");
        if ((err = transpose_split_f16(p.Shat, M, nb_dev, p.nbp, p.St_p, p.ldt, s,
                                       p.cen_S, p.colmax, p.isc_St, true)) != cudaSuccess)
            return err;
        ++*nl;
        prof_mark(s, "transpose_S");
        cudaMemsetAsync(p.dal_gemm, 0, sizeof(float) * (size_t)M * M, s);
        // split K so that the blocks (one per SM) fill whole waves: minimise
        // waves x (k-tiles per block + the cost of its atomic output, ~4 k-tiles)
        const int64_t tiles = ((M + 127) / 128) * ((M + 255) / 256);
        const int64_t ktiles = (p.nbp + 63) / 64;
        int splits = 1;
        int64_t best = -1;
        for (int64_t sp = 1; sp <= 64 && sp <= ktiles; ++sp) {
            const int64_t waves = (tiles * sp + sms - 1) / sms;
            const int64_t cost = waves * ((ktiles + sp - 1) / sp + 4);
            if (best < 0 || cost < best) { best = cost; splits = (int)sp; }
        }
        if ((err = tc_gemm_f16x3(p.Wt_p, p.ldt, p.St_p, p.ldt, p.dal_gemm, M,
                                 (int)M, (int)M, p.nbp, splits, true, p.hdr, s, nullptr,
                                 p.isc_Wt, p.isc_St)) != cudaSuccess)
            return err;
        ++*nl;
        prof_mark(s, "gemm_dalpha");
    }
    return launch_finalize_mode(p, s, 1, nl);
}

// ---------------------------------------------------------------------------
// Several decay kernels (paper, Eq. hawkes_excitation with its sum over kernels q):
//     lambda_k = mu_{c_k} + sum_q beta_q (e^(q)_k Y^(q)_b[c_k] + A^(q)_k),
// every kernel's Y, Z, A, B coming from its own workspace slice.  With w_k = 1 / lambda_k
// shared by the kernels, each kernel q gets its own W rows (w_k e^(q)_k), decay-gradient
// sum w_k (e^(q)_k (Z^(q)_b[c_k] - beta_q delta_k Y^(q)_b[c_k]) + A^(q)_k - beta_q B^(q)_k)
// and compensator sums, in its own slice, so that the
// slice's backward part and finalisation then produce dalpha^(q) and dbeta_q; the
// log-sum and dmu go to slice 0.
// ---------------------------------------------------------------------------
template <bool GRAD>
__global__ void __launch_bounds__(512) k_epilogue_multi(Problem p, MultiSlices ms, float* wbuf) {
    extern __shared__ float sh[];
    const int M = p.M, K = ms.K, C = p.C;
    float* hEt = sh;                           // [K][M]
    float* hF = hEt + K * M;                   // [K][M]
    float* hmu = hF + K * M;                   // [M]
    uint32_t* hcnt = (uint32_t*)(hmu + M);     // [M]
    __shared__ double red_ll[16];
    __shared__ double red_db[kMaxKernels][16];
    for (int q = 0; q < K; ++q)
        if (failed(ms.k[q].hdr)) return;
    const int64_t N = p.N, ldw = p.nbp;
    const bool counted = p.validated != 0;
    float beta[kMaxKernels], bmin = 0.f;      // the smallest decay has the longest tail
#pragma unroll
    for (int q = 0; q < kMaxKernels; ++q) {
        beta[q] = q < K ? ms.k[q].beta[0] : 0.f;
        if (q < K) bmin = q == 0 ? beta[q] : fminf(bmin, beta[q]);
    }
    const double T = p.Tarr[0];
    for (int j = threadIdx.x; j < (2 * K + 2) * M; j += blockDim.x) sh[j] = 0.f;
    __syncthreads();
    LogProd lp;
    double db[kMaxKernels] = {0.0, 0.0, 0.0, 0.0};   // FP32 terms summed in FP64
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = chunk_of(k, C, N);
        const int ck = p.c[k];
        const float delta = p.delta[k];
        float e[kMaxKernels], y[kMaxKernels];
        float exc = 0.f;
#pragma unroll
        for (int q = 0; q < kMaxKernels; ++q) {
            if (q < K) {
                e[q] = exp_unbiased(-beta[q] * delta);
                y[q] = ms.k[q].Y[b * M + ck];
                exc += beta[q] * (e[q] * y[q] + ms.k[q].A[k]);
            }
        }
        const float lam = p.mu[ck] + exc;
        if (!(lam > 0.f)) set_status(p.hdr, HAWKES_ERR_NONPOS_INTENSITY);
        lp.mul(lam);
        if (!counted) atomicAdd(&hcnt[ck], 1u);
        if (bmin * (p.Tmt[b] - delta) < kTailLimit + 1.f) {       // T - t_k, to within rounding
            const float xT = (float)(T - p.t[k]);
#pragma unroll
            for (int q = 0; q < kMaxKernels; ++q) {
                if (q < K && beta[q] * xT < kTailLimit) {
                    const float eT = exp_unbiased(-beta[q] * xT);
                    atomicAdd(&hEt[q * M + ck], eT);
                    if (GRAD) atomicAdd(&hF[q * M + ck], xT * eT);
                }
            }
        }
        if (GRAD) {
            const float w = 1.f / lam;
            wbuf[k] = w;
            atomicAdd(&hmu[ck], w);
#pragma unroll
            for (int q = 0; q < kMaxKernels; ++q) {
                if (q < K) {
                    const float x = ms.k[q].Z[b * M + ck];
                    db[q] += (double)(w * (e[q] * (x - beta[q] * delta * y[q]) +
                                           (ms.k[q].A[k] - beta[q] * ms.k[q].B[k])));
                    atomicAdd(&ms.k[q].W[(int64_t)ck * ldw + b], w * e[q]);
                }
            }
        }
    }
    double ll = lp.log_value();
    double dbd[kMaxKernels];
#pragma unroll
    for (int q = 0; q < kMaxKernels; ++q) dbd[q] = db[q];
    for (int o = 16; o >= 1; o >>= 1) {
        ll += __shfl_xor_sync(HK_FULL, ll, o);
#pragma unroll
        for (int q = 0; q < kMaxKernels; ++q) dbd[q] += __shfl_xor_sync(HK_FULL, dbd[q], o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_ll[threadIdx.x >> 5] = ll;
#pragma unroll
        for (int q = 0; q < kMaxKernels; ++q) red_db[q][threadIdx.x >> 5] = dbd[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red_ll[w];
        atomicAdd(&p.ll_acc[0], a);
        if (GRAD)
            for (int q = 0; q < K; ++q) {
                double d = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) d += red_db[q][w];
                atomicAdd(&ms.k[q].dbe_acc[0], d);
            }
    }
    for (int e = threadIdx.x; e < K * M; e += blockDim.x) {
        const int q = e / M, j = e % M;
        const double n = counted ? (blockIdx.x == 0 ? (double)p.counts[j] : 0.0) : (double)hcnt[j];
        const double ev = n - (double)hEt[e];
        if (ev != 0.0) atomicAdd(&ms.k[q].E_acc[j], ev);
        if (GRAD && hF[e] != 0.f) atomicAdd(&ms.k[q].F_acc[j], (double)hF[e]);
    }
    if (GRAD)
        for (int j = threadIdx.x; j < M; j += blockDim.x)
            if (hmu[j] != 0.f) atomicAdd(&p.dmu_acc[j], (double)hmu[j]);
}

cudaError_t launch_epilogue_multi(const Problem& p, const MultiSlices& ms, cudaStream_t s, int* nl) {
    const int64_t M = p.M;
    if (p.grad)
        for (int q = 0; q < ms.K; ++q)
            cudaMemsetAsync(ms.k[q].W, 0, sizeof(float) * (size_t)M * (size_t)p.nbp, s);
    const size_t smem = sizeof(float) * (2 * (size_t)ms.K + 2) * (size_t)M;
    auto kern = p.grad ? k_epilogue_multi<true> : k_epilogue_multi<false>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)epilogue_blocks(p.N), 512, smem, s>>>(p, ms, p.wbuf);
    ++*nl;
    prof_mark(s, "epilogue");
    return cudaGetLastError();
}

cudaError_t launch_gemm_path(const Problem& p0, cudaStream_t s, int* nl) {
    Problem p = p0;
    p.w_rowstats = p.grad && epi_groups(p) ? 1 : 0;
    cudaError_t err = launch_gemm_forward(p, s, nl);
    if (err == cudaSuccess) err = launch_gemm_epilogue(p, s, nl);
    if (err == cudaSuccess) err = launch_gemm_backward(p, s, nl);
    return err;
}

}  // namespace hk
