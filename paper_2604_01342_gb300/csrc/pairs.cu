// Intra-chunk pairs of the chunk-GEMM path.
//
// Inside a chunk every event k receives the excitation of the earlier events l of the same
// chunk directly (paper, Eq. hawkes_excitation restricted to the pairs of one chunk):
//     A_k = sum_{l<k} P_kl alpha[c_k][c_l],   B_k = sum_{l<k} (t_k - t_l) P_kl alpha[c_k][c_l],
// with P_kl = exp(-beta (t_k - t_l)) = em_k ep_l, and the backward pass adds
//     dalpha_pairs[c_k][c_l] += w_k P_kl        (w_k = 1 / lambda_k; Appendix B, Eq. grad_alpha).
// Gathering alpha[c_k][c_l] from L2 would cost a 32-byte sector per pair, so both passes
// keep part of alpha (forward) or of dalpha_pairs (backward) in shared memory.
//
// Forward: square tiles (I, J) of alpha, 128 x 128, one at a time per block; the lanes hold
// the targets of bucket I and the sources of bucket J are broadcast to them (k_pairs_fwd).
//
// Backward, by row block: R target marks (marks I + P pos, pos in [q R, q R + R) of mark
// block I) with all M source marks, an R x M tile of dalpha_pairs that one block of threads
// keeps for a whole run of chunks.  In a chunk the targets of a row block are a contiguous
// run of bucket I (sorted by (position, index)); a warp takes them one at a time, and with
// the row groups of k_bwd_prep target k owes U_k ep_l only for the sources l between the
// previous target of its mark and k, which its lanes take 32 at a time in index order (the
// source records read coalesced, every add of one step in one row, at the sources' marks).
// The blocks' work is balanced by a plan (k_pair_plan): the work of every (row block,
// chunk) - the 32-source steps of its targets plus one per target, counted by k_bwd_prep -
// is summed over the chunks; every row block gets a number of thread blocks in proportion to
// its total and each of them takes the run of chunks holding its share.
#include "common.cuh"

namespace hk {

constexpr int kPairRowThreads = 1024;
constexpr int kBwdStage = 256;          // sources of one chunk staged per warp (at most)

// Inclusive scan over the block (1024 threads) of one int64 value per thread; *total gets
// the block's sum.  Uses the 33 words of `sh`.
__device__ __forceinline__ int64_t block_scan_i64(int64_t v, int64_t* sh, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(HK_FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(HK_FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;
        if (lane == 31) sh[32] = w;
    }
    __syncthreads();
    const int64_t r = x + (wid > 0 ? sh[wid - 1] : 0);
    *total = sh[32];
    __syncthreads();
    return r;
}

// One block per row block: the prefix of its work over the chunks (pcum) and its total;
// the last block to finish then lays out the plan: nr_rb = ceil(total_rb B / W) blocks for a
// row block with work (at least one, at most one per chunk; B chosen so that they add up to
// at most nb_target), their first block, and for every block x its (row block, share) as
// rb << 16 | k.
__global__ void __launch_bounds__(kPairRowThreads) k_pair_plan(Problem p, int32_t* plan,
                                                               int nb_target, unsigned* ticket) {
    __shared__ int64_t sh[33];
    __shared__ int last_sh;
    if (failed(p.hdr)) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n_rb = p.n_rb;
    const int64_t nbc = num_chunks(p);
    const int64_t ldc = p.nb_max + 1;
    {
        // each warp scans a contiguous segment of the chunks, 32 at a time (coalesced reads):
        // its segment's sum, the warps' prefix over the block, then the segment's prefixes
        const int rb = blockIdx.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
        const int32_t* w = p.pwork + (int64_t)rb * p.nb_max;
        int64_t* cum = p.pcum + (int64_t)rb * ldc;
        const int64_t per = ((nbc + nw - 1) / nw + 31) / 32 * 32;
        const int64_t b0 = min((int64_t)wid * per, nbc), b1 = min(b0 + per, nbc);
        int64_t run = 0;
        for (int64_t b = b0 + lane; b < b1; b += 32) run += w[b];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) run += __shfl_xor_sync(HK_FULL, run, o);
        int64_t total;
        const int64_t incl = block_scan_i64(lane == 0 ? run : 0, sh, &total);
        int64_t at = __shfl_sync(HK_FULL, incl, 0) - run;     // before this warp's segment
        for (int64_t b = b0; b < b1; b += 32) {
            const int64_t x = b + lane < b1 ? w[b + lane] : 0;
            int64_t y = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t z = __shfl_up_sync(HK_FULL, y, o);
                if (lane >= o) y += z;
            }
            if (b + lane < b1) cum[b + lane] = at + y - x;
            at += __shfl_sync(HK_FULL, y, 31);
        }
        if (tid == 0) {
            cum[nbc] = total;
            p.ptot[rb] = total;
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last_sh = atomicAdd(ticket, 1u) == (unsigned)(n_rb - 1);
    __syncthreads();
    if (!last_sh) return;
    __threadfence();
    int64_t part = 0;
    for (int r = tid; r < n_rb; r += nt) part += __ldcg(p.ptot + r);
    int64_t W;
    block_scan_i64(part, sh, &W);
    // blocks of a row block with work: ceil(t B / W) for the largest B <= nb_target whose
    // blocks add up to at most nb_target (each ceil adds less than one, so B lies within
    // n_rb below nb_target), so that the blocks fill whole waves
    auto blocks_of = [&](int64_t t, int64_t B) -> int64_t {
        if (t <= 0 || W <= 0) return 0;
        int64_t nr = (t * B + W - 1) / W;
        if (nr > nbc) nr = nbc;
        return nr < 1 ? 1 : nr;
    };
    int64_t lo = nb_target - n_rb > 1 ? nb_target - n_rb : 1, hi = nb_target;
    while (lo < hi) {                       // the largest B in [lo, hi] that fits (lo always does)
        const int64_t mid = (lo + hi + 1) / 2;
        int64_t cnt = 0;
        for (int r = tid; r < n_rb; r += nt) cnt += blocks_of(__ldcg(p.ptot + r), mid);
        int64_t sum;
        block_scan_i64(cnt, sh, &sum);
        if (sum <= nb_target) lo = mid;
        else hi = mid - 1;
    }
    const int64_t Bsel = lo;
    int64_t carry = 0;
    for (int r0 = 0; r0 < n_rb; r0 += nt) {
        const int r = r0 + tid;
        const int64_t nr = r < n_rb ? blocks_of(__ldcg(p.ptot + r), Bsel) : 0;
        int64_t sum;
        const int64_t incl = block_scan_i64(nr, sh, &sum);
        const int64_t base = carry + incl - nr;
        if (r < n_rb) {
            plan[1 + r] = (int32_t)nr;
            plan[1 + n_rb + r] = (int32_t)base;
            for (int k = 0; k < (int)nr; ++k) plan[1 + 2 * n_rb + base + k] = (r << 16) | k;
        }
        carry += sum;
    }
    if (tid == 0) plan[0] = (int32_t)carry;
}

// First chunk b in [0, nbc] with cum[b] nr >= k tot (b = nbc always qualifies): a 32-way
// search by one warp, every lane probing one point per round.
__device__ int64_t pair_range_start(const int64_t* cum, int64_t nbc, int64_t tot, int nr, int k) {
    const int lane = threadIdx.x & 31;
    const int64_t want = (int64_t)k * tot;
    int64_t lo = -1, hi = nbc;          // the answer lies in (lo, hi]
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        int64_t b = lo + step * (lane + 1);
        if (b > hi) b = hi;
        const bool ok = b == hi || __ldcg(cum + b) * nr >= want;
        const unsigned m = __ballot_sync(HK_FULL, ok);   // lane 31 probes hi: never 0
        const int f = __ffs(m) - 1;
        const int64_t nhi = min(lo + step * (f + 1), hi);
        if (f > 0) lo = lo + step * f;
        hi = nhi;
    }
    return hi;
}

// This block's row block, share and run of chunks [c0, c1); false if the plan has no work
// for it.
struct PairBlock {
    int rb, k, I, r0, rows;
    int64_t c0, c1;
};
__device__ __forceinline__ bool pair_block(const Problem& p, const int32_t* plan, PairBlock& pb,
                                           int64_t* range_sh) {
    const int x = blockIdx.x;
    if (x >= plan[0]) return false;
    const int n_rb = p.n_rb;
    const int code = plan[1 + 2 * n_rb + x];
    pb.rb = code >> 16;
    pb.k = code & 0xffff;
    pb.I = pb.rb / p.nrb;
    pb.r0 = (pb.rb - pb.I * p.nrb) << p.lgR;
    const int TR = (p.M + p.P - 1) / p.P;
    pb.rows = min(1 << p.lgR, TR - pb.r0);
    if ((threadIdx.x >> 5) == 0) {
        const int nr = plan[1 + pb.rb];
        const int64_t nbc = num_chunks(p);
        const int64_t* cum = p.pcum + (int64_t)pb.rb * (p.nb_max + 1);
        const int64_t tot = __ldcg(cum + nbc);
        const int64_t c0 = pair_range_start(cum, nbc, tot, nr, pb.k);
        const int64_t c1 = pair_range_start(cum, nbc, tot, nr, pb.k + 1);
        if ((threadIdx.x & 31) == 0) {
            range_sh[0] = c0;
            range_sh[1] = c1;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Forward pairs, through square tiles of alpha: tile (I, J) holds alpha[I + P i][J + P j]
// for i, j < 128, and a work item (row block I, kFwdChunksPerItem chunks) pairs, for every
// column block J in turn, the chunk's bucket-I events (one per lane) with its bucket-J
// events (staged in shared memory, broadcast to the lanes).
// ---------------------------------------------------------------------------
constexpr int kTile = 128;
constexpr int kTileLd = kTile + 1;      // padded row stride against bank conflicts
constexpr int kFwdChunksPerItem = 256;
constexpr int kStage = 64;              // source records staged per warp at a time

// a source record as the pair loops read it: (delta, ep, column, index)
__device__ __forceinline__ float4 unpack_rec(float4 r) {
    return make_float4(r.x, r.z, __int_as_float(rec_pos(r)), __int_as_float(rec_idx(r)));
}

// alpha in tile-major order, arranged for conflict-free staging into shared memory:
// float4 number e = rr * 128 + q of tile (I, J) holds column q of rows rr, rr + 32, rr + 64,
// rr + 96, that is at[(((I * P + J) * 4096 + e) * 4 + s] = alpha[I + P (rr + 32 s)][J + P q]
// (zero outside the matrix).
__global__ void k_alpha_tiles(Problem p, float* at) {
    const int M = p.M, P = p.P;
    const int64_t total = (int64_t)P * P * kTile * kTile;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(e & 3);
        const int f = (int)((e >> 2) % (kTile * kTile / 4));
        const int tile = (int)(e / ((int64_t)kTile * kTile));
        const int rr = f >> 7, q = f & 127;
        const int I = tile / P, J = tile % P;
        const int i = I + P * (rr + 32 * s), j = J + P * q;
        at[e] = (i < M && j < M) ? p.alpha[(int64_t)i * M + j] : 0.f;
    }
}

// Forward pairs: for every event k,
//   A_k = sum_{l<k in chunk} P_kl alpha[c_k][c_l],  B_k = sum (t_k - t_l) P_kl alpha[c_k][c_l].
// With P_kl = em_k ep_l the lane of k sums a = sum ep_l alpha and d = sum delta_l ep_l alpha
// and returns A_k = em_k a, B_k = em_k (delta_k a - d).  One thread owns A_k and B_k for all
// column blocks J, so its updates for J > 0 (reductions without a returned value, issued
// in J order) keep a fixed summation order.
constexpr int kPairThreads = 512;
constexpr int kPairWarps = kPairThreads / 32;

// Stage tile (I, J) of alpha (laid out by k_alpha_tiles) into rows of kTileLd floats.
__device__ __forceinline__ void load_alpha_tile(float* tile, const float* __restrict__ at, int tile_id) {
    const float4* src = (const float4*)(at + (int64_t)tile_id * kTile * kTile);
    for (int e = threadIdx.x; e < kTile * kTile / 4; e += blockDim.x) {
        const float4 v = __ldg(src + e);
        float* d = tile + (e >> 7) * kTileLd + (e & 127);
        d[0] = v.x;
        d[32 * kTileLd] = v.y;
        d[64 * kTileLd] = v.z;
        d[96 * kTileLd] = v.w;
    }
}

__global__ void __launch_bounds__(kPairThreads, 2) k_pairs_fwd(Problem p, const float4* __restrict__ recs,
                                                   const int32_t* __restrict__ bstart,
                                                   const uint8_t* __restrict__ wide,
                                                   const float* __restrict__ at, float* Aout,
                                                   float* Bout, int* counter) {
    extern __shared__ float tile[];       // [kTile][kTileLd], then per-warp staging
    __shared__ int item_sh;
    if (failed(p.hdr)) return;
    const int P = p.P;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    float4* stage = (float4*)(tile + kTile * kTileLd) + warp * kStage;
    const int nb = (int)num_chunks(p);
    const int nranges = (nb + kFwdChunksPerItem - 1) / kFwdChunksPerItem;
    const int nitems = nranges * P;
    const float beta = p.beta[0];
    const int C = p.C;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item_sh = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_sh;
        if (item >= nitems) break;
        const int I = item % P, range = item / P;
        const int b0 = range * kFwdChunksPerItem;
        const int b1 = min(b0 + kFwdChunksPerItem, nb);
        for (int J = 0; J < P; ++J) {
            __syncthreads();
            load_alpha_tile(tile, at, I * P + J);
            __syncthreads();
            for (int b = b0 + warp; b < b1; b += nwarps) {
                const int64_t s0 = (int64_t)b * C;
                const int32_t* bs = bstart + (int64_t)b * (P + 1);
                const int k0 = bs[I], k1 = bs[I + 1];
                const int l0 = bs[J], nJ = bs[J + 1] - l0;
                const bool isw = wide[b] != 0;
                for (int kb = k0; kb < k1; kb += 32) {
                    const int kk = kb + lane;
                    const bool have = kk < k1;
                    const float4 rk = have ? recs[s0 + kk] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const int ik = have ? rec_idx(rk) : -1;
                    const float* trow = tile + rec_pos(rk) * kTileLd;
                    float a = 0.f, d = 0.f;
                    for (int lb = 0; lb < nJ; lb += kStage) {
                        const int ns = min(kStage, nJ - lb);
                        __syncwarp();
                        for (int q = lane; q < ns; q += 32)
                            stage[q] = unpack_rec(__ldg(recs + s0 + l0 + lb + q));
                        __syncwarp();
                        if (!isw) {
                            float a2 = 0.f, d2 = 0.f;
                            int l = 0;
#pragma unroll 2
                            for (; l + 1 < ns; l += 2) {
                                const float4 r0 = stage[l], r1 = stage[l + 1];
                                const float v0 = r0.y * trow[__float_as_int(r0.z)];
                                const float v1 = r1.y * trow[__float_as_int(r1.z)];
                                if (__float_as_int(r0.w) < ik) { a += v0; d = fmaf(r0.x, v0, d); }
                                if (__float_as_int(r1.w) < ik) { a2 += v1; d2 = fmaf(r1.x, v1, d2); }
                            }
                            if (l < ns) {
                                const float4 r0 = stage[l];
                                const float v0 = r0.y * trow[__float_as_int(r0.z)];
                                if (__float_as_int(r0.w) < ik) { a += v0; d = fmaf(r0.x, v0, d); }
                            }
                            a += a2;
                            d += d2;
                        } else {
                            for (int l = 0; l < ns; ++l) {
                                const float4 rl = stage[l];
                                if (__float_as_int(rl.w) < ik) {
                                    const float v = expf(-beta * (rk.x - rl.x)) * trow[__float_as_int(rl.z)];
                                    a += v;
                                    d = fmaf(rl.x, v, d);
                                }
                            }
                        }
                    }
                    if (have) {
                        const float em = isw ? 1.f : rk.y;
                        const float A = em * a, B = em * fmaf(rk.x, a, -d);
                        const int64_t k = s0 + ik;
                        if (J == 0) { Aout[k] = A; Bout[k] = B; }
                        else { atomicAdd(Aout + k, A); atomicAdd(Bout + k, B); }
                    }
                }
            }
        }
    }
}

// Backward pairs into a row block's R x M tile of dalpha_pairs.
// FIXED: the tile holds unsigned fixed-point numbers (value x 2^s, rounded to nearest) and
// every add is a native 32-bit shared-memory atomic (an FP32 shared-memory atomic is a load
// and a compare-and-swap on this part, a third of the rate).  Every add is at most 32 w_max
// (w_max = the largest 1 / lambda_k: U_k ep_l <= sum of w over the row group; in a wide chunk
// w_k P_kl <= w_max), and s puts 64 such adds below 2^32 (s from k_pair_scale); an add that
// would wrap is detected from the atomic's returned value and marks the block, which the
// FP32 variant (FIXED = false, marked blocks only) then recomputes.
__device__ __forceinline__ void pair_add(float* t, int at, float v, bool&) { atomicAdd(t + at, v); }
__device__ __forceinline__ void pair_add(uint32_t* t, int at, float v, bool& wrap) {
    const uint32_t x = __float2uint_rn(v);
    const uint32_t old = atomicAdd(t + at, x);
    wrap |= old > 0xffffffffu - x;
}

template <bool FIXED>
__global__ void __launch_bounds__(kPairRowThreads, 1) k_pairs_bwd_rows(Problem p,
                                                                       const float4* __restrict__ recs,
                                                                       const float2* __restrict__ src,
                                                                       const int4* __restrict__ kprep,
                                                                       const float* __restrict__ wbuf,
                                                                       int* redo) {
    using TileT = typename std::conditional<FIXED, uint32_t, float>::type;
    extern __shared__ float sm_rows[];
    TileT* tile = (TileT*)sm_rows;          // [rows][M]
    __shared__ int64_t range_sh[2];
    __shared__ unsigned long long next_sh;
    __shared__ int wrap_sh;
    if (failed(p.hdr)) return;
    const int x = blockIdx.x;
    if (x < p.plan_b[0] && (FIXED ? redo[x] != 0 : !redo[x])) return;   // the other variant's
    PairBlock pb;
    if (!pair_block(p, p.plan_b, pb, range_sh)) return;
    const int M = p.M, C = p.C, n_rb = p.n_rb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // 2^s of the fixed-point tile, from the exponent k_pair_scale left in the header
    const int sexp = FIXED ? (int)p.hdr->pad[10] : 0;
    const float scale = FIXED ? ldexpf(1.f, sexp) : 1.f;
    const int ntile = pb.rows * M;
    float2* stage = (float2*)(sm_rows + ((ntile + 3) & ~3)) + warp * kBwdStage;   // this warp's sources
    for (int e = threadIdx.x; e < ntile; e += blockDim.x) tile[e] = (TileT)0;
    if (threadIdx.x == 0) {
        wrap_sh = 0;
        next_sh = range_sh[0];
    }
    __syncthreads();
    const int64_t c1 = range_sh[1];
    const float beta = p.beta[0];
    bool wrap = false;
    for (;;) {
        // the block's warps take its chunks one at a time
        int64_t b = 0;
        if (lane == 0) b = (int64_t)atomicAdd(&next_sh, 1ull);
        b = __shfl_sync(HK_FULL, b, 0);
        if (b >= c1) break;
        const int64_t s0 = b * C;
        const int32_t* bs = p.bsub + b * (n_rb + 1);
        const int ka = bs[pb.rb], kb = bs[pb.rb + 1];
        if (ka >= kb) continue;
        const float2* sc = src + s0;
        if (!p.wide[b]) {
            for (int t0 = ka; t0 < kb; t0 += 32) {
                // up to 32 targets on the lanes: (position, U_k, index, previous index)
                const int nt = min(32, kb - t0);
                const int4 kl = lane < nt ? __ldg(kprep + s0 + t0 + lane) : make_int4(0, 0, 0, 0);
                const int lmax = __reduce_max_sync(HK_FULL, kl.z);
                const bool staged = lmax <= kBwdStage;
                if (staged) {
                    for (int l = lane; l < lmax; l += 32) stage[l] = __ldg(sc + l);
                    __syncwarp();
                }
                for (int t = 0; t < nt; ++t) {
                    const int ro = (__shfl_sync(HK_FULL, kl.x, t) - pb.r0) * M;
                    const float U = __int_as_float(__shfl_sync(HK_FULL, kl.y, t)) * scale;
                    const int hi = __shfl_sync(HK_FULL, kl.z, t);
                    const int lo = __shfl_sync(HK_FULL, kl.w, t);
                    const int l0 = (lo > 0 ? lo : 0) + lane;
                    if (staged) {
#pragma unroll 2
                        for (int l = l0; l < hi; l += 32) {
                            const float2 sl = stage[l];
                            pair_add(tile, ro + __float_as_int(sl.y), U * sl.x, wrap);
                        }
                    } else {
                        for (int l = l0; l < hi; l += 32) {
                            const float2 sl = __ldg(sc + l);
                            pair_add(tile, ro + __float_as_int(sl.y), U * sl.x, wrap);
                        }
                    }
                }
                __syncwarp();
            }
        } else {
            const float* dc = p.delta + s0;
            for (int t = ka; t < kb; ++t) {
                const float4 rk = recs[s0 + t];
                const int ik = rec_idx(rk);
                const int ro = (rec_pos(rk) - pb.r0) * M;
                const float wk = wbuf[s0 + ik] * scale;
                for (int l = lane; l < ik; l += 32) {
                    const float2 sl = __ldg(sc + l);
                    pair_add(tile, ro + __float_as_int(sl.y), wk * expf(-beta * (rk.x - __ldg(dc + l))),
                             wrap);
                }
            }
        }
    }
    if (FIXED && wrap) atomicOr(&wrap_sh, 1);
    __syncthreads();
    if (FIXED && wrap_sh) {                 // recomputed by the FP32 variant
        if (threadIdx.x == 0) redo[x] = 1;
        return;
    }
    // the block's share of its rows, summed over the shares in a fixed order by the
    // finalisation
    float* out = p.dal_part + ((int64_t)x << p.lgR) * M;
    const float inv = FIXED ? ldexpf(1.f, -sexp) : 1.f;
    for (int e = threadIdx.x; e < ntile; e += blockDim.x) out[e] = (float)tile[e] * inv;
}

// The exponent s of the fixed-point pair tiles: w_max = the largest w_k (one pass over w),
// then s with 32 w_max 2^s <= 2^26; written to the header.  A tile whose adds would wrap is
// still exact (the FP32 variant redoes it); s below kFixedMinExp (w_max above ~2^9) sends
// every block to the FP32 variant, so that the fixed-point resolution 2^-s stays fine.
constexpr int kFixedMinExp = 8;
__global__ void k_pair_wmax(Problem p, const float* __restrict__ w, unsigned* wmax_bits) {
    float m = 0.f;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p.N;
         k += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, w[k]);
    for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(HK_FULL, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(wmax_bits, __float_as_uint(m));
}
__global__ void k_pair_scale(Problem p, const unsigned* wmax_bits, int* redo, int nblocks) {
    const float wmax = __uint_as_float(*wmax_bits);
    int e = 0;
    if (wmax > 0.f && isfinite(wmax)) frexpf(32.f * wmax, &e);     // 32 wmax < 2^e
    const int s = 26 - e;
    if (blockIdx.x == 0 && threadIdx.x == 0) p.hdr->pad[10] = s;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblocks; b += gridDim.x * blockDim.x)
        redo[b] = s < kFixedMinExp ? 1 : 0;
}

static int pair_target_blocks() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = 2 * sms;        // two waves of one 1024-thread block per SM
    return nb < kPairBlocksMax ? nb : kPairBlocksMax;
}

static size_t pair_smem(const Problem& p) {
    return sizeof(float) * (((size_t)p.M << p.lgR) + 4) + sizeof(float2) * kBwdStage * (kPairRowThreads / 32);
}

cudaError_t launch_pairs_forward(const Problem& p, cudaStream_t s, int* nl) {
    cudaError_t err;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int P = p.P;
    // alpha in tile-major order
    int64_t total = (int64_t)P * P * kTile * kTile;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_alpha_tiles<<<(unsigned)blocks, 256, 0, s>>>(p, p.at);
    ++*nl;
    // work items (row block, kFwdChunksPerItem chunks) from a counter in the header
    const size_t smem = sizeof(float) * kTile * kTileLd + sizeof(float4) * kStage * kPairWarps;
    err = cudaFuncSetAttribute(k_pairs_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_pairs_fwd<<<(unsigned)(sms * 2), kPairThreads, smem, s>>>(p, p.recs, p.bstart, p.wide, p.at,
                                                               p.Aint, p.Bint, (int*)&p.hdr->pad[8]);
    ++*nl;
    prof_mark(s, "pairs_fwd");
    return cudaGetLastError();
}

cudaError_t launch_pairs_backward(const Problem& p, cudaStream_t s, int* nl) {
    cudaError_t err;
    const int nbt = pair_target_blocks();
    const int nblocks = nbt + p.n_rb;
    k_pair_plan<<<p.n_rb, kPairRowThreads, 0, s>>>(p, p.plan_b, nbt, (unsigned*)&p.hdr->pad[12]);
    ++*nl;
    prof_mark(s, "pair_plan_bwd");
    const size_t smem = pair_smem(p);
    for (const void* k : {(const void*)k_pairs_bwd_rows<true>, (const void*)k_pairs_bwd_rows<false>}) {
        err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    // the fixed-point scale from the largest w, then the fixed-point pass, then the FP32
    // pass over the blocks it could not hold
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned* wmax_bits = (unsigned*)&p.hdr->pad[11];
    cudaMemsetAsync(wmax_bits, 0, sizeof(unsigned), s);
    int64_t wb = (p.N + 255) / 256;
    if (wb > (int64_t)sms * 4) wb = (int64_t)sms * 4;
    k_pair_wmax<<<(unsigned)(wb > 0 ? wb : 1), 256, 0, s>>>(p, p.wbuf, wmax_bits);
    k_pair_scale<<<(unsigned)((nblocks + 255) / 256), 256, 0, s>>>(p, wmax_bits, p.pair_redo, nblocks);
    k_pairs_bwd_rows<true><<<nblocks, kPairRowThreads, smem, s>>>(p, p.recs, p.src, p.kprep, p.wbuf,
                                                                 p.pair_redo);
    k_pairs_bwd_rows<false><<<nblocks, kPairRowThreads, smem, s>>>(p, p.recs, p.src, p.kprep, p.wbuf,
                                                                  p.pair_redo);
    *nl += 4;
    prof_mark(s, "pairs_bwd");
    return cudaGetLastError();
}

}  // namespace hk
