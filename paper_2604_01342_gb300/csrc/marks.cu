// Mark-major walk: one decay per source and large M, with the excitation matrix read
// through its support (the entries alpha[i][j] != 0; every entry when the caller asks for
// the dense gradient).
//
// The intensity of an event of mark i reads only the components j of the source-indexed
// state with alpha[i][j] != 0 (paper, Section 2, Eq. hawkes_excitation):
//     lambda_k = mu_i + sum_{j in supp(i)} alpha[i][j] beta_j S_{k,j},
//     S_{k,j} = sum_{l < k, c_l = j} exp(-beta_j (t_k - t_l)),
// and between two events of mark j the component S_j only decays, so it is known at any
// time from its value just after the last event of mark j (the closed form of the
// recurrence of Appendix B, Eq. alpha_grad_recurrence, between its jumps).  So the events
// are sorted, stably, by (segment, mark), and one warp takes one (segment, target mark i):
// it walks the segment's events of mark i in index order, while lane g of its row (source
// j) walks the segment's events of mark j in index order and keeps S_j, G_j just after the
// last of them that precedes the current target event.  The gradient sums of Appendix B
// (Eqs. grad_mu, grad_alpha, grad_gamma)
//     dL/dalpha_ij  += beta_j w_k S_{k,j},   dL/dbeta_j += w_k alpha[i][j] (S_{k,j} - beta_j G_{k,j})
// then stay in the lane's registers for the whole segment: no atomics per event, no dense
// state per event, and O(|supp(i)|) work per event.  The state at each segment start comes
// from the segments before it (Section 3.3: a batch depends on the earlier ones through
// one carried state): per (segment, mark) the contribution of its events at the next
// segment start, then a scan over the segments per mark.
//
// Times: each event carries its offset from its segment's first event as an FP32 pair
// (hi, lo) with hi + lo = t - t_0 to about 2^-48 relative (one FP64 subtraction per event,
// in the sort), so that a time difference inside a segment is (hi_a - hi_b) + (lo_a - lo_b)
// in FP32 arithmetic: the high parts of two nearby times subtract exactly, and the result
// has FP32 relative accuracy however large the absolute times are.
#include "common.cuh"

namespace hk {

constexpr int kTileEv = 16384;          // events per tile: one warp histograms and scatters it
constexpr int kMarkGroups = 4;          // 32-lane groups of a row: up to 128 support entries
constexpr int kMarkRowMax = 32 * kMarkGroups;
constexpr int kRowMaxWord = 9;          // header word: the longest support row (device)
constexpr float kMarkTail = 104.f;      // exp(-x) is 0 in FP32 for x above this

__device__ __forceinline__ float4 mark_sentinel() {
    return make_float4(0.f, 0.f, __int_as_float(0x7fffffff), 0.f);
}

// ---------------------------------------------------------------- support of alpha
// One warp per row: the number of support entries (every entry when the gradient is dense),
// stored at row_ptr[i + 1]; a row longer than the walk's lane groups is reported.
__global__ void k_csr_count(Problem p) {
    const int M = p.M, lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < M; i += warps) {
        int n = M;
        if (p.support) {
            n = 0;
            for (int j0 = 0; j0 < M; j0 += 32) {
                const int j = j0 + lane;
                n += __popc(__ballot_sync(HK_FULL, j < M && p.alpha[(int64_t)i * M + j] != 0.f));
            }
        }
        if (lane == 0) {
            p.row_ptr[i + 1] = n;
            if (n > kMarkRowMax) set_status(p.hdr, HAWKES_ERR_UNSUPPORTED);
            atomicMax((unsigned long long*)&p.hdr->pad[kRowMaxWord], (unsigned long long)n);
        }
        if (i == 0 && lane == 0) p.row_ptr[0] = 0;
    }
}

// Inclusive scan of row_ptr[1..M] in place (one block of 1024 threads).
__global__ void k_csr_scan(Problem p) {
    __shared__ int part[1024];
    const int M = p.M;
    const int per = (M + blockDim.x - 1) / blockDim.x;
    const int a = threadIdx.x * per, b = min(a + per, M);
    int s = 0;
    for (int i = a; i < b; ++i) s += p.row_ptr[i + 1];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int i = a; i < b; ++i) {
        run += p.row_ptr[i + 1];
        p.row_ptr[i + 1] = run;
    }
}

// One warp per row: the support entries in column order (column, value).
__global__ void k_csr_fill(Problem p) {
    const int M = p.M, lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    if (failed(p.hdr)) return;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < M; i += warps) {
        int at = p.row_ptr[i];
        for (int j0 = 0; j0 < M; j0 += 32) {
            const int j = j0 + lane;
            const float a = j < M ? p.alpha[(int64_t)i * M + j] : 0.f;
            const bool in = j < M && (!p.support || a != 0.f);
            const uint32_t m = __ballot_sync(HK_FULL, in);
            if (in) {
                const int e = at + __popc(m & ((1u << lane) - 1u));
                p.sup_col[e] = j;
                p.sup_val[e] = a;
            }
            at += __popc(m);
        }
    }
}

// ---------------------------------------------------------------- segments
// Per segment s (events [s L, min((s + 1) L, N))): its first time t0, the span D to the next
// segment's first event (0 for the last), and T - t0, as FP64 and as FP32 (hi, lo) pairs:
// seg_time[3 s + {0, 1, 2}] = t0, D, T - t0; seg_f[4 s + {0, 1, 2, 3}] = D hi, D lo, (T-t0) hi, lo.
__global__ void k_seg_times(Problem p, int64_t L) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.nseg || failed(p.hdr)) return;
    const double T = p.Tarr[0];
    const int64_t s0 = (int64_t)s * L, s1 = s0 + L;
    const double t0 = p.t[s0];
    const double D = s1 < p.N ? p.t[s1] - t0 : 0.0;
    const double Tm = T - t0;
    p.seg_time[3 * s] = t0;
    p.seg_time[3 * s + 1] = D;
    p.seg_time[3 * s + 2] = Tm;
    const float Dh = (float)D, Th = (float)Tm;
    p.seg_f[4 * s] = Dh;
    p.seg_f[4 * s + 1] = (float)(D - (double)Dh);
    p.seg_f[4 * s + 2] = Th;
    p.seg_f[4 * s + 3] = (float)(Tm - (double)Th);
}

// Per-warp tile of kTileEv events: its events per mark (shared-memory histogram), written
// as tile_cnt[tile][M].  Marks are loaded four rounds ahead.
__global__ void k_tile_hist(Problem p) {
    extern __shared__ int32_t hist_sm[];
    const int M = p.M, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t* h = hist_sm + (int64_t)w * M;
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;
    if (failed(p.hdr) || tile >= p.ntiles) return;
    for (int m = lane; m < M; m += 32) h[m] = 0;
    __syncwarp();
    const int64_t k0 = tile * kTileEv, k1 = min(k0 + kTileEv, p.N);
    for (int64_t kb = k0; kb < k1; kb += 128) {
        int cs[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t k = kb + 32 * r + lane;
            cs[r] = k < k1 ? __ldg(p.c + k) : -1;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)       // (a mark outside [0, M) is skipped: unvalidated input)
            if ((unsigned)cs[r] < (unsigned)M) atomicAdd(&h[cs[r]], 1);
    }
    __syncwarp();
    int32_t* out = p.tile_cnt + tile * M;
    for (int m = lane; m < M; m += 32) out[m] = h[m];
}

// One thread per (segment, mark): the exclusive prefix of its tiles' counts inside the
// segment (in place), and the segment total into seg_off[s M + m].
__global__ void k_seg_counts(Problem p) {
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int M = p.M;
    if (x >= (int64_t)p.nseg * M || failed(p.hdr)) return;
    const int s = (int)(x / M), m = (int)(x % M);
    const int64_t ta = (int64_t)s * p.seg_tiles, tb = min(ta + p.seg_tiles, (int64_t)p.ntiles);
    int run = 0;
    for (int64_t tl = ta; tl < tb; ++tl) {
        const int v = p.tile_cnt[tl * M + m];
        p.tile_cnt[tl * M + m] = run;
        run += v;
    }
    p.seg_off[x] = run;
}

// Exclusive scan of seg_off[0 .. n) in place, the total at seg_off[n] (one block).
__global__ void k_seg_off_scan(Problem p) {
    __shared__ int part[1024];
    const int64_t n = (int64_t)p.nseg * p.M;
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t a = threadIdx.x * per, b = min(a + per, n);
    int s = 0;
    for (int64_t i = a; i < b; ++i) s += p.seg_off[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int64_t i = a; i < b; ++i) {
        const int v = p.seg_off[i];
        p.seg_off[i] = run;
        run += v;
    }
    if (threadIdx.x == blockDim.x - 1) p.seg_off[n] = run;
}

// Per-warp tile: every event to its slot in the (segment, mark) order, stably (the tile's
// events of one mark in index order after those of the earlier tiles of the segment): the
// warp's running slot per mark starts at seg_off + the tile's prefix, and the lanes of one
// mark in one 32-event round take consecutive slots in lane order.  Record: (hi, lo) offset
// from the segment's first time, the event index, the mark.
__global__ void k_mark_scatter(Problem p, int64_t L) {
    extern __shared__ int32_t slot_sm[];
    const int M = p.M, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t* slot = slot_sm + (int64_t)w * M;
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;
    if (failed(p.hdr) || tile >= p.ntiles) return;
    const int64_t k0 = tile * kTileEv, k1 = min(k0 + kTileEv, p.N);
    const int s = (int)(k0 / L);
    for (int m = lane; m < M; m += 32)
        slot[m] = p.seg_off[(int64_t)s * M + m] + p.tile_cnt[tile * M + m];
    __syncwarp();
    const double t0 = p.seg_time[3 * s];
    for (int64_t kb = k0; kb < k1; kb += 128) {
        int cs[4];
        double ts[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t k = kb + 32 * r + lane;
            const int cv = k < k1 ? __ldg(p.c + k) : -1;
            cs[r] = (unsigned)cv < (unsigned)M ? cv : -1 - lane;    // skipped as in k_tile_hist
            ts[r] = k < k1 ? __ldg(p.t + k) : 0.0;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t peers = __match_any_sync(HK_FULL, cs[r]);
            const int leader = __ffs(peers) - 1;
            int first = 0;
            if (lane == leader && cs[r] >= 0) first = atomicAdd(&slot[cs[r]], __popc(peers));
            first = __shfl_sync(HK_FULL, first, leader);
            if (cs[r] >= 0) {
                const int at = first + __popc(peers & ((1u << lane) - 1u));
                const double d = ts[r] - t0;
                const float hi = (float)d;
                const float lo = (float)(d - (double)hi);
                p.recs[at] = make_float4(hi, lo, __int_as_float((int)(kb + 32 * r + lane)),
                                         __int_as_float(cs[r]));
            }
        }
    }
}

// One warp per (segment s < nseg - 1, mark m): the contribution of the segment's events of
// mark m to the state at the next segment start,
//     v = sum exp(-beta_m x),  g = sum x exp(-beta_m x),  x = t_{next start} - t_l,
// walking the list backwards from its end (x grows) and stopping when every lane's x is
// past the point where exp(-beta_m x) is 0 in FP32.  Written to Shat/Ghat[s + 1][m].
__global__ void k_seg_aggregate(Problem p) {
    const int M = p.M, lane = threadIdx.x & 31;
    const int64_t nlist = (int64_t)(p.nseg - 1) * M;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (failed(p.hdr)) return;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < nlist; x += warps) {
        const int s = (int)(x / M), m = (int)(x % M);
        const int a = p.seg_off[x], b = p.seg_off[x + 1];
        const float be = beta_of(p, 0, m);
        const float Dh = p.seg_f[4 * s], Dl = p.seg_f[4 * s + 1];
        float v = 0.f, g = 0.f;
        for (int e1 = b; e1 > a; e1 -= 32) {
            const int e = e1 - 1 - lane;
            float xx = 0.f;
            bool live = false;
            if (e >= a) {
                const float4 r = p.recs[e];
                xx = (Dh - r.x) + (Dl - r.y);
                live = be * xx < kMarkTail;
                if (live) {
                    const float d = exp_unbiased(-be * xx);
                    v += d;
                    g += xx * d;
                }
            }
            if (!__any_sync(HK_FULL, live)) break;
        }
        for (int o = 16; o >= 1; o >>= 1) {
            v += __shfl_xor_sync(HK_FULL, v, o);
            g += __shfl_xor_sync(HK_FULL, g, o);
        }
        if (lane == 0) {
            p.Shat[(int64_t)(s + 1) * M + m] = v;
            if (p.Ghat) p.Ghat[(int64_t)(s + 1) * M + m] = g;
        }
    }
}

// One thread per mark: the states at every segment start from the aggregates, in place:
//     S^_{s+1} = d_s S^_s + v_s,  G^_{s+1} = d_s (G^_s + D_s S^_s) + g_s,  d_s = exp(-beta D_s)
// (the composition rule of Section 3 with a diagonal transition), S^_0 = G^_0 = 0.
__global__ void k_seg_carry(Problem p) {
    const int M = p.M;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M || failed(p.hdr) || p.nseg <= 0) return;
    const float be = beta_of(p, 0, m);
    float S = 0.f, G = 0.f;
    p.Shat[m] = 0.f;
    if (p.Ghat) p.Ghat[m] = 0.f;
    for (int s = 0; s + 1 < p.nseg; ++s) {
        const float D = (float)p.seg_time[3 * s + 1];
        const float d = be * D < kMarkTail ? exp_unbiased(-be * D) : 0.f;
        const int64_t at = (int64_t)(s + 1) * M + m;
        const float v = p.Shat[at];
        const float g = p.Ghat ? p.Ghat[at] : 0.f;
        G = d * (G + D * S) + g;
        S = d * S + v;
        p.Shat[at] = S;
        if (p.Ghat) p.Ghat[at] = G;
    }
}

// ---------------------------------------------------------------- the walk
// Work items (segment, target mark) in segment-major order, taken from a counter so that the
// warps work on the same few segments at a time (their sorted events stay in L2).  GRAD
// adds the gradient sums; without it only lambda, its log and the compensator are formed.
// R lane groups hold rows of up to 32 R support entries; both variants are launched and the
// one whose R fits the longest row (a header word written by k_csr_count) does the work, so
// that rows of at most 64 entries run with half the registers and twice the warps per SM.
// Each lane keeps the next two records of its source list in flight, and the warp the next
// target record, because a walk step waits on little else than those loads.
// A lane's state is its component at the previous target's time t' (the segment start
// before the first target): at target k, S = exp(-beta_j (t_k - t')) S + sum of
// exp(-beta_j (t_k - t_l)) over its source events l with index in [index of the previous
// target, k), and G likewise with the weights (t_k - t_l) (G takes (t_k - t') S first).  The
// one factor per target that multiplies the state goes through exp_unbiased (it is chained
// along the targets); each source event's own term is used once and takes expf (nothing
// chained), which keeps a source step to a handful of instructions.
template <bool GRAD, int R>
__global__ void __launch_bounds__(256, R == 2 ? 4 : 2) k_walk_marks(Problem p,
                                                                    unsigned long long* counter) {
    if (failed(p.hdr)) return;
    const unsigned long long rowmax = *(volatile unsigned long long*)&p.hdr->pad[kRowMaxWord];
    if (R == 2 ? rowmax > 64 : rowmax <= 64) return;      // the other variant's work
    const int M = p.M, lane = threadIdx.x & 31;
    const int64_t nitems = (int64_t)p.nseg * M;
    const float4* __restrict__ rec = p.recs;
    const int32_t* __restrict__ soff = p.seg_off;
    const float4 sentinel = mark_sentinel();
    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = (int64_t)atomicAdd(counter, 1ull);
        item = __shfl_sync(HK_FULL, item, 0);
        if (item >= nitems) break;
        const int s = (int)(item / M), i = (int)(item % M);
        const int ta = soff[item], tb = soff[item + 1];
        if (ta == tb) continue;
        const int r0 = p.row_ptr[i], r1 = p.row_ptr[i + 1];
        const int ng = (r1 - r0 + 31) >> 5;
        float Sv[R], Gv[R], av[R], bv[R], dal[R], dbe[R];
        int q[R], qe[R], jv[R];
        float4 nx[R], nx2[R];
#pragma unroll
        for (int g = 0; g < R; ++g) {
            const int e = r0 + 32 * g + lane;
            const bool valid = g < ng && e < r1;
            jv[g] = valid ? p.sup_col[e] : -1;
            av[g] = valid ? p.sup_val[e] : 0.f;
            bv[g] = valid ? beta_of(p, 0, jv[g]) : 0.f;
            const int64_t at = (int64_t)s * M + (valid ? jv[g] : 0);
            Sv[g] = valid ? p.Shat[at] : 0.f;
            Gv[g] = (GRAD && valid) ? p.Ghat[at] : 0.f;
            q[g] = valid ? soff[at] : 0;
            qe[g] = valid ? soff[at + 1] : 0;
            nx[g] = q[g] < qe[g] ? rec[q[g]] : sentinel;
            nx2[g] = q[g] + 1 < qe[g] ? rec[q[g] + 1] : sentinel;
            dal[g] = 0.f;
            dbe[g] = 0.f;
        }
        const float mu_i = p.mu[i];
        LogProd lp;
        float dmu = 0.f;
        bool bad = false;
        float4 tnext = rec[ta];
        float ph = 0.f, pl = 0.f;          // the previous target's time (segment start first)
        for (int k = ta; k < tb; ++k) {
            const float4 tk = tnext;
            if (k + 1 < tb) tnext = rec[k + 1];
            const int ik = __float_as_int(tk.z);
            const float dtp = (tk.x - ph) + (tk.y - pl);
            ph = tk.x;
            pl = tk.y;
            float part = 0.f;
#pragma unroll
            for (int g = 0; g < R; ++g) {
                if (g < ng) {
                    // the state carried from the previous target ...
                    const float d = exp_unbiased(-bv[g] * dtp);
                    if (GRAD) Gv[g] = d * fmaf(dtp, Sv[g], Gv[g]);
                    Sv[g] *= d;
                    // ... plus the source's events since then
                    while (__float_as_int(nx[g].z) < ik) {
                        const float x = (tk.x - nx[g].x) + (tk.y - nx[g].y);
                        const float e = expf(-bv[g] * x);
                        Sv[g] += e;
                        if (GRAD) Gv[g] = fmaf(x, e, Gv[g]);
                        ++q[g];
                        nx[g] = nx2[g];
                        nx2[g] = q[g] + 1 < qe[g] ? rec[q[g] + 1] : sentinel;
                    }
                    part = fmaf(av[g] * bv[g], Sv[g], part);
                }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(HK_FULL, part, o);
            const float lam = mu_i + part;
            bad |= !(lam > 0.f);
            if (lane == 0) lp.mul(lam);
            if (GRAD) {
                const float w = 1.f / lam;
                if (lane == 0) dmu += w;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    dal[g] = fmaf(w, Sv[g], dal[g]);
                    dbe[g] = fmaf(w * av[g], fmaf(-bv[g], Gv[g], Sv[g]), dbe[g]);
                }
            }
        }
        // compensator sums of the target events (mark i as a source): events with
        // beta_i (T - t) >= kMarkTail add 1 to E_i and 0 to F_i
        const float bi = beta_of(p, 0, i);
        const float Th = p.seg_f[4 * s + 2], Tl = p.seg_f[4 * s + 3];
        float Et = 0.f, Ft = 0.f;
        if (bi * (Th - rec[tb - 1].x) < kMarkTail + 1.f) {       // T - t of the last, roughly
            for (int k = ta + lane; k < tb; k += 32) {
                const float4 r = rec[k];
                const float x = (Th - r.x) + (Tl - r.y);
                if (bi * x < kMarkTail) {
                    const float e = exp_unbiased(-bi * x);
                    Et += e;
                    Ft = fmaf(x, e, Ft);
                }
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            Et += __shfl_xor_sync(HK_FULL, Et, o);
            Ft += __shfl_xor_sync(HK_FULL, Ft, o);
        }
        if (GRAD) {
#pragma unroll
            for (int g = 0; g < R; ++g) {
                if (jv[g] >= 0) {
                    atomicAdd(&p.dal_acc[(int64_t)i * M + jv[g]], (double)(bv[g] * dal[g]));
                    atomicAdd(&p.dbe_acc[jv[g]], (double)dbe[g]);
                }
            }
        }
        if (__any_sync(HK_FULL, bad) && lane == 0) set_status(p.hdr, HAWKES_ERR_NONPOS_INTENSITY);
        if (lane == 0) {
            atomicAdd(&p.ll_acc[0], lp.log_value());
            atomicAdd(&p.E_acc[i], (double)(tb - ta) - (double)Et);
            if (GRAD) {
                atomicAdd(&p.dmu_acc[i], (double)dmu);
                if (Ft != 0.f) atomicAdd(&p.F_acc[i], (double)Ft);
            }
        }
    }
}

template <bool GRAD, int R>
static cudaError_t launch_walk_marks(const Problem& p, int sms, int64_t nsm, cudaStream_t s) {
    auto kern = k_walk_marks<GRAD, R>;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    if (err != cudaSuccess) return err;
    int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (nsm + 7) / 8;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(p, (unsigned long long*)&p.hdr->pad[8]);
    return cudaGetLastError();
}

int marks_row_max() { return kMarkRowMax; }
int marks_tile_events() { return kTileEv; }

cudaError_t launch_marks(const Problem& p, int64_t L, cudaStream_t s, int* nl) {
    cudaError_t err;
    const int M = p.M;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // support of alpha as rows of (column, value)
    const unsigned rows_grid = (unsigned)((M + 7) / 8);
    k_csr_count<<<rows_grid, 256, 0, s>>>(p);
    k_csr_scan<<<1, 1024, 0, s>>>(p);
    k_csr_fill<<<rows_grid, 256, 0, s>>>(p);
    *nl += 3;
    prof_mark(s, "support");
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (p.N > 0) {
        // stable counting sort of the events by (segment, mark)
        k_seg_times<<<(unsigned)((p.nseg + 127) / 128), 128, 0, s>>>(p, L);
        const int wpb = p.tile_warps;
        const size_t smem = sizeof(int32_t) * (size_t)wpb * M;
        if (smem > 48 * 1024) {
            if ((err = cudaFuncSetAttribute(k_tile_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem)) != cudaSuccess)
                return err;
            if ((err = cudaFuncSetAttribute(k_mark_scatter,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem)) != cudaSuccess)
                return err;
        }
        const unsigned tgrid = (unsigned)((p.ntiles + wpb - 1) / wpb);
        k_tile_hist<<<tgrid, 32 * wpb, smem, s>>>(p);
        const int64_t nsm = (int64_t)p.nseg * M;
        k_seg_counts<<<(unsigned)((nsm + 255) / 256), 256, 0, s>>>(p);
        k_seg_off_scan<<<1, 1024, 0, s>>>(p);
        k_mark_scatter<<<tgrid, 32 * wpb, smem, s>>>(p, L);
        *nl += 5;
        prof_mark(s, "mark_sort");
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        // segment-start states
        if (p.nseg > 1) {
            int64_t blocks = ((int64_t)(p.nseg - 1) * M + 7) / 8;
            if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
            k_seg_aggregate<<<(unsigned)blocks, 256, 0, s>>>(p);
            ++*nl;
        }
        k_seg_carry<<<(unsigned)((M + 127) / 128), 128, 0, s>>>(p);
        ++*nl;
        prof_mark(s, "seg_states");
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        // the walk: both variants when the support's longest row is known only on the
        // device, the one that fits when every row is dense (M entries)
        const bool two = !p.support ? M <= 64 : true, four = !p.support ? M > 64 : true;
        if (two) {
            err = p.grad ? launch_walk_marks<true, 2>(p, sms, nsm, s)
                         : launch_walk_marks<false, 2>(p, sms, nsm, s);
            if (err != cudaSuccess) return err;
            ++*nl;
        }
        if (four) {
            err = p.grad ? launch_walk_marks<true, 4>(p, sms, nsm, s)
                         : launch_walk_marks<false, 4>(p, sms, nsm, s);
            if (err != cudaSuccess) return err;
            ++*nl;
        }
        prof_mark(s, "walk_marks");
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return launch_finalize_mode(p, s, 0, nl);
}

}  // namespace hk
