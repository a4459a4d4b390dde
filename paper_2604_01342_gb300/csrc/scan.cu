// Inter-chunk carry: the chunk-start states S^_b (and G^_b for the gradient)
// of the source-indexed recurrence
//     S_k = D_k (S_{k-1} + e_{c_{k-1}}),  D_k = diag(exp(-beta_j (t_k - t_{k-1})))
// (paper, Appendix B, Eq. alpha_grad_recurrence, with one decay per source),
// evaluated with the composition rule of the paper's associative operator
// (Section 3, (s_A, v_A) (.) (s_B, v_B) = (s_A s_B, s_A v_B + v_A), here with a
// diagonal s).  Chunk b starts at event s_b; its map to the next chunk start is
//     S^_{b+1} = d_b S^_b + v_b,         d_b = exp(-beta (t_{s_{b+1}} - t_{s_b}))
//     G^_{b+1} = d_b (G^_b + D_b S^_b) + g_b,  D_b = t_{s_{b+1}} - t_{s_b}
// with v_b = sum_{l in b} exp(-beta_{c_l}(t_{s_{b+1}} - t_l)) e_{c_l} and g_b the
// same weighted by (t_{s_{b+1}} - t_l).  G is the derivative state
// G_{k,j} = sum_{l<k, c_l=j} (t_k - t_l) exp(-beta_j (t_k - t_l)) = -dS_{k,j}/dbeta_j.
// The last chunk of each sequence maps to the zero state, so one plain scan
// over all chunks of all sequences restarts at every sequence.
//
// Three passes (reduce, scan, re-walk) instead of a serial chain:
//   A: each block composes a group of Gc chunks from a zero state -> (v, g, span, reset)
//   B: the group composites are scanned in order per mark (in Q segments composed in
//      parallel, then walked from the composites before them) -> carry into each group
//   C: each block re-walks its group from the carry and writes S^_b, G^_b per chunk.
// Within a chunk the decay is applied to the whole state once and the chunk's
// events are added with shared-memory atomics, so S is never held per event.
#include "common.cuh"

namespace hk {

// PHASE 0 = A (compose from zero), 1 = C (re-walk from carry and write states).
// With few marks (M <= kScanSplitM) the events of a chunk pile their contributions onto a
// handful of state entries, so each warp adds into its own copy of the state and the
// copies are folded into S, G once per chunk.
constexpr int kScanSplitM = 64;
__host__ __device__ inline size_t scan_smem_floats(int M, int threads) {
    return 2 * (size_t)M + (M <= kScanSplitM ? 2 * (size_t)M * (threads / 32) : 0);
}

template <int PHASE, bool GRAD>
__global__ void __launch_bounds__(256) k_scan_group(Problem p, int64_t g_begin) {
    extern __shared__ float sm[];
    float* S = sm;
    float* G = sm + p.M;
    const bool split = p.M <= kScanSplitM;
    const int nwarps = blockDim.x >> 5;
    float* Sw = sm + 2 * p.M + (threadIdx.x >> 5) * p.M;     // this warp's copies (split only)
    float* Gw = sm + 2 * p.M + (nwarps + (threadIdx.x >> 5)) * p.M;
    __shared__ double span_sh;
    __shared__ int reset_sh;
    if (failed(p.hdr)) return;
    const int64_t nb = num_chunks(p);
    const int64_t g = g_begin + blockIdx.x;
    const int64_t b0 = g * p.Gc;
    if (b0 >= nb) return;
    const int64_t b1 = b0 + p.Gc < nb ? b0 + p.Gc : nb;
    const int M = p.M;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        if (PHASE == 0) {
            S[j] = 0.f;
            if (GRAD) G[j] = 0.f;
        } else {
            S[j] = p.carry_S[g * M + j];
            if (GRAD) G[j] = p.carry_G[g * M + j];
        }
    }
    if (split)
        for (int j = threadIdx.x; j < 2 * nwarps * M; j += blockDim.x) sm[2 * M + j] = 0.f;
    if (threadIdx.x == 0) { span_sh = 0.0; reset_sh = 0; }
    __syncthreads();
    // Chunk-GEMM path (p.delta set): the per-event offsets delta_l = t_l - t_0 from the chunk
    // start are taken here once in FP64 (this part's FP64 rate is 1/64 of its FP32 rate) and
    // stored for the later kernels, with the chunk span D = t_n - t_0 and T - t_0; the offset
    // to the next chunk start is then D - delta_l in FP32 (an absolute error of about one ulp
    // of D, i.e. a relative error below 1e-6 of exp(-beta x) while beta D <= 16; wider chunks
    // take it in FP64).  The state walk's scan keeps one FP64 difference per event.
    __shared__ float D_sh;
    __shared__ int narrow_sh;
    const bool fast = p.delta != nullptr;
    for (int64_t b = b0; b < b1; ++b) {
        const int32_t seq = p.chunk_seq[b];
        int64_t s0, s1;
        chunk_range(p, b, seq, s0, s1);
        const bool last = (s1 == p.off[seq + 1]);
        if (PHASE == 1) {
            for (int j = threadIdx.x; j < M; j += blockDim.x) {
                p.Shat[b * M + j] = S[j];
                if (GRAD) p.Ghat[b * M + j] = G[j];
            }
        }
        const double t0 = s0 < s1 ? p.t[s0] : 0.0;
        if (last) {
            if (PHASE == 0 && fast) {
                if (threadIdx.x == 0 && s0 < s1) p.Tmt[b] = (float)tdiff(p, p.Tarr[seq], t0);
                for (int64_t l = s0 + threadIdx.x; l < s1; l += blockDim.x)
                    p.delta[l] = (float)tdiff(p, p.t[l], t0);
            }
            for (int j = threadIdx.x; j < M; j += blockDim.x) {
                S[j] = 0.f;
                if (GRAD) G[j] = 0.f;
            }
            if (threadIdx.x == 0) { span_sh = 0.0; reset_sh = 1; }
            __syncthreads();
            continue;
        }
        const double tn = p.t[s1];            // start of the next chunk
        float D;
        bool narrow;
        if (PHASE == 1 && fast) {
            D = p.Dspan[b];
            narrow = beta_of(p, seq, 0) * D <= 16.f;
        } else {
            if (threadIdx.x == 0) {
                const double span = fast ? tdiff(p, tn, t0) : tn - t0;
                D_sh = (float)span;
                narrow_sh = fast && beta_of(p, seq, 0) * D_sh <= 16.f;
                span_sh += span;
                if (PHASE == 0 && fast) {
                    p.Dspan[b] = D_sh;
                    p.Tmt[b] = (float)tdiff(p, p.Tarr[seq], t0);
                }
            }
            __syncthreads();
            D = D_sh;
            narrow = narrow_sh != 0;
        }
        const float dsh = p.shared ? exp_unbiased(-beta_of(p, seq, 0) * D) : 0.f;
        for (int j = threadIdx.x; j < M; j += blockDim.x) {
            float d = p.shared ? dsh : exp_unbiased(-beta_of(p, seq, j) * D);
            float s = S[j];
            if (GRAD) G[j] = d * (G[j] + D * s);
            S[j] = d * s;
        }
        __syncthreads();
        for (int64_t l = s0 + threadIdx.x; l < s1; l += blockDim.x) {
            int32_t cl = p.c[l];
            float x;
            if (fast) {
                float dl;
                if (PHASE == 0) {
                    dl = (float)tdiff(p, p.t[l], t0);
                    p.delta[l] = dl;
                } else {
                    dl = p.delta[l];
                }
                x = narrow ? D - dl : (float)tdiff(p, tn, p.t[l]);
            } else {
                x = (float)(tn - p.t[l]);
            }
            float e = exp_unbiased(-beta_of(p, seq, cl) * x);
            atomicAdd(split ? &Sw[cl] : &S[cl], e);
            if (GRAD) atomicAdd(split ? &Gw[cl] : &G[cl], x * e);
        }
        __syncthreads();
        if (split)      // fold the warps' copies (same thread-to-entry map as every other pass)
            for (int j = threadIdx.x; j < M; j += blockDim.x) {
                float sv = S[j], gv = GRAD ? G[j] : 0.f;
                for (int w = 0; w < nwarps; ++w) {
                    float* sw = sm + 2 * M + w * M;
                    sv += sw[j];
                    sw[j] = 0.f;
                    if (GRAD) {
                        float* gw = sm + 2 * M + (nwarps + w) * M;
                        gv += gw[j];
                        gw[j] = 0.f;
                    }
                }
                S[j] = sv;
                if (GRAD) G[j] = gv;
            }
    }
    if (PHASE == 0) {
        for (int j = threadIdx.x; j < M; j += blockDim.x) {
            p.grp_v[g * M + j] = S[j];
            if (GRAD) p.grp_g[g * M + j] = G[j];
        }
        if (threadIdx.x == 0) {
            p.grp_dt[g] = span_sh;
            p.grp_reset[g] = reset_sh;
        }
    }
}

// One thread per mark j: exclusive scan of the group composites.
// Pass B in parallel: the groups are cut into Q segments.  The map of group g on the
// state of mark j is S' = d S + v_g, G' = d (G + dt S) + g_g (or the constant map
// S' = v_g, G' = g_g at a sequence start); maps of the form
//     S' = a S + v,  G' = b S + c G + w
// compose into the same form.  k_carry_compose builds every segment's composite (one
// thread per (mark, segment)); k_carry_walk starts each (mark, segment) from the
// composites of the segments before it and walks its groups, writing the carry into each.
__device__ __forceinline__ void group_map(const Problem& p, int64_t g, int j, float& d,
                                          float& dt, float& v, float& gg, bool& reset) {
    const int M = p.M;
    v = p.grp_v[g * M + j];
    gg = p.grp_g ? p.grp_g[g * M + j] : 0.f;
    dt = (float)p.grp_dt[g];
    reset = p.grp_reset[g] != 0;
    d = reset ? 0.f : exp_unbiased(-beta_of(p, p.chunk_seq[g * p.Gc], j) * dt);
}

template <bool GRAD>
__global__ void k_carry_compose(Problem p, int Q, float* comp) {
    if (failed(p.hdr)) return;
    const int M = p.M;
    const int j = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (j >= M) return;
    const int64_t ng = (num_chunks(p) + p.Gc - 1) / p.Gc;
    const int64_t per = (ng + Q - 1) / Q;
    const int64_t g0 = q * per, g1 = min(ng, g0 + per);
    float a = 1.f, b = 0.f, c = 1.f, v = 0.f, w = 0.f;
    for (int64_t g = g0; g < g1; ++g) {
        float d, dt, vg, gg;
        bool reset;
        group_map(p, g, j, d, dt, vg, gg, reset);
        if (reset) {
            a = b = c = 0.f;
            v = vg;
            w = GRAD ? gg : 0.f;
        } else {
            if (GRAD) {
                b = d * (dt * a + b);
                c = d * c;
                w = d * (dt * v + w) + gg;
            }
            a = d * a;
            v = d * v + vg;
        }
    }
    const int64_t at = (int64_t)q * M + j, st = (int64_t)Q * M;
    comp[at] = a;
    comp[st + at] = v;
    if (GRAD) {
        comp[2 * st + at] = b;
        comp[3 * st + at] = c;
        comp[4 * st + at] = w;
    }
}

template <bool GRAD>
__global__ void k_carry_walk(Problem p, int Q, const float* comp) {
    if (failed(p.hdr)) return;
    const int M = p.M;
    const int j = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (j >= M) return;
    const int64_t ng = (num_chunks(p) + p.Gc - 1) / p.Gc;
    const int64_t per = (ng + Q - 1) / Q;
    const int64_t g0 = q * per, g1 = min(ng, g0 + per);
    // a slice of a longer sequence starts from the carried-in state (single sequence)
    float cS = p.init_S ? p.init_S[j] : 0.f;
    float cG = (GRAD && p.init_G) ? p.init_G[j] : 0.f;
    const int64_t st = (int64_t)Q * M;
    for (int r = 0; r < q; ++r) {
        const int64_t at = (int64_t)r * M + j;
        const float a = comp[at], v = comp[st + at];
        if (GRAD) cG = comp[2 * st + at] * cS + comp[3 * st + at] * cG + comp[4 * st + at];
        cS = a * cS + v;
    }
    for (int64_t g = g0; g < g1; ++g) {
        p.carry_S[g * M + j] = cS;
        if (GRAD) p.carry_G[g * M + j] = cG;
        float d, dt, vg, gg;
        bool reset;
        group_map(p, g, j, d, dt, vg, gg, reset);
        if (reset) {
            cS = vg;
            cG = gg;
        } else {
            if (GRAD) cG = d * (cG + dt * cS) + gg;
            cS = d * cS + vg;
        }
    }
}

// State contributions of all events at time t_next >= the last event (one slice's
// aggregate for the carry exchange): agg_S[j] = sum_{l: c_l = j} exp(-beta_j (t_next - t_l)),
// agg_G[j] = the same weighted by (t_next - t_l).  Block-level shared histograms.
__global__ void k_slice_aggregate(Problem p, double t_next, float* agg_S, float* agg_G) {
    extern __shared__ float hs[];
    float* hS = hs;
    float* hG = hs + p.M;
    if (failed(p.hdr)) return;
    for (int j = threadIdx.x; j < 2 * p.M; j += blockDim.x) hs[j] = 0.f;
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p.N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int ck = p.c[k];
        const float x = (float)(t_next - p.t[k]);
        const float e = exp_unbiased(-beta_of(p, 0, ck) * x);
        atomicAdd(&hS[ck], e);
        atomicAdd(&hG[ck], x * e);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < p.M; j += blockDim.x) {
        if (hS[j] != 0.f) atomicAdd(&agg_S[j], hS[j]);
        if (hG[j] != 0.f) atomicAdd(&agg_G[j], hG[j]);
    }
}

cudaError_t launch_slice_aggregate(const Problem& p, double t_next, float* agg_S, float* agg_G,
                                   cudaStream_t s, int* nl) {
    cudaMemsetAsync(agg_S, 0, sizeof(float) * (size_t)p.M, s);
    cudaMemsetAsync(agg_G, 0, sizeof(float) * (size_t)p.M, s);
    int64_t blocks = (p.N + 255) / 256;
    if (blocks > 152 * 4) blocks = 152 * 4;
    if (blocks < 1) blocks = 1;
    size_t smem = sizeof(float) * 2 * (size_t)p.M;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_slice_aggregate,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_slice_aggregate<<<(unsigned)blocks, 256, smem, s>>>(p, t_next, agg_S, agg_G);
    ++*nl;
    return cudaGetLastError();
}

// Pass C on the chunk-GEMM path (one sequence, one shared decay, offsets from pass A):
// the same re-walk as k_scan_group<1>, with chunk k at events [k C, min((k+1) C, N)) and
// the next chunk's span and first event slot loaded one chunk ahead, so that the loads
// overlap the state writes and the decay of the current chunk.
template <bool GRAD>
__global__ void __launch_bounds__(256) k_scan_states_fast(Problem p) {
    extern __shared__ float sm[];
    float* S = sm;
    float* G = sm + p.M;
    if (failed(p.hdr)) return;
    const int64_t nb = num_chunks(p);
    const int64_t g = blockIdx.x;
    const int64_t b0 = g * p.Gc;
    if (b0 >= nb) return;
    const int64_t b1 = b0 + p.Gc < nb ? b0 + p.Gc : nb;
    const int M = p.M, C = p.C, tid = threadIdx.x;
    const int64_t N = p.N;
    const float beta = p.beta[0];
    for (int j = tid; j < M; j += blockDim.x) {
        S[j] = p.carry_S[g * M + j];
        if (GRAD) G[j] = p.carry_G[g * M + j];
    }
    auto slot = [&](int64_t b, float& Dn, int& cn, float& dn) {
        const int64_t s1 = (b + 1) * C < N ? (b + 1) * C : N;
        Dn = s1 < N ? __ldg(p.Dspan + b) : 0.f;
        const int64_t l = b * C + tid;
        cn = l < s1 ? __ldg(p.c + l) : 0;
        dn = l < s1 ? __ldg(p.delta + l) : 0.f;
    };
    float Dn, dn;
    int cn;
    slot(b0, Dn, cn, dn);
    __syncthreads();
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t s0 = b * C, s1 = s0 + C < N ? s0 + C : N;
        const float D = Dn, d0 = dn;
        const int c0 = cn;
        if (b + 1 < b1) slot(b + 1, Dn, cn, dn);
        // the chunk-start state out and decayed to the next chunk start in one pass (each
        // thread its own entries)
        const bool last = s1 == N;              // the last chunk maps to the zero state
        const float d = last ? 0.f : exp_unbiased(-beta * D);
        for (int j = tid; j < M; j += blockDim.x) {
            const float sv = S[j];
            p.Shat[b * M + j] = sv;
            if (GRAD) {
                const float gv = G[j];
                p.Ghat[b * M + j] = gv;
                G[j] = d * (gv + D * sv);
            }
            S[j] = d * sv;
        }
        if (last) break;
        __syncthreads();
        const bool narrow = beta * D <= 16.f;
        for (int64_t l = s0 + tid; l < s1; l += blockDim.x) {
            const int cl = l == s0 + tid ? c0 : __ldg(p.c + l);
            const float dl = l == s0 + tid ? d0 : __ldg(p.delta + l);
            const float x = narrow ? D - dl : (float)tdiff(p, p.t[s1], p.t[l]);
            const float e = exp_unbiased(-beta * x);
            atomicAdd(&S[cl], e);
            if (GRAD) atomicAdd(&G[cl], x * e);
        }
        __syncthreads();
    }
}

// Pass A on the chunk-GEMM path (one sequence, one shared decay): the composite of a group
// of chunks [b0, b1) taken straight from its events, each scaled to the group's end t_E (the
// first event of chunk b1).  An event l of chunk b adds
//     e_l = F_b exp(-beta x_l) to S[c_l] and (X_b + x_l) e_l to G[c_l],
// with x_l = t_{s_{b+1}} - t_l (the chunk's span D_b minus the event's offset delta_l while
// beta D_b <= 16, else in FP64), X_b = t_E - t_{s_{b+1}} and F_b = exp(-beta X_b): the sums
// that the chunk-by-chunk walk forms through its chain of decays, without a pass over the
// whole state and a barrier per chunk.  One thread per chunk first lays out the chunk table
// (the offsets t_{s_b}, spans, X_b, F_b; D_b and T - t_{s_b} stored for the later kernels).
// A group that holds the sequence's last chunk maps to the zero state (the walk resets there)
// and only stores the offsets.
constexpr int kMaxGroupChunks = 64;

template <bool GRAD>
__global__ void __launch_bounds__(128) k_scan_reduce_fast(Problem p, int64_t g_begin) {
    extern __shared__ float sm[];
    float* S = sm;
    float* G = sm + p.M;
    const bool split = p.M <= kScanSplitM;
    const int nwarps = blockDim.x >> 5;
    float* Sw = sm + 2 * p.M + (threadIdx.x >> 5) * p.M;     // this warp's copies (split only)
    float* Gw = sm + 2 * p.M + (nwarps + (threadIdx.x >> 5)) * p.M;
    __shared__ double t0_sh[kMaxGroupChunks], tn_sh[kMaxGroupChunks];
    __shared__ float D_sh[kMaxGroupChunks], X_sh[kMaxGroupChunks], F_sh[kMaxGroupChunks];
    __shared__ int narrow_sh[kMaxGroupChunks];
    if (failed(p.hdr)) return;
    const int64_t nb = num_chunks(p);
    const int64_t g = g_begin + blockIdx.x;
    const int64_t b0 = g * p.Gc;
    if (b0 >= nb) return;
    const int64_t b1 = b0 + p.Gc < nb ? b0 + p.Gc : nb;
    const int M = p.M, C = p.C, tid = threadIdx.x, nbg = (int)(b1 - b0);
    const int64_t N = p.N;
    const float beta = p.beta[0];
    const bool final = b1 == nb;              // holds the last chunk
    const double tE = final ? 0.0 : p.t[b1 * C];
    for (int j = tid; j < M; j += blockDim.x) {
        S[j] = 0.f;
        if (GRAD) G[j] = 0.f;
    }
    if (split)
        for (int j = tid; j < 2 * nwarps * M; j += blockDim.x) sm[2 * M + j] = 0.f;
    for (int i = tid; i < nbg; i += blockDim.x) {
        const int64_t b = b0 + i, s0 = b * C, s1 = s0 + C < N ? s0 + C : N;
        const double t0 = p.t[s0];
        t0_sh[i] = t0;
        p.Tmt[b] = (float)tdiff(p, p.Tarr[0], t0);
        if (s1 < N) {
            const double tn = p.t[s1];
            const float D = (float)tdiff(p, tn, t0);
            p.Dspan[b] = D;
            tn_sh[i] = tn;
            D_sh[i] = D;
            narrow_sh[i] = beta * D <= 16.f;
            if (!final) {
                const float X = (float)tdiff(p, tE, tn);
                X_sh[i] = X;
                F_sh[i] = exp_unbiased(-beta * X);
            }
        }
    }
    if (tid == 0) {
        p.grp_dt[g] = final ? 0.0 : tdiff(p, tE, p.t[b0 * C]);
        p.grp_reset[g] = final ? 1 : 0;
    }
    __syncthreads();
    // four events per thread and step, their loads issued before any of their stores
    constexpr int U = 4;
    const int64_t k0 = b0 * C, k1 = b1 * C < N ? b1 * C : N;
    const int nt = blockDim.x;
    for (int64_t lb = k0 + tid; lb < k1; lb += (int64_t)U * nt) {
        double tl[U];
        int cl[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t l = lb + (int64_t)u * nt;
            tl[u] = l < k1 ? __ldg(p.t + l) : 0.0;
            cl[u] = (!final && l < k1) ? __ldg(p.c + l) : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t l = lb + (int64_t)u * nt;
            if (l >= k1) break;
            const int i = (int)((uint64_t)(l - k0) / (uint64_t)C);
            const float dl = (float)tdiff(p, tl[u], t0_sh[i]);
            p.delta[l] = dl;
            if (final) continue;
            const float x = narrow_sh[i] ? D_sh[i] - dl : (float)tdiff(p, tn_sh[i], tl[u]);
            const float e = F_sh[i] * exp_unbiased(-beta * x);
            atomicAdd(split ? &Sw[cl[u]] : &S[cl[u]], e);
            if (GRAD) atomicAdd(split ? &Gw[cl[u]] : &G[cl[u]], (X_sh[i] + x) * e);
        }
    }
    __syncthreads();
    if (split)      // fold the warps' copies
        for (int j = tid; j < M; j += blockDim.x) {
            float sv = S[j], gv = GRAD ? G[j] : 0.f;
            for (int w = 0; w < nwarps; ++w) {
                sv += sm[2 * M + w * M + j];
                if (GRAD) gv += sm[2 * M + (nwarps + w) * M + j];
            }
            S[j] = sv;
            if (GRAD) G[j] = gv;
        }
    for (int j = tid; j < M; j += blockDim.x) {
        p.grp_v[g * M + j] = S[j];
        if (GRAD) p.grp_g[g * M + j] = G[j];
    }
}

// the chunk-GEMM path's pass C: one sequence, one shared decay, offsets written by pass A
static bool fast_states(const Problem& p) { return p.delta != nullptr && p.shared && p.B == 1; }

static size_t scan_smem_bytes(const Problem& p) {
    return sizeof(float) * scan_smem_floats(p.M, 128);
}

static cudaError_t scan_attributes(const Problem& p) {
    const size_t smem = scan_smem_bytes(p);
    if (smem > 48 * 1024) {       // large M on the chunk-GEMM path: opt in to more shared memory
        const void* kerns[] = {(const void*)k_scan_group<0, true>, (const void*)k_scan_group<1, true>,
                               (const void*)k_scan_group<0, false>, (const void*)k_scan_group<1, false>,
                               (const void*)k_scan_states_fast<true>, (const void*)k_scan_states_fast<false>,
                               (const void*)k_scan_reduce_fast<true>, (const void*)k_scan_reduce_fast<false>};
        for (const void* k : kerns) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Pass A over the scan groups [g_begin, g_end) (clipped to the groups of the call).
cudaError_t launch_scan_reduce(const Problem& p, cudaStream_t s, int64_t g_begin, int64_t g_end,
                               int* nl) {
    cudaError_t err = scan_attributes(p);
    if (err != cudaSuccess) return err;
    if (g_end > p.ng_max) g_end = p.ng_max;
    const unsigned grid = (unsigned)(g_end > g_begin ? g_end - g_begin : 1);
    if (fast_states(p) && p.Gc <= kMaxGroupChunks) {
        if (p.grad) k_scan_reduce_fast<true><<<grid, 128, scan_smem_bytes(p), s>>>(p, g_begin);
        else k_scan_reduce_fast<false><<<grid, 128, scan_smem_bytes(p), s>>>(p, g_begin);
    } else if (p.grad) {
        k_scan_group<0, true><<<grid, 128, scan_smem_bytes(p), s>>>(p, g_begin);
    } else {
        k_scan_group<0, false><<<grid, 128, scan_smem_bytes(p), s>>>(p, g_begin);
    }
    ++*nl;
    prof_mark(s, "scan_reduce");
    return cudaGetLastError();
}

// Passes B and C: the carry into every group, then the chunk-start states.
cudaError_t launch_scan_rest(const Problem& p, cudaStream_t s, int* nl) {
    cudaError_t err = scan_attributes(p);
    if (err != cudaSuccess) return err;
    const size_t smem_fast = sizeof(float) * 2 * (size_t)p.M;
    const size_t smem = scan_smem_bytes(p);
    unsigned grid = (unsigned)(p.ng_max > 0 ? p.ng_max : 1);
    // segments of the carry pass: enough (mark, segment) threads for every SM, at least
    // four groups per segment
    int64_t Q = (152 * 512 + p.M - 1) / p.M;
    if (Q > kCarrySegments) Q = kCarrySegments;
    if (Q > (p.ng_max + 3) / 4) Q = (p.ng_max + 3) / 4;
    if (Q < 1) Q = 1;
    const dim3 cgrid((unsigned)((p.M + 127) / 128), (unsigned)Q);
    if (p.grad) {
        k_carry_compose<true><<<cgrid, 128, 0, s>>>(p, (int)Q, p.seg_comp);
        k_carry_walk<true><<<cgrid, 128, 0, s>>>(p, (int)Q, p.seg_comp);
        prof_mark(s, "scan_carry");
        if (fast_states(p)) k_scan_states_fast<true><<<grid, 128, smem_fast, s>>>(p);
        else k_scan_group<1, true><<<grid, 128, smem, s>>>(p, 0);
        prof_mark(s, "scan_states");
    } else {
        k_carry_compose<false><<<cgrid, 128, 0, s>>>(p, (int)Q, p.seg_comp);
        k_carry_walk<false><<<cgrid, 128, 0, s>>>(p, (int)Q, p.seg_comp);
        prof_mark(s, "scan_carry");
        if (fast_states(p)) k_scan_states_fast<false><<<grid, 128, smem_fast, s>>>(p);
        else k_scan_group<1, false><<<grid, 128, smem, s>>>(p, 0);
        prof_mark(s, "scan_states");
    }
    *nl += 3;
    return cudaGetLastError();
}

cudaError_t launch_scan(const Problem& p, cudaStream_t s, int* nl) {
    cudaError_t err = launch_scan_reduce(p, s, 0, p.ng_max, nl);
    if (err == cudaSuccess) err = launch_scan_rest(p, s, nl);
    return err;
}

}  // namespace hk

namespace hk {
__global__ void k_test_exp_unbiased(const float* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = exp_unbiased(x[i]);
}
}  // namespace hk

// Test hook (declared in no public header): y[i] = exp_unbiased(x[i]) for i < n on device
// buffers, so a GPU test can measure its rounding against FP64.  Returns 0 on success.
extern "C" int hawkes_test_exp_unbiased(const float* x, float* y, int64_t n, void* stream) {
    if (n <= 0) return 0;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    hk::k_test_exp_unbiased<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, y, n);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
