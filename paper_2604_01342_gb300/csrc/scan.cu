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
//   B: one thread per mark scans the group composites in order -> carry into each group
//   C: each block re-walks its group from the carry and writes S^_b, G^_b per chunk.
// Within a chunk the decay is applied to the whole state once and the chunk's
// events are added with shared-memory atomics, so S is never held per event.
#include "common.cuh"

namespace hk {

// PHASE 0 = A (compose from zero), 1 = C (re-walk from carry and write states).
template <int PHASE, bool GRAD>
__global__ void __launch_bounds__(256) k_scan_group(Problem p) {
    extern __shared__ float sm[];
    float* S = sm;
    float* G = sm + p.M;
    __shared__ double span_sh;
    __shared__ int reset_sh;
    if (failed(p.hdr)) return;
    const int64_t nb = num_chunks(p);
    const int64_t g = blockIdx.x;
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
    if (threadIdx.x == 0) { span_sh = 0.0; reset_sh = 0; }
    __syncthreads();
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
        if (last) {
            for (int j = threadIdx.x; j < M; j += blockDim.x) {
                S[j] = 0.f;
                if (GRAD) G[j] = 0.f;
            }
            if (threadIdx.x == 0) { span_sh = 0.0; reset_sh = 1; }
            __syncthreads();
            continue;
        }
        const double tn = p.t[s1];            // start of the next chunk
        const float D = (float)(tn - p.t[s0]);
        for (int j = threadIdx.x; j < M; j += blockDim.x) {
            float d = expf(-beta_of(p, seq, j) * D);
            float s = S[j];
            if (GRAD) G[j] = d * (G[j] + D * s);
            S[j] = d * s;
        }
        if (threadIdx.x == 0) span_sh += (tn - p.t[s0]);
        __syncthreads();
        for (int64_t l = s0 + threadIdx.x; l < s1; l += blockDim.x) {
            int32_t cl = p.c[l];
            float x = (float)(tn - p.t[l]);
            float e = expf(-beta_of(p, seq, cl) * x);
            atomicAdd(&S[cl], e);
            if (GRAD) atomicAdd(&G[cl], x * e);
        }
        __syncthreads();
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
template <bool GRAD>
__global__ void k_scan_carry(Problem p) {
    if (failed(p.hdr)) return;
    const int64_t nb = num_chunks(p);
    const int64_t ng = (nb + p.Gc - 1) / p.Gc;
    const int M = p.M;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        float cS = 0.f, cG = 0.f;
        constexpr int U = 8;
        for (int64_t g0 = 0; g0 < ng; g0 += U) {
            float v[U], gg[U], dt[U];
            int rs[U], sq[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int64_t g = g0 + u;
                if (g < ng) {
                    v[u] = p.grp_v[g * M + j];
                    gg[u] = GRAD ? p.grp_g[g * M + j] : 0.f;
                    dt[u] = (float)p.grp_dt[g];
                    rs[u] = p.grp_reset[g];
                    sq[u] = p.chunk_seq[g * p.Gc];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int64_t g = g0 + u;
                if (g < ng) {
                    p.carry_S[g * M + j] = cS;
                    if (GRAD) p.carry_G[g * M + j] = cG;
                    if (rs[u]) {
                        cS = v[u];
                        cG = gg[u];
                    } else {
                        float d = expf(-beta_of(p, sq[u], j) * dt[u]);
                        if (GRAD) cG = d * (cG + dt[u] * cS) + gg[u];
                        cS = d * cS + v[u];
                    }
                }
            }
        }
    }
}

cudaError_t launch_scan(const Problem& p, cudaStream_t s, int* nl) {
    size_t smem = sizeof(float) * 2 * (size_t)p.M;
    unsigned grid = (unsigned)(p.ng_max > 0 ? p.ng_max : 1);
    unsigned cgrid = (unsigned)((p.M + 127) / 128);
    if (p.grad) {
        k_scan_group<0, true><<<grid, 256, smem, s>>>(p);
        prof_mark(s, "scan_reduce");
        k_scan_carry<true><<<cgrid, 128, 0, s>>>(p);
        prof_mark(s, "scan_carry");
        k_scan_group<1, true><<<grid, 256, smem, s>>>(p);
        prof_mark(s, "scan_states");
    } else {
        k_scan_group<0, false><<<grid, 256, smem, s>>>(p);
        prof_mark(s, "scan_reduce");
        k_scan_carry<false><<<cgrid, 128, 0, s>>>(p);
        prof_mark(s, "scan_carry");
        k_scan_group<1, false><<<grid, 256, smem, s>>>(p);
        prof_mark(s, "scan_states");
    }
    *nl += 3;
    return cudaGetLastError();
}

}  // namespace hk
