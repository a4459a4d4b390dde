// State-walk kernel (any decay mode, M <= 64 with gradient, M <= 256 without).
//
// One warp walks one chunk at a time, starting from the chunk-start states
// S^_b, G^_b of the scan.  Lane l of a walker owns marks j = l + W r.  Per event k
// (paper, Appendix B, Eq. alpha_grad_recurrence with one decay per source):
//     S_k = D_k (S_{k-1} + e_{c_{k-1}}),   G_k = D_k (G_{k-1} + dt_k (S_{k-1} + e_{c_{k-1}}))
//     lambda_k = mu_{c_k} + sum_j alpha[c_k][j] beta_j S_{k,j}      (Eq. hawkes_excitation)
// and, with w_k = 1 / lambda_k (Eqs. grad_mu, grad_alpha, grad_gamma):
//     dmu[c_k] += w_k,  dalpha[c_k][j] += w_k beta_j S_{k,j},
//     dbeta_j += w_k alpha[c_k][j] (S_{k,j} - beta_j G_{k,j}).
// The compensator pieces of event k as a source, 1 - exp(-beta (T - t_k)) and
// (T - t_k) exp(-beta (T - t_k)), are summed per source mark.
//
// A walker is a group of W lanes (W = 32, or 8 / 16 when every mark fits one lane of the
// group, so that a warp walks 32 / W chunks at once; every shuffle and warp barrier names
// the group's lanes only, and all control flow is uniform within a group).  Events are
// processed W at a time: lane e loads event e (coalesced), each lane accumulates its marks'
// share of all W dot products, and one transposing butterfly leaves lane e with the sum for
// event e.  The gradient needs w_k, so the 32 events are walked a second time
// from the saved batch-start state (recomputing the decays is cheaper than
// keeping 32 states per lane).  dt_k and T - t_k are FP64 differences rounded to
// FP32; the log-sum is taken as the log of a running product (LogProd: FP32 mantissa,
// integer exponent).
//
// Within a batch the recurrence is taken in factorised form from the state (S0, G0)
// seen by its first event (time t_0; Delta_e = t_e - t_0):
//     S_e = exp(-beta_j Delta_e) (S0_j + U_j),
//     G_e = exp(-beta_j Delta_e) (G0_j + Delta_e (S0_j + U_j) - V_j),
// with U_j, V_j the sums of exp(beta_j Delta_l) and Delta_l exp(beta_j Delta_l) over the
// batch's earlier events l of mark j.  Each factor exp(-beta Delta_e) is used once, so
// the one-signed sub-ulp error of expf (kept for the 32 M per-source factors of a batch,
// the walk's most frequent operation) does not compound along the chain of events; the
// chained step from one batch start to the next, and the per-event factors, are taken
// with exp_unbiased.  A batch with beta * (t_last - t_0) above kWalkFactorLimit (where the
// growing factors exp(beta Delta) would lose range or precision) is walked event by
// event with exp_unbiased steps.
#include "common.cuh"

namespace hk {

int walk_max_m(int grad) { return grad ? 64 : 256; }

// Largest beta * (t_last - t_first) of a batch walked in the factorised form: keeps
// exp(+beta Delta) below e^64, so the sums U, V of 32 such terms and the factors
// exp(-beta Delta) stay normal FP32 numbers (the chunk-GEMM path uses the same bound).
// Delta_e U - V = sum_l (Delta_e - Delta_l) exp(beta Delta_l) loses about
// beta Delta_e / (beta (t_e - t_l)) ulps for a close pair (l, e) late in a wide batch: a
// relative error of at most ~1e-5 of that pair's term of G at beta (t_e - t_l) >= 0.01,
// of either sign, and G enters the decay gradient only as beta G next to S.
constexpr float kWalkFactorLimit = 64.f;

// Shared memory of one warp: E, F (and dmu, dalpha with the gradient) per-mark sums.
__host__ __device__ inline int walk_floats_per_warp(int M, bool grad) {
    return 2 * M + (grad ? M + M * M : 0);
}

// Lanes l of a group of W: v[e] holds lane l's share of event e's sum; afterwards lane l
// returns the total for event l (a transposing butterfly within the group).
template <int W>
__device__ __forceinline__ float group_transpose_reduce(float (&v)[W], int gl, unsigned gmask) {
#pragma unroll
    for (int o = W / 2; o >= 1; o >>= 1) {
        const bool upper = (gl & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            float send = upper ? v[i] : v[i + o];
            float keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(gmask, send, o, W);
        }
    }
    return v[0];
}

template <int R, bool GRAD, int W>
__device__ void flush(const Problem& p, int32_t seq, float* E_s, float* F_s, float* dmu_s,
                      float* dal_s, float (&dbr)[R], LogProd& lp, int gl, unsigned gmask) {
    const int M = p.M;
    for (int j = gl; j < M; j += W) {
        float e = E_s[j], f = F_s[j];
        if (e != 0.f) atomicAdd(&p.E_acc[(int64_t)seq * M + j], (double)e);
        if (GRAD && f != 0.f) atomicAdd(&p.F_acc[(int64_t)seq * M + j], (double)f);
        E_s[j] = 0.f;
        F_s[j] = 0.f;
        if (GRAD) {
            float m = dmu_s[j];
            if (m != 0.f) atomicAdd(&p.dmu_acc[(int64_t)seq * M + j], (double)m);
            dmu_s[j] = 0.f;
        }
    }
    if (GRAD) {
        for (int i = gl; i < M * M; i += W) {
            float a = dal_s[i];
            if (a != 0.f) atomicAdd(&p.dal_acc[(int64_t)seq * M * M + i], (double)a);
            dal_s[i] = 0.f;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int j = gl + W * r;
            if (j < M && dbr[r] != 0.f) atomicAdd(&p.dbe_acc[(int64_t)seq * M + j], (double)dbr[r]);
            dbr[r] = 0.f;
        }
    }
    double ll = lp.log_value();
#pragma unroll
    for (int o = W / 2; o >= 1; o >>= 1) ll += __shfl_xor_sync(gmask, ll, o, W);
    if (gl == 0 && ll != 0.0) atomicAdd(&p.ll_acc[seq], ll);
    lp = LogProd();
    __syncwarp(gmask);
}

template <int R, bool GRAD, int W>
__global__ void __launch_bounds__(128) k_walk(Problem p, int64_t chunks_per_warp) {
    extern __shared__ float sm[];
    constexpr int kGroups = 32 / W;               // groups of W lanes per warp, each a walker
    const int lane = threadIdx.x & 31, gl = lane % W, grp = lane / W;
    const unsigned gmask = W == 32 ? HK_FULL : (((1u << W) - 1u) << (grp * W));
    const int M = p.M;
    const int per_warp = walk_floats_per_warp(M, GRAD);
    float* E_s = sm + ((threadIdx.x >> 5) * kGroups + grp) * per_warp;
    float* F_s = E_s + M;
    float* dmu_s = F_s + M;
    float* dal_s = dmu_s + M;
    if (failed(p.hdr)) return;
    for (int i = gl; i < per_warp; i += W) E_s[i] = 0.f;
    __syncwarp(gmask);

    const int64_t nb = num_chunks(p);
    const int64_t gw = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * kGroups + grp;
    int64_t b = gw * chunks_per_warp;
    const int64_t b_end = b + chunks_per_warp < nb ? b + chunks_per_warp : nb;

    int32_t cur = -1;
    float bj[R], dbr[R], bmax = 0.f;
    LogProd lp;
    double T = 0.0;
    const float* mu = nullptr;
    const float* alpha = nullptr;
    const float* beta_row = nullptr;
#pragma unroll
    for (int r = 0; r < R; ++r) { bj[r] = 0.f; dbr[r] = 0.f; }

    for (; b < b_end; ++b) {
        const int32_t seq = p.chunk_seq[b];
        if (seq != cur) {
            if (cur >= 0) flush<R, GRAD, W>(p, cur, E_s, F_s, dmu_s, dal_s, dbr, lp, gl, gmask);
            cur = seq;
            T = p.Tarr[seq];
            mu = p.mu + (int64_t)seq * M;
            alpha = p.alpha + (int64_t)seq * M * M;
            beta_row = p.shared ? p.beta + seq : p.beta + (int64_t)seq * M;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int j = gl + W * r;
                bj[r] = p.shared ? beta_row[0] : (j < M ? beta_row[j] : 0.f);
            }
            float bm = 0.f;
#pragma unroll
            for (int r = 0; r < R; ++r) bm = fmaxf(bm, bj[r]);
#pragma unroll
            for (int o = W / 2; o >= 1; o >>= 1) bm = fmaxf(bm, __shfl_xor_sync(gmask, bm, o, W));
            bmax = bm;
        }
        int64_t s0, s1;
        chunk_range(p, b, seq, s0, s1);
        // S0, G0: the state seen by the first event of the current batch
        float S0[R], G0[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int j = gl + W * r;
            S0[r] = j < M ? p.Shat[b * M + j] : 0.f;
            G0[r] = (GRAD && j < M) ? p.Ghat[b * M + j] : 0.f;
        }
        for (int64_t base = s0; base < s1; base += W) {
            const int64_t k = base + gl;
            const bool valid = k < s1;
            const int nvalid = (int)(s1 - base < W ? s1 - base : W);
            const double tk = valid ? p.t[k] : p.t[base];
            const int32_t ck = valid ? p.c[k] : 0;
            const double t0 = __shfl_sync(gmask, tk, 0, W);
            const double tl = __shfl_sync(gmask, tk, nvalid - 1, W);
            const float De = (float)(tk - t0);             // Delta_e = t_e - t_0
            const float bc = p.shared ? bj[0] : __ldg(beta_row + ck);
            const bool fact = bmax * (float)(tl - t0) <= kWalkFactorLimit;   // group-uniform
            // factorised: exp(+beta_{c_e} Delta_e) of the own mark, and (one decay) exp(-beta Delta_e)
            const float ep = fact ? exp_unbiased(bc * De) : 0.f;
            const float emsh = (fact && p.shared) ? exp_unbiased(-bj[0] * De) : 0.f;
            // chained (batches spanning beta * span > kWalkFactorLimit): step from the previous event
            double tp = __shfl_up_sync(gmask, tk, 1, W);
            const int32_t cp = __shfl_up_sync(gmask, ck, 1, W);
            const float dt = gl == 0 ? 0.f : (float)(tk - tp);
            const float dsh = (!fact && p.shared) ? exp_unbiased(-bj[0] * dt) : 0.f;

            float U[R], V[R], S[R], G[R];
#pragma unroll
            for (int r = 0; r < R; ++r) { U[r] = 0.f; V[r] = 0.f; S[r] = S0[r]; G[r] = G0[r]; }
            float exc = 0.f;
            if (fact) {
                float pp[W];
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    pp[e] = 0.f;
                    const int32_t cee = __shfl_sync(gmask, ck, e, W);
                    const float Dee = __shfl_sync(gmask, De, e, W);
                    const float epe = __shfl_sync(gmask, ep, e, W);
                    const float eme = p.shared ? __shfl_sync(gmask, emsh, e, W) : 0.f;
                    if (e < nvalid) {
                        const float* arow = alpha + (int64_t)cee * M;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            int j = gl + W * r;
                            const float em = p.shared ? eme : expf(-bj[r] * Dee);
                            const float Sv = em * (S0[r] + U[r]);
                            if (j == cee) {
                                U[r] += epe;
                                if (GRAD) V[r] = fmaf(Dee, epe, V[r]);
                            }
                            if (j < M) pp[e] += __ldg(arow + j) * bj[r] * Sv;
                        }
                    }
                }
                exc = group_transpose_reduce<W>(pp, gl, gmask);
            } else {
                // event by event (rare): the dot product of event e by a warp sum
                for (int e = 0; e < nvalid; ++e) {
                    const int32_t cee = __shfl_sync(gmask, ck, e, W);
                    const float dte = __shfl_sync(gmask, dt, e, W);
                    const int32_t cpe = __shfl_sync(gmask, cp, e, W);
                    const float de = __shfl_sync(gmask, dsh, e, W);
                    const float* arow = alpha + (int64_t)cee * M;
                    float part = 0.f;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        int j = gl + W * r;
                        if (e > 0) {
                            const float d = p.shared ? de : exp_unbiased(-bj[r] * dte);
                            const float P = S[r] + (j == cpe ? 1.f : 0.f);
                            if (GRAD) G[r] = d * (G[r] + dte * P);
                            S[r] = d * P;
                        }
                        if (j < M) part += __ldg(arow + j) * bj[r] * S[r];
                    }
#pragma unroll
                    for (int o = W / 2; o >= 1; o >>= 1) part += __shfl_xor_sync(gmask, part, o, W);
                    if (gl == e) exc = part;
                }
            }
            float w = 0.f;
            if (valid) {
                const float lam = __ldg(mu + ck) + exc;
                if (!(lam > 0.f)) set_status(p.hdr, HAWKES_ERR_NONPOS_INTENSITY);
                lp.mul(lam);
                w = 1.f / lam;
                const float x = (float)(T - tk);
                atomicAdd(&E_s[ck], -expm1f(-bc * x));
                if (GRAD) {
                    atomicAdd(&F_s[ck], x * exp_unbiased(-bc * x));
                    atomicAdd(&dmu_s[ck], w);
                }
            }
            if (GRAD) {
#pragma unroll
                for (int r = 0; r < R; ++r) { U[r] = 0.f; V[r] = 0.f; S[r] = S0[r]; G[r] = G0[r]; }
                if (fact) {
#pragma unroll
                    for (int e = 0; e < W; ++e) {
                        const int32_t cee = __shfl_sync(gmask, ck, e, W);
                        const float Dee = __shfl_sync(gmask, De, e, W);
                        const float epe = __shfl_sync(gmask, ep, e, W);
                        const float eme = p.shared ? __shfl_sync(gmask, emsh, e, W) : 0.f;
                        const float we = __shfl_sync(gmask, w, e, W);
                        if (e < nvalid) {
                            const float* arow = alpha + (int64_t)cee * M;
#pragma unroll
                            for (int r = 0; r < R; ++r) {
                                int j = gl + W * r;
                                const float em = p.shared ? eme : expf(-bj[r] * Dee);
                                const float Sx = S0[r] + U[r];
                                const float Sv = em * Sx;
                                const float Gv = em * (G0[r] + fmaf(Dee, Sx, -V[r]));
                                if (j == cee) {
                                    U[r] += epe;
                                    V[r] = fmaf(Dee, epe, V[r]);
                                }
                                if (j < M) {
                                    dal_s[cee * M + j] += we * bj[r] * Sv;
                                    dbr[r] += we * __ldg(arow + j) * (Sv - bj[r] * Gv);
                                }
                            }
                        }
                    }
                } else {
                    for (int e = 0; e < nvalid; ++e) {
                        const int32_t cee = __shfl_sync(gmask, ck, e, W);
                        const float dte = __shfl_sync(gmask, dt, e, W);
                        const int32_t cpe = __shfl_sync(gmask, cp, e, W);
                        const float de = __shfl_sync(gmask, dsh, e, W);
                        const float we = __shfl_sync(gmask, w, e, W);
                        const float* arow = alpha + (int64_t)cee * M;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            int j = gl + W * r;
                            if (e > 0) {
                                const float d = p.shared ? de : exp_unbiased(-bj[r] * dte);
                                const float P = S[r] + (j == cpe ? 1.f : 0.f);
                                G[r] = d * (G[r] + dte * P);
                                S[r] = d * P;
                            }
                            if (j < M) {
                                dal_s[cee * M + j] += we * bj[r] * S[r];
                                dbr[r] += we * __ldg(arow + j) * (S[r] - bj[r] * G[r]);
                            }
                        }
                    }
                }
            }
            // advance to the first event of the next batch of this chunk
            if (base + W < s1) {
                const double tn = p.t[base + W];
                const int32_t cl = __shfl_sync(gmask, ck, W - 1, W);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int j = gl + W * r;
                    if (fact) {
                        // S0' = D (S0 + U), G0' = D (G0 + Dn (S0 + U) - V), one decay over t_0 -> t_n
                        const float Dn = (float)(tn - t0);
                        const float D = exp_unbiased(-bj[r] * Dn);
                        const float Sx = S0[r] + U[r];
                        if (GRAD) G0[r] = D * (G0[r] + fmaf(Dn, Sx, -V[r]));
                        S0[r] = D * Sx;
                    } else {
                        const float dn = (float)(tn - tl);
                        const float D = exp_unbiased(-bj[r] * dn);
                        const float P = S[r] + (j == cl ? 1.f : 0.f);
                        if (GRAD) G0[r] = D * (G[r] + dn * P);
                        S0[r] = D * P;
                    }
                }
            }
            __syncwarp(gmask);
        }
    }
    if (cur >= 0) flush<R, GRAD, W>(p, cur, E_s, F_s, dmu_s, dal_s, dbr, lp, gl, gmask);
}

cudaError_t launch_walk(const Problem& p, cudaStream_t s, int* nl) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // a walker is a group of W lanes (W = 8 or 16 when every mark fits one lane of it, so
    // that a warp walks 32 / W chunks at a time)
    const int W = p.walk_lanes ? p.walk_lanes : (p.M <= 8 ? 8 : (p.M <= 16 ? 16 : 32));
    const int groups = 32 / W;
    const int warps_per_block = 4;
    const int per_walker = walk_floats_per_warp(p.M, p.grad != 0);
    size_t smem = sizeof(float) * (size_t)per_walker * warps_per_block * groups;
    int64_t walkers = (int64_t)sms * 16 * groups;
    if (walkers > p.nb_max) walkers = p.nb_max > 0 ? p.nb_max : 1;
    int64_t q = (p.nb_max + walkers - 1) / walkers;
    if (q < 1) q = 1;
    const int64_t per_block = (int64_t)warps_per_block * groups;
    unsigned grid = (unsigned)((walkers + per_block - 1) / per_block);
    cudaError_t err = cudaSuccess;
#define HK_WALK(RR, GG, WW)                                                                  \
    do {                                                                                     \
        auto kern = k_walk<RR, GG, WW>;                                                      \
        if (smem > 48 * 1024)                                                                \
            err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                       (int)smem);                                           \
        if (err == cudaSuccess) kern<<<grid, 32 * warps_per_block, smem, s>>>(p, q);         \
    } while (0)
    const int R = (p.M + 31) / 32;
    if (p.grad) {
        if (W == 8) HK_WALK(1, true, 8);
        else if (W == 16) HK_WALK(1, true, 16);
        else if (R <= 1) HK_WALK(1, true, 32);
        else HK_WALK(2, true, 32);
    } else {
        if (W == 8) HK_WALK(1, false, 8);
        else if (W == 16) HK_WALK(1, false, 16);
        else if (R <= 1) HK_WALK(1, false, 32);
        else if (R <= 2) HK_WALK(2, false, 32);
        else if (R <= 4) HK_WALK(4, false, 32);
        else HK_WALK(8, false, 32);
    }
#undef HK_WALK
    ++*nl;
    prof_mark(s, "walk");
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace hk
