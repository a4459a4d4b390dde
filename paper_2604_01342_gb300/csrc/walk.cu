// State-walk kernel (any decay mode, M <= 64 with gradient, M <= 256 without).
//
// One warp walks one chunk at a time, starting from the chunk-start states
// S^_b, G^_b of the scan.  Lane l owns marks j = l + 32 r.  Per event k
// (paper, Appendix B, Eq. alpha_grad_recurrence with one decay per source):
//     S_k = D_k (S_{k-1} + e_{c_{k-1}}),   G_k = D_k (G_{k-1} + dt_k (S_{k-1} + e_{c_{k-1}}))
//     lambda_k = mu_{c_k} + sum_j alpha[c_k][j] beta_j S_{k,j}      (Eq. hawkes_excitation)
// and, with w_k = 1 / lambda_k (Eqs. grad_mu, grad_alpha, grad_gamma):
//     dmu[c_k] += w_k,  dalpha[c_k][j] += w_k beta_j S_{k,j},
//     dbeta_j += w_k alpha[c_k][j] (S_{k,j} - beta_j G_{k,j}).
// The compensator pieces of event k as a source, 1 - exp(-beta (T - t_k)) and
// (T - t_k) exp(-beta (T - t_k)), are summed per source mark.
//
// Events are processed 32 at a time: lane e loads event e (coalesced), each
// lane accumulates its marks' share of all 32 dot products, and one
// transposing butterfly (31 shuffles per lane) leaves lane e with the sum for
// event e.  The gradient needs w_k, so the 32 events are walked a second time
// from the saved batch-start state (recomputing the decays is cheaper than
// keeping 32 states per lane).  dt_k and T - t_k are FP64 differences rounded to
// FP32; the log-sum is taken as the log of an FP64 product (LogProd).
#include "common.cuh"

namespace hk {

int walk_max_m(int grad) { return grad ? 64 : 256; }

__device__ __forceinline__ float warp_transpose_reduce(float (&v)[32], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            float send = upper ? v[i] : v[i + o];
            float keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(HK_FULL, send, o);
        }
    }
    return v[0];
}

template <int R, bool GRAD>
__device__ void flush(const Problem& p, int32_t seq, float* E_s, float* F_s, float* dmu_s,
                      float* dal_s, float (&dbr)[R], LogProd& lp, int lane) {
    const int M = p.M;
    for (int j = lane; j < M; j += 32) {
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
        for (int i = lane; i < M * M; i += 32) {
            float a = dal_s[i];
            if (a != 0.f) atomicAdd(&p.dal_acc[(int64_t)seq * M * M + i], (double)a);
            dal_s[i] = 0.f;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int j = lane + 32 * r;
            if (j < M && dbr[r] != 0.f) atomicAdd(&p.dbe_acc[(int64_t)seq * M + j], (double)dbr[r]);
            dbr[r] = 0.f;
        }
    }
    double ll = lp.log_value();
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) ll += __shfl_xor_sync(HK_FULL, ll, o);
    if (lane == 0 && ll != 0.0) atomicAdd(&p.ll_acc[seq], ll);
    lp = LogProd();
    __syncwarp();
}

template <int R, bool GRAD>
__global__ void __launch_bounds__(128) k_walk(Problem p, int64_t chunks_per_warp) {
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31;
    const int M = p.M;
    const int per_warp = 2 * M + (GRAD ? M + M * M : 0);
    float* E_s = sm + (threadIdx.x >> 5) * per_warp;
    float* F_s = E_s + M;
    float* dmu_s = F_s + M;
    float* dal_s = dmu_s + M;
    if (failed(p.hdr)) return;
    for (int i = lane; i < per_warp; i += 32) E_s[i] = 0.f;
    __syncwarp();

    const int64_t nb = num_chunks(p);
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t b = gw * chunks_per_warp;
    const int64_t b_end = b + chunks_per_warp < nb ? b + chunks_per_warp : nb;

    int32_t cur = -1;
    float bj[R], dbr[R];
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
            if (cur >= 0) flush<R, GRAD>(p, cur, E_s, F_s, dmu_s, dal_s, dbr, lp, lane);
            cur = seq;
            T = p.Tarr[seq];
            mu = p.mu + (int64_t)seq * M;
            alpha = p.alpha + (int64_t)seq * M * M;
            beta_row = p.shared ? p.beta + seq : p.beta + (int64_t)seq * M;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int j = lane + 32 * r;
                bj[r] = p.shared ? beta_row[0] : (j < M ? beta_row[j] : 0.f);
            }
        }
        int64_t s0, s1;
        chunk_range(p, b, seq, s0, s1);
        float S[R], G[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int j = lane + 32 * r;
            S[r] = j < M ? p.Shat[b * M + j] : 0.f;
            G[r] = (GRAD && j < M) ? p.Ghat[b * M + j] : 0.f;
        }
        double t_carry = p.t[s0];
        int32_t c_carry = -1;
        for (int64_t base = s0; base < s1; base += 32) {
            const int64_t k = base + lane;
            const bool valid = k < s1;
            const int nvalid = (int)(s1 - base < 32 ? s1 - base : 32);
            const double tk = valid ? p.t[k] : t_carry;
            const int32_t ck = valid ? p.c[k] : 0;
            double tp = __shfl_up_sync(HK_FULL, tk, 1);
            int32_t cp = __shfl_up_sync(HK_FULL, ck, 1);
            if (lane == 0) { tp = t_carry; cp = c_carry; }
            const float dt = (k == s0) ? 0.f : (float)(tk - tp);
            const bool first = (k == s0);
            float dsh = 0.f;
            if (p.shared) dsh = expf(-bj[0] * dt);
            t_carry = __shfl_sync(HK_FULL, tk, 31);
            c_carry = __shfl_sync(HK_FULL, ck, 31);

            float S0[R], G0[R];
#pragma unroll
            for (int r = 0; r < R; ++r) { S0[r] = S[r]; G0[r] = G[r]; }

            float pp[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                pp[e] = 0.f;
                const float dte = __shfl_sync(HK_FULL, dt, e);
                const int32_t cpe = __shfl_sync(HK_FULL, cp, e);
                const int32_t cee = __shfl_sync(HK_FULL, ck, e);
                const bool fe = __shfl_sync(HK_FULL, first, e);
                const float de = __shfl_sync(HK_FULL, dsh, e);
                if (e < nvalid) {
                    const float* arow = alpha + (int64_t)cee * M;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        int j = lane + 32 * r;
                        if (!fe) {
                            float d = p.shared ? de : expf(-bj[r] * dte);
                            float P = S[r] + (j == cpe ? 1.f : 0.f);
                            if (GRAD) G[r] = d * (G[r] + dte * P);
                            S[r] = d * P;
                        }
                        if (j < M) pp[e] += __ldg(arow + j) * bj[r] * S[r];
                    }
                }
            }
            const float exc = warp_transpose_reduce(pp, lane);
            float w = 0.f;
            if (valid) {
                const float lam = __ldg(mu + ck) + exc;
                if (!(lam > 0.f)) set_status(p.hdr, HAWKES_ERR_NONPOS_INTENSITY);
                lp.mul(lam);
                w = 1.f / lam;
                const float bc = p.shared ? bj[0] : __ldg(beta_row + ck);
                const float x = (float)(T - tk);
                atomicAdd(&E_s[ck], -expm1f(-bc * x));
                if (GRAD) {
                    atomicAdd(&F_s[ck], x * expf(-bc * x));
                    atomicAdd(&dmu_s[ck], w);
                }
            }
            if (GRAD) {
#pragma unroll
                for (int r = 0; r < R; ++r) { S[r] = S0[r]; G[r] = G0[r]; }
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const float dte = __shfl_sync(HK_FULL, dt, e);
                    const int32_t cpe = __shfl_sync(HK_FULL, cp, e);
                    const int32_t cee = __shfl_sync(HK_FULL, ck, e);
                    const bool fe = __shfl_sync(HK_FULL, first, e);
                    const float de = __shfl_sync(HK_FULL, dsh, e);
                    const float we = __shfl_sync(HK_FULL, w, e);
                    if (e < nvalid) {
                        const float* arow = alpha + (int64_t)cee * M;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            int j = lane + 32 * r;
                            if (!fe) {
                                float d = p.shared ? de : expf(-bj[r] * dte);
                                float P = S[r] + (j == cpe ? 1.f : 0.f);
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
            __syncwarp();
        }
    }
    if (cur >= 0) flush<R, GRAD>(p, cur, E_s, F_s, dmu_s, dal_s, dbr, lp, lane);
}

cudaError_t launch_walk(const Problem& p, cudaStream_t s, int* nl) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int warps_per_block = 4;
    const int per_warp = 2 * p.M + (p.grad ? p.M + p.M * p.M : 0);
    size_t smem = sizeof(float) * (size_t)per_warp * warps_per_block;
    int64_t warps = (int64_t)sms * 16;
    if (warps > p.nb_max) warps = p.nb_max > 0 ? p.nb_max : 1;
    int64_t q = (p.nb_max + warps - 1) / warps;
    if (q < 1) q = 1;
    unsigned grid = (unsigned)((warps + warps_per_block - 1) / warps_per_block);
    cudaError_t err = cudaSuccess;
#define HK_WALK(RR, GG)                                                                      \
    do {                                                                                     \
        auto kern = k_walk<RR, GG>;                                                          \
        if (smem > 48 * 1024)                                                                \
            err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                       (int)smem);                                           \
        if (err == cudaSuccess) kern<<<grid, 32 * warps_per_block, smem, s>>>(p, q);         \
    } while (0)
    const int R = (p.M + 31) / 32;
    if (p.grad) {
        if (R <= 1) HK_WALK(1, true); else HK_WALK(2, true);
    } else {
        if (R <= 1) HK_WALK(1, false);
        else if (R <= 2) HK_WALK(2, false);
        else if (R <= 4) HK_WALK(4, false);
        else HK_WALK(8, false);
    }
#undef HK_WALK
    ++*nl;
    prof_mark(s, "walk");
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace hk
