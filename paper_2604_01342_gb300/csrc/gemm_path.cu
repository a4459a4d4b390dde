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
#include "common.cuh"

namespace hk {

cudaError_t launch_finalize_mode(const Problem& p, cudaStream_t s, int mode, int* nl);

// ---------------------------------------------------------------------------
// FP32 CUDA-core GEMM  C[m][n] (+)= sum_k A(m, k) B(n, k) with general strides.
// 64 x 64 tile, 256 threads, 4 x 4 outputs per thread, k-step 16.
// ---------------------------------------------------------------------------
struct GemmArgs {
    const float* A; int64_t a_m, a_k;   // A(m,k) = A[m*a_m + k*a_k]
    const float* B; int64_t b_n, b_k;   // B(n,k) = B[n*b_n + k*b_k]
    float* C; int64_t c_m, c_n;         // C(m,n) = C[m*c_m + n*c_n]
    int64_t Mdim, Ndim, Kdim;
    int64_t k_per_split;                // split-K slice length (atomic accumulate if split)
    const int64_t* kdim_dev;            // if set, K is clipped to *kdim_dev (device count)
    int atomic;
};

__global__ void __launch_bounds__(256) k_sgemm(GemmArgs g, const WsHeader* hdr) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    if (failed(hdr)) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    const int64_t k_begin = (int64_t)blockIdx.z * g.k_per_split;
    int64_t k_end = k_begin + g.k_per_split;
    int64_t kdim = g.Kdim;
    if (g.kdim_dev && *g.kdim_dev < kdim) kdim = *g.kdim_dev;
    if (k_end > kdim) k_end = kdim;
    float acc[4][4] = {};
    for (int64_t k0 = k_begin; k0 < k_end; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            int kk = i & 15, mm = i >> 4;
            int64_t gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < g.Mdim && gk < k_end) ? g.A[gm * g.a_m + gk * g.a_k] : 0.f;
            int64_t gn = n0 + mm;
            Bs[kk][mm] = (gn < g.Ndim && gk < k_end) ? g.B[gn * g.b_n + gk * g.b_k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < g.Mdim && gn < g.Ndim) {
                float* dst = g.C + gm * g.c_m + gn * g.c_n;
                if (g.atomic) atomicAdd(dst, acc[i][j]);
                else *dst = acc[i][j];
            }
        }
}

static cudaError_t sgemm(const GemmArgs& g0, int splits, const WsHeader* hdr, cudaStream_t s) {
    GemmArgs g = g0;
    if (splits < 1) splits = 1;
    g.k_per_split = ((g.Kdim + splits - 1) / splits + 15) / 16 * 16;
    if (g.k_per_split < 16) g.k_per_split = 16;
    splits = (int)((g.Kdim + g.k_per_split - 1) / g.k_per_split);
    if (splits < 1) splits = 1;
    g.atomic = splits > 1 ? 1 : g.atomic;
    dim3 grid((unsigned)((g.Ndim + 63) / 64), (unsigned)((g.Mdim + 63) / 64), (unsigned)splits);
    k_sgemm<<<grid, 256, 0, s>>>(g, hdr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-chunk epilogue: intra-chunk pairs, lambda, log, weights, gradient pieces.
// One block per chunk; the chunk's events are staged in shared memory.
// ---------------------------------------------------------------------------
template <bool GRAD>
__global__ void __launch_bounds__(256) k_chunk_epilogue(Problem p) {
    extern __shared__ unsigned char smraw[];
    const int M = p.M;
    const int C = p.C;
    double* tsh = (double*)smraw;                // [C]
    int32_t* csh = (int32_t*)(tsh + C);          // [C]
    float* wsh = (float*)(csh + C);              // [C]  w_k
    float* Wrow = wsh + C;                       // [M]  W[b][:]
    __shared__ double red_ll[8];
    __shared__ float red_db[8];
    if (failed(p.hdr)) return;
    const int64_t nb = num_chunks(p);
    const float beta = p.beta[0];
    const double T = p.Tarr[0];
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        int64_t s0, s1;
        chunk_range(p, b, 0, s0, s1);
        const int n = (int)(s1 - s0);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            tsh[i] = p.t[s0 + i];
            csh[i] = p.c[s0 + i];
        }
        if (GRAD)
            for (int j = threadIdx.x; j < M; j += blockDim.x) Wrow[j] = 0.f;
        __syncthreads();
        const double tau = tsh[0];
        double ll = 0.0;
        float db = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double tk = tsh[i];
            const int ck = csh[i];
            const float* arow = p.alpha + (int64_t)ck * M;
            float A = 0.f, Bp = 0.f;
            for (int l = 0; l < i; ++l) {
                const float x = (float)(tk - tsh[l]);
                const float e = expf(-beta * x) * __ldg(arow + csh[l]);
                A += e;
                if (GRAD) Bp += x * e;
            }
            const float delta = (float)(tk - tau);
            const float ek = expf(-beta * delta);
            const float y = p.Y[b * M + ck];
            const float aS = ek * y + A;
            const float lam = p.mu[ck] + beta * aS;
            if (!(lam > 0.f)) set_status(p.hdr, HAWKES_ERR_NONPOS_INTENSITY);
            ll += (double)logf(lam);
            const float w = 1.f / lam;
            const float xT = (float)(T - tk);
            atomicAdd(&p.E_acc[ck], (double)(-expm1f(-beta * xT)));
            if (GRAD) {
                const float z = p.Z[b * M + ck];
                const float aG = ek * (delta * y + z) + Bp;
                db += w * (aS - beta * aG);
                wsh[i] = w;
                atomicAdd(&Wrow[ck], w * ek);
                atomicAdd(&p.dmu_acc[ck], (double)w);
                atomicAdd(&p.F_acc[ck], (double)(xT * expf(-beta * xT)));
            }
        }
        // block reductions
        for (int o = 16; o >= 1; o >>= 1) {
            ll += __shfl_xor_sync(HK_FULL, ll, o);
            db += __shfl_xor_sync(HK_FULL, db, o);
        }
        if ((threadIdx.x & 31) == 0) { red_ll[threadIdx.x >> 5] = ll; red_db[threadIdx.x >> 5] = db; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, d = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red_ll[w]; d += red_db[w]; }
            atomicAdd(&p.ll_acc[0], a);
            if (GRAD) atomicAdd(&p.dbe_acc[0], d);
        }
        if (GRAD) {
            // intra-chunk pairs of dalpha (without the factor beta)
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const double tk = tsh[i];
                const float w = wsh[i];
                double* drow = p.dal_acc + (int64_t)csh[i] * M;
                for (int l = 0; l < i; ++l) {
                    const float x = (float)(tk - tsh[l]);
                    atomicAdd(drow + csh[l], (double)(w * expf(-beta * x)));
                }
            }
            for (int j = threadIdx.x; j < M; j += blockDim.x) p.W[b * M + j] = Wrow[j];
        }
        __syncthreads();
    }
}

cudaError_t launch_gemm_path(const Problem& p, cudaStream_t s, int* nl) {
    cudaError_t err;
    const int64_t M = p.M, nb = p.nb_max;
    // Y = Shat alpha^T, Z = Ghat alpha^T   (rows = chunks)
    {
        GemmArgs g{};
        g.A = p.Shat; g.a_m = M; g.a_k = 1;
        g.B = p.alpha; g.b_n = M; g.b_k = 1;
        g.C = p.Y; g.c_m = M; g.c_n = 1;
        g.Mdim = nb; g.Ndim = M; g.Kdim = M; g.atomic = 0;
        if ((err = sgemm(g, 1, p.hdr, s)) != cudaSuccess) return err;
        ++*nl;
        prof_mark(s, "gemm_Y");
        if (p.grad) {
            g.A = p.Ghat; g.C = p.Z;
            if ((err = sgemm(g, 1, p.hdr, s)) != cudaSuccess) return err;
            ++*nl;
            prof_mark(s, "gemm_Z");
        }
    }
    {
        size_t smem = (size_t)p.C * (8 + 4 + 4) + sizeof(float) * (size_t)M;
        auto kern = p.grad ? k_chunk_epilogue<true> : k_chunk_epilogue<false>;
        if (smem > 48 * 1024) {
            err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
        }
        int64_t grid = nb < 65535 * 16 ? nb : 65535 * 16;
        kern<<<(unsigned)(grid > 0 ? grid : 1), 256, smem, s>>>(p);
        ++*nl;
        prof_mark(s, "chunk_epilogue");
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (p.grad) {
        // dal_gemm[i][j] = sum_b W[b][i] Shat[b][j]   (split over chunks, atomic accumulate)
        cudaMemsetAsync(p.dal_gemm, 0, sizeof(float) * (size_t)M * M, s);
        GemmArgs g{};
        g.A = p.W; g.a_m = 1; g.a_k = M;
        g.B = p.Shat; g.b_n = 1; g.b_k = M;
        g.C = p.dal_gemm; g.c_m = M; g.c_n = 1;
        g.Mdim = M; g.Ndim = M; g.Kdim = nb; g.atomic = 1;
        g.kdim_dev = p.chunk_base + p.B;
        int splits = (int)((nb + 1023) / 1024);
        if ((err = sgemm(g, splits, p.hdr, s)) != cudaSuccess) return err;
        ++*nl;
        prof_mark(s, "gemm_dalpha");
    }
    return launch_finalize_mode(p, s, 1, nl);
}

}  // namespace hk
