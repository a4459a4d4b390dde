// Assemble L and the gradient from the accumulated sums (one block per sequence).
//   L          = sum_k log lambda_k - T sum_i mu_i - sum_j colsum_j E_j
//                (paper, Eq. general_hawkes_likelihood with the closed-form compensator)
//   dL/dmu_i   = sum_{k: c_k = i} w_k - T                                  (Eq. grad_mu)
//   dL/dalpha  = X_ij - E_j,  X_ij = beta_j sum_{k: c_k = i} w_k S_{k,j}     (Eq. grad_alpha)
//   dL/dbeta_j = Y_j - colsum_j F_j                                        (Eq. grad_gamma,
//                rewritten with the derivative state G)
// with colsum_j = sum_i alpha[i][j], E_j = sum_{l: c_l = j} (1 - exp(-beta_j (T - t_l))),
// F_j = sum_{l: c_l = j} (T - t_l) exp(-beta_j (T - t_l)).  A shared decay sums
// dbeta over j.  If the device status word is set, every output is NaN.
#include "common.cuh"

namespace hk {

// mode 0: X = dal_acc (already carries beta_j);
// mode 1: X = beta * (dal_gemm + dal_acc)  (chunk-GEMM path, one shared beta)
__global__ void k_finalize(Problem p, int mode) {
    const int s = blockIdx.x;
    const int M = p.M;
    const bool bad = failed(p.hdr);
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    const float* alpha = p.alpha + (int64_t)s * M * M;
    const float* mu = p.mu + (int64_t)s * M;
    const double T = p.Tarr[s];
    __shared__ double red_comp[32], red_mu[32], red_be[32];
    double comp = 0.0, summu = 0.0, dbsum = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        double cs = 0.0;
        for (int i = 0; i < M; ++i) cs += (double)alpha[(int64_t)i * M + j];
        const double E = p.E_acc[(int64_t)s * M + j];
        comp += cs * E;
        summu += (double)mu[j];
        if (p.grad) {
            double db = p.dbe_acc[(int64_t)s * M + j] - cs * p.F_acc[(int64_t)s * M + j];
            if (p.shared) dbsum += db;
            else p.d_beta[(int64_t)s * M + j] = bad ? (float)nanv : (float)db;
            p.d_mu[(int64_t)s * M + j] =
                bad ? (float)nanv : (float)(p.dmu_acc[(int64_t)s * M + j] - T);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o >= 1; o >>= 1) {
        comp += __shfl_xor_sync(HK_FULL, comp, o);
        summu += __shfl_xor_sync(HK_FULL, summu, o);
        dbsum += __shfl_xor_sync(HK_FULL, dbsum, o);
    }
    if (lane == 0) { red_comp[wid] = comp; red_mu[wid] = summu; red_be[wid] = dbsum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double c = 0.0, m = 0.0, b = 0.0;
        for (int w = 0; w < nw; ++w) { c += red_comp[w]; m += red_mu[w]; b += red_be[w]; }
        p.out_ll[s] = bad ? nanv : p.ll_acc[s] - T * m - c;
        if (p.grad && p.shared) p.d_beta[s] = bad ? (float)nanv : (float)b;
    }
    if (p.grad) {
        const float beta = p.shared ? p.beta[s] : 0.f;
        for (int64_t e = threadIdx.x; e < (int64_t)M * M; e += blockDim.x) {
            const int j = (int)(e % M);
            double x;
            if (mode == 0) x = p.dal_acc[(int64_t)s * M * M + e];
            else x = (double)beta * ((double)p.dal_gemm[e] + p.dal_acc[e]);
            const double v = x - p.E_acc[(int64_t)s * M + j];
            p.d_alpha[(int64_t)s * M * M + e] = bad ? (float)nanv : (float)v;
        }
    }
}

cudaError_t launch_finalize_mode(const Problem& p, cudaStream_t s, int mode, int* nl) {
    k_finalize<<<p.B, 256, 0, s>>>(p, mode);
    ++*nl;
    prof_mark(s, "finalize");
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Problem& p, cudaStream_t s, int* nl) {
    return launch_finalize_mode(p, s, 0, nl);
}

}  // namespace hk
