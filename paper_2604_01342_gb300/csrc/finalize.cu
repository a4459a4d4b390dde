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

// Column sums colsum[s][j] = sum_i alpha[s][i][j] in FP64: block (32 columns x 8 row groups).
__global__ void k_colsum(Problem p, double* colsum) {
    __shared__ double part[8][33];
    const int M = p.M, s = blockIdx.y;
    const int j = blockIdx.x * 32 + threadIdx.x;
    const float* alpha = p.alpha + (int64_t)s * M * M;
    double acc = 0.0;
    if (j < M)
        for (int i = threadIdx.y; i < M; i += 8) acc += (double)alpha[(int64_t)i * M + j];
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && j < M) {
        double t = 0.0;
        for (int r = 0; r < 8; ++r) t += part[r][threadIdx.x];
        colsum[(int64_t)s * M + j] = t;
    }
}

// Per-sequence scalars and vectors: L, dmu, dbeta.  One block per sequence.
__global__ void k_finalize_vec(Problem p, const double* colsum) {
    const int s = blockIdx.x;
    const int M = p.M;
    const bool bad = failed(p.hdr);
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    const float* mu = p.mu + (int64_t)s * M;
    const double T = p.Tarr[s];
    __shared__ double red_comp[32], red_mu[32], red_be[32];
    double comp = 0.0, summu = 0.0, dbsum = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const double cs = colsum[(int64_t)s * M + j];
        comp += cs * p.E_acc[(int64_t)s * M + j];
        summu += (double)mu[j];
        if (p.grad) {
            const double db = p.dbe_acc[(int64_t)s * M + j] - cs * p.F_acc[(int64_t)s * M + j];
            if (p.shared) dbsum += db;
            else p.d_beta[(int64_t)s * M + j] = bad ? (float)nanv : (float)db;
            p.d_mu[(int64_t)s * M + j] =
                bad ? (float)nanv
                    : (float)(p.dmu_acc[(int64_t)s * M + j] - (p.base_term ? T : 0.0));
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
        p.out_ll[s] = bad ? nanv : p.ll_acc[s] - (p.base_term ? T * m : 0.0) - c;
        if (p.grad && p.shared) p.d_beta[s] = bad ? (float)nanv : (float)b;
    }
}

// dalpha for all sequences, elementwise.
// Entries outside alpha's support are 0 when the caller asked for the gradient on the
// support (p.support).
// mode 0: X = dal_acc (already carries beta_j);
// mode 1: X = beta * (dal_gemm + m_j wsum_i + sum_k part_k[i][j])  (chunk-GEMM path, one
//         shared beta; the GEMM ran on S^ - m, so m_j sum_b W[b][i] restores the centre;
//         part_k are the shares of row i's row block written by the backward pair blocks of
//         the plan, rows of M floats, summed in share order).
__global__ void k_finalize_alpha(Problem p, int mode) {
    const int M = p.M;
    const bool bad = failed(p.hdr);
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    if (mode == 0) {
        const int64_t total = (int64_t)p.B * M * M;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
             e += (int64_t)gridDim.x * blockDim.x) {
            const int64_t s = e / ((int64_t)M * M), ij = e % ((int64_t)M * M);
            const int j = (int)(ij % M);
            double v = p.dal_acc[e] - p.E_acc[s * M + j];
            if (p.support && p.alpha[e] == 0.f) v = 0.0;     // outside alpha's support
            p.d_alpha[e] = bad ? (float)nanv : (float)v;
        }
        return;
    }
    // one block row per dalpha row i (blockIdx.y), its columns over blockIdx.x and the threads
    const float beta = p.beta[0];
    const int i = blockIdx.y;
    const int P = p.P, R = 1 << p.lgR;
    // row i = I + P pos is row pos mod R of row block I nrb + pos / R
    const int I = i % P, pos = i / P;
    const int rb = I * p.nrb + (pos >> p.lgR);
    const int nr = bad ? 0 : p.plan_b[1 + rb];
    const int base = bad ? 0 : p.plan_b[1 + p.n_rb + rb];
    const double wsum = p.wsum_acc[i];
    const int64_t step = (int64_t)R * M;
    const float* part0 = p.dal_part + (((int64_t)base << p.lgR) + (pos & (R - 1))) * M;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const int64_t ij = (int64_t)i * M + j;
        // compensated FP32 sum of the shares, in share order (FP64 arithmetic runs at 1/64 of
        // the FP32 rate here); four shares loaded at a time
        float pairs = 0.f, comp = 0.f;
        const float* part = part0 + j;
        int k = 0;
        for (; k + 4 <= nr; k += 4) {
            const float y4[4] = {part[k * step], part[(k + 1) * step], part[(k + 2) * step],
                                 part[(k + 3) * step]};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float y = y4[u] - comp;
                const float t = pairs + y;
                comp = (t - pairs) - y;
                pairs = t;
            }
        }
        for (; k < nr; ++k) {
            const float y = part[k * step] - comp;
            const float t = pairs + y;
            comp = (t - pairs) - y;
            pairs = t;
        }
        const double x = (double)beta * ((double)p.dal_gemm[ij] + (double)p.cen_S[j] * wsum +
                                         (double)pairs);
        double v = x - p.E_acc[j];
        if (p.support && p.alpha[ij] == 0.f) v = 0.0;       // outside alpha's support
        p.d_alpha[ij] = bad ? (float)nanv : (float)v;
    }
}

cudaError_t launch_finalize_mode(const Problem& p, cudaStream_t s, int mode, int* nl) {
    k_colsum<<<dim3((unsigned)((p.M + 31) / 32), (unsigned)p.B), dim3(32, 8), 0, s>>>(p, p.colsum);
    k_finalize_vec<<<p.B, 256, 0, s>>>(p, p.colsum);
    *nl += 2;
    if (p.grad) {
        int64_t total = (int64_t)p.B * p.M * p.M;
        int64_t blocks = (total + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        if (mode == 0)
            k_finalize_alpha<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(p, mode);
        else
            k_finalize_alpha<<<dim3((unsigned)((p.M + 255) / 256), (unsigned)p.M), 256, 0, s>>>(p, mode);
        ++*nl;
    }
    prof_mark(s, "finalize");
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Problem& p, cudaStream_t s, int* nl) {
    return launch_finalize_mode(p, s, 0, nl);
}

// Last step for several decay kernels: L = slice 0's value (its log-sum, -T sum mu and its
// compensator) + every other slice's (minus its compensator); the first (smallest) error
// code of any slice becomes the caller's, and then every output is NaN.
__global__ void k_finalize_multi(Problem p, MultiSlices ms) {
    __shared__ int code_sh;
    if (threadIdx.x == 0) {
        int code = 0;
        for (int q = 0; q < ms.K; ++q) {
            const int s = ms.k[q].hdr->status;
            if (s != 0 && (code == 0 || s < code)) code = s;
        }
        code_sh = code;
        if (code != 0) p.hdr->status = code;
        if (blockIdx.x == 0 && code == 0) {
            double ll = ms.k[0].out_ll[0];
            for (int q = 1; q < ms.K; ++q) ll += ms.k[q].out_ll[0];
            p.out_ll[0] = ll;
        }
    }
    __syncthreads();
    if (code_sh == 0) return;
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    const float nanf = (float)nanv;
    const int64_t M = p.M, KM2 = (int64_t)ms.K * M * M;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i0 == 0) p.out_ll[0] = nanv;
    if (p.grad) {
        for (int64_t i = i0; i < M; i += stride) p.d_mu[i] = nanf;
        for (int64_t i = i0; i < KM2; i += stride) p.d_alpha[i] = nanf;
        for (int64_t i = i0; i < ms.K; i += stride) p.d_beta[i] = nanf;
    }
}

// p: the caller's view (slice 0's workspace, all K kernels' gradient outputs).
cudaError_t launch_finalize_multi(const Problem& p, const MultiSlices& ms, cudaStream_t s, int* nl) {
    int64_t total = (int64_t)ms.K * p.M * p.M;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_finalize_multi<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(p, ms);
    ++*nl;
    return cudaGetLastError();
}

}  // namespace hk
