// Ingest and validation (integer work, bit-exact):
//   - parameter domain checks (mu > 0, alpha >= 0, beta > 0, all finite; T finite >= 0)
//   - the chunk table: per-sequence chunk counts ceil(len / C), their exclusive scan
//     (chunk_base) and the owning sequence of every chunk (chunk_seq)
//   - event checks: sorted inside each sequence, 0 <= t <= T, 0 <= c < M, and
//     per-(sequence, mark) event counts.
// Paper, Section 2: the event sequence H = {(t_i, m_i)} is ordered in time on
// [0, T] with marks in {1..M} (0-based here); Section 3.3 splits it into
// contiguous batches, which are the chunks below.
#include "common.cuh"

namespace hk {

__global__ void k_init(Problem p, double* acc, int64_t n_acc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (i == 0) {
        p.hdr->status = 0;
        p.hdr->validated = 0;
        p.hdr->nb = 0;
        p.hdr->pad[8] = 0;   // work counter of the forward pair kernel / the mark-major walk
        p.hdr->pad[9] = 0;   // longest support row (mark-major walk)
        p.hdr->pad[12] = 0;  // ticket of the backward pair plan
        if (p.single) {
            p.hdr->pad[0] = 0;
            p.hdr->pad[1] = p.N;
            p.hdr->pad[2] = __double_as_longlong(p.T_single);
        }
    }
    for (; i < n_acc; i += stride) acc[i] = 0.0;
}

__global__ void k_check_params(Problem p) {
    int64_t nmu = (int64_t)p.B * p.M;
    int64_t nal = nmu * p.M;
    int64_t nbe = p.shared ? p.B : nmu;
    int64_t total = nmu + nal + nbe + p.B;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += stride) {
        bool ok;
        if (i < nmu) {
            float v = p.mu[i];
            ok = v > 0.f && isfinite(v);
        } else if (i < nmu + nal) {
            float v = p.alpha[i - nmu];
            ok = v >= 0.f && isfinite(v);
        } else if (i < nmu + nal + nbe) {
            float v = p.beta[i - nmu - nal];
            ok = v > 0.f && isfinite(v);
        } else {
            double T = p.Tarr[i - nmu - nal - nbe];
            ok = T >= 0.0 && isfinite(T);
            if (!ok) { set_status(p.hdr, HAWKES_ERR_INVALID_ARG); continue; }
        }
        if (!ok) set_status(p.hdr, HAWKES_ERR_PARAM_DOMAIN);
    }
}

// One block: chunk counts per sequence and their exclusive scan.
__global__ void k_chunk_table(Problem p) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        carry = 0;
        if (p.off[0] != 0 || p.off[p.B] != p.N) set_status(p.hdr, HAWKES_ERR_INVALID_ARG);
    }
    __syncthreads();
    for (int64_t base = 0; base < p.B; base += blockDim.x) {
        int64_t s = base + threadIdx.x;
        int64_t n = 0;
        if (s < p.B) {
            int64_t len = p.off[s + 1] - p.off[s];
            if (len < 0) { set_status(p.hdr, HAWKES_ERR_INVALID_ARG); len = 0; }
            n = (len + p.C - 1) / p.C;
        }
        // inclusive warp scan
        int64_t x = n;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(HK_FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int64_t w = lane < nw ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(HK_FULL, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) warp_tot[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        int64_t excl = carry + x - n + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (s < p.B) p.chunk_base[s] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + n;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int64_t nb = carry;
        if (nb > p.nb_max) { set_status(p.hdr, HAWKES_ERR_INVALID_ARG); nb = p.nb_max; }
        p.chunk_base[p.B] = nb;
        p.hdr->nb = nb;
    }
}

__global__ void k_chunk_seq(Problem p) {
    if (failed(p.hdr)) return;
    for (int64_t s = blockIdx.x; s < p.B; s += gridDim.x) {
        int64_t b0 = p.chunk_base[s], b1 = p.chunk_base[s + 1];
        for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) p.chunk_seq[b] = (int32_t)s;
    }
}

// Event checks and per-(sequence, mark) counts.  Each block takes a run of
// chunks; counts go through a shared-memory histogram when the run's
// sequences fit in it, else straight to global atomics.
constexpr int kHistMax = 4096;

// Order key of a time: the bit pattern of a non-negative double (-0 as +0); a negative value
// or a NaN maps above every finite non-negative time.
__device__ __forceinline__ uint64_t time_key(double t) {
    const uint64_t u = (uint64_t)__double_as_longlong(t);
    if (u == 0x8000000000000000ull) return 0ull;
    return (u >> 63) ? ~0ull : u;
}

// Chunks [b_begin, b_end) of the call (b_end clipped to the number of chunks).
__global__ void k_validate_events(Problem p, int chunks_per_block, int64_t b_begin, int64_t b_end) {
    __shared__ int32_t hist[kHistMax];
    if (failed(p.hdr)) return;
    const int64_t nb = num_chunks(p) < b_end ? num_chunks(p) : b_end;
    const int64_t b0 = b_begin + (int64_t)blockIdx.x * chunks_per_block;
    if (b0 >= nb) return;
    const int64_t b1 = b0 + chunks_per_block < nb ? b0 + chunks_per_block : nb;
    const int32_t seq0 = p.chunk_seq[b0], seq1 = p.chunk_seq[b1 - 1];
    const int64_t span = (int64_t)(seq1 - seq0 + 1) * p.M;
    const bool use_hist = span <= kHistMax;
    if (use_hist)
        for (int i = threadIdx.x; i < span; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    int bad = 0;
    if (p.B == 1) {
        // one sequence: the block's chunks are one run of events [e0, e1), taken four events
        // per thread and step with their loads issued together
        int64_t e0, e1, x0, x1;
        chunk_range(p, b0, 0, e0, x0);
        chunk_range(p, b1 - 1, 0, x1, e1);
        const uint64_t Tkey = time_key(p.Tarr[0]);
        const int64_t first = p.off[0];
        constexpr int U = 4;
        const int nt = blockDim.x;
        for (int64_t kb = e0 + threadIdx.x; kb < e1; kb += (int64_t)U * nt) {
            uint64_t key[U], prev[U];
            int32_t ck[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = kb + (int64_t)u * nt;
                const bool in = k < e1;
                key[u] = in ? time_key(__ldg(p.t + k)) : 0ull;
                prev[u] = (in && k > first) ? time_key(__ldg(p.t + k - 1)) : 0ull;
                ck[u] = in ? __ldg(p.c + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (kb + (int64_t)u * nt >= e1) break;
                if (key[u] > Tkey) bad = bad ? bad : HAWKES_ERR_TIME_RANGE;
                if (key[u] < prev[u]) bad = bad ? bad : HAWKES_ERR_UNSORTED;
                if (ck[u] < 0 || ck[u] >= p.M) { bad = bad ? bad : HAWKES_ERR_MARK_RANGE; continue; }
                if (use_hist) atomicAdd(&hist[ck[u]], 1);
                else atomicAdd((unsigned long long*)&p.counts[ck[u]], 1ull);
            }
        }
    }
    for (int64_t b = b0; b < b1 && p.B != 1; ++b) {
        int32_t seq = p.chunk_seq[b];
        int64_t s0, s1;
        chunk_range(p, b, seq, s0, s1);
        const double T = p.Tarr[seq];
        const int64_t first = p.off[seq];
        // Times compare as integers: for non-negative doubles (and -0 read as +0) the order of
        // the bit patterns is the numeric order, and a NaN or a negative value falls outside
        // [0, T] (FP64 compares run at 1/64 of the FP32 rate on this part).  T itself is
        // checked on the host to be finite and non-negative.
        const uint64_t Tkey = time_key(T);
        for (int64_t k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
            const uint64_t key = time_key(p.t[k]);
            int32_t ck = p.c[k];
            if (key > Tkey) bad = bad ? bad : HAWKES_ERR_TIME_RANGE;
            if (k > first && key < time_key(p.t[k - 1])) bad = bad ? bad : HAWKES_ERR_UNSORTED;
            if (ck < 0 || ck >= p.M) { bad = bad ? bad : HAWKES_ERR_MARK_RANGE; continue; }
            if (use_hist)
                atomicAdd(&hist[(seq - seq0) * p.M + ck], 1);
            else
                atomicAdd((unsigned long long*)&p.counts[(int64_t)seq * p.M + ck], 1ull);
        }
    }
    if (bad) set_status(p.hdr, bad);
    __syncthreads();
    if (use_hist)
        for (int i = threadIdx.x; i < span; i += blockDim.x)
            if (hist[i])
                atomicAdd((unsigned long long*)&p.counts[(int64_t)seq0 * p.M + i],
                          (unsigned long long)hist[i]);
    if (b0 == 0 && threadIdx.x == 0) p.hdr->validated = 1;
}

// Everything of the preparation that reads no event: accumulators, header, parameter checks,
// chunk table.
cudaError_t launch_prepare_head(const Problem& p, cudaStream_t s, int validate, int* nl) {
    // accumulators are one contiguous run of doubles starting at ll_acc
    int64_t n_acc = (int64_t)p.B * (1 + 4 * (int64_t)p.M) +
                    (p.grad ? (int64_t)p.B * p.M * p.M : 0);
    k_init<<<256, 256, 0, s>>>(p, p.ll_acc, n_acc);
    ++*nl;
    prof_mark(s, "init");
    if (validate) {
        cudaMemsetAsync(p.counts, 0, sizeof(int64_t) * (size_t)p.B * p.M, s);
        k_check_params<<<128, 256, 0, s>>>(p);
        ++*nl;
        prof_mark(s, "check_params");
    }
    k_chunk_table<<<1, 1024, 0, s>>>(p);
    prof_mark(s, "chunk_table");
    k_chunk_seq<<<p.B < 4096 ? p.B : 4096, 128, 0, s>>>(p);
    *nl += 2;
    prof_mark(s, "chunk_seq");
    return cudaGetLastError();
}

// The event checks and counts of chunks [b_begin, b_end).
cudaError_t launch_validate_chunks(const Problem& p, cudaStream_t s, int64_t b_begin,
                                   int64_t b_end, int* nl) {
    if (b_end > p.nb_max) b_end = p.nb_max;
    // one sequence: about 12,288 events per block (one mark-histogram flush per block), but
    // at least two blocks per SM
    int cpb = 16;
    if (p.B == 1) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int64_t per = (12288 + p.C - 1) / p.C;
        const int64_t spread = (b_end - b_begin) / (2 * (int64_t)sms);
        if (per > spread) per = spread;
        cpb = (int)(per < 1 ? 1 : (per > 64 ? 64 : per));
    }
    int64_t blocks = (b_end - b_begin + cpb - 1) / cpb;
    if (blocks < 1) blocks = 1;
    k_validate_events<<<(unsigned)blocks, 256, 0, s>>>(p, cpb, b_begin, b_end);
    ++*nl;
    prof_mark(s, "validate_events");
    return cudaGetLastError();
}

cudaError_t launch_prepare(const Problem& p, cudaStream_t s, int validate, int* nl) {
    cudaError_t err = launch_prepare_head(p, s, validate, nl);
    if (err == cudaSuccess && validate) err = launch_validate_chunks(p, s, 0, p.nb_max, nl);
    return err;
}

}  // namespace hk
