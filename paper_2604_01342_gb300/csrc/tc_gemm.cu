// Tensor-core GEMM for sm_103a:  D[m][n] (+)= sum_k A[m][k] B[n][k]
// with FP32-class accuracy from BF16 operands split in two:
//     A = Ah + Al,  B = Bh + Bl  (Ah = bf16(A), Al = bf16(A - Ah))
//     A B^T ~= Ah Bh^T + Ah Bl^T + Al Bh^T        (the Al Bl^T term is ~2^-18 relative)
// All three products accumulate into one FP32 accumulator in tensor memory.
//
// Used for the two dense contractions of the chunk-GEMM path: alpha . S^_b over
// all chunk-start states, and the dalpha contraction W^T S^ over all chunks.
//
// One CTA computes one 128 x 256 output tile over a slice of K (split-K with
// atomic accumulation when there is more than one slice).  Thread 0 issues the TMA
// loads (cp.async.bulk.tensor, 128-byte swizzle, 64 bf16 of K per row) into a
// two-stage ring and the tcgen05.mma instructions (kind::f16, bf16 in, f32
// accumulate, M=128, N=256, K=16); tcgen05.commit arrives on the stage's "empty"
// mbarrier when the MMAs that read it are done.  All four warps then read the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows) and
// store it.  Every mbarrier wait is bounded; on timeout the kernel records an
// error in the status word, waits (bounded) for its MMAs, frees its tensor memory
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "common.cuh"

namespace hk {

namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;                  // bf16 elements = 128 bytes = one swizzle row
constexpr int STAGES = 2;
constexpr int A_TILE = BM * BK * 2;     // 16 KB
constexpr int B_TILE = BN * BK * 2;     // 32 KB
constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;   // Ah, Al, Bh, Bl
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t kSpinLimit = 1u << 26;   // bounded waits (~ seconds)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: returns false if the phase did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(const void* tile) {
    uint64_t a = smem_u32(tile);
    uint64_t d = 0;
    d |= (a >> 4) & 0x3FFFull;          // start address
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: f32 accumulate, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct Maps {
    CUtensorMap ah, al, bh, bl;
};

__global__ void __launch_bounds__(128, 1)
k_gemm_bf16x3(const __grid_constant__ Maps maps, float* D, int64_t ldd, int Mdim, int Ndim,
              int k_tiles_total, int k_tiles_per_split, int atomic_out, WsHeader* hdr) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kt0 = blockIdx.z * k_tiles_per_split;
    int kt1 = kt0 + k_tiles_per_split;
    if (kt1 > k_tiles_total) kt1 = k_tiles_total;
    const int KT = kt1 > kt0 ? kt1 - kt0 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0 && KT > 0) {
        const uint32_t idesc = idesc_bf16(BM, BN);
        auto load_stage = [&](int s, int kt) {
            uint8_t* st = smem + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            const int kx = kt * BK;
            tma_load_2d(st, &maps.ah, &full[s], kx, m0);
            tma_load_2d(st + A_TILE, &maps.al, &full[s], kx, m0);
            tma_load_2d(st + 2 * A_TILE, &maps.bh, &full[s], kx, n0);
            tma_load_2d(st + 2 * A_TILE + B_TILE, &maps.bl, &full[s], kx, n0);
        };
        // per stage: index of the k-tile whose load is in flight and not yet consumed
        int inflight[STAGES];
        for (int s2 = 0; s2 < STAGES; ++s2) inflight[s2] = -1;
        for (int i = 0; i < STAGES && i < KT; ++i) { load_stage(i, kt0 + i); inflight[i] = i; }
        bool ok = true;
        for (int i = 0; i < KT && ok; ++i) {
            const int s = i % STAGES;
            if (!mbar_wait(&full[s], (uint32_t)((i / STAGES) & 1))) { ok = false; break; }
            inflight[s] = -1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint8_t* st = smem + s * STAGE_BYTES;
            const uint64_t dah = sw128_desc(st), dal = sw128_desc(st + A_TILE);
            const uint64_t dbh = sw128_desc(st + 2 * A_TILE);
            const uint64_t dbl = sw128_desc(st + 2 * A_TILE + B_TILE);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t off = (uint64_t)(kk * 32) >> 4;   // 16 bf16 = 32 bytes
                const uint32_t acc0 = (i > 0 || kk > 0) ? 1u : 0u;
                mma_bf16(tmem, dah + off, dbh + off, idesc, acc0);
                mma_bf16(tmem, dah + off, dbl + off, idesc, 1u);
                mma_bf16(tmem, dal + off, dbh + off, idesc, 1u);
            }
            mma_commit(&empty[s]);
            // refill the stage the previous k-tile used once its MMAs are done
            if (i >= 1) {
                const int ps = (i - 1) % STAGES;
                const int nxt = i - 1 + STAGES;
                if (nxt < KT) {
                    if (!mbar_wait(&empty[ps], (uint32_t)(((i - 1) / STAGES) & 1))) {
                        ok = false;
                        break;
                    }
                    load_stage(ps, kt0 + nxt);
                    inflight[ps] = nxt;
                }
            }
        }
        mma_commit(done);
        if (!ok) {
            // let the copies still in flight land before the block's smem is released
            for (int s2 = 0; s2 < STAGES; ++s2)
                if (inflight[s2] >= 0) mbar_wait(&full[s2], (uint32_t)((inflight[s2] / STAGES) & 1));
            *abort_flag = 1;
            if (hdr) set_status(hdr, HAWKES_ERR_CUDA);
        }
    }
    __syncthreads();
    bool have = KT > 0 && !*abort_flag;
    if (KT > 0) {
        // all issued MMAs complete before the accumulator is read or freed
        if (!mbar_wait(done, 0)) {
            have = false;
            if (lane == 0 && hdr) set_status(hdr, HAWKES_ERR_CUDA);
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (have) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            tmem_ld32(tbase + (uint32_t)c0, v);
            if (row < Mdim) {
                float* drow = D + (int64_t)row * ldd + n0 + c0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (n0 + c0 + j < Ndim) {
                        if (atomic_out) atomicAdd(drow + j, v[j]);
                        else drow[j] = v[j];
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D bf16 tensor [rows][k] with row stride ld (elements), box {64, box_rows}.
static bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t k, int64_t ld,
                     int box_rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace tc

// D[m][n] (+)= sum_k A[m][k] B[n][k] over m < Mdim, n < Ndim, k < Kdim; A and B given as
// bf16 hi/lo pairs with row strides lda, ldb (elements, multiples of 8; bases 16-byte aligned).
cudaError_t tc_gemm_bf16x3(const __nv_bfloat16* Ah, const __nv_bfloat16* Al, int64_t lda,
                           const __nv_bfloat16* Bh, const __nv_bfloat16* Bl, int64_t ldb,
                           float* D, int64_t ldd, int Mdim, int Ndim, int64_t Kdim, int splits,
                           bool accumulate, WsHeader* hdr, cudaStream_t s) {
    using namespace tc;
    if (Mdim <= 0 || Ndim <= 0 || Kdim <= 0) return cudaSuccess;
    if ((lda % 8) || (ldb % 8)) return cudaErrorInvalidValue;
    Maps maps;
    if (!make_map(&maps.ah, Ah, Mdim, Kdim, lda, BM) || !make_map(&maps.al, Al, Mdim, Kdim, lda, BM) ||
        !make_map(&maps.bh, Bh, Ndim, Kdim, ldb, BN) || !make_map(&maps.bl, Bl, Ndim, Kdim, ldb, BN))
        return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16x3,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int kt_total = (int)((Kdim + BK - 1) / BK);
    if (splits < 1) splits = 1;
    if (splits > kt_total) splits = kt_total;
    const int per = (kt_total + splits - 1) / splits;
    splits = (kt_total + per - 1) / per;
    dim3 grid((unsigned)((Ndim + BN - 1) / BN), (unsigned)((Mdim + BM - 1) / BM), (unsigned)splits);
    const int atomic_out = (splits > 1 || accumulate) ? 1 : 0;
    k_gemm_bf16x3<<<grid, 128, SMEM_BYTES, s>>>(maps, D, ldd, Mdim, Ndim, kt_total, per,
                                                 atomic_out, hdr);
    return cudaGetLastError();
}

// Split an FP32 matrix [rows][cols] (row stride lds) into bf16 hi/lo [rows][ldd].
__global__ void k_split_bf16(const float* __restrict__ src, int64_t lds, __nv_bfloat16* hi,
                             __nv_bfloat16* lo, int64_t ldd, int64_t rows, int64_t cols) {
    const int64_t n = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, c = i % cols;
        const float x = src[r * lds + c];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[r * ldd + c] = h;
        lo[r * ldd + c] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

cudaError_t split_bf16(const float* src, int64_t lds, __nv_bfloat16* hi, __nv_bfloat16* lo,
                       int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    int64_t n = rows * cols;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_split_bf16<<<(unsigned)blocks, 256, 0, s>>>(src, lds, hi, lo, ldd, rows, cols);
    return cudaGetLastError();
}

}  // namespace hk

// Test hook (declared in no public header): the same GEMM on caller buffers, so a GPU
// test can compare it with a reference product.  D[m][n] = sum_k A[m][k] B[n][k] from
// FP32 A [M][K] and B [N][K]; scratch must hold 2*(M+N)*K bf16 (row stride K rounded up
// to 8).  Returns 0 on success.
extern "C" int hawkes_test_tc_gemm(const float* A, const float* B, float* D, int M, int N,
                                   int K, int splits, void* scratch, void* stream) {
    using namespace hk;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ld = (K + 7) / 8 * 8;
    __nv_bfloat16* p = (__nv_bfloat16*)scratch;
    __nv_bfloat16 *Ah = p, *Al = Ah + (int64_t)M * ld, *Bh = Al + (int64_t)M * ld,
                  *Bl = Bh + (int64_t)N * ld;
    if (split_bf16(A, K, Ah, Al, ld, M, K, s) != cudaSuccess) return 1;
    if (split_bf16(B, K, Bh, Bl, ld, N, K, s) != cudaSuccess) return 1;
    if (splits > 1) cudaMemsetAsync(D, 0, sizeof(float) * (size_t)M * N, s);
    return tc_gemm_bf16x3(Ah, Al, ld, Bh, Bl, ld, D, N, M, N, K, splits, false, nullptr, s) ==
                   cudaSuccess
               ? 0
               : 2;
}
