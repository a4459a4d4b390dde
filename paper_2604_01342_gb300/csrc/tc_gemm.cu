// Tensor-core GEMM for sm_103a:  D[m][n] (+)= sum_k A[m][k] B[n][k]
// with FP32-class accuracy from FP16 operands split in two.  Every row of A and of B is
// first scaled by a power of two 2^a_m (2^b_n) that brings its largest magnitude into
// [2^13, 2^14), then split:
//     A[m][k] 2^a_m = Ah + Al,  Ah = fp16(.), Al = fp16(. - Ah)   (both rounded to nearest)
//     A B^T ~= 2^-(a_m + b_n) (Ah Bh^T + Ah Bl^T + Al Bh^T)   (the Al Bl^T term is ~2^-22)
// FP16 carries the same 11 significant bits as TF32 and runs at twice its tensor rate;
// the row scaling keeps every split part of an entry larger than 2^-17 of its row's
// maximum in the normal FP16 range, and the scaling and its inverse are exact.  All three
// products accumulate into FP32 accumulators in tensor memory.
//
// Operand layout ("paired" rows): for every group of 32 consecutive k the 32 high parts are
// followed by the 32 low parts, so element k of a row has its high part at
// 64 (k / 32) + k % 32 and its low part 32 halves later; a row of K elements takes
// 64 ceil(K / 32) halves, the positions past K holding zeros.  One 128-byte TMA row
// (128-byte swizzle) then carries both parts of a k-tile of 32.
//
// Used for the two dense contractions of the chunk-GEMM path: alpha . S^_b over
// all chunk-start states, and the dalpha contraction W^T S^ over all chunks.
//
// One CTA computes one 128 x 256 output tile over a slice of K (split-K with
// atomic accumulation when there is more than one slice).  One thread issues the TMA
// loads (cp.async.bulk.tensor, 128-byte swizzle, one paired k-tile per row) into a
// four-stage ring; a thread of another warp issues the tcgen05.mma instructions
// (kind::f16, f32 accumulate, M=128, N=256, K=16); tcgen05.commit arrives on the stage's
// "empty" mbarrier when the MMAs that read it are done, and the loading thread refills it.
// The tensor-core accumulator loses precision with the number of accumulation steps
// (measured with TF32 operands: ~1.6e-6 after 64 of K, ~2.6e-5 after 1024), so every 64 of
// K (two k-tiles) is accumulated into one of two TMEM banks and then promoted: eight warps
// read the finished bank with tcgen05.ld and add it to FP32 registers while the MMAs fill
// the other bank.  The output tile is staged in the (then free) stage buffers and stored as
// whole row pieces.  Every mbarrier wait is bounded; on timeout the kernel records an error
// in the status word, waits (bounded) for its MMAs and copies, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "common.cuh"

namespace hk {

namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 32;                  // k per tile: 32 high + 32 low fp16 = 128 bytes per row
constexpr int ROW_BYTES = 4 * BK;
constexpr int STAGES = 4;
constexpr int A_TILE = BM * ROW_BYTES;  // 16 KB
constexpr int B_TILE = BN * ROW_BYTES;  // 32 KB
constexpr int kTilesPerGroup = 2;       // k-tiles accumulated in TMEM before promotion (64 of K)
// unused bytes between the stages and the barriers, so that no operand descriptor of the
// last stage can reach the barriers or the end of the allocation
constexpr int kSlack = 24 * 1024;
constexpr int STAGE_BYTES = A_TILE + B_TILE;
// then the barriers (256 B) and the tile's column factors (inverse scale, bias: 2 x BN floats)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + kSlack + 1024 /*align*/ + 256 + 2 * BN * 4;
// row stride (floats) of the output tile staged in the stage buffers: 16 bytes of padding
// per row, so that the rows' float4 writes (one row per lane) fall in distinct banks
constexpr int kOutLd = BN + 4;
static_assert(BM * kOutLd * 4 <= STAGES * STAGE_BYTES, "the output tile fits the stages");
constexpr uint32_t TMEM_COLS = 512;      // two accumulator banks of BN columns
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

// Bounded wait that also gives up as soon as *abort is set.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity,
                                                   volatile int* abort) {
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
    }
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

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
// (tiles 1024-byte aligned, so the base offset is 0).
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

// Instruction descriptor, kind::f16: f32 accumulate, fp16 A and B (format 0), both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
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
    CUtensorMap a, b;
};

// Threads: warps 0-7 read and promote the accumulator (warp w owns TMEM lanes
// 32 (w % 4) .. +31 = rows, and columns (w / 4) * 128 .. +127); warp 8 allocates the
// tensor memory and one of its threads issues the MMAs; one thread of warp 9 issues the
// TMA loads, refilling each stage as soon as the MMAs that read it are done, so that the
// MMA thread never waits for a refill and can queue MMAs up to the ring's depth ahead.
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = kEpiWarps, kTmaWarp = kEpiWarps + 1;
constexpr int kThreads = (kEpiWarps + 2) * 32;

__global__ void __launch_bounds__(kThreads, 1)
k_gemm_f16x3(const __grid_constant__ Maps maps, float* D, int64_t ldd, int Mdim, int Ndim,
             int k_tiles_total, int k_tiles_per_split, int atomic_out, const float* bias,
             const float* __restrict__ inv_sa, const float* __restrict__ inv_sb, WsHeader* hdr) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES + kSlack);
    uint64_t* empty = full + STAGES;
    uint64_t* bank_full = empty + STAGES;     // [2] accumulator bank holds a finished group
    uint64_t* bank_empty = bank_full + 2;     // [2] bank has been read by all epilogue warps
    uint64_t* done = bank_empty + 2;          // every MMA of this block has completed
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    float* col_scale = (float*)(smem + STAGES * STAGE_BYTES + kSlack + 256);   // [BN]
    float* col_bias = col_scale + BN;                                         // [BN]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kt0 = blockIdx.z * k_tiles_per_split;
    int kt1 = kt0 + k_tiles_per_split;
    if (kt1 > k_tiles_total) kt1 = k_tiles_total;
    const int KT = kt1 > kt0 ? kt1 - kt0 : 0;
    const int ngroups = (KT + kTilesPerGroup - 1) / kTilesPerGroup;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&bank_full[q], 1);
            mbar_init(&bank_empty[q], kEpiWarps);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < BN) {
        const int col = n0 + threadIdx.x;
        col_scale[threadIdx.x] = col < Ndim ? __ldg(inv_sb + col) : 0.f;
        col_bias[threadIdx.x] = (bias && blockIdx.z == 0 && col < Ndim) ? __ldg(bias + col) : 0.f;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == kMmaWarp) {
        if (lane == 0 && KT > 0) {
            const uint32_t idesc = idesc_f16(BM, BN);
            bool ok = true;
            for (int i = 0; i < KT; ++i) {
                const int s = i % STAGES;
                if (!mbar_wait_or_abort(&full[s], (uint32_t)((i / STAGES) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint8_t* st = smem + s * STAGE_BYTES;
                const uint64_t da = sw128_desc(st), db = sw128_desc(st + A_TILE);
                const int g = i / kTilesPerGroup, bank = g & 1;
                const bool first_in_group = (i % kTilesPerGroup) == 0;
                if (first_in_group && g >= 2) {
                    // the epilogue must have read this bank's previous group
                    if (!mbar_wait(&bank_empty[bank], (uint32_t)(((g >> 1) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                const uint32_t acc_t = tmem + (uint32_t)(bank * BN);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    // 16 fp16 = 32 bytes along the 128-byte swizzled row: the high parts
                    // at bytes 0-63, the low parts at 64-127
                    const uint64_t oh = (uint64_t)(kk * 32) >> 4;
                    const uint64_t ol = (uint64_t)(64 + kk * 32) >> 4;
                    const uint32_t acc0 = (!first_in_group || kk > 0) ? 1u : 0u;
                    mma_f16(acc_t, da + oh, db + oh, idesc, acc0);
                    mma_f16(acc_t, da + oh, db + ol, idesc, 1u);
                    mma_f16(acc_t, da + ol, db + oh, idesc, 1u);
                }
                if ((i % kTilesPerGroup) == kTilesPerGroup - 1 || i == KT - 1) mma_commit(&bank_full[bank]);
                mma_commit(&empty[s]);           // the stage may be refilled once these are done
            }
            if (!ok) {
                *abort_flag = 1;
                if (hdr) set_status(hdr, HAWKES_ERR_CUDA);
                // release the epilogue warps waiting on the banks
                mma_commit(&bank_full[0]);
                mma_commit(&bank_full[1]);
            }
            // no MMA may still be writing tensor memory when it is freed
            mma_commit(done);
            mbar_wait(done, 0);
        }
    } else if (warp == kTmaWarp) {
        if (lane == 0 && KT > 0) {
            int last[STAGES];                    // the last k-tile loaded into each stage
            for (int s2 = 0; s2 < STAGES; ++s2) last[s2] = -1;
            for (int i = 0; i < KT; ++i) {
                const int s = i % STAGES;
                if (i >= STAGES &&
                    !mbar_wait_or_abort(&empty[s], (uint32_t)(((i / STAGES) - 1) & 1), abort_flag)) {
                    if (!*abort_flag) {
                        *abort_flag = 1;
                        if (hdr) set_status(hdr, HAWKES_ERR_CUDA);
                    }
                    break;
                }
                if (*abort_flag) break;
                uint8_t* st = smem + s * STAGE_BYTES;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                const int kx = (kt0 + i) * 2 * BK;   // halves: 128-byte aligned
                tma_load_2d(st, &maps.a, &full[s], kx, m0);
                tma_load_2d(st + A_TILE, &maps.b, &full[s], kx, n0);
                last[s] = i;
            }
            // no copy may still be writing shared memory when the block exits
            for (int s2 = 0; s2 < STAGES; ++s2)
                if (last[s2] >= 0) mbar_wait(&full[s2], (uint32_t)((last[s2] / STAGES) & 1));
        }
    } else if (KT > 0) {
        // epilogue warps: promote each group's partial sum into FP32 registers
        const int lane_base = 32 * (warp & 3);
        const int col_base = 128 * (warp >> 2);
        float run[128];
#pragma unroll
        for (int j = 0; j < 128; ++j) run[j] = 0.f;
        bool good = true;
        for (int g = 0; g < ngroups && good; ++g) {
            const int bank = g & 1;
            if (!mbar_wait(&bank_full[bank], (uint32_t)((g >> 1) & 1))) { good = false; break; }
            if (*abort_flag) { good = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t tb = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(bank * BN + col_base);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float v[32];
                tmem_ld32(tb + (uint32_t)(32 * c), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) run[32 * c + j] += v[j];
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                            smem_u32(&bank_empty[bank]))
                                        : "memory");
        }
        if (!good && lane == 0 && hdr) set_status(hdr, HAWKES_ERR_CUDA);
        // Output: undo the row scalings (exact powers of two) and add the bias into a row-major
        // copy of the tile in the stage buffers (free now: the last group's commit means every
        // load was consumed and every MMA has completed), then store whole row pieces: with
        // one row per thread, direct stores would be 32 separate 16-byte pieces per warp
        // instruction.
        const int rloc = lane_base + lane;
        const int row = m0 + rloc;
        const float fa = row < Mdim ? __ldg(inv_sa + row) : 0.f;
        float* otile = (float*)smem;                       // [BM][kOutLd]
        if (good) {
            float* orow = otile + rloc * kOutLd + col_base;
#pragma unroll
            for (int j = 0; j < 128; j += 4) {
                float4 o;
                o.x = run[j] * (fa * col_scale[col_base + j]) + col_bias[col_base + j];
                o.y = run[j + 1] * (fa * col_scale[col_base + j + 1]) + col_bias[col_base + j + 1];
                o.z = run[j + 2] * (fa * col_scale[col_base + j + 2]) + col_bias[col_base + j + 2];
                o.w = run[j + 3] * (fa * col_scale[col_base + j + 3]) + col_bias[col_base + j + 3];
                *(float4*)(orow + j) = o;
            }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory");   // epilogue warps only
        if (good) {
            const bool vec = (ldd & 3) == 0 && ((uintptr_t)D & 15) == 0;
            // warp w stores rows w, w + 8, ...: 256 columns as two 512-byte pieces per row
            for (int rr = warp; rr < BM && m0 + rr < Mdim; rr += kEpiWarps) {
                float* drow = D + (int64_t)(m0 + rr) * ldd + n0;
                const float* srow = otile + rr * kOutLd;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = 128 * h + 4 * lane;
                    const float4 v = *(const float4*)(srow + c);
                    if (vec && n0 + c + 4 <= Ndim) {
                        if (atomic_out) atomicAdd((float4*)(drow + c), v);
                        else *(float4*)(drow + c) = v;
                    } else {
                        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (n0 + c + q < Ndim) {
                                if (atomic_out) atomicAdd(drow + c + q, vv[q]);
                                else drow[c + q] = vv[q];
                            }
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp)
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

// 2-D fp16 tensor of paired rows [rows][2 * BK * k_tiles] with row stride ld (halves),
// box {2 * BK, box_rows} (128 bytes per box row).
static bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t k_tiles,
                     int64_t ld, int box_rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * BK * k_tiles), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)(2 * BK), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Power-of-two exponent a with max * 2^a in [2^13, 2^14) (0 for a zero or non-finite max).
__device__ __forceinline__ int row_exponent(float amax) {
    if (!(amax > 0.f) || !isfinite(amax)) return 0;
    int e;
    frexpf(amax, &e);                    // amax = f 2^e, f in [0.5, 1)
    return max(-100, min(100, 14 - e));
}

__device__ __forceinline__ void split_f16(float x, __half& hi, __half& lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// Position of the high part of element c in a paired row (the low part is 32 further on).
__host__ __device__ __forceinline__ int64_t pidx(int64_t c) { return c + (c & ~(int64_t)31); }
__host__ __device__ __forceinline__ int64_t round32(int64_t c) { return (c + 31) & ~(int64_t)31; }

// Split of four consecutive values: their high parts (h01, h23) and low parts (l01, l23)
// as pairs of halves.
struct Split4 {
    uint32_t h01, h23, l01, l23;
};
__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
    const __half2 v = __halves2half2(a, b);
    return *(const uint32_t*)&v;
}
__device__ __forceinline__ Split4 split4(float4 x) {
    __half h0, l0, h1, l1, h2, l2, h3, l3;
    split_f16(x.x, h0, l0);
    split_f16(x.y, h1, l1);
    split_f16(x.z, h2, l2);
    split_f16(x.w, h3, l3);
    return Split4{pack2(h0, h1), pack2(h2, h3), pack2(l0, l1), pack2(l2, l3)};
}

// A warp whose lane L holds the split of elements c0 + 4 L + {0, 1, 2, 3} of a paired row
// (c0 a multiple of 64) stores elements [c0, c0 + 128) as two contiguous 256-byte stores:
// in store s, lane L writes 8 bytes at byte 8 L of the run, the high (L % 16 < 8) or low
// parts of elements c0 + 64 s + 32 (L / 16) + 4 (L % 8) + {0..3}, received by shuffles from
// the lane that split them.  Elements at or past cpad (a multiple of 32) are not stored.
// Every lane of the warp must call it.
__device__ __forceinline__ void p128_store(__half* row, int64_t c0, int64_t cpad, int lane,
                                           const Split4& v) {
    const bool low = ((lane >> 3) & 1) != 0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int src = 16 * s + 8 * (lane >> 4) + (lane & 7);
        const uint32_t a = __shfl_sync(0xffffffffu, v.h01, src);
        const uint32_t b = __shfl_sync(0xffffffffu, v.h23, src);
        const uint32_t c = __shfl_sync(0xffffffffu, v.l01, src);
        const uint32_t d = __shfl_sync(0xffffffffu, v.l23, src);
        const int64_t e = c0 + 64 * s + 32 * (lane >> 4) + 4 * (lane & 7);
        if (e < cpad) *(uint2*)(row + pidx(e) + (low ? 32 : 0)) = low ? make_uint2(c, d) : make_uint2(a, b);
    }
}

// four consecutive values p[c .. c + 3] (0 at or past n); vec: p is 16-byte aligned and
// c a multiple of 4
__device__ __forceinline__ float4 load4(const float* __restrict__ p, int64_t c, int64_t n, bool vec) {
    if (vec && c + 4 <= n) return __ldg((const float4*)(p + c));
    return make_float4(c < n ? p[c] : 0.f, c + 1 < n ? p[c + 1] : 0.f, c + 2 < n ? p[c + 2] : 0.f,
                       c + 3 < n ? p[c + 3] : 0.f);
}

__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace tc

// D[m][n] (+)= inv_sa[m] inv_sb[n] sum_k A[m][k] B[n][k] over m < Mdim, n < Ndim, k < Kdim;
// A and B given as paired fp16 hi/lo rows of the scaled matrices (row strides lda, ldb in
// halves, multiples of 8 and at least 64 ceil(Kdim / 32); bases 16-byte aligned; zeros
// past Kdim), inv_sa / inv_sb the inverse scales.
cudaError_t tc_gemm_f16x3(const __half* A, int64_t lda, const __half* B, int64_t ldb, float* D,
                          int64_t ldd, int Mdim, int Ndim, int64_t Kdim, int splits,
                          bool accumulate, WsHeader* hdr, cudaStream_t s, const float* bias,
                          const float* inv_sa, const float* inv_sb) {
    using namespace tc;
    if (Mdim <= 0 || Ndim <= 0 || Kdim <= 0) return cudaSuccess;
    const int64_t kt_total64 = (Kdim + BK - 1) / BK;
    if ((lda % 8) || (ldb % 8) || lda < 2 * BK * kt_total64 || ldb < 2 * BK * kt_total64)
        return cudaErrorInvalidValue;
    Maps maps;
    if (!make_map(&maps.a, A, Mdim, kt_total64, lda, BM) ||
        !make_map(&maps.b, B, Ndim, kt_total64, ldb, BN))
        return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_f16x3,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int kt_total = (int)kt_total64;
    if (splits < 1) splits = 1;
    if (splits > kt_total) splits = kt_total;
    const int per = (kt_total + splits - 1) / splits;
    splits = (kt_total + per - 1) / per;
    dim3 grid((unsigned)((Ndim + BN - 1) / BN), (unsigned)((Mdim + BM - 1) / BM), (unsigned)splits);
    const int atomic_out = (splits > 1 || accumulate) ? 1 : 0;
    k_gemm_f16x3<<<grid, kThreads, SMEM_BYTES, s>>>(maps, D, ldd, Mdim, Ndim, kt_total, per,
                                                atomic_out, bias, inv_sa, inv_sb, hdr);
    return cudaGetLastError();
}

// One warp per row r < rows of an FP32 matrix [rows][cols] (row stride lds), minus an
// optional per-column centre and minus an optional (*coef) * sub[r][c] (same layout as
// src; coef on the device): the row's scale exponent from its largest magnitude, the
// paired fp16 hi/lo rows of the scaled row in dst [rows][ldd], and inv_scale[r] = 2^-a.
// Rows at or past *rows_valid (when given) are written as zeros.
__global__ void k_split_f16_rows(const float* __restrict__ src, int64_t lds, __half* dst,
                                 int64_t ldd, int64_t rows, int64_t cols,
                                 const float* __restrict__ centre, const int64_t* rows_valid,
                                 float* inv_scale, const float* __restrict__ sub,
                                 const float* __restrict__ coef) {
    const int lane = threadIdx.x & 31;
    const int64_t nvalid = rows_valid ? *rows_valid : rows;
    const float cf = sub ? *coef : 0.f;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t cpad = tc::round32(cols);
    for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
        const float* sr = src + r * lds;
        const float* ur = sub ? sub + r * lds : nullptr;
        auto val = [&](int64_t c) {
            float v = sr[c] - (centre ? centre[c] : 0.f);
            return ur ? v - cf * ur[c] : v;
        };
        __half* dr = dst + r * ldd;
        const bool valid = r < nvalid;
        float amax = 0.f;
        if (valid)
            for (int64_t c = lane; c < cols; c += 32) amax = fmaxf(amax, fabsf(val(c)));
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        const int a = tc::row_exponent(amax);
        const float sc = ldexpf(1.f, a);
        // 128 elements per two warp stores (zeros past cols, and for the rows past the valid ones)
        for (int64_t c0 = 0; c0 < cpad; c0 += 128) {
            const int64_t c = c0 + 4 * lane;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid) {
                x.x = c < cols ? val(c) * sc : 0.f;
                x.y = c + 1 < cols ? val(c + 1) * sc : 0.f;
                x.z = c + 2 < cols ? val(c + 2) * sc : 0.f;
                x.w = c + 3 < cols ? val(c + 3) * sc : 0.f;
            }
            tc::p128_store(dr, c0, cpad, lane, tc::split4(x));
        }
        if (lane == 0) inv_scale[r] = valid ? ldexpf(1.f, -a) : 1.f;
    }
}

// Two row-scaled splits of one matrix in one pass over it (one warp per row): out1 = src -
// centre (per column) and out2 = src - (*coef) sub - centre2 (per column), each with its own
// row exponent and inverse scale, as paired rows; rows at or past *rows_valid are written as
// zeros.
__global__ void k_split_f16_rows_pair(const float* __restrict__ src, const float* __restrict__ sub,
                                      int64_t lds, const float* __restrict__ centre,
                                      const float* __restrict__ centre2,
                                      const float* __restrict__ coef, __half* out1, float* isc1,
                                      __half* out2, float* isc2, int64_t ldd, int64_t rows,
                                      int64_t cols, const int64_t* rows_valid, uint32_t* colmax) {
    extern __shared__ uint32_t cmax_sh[];     // [cols] this block's column maxima of |out1|
    const int lane = threadIdx.x & 31;
    const int64_t nvalid = rows_valid ? *rows_valid : rows;
    const float cf = *coef;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t cpad = tc::round32(cols);
    const bool vec = (lds & 3) == 0 && tc::aligned16(src) && tc::aligned16(sub) &&
                     tc::aligned16(centre) && tc::aligned16(centre2);
    if (colmax) {
        for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) cmax_sh[c] = 0u;
        __syncthreads();
    }
    for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
        const float* sr = src + r * lds;
        const float* ur = sub + r * lds;
        __half *d1 = out1 + r * ldd, *d2 = out2 + r * ldd;
        if (r >= nvalid) {
            const tc::Split4 z = tc::split4(make_float4(0.f, 0.f, 0.f, 0.f));
            for (int64_t c0 = 0; c0 < cpad; c0 += 128) {
                tc::p128_store(d1, c0, cpad, lane, z);
                tc::p128_store(d2, c0, cpad, lane, z);
            }
            if (lane == 0) { isc1[r] = 1.f; isc2[r] = 1.f; }
            continue;
        }
        float m1 = 0.f, m2 = 0.f;
        for (int64_t c = lane; c < cols; c += 32) {
            const float v = sr[c];
            const float a1 = fabsf(v - centre[c]);
            m1 = fmaxf(m1, a1);
            m2 = fmaxf(m2, fabsf((v - cf * ur[c]) - centre2[c]));
            if (colmax && a1 > 0.f) atomicMax(&cmax_sh[c], __float_as_uint(a1));
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        }
        const int a1 = tc::row_exponent(m1), a2 = tc::row_exponent(m2);
        const float sc1 = ldexpf(1.f, a1), sc2 = ldexpf(1.f, a2);
        // 128 elements per two warp stores per output (zeros past cols)
        for (int64_t c0 = 0; c0 < cpad; c0 += 128) {
            const int64_t c = c0 + 4 * lane;
            const float4 v = tc::load4(sr, c, cols, vec);
            const float4 m = tc::load4(centre, c, cols, vec);
            const float4 u = tc::load4(ur, c, cols, vec);
            const float4 m2c = tc::load4(centre2, c, cols, vec);
            tc::p128_store(d1, c0, cpad, lane,
                           tc::split4(make_float4((v.x - m.x) * sc1, (v.y - m.y) * sc1,
                                                  (v.z - m.z) * sc1, (v.w - m.w) * sc1)));
            tc::p128_store(d2, c0, cpad, lane,
                           tc::split4(make_float4(((v.x - cf * u.x) - m2c.x) * sc2,
                                                  ((v.y - cf * u.y) - m2c.y) * sc2,
                                                  ((v.z - cf * u.z) - m2c.z) * sc2,
                                                  ((v.w - cf * u.w) - m2c.w) * sc2)));
        }
        if (lane == 0) {
            isc1[r] = ldexpf(1.f, -a1);
            isc2[r] = ldexpf(1.f, -a2);
        }
    }
    if (colmax) {
        __syncthreads();
        for (int64_t c = threadIdx.x; c < cols; c += blockDim.x)
            if (cmax_sh[c]) atomicMax(colmax + c, cmax_sh[c]);
    }
}

// colmax (optional, [cols] uint bits, zeroed here): the largest |out1| of every column over
// the valid rows, for a later transposed split of the same matrix.
cudaError_t split_f16_rows_pair(const float* src, const float* sub, int64_t lds,
                                const float* centre, const float* centre2, const float* coef,
                                __half* out1, float* isc1, __half* out2, float* isc2,
                                int64_t ldd, int64_t rows, int64_t cols,
                                const int64_t* rows_valid, uint32_t* colmax, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (!src || !sub || !centre || !centre2 || !coef || (ldd & 1) ||
        ldd < 2 * tc::round32(cols))
        return cudaErrorInvalidValue;
    const size_t smem = colmax ? sizeof(uint32_t) * (size_t)cols : 0;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    if (colmax) {
        cudaError_t e = cudaMemsetAsync(colmax, 0, sizeof(uint32_t) * (size_t)cols, s);
        if (e != cudaSuccess) return e;
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(k_split_f16_rows_pair,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
    }
    int64_t blocks = (rows + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_split_f16_rows_pair<<<(unsigned)blocks, 256, smem, s>>>(src, sub, lds, centre, centre2,
                                                              coef, out1,
                                                              isc1, out2, isc2, ldd, rows, cols,
                                                              rows_valid, colmax);
    return cudaGetLastError();
}

// Long rows (cols >> 32): one block per row at a time, two passes over it (the row maximum
// and, if asked, the FP64 row sum; then the split into a paired row), no centre or
// subtrahend.  Two blocks per SM, so that the rows being split (2 x 152 at a time) stay in
// L2 between the passes while they are at most a few hundred KB long.
constexpr int kLongRowThreads = 512;
__global__ void __launch_bounds__(kLongRowThreads) k_split_f16_long_rows(
    const float* __restrict__ src, int64_t lds, __half* dst, int64_t ldd, int64_t rows,
    int64_t cols, float* inv_scale, double* row_sum, const uint32_t* __restrict__ row_max) {
    __shared__ float red[kLongRowThreads / 32];
    __shared__ double reds[kLongRowThreads / 32];
    const int64_t cpad = tc::round32(cols);
    const bool vec = (lds & 3) == 0 && tc::aligned16(src);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const float* sr = src + r * lds;
        float amax = 0.f;
        if (row_max) {
            // the row's largest magnitude is given (non-negative rows): one pass
            amax = __uint_as_float(row_max[r]);
        } else {
        float part = 0.f;                     // FP32 partial sums per thread, FP64 across
        const int64_t c4end = vec ? (cols & ~(int64_t)3) : 0;
#pragma unroll 4
        for (int64_t c = 4 * (int64_t)threadIdx.x; c < c4end; c += 4 * (int64_t)blockDim.x) {
            const float4 v = __ldg((const float4*)(sr + c));
            amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            part += (v.x + v.y) + (v.z + v.w);
        }
        for (int64_t c = c4end + threadIdx.x; c < cols; c += blockDim.x) {
            const float v = sr[c];
            amax = fmaxf(amax, fabsf(v));
            part += v;
        }
        double sum = (double)part;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
        }
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = amax; reds[threadIdx.x >> 5] = sum; }
        __syncthreads();
        amax = 0.f;
        sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { amax = fmaxf(amax, red[w]); sum += reds[w]; }
        __syncthreads();                                  // red is reused by the next row
        if (row_sum && threadIdx.x == 0) row_sum[r] = sum;
        }
        const int a = tc::row_exponent(amax);
        const float sc = ldexpf(1.f, a);
        __half* dr = dst + r * ldd;
        // 128 elements per two warp stores (zeros past cols)
#pragma unroll 4
        for (int64_t c0 = 128 * (int64_t)warp; c0 < cpad; c0 += 128 * (int64_t)nwarps) {
            const float4 v = tc::load4(sr, c0 + 4 * lane, cols, vec);
            tc::p128_store(dr, c0, cpad, lane,
                           tc::split4(make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc)));
        }
        if (threadIdx.x == 0) inv_scale[r] = ldexpf(1.f, -a);
    }
}

// row_max (optional): the largest magnitude of every row as float bits, taken by the caller;
// the rows are then read once (row_sum is not formed).
cudaError_t split_f16_long_rows(const float* src, int64_t lds, __half* dst, int64_t ldd,
                                int64_t rows, int64_t cols, cudaStream_t s, float* inv_scale,
                                double* row_sum, const uint32_t* row_max) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if ((ldd & 1) || ldd < 2 * tc::round32(cols)) return cudaErrorInvalidValue;
    const int64_t blocks = rows < 152 * 2 ? rows : 152 * 2;
    k_split_f16_long_rows<<<(unsigned)blocks, kLongRowThreads, 0, s>>>(src, lds, dst, ldd, rows,
                                                                       cols, inv_scale, row_sum,
                                                                       row_max);
    return cudaGetLastError();
}

cudaError_t split_f16_rows(const float* src, int64_t lds, __half* dst, int64_t ldd,
                           int64_t rows, int64_t cols, cudaStream_t s, const float* centre,
                           const int64_t* rows_valid, float* inv_scale, const float* sub,
                           const float* coef) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if ((sub == nullptr) != (coef == nullptr) || (ldd & 1) || ldd < 2 * tc::round32(cols))
        return cudaErrorInvalidValue;
    if (cols >= 4096 && !centre && !rows_valid && !sub)
        return split_f16_long_rows(src, lds, dst, ldd, rows, cols, s, inv_scale, nullptr, nullptr);
    int64_t blocks = (rows + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_split_f16_rows<<<(unsigned)blocks, 256, 0, s>>>(src, lds, dst, ldd, rows, cols, centre,
                                                      rows_valid, inv_scale, sub, coef);
    return cudaGetLastError();
}

// Largest |src[r][c] - centre[c]| over the valid rows of every column c, as the bits of a
// non-negative float (so that an unsigned maximum orders them); amax_bits starts at 0.
__global__ void k_colmax(const float* __restrict__ src, int64_t cols, const int64_t* rows_valid,
                         const float* __restrict__ centre, uint32_t* amax_bits) {
    const int64_t nvalid = *rows_valid;
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    if (c >= cols) return;
    const float cc = centre ? centre[c] : 0.f;
    float m = 0.f;
    for (int64_t r = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; r < nvalid;
         r += (int64_t)gridDim.y * blockDim.y)
        m = fmaxf(m, fabsf(src[r * cols + c] - cc));
    if (m > 0.f) atomicMax(amax_bits + c, __float_as_uint(m));
}

// dst row c, element r = split(2^a_c (src[r][c] - centre[c])) for r < kpad (zero for
// r >= *rows_valid), a_c from the column's largest magnitude: transposes a chunk-major
// [rows][cols] FP32 matrix into cols paired rows with chunks contiguous, and
// inv_scale[c] = 2^-a_c.  Tiles of 64 rows x 32 columns; each thread stores two adjacent
// rows as one half2 per part (kpad is a multiple of 32, ldd even).
__global__ void k_transpose_split_f16(const float* __restrict__ src, int64_t cols,
                                      const int64_t* rows_valid, int64_t kpad, __half* dst,
                                      int64_t ldd, const float* centre,
                                      const uint32_t* __restrict__ amax_bits, float* inv_scale) {
    __shared__ float tile[64][33];
    __shared__ float sc[32];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 32;
    const int64_t nvalid = *rows_valid;
    if (threadIdx.y == 0) {
        const int64_t c = c0 + threadIdx.x;
        const int a = c < cols ? tc::row_exponent(__uint_as_float(amax_bits[c])) : 0;
        sc[threadIdx.x] = ldexpf(1.f, a);
        if (blockIdx.y == 0 && c < cols) inv_scale[c] = ldexpf(1.f, -a);
    }
    const int64_t c_ld = c0 + threadIdx.x;
    const float cen = (centre && c_ld < cols) ? centre[c_ld] : 0.f;
    for (int i = threadIdx.y; i < 64; i += blockDim.y) {
        const int64_t r = r0 + i;
        tile[i][threadIdx.x] = (r < nvalid && c_ld < cols) ? src[r * cols + c_ld] - cen : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + 2 * threadIdx.x;
        if (c < cols && r < kpad) {
            __half h0, l0, h1, l1;
            tc::split_f16(tile[2 * threadIdx.x][i] * sc[i], h0, l0);
            tc::split_f16(tile[2 * threadIdx.x + 1][i] * sc[i], h1, l1);
            __half* d = dst + c * ldd + tc::pidx(r);      // r even: one group, 4-byte aligned
            *(__half2*)d = __halves2half2(h0, h1);
            *(__half2*)(d + 32) = __halves2half2(l0, l1);
        }
    }
}

// have_max: amax_bits already holds the column maxima (taken by an earlier pass over src).
// The paired rows cover rows_pad chunks rounded up to 32 (ldd halves each, at least twice that).
cudaError_t transpose_split_f16(const float* src, int64_t cols, const int64_t* rows_valid,
                                int64_t rows_pad, __half* dst, int64_t ldd, cudaStream_t s,
                                const float* centre, uint32_t* amax_bits, float* inv_scale,
                                bool have_max) {
    if (cols <= 0 || rows_pad <= 0) return cudaSuccess;
    const int64_t kpad = tc::round32(rows_pad);
    if ((ldd & 1) || ldd < 2 * kpad) return cudaErrorInvalidValue;
    const int64_t cb = (cols + 31) / 32;
    if (!have_max) {
        cudaError_t e = cudaMemsetAsync(amax_bits, 0, sizeof(uint32_t) * (size_t)cols, s);
        if (e != cudaSuccess) return e;
        int64_t rb = (152 * 8 + cb - 1) / cb;
        if (rb < 1) rb = 1;
        k_colmax<<<dim3((unsigned)cb, (unsigned)rb), dim3(32, 8), 0, s>>>(src, cols, rows_valid,
                                                                         centre, amax_bits);
    }
    dim3 grid((unsigned)cb, (unsigned)((kpad + 63) / 64));
    k_transpose_split_f16<<<grid, dim3(32, 8), 0, s>>>(src, cols, rows_valid, kpad, dst, ldd,
                                                       centre, amax_bits, inv_scale);
    return cudaGetLastError();
}

}  // namespace hk

// Test hook (declared in no public header): the same GEMM on caller buffers, so a GPU
// test can compare it with a reference product.  D[m][n] = sum_k A[m][k] B[n][k] from
// FP32 A [M][K] and B [N][K]; scratch must hold (M+N)*ld halves (ld = 64 ceil(K / 32))
// followed by M+N floats.  Returns 0 on success.
extern "C" int hawkes_test_tc_gemm(const float* A, const float* B, float* D, int M, int N,
                                   int K, int splits, void* scratch, void* stream) {
    using namespace hk;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ld = 2 * tc::round32(K);
    __half* Ap = (__half*)scratch;
    __half* Bp = Ap + (int64_t)M * ld;
    float* inv_a = (float*)(Bp + (int64_t)N * ld);
    float* inv_b = inv_a + M;
    if (split_f16_rows(A, K, Ap, ld, M, K, s, nullptr, nullptr, inv_a, nullptr, nullptr) != cudaSuccess) return 1;
    if (split_f16_rows(B, K, Bp, ld, N, K, s, nullptr, nullptr, inv_b, nullptr, nullptr) != cudaSuccess) return 1;
    if (splits > 1) cudaMemsetAsync(D, 0, sizeof(float) * (size_t)M * N, s);
    return tc_gemm_f16x3(Ap, ld, Bp, ld, D, N, M, N, K, splits, false, nullptr, s, nullptr, inv_a,
                         inv_b) == cudaSuccess
               ? 0
               : 2;
}
