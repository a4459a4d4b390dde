// Host side of the C ABI (include/hawkes_gb300.h): argument checks, workspace
// layout, path choice and the launch sequence.  No memory is allocated here.
#include <stdio.h>
#include <string.h>

#include "common.cuh"

namespace {

thread_local int32_t g_last_launches = 0;

// per-kernel timing (off unless hawkes_profile_enable(1))
constexpr int kProfMax = 64;
struct Prof {
    int on = 0;
    int n = 0;
    cudaEvent_t ev[kProfMax + 1];
    const char* name[kProfMax];
    bool created = false;
};
thread_local Prof g_prof;

constexpr size_t kAlign = 256;
constexpr size_t kMaxDynamicSmem = 227 * 1024;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr int kDefaultChunkWalk = 128;
constexpr int kDefaultChunkGemm = 192;

enum Path { PATH_WALK = 1, PATH_GEMM = 2, PATH_MARKS = 3 };
constexpr int kMarksPrepChunk = 4096;   // chunks of the validation pass on the mark-major path

struct Plan {
    int path;
    int C;
    int P;
    int Gc;
    int64_t nb_max, ng_max;
    size_t off_counts, off_chunk_base, off_chunk_seq, off_Shat, off_Ghat, off_grp_v, off_grp_g,
        off_grp_dt, off_grp_reset, off_seg_comp, off_carry_S, off_carry_G, off_acc, off_Y, off_Z, off_W,
        off_dal_gemm, off_al_p, off_S_p, off_G_p, off_Wt_p, off_St_p, off_recs, off_src, off_kprep, off_dal_part, off_bstart, off_bsub, off_pwork, off_pcum, off_ptot, off_plan_b, off_wide, off_Aint, off_Bint, off_wbuf, off_delta, off_Dspan, off_Tmt,
        off_cen, off_wsum, off_colsum, off_at, off_isc, off_colmax, total;
    // mark-major walk
    size_t off_rowptr, off_supcol, off_supval, off_tcnt, off_segoff, off_segt, off_segf;
    size_t off_llpart, off_redo;
    int64_t seg_len;
    int nseg, ntiles, seg_tiles, tile_warps;
    int64_t ldk, ldt, nbp;
    hk::PairRows rows;     // row blocks of the pair kernels
    int K;                 // decay kernels (one workspace slice each)
    size_t scratch_off;
    size_t slice;          // bytes of one slice
};

// Returns 0 and fills the plan, or a hawkes_status.
int make_plan(int64_t N, int32_t M, int32_t B, int grad, const hawkes_opts* o, Plan* pl) {
    if (N < 0 || M <= 0 || B <= 0) return HAWKES_ERR_INVALID_ARG;
    const int shared = o ? o->beta_shared : 0;
    int path = o ? o->path : 0;
    const int K = (o && o->kernels > 1) ? o->kernels : 1;
    const int support = o ? o->support : 0;
    const int reduce = o ? o->reduce : 0, fp32_times = o ? o->fp32_times : 0;
    const int lanes = o ? o->walk_lanes : 0;
    if (lanes != 0 && lanes != 8 && lanes != 16 && lanes != 32) return HAWKES_ERR_INVALID_ARG;
    if (lanes != 0 && lanes < 32 && lanes < M) return HAWKES_ERR_INVALID_ARG;   // one mark per lane
    if (reduce < 0 || reduce > 2 || fp32_times < 0 || fp32_times > 1) return HAWKES_ERR_INVALID_ARG;
    if (K > hk::kMaxKernels) return HAWKES_ERR_INVALID_ARG;
    if (K > 1) {
        // several kernels, each with one shared decay: chunk-GEMM path, one sequence
        if (!shared || B != 1 || path == PATH_WALK) return HAWKES_ERR_UNSUPPORTED;
        path = PATH_GEMM;
    }
    if (path == 0) {
        if (M <= hk::walk_max_m(grad)) path = PATH_WALK;
        else path = shared ? PATH_GEMM : PATH_MARKS;
    }
    if (path == PATH_WALK && M > hk::walk_max_m(grad)) return HAWKES_ERR_UNSUPPORTED;
    if (path == PATH_GEMM && (!shared || B != 1)) return HAWKES_ERR_UNSUPPORTED;
    if (path == PATH_MARKS) {
        // one sequence, one kernel; dense rows must fit the walk's lane groups (the rows of a
        // support are checked on the device); slots and indices are int32
        if (B != 1 || K > 1) return HAWKES_ERR_UNSUPPORTED;
        if (!support && M > hk::marks_row_max()) return HAWKES_ERR_UNSUPPORTED;
        if (N >= ((int64_t)1 << 31) - hk::marks_tile_events() || M > 32768)
            return HAWKES_ERR_UNSUPPORTED;
        if (o && o->chunk < 0) return HAWKES_ERR_INVALID_ARG;
    }
    if (path != PATH_WALK && path != PATH_GEMM && path != PATH_MARKS) return HAWKES_ERR_INVALID_ARG;
    // the FP32 log-sums and the FP32-times ablation exist on the one-kernel chunk-GEMM path
    if ((reduce != 0 || fp32_times != 0) && (path != PATH_GEMM || K > 1)) return HAWKES_ERR_UNSUPPORTED;
    int C = path == PATH_MARKS ? kMarksPrepChunk
                               : (o && o->chunk > 0) ? o->chunk
                                                     : (path == PATH_WALK ? kDefaultChunkWalk
                                                                          : kDefaultChunkGemm);
    if (C < 1 || C > 4096) return HAWKES_ERR_INVALID_ARG;
    if (path == PATH_GEMM && C > 1024) return HAWKES_ERR_INVALID_ARG;
    if (path == PATH_GEMM && M > 128 * 128) return HAWKES_ERR_UNSUPPORTED;
    // per-mark shared-memory histograms of the epilogue: (2 K + 2) M words
    if (path == PATH_GEMM && sizeof(float) * (2 * (size_t)K + 2) * (size_t)M > kMaxDynamicSmem)
        return HAWKES_ERR_UNSUPPORTED;
    pl->path = path;
    pl->C = C;
    // mark blocks for the pair kernels: at most 128 marks per block, and about 26 events
    // of a chunk per block so that one bucket mostly fits one 32-lane group
    {
        int64_t Pm = ((int64_t)M + 127) / 128, Pc = ((int64_t)C + 25) / 26;
        int64_t P = Pm > Pc ? Pm : Pc;
        if (P > M) P = M;
        pl->P = (int)P;
    }
    pl->nb_max = (N + C - 1) / C + B;
    pl->off_rowptr = pl->off_supcol = pl->off_supval = pl->off_tcnt = pl->off_segoff = 0;
    pl->off_segt = pl->off_segf = 0;
    pl->off_llpart = 0;
    pl->off_redo = 0;
    pl->seg_len = 0;
    pl->nseg = pl->ntiles = pl->seg_tiles = pl->tile_warps = 0;
    if (path == PATH_MARKS) {
        // tiles of the sort, and segments of whole tiles: enough (segment, mark) work items for
        // about 64 warps per SM, at most 64 tiles (1M events) per segment, or the caller's
        // segment length (opts->chunk events, rounded up to whole tiles)
        const int64_t TE = hk::marks_tile_events();
        const int64_t ntiles = (N + TE - 1) / TE;
        int64_t tps;
        if (o && o->chunk > 0) {
            tps = ((int64_t)o->chunk + TE - 1) / TE;
        } else {
            const int64_t want_seg = (152 * 64 + (int64_t)M - 1) / M;
            tps = (ntiles + want_seg - 1) / want_seg;
            if (tps > 64) tps = 64;
        }
        if (tps < 1) tps = 1;
        pl->ntiles = (int)ntiles;
        pl->seg_tiles = (int)tps;
        pl->nseg = (int)((ntiles + tps - 1) / tps);
        pl->seg_len = tps * TE;
        int wpb = (int)((200 * 1024) / (4 * (int64_t)M));
        pl->tile_warps = wpb < 1 ? 1 : (wpb > 4 ? 4 : wpb);
    }
    int64_t target_groups = 2432;  // ~16 blocks of 128 threads per SM on 152 SMs
    int64_t gc = (pl->nb_max + target_groups - 1) / target_groups;
    if (gc < 1) gc = 1;
    if (gc > 64) gc = 64;
    pl->Gc = (int)gc;
    pl->ng_max = (pl->nb_max + gc - 1) / gc;
    const size_t nbM = (size_t)(path == PATH_MARKS ? pl->nseg : pl->nb_max) * M;
    const size_t ngM = (size_t)(path == PATH_MARKS ? 0 : pl->ng_max) * M;
    size_t o_ = align_up(sizeof(hk::WsHeader));
    auto take = [&](size_t bytes) { size_t at = o_; o_ = align_up(o_ + bytes); return at; };
    pl->off_counts = take(sizeof(int64_t) * (size_t)B * M);
    pl->off_chunk_base = take(sizeof(int64_t) * ((size_t)B + 1));
    pl->off_chunk_seq = take(sizeof(int32_t) * (size_t)pl->nb_max);
    pl->off_Shat = take(sizeof(float) * nbM);
    pl->off_Ghat = grad ? take(sizeof(float) * nbM) : 0;
    pl->off_grp_v = take(sizeof(float) * ngM);
    pl->off_grp_g = grad ? take(sizeof(float) * ngM) : 0;
    pl->off_grp_dt = take(sizeof(double) * (size_t)pl->ng_max);
    pl->off_grp_reset = take(sizeof(int32_t) * (size_t)pl->ng_max);
    pl->off_seg_comp = path == PATH_MARKS ? 0 : take(sizeof(float) * 5 * (size_t)hk::kCarrySegments * M);
    pl->off_carry_S = take(sizeof(float) * ngM);
    pl->off_carry_G = grad ? take(sizeof(float) * ngM) : 0;
    size_t n_acc = (size_t)B * (1 + 4 * (size_t)M) + (grad ? (size_t)B * M * M : 0);
    pl->off_acc = take(sizeof(double) * n_acc);
    pl->off_colsum = take(sizeof(double) * (size_t)B * M);
    pl->nbp = (pl->nb_max + 7) / 8 * 8;
    pl->ldk = ((int64_t)M + 31) / 32 * 64;          // paired fp16 rows (tc_gemm.cu)
    pl->ldt = (pl->nbp + 31) / 32 * 64;
    pl->off_Y = pl->off_Z = pl->off_W = pl->off_dal_gemm = 0;
    pl->off_al_p = pl->off_S_p = pl->off_G_p = pl->off_Wt_p = pl->off_St_p = 0;
    pl->off_recs = pl->off_src = pl->off_kprep = pl->off_dal_part = pl->off_bstart = pl->off_wide = pl->off_Aint = pl->off_Bint = pl->off_wbuf = 0;
    pl->off_bsub = pl->off_pwork = pl->off_pcum = pl->off_ptot = pl->off_plan_b = 0;
    pl->off_delta = pl->off_Dspan = pl->off_Tmt = 0;
    pl->off_cen = pl->off_wsum = pl->off_at = pl->off_isc = pl->off_colmax = 0;
    pl->rows = hk::pair_rows(M, pl->P);
    if (path == PATH_GEMM) {
        const size_t h = 2;   // fp16 operand halves
        const size_t P = (size_t)pl->P;
        pl->off_recs = take(16 * (size_t)(N > 0 ? N : 1));
        pl->off_src = take(8 * (size_t)(N > 0 ? N : 1));
        if (grad) pl->off_kprep = take(16 * (size_t)(N > 0 ? N : 1));
        // row blocks of the backward pairs: their first slots per chunk, work per chunk and
        // its prefix, the plan, and one R x M partial per plan block
        {
            const size_t n_rb = (size_t)pl->rows.n_rb, slots = (size_t)pl->rows.slots;
            pl->off_bsub = take(sizeof(int32_t) * (size_t)pl->nb_max * (n_rb + 1));
            pl->off_pwork = take(sizeof(int32_t) * n_rb * (size_t)pl->nb_max);
            pl->off_pcum = take(sizeof(int64_t) * n_rb * ((size_t)pl->nb_max + 1));
            pl->off_ptot = take(sizeof(int64_t) * n_rb);
            pl->off_plan_b = take(sizeof(int32_t) * (1 + 2 * n_rb + slots));
            if (grad) pl->off_dal_part = take(sizeof(float) * slots * ((size_t)M << pl->rows.lgR));
            if (grad) pl->off_redo = take(sizeof(int32_t) * slots);
        }
        pl->off_at = take(sizeof(float) * P * P * 128 * 128);
        pl->off_bstart = take(sizeof(int32_t) * (size_t)pl->nb_max * (P + 1));
        pl->off_wide = take((size_t)pl->nb_max);
        pl->off_Aint = take(sizeof(float) * (size_t)(N > 0 ? N : 1));
        pl->off_Bint = take(sizeof(float) * (size_t)(N > 0 ? N : 1));
        if (grad) pl->off_wbuf = take(sizeof(float) * (size_t)(N > 0 ? N : 1));
        pl->off_delta = take(sizeof(float) * (size_t)(N > 0 ? N : 1));
        pl->off_Dspan = take(sizeof(float) * (size_t)pl->nb_max);
        pl->off_Tmt = take(sizeof(float) * (size_t)pl->nb_max);
        pl->off_cen = take(sizeof(float) * ((4 + 2 * 32) * (size_t)M + 1));   // 32 = kCentreSlices
        pl->off_wsum = take(sizeof(double) * (size_t)M);
        pl->off_Y = take(sizeof(float) * nbM);
        pl->off_llpart = take(sizeof(float) * 2 * (size_t)hk::kLogSumBlocks);
        pl->off_isc = take(sizeof(float) * (3 * (size_t)M + 2 * (size_t)pl->nb_max));
        pl->off_colmax = take(sizeof(uint32_t) * 2 * (size_t)M);   // colmax, then wmax
        pl->off_al_p = take(h * (size_t)M * pl->ldk);
        pl->off_S_p = take(h * (size_t)pl->nb_max * pl->ldk);
        if (grad) {
            pl->off_Z = take(sizeof(float) * nbM);
            pl->off_W = take(sizeof(float) * (size_t)M * pl->nbp);   // transposed: [M][nbp]
            pl->off_dal_gemm = take(sizeof(float) * (size_t)M * M);
            pl->off_G_p = take(h * (size_t)pl->nb_max * pl->ldk);
            pl->off_Wt_p = take(h * (size_t)M * pl->ldt);
            pl->off_St_p = take(h * (size_t)M * pl->ldt);
        }
    }
    if (path == PATH_MARKS) {
        const size_t nnz_max = (size_t)M * M;
        pl->off_rowptr = take(sizeof(int32_t) * ((size_t)M + 1));
        pl->off_supcol = take(sizeof(int32_t) * nnz_max);
        pl->off_supval = take(sizeof(float) * nnz_max);
        pl->off_tcnt = take(sizeof(int32_t) * (size_t)pl->ntiles * M);
        pl->off_segoff = take(sizeof(int32_t) * ((size_t)pl->nseg * M + 1));
        pl->off_segt = take(sizeof(double) * 3 * (size_t)pl->nseg);
        pl->off_segf = take(sizeof(float) * 4 * (size_t)pl->nseg);
        pl->off_recs = take(16 * (size_t)(N > 0 ? N : 1));
    }
    pl->scratch_off = path == PATH_GEMM ? take(sizeof(float) * ((size_t)M + 2)) : 0;
    pl->K = K;
    pl->slice = align_up(o_);
    pl->total = (size_t)K * pl->slice;
    return 0;
}

template <typename T>
T* at(void* ws, size_t off) { return off ? (T*)((char*)ws + off) : nullptr; }

// Events of a single sequence that arrive on the device in pieces (the host-buffer entry
// point): events [0, end[i]) (and the one event after, when there is one) are on the device
// once ev[i] has completed.  Piece ends are whole scan groups.
constexpr int kMaxPieces = 8;
struct Pieces {
    int n;
    int64_t end[kMaxPieces];
    cudaEvent_t ev[kMaxPieces];
};

void bind(hk::Problem& p, void* ws, const Plan& pl, int32_t B, int32_t M, int grad) {
    p.hdr = (hk::WsHeader*)ws;
    p.counts = at<int64_t>(ws, pl.off_counts);
    p.chunk_base = at<int64_t>(ws, pl.off_chunk_base);
    p.chunk_seq = at<int32_t>(ws, pl.off_chunk_seq);
    p.Shat = at<float>(ws, pl.off_Shat);
    p.Ghat = at<float>(ws, pl.off_Ghat);
    p.grp_v = at<float>(ws, pl.off_grp_v);
    p.grp_g = at<float>(ws, pl.off_grp_g);
    p.grp_dt = at<double>(ws, pl.off_grp_dt);
    p.grp_reset = at<int32_t>(ws, pl.off_grp_reset);
    p.carry_S = at<float>(ws, pl.off_carry_S);
    p.seg_comp = at<float>(ws, pl.off_seg_comp);
    p.carry_G = at<float>(ws, pl.off_carry_G);
    double* acc = at<double>(ws, pl.off_acc);
    const size_t BM = (size_t)B * M;
    p.ll_acc = acc;
    p.dmu_acc = acc + B;
    p.dbe_acc = p.dmu_acc + BM;
    p.E_acc = p.dbe_acc + BM;
    p.F_acc = p.E_acc + BM;
    p.dal_acc = grad ? p.F_acc + BM : nullptr;
    p.colsum = at<double>(ws, pl.off_colsum);
    p.Y = at<float>(ws, pl.off_Y);
    p.Z = at<float>(ws, pl.off_Z);
    p.W = at<float>(ws, pl.off_W);
    p.dal_gemm = at<float>(ws, pl.off_dal_gemm);
    p.al_p = at<__half>(ws, pl.off_al_p);
    p.S_p = at<__half>(ws, pl.off_S_p);
    p.G_p = at<__half>(ws, pl.off_G_p);
    p.Wt_p = at<__half>(ws, pl.off_Wt_p);
    p.St_p = at<__half>(ws, pl.off_St_p);
    p.recs = at<float4>(ws, pl.off_recs);
    p.src = at<float2>(ws, pl.off_src);
    p.kprep = at<int4>(ws, pl.off_kprep);
    p.dal_part = at<float>(ws, pl.off_dal_part);
    p.scratch = at<float>(ws, pl.scratch_off);
    p.bsub = at<int32_t>(ws, pl.off_bsub);
    p.pwork = at<int32_t>(ws, pl.off_pwork);
    p.pcum = at<int64_t>(ws, pl.off_pcum);
    p.ptot = at<int64_t>(ws, pl.off_ptot);
    p.at = at<float>(ws, pl.off_at);
    p.plan_b = at<int32_t>(ws, pl.off_plan_b);
    p.lgR = pl.rows.lgR;
    p.nrb = pl.rows.nrb;
    p.n_rb = pl.rows.n_rb;
    p.pair_slots = pl.rows.slots;
    p.bstart = at<int32_t>(ws, pl.off_bstart);
    p.wide = at<uint8_t>(ws, pl.off_wide);
    p.Aint = at<float>(ws, pl.off_Aint);
    p.Bint = at<float>(ws, pl.off_Bint);
    p.wbuf = at<float>(ws, pl.off_wbuf);
    p.delta = at<float>(ws, pl.off_delta);
    p.Dspan = at<float>(ws, pl.off_Dspan);
    p.Tmt = at<float>(ws, pl.off_Tmt);
    p.cen_S = at<float>(ws, pl.off_cen);
    p.bias_Y = p.cen_S ? p.cen_S + M : nullptr;
    p.cen_Z = p.cen_S ? p.cen_S + 2 * (size_t)M : nullptr;
    p.bias_Z = p.cen_S ? p.cen_S + 3 * (size_t)M : nullptr;
    p.cen_acc = p.cen_S ? p.cen_S + 4 * (size_t)M : nullptr;
    p.wsum_acc = at<double>(ws, pl.off_wsum);
    p.isc_al = at<float>(ws, pl.off_isc);
    p.isc_S = p.isc_al ? p.isc_al + M : nullptr;
    p.isc_G = p.isc_S ? p.isc_S + pl.nb_max : nullptr;
    p.isc_Wt = p.isc_G ? p.isc_G + pl.nb_max : nullptr;
    p.isc_St = p.isc_Wt ? p.isc_Wt + M : nullptr;
    p.colmax = at<uint32_t>(ws, pl.off_colmax);
    p.wmax = p.colmax ? p.colmax + M : nullptr;
    p.w_rowstats = 0;
    p.ldk = pl.ldk;
    p.ldt = pl.ldt;
    p.nbp = pl.nbp;
    p.C = pl.C;
    p.P = pl.P;
    p.Gc = pl.Gc;
    p.nb_max = pl.nb_max;
    p.ng_max = pl.ng_max;
    p.row_ptr = at<int32_t>(ws, pl.off_rowptr);
    p.sup_col = at<int32_t>(ws, pl.off_supcol);
    p.sup_val = at<float>(ws, pl.off_supval);
    p.tile_cnt = at<int32_t>(ws, pl.off_tcnt);
    p.seg_off = at<int32_t>(ws, pl.off_segoff);
    p.seg_time = at<double>(ws, pl.off_segt);
    p.seg_f = at<float>(ws, pl.off_segf);
    p.nseg = pl.nseg;
    p.ntiles = pl.ntiles;
    p.seg_tiles = pl.seg_tiles;
    p.tile_warps = pl.tile_warps;
    p.ll_part = at<float>(ws, pl.off_llpart);
    p.pair_redo = at<int32_t>(ws, pl.off_redo);
}

int run(hk::Problem& p, const hawkes_opts* o, void* ws, size_t ws_bytes, cudaStream_t s,
        const Pieces* pieces = nullptr) {
    Plan pl;
    int rc = make_plan(p.N, p.M, p.B, p.grad, o, &pl);
    if (rc) return rc;
    if (!ws || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < pl.total) return HAWKES_ERR_WORKSPACE;
    bind(p, ws, pl, p.B, p.M, p.grad);
    int nl = 0;
    const int validate = o ? o->validate : 1;
    p.validated = validate ? 1 : 0;
    if (g_prof.on) {
        g_prof.n = 0;
        cudaEventRecord(g_prof.ev[0], s);
    }
    p.support = o ? o->support : 0;
    p.reduce = o ? o->reduce : 0;
    p.fp32_times = o ? o->fp32_times : 0;
    p.walk_lanes = o ? o->walk_lanes : 0;
    cudaError_t err;
    if (!pieces) {
        err = hk::launch_prepare(p, s, validate, &nl);
        if (err == cudaSuccess && pl.path != PATH_MARKS) err = hk::launch_scan_reduce(p, s, 0, pl.ng_max, &nl);
    } else {
        // every piece's events are checked, then composed by the scan's reduce pass, as soon as
        // they are on the device, while the later pieces are still being copied; the checks of
        // a piece come before any kernel that indexes with its marks
        err = hk::launch_prepare_head(p, s, validate, &nl);
        int64_t b_done = 0, g_done = 0;
        for (int i = 0; i < pieces->n && err == cudaSuccess; ++i) {
            const bool last = i == pieces->n - 1;
            const int64_t b_end = last ? pl.nb_max : pieces->end[i] / pl.C;
            err = cudaStreamWaitEvent(s, pieces->ev[i], 0);
            if (err == cudaSuccess && validate) err = hk::launch_validate_chunks(p, s, b_done, b_end, &nl);
            if (err == cudaSuccess && pl.path != PATH_MARKS) {
                const int64_t g_end = last ? pl.ng_max : b_end / pl.Gc;
                err = hk::launch_scan_reduce(p, s, g_done, g_end, &nl);
                g_done = g_end;
            }
            if (err == cudaSuccess && pl.path == PATH_GEMM)
                err = hk::launch_bucket_range(p, s, b_done, b_end, &nl);
            b_done = b_end;
        }
        p.bucket_done = pl.path == PATH_GEMM ? 1 : 0;
    }
    if (err == cudaSuccess) {
        if (pl.path == PATH_MARKS) {
            err = hk::launch_marks(p, pl.seg_len, s, &nl);
        } else {
            err = hk::launch_scan_rest(p, s, &nl);
            if (err == cudaSuccess && pl.path == PATH_WALK) {
                err = hk::launch_walk(p, s, &nl);
                if (err == cudaSuccess) err = hk::launch_finalize(p, s, &nl);
            } else if (err == cudaSuccess) {
                err = hk::launch_gemm_path(p, s, &nl);
            }
        }
    }
    g_last_launches = nl;
    if (err != cudaSuccess) {
        fprintf(stderr, "hawkes_gb300: CUDA error %s\n", cudaGetErrorString(err));
        return HAWKES_ERR_CUDA;
    }
    return HAWKES_OK;
}

// Several decay kernels: slice q of the workspace is a complete one-kernel problem for
// (alpha_q, beta_q); the slices run their forward parts, one epilogue combines them, they
// run their backward parts (each writing d_alpha_q, d_beta_q), and a last kernel assembles
// L and the status.  Slices q > 0 leave out -T sum(mu) and write L and dmu to scratch.
int run_multi(hk::Problem& base, const hawkes_opts* o, void* ws, size_t ws_bytes, cudaStream_t s) {
    Plan pl;
    int rc = make_plan(base.N, base.M, 1, base.grad, o, &pl);
    if (rc) return rc;
    if (!ws || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < pl.total) return HAWKES_ERR_WORKSPACE;
    const int K = pl.K, M = base.M;
    const int validate = o ? o->validate : 1;
    hk::Problem p[hk::kMaxKernels];
    hk::MultiSlices ms{};
    ms.K = K;
    for (int q = 0; q < K; ++q) {
        void* wq = (char*)ws + (size_t)q * pl.slice;
        hk::WsHeader* hdr = (hk::WsHeader*)wq;
        p[q] = base;
        bind(p[q], wq, pl, 1, M, base.grad);
        p[q].off = (const int64_t*)&hdr->pad[0];
        p[q].Tarr = (const double*)&hdr->pad[2];
        p[q].alpha = base.alpha + (size_t)q * M * M;
        p[q].beta = base.beta + q;
        p[q].validated = validate ? 1 : 0;
        p[q].support = o ? o->support : 0;
        if (base.grad) {
            p[q].d_alpha = base.d_alpha + (size_t)q * M * M;
            p[q].d_beta = base.d_beta + q;
        }
        if (q > 0) {
            p[q].base_term = 0;
            p[q].out_ll = (double*)p[q].scratch;     // 8-byte aligned: the region is 256-aligned
            if (base.grad) p[q].d_mu = p[q].scratch + 2;
            p[q].wbuf = p[0].wbuf;                   // one w per event, written by the epilogue
        }
        ms.k[q].Y = p[q].Y;
        ms.k[q].Z = p[q].Z;
        ms.k[q].A = p[q].Aint;
        ms.k[q].B = p[q].Bint;
        ms.k[q].W = p[q].W;
        ms.k[q].E_acc = p[q].E_acc;
        ms.k[q].F_acc = p[q].F_acc;
        ms.k[q].dbe_acc = p[q].dbe_acc;
        ms.k[q].wsum_acc = p[q].wsum_acc;
        ms.k[q].beta = p[q].beta;
        ms.k[q].hdr = p[q].hdr;
        ms.k[q].out_ll = p[q].out_ll;
    }
    int nl = 0;
    if (g_prof.on) {
        g_prof.n = 0;
        cudaEventRecord(g_prof.ev[0], s);
    }
    cudaError_t err = cudaSuccess;
    for (int q = 0; q < K && err == cudaSuccess; ++q) {
        err = hk::launch_prepare(p[q], s, validate, &nl);
        if (err == cudaSuccess) err = hk::launch_scan(p[q], s, &nl);
        if (err == cudaSuccess) err = hk::launch_gemm_forward(p[q], s, &nl);
    }
    if (err == cudaSuccess) err = hk::launch_epilogue_multi(p[0], ms, s, &nl);
    for (int q = 0; q < K && err == cudaSuccess; ++q) err = hk::launch_gemm_backward(p[q], s, &nl);
    if (err == cudaSuccess) {
        hk::Problem caller = p[0];
        caller.out_ll = base.out_ll;
        caller.d_alpha = base.d_alpha;
        caller.d_beta = base.d_beta;
        err = hk::launch_finalize_multi(caller, ms, s, &nl);
    }
    g_last_launches = nl;
    if (err != cudaSuccess) {
        fprintf(stderr, "hawkes_gb300: CUDA error %s\n", cudaGetErrorString(err));
        return HAWKES_ERR_CUDA;
    }
    return HAWKES_OK;
}

bool bad_ptrs(std::initializer_list<const void*> ps) {
    for (const void* q : ps)
        if (!q) return true;
    return false;
}

}  // namespace

namespace hk {
void prof_mark(cudaStream_t s, const char* name) {
    if (!g_prof.on || g_prof.n >= kProfMax) return;
    g_prof.name[g_prof.n] = name;
    cudaEventRecord(g_prof.ev[g_prof.n + 1], s);
    ++g_prof.n;
}
}  // namespace hk

extern "C" {

hawkes_opts hawkes_default_opts(void) {
    hawkes_opts o;
    o.beta_shared = 0;
    o.chunk = 0;
    o.validate = 1;
    o.path = 0;
    o.kernels = 1;
    o.support = 0;
    o.reduce = 0;
    o.fp32_times = 0;
    o.walk_lanes = 0;
    return o;
}

size_t hawkes_workspace_size(int64_t N, int32_t M, int32_t B, int32_t grad,
                             const hawkes_opts* opts) {
    Plan pl;
    if (make_plan(N, M, B, grad ? 1 : 0, opts, &pl)) return 0;
    return pl.total;
}

}  // extern "C"

namespace hk {
// The host-side checks of one single-sequence call, in the order hawkes_loglik_grad makes
// them: sizes and T, null pointers, then the configuration (make_plan).  Returns 0 or the
// status that call would return before touching the workspace.
int check_single_args(const double* t, const int32_t* c, int64_t N, double T, int32_t M,
                      const float* mu, const float* alpha, const float* beta,
                      const hawkes_opts* opts, const double* out_ll, const float* d_mu,
                      const float* d_alpha, const float* d_beta, int grad) {
    if (N < 0 || M <= 0 || !(T >= 0.0)) return HAWKES_ERR_INVALID_ARG;
    if (bad_ptrs({mu, alpha, beta, out_ll})) return HAWKES_ERR_INVALID_ARG;
    if (N > 0 && bad_ptrs({t, c})) return HAWKES_ERR_INVALID_ARG;
    if (grad && bad_ptrs({d_mu, d_alpha, d_beta})) return HAWKES_ERR_INVALID_ARG;
    Plan pl;
    return make_plan(N, M, 1, grad, opts, &pl);
}
}  // namespace hk

extern "C" {

static hawkes_status single(const double* t, const int32_t* c, int64_t N, double T, int32_t M,
                            const float* mu, const float* alpha, const float* beta,
                            const hawkes_opts* opts, void* ws, size_t ws_bytes, double* out_ll,
                            float* d_mu, float* d_alpha, float* d_beta, int grad, void* stream,
                            const float* carry_S = nullptr, const float* carry_G = nullptr,
                            int base_term = 1, const Pieces* pieces = nullptr) {
    int rc = hk::check_single_args(t, c, N, T, M, mu, alpha, beta, opts, out_ll, d_mu, d_alpha,
                                   d_beta, grad);
    if (rc) return (hawkes_status)rc;
    Plan pl;
    make_plan(N, M, 1, grad, opts, &pl);
    if (!ws || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < pl.total) return HAWKES_ERR_WORKSPACE;
    // single sequence: offsets {0, N} and T are written into the header's spare
    // words by the first kernel, so the call issues no host-to-device copy
    hk::WsHeader* hdr = (hk::WsHeader*)ws;
    cudaStream_t s = (cudaStream_t)stream;
    hk::Problem p{};
    p.t = t; p.c = c; p.off = (const int64_t*)&hdr->pad[0]; p.Tarr = (const double*)&hdr->pad[2];
    p.N = N; p.B = 1; p.M = M;
    p.single = 1; p.T_single = T;
    p.base_term = base_term;
    p.init_S = carry_S;
    p.init_G = carry_G;
    p.mu = mu; p.alpha = alpha; p.beta = beta;
    p.shared = opts ? opts->beta_shared : 0;
    p.grad = grad;
    p.out_ll = out_ll; p.d_mu = d_mu; p.d_alpha = d_alpha; p.d_beta = d_beta;
    if (pl.K > 1) {
        if (carry_S || carry_G || !base_term) return HAWKES_ERR_UNSUPPORTED;
        return (hawkes_status)run_multi(p, opts, ws, ws_bytes, s);
    }
    return (hawkes_status)run(p, opts, ws, ws_bytes, s, pieces);
}

hawkes_status hawkes_loglik(const double* t, const int32_t* c, int64_t N, double T, int32_t M,
                            const float* mu, const float* alpha, const float* beta,
                            const hawkes_opts* opts, void* workspace, size_t workspace_bytes,
                            double* out_ll, void* stream) {
    return single(t, c, N, T, M, mu, alpha, beta, opts, workspace, workspace_bytes, out_ll,
                  nullptr, nullptr, nullptr, 0, stream);
}

hawkes_status hawkes_loglik_grad(const double* t, const int32_t* c, int64_t N, double T,
                                 int32_t M, const float* mu, const float* alpha,
                                 const float* beta, const hawkes_opts* opts, void* workspace,
                                 size_t workspace_bytes, double* out_ll, float* d_mu,
                                 float* d_alpha, float* d_beta, void* stream) {
    return single(t, c, N, T, M, mu, alpha, beta, opts, workspace, workspace_bytes, out_ll,
                  d_mu, d_alpha, d_beta, 1, stream);
}

static hawkes_status varlen(const double* t, const int32_t* c, const int64_t* offsets,
                            int32_t B, int64_t N, const double* T, int32_t M, const float* mu,
                            const float* alpha, const float* beta, const hawkes_opts* opts,
                            void* ws, size_t ws_bytes, double* out_ll, float* d_mu,
                            float* d_alpha, float* d_beta, int grad, void* stream) {
    if (N < 0 || M <= 0 || B <= 0) return HAWKES_ERR_INVALID_ARG;
    if (bad_ptrs({offsets, T, mu, alpha, beta, out_ll})) return HAWKES_ERR_INVALID_ARG;
    if (N > 0 && bad_ptrs({t, c})) return HAWKES_ERR_INVALID_ARG;
    if (grad && bad_ptrs({d_mu, d_alpha, d_beta})) return HAWKES_ERR_INVALID_ARG;
    hk::Problem p{};
    p.t = t; p.c = c; p.off = offsets; p.Tarr = T;
    p.N = N; p.B = B; p.M = M;
    p.base_term = 1;
    p.mu = mu; p.alpha = alpha; p.beta = beta;
    p.shared = opts ? opts->beta_shared : 0;
    p.grad = grad;
    p.out_ll = out_ll; p.d_mu = d_mu; p.d_alpha = d_alpha; p.d_beta = d_beta;
    return (hawkes_status)run(p, opts, ws, ws_bytes, (cudaStream_t)stream);
}

hawkes_status hawkes_loglik_varlen(const double* t, const int32_t* c, const int64_t* offsets,
                                   int32_t B, int64_t N, const double* T, int32_t M,
                                   const float* mu, const float* alpha, const float* beta,
                                   const hawkes_opts* opts, void* workspace,
                                   size_t workspace_bytes, double* out_ll, void* stream) {
    return varlen(t, c, offsets, B, N, T, M, mu, alpha, beta, opts, workspace, workspace_bytes,
                  out_ll, nullptr, nullptr, nullptr, 0, stream);
}

hawkes_status hawkes_loglik_grad_varlen(const double* t, const int32_t* c,
                                        const int64_t* offsets, int32_t B, int64_t N,
                                        const double* T, int32_t M, const float* mu,
                                        const float* alpha, const float* beta,
                                        const hawkes_opts* opts, void* workspace,
                                        size_t workspace_bytes, double* out_ll, float* d_mu,
                                        float* d_alpha, float* d_beta, void* stream) {
    return varlen(t, c, offsets, B, N, T, M, mu, alpha, beta, opts, workspace, workspace_bytes,
                  out_ll, d_mu, d_alpha, d_beta, 1, stream);
}

hawkes_status hawkes_loglik_grad_slice(const double* t, const int32_t* c, int64_t N, double T,
                                       int32_t M, const float* mu, const float* alpha,
                                       const float* beta, const hawkes_opts* opts,
                                       const float* carry_S, const float* carry_G,
                                       int32_t base_term, void* workspace,
                                       size_t workspace_bytes, double* out_ll, float* d_mu,
                                       float* d_alpha, float* d_beta, void* stream) {
    if ((carry_S == nullptr) != (carry_G == nullptr)) return HAWKES_ERR_INVALID_ARG;
    return single(t, c, N, T, M, mu, alpha, beta, opts, workspace, workspace_bytes, out_ll, d_mu,
                  d_alpha, d_beta, 1, stream, carry_S, carry_G, base_term ? 1 : 0);
}

hawkes_status hawkes_slice_aggregate(const double* t, const int32_t* c, int64_t N, int32_t M,
                                     const float* beta, const hawkes_opts* opts, double t_next,
                                     void* workspace, size_t workspace_bytes, float* agg_S,
                                     float* agg_G, void* stream) {
    if (N < 0 || M <= 0 || !beta || !agg_S || !agg_G) return HAWKES_ERR_INVALID_ARG;
    if (N > 0 && (!t || !c)) return HAWKES_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0 ||
        workspace_bytes < align_up(sizeof(hk::WsHeader)))
        return HAWKES_ERR_WORKSPACE;
    hk::Problem p{};
    p.t = t; p.c = c; p.N = N; p.B = 1; p.M = M;
    p.beta = beta;
    p.shared = opts ? opts->beta_shared : 0;
    p.hdr = (hk::WsHeader*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    // the header's status word is cleared here; the events are assumed to have been
    // validated by the caller's hawkes_loglik_grad_slice on the same slice
    if (cudaMemsetAsync(workspace, 0, sizeof(int32_t), s) != cudaSuccess) return HAWKES_ERR_CUDA;
    int nl = 0;
    cudaError_t e = hk::launch_slice_aggregate(p, t_next, agg_S, agg_G, s, &nl);
    g_last_launches = nl;
    return e == cudaSuccess ? HAWKES_OK : HAWKES_ERR_CUDA;
}

// Host-buffer form: staging for inputs and outputs sits after the device workspace.
static size_t host_staging_bytes(int64_t N, int32_t M, int shared) {
    size_t b = align_up(sizeof(double) * (size_t)N) + align_up(sizeof(int32_t) * (size_t)N);
    b += align_up(sizeof(float) * (size_t)M) * 2 + align_up(sizeof(float) * (size_t)M * M) * 2;
    b += align_up(sizeof(float) * (size_t)(shared ? 1 : M)) * 2 + align_up(sizeof(double));
    return b;
}

size_t hawkes_workspace_size_host(int64_t N, int32_t M, const hawkes_opts* opts) {
    size_t dev = hawkes_workspace_size(N, M, 1, 1, opts);
    if (!dev) return 0;
    return align_up(dev) + host_staging_bytes(N, M, opts ? opts->beta_shared : 0);
}

// The host entry point's copy stream and events, created once per thread and device.
struct HostPipe {
    int dev = -1;
    cudaStream_t copy = nullptr;
    cudaEvent_t start = nullptr;
    cudaEvent_t ev[kMaxPieces] = {};
};
thread_local HostPipe g_pipe;

static cudaError_t host_pipe() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (g_pipe.dev == dev) return cudaSuccess;
    HostPipe h;
    h.dev = dev;
    e = cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming);
    for (int i = 0; i < kMaxPieces && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&h.ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) g_pipe = h;     // (a thread that changes devices keeps the old ones)
    return e;
}

hawkes_status hawkes_loglik_grad_host(const double* t, const int32_t* c, int64_t N, double T,
                                      int32_t M, const float* mu, const float* alpha,
                                      const float* beta, const hawkes_opts* opts,
                                      void* workspace, size_t workspace_bytes, double* out_ll,
                                      float* d_mu, float* d_alpha, float* d_beta,
                                      void* stream) {
    if (N < 0 || M <= 0) return HAWKES_ERR_INVALID_ARG;
    if (bad_ptrs({mu, alpha, beta, out_ll, d_mu, d_alpha, d_beta})) return HAWKES_ERR_INVALID_ARG;
    if (N > 0 && bad_ptrs({t, c})) return HAWKES_ERR_INVALID_ARG;
    if (opts && opts->kernels > 1) return HAWKES_ERR_UNSUPPORTED;   // one kernel only here
    size_t dev = hawkes_workspace_size(N, M, 1, 1, opts);
    if (!dev) return HAWKES_ERR_UNSUPPORTED;
    if (!workspace || workspace_bytes < hawkes_workspace_size_host(N, M, opts))
        return HAWKES_ERR_WORKSPACE;
    Plan pl;
    make_plan(N, M, 1, 1, opts, &pl);
    const int shared = opts ? opts->beta_shared : 0;
    const size_t nbeta = shared ? 1 : (size_t)M;
    char* st = (char*)workspace + align_up(dev);
    auto take = [&](size_t bytes) { char* q = st; st += align_up(bytes); return q; };
    double* t_d = (double*)take(sizeof(double) * (size_t)N);
    int32_t* c_d = (int32_t*)take(sizeof(int32_t) * (size_t)N);
    float* mu_d = (float*)take(sizeof(float) * (size_t)M);
    float* dmu_d = (float*)take(sizeof(float) * (size_t)M);
    float* al_d = (float*)take(sizeof(float) * (size_t)M * M);
    float* dal_d = (float*)take(sizeof(float) * (size_t)M * M);
    float* be_d = (float*)take(sizeof(float) * nbeta);
    float* dbe_d = (float*)take(sizeof(float) * nbeta);
    double* ll_d = (double*)take(sizeof(double));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // The events go to the device in pieces of whole scan groups on a second stream (one
    // cudaMemcpyAsync per array and piece), each followed by an event that the kernels wait
    // for, so that the checks and the scan's reduce pass of a piece run while the next
    // piece is copied.  The copies wait for the work queued on `stream` before this call.
    Pieces pieces{};
    if (N > 0) {
        e = host_pipe();
        const int64_t unit = pl.path == PATH_MARKS ? (int64_t)pl.C : (int64_t)pl.Gc * pl.C;
        int64_t np = N / ((int64_t)1 << 21);
        if (np < 1) np = 1;
        if (np > kMaxPieces) np = kMaxPieces;
        int64_t len = (N + np - 1) / np;
        len = (len + unit - 1) / unit * unit;
        if (e == cudaSuccess) e = cudaEventRecord(g_pipe.start, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g_pipe.copy, g_pipe.start, 0);
        for (int64_t a0 = 0; a0 < N && e == cudaSuccess; a0 += len) {
            const int64_t b0 = a0 + len < N ? a0 + len : N;
            const int64_t tb = b0 < N ? b0 + 1 : N;     // and the next piece's first time
            e = cudaMemcpyAsync(t_d + a0, t + a0, sizeof(double) * (size_t)(tb - a0),
                                cudaMemcpyHostToDevice, g_pipe.copy);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c_d + a0, c + a0, sizeof(int32_t) * (size_t)(b0 - a0),
                                    cudaMemcpyHostToDevice, g_pipe.copy);
            if (e == cudaSuccess) e = cudaEventRecord(g_pipe.ev[pieces.n], g_pipe.copy);
            pieces.end[pieces.n] = b0;
            pieces.ev[pieces.n] = g_pipe.ev[pieces.n];
            ++pieces.n;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mu_d, mu, sizeof(float) * M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(al_d, alpha, sizeof(float) * (size_t)M * M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(be_d, beta, sizeof(float) * nbeta, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return HAWKES_ERR_CUDA;
    hawkes_status rc = single(t_d, c_d, N, T, M, mu_d, al_d, be_d, opts, workspace, dev, ll_d,
                              dmu_d, dal_d, dbe_d, 1, stream, nullptr, nullptr, 1,
                              pieces.n > 0 ? &pieces : nullptr);
    if (rc != HAWKES_OK) {
        cudaStreamSynchronize(g_pipe.copy);      // no copy may outlive the call
        return rc;
    }
    e = cudaMemcpyAsync(out_ll, ll_d, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mu, dmu_d, sizeof(float) * M, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_alpha, dal_d, sizeof(float) * (size_t)M * M, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_beta, dbe_d, sizeof(float) * nbeta, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return HAWKES_ERR_CUDA;
    return hawkes_last_device_status(workspace, stream);
}

hawkes_status hawkes_last_device_status(void* workspace, void* stream) {
    if (!workspace) return HAWKES_ERR_WORKSPACE;
    int32_t st = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&st, workspace, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return HAWKES_ERR_CUDA;
    return (hawkes_status)st;
}

const int64_t* hawkes_mark_counts(void* workspace) {
    if (!workspace) return nullptr;
    return (const int64_t*)((char*)workspace + align_up(sizeof(hk::WsHeader)));
}

hawkes_status hawkes_integer_tables(void* workspace, int64_t N, int32_t M, int32_t B,
                                    int32_t grad, const hawkes_opts* opts, hawkes_tables* out) {
    if (!workspace || !out) return HAWKES_ERR_INVALID_ARG;
    Plan pl;
    int rc = make_plan(N, M, B, grad ? 1 : 0, opts, &pl);
    if (rc) return (hawkes_status)rc;
    out->mark_counts = at<int64_t>(workspace, pl.off_counts);
    out->chunk_base = at<int64_t>(workspace, pl.off_chunk_base);
    out->chunk_seq = at<int32_t>(workspace, pl.off_chunk_seq);
    const bool gemm = pl.path == PATH_GEMM, marks = pl.path == PATH_MARKS;
    out->bucket_start = gemm ? at<int32_t>(workspace, pl.off_bstart) : nullptr;
    out->bucket_slots = gemm ? at<uint32_t>(workspace, pl.off_recs) : nullptr;
    out->chunk = pl.C;
    out->mark_blocks = gemm ? pl.P : 0;
    out->support_row_ptr = marks ? at<int32_t>(workspace, pl.off_rowptr) : nullptr;
    out->support_col = marks ? at<int32_t>(workspace, pl.off_supcol) : nullptr;
    out->mark_start = marks ? at<int32_t>(workspace, pl.off_segoff) : nullptr;
    out->mark_slots = marks ? at<uint32_t>(workspace, pl.off_recs) : nullptr;
    out->segment_events = marks ? pl.seg_len : 0;
    out->segments = marks ? pl.nseg : 0;
    out->reserved = 0;
    return HAWKES_OK;
}

const char* hawkes_status_str(hawkes_status s) {
    switch (s) {
        case HAWKES_OK: return "ok";
        case HAWKES_ERR_INVALID_ARG: return "invalid argument";
        case HAWKES_ERR_UNSORTED: return "event times not sorted";
        case HAWKES_ERR_MARK_RANGE: return "mark outside [0, M)";
        case HAWKES_ERR_TIME_RANGE: return "event time outside [0, T]";
        case HAWKES_ERR_PARAM_DOMAIN: return "parameter outside its domain";
        case HAWKES_ERR_NONPOS_INTENSITY: return "non-positive intensity";
        case HAWKES_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case HAWKES_ERR_UNSUPPORTED: return "configuration not supported";
        case HAWKES_ERR_CUDA: return "CUDA runtime error";
    }
    return "unknown status";
}

int32_t hawkes_last_launch_count(void) { return g_last_launches; }

int32_t hawkes_profile_enable(int32_t on) {
    if (on && !g_prof.created) {
        for (int i = 0; i <= kProfMax; ++i)
            if (cudaEventCreate(&g_prof.ev[i]) != cudaSuccess) return HAWKES_ERR_CUDA;
        g_prof.created = true;
    }
    g_prof.on = on ? 1 : 0;
    g_prof.n = 0;
    return HAWKES_OK;
}

int32_t hawkes_profile_read(float* ms, const char** names, int32_t cap) {
    if (!g_prof.created) return 0;
    int n = g_prof.n < cap ? g_prof.n : cap;
    if (n > 0 && cudaEventSynchronize(g_prof.ev[n]) != cudaSuccess) return -HAWKES_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        float t = 0.f;
        cudaEventElapsedTime(&t, g_prof.ev[i], g_prof.ev[i + 1]);
        ms[i] = t;
        names[i] = g_prof.name[i];
    }
    return n;
}

}  // extern "C"
