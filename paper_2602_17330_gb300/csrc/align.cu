// (a3) Affine-gap local alignment (Smith-Waterman with Gotoh's three states)
// for every candidate pair -- the alignment channel of Algorithm 1's affinity
// loop.
//
// Inter-pair parallelism: one pair per thread.  The shorter sequence (the
// "query", when the scoring matrix is symmetric) runs down the rows and is
// fully unrolled at a compile-time height NQ picked per warp (the warp's
// longest query rounded up to 4; shorter queries are padded with a residue
// whose scores are hugely negative, which can never raise the maximum).  The
// other sequence streams through the columns.  Per row the thread keeps
// E(i, j-1) and H(i, j-1) - o in registers, and the substitution scores come
// from a lane-replicated table in shared memory (entry (a, b) of lane l at word
// (a*20 + b)*32 + l, so a warp's 32 lookups hit 32 distinct banks) that already
// holds M[a][b] + o.  E and F are clamped at 0 (values below 0 can never lift
// H above its floor of 0, so the maximum is unchanged), and each cell is
//   t = (H(i-1,j-1) - o) + (M + o)
//   E = max(E - e, H(i,j-1) - o, 0)           (DPX add-max-relu)
//   F = max(F - e, H(i-1,j) - o, 0)           (DPX add-max-relu)
//   H = max(t, E, F, 0)                       (DPX max3-relu)
#include <string.h>

#include "internal.cuh"

namespace {

constexpr int kLanes = 32;
constexpr int kTabRows = 21;  // 20 residues + the padding residue
constexpr int kTabWords = kTabRows * 20 * kLanes;
constexpr int32_t kPadScore = -30000;
constexpr int kAlignThreads = 256;

template <int WORDS>
struct Rec {
    uint64_t w[WORDS];
    __device__ __forceinline__ void load(const uint64_t *__restrict__ packed, int64_t i)
    {
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(packed + i * WORDS);
        ulonglong2 a = p[0];
        w[0] = a.x;
        w[1] = a.y;
        if (WORDS == 4) {
            ulonglong2 b = p[1];
            w[2 % WORDS] = b.x;
            w[3 % WORDS] = b.y;
        }
    }
    __device__ __forceinline__ int len() const { return sq_record_len(w[0], w[1]); }
};

template <int WORDS, int NQ>
__device__ __forceinline__ int32_t sw_pair(const Rec<WORDS> &q, int Lq, const Rec<WORDS> &t, int Lt,
                                           const char *__restrict__ s_tab, int lane, int o, int e)
{
    uint32_t qoff[NQ];
    int32_t E[NQ], HM[NQ];
#pragma unroll
    for (int p = 0; p < NQ; ++p) {
        uint32_t code = (uint32_t)(q.w[p / 12] >> (5 * (p % 12))) & 31u;
        code = p < Lq ? min(code, 19u) : 20u;  // records from subquad_pack hold codes < 20
        qoff[p] = (code * 20u * kLanes + (uint32_t)lane) * 4u;
        E[p] = 0;
        HM[p] = -o;
    }
    int32_t best = 0;
    uint64_t cur = t.w[0];
    int left = 12, word = 0;
    for (int j = 0; j < Lt; ++j) {
        const uint32_t b = min((uint32_t)cur & 31u, 19u);
        cur >>= 5;
        if (--left == 0) {
            ++word;
            cur = word == 1 ? t.w[1] : t.w[2 % WORDS];
            left = 12;
        }
        const char *col = s_tab + b * (kLanes * 4);
        int32_t hm_diag = -o, hm_up = -o, F = 0;
#pragma unroll
        for (int p = 0; p < NQ; ++p) {
            const int32_t s_o = *reinterpret_cast<const int32_t *>(col + qoff[p]);
            const int32_t tdiag = hm_diag + s_o;
            const int32_t e_new = __viaddmax_s32_relu(E[p], -e, HM[p]);
            F = __viaddmax_s32_relu(F, -e, hm_up);
            const int32_t h = __vimax3_s32_relu(tdiag, e_new, F);
            hm_diag = HM[p];
            HM[p] = h - o;
            hm_up = HM[p];
            E[p] = e_new;
            best = max(best, h);
        }
    }
    return best;
}

template <int WORDS, bool SELF>
__global__ void __launch_bounds__(kAlignThreads, 2)
    align_plain_kernel(const uint64_t *__restrict__ packed, const uint32_t *__restrict__ pairs, int64_t m,
                       const int32_t *__restrict__ table, int o, int e, bool symmetric, int32_t *__restrict__ out)
{
    extern __shared__ int32_t s_tab_words[];
    for (int q = threadIdx.x; q < kTabWords / 4; q += blockDim.x)
        reinterpret_cast<int4 *>(s_tab_words)[q] = reinterpret_cast<const int4 *>(table)[q];
    __syncthreads();
    const char *s_tab = reinterpret_cast<const char *>(s_tab_words);
    constexpr int MAXLEN = WORDS == 2 ? 24 : 30;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
        const int64_t p = base + threadIdx.x;
        const bool valid = p < m;
        Rec<WORDS> A, B;
        int La = 0, Lb = 0;
        if (valid) {
            uint32_t i, j;
            if (SELF) {
                i = j = (uint32_t)p;
            } else {
                uint2 ij = reinterpret_cast<const uint2 *>(pairs)[p];
                i = ij.x;
                j = ij.y;
            }
            A.load(packed, i);
            La = min(A.len(), MAXLEN);
            if (SELF) {
                B = A;
                Lb = La;
            } else {
                B.load(packed, j);
                Lb = min(B.len(), MAXLEN);
            }
            if (symmetric && Lb < La) {
                Rec<WORDS> T = A;
                A = B;
                B = T;
                int tl = La;
                La = Lb;
                Lb = tl;
            }
        }
        const int wmax = __reduce_max_sync(0xffffffffu, La);
        if (!valid) continue;
        int32_t s;
        if (wmax <= 8) s = sw_pair<WORDS, 8>(A, La, B, Lb, s_tab, lane, o, e);
        else if (wmax <= 12) s = sw_pair<WORDS, 12>(A, La, B, Lb, s_tab, lane, o, e);
        else if (wmax <= 16) s = sw_pair<WORDS, 16>(A, La, B, Lb, s_tab, lane, o, e);
        else if (wmax <= 20) s = sw_pair<WORDS, 20>(A, La, B, Lb, s_tab, lane, o, e);
        else if (wmax <= 24) s = sw_pair<WORDS, 24>(A, La, B, Lb, s_tab, lane, o, e);
        else s = sw_pair<WORDS, MAXLEN>(A, La, B, Lb, s_tab, lane, o, e);
        out[p] = s;
    }
}

// Build (or reuse) the lane-replicated table for the context's matrix and o.
int ensure_table(subquad_ctx *ctx, int gap_open)
{
    if (ctx->d_table && ctx->table_gap_open == gap_open) return SUBQUAD_OK;
    static thread_local int32_t host[kTabWords];
    for (int a = 0; a < kTabRows; ++a)
        for (int b = 0; b < 20; ++b) {
            int32_t v = a < 20 ? (int32_t)ctx->h_matrix[20 * a + b] + gap_open : kPadScore;
            for (int l = 0; l < kLanes; ++l) host[(a * 20 + b) * kLanes + l] = v;
        }
    if (!ctx->d_table) SQ_TRY_CUDA(cudaMalloc(&ctx->d_table, sizeof(int32_t) * kTabWords));
    // earlier work on the stream may still read the previous table
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    SQ_TRY_CUDA(cudaMemcpy(ctx->d_table, host, sizeof(int32_t) * kTabWords, cudaMemcpyHostToDevice));
    ctx->table_gap_open = gap_open;
    return SUBQUAD_OK;
}

template <bool SELF>
int launch_align(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs, int64_t m, int o, int e,
                 int32_t *out)
{
    const size_t smem = sizeof(int32_t) * kTabWords;
    const unsigned grid = sq_grid(ctx, m, kAlignThreads, 2);
    if (pack_stride == 16) {
        auto k = align_plain_kernel<2, SELF>;
        SQ_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, kAlignThreads, smem, ctx->stream>>>((const uint64_t *)packed, pairs, m, ctx->d_table, o, e,
                                                      ctx->matrix_symmetric, out);
    } else {
        auto k = align_plain_kernel<4, SELF>;
        SQ_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, kAlignThreads, smem, ctx->stream>>>((const uint64_t *)packed, pairs, m, ctx->d_table, o, e,
                                                      ctx->matrix_symmetric, out);
    }
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

}  // namespace

extern "C" int subquad_align_score(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs,
                                   int64_t m, int gap_open, int gap_extend, int32_t *scores_out)
{
    SQ_ENTER(ctx);
    if (m < 0 || gap_open < 0 || gap_open > 1000 || gap_extend < 0 || gap_extend > 1000) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (m == 0) return SUBQUAD_OK;
    if (!packed || !pairs || !scores_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8) return SUBQUAD_ERR_ARG;
    SQ_TRY(ensure_table(ctx, gap_open));
    return launch_align<false>(ctx, packed, pack_stride, pairs, m, gap_open, gap_extend, scores_out);
}

extern "C" int subquad_self_scores(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n, int gap_open,
                                   int gap_extend, int32_t *self_out)
{
    SQ_ENTER(ctx);
    if (n < 0 || gap_open < 0 || gap_open > 1000 || gap_extend < 0 || gap_extend > 1000) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (n == 0) return SUBQUAD_OK;
    if (!packed || !self_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16) return SUBQUAD_ERR_ARG;
    SQ_TRY(ensure_table(ctx, gap_open));
    return launch_align<true>(ctx, packed, pack_stride, nullptr, n, gap_open, gap_extend, self_out);
}
