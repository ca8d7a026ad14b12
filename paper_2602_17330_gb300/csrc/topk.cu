// (a7) Cross-donor retrieval: the k best partners of each query among the
// sequences of other donors, ranked by (alignment score desc, id asc).
//
// Two producers feed one warp-level top-k structure:
//  * subquad_topk_candidates -- the query's partners in the candidate graph
//    (its runs in the pair index), with the alignment scores already computed;
//  * subquad_topk_bruteforce -- every sequence of another donor, aligned on
//    the fly (all lanes of a warp share the query, so the query's score-table
//    offsets are warp-uniform): the exhaustive reference that recall@k of the
//    candidate route is measured against.
// A candidate is one 64-bit key, (score + 2^31) << 32 | (0xffffffff - id), so a
// larger key is a better candidate and keys of one query are unique.  Each
// warp keeps its current best k keys sorted in shared memory; every round of
// 32 new keys is sorted with a warp bitonic network and merged by rank
// (binary searches in both sorted lists), keeping the first k.
#include "internal.cuh"

namespace {

constexpr int kTopThreads = 256;
constexpr int kTopWarps = kTopThreads / 32;
constexpr int kMaxK = 256;

__device__ __forceinline__ uint64_t make_key(int32_t score, uint32_t id)
{
    return ((uint64_t)((uint32_t)score + 0x80000000u) << 32) | (uint64_t)(0xffffffffu - id);
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src_lane_xor)
{
    return __shfl_xor_sync(0xffffffffu, v, src_lane_xor);
}

// Bitonic sort of one key per lane, descending across lanes.
__device__ __forceinline__ uint64_t warp_sort_desc(uint64_t x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t y = shfl64(x, stride);
            const bool lower = (lane & stride) == 0;
            const bool desc = (lane & size) == 0;  // direction of this bitonic block
            const bool keep_max = (lower == desc);
            x = keep_max ? (x > y ? x : y) : (x < y ? x : y);
        }
    }
    return x;
}

// Number of entries of the descending array a[0..len) that are > x.
__device__ __forceinline__ int count_greater(const uint64_t *a, int len, uint64_t x)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] > x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

struct WarpTopK {
    uint64_t *list;   // current best keys, descending, `size` valid
    uint64_t *next;   // scratch for the merge
    uint64_t *chunk;  // 32 sorted new keys
    int size, k;

    // Warp-collective: every lane offers one key (0 = nothing).
    __device__ __forceinline__ void offer(uint64_t x)
    {
        const int lane = threadIdx.x & 31;
        if (size == k && x <= list[k - 1]) x = 0;  // cannot enter the list
        if (!__any_sync(0xffffffffu, x != 0)) return;
        x = warp_sort_desc(x);
        const int nnew = __popc(__ballot_sync(0xffffffffu, x != 0));
        chunk[lane] = x;
        __syncwarp();
        if (x != 0) {
            const int pos = lane + count_greater(list, size, x);
            if (pos < k) next[pos] = x;
        }
        for (int l = lane; l < size; l += 32) {
            const uint64_t y = list[l];
            const int pos = l + count_greater(chunk, nnew, y);
            if (pos < k) next[pos] = y;
        }
        __syncwarp();
        size = min(k, size + nnew);
        uint64_t *t = list;
        list = next;
        next = t;
    }

    __device__ __forceinline__ void write(int64_t qi, uint32_t *top_id, int32_t *top_score) const
    {
        const int lane = threadIdx.x & 31;
        for (int r = lane; r < k; r += 32) {
            uint32_t id = 0xffffffffu;
            int32_t sc = -1;
            if (r < size) {
                const uint64_t key = list[r];
                id = 0xffffffffu - (uint32_t)(key & 0xffffffffu);
                sc = (int32_t)((uint32_t)(key >> 32) - 0x80000000u);
            }
            top_id[qi * k + r] = id;
            top_score[qi * k + r] = sc;
        }
    }
};

__global__ void __launch_bounds__(kTopThreads) topk_candidates_kernel(
    const uint32_t *__restrict__ pairs, const int32_t *__restrict__ scores, const int32_t *__restrict__ donor,
    const uint32_t *__restrict__ perm_i, const uint32_t *__restrict__ off_i, const uint32_t *__restrict__ perm_j,
    const uint32_t *__restrict__ off_j, const uint32_t *__restrict__ queries, int64_t nq, int64_t n, int k,
    uint32_t *__restrict__ top_id, int32_t *__restrict__ top_score, uint32_t *err)
{
    __shared__ uint64_t s_buf[kTopWarps][2 * kMaxK + 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint2 *pr = reinterpret_cast<const uint2 *>(pairs);
    for (int64_t qi = gw; qi < nq; qi += nw) {
        const uint32_t q = queries[qi];
        if (q >= (uint64_t)n) {
            if (lane == 0) atomicOr(err, SQ_DEVERR_INPUT);
            continue;
        }
        WarpTopK top{s_buf[warp], s_buf[warp] + kMaxK, s_buf[warp] + 2 * kMaxK, 0, k};
        const int32_t dq = donor[q];
        for (int side = 0; side < 2; ++side) {
            const uint32_t *perm = side == 0 ? perm_i : perm_j;
            const uint32_t *off = side == 0 ? off_i : off_j;
            const uint32_t q0 = off[q], q1 = off[q + 1];
            for (uint32_t b = q0; b < q1; b += 32) {
                uint64_t key = 0;
                if (b + lane < q1) {
                    const uint32_t p = perm[b + lane];
                    const uint2 ij = pr[p];
                    const uint32_t other = side == 0 ? ij.y : ij.x;
                    if (donor[other] != dq) key = make_key(scores[p], other);
                }
                top.offer(key);
            }
        }
        top.write(qi, top_id, top_score);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Exhaustive reference: every query against every sequence of another donor.
// ---------------------------------------------------------------------------
constexpr int kLanes = 32;
constexpr int kTabRows = 21;
constexpr int kTabWords = kTabRows * kTabRows * kLanes;

template <int NQ>
__device__ __forceinline__ int32_t sw_query(const uint32_t (&qoff)[30], uint64_t t0, uint64_t t1, uint64_t t2, int Lt,
                                            const char *__restrict__ s_tab, int o, int e)
{
    int32_t E[NQ], HM[NQ];
#pragma unroll
    for (int p = 0; p < NQ; ++p) {
        E[p] = 0;
        HM[p] = -o;
    }
    int32_t best = 0;
    uint64_t cur = t0;
    int left = 12, word = 0;
    for (int j = 0; j < Lt; ++j) {
        const uint32_t b = min((uint32_t)cur & 31u, 19u);
        cur >>= 5;
        if (--left == 0) {
            ++word;
            cur = word == 1 ? t1 : t2;
            left = 12;
        }
        const char *col = s_tab + b * (kLanes * 4);
        int32_t hm_diag = -o, hm_up = -o, F = 0;
#pragma unroll
        for (int p = 0; p < NQ; ++p) {
            const int32_t s_o = *reinterpret_cast<const int32_t *>(col + qoff[p]);
            const int32_t e_new = __viaddmax_s32_relu(E[p], -e, HM[p]);
            F = __viaddmax_s32_relu(F, -e, hm_up);
            const int32_t h = __viaddmax_s32_relu(hm_diag, s_o, max(e_new, F));
            hm_diag = HM[p];
            HM[p] = h - o;
            hm_up = HM[p];
            E[p] = e_new;
            best = max(best, h);
        }
    }
    return best;
}

template <int WORDS>
__global__ void __launch_bounds__(kTopThreads) topk_bruteforce_kernel(
    const uint64_t *__restrict__ packed, int64_t n, const int32_t *__restrict__ donor,
    const int32_t *__restrict__ table, int o, int e, const uint32_t *__restrict__ queries, int64_t nq, int k,
    uint32_t *__restrict__ top_id, int32_t *__restrict__ top_score, uint32_t *err)
{
    extern __shared__ uint64_t s_dyn[];
    int32_t *s_tab_words = reinterpret_cast<int32_t *>(s_dyn);
    uint64_t *s_lists = s_dyn + kTabWords / 2;
    for (int q = threadIdx.x; q < kTabWords / 4; q += blockDim.x)
        reinterpret_cast<int4 *>(s_tab_words)[q] = reinterpret_cast<const int4 *>(table)[q];
    __syncthreads();
    const char *s_tab = reinterpret_cast<const char *>(s_tab_words);
    constexpr int MAXLEN = WORDS == 2 ? 24 : 30;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t *mine = s_lists + (size_t)warp * (2 * kMaxK + 32);
    for (int64_t qi = gw; qi < nq; qi += nw) {
        const uint32_t q = queries[qi];
        if (q >= (uint64_t)n) {
            if (lane == 0) atomicOr(err, SQ_DEVERR_INPUT);
            continue;
        }
        uint64_t qw[WORDS];
        const ulonglong2 *rq = reinterpret_cast<const ulonglong2 *>(packed + (int64_t)q * WORDS);
        const ulonglong2 r0 = rq[0];
        qw[0] = r0.x;
        qw[1 % WORDS] = r0.y;
        if (WORDS == 4) {
            const ulonglong2 r1 = rq[1];
            qw[2 % WORDS] = r1.x;
            qw[3 % WORDS] = r1.y;
        }
        const int Lq = min(sq_record_len(qw[0], qw[1 % WORDS]), MAXLEN);
        uint32_t qoff[30];
#pragma unroll
        for (int p = 0; p < 30; ++p) {
            uint32_t code = (uint32_t)(qw[(p / 12) < WORDS ? p / 12 : 0] >> (5 * (p % 12))) & 31u;
            code = p < Lq ? min(code, 19u) : 20u;
            qoff[p] = (code * kTabRows * kLanes + (uint32_t)lane) * 4u;
        }
        const int32_t dq = donor[q];
        WarpTopK top{mine, mine + kMaxK, mine + 2 * kMaxK, 0, k};
        for (int64_t b = 0; b < n; b += 32) {
            const int64_t t = b + lane;
            uint64_t key = 0;
            bool take = t < n && donor[t] != dq;
            uint64_t tw[WORDS];
            int Lt = 0;
            if (take) {
                const ulonglong2 *rt = reinterpret_cast<const ulonglong2 *>(packed + t * WORDS);
                const ulonglong2 a = rt[0];
                tw[0] = a.x;
                tw[1 % WORDS] = a.y;
                if (WORDS == 4) {
                    const ulonglong2 c = rt[1];
                    tw[2 % WORDS] = c.x;
                    tw[3 % WORDS] = c.y;
                }
                Lt = min(sq_record_len(tw[0], tw[1 % WORDS]), MAXLEN);
            } else {
#pragma unroll
                for (int w = 0; w < WORDS; ++w) tw[w] = 0;
            }
            int32_t sc;
            const uint64_t t0 = tw[0], t1 = tw[1 % WORDS], t2 = WORDS == 4 ? tw[2 % WORDS] : 0ull;
            // the query's height is warp-uniform
            if (Lq <= 12) sc = sw_query<12>(qoff, t0, t1, t2, Lt, s_tab, o, e);
            else if (Lq <= 16) sc = sw_query<16>(qoff, t0, t1, t2, Lt, s_tab, o, e);
            else if (Lq <= 20) sc = sw_query<20>(qoff, t0, t1, t2, Lt, s_tab, o, e);
            else if (Lq <= 24) sc = sw_query<24>(qoff, t0, t1, t2, Lt, s_tab, o, e);
            else sc = sw_query<(WORDS == 2 ? 24 : 30)>(qoff, t0, t1, t2, Lt, s_tab, o, e);
            if (take) key = make_key(sc, (uint32_t)t);
            top.offer(key);
        }
        top.write(qi, top_id, top_score);
        __syncwarp();
    }
}

}  // namespace

extern "C" int subquad_topk_candidates(subquad_ctx *ctx, const uint32_t *pairs, const int32_t *scores, int64_t m,
                                       int64_t n, const int32_t *donor, const uint32_t *perm_i,
                                       const uint32_t *off_i, const uint32_t *perm_j, const uint32_t *off_j,
                                       const uint32_t *queries, int64_t nq, int k, uint32_t *top_id,
                                       int32_t *top_score)
{
    SQ_ENTER(ctx);
    if (m < 0 || n < 1 || nq < 0 || k < 1 || k > kMaxK) return SUBQUAD_ERR_ARG;
    if (nq == 0) return SUBQUAD_OK;
    if (!donor || !off_i || !off_j || !queries || !top_id || !top_score) return SUBQUAD_ERR_ARG;
    if (m > 0 && (!pairs || !scores || !perm_i || !perm_j)) return SUBQUAD_ERR_ARG;
    const unsigned grid = sq_grid(ctx, nq * 32, kTopThreads, 8);
    topk_candidates_kernel<<<grid, kTopThreads, 0, ctx->stream>>>(pairs, scores, donor, perm_i, off_i, perm_j, off_j,
                                                                  queries, nq, n, k, top_id, top_score, ctx->d_err);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

extern "C" int subquad_topk_bruteforce(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n,
                                       const int32_t *donor, int gap_open, int gap_extend, const uint32_t *queries,
                                       int64_t nq, int k, uint32_t *top_id, int32_t *top_score)
{
    SQ_ENTER(ctx);
    if (n < 1 || nq < 0 || k < 1 || k > kMaxK || gap_open < 0 || gap_open > 1000 || gap_extend < 0 ||
        gap_extend > 1000)
        return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (nq == 0) return SUBQUAD_OK;
    if (!packed || !donor || !queries || !top_id || !top_score) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16) return SUBQUAD_ERR_ARG;
    SQ_TRY(sq_ensure_align_table(ctx, gap_open));
    const size_t smem = sizeof(int32_t) * kTabWords + sizeof(uint64_t) * kTopWarps * (2 * kMaxK + 32);
    const unsigned grid = sq_grid(ctx, nq * 32, kTopThreads, 1);
    if (pack_stride == 16) {
        auto kern = topk_bruteforce_kernel<2>;
        SQ_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, kTopThreads, smem, ctx->stream>>>((const uint64_t *)packed, n, donor, ctx->d_table, gap_open,
                                                       gap_extend, queries, nq, k, top_id, top_score, ctx->d_err);
    } else {
        auto kern = topk_bruteforce_kernel<4>;
        SQ_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, kTopThreads, smem, ctx->stream>>>((const uint64_t *)packed, n, donor, ctx->d_table, gap_open,
                                                       gap_extend, queries, nq, k, top_id, top_score, ctx->d_err);
    }
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}
