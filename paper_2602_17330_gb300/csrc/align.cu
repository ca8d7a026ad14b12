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
// (a*21 + b)*32 + l, so a warp's 32 lookups hit 32 distinct banks) that already
// holds M[a][b] + o (a and b = 20 is the padding residue).  E and F are clamped at 0 (values below 0 can never lift
// H above its floor of 0, so the maximum is unchanged), and each cell is
//   t = (H(i-1,j-1) - o) + (M + o)
//   E = max(E - e, H(i,j-1) - o, 0)           (DPX add-max-relu)
//   F = max(F - e, H(i-1,j) - o, 0)           (DPX add-max-relu)
//   H = max(t, E, F, 0)                       (DPX max3-relu)
#include <string.h>

#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kLanes = 32;
constexpr int kTabRows = 21;  // 20 residues + the padding residue (rows and columns)
constexpr int kTabWords = kTabRows * kTabRows * kLanes;
// Substitution score of the padding residue.  Any value <= 0 keeps padded
// rows/columns from raising the maximum (their cells are bounded by the real
// cells above/left of them); -64 keeps every 16-bit intermediate in range.
constexpr int32_t kPadScore = -64;
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
        qoff[p] = (code * kTabRows * kLanes + (uint32_t)lane) * 4u;
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
        for (int b = 0; b < kTabRows; ++b) {
            const int32_t v = (a < 20 && b < 20 ? (int32_t)ctx->h_matrix[20 * a + b] : kPadScore) + gap_open;
            for (int l = 0; l < kLanes; ++l) host[(a * kTabRows + b) * kLanes + l] = v;
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
    SqProfScope prof(ctx, SELF ? SUBQUAD_PROF_SELF : SUBQUAD_PROF_ALIGN);
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

// ---------------------------------------------------------------------------
// Length-binned scheduling.  Pairs are counted into bins by (query length,
// target length), a single block turns the counts into offsets, and a
// warp-aggregated scatter writes the bin-ordered work list.  The alignment
// kernel then gives each warp 32 consecutive entries of the list: their
// lengths agree, so the unrolled height is the exact query length and no lane
// idles waiting for a longer target.
// ---------------------------------------------------------------------------
constexpr int kBins = 32 * 32;

// Item count of a launch sized for m_max: *d_m when the caller keeps the count
// on the device (graph-captured pipelines), else m_max.
__device__ __forceinline__ int64_t items(int64_t m_max, const unsigned long long *d_m)
{
    if (!d_m) return m_max;
    const int64_t c = (int64_t)*d_m;
    return c < m_max ? c : m_max;
}

// Sequence ids of work item p, and its bin: (query length, target length)
// after orientation.
template <bool SELF>
__device__ __forceinline__ uint2 ids_of_item(const uint32_t *__restrict__ pairs, int64_t p)
{
    if (SELF) return make_uint2((uint32_t)p, (uint32_t)p);
    return reinterpret_cast<const uint2 *>(pairs)[p];
}

template <int WORDS>
__device__ __forceinline__ uint32_t bin_of_ids(const uint64_t *__restrict__ packed, uint2 ij, bool symmetric)
{
    constexpr int MAXLEN = WORDS == 2 ? 24 : 30;
    const uint32_t i = ij.x, j = ij.y;
    const ulonglong2 ri = reinterpret_cast<const ulonglong2 *>(packed + (int64_t)i * WORDS)[0];
    const ulonglong2 rj = reinterpret_cast<const ulonglong2 *>(packed + (int64_t)j * WORDS)[0];
    const int La = min(sq_record_len(ri.x, ri.y), MAXLEN), Lb = min(sq_record_len(rj.x, rj.y), MAXLEN);
    const int Lq = symmetric ? min(La, Lb) : La, Lt = symmetric ? max(La, Lb) : Lb;
    return (uint32_t)(Lq * 32 + Lt);
}

// Shared-memory add of one item to its bin; returns the item's position
// among the bin's adds (any order).
__device__ __forceinline__ uint32_t smem_bin_add(uint32_t *s_arr, uint32_t bin, bool valid)
{
    return valid ? atomicAdd(&s_arr[bin], 1u) : 0u;
}

// Each block histograms one contiguous range of items in shared memory and
// adds its non-zero bins to the global counts: one global atomic per block
// and bin, instead of one per warp on a few hot bins.
template <int WORDS, bool SELF>
__global__ void __launch_bounds__(256) bin_count_kernel(const uint64_t *__restrict__ packed,
                                                        const uint32_t *__restrict__ pairs, int64_t m_max,
                                                        const unsigned long long *__restrict__ d_m, bool symmetric,
                                                        uint16_t *__restrict__ bin_of, uint32_t *__restrict__ counts)
{
    __shared__ uint32_t s_hist[kBins];
    const int64_t m = items(m_max, d_m);
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) s_hist[b] = 0;
    __syncthreads();
    const int64_t per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(m, lo + per);
    // four items per thread and iteration (their record gathers in flight
    // together); the next iteration's ids are loaded one iteration ahead
    constexpr int H = 4;
    uint2 nxt[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int64_t p = lo + h * (int64_t)blockDim.x + threadIdx.x;
        nxt[h] = p < hi ? ids_of_item<SELF>(pairs, p) : make_uint2(0, 0);
    }
    for (int64_t base = lo; base < hi; base += (int64_t)blockDim.x * H) {
        uint2 cur[H];
        uint32_t bin[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            cur[h] = nxt[h];
            const int64_t pn = base + (int64_t)blockDim.x * H + h * (int64_t)blockDim.x + threadIdx.x;
            nxt[h] = pn < hi ? ids_of_item<SELF>(pairs, pn) : make_uint2(0, 0);
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int64_t p = base + h * (int64_t)blockDim.x + threadIdx.x;
            bin[h] = p < hi ? bin_of_ids<WORDS>(packed, cur[h], symmetric) : kBins;
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int64_t p = base + h * (int64_t)blockDim.x + threadIdx.x;
            if (bin[h] < (uint32_t)kBins) {
                bin_of[p] = (uint16_t)bin[h];
                smem_bin_add(s_hist, bin[h], true);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x)
        if (s_hist[b]) atomicAdd(&counts[b], s_hist[b]);
}

// Exclusive scan of the kBins counts (one thread per bin, 32 warps).
__global__ void __launch_bounds__(kBins) bin_offsets_kernel(uint32_t *__restrict__ counts)
{
    static_assert(kBins == 32 * 32, "one warp per 32 bins, 32 warps");
    __shared__ uint32_t s_w[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t v = counts[threadIdx.x];
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += y;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = s_w[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if ((int)lane >= o) wi += y;
        }
        s_w[lane] = wi - w;
    }
    __syncthreads();
    counts[threadIdx.x] = s_w[warp] + inc - v;
}

// Same block ranges as bin_count_kernel: the block reserves one slice of each
// bin with a single global atomic, then places its items in shared memory.
__global__ void __launch_bounds__(256) bin_scatter_kernel(const uint16_t *__restrict__ bin_of, int64_t m_max,
                                                          const unsigned long long *__restrict__ d_m,
                                                          uint32_t *__restrict__ cursor, uint32_t *__restrict__ order)
{
    __shared__ uint32_t s_cnt[kBins];
    const int64_t m = items(m_max, d_m);
    __shared__ uint32_t s_base[kBins];
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    const int64_t per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(m, lo + per);
    constexpr int H = 4;
    for (int64_t base = lo; base < hi; base += (int64_t)blockDim.x * H) {
        uint32_t bin[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int64_t p = base + h * (int64_t)blockDim.x + threadIdx.x;
            bin[h] = p < hi ? bin_of[p] : (uint32_t)kBins;
        }
#pragma unroll
        for (int h = 0; h < H; ++h)
            if (bin[h] < (uint32_t)kBins) smem_bin_add(s_cnt, bin[h], true);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) {
        s_base[b] = s_cnt[b] ? atomicAdd(&cursor[b], s_cnt[b]) : 0u;
        s_cnt[b] = 0;
    }
    __syncthreads();
    for (int64_t base = lo; base < hi; base += (int64_t)blockDim.x * H) {
        uint32_t bin[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int64_t p = base + h * (int64_t)blockDim.x + threadIdx.x;
            bin[h] = p < hi ? bin_of[p] : (uint32_t)kBins;
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int64_t p = base + h * (int64_t)blockDim.x + threadIdx.x;
            if (bin[h] < (uint32_t)kBins) order[s_base[bin[h]] + smem_bin_add(s_cnt, bin[h], true)] = (uint32_t)p;
        }
    }
}

// Two pairs per thread in packed 16-bit halves (pair P low, pair Q high).  Per
// cell: two table lookups combined with one bitwise select, then
//   E = max(E - e, H(i,j-1) - o, 0)   F = max(F - e, H(i-1,j) - o, 0)  (DPX add-max-relu)
//   H = max((H(i-1,j-1) - o) + (M + o), max(E, F), 0)                  (packed max, DPX add-max-relu)
// Every intermediate lies in [-1064, 2953] for |M| <= 64, o, e <= 1000 and
// lengths <= 30, so 16-bit lanes are exact.  A pair shorter than the other
// one in its thread is padded with the padding residue in both dimensions.
__device__ __forceinline__ uint32_t pack2(int32_t lo, int32_t hi)
{
    return ((uint32_t)lo & 0xffffu) | ((uint32_t)hi << 16);
}

template <int WORDS>
struct TargetStream {
    uint64_t cur;
    int left, word;
    const Rec<WORDS> *t;
    __device__ __forceinline__ explicit TargetStream(const Rec<WORDS> &r) : cur(r.w[0]), left(12), word(0), t(&r) {}
    __device__ __forceinline__ uint32_t next()
    {
        const uint32_t b = min((uint32_t)cur & 31u, 19u);
        cur >>= 5;
        if (--left == 0) {
            ++word;
            cur = word == 1 ? t->w[1] : t->w[2 % WORDS];
            left = 12;
        }
        return b;
    }
};

// SPLIT (launch shape 2): the table is staged twice, scores in the low half
// of each word (zero above) and in the high half (zero below); a pair of
// lookups combines with one integer multiply-add by the runtime constant
// `unit` (= 1), and the lookup addresses are formed the same way, so this
// arithmetic runs on the FMA pipe and leaves the ALU pipe (where the DPX and
// packed max operations run) to the recurrence.
template <int WORDS, int NQ, bool SPLIT = false>
__device__ __forceinline__ uint32_t sw_pair2(const Rec<WORDS> &qP, int LqP, const Rec<WORDS> &tP, int LtP,
                                             const Rec<WORDS> &qQ, int LqQ, const Rec<WORDS> &tQ, int LtQ,
                                             const char *__restrict__ s_tab, int lane, int o, int e, uint32_t unit = 1)
{
    uint32_t qoffP[NQ], qoffQ[NQ], E[NQ], HM[NQ];
    const uint32_t neg_o = pack2(-o, -o), neg_e = pack2(-e, -e);
#pragma unroll
    for (int p = 0; p < NQ; ++p) {
        uint32_t cp = (uint32_t)(qP.w[p / 12] >> (5 * (p % 12))) & 31u;
        uint32_t cq = (uint32_t)(qQ.w[p / 12] >> (5 * (p % 12))) & 31u;
        cp = p < LqP ? min(cp, 19u) : 20u;
        cq = p < LqQ ? min(cq, 19u) : 20u;
        qoffP[p] = (cp * kTabRows * kLanes + (uint32_t)lane) * 4u;
        qoffQ[p] = (cq * kTabRows * kLanes + (uint32_t)lane) * 4u;
        E[p] = 0u;
        HM[p] = neg_o;
    }
    // Two target columns per iteration, the second one row behind the first:
    // column j's row p and column j+1's row p-1 are independent, so each step
    // carries two dependency chains (F -> max -> H -> H-o) instead of one.  A
    // column beyond the target's length scores every cell with the padding
    // residue and can never raise the maximum.
    uint32_t best = 0u;
    TargetStream<WORDS> sP(tP), sQ(tQ);
    const int Lt = max(LtP, LtQ);
    for (int j = 0; j < Lt; j += 2) {
        const uint32_t aP = sP.next(), aQ = sQ.next();
        const uint32_t bP = sP.next(), bQ = sQ.next();
        const uint32_t offAP = (j < LtP ? aP : 20u) * (kLanes * 4);
        const uint32_t offAQ = (j < LtQ ? aQ : 20u) * (kLanes * 4) + (SPLIT ? kTabWords * 4u : 0u);
        const uint32_t offBP = (j + 1 < LtP ? bP : 20u) * (kLanes * 4);
        const uint32_t offBQ = (j + 1 < LtQ ? bQ : 20u) * (kLanes * 4) + (SPLIT ? kTabWords * 4u : 0u);
        const char *colAP = s_tab + offAP, *colAQ = s_tab + offAQ;
        const char *colBP = s_tab + offBP, *colBQ = s_tab + offBQ;
        uint32_t dA = neg_o, upA = neg_o, FA = 0u;
        uint32_t dB = neg_o, upB = neg_o, FB = 0u;
#pragma unroll
        for (int p = 0; p <= NQ; ++p) {
            uint32_t hA = 0u, hB = 0u;
            if (p < NQ) {  // column j, row p
                uint32_t s_o;
                if (SPLIT) {
                    const uint32_t lo = *reinterpret_cast<const uint32_t *>(s_tab + (qoffP[p] * unit + offAP));
                    const uint32_t hi = *reinterpret_cast<const uint32_t *>(s_tab + (qoffQ[p] * unit + offAQ));
                    s_o = hi * unit + lo;
                } else {
                    const uint32_t lo = *reinterpret_cast<const uint32_t *>(colAP + qoffP[p]);
                    const uint32_t hi = *reinterpret_cast<const uint32_t *>(colAQ + qoffQ[p]);
                    s_o = (lo & 0x0000ffffu) | (hi & 0xffff0000u);
                }
                const uint32_t e_new = __viaddmax_s16x2_relu(E[p], neg_e, HM[p]);
                FA = __viaddmax_s16x2_relu(FA, neg_e, upA);
                hA = __viaddmax_s16x2_relu(dA, s_o, __vmaxs2(e_new, FA));
                dA = HM[p];
                HM[p] = __vadd2(hA, neg_o);
                upA = HM[p];
                E[p] = e_new;
            }
            if (p >= 1) {  // column j + 1, row p - 1
                const int r = p >= 1 ? p - 1 : 0;
                uint32_t s_o;
                if (SPLIT) {
                    const uint32_t lo = *reinterpret_cast<const uint32_t *>(s_tab + (qoffP[r] * unit + offBP));
                    const uint32_t hi = *reinterpret_cast<const uint32_t *>(s_tab + (qoffQ[r] * unit + offBQ));
                    s_o = hi * unit + lo;
                } else {
                    const uint32_t lo = *reinterpret_cast<const uint32_t *>(colBP + qoffP[r]);
                    const uint32_t hi = *reinterpret_cast<const uint32_t *>(colBQ + qoffQ[r]);
                    s_o = (lo & 0x0000ffffu) | (hi & 0xffff0000u);
                }
                const uint32_t e_new = __viaddmax_s16x2_relu(E[r], neg_e, HM[r]);
                FB = __viaddmax_s16x2_relu(FB, neg_e, upB);
                hB = __viaddmax_s16x2_relu(dB, s_o, __vmaxs2(e_new, FB));
                dB = HM[r];
                HM[r] = __vadd2(hB, neg_o);
                upB = HM[r];
                E[r] = e_new;
            }
            // the running maximum takes both chains' cells with one 3-input max
            // (a cell outside its chain's range is 0 and changes nothing)
            best = __vimax3_s16x2_relu(best, hA, hB);
        }
    }
    return best;
}

// Launch shapes of the batched kernel: 0 = 256 threads, 2 blocks per SM (128
// registers); 1 = 128 threads, 3 blocks per SM (168 registers, no spills up
// to 24 rows); 2 = one block of 384 threads per SM (168 registers) sharing
// the two staged tables of the split lookup.  Chosen by the context's tuning
// (see subquad_set_tuning).
template <int CFG>
struct BinnedShape {
    static constexpr int threads = CFG == 0 ? 256 : CFG == 1 ? 128 : 384;
    static constexpr int blocks = CFG == 0 ? 2 : CFG == 1 ? 3 : 1;
    static constexpr bool split = CFG == 2;  // two staged tables (see sw_pair2)
    static constexpr int tables = split ? 2 : 1;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Sequence ids (i, j) of work-list entry q and the pair index it came from.
template <bool SELF>
__device__ __forceinline__ uint4 entry_ids(const uint32_t *__restrict__ order, const uint32_t *__restrict__ pairs,
                                           int64_t q, int64_t m)
{
    if (q >= m) return make_uint4(0u, 0u, 0u, 0u);
    const uint32_t p = order[q];
    if (SELF) return make_uint4(p, p, p, 1u);
    const uint2 ij = reinterpret_cast<const uint2 *>(pairs)[p];
    return make_uint4(ij.x, ij.y, p, 1u);
}

template <int WORDS>
__device__ __forceinline__ void orient(Rec<WORDS> &A, int &La, Rec<WORDS> &B, int &Lb, bool symmetric)
{
    constexpr int MAXLEN = WORDS == 2 ? 24 : 30;
    La = min(A.len(), MAXLEN);
    Lb = min(B.len(), MAXLEN);
    if (symmetric && Lb < La) {
        const Rec<WORDS> T = A;
        A = B;
        B = T;
        const int tl = La;
        La = Lb;
        Lb = tl;
    }
}

template <int WORDS, bool SELF, int CFG>
__global__ void __launch_bounds__(BinnedShape<CFG>::threads, BinnedShape<CFG>::blocks)
    align_binned_kernel(const uint64_t *__restrict__ packed, const uint32_t *__restrict__ pairs,
                        const uint32_t *__restrict__ order, int64_t m_max, const unsigned long long *__restrict__ d_m,
                        const int32_t *__restrict__ table, int o, int e, bool symmetric, int32_t *__restrict__ out,
                        uint32_t unit)
{
    extern __shared__ int32_t s_tab_words[];
    const int64_t m = items(m_max, d_m);
    // each staged word holds its 16-bit score in both halves, so the two
    // pairs' scores combine with one bitwise select (low half of the first
    // word, high half of the second); the split shape stages the low halves
    // and the high halves as two tables instead
    constexpr bool kSplit = BinnedShape<CFG>::split;
    for (int q = threadIdx.x; q < kTabWords / 4; q += blockDim.x) {
        const int4 v = reinterpret_cast<const int4 *>(table)[q];
        const uint32_t x = (uint32_t)v.x & 0xffffu, y = (uint32_t)v.y & 0xffffu, z = (uint32_t)v.z & 0xffffu,
                       w = (uint32_t)v.w & 0xffffu;
        if (kSplit) {
            reinterpret_cast<uint4 *>(s_tab_words)[q] = make_uint4(x, y, z, w);
            reinterpret_cast<uint4 *>(s_tab_words + kTabWords)[q] = make_uint4(x << 16, y << 16, z << 16, w << 16);
        } else {
            reinterpret_cast<uint4 *>(s_tab_words)[q] = make_uint4(x * 0x10001u, y * 0x10001u, z * 0x10001u,
                                                                   w * 0x10001u);
        }
    }
    __syncthreads();
    const char *s_tab = reinterpret_cast<const char *>(s_tab_words);
    constexpr int MAXLEN = WORDS == 2 ? 24 : 30;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t stride = nwarps * 64;
    // Per thread, a double buffer of its two entries' four records in shared
    // memory (after the table).  Each warp takes 64 consecutive entries of the
    // bin-ordered list per iteration (entry base + lane in the low halves,
    // base + 32 + lane in the high halves); the records of iteration k+1 are
    // copied with cp.async while iteration k computes, and the ids of
    // iteration k+2 are loaded meanwhile.  A thread reads only what it copied.
    Rec<WORDS> *buf =
        reinterpret_cast<Rec<WORDS> *>(s_tab_words + BinnedShape<CFG>::tables * kTabWords) + threadIdx.x * 8;
    auto issue = [&](int slot, uint4 idP, uint4 idQ) {
        Rec<WORDS> *d = buf + slot * 4;
        if (idP.w) {
#pragma unroll
            for (int c = 0; c < WORDS / 2; ++c) {
                cp_async16(reinterpret_cast<char *>(d + 0) + 16 * c, packed + (int64_t)idP.x * WORDS + 2 * c);
                cp_async16(reinterpret_cast<char *>(d + 1) + 16 * c, packed + (int64_t)idP.y * WORDS + 2 * c);
            }
        }
        if (idQ.w) {
#pragma unroll
            for (int c = 0; c < WORDS / 2; ++c) {
                cp_async16(reinterpret_cast<char *>(d + 2) + 16 * c, packed + (int64_t)idQ.x * WORDS + 2 * c);
                cp_async16(reinterpret_cast<char *>(d + 3) + 16 * c, packed + (int64_t)idQ.y * WORDS + 2 * c);
            }
        }
        cp_async_commit();
    };
    int64_t base = warp * 64;
    uint4 curP = entry_ids<SELF>(order, pairs, base + lane, m), curQ = entry_ids<SELF>(order, pairs, base + 32 + lane, m);
    issue(0, curP, curQ);
    uint4 nxtP = entry_ids<SELF>(order, pairs, base + stride + lane, m);
    uint4 nxtQ = entry_ids<SELF>(order, pairs, base + stride + 32 + lane, m);
    for (int k = 0; base < m; ++k, base += stride) {
        issue((k + 1) & 1, nxtP, nxtQ);  // empty group past the end
        const uint4 farP = entry_ids<SELF>(order, pairs, base + 2 * stride + lane, m);
        const uint4 farQ = entry_ids<SELF>(order, pairs, base + 2 * stride + 32 + lane, m);
        cp_async_wait1();  // this iteration's records have landed
        const bool vP = curP.w != 0, vQ = curQ.w != 0;
        const Rec<WORDS> *r = buf + (k & 1) * 4;
        Rec<WORDS> AP, BP, AQ, BQ;
        int LaP = 0, LbP = 0, LaQ = 0, LbQ = 0;
        if (vP) {
            AP = r[0];
            BP = r[1];
            orient<WORDS>(AP, LaP, BP, LbP, symmetric);
        } else {
#pragma unroll
            for (int w = 0; w < WORDS; ++w) AP.w[w] = BP.w[w] = 0;
        }
        if (vQ) {
            AQ = r[2];
            BQ = r[3];
            orient<WORDS>(AQ, LaQ, BQ, LbQ, symmetric);
        } else {
            AQ = AP;
            BQ = BP;
            LaQ = LaP;
            LbQ = LbP;
        }
        const int wmax = __reduce_max_sync(0xffffffffu, max(LaP, LaQ));
        if (vP) {
            uint32_t sc;
            // rows: the warp's longest query, exactly for the pair lists' common
            // lengths (7..24 with 16-byte records), else rounded up to even
            constexpr bool kExact = WORDS == 2 && !SELF;
            if (kExact && wmax >= 7) {
                switch (wmax) {
#define SQ_EXACT(N)                                                                                                \
    case N:                                                                                                        \
        sc = sw_pair2<WORDS, (N <= MAXLEN ? N : MAXLEN), kSplit>(AP, LaP, BP, LbP, AQ, LaQ, BQ, LbQ, s_tab, lane, o, \
                                                                e, unit);                                          \
        break;
                    SQ_EXACT(7) SQ_EXACT(8) SQ_EXACT(9) SQ_EXACT(10) SQ_EXACT(11) SQ_EXACT(12) SQ_EXACT(13)
                    SQ_EXACT(14) SQ_EXACT(15) SQ_EXACT(16) SQ_EXACT(17) SQ_EXACT(18) SQ_EXACT(19) SQ_EXACT(20)
                    SQ_EXACT(21) SQ_EXACT(22) SQ_EXACT(23)
#undef SQ_EXACT
                default:
                    sc = sw_pair2<WORDS, MAXLEN, kSplit>(AP, LaP, BP, LbP, AQ, LaQ, BQ, LbQ, s_tab, lane, o, e, unit);
                    break;
                }
            } else {
                switch ((wmax + 1) >> 1) {
#define SQ_CASE(H)                                                                                                 \
    case H:                                                                                                        \
        sc = sw_pair2<WORDS, (H < 1 ? 2 : (2 * H <= MAXLEN ? 2 * H : MAXLEN)), kSplit>(                            \
            AP, LaP, BP, LbP, AQ, LaQ, BQ, LbQ, s_tab, lane, o, e, unit);                                          \
        break;
                    SQ_CASE(0) SQ_CASE(1) SQ_CASE(2) SQ_CASE(3) SQ_CASE(4) SQ_CASE(5) SQ_CASE(6) SQ_CASE(7)
                    SQ_CASE(8) SQ_CASE(9) SQ_CASE(10) SQ_CASE(11) SQ_CASE(12)
#undef SQ_CASE
                default:
                    sc = sw_pair2<WORDS, MAXLEN, kSplit>(AP, LaP, BP, LbP, AQ, LaQ, BQ, LbQ, s_tab, lane, o, e, unit);
                    break;
                }
            }
            out[curP.z] = (int32_t)(sc & 0xffffu);
            if (vQ) out[curQ.z] = (int32_t)(sc >> 16);
        }
        curP = nxtP;
        curQ = nxtQ;
        nxtP = farP;
        nxtQ = farQ;
    }
}

// Length-binned work list of m items in context scratch: *order_out lists the
// item indices grouped by (query length, target length) bin.  The bins are
// the scheduler shared by the batched alignment and edit-distance kernels.
template <bool SELF>
int build_work_list(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs, int64_t m,
                    const unsigned long long *d_m, bool symmetric, uint32_t **order_out)
{
    if (m >= (int64_t(1) << 32)) return SUBQUAD_ERR_ARG;
    SqArena measure(nullptr);
    measure.take<uint32_t>(kBins);
    measure.take<uint16_t>(m);
    measure.take<uint32_t>(m);
    SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    SqArena a(ctx->scratch);
    uint32_t *counts = a.take<uint32_t>(kBins);
    uint16_t *bin_of = a.take<uint16_t>(m);
    uint32_t *order = a.take<uint32_t>(m);
    SqProfScope prof_bin(ctx, SUBQUAD_PROF_ALIGN_BIN);
    SQ_TRY_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * kBins, ctx->stream));
    const unsigned g = sq_grid(ctx, m, 256, 8);
    const uint64_t *pk = static_cast<const uint64_t *>(packed);
    if (pack_stride == 16)
        bin_count_kernel<2, SELF><<<g, 256, 0, ctx->stream>>>(pk, pairs, m, d_m, symmetric, bin_of, counts);
    else
        bin_count_kernel<4, SELF><<<g, 256, 0, ctx->stream>>>(pk, pairs, m, d_m, symmetric, bin_of, counts);
    SQ_LAUNCH_CHECK();
    bin_offsets_kernel<<<1, kBins, 0, ctx->stream>>>(counts);
    SQ_LAUNCH_CHECK();
    bin_scatter_kernel<<<g, 256, 0, ctx->stream>>>(bin_of, m, d_m, counts, order);
    SQ_LAUNCH_CHECK();
    *order_out = order;
    return SUBQUAD_OK;
}

template <bool SELF>
int launch_binned(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs, int64_t m, int o,
                  int e, int32_t *out, const unsigned long long *d_m = nullptr)
{
    uint32_t *order = nullptr;
    SQ_TRY(build_work_list<SELF>(ctx, packed, pack_stride, pairs, m, d_m, ctx->matrix_symmetric, &order));
    const uint64_t *pk = static_cast<const uint64_t *>(packed);
    SqProfScope prof(ctx, SELF ? SUBQUAD_PROF_SELF : SUBQUAD_PROF_ALIGN);
#define SQ_BINNED(W, C)                                                                                            \
    do {                                                                                                           \
        auto k = align_binned_kernel<W, SELF, C>;                                                                  \
        const size_t smem = sizeof(int32_t) * kTabWords * BinnedShape<C>::tables +                                \
                            sizeof(uint64_t) * W * 8 * BinnedShape<C>::threads;                                    \
        static std::mutex attr_mutex;                                                                              \
        static bool attr_set[64] = {};                                                                             \
        const bool slot_ok = ctx->device >= 0 && ctx->device < 64;                                                 \
        bool need_attr;                                                                                            \
        {                                                                                                          \
            std::lock_guard<std::mutex> lock(attr_mutex);                                                          \
            need_attr = !slot_ok || !attr_set[ctx->device];                                                        \
        }                                                                                                          \
        if (need_attr) { /* racing first launches both set it: harmless */                                         \
            SQ_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));         \
            if (slot_ok) {                                                                                         \
                std::lock_guard<std::mutex> lock(attr_mutex);                                                      \
                attr_set[ctx->device] = true;                                                                      \
            }                                                                                                      \
        }                                                                                                          \
        const unsigned grid = sq_grid(ctx, (m + 1) / 2, BinnedShape<C>::threads, BinnedShape<C>::blocks);         \
        k<<<grid, BinnedShape<C>::threads, smem, ctx->stream>>>(pk, pairs, order, m, d_m, ctx->d_table, o, e,      \
                                                               ctx->matrix_symmetric, out, 1u);                    \
    } while (0)
    const int cfg = ctx->tune[SUBQUAD_TUNE_ALIGN_SHAPE];
    if (pack_stride == 16) {
        if (cfg == 0) SQ_BINNED(2, 0);
        else if (cfg == 1) SQ_BINNED(2, 1);
        else SQ_BINNED(2, 2);
    } else {
        if (cfg == 0) SQ_BINNED(4, 0);
        else if (cfg == 1) SQ_BINNED(4, 1);
        else SQ_BINNED(4, 2);
    }
#undef SQ_BINNED
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

}  // namespace

int sq_ensure_align_table(subquad_ctx *ctx, int gap_open) { return ensure_table(ctx, gap_open); }

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

namespace {

struct DiagScores {
    int8_t d[20];
};

// Self-scores when the matrix is diagonally dominant (see subquad_ctx): the
// sum of the diagonal entries over the residues, one thread per sequence.
template <int WORDS>
__global__ void self_diag_kernel(const uint64_t *__restrict__ packed, int64_t n, DiagScores diag,
                                 int32_t *__restrict__ out)
{
    constexpr int MAXLEN = WORDS == 2 ? 24 : 30;
    __shared__ int32_t s_d[32];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < 20; ++a) s_d[a] = diag.d[a];
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Rec<WORDS> r;
        r.load(packed, i);
        const int L = min(r.len(), MAXLEN);
        int32_t s = 0;
#pragma unroll
        for (int p = 0; p < MAXLEN; ++p) {
            const uint32_t c = min((uint32_t)(r.w[p / 12] >> (5 * (p % 12))) & 31u, 19u);
            s += p < L ? s_d[c] : 0;
        }
        out[i] = s;
    }
}

int launch_self_diag(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n, int32_t *out)
{
    DiagScores d;
    for (int a = 0; a < 20; ++a) d.d[a] = ctx->h_matrix[21 * a];
    const unsigned grid = sq_grid(ctx, n, 256, 8);
    SqProfScope prof(ctx, SUBQUAD_PROF_SELF);
    if (pack_stride == 16)
        self_diag_kernel<2><<<grid, 256, 0, ctx->stream>>>(static_cast<const uint64_t *>(packed), n, d, out);
    else
        self_diag_kernel<4><<<grid, 256, 0, ctx->stream>>>(static_cast<const uint64_t *>(packed), n, d, out);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

}  // namespace

extern "C" int subquad_self_scores(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n, int gap_open,
                                   int gap_extend, int32_t *self_out)
{
    SQ_ENTER(ctx);
    if (n < 0 || gap_open < 0 || gap_open > 1000 || gap_extend < 0 || gap_extend > 1000) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (n == 0) return SUBQUAD_OK;
    if (!packed || !self_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16) return SUBQUAD_ERR_ARG;
    if (ctx->self_is_diagonal) return launch_self_diag(ctx, packed, pack_stride, n, self_out);
    SQ_TRY(ensure_table(ctx, gap_open));
    return launch_align<true>(ctx, packed, pack_stride, nullptr, n, gap_open, gap_extend, self_out);
}

extern "C" int subquad_align_score_binned(subquad_ctx *ctx, const void *packed, int pack_stride,
                                          const uint32_t *pairs, int64_t m, int gap_open, int gap_extend,
                                          int32_t *scores_out)
{
    SQ_ENTER(ctx);
    if (m < 0 || gap_open < 0 || gap_open > 1000 || gap_extend < 0 || gap_extend > 1000) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (m == 0) return SUBQUAD_OK;
    if (!packed || !pairs || !scores_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8) return SUBQUAD_ERR_ARG;
    SQ_TRY(ensure_table(ctx, gap_open));
    return launch_binned<false>(ctx, packed, pack_stride, pairs, m, gap_open, gap_extend, scores_out);
}

extern "C" int subquad_self_scores_binned(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n,
                                          int gap_open, int gap_extend, int32_t *self_out)
{
    SQ_ENTER(ctx);
    if (n < 0 || gap_open < 0 || gap_open > 1000 || gap_extend < 0 || gap_extend > 1000) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (n == 0) return SUBQUAD_OK;
    if (!packed || !self_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16) return SUBQUAD_ERR_ARG;
    if (ctx->self_is_diagonal) return launch_self_diag(ctx, packed, pack_stride, n, self_out);
    SQ_TRY(ensure_table(ctx, gap_open));
    return launch_binned<true>(ctx, packed, pack_stride, nullptr, n, gap_open, gap_extend, self_out);
}

extern "C" int subquad_align_score_binned_async(subquad_ctx *ctx, const void *packed, int pack_stride,
                                                const uint32_t *pairs, const uint64_t *d_m, int64_t m_max,
                                                int gap_open, int gap_extend, int32_t *scores_out)
{
    SQ_ENTER(ctx);
    if (!d_m || m_max < 0 || gap_open < 0 || gap_open > 1000 || gap_extend < 0 || gap_extend > 1000)
        return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (m_max == 0) return SUBQUAD_OK;
    if (!packed || !pairs || !scores_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8) return SUBQUAD_ERR_ARG;
    SQ_TRY(ensure_table(ctx, gap_open));
    return launch_binned<false>(ctx, packed, pack_stride, pairs, m_max, gap_open, gap_extend, scores_out,
                                reinterpret_cast<const unsigned long long *>(d_m));
}

namespace {

// ---------------------------------------------------------------------------
// Edit distance (the GPU appendix's edit-distance recurrence) as a second
// alignment mode on the same length-binned scheduler:
//   D(x, y) = min(D(x-1, y) + indel, D(x, y-1) + indel,
//                 D(x-1, y-1) + sub(a_x, b_y)),   D(x, 0) = x indel,
//   D(0, y) = y indel,  distance = D(La, Lb),
// with the context's costs (sub symmetric, zero on the diagonal).  Two pairs
// per thread in packed 16-bit halves, the shorter sequence unrolled down the
// rows at the warp's common height, the longer streamed through the columns.
// Rows below a pair's query and columns right of its target are made
// transparent: a move down into a padding row and a move right into a padding
// column cost 0, and the padding residue's substitution cost is indel against
// a real residue and 0 against itself; every path to the bottom-right corner
// of the padded grid then costs at least D(La, Lb) and one costs exactly that,
// so the corner holds the distance.  Per cell (DPX):
//   t = D(x-1, y-1) + sub;  m = min(D(x, y-1) + h_y, t);  D = min(D(x-1, y) + v_x, m).
// Every value is at most 60 x 255 < 2^15, so 16-bit lanes are exact.
// ---------------------------------------------------------------------------
constexpr int kEdRows = 21;  // 20 residues + the padding residue
constexpr int kEdWords = kEdRows * kEdRows * kLanes;

int ensure_edit_table(subquad_ctx *ctx)
{
    if (ctx->d_edit_table && ctx->edit_table_valid) return SUBQUAD_OK;
    static thread_local uint32_t host[kEdWords];
    for (int a = 0; a < kEdRows; ++a)
        for (int b = 0; b < kEdRows; ++b) {
            uint32_t v;
            if (a < 20 && b < 20) v = ctx->h_edit_sub[20 * a + b];
            else if (a == 20 && b == 20) v = 0;
            else v = (uint32_t)ctx->edit_indel;
            for (int l = 0; l < kLanes; ++l) host[(a * kEdRows + b) * kLanes + l] = v * 0x10001u;
        }
    if (!ctx->d_edit_table) SQ_TRY_CUDA(cudaMalloc(&ctx->d_edit_table, sizeof(uint32_t) * kEdWords));
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));  // earlier work may still read the old table
    SQ_TRY_CUDA(cudaMemcpy(ctx->d_edit_table, host, sizeof(uint32_t) * kEdWords, cudaMemcpyHostToDevice));
    ctx->edit_table_valid = true;
    return SUBQUAD_OK;
}

// SPLIT: the cost table staged as low halves and high halves (see sw_pair2).
template <int WORDS, int NQ, bool SPLIT = false>
__device__ __forceinline__ uint32_t ed_pair2(const Rec<WORDS> &qP, int LqP, const Rec<WORDS> &tP, int LtP,
                                             const Rec<WORDS> &qQ, int LqQ, const Rec<WORDS> &tQ, int LtQ,
                                             const char *__restrict__ s_tab, int lane, int indel, uint32_t unit = 1)
{
    uint32_t qoffP[NQ], qoffQ[NQ], D[NQ], vc[NQ];
    uint32_t acc = 0u;
#pragma unroll
    for (int p = 0; p < NQ; ++p) {
        uint32_t cp = (uint32_t)(qP.w[p / 12] >> (5 * (p % 12))) & 31u;
        uint32_t cq = (uint32_t)(qQ.w[p / 12] >> (5 * (p % 12))) & 31u;
        cp = p < LqP ? min(cp, 19u) : 20u;
        cq = p < LqQ ? min(cq, 19u) : 20u;
        qoffP[p] = (cp * kEdRows * kLanes + (uint32_t)lane) * 4u;
        qoffQ[p] = (cq * kEdRows * kLanes + (uint32_t)lane) * 4u;
        vc[p] = pack2(p < LqP ? indel : 0, p < LqQ ? indel : 0);
        acc = __vadd2(acc, vc[p]);
        D[p] = acc;  // D(p + 1, 0)
    }
    TargetStream<WORDS> sP(tP), sQ(tQ);
    const int Lt = max(LtP, LtQ);
    uint32_t top = 0u;  // D(0, y)
    for (int j = 0; j < Lt; ++j) {
        const uint32_t aP = sP.next(), aQ = sQ.next();
        const uint32_t offP = (j < LtP ? aP : 20u) * (kLanes * 4);
        const uint32_t offQ = (j < LtQ ? aQ : 20u) * (kLanes * 4) + (SPLIT ? kEdWords * 4u : 0u);
        const char *colP = s_tab + offP, *colQ = s_tab + offQ;
        const uint32_t hc = pack2(j < LtP ? indel : 0, j < LtQ ? indel : 0);
        uint32_t diag = top;
        top = __vadd2(top, hc);
        uint32_t up = top;
#pragma unroll
        for (int p = 0; p < NQ; ++p) {
            uint32_t sub;
            if (SPLIT) {
                const uint32_t lo = *reinterpret_cast<const uint32_t *>(s_tab + (qoffP[p] * unit + offP));
                const uint32_t hi = *reinterpret_cast<const uint32_t *>(s_tab + (qoffQ[p] * unit + offQ));
                sub = hi * unit + lo;
            } else {
                const uint32_t lo = *reinterpret_cast<const uint32_t *>(colP + qoffP[p]);
                const uint32_t hi = *reinterpret_cast<const uint32_t *>(colQ + qoffQ[p]);
                sub = (lo & 0x0000ffffu) | (hi & 0xffff0000u);
            }
            const uint32_t t = __vadd2(diag, sub);
            const uint32_t mleft = __viaddmin_s16x2(D[p], hc, t);
            const uint32_t d = __viaddmin_s16x2(up, vc[p], mleft);
            diag = D[p];
            D[p] = d;
            up = d;
        }
    }
    return NQ > 0 ? D[NQ - 1] : top;
}

template <int WORDS, int CFG>
__global__ void __launch_bounds__(BinnedShape<CFG>::threads, BinnedShape<CFG>::blocks)
    edit_binned_kernel(const uint64_t *__restrict__ packed, const uint32_t *__restrict__ pairs,
                       const uint32_t *__restrict__ order, int64_t m_max, const unsigned long long *__restrict__ d_m,
                       const uint32_t *__restrict__ table, int indel, int32_t *__restrict__ out, uint32_t unit)
{
    extern __shared__ int32_t s_tab_words[];
    const int64_t m = items(m_max, d_m);
    constexpr bool kSplit = BinnedShape<CFG>::split;
    for (int q = threadIdx.x; q < kEdWords / 4; q += blockDim.x) {
        const uint4 v = reinterpret_cast<const uint4 *>(table)[q];  // cost in both halves
        if (kSplit) {
            reinterpret_cast<uint4 *>(s_tab_words)[q] =
                make_uint4(v.x & 0xffffu, v.y & 0xffffu, v.z & 0xffffu, v.w & 0xffffu);
            reinterpret_cast<uint4 *>(s_tab_words + kEdWords)[q] =
                make_uint4(v.x << 16, v.y << 16, v.z << 16, v.w << 16);
        } else {
            reinterpret_cast<uint4 *>(s_tab_words)[q] = v;
        }
    }
    __syncthreads();
    const char *s_tab = reinterpret_cast<const char *>(s_tab_words);
    constexpr int MAXLEN = WORDS == 2 ? 24 : 30;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t stride = nwarps * 64;
    // the record double buffer of the batched alignment kernel (see there)
    Rec<WORDS> *buf =
        reinterpret_cast<Rec<WORDS> *>(s_tab_words + BinnedShape<CFG>::tables * kEdWords) + threadIdx.x * 8;
    auto issue = [&](int slot, uint4 idP, uint4 idQ) {
        Rec<WORDS> *dst = buf + slot * 4;
        if (idP.w) {
#pragma unroll
            for (int c = 0; c < WORDS / 2; ++c) {
                cp_async16(reinterpret_cast<char *>(dst + 0) + 16 * c, packed + (int64_t)idP.x * WORDS + 2 * c);
                cp_async16(reinterpret_cast<char *>(dst + 1) + 16 * c, packed + (int64_t)idP.y * WORDS + 2 * c);
            }
        }
        if (idQ.w) {
#pragma unroll
            for (int c = 0; c < WORDS / 2; ++c) {
                cp_async16(reinterpret_cast<char *>(dst + 2) + 16 * c, packed + (int64_t)idQ.x * WORDS + 2 * c);
                cp_async16(reinterpret_cast<char *>(dst + 3) + 16 * c, packed + (int64_t)idQ.y * WORDS + 2 * c);
            }
        }
        cp_async_commit();
    };
    int64_t base = warp * 64;
    uint4 curP = entry_ids<false>(order, pairs, base + lane, m), curQ = entry_ids<false>(order, pairs, base + 32 + lane, m);
    issue(0, curP, curQ);
    uint4 nxtP = entry_ids<false>(order, pairs, base + stride + lane, m);
    uint4 nxtQ = entry_ids<false>(order, pairs, base + stride + 32 + lane, m);
    for (int k = 0; base < m; ++k, base += stride) {
        issue((k + 1) & 1, nxtP, nxtQ);
        const uint4 farP = entry_ids<false>(order, pairs, base + 2 * stride + lane, m);
        const uint4 farQ = entry_ids<false>(order, pairs, base + 2 * stride + 32 + lane, m);
        cp_async_wait1();
        const bool vP = curP.w != 0, vQ = curQ.w != 0;
        const Rec<WORDS> *r = buf + (k & 1) * 4;
        Rec<WORDS> AP, BP, AQ, BQ;
        int LaP = 0, LbP = 0, LaQ = 0, LbQ = 0;
        if (vP) {
            AP = r[0];
            BP = r[1];
            orient<WORDS>(AP, LaP, BP, LbP, true);
        } else {
#pragma unroll
            for (int w = 0; w < WORDS; ++w) AP.w[w] = BP.w[w] = 0;
        }
        if (vQ) {
            AQ = r[2];
            BQ = r[3];
            orient<WORDS>(AQ, LaQ, BQ, LbQ, true);
        } else {
            AQ = AP;
            BQ = BP;
            LaQ = LaP;
            LbQ = LbP;
        }
        const int wmax = __reduce_max_sync(0xffffffffu, max(LaP, LaQ));
        if (vP) {
            uint32_t dist;
            switch ((wmax + 1) >> 1) {
#define SQ_ED(H)                                                                                                   \
    case H:                                                                                                        \
        dist = ed_pair2<WORDS, (H < 1 ? 2 : (2 * H <= MAXLEN ? 2 * H : MAXLEN)), kSplit>(                          \
            AP, LaP, BP, LbP, AQ, LaQ, BQ, LbQ, s_tab, lane, indel, unit);                                         \
        break;
                SQ_ED(0) SQ_ED(1) SQ_ED(2) SQ_ED(3) SQ_ED(4) SQ_ED(5) SQ_ED(6) SQ_ED(7) SQ_ED(8) SQ_ED(9) SQ_ED(10)
                SQ_ED(11) SQ_ED(12)
#undef SQ_ED
            default:
                dist = ed_pair2<WORDS, MAXLEN, kSplit>(AP, LaP, BP, LbP, AQ, LaQ, BQ, LbQ, s_tab, lane, indel, unit);
                break;
            }
            out[curP.z] = (int32_t)(dist & 0xffffu);
            if (vQ) out[curQ.z] = (int32_t)(dist >> 16);
        }
        curP = nxtP;
        curQ = nxtQ;
        nxtP = farP;
        nxtQ = farQ;
    }
}

int launch_edit(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs, int64_t m,
                int32_t *out, const unsigned long long *d_m)
{
    SQ_TRY(ensure_edit_table(ctx));
    uint32_t *order = nullptr;
    SQ_TRY(build_work_list<false>(ctx, packed, pack_stride, pairs, m, d_m, true, &order));
    const uint64_t *pk = static_cast<const uint64_t *>(packed);
    SqProfScope prof(ctx, SUBQUAD_PROF_EDIT);
#define SQ_EDL(W, C)                                                                                               \
    do {                                                                                                           \
        auto k = edit_binned_kernel<W, C>;                                                                         \
        const size_t smem = sizeof(uint32_t) * kEdWords * BinnedShape<C>::tables +                                \
                            sizeof(uint64_t) * W * 8 * BinnedShape<C>::threads;                                    \
        SQ_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));             \
        const unsigned grid = sq_grid(ctx, (m + 1) / 2, BinnedShape<C>::threads, BinnedShape<C>::blocks);         \
        k<<<grid, BinnedShape<C>::threads, smem, ctx->stream>>>(pk, pairs, order, m, d_m, ctx->d_edit_table,       \
                                                               ctx->edit_indel, out, 1u);                         \
    } while (0)
    const int cfg = ctx->tune[SUBQUAD_TUNE_ALIGN_SHAPE];
    if (pack_stride == 16) {
        if (cfg == 0) SQ_EDL(2, 0);
        else if (cfg == 1) SQ_EDL(2, 1);
        else SQ_EDL(2, 2);
    } else {
        if (cfg == 0) SQ_EDL(4, 0);
        else if (cfg == 1) SQ_EDL(4, 1);
        else SQ_EDL(4, 2);
    }
#undef SQ_EDL
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

}  // namespace

extern "C" int subquad_edit_distance(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs,
                                     int64_t m, int32_t *dist_out)
{
    SQ_ENTER(ctx);
    if (m < 0 || (pack_stride != 16 && pack_stride != 32)) return SUBQUAD_ERR_ARG;
    if (m == 0) return SUBQUAD_OK;
    if (!packed || !pairs || !dist_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8) return SUBQUAD_ERR_ARG;
    return launch_edit(ctx, packed, pack_stride, pairs, m, dist_out, nullptr);
}

extern "C" int subquad_edit_distance_async(subquad_ctx *ctx, const void *packed, int pack_stride,
                                           const uint32_t *pairs, const uint64_t *d_m, int64_t m_max,
                                           int32_t *dist_out)
{
    SQ_ENTER(ctx);
    if (!d_m || m_max < 0 || (pack_stride != 16 && pack_stride != 32)) return SUBQUAD_ERR_ARG;
    if (m_max == 0) return SUBQUAD_OK;
    if (!packed || !pairs || !dist_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8) return SUBQUAD_ERR_ARG;
    return launch_edit(ctx, packed, pack_stride, pairs, m_max, dist_out, reinterpret_cast<const unsigned long long *>(d_m));
}
