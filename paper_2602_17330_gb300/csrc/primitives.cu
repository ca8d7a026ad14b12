// Device-wide scan (banding, binning) and stable LSD radix sort (pair index of
// the gate training).
//
// Scan: one pass over tiles of 4096 elements (256 threads x 16) with
// decoupled look-back between tiles.  Radix sort: 8-bit digits; per pass
// a digit histogram per tile (warp-aggregated shared-memory counts), a scan of
// the digit-major histogram, and a stable scatter in which each warp ranks its
// 256 elements round by round with __match_any_sync so equal digits keep their
// input order.
#include "internal.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
// one padding word per 32 keeps blocked (thread-major) accesses conflict-free
__device__ __forceinline__ int pad(int q) { return q + (q >> 5); }
constexpr int kScanTilePadded = kScanTile + kScanTile / 32;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;

// Element count of a launch sized for count_max: the device-side count when one
// is given (the producer of the data wrote it), else count_max.
__device__ __forceinline__ int64_t eff_count(int64_t count_max, const uint32_t *d_count)
{
    if (!d_count) return count_max;
    int64_t c = (int64_t)*d_count;
    return c < count_max ? c : count_max;
}

template <typename T, bool MAX>
__device__ __forceinline__ T op(T a, T b)
{
    return MAX ? (a > b ? a : b) : a + b;
}

template <typename T, bool MAX>
__device__ __forceinline__ T warp_inclusive(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v = op<T, MAX>(v, o);
    }
    return v;
}

// Exclusive scan of one value per thread across the block; returns the block
// total through *total.
template <typename T, bool MAX>
__device__ __forceinline__ T block_exclusive(T v, T *total)
{
    __shared__ T s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_inclusive<T, MAX>(v);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? s_warp[lane] : T(0);
        T wi = warp_inclusive<T, MAX>(w);
        if (lane < nw) s_warp[lane] = wi;  // inclusive per warp
    }
    __syncthreads();
    T warp_prefix = warp > 0 ? s_warp[warp - 1] : T(0);
    *total = s_warp[nw - 1];
    T exc_in_warp = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc_in_warp = T(0);
    T res = op<T, MAX>(warp_prefix, exc_in_warp);
    __syncthreads();
    return res;
}

template <typename T>
__device__ __forceinline__ void load_tile(const T *in, int64_t base, int64_t count, T *s_buf, T items[kScanItems])
{
    for (int q = threadIdx.x; q < kScanTile; q += kScanThreads) {
        int64_t g = base + q;
        s_buf[pad(q)] = g < count ? in[g] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) items[q] = s_buf[pad(threadIdx.x * kScanItems + q)];
    __syncthreads();
}

// Single-pass scan with decoupled look-back: each CTA takes the next tile
// index from a counter (so every lower tile belongs to a CTA already
// running), publishes its tile total, then warp 0 reads the status words of
// the 32 preceding tiles at a time: a tile that has published its inclusive
// prefix ends the walk, tiles with only a total are added and the window
// moves back.  Status word: flag in bits 62..63, value below (values and
// totals stay under 2^62).  Spins on an unpublished tile are bounded;
// running out sets the TIMEOUT error bit instead of waiting forever.
constexpr unsigned long long kScanFlagAgg = 1ull << 62;
constexpr unsigned long long kScanFlagPre = 2ull << 62;
constexpr unsigned long long kScanValue = (1ull << 62) - 1ull;
constexpr long long kScanSpinLimit = 1ll << 22;

template <typename T, bool MAX>
__device__ __forceinline__ T warp_reduce(T v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = op<T, MAX>(v, __shfl_xor_sync(0xffffffffu, v, d));
    return v;
}

template <typename T, bool MAX>
__global__ void __launch_bounds__(kScanThreads) scan_onepass_kernel(const T *__restrict__ in, T *__restrict__ out,
                                                                    int64_t count_max,
                                                                    const uint32_t *__restrict__ d_count,
                                                                    bool inclusive, unsigned long long *status,
                                                                    uint32_t *tile_counter, T *total_out,
                                                                    uint32_t *err)
{
    __shared__ T s_buf[kScanTilePadded];
    __shared__ uint32_t s_tile;
    __shared__ T s_prefix;
    const int64_t count = eff_count(count_max, d_count);
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    const int64_t base = t * kScanTile;
    if (base >= count) {
        if (t == 0 && threadIdx.x == 0 && total_out) *total_out = T(0);  // empty input
        return;
    }
    T items[kScanItems];
    load_tile(in, base, count, s_buf, items);
    T acc = items[0];
#pragma unroll
    for (int q = 1; q < kScanItems; ++q) acc = op<T, MAX>(acc, items[q]);
    T total;
    const T excl = block_exclusive<T, MAX>(acc, &total);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        T prefix = T(0);
        if (t == 0) {
            if (lane == 0) atomicExch(&status[0], kScanFlagPre | (unsigned long long)total);
        } else {
            if (lane == 0) atomicExch(&status[t], kScanFlagAgg | (unsigned long long)total);
            T run = T(0);
            int64_t j = t - 1;
            long long spins = 0;
            for (;;) {
                const int64_t idx = j - lane;
                unsigned long long v = kScanFlagPre;
                if (idx >= 0) v = *(volatile unsigned long long *)&status[idx];
                while (__any_sync(0xffffffffu, (v >> 62) == 0)) {
                    if ((v >> 62) == 0) v = *(volatile unsigned long long *)&status[idx];
                    if (++spins > kScanSpinLimit) {
                        if (lane == 0) atomicOr(err, SQ_DEVERR_TIMEOUT);
                        v = kScanFlagPre;  // give up: the error bit is set
                    }
                }
                const uint32_t pmask = __ballot_sync(0xffffffffu, (v & kScanFlagPre) != 0);
                const T val = (T)(v & kScanValue);
                if (pmask) {
                    const int k = __ffs(pmask) - 1;  // nearest tile with its inclusive prefix
                    run = op<T, MAX>(run, warp_reduce<T, MAX>(lane <= k ? val : T(0)));
                    break;
                }
                run = op<T, MAX>(run, warp_reduce<T, MAX>(val));
                j -= 32;
            }
            prefix = run;
            if (lane == 0) atomicExch(&status[t], kScanFlagPre | (unsigned long long)op<T, MAX>(prefix, total));
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (total_out && base + kScanTile >= count) *total_out = op<T, MAX>(prefix, total);
        }
    }
    __syncthreads();
    T run = op<T, MAX>(s_prefix, excl);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const T next = op<T, MAX>(run, items[q]);
        s_buf[pad(threadIdx.x * kScanItems + q)] = inclusive ? next : run;
        run = next;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kScanTile; q += kScanThreads) {
        const int64_t g = base + q;
        if (g < count) out[g] = s_buf[pad(q)];
    }
}

template <typename T, bool MAX>
int scan_impl(subquad_ctx *ctx, const T *in, T *out, int64_t count, const uint32_t *d_count, bool inclusive,
              T *total_out, void *tmp, size_t tmp_bytes)
{
    if (count <= 0) {
        if (total_out) SQ_TRY_CUDA(cudaMemsetAsync(total_out, 0, sizeof(T), ctx->stream));
        return SUBQUAD_OK;
    }
    const int64_t ntiles = (count + kScanTile - 1) / kScanTile;
    const size_t need = (size_t)(ntiles + 1) * sizeof(unsigned long long);
    if (need > tmp_bytes) return SUBQUAD_ERR_ARG;
    unsigned long long *status = static_cast<unsigned long long *>(tmp);
    uint32_t *counter = reinterpret_cast<uint32_t *>(status + ntiles);
    SQ_TRY_CUDA(cudaMemsetAsync(tmp, 0, need, ctx->stream));
    scan_onepass_kernel<T, MAX><<<(unsigned)ntiles, kScanThreads, 0, ctx->stream>>>(
        in, out, count, d_count, inclusive, status, counter, total_out, ctx->d_err);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift)
{
    return (uint32_t)(key >> shift) & (kRadix - 1);
}

// hist[d * ntiles + tile] = number of elements of the tile with digit d
template <typename K>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const K *__restrict__ keys, int64_t count_max,
                                                                  const uint32_t *__restrict__ d_count, int shift,
                                                                  uint32_t *__restrict__ hist, int64_t ntiles)
{
    __shared__ uint32_t s_hist[kRadix];
    const int64_t count = eff_count(count_max, d_count);
    if ((int64_t)blockIdx.x * kSortTile >= count) {
        for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = 0;
        return;
    }
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) s_hist[d] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)blockIdx.x * kSortTile + warp * 32 * kSortItems;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t g = wbase + r * 32 + lane;
        bool valid = g < count;
        uint32_t d = valid ? digit_of(keys[g], shift) : 0xffffu;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = s_hist[d];
}

template <typename K, bool HAS_VAL>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const K *__restrict__ keys_in,
                                                                     const uint32_t *__restrict__ vals_in,
                                                                     K *__restrict__ keys_out,
                                                                     uint32_t *__restrict__ vals_out, int64_t count_max,
                                                                     const uint32_t *__restrict__ d_count, int shift,
                                                                     const uint32_t *__restrict__ offsets,
                                                                     int64_t ntiles)
{
    __shared__ uint32_t s_wcnt[kSortThreads / 32][kRadix];
    __shared__ uint32_t s_gofs[kRadix];
    const int64_t count = eff_count(count_max, d_count);
    if ((int64_t)blockIdx.x * kSortTile >= count) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < (kSortThreads / 32) * kRadix; q += blockDim.x) (&s_wcnt[0][0])[q] = 0;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) s_gofs[d] = offsets[(int64_t)d * ntiles + blockIdx.x];
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * kSortTile + warp * 32 * kSortItems;
    const uint32_t lt_mask = (1u << lane) - 1u;
    K key[kSortItems];
    uint32_t val[kSortItems], dig[kSortItems], rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t g = wbase + r * 32 + lane;
        bool valid = g < count;
        key[r] = valid ? keys_in[g] : K(0);
        val[r] = (HAS_VAL && valid) ? vals_in[g] : 0u;
        dig[r] = valid ? digit_of(key[r], shift) : 0xffffu;
        uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
        uint32_t before = __popc(peers & lt_mask);
        uint32_t base = valid ? s_wcnt[warp][dig[r]] : 0u;
        rank[r] = base + before;
        __syncwarp();
        if (valid && before == 0) s_wcnt[warp][dig[r]] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps (warp order = input order)
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            uint32_t c = s_wcnt[w][d];
            s_wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (dig[r] < (uint32_t)kRadix) {
            uint32_t pos = s_gofs[dig[r]] + s_wcnt[warp][dig[r]] + rank[r];
            keys_out[pos] = key[r];
            if (HAS_VAL) vals_out[pos] = val[r];
        }
    }
}

template <typename K, bool HAS_VAL>
int radix_impl(subquad_ctx *ctx, K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, int64_t count,
               const uint32_t *d_count, int begin_bit, int end_bit, bool *result_in_alt, void *tmp, size_t tmp_bytes)
{
    *result_in_alt = false;
    if (count <= 1 || end_bit <= begin_bit) return SUBQUAD_OK;
    if (count >= (int64_t(1) << 32)) return SUBQUAD_ERR_ARG;
    const int64_t ntiles = (count + kSortTile - 1) / kSortTile;
    const int64_t hist_len = ntiles * kRadix;
    const size_t scan_bytes = sq_scan_tmp_bytes(hist_len);
    size_t need = (size_t)hist_len * sizeof(uint32_t) * 2 + scan_bytes + 1024;
    if (need > tmp_bytes) return SUBQUAD_ERR_ARG;
    SqArena arena(tmp);
    uint32_t *hist = arena.take<uint32_t>(hist_len);
    uint32_t *offs = arena.take<uint32_t>(hist_len);
    char *scan_tmp = arena.take<char>(scan_bytes);
    K *src_k = keys, *dst_k = keys_alt;
    uint32_t *src_v = vals, *dst_v = vals_alt;
    bool in_alt = false;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        radix_hist_kernel<K><<<(unsigned)ntiles, kSortThreads, 0, ctx->stream>>>(src_k, count, d_count, shift, hist,
                                                                                ntiles);
        SQ_LAUNCH_CHECK();
        SQ_TRY((scan_impl<uint32_t, false>(ctx, hist, offs, hist_len, nullptr, false, nullptr, scan_tmp,
                                           scan_bytes)));
        radix_scatter_kernel<K, HAS_VAL><<<(unsigned)ntiles, kSortThreads, 0, ctx->stream>>>(
            src_k, src_v, dst_k, dst_v, count, d_count, shift, offs, ntiles);
        SQ_LAUNCH_CHECK();
        K *tk = src_k;
        src_k = dst_k;
        dst_k = tk;
        uint32_t *tv = src_v;
        src_v = dst_v;
        dst_v = tv;
        in_alt = !in_alt;
    }
    *result_in_alt = in_alt;
    return SUBQUAD_OK;
}

}  // namespace

size_t sq_scan_tmp_bytes(int64_t count)
{
    return (size_t)((count + kScanTile - 1) / kScanTile + 2) * sizeof(uint64_t) + 256;
}

size_t sq_radix_tmp_bytes(int64_t count)
{
    int64_t ntiles = (count + kSortTile - 1) / kSortTile;
    int64_t hist_len = ntiles * kRadix;
    return (size_t)hist_len * sizeof(uint32_t) * 2 + sq_scan_tmp_bytes(hist_len) + 4096;
}

int sq_scan_u32(subquad_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t count, const uint32_t *d_count,
                bool inclusive, bool max_op, uint32_t *total_out, void *tmp, size_t tmp_bytes)
{
    if (max_op) return scan_impl<uint32_t, true>(ctx, in, out, count, d_count, inclusive, total_out, tmp, tmp_bytes);
    return scan_impl<uint32_t, false>(ctx, in, out, count, d_count, inclusive, total_out, tmp, tmp_bytes);
}

int sq_scan_u64(subquad_ctx *ctx, const uint64_t *in, uint64_t *out, int64_t count, const uint32_t *d_count,
                uint64_t *total_out, void *tmp, size_t tmp_bytes)
{
    return scan_impl<uint64_t, false>(ctx, in, out, count, d_count, false, total_out, tmp, tmp_bytes);
}

int sq_radix_sort_u32(subquad_ctx *ctx, uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      int64_t count, const uint32_t *d_count, int begin_bit, int end_bit, bool *result_in_alt,
                      void *tmp, size_t tmp_bytes)
{
    if (vals)
        return radix_impl<uint32_t, true>(ctx, keys, vals, keys_alt, vals_alt, count, d_count, begin_bit, end_bit,
                                          result_in_alt, tmp, tmp_bytes);
    return radix_impl<uint32_t, false>(ctx, keys, nullptr, keys_alt, nullptr, count, d_count, begin_bit, end_bit,
                                       result_in_alt, tmp, tmp_bytes);
}
