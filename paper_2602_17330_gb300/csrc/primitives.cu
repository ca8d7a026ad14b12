// Device-wide scan (banding, binning) and stable LSD radix sort (pair index of
// the gate training).
//
// Scan: reduce-then-scan over at most eight chunks per SM, each chunk scanned
// in tiles of 4096 elements (256 threads x 16).  Radix sort: 8-bit digits; per pass
// a digit histogram per tile (warp-aggregated shared-memory counts), a scan of
// the digit-major histogram, and a stable scatter in which each warp ranks its
// 256 elements round by round with __match_any_sync so equal digits keep their
// input order.
#include <algorithm>

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

// A tile's loads, all issued before any is used: element base + q * 256 + t
// of thread t (zero at or past count).
template <typename T>
__device__ __forceinline__ void fetch_tile(const T *in, int64_t base, int64_t count, T v[kScanItems])
{
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t g = base + q * kScanThreads + threadIdx.x;
        v[q] = g < count ? in[g] : T(0);
    }
}

// Fetched (strided) elements to the blocked order: thread t's items are
// elements t * 16 .. t * 16 + 15 of the tile.
template <typename T>
__device__ __forceinline__ void stage_tile(const T v[kScanItems], T *s_buf, T items[kScanItems])
{
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) s_buf[pad(q * kScanThreads + threadIdx.x)] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) items[q] = s_buf[pad(threadIdx.x * kScanItems + q)];
    __syncthreads();
}

// Reduce-then-scan over G contiguous chunks (whole tiles of kScanTile
// elements; G at most kScanChunksPerSm per SM, so that small inputs still
// spread over many CTAs): one kernel reduces every chunk, a second one gives
// each chunk its prefix (the reduction of the chunk totals before it) and
// scans the chunk tile by tile with a running carry.  Two passes over the
// input, one over the output, and no waiting between CTAs.  Both kernels
// issue a whole tile's loads (16 per thread) before using any of them: the
// scans are small and latency-bound.
constexpr int kScanChunksPerSm = 8;
template <typename T, bool MAX>
__device__ __forceinline__ T block_reduce(T v, T *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = op<T, MAX>(v, __shfl_xor_sync(0xffffffffu, v, d));
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    T r = T(0);
    for (int w = 0; w < nw; ++w) r = op<T, MAX>(r, s_warp[w]);
    __syncthreads();
    return r;
}

// Chunk [lo, hi) of chunk b: chunks are whole tiles, the last one ragged.
__device__ __forceinline__ void scan_chunk(int64_t count, int64_t b, int64_t G, int64_t &lo, int64_t &hi)
{
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    const int64_t per = (tiles + G - 1) / G;
    lo = min(count, b * per * kScanTile);
    hi = min(count, lo + per * kScanTile);
}

template <typename T, bool MAX>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const T *__restrict__ in, int64_t count_max,
                                                                   const uint32_t *__restrict__ d_count,
                                                                   T *__restrict__ partial)
{
    __shared__ T s_warp[32];
    const int64_t count = eff_count(count_max, d_count);
    int64_t lo, hi;
    scan_chunk(count, blockIdx.x, gridDim.x, lo, hi);
    T acc = T(0);
    for (int64_t base = lo; base < hi; base += kScanTile) {
        T v[kScanItems];
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            const int64_t g = base + q * kScanThreads + threadIdx.x;
            v[q] = g < hi ? in[g] : T(0);
        }
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) acc = op<T, MAX>(acc, v[q]);
    }
    const T r = block_reduce<T, MAX>(acc, s_warp);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

template <typename T, bool MAX>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const T *__restrict__ in, T *__restrict__ out,
                                                                  int64_t count_max,
                                                                  const uint32_t *__restrict__ d_count,
                                                                  bool inclusive, const T *__restrict__ partial,
                                                                  T *total_out)
{
    __shared__ T s_buf[kScanTilePadded];
    __shared__ T s_warp[32];
    const int64_t count = eff_count(count_max, d_count);
    int64_t lo, hi;
    scan_chunk(count, blockIdx.x, gridDim.x, lo, hi);
    // the first tile's loads in flight while the prefix of this chunk (the
    // chunk totals before it) is summed; each later tile's while the tile
    // before it is scanned
    T v[kScanItems];
    fetch_tile(in, lo, hi, v);
    T pre = T(0);
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += kScanThreads) pre = op<T, MAX>(pre, partial[k]);
    T carry = block_reduce<T, MAX>(pre, s_warp);
    for (int64_t base = lo; base < hi; base += kScanTile) {
        T items[kScanItems];
        stage_tile(v, s_buf, items);
        if (base + kScanTile < hi) fetch_tile(in, base + kScanTile, hi, v);
        T acc = items[0];
#pragma unroll
        for (int q = 1; q < kScanItems; ++q) acc = op<T, MAX>(acc, items[q]);
        T total;
        const T excl = block_exclusive<T, MAX>(acc, &total);
        T run = op<T, MAX>(carry, excl);
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            const T next = op<T, MAX>(run, items[q]);
            s_buf[pad(threadIdx.x * kScanItems + q)] = inclusive ? next : run;
            run = next;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kScanTile; q += kScanThreads) {
            const int64_t g = base + q;
            if (g < hi) out[g] = s_buf[pad(q)];
        }
        __syncthreads();
        carry = op<T, MAX>(carry, total);
    }
    if (total_out && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *total_out = carry;
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
    const int64_t G = std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * kScanChunksPerSm);
    if ((size_t)G * sizeof(T) > tmp_bytes) return SUBQUAD_ERR_ARG;
    T *partial = static_cast<T *>(tmp);
    scan_reduce_kernel<T, MAX><<<(unsigned)G, kScanThreads, 0, ctx->stream>>>(in, count, d_count, partial);
    SQ_LAUNCH_CHECK();
    scan_apply_kernel<T, MAX><<<(unsigned)G, kScanThreads, 0, ctx->stream>>>(in, out, count, d_count, inclusive,
                                                                            partial, total_out);
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
