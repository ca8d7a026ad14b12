// (a2) LSH banding, candidate emission and deduplication (Algorithm 1,
// preprocessing: "build MinHash index; generate candidate list CAND").
//
// Bands are inserted in groups whose hash tables fit a share of L2:
//  1. insert every (band, sequence) key -- the exact R-tuple -- into a
//     per-band open-addressing table whose slots hold the id of the first
//     inserter; equal keys meet at one slot, so the slot index is an exact
//     bucket id; count the members of every bucket;
//  2. keep only members of buckets with >= 2 members (on the 1M-sequence
//     donor about 10% of the keys) and radix-sort them by (bucket, id): each
//     bucket becomes one contiguous run with its members in ascending id order
//     (the contiguous bucket blocks of the paper's index);
//  3. run starts by a max-scan of head positions; rank in bucket = position -
//     run start; chunk = rank / cap; every kept element records, per band, the
//     sorted position of its chunk head (its chunk id G[i][b]; singletons keep
//     a sentinel that matches nothing);
//  4. chunks with >= 2 members are compacted and their pair counts scanned;
//  5. each warp takes 32 consecutive pair indices, finds their chunks, decodes
//     (u, v) and keeps pair (i, j) only if no earlier band already puts i and j
//     in one chunk (first-band ownership), so every pair of C is emitted once;
//  6. after all groups: read back |C| (the call's only host synchronisation),
//     then radix-sort the pairs into lexicographic order.
// Element counts produced on the device (kept keys, chunks, raw pairs) are
// consumed on the device: the kernels after them are sized for the upper
// bound and read the actual count.
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr uint32_t kEmpty = 0xffffffffu;
constexpr uint32_t kNoChunk = 0xffffffffu;  // chunk id of a singleton (matches nothing)

__device__ __forceinline__ uint32_t mix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ void load_key(const uint32_t *__restrict__ p, int rows, uint32_t k[8])
{
    if (rows == 4) {
        uint4 v = *reinterpret_cast<const uint4 *>(p);
        k[0] = v.x;
        k[1] = v.y;
        k[2] = v.z;
        k[3] = v.w;
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (r < rows) k[r] = p[r];
    }
}

__device__ __forceinline__ bool key_equal(const uint32_t *__restrict__ p, int rows, const uint32_t k[8])
{
    uint32_t o[8];
    load_key(p, rows, o);
    bool eq = true;
#pragma unroll
    for (int r = 0; r < 8; ++r)
        if (r < rows) eq = eq && o[r] == k[r];
    return eq;
}

// Block-wide exclusive position of each flagged thread in an append buffer:
// one global atomic per block instead of one per warp, so a single hot counter
// is touched 8x less often.
__device__ __forceinline__ unsigned long long block_append(bool flag, unsigned long long *counter,
                                                           unsigned long long *s_base, uint32_t *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t mask = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) s_warp[warp] = __popc(mask);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < nw; ++w) {
            const uint32_t c = s_warp[w];
            s_warp[w] = run;
            run += c;
        }
        *s_base = run ? atomicAdd(counter, (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    const unsigned long long pos = *s_base + s_warp[warp] + __popc(mask & ((1u << lane) - 1u));
    __syncthreads();
    return pos;
}

// Step 1: exact bucket id (= table slot) per (band, sequence).  A slot holds
// the id of its first inserter (whose key it stands for) in bits 0..30; bit 31
// is set, by a plain store, as soon as a second member arrives.  Only the
// first member of a bucket uses an atomic (the claiming CAS), so a bucket of
// hundreds of members adds no contended atomics.  blockIdx.y = band in group.
constexpr uint32_t kShared = 0x80000000u;

constexpr int kInsIlp = 4;  // elements per thread in the singleton filter

__device__ __forceinline__ uint32_t key_hash(const uint32_t k[8], int rows)
{
    uint32_t h = 0x9e3779b9u ^ (uint32_t)rows;
#pragma unroll
    for (int r = 0; r < 8; ++r)
        if (r < rows) h = mix32(h ^ k[r]);
    return h;
}

// Probe from `slot` until the element's key is claimed or found (the slow path
// after a first probe that hit another key).
// Equal keys: the same R-tuple and, in a batch of donors, the same donor.
__device__ __forceinline__ bool same_key(const uint32_t *band_sig, int rows, uint32_t owner, const uint32_t k[8],
                                         const int32_t *donor, int32_t my_donor)
{
    return key_equal(band_sig + (int64_t)owner * rows, rows, k) && (!donor || donor[owner] == my_donor);
}

__device__ __forceinline__ uint32_t probe_from(uint32_t *tab, uint32_t slot, uint32_t smask, const uint32_t k[8],
                                               uint32_t i, const uint32_t *band_sig, int rows, const int32_t *donor,
                                               int32_t my_donor, uint32_t *err)
{
    for (uint32_t probe = 0; probe <= smask; ++probe) {
        uint32_t cur = tab[slot];
        if (cur == kEmpty) {
            cur = atomicCAS(&tab[slot], kEmpty, i);
            if (cur == kEmpty) return slot;
        }
        if (same_key(band_sig, rows, cur & ~kShared, k, donor, my_donor)) {
            if (!(cur & kShared)) tab[slot] = cur | kShared;
            return slot;
        }
        slot = (slot + 1) & smask;
    }
    atomicOr(err, SQ_DEVERR_TIMEOUT);  // unreachable: the table is at most half full
    return 0;
}

__global__ void __launch_bounds__(256) band_insert_kernel(const uint32_t *__restrict__ sig, int64_t n, int rows,
                                                          int band0, int log_s, const int32_t *__restrict__ donor,
                                                          uint32_t *__restrict__ table, uint32_t *__restrict__ slot_of,
                                                          uint32_t *err)
{
    const int gb = blockIdx.y;
    const uint32_t smask = (1u << log_s) - 1u;
    const uint32_t *band_sig = sig + (int64_t)(band0 + gb) * n * rows;
    uint32_t *tab = table + ((int64_t)gb << log_s);
    uint32_t *slots = slot_of + (int64_t)gb * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t k[8];
        load_key(band_sig + i * rows, rows, k);
        const int32_t dn = donor ? donor[i] : 0;
        const uint32_t home = mix32(key_hash(k, rows) ^ (uint32_t)dn) & smask;
        slots[i] = probe_from(tab, home, smask, k, (uint32_t)i, band_sig, rows, donor, dn, err);
    }
}

// Step 1b: keep the members of buckets with >= 2 members (singletons can form
// no pair), as keys ((band << log_s | slot) << nbits) | id, appended in any
// order -- the sort that follows orders them by band, bucket, then id.  A
// member is kept if its bucket's slot is flagged shared.
__global__ void __launch_bounds__(256) band_filter_kernel(const uint32_t *__restrict__ slot_of,
                                                          const uint32_t *__restrict__ table, int64_t n, int band0,
                                                          int log_s, int nbits, uint64_t *__restrict__ keys,
                                                          unsigned long long *__restrict__ d_kept)
{
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_warp[32];
    const int gb = blockIdx.y;
    const uint32_t *tab = table + ((int64_t)gb << log_s);
    const uint32_t *slots = slot_of + (int64_t)gb * n;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * kInsIlp;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kInsIlp + threadIdx.x;
         base - threadIdx.x < n; base += step) {
        uint32_t slot[kInsIlp];
        bool keep[kInsIlp];
#pragma unroll
        for (int q = 0; q < kInsIlp; ++q) {
            const int64_t i = base + (int64_t)q * blockDim.x;
            slot[q] = i < n ? slots[i] : 0u;
        }
#pragma unroll
        for (int q = 0; q < kInsIlp; ++q) {
            const int64_t i = base + (int64_t)q * blockDim.x;
            keep[q] = i < n && (tab[slot[q]] & kShared) != 0u;
        }
#pragma unroll
        for (int q = 0; q < kInsIlp; ++q) {
            const int64_t i = base + (int64_t)q * blockDim.x;
            const unsigned long long pos = block_append(keep[q], d_kept, &s_base, s_warp);
            if (keep[q]) keys[pos] = ((((uint64_t)(band0 + gb) << log_s) | slot[q]) << nbits) | (uint64_t)i;
        }
    }
}

__device__ __forceinline__ int64_t dev_count(int64_t count_max, const uint32_t *d_count)
{
    const int64_t c = (int64_t)*d_count;
    return c < count_max ? c : count_max;
}

// Step 3a: head positions of runs of equal buckets (0 elsewhere), for a max-scan.
__global__ void band_heads_kernel(const uint64_t *__restrict__ keys, int nbits, int64_t count_max,
                                  const uint32_t *__restrict__ d_count, uint32_t *__restrict__ head_pos)
{
    const int64_t count = dev_count(count_max, d_count);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        head_pos[e] = (e == 0 || (keys[e] >> nbits) != (keys[e - 1] >> nbits)) ? (uint32_t)e : 0u;
}

struct ChunkInfo {
    uint32_t head;  // sorted position of the element's chunk head
    bool is_head, is_last;
};

__device__ __forceinline__ ChunkInfo chunk_info(const uint32_t *__restrict__ run_start, int64_t count, int64_t e,
                                                int cap)
{
    ChunkInfo c;
    const uint32_t rs = run_start[e];
    const uint32_t rank = (uint32_t)e - rs;
    c.head = cap > 0 ? rs + (rank / (uint32_t)cap) * (uint32_t)cap : rs;
    c.is_head = (uint32_t)e == c.head;
    c.is_last = e + 1 == count || run_start[e + 1] != rs || (cap > 0 && (rank + 1) % (uint32_t)cap == 0);
    return c;
}

// Step 3b: chunk ids per (sequence, band) and flags of chunks with >= 2 members.
__global__ void band_chunks_kernel(const uint64_t *__restrict__ keys, int nbits, const uint32_t *__restrict__ run_start,
                                   int64_t count_max, const uint32_t *__restrict__ d_count, int cap, int log_s,
                                   int band0, int bands, uint32_t *__restrict__ chunk_of, uint32_t *__restrict__ flags)
{
    const int64_t count = dev_count(count_max, d_count);
    const uint64_t idmask = (1ull << nbits) - 1ull;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        ChunkInfo c = chunk_info(run_start, count, e, cap);
        const uint64_t k = keys[e];
        const int b = (int)((k >> nbits) >> log_s);
        chunk_of[(int64_t)(k & idmask) * bands + b] = c.head;
        flags[e] = (c.is_head && !c.is_last) ? 1u : 0u;
    }
}

// Step 4: compacted chunk heads, sizes and pair counts.
__global__ void band_chunk_list_kernel(const uint32_t *__restrict__ run_start, const uint32_t *__restrict__ flags,
                                       const uint32_t *__restrict__ cidx, int64_t count_max,
                                       const uint32_t *__restrict__ d_count, int cap, uint32_t *__restrict__ heads,
                                       uint32_t *__restrict__ sizes, uint64_t *__restrict__ npairs)
{
    const int64_t count = dev_count(count_max, d_count);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        if (flags[e]) heads[cidx[e]] = (uint32_t)e;
        ChunkInfo c = chunk_info(run_start, count, e, cap);
        if (c.is_last && !c.is_head) {
            const uint32_t s = (uint32_t)e - c.head + 1;
            const uint32_t ci = cidx[c.head];
            sizes[ci] = s;
            npairs[ci] = (uint64_t)s * (s - 1) / 2;
        }
    }
}

// (u, v), u < v, of the t-th pair of a chunk of size s in row-major order.
__device__ __forceinline__ void decode_pair(uint64_t t, uint32_t s, uint32_t &u, uint32_t &v)
{
    // estimate u from the quadratic in float, then correct it exactly
    const uint64_t twos1 = 2 * (uint64_t)s - 1;
    const uint64_t d = twos1 * twos1 - 8 * t;  // > 0 for t < s(s-1)/2
    int64_t ue = (int64_t)(((float)twos1 - sqrtf((float)d)) * 0.5f);
    if (ue < 0) ue = 0;
    if (ue > (int64_t)s - 2) ue = (int64_t)s - 2;
    auto row_start = [s](int64_t uu) { return (uint64_t)uu * (2 * (uint64_t)s - uu - 1) / 2; };
    for (int it = 0; it < 64 && ue > 0 && row_start(ue) > t; ++it) --ue;
    for (int it = 0; it < 64 && ue + 1 <= (int64_t)s - 2 && row_start(ue + 1) <= t; ++it) ++ue;
    u = (uint32_t)ue;
    v = (uint32_t)(ue + 1 + (int64_t)(t - row_start(ue)));
}

// Step 5: owned pairs of this band group, appended to out.
__global__ void __launch_bounds__(256) band_emit_kernel(
    const uint64_t *__restrict__ keys, int nbits, const uint32_t *__restrict__ heads,
    const uint32_t *__restrict__ sizes, const uint64_t *__restrict__ poff, const uint32_t *__restrict__ d_nchunks,
    const uint64_t *__restrict__ d_total, int log_s, int band0, int bands, const uint32_t *__restrict__ chunk_of,
    uint32_t *__restrict__ out, int64_t capacity, unsigned long long *__restrict__ d_count, uint32_t *err)
{
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_warp[32];
    const uint32_t nc = *d_nchunks;
    const uint64_t total = *d_total;
    const int lane = threadIdx.x & 31;
    // block-uniform trip count (block_append synchronises the block)
    for (uint64_t b0 = (uint64_t)blockIdx.x * blockDim.x; b0 < total; b0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q0 = b0 + (threadIdx.x & ~31u);
        // chunk of q0: largest c with poff[c] <= q0 (every chunk has >= 1 pair)
        uint32_t c0 = 0;
        if (lane == 0 && q0 < total) {
            uint32_t lo = 0, hi = nc;
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (poff[mid] <= q0) lo = mid;
                else hi = mid;
            }
            c0 = lo;
        }
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        const uint64_t q = q0 + lane;
        bool owned = false;
        uint32_t i = 0, j = 0;
        if (q < total) {
            uint32_t lo = c0, hi = min(nc, c0 + (uint32_t)lane + 1);
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (poff[mid] <= q) lo = mid;
                else hi = mid;
            }
            const uint32_t h = heads[lo], s = sizes[lo];
            uint32_t u, v;
            decode_pair(q - poff[lo], s, u, v);
            if (u >= v || v >= s) {  // cannot happen for a consistent chunk list
                atomicOr(err, SQ_DEVERR_TIMEOUT);
                u = 0;
                v = 1;
            }
            const uint64_t idmask = (1ull << nbits) - 1ull;
            i = (uint32_t)(keys[h + u] & idmask);
            j = (uint32_t)(keys[h + v] & idmask);
            const int b = (int)((keys[h] >> nbits) >> log_s);
            owned = true;
            const uint32_t *gi = chunk_of + (int64_t)i * bands;
            const uint32_t *gj = chunk_of + (int64_t)j * bands;
            for (int bb = 0; bb < b; ++bb)
                if (gi[bb] == gj[bb] && gi[bb] != kNoChunk) {
                    owned = false;
                    break;
                }
        }
        const unsigned long long pos = block_append(owned, d_count, &s_base, s_warp);
        if (owned && pos < (unsigned long long)capacity) reinterpret_cast<uint2 *>(out)[pos] = make_uint2(i, j);
    }
}

// raw pair count of the group = offset of the last chunk + its pairs
__global__ void band_total_kernel(const uint64_t *__restrict__ poff, const uint32_t *__restrict__ sizes,
                                  const uint32_t *__restrict__ d_nchunks, uint64_t *__restrict__ d_total)
{
    const uint32_t nc = *d_nchunks;
    uint64_t total = 0;
    if (nc > 0) {
        const uint64_t s = sizes[nc - 1];
        total = poff[nc - 1] + s * (s - 1) / 2;
    }
    *d_total = total;
}

__device__ __forceinline__ int64_t count_or(int64_t m, const unsigned long long *d_m)
{
    if (!d_m) return m;
    const int64_t c = (int64_t)*d_m;
    return c < m ? c : m;
}

__global__ void pairs_to_keys_kernel(const uint32_t *__restrict__ pairs, int64_t m_max,
                                     const unsigned long long *__restrict__ d_m, int nbits, uint64_t *__restrict__ keys)
{
    const int64_t m = count_or(m_max, d_m);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        uint2 ij = reinterpret_cast<const uint2 *>(pairs)[p];
        keys[p] = ((uint64_t)ij.x << nbits) | ij.y;
    }
}

__global__ void keys_to_pairs_kernel(const uint64_t *__restrict__ keys, int64_t m_max,
                                     const unsigned long long *__restrict__ d_m, int nbits,
                                     uint32_t *__restrict__ pairs)
{
    const int64_t m = count_or(m_max, d_m);
    const uint64_t mask = (nbits >= 64) ? ~0ull : ((1ull << nbits) - 1ull);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[p];
        reinterpret_cast<uint2 *>(pairs)[p] = make_uint2((uint32_t)(k >> nbits), (uint32_t)(k & mask));
    }
}

// Async finish: publish |C|, flag an overflow, clamp the count used below.
__global__ void band_finish_kernel(const unsigned long long *__restrict__ d_count, int64_t capacity,
                                   unsigned long long *__restrict__ d_out, unsigned long long *__restrict__ d_clamped,
                                   uint32_t *err)
{
    const unsigned long long c = *d_count;
    if (d_out) *d_out = c;
    if (c > (unsigned long long)capacity) atomicOr(err, SQ_DEVERR_CAPACITY);
    *d_clamped = c < (unsigned long long)capacity ? c : (unsigned long long)capacity;
}

int bits_for(uint64_t v)  // number of bits needed to hold values 0..v
{
    int b = 1;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

}  // namespace

namespace {

// The banding stage.  Synchronous form (d_num_pairs == nullptr): reads back the
// kept-key count (to size the sort) and |C| (to size the final sort and check
// the capacity).  Asynchronous form: no host synchronisation at all -- the
// counts stay on the device, kernels are sized for their upper bounds and read
// the actual counts, |C| goes to *d_num_pairs and an overflow of the capacity
// sets the sticky CAPACITY error -- so the call can be captured in a graph once
// a call of the same shape has reserved the scratch.
int band_run(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows, int32_t bucket_cap,
             const int32_t *donor, uint32_t *pairs_out, int64_t pairs_capacity, int64_t *num_pairs_out,
             unsigned long long *d_num_pairs)
{
    const bool async = d_num_pairs != nullptr;
    const int cap = (bucket_cap <= 0 || bucket_cap >= n) ? 0 : bucket_cap;
    SqProfScope prof(ctx, SUBQUAD_PROF_BAND);

    // Table of S >= 2n 32-bit slots per band.  Bands are inserted in groups
    // whose tables fit a share of L2 (the random probes then stay on chip);
    // the kept keys of all bands are sorted and chunked together.
    const int log_s = bits_for((uint64_t)(2 * n - 1));
    const int64_t S = int64_t(1) << log_s;
    const int nbits = bits_for((uint64_t)(n - 1));
    const int key_bits = nbits + log_s + bits_for((uint64_t)(bands - 1));
    if (key_bits > 64) return SUBQUAD_ERR_ARG;
    const int64_t l2_budget = (int64_t)ctx->tune[SUBQUAD_TUNE_BAND_L2_MB] << 20;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(bands, l2_budget / (S * 4)));
    const int64_t mg = (int64_t)G * n;       // elements per insert group
    const int64_t mall = (int64_t)bands * n;  // upper bound of kept keys
    const int nb = bits_for((uint64_t)(n - 1));
    const int64_t final_cap = std::max<int64_t>(pairs_capacity, 1);

    auto layout = [&](SqArena &a) {
        struct L {
            uint32_t *chunk_of, *table, *slot_of, *run_start, *flags, *cidx, *heads, *sizes;
            uint64_t *k0, *k1, *npairs, *p0, *p1;
            void *tmp, *ptmp;
        } l;
        l.chunk_of = a.take<uint32_t>((size_t)n * bands);
        l.table = a.take<uint32_t>((size_t)G * S);
        l.slot_of = a.take<uint32_t>(mg);
        l.k0 = a.take<uint64_t>(mall);
        l.k1 = a.take<uint64_t>(mall);
        l.run_start = a.take<uint32_t>(mall);
        l.flags = a.take<uint32_t>(mall);
        l.cidx = a.take<uint32_t>(mall);
        l.heads = a.take<uint32_t>(mall);
        l.sizes = a.take<uint32_t>(mall);
        l.npairs = a.take<uint64_t>(mall);
        l.tmp = a.take<char>(std::max(sq_radix_tmp_bytes(mall), sq_scan_tmp_bytes(mall)));
        // the asynchronous form sorts the pairs in its own scratch (sized by the capacity)
        l.p0 = async ? a.take<uint64_t>(final_cap) : nullptr;
        l.p1 = async ? a.take<uint64_t>(final_cap) : nullptr;
        l.ptmp = async ? a.take<char>(sq_radix_tmp_bytes(final_cap)) : nullptr;
        return l;
    };
    SqArena measure(nullptr);
    layout(measure);
    SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    SqArena arena(ctx->scratch);
    auto L = layout(arena);
    const size_t tmp_bytes = std::max(sq_radix_tmp_bytes(mall), sq_scan_tmp_bytes(mall));

    unsigned long long *d_count = reinterpret_cast<unsigned long long *>(ctx->d_small);
    uint32_t *d_nchunks = reinterpret_cast<uint32_t *>(ctx->d_small + 1);
    uint64_t *d_total = ctx->d_small + 2;
    unsigned long long *d_kept64 = reinterpret_cast<unsigned long long *>(ctx->d_small + 3);
    const uint32_t *d_kept = reinterpret_cast<const uint32_t *>(ctx->d_small + 3);  // low word (< 2^32 keys)
    unsigned long long *d_clamped = reinterpret_cast<unsigned long long *>(ctx->d_small + 4);
    SQ_TRY_CUDA(cudaMemsetAsync(ctx->d_small, 0, 8 * sizeof(uint64_t), ctx->stream));
    SQ_TRY_CUDA(cudaMemsetAsync(L.chunk_of, 0xff, (size_t)n * bands * sizeof(uint32_t), ctx->stream));

    for (int band0 = 0; band0 < bands; band0 += G) {
        const int gb = std::min(G, bands - band0);
        const dim3 grid(sq_grid(ctx, n, 256, (8 + gb - 1) / gb), gb);
        const dim3 fgrid(sq_grid(ctx, (n + kInsIlp - 1) / kInsIlp, 256, (8 + gb - 1) / gb), gb);
        SqProfScope prof_ins(ctx, SUBQUAD_PROF_BAND_INSERT);
        SQ_TRY_CUDA(cudaMemsetAsync(L.table, 0xff, (size_t)gb * S * sizeof(uint32_t), ctx->stream));
        band_insert_kernel<<<grid, 256, 0, ctx->stream>>>(sig, n, rows, band0, log_s, donor, L.table, L.slot_of,
                                                          ctx->d_err);
        SQ_LAUNCH_CHECK();
        band_filter_kernel<<<fgrid, 256, 0, ctx->stream>>>(L.slot_of, L.table, n, band0, log_s, nbits, L.k0, d_kept64);
        SQ_LAUNCH_CHECK();
    }
    {
        // synchronous form: read the kept count back so the sort and scans
        // below launch grids for the kept keys (~10% of bands*n)
        int64_t kept = mall;
        const uint32_t *dk = d_kept;
        if (!async) {
            SQ_TRY_CUDA(cudaMemcpyAsync(ctx->h_pinned + 3, ctx->d_small + 3, sizeof(uint64_t),
                                        cudaMemcpyDeviceToHost, ctx->stream));
            SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
            kept = std::min<int64_t>((int64_t)ctx->h_pinned[3], mall);
            dk = nullptr;
        }
        const unsigned grid = sq_grid(ctx, std::max<int64_t>(kept, 1), 256, 8);
        bool in_alt = false;
        {
            SqProfScope prof_sort(ctx, SUBQUAD_PROF_BAND_SORT);
            SQ_TRY(sq_radix_sort_u64(ctx, L.k0, L.k1, kept, dk, 0, key_bits, &in_alt, L.tmp, tmp_bytes));
        }
        SqProfScope prof_emit(ctx, SUBQUAD_PROF_BAND_EMIT);
        const uint64_t *K = in_alt ? L.k1 : L.k0;
        band_heads_kernel<<<grid, 256, 0, ctx->stream>>>(K, nbits, kept, d_kept, L.run_start);
        SQ_LAUNCH_CHECK();
        SQ_TRY(sq_scan_u32(ctx, L.run_start, L.run_start, kept, dk, true, true, nullptr, L.tmp, tmp_bytes));
        band_chunks_kernel<<<grid, 256, 0, ctx->stream>>>(K, nbits, L.run_start, kept, d_kept, cap, log_s, 0, bands,
                                                          L.chunk_of, L.flags);
        SQ_LAUNCH_CHECK();
        SQ_TRY(sq_scan_u32(ctx, L.flags, L.cidx, kept, dk, false, false, d_nchunks, L.tmp, tmp_bytes));
        band_chunk_list_kernel<<<grid, 256, 0, ctx->stream>>>(L.run_start, L.flags, L.cidx, kept, d_kept, cap,
                                                              L.heads, L.sizes, L.npairs);
        SQ_LAUNCH_CHECK();
        // pair counts -> offsets.  Only the first nchunks entries are written;
        // an exclusive prefix at entry c depends on entries < c only, so the
        // unwritten tail never reaches a used offset.
        SQ_TRY(sq_scan_u64(ctx, L.npairs, L.npairs, kept, dk, nullptr, L.tmp, tmp_bytes));
        band_total_kernel<<<1, 1, 0, ctx->stream>>>(L.npairs, L.sizes, d_nchunks, d_total);
        SQ_LAUNCH_CHECK();
        band_emit_kernel<<<(unsigned)ctx->num_sms * 8, 256, 0, ctx->stream>>>(
            K, nbits, L.heads, L.sizes, L.npairs, d_nchunks, d_total, log_s, 0, bands, L.chunk_of, pairs_out,
            pairs_capacity, d_count, ctx->d_err);
        SQ_LAUNCH_CHECK();
    }
    if (async) {
        band_finish_kernel<<<1, 1, 0, ctx->stream>>>(d_count, pairs_capacity, d_num_pairs, d_clamped, ctx->d_err);
        SQ_LAUNCH_CHECK();
        if (pairs_capacity > 1) {
            const unsigned grid = sq_grid(ctx, pairs_capacity, 256, 8);
            pairs_to_keys_kernel<<<grid, 256, 0, ctx->stream>>>(pairs_out, pairs_capacity, d_clamped, nb, L.p0);
            SQ_LAUNCH_CHECK();
            bool in_alt = false;
            SQ_TRY(sq_radix_sort_u64(ctx, L.p0, L.p1, pairs_capacity, reinterpret_cast<const uint32_t *>(d_clamped),
                                     0, 2 * nb, &in_alt, L.ptmp, sq_radix_tmp_bytes(final_cap)));
            keys_to_pairs_kernel<<<grid, 256, 0, ctx->stream>>>(in_alt ? L.p1 : L.p0, pairs_capacity, d_clamped, nb,
                                                                pairs_out);
            SQ_LAUNCH_CHECK();
        }
        return SUBQUAD_OK;
    }
    SQ_TRY_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_small, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_TRY_CUDA(cudaMemcpyAsync(ctx->h_pinned + 1, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    const int64_t count = (int64_t)ctx->h_pinned[0];
    const uint32_t err = (uint32_t)(ctx->h_pinned[1] & 0xffffffffu);
    *num_pairs_out = count;
    if (err) return subquad_check(ctx);
    if (count > pairs_capacity) return SUBQUAD_ERR_CAPACITY;
    if (count > 1) {
        SqArena a2(nullptr);
        a2.take<uint64_t>(count);
        a2.take<uint64_t>(count);
        a2.take<char>(sq_radix_tmp_bytes(count));
        SQ_TRY(sq_scratch_reserve(ctx, a2.off));
        SqArena a3(ctx->scratch);
        uint64_t *k0 = a3.take<uint64_t>(count);
        uint64_t *k1 = a3.take<uint64_t>(count);
        void *tmp = a3.take<char>(sq_radix_tmp_bytes(count));
        const unsigned grid = sq_grid(ctx, count, 256, 8);
        SqProfScope prof_ps(ctx, SUBQUAD_PROF_BAND_PAIRSORT);
        pairs_to_keys_kernel<<<grid, 256, 0, ctx->stream>>>(pairs_out, count, nullptr, nb, k0);
        SQ_LAUNCH_CHECK();
        bool in_alt = false;
        SQ_TRY(sq_radix_sort_u64(ctx, k0, k1, count, nullptr, 0, 2 * nb, &in_alt, tmp, sq_radix_tmp_bytes(count)));
        keys_to_pairs_kernel<<<grid, 256, 0, ctx->stream>>>(in_alt ? k1 : k0, count, nullptr, nb, pairs_out);
        SQ_LAUNCH_CHECK();
    }
    return SUBQUAD_OK;
}

int band_args(int64_t n, int bands, int rows, int64_t pairs_capacity, const uint32_t *sig, const uint32_t *pairs_out)
{
    if (n < 0 || n >= (int64_t(1) << 31) || bands < 1 || rows < 1 || rows > 8 || bands * rows > 512 ||
        pairs_capacity < 0)
        return SUBQUAD_ERR_ARG;
    if (n >= 2 && (!sig || (pairs_capacity > 0 && !pairs_out))) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(sig) % 16 || reinterpret_cast<uintptr_t>(pairs_out) % 8) return SUBQUAD_ERR_ARG;
    return SUBQUAD_OK;
}

}  // namespace

extern "C" int subquad_band_candidates(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows,
                                       int32_t bucket_cap, uint32_t *pairs_out, int64_t pairs_capacity,
                                       int64_t *num_pairs_out)
{
    SQ_ENTER(ctx);
    if (!num_pairs_out) return SUBQUAD_ERR_ARG;
    *num_pairs_out = 0;
    SQ_TRY(band_args(n, bands, rows, pairs_capacity, sig, pairs_out));
    if (n < 2) return subquad_check(ctx);
    return band_run(ctx, sig, n, bands, rows, bucket_cap, nullptr, pairs_out, pairs_capacity, num_pairs_out, nullptr);
}

extern "C" int subquad_band_candidates_async(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows,
                                             int32_t bucket_cap, const int32_t *donor, uint32_t *pairs_out,
                                             int64_t pairs_capacity, uint64_t *d_num_pairs)
{
    SQ_ENTER(ctx);
    if (!d_num_pairs) return SUBQUAD_ERR_ARG;
    SQ_TRY(band_args(n, bands, rows, pairs_capacity, sig, pairs_out));
    if (n < 2) {
        SQ_TRY_CUDA(cudaMemsetAsync(d_num_pairs, 0, sizeof(uint64_t), ctx->stream));
        return SUBQUAD_OK;
    }
    return band_run(ctx, sig, n, bands, rows, bucket_cap, donor, pairs_out, pairs_capacity, nullptr,
                    reinterpret_cast<unsigned long long *>(d_num_pairs));
}
