// (a2) LSH banding, candidate emission and deduplication (Algorithm 1,
// preprocessing: "build MinHash index; generate candidate list CAND").
//
//  1. every (band, sequence) key -- the exact R-tuple, plus the donor in a
//     batch of donors -- is hashed to a 32-bit fingerprint and a partition
//     digit; a per-tile histogram, a scan and a scatter lay the records
//     (fingerprint, id) of each partition out contiguously;
//  2. one CTA per partition (about 2048 records) groups equal keys in a
//     shared-memory hash table (fingerprint match confirmed on the exact
//     keys); buckets of >= 2 members get contiguous kept positions, their
//     chunks (runs of cap members in id order; the whole bucket when it is
//     within cap) go to a chunk list, and each member records its chunk id
//     G[i][b] for the band (singletons keep a sentinel that matches nothing);
//  3. the chunk pair counts are scanned; each warp takes 32 consecutive pair
//     indices, finds their chunks, decodes (u, v) and keeps pair (i, j) only
//     if no earlier band already puts i and j in one chunk (first-band
//     ownership), so every pair of C is emitted once;
//  4. lexicographic order: degrees counted by the emitter give row offsets,
//     the second members are scattered into their rows and every row is
//     sorted (registers, a warp, a CTA, or in place in global memory);
//     the synchronous form then reads back |C| (its only host
//     synchronisation).
// Counts produced on the device (chunks, raw pairs) are consumed on the
// device: the kernels after them are sized for the upper bound and read the
// actual count.
#include <algorithm>
#include <new>

#include "internal.cuh"

namespace {

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

// Equal keys: the same R-tuple and, in a batch of donors, the same donor.
__device__ __forceinline__ bool same_key(const uint32_t *band_sig, int rows, uint32_t owner, const uint32_t k[8],
                                         const int32_t *donor, int32_t my_donor)
{
    return key_equal(band_sig + (int64_t)owner * rows, rows, k) && (!donor || donor[owner] == my_donor);
}

// Steps 1-2: hash partition of the (band, sequence) keys.
//
// Every key gets a 32-bit fingerprint fp (a hash of the R-tuple and, in a
// batch of donors, the donor) and a partition digit (pbits of an independent
// second hash).
// A per-tile digit histogram, an exclusive scan of the digit-major histogram
// and a scatter place the records (fp << 32 | id) of every partition
// contiguously (tile by tile; within a tile in any order).  Equal keys have
// equal fingerprints and so land in one partition.
constexpr int kPartThreads = 256;
constexpr int kPartItems = 16;
constexpr int kPartTile = kPartThreads * kPartItems;
constexpr int kPartMaxBits = 10;

struct KeyHash {
    uint32_t fp, digit;
};

// Two 32-bit hashes of the key: every word is pre-mixed (w ^ w >> 16, a
// bijection, so the low bits depend on the high ones), the words are summed
// in two polynomials mod 2^32 (Horner with two different odd multipliers)
// and each sum is finished by mix32: the fingerprint and the partition digit.
// Distinct keys share a partition and a fingerprint with probability about
// 2^-(32 + pbits) (a shared fingerprint is caught by the exact-key check).
constexpr uint32_t kFpMul = 0x9e3779b1u;
constexpr uint32_t kDigitMul = 0x85ebca77u;

__device__ __forceinline__ KeyHash hash_key(const uint32_t k[8], int rows, int32_t dn, int pbits)
{
    uint32_t a = 0x7f4a7c15u ^ (uint32_t)rows, g = 0x165667b1u ^ (uint32_t)rows;
#pragma unroll
    for (int r = 0; r < 8; ++r)
        if (r < rows) {
            const uint32_t w = k[r] ^ (k[r] >> 16);
            a = (a + w) * kFpMul;
            g = (g + w) * kDigitMul;
        }
    KeyHash h;
    h.fp = mix32(a ^ (uint32_t)dn);
    h.digit = pbits ? mix32(g ^ ((uint32_t)dn * 0x27d4eb2fu)) >> (32 - pbits) : 0u;
    return h;
}

// fd[gb * n + i] = (digit << 32 | fingerprint) of key (band0 + gb, i);
// hist[(gb * P + digit) * ntiles + tile] = members of the digit in the tile
__global__ void __launch_bounds__(kPartThreads) part_hist_kernel(const uint32_t *__restrict__ sig, int64_t n, int rows,
                                                                 int band0, int pbits, const int32_t *__restrict__ donor,
                                                                 int64_t ntiles, uint32_t *__restrict__ hist,
                                                                 uint64_t *__restrict__ fd)
{
    extern __shared__ uint32_t s_hist[];
    const int P = 1 << pbits, gb = blockIdx.y;
    for (int q = threadIdx.x; q < P; q += blockDim.x) s_hist[q] = 0;
    __syncthreads();
    const uint32_t *band_sig = sig + (int64_t)(band0 + gb) * n * rows;
    const int64_t tile = blockIdx.x;
    // all loads first (independent, so they are in flight together), then the counts
    uint32_t dg[kPartItems];
#pragma unroll
    for (int r = 0; r < kPartItems; ++r) {
        const int64_t i = tile * kPartTile + r * kPartThreads + threadIdx.x;
        dg[r] = 0x80000000u;
        if (i < n) {
            uint32_t k[8];
            load_key(band_sig + i * rows, rows, k);
            const KeyHash h = hash_key(k, rows, donor ? donor[i] : 0, pbits);
            dg[r] = h.digit;
            fd[(int64_t)gb * n + i] = ((uint64_t)h.digit << 32) | h.fp;
        }
    }
#pragma unroll
    for (int r = 0; r < kPartItems; ++r)
        if (dg[r] < 0x80000000u) atomicAdd(&s_hist[dg[r]], 1u);
    __syncthreads();
    for (int q = threadIdx.x; q < P; q += blockDim.x) hist[((int64_t)gb * P + q) * ntiles + tile] = s_hist[q];
}

// Scatter, staged in shared memory: every record takes a rank within its
// digit (shared-memory atomic), the tile's digit counts are scanned into
// local run starts, and the records are laid out digit by digit in shared
// memory (fingerprint, digit and index within the tile in one word); thread t
// then stores entry t of that layout at its run's scanned global offset.
// Consecutive threads store consecutive positions of a run, so a run leaves
// as one burst instead of one scattered 8-byte store per record.  A
// partition's records come tile by tile, in any order within a tile.
constexpr size_t part_scatter_smem(int P)
{
    return (size_t)kPartTile * sizeof(uint64_t) + 2 * (size_t)P * sizeof(uint32_t);
}
static_assert(part_scatter_smem(1 << kPartMaxBits) <= 48 * 1024, "the scatter needs no shared-memory opt-in");
static_assert(kPartTile <= 4096 && kPartMaxBits <= 20, "index within the tile (12 bits) and digit fit one word");

__global__ void __launch_bounds__(kPartThreads, 4) part_scatter_kernel(const uint64_t *__restrict__ fd, int64_t n,
                                                                    int pbits, int64_t ntiles,
                                                                    const uint32_t *__restrict__ offs,
                                                                    uint64_t *__restrict__ recs)
{
    extern __shared__ uint64_t s_stage[];  // [kPartTile] entries | [P] run starts | [P] global offsets
    uint32_t *s_run = reinterpret_cast<uint32_t *>(s_stage + kPartTile);
    const int P = 1 << pbits, gb = blockIdx.y;
    uint32_t *s_goff = s_run + P;
    __shared__ uint32_t s_warp[kPartThreads / 32];
    const int64_t tile = blockIdx.x;
    const int64_t t0 = tile * kPartTile;
    const int cnt = n - t0 < kPartTile ? (int)(n - t0) : kPartTile;
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        s_run[q] = 0;
        s_goff[q] = offs[((int64_t)gb * P + q) * ntiles + tile];
    }
    const uint64_t *band_fd = fd + (int64_t)gb * n + t0;
    uint64_t v[kPartItems];
    uint32_t rank[kPartItems];
#pragma unroll
    for (int r = 0; r < kPartItems; ++r) {
        const int t = r * kPartThreads + threadIdx.x;
        v[r] = t < cnt ? band_fd[t] : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPartItems; ++r) {
        const int t = r * kPartThreads + threadIdx.x;
        rank[r] = t < cnt ? atomicAdd(&s_run[(uint32_t)(v[r] >> 32)], 1u) : 0u;
    }
    __syncthreads();
    // exclusive scan of the P <= 1024 counts: runs of P / 256 (at least one)
    // consecutive digits per thread, then across the warps
    {
        const int per = (P + kPartThreads - 1) / kPartThreads;
        const int q0 = threadIdx.x * per;
        uint32_t own = 0;
        for (int q = q0; q < q0 + per && q < P; ++q) own += s_run[q];
        const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint32_t inc = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        uint32_t wbase = 0;
        for (uint32_t w = 0; w < warp; ++w) wbase += s_warp[w];
        uint32_t run = wbase + inc - own;
        for (int q = q0; q < q0 + per && q < P; ++q) {
            const uint32_t c = s_run[q];
            s_run[q] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPartItems; ++r) {
        const int t = r * kPartThreads + threadIdx.x;
        const uint32_t dg = (uint32_t)(v[r] >> 32);
        if (t < cnt) s_stage[s_run[dg] + rank[r]] = (v[r] << 32) | ((uint64_t)dg << 12) | (uint32_t)t;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += kPartThreads) {
        const uint64_t e = s_stage[t];
        const uint32_t dg = (uint32_t)(e >> 12) & 0xfffffu;
        recs[s_goff[dg] + (uint32_t)t - s_run[dg]] = (e & 0xffffffff00000000ull) | (uint32_t)(t0 + (e & 0xfffu));
    }
}

// Steps 3-4: one CTA per partition groups its records in a shared-memory
// hash table keyed by fingerprint; a fingerprint match is confirmed by
// comparing the two exact keys (and donors), so distinct keys never merge.
// Per bucket of c >= 2 members the CTA reserves c contiguous kept positions
// and writes its chunks (c members, or runs of cap members in id order when
// c > cap) to the chunk list; every kept member records its chunk head as its
// chunk id for the band.  Members are placed in any order; a bucket above
// the cap is then sorted by id in place, so chunk m holds ranks
// [m*cap, (m+1)*cap) (order_bucket).
// A partition holding more than kGrpDistinct distinct keys is split by
// further fingerprint bits into sub-ranges processed one after another.
constexpr int kGrpThreads = 256;
constexpr int kGrpSlots = 4096;
constexpr int kGrpDistinct = 3072;
constexpr int kGrpFast = 3072;       // partitions up to this size are grouped with records in shared memory
constexpr int kGrpFastSurv = 1024;   // ... when at most this many records pass the filter
constexpr int kGrpFastSlots = 2048;  // their table (load <= 1/2)
constexpr int kGrpVerify = 160;      // deferred key comparisons held in shared memory (more: compared at once)
constexpr int kGrpBloomWords = 1024;  // 32768-bit filter bitmaps (two), aliased on the table
constexpr uint32_t kFastEmpty = 0xffffffffu;
constexpr uint16_t kNoSlot = 0xffffu;
// fast-path layout: tab u32[2048] | cnt u32[2048] | rec u64[3072] | slot u16[3072] | surv u16[3072] |
//                   keys u16[1024] | vlist uint2[160]  (under 56 KB: four CTAs per SM)
constexpr size_t kGrpFastSmem = (size_t)kGrpFastSlots * 8 + (size_t)kGrpFast * 8 + (size_t)kGrpFast * 4 +
                                (size_t)kGrpFastSurv * 2 + (size_t)kGrpVerify * 8;
// exact-path layout: tab u64[4096] | cnt u32[4096]
constexpr size_t kGrpExactSmem = (size_t)kGrpSlots * (sizeof(unsigned long long) + sizeof(uint32_t));
constexpr size_t kGrpSmem = kGrpFastSmem > kGrpExactSmem ? kGrpFastSmem : kGrpExactSmem;
static_assert(kGrpFastSurv * 2 <= kGrpFastSlots, "a fast-path table is never more than half full");
static_assert(2 * kGrpBloomWords <= kGrpFastSlots, "the two filter bitmaps fit in the table's words");
static_assert(kGrpFast <= 4096, "record indices fit the 12 low bits of a fast-path table entry");
static_assert(kGrpFastSmem <= 56 * 1024, "four fast-path CTAs share an SM");
constexpr int kGrpStack = 48;
constexpr int kGrpMaxLevel = 20;  // sub-ranges select fingerprint bits 12..31
constexpr uint64_t kGrpEmpty = ~0ull;

__device__ __forceinline__ uint64_t block_exclusive_u64(uint64_t v, uint64_t *total, uint64_t *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (int w = 0; w < nw; ++w) {
            const uint64_t c = s_warp[w];
            s_warp[w] = run;
            run += c;
        }
        s_warp[32] = run;
    }
    __syncthreads();
    const uint64_t res = s_warp[warp] + inc - v;
    *total = s_warp[32];
    __syncthreads();
    return res;
}

struct GroupOut {
    uint32_t *kept_ids;
    unsigned long long *d_kept;
    uint32_t *d_nchunks;
    uint32_t *heads, *sizes, *cband;
    uint64_t *npairs;
    uint32_t *chunk_of;
    uint32_t *kept_mask;  // bit b (b < 32): the sequence is in a chunk of >= 2 members in band b
    uint32_t *rslot;
};

// Records that member id has chunk `head` in band b.
__device__ __forceinline__ void set_chunk(const GroupOut &o, uint32_t id, int b, int bands, uint32_t head)
{
    o.chunk_of[(int64_t)id * bands + b] = head;
    if (b < 32) atomicOr(&o.kept_mask[id], 1u << b);
}

struct GroupShared {
    unsigned long long *tab;  // (fp << 32 | owner id) while inserting; (kept offset << 32 | count) after
    uint32_t *cnt;            // member counts, then fill cursors
    uint64_t *scan;           // [33]
    uint32_t *distinct, *overflow, *big;
    unsigned long long *kbase;
    uint32_t *cbase;
};

// Slot of the record's key in the table, claiming an empty slot for a new
// key.  Table entries hold (fingerprint, owner id); a fingerprint match is
// confirmed on the exact keys.  Returns kGrpSlots if the table is declared
// overflowed (more than kGrpDistinct keys) before the key is placed.
__device__ __forceinline__ uint32_t find_or_claim(const GroupShared &g, uint32_t fp, uint32_t id,
                                                  const uint32_t *band_sig, int rows, const int32_t *donor)
{
    uint32_t slot = fp & (kGrpSlots - 1);
    bool have = false;
    uint32_t key[8];
    int32_t dn = 0;
    for (int probe = 0; probe < kGrpSlots; ++probe) {
        if (*(volatile uint32_t *)g.overflow) return kGrpSlots;
        unsigned long long e = g.tab[slot];
        if (e == kGrpEmpty) {
            const unsigned long long mine = ((unsigned long long)fp << 32) | id;
            e = atomicCAS(&g.tab[slot], kGrpEmpty, mine);
            if (e == kGrpEmpty) {
                if (atomicAdd(g.distinct, 1u) >= (uint32_t)kGrpDistinct) *g.overflow = 1;
                return slot;
            }
        }
        if ((uint32_t)(e >> 32) == fp) {
            if (!have) {
                load_key(band_sig + (int64_t)id * rows, rows, key);
                dn = donor ? donor[id] : 0;
                have = true;
            }
            if (same_key(band_sig, rows, (uint32_t)e, key, donor, dn)) return slot;
        }
        slot = (slot + 1) & (kGrpSlots - 1);
    }
    return kGrpSlots;
}

// Bucket offsets (kept members and chunks of >= 2 members per slot), one
// reservation of kept positions and chunk-list entries per table, chunk list
// entries, and the table rewritten to (kept offset << 32 | count).  Sets
// *g.big if a bucket exceeds the cap.  Ends with the block synchronised.
__device__ __forceinline__ void bucket_phase(const GroupShared &g, int cap, int b, const GroupOut &o)
{
    constexpr int kPer = kGrpSlots / kGrpThreads;
    uint32_t c[kPer];
    uint64_t mine = 0;
    bool big = false;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        c[j] = g.cnt[j * kGrpThreads + threadIdx.x];
        if (c[j] >= 2) {
            uint32_t nch = 1;
            if (cap > 0 && c[j] > (uint32_t)cap) {
                nch = (cap >= 2 ? c[j] / (uint32_t)cap : 0u) + ((c[j] % (uint32_t)cap) >= 2 ? 1u : 0u);
                big = true;
            }
            mine += ((uint64_t)c[j] << 32) | nch;
        }
    }
    uint64_t total;
    const uint64_t excl = block_exclusive_u64(mine, &total, g.scan);
    if (big) *g.big = 1;
    if (threadIdx.x == 0) {
        *g.kbase = (total >> 32) ? atomicAdd(o.d_kept, (unsigned long long)(total >> 32)) : 0ull;
        *g.cbase = (uint32_t)total ? atomicAdd(o.d_nchunks, (uint32_t)total) : 0u;
    }
    __syncthreads();
    uint32_t koff = (uint32_t)(excl >> 32), coff = (uint32_t)excl;
    const uint64_t kbase = *g.kbase;
    const uint32_t cbase = *g.cbase;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int slot = j * kGrpThreads + threadIdx.x;
        if (c[j] >= 2) {
            const uint32_t head = (uint32_t)(kbase + koff);
            const uint32_t step = (cap > 0 && c[j] > (uint32_t)cap) ? (uint32_t)cap : c[j];
            for (uint32_t m0 = 0; m0 < c[j]; m0 += step) {
                const uint32_t sz = min(step, c[j] - m0);
                if (sz < 2) continue;
                o.heads[cbase + coff] = head + m0;
                o.sizes[cbase + coff] = sz;
                o.cband[cbase + coff] = (uint32_t)b;
                o.npairs[cbase + coff] = (uint64_t)sz * (sz - 1) / 2;
                ++coff;
            }
            g.tab[slot] = ((unsigned long long)koff << 32) | c[j];
            koff += c[j];
        } else {
            g.tab[slot] = c[j];  // 0 or 1 member: nothing kept
        }
        g.cnt[slot] = 0;  // becomes the fill cursor
    }
    __syncthreads();
}

// Kept position of a member of a bucket (any order).  A member of a bucket
// within the cap records the bucket's single chunk; chunk ids of the members
// of a bucket above the cap follow once the bucket is ordered (order_bucket).
__device__ __forceinline__ void place_any(const GroupShared &g, uint32_t slot, uint32_t id, int cap, int b, int bands,
                                          const GroupOut &o)
{
    const unsigned long long e = g.tab[slot];
    const uint32_t cc = (uint32_t)e;
    if (cc < 2) return;
    const uint32_t r = atomicAdd(&g.cnt[slot], 1u);
    const uint64_t head = *g.kbase + (e >> 32);
    o.kept_ids[head + r] = id;
    if (cap > 0 && cc > (uint32_t)cap) return;
    set_chunk(o, id, b, bands, (uint32_t)head);
}

// A bucket above the cap: its c kept members (at v, kept position head) are
// sorted by id in place -- an all-ascending bitonic network over the next
// power of two, positions >= c acting as +infinity that never move -- and the
// member of rank r records chunk head + (r / cap) * cap, so chunk m holds
// ranks [m*cap, (m+1)*cap).  Called by every thread of the block.
__device__ void order_bucket(uint32_t *v, uint32_t c, uint32_t head, int cap, int b, int bands, const GroupOut &o)
{
    uint64_t P2 = 2;
    while (P2 < c) P2 <<= 1;
    for (uint64_t k = 2; k <= P2; k <<= 1) {
        for (uint64_t j = k >> 1; j > 0; j >>= 1) {
            for (uint64_t t = threadIdx.x; t < P2 / 2; t += blockDim.x) {
                const uint64_t a = (t / j) * 2 * j + (t % j);
                const uint64_t bb = j == (k >> 1) ? (a | (k - 1)) - (a & (k - 1)) : a + j;  // flip, then half-cleaners
                if (bb < c) {
                    const uint32_t x = v[a], y = v[bb];
                    if (x > y) {
                        v[a] = y;
                        v[bb] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t r = threadIdx.x; r < c; r += blockDim.x)
        set_chunk(o, v[r], b, bands, head + (r / (uint32_t)cap) * (uint32_t)cap);
    __syncthreads();
}

// Fast path for a partition of at most kGrpFast records, staged in shared
// memory.  A two-bitmap filter on fingerprint bits first drops the records
// whose key certainly occurs once (a record passes when another record set
// its bit before it, or it set a bit another record hits later); the
// passing records (about 15% on a donor repertoire, at most kGrpFastSurv)
// are grouped in a table of at least 2x their number (u32 entries: the upper
// 20 fingerprint bits and the owner's record index; the full fingerprint is
// compared through the staged record).  Every member that is not its
// bucket's owner then compares its exact key with the owner's (a deferred
// list processed by the whole block, so the loads overlap).  Returns false,
// with nothing written, if two distinct keys share a fingerprint or too many
// records pass: the caller then runs the exact path.
__device__ __forceinline__ bool group_fast(const uint64_t *__restrict__ prec, uint32_t cnt,
                                        const uint32_t *__restrict__ band_sig, int rows,
                                        const int32_t *__restrict__ donor, int cap, int b, int bands,
                                        const GroupOut &o, unsigned long long *s_dyn, uint64_t *s_scan,
                                        uint32_t &s_nk, uint32_t &s_nv, uint32_t &s_clash, uint32_t &s_big,
                                        unsigned long long &s_kbase, uint32_t &s_cbase)
{
    uint32_t *tab = reinterpret_cast<uint32_t *>(s_dyn);
    uint32_t *cntv = tab + kGrpFastSlots;
    uint64_t *srec = reinterpret_cast<uint64_t *>(cntv + kGrpFastSlots);
    uint16_t *sslot = reinterpret_cast<uint16_t *>(srec + kGrpFast);
    uint16_t *surv = sslot + kGrpFast;
    uint16_t *keys = surv + kGrpFast;
    uint2 *vlist = reinterpret_cast<uint2 *>(keys + kGrpFastSurv);
    uint32_t *bloom1 = tab, *bloom2 = tab + kGrpBloomWords;
    __shared__ uint32_t s_ns;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = (1u << lane) - 1u;

    for (uint32_t q = threadIdx.x; q < 2 * kGrpBloomWords; q += blockDim.x) tab[q] = 0u;
    if (threadIdx.x == 0) {
        s_ns = 0;
        s_nk = 0;
        s_nv = 0;
        s_clash = 0;
        s_big = 0;
    }
    __syncthreads();
    // records staged and entered in the filter in one pass: equal keys have
    // equal fingerprints, hence equal bits
    for (uint32_t q0 = threadIdx.x; q0 < cnt; q0 += 4 * blockDim.x) {
        uint64_t rec[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t q = q0 + u * blockDim.x;
            rec[u] = q < cnt ? prec[q] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t q = q0 + u * blockDim.x;
            if (q < cnt) {
                srec[q] = rec[u];
                const uint32_t bi = (uint32_t)(rec[u] >> 32) & (32u * kGrpBloomWords - 1u);
                const uint32_t bit = 1u << (bi & 31);
                if (atomicOr(&bloom1[bi >> 5], bit) & bit) atomicOr(&bloom2[bi >> 5], bit);
            }
        }
    }
    __syncthreads();
    for (uint32_t q0 = warp * 32; q0 < cnt; q0 += blockDim.x) {
        const uint32_t q = q0 + lane;
        bool pass = false;
        if (q < cnt) {
            const uint32_t bi = (uint32_t)(srec[q] >> 32) & (32u * kGrpBloomWords - 1u);
            pass = (bloom2[bi >> 5] >> (bi & 31)) & 1u;
            sslot[q] = kNoSlot;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, pass);
        uint32_t base = 0;
        if (lane == 0 && m) base = atomicAdd(&s_ns, (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint32_t at = base + __popc(m & lt);
        if (pass && at < (uint32_t)kGrpFast) surv[at] = (uint16_t)q;
    }
    __syncthreads();
    const uint32_t ns = s_ns;
    if (ns > (uint32_t)kGrpFastSurv) return false;  // uniform: too many keys repeat
    uint32_t tslots = 64;
    while (tslots < 2 * ns) tslots <<= 1;
    const int tshift = 33 - __ffs(tslots);
    for (uint32_t q = threadIdx.x; q < tslots; q += blockDim.x) {
        tab[q] = kFastEmpty;
        cntv[q] = 0;
    }
    __syncthreads();
    bool clash = false;
    // insert the passing records; warp-uniform trip count so the ballots see the whole warp
    for (uint32_t t0 = warp * 32; t0 < ns; t0 += blockDim.x) {
        const uint32_t t = t0 + lane;
        const bool valid = t < ns;
        const uint32_t q = valid ? surv[t] : 0u;
        uint32_t owner = q;
        if (valid) {
            const uint32_t fp = (uint32_t)(srec[q] >> 32);
            const uint32_t mine = (fp & ~0xfffu) | q;
            uint32_t sl = fp >> tshift;
#pragma unroll 1
            for (uint32_t probe = 0; probe < tslots; ++probe) {
                uint32_t e = tab[sl];
                if (e == kFastEmpty) {
                    e = atomicCAS(&tab[sl], kFastEmpty, mine);
                    if (e == kFastEmpty) break;
                }
                if (((e ^ fp) & ~0xfffu) == 0 && (uint32_t)(srec[e & 0xfffu] >> 32) == fp) {
                    owner = e & 0xfffu;
                    break;
                }
                sl = (sl + 1) & (tslots - 1);
            }
            sslot[q] = (uint16_t)sl;
            atomicAdd(&cntv[sl], 1u);
        }
        const bool need = valid && owner != q;
        const uint32_t m = __ballot_sync(0xffffffffu, need);
        uint32_t base = 0;
        if (lane == 0 && m) base = atomicAdd(&s_nv, (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (need) {
            const uint32_t v = base + __popc(m & lt);
            if (v < (uint32_t)kGrpVerify) {
                vlist[v] = make_uint2(q, owner);
            } else {
                const uint32_t id = (uint32_t)srec[q];
                uint32_t key[8];
                load_key(band_sig + (int64_t)id * rows, rows, key);
                clash = clash || !same_key(band_sig, rows, (uint32_t)srec[owner], key, donor, donor ? donor[id] : 0);
            }
        }
    }
    __syncthreads();
    const uint32_t nv = min(s_nv, (uint32_t)kGrpVerify);
    for (uint32_t t = threadIdx.x; t < nv; t += blockDim.x) {
        const uint2 pr = vlist[t];
        const uint32_t id = (uint32_t)srec[pr.x];
        uint32_t key[8];
        load_key(band_sig + (int64_t)id * rows, rows, key);
        clash = clash || !same_key(band_sig, rows, (uint32_t)srec[pr.y], key, donor, donor ? donor[id] : 0);
    }
    // buckets of >= 2 members listed (warp-aggregated appends); every other
    // slot's entry becomes its member count (0 or 1)
    for (uint32_t t0 = 0; t0 < tslots; t0 += blockDim.x) {
        const uint32_t sl = t0 + threadIdx.x;
        const bool in = sl < tslots;
        const uint32_t c = in ? cntv[sl] : 0u;
        const bool kept = c >= 2;
        if (in && !kept) tab[sl] = c;
        const uint32_t m = __ballot_sync(0xffffffffu, kept);
        uint32_t base = 0;
        if (lane == 0 && m) base = atomicAdd(&s_nk, (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (kept) keys[base + __popc(m & lt)] = (uint16_t)sl;
    }
    if (clash) s_clash = 1;
    __syncthreads();
    if (s_clash) return false;  // uniform: read after the barrier

    // kept offsets and chunk counts over the listed buckets
    const uint32_t nk = s_nk;
    uint64_t sum = 0;
    bool big = false;
    for (uint32_t t = threadIdx.x; t < nk; t += blockDim.x) {
        const uint32_t c = cntv[keys[t]];
        uint32_t nch = 1;
        if (cap > 0 && c > (uint32_t)cap) {
            nch = (cap >= 2 ? c / (uint32_t)cap : 0u) + ((c % (uint32_t)cap) >= 2 ? 1u : 0u);
            big = true;
        }
        sum += ((uint64_t)c << 32) | nch;
    }
    uint64_t total;
    const uint64_t excl = block_exclusive_u64(sum, &total, s_scan);
    if (big) s_big = 1;
    if (threadIdx.x == 0) {
        s_kbase = (total >> 32) ? atomicAdd(o.d_kept, (unsigned long long)(total >> 32)) : 0ull;
        s_cbase = (uint32_t)total ? atomicAdd(o.d_nchunks, (uint32_t)total) : 0u;
    }
    __syncthreads();
    const uint64_t kbase = s_kbase;
    {
        uint32_t koff = (uint32_t)(excl >> 32), coff = (uint32_t)excl;
        const uint32_t cbase = s_cbase;
        for (uint32_t t = threadIdx.x; t < nk; t += blockDim.x) {
            const uint32_t sl = keys[t];
            const uint32_t c = cntv[sl];
            const uint32_t head = (uint32_t)(kbase + koff);
            const uint32_t step = (cap > 0 && c > (uint32_t)cap) ? (uint32_t)cap : c;
            for (uint32_t m0 = 0; m0 < c; m0 += step) {
                const uint32_t sz = min(step, c - m0);
                if (sz < 2) continue;
                o.heads[cbase + coff] = head + m0;
                o.sizes[cbase + coff] = sz;
                o.cband[cbase + coff] = (uint32_t)b;
                o.npairs[cbase + coff] = (uint64_t)sz * (sz - 1) / 2;
                ++coff;
            }
            tab[sl] = (koff << 16) | c;  // koff, c < 2^12
            koff += c;
            cntv[sl] = 0;  // becomes the fill cursor
        }
    }
    __syncthreads();
    // kept positions in any order; members of buckets within the cap record
    // their chunk now, those of buckets above it once the bucket is ordered
    for (uint32_t t = threadIdx.x; t < ns; t += blockDim.x) {
        const uint32_t q = surv[t];
        const uint32_t e = tab[sslot[q]];
        const uint32_t c = e & 0xffffu;
        if (c < 2 || e == kFastEmpty) continue;
        const uint32_t r = atomicAdd(&cntv[sslot[q]], 1u);
        const uint64_t head = kbase + (e >> 16);
        const uint32_t id = (uint32_t)srec[q];
        o.kept_ids[head + r] = id;
        if (cap > 0 && c > (uint32_t)cap) continue;
        set_chunk(o, id, b, bands, (uint32_t)head);
    }
    if (s_big) {  // uniform: set before a barrier
        // the buckets above the cap, listed (surv is free), then ordered one by one
        if (threadIdx.x == 0) s_ns = 0;
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < nk; t += blockDim.x) {
            const uint32_t c = tab[keys[t]] & 0xffffu;
            if (c > (uint32_t)cap) surv[atomicAdd(&s_ns, 1u)] = keys[t];
        }
        __syncthreads();
        const uint32_t nbig = s_ns;
        for (uint32_t k = 0; k < nbig; ++k) {
            const uint32_t e = tab[surv[k]];
            const uint32_t head = (uint32_t)(kbase + (e >> 16));
            order_bucket(o.kept_ids + head, e & 0xffffu, head, cap, b, bands, o);
        }
    }
    return true;
}

__global__ void __launch_bounds__(kGrpThreads, 4) part_group_kernel(
    const uint64_t *__restrict__ recs, const uint32_t *__restrict__ offs, int64_t ntiles, int64_t total_recs,
    int pbits, int band0, int bands, const uint32_t *__restrict__ sig, int64_t n, int rows,
    const int32_t *__restrict__ donor, int cap, GroupOut o, uint32_t *err)
{
    extern __shared__ unsigned long long s_dyn[];
    __shared__ uint64_t s_scan[33];
    __shared__ uint32_t s_stack[kGrpStack][2];
    __shared__ int s_top;
    __shared__ uint32_t s_distinct, s_overflow, s_big, s_nv;
    __shared__ unsigned long long s_kbase;
    __shared__ uint32_t s_cbase;
    GroupShared g;
    g.tab = s_dyn;
    g.cnt = reinterpret_cast<uint32_t *>(s_dyn + kGrpSlots);
    g.scan = s_scan;
    g.distinct = &s_distinct;
    g.overflow = &s_overflow;
    g.big = &s_big;
    g.kbase = &s_kbase;
    g.cbase = &s_cbase;

    const int64_t p = blockIdx.x;
    const int gb = (int)(p >> pbits), b = band0 + gb;
    const int64_t start = offs[p * ntiles];
    const int64_t end = p + 1 < (int64_t)gridDim.x ? (int64_t)offs[(p + 1) * ntiles] : total_recs;
    const int64_t cnt = end - start;
    if (cnt < 2) return;
    const uint32_t *band_sig = sig + (int64_t)b * n * rows;
    const uint64_t *prec = recs + start;

    if (cnt <= kGrpFast &&
        group_fast(prec, (uint32_t)cnt, band_sig, rows, donor, cap, b, bands, o, s_dyn, s_scan, s_distinct, s_nv,
                   s_overflow, s_big, s_kbase, s_cbase))
        return;

    // Large partition (or a fingerprint clash): records streamed from global
    // memory, every fingerprint match confirmed on the exact keys before it
    // joins a bucket; the partition is split into fingerprint sub-ranges (a stack of (level, k): the records
    // with ((fp >> 12) mod 2^level) == k) while one holds too many keys.
    uint32_t *rslot = o.rslot + start;
    if (threadIdx.x == 0) {
        s_stack[0][0] = 0;
        s_stack[0][1] = 0;
        s_top = 1;
    }
    for (;;) {
        __syncthreads();
        const int top = s_top;
        if (top == 0) break;
        const uint32_t level = s_stack[top - 1][0], k = s_stack[top - 1][1];
        const uint32_t kmask = (1u << level) - 1u;
        __syncthreads();  // every thread has read the node before it is popped
        for (int q = threadIdx.x; q < kGrpSlots; q += blockDim.x) {
            g.tab[q] = kGrpEmpty;
            g.cnt[q] = 0;
        }
        if (threadIdx.x == 0) {
            s_top = top - 1;
            s_distinct = 0;
            s_overflow = 0;
            s_big = 0;
        }
        __syncthreads();
        for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
            const uint64_t rec = prec[q];
            const uint32_t fp = (uint32_t)(rec >> 32);
            if (((fp >> 12) & kmask) != k) continue;
            const uint32_t sl = find_or_claim(g, fp, (uint32_t)rec, band_sig, rows, donor);
            if (sl < (uint32_t)kGrpSlots) {
                rslot[q] = sl;
                atomicAdd(&g.cnt[sl], 1u);
            } else {
                s_overflow = 1;
            }
        }
        __syncthreads();
        if (s_overflow) {
            if (threadIdx.x == 0) {
                if (level + 1 > (uint32_t)kGrpMaxLevel || s_top + 2 > kGrpStack) {
                    atomicOr(err, SQ_DEVERR_CAPACITY);
                } else {
                    s_stack[s_top][0] = level + 1;
                    s_stack[s_top][1] = k + (1u << level);
                    s_stack[s_top + 1][0] = level + 1;
                    s_stack[s_top + 1][1] = k;
                    s_top += 2;
                }
            }
            continue;
        }
        bucket_phase(g, cap, b, o);
        for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
            const uint64_t rec = prec[q];
            if ((((uint32_t)(rec >> 32) >> 12) & kmask) != k) continue;
            place_any(g, rslot[q], (uint32_t)rec, cap, b, bands, o);
        }
        if (s_big) {  // uniform: set before the barrier that ends bucket_phase
            // the buckets above the cap, listed in the free cursor array, then ordered one by one
            __syncthreads();
            if (threadIdx.x == 0) s_distinct = 0;
            __syncthreads();
            for (int q = threadIdx.x; q < kGrpSlots; q += blockDim.x) {
                const uint32_t c = (uint32_t)g.tab[q];
                if (c >= 2 && c > (uint32_t)cap) g.cnt[atomicAdd(&s_distinct, 1u)] = (uint32_t)q;
            }
            __syncthreads();
            const uint32_t nbig = s_distinct;
            for (uint32_t t = 0; t < nbig; ++t) {
                const unsigned long long e = g.tab[g.cnt[t]];
                const uint32_t head = (uint32_t)(*g.kbase + (e >> 32));
                order_bucket(o.kept_ids + head, (uint32_t)e, head, cap, b, bands, o);
            }
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

// Chunk holding the first raw pair of every group of 32 (one binary search
// per group, all in parallel).
__device__ __forceinline__ uint32_t chunk_of_raw(const uint64_t *__restrict__ poff, uint32_t nc, uint64_t q)
{
    uint32_t lo = 0, hi = nc;  // largest c with poff[c] <= q (every chunk has >= 1 pair)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (poff[mid] <= q) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void band_warp_chunk_kernel(const uint64_t *__restrict__ poff, const uint32_t *__restrict__ d_nchunks,
                                       const uint64_t *__restrict__ d_total, uint32_t *__restrict__ wchunk,
                                       int64_t wmax)
{
    const uint32_t nc = *d_nchunks;
    const uint64_t groups = min((*d_total + 31) / 32, (uint64_t)wmax);
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < groups;
         w += (uint64_t)gridDim.x * blockDim.x)
        wchunk[w] = chunk_of_raw(poff, nc, w * 32);
}

// Lanes of the warp holding the same value as their neighbours form runs;
// run_of returns the lane mask of the calling lane's run and its first lane.
// Every lane of the warp must call it.
struct RunOf {
    uint32_t mask, first;
};
__device__ __forceinline__ RunOf run_of(uint32_t key, uint32_t lane)
{
    const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
    const uint32_t upto = (2u << lane) - 1u;  // lanes 0..lane (all lanes for lane 31)
    const uint32_t first = 31u - __clz(heads & upto);
    const uint32_t later = heads & ~upto;
    const uint32_t end = later ? (uint32_t)__ffs(later) - 1u : 32u;
    const uint32_t mask = (end == 32u ? 0xffffffffu : ((1u << end) - 1u)) & ~((1u << first) - 1u);
    return {mask, first};
}

// Positions of up to two appends per thread in one block-wide reservation:
// the block's f0 appends first (in thread order), then its f1 appends, so the
// output keeps the order of each span.  Every thread of the block must call it.
__device__ __forceinline__ void block_append2(bool f0, bool f1, unsigned long long *counter,
                                              unsigned long long *s_base, uint32_t *s_warp,
                                              unsigned long long &p0, unsigned long long &p1)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t c = (uint32_t)f0 | ((uint32_t)f1 << 16);  // two counters of < 2^16 (blockDim <= 1024)
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= (uint32_t)d) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (uint32_t w = 0; w < nw; ++w) {
            const uint32_t t = s_warp[w];
            s_warp[w] = run;
            run += t;
        }
        const uint32_t n0 = run & 0xffffu, n1 = run >> 16;
        s_warp[nw] = n0;
        *s_base = n0 + n1 ? atomicAdd(counter, (unsigned long long)(n0 + n1)) : 0ull;
    }
    __syncthreads();
    const uint32_t excl = s_warp[warp] + inc - c;
    p0 = *s_base + (excl & 0xffffu);
    p1 = *s_base + s_warp[nw] + (excl >> 16);
    __syncthreads();
}

// Step 5: owned pairs, appended to out.  Each warp takes 32 consecutive raw
// pair indices; their chunks are c0 (looked up) plus the chunks starting
// inside the group (one load per lane and a warp OR of start positions); each
// lane decodes its (u, v) and keeps pair (i, j) only if no earlier band
// already puts i and j in one chunk (first-band ownership), so every pair of
// C is emitted exactly once.
// Each block iteration takes two spans of blockDim raw pairs, so every thread
// carries two independent chains of dependent loads (chunk -> chunk entry ->
// member ids -> masks and chunk ids) in flight.
__global__ void __launch_bounds__(256) band_emit_kernel(
    const uint32_t *__restrict__ kept_ids, const uint32_t *__restrict__ heads, const uint32_t *__restrict__ sizes,
    const uint32_t *__restrict__ cband, const uint64_t *__restrict__ poff, const uint32_t *__restrict__ wchunk,
    int64_t wmax, const uint32_t *__restrict__ d_nchunks, const uint64_t *__restrict__ d_total, int bands,
    const uint32_t *__restrict__ chunk_of, const uint32_t *__restrict__ kept_mask, uint64_t raw0, uint64_t raw1,
    uint32_t *__restrict__ out, int64_t capacity, unsigned long long *__restrict__ d_count,
    uint32_t *__restrict__ deg, uint32_t *err)
{
    constexpr int H = 2;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_warp[33];
    const uint32_t nc = *d_nchunks;
    const uint64_t total = min(*d_total, raw1);  // raw pairs [raw0, total) of this call; raw0 % 32 == 0
    const uint32_t lane = threadIdx.x & 31;
    // block-uniform trip count (block_append2 synchronises the block)
    for (uint64_t b0 = raw0 + (uint64_t)blockIdx.x * blockDim.x * H; b0 < total;
         b0 += (uint64_t)gridDim.x * blockDim.x * H) {
        uint64_t q0[H], q[H];
        uint32_t c0[H], starts[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            q0[h] = b0 + (uint64_t)h * blockDim.x + (threadIdx.x & ~31u);
            q[h] = q0[h] + lane;
            c0[h] = 0;
            starts[h] = 0;
            if (q0[h] < total) {
                c0[h] = q0[h] / 32 < (uint64_t)wmax ? wchunk[q0[h] / 32] : chunk_of_raw(poff, nc, q0[h]);
                const uint32_t c = c0[h] + 1 + lane;
                if (c < nc) {
                    const uint64_t d = poff[c] - q0[h];  // >= 1: chunk c starts after q0
                    if (d < 32) starts[h] = 1u << d;
                }
            }
        }
        bool owned[H];
        uint32_t i[H], j[H], b[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            starts[h] = __reduce_or_sync(0xffffffffu, starts[h]);
            owned[h] = false;
            i[h] = j[h] = b[h] = 0;
            if (q[h] < total) {
                const uint32_t cl = c0[h] + __popc(starts[h] & ((2u << lane) - 1u));
                const uint32_t hd = heads[cl], sz = sizes[cl];
                b[h] = cband[cl];
                uint32_t u, v;
                decode_pair(q[h] - poff[cl], sz, u, v);
                if (u >= v || v >= sz) {  // cannot happen for a consistent chunk list
                    atomicOr(err, SQ_DEVERR_INTERNAL);
                    u = 0;
                    v = 1;
                }
                i[h] = kept_ids[hd + u];
                j[h] = kept_ids[hd + v];
                owned[h] = true;
            }
        }
        uint32_t common[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if (i[h] > j[h]) {
                const uint32_t t = i[h];
                i[h] = j[h];
                j[h] = t;
            }
            // earlier bands where both are in some chunk (mask), then their chunk ids
            common[h] = owned[h] ? kept_mask[i[h]] & kept_mask[j[h]] &
                                       (b[h] >= 32 ? 0xffffffffu : ((1u << b[h]) - 1u))
                                 : 0u;
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if (!owned[h]) continue;
            const uint32_t *gi = chunk_of + (int64_t)i[h] * bands;
            const uint32_t *gj = chunk_of + (int64_t)j[h] * bands;
            while (common[h]) {
                const int bb = __ffs(common[h]) - 1;
                common[h] &= common[h] - 1u;
                if (gi[bb] == gj[bb]) {
                    owned[h] = false;
                    break;
                }
            }
            for (int bb = 32; owned[h] && bb < (int)b[h]; ++bb) {
                const uint32_t x = gi[bb], y = gj[bb];
                if (x == y && x != kNoChunk) owned[h] = false;
            }
        }
        unsigned long long pos[H];
        block_append2(owned[0], owned[1], d_count, &s_base, s_warp, pos[0], pos[1]);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const bool written = owned[h] && pos[h] < (unsigned long long)capacity;
            if (written) reinterpret_cast<uint2 *>(out)[pos[h]] = make_uint2(i[h], j[h]);
            if (deg) {
                // one count per run of equal first members (a chunk's pairs come
                // in runs sharing i): the run's first written lane adds them all
                const RunOf r = run_of(q[h] < total ? i[h] : 0xffffffffu, lane);
                const uint32_t mine = __ballot_sync(0xffffffffu, written) & r.mask;
                if (written && lane == (uint32_t)__ffs(mine) - 1u) atomicAdd(&deg[i[h]], (uint32_t)__popc(mine));
            }
        }
    }
}

// Lexicographic order of the emitted pairs: a counting pass by first member
// i (degrees counted by the emitter, scanned into row offsets), a scatter of
// the second members into their rows, and a sort of every row, the rows
// listed by size class first: by one thread in registers for rows of at most
// kRowSmall partners (four classes, so the lanes of a warp sort rows of one
// size), by one warp up to kRowWarp, by one CTA in shared memory up to
// kRowMid, in place in global memory beyond.
// Every count stays on the device.
constexpr int kRowSmall = 32;
constexpr int kRowWarp = 512;   // rows up to this size: one warp, registers
constexpr int kRowMid = 8192;   // rows up to this size: one CTA, radix sort in shared memory
constexpr int kRowThreads = 256;

__device__ __forceinline__ uint64_t row_end(const uint32_t *rowoff, int64_t n, uint64_t m, int64_t i)
{
    return i + 1 < n ? rowoff[i + 1] : m;
}

// Row classes by partner count d: 2..4, 5..8, 9..16, 17..32 (sorted by one
// thread per row in registers), 33..kRowWarp (one warp), kRowWarp+1..kRowMid
// (one CTA), longer (in place in global memory).  Each class is listed so a
// warp of a sorting kernel takes rows of one class only.
constexpr int kRowClasses = 7;
enum { kClsS4 = 0, kClsS8, kClsS16, kClsS32, kClsWarp, kClsCta, kClsLong };

__device__ __forceinline__ int row_class(uint64_t d)
{
    if (d <= 1) return -1;
    if (d <= 4) return kClsS4;
    if (d <= 8) return kClsS8;
    if (d <= 16) return kClsS16;
    if (d <= (uint64_t)kRowSmall) return kClsS32;
    if (d <= (uint64_t)kRowWarp) return kClsWarp;
    if (d <= (uint64_t)kRowMid) return kClsCta;
    return kClsLong;
}

// Positions of the block's threads in per-class lists: one ballot per class
// per warp, one atomic per class per block (cls < 0: no list).
__device__ __forceinline__ unsigned long long block_append_class(int cls, unsigned long long *counters,
                                                                 unsigned long long *s_base,
                                                                 uint32_t (*s_wc)[32])
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t rank = 0;
#pragma unroll
    for (int c = 0; c < kRowClasses; ++c) {
        const uint32_t mk = __ballot_sync(0xffffffffu, cls == c);
        if (cls == c) rank = __popc(mk & ((1u << lane) - 1u));
        if (lane == 0) s_wc[c][warp] = __popc(mk);
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)kRowClasses) {
        const int c = threadIdx.x;
        uint32_t run = 0;
        for (uint32_t w = 0; w < nw; ++w) {
            const uint32_t t = s_wc[c][w];
            s_wc[c][w] = run;
            run += t;
        }
        s_base[c] = run ? atomicAdd(&counters[c], (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    const unsigned long long pos = cls >= 0 ? s_base[cls] + s_wc[cls][warp] + rank : 0ull;
    __syncthreads();
    return pos;
}

// Lists: classes S4/S8 from the front/back of sa, S16/S32 of sb, Warp/Cta
// of mid, Long in lng.  Rows of one partner are written out here (the row
// columns are in place).
__global__ void __launch_bounds__(kRowThreads) rows_classify_kernel(const uint32_t *__restrict__ rowoff, int64_t n,
                                                                    const unsigned long long *__restrict__ d_m,
                                                                    const uint32_t *__restrict__ col,
                                                                    uint32_t *__restrict__ out,
                                                                    uint32_t *__restrict__ sa, uint32_t *__restrict__ sb,
                                                                    uint32_t *__restrict__ mid,
                                                                    uint32_t *__restrict__ lng,
                                                                    unsigned long long *__restrict__ d_cls)
{
    __shared__ unsigned long long s_base[kRowClasses];
    __shared__ uint32_t s_wc[kRowClasses][32];
    const uint64_t m = *d_m;
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < n; b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        uint64_t d = 0, r0 = 0;
        if (i < n) {
            r0 = rowoff[i];
            d = row_end(rowoff, n, m, i) - r0;
        }
        if (d == 1) reinterpret_cast<uint2 *>(out)[r0] = make_uint2((uint32_t)i, col[r0]);
        const int cls = row_class(d);
        const unsigned long long pos = block_append_class(cls, d_cls, s_base, s_wc);
        switch (cls) {
        case kClsS4: sa[pos] = (uint32_t)i; break;
        case kClsS8: sa[n - 1 - (int64_t)pos] = (uint32_t)i; break;
        case kClsS16: sb[pos] = (uint32_t)i; break;
        case kClsS32: sb[n - 1 - (int64_t)pos] = (uint32_t)i; break;
        case kClsWarp: mid[pos] = (uint32_t)i; break;
        case kClsCta: mid[n - 1 - (int64_t)pos] = (uint32_t)i; break;
        case kClsLong: lng[pos] = (uint32_t)i; break;
        default: break;
        }
    }
}

// The emitter's owned count is also finished here, by the first thread: it
// is published (with the sticky CAPACITY error when it exceeds the
// capacity) and clamped to the capacity for the kernels after this one; the
// scatter itself takes the clamped count directly.
__global__ void pairs_scatter_kernel(const uint32_t *__restrict__ pairs, const unsigned long long *__restrict__ d_count,
                                     int64_t capacity, unsigned long long *__restrict__ d_out,
                                     unsigned long long *__restrict__ d_clamped, uint32_t *err,
                                     const uint32_t *__restrict__ rowoff, uint32_t *__restrict__ fill,
                                     uint32_t *__restrict__ col)
{
    constexpr int H = 4;  // groups of 32 pairs per warp and iteration, their loads in flight together
    const unsigned long long c = *d_count;
    const unsigned long long clamped = c < (unsigned long long)capacity ? c : (unsigned long long)capacity;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (d_out) *d_out = c;
        if (d_out && c > (unsigned long long)capacity) atomicOr(err, SQ_DEVERR_CAPACITY);
        *d_clamped = clamped;
    }
    const int64_t m = (int64_t)clamped;
    const uint32_t lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // warp-uniform trip count; a run of equal first members takes its slots
    // with one atomic (positions old-1, old-2, ... in lane order)
    // (the next iteration's pairs are loaded one iteration ahead)
    uint2 nxt[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int64_t p = warp * 32 * H + h * 32 + lane;
        nxt[h] = p < m ? reinterpret_cast<const uint2 *>(pairs)[p] : make_uint2(0xffffffffu, 0u);
    }
    for (int64_t pb = warp * 32 * H; pb < m; pb += nwarps * 32 * H) {
        uint2 ij[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            ij[h] = nxt[h];
            const int64_t p = pb + nwarps * 32 * H + h * 32 + lane;
            nxt[h] = p < m ? reinterpret_cast<const uint2 *>(pairs)[p] : make_uint2(0xffffffffu, 0u);
        }
        uint32_t top[H], first[H], off[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const RunOf r = run_of(ij[h].x, lane);
            first[h] = r.first;
            top[h] = 0;
            off[h] = 0;
            if (ij[h].x != 0xffffffffu) {
                if (lane == r.first) top[h] = atomicSub(&fill[ij[h].x], (uint32_t)__popc(r.mask));
                off[h] = rowoff[ij[h].x];
            }
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const uint32_t t = __shfl_sync(0xffffffffu, top[h], first[h]);
            if (ij[h].x != 0xffffffffu) col[off[h] + t - 1u - (lane - first[h])] = ij[h].y;
        }
    }
}

template <int N>
__device__ __forceinline__ void bitonic_regs(uint32_t (&v)[N])
{
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const int b = a ^ j;
                if (b > a) {
                    const uint32_t lo = min(v[a], v[b]), hi = max(v[a], v[b]);
                    const bool asc = (a & k) == 0;
                    v[a] = asc ? lo : hi;
                    v[b] = asc ? hi : lo;
                }
            }
}

template <int N>
__device__ __forceinline__ void sort_row_regs(const uint32_t *__restrict__ col, uint64_t r0, uint32_t d, uint32_t i,
                                              uint32_t *__restrict__ out)
{
    uint32_t v[N];
#pragma unroll
    for (int t = 0; t < N; ++t) v[t] = (uint32_t)t < d ? col[r0 + t] : 0xffffffffu;
    bitonic_regs<N>(v);
#pragma unroll
    for (int t = 0; t < N; ++t)
        if ((uint32_t)t < d) reinterpret_cast<uint2 *>(out)[r0 + t] = make_uint2(i, v[t]);
}

// One thread per row of 2..32 partners; the four class lists are walked in
// turn so the lanes of a warp (nearly always) sort rows of one class.
__global__ void __launch_bounds__(kRowThreads) rows_sort_small_kernel(const uint32_t *__restrict__ rowoff, int64_t n,
                                                                      const unsigned long long *__restrict__ d_m,
                                                                      const uint32_t *__restrict__ sa,
                                                                      const uint32_t *__restrict__ sb,
                                                                      const unsigned long long *__restrict__ d_cls,
                                                                      const uint32_t *__restrict__ col,
                                                                      uint32_t *__restrict__ out)
{
    const uint64_t m = *d_m;
    const uint64_t e0 = d_cls[kClsS4], e1 = e0 + d_cls[kClsS8], e2 = e1 + d_cls[kClsS16], e3 = e2 + d_cls[kClsS32];
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < e3; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = v < e0 ? sa[v] : v < e1 ? sa[n - 1 - (int64_t)(v - e0)]
                         : v < e2 ? sb[v - e1] : sb[n - 1 - (int64_t)(v - e2)];
        const uint64_t r0 = rowoff[i];
        const uint32_t d = (uint32_t)(row_end(rowoff, n, m, i) - r0);
        if (v < e0) sort_row_regs<4>(col, r0, d, i, out);
        else if (v < e1) sort_row_regs<8>(col, r0, d, i, out);
        else if (v < e2) sort_row_regs<16>(col, r0, d, i, out);
        else sort_row_regs<32>(col, r0, d, i, out);
    }
}

// One warp per row of 33..kRowWarp partners: E values per lane in striped
// order (element a = e * 32 + lane), bitonic network over 32 E elements with
// register exchanges for distances >= 32 and lane shuffles below.
template <int E>
__device__ __forceinline__ void sort_row_warp(const uint32_t *__restrict__ col, uint64_t r0, uint32_t d, uint32_t i,
                                              uint32_t *__restrict__ out)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t a = e * 32 + lane;
        v[e] = a < d ? col[r0 + a] : 0xffffffffu;
    }
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jr = j >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int e2 = e ^ jr;
                    if (e2 > e) {
                        const bool asc = ((e * 32 + lane) & k) == 0;
                        const uint32_t lo = min(v[e], v[e2]), hi = max(v[e], v[e2]);
                        v[e] = asc ? lo : hi;
                        v[e2] = asc ? hi : lo;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t y = __shfl_xor_sync(0xffffffffu, v[e], j);
                    const bool asc = ((e * 32 + lane) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    v[e] = (lower == asc) ? min(v[e], y) : max(v[e], y);
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t a = e * 32 + lane;
        if (a < d) reinterpret_cast<uint2 *>(out)[r0 + a] = make_uint2(i, v[e]);
    }
}

__global__ void __launch_bounds__(kRowThreads) rows_sort_warp_kernel(const uint32_t *__restrict__ rowoff, int64_t n,
                                                                     const unsigned long long *__restrict__ d_m,
                                                                     const uint32_t *__restrict__ mid,
                                                                     const unsigned long long *__restrict__ d_warp,
                                                                     const uint32_t *__restrict__ col,
                                                                     uint32_t *__restrict__ out)
{
    const uint64_t m = *d_m, nrows = *d_warp;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t wstep = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = w0; r < nrows; r += wstep) {
        const uint32_t i = mid[r];
        const uint64_t r0 = rowoff[i];
        const uint32_t d = (uint32_t)(row_end(rowoff, n, m, i) - r0);
        if (d <= 64) sort_row_warp<2>(col, r0, d, i, out);
        else if (d <= 128) sort_row_warp<4>(col, r0, d, i, out);
        else if (d <= 256) sort_row_warp<8>(col, r0, d, i, out);
        else if (d <= 512) sort_row_warp<16>(col, r0, d, i, out);
        else sort_row_warp<32>(col, r0, d, i, out);
    }
}

// One CTA per row of kRowWarp+1..kRowMid partners (listed from the back of
// `mid`): LSD radix sort in shared memory of the keys v - (i + 1) < n, 8-bit
// digits, as many passes as n needs.  Each pass: every warp counts the digits
// of its contiguous slice, one scan over (digit, warp) gives stable bases,
// then every warp scatters its slice in order, ranking equal digits within a
// round of 32 by one ballot per digit bit.
constexpr int kRadixWarps = kRowThreads / 32;

__global__ void __launch_bounds__(kRowThreads) rows_sort_mid_kernel(const uint32_t *__restrict__ rowoff, int64_t n,
                                                                    const unsigned long long *__restrict__ d_m,
                                                                    const uint32_t *__restrict__ mid,
                                                                    const unsigned long long *__restrict__ d_mid,
                                                                    const uint32_t *__restrict__ col,
                                                                    uint32_t *__restrict__ out)
{
    extern __shared__ uint32_t s_rs[];  // [2][kRowMid] keys, then [kRadixWarps][256] counts
    uint32_t *bufA = s_rs, *bufB = s_rs + kRowMid, *wcnt = s_rs + 2 * kRowMid;
    __shared__ uint32_t s_dtot[256];
    const uint64_t m = *d_m, nmid = *d_mid;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = (1u << lane) - 1u;
    for (uint64_t r = blockIdx.x; r < nmid; r += gridDim.x) {
        const uint32_t i = mid[n - 1 - (int64_t)r];
        const uint64_t r0 = rowoff[i];
        const uint32_t d = (uint32_t)(row_end(rowoff, n, m, i) - r0);
        const uint32_t lo = i + 1;  // every partner is above i
        const uint32_t range = (uint32_t)n - lo;
        const int nbits = range > 1 ? 32 - __clz(range - 1) : 1;
        for (uint32_t t = threadIdx.x; t < d; t += blockDim.x) bufA[t] = col[r0 + t] - lo;
        // warp slices of whole rounds of 32
        const uint32_t slice = ((d + kRadixWarps * 32 - 1) / (kRadixWarps * 32)) * 32;
        const uint32_t s0 = warp * slice, s1 = min(d, s0 + slice);
        for (int shift = 0; shift < nbits; shift += 8) {
            for (uint32_t t = threadIdx.x; t < kRadixWarps * 256; t += blockDim.x) wcnt[t] = 0;
            __syncthreads();
            uint32_t *wc = wcnt + warp * 256;
            for (uint32_t t = s0 + lane; t < s1; t += 32) atomicAdd(&wc[(bufA[t] >> shift) & 255u], 1u);
            __syncthreads();
            {
                // thread = digit: exclusive over warps, then over digits
                const uint32_t dg = threadIdx.x;
                uint32_t run = 0;
#pragma unroll
                for (int w = 0; w < kRadixWarps; ++w) {
                    const uint32_t c = wcnt[w * 256 + dg];
                    wcnt[w * 256 + dg] = run;
                    run += c;
                }
                s_dtot[dg] = run;
                __syncthreads();
                if (warp == 0) {
                    uint32_t carry = 0;
                    for (int base = 0; base < 256; base += 32) {
                        const uint32_t v = s_dtot[base + lane];
                        uint32_t inc = v;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                            if ((int)lane >= o) inc += y;
                        }
                        s_dtot[base + lane] = carry + inc - v;
                        carry += __shfl_sync(0xffffffffu, inc, 31);
                    }
                }
                __syncthreads();
                const uint32_t dbase = s_dtot[dg];
#pragma unroll
                for (int w = 0; w < kRadixWarps; ++w) wcnt[w * 256 + dg] += dbase;
            }
            __syncthreads();
            for (uint32_t t0 = s0; t0 < s1; t0 += 32) {
                const uint32_t t = t0 + lane;
                const bool valid = t < s1;
                const uint32_t key = valid ? bufA[t] : 0u;
                const uint32_t dgt = valid ? (key >> shift) & 255u : 256u;
                uint32_t peers = 0xffffffffu;
#pragma unroll
                for (int bit = 0; bit < 9; ++bit) {
                    const uint32_t mb = __ballot_sync(0xffffffffu, (dgt >> bit) & 1u);
                    peers &= ((dgt >> bit) & 1u) ? mb : ~mb;
                }
                const uint32_t before = __popc(peers & lt);
                const uint32_t base = valid ? wc[dgt] : 0u;
                __syncwarp();
                if (valid && before == 0) wc[dgt] = base + __popc(peers);
                __syncwarp();
                if (valid) bufB[base + before] = key;
            }
            __syncthreads();
            uint32_t *tmp = bufA;
            bufA = bufB;
            bufB = tmp;
        }
        for (uint32_t t = threadIdx.x; t < d; t += blockDim.x)
            reinterpret_cast<uint2 *>(out)[r0 + t] = make_uint2(i, bufA[t] + lo);
        __syncthreads();
    }
}

// One CTA per row of more than kRowMid partners, sorted in place in global
// memory by a bitonic network whose comparators all put the smaller value at
// the lower index (a "flip" step, then half-cleaners), so positions past the
// row's end act as +infinity and are never touched.
__global__ void __launch_bounds__(1024) rows_sort_long_kernel(const uint32_t *__restrict__ rowoff, int64_t n,
                                                              const unsigned long long *__restrict__ d_m,
                                                              const uint32_t *__restrict__ lng,
                                                              const unsigned long long *__restrict__ d_long,
                                                              uint32_t *__restrict__ col, uint32_t *__restrict__ out)
{
    const uint64_t m = *d_m, nl = *d_long;
    for (uint64_t r = blockIdx.x; r < nl; r += gridDim.x) {
        const uint32_t i = lng[r];
        const uint64_t r0 = rowoff[i];
        const uint64_t d = row_end(rowoff, n, m, i) - r0;
        uint32_t *v = col + r0;
        uint64_t P2 = 2;
        while (P2 < d) P2 <<= 1;
        for (uint64_t k = 2; k <= P2; k <<= 1) {
            for (uint64_t j = k >> 1; j > 0; j >>= 1) {
                for (uint64_t t = threadIdx.x; t < P2 / 2; t += blockDim.x) {
                    const uint64_t a = (t / j) * 2 * j + (t % j);
                    const uint64_t b = j == (k >> 1) ? (a | (k - 1)) - (a & (k - 1)) : a + j;  // flip, then half-cleaners
                    if (b < d) {
                        const uint32_t x = v[a], y = v[b];
                        if (x > y) {
                            v[a] = y;
                            v[b] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint64_t t = threadIdx.x; t < d; t += blockDim.x)
            reinterpret_cast<uint2 *>(out)[r0 + t] = make_uint2(i, v[t]);
        __syncthreads();
    }
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
// The chunk structure of one banding (device arrays): per (sequence, band)
// chunk ids and kept-band masks, kept members, the chunk list with its
// scanned pair counts, the start chunk of every 32nd raw pair, and the
// device counts (chunks, raw pairs, kept members).
struct BandIndex {
    int64_t n = 0, mall = 0, cmax = 0, wmax = 0;
    int bands = 0;
    uint32_t *chunk_of, *kept_mask, *kept, *heads, *sizes, *cband, *wchunk;
    uint64_t *poff;
    uint64_t *counters;  // [0] chunks (low word), [1] raw pairs, [2] kept members
};

BandIndex take_index(SqArena &a, int64_t n, int bands)
{
    BandIndex I;
    I.n = n;
    I.bands = bands;
    I.mall = (int64_t)bands * n;
    I.cmax = I.mall / 2 + 1;  // chunks of >= 2 members
    I.wmax = I.mall / 8 + 64;  // start chunks of the first 4 * bands * n raw pairs
    I.chunk_of = a.take<uint32_t>((size_t)n * bands);
    I.kept_mask = a.take<uint32_t>(n);
    I.kept = a.take<uint32_t>(I.mall);
    I.heads = a.take<uint32_t>(I.cmax);
    I.sizes = a.take<uint32_t>(I.cmax);
    I.cband = a.take<uint32_t>(I.cmax);
    I.poff = a.take<uint64_t>(I.cmax);
    I.wchunk = a.take<uint32_t>(I.wmax);
    I.counters = a.take<uint64_t>(4);
    return I;
}

struct GroupScratch {
    int pbits = 0, G = 0;
    int64_t P = 0, ntiles = 0, mg = 0, hlen = 0;
    uint64_t *recs, *fd;
    uint32_t *rslot, *offs;
    void *tmp;
    size_t tmp_bytes = 0;
};

GroupScratch plan_group(subquad_ctx *ctx, int64_t n, int bands)
{
    GroupScratch S;
    // Partitions of at most 2^part_log2 keys on average (the tuning knob;
    // default 2048): P = 2^pbits per band.  Bands are partitioned in groups
    // of at most 2^28 keys (bounding the record buffers); kept members,
    // chunk ids and the chunk list span all bands.
    const int part_log2 = ctx->tune[SUBQUAD_TUNE_BAND_PART_LOG2];
    while ((n >> S.pbits) > (int64_t(1) << part_log2) && S.pbits < kPartMaxBits) ++S.pbits;
    S.P = int64_t(1) << S.pbits;
    S.ntiles = (n + kPartTile - 1) / kPartTile;
    S.G = (int)std::max<int64_t>(1, std::min<int64_t>(bands, (int64_t(1) << 28) / n));
    S.mg = (int64_t)S.G * n;
    S.hlen = (int64_t)S.G * S.P * S.ntiles;
    S.tmp_bytes = std::max(sq_scan_tmp_bytes(S.hlen), sq_scan_tmp_bytes((int64_t)bands * n / 2 + 1));
    return S;
}

void take_group(SqArena &a, GroupScratch &S)
{
    S.recs = a.take<uint64_t>(S.mg);
    S.fd = a.take<uint64_t>(S.mg);
    S.rslot = a.take<uint32_t>(S.mg);
    S.offs = a.take<uint32_t>(S.hlen);
    S.tmp = a.take<char>(S.tmp_bytes);
}

// Steps 1-3: partition, group, chunk list, pair offsets, start chunks.
int band_index_build(subquad_ctx *ctx, const uint32_t *sig, int rows, int cap, const int32_t *donor,
                     const BandIndex &I, const GroupScratch &S)
{
    const int64_t n = I.n;
    const int bands = I.bands;
    uint32_t *d_nchunks = reinterpret_cast<uint32_t *>(I.counters);
    uint64_t *d_total = I.counters + 1;
    unsigned long long *d_kept = reinterpret_cast<unsigned long long *>(I.counters + 2);
    SQ_TRY_CUDA(cudaMemsetAsync(I.counters, 0, 4 * sizeof(uint64_t), ctx->stream));
    // chunk ids of bands below 32 are read only where kept_mask says the
    // member was placed in that band (so written); bands from 32 on are
    // compared without a mask and start as kNoChunk
    if (bands > 32)
        SQ_TRY_CUDA(cudaMemsetAsync(I.chunk_of, 0xff, (size_t)n * bands * sizeof(uint32_t), ctx->stream));
    SQ_TRY_CUDA(cudaMemsetAsync(I.kept_mask, 0, (size_t)n * sizeof(uint32_t), ctx->stream));
    GroupOut go{I.kept, d_kept, d_nchunks, I.heads, I.sizes, I.cband, I.poff, I.chunk_of, I.kept_mask, S.rslot};
    for (int band0 = 0; band0 < bands; band0 += S.G) {
        const int gb = std::min(S.G, bands - band0);
        const int64_t recs = (int64_t)gb * n;
        const int64_t hl = (int64_t)gb * S.P * S.ntiles;
        const dim3 grid((unsigned)S.ntiles, gb);
        {
            SqProfScope prof_ins(ctx, SUBQUAD_PROF_BAND_PARTITION);
            part_hist_kernel<<<grid, kPartThreads, S.P * sizeof(uint32_t), ctx->stream>>>(
                sig, n, rows, band0, S.pbits, donor, S.ntiles, S.offs, S.fd);
            SQ_LAUNCH_CHECK();
            SQ_TRY(sq_scan_u32(ctx, S.offs, S.offs, hl, nullptr, false, false, nullptr, S.tmp, S.tmp_bytes));
            part_scatter_kernel<<<grid, kPartThreads, part_scatter_smem((int)S.P), ctx->stream>>>(
                S.fd, n, S.pbits, S.ntiles, S.offs, S.recs);
            SQ_LAUNCH_CHECK();
        }
        SqProfScope prof_grp(ctx, SUBQUAD_PROF_BAND_GROUP);
        SQ_TRY_CUDA(cudaFuncSetAttribute(part_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGrpSmem));
        part_group_kernel<<<(unsigned)(gb * S.P), kGrpThreads, kGrpSmem, ctx->stream>>>(
            S.recs, S.offs, S.ntiles, recs, S.pbits, band0, bands, sig, n, rows, donor, cap, go, ctx->d_err);
        SQ_LAUNCH_CHECK();
    }
    SqProfScope prof_emit(ctx, SUBQUAD_PROF_BAND_EMIT);
    // pair counts -> offsets, and their sum (the raw pair count) -> d_total.
    // The scan reads the first nchunks entries only (the device count), the
    // ones the grouping wrote.
    SQ_TRY(sq_scan_u64(ctx, I.poff, I.poff, I.cmax, d_nchunks, d_total, S.tmp, S.tmp_bytes));
    band_warp_chunk_kernel<<<(unsigned)ctx->num_sms * 8, 256, 0, ctx->stream>>>(I.poff, d_nchunks, d_total, I.wchunk,
                                                                                I.wmax);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

struct EmitScratch {
    uint32_t *deg, *rowoff, *sa, *sb, *mid, *lng, *col;
    void *tmp;
    size_t tmp_bytes = 0;
};

void take_emit(SqArena &a, EmitScratch &E, int64_t n, int64_t capacity, uint32_t *col_alias, int64_t alias_words)
{
    E.deg = a.take<uint32_t>(n);
    E.rowoff = a.take<uint32_t>(n);
    E.sa = a.take<uint32_t>(n);
    E.sb = a.take<uint32_t>(n);
    E.mid = a.take<uint32_t>(n);
    E.lng = a.take<uint32_t>((capacity >> 13) + 1);
    // row columns: in a free buffer of the caller when it is large enough
    E.col = capacity <= alias_words ? col_alias : a.take<uint32_t>(capacity);
    E.tmp_bytes = sq_scan_tmp_bytes(n);
    E.tmp = a.take<char>(E.tmp_bytes);
}

// Step 4: the owned pairs among raw pairs [raw0, raw1) (raw0 % 32 == 0),
// appended to pairs_out (at most capacity written; d_count receives the
// owned count) and sorted lexicographically.  d_publish, when given, receives
// the owned count with the sticky CAPACITY bit on an overflow.
int band_emit_sorted(subquad_ctx *ctx, const BandIndex &I, uint64_t raw0, uint64_t raw1, uint32_t *pairs_out,
                     int64_t capacity, unsigned long long *d_publish, const EmitScratch &E)
{
    const int64_t n = I.n;
    const int64_t cap1 = std::max<int64_t>(capacity, 1);
    unsigned long long *d_count = reinterpret_cast<unsigned long long *>(ctx->d_small);
    unsigned long long *d_clamped = reinterpret_cast<unsigned long long *>(ctx->d_small + 4);
    unsigned long long *d_cls = reinterpret_cast<unsigned long long *>(ctx->d_small + 8);  // kRowClasses counters
    SQ_TRY_CUDA(cudaMemsetAsync(ctx->d_small, 0, 16 * sizeof(uint64_t), ctx->stream));
    SQ_TRY_CUDA(cudaMemsetAsync(E.deg, 0, (size_t)n * sizeof(uint32_t), ctx->stream));
    {
        SqProfScope prof_emit(ctx, SUBQUAD_PROF_BAND_EMIT);
        band_emit_kernel<<<(unsigned)ctx->num_sms * 8, 256, 0, ctx->stream>>>(
            I.kept, I.heads, I.sizes, I.cband, I.poff, I.wchunk, I.wmax, reinterpret_cast<const uint32_t *>(I.counters),
            I.counters + 1, I.bands, I.chunk_of, I.kept_mask, raw0, raw1, pairs_out, capacity, d_count, E.deg,
            ctx->d_err);
        SQ_LAUNCH_CHECK();
    }
    // lexicographic order: row offsets by first member, the second members
    // scattered into their rows, row class lists, every row sorted
    SqProfScope prof_ps(ctx, SUBQUAD_PROF_BAND_PAIRSORT);
    const unsigned rgrid = sq_grid(ctx, n, kRowThreads, 8);
    SQ_TRY(sq_scan_u32(ctx, E.deg, E.rowoff, n, nullptr, false, false, nullptr, E.tmp, E.tmp_bytes));
    // the scatter also publishes the owned count, flags an overflow and
    // leaves the count of written pairs, clamped to the capacity, for the
    // sort below
    pairs_scatter_kernel<<<sq_grid(ctx, cap1, 256, 8), 256, 0, ctx->stream>>>(
        pairs_out, d_count, capacity, d_publish, d_clamped, ctx->d_err, E.rowoff, E.deg, E.col);
    SQ_LAUNCH_CHECK();
    rows_classify_kernel<<<rgrid, kRowThreads, 0, ctx->stream>>>(E.rowoff, n, d_clamped, E.col, pairs_out, E.sa, E.sb,
                                                                 E.mid, E.lng, d_cls);
    SQ_LAUNCH_CHECK();
    // the classes are sorted concurrently (disjoint rows): the CTA radix and
    // in-place sorts on the context stream, the register and warp sorts on
    // the side stream, which fill the SMs around the radix CTAs
    SQ_TRY_CUDA(cudaEventRecord(ctx->fork, ctx->stream));
    SQ_TRY_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork, 0));
    constexpr size_t kRadixSmem = (2 * (size_t)kRowMid + (size_t)kRadixWarps * 256) * sizeof(uint32_t);
    SQ_TRY_CUDA(cudaFuncSetAttribute(rows_sort_mid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRadixSmem));
    rows_sort_mid_kernel<<<(unsigned)ctx->num_sms * 3, kRowThreads, kRadixSmem, ctx->stream>>>(
        E.rowoff, n, d_clamped, E.mid, d_cls + kClsCta, E.col, pairs_out);
    SQ_LAUNCH_CHECK();
    rows_sort_small_kernel<<<rgrid, kRowThreads, 0, ctx->side>>>(E.rowoff, n, d_clamped, E.sa, E.sb, d_cls, E.col,
                                                                 pairs_out);
    SQ_LAUNCH_CHECK();
    rows_sort_warp_kernel<<<(unsigned)ctx->num_sms * 8, kRowThreads, 0, ctx->side>>>(
        E.rowoff, n, d_clamped, E.mid, d_cls + kClsWarp, E.col, pairs_out);
    SQ_LAUNCH_CHECK();
    rows_sort_long_kernel<<<(unsigned)ctx->num_sms, 1024, 0, ctx->stream>>>(E.rowoff, n, d_clamped, E.lng, d_cls + kClsLong,
                                                                           E.col, pairs_out);
    SQ_LAUNCH_CHECK();
    SQ_TRY_CUDA(cudaEventRecord(ctx->join, ctx->side));
    SQ_TRY_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->join, 0));
    return SUBQUAD_OK;
}

// Synchronous form (d_num_pairs == nullptr): reads back |C| once at the end.
// Asynchronous form: no host synchronisation -- |C| goes to *d_num_pairs and
// an overflow of the capacity sets the sticky CAPACITY error -- so the call
// can be captured in a graph once a call of the same shape has reserved the
// scratch.
int band_run(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows, int32_t bucket_cap,
             const int32_t *donor, uint32_t *pairs_out, int64_t pairs_capacity, int64_t *num_pairs_out,
             unsigned long long *d_num_pairs)
{
    const bool async = d_num_pairs != nullptr;
    const int cap = (bucket_cap <= 0 || bucket_cap >= n) ? 0 : bucket_cap;
    SqProfScope prof(ctx, SUBQUAD_PROF_BAND);
    GroupScratch S = plan_group(ctx, n, bands);
    const int64_t cap1 = std::max<int64_t>(pairs_capacity, 1);
    auto layout = [&](SqArena &a, BandIndex &I, EmitScratch &E) {
        I = take_index(a, n, bands);
        take_group(a, S);
        // the record buffer is free after the grouping: it holds the row columns when large enough
        take_emit(a, E, n, cap1, reinterpret_cast<uint32_t *>(S.recs), 2 * S.mg);
    };
    BandIndex I;
    EmitScratch E;
    {
        SqArena measure(nullptr);
        layout(measure, I, E);
        SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    }
    SqArena arena(ctx->scratch);
    layout(arena, I, E);
    SQ_TRY(band_index_build(ctx, sig, rows, cap, donor, I, S));
    SQ_TRY(band_emit_sorted(ctx, I, 0, ~0ull, pairs_out, pairs_capacity, async ? d_num_pairs : nullptr, E));
    if (async) return SUBQUAD_OK;
    SQ_TRY_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_small, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_TRY_CUDA(cudaMemcpyAsync(ctx->h_pinned + 1, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    const int64_t count = (int64_t)ctx->h_pinned[0];
    const uint32_t err = (uint32_t)(ctx->h_pinned[1] & 0xffffffffu);
    *num_pairs_out = count;
    if (err) return subquad_check(ctx);
    if (count > pairs_capacity) return SUBQUAD_ERR_CAPACITY;  // the status reports it (no sticky bit)
    return SUBQUAD_OK;
}

int band_args(int64_t n, int bands, int rows, int64_t pairs_capacity, const uint32_t *sig, const uint32_t *pairs_out)
{
    if (n < 0 || n >= (int64_t(1) << 31) || bands < 1 || rows < 1 || rows > 8 || bands * rows > 512 ||
        pairs_capacity < 0 || pairs_capacity >= (int64_t)0xffffffffLL || (int64_t)bands * n >= (int64_t)0xffffffffLL)
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

// ---------------------------------------------------------------------------
// Streamed candidates: the chunk structure is built once and kept in the
// stream's own device memory; every call emits, in lexicographic order, the
// owned pairs among the next block of raw pairs (at most `capacity` of them,
// so the batch always fits).  Ownership is decided against all bands, so the
// batches partition C: every pair of C comes out exactly once.
// ---------------------------------------------------------------------------
struct subquad_band_stream {
    int device = 0;
    void *mem = nullptr;
    BandIndex index;
    uint64_t next = 0, total = 0;
};

extern "C" int subquad_band_stream_create(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows,
                                          int32_t bucket_cap, const int32_t *donor, subquad_band_stream **out,
                                          uint64_t *total_raw_out)
{
    SQ_ENTER(ctx);
    if (!out) return SUBQUAD_ERR_ARG;
    *out = nullptr;
    if (total_raw_out) *total_raw_out = 0;
    SQ_TRY(band_args(n, bands, rows, 0, sig, nullptr));
    auto *st = new (std::nothrow) subquad_band_stream;
    if (!st) return SUBQUAD_ERR_NOMEM;
    st->device = ctx->device;
    if (n >= 2) {
        SqArena m(nullptr);
        take_index(m, n, bands);
        if (cudaMalloc(&st->mem, m.off) != cudaSuccess) {
            cudaGetLastError();
            delete st;
            return SUBQUAD_ERR_NOMEM;
        }
        SqArena a(st->mem);
        st->index = take_index(a, n, bands);
        GroupScratch S = plan_group(ctx, n, bands);
        {
            SqArena measure(nullptr);
            take_group(measure, S);
            const int rc = sq_scratch_reserve(ctx, measure.off);
            if (rc != SUBQUAD_OK) {
                cudaFree(st->mem);
                delete st;
                return rc;
            }
        }
        SqArena arena(ctx->scratch);
        take_group(arena, S);
        const int cap = (bucket_cap <= 0 || bucket_cap >= n) ? 0 : bucket_cap;
        int rc = band_index_build(ctx, sig, rows, cap, donor, st->index, S);
        uint64_t total = 0;
        if (rc == SUBQUAD_OK) {
            // (subquad_check reuses the first staging word: read the total first)
            rc = cudaMemcpyAsync(ctx->h_pinned + 2, st->index.counters + 1, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                 ctx->stream) == cudaSuccess &&
                         cudaStreamSynchronize(ctx->stream) == cudaSuccess
                     ? SUBQUAD_OK
                     : SUBQUAD_ERR_CUDA;
            total = ctx->h_pinned[2];
            if (rc == SUBQUAD_OK) rc = subquad_check(ctx);
        }
        if (rc != SUBQUAD_OK) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(st->mem);
            delete st;
            return rc;
        }
        st->total = total;
    }
    if (total_raw_out) *total_raw_out = st->total;
    *out = st;
    return SUBQUAD_OK;
}

extern "C" int subquad_band_stream_next(subquad_ctx *ctx, subquad_band_stream *st, uint32_t *pairs_out,
                                        int64_t capacity, int64_t *num_pairs_out, int *done)
{
    SQ_ENTER(ctx);
    if (!st || !num_pairs_out || !done) return SUBQUAD_ERR_ARG;
    *num_pairs_out = 0;
    *done = 0;
    if (st->device != ctx->device || capacity < 32 || capacity >= (int64_t)0xffffffffLL || !pairs_out ||
        reinterpret_cast<uintptr_t>(pairs_out) % 8)
        return SUBQUAD_ERR_ARG;
    if (st->next >= st->total) {
        *done = 1;
        return SUBQUAD_OK;
    }
    const uint64_t batch = (uint64_t)capacity & ~31ull;  // owned <= raw: the batch fits
    const BandIndex &I = st->index;
    EmitScratch E;
    {
        SqArena measure(nullptr);
        take_emit(measure, E, I.n, capacity, nullptr, 0);
        SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    }
    SqArena arena(ctx->scratch);
    take_emit(arena, E, I.n, capacity, nullptr, 0);
    SQ_TRY(band_emit_sorted(ctx, I, st->next, st->next + batch, pairs_out, capacity, nullptr, E));
    SQ_TRY_CUDA(
        cudaMemcpyAsync(ctx->h_pinned + 2, ctx->d_small, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    const int64_t count = (int64_t)ctx->h_pinned[2];  // read before subquad_check reuses the staging words
    SQ_TRY(subquad_check(ctx));
    *num_pairs_out = count;
    st->next += batch;
    *done = st->next >= st->total ? 1 : 0;
    return SUBQUAD_OK;
}

extern "C" int subquad_band_stream_reset(subquad_band_stream *st)
{
    if (!st) return SUBQUAD_ERR_ARG;
    st->next = 0;
    return SUBQUAD_OK;
}

extern "C" void subquad_band_stream_destroy(subquad_band_stream *st)
{
    if (!st) return;
    if (st->mem) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(st->device);
        cudaFree(st->mem);
        if (prev >= 0) cudaSetDevice(prev);
    }
    delete st;
}
