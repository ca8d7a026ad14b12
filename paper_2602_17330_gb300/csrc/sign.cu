// (a1) MinHash signatures over amino-acid k-mers (Algorithm 1, preprocessing).
//
// One thread per sequence.  The k-mer values of the sequence are held in
// registers (a compile-time count NK, chosen per warp as the warp's largest
// k-mer count rounded up to 4; lanes with fewer k-mers repeat their first one,
// which leaves the minimum unchanged).  For each hash t the thread evaluates
// (a_t x + b_t) mod (2^31 - 1) exactly with one 32x32->64 multiply-add and a
// Mersenne fold, keeps the running minimum, and stores each band's R minima as
// one vector store into the band-major output sig[b][i][r].
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr uint32_t kP31 = 0x7fffffffu;

// min(best, (a*x + b) mod P) for x < 20^6, given a2 = 2a and b2 = 2b with
// a, b < P.  w = a2*x + b2 = 2v for v = a*x + b < 2^57, so the high word of w
// is v >> 31 and the low word shifted right by one is v mod 2^31; their sum
// r < P + 2^26 < 2P, so one conditional subtract finishes the reduction, and
// min3 over (r, r - P) picks it (r - P wraps above r when r < P).
// The low word's shift is formed as the high half of a multiply by 2^31 and
// r - P as a multiply-add by the runtime constant unit (= 1), so both run on
// the FMA pipe beside the minima on the ALU pipe.
__device__ __forceinline__ uint32_t hash_min(uint32_t best, uint32_t a2, uint32_t b2, uint32_t x, uint32_t unit)
{
    const uint64_t w = (uint64_t)a2 * x + b2;
    const uint32_t r = __umulhi((uint32_t)w, 0x80000000u) + (uint32_t)(w >> 32);
    return min(best, min(r, r * unit - kP31));
}

template <int WORDS, int NK>
__device__ __forceinline__ void sign_one(const uint64_t *__restrict__ w, int L, int k, int64_t i, int64_t n,
                                         int bands, int rows, const uint2 *__restrict__ s_ab,
                                         uint32_t *__restrict__ sig, uint32_t unit)
{
    constexpr int MAXLEN = WORDS == 2 ? 24 : 30;
    uint32_t c[MAXLEN];
#pragma unroll
    for (int p = 0; p < MAXLEN; ++p) c[p] = (uint32_t)(w[p / 12] >> (5 * (p % 12))) & 31u;
    const int nk = L - k + 1;
    uint32_t x[NK];
#pragma unroll
    for (int p = 0; p < NK; ++p) {
        uint32_t v = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            uint32_t cm = (p + m < MAXLEN) ? c[(p + m < MAXLEN) ? p + m : 0] : 0u;
            v = (m < k) ? v * 20u + cm : v;
        }
        x[p] = v;
    }
#pragma unroll
    for (int p = 1; p < NK; ++p) x[p] = (p < nk) ? x[p] : x[0];
    for (int bnd = 0; bnd < bands; ++bnd) {
        uint32_t out[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            out[r] = 0xffffffffu;
            if (r < rows) {
                uint2 ab = s_ab[bnd * rows + r];
                uint32_t best = 0xffffffffu;
#pragma unroll
                for (int p = 0; p < NK; ++p) best = hash_min(best, ab.x, ab.y, x[p], unit);
                out[r] = nk > 0 ? best : 0xffffffffu;
            }
        }
        uint32_t *dst = sig + ((int64_t)bnd * n + i) * rows;
        if (rows == 4) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(out[0], out[1], out[2], out[3]);
        } else if (rows == 2) {
            *reinterpret_cast<uint2 *>(dst) = make_uint2(out[0], out[1]);
        } else {
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (r < rows) dst[r] = out[r];
        }
    }
}

// One CTA handles tiles of kSignTile consecutive sequences: it counting-sorts
// the tile by k-mer count in shared memory, so each warp takes 32 sequences
// of (nearly) equal count and the per-warp k-mer count NK wastes almost no
// evaluations; signatures are written back at the sequences' own ids (a tile
// covers one contiguous id range).
constexpr int kSignThreads = 256;
constexpr int kSignPer = 1;
constexpr int kSignTile = kSignThreads * kSignPer;

template <int WORDS>
__global__ void __launch_bounds__(kSignThreads) sign_kernel(const uint64_t *__restrict__ packed, int64_t n, int k,
                                                            int bands, int rows, const uint32_t *__restrict__ a,
                                                            const uint32_t *__restrict__ b, uint32_t *__restrict__ sig)
{
    extern __shared__ uint2 s_ab[];
    __shared__ uint32_t s_cnt[32];
    __shared__ uint16_t s_order[kSignTile];
    const int H = bands * rows;
    // coefficients reduced mod P (same hash) and doubled for hash_min
    for (int t = threadIdx.x; t < H; t += blockDim.x) s_ab[t] = make_uint2(2u * (a[t] % kP31), 2u * (b[t] % kP31));
    for (int64_t base = (int64_t)blockIdx.x * kSignTile; base < n; base += (int64_t)gridDim.x * kSignTile) {
        if (threadIdx.x < 32) s_cnt[threadIdx.x] = 0;
        __syncthreads();
        uint32_t bin[kSignPer];
#pragma unroll
        for (int r = 0; r < kSignPer; ++r) {
            const int64_t i = base + r * kSignThreads + threadIdx.x;
            bin[r] = 31;  // past the end: sorted last
            if (i < n) {
                const ulonglong2 w01 = reinterpret_cast<const ulonglong2 *>(packed + i * WORDS)[0];
                bin[r] = (uint32_t)max(sq_record_len(w01.x, w01.y) - k + 1, 0);
            }
            atomicAdd(&s_cnt[bin[r]], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const uint32_t c = s_cnt[threadIdx.x];
            uint32_t inc = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
                if ((int)threadIdx.x >= d) inc += o;
            }
            s_cnt[threadIdx.x] = inc - c;  // exclusive
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSignPer; ++r) s_order[atomicAdd(&s_cnt[bin[r]], 1u)] = (uint16_t)(r * kSignThreads + threadIdx.x);
        __syncthreads();
#pragma unroll 1
        for (int r = 0; r < kSignPer; ++r) {
            const int64_t i = base + s_order[r * kSignThreads + threadIdx.x];
            const bool valid = i < n;
            uint64_t w[WORDS];
#pragma unroll
            for (int q = 0; q < WORDS; ++q) w[q] = 0;
            if (valid) {
                const ulonglong2 *rec = reinterpret_cast<const ulonglong2 *>(packed + i * WORDS);
                const ulonglong2 r0 = rec[0];
                w[0] = r0.x;
                w[1] = r0.y;
                if (WORDS == 4) {
                    const ulonglong2 r1 = rec[1];
                    w[2 % WORDS] = r1.x;
                    w[3 % WORDS] = r1.y;
                }
            }
            const int L = sq_record_len(w[0], w[1]);
            const int nk = valid ? L - k + 1 : 0;
            const int wmax = __reduce_max_sync(0xffffffffu, nk > 0 ? nk : 0);
            const uint32_t unit = blockDim.x / kSignThreads;  // 1: the kernel is launched with kSignThreads
            if (valid) {
                if (wmax <= 4) sign_one<WORDS, 4>(w, L, k, i, n, bands, rows, s_ab, sig, unit);
                else if (wmax <= 8) sign_one<WORDS, 8>(w, L, k, i, n, bands, rows, s_ab, sig, unit);
                else if (wmax <= 12) sign_one<WORDS, 12>(w, L, k, i, n, bands, rows, s_ab, sig, unit);
                else if (wmax <= 16) sign_one<WORDS, 16>(w, L, k, i, n, bands, rows, s_ab, sig, unit);
                else if (wmax <= 20) sign_one<WORDS, 20>(w, L, k, i, n, bands, rows, s_ab, sig, unit);
                else if (wmax <= 24) sign_one<WORDS, 24>(w, L, k, i, n, bands, rows, s_ab, sig, unit);
                else sign_one<WORDS, (WORDS == 2 ? 24 : 30)>(w, L, k, i, n, bands, rows, s_ab, sig, unit);
            }
        }
        __syncthreads();  // s_order and s_cnt are reused by the next tile
    }
}

}  // namespace

extern "C" int subquad_sign(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n, int k, int bands,
                            int rows, const uint32_t *a, const uint32_t *b, uint32_t *sig_out)
{
    SQ_ENTER(ctx);
    if (n < 0 || k < 1 || k > 6 || bands < 1 || rows < 1 || rows > 8 || bands * rows > 512) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (n == 0) return SUBQUAD_OK;
    if (!packed || !a || !b || !sig_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed) % 16 || reinterpret_cast<uintptr_t>(sig_out) % 16) return SUBQUAD_ERR_ARG;
    const size_t smem = (size_t)bands * rows * sizeof(uint2);
    unsigned grid = (unsigned)std::min<int64_t>((n + kSignTile - 1) / kSignTile, int64_t(1) << 30);
    SqProfScope prof(ctx, SUBQUAD_PROF_SIGN);
    if (pack_stride == 16)
        sign_kernel<2><<<grid, kSignThreads, smem, ctx->stream>>>((const uint64_t *)packed, n, k, bands, rows, a, b, sig_out);
    else
        sign_kernel<4><<<grid, kSignThreads, smem, ctx->stream>>>((const uint64_t *)packed, n, k, bands, rows, a, b, sig_out);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}
