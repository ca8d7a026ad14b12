// Context, scoring matrix, error reporting and sequence packing.
#include <stdlib.h>
#include <string.h>

#include <new>

#include <algorithm>

#include "internal.cuh"

static thread_local cudaError_t g_last_cuda = cudaSuccess;

void sq_note_cuda_error(cudaError_t e) { g_last_cuda = e; }

// BLOSUM62 (Henikoff & Henikoff 1992), typed here in the alphabetical code
// order ACDEFGHIKLMNPQRSTVWY, row = first residue.
static const int8_t kBlosum62[20][20] = {
    //  A   C   D   E   F   G   H   I   K   L   M   N   P   Q   R   S   T   V   W   Y
    {4, 0, -2, -1, -2, 0, -2, -1, -1, -1, -1, -2, -1, -1, -1, 1, 0, 0, -3, -2},           // A
    {0, 9, -3, -4, -2, -3, -3, -1, -3, -1, -1, -3, -3, -3, -3, -1, -1, -1, -2, -2},       // C
    {-2, -3, 6, 2, -3, -1, -1, -3, -1, -4, -3, 1, -1, 0, -2, 0, -1, -3, -4, -3},          // D
    {-1, -4, 2, 5, -3, -2, 0, -3, 1, -3, -2, 0, -1, 2, 0, 0, -1, -2, -3, -2},             // E
    {-2, -2, -3, -3, 6, -3, -1, 0, -3, 0, 0, -3, -4, -3, -3, -2, -2, -1, 1, 3},           // F
    {0, -3, -1, -2, -3, 6, -2, -4, -2, -4, -3, 0, -2, -2, -2, 0, -2, -3, -2, -3},         // G
    {-2, -3, -1, 0, -1, -2, 8, -3, -1, -3, -2, 1, -2, 0, 0, -1, -2, -3, -2, 2},           // H
    {-1, -1, -3, -3, 0, -4, -3, 4, -3, 2, 1, -3, -3, -3, -3, -2, -1, 3, -3, -1},          // I
    {-1, -3, -1, 1, -3, -2, -1, -3, 5, -2, -1, 0, -1, 1, 2, 0, -1, -2, -3, -2},           // K
    {-1, -1, -4, -3, 0, -4, -3, 2, -2, 4, 2, -3, -3, -2, -2, -2, -1, 1, -2, -1},          // L
    {-1, -1, -3, -2, 0, -3, -2, 1, -1, 2, 5, -2, -2, 0, -1, -1, -1, 1, -1, -1},           // M
    {-2, -3, 1, 0, -3, 0, 1, -3, 0, -3, -2, 6, -2, 0, 0, 1, 0, -3, -4, -2},               // N
    {-1, -3, -1, -1, -4, -2, -2, -3, -1, -3, -2, -2, 7, -1, -2, -1, -1, -2, -4, -3},      // P
    {-1, -3, 0, 2, -3, -2, 0, -3, 1, -2, 0, 0, -1, 5, 1, 0, -1, -2, -2, -1},              // Q
    {-1, -3, -2, 0, -3, -2, 0, -3, 2, -2, -1, 0, -2, 1, 5, -1, -1, -3, -3, -2},           // R
    {1, -1, 0, 0, -2, 0, -1, -2, 0, -2, -1, 1, -1, 0, -1, 4, 1, -2, -3, -2},              // S
    {0, -1, -1, -1, -2, -2, -2, -1, -1, -1, -1, 0, -1, -1, -1, 1, 5, 0, -2, -2},          // T
    {0, -1, -3, -2, -1, -3, -3, 3, -2, 1, 1, -3, -2, -2, -3, -2, 0, 4, -3, -1},           // V
    {-3, -2, -4, -3, 1, -2, -2, -3, -3, -2, -1, -4, -4, -2, -3, -3, -2, -3, 11, 2},       // W
    {-2, -2, -3, -2, 3, -3, 2, -1, -2, -1, -1, -2, -3, -1, -2, -2, -2, -1, 2, 7},         // Y
};

extern "C" const char *subquad_strerror(int status)
{
    switch (status) {
    case SUBQUAD_OK: return "ok";
    case SUBQUAD_ERR_ARG: return "invalid argument";
    case SUBQUAD_ERR_CAPACITY: return "output capacity too small";
    case SUBQUAD_ERR_CUDA: return g_last_cuda != cudaSuccess ? cudaGetErrorString(g_last_cuda) : "CUDA error";
    case SUBQUAD_ERR_TIMEOUT: return "device loop exceeded its iteration bound";
    case SUBQUAD_ERR_NOMEM: return "scratch allocation failed";
    case SUBQUAD_ERR_INPUT: return "invalid input data (residue code or length)";
    case SUBQUAD_ERR_INTERNAL: return "internal consistency check failed in a kernel";
    default: return "unknown status";
    }
}

extern "C" int subquad_version(void) { return 100; }

extern "C" int subquad_default_matrix(int8_t *out)
{
    if (!out) return SUBQUAD_ERR_ARG;
    memcpy(out, kBlosum62, sizeof(kBlosum62));
    return SUBQUAD_OK;
}

extern "C" int subquad_create(subquad_ctx **out, int device, void *cuda_stream)
{
    if (!out) return SUBQUAD_ERR_ARG;
    *out = nullptr;
    int count = 0;
    SQ_TRY_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return SUBQUAD_ERR_ARG;
    subquad_ctx *ctx = new (std::nothrow) subquad_ctx();
    if (!ctx) return SUBQUAD_ERR_NOMEM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    memcpy(ctx->h_matrix, kBlosum62, sizeof(kBlosum62));
    sq_update_matrix_flags(ctx);
    sq_default_edit_costs(ctx->h_edit_sub);
    ctx->edit_indel = 2;
    for (int k = 0; k < SUBQUAD_TUNE_COUNT; ++k) ctx->tune[k] = 0;
    ctx->tune[SUBQUAD_TUNE_ALIGN_SHAPE] = 2;
    ctx->tune[SUBQUAD_TUNE_BAND_PART_LOG2] = 11;
    ctx->tune[SUBQUAD_TUNE_FUSE_LANES] = 4;
    SqDeviceGuard guard(ctx);
    cudaError_t e = guard.ok ? cudaSuccess : cudaErrorInvalidDevice;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, 256);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_small, 16 * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, 8 * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err, 0, 256, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        sq_note_cuda_error(e);
        subquad_destroy(ctx);
        return SUBQUAD_ERR_CUDA;
    }
    *out = ctx;
    return SUBQUAD_OK;
}

cudaEvent_t sq_prof_event(subquad_ctx *ctx)
{
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

static void prof_recycle(subquad_ctx *ctx)
{
    for (auto &r : ctx->prof_records) {
        ctx->prof_pool.push_back(r.start);
        ctx->prof_pool.push_back(r.stop);
    }
    ctx->prof_records.clear();
}

extern "C" int subquad_profile_enable(subquad_ctx *ctx, int on)
{
    SQ_ENTER(ctx);
    ctx->prof_on = on != 0;
    return SUBQUAD_OK;
}

extern "C" int subquad_profile_reset(subquad_ctx *ctx)
{
    SQ_ENTER(ctx);
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    prof_recycle(ctx);
    return SUBQUAD_OK;
}

extern "C" int subquad_profile_read(subquad_ctx *ctx, int kernel, double *total_ms, int64_t *launches)
{
    SQ_ENTER(ctx);
    if (!total_ms || !launches || kernel < 0 || kernel >= SUBQUAD_PROF_COUNT) return SUBQUAD_ERR_ARG;
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    double t = 0.0;
    int64_t c = 0;
    for (auto &r : ctx->prof_records) {
        if (r.kernel != kernel) continue;
        float ms = 0.f;
        SQ_TRY_CUDA(cudaEventElapsedTime(&ms, r.start, r.stop));
        t += ms;
        ++c;
    }
    *total_ms = t;
    *launches = c;
    return SUBQUAD_OK;
}

extern "C" int subquad_destroy(subquad_ctx *ctx)
{
    if (!ctx) return SUBQUAD_OK;
    {
        SqDeviceGuard guard(ctx);
        if (guard.ok) {
            cudaStreamSynchronize(ctx->stream);
            prof_recycle(ctx);
            for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
            ctx->prof_pool.clear();
            cudaFree(ctx->scratch);
            cudaFree(ctx->d_table);
            cudaFree(ctx->d_edit_table);
            cudaFree(ctx->d_err);
            cudaFree(ctx->d_small);
            cudaFreeHost(ctx->h_pinned);
            if (ctx->side) {
                cudaStreamSynchronize(ctx->side);
                cudaStreamDestroy(ctx->side);
            }
            if (ctx->fork) cudaEventDestroy(ctx->fork);
            if (ctx->join) cudaEventDestroy(ctx->join);
        }
    }
    delete ctx;
    return SUBQUAD_OK;
}

extern "C" int subquad_set_stream(subquad_ctx *ctx, void *cuda_stream)
{
    SQ_ENTER(ctx);
    // scratch is reused in stream order: finish the old stream's work first
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return SUBQUAD_OK;
}

extern "C" int subquad_check(subquad_ctx *ctx)
{
    SQ_ENTER(ctx);
    SQ_TRY_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    uint32_t err = (uint32_t)(ctx->h_pinned[0] & 0xffffffffu);
    SQ_TRY_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream));
    if (err & SQ_DEVERR_INPUT) return SUBQUAD_ERR_INPUT;
    if (err & SQ_DEVERR_TIMEOUT) return SUBQUAD_ERR_TIMEOUT;
    if (err & SQ_DEVERR_INTERNAL) return SUBQUAD_ERR_INTERNAL;
    if (err & SQ_DEVERR_CAPACITY) return SUBQUAD_ERR_CAPACITY;
    return SUBQUAD_OK;
}

extern "C" int64_t subquad_scratch_bytes(const subquad_ctx *ctx) { return ctx ? (int64_t)ctx->scratch_cap : -1; }

extern "C" int64_t subquad_launch_count(const subquad_ctx *ctx) { return ctx ? ctx->launches : -1; }

int sq_scratch_reserve(subquad_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->scratch_cap) return SUBQUAD_OK;
    size_t want = bytes + bytes / 4 + (1u << 20);
    // in-flight work on this stream may still use the old block
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SUBQUAD_ERR_NOMEM;
    }
    ctx->scratch_cap = want;
    return SUBQUAD_OK;
}

extern "C" int subquad_set_tuning(subquad_ctx *ctx, int key, int value)
{
    if (!ctx || key < 0 || key >= SUBQUAD_TUNE_COUNT) return SUBQUAD_ERR_ARG;
    if (key == SUBQUAD_TUNE_ALIGN_SHAPE && (value < 0 || value > 2)) return SUBQUAD_ERR_ARG;
    if (key == SUBQUAD_TUNE_BAND_PART_LOG2 && (value < 6 || value > 16)) return SUBQUAD_ERR_ARG;
    if (key == SUBQUAD_TUNE_FUSE_LANES && value != 4 && value != 8) return SUBQUAD_ERR_ARG;
    ctx->tune[key] = value;
    return SUBQUAD_OK;
}

extern "C" int subquad_get_tuning(const subquad_ctx *ctx, int key, int *value)
{
    if (!ctx || !value || key < 0 || key >= SUBQUAD_TUNE_COUNT) return SUBQUAD_ERR_ARG;
    *value = ctx->tune[key];
    return SUBQUAD_OK;
}

extern "C" int subquad_set_matrix(subquad_ctx *ctx, const int8_t *matrix)
{
    SQ_ENTER(ctx);
    const int8_t *src = matrix ? matrix : &kBlosum62[0][0];
    for (int k = 0; k < 400; ++k)
        if (src[k] < -64 || src[k] > 63) return SUBQUAD_ERR_ARG;
    memcpy(ctx->h_matrix, src, 400);
    sq_update_matrix_flags(ctx);
    ctx->table_gap_open = -1;  // rebuild the device table on next use
    return SUBQUAD_OK;
}

void sq_default_edit_costs(uint8_t *out)
{
    for (int a = 0; a < 20; ++a)
        for (int b = 0; b < 20; ++b) out[20 * a + b] = (uint8_t)(a == b ? 0 : (kBlosum62[a][b] > 0 ? 1 : 2));
}

extern "C" int subquad_default_edit_costs(uint8_t *out)
{
    if (!out) return SUBQUAD_ERR_ARG;
    sq_default_edit_costs(out);
    return SUBQUAD_OK;
}

extern "C" int subquad_set_edit_costs(subquad_ctx *ctx, int indel, const uint8_t *sub)
{
    SQ_ENTER(ctx);
    if (indel < 0 || indel > 255) return SUBQUAD_ERR_ARG;
    uint8_t costs[400];
    if (sub) memcpy(costs, sub, 400);
    else sq_default_edit_costs(costs);
    for (int a = 0; a < 20; ++a) {
        if (costs[21 * a] != 0) return SUBQUAD_ERR_ARG;
        for (int b = 0; b < 20; ++b)
            if (costs[20 * a + b] != costs[20 * b + a]) return SUBQUAD_ERR_ARG;
    }
    memcpy(ctx->h_edit_sub, costs, 400);
    ctx->edit_indel = indel;
    ctx->edit_table_valid = false;
    return SUBQUAD_OK;
}

void sq_update_matrix_flags(subquad_ctx *ctx)
{
    const int8_t *m = ctx->h_matrix;
    bool sym = true, diag = true;
    for (int a = 0; a < 20; ++a) {
        diag = diag && m[21 * a] > 0;
        for (int b = 0; b < 20; ++b) {
            sym = sym && m[20 * a + b] == m[20 * b + a];
            diag = diag && 2 * (int)m[20 * a + b] <= (int)m[21 * a] + (int)m[21 * b];
        }
    }
    ctx->matrix_symmetric = sym;
    ctx->self_is_diagonal = diag;
}

extern "C" int subquad_pack_stride(int max_len)
{
    if (max_len >= 1 && max_len <= 24) return 16;
    if (max_len >= 1 && max_len <= 30) return 32;
    return 0;
}

// One thread per sequence: validate, then write 2 or 4 little-endian 64-bit
// words with 12 five-bit residues each and the length split over the top
// nibbles of words 0 and 1.
template <int WORDS>
__global__ void pack_kernel(const uint8_t *__restrict__ codes, int code_stride, const uint8_t *__restrict__ lens,
                            int64_t n, uint64_t *__restrict__ out, uint32_t *err)
{
    const int max_len = WORDS == 2 ? 24 : 30;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int L = lens[i];
        bool bad = L < 1 || L > max_len || L > code_stride;
        uint64_t w[WORDS];
#pragma unroll
        for (int k = 0; k < WORDS; ++k) w[k] = 0;
        const uint8_t *row = codes + i * (int64_t)code_stride;
        for (int p = 0; p < L && p < max_len && p < code_stride; ++p) {
            uint32_t c = row[p];
            bad |= c >= 20u;
            uint64_t v = (uint64_t)(c & 31u) << (5 * (p % 12));
#pragma unroll
            for (int k = 0; k < WORDS; ++k)
                if (p / 12 == k) w[k] |= v;
        }
        if (bad) {
            atomicOr(err, SQ_DEVERR_INPUT);
#pragma unroll
            for (int k = 0; k < WORDS; ++k) w[k] = 0;
            L = 0;
        }
        w[0] |= (uint64_t)(L & 15) << 60;
        w[1] |= (uint64_t)(L >> 4) << 60;
        uint64_t *dst = out + i * WORDS;
        if (WORDS == 2) {
            reinterpret_cast<ulonglong2 *>(dst)[0] = make_ulonglong2(w[0], w[1]);
        } else {
            reinterpret_cast<ulonglong2 *>(dst)[0] = make_ulonglong2(w[0], w[1]);
            reinterpret_cast<ulonglong2 *>(dst)[1] = make_ulonglong2(w[2 % WORDS], w[3 % WORDS]);
        }
    }
}

// The same packing for code rows of a multiple of 4 bytes (codes 4-byte
// aligned): each block stages its 256 rows with coalesced 32-bit loads into
// shared memory (row pitch of an odd number of words, so the per-thread row
// reads hit distinct banks), then every thread packs its row from there.
constexpr int kPackRows = 256;
constexpr int kPackMaxStrideWords = 16;  // code rows of up to 64 bytes take the staged path

template <int WORDS>
__global__ void __launch_bounds__(kPackRows) pack_staged_kernel(const uint32_t *__restrict__ codes, int stride_words,
                                                                const uint8_t *__restrict__ lens, int64_t n,
                                                                uint64_t *__restrict__ out, uint32_t *err)
{
    __shared__ uint32_t s_rows[kPackRows * (kPackMaxStrideWords + 1)];
    const int max_len = WORDS == 2 ? 24 : 30;
    const int pitch = stride_words | 1;  // odd
    for (int64_t r0 = (int64_t)blockIdx.x * kPackRows; r0 < n; r0 += (int64_t)gridDim.x * kPackRows) {
        const int rows = (int)(n - r0 < kPackRows ? n - r0 : kPackRows);
        const uint32_t *src = codes + r0 * stride_words;
        const int words = rows * stride_words;
        if ((stride_words & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            // 16-byte loads (a multiple of 4 words per row keeps them inside one row)
            for (int w = 4 * threadIdx.x; w < words; w += 4 * blockDim.x) {
                const uint4 v = *reinterpret_cast<const uint4 *>(src + w);
                const int row = w / stride_words, col = w - row * stride_words;
                uint32_t *d = s_rows + row * pitch + col;
                d[0] = v.x;
                d[1] = v.y;
                d[2] = v.z;
                d[3] = v.w;
            }
        } else {
            for (int w = threadIdx.x; w < words; w += blockDim.x) {
                const int row = w / stride_words, col = w - row * stride_words;
                s_rows[row * pitch + col] = src[w];
            }
        }
        __syncthreads();
        const int t = threadIdx.x;
        if (t < rows) {
            const int64_t i = r0 + t;
            int L = lens[i];
            bool bad = L < 1 || L > max_len || L > 4 * stride_words;
            uint64_t w[WORDS];
#pragma unroll
            for (int k = 0; k < WORDS; ++k) w[k] = 0;
            const uint32_t *row = s_rows + t * pitch;
            const int Lc = min(min(L, max_len), 4 * stride_words);
            for (int q = 0; q * 4 < Lc; ++q) {
                const uint32_t word = row[q];
#pragma unroll
                for (int bpos = 0; bpos < 4; ++bpos) {
                    const int p = 4 * q + bpos;
                    if (p < Lc) {
                        const uint32_t c = (word >> (8 * bpos)) & 0xffu;
                        bad |= c >= 20u;
                        const uint64_t v = (uint64_t)(c & 31u) << (5 * (p % 12));
#pragma unroll
                        for (int k = 0; k < WORDS; ++k)
                            if (p / 12 == k) w[k] |= v;
                    }
                }
            }
            if (bad) {
                atomicOr(err, SQ_DEVERR_INPUT);
#pragma unroll
                for (int k = 0; k < WORDS; ++k) w[k] = 0;
                L = 0;
            }
            w[0] |= (uint64_t)(L & 15) << 60;
            w[1] |= (uint64_t)(L >> 4) << 60;
            uint64_t *dst = out + i * WORDS;
            reinterpret_cast<ulonglong2 *>(dst)[0] = make_ulonglong2(w[0], w[1]);
            if (WORDS == 4) reinterpret_cast<ulonglong2 *>(dst)[1] = make_ulonglong2(w[2 % WORDS], w[3 % WORDS]);
        }
        __syncthreads();
    }
}

extern "C" int subquad_pack(subquad_ctx *ctx, const uint8_t *codes, int code_stride, const uint8_t *lens, int64_t n,
                            int pack_stride, void *packed_out)
{
    SQ_ENTER(ctx);
    if (n < 0 || (n > 0 && (!codes || !lens || !packed_out)) || code_stride < 1) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(packed_out) % 16) return SUBQUAD_ERR_ARG;
    if (n == 0) return SUBQUAD_OK;
    unsigned grid = sq_grid(ctx, n, 256);
    const bool staged = code_stride % 4 == 0 && code_stride / 4 <= kPackMaxStrideWords &&
                        reinterpret_cast<uintptr_t>(codes) % 4 == 0;
    if (staged) {
        const unsigned sgrid = (unsigned)std::min<int64_t>((n + kPackRows - 1) / kPackRows, (int64_t)ctx->num_sms * 8);
        const uint32_t *cw = reinterpret_cast<const uint32_t *>(codes);
        if (pack_stride == 16)
            pack_staged_kernel<2><<<sgrid, kPackRows, 0, ctx->stream>>>(cw, code_stride / 4, lens, n,
                                                                        (uint64_t *)packed_out, ctx->d_err);
        else
            pack_staged_kernel<4><<<sgrid, kPackRows, 0, ctx->stream>>>(cw, code_stride / 4, lens, n,
                                                                        (uint64_t *)packed_out, ctx->d_err);
    } else if (pack_stride == 16) {
        pack_kernel<2><<<grid, 256, 0, ctx->stream>>>(codes, code_stride, lens, n, (uint64_t *)packed_out, ctx->d_err);
    } else {
        pack_kernel<4><<<grid, 256, 0, ctx->stream>>>(codes, code_stride, lens, n, (uint64_t *)packed_out, ctx->d_err);
    }
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}
