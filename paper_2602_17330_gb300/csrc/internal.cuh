// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "subquad.h"

// Sticky device-side error bits (OR-ed by kernels, read by subquad_check and
// by synchronising calls).
enum : uint32_t {
    SQ_DEVERR_INPUT = 1u,
    SQ_DEVERR_TIMEOUT = 2u,
    SQ_DEVERR_CAPACITY = 4u,
    SQ_DEVERR_INTERNAL = 8u,  // a consistency check inside a kernel failed
};

#include <vector>

struct SqProfRecord {
    int kernel;
    cudaEvent_t start, stop;
};

struct subquad_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // a second stream of the library's own, forked from and joined back to
    // `stream` by events inside one call, for independent kernels that can
    // share the GPU (graph capture records the fork as parallel branches)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int num_sms = 0;
    int8_t h_matrix[400];   // scoring matrix, row = first sequence's residue
    bool matrix_symmetric = true;
    // Self-alignment shortcut: true when every diagonal entry is positive and
    // 2 M(a, b) <= M(a, a) + M(b, b) for all a, b; then (with gap costs >= 0)
    // the best local alignment of a sequence with itself is the ungapped
    // identity alignment, whose score is the sum of the diagonal entries.
    bool self_is_diagonal = true;
    int32_t *d_table = nullptr;  // lane-replicated alignment table (see align.cu)
    int table_gap_open = -1;     // gap-open folded into d_table (-1: not built)
    // edit-distance costs (subquad_set_edit_costs) and their lane-replicated
    // device table (built on first use after a change)
    uint8_t h_edit_sub[400];
    int edit_indel = 2;
    uint32_t *d_edit_table = nullptr;
    bool edit_table_valid = false;
    uint32_t *d_err = nullptr;   // sticky device error word
    uint64_t *h_pinned = nullptr;  // pinned host staging, 8 words
    uint64_t *d_small = nullptr;   // small device scalars (counters), 16 words
    void *scratch = nullptr;
    size_t scratch_cap = 0;
    int64_t launches = 0;  // kernels launched through this context
    int tune[SUBQUAD_TUNE_COUNT];  // tuning knobs, see subquad_set_tuning
    bool prof_on = false;          // per-kernel event timing (subquad_profile_*)
    std::vector<SqProfRecord> prof_records;
    std::vector<cudaEvent_t> prof_pool;
};

// Opt-in per-kernel timing: events recorded on the context stream around one
// launch (or launch sequence) tagged with a SUBQUAD_PROF_* id.
cudaEvent_t sq_prof_event(subquad_ctx *ctx);
// Name of a profiled kernel tag (NVTX range and diagnostics).
inline const char *sq_prof_name(int k)
{
    static const char *const names[SUBQUAD_PROF_COUNT] = {"subquad.sign", "subquad.band", "subquad.band_partition",
                                                          "subquad.band_group", "subquad.band_emit",
                                                          "subquad.band_pairsort", "subquad.align",
                                                          "subquad.align_bin", "subquad.self", "subquad.fuse",
                                                          "subquad.edit"};
    return k >= 0 && k < SUBQUAD_PROF_COUNT ? names[k] : "subquad";
}

// Every tagged region is an NVTX range (free unless a tool is attached);
// with the context's profiler on it is also timed by events on its stream.
struct SqProfScope {
    subquad_ctx *ctx;
    int kernel;
    cudaEvent_t stop = nullptr;
    bool ranged = false;
    SqProfScope(subquad_ctx *c, int k) : ctx(c), kernel(k)
    {
        nvtxRangePushA(sq_prof_name(k));
        ranged = true;
        if (!ctx->prof_on) return;
        cudaEvent_t start = sq_prof_event(ctx);
        stop = sq_prof_event(ctx);
        if (!start || !stop) {
            stop = nullptr;
            return;
        }
        cudaEventRecord(start, ctx->stream);
        ctx->prof_records.push_back({kernel, start, stop});
    }
    void finish()
    {
        if (stop) cudaEventRecord(stop, ctx->stream);
        stop = nullptr;
        if (ranged) nvtxRangePop();
        ranged = false;
    }
    ~SqProfScope() { finish(); }
};

// Last CUDA error seen by the library on this thread (for diagnostics).
void sq_note_cuda_error(cudaError_t e);

#define SQ_TRY_CUDA(call)                                  \
    do {                                                   \
        cudaError_t sq_e_ = (call);                        \
        if (sq_e_ != cudaSuccess) {                        \
            sq_note_cuda_error(sq_e_);                     \
            return SUBQUAD_ERR_CUDA;                       \
        }                                                  \
    } while (0)

#define SQ_TRY(call)                                       \
    do {                                                   \
        int sq_s_ = (call);                                \
        if (sq_s_ != SUBQUAD_OK) return sq_s_;             \
    } while (0)

#define SQ_LAUNCH_CHECK()                                  \
    do {                                                   \
        ++ctx->launches;                                   \
        SQ_TRY_CUDA(cudaGetLastError());                   \
    } while (0)

// Makes ctx->device current for the scope of an entry point and restores the
// caller's device afterwards.
struct SqDeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit SqDeviceGuard(const subquad_ctx *ctx)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != ctx->device) ok = cudaSetDevice(ctx->device) == cudaSuccess;
    }
    ~SqDeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define SQ_ENTER(ctx)                                      \
    if (!(ctx)) return SUBQUAD_ERR_ARG;                    \
    SqDeviceGuard sq_guard_(ctx);                          \
    if (!sq_guard_.ok) return SUBQUAD_ERR_CUDA

// Make sure ctx->scratch holds at least `bytes` (stream-ordered reallocation).
int sq_scratch_reserve(subquad_ctx *ctx, size_t bytes);

// Bump allocator over a scratch block.  With base == nullptr it only measures.
struct SqArena {
    char *base;
    size_t off = 0;
    explicit SqArena(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// Grid size for a grid-stride kernel: enough CTAs to fill the machine.
inline unsigned sq_grid(const subquad_ctx *ctx, int64_t work, int threads, int per_sm = 8)
{
    int64_t need = (work + threads - 1) / threads;
    int64_t cap = (int64_t)ctx->num_sms * per_sm;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

// Blocks for a grid-stride kernel: at most `need`, and at most one wave of
// the blocks that fit on the device at once (the kernel's occupancy times the
// SM count), so no partial last wave trails the others.
template <typename K>
inline unsigned sq_resident_grid(const subquad_ctx *ctx, K kernel, int threads, size_t smem, int64_t need)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t cap = (int64_t)ctx->num_sms * per_sm;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

// Packed sequence records (see subquad_pack in subquad.h).
__device__ __forceinline__ int sq_record_len(uint64_t w0, uint64_t w1)
{
    return (int)((w0 >> 60) | ((w1 >> 60) << 4));
}

// Device-wide primitives (primitives.cu).  `count` is the host-side element
// count (or an upper bound); when `d_count` is given the kernels process
// min(*d_count, count) elements, so a producer kernel can size the work
// without a host round trip.
int sq_scan_u32(subquad_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t count, const uint32_t *d_count,
                bool inclusive, bool max_op, uint32_t *total_out /* device, nullable */, void *tmp, size_t tmp_bytes);
int sq_scan_u64(subquad_ctx *ctx, const uint64_t *in, uint64_t *out, int64_t count, const uint32_t *d_count,
                uint64_t *total_out, void *tmp, size_t tmp_bytes);
size_t sq_scan_tmp_bytes(int64_t count);
// Stable LSD radix sort of (key, value) uint32 pairs on bits [begin_bit, end_bit).
// Returns via *result_in_alt whether the sorted data ended in the alt buffers.
int sq_radix_sort_u32(subquad_ctx *ctx, uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      int64_t count, const uint32_t *d_count, int begin_bit, int end_bit, bool *result_in_alt,
                      void *tmp, size_t tmp_bytes);
size_t sq_radix_tmp_bytes(int64_t count);

// Lane-replicated alignment score table for the context's matrix and gap_open
// (align.cu); shared by the alignment and the brute-force retrieval kernels.
void sq_update_matrix_flags(subquad_ctx *ctx);
// Default edit-distance substitution costs from the built-in BLOSUM62 (half
// units): 0 on the diagonal, 1 where the score is positive, else 2.
void sq_default_edit_costs(uint8_t *out);
int sq_ensure_align_table(subquad_ctx *ctx, int gap_open);
