// (a5) Gate training around the fusion adjoint: pair labels and subgroup
// weights, the weighted binary cross-entropy with its gradient, the pair index
// used for the deterministic embedding-gradient reduction, and Adam.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr double kClamp = 1e-7;

__global__ void pair_labels_kernel(const uint32_t *__restrict__ pairs, int64_t m, const int32_t *__restrict__ family,
                                   const int32_t *__restrict__ subgroup, uint8_t *__restrict__ label,
                                   int32_t *__restrict__ group)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const uint2 ij = reinterpret_cast<const uint2 *>(pairs)[p];
        const int32_t fi = family[ij.x], fj = family[ij.y];
        label[p] = (uint8_t)(fi >= 0 && fi == fj);
        const int32_t gi = subgroup[ij.x];
        group[p] = gi != 0 ? gi : subgroup[ij.y];
    }
}

// Per block: a shared-memory histogram of the groups (most pairs fall in a
// handful of groups, so global atomics per pair serialise on those few
// counters), then one global atomic per group and block.
__global__ void group_count_kernel(const int32_t *__restrict__ group, int64_t m, int num_groups,
                                   uint32_t *__restrict__ counts, uint32_t *err)
{
    extern __shared__ uint32_t s_hist[];
    for (int g = threadIdx.x; g < num_groups; g += blockDim.x) s_hist[g] = 0;
    __syncthreads();
    bool bad = false;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = group[p];
        if (g < 0 || g >= num_groups) {
            bad = true;
            continue;
        }
        atomicAdd(&s_hist[g], 1u);
    }
    if (bad) atomicOr(err, SQ_DEVERR_INPUT);
    __syncthreads();
    for (int g = threadIdx.x; g < num_groups; g += blockDim.x)
        if (s_hist[g]) atomicAdd(&counts[g], s_hist[g]);
}

// w_p = (m / count_g) * m / sum_q (m / count_{g(q)}) = m / (count_g * groups_present)
__global__ void group_weight_kernel(const int32_t *__restrict__ group, int64_t m, int num_groups,
                                    const uint32_t *__restrict__ counts, float *__restrict__ weight)
{
    extern __shared__ uint32_t s_cnt[];
    __shared__ int s_present;
    if (threadIdx.x == 0) s_present = 0;
    __syncthreads();
    int local = 0;
    for (int g = threadIdx.x; g < num_groups; g += blockDim.x) {
        s_cnt[g] = counts[g];
        local += s_cnt[g] > 0;
    }
    atomicAdd(&s_present, local);
    __syncthreads();
    const double present = (double)s_present;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = group[p];
        const uint32_t c = (g >= 0 && g < num_groups) ? s_cnt[g] : 0u;
        weight[p] = c ? (float)((double)m / ((double)c * present)) : 0.f;
    }
}

// The clamp of the loss and of its adjoint, for a float fused score q, as
// float comparisons that decide exactly as the FP64 ones on the widened q:
// q < c  <=>  q < lo_in, q > 1 - c  <=>  q > hi_in (loss), q > c  <=>  q >
// lo_out, q < 1 - c  <=>  q < hi_out (adjoint), and the logarithm arguments
// of the clamped cases as the FP64 clamp rounds them to float.
struct BceClamp {
    float lo_in, hi_in, lo_out, hi_out;
    float arg_lo1, arg_hi1, arg_lo0, arg_hi0;  // label 1 / label 0 at the low / high clamp
};

BceClamp bce_clamp()
{
    auto ceil_f = [](double c) {  // smallest float >= c
        float f = (float)c;
        return (double)f < c ? nextafterf(f, INFINITY) : f;
    };
    auto floor_f = [](double c) {  // largest float <= c
        float f = (float)c;
        return (double)f > c ? nextafterf(f, -INFINITY) : f;
    };
    BceClamp k;
    k.lo_in = ceil_f(kClamp);
    k.hi_in = floor_f(1.0 - kClamp);
    k.lo_out = floor_f(kClamp);
    k.hi_out = ceil_f(1.0 - kClamp);
    k.arg_lo1 = (float)kClamp;
    k.arg_hi1 = (float)(1.0 - kClamp);
    k.arg_lo0 = (float)(1.0 - kClamp);
    k.arg_hi0 = (float)(1.0 - (1.0 - kClamp));
    return k;
}

// Per block: partial sums of w and w * l in a fixed order.  The label is 0
// or 1, so each pair's loss is one logarithm, -log(q) or -log(1 - q), taken in
// FP32 (one or two ulps of a term, far inside the loss tolerance); each thread
// sums its pairs with compensated FP32 additions and the block adds the
// threads' sums in FP64 (the FP64 pipe is slow on this part).
__global__ void __launch_bounds__(kThreads) bce_partial_kernel(const float *__restrict__ fused,
                                                               const uint8_t *__restrict__ label,
                                                               const float *__restrict__ weight, int64_t m,
                                                               BceClamp k, double *__restrict__ partials)
{
    __shared__ double s_w[kThreads], s_l[kThreads];
    float sw = 0.f, cw = 0.f, sl = 0.f, cl = 0.f;  // compensated sums
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const float w = weight[p], q = fused[p];
        float arg;
        if (label[p])
            arg = q < k.lo_in ? k.arg_lo1 : (q > k.hi_in ? k.arg_hi1 : q);
        else
            arg = q < k.lo_in ? k.arg_lo0 : (q > k.hi_in ? k.arg_hi0 : 1.f - q);  // 1 - q: one correctly rounded op
        const float term = w * -logf(arg);
        float y = w - cw, t = sw + y;
        cw = (t - sw) - y;
        sw = t;
        y = term - cl;
        t = sl + y;
        cl = (t - sl) - y;
        sl = t;
    }
    s_w[threadIdx.x] = (double)sw - (double)cw;
    s_l[threadIdx.x] = (double)sl - (double)cl;
    __syncthreads();
    for (int stride = kThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            s_w[threadIdx.x] += s_w[threadIdx.x + stride];
            s_l[threadIdx.x] += s_l[threadIdx.x + stride];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s_w[0];
        partials[2 * blockIdx.x + 1] = s_l[0];
    }
}

__global__ void bce_final_kernel(const double *__restrict__ partials, int blocks, float *__restrict__ loss_out,
                                 double *__restrict__ wsum_out)
{
    if (threadIdx.x != 0) return;
    double sw = 0.0, sl = 0.0;
    for (int b = 0; b < blocks; ++b) {
        sw += partials[2 * b];
        sl += partials[2 * b + 1];
    }
    *wsum_out = sw;
    if (loss_out) *loss_out = sw > 0.0 ? (float)(sl / sw) : 0.f;
}

__global__ void bce_grad_kernel(const float *__restrict__ fused, const uint8_t *__restrict__ label,
                                const float *__restrict__ weight, int64_t m, BceClamp k,
                                const double *__restrict__ wsum, float *__restrict__ dL)
{
    // the clamp test as the loss's (exact float thresholds), the adjoint
    // w (q - y) / (q (1 - q)) / sum(w) in FP32: q - y is exact for y in {0, 1}
    // and q in [1/2, 1] or y = 0, the rest a few roundings, far inside the
    // gradient tolerance
    const float inv = *wsum > 0.0 ? (float)(1.0 / *wsum) : 0.f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const float q = fused[p];
        const bool inside = q > k.lo_out && q < k.hi_out;
        const float y = label[p] ? 1.f : 0.f;
        dL[p] = inside ? weight[p] * (q - y) / (q * (1.f - q)) * inv : 0.f;
    }
}

__global__ void member_keys_kernel(const uint32_t *__restrict__ pairs, int64_t m, int which, uint32_t *__restrict__ keys,
                                   uint32_t *__restrict__ vals, uint32_t *__restrict__ counts)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = pairs[2 * p + which];
        keys[p] = v;
        vals[p] = (uint32_t)p;
        atomicAdd(&counts[v], 1u);
    }
}

__global__ void adam_kernel(float *__restrict__ param, const float *__restrict__ grad, float *__restrict__ m1,
                            float *__restrict__ m2, int64_t count, float beta1, float beta2, float lr_t, float bc2_sqrt,
                            float eps)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[k];
        const float a = beta1 * m1[k] + (1.f - beta1) * g;
        const float b = beta2 * m2[k] + (1.f - beta2) * g * g;
        m1[k] = a;
        m2[k] = b;
        param[k] -= lr_t * a / (sqrtf(b) / bc2_sqrt + eps);
    }
}

// The same update, four elements per thread with 16-byte loads and stores
// (count4 = count / 4 vectors; the caller handles the tail).
__device__ __forceinline__ float adam_one(float &p, float g, float &a1, float &a2, float beta1, float beta2,
                                          float lr_t, float bc2_sqrt, float eps)
{
    const float a = beta1 * a1 + (1.f - beta1) * g;
    const float b = beta2 * a2 + (1.f - beta2) * g * g;
    a1 = a;
    a2 = b;
    p -= lr_t * a / (sqrtf(b) / bc2_sqrt + eps);
    return p;
}

__global__ void adam4_kernel(float4 *__restrict__ param, const float4 *__restrict__ grad, float4 *__restrict__ m1,
                             float4 *__restrict__ m2, int64_t count4, float beta1, float beta2, float lr_t,
                             float bc2_sqrt, float eps)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count4; k += (int64_t)gridDim.x * blockDim.x) {
        const float4 g = grad[k];
        float4 a = m1[k], b = m2[k], p = param[k];
        adam_one(p.x, g.x, a.x, b.x, beta1, beta2, lr_t, bc2_sqrt, eps);
        adam_one(p.y, g.y, a.y, b.y, beta1, beta2, lr_t, bc2_sqrt, eps);
        adam_one(p.z, g.z, a.z, b.z, beta1, beta2, lr_t, bc2_sqrt, eps);
        adam_one(p.w, g.w, a.w, b.w, beta1, beta2, lr_t, bc2_sqrt, eps);
        m1[k] = a;
        m2[k] = b;
        param[k] = p;
    }
}

int bits_for(uint64_t v)
{
    int b = 1;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

}  // namespace

extern "C" int subquad_pair_labels(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *family,
                                   const int32_t *subgroup, uint8_t *label_out, int32_t *group_out)
{
    SQ_ENTER(ctx);
    if (m < 0) return SUBQUAD_ERR_ARG;
    if (m == 0) return SUBQUAD_OK;
    if (!pairs || !family || !subgroup || !label_out || !group_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(pairs) % 8) return SUBQUAD_ERR_ARG;
    pair_labels_kernel<<<sq_grid(ctx, m, kThreads), kThreads, 0, ctx->stream>>>(pairs, m, family, subgroup, label_out,
                                                                               group_out);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

extern "C" int subquad_pair_weights(subquad_ctx *ctx, const int32_t *group, int64_t m, int num_groups,
                                    float *weight_out)
{
    SQ_ENTER(ctx);
    if (m < 0 || num_groups < 1 || num_groups > 4096) return SUBQUAD_ERR_ARG;
    if (m == 0) return SUBQUAD_OK;
    if (!group || !weight_out) return SUBQUAD_ERR_ARG;
    SQ_TRY(sq_scratch_reserve(ctx, sizeof(uint32_t) * num_groups));
    uint32_t *counts = static_cast<uint32_t *>(ctx->scratch);
    SQ_TRY_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * num_groups, ctx->stream));
    const unsigned grid = sq_grid(ctx, m, kThreads);
    group_count_kernel<<<grid, kThreads, sizeof(uint32_t) * num_groups, ctx->stream>>>(group, m, num_groups, counts,
                                                                                        ctx->d_err);
    SQ_LAUNCH_CHECK();
    group_weight_kernel<<<grid, kThreads, sizeof(uint32_t) * num_groups, ctx->stream>>>(group, m, num_groups, counts,
                                                                                        weight_out);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

extern "C" int subquad_bce_loss(subquad_ctx *ctx, const float *fused, const uint8_t *label, const float *weight,
                                int64_t m, float *loss_out, float *dL_dfused)
{
    SQ_ENTER(ctx);
    if (m < 0 || !loss_out) return SUBQUAD_ERR_ARG;
    if (m > 0 && (!fused || !label || !weight)) return SUBQUAD_ERR_ARG;
    // a fixed grid keeps the summation order independent of the launch
    const int blocks = ctx->num_sms * 2;
    SQ_TRY(sq_scratch_reserve(ctx, sizeof(double) * (2 * blocks + 1)));
    double *partials = static_cast<double *>(ctx->scratch);
    double *wsum = partials + 2 * blocks;
    const BceClamp k = bce_clamp();
    bce_partial_kernel<<<blocks, kThreads, 0, ctx->stream>>>(fused, label, weight, m, k, partials);
    SQ_LAUNCH_CHECK();
    bce_final_kernel<<<1, 32, 0, ctx->stream>>>(partials, blocks, loss_out, wsum);
    SQ_LAUNCH_CHECK();
    if (dL_dfused && m > 0) {
        bce_grad_kernel<<<sq_grid(ctx, m, kThreads), kThreads, 0, ctx->stream>>>(fused, label, weight, m, k, wsum,
                                                                                 dL_dfused);
        SQ_LAUNCH_CHECK();
    }
    return SUBQUAD_OK;
}

extern "C" int subquad_pair_index(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, int64_t n, uint32_t *perm_i,
                                  uint32_t *off_i, uint32_t *perm_j, uint32_t *off_j)
{
    SQ_ENTER(ctx);
    if (m < 0 || n < 1 || m >= (int64_t(1) << 32) || n >= (int64_t(1) << 31)) return SUBQUAD_ERR_ARG;
    if (!off_i || !off_j || (m > 0 && (!pairs || !perm_i || !perm_j))) return SUBQUAD_ERR_ARG;
    const int64_t cm = std::max<int64_t>(m, 1);
    SqArena measure(nullptr);
    measure.take<uint32_t>(cm);
    measure.take<uint32_t>(cm);
    measure.take<uint32_t>(cm);
    measure.take<uint32_t>(n + 1);
    measure.take<char>(std::max(sq_radix_tmp_bytes(cm), sq_scan_tmp_bytes(n + 1)));
    SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    SqArena a(ctx->scratch);
    uint32_t *keys = a.take<uint32_t>(cm);
    uint32_t *keys_alt = a.take<uint32_t>(cm);
    uint32_t *vals_alt = a.take<uint32_t>(cm);
    uint32_t *counts = a.take<uint32_t>(n + 1);
    const size_t tmp_bytes = std::max(sq_radix_tmp_bytes(cm), sq_scan_tmp_bytes(n + 1));
    void *tmp = a.take<char>(tmp_bytes);
    const int nb = bits_for((uint64_t)(n - 1));
    for (int which = 0; which < 2; ++which) {
        uint32_t *perm = which == 0 ? perm_i : perm_j;
        uint32_t *off = which == 0 ? off_i : off_j;
        SQ_TRY_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (n + 1), ctx->stream));
        if (m > 0) {
            member_keys_kernel<<<sq_grid(ctx, m, kThreads), kThreads, 0, ctx->stream>>>(pairs, m, which, keys, perm,
                                                                                        counts);
            SQ_LAUNCH_CHECK();
            bool in_alt = false;
            SQ_TRY(sq_radix_sort_u32(ctx, keys, perm, keys_alt, vals_alt, m, nullptr, 0, nb, &in_alt, tmp, tmp_bytes));
            if (in_alt)
                SQ_TRY_CUDA(cudaMemcpyAsync(perm, vals_alt, sizeof(uint32_t) * m, cudaMemcpyDeviceToDevice,
                                            ctx->stream));
        }
        // counts[n] = 0, so the exclusive scan's entry n is m
        SQ_TRY(sq_scan_u32(ctx, counts, off, n + 1, nullptr, false, false, nullptr, tmp, tmp_bytes));
    }
    return SUBQUAD_OK;
}

extern "C" int subquad_adam_step(subquad_ctx *ctx, float *param, const float *grad, float *m1, float *m2,
                                 int64_t count, int t, float lr, float beta1, float beta2, float eps)
{
    SQ_ENTER(ctx);
    if (count < 0 || t < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f)) return SUBQUAD_ERR_ARG;
    if (count == 0) return SUBQUAD_OK;
    if (!param || !grad || !m1 || !m2) return SUBQUAD_ERR_ARG;
    const double bc1 = 1.0 - pow((double)beta1, (double)t);
    const double bc2 = 1.0 - pow((double)beta2, (double)t);
    const float lr_t = (float)(lr / bc1), bc2_sqrt = (float)sqrt(bc2);
    const bool aligned = (reinterpret_cast<uintptr_t>(param) | reinterpret_cast<uintptr_t>(grad) |
                          reinterpret_cast<uintptr_t>(m1) | reinterpret_cast<uintptr_t>(m2)) % 16 == 0;
    int64_t head = 0;  // elements done by the vector kernel
    if (aligned && count >= 4) {
        const int64_t count4 = count / 4;
        adam4_kernel<<<sq_grid(ctx, count4, kThreads), kThreads, 0, ctx->stream>>>(
            reinterpret_cast<float4 *>(param), reinterpret_cast<const float4 *>(grad), reinterpret_cast<float4 *>(m1),
            reinterpret_cast<float4 *>(m2), count4, beta1, beta2, lr_t, bc2_sqrt, eps);
        SQ_LAUNCH_CHECK();
        head = 4 * count4;
    }
    if (head < count) {
        adam_kernel<<<sq_grid(ctx, count - head, kThreads), kThreads, 0, ctx->stream>>>(
            param + head, grad + head, m1 + head, m2 + head, count - head, beta1, beta2, lr_t, bc2_sqrt, eps);
        SQ_LAUNCH_CHECK();
    }
    return SUBQUAD_OK;
}
