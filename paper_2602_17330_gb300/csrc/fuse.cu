// (a4) Per-pair gated fusion of the alignment and embedding channels
// (Eq. alpha, Eq. wm, Eq. afused with M = 2 channels).
//
// A half-warp (16 lanes) owns one pair: each lane loads float4 slices of e_i
// and e_j (coalesced 256-byte rows for d = 64), the dot product and both
// squared norms are reduced with shuffles (a pairwise tree, so FP32 rounding
// grows with log2(d)), each lane then evaluates hidden units k = lane,
// lane + 16, ... of the gate MLP from parameters staged in shared memory, and
// a second shuffle tree gives the logit g.  alpha = sigmoid(g) is the
// two-logit softmax of Eq. wm with logits (g, 0).
#include "internal.cuh"

namespace {

constexpr int kFuseThreads = 256;
constexpr int kTpp = 16;  // threads per pair
constexpr int kMaxHidden = 64;

__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int d = kTpp / 2; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d, kTpp);
    return v;
}

template <int WORDS>
__device__ __forceinline__ int record_len(const uint64_t *__restrict__ packed, uint32_t i)
{
    ulonglong2 r = reinterpret_cast<const ulonglong2 *>(packed + (int64_t)i * WORDS)[0];
    return sq_record_len(r.x, r.y);
}

template <int WORDS>
__global__ void __launch_bounds__(kFuseThreads) fuse_forward_kernel(
    const uint32_t *__restrict__ pairs, int64_t m, const int32_t *__restrict__ sw, const int32_t *__restrict__ self_sc,
    const uint64_t *__restrict__ packed, const float *__restrict__ emb, int d, const float *__restrict__ params,
    int hidden, float *__restrict__ fused, float *__restrict__ alpha_out)
{
    __shared__ float s_par[5 * kMaxHidden + 1];
    for (int q = threadIdx.x; q < 5 * hidden + 1; q += blockDim.x) s_par[q] = params[q];
    __syncthreads();
    const float *W1 = s_par, *b1 = s_par + 3 * hidden, *w2 = s_par + 4 * hidden;
    const float b2 = s_par[5 * hidden];
    const int sub = threadIdx.x & (kTpp - 1);
    const int half = (threadIdx.x >> 4) & 1;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d4 = d >> 2;
    // the trip count is uniform per warp, so full-warp shuffles are safe
    for (int64_t pbase = warp * 2; pbase < m; pbase += nwarps * 2) {
        const int64_t p = pbase + half;
        const bool valid = p < m;
        uint2 ij = valid ? reinterpret_cast<const uint2 *>(pairs)[p] : make_uint2(0, 0);
        const float4 *ei = reinterpret_cast<const float4 *>(emb + (int64_t)ij.x * d);
        const float4 *ej = reinterpret_cast<const float4 *>(emb + (int64_t)ij.y * d);
        float dot = 0.f, sii = 0.f, sjj = 0.f;
        if (valid) {
            for (int k = sub; k < d4; k += kTpp) {
                float4 a = ei[k], b = ej[k];
                dot = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w))) + dot;
                sii = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, a.w * a.w))) + sii;
                sjj = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, b.w * b.w))) + sjj;
            }
        }
        dot = group_sum(dot);
        sii = group_sum(sii);
        sjj = group_sum(sjj);
        float s = 0.f, c = 0.f, delta = 0.f;
        if (valid) {
            const float prod = (float)self_sc[ij.x] * (float)self_sc[ij.y];
            s = prod > 0.f ? (float)sw[p] / sqrtf(prod) : 0.f;
            const float nn = sii * sjj;
            c = nn > 0.f ? dot / sqrtf(nn) : 0.f;
            delta = fabsf((float)(record_len<WORDS>(packed, ij.x) - record_len<WORDS>(packed, ij.y)));
        }
        float acc = 0.f;
        for (int k = sub; k < hidden; k += kTpp) {
            float z = fmaf(W1[3 * k], s, fmaf(W1[3 * k + 1], c, fmaf(W1[3 * k + 2], delta, b1[k])));
            acc = fmaf(w2[k], fmaxf(z, 0.f), acc);
        }
        const float g = group_sum(acc) + b2;
        if (valid && sub == 0) {
            const float a = 1.f / (1.f + expf(-g));
            fused[p] = a * s + (1.f - a) * 0.5f * (1.f + c);
            if (alpha_out) alpha_out[p] = a;
        }
    }
}

}  // namespace

extern "C" int subquad_fuse_forward(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                                    const int32_t *self_scores, const void *packed, int pack_stride, const float *emb,
                                    int d, const float *gate_params, int hidden, float *fused_out, float *alpha_out)
{
    SQ_ENTER(ctx);
    if (m < 0 || d < 4 || d > 1024 || d % 4 || hidden < 1 || hidden > kMaxHidden) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (m == 0) return SUBQUAD_OK;
    if (!pairs || !sw || !self_scores || !packed || !emb || !gate_params || !fused_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(emb) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8 ||
        reinterpret_cast<uintptr_t>(packed) % 16)
        return SUBQUAD_ERR_ARG;
    const unsigned grid = sq_grid(ctx, (m + 1) / 2 * 32, kFuseThreads, 8);
    if (pack_stride == 16)
        fuse_forward_kernel<2><<<grid, kFuseThreads, 0, ctx->stream>>>(pairs, m, sw, self_scores,
                                                                      (const uint64_t *)packed, emb, d, gate_params,
                                                                      hidden, fused_out, alpha_out);
    else
        fuse_forward_kernel<4><<<grid, kFuseThreads, 0, ctx->stream>>>(pairs, m, sw, self_scores,
                                                                      (const uint64_t *)packed, emb, d, gate_params,
                                                                      hidden, fused_out, alpha_out);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}
