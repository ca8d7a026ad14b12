// (a4) Per-pair gated fusion of the alignment and embedding channels
// (Eq. alpha, Eq. wm, Eq. afused with M = 2 channels), and its adjoint.
//
// Forward: four lanes own one pair (eight pairs per warp).  When d % 8 == 0
// (and d <= 128) each lane reads 32-byte chunks of e_i and e_j with 256-bit
// loads, so a pair's four lanes read one whole 128-byte line of a row per
// load (for d = 64, two loads per row); otherwise 16-byte chunks.  Each lane
// accumulates the dot product and both squared norms, and two shuffle levels
// finish them; each lane then evaluates hidden units
// k = lane, lane + 4, ... of the gate MLP from parameters staged in shared
// memory, and two more shuffle levels give the logit g.  alpha = sigmoid(g)
// is the two-logit softmax of Eq. wm with logits (g, 0).  The kernel is
// instruction-bound at 16 lanes per pair, so the split favours fewer
// shuffles and more work per lane.
#include <algorithm>
#include <mutex>

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

constexpr int kTppF = 4;  // lanes per pair in the forward kernels (default)

__device__ __forceinline__ float quad_sum(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 2, kTppF);
    v += __shfl_xor_sync(0xffffffffu, v, 1, kTppF);
    return v;
}

// Sum over the T lanes of one pair (T a power of two <= 32).
template <int T>
__device__ __forceinline__ float lanes_sum(float v)
{
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, T);
    return v;
}

// One 32-byte load (a 256-bit vector load of the read-only path) into two
// float4; p must be 32-byte aligned.
__device__ __forceinline__ void ldg_v8(const float *p, float4 &lo, float4 &hi)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
        : "l"(p));
}

__device__ __forceinline__ void ldg_v8u(const uint32_t *p, uint4 &lo, uint4 &hi)
{
    asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
        : "l"(p));
}

// Per-pair inputs of the fusion, all loads issued together so one round trip
// to memory (after the pair indices) covers the embedding rows, the alignment
// score, both self-scores and both lengths.  A lane loads CPL chunks of V
// float4 from each row: V = 1 (16-byte loads; chunk k = float4 k) or V = 2
// (32-byte loads, rows 32-byte aligned; chunk k = floats 8k .. 8k + 7), the
// pair's TPP lanes taking consecutive chunks.
template <int WORDS, int CPL, int TPP = kTpp, int V = 1>
struct PairInputs {
    float4 a[CPL * V], b[CPL * V];
    int32_t sw, self_i, self_j;
    int len_i, len_j;

    __device__ __forceinline__ void load(uint2 ij, int64_t p, bool valid, int sub, int d4, const float *__restrict__ emb,
                                         int d, const int32_t *__restrict__ sw_in, const int32_t *__restrict__ self_sc,
                                         const uint64_t *__restrict__ packed)
    {
        if (V == 2) {
            const float *ei = emb + (int64_t)ij.x * d, *ej = emb + (int64_t)ij.y * d;
            const int d8 = d4 >> 1;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int k = sub + c * TPP;
                if (valid && k < d8) {
                    ldg_v8(ei + 8 * k, a[V * c], a[V * c + V - 1]);
                    ldg_v8(ej + 8 * k, b[V * c], b[V * c + V - 1]);
                } else {
                    a[V * c] = a[V * c + V - 1] = b[V * c] = b[V * c + V - 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        } else {
            const float4 *ei = reinterpret_cast<const float4 *>(emb + (int64_t)ij.x * d);
            const float4 *ej = reinterpret_cast<const float4 *>(emb + (int64_t)ij.y * d);
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int k = sub + c * TPP;
                const bool ok = valid && k < d4;
                a[c] = ok ? __ldg(ei + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                b[c] = ok ? __ldg(ej + k) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        sw = 0;
        self_i = self_j = 0;
        len_i = len_j = 0;
        if (valid) {
            sw = __ldg(sw_in + p);
            self_i = __ldg(self_sc + ij.x);
            self_j = __ldg(self_sc + ij.y);
            const ulonglong2 ri = __ldg(reinterpret_cast<const ulonglong2 *>(packed + (int64_t)ij.x * WORDS));
            const ulonglong2 rj = __ldg(reinterpret_cast<const ulonglong2 *>(packed + (int64_t)ij.y * WORDS));
            len_i = sq_record_len(ri.x, ri.y);
            len_j = sq_record_len(rj.x, rj.y);
        }
    }
};

template <int WORDS, int CPL, int TPPF, int V = 1>
__global__ void __launch_bounds__(kFuseThreads) fuse_forward_kernel(
    const uint32_t *__restrict__ pairs, int64_t m_max, const unsigned long long *__restrict__ d_m,
    const int32_t *__restrict__ sw, const int32_t *__restrict__ self_sc, const uint64_t *__restrict__ packed,
    const float *__restrict__ emb, int d, const float *__restrict__ params, int hidden, float *__restrict__ fused,
    float *__restrict__ alpha_out)
{
    // hidden unit k as one 16-byte word (W1[k][0..2], b1[k]) and w2[k]: two
    // shared-memory loads per unit instead of five
    __shared__ float4 s_unit[kMaxHidden];
    __shared__ float s_w2[kMaxHidden];
    __shared__ float s_b2;
    int64_t m = m_max;
    if (d_m) m = (int64_t)*d_m < m_max ? (int64_t)*d_m : m_max;
    for (int k = threadIdx.x; k < hidden; k += blockDim.x) {
        s_unit[k] = make_float4(params[3 * k], params[3 * k + 1], params[3 * k + 2], params[3 * hidden + k]);
        s_w2[k] = params[4 * hidden + k];
    }
    if (threadIdx.x == 0) s_b2 = params[5 * hidden];
    __syncthreads();
    const float b2 = s_b2;
    constexpr int kPairsPerWarp = 32 / TPPF;
    const int sub = threadIdx.x & (TPPF - 1);
    const int slot = (threadIdx.x & 31) / TPPF;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d4 = d >> 2;
    // the trip count is uniform per warp, so full-warp shuffles are safe; the
    // next iteration's pair is loaded one iteration ahead
    const int64_t pstep = nwarps * kPairsPerWarp;
    uint2 ij_next = warp * kPairsPerWarp + slot < m
                        ? __ldg(reinterpret_cast<const uint2 *>(pairs) + warp * kPairsPerWarp + slot)
                        : make_uint2(0, 0);
    for (int64_t pbase = warp * kPairsPerWarp; pbase < m; pbase += pstep) {
        const int64_t p = pbase + slot;
        const bool valid = p < m;
        const uint2 ij = valid ? ij_next : make_uint2(0, 0);
        ij_next = p + pstep < m ? __ldg(reinterpret_cast<const uint2 *>(pairs) + p + pstep) : make_uint2(0, 0);
        PairInputs<WORDS, CPL, TPPF, V> in;
        in.load(ij, p, valid, sub, d4, emb, d, sw, self_sc, packed);
        float dot = 0.f, sii = 0.f, sjj = 0.f;
#pragma unroll
        for (int c = 0; c < CPL * V; ++c) {
            const float4 a = in.a[c], b = in.b[c];
            dot = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, dot))));
            sii = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, sii))));
            sjj = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, sjj))));
        }
        dot = lanes_sum<TPPF>(dot);
        sii = lanes_sum<TPPF>(sii);
        sjj = lanes_sum<TPPF>(sjj);
        const float prod = (float)in.self_i * (float)in.self_j;
        const float s = prod > 0.f ? (float)in.sw * rsqrtf(prod) : 0.f;
        const float nn = sii * sjj;
        const float c = nn > 0.f ? dot * rsqrtf(nn) : 0.f;
        const float delta = fabsf((float)(in.len_i - in.len_j));
        float acc = 0.f;
        for (int k = sub; k < hidden; k += TPPF) {
            const float4 u = s_unit[k];
            float z = fmaf(u.x, s, fmaf(u.y, c, fmaf(u.z, delta, u.w)));
            acc = fmaf(s_w2[k], fmaxf(z, 0.f), acc);
        }
        const float g = lanes_sum<TPPF>(acc) + b2;
        if (valid && sub == 0) {
            const float a = __fdividef(1.f, 1.f + __expf(-g));
            fused[p] = fmaf(a, s - 0.5f * (1.f + c), 0.5f * (1.f + c));
            if (alpha_out) alpha_out[p] = a;
        }
    }
}

template <int WORDS, int TPPF>
int launch_forward_t(subquad_ctx *ctx, unsigned grid, const uint32_t *pairs, int64_t m, const int32_t *sw,
                     const int32_t *self_scores, const void *packed, const float *emb, int d, const float *gate_params,
                     int hidden, float *fused_out, float *alpha_out, const unsigned long long *d_m)
{
    if (d % 8 == 0 && d <= 8 * 4 * TPPF && reinterpret_cast<uintptr_t>(emb) % 32 == 0) {
        // 32-byte lane loads: four lanes read a 128-byte line of a row per load
        const int cpl8 = (d / 8 + TPPF - 1) / TPPF;
#define SQ_FWD8(C)                                                                                                 \
    fuse_forward_kernel<WORDS, C, TPPF, 2><<<grid, kFuseThreads, 0, ctx->stream>>>(                                \
        pairs, m, d_m, sw, self_scores, (const uint64_t *)packed, emb, d, gate_params, hidden, fused_out, alpha_out)
        if (cpl8 <= 1) SQ_FWD8(1);
        else if (cpl8 <= 2) SQ_FWD8(2);
        else SQ_FWD8(4);
#undef SQ_FWD8
        SQ_LAUNCH_CHECK();
        return SUBQUAD_OK;
    }
    const int cpl = (d / 4 + TPPF - 1) / TPPF;  // float4 chunks per lane
#define SQ_FWD(C)                                                                                                  \
    fuse_forward_kernel<WORDS, C, TPPF><<<grid, kFuseThreads, 0, ctx->stream>>>(                                   \
        pairs, m, d_m, sw, self_scores, (const uint64_t *)packed, emb, d, gate_params, hidden, fused_out, alpha_out)
    if (cpl <= 1) SQ_FWD(1);
    else if (cpl <= 2) SQ_FWD(2);
    else if (cpl <= 4) SQ_FWD(4);
    else if (cpl <= 8) SQ_FWD(8);
    else if (cpl <= 16) SQ_FWD(16);
    else if (cpl <= 32) SQ_FWD(32);
    else SQ_FWD(64);
#undef SQ_FWD
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

// Lanes per pair from the context's tuning: 4 (eight pairs per warp) or 8
// (four pairs per warp).
template <int WORDS>
int launch_forward(subquad_ctx *ctx, unsigned grid, const uint32_t *pairs, int64_t m, const int32_t *sw,
                   const int32_t *self_scores, const void *packed, const float *emb, int d, const float *gate_params,
                   int hidden, float *fused_out, float *alpha_out, const unsigned long long *d_m = nullptr)
{
    SqProfScope prof(ctx, SUBQUAD_PROF_FUSE);
    if (ctx->tune[SUBQUAD_TUNE_FUSE_LANES] == 8)
        return launch_forward_t<WORDS, 8>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden,
                                          fused_out, alpha_out, d_m);
    return launch_forward_t<WORDS, 4>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden,
                                      fused_out, alpha_out, d_m);
}


// ---------------------------------------------------------------------------
// Adjoint (gate training).  Pass 1: per pair, recompute the forward, then
// accumulate the parameter gradient per lane (compensated FP32), and store
// three per-pair coefficients of the cosine adjoint,
//   dL/de_i = k0 e_j + k1 e_i,  dL/de_j = k0 e_i + k2 e_j,
//   k0 = dc / (|e_i||e_j|), k1 = -dc c / |e_i|^2, k2 = -dc c / |e_j|^2,
// with dc = dL/dc.  Each block then reduces its lanes in FP64 in a fixed
// order.  Pass 2: one block sums the block partials in FP64 in block order.
// Pass 3 (optional): one half-warp per sequence gathers its pairs through the
// pair index and writes its embedding-gradient row once.
// ---------------------------------------------------------------------------

struct Kahan {
    float sum = 0.f, comp = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    __device__ __forceinline__ double value() const { return (double)sum - (double)comp; }
};

constexpr int kGroups = kFuseThreads / kTpp;  // pair groups (half-warps) per block

// The adjoint runs on a fixed grid of four blocks per SM (its reduction order
// must not depend on m); at most two float4 chunks and two hidden units per
// lane fit the 64 registers that keep all four resident (no spill), where 76
// left a second, quarter-full wave of blocks.
template <int CPL, int HPL>
constexpr int bwd_min_blocks()
{
    return CPL <= 2 && HPL <= 2 ? 4 : 1;
}

template <int WORDS, int CPL, int HPL>
__global__ void __launch_bounds__(kFuseThreads, bwd_min_blocks<CPL, HPL>()) fuse_backward_kernel(
    const uint32_t *__restrict__ pairs, int64_t m, const int32_t *__restrict__ sw, const int32_t *__restrict__ self_sc,
    const uint64_t *__restrict__ packed, const float *__restrict__ emb, int d, const float *__restrict__ params,
    int hidden, const float *__restrict__ dL, float4 *__restrict__ coef, double *__restrict__ partials)
{
    __shared__ float s_par[5 * kMaxHidden + 1];
    extern __shared__ double s_red[];  // [kGroups][5 * hidden + 1]
    const int P = 5 * hidden + 1;
    for (int q = threadIdx.x; q < P; q += blockDim.x) s_par[q] = params[q];
    __syncthreads();
    const float *W1 = s_par, *b1 = s_par + 3 * hidden, *w2 = s_par + 4 * hidden;
    const float b2 = s_par[5 * hidden];
    const int sub = threadIdx.x & (kTpp - 1);
    const int half = (threadIdx.x >> 4) & 1;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d4 = d >> 2;
    Kahan gW[HPL][3], gb1[HPL], gw2[HPL], gb2;
    // the next iteration's pair is loaded one iteration ahead, so an
    // iteration waits on one round trip (its rows) instead of two
    const uint2 *pr = reinterpret_cast<const uint2 *>(pairs);
    uint2 ij_next = warp * 2 + half < m ? __ldg(pr + warp * 2 + half) : make_uint2(0, 0);
    for (int64_t pbase = warp * 2; pbase < m; pbase += nwarps * 2) {
        const int64_t p = pbase + half;
        const bool valid = p < m;
        const uint2 ij = valid ? ij_next : make_uint2(0, 0);
        ij_next = p + nwarps * 2 < m ? __ldg(pr + p + nwarps * 2) : make_uint2(0, 0);
        PairInputs<WORDS, CPL> in;
        in.load(ij, p, valid, sub, d4, emb, d, sw, self_sc, packed);
        const float dA = valid ? __ldg(dL + p) : 0.f;
        float dot = 0.f, sii = 0.f, sjj = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const float4 a = in.a[c], b = in.b[c];
            dot = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w))) + dot;
            sii = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, a.w * a.w))) + sii;
            sjj = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, b.w * b.w))) + sjj;
        }
        dot = group_sum(dot);
        sii = group_sum(sii);
        sjj = group_sum(sjj);
        const float prod = (float)in.self_i * (float)in.self_j;
        // the same approximate reciprocal square roots and quotients as the
        // forward (a few ulps, far inside the gradient tolerance; the
        // correctly rounded forms are long instruction sequences in an
        // instruction-bound kernel)
        const float s = prod > 0.f ? (float)in.sw * rsqrtf(prod) : 0.f;
        const float nn = sii * sjj;
        const float c = nn > 0.f ? dot * rsqrtf(nn) : 0.f;
        const float delta = fabsf((float)(in.len_i - in.len_j));
        float z[HPL];
        float acc = 0.f;
#pragma unroll
        for (int hh = 0; hh < HPL; ++hh) {
            const int k = sub + hh * kTpp;
            z[hh] = 0.f;
            if (k < hidden) {
                z[hh] = fmaf(W1[3 * k], s, fmaf(W1[3 * k + 1], c, fmaf(W1[3 * k + 2], delta, b1[k])));
                acc = fmaf(w2[k], fmaxf(z[hh], 0.f), acc);
            }
        }
        const float g = group_sum(acc) + b2;
        const float a = __fdividef(1.f, 1.f + __expf(-g));
        const float d_g = dA * (s - 0.5f * (1.f + c)) * a * (1.f - a);
        float dc = 0.f;
#pragma unroll
        for (int hh = 0; hh < HPL; ++hh) {
            const int k = sub + hh * kTpp;
            if (k < hidden && valid) {
                const float u = fmaxf(z[hh], 0.f);
                gw2[hh].add(d_g * u);
                const float dz = z[hh] > 0.f ? d_g * w2[k] : 0.f;
                gW[hh][0].add(dz * s);
                gW[hh][1].add(dz * c);
                gW[hh][2].add(dz * delta);
                gb1[hh].add(dz);
                dc = fmaf(dz, W1[3 * k + 1], dc);
            }
        }
        dc = group_sum(dc) + dA * (1.f - a) * 0.5f;
        if (sub == 0 && valid) {
            gb2.add(d_g);
            if (coef) {
                float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
                if (sii > 0.f && sjj > 0.f) {
                    cf.x = dc * rsqrtf(sii * sjj);
                    cf.y = __fdividef(-dc * c, sii);
                    cf.z = __fdividef(-dc * c, sjj);
                }
                coef[p] = cf;
            }
        }
    }
    // block reduction: group-major partials in shared memory, then a fixed-order
    // FP64 sum over the groups for every parameter
    const int grp = threadIdx.x / kTpp;
    double *mine = s_red + (size_t)grp * P;
#pragma unroll
    for (int hh = 0; hh < HPL; ++hh) {
        const int k = sub + hh * kTpp;
        if (k < hidden) {
            mine[3 * k] = gW[hh][0].value();
            mine[3 * k + 1] = gW[hh][1].value();
            mine[3 * k + 2] = gW[hh][2].value();
            mine[3 * hidden + k] = gb1[hh].value();
            mine[4 * hidden + k] = gw2[hh].value();
        }
    }
    if (sub == 0) mine[5 * hidden] = gb2.value();
    __syncthreads();
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        double t = 0.0;
        for (int gi = 0; gi < kGroups; ++gi) t += s_red[(size_t)gi * P + q];
        partials[(int64_t)blockIdx.x * P + q] = t;
    }
}

__global__ void reduce_partials_kernel(const double *__restrict__ partials, int blocks, int P, float *__restrict__ out)
{
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < blocks; ++b) t += partials[(int64_t)b * P + q];
        out[q] = (float)t;
    }
}

// One half-warp per sequence v: its pairs (through the pair index, in index
// order) are taken sixteen at a time -- each lane loads one entry's pair id,
// pair and coefficients, so the dependent loads of sixteen pairs overlap --
// and the partners' rows up to four at a time, then accumulated in index order, so
// the sums are those of a sequential walk over the pairs (bitwise).  A
// sequence in a bucket of 2,000 members has thousands of pairs; walking them
// one dependent chain at a time made it the kernel's tail.
template <int CPL>
__global__ void __launch_bounds__(kFuseThreads) emb_grad_kernel(
    const uint32_t *__restrict__ pairs, const float4 *__restrict__ coef, const float *__restrict__ emb, int64_t n, int d,
    const uint32_t *__restrict__ perm_i, const uint32_t *__restrict__ off_i, const uint32_t *__restrict__ perm_j,
    const uint32_t *__restrict__ off_j, float *__restrict__ grad_emb, uint32_t heavy_min)
{
    constexpr int kRows = CPL <= 2 ? 4 : CPL <= 4 ? 2 : 1;  // partner rows in flight per step
    const int sub = threadIdx.x & (kTpp - 1);
    const unsigned hmask = 0xffffu << (threadIdx.x & 16);  // this half-warp's lanes
    const int d4 = d >> 2;
    const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kTpp;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / kTpp;
    const uint2 *pr = reinterpret_cast<const uint2 *>(pairs);
    const float4 *e4 = reinterpret_cast<const float4 *>(emb);
    for (int64_t v = grp; v < n; v += ngrp) {  // uniform per half-warp
        // sequences of more than heavy_min pairs are left to emb_grad_heavy_kernel
        if ((__ldg(off_i + v + 1) - __ldg(off_i + v)) + (__ldg(off_j + v + 1) - __ldg(off_j + v)) > heavy_min) continue;
        float4 acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        float beta = 0.f;
        for (int side = 0; side < 2; ++side) {
            const uint32_t *perm = side == 0 ? perm_i : perm_j;
            const uint32_t *off = side == 0 ? off_i : off_j;
            const uint32_t q0 = __ldg(off + v), q1 = __ldg(off + v + 1);
            for (uint32_t qb = q0; qb < q1; qb += kTpp) {
                const int cnt = (int)min((uint32_t)kTpp, q1 - qb);
                uint32_t other = 0;
                float cfx = 0.f, cfb = 0.f;
                if (sub < cnt) {
                    const uint32_t p = __ldg(perm + qb + sub);
                    const uint2 ij = __ldg(pr + p);
                    const float4 cf = __ldg(coef + p);
                    other = side == 0 ? ij.y : ij.x;
                    cfx = cf.x;
                    cfb = side == 0 ? cf.y : cf.z;
                }
                for (int t0 = 0; t0 < cnt; t0 += kRows) {
                    float4 row[kRows][CPL];
                    float cx[kRows], cb[kRows];
#pragma unroll
                    for (int u = 0; u < kRows; ++u) {
                        const int t = t0 + u;
                        const uint32_t o = __shfl_sync(hmask, other, t & (kTpp - 1), kTpp);
                        cx[u] = __shfl_sync(hmask, cfx, t & (kTpp - 1), kTpp);
                        cb[u] = __shfl_sync(hmask, cfb, t & (kTpp - 1), kTpp);
                        const float4 *eo = e4 + (int64_t)o * d4;
#pragma unroll
                        for (int c = 0; c < CPL; ++c) {
                            const int k = sub + c * kTpp;
                            row[u][c] = t < cnt && k < d4 ? __ldg(eo + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kRows; ++u) {
                        if (t0 + u >= cnt) break;
                        beta += cb[u];
#pragma unroll
                        for (int c = 0; c < CPL; ++c) {
                            acc[c].x = fmaf(cx[u], row[u][c].x, acc[c].x);
                            acc[c].y = fmaf(cx[u], row[u][c].y, acc[c].y);
                            acc[c].z = fmaf(cx[u], row[u][c].z, acc[c].z);
                            acc[c].w = fmaf(cx[u], row[u][c].w, acc[c].w);
                        }
                    }
                }
            }
        }
        const float4 *ev = e4 + v * d4;
        float4 *gv = reinterpret_cast<float4 *>(grad_emb + v * d);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int k = sub + c * kTpp;
            if (k < d4) {
                const float4 e = __ldg(ev + k);
                gv[k] = make_float4(fmaf(beta, e.x, acc[c].x), fmaf(beta, e.y, acc[c].y), fmaf(beta, e.z, acc[c].z),
                                    fmaf(beta, e.w, acc[c].w));
            }
        }
    }
}

// Sequences with more than heavy_min pairs, listed (in any order: each is
// computed on its own).
__global__ void heavy_list_kernel(const uint32_t *__restrict__ off_i, const uint32_t *__restrict__ off_j, int64_t n,
                                  uint32_t heavy_min, uint32_t *__restrict__ list, uint32_t *__restrict__ count)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if ((off_i[v + 1] - off_i[v]) + (off_j[v + 1] - off_j[v]) > heavy_min) list[atomicAdd(count, 1u)] = (uint32_t)v;
}

// One block per listed sequence: its D pairs (first-member side, then
// second-member side, each in index order) are cut into 16 consecutive
// parts, one per half-warp, each walked as in emb_grad_kernel; the 16 partial
// rows are summed in part order in shared memory, so the result is fixed by
// D alone.  Rows of at most 256 floats.
template <int CPL>
__global__ void __launch_bounds__(kFuseThreads) emb_grad_heavy_kernel(
    const uint32_t *__restrict__ pairs, const float4 *__restrict__ coef, const float *__restrict__ emb, int d,
    const uint32_t *__restrict__ perm_i, const uint32_t *__restrict__ off_i, const uint32_t *__restrict__ perm_j,
    const uint32_t *__restrict__ off_j, const uint32_t *__restrict__ list, const uint32_t *__restrict__ d_count,
    float *__restrict__ grad_emb)
{
    constexpr int kHalves = kFuseThreads / kTpp;
    constexpr int kRows = CPL <= 2 ? 4 : CPL <= 4 ? 2 : 1;
    extern __shared__ float s_part[];  // [kHalves][d + 1]: partial row, then partial beta
    const int half = threadIdx.x / kTpp, sub = threadIdx.x & (kTpp - 1);
    const unsigned hmask = 0xffffu << (threadIdx.x & 16);
    const int d4 = d >> 2;
    const uint2 *pr = reinterpret_cast<const uint2 *>(pairs);
    const float4 *e4 = reinterpret_cast<const float4 *>(emb);
    const uint32_t count = *d_count;
    for (uint32_t e = blockIdx.x; e < count; e += gridDim.x) {
        const uint32_t v = list[e];
        const uint32_t a0 = __ldg(off_i + v), b0 = __ldg(off_j + v);
        const uint32_t Di = __ldg(off_i + v + 1) - a0, D = Di + (__ldg(off_j + v + 1) - b0);
        const uint32_t t0 = (uint32_t)((uint64_t)D * half / kHalves);
        const uint32_t t1 = (uint32_t)((uint64_t)D * (half + 1) / kHalves);
        float4 acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        float beta = 0.f;
        for (uint32_t tb = t0; tb < t1; tb += kTpp) {  // uniform per half-warp
            const int cnt = (int)min((uint32_t)kTpp, t1 - tb);
            uint32_t other = 0;
            float cfx = 0.f, cfb = 0.f;
            if (sub < cnt) {
                const uint32_t t = tb + sub;
                const bool first = t < Di;
                const uint32_t p = first ? __ldg(perm_i + a0 + t) : __ldg(perm_j + b0 + (t - Di));
                const uint2 ij = __ldg(pr + p);
                const float4 cf = __ldg(coef + p);
                other = first ? ij.y : ij.x;
                cfx = cf.x;
                cfb = first ? cf.y : cf.z;
            }
            for (int u0 = 0; u0 < cnt; u0 += kRows) {
                float4 row[kRows][CPL];
                float cx[kRows], cb[kRows];
#pragma unroll
                for (int u = 0; u < kRows; ++u) {
                    const int t = u0 + u;
                    const uint32_t o = __shfl_sync(hmask, other, t & (kTpp - 1), kTpp);
                    cx[u] = __shfl_sync(hmask, cfx, t & (kTpp - 1), kTpp);
                    cb[u] = __shfl_sync(hmask, cfb, t & (kTpp - 1), kTpp);
                    const float4 *eo = e4 + (int64_t)o * d4;
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        const int k = sub + c * kTpp;
                        row[u][c] = t < cnt && k < d4 ? __ldg(eo + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int u = 0; u < kRows; ++u) {
                    if (u0 + u >= cnt) break;
                    beta += cb[u];
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        acc[c].x = fmaf(cx[u], row[u][c].x, acc[c].x);
                        acc[c].y = fmaf(cx[u], row[u][c].y, acc[c].y);
                        acc[c].z = fmaf(cx[u], row[u][c].z, acc[c].z);
                        acc[c].w = fmaf(cx[u], row[u][c].w, acc[c].w);
                    }
                }
            }
        }
        float *mine = s_part + half * (d + 1);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int k = sub + c * kTpp;
            if (k < d4) {
                mine[4 * k] = acc[c].x;
                mine[4 * k + 1] = acc[c].y;
                mine[4 * k + 2] = acc[c].z;
                mine[4 * k + 3] = acc[c].w;
            }
        }
        if (sub == 0) mine[d] = beta;
        __syncthreads();
        for (int f = threadIdx.x; f < d; f += blockDim.x) {
            float a = 0.f, bsum = 0.f;
            for (int h = 0; h < kHalves; ++h) {
                a += s_part[h * (d + 1) + f];
                bsum += s_part[h * (d + 1) + d];
            }
            grad_emb[(int64_t)v * d + f] = fmaf(bsum, __ldg(emb + (int64_t)v * d + f), a);
        }
        __syncthreads();  // s_part is rewritten for the next sequence
    }
}

// Embedding gradient through the pair index: sequences of at most
// kHeavyPairs pairs by one half-warp each (emb_grad_kernel), longer ones by a
// block each (emb_grad_heavy_kernel, rows of at most 256 floats); list and
// count in the caller's scratch.
constexpr uint32_t kHeavyPairs = 128;

int launch_emb_grad(subquad_ctx *ctx, const uint32_t *pairs, const float4 *coef, const float *emb, int64_t n, int d,
                    const uint32_t *perm_i, const uint32_t *off_i, const uint32_t *perm_j, const uint32_t *off_j,
                    float *grad_emb, uint32_t *heavy_list, uint32_t *heavy_count)
{
    const int cpl = (d / 4 + kTpp - 1) / kTpp;
    const bool heavy = d <= 4 * 4 * kTpp;
    const uint32_t heavy_min = heavy ? kHeavyPairs : 0xffffffffu;
    const unsigned g2 = sq_grid(ctx, n * kTpp, kFuseThreads, 8);
#define SQ_EMB(C)                                                                                                  \
    emb_grad_kernel<C><<<sq_resident_grid(ctx, emb_grad_kernel<C>, kFuseThreads, 0, g2), kFuseThreads, 0,          \
                         ctx->stream>>>(pairs, coef, emb, n, d, perm_i, off_i, perm_j, off_j, grad_emb, heavy_min)
    if (cpl <= 1) SQ_EMB(1);
    else if (cpl <= 2) SQ_EMB(2);
    else if (cpl <= 4) SQ_EMB(4);
    else if (cpl <= 8) SQ_EMB(8);
    else SQ_EMB(16);
#undef SQ_EMB
    SQ_LAUNCH_CHECK();
    if (!heavy) return SUBQUAD_OK;
    SQ_TRY_CUDA(cudaMemsetAsync(heavy_count, 0, sizeof(uint32_t), ctx->stream));
    heavy_list_kernel<<<sq_grid(ctx, n, 256, 8), 256, 0, ctx->stream>>>(off_i, off_j, n, heavy_min, heavy_list,
                                                                          heavy_count);
    SQ_LAUNCH_CHECK();
    const size_t smem = sizeof(float) * (kFuseThreads / kTpp) * (size_t)(d + 1);
    const unsigned g3 = (unsigned)ctx->num_sms * 4;
#define SQ_EMBH(C)                                                                                                 \
    emb_grad_heavy_kernel<C><<<g3, kFuseThreads, smem, ctx->stream>>>(pairs, coef, emb, d, perm_i, off_i, perm_j,   \
                                                                     off_j, heavy_list, heavy_count, grad_emb)
    if (cpl <= 1) SQ_EMBH(1);
    else if (cpl <= 2) SQ_EMBH(2);
    else SQ_EMBH(4);
#undef SQ_EMBH
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

template <int WORDS, int CPL>
int launch_backward_cpl(subquad_ctx *ctx, unsigned grid, const uint32_t *pairs, int64_t m, const int32_t *sw,
                        const int32_t *self_scores, const void *packed, const float *emb, int d,
                        const float *gate_params, int hidden, const float *dL, float4 *coef, double *partials)
{
    const int hpl = (hidden + kTpp - 1) / kTpp;
    const size_t smem = sizeof(double) * kGroups * (5 * hidden + 1);
#define SQ_BWD(H)                                                                                                  \
    do {                                                                                                           \
        auto kern = fuse_backward_kernel<WORDS, CPL, H>;                                                           \
        SQ_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));           \
        kern<<<grid, kFuseThreads, smem, ctx->stream>>>(pairs, m, sw, self_scores, (const uint64_t *)packed, emb, d,  \
                                                        gate_params, hidden, dL, coef, partials);                  \
    } while (0)
    if (hpl <= 1) SQ_BWD(1);
    else if (hpl <= 2) SQ_BWD(2);
    else SQ_BWD(4);
#undef SQ_BWD
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

template <int WORDS>
int launch_backward(subquad_ctx *ctx, unsigned grid, const uint32_t *pairs, int64_t m, const int32_t *sw,
                    const int32_t *self_scores, const void *packed, const float *emb, int d, const float *gate_params,
                    int hidden, const float *dL, float4 *coef, double *partials)
{
    const int cpl = (d / 4 + kTpp - 1) / kTpp;
    if (cpl <= 1)
        return launch_backward_cpl<WORDS, 1>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden,
                                             dL, coef, partials);
    if (cpl <= 2)
        return launch_backward_cpl<WORDS, 2>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden,
                                             dL, coef, partials);
    if (cpl <= 4)
        return launch_backward_cpl<WORDS, 4>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden,
                                             dL, coef, partials);
    if (cpl <= 8)
        return launch_backward_cpl<WORDS, 8>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden,
                                             dL, coef, partials);
    return launch_backward_cpl<WORDS, 16>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden, dL,
                                          coef, partials);
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
    const unsigned grid = sq_grid(ctx, (m + 7) / 8 * 32, kFuseThreads, 8);
    if (pack_stride == 16)
        return launch_forward<2>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden, fused_out,
                                 alpha_out);
    return launch_forward<4>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden, fused_out,
                             alpha_out);
}

extern "C" int subquad_fuse_backward(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                                     const int32_t *self_scores, const void *packed, int pack_stride, const float *emb,
                                     int64_t n, int d, const float *gate_params, int hidden, const float *dL_dfused,
                                     const uint32_t *perm_i, const uint32_t *off_i, const uint32_t *perm_j,
                                     const uint32_t *off_j, float *grad_params, float *grad_emb)
{
    SQ_ENTER(ctx);
    if (m < 0 || n < 0 || d < 4 || d > 1024 || d % 4 || hidden < 1 || hidden > kMaxHidden) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (!grad_params || !gate_params) return SUBQUAD_ERR_ARG;
    if (m > 0 && (!pairs || !sw || !self_scores || !packed || !emb || !dL_dfused)) return SUBQUAD_ERR_ARG;
    if (grad_emb && (!perm_i || !off_i || !perm_j || !off_j || !emb)) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(emb) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8 ||
        reinterpret_cast<uintptr_t>(packed) % 16 || reinterpret_cast<uintptr_t>(grad_emb) % 16)
        return SUBQUAD_ERR_ARG;
    const int P = 5 * hidden + 1;
    // a fixed grid keeps the reduction order (and so the result) independent of m
    const unsigned grid = (unsigned)ctx->num_sms * 4;
    SqArena measure(nullptr);
    measure.take<double>((size_t)grid * P);
    if (grad_emb) {
        measure.take<float4>((size_t)m);
        measure.take<uint32_t>((size_t)n + 1);
    }
    SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    SqArena arena(ctx->scratch);
    double *partials = arena.take<double>((size_t)grid * P);
    float4 *coef = grad_emb ? arena.take<float4>((size_t)m) : nullptr;
    uint32_t *heavy_list = grad_emb ? arena.take<uint32_t>((size_t)n + 1) : nullptr;
    uint32_t *heavy_count = heavy_list ? heavy_list + n : nullptr;
    if (pack_stride == 16)
        SQ_TRY(launch_backward<2>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden, dL_dfused,
                                  coef, partials));
    else
        SQ_TRY(launch_backward<4>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden, dL_dfused,
                                  coef, partials));
    reduce_partials_kernel<<<1, 352, 0, ctx->stream>>>(partials, (int)grid, P, grad_params);
    SQ_LAUNCH_CHECK();
    if (grad_emb && n > 0)
        SQ_TRY(launch_emb_grad(ctx, pairs, coef, emb, n, d, perm_i, off_i, perm_j, off_j, grad_emb, heavy_list,
                               heavy_count));
    return SUBQUAD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free parameter gradient
// ---------------------------------------------------------------------------
// Some callers cannot let a library call cudaMalloc: a training step that runs
// while a caching allocator owns the device's free memory, code that must not
// take cudaMalloc's implicit device synchronisation inside a latency-bound
// loop, or hosts whose allocation policy forbids driver allocations.  For them
// the parameter gradient of the fusion adjoint can keep its block partials in
// this file-scope device array instead of context scratch.  Every GPU that
// loads the library holds the array until the process exits.
constexpr size_t kStaticPartialBytes = size_t(2) << 20;  // 2 MiB
constexpr size_t kStaticPartialDoubles = kStaticPartialBytes / sizeof(double);
static __device__ __align__(256) double g_static_partials[kStaticPartialDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double *g_static_ptr[kMaxDevices] = {};

// Device address of g_static_partials on `device` (which must be current):
// the host-side symbol is only a stand-in, so the address is looked up once
// per device and cached for the life of the process (a device reset, which
// reloads the module, would leave the cached address stale).
int static_partials(int device, double **out)
{
    if (device < 0 || device >= kMaxDevices) return SUBQUAD_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[device]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_partials);
        if (e != cudaSuccess) {
            sq_note_cuda_error(e);
            return SUBQUAD_ERR_CUDA;
        }
        g_static_ptr[device] = static_cast<double *>(ptr);
    }
    *out = g_static_ptr[device];
    return SUBQUAD_OK;
}

}  // namespace

extern "C" int subquad_fuse_backward_params_noalloc(subquad_ctx *ctx, const uint32_t *pairs, int64_t m,
                                                    const int32_t *sw, const int32_t *self_scores, const void *packed,
                                                    int pack_stride, const float *emb, int d,
                                                    const float *gate_params, int hidden, const float *dL_dfused,
                                                    float *grad_params)
{
    SQ_ENTER(ctx);
    if (m < 0 || d < 4 || d > 1024 || d % 4 || hidden < 1 || hidden > kMaxHidden) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (!grad_params || !gate_params) return SUBQUAD_ERR_ARG;
    if (m > 0 && (!pairs || !sw || !self_scores || !packed || !emb || !dL_dfused)) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(emb) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8 ||
        reinterpret_cast<uintptr_t>(packed) % 16)
        return SUBQUAD_ERR_ARG;
    const int P = 5 * hidden + 1;
    const unsigned grid = (unsigned)ctx->num_sms * 4;  // the same grid as subquad_fuse_backward
    if ((size_t)grid * P > kStaticPartialDoubles) return SUBQUAD_ERR_ARG;  // partials would not fit
    double *partials = nullptr;
    SQ_TRY(static_partials(ctx->device, &partials));
    // every block overwrites all of its P partials, so nothing needs clearing
    if (pack_stride == 16)
        SQ_TRY(launch_backward<2>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden, dL_dfused,
                                  nullptr, partials));
    else
        SQ_TRY(launch_backward<4>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, gate_params, hidden, dL_dfused,
                                  nullptr, partials));
    reduce_partials_kernel<<<1, 352, 0, ctx->stream>>>(partials, (int)grid, P, grad_params);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

extern "C" int subquad_fuse_forward_async(subquad_ctx *ctx, const uint32_t *pairs, const uint64_t *d_m, int64_t m_max,
                                          const int32_t *sw, const int32_t *self_scores, const void *packed,
                                          int pack_stride, const float *emb, int d, const float *gate_params,
                                          int hidden, float *fused_out, float *alpha_out)
{
    SQ_ENTER(ctx);
    if (!d_m || m_max < 0 || d < 4 || d > 1024 || d % 4 || hidden < 1 || hidden > kMaxHidden) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (m_max == 0) return SUBQUAD_OK;
    if (!pairs || !sw || !self_scores || !packed || !emb || !gate_params || !fused_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(emb) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8 ||
        reinterpret_cast<uintptr_t>(packed) % 16)
        return SUBQUAD_ERR_ARG;
    const unsigned grid = sq_grid(ctx, (m_max + 7) / 8 * 32, kFuseThreads, 8);
    const auto *dm = reinterpret_cast<const unsigned long long *>(d_m);
    if (pack_stride == 16)
        return launch_forward<2>(ctx, grid, pairs, m_max, sw, self_scores, packed, emb, d, gate_params, hidden,
                                 fused_out, alpha_out, dm);
    return launch_forward<4>(ctx, grid, pairs, m_max, sw, self_scores, packed, emb, d, gate_params, hidden, fused_out,
                             alpha_out, dm);
}

// ---------------------------------------------------------------------------
// M-channel fusion (Eq. wm with M > 2, Eq. afused): channels s, c' = (1+c)/2
// and, for M = 3, J = the fraction of the H MinHash rows on which the two
// signatures agree (the sketch's estimate of the k-mer Jaccard index).  One
// gate MLP scores the channels from f = [s, c, |dL|, J]: its M - 1 outputs
// are the logits of channels 1 and 3, channel 2 keeps logit 0, and the
// weights are the softmax of the logits.  Parameters: W1 [h][M+1], b1 [h],
// W2 [M-1][h], b2 [M-1] (for M = 2 the layout of the two-channel gate).
// The forward uses four lanes per pair like the two-channel kernel; the
// signature rows of a band are one 16-byte vector per sequence when rows ==
// 4 (the library's layout [band][n][rows]), so lane q compares bands q,
// q + 4, ... with one vector load per member.
// ---------------------------------------------------------------------------
namespace {

// Agreeing signature rows of sequences i and j, summed over the hashes this
// lane owns.  sig_seq is sequence-major (uint32 [n][H], the layout of
// subquad_sig_sequence_major), so a member's H words are one contiguous row:
// with H % 4 == 0 lane q compares 16-byte chunks q, q + LANES, ... of the two
// rows (a pair's lanes read consecutive chunks), else single words.
template <int LANES, int V = 1>
__device__ __forceinline__ int sig_agree(const uint32_t *__restrict__ sig_seq, int H, uint32_t i, uint32_t j, int sub,
                                         bool valid)
{
    int agree = 0;
    if (!valid) return 0;
    if (V == 2) {  // H % 8 == 0, rows 32-byte aligned: 32-byte chunks, a pair's lanes read whole lines
        const int H8 = H >> 3;
        const uint32_t *ri = sig_seq + (int64_t)i * H, *rj = sig_seq + (int64_t)j * H;
        for (int c = sub; c < H8; c += LANES) {
            uint4 x0, x1, y0, y1;
            ldg_v8u(ri + 8 * c, x0, x1);
            ldg_v8u(rj + 8 * c, y0, y1);
            agree += (x0.x == y0.x) + (x0.y == y0.y) + (x0.z == y0.z) + (x0.w == y0.w) + (x1.x == y1.x) +
                     (x1.y == y1.y) + (x1.z == y1.z) + (x1.w == y1.w);
        }
    } else if ((H & 3) == 0) {
        const int H4 = H >> 2;
        const uint4 *ri = reinterpret_cast<const uint4 *>(sig_seq) + (int64_t)i * H4;
        const uint4 *rj = reinterpret_cast<const uint4 *>(sig_seq) + (int64_t)j * H4;
        for (int c = sub; c < H4; c += LANES) {
            const uint4 x = __ldg(ri + c), y = __ldg(rj + c);
            agree += (x.x == y.x) + (x.y == y.y) + (x.z == y.z) + (x.w == y.w);
        }
    } else {
        for (int t = sub; t < H; t += LANES)
            agree += __ldg(sig_seq + (int64_t)i * H + t) == __ldg(sig_seq + (int64_t)j * H + t);
    }
    return agree;
}

// [bands][n][rows] -> [n][bands * rows].  rows == 4: a block takes 64
// sequences, reads every band's 16-byte vectors of them (64 consecutive
// vectors per band: coalesced) into shared memory, then writes the 64 rows,
// which are contiguous in the output, as consecutive 16-byte chunks
// (coalesced).  Other rows: one thread per sequence, word by word.
constexpr int kTrSeq = 64;

__global__ void __launch_bounds__(256) sig_transpose4_kernel(const uint4 *__restrict__ sig, int64_t n, int bands,
                                                              uint4 *__restrict__ out)
{
    extern __shared__ uint4 s_v[];  // [kTrSeq][bands]
    for (int64_t i0 = (int64_t)blockIdx.x * kTrSeq; i0 < n; i0 += (int64_t)gridDim.x * kTrSeq) {
        const int cnt = n - i0 < kTrSeq ? (int)(n - i0) : kTrSeq;
        for (int q = threadIdx.x; q < cnt * bands; q += blockDim.x) {
            const int b = q / cnt, il = q - b * cnt;
            s_v[il * bands + b] = __ldg(sig + (int64_t)b * n + i0 + il);
        }
        __syncthreads();
        uint4 *dst = out + i0 * bands;
        for (int q = threadIdx.x; q < cnt * bands; q += blockDim.x) dst[q] = s_v[q];
        __syncthreads();
    }
}

__global__ void sig_transpose_kernel(const uint32_t *__restrict__ sig, int64_t n, int bands, int rows,
                                     uint32_t *__restrict__ out)
{
    const int H = bands * rows;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int b = 0; b < bands; ++b)
            for (int r = 0; r < rows; ++r) out[i * H + b * rows + r] = __ldg(sig + ((int64_t)b * n + i) * rows + r);
}

// Parameter offsets of the M-channel gate.
struct McLayout {
    int F, W1, b1, W2, b2, P;
    __host__ __device__ McLayout(int M, int h)
        : F(M + 1), W1(0), b1((M + 1) * h), W2((M + 2) * h), b2((2 * M + 1) * h), P((2 * M + 1) * h + M - 1)
    {
    }
};

template <int M, int WORDS, int CPL, int V = 1>
__global__ void __launch_bounds__(kFuseThreads) fuse_forward_mc_kernel(
    const uint32_t *__restrict__ pairs, int64_t m, const int32_t *__restrict__ sw, const int32_t *__restrict__ self_sc,
    const uint64_t *__restrict__ packed, const float *__restrict__ emb, int d, const uint32_t *__restrict__ sig,
    int H, const float *__restrict__ params, int hidden, float *__restrict__ fused, float *__restrict__ weights)
{
    constexpr int F = M + 1;
    __shared__ float s_w1[kMaxHidden * F];
    __shared__ float s_b1[kMaxHidden];
    __shared__ float s_w2[(M - 1) * kMaxHidden];
    __shared__ float s_b2[M - 1];
    const McLayout L(M, hidden);
    for (int q = threadIdx.x; q < hidden * F; q += blockDim.x) s_w1[q] = params[L.W1 + q];
    for (int q = threadIdx.x; q < hidden; q += blockDim.x) s_b1[q] = params[L.b1 + q];
    for (int q = threadIdx.x; q < (M - 1) * hidden; q += blockDim.x) s_w2[q] = params[L.W2 + q];
    if (threadIdx.x < M - 1) s_b2[threadIdx.x] = params[L.b2 + threadIdx.x];
    __syncthreads();
    constexpr int kPairsPerWarp = 32 / kTppF;
    const int sub = threadIdx.x & (kTppF - 1);
    const int slot = (threadIdx.x & 31) / kTppF;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d4 = d >> 2;
    for (int64_t pbase = warp * kPairsPerWarp; pbase < m; pbase += nwarps * kPairsPerWarp) {
        const int64_t p = pbase + slot;
        const bool valid = p < m;
        const uint2 ij = valid ? __ldg(reinterpret_cast<const uint2 *>(pairs) + p) : make_uint2(0, 0);
        PairInputs<WORDS, CPL, kTppF, V> in;
        in.load(ij, p, valid, sub, d4, emb, d, sw, self_sc, packed);
        int agree = M == 3 ? sig_agree<kTppF, V>(sig, H, ij.x, ij.y, sub, valid) : 0;
        float dot = 0.f, sii = 0.f, sjj = 0.f;
#pragma unroll
        for (int c = 0; c < CPL * V; ++c) {
            const float4 a = in.a[c], b = in.b[c];
            dot = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, dot))));
            sii = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, sii))));
            sjj = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, sjj))));
        }
        dot = quad_sum(dot);
        sii = quad_sum(sii);
        sjj = quad_sum(sjj);
        if (M == 3) {
            agree += __shfl_xor_sync(0xffffffffu, agree, 2, kTppF);
            agree += __shfl_xor_sync(0xffffffffu, agree, 1, kTppF);
        }
        const float prod = (float)in.self_i * (float)in.self_j;
        const float s = prod > 0.f ? (float)in.sw * rsqrtf(prod) : 0.f;
        const float nn = sii * sjj;
        const float c = nn > 0.f ? dot * rsqrtf(nn) : 0.f;
        const float delta = fabsf((float)(in.len_i - in.len_j));
        const float J = M == 3 ? (float)agree / (float)H : 0.f;
        float acc0 = 0.f, acc1 = 0.f;
        for (int k = sub; k < hidden; k += kTppF) {
            const float *w = s_w1 + k * F;
            float z = fmaf(w[0], s, fmaf(w[1], c, fmaf(w[2], delta, s_b1[k])));
            if (M == 3) z = fmaf(w[3], J, z);
            const float u = fmaxf(z, 0.f);
            acc0 = fmaf(s_w2[k], u, acc0);
            if (M == 3) acc1 = fmaf(s_w2[hidden + k], u, acc1);
        }
        const float g1 = quad_sum(acc0) + s_b2[0];
        const float g3 = M == 3 ? quad_sum(acc1) + s_b2[M - 2] : 0.f;
        if (valid && sub == 0) {
            const float cp = 0.5f * (1.f + c);
            const float mx = M == 3 ? fmaxf(fmaxf(g1, 0.f), g3) : fmaxf(g1, 0.f);
            const float e1 = __expf(g1 - mx), e2 = __expf(-mx), e3 = M == 3 ? __expf(g3 - mx) : 0.f;
            const float inv = __fdividef(1.f, e1 + e2 + e3);
            const float w1 = e1 * inv, w2 = e2 * inv, w3 = e3 * inv;
            fused[p] = M == 3 ? fmaf(w1, s, fmaf(w2, cp, w3 * J)) : fmaf(w1, s, w2 * cp);
            if (weights) {
                weights[p * M] = w1;
                weights[p * M + 1] = w2;
                if (M == 3) weights[p * M + 2] = w3;
            }
        }
    }
}

// Adjoint of the M-channel fusion: sixteen lanes per pair as in the
// two-channel adjoint; d fused / d g_k = w_k (a_k - fused) for the two MLP
// outputs, then W2, the ReLU and W1; the cosine receives w_2 / 2 from the
// channel c' and W1[k][1] dz_k from the feature c.
template <int M, int WORDS, int CPL, int HPL>
__global__ void __launch_bounds__(kFuseThreads) fuse_backward_mc_kernel(
    const uint32_t *__restrict__ pairs, int64_t m, const int32_t *__restrict__ sw, const int32_t *__restrict__ self_sc,
    const uint64_t *__restrict__ packed, const float *__restrict__ emb, int d, const uint32_t *__restrict__ sig,
    int H, const float *__restrict__ params, int hidden, const float *__restrict__ dL, float4 *__restrict__ coef,
    double *__restrict__ partials)
{
    constexpr int F = M + 1;
    __shared__ float s_par[(2 * M + 1) * kMaxHidden + M - 1];
    extern __shared__ double s_red[];  // [kGroups][P]
    const McLayout L(M, hidden);
    const int P = L.P;
    for (int q = threadIdx.x; q < P; q += blockDim.x) s_par[q] = params[q];
    __syncthreads();
    const float *W1 = s_par + L.W1, *b1 = s_par + L.b1, *W2 = s_par + L.W2, *b2 = s_par + L.b2;
    const int sub = threadIdx.x & (kTpp - 1);
    const int half = (threadIdx.x >> 4) & 1;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d4 = d >> 2;
    Kahan gW1[HPL][F], gb1[HPL], gW2[HPL][M - 1], gb2[M - 1];
    const uint2 *pr = reinterpret_cast<const uint2 *>(pairs);
    uint2 ij_next = warp * 2 + half < m ? __ldg(pr + warp * 2 + half) : make_uint2(0, 0);  // one iteration ahead
    for (int64_t pbase = warp * 2; pbase < m; pbase += nwarps * 2) {
        const int64_t p = pbase + half;
        const bool valid = p < m;
        const uint2 ij = valid ? ij_next : make_uint2(0, 0);
        ij_next = p + nwarps * 2 < m ? __ldg(pr + p + nwarps * 2) : make_uint2(0, 0);
        PairInputs<WORDS, CPL> in;
        in.load(ij, p, valid, sub, d4, emb, d, sw, self_sc, packed);
        const float dA = valid ? __ldg(dL + p) : 0.f;
        int agree = M == 3 ? sig_agree<kTpp>(sig, H, ij.x, ij.y, sub, valid) : 0;
        float dot = 0.f, sii = 0.f, sjj = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const float4 a = in.a[c], b = in.b[c];
            dot = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w))) + dot;
            sii = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, a.w * a.w))) + sii;
            sjj = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, b.w * b.w))) + sjj;
        }
        dot = group_sum(dot);
        sii = group_sum(sii);
        sjj = group_sum(sjj);
        if (M == 3) {
#pragma unroll
            for (int o = kTpp / 2; o > 0; o >>= 1) agree += __shfl_xor_sync(0xffffffffu, agree, o, kTpp);
        }
        const float prod = (float)in.self_i * (float)in.self_j;
        const float s = prod > 0.f ? (float)in.sw * rsqrtf(prod) : 0.f;  // as the forward
        const float nn = sii * sjj;
        const float c = nn > 0.f ? dot * rsqrtf(nn) : 0.f;
        const float f[4] = {s, c, fabsf((float)(in.len_i - in.len_j)), M == 3 ? (float)agree / (float)H : 0.f};
        float z[HPL];
        float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
        for (int hh = 0; hh < HPL; ++hh) {
            const int k = sub + hh * kTpp;
            z[hh] = 0.f;
            if (k < hidden) {
                float t = b1[k];
#pragma unroll
                for (int q = F - 1; q >= 0; --q) t = fmaf(W1[k * F + q], f[q], t);
                z[hh] = t;
                const float u = fmaxf(t, 0.f);
                acc0 = fmaf(W2[k], u, acc0);
                if (M == 3) acc1 = fmaf(W2[hidden + k], u, acc1);
            }
        }
        const float g1 = group_sum(acc0) + b2[0];
        const float g3 = M == 3 ? group_sum(acc1) + b2[M - 2] : 0.f;
        const float mx = M == 3 ? fmaxf(fmaxf(g1, 0.f), g3) : fmaxf(g1, 0.f);
        const float e1 = __expf(g1 - mx), e2 = __expf(-mx), e3 = M == 3 ? __expf(g3 - mx) : 0.f;
        const float den = e1 + e2 + e3;
        const float inv_den = __fdividef(1.f, den);
        const float w1 = e1 * inv_den, w2 = e2 * inv_den, w3 = e3 * inv_den;
        const float cp = 0.5f * (1.f + c);
        const float fused = M == 3 ? w1 * s + w2 * cp + w3 * f[3] : w1 * s + w2 * cp;
        const float d0 = dA * w1 * (s - fused);
        const float d1 = M == 3 ? dA * w3 * (f[3] - fused) : 0.f;
        float dc = 0.f;
#pragma unroll
        for (int hh = 0; hh < HPL; ++hh) {
            const int k = sub + hh * kTpp;
            if (k < hidden && valid) {
                const float u = fmaxf(z[hh], 0.f);
                gW2[hh][0].add(d0 * u);
                float du = d0 * W2[k];
                if (M == 3) {
                    gW2[hh][M - 2].add(d1 * u);
                    du = fmaf(d1, W2[hidden + k], du);
                }
                const float dz = z[hh] > 0.f ? du : 0.f;
#pragma unroll
                for (int q = 0; q < F; ++q) gW1[hh][q].add(dz * f[q]);
                gb1[hh].add(dz);
                dc = fmaf(dz, W1[k * F + 1], dc);
            }
        }
        dc = group_sum(dc) + dA * w2 * 0.5f;
        if (sub == 0 && valid) {
            gb2[0].add(d0);
            if (M == 3) gb2[M - 2].add(d1);
            if (coef) {
                float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
                if (sii > 0.f && sjj > 0.f) {
                    cf.x = dc * rsqrtf(sii * sjj);
                    cf.y = __fdividef(-dc * c, sii);
                    cf.z = __fdividef(-dc * c, sjj);
                }
                coef[p] = cf;
            }
        }
    }
    const int grp = threadIdx.x / kTpp;
    double *mine = s_red + (size_t)grp * P;
#pragma unroll
    for (int hh = 0; hh < HPL; ++hh) {
        const int k = sub + hh * kTpp;
        if (k < hidden) {
#pragma unroll
            for (int q = 0; q < F; ++q) mine[L.W1 + k * F + q] = gW1[hh][q].value();
            mine[L.b1 + k] = gb1[hh].value();
#pragma unroll
            for (int r = 0; r < M - 1; ++r) mine[L.W2 + r * hidden + k] = gW2[hh][r].value();
        }
    }
    if (sub == 0)
        for (int r = 0; r < M - 1; ++r) mine[L.b2 + r] = gb2[r].value();
    __syncthreads();
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        double t = 0.0;
        for (int gi = 0; gi < kGroups; ++gi) t += s_red[(size_t)gi * P + q];
        partials[(int64_t)blockIdx.x * P + q] = t;
    }
}

template <int M, int WORDS>
int launch_forward_mc(subquad_ctx *ctx, unsigned grid, const uint32_t *pairs, int64_t m, const int32_t *sw,
                      const int32_t *self_scores, const void *packed, const float *emb, int d, const uint32_t *sig,
                      int H, const float *params, int hidden, float *fused, float *weights)
{
    SqProfScope prof(ctx, SUBQUAD_PROF_FUSE);
    if (d % 8 == 0 && d <= 8 * 4 * kTppF && reinterpret_cast<uintptr_t>(emb) % 32 == 0 &&
        (M == 2 || (H % 8 == 0 && reinterpret_cast<uintptr_t>(sig) % 32 == 0))) {
        // 32-byte lane loads of the rows and signatures (whole lines per pair and load)
        const int cpl8 = (d / 8 + kTppF - 1) / kTppF;
#define SQ_FWDMC8(C)                                                                                               \
    fuse_forward_mc_kernel<M, WORDS, C, 2><<<sq_resident_grid(ctx, fuse_forward_mc_kernel<M, WORDS, C, 2>,          \
                                                              kFuseThreads, 0, grid),                              \
                                             kFuseThreads, 0, ctx->stream>>>(                                      \
        pairs, m, sw, self_scores, (const uint64_t *)packed, emb, d, sig, H, params, hidden, fused, weights)
        if (cpl8 <= 1) SQ_FWDMC8(1);
        else if (cpl8 <= 2) SQ_FWDMC8(2);
        else SQ_FWDMC8(4);
#undef SQ_FWDMC8
        SQ_LAUNCH_CHECK();
        return SUBQUAD_OK;
    }
    const int cpl = (d / 4 + kTppF - 1) / kTppF;
#define SQ_FWDMC(C)                                                                                                \
    fuse_forward_mc_kernel<M, WORDS, C><<<sq_resident_grid(ctx, fuse_forward_mc_kernel<M, WORDS, C>, kFuseThreads, \
                                                           0, grid),                                               \
                                          kFuseThreads, 0, ctx->stream>>>(                                         \
        pairs, m, sw, self_scores, (const uint64_t *)packed, emb, d, sig, H, params, hidden, fused, weights)
    if (cpl <= 1) SQ_FWDMC(1);
    else if (cpl <= 2) SQ_FWDMC(2);
    else if (cpl <= 4) SQ_FWDMC(4);
    else if (cpl <= 8) SQ_FWDMC(8);
    else if (cpl <= 16) SQ_FWDMC(16);
    else if (cpl <= 32) SQ_FWDMC(32);
    else SQ_FWDMC(64);
#undef SQ_FWDMC
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

template <int M, int WORDS, int CPL>
int launch_backward_mc_cpl(subquad_ctx *ctx, unsigned grid, const uint32_t *pairs, int64_t m, const int32_t *sw,
                           const int32_t *self_scores, const void *packed, const float *emb, int d,
                           const uint32_t *sig, int H, const float *params, int hidden, const float *dL, float4 *coef,
                           double *partials)
{
    const int hpl = (hidden + kTpp - 1) / kTpp;
    const size_t smem = sizeof(double) * kGroups * McLayout(M, hidden).P;
#define SQ_BWDMC(HH)                                                                                               \
    do {                                                                                                           \
        auto kern = fuse_backward_mc_kernel<M, WORDS, CPL, HH>;                                                    \
        SQ_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));           \
        kern<<<grid, kFuseThreads, smem, ctx->stream>>>(pairs, m, sw, self_scores, (const uint64_t *)packed, emb, d,  \
                                                        sig, H, params, hidden, dL, coef, partials);               \
    } while (0)
    if (hpl <= 1) SQ_BWDMC(1);
    else if (hpl <= 2) SQ_BWDMC(2);
    else SQ_BWDMC(4);
#undef SQ_BWDMC
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

template <int M, int WORDS>
int launch_backward_mc(subquad_ctx *ctx, unsigned grid, const uint32_t *pairs, int64_t m, const int32_t *sw,
                       const int32_t *self_scores, const void *packed, const float *emb, int d, const uint32_t *sig,
                       int H, const float *params, int hidden, const float *dL, float4 *coef, double *partials)
{
    const int cpl = (d / 4 + kTpp - 1) / kTpp;
#define SQ_BMC(C)                                                                                                  \
    return launch_backward_mc_cpl<M, WORDS, C>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, sig, H, params, \
                                               hidden, dL, coef, partials)
    if (cpl <= 1) SQ_BMC(1);
    if (cpl <= 2) SQ_BMC(2);
    if (cpl <= 4) SQ_BMC(4);
    if (cpl <= 8) SQ_BMC(8);
    SQ_BMC(16);
#undef SQ_BMC
}

int check_mc_args(int64_t m, int64_t n, int d, int hidden, int channels, int pack_stride, const uint32_t *sig, int H)
{
    if (m < 0 || n < 0 || d < 4 || d > 1024 || d % 4 || hidden < 1 || hidden > kMaxHidden) return SUBQUAD_ERR_ARG;
    if (channels != 2 && channels != 3) return SUBQUAD_ERR_ARG;
    if (pack_stride != 16 && pack_stride != 32) return SUBQUAD_ERR_ARG;
    if (channels == 3) {
        if (!sig || H < 1 || H > 512) return SUBQUAD_ERR_ARG;
        if (reinterpret_cast<uintptr_t>(sig) % ((H & 3) == 0 ? 16 : 4)) return SUBQUAD_ERR_ARG;
    }
    return SUBQUAD_OK;
}

}  // namespace

extern "C" int subquad_fuse_forward_mc(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                                       const int32_t *self_scores, const void *packed, int pack_stride,
                                       const float *emb, int d, const uint32_t *sig_seq, int hashes,
                                       const float *gate_params, int hidden, int channels, float *fused_out,
                                       float *weights_out)
{
    SQ_ENTER(ctx);
    SQ_TRY(check_mc_args(m, 0, d, hidden, channels, pack_stride, sig_seq, hashes));
    if (m == 0) return SUBQUAD_OK;
    if (!pairs || !sw || !self_scores || !packed || !emb || !gate_params || !fused_out) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(emb) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8 ||
        reinterpret_cast<uintptr_t>(packed) % 16)
        return SUBQUAD_ERR_ARG;
    const unsigned grid = sq_grid(ctx, (m + 7) / 8 * 32, kFuseThreads, 8);
#define SQ_MCF(MM, W)                                                                                              \
    return launch_forward_mc<MM, W>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, sig_seq, hashes,         \
                                    gate_params, hidden, fused_out, weights_out)
    if (channels == 2) {
        if (pack_stride == 16) SQ_MCF(2, 2);
        SQ_MCF(2, 4);
    }
    if (pack_stride == 16) SQ_MCF(3, 2);
    SQ_MCF(3, 4);
#undef SQ_MCF
}

extern "C" int subquad_fuse_backward_mc(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                                        const int32_t *self_scores, const void *packed, int pack_stride,
                                        const float *emb, int64_t n, int d, const uint32_t *sig_seq, int hashes,
                                        const float *gate_params, int hidden, int channels, const float *dL_dfused,
                                        const uint32_t *perm_i, const uint32_t *off_i, const uint32_t *perm_j,
                                        const uint32_t *off_j, float *grad_params, float *grad_emb)
{
    SQ_ENTER(ctx);
    SQ_TRY(check_mc_args(m, n, d, hidden, channels, pack_stride, sig_seq, hashes));
    if (!grad_params || !gate_params) return SUBQUAD_ERR_ARG;
    if (m > 0 && (!pairs || !sw || !self_scores || !packed || !emb || !dL_dfused)) return SUBQUAD_ERR_ARG;
    if (grad_emb && (!perm_i || !off_i || !perm_j || !off_j || !emb)) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(emb) % 16 || reinterpret_cast<uintptr_t>(pairs) % 8 ||
        reinterpret_cast<uintptr_t>(packed) % 16 || reinterpret_cast<uintptr_t>(grad_emb) % 16)
        return SUBQUAD_ERR_ARG;
    const int P = McLayout(channels, hidden).P;
    const unsigned grid = (unsigned)ctx->num_sms * 4;  // fixed: the reduction order does not depend on m
    SqArena measure(nullptr);
    measure.take<double>((size_t)grid * P);
    if (grad_emb) {
        measure.take<float4>((size_t)m);
        measure.take<uint32_t>((size_t)n + 1);
    }
    SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    SqArena arena(ctx->scratch);
    double *partials = arena.take<double>((size_t)grid * P);
    float4 *coef = grad_emb ? arena.take<float4>((size_t)m) : nullptr;
    uint32_t *heavy_list = grad_emb ? arena.take<uint32_t>((size_t)n + 1) : nullptr;
    uint32_t *heavy_count = heavy_list ? heavy_list + n : nullptr;
#define SQ_MCB(MM, W)                                                                                              \
    SQ_TRY((launch_backward_mc<MM, W>(ctx, grid, pairs, m, sw, self_scores, packed, emb, d, sig_seq, hashes,       \
                                      gate_params, hidden, dL_dfused, coef, partials)))
    if (channels == 2) {
        if (pack_stride == 16) SQ_MCB(2, 2);
        else SQ_MCB(2, 4);
    } else {
        if (pack_stride == 16) SQ_MCB(3, 2);
        else SQ_MCB(3, 4);
    }
#undef SQ_MCB
    reduce_partials_kernel<<<1, 352, 0, ctx->stream>>>(partials, (int)grid, P, grad_params);
    SQ_LAUNCH_CHECK();
    if (grad_emb && n > 0)
        SQ_TRY(launch_emb_grad(ctx, pairs, coef, emb, n, d, perm_i, off_i, perm_j, off_j, grad_emb, heavy_list,
                               heavy_count));
    return SUBQUAD_OK;
}

extern "C" int subquad_sig_sequence_major(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows,
                                          uint32_t *sig_seq_out)
{
    SQ_ENTER(ctx);
    if (n < 0 || bands < 1 || rows < 1 || rows > 8 || bands * rows > 512) return SUBQUAD_ERR_ARG;
    if (n == 0) return SUBQUAD_OK;
    if (!sig || !sig_seq_out) return SUBQUAD_ERR_ARG;
    if (rows == 4 && (reinterpret_cast<uintptr_t>(sig) % 16 || reinterpret_cast<uintptr_t>(sig_seq_out) % 16))
        return SUBQUAD_ERR_ARG;
    if (rows == 4) {
        const size_t smem = sizeof(uint4) * kTrSeq * bands;  // <= 128 bands: 128 KB
        SQ_TRY_CUDA(cudaFuncSetAttribute(sig_transpose4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const unsigned grid = (unsigned)std::min<int64_t>((n + kTrSeq - 1) / kTrSeq, (int64_t)ctx->num_sms * 8);
        sig_transpose4_kernel<<<grid, 256, smem, ctx->stream>>>(reinterpret_cast<const uint4 *>(sig), n, bands,
                                                                reinterpret_cast<uint4 *>(sig_seq_out));
    } else {
        sig_transpose_kernel<<<sq_grid(ctx, n, 256, 8), 256, 0, ctx->stream>>>(sig, n, bands, rows, sig_seq_out);
    }
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}
