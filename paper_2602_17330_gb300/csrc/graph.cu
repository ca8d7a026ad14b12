// Graph construction and RMT-based thresholding (the graph-construction
// section and Algorithm 1's graph step): the fused scores of the candidate
// pairs form a symmetric sparse matrix A; its spectrum decides the threshold
// below which edges are removed.
//
// A_tau (entries >= tau) is block-diagonal over the connected components of
// its graph, so its spectrum is the union of the components' spectra:
//   1. components by lock-free union-find (hooks always point to the smaller
//      root, so a component's root is its smallest vertex id);
//   2. the vertices of components with >= 2 vertices grouped by component
//      (stable radix sort on the label: vertex ids ascending inside a
//      component), each component's dense block scattered into scratch;
//   3. every block's eigenvalues by a cyclic parallel Jacobi method in FP64,
//      one warp per component (round-robin pairing, n/2 disjoint rotations
//      per step, the block in shared memory), up to 64 vertices;
//   4. the union of the levels sorted (64-bit order-preserving keys through
//      two stable 32-bit radix passes), levels within 1e-9 of their
//      predecessor dropped as degenerate, and the mean ratio of consecutive
//      spacings <r> = mean min(d_k, d_{k+1}) / max(d_k, d_{k+1}) reduced in
//      FP64 in a fixed order.
// The scan over thresholds stops at the first tau whose components all have
// <= s_max vertices and whose <r> is at most the midpoint of the Poisson and
// GOE reference values.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int kUfLimit = 1 << 20;  // bound on the steps of one find or union
constexpr int kMaxComp = 64;       // largest component the Jacobi kernel takes
constexpr int kJacWarps = 8;       // components (warps) per Jacobi block
constexpr int kJacSweeps = 60;
constexpr double kEpsLevel = 1e-9;

__global__ void uf_init_kernel(uint32_t *__restrict__ parent, int64_t n)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = (uint32_t)v;
}

__device__ __forceinline__ uint32_t uf_find(uint32_t *parent, uint32_t x, uint32_t *err)
{
    for (int it = 0; it < kUfLimit; ++it) {
        const uint32_t p = parent[x];
        if (p == x) return x;
        const uint32_t g = parent[p];
        if (g != p) parent[x] = g;  // path halving: g is an ancestor of x as well
        x = g;
    }
    atomicOr(err, SQ_DEVERR_TIMEOUT);
    return x;
}

__global__ void uf_union_kernel(const uint32_t *__restrict__ pairs, const float *__restrict__ w, int64_t m, double tau,
                                uint32_t *parent, uint32_t *err)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        if (!((double)w[p] >= tau)) continue;
        const uint2 ij = reinterpret_cast<const uint2 *>(pairs)[p];
        uint32_t a = ij.x, b = ij.y;
        int it = 0;
        for (; it < kUfLimit; ++it) {
            a = uf_find(parent, a, err);
            b = uf_find(parent, b, err);
            if (a == b) break;
            const uint32_t hi = a > b ? a : b, lo = a > b ? b : a;
            if (atomicCAS(&parent[hi], hi, lo) == hi) break;  // hooked; else hi gained a parent meanwhile
        }
        if (it == kUfLimit) atomicOr(err, SQ_DEVERR_TIMEOUT);
    }
}

// label[v] = root of v; size[root] += 1.
__global__ void uf_flatten_kernel(uint32_t *parent, uint32_t *__restrict__ label, uint32_t *__restrict__ size,
                                  int64_t n, uint32_t *err)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = uf_find(parent, (uint32_t)v, err);
        label[v] = r;
        atomicAdd(&size[r], 1u);
    }
}

// flag[v] = 1 for a vertex of a component with >= 2 vertices; stats[0] = the
// largest such component's size.
__global__ void active_kernel(const uint32_t *__restrict__ label, const uint32_t *__restrict__ size, int64_t n,
                              uint32_t *__restrict__ flag, uint32_t *__restrict__ stats)
{
    uint32_t mx = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = size[label[v]];
        flag[v] = s >= 2 ? 1u : 0u;
        if (s >= 2 && s > mx) mx = s;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&stats[0], mx);
}

__global__ void compact_kernel(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                               const uint32_t *__restrict__ label, int64_t n, uint32_t *__restrict__ keys,
                               uint32_t *__restrict__ vals)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (flag[v]) {
            keys[pos[v]] = label[v];
            vals[pos[v]] = (uint32_t)v;
        }
}

__global__ void seg_start_kernel(const uint32_t *__restrict__ keys, int64_t A, uint32_t *__restrict__ start_flag)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A; k += (int64_t)gridDim.x * blockDim.x)
        start_flag[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1u : 0u;
}

// comp_start[c] = first position of component c; vpos[v] = position of v in
// the grouped order; vcomp[v] = component index of v.
__global__ void seg_index_kernel(const uint32_t *__restrict__ start_flag, const uint32_t *__restrict__ start_scan,
                                 const uint32_t *__restrict__ vals, int64_t A, uint32_t *__restrict__ comp_start,
                                 uint32_t *__restrict__ vpos, uint32_t *__restrict__ vcomp)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = start_scan[k] + start_flag[k] - 1u;  // inclusive count - 1
        if (start_flag[k]) comp_start[c] = (uint32_t)k;
        vpos[vals[k]] = (uint32_t)k;
        vcomp[vals[k]] = c;
    }
}

__global__ void mat_size_kernel(const uint32_t *__restrict__ comp_start, int64_t ncomp, int64_t A,
                                uint64_t *__restrict__ msz)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncomp; c += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t s = (c + 1 < ncomp ? comp_start[c + 1] : (uint32_t)A) - comp_start[c];
        msz[c] = s * s;
    }
}

__global__ void mat_scatter_kernel(const uint32_t *__restrict__ pairs, const float *__restrict__ w, int64_t m,
                                   double tau, const uint32_t *__restrict__ vpos, const uint32_t *__restrict__ vcomp,
                                   const uint32_t *__restrict__ comp_start, const uint64_t *__restrict__ mat_off,
                                   int64_t ncomp, int64_t A, double *__restrict__ mats)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)w[p];
        if (!(x >= tau)) continue;
        const uint2 ij = reinterpret_cast<const uint2 *>(pairs)[p];
        const uint32_t c = vcomp[ij.x];
        const uint32_t base = comp_start[c];
        const uint32_t s = (c + 1 < ncomp ? comp_start[c + 1] : (uint32_t)A) - base;
        const uint32_t li = vpos[ij.x] - base, lj = vpos[ij.y] - base;
        double *M = mats + mat_off[c];
        M[(uint64_t)li * s + lj] = x;
        M[(uint64_t)lj * s + li] = x;
    }
}

// One warp per component: cyclic parallel Jacobi in FP64 on the block held in
// shared memory (row pitch nmax + 1, nmax = the largest component rounded up
// to even, so small components leave room for more warps per SM), round-robin
// pairing (player 0 fixed, the others rotate), rows then columns updated per
// step; sweeps until the off-diagonal sum of squares is <= 1e-26 of the total
// (or kJacSweeps).
__global__ void __launch_bounds__(32 * kJacWarps) jacobi_kernel(const uint32_t *__restrict__ comp_start,
                                                                 int64_t ncomp, int64_t A,
                                                                 const uint64_t *__restrict__ mat_off,
                                                                 const double *__restrict__ mats, int nmax,
                                                                 double *__restrict__ levels, uint32_t *err)
{
    extern __shared__ double s_mem[];
    const int P = nmax + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *S = s_mem + (size_t)warp * nmax * P;
    __shared__ int s_p[kJacWarps][kMaxComp / 2], s_q[kJacWarps][kMaxComp / 2];
    __shared__ double s_c[kJacWarps][kMaxComp / 2], s_s[kJacWarps][kMaxComp / 2];
    const int wpb = blockDim.x >> 5;  // warps (components in flight) per block
    for (int64_t c = blockIdx.x * (int64_t)wpb + warp; c < ncomp; c += (int64_t)gridDim.x * wpb) {
        const uint32_t base = comp_start[c];
        const int s = (int)((c + 1 < ncomp ? comp_start[c + 1] : (uint32_t)A) - base);
        const int N = s + (s & 1);
        const double *M = mats + mat_off[c];
        for (int q = lane; q < N * N; q += 32) {
            const int i = q / N, j = q - i * N;
            S[i * P + j] = (i < s && j < s) ? M[(uint64_t)i * s + j] : 0.0;
        }
        __syncwarp();
        double tot = 0.0;
        for (int q = lane; q < N * N; q += 32) tot += S[(q / N) * P + q % N] * S[(q / N) * P + q % N];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        int sweep = 0;
        for (; sweep < kJacSweeps; ++sweep) {
            double off = 0.0;
            for (int q = lane; q < N * N; q += 32) {
                const int i = q / N, j = q - i * N;
                if (i != j) off += S[i * P + j] * S[i * P + j];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
            if (off <= 1e-26 * tot) break;
            for (int r = 0; r < N - 1; ++r) {
                for (int k = lane; k < N / 2; k += 32) {
                    int a, b;
                    if (k == 0) {
                        a = 0;
                        b = r % (N - 1) + 1;
                    } else {
                        a = (r + k) % (N - 1) + 1;
                        b = (r - k + (N - 1)) % (N - 1) + 1;
                    }
                    const int p = a < b ? a : b, q = a < b ? b : a;
                    const double apq = S[p * P + q];
                    double cs = 1.0, sn = 0.0;
                    if (fabs(apq) > 1e-300) {
                        const double th = (S[q * P + q] - S[p * P + p]) / (2.0 * apq);
                        const double t = fabs(th) < 1e150 ? (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0))
                                                          : 0.5 / th;
                        cs = 1.0 / sqrt(t * t + 1.0);
                        sn = t * cs;
                    }
                    s_p[warp][k] = p;
                    s_q[warp][k] = q;
                    s_c[warp][k] = cs;
                    s_s[warp][k] = sn;
                }
                __syncwarp();
                // rows p and q of every pair: column j per lane
                for (int j = lane; j < N; j += 32)
                    for (int k = 0; k < N / 2; ++k) {
                        const int p = s_p[warp][k], q = s_q[warp][k];
                        const double cs = s_c[warp][k], sn = s_s[warp][k];
                        const double xp = S[p * P + j], xq = S[q * P + j];
                        S[p * P + j] = cs * xp - sn * xq;
                        S[q * P + j] = sn * xp + cs * xq;
                    }
                __syncwarp();
                // columns p and q: row i per lane
                for (int i = lane; i < N; i += 32)
                    for (int k = 0; k < N / 2; ++k) {
                        const int p = s_p[warp][k], q = s_q[warp][k];
                        const double cs = s_c[warp][k], sn = s_s[warp][k];
                        const double xp = S[i * P + p], xq = S[i * P + q];
                        S[i * P + p] = cs * xp - sn * xq;
                        S[i * P + q] = sn * xp + cs * xq;
                    }
                __syncwarp();
            }
        }
        if (sweep == kJacSweeps && lane == 0) atomicOr(err, SQ_DEVERR_TIMEOUT);
        for (int k = lane; k < s; k += 32) levels[base + k] = S[k * P + k];
        __syncwarp();
    }
}

__device__ __forceinline__ uint64_t order_key(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | (uint64_t(1) << 63));
}

__global__ void level_keys_kernel(const double *__restrict__ levels, int64_t A, uint32_t *__restrict__ lo,
                                  uint32_t *__restrict__ idx)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A; k += (int64_t)gridDim.x * blockDim.x) {
        lo[k] = (uint32_t)order_key(levels[k]);
        idx[k] = (uint32_t)k;
    }
}

__global__ void level_hi_kernel(const double *__restrict__ levels, const uint32_t *__restrict__ idx, int64_t A,
                                uint32_t *__restrict__ hi)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A; k += (int64_t)gridDim.x * blockDim.x)
        hi[k] = (uint32_t)(order_key(levels[idx[k]]) >> 32);
}

__global__ void level_gather_kernel(const double *__restrict__ levels, const uint32_t *__restrict__ idx, int64_t A,
                                    double *__restrict__ sorted, uint32_t *__restrict__ kept)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A; k += (int64_t)gridDim.x * blockDim.x) {
        const double x = levels[idx[k]];
        sorted[k] = x;
        kept[k] = (k == 0 || x - levels[idx[k - 1]] > kEpsLevel) ? 1u : 0u;
    }
}

__global__ void level_compact_kernel(const double *__restrict__ sorted, const uint32_t *__restrict__ kept,
                                     const uint32_t *__restrict__ kpos, int64_t A, double *__restrict__ out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A; k += (int64_t)gridDim.x * blockDim.x)
        if (kept[k]) out[kpos[k]] = sorted[k];
}

constexpr int kRThreads = 256;

// Per block, the FP64 sum of the spacing ratios of its grid-stride share
// (fixed grid: the summation order does not depend on anything but K).
__global__ void __launch_bounds__(kRThreads) r_partial_kernel(const double *__restrict__ K, const uint32_t *__restrict__ d_K,
                                                              double *__restrict__ partial)
{
    __shared__ double s_sum[kRThreads];
    const int64_t nk = (int64_t)*d_K;
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q + 2 < nk; q += (int64_t)gridDim.x * blockDim.x) {
        const double d1 = K[q + 1] - K[q], d2 = K[q + 2] - K[q + 1];
        acc += fmin(d1, d2) / fmax(d1, d2);
    }
    s_sum[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kRThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s_sum[0];
}

__global__ void r_final_kernel(const double *__restrict__ partial, int blocks, double *__restrict__ out)
{
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < blocks; ++b) t += partial[b];
        out[0] = t;
    }
}

__global__ void prune_flag_kernel(const float *__restrict__ w, int64_t m, double tau, uint32_t *__restrict__ flag)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = (double)w[p] >= tau ? 1u : 0u;
}

__global__ void prune_scatter_kernel(const uint32_t *__restrict__ pairs, const float *__restrict__ w, int64_t m,
                                     const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                                     uint32_t *__restrict__ pairs_out, float *__restrict__ w_out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
        if (flag[p]) {
            reinterpret_cast<uint2 *>(pairs_out)[pos[p]] = reinterpret_cast<const uint2 *>(pairs)[p];
            if (w_out) w_out[pos[p]] = w[p];
        }
}

__global__ void u32_to_u64_kernel(const uint32_t *__restrict__ in, uint64_t *__restrict__ out)
{
    if (threadIdx.x == 0) out[0] = in[0];
}

// Scratch of one threshold evaluation.
struct GraphScratch {
    uint32_t *parent, *label, *size, *flag, *pos, *keys, *vals, *keys_alt, *vals_alt, *start_flag, *start_scan,
        *comp_start, *vpos, *vcomp, *stats, *kept, *kpos, *totals;
    uint64_t *msz, *mat_off;
    double *mats, *levels, *sorted, *kept_levels, *partial, *rsum;
    void *tmp;
    size_t tmp_bytes;
};

constexpr int kRBlocks = 512;

int graph_scratch(subquad_ctx *ctx, int64_t n, int64_t m, bool with_spectrum, GraphScratch &g)
{
    const int64_t nn = n > 0 ? n : 1;
    const size_t tmp_bytes = std::max(std::max(sq_scan_tmp_bytes(nn + 1), sq_radix_tmp_bytes(nn)),
                                      sq_scan_tmp_bytes(m > 0 ? m : 1));
    auto lay = [&](SqArena &a) {
        g.parent = a.take<uint32_t>(nn);
        g.label = a.take<uint32_t>(nn);
        g.size = a.take<uint32_t>(nn);
        g.flag = a.take<uint32_t>(std::max<int64_t>(nn, m) + 1);
        g.pos = a.take<uint32_t>(std::max<int64_t>(nn, m) + 1);
        g.stats = a.take<uint32_t>(8);
        g.totals = a.take<uint32_t>(8);
        g.tmp = a.take<char>(tmp_bytes);
        if (with_spectrum) {
            g.keys = a.take<uint32_t>(nn);
            g.vals = a.take<uint32_t>(nn);
            g.keys_alt = a.take<uint32_t>(nn);
            g.vals_alt = a.take<uint32_t>(nn);
            g.start_flag = a.take<uint32_t>(nn);
            g.start_scan = a.take<uint32_t>(nn);
            g.comp_start = a.take<uint32_t>(nn + 1);
            g.vpos = a.take<uint32_t>(nn);
            g.vcomp = a.take<uint32_t>(nn);
            g.kept = a.take<uint32_t>(nn);
            g.kpos = a.take<uint32_t>(nn);
            g.msz = a.take<uint64_t>(nn);
            g.mat_off = a.take<uint64_t>(nn + 1);
            g.levels = a.take<double>(nn);
            g.sorted = a.take<double>(nn);
            g.kept_levels = a.take<double>(nn);
            g.partial = a.take<double>(kRBlocks);
            g.rsum = a.take<double>(1);
            g.mats = a.take<double>((size_t)nn * kMaxComp);  // sum of s^2 <= s_max * sum of s
        }
    };
    SqArena measure(nullptr);
    lay(measure);
    SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    SqArena a(ctx->scratch);
    lay(a);
    g.tmp_bytes = tmp_bytes;
    return SUBQUAD_OK;
}

int run_components(subquad_ctx *ctx, const uint32_t *pairs, const float *w, int64_t m, int64_t n, double tau,
                   GraphScratch &g)
{
    const unsigned gn = sq_grid(ctx, n, 256, 8), gm = sq_grid(ctx, m, 256, 8);
    uf_init_kernel<<<gn, 256, 0, ctx->stream>>>(g.parent, n);
    SQ_LAUNCH_CHECK();
    if (m > 0) {
        uf_union_kernel<<<gm, 256, 0, ctx->stream>>>(pairs, w, m, tau, g.parent, ctx->d_err);
        SQ_LAUNCH_CHECK();
    }
    SQ_TRY_CUDA(cudaMemsetAsync(g.size, 0, sizeof(uint32_t) * n, ctx->stream));
    uf_flatten_kernel<<<gn, 256, 0, ctx->stream>>>(g.parent, g.label, g.size, n, ctx->d_err);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

int read_u32(subquad_ctx *ctx, const uint32_t *d, uint32_t *h, int count)
{
    SQ_TRY_CUDA(cudaMemcpyAsync(ctx->h_pinned, d, sizeof(uint32_t) * count, cudaMemcpyDeviceToHost, ctx->stream));
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    memcpy(h, ctx->h_pinned, sizeof(uint32_t) * count);
    return SUBQUAD_OK;
}

// One threshold: max component size (*max_comp), and when every component has
// <= s_max vertices the spectrum's <r> and number of ratios.
int evaluate_threshold(subquad_ctx *ctx, const uint32_t *pairs, const float *w, int64_t m, int64_t n, double tau,
                       int s_max, GraphScratch &g, int32_t *max_comp, int64_t *levels_out, int64_t *ratios_out,
                       double *r_mean_out)
{
    *levels_out = 0;
    *ratios_out = 0;
    *r_mean_out = NAN;
    SQ_TRY(run_components(ctx, pairs, w, m, n, tau, g));
    const unsigned gn = sq_grid(ctx, n, 256, 8);
    SQ_TRY_CUDA(cudaMemsetAsync(g.stats, 0, sizeof(uint32_t) * 8, ctx->stream));
    active_kernel<<<gn, 256, 0, ctx->stream>>>(g.label, g.size, n, g.flag, g.stats);
    SQ_LAUNCH_CHECK();
    SQ_TRY(sq_scan_u32(ctx, g.flag, g.pos, n, nullptr, false, false, g.totals, g.tmp, g.tmp_bytes));
    uint32_t h[2];
    SQ_TRY(read_u32(ctx, g.stats, &h[0], 1));
    SQ_TRY(read_u32(ctx, g.totals, &h[1], 1));
    *max_comp = (int32_t)h[0];
    const int64_t A = h[1];
    if ((int)h[0] > s_max || A == 0) return SUBQUAD_OK;
    compact_kernel<<<gn, 256, 0, ctx->stream>>>(g.flag, g.pos, g.label, n, g.keys, g.vals);
    SQ_LAUNCH_CHECK();
    int bits = 1;
    while (bits < 32 && (int64_t(1) << bits) < n) ++bits;
    bool in_alt = false;
    SQ_TRY(sq_radix_sort_u32(ctx, g.keys, g.vals, g.keys_alt, g.vals_alt, A, nullptr, 0, bits, &in_alt, g.tmp,
                             g.tmp_bytes));
    uint32_t *keys = in_alt ? g.keys_alt : g.keys, *vals = in_alt ? g.vals_alt : g.vals;
    const unsigned ga = sq_grid(ctx, A, 256, 8);
    seg_start_kernel<<<ga, 256, 0, ctx->stream>>>(keys, A, g.start_flag);
    SQ_LAUNCH_CHECK();
    SQ_TRY(sq_scan_u32(ctx, g.start_flag, g.start_scan, A, nullptr, false, false, g.totals + 1, g.tmp, g.tmp_bytes));
    seg_index_kernel<<<ga, 256, 0, ctx->stream>>>(g.start_flag, g.start_scan, vals, A, g.comp_start, g.vpos, g.vcomp);
    SQ_LAUNCH_CHECK();
    uint32_t ncomp32 = 0;
    SQ_TRY(read_u32(ctx, g.totals + 1, &ncomp32, 1));
    const int64_t ncomp = ncomp32;
    mat_size_kernel<<<sq_grid(ctx, ncomp, 256, 8), 256, 0, ctx->stream>>>(g.comp_start, ncomp, A, g.msz);
    SQ_LAUNCH_CHECK();
    SQ_TRY(sq_scan_u64(ctx, g.msz, g.mat_off, ncomp, nullptr, nullptr, g.tmp, g.tmp_bytes));
    SQ_TRY_CUDA(cudaMemsetAsync(g.mats, 0, sizeof(double) * (size_t)A * kMaxComp, ctx->stream));
    mat_scatter_kernel<<<sq_grid(ctx, m, 256, 8), 256, 0, ctx->stream>>>(pairs, w, m, tau, g.vpos, g.vcomp,
                                                                         g.comp_start, g.mat_off, ncomp, A, g.mats);
    SQ_LAUNCH_CHECK();
    const int nmax = (int)h[0] + ((int)h[0] & 1);
    const size_t per_warp = sizeof(double) * nmax * (nmax + 1);
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(kJacWarps, (size_t)(200 << 10) / per_warp));
    const size_t smem = per_warp * wpb;
    SQ_TRY_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned gj = (unsigned)std::min<int64_t>((ncomp + wpb - 1) / wpb, (int64_t)ctx->num_sms * 16);
    jacobi_kernel<<<gj, 32 * wpb, smem, ctx->stream>>>(g.comp_start, ncomp, A, g.mat_off, g.mats, nmax, g.levels,
                                                       ctx->d_err);
    SQ_LAUNCH_CHECK();
    // sort the levels: low words, then high words (both stable)
    level_keys_kernel<<<ga, 256, 0, ctx->stream>>>(g.levels, A, g.keys, g.vals);
    SQ_LAUNCH_CHECK();
    SQ_TRY(sq_radix_sort_u32(ctx, g.keys, g.vals, g.keys_alt, g.vals_alt, A, nullptr, 0, 32, &in_alt, g.tmp,
                             g.tmp_bytes));
    uint32_t *idx = in_alt ? g.vals_alt : g.vals;
    uint32_t *hk = in_alt ? g.keys_alt : g.keys;
    uint32_t *idx_alt = in_alt ? g.vals : g.vals_alt, *hk_alt = in_alt ? g.keys : g.keys_alt;
    level_hi_kernel<<<ga, 256, 0, ctx->stream>>>(g.levels, idx, A, hk);
    SQ_LAUNCH_CHECK();
    SQ_TRY(sq_radix_sort_u32(ctx, hk, idx, hk_alt, idx_alt, A, nullptr, 0, 32, &in_alt, g.tmp, g.tmp_bytes));
    const uint32_t *order = in_alt ? idx_alt : idx;
    level_gather_kernel<<<ga, 256, 0, ctx->stream>>>(g.levels, order, A, g.sorted, g.kept);
    SQ_LAUNCH_CHECK();
    SQ_TRY(sq_scan_u32(ctx, g.kept, g.kpos, A, nullptr, false, false, g.totals + 2, g.tmp, g.tmp_bytes));
    level_compact_kernel<<<ga, 256, 0, ctx->stream>>>(g.sorted, g.kept, g.kpos, A, g.kept_levels);
    SQ_LAUNCH_CHECK();
    r_partial_kernel<<<kRBlocks, kRThreads, 0, ctx->stream>>>(g.kept_levels, g.totals + 2, g.partial);
    SQ_LAUNCH_CHECK();
    r_final_kernel<<<1, 32, 0, ctx->stream>>>(g.partial, kRBlocks, g.rsum);
    SQ_LAUNCH_CHECK();
    uint32_t nk = 0;
    SQ_TRY(read_u32(ctx, g.totals + 2, &nk, 1));
    double rsum = 0.0;
    SQ_TRY_CUDA(cudaMemcpyAsync(ctx->h_pinned, g.rsum, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    memcpy(&rsum, ctx->h_pinned, sizeof(double));
    *levels_out = A;
    if (nk >= 3) {
        *ratios_out = (int64_t)nk - 2;
        *r_mean_out = rsum / (double)(nk - 2);
    }
    return SUBQUAD_OK;
}

// ---------------------------------------------------------------------------
// Cluster-mass Jensen-Shannon repertoire distance (appendix on repertoire-
// level distances).  With p_d(k) = |cluster k n donor d| / |donor d| and
// M = (p_a + p_b) / 2, JS(a, b) = 1/2 KL(p_a || M) + 1/2 KL(p_b || M)
// (natural log).  A cluster present in only one of the two donors adds
// 1/2 p log 2, and sum_k p_d(k) = 1, so
//   JS(a, b) = log 2 + sum over clusters with both present of
//              [1/2 p_a log(2 p_a / (p_a + p_b)) + 1/2 p_b log(2 p_b / (p_a + p_b)) - 1/2 (p_a + p_b) log 2],
// which touches only the (cluster, donor pair) combinations that occur.  The
// (label, donor) keys are sorted (two stable radix passes), runs of equal
// keys counted, and one warp per cluster adds its donor pairs' terms.
// ---------------------------------------------------------------------------
__global__ void run_start_kernel(const uint32_t *__restrict__ lab, const uint32_t *__restrict__ don, int64_t n,
                                 uint32_t *__restrict__ run_flag, uint32_t *__restrict__ clu_flag)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const bool new_label = k == 0 || lab[k] != lab[k - 1];
        run_flag[k] = (new_label || don[k] != don[k - 1]) ? 1u : 0u;
        clu_flag[k] = new_label ? 1u : 0u;
    }
}

// run r: first position run_pos[r], donor run_don[r]; cluster of run r starts
// at run clu_first[c]; run lengths follow from consecutive positions.
__global__ void run_index_kernel(const uint32_t *__restrict__ run_flag, const uint32_t *__restrict__ run_scan,
                                 const uint32_t *__restrict__ clu_flag, const uint32_t *__restrict__ clu_scan,
                                 const uint32_t *__restrict__ don, int64_t n, uint32_t *__restrict__ run_pos,
                                 uint32_t *__restrict__ run_don, uint32_t *__restrict__ clu_first)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (!run_flag[k]) continue;
        const uint32_t r = run_scan[k];
        run_pos[r] = (uint32_t)k;
        run_don[r] = don[k];
        if (clu_flag[k]) clu_first[clu_scan[k]] = r;
    }
}

__global__ void donor_size_kernel(const int32_t *__restrict__ donor, int64_t n, int num_donors,
                                  uint32_t *__restrict__ dsize, uint32_t *__restrict__ don_u, uint32_t *err)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = donor[v];
        if (d < 0 || d >= num_donors) {
            atomicOr(err, SQ_DEVERR_INPUT);
            don_u[v] = 0;
            continue;
        }
        don_u[v] = (uint32_t)d;
        atomicAdd(&dsize[d], 1u);
    }
}

__global__ void js_pairs_kernel(const uint32_t *__restrict__ clu_first, const uint32_t *__restrict__ d_nclu,
                                const uint32_t *__restrict__ d_nrun, const uint32_t *__restrict__ run_pos,
                                const uint32_t *__restrict__ run_don, int64_t n, const uint32_t *__restrict__ dsize,
                                int num_donors, double *__restrict__ acc)
{
    const int64_t nclu = *d_nclu, nrun = *d_nrun;
    const int lane = threadIdx.x & 31;
    const double ln2 = 0.69314718055994530942;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < nclu;
         c += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const uint32_t r0 = clu_first[c], r1 = c + 1 < nclu ? clu_first[c + 1] : (uint32_t)nrun;
        const uint32_t R = r1 - r0;
        if (R < 2) continue;
        for (uint64_t t = lane; t < (uint64_t)R * R; t += 32) {
            const uint32_t x = (uint32_t)(t / R), y = (uint32_t)(t % R);
            if (x >= y) continue;
            const uint32_t ra = r0 + x, rb = r0 + y;
            const uint32_t ca = (ra + 1 < (uint32_t)nrun ? run_pos[ra + 1] : (uint32_t)n) - run_pos[ra];
            const uint32_t cb = (rb + 1 < (uint32_t)nrun ? run_pos[rb + 1] : (uint32_t)n) - run_pos[rb];
            const uint32_t a = run_don[ra], b = run_don[rb];
            const double pa = (double)ca / (double)dsize[a], pb = (double)cb / (double)dsize[b];
            const double s = pa + pb;
            const double term = 0.5 * pa * log(2.0 * pa / s) + 0.5 * pb * log(2.0 * pb / s) - 0.5 * s * ln2;
            atomicAdd(&acc[(size_t)a * num_donors + b], term);
        }
    }
}

__global__ void js_finish_kernel(const double *__restrict__ acc, const uint32_t *__restrict__ dsize, int num_donors,
                                 double *__restrict__ out)
{
    const double ln2 = 0.69314718055994530942;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < num_donors * num_donors; q += gridDim.x * blockDim.x) {
        const int a = q / num_donors, b = q % num_donors;
        double v;
        if (!dsize[a] || !dsize[b]) v = NAN;
        else if (a == b) v = 0.0;
        else {
            const double js = ln2 + (a < b ? acc[(size_t)a * num_donors + b] : acc[(size_t)b * num_donors + a]);
            v = sqrt(js > 0.0 ? js : 0.0);
        }
        out[q] = v;
    }
}

bool graph_args_ok(const uint32_t *pairs, const float *w, int64_t m, int64_t n)
{
    if (m < 0 || n < 0 || n >= (int64_t(1) << 31) || m >= (int64_t(1) << 32)) return false;
    if (m > 0 && (!pairs || !w)) return false;
    return reinterpret_cast<uintptr_t>(pairs) % 8 == 0;
}

}  // namespace

extern "C" int subquad_graph_components(subquad_ctx *ctx, const uint32_t *pairs, const float *weights, int64_t m,
                                        int64_t n, double tau, uint32_t *labels_out, uint32_t *sizes_out)
{
    SQ_ENTER(ctx);
    if (!graph_args_ok(pairs, weights, m, n) || (n > 0 && !labels_out)) return SUBQUAD_ERR_ARG;
    if (n == 0) return SUBQUAD_OK;
    GraphScratch g;
    SQ_TRY(graph_scratch(ctx, n, m, false, g));
    SQ_TRY(run_components(ctx, pairs, weights, m, n, tau, g));
    SQ_TRY_CUDA(cudaMemcpyAsync(labels_out, g.label, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    if (sizes_out)
        SQ_TRY_CUDA(cudaMemcpyAsync(sizes_out, g.size, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return SUBQUAD_OK;
}

extern "C" int subquad_rmt_threshold(subquad_ctx *ctx, const uint32_t *pairs, const float *weights, int64_t m,
                                     int64_t n, const double *taus, int num_taus, int s_max, double r_mid,
                                     double *tau_star, double *r_mean, int64_t *num_ratios, int64_t *num_levels,
                                     int32_t *max_comp)
{
    SQ_ENTER(ctx);
    if (!graph_args_ok(pairs, weights, m, n) || !taus || num_taus < 1 || !tau_star) return SUBQUAD_ERR_ARG;
    if (s_max < 2 || s_max > kMaxComp) return SUBQUAD_ERR_ARG;
    for (int t = 1; t < num_taus; ++t)
        if (!(taus[t] > taus[t - 1])) return SUBQUAD_ERR_ARG;
    for (int t = 0; t < num_taus; ++t) {
        if (r_mean) r_mean[t] = NAN;
        if (num_ratios) num_ratios[t] = 0;
        if (num_levels) num_levels[t] = 0;
        if (max_comp) max_comp[t] = -1;
    }
    *tau_star = taus[num_taus - 1];
    if (n == 0) return SUBQUAD_OK;
    GraphScratch g;
    SQ_TRY(graph_scratch(ctx, n, m, true, g));
    for (int t = 0; t < num_taus; ++t) {
        int32_t mc = 0;
        int64_t nl = 0, nr = 0;
        double rm = NAN;
        SQ_TRY(evaluate_threshold(ctx, pairs, weights, m, n, taus[t], s_max, g, &mc, &nl, &nr, &rm));
        SQ_TRY(subquad_check(ctx));
        if (r_mean) r_mean[t] = rm;
        if (num_ratios) num_ratios[t] = nr;
        if (num_levels) num_levels[t] = nl;
        if (max_comp) max_comp[t] = mc;
        if (mc <= s_max && nr > 0 && rm <= r_mid) {
            *tau_star = taus[t];
            break;
        }
    }
    return SUBQUAD_OK;
}

extern "C" int subquad_graph_prune(subquad_ctx *ctx, const uint32_t *pairs, const float *weights, int64_t m,
                                   double tau, uint32_t *pairs_out, float *weights_out, uint64_t *d_count)
{
    SQ_ENTER(ctx);
    if (!graph_args_ok(pairs, weights, m, 0) || !d_count || (m > 0 && !pairs_out)) return SUBQUAD_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(pairs_out) % 8) return SUBQUAD_ERR_ARG;
    GraphScratch g;
    SQ_TRY(graph_scratch(ctx, 1, m, false, g));
    if (m == 0) {
        SQ_TRY_CUDA(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), ctx->stream));
        return SUBQUAD_OK;
    }
    const unsigned gm = sq_grid(ctx, m, 256, 8);
    prune_flag_kernel<<<gm, 256, 0, ctx->stream>>>(weights, m, tau, g.flag);
    SQ_LAUNCH_CHECK();
    SQ_TRY(sq_scan_u32(ctx, g.flag, g.pos, m, nullptr, false, false, g.totals, g.tmp, g.tmp_bytes));
    prune_scatter_kernel<<<gm, 256, 0, ctx->stream>>>(pairs, weights, m, g.flag, g.pos, pairs_out, weights_out);
    SQ_LAUNCH_CHECK();
    u32_to_u64_kernel<<<1, 32, 0, ctx->stream>>>(g.totals, d_count);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}

extern "C" int subquad_cluster_js(subquad_ctx *ctx, const uint32_t *labels, const int32_t *donor, int64_t n,
                                  int num_donors, double *dist_out)
{
    SQ_ENTER(ctx);
    if (n < 1 || n >= (int64_t(1) << 31) || num_donors < 1 || num_donors > 4096) return SUBQUAD_ERR_ARG;
    if (!labels || !donor || !dist_out) return SUBQUAD_ERR_ARG;
    const int D = num_donors;
    const size_t tmp_bytes = std::max(sq_radix_tmp_bytes(n), sq_scan_tmp_bytes(n));
    auto lay = [&](SqArena &a, uint32_t **k0, uint32_t **v0, uint32_t **k1, uint32_t **v1, uint32_t **f1,
                   uint32_t **s1, uint32_t **f2, uint32_t **s2, uint32_t **rp, uint32_t **rd, uint32_t **cf,
                   uint32_t **ds, uint32_t **tot, double **acc, void **tmp) {
        *k0 = a.take<uint32_t>(n);
        *v0 = a.take<uint32_t>(n);
        *k1 = a.take<uint32_t>(n);
        *v1 = a.take<uint32_t>(n);
        *f1 = a.take<uint32_t>(n);
        *s1 = a.take<uint32_t>(n);
        *f2 = a.take<uint32_t>(n);
        *s2 = a.take<uint32_t>(n);
        *rp = a.take<uint32_t>(n);
        *rd = a.take<uint32_t>(n);
        *cf = a.take<uint32_t>(n);
        *ds = a.take<uint32_t>(D);
        *tot = a.take<uint32_t>(4);
        *acc = a.take<double>((size_t)D * D);
        *tmp = a.take<char>(tmp_bytes);
    };
    uint32_t *k0, *v0, *k1, *v1, *f1, *s1, *f2, *s2, *rp, *rd, *cf, *ds, *tot;
    double *acc;
    void *tmp;
    SqArena measure(nullptr);
    lay(measure, &k0, &v0, &k1, &v1, &f1, &s1, &f2, &s2, &rp, &rd, &cf, &ds, &tot, &acc, &tmp);
    SQ_TRY(sq_scratch_reserve(ctx, measure.off));
    SqArena a(ctx->scratch);
    lay(a, &k0, &v0, &k1, &v1, &f1, &s1, &f2, &s2, &rp, &rd, &cf, &ds, &tot, &acc, &tmp);
    const unsigned gn = sq_grid(ctx, n, 256, 8);
    SQ_TRY_CUDA(cudaMemsetAsync(ds, 0, sizeof(uint32_t) * D, ctx->stream));
    SQ_TRY_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * D * D, ctx->stream));
    // keys: donor first (stable), then label, so runs are (label, donor) ascending
    donor_size_kernel<<<gn, 256, 0, ctx->stream>>>(donor, n, D, ds, k0, ctx->d_err);
    SQ_LAUNCH_CHECK();
    SQ_TRY_CUDA(cudaMemcpyAsync(v0, labels, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    int dbits = 1;
    while ((1 << dbits) < D) ++dbits;
    bool alt = false;
    SQ_TRY(sq_radix_sort_u32(ctx, k0, v0, k1, v1, n, nullptr, 0, dbits, &alt, tmp, tmp_bytes));
    // now (donor, label) in (k, v) of the current buffers: swap roles, sort by label
    uint32_t *don = alt ? k1 : k0, *lab = alt ? v1 : v0;
    uint32_t *don_alt = alt ? k0 : k1, *lab_alt = alt ? v0 : v1;
    SQ_TRY(sq_radix_sort_u32(ctx, lab, don, lab_alt, don_alt, n, nullptr, 0, 31, &alt, tmp, tmp_bytes));
    const uint32_t *L = alt ? lab_alt : lab, *Dn = alt ? don_alt : don;
    run_start_kernel<<<gn, 256, 0, ctx->stream>>>(L, Dn, n, f1, f2);
    SQ_LAUNCH_CHECK();
    SQ_TRY(sq_scan_u32(ctx, f1, s1, n, nullptr, false, false, tot, tmp, tmp_bytes));
    SQ_TRY(sq_scan_u32(ctx, f2, s2, n, nullptr, false, false, tot + 1, tmp, tmp_bytes));
    run_index_kernel<<<gn, 256, 0, ctx->stream>>>(f1, s1, f2, s2, Dn, n, rp, rd, cf);
    SQ_LAUNCH_CHECK();
    js_pairs_kernel<<<sq_grid(ctx, n * 32, 256, 8), 256, 0, ctx->stream>>>(cf, tot + 1, tot, rp, rd, n, ds, D, acc);
    SQ_LAUNCH_CHECK();
    js_finish_kernel<<<sq_grid(ctx, (int64_t)D * D, 256, 8), 256, 0, ctx->stream>>>(acc, ds, D, dist_out);
    SQ_LAUNCH_CHECK();
    return SUBQUAD_OK;
}
