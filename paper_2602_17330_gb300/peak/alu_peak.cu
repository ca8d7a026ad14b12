// Integer / min-max issue-rate microbenchmark for the alignment roofline.
//
// Each kernel runs long chains of one operation on 8 independent registers per
// thread, in CTAs that are all resident at once (8 per SM).  Every CTA records
// its SM id and clock64() at start and end; per SM, lane-operations divided by
// the SM's busy cycles gives operations per SM per clock, independent of the
// clock frequency.
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA error %s at %d\n", cudaGetErrorString(e), __LINE__); exit(1); } } while (0)

constexpr int kThreads = 256;
constexpr int kIters = 4096;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned smid() { unsigned r; asm volatile("mov.u32 %0, %%smid;" : "=r"(r)); return r; }

template <int OP>
__global__ void __launch_bounds__(kThreads) probe(int *out, long long *rec, int seed)
{
    int v[kChains];
    const int t = threadIdx.x + seed;
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = t * (c + 3) + c;
    const int a = seed & 7, b = (seed >> 3) | 1;
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) v[c] = v[c] + v[(c + 1) & 7] + it;                     // 3-input add
            if (OP == 1) v[c] = max(v[c], a + it);                              // plain int max (loop-variant operand)
            if (OP == 2) v[c] = __vimax3_s32_relu(v[c], a, b + it);             // max of three, relu
            if (OP == 3) v[c] = __viaddmax_s32_relu(v[c], -b, a + it);          // add then max, relu
            if (OP == 4) v[c] = __vimax3_s16x2_relu(v[c], a, b + it);           // packed 16-bit max3
            if (OP == 5) v[c] = __viaddmax_s16x2_relu(v[c], b, a + it);         // packed 16-bit add-max
            if (OP == 6) v[c] = v[c] * b + a;                                   // integer multiply-add
            if (OP == 7) v[c] = __float_as_int(fmaxf(__int_as_float(v[c]), __int_as_float(a + it)));  // fp32 max
            if (OP == 8) v[c] = max(max(v[c], a + it), v[(c + 3) & 7]);                 // two-level int max
            if (OP == 9) v[c] = __vmaxs2(v[c], a + it);                                 // packed 16-bit max
            if (OP == 10) v[c] = __vadd2(v[c], v[(c + 1) & 7]);                         // packed 16-bit add
            if (OP == 11) v[c] = __vimax_s32_relu(v[c], v[(c + 5) & 7]);                // max with 0
            if (OP >= 12 && OP <= 14) {
                __half2 x = *reinterpret_cast<__half2 *>(&v[c]);
                __half2 y = *reinterpret_cast<__half2 *>(&v[(c + 1) & 7]);
                __half2 r = OP == 12 ? __hadd2(x, y) : OP == 13 ? __hmax2(x, y) : __hfma2(x, y, x);
                v[c] = *reinterpret_cast<int *>(&r);
            }
            if (OP == 15) v[c] = __float_as_int(__int_as_float(v[c]) + __int_as_float(v[(c + 1) & 7]));   // fadd
            if (OP == 16) v[c] = __float_as_int(fmaf(__int_as_float(v[c]), __int_as_float(b), __int_as_float(v[(c + 1) & 7])));
            if (OP == 17) v[c] = __byte_perm(v[c], v[(c + 1) & 7], 0x5410);              // prmt
            if (OP == 18) v[c] = (v[c] ^ v[(c + 1) & 7]) & (v[(c + 2) & 7] | a);        // lop3
            if (OP == 19) v[c] = __float_as_int(fmaxf(fmaxf(__int_as_float(v[c]), __int_as_float(v[(c + 1) & 7])),
                                                      __int_as_float(v[(c + 2) & 7])));  // two fp32 max
            if (OP == 20) v[c] = __vmaxs2(__vmaxs2(v[c], v[(c + 1) & 7]), v[(c + 2) & 7]);  // two packed maxes
            if (OP == 21) v[c] = v[c] + v[(c + 1) & 7];                                  // 2-input add
            if (OP == 22) v[c] = __viaddmin_s16x2(v[c], b, a + it);                        // packed 16-bit add-min
            if (OP == 23) v[c] = __vimin3_s16x2(v[c], a, b + it);                          // packed 16-bit min3
            if (OP == 24) v[c] = __vmins2(v[c], a + it);                                   // packed 16-bit min
        }
    }
    long long t1 = clock64();
    int s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= v[c];
    if (s == 0x7fffffff) out[0] = s;
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = smid();
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

template <int OP>
double run(int sms, int per_sm, int *out, long long *rec, const char *name)
{
    int blocks = sms * per_sm;
    probe<OP><<<blocks, kThreads>>>(out, rec, 1);  // warm
    CK(cudaDeviceSynchronize());
    probe<OP><<<blocks, kThreads>>>(out, rec, 5);
    CK(cudaDeviceSynchronize());
    std::vector<long long> h(3 * blocks);
    CK(cudaMemcpy(h.data(), rec, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost));
    const int kMaxSm = 4096;
    std::vector<long long> lo(kMaxSm, -1), hi(kMaxSm, -1);
    std::vector<int> cnt(kMaxSm, 0);
    for (int k = 0; k < blocks; ++k) {
        int s = (int)h[3 * k];
        if (s < 0 || s >= kMaxSm) continue;
        if (lo[s] < 0 || h[3 * k + 1] < lo[s]) lo[s] = h[3 * k + 1];
        if (hi[s] < 0 || h[3 * k + 2] > hi[s]) hi[s] = h[3 * k + 2];
        cnt[s]++;
    }
    double sum = 0; int used = 0;
    for (int s = 0; s < kMaxSm; ++s) if (cnt[s] > 0 && hi[s] > lo[s]) {
        double ops = (double)cnt[s] * kThreads * kIters * kChains;
        sum += ops / (double)(hi[s] - lo[s]);
        ++used;
    }
    double per_sm_clk = sum / used;
    printf("%-28s %8.1f lane-ops/SM/clk  (%d SMs, %d CTAs/SM)\n", name, per_sm_clk, used, per_sm);
    return per_sm_clk;
}

// Shared-memory lookups with the alignment kernel's pattern: a lane-replicated
// table (word index * 32 + lane), data-dependent word index per lookup.
__global__ void __launch_bounds__(kThreads) lds_probe_kernel(int *out, long long *rec, int seed)
{
    __shared__ int tab[420 * 32];
    for (int q = threadIdx.x; q < 420 * 32; q += blockDim.x) tab[q] = (q * 7 + seed) % 419;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int idx[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) idx[c] = (threadIdx.x * 13 + c * 29 + seed) % 419;
    long long t0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) idx[c] = tab[idx[c] * 32 + lane];
    }
    long long t1 = clock64();
    int s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= idx[c];
    if (s == 0x7fffffff) out[0] = s;
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = smid();
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

void lds_probe(int sms, int *out, long long *rec)
{
    const int per_sm = 4;  // 53.8 KB of shared memory per CTA
    const int blocks = sms * per_sm;
    lds_probe_kernel<<<blocks, kThreads>>>(out, rec, 1);
    CK(cudaDeviceSynchronize());
    lds_probe_kernel<<<blocks, kThreads>>>(out, rec, 3);
    CK(cudaDeviceSynchronize());
    std::vector<long long> h(3 * blocks);
    CK(cudaMemcpy(h.data(), rec, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost));
    const int kMaxSm = 4096;
    std::vector<long long> lo(kMaxSm, -1), hi(kMaxSm, -1);
    std::vector<int> cnt(kMaxSm, 0);
    for (int k = 0; k < blocks; ++k) {
        int s = (int)h[3 * k];
        if (s < 0 || s >= kMaxSm) continue;
        if (lo[s] < 0 || h[3 * k + 1] < lo[s]) lo[s] = h[3 * k + 1];
        if (hi[s] < 0 || h[3 * k + 2] > hi[s]) hi[s] = h[3 * k + 2];
        cnt[s]++;
    }
    double sum = 0; int used = 0;
    for (int s = 0; s < kMaxSm; ++s) if (cnt[s] > 0 && hi[s] > lo[s]) {
        sum += (double)cnt[s] * kThreads * kIters * kChains / (double)(hi[s] - lo[s]);
        ++used;
    }
    printf("%-28s %8.1f lane-loads/SM/clk  (%d SMs, %d CTAs/SM; dependent chains)\n", "lds lane-replicated", sum / used,
           used, per_sm);
}

int main()
{
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, 0));
    printf("device %s, %d SMs, cc %d.%d\n", p.name, p.multiProcessorCount, p.major, p.minor);
    int sms = p.multiProcessorCount, per_sm = 8;
    int *out; long long *rec;
    CK(cudaMalloc(&out, 64));
    CK(cudaMalloc(&rec, sizeof(long long) * 3 * sms * per_sm));
    run<0>(sms, per_sm, out, rec, "iadd3 (a+b+c)");
    run<1>(sms, per_sm, out, rec, "imax");
    run<2>(sms, per_sm, out, rec, "__vimax3_s32_relu");
    run<3>(sms, per_sm, out, rec, "__viaddmax_s32_relu");
    run<4>(sms, per_sm, out, rec, "__vimax3_s16x2_relu");
    run<5>(sms, per_sm, out, rec, "__viaddmax_s16x2_relu");
    run<6>(sms, per_sm, out, rec, "imad (a*b+c)");
    run<7>(sms, per_sm, out, rec, "fmaxf");
    run<8>(sms, per_sm, out, rec, "max(max(a,b),c)");
    run<9>(sms, per_sm, out, rec, "__vmaxs2");
    run<10>(sms, per_sm, out, rec, "__vadd2");
    run<11>(sms, per_sm, out, rec, "__vimax_s32_relu");
    run<12>(sms, per_sm, out, rec, "__hadd2");
    run<13>(sms, per_sm, out, rec, "__hmax2");
    run<14>(sms, per_sm, out, rec, "__hfma2");
    run<15>(sms, per_sm, out, rec, "fadd");
    run<16>(sms, per_sm, out, rec, "ffma");
    run<17>(sms, per_sm, out, rec, "prmt");
    run<18>(sms, per_sm, out, rec, "lop3 (xor/and/or)");
    run<19>(sms, per_sm, out, rec, "fmaxf(fmaxf(a,b),c)");
    run<20>(sms, per_sm, out, rec, "__vmaxs2(__vmaxs2(a,b),c)");
    run<21>(sms, per_sm, out, rec, "iadd (2-input)");
    run<22>(sms, per_sm, out, rec, "__viaddmin_s16x2");
    run<23>(sms, per_sm, out, rec, "__vimin3_s16x2");
    run<24>(sms, per_sm, out, rec, "__vmins2");
    lds_probe(sms, out, rec);
    CK(cudaFree(out));
    CK(cudaFree(rec));
    return 0;
}
