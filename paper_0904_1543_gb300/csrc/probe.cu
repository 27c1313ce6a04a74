// Arithmetic-pipe peak probe: the rate of independent FMA chains on this GPU,
// the denominator of the FP64 and FP32 rooflines (no counterpart in the paper,
// whose Sec. "Performance evaluation of GPU convolution routines" quotes
// rates against its own hardware's peak).  Every thread runs NCH independent
// chains a <- a * b + c, so the pipe, not the dependency latency, bounds the
// kernel; FP32 uses packed FMAs (two per lane per instruction), so the issue
// slots do not bound it either.
#include <algorithm>

#include <cuda_runtime.h>

#include "wvl.h"
#include "wvl_internal.h"

namespace wvl {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int UNROLL = 16;  // FMAs per chain per loop trip

__device__ double g_probe_sink;

// NCH independent chains per thread
template <int NCH>
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_f64(long long trips, double b, double c) {
    double a[NCH];
    #pragma unroll
    for (int k = 0; k < NCH; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (long long t = 0; t < trips; ++t) {
        #pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            #pragma unroll
            for (int k = 0; k < NCH; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
    #pragma unroll
    for (int k = 0; k < NCH; ++k) s += a[k];
    if (s == 1234.5678) g_probe_sink = s;   // keeps the chains live; never true in practice
}

template <int NCH>
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_f32(long long trips, float b, float c) {
    float2 a[NCH];
    #pragma unroll
    for (int k = 0; k < NCH; ++k) a[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (long long t = 0; t < trips; ++t) {
        #pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            #pragma unroll
            for (int k = 0; k < NCH; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
    }
    float s = 0.f;
    #pragma unroll
    for (int k = 0; k < NCH; ++k) s += a[k].x + a[k].y;
    if (s == 1234.5678f) g_probe_sink = s;
}

// one launch of a probe variant: chains per thread 4 / 8 / 16 (v = 0 / 1 / 2)
cudaError_t launch_probe(int prec, int v, long long blocks, long long trips, cudaStream_t st) {
    const unsigned g = (unsigned)blocks;
    if (prec == WVL_F64) {
        if (v == 0) fma_probe_f64<4><<<g, PROBE_THREADS, 0, st>>>(trips, 0.999999, 1e-7);
        else if (v == 1) fma_probe_f64<8><<<g, PROBE_THREADS, 0, st>>>(trips, 0.999999, 1e-7);
        else fma_probe_f64<16><<<g, PROBE_THREADS, 0, st>>>(trips, 0.999999, 1e-7);
    } else {
        if (v == 0) fma_probe_f32<4><<<g, PROBE_THREADS, 0, st>>>(trips, 0.999999f, 1e-7f);
        else if (v == 1) fma_probe_f32<8><<<g, PROBE_THREADS, 0, st>>>(trips, 0.999999f, 1e-7f);
        else fma_probe_f32<16><<<g, PROBE_THREADS, 0, st>>>(trips, 0.999999f, 1e-7f);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace
}  // namespace wvl

using namespace wvl;

extern "C" wvl_status wvl_fma_peak(int prec, double seconds, double* tflops, double* ms,
                                   void* stream) {
    if (!tflops) return WVL_EINVAL;
    if (prec != WVL_F64 && prec != WVL_F32) return WVL_EINVAL;
    if (!(seconds > 0.0) || seconds > 10.0) return WVL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return WVL_ECUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return WVL_ECUDA;
    static const int kChains[3] = {4, 8, 16};
    // flops/s of one launch; trips is raised until the launch takes >= 20 ms
    auto rate = [&](int v, long long blocks, long long& trips, float& t) -> double {
        for (int k = 0; k < 14; ++k) {
            cudaEventRecord(e0, st);
            if (launch_probe(prec, v, blocks, trips, st) != cudaSuccess) return -1.0;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                return -1.0;
            if (t >= 20.f) break;
            trips *= 4;
        }
        const double fmas = (double)blocks * PROBE_THREADS * kChains[v] * UNROLL * (double)trips *
                            (prec == WVL_F32 ? 2.0 : 1.0);
        return 2.0 * fmas / (t * 1e-3);
    };
    // the variant (chains per thread, CTAs per SM: 1, 2, 4 or 8 of 256
    // threads) that runs fastest, then that one for about `seconds`, best of 3
    double best = 0.0, best_ms = 0.0;
    int bv = 1;
    long long bblocks = nsm, btrips = 16;
    wvl_status rs = WVL_OK;
    for (int v = 0; v < 3 && rs == WVL_OK; ++v)
        for (int per = 1; per <= 8; per *= 2) {
            long long trips = 16;
            float t = 0.f;
            const double r = rate(v, (long long)nsm * per, trips, t);
            if (r < 0.0) { rs = WVL_ECUDA; break; }
            if (r > best) { best = r; bv = v; bblocks = (long long)nsm * per; btrips = trips; best_ms = t; }
        }
    if (rs == WVL_OK) {
        long long trips = std::max(1LL, (long long)(btrips * (seconds * 1e3 / std::max(best_ms, 1e-3))));
        for (int k = 0; k < 3; ++k) {
            float t = 0.f;
            long long tr = trips;
            const double r = rate(bv, bblocks, tr, t);
            if (r < 0.0) { rs = WVL_ECUDA; break; }
            if (r > best) { best = r; best_ms = t; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != WVL_OK) return rs;
    *tflops = best / 1e12;
    if (ms) *ms = best_ms;
    return WVL_OK;
}
