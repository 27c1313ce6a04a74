// Deterministic second-stage reductions (paper Sec. "Three dimensional
// operators": the energies are reductions over the grid).  Fixed summation
// order for a fixed launch configuration: no floating-point atomics.
#include <cuda_runtime.h>

#include "wvl_internal.h"

namespace wvl {

// out[o] = sum_t part[o][t] - (minus ? minus[o] : 0); one warp per orbital.
__global__ void reduce_parts_kernel(const double* __restrict__ part,
                                    const double* __restrict__ minus, int tiles,
                                    int norb, double* __restrict__ out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= norb) return;
    const double* p = part + (long long)warp * tiles;
    double s = 0.0;
    for (int t = lane; t < tiles; t += 32) s += p[t];
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[warp] = s - (minus ? minus[warp] : 0.0);
}

// rho[i] += sum_g parts[g * P + i], g in increasing order.
__global__ void rho_reduce_kernel(const double* __restrict__ parts, long long P,
                                  int ngroups, double* __restrict__ rho) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        double s = rho[i];
        for (int g = 0; g < ngroups; ++g) s += parts[g * P + i];
        rho[i] = s;
    }
}

cudaError_t launch_reduce_parts(const double* part, const double* minus, int tiles,
                                int norb, double* out, cudaStream_t st) {
    if (norb <= 0) return cudaSuccess;
    const int threads = 128;
    const int blocks = (norb * 32 + threads - 1) / threads;
    reduce_parts_kernel<<<blocks, threads, 0, st>>>(part, minus, tiles, norb, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rho_reduce(const double* parts, long long P, int ngroups,
                              double* rho, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const int threads = 256;
    long long blocks = (P + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    rho_reduce_kernel<<<(unsigned)blocks, threads, 0, st>>>(parts, P, ngroups, rho);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wvl
