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

// Several of those sums in one launch, one warp per (task, orbital):
// out[o] = sum_t part[o][t] - sum_t mpart[o][t] (the second sum where mpart
// is set, formed by the same warp in the same order as its own task forms
// it, so the result equals the two launches' bit for bit).
__device__ __forceinline__ double warp_row_sum(const double* __restrict__ p, int tiles, int lane) {
    double s = 0.0;
    for (int t = lane; t < tiles; t += 32) s += p[t];
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}
__global__ void reduce_parts_multi_kernel(const __grid_constant__ PartTasks T) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= T.nwarps) return;
    int k = 0;
    while (k + 1 < T.ntask && warp >= T.t[k + 1].warp0) ++k;
    const PartTask& q = T.t[k];
    const int o = warp - q.warp0;
    double s = warp_row_sum(q.part + (long long)o * q.tiles, q.tiles, lane);
    if (q.mpart != nullptr) s = s - warp_row_sum(q.mpart + (long long)o * q.mtiles, q.mtiles, lane);
    else s = s - 0.0;
    if (lane == 0) q.out[o] = s;
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

// E_loc = sum_o occ[o] (ekin[o] + epot[o]) (Sec. "Full local hamiltonian":
// the local energy of the occupied orbitals): one CTA, thread t sums the
// orbitals t, t + 256, ... in order, then a fixed tree over the threads.
__global__ void eloc_total_kernel(const double* __restrict__ occ,
                                  const double* __restrict__ ekin,
                                  const double* __restrict__ epot, int norb,
                                  double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int o = threadIdx.x; o < norb; o += blockDim.x) s += occ[o] * (ekin[o] + epot[o]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// dE_loc/dV = gbar rho (E_loc is linear in V with coefficient rho in grid
// units), written in the potential's precision.
template <typename T>
__global__ void scale_density_kernel(const double* __restrict__ rho,
                                     const double* __restrict__ gbar, long long P,
                                     T* __restrict__ dV) {
    const double g = *gbar;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride)
        dV[i] = (T)(g * rho[i]);
}

cudaError_t launch_eloc_total(const double* occ, const double* ekin, const double* epot,
                              int norb, double* out, cudaStream_t st) {
    eloc_total_kernel<<<1, 256, 0, st>>>(occ, ekin, epot, norb, out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_density(const double* rho, const double* gbar, long long P, T* dV,
                                 cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const int threads = 256;
    long long blocks = (P + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    scale_density_kernel<T><<<(unsigned)blocks, threads, 0, st>>>(rho, gbar, P, dV);
    count_launches(1);
    return cudaGetLastError();
}
template cudaError_t launch_scale_density<double>(const double*, const double*, long long,
                                                  double*, cudaStream_t);
template cudaError_t launch_scale_density<float>(const double*, const double*, long long,
                                                 float*, cudaStream_t);

cudaError_t launch_reduce_parts(const double* part, const double* minus, int tiles,
                                int norb, double* out, cudaStream_t st) {
    if (norb <= 0) return cudaSuccess;
    const int threads = 128;
    const int blocks = (norb * 32 + threads - 1) / threads;
    reduce_parts_kernel<<<blocks, threads, 0, st>>>(part, minus, tiles, norb, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_reduce_parts_multi(const PartTasks& t, cudaStream_t st) {
    if (t.ntask <= 0 || t.nwarps <= 0) return cudaSuccess;
    const int threads = 128;
    const int blocks = (t.nwarps * 32 + threads - 1) / threads;
    reduce_parts_multi_kernel<<<blocks, threads, 0, st>>>(t);
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
