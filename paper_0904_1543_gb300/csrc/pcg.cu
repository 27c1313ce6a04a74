// Vector kernels of the preconditioned conjugate gradient that solves the
// Helmholtz equation of the preconditioning step (paper Eq. precon), one
// independent system per orbital, on compressed coefficients.
//
// Every orbital has its own scalars (alpha, beta, r.z) kept on the device, so
// the iteration never synchronises with the host.  Dot products are two-stage
// and deterministic: per-block partials (products and sums in FP64 in both
// modes), then the fixed-order warp reduction of reduce.cu.
#include <cuda_runtime.h>

#include "pass_kernel.cuh"
#include "wvl_internal.h"

namespace wvl {

constexpr int PCG_THREADS = 256;

// compressed position k of a cell with m coarse points -> component mu
__device__ __forceinline__ int comp_mu(long long k, long long m) {
    return k < m ? 0 : (int)((k - m) % 7) + 1;
}

template <typename T>
__device__ __forceinline__ void block_partial(double v, double* out) {
    __shared__ double red[PCG_THREADS / 32];
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < PCG_THREADS / 32; ++w) t += red[w];
        *out = t;
    }
}

// 1 / (d_mu - eps_o) for the 8 components, in shared memory
template <typename T>
__device__ __forceinline__ void load_minv(const PcgParams& q, int o, T* minv) {
    if (threadIdx.x < 8) minv[threadIdx.x] = T(1.0 / (q.diag[threadIdx.x] - q.eps[o]));
    __syncthreads();
}

// x = 0, r = g, z = M^-1 r, p = z; partial r.z
template <typename T>
__global__ void __launch_bounds__(PCG_THREADS)
pcg_init_kernel(const PcgParams q, const T* __restrict__ g, T* x, T* r, T* z, T* p) {
    __shared__ T minv[8];
    const int o = blockIdx.y;
    load_minv<T>(q, o, minv);
    const long long base = (long long)o * q.len;
    Acc<T> acc;
    for (long long k = (long long)blockIdx.x * PCG_THREADS + threadIdx.x; k < q.len;
         k += (long long)gridDim.x * PCG_THREADS) {
        const T gv = g[base + k];
        const T zv = minv[comp_mu(k, q.m)] * gv;
        x[base + k] = T(0);
        r[base + k] = gv;
        z[base + k] = zv;
        p[base + k] = zv;
        acc.fma_add(gv, zv);
    }
    block_partial<T>(acc.get(), q.part + (long long)o * gridDim.x + blockIdx.x);
}

// partial a.b per orbital
template <typename T>
__global__ void __launch_bounds__(PCG_THREADS)
pcg_dot_kernel(const PcgParams q, const T* __restrict__ a, const T* __restrict__ b) {
    const int o = blockIdx.y;
    const long long base = (long long)o * q.len;
    Acc<T> acc;
    for (long long k = (long long)blockIdx.x * PCG_THREADS + threadIdx.x; k < q.len;
         k += (long long)gridDim.x * PCG_THREADS)
        acc.fma_add(a[base + k], b[base + k]);
    block_partial<T>(acc.get(), q.part + (long long)o * gridDim.x + blockIdx.x);
}

// alpha = rz / pq; x += alpha p; r -= alpha Ap; z = M^-1 r; partial r.z
template <typename T>
__global__ void __launch_bounds__(PCG_THREADS)
pcg_step_kernel(const PcgParams q, T* x, T* r, T* z, const T* __restrict__ p,
                const T* __restrict__ Ap, const double* __restrict__ rz,
                const double* __restrict__ pq) {
    __shared__ T minv[8];
    const int o = blockIdx.y;
    load_minv<T>(q, o, minv);
    const T alpha = T(rz[o] / pq[o]);
    const long long base = (long long)o * q.len;
    Acc<T> acc;
    for (long long k = (long long)blockIdx.x * PCG_THREADS + threadIdx.x; k < q.len;
         k += (long long)gridDim.x * PCG_THREADS) {
        x[base + k] += alpha * p[base + k];
        const T rv = r[base + k] - alpha * Ap[base + k];
        r[base + k] = rv;
        const T zv = minv[comp_mu(k, q.m)] * rv;
        z[base + k] = zv;
        acc.fma_add(rv, zv);
    }
    block_partial<T>(acc.get(), q.part + (long long)o * gridDim.x + blockIdx.x);
}

// beta = rz_new / rz_old; p = z + beta p
template <typename T>
__global__ void __launch_bounds__(PCG_THREADS)
pcg_dir_kernel(const PcgParams q, T* p, const T* __restrict__ z,
               const double* __restrict__ rz_new, const double* __restrict__ rz_old) {
    const int o = blockIdx.y;
    const T beta = T(rz_new[o] / rz_old[o]);
    const long long base = (long long)o * q.len;
    for (long long k = (long long)blockIdx.x * PCG_THREADS + threadIdx.x; k < q.len;
         k += (long long)gridDim.x * PCG_THREADS)
        p[base + k] = z[base + k] + beta * p[base + k];
}

static dim3 pcg_grid(const PcgParams& q) { return dim3(q.nblk, q.norb); }

template <typename T>
cudaError_t launch_pcg(int which, const PcgParams& q, T* a, T* b, T* c, T* d, const T* e,
                       const double* s1, const double* s2, cudaStream_t st) {
    if (q.norb <= 0) return cudaSuccess;
    switch (which) {
    case PCG_INIT:
        pcg_init_kernel<T><<<pcg_grid(q), PCG_THREADS, 0, st>>>(q, e, a, b, c, d);
        break;
    case PCG_DOT:
        pcg_dot_kernel<T><<<pcg_grid(q), PCG_THREADS, 0, st>>>(q, a, b);
        break;
    case PCG_STEP:
        pcg_step_kernel<T><<<pcg_grid(q), PCG_THREADS, 0, st>>>(q, a, b, c, d, e, s1, s2);
        break;
    case PCG_DIR:
        pcg_dir_kernel<T><<<pcg_grid(q), PCG_THREADS, 0, st>>>(q, a, c, s1, s2);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_pcg<double>(int, const PcgParams&, double*, double*, double*,
                                        double*, const double*, const double*, const double*,
                                        cudaStream_t);
template cudaError_t launch_pcg<float>(int, const PcgParams&, float*, float*, float*, float*,
                                       const float*, const double*, const double*,
                                       cudaStream_t);

}  // namespace wvl
