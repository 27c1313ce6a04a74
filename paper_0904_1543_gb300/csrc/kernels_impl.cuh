// Dispatch of the pass kernels for one element type (included once per type
// by kernels_f64.cu / kernels_f32.cu so the two compile in parallel).
#pragma once
#include <atomic>

#include "pass_kernel.cuh"

namespace wvl {

template <typename T, int KIND, int MODE, int R>
static cudaError_t ensure_attr() {
    // opt in to large dynamic shared memory once per device
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        err = cudaFuncSetAttribute(pass_kernel<T, KIND, MODE, R>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (err != cudaSuccess) return err;
        done.fetch_or(bit);
    }
    return cudaSuccess;
}

// Persistent launch: as many CTAs as fit on the device at once (never more
// than there are work units); each walks its units with a stride of the grid.
template <typename T, int KIND, int MODE, int R>
static cudaError_t launch_one(const PassParams<T>& p, long long nunits, size_t smem,
                              cudaStream_t st, bool persistent) {
    cudaError_t err = ensure_attr<T, KIND, MODE, R>();
    if (err != cudaSuccess) return err;
    if (nunits <= 0) return cudaSuccess;
    int dev = 0, nsm = 0, occ = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pass_kernel<T, KIND, MODE, R>,
                                                        NTHREADS, smem);
    if (err != cudaSuccess) return err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    long long grid = persistent ? (long long)occ * nsm : nunits;
    if (grid > nunits) grid = nunits;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if constexpr (sizeof(T) == 4) {
        PassParams<T> q = p;
        tap_pairs<KIND>(q.f, q.tp);
        pass_kernel<T, KIND, MODE, R><<<dim3((unsigned)grid), dim3(NTHREADS), smem, st>>>(q);
    } else {
        pass_kernel<T, KIND, MODE, R><<<dim3((unsigned)grid), dim3(NTHREADS), smem, st>>>(p);
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int R>
static cudaError_t prepare_r() {
    cudaError_t e;
    if ((e = ensure_attr<T, K_SYN, M_UNCOMP, R>()) != cudaSuccess) return e;
    if ((e = ensure_attr<T, K_SYN, M_PLAIN, R>()) != cudaSuccess) return e;
    if ((e = ensure_attr<T, K_ANA, M_COMP, R>()) != cudaSuccess) return e;
    if ((e = ensure_attr<T, K_ANA, M_PLAIN, R>()) != cudaSuccess) return e;
    if ((e = ensure_attr<T, K_MF, M_POT, R>()) != cudaSuccess) return e;
    if ((e = ensure_attr<T, K_MF, M_PLAIN, R>()) != cudaSuccess) return e;
    if ((e = ensure_attr<T, K_MFT, M_PLAIN, R>()) != cudaSuccess) return e;
    if ((e = ensure_attr<T, K_KIN, M_KMID, R>()) != cudaSuccess) return e;
    return ensure_attr<T, K_KIN, M_KLAST, R>();
}

template <typename T, int R>
static cudaError_t launch_r(int kind, int mode, const PassParams<T>& p, long long nb,
                            size_t smem, cudaStream_t st, bool ps) {
    switch (kind) {
    case K_SYN:
        if (mode == M_UNCOMP) return launch_one<T, K_SYN, M_UNCOMP, R>(p, nb, smem, st, ps);
        if (mode == M_PLAIN) return launch_one<T, K_SYN, M_PLAIN, R>(p, nb, smem, st, ps);
        break;
    case K_ANA:
        if (mode == M_COMP) return launch_one<T, K_ANA, M_COMP, R>(p, nb, smem, st, ps);
        if (mode == M_PLAIN) return launch_one<T, K_ANA, M_PLAIN, R>(p, nb, smem, st, ps);
        break;
    case K_MF:
        if (mode == M_POT) return launch_one<T, K_MF, M_POT, R>(p, nb, smem, st, ps);
        if (mode == M_PLAIN) return launch_one<T, K_MF, M_PLAIN, R>(p, nb, smem, st, ps);
        break;
    case K_MFT:
        if (mode == M_PLAIN) return launch_one<T, K_MFT, M_PLAIN, R>(p, nb, smem, st, ps);
        break;
    case K_KIN:
        if (mode == M_KMID) return launch_one<T, K_KIN, M_KMID, R>(p, nb, smem, st, ps);
        if (mode == M_KLAST) return launch_one<T, K_KIN, M_KLAST, R>(p, nb, smem, st, ps);
        break;
    }
    return cudaErrorInvalidValue;
}

#define WVL_INSTANTIATE_LAUNCH(T)                                                    \
    template <>                                                                      \
    cudaError_t launch_pass<T>(int kind, int mode, int R, const PassParams<T>& p,    \
                               long long nblocks, size_t smem, cudaStream_t st,      \
                               bool ps) {                                            \
        if (R == 4) return launch_r<T, 4>(kind, mode, p, nblocks, smem, st, ps);     \
        if (R == 8) return launch_r<T, 8>(kind, mode, p, nblocks, smem, st, ps);     \
        return cudaErrorInvalidValue;                                                \
    }                                                                                \
    template <>                                                                      \
    cudaError_t prepare_pass_kernels<T>() {                                          \
        cudaError_t e = prepare_r<T, 4>();                                           \
        return e != cudaSuccess ? e : prepare_r<T, 8>();                             \
    }

}  // namespace wvl
