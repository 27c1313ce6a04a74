// Orbital scalar products in compressed form.  The wavelet basis is
// orthonormal (Sec. "Daubechies basis and wavelet transformation": the
// scaling functions and wavelets of Eq. wavef0 are orthonormal, so the scalar
// product of two orbitals is the sum of the products of their coefficients,
// taken directly on the compressed vectors).
//
// S[i][j] = sum_k a_i[k] b_j[k] for blocks of orbitals.  Every product is
// formed in FP64 (FP32 coefficients are converted exactly, and the product of
// two FP32 values is exact in FP64) and accumulated in FP64, by a fixed-order
// two-stage reduction: CTAs own a 32 x 32 tile of S and a slice of k and
// write one partial per tile entry; a second kernel sums the slices in order.
// The contraction is bound by the FP64 pipe (na nb len FMAs for (na + nb) len
// loaded values), so the slices are staged in shared memory as doubles and
// each thread keeps a 2 x 2 block of S in registers.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "wvl.h"
#include "wvl_internal.h"

namespace wvl {
namespace {

constexpr int OV_T = 32;          // tile of S: OV_T x OV_T
constexpr int OV_KC = 64;         // k per shared-memory stage
constexpr int OV_THREADS = 256;   // 16 x 16 threads, 2 x 2 outputs each
constexpr int OV_RS = OV_KC + 1;  // row stride (doubles): rows fall on distinct banks

struct OvParams {
    const void* a;
    const void* b;
    double* part;      // [nsplit][na][nb] partials
    long long len;     // coefficients per orbital
    long long kper;    // k per split (a multiple of OV_KC)
    int na, nb, nsplit;
    int tiles_j;       // tiles along j
    int sym;           // a == b: only tiles with tj >= ti are computed
};

template <typename T>
__global__ void __launch_bounds__(OV_THREADS) overlap_part_kernel(const OvParams q) {
    __shared__ double As[OV_T * OV_RS];
    __shared__ double Bs[OV_T * OV_RS];
    // tile (ti, tj) of this CTA (upper triangle only when symmetric)
    int ti, tj;
    if (q.sym) {
        // blockIdx.y enumerates (ti, tj), tj >= ti, row by row
        int r = blockIdx.y, t = 0;
        const int nt = q.tiles_j;
        while (r >= nt - t) { r -= nt - t; ++t; }
        ti = t;
        tj = t + r;
    } else {
        ti = blockIdx.y / q.tiles_j;
        tj = blockIdx.y - ti * q.tiles_j;
    }
    const int split = blockIdx.x;
    const long long k0 = (long long)split * q.kper;
    const long long k1 = min(q.len, k0 + q.kper);
    const T* A = static_cast<const T*>(q.a);
    const T* B = static_cast<const T*>(q.b);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = ti * OV_T, j0 = tj * OV_T;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (long long kb = k0; kb < k1; kb += OV_KC) {
        // stage 32 rows x 64 k of each block (zero past the ends)
        for (int e = threadIdx.x; e < OV_T * OV_KC; e += OV_THREADS) {
            const int row = e / OV_KC, kk = e - row * OV_KC;
            const long long k = kb + kk;
            const int i = i0 + row, j = j0 + row;
            As[row * OV_RS + kk] = (i < q.na && k < k1) ? (double)A[(long long)i * q.len + k] : 0.0;
            Bs[row * OV_RS + kk] = (j < q.nb && k < k1) ? (double)B[(long long)j * q.len + k] : 0.0;
        }
        __syncthreads();
        #pragma unroll 8
        for (int kk = 0; kk < OV_KC; ++kk) {
            const double a0 = As[(2 * ty) * OV_RS + kk], a1 = As[(2 * ty + 1) * OV_RS + kk];
            const double b0 = Bs[(2 * tx) * OV_RS + kk], b1 = Bs[(2 * tx + 1) * OV_RS + kk];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    double* P = q.part + (long long)split * q.na * q.nb;
    #pragma unroll
    for (int r = 0; r < 2; ++r)
        #pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = i0 + 2 * ty + r, j = j0 + 2 * tx + c;
            if (i < q.na && j < q.nb) P[(long long)i * q.nb + j] = acc[r][c];
        }
}

// S[i][j] = sum_s part[s][i][j], s in increasing order; when symmetric the
// lower-triangle tiles were not computed and take the mirrored entry
__global__ void overlap_reduce_kernel(const double* __restrict__ part, int na, int nb,
                                      int nsplit, int sym, double* __restrict__ S) {
    const long long n = (long long)na * nb;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e / nb), j = (int)(e - (long long)i * nb);
        if (sym && i / OV_T > j / OV_T) { const int t = i; i = j; j = t; }
        double s = 0.0;
        for (int p = 0; p < nsplit; ++p) s += part[(long long)p * n + (long long)i * nb + j];
        S[e] = s;
    }
}

// d[o] partials: block b of orbital o sums a[o][k] b[o][k] over its k
template <typename T>
__global__ void __launch_bounds__(256) dot_part_kernel(const T* __restrict__ a,
                                                       const T* __restrict__ b, long long len,
                                                       double* __restrict__ part) {
    __shared__ double red[8];
    const int o = blockIdx.y;
    const T* x = a + (long long)o * len;
    const T* y = b + (long long)o * len;
    double s = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < len;
         k += (long long)gridDim.x * blockDim.x)
        s = fma((double)x[k], (double)y[k], s);
    #pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[(long long)o * gridDim.x + blockIdx.x] = t;
    }
}

// splits of k: about 608 CTAs (4 per SM of a 152-SM GB300), each slice at
// least 4 stages; the same shape on every GPU, so the workspace bound holds
void overlap_shape(int na, int nb, long long len, bool sym, int& nsplit, long long& kper,
                   int& tiles) {
    const int ti = (na + OV_T - 1) / OV_T, tj = (nb + OV_T - 1) / OV_T;
    tiles = sym ? ti * (ti + 1) / 2 : ti * tj;
    long long ns = std::max(1LL, (608LL + tiles - 1) / tiles);
    ns = std::min(ns, std::max(1LL, len / (4 * OV_KC)));
    kper = (len + ns - 1) / ns;
    kper = (kper + OV_KC - 1) / OV_KC * OV_KC;
    nsplit = (int)std::max(1LL, (len + kper - 1) / kper);
}

constexpr int DOT_BLOCKS = 64;   // partials per orbital of wvl_dot

}  // namespace
}  // namespace wvl

using namespace wvl;

namespace {
wvl_status ov_fail(wvl_status s, const char* msg) { return set_error(s, msg); }
bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }
bool bad_prec(int prec) { return prec != WVL_F64 && prec != WVL_F32 && prec != WVL_F64_EMU; }
}  // namespace

extern "C" wvl_status wvl_overlap_workspace_size(int prec, int na, int nb, long long len,
                                                 size_t* bytes) {
    clear_error();
    if (!bytes) return ov_fail(WVL_EINVAL, "bytes is NULL");
    if (bad_prec(prec)) return ov_fail(WVL_EINVAL, "prec must be WVL_F64, WVL_F32 or WVL_F64_EMU");
    if (na < 0 || nb < 0 || len < 0) return ov_fail(WVL_EINVAL, "negative size");
    const int a1 = std::max(na, 1), b1 = std::max(nb, 1);
    const long long l1 = std::max(len, 1LL);
    int ns0 = 1, ns1 = 1, tiles = 0;
    long long kper = 0;
    overlap_shape(a1, b1, l1, false, ns0, kper, tiles);
    if (a1 == b1) overlap_shape(a1, b1, l1, true, ns1, kper, tiles);
    const size_t ov = (size_t)std::max(ns0, ns1) * (size_t)a1 * (size_t)b1 * sizeof(double);
    const size_t dot = (size_t)std::max(na, 1) * DOT_BLOCKS * sizeof(double);
    *bytes = std::max(ov, dot);
    return WVL_OK;
}

extern "C" wvl_status wvl_overlap(int prec, int na, const void* a, int nb, const void* b,
                                  long long len, double* S, void* ws, size_t ws_bytes,
                                  void* stream) {
    clear_error();
    if (bad_prec(prec)) return ov_fail(WVL_EINVAL, "prec must be WVL_F64, WVL_F32 or WVL_F64_EMU");
    if (na < 0 || nb < 0 || len < 0) return ov_fail(WVL_EINVAL, "negative size");
    if (na == 0 || nb == 0) return WVL_OK;
    if (!a || !b || !S || !ws) return ov_fail(WVL_EINVAL, "a, b, S and ws must not be NULL");
    if (misaligned(a) || misaligned(b) || misaligned(S) || misaligned(ws))
        return ov_fail(WVL_EINVAL, "a, b, S and ws must be 16-byte aligned");
    if (na > (1 << 20) || nb > (1 << 20)) return ov_fail(WVL_EUNSUPPORTED, "too many orbitals");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool sym = (a == b) && (na == nb);
    OvParams q;
    q.a = a;
    q.b = b;
    q.len = len;
    q.na = na;
    q.nb = nb;
    q.sym = sym ? 1 : 0;
    q.tiles_j = (nb + OV_T - 1) / OV_T;
    int tiles = 0;
    overlap_shape(na, nb, std::max(len, 1LL), sym, q.nsplit, q.kper, tiles);
    const size_t need = (size_t)q.nsplit * na * nb * sizeof(double);
    if (ws_bytes < need) return ov_fail(WVL_ENOMEM_WS, "workspace smaller than wvl_overlap_workspace_size()");
    q.part = static_cast<double*>(ws);
    if (tiles > 65535) return ov_fail(WVL_EUNSUPPORTED, "too many tiles");
    const dim3 grid((unsigned)q.nsplit, (unsigned)tiles);
    if (prec == WVL_F32)
        overlap_part_kernel<float><<<grid, OV_THREADS, 0, st>>>(q);
    else
        overlap_part_kernel<double><<<grid, OV_THREADS, 0, st>>>(q);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ov_fail(WVL_ECUDA, cudaGetErrorString(e));
    const long long n = (long long)na * nb;
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 8);
    overlap_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(q.part, na, nb, q.nsplit, q.sym, S);
    count_launches(1);
    e = cudaGetLastError();
    return e == cudaSuccess ? WVL_OK : ov_fail(WVL_ECUDA, cudaGetErrorString(e));
}

extern "C" wvl_status wvl_dot(int prec, int n, const void* a, const void* b, long long len,
                              double* d, void* ws, size_t ws_bytes, void* stream) {
    clear_error();
    if (bad_prec(prec)) return ov_fail(WVL_EINVAL, "prec must be WVL_F64, WVL_F32 or WVL_F64_EMU");
    if (n < 0 || len < 0) return ov_fail(WVL_EINVAL, "negative size");
    if (n == 0) return WVL_OK;
    if (!a || !b || !d || !ws) return ov_fail(WVL_EINVAL, "a, b, d and ws must not be NULL");
    if (misaligned(a) || misaligned(b) || misaligned(d) || misaligned(ws))
        return ov_fail(WVL_EINVAL, "a, b, d and ws must be 16-byte aligned");
    if (n > 65535) return ov_fail(WVL_EUNSUPPORTED, "more than 65535 orbitals");
    if (ws_bytes < (size_t)n * DOT_BLOCKS * sizeof(double))
        return ov_fail(WVL_ENOMEM_WS, "workspace smaller than wvl_overlap_workspace_size()");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* part = static_cast<double*>(ws);
    const dim3 grid(DOT_BLOCKS, (unsigned)n);
    if (prec == WVL_F32)
        dot_part_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(a),
                                                     static_cast<const float*>(b), len, part);
    else
        dot_part_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(a),
                                                      static_cast<const double*>(b), len, part);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ov_fail(WVL_ECUDA, cudaGetErrorString(e));
    e = launch_reduce_parts(part, nullptr, DOT_BLOCKS, n, d, st);
    return e == cudaSuccess ? WVL_OK : ov_fail(WVL_ECUDA, cudaGetErrorString(e));
}
