// The emulated FP64 pass (see emu.cuh for the arithmetic) as a tcgen05
// kernel for sm_103a.
//
// A window is 128 lines x N outputs (N = 32, or 16 for the kinetic filter)
// reading 48 input positions, three 16-position slabs.  A work unit is a
// whole 128-line tile of one orbital (of each orbital of a group in turn in
// the potential pass, whose density partial it updates in place), walked
// window by window.  A persistent CTA of 256 threads, two per SM, per window
//   1. slices the window's new slabs: reads them (wrapped periodically, or
//      gathered from the compressed layout in synthesis pass 1), scales every
//      line by its largest exponent (taken once per unit), and writes six
//      FP16 digit planes into a ring of three slab slots in shared memory, in
//      the MMA's K-major layout (8 x 16 B core matrices);
//   2. issues, from one thread, 6 data digits x 3 K-steps of MMAs
//      (M = 128, K = 16), each over the filter digits side by side along N,
//      adding the 26 digit pairs' products into seven FP32 accumulators
//      (one per diagonal, N columns each) in tensor memory, and commits them
//      to an mbarrier, polled with a bound; meanwhile every thread loads the
//      epilogue's other inputs;
//   3. reads the accumulators (warp w: lines 32 (w % 4) + lane, half of the
//      outputs), recombines them into 64-bit integers, scales to FP64 and
//      runs the pass's epilogue (transposed store, compressed scatter, V psi
//      with density and Epot, kinetic K_p and Ekin) as the FP64 pass does.
// The filter digit planes are built once per CTA from the launch's taps.
#include <cmath>

#include <cuda_fp16.h>

#include "emu.cuh"
#include "pass_kernel.cuh"

namespace wvl {

__device__ unsigned int g_emu_timeouts = 0;

namespace emu {

constexpr long long WAIT_CYCLES = 4000000000LL;   // about two seconds

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: no swizzle, K-major core matrices
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor: kind::f16, FP16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t accumulate) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(mbar) : "memory");
}
__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
        if (clock64() - t0 > WAIT_CYCLES) return false;
    }
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tld8(uint32_t addr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(addr));
}
__device__ __forceinline__ void tld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// input value at position x (0 <= x < n) of line a of orbital orb
template <int MODE>
__device__ __forceinline__ double load_in(const Seg<double>& S, int orb, int a, int x) {
    if (MODE == M_UNCOMP) {
        // line a = (x3, x2) of the interleaved coarse array: element x is
        // c^mu[x3/2][x2/2][x/2], mu = (x & 1) + 2 (x2 & 1) + 4 (x3 & 1)
        const int x3 = a / S.N2, x2 = a - x3 * S.N2;
        const int mu = (x & 1) + 2 * (x2 & 1) + 4 * (x3 & 1);
        const double* cc = S.in + (long long)orb * S.clen;
        const long long ci = ((long long)(x3 >> 1) * S.n2 + (x2 >> 1)) * S.n1 + (x >> 1);
        if (S.mapc == nullptr && S.bx1 == 0)
            return (mu == 0) ? cc[ci] : cc[S.ncoarse + ci * 7 + mu - 1];
        const int k = stored_index(S, ci, x >> 1, x2 >> 1, x3 >> 1, mu);
        if (k < 0) return 0.0;
        return (mu == 0) ? cc[k] : cc[S.ncoarse + (long long)k * 7 + mu - 1];
    }
    return S.in[(long long)orb * S.P + (long long)a * S.n + x];
}

// One job: orbital orb of work unit u (line tile x output window).
struct EJob {
    long long u;
    int si, grp, tt, a0, o, lt, orb, oe;
    bool valid;
};

__device__ __forceinline__ void decode_unit(const PassParams<double>& p, int mode, EJob& J) {
    J.valid = J.u < p.nunits;
    if (!J.valid) return;
    int si = 0;
    while (si + 1 < p.nseg && J.u >= p.seg[si + 1].blk0) ++si;
    const Seg<double>& S = p.seg[si];
    const long long loc = J.u - S.blk0;
    J.si = si;
    J.grp = (int)(loc / S.tiles);
    J.tt = (int)(loc - (long long)J.grp * S.tiles);
    // unit = (orbital, or orbital group in the potential pass) x a whole
    // tile of lines; the kernel walks the tile's windows
    J.a0 = J.tt * M;
    J.o = 0;
    J.lt = min(M, S.N - J.a0);
    if (mode == M_POT) {
        J.orb = J.grp * S.opg;
        J.oe = min(S.norb, J.orb + S.opg);
    } else {
        J.orb = J.grp;
        J.oe = J.grp + 1;
    }
}
__device__ __forceinline__ void first_job(const PassParams<double>& p, int mode, EJob& J) {
    J.u = blockIdx.x;
    decode_unit(p, mode, J);
}
// returns true when J was the last orbital of its unit
__device__ __forceinline__ bool next_job(const PassParams<double>& p, int mode, EJob& J) {
    if (J.orb + 1 < J.oe) {
        ++J.orb;
        return false;
    }
    J.u += gridDim.x;
    decode_unit(p, mode, J);
    return true;
}

// The 26 digit pairs of the canonical schedule (diagonal d = 2..8, i.e.
// dq + fp = d - 2 <= 6, accumulating in tensor-memory columns (d - 2) N..)
// as 6 data digits x 3 K-steps: the MMA of data digit dq multiplies it by the
// filter digits fp = 0 .. 6 - dq side by side (N (7 - dq) columns from column
// dq N), so one instruction adds the products of every pair with that dq to
// their diagonals.  The first one (dq = 0, K-step 0) also meets the zero
// block (fp = 6) and so starts all seven accumulators.  Every exact
// diagonal's partial sums stay integers below 2^24 in any order, so the
// order of the pairs does not change the result.  K-step k reads the data
// planes' slab slot (slot0 + k) mod 3; the shared-memory descriptors are base
// + compile-time offsets.
template <int KIND, int MODE>
__device__ __forceinline__ void issue_window_mmas(uint32_t tm, uint32_t a_base, uint32_t b_base,
                                                  int slot0) {
    constexpr int LBOA = lboa(MODE);
    constexpr int APL = plane_a_bytes(KIND, MODE);
    constexpr int N = window_n(KIND), LBOB = lbo_b(KIND), K = window_k(KIND);
    static_assert(S == 6 && DMAX - 2 == S, "one block per filter digit plus the zero block");
    const uint64_t a0d = mdesc(a_base, LBOA, 128), b0d = mdesc(b_base, LBOB, 128);
    uint32_t aoff[K / 16];
#pragma unroll
    for (int k = 0; k < K / 16; ++k) {
        int sl = slot0 + k;
        sl -= (sl >= K / 16) ? K / 16 : 0;
        aoff[k] = (uint32_t)(sl * 2 * LBOA) >> 4;
    }
#pragma unroll
    for (int dq = 0; dq < S; ++dq) {
        const uint32_t idesc = idesc_f16(M, N * (S + 1 - dq));
#pragma unroll
        for (int k = 0; k < K / 16; ++k)
            mma(tm + dq * N, a0d + (uint64_t)(((uint32_t)(dq * APL) >> 4) + aoff[k]),
                b0d + (uint64_t)((2 * k * LBOB) >> 4), idesc, (dq == 0 && k == 0) ? 0u : 1u);
    }
}

// digits of two consecutive inputs of line r into the data planes at the
// given chunk (8 positions) and pair within it
template <int LBOA>
__device__ __forceinline__ void store_pair_digits(unsigned char* Asm, int apl, int chunk, int r,
                                                  int pair4, double v0, double v1, int E) {
    uint32_t h[S];
    digit_pairs(quantize(v0, E), quantize(v1, E), h);
    unsigned char* dst = Asm + chunk * LBOA + r * 16 + pair4 * 4;
#pragma unroll
    for (int q = 0; q < S; ++q) *reinterpret_cast<uint32_t*>(dst + q * apl) = h[q];
}

// The epilogue's other inputs for this thread's outputs (line er, outputs
// o0 .. o0 + N/2 - 1), loaded while the MMAs run: the kinetic passes' G and
// K_{p-1} (line-major, 16-byte loads) and K_0; the potential pass's V and
// the density accumulated so far.
template <int KIND, int MODE>
__device__ __forceinline__ void prefetch_epilogue(const Seg<double>& Sg, int o0, int er, int lt,
                                                  int a0, int orb, int grp,
                                                  double (&pa)[window_n(KIND) / 2],
                                                  double (&pb)[window_n(KIND) / 2],
                                                  double (&pc)[window_n(KIND) / 2]) {
    constexpr int NH = window_n(KIND) / 2;
    constexpr bool KM = (MODE == M_KMID || MODE == M_KLAST);
    if (!(KM || MODE == M_POT)) return;
    const int n = Sg.n, NL = Sg.N;
    const int a = a0 + er;
    const long long obase = (long long)orb * Sg.P;
    const bool full = er < lt && o0 + NH <= n;   // all outputs exist: vector loads
#pragma unroll
    for (int c = 0; c < NH; ++c) pa[c] = pb[c] = pc[c] = 0.0;
    if (er >= lt) return;
    if (KM) {
        const double* gi = Sg.in + obase + (long long)a * n + o0;
        const double* ki = Sg.in2 ? Sg.in2 + obase + (long long)a * n + o0 : nullptr;
        if (full) {
#pragma unroll
            for (int c = 0; c < NH; c += 2) {
                const double2 g2 = *reinterpret_cast<const double2*>(gi + c);
                pa[c] = g2.x;
                pa[c + 1] = g2.y;
                if (ki) {
                    const double2 k2 = *reinterpret_cast<const double2*>(ki + c);
                    pb[c] = k2.x;
                    pb[c + 1] = k2.y;
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < NH; ++c)
                if (o0 + c < n) {
                    pa[c] = gi[c];
                    if (ki) pb[c] = ki[c];
                }
        }
        if (MODE == M_KLAST && Sg.aux)
#pragma unroll
            for (int c = 0; c < NH; ++c)
                if (o0 + c < n) pc[c] = Sg.aux[obase + (long long)(o0 + c) * NL + a];
    } else if (MODE == M_POT) {
        if (Sg.aux)
#pragma unroll
            for (int c = 0; c < NH; ++c)
                if (o0 + c < n) pa[c] = Sg.aux[(long long)(o0 + c) * NL + a];
        // the density so far is read in the epilogue: prefetched too, it
        // would stay live across the MMAs beside V and spill
    }
}

// one window's outputs of this thread (line er, outputs o0 .. o0 + N/2 - 1):
// accumulators -> FP64 -> the pass's epilogue; returns the energy partial
template <int KIND, int MODE>
__device__ __forceinline__ double window_epilogue(const Seg<double>& Sg, uint32_t tl, int o0,
                                                  int er, int lt, int a0, int orb, int grp, int se,
                                                  const double (&pa)[window_n(KIND) / 2],
                                                  const double (&pb)[window_n(KIND) / 2],
                                                  const double (&pc)[window_n(KIND) / 2]) {
    constexpr int N = window_n(KIND), NH = N / 2;
    constexpr bool KM = (MODE == M_KMID || MODE == M_KLAST);
    const int n = Sg.n, NL = Sg.N;
    se = max(-1022, min(1023, se));
    // 2^se as a double: the FP64 pipe is idle here, the integer pipes are not
    const double scale = __longlong_as_double((long long)(se + 1023) << 52);
    const bool row_ok = er < lt;
    const int a = a0 + er;
    const long long obase = (long long)orb * Sg.P;
    double occ = 1.0;
    if (MODE == M_POT) occ = Sg.occ ? Sg.occ[orb] : 1.0;
    // M_COMP for the adjoint of E_loc: H psi scaled by 2 occ g
    double osc = 1.0;
    if (MODE == M_COMP && Sg.gscale != nullptr) osc = 2.0 * Sg.occ[orb] * Sg.gscale[0];
    double eacc = 0.0;
#pragma unroll
    for (int c8 = 0; c8 < NH / 8; ++c8) {
        uint32_t dv[NACC][8];
#pragma unroll
        for (int ac = 0; ac < NACC; ++ac) tld8(tl + ac * N + c8 * 8, dv[ac]);
        tld_wait();
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            long long t = 0;
            float low = 0.f;
#pragma unroll
            for (int ac = 0; ac < NACC; ++ac) {
                const float v = __uint_as_float(dv[ac][jj]);
                // shifts and weights of the canonical schedule (checked on the host)
                if (ac < NEXACT) t += (long long)__float2int_rn(v) << (DBITS * (DMAX - 2 - ac) - TSHIFT);
                else low = fmaf(v, __int_as_float((127 + DBITS * (DMAX - 2 - ac) - TSHIFT) << 23), low);
            }
            t += __float2int_rn(low);
            const double val = (double)t * scale;
            const int c = c8 * 8 + jj;
            const int I = o0 + c;
            if (!row_ok || I >= n) continue;
            const long long oidx = (long long)I * NL + a;
            if (MODE == M_PLAIN || MODE == M_UNCOMP) {
                Sg.out[obase + oidx] = val;
            } else if (MODE == M_COMP) {
                const int X2 = a / Sg.N1, X1 = a - X2 * Sg.N1;
                const int mu = (X1 & 1) + 2 * (X2 & 1) + 4 * (I & 1);
                const long long ci = ((long long)(I >> 1) * Sg.n2 + (X2 >> 1)) * Sg.n1 + (X1 >> 1);
                double* cc0 = Sg.out + (long long)orb * Sg.clen;
                const double sv = Sg.gscale != nullptr ? val * osc : val;
                if (Sg.mapc == nullptr && Sg.bx1 == 0) {
                    if (mu == 0) cc0[ci] = sv;
                    else cc0[Sg.ncoarse + ci * 7 + mu - 1] = sv;
                } else {
                    const int k = stored_index(Sg, ci, X1 >> 1, X2 >> 1, I >> 1, mu);
                    if (k >= 0) {
                        if (mu == 0) cc0[k] = sv;
                        else cc0[Sg.ncoarse + (long long)k * 7 + mu - 1] = sv;
                    }
                }
            } else if (KM) {
                const double g = pa[c];
                double kin = pb[c];
                if (MODE == M_KMID && Sg.in2 == nullptr && Sg.eps != nullptr) kin = -Sg.eps[orb] * g;
                const double acc = val + kin;
                if (MODE == M_KMID) {
                    Sg.out[obase + oidx] = acc;
                    Sg.out2[obase + oidx] = g;
                } else {
                    if (Sg.out) Sg.out[obase + oidx] = acc;
                    eacc = fma(g, acc - pc[c], eacc);
                }
            } else if (MODE == M_POT) {
                if (Sg.aux) {
                    const double y = pa[c] * val;
                    if (Sg.out) Sg.out[obase + oidx] = y;
                    eacc = fma(y, val, eacc);
                }
                // the unit owns these density elements: one thread updates
                // each, orbital after orbital, in a fixed order; the density
                // so far is the caller's rho, or this group's partial after
                // the group's first orbital
                if (Sg.rho != nullptr) {
                    double* const rp = Sg.rho + (long long)grp * Sg.rho_gstride + oidx;
                    const double prev = (Sg.rho_gstride == 0 || orb != grp * Sg.opg) ? *rp : 0.0;
                    *rp = fma(occ * val, val, prev);
                }
            }
        }
    }
    return eacc;
}

// fixed-order CTA sum of one value per thread
__device__ __forceinline__ double cta_sum(double v, double* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
#pragma unroll
        for (int w = 0; w < WARPS; ++w) t += red[w];
    return t;
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(THREADS, 2)
emu_pass_kernel(const __grid_constant__ Params ep) {
    constexpr int K = window_k(KIND), HA = window_ha(KIND);
    constexpr int LBOA = lboa(MODE);
    constexpr int APL = plane_a_bytes(KIND, MODE);
    constexpr int NT = KT<KIND>::NT;
    constexpr int N = window_n(KIND), LBOB = lbo_b(KIND), TCOLS = tmem_cols(KIND);
    constexpr int NH = N / 2;                // outputs per epilogue thread
    constexpr int RPW = M / WARPS;           // lines per slicing warp
    constexpr int NSLOT = K / 16;            // 16-position slabs per window (3)
    static_assert(K == 48 && N % 16 == 0 && (HA - (KIND == K_KIN ? 0 : 8)) % 16 == 0, "window");
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* const Asm = sm;                // [S][APL]: NSLOT slab slots of 2 chunks
    unsigned char* const Bsm = sm + S * APL;      // K / 8 chunks of (S + 1) N rows
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int rowE[M];
    __shared__ double red[WARPS];

    const PassParams<double>& p = ep.p;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---------------------------------------------- filter digit planes
    int ebf = 0;
    for (int e = 0; e < 2; ++e)
        for (int t = 0; t < NT; ++t) ebf = max(ebf, bexp(p.f[e][t]));
    const int Ef = scale_of(ebf);
    for (int i = tid; i < N * K; i += THREADS) {
        const int j = i / K, k = i - j * K;
        const int e = j & 1;
        const int t = k - j - (HA - p.hl) - (e ? KT<KIND>::OFF1 : KT<KIND>::OFF0);
        const double f = (t >= 0 && t < NT) ? p.f[e][t] : 0.0;
        int d[S];
        digits(quantize(f, Ef), d);
        unsigned char* const b = Bsm + (k >> 3) * LBOB + j * 16 + (k & 7) * 2;
#pragma unroll
        for (int q = 0; q < S; ++q)
            *reinterpret_cast<__half*>(b + q * N * 16) = __int2half_rn(d[q]);
        *reinterpret_cast<__half*>(b + S * N * 16) = __float2half(0.f);   // the zero block
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&tslot)), "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tm = tslot;
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (lines)
    // and one half of the window's outputs
    const int quarter = warp & 3, half = warp >> 2;
    const int er = 32 * quarter + lane;
    const uint32_t tl = tm + ((uint32_t)(32 * quarter) << 16) + NH * half;
    const uint32_t a_base = su32(Asm), b_base = su32(Bsm);
    uint32_t phase = 0;
    bool failed = false;

    // MMAs of one window, then the wait: one thread polls, the others sleep
    // in the barrier instead of taking issue slots from the co-resident CTA
    auto issue_mmas = [&](int slot0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            issue_window_mmas<KIND, MODE>(tm, a_base, b_base, slot0);
            commit(su32(&mbar));
        }
    };
    auto wait_mmas = [&]() -> bool {
        bool ok = true;
        if (tid == 0) ok = wait_parity(su32(&mbar), phase);
        if (__syncthreads_or(!ok)) return false;
        phase ^= 1u;
        fence_after();
        return true;
    };

    EJob J;
    first_job(p, MODE, J);
#pragma unroll 1
    while (J.valid) {
        const Seg<double>& Sg = p.seg[J.si];
        const int n = Sg.n;
        {
            // ---------------------------- one exponent per line: given (synthesis
            // pass 1 on the full grid), or the whole line read, 8 lines in flight per warp
            if (MODE == M_UNCOMP && Sg.lexp != nullptr) {
                for (int r = tid; r < M; r += THREADS)
                    rowE[r] = scale_of(r < J.lt ? Sg.lexp[(long long)J.orb * Sg.N + J.a0 + r] : 0);
            } else
#pragma unroll 1
            for (int i = 0; i < RPW; i += 8) {
                int eb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 1
                for (int x = 2 * lane; x < n; x += 64) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int r = warp + WARPS * (i + k);
                        if (r >= J.lt) continue;
                        if (MODE == M_UNCOMP) {
                            eb[k] = max(eb[k], bexp(load_in<MODE>(Sg, J.orb, J.a0 + r, x)));
                            eb[k] = max(eb[k], bexp(load_in<MODE>(Sg, J.orb, J.a0 + r, x + 1)));
                        } else {
                            // n is even: x, x + 1 are in the line and 16-byte aligned
                            const double2 v = *reinterpret_cast<const double2*>(
                                Sg.in + (long long)J.orb * Sg.P + (long long)(J.a0 + r) * n + x);
                            eb[k] = max(eb[k], max(bexp(v.x), bexp(v.y)));
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = (int)__reduce_max_sync(0xffffffffu, (unsigned)eb[k]);
                    if (lane == 0) rowE[warp + WARPS * (i + k)] = scale_of(e);
                }
            }
            __syncthreads();
            // ---------------------------- windows; each slab sliced once
            // slab s covers positions 16 s + P0 .. + 15; window w reads slabs
            // s0(w) .. s0(w) + 2 from slots (slab mod 3)
            constexpr int P0 = (KIND == K_KIN) ? 0 : -8;
            const int nwin = Sg.nwin;
            constexpr int NEW = N / 16;          // new slabs per window after the first
            // raw inputs of one slab for this lane: lines warp * RPW + 4 g + lane / 8,
            // positions 2 (lane % 8), + 1 of the slab
            auto load_slab = [&](int sb, double (&v)[RPW / 4][2]) {
                const int pair = lane & 7;
                int x = (16 * sb + P0 + 2 * pair) % n;
                if (x < 0) x += n;
                int x1 = x + 1;
                if (x1 >= n) x1 -= n;
#pragma unroll
                for (int g4 = 0; g4 < RPW / 4; ++g4) {
                    const int r = warp * RPW + 4 * g4 + (lane >> 3);
                    v[g4][0] = v[g4][1] = 0.0;
                    if (r >= J.lt) continue;
                    if (MODE == M_UNCOMP) {
                        v[g4][0] = load_in<MODE>(Sg, J.orb, J.a0 + r, x);
                        v[g4][1] = load_in<MODE>(Sg, J.orb, J.a0 + r, x1);
                    } else {
                        // x is even and n is even: x1 = x + 1, 16-byte aligned
                        const double2 d2 = *reinterpret_cast<const double2*>(
                            Sg.in + (long long)J.orb * Sg.P + (long long)(J.a0 + r) * n + x);
                        v[g4][0] = d2.x;
                        v[g4][1] = d2.y;
                    }
                }
            };
            auto slice_slab = [&](int sb, const double (&v)[RPW / 4][2]) {
                const int slot = ((sb % NSLOT) + NSLOT) % NSLOT;
                const int pair = lane & 7;
#pragma unroll
                for (int g4 = 0; g4 < RPW / 4; ++g4) {
                    const int r = warp * RPW + 4 * g4 + (lane >> 3);
                    store_pair_digits<LBOA>(Asm, APL, 2 * slot + (pair >> 2), r, pair & 3, v[g4][0],
                                            v[g4][1], rowE[r]);
                }
            };
            double eacc = 0.0;
#pragma unroll 1
            for (int w = 0; w < nwin && !failed; ++w) {
                const int o = w * N;
                const int s0 = (o - HA - P0) / 16;
                if (w == 0) {
                    if constexpr (KIND == K_KIN) {
                        // the kinetic pass's tiles have 5 to 7 windows, so the
                        // first window's three slabs weigh: their loads first
                        // (8.82 -> 8.47 ms per headline step; the 16-tap passes,
                        // with 3 to 4 windows, measured no gain)
                        double v[NSLOT][RPW / 4][2];
#pragma unroll
                        for (int k = 0; k < NSLOT; ++k) load_slab(s0 + k, v[k]);
#pragma unroll
                        for (int k = 0; k < NSLOT; ++k) slice_slab(s0 + k, v[k]);
                    } else {
#pragma unroll 1
                        for (int sb = s0; sb < s0 + NSLOT; ++sb) {
                            double v[RPW / 4][2];
                            load_slab(sb, v);
                            slice_slab(sb, v);
                        }
                    }
                } else {
#pragma unroll 1
                    for (int k = 0; k < NEW; ++k) {
                        double v[RPW / 4][2];
                        load_slab(s0 + NSLOT - NEW + k, v);
                        slice_slab(s0 + NSLOT - NEW + k, v);
                    }
                }
                issue_mmas(((s0 % NSLOT) + NSLOT) % NSLOT);
                double pa[NH], pb[NH], pc[NH];
                prefetch_epilogue<KIND, MODE>(Sg, o + NH * half, er, J.lt, J.a0, J.orb, J.grp, pa,
                                              pb, pc);

                if (!wait_mmas()) {
                    failed = true;
                    break;
                }
                eacc += window_epilogue<KIND, MODE>(Sg, tl, o + NH * half, er, J.lt, J.a0, J.orb,
                                                    J.grp, rowE[er] + Ef - OUT_EXP, pa, pb, pc);
                fence_before();
                __syncthreads();   // accumulators are rewritten by the next window's MMAs
            }
            if (failed) break;
            if (MODE == M_KLAST || (MODE == M_POT && Sg.aux)) {
                const double t = cta_sum(eacc, red);
                if (tid == 0) Sg.part[(long long)J.orb * Sg.tiles + J.tt] = t;
                __syncthreads();
            }
            __syncthreads();   // rowE and the slab ring are reused by the next job
            next_job(p, MODE, J);
        }
    }

    if (failed) {
        // let the MMAs still in flight finish before the accumulators are freed
        if (tid == 0) {
            atomicAdd(&g_emu_timeouts, 1u);
            wait_parity(su32(&mbar), phase);
        }
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tm), "r"(TCOLS));
}

// ------------------------------------------------------------------ host
// The kernel's schedule for a launch's taps (emu.cuh: build_sched).
static bool build_sched(int kind, const PassParams<double>& p, Sched& s) {
    return emu::build_sched(p.f, kind_geom(kind).nt, s);
}

template <int KIND, int MODE>
static cudaError_t ensure_emu_attr() {
    static unsigned long long done = 0;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(__atomic_load_n(&done, __ATOMIC_ACQUIRE) & bit)) {
        err = cudaFuncSetAttribute(emu_pass_kernel<KIND, MODE>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(KIND, MODE));
        if (err != cudaSuccess) return err;
        err = cudaFuncSetAttribute(emu_pass_kernel<KIND, MODE>,
                                   cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared);
        if (err != cudaSuccess) return err;
        __atomic_fetch_or(&done, bit, __ATOMIC_ACQ_REL);
    }
    return cudaSuccess;
}

template <int KIND, int MODE>
static cudaError_t launch_emu(const Params& ep, long long nunits, cudaStream_t st) {
    cudaError_t err = ensure_emu_attr<KIND, MODE>();
    if (err != cudaSuccess) return err;
    if (nunits <= 0) return cudaSuccess;
    int dev = 0, nsm = 0, occ = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return err;
    // CTAs per SM from shared memory, registers and tensor memory (512
    // columns); the occupancy calculator undercounts these kernels
    static int regs[64] = {0};
    if (!regs[dev & 63]) {
        cudaFuncAttributes fa;
        if ((err = cudaFuncGetAttributes(&fa, emu_pass_kernel<KIND, MODE>)) != cudaSuccess) return err;
        regs[dev & 63] = std::max(fa.numRegs, 1);
    }
    int smem_sm = 0;
    if ((err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
        cudaSuccess)
        return err;
    const int per_cta = smem_bytes(KIND, MODE) + 1024 + 1024;   // + static + reserved
    const int by_smem = smem_sm / per_cta;
    const int by_regs = 65536 / (((regs[dev & 63] + 7) / 8 * 8) * THREADS);
    occ = std::min(std::min(by_smem, by_regs), 512 / tmem_cols(KIND));
    if (occ < 1) return cudaErrorInvalidConfiguration;
    long long grid = std::min<long long>((long long)occ * nsm, nunits);
    emu_pass_kernel<KIND, MODE><<<dim3((unsigned)grid), dim3(THREADS), smem_bytes(KIND, MODE), st>>>(ep);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace emu

// One warp per (orbital, i3, i2) row of coarse points reads the row's scaling
// coefficients and 7-component wavelet records as contiguous runs; the
// coefficient c^mu of point (i1, i2, i3) lies on line (x3, x2) = (2 i3 + a3,
// 2 i2 + a2) of the interleaved array, mu = a1 + 2 a2 + 4 a3, so the row
// gives the maxima of four lines.
__global__ void line_exp_kernel(const double* __restrict__ in, int* __restrict__ lexp, int n1,
                                int n2, int n3, long long P, long long nrows) {
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    const long long rows_orb = (long long)n3 * n2;
    const int orb = (int)(row / rows_orb);
    const int rem = (int)(row - orb * rows_orb);
    const int i3 = rem / n2, i2 = rem - i3 * n2;
    const double* cc = in + (long long)orb * P;
    const long long k0 = ((long long)i3 * n2 + i2) * n1;
    const double* cf = cc + P / 8 + 7 * k0;
    int m[4] = {0, 0, 0, 0};   // line (a3, a2) -> m[2 a3 + a2]
    for (int i1 = lane; i1 < n1; i1 += 32) m[0] = max(m[0], emu::bexp(cc[k0 + i1]));
    for (int pos = lane; pos < 7 * n1; pos += 32) {
        const int mu = pos % 7 + 1;
        const int e = emu::bexp(cf[pos]);
        const int l = 2 * (mu >> 2) + ((mu >> 1) & 1);
        m[0] = l == 0 ? max(m[0], e) : m[0];
        m[1] = l == 1 ? max(m[1], e) : m[1];
        m[2] = l == 2 ? max(m[2], e) : m[2];
        m[3] = l == 3 ? max(m[3], e) : m[3];
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) m[l] = (int)__reduce_max_sync(0xffffffffu, (unsigned)m[l]);
    if (lane < 4) {
        const int a3 = lane >> 1, a2 = lane & 1;
        const int N2 = 2 * n2, N3 = 2 * n3;
        const int v = lane == 0 ? m[0] : lane == 1 ? m[1] : lane == 2 ? m[2] : m[3];
        lexp[(long long)orb * N2 * N3 + (long long)(2 * i3 + a3) * N2 + 2 * i2 + a2] = v;
    }
}

cudaError_t launch_line_exp(const double* in, int* lexp, int n1, int n2, int n3, int norb,
                            long long P, cudaStream_t st) {
    const long long nrows = (long long)norb * n3 * n2;
    if (nrows <= 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (nrows * 32 + threads - 1) / threads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    line_exp_kernel<<<(unsigned)blocks, threads, 0, st>>>(in, lexp, n1, n2, n3, P, nrows);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pass_emu(int kind, int mode, const PassParams<double>& p, long long nunits,
                            cudaStream_t st) {
    emu::Params ep;
    std::memset(&ep, 0, sizeof ep);
    ep.p = p;
    if (!emu::build_sched(kind, p, ep.s)) return cudaErrorInvalidValue;
    using namespace emu;
    switch (kind) {
    case K_SYN:
        if (mode == M_UNCOMP) return launch_emu<K_SYN, M_UNCOMP>(ep, nunits, st);
        if (mode == M_PLAIN) return launch_emu<K_SYN, M_PLAIN>(ep, nunits, st);
        break;
    case K_ANA:
        if (mode == M_COMP) return launch_emu<K_ANA, M_COMP>(ep, nunits, st);
        if (mode == M_PLAIN) return launch_emu<K_ANA, M_PLAIN>(ep, nunits, st);
        break;
    case K_MF:
        if (mode == M_POT) return launch_emu<K_MF, M_POT>(ep, nunits, st);
        if (mode == M_PLAIN) return launch_emu<K_MF, M_PLAIN>(ep, nunits, st);
        break;
    case K_MFT:
        if (mode == M_PLAIN) return launch_emu<K_MFT, M_PLAIN>(ep, nunits, st);
        break;
    case K_KIN:
        if (mode == M_KMID) return launch_emu<K_KIN, M_KMID>(ep, nunits, st);
        if (mode == M_KLAST) return launch_emu<K_KIN, M_KLAST>(ep, nunits, st);
        break;
    }
    return cudaErrorInvalidValue;
}

cudaError_t prepare_emu_kernels() {
    using namespace emu;
    cudaError_t e;
    if ((e = ensure_emu_attr<K_SYN, M_UNCOMP>()) != cudaSuccess) return e;
    if ((e = ensure_emu_attr<K_SYN, M_PLAIN>()) != cudaSuccess) return e;
    if ((e = ensure_emu_attr<K_ANA, M_COMP>()) != cudaSuccess) return e;
    if ((e = ensure_emu_attr<K_ANA, M_PLAIN>()) != cudaSuccess) return e;
    if ((e = ensure_emu_attr<K_MF, M_POT>()) != cudaSuccess) return e;
    if ((e = ensure_emu_attr<K_MF, M_PLAIN>()) != cudaSuccess) return e;
    if ((e = ensure_emu_attr<K_MFT, M_PLAIN>()) != cudaSuccess) return e;
    if ((e = ensure_emu_attr<K_KIN, M_KMID>()) != cudaSuccess) return e;
    return ensure_emu_attr<K_KIN, M_KLAST>();
}

namespace emu {
// An mbarrier that nothing arrives on, waited for with a bound of `cycles`:
// the expiry path of the bounded waits, exercised without a fault.
__global__ void wait_probe_kernel(long long cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&bar)), "r"(1));
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(su32(&bar)), "r"(0u) : "memory");
        if (ok) return;
        if (clock64() - t0 > cycles) {
            atomicAdd(&g_emu_timeouts, 1u);
            return;
        }
    }
}
}  // namespace emu

cudaError_t emu_wait_probe(double ms, cudaStream_t st) {
    int dev = 0, khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0)
        khz = 2000000;   // SM clock unknown: assume 2 GHz
    const long long cycles = (long long)(ms * (double)khz);
    emu::wait_probe_kernel<<<1, 32, 0, st>>>(cycles);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t emu_take_timeouts(unsigned* count) {
    unsigned v = 0, z = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_emu_timeouts, sizeof v);
    if (e != cudaSuccess) return e;
    if (v) e = cudaMemcpyToSymbol(g_emu_timeouts, &z, sizeof z);
    *count = v;
    return e;
}

}  // namespace wvl
