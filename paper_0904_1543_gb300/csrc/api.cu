// Host side of the C ABI declared in include/wvl.h: argument validation,
// workspace carving, the order of the 1D passes for each operator (paper
// Sec. "Full local hamiltonian", Sec. "Local density calculation",
// Sec. "Kinetic convolution"), the second-stage reductions, batched plans
// (segments of equal-size cells, CUDA-graph replay, autotuning, tracing).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "wvl.h"
#include "wvl_internal.h"
#include "emu.cuh"

namespace wvl {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

static wvl_status fail(wvl_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}
wvl_status set_error(wvl_status s, const char* msg) { return fail(s, "%s", msg); }
void clear_error() { g_err[0] = 0; }

static wvl_status cuda_fail(cudaError_t e, const char* where) {
    return fail(WVL_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ------------------------------------------------------------------ filters
KindGeom kind_geom(int kind) {
    const int k0 = filters().k0;
    switch (kind) {
    case K_MF:  return {16, 0, 0, 0, k0 + 15, -k0};
    case K_MFT: return {16, 0, 0, 0, -k0, k0 + 15};
    case K_KIN: return {29, 0, 0, 0, 14, 14};
    case K_SYN: return {16, 0, 1, 1, 8, 8};
    case K_ANA: return {16, 1, 0, 1, 8, 8};
    }
    return {0, 0, 0, 0, 0, 0};
}

// Tap t of parity e multiplies the input at position i - hl + off_e + t.
template <typename T>
void fill_taps(PassParams<T>& p, int kind, double hgrid) {
    const FilterSet& F = filters();
    auto H = [&](int j) { return F.h[j + 7]; };   // h_j, j = -7..8
    auto G = [&](int j) { return F.g[j + 7]; };
    for (int e = 0; e < 2; ++e)
        for (int t = 0; t < 32; ++t) p.f[e][t] = T(0);
    for (int t = 0; t < 16; ++t) {
        switch (kind) {
        case K_MF:  // psi_r(I) = sum_k w_k s(I - k), k = k0 + 15 - t
            p.f[0][t] = p.f[1][t] = T(F.w[15 - t]);
            break;
        case K_MFT: // y(J) = sum_k w_k y_r(J + k), k = k0 + t
            p.f[0][t] = p.f[1][t] = T(F.w[t]);
            break;
        case K_SYN: // s_i = sum_j h_{i-2j} c_j + g_{i-2j} d_j (interleaved c, d)
            p.f[0][t] = T((t % 2 == 0) ? H(8 - t) : G(9 - t));
            p.f[1][t] = T((t % 2 == 0) ? H(7 - t) : G(8 - t));
            break;
        case K_ANA: // c_j = sum_i h_{i-2j} s_i, d_j = sum_i g_{i-2j} s_i
            p.f[0][t] = T(H(t - 7));
            p.f[1][t] = T(G(t - 7));
            break;
        }
    }
    if (kind == K_KIN) {
        // out(I) = sum_l T_l s(I - l), T_l = -a_l / (2 h'^2), l = 14 - t
        const double sc = 2.0 * hgrid * hgrid;
        for (int t = 0; t < 29; ++t) p.f[0][t] = p.f[1][t] = T(-F.a[28 - t] / sc);
    }
    p.hl = kind_geom(kind).hl;
}
template void fill_taps<double>(PassParams<double>&, int, double);
template void fill_taps<float>(PassParams<float>&, int, double);

static int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    dev &= 63;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        cached[dev] = v;
    }
    return cached[dev];
}

// ------------------------------------------------------------------ passes
struct Tune {
    int R = 8;
    int LT = 32;
    bool persist = false;   // persistent double-buffered grid vs one CTA per job
};

// FP32 potential pass: compensated density sums in shared memory, one float
// pair per (output, line) of a tile
template <typename T>
static size_t pot_smem(int mode, int LT, int n) {
    return (mode == M_POT && sizeof(T) == 4) ? (size_t)LT * n * 8 : 0;
}

// one staging buffer per CTA unless it prefetches (persistent grid, or the
// orbital walk of the potential pass)
static int nbuf(int mode, const Tune& t) { return (t.persist || mode == M_POT) ? 2 : 1; }

enum Op { OP_HPSI, OP_ENERGY, OP_DENSITY, OP_SYN, OP_ANA, OP_MF, OP_MFT, OP_KIN, OP_HELM };
enum Stage { ST_SYN = 0, ST_MF = 1, ST_MFT = 2, ST_KIN = 3, ST_ANA = 4, ST_RED = 5 };

constexpr int GMAX = 16;   // orbital groups per cell in the potential pass
constexpr int LT_MIN = 4;

static void pass_dims(const int Nf[3], int pass, int& n, int& N) {
    if (pass == 1) { n = Nf[0]; N = Nf[2] * Nf[1]; }
    else if (pass == 2) { n = Nf[1]; N = Nf[0] * Nf[2]; }
    else { n = Nf[2]; N = Nf[1] * Nf[0]; }
}

template <typename T>
struct SegDesc {
    Seg<T> s{};
    int Nf[3] = {0, 0, 0};
    int gn = 0, gN = 0;      // free lines: the pass's output line length and line count
    double hax = 0.0;        // spacing of the pass axis (kinetic)
    double* user_rho = nullptr;
    double* rho_part = nullptr;
    int groups = 1;          // M_POT: groups actually launched
    bool rho_shared = false; // M_POT: write partials even with one group
};

template <typename T>
struct PassCall {
    int kind, mode, pass, stage;
    std::vector<SegDesc<T>> segs;
    bool emu = false;        // FP64 convolutions on the tensor cores (emu.cuh)
};

// shared-memory row length of a staged line, in elements
static int rowlen_of(int n, int R, const KindGeom& g, size_t elt) {
    int nch = (n + R - 1) / R;
    int rl = nch * R + g.hl + g.hr;
    if (elt == 4) {
        // FP32: the left halo is rounded up to 4 words (16-byte staging of the
        // interior), windows are read as 16-byte vectors from the chunk start
        // (past the window by up to 3 words); rows 16-byte aligned, stride
        // = 4 mod 8 words so the 8 lanes of a 16-byte load phase hit
        // distinct banks
        const int hla = (g.hl + 3) / 4 * 4;
        const int w4 = (R + g.nt - 1 + g.extra + (hla - g.hl) + 3) / 4 * 4;
        rl = std::max(nch * R + hla + g.hr, nch * R - R + w4);
        rl = (rl + 3) / 4 * 4;
        if ((rl & 7) == 0) rl += 4;
        return rl;
    }
    if ((rl & 1) == 0) rl += 1;   // odd stride: conflict-free lane-per-line reads
    return rl;
}

template <typename T>
static bool tune_valid(const PassCall<T>& c, const Tune& t) {
    const KindGeom g = kind_geom(c.kind);
    for (const auto& d : c.segs) {
        int n, N;
        pass_dims(d.Nf, c.pass, n, N);
        // the staging buffers (and the FP32 potential pass's density sums) must fit
        if (nbuf(c.mode, t) * ((size_t)t.LT * rowlen_of(n, t.R, g, sizeof(T)) + 2) * sizeof(T) +
                pot_smem<T>(c.mode, t.LT, n) > 200 * 1024)
            return false;
        if (c.mode == M_POT && sizeof(T) == 8) {
            const int nslots = (NTHREADS / 32) * (32 / t.LT);
            const int cpt = pot_out<T>() / t.R;
            if ((long long)cpt * nslots < (n + t.R - 1) / t.R) return false;
        }
    }
    return true;
}

template <typename T>
static long long blocks_of(const PassCall<T>& c, const Tune& t) {
    long long b = 0;
    for (const auto& d : c.segs) {
        int n, N;
        pass_dims(d.Nf, c.pass, n, N);
        const long long units = (c.mode == M_POT) ? std::min(d.s.norb, GMAX) : d.s.norb;
        b += (long long)((N + t.LT - 1) / t.LT) * units;
    }
    return b;
}

// Untuned choice, ordered by what the autotuner measures on GB300: FP64
// 16-tap passes R = 4 on small tiles (LT = 8), FP64 kinetic passes R = 8,
// LT = 16, FP32 passes R = 8, LT = 32; one CTA per job.  A tile size is
// skipped when it leaves fewer than two CTAs per SM.
template <typename T>
static Tune default_tune(const PassCall<T>& c) {
    const long long want = 2LL * num_sms();
    const bool f64 = sizeof(T) == 8;
    const bool kin = c.kind == K_KIN;
    const int R0 = (f64 && !kin) ? 4 : 8;
    static const int pref64[4] = {8, 16, 32, 4}, pref64k[4] = {16, 32, 8, 4},
                     pref32[4] = {32, 16, 8, 4};
    const int* lts = !f64 ? pref32 : (kin ? pref64k : pref64);
    for (int R : {R0, 12 - R0}) {
        Tune fallback;
        bool have = false;
        for (int k = 0; k < 4; ++k) {
            Tune t;
            t.R = R;
            t.LT = lts[k];
            t.persist = false;
            if (!tune_valid(c, t)) continue;
            if (blocks_of(c, t) >= want) return t;
            if (!have) fallback = t;
            have = true;
        }
        if (have) return fallback;
    }
    Tune t;
    t.R = 4;
    t.LT = LT_MIN;
    return t;
}

static cudaError_t launch_emu_t(int kind, int mode, const PassParams<double>& p, long long n,
                               cudaStream_t st) {
    return launch_pass_emu(kind, mode, p, n, st);
}
static cudaError_t launch_emu_t(int, int, const PassParams<float>&, long long, cudaStream_t) {
    return cudaErrorInvalidValue;
}
static cudaError_t launch_line_exp_t(const double* in, int* lexp, int n1, int n2, int n3,
                                     int norb, long long P, cudaStream_t st) {
    return launch_line_exp(in, lexp, n1, n2, n3, norb, P, st);
}
static cudaError_t launch_line_exp_t(const float*, int*, int, int, int, int, long long,
                                     cudaStream_t) {
    return cudaErrorInvalidValue;
}

template <typename T>
static wvl_status exec_call(PassCall<T>& c, const Tune& tn, cudaStream_t st) {
    const KindGeom g = kind_geom(c.kind);
    // the kernels fix the left halos at compile time (magic filter k0 = -7)
    if (kind_geom(K_MF).hl != 8 || kind_geom(K_MFT).hl != 7)
        return fail(WVL_EUNSUPPORTED, "magic filter offset k0 = %d, kernels assume -7", filters().k0);
    const bool emu = c.emu;
    size_t i = 0;
    while (i < c.segs.size()) {
        PassParams<T> p;
        std::memset(&p, 0, sizeof p);
        const double hax = c.segs[i].hax;
        fill_taps(p, c.kind, hax);
        p.LT = emu ? emu::M : tn.LT;
        long long blk = 0;
        size_t smem = 0;
        int nmax = 0;
        int k = 0;
        const size_t first = i;
        for (; i < c.segs.size() && k < MAXSEG; ++i, ++k) {
            SegDesc<T>& d = c.segs[i];
            if (c.kind == K_KIN && i > first && d.hax != hax) break;
            Seg<T>& s = d.s;
            pass_dims(d.Nf, c.pass, s.n, s.N);
            if (d.gn > 0) {
                s.n = d.gn;
                s.N = d.gN;
            }
            if (emu) {
                // units: 128-line tiles (the kernel walks their output windows)
                s.nwin = (s.n + emu::window_n(c.kind) - 1) / emu::window_n(c.kind);
                s.tiles = (s.N + emu::M - 1) / emu::M;
                s.rowlen = 0;
            } else {
                s.nwin = 1;
                s.tiles = (s.N + tn.LT - 1) / tn.LT;
                s.rowlen = rowlen_of(s.n, tn.R, g, sizeof(T));
            }
            long long units = s.norb;
            if (c.mode == M_POT) {
                // orbital groups: enough units to fill the SMs (the FP32 pass
                // is latency-bound and fits more CTAs per SM); each group adds
                // one density partial of P doubles
                const long long want = (sizeof(T) == 4 ? 16LL : 4LL) * num_sms();
                int gmax = s.norb;
                if (d.user_rho) gmax = d.rho_part ? std::min(GMAX, s.norb) : 1;
                long long G = (want + s.tiles - 1) / s.tiles;
                G = std::max(1LL, std::min<long long>(G, gmax));
                s.opg = (int)((s.norb + G - 1) / G);
                G = (s.norb + s.opg - 1) / s.opg;
                d.groups = (int)G;
                units = G;
                if (d.user_rho == nullptr) {
                    s.rho = nullptr;
                    s.rho_gstride = 0;
                } else if (G == 1 && !d.rho_shared) {
                    s.rho = d.user_rho;
                    s.rho_gstride = 0;
                } else {
                    s.rho = d.rho_part;
                    s.rho_gstride = s.vN1 > 0 ? s.vP : s.P;
                }
            }
            if (c.mode == M_POT && s.vN1 > 0 && s.rho != nullptr && s.rho_gstride > 0) {
                // free lines cover part of the grid of rho only: the groups'
                // partials start at zero everywhere, as the reduction adds them all
                cudaError_t e = cudaMemsetAsync(s.rho, 0, (size_t)d.groups * s.vP * sizeof(double), st);
                if (e != cudaSuccess) return cuda_fail(e, "density partials");
            }
            s.blk0 = blk;
            blk += units * s.tiles;
            if (!emu) smem = std::max(smem, (size_t)tn.LT * s.rowlen);
            nmax = std::max(nmax, s.n);
            p.seg[k] = s;
        }
        p.nseg = k;
        p.nunits = blk;
        if (emu) {
            if (c.mode == M_UNCOMP)
                for (int q = 0; q < k; ++q) {
                    const Seg<T>& s = p.seg[q];
                    if (s.lexp == nullptr) continue;
                    cudaError_t e = launch_line_exp_t(s.in, const_cast<int*>(s.lexp), s.n1, s.n2,
                                                      c.segs[first + q].Nf[2] / 2, s.norb, s.P, st);
                    if (e != cudaSuccess) return cuda_fail(e, "line exponent launch");
                }
            cudaError_t e = launch_emu_t(c.kind, c.mode, p, blk, st);
            if (e == cudaErrorInvalidValue)
                return fail(WVL_EUNSUPPORTED, "tensor-core pass: filter digit schedule not supported");
            if (e != cudaSuccess) return cuda_fail(e, "emulated pass launch");
            continue;
        }
        // two staging buffers, each rounded to 16 bytes
        const size_t per16 = 16 / sizeof(T);
        p.bufelems = (int)((smem + per16 - 1) / per16 * per16);
        smem = nbuf(c.mode, tn) * (size_t)p.bufelems * sizeof(T) + pot_smem<T>(c.mode, tn.LT, nmax);
        cudaError_t e = launch_pass<T>(c.kind, c.mode, tn.R, p, blk, smem, st, tn.persist);
        if (e != cudaSuccess) return cuda_fail(e, "pass launch");
    }
    return WVL_OK;
}

// ------------------------------------------------------------------ runs
template <typename T>
struct CellRun {
    int n[3];
    int Nf[3];
    double hg[3];
    int norb;
    long long P;
    const T* in;       // psi_c (or the op's input)
    T* out;            // hpsi_c (or the op's output)
    const T* V;        // potential (OP_HPSI/OP_ENERGY) or K0 (OP_KIN)
    double* rho;
    const double* occ;
    double* ekin;
    double* epot;
    T* buf[4];
    double* epart;
    double* kpart;
    double* rpart;
    const double* eps = nullptr;   // OP_HELM: per-orbital shift
    const double* gscale = nullptr;// OP_HPSI: scale H psi of orbital o by 2 occ[o] gscale[0]
                                   //   in the last pass (the adjoint of E_loc)
    const int* mapc = nullptr;     // localisation region (nullptr: full grid)
    const int* mapf = nullptr;
    long long clen = 0;            // region: compressed length per orbital
    long long ncoarse = 0;         // region: stored scaling coefficients
    int bx[3] = {0, 0, 0};         // free/surface BC: box extents inside the padded cell
    int bo[3] = {0, 0, 0};         // free/surface BC: padding per side along each axis
    bool emu = false;              // FP64 convolutions on the tensor cores (emu.cuh)
    int chain = 0;                 // OP_HPSI: CHAIN_AUTO, CHAIN_PASSES or CHAIN_FUSED
    bool rho_shared = false;       // another run of the same call adds into the same rho:
                                   //   the density goes through the run's partials
    // free boundary conditions computed on supports that grow pass by pass
    // (grow_seg): the box's coarse extents and which axes are free; the cell
    // fields (n, Nf, P) are those of the padded cell that V and rho cover
    bool grow = false;
    int gb[3] = {0, 0, 0};
    bool gfree[3] = {false, false, false};
    int go[3] = {0, 0, 0};         // region runs: the box origin in the cell (coarse)
    int vlo[3] = {0, 0, 0};        // fine coordinate, relative to the box, of V's index 0
};

// Runs that add into one density array must not do so from one launch (their
// read-modify-writes would race): such runs write partials, which the
// reductions (one launch per run, in order) add into rho.
template <typename T>
static void mark_shared_rho(std::vector<CellRun<T>>& runs) {
    for (auto& r : runs) {
        r.rho_shared = false;
        if (!r.rho) continue;
        int uses = 0;
        for (const auto& q : runs) uses += (q.rho == r.rho);
        r.rho_shared = uses > 1;
    }
}

// Which kernels run the local Hamiltonian: the fifteen transposing 1D passes,
// or the five plane/column kernels of fused_kernel.cu (where every cell fits
// them).  CHAIN_AUTO takes the fused chain for FP32 and the passes for FP64
// (bound by the FP64 pipe, where the fused chain saves no arithmetic); a
// plan's autotuner may replace that choice by a measured one.
enum Chain { CHAIN_AUTO = 0, CHAIN_PASSES = 1, CHAIN_FUSED = 2 };

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// partial sums per orbital of the passes that write them (the last axis):
// tiles of LT_MIN lines, or 128-line tiles x 32-output windows when emulated
static long long tiles_max(const int Nf[3]) {
    long long N = (long long)Nf[1] * Nf[0];
    const long long emu_tiles = (N + emu::M - 1) / emu::M * ((Nf[2] + emu::NMIN - 1) / emu::NMIN);
    return std::max((N + LT_MIN - 1) / LT_MIN, emu_tiles);
}

// workspace bytes of one cell run
static size_t run_ws_bytes(const int Nf[3], int norb, size_t elt) {
    const long long P = (long long)Nf[0] * Nf[1] * Nf[2];
    size_t b = 4 * align256((size_t)norb * P * elt);
    b += 2 * align256((size_t)norb * tiles_max(Nf) * sizeof(double));
    b += align256((size_t)std::min(GMAX, std::max(norb, 1)) * P * sizeof(double));
    return b;
}

template <typename T>
static void carve(CellRun<T>& r, char* ws) {
    const size_t fb = align256((size_t)r.norb * r.P * sizeof(T));
    for (int k = 0; k < 4; ++k) r.buf[k] = reinterpret_cast<T*>(ws + k * fb);
    char* q = ws + 4 * fb;
    const size_t pb = align256((size_t)r.norb * tiles_max(r.Nf) * sizeof(double));
    r.epart = reinterpret_cast<double*>(q);
    r.kpart = reinterpret_cast<double*>(q + pb);
    r.rpart = reinterpret_cast<double*>(q + 2 * pb);
}

template <typename T>
static SegDesc<T> seg_for(const CellRun<T>& c, const T* in, T* out) {
    SegDesc<T> d;
    d.s.in = in;
    d.s.out = out;
    d.s.P = c.P;
    d.s.N1 = c.Nf[0];
    d.s.N2 = c.Nf[1];
    d.s.n1 = c.n[0];
    d.s.n2 = c.n[1];
    d.s.norb = c.norb;
    d.s.opg = 1;
    // compressed form: full grid unless a localisation region or the box of
    // free boundary conditions is given
    const bool reg = c.mapc != nullptr || c.bx[0] > 0;
    d.s.mapc = c.mapc;
    d.s.mapf = c.mapf;
    d.s.clen = reg ? c.clen : c.P;
    d.s.ncoarse = reg ? c.ncoarse : c.P / 8;
    d.s.bx1 = c.bx[0];
    d.s.bx2 = c.bx[1];
    d.s.bx3 = c.bx[2];
    d.s.bo1 = c.bo[0];
    d.s.bo2 = c.bo[1];
    d.s.bo3 = c.bo[2];
    for (int k = 0; k < 3; ++k) d.Nf[k] = c.Nf[k];
    return d;
}

// Free boundary conditions on growing supports.  Along a free axis with b
// box coarse points (fine [0, 2b)) each array of the chain is nonzero, or
// needed, only on a fine interval [lo, lo + len):
//   C   the box's coefficients (interleaved coarse layout)   [0, 2b)
//   S   s = synthesis, and y, the kinetic terms K_p and z  [-8, 2b + 8)
//       (h_j, j = -7..8, moves coarse point j to fine 2j - 7 .. 2j + 8, so s
//       is nonzero on [-7, 2b + 6]; the analysis of outputs on the box reads
//       that interval back; the interval starts on an even point because
//       the synthesis and analysis taps follow the parity of the fine point)
//   PSI psi_r = MF s and V psi_r                          [-14, 2b + 15)
//       (magic filter taps k = -7..8 widen [-7, 2b + 6] by 7 / 8; the
//       transposed filter maps this interval back onto S)
//   BOX the analysis output, the box                      [0, 2b)
// so each 1D pass reads a line of the source interval, zero outside it
// (free lines), and writes the target interval.  Periodic axes keep the
// whole periodic line [0, 2b) at every stage.  V and rho live on the cell
// padded by WVL_FREE_PAD coarse points per side along the free axes.
enum GrowDom { GD_C = 0, GD_S = 1, GD_PSI = 2, GD_BOX = 3 };
static void grow_dom(int dom, int b, bool fr, int& lo, int& len) {
    if (!fr || dom == GD_C || dom == GD_BOX) { lo = 0; len = 2 * b; return; }
    if (dom == GD_S) { lo = -8; len = 2 * b + 16; return; }
    lo = -14;
    len = 2 * b + 29;
}

template <typename T>
static void grow_seg(SegDesc<T>& d, const CellRun<T>& r, int kind, int mode, int pass) {
    int from = GD_S, to = GD_S;
    switch (kind) {
    case K_SYN: from = GD_C; to = GD_S; break;
    case K_MF: from = GD_S; to = GD_PSI; break;
    case K_MFT: from = GD_PSI; to = GD_S; break;
    case K_KIN: from = GD_S; to = GD_S; break;
    case K_ANA: from = GD_S; to = GD_BOX; break;
    }
    int flo[3], flen[3], tlo[3], tlen[3];
    for (int a = 0; a < 3; ++a) {
        grow_dom(from, r.gb[a], r.gfree[a], flo[a], flen[a]);
        grow_dom(to, r.gb[a], r.gfree[a], tlo[a], tlen[a]);
    }
    // pass 1 runs along x over the source extents, pass 2 along y with x
    // already at the target, pass 3 along z with x and y at the target
    const int ax = pass - 1;
    int N;
    if (pass == 1) N = flen[2] * flen[1];
    else if (pass == 2) N = tlen[0] * flen[2];
    else N = tlen[1] * tlen[0];
    Seg<T>& s = d.s;
    d.gn = tlen[ax];
    d.gN = N;
    s.P = (long long)tlen[ax] * N;
    s.Pin = (long long)flen[ax] * N;
    if (r.gfree[ax]) {
        s.nin = flen[ax];
        s.inoff = tlo[ax] - flo[ax];
    }
    // index decoding of the modes that need it: M_UNCOMP lines (x3, x2) of
    // the box, M_COMP / M_POT outputs (X1, X2) in pass 3
    s.N2 = flen[1];
    s.N1 = tlen[0];
    s.n1 = r.gb[0];
    s.n2 = r.gb[1];
    s.bx1 = s.bx2 = s.bx3 = 0;
    s.bo1 = s.bo2 = s.bo3 = 0;
    if (r.mapc != nullptr) {
        // a region's box inside the periodic cell: index lookups in the cell
        s.go1 = r.go[0];
        s.go2 = r.go[1];
        s.go3 = r.go[2];
        s.gc1 = r.n[0];
        s.gc2 = r.n[1];
        s.gc3 = r.n[2];
    } else {
        s.ncoarse = (long long)r.gb[0] * r.gb[1] * r.gb[2];
        s.clen = 8 * s.ncoarse;
    }
    if (mode == M_POT) {
        // V and rho on the cell (region) or the padded cell (free conditions),
        // whose index 0 sits at fine coordinate vlo of the box
        s.vN1 = r.Nf[0];
        s.vN2 = r.Nf[1];
        s.vN3 = r.Nf[2];
        s.vP = r.P;
        int vo[3];
        for (int a = 0; a < 3; ++a) vo[a] = ((tlo[a] - r.vlo[a]) % r.Nf[a] + r.Nf[a]) % r.Nf[a];
        s.vo1 = vo[0];
        s.vo2 = vo[1];
        s.vo3 = vo[2];
    }
}

template <typename T>
static std::vector<PassCall<T>> build_calls(int op, std::vector<CellRun<T>>& runs) {
    std::vector<PassCall<T>> calls;
    auto add = [&](int kind, int mode, int pass, int stage, auto&& make) {
        PassCall<T> c{kind, mode, pass, stage, {}};
        c.emu = !runs.empty() && runs.front().emu;
        for (auto& r : runs) {
            SegDesc<T> d = make(r);
            if (r.grow) grow_seg(d, r, kind, mode, pass);
            c.segs.push_back(d);
        }
        calls.push_back(std::move(c));
    };
    auto B = [](CellRun<T>& r, int k) { return r.buf[k]; };
    const int A_ = 0, B_ = 1, C_ = 2, D_ = 3;

    auto synthesis = [&](bool to_user) {
        add(K_SYN, M_UNCOMP, 1, ST_SYN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for(r, r.in, B(r, A_));
            // the tensor-core pass takes its line exponents from a coalesced
            // read of the compressed form (into buffer C, free until the
            // kinetic or density passes)
            if (r.emu && r.mapc == nullptr && r.bx[0] == 0)
                d.s.lexp = reinterpret_cast<const int*>(B(r, C_));
            return d;
        });
        add(K_SYN, M_PLAIN, 2, ST_SYN, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), B(r, B_)); });
        add(K_SYN, M_PLAIN, 3, ST_SYN, [&](CellRun<T>& r) {
            return seg_for<T>(r, B(r, B_), to_user ? r.out : B(r, D_));
        });
    };
    auto mf_pot = [&](bool with_v, bool write_y) {
        add(K_MF, M_PLAIN, 1, ST_MF, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, D_), B(r, A_)); });
        add(K_MF, M_PLAIN, 2, ST_MF, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), B(r, B_)); });
        add(K_MF, M_POT, 3, ST_MF, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, B_), write_y ? B(r, A_) : nullptr);
            d.s.aux = with_v ? r.V : nullptr;
            d.s.occ = r.occ;
            d.s.part = r.epart;
            d.user_rho = r.rho;
            d.rho_part = r.rpart;
            d.rho_shared = r.rho_shared;
            return d;
        });
    };

    switch (op) {
    case OP_SYN:
        synthesis(true);
        break;
    case OP_HELM:
        // A c = S^T (K s - eps s), s = S c: the kinetic passes with K_0 = -eps s
        // (Eq. kinetic1d), between synthesis and analysis
        synthesis(false);                      // s -> D
        add(K_KIN, M_KMID, 1, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, D_), B(r, A_));
            d.s.eps = r.eps;
            d.s.out2 = B(r, C_);
            d.hax = r.hg[0];
            return d;
        });
        add(K_KIN, M_KMID, 2, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, C_), B(r, B_));
            d.s.in2 = B(r, A_);
            d.s.out2 = B(r, D_);
            d.hax = r.hg[1];
            return d;
        });
        add(K_KIN, M_KLAST, 3, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, D_), B(r, A_));
            d.s.in2 = B(r, B_);
            d.s.part = r.kpart;
            d.hax = r.hg[2];
            return d;
        });
        add(K_ANA, M_PLAIN, 1, ST_ANA, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), B(r, B_)); });
        add(K_ANA, M_PLAIN, 2, ST_ANA, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, B_), B(r, A_)); });
        add(K_ANA, M_COMP, 3, ST_ANA, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), r.out); });
        break;
    case OP_ANA:
        add(K_ANA, M_PLAIN, 1, ST_ANA, [&](CellRun<T>& r) { return seg_for(r, r.in, B(r, A_)); });
        add(K_ANA, M_PLAIN, 2, ST_ANA, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), B(r, B_)); });
        add(K_ANA, M_COMP, 3, ST_ANA, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, B_), r.out); });
        break;
    case OP_MF:
    case OP_MFT: {
        const int kd = (op == OP_MF) ? K_MF : K_MFT;
        const int st = (op == OP_MF) ? ST_MF : ST_MFT;
        add(kd, M_PLAIN, 1, st, [&](CellRun<T>& r) { return seg_for(r, r.in, B(r, A_)); });
        add(kd, M_PLAIN, 2, st, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), B(r, B_)); });
        add(kd, M_PLAIN, 3, st, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, B_), r.out); });
        break;
    }
    case OP_KIN: {
        // K_1 = T_x s + K0 -> A, G_1 = s^T -> B; K_2 -> C, G_2 -> D; K_3 -> out
        add(K_KIN, M_KMID, 1, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for(r, r.in, B(r, A_));
            d.s.in2 = r.V;
            d.s.out2 = B(r, B_);
            d.hax = r.hg[0];
            return d;
        });
        add(K_KIN, M_KMID, 2, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, B_), B(r, C_));
            d.s.in2 = B(r, A_);
            d.s.out2 = B(r, D_);
            d.hax = r.hg[1];
            return d;
        });
        add(K_KIN, M_KLAST, 3, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, D_), r.out);
            d.s.in2 = B(r, C_);
            d.s.aux = r.V;
            d.s.part = r.kpart;
            d.hax = r.hg[2];
            return d;
        });
        break;
    }
    case OP_DENSITY:
        synthesis(false);
        mf_pot(false, false);
        break;
    case OP_ENERGY:
        synthesis(false);
        mf_pot(true, false);
        // kinetic with K0 = 0 on s (D): K_1 -> A, G_1 -> C, K_2 -> B, G_2 -> D
        add(K_KIN, M_KMID, 1, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, D_), B(r, A_));
            d.s.out2 = B(r, C_);
            d.hax = r.hg[0];
            return d;
        });
        add(K_KIN, M_KMID, 2, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, C_), B(r, B_));
            d.s.in2 = B(r, A_);
            d.s.out2 = B(r, D_);
            d.hax = r.hg[1];
            return d;
        });
        add(K_KIN, M_KLAST, 3, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, D_), nullptr);
            d.s.in2 = B(r, B_);
            d.s.part = r.kpart;
            d.hax = r.hg[2];
            return d;
        });
        break;
    case OP_HPSI:
        synthesis(false);                      // s -> D
        mf_pot(true, true);                    // V psi_r -> A
        add(K_MFT, M_PLAIN, 1, ST_MFT, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), B(r, B_)); });
        add(K_MFT, M_PLAIN, 2, ST_MFT, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, B_), B(r, A_)); });
        add(K_MFT, M_PLAIN, 3, ST_MFT, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), B(r, B_)); });
        // kinetic on s (D) with K_0 = y (B), Eq. (kinetic1d) with K_0 != 0
        add(K_KIN, M_KMID, 1, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, D_), B(r, A_));
            d.s.in2 = B(r, B_);
            d.s.out2 = B(r, C_);
            d.hax = r.hg[0];
            return d;
        });
        add(K_KIN, M_KMID, 2, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, C_), B(r, B_));
            d.s.in2 = B(r, A_);
            d.s.out2 = B(r, D_);
            d.hax = r.hg[1];
            return d;
        });
        // K_3 = z -> A; partials of <s, K_3> = Ekin + Epot
        add(K_KIN, M_KLAST, 3, ST_KIN, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, D_), B(r, A_));
            d.s.in2 = B(r, B_);
            d.s.part = r.kpart;
            d.hax = r.hg[2];
            return d;
        });
        add(K_ANA, M_PLAIN, 1, ST_ANA, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, A_), B(r, B_)); });
        add(K_ANA, M_PLAIN, 2, ST_ANA, [&](CellRun<T>& r) { return seg_for<T>(r, B(r, B_), B(r, A_)); });
        add(K_ANA, M_COMP, 3, ST_ANA, [&](CellRun<T>& r) {
            SegDesc<T> d = seg_for<T>(r, B(r, A_), r.out);
            d.s.occ = r.occ;
            d.s.gscale = r.gscale;
            return d;
        });
        break;
    }
    return calls;
}

template <typename T>
static wvl_status exec_reductions(int op, std::vector<CellRun<T>>& runs,
                                  std::vector<PassCall<T>>& calls, cudaStream_t st) {
    const PassCall<T>* pot = nullptr;
    const PassCall<T>* kl = nullptr;
    for (auto& c : calls) {
        if (c.mode == M_POT) pot = &c;
        if (c.mode == M_KLAST) kl = &c;
    }
    // the energy sums of every cell in as few launches as the task table allows
    PartTasks tasks;
    auto add_task = [&](const double* part, int tiles, const double* mpart, int mtiles, double* out,
                        int norb) -> cudaError_t {
        if (!tasks.add(part, tiles, mpart, mtiles, out, norb)) {
            cudaError_t e = launch_reduce_parts_multi(tasks, st);
            if (e != cudaSuccess) return e;
            tasks = PartTasks();
            tasks.add(part, tiles, mpart, mtiles, out, norb);
        }
        return cudaSuccess;
    };
    for (size_t i = 0; i < runs.size(); ++i) {
        CellRun<T>& r = runs[i];
        cudaError_t e = cudaSuccess;
        if (pot) {
            const SegDesc<T>& d = pot->segs[i];
            if (r.rho && (d.groups > 1 || d.rho_shared)) {
                e = launch_rho_reduce(r.rpart, r.P, d.groups, r.rho, st);
                if (e != cudaSuccess) return cuda_fail(e, "density reduction");
            }
            if ((op == OP_HPSI || op == OP_ENERGY) && r.epot) {
                e = add_task(r.epart, d.s.tiles, nullptr, 0, r.epot, r.norb);
                if (e != cudaSuccess) return cuda_fail(e, "energy reduction");
            }
        }
        if (kl && r.ekin) {
            const SegDesc<T>& d = kl->segs[i];
            // OP_HPSI accumulates <s, z> = Ekin + Epot; subtract Epot, formed
            // again from its partials in the order of its own reduction
            const bool sub = op == OP_HPSI && pot != nullptr;
            e = add_task(r.kpart, d.s.tiles, sub ? r.epart : nullptr, sub ? pot->segs[i].s.tiles : 0,
                         r.ekin, r.norb);
            if (e != cudaSuccess) return cuda_fail(e, "energy reduction");
        }
    }
    cudaError_t e = launch_reduce_parts_multi(tasks, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy reduction");
    return WVL_OK;
}

// --------------------------------------------------------------- tracing
struct Prof {
    bool on = false;
    std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> pool;
    double ms[WVL_NSTAGE] = {0};
    int cnt[WVL_NSTAGE] = {0};

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void flush() {
        for (auto& t : pending) {
            float v = 0.f;
            cudaEventSynchronize(std::get<2>(t));
            if (cudaEventElapsedTime(&v, std::get<1>(t), std::get<2>(t)) == cudaSuccess) {
                ms[std::get<0>(t)] += v;
                cnt[std::get<0>(t)] += 1;
            }
            pool.push_back(std::get<1>(t));
            pool.push_back(std::get<2>(t));
        }
        pending.clear();
    }
    ~Prof() {
        for (auto& t : pending) {
            cudaEventDestroy(std::get<1>(t));
            cudaEventDestroy(std::get<2>(t));
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// ----------------------------------------------------------- fused chain
// every fine extent a multiple of 8 in [FZ_MIN_FINE, FZ_MAX_FINE], periodic
// full-grid cells, the planes within the shared memory of one CTA
static constexpr size_t FZ_SMEM_MAX = 224 * 1024;
template <typename T>
static bool fused_cell_ok(const int Nf[3]) {
    for (int d = 0; d < 3; ++d)
        if (Nf[d] % 8 != 0 || Nf[d] < FZ_MIN_FINE || Nf[d] > FZ_MAX_FINE) return false;
    for (int prog = 0; prog < FZ_NPROG; ++prog)
        if (fz_smem<T>(prog, Nf[0], Nf[1], Nf[2]) > FZ_SMEM_MAX) return false;
    return true;
}
template <typename T>
static bool fused_ok(const std::vector<CellRun<T>>& runs) {
    if (runs.empty()) return false;
    for (const auto& r : runs)
        if (r.emu || r.mapc != nullptr || r.bx[0] > 0 || r.grow || !fused_cell_ok<T>(r.Nf))
            return false;
    return true;
}

struct StageClock {
    Prof* prof;
    cudaStream_t st;
    int cur = -1;
    cudaEvent_t ev0 = nullptr;
    void begin(int stg) {
        if (!prof || !prof->on || stg == cur) return;
        end();
        cur = stg;
        ev0 = prof->get();
        cudaEventRecord(ev0, st);
    }
    void end() {
        if (!prof || !prof->on || cur < 0) return;
        cudaEvent_t e1 = prof->get();
        cudaEventRecord(e1, st);
        prof->pending.emplace_back(cur, ev0, e1);
        cur = -1;
    }
};

// The local Hamiltonian by the five kernels of fused_kernel.cu.  Buffers of a
// run: A = buf[0] .. D = buf[3]:  SYN3 c -> a A;  SKM12 A -> v C, t D;
// POT3 D -> x B;  MFTA12 B (+ C) -> w' D;  TA3 D (+ A) -> H psi.
// Ekin partials: [norb][N3 (SKM12) + N2/2 ncb (TA3)]; Epot: [norb][N2 ncb].
// Profiling stages: synthesis = SYN3 + SKM12 (which also applies T_1, T_2 and
// MF_1, MF_2), magic filter + potential = POT3 (MF_3, V, rho, MFT_3),
// transposed magic filter = MFTA12 (MFT_1, MFT_2 and the analysis A_1, A_2),
// kinetic = TA3 (T_3, A_3, compression); the analysis stage stays empty.
// OP_ENERGY runs SYN3, SKM12 without v, POT3 without x and TA3 for <a, T_3 a>
// alone; OP_DENSITY runs SYN3, SKM12 (t only) and POT3 (rho only).
template <typename T>
static wvl_status run_fused(int op, std::vector<CellRun<T>>& runs, Prof* prof, cudaStream_t st) {
    static const int kStage[FZ_NPROG] = {ST_SYN, ST_SYN, ST_MF, ST_MFT, ST_KIN};
    StageClock clk{prof, st};
    constexpr int LTC = fz_ltc<T>();
    auto taps = [](int kind, double h, T (&dst)[2][32]) {
        PassParams<T> tp;
        std::memset(&tp, 0, sizeof tp);
        fill_taps(tp, kind, h);
        std::memcpy(dst, tp.f, sizeof dst);
    };
    std::vector<int> groups(runs.size(), 1);
    const bool hpsi = op == OP_HPSI, energy = op != OP_DENSITY;
    for (int prog = 0; prog < FZ_NPROG; ++prog) {
        if (!hpsi && prog == FZ_MFTA12) continue;
        if (!energy && prog == FZ_TA3) continue;
        clk.begin(kStage[prog]);
        size_t i = 0;
        while (i < runs.size()) {
            FzParams<T> p;
            std::memset(&p, 0, sizeof p);
            const CellRun<T>& r0 = runs[i];
            switch (prog) {
            case FZ_SYN3: taps(K_SYN, 0.0, p.tap[0]); break;
            case FZ_SKM12:
                taps(K_SYN, 0.0, p.tap[0]);
                taps(K_KIN, r0.hg[0], p.tap[1]);
                taps(K_KIN, r0.hg[1], p.tap[2]);
                taps(K_MF, 0.0, p.tap[3]);
                break;
            case FZ_POT3: taps(K_MF, 0.0, p.tap[0]); taps(K_MFT, 0.0, p.tap[1]); break;
            case FZ_MFTA12: taps(K_MFT, 0.0, p.tap[0]); taps(K_ANA, 0.0, p.tap[1]); break;
            case FZ_TA3: taps(K_KIN, r0.hg[2], p.tap[0]); taps(K_ANA, 0.0, p.tap[1]); break;
            }
            long long jobs = 0;
            size_t smem = 0;
            int k = 0;
            for (; i < runs.size() && k < MAXSEG; ++i, ++k) {
                CellRun<T>& r = runs[i];
                // the kinetic taps are per launch: one axis spacing per launch
                if (k > 0 && (r.hg[0] != r0.hg[0] || r.hg[1] != r0.hg[1] || r.hg[2] != r0.hg[2]))
                    break;
                FzSeg<T>& s = p.seg[k];
                s.P = r.P;
                s.N1 = r.Nf[0];
                s.N2 = r.Nf[1];
                s.N3 = r.Nf[2];
                s.n1 = r.n[0];
                s.n2 = r.n[1];
                s.norb = r.norb;
                s.opg = 1;
                s.ncb = (s.N1 + LTC - 1) / LTC;
                const int ctiles = s.N2 * s.ncb;
                const int ktiles = s.N3 + (s.N2 / 2) * s.ncb;   // Ekin partials per orbital
                const bool plane = prog == FZ_SKM12 || prog == FZ_MFTA12;
                s.RS = plane ? fz_plane_rs<T>(s.N1) : LTC;
                long long units = r.norb;
                T* const A = r.buf[0];
                T* const B = r.buf[1];
                T* const C = r.buf[2];
                T* const D = r.buf[3];
                switch (prog) {
                case FZ_SYN3: {
                    s.in = r.in; s.out = A;
                    // orbital groups of about four jobs per SM: each job walks
                    // its group on one tile, the next orbital's gather under
                    // this one's filter
                    long long G = (4LL * num_sms() + ctiles - 1) / ctiles;
                    G = std::max(1LL, std::min<long long>(G, std::max(r.norb, 1)));
                    s.opg = (int)((r.norb + G - 1) / G);
                    units = (r.norb + s.opg - 1) / s.opg;
                    break;
                }
                case FZ_SKM12:
                    s.in = A; s.out2 = hpsi ? C : nullptr; s.out3 = D;
                    s.part = energy ? r.kpart : nullptr; s.ptiles = ktiles; s.poff = 0;
                    break;
                case FZ_POT3: {
                    s.in = D; s.out = hpsi ? B : nullptr; s.V = energy ? r.V : nullptr;
                    s.occ = r.occ;
                    s.part = energy ? r.epart : nullptr; s.ptiles = ctiles; s.poff = 0;
                    // orbital groups, each adding one density partial of P doubles;
                    // about 4 jobs per SM: longer jobs amortise the potential tile
                    // and the density flush, and fewer partials cut the reduction
                    // (FP32 headline step 3.30 -> 3.25 ms against 16 jobs per SM)
                    const long long want = 4LL * num_sms();
                    const int gmax = r.rho ? std::min(GMAX, r.norb) : r.norb;
                    long long G = (want + ctiles - 1) / ctiles;
                    G = std::max(1LL, std::min<long long>(G, std::max(gmax, 1)));
                    s.opg = (int)((r.norb + G - 1) / G);
                    G = (r.norb + s.opg - 1) / s.opg;
                    groups[i] = (int)G;
                    units = G;
                    if (r.rho == nullptr) {
                        s.rho = nullptr;
                    } else if (G == 1 && !r.rho_shared) {
                        s.rho = r.rho;
                        s.rho_gstride = 0;
                    } else {
                        s.rho = r.rpart;
                        s.rho_gstride = r.P;
                    }
                    break;
                }
                case FZ_MFTA12: s.in = B; s.in2 = C; s.out = D; break;
                case FZ_TA3:
                    s.in = hpsi ? D : nullptr; s.in2 = A; s.out = hpsi ? r.out : nullptr;
                    s.part = r.kpart; s.ptiles = ktiles; s.poff = s.N3;
                    s.occ = r.occ; s.gscale = hpsi ? r.gscale : nullptr;
                    break;
                }
                s.blk0 = jobs;
                jobs += units * (plane ? s.N3 : prog == FZ_TA3 ? ctiles / 2 : ctiles);
                smem = std::max(smem, fz_smem<T>(prog, s.N1, s.N2, s.N3));
            }
            p.nseg = k;
            p.njobs = jobs;
            cudaError_t e = launch_fused<T>(prog, p, smem, st);
            if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
        }
    }
    clk.begin(ST_RED);
    // the energy sums of every cell in as few launches as the task table allows
    PartTasks tasks;
    auto add_task = [&](const double* part, int tiles, const double* mpart, int mtiles, double* out,
                        int norb) -> cudaError_t {
        if (!tasks.add(part, tiles, mpart, mtiles, out, norb)) {
            cudaError_t e = launch_reduce_parts_multi(tasks, st);
            if (e != cudaSuccess) return e;
            tasks = PartTasks();
            tasks.add(part, tiles, mpart, mtiles, out, norb);
        }
        return cudaSuccess;
    };
    for (size_t i = 0; i < runs.size(); ++i) {
        CellRun<T>& r = runs[i];
        const int ctiles = r.Nf[1] * ((r.Nf[0] + LTC - 1) / LTC);
        cudaError_t e = cudaSuccess;
        if (r.rho && (groups[i] > 1 || r.rho_shared)) {
            e = launch_rho_reduce(r.rpart, r.P, groups[i], r.rho, st);
            if (e != cudaSuccess) return cuda_fail(e, "density reduction");
        }
        if (r.epot && energy) {
            e = add_task(r.epart, ctiles, nullptr, 0, r.epot, r.norb);
            if (e != cudaSuccess) return cuda_fail(e, "energy reduction");
        }
        if (r.ekin && energy) {
            e = add_task(r.kpart, r.Nf[2] + ctiles / 2, nullptr, 0, r.ekin, r.norb);
            if (e != cudaSuccess) return cuda_fail(e, "energy reduction");
        }
    }
    {
        cudaError_t e = launch_reduce_parts_multi(tasks, st);
        if (e != cudaSuccess) return cuda_fail(e, "energy reduction");
    }
    clk.end();
    return WVL_OK;
}

using TuneTable = std::map<int, Tune>;
static int tune_key(int kind, int mode, int pass) { return kind * 100 + mode * 10 + pass; }

template <typename T>
static wvl_status run_op(int op, std::vector<CellRun<T>>& runs, const TuneTable* tt,
                         Prof* prof, cudaStream_t st) {
    mark_shared_rho(runs);
    if ((op == OP_HPSI || op == OP_ENERGY || op == OP_DENSITY) && !runs.empty()) {
        const int ch = runs.front().chain;
        const bool ok = fused_ok(runs);
        if (ch == CHAIN_FUSED && !ok)
            return fail(WVL_EUNSUPPORTED, "fused chain: every fine extent must be a multiple of 8 "
                        "in [%d, %d] on a periodic full-grid cell, in FP64 or FP32",
                        FZ_MIN_FINE, FZ_MAX_FINE);
        if (ok && (ch == CHAIN_FUSED || (ch == CHAIN_AUTO && sizeof(T) == 4)))
            return run_fused<T>(op, runs, prof, st);
    }
    std::vector<PassCall<T>> calls = build_calls<T>(op, runs);
    int cur_stage = -1;
    cudaEvent_t ev0 = nullptr;
    auto stage_begin = [&](int stg) {
        if (!prof || !prof->on || stg == cur_stage) return;
        if (cur_stage >= 0) {
            cudaEvent_t e1 = prof->get();
            cudaEventRecord(e1, st);
            prof->pending.emplace_back(cur_stage, ev0, e1);
        }
        cur_stage = stg;
        ev0 = prof->get();
        cudaEventRecord(ev0, st);
    };
    for (auto& c : calls) {
        stage_begin(c.stage);
        Tune t = default_tune(c);
        if (tt) {
            auto it = tt->find(tune_key(c.kind, c.mode, c.pass));
            if (it != tt->end() && tune_valid(c, it->second)) t = it->second;
        }
        wvl_status s = exec_call(c, t, st);
        if (s != WVL_OK) return s;
    }
    stage_begin(ST_RED);
    wvl_status s = exec_reductions(op, runs, calls, st);
    if (prof && prof->on && cur_stage >= 0) {
        cudaEvent_t e1 = prof->get();
        cudaEventRecord(e1, st);
        prof->pending.emplace_back(cur_stage, ev0, e1);
    }
    return s;
}

// ------------------------------------------------------------ validation
static wvl_status check_prec(int prec) {
    if (prec != WVL_F64 && prec != WVL_F32 && prec != WVL_F64_EMU)
        return fail(WVL_EINVAL, "prec must be WVL_F64, WVL_F32 or WVL_F64_EMU");
    return WVL_OK;
}
static wvl_status check_grid(const wvl_grid* g) {
    if (!g) return fail(WVL_EINVAL, "grid is NULL");
    const int n[3] = {g->n1, g->n2, g->n3};
    const double h[3] = {g->h1, g->h2, g->h3};
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 1) return fail(WVL_EINVAL, "grid extent n%d = %d < 1", d + 1, n[d]);
        if (2LL * n[d] > MAX_FINE)
            return fail(WVL_EUNSUPPORTED, "fine extent 2*n%d = %lld exceeds %d", d + 1,
                        2LL * n[d], MAX_FINE);
        if (!(h[d] > 0.0) || !std::isfinite(h[d]))
            return fail(WVL_EINVAL, "fine spacing h%d must be positive and finite", d + 1);
    }
    const long long P = 8LL * n[0] * n[1] * n[2];
    if (P > (1LL << 40)) return fail(WVL_EUNSUPPORTED, "grid too large");
    return WVL_OK;
}
static wvl_status check_ptr(const void* p, const char* name, bool required) {
    if (!p) return required ? fail(WVL_EINVAL, "%s is NULL", name) : WVL_OK;
    if (reinterpret_cast<uintptr_t>(p) & 15) return fail(WVL_EINVAL, "%s is not 16-byte aligned", name);
    return WVL_OK;
}

#define WVL_TRY(x)                          \
    do {                                    \
        wvl_status _s = (x);                \
        if (_s != WVL_OK) return _s;        \
    } while (0)

static void grid_dims(const wvl_grid* g, int n[3], int Nf[3], double hg[3], long long& P) {
    n[0] = g->n1; n[1] = g->n2; n[2] = g->n3;
    hg[0] = g->h1; hg[1] = g->h2; hg[2] = g->h3;
    for (int d = 0; d < 3; ++d) Nf[d] = 2 * n[d];
    P = (long long)Nf[0] * Nf[1] * Nf[2];
}

template <typename T>
static wvl_status single_cell(int op, const wvl_grid* grid, int norb, const void* in,
                              void* out, const void* V, const double* occ, double* rho,
                              double* ekin, double* epot, void* ws, size_t ws_bytes,
                              void* stream, const wvl_region* reg, bool emu,
                              const double* gscale = nullptr) {
    CellRun<T> r;
    grid_dims(grid, r.n, r.Nf, r.hg, r.P);
    r.norb = norb;
    r.emu = emu;
    if (reg) {
        r.mapc = reg->coarse_index;
        r.mapf = reg->fine_index;
        r.ncoarse = reg->ncoarse;
        r.clen = reg->ncoarse + 7 * reg->nfine;
        // a region whose periodic bounding box leaves at least 15 coarse
        // points to the cell along an axis is computed on that box along it
        // (free lines, grow_seg): H couples coarse points at most 15 apart,
        // so no periodic image of the box reaches it and the periodic
        // operator restricted to the region is the box's free-space one
        bool any = false;
        int box[3], lo[3];
        for (int d = 0; d < 3; ++d) {
            const bool fr = reg->len[d] > 0 && reg->len[d] <= r.n[d] - 15 && !emu;
            box[d] = fr ? reg->len[d] : r.n[d];
            lo[d] = fr ? reg->lo[d] : 0;
            any = any || fr;
            r.gfree[d] = fr;
        }
        if (any) {
            r.grow = true;
            for (int d = 0; d < 3; ++d) {
                r.gb[d] = box[d];
                r.go[d] = lo[d];
                r.vlo[d] = -2 * lo[d];
            }
        }
    }
    r.in = static_cast<const T*>(in);
    r.out = static_cast<T*>(out);
    r.V = static_cast<const T*>(V);
    r.rho = rho;
    r.occ = occ;
    r.ekin = ekin;
    r.epot = epot;
    r.gscale = gscale;
    const size_t need = run_ws_bytes(r.Nf, norb, sizeof(T));
    if (!ws) return fail(WVL_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(WVL_EINVAL, "workspace is not 256-byte aligned");
    if (ws_bytes < need)
        return fail(WVL_ENOMEM_WS, "workspace has %zu bytes, %zu needed", ws_bytes, need);
    carve(r, static_cast<char*>(ws));
    std::vector<CellRun<T>> runs(1, r);
    return run_op<T>(op, runs, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

// -------------------------------------------------- free / surface boundaries
// Free (isolated) boundary conditions along an axis: the orbital lives on the
// coarse points of the box; every operator acts on the whole line.  The
// interaction range of H is 15 coarse points (synthesis 8 + magic filter 8
// fine points out, then back), so the periodic operator on a cell padded by
// FREE_PAD >= 8 coarse points per side along each free axis, restricted to
// the box, is the free-space operator exactly; V and rho cover the padded
// cell.  Surface conditions: one free axis, two periodic.
constexpr int FREE_PAD = WVL_FREE_PAD;

static void padded_grid(const wvl_grid* g, const int fa[3], wvl_grid* out) {
    *out = *g;
    out->n1 += fa[0] ? 2 * FREE_PAD : 0;
    out->n2 += fa[1] ? 2 * FREE_PAD : 0;
    out->n3 += fa[2] ? 2 * FREE_PAD : 0;
}

template <typename T>
static wvl_status bc_cell(int op, const wvl_grid* box, const int fa[3], int norb, const void* in,
                         void* out, const void* V, const double* occ, double* rho, double* ekin,
                         double* epot, void* ws, size_t ws_bytes, void* stream, bool emu) {
    wvl_grid g;
    padded_grid(box, fa, &g);
    CellRun<T> r;
    grid_dims(&g, r.n, r.Nf, r.hg, r.P);
    r.norb = norb;
    r.emu = emu;
    r.in = static_cast<const T*>(in);
    r.out = static_cast<T*>(out);
    r.V = static_cast<const T*>(V);
    r.rho = rho;
    r.occ = occ;
    r.ekin = ekin;
    r.epot = epot;
    r.ncoarse = (long long)box->n1 * box->n2 * box->n3;
    r.clen = 8 * r.ncoarse;
    if (emu) {
        // the tensor-core passes run the periodic operator on the padded
        // cell, restricted to the box
        r.bx[0] = box->n1;
        r.bx[1] = box->n2;
        r.bx[2] = box->n3;
        for (int d = 0; d < 3; ++d) r.bo[d] = fa[d] ? FREE_PAD : 0;
    } else {
        // every pass on the support its stage needs (grow_seg)
        r.grow = true;
        r.gb[0] = box->n1;
        r.gb[1] = box->n2;
        r.gb[2] = box->n3;
        for (int d = 0; d < 3; ++d) {
            r.gfree[d] = fa[d] != 0;
            r.vlo[d] = fa[d] ? -2 * FREE_PAD : 0;
        }
    }
    const size_t need = run_ws_bytes(r.Nf, norb, sizeof(T));
    if (!ws) return fail(WVL_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(WVL_EINVAL, "workspace is not 256-byte aligned");
    if (ws_bytes < need)
        return fail(WVL_ENOMEM_WS, "workspace has %zu bytes, %zu needed", ws_bytes, need);
    carve(r, static_cast<char*>(ws));
    std::vector<CellRun<T>> runs(1, r);
    return run_op<T>(op, runs, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------ preconditioner
// Diagonal of S_d^T T_d S_d on a periodic line of 2 nc fine points for the
// scaling (a = 0) and wavelet (a = 1) component of coarse point 0: the
// synthesis of that unit coefficient, the 29-tap kinetic filter, and the
// analysis entry.  By Eq. (fprod) and S_d^T S_d = 1, the diagonal of
// S^T K S for component mu = a1 + 2 a2 + 4 a3 is D_1[a1] + D_2[a2] + D_3[a3].
static void diag1d(int nc, double hgrid, double out[2]) {
    const FilterSet& F = filters();
    const int N = 2 * nc;
    auto wrap = [N](int i) { return ((i % N) + N) % N; };
    std::vector<double> s(N), t(N);
    const double sc = -1.0 / (2.0 * hgrid * hgrid);
    for (int a = 0; a < 2; ++a) {
        const double* f = (a == 0) ? F.h : F.g;
        std::fill(s.begin(), s.end(), 0.0);
        for (int k = -7; k <= 8; ++k) s[wrap(k)] += f[k + 7];
        for (int I = 0; I < N; ++I) {
            double v = 0.0;
            for (int l = -14; l <= 14; ++l) v += sc * F.a[l + 14] * s[wrap(I - l)];
            t[I] = v;
        }
        double y = 0.0;
        for (int k = -7; k <= 8; ++k) y += f[k + 7] * t[wrap(k)];
        out[a] = y;
    }
}

static void helmholtz_diag(const int n[3], const double hg[3], double d[8]) {
    double D[3][2];
    for (int ax = 0; ax < 3; ++ax) diag1d(n[ax], hg[ax], D[ax]);
    for (int mu = 0; mu < 8; ++mu) d[mu] = D[0][mu & 1] + D[1][(mu >> 1) & 1] + D[2][mu >> 2];
}

static int pcg_blocks(long long len) {
    long long b = (len + 4 * 256 - 1) / (4 * 256);
    return (int)std::max(1LL, std::min(b, 64LL));
}

static size_t precond_ws_bytes(const int Nf[3], int norb, size_t elt) {
    const long long P = (long long)Nf[0] * Nf[1] * Nf[2];
    size_t b = run_ws_bytes(Nf, norb, elt);
    b += 4 * align256((size_t)norb * P * elt);
    b += align256((size_t)norb * pcg_blocks(P) * sizeof(double));
    b += 3 * align256((size_t)norb * sizeof(double));
    return b;
}

template <typename T>
static wvl_status run_precond(const wvl_grid* grid, int norb, const T* g, const double* eps,
                              int ncg, T* x, double* rr, void* ws, size_t ws_bytes,
                              cudaStream_t st, bool emu) {
    CellRun<T> r;
    grid_dims(grid, r.n, r.Nf, r.hg, r.P);
    r.norb = norb;
    r.emu = emu;
    r.eps = eps;
    r.V = nullptr;
    r.rho = nullptr;
    r.occ = nullptr;
    r.ekin = nullptr;
    r.epot = nullptr;
    const size_t need = precond_ws_bytes(r.Nf, norb, sizeof(T));
    if (!ws) return fail(WVL_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(WVL_EINVAL, "workspace is not 256-byte aligned");
    if (ws_bytes < need)
        return fail(WVL_ENOMEM_WS, "workspace has %zu bytes, %zu needed", ws_bytes, need);
    char* w = static_cast<char*>(ws);
    carve(r, w);
    w += run_ws_bytes(r.Nf, norb, sizeof(T));
    const size_t vb = align256((size_t)norb * r.P * sizeof(T));
    T* rv = reinterpret_cast<T*>(w);
    T* zv = reinterpret_cast<T*>(w + vb);
    T* pv = reinterpret_cast<T*>(w + 2 * vb);
    T* Ap = reinterpret_cast<T*>(w + 3 * vb);
    w += 4 * vb;
    PcgParams q;
    helmholtz_diag(r.n, r.hg, q.diag);
    q.eps = eps;
    q.len = r.P;
    q.m = r.P / 8;
    q.norb = norb;
    q.nblk = pcg_blocks(r.P);
    q.part = reinterpret_cast<double*>(w);
    w += align256((size_t)norb * q.nblk * sizeof(double));
    double* rz0 = reinterpret_cast<double*>(w);
    double* rz1 = reinterpret_cast<double*>(w + align256(norb * sizeof(double)));
    double* pq = reinterpret_cast<double*>(w + 2 * align256(norb * sizeof(double)));

    cudaError_t e;
#define WVL_CU(call, what)                                  \
    do {                                                    \
        if ((e = (call)) != cudaSuccess) return cuda_fail(e, what); \
    } while (0)
    WVL_CU(launch_pcg<T>(PCG_INIT, q, x, rv, zv, pv, g, nullptr, nullptr, st), "pcg init");
    WVL_CU(launch_reduce_parts(q.part, nullptr, q.nblk, norb, rz0, st), "pcg r.z");
    for (int it = 0; it < ncg; ++it) {
        r.in = pv;
        r.out = Ap;
        std::vector<CellRun<T>> runs(1, r);
        wvl_status s = run_op<T>(OP_HELM, runs, nullptr, nullptr, st);
        if (s != WVL_OK) return s;
        WVL_CU(launch_pcg<T>(PCG_DOT, q, pv, Ap, nullptr, nullptr, nullptr, nullptr, nullptr, st),
               "pcg p.Ap");
        WVL_CU(launch_reduce_parts(q.part, nullptr, q.nblk, norb, pq, st), "pcg p.Ap");
        WVL_CU(launch_pcg<T>(PCG_STEP, q, x, rv, zv, pv, Ap, rz0, pq, st), "pcg step");
        WVL_CU(launch_reduce_parts(q.part, nullptr, q.nblk, norb, rz1, st), "pcg r.z");
        WVL_CU(launch_pcg<T>(PCG_DIR, q, pv, nullptr, zv, nullptr, nullptr, rz1, rz0, st),
               "pcg direction");
        std::swap(rz0, rz1);
    }
    if (rr) {
        WVL_CU(launch_pcg<T>(PCG_DOT, q, rv, rv, nullptr, nullptr, nullptr, nullptr, nullptr, st),
               "pcg r.r");
        WVL_CU(launch_reduce_parts(q.part, nullptr, q.nblk, norb, rr, st), "pcg r.r");
    }
#undef WVL_CU
    return WVL_OK;
}

static wvl_status dispatch_single(int op, const wvl_grid* grid, int prec, int norb,
                                  const void* in, void* out, const void* V,
                                  const double* occ, double* rho, double* ekin,
                                  double* epot, void* ws, size_t ws_bytes, void* stream,
                                  const wvl_region* reg = nullptr,
                                  const double* gscale = nullptr) {
    g_err[0] = 0;
    if (prec != WVL_F32)
        return single_cell<double>(op, grid, norb, in, out, V, occ, rho, ekin, epot, ws,
                                   ws_bytes, stream, reg, prec == WVL_F64_EMU, gscale);
    return single_cell<float>(op, grid, norb, in, out, V, occ, rho, ekin, epot, ws,
                              ws_bytes, stream, reg, false, gscale);
}

static wvl_status check_region(const wvl_grid* grid, const wvl_region* reg) {
    if (!reg) return fail(WVL_EINVAL, "region is NULL");
    WVL_TRY(check_ptr(reg->coarse_index, "region coarse_index", true));
    WVL_TRY(check_ptr(reg->fine_index, "region fine_index", true));
    const long long m = (long long)grid->n1 * grid->n2 * grid->n3;
    if (reg->ncoarse < 0 || reg->ncoarse > m || reg->nfine < 0 || reg->nfine > m)
        return fail(WVL_EINVAL, "region counts out of range (ncoarse %lld, nfine %lld, %lld points)",
                    reg->ncoarse, reg->nfine, m);
    const int n[3] = {grid->n1, grid->n2, grid->n3};
    for (int d = 0; d < 3; ++d)
        if (reg->len[d] < 0 || reg->len[d] > n[d] || reg->lo[d] < 0 || reg->lo[d] >= n[d])
            return fail(WVL_EINVAL, "region box out of range on axis %d (lo %d, len %d)", d + 1,
                        reg->lo[d], reg->len[d]);
    return WVL_OK;
}

}  // namespace wvl

// ==================================================================== C ABI
using namespace wvl;

struct wvl_plan {
    int prec = 0;
    unsigned flags = 0;
    std::vector<wvl_grid> cells;
    std::vector<int> cell_of_orb;
    int norb = 0;
    std::vector<size_t> orb_off;
    size_t total = 0;
    struct Run {
        int cell, o0, cnt;
        size_t off, ws_off;
    };
    std::vector<Run> runs;
    size_t ws_bytes = 0;
    TuneTable tune;
    bool tuned = false;
    int chain = CHAIN_AUTO;        // forced by the flags, or the autotuner's choice
    Prof prof;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const void*> gkey;
    size_t gnodes = 0;
    std::mutex mu;
    ~wvl_plan() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
    }
};

extern "C" {

const char* wvl_status_string(int s) {
    switch (s) {
    case WVL_OK: return "WVL_OK";
    case WVL_EINVAL: return "WVL_EINVAL: invalid argument";
    case WVL_ENOMEM_WS: return "WVL_ENOMEM_WS: workspace too small";
    case WVL_ECUDA: return "WVL_ECUDA: CUDA runtime error";
    case WVL_ETIMEOUT: return "WVL_ETIMEOUT: bounded device wait expired";
    case WVL_EUNSUPPORTED: return "WVL_EUNSUPPORTED: unsupported size or option";
    }
    return "unknown wvl status";
}

const char* wvl_last_error(void) { return g_err; }

int wvl_version(void) { return 10000; }

unsigned long long wvl_kernel_launches(void) { return g_launches.load(); }

wvl_status wvl_selftest_timeout(double ms, void* stream) {
    g_err[0] = 0;
    if (!(ms > 0.0) || ms > 10000.0) return fail(WVL_EINVAL, "ms must be in (0, 10000]");
    cudaError_t e = emu_wait_probe(ms, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? WVL_OK : cuda_fail(e, "timeout self-test");
}

wvl_status wvl_wait_timeouts(unsigned* count) {
    g_err[0] = 0;
    if (!count) return fail(WVL_EINVAL, "count is NULL");
    *count = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    e = emu_take_timeouts(count);
    if (e != cudaSuccess) return cuda_fail(e, "timeout counter");
    return *count ? fail(WVL_ETIMEOUT, "%u bounded device waits gave up", *count) : WVL_OK;
}

int wvl_device_count(void) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

wvl_status wvl_filters(double* h, double* g, double* w, int* k0, double* a) {
    const FilterSet& F = filters();
    if (h) std::memcpy(h, F.h, sizeof F.h);
    if (g) std::memcpy(g, F.g, sizeof F.g);
    if (w) std::memcpy(w, F.w, sizeof F.w);
    if (k0) *k0 = F.k0;
    if (a) std::memcpy(a, F.a, sizeof F.a);
    return WVL_OK;
}

wvl_status wvl_workspace_size(const wvl_grid* grid, int prec, int norb, size_t* bytes) {
    g_err[0] = 0;
    WVL_TRY(check_grid(grid));
    WVL_TRY(check_prec(prec));
    if (norb < 0) return fail(WVL_EINVAL, "norb < 0");
    if (!bytes) return fail(WVL_EINVAL, "bytes is NULL");
    int n[3], Nf[3];
    double hg[3];
    long long P;
    grid_dims(grid, n, Nf, hg, P);
    *bytes = run_ws_bytes(Nf, std::max(norb, 1), prec != WVL_F32 ? 8 : 4);
    return WVL_OK;
}

#define WVL_COMMON_CHECKS()                        \
    g_err[0] = 0;                                  \
    WVL_TRY(check_grid(grid));                     \
    WVL_TRY(check_prec(prec));                     \
    if (norb < 0) return fail(WVL_EINVAL, "norb < 0"); \
    if (norb == 0) return WVL_OK;

wvl_status wvl_synthesis(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                         void* s, void* ws, size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(s, "s", true));
    return dispatch_single(OP_SYN, grid, prec, norb, psi_c, s, nullptr, nullptr, nullptr,
                           nullptr, nullptr, ws, ws_bytes, stream);
}

wvl_status wvl_analysis(const wvl_grid* grid, int prec, int norb, const void* z,
                        void* psi_c, void* ws, size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(z, "z", true));
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    return dispatch_single(OP_ANA, grid, prec, norb, z, psi_c, nullptr, nullptr, nullptr,
                           nullptr, nullptr, ws, ws_bytes, stream);
}

wvl_status wvl_magicfilter(const wvl_grid* grid, int prec, int norb, const void* s,
                           void* psi_r, void* ws, size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(s, "s", true));
    WVL_TRY(check_ptr(psi_r, "psi_r", true));
    return dispatch_single(OP_MF, grid, prec, norb, s, psi_r, nullptr, nullptr, nullptr,
                           nullptr, nullptr, ws, ws_bytes, stream);
}

wvl_status wvl_magicfilter_T(const wvl_grid* grid, int prec, int norb, const void* y_r,
                             void* y, void* ws, size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(y_r, "y_r", true));
    WVL_TRY(check_ptr(y, "y", true));
    return dispatch_single(OP_MFT, grid, prec, norb, y_r, y, nullptr, nullptr, nullptr,
                           nullptr, nullptr, ws, ws_bytes, stream);
}

wvl_status wvl_kinetic(const wvl_grid* grid, int prec, int norb, const void* s,
                       const void* k0, void* out, double* ekin, void* ws, size_t ws_bytes,
                       void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(s, "s", true));
    WVL_TRY(check_ptr(k0, "k0", false));
    WVL_TRY(check_ptr(out, "out", true));
    WVL_TRY(check_ptr(ekin, "ekin", false));
    return dispatch_single(OP_KIN, grid, prec, norb, s, out, k0, nullptr, nullptr, ekin,
                           nullptr, ws, ws_bytes, stream);
}

wvl_status wvl_density(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                       const double* occ, double* rho, void* ws, size_t ws_bytes,
                       void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(occ, "occ", true));
    WVL_TRY(check_ptr(rho, "rho", true));
    return dispatch_single(OP_DENSITY, grid, prec, norb, psi_c, nullptr, nullptr, occ, rho,
                           nullptr, nullptr, ws, ws_bytes, stream);
}

wvl_status wvl_hpsi_local(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                          const void* V, const double* occ, void* hpsi_c, double* rho,
                          double* ekin, double* epot, void* ws, size_t ws_bytes,
                          void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(V, "V", true));
    WVL_TRY(check_ptr(occ, "occ", true));
    WVL_TRY(check_ptr(hpsi_c, "hpsi_c", true));
    WVL_TRY(check_ptr(rho, "rho", false));
    WVL_TRY(check_ptr(ekin, "ekin", true));
    WVL_TRY(check_ptr(epot, "epot", true));
    return dispatch_single(OP_HPSI, grid, prec, norb, psi_c, hpsi_c, V, occ, rho, ekin, epot,
                           ws, ws_bytes, stream);
}

wvl_status wvl_energy(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                      const void* V, const double* occ, double* rho, double* ekin,
                      double* epot, void* ws, size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(V, "V", true));
    WVL_TRY(check_ptr(occ, "occ", true));
    WVL_TRY(check_ptr(rho, "rho", false));
    WVL_TRY(check_ptr(ekin, "ekin", true));
    WVL_TRY(check_ptr(epot, "epot", true));
    return dispatch_single(OP_ENERGY, grid, prec, norb, psi_c, nullptr, V, occ, rho, ekin,
                           epot, ws, ws_bytes, stream);
}

wvl_status wvl_eloc(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                    const void* V, const double* occ, double* rho, double* ekin, double* epot,
                    double* eloc, void* ws, size_t ws_bytes, void* stream) {
    g_err[0] = 0;
    WVL_TRY(check_grid(grid));
    WVL_TRY(check_prec(prec));
    if (norb < 0) return fail(WVL_EINVAL, "norb < 0");
    WVL_TRY(check_ptr(eloc, "eloc", true));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (norb > 0) {
        WVL_TRY(check_ptr(psi_c, "psi_c", true));
        WVL_TRY(check_ptr(V, "V", true));
        WVL_TRY(check_ptr(occ, "occ", true));
        WVL_TRY(check_ptr(rho, "rho", false));
        WVL_TRY(check_ptr(ekin, "ekin", true));
        WVL_TRY(check_ptr(epot, "epot", true));
        WVL_TRY(dispatch_single(OP_ENERGY, grid, prec, norb, psi_c, nullptr, V, occ, rho, ekin,
                                epot, ws, ws_bytes, stream));
    }
    cudaError_t e = launch_eloc_total(occ, ekin, epot, norb, eloc, st);
    return e == cudaSuccess ? WVL_OK : cuda_fail(e, "E_loc reduction");
}

wvl_status wvl_eloc_backward(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                             const void* V, const double* occ, const double* rho,
                             const double* gbar, void* dpsi_c, void* dV, void* ws,
                             size_t ws_bytes, void* stream) {
    g_err[0] = 0;
    WVL_TRY(check_grid(grid));
    WVL_TRY(check_prec(prec));
    if (norb < 0) return fail(WVL_EINVAL, "norb < 0");
    WVL_TRY(check_ptr(gbar, "gbar", true));
    WVL_TRY(check_ptr(dpsi_c, "dpsi_c", false));
    WVL_TRY(check_ptr(dV, "dV", false));
    if (dV) WVL_TRY(check_ptr(rho, "rho (needed for dV)", true));
    if (dpsi_c && norb > 0) {
        WVL_TRY(check_ptr(psi_c, "psi_c", true));
        WVL_TRY(check_ptr(V, "V", true));
        WVL_TRY(check_ptr(occ, "occ", true));
        // the whole chain again (real-space psi recomputed, not stored), its
        // last pass writing 2 occ gbar H psi; no density, no energies
        WVL_TRY(dispatch_single(OP_HPSI, grid, prec, norb, psi_c, dpsi_c, V, occ, nullptr,
                                nullptr, nullptr, ws, ws_bytes, stream, nullptr, gbar));
    }
    if (dV) {
        const long long P = 8LL * grid->n1 * grid->n2 * grid->n3;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        cudaError_t e = prec == WVL_F32
                            ? launch_scale_density<float>(rho, gbar, P, static_cast<float*>(dV), st)
                            : launch_scale_density<double>(rho, gbar, P, static_cast<double*>(dV), st);
        if (e != cudaSuccess) return cuda_fail(e, "dE/dV");
    }
    return WVL_OK;
}

wvl_status wvl_precondition_workspace_size(const wvl_grid* grid, int prec, int norb,
                                           size_t* bytes) {
    g_err[0] = 0;
    WVL_TRY(check_grid(grid));
    WVL_TRY(check_prec(prec));
    if (norb < 0) return fail(WVL_EINVAL, "norb < 0");
    if (!bytes) return fail(WVL_EINVAL, "bytes is NULL");
    int n[3], Nf[3];
    double hg[3];
    long long P;
    grid_dims(grid, n, Nf, hg, P);
    *bytes = precond_ws_bytes(Nf, std::max(norb, 1), prec != WVL_F32 ? 8 : 4);
    return WVL_OK;
}

wvl_status wvl_precondition(const wvl_grid* grid, int prec, int norb, const void* g,
                            const double* eps, int ncg, void* x, double* rr, void* ws,
                            size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_ptr(g, "g", true));
    WVL_TRY(check_ptr(eps, "eps", true));
    WVL_TRY(check_ptr(x, "x", true));
    WVL_TRY(check_ptr(rr, "rr", false));
    if (ncg < 0 || ncg > 10000) return fail(WVL_EINVAL, "ncg = %d out of range", ncg);
    if (g == x) return fail(WVL_EINVAL, "g and x must not alias");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec != WVL_F32)
        return run_precond<double>(grid, norb, static_cast<const double*>(g), eps, ncg,
                                   static_cast<double*>(x), rr, ws, ws_bytes, st,
                                   prec == WVL_F64_EMU);
    return run_precond<float>(grid, norb, static_cast<const float*>(g), eps, ncg,
                              static_cast<float*>(x), rr, ws, ws_bytes, st, false);
}

// ------------------------------------------------- free / surface boundaries
static const int kAllFree[3] = {1, 1, 1};

static wvl_status bc_checks(const wvl_grid* grid, const int* fa, int prec, int norb) {
    g_err[0] = 0;
    if (!fa) return fail(WVL_EINVAL, "free_axes is NULL");
    for (int d = 0; d < 3; ++d)
        if (fa[d] != 0 && fa[d] != 1) return fail(WVL_EINVAL, "free_axes[%d] must be 0 or 1", d);
    WVL_TRY(check_grid(grid));
    WVL_TRY(check_prec(prec));
    wvl_grid g;
    padded_grid(grid, fa, &g);
    WVL_TRY(check_grid(&g));
    if (norb < 0) return fail(WVL_EINVAL, "norb < 0");
    return WVL_OK;
}

wvl_status wvl_bc_workspace_size(const wvl_grid* grid, const int* free_axes, int prec, int norb,
                                 size_t* bytes) {
    WVL_TRY(bc_checks(grid, free_axes, prec, std::max(norb, 0)));
    wvl_grid g;
    padded_grid(grid, free_axes, &g);
    return wvl_workspace_size(&g, prec, norb, bytes);
}

wvl_status wvl_hpsi_local_bc(const wvl_grid* grid, const int* free_axes, int prec, int norb,
                             const void* psi_c, const void* V, const double* occ, void* hpsi_c,
                             double* rho, double* ekin, double* epot, void* ws, size_t ws_bytes,
                             void* stream) {
    WVL_TRY(bc_checks(grid, free_axes, prec, norb));
    if (norb == 0) return WVL_OK;
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(V, "V", true));
    WVL_TRY(check_ptr(occ, "occ", true));
    WVL_TRY(check_ptr(hpsi_c, "hpsi_c", true));
    WVL_TRY(check_ptr(rho, "rho", false));
    WVL_TRY(check_ptr(ekin, "ekin", true));
    WVL_TRY(check_ptr(epot, "epot", true));
    if (prec != WVL_F32)
        return bc_cell<double>(OP_HPSI, grid, free_axes, norb, psi_c, hpsi_c, V, occ, rho, ekin,
                               epot, ws, ws_bytes, stream, prec == WVL_F64_EMU);
    return bc_cell<float>(OP_HPSI, grid, free_axes, norb, psi_c, hpsi_c, V, occ, rho, ekin, epot,
                          ws, ws_bytes, stream, false);
}

wvl_status wvl_density_bc(const wvl_grid* grid, const int* free_axes, int prec, int norb,
                          const void* psi_c, const double* occ, double* rho, void* ws,
                          size_t ws_bytes, void* stream) {
    WVL_TRY(bc_checks(grid, free_axes, prec, norb));
    if (norb == 0) return WVL_OK;
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(occ, "occ", true));
    WVL_TRY(check_ptr(rho, "rho", true));
    if (prec != WVL_F32)
        return bc_cell<double>(OP_DENSITY, grid, free_axes, norb, psi_c, nullptr, nullptr, occ,
                               rho, nullptr, nullptr, ws, ws_bytes, stream, prec == WVL_F64_EMU);
    return bc_cell<float>(OP_DENSITY, grid, free_axes, norb, psi_c, nullptr, nullptr, occ, rho,
                          nullptr, nullptr, ws, ws_bytes, stream, false);
}

wvl_status wvl_free_workspace_size(const wvl_grid* grid, int prec, int norb, size_t* bytes) {
    return wvl_bc_workspace_size(grid, kAllFree, prec, norb, bytes);
}

wvl_status wvl_hpsi_local_free(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                               const void* V, const double* occ, void* hpsi_c, double* rho,
                               double* ekin, double* epot, void* ws, size_t ws_bytes,
                               void* stream) {
    return wvl_hpsi_local_bc(grid, kAllFree, prec, norb, psi_c, V, occ, hpsi_c, rho, ekin, epot,
                             ws, ws_bytes, stream);
}

wvl_status wvl_density_free(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                            const double* occ, double* rho, void* ws, size_t ws_bytes,
                            void* stream) {
    return wvl_density_bc(grid, kAllFree, prec, norb, psi_c, occ, rho, ws, ws_bytes, stream);
}

// ------------------------------------------------------ localisation regions
wvl_status wvl_region_index(const wvl_grid* grid, const unsigned char* coarse_mask,
                            const unsigned char* fine_mask, int* coarse_index,
                            int* fine_index, long long* ncoarse, long long* nfine) {
    g_err[0] = 0;
    WVL_TRY(check_grid(grid));
    if (!coarse_mask || !fine_mask || !coarse_index || !fine_index || !ncoarse || !nfine)
        return fail(WVL_EINVAL, "NULL argument");
    const long long m = (long long)grid->n1 * grid->n2 * grid->n3;
    if (m > 0x7fffffffLL) return fail(WVL_EUNSUPPORTED, "grid too large for int32 indices");
    long long c = 0, f = 0;
    for (long long p = 0; p < m; ++p) {
        coarse_index[p] = coarse_mask[p] ? (int)c++ : -1;
        fine_index[p] = fine_mask[p] ? (int)f++ : -1;
    }
    *ncoarse = c;
    *nfine = f;
    return WVL_OK;
}

wvl_status wvl_region_bounds(const wvl_grid* grid, const unsigned char* coarse_mask,
                             const unsigned char* fine_mask, int* lo, int* len) {
    g_err[0] = 0;
    WVL_TRY(check_grid(grid));
    if (!coarse_mask || !fine_mask || !lo || !len) return fail(WVL_EINVAL, "NULL argument");
    const int n[3] = {grid->n1, grid->n2, grid->n3};
    for (int d = 0; d < 3; ++d) {
        // coordinates along axis d that some region point occupies
        std::vector<char> occ(n[d], 0);
        for (int i3 = 0; i3 < n[2]; ++i3)
            for (int i2 = 0; i2 < n[1]; ++i2)
                for (int i1 = 0; i1 < n[0]; ++i1) {
                    const long long p = ((long long)i3 * n[1] + i2) * n[0] + i1;
                    if (coarse_mask[p] || fine_mask[p]) occ[d == 0 ? i1 : d == 1 ? i2 : i3] = 1;
                }
        // the box is the complement of the longest periodic run of free coordinates
        int best = 0, best_end = -1;
        for (int s = 0; s < n[d]; ++s) {
            if (occ[s]) continue;
            int l = 0;
            while (l < n[d] && !occ[(s + l) % n[d]]) ++l;
            if (l > best) { best = l; best_end = (s + l) % n[d]; }
        }
        if (best == n[d]) { lo[d] = 0; len[d] = 0; continue; }   // empty region
        lo[d] = best == 0 ? 0 : best_end;
        len[d] = n[d] - best;
    }
    return WVL_OK;
}

wvl_status wvl_synthesis_region(const wvl_grid* grid, const wvl_region* region, int prec,
                                int norb, const void* psi_c, void* s, void* ws,
                                size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_region(grid, region));
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(s, "s", true));
    return dispatch_single(OP_SYN, grid, prec, norb, psi_c, s, nullptr, nullptr, nullptr,
                           nullptr, nullptr, ws, ws_bytes, stream, region);
}

wvl_status wvl_analysis_region(const wvl_grid* grid, const wvl_region* region, int prec,
                               int norb, const void* z, void* psi_c, void* ws,
                               size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_region(grid, region));
    WVL_TRY(check_ptr(z, "z", true));
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    return dispatch_single(OP_ANA, grid, prec, norb, z, psi_c, nullptr, nullptr, nullptr,
                           nullptr, nullptr, ws, ws_bytes, stream, region);
}

wvl_status wvl_density_region(const wvl_grid* grid, const wvl_region* region, int prec,
                              int norb, const void* psi_c, const double* occ, double* rho,
                              void* ws, size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_region(grid, region));
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(occ, "occ", true));
    WVL_TRY(check_ptr(rho, "rho", true));
    return dispatch_single(OP_DENSITY, grid, prec, norb, psi_c, nullptr, nullptr, occ, rho,
                           nullptr, nullptr, ws, ws_bytes, stream, region);
}

wvl_status wvl_hpsi_local_region(const wvl_grid* grid, const wvl_region* region, int prec,
                                 int norb, const void* psi_c, const void* V, const double* occ,
                                 void* hpsi_c, double* rho, double* ekin, double* epot,
                                 void* ws, size_t ws_bytes, void* stream) {
    WVL_COMMON_CHECKS();
    WVL_TRY(check_region(grid, region));
    WVL_TRY(check_ptr(psi_c, "psi_c", true));
    WVL_TRY(check_ptr(V, "V", true));
    WVL_TRY(check_ptr(occ, "occ", true));
    WVL_TRY(check_ptr(hpsi_c, "hpsi_c", true));
    WVL_TRY(check_ptr(rho, "rho", false));
    WVL_TRY(check_ptr(ekin, "ekin", true));
    WVL_TRY(check_ptr(epot, "epot", true));
    return dispatch_single(OP_HPSI, grid, prec, norb, psi_c, hpsi_c, V, occ, rho, ekin, epot,
                           ws, ws_bytes, stream, region);
}

// ----------------------------------------------------------------- plans
wvl_status wvl_plan_create(const wvl_grid* cells, int ncell, const int* cell_of_orb,
                           int norb, int prec, unsigned flags, wvl_plan** out) {
    g_err[0] = 0;
    if (!out) return fail(WVL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cells || ncell < 1) return fail(WVL_EINVAL, "need at least one cell");
    if (norb < 0 || (norb > 0 && !cell_of_orb)) return fail(WVL_EINVAL, "bad orbital list");
    WVL_TRY(check_prec(prec));
    if (flags & ~(WVL_PLAN_GRAPH | WVL_PLAN_AUTOTUNE | WVL_PLAN_FUSED | WVL_PLAN_PASSES))
        return fail(WVL_EINVAL, "unknown plan flags");
    if ((flags & WVL_PLAN_FUSED) && (flags & WVL_PLAN_PASSES))
        return fail(WVL_EINVAL, "WVL_PLAN_FUSED and WVL_PLAN_PASSES exclude each other");
    for (int c = 0; c < ncell; ++c) WVL_TRY(check_grid(&cells[c]));
    for (int o = 0; o < norb; ++o)
        if (cell_of_orb[o] < 0 || cell_of_orb[o] >= ncell)
            return fail(WVL_EINVAL, "cell_of_orb[%d] = %d out of range", o, cell_of_orb[o]);
    if (flags & WVL_PLAN_FUSED) {
        if (prec == WVL_F64_EMU)
            return fail(WVL_EUNSUPPORTED, "the fused chain has no tensor-core form");
        for (int c = 0; c < ncell; ++c) {
            int n[3], Nf[3];
            double hg[3];
            long long P;
            grid_dims(&cells[c], n, Nf, hg, P);
            const bool ok = prec == WVL_F32 ? fused_cell_ok<float>(Nf) : fused_cell_ok<double>(Nf);
            if (!ok)
                return fail(WVL_EUNSUPPORTED, "cell %d: the fused chain needs fine extents that are "
                            "multiples of 8 in [%d, %d] (and planes that fit one CTA)", c,
                            FZ_MIN_FINE, FZ_MAX_FINE);
        }
    }
    wvl_plan* p = new (std::nothrow) wvl_plan;
    if (!p) return fail(WVL_EINVAL, "host allocation failed");
    p->prec = prec;
    p->flags = flags;
    p->chain = (flags & WVL_PLAN_FUSED) ? CHAIN_FUSED : (flags & WVL_PLAN_PASSES) ? CHAIN_PASSES : CHAIN_AUTO;
    p->cells.assign(cells, cells + ncell);
    p->cell_of_orb.assign(cell_of_orb, cell_of_orb + norb);
    p->norb = norb;
    const size_t elt = prec != WVL_F32 ? 8 : 4;
    size_t off = 0, wsoff = 0;
    for (int o = 0; o < norb;) {
        const int c = cell_of_orb[o];
        int e = o;
        while (e < norb && cell_of_orb[e] == c) ++e;
        const wvl_grid& g = cells[c];
        int n[3], Nf[3];
        double hg[3];
        long long P;
        grid_dims(&g, n, Nf, hg, P);
        wvl_plan::Run r{c, o, e - o, off, wsoff};
        p->runs.push_back(r);
        for (int k = o; k < e; ++k) {
            p->orb_off.push_back(off);
            off += (size_t)P;
        }
        wsoff += align256(run_ws_bytes(Nf, e - o, elt));
        o = e;
    }
    p->total = off;
    p->ws_bytes = std::max<size_t>(wsoff, 256);
    *out = p;
    return WVL_OK;
}

wvl_status wvl_plan_destroy(wvl_plan* plan) {
    delete plan;
    return WVL_OK;
}

wvl_status wvl_plan_workspace_size(const wvl_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return fail(WVL_EINVAL, "NULL argument");
    *bytes = plan->ws_bytes;
    return WVL_OK;
}

wvl_status wvl_plan_orbital_offset(const wvl_plan* plan, int o, size_t* offset) {
    if (!plan || !offset) return fail(WVL_EINVAL, "NULL argument");
    if (o < 0 || o > plan->norb) return fail(WVL_EINVAL, "orbital index out of range");
    *offset = (o == plan->norb) ? plan->total : plan->orb_off[o];
    return WVL_OK;
}

}  // extern "C"

template <typename T>
static wvl_status plan_runs(wvl_plan* plan, const void* psi, const void* const* V,
                            const double* occ, void* hpsi, double* const* rho, double* ekin,
                            double* epot, void* ws, std::vector<CellRun<T>>& runs) {
    for (const auto& pr : plan->runs) {
        CellRun<T> r;
        grid_dims(&plan->cells[pr.cell], r.n, r.Nf, r.hg, r.P);
        r.norb = pr.cnt;
        r.in = static_cast<const T*>(psi) + pr.off;
        r.out = static_cast<T*>(hpsi) + pr.off;
        r.V = static_cast<const T*>(V[pr.cell]);
        r.rho = rho ? rho[pr.cell] : nullptr;
        r.occ = occ + pr.o0;
        r.ekin = ekin + pr.o0;
        r.epot = epot + pr.o0;
        r.emu = plan->prec == WVL_F64_EMU;
        r.chain = plan->chain;
        carve(r, static_cast<char*>(ws) + pr.ws_off);
        runs.push_back(r);
    }
    return WVL_OK;
}

static wvl_status plan_check(wvl_plan* plan, const void* psi, const void* const* V,
                             const double* occ, void* hpsi, double* const* rho, double* ekin,
                             double* epot, void* ws, size_t ws_bytes) {
    if (!plan) return fail(WVL_EINVAL, "plan is NULL");
    WVL_TRY(check_ptr(psi, "psi", true));
    WVL_TRY(check_ptr(hpsi, "hpsi", true));
    WVL_TRY(check_ptr(occ, "occ", true));
    WVL_TRY(check_ptr(ekin, "ekin", true));
    WVL_TRY(check_ptr(epot, "epot", true));
    if (!V) return fail(WVL_EINVAL, "V is NULL");
    for (size_t c = 0; c < plan->cells.size(); ++c) {
        WVL_TRY(check_ptr(V[c], "V[cell]", true));
        if (rho) WVL_TRY(check_ptr(rho[c], "rho[cell]", false));
    }
    if (!ws) return fail(WVL_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(WVL_EINVAL, "workspace is not 256-byte aligned");
    if (ws_bytes < plan->ws_bytes)
        return fail(WVL_ENOMEM_WS, "workspace has %zu bytes, %zu needed", ws_bytes, plan->ws_bytes);
    return WVL_OK;
}

template <typename T>
static wvl_status plan_exec(wvl_plan* plan, const void* psi, const void* const* V,
                            const double* occ, void* hpsi, double* const* rho, double* ekin,
                            double* epot, void* ws, cudaStream_t st) {
    std::vector<CellRun<T>> runs;
    plan_runs<T>(plan, psi, V, occ, hpsi, rho, ekin, epot, ws, runs);
    const bool graph = (plan->flags & WVL_PLAN_GRAPH) && !plan->prof.on && st != nullptr;
    if (!graph) return run_op<T>(OP_HPSI, runs, &plan->tune, &plan->prof, st);

    std::vector<const void*> key = {psi, occ, hpsi, ekin, epot, ws};
    for (size_t c = 0; c < plan->cells.size(); ++c) {
        key.push_back(V[c]);
        key.push_back(rho ? rho[c] : nullptr);
    }
    if (plan->gexec && key == plan->gkey) {
        cudaError_t e = cudaGraphLaunch(plan->gexec, st);
        if (e == cudaSuccess) count_launches(plan->gnodes);
        return e == cudaSuccess ? WVL_OK : cuda_fail(e, "cudaGraphLaunch");
    }
    const unsigned long long before = g_launches.load();
    // capture the enqueue sequence into a graph; the kernels' shared-memory
    // attributes are set before capture (host-only calls)
    cudaError_t e = (plan->prec == WVL_F64_EMU) ? prepare_emu_kernels() : prepare_pass_kernels<T>();
    if (e == cudaSuccess && plan->prec != WVL_F64_EMU) e = prepare_fused_kernels<T>();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    wvl_status s = run_op<T>(OP_HPSI, runs, &plan->tune, nullptr, st);
    e = cudaStreamEndCapture(st, &g);
    if (s != WVL_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    plan->graph = g;
    plan->gexec = ge;
    plan->gkey = key;
    // the capture counted its kernels once; they run now, on the replay
    plan->gnodes = (size_t)(g_launches.load() - before);
    e = cudaGraphLaunch(ge, st);
    return e == cudaSuccess ? WVL_OK : cuda_fail(e, "cudaGraphLaunch");
}

extern "C" {

wvl_status wvl_plan_hpsi(wvl_plan* plan, const void* psi, const void* const* V,
                         const double* occ, void* hpsi, double* const* rho, double* ekin,
                         double* epot, void* ws, size_t ws_bytes, void* stream) {
    g_err[0] = 0;
    WVL_TRY(plan_check(plan, psi, V, occ, hpsi, rho, ekin, epot, ws, ws_bytes));
    if (plan->norb == 0) return WVL_OK;
    std::lock_guard<std::mutex> lk(plan->mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (plan->prec != WVL_F32) return plan_exec<double>(plan, psi, V, occ, hpsi, rho, ekin, epot, ws, st);
    return plan_exec<float>(plan, psi, V, occ, hpsi, rho, ekin, epot, ws, st);
}

}  // extern "C"

template <typename T>
static wvl_status plan_tune(wvl_plan* plan, const void* psi, const void* const* V,
                            const double* occ, void* hpsi, double* const* rho, double* ekin,
                            double* epot, void* ws, cudaStream_t st) {
    std::vector<CellRun<T>> runs;
    plan_runs<T>(plan, psi, V, occ, hpsi, rho, ekin, epot, ws, runs);
    // one full run leaves realistic values in every buffer
    WVL_TRY(run_op<T>(OP_HPSI, runs, &plan->tune, nullptr, st));
    if (plan->prec == WVL_F64_EMU) {
        // the emulated passes have one launch shape: nothing to tune
        plan->tuned = true;
        cudaError_t e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? WVL_OK : cuda_fail(e, "autotune");
    }
    std::vector<PassCall<T>> calls = build_calls<T>(OP_HPSI, runs);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    TuneTable best;
    for (auto& c : calls) {
        float bt = 1e30f;
        Tune bv = default_tune(c);
        for (int R : {4, 8})
            for (int lt : {32, 16, 8, 4})
            for (int ps = 0; ps < 2; ++ps) {
                Tune t;
                t.R = R;
                t.LT = lt;
                t.persist = ps != 0;
                if (!tune_valid(c, t)) continue;
                float tot = 0.f;
                bool ok = true;
                for (int rep = 0; rep < 3 && ok; ++rep) {
                    cudaEventRecord(e0, st);
                    ok = exec_call(c, t, st) == WVL_OK;
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) tot += ms;   // first repetition is a warm-up
                }
                if (ok && tot < bt) {
                    bt = tot;
                    bv = t;
                }
            }
        best[tune_key(c.kind, c.mode, c.pass)] = bv;
    }
    plan->tune = best;
    // the chain: time both where the flags leave the choice and the cells allow
    if (!(plan->flags & (WVL_PLAN_FUSED | WVL_PLAN_PASSES)) && fused_ok(runs)) {
        float tc[2] = {0.f, 0.f};
        for (int ch = 0; ch < 2; ++ch) {
            for (auto& r : runs) r.chain = ch == 0 ? CHAIN_PASSES : CHAIN_FUSED;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, st);
                wvl_status s = run_op<T>(OP_HPSI, runs, &plan->tune, nullptr, st);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                if (s != WVL_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return s;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tc[ch] += ms;
            }
        }
        plan->chain = tc[1] < tc[0] ? CHAIN_FUSED : CHAIN_PASSES;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan->tuned = true;
    if (plan->gexec) {
        cudaGraphExecDestroy(plan->gexec);
        plan->gexec = nullptr;
    }
    if (plan->graph) {
        cudaGraphDestroy(plan->graph);
        plan->graph = nullptr;
    }
    plan->gkey.clear();
    cudaError_t e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? WVL_OK : cuda_fail(e, "autotune");
}

extern "C" {

wvl_status wvl_plan_autotune(wvl_plan* plan, const void* psi, const void* const* V,
                             const double* occ, void* hpsi, double* const* rho, double* ekin,
                             double* epot, void* ws, size_t ws_bytes, void* stream) {
    g_err[0] = 0;
    WVL_TRY(plan_check(plan, psi, V, occ, hpsi, rho, ekin, epot, ws, ws_bytes));
    if (!(plan->flags & WVL_PLAN_AUTOTUNE)) return fail(WVL_EINVAL, "plan created without WVL_PLAN_AUTOTUNE");
    if (plan->norb == 0) return WVL_OK;
    std::lock_guard<std::mutex> lk(plan->mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (plan->prec != WVL_F32) return plan_tune<double>(plan, psi, V, occ, hpsi, rho, ekin, epot, ws, st);
    return plan_tune<float>(plan, psi, V, occ, hpsi, rho, ekin, epot, ws, st);
}

wvl_status wvl_plan_describe(const wvl_plan* plan, char* buf, size_t len) {
    if (!plan || !buf || len == 0) return fail(WVL_EINVAL, "NULL argument");
    static const char* kn[] = {"synthesis", "analysis", "magicfilter", "magicfilter_T", "kinetic"};
    std::string s = plan->tuned ? "autotuned\n" : "defaults\n";
    s += plan->chain == CHAIN_FUSED ? "chain: fused plane/column kernels\n"
         : plan->chain == CHAIN_PASSES ? "chain: transposing 1D passes\n"
         : "chain: automatic (fused plane/column kernels for FP32 where the cells allow)\n";
    for (const auto& kv : plan->tune) {
        char line[128];
        snprintf(line, sizeof line, "%s mode %d pass %d: R=%d LT=%d %s\n", kn[kv.first / 100],
                 (kv.first / 10) % 10, kv.first % 10, kv.second.R, kv.second.LT,
                 kv.second.persist ? "persistent" : "one CTA per job");
        s += line;
    }
    std::strncpy(buf, s.c_str(), len - 1);
    buf[len - 1] = 0;
    return WVL_OK;
}

wvl_status wvl_plan_set_profiling(wvl_plan* plan, int on) {
    if (!plan) return fail(WVL_EINVAL, "plan is NULL");
    std::lock_guard<std::mutex> lk(plan->mu);
    plan->prof.on = on != 0;
    return WVL_OK;
}

wvl_status wvl_plan_profile(wvl_plan* plan, double* ms, int* launches, int nstage) {
    if (!plan) return fail(WVL_EINVAL, "plan is NULL");
    std::lock_guard<std::mutex> lk(plan->mu);
    plan->prof.flush();
    for (int k = 0; k < nstage && k < WVL_NSTAGE; ++k) {
        if (ms) ms[k] = plan->prof.ms[k];
        if (launches) launches[k] = plan->prof.cnt[k];
        plan->prof.ms[k] = 0;
        plan->prof.cnt[k] = 0;
    }
    return WVL_OK;
}

}  // extern "C"
