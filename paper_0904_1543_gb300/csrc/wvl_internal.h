// Internal declarations shared by the host API and the kernel translation
// units.  Not part of the public ABI (see include/wvl.h).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime_api.h>

#include "wvl.h"

namespace wvl {

// Filters of the method, derived on the host (filters.cpp).
struct FilterSet {
    double h[16];   // h_j, j = -7..8         (Eq. refinement)
    double g[16];   // g_j = (-1)^j h_{1-j}
    double w[16];   // w_k, k = k0..k0+15     (Eq. magicfilter)
    double a[29];   // a_l, l = -14..14       (Eqs. kiner, fprod)
    int k0;
};
const FilterSet& filters();

// The five 1D operators.  Each 3D operator is three passes of
// F(I, a) = sum_t f_t G(a, I - HL + off + t), output written transposed
// (Eqs. 1dconvtrans and kinetic1d).
enum Kind { K_SYN = 0, K_ANA = 1, K_MF = 2, K_MFT = 3, K_KIN = 4, NKIND = 5 };

// Load/epilogue variants of a pass.
enum Mode {
    M_PLAIN = 0,   // read lines, write transposed
    M_UNCOMP = 1,  // synthesis pass 1: gather lines from the compressed layout
    M_COMP = 2,    // analysis pass 3: scatter into the compressed layout
    M_POT = 3,     // magic-filter pass 3: V*psi, rho += occ psi^2, Epot partials
    M_KMID = 4,    // kinetic pass 1/2: K_p = T*G + K_{p-1}, G_p = G^T
    M_KLAST = 5,   // kinetic pass 3: K_3 and sum s*(K_3 - K0) partials
    NMODE = 6
};

constexpr int MAXSEG = 8;      // cells (segments) per launch
constexpr int NTHREADS = 128;  // threads per CTA (4 warps)
// register-resident density outputs per thread in the FP64 M_POT pass (the
// FP32 pass keeps its compensated density sums in shared memory)
template <typename T>
__host__ __device__ constexpr int pot_out() { return sizeof(T) == 8 ? 32 : 16; }
constexpr int MAX_FINE = 1024; // largest fine extent of one axis

// One cell's orbitals inside one pass launch.  Element offsets are per
// orbital; orbital o of the segment starts at o * P in every array (P = fine
// points = compressed length).
template <typename T>
struct Seg {
    const T* in;          // pass input (orbital 0 of the segment)
    T* out;               // pass output (may be null for reduction-only M_POT/M_KLAST)
    const T* in2;         // K_{p-1} for M_KMID/M_KLAST (null = 0)
    T* out2;              // G_p for M_KMID
    const T* aux;         // M_POT: V (null = no potential);  M_KLAST: K0 (null = 0)
    double* rho;          // M_POT: density target (null = none)
    double* part;         // per (orbital, tile) partial sums, [norb][tiles]
    const double* occ;    // M_POT: occupations of the segment's orbitals
    const double* gscale; // M_COMP: when set, output o is scaled by 2 occ[o] gscale[0]
                          //   (dE_loc/dpsi = 2 occ g H psi, the adjoint of E_loc)
    const double* eps;    // M_KMID pass 1 without in2: K_0 = -eps[o] G (Helmholtz shift)
    const int* mapc;      // M_UNCOMP/M_COMP with a localisation region: coarse point ->
    const int* mapf;      //   position of c^0 / index k of c^{1..7} (ncoarse + 7k), or -1
    const int* lexp;      // emulated M_UNCOMP: largest biased exponent of each input line,
                          //   [orbital][line] (null: the pass scans its lines)
    long long clen;       // compressed length of one orbital (orbital stride there)
    long long ncoarse;    // scaling coefficients stored (start of the wavelet block)
    int bx1, bx2, bx3;    // free/surface boundary conditions: box extents inside the
    int bo1, bo2, bo3;    //   padded cell and its offsets (coarse points); bx1 = 0 otherwise
    int nin;              // free lines (no wrap; 0 = periodic lines): input line length;
    int inoff;            //   row slot j holds input element j - hl + inoff, zero outside
    long long Pin;        //   [0, nin); Pin = input elements per orbital
    int vN1, vN2, vN3;    // M_POT on free lines: V and rho live on another grid (extents
    int vo1, vo2, vo3;    //   vN1, vN2, vN3, vP elements); output (X1, X2, I) sits there at
    long long vP;         //   (X1 + vo1, X2 + vo2, I + vo3) modulo the extents; vN1 = 0: same
                          //   layout as the output
    int go1, go2, go3;    // free lines over a region's box: the box origin in the cell and
    int gc1, gc2, gc3;    //   the cell's coarse extents (region index lookups, with wrap);
                          //   gc1 = 0 otherwise
    long long P;          // elements per orbital
    long long rho_gstride;// M_POT: 0 -> rho += (direct), else group g writes rho[g*stride]
    long long blk0;       // first work unit of the segment in the launch
    int n, N;             // line length and line count of this pass
    int N1, N2;           // fine extents (index decoding)
    int n1, n2;           // coarse extents (compressed layout)
    int norb;
    int tiles;            // work units per orbital (group): ceil(N / LT), times nwin when emulated
    int nwin;             // emulated FP64 passes: output windows per line
    int opg;              // M_POT: orbitals per group
    int rowlen;           // shared-memory row length in elements
};

// A work unit is one (orbital, tile) -- or, for M_POT, one (orbital group,
// tile) whose orbitals the CTA walks in order.  The kernel is persistent:
// CTA b takes units b, b + gridDim.x, ... and stages the next job in the
// second shared-memory buffer while it computes the current one.
template <typename T>
struct PassParams {
    T f[2][32];           // taps per output parity (single-parity kinds: both equal)
    float2 tp[32];        // FP32: tap pairs of outputs 2m, 2m + 1 (pass_kernel.cuh)
    long long nunits;     // work units over all segments
    int bufelems;         // elements of one staging buffer (two are allocated)
    int hl;               // left halo
    int LT;               // lines per tile (power of two, 4..32)
    int nseg;
    Seg<T> seg[MAXSEG];
};

// ------------------------------------------------ fused plane/column chain
// The local Hamiltonian chain as five kernels (fused_kernel.cu): each xy plane
// kernel keeps one fine-grid plane of an orbital in shared memory and applies
// the axis-1 and axis-2 filters of one or more operators to it; each column
// kernel keeps N3 x 32-column (FP64: 16) tiles and applies the axis-3
// filters.  Programs, in chain order (a = S3 c, s = S1 S2 a):
enum FzProg {
    FZ_SYN3 = 0,    // column: gather c from the compressed form, a = S3 c
    FZ_SKM12 = 1,   // plane:  s = S1 S2 a;  v = (T1 + T2) s (Ekin part);  t = MF1 MF2 s
    FZ_POT3 = 2,    // column: psi_r = MF3 t;  V psi_r, rho, Epot;  x = MFT3 (V psi_r)
    FZ_MFTA12 = 3,  // plane:  w' = A1 A2 (MFT1 MFT2 x + v)
    FZ_TA3 = 4,     // column, two I2 rows: H psi = A3 (w' + T3 a) (Ekin part), compressed
    FZ_NPROG = 5
};
constexpr int FZ_PTHREADS = 256;   // plane kernels
constexpr int FZ_CTHREADS = 128;   // column kernels
constexpr int FZ_RR = 8;           // row-pass outputs per thread (along the row)
constexpr int FZ_RC = 8;           // column-pass outputs per thread (along the column)
constexpr int FZ_MIN_FINE = 32;    // fine extents the fused chain takes: multiples
constexpr int FZ_MAX_FINE = 128;   //   of 8 in [32, 128]
constexpr int FZ_EPW = 64;         // FZ_POT3: orbitals whose Epot partials are held at once
template <typename T>
__host__ __device__ constexpr int fz_ltc() { return 128 / (int)sizeof(T); }   // tile columns

template <typename T>
struct FzSeg {
    const T* in;          // program input (FZ_SYN3: compressed psi)
    const T* in2;         // FZ_MFTA12: v;  FZ_TA3: a
    T* out;               // program output (FZ_TA3: compressed H psi)
    T* out2;              // FZ_SKM12: v
    T* out3;              // FZ_SKM12: t
    const T* V;           // FZ_POT3: potential
    double* rho;          // FZ_POT3: density target (null = none)
    long long rho_gstride;// 0 -> rho += ; else group g writes rho[g * stride]
    const double* occ;    // FZ_POT3: occupations;  FZ_TA3 with gscale: the scale's occ
    const double* gscale; // FZ_TA3: when set, H psi of orbital o is scaled by 2 occ[o] gscale[0]
    double* part;         // energy partials [norb][ptiles]; this program writes from poff
    long long P;          // fine points per orbital
    long long blk0;       // first job of the segment in the launch
    int N1, N2, N3, n1, n2;
    int norb, opg;        // FZ_POT3: orbitals per group
    int ncb;              // column blocks per row, ceil(N1 / fz_ltc)
    int ptiles, poff;
    int RS;               // shared-memory row stride in elements
};

template <typename T>
struct FzParams {
    T tap[4][2][32];      // the program's filters, per output parity (see fused_kernel.cu)
    float2 tp[4][32];     // FP32 row passes: tap pairs of outputs 2m, 2m + 1 (fused_kernel.cu)
    long long njobs;
    int nseg;
    FzSeg<T> seg[MAXSEG];
};

// shared-memory row stride of an xy plane with N1 columns: a 16-byte multiple
// whose count of 16-byte words is odd (lane-per-row vector loads hit distinct banks)
template <typename T>
inline int fz_plane_rs(int N1) {
    const int v = 16 / (int)sizeof(T);
    int w = (N1 + v - 1) / v;
    if ((w & 1) == 0) ++w;
    return w * v;
}
template <typename T>
size_t fz_smem(int prog, int N1, int N2, int N3);
template <typename T>
cudaError_t launch_fused(int prog, const FzParams<T>& p, size_t smem, cudaStream_t st);
template <typename T>
cudaError_t prepare_fused_kernels();

// Per-kind geometry: taps, parity offsets, left/right halo.
struct KindGeom {
    int nt, off0, off1, extra, hl, hr;
};
KindGeom kind_geom(int kind);

// Fills p.f and p.hl for a kind and axis spacing (kinetic only).
template <typename T>
void fill_taps(PassParams<T>& p, int kind, double hgrid);

// Launches one pass.  R (outputs per thread) must be 4 or 8.
template <typename T>
cudaError_t launch_pass(int kind, int mode, int R, const PassParams<T>& p,
                        long long nunits, size_t smem, cudaStream_t st, bool persistent);

// Sets the dynamic shared-memory attribute of every pass kernel on the
// current device (done lazily by launch_pass too; needed before capture).
template <typename T>
cudaError_t prepare_pass_kernels();

// Preconditioned conjugate gradient on compressed coefficients (pcg.cu).
struct PcgParams {
    double diag[8];       // diagonal of S^T K S per component mu
    const double* eps;    // per-orbital shift (device)
    double* part;         // block partials [norb][nblk]
    long long len;        // compressed length per orbital (8 m)
    long long m;          // coarse points
    int norb;
    int nblk;             // blocks per orbital
};
enum PcgOp { PCG_INIT = 0, PCG_DOT = 1, PCG_STEP = 2, PCG_DIR = 3 };
// INIT: (a=x, b=r, c=z, d=p, e=g);  DOT: (a, b) -> partials;
// STEP: (a=x, b=r, c=z, d=p, e=Ap, s1=rz, s2=pq);  DIR: (a=p, c=z, s1=rz_new, s2=rz_old)
template <typename T>
cudaError_t launch_pcg(int which, const PcgParams& q, T* a, T* b, T* c, T* d, const T* e,
                       const double* s1, const double* s2, cudaStream_t st);

// Kernel-launch counter behind wvl_kernel_launches().
void count_launches(unsigned long long k);
// Status with a detail string for wvl_last_error() (thread-local), and its reset.
wvl_status set_error(wvl_status s, const char* msg);
void clear_error();

// ekin/epot finalisation and density reduction.
cudaError_t launch_reduce_parts(const double* part, const double* minus, int tiles,
                                int norb, double* out, cudaStream_t st);
cudaError_t launch_rho_reduce(const double* parts, long long P, int ngroups,
                              double* rho, cudaStream_t st);
// several reduce_parts sums in one launch: task k covers warps
// warp0 .. warp0 + norb - 1, out[o] = sum part[o][*] - sum mpart[o][*]
struct PartTask {
    const double* part;
    const double* mpart;  // null: nothing subtracted
    double* out;
    int tiles, mtiles, norb, warp0;
};
constexpr int MAXTASK = 2 * MAXSEG;
struct PartTasks {
    PartTask t[MAXTASK];
    int ntask = 0;
    int nwarps = 0;
    // append a task; false when the table is full
    bool add(const double* part, int tiles, const double* mpart, int mtiles, double* out, int norb) {
        if (ntask >= MAXTASK) return false;
        t[ntask] = PartTask{part, mpart, out, tiles, mtiles, norb, nwarps};
        ++ntask;
        nwarps += norb;
        return true;
    }
};
cudaError_t launch_reduce_parts_multi(const PartTasks& t, cudaStream_t st);
// E_loc = sum_o occ (ekin + epot) into *out (one fixed-order CTA), and
// dV = gbar rho in the potential's precision (the adjoint of E_loc in V).
cudaError_t launch_eloc_total(const double* occ, const double* ekin, const double* epot,
                              int norb, double* out, cudaStream_t st);
template <typename T>
cudaError_t launch_scale_density(const double* rho, const double* gbar, long long P, T* dV,
                                 cudaStream_t st);

}  // namespace wvl
