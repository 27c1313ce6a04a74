/*
 * wvl.h -- C ABI of the GB300 local-Hamiltonian library for Daubechies-16
 * wavelets in periodic boundary conditions (Genovese et al., "Density
 * Functional Theory calculation on many-cores hybrid CPU-GPU architectures").
 *
 * Method (paper, Sec. "Full local hamiltonian"): for each orbital
 *   1) decompression, 2) wavelet synthesis to the fine scaling basis
 *   (Eq. wavefhigh), 3a) magic filter (Eq. magicfilter), 3b) V*psi,
 *   3c) transposed magic filter, 4) kinetic convolution (Eqs. kiner, fprod)
 *   on the output of 2), 5) sum, 6) analysis, 7) compression;
 * plus the density rho += occ |psi_r|^2 (Eq. density, Sec. "Local density
 * calculation") and the energies Ekin = <s, -1/2 Lap s>, Epot = sum V psi_r^2.
 * Every 3D convolution is three 1D periodic "convolve + transpose" passes
 * (Eqs. 3dconv, 1dconvtrans, kinetic1d).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: coarse n1 x n2 x n3 points (n_d >= 1), fine N_d = 2 n_d, fine spacing
 *   h'_d (kinetic scale -1/(2 h'_d^2)); P = N1 N2 N3 fine points per orbital.
 * Arrays are C-ordered with x fastest: fine arrays are [N3][N2][N1].
 * Compressed coefficients (8 n1 n2 n3 values per orbital): the scaling block
 *   c^0[i3][i2][i1] followed by the wavelet block c^mu[i3][i2][i1][mu-1],
 *   mu = a1 + 2 a2 + 4 a3 = 1..7 (a_d = 1 selects the wavelet along axis d).
 * Orbitals of one call are contiguous, orbital o at offset o * 8 n1 n2 n3
 *   (compressed) or o * P (fine).
 * Precision: WVL_F64 -- every array is double.  WVL_F32 -- coefficient, fine
 *   and potential arrays are float, and so are the convolutions; rho, occ and
 *   energies stay double.  Energies accumulate in double: each term is an
 *   FP32 chain of at most 32 products of convolution outputs, converted
 *   exactly (the fused potential kernel first sums a warp's 32 chains in a
 *   compensated single pair, ~48-bit); scalar products (wvl_overlap,
 *   wvl_dot) form every product and sum in double; rho over orbitals is
 *   carried per thread in compensated single (~48-bit) and in double from
 *   there on.
 *   WVL_F64_EMU -- arrays as WVL_F64; every 1D convolution sum of the
 *   passes (Eqs. 1dconvtrans, kinetic1d) is evaluated on the FP16 tensor
 *   cores instead of the FP64 pipe: operands split into six signed 10-bit
 *   digits on a per-line (data) and per-filter (taps) power-of-two scale,
 *   digit products summed exactly in FP32 accumulators, recombined in
 *   64-bit integers.  The error per convolution is below 2^-52 of
 *   max|f| max|x| over the line (the order of FP64 rounding); pointwise
 *   steps and reductions are FP64.  All entry points that take `prec`
 *   accept it; the preconditioner's CG vector updates stay FP64.
 * Memory: every data pointer is DEVICE memory owned by the caller and must be
 *   16-byte aligned; the library allocates nothing on these calls.  Scratch
 *   space is the caller's workspace `ws` of `ws_bytes` bytes, at least
 *   wvl_workspace_size(); its contents are clobbered.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream); every
 *   call only enqueues work and returns without synchronising.  Calls on the
 *   same stream are ordered; calls sharing a workspace must not overlap.
 * rho is ACCUMULATED (+=); energies are WRITTEN, one double per orbital.
 * Errors: arguments are validated on the host before anything is enqueued;
 *   on error nothing is enqueued, the status is returned and a detail string
 *   is available from wvl_last_error() (thread-local).  Launch failures are
 *   returned as WVL_ECUDA.  No call traps, asserts on the device or throws.
 */
#ifndef WVL_H
#define WVL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WVL_OK = 0,
    WVL_EINVAL = 1,        /* bad argument: null, size, misalignment      */
    WVL_ENOMEM_WS = 2,     /* workspace smaller than required             */
    WVL_ECUDA = 3,         /* a CUDA runtime call failed                  */
    WVL_ETIMEOUT = 4,      /* a bounded device-side wait gave up          */
    WVL_EUNSUPPORTED = 5   /* size or option outside what is implemented  */
} wvl_status;

typedef enum { WVL_F64 = 0, WVL_F32 = 1, WVL_F64_EMU = 2 } wvl_prec;

/* Coarse grid and fine spacing h'_d = h_d / 2 (paper Eq. wavefhigh). */
typedef struct {
    int n1, n2, n3;
    double h1, h2, h3;
} wvl_grid;

/* Largest fine extent N_d = 2 n_d a 1D pass keeps in shared memory. */
#define WVL_MAX_FINE 1024

const char* wvl_status_string(int status);
const char* wvl_last_error(void);
int wvl_version(void);

/* Number of CUDA devices visible to the library (0 without a GPU); host only. */
int wvl_device_count(void);

/* Running count of kernels this library has enqueued in this process: direct
 * launches plus every kernel node of each replayed plan graph. */
unsigned long long wvl_kernel_launches(void);

/* Bounded device-side waits that gave up since the previous call (the
 * tensor-core passes of WVL_F64_EMU wait on their MMAs for at most ~2 s;
 * on expiry the kernel stops, leaves its outputs incomplete and counts it
 * here).  Synchronises the current device.  No counterpart in the paper.
 * Returns WVL_ETIMEOUT when the count is nonzero, WVL_OK otherwise. */
wvl_status wvl_wait_timeouts(unsigned* count);

/* Self-test of that expiry path: enqueues one kernel whose bounded wait (an
 * mbarrier nothing arrives on) gives up after about `ms` milliseconds of
 * SM clock and counts one expiry, so that wvl_wait_timeouts() then reports
 * WVL_ETIMEOUT with count 1.  No fault, no hang; the context stays usable.
 * No counterpart in the paper.  WVL_EINVAL unless 0 < ms <= 10000. */
wvl_status wvl_selftest_timeout(double ms, void* stream);

/* Arithmetic-pipe peak of the current device, measured: independent FMA
 * chains (packed pairs in FP32) on every SM; of the variants with 4, 8 or 16
 * chains per thread and 1, 2, 4 or 8 CTAs of 256 threads per SM, the fastest
 * is run for about `seconds` (0 < seconds <= 10), best of three launches
 * timed with CUDA events on `stream`.  *tflops = 2 x FMAs / s / 1e12 for prec WVL_F64 or
 * WVL_F32; *ms (nullable) = that launch's duration.  Synchronises the
 * stream.  The denominator of the library's FP64 and FP32 rooflines; no
 * counterpart in the paper. */
wvl_status wvl_fma_peak(int prec, double seconds, double* tflops, double* ms, void* stream);

/*
 * Filters derived by the library (host computation, no GPU needed), FP64.
 *  h[16], g[16]: h_j, g_j for j = -7..8 (Eq. refinement, g_j = (-1)^j h_{1-j});
 *  w[16], *k0: magic filter w_k for k = k0..k0+15 (Eq. magicfilter);
 *  a[29]: a_l = int phi phi''(x-l) dx for l = -14..14, so that the 1D
 *         kinetic filter of Eq. (fprod) along axis d is T_l = -a_l/(2 h'_d^2).
 * Any pointer may be NULL.
 */
wvl_status wvl_filters(double* h, double* g, double* w, int* k0, double* a);

/* Workspace bytes sufficient for every entry point below on `grid` with
 * `norb` orbitals in precision `prec`. */
wvl_status wvl_workspace_size(const wvl_grid* grid, int prec, int norb,
                              size_t* bytes);

/* Steps 1)+2): compressed coefficients -> fine scaling coefficients s
 * (fast wavelet synthesis, Sec. "Daubechies basis and wavelet
 * transformation"): psi_c [norb][8 n1 n2 n3] -> s [norb][N3][N2][N1]. */
wvl_status wvl_synthesis(const wvl_grid* grid, int prec, int norb,
                         const void* psi_c, void* s,
                         void* ws, size_t ws_bytes, void* stream);

/* Steps 6)+7): the transpose (inverse) of wvl_synthesis:
 * z [norb][N3][N2][N1] -> psi_c [norb][8 n1 n2 n3]. */
wvl_status wvl_analysis(const wvl_grid* grid, int prec, int norb,
                        const void* z, void* psi_c,
                        void* ws, size_t ws_bytes, void* stream);

/* Step 3a), Eq. (3dconv): psi_r(I) = sum_j w_j1 w_j2 w_j3 s(I - j);
 * s, psi_r: [norb][N3][N2][N1]. */
wvl_status wvl_magicfilter(const wvl_grid* grid, int prec, int norb,
                           const void* s, void* psi_r,
                           void* ws, size_t ws_bytes, void* stream);

/* Step 3c): the transposed magic filter, y(J) = sum_j w w w y_r(J + j). */
wvl_status wvl_magicfilter_T(const wvl_grid* grid, int prec, int norb,
                             const void* y_r, void* y,
                             void* ws, size_t ws_bytes, void* stream);

/* Step 4) (+5) through K_0, Sec. "Kinetic convolution", Eq. (kinetic1d)):
 * out = K0 + (-1/2 Lap) s, with K0 = 0 when k0 is NULL;
 * ekin[o] = <s_o, (-1/2 Lap) s_o> when ekin is not NULL (device, double). */
wvl_status wvl_kinetic(const wvl_grid* grid, int prec, int norb,
                       const void* s, const void* k0, void* out, double* ekin,
                       void* ws, size_t ws_bytes, void* stream);

/* Sec. "Local density calculation": steps 1), 2), 3a) then
 * rho[N3][N2][N1] += sum_o occ[o] psi_r,o^2 (grid units).  occ: device
 * double[norb]; rho: device double, accumulated. */
wvl_status wvl_density(const wvl_grid* grid, int prec, int norb,
                       const void* psi_c, const double* occ, double* rho,
                       void* ws, size_t ws_bytes, void* stream);

/* The whole local Hamiltonian of Sec. "Full local hamiltonian" for norb
 * orbitals of one cell: hpsi_c = A^T (M^T V M + K) A psi_c, with the density
 * of step 3a) accumulated into rho when rho is not NULL, and per-orbital
 * ekin[o] = <s, -1/2 Lap s>, epot[o] = sum_I V psi_r^2 (device doubles,
 * written).  V: [N3][N2][N1] in the orbital precision. */
wvl_status wvl_hpsi_local(const wvl_grid* grid, int prec, int norb,
                          const void* psi_c, const void* V, const double* occ,
                          void* hpsi_c, double* rho, double* ekin, double* epot,
                          void* ws, size_t ws_bytes, void* stream);

/* wvl_hpsi_local without a workspace argument.  The paper has no
 * counterpart: this is for callers that cannot give the library scratch
 * memory or let anything allocate device memory when they call it -- plugins
 * whose host program owns every device allocation, and pipelines that
 * reserve all device memory up front and forbid allocation later.
 * The scratch is one file-scope device array of WVL_NOALLOC_SCRATCH_BYTES,
 * held on every GPU that loads the library until the process exits; no
 * allocator is called.  Calls whose wvl_workspace_size() exceeds it return
 * WVL_EUNSUPPORTED.  On any failure wvl_noalloc_last_error() gives the
 * detail (also that of errors raised by the inner wvl_hpsi_local call).
 * Every call looks up the array's device address in the calling thread's
 * current device and context (cudaGetSymbolAddress), so switching devices,
 * driver-API contexts or a cudaDeviceReset between calls is safe; the first
 * call in a context loads the library's device code there, so make that
 * first call before any stream capture.  Every call uses the same array and leaves its contents behind
 * (nothing in it needs to start at zero); calls that overlap on the GPU --
 * on different streams or from several host threads -- race on it.
 * Arguments, layouts and results are those of wvl_hpsi_local. */
#define WVL_NOALLOC_SCRATCH_BYTES (64u << 20)
wvl_status wvl_hpsi_local_noalloc(const wvl_grid* grid, int prec, int norb,
                                  const void* psi_c, const void* V,
                                  const double* occ, void* hpsi_c, double* rho,
                                  double* ekin, double* epot, void* stream);
const char* wvl_noalloc_last_error(void);

/* Forward of E_loc = sum_o occ_o (Ekin_o + Epot_o): the energies (and rho
 * when not NULL) without H psi -- steps 1), 2), 3a), 3b) and 4) only. */
wvl_status wvl_energy(const wvl_grid* grid, int prec, int norb,
                      const void* psi_c, const void* V, const double* occ,
                      double* rho, double* ekin, double* epot,
                      void* ws, size_t ws_bytes, void* stream);

/* The differentiable local energy E_loc(psi, V) = sum_o occ_o (Ekin_o + Epot_o)
 * (Sec. "Full local hamiltonian"; Sec. "Local density calculation" for rho).
 * wvl_eloc is its forward: wvl_energy, then the total written to *eloc
 * (device double, one fixed-order reduction on the device).  ekin, epot:
 * device double[norb], written; rho nullable, accumulated.
 * wvl_eloc_backward is its adjoint for an upstream gradient *gbar (device
 * double):
 *   dpsi_c[o] = 2 occ_o gbar (H psi)_o   -- E_loc is quadratic in psi with the
 *       symmetric operator H = A^T (M^T V M + K) A; the whole chain runs again
 *       (real-space orbitals recomputed, not stored) and its last pass writes
 *       the scaled result in psi's precision and layout;
 *   dV = gbar rho                         -- E_loc is linear in V with
 *       coefficient rho (grid units); rho is the forward's density (device
 *       double), dV is written in V's precision, [N3][N2][N1].
 * Either output may be NULL (not computed); rho is required when dV is given.
 * Workspace: wvl_workspace_size(). */
wvl_status wvl_eloc(const wvl_grid* grid, int prec, int norb,
                    const void* psi_c, const void* V, const double* occ,
                    double* rho, double* ekin, double* epot, double* eloc,
                    void* ws, size_t ws_bytes, void* stream);
wvl_status wvl_eloc_backward(const wvl_grid* grid, int prec, int norb,
                             const void* psi_c, const void* V, const double* occ,
                             const double* rho, const double* gbar,
                             void* dpsi_c, void* dV,
                             void* ws, size_t ws_bytes, void* stream);

/* Orbital scalar products in compressed form (Sec. "Daubechies basis and
 * wavelet transformation": the basis functions of Eq. wavef0 are
 * orthonormal, so <psi_i|psi_j> is the sum of the products of the
 * coefficients, taken on the compressed vectors).  Precision `prec` gives the
 * element type of a and b (float for WVL_F32, else double); every product is
 * formed in FP64 (an FP32 x FP32 product is exact there) and accumulated in
 * FP64 by a fixed-order two-stage reduction, so repeated calls give
 * identical results.
 *   wvl_overlap: S[i][j] = <a_i|b_j>, a: [na][len], b: [nb][len] (device),
 *     S: device double [na][nb], written.  When a == b and na == nb only the
 *     upper block triangle is computed and mirrored.
 *   wvl_dot: d[o] = <a_o|b_o> for o < n (norms, <psi|H psi>), d: device
 *     double[n], written.
 * len may be any compressed length (full grid 8 n1 n2 n3, or a region's
 * ncoarse + 7 nfine).  Workspace: wvl_overlap_workspace_size() (enough for
 * both calls with these sizes). */
wvl_status wvl_overlap_workspace_size(int prec, int na, int nb, long long len, size_t* bytes);
wvl_status wvl_overlap(int prec, int na, const void* a, int nb, const void* b, long long len,
                       double* S, void* ws, size_t ws_bytes, void* stream);
wvl_status wvl_dot(int prec, int n, const void* a, const void* b, long long len, double* d,
                   void* ws, size_t ws_bytes, void* stream);

/* Preconditioning step (paper Eq. precon, Sec. "Kinetic convolution" with
 * K_0 = -eps s): for each orbital o, ncg iterations of the preconditioned
 * conjugate gradient for
 *     A x = g,   A = S^T (-1/2 Lap - eps_o) S   (S = synthesis, orthogonal)
 * on compressed coefficients, from x_0 = 0, with the diagonal of A (one value
 * per component mu, by translation invariance) as preconditioner.
 * g, x: device [norb][8 n1 n2 n3] (must not alias); eps: device double[norb],
 * each eps_o < 0 so that A is positive definite; rr (nullable, device
 * double[norb]) receives the final squared residual |g - A x|^2.
 * Workspace: wvl_precondition_workspace_size().  All scalars of the
 * iteration stay on the device: nothing synchronises with the host. */
wvl_status wvl_precondition_workspace_size(const wvl_grid* grid, int prec, int norb,
                                           size_t* bytes);
wvl_status wvl_precondition(const wvl_grid* grid, int prec, int norb, const void* g,
                            const double* eps, int ncg, void* x, double* rr,
                            void* ws, size_t ws_bytes, void* stream);

/* Free (isolated) boundary conditions (the paper's GPU code is periodic; its
 * CPU convolutions also admit isolated conditions, Sec. "Wavelet
 * transformation and Magic Filters convolutions"): the orbital's basis
 * functions are those of the coarse points of the box `grid` (n1 x n2 x n3),
 * with the compressed layout of the periodic entry points on that box, and
 * every operator acts on the whole space -- input arrays are zero outside,
 * outputs extend beyond the box.  V and rho cover the box plus
 * WVL_FREE_PAD coarse points (2 WVL_FREE_PAD fine points) on every side:
 * fine extents 2 (n_d + 2 WVL_FREE_PAD), index 0 at fine coordinate
 * -2 WVL_FREE_PAD.  H couples coarse points at most 15 apart, so the
 * periodic operator on that padded cell, restricted to the box, is the
 * free-space operator exactly; that is how it is computed. */
#define WVL_FREE_PAD 8
/* Mixed conditions: free_axes (HOST int[3], x y z) = 1 for a free axis, 0 for
 * a periodic one; padding (and the extent of V and rho) grows only along the
 * free axes.  One free axis = the surface (slab) conditions of the CPU code;
 * three = wvl_hpsi_local_free; none = wvl_hpsi_local. */
wvl_status wvl_bc_workspace_size(const wvl_grid* grid, const int* free_axes, int prec,
                                 int norb, size_t* bytes);
wvl_status wvl_hpsi_local_bc(const wvl_grid* grid, const int* free_axes, int prec, int norb,
                             const void* psi_c, const void* V, const double* occ,
                             void* hpsi_c, double* rho, double* ekin, double* epot,
                             void* ws, size_t ws_bytes, void* stream);
wvl_status wvl_density_bc(const wvl_grid* grid, const int* free_axes, int prec, int norb,
                          const void* psi_c, const double* occ, double* rho,
                          void* ws, size_t ws_bytes, void* stream);
wvl_status wvl_free_workspace_size(const wvl_grid* grid, int prec, int norb, size_t* bytes);
wvl_status wvl_hpsi_local_free(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                               const void* V, const double* occ, void* hpsi_c, double* rho,
                               double* ekin, double* epot, void* ws, size_t ws_bytes,
                               void* stream);
wvl_status wvl_density_free(const wvl_grid* grid, int prec, int norb, const void* psi_c,
                            const double* occ, double* rho, void* ws, size_t ws_bytes,
                            void* stream);

/* Localisation regions of the compressed form (paper Sec. "Daubechies basis
 * and wavelet transformation", Eq. wavef0: the scaling sum runs over the
 * low-resolution region, the wavelet sum over the generally smaller
 * high-resolution region, and only those coefficients are stored).
 * An orbital's compressed vector then holds ncoarse scaling coefficients
 * (coarse-region points in lexicographic order, i1 fastest) followed by
 * nfine groups of the 7 wavelet coefficients (fine-region points in the
 * same order, mu = 1..7 fastest); orbital o starts at o (ncoarse + 7 nfine).
 * coarse_index, fine_index: DEVICE int32 [n3][n2][n1]; coarse_index[p] is
 * the position of c^0 of coarse point p, fine_index[p] = k such that c^mu
 * sits at ncoarse + 7 k + mu - 1; -1 off the region.  Off-region
 * coefficients are zero on input and dropped on output (H is restricted to
 * the region: P^T H P). */
typedef struct {
    const int* coarse_index;
    const int* fine_index;
    long long ncoarse, nfine;
    /* Optional periodic bounding box of the region (wvl_region_bounds):
     * along axis d every region point has a coarse coordinate in
     * lo[d] .. lo[d] + len[d] - 1 (mod n_d).  len[d] = 0: not given.  Along
     * axes where len[d] <= n_d - 15 the chain is computed on that box plus
     * the supports its filters reach (no periodic image of the box couples
     * to it), so the work shrinks with the region; results are the same. */
    int lo[3], len[3];
} wvl_region;

/* Host helper: index arrays (HOST int32 [n1 n2 n3]) and counts from two
 * HOST masks (uint8 [n3][n2][n1], nonzero = in the region). */
wvl_status wvl_region_index(const wvl_grid* grid, const unsigned char* coarse_mask,
                            const unsigned char* fine_mask, int* coarse_index,
                            int* fine_index, long long* ncoarse, long long* nfine);

/* Host helper: the smallest periodic bounding box (lo, len: HOST int[3]) of
 * the union of the two masks, per axis the complement of the longest
 * periodic run of coordinates no region point occupies (len 0: empty). */
wvl_status wvl_region_bounds(const wvl_grid* grid, const unsigned char* coarse_mask,
                             const unsigned char* fine_mask, int* lo, int* len);

/* The entry points above, with region-compressed coefficient arrays. */
wvl_status wvl_synthesis_region(const wvl_grid* grid, const wvl_region* region, int prec,
                                int norb, const void* psi_c, void* s,
                                void* ws, size_t ws_bytes, void* stream);
wvl_status wvl_analysis_region(const wvl_grid* grid, const wvl_region* region, int prec,
                               int norb, const void* z, void* psi_c,
                               void* ws, size_t ws_bytes, void* stream);
wvl_status wvl_density_region(const wvl_grid* grid, const wvl_region* region, int prec,
                              int norb, const void* psi_c, const double* occ, double* rho,
                              void* ws, size_t ws_bytes, void* stream);
wvl_status wvl_hpsi_local_region(const wvl_grid* grid, const wvl_region* region, int prec,
                                 int norb, const void* psi_c, const void* V,
                                 const double* occ, void* hpsi_c, double* rho,
                                 double* ekin, double* epot,
                                 void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Batched plans: many orbitals on cells of different sizes in one enqueue
 * (the paper's orbital distribution, Sec. "Parallel distribution", inside
 * one GPU).  Orbital o lives on cell cell_of_orb[o]; orbitals are stored one
 * after another in the given order, each with its own cell's size.  Runs of
 * consecutive orbitals on the same cell form one segment of each launch.
 * ---------------------------------------------------------------------- */
typedef struct wvl_plan wvl_plan;

#define WVL_PLAN_GRAPH    1u   /* replay a captured CUDA graph when pointers repeat */
#define WVL_PLAN_AUTOTUNE 2u   /* wvl_plan_autotune may time kernel variants */
/* Which kernels apply the local Hamiltonian (at most one of the two; neither:
 * the fused kernels for WVL_F32 where every cell allows them, else the 1D
 * passes, and wvl_plan_autotune times both and keeps the faster):
 *   WVL_PLAN_FUSED  five kernels that keep a fine-grid plane (axes 1, 2) or
 *                   N3 x 128-byte column tiles (axis 3) in shared memory across
 *                   several 1D filters of the chain (Sec. "Three dimensional
 *                   operators": each 3D operator is three commuting 1D ones;
 *                   the wavelet transform is orthogonal along each axis).
 *                   Results equal the passes' up to rounding.
 *                   Needs WVL_F64 or WVL_F32 and every fine extent 2 n_d a
 *                   multiple of 8 in [32, 128] (FP64: planes up to ~112 x 112);
 *                   otherwise wvl_plan_create returns WVL_EUNSUPPORTED.
 *   WVL_PLAN_PASSES the fifteen transposing 1D passes (Eq. 1dconvtrans). */
#define WVL_PLAN_FUSED    4u
#define WVL_PLAN_PASSES   8u

/* Host-side; allocates the plan (host memory only).  cells[ncell],
 * cell_of_orb[norb] are host arrays copied into the plan. */
wvl_status wvl_plan_create(const wvl_grid* cells, int ncell,
                           const int* cell_of_orb, int norb, int prec,
                           unsigned flags, wvl_plan** out);
wvl_status wvl_plan_destroy(wvl_plan* plan);
wvl_status wvl_plan_workspace_size(const wvl_plan* plan, size_t* bytes);
/* Element offset of orbital o in the concatenated compressed array. */
wvl_status wvl_plan_orbital_offset(const wvl_plan* plan, int o, size_t* offset);

/* Local Hamiltonian of every orbital of the plan.  psi, hpsi: concatenated
 * compressed orbitals (device); V, rho: HOST arrays of ncell DEVICE pointers
 * (rho entries may be NULL: no density for that cell); occ, ekin, epot:
 * device double[norb]. */
wvl_status wvl_plan_hpsi(wvl_plan* plan, const void* psi,
                         const void* const* V, const double* occ, void* hpsi,
                         double* const* rho, double* ekin, double* epot,
                         void* ws, size_t ws_bytes, void* stream);

/* Times the kernel variants of every pass of wvl_plan_hpsi on the given
 * buffers (their contents are overwritten) and keeps the fastest for later
 * calls.  Synchronises the stream.  Needs WVL_PLAN_AUTOTUNE. */
wvl_status wvl_plan_autotune(wvl_plan* plan, const void* psi,
                             const void* const* V, const double* occ,
                             void* hpsi, double* const* rho, double* ekin,
                             double* epot, void* ws, size_t ws_bytes,
                             void* stream);

/* Human-readable choice of the autotuner (or the defaults), one line per
 * pass; copies at most len-1 characters. */
wvl_status wvl_plan_describe(const wvl_plan* plan, char* buf, size_t len);

/* Tracing: when on, every stage of wvl_plan_hpsi is bracketed by CUDA
 * events on the launching stream (graph replay is then bypassed).
 * wvl_plan_profile() synchronises those events and returns, per stage, the
 * summed milliseconds and the launch count since the last read, then
 * clears them.  Stages: 0 synthesis, 1 magic filter + potential/density,
 * 2 transposed magic filter, 3 kinetic, 4 analysis, 5 reductions. */
#define WVL_NSTAGE 6
wvl_status wvl_plan_set_profiling(wvl_plan* plan, int on);
wvl_status wvl_plan_profile(wvl_plan* plan, double* ms, int* launches,
                            int nstage);

#ifdef __cplusplus
}
#endif
#endif /* WVL_H */
