// wvl_hpsi_local_noalloc: the local Hamiltonian with library-owned scratch.
//
// Some callers cannot hand the library a workspace or let anything allocate
// device memory when they call it: plugins whose host program owns and
// accounts for every device allocation, and fixed-memory pipelines that
// reserve all device memory at start-up and forbid allocation afterwards.
// For them this entry point keeps its scratch in one file-scope device array
// of a fixed size, reserved on every GPU that loads the library until the
// process exits, and calls no allocator at all.
#include <cstdio>
#include <cstring>

#include <cuda_runtime.h>

#include "wvl.h"

namespace {

constexpr size_t kScratchBytes = (size_t)WVL_NOALLOC_SCRATCH_BYTES;

// In host code this name is only a host-side stand-in; the kernels get the
// device address that cudaGetSymbolAddress returns for the current device
// and context.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

thread_local char g_msg[256];

}  // namespace

extern "C" const char* wvl_noalloc_last_error(void) { return g_msg; }

extern "C" wvl_status wvl_hpsi_local_noalloc(const wvl_grid* grid, int prec, int norb,
                                             const void* psi_c, const void* V,
                                             const double* occ, void* hpsi_c, double* rho,
                                             double* ekin, double* epot, void* stream) {
    g_msg[0] = 0;
    if (norb == 0) return WVL_OK;
    size_t need = 0;
    wvl_status st = wvl_workspace_size(grid, prec, norb, &need);
    if (st != WVL_OK) {
        std::snprintf(g_msg, sizeof g_msg, "wvl_hpsi_local_noalloc: %s", wvl_last_error());
        return st;
    }
    if (need > kScratchBytes) {
        std::snprintf(g_msg, sizeof g_msg,
                      "wvl_hpsi_local_noalloc: this grid and orbital count need %zu bytes of "
                      "scratch, more than the fixed %zu; use wvl_hpsi_local with a workspace",
                      need, kScratchBytes);
        return WVL_EUNSUPPORTED;
    }
    // The array's address belongs to the current device's context, so it is
    // looked up on every call (a host-side table lookup once the module is
    // loaded): a caller that switches devices, runs under its own driver
    // context or resets the device always gets the address valid for the
    // context it calls from.  The first lookup in a context loads the
    // library's device code there.
    void* scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&scratch, g_scratch);
    if (e != cudaSuccess || scratch == nullptr) {
        std::snprintf(g_msg, sizeof g_msg, "wvl_hpsi_local_noalloc: cudaGetSymbolAddress: %s",
                      cudaGetErrorString(e));
        return WVL_ECUDA;
    }
    // Nothing in the scratch has to start at zero: every word the chain reads
    // is first written by the same call.
    st = wvl_hpsi_local(grid, prec, norb, psi_c, V, occ, hpsi_c, rho, ekin, epot, scratch,
                        kScratchBytes, stream);
    if (st != WVL_OK)
        std::snprintf(g_msg, sizeof g_msg, "wvl_hpsi_local_noalloc: %s", wvl_last_error());
    return st;
}
