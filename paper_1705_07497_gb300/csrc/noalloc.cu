// ct_cg_solve_noalloc: the single-slice CG solve of ct_cg_solve, run on a
// fixed scratch area that is part of the library image, so the call itself
// never allocates device memory.  The paper has no counterpart; this exists
// for callers that cannot allocate (see include/ct.h).
//
// The scratch is one file-scope __device__ array.  Every device that loads
// the library holds it until the process exits.  Host code cannot use the
// array's name as a device address (on the host it names a stand-in object),
// so the address is asked of the runtime with cudaGetSymbolAddress, with the
// device current.  The runtime loads a module's device image (and with it
// backs this array) on its first use, so the matrix builders ask for the
// address once on the handle's device, where allocating is allowed; every
// call asks again (cheap once the image is loaded), so no address outlives a
// device reset.
#include <algorithm>
#include <string>

#include "ct_internal.cuh"

namespace ct {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CT_NOALLOC_SCRATCH_BYTES];

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device.
int scratch_address(unsigned char** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return fail(CT_ERR_OOM, "the device has no room for the allocation-free scratch array (" +
                                    std::to_string((size_t)CT_NOALLOC_SCRATCH_BYTES) + " bytes)");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
    *out = static_cast<unsigned char*>(p);
    return CT_OK;
}

// Byte layout of the scratch for one solve: five image vectors, the sinogram
// temp, reduction partials, the block counter and the CG scalars.
struct Layout {
    size_t vec, y, partials, counter, cg, total;
};

Layout layout_for(const ct_matrix* M)
{
    Layout L;
    const size_t n2 = (size_t)M->npad, rows = (size_t)M->rows;
    // two partials per block of the widest reduction (the fused adjoint: one block per tile)
    const size_t nparts = std::max((size_t)4 * (M->sm_count > 0 ? M->sm_count : 148) * 8,
                                   (size_t)2 * M->tn * M->tn);
    L.vec = round256(n2 * sizeof(float2));
    L.y = round256(rows * sizeof(float2));
    L.partials = round256(nparts * sizeof(float2));
    L.counter = 256;
    L.cg = round256(sizeof(CgSlice));
    L.total = 5 * L.vec + L.y + L.partials + L.counter + L.cg;
    return L;
}

bool on_device(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// Commits the scratch array on the current device (loads this file's device
// image).  Called by the matrix builders, where allocating is allowed; a
// failure is left for ct_cg_solve_noalloc to report.
void noalloc_reserve()
{
    unsigned char* p = nullptr;
    if (scratch_address(&p) != CT_OK) {
        (void)cudaGetLastError();
        set_error("");
    }
}

}  // namespace ct

using namespace ct;

extern "C" int ct_cg_solve_noalloc(ct_matrix_t A, const ct_cg_params* params, const float* rhs, float* u,
                                   ct_cg_stats* stats, void* cuda_stream)
{
    if (!A) return fail(CT_ERR_ARG, "NULL matrix handle");
    if (!params) return fail(CT_ERR_ARG, "NULL params");
    if (params->max_iters < 0) return fail(CT_ERR_ARG, "max_iters < 0");
    if (params->surrogate_r != 0)
        return fail(CT_ERR_UNSUPPORTED, "ct_cg_solve_noalloc supports the exact operator only (surrogate_r = 0)");
    int dev = -1;
    CT_CUDA(cudaGetDevice(&dev));
    if (dev != A->device) return fail(CT_ERR_ARG, "matrix lives on another device than the current one");
    if (!rhs || !u || !on_device(rhs) || !on_device(u))
        return fail(CT_ERR_ARG, "ct_cg_solve_noalloc needs device pointers for rhs and u");
    const Layout L = layout_for(A);
    if (L.total > (size_t)CT_NOALLOC_SCRATCH_BYTES)
        return fail(CT_ERR_ARG, "problem needs " + std::to_string(L.total) + " bytes of scratch; the limit is " +
                                    std::to_string((size_t)CT_NOALLOC_SCRATCH_BYTES) + " (CT_NOALLOC_SCRATCH_BYTES)");
    unsigned char* base = nullptr;
    CT_CHECK(scratch_address(&base));
    Workspace w;
    w.batch = 1;
    w.n2 = A->npad;
    w.rows = A->rows;
    unsigned char* at = base;
    float2** vecs[] = {&w.u, &w.r, &w.p, &w.q, &w.rhs};
    for (float2** v : vecs) {
        *v = reinterpret_cast<float2*>(at);
        at += L.vec;
    }
    w.y = reinterpret_cast<float2*>(at);
    at += L.y;
    w.partials = reinterpret_cast<float2*>(at);
    w.partials_len = (int64_t)(L.partials / sizeof(float2));
    at += L.partials;
    w.counter = reinterpret_cast<unsigned*>(at);
    at += L.counter;
    w.cg = reinterpret_cast<CgSlice*>(at);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the block counter must start at zero; everything else is written before it is read
    CT_CUDA(cudaMemsetAsync(w.counter, 0, L.counter, st));
    return cg_solve_in(A, w, params, rhs, u, stats, st);
}
