// Allocation-free descriptor range.
//
// nep_descriptor_range() allocates a temporary buffer for the raw descriptors on every
// call.  Some callers cannot allocate device memory at that point: code that runs
// while a CUDA stream is being captured into a graph (cudaMalloc/cudaFree are not
// allowed there), code embedded in a host program whose memory manager owns all
// device allocations, and real-time loops that must not hit the driver's allocator.
// This entry point does the same work with its scratch in a fixed, file-scope device
// array instead, so the call itself allocates nothing.
#include <mutex>

#include "nep_ctx.cuh"

using namespace nep;

struct nep_ctx : public nep::Ctx {};

namespace {

// Scratch for the raw descriptors, [N_a][padded N_des] floats.  Every GPU that loads
// the library keeps this array for the life of the process.
constexpr size_t NOALLOC_QMAX = 8u * 1024u * 1024u;  // floats (32 MiB)
static __device__ __align__(256) float g_noalloc_q[NOALLOC_QMAX];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
float *g_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device;
// in host code the array's name is only a host-side stand-in, not a device address).
int scratch_address(Ctx *c, float **out) {
    if (c->dev < 0 || c->dev >= MAX_DEVICES) return c->fail(NEP_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[c->dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_q);
        if (e != cudaSuccess) return c->fail_cuda(e, "cudaGetSymbolAddress(descriptor scratch)");
        g_ptr[c->dev] = (float *)p;
    }
    *out = g_ptr[c->dev];
    return NEP_OK;
}

}  // namespace

extern "C" int nep_descriptor_range_noalloc(nep_ctx *c, float *qmin, float *qmax) {
    if (!c) return NEP_EINVAL;
    if (!c->have_batch) return c->fail(NEP_ESTATE, "no structures (call nep_set_structures)");
    if (!c->have_params) return c->fail(NEP_ESTATE, "no parameters (call nep_set_params)");
    if (!qmin || !qmax) return c->fail(NEP_EINVAL, "null output");
    if ((size_t)c->n_atoms * (size_t)c->NDP > NOALLOC_QMAX)
        return c->fail(NEP_EINVAL, "batch too large for the fixed descriptor scratch "
                                   "(atoms x padded descriptor length must be at most 8,388,608)");
    CK(cudaSetDevice(c->dev));
    float *q = nullptr;
    int rc = scratch_address(c, &q);
    if (rc) return rc;
    // Every scratch entry the range kernel reads is written by the forward's descriptor
    // stage in this same call, so nothing has to be cleared between calls.
    if ((rc = launch_expand(c))) return rc;
    if ((rc = launch_forward(c, q, 0))) return rc;
    return launch_range(c, q, qmin, qmax);
}
