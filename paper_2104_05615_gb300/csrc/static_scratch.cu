// dwf_apply_packed_static: the global operators (D, D^+, D^+D) on packed
// fields with their three intermediate fields in a fixed, file-scope device
// array instead of memory the library allocates.
//
// Some callers cannot allocate device memory at the point where they apply the
// operator: code running inside a memory pool or arena that owns all device
// memory, callers that must not let a library touch the allocator while other
// work is in flight, and embedded or safety-certified hosts that forbid
// allocation after start-up.  This entry point serves them.  The price is a
// fixed block of device memory (kStaticScratchBytes) that every GPU which
// loads this library keeps until the process exits.
#include <mutex>

#include "engine.h"

namespace {

// 24 MiB: room for the three intermediate fields (each dwf_packed_bytes, one
// checkerboard) of lattices up to, e.g., 8^4 x Ls = 12 in FP32 (3 x 2.4 MB)
// or 12^4 x Ls = 12 in FP16 (3 x 6.5 MB); 12^4 x Ls = 12 in FP32 (3 x 11.9 MB)
// does not fit.
constexpr size_t kStaticScratchBytes = 24u << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};  // device address of g_static_scratch per device

// The device address of the array on the current device.  In host code the
// symbol is only a host-side stand-in, so its address must be looked up once
// per device, with that device current.  The address is kept for the life of
// the process: after cudaDeviceReset (or a release of the device's primary
// context) the module is loaded again and the kept address is stale, so this
// entry point must not be used across a device reset.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" dwf_status dwf_apply_packed_static(dwf_handle *h, void *out, const void *in,
                                              dwf_op op, dwf_prec prec, void *stream);

// Defined in api.cu: the handle's engine and error string.
dwf::Engine *dwf_handle_engine(dwf_handle *h);
void dwf_handle_set_error(dwf_handle *h, const char *msg);

extern "C" dwf_status dwf_apply_packed_static(dwf_handle *h, void *out, const void *in,
                                              dwf_op op, dwf_prec prec, void *stream)
{
    using namespace dwf;
    if (!h || !out || !in || out == in || prec < DWF_F64 || prec > DWF_FX8) return DWF_EINVAL;
    if (op != DWF_OP_D && op != DWF_OP_DDAG && op != DWF_OP_DDAGD) {
        dwf_handle_set_error(h, "static-scratch apply supports D, D^+ and D^+D only");
        return DWF_EINVAL;
    }
    Engine &E = *dwf_handle_engine(h);
    const size_t fb = (field_bytes((Prec)prec, E.ne, E.Ls) + 255) & ~size_t(255);
    if (3 * fb > kStaticScratchBytes) {
        dwf_handle_set_error(h, "lattice too large for the static scratch (3 fields > 24 MiB)");
        return DWF_EINVAL;
    }
    if (!E.global_ready((Prec)prec)) {
        dwf_handle_set_error(h, "call dwf_apply_packed once with this precision first "
                                "(it builds the link copies and launch configuration)");
        return DWF_EINVAL;
    }
    void *base = nullptr;
    cudaError_t ce = scratch_address(&base);
    if (ce != cudaSuccess) {
        dwf_handle_set_error(h, cudaGetErrorString(ce));
        return DWF_ECUDA;
    }
    void *scr[3] = {base, (char *)base + fb, (char *)base + 2 * fb};
    try {
        StreamSwap sw(E, stream);  // the handle's stream is restored on every exit path
        E.apply_global((Prec)prec, op, out, in, nullptr, scr);
    } catch (const CudaError &e) {
        dwf_handle_set_error(h, cudaGetErrorString(e.err));
        return e.err == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA;
    } catch (const std::exception &e) {
        dwf_handle_set_error(h, e.what());
        return DWF_EINVAL;
    }
    return DWF_OK;
}
