// Dhat (Eq. 2) on native fields with its odd-site intermediate held in a
// statically sized device array rather than the context's grow-on-demand
// workspace.  Callers that must not allocate device memory while they run
// (a driver that has given the rest of the device to its own pool, or one
// that cannot pay for the synchronisation cudaMalloc may imply) use this
// entry point; it launches the same two stencil kernels as
// lqcd_apply_Dhat_native.
#include <mutex>

#include "lqcd_internal.cuh"

namespace {

constexpr size_t kScratchBytes = LQCD_DHAT_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The odd-site intermediate: DHAT1 writes every odd site of every right-hand
// side before DHAT2 reads any, so the array needs no clearing.
static __device__ __align__(256) unsigned char g_dhat_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_dhat_scratch on the current device, looked up once per
// device (cudaGetSymbolAddress allocates nothing).
lqcd_status scratch_address(lqcd_ctx *c, void **out)
{
    int dev = -1;
    LQCD_CUDA_CHECK(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_err(c, LQCD_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dhat_scratch);
        if (e != cudaSuccess || !p)
            return set_err(c, LQCD_ERR_CUDA, "static Dhat scratch: cudaGetSymbolAddress failed: %s",
                           cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LQCD_OK;
}

}  // namespace

extern "C" lqcd_status lqcd_apply_Dhat_native_static(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, int nrhs)
{
    if (!c || !in || !out || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (p != LQCD_F64 && p != LQCD_F32 && p != LQCD_F16S)
        return set_err(c, LQCD_ERR_ARG, "static Dhat: precision %d is not a stencil precision", (int)p);
    const size_t need = native_half_bytes(c, p) * (size_t)nrhs;
    if (need > kScratchBytes)
        return set_err(c, LQCD_ERR_ARG,
                       "static Dhat scratch: %d right-hand side(s) at this lattice and precision need %zu bytes, "
                       "the fixed array holds %zu (at most %zu right-hand side(s))",
                       nrhs, need, kScratchBytes, kScratchBytes / native_half_bytes(c, p));
    void *tmp = nullptr;
    LQCD_TRY(scratch_address(c, &tmp));
    return dirac_dhat(c, p, in, out, tmp, nrhs);
}
