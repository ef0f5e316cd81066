// noalloc.cu -- fhe_relinearise_noalloc: relinearisation whose scratch comes
// from a fixed device array instead of the context workspace.
//
// Who needs it: callers that must not allocate device memory at call time --
// for instance a serving loop whose device memory is fully owned by another
// allocator (a framework's caching pool), or code that must not pay for, or
// wait on, the device-wide synchronisation that growing a workspace with
// cudaMalloc / cudaFree can cause.  fhe_relinearise grows the context
// workspace on demand; this variant never does.
//
// The scratch is the file-scope array below: kNoAllocScratchBytes on every
// GPU that loads the library, held until the process exits.  Host code may not
// use the array's name as a device address (on the host it names a host-side
// stand-in), so the first call on each device looks the device address up
// with cudaGetSymbolAddress while that device is current, and passes that
// address to the kernels.  Under lazy module loading (CUDA's default) that
// lookup is also what loads the module on the device and reserves the array,
// so the first call can allocate (and fail for lack of device memory); make
// one warm-up call per device before another allocator takes the memory and
// before any stream capture.  All calls share the array and it keeps the previous call's
// contents; the relinearisation kernels write every scratch word before they
// read it, so nothing has to be cleared.  Calls whose work overlaps on the GPU
// (two streams, or two threads) race on the array: serialise them.
#include <mutex>
#include <string>

#include "../../include/fhe.h"
#include "ctx.h"

using namespace fhe;

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;    // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

int scratch_for_current_device(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(FHE_EUNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return FHE_OK;
}

}  // namespace

extern "C" int fhe_relinearise_noalloc(fhe_ctx* c, const uint64_t* d3, uint32_t n_ct, uint32_t level, uint64_t* d_out,
                                       void* stream)
{
    if (!c) return fail(FHE_EINVAL, "null context");
    if (!c->has_keys) return fail(FHE_ENOKEY, "fhe_keygen has not run");
    if (level < 1 || level > c->L_top) return fail(FHE_ELEVEL, "level out of range");
    if (n_ct == 0) return FHE_OK;
    if (!d3 || !d_out) return fail(FHE_EINVAL, "null buffer");
    if (c->N > kMaxSinglePassN) return fail(FHE_EUNSUPPORTED, "fhe_relinearise_noalloc supports N <= 16384");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev != c->device) return fail(FHE_EINVAL, "make the context's device current before this call");
    const size_t need = relin_scratch_bytes(c, n_ct, level);
    if (need > kNoAllocScratchBytes)
        return fail(FHE_EINVAL, "fhe_relinearise_noalloc: this batch needs " + std::to_string(need) +
                                    " bytes of scratch; the fixed area holds " +
                                    std::to_string(kNoAllocScratchBytes) + " (use fewer ciphertexts per call)");
    void* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    // single-pass transforms only: the two-pass schedule would use the
    // context's intermediate buffer in addition to the fixed array
    k_relin(c, (const u64*)d3, (u64*)d_out, n_ct, level, scratch, (cudaStream_t)stream, nullptr, true);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, "relinearise_noalloc launch");
    return FHE_OK;
}
