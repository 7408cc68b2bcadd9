// noalloc.cu -- a negacyclic product that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they call into
// the library: a serving thread that must not block or fail on cudaMalloc
// (cudaMalloc may synchronise the device and can run out of memory at any
// time), and code whose device memory is owned and accounted by a host
// framework or pool that forbids allocations behind its back.  fg_poly_mul
// needs scratch for the transformed operands and takes it from the
// context's workspace, which grows with cudaMalloc on first use.
// fg_poly_mul_noalloc does the same product with its scratch in a fixed
// array compiled into the library.
//
// The array below lives in every GPU that loads the library, for as long as
// the process runs.  Host code cannot use its name as a device address (the
// name denotes a host-side shadow), so the address is looked up with
// cudaGetSymbolAddress, once per device, with that device current.
#include <mutex>

#include "fg_internal.h"
#include "modarith.cuh"

namespace {

// Two operands of at most kNoAllocWords words each: (level + 1) * N <= 2^18,
// e.g. 16 limbs at N = 2^14, 4 limbs at N = 2^16.  4 MiB in total.
constexpr size_t kNoAllocWords = size_t(1) << 18;

static __device__ __align__(256) u64 g_noalloc_scratch[2 * kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
u64 *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device`.  The first call for a
// device makes that device current, looks the address up and restores the
// caller's device; later calls reuse the address.
u64 *noalloc_scratch(int device)
{
    FG_CHECK(device >= 0 && device < kMaxDevices, FG_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        int prev = 0;
        CUDA_TRY(cudaGetDevice(&prev));
        CUDA_TRY(cudaSetDevice(device));
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        cudaSetDevice(prev);
        if (e != cudaSuccess)
            throw fg_error(FG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[device] = (u64 *)p;
    }
    return g_noalloc_ptr[device];
}

// true when p is device (or managed) memory of GPU `device`
bool on_device(const void *p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

}  // namespace

extern "C" int fg_poly_mul_noalloc(fg_ctx *ctx, const uint64_t *a, const uint64_t *b, int level,
                                   uint64_t *c)
{
    if (!ctx) return FG_EINVAL;
    try {
        FG_CHECK(level >= 0 && level < ctx->nq, FG_ELEVEL, "level out of range");
        const int N = ctx->n, nl = level + 1;
        FG_CHECK((size_t)nl * N <= kNoAllocWords, FG_EINVAL,
                 "fg_poly_mul_noalloc: (level + 1) * N exceeds 2^18 words");
        const int dev = ctx->device;
        FG_CHECK(a && b && c && on_device(a, dev) && on_device(b, dev) && on_device(c, dev), FG_EINVAL,
                 "fg_poly_mul_noalloc takes device pointers on the context's GPU only");
        u64 *ta = noalloc_scratch(dev);
        u64 *tb = ta + kNoAllocWords;
        // every scratch word read below is written first by the forward
        // transforms, so nothing has to be cleared between calls
        std::vector<int> pid(nl);
        for (int i = 0; i < nl; i++) pid[i] = i;
        kern::LimbSet sa{const_cast<u64 *>(a), nl, nl, 1, pid}, sb{const_cast<u64 *>(b), nl, nl, 1, pid};
        kern::LimbSet da{ta, nl, nl, 1, pid}, db{tb, nl, nl, 1, pid}, dc{c, nl, nl, 1, pid};
        kern::ntt_fwd(ctx, sa, da);
        kern::ntt_fwd(ctx, sb, db);
        kern::pointwise(ctx, ta, tb, ta, nl, pid);
        kern::ntt_inv(ctx, da, dc);
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    } catch (const fg_error &e) {
        ctx->err = e.what();
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        return FG_EINVAL;
    }
    return FG_OK;
}
