// peak.cu -- measured integer-multiply throughput of the GPU: the ALU
// roofline the modular kernels are compared against.
//
// Every thread runs eight independent chains of one 32-bit multiply
// instruction (no chain waits on another, so the pipe, not latency, bounds
// the rate) on a grid of eight 256-thread CTAs per SM.  The chains' results
// are folded into one word per thread that is written out, so no multiply
// can be dropped.  Rates are instructions (one per thread and operation) per
// second over the whole GPU, timed with CUDA events on the context's stream
// after one warm-up launch.
#include "fg_internal.h"
#include "modarith.cuh"

namespace {

constexpr int kPeakChains = 8;
constexpr int kPeakIters = 4096;

template <int OP>
__global__ void __launch_bounds__(256) k_mul_peak(u64 *out, u32 seed)
{
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u32 a[kPeakChains], b = seed ^ (t * 2654435761u);
    u64 acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) {
        a[c] = t + 977u * c + 1u;
        acc[c] = (u64)c * 0x9E3779B9u;
    }
    for (int it = 0; it < kPeakIters; it++) {
#pragma unroll
        for (int c = 0; c < kPeakChains; c++) {
            if (OP == 0) {   // 32 x 32 -> 64-bit multiply-add (the split products' step)
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[c]) : "r"(a[c]), "r"(b));
            } else if (OP == 1) {   // high word of a 32 x 32 product
                u32 h;
                asm volatile("mul.hi.u32 %0, %1, %2;" : "=r"(h) : "r"(a[c]), "r"(b));
                a[c] = h ^ (u32)it;
            } else if (OP == 2) {   // 32-bit multiply-add, low word
                u32 l;
                asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(l) : "r"(a[c]), "r"(b), "r"((u32)acc[c]));
                acc[c] = l;
            } else {   // 32 x 32 -> 64-bit product added to a 64-bit sum by a carry-chained
                       // pair (the step of the split products): counted as one
                asm volatile("{\n\t.reg .u32 l, h;\n\tmov.b64 {l, h}, %0;\n\t"
                             "mad.lo.cc.u32 l, %1, %2, l;\n\tmadc.hi.u32 h, %1, %2, h;\n\t"
                             "mov.b64 %0, {l, h};\n\t}"
                             : "+l"(acc[c]) : "r"(a[c]), "r"(b));
            }
        }
    }
    u64 r = 0;
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) r += acc[c] + a[c];
    out[t] = r;
}

}  // namespace

extern "C" int fg_int_mul_peak(fg_ctx *ctx, int op, double *ops_per_s)
{
    if (!ctx || !ops_per_s || op < 0 || op > 3) return FG_EINVAL;
    try {
        int sms = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        const int blocks = sms * 8, threads = 256;
        u64 *out = (u64 *)ctx->buf("peak_out", (size_t)blocks * threads * 8);
        cudaEvent_t e0, e1;
        CUDA_TRY(cudaEventCreate(&e0));
        CUDA_TRY(cudaEventCreate(&e1));
        float ms = 0;
        for (int rep = 0; rep < 2; rep++) {   // first launch warms up
            CUDA_TRY(cudaEventRecord(e0, ctx->stream));
            if (op == 0) k_mul_peak<0><<<blocks, threads, 0, ctx->stream>>>(out, 12345u + rep);
            else if (op == 1) k_mul_peak<1><<<blocks, threads, 0, ctx->stream>>>(out, 12345u + rep);
            else if (op == 2) k_mul_peak<2><<<blocks, threads, 0, ctx->stream>>>(out, 12345u + rep);
            else k_mul_peak<3><<<blocks, threads, 0, ctx->stream>>>(out, 12345u + rep);
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(cudaEventRecord(e1, ctx->stream));
            CUDA_TRY(cudaEventSynchronize(e1));
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->launches += 2;
        *ops_per_s = (double)blocks * threads * kPeakChains * kPeakIters / (ms * 1e-3);
    } catch (const fg_error &e) {
        ctx->err = e.what();
        return e.code;
    }
    return FG_OK;
}
