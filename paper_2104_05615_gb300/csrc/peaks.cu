// dwf_fma_peak: the CUDA cores' fused multiply-add rate, measured on the
// device at the clocks it actually runs.
//
// The FP32 stages and the FP64 operator of the reliable updates run on the
// CUDA cores, so their rooflines need the FP32 and FP64 FMA rates; no data
// sheet figure gives them at the clocks reached under load.  Every thread
// runs kChains independent recurrences x <- x * a + b (enough independent
// work to hide the FMA latency at full occupancy), unrolled so the loop
// control costs a few percent of the issue slots; one FMA = 2 flops.
#include <cfloat>
#include <new>

#include "engine.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 8;
constexpr int kThreads = 512;

template <typename R>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(R *sink, int iters, R a, R b)
{
    R x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = R(threadIdx.x) * R(1e-3) + R(c);
    for (int it = 0; it < iters; it += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
    }
    R s = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    // the recurrences stay near 1 (fixed point b / (1 - a)), so this store
    // never happens; it keeps the compiler from dropping the chains
    if (s < R(-1)) sink[0] = s;
}

template <typename R>
double measure(dwf::Engine &E, int iters)
{
    using namespace dwf;
    int dev = 0, sms = 0, per_sm = 0;
    DWF_CUDA(cudaGetDevice(&dev));
    DWF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<R>, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;  // one full wave: no tail
    R *sink = static_cast<R *>(E.ws("fma_peak_sink", 64));
    EventPair ev;
    float best = FLT_MAX;
    for (int rep = 0; rep < 4; rep++) {  // the first is a warm-up
        DWF_CUDA(cudaEventRecord(ev.e0, E.st));
        fma_peak_kernel<R><<<blocks, kThreads, 0, E.st>>>(sink, iters, R(0.9999999), R(1e-7));
        DWF_CUDA(cudaGetLastError());
        DWF_CUDA(cudaEventRecord(ev.e1, E.st));
        DWF_CUDA(cudaEventSynchronize(ev.e1));
        float ms = 0.f;
        DWF_CUDA(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
        if (rep > 0 && ms < best) best = ms;
    }
    count_launch(4);
    const double flops = 2.0 * kChains * (double)iters * kThreads * (double)blocks;
    return flops / (best * 1e-3) / 1e12;
}

}  // namespace

dwf::Engine *dwf_handle_engine(dwf_handle *h);
void dwf_handle_set_error(dwf_handle *h, const char *msg);

extern "C" dwf_status dwf_fma_peak(dwf_handle *h, dwf_prec prec, double *tflops)
{
    using namespace dwf;
    if (!h || !tflops || (prec != DWF_F32 && prec != DWF_F64)) return DWF_EINVAL;
    Engine &E = *dwf_handle_engine(h);
    try {
        // about 4 ms (FP32) and 15 ms (FP64) per launch on a GB300
        *tflops = prec == DWF_F32 ? measure<float>(E, 1 << 16) : measure<double>(E, 1 << 12);
    } catch (const CudaError &e) {
        dwf_handle_set_error(h, cudaGetErrorString(e.err));
        return e.err == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA;
    } catch (const std::bad_alloc &) {
        dwf_handle_set_error(h, "host allocation failed");
        return DWF_ENOMEM;
    } catch (const std::exception &e) {
        dwf_handle_set_error(h, e.what());
        return DWF_ECUDA;
    }
    return DWF_OK;
}
