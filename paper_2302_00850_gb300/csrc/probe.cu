// FP64 arithmetic-peak probe: a kernel of independent FP64 fused
// multiply-add chains, timed by the caller, that measures the FP64 rate the
// hopping term's FP64 instantiation is bound by on this part.  It has no
// counterpart in the paper; it exists so that the FP64 roofline is a
// measured number, not one derived from unit counts and clocks.
//
// Each thread runs kChains independent chains x <- x * m + c (the update
// has the fixed point c / (1 - m), so values stay bounded and normal), each
// chain advancing once per step, for `steps` steps: exactly
// kChains * steps DFMA instructions per thread, 2 flop each.  The chains
// are independent, so enough of them are in flight per warp to keep the FP64
// pipe busy without depending on its latency; the final sum is stored so
// that nothing is optimised away.
#include "cola_impl.h"

namespace cola {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_chains_kernel(double *out, int steps, double m, double c) {
    double x[kChains];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (double)((tid + k) & 63);
    for (int s = 0; s < steps; s += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], m, c);
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += x[k];
    out[tid] = acc;
}

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" cola_status cola_probe_fp64_fma(double *out, int blocks, int threads, int steps, cudaStream_t stream,
                                           double *flop) {
    if (!out || !flop) {
        set_error("null argument to cola_probe_fp64_fma");
        return COLA_ERR_ARG;
    }
    if (blocks < 1 || blocks > (1 << 20) || threads < 32 || threads > 256 || threads % 32 != 0 || steps < 4 ||
        steps % 4 != 0) {
        set_error("cola_probe_fp64_fma: blocks in 1..2^20, threads a multiple of 32 in 32..256, steps a positive "
                  "multiple of 4");
        return COLA_ERR_ARG;
    }
    fp64_fma_chains_kernel<<<blocks, threads, 0, stream>>>(out, steps, 0.999999, 1e-7);
    *flop = 2.0 * kChains * (double)steps * (double)threads * (double)blocks;
    return cuda_check(cudaGetLastError(), "fp64 probe launch");
}
