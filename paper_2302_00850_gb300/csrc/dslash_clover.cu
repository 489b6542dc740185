// Clover epilogues of the hopping term (EPI_CLOVER_X: out = a A xin + b H in,
// EPI_CLOVER_INV: out = A^-1 b H in).  Kept apart from dslash.cu so that the
// two sets of kernel instantiations compile in parallel.
#include "dslash_kernel.cuh"

namespace cola {

cudaError_t launch_dslash_clover(int prec, int recon, const DslashArgs &A, int nparity, bool dagger, int epi, int bx,
                                 int nb, cudaStream_t s) {
    return launch_pr<EPI_CLOVER_X, EPI_CLOVER_INV>(prec, recon, A, nparity, dagger, epi, bx, nb, s);
}

}  // namespace cola
