// Failure detection exercised on purpose, without a GPU fault: a cooperative
// launch of two CTAs in which the second returns at once and never arrives
// at the grid barrier the first one waits at.  The first gives up after the
// barrier's spin limit (SPIN_LIMIT_CYCLES, about two seconds), records
// DERR_TIMEOUT and returns, exactly as a persistent kernel of the library
// would if a peer CTA never showed up.
#include "ps_internal.cuh"

namespace ps {

__global__ void __launch_bounds__(32) k_wait_probe(Ctr* C)
{
    if (blockIdx.x == 1) return;   // this CTA never arrives
    grid_barrier(C);
}

cudaError_t launch_wait_probe(Ctr* C, cudaStream_t s)
{
    void* args[] = {(void*)&C};
    return cudaLaunchCooperativeKernel((const void*)k_wait_probe, dim3(2), dim3(32), args, 0, s);
}

}  // namespace ps
