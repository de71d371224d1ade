// FP32 time step of the LBRS solver (distributions stored and updated in FP32).
//
// Compiled with FMA contraction allowed; velocities use one correctly rounded
// reciprocal per cell.  The numerics differ from the FP64 path by rounding
// only; their distance to the FP64 oracle is measured, not assumed.
#include "lbrs_kernels.cuh"
#include "lbrs_launch.h"

namespace lbrs {

cudaError_t launch_step_f32(int lattice, const StepArgs<float>& a, cudaStream_t s)
{
    if (lattice == LAT_D2Q4) {
        const dim3 block(128, 2);
        const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
        step2d_kernel<float><<<grid, block, 0, s>>>(a);
    } else {
        step1d_kernel<float><<<(unsigned)((a.nx + 255) / 256), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lbrs
