// Launches of the ray marcher for 4, 8 and 16 wavelengths.  They live in a
// translation unit of their own (march_wide.cu) so that the library's two
// halves compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace dartray {

struct MarchArgs;

// Launch one wave of the marcher (mode: step 1, step 2 or a scattering
// iteration; det: the fixed-point deterministic mode; smem: dynamic shared
// memory bytes) with nl in {4, 8, 16};
// returns false for any other nl.
bool launch_march_wide(int nl, int mode, bool det, int blocks, int block, int smem, cudaStream_t st,
                       const DevGrid &G, const MarchArgs &A);

// Resident blocks per SM of the scattering-iteration marcher for nl in
// {4, 8, 16} with smem bytes of dynamic shared memory (0 for any other nl).
int march_wide_blocks_per_sm(int nl, int block, int smem);

}  // namespace dartray
