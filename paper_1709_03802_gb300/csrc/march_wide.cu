// The ray marcher instantiated for 4, 8 and 16 wavelengths (see
// march_wide.h).
#include "march_kernel.cuh"
#include "march_wide.h"

namespace dartray {

namespace {

template <int NL, bool DET>
void launch(int mode, int blocks, int block, int smem, cudaStream_t st, const DevGrid &G, const MarchArgs &A) {
    if (mode == MODE_LL) march_kernel<NL, MODE_LL, DET><<<blocks, block, smem, st>>>(G, A);
    else if (mode == MODE_DIRECT) march_kernel<NL, MODE_DIRECT, DET><<<blocks, block, smem, st>>>(G, A);
    else march_kernel<NL, MODE_SCATTER, DET><<<blocks, block, smem, st>>>(G, A);
}

template <int NL>
void launch_nl(int mode, bool det, int blocks, int block, int smem, cudaStream_t st, const DevGrid &G,
               const MarchArgs &A) {
    if (det) launch<NL, true>(mode, blocks, block, smem, st, G, A);
    else launch<NL, false>(mode, blocks, block, smem, st, G, A);
}

}  // namespace

bool launch_march_wide(int nl, int mode, bool det, int blocks, int block, int smem, cudaStream_t st,
                       const DevGrid &G, const MarchArgs &A) {
    switch (nl) {
    case 4: launch_nl<4>(mode, det, blocks, block, smem, st, G, A); return true;
    case 8: launch_nl<8>(mode, det, blocks, block, smem, st, G, A); return true;
    case 16: launch_nl<16>(mode, det, blocks, block, smem, st, G, A); return true;
    default: return false;
    }
}

int march_wide_blocks_per_sm(int nl, int block, int smem) {
    int n = 0;
    switch (nl) {
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<4, MODE_SCATTER, false>, block, smem); break;
    case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<8, MODE_SCATTER, false>, block, smem); break;
    case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<16, MODE_SCATTER, false>, block, smem); break;
    default: break;
    }
    return n;
}

}  // namespace dartray
