// Instantiations of the line pass kernel (lines_kernel.cuh) for m = 3, tau = 1:
// the diagonal pass with register windows of 8, 16 and 32 diagonals (each also
// for a full sweep of LINE_KMAX thresholds), and the vertical pass.  One group
// per translation unit, so they compile in parallel.
#include "lines_kernel.cuh"

namespace rqa {

LinesKernel lines_kernel_m3t1(int tile, bool vert, bool full)
{
    if (vert) return k_lines<3, 1, LINE_TILE_DEFAULT, true>;
    switch (tile) {
    case 8: return full ? k_lines<3, 1, 8, false, false, true> : k_lines<3, 1, 8, false>;
    case 32: return full ? k_lines<3, 1, 32, false, false, true> : k_lines<3, 1, 32, false>;
    default:
        return full ? k_lines<3, 1, LINE_TILE_DEFAULT, false, false, true>
                    : k_lines<3, 1, LINE_TILE_DEFAULT, false>;
    }
}

}  // namespace rqa
