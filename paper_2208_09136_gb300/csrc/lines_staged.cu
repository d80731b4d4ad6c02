// Instantiations of the line pass kernel (lines_kernel.cuh) with staged
// series windows (bulk copies into shared memory): the diagonal pass of
// m = 3, tau = 3 and m = 3, tau = 1 with register windows of 16 and 32
// diagonals.  A translation unit of their own, compiled in parallel with the rest.
#include "lines_kernel.cuh"

namespace rqa {

LinesKernel lines_kernel_staged(int embed, int tile)
{
    if (tile != 16 && tile != 32) return nullptr;
    switch (embed) {
    case E_M3T3: return tile == 32 ? k_lines<3, 3, 32, false, true> : k_lines<3, 3, 16, false, true>;
    case E_M3T1: return tile == 32 ? k_lines<3, 1, 32, false, true> : k_lines<3, 1, 16, false, true>;
    default: return nullptr;
    }
}

}  // namespace rqa
