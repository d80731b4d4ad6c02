// Instantiations of the line pass kernel (lines_kernel.cuh) for the other
// embeddings: compile-time m with the delay read at run time (any tau), and
// the fully generic one (m and tau at run time), which the vertical pass uses
// for every embedding but the specialised ones.
#include "lines_kernel.cuh"

namespace rqa {

LinesKernel lines_kernel_generic(int m, bool vert)
{
    constexpr int T = LINE_TILE_DEFAULT;
    if (vert) return k_lines<0, 0, T, true>;
    switch (m) {
    case 1: return k_lines<1, 0, T, false>;
    case 2: return k_lines<2, 0, T, false>;
    case 3: return k_lines<3, 0, T, false>;
    case 4: return k_lines<4, 0, T, false>;
    default: return k_lines<0, 0, T, false>;
    }
}

}  // namespace rqa
