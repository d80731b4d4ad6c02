// Line pass launches: the kernel variant for the batch's embedding and the
// register window, on a persistent grid (the kernel is in lines_kernel.cuh,
// its instantiations in lines_*.cu).
#include <algorithm>

#include "lines_kernel.cuh"

namespace rqa {


// Window widths the cell phase supports for an embedding variant: 8, 16 and
// 32 diagonals for the compile-time embeddings of the diagonal pass, 16
// otherwise.
bool lines_tile_ok(int embed, int tile)
{
    if (tile == LINE_TILE_DEFAULT) return true;
    const bool special = embed == E_M1T1 || embed == E_M3T1 || embed == E_M3T3;
    return special && (tile == 8 || tile == 32);
}

bool lines_stage_ok(int embed, int tile)
{
    return lines_kernel_staged(embed, tile) != nullptr;
}

// The kernel of an embedding variant and register window (full: a sweep of
// LINE_KMAX thresholds, which the special embeddings' diagonal pass has its
// own variant for).
static LinesKernel lines_kernel(int embed, int tile, bool vert, bool stage, bool full)
{
    if (stage) return lines_kernel_staged(embed, tile);
    switch (embed) {
    case E_M3T3: return lines_kernel_m3t3(tile, vert, full);
    case E_M3T1: return lines_kernel_m3t1(tile, vert, full);
    case E_M1T1: return lines_kernel_m1t1(tile, vert, full);
    case E_M1: case E_M2: case E_M3: case E_M4: return lines_kernel_generic(embed, vert);
    default: return lines_kernel_generic(0, vert);
    }
}

template <bool VERT>
static cudaError_t launch_lines_v(const CellArgs &a, const LineBufs &lb, int K, int grid, int embed,
                                  cudaStream_t st)
{
    if ((!VERT && !lines_tile_ok(embed, a.line_tile)) || (VERT && a.line_tile != LINE_TILE_DEFAULT))
        return cudaErrorInvalidValue;
    if (!a.y || !a.series || !a.order || !a.uprefix || !a.queue || !a.status || !lb.eps ||
        !lb.count || !lb.lmax || !lb.hshort || (lb.hist && !lb.hist_off) || K < 1 ||
        K > LINE_KMAX || lb.k0 < 0 || lb.k0 + K > lb.kstride || grid < 1 || a.n_units < 1 ||
        a.n_pos < 1 || a.chunk < 1)
        return cudaErrorInvalidValue;
    // staging where the variant exists; elsewhere the flag is ignored
    const bool stage = !VERT && a.line_stage && lines_stage_ok(embed, a.line_tile);
    if (stage && a.y_len < 1) return cudaErrorInvalidValue;
    LinesKernel kern = lines_kernel(embed, a.line_tile, VERT, stage, K == LINE_KMAX);
    const int smem = lines_smem_bytes_impl(stage);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    grid *= WARPS / LWARPS;  // the caller counts CTAs of WARPS warps
    grid = persistent_cap(reinterpret_cast<const void *>(kern), smem, grid, LTHREADS);
    if (a.line_ctas > 0) grid = std::min(grid, sm_count_current() * a.line_ctas);
    kern<<<grid, LTHREADS, smem, st>>>(a, lb, K);
    return cudaGetLastError();
}

cudaError_t launch_lines(const CellArgs &a, const LineBufs &lb, int K, int grid, int embed,
                         cudaStream_t st)
{
    return launch_lines_v<false>(a, lb, K, grid, embed, st);
}

cudaError_t launch_vlines(const CellArgs &a, const LineBufs &lb, int K, int grid, int embed,
                          cudaStream_t st)
{
    return launch_lines_v<true>(a, lb, K, grid, embed, st);
}

}  // namespace rqa
