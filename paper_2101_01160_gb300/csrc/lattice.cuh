// Device helpers of the MDLG lattice mapping (Sec. 2).  The integer results
// (lattice cell, displacement class) depend on FP64 arithmetic, so each
// operation is an explicitly rounded intrinsic: no contraction into FMA, the
// same rounding as a plain IEEE evaluation of x = cx*h + off and
// floor(x / dxl) on the host.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdlg {

// Position encoded as (cell coordinate, offset): x = c*h + off.
__device__ __forceinline__ double cell_position(int c, double h, double off) {
    return __dadd_rn(__dmul_rn((double)c, h), off);
}

// Lattice cell of coordinate x: floor(x / dxl) reduced modulo lx (a point on
// a cell boundary belongs to the upper cell).
__device__ __forceinline__ long long lattice_cell(double x, double dxl, int lx) {
    long long l = (long long)floor(__ddiv_rn(x, dxl));
    l %= lx;
    if (l < 0) l += lx;
    return l;
}

// Lattice displacement reduced to the nearest periodic image, in
// (-lx/2, lx/2].
__device__ __forceinline__ long long lattice_shift(long long d, int lx) {
    d %= lx;
    if (d < 0) d += lx;
    if (d > lx / 2) d -= lx;
    return d;
}

__device__ __forceinline__ double nearest_image(double d, double L) {
    return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

// Adds one count to sh[bin] for every lane with bin >= 0; lanes holding the
// same bin are merged into one shared-memory atomic.  All 32 lanes of the
// warp must call it.
__device__ __forceinline__ void warp_hist_add(int *sh, int bin, int lane) {
    const unsigned m = __match_any_sync(0xffffffffu, bin);
    if (bin >= 0 && lane == __ffs(m) - 1) atomicAdd(&sh[bin], __popc(m));
}

// Sum of two doubles over the CTA; the result is valid in thread 0.
// Fixed reduction tree (warp shuffles, then warp 0), so the result is the
// same on every run.
__device__ __forceinline__ void block_sum2(double &a, double &b) {
    __shared__ double s_a[32], s_b[32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        s_a[w] = a;
        s_b[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = lane < nw ? s_a[lane] : 0.0;
        b = lane < nw ? s_b[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
}

}  // namespace mdlg
