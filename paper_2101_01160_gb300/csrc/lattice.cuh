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

// The same lattice cell, floor(RN(x / dxl)) mod lx, with the division
// replaced by a product with inv = RN(1 / dxl) wherever that cannot change
// the result.  q = RN(x * inv) and RN(x / dxl) both lie within |q| 2^-51 of
// the exact quotient x / dxl (each is one or two roundings of relative size
// 2^-53 away from it), so when q is more than |q| 2^-50 from the nearest
// integer no integer separates them and floor(q) is the answer; otherwise
// (points on or next to a lattice line, x = 0, and |q| < 2^-900, where
// underflow would void the relative bounds) the division is done.
// Bit-identical to lattice_cell for every finite x; one FP64 product, a rint
// and a compare in place of a division on all but those cases.
__device__ __forceinline__ long long lattice_cell_mul(double x, double dxl, double inv, int lx) {
    const double q = __dmul_rn(x, inv);
    const double t = rint(q);
    const double fq = fabs(q);
    double f;
    if (fq > 0x1p-900 && fabs(__dsub_rn(q, t)) > __dmul_rn(fq, 0x1p-50))
        f = floor(q);
    else
        f = floor(__ddiv_rn(x, dxl));
    long long l = (long long)f;
    l %= lx;
    if (l < 0) l += lx;
    return l;
}

// The lattice cell of the position encoded as (cell coordinate c, offset
// off), floor(RN(RN(c*h + off) / dxl)) mod lx as lattice_cell computes it,
// decided in FP32 wherever FP32 provably gives the same cell.  With a =
// RN32(c * hf), hf = RN32(h), invf = RN32(1/dxl):
//     q = RN32(RN32(a + off) * invf),   S = RN32(RN32(|a| + |off|) * invf),
// the distance of q from the exact quotient (c*h + off)/dxl is below
// S 2^-21 (a: two roundings of c*h, the sum one, the offset one if it is
// FP64, the product two -- each at most 2^-24 relative to |a| + |off|), and
// the FP64 reference lies within a few 2^-53 relative of the same quotient.
// So when q is more than S 2^-20 from the nearest integer, floor(q) is the
// cell; otherwise (points on or within about S 1e-6 of a lattice line) the
// FP64 evaluation of lattice_cell decides.  Bit-identical to lattice_cell
// for every finite encoded position; in the common case a few FP32 and
// 32-bit integer operations replace the FP64 ones and the 64-bit modulo
// (GB300's FP64 rate is a small fraction of its FP32 rate).  lx < 2^22.
// The FP64 evaluation, out of line: it runs only near lattice lines, and
// keeping it out of the unrolled callers keeps their code small.
static __device__ __noinline__ int lattice_cell_slow(int c, double off, double h, double dxl, int lx) {
    return (int)lattice_cell(cell_position(c, h, off), dxl, lx);
}

template <typename T>
__device__ __forceinline__ int lattice_cell_f32(int c, T off, double h, float hf, double dxl, float invf,
                                                int lx) {
    const float a = __fmul_rn((float)c, hf);
    const float o = (float)off;
    const float q = __fmul_rn(__fadd_rn(a, o), invf);
    const float S = __fmul_rn(__fadd_rn(fabsf(a), fabsf(o)), invf);
    if (S < 0x1p22f && fabsf(__fsub_rn(q, rintf(q))) > __fmul_rn(S, 0x1p-20f)) {
        int l = __float2int_rd(q);   // |q| < 2^22: floor in one 32-bit conversion
        // positions within a box edge of the box need one wrap; others the
        // general reduction
        if (l < 0) l += lx;
        else if (l >= lx) l -= lx;
        if (l < 0 || l >= lx) {
            l %= lx;
            if (l < 0) l += lx;
        }
        return l;
    }
    return lattice_cell_slow(c, (double)off, h, dxl, lx);
}

// Splits a linear cell index c = cy * ncell + cx (0 <= cx, cy < ncell,
// ncell^2 < 2^31) without an integer division: the float estimate of
// c / ncell (< 46341) carries a relative error below 2^-22, so it is off by
// at most one, and one multiply-subtract with a fix-up makes it exact.
__device__ __forceinline__ void split_cell(int c, int ncell, float inv_ncell, int &cx, int &cy) {
    int y = (int)__fmul_rz((float)c, inv_ncell);
    int x = c - y * ncell;
    if (x < 0) {
        --y;
        x += ncell;
    } else if (x >= ncell) {
        ++y;
        x -= ncell;
    }
    cx = x;
    cy = y;
}

// Nearest periodic image of a lattice displacement d in (-lx, lx) (two
// cells of [0, lx)), in (-lx/2, lx/2]: lattice_shift without the modulo.
__device__ __forceinline__ int lattice_shift_near(int d, int lx) {
    if (d < 0) d += lx;
    if (d > lx / 2) d -= lx;
    return d;
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
