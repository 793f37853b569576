// Local MDLG fields (Sec. 2): the occupation numbers n_i(x, t) of Eq. n_i
// per lattice site, and the lattice-gas collision operator of Eq.
// mdlg_evolution, Xi_i(x, t) = n_i(x + v_i, t + dt) - n_i(x, t), with its
// ensemble average Omega_i = <Xi_i> over replicas of one box.
//
// Layout: a field is int32 [Q][lx][lx], class-major (class i = (vy+W)(2W+1)
// + (vx+W), site ly*lx + lx_), so that each class is one contiguous lattice
// plane: the collision kernel reads plane i of n(t + dt) shifted by v_i,
// which stays coalesced except at the periodic wrap.
//
// The occupation kernel maps both snapshots to lattice sites exactly as the
// global binning does (lattice.cuh: the FP64 cell of each position, decided
// in FP32 wherever FP32 provably gives the same cell), so summing a field
// over its sites gives mdlg_bin's histogram bit for bit.
// Each particle adds one count at its arrival site with one atomic; integer
// counts do not depend on the launch.  The arithmetic is FP32 and 32-bit
// integer except near lattice lines, so the kernel is bound by its loads
// (24 bytes per FP32 particle pair) and the field's atomics in L2.
#include "common.cuh"
#include "lattice.cuh"

namespace mdlg {

struct LocSnap {
    const int32_t *cell;
    const void *ox, *oy;
};

struct OccParams {
    int ncell, lx, W;
    float inv_ncell, hf, invf;
    double h, dxl;
};

// Field index of one particle (class-major, at its arrival site), or -1 with
// the arrival site in *oi when the displacement leaves the window.
template <typename T>
__device__ __forceinline__ int occ_index(const OccParams &P, int c0, T ox0, T oy0, int c1, T ox1, T oy1,
                                         int &oi) {
    int cx0, cy0, cx1, cy1;
    split_cell(c0, P.ncell, P.inv_ncell, cx0, cy0);
    split_cell(c1, P.ncell, P.inv_ncell, cx1, cy1);
    const int sx1 = lattice_cell_f32<T>(cx1, ox1, P.h, P.hf, P.dxl, P.invf, P.lx);
    const int sy1 = lattice_cell_f32<T>(cy1, oy1, P.h, P.hf, P.dxl, P.invf, P.lx);
    const int vx = lattice_shift_near(sx1 - lattice_cell_f32<T>(cx0, ox0, P.h, P.hf, P.dxl, P.invf, P.lx), P.lx);
    const int vy = lattice_shift_near(sy1 - lattice_cell_f32<T>(cy0, oy0, P.h, P.hf, P.dxl, P.invf, P.lx), P.lx);
    const int site = sy1 * P.lx + sx1;
    oi = -1;
    if (vx >= -P.W && vx <= P.W && vy >= -P.W && vy <= P.W)
        return ((vy + P.W) * (2 * P.W + 1) + (vx + P.W)) * (P.lx * P.lx) + site;
    oi = site;
    return -1;
}

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void load(const float *p, float (&v)[4]) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Vec4<double> {
    static __device__ __forceinline__ void load(const double *p, double (&v)[4]) {
        const double2 q0 = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 q1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
};

__device__ __forceinline__ void occ_add(int fi, int oi, int *field, int *ovf) {
    if (fi >= 0)
        atomicAdd(&field[fi], 1);
    else
        atomicAdd(&ovf[oi], 1);
}

// Grid-stride over groups of four consecutive particles (VEC: the six
// arrays are 16-byte aligned and read with vector loads, all loads of a
// group issued before any arithmetic), then the last n % 4 particles one
// per thread.  One plain atomic per particle: the sites of consecutive
// particles are scattered once the gas has mixed, so merging equal
// addresses within a warp first does not pay.
template <typename T, bool VEC>
__global__ void k_site_occupation(LocSnap a, LocSnap b, int n, OccParams P, int *field, int *ovf) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const T *ax = static_cast<const T *>(a.ox), *ay = static_cast<const T *>(a.oy);
    const T *bx = static_cast<const T *>(b.ox), *by = static_cast<const T *>(b.oy);
    const long long ngroup = VEC ? n / 4 : 0;
    for (long long g = tid; g < ngroup; g += stride) {
        const int4 q0 = __ldg(reinterpret_cast<const int4 *>(a.cell) + g);
        const int4 q1 = __ldg(reinterpret_cast<const int4 *>(b.cell) + g);
        const int c0[4] = {q0.x, q0.y, q0.z, q0.w}, c1[4] = {q1.x, q1.y, q1.z, q1.w};
        T x0[4], y0[4], x1[4], y1[4];
        Vec4<T>::load(ax + 4 * g, x0);
        Vec4<T>::load(ay + 4 * g, y0);
        Vec4<T>::load(bx + 4 * g, x1);
        Vec4<T>::load(by + 4 * g, y1);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int oi;
            const int fi = occ_index<T>(P, c0[u], x0[u], y0[u], c1[u], x1[u], y1[u], oi);
            occ_add(fi, oi, field, ovf);
        }
    }
    for (long long j = 4 * ngroup + tid; j < n; j += stride) {
        int oi;
        const int fi = occ_index<T>(P, a.cell[j], ax[j], ay[j], b.cell[j], bx[j], by[j], oi);
        occ_add(fi, oi, field, ovf);
    }
}

// Grid (row tiles of `rows` rows, class i): each thread walks the tile's
// entries (y, x) in steps of the block size, keeping (y, x) incrementally,
// and writes xi = n_next[i][(y + vy) mod lx][(x + vx) mod lx] - n_t[i][y][x].
// The class shift is reduced into [0, lx) once per thread, so the periodic
// wrap is one conditional subtract per coordinate.
// entries of whole rows per block of k_collision (measured: 1024 and 4096-16384 slower)
constexpr int COLLISION_BLOCK_ENTRIES = 2048;
__global__ void k_collision(const int *nt, const int *nn, int lx, int W, int rows, double scale,
                            int *xi_out, double *omega_out) {
    const int side = 2 * W + 1;
    const int i = blockIdx.y;
    int sx = (i % side - W) % lx, sy = (i / side - W) % lx;
    if (sx < 0) sx += lx;
    if (sy < 0) sy += lx;
    const int y0 = blockIdx.x * rows;
    const int y1 = min(lx, y0 + rows);
    const long long plane = (long long)i * lx * lx;
    int y = y0 + (int)(threadIdx.x / lx), x = (int)(threadIdx.x % lx);
    const int step_y = (int)(blockDim.x / lx), step_x = (int)(blockDim.x % lx);
    auto advance = [&](int &ax, int &ay) {
        ax += step_x;
        ay += step_y;
        if (ax >= lx) {
            ax -= lx;
            ++ay;
        }
    };
    auto source = [&](int ax, int ay) {
        int xd = ax + sx, yd = ay + sy;
        if (xd >= lx) xd -= lx;
        if (yd >= lx) yd -= lx;
        return plane + (long long)yd * lx + xd;
    };
    // four entries per iteration, their eight loads issued together
    constexpr int U = 4;
    while (y < y1) {
        int ex[U], ey[U];
        ex[0] = x;
        ey[0] = y;
#pragma unroll
        for (int u = 1; u < U; ++u) {
            ex[u] = ex[u - 1];
            ey[u] = ey[u - 1];
            advance(ex[u], ey[u]);
        }
        int a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[u] = 0;
            b[u] = 0;
            if (ey[u] < y1) {
                a[u] = nn[source(ex[u], ey[u])];
                b[u] = nt[plane + (long long)ey[u] * lx + ex[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (ey[u] < y1) {
                const long long e = plane + (long long)ey[u] * lx + ex[u];
                const int v = a[u] - b[u];
                if (xi_out) xi_out[e] = v;
                if (omega_out) omega_out[e] = scale * (double)v;
            }
        }
        x = ex[U - 1];
        y = ey[U - 1];
        advance(x, y);
    }
}

// One wave of resident CTAs (occupancy of the instantiation times the SM
// count), fewer when there is less work.
template <typename K>
int occ_grid(K kernel, long long work) {
    int dev = 0, nsm = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
    long long g = (long long)(nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1);
    const long long need = (work + 255) / 256;
    if (need < g) g = need;
    return (int)(g < 1 ? 1 : g);
}

template <typename T>
void occ_launch_t(bool vec, LocSnap a, LocSnap b, int n, const OccParams &P, int *f, int *o, cudaStream_t st) {
    if (vec) {
        auto k = k_site_occupation<T, true>;
        k<<<occ_grid(k, (n + 3) / 4), 256, 0, st>>>(a, b, n, P, f, o);
    } else {
        auto k = k_site_occupation<T, false>;
        k<<<occ_grid(k, n), 256, 0, st>>>(a, b, n, P, f, o);
    }
}

void occ_launch(bool f64, bool vec, LocSnap a, LocSnap b, int n, const OccParams &P, int *f, int *o,
                cudaStream_t st) {
    if (f64)
        occ_launch_t<double>(vec, a, b, n, P, f, o, st);
    else
        occ_launch_t<float>(vec, a, b, n, P, f, o, st);
}

}  // namespace mdlg

using namespace mdlg;

extern "C" int mdlg_site_occupation(const md_snapshot *t0, const md_snapshot *t1, int64_t n, int32_t lx,
                                    int32_t W, int32_t *n_out, int32_t *overflow_out, void *stream) {
    mdlg::Range range_("mdlg_site_occupation");
    if (!t0 || !t1 || !n_out || !overflow_out) return fail(MD_E_ARG, "mdlg_site_occupation: NULL argument");
    if (n < 0 || n >= (int64_t)1 << 31) return fail(MD_E_ARG, "mdlg_site_occupation: n out of [0, 2^31)");
    if (n > 0 && (!t0->cell || !t0->off_x || !t0->off_y || !t1->cell || !t1->off_x || !t1->off_y))
        return fail(MD_E_ARG, "mdlg_site_occupation: NULL snapshot array");
    if (t0->ncell != t1->ncell || t0->h != t1->h || t0->off_is_f64 != t1->off_is_f64)
        return fail(MD_E_ARG, "mdlg_site_occupation: snapshots differ in ncell, h or offset type");
    if (t0->ncell < 1 || !(t0->h > 0.0) || (int64_t)t0->ncell * t0->ncell >= (int64_t)1 << 31)
        return fail(MD_E_ARG, "mdlg_site_occupation: bad ncell or h");
    if (lx < 1) return fail(MD_E_ARG, "mdlg_site_occupation: lx must be >= 1");
    if (W < 0 || W > MD_MAX_W) return fail(MD_E_ARG, "mdlg_site_occupation: W out of [0,%d]", MD_MAX_W);
    const int64_t side = 2 * (int64_t)W + 1;
    if (side * side * (int64_t)lx * lx >= (int64_t)1 << 31)
        return fail(MD_E_LIMIT, "mdlg_site_occupation: (2W+1)^2 lx^2 must be < 2^31");
    if (n == 0) return MD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    LocSnap a{t0->cell, t0->off_x, t0->off_y};
    LocSnap b{t1->cell, t1->off_x, t1->off_y};
    OccParams P;
    P.ncell = t0->ncell;
    P.lx = lx;
    P.W = W;
    P.h = t0->h;
    P.dxl = (double)t0->ncell * t0->h / (double)lx;
    P.inv_ncell = 1.0f / (float)t0->ncell;
    P.hf = (float)t0->h;
    P.invf = (float)(1.0 / P.dxl);
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    const bool vec = al16(a.cell) && al16(a.ox) && al16(a.oy) && al16(b.cell) && al16(b.ox) && al16(b.oy);
    occ_launch(t0->off_is_f64 != 0, vec, a, b, (int)n, P, n_out, overflow_out, st);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" int mdlg_collision(const int32_t *n_t, const int32_t *n_next, int32_t lx, int32_t W, double scale,
                              int32_t *xi_out, double *omega_out, void *stream) {
    mdlg::Range range_("mdlg_collision");
    if (!n_t || !n_next || (!xi_out && !omega_out)) return fail(MD_E_ARG, "mdlg_collision: NULL argument");
    if (lx < 1) return fail(MD_E_ARG, "mdlg_collision: lx must be >= 1");
    if (W < 0 || W > MD_MAX_W) return fail(MD_E_ARG, "mdlg_collision: W out of [0,%d]", MD_MAX_W);
    const int64_t side = 2 * (int64_t)W + 1;
    const int64_t total = side * side * (int64_t)lx * lx;
    if (total >= (int64_t)1 << 31) return fail(MD_E_LIMIT, "mdlg_collision: (2W+1)^2 lx^2 must be < 2^31");
    // about COLLISION_BLOCK_ENTRIES entries (whole rows) per block
    const int rows = lx >= COLLISION_BLOCK_ENTRIES ? 1 : COLLISION_BLOCK_ENTRIES / lx;
    const dim3 grid((unsigned)((lx + rows - 1) / rows), (unsigned)(side * side));
    k_collision<<<grid, 256, 0, (cudaStream_t)stream>>>(n_t, n_next, lx, W, rows, scale, xi_out, omega_out);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
