// MDLG binning of two position snapshots (Sec. 2, Eq. n_i summed over the
// lattice sites): standalone entry point mdlg_bin.  The fused variant that
// runs inside the MD step lives in md.cu; both share the device helpers of
// lattice.cuh.
//
// Design: grid-stride over particles; the (2W+1)^2 histogram is privatised
// per CTA in shared memory with warp-aggregated integer atomics (most
// particles fall in the few central classes, so lanes of a warp usually agree
// and one atomic per distinct class is issued); the FP64 moment sums are
// reduced per CTA into a scratch array and summed in CTA order by a second
// one-block kernel, so the result does not depend on scheduling.
#include <mutex>

#include "common.cuh"
#include "lattice.cuh"

namespace mdlg {

struct SnapDev {
    const int32_t *cell;
    const void *ox;
    const void *oy;
    int f64;
};

__device__ __forceinline__ double snap_off(const void *p, int f64, int j) {
    return f64 ? static_cast<const double *>(p)[j] : (double)static_cast<const float *>(p)[j];
}

__global__ void k_bin_snapshots(SnapDev s0, SnapDev s1, int n, int ncell, double h, double L,
                                int lx, double dxl, double inv, int W, int *hist,
                                unsigned long long *ovf, double *part) {
    extern __shared__ int sh[];
    const int side = 2 * W + 1, nb = side * side;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    double m2 = 0.0, m4 = 0.0;
    unsigned my_ovf = 0;
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    // Whole warps iterate together so that the warp-aggregated atomics see
    // every lane.
    const int nround = (n + stride - 1) / stride;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = 0; r < nround; ++r, j += stride) {
        int bin = -1;
        if (j < n) {
            const int c0 = s0.cell[j], c1 = s1.cell[j];
            const int cx0 = c0 % ncell, cy0 = c0 / ncell;
            const int cx1 = c1 % ncell, cy1 = c1 / ncell;
            const double x0 = cell_position(cx0, h, snap_off(s0.ox, s0.f64, j));
            const double y0 = cell_position(cy0, h, snap_off(s0.oy, s0.f64, j));
            const double x1 = cell_position(cx1, h, snap_off(s1.ox, s1.f64, j));
            const double y1 = cell_position(cy1, h, snap_off(s1.oy, s1.f64, j));
            const long long ddx = lattice_shift(
                lattice_cell_mul(x1, dxl, inv, lx) - lattice_cell_mul(x0, dxl, inv, lx), lx);
            const long long ddy = lattice_shift(
                lattice_cell_mul(y1, dxl, inv, lx) - lattice_cell_mul(y0, dxl, inv, lx), lx);
            if (ddx >= -W && ddx <= W && ddy >= -W && ddy <= W)
                bin = (int)((ddy + W) * side + (ddx + W));
            else
                ++my_ovf;
            const double ex = nearest_image(x1 - x0, L), ey = nearest_image(y1 - y0, L);
            const double ex2 = ex * ex, ey2 = ey * ey;
            m2 += ex2 + ey2;
            m4 += ex2 * ex2 + ey2 * ey2;
        }
        warp_hist_add(sh, bin, lane);
    }
    // overflow: exact integer sum
    for (int o = 16; o > 0; o >>= 1) my_ovf += __shfl_xor_sync(0xffffffffu, my_ovf, o);
    if (lane == 0 && my_ovf) atomicAdd(ovf, (unsigned long long)my_ovf);
    block_sum2(m2, m4);
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = m2;
        part[2 * blockIdx.x + 1] = m4;
    }
}

// Sums the per-CTA moment partials in CTA order (one warp, fixed tree).
__global__ void k_sum_partials(const double *part, int nparts, double *mom) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 32) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
        mom[0] = a;
        mom[1] = b;
    }
}

int bin_check_args(const md_snapshot *t0, const md_snapshot *t1, int64_t n, int32_t lx, int32_t W,
                   const void *hist_out, const void *overflow_out, const void *mom_out) {
    if (!t0 || !t1 || !hist_out || !overflow_out || !mom_out)
        return fail(MD_E_ARG, "mdlg_bin: NULL argument");
    if (n < 0 || n >= (int64_t)1 << 31) return fail(MD_E_ARG, "mdlg_bin: n out of [0, 2^31)");
    if (n > 0 && (!t0->cell || !t0->off_x || !t0->off_y || !t1->cell || !t1->off_x || !t1->off_y))
        return fail(MD_E_ARG, "mdlg_bin: NULL snapshot array");
    if (t0->ncell != t1->ncell || t0->h != t1->h || t0->off_is_f64 != t1->off_is_f64)
        return fail(MD_E_ARG, "mdlg_bin: snapshots differ in ncell, h or offset type");
    if (t0->ncell < 1 || !(t0->h > 0.0)) return fail(MD_E_ARG, "mdlg_bin: bad ncell or h");
    if ((int64_t)t0->ncell * t0->ncell >= (int64_t)1 << 31)
        return fail(MD_E_ARG, "mdlg_bin: ncell^2 must fit in int32");
    if (lx < 1) return fail(MD_E_ARG, "mdlg_bin: lx must be >= 1");
    if (W < 0 || W > MD_MAX_W) return fail(MD_E_ARG, "mdlg_bin: W out of [0,%d]", MD_MAX_W);
    return MD_OK;
}

// Enqueues the two binning kernels with the moment partials in `part`
// (>= 2*grid doubles of device memory).  Outputs must be zeroed by the
// caller's stream order beforehand.
int bin_launch(const md_snapshot *t0, const md_snapshot *t1, int64_t n, int32_t lx, int32_t W,
               int32_t *hist_out, int64_t *overflow_out, double *mom_out, double *part, int grid,
               cudaStream_t st) {
    const int nb = (2 * W + 1) * (2 * W + 1);
    SnapDev a{t0->cell, t0->off_x, t0->off_y, t0->off_is_f64};
    SnapDev b{t1->cell, t1->off_x, t1->off_y, t1->off_is_f64};
    const double L = (double)t0->ncell * t0->h;
    const double dxl = L / (double)lx;
    k_bin_snapshots<<<grid, 256, nb * sizeof(int), st>>>(a, b, (int)n, t0->ncell, t0->h, L, lx, dxl,
                                                        1.0 / dxl, W, hist_out,
                                                        (unsigned long long *)overflow_out, part);
    MD_CUDA_TRY(cudaGetLastError());
    k_sum_partials<<<1, 32, 0, st>>>(part, grid, mom_out);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

// Moment partials of mdlg_bin_noalloc, for callers that cannot allocate
// device memory while they run (their memory belongs to a framework's
// caching allocator or a fixed budget, or their loop must not stall on
// allocator calls): a fixed device array instead of a per-call allocation
// (2 doubles per CTA, room for BIN_SCRATCH_CTAS CTAs, 32 KiB, held by every
// GPU that loads the library until the process exits).  Every CTA of a
// launch overwrites its own two entries and the reduction reads only the
// first `grid`, so it never needs clearing.  Host code must not pass the
// array's name to a kernel (on the host it only stands in for the symbol);
// it passes the device address that cudaGetSymbolAddress returns.
constexpr int BIN_SCRATCH_CTAS = 2048;
static __device__ __align__(256) double g_bin_scratch[2 * BIN_SCRATCH_CTAS];

// CTAs of one binning launch: one per 256 particles, at most 8 per SM of
// the current device (SM count queried per call: a process may bin on GPUs
// of different sizes).
int bin_grid(int64_t n) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        nsm = 1;
    int64_t want = (n + 255) / 256;
    int64_t cap = (int64_t)nsm * 8;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

// Device address of g_bin_scratch on the current device.  Looked up with
// that device current on the first call made on it, and looked up again
// when the device's context has changed since (after a cudaDeviceReset the
// module is loaded afresh and the array may live elsewhere).  The table is
// guarded by a mutex, so host threads may call concurrently.
using CtxGetCurrentFn = int (*)(void **);
constexpr int BIN_MAX_DEV = 64;
struct ScratchSlot {
    const void *ctx = nullptr;
    double *ptr = nullptr;
};
std::mutex g_scratch_mu;
ScratchSlot g_scratch[BIN_MAX_DEV];

CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    return fn;
}

int scratch_address(double **out) {
    int dev = 0;
    MD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= BIN_MAX_DEV)
        return fail(MD_E_LIMIT, "mdlg_bin_noalloc: device %d >= %d", dev, BIN_MAX_DEV);
    const CtxGetCurrentFn get = ctx_get_current();
    auto current = [get]() {
        void *c = nullptr;
        if (!get || get(&c) != 0) c = nullptr;
        return c;
    };
    // no current context yet on this thread (or no way to ask): look up,
    // which also makes the device's primary context current
    const void *ctx = current();
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    ScratchSlot &sl = g_scratch[dev];
    if (!sl.ptr || !ctx || sl.ctx != ctx) {
        double *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_bin_scratch);
        if (e != cudaSuccess)
            return fail(MD_E_CUDA, "mdlg_bin_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        sl.ptr = p;
        sl.ctx = current();
    }
    *out = sl.ptr;
    return MD_OK;
}

}  // namespace mdlg

using namespace mdlg;

extern "C" int mdlg_bin(const md_snapshot *t0, const md_snapshot *t1, int64_t n, int32_t lx,
                        int32_t W, int32_t *hist_out, int64_t *overflow_out, double *mom_out,
                        void *stream) {
    mdlg::Range range_("mdlg_bin");
    int rc = bin_check_args(t0, t1, n, lx, W, hist_out, overflow_out, mom_out);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (2 * W + 1) * (2 * W + 1);
    const int grid = bin_grid(n);
    MD_CUDA_TRY(cudaMemsetAsync(hist_out, 0, nb * sizeof(int32_t), st));
    MD_CUDA_TRY(cudaMemsetAsync(overflow_out, 0, sizeof(int64_t), st));
    double *part = nullptr;
    MD_CUDA_TRY(cudaMallocAsync((void **)&part, 2 * sizeof(double) * grid, st));
    rc = bin_launch(t0, t1, n, lx, W, hist_out, overflow_out, mom_out, part, grid, st);
    cudaError_t e = cudaFreeAsync(part, st);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(MD_E_CUDA, "mdlg_bin: cudaFreeAsync: %s", cudaGetErrorString(e));
    return MD_OK;
}

// Same computation as mdlg_bin with the partials in g_bin_scratch.  The
// array's device address is looked up on the first call on each device
// (with that device current), and again after a cudaDeviceReset, so that
// first call should come before any stream capture; nothing is allocated.
// Calls that overlap on the GPU share the array and race.
extern "C" int mdlg_bin_noalloc(const md_snapshot *t0, const md_snapshot *t1, int64_t n, int32_t lx,
                                int32_t W, int32_t *hist_out, int64_t *overflow_out, double *mom_out,
                                void *stream) {
    mdlg::Range range_("mdlg_bin_noalloc");
    int rc = bin_check_args(t0, t1, n, lx, W, hist_out, overflow_out, mom_out);
    if (rc) return rc;
    const int grid = bin_grid(n);
    if (grid > BIN_SCRATCH_CTAS)
        return fail(MD_E_LIMIT, "mdlg_bin_noalloc: %d CTAs exceed the scratch capacity of %d", grid,
                    BIN_SCRATCH_CTAS);
    double *scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (2 * W + 1) * (2 * W + 1);
    MD_CUDA_TRY(cudaMemsetAsync(hist_out, 0, nb * sizeof(int32_t), st));
    MD_CUDA_TRY(cudaMemsetAsync(overflow_out, 0, sizeof(int64_t), st));
    return bin_launch(t0, t1, n, lx, W, hist_out, overflow_out, mom_out, scratch, grid, st);
}
