// Displacement-PDF diagnostics (Sec. 3(b), Fig. 2): the histogram of the
// continuous one-dimensional displacement component between two snapshots
// over bins X_i, the bin masses of the Gaussian (Eq. gaussian_df) and
// Poisson WSG (Eqs. poisson_v2, p_wsg_one) displacement PDFs, and the
// element-wise K(X_i) of Eq. k_Xi.
//
// The displacement is taken in the cell frame, wrap(c1 - c0) * h +
// (off1 - off0) with the cell difference wrapped to the nearest image, and
// its bin is floor(delta / width), every operation of that FP64 definition
// rounded on its own.  The kernel decides the bin in FP32 with a proven
// error bound and falls back to the FP64 definition only near bin edges
// (GB300's FP64 rate is a small fraction of its FP32 rate), so bin indices
// are exact.  The histogram is privatised per CTA in shared memory and
// flushed with 64-bit atomics: integer counts do not depend on the launch.
#include <cmath>

#include "common.cuh"
#include "equilibria.cuh"
#include "lattice.cuh"

namespace mdlg {

constexpr int PDF_MAX_BINS = 8192;    // 32 KB of shared counters per CTA

struct PdfSnap {
    const int32_t *cell;
    const void *ox, *oy;
    int f64;
};

// Bin index of one displacement component, floor(RN(d / w)) with d =
// RN(RN(dc * h) + RN(o1 - o0)) in FP64 (the definition), decided in FP32
// wherever FP32 provably gives the same integer.  With a = RN32(dc * hf),
// hf = RN32(h), invwf = RN32(1 / w):
//     q = RN32(RN32(a + RN32(o1 - o0)) * invwf),
//     S = RN32((|a| + |o1| + |o0|) * invwf),
// q differs from the exact quotient (dc h + o1 - o0) / w by less than
// S 2^-21 (two roundings of dc h, one of the offset difference, one of the
// sum, two of the product with the rounded reciprocal, one per offset if
// they are FP64 -- each at most 2^-24 relative to |a| + |o1| + |o0|), and
// the FP64 definition lies within a few 2^-53 of the same magnitude of that
// quotient.  So when q is more than S 2^-20 from the nearest integer, no
// integer separates the two and floor(q) is the bin; otherwise (values on or
// within about S 1e-6 of a bin edge) the FP64 division decides.
// Bit-identical to the FP64 definition for finite inputs.
// The FP64 definition, out of line (it runs only near bin edges).
__device__ __noinline__ long long disp_bin_slow(int dc, double o1, double o0, double h, double w) {
    const double doff = __dsub_rn(o1, o0);
    const double d = __dadd_rn(__dmul_rn((double)dc, h), doff);
    // floor as an integer in one round-down conversion
    return __double2ll_rd(__ddiv_rn(d, w));
}

template <typename T>
__device__ __forceinline__ long long disp_bin(int dc, T o1, T o0, double h, float hf, double w,
                                              float invwf) {
    const float a = __fmul_rn((float)dc, hf);
    const float f1 = (float)o1, f0 = (float)o0;
    const float q = __fmul_rn(__fadd_rn(a, __fsub_rn(f1, f0)), invwf);
    const float S = __fmul_rn(__fadd_rn(__fadd_rn(fabsf(a), fabsf(f1)), fabsf(f0)), invwf);
    // |q| < 2^22 here: a 32-bit round-down conversion (a 64-bit one would
    // run on the FP64 pipe)
    if (S < 0x1p22f && fabsf(__fsub_rn(q, rintf(q))) > __fmul_rn(S, 0x1p-20f))
        return __float2int_rd(q);
    return disp_bin_slow(dc, (double)o1, (double)o0, h, w);
}

template <typename T> struct PdfVec4;
template <> struct PdfVec4<float> {
    static __device__ __forceinline__ void load(const float *p, float (&v)[4]) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct PdfVec4<double> {
    static __device__ __forceinline__ void load(const double *p, double (&v)[4]) {
        const double2 q0 = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 q1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
};

struct DispParams {
    int ncell, nbins;
    float inv_ncell, hf, invwf;
    double h, w;
};

// Counts both displacement components of one particle into the CTA's bins.
template <typename T>
__device__ __forceinline__ void disp_count(const DispParams &P, int c0, int c1, T x0, T y0, T x1, T y1,
                                           unsigned *sh_bins, unsigned &my_out) {
    int cc0[2], cc1[2];
    split_cell(c0, P.ncell, P.inv_ncell, cc0[0], cc0[1]);
    split_cell(c1, P.ncell, P.inv_ncell, cc1[0], cc1[1]);
    const T o0[2] = {x0, y0}, o1[2] = {x1, y1};
    const long long lo = -(long long)(P.nbins / 2), hi = (long long)P.nbins - P.nbins / 2;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        int dc = cc1[ax] - cc0[ax];
        if (dc > P.ncell / 2) dc -= P.ncell;
        if (dc < -(P.ncell / 2)) dc += P.ncell;
        const long long k = disp_bin<T>(dc, o1[ax], o0[ax], P.h, P.hf, P.w, P.invwf);
        if (k >= lo && k < hi)
            atomicAdd(&sh_bins[(int)(k - lo)], 1u);
        else
            ++my_out;
    }
}

// Grid-stride over groups of four consecutive particles (VEC: 16-byte
// aligned arrays read with vector loads, all loads of a group issued before
// any arithmetic), then the last n % 4 particles one per thread.
template <typename T, bool VEC>
__global__ void k_disp_hist(PdfSnap a, PdfSnap b, int n, DispParams P, unsigned long long *hist,
                            unsigned long long *outside) {
    extern __shared__ unsigned int sh_bins[];
    for (int k = threadIdx.x; k < P.nbins; k += blockDim.x) sh_bins[k] = 0u;
    __syncthreads();
    unsigned my_out = 0;
    const T *ax = static_cast<const T *>(a.ox), *ay = static_cast<const T *>(a.oy);
    const T *bx = static_cast<const T *>(b.ox), *by = static_cast<const T *>(b.oy);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long ngroup = VEC ? n / 4 : 0;
    for (long long g = tid; g < ngroup; g += stride) {
        const int4 q0 = __ldg(reinterpret_cast<const int4 *>(a.cell) + g);
        const int4 q1 = __ldg(reinterpret_cast<const int4 *>(b.cell) + g);
        const int c0[4] = {q0.x, q0.y, q0.z, q0.w}, c1[4] = {q1.x, q1.y, q1.z, q1.w};
        T x0[4], y0[4], x1[4], y1[4];
        PdfVec4<T>::load(ax + 4 * g, x0);
        PdfVec4<T>::load(ay + 4 * g, y0);
        PdfVec4<T>::load(bx + 4 * g, x1);
        PdfVec4<T>::load(by + 4 * g, y1);
#pragma unroll
        for (int u = 0; u < 4; ++u) disp_count<T>(P, c0[u], c1[u], x0[u], y0[u], x1[u], y1[u], sh_bins, my_out);
    }
    for (long long j = 4 * ngroup + tid; j < n; j += stride)
        disp_count<T>(P, a.cell[j], b.cell[j], ax[j], ay[j], bx[j], by[j], sh_bins, my_out);
    for (int o = 16; o > 0; o >>= 1) my_out += __shfl_xor_sync(0xffffffffu, my_out, o);
    if ((threadIdx.x & 31) == 0 && my_out) atomicAdd(outside, (unsigned long long)my_out);
    __syncthreads();
    for (int k = threadIdx.x; k < P.nbins; k += blockDim.x)
        if (sh_bins[k]) atomicAdd(&hist[k], (unsigned long long)sh_bins[k]);
}

// Mass of a centred normal distribution of variance var in [lo, hi).
__device__ __forceinline__ double normal_mass(double lo, double hi, double var) {
    const double s = sqrt(__dmul_rn(2.0, var));
    return 0.5 * (erf(hi / s) - erf(lo / s));
}

// One thread per bin: Gaussian of variance mu2 and the Poisson mixture of
// Gaussians of variance (c + 1) mu2 / (lambda + 1) over the window of c.
__global__ void k_pdf_models(double mu2, double lam, double width, int nbins, double *pg, double *pwsg) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nbins) return;
    const double lo = __dmul_rn((double)(k - nbins / 2), width);
    const double hi = __dadd_rn(lo, width);
    pg[k] = normal_mass(lo, hi, mu2);
    double s = 0.0;
    const int c1 = wsg_cmax(lam);
    for (int c = wsg_cmin(lam); c <= c1; ++c)
        s += poisson_weight(c, lam) * normal_mass(lo, hi, (double)(c + 1) * mu2 / (lam + 1.0));
    pwsg[k] = s;
}

__global__ void k_kl_terms(const double *R, const double *Q, int n, double *K) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) K[i] = R[i] > 0.0 ? R[i] * log(R[i] / Q[i]) : 0.0;
}

// One wave of resident CTAs of the histogram kernel (its occupancy with
// `smem` bytes of bins times the SM count), fewer when there is less work.
template <typename K>
int disp_grid(K kernel, long long work, size_t smem) {
    int dev = 0, nsm = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem);
    long long g = (long long)(nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1);
    const long long need = (work + 255) / 256;
    if (need < g) g = need;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace mdlg

using namespace mdlg;

extern "C" int mdlg_disp_hist(const md_snapshot *t0, const md_snapshot *t1, int64_t n, double width,
                              int32_t nbins, int64_t *hist_out, int64_t *outside_out, void *stream) {
    mdlg::Range range_("mdlg_disp_hist");
    if (!t0 || !t1 || !hist_out || !outside_out) return fail(MD_E_ARG, "mdlg_disp_hist: NULL argument");
    if (n < 0 || n >= (int64_t)1 << 31) return fail(MD_E_ARG, "mdlg_disp_hist: n out of [0, 2^31)");
    if (n > 0 && (!t0->cell || !t0->off_x || !t0->off_y || !t1->cell || !t1->off_x || !t1->off_y))
        return fail(MD_E_ARG, "mdlg_disp_hist: NULL snapshot array");
    if (t0->ncell != t1->ncell || t0->h != t1->h || t0->off_is_f64 != t1->off_is_f64)
        return fail(MD_E_ARG, "mdlg_disp_hist: snapshots differ in ncell, h or offset type");
    if (t0->ncell < 1 || !(t0->h > 0.0) || (int64_t)t0->ncell * t0->ncell >= (int64_t)1 << 31)
        return fail(MD_E_ARG, "mdlg_disp_hist: bad ncell or h");
    if (!(width > 0.0) || !std::isfinite(width)) return fail(MD_E_ARG, "mdlg_disp_hist: width must be > 0");
    if (nbins < 1 || nbins > PDF_MAX_BINS)
        return fail(MD_E_ARG, "mdlg_disp_hist: nbins out of [1, %d]", PDF_MAX_BINS);
    cudaStream_t st = (cudaStream_t)stream;
    MD_CUDA_TRY(cudaMemsetAsync(hist_out, 0, sizeof(int64_t) * nbins, st));
    MD_CUDA_TRY(cudaMemsetAsync(outside_out, 0, sizeof(int64_t), st));
    if (n == 0) return MD_OK;
    PdfSnap a{t0->cell, t0->off_x, t0->off_y, t0->off_is_f64};
    PdfSnap b{t1->cell, t1->off_x, t1->off_y, t1->off_is_f64};
    DispParams P;
    P.ncell = t0->ncell;
    P.nbins = nbins;
    P.h = t0->h;
    P.w = width;
    P.hf = (float)t0->h;
    P.invwf = (float)(1.0 / width);
    P.inv_ncell = 1.0f / (float)t0->ncell;
    const size_t smem = sizeof(unsigned) * nbins;
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    const bool vec = al16(a.cell) && al16(a.ox) && al16(a.oy) && al16(b.cell) && al16(b.ox) && al16(b.oy);
    unsigned long long *h64 = (unsigned long long *)hist_out, *o64 = (unsigned long long *)outside_out;
    const long long work = vec ? (n + 3) / 4 : n;
    auto go = [&](auto kernel) {
        kernel<<<disp_grid(kernel, work, smem), 256, smem, st>>>(a, b, (int)n, P, h64, o64);
    };
    if (t0->off_is_f64) {
        if (vec) go(k_disp_hist<double, true>);
        else go(k_disp_hist<double, false>);
    } else {
        if (vec) go(k_disp_hist<float, true>);
        else go(k_disp_hist<float, false>);
    }
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" int disp_pdf_models(double mu2, double lambda, double width, int32_t nbins, double *pg_out,
                               double *pwsg_out, void *stream) {
    if (!pg_out || !pwsg_out) return fail(MD_E_ARG, "disp_pdf_models: NULL output");
    if (!(mu2 > 0.0) || !std::isfinite(mu2)) return fail(MD_E_ARG, "disp_pdf_models: mu2 must be > 0");
    if (!(lambda >= 0.0) || !(lambda <= 1e5)) return fail(MD_E_ARG, "disp_pdf_models: lambda out of [0, 1e5]");
    if (!(width > 0.0) || !std::isfinite(width)) return fail(MD_E_ARG, "disp_pdf_models: width must be > 0");
    if (nbins < 1 || nbins > PDF_MAX_BINS)
        return fail(MD_E_ARG, "disp_pdf_models: nbins out of [1, %d]", PDF_MAX_BINS);
    cudaStream_t st = (cudaStream_t)stream;
    k_pdf_models<<<(nbins + 127) / 128, 128, 0, st>>>(mu2, lambda, width, nbins, pg_out, pwsg_out);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" int kl_terms(const double *R, const double *Q, int32_t n, double *K_out, void *stream) {
    if (!R || !Q || !K_out || n < 0) return fail(MD_E_ARG, "kl_terms: bad arguments");
    if (n == 0) return MD_OK;
    k_kl_terms<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(R, Q, n, K_out);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
