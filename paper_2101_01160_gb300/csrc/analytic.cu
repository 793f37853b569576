// Analytic MDLG equilibria (Sec. 3) and distribution comparison, FP64 on
// the device.  The Gaussian takes one thread per lattice velocity, the WSG
// one CTA per lattice velocity over its Poisson terms.  These are tiny
// launches (at most (2*MD_MAX_W+1)^2 = 441 classes).
#include <cstdarg>
#include <cmath>

#include "common.cuh"
#include "equilibria.cuh"

namespace mdlg {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

__global__ void k_feq_gaussian(double a2, double ux, double uy, int W, double *P) {
    const int side = 2 * W + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= side * side) return;
    const int ix = i % side, iy = i / side;
    P[i] = cell_gauss_1d((double)(ix - W) - ux, a2) * cell_gauss_1d((double)(iy - W) - uy, a2);
}

// One CTA per lattice velocity; its threads share the Poisson terms
// c = cmin..cmax (terms outside the window weigh < 1e-16 in total: the
// Poisson tails beyond 12 sqrt(lambda) + 20 of the mean).  Fixed-order
// reduction, so the result is reproducible.
constexpr int WSG_THREADS = 128;

__global__ void __launch_bounds__(WSG_THREADS) k_feq_wsg(double a2, double lam, double ux, double uy,
                                                         int W, int cmin, int cmax, double *P) {
    __shared__ double red[WSG_THREADS];
    const int side = 2 * W + 1;
    const int i = blockIdx.x;
    const double vx = (double)(i % side - W) - ux, vy = (double)(i / side - W) - uy;
    double acc = 0.0;
    for (int c = cmin + (int)threadIdx.x; c <= cmax; c += WSG_THREADS) {
        const double w = poisson_weight(c, lam);
        const double var = a2 * ((double)c + 1.0) / (lam + 1.0);
        acc += w * (cell_gauss_1d(vx, var) * cell_gauss_1d(vy, var));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = WSG_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) P[i] = red[0];
}

// Roots of Eq. (lambda_eq) in the printed form; root 1: '+' branch, root 2:
// '-' branch.  mode 1 / 2 writes the fixed degenerate values.
__global__ void k_wsg_lambda(double mu2, double mu4, int root, int mode, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (mode == 1) { *out = 0.0; return; }
    if (mode == 2) { *out = 1.0; return; }
    *out = lambda_root(mu2, mu4, root);
}

__global__ void k_compare(const double *R, const double *Q, int n, double *out) {
    __shared__ double smax[256], skl[256], ssum[256];
    double mx = 0.0, kl = 0.0, sm = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = R[i], q = Q[i];
        mx = fmax(mx, fabs(r - q));
        if (r > 0.0) kl += r * log(r / q);
        sm += r;
    }
    smax[threadIdx.x] = mx;
    skl[threadIdx.x] = kl;
    ssum[threadIdx.x] = sm;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            skl[threadIdx.x] += skl[threadIdx.x + o];
            ssum[threadIdx.x] += ssum[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = smax[0];
        out[1] = skl[0];
        out[2] = ssum[0];
    }
}



}  // namespace mdlg

using namespace mdlg;

extern "C" {

const char *md_last_error(void) { return g_last_error.c_str(); }

int feq_gaussian(double a2, double ux, double uy, int32_t W, double *P_out, void *stream) {
    if (!(a2 > 0.0) || !std::isfinite(a2)) return fail(MD_E_ARG, "feq_gaussian: a2 must be > 0");
    if (W < 0 || W > MD_MAX_W) return fail(MD_E_ARG, "feq_gaussian: W out of [0,%d]", MD_MAX_W);
    if (!P_out) return fail(MD_E_ARG, "feq_gaussian: P_out is NULL");
    const int nb = (2 * W + 1) * (2 * W + 1);
    k_feq_gaussian<<<(nb + 127) / 128, 128, 0, (cudaStream_t)stream>>>(a2, ux, uy, W, P_out);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

int feq_wsg(double a2, double lambda, double ux, double uy, int32_t W, double *P_out,
            void *stream) {
    if (!(a2 > 0.0) || !std::isfinite(a2)) return fail(MD_E_ARG, "feq_wsg: a2 must be > 0");
    if (!(lambda >= 0.0) || !(lambda < 1e6)) return fail(MD_E_ARG, "feq_wsg: lambda out of [0,1e6)");
    if (W < 0 || W > MD_MAX_W) return fail(MD_E_ARG, "feq_wsg: W out of [0,%d]", MD_MAX_W);
    if (!P_out) return fail(MD_E_ARG, "feq_wsg: P_out is NULL");
    const int nb = (2 * W + 1) * (2 * W + 1);
    k_feq_wsg<<<nb, WSG_THREADS, 0, (cudaStream_t)stream>>>(a2, lambda, ux, uy, W, wsg_cmin(lambda),
                                                            wsg_cmax(lambda), P_out);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

int wsg_lambda(double mu2, double mu4, int32_t root, double *lambda_out, void *stream) {
    if (!(mu2 > 0.0) || !(mu4 > 0.0)) return fail(MD_E_ARG, "wsg_lambda: moments must be > 0");
    if (root != 1 && root != 2) return fail(MD_E_ARG, "wsg_lambda: root must be 1 or 2");
    if (!lambda_out) return fail(MD_E_ARG, "wsg_lambda: lambda_out is NULL");
    const double k = mu4 / (mu2 * mu2);
    int mode = 0, rc = MD_OK;
    if (k <= 3.0) {
        mode = 1;
        rc = fail(MD_E_DOMAIN, "wsg_lambda: kurtosis %.17g <= 3, lambda set to 0", k);
    } else if (k > 3.75) {
        mode = 2;
        rc = fail(MD_E_DOMAIN, "wsg_lambda: kurtosis %.17g > 3.75, lambda set to 1", k);
    }
    k_wsg_lambda<<<1, 32, 0, (cudaStream_t)stream>>>(mu2, mu4, root, mode, lambda_out);
    MD_CUDA_TRY(cudaGetLastError());
    return rc;
}

int feq_compare(const double *R, const double *Q, int32_t n, double *out3, void *stream) {
    if (!R || !Q || !out3 || n < 1) return fail(MD_E_ARG, "feq_compare: bad arguments");
    k_compare<<<1, 256, 0, (cudaStream_t)stream>>>(R, Q, n, out3);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

}  // extern "C"
