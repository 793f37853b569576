// Host side of the MD system: md_init / md_init_batch / md_step / readouts.
//
// One system holds one or more replicas.  md_step enqueues a single
// cooperative launch of the persistent kernel (md_kernels.cuh) that runs all
// requested steps, sampling and cell-list rebuilds on the device; control
// returns to the host only at md_sync or at a readout.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "equilibria.cuh"
#include "md_kernels.cuh"
#include "md_resident.cuh"

namespace mdlg {

template <typename T>
__global__ void k_init(SysDev S, const double *x, const double *y, const double *vx,
                       const double *vy) {
    using V = typename V2<T>::type;
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot < S.nrep) {
        const RepDev &R = S.reps[slot];
        S.cellcnt[R.cbase + R.nc * R.nc] = R.cap - R.n;
    }
    if (slot >= S.nslots) return;
    const RepDev &R = S.reps[S.gran_rep[slot / GRAN]];
    const int local = slot - R.pbase;
    V *pos = static_cast<V *>(S.pos[0][0]);
    V *vel = static_cast<V *>(S.vel[0]);
    if (local >= R.n) {
        pos[slot] = V{T(0), T(0)};
        vel[slot] = V{T(0), T(0)};
        S.cell[0][slot] = 0u;
        S.pid[0][slot] = -1;
        return;
    }
    const int id = R.ibase + local;
    double X = x[id], Y = y[id];
    X -= R.L * floor(X / R.L);
    Y -= R.L * floor(Y / R.L);
    if (X >= R.L) X -= R.L;
    if (Y >= R.L) Y -= R.L;
    int cx = (int)floor(X / R.h), cy = (int)floor(Y / R.h);
    cx = min(max(cx, 0), R.nc - 1);
    cy = min(max(cy, 0), R.nc - 1);
    pos[slot] = V{(T)(X - (double)cx * R.h), (T)(Y - (double)cy * R.h)};
    vel[slot] = V{(T)vx[id], (T)vy[id]};
    S.cell[0][slot] = (uint32_t)cx | ((uint32_t)cy << 16);
    S.pid[0][slot] = id;
}

// Energy partials of one replica summed in a fixed order by one CTA.
__device__ __forceinline__ void sum_energy_cta(const double *epart, int g0, int g1, double *out4) {
    __shared__ double sh[4][256];
    double a[4] = {0, 0, 0, 0};
    for (int g = g0 + threadIdx.x; g < g1; g += 256)
        for (int k = 0; k < 4; ++k) a[k] += epart[(long long)g * 4 + k];
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 4) out4[threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_sum_energy(const double *epart, int g0, int g1, double *out4) {
    sum_energy_cta(epart, g0, g1, out4);
}

// every replica at once, one CTA per replica: the same sums as k_sum_energy
__global__ void k_sum_energy_batch(const double *epart, const RepDev *reps, double *out) {
    const RepDev &R = reps[blockIdx.x];
    sum_energy_cta(epart, R.pbase / 32, (R.pbase + R.cap) / 32, out + 4 * (size_t)blockIdx.x);
}

struct FeqArgs {
    const int32_t *hist;          // [MD_NBLK][nb] of one (rep, lg, dx)
    const unsigned long long *ovf;
    const double *mom;            // [ngran32][n_lg][2]
    int g0, g1, n_lg, lg, nb, W, sym;
    double n;                     // particles of the replica
    long long nwin;
    long long wblk[MD_NBLK];      // windows per block
    double dx_eff;
    double *out;                  // [nb] P, [nb] stderr, [8] stats
};

// Normalised measured equilibrium (Eq. theory_feq per particle), batch-means
// error bars over blocks of windows, optional symmetric-set averaging
// (Sec. 5), moments mu2, mu4 and a^2 (Eq. a2_n_ua).  One CTA.
constexpr int FEQ_THREADS = 128;

__global__ void __launch_bounds__(FEQ_THREADS) k_feq_measured(FeqArgs A) {
    __shared__ double s2[FEQ_THREADS], s4[FEQ_THREADS];
    double m2 = 0.0, m4 = 0.0;
    for (int g = A.g0 + threadIdx.x; g < A.g1; g += blockDim.x) {
        m2 += A.mom[((long long)g * A.n_lg + A.lg) * 2];
        m4 += A.mom[((long long)g * A.n_lg + A.lg) * 2 + 1];
    }
    s2[threadIdx.x] = m2;
    s4[threadIdx.x] = m4;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s2[threadIdx.x] += s2[threadIdx.x + o];
            s4[threadIdx.x] += s4[threadIdx.x + o];
        }
        __syncthreads();
    }
    const double samples = A.n * (double)A.nwin;
    const int side = 2 * A.W + 1;
    for (int i = threadIdx.x; i < A.nb; i += blockDim.x) {
        int mem[8];
        int nm = 0;
        if (A.sym) {
            const int a = abs(i % side - A.W), b = abs(i / side - A.W);
            const int lo = min(a, b), hi = max(a, b);
            for (int j = 0; j < A.nb && nm < 8; ++j) {
                const int c = abs(j % side - A.W), d = abs(j / side - A.W);
                if (min(c, d) == lo && max(c, d) == hi) mem[nm++] = j;
            }
        } else {
            mem[nm++] = i;
        }
        long long tot = 0;
        double pb[MD_NBLK];
        for (int b = 0; b < MD_NBLK; ++b) {
            long long hb = 0;
            for (int m = 0; m < nm; ++m) hb += A.hist[b * A.nb + mem[m]];
            tot += hb;
            pb[b] = A.wblk[b] > 0 ? (double)hb / ((double)nm * A.n * (double)A.wblk[b]) : 0.0;
        }
        const double P = samples > 0 ? (double)tot / ((double)nm * samples) : 0.0;
        double num = 0.0, wsum = 0.0;
        int used = 0;
        for (int b = 0; b < MD_NBLK; ++b) {
            if (A.wblk[b] <= 0) continue;
            const double w = (double)A.wblk[b];
            num += w * w * (pb[b] - P) * (pb[b] - P);
            wsum += w;
            ++used;
        }
        A.out[i] = P;
        A.out[A.nb + i] = used > 1 ? sqrt(num / (wsum * wsum) * (double)used / (double)(used - 1)) : 0.0;
    }
    if (threadIdx.x == 0) {
        double *st = A.out + 2 * A.nb;
        const double mu2 = samples > 0 ? s2[0] / (2.0 * samples) : 0.0;
        const double mu4 = samples > 0 ? s4[0] / (2.0 * samples) : 0.0;
        st[0] = mu2;
        st[1] = mu4;
        st[2] = mu2 / (A.dx_eff * A.dx_eff);
        st[3] = (double)(*A.ovf);
    }
}

__global__ void k_hist_total(const int32_t *hist, int nb, long long *out) {
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        long long t = 0;
        for (int b = 0; b < MD_NBLK; ++b) t += hist[b * nb + i];
        out[i] = t;
    }
}

__global__ void k_copy_snapshot(const uint32_t *sc, const void *so, int f64, long long ntot,
                                const int32_t *nc_of_id, int32_t *cell, void *ox, void *oy) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    const uint32_t pk = sc[i];
    cell[i] = (int32_t)(pk >> 16) * nc_of_id[i] + (int32_t)(pk & 0xffffu);
    if (f64) {
        const double2 v = static_cast<const double2 *>(so)[i];
        static_cast<double *>(ox)[i] = v.x;
        static_cast<double *>(oy)[i] = v.y;
    } else {
        const float2 v = static_cast<const float2 *>(so)[i];
        static_cast<float *>(ox)[i] = v.x;
        static_cast<float *>(oy)[i] = v.y;
    }
}

__global__ void k_nc_of_id(SysDev S, int32_t *nc_of_id) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= S.nslots) return;
    const RepDev &R = S.reps[S.gran_rep[slot / GRAN]];
    const int local = slot - R.pbase;
    if (local < R.n) nc_of_id[R.ibase + local] = R.nc;
}


// ---------------------------------------------------------------- batched f_eq stage
// For every replica, on the device (k_feq_params: the moments and lambda;
// k_feq_terms: the WSG sums over the Poisson window, split over CTAs;
// k_feq_batch: one CTA per replica for the rest): the measured equilibrium
// (Eq. theory_feq per particle, optionally averaged over symmetric sets),
// the moments mu2, mu4 and a^2 (Eq. a2_n_ua), lambda from Eq. (lambda_eq)
// (root 2), the Gaussian (Eq. feq_gaussian) and WSG (Eq. f_eq_wsg)
// equilibria at that a^2 and lambda, and their distance to the measured one
// (max |difference| and Eq. kullback_leibler).
constexpr int FEQB_THREADS = 128;
constexpr int FEQB_STATS = 16;

struct FeqBatchArgs {
    const RepDev *reps;
    const int32_t *hist;           // [nrep][n_lg][n_dx][MD_NBLK][nb]
    const unsigned long long *ovf; // [nrep][n_lg][n_dx]
    const double *mom;             // [ngran32][n_lg][2]
    int n_lg, n_dx, lg, dxi, nb, W, sym;
    long long nwin;
    double *out;                   // [nrep][3 nb + FEQB_STATS]
};

// The WSG sum of one replica is spread over up to FEQB_SPLIT CTAs of
// FEQB_SPLIT_TERMS Poisson terms each (the last takes any remainder): with
// lambda capped at 1e5 the window holds at most 7,631 terms, and a single
// CTA would carry them all on one SM's FP64 pipe.
constexpr int FEQB_SPLIT = 64;
constexpr int FEQB_SPLIT_TERMS = FEQB_THREADS;

// Splits that hold terms for lambda (the others add nothing).
__device__ inline int feqb_splits_used(double lam) {
    const int n = wsg_cmax(lam) - wsg_cmin(lam) + 1;
    return min(FEQB_SPLIT, (n + FEQB_SPLIT_TERMS - 1) / FEQB_SPLIT_TERMS);
}

// Moments, a^2 and lambda of replica r into s_par = {mu2, a^2, lambda}
// (every thread calls it; s_a, s_b: FEQB_THREADS doubles of scratch); with
// out != nullptr thread 0 also writes the replica's statistics.
__device__ void feqb_params(const FeqBatchArgs &A, const RepDev &R, int r, double *s_a, double *s_b,
                            double *s_par, double *out) {
    const int tid = threadIdx.x;
    const double samples = (double)R.n * (double)A.nwin;
    double m2 = 0.0, m4 = 0.0;
    for (int g = R.pbase / 32 + tid; g < (R.pbase + R.cap) / 32; g += FEQB_THREADS) {
        m2 += A.mom[((long long)g * A.n_lg + A.lg) * 2];
        m4 += A.mom[((long long)g * A.n_lg + A.lg) * 2 + 1];
    }
    s_a[tid] = m2;
    s_b[tid] = m4;
    __syncthreads();
    for (int o = FEQB_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o) {
            s_a[tid] += s_a[tid + o];
            s_b[tid] += s_b[tid + o];
        }
        __syncthreads();
    }
    if (tid == 0) {
        const double mu2 = samples > 0 ? s_a[0] / (2.0 * samples) : 0.0;
        const double mu4 = samples > 0 ? s_b[0] / (2.0 * samples) : 0.0;
        const double dx = R.dxl[A.dxi];
        double lam = 0.0, st = 0.0;
        const double k = mu2 > 0 ? mu4 / (mu2 * mu2) : 0.0;
        if (!(k > 3.0)) {
            st = 1.0;
        } else if (k > 3.75) {
            lam = 1.0;
            st = 2.0;
        } else {
            lam = lambda_root(mu2, mu4, 2);
            if (lam > 1e5) {
                lam = 1e5;   // the mixture is then a single Gaussian to ~1e-5
                st = 3.0;
            }
        }
        s_par[0] = mu2;
        s_par[1] = mu2 / (dx * dx);
        s_par[2] = lam;
        if (out) {
            out[3 * A.nb + 0] = mu2;
            out[3 * A.nb + 1] = mu4;
            out[3 * A.nb + 2] = s_par[1];
            out[3 * A.nb + 3] = lam;
            out[3 * A.nb + 8] = (double)A.nwin;
            out[3 * A.nb + 9] = samples;
            out[3 * A.nb + 10] = (double)A.ovf[((long long)r * A.n_lg + A.lg) * A.n_dx + A.dxi];
            out[3 * A.nb + 11] = dx;
            out[3 * A.nb + 12] = st;
        }
    }
    __syncthreads();
}

constexpr int FEQB_CPT = ((2 * MD_MAX_W + 1) * (2 * MD_MAX_W + 1) + FEQB_THREADS - 1) / FEQB_THREADS;

// One CTA per replica: par[4 r + {0, 1, 2}] = mu2, a^2, lambda.
__global__ void __launch_bounds__(FEQB_THREADS) k_feq_params(FeqBatchArgs A, double *par) {
    __shared__ double s_a[FEQB_THREADS], s_b[FEQB_THREADS], s_par[4];
    const int r = blockIdx.x;
    feqb_params(A, A.reps[r], r, s_a, s_b, s_par, nullptr);
    if (threadIdx.x < 3) par[4 * r + threadIdx.x] = s_par[threadIdx.x];
}

// Grid (replica, split): the split's Poisson terms c, one per thread in
// chunks of FEQB_THREADS; the 1D factors of one term are evaluated once for
// the 2W+1 displacements and shared by all classes (the 2D value is their
// outer product); each class sums the chunk's terms in increasing c.
// part[(r * FEQB_SPLIT + split) * nb + i] = the split's partial sum, written
// by the splits that hold terms (feqb_splits_used); the others return at
// once.
__global__ void __launch_bounds__(FEQB_THREADS) k_feq_terms(FeqBatchArgs A, const double *par,
                                                            double *part) {
    __shared__ double s_w[FEQB_THREADS];
    __shared__ double s_F[FEQB_THREADS][2 * MD_MAX_W + 1];
    const int r = blockIdx.x, split = blockIdx.y, tid = threadIdx.x;
    const double a2 = par[4 * r + 1], lam = par[4 * r + 2];
    if (split >= feqb_splits_used(lam)) return;
    const int side = 2 * A.W + 1;
    double accW[FEQB_CPT];
#pragma unroll
    for (int q = 0; q < FEQB_CPT; ++q) accW[q] = 0.0;
    const int cmin = wsg_cmin(lam), cmax = wsg_cmax(lam);
    const int lo = cmin + split * FEQB_SPLIT_TERMS;
    const int hi = split == FEQB_SPLIT - 1 ? cmax : min(cmax, lo + FEQB_SPLIT_TERMS - 1);
    for (int c0 = lo; c0 <= hi && a2 > 0; c0 += FEQB_THREADS) {
        const int c = c0 + tid;
        if (c <= hi) {
            s_w[tid] = poisson_weight(c, lam);
            cell_gauss_row(a2 * ((double)c + 1.0) / (lam + 1.0), A.W, s_F[tid]);
        }
        __syncthreads();
        const int nterm = min(FEQB_THREADS, hi - c0 + 1);
#pragma unroll
        for (int q = 0; q < FEQB_CPT; ++q) {
            const int i = tid + q * FEQB_THREADS;
            if (i < A.nb) {
                const int ix = i % side, iy = i / side;
                double acc = accW[q];
                for (int t = 0; t < nterm; ++t) acc += s_w[t] * (s_F[t][ix] * s_F[t][iy]);
                accW[q] = acc;
            }
        }
        __syncthreads();
    }
    double *dst = part + ((long long)r * FEQB_SPLIT + split) * A.nb;
#pragma unroll
    for (int q = 0; q < FEQB_CPT; ++q) {
        const int i = tid + q * FEQB_THREADS;
        if (i < A.nb) dst[i] = accW[q];
    }
}

// One CTA per replica: the statistics, the WSG sum of the splits' partials
// (in split order), the measured and Gaussian equilibria and the distances.
__global__ void __launch_bounds__(FEQB_THREADS) k_feq_batch(FeqBatchArgs A, const double *part) {
    __shared__ double s_a[FEQB_THREADS], s_b[FEQB_THREADS], s_c[FEQB_THREADS], s_d[FEQB_THREADS];
    __shared__ double s_par[4];
    const int r = blockIdx.x, tid = threadIdx.x;
    const RepDev &R = A.reps[r];
    const int stride = 3 * A.nb + FEQB_STATS;
    double *out = A.out + (long long)r * stride;
    const int32_t *hist = A.hist + ((((long long)r * A.n_lg + A.lg) * A.n_dx + A.dxi) * MD_NBLK) * A.nb;
    const double samples = (double)R.n * (double)A.nwin;
    feqb_params(A, R, r, s_a, s_b, s_par, out);
    const double a2 = s_par[1];
    const int side = 2 * A.W + 1;
    const int used = feqb_splits_used(s_par[2]);
    // the Gaussian's 1D factors, one row shared by all classes
    __shared__ double s_G[2 * MD_MAX_W + 1];
    if (tid == 0 && a2 > 0) cell_gauss_row(a2, A.W, s_G);
    __syncthreads();
    constexpr int CPT = FEQB_CPT;
    double accW[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int i = tid + q * FEQB_THREADS;
        double acc = 0.0;
        if (i < A.nb && a2 > 0)
            for (int sp = 0; sp < used; ++sp) acc += part[((long long)r * FEQB_SPLIT + sp) * A.nb + i];
        accW[q] = acc;
    }
    double mg = 0.0, kg = 0.0, mw = 0.0, kw = 0.0, sum = 0.0;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int i = tid + q * FEQB_THREADS;
        if (i >= A.nb) continue;
        int mem[8], nm = 0;
        if (A.sym) {
            const int a = abs(i % side - A.W), b = abs(i / side - A.W);
            const int lo = min(a, b), hi = max(a, b);
            for (int j = 0; j < A.nb && nm < 8; ++j) {
                const int c = abs(j % side - A.W), d = abs(j / side - A.W);
                if (min(c, d) == lo && max(c, d) == hi) mem[nm++] = j;
            }
        } else {
            mem[nm++] = i;
        }
        long long tot = 0;
        for (int b = 0; b < MD_NBLK; ++b)
            for (int m = 0; m < nm; ++m) tot += hist[b * A.nb + mem[m]];
        const double P = samples > 0 ? (double)tot / ((double)nm * samples) : 0.0;
        const double G = a2 > 0 ? s_G[i % side] * s_G[i / side] : 0.0;
        const double Wg = accW[q];
        out[i] = P;
        out[A.nb + i] = G;
        out[2 * A.nb + i] = Wg;
        mg = fmax(mg, fabs(P - G));
        mw = fmax(mw, fabs(P - Wg));
        if (P > 0.0) {
            kg += P * log(P / G);
            kw += P * log(P / Wg);
        }
        sum += P;
    }
    s_a[tid] = mg;
    s_b[tid] = kg;
    s_c[tid] = mw;
    s_d[tid] = kw;
    __syncthreads();
    for (int o = FEQB_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o) {
            s_a[tid] = fmax(s_a[tid], s_a[tid + o]);
            s_b[tid] += s_b[tid + o];
            s_c[tid] = fmax(s_c[tid], s_c[tid + o]);
            s_d[tid] += s_d[tid + o];
        }
        __syncthreads();
    }
    // the sum of P goes through the same fixed tree
    if (tid == 0) {
        out[3 * A.nb + 4] = s_a[0];
        out[3 * A.nb + 5] = s_b[0];
        out[3 * A.nb + 6] = s_c[0];
        out[3 * A.nb + 7] = s_d[0];
    }
    __syncthreads();
    s_a[tid] = sum;
    __syncthreads();
    for (int o = FEQB_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o) s_a[tid] += s_a[tid + o];
        __syncthreads();
    }
    if (tid == 0) out[3 * A.nb + 13] = s_a[0];
}

// ---------------------------------------------------------------- bootstrap
// Block-bootstrap standard error of the measured equilibrium of every
// replica: the error-bar blocks of windows that hold data are resampled with
// replacement (as many draws as used blocks), each resample's P_i = drawn
// counts / (n * drawn windows), optionally averaged over i's symmetric set;
// sigma_i = sample standard deviation over the B resamples (divisor B - 1).
// Draw c of replica rep is SplitMix64 (Steele, Lea and Flood 2014) used as a
// counter-based generator: the output function of seed + (c + 1) * gamma,
// gamma = 0x9e3779b97f4a7c15, c = ((rep * 2^20 + b) * 64 + k) for slot k of
// resample b; block = (draw >> 32) * used >> 32.  One CTA per replica, one
// thread per class; every thread walks the resamples in order.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1u) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct BootArgs {
    const RepDev *reps;
    const int32_t *hist;   // [nrep][n_lg][n_dx][MD_NBLK][nb]
    int n_lg, n_dx, lg, dxi, nb, W, sym, B;
    uint64_t seed;
    long long wblk[MD_NBLK];
    double *sigma;         // [nrep][nb]
};

__global__ void k_feq_bootstrap(BootArgs A) {
    __shared__ int s_used[MD_NBLK];
    __shared__ int s_nu;
    const int r = blockIdx.x;
    if (threadIdx.x == 0) {
        int nu = 0;
        for (int k = 0; k < MD_NBLK; ++k)
            if (A.wblk[k] > 0) s_used[nu++] = k;
        s_nu = nu;
    }
    __syncthreads();
    const int nu = s_nu, side = 2 * A.W + 1;
    const double n = (double)A.reps[r].n;
    const int32_t *h = A.hist + ((((long long)r * A.n_lg + A.lg) * A.n_dx + A.dxi) * MD_NBLK) * A.nb;
    for (int i = threadIdx.x; i < A.nb; i += blockDim.x) {
        int mem[8], nm = 0;
        if (A.sym) {
            const int a = abs(i % side - A.W), b = abs(i / side - A.W);
            const int lo = min(a, b), hi = max(a, b);
            for (int j = 0; j < A.nb && nm < 8; ++j) {
                const int c = abs(j % side - A.W), d = abs(j / side - A.W);
                if (min(c, d) == lo && max(c, d) == hi) mem[nm++] = j;
            }
        } else {
            mem[nm++] = i;
        }
        double sig = 0.0;
        if (nu > 0) {
            // two passes over the resamples (mean, then squared deviations),
            // each resample recomputed from its draws
            double mean = 0.0, ss = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                for (int b = 0; b < A.B; ++b) {
                    long long hs = 0, ws = 0;
                    for (int k = 0; k < nu; ++k) {
                        const uint64_t c = (((uint64_t)r << 20) + (uint64_t)b) * 64u + (uint64_t)k;
                        const uint64_t x = splitmix64(A.seed, c);
                        const int u = s_used[(int)(((x >> 32) * (uint64_t)nu) >> 32)];
                        ws += A.wblk[u];
                        for (int m = 0; m < nm; ++m) hs += h[(long long)u * A.nb + mem[m]];
                    }
                    const double P = (double)hs / ((double)nm * n * (double)ws);
                    if (pass == 0) {
                        mean += P;
                    } else {
                        const double d = P - mean;
                        ss = __dadd_rn(ss, __dmul_rn(d, d));   // rounded as the plain definition
                    }
                }
                if (pass == 0) mean /= (double)A.B;
            }
            sig = sqrt(ss / (double)(A.B - 1));
        }
        A.sigma[(long long)r * A.nb + i] = sig;
    }
}

}  // namespace mdlg

using namespace mdlg;

struct md_system {
    int prec = 0, nrep = 0, W = 0, nb = 0, n_lg = 0, n_dx = 0, block_windows = 1;
    int lg_every[MD_MAX_LG] = {0};
    long long n_equil = 0;
    std::vector<RepDev> reps;
    long long ntot = 0;
    int nslots = 0, total_cells = 0;
    cudaStream_t st = nullptr;
    int dev = 0, nsm = 1;
    int block = 256, grid = 1, ppt = 1, K = 16, stage = 1;
    long long chunk_cap = 0;
    int4 *d_chunks = nullptr;
    size_t smem = 0;
    long long step = 0;
    int phase_half = 0;
    std::vector<void *> allocs;
    SysDev sd{};
    RepDev *d_reps = nullptr;
    int32_t *d_gran = nullptr;
    Control *d_ctl = nullptr;
    double *d_epart = nullptr;
    double *d_small = nullptr;   // readout scratch (2*nb + 8 doubles, 4 energy)
    double *d_feq_part = nullptr;   // WSG partial sums of the f_eq stage [nrep][FEQB_SPLIT][nb]
    double *d_feq_par = nullptr;    // per replica mu2, a^2, lambda of the f_eq stage [nrep][4]
    long long *d_hist64 = nullptr;
    int32_t *d_nc_of_id = nullptr;
    // resident engine (md_tune staging 4): plan, buffers, launch shape; the
    // global engine's cell lists need a sort-only rebuild after its launches
    int engine = 0;                   // 0 = k_md_persistent, 1 = k_md_resident
    bool needs_sort = false;
    // the neighbour lists' layout depends on the launch shape (staged: slot
    // order; global: sorted within each chunk of the chunk table), so a new
    // shape's first launch rebuilds them (sort only)
    bool lists_valid = false;
    std::vector<void *> res_allocs;
    ResDev rd{};
    int res_grid = 0;
    size_t res_smem = 0;
    int res_slabs = 0, res_max_g = 0;
    std::vector<ResJob> res_jobs;     // the plan's slabs, in device order
    std::vector<double> res_cost;     // measured per-replica slab times of the current plan, if any
};

namespace {

int dalloc(md_system *s, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(MD_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    s->allocs.push_back(*p);
    return MD_OK;
}

// staging 3 = global staging with the full-occupancy register budget (FP32
// only; in FP64 it is the same kernel as staging 2)
const void *persistent_fn(int prec, int block, int stage) {
    if (prec == MD_FP64)
        return block == 128 ? (const void *)k_md_persistent<double, 128, false>
                            : (const void *)k_md_persistent<double, 256, false>;
    if (stage == 3)
        return block == 128 ? (const void *)k_md_persistent<float, 128, true>
                            : (const void *)k_md_persistent<float, 256, true>;
    return block == 128 ? (const void *)k_md_persistent<float, 128, false>
                        : (const void *)k_md_persistent<float, 256, false>;
}

// Per-replica constants from the parameters (slot, cell and id bases are
// set by the caller).
RepDev make_rep(const md_params &q, int prec, int n_dx) {
    RepDev R{};
    R.nc = (int)std::floor(q.box_L / (q.rc + q.skin));
    double h = q.box_L / R.nc;
    if (prec == MD_FP32_CELLOFF) h = (double)(float)h;
    R.h = h;
    R.L = (double)R.nc * h;
    R.n = (int)q.n;
    R.cap = (int)((q.n + SLOT_PAD - 1) / SLOT_PAD * SLOT_PAD);
    R.dt = q.dt;
    R.hk = q.dt / (2.0 * q.mass);
    R.rc2 = q.rc * q.rc;
    R.eps = q.eps;
    R.sig2 = q.sigma * q.sigma;
    const double sc2 = q.sigma * q.sigma / (q.rc * q.rc), sc6 = sc2 * sc2 * sc2;
    R.vshift = 4.0 * q.eps * (sc6 * sc6 - sc6);
    R.mass = q.mass;
    R.rv2 = (q.rc + q.skin) * (q.rc + q.skin);
    R.half_skin = 0.5 * q.skin;
    for (int d = 0; d < n_dx; ++d) {
        R.lx[d] = q.lx[d];
        R.dxl[d] = R.L / (double)q.lx[d];
        R.dxl_invf[d] = (float)(1.0 / R.dxl[d]);
    }
    R.hf = (float)h;
    R.dtf = (float)R.dt;
    R.hkf = (float)R.hk;
    R.rc2f = (float)R.rc2;
    R.epsf = (float)R.eps;
    R.sig2f = (float)R.sig2;
    R.rv2f = (float)R.rv2;
    return R;
}

// ---- resident engine plan -------------------------------------------------
// Cuts every replica into g slabs of whole MD-cell rows, the fewest that fit
// one CTA's shared memory each with room to spare (particles 1.2x the
// expected count of the largest slab plus 64, halo rows twice the mean row
// population plus 64, list entries 1.8x the mean neighbour count within
// rc + skin), then deals the slabs to `grid` CTAs by list scheduling: the
// replicas in order of decreasing g and estimated time, each on the
// contiguous CTA range that frees up first.  Every CTA runs its slabs in
// order of their planned start, so the slabs of one replica meet in the
// same order on all their CTAs (no cycle of waits).
struct ResPlan {
    std::vector<ResJob> jobs;        // by CTA, in execution order
    std::vector<int32_t> start;      // [grid + 1]
    int hmax = 0, slabs = 0, max_g = 0;
    double makespan = 0.0;
};

static int round_up(long long v, int m) { return (int)((v + m - 1) / m * m); }

int plan_resident(const std::vector<RepDev> &all, int grid, size_t avail, ResPlan &P,
                  const std::vector<double> *measured = nullptr) {
    struct Rep {
        int r, g, p_cap, h_cap;
        double cost;
    };
    std::vector<Rep> reps;
    for (int r = 0; r < (int)all.size(); ++r) {
        const RepDev &R = all[r];
        const double dens = (double)R.n / (R.L * R.L);
        const double cbar = M_PI * R.rv2 * dens;
        const double rowpop = (double)R.n / R.nc;
        Rep best{r, 0, 0, 0, 0.0};
        for (int g = 1; g <= 1024; ++g) {
            if (g > 1 && (R.nc / g < 2 || g > R.cap / 32)) break;
            const int rows = (R.nc + g - 1) / g;
            if ((g == 1 ? R.nc : rows + 2) > RES_NCC) continue;
            const double pmax = (double)R.n * rows / R.nc;
            const double want = 1.2 * pmax + 64.0;
            if (want > RES_PCAP) continue;
            const int p_cap = std::min(RES_PCAP, round_up((long long)std::ceil(want), 32));
            const int h_cap = g == 1 ? 0 : std::min(4096, round_up((long long)std::ceil(2.0 * rowpop + 64.0), 32));
            if (p_cap + 2 * h_cap > (int)RES_IDX + 1) continue;   // 14-bit list indices
            const long long e_need = (long long)std::ceil(1.8 * cbar * p_cap) + 256;
            if (res_slab_bytes(p_cap, h_cap, (int)std::min<long long>(e_need, 1 << 30)) > avail) continue;
            best = Rep{r, g, p_cap, h_cap, pmax * (40.0 + 14.0 * cbar) + (g > 1 ? 4000.0 : 0.0)};
            // a measured time of the replica's slabs replaces the model
            if (measured && r < (int)measured->size() && (*measured)[r] > 0.0) best.cost = (*measured)[r];
            break;
        }
        if (best.g == 0)
            return fail(MD_E_LIMIT, "resident engine: replica %d (n = %d, %d cell rows) fits no slab plan", r, R.n,
                        R.nc);
        reps.push_back(best);
    }
    std::stable_sort(reps.begin(), reps.end(), [](const Rep &a, const Rep &b) {
        return a.g != b.g ? a.g > b.g : a.cost > b.cost;
    });
    std::vector<double> free_at(grid, 0.0);
    struct Placed {
        double t;
        ResJob j;
    };
    std::vector<std::vector<Placed>> per_cta(grid);
    P.hmax = 32;
    P.slabs = 0;
    P.max_g = 0;
    for (const Rep &q : reps) {
        if (q.g > grid) return fail(MD_E_LIMIT, "resident engine: replica %d needs %d CTAs > %d", q.r, q.g, grid);
        int c0 = 0;
        double best_t = 1e300, best_idle = 1e300;
        for (int c = 0; c + q.g <= grid; ++c) {
            double t = 0.0;
            for (int k = 0; k < q.g; ++k) t = std::max(t, free_at[c + k]);
            double idle = 0.0;
            for (int k = 0; k < q.g; ++k) idle += t - free_at[c + k];
            if (t < best_t || (t == best_t && idle < best_idle)) {
                best_t = t;
                best_idle = idle;
                c0 = c;
            }
        }
        const RepDev &R = all[q.r];
        for (int k = 0; k < q.g; ++k) {
            ResJob j;
            j.rep = q.r;
            j.g = q.g;
            j.k = k;
            j.r0 = (int)((long long)k * R.nc / q.g);
            j.r1 = (int)((long long)(k + 1) * R.nc / q.g);
            j.p_cap = q.p_cap;
            j.h_cap = q.h_cap;
            j.cta0 = c0;
            per_cta[c0 + k].push_back(Placed{best_t, j});
            free_at[c0 + k] = best_t + q.cost;
        }
        P.hmax = std::max(P.hmax, q.h_cap);
        P.slabs += q.g;
        P.max_g = std::max(P.max_g, q.g);
    }
    P.jobs.clear();
    P.start.assign(grid + 1, 0);
    P.makespan = 0.0;
    for (int c = 0; c < grid; ++c) {
        std::stable_sort(per_cta[c].begin(), per_cta[c].end(),
                         [](const Placed &a, const Placed &b) { return a.t < b.t; });
        P.start[c] = (int)P.jobs.size();
        for (const Placed &x : per_cta[c]) P.jobs.push_back(x.j);
        P.makespan = std::max(P.makespan, free_at[c]);
    }
    P.start[grid] = (int)P.jobs.size();
    return MD_OK;
}

void free_resident(md_system *s) {
    for (void *p : s->res_allocs) cudaFree(p);
    s->res_allocs.clear();
    s->rd = ResDev{};
    s->res_grid = 0;
}

int configure_resident(md_system *s, const std::vector<double> *measured = nullptr) {
    if (s->prec != MD_FP32_CELLOFF) return fail(MD_E_ARG, "the resident engine (staging 4) is FP32 only");
    int optin = 0, per_sm = 0;
    MD_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->dev));
    MD_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->dev));
    cudaFuncAttributes fa{};
    MD_CUDA_TRY(cudaFuncGetAttributes(&fa, k_md_resident));
    // RES_CTAS_PER_SM CTAs share an SM's shared memory (1 KB of it is
    // reserved per CTA)
    const size_t smem = std::min((size_t)optin, (size_t)per_sm / RES_CTAS_PER_SM - 1024) - fa.sharedSizeBytes;
    const size_t hb = smem_hist_bytes(s->n_lg, s->n_dx, s->nb);
    if (hb + 4096 > smem) return fail(MD_E_LIMIT, "resident engine: histograms leave no shared memory");
    MD_CUDA_TRY(cudaFuncSetAttribute(k_md_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    MD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_md_resident, RES_THREADS, smem));
    if (occ < RES_CTAS_PER_SM) return fail(MD_E_CUDA, "resident kernel: %d of %d CTAs fit on an SM", occ, RES_CTAS_PER_SM);
    const int grid = s->nsm * RES_CTAS_PER_SM;
    ResPlan P;
    int rc = plan_resident(s->reps, grid, smem - hb, P, measured);
    if (rc) return rc;
    MD_CUDA_TRY(cudaStreamSynchronize(s->st));   // no launch may still use the old buffers
    free_resident(s);
    ResDev &D = s->rd;
    auto A = [&](void **ptr, size_t bytes) {
        if (rc) return;
        if (cudaMalloc(ptr, bytes ? bytes : 16) != cudaSuccess) {
            *ptr = nullptr;
            rc = fail(MD_E_NOMEM, "resident engine: cudaMalloc(%zu)", bytes);
            return;
        }
        s->res_allocs.push_back(*ptr);
    };
    const size_t hm = (size_t)P.hmax;
    A((void **)&D.jobs, sizeof(ResJob) * P.jobs.size());
    A((void **)&D.job_start, sizeof(int32_t) * P.start.size());
    A((void **)&D.halo_off, sizeof(float2) * grid * 4 * hm);
    A((void **)&D.halo_ci, sizeof(uint2) * grid * 2 * hm);
    A((void **)&D.halo_n, sizeof(int32_t) * grid * 2);
    A((void **)&D.mig_a, sizeof(float4) * grid * 2 * hm);
    A((void **)&D.mig_b, sizeof(uint2) * grid * 2 * hm);
    A((void **)&D.mig_n, sizeof(int32_t) * grid * 2);
    A((void **)&D.slab_n, sizeof(int32_t) * grid);
    A((void **)&D.gbar, sizeof(unsigned) * 2 * (size_t)s->nrep);
    A((void **)&D.job_ns, sizeof(unsigned long long) * std::max<size_t>(1, P.jobs.size()));
    if (rc) {
        free_resident(s);
        return rc;
    }
    D.hmax = P.hmax;
    D.smem_bytes = (int)smem;
    MD_CUDA_TRY(cudaMemcpyAsync((void *)D.jobs, P.jobs.data(), sizeof(ResJob) * P.jobs.size(),
                                cudaMemcpyHostToDevice, s->st));
    MD_CUDA_TRY(cudaMemcpyAsync((void *)D.job_start, P.start.data(), sizeof(int32_t) * P.start.size(),
                                cudaMemcpyHostToDevice, s->st));
    MD_CUDA_TRY(cudaMemsetAsync(D.gbar, 0, sizeof(unsigned) * 2 * (size_t)s->nrep, s->st));
    s->res_grid = grid;
    s->res_smem = smem;
    s->res_slabs = P.slabs;
    s->res_max_g = P.max_g;
    s->res_jobs = P.jobs;
    s->res_cost = measured ? *measured : std::vector<double>();
    s->engine = 1;   // the global engine keeps its own launch shape for its other uses
    return MD_OK;
}

int launch_resident(md_system *s, long long nsteps) {
    for (long long done = 0; done < nsteps;) {
        long long step0 = s->step + done;
        long long n = std::min(RES_MAX_STEPS, nsteps - done);
        int phase = done ? 1 : s->phase_half;
        void *args[] = {&s->sd, &s->rd, &step0, &n, &phase};
        MD_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_md_resident, dim3(s->res_grid), dim3(RES_THREADS),
                                                args, s->res_smem, s->st));
        k_res_flip<<<1, 1, 0, s->st>>>(s->d_ctl);
        MD_CUDA_TRY(cudaGetLastError());
        done += n;
    }
    s->needs_sort = true;
    return MD_OK;
}

int configure_launch(md_system *s, int block, int ppt, int stage) {
    if (stage == 4) return configure_resident(s);
    if (block != 128 && block != 256) return fail(MD_E_ARG, "block_threads must be 128 or 256");
    if (ppt < 1 || ppt > 8) return fail(MD_E_ARG, "per_thread must be in [1, 8]");
    if (stage < 1 || stage > 3) return fail(MD_E_ARG, "staging must be 1, 2, 3 or 4");
    const void *fn = persistent_fn(s->prec, block, stage);
    const int chunk = ppt * block;
    // chunk table: ppt*block consecutive slots of one replica
    std::vector<int4> ch;
    for (int r = 0; r < s->nrep; ++r) {
        const RepDev &R = s->reps[r];
        for (int a = R.pbase; a < R.pbase + R.n; a += chunk)
            ch.push_back(make_int4(r, a, std::min(a + chunk, R.pbase + R.n), 0));
    }
    if ((long long)ch.size() > s->chunk_cap) return fail(MD_E_LIMIT, "chunk table overflow");
    const long long nch = (long long)ch.size();
    const size_t smem = s->prec == MD_FP64
                            ? smem_bytes<double>(s->n_lg, s->n_dx, s->nb, chunk, stage == 1)
                            : smem_bytes<float>(s->n_lg, s->n_dx, s->nb, chunk, stage == 1);
    if (smem > 227 * 1024) return fail(MD_E_LIMIT, "shared memory per CTA exceeds 227 KB");
    MD_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    MD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, smem));
    if (occ < 1) return fail(MD_E_CUDA, "persistent kernel does not fit on an SM");
    const long long maxco = (long long)occ * s->nsm;
    // Every SM gets the same number of CTAs (the full resident grid, unless
    // there are fewer chunks): an SM finishes a step's force pass when all of
    // its CTAs' work is done, so an SM with one CTA more would set the pace
    // of the grid barrier.  The chunk dealing below evens out the per-CTA sums.
    const long long q = (nch + maxco - 1) / maxco;
    const long long grid = std::min<long long>(4096, std::max<long long>(1, std::min<long long>(maxco, nch)));
    if (q > MAX_CPC) return fail(MD_E_LIMIT, "more than %d chunks per CTA: raise per_thread", MAX_CPC);
    // CTA b owns table entries b, b + grid, b + 2 grid, ... (staged shapes;
    // also the sampling pass and the sort of a rebuild).  Chunks differ in
    // cost by the replicas' densities (neighbours per particle), so they are
    // dealt by decreasing estimated cost, the CTA order reversed every other
    // round, which evens out the per-CTA sums and the wait at the step's grid
    // barrier.  The dynamic distribution of the global-memory shapes takes
    // the chunks in table order, so the costliest come first.  Which CTA
    // computes a chunk does not change any result.
    {
        std::vector<double> cost(nch);
        for (long long k = 0; k < nch; ++k) {
            const RepDev &R = s->reps[ch[k].x];
            const double nbr = M_PI * R.rv2 * (double)R.n / (R.L * R.L);
            cost[k] = (double)(ch[k].z - ch[k].y) * (6.0 + nbr);
        }
        std::vector<long long> order(nch);
        for (long long k = 0; k < nch; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(),
                         [&](long long a, long long b) { return cost[a] > cost[b]; });
        std::vector<int4> dealt(nch);
        for (long long k = 0; k < nch; ++k) {
            const long long round = k / grid, w = k % grid;
            const bool full = (round + 1) * grid <= nch;
            const long long b = (full && (round & 1)) ? grid - 1 - w : w;
            dealt[round * grid + b] = ch[order[k]];
        }
        ch.swap(dealt);
    }
    MD_CUDA_TRY(cudaMemcpyAsync(s->d_chunks, ch.data(), sizeof(int4) * ch.size(),
                                cudaMemcpyHostToDevice, s->st));
    s->smem = smem;
    s->grid = (int)grid;
    s->block = block;
    s->ppt = ppt;
    s->sd.chunks = s->d_chunks;
    s->sd.nchunks = (int)nch;
    // global-memory shapes: the later half of the dealing's rounds (its
    // cheapest chunks) is claimed (a measured choice on a 256-replica batch:
    // a third and a half claimed about equal, none or all 3-10 % slower)
    {
        const long long rounds = (nch + grid - 1) / grid;
        const long long keep = stage == 1 ? rounds : rounds / 2;
        // the shared work word holds a claimed chunk's index in 22 bits
        s->sd.nstatic = (int)std::min<long long>(nch, std::max(keep * grid, nch - (1ll << 21)));
    }
    s->sd.ppt = ppt;
    s->sd.stage = stage == 1;
    s->stage = stage;
    s->engine = 0;
    s->lists_valid = false;   // chunk table and list layout change with the shape
    return MD_OK;
}

int launch_persistent(md_system *s, long long nsteps, int force_rebuild);

// The global engine's invariants (slots sorted by cell, by id inside a cell,
// cell_start, Verlet lists) after a resident launch: a sort-only rebuild,
// which moves no particle's cell and changes no value.
int ensure_sorted(md_system *s) {
    if (!s->needs_sort) return MD_OK;
    s->needs_sort = false;
    return launch_persistent(s, 0, RB_NONE);
}

int launch_persistent(md_system *s, long long nsteps, int force_rebuild) {
    if (force_rebuild != RB_ALL) {
        if (s->needs_sort || !s->lists_valid) force_rebuild = RB_NONE;
        s->needs_sort = false;
    } else {
        s->needs_sort = false;
    }
    s->lists_valid = true;
    const void *fn = persistent_fn(s->prec, s->block, s->stage);
    long long step0 = s->step;
    int phase = s->phase_half;
    void *args[] = {&s->sd, &step0, &nsteps, &phase, &force_rebuild};
    MD_CUDA_TRY(cudaMemsetAsync(&s->d_ctl->claims, 0, sizeof(unsigned long long), s->st));
    MD_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(s->grid), dim3(s->block), args, s->smem, s->st));
    return MD_OK;
}

int status_to_code(int ds) {
    if (ds & DS_TIMEOUT) return fail(MD_E_TIMEOUT, "device barrier wait timed out");
    if (ds & DS_CAPACITY)
        return fail(MD_E_LIMIT, "resident engine: a slab outgrew its planned capacity (state undefined)");
    if (ds & DS_NONFINITE) return fail(MD_E_NONFINITE, "non-finite position encountered");
    if (ds & DS_SKIN) return fail(MD_E_SKIN, "a particle moved more than one cell in one step");
    if (ds & DS_NBR_OVERFLOW)
        return fail(MD_E_LIMIT, "neighbour list overflow: raise md_params.nbr_max");
    return MD_OK;
}

int sync_status(md_system *s) {
    MD_CUDA_TRY(cudaStreamSynchronize(s->st));
    int ds = 0;
    MD_CUDA_TRY(cudaMemcpy(&ds, &s->d_ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (ds) {
        MD_CUDA_TRY(cudaMemset(&s->d_ctl->status, 0, sizeof(int)));
        // a wait that gave up leaves the arrival count behind; no kernel of
        // the system runs now, so it is cleared for the next launch
        if (ds & DS_TIMEOUT) MD_CUDA_TRY(cudaMemset(&s->d_ctl->bar_count, 0, sizeof(unsigned)));
        if ((ds & (DS_TIMEOUT | DS_CAPACITY)) && s->rd.gbar)
            MD_CUDA_TRY(cudaMemset(s->rd.gbar, 0, sizeof(unsigned) * 2 * (size_t)s->nrep));
        return status_to_code(ds);
    }
    return MD_OK;
}

int check_params(const md_params *p, int r, const md_params *p0) {
    if (p->n < 2 || p->n > (1ll << 30)) return fail(MD_E_ARG, "replica %d: n out of [2, 2^30]", r);
    if (!(p->box_L > 0) || !(p->dt > 0) || !(p->rc > 0) || !(p->sigma > 0) || !(p->mass > 0) ||
        !(p->eps >= 0) || !(p->skin > 0))
        return fail(MD_E_ARG, "replica %d: box_L, dt, rc, sigma, mass, skin must be > 0, eps >= 0", r);
    if (p->precision != MD_FP64 && p->precision != MD_FP32_CELLOFF)
        return fail(MD_E_ARG, "replica %d: unknown precision", r);
    if (p->W < 1 || p->W > MD_MAX_W) return fail(MD_E_ARG, "W out of [1,%d]", MD_MAX_W);
    if (p->n_lg < 0 || p->n_lg > MD_MAX_LG) return fail(MD_E_ARG, "n_lg out of [0,%d]", MD_MAX_LG);
    if (p->n_dx < 1 || p->n_dx > MD_MAX_DX) return fail(MD_E_ARG, "n_dx out of [1,%d]", MD_MAX_DX);
    for (int k = 0; k < p->n_lg; ++k)
        if (p->lg_every[k] < 1) return fail(MD_E_ARG, "lg_every[%d] must be >= 1", k);
    for (int d = 0; d < p->n_dx; ++d)
        if (p->lx[d] < 1) return fail(MD_E_ARG, "replica %d: lx[%d] must be >= 1", r, d);
    if (p->n_equil < 0) return fail(MD_E_ARG, "n_equil must be >= 0");
    if (p->block_windows < 1) return fail(MD_E_ARG, "block_windows must be >= 1");
    const long long nc = (long long)std::floor(p->box_L / (p->rc + p->skin));
    if (nc < 3) return fail(MD_E_ARG, "replica %d: box must hold >= 3 cells of rc+skin", r);
    if (nc > 32767) return fail(MD_E_LIMIT, "replica %d: more than 32767 cells per edge", r);
    if (p0) {
        if (p->precision != p0->precision || p->W != p0->W || p->n_equil != p0->n_equil ||
            p->n_lg != p0->n_lg || p->n_dx != p0->n_dx || p->block_windows != p0->block_windows)
            return fail(MD_E_ARG, "replica %d: batch-wide parameters differ from replica 0", r);
        for (int k = 0; k < p->n_lg; ++k)
            if (p->lg_every[k] != p0->lg_every[k])
                return fail(MD_E_ARG, "replica %d: lg_every differs from replica 0", r);
    }
    return MD_OK;
}

int observe(md_system *s, ObsArgs a);

int upload_state(md_system *s, const double *x, const double *y, const double *vx,
                 const double *vy) {
    if (!x || !y || !vx || !vy) return fail(MD_E_ARG, "state arrays must not be NULL");
    const size_t bytes = sizeof(double) * (size_t)s->ntot;
    double *tmp = nullptr;
    MD_CUDA_TRY(cudaMallocAsync((void **)&tmp, 4 * bytes, s->st));
    int rc = MD_OK;
    const double *src[4] = {x, y, vx, vy};
    for (int k = 0; k < 4 && rc == MD_OK; ++k) {
        cudaError_t e = cudaMemcpyAsync(tmp + k * s->ntot, src[k], bytes, cudaMemcpyDefault, s->st);
        if (e != cudaSuccess) rc = fail(MD_E_CUDA, "state upload: %s", cudaGetErrorString(e));
    }
    if (rc == MD_OK) {
        // fresh cell list: positions go to set 0, buffer 0
        cudaMemsetAsync(&s->d_ctl->set, 0, 2 * sizeof(int), s->st);
        const int nthr = 256;
        const int nblk = (s->nslots + nthr - 1) / nthr;
        if (s->prec == MD_FP64)
            k_init<double><<<nblk, nthr, 0, s->st>>>(s->sd, tmp, tmp + s->ntot, tmp + 2 * s->ntot,
                                                     tmp + 3 * s->ntot);
        else
            k_init<float><<<nblk, nthr, 0, s->st>>>(s->sd, tmp, tmp + s->ntot, tmp + 2 * s->ntot,
                                                    tmp + 3 * s->ntot);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = fail(MD_E_CUDA, "init kernel: %s", cudaGetErrorString(e));
    }
    if (rc == MD_OK) rc = launch_persistent(s, 0, 1);
    cudaFreeAsync(tmp, s->st);
    if (rc) return rc;
    s->phase_half = 0;
    // a state placed on a sampling boundary starts the next window there
    unsigned mask = 0;
    for (int k = 0; k < s->n_lg; ++k)
        if (s->step >= s->n_equil && (s->step - s->n_equil) % s->lg_every[k] == 0) mask |= 1u << k;
    if (mask) {
        ObsArgs a{};
        a.snap_mask = mask;
        rc = observe(s, a);
        if (rc) return rc;
    }
    return sync_status(s);
}

// Runs the observation kernel; completes the half kick when needed.
int observe(md_system *s, ObsArgs a) {
    int rc = ensure_sorted(s);
    if (rc) return rc;
    a.complete = s->phase_half;
    const int nthr = 256;
    const int nblk = s->nslots / nthr;
    if (s->prec == MD_FP64)
        k_observe<double><<<nblk, nthr, 0, s->st>>>(s->sd, a);
    else
        k_observe<float><<<nblk, nthr, 0, s->st>>>(s->sd, a);
    MD_CUDA_TRY(cudaGetLastError());
    s->phase_half = 0;
    return MD_OK;
}

// Particles per thread in a chunk: one, i.e. chunks of one block, which
// keeps the staging buffers small and deals the most chunks round-robin.
int default_ppt(const md_system *) { return 1; }

long long windows_done(const md_system *s, int k) {
    const long long t = s->step - s->n_equil;
    if (t < 0) return 0;
    return t / s->lg_every[k];
}

}  // namespace

extern "C" {

int md_init_batch(const md_params *p, int32_t n_rep, const double *x, const double *y,
                  const double *vx, const double *vy, void *stream, md_system **out) {
    mdlg::Range range_("md_init_batch");
    if (!p || !out || n_rep < 1) return fail(MD_E_ARG, "md_init_batch: bad arguments");
    if (n_rep > MD_MAX_REP) return fail(MD_E_LIMIT, "md_init_batch: more than %d replicas", MD_MAX_REP);
    *out = nullptr;
    for (int r = 0; r < n_rep; ++r) {
        int rc = check_params(&p[r], r, r ? &p[0] : nullptr);
        if (rc) return rc;
    }
    md_system *s = new md_system();
    s->st = (cudaStream_t)stream;
    s->prec = p[0].precision;
    s->nrep = n_rep;
    s->W = p[0].W;
    s->nb = (2 * s->W + 1) * (2 * s->W + 1);
    s->n_lg = p[0].n_lg;
    s->n_dx = p[0].n_dx;
    s->block_windows = p[0].block_windows;
    s->n_equil = p[0].n_equil;
    for (int k = 0; k < s->n_lg; ++k) s->lg_every[k] = p[0].lg_every[k];
    long long pbase = 0, cbase = 0, ibase = 0;
    for (int r = 0; r < n_rep; ++r) {
        const md_params &q = p[r];
        RepDev R = make_rep(q, s->prec, s->n_dx);
        R.pbase = (int)pbase;
        R.cbase = (int)cbase;
        R.ibase = (int)ibase;
        s->reps.push_back(R);
        pbase += R.cap;
        cbase += (long long)R.nc * R.nc + 1;
        ibase += q.n;
    }
    if (pbase >= (1ll << 31) - SLOT_PAD || cbase >= (1ll << 31) - 1) {
        delete s;
        return fail(MD_E_LIMIT, "md_init_batch: more than 2^31 slots or cells");
    }
    // neighbour-list capacity: three times the mean count within rv plus
    // eight standard deviations (clustered replicas), or the caller's value
    double kmax = 16.0;
    for (int r = 0; r < n_rep; ++r) {
        const md_params &q = p[r];
        const double rv = q.rc + q.skin;
        const double mean = M_PI * rv * rv * (double)q.n / (s->reps[r].L * s->reps[r].L);
        kmax = std::max(kmax, 3.0 * mean + 8.0 * std::sqrt(mean) + 8.0);
        if (q.nbr_max > 0) kmax = std::max(kmax, (double)q.nbr_max);
    }
    s->K = (int)std::min(1024.0, std::ceil(kmax / 4.0) * 4.0);
    s->nslots = (int)pbase;
    s->total_cells = (int)cbase;
    s->ntot = ibase;
    int rc = MD_OK;
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->dev);
    if (e != cudaSuccess) {
        delete s;
        return fail(MD_E_CUDA, "md_init_batch: %s", cudaGetErrorString(e));
    }
    const size_t vsz = s->prec == MD_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t ns = (size_t)s->nslots, nlg = (size_t)std::max(1, s->n_lg);
    const size_t ngr = ns / 32;
    SysDev &S = s->sd;
#define ALLOC(ptr, bytes) \
    if (rc == MD_OK) rc = dalloc(s, (void **)&(ptr), (bytes))
    ALLOC(s->d_reps, sizeof(RepDev) * n_rep);
    ALLOC(s->d_gran, sizeof(int32_t) * (ns / GRAN));
    ALLOC(s->d_ctl, sizeof(Control));
    for (int k = 0; k < 2; ++k) {
        ALLOC(S.cell[k], sizeof(uint32_t) * ns);
        ALLOC(S.pid[k], sizeof(int32_t) * ns);
        ALLOC(S.vel[k], vsz * ns);
        ALLOC(S.pos[k][0], vsz * ns);
        ALLOC(S.pos[k][1], vsz * ns);
    }
    ALLOC(S.cellcnt, sizeof(int32_t) * s->total_cells);
    ALLOC(S.cell_start, sizeof(int32_t) * (s->total_cells + 1));
    ALLOC(S.newcell, sizeof(int32_t) * ns);
    ALLOC(S.rank, sizeof(int32_t) * ns);
    ALLOC(S.perm, sizeof(int32_t) * ns);
    ALLOC(S.nbr, sizeof(uint32_t) * ns * (size_t)s->K);
    ALLOC(S.nn, sizeof(int32_t) * (ns + 16));   // staged four at a time
    ALLOC(S.cnt_id, sizeof(int32_t) * (size_t)s->ntot);
    s->chunk_cap = (long long)(ns / 128) + n_rep + 1;
    ALLOC(s->d_chunks, sizeof(int4) * s->chunk_cap);
    ALLOC(S.blocksum, sizeof(int32_t) * 4096);
    ALLOC(S.snap_cell, sizeof(uint32_t) * nlg * s->ntot);
    ALLOC(S.snap_off, vsz * nlg * s->ntot);
    const size_t nhist = (size_t)n_rep * nlg * s->n_dx * MD_NBLK * s->nb;
    ALLOC(S.hist, sizeof(int32_t) * nhist);
    ALLOC(S.ovf, sizeof(unsigned long long) * n_rep * nlg * s->n_dx);
    ALLOC(S.mom, sizeof(double) * ngr * nlg * 2);
    ALLOC(S.vmax_rep, sizeof(unsigned) * 3 * (size_t)n_rep);
    ALLOC(S.disp_rep, sizeof(double) * (size_t)n_rep);
    ALLOC(s->d_epart, sizeof(double) * ngr * 4);
    ALLOC(s->d_small, sizeof(double) * (2 * s->nb + 16));
    ALLOC(s->d_feq_part, sizeof(double) * (size_t)n_rep * FEQB_SPLIT * s->nb);
    ALLOC(s->d_feq_par, sizeof(double) * 4 * (size_t)n_rep);
    ALLOC(s->d_hist64, sizeof(long long) * s->nb);
    ALLOC(s->d_nc_of_id, sizeof(int32_t) * s->ntot);
#undef ALLOC
    if (rc) {
        md_destroy(s);
        return rc;
    }
    std::vector<int32_t> gran(ns / GRAN);
    for (int r = 0; r < n_rep; ++r)
        for (int g = s->reps[r].pbase / GRAN; g < (s->reps[r].pbase + s->reps[r].cap) / GRAN; ++g)
            gran[g] = r;
    S.reps = s->d_reps;
    S.gran_rep = s->d_gran;
    S.ctl = s->d_ctl;
    S.nslots = s->nslots;
    S.nrep = n_rep;
    S.total_cells = s->total_cells;
    S.n_lg = s->n_lg;
    S.n_dx = s->n_dx;
    S.W = s->W;
    S.nb = s->nb;
    S.block_windows = s->block_windows;
    S.n_equil = s->n_equil;
    for (int k = 0; k < MD_MAX_LG; ++k) S.lg_every[k] = s->lg_every[k];
    S.ntot = s->ntot;
    S.K = s->K;
    S.timeout_ns = 4000000000ull;
    S.dbg_leave_cta = -1;
    auto tryc = [&](cudaError_t er) {
        if (er != cudaSuccess && rc == MD_OK) rc = fail(MD_E_CUDA, "md_init_batch: %s", cudaGetErrorString(er));
    };
    tryc(cudaMemcpyAsync(s->d_reps, s->reps.data(), sizeof(RepDev) * n_rep, cudaMemcpyHostToDevice, s->st));
    tryc(cudaMemcpyAsync(s->d_gran, gran.data(), sizeof(int32_t) * gran.size(), cudaMemcpyHostToDevice, s->st));
    tryc(cudaMemsetAsync(s->d_ctl, 0, sizeof(Control), s->st));
    tryc(cudaMemsetAsync(S.perm, 0xff, sizeof(int32_t) * ns, s->st));   // padding slots: -1
    tryc(cudaMemsetAsync(S.nn, 0, sizeof(int32_t) * (ns + 16), s->st));
    tryc(cudaMemsetAsync(S.cnt_id, 0, sizeof(int32_t) * (size_t)s->ntot, s->st));
    tryc(cudaMemsetAsync(S.cellcnt, 0, sizeof(int32_t) * s->total_cells, s->st));
    tryc(cudaMemsetAsync(S.hist, 0, sizeof(int32_t) * nhist, s->st));
    tryc(cudaMemsetAsync(S.ovf, 0, sizeof(unsigned long long) * n_rep * nlg * s->n_dx, s->st));
    tryc(cudaMemsetAsync(S.mom, 0, sizeof(double) * ngr * nlg * 2, s->st));
    tryc(cudaMemsetAsync(S.vmax_rep, 0, sizeof(unsigned) * 3 * (size_t)n_rep, s->st));
    tryc(cudaMemsetAsync(S.disp_rep, 0, sizeof(double) * (size_t)n_rep, s->st));
    tryc(cudaMemsetAsync(S.snap_cell, 0, sizeof(uint32_t) * nlg * s->ntot, s->st));
    tryc(cudaMemsetAsync(S.snap_off, 0, vsz * nlg * s->ntot, s->st));
    if (rc == MD_OK) {
        k_nc_of_id<<<(s->nslots + 255) / 256, 256, 0, s->st>>>(S, s->d_nc_of_id);
        tryc(cudaGetLastError());
    }
    if (rc == MD_OK) rc = configure_launch(s, 256, default_ppt(s), 1);
    if (rc == MD_OK) rc = upload_state(s, x, y, vx, vy);
    if (rc) {
        md_destroy(s);
        return rc;
    }
    *out = s;
    return MD_OK;
}

int md_resident_plan(const md_params *p, int32_t n_rep, int32_t grid, int64_t smem_bytes, int32_t *jobs_out,
                     int32_t max_jobs, int32_t *start_out, double *makespan) {
    if (!p || n_rep < 1 || n_rep > MD_MAX_REP || grid < 1 || smem_bytes < 4096 || !jobs_out || !start_out ||
        max_jobs < 0)
        return fail(MD_E_ARG, "md_resident_plan: bad arguments");
    std::vector<RepDev> reps;
    for (int r = 0; r < n_rep; ++r) {
        int rc = check_params(&p[r], r, r ? &p[0] : nullptr);
        if (rc) return rc;
        reps.push_back(make_rep(p[r], p[0].precision, p[0].n_dx));
    }
    const int nb = (2 * p[0].W + 1) * (2 * p[0].W + 1);
    const size_t hb = smem_hist_bytes(p[0].n_lg, p[0].n_dx, nb);
    if ((size_t)smem_bytes <= hb) return fail(MD_E_LIMIT, "md_resident_plan: no shared memory left");
    ResPlan P;
    int rc = plan_resident(reps, grid, (size_t)smem_bytes - hb, P);
    if (rc) return rc;
    if ((int)P.jobs.size() > max_jobs) return fail(MD_E_LIMIT, "md_resident_plan: %d slabs > max_jobs", (int)P.jobs.size());
    for (size_t j = 0; j < P.jobs.size(); ++j) {
        const ResJob &J = P.jobs[j];
        const int32_t v[8] = {J.rep, J.g, J.k, J.r0, J.r1, J.p_cap, J.h_cap, J.cta0};
        std::memcpy(jobs_out + 8 * j, v, sizeof(v));
    }
    std::memcpy(start_out, P.start.data(), sizeof(int32_t) * P.start.size());
    if (makespan) *makespan = P.makespan;
    return MD_OK;
}

int md_init(const md_params *p, const double *x, const double *y, const double *vx,
            const double *vy, void *stream, md_system **out) {
    return md_init_batch(p, 1, x, y, vx, vy, stream, out);
}

void md_destroy(md_system *s) {
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    free_resident(s);
    for (void *p : s->allocs) cudaFree(p);
    delete s;
}

int md_step(md_system *s, int64_t nsteps) {
    mdlg::Range range_("md_step");
    if (!s || nsteps < 0) return fail(MD_E_ARG, "md_step: bad arguments");
    if (nsteps == 0) return MD_OK;
    int rc = s->engine == 1 ? launch_resident(s, nsteps) : launch_persistent(s, nsteps, 0);
    if (rc) return rc;
    s->step += nsteps;
    s->phase_half = 1;
    return MD_OK;
}

int md_tune(md_system *s, int32_t block_threads, int32_t per_thread, int32_t staging) {
    if (!s) return fail(MD_E_ARG, "md_tune: NULL system");
    if (block_threads == 0) block_threads = 256;
    if (per_thread == 0) per_thread = default_ppt(s);
    if (staging == 0) staging = 1;
    return configure_launch(s, block_threads, per_thread, staging);
}

// ---- checkpoint ---------------------------------------------------------------
// Layout of a checkpoint (host memory): header, then the arrays in the order
// of ckpt_parts.  The state is stored slot by slot in the current set, sorted
// by cell and by id inside a cell (a resident launch's order is sorted
// first), so a load followed by a sort that moves nothing restores the slot
// order, and with it every later force sum and moment partial.
struct CkptHeader {
    uint64_t magic;
    int64_t step, ntot, n_rebuilds;
    int32_t version, prec, nrep, nslots, n_lg, n_dx, nb, phase_half;
};
constexpr uint64_t CKPT_MAGIC = 0x4d444c4743484b31ull;   // "MDLGCHK1"

struct CkptPart {
    void *dev;
    size_t bytes;
};

static std::vector<CkptPart> ckpt_parts(md_system *s, int set, int cur) {
    const SysDev &S = s->sd;
    const size_t vsz = s->prec == MD_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t ns = (size_t)s->nslots, nlg = (size_t)std::max(1, s->n_lg);
    const size_t nhist = (size_t)s->nrep * nlg * s->n_dx * MD_NBLK * s->nb;
    return {{S.cell[set], sizeof(uint32_t) * ns},
            {S.pid[set], sizeof(int32_t) * ns},
            {S.vel[set], vsz * ns},
            {S.pos[set][cur], vsz * ns},
            {S.disp_rep, sizeof(double) * (size_t)s->nrep},
            {S.snap_cell, sizeof(uint32_t) * nlg * (size_t)s->ntot},
            {S.snap_off, vsz * nlg * (size_t)s->ntot},
            {S.hist, sizeof(int32_t) * nhist},
            {S.ovf, sizeof(unsigned long long) * (size_t)s->nrep * nlg * s->n_dx},
            {S.mom, sizeof(double) * (ns / 32) * nlg * 2}};
}

int md_checkpoint_bytes(md_system *s, int64_t *bytes) {
    if (!s || !bytes) return fail(MD_E_ARG, "md_checkpoint_bytes: NULL argument");
    size_t b = sizeof(CkptHeader);
    for (const CkptPart &p : ckpt_parts(s, 0, 0)) b += p.bytes;
    *bytes = (int64_t)b;
    return MD_OK;
}

int md_checkpoint_save(md_system *s, void *buf) {
    mdlg::Range range_("md_checkpoint_save");
    if (!s || !buf) return fail(MD_E_ARG, "md_checkpoint_save: NULL argument");
    int rc = ensure_sorted(s);
    if (rc) return rc;
    rc = sync_status(s);
    if (rc) return rc;
    Control c;
    MD_CUDA_TRY(cudaMemcpy(&c, s->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost));
    CkptHeader h{};
    h.magic = CKPT_MAGIC;
    h.version = 1;
    h.step = s->step;
    h.ntot = s->ntot;
    h.n_rebuilds = c.n_rebuilds;
    h.prec = s->prec;
    h.nrep = s->nrep;
    h.nslots = s->nslots;
    h.n_lg = s->n_lg;
    h.n_dx = s->n_dx;
    h.nb = s->nb;
    h.phase_half = s->phase_half;
    unsigned char *o = static_cast<unsigned char *>(buf);
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    for (const CkptPart &p : ckpt_parts(s, c.set, c.cur)) {
        MD_CUDA_TRY(cudaMemcpy(o, p.dev, p.bytes, cudaMemcpyDeviceToHost));
        o += p.bytes;
    }
    return MD_OK;
}

int md_checkpoint_load(md_system *s, const void *buf) {
    mdlg::Range range_("md_checkpoint_load");
    if (!s || !buf) return fail(MD_E_ARG, "md_checkpoint_load: NULL argument");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != CKPT_MAGIC || h.version != 1) return fail(MD_E_ARG, "md_checkpoint_load: not a checkpoint");
    if (h.ntot != s->ntot || h.prec != s->prec || h.nrep != s->nrep || h.nslots != s->nslots ||
        h.n_lg != s->n_lg || h.n_dx != s->n_dx || h.nb != s->nb)
        return fail(MD_E_ARG, "md_checkpoint_load: the checkpoint was made by a system of other parameters");
    int rc = sync_status(s);
    if (rc) return rc;
    // the state goes to set 0, buffer 0; then a sort that moves no particle
    MD_CUDA_TRY(cudaMemset(&s->d_ctl->set, 0, 2 * sizeof(int)));
    const unsigned char *o = static_cast<const unsigned char *>(buf) + sizeof(h);
    for (const CkptPart &p : ckpt_parts(s, 0, 0)) {
        MD_CUDA_TRY(cudaMemcpy(p.dev, o, p.bytes, cudaMemcpyHostToDevice));
        o += p.bytes;
    }
    MD_CUDA_TRY(cudaMemcpy(&s->d_ctl->n_rebuilds, &h.n_rebuilds, sizeof(long long), cudaMemcpyHostToDevice));
    MD_CUDA_TRY(cudaMemset(s->d_ctl->vmax, 0, sizeof(s->d_ctl->vmax)));
    MD_CUDA_TRY(cudaMemset(s->sd.vmax_rep, 0, sizeof(unsigned) * 3 * (size_t)s->nrep));
    s->step = h.step;
    s->phase_half = h.phase_half;
    s->needs_sort = true;
    rc = ensure_sorted(s);
    if (rc) return rc;
    return sync_status(s);
}

int md_barrier_selftest(md_system *s, double limit_s) {
    if (!s || !(limit_s > 0.0) || !(limit_s <= 4.0)) return fail(MD_E_ARG, "md_barrier_selftest: bad arguments");
    if (s->grid < 2) return fail(MD_E_ARG, "md_barrier_selftest: needs a launch of at least 2 CTAs");
    int rc = sync_status(s);
    if (rc) return rc;
    const uint64_t keep = s->sd.timeout_ns;
    s->sd.timeout_ns = (uint64_t)(limit_s * 1e9);
    s->sd.dbg_leave_cta = 0;
    rc = launch_persistent(s, 1, 0);   // the global engine's grid barrier
    s->sd.dbg_leave_cta = -1;
    s->sd.timeout_ns = keep;
    if (rc) return rc;
    s->step += 1;
    s->phase_half = 1;
    return sync_status(s);
}

int md_sync(md_system *s) {
    if (!s) return fail(MD_E_ARG, "md_sync: NULL system");
    return sync_status(s);
}

int md_info(md_system *s, md_info_t *o) {
    if (!s || !o) return fail(MD_E_ARG, "md_info: NULL argument");
    MD_CUDA_TRY(cudaStreamSynchronize(s->st));
    Control c;
    MD_CUDA_TRY(cudaMemcpy(&c, s->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost));
    o->n_total = s->ntot;
    o->step = s->step;
    o->n_rebuilds = c.n_rebuilds;
    o->n_rep = s->nrep;
    o->precision = s->prec;
    o->grid_blocks = s->grid;
    o->block_threads = s->block;
    return MD_OK;
}

int md_rep_info(md_system *s, int32_t rep, md_rep_info_t *o) {
    if (!s || !o || rep < 0 || rep >= s->nrep) return fail(MD_E_ARG, "md_rep_info: bad arguments");
    const RepDev &R = s->reps[rep];
    o->n = R.n;
    o->L_eff = R.L;
    o->h = R.h;
    o->ncell = R.nc;
    o->reserved = 0;
    for (int d = 0; d < MD_MAX_DX; ++d) o->dx_eff[d] = d < s->n_dx ? R.dxl[d] : 0.0;
    return MD_OK;
}

int md_get_state(md_system *s, double *x, double *y, double *vx, double *vy) {
    if (!s || !x || !y || !vx || !vy) return fail(MD_E_ARG, "md_get_state: NULL argument");
    const size_t bytes = sizeof(double) * s->ntot;
    double *tmp = nullptr;
    MD_CUDA_TRY(cudaMallocAsync((void **)&tmp, 4 * bytes, s->st));
    ObsArgs a{};
    a.x = tmp;
    a.y = tmp + s->ntot;
    a.vx = tmp + 2 * s->ntot;
    a.vy = tmp + 3 * s->ntot;
    int rc = observe(s, a);
    double *dst[4] = {x, y, vx, vy};
    for (int k = 0; k < 4 && rc == MD_OK; ++k) {
        cudaError_t e = cudaMemcpyAsync(dst[k], tmp + k * s->ntot, bytes, cudaMemcpyDefault, s->st);
        if (e != cudaSuccess) rc = fail(MD_E_CUDA, "md_get_state: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(tmp, s->st);
    if (rc) return rc;
    return sync_status(s);
}

int md_set_state(md_system *s, const double *x, const double *y, const double *vx,
                 const double *vy) {
    if (!s) return fail(MD_E_ARG, "md_set_state: NULL system");
    return upload_state(s, x, y, vx, vy);
}

int md_get_raw(md_system *s, int32_t *cell, void *off_x, void *off_y) {
    if (!s || !cell || !off_x || !off_y) return fail(MD_E_ARG, "md_get_raw: NULL argument");
    ObsArgs a{};
    a.raw_cell = cell;
    a.raw_x = off_x;
    a.raw_y = off_y;
    int rc = observe(s, a);
    if (rc) return rc;
    return sync_status(s);
}

int md_get_snapshot(md_system *s, int32_t lg, int32_t *cell, void *off_x, void *off_y) {
    if (!s || !cell || !off_x || !off_y || lg < 0 || lg >= s->n_lg)
        return fail(MD_E_ARG, "md_get_snapshot: bad arguments");
    const size_t vsz = s->prec == MD_FP64 ? sizeof(double2) : sizeof(float2);
    k_copy_snapshot<<<(unsigned)((s->ntot + 255) / 256), 256, 0, s->st>>>(
        s->sd.snap_cell + (size_t)lg * s->ntot, (const char *)s->sd.snap_off + vsz * lg * s->ntot,
        s->prec == MD_FP64, s->ntot, s->d_nc_of_id, cell, off_x, off_y);
    MD_CUDA_TRY(cudaGetLastError());
    return sync_status(s);
}

int md_forces(md_system *s, double *fx, double *fy, double *fabs_sum) {
    if (!s || !fx || !fy) return fail(MD_E_ARG, "md_forces: NULL argument");
    const size_t bytes = sizeof(double) * s->ntot;
    double *tmp = nullptr;
    MD_CUDA_TRY(cudaMallocAsync((void **)&tmp, 3 * bytes, s->st));
    ObsArgs a{};
    a.fx = tmp;
    a.fy = tmp + s->ntot;
    a.fabs_sum = tmp + 2 * s->ntot;
    int rc = observe(s, a);
    double *dst[3] = {fx, fy, fabs_sum};
    for (int k = 0; k < 3 && rc == MD_OK; ++k) {
        if (!dst[k]) continue;
        cudaError_t e = cudaMemcpyAsync(dst[k], tmp + k * s->ntot, bytes, cudaMemcpyDefault, s->st);
        if (e != cudaSuccess) rc = fail(MD_E_CUDA, "md_forces: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(tmp, s->st);
    if (rc) return rc;
    return sync_status(s);
}

int md_step_forces(md_system *s, int64_t nsteps, double *fx, double *fy) {
    mdlg::Range range_("md_step_forces");
    if (!s || nsteps < 1 || !fx || !fy) return fail(MD_E_ARG, "md_step_forces: bad arguments");
    const size_t bytes = sizeof(double) * s->ntot;
    double *tmp = nullptr;
    MD_CUDA_TRY(cudaMallocAsync((void **)&tmp, 2 * bytes, s->st));
    s->sd.dbg_fx = tmp;
    s->sd.dbg_fy = tmp + s->ntot;
    int rc = md_step(s, nsteps);
    s->sd.dbg_fx = s->sd.dbg_fy = nullptr;
    double *dst[2] = {fx, fy};
    for (int k = 0; k < 2 && rc == MD_OK; ++k) {
        cudaError_t e = cudaMemcpyAsync(dst[k], tmp + k * s->ntot, bytes, cudaMemcpyDefault, s->st);
        if (e != cudaSuccess) rc = fail(MD_E_CUDA, "md_step_forces: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(tmp, s->st);
    if (rc) return rc;
    return sync_status(s);
}

int md_energy(md_system *s, int32_t rep, double *out4) {
    if (!s || !out4 || rep < 0 || rep >= s->nrep) return fail(MD_E_ARG, "md_energy: bad arguments");
    ObsArgs a{};
    a.epart = s->d_epart;
    int rc = observe(s, a);
    if (rc) return rc;
    const RepDev &R = s->reps[rep];
    k_sum_energy<<<1, 256, 0, s->st>>>(s->d_epart, R.pbase / 32, (R.pbase + R.cap) / 32, s->d_small);
    MD_CUDA_TRY(cudaGetLastError());
    MD_CUDA_TRY(cudaMemcpyAsync(out4, s->d_small, 4 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    return sync_status(s);
}

int md_energy_batch(md_system *s, double *out) {
    mdlg::Range range_("md_energy_batch");
    if (!s || !out) return fail(MD_E_ARG, "md_energy_batch: bad arguments");
    ObsArgs a{};
    a.epart = s->d_epart;
    int rc = observe(s, a);
    if (rc) return rc;
    const size_t bytes = sizeof(double) * 4 * (size_t)s->nrep;
    cudaPointerAttributes at{};
    const bool dev = cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    double *dst = out;
    if (!dev) MD_CUDA_TRY(cudaMallocAsync((void **)&dst, bytes, s->st));
    k_sum_energy_batch<<<s->nrep, 256, 0, s->st>>>(s->d_epart, s->d_reps, dst);
    cudaError_t e = cudaGetLastError();
    if (!dev) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, s->st);
        cudaFreeAsync(dst, s->st);
    }
    if (e != cudaSuccess) return fail(MD_E_CUDA, "md_energy_batch: %s", cudaGetErrorString(e));
    return sync_status(s);
}

int md_hist_raw(md_system *s, int32_t rep, int32_t lg, int32_t dxi, int64_t *hist,
                int64_t *overflow, int64_t *n_windows) {
    if (!s || !hist || rep < 0 || rep >= s->nrep || lg < 0 || lg >= s->n_lg || dxi < 0 ||
        dxi >= s->n_dx)
        return fail(MD_E_ARG, "md_hist_raw: bad arguments");
    const size_t base = ((size_t)(rep * s->n_lg + lg) * s->n_dx + dxi);
    k_hist_total<<<1, 256, 0, s->st>>>(s->sd.hist + base * MD_NBLK * s->nb, s->nb, s->d_hist64);
    MD_CUDA_TRY(cudaGetLastError());
    MD_CUDA_TRY(cudaMemcpyAsync(hist, s->d_hist64, sizeof(int64_t) * s->nb, cudaMemcpyDeviceToHost, s->st));
    unsigned long long ov = 0;
    MD_CUDA_TRY(cudaMemcpyAsync(&ov, s->sd.ovf + base, sizeof(ov), cudaMemcpyDeviceToHost, s->st));
    int rc = sync_status(s);
    if (rc) return rc;
    if (overflow) *overflow = (int64_t)ov;
    if (n_windows) *n_windows = windows_done(s, lg);
    return MD_OK;
}

int feq_measured(md_system *s, int32_t rep, int32_t lg, int32_t dxi, int32_t symmetrize,
                 double *P_out, double *stderr_out, md_feq_stats *stats) {
    mdlg::Range range_("feq_measured");
    if (!s || !P_out || rep < 0 || rep >= s->nrep || lg < 0 || lg >= s->n_lg || dxi < 0 ||
        dxi >= s->n_dx)
        return fail(MD_E_ARG, "feq_measured: bad arguments");
    const RepDev &R = s->reps[rep];
    const size_t base = ((size_t)(rep * s->n_lg + lg) * s->n_dx + dxi);
    FeqArgs A{};
    A.hist = s->sd.hist + base * MD_NBLK * s->nb;
    A.ovf = s->sd.ovf + base;
    A.mom = s->sd.mom;
    A.g0 = R.pbase / 32;
    A.g1 = (R.pbase + R.cap) / 32;
    A.n_lg = s->n_lg;
    A.lg = lg;
    A.nb = s->nb;
    A.W = s->W;
    A.sym = symmetrize != 0;
    A.n = (double)R.n;
    A.nwin = windows_done(s, lg);
    int used = 0;
    for (long long w = 0; w < A.nwin; ++w) {
        const int b = (int)((w / s->block_windows) % MD_NBLK);
        if (A.wblk[b]++ == 0) ++used;
    }
    A.dx_eff = R.dxl[dxi];
    A.out = s->d_small;
    k_feq_measured<<<1, FEQ_THREADS, 0, s->st>>>(A);
    MD_CUDA_TRY(cudaGetLastError());
    std::vector<double> h(2 * s->nb + 8);
    MD_CUDA_TRY(cudaMemcpyAsync(h.data(), s->d_small, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s->st));
    int rc = sync_status(s);
    if (rc) return rc;
    std::memcpy(P_out, h.data(), sizeof(double) * s->nb);
    if (stderr_out) std::memcpy(stderr_out, h.data() + s->nb, sizeof(double) * s->nb);
    if (stats) {
        const double *st = h.data() + 2 * s->nb;
        stats->mu2 = st[0];
        stats->mu4 = st[1];
        stats->a2 = st[2];
        stats->dx_eff = A.dx_eff;
        stats->n_windows = A.nwin;
        stats->n_overflow = (int64_t)st[3];
        stats->n_samples = (int64_t)R.n * A.nwin;
        stats->n_blocks_used = used;
    }
    return MD_OK;
}

int md_hist_blocks(md_system *s, int32_t rep, int32_t lg, int32_t dxi, int32_t *hist, int64_t *wblk) {
    if (!s || !hist || !wblk || rep < 0 || rep >= s->nrep || lg < 0 || lg >= s->n_lg || dxi < 0 ||
        dxi >= s->n_dx)
        return fail(MD_E_ARG, "md_hist_blocks: bad arguments");
    const size_t base = ((size_t)(rep * s->n_lg + lg) * s->n_dx + dxi);
    MD_CUDA_TRY(cudaMemcpyAsync(hist, s->sd.hist + base * MD_NBLK * s->nb, sizeof(int32_t) * MD_NBLK * s->nb,
                                cudaMemcpyDeviceToHost, s->st));
    int rc = sync_status(s);
    if (rc) return rc;
    for (int b = 0; b < MD_NBLK; ++b) wblk[b] = 0;
    for (long long w = 0; w < windows_done(s, lg); ++w) wblk[(w / s->block_windows) % MD_NBLK] += 1;
    return MD_OK;
}

int feq_bootstrap(md_system *s, int32_t lg, int32_t dxi, int32_t symmetrize, int32_t n_resamples, uint64_t seed,
                  double *sigma_out) {
    mdlg::Range range_("feq_bootstrap");
    if (!s || !sigma_out || lg < 0 || lg >= s->n_lg || dxi < 0 || dxi >= s->n_dx || n_resamples < 2 ||
        n_resamples > (1 << 20))
        return fail(MD_E_ARG, "feq_bootstrap: bad arguments");
    BootArgs A{};
    A.reps = s->d_reps;
    A.hist = s->sd.hist;
    A.n_lg = s->n_lg;
    A.n_dx = s->n_dx;
    A.lg = lg;
    A.dxi = dxi;
    A.nb = s->nb;
    A.W = s->W;
    A.sym = symmetrize != 0;
    A.B = n_resamples;
    A.seed = seed;
    for (long long w = 0; w < windows_done(s, lg); ++w) A.wblk[(w / s->block_windows) % MD_NBLK] += 1;
    const size_t bytes = sizeof(double) * (size_t)s->nrep * s->nb;
    cudaPointerAttributes at{};
    const bool dev = cudaPointerGetAttributes(&at, sigma_out) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    double *dst = sigma_out;
    if (!dev) MD_CUDA_TRY(cudaMallocAsync((void **)&dst, bytes, s->st));
    A.sigma = dst;
    k_feq_bootstrap<<<s->nrep, 128, 0, s->st>>>(A);
    cudaError_t e = cudaGetLastError();
    if (!dev) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(sigma_out, dst, bytes, cudaMemcpyDeviceToHost, s->st);
        cudaFreeAsync(dst, s->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    }
    if (e != cudaSuccess) return fail(MD_E_CUDA, "feq_bootstrap: %s", cudaGetErrorString(e));
    return MD_OK;
}

int feq_batch(md_system *s, int32_t lg, int32_t dxi, int32_t symmetrize, double *out) {
    mdlg::Range range_("feq_batch");
    if (!s || !out || lg < 0 || lg >= s->n_lg || dxi < 0 || dxi >= s->n_dx)
        return fail(MD_E_ARG, "feq_batch: bad arguments");
    FeqBatchArgs A{};
    A.reps = s->d_reps;
    A.hist = s->sd.hist;
    A.ovf = s->sd.ovf;
    A.mom = s->sd.mom;
    A.n_lg = s->n_lg;
    A.n_dx = s->n_dx;
    A.lg = lg;
    A.dxi = dxi;
    A.nb = s->nb;
    A.W = s->W;
    A.sym = symmetrize != 0;
    A.nwin = windows_done(s, lg);
    const size_t bytes = sizeof(double) * (size_t)s->nrep * (3 * s->nb + FEQB_STATS);
    cudaPointerAttributes at{};
    const bool dev = cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    double *dst = out;
    if (!dev) MD_CUDA_TRY(cudaMallocAsync((void **)&dst, bytes, s->st));
    A.out = dst;
    k_feq_params<<<s->nrep, FEQB_THREADS, 0, s->st>>>(A, s->d_feq_par);
    k_feq_terms<<<dim3(s->nrep, FEQB_SPLIT), FEQB_THREADS, 0, s->st>>>(A, s->d_feq_par, s->d_feq_part);
    k_feq_batch<<<s->nrep, FEQB_THREADS, 0, s->st>>>(A, s->d_feq_part);
    cudaError_t e = cudaGetLastError();
    if (!dev) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, s->st);
        cudaFreeAsync(dst, s->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    }
    if (e != cudaSuccess) return fail(MD_E_CUDA, "feq_batch: %s", cudaGetErrorString(e));
    return MD_OK;
}

// ---- autotuner ------------------------------------------------------------
// Launch shapes tried: block {256, 128} x per_thread {1, 2, 4} x staging
// {shared, global}.  The best shape per (precision, replicas, particle
// count rounded to a power of two, list capacity) is kept for the process.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::tuple<int, int, int>> g_tune_cache;
std::map<std::tuple<int, int, int, int>, std::vector<double>> g_tune_costs;   // resident slab times
}

int md_autotune(md_system *s, int64_t steps_per_trial, int32_t *best3) {
    mdlg::Range range_("md_autotune");
    if (!s || steps_per_trial < 1) return fail(MD_E_ARG, "md_autotune: bad arguments");
    int lg2 = 0;
    while ((1ll << lg2) < s->ntot) ++lg2;
    const auto key = std::make_tuple(s->prec, s->nrep, lg2, s->K);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            auto ic = g_tune_costs.find(key);
            int rc = std::get<2>(it->second) == 4 && ic != g_tune_costs.end() && !ic->second.empty() &&
                             (int)ic->second.size() == s->nrep
                         ? configure_resident(s, &ic->second)
                         : configure_launch(s, std::get<0>(it->second), std::get<1>(it->second),
                                            std::get<2>(it->second));
            if (rc) return rc;
            if (best3) {
                best3[0] = std::get<0>(it->second);
                best3[1] = std::get<1>(it->second);
                best3[2] = std::get<2>(it->second);
            }
            return MD_OK;
        }
    }
    cudaEvent_t e0, e1;
    MD_CUDA_TRY(cudaEventCreate(&e0));
    MD_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int bb = 256, bp = 1, bs = 1;
    const int blocks[2] = {256, 128}, ppts[3] = {1, 2, 4}, stages[3] = {1, 2, 3};
    int rc = MD_OK;
    for (int b : blocks)
        for (int p : ppts)
            for (int st : stages) {
                if (st == 3 && s->prec == MD_FP64) continue;               // same kernel as 2
                if (configure_launch(s, b, p, st) != MD_OK) continue;   // shape does not fit
                rc = md_step(s, steps_per_trial);                          // settles caches
                if (rc) break;
                cudaEventRecord(e0, s->st);
                rc = md_step(s, steps_per_trial);
                if (rc) break;
                cudaEventRecord(e1, s->st);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    bb = b;
                    bp = p;
                    bs = st;
                }
            }
    // the shared-memory-resident engine (batched FP32 ensembles): a trial
    // with the modelled slab costs, then one with the schedule re-planned
    // from the slabs' measured times (the per-replica work split this
    // tunes; no result depends on the schedule)
    std::vector<double> res_cost;
    if (rc == MD_OK && s->prec == MD_FP32_CELLOFF && s->nrep >= 2 && configure_launch(s, 256, 1, 4) == MD_OK) {
        for (int trial = 0; trial < 2 && rc == MD_OK; ++trial) {
            rc = md_step(s, steps_per_trial);
            if (rc) break;
            cudaEventRecord(e0, s->st);
            rc = md_step(s, steps_per_trial);
            cudaEventRecord(e1, s->st);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rc == MD_OK && ms < best_ms) {
                best_ms = ms;
                bb = 256;
                bp = 1;
                bs = 4;
                res_cost.clear();
                if (trial == 1) res_cost = s->res_cost;
            }
            if (trial == 0 && rc == MD_OK) {
                // per replica: the longest of its slabs in the last launch
                std::vector<unsigned long long> ns(s->res_jobs.size());
                if (cudaMemcpy(ns.data(), s->rd.job_ns, sizeof(unsigned long long) * ns.size(),
                               cudaMemcpyDeviceToHost) != cudaSuccess)
                    break;
                std::vector<double> cost(s->nrep, 0.0);
                for (size_t j = 0; j < ns.size(); ++j)
                    cost[s->res_jobs[j].rep] = std::max(cost[s->res_jobs[j].rep], (double)ns[j]);
                if (configure_resident(s, &cost) != MD_OK) break;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = sync_status(s);
    if (rc) return rc;
    rc = bs == 4 && !res_cost.empty() ? configure_resident(s, &res_cost) : configure_launch(s, bb, bp, bs);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = std::make_tuple(bb, bp, bs);
        g_tune_costs[key] = res_cost;
    }
    if (best3) {
        best3[0] = bb;
        best3[1] = bp;
        best3[2] = bs;
    }
    return MD_OK;
}

}  // extern "C"

