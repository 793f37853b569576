/*
 * mdlg_oracle.c -- plain FP64 CPU oracle of the MDLG hot path
 * (Pachalieva & Wagner, "Molecular dynamics lattice gas equilibrium
 * distribution function for Lennard-Jones particles", arXiv 2101.01160).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  The product
 * path (libmdlg.so and its Python binding) never calls it, and it shares no
 * source, header, helper or constant with the CUDA path.
 *
 * Written for clarity, not speed: FP64 throughout, one plain loop per
 * definition, compiled with -ffp-contract=off so every product and sum is
 * rounded on its own (the CUDA path uses the same discipline where an integer
 * result depends on floating point: the lattice mapping).
 *
 * Contents and the passage each follows:
 *   or_bin_xy / or_bin_celloff   occupation numbers n_i of Eq. (n_i) (Sec. 2)
 *                                summed over all lattice sites x, i.e. the
 *                                unnormalised global histogram behind
 *                                f_i^eq of Eq. (theory_feq), plus the
 *                                displacement moments mu2, mu4 of Sec. 3(b)
 *   or_feq_g1 / or_feq_gaussian  Eq. (feq_gaussian) with Eq. (a2_n_ua), the
 *                                2D product of Eq. (feq_prod)
 *   or_feq_wsg                   the Poisson weighted sum of Eq. (f_eq_wsg)
 *                                with N_c of Sec. 3(b), sum over c outside
 *                                the 2D product
 *   or_wsg_lambda                the roots lambda_{1,2} of Eq. (lambda_eq)
 *   or_wsg_mu4                   Eq. (fourth_order)
 *   or_kl                        Eq. (kullback_leibler) / Eq. (k_Xi)
 *   or_site_occupation           the local occupation numbers n_i(x, t) of
 *                                Eq. (n_i) per lattice site (Sec. 2)
 *   or_collision                 the lattice-gas collision operator Xi_i of
 *                                Eq. (mdlg_evolution) (Sec. 2)
 *   or_disp_hist                 histogram of the continuous one-dimensional
 *                                displacement component over bins X_i (the
 *                                measured PDF of Sec. 3(b), Fig. 2)
 *   or_pdf_gauss_bins            bin masses of the Gaussian displacement PDF,
 *                                Eq. (gaussian_df), d = 1, u = 0
 *   or_pdf_wsg_bins              bin masses of the Poisson WSG displacement
 *                                PDF, Eqs. (poisson_v2) and (p_wsg_one)
 *   or_kl_terms                  element-wise K(X_i) of Eq. (k_Xi)
 *   or_symmetrize                the symmetric-set averaging of Sec. 5
 *   or_bootstrap_feq             block-bootstrap standard error of the
 *                                measured equilibrium (the run averages of
 *                                Sec. 2 are finite), draws by SplitMix64
 *   or_forces_brute              the Lennard-Jones force of Sec. 4, all
 *                                pairs, minimum image, cutoff rc, potential
 *                                shifted to zero at rc (force not shifted)
 *   or_forces_cells              the same force through a plain cell list
 *   or_md_run                    velocity-Verlet NVE dynamics (Sec. 4) with
 *                                MDLG sampling every S steps
 *   or_mlp_*                     the MLP surrogate (a project addition, not
 *                                in the paper): forward, softmax, KL loss and
 *                                backward in FP64
 *
 * Pins (tests/test_oracle_*.py, run with -m "not gpu"): brute-force counts on
 * hand-made snapshots and boundary ties, histogram mass conservation, the
 * closed forms against numerical quadrature of their defining integral,
 * normalisation and first moment, WSG(lambda=0) = G, WSG moments against
 * Eq. (fourth_order), lambda1*lambda2 = 1, the LJ force against a finite
 * difference of the potential and known potential values, Newton's third law,
 * the cell list against all pairs, NVE energy drift scaling as dt^2, exact
 * time reversal, the ballistic ideal gas against the Gaussian equilibrium,
 * the local occupation numbers against their indicator sum and the global
 * histogram, and mass conservation and free streaming of the collision
 * operator.  Parity of the measured f_eq of the interacting gas has no
 * printed values to pin to (the paper ships no data): only statistical
 * agreement and the qualitative claims of Sec. 5 are checked.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Lattice mapping (Sec. 2): cell indicator Delta_x[x_j(t)] = 1 iff particle j
 * lies in lattice cell x.  Reading: l = floor(x / dx) reduced mod lx, a point
 * exactly on a cell boundary belongs to the upper cell. */
static int64_t lattice_index(double x, double dxl, int64_t lx)
{
    double t = x / dxl;
    int64_t l = (int64_t)floor(t);
    l %= lx;
    if (l < 0) l += lx;
    return l;
}

/* Lattice displacement l1 - l0 reduced to the nearest periodic image. */
static int64_t nearest_image_int(int64_t d, int64_t lx)
{
    d %= lx;
    if (d < 0) d += lx;
    if (d > lx / 2) d -= lx;
    return d;
}

static double nearest_image(double d, double L)
{
    return d - L * nearbyint(d / L);
}

/* Global displacement histogram from two snapshots of absolute positions.
 * hist has (2W+1)^2 entries, index (dy+W)*(2W+1) + (dx+W); a particle whose
 * lattice displacement leaves the window counts in *overflow, so that
 * sum(hist) + overflow = n.  mom[0] += sum over particles and both axes of
 * delta^2, mom[1] += delta^4, delta the continuous nearest-image
 * displacement.  Accumulates into hist, overflow, mom. */
void or_bin_xy(int64_t n, const double *x0, const double *y0, const double *x1,
               const double *y1, double L, int64_t lx, int32_t W, int64_t *hist,
               int64_t *overflow, double *mom)
{
    double dxl = L / (double)lx;
    int64_t side = 2 * (int64_t)W + 1;
    for (int64_t j = 0; j < n; ++j) {
        int64_t lx0 = lattice_index(x0[j], dxl, lx);
        int64_t ly0 = lattice_index(y0[j], dxl, lx);
        int64_t lx1 = lattice_index(x1[j], dxl, lx);
        int64_t ly1 = lattice_index(y1[j], dxl, lx);
        int64_t ddx = nearest_image_int(lx1 - lx0, lx);
        int64_t ddy = nearest_image_int(ly1 - ly0, lx);
        if (ddx >= -W && ddx <= W && ddy >= -W && ddy <= W)
            hist[(ddy + W) * side + (ddx + W)] += 1;
        else
            *overflow += 1;
        double ex = nearest_image(x1[j] - x0[j], L);
        double ey = nearest_image(y1[j] - y0[j], L);
        mom[0] += ex * ex + ey * ey;
        mom[1] += ex * ex * ex * ex + ey * ey * ey * ey;
    }
}

/* Same, for snapshots stored as (linear MD-cell index cy*ncell+cx, in-cell
 * offset).  The encoded position is x = cx*h + off, evaluated in FP64 with
 * separate roundings; the periodic box edge is L = ncell*h as given. */
static void decode(int64_t n, const int32_t *cell, const void *ox, const void *oy, int f64,
                   int32_t ncell, double h, double *x, double *y)
{
    for (int64_t j = 0; j < n; ++j) {
        int32_t cx = cell[j] % ncell;
        int32_t cy = cell[j] / ncell;
        double ofx = f64 ? ((const double *)ox)[j] : (double)((const float *)ox)[j];
        double ofy = f64 ? ((const double *)oy)[j] : (double)((const float *)oy)[j];
        double px = (double)cx * h;
        double py = (double)cy * h;
        x[j] = px + ofx;
        y[j] = py + ofy;
    }
}

int or_bin_celloff(int64_t n, const int32_t *c0, const void *ox0, const void *oy0,
                   const int32_t *c1, const void *ox1, const void *oy1, int32_t f64,
                   int32_t ncell, double h, double L, int64_t lx, int32_t W,
                   int64_t *hist, int64_t *overflow, double *mom)
{
    double *b = (double *)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
    if (!b) return -1;
    decode(n, c0, ox0, oy0, f64, ncell, h, b, b + n);
    decode(n, c1, ox1, oy1, f64, ncell, h, b + 2 * n, b + 3 * n);
    or_bin_xy(n, b, b + n, b + 2 * n, b + 3 * n, L, lx, W, hist, overflow, mom);
    free(b);
    return 0;
}

/* Local occupation numbers of Eq. (n_i), Sec. 2: n_i(x, t1) counts the
 * particles that are in lattice cell x at t1 and were in cell x - v_i at t0
 * (v_i taken as the nearest periodic image of the lattice displacement).
 * nfield has (2W+1)^2 * lx^2 entries, class-major: class i = (vy+W)(2W+1) +
 * (vx+W), site x = ly*lx + lx_; a particle whose displacement leaves the
 * window counts in ovf[x] of its arrival site, so that summed over x and i
 * this is or_bin_celloff's histogram.  Accumulates. */
int or_site_occupation(int64_t n, const int32_t *c0, const void *ox0, const void *oy0,
                       const int32_t *c1, const void *ox1, const void *oy1, int32_t f64,
                       int32_t ncell, double h, double L, int64_t lx, int32_t W,
                       int64_t *nfield, int64_t *ovf)
{
    double *b = (double *)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
    if (!b) return -1;
    decode(n, c0, ox0, oy0, f64, ncell, h, b, b + n);
    decode(n, c1, ox1, oy1, f64, ncell, h, b + 2 * n, b + 3 * n);
    double dxl = L / (double)lx;
    int64_t side = 2 * (int64_t)W + 1;
    int64_t nsite = lx * lx;
    for (int64_t j = 0; j < n; ++j) {
        int64_t sx0 = lattice_index(b[j], dxl, lx);
        int64_t sy0 = lattice_index(b[n + j], dxl, lx);
        int64_t sx1 = lattice_index(b[2 * n + j], dxl, lx);
        int64_t sy1 = lattice_index(b[3 * n + j], dxl, lx);
        int64_t vx = nearest_image_int(sx1 - sx0, lx);
        int64_t vy = nearest_image_int(sy1 - sy0, lx);
        int64_t site = sy1 * lx + sx1;
        if (vx >= -W && vx <= W && vy >= -W && vy <= W)
            nfield[((vy + W) * side + (vx + W)) * nsite + site] += 1;
        else
            ovf[site] += 1;
    }
    free(b);
    return 0;
}

/* Lattice-gas collision operator of Eq. (mdlg_evolution), Sec. 2:
 * Xi_i(x, t) = n_i(x + v_i, t + dt) - n_i(x, t), x + v_i periodic, for the
 * occupation fields nt = n(., t) and nn = n(., t + dt) in the layout of
 * or_site_occupation. */
void or_collision(const int64_t *nt, const int64_t *nn, int64_t lx, int32_t W, int64_t *xi)
{
    int64_t side = 2 * (int64_t)W + 1;
    int64_t nsite = lx * lx;
    for (int64_t vy = -W; vy <= W; ++vy)
        for (int64_t vx = -W; vx <= W; ++vx) {
            int64_t i = (vy + W) * side + (vx + W);
            for (int64_t y = 0; y < lx; ++y)
                for (int64_t x = 0; x < lx; ++x) {
                    int64_t xd = ((x + vx) % lx + lx) % lx;
                    int64_t yd = ((y + vy) % lx + lx) % lx;
                    xi[i * nsite + y * lx + x] = nn[i * nsite + yd * lx + xd] - nt[i * nsite + y * lx + x];
                }
        }
}

/* Histogram of the continuous one-dimensional displacement component over
 * bins X_i.  For every particle and both axes the displacement is taken in
 * the cell frame: the cell-index difference wrapped to the nearest periodic
 * image (into [-ncell/2, ncell/2]) times h, plus the offset difference,
 *     delta = wrap(c1 - c0) * h + (off1 - off0),
 * which has a single rounding (none in the product and the offset
 * difference when the offsets are FP32), instead of decoding two absolute
 * positions near the box size.  Its bin is floor(delta / width) + nbins / 2:
 * bin k covers [(k - nbins/2) width, (k - nbins/2 + 1) width), the bins
 * X_i whose model masses or_pdf_gauss_bins and or_pdf_wsg_bins integrate,
 * and a value on an edge belongs to the upper bin.  Values outside all bins
 * count in *outside, so sum(hist) + *outside = 2n.  Accumulates. */
int or_disp_hist(int64_t n, const int32_t *c0, const void *ox0, const void *oy0,
                 const int32_t *c1, const void *ox1, const void *oy1, int32_t f64,
                 int32_t ncell, double h, double L, double width, int32_t nbins,
                 int64_t *hist, int64_t *outside)
{
    (void)L;
    for (int64_t j = 0; j < n; ++j) {
        int32_t cell0[2] = {c0[j] % ncell, c0[j] / ncell};
        int32_t cell1[2] = {c1[j] % ncell, c1[j] / ncell};
        const void *o0[2] = {ox0, oy0}, *o1[2] = {ox1, oy1};
        for (int axis = 0; axis < 2; ++axis) {
            int32_t dc = cell1[axis] - cell0[axis];
            if (dc > ncell / 2) dc -= ncell;
            if (dc < -(ncell / 2)) dc += ncell;
            double a = f64 ? ((const double *)o0[axis])[j] : (double)((const float *)o0[axis])[j];
            double b = f64 ? ((const double *)o1[axis])[j] : (double)((const float *)o1[axis])[j];
            double d = (double)dc * h + (b - a);
            double k = floor(d / width) + (double)(nbins / 2);
            if (k >= 0.0 && k < (double)nbins)
                hist[(int64_t)k] += 1;
            else
                *outside += 1;
        }
    }
    return 0;
}

int32_t or_wsg_cmax(double lambda);
double or_poisson(int32_t c, double lambda);

/* Mass of a centred normal distribution of variance var in [a, b). */
static double normal_mass(double a, double b, double var)
{
    double s = sqrt(2.0 * var);
    return 0.5 * (erf(b / s) - erf(a / s));
}

/* Eq. (gaussian_df) with d = 1, u = 0 and <dx^2> = mu2, integrated over the
 * bins of or_disp_hist. */
void or_pdf_gauss_bins(double mu2, double width, int32_t nbins, double *P)
{
    for (int32_t k = 0; k < nbins; ++k) {
        double a = (double)(k - nbins / 2) * width;
        P[k] = normal_mass(a, a + width, mu2);
    }
}

/* Eq. (poisson_v2) with the one-dimensional Gaussians of Eq. (p_wsg_one)
 * (d = 1, u = 0): Poisson weights of the number c of collisions times a
 * Gaussian of variance (c + 1) mu2 / (lambda + 1), integrated over the bins
 * of or_disp_hist; c = 0 .. or_wsg_cmax(lambda). */
void or_pdf_wsg_bins(double mu2, double lambda, double width, int32_t nbins, double *P)
{
    int32_t cmax = or_wsg_cmax(lambda);
    for (int32_t k = 0; k < nbins; ++k) {
        double a = (double)(k - nbins / 2) * width;
        double s = 0.0;
        for (int32_t c = 0; c <= cmax; ++c)
            s += or_poisson(c, lambda) * normal_mass(a, a + width, (double)(c + 1) * mu2 / (lambda + 1.0));
        P[k] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. (feq_gaussian): one-dimensional Gaussian equilibrium for the shifted
 * lattice velocity u = v_i - u_alpha (lattice units) and a^2 = <dx^2>/dx^2,
 * with N = a / sqrt(2 pi) of Eq. (a2_n_ua). */
double or_feq_g1(double u, double a2)
{
    double a = sqrt(a2);
    double Nn = a / sqrt(2.0 * M_PI);
    double s = a * sqrt(2.0);
    double e_m = exp(-((u - 1.0) * (u - 1.0)) / (2.0 * a2));
    double e_0 = exp(-(u * u) / (2.0 * a2));
    double e_p = exp(-((u + 1.0) * (u + 1.0)) / (2.0 * a2));
    double t1 = Nn * (e_m - 2.0 * e_0 + e_p);
    double t2 = (u - 1.0) / 2.0 * (erf((u - 1.0) / s) - erf(u / s));
    double t3 = (u + 1.0) / 2.0 * (erf((u + 1.0) / s) - erf(u / s));
    return t1 + t2 + t3;
}

/* Eq. (feq_prod): f_i / rho = f_{i,x} f_{i,y}, for the (2W+1)^2 lattice
 * velocities v_i = (vx, vy), |vx|,|vy| <= W, index (vy+W)(2W+1) + (vx+W). */
void or_feq_gaussian(double a2, double ux, double uy, int32_t W, double *P)
{
    int32_t side = 2 * W + 1;
    for (int32_t iy = 0; iy < side; ++iy)
        for (int32_t ix = 0; ix < side; ++ix) {
            double gx = or_feq_g1((double)(ix - W) - ux, a2);
            double gy = or_feq_g1((double)(iy - W) - uy, a2);
            P[iy * side + ix] = gx * gy;
        }
}

/* Number of Poisson terms kept: c = 0..cmax with cmax = ceil(lambda +
 * 12 sqrt(lambda) + 20); the omitted tail mass is below 1e-16 for every
 * lambda in use (checked in the tests against the exact Poisson CDF). */
int32_t or_wsg_cmax(double lambda)
{
    if (lambda <= 0.0) return 0;
    return (int32_t)ceil(lambda + 12.0 * sqrt(lambda) + 20.0);
}

double or_poisson(int32_t c, double lambda)
{
    if (lambda <= 0.0) return c == 0 ? 1.0 : 0.0;
    return exp(-lambda + (double)c * log(lambda) - lgamma((double)c + 1.0));
}

/* Poisson WSG equilibrium (Sec. 3(b)): f_i / rho = sum_c Pois(c; lambda)
 * f^c_{i,x} f^c_{i,y}, where f^c is Eq. (f_eq_wsg) with
 * N_c = sqrt(2 a^2 (c+1)/(lambda+1)); written out, f^c is the expression of
 * Eq. (f_eq_wsg) itself. */
static double feq_c1(double u, double Nc)
{
    double e_m = exp(-((u - 1.0) * (u - 1.0)) / (Nc * Nc));
    double e_0 = exp(-(u * u) / (Nc * Nc));
    double e_p = exp(-((u + 1.0) * (u + 1.0)) / (Nc * Nc));
    double t1 = Nc / (2.0 * sqrt(M_PI)) * (e_m - 2.0 * e_0 + e_p);
    double t2 = (u - 1.0) / 2.0 * (erf((u - 1.0) / Nc) - erf(u / Nc));
    double t3 = (u + 1.0) / 2.0 * (erf((u + 1.0) / Nc) - erf(u / Nc));
    return t1 + t2 + t3;
}

double or_feq_wsg1(double u, double a2, double lambda, int32_t c)
{
    double Nc = sqrt(2.0 * a2 * ((double)c + 1.0) / (lambda + 1.0));
    return feq_c1(u, Nc);
}

void or_feq_wsg(double a2, double lambda, double ux, double uy, int32_t W, double *P)
{
    int32_t side = 2 * W + 1;
    int32_t cmax = or_wsg_cmax(lambda);
    for (int32_t k = 0; k < side * side; ++k) P[k] = 0.0;
    for (int32_t c = 0; c <= cmax; ++c) {
        double w = or_poisson(c, lambda);
        for (int32_t iy = 0; iy < side; ++iy)
            for (int32_t ix = 0; ix < side; ++ix) {
                double fx = or_feq_wsg1((double)(ix - W) - ux, a2, lambda, c);
                double fy = or_feq_wsg1((double)(iy - W) - uy, a2, lambda, c);
                P[iy * side + ix] += w * (fx * fy);
            }
    }
}

/* Eq. (fourth_order). */
double or_wsg_mu4(double mu2, double lambda)
{
    return 3.0 * mu2 * mu2 / ((lambda + 1.0) * (lambda + 1.0)) *
           (lambda * lambda + 3.0 * lambda + 1.0);
}

/* Roots of Eq. (lambda_eq), in the paper's printed form: lambda_1 takes the
 * '+' sign of the square root, lambda_2 the '-' sign.  Returns 0 on success,
 * -1 if 3 mu2^2 = mu4 (no quadratic), -2 if the discriminant is negative
 * (kurtosis mu4/mu2^2 > 3.75, no real root). */
int or_wsg_lambda(double mu2, double mu4, double *l1, double *l2)
{
    double m22 = mu2 * mu2;
    double den = 2.0 * (3.0 * m22 - mu4);
    double disc = 3.0 * (15.0 * m22 * m22 - 4.0 * m22 * mu4);
    if (den == 0.0) return -1;
    if (disc < 0.0) return -2;
    double r = sqrt(disc);
    *l1 = (-9.0 * m22 + r + 2.0 * mu4) / den;
    *l2 = (-9.0 * m22 - r + 2.0 * mu4) / den;
    return 0;
}

/* Eq. (k_Xi): K(X_i) = R_i log(R_i / Q_i) per bin, 0 where R_i = 0. */
void or_kl_terms(const double *R, const double *Q, int64_t n, double *K)
{
    for (int64_t i = 0; i < n; ++i) K[i] = R[i] > 0.0 ? R[i] * log(R[i] / Q[i]) : 0.0;
}

/* Eq. (kullback_leibler), with the convention 0 log 0 = 0. */
double or_kl(const double *R, const double *Q, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (R[i] > 0.0) s += R[i] * log(R[i] / Q[i]);
    return s;
}

/* Symmetric-set averaging (Sec. 5): each value is replaced by the mean over
 * the lattice velocities of the same set, a set being the velocities that
 * the symmetries of the square map onto each other, i.e. equal
 * (min(|vx|,|vy|), max(|vx|,|vy|)). */
void or_symmetrize(const double *P, int32_t W, double *out)
{
    int32_t side = 2 * W + 1;
    for (int32_t iy = 0; iy < side; ++iy)
        for (int32_t ix = 0; ix < side; ++ix) {
            int32_t a = abs(ix - W), b = abs(iy - W);
            int32_t lo = a < b ? a : b, hi = a < b ? b : a;
            double s = 0.0;
            int32_t m = 0;
            for (int32_t jy = 0; jy < side; ++jy)
                for (int32_t jx = 0; jx < side; ++jx) {
                    int32_t c = abs(jx - W), d = abs(jy - W);
                    int32_t lo2 = c < d ? c : d, hi2 = c < d ? d : c;
                    if (lo2 == lo && hi2 == hi) {
                        s += P[jy * side + jx];
                        ++m;
                    }
                }
            out[iy * side + ix] = s / (double)m;
        }
}

/* ------------------------------------------------------------------------ */
/* Statistical error of the measured equilibrium by the block bootstrap (the
 * averages over iterations of Sec. 2 are estimated from a finite run): the
 * error-bar blocks of windows that hold data are resampled with replacement,
 * nblk_used draws per resample, and each resample's P_i = sum of the drawn
 * blocks' counts / (n * drawn windows) (optionally averaged over the
 * symmetric set of i, as or_symmetrize does); sigma_i is the sample
 * standard deviation of P_i over the B resamples (divisor B - 1).
 *
 * Draws come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: draw number c of a stream gives the output function applied
 * to seed + (c + 1) * 0x9e3779b97f4a7c15; block index = the draw's top 32
 * bits times nblk_used, shifted right by 32.  The draw of resample b, slot k
 * of replica rep has c = ((rep * 2^20 + b) * 64 + k). */
uint64_t or_splitmix64(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1u) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

int or_bootstrap_feq(const int64_t *hist, const int64_t *wblk, int32_t nblk, int32_t W, double n,
                     int32_t sym, int32_t B, uint64_t seed, int32_t rep, double *sigma)
{
    int32_t side = 2 * W + 1, nb = side * side;
    int32_t used[64];
    int32_t nu = 0;
    if (nblk > 64 || B < 2) return -1;
    for (int32_t k = 0; k < nblk; ++k)
        if (wblk[k] > 0) used[nu++] = k;
    double *P = (double *)malloc(sizeof(double) * (size_t)B * (size_t)nb);
    int64_t *Hs = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
    if (!P || !Hs) {
        free(P);
        free(Hs);
        return -2;
    }
    for (int32_t i = 0; i < nb; ++i) sigma[i] = 0.0;
    if (nu == 0) {
        free(P);
        free(Hs);
        return 0;
    }
    for (int32_t b = 0; b < B; ++b) {
        int64_t wsum = 0;
        for (int32_t i = 0; i < nb; ++i) Hs[i] = 0;
        for (int32_t k = 0; k < nu; ++k) {
            uint64_t c = (((uint64_t)rep << 20) + (uint64_t)b) * 64u + (uint64_t)k;
            uint64_t r = or_splitmix64(seed, c);
            int32_t u = used[(int32_t)(((r >> 32) * (uint64_t)nu) >> 32)];
            wsum += wblk[u];
            for (int32_t i = 0; i < nb; ++i) Hs[i] += hist[(int64_t)u * nb + i];
        }
        for (int32_t iy = 0; iy < side; ++iy)
            for (int32_t ix = 0; ix < side; ++ix) {
                int64_t h = 0;
                int32_t m = 0;
                if (sym) {
                    int32_t a = abs(ix - W), bb = abs(iy - W);
                    int32_t lo = a < bb ? a : bb, hi = a < bb ? bb : a;
                    for (int32_t jy = 0; jy < side; ++jy)
                        for (int32_t jx = 0; jx < side; ++jx) {
                            int32_t c2 = abs(jx - W), d2 = abs(jy - W);
                            int32_t lo2 = c2 < d2 ? c2 : d2, hi2 = c2 < d2 ? d2 : c2;
                            if (lo2 == lo && hi2 == hi) {
                                h += Hs[jy * side + jx];
                                ++m;
                            }
                        }
                } else {
                    h = Hs[iy * side + ix];
                    m = 1;
                }
                P[(int64_t)b * nb + iy * side + ix] = (double)h / ((double)m * n * (double)wsum);
            }
    }
    for (int32_t i = 0; i < nb; ++i) {
        double mean = 0.0, ss = 0.0;
        for (int32_t b = 0; b < B; ++b) mean += P[(int64_t)b * nb + i];
        mean /= (double)B;
        for (int32_t b = 0; b < B; ++b) {
            double d = P[(int64_t)b * nb + i] - mean;
            ss += d * d;
        }
        sigma[i] = sqrt(ss / (double)(B - 1));
    }
    free(P);
    free(Hs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lennard-Jones pair (Sec. 4): V(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6],
 * truncated at rc and shifted by V(rc); the force -dV/dr is not shifted.
 * Returns the shifted pair energy; *fr = (-dV/dr) / r, so the force on the
 * particle at x_i from the one at x_j is fr * (x_i - x_j). */
double or_lj_pair(double r2, double rc, double eps, double sigma, double *fr)
{
    double sr2 = sigma * sigma / r2;
    double sr6 = sr2 * sr2 * sr2;
    double sc2 = sigma * sigma / (rc * rc);
    double sc6 = sc2 * sc2 * sc2;
    *fr = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
    double v = 4.0 * eps * (sr6 * sr6 - sr6);
    double vc = 4.0 * eps * (sc6 * sc6 - sc6);
    return v - vc;
}

/* All pairs, nearest periodic image.  fx, fy receive the total force; if
 * pe is non-NULL, pe[i] = half the sum of pair energies of i (so sum(pe) is
 * the system energy); if fabs_sum is non-NULL it receives sum_j |F_ij|. */
void or_forces_brute(int64_t n, const double *x, const double *y, double L, double rc,
                     double eps, double sigma, double *fx, double *fy, double *pe,
                     double *fabs_sum)
{
    double rc2 = rc * rc;
    for (int64_t i = 0; i < n; ++i) {
        double sx = 0.0, sy = 0.0, se = 0.0, sa = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = nearest_image(x[i] - x[j], L);
            double dy = nearest_image(y[i] - y[j], L);
            double r2 = dx * dx + dy * dy;
            if (r2 >= rc2) continue;
            double fr;
            double v = or_lj_pair(r2, rc, eps, sigma, &fr);
            sx += fr * dx;
            sy += fr * dy;
            se += 0.5 * v;
            sa += fabs(fr) * sqrt(r2);
        }
        fx[i] = sx;
        fy[i] = sy;
        if (pe) pe[i] = se;
        if (fabs_sum) fabs_sum[i] = sa;
    }
}

/* The same force through a cell list: cells of edge L/floor(L/rc) >= rc,
 * a particle interacts only with particles of the 3x3 block of cells around
 * its own.  With fewer than 3 cells per edge it falls back to all pairs.
 * If sub/nsub are given, forces are computed only for those particle indices
 * (outputs still indexed by particle), the others are left untouched. */
int or_forces_cells(int64_t n, const double *x, const double *y, double L, double rc,
                    double eps, double sigma, double *fx, double *fy, double *pe,
                    double *fabs_sum, int64_t nsub, const int64_t *sub)
{
    int64_t nc = (int64_t)floor(L / rc);
    if (nc < 3) {
        if (sub) return -1;
        or_forces_brute(n, x, y, L, rc, eps, sigma, fx, fy, pe, fabs_sum);
        return 0;
    }
    double cw = L / (double)nc;
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc * nc));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!head || !next || !cid) {
        free(head); free(next); free(cid);
        return -2;
    }
    for (int64_t c = 0; c < nc * nc; ++c) head[c] = -1;
    for (int64_t j = n - 1; j >= 0; --j) {
        double px = x[j] - L * floor(x[j] / L);
        double py = y[j] - L * floor(y[j] / L);
        int64_t cx = (int64_t)floor(px / cw), cy = (int64_t)floor(py / cw);
        if (cx >= nc) cx = nc - 1;
        if (cy >= nc) cy = nc - 1;
        if (cx < 0) cx = 0;
        if (cy < 0) cy = 0;
        cid[j] = cy * nc + cx;
        next[j] = head[cid[j]];
        head[cid[j]] = j;
    }
    double rc2 = rc * rc;
    int64_t m = sub ? nsub : n;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = sub ? sub[k] : k;
        int64_t cx = cid[i] % nc, cy = cid[i] / nc;
        double sx = 0.0, sy = 0.0, se = 0.0, sa = 0.0;
        for (int64_t oy = -1; oy <= 1; ++oy)
            for (int64_t ox = -1; ox <= 1; ++ox) {
                int64_t qx = (cx + ox + nc) % nc, qy = (cy + oy + nc) % nc;
                for (int64_t j = head[qy * nc + qx]; j >= 0; j = next[j]) {
                    if (j == i) continue;
                    double dx = nearest_image(x[i] - x[j], L);
                    double dy = nearest_image(y[i] - y[j], L);
                    double r2 = dx * dx + dy * dy;
                    if (r2 >= rc2) continue;
                    double fr;
                    double v = or_lj_pair(r2, rc, eps, sigma, &fr);
                    sx += fr * dx;
                    sy += fr * dy;
                    se += 0.5 * v;
                    sa += fabs(fr) * sqrt(r2);
                }
            }
        fx[i] = sx;
        fy[i] = sy;
        if (pe) pe[i] = se;
        if (fabs_sum) fabs_sum[i] = sa;
    }
    free(head); free(next); free(cid);
    return 0;
}

/* Kinetic energy, shifted potential energy and total momentum. */
int or_energy(int64_t n, const double *x, const double *y, const double *vx, const double *vy,
              double L, double rc, double eps, double sigma, double mass, double *out4)
{
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!f) return -1;
    int rcode = or_forces_cells(n, x, y, L, rc, eps, sigma, f, f + n, f + 2 * n, NULL, 0, NULL);
    double ke = 0.0, pe = 0.0, px = 0.0, py = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        ke += 0.5 * mass * (vx[i] * vx[i] + vy[i] * vy[i]);
        pe += f[2 * n + i];
        px += mass * vx[i];
        py += mass * vy[i];
    }
    out4[0] = ke; out4[1] = pe; out4[2] = px; out4[3] = py;
    free(f);
    return rcode;
}

/* ------------------------------------------------------------------------ */
/* NVE velocity-Verlet dynamics (Sec. 4) with MDLG sampling.
 *
 * Each step: v += (dt/2m) F; x += dt v (wrapped into [0, L)); F = F(x);
 * v += (dt/2m) F.  Step counter s counts completed steps.  Sampling slot k has
 * period every[k] steps: at s == n_equil its snapshot is taken, and at every
 * s = n_equil + m*every[k] (m >= 1) the positions are binned against the
 * snapshot on each lattice lx[d] (Eq. (n_i) summed over x) and the snapshot
 * is replaced.  hist is [n_lg][n_dx][(2W+1)^2], overflow [n_lg][n_dx],
 * mom [n_lg][2], nwin [n_lg]; all accumulate.  If elog is non-NULL it
 * receives (KE, PE, Px, Py) at s = 0..nsteps ([nsteps+1][4]).
 * x, y, vx, vy are updated in place to the state after nsteps steps. */
int or_md_run(int64_t n, double *x, double *y, double *vx, double *vy, double L, double rc,
              double eps, double sigma, double mass, double dt, int64_t nsteps, int64_t n_equil,
              int32_t n_lg, const int32_t *every, int32_t n_dx, const int64_t *lx, int32_t W,
              int64_t *hist, int64_t *overflow, double *mom, int64_t *nwin, double *elog)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *fx = (double *)malloc(sizeof(double) * nn);
    double *fy = (double *)malloc(sizeof(double) * nn);
    double *pe = (double *)malloc(sizeof(double) * nn);
    double *snap = (double *)malloc(sizeof(double) * 2 * nn * (size_t)(n_lg > 0 ? n_lg : 1));
    if (!fx || !fy || !pe || !snap) {
        free(fx); free(fy); free(pe); free(snap);
        return -2;
    }
    int32_t nb = (2 * W + 1) * (2 * W + 1);
    double hk = dt / (2.0 * mass);
    int rcode = or_forces_cells(n, x, y, L, rc, eps, sigma, fx, fy, pe, NULL, 0, NULL);
    if (rcode) goto done;
    for (int64_t s = 0;; ++s) {
        if (elog) {
            double ke = 0.0, pt = 0.0, px = 0.0, py = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                ke += 0.5 * mass * (vx[i] * vx[i] + vy[i] * vy[i]);
                pt += pe[i];
                px += mass * vx[i];
                py += mass * vy[i];
            }
            elog[4 * s + 0] = ke; elog[4 * s + 1] = pt;
            elog[4 * s + 2] = px; elog[4 * s + 3] = py;
        }
        for (int32_t k = 0; k < n_lg; ++k) {
            if (s < n_equil || (s - n_equil) % every[k] != 0) continue;
            double *sx = snap + 2 * nn * (size_t)k, *sy = sx + nn;
            if (s > n_equil) {
                /* the displacement moments belong to the interval, not to a
                 * lattice: they are accumulated once per window */
                for (int32_t d = 0; d < n_dx; ++d) {
                    double dummy[2] = {0.0, 0.0};
                    or_bin_xy(n, sx, sy, x, y, L, lx[d], W,
                              hist + ((int64_t)k * n_dx + d) * nb,
                              overflow + (int64_t)k * n_dx + d, d == 0 ? mom + 2 * k : dummy);
                }
                nwin[k] += 1;
            }
            memcpy(sx, x, sizeof(double) * (size_t)n);
            memcpy(sy, y, sizeof(double) * (size_t)n);
        }
        if (s == nsteps) break;
        for (int64_t i = 0; i < n; ++i) {
            vx[i] = vx[i] + hk * fx[i];
            vy[i] = vy[i] + hk * fy[i];
            x[i] = x[i] + dt * vx[i];
            y[i] = y[i] + dt * vy[i];
            x[i] = x[i] - L * floor(x[i] / L);
            y[i] = y[i] - L * floor(y[i] / L);
            if (x[i] >= L) x[i] -= L;
            if (y[i] >= L) y[i] -= L;
        }
        rcode = or_forces_cells(n, x, y, L, rc, eps, sigma, fx, fy, pe, NULL, 0, NULL);
        if (rcode) goto done;
        for (int64_t i = 0; i < n; ++i) {
            vx[i] = vx[i] + hk * fx[i];
            vy[i] = vy[i] + hk * fy[i];
        }
    }
done:
    free(fx); free(fy); free(pe); free(snap);
    return rcode;
}
