// Device functions of the analytic equilibria (Sec. 3), shared by the
// single-distribution entry points and the batched f_eq stage.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace mdlg {

// One-dimensional equilibrium of a particle uniform in a unit lattice cell
// displaced by a Gaussian of variance var (lattice units), landing u cells
// away: Eq. (feq_gaussian) with a^2 = var, N = a / sqrt(2 pi).  The WSG
// component f^c of Eq. (f_eq_wsg) is this with var = a^2 (c+1)/(lambda+1)
// (N_c^2 = 2 var).
__device__ inline double cell_gauss_1d(double u, double var) {
    const double s = sqrt(2.0 * var);             // a sqrt(2) = N_c
    const double norm = sqrt(var) * 0.39894228040143267794;   // a / sqrt(2 pi)
    const double um = u - 1.0, up = u + 1.0;
    const double e = exp(-(um * um) / (2.0 * var)) - 2.0 * exp(-(u * u) / (2.0 * var)) +
                     exp(-(up * up) / (2.0 * var));
    const double eu = erf(u / s);
    return norm * e + 0.5 * um * (erf(um / s) - eu) + 0.5 * up * (erf(up / s) - eu);
}

// cell_gauss_1d(v, var) for the 2W+1 displacements v = -W..W into out[0..2W]
// (W <= 10).  Neighbouring v share two of their three points u-1, u, u+1, so
// the exponentials and error functions are evaluated once at each of the
// 2W+3 points -W-1..W+1 and combined with the arithmetic of cell_gauss_1d.
__device__ inline void cell_gauss_row(double var, int W, double *out) {
    const double s = sqrt(2.0 * var);
    const double norm = sqrt(var) * 0.39894228040143267794;
    double E[23], R[23];
    for (int k = 0; k < 2 * W + 3; ++k) {
        const double p = (double)(k - W - 1);
        E[k] = exp(-(p * p) / (2.0 * var));
        R[k] = erf(p / s);
    }
    for (int v = 0; v <= 2 * W; ++v) {
        const double u = (double)(v - W), um = u - 1.0, up = u + 1.0;
        const double e = E[v] - 2.0 * E[v + 1] + E[v + 2];
        const double eu = R[v + 1];
        out[v] = norm * e + 0.5 * um * (R[v] - eu) + 0.5 * up * (R[v + 2] - eu);
    }
}

// Root of Eq. (lambda_eq) in the printed form: root 1 takes the '+' sign of
// the square root, root 2 (the paper's choice) the '-' sign.
__device__ inline double lambda_root(double mu2, double mu4, int root) {
    const double m22 = mu2 * mu2;
    const double r = sqrt(3.0 * (15.0 * m22 * m22 - 4.0 * m22 * mu4));
    const double num = -9.0 * m22 + 2.0 * mu4 + (root == 1 ? r : -r);
    return num / (2.0 * (3.0 * m22 - mu4));
}

// Poisson terms kept: |c - lambda| <= 12 sqrt(lambda) + 20 (tails < 1e-16).
__host__ __device__ inline int wsg_cmax(double lam) {
    return lam <= 0.0 ? 0 : (int)ceil(lam + 12.0 * sqrt(lam) + 20.0);
}
__host__ __device__ inline int wsg_cmin(double lam) {
    const double c = floor(lam - 12.0 * sqrt(lam) - 20.0);
    return c > 0.0 ? (int)c : 0;
}

// Poisson weight Pois(c; lambda).
__device__ inline double poisson_weight(int c, double lam) {
    return lam > 0.0 ? exp(-lam + (double)c * log(lam) - lgamma((double)c + 1.0)) : (c == 0 ? 1.0 : 0.0);
}

}  // namespace mdlg
