/*
 * mlp_oracle.c -- plain FP64 CPU oracle of the f_eq surrogate (a project
 * addition, not in the paper): a multilayer perceptron mapping the state
 * point (phi, T, Delta t_LG, Delta x) to the equilibrium probabilities of the
 * (2W+1)^2 displacement classes.
 *
 * TEST INFRASTRUCTURE, like mdlg_oracle.c: loaded only by tests/ (and
 * bench.py's baseline legs); shares nothing with the CUDA path.
 *
 * Model (fixed for both sides):
 *   features  x_f = (x - shift) / scale                 (4 inputs)
 *   hidden    h_l = silu(W_l h_{l-1} + b_l), silu(z) = z / (1 + exp(-z))
 *   output    p = softmax(W_L h_{L-1} + b_L)
 *   loss      mean over the batch of the Kullback-Leibler divergence
 *             D_KL(t || p) = sum_i t_i log(t_i / p_i)   (Eq. kullback_leibler)
 * Weights are row-major [out][in].  sizes[0..nl] are the layer widths
 * (sizes[0] = 4 inputs, sizes[nl] = classes).
 *
 * Pin (tests/test_oracle_mlp.py): the gradient equals a central finite
 * difference of the loss for every parameter tensor, and the forward pass
 * is a probability distribution.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double silu_grad(double z)
{
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

/* Forward pass for row m; z and h receive pre- and post-activations of
 * every layer (offsets off[l]).  Returns the probability vector in p. */
static void forward_row(int32_t nl, const int32_t *sizes, const double *x, const double *shift,
                        const double *scale, const double *const *W, const double *const *b,
                        double *z, double *h, const int64_t *off, double *p)
{
    for (int32_t i = 0; i < sizes[0]; ++i) h[off[0] + i] = (x[i] - shift[i]) / scale[i];
    for (int32_t l = 1; l <= nl; ++l) {
        int32_t in = sizes[l - 1], out = sizes[l];
        for (int32_t o = 0; o < out; ++o) {
            double a = b[l - 1][o];
            for (int32_t i = 0; i < in; ++i) a += W[l - 1][(int64_t)o * in + i] * h[off[l - 1] + i];
            z[off[l] + o] = a;
            h[off[l] + o] = l < nl ? silu(a) : a;
        }
    }
    int32_t nc = sizes[nl];
    double mx = -INFINITY;
    for (int32_t c = 0; c < nc; ++c) mx = fmax(mx, h[off[nl] + c]);
    double s = 0.0;
    for (int32_t c = 0; c < nc; ++c) {
        p[c] = exp(h[off[nl] + c] - mx);
        s += p[c];
    }
    for (int32_t c = 0; c < nc; ++c) p[c] /= s;
}

static int64_t offsets(int32_t nl, const int32_t *sizes, int64_t *off)
{
    int64_t t = 0;
    for (int32_t l = 0; l <= nl; ++l) {
        off[l] = t;
        t += sizes[l];
    }
    return t;
}

/* params: W_1, b_1, W_2, b_2, ... packed back to back. */
static void unpack(int32_t nl, const int32_t *sizes, const double *params, const double **W,
                   const double **b)
{
    const double *q = params;
    for (int32_t l = 1; l <= nl; ++l) {
        W[l - 1] = q;
        q += (int64_t)sizes[l] * sizes[l - 1];
        b[l - 1] = q;
        q += sizes[l];
    }
}

int or_mlp_forward(int32_t nl, const int32_t *sizes, int64_t M, const double *X,
                   const double *shift, const double *scale, const double *params, double *P)
{
    if (nl < 1 || nl > 16) return -1;
    const double *W[16], *b[16];
    int64_t off[17];
    unpack(nl, sizes, params, W, b);
    int64_t tot = offsets(nl, sizes, off);
    double *z = (double *)malloc(sizeof(double) * (size_t)tot);
    double *h = (double *)malloc(sizeof(double) * (size_t)tot);
    if (!z || !h) {
        free(z);
        free(h);
        return -2;
    }
    for (int64_t m = 0; m < M; ++m)
        forward_row(nl, sizes, X + m * sizes[0], shift, scale, W, b, z, h, off,
                    P + m * sizes[nl]);
    free(z);
    free(h);
    return 0;
}

/* Loss (returned) and its gradient with respect to every parameter (grad,
 * packed like params). */
double or_mlp_loss_backward(int32_t nl, const int32_t *sizes, int64_t M, const double *X,
                            const double *shift, const double *scale, const double *params,
                            const double *T, double *grad)
{
    if (nl < 1 || nl > 16) return NAN;
    const double *W[16], *b[16];
    int64_t off[17];
    unpack(nl, sizes, params, W, b);
    int64_t tot = offsets(nl, sizes, off);
    int64_t np = 0;
    for (int32_t l = 1; l <= nl; ++l) np += (int64_t)sizes[l] * sizes[l - 1] + sizes[l];
    memset(grad, 0, sizeof(double) * (size_t)np);
    double *gW[16], *gb[16];
    {
        double *q = grad;
        for (int32_t l = 1; l <= nl; ++l) {
            gW[l - 1] = q;
            q += (int64_t)sizes[l] * sizes[l - 1];
            gb[l - 1] = q;
            q += sizes[l];
        }
    }
    double *z = (double *)malloc(sizeof(double) * (size_t)tot);
    double *h = (double *)malloc(sizeof(double) * (size_t)tot);
    double *d = (double *)malloc(sizeof(double) * (size_t)tot);
    double *p = (double *)malloc(sizeof(double) * (size_t)sizes[nl]);
    if (!z || !h || !d || !p) {
        free(z); free(h); free(d); free(p);
        return NAN;
    }
    double loss = 0.0;
    int32_t nc = sizes[nl];
    for (int64_t m = 0; m < M; ++m) {
        const double *t = T + m * nc;
        forward_row(nl, sizes, X + m * sizes[0], shift, scale, W, b, z, h, off, p);
        for (int32_t c = 0; c < nc; ++c)
            if (t[c] > 0.0) loss += t[c] * log(t[c] / p[c]) / (double)M;
        /* d loss / d logits = (p - t) sum(t) / M ... for normalised targets
         * sum(t) = 1; the general form keeps the softmax Jacobian exact */
        double st = 0.0;
        for (int32_t c = 0; c < nc; ++c) st += t[c];
        for (int32_t c = 0; c < nc; ++c) d[off[nl] + c] = (p[c] * st - t[c]) / (double)M;
        for (int32_t l = nl; l >= 1; --l) {
            int32_t in = sizes[l - 1], out = sizes[l];
            for (int32_t o = 0; o < out; ++o) {
                double g = d[off[l] + o];
                gb[l - 1][o] += g;
                for (int32_t i = 0; i < in; ++i) gW[l - 1][(int64_t)o * in + i] += g * h[off[l - 1] + i];
            }
            if (l > 1) {
                for (int32_t i = 0; i < in; ++i) {
                    double a = 0.0;
                    for (int32_t o = 0; o < out; ++o) a += W[l - 1][(int64_t)o * in + i] * d[off[l] + o];
                    d[off[l - 1] + i] = a * silu_grad(z[off[l - 1] + i]);
                }
            }
        }
    }
    free(z); free(h); free(d); free(p);
    return loss;
}
