/*
 * tvl1_oracle.c -- plain, slow, FP64 CPU oracle for the TV-L1 optical-flow solvers of
 * H. Sun, X.-C. Tai, J. Yuan, "Variational Image Motion Estimation by Accelerated Dual
 * Optimization" (arXiv 2011.10979).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant with the CUDA library: every
 * operator below is written out again from the paper's definitions, in double precision,
 * without blocking, fusion or reordering beyond what the paper states.
 *
 * Conventions (Sec. 2.2, discrete grid): an image is H rows x W columns, row-major,
 * element (i, j) at index i*W + j; x runs along columns j, y along rows i.  A dual field
 * p = (p1, p2) holds the x-component p1 and the y-component p2.  q1 = (q11, q12) is the dual
 * of u, q2 = (q21, q22) the dual of v.
 *
 * Where the paper is silent (pyramid, warping, linearisation point, dual warm start, which
 * image's gradient, boundary handling) the oracle takes one fixed reading; each reading is
 * marked "reading:" at the place it is used.
 *
 * Parity pins: every function here is pinned by a CPU test against a property fixed by the
 * paper or by mathematics (adjointness, projection invariants, brute-force prox, direct
 * solve for the Gauss-Seidel sweeps, subproblem optimality, strong duality at convergence).
 * The pyramid and warping readings are pinned against library routines (scipy.ndimage's
 * Gaussian filter and bilinear map_coordinates) and the whole schedule by a hand-computed
 * single-pixel solve and a step-by-step composition; the absolute flow values on the paper's
 * own sequences stay unpinned because those data sets are not available.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_AT(a, i, j) ((a)[(size_t)(i) * (size_t)W + (size_t)(j)])

/* ------------------------------------------------------------------------------------- */
/* Discrete operators, Sec. 2.2 (forward-difference gradient, divergence = -adjoint).     */
/* ------------------------------------------------------------------------------------- */

/* Forward-difference gradient with zero at the last column / row (Sec. 2.2, the
 * discretisation the paper takes from Chambolle-Pock). */
void orc_grad(int H, int W, const double *f, double *gx, double *gy)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            ORC_AT(gx, i, j) = (j < W - 1) ? ORC_AT(f, i, j + 1) - ORC_AT(f, i, j) : 0.0;
            ORC_AT(gy, i, j) = (i < H - 1) ? ORC_AT(f, i + 1, j) - ORC_AT(f, i, j) : 0.0;
        }
}

/* Discrete divergence, the unique map with <grad u, p> = -<u, div p> (Sec. 2.2). */
void orc_div(int H, int W, const double *px, const double *py, double *d)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double v = 0.0;
            if (j < W - 1) v += ORC_AT(px, i, j);
            if (j > 0) v -= ORC_AT(px, i, j - 1);
            if (i < H - 1) v += ORC_AT(py, i, j);
            if (i > 0) v -= ORC_AT(py, i - 1, j);
            ORC_AT(d, i, j) = v;
        }
}

/* ------------------------------------------------------------------------------------- */
/* Projections onto the dual balls, Sec. 3.1.1 (after eq. rpADMMI) with the norms of      */
/* eq. (euclid:norm).  Reading: the radius alpha is lambda for s and 1 for p and q.       */
/* ------------------------------------------------------------------------------------- */

void orc_proj_p(size_t n, double *p1, double *p2)
{
    for (size_t k = 0; k < n; ++k) {
        double nrm = sqrt(p1[k] * p1[k] + p2[k] * p2[k]);
        double f = nrm > 1.0 ? nrm : 1.0;
        p1[k] /= f;
        p2[k] /= f;
    }
}

/* Joint 4-component norm |q| = sqrt(q11^2 + q12^2 + q21^2 + q22^2) (eq. euclid:norm). */
void orc_proj_q(size_t n, double *q11, double *q12, double *q21, double *q22)
{
    for (size_t k = 0; k < n; ++k) {
        double nrm = sqrt(q11[k] * q11[k] + q12[k] * q12[k] + q21[k] * q21[k] + q22[k] * q22[k]);
        double f = nrm > 1.0 ? nrm : 1.0;
        q11[k] /= f;
        q12[k] /= f;
        q21[k] /= f;
        q22[k] /= f;
    }
}

void orc_proj_s(size_t n, double *s, double lambda)
{
    for (size_t k = 0; k < n; ++k) {
        double f = fabs(s[k]) / lambda;
        if (f < 1.0) f = 1.0;
        s[k] /= f;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Closed-form resolvent (I + sigma dF)^{-1} of F = lambda ||rho(w, d)||_1, eq. (resolvent) */
/* and its proof in the appendix.  e = (beta, Ix, Iy), |e|^2 = beta^2 + Ix^2 + Iy^2.      */
/* Inputs Z = (zw, zu, zv) are overwritten with the result.                               */
/* ------------------------------------------------------------------------------------- */

void orc_prox_l1(size_t n, double *zw, double *zu, double *zv, const double *Ix,
                 const double *Iy, const double *It, double beta, double lambda, double sigma)
{
    for (size_t k = 0; k < n; ++k) {
        double e2 = beta * beta + Ix[k] * Ix[k] + Iy[k] * Iy[k];
        double rho = It[k] + beta * zw[k] + Ix[k] * zu[k] + Iy[k] * zv[k];
        double t; /* X = Z + t * e */
        if (e2 <= 0.0)
            t = 0.0; /* rho does not depend on X: F is constant, the resolvent is the identity */
        else if (rho < -sigma * lambda * e2)
            t = sigma * lambda;
        else if (rho > sigma * lambda * e2)
            t = -sigma * lambda;
        else
            t = -rho / e2;
        zw[k] += t * beta;
        zu[k] += t * Ix[k];
        zv[k] += t * Iy[k];
    }
}

/* ------------------------------------------------------------------------------------- */
/* Red-black symmetric Gauss-Seidel for (I - st*Laplace) x = b with Neumann boundary,     */
/* Sec. 3.1.2, eq. (neumann:boudary).  Laplace = div grad with the operators above, so    */
/* row (i,j) of T reads (1 + st*n_ij) x_ij - st * sum of in-domain 4-neighbours.          */
/* One symmetric sweep = forward red-black pass (red, black) followed by the backward    */
/* pass (black, red).  Red pixels are (i + j) even.                                        */
/* ------------------------------------------------------------------------------------- */

static void orc_gs_colour(int H, int W, double *x, const double *b, double st, int colour)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            if (((i + j) & 1) != colour) continue;
            double acc = 0.0;
            int nb = 0;
            if (j > 0) { acc += ORC_AT(x, i, j - 1); ++nb; }
            if (j < W - 1) { acc += ORC_AT(x, i, j + 1); ++nb; }
            if (i > 0) { acc += ORC_AT(x, i - 1, j); ++nb; }
            if (i < H - 1) { acc += ORC_AT(x, i + 1, j); ++nb; }
            ORC_AT(x, i, j) = (ORC_AT(b, i, j) + st * acc) / (1.0 + st * nb);
        }
}

void orc_srbgs(int H, int W, double *x, const double *b, double st, int sweeps)
{
    for (int s = 0; s < sweeps; ++s) {
        orc_gs_colour(H, W, x, b, st, 0); /* forward: red   */
        orc_gs_colour(H, W, x, b, st, 1); /* forward: black */
        orc_gs_colour(H, W, x, b, st, 1); /* backward: black */
        orc_gs_colour(H, W, x, b, st, 0); /* backward: red   */
    }
}

/* ------------------------------------------------------------------------------------- */
/* Coarse-to-fine pyramid (Sec. 4 names a standard pyramid and gives no details).          */
/* Reading: H_{l+1} = max(1, floor(H_l*eta + 0.5)); pre-smoothing by a separable           */
/* normalised Gaussian with sigma_g = 0.6*sqrt(eta^-2 - 1), radius ceil(3*sigma_g),        */
/* half-sample symmetric extension; then bilinear sampling at                              */
/* x_f = (x_c + 0.5) * W_f / W_c - 0.5, clamped to [0, W_f - 1].                            */
/* ------------------------------------------------------------------------------------- */

int orc_level_size(int n, double eta) /* size of the next coarser level */
{
    int m = (int)floor((double)n * eta + 0.5);
    return m < 1 ? 1 : m;
}

static int orc_reflect(int k, int n) /* half-sample symmetric extension, any integer k */
{
    int period = 2 * n;
    int m = k % period;
    if (m < 0) m += period;
    return m < n ? m : period - 1 - m;
}

/* Bilinear value of f (H x W) at real position (x, y) already inside [0,W-1]x[0,H-1]. */
static double orc_bilinear(int H, int W, const double *f, double x, double y)
{
    int x0 = (int)floor(x), y0 = (int)floor(y);
    double fx = x - x0, fy = y - y0;
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
    int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    double top = (1.0 - fx) * ORC_AT(f, y0, x0) + fx * ORC_AT(f, y0, x1);
    double bot = (1.0 - fx) * ORC_AT(f, y1, x0) + fx * ORC_AT(f, y1, x1);
    return (1.0 - fy) * top + fy * bot;
}

static double orc_clamp(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Gaussian pre-smoothing of a Hf x Wf image (separable: along rows first, then columns). */
void orc_gauss_smooth(int H, int W, const double *in, double *out, double eta)
{
    double sg = 0.6 * sqrt(1.0 / (eta * eta) - 1.0);
    int R = (int)ceil(3.0 * sg);
    double *g = (double *)malloc(sizeof(double) * (size_t)(2 * R + 1));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)H * (size_t)W);
    double sum = 0.0;
    for (int k = -R; k <= R; ++k) { g[k + R] = exp(-(double)(k * k) / (2.0 * sg * sg)); sum += g[k + R]; }
    for (int k = 0; k <= 2 * R; ++k) g[k] /= sum;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int k = -R; k <= R; ++k) acc += g[k + R] * ORC_AT(in, i, orc_reflect(j + k, W));
            ORC_AT(tmp, i, j) = acc;
        }
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int k = -R; k <= R; ++k) acc += g[k + R] * ORC_AT(tmp, orc_reflect(i + k, H), j);
            ORC_AT(out, i, j) = acc;
        }
    free(tmp);
    free(g);
}

/* One pyramid step: fine (Hf x Wf) -> coarse (Hc x Wc). */
void orc_downsample(int Hf, int Wf, const double *fine, int Hc, int Wc, double *coarse, double eta)
{
    double *sm = (double *)malloc(sizeof(double) * (size_t)Hf * (size_t)Wf);
    orc_gauss_smooth(Hf, Wf, fine, sm, eta);
    int W = Wc;
    for (int i = 0; i < Hc; ++i)
        for (int j = 0; j < Wc; ++j) {
            double xf = orc_clamp((j + 0.5) * (double)Wf / (double)Wc - 0.5, 0.0, (double)(Wf - 1));
            double yf = orc_clamp((i + 0.5) * (double)Hf / (double)Hc - 0.5, 0.0, (double)(Hf - 1));
            ORC_AT(coarse, i, j) = orc_bilinear(Hf, Wf, sm, xf, yf);
        }
    free(sm);
}

/* Level transfer of a field: bilinear sampling at x_c = (x_f + 0.5) * W_c / W_f - 0.5,
 * clamped, times `scale` (W_f/W_c for u, H_f/H_c for v, 1 for w).  Reading of Sec. 4. */
void orc_upsample(int Hc, int Wc, const double *coarse, int Hf, int Wf, double *fine, double scale)
{
    int W = Wf;
    for (int i = 0; i < Hf; ++i)
        for (int j = 0; j < Wf; ++j) {
            double xc = orc_clamp((j + 0.5) * (double)Wc / (double)Wf - 0.5, 0.0, (double)(Wc - 1));
            double yc = orc_clamp((i + 0.5) * (double)Hc / (double)Hf - 0.5, 0.0, (double)(Hc - 1));
            ORC_AT(fine, i, j) = scale * orc_bilinear(Hc, Wc, coarse, xc, yc);
        }
}

/* ------------------------------------------------------------------------------------- */
/* Derivative images and warping (Sec. 1, the optical-flow constraint; Sec. 4 warping).   */
/* ------------------------------------------------------------------------------------- */

/* Reading: central differences of I1 with clamped indices, once per level. */
void orc_derivatives(int H, int W, const double *I, double *Ix, double *Iy)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            int jl = j > 0 ? j - 1 : 0, jr = j < W - 1 ? j + 1 : W - 1;
            int iu = i > 0 ? i - 1 : 0, id = i < H - 1 ? i + 1 : H - 1;
            ORC_AT(Ix, i, j) = 0.5 * (ORC_AT(I, i, jr) - ORC_AT(I, i, jl));
            ORC_AT(Iy, i, j) = 0.5 * (ORC_AT(I, id, j) - ORC_AT(I, iu, j));
        }
}

/* Warp I1 and its derivatives to (j + u0, i + v0) (clamped to the image), and linearise the
 * constraint I1(x + d) - I0(x) around d0 = (u0, v0):
 *   rho(w, d) = Ix*u + Iy*v + beta*w + It,  It = I1w - I0 - Ix*u0 - Iy*v0.
 * Reading of eq. (l1:optical:flow) inside the warping loop.  Returns max M_s with
 * M_s = beta^2 + Ix^2 + Iy^2 (Sec. 3.1.1 after eq. aug:pre1:vector). */
double orc_warp_linearise(int H, int W, const double *I0, const double *I1, const double *I1x,
                          const double *I1y, const double *u0, const double *v0, double beta,
                          double *Ix, double *Iy, double *It)
{
    double msmax = 0.0;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double xs = orc_clamp(j + ORC_AT(u0, i, j), 0.0, (double)(W - 1));
            double ys = orc_clamp(i + ORC_AT(v0, i, j), 0.0, (double)(H - 1));
            double w1 = orc_bilinear(H, W, I1, xs, ys);
            double gx = orc_bilinear(H, W, I1x, xs, ys);
            double gy = orc_bilinear(H, W, I1y, xs, ys);
            ORC_AT(Ix, i, j) = gx;
            ORC_AT(Iy, i, j) = gy;
            ORC_AT(It, i, j) = w1 - ORC_AT(I0, i, j) - gx * ORC_AT(u0, i, j) - gy * ORC_AT(v0, i, j);
            double ms = beta * beta + gx * gx + gy * gy;
            if (ms > msmax) msmax = ms;
        }
    return msmax;
}

/* ------------------------------------------------------------------------------------- */
/* Solver state and parameters                                                             */
/* ------------------------------------------------------------------------------------- */

typedef struct {
    int method;        /* 0 = rpADMMI (pADMM if r = 1), 1 = rpADMMII, 2 = pDR, 3 = ALG1 (primal-dual) */
    double lambda;     /* data weight, |s| <= lambda */
    double beta;       /* illumination weight; 0 = the beta = 0 model (no w, no p) */
    double c;          /* ADMM penalty c */
    double a;          /* preconditioner a of the y block */
    double a_tilde;    /* preconditioner of the s block; <= 0: max M_s per warp */
    double r;          /* rpADMMI relaxation */
    double rho;        /* rpADMMII relaxation */
    double sigma, tau; /* pDR step sizes */
    int gs_sweeps;     /* symmetric red-black Gauss-Seidel sweeps per pDR iteration */
    double eta;        /* pyramid scale */
    int levels, warps, iters;
    double tol;        /* > 0: stop a warp's inner loop once the residual < tol (checked every 10) */
    int out_level;     /* stop after this pyramid level and return its flow */
    double cp_tau;     /* ALG1 dual step */
    double cp_sigma;   /* ALG1 primal step */
    int a_tilde_mode;  /* 0: one a~ per warp (the paper's ||M_s||); 1: per-pixel a~_ij = M_s(ij) */
    int c_adapt_iters; /* 0: fixed steps; K > 0: residual balancing in the first K iterations of
                          every level's first warp, frozen afterwards (an extension): the ADMM
                          step c, or pDR's sigma and tau with sigma tau fixed */
} orc_params;

typedef struct {
    /* ADMM: Lagrange multipliers (w, u, v), duals p, q, s.
     * pDR: X = (w, u, v), Xbar = (wb, ub, vb), ybar = (p, q); s unused.
     * ALG1: X = (w, u, v), the extrapolated Xbar = (wb, ub, vb), y = (p, q); s unused. */
    double *w, *u, *v;
    double *p1, *p2, *q11, *q12, *q21, *q22, *s;
    double *wb, *ub, *vb;
} orc_state;

typedef struct {
    long long iters_run;
    double residual, energy, dual_value;
    double c_final;      /* ADMM step c (pDR: the primal step sigma) at the end of the solve */
    double adapt_margin; /* smallest |log| distance of a balancing test from its thresholds
                            (HUGE_VAL when no test ran): how far each decision was from a tie */
} orc_stats;

static double *orc_alloc(size_t n) { return (double *)calloc(n, sizeof(double)); }

/* ------------------------------------------------------------------------------------- */
/* rpADMMI (Sec. 3.1.1, eq. rpADMMI): one iteration, component form.  pADMM is r = 1;     */
/* the beta = 0 case drops w and p and is Zach-pADMM (eq. Zach-pADMM) when r = 1.         */
/* rpADMMII (eq. rpADMMII) differs in the s-update weights and the multiplier update.     */
/* Reading: (I - (1/a) grad grad^*) p = p + (1/a) grad(div p), because grad^* = -div.       */
/* Returns the squared constraint residual ||A s + B y||^2 after the step.                 */
/* ------------------------------------------------------------------------------------- */

double orc_admm_step(int H, int W, orc_state *st, const double *Ix, const double *Iy,
                     const double *It, double a_tilde, const orc_params *P)
{
    size_t N = (size_t)H * (size_t)W;
    int has_w = P->beta != 0.0;
    double a = P->a, c = P->c, beta = P->beta;
    double *d = orc_alloc(N), *gx = orc_alloc(N), *gy = orc_alloc(N), *hx = orc_alloc(N), *hy = orc_alloc(N);
    double *sIx = orc_alloc(N), *sIy = orc_alloc(N);
    double *np1 = orc_alloc(N), *np2 = orc_alloc(N);
    double *nq11 = orc_alloc(N), *nq12 = orc_alloc(N), *nq21 = orc_alloc(N), *nq22 = orc_alloc(N);
    double *dp = orc_alloc(N), *dq1 = orc_alloc(N), *dq2 = orc_alloc(N);

    /* y-update: p^{k+1} = P_p[p + (1/a) grad div p + (1/a)(grad w / c - beta grad s)] */
    if (has_w) {
        orc_div(H, W, st->p1, st->p2, d);
        orc_grad(H, W, d, gx, gy);                       /* grad div p^k */
        orc_grad(H, W, st->w, hx, hy);                   /* grad w^k     */
        double *sx = orc_alloc(N), *sy = orc_alloc(N);
        orc_grad(H, W, st->s, sx, sy);                   /* grad s^k     */
        for (size_t k = 0; k < N; ++k) {
            np1[k] = st->p1[k] + gx[k] / a + (hx[k] / c - beta * sx[k]) / a;
            np2[k] = st->p2[k] + gy[k] / a + (hy[k] / c - beta * sy[k]) / a;
        }
        free(sx);
        free(sy);
        orc_proj_p(N, np1, np2);
    }
    /* q1, q2 with grad(s Ix), grad(s Iy), then the joint projection P_q */
    for (size_t k = 0; k < N; ++k) { sIx[k] = st->s[k] * Ix[k]; sIy[k] = st->s[k] * Iy[k]; }
    {
        double *sx = orc_alloc(N), *sy = orc_alloc(N);
        orc_div(H, W, st->q11, st->q12, d);
        orc_grad(H, W, d, gx, gy);
        orc_grad(H, W, st->u, hx, hy);
        orc_grad(H, W, sIx, sx, sy);
        for (size_t k = 0; k < N; ++k) {
            nq11[k] = st->q11[k] + gx[k] / a + (hx[k] / c - sx[k]) / a;
            nq12[k] = st->q12[k] + gy[k] / a + (hy[k] / c - sy[k]) / a;
        }
        orc_div(H, W, st->q21, st->q22, d);
        orc_grad(H, W, d, gx, gy);
        orc_grad(H, W, st->v, hx, hy);
        orc_grad(H, W, sIy, sx, sy);
        for (size_t k = 0; k < N; ++k) {
            nq21[k] = st->q21[k] + gx[k] / a + (hx[k] / c - sx[k]) / a;
            nq22[k] = st->q22[k] + gy[k] / a + (hy[k] / c - sy[k]) / a;
        }
        free(sx);
        free(sy);
        orc_proj_q(N, nq11, nq12, nq21, nq22);
    }
    /* divergences of y^{k+1} */
    if (has_w) orc_div(H, W, np1, np2, dp);
    orc_div(H, W, nq11, nq12, dq1);
    orc_div(H, W, nq21, nq22, dq2);

    /* s-update with the old multipliers Lambda^k and the new y^{k+1}, then P_s.
     * Per-pixel preconditioner (a_tilde_mode 1): M_s is diagonal, so the s-block proximal matrix
     * c(diag(a~) - M_s) stays positive semidefinite with a~_ij = M_s(ij) (floored at 1e-12),
     * the pointwise form of the paper's a~ = ||M_s|| (Prop. 3.1). */
    double res2 = 0.0;
    for (size_t k = 0; k < N; ++k) {
        double ms = beta * beta + Ix[k] * Ix[k] + Iy[k] * Iy[k];
        double a_tilde_k = P->a_tilde_mode == 1 ? (ms > 1e-12 ? ms : 1e-12) : a_tilde;
        double lin = It[k] + Ix[k] * st->u[k] + Iy[k] * st->v[k] + (has_w ? beta * st->w[k] : 0.0);
        double divterm = Ix[k] * dq1[k] + Iy[k] * dq2[k] + (has_w ? beta * dp[k] : 0.0);
        double s_old = st->s[k], s_new;
        if (P->method == 1) {
            double rho = P->rho;
            s_new = (1.0 - rho * ms / a_tilde_k) * s_old + (lin + c * rho * divterm) / (a_tilde_k * c);
        } else {
            s_new = (1.0 - ms / a_tilde_k) * s_old + (lin + c * divterm) / (a_tilde_k * c);
        }
        {
            double f = fabs(s_new) / P->lambda;
            if (f < 1.0) f = 1.0;
            s_new /= f; /* P_s */
        }
        /* multiplier update */
        double cw, cu, cv; /* A s^{k+1} + B y^{k+1}, the constraint of eq. (dual:l1:flow:constaint) */
        cw = has_w ? beta * s_new - dp[k] : 0.0;
        cu = Ix[k] * s_new - dq1[k];
        cv = Iy[k] * s_new - dq2[k];
        if (P->method == 1) {
            double rho = P->rho;
            if (has_w) st->w[k] -= c * (beta * s_new - rho * dp[k] - (1.0 - rho) * beta * s_old);
            st->u[k] -= c * (Ix[k] * s_new - rho * dq1[k] - (1.0 - rho) * Ix[k] * s_old);
            st->v[k] -= c * (Iy[k] * s_new - rho * dq2[k] - (1.0 - rho) * Iy[k] * s_old);
        } else {
            double rc = P->r * c;
            if (has_w) st->w[k] -= rc * cw;
            st->u[k] -= rc * cu;
            st->v[k] -= rc * cv;
        }
        st->s[k] = s_new;
        res2 += cw * cw + cu * cu + cv * cv;
    }
    if (has_w) { memcpy(st->p1, np1, N * sizeof(double)); memcpy(st->p2, np2, N * sizeof(double)); }
    memcpy(st->q11, nq11, N * sizeof(double));
    memcpy(st->q12, nq12, N * sizeof(double));
    memcpy(st->q21, nq21, N * sizeof(double));
    memcpy(st->q22, nq22, N * sizeof(double));

    free(d); free(gx); free(gy); free(hx); free(hy); free(sIx); free(sIy);
    free(np1); free(np2); free(nq11); free(nq12); free(nq21); free(nq22);
    free(dp); free(dq1); free(dq2);
    return res2;
}

/* ------------------------------------------------------------------------------------- */
/* pDR (Sec. 3.1.2, eq. pDR for the flow model): one iteration.                            */
/*   b = Xbar + sigma div ybar;  X^{k+1} = SRBGS^n(T, b, X^k),  T = I - sigma tau Laplace;  */
/*   Xbar^{k+1} = Xbar + prox_{sigma F}(2 X^{k+1} - Xbar) - X^{k+1};                        */
/*   pbar^{k+1} = P_p(pbar + 2 tau grad w^{k+1}) - tau grad w^{k+1}; likewise qbar (joint). */
/* Reading: the dual variables entering b are the barred ones (generic pDR, first line).    */
/* Returns ||X^{k+1} - X^k||^2.                                                              */
/* ------------------------------------------------------------------------------------- */

double orc_pdr_step(int H, int W, orc_state *st, const double *Ix, const double *Iy,
                    const double *It, const orc_params *P)
{
    size_t N = (size_t)H * (size_t)W;
    int has_w = P->beta != 0.0;
    double sg = P->sigma, ta = P->tau;
    double *b = orc_alloc(N), *d = orc_alloc(N), *old = orc_alloc(N);
    double *zw = orc_alloc(N), *zu = orc_alloc(N), *zv = orc_alloc(N);
    double *gx = orc_alloc(N), *gy = orc_alloc(N);
    double diff2 = 0.0;

    double *X[3] = {st->w, st->u, st->v};
    double *Xb[3] = {st->wb, st->ub, st->vb};
    double *Y1[3] = {st->p1, st->q11, st->q21};
    double *Y2[3] = {st->p2, st->q12, st->q22};
    for (int c = has_w ? 0 : 1; c < 3; ++c) {
        orc_div(H, W, Y1[c], Y2[c], d);
        for (size_t k = 0; k < N; ++k) b[k] = Xb[c][k] + sg * d[k];
        memcpy(old, X[c], N * sizeof(double));
        orc_srbgs(H, W, X[c], b, sg * ta, P->gs_sweeps);
        for (size_t k = 0; k < N; ++k) { double e = X[c][k] - old[k]; diff2 += e * e; }
    }
    /* Xbar update through the L1 resolvent at Z = 2 X^{k+1} - Xbar^k */
    for (size_t k = 0; k < N; ++k) {
        zw[k] = has_w ? 2.0 * st->w[k] - st->wb[k] : 0.0;
        zu[k] = 2.0 * st->u[k] - st->ub[k];
        zv[k] = 2.0 * st->v[k] - st->vb[k];
    }
    orc_prox_l1(N, zw, zu, zv, Ix, Iy, It, P->beta, P->lambda, sg);
    for (size_t k = 0; k < N; ++k) {
        if (has_w) st->wb[k] += zw[k] - st->w[k];
        st->ub[k] += zu[k] - st->u[k];
        st->vb[k] += zv[k] - st->v[k];
    }
    /* ybar update */
    if (has_w) {
        orc_grad(H, W, st->w, gx, gy);
        for (size_t k = 0; k < N; ++k) { zu[k] = st->p1[k] + 2.0 * ta * gx[k]; zv[k] = st->p2[k] + 2.0 * ta * gy[k]; }
        orc_proj_p(N, zu, zv);
        for (size_t k = 0; k < N; ++k) { st->p1[k] = zu[k] - ta * gx[k]; st->p2[k] = zv[k] - ta * gy[k]; }
    }
    {
        double *ux = orc_alloc(N), *uy = orc_alloc(N), *vx = orc_alloc(N), *vy = orc_alloc(N);
        double *t11 = orc_alloc(N), *t12 = orc_alloc(N), *t21 = orc_alloc(N), *t22 = orc_alloc(N);
        orc_grad(H, W, st->u, ux, uy);
        orc_grad(H, W, st->v, vx, vy);
        for (size_t k = 0; k < N; ++k) {
            t11[k] = st->q11[k] + 2.0 * ta * ux[k];
            t12[k] = st->q12[k] + 2.0 * ta * uy[k];
            t21[k] = st->q21[k] + 2.0 * ta * vx[k];
            t22[k] = st->q22[k] + 2.0 * ta * vy[k];
        }
        orc_proj_q(N, t11, t12, t21, t22);
        for (size_t k = 0; k < N; ++k) {
            st->q11[k] = t11[k] - ta * ux[k];
            st->q12[k] = t12[k] - ta * uy[k];
            st->q21[k] = t21[k] - ta * vx[k];
            st->q22[k] = t22[k] - ta * vy[k];
        }
        free(ux); free(uy); free(vx); free(vy); free(t11); free(t12); free(t21); free(t22);
    }
    free(b); free(d); free(old); free(zw); free(zu); free(zv); free(gx); free(gy);
    return diff2;
}

/* ------------------------------------------------------------------------------------- */
/* ALG1 (Sec. 4): the first-order primal-dual method of Chambolle and Pock with constant   */
/* steps and theta = 1, applied to the saddle-point form eq. (primal-dual:optical:o) with   */
/* K = (grad w, grad u, grad v), F(X) = lambda ||rho(w, d)||_1, G^* = the indicators of     */
/* the unit balls of p and (jointly) q.  One iteration:                                     */
/*   y^{k+1}    = P(y^k + tau K Xbar^k)              (P_p on p, P_q on q)                    */
/*   X^{k+1}    = prox_{sigma F}(X^k - sigma K^* y^{k+1}) = prox_{sigma F}(X^k + sigma div y) */
/*   Xbar^{k+1} = 2 X^{k+1} - X^k.                                                           */
/* Reading: the printed step rule "sigma = 1/(L^2 sigma)" is sigma = 1/(L^2 tau), L^2 = 8,   */
/* with tau = 0.1 the dual step, so sigma = 1.25.  Returns ||X^{k+1} - X^k||^2.              */
/* ------------------------------------------------------------------------------------- */

double orc_cp_step(int H, int W, orc_state *st, const double *Ix, const double *Iy,
                   const double *It, const orc_params *P)
{
    size_t N = (size_t)H * (size_t)W;
    int has_w = P->beta != 0.0;
    double ta = P->cp_tau, sg = P->cp_sigma;
    double *gx = orc_alloc(N), *gy = orc_alloc(N), *gx2 = orc_alloc(N), *gy2 = orc_alloc(N);
    double *d = orc_alloc(N), *zw = orc_alloc(N), *zu = orc_alloc(N), *zv = orc_alloc(N);
    double diff2 = 0.0;

    /* dual ascent on the extrapolated primal point, then projection */
    if (has_w) {
        orc_grad(H, W, st->wb, gx, gy);
        for (size_t k = 0; k < N; ++k) { st->p1[k] += ta * gx[k]; st->p2[k] += ta * gy[k]; }
        orc_proj_p(N, st->p1, st->p2);
    }
    orc_grad(H, W, st->ub, gx, gy);
    orc_grad(H, W, st->vb, gx2, gy2);
    for (size_t k = 0; k < N; ++k) {
        st->q11[k] += ta * gx[k];
        st->q12[k] += ta * gy[k];
        st->q21[k] += ta * gx2[k];
        st->q22[k] += ta * gy2[k];
    }
    orc_proj_q(N, st->q11, st->q12, st->q21, st->q22);
    /* primal descent along div y^{k+1}, then the L1 resolvent */
    if (has_w) {
        orc_div(H, W, st->p1, st->p2, d);
        for (size_t k = 0; k < N; ++k) zw[k] = st->w[k] + sg * d[k];
    }
    orc_div(H, W, st->q11, st->q12, d);
    for (size_t k = 0; k < N; ++k) zu[k] = st->u[k] + sg * d[k];
    orc_div(H, W, st->q21, st->q22, d);
    for (size_t k = 0; k < N; ++k) zv[k] = st->v[k] + sg * d[k];
    orc_prox_l1(N, zw, zu, zv, Ix, Iy, It, P->beta, P->lambda, sg);
    /* extrapolation */
    for (size_t k = 0; k < N; ++k) {
        double e;
        if (has_w) {
            e = zw[k] - st->w[k];
            diff2 += e * e;
            st->wb[k] = 2.0 * zw[k] - st->w[k];
            st->w[k] = zw[k];
        }
        e = zu[k] - st->u[k];
        diff2 += e * e;
        st->ub[k] = 2.0 * zu[k] - st->u[k];
        st->u[k] = zu[k];
        e = zv[k] - st->v[k];
        diff2 += e * e;
        st->vb[k] = 2.0 * zv[k] - st->v[k];
        st->v[k] = zv[k];
    }
    free(gx); free(gy); free(gx2); free(gy2); free(d); free(zw); free(zu); free(zv);
    return diff2;
}

/* ------------------------------------------------------------------------------------- */
/* Energy of the discrete primal problem, eq. (l1:finite): ||grad w||_1 + ||grad d||_1     */
/* + lambda ||rho(w, d)||_1, with the pointwise norms of eq. (euclid:norm) (joint for d),  */
/* and the dual objective <It, s> of eq. (dual:l1:flow:cons).                              */
/* ------------------------------------------------------------------------------------- */

double orc_energy(int H, int W, const double *w, const double *u, const double *v,
                  const double *Ix, const double *Iy, const double *It, double beta, double lambda)
{
    size_t N = (size_t)H * (size_t)W;
    double *ux = orc_alloc(N), *uy = orc_alloc(N), *vx = orc_alloc(N), *vy = orc_alloc(N);
    double E = 0.0;
    orc_grad(H, W, u, ux, uy);
    orc_grad(H, W, v, vx, vy);
    for (size_t k = 0; k < N; ++k) {
        E += sqrt(ux[k] * ux[k] + uy[k] * uy[k] + vx[k] * vx[k] + vy[k] * vy[k]);
        double rho = Ix[k] * u[k] + Iy[k] * v[k] + It[k] + (beta != 0.0 ? beta * w[k] : 0.0);
        E += lambda * fabs(rho);
    }
    if (beta != 0.0) {
        orc_grad(H, W, w, ux, uy);
        for (size_t k = 0; k < N; ++k) E += sqrt(ux[k] * ux[k] + uy[k] * uy[k]);
    }
    free(ux); free(uy); free(vx); free(vy);
    return E;
}

double orc_dual_value(size_t n, const double *It, const double *s)
{
    double acc = 0.0;
    for (size_t k = 0; k < n; ++k) acc += It[k] * s[k];
    return acc;
}

/* ------------------------------------------------------------------------------------- */
/* Residual balancing of the ADMM step c (an extension: the paper keeps c fixed).  The    */
/* stepsize conditions (eq. stepsize:constraint, Prop. 3.1) bound only a and a~, so every  */
/* c > 0 keeps the proximal metrics c(aI - grad grad^*) and c(a~ - M_s) positive           */
/* semidefinite, and the multipliers are unscaled, so c may change between iterations.     */
/* Residuals after the step prev -> cur of eq. (aug:pre1:vector), from the optimality      */
/* conditions of its two subproblems (B^*A ds = grad(beta ds), grad(Ix ds), grad(Iy ds);   */
/* B^*B = grad grad^* = -grad div per component):                                          */
/*   primal   r = A s + B y                     = (beta s - div p, Ix s - div q1, Iy s - div q2) */
/*   dual     d_y = c(B^*A ds - (aI - B^*B) dy) = c(grad(A_k ds) - a dy_k - grad div dy_k)  */
/*            d_s = c(M_s - a~) ds                                                          */
/* Reading: the same residuals serve rpADMMI with r != 1 and rpADMMII.                      */
/* ------------------------------------------------------------------------------------- */

void orc_adapt_residuals(int H, int W, const orc_state *prev, const orc_state *cur, const double *Ix,
                         const double *Iy, double a_tilde, double c, const orc_params *P, double *r_norm,
                         double *d_norm)
{
    size_t N = (size_t)H * (size_t)W;
    int has_w = P->beta != 0.0;
    double a = P->a, beta = P->beta;
    double *d = orc_alloc(N), *gx = orc_alloc(N), *gy = orc_alloc(N), *hx = orc_alloc(N), *hy = orc_alloc(N);
    double *ds = orc_alloc(N), *t = orc_alloc(N), *e1 = orc_alloc(N), *e2 = orc_alloc(N);
    double r2 = 0.0, d2 = 0.0;

    /* primal residual at cur */
    for (int comp = has_w ? 0 : 1; comp < 3; ++comp) {
        const double *x = comp == 0 ? cur->p1 : comp == 1 ? cur->q11 : cur->q21;
        const double *y = comp == 0 ? cur->p2 : comp == 1 ? cur->q12 : cur->q22;
        orc_div(H, W, x, y, d);
        for (size_t k = 0; k < N; ++k) {
            double ak = comp == 0 ? beta : comp == 1 ? Ix[k] : Iy[k];
            double rk = ak * cur->s[k] - d[k];
            r2 += rk * rk;
        }
    }
    /* dual residual, y block: one 2-vector dual per component (p; q1; q2) */
    for (size_t k = 0; k < N; ++k) ds[k] = cur->s[k] - prev->s[k];
    for (int comp = has_w ? 0 : 1; comp < 3; ++comp) {
        const double *xc = comp == 0 ? cur->p1 : comp == 1 ? cur->q11 : cur->q21;
        const double *yc = comp == 0 ? cur->p2 : comp == 1 ? cur->q12 : cur->q22;
        const double *xp = comp == 0 ? prev->p1 : comp == 1 ? prev->q11 : prev->q21;
        const double *yp = comp == 0 ? prev->p2 : comp == 1 ? prev->q12 : prev->q22;
        for (size_t k = 0; k < N; ++k) {
            e1[k] = xc[k] - xp[k];
            e2[k] = yc[k] - yp[k];
            t[k] = (comp == 0 ? beta : comp == 1 ? Ix[k] : Iy[k]) * ds[k]; /* A_comp ds */
        }
        orc_grad(H, W, t, hx, hy);  /* B^*A ds, this component */
        orc_div(H, W, e1, e2, d);
        orc_grad(H, W, d, gx, gy);  /* grad div dy = -B^*B dy */
        for (size_t k = 0; k < N; ++k) {
            double dx = c * (hx[k] - a * e1[k] - gx[k]);
            double dy = c * (hy[k] - a * e2[k] - gy[k]);
            d2 += dx * dx + dy * dy;
        }
    }
    /* dual residual, s block */
    for (size_t k = 0; k < N; ++k) {
        double ms = beta * beta + Ix[k] * Ix[k] + Iy[k] * Iy[k];
        double at = P->a_tilde_mode == 1 ? (ms > 1e-12 ? ms : 1e-12) : a_tilde;
        double dk = c * (ms - at) * ds[k];
        d2 += dk * dk;
    }
    free(d); free(gx); free(gy); free(hx); free(hy); free(ds); free(t); free(e1); free(e2);
    *r_norm = sqrt(r2);
    *d_norm = sqrt(d2);
}

/* The balancing rule: c doubled when ||r|| > 10 ||d||, halved when ||d|| > 10 ||r||,
 * kept otherwise (residual balancing with mu = 10 and factor 2). */
double orc_adapt_rule(double c, double r_norm, double d_norm)
{
    if (r_norm > 10.0 * d_norm) return 2.0 * c;
    if (d_norm > 10.0 * r_norm) return 0.5 * c;
    return c;
}

/* Runs `iters` inner iterations at one linearisation; the stopping test of the schedule
 * (residual < tol, checked every 10 iterations) applies when tol > 0.  Returns iterations
 * run; *res_out gets the last residual sqrt(||.||^2 / n_rows). */
long long orc_inner(int H, int W, orc_state *st, const double *Ix, const double *Iy,
                    const double *It, double a_tilde, const orc_params *P, int iters, double *res_out)
{
    size_t N = (size_t)H * (size_t)W;
    double nrows = (double)N * (P->beta != 0.0 ? 3.0 : 2.0);
    double res = 0.0;
    long long k;
    for (k = 0; k < iters; ++k) {
        double r2 = P->method == 2   ? orc_pdr_step(H, W, st, Ix, Iy, It, P)
                     : P->method == 3 ? orc_cp_step(H, W, st, Ix, Iy, It, P)
                                      : orc_admm_step(H, W, st, Ix, Iy, It, a_tilde, P);
        res = sqrt(r2 / nrows);
        if (P->tol > 0.0 && (k + 1) % 10 == 0 && res < P->tol) { ++k; break; }
    }
    if (res_out) *res_out = res;
    return k;
}

/* pDR (Sec. 3.1.2) leaves sigma and tau free.  The SRBGS preconditioner is built for
 * T = I - sigma tau Laplace, so the balancing keeps sigma tau fixed and moves their ratio:
 * sigma -> theta sigma, tau -> tau / theta.  Its residuals after the step prev -> cur are the
 * primal change ||X^{k+1} - X^k|| / sigma and the dual change ||ybar^{k+1} - ybar^k|| / tau
 * (each a change of its block's iterate per unit step); the rule of orc_adapt_rule then doubles
 * theta when the primal change is more than 10 times the dual one and halves it in the opposite
 * case.  Reading: a heuristic in the spirit of residual balancing for primal-dual methods; the
 * paper gives no rule. */
void orc_pdr_adapt_residuals(int H, int W, const orc_state *prev, const orc_state *cur, double sigma,
                             double tau, const orc_params *P, double *rx, double *ry)
{
    size_t N = (size_t)H * (size_t)W;
    int has_w = P->beta != 0.0;
    const double *xp[3] = {prev->w, prev->u, prev->v}, *xc[3] = {cur->w, cur->u, cur->v};
    const double *yp[6] = {prev->p1, prev->p2, prev->q11, prev->q12, prev->q21, prev->q22};
    const double *yc[6] = {cur->p1, cur->p2, cur->q11, cur->q12, cur->q21, cur->q22};
    double x2 = 0.0, y2 = 0.0;
    for (int c = has_w ? 0 : 1; c < 3; ++c)
        for (size_t k = 0; k < N; ++k) { double e = xc[c][k] - xp[c][k]; x2 += e * e; }
    for (int c = has_w ? 0 : 2; c < 6; ++c)
        for (size_t k = 0; k < N; ++k) { double e = yc[c][k] - yp[c][k]; y2 += e * e; }
    *rx = sqrt(x2) / sigma;
    *ry = sqrt(y2) / tau;
}

/* The first warp of a level under pDR's adaptive steps: like orc_inner_adapt, with theta (the
 * factor on sigma, 1 / theta on tau) carried in *theta. */
long long orc_inner_adapt_pdr(int H, int W, orc_state *st, const double *Ix, const double *Iy,
                              const double *It, const orc_params *P, int iters, int window, double *theta,
                              double *margin, double *res_out)
{
    size_t N = (size_t)H * (size_t)W;
    double nrows = (double)N * (P->beta != 0.0 ? 3.0 : 2.0);
    orc_params Q = *P;
    orc_state prev;
    memset(&prev, 0, sizeof(prev));
    double **pk[9] = {&prev.w, &prev.u, &prev.v, &prev.p1, &prev.p2, &prev.q11, &prev.q12, &prev.q21, &prev.q22};
    double *ps[9] = {st->w, st->u, st->v, st->p1, st->p2, st->q11, st->q12, st->q21, st->q22};
    for (int f = 0; f < 9; ++f) *pk[f] = orc_alloc(N);
    int kw = window < iters ? window : iters;
    double res = 0.0;
    for (int k = 0; k < kw; ++k) {
        int test = (k + 1) % 10 == 0;
        Q.sigma = P->sigma * *theta;
        Q.tau = P->tau / *theta;
        if (test)
            for (int f = 0; f < 9; ++f) memcpy(*pk[f], ps[f], N * sizeof(double));
        res = sqrt(orc_pdr_step(H, W, st, Ix, Iy, It, &Q) / nrows);
        if (test) {
            double rx, ry;
            orc_pdr_adapt_residuals(H, W, &prev, st, Q.sigma, Q.tau, P, &rx, &ry);
            double m1 = fabs(log(rx / (10.0 * ry))), m2 = fabs(log(ry / (10.0 * rx)));
            if (m1 < *margin) *margin = m1;
            if (m2 < *margin) *margin = m2;
            *theta = orc_adapt_rule(*theta, rx, ry);
        }
    }
    for (int f = 0; f < 9; ++f) free(*pk[f]);
    Q.sigma = P->sigma * *theta;
    Q.tau = P->tau / *theta;
    long long n = kw;
    if (iters > kw) n += orc_inner(H, W, st, Ix, Iy, It, 1.0, &Q, iters - kw, &res);
    if (res_out) *res_out = res;
    return n;
}

/* The first warp of a level under the adaptive step: the first `window` iterations run
 * without the stopping test and rebalance c after every 10th (residuals of that iteration,
 * with the c it used); the remaining iterations run with c frozen, their stopping test counted
 * from the window's end.  *c carries the step in and out; *margin is lowered to the smallest
 * |log| distance of a test from its two thresholds. */
long long orc_inner_adapt(int H, int W, orc_state *st, const double *Ix, const double *Iy,
                          const double *It, double a_tilde, const orc_params *P, int iters, int window,
                          double *c, double *margin, double *res_out)
{
    size_t N = (size_t)H * (size_t)W;
    double nrows = (double)N * (P->beta != 0.0 ? 3.0 : 2.0);
    orc_params Q = *P;
    orc_state prev;
    memset(&prev, 0, sizeof(prev));
    double **yk[7] = {&prev.p1, &prev.p2, &prev.q11, &prev.q12, &prev.q21, &prev.q22, &prev.s};
    double *ys[7] = {st->p1, st->p2, st->q11, st->q12, st->q21, st->q22, st->s};
    for (int f = 0; f < 7; ++f) *yk[f] = orc_alloc(N);
    int kw = window < iters ? window : iters;
    double res = 0.0;
    for (int k = 0; k < kw; ++k) {
        int test = (k + 1) % 10 == 0;
        Q.c = *c;
        if (test)
            for (int f = 0; f < 7; ++f) memcpy(*yk[f], ys[f], N * sizeof(double));
        res = sqrt(orc_admm_step(H, W, st, Ix, Iy, It, a_tilde, &Q) / nrows);
        if (test) {
            double rn, dn;
            orc_adapt_residuals(H, W, &prev, st, Ix, Iy, a_tilde, *c, P, &rn, &dn);
            double m1 = fabs(log(rn / (10.0 * dn))), m2 = fabs(log(dn / (10.0 * rn)));
            if (m1 < *margin) *margin = m1;
            if (m2 < *margin) *margin = m2;
            *c = orc_adapt_rule(*c, rn, dn);
        }
    }
    for (int f = 0; f < 7; ++f) free(*yk[f]);
    Q.c = *c;
    long long n = kw;
    if (iters > kw) n += orc_inner(H, W, st, Ix, Iy, It, a_tilde, &Q, iters - kw, &res);
    if (res_out) *res_out = res;
    return n;
}

/* ------------------------------------------------------------------------------------- */
/* The whole schedule: pyramid, coarse-to-fine levels, warps, inner iterations.           */
/* Reading (Sec. 4 gives no details): state is zero at the coarsest level; at each finer   */
/* level (w, u, v) are upsampled (u, v scaled by the size ratio) and the dual variables    */
/* restart at zero (pDR: Xbar = X, ybar = 0); within a level all state carries over from   */
/* one warp to the next.  Output: (u, v, w) at level out_level, of size H_l x W_l.          */
/* ------------------------------------------------------------------------------------- */

int orc_solve(int H, int W, const double *I0, const double *I1, const orc_params *P,
              double *u_out, double *v_out, double *w_out, orc_stats *stats)
{
    int L = P->levels;
    if (H < 1 || W < 1 || L < 1 || L > 32 || P->out_level < 0 || P->out_level >= L) return 1;
    if (P->c_adapt_iters < 0 || P->c_adapt_iters % 10 != 0 || (P->c_adapt_iters > 0 && P->method == 3)) return 2;
    int Hs[32], Ws[32];
    double *P0[32], *P1[32];
    Hs[0] = H; Ws[0] = W;
    for (int l = 1; l < L; ++l) { Hs[l] = orc_level_size(Hs[l - 1], P->eta); Ws[l] = orc_level_size(Ws[l - 1], P->eta); }
    P0[0] = orc_alloc((size_t)H * W); P1[0] = orc_alloc((size_t)H * W);
    memcpy(P0[0], I0, sizeof(double) * (size_t)H * W);
    memcpy(P1[0], I1, sizeof(double) * (size_t)H * W);
    for (int l = 1; l < L; ++l) {
        size_t n = (size_t)Hs[l] * Ws[l];
        P0[l] = orc_alloc(n); P1[l] = orc_alloc(n);
        orc_downsample(Hs[l - 1], Ws[l - 1], P0[l - 1], Hs[l], Ws[l], P0[l], P->eta);
        orc_downsample(Hs[l - 1], Ws[l - 1], P1[l - 1], Hs[l], Ws[l], P1[l], P->eta);
    }
    size_t Nmax = (size_t)H * W;
    orc_state st;
    double **fields[13] = {&st.w, &st.u, &st.v, &st.p1, &st.p2, &st.q11, &st.q12, &st.q21, &st.q22, &st.s, &st.wb, &st.ub, &st.vb};
    for (int f = 0; f < 13; ++f) *fields[f] = orc_alloc(Nmax);
    double *cw = orc_alloc(Nmax), *cu = orc_alloc(Nmax), *cv = orc_alloc(Nmax);
    double *I1x = orc_alloc(Nmax), *I1y = orc_alloc(Nmax), *Ix = orc_alloc(Nmax), *Iy = orc_alloc(Nmax), *It = orc_alloc(Nmax);
    double *u0 = orc_alloc(Nmax), *v0 = orc_alloc(Nmax);
    long long total = 0;
    double res = 0.0, a_tilde = 1.0;
    double c_cur = P->c, theta = 1.0, margin = HUGE_VAL; /* the steps carry from level to level */
    orc_params Q = *P;

    for (int l = L - 1; l >= P->out_level; --l) {
        int h = Hs[l], w = Ws[l];
        size_t n = (size_t)h * w;
        if (l == L - 1) {
            for (int f = 0; f < 13; ++f) memset(*fields[f], 0, n * sizeof(double));
        } else {
            int hc = Hs[l + 1], wc = Ws[l + 1];
            size_t nc = (size_t)hc * wc;
            memcpy(cw, st.w, nc * sizeof(double)); memcpy(cu, st.u, nc * sizeof(double)); memcpy(cv, st.v, nc * sizeof(double));
            orc_upsample(hc, wc, cw, h, w, st.w, 1.0);
            orc_upsample(hc, wc, cu, h, w, st.u, (double)w / (double)wc);
            orc_upsample(hc, wc, cv, h, w, st.v, (double)h / (double)hc);
            for (int f = 3; f < 13; ++f) memset(*fields[f], 0, n * sizeof(double));
        }
        if (P->beta == 0.0) memset(st.w, 0, n * sizeof(double));
        if (P->method == 2 || P->method == 3) { /* pDR: Xbar = X; ALG1: the extrapolated point starts at X */
            memcpy(st.wb, st.w, n * sizeof(double)); memcpy(st.ub, st.u, n * sizeof(double)); memcpy(st.vb, st.v, n * sizeof(double));
        }
        orc_derivatives(h, w, P1[l], I1x, I1y);
        for (int wp = 0; wp < P->warps; ++wp) {
            memcpy(u0, st.u, n * sizeof(double));
            memcpy(v0, st.v, n * sizeof(double));
            double msmax = orc_warp_linearise(h, w, P0[l], P1[l], I1x, I1y, u0, v0, P->beta, Ix, Iy, It);
            a_tilde = P->a_tilde > 0.0 ? P->a_tilde : (msmax > 1e-12 ? msmax : 1e-12);
            if (P->c_adapt_iters > 0 && wp == 0 && P->method == 2) {
                total += orc_inner_adapt_pdr(h, w, &st, Ix, Iy, It, P, P->iters, P->c_adapt_iters, &theta, &margin,
                                             &res);
            } else if (P->c_adapt_iters > 0 && wp == 0) {
                total += orc_inner_adapt(h, w, &st, Ix, Iy, It, a_tilde, P, P->iters, P->c_adapt_iters, &c_cur,
                                         &margin, &res);
            } else {
                Q.c = c_cur;
                Q.sigma = P->sigma * theta;
                Q.tau = P->tau / theta;
                total += orc_inner(h, w, &st, Ix, Iy, It, a_tilde, &Q, P->iters, &res);
            }
        }
        if (l == P->out_level) {
            memcpy(u_out, st.u, n * sizeof(double));
            memcpy(v_out, st.v, n * sizeof(double));
            if (w_out) memcpy(w_out, st.w, n * sizeof(double));
            if (stats) {
                stats->iters_run = total;
                stats->residual = res;
                stats->energy = orc_energy(h, w, st.w, st.u, st.v, Ix, Iy, It, P->beta, P->lambda);
                stats->dual_value = P->method >= 2 ? NAN : orc_dual_value(n, It, st.s);
                stats->c_final = P->method == 2 ? P->sigma * theta : c_cur;
                stats->adapt_margin = margin;
            }
        }
    }
    for (int f = 0; f < 13; ++f) free(*fields[f]);
    free(cw); free(cu); free(cv); free(I1x); free(I1y); free(Ix); free(Iy); free(It); free(u0); free(v0);
    for (int l = 0; l < L; ++l) { free(P0[l]); free(P1[l]); }
    return 0;
}

/* Flat-argument wrappers for the ctypes loader (arrays of 13 state pointers). */
static void orc_state_from(orc_state *st, double **f)
{
    st->w = f[0]; st->u = f[1]; st->v = f[2]; st->p1 = f[3]; st->p2 = f[4]; st->q11 = f[5];
    st->q12 = f[6]; st->q21 = f[7]; st->q22 = f[8]; st->s = f[9]; st->wb = f[10]; st->ub = f[11]; st->vb = f[12];
}

double orc_admm_step_flat(int H, int W, double **fields, const double *Ix, const double *Iy,
                          const double *It, double a_tilde, const orc_params *P)
{
    orc_state st;
    orc_state_from(&st, fields);
    return orc_admm_step(H, W, &st, Ix, Iy, It, a_tilde, P);
}

double orc_pdr_step_flat(int H, int W, double **fields, const double *Ix, const double *Iy,
                         const double *It, const orc_params *P)
{
    orc_state st;
    orc_state_from(&st, fields);
    return orc_pdr_step(H, W, &st, Ix, Iy, It, P);
}

double orc_cp_step_flat(int H, int W, double **fields, const double *Ix, const double *Iy,
                        const double *It, const orc_params *P)
{
    orc_state st;
    orc_state_from(&st, fields);
    return orc_cp_step(H, W, &st, Ix, Iy, It, P);
}

long long orc_inner_flat(int H, int W, double **fields, const double *Ix, const double *Iy,
                         const double *It, double a_tilde, const orc_params *P, int iters, double *res_out)
{
    orc_state st;
    orc_state_from(&st, fields);
    return orc_inner(H, W, &st, Ix, Iy, It, a_tilde, P, iters, res_out);
}

double orc_adapt_residuals_flat(int H, int W, double **prev_fields, double **cur_fields, const double *Ix,
                                const double *Iy, double a_tilde, double c, const orc_params *P, double *r_norm,
                                double *d_norm)
{
    orc_state prev, cur;
    orc_state_from(&prev, prev_fields);
    orc_state_from(&cur, cur_fields);
    orc_adapt_residuals(H, W, &prev, &cur, Ix, Iy, a_tilde, c, P, r_norm, d_norm);
    return *r_norm;
}

long long orc_inner_adapt_flat(int H, int W, double **fields, const double *Ix, const double *Iy,
                               const double *It, double a_tilde, const orc_params *P, int iters, int window,
                               double *c, double *margin, double *res_out)
{
    orc_state st;
    orc_state_from(&st, fields);
    return orc_inner_adapt(H, W, &st, Ix, Iy, It, a_tilde, P, iters, window, c, margin, res_out);
}

double orc_pdr_adapt_residuals_flat(int H, int W, double **prev_fields, double **cur_fields, double sigma,
                                    double tau, const orc_params *P, double *rx, double *ry)
{
    orc_state prev, cur;
    orc_state_from(&prev, prev_fields);
    orc_state_from(&cur, cur_fields);
    orc_pdr_adapt_residuals(H, W, &prev, &cur, sigma, tau, P, rx, ry);
    return *rx;
}

long long orc_inner_adapt_pdr_flat(int H, int W, double **fields, const double *Ix, const double *Iy,
                                   const double *It, const orc_params *P, int iters, int window, double *theta,
                                   double *margin, double *res_out)
{
    orc_state st;
    orc_state_from(&st, fields);
    return orc_inner_adapt_pdr(H, W, &st, Ix, Iy, It, P, iters, window, theta, margin, res_out);
}
