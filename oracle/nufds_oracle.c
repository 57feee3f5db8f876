/*
 * FP64 reference ("oracle") for NU-FDS reconstruction of wide-angle CGHs.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU product path
 * neither links nor calls it, and this file shares no code, table or helper
 * with the CUDA sources.
 *
 * Plain, slow and direct: FP64 throughout, a naive recursive mixed-radix FFT,
 * the Gauss hypergeometric function from its series, a 2-D Newton solve for
 * the inverse of the frequency stretch, and a Gaussian-gridding type-2 NUFFT
 * (oversampling 2, half-width 14 cells, error ~1e-12 relative to sum|c|) to
 * evaluate trigonometric polynomials off the grid (or, for the paper-literal
 * variant, bilinear interpolation between their grid values).
 *
 * Paper: Kozacki et al., "Non-uniform Fourier Domain Stretching method for
 * ultra-wide-angle wave propagation".  Each function cites the equation it
 * follows.  Readings of ambiguous passages (sign conventions, grid spacing,
 * band rule, masking, normalisation) are listed in the repository's design
 * notes and summarised at each use below.
 *
 * Conventions: centred sample positions x_n = (n - N/2) * pitch, centred
 * frequencies f_k = (k - N/2)/(N pitch); forward transform kernel
 * e^{-2 pi i x f}; chirps e^{+i pi r^2/(lambda z)}.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Naive recursive mixed-radix FFT (decimation in time).                     */
/* X[k] = sum_n x[n] e^{sign * 2 pi i n k / n_total}, unnormalised.          */
/* ------------------------------------------------------------------------ */

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* tw[e] = e^{sign 2 pi i e / ntot}; a length-n sub-transform uses stride ntot/n. */
static void fft_rec(const cplx *x, int xstride, cplx *out, int n, const cplx *tw,
                    int ntot, cplx *scratch) {
    if (n == 1) {
        out[0] = x[0];
        return;
    }
    int p = smallest_factor(n);
    int m = n / p;
    int twstep = ntot / n;
    /* sub-transforms of the p decimated sequences, written contiguously */
    for (int j = 0; j < p; ++j)
        fft_rec(x + (size_t)j * xstride, xstride * p, scratch + (size_t)j * m, m, tw, ntot,
                out);
    /* combine: X[k + m q] = sum_j W_n^{j (k + m q)} Y_j[k] */
    for (int k = 0; k < m; ++k) {
        for (int q = 0; q < p; ++q) {
            int kk = k + m * q;
            cplx acc = 0;
            for (int j = 0; j < p; ++j) {
                long e = ((long)j * kk) % n;
                acc += tw[(size_t)e * twstep] * scratch[(size_t)j * m + k];
            }
            out[kk] = acc;
        }
    }
}

static cplx *twiddles(int n, int sign) {
    cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int e = 0; e < n; ++e) {
        double a = 2.0 * OR_PI * (double)e / (double)n;
        tw[e] = cos(a) + sign * I * sin(a);
    }
    return tw;
}

/* In-place 1-D FFT of interleaved complex data; sign = -1 forward, +1 inverse. */
void or_fft(double *re_im, int n, int sign) {
    cplx *x = (cplx *)re_im;
    cplx *tw = twiddles(n, sign);
    cplx *in = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *scratch = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    memcpy(in, x, sizeof(cplx) * (size_t)n);
    fft_rec(in, 1, x, n, tw, n, scratch);
    free(scratch);
    free(in);
    free(tw);
}

/* 2-D FFT (rows of length nx, ny rows) in place, along both axes. */
static void fft2(cplx *a, int nx, int ny, int sign) {
    cplx *twx = twiddles(nx, sign), *twy = twiddles(ny, sign);
#pragma omp parallel
    {
        int mx = nx > ny ? nx : ny;
        cplx *in = (cplx *)malloc(sizeof(cplx) * (size_t)mx);
        cplx *scr = (cplx *)malloc(sizeof(cplx) * (size_t)mx);
#pragma omp for schedule(dynamic, 4)
        for (int r = 0; r < ny; ++r) {
            memcpy(in, a + (size_t)r * nx, sizeof(cplx) * (size_t)nx);
            fft_rec(in, 1, a + (size_t)r * nx, nx, twx, nx, scr);
        }
        cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)ny);
#pragma omp for schedule(dynamic, 4)
        for (int c = 0; c < nx; ++c) {
            for (int r = 0; r < ny; ++r) in[r] = a[(size_t)r * nx + c];
            fft_rec(in, 1, col, ny, twy, ny, scr);
            for (int r = 0; r < ny; ++r) a[(size_t)r * nx + c] = col[r];
        }
        free(col);
        free(scr);
        free(in);
    }
    free(twx);
    free(twy);
}

/*
 * Centred 2-D DFT of an ny x nx array (Section 4, step two, "FT of the
 * hologram"; sampling of Eq. 2):
 *   Ht[ky][kx] = sum_n a[ny][nx] e^{-2 pi i ((nx-Nx/2)(kx-Nx/2)/Nx + (ny-Ny/2)(ky-Ny/2)/Ny)}
 * computed by shifting the index origin (roll by N/2 before and after).
 * sign = +1 gives the centred inverse kernel (unnormalised).
 */
static void centred_dft2(cplx *a, int nx, int ny, int sign) {
    size_t total = (size_t)nx * ny;
    cplx *t = (cplx *)malloc(sizeof(cplx) * total);
    for (int r = 0; r < ny; ++r)
        for (int c = 0; c < nx; ++c)
            t[(size_t)((r + ny / 2) % ny) * nx + (c + nx / 2) % nx] = a[(size_t)r * nx + c];
    fft2(t, nx, ny, sign);
    for (int r = 0; r < ny; ++r)
        for (int c = 0; c < nx; ++c)
            a[(size_t)r * nx + c] = t[(size_t)((r + ny / 2) % ny) * nx + (c + nx / 2) % nx];
    free(t);
}

void or_centred_dft2(double *re_im, int nx, int ny, int sign) {
    centred_dft2((cplx *)re_im, nx, ny, sign);
}

/* ------------------------------------------------------------------------ */
/* Gauss hypergeometric 2F1(1/2, 3/4; 3/2; w), the function of Eq. 16.       */
/* ------------------------------------------------------------------------ */

/* plain power series sum_n (a)_n (b)_n / ((c)_n n!) w^n, |w| <= 1/2 */
static double f21_series(double a, double b, double c, double w) {
    double term = 1.0, sum = 1.0;
    for (int n = 0; n < 400; ++n) {
        term *= (a + n) * (b + n) / ((c + n) * (n + 1.0)) * w;
        sum += term;
        if (fabs(term) <= 1e-18 * fabs(sum)) break;
    }
    return sum;
}

/*
 * F(w) = 2F1(1/2, 3/4; 3/2; w) for 0 <= w <= 1.  Power series for w <= 1/2;
 * for w > 1/2 the connection formula of Abramowitz & Stegun 15.3.6
 * (c - a - b = 1/4 is not an integer) maps it to series in 1 - w.
 * Returns NaN for w > 1 (evanescent: no real value of Eq. 16).
 */
double or_hyp2f1(double w) {
    const double a = 0.5, b = 0.75, c = 1.5;
    if (w < 0.0 || w > 1.0) return NAN;
    if (w <= 0.5) return f21_series(a, b, c, w);
    double v = 1.0 - w;
    double A = tgamma(c) * tgamma(c - a - b) / (tgamma(c - a) * tgamma(c - b));
    double B = tgamma(c) * tgamma(a + b - c) / (tgamma(a) * tgamma(b));
    double t1 = A * f21_series(a, b, a + b - c + 1.0, v);
    double t2 = (v > 0.0) ? B * pow(v, c - a - b) * f21_series(c - a, c - b, c - a - b + 1.0, v)
                          : 0.0;
    return t1 + t2;
}

/* ------------------------------------------------------------------------ */
/* The paper's polynomial surrogate for 2F1 (Section 4, initialisation step  */
/* 1): a degree-8 polynomial fitted to 51 frequencies uniformly spread over  */
/* the hologram's band.  Reading: samples at f_y = 0, f_x = -1/(2 pitch) ..  */
/* 1/(2 pitch), variable s = lambda f_x (so w = s^2), least squares; applied */
/* in Eq. 16 as F(w) ~ P(lambda f_x / a_y).  Off by default.                 */
/* ------------------------------------------------------------------------ */
#define OR_POLY_DEG 8
#define OR_POLY_SAMPLES 51
static int g_poly = 0;
static double g_pc[OR_POLY_DEG + 1];

/* least squares by Householder QR of the 51 x 9 Vandermonde system */
static void poly_fit(const double *x, const double *y, int m, int n, double *c) {
    double A[OR_POLY_SAMPLES][OR_POLY_DEG + 1], b[OR_POLY_SAMPLES];
    for (int i = 0; i < m; ++i) {
        double t = 1.0;
        for (int j = 0; j < n; ++j, t *= x[i]) A[i][j] = t;
        b[i] = y[i];
    }
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += A[i][k] * A[i][k];
        nrm = sqrt(nrm);
        double alpha = A[k][k] > 0 ? -nrm : nrm;
        double v[OR_POLY_SAMPLES];
        for (int i = 0; i < m; ++i) v[i] = i < k ? 0.0 : A[i][k];
        v[k] -= alpha;
        double vv = 0.0;
        for (int i = k; i < m; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        for (int j = k; j < n; ++j) {
            double d = 0.0;
            for (int i = k; i < m; ++i) d += v[i] * A[i][j];
            for (int i = k; i < m; ++i) A[i][j] -= 2.0 * d / vv * v[i];
        }
        double d = 0.0;
        for (int i = k; i < m; ++i) d += v[i] * b[i];
        for (int i = k; i < m; ++i) b[i] -= 2.0 * d / vv * v[i];
    }
    for (int j = n - 1; j >= 0; --j) { /* back substitution, R c = Q^T b */
        double t = b[j];
        for (int k = j + 1; k < n; ++k) t -= A[j][k] * c[k];
        c[j] = t / A[j][j];
    }
}

/* enable (1) or disable (0) the polynomial for a geometry; coefficients out (9) */
void or_set_paper_poly(int enable, double lam, double pitch, double *coef_out) {
    g_poly = 0;
    if (!enable) return;
    double x[OR_POLY_SAMPLES], y[OR_POLY_SAMPLES];
    for (int i = 0; i < OR_POLY_SAMPLES; ++i) {
        double f = (-0.5 + (double)i / (OR_POLY_SAMPLES - 1)) / pitch;
        x[i] = lam * f;
        y[i] = or_hyp2f1(x[i] * x[i]);
    }
    poly_fit(x, y, OR_POLY_SAMPLES, OR_POLY_DEG + 1, g_pc);
    if (coef_out)
        for (int k = 0; k <= OR_POLY_DEG; ++k) coef_out[k] = g_pc[k];
    g_poly = 1;
}

static double poly_val(double s) {
    double p = g_pc[OR_POLY_DEG];
    for (int k = OR_POLY_DEG - 1; k >= 0; --k) p = p * s + g_pc[k];
    return p;
}

static double poly_der(double s) {
    double p = OR_POLY_DEG * g_pc[OR_POLY_DEG];
    for (int k = OR_POLY_DEG - 1; k >= 1; --k) p = p * s + k * g_pc[k];
    return p;
}

/* F(w) of Eq. 16, w = s^2 (s carries the frequency's sign): exact or the surrogate */
static double F_of(double w, double s) { return g_poly ? poly_val(s) : or_hyp2f1(w); }

/* ------------------------------------------------------------------------ */
/* Magnification and the non-uniform stretch (Eqs. 9, 10, 15, 16).          */
/* ------------------------------------------------------------------------ */

/* Eq. 16: m_x = (1 - l^2 fy^2)^(-1/4) F(l^2 fx^2 / (1 - l^2 fy^2)); m_y swaps x,y. */
void or_mag(double lam, double fx, double fy, double *mx, double *my) {
    double ax = 1.0 - lam * lam * fx * fx, ay = 1.0 - lam * lam * fy * fy;
    *mx = pow(ay, -0.25) * F_of(lam * lam * fx * fx / ay, g_poly ? lam * fx / sqrt(ay) : 0.0);
    *my = pow(ax, -0.25) * F_of(lam * lam * fy * fy / ax, g_poly ? lam * fy / sqrt(ax) : 0.0);
}

/* Eqs. 9-10: f' = (fx m_x, fy m_y). */
void or_forward(double lam, double fx, double fy, double *fpx, double *fpy) {
    double mx, my;
    or_mag(lam, fx, fy, &mx, &my);
    *fpx = fx * mx;
    *fpy = fy * my;
}

/* F'(w): from Eq. 15, d/ds [s F(s^2)] = (1 - s^2)^(-3/4), i.e.
 * F + 2 w F' = (1 - w)^(-3/4); the series derivative near w = 0. */
static double hyp2f1_deriv(double w) {
    if (w < 0.05) {
        double term = 1.0, sum = 0.0;   /* d/dw sum t_n w^n = sum n t_n w^(n-1) */
        double tn = 1.0;
        for (int n = 1; n < 200; ++n) {
            tn *= (0.5 + n - 1) * (0.75 + n - 1) / ((1.5 + n - 1) * n);
            term = n * tn * pow(w, n - 1);
            sum += term;
            if (fabs(term) <= 1e-18 * fabs(sum)) break;
        }
        return sum;
    }
    return (pow(1.0 - w, -0.75) - or_hyp2f1(w)) / (2.0 * w);
}

/* Jacobian of f' = Phi(f) w.r.t. f, dimensionless (u = l fx, v = l fy). */
static void jacobian(double u, double v, double J[2][2]) {
    double ay = 1.0 - v * v, ax = 1.0 - u * u;
    if (g_poly) {
        /* d/du [u ay^(-1/4) P(s)] = ay^(-1/4) (P + s P'), s = u / sqrt(ay);
         * d/dv [u ay^(-1/4) P(s)] = u v ay^(-5/4) (P / 2 + s P') */
        double sx = u / sqrt(ay), sy = v / sqrt(ax);
        J[0][0] = pow(ay, -0.25) * (poly_val(sx) + sx * poly_der(sx));
        J[1][1] = pow(ax, -0.25) * (poly_val(sy) + sy * poly_der(sy));
        J[0][1] = u * v * pow(ay, -1.25) * (0.5 * poly_val(sx) + sx * poly_der(sx));
        J[1][0] = u * v * pow(ax, -1.25) * (0.5 * poly_val(sy) + sy * poly_der(sy));
        return;
    }
    double wx = u * u / ay, wy = v * v / ax;
    double r = 1.0 - u * u - v * v;
    /* diagonal: Eq. 15 */
    J[0][0] = sqrt(ay) * pow(r, -0.75);
    J[1][1] = sqrt(ax) * pow(r, -0.75);
    /* off-diagonal: d/dv [u ay^(-1/4) F(u^2/ay)] */
    J[0][1] = u * (0.5 * v * pow(ay, -1.25) * or_hyp2f1(wx) +
                   pow(ay, -0.25) * hyp2f1_deriv(wx) * 2.0 * u * u * v / (ay * ay));
    J[1][0] = v * (0.5 * u * pow(ax, -1.25) * or_hyp2f1(wy) +
                   pow(ax, -0.25) * hyp2f1_deriv(wy) * 2.0 * v * v * u / (ax * ax));
}

static void phi_uv(double u, double v, double *up, double *vp) {
    /* Eqs. 9, 10, 16 with u = lambda fx, v = lambda fy */
    double ay = 1.0 - v * v, ax = 1.0 - u * u;
    *up = u * pow(ay, -0.25) * F_of(u * u / ay, g_poly ? u / sqrt(ay) : 0.0);
    *vp = v * pow(ax, -0.25) * F_of(v * v / ax, g_poly ? v / sqrt(ax) : 0.0);
}

/*
 * Inverse of the stretch (Section 4, step two read as a pull-back): find f
 * with f m(f) = f' by damped 2-D Newton on u = lambda f.  Returns 1 and f on
 * success, 0 if f' has no pre-image in the propagating region
 * (lambda^2 |f|^2 < 1).  Converged when |du| <= 1e-13 lambda / pitch... in
 * dimensionless units: |du| <= tol_u.
 */
static int pullback_uv(double up, double vp, double tol_u, double *uo, double *vo) {
    /* start inside the disc, shrunk towards the origin (m >= 1 => |u| <= |u'|) */
    double u = up, v = vp;
    double rr = u * u + v * v;
    if (rr > 0.81) {
        double s = 0.9 / sqrt(rr);
        u *= s;
        v *= s;
    }
    double fu, fv;
    phi_uv(u, v, &fu, &fv);
    double res = hypot(fu - up, fv - vp);
    for (int it = 0; it < 200; ++it) {
        double J[2][2];
        jacobian(u, v, J);
        double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        double ru = up - fu, rv = vp - fv;
        double du = (J[1][1] * ru - J[0][1] * rv) / det;
        double dv = (-J[1][0] * ru + J[0][0] * rv) / det;
        double lam = 1.0;
        int accepted = 0;
        for (int h = 0; h < 60; ++h) {
            double un = u + lam * du, vn = v + lam * dv;
            if (un * un + vn * vn < 1.0) {
                double gu, gv;
                phi_uv(un, vn, &gu, &gv);
                double rn = hypot(gu - up, gv - vp);
                if (rn < res || rn == 0.0 || (lam * hypot(du, dv) <= tol_u)) {
                    u = un;
                    v = vn;
                    fu = gu;
                    fv = gv;
                    res = rn;
                    accepted = 1;
                    break;
                }
            }
            lam *= 0.5;
        }
        if (!accepted) return 0;
        if (lam * hypot(du, dv) <= tol_u) {
            *uo = u;
            *vo = v;
            /* accept only a true root (residual at rounding level) */
            return res <= 1e-12 * (1.0 + hypot(up, vp));
        }
    }
    return 0;
}

/* Pull-back in frequency units (1/m).  Returns 1 if a pre-image exists. */
int or_pullback(double lam, double pitch, double fpx, double fpy, double *fx, double *fy) {
    double u, v;
    int ok = pullback_uv(lam * fpx, lam * fpy, 1e-13 * lam / pitch, &u, &v);
    *fx = ok ? u / lam : NAN;
    *fy = ok ? v / lam : NAN;
    return ok;
}

/* ------------------------------------------------------------------------ */
/* Output coordinate map (Eqs. 17, 18) and its 4-step inverse iteration.     */
/* ------------------------------------------------------------------------ */

/* Eqs. 17-18: x_o' = z lambda f_x0 m_x(f_0), f_0 = (x_o, y_o)/(lambda R_0). */
void or_output_map(double lam, double z, double xo, double yo, double *xop, double *yop) {
    double R0 = sqrt(xo * xo + yo * yo + z * z);
    double fx0 = xo / (lam * R0), fy0 = yo / (lam * R0);
    double fpx, fpy;
    or_forward(lam, fx0, fy0, &fpx, &fpy);
    *xop = z * lam * fpx;
    *yop = z * lam * fpy;
}

/*
 * The paper's fixed-point iteration for the inverse output map (the second
 * equation numbered (18) in Section 4): x_o(k) = x_o' R(k-1) / (z m_x(f_0(k-1))),
 * with x_o(1) = x_o'.  'steps' iterations; returns x_o(steps).
 */
void or_output_map_iterative_inverse(double lam, double z, double xop, double yop, int steps,
                                     double *xo, double *yo) {
    double x = xop, y = yop;
    for (int k = 2; k <= steps; ++k) {
        double R = sqrt(x * x + y * y + z * z);
        double mx, my;
        or_mag(lam, x / (lam * R), y / (lam * R), &mx, &my);
        double xn = xop * R / (z * mx), yn = yop * R / (z * my);
        x = xn;
        y = yn;
    }
    *xo = x;
    *yo = y;
}

/* Phase-space tools at the hologram centre for a point (xo, yo, zo), Eqs. 4-5:
 * f_xl(0,0) = xo/(lambda R), c_xl(0,0) = -(yo^2 + zo^2)/R^3. */
void or_ps_tools(double lam, double xo, double yo, double zo, double *fxl, double *cxl) {
    double R = sqrt(xo * xo + yo * yo + zo * zo);
    *fxl = -(0.0 - xo) / (lam * R);
    *cxl = -(yo * yo + zo * zo) / (R * R * R);
}

/*
 * Wavefront error of one object point along the hologram's central row
 * (Section 2, Figs. 2c/2f; Section 4, Fig. 5), in waves.
 *
 * Reading (the paper gives the idea, not the formula): the error is the
 * phase of the point's spectrum minus the phase of the paraxial spectrum the
 * Fresnel transform focuses, taken where the spectrum carries the point.
 *   - The hologram e^{-ikR_o} has, by stationary phase, the spectrum phase
 *     psi(f) = -(f . x_o + z_o sqrt(1/lambda^2 - |f|^2)) cycles, sampled at
 *     the local frequency f(x) of Eq. 4 of each hologram pixel x.
 *   - The Fresnel transform at distance z_r focuses the paraxial spectrum
 *     psi_p(q) = -(q . x_r + z_r (1/lambda - lambda |q|^2 / 2)).
 *   - NU-FDS (method 0) moves f to q = f' of Eqs. 9-10 and focuses at
 *     z_r = z_o, x_r = x_o' of Eq. 17; the plain Fresnel transform (method 1)
 *     keeps q = f and focuses at the given z_r, x_r = z_r lambda f_l(0,0)
 *     (z_r <= 0: z_r = z_o, the paper's wrong-coordinate reconstruction).
 *   - W(x) = psi(f(x)) - psi_p(q(x)) - [the same at the hologram centre].
 * x[j] = (j - (ns-1)/2) (n pitch)/ns across the aperture; samples whose local
 * frequency leaves the band (|f| >= 1/(2 pitch) on an axis) or is evanescent
 * get W = NaN.  Returns max |W| over the rest (0 when none).
 */
static double wfe_psi(double lam, double fx, double fy, double xo, double yo, double zo) {
    return -(fx * xo + fy * yo + zo * sqrt(1.0 / (lam * lam) - fx * fx - fy * fy));
}

static double wfe_psi_p(double lam, double qx, double qy, double xr, double yr, double zr) {
    return -(qx * xr + qy * yr + zr * (1.0 / lam - 0.5 * lam * (qx * qx + qy * qy)));
}

/* W before the piston is removed, at local frequency (fx, fy) */
static double wfe_raw(double lam, double fx, double fy, double xo, double yo, double zo, int method,
                      double zr, double xr, double yr) {
    double qx = fx, qy = fy;
    if (method == 0) or_forward(lam, fx, fy, &qx, &qy);
    return wfe_psi(lam, fx, fy, xo, yo, zo) - wfe_psi_p(lam, qx, qy, xr, yr, zr);
}

double or_wavefront_error(double lam, double pitch, int n, double xo, double yo, double zo,
                          int method, double zr, int ns, double *x, double *w) {
    double R0 = sqrt(xo * xo + yo * yo + zo * zo);
    double f0x = xo / (lam * R0), f0y = yo / (lam * R0); /* Eq. 4 at the centre */
    double xr, yr;
    if (method == 0) {
        zr = zo;
        or_output_map(lam, zo, xo, yo, &xr, &yr); /* Eq. 17 */
    } else {
        if (zr <= 0.0) zr = zo;
        xr = zr * lam * f0x;
        yr = zr * lam * f0y;
    }
    double w0 = wfe_raw(lam, f0x, f0y, xo, yo, zo, method, zr, xr, yr);
    double fb = 0.5 / pitch, mx = 0.0;
    for (int j = 0; j < ns; ++j) {
        double xh = (j - 0.5 * (ns - 1)) * (n * pitch) / ns;
        double R = sqrt((xh - xo) * (xh - xo) + yo * yo + zo * zo);
        double fx = -(xh - xo) / (lam * R), fy = yo / (lam * R); /* Eq. 4, y = 0 */
        double v = NAN;
        if (fabs(fx) < fb && fabs(fy) < fb && lam * lam * (fx * fx + fy * fy) < 1.0) {
            v = wfe_raw(lam, fx, fy, xo, yo, zo, method, zr, xr, yr) - w0;
            if (fabs(v) > mx) mx = fabs(v);
        }
        if (x) x[j] = xh;
        if (w) w[j] = v;
    }
    return mx;
}

/* ------------------------------------------------------------------------ */
/* View planning (Eq. 1, Eq. 17, Section 4 output-grid choice).              */
/* ------------------------------------------------------------------------ */

/* smallest 2^a 3^b 5^c >= n with a >= 6, b <= 2, c <= 1 */
int64_t or_nice(int64_t n) {
    int64_t best = -1;
    for (int b = 0; b <= 2; ++b)
        for (int c = 0; c <= 1; ++c) {
            int64_t base = (b == 0 ? 1 : (b == 1 ? 3 : 9)) * (c ? 5 : 1);
            int64_t v = 64 * base;
            while (v < n) v *= 2;
            if (best < 0 || v < best) best = v;
        }
    return best;
}

/*
 * Plan of one view.  In: lambda, pitch, Nx, Ny, z, view centre (cx, cy),
 * view size (w, h; 0,0 = full view of Eq. 1), output pixels (ox, oy; 0,0 = N).
 * stretch = 0 plans the plain Fresnel transform (x' = x_o).
 * Out (int64 iout[8]): ox, oy, k_lo_x, k_hi_x, k_lo_y, k_hi_y, Np_x, Np_y;
 *     (double dout[4]): pitch_out_x, pitch_out_y, window_w, window_h.
 * Band in stretched-lattice units (spacing 1/(N pitch)): the Eq. 17 image of
 * every boundary pixel centre, floored/ceiled.  FFT size: nice(max(band
 * width, ceil((N pitch)^2/(lambda z)))).  Band centre k_c = floor((lo+hi)/2).
 * Returns 0, or -1 on invalid input.
 */
int or_plan_view_ex(double lam, double pitch, int nx, int ny, double z, double cx, double cy,
                    double w, double h, int ox, int oy, int stretch, int64_t *iout,
                    double *dout) {
    if (!(lam > 0 && pitch > 0 && lam < 2.0 * pitch && z > 0 && nx > 0 && ny > 0)) return -1;
    double st = lam / (2.0 * pitch);
    double B = 2.0 * z * st / sqrt(1.0 - st * st); /* Eq. 1 */
    if (w <= 0 || h <= 0) {
        w = B;
        h = B;
    }
    if (ox <= 0 || oy <= 0) {
        ox = nx;
        oy = ny;
    }
    double px = w / ox, py = h / oy;
    double kmin[2] = {1e300, 1e300}, kmax[2] = {-1e300, -1e300};
    int64_t nb = 2LL * ox + 2LL * oy;
    for (int64_t t = 0; t < nb; ++t) {
        int i, j;
        if (t < ox) { i = (int)t; j = 0; }
        else if (t < 2 * ox) { i = (int)(t - ox); j = oy - 1; }
        else if (t < 2 * ox + oy) { i = 0; j = (int)(t - 2 * ox); }
        else { i = ox - 1; j = (int)(t - 2 * ox - oy); }
        double xo = cx + (i - 0.5 * ox) * px, yo = cy + (j - 0.5 * oy) * py;
        double xp = xo, yp = yo;
        if (stretch) or_output_map(lam, z, xo, yo, &xp, &yp);
        double kx = xp * nx * pitch / (lam * z), ky = yp * ny * pitch / (lam * z);
        if (kx < kmin[0]) kmin[0] = kx;
        if (kx > kmax[0]) kmax[0] = kx;
        if (ky < kmin[1]) kmin[1] = ky;
        if (ky > kmax[1]) kmax[1] = ky;
    }
    int64_t klo_x = (int64_t)floor(kmin[0]), khi_x = (int64_t)ceil(kmax[0]);
    int64_t klo_y = (int64_t)floor(kmin[1]), khi_y = (int64_t)ceil(kmax[1]);
    double chx = ceil((nx * pitch) * (nx * pitch) / (lam * z));
    double chy = ceil((ny * pitch) * (ny * pitch) / (lam * z));
    int64_t wx = khi_x - klo_x + 1, wy = khi_y - klo_y + 1;
    iout[0] = ox;
    iout[1] = oy;
    iout[2] = klo_x;
    iout[3] = khi_x;
    iout[4] = klo_y;
    iout[5] = khi_y;
    iout[6] = or_nice(wx > (int64_t)chx ? wx : (int64_t)chx);
    iout[7] = or_nice(wy > (int64_t)chy ? wy : (int64_t)chy);
    dout[0] = px;
    dout[1] = py;
    dout[2] = w;
    dout[3] = h;
    return 0;
}

/* The view plan of the NU-FDS method (band from Eq. 17). */
int or_plan_view(double lam, double pitch, int nx, int ny, double z, double cx, double cy,
                 double w, double h, int ox, int oy, int64_t *iout, double *dout) {
    return or_plan_view_ex(lam, pitch, nx, ny, z, cx, cy, w, h, ox, oy, 1, iout, dout);
}

/* ------------------------------------------------------------------------ */
/* Trigonometric-polynomial evaluation off the grid.                         */
/*   F(tx, ty) = sum_{n} c[ny][nx] e^{-2 pi i ((nx - Nx/2) tx / Nx + (ny - Ny/2) ty / Ny)} */
/* ------------------------------------------------------------------------ */

/* Direct sum (O(N^2) per target), separable phasors.  The plain definition. */
void or_dtft2_direct(const double *c_re_im, int nx, int ny, const double *tx, const double *ty,
                     int64_t nt, double *out_re_im) {
    const cplx *c = (const cplx *)c_re_im;
    cplx *out = (cplx *)out_re_im;
#pragma omp parallel
    {
        cplx *ex = (cplx *)malloc(sizeof(cplx) * (size_t)nx);
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < nt; ++t) {
            for (int n = 0; n < nx; ++n) {
                double a = -2.0 * OR_PI * (n - nx / 2) * tx[t] / nx;
                ex[n] = cos(a) + I * sin(a);
            }
            cplx acc = 0;
            for (int m = 0; m < ny; ++m) {
                double a = -2.0 * OR_PI * (m - ny / 2) * ty[t] / ny;
                cplx ey = cos(a) + I * sin(a);
                cplx row = 0;
                const cplx *cr = c + (size_t)m * nx;
                for (int n = 0; n < nx; ++n) row += cr[n] * ex[n];
                acc += ey * row;
            }
            out[t] = acc;
        }
        free(ex);
    }
}

/*
 * Same sum by Gaussian gridding (type-2 NUFFT): deapodise c by the Gaussian's
 * Fourier transform, zero-pad to 2N per axis, FFT, and interpolate with the
 * Gaussian exp(-s^2/(2 a^2)), |s| <= 14 fine cells, a^2 = 14/(pi sqrt 2).
 * Aliasing and truncation are both ~ exp(-pi*14/sqrt2) ~ 3e-14 (times the
 * deapodisation range ~50).
 */
#define GG_HALF 14
typedef struct {
    int nx, ny, mx, my;
    double a2;
    cplx *grid; /* my x mx, unshifted FFT output A_q */
} gg_plan;

static double gauss_ft(double a2, double x, int m) {
    /* int exp(-s^2/(2a^2)) e^{2 pi i x s / m} ds over the real line */
    return sqrt(2.0 * OR_PI * a2) * exp(-2.0 * OR_PI * OR_PI * a2 * x * x / ((double)m * m));
}

static void gg_prepare(gg_plan *p, const cplx *c, int nx, int ny) {
    p->nx = nx;
    p->ny = ny;
    p->mx = 2 * nx;
    p->my = 2 * ny;
    p->a2 = GG_HALF / (OR_PI * sqrt(2.0));
    size_t tot = (size_t)p->mx * p->my;
    p->grid = (cplx *)calloc(tot, sizeof(cplx));
    double *dx = (double *)malloc(sizeof(double) * nx), *dy = (double *)malloc(sizeof(double) * ny);
    for (int n = 0; n < nx; ++n) dx[n] = 1.0 / gauss_ft(p->a2, n - nx / 2, p->mx);
    for (int n = 0; n < ny; ++n) dy[n] = 1.0 / gauss_ft(p->a2, n - ny / 2, p->my);
    for (int m = 0; m < ny; ++m) {
        int qy = ((m - ny / 2) % p->my + p->my) % p->my;
        for (int n = 0; n < nx; ++n) {
            int qx = ((n - nx / 2) % p->mx + p->mx) % p->mx;
            p->grid[(size_t)qy * p->mx + qx] = c[(size_t)m * nx + n] * dx[n] * dy[m];
        }
    }
    free(dx);
    free(dy);
    fft2(p->grid, p->mx, p->my, -1);
}

static cplx gg_eval(const gg_plan *p, double tx, double ty) {
    /* fine coordinates s = 2 t; F ~ sum_q A_q psi(s - q), q wrapped mod M */
    double sx = 2.0 * tx, sy = 2.0 * ty;
    long qx0 = (long)floor(sx) - GG_HALF + 1, qy0 = (long)floor(sy) - GG_HALF + 1;
    double wx[2 * GG_HALF], wy[2 * GG_HALF];
    for (int i = 0; i < 2 * GG_HALF; ++i) {
        double d = sx - (double)(qx0 + i);
        wx[i] = exp(-d * d / (2.0 * p->a2));
        d = sy - (double)(qy0 + i);
        wy[i] = exp(-d * d / (2.0 * p->a2));
    }
    cplx acc = 0;
    for (int j = 0; j < 2 * GG_HALF; ++j) {
        long qy = ((qy0 + j) % p->my + p->my) % p->my;
        const cplx *row = p->grid + (size_t)qy * p->mx;
        cplx racc = 0;
        for (int i = 0; i < 2 * GG_HALF; ++i) {
            long qx = ((qx0 + i) % p->mx + p->mx) % p->mx;
            racc += wx[i] * row[qx];
        }
        acc += wy[j] * racc;
    }
    return acc;
}

void or_nufft2(const double *c_re_im, int nx, int ny, const double *tx, const double *ty,
               int64_t nt, double *out_re_im) {
    gg_plan p;
    gg_prepare(&p, (const cplx *)c_re_im, nx, ny);
    cplx *out = (cplx *)out_re_im;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) out[t] = gg_eval(&p, tx[t], ty[t]);
    free(p.grid);
}

/*
 * Paper-literal resampling variant (Section 4, steps two and five name an
 * interpolation without its kernel; read as linear, separable in x and y):
 * the trigonometric polynomial F above is taken on its integer grid only --
 * the centred DFT -- and interpolated bilinearly between the four grid
 * points around (tx, ty), periodically like the DFT.  Exact at grid points.
 */
static int64_t pmod(int64_t a, int64_t m) { return ((a % m) + m) % m; }

void or_lerp2(const double *c_re_im, int nx, int ny, const double *tx, const double *ty,
              int64_t nt, double *out_re_im) {
    size_t total = (size_t)nx * ny;
    cplx *g = (cplx *)malloc(sizeof(cplx) * total);
    memcpy(g, c_re_im, sizeof(cplx) * total);
    centred_dft2(g, nx, ny, -1); /* g[ky][kx] = F(kx - nx/2, ky - ny/2) */
    cplx *out = (cplx *)out_re_im;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) {
        double x0 = floor(tx[t]), y0 = floor(ty[t]);
        double ax = tx[t] - x0, ay = ty[t] - y0;
        cplx v[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                int64_t kx = pmod((int64_t)x0 + b + nx / 2, nx);
                int64_t ky = pmod((int64_t)y0 + a + ny / 2, ny);
                v[a][b] = g[(size_t)ky * nx + kx];
            }
        out[t] = (1 - ay) * ((1 - ax) * v[0][0] + ax * v[0][1]) +
                 ay * ((1 - ax) * v[1][0] + ax * v[1][1]);
    }
    free(g);
}

static int g_linear = 0;

/* Select the resampling of steps two and five: 0 ideal (NUFFT), 1 bilinear. */
void or_set_paper_linear(int enable) { g_linear = enable != 0; }

static void off_grid(const double *c, int nx, int ny, const double *tx, const double *ty,
                     int64_t nt, double *out) {
    if (g_linear) or_lerp2(c, nx, ny, tx, ty, nt, out);
    else or_nufft2(c, nx, ny, tx, ty, nt, out);
}

/* ------------------------------------------------------------------------ */
/* The NU-FDS reconstruction (Section 4, Fig. 3: steps 2, 3 and 5).          */
/* ------------------------------------------------------------------------ */

/*
 * holo: ny x nx complex64 (interleaved float), as the GPU receives it.
 * View as in or_plan_view.  stretch = 0 skips the non-uniform stretch and
 * the output remap (plain FrT of Eq. 2 at z on the same grid; a comparison
 * mode, Fig. 10b).  Outputs (oy x ox): field (interleaved complex128, may be
 * NULL) and intensity (float64, may be NULL).  threads <= 0: OpenMP default.
 * Returns 0 or -1.
 */
/* One view of the hologram H (FP64, ny x nx); gH, if not NULL, is H's
 * gridding plan shared by several views (the ideal resampling only). */
static int recon_view(double lam, double pitch, int nx, int ny, const cplx *H, const gg_plan *gH,
                      double z, double cx, double cy, double w, double h, int ox_in, int oy_in,
                      int stretch, double *field_out, double *intensity_out) {
    int64_t iv[8];
    double dv[4];
    if (or_plan_view_ex(lam, pitch, nx, ny, z, cx, cy, w, h, ox_in, oy_in, stretch, iv, dv))
        return -1;
    const int ox = (int)iv[0], oy = (int)iv[1];
    const int64_t klo_x = iv[2], khi_x = iv[3], klo_y = iv[4], khi_y = iv[5];
    const int npx = (int)iv[6], npy = (int)iv[7];
    const int64_t kcx = (int64_t)floor(0.5 * (double)(klo_x + khi_x));
    const int64_t kcy = (int64_t)floor(0.5 * (double)(klo_y + khi_y));
    const double px = dv[0], py = dv[1];
    const double dfx = 1.0 / (nx * pitch), dfy = 1.0 / (ny * pitch); /* stretched lattice */

    /* Step two: S(f'_k) = DTFT of H at the pulled-back f(f'_k); zero outside
     * the band, where no pre-image exists, or outside |f| <= 1/(2 pitch). */
    size_t nS = (size_t)npx * npy;
    double *tx = (double *)malloc(sizeof(double) * nS), *ty = (double *)malloc(sizeof(double) * nS);
    unsigned char *keep = (unsigned char *)calloc(nS, 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int jy = 0; jy < npy; ++jy) {
        int64_t ky = kcy + jy - npy / 2;
        for (int jx = 0; jx < npx; ++jx) {
            int64_t kx = kcx + jx - npx / 2;
            size_t s = (size_t)jy * npx + jx;
            tx[s] = 0.0;
            ty[s] = 0.0;
            if (kx < klo_x || kx > khi_x || ky < klo_y || ky > khi_y) continue;
            double fx, fy;
            if (stretch) {
                if (!or_pullback(lam, pitch, kx * dfx, ky * dfy, &fx, &fy)) continue;
            } else {
                fx = kx * dfx;
                fy = ky * dfy;
            }
            double gx = fx * nx * pitch, gy = fy * ny * pitch; /* grid units */
            if (fabs(gx) > 0.5 * nx || fabs(gy) > 0.5 * ny) continue;
            tx[s] = gx;
            ty[s] = gy;
            keep[s] = 1;
        }
    }
    cplx *S = (cplx *)malloc(sizeof(cplx) * nS);
    if (gH) {
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < (int64_t)nS; ++t) S[t] = gg_eval(gH, tx[t], ty[t]);
    } else {
        off_grid((const double *)H, nx, ny, tx, ty, (int64_t)nS, (double *)S);
    }
    for (size_t s = 0; s < nS; ++s)
        if (!keep[s]) S[s] = 0;
    free(keep);
    free(tx);
    free(ty);

    /* inverse transform: H'_v = centred IDFT(S) / (Npx Npy), demodulated by f'_c */
    centred_dft2(S, npx, npy, +1);
    const double inv = 1.0 / ((double)npx * npy);
    /* step three, Eq. 2 input side: multiply by e^{i pi (x^2 + y^2)/(lambda z)},
     * x_n = (n - Np/2) * N pitch / Np */
    const double hx = nx * pitch / npx, hy = ny * pitch / npy;
    for (int m = 0; m < npy; ++m) {
        double y = (m - npy / 2) * hy;
        for (int n = 0; n < npx; ++n) {
            double x = (n - npx / 2) * hx;
            double ph = OR_PI * (x * x + y * y) / (lam * z);
            S[(size_t)m * npx + n] *= inv * (cos(ph) + I * sin(ph));
        }
    }

    /* Steps three and five: P(x') = sum_n c_n e^{-2 pi i x_n (x' - lambda z f'_c)/(lambda z)}
     * evaluated at x'(x_o) of Eq. 17, then O = e^{i pi |x'|^2/(lambda z)} P. */
    size_t nO = (size_t)ox * oy;
    double *ux = (double *)malloc(sizeof(double) * nO), *uy = (double *)malloc(sizeof(double) * nO);
    double *xq = (double *)malloc(sizeof(double) * nO), *yq = (double *)malloc(sizeof(double) * nO);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < oy; ++j) {
        double yo = cy + (j - 0.5 * oy) * py;
        for (int i = 0; i < ox; ++i) {
            double xo = cx + (i - 0.5 * ox) * px;
            double xp, yp;
            if (stretch) or_output_map(lam, z, xo, yo, &xp, &yp);
            else { xp = xo; yp = yo; }
            size_t o = (size_t)j * ox + i;
            xq[o] = xp;
            yq[o] = yp;
            ux[o] = xp * nx * pitch / (lam * z) - (double)kcx;
            uy[o] = yp * ny * pitch / (lam * z) - (double)kcy;
        }
    }
    cplx *P = (cplx *)malloc(sizeof(cplx) * nO);
    off_grid((const double *)S, npx, npy, ux, uy, (int64_t)nO, (double *)P);
    for (size_t o = 0; o < nO; ++o) {
        double ph = OR_PI * (xq[o] * xq[o] + yq[o] * yq[o]) / (lam * z);
        cplx O = (cos(ph) + I * sin(ph)) * P[o];
        if (field_out) ((cplx *)field_out)[o] = O;
        if (intensity_out) intensity_out[o] = creal(O) * creal(O) + cimag(O) * cimag(O);
    }
    free(P);
    free(S);
    free(ux);
    free(uy);
    free(xq);
    free(yq);
    return 0;
}

/* O0: the c64 hologram as the GPU receives it, promoted to FP64 */
static cplx *promote(const float *holo, int nx, int ny) {
    size_t nh = (size_t)nx * ny;
    cplx *H = (cplx *)malloc(sizeof(cplx) * nh);
    for (size_t i = 0; i < nh; ++i) H[i] = (double)holo[2 * i] + I * (double)holo[2 * i + 1];
    return H;
}

int or_reconstruct(double lam, double pitch, int nx, int ny, const float *holo, double z,
                   double cx, double cy, double w, double h, int ox_in, int oy_in, int stretch,
                   int threads, double *field_out, double *intensity_out) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    cplx *H = promote(holo, nx, ny);
    int r = recon_view(lam, pitch, nx, ny, H, NULL, z, cx, cy, w, h, ox_in, oy_in, stretch,
                       field_out, intensity_out);
    free(H);
    return r;
}

/*
 * Several views of one hologram (arrays of nv view arguments and output
 * pointers, as in or_reconstruct).  The same arithmetic as nv calls of
 * or_reconstruct; the gridded oversampled transform of the hologram that
 * step two evaluates is computed once and shared by the views.
 */
int or_reconstruct_views(double lam, double pitch, int nx, int ny, const float *holo, int nv,
                         const double *z, const double *cx, const double *cy, const double *w,
                         const double *h, const int *ox, const int *oy, int stretch, int threads,
                         double *const *field_out, double *const *intensity_out) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    cplx *H = promote(holo, nx, ny);
    gg_plan gH;
    const gg_plan *pg = NULL;
    if (!g_linear) {
        gg_prepare(&gH, H, nx, ny);
        pg = &gH;
    }
    int r = 0;
    for (int v = 0; v < nv && !r; ++v)
        r = recon_view(lam, pitch, nx, ny, H, pg, z[v], cx[v], cy[v], w[v], h[v], ox[v], oy[v],
                       stretch, field_out ? field_out[v] : NULL,
                       intensity_out ? intensity_out[v] : NULL);
    if (pg) free(gH.grid);
    free(H);
    return r;
}

/* Number of OpenMP threads the oracle will use. */
int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
