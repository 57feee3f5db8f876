// FP64 coordinate maps of the NU-FDS method and the tables built from them.
//
// With u = lambda f_x, v = lambda f_y, the stretch of Eqs. 9, 10 with the
// magnification of Eq. 16 reads
//   lambda f_x' = (1 - v^2)^(1/4) g(u / sqrt(1 - v^2)),
//   lambda f_y' = (1 - u^2)^(1/4) g(v / sqrt(1 - u^2)),
// where g(s) = s 2F1(1/2, 3/4; 3/2; s^2) = int_0^s (1 - t^2)^(-3/4) dt
// (integrating Eq. 15 in f_x).  g is evaluated from two series of that
// integral: the binomial series of the integrand around t = 0 for |s| <= 1/2,
// and around t = 1 (in powers of 1 - s) above, with g(1) = B(1/2, 1/4) / 2;
// either needs at most ~30 terms for 1e-18.
//
// Every value that sets a sampling position is computed here in FP64, once
// per plan (or per off-lattice view), and stored as an integer base on the
// 2x oversampled grid plus an FP32 fraction in [0, 1), which keeps ~1e-7 of
// a fine cell after the FP32 kernels take over.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "internal.cuh"

namespace nufds {

// Coefficients of the two series, c_n = (3/4)_n / n! by its recurrence in FP64:
// a_n = c_n / (2n + 1) (about t = 0) and b_n = c_n / (n + 1/4) (about t = 1),
// tabulated once so the series loops carry no FP64 division (slow on this GPU).
constexpr int kGTerms = 200;
struct GCoef {
    double a[kGTerms], b[kGTerms];
};
static GCoef make_gcoef() {
    GCoef t;
    double c = 1.0;
    for (int n = 0; n < kGTerms; ++n) {
        if (n > 0) c *= (n - 0.25) / n;
        t.a[n] = c / (2.0 * n + 1.0);
        t.b[n] = c / (n + 0.25);
    }
    return t;
}
static const GCoef h_gcoef = make_gcoef();
__constant__ GCoef c_gcoef;

static int gcoef_init() {
    static std::mutex mu;
    static std::map<int, bool> ready;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return -4;
    std::lock_guard<std::mutex> lk(mu);
    if (ready[dev]) return 0;
    if (cudaMemcpyToSymbol(c_gcoef, &h_gcoef, sizeof(GCoef)) != cudaSuccess) return -4;
    ready[dev] = true;
    return 0;
}

__host__ __device__ inline double g_series(double s, double g1) {
#ifdef __CUDA_ARCH__
    const GCoef &k = c_gcoef;
#else
    const GCoef &k = h_gcoef;
#endif
    double a = fabs(s);
    double r;
    if (a <= 0.5) {
        // sum_n c_n s^(2n+1) / (2n+1): terms fall by s^2 <= 1/4
        double s2 = a * a, p = a, sum = a;
        for (int n = 1; n < kGTerms; ++n) {
            p *= s2;
            double t = k.a[n] * p;
            sum += t;
            if (t < 1e-18 * sum) break;
        }
        r = sum;
    } else {
        // g(1) - 2^(-3/4) sum_n c_n 2^(-n) e^(n + 1/4) / (n + 1/4), e = 1 - s:
        // terms fall by e/2 < 1/4
        double e = 1.0 - a;
        if (e <= 0.0) {
            r = g1;
        } else {
            double q = sqrt(sqrt(e)), h = 1.0, sum = 0.0;
            for (int n = 0; n < kGTerms; ++n) {
                if (n > 0) h *= 0.5 * e;
                double t = k.b[n] * h * q;
                sum += t;
                if (t < 1e-18 * sum) break;
            }
            r = g1 - 0.59460355750136053336 * sum;  // 2^(-3/4)
        }
    }
    return s < 0 ? -r : r;
}

double g_at_one() {
    // B(1/2, 1/4) / 2 = Gamma(1/2) Gamma(1/4) / (2 Gamma(3/4))
    return tgamma(0.5) * tgamma(0.25) / (2.0 * tgamma(0.75));
}

double host_g(double s) { return g_series(s, g_at_one()); }

// Surrogate g(s) = s P(s) and g'(s) = P(s) + s P'(s) (Horner, degree 8)
__host__ __device__ inline void poly_g(const MapFn &m, double s, double *g, double *gp) {
    double p = m.c[8], d = 8.0 * m.c[8];
    for (int k = 7; k >= 0; --k) {
        p = p * s + m.c[k];
        if (k >= 1) d = d * s + k * m.c[k];
    }
    *g = s * p;
    *gp = p + s * d;
}

// gs (optional): the two g values of the exact map, g(u / sqrt(ay)) and
// g(v / sqrt(ax)), which the Jacobian at the same point reuses
__host__ __device__ inline void phi_uv(double u, double v, double g1, const MapFn &m, double *up,
                                       double *vp, double *gs = nullptr) {
    double ay = 1.0 - v * v, ax = 1.0 - u * u;
    if (m.poly) {
        double gx, gy, d;
        poly_g(m, u / sqrt(ay), &gx, &d);
        poly_g(m, v / sqrt(ax), &gy, &d);
        *up = sqrt(sqrt(ay)) * gx;
        *vp = sqrt(sqrt(ax)) * gy;
        return;
    }
    const double gu = g_series(u / sqrt(ay), g1), gv = g_series(v / sqrt(ax), g1);
    *up = sqrt(sqrt(ay)) * gu;
    *vp = sqrt(sqrt(ax)) * gv;
    if (gs) {
        gs[0] = gu;
        gs[1] = gv;
    }
}

void host_phi(double u, double v, double *up, double *vp, const MapFn &m) {
    phi_uv(u, v, g_at_one(), m, up, vp);
}

// Least-squares fit of the surrogate: modified Gram-Schmidt on the augmented
// 51 x (9 + 1) Vandermonde system [A | b] in s = lambda f, b = 2F1(s^2) =
// g(s) / s from the series above (1 at s = 0).
void map_fit_paper_poly(double lam, double pitch, MapFn *m) {
    const int M = 51, N = 9;
    double A[51][10];
    const double g1 = g_at_one();
    for (int i = 0; i < M; ++i) {
        const double s = lam * (-0.5 + (double)i / (M - 1)) / pitch;
        double t = 1.0;
        for (int j = 0; j < N; ++j, t *= s) A[i][j] = t;
        A[i][N] = s == 0.0 ? 1.0 : g_series(s, g1) / s;
    }
    double R[10][10] = {};
    for (int j = 0; j <= N; ++j) {
        for (int k = 0; k < j && k < N; ++k) {  // remove the earlier directions
            double d = 0.0;
            for (int i = 0; i < M; ++i) d += A[i][k] * A[i][j];
            R[k][j] = d;
            for (int i = 0; i < M; ++i) A[i][j] -= d * A[i][k];
        }
        if (j < N) {
            double nrm = 0.0;
            for (int i = 0; i < M; ++i) nrm += A[i][j] * A[i][j];
            nrm = sqrt(nrm);
            R[j][j] = nrm;
            for (int i = 0; i < M; ++i) A[i][j] /= nrm;
        }
    }
    for (int j = N - 1; j >= 0; --j) {  // R c = Q^T b (column N of R)
        double t = R[j][N];
        for (int k = j + 1; k < N; ++k) t -= R[j][k] * m->c[k];
        m->c[j] = t / R[j][j];
    }
    m->poly = 1;
}

// Jacobian d(u', v')/d(u, v) of the stretch (Eq. 15 on the diagonal).  For the
// surrogate: du'/du = ay^(-1/4) g'(s), du'/dv = -v/2 ay^(-3/4) g(s) +
// u v ay^(-5/4) g'(s), s = u / sqrt(ay) (and x <-> y).
__device__ inline void jac_uv(double u, double v, double g1, const MapFn &m, double J[4],
                              const double *gs = nullptr) {
    double ay = 1.0 - v * v, ax = 1.0 - u * u;
    if (m.poly) {
        double gy, dy, gx, dx;
        poly_g(m, u / sqrt(ay), &gy, &dy);
        poly_g(m, v / sqrt(ax), &gx, &dx);
        J[0] = dy / sqrt(sqrt(ay));
        J[3] = dx / sqrt(sqrt(ax));
        J[1] = -0.5 * v * gy / sqrt(sqrt(ay * ay * ay)) + u * v * dy / (ay * sqrt(sqrt(ay)));
        J[2] = -0.5 * u * gx / sqrt(sqrt(ax * ax * ax)) + u * v * dx / (ax * sqrt(sqrt(ax)));
        return;
    }
    double r = 1.0 - u * u - v * v;
    double r34 = 1.0 / sqrt(sqrt(r * r * r));  // r^(-3/4)
    J[0] = sqrt(ay) * r34;
    J[3] = sqrt(ax) * r34;
    double gy = gs ? gs[0] : g_series(u / sqrt(ay), g1);
    double gx = gs ? gs[1] : g_series(v / sqrt(ax), g1);
    J[1] = -0.5 * v * gy / sqrt(sqrt(ay * ay * ay)) + u * v * r34 / sqrt(ay);
    J[2] = -0.5 * u * gx / sqrt(sqrt(ax * ax * ax)) + u * v * r34 / sqrt(ax);
}

// Inverse of the stretch: solve phi(u, v) = (up, vp) inside the unit disc by
// damped Newton, from (u0, v0) when given inside the disc (an interpolated
// neighbouring solution), else from (up, vp) pulled inside radius 0.9.
// Returns false when (up, vp) has no pre-image.
__device__ bool pullback_uv(double up, double vp, double g1, const MapFn &m, double tol, double *uo,
                            double *vo, double u0 = 2.0, double v0 = 0.0) {
    double u = up, v = vp;
    if (u0 * u0 + v0 * v0 < 0.99) {
        u = u0;
        v = v0;
    }
    double rr = u * u + v * v;
    if (rr > 0.81 && !(u0 * u0 + v0 * v0 < 0.99)) {
        double sc = 0.9 * rsqrt(rr);
        u *= sc;
        v *= sc;
    }
    double fu, fv, gs[2] = {0.0, 0.0};  // gs: the g values at (u, v), for the Jacobian
    phi_uv(u, v, g1, m, &fu, &fv, gs);
    double res = fabs(fu - up) + fabs(fv - vp);
    for (int it = 0; it < 100; ++it) {
        double J[4];
        jac_uv(u, v, g1, m, J, gs);
        double det = J[0] * J[3] - J[1] * J[2];
        double ru = up - fu, rv = vp - fv;
        double du = (J[3] * ru - J[1] * rv) / det;
        double dv = (J[0] * rv - J[2] * ru) / det;
        double step = 1.0;
        bool ok = false;
        for (int h = 0; h < 60; ++h) {
            double un = u + step * du, vn = v + step * dv;
            if (un * un + vn * vn < 1.0) {
                double gu, gv, gsn[2] = {0.0, 0.0};
                phi_uv(un, vn, g1, m, &gu, &gv, gsn);
                double rn = fabs(gu - up) + fabs(gv - vp);
                if (rn < res || rn == 0.0 || step * (fabs(du) + fabs(dv)) <= tol) {
                    u = un;
                    v = vn;
                    fu = gu;
                    fv = gv;
                    gs[0] = gsn[0];
                    gs[1] = gsn[1];
                    res = rn;
                    ok = true;
                    break;
                }
            }
            step *= 0.5;
        }
        if (!ok) return false;
        if (step * (fabs(du) + fabs(dv)) <= tol) {
            *uo = u;
            *vo = v;
            return res <= 2e-12 * (1.0 + fabs(up) + fabs(vp));
        }
    }
    return false;
}

// the fine base as an offset from 2k (the identity map) and the FP32 fraction
__device__ inline void split_fine(double t2, long k2, short *base, float *frac) {
    double b = floor(t2);
    *base = (short)((long)b - k2);
    *frac = (float)(t2 - b);
}

// Coarse solutions for the pull-back table: the pre-image (u, v) of every
// step-th lattice point of the band (and of its last row and column), NaN
// where there is none.  Node c of an axis sits at min(c step, n - 1).
__global__ void k_pullback_coarse(double lam, double pitch, int nx, int ny, long kx0, int nkx,
                                  long ky0, int nky, int step, int ncx, int ncy, double g1,
                                  MapFn m, double2 *cuv) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)ncx * ncy) return;
    const int cx = (int)(idx / ncy), cy = (int)(idx - (long)cx * ncy);
    const int ix = min(cx * step, nkx - 1), iy = min(cy * step, nky - 1);
    const double up = lam * (double)(kx0 + ix) / (nx * pitch);
    const double vp = lam * (double)(ky0 + iy) / (ny * pitch);
    double u, v;
    if (pullback_uv(up, vp, g1, m, 1e-13 * lam / pitch, &u, &v)) cuv[idx] = make_double2(u, v);
    else cuv[idx] = make_double2(NAN, NAN);
}

// Table of f(f'_k) for lattice points k of the stretched band, layout [kx][ky]:
// fine coordinates 2 t with t = N pitch f (centred grid units), the integer
// base stored as its offset from 2 k (|2 t - 2 k| stays far below 2^15 while
// 2 t itself reaches +-N), the fraction in FP32.  Masked (base.x = kMasked)
// where there is no pre-image or |t_x| > N_x/2 or |t_y| > N_y/2.  With coarse
// solutions (cuv), Newton starts from their bilinear interpolation when the
// four surrounding ones exist (one or two steps instead of several from the
// identity; the same root and the same stopping rule).
__global__ void k_pullback_table(double lam, double pitch, int nx, int ny, long kx0, int nkx,
                                 long ky0, int nky, double g1, MapFn m, short2 *base,
                                 float2 *frac, const double2 *cuv, int step, int ncx, int ncy) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nkx * nky) return;
    int ix = (int)(idx / nky), iy = (int)(idx - (long)ix * nky);
    double up = lam * (double)(kx0 + ix) / (nx * pitch);
    double vp = lam * (double)(ky0 + iy) / (ny * pitch);
    double u0 = 2.0, v0 = 0.0;  // no start given
    if (cuv) {
        const int cx = min(ix / step, ncx - 2), cy = min(iy / step, ncy - 2);
        const int x0 = cx * step, x1 = min((cx + 1) * step, nkx - 1);
        const int y0 = cy * step, y1 = min((cy + 1) * step, nky - 1);
        const double ax = x1 > x0 ? (double)(ix - x0) / (x1 - x0) : 0.0;
        const double ay = y1 > y0 ? (double)(iy - y0) / (y1 - y0) : 0.0;
        const double2 c00 = cuv[(long)cx * ncy + cy], c01 = cuv[(long)cx * ncy + cy + 1];
        const double2 c10 = cuv[(long)(cx + 1) * ncy + cy], c11 = cuv[(long)(cx + 1) * ncy + cy + 1];
        const double su = (1 - ax) * ((1 - ay) * c00.x + ay * c01.x) + ax * ((1 - ay) * c10.x + ay * c11.x);
        const double sv = (1 - ax) * ((1 - ay) * c00.y + ay * c01.y) + ax * ((1 - ay) * c10.y + ay * c11.y);
        if (su == su && sv == sv) {  // all four corners solved (NaN propagates)
            u0 = su;
            v0 = sv;
        }
    }
    double u, v;
    short2 b = make_short2(kMasked, kMasked);
    float2 f = make_float2(0.f, 0.f);
    if (pullback_uv(up, vp, g1, m, 1e-13 * lam / pitch, &u, &v, u0, v0)) {
        double tx = nx * pitch * u / lam, ty = ny * pitch * v / lam;
        if (fabs(tx) <= 0.5 * nx && fabs(ty) <= 0.5 * ny) {
            split_fine(2.0 * tx, 2 * (kx0 + ix), &b.x, &f.x);
            split_fine(2.0 * ty, 2 * (ky0 + iy), &b.y, &f.y);
        }
    }
    base[idx] = b;
    frac[idx] = f;
}

// floor and 0.32 fixed-point fraction (truncated, so the fraction is < 1)
__device__ inline void split_fine_fx(double t2, int *base, unsigned int *frac) {
    double b = floor(t2);
    *base = (int)b;
    double q = floor((t2 - b) * 4294967296.0);
    *frac = q >= 4294967295.0 ? 0xffffffffu : (unsigned int)q;
}

// Output map of Eq. 17 in stretched-lattice units t' = N pitch f_0 m(f_0),
// f_0 = (x_o, y_o) / (lambda R_0), for view pixels; layout [j][i].
__global__ void k_remap_table(double lam, double pitch, int nx, int ny, double z, double cx,
                              double cy, double px, double py, int ox, int oy, double g1,
                              MapFn m, int2 *base, uint2 *frac, int plain) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)ox * oy) return;
    int j = (int)(idx / ox), i = (int)(idx - (long)j * ox);
    double xo = cx + (i - 0.5 * ox) * px, yo = cy + (j - 0.5 * oy) * py;
    double up, vp;
    if (plain) {  // x' = x_o: lambda f' = x_o / z
        up = xo / z;
        vp = yo / z;
    } else {
        double R0 = sqrt(xo * xo + yo * yo + z * z);
        phi_uv(xo / R0, yo / R0, g1, m, &up, &vp);
    }
    double tx = nx * pitch * up / lam, ty = ny * pitch * vp / lam;
    int2 b;
    uint2 f;
    split_fine_fx(2.0 * tx, &b.x, &f.x);
    split_fine_fx(2.0 * ty, &b.y, &f.y);
    base[idx] = b;
    frac[idx] = f;
}

// chirp at the group-major position of each slot:
// e^{i pi x_n^2/(lambda z)} deapod[n] / L, x_n = (n - L/2) window / L,
// n the natural index of the slot in the digit-reversed order of the row FFT
__device__ inline void chirp_entry(const FftPlan &fp, double window, double lam, double z,
                                   int linear, int slot, float2 *chirp) {
    const int L = fp.L;
    if (slot >= L) return;
    const int n = fft_index_of_slot(fp, slot);
    const double *deapod = fp.deapod;
    double x = (n - L / 2) * (window / L);
    double ph = M_PI * x * x / (lam * z);
    ph -= 2.0 * M_PI * rint(ph / (2.0 * M_PI));
    double s, c;
    sincos(ph, &s, &c);
    double a = (linear ? 1.0 : deapod[n]) / L;
    chirp[fft_gm_pos(fp, slot)] = make_float2((float)(c * a), (float)(s * a));
}

__global__ void k_chirp_table(FftPlan fp, double window, double lam, double z, int linear,
                              float2 *chirp) {
    chirp_entry(fp, window, lam, z, linear, blockIdx.x * blockDim.x + threadIdx.x, chirp);
}

__global__ void k_chirp_table_batch(const ChirpItem *__restrict__ items,
                                    const int *__restrict__ off, int nitems) {
    int lo = 0, hi = nitems - 1;  // last item with off <= blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const ChirpItem &c = items[lo];
    chirp_entry(c.fp, c.window_m, c.lam, c.z, c.linear,
                ((int)blockIdx.x - off[lo]) * blockDim.x + threadIdx.x, c.chirp);
}

int launch_chirp_table_batch(const ChirpItem *d_items, const int *d_off, int nitems,
                             int total_blocks, cudaStream_t st) {
    if (total_blocks <= 0) return 0;
    k_chirp_table_batch<<<total_blocks, 256, 0, st>>>(d_items, d_off, nitems);
    count_launch();
    return check_launch();
}

__global__ void k_outchirp_table(double kappa, long b0, int nb, OutChirp *E) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double b = (double)(b0 + i);
    double ph = 0.25 * kappa * b * b;
    ph -= 2.0 * M_PI * rint(ph / (2.0 * M_PI));
    double s, c;
    sincos(ph, &s, &c);
    OutChirp o;
    o.e = make_float2((float)c, (float)s);
    const long long k = llrint(kappa * b / (4.0 * M_PI) * 4294967296.0);
    o.klo = (unsigned int)(k & 0xffffffffLL);
    o.khi = (int)(k >> 32);
    E[i] = o;
}

int pullback_coarse_count(int nkx, int nky) {
    const int ncx = (nkx - 1 + kPullbackStep - 1) / kPullbackStep + 1;
    const int ncy = (nky - 1 + kPullbackStep - 1) / kPullbackStep + 1;
    return ncx * ncy;
}

int launch_pullback_table(double lam, double pitch, int nx, int ny, long kx0, int nkx, long ky0,
                          int nky, short2 *base, float2 *frac, cudaStream_t st, const MapFn &m,
                          double2 *coarse) {
    long n = (long)nkx * nky;
    if (n <= 0) return 0;
    if (gcoef_init()) return -4;
    const int step = kPullbackStep;
    const int ncx = (nkx - 1 + step - 1) / step + 1, ncy = (nky - 1 + step - 1) / step + 1;
    if (coarse && (ncx < 2 || ncy < 2)) coarse = nullptr;
    if (coarse) {
        const long nc = (long)ncx * ncy;
        k_pullback_coarse<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(
            lam, pitch, nx, ny, kx0, nkx, ky0, nky, step, ncx, ncy, g_at_one(), m, coarse);
        count_launch();
        if (check_launch()) return -4;
    }
    k_pullback_table<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
        lam, pitch, nx, ny, kx0, nkx, ky0, nky, g_at_one(), m, base, frac, coarse, step, ncx, ncy);
    count_launch();
    return check_launch();
}

int launch_remap_table(double lam, double pitch, int nx, int ny, double z, double cx, double cy,
                       double px, double py, int ox, int oy, int2 *base, uint2 *frac,
                       cudaStream_t st, int plain, const MapFn &m) {
    long n = (long)ox * oy;
    if (n <= 0) return 0;
    if (gcoef_init()) return -4;
    k_remap_table<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(lam, pitch, nx, ny, z, cx, cy, px,
                                                              py, ox, oy, g_at_one(), m, base, frac, plain);
    count_launch();
    return check_launch();
}

int launch_chirp_table(const FftPlan &fp, double window_m, double lam, double z, float2 *chirp,
                       cudaStream_t st, int linear) {
    k_chirp_table<<<(fp.L + 255) / 256, 256, 0, st>>>(fp, window_m, lam, z, linear, chirp);
    count_launch();
    return check_launch();
}

int launch_outchirp_table(double kappa, long b0, int nb, OutChirp *E, cudaStream_t st) {
    const double bmax = (double)std::max(std::labs(b0), std::labs(b0 + nb));
    if (!(fabs(kappa) * bmax / (4.0 * M_PI) < 1073741824.0)) return -3;
    k_outchirp_table<<<(nb + 255) / 256, 256, 0, st>>>(kappa, b0, nb, E);
    count_launch();
    return check_launch();
}

}  // namespace nufds
