/*
 * Seeded synthetic inputs: point clouds and their point-source holograms.
 *
 * This module only makes inputs.  It holds none of the reconstruction
 * method's arithmetic (no spectra, no magnification maps, no Fresnel
 * transform), so both the FP64 oracle and the CUDA path may consume what it
 * produces.
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), the top 53 bits scaled to a
 * uniform double in [0, 1).
 *
 * Point model: Eq. 3 of the paper, a spherical wave e^{-ikR} per object
 * point, unit amplitude and no 1/R factor, multiplied by the point's complex
 * weight a*e^{i*theta}.  Hologram sample n sits at x_n = (n - N/2)*pitch.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static uint64_t splitmix64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double uniform01(uint64_t *s) {
    return (double)(splitmix64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

/* n uniform doubles in [0,1) from seed (exposed for tests of the stream). */
void synth_uniform(uint64_t seed, int64_t n, double *out) {
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) out[i] = uniform01(&s);
}

/*
 * Point cloud inside the square pyramid of the full view.
 * Draw order per point: z, x, y, amplitude, phase.
 *   z  ~ U[z_min, z_max]
 *   x,y ~ U[-z*tan_half_fov, +z*tan_half_fov] * spread   (spread <= 1)
 *   a  ~ U[a_min, a_max]
 *   theta ~ U[0, 2*pi)
 * pts is n_points x 5 doubles: x, y, z, a, theta.
 */
void synth_points(uint64_t seed, int32_t n_points, double z_min, double z_max,
                  double tan_half_fov, double spread, double a_min, double a_max,
                  double *pts) {
    uint64_t s = seed;
    for (int32_t j = 0; j < n_points; ++j) {
        double z = z_min + (z_max - z_min) * uniform01(&s);
        double half = z * tan_half_fov * spread;
        double x = -half + 2.0 * half * uniform01(&s);
        double y = -half + 2.0 * half * uniform01(&s);
        double a = a_min + (a_max - a_min) * uniform01(&s);
        double th = 2.0 * M_PI * uniform01(&s);
        pts[5 * j + 0] = x;
        pts[5 * j + 1] = y;
        pts[5 * j + 2] = z;
        pts[5 * j + 3] = a;
        pts[5 * j + 4] = th;
    }
}

/*
 * H[iy*nx + ix] = sum_j a_j e^{i theta_j} e^{-i k R_j},
 * R_j = sqrt((x - x_j)^2 + (y - y_j)^2 + z_j^2), summed in FP64 and rounded
 * to complex64 (interleaved re, im floats).
 * Rows [row0, row0 + nrows) only, written to out from row 0 (lets a caller
 * generate a big hologram in slabs).
 */
void synth_hologram_rows(const double *pts, int32_t n_points, double wavelength,
                         double pitch, int32_t nx, int32_t ny, int32_t row0,
                         int32_t nrows, int32_t threads, float *out) {
    const double k = 2.0 * M_PI / wavelength;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t r = 0; r < nrows; ++r) {
        const int32_t iy = row0 + r;
        const double y = ((double)iy - 0.5 * ny) * pitch;
        double *acc = (double *)calloc(2 * (size_t)nx, sizeof(double));
        for (int32_t j = 0; j < n_points; ++j) {
            const double xj = pts[5 * j], yj = pts[5 * j + 1], zj = pts[5 * j + 2];
            const double a = pts[5 * j + 3], th = pts[5 * j + 4];
            const double dy2z2 = (y - yj) * (y - yj) + zj * zj;
            for (int32_t ix = 0; ix < nx; ++ix) {
                const double x = ((double)ix - 0.5 * nx) * pitch;
                const double R = sqrt((x - xj) * (x - xj) + dy2z2);
                const double ph = th - k * R;
                acc[2 * ix] += a * cos(ph);
                acc[2 * ix + 1] += a * sin(ph);
            }
        }
        float *o = out + 2 * (size_t)r * nx;
        for (int32_t ix = 0; ix < 2 * nx; ++ix) o[ix] = (float)acc[ix];
        free(acc);
    }
}

void synth_hologram(const double *pts, int32_t n_points, double wavelength,
                    double pitch, int32_t nx, int32_t ny, int32_t threads,
                    float *out) {
    synth_hologram_rows(pts, n_points, wavelength, pitch, nx, ny, 0, ny,
                        threads, out);
}

/* Exact FP64 value of one hologram sample (for sampled checks). */
void synth_sample(const double *pts, int32_t n_points, double wavelength,
                  double pitch, int32_t nx, int32_t ny, int32_t ix, int32_t iy,
                  double *re_im) {
    const double k = 2.0 * M_PI / wavelength;
    const double x = ((double)ix - 0.5 * nx) * pitch;
    const double y = ((double)iy - 0.5 * ny) * pitch;
    double re = 0.0, im = 0.0;
    for (int32_t j = 0; j < n_points; ++j) {
        const double dx = x - pts[5 * j], dy = y - pts[5 * j + 1], z = pts[5 * j + 2];
        const double ph = pts[5 * j + 4] - k * sqrt(dx * dx + dy * dy + z * z);
        re += pts[5 * j + 3] * cos(ph);
        im += pts[5 * j + 3] * sin(ph);
    }
    re_im[0] = re;
    re_im[1] = im;
}
