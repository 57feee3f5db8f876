// GPU generator of point-source holograms (Eq. 3), for inputs too large to
// sum on the host (16K x 16K x 20000 points).  Input generation only: no
// arithmetic of the reconstruction method lives here.
//
// H(x, y) = sum_j a_j e^{i theta_j} e^{-i k R_j(x, y)}.  Per 128 x 128 pixel
// tile and point, the phase at the tile centre is formed in FP64 and reduced
// to [-pi, pi]; inside the tile the phase offset k (R - R_c) is formed in FP32
// from R - R_c = (R^2 - R_c^2)/(R + R_c), exact to ~3e-5 rad for tiles of
// ~20 um half-width.  Tiles accumulate in shared memory (FP32) over chunks of
// points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

constexpr int kTile = 128;
constexpr int kChunk = 512;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_holo(const double *__restrict__ pts, int n, double k,
                                                   double pitch, int nx, int ny,
                                                   float2 *__restrict__ out) {
    extern __shared__ float smem[];
    float2 *acc = reinterpret_cast<float2 *>(smem);           // kTile * kTile
    float *sp = smem + 2 * kTile * kTile;                      // kChunk * 6
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const double xc = ((double)(x0 + kTile / 2) - 0.5 * nx) * pitch;
    const double yc = ((double)(y0 + kTile / 2) - 0.5 * ny) * pitch;
    for (int p = threadIdx.x; p < kTile * kTile; p += kThreads) acc[p] = make_float2(0.f, 0.f);
    const float kf = (float)k, pf = (float)pitch;
    const float two_pi = 6.28318530717958648f, inv_two_pi = 0.159154943091895336f;
    for (int c0 = 0; c0 < n; c0 += kChunk) {
        const int m = min(kChunk, n - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kThreads) {
            const double *q = pts + 5 * (size_t)(c0 + j);
            double dx = xc - q[0], dy = yc - q[1], z = q[2];
            double rc2 = dx * dx + dy * dy + z * z;
            double rc = sqrt(rc2);
            double ph = q[4] - k * rc;
            ph -= 2.0 * M_PI * rint(ph / (2.0 * M_PI));
            float *s = sp + 6 * j;
            s[0] = (float)ph;
            s[1] = (float)(2.0 * dx);
            s[2] = (float)(2.0 * dy);
            s[3] = (float)rc2;
            s[4] = (float)rc;
            s[5] = (float)q[3];
        }
        __syncthreads();
        for (int p = threadIdx.x; p < kTile * kTile; p += kThreads) {
            const int ix = p % kTile, iy = p / kTile;
            const float a = (float)(ix - kTile / 2) * pf, c = (float)(iy - kTile / 2) * pf;
            float re = 0.f, im = 0.f;
            for (int j = 0; j < m; ++j) {
                const float *s = sp + 6 * j;
                float b = a + s[1], d = c + s[2];
                float num = fmaf(a, b, c * d);
                float R = sqrtf(s[3] + num);
                float dR = __fdividef(num, R + s[4]);
                float ph = fmaf(-kf, dR, s[0]);
                ph = fmaf(-two_pi, rintf(ph * inv_two_pi), ph);
                float sn, cs;
                __sincosf(ph, &sn, &cs);
                re = fmaf(s[5], cs, re);
                im = fmaf(s[5], sn, im);
            }
            acc[p].x += re;
            acc[p].y += im;
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < kTile * kTile; p += kThreads) {
        const int ix = x0 + p % kTile, iy = y0 + p / kTile;
        if (ix < nx && iy < ny) out[(size_t)iy * nx + ix] = acc[p];
    }
}

}  // namespace

extern "C" int synth_gpu_hologram(const double *d_pts, int n_points, double wavelength,
                                  double pitch, int nx, int ny, void *d_out, void *stream) {
    const size_t smem = sizeof(float) * (2 * kTile * kTile + 6 * kChunk);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_holo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    dim3 grid((nx + kTile - 1) / kTile, (ny + kTile - 1) / kTile);
    k_holo<<<grid, kThreads, smem, (cudaStream_t)stream>>>(d_pts, n_points, 2.0 * M_PI / wavelength,
                                                           pitch, nx, ny, (float2 *)d_out);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -4;
}
