// The two off-grid resampling steps of NU-FDS as gathers on 2x oversampled grids.
//
// Step two (Section 4): S(f'_k) = H~(f(f'_k)), the hologram spectrum at the
// pulled-back frequency of every stretched-lattice point, i.e. the DTFT of
// the hologram evaluated off its DFT grid.  The spectrum is cached on a 2x
// oversampled grid of the deapodised hologram, so the value at any frequency
// is a short separable sum with the ES kernel (W x W taps).
//
// Step five: O(x_o) = O'(x_o'(x_o)), the Fresnel-transform output evaluated
// at the Eq. 17 image of every output pixel, from the 2x oversampled FrT grid
// the same way; then |O|^2 or O times the output chirp.
//
// Both read a coordinate table (integer fine-grid base + FP32 fraction,
// derived in FP64) and wrap indices periodically (the DTFT is periodic).
// The 2x grids are stored plane-wise per axis (fine index m at
// (m & 1) * L + m / 2), as the row passes write them, except the columns of
// the spectrum G, which are in natural order: a warp of the stretch covers 32
// consecutive band points along y whose windows step by ~1.5 fine columns, so
// one contiguous run per row touches fewer sectors than two planes do.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>

#include "internal.cuh"

namespace nufds {

// Kernel weights of the kW taps for a fractional offset f in [0, 1): tap i is
// at distance d_i = f + kW/2 - 1 - i and weighs psi(d_i) =
// exp(beta (sqrt(1 - (2 d_i / kW)^2) - 1)).  Each psi(f + c_i) is smooth in f,
// so it is evaluated as a degree-kEsDeg polynomial P_i in t = 2f - 1 whose
// coefficients are Chebyshev interpolants built in FP64 on the host (max
// error ~1e-7 absolute, weights <= 1).  psi is even, so tap kW-1-i at f is
// tap i at 1 - f: P_{kW-1-i}(t) = P_i(-t).  With P_i(t) = E_i(t^2) + t O_i(t^2)
// both taps come from one evaluation of E_i and O_i.
constexpr int kEsDeg = 12;
constexpr int kEsEven = kEsDeg / 2 + 1;  // coefficients of E_i (t^0, t^2, ..)
constexpr int kEsOdd = kEsDeg / 2;       // coefficients of O_i (t^1, t^3, ..)
__constant__ float c_es_e[kW / 2][kEsEven];
__constant__ float c_es_o[kW / 2][kEsOdd];

__device__ __forceinline__ void es_weights(float f, float *w) {
    const float t = 2.0f * f - 1.0f, u = t * t;
#pragma unroll
    for (int i = 0; i < kW / 2; ++i) {
        float e = c_es_e[i][kEsEven - 1];
#pragma unroll
        for (int k = kEsEven - 2; k >= 0; --k) e = fmaf(e, u, c_es_e[i][k]);
        float o = c_es_o[i][kEsOdd - 1];
#pragma unroll
        for (int k = kEsOdd - 2; k >= 0; --k) o = fmaf(o, u, c_es_o[i][k]);
        w[i] = fmaf(t, o, e);
        w[kW - 1 - i] = fmaf(-t, o, e);
    }
}

static double psi_host(double d) {
    const double u = 2.0 * d / kW, q = 1.0 - u * u;
    return q > 0.0 ? exp(kBeta * (sqrt(q) - 1.0)) : 0.0;
}

// Chebyshev interpolation of the weight of taps 0 .. kW/2-1 on kEsDeg + 1
// nodes, converted to monomial coefficients in t and split into even and odd
// parts; uploaded once per device.
static int es_init() {
    static std::mutex mu;
    static std::map<int, bool> ready;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return -4;
    std::lock_guard<std::mutex> lk(mu);
    if (ready[dev]) return 0;
    const int n = kEsDeg + 1;
    float he[kW / 2][kEsEven], ho[kW / 2][kEsOdd];
    for (int i = 0; i < kW / 2; ++i) {
        double a[kEsDeg + 1] = {0};
        for (int k = 0; k < n; ++k) {
            double s = 0;
            for (int j = 0; j < n; ++j) {
                const double x = cos(M_PI * (j + 0.5) / n);
                s += psi_host(0.5 * (x + 1.0) + (kW / 2 - 1 - i)) * cos(k * M_PI * (j + 0.5) / n);
            }
            a[k] = 2.0 * s / n;
        }
        a[0] *= 0.5;
        // sum a_k T_k(t) -> monomials, T_{k+1} = 2 t T_k - T_{k-1}
        double mono[kEsDeg + 1] = {0}, tk[kEsDeg + 1] = {0}, tkm1[kEsDeg + 1] = {0};
        tkm1[0] = 1.0;  // T_0
        tk[1] = 1.0;    // T_1
        mono[0] += a[0];
        if (kEsDeg >= 1) mono[1] += a[1];
        for (int k = 2; k <= kEsDeg; ++k) {
            double nx[kEsDeg + 1] = {0};
            for (int m = 0; m <= kEsDeg; ++m) {
                if (m >= 1) nx[m] += 2.0 * tk[m - 1];
                nx[m] -= tkm1[m];
            }
            for (int m = 0; m <= kEsDeg; ++m) {
                tkm1[m] = tk[m];
                tk[m] = nx[m];
                mono[m] += a[k] * nx[m];
            }
        }
        for (int m = 0; m < kEsEven; ++m) he[i][m] = (float)mono[2 * m];
        for (int m = 0; m < kEsOdd; ++m) ho[i][m] = (float)mono[2 * m + 1];
    }
    if (cudaMemcpyToSymbol(c_es_e, he, sizeof(he)) != cudaSuccess ||
        cudaMemcpyToSymbol(c_es_o, ho, sizeof(ho)) != cudaSuccess)
        return -4;
    ready[dev] = true;
    return 0;
}

// m in [-M, 2M): periodic index without integer division
__device__ __forceinline__ int wrap(int m, int M) {
    return m < 0 ? m + M : (m >= M ? m - M : m);
}

// Debug build (NUFDS_BOUNDS_CHECK): every gather read is checked against the
// extent of the array it reads; a read outside is skipped (its taps count as
// zero), counted, and the first offending element offset recorded, so the
// host can ask (bounds_violations) instead of the kernel faulting.  In the
// product build the check is compiled out.
#ifdef NUFDS_BOUNDS_CHECK
__device__ unsigned long long g_oob_count = 0;
__device__ unsigned long long g_oob_first = ~0ull;
// [lo, hi) inside [0, total)
__device__ __forceinline__ bool in_bounds(long lo, long hi, long total) {
    if (lo >= 0 && lo <= hi && hi <= total) return true;
    atomicAdd(&g_oob_count, 1ull);
    atomicCAS(&g_oob_first, ~0ull, (unsigned long long)lo);
    return false;
}
// columns [c_lo, c_hi) of the row at element offset roff (row length ld)
// inside that row, and the row inside [0, total)
__device__ __forceinline__ bool in_row(long roff, long c_lo, long c_hi, long ld, long total) {
    if (c_lo >= 0 && c_lo <= c_hi && c_hi <= ld && roff >= 0 && roff + ld <= total) return true;
    atomicAdd(&g_oob_count, 1ull);
    atomicCAS(&g_oob_first, ~0ull, (unsigned long long)(roff + c_lo));
    return false;
}
#else
__device__ __forceinline__ bool in_bounds(long, long, long) { return true; }
__device__ __forceinline__ bool in_row(long, long, long, long, long) { return true; }
#endif

int bounds_violations(int reset, long long *first) {
#ifdef NUFDS_BOUNDS_CHECK
    unsigned long long n = 0, f = ~0ull;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(&n, g_oob_count, sizeof n) != cudaSuccess ||
        cudaMemcpyFromSymbol(&f, g_oob_first, sizeof f) != cudaSuccess)
        return -4;
    if (first) *first = f == ~0ull ? -1 : (long long)f;
    if (reset) {
        const unsigned long long z = 0, m = ~0ull;
        if (cudaMemcpyToSymbol(g_oob_count, &z, sizeof z) != cudaSuccess ||
            cudaMemcpyToSymbol(g_oob_first, &m, sizeof m) != cudaSuccess)
            return -4;
    }
    return (int)(n > 0x7fffffffull ? 0x7fffffffull : n);
#else
    if (first) *first = -1;
    (void)reset;
    return -3;  // not a checking build
#endif
}

// sum_{i,j} wr[i] wc[j] A[row r0 + i][column c0 + j] for a window inside a
// grid stored plane-wise on both axes (fine row m at row (m & 1) Lr + (m >> 1),
// pitch ld; fine column m at (m & 1) Lc + (m >> 1)): 0 <= r0, r0 + kW <= 2 Lr,
// 0 <= c0, c0 + kW <= 2 Lc.  The kW columns of a row are two runs of kW/2
// consecutive elements (even taps in one plane, odd taps in the other), so
// each run is one pointer and its loads take immediate offsets.  Same
// summation order as the general path.
// Four consecutive elements row[s .. s+3] as two 2-element vector loads from
// the aligned-down start, plus one single load of the last element when s is
// odd (rows start on 2-element boundaries: A is 256-byte aligned and every
// pitch is even).  Fewer, wider requests than four single loads: fewer L1
// tag lookups, more data-pipe wavefronts per request -- a gain where lanes
// are far apart (the remap), a loss where their windows overlap (the stretch).
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ void load_run4(const float2 *__restrict__ row, int s, float2 *v) {
    const bool odd = s & 1;
    const float4 *q = reinterpret_cast<const float4 *>(row + (s & ~1));
    const float4 f0 = __ldg(q), f1 = __ldg(q + 1);
    float2 f2 = make_float2(0.f, 0.f);
    if (odd) f2 = __ldg(row + s + 3);
    v[0] = odd ? hi2(f0) : lo2(f0);
    v[1] = odd ? lo2(f1) : hi2(f0);
    v[2] = odd ? hi2(f1) : lo2(f1);
    v[3] = odd ? f2 : hi2(f1);
}
__device__ __forceinline__ float2 cvt_c(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 cvt_c(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <class H>
__device__ __forceinline__ void load_run4_16(const H *__restrict__ row, int s, float2 *v) {
    const bool odd = s & 1;
    const uint2 *q = reinterpret_cast<const uint2 *>(row + (s & ~1));
    const uint2 f0 = __ldg(q), f1 = __ldg(q + 1);
    unsigned int f2 = 0u;
    if (odd) f2 = __ldg(reinterpret_cast<const unsigned int *>(row + s + 3));
    const unsigned int w[5] = {f0.x, f0.y, f1.x, f1.y, f2};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned int u = odd ? w[k + 1] : w[k];
        H h;
        memcpy(&h, &u, sizeof(h));
        v[k] = cvt_c(h);
    }
}
__device__ __forceinline__ void load_run4(const __half2 *__restrict__ row, int s, float2 *v) {
    load_run4_16(row, s, v);
}
__device__ __forceinline__ void load_run4(const __nv_bfloat162 *__restrict__ row, int s,
                                          float2 *v) {
    load_run4_16(row, s, v);
}

template <bool WIDE, class T>
__device__ __forceinline__ float2 window_sum_inside(const T *__restrict__ A, long ld, int Lr,
                                                   int Lc, int r0, int c0, const float *wr,
                                                   const float *wc, long total) {
    const int e = c0 & 1;
    const int ca = e * Lc + (c0 >> 1), cb = (1 - e) * Lc + ((c0 + 1) >> 1);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kW; ++i) {
        const int r = r0 + i;
        const long roff = (long)((r & 1) * Lr + (r >> 1)) * ld;
        // load_run4 reads [s & ~1, s + kW/2) of each plane run s = ca, cb
        if (!in_row(roff, min(ca, cb) & ~1, max(ca, cb) + kW / 2, ld, total)) continue;
        const T *row = A + roff;
        float2 va[kW / 2], vb[kW / 2];
        if (WIDE) {
            load_run4(row, ca, va);
            load_run4(row, cb, vb);
        } else {
#pragma unroll
            for (int q = 0; q < kW / 2; ++q) {
                va[q] = ld_c(row + ca, q, 1.0f);
                vb[q] = ld_c(row + cb, q, 1.0f);
            }
        }
        float2 sum = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < kW / 2; ++q) {
            const float2 ga = va[q], gb = vb[q];
            sum.x = fmaf(wc[2 * q], ga.x, sum.x);
            sum.y = fmaf(wc[2 * q], ga.y, sum.y);
            sum.x = fmaf(wc[2 * q + 1], gb.x, sum.x);
            sum.y = fmaf(wc[2 * q + 1], gb.y, sum.y);
        }
        acc.x = fmaf(wr[i], sum.x, acc.x);
        acc.y = fmaf(wr[i], sum.y, acc.y);
    }
    return acc;
}

// Eight consecutive elements row[s .. s+7] as four 2-element vector loads
// from the aligned-down start plus the ninth element when s is odd.
__device__ __forceinline__ void load_run8(const float2 *__restrict__ row, int s, float2 *v) {
    const bool odd = s & 1;
    const float4 *q = reinterpret_cast<const float4 *>(row + (s & ~1));
    float2 e[9];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 f = __ldg(q + k);
        e[2 * k] = lo2(f);
        e[2 * k + 1] = hi2(f);
    }
    e[8] = make_float2(0.f, 0.f);
    if (odd) e[8] = __ldg(row + s + 7);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = odd ? e[k + 1] : e[k];
}
template <class H>
__device__ __forceinline__ void load_run8_16(const H *__restrict__ row, int s, float2 *v) {
    const bool odd = s & 1;
    const uint2 *q = reinterpret_cast<const uint2 *>(row + (s & ~1));
    unsigned int e[9];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint2 f = __ldg(q + k);
        e[2 * k] = f.x;
        e[2 * k + 1] = f.y;
    }
    e[8] = 0u;
    if (odd) e[8] = __ldg(reinterpret_cast<const unsigned int *>(row + s + 7));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const unsigned int u = odd ? e[k + 1] : e[k];
        H h;
        memcpy(&h, &u, sizeof(h));
        v[k] = cvt_c(h);
    }
}
__device__ __forceinline__ void load_run8(const __half2 *__restrict__ row, int s, float2 *v) {
    load_run8_16(row, s, v);
}
__device__ __forceinline__ void load_run8(const __nv_bfloat162 *__restrict__ row, int s,
                                          float2 *v) {
    load_run8_16(row, s, v);
}

// As window_sum_inside, for a grid whose columns are in natural order (rows
// still plane-wise): the kW columns of a row are one run of kW elements.
template <class T>
__device__ __forceinline__ float2 window_sum_natcols(const T *__restrict__ A, long ld, int Lr,
                                                    int r0, int c0, const float *wr,
                                                    const float *wc, long total) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kW; ++i) {
        const int r = r0 + i;
        const long roff = (long)((r & 1) * Lr + (r >> 1)) * ld;
        // load_run8 reads [c0 & ~1, c0 + kW)
        if (!in_row(roff, c0 & ~1, c0 + kW, ld, total)) continue;
        const T *row = A + roff;
        float2 v[kW];
        load_run8(row, c0, v);
        float2 sum = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kW; ++j) {
            sum.x = fmaf(wc[j], v[j].x, sum.x);
            sum.y = fmaf(wc[j], v[j].y, sum.y);
        }
        acc.x = fmaf(wr[i], sum.x, acc.x);
        acc.y = fmaf(wr[i], sum.y, acc.y);
    }
    return acc;
}

template <class T>
__device__ __forceinline__ void stretch_body(const StretchArgs &a, int bx, int by) {
    const T *G = (const T *)a.G;
    const float ginv = a.sc_g ? 1.0f / *a.sc_g : 1.0f, ssc = a.sc_s ? *a.sc_s : 1.0f;
    // a warp covers 32 consecutive band points along y (measured faster than
    // 8 x 4 blocks, whose lanes' windows spread over more lines of G)
    const int jy = bx * 32 + threadIdx.x;
    const int jx = a.jx0 + by * kStretchRows + threadIdx.y;
    const bool inside = jx - a.jx0 < (a.jn ? a.jn : a.npx) && jx < a.npx && jy < a.npy;
    const long kx = a.kc_x + jx - a.npx / 2, ky = a.kc_y + jy - a.npy / 2;
    bool valid = false;
    int2 b = make_int2(0, 0);
    float2 f = make_float2(0.f, 0.f);
    if (inside && kx >= a.klo_x && kx <= a.khi_x && ky >= a.klo_y && ky <= a.khi_y) {
        if (a.plain) {  // f = f'_k: fine position 2k, zero outside |f| <= 1/(2 pitch)
            if (2 * labs(kx) <= a.Nx && 2 * labs(ky) <= a.Ny) {
                b = make_int2((int)(2 * kx), (int)(2 * ky));
                valid = true;
            }
        } else {
            const long t = (kx - a.pb_kx0) * a.pb_nky + (ky - a.pb_ky0);
            if (in_bounds(t, t + 1, (long)a.pb_nkx * a.pb_nky)) {
                const short2 e = a.pb_base[t];
                if (e.x != kMasked) {
                    b = make_int2(e.x + (int)(2 * kx), e.y + (int)(2 * ky));
                    f = a.pb_frac[t];
                    valid = true;
                }
            }
        }
    }
    const int Mx = 2 * a.Nx, My = 2 * a.Ny;
    const long gtot = (long)Mx * My;
    // first taps on the fine grid, unwrapped (rows = x, columns = y)
    const int r0 = b.x - kW / 2 + 1 + a.Nx, c0 = b.y - kW / 2 + 1 + a.Ny;
    float2 acc = make_float2(0.f, 0.f);
    if (valid) {
        float wx[kW], wy[kW];
        es_weights(f.x, wx);
        es_weights(f.y, wy);
        if (r0 >= 0 && r0 + kW <= Mx && c0 >= 0 && c0 + kW <= My) {
            acc = window_sum_natcols(G, My, a.Nx, r0, c0, wx, wy, gtot);
        } else {  // the window wraps around the periodic grid
            int cols[kW];
#pragma unroll
            for (int j = 0; j < kW; ++j) cols[j] = wrap(c0 + j, My);
#pragma unroll
            for (int i = 0; i < kW; ++i) {
                const long row = (long)fine_pos(wrap(r0 + i, Mx), a.Nx) * My;
                float2 r = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < kW; ++j) {
                    if (!in_row(row, cols[j], cols[j] + 1, My, gtot)) continue;
                    float2 gv = ld_c(G, row + cols[j], 1.0f);
                    r.x = fmaf(wy[j], gv.x, r.x);
                    r.y = fmaf(wy[j], gv.y, r.y);
                }
                acc.x = fmaf(wx[i], r.x, acc.x);
                acc.y = fmaf(wx[i], r.y, acc.y);
            }
        }
        // (-1)^(jx + jy): centring of the inverse transforms that follow
        if ((jx + jy) & 1) acc = make_float2(-acc.x, -acc.y);
        acc = make_float2(acc.x * ginv, acc.y * ginv);
    }
    if (inside) st_c((T *)a.S, (long)jx * a.npy + jy, acc, ssc);
}

template <class T>
__global__ void __launch_bounds__(32 * kStretchRows, 32 / kStretchRows) k_stretch(StretchArgs a) {
    stretch_body<T>(a, blockIdx.x, blockIdx.y);
}

__device__ __forceinline__ int find_item(const int *off, int nitems, int b) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class T>
__global__ void __launch_bounds__(32 * kStretchRows, 32 / kStretchRows) k_stretch_batch(const StretchArgs *__restrict__ items,
                                                       const int *__restrict__ off, int nitems) {
    const int it = find_item(off, nitems, blockIdx.x);
    const StretchArgs &a = items[it];
    const int t = blockIdx.x - off[it], tx = (a.npy + 31) / 32;
    stretch_body<T>(a, t % tx, t / tx);
}

__device__ __forceinline__ void remap_store(const RemapArgs &a, long o, float2 acc, int2 b,
                                            uint2 F);

template <class T>
__device__ __forceinline__ void remap_body(const RemapArgs &a, int bx, int by) {
    const T *Q = (const T *)a.Q;
    const float qinv = a.sc_q ? 1.0f / *a.sc_q : 1.0f;
    const int i = bx * 32 + threadIdx.x;
    const int j = by * kRemapRows + threadIdx.y;
    const bool valid = i < a.ox && j < a.oy;
    int2 b = make_int2(0, 0);
    uint2 F = make_uint2(0u, 0u);
    if (valid) {
        const long t = (long)(j + a.rm_j0) * a.rm_ld + (i + a.rm_i0);
        if (in_bounds(t, t + 1, a.rm_count)) {
            b = a.rm_base[t];
            F = a.rm_frac[t];
        }
    }
    // the fraction in FP32 for the weights (rounded toward zero: stays < 1)
    const float2 f = make_float2(__uint2float_rz(F.x) * 0x1p-32f, __uint2float_rz(F.y) * 0x1p-32f);
    const int Mx = 2 * a.npx, My = 2 * a.npy;
    // first taps on the fine grid, unwrapped (rows = y, columns = x)
    const int c0 = (int)(b.x - 2 * a.kc_x) + a.npx - kW / 2 + 1;
    const int r0 = (int)(b.y - 2 * a.kc_y) + a.npy - kW / 2 + 1;
    float2 acc = make_float2(0.f, 0.f);
    if (!valid) return;
    float wx[kW], wy[kW];
    es_weights(f.x, wx);
    es_weights(f.y, wy);
    if (r0 >= 0 && r0 + kW <= My && c0 >= 0 && c0 + kW <= Mx) {
        acc = window_sum_inside<true>(Q, Mx, a.npy, a.npx, r0, c0, wy, wx, (long)Mx * My);
    } else {  // the window wraps around the periodic grid
        int cols[kW];
#pragma unroll
        for (int q = 0; q < kW; ++q) cols[q] = fine_pos(wrap(c0 + q, Mx), a.npx);
#pragma unroll
        for (int p = 0; p < kW; ++p) {
            const long row = (long)fine_pos(wrap(r0 + p, My), a.npy) * Mx;
            float2 r = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < kW; ++q) {
                if (!in_row(row, cols[q], cols[q] + 1, Mx, (long)Mx * My)) continue;
                float2 g = ld_c(Q, row + cols[q], 1.0f);
                r.x = fmaf(wx[q], g.x, r.x);
                r.y = fmaf(wx[q], g.y, r.y);
            }
            acc.x = fmaf(wy[p], r.x, acc.x);
            acc.y = fmaf(wy[p], r.y, acc.y);
        }
    }
    acc = make_float2(acc.x * qinv, acc.y * qinv);
    remap_store(a, (long)j * a.ox + i, acc, b, F);
}

// O = P at the output pixel o: |O|^2, added |O|^2, or O times the output chirp
// of the fine position b + F 2^-32
__device__ __forceinline__ void remap_store(const RemapArgs &a, long o, float2 acc, int2 b,
                                            uint2 F) {
    if (a.kind == 0) {
        ((float *)a.out)[o] = fmaf(acc.x, acc.x, acc.y * acc.y);
    } else if (a.kind == 2) {  // accumulate |O|^2 (speckle averaging)
        ((float *)a.out)[o] += fmaf(acc.x, acc.x, acc.y * acc.y);
    } else {
        // e^{i kappa (b + f)^2 / 4} per axis: the b^2 part from the table, the
        // rest, kappa b f / 2 + kappa f^2 / 4, in turns reduced mod 1 exactly:
        // bits 32..63 of K * F (K = kappa b / (4 pi) in 32.32, F = f 2^32) and
        // of K2 * G (K2 = kappa / (8 pi), G = f^2 2^32).
        const OutChirp cx = a.Ex[b.x - a.ex_b0], cy = a.Ey[b.y - a.ey_b0];
        const unsigned int gx = __umulhi(F.x, F.x), gy = __umulhi(F.y, F.y);
        unsigned int tq = __umulhi(cx.klo, F.x) + (unsigned int)cx.khi * F.x;
        tq += __umulhi(cy.klo, F.y) + (unsigned int)cy.khi * F.y;
        tq += __umulhi(a.k2x.x, gx) + a.k2x.y * gx;
        tq += __umulhi(a.k2y.x, gy) + a.k2y.y * gy;
        float s, c;
        sincospif((float)(int)tq * 0x1p-31f, &s, &c);  // 2 pi (tq / 2^32), in (-pi, pi]
        const float2 ex = cx.e, ey = cy.e;
        float2 e = make_float2(ex.x * ey.x - ex.y * ey.y, ex.x * ey.y + ex.y * ey.x);
        float2 w = make_float2(e.x * c - e.y * s, e.x * s + e.y * c);
        ((float2 *)a.out)[o] = make_float2(acc.x * w.x - acc.y * w.y, acc.x * w.y + acc.y * w.x);
    }
}

// ------------------------------------------------------------------------
// Paper-literal variant (plan flag NUFDS_FLAG_PAPER_LINEAR, FP32 storage):
// linear interpolation, separable in x and y, on the unpadded grids instead
// of the ideal resampling above (Section 4 names interpolation in steps two
// and five without its kernel).  The even fine samples of G are the centred
// DFT of the hologram when it is loaded without deapodisation, and the even
// fine samples of Q the native FrT output when the chirp carries none; both
// are periodic like the DFT.
// ------------------------------------------------------------------------

// floor(m / 2) for any sign
__device__ __forceinline__ int floor_half(int m) { return (m - (m & 1)) / 2; }

// bilinear of a periodic coarse grid (C rows x D columns) stored at
// A[r * ld + c * cs], at coarse position (i + ax, j + ay), i, j centred
__device__ __forceinline__ float2 lerp2(const float2 *__restrict__ A, long ld, int cs, int C,
                                        int D, int i, float ax, int j, float ay) {
    const int r0 = wrap(i + C / 2, C), r1 = wrap(i + 1 + C / 2, C);
    const int c0 = wrap(j + D / 2, D), c1 = wrap(j + 1 + D / 2, D);
    if (!in_bounds(min(r0, r1), max(r0, r1) + 1, C) || !in_bounds(min(c0, c1), max(c0, c1) + 1, D))
        return make_float2(0.f, 0.f);
    const float2 v00 = __ldg(A + r0 * ld + (long)c0 * cs), v01 = __ldg(A + r0 * ld + (long)c1 * cs);
    const float2 v10 = __ldg(A + r1 * ld + (long)c0 * cs), v11 = __ldg(A + r1 * ld + (long)c1 * cs);
    const float bx = 1.0f - ax, by = 1.0f - ay;
    const float2 u0 = make_float2(by * v00.x + ay * v01.x, by * v00.y + ay * v01.y);
    const float2 u1 = make_float2(by * v10.x + ay * v11.x, by * v10.y + ay * v11.y);
    return make_float2(bx * u0.x + ax * u1.x, bx * u0.y + ax * u1.y);
}

// step two: S(f'_k) = bilinear of the unpadded spectrum at the pulled-back f
__global__ void __launch_bounds__(256) k_stretch_linear(StretchArgs a) {
    const int jy = blockIdx.x * 32 + threadIdx.x, jx = a.jx0 + blockIdx.y * 8 + threadIdx.y;
    if (jx - a.jx0 >= (a.jn ? a.jn : a.npx) || jx >= a.npx || jy >= a.npy) return;
    const long kx = a.kc_x + jx - a.npx / 2, ky = a.kc_y + jy - a.npy / 2;
    float2 acc = make_float2(0.f, 0.f);
    bool valid = false;
    int2 b = make_int2(0, 0);
    float2 f = make_float2(0.f, 0.f);
    if (kx >= a.klo_x && kx <= a.khi_x && ky >= a.klo_y && ky <= a.khi_y) {
        if (a.plain) {
            if (2 * labs(kx) <= a.Nx && 2 * labs(ky) <= a.Ny) {
                b = make_int2((int)(2 * kx), (int)(2 * ky));
                valid = true;
            }
        } else {
            const long t = (kx - a.pb_kx0) * a.pb_nky + (ky - a.pb_ky0);
            const short2 e = in_bounds(t, t + 1, (long)a.pb_nkx * a.pb_nky)
                                 ? a.pb_base[t] : make_short2(kMasked, kMasked);
            if (e.x != kMasked) {
                b = make_int2(e.x + (int)(2 * kx), e.y + (int)(2 * ky));
                f = a.pb_frac[t];
                valid = true;
            }
        }
    }
    if (valid) {
        // fine position b + f = 2 (coarse position): rows plane-wise (even
        // fine row 2c is row c), columns natural (even fine column 2c)
        acc = lerp2((const float2 *)a.G, 2L * a.Ny, 2, a.Nx, a.Ny, floor_half(b.x),
                    ((b.x & 1) + f.x) * 0.5f, floor_half(b.y), ((b.y & 1) + f.y) * 0.5f);
        if ((jx + jy) & 1) acc = make_float2(-acc.x, -acc.y);
    }
    ((float2 *)a.S)[(long)jx * a.npy + jy] = acc;
}

// step five: O(x_o) = bilinear of the native FrT output at x'(x_o)
__global__ void __launch_bounds__(256) k_remap_linear(RemapArgs a) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    if (i >= a.ox || j >= a.oy) return;
    const long t = (long)(j + a.rm_j0) * a.rm_ld + (i + a.rm_i0);
    if (!in_bounds(t, t + 1, a.rm_count)) return;
    const int2 b = a.rm_base[t];
    const uint2 F = a.rm_frac[t];
    const int px = (int)(b.x - 2 * a.kc_x), py = (int)(b.y - 2 * a.kc_y);
    const float fx = __uint2float_rz(F.x) * 0x1p-32f, fy = __uint2float_rz(F.y) * 0x1p-32f;
    // Q: rows = y, columns = x, both plane-wise: even fine index 2c at c
    const float2 acc = lerp2((const float2 *)a.Q, 2L * a.npx, 1, a.npy, a.npx, floor_half(py),
                             ((py & 1) + fy) * 0.5f, floor_half(px), ((px & 1) + fx) * 0.5f);
    remap_store(a, (long)j * a.ox + i, acc, b, F);
}

template <class T>
__global__ void __launch_bounds__(32 * kRemapRows, 32 / kRemapRows) k_remap(RemapArgs a) {
    remap_body<T>(a, blockIdx.x, blockIdx.y);
}

template <class T>
__global__ void __launch_bounds__(32 * kRemapRows, 32 / kRemapRows) k_remap_batch(const RemapArgs *__restrict__ items,
                                                     const int *__restrict__ off, int nitems) {
    const int it = find_item(off, nitems, blockIdx.x);
    const RemapArgs &a = items[it];
    const int t = blockIdx.x - off[it], tx = (a.ox + 31) / 32;
    remap_body<T>(a, t % tx, t / tx);
}

int launch_stretch(const StretchArgs &a, cudaStream_t st) {
    if (es_init()) return -4;
    const int rows = a.jn ? a.jn : a.npx;
    const dim3 grid((a.npy + 31) / 32, (rows + kStretchRows - 1) / kStretchRows),
        blk(32, kStretchRows);
    if (a.linear && a.prec != PREC_F32) return -3;
    if (a.linear)
        k_stretch_linear<<<dim3((a.npy + 31) / 32, (rows + 7) / 8), dim3(32, 8), 0, st>>>(a);
    else if (a.prec == PREC_F32) k_stretch<float2><<<grid, blk, 0, st>>>(a);
    else if (a.prec == PREC_F16) k_stretch<__half2><<<grid, blk, 0, st>>>(a);
    else k_stretch<__nv_bfloat162><<<grid, blk, 0, st>>>(a);
    count_launch();
    return check_launch();
}

int launch_stretch_batch(const StretchArgs *d_items, const int *d_off, int nitems, int total,
                         int prec, cudaStream_t st) {
    if (es_init()) return -4;
    if (total <= 0) return 0;
    if (prec == PREC_F32) k_stretch_batch<float2><<<total, dim3(32, kStretchRows), 0, st>>>(d_items, d_off, nitems);
    else if (prec == PREC_F16) k_stretch_batch<__half2><<<total, dim3(32, kStretchRows), 0, st>>>(d_items, d_off, nitems);
    else k_stretch_batch<__nv_bfloat162><<<total, dim3(32, kStretchRows), 0, st>>>(d_items, d_off, nitems);
    count_launch();
    return check_launch();
}

int launch_remap_batch(const RemapArgs *d_items, const int *d_off, int nitems, int total, int prec,
                       cudaStream_t st) {
    if (es_init()) return -4;
    if (total <= 0) return 0;
    if (prec == PREC_F32) k_remap_batch<float2><<<total, dim3(32, kRemapRows), 0, st>>>(d_items, d_off, nitems);
    else if (prec == PREC_F16) k_remap_batch<__half2><<<total, dim3(32, kRemapRows), 0, st>>>(d_items, d_off, nitems);
    else k_remap_batch<__nv_bfloat162><<<total, dim3(32, kRemapRows), 0, st>>>(d_items, d_off, nitems);
    count_launch();
    return check_launch();
}

int launch_remap(const RemapArgs &a, cudaStream_t st) {
    if (es_init()) return -4;
    const dim3 grid((a.ox + 31) / 32, (a.oy + kRemapRows - 1) / kRemapRows), blk(32, kRemapRows);
    if (a.linear && a.prec != PREC_F32) return -3;
    if (a.linear)
        k_remap_linear<<<dim3((a.ox + 31) / 32, (a.oy + 7) / 8), dim3(32, 8), 0, st>>>(a);
    else if (a.prec == PREC_F32) k_remap<float2><<<grid, blk, 0, st>>>(a);
    else if (a.prec == PREC_F16) k_remap<__half2><<<grid, blk, 0, st>>>(a);
    else k_remap<__nv_bfloat162><<<grid, blk, 0, st>>>(a);
    count_launch();
    return check_launch();
}

}  // namespace nufds
