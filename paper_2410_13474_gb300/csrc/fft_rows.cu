// Batched 1-D FFT passes along rows, with the fused pre/post operations of
// the NU-FDS path (Section 4, steps two and three of Fig. 3).
//
// One CTA owns one row at a time (grid-stride over rows).  The row lives in
// shared memory; the transform is a mixed-radix in-place decomposition
// L = r_1 r_2 ... r_P with radices in {2,3,4,5,6,8,9,10,12,15,16}:
//   * decimation in frequency (DIF) takes natural order to digit-reversed
//     order, the first pass reading straight from global memory;
//   * decimation in time (DIT) with the same radices takes digit-reversed
//     order back to natural order, the last pass writing straight to global
//     memory.
// So "inverse FFT -> pointwise chirp -> forward FFT" needs no reordering
// pass.  Each pass: a thread loads the r elements of a group into registers,
// runs an unrolled r-point DFT, applies the inter-pass twiddles and stores
// back to the same shared-memory slots.  Shared memory is padded by one
// element per 16 to spread strided accesses over the banks.
//
// Twiddles: W_L^q = coarse[q >> 6] * fine[q & 63] from two small tables
// built in FP64 on the host (about 2 ulp).  Constants inside the small DFTs
// come from a __constant__ table, also built in FP64.
#include <math.h>

#include <cstdio>
#include <map>
#include <mutex>

#include "internal.cuh"

namespace nufds {

// ------------------------------------------------------------------------
// in-register small DFTs
// ------------------------------------------------------------------------
// W_R^j = e^{-2 pi i j / R} for the composite radices, concatenated
__constant__ float2 c_tw[6 + 8 + 9 + 10 + 12 + 15 + 16];

template <int R> struct TwOff;
template <> struct TwOff<6> { static constexpr int v = 0; };
template <> struct TwOff<8> { static constexpr int v = 6; };
template <> struct TwOff<9> { static constexpr int v = 14; };
template <> struct TwOff<10> { static constexpr int v = 23; };
template <> struct TwOff<12> { static constexpr int v = 33; };
template <> struct TwOff<15> { static constexpr int v = 45; };
template <> struct TwOff<16> { static constexpr int v = 60; };
static const int kCompositeR[7] = {6, 8, 9, 10, 12, 15, 16};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <bool INV> __device__ __forceinline__ float2 twmul(float2 a, float2 w) {
    return INV ? cmulc(a, w) : cmul(a, w);
}

constexpr int smallest_prime(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<1, INV> {
    static __device__ __forceinline__ void run(float2 *) {}
};
template <bool INV> struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2 *x) {
        float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};
template <bool INV> struct Dft<3, INV> {
    static __device__ __forceinline__ void run(float2 *x) {
        const float h = 0.86602540378443864676f;  // sin(2 pi / 3)
        float2 a = x[0], b = x[1], c = x[2];
        float2 t1 = cadd(b, c);
        float2 t2 = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
        float2 t3 = cscale(csub(b, c), h);
        x[0] = cadd(a, t1);
        x[1] = cadd(t2, mul_mi<INV>(t3));
        x[2] = csub(t2, mul_mi<INV>(t3));
    }
};
template <bool INV> struct Dft<4, INV> {
    static __device__ __forceinline__ void run(float2 *x) {
        float2 a = x[0], b = x[1], c = x[2], d = x[3];
        float2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = mul_mi<INV>(csub(b, d));
        x[0] = cadd(s0, s2);
        x[2] = csub(s0, s2);
        x[1] = cadd(s1, s3);
        x[3] = csub(s1, s3);
    }
};
template <bool INV> struct Dft<5, INV> {
    static __device__ __forceinline__ void run(float2 *x) {
        const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
        const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
        float2 a = x[0];
        float2 t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
        float2 t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
        float2 r1 = make_float2(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
        float2 r2 = make_float2(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
        float2 i1 = mul_mi<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
        float2 i2 = mul_mi<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
        x[0] = cadd(a, cadd(t1, t2));
        x[1] = cadd(r1, i1);
        x[4] = csub(r1, i1);
        x[2] = cadd(r2, i2);
        x[3] = csub(r2, i2);
    }
};
// composite R = A * B: X[k1 + A k2] = sum_{n2} W_R^{n2 k1} W_B^{n2 k2} sum_{n1} x[B n1 + n2] W_A^{n1 k1}
template <int R, bool INV> struct Dft {
    static __device__ __forceinline__ void run(float2 *x) {
        constexpr int A = smallest_prime(R);
        constexpr int B = R / A;
        float2 y[R];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) {
            float2 t[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) t[n1] = x[B * n1 + n2];
            Dft<A, INV>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1)
                y[k1 * B + n2] = (n2 * k1 == 0) ? t[k1] : twmul<INV>(t[k1], c_tw[TwOff<R>::v + n2 * k1]);
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            float2 t[B];
#pragma unroll
            for (int n2 = 0; n2 < B; ++n2) t[n2] = y[k1 * B + n2];
            Dft<B, INV>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = t[k2];
        }
    }
};

// ------------------------------------------------------------------------
// passes
// ------------------------------------------------------------------------
struct PassArgs {
    int L, npass;
    int radix[kMaxPasses], stride[kMaxPasses], prefix[kMaxPasses];
    const float2 *tw_fine, *tw_coarse, *mod1;
    const float *pad_pre;
};

__device__ __forceinline__ int phys(int p) { return p + (p >> 4); }

__device__ __forceinline__ float2 twiddle(const PassArgs &P, int q) {
    return cmul(__ldg(P.tw_coarse + (q >> 6)), __ldg(P.tw_fine + (q & 63)));
}

// natural index n -> DIF output / DIT input slot
__device__ __forceinline__ int slot_of_index(const PassArgs &P, int n) {
    int p = 0;
#pragma unroll
    for (int j = 0; j < kMaxPasses; ++j) {
        if (j >= P.npass) break;
        int d = (n / P.prefix[j]) % P.radix[j];
        p += d * P.stride[j];
    }
    return p;
}
// slot -> natural index
__device__ __forceinline__ int index_of_slot(const PassArgs &P, int p) {
    int n = 0;
#pragma unroll
    for (int j = 0; j < kMaxPasses; ++j) {
        if (j >= P.npass) break;
        int d = (p / P.stride[j]) % P.radix[j];
        n += d * P.prefix[j];
    }
    return n;
}

// One pass j over all groups.  DIT: twiddle then DFT; DIF: DFT then twiddle.
// Group g: b = g / s, o = g % s, slots b*(R*s) + o + i*s.
// load(i, slot) -> float2, store(k, slot, value).
template <int R, bool INV, bool DIT, class Load, class Store>
__device__ __forceinline__ void pass_r(const PassArgs &P, int j, Load load, Store store) {
    const int s = P.stride[j];
    const int B = R * s;
    const int tstep = P.L / B;  // W_B^e = W_L^{e * tstep}
    const int ngroups = P.L / R;
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const int b = g / s, o = g - b * s;
        const int base = b * B + o;
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = load(i, base + i * s);
        if (DIT) {
#pragma unroll
            for (int i = 1; i < R; ++i)
                if (o) x[i] = twmul<INV>(x[i], twiddle(P, o * i * tstep));
            Dft<R, INV>::run(x);
        } else {
            Dft<R, INV>::run(x);
#pragma unroll
            for (int k = 1; k < R; ++k)
                if (o) x[k] = twmul<INV>(x[k], twiddle(P, o * k * tstep));
        }
#pragma unroll
        for (int k = 0; k < R; ++k) store(k, base + k * s, x[k]);
    }
}

template <bool INV, bool DIT, class Load, class Store>
__device__ void pass_any(const PassArgs &P, int j, Load load, Store store) {
    switch (P.radix[j]) {
        case 2: pass_r<2, INV, DIT>(P, j, load, store); break;
        case 3: pass_r<3, INV, DIT>(P, j, load, store); break;
        case 4: pass_r<4, INV, DIT>(P, j, load, store); break;
        case 5: pass_r<5, INV, DIT>(P, j, load, store); break;
        case 6: pass_r<6, INV, DIT>(P, j, load, store); break;
        case 8: pass_r<8, INV, DIT>(P, j, load, store); break;
        case 9: pass_r<9, INV, DIT>(P, j, load, store); break;
        case 10: pass_r<10, INV, DIT>(P, j, load, store); break;
        case 12: pass_r<12, INV, DIT>(P, j, load, store); break;
        case 15: pass_r<15, INV, DIT>(P, j, load, store); break;
        case 16: pass_r<16, INV, DIT>(P, j, load, store); break;
        default: break;
    }
}

// forward DIT over passes npass-1 .. 1 in shared memory; pass 0 writes
// out[(2k + a)] * (-1)^k for natural frequency k
__device__ __forceinline__ void dit_forward_to_global(const PassArgs &P, float2 *sm, float2 *orow,
                                                      int a) {
    auto lsm = [&](int, int p) { return sm[phys(p)]; };
    auto ssm = [&](int, int p, float2 v) { sm[phys(p)] = v; };
    for (int j = P.npass - 1; j >= 1; --j) {
        pass_any<false, true>(P, j, lsm, ssm);
        __syncthreads();
    }
    auto sgl = [&](int, int k, float2 v) {
        if (k & 1) v = make_float2(-v.x, -v.y);
        orow[2 * k + a] = v;
    };
    pass_any<false, true>(P, 0, lsm, sgl);
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_rows_pad2(PassArgs P, const float2 *__restrict__ in,
                                                    long in_ld, float2 *__restrict__ out,
                                                    long out_ld, int rows) {
    extern __shared__ float2 sm[];
    const int L = P.L;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const float2 *irow = in + (long)r * in_ld;
        float2 *orow = out + (long)r * out_ld;
        for (int a = 0; a < 2; ++a) {
            for (int n = threadIdx.x; n < L; n += blockDim.x) {
                float2 v = cscale(irow[n], __ldg(P.pad_pre + n));
                if (a) v = cmul(v, __ldg(P.mod1 + n));
                sm[phys(slot_of_index(P, n))] = v;
            }
            __syncthreads();
            dit_forward_to_global(P, sm, orow, a);
        }
    }
}

__global__ void __launch_bounds__(1024) k_rows_view(PassArgs P, const float2 *__restrict__ in,
                                                    long in_ld, const float2 *__restrict__ chirp,
                                                    float2 *__restrict__ out, long out_ld, int rows,
                                                    float2 *__restrict__ scratch) {
    extern __shared__ float2 sm[];
    const int L = P.L;
    float2 *scr = scratch + (long)blockIdx.x * L;
    auto lsm = [&](int, int p) { return sm[phys(p)]; };
    auto ssm = [&](int, int p, float2 v) { sm[phys(p)] = v; };
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const float2 *irow = in + (long)r * in_ld;
        float2 *orow = out + (long)r * out_ld;
        // inverse DFT (DIF): natural -> digit-reversed
        auto lgl = [&](int, int p) { return irow[p]; };
        pass_any<true, false>(P, 0, lgl, ssm);
        __syncthreads();
        for (int j = 1; j < P.npass; ++j) {
            pass_any<true, false>(P, j, lsm, ssm);
            __syncthreads();
        }
        // chirp (with deapodisation and 1/L); keep a copy for the odd half
        for (int p = threadIdx.x; p < L; p += blockDim.x) {
            float2 v = cmul(sm[phys(p)], __ldg(chirp + index_of_slot(P, p)));
            sm[phys(p)] = v;
            scr[p] = v;
        }
        __syncthreads();
        dit_forward_to_global(P, sm, orow, 0);
        for (int p = threadIdx.x; p < L; p += blockDim.x)
            sm[phys(p)] = cmul(scr[p], __ldg(P.mod1 + index_of_slot(P, p)));
        __syncthreads();
        dit_forward_to_global(P, sm, orow, 1);
    }
}

// ------------------------------------------------------------------------
// host side: plans and tables
// ------------------------------------------------------------------------
static const int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

// fewest passes, then the largest smallest radix
static bool factor(int L, int depth, int *out, int &best_n, int *best, int *cur) {
    if (L == 1) {
        if (depth < best_n) {
            best_n = depth;
            for (int i = 0; i < depth; ++i) best[i] = cur[i];
        }
        return true;
    }
    if (depth + 1 >= best_n || depth >= kMaxPasses) return false;
    for (int r : kRadices) {
        if (L % r) continue;
        if (depth > 0 && r > cur[depth - 1]) continue;  // non-increasing: avoid permutations
        cur[depth] = r;
        factor(L / r, depth + 1, out, best_n, best, cur);
    }
    (void)out;
    return best_n <= kMaxPasses;
}

static double psi_es(double s) {
    double t = 2.0 * s / kW;
    if (fabs(t) >= 1.0) return 0.0;
    return exp(kBeta * (sqrt(1.0 - t * t) - 1.0));
}

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on the three-term recurrence)
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

// psi_hat(x) = int psi(s) e^{2 pi i x s / M} ds, M = 2L fine cells; with
// s = (W/2) sin(theta) the integrand is smooth on [0, pi/2].
static void es_fourier(int L, std::vector<double> &ft) {
    static std::vector<double> gx, gw;
    if (gx.empty()) gauss_legendre(128, gx, gw);
    const double M = 2.0 * L, h = 0.5 * kW;
    ft.assign(L, 0.0);
    for (int n = 0; n < L; ++n) {
        double x = n - L / 2;
        double acc = 0.0;
        for (size_t q = 0; q < gx.size(); ++q) {
            double th = 0.25 * M_PI * (gx[q] + 1.0);
            double s = h * sin(th);
            acc += gw[q] * 0.25 * M_PI * psi_es(s) * h * cos(th) * cos(2.0 * M_PI * x * s / M);
        }
        ft[n] = 2.0 * acc;
    }
}

struct LenEntry {
    FftPlan plan;
    float2 *dev = nullptr;  // tw_fine | tw_coarse | mod1
    double *deapod = nullptr;
    float *pad_pre = nullptr;
};

static std::mutex g_mu;
static std::map<std::pair<int, int>, LenEntry *> g_cache;  // (device, L)
static std::map<int, bool> g_const_ready;

static int init_constants() {
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return -4;
    if (g_const_ready[dev]) return 0;
    float2 h[6 + 8 + 9 + 10 + 12 + 15 + 16];
    int off = 0;
    for (int R : kCompositeR)
        for (int j = 0; j < R; ++j, ++off) {
            double a = -2.0 * M_PI * j / R;
            h[off] = make_float2((float)cos(a), (float)sin(a));
        }
    if (cudaMemcpyToSymbol(c_tw, h, sizeof(h)) != cudaSuccess) return -4;
    g_const_ready[dev] = true;
    return 0;
}

int fft_plan_get(int L, const FftPlan **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = init_constants();
    if (rc) return rc;
    int dev;
    cudaGetDevice(&dev);
    auto key = std::make_pair(dev, L);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = &it->second->plan;
        return 0;
    }
    int best[kMaxPasses], cur[kMaxPasses], best_n = kMaxPasses + 1;
    factor(L, 0, nullptr, best_n, best, cur);
    if (best_n > kMaxPasses || L < 16 || (L % 4)) return -3;
    LenEntry *e = new LenEntry();
    FftPlan &p = e->plan;
    p.L = L;
    p.npass = best_n;
    int pre = 1, rem = L;
    for (int j = 0; j < best_n; ++j) {
        p.radix[j] = best[j];
        p.prefix[j] = pre;
        pre *= best[j];
        rem /= best[j];
        p.stride[j] = rem;
    }
    int t = (L / 16 + 31) / 32 * 32;
    p.threads = t < 64 ? 64 : (t > 1024 ? 1024 : t);
    p.smem_bytes = sizeof(float2) * (size_t)(L + L / 16 + 1);
    // tables
    int ncoarse = (L + 63) / 64;
    std::vector<float2> h(64 + ncoarse + L);
    for (int j = 0; j < 64; ++j) {
        double a = -2.0 * M_PI * j / L;
        h[j] = make_float2((float)cos(a), (float)sin(a));
    }
    for (int i = 0; i < ncoarse; ++i) {
        double a = -2.0 * M_PI * (double)(64L * i % L) / L;
        h[64 + i] = make_float2((float)cos(a), (float)sin(a));
    }
    for (int n = 0; n < L; ++n) {
        double a = -M_PI * (n - L / 2) / (double)L;
        h[64 + ncoarse + n] = make_float2((float)cos(a), (float)sin(a));
    }
    std::vector<double> ft;
    es_fourier(L, ft);
    std::vector<double> dea(L);
    std::vector<float> pp(L);
    for (int n = 0; n < L; ++n) {
        dea[n] = 1.0 / ft[n];
        pp[n] = (float)((n & 1) ? -dea[n] : dea[n]);
    }
    if (cudaMalloc(&e->dev, sizeof(float2) * h.size()) != cudaSuccess ||
        cudaMalloc(&e->deapod, sizeof(double) * L) != cudaSuccess ||
        cudaMalloc(&e->pad_pre, sizeof(float) * L) != cudaSuccess) {
        delete e;
        return -2;
    }
    cudaMemcpy(e->dev, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(e->deapod, dea.data(), sizeof(double) * L, cudaMemcpyHostToDevice);
    cudaMemcpy(e->pad_pre, pp.data(), sizeof(float) * L, cudaMemcpyHostToDevice);
    p.tw_fine = e->dev;
    p.tw_coarse = e->dev + 64;
    p.mod1 = e->dev + 64 + ncoarse;
    p.deapod = e->deapod;
    p.pad_pre = e->pad_pre;
    if (p.smem_bytes > 48 * 1024) {
        cudaFuncSetAttribute(k_rows_pad2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
        cudaFuncSetAttribute(k_rows_view, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
    }
    if (p.smem_bytes > 227 * 1024) {
        delete e;
        return -3;
    }
    g_cache[key] = e;
    *out = &p;
    return 0;
}

// Plan and tables of length L written into caller-provided device memory
// (no allocation): d_tw holds 64 + ceil(L/64) + L float2, d_deapod L doubles,
// d_pad L floats.  Tables are computed on the host in FP64 and copied on st.
int fft_plan_fill(int L, FftPlan *p, float2 *d_tw, double *d_deapod, float *d_pad,
                  cudaStream_t st) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        int rc = init_constants();
        if (rc) return rc;
    }
    int best[kMaxPasses], cur[kMaxPasses], best_n = kMaxPasses + 1;
    factor(L, 0, nullptr, best_n, best, cur);
    if (best_n > kMaxPasses || L < 16 || (L % 4)) return -3;
    *p = FftPlan();
    p->L = L;
    p->npass = best_n;
    int pre = 1, rem = L;
    for (int j = 0; j < best_n; ++j) {
        p->radix[j] = best[j];
        p->prefix[j] = pre;
        pre *= best[j];
        rem /= best[j];
        p->stride[j] = rem;
    }
    int t = (L / 16 + 31) / 32 * 32;
    p->threads = t < 64 ? 64 : (t > 1024 ? 1024 : t);
    p->smem_bytes = sizeof(float2) * (size_t)(L + L / 16 + 1);
    if (p->smem_bytes > 48 * 1024) return -3;
    int ncoarse = (L + 63) / 64;
    std::vector<float2> h(64 + ncoarse + L);
    for (int j = 0; j < 64; ++j) {
        double a = -2.0 * M_PI * j / L;
        h[j] = make_float2((float)cos(a), (float)sin(a));
    }
    for (int i = 0; i < ncoarse; ++i) {
        double a = -2.0 * M_PI * (double)(64L * i % L) / L;
        h[64 + i] = make_float2((float)cos(a), (float)sin(a));
    }
    for (int n = 0; n < L; ++n) {
        double a = -M_PI * (n - L / 2) / (double)L;
        h[64 + ncoarse + n] = make_float2((float)cos(a), (float)sin(a));
    }
    std::vector<double> ft;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        es_fourier(L, ft);
    }
    std::vector<double> dea(L);
    std::vector<float> pp(L);
    for (int n = 0; n < L; ++n) {
        dea[n] = 1.0 / ft[n];
        pp[n] = (float)((n & 1) ? -dea[n] : dea[n]);
    }
    if (cudaMemcpyAsync(d_tw, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_deapod, dea.data(), sizeof(double) * L, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_pad, pp.data(), sizeof(float) * L, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return -4;
    // pageable sources: keep them alive until the copies have been consumed
    if (cudaStreamSynchronize(st) != cudaSuccess) return -4;
    p->tw_fine = d_tw;
    p->tw_coarse = d_tw + 64;
    p->mod1 = d_tw + 64 + ncoarse;
    p->deapod = d_deapod;
    p->pad_pre = d_pad;
    return 0;
}

static PassArgs pass_args(const FftPlan &p) {
    PassArgs a;
    a.L = p.L;
    a.npass = p.npass;
    for (int j = 0; j < kMaxPasses; ++j) {
        a.radix[j] = p.radix[j];
        a.stride[j] = p.stride[j];
        a.prefix[j] = p.prefix[j];
    }
    a.tw_fine = p.tw_fine;
    a.tw_coarse = p.tw_coarse;
    a.mod1 = p.mod1;
    a.pad_pre = p.pad_pre;
    return a;
}

static int grid_for(const void *fn, const FftPlan &p, int rows) {
    int dev, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, p.threads, p.smem_bytes);
    if (per < 1) per = 1;
    long g = (long)sms * per;
    return (int)(g < rows ? g : rows);
}

int rows_view_grid(const FftPlan &p, int rows) { return grid_for((const void *)k_rows_view, p, rows); }

int launch_rows_pad2(const FftPlan &p, const float2 *in, long in_ld, float2 *out, long out_ld,
                     int rows, cudaStream_t st) {
    if (rows <= 0) return 0;
    int grid = grid_for((const void *)k_rows_pad2, p, rows);
    k_rows_pad2<<<grid, p.threads, p.smem_bytes, st>>>(pass_args(p), in, in_ld, out, out_ld, rows);
    count_launch();
    return check_launch();
}

int launch_rows_view(const FftPlan &p, const float2 *in, long in_ld, const float2 *chirp,
                     float2 *out, long out_ld, int rows, float2 *scratch, int grid,
                     cudaStream_t st) {
    if (rows <= 0) return 0;
    k_rows_view<<<grid, p.threads, p.smem_bytes, st>>>(pass_args(p), in, in_ld, chirp, out, out_ld,
                                                       rows, scratch);
    count_launch();
    return check_launch();
}

// ------------------------------------------------------------------------
// transpose
// ------------------------------------------------------------------------
__global__ void k_transpose(const float2 *__restrict__ in, long in_ld, float2 *__restrict__ out,
                            long out_ld, int rows, int cols) {
    __shared__ float2 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[(long)r * in_ld + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(long)c * out_ld + r] = tile[threadIdx.x][i];
    }
}

int launch_transpose(const float2 *in, long in_ld, float2 *out, long out_ld, int rows, int cols,
                     cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return 0;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, in_ld, out, out_ld, rows, cols);
    count_launch();
    return check_launch();
}

}  // namespace nufds
