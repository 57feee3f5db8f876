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

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

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

__host__ __device__ constexpr int smallest_prime(int n) {
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
// x W_R^m for the quarter turns (4 m % R == 0): W = (-i)^q, q = 4 m / R (the
// conjugate for the inverse) -- a swap and sign, no multiply
template <bool INV> __device__ __forceinline__ float2 rot_quarter(float2 a, int q) {
    return q == 0 ? a : (q == 2 ? make_float2(-a.x, -a.y) : (q == 1 ? mul_mi<INV>(a) : mul_mi<!INV>(a)));
}

// Split of a composite radix: 4 x (R/4) where R is a multiple of 4 (more
// quarter-turn twiddles than 2 x (R/2)), else smallest prime x rest.
__host__ __device__ constexpr int split_of(int R) {
    return (R % 4 == 0 && R > 4) ? 4 : smallest_prime(R);
}

template <int R, bool INV> struct Dft {
    static __device__ __forceinline__ void run(float2 *x) {
        constexpr int A = split_of(R);
        constexpr int B = R / A;
        float2 y[R];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) {
            float2 t[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) t[n1] = x[B * n1 + n2];
            Dft<A, INV>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) {
                const int m = n2 * k1;  // a constant after unrolling
                y[k1 * B + n2] = (4 * m) % R == 0 ? rot_quarter<INV>(t[k1], (4 * m / R) & 3)
                                                  : twmul<INV>(t[k1], c_tw[TwOff<R>::v + m]);
            }
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


// exact n / d for n * d < 2^32 (host check in fft_plan_*); m == 0 means d == 1
__device__ __forceinline__ uint32_t udiv(uint32_t n, uint32_t m) { return m ? __umulhi(n, m) : n; }

// shared-memory slot -> padded index (two-level padding: every 16th and 256th)
__device__ __forceinline__ int phys(int p) { return p + (p >> 4) + (p >> 8); }

__device__ __forceinline__ float2 tw_base(const float2 *tws, int q) {
    return cmul(tws[64 + (q >> 6)], tws[q & 63]);
}

// W[k] = w^k for k < R (W[0] unused) by a binary tree of products
template <int R> __device__ __forceinline__ void tw_powers(float2 w, float2 *W) {
    W[1] = w;
#pragma unroll
    for (int k = 2; k < R; ++k) {
        int h = 1;
        while (2 * h <= k) h *= 2;
        W[k] = (h == k) ? cmul(W[h / 2], W[h / 2]) : cmul(W[h], W[k - h]);
    }
}

// A middle pass j (shared -> shared).  Group g: b = g / s, o = g % s, slots
// b*R*s + o + i*s.  DIT: twiddle W_{Rs}^{o i} then DFT; DIF: DFT then W^{o k}.
template <int R, bool INV, bool DIT>
__device__ __forceinline__ void mid_pass_r(const PassArgs &P, int j, float2 *sm,
                                           const float2 *tws) {
    const int s = P.stride[j], B = R * s, tstep = P.L / B, ng = P.L / R;
    const uint32_t ms = P.mag_stride[j];
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int b = (int)udiv(g, ms), o = g - b * s, base = b * B + o;
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = sm[phys(base + i * s)];
        if (!DIT) Dft<R, INV>::run(x);
        if (o) {
            float2 W[R];
            tw_powers<R>(tw_base(tws, o * tstep), W);
#pragma unroll
            for (int i = 1; i < R; ++i) x[i] = twmul<INV>(x[i], W[i]);
        }
        if (DIT) Dft<R, INV>::run(x);
#pragma unroll
        for (int k = 0; k < R; ++k) sm[phys(base + k * s)] = x[k];
    }
}

// pass 0 of the inverse DIF, reading the natural-order row from global memory
// (elements outside [lo, hi) are zero and not read)
template <int R, class TI>
__device__ __forceinline__ void dif_first_r(const PassArgs &P, const TI *__restrict__ irow,
                                            float inv, float2 *sm, const float2 *tws, int lo,
                                            int hi) {
    const int s = P.stride[0];
    for (int o = threadIdx.x; o < s; o += blockDim.x) {
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int n = o + i * s;
            x[i] = n >= lo && n < hi ? ld_cs(irow, n, inv) : make_float2(0.f, 0.f);
        }
        Dft<R, true>::run(x);
        if (o) {
            float2 W[R];
            tw_powers<R>(tw_base(tws, o), W);
#pragma unroll
            for (int k = 1; k < R; ++k) x[k] = twmul<true>(x[k], W[k]);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) sm[phys(o + k * s)] = x[k];
    }
}

// last pass (P-1, stride 1) of the inverse DIF fused with the chirp, a copy
// of the result to scratch, and the first forward DIT pass; chirp and
// scratch in group-major order (slot g R + k at k ng + g: coalesced)
template <int R>
__device__ __forceinline__ void fused_mid_r(const PassArgs &P, float2 *sm,
                                            const float2 *__restrict__ chirp_gm,
                                            float2 *__restrict__ scr) {
    const int ng = P.L / R;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int base = g * R;
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = sm[phys(base + i)];
        Dft<R, true>::run(x);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            x[k] = cmul(x[k], __ldg(chirp_gm + k * ng + g));
            scr[k * ng + g] = x[k];
        }
        Dft<R, false>::run(x);
#pragma unroll
        for (int k = 0; k < R; ++k) sm[phys(base + k)] = x[k];
    }
}

// the odd half: reload the chirped samples, modulate (mod: per slot, group-major),
// first forward DIT pass
template <int R>
__device__ __forceinline__ void odd_first_r(const PassArgs &P, float2 *sm,
                                            const float2 *__restrict__ scr,
                                            const float2 *__restrict__ mod) {
    const int ng = P.L / R;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int base = g * R;
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = cmul(scr[i * ng + g], __ldg(mod + i * ng + g));
        Dft<R, false>::run(x);
#pragma unroll
        for (int k = 0; k < R; ++k) sm[phys(base + k)] = x[k];
    }
}

// padded forward pass, first step: natural-order loads (thread <-> n_b), the
// deapodisation and modulation, the first DIT pass, stored at slot(n_b) + k
template <int R, class TI>
__device__ __forceinline__ void pad_first_r(const PassArgs &P, const TI *__restrict__ irow,
                                            float inv, float2 *sm, int a) {
    const int nb = P.L / R;
    for (int n = threadIdx.x; n < nb; n += blockDim.x) {
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int m = n + i * nb;
            float2 v = cscale(ld_cs(irow, m, inv), __ldg(P.pad_pre + m));
            x[i] = a ? cmul(v, __ldg(P.mod1 + m)) : v;
        }
        Dft<R, false>::run(x);
        // slot of n: digits in radices 0..P-2
        uint32_t q = n;
        int base = 0;
        for (int j = 0; j < P.npass - 1; ++j) {
            uint32_t q2 = udiv(q, P.mag_radix[j]);
            base += (int)(q - q2 * P.radix[j]) * P.stride[j];
            q = q2;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) sm[phys(base + k)] = x[k];
    }
}

// pass 0 of the forward DIT: shared -> global, fine index 2k + a = (-1)^k X[k],
// stored in the plane layout at a L + k (or at 2k + a when P.natural_out)
// fine samples 2f and 2f + 1 of a natural-order padded row in one store
__device__ __forceinline__ void st_pair(float2 *p, long f, float2 e, float2 o, float) {
    __stcs(reinterpret_cast<float4 *>(p) + f, make_float4(e.x, e.y, o.x, o.y));
}
template <class H>
__device__ __forceinline__ void st_pair_16(H *p, long f, H e, H o) {
    uint2 u;
    memcpy(&u.x, &e, sizeof(H));
    memcpy(&u.y, &o, sizeof(H));
    __stcs(reinterpret_cast<uint2 *>(p) + f, u);
}
__device__ __forceinline__ void st_pair(__half2 *p, long f, float2 e, float2 o, float sc) {
    st_pair_16(p, f, __float22half2_rn(make_float2(e.x * sc, e.y * sc)),
               __float22half2_rn(make_float2(o.x * sc, o.y * sc)));
}
__device__ __forceinline__ void st_pair(__nv_bfloat162 *p, long f, float2 e, float2 o, float) {
    st_pair_16(p, f, __float22bfloat162_rn(e), __float22bfloat162_rn(o));
}

template <int R, class TO>
__device__ __forceinline__ void dit_last_r(const PassArgs &P, const float2 *sm, const float2 *tws,
                                           TO *__restrict__ orow, float sc, int a,
                                           float2 *__restrict__ pscr) {
    const int s = P.stride[0];
    for (int o = threadIdx.x; o < s; o += blockDim.x) {
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = sm[phys(o + i * s)];
        if (o) {
            float2 W[R];
            tw_powers<R>(tw_base(tws, o), W);
#pragma unroll
            for (int i = 1; i < R; ++i) x[i] = twmul<false>(x[i], W[i]);
        }
        Dft<R, false>::run(x);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int f = o + k * s;
            float2 v = x[k];
            if (f & 1) v = make_float2(-v.x, -v.y);
            if (P.natural_out == 2) {
                // paired natural order: the even half waits in this CTA's
                // scratch row (written and read by the same thread), the odd
                // half's pass stores fine samples 2f, 2f + 1 together
                if (a == 0) pscr[f] = v;
                else st_pair(orow, f, pscr[f], v, sc);
            } else {
                st_cs(orow, P.natural_out ? 2 * f + a : a * P.L + f, v, sc);
            }
        }
    }
}

#define NUFDS_RADIX_SWITCH(R_, CALL)                   \
    switch (R_) {                                      \
        case 2: CALL(2); break;                        \
        case 3: CALL(3); break;                        \
        case 4: CALL(4); break;                        \
        case 5: CALL(5); break;                        \
        case 6: CALL(6); break;                        \
        case 8: CALL(8); break;                        \
        case 9: CALL(9); break;                        \
        case 10: CALL(10); break;                      \
        case 12: CALL(12); break;                      \
        case 15: CALL(15); break;                      \
        case 16: CALL(16); break;                      \
        default: break;                                \
    }

template <bool INV, bool DIT>
__device__ void mid_pass(const PassArgs &P, int j, float2 *sm, const float2 *tws) {
#define C_(R) mid_pass_r<R, INV, DIT>(P, j, sm, tws)
    NUFDS_RADIX_SWITCH(P.radix[j], C_)
#undef C_
}

template <class TO>
__device__ void forward_tail(const PassArgs &P, float2 *sm, const float2 *tws, TO *orow, float sc,
                             int a, float2 *pscr = nullptr) {
    for (int j = P.npass - 2; j >= 1; --j) {
        mid_pass<false, true>(P, j, sm, tws);
        __syncthreads();
    }
#define C_(R) dit_last_r<R, TO>(P, sm, tws, orow, sc, a, pscr)
    NUFDS_RADIX_SWITCH(P.radix[0], C_)
#undef C_
    __syncthreads();
}

// dynamic shared memory: padded row, then the twiddle tables
__device__ __forceinline__ float2 *load_tw(const PassArgs &P, float2 *sm) {
    float2 *tws = sm + phys(P.L) + 1;
    for (int i = threadIdx.x; i < 64 + P.ncoarse; i += blockDim.x) tws[i] = P.tw[i];
    __syncthreads();
    return tws;
}

template <class TI, class TO>
__global__ void __launch_bounds__(512) k_rows_pad2(PassArgs P, const TI *__restrict__ in,
                                                   long in_ld, TO *__restrict__ out, long out_ld,
                                                   int rows, const float *sc_in,
                                                   const float *sc_out, float2 *pair_scr) {
    extern __shared__ float2 sm[];
    const float2 *tws = load_tw(P, sm);
    const float inv = sc_in ? 1.0f / *sc_in : 1.0f, sc = sc_out ? *sc_out : 1.0f;
    const int RL = P.radix[P.npass - 1];
    float2 *pscr = pair_scr ? pair_scr + (long)blockIdx.x * P.L : nullptr;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const TI *irow = in + (long)r * in_ld;
        TO *orow = out + (long)r * out_ld;
        for (int a = 0; a < 2; ++a) {
#define C_(R) pad_first_r<R, TI>(P, irow, inv, sm, a)
            NUFDS_RADIX_SWITCH(RL, C_)
#undef C_
            __syncthreads();
            forward_tail<TO>(P, sm, tws, orow, sc, a, pscr);
        }
    }
}

// one row of the view pass: inverse DFT, chirp, the two half-grid forward DFTs
// (input elements outside [lo, hi) are zero)
template <class T>
__device__ __forceinline__ void row_view_body(const PassArgs &P, const T *__restrict__ irow,
                                              T *__restrict__ orow,
                                              const float2 *__restrict__ chirp_slot,
                                              float2 *__restrict__ scr, float2 *sm,
                                              const float2 *tws, float inv, float sc, int lo,
                                              int hi) {
    const int RL = P.radix[P.npass - 1];
    // inverse DFT (DIF): natural -> slot order
#define C_(R) dif_first_r<R, T>(P, irow, inv, sm, tws, lo, hi)
    NUFDS_RADIX_SWITCH(P.radix[0], C_)
#undef C_
    __syncthreads();
    for (int j = 1; j < P.npass - 1; ++j) {
        mid_pass<true, false>(P, j, sm, tws);
        __syncthreads();
    }
    // last inverse pass + chirp + first forward pass
#define C_(R) fused_mid_r<R>(P, sm, chirp_slot, scr)
    NUFDS_RADIX_SWITCH(RL, C_)
#undef C_
    __syncthreads();
    forward_tail<T>(P, sm, tws, orow, sc, 0);
#define C_(R) odd_first_r<R>(P, sm, scr, P.mod1_slot)
    NUFDS_RADIX_SWITCH(RL, C_)
#undef C_
    __syncthreads();
    forward_tail<T>(P, sm, tws, orow, sc, 1);
}

template <class T>
__global__ void __launch_bounds__(512) k_rows_view(PassArgs P, const T *__restrict__ in,
                                                   long in_ld,
                                                   const float2 *__restrict__ chirp_slot,
                                                   T *__restrict__ out, long out_ld, int rows,
                                                   float2 *__restrict__ scratch,
                                                   const float *sc_in, const float *sc_out,
                                                   int lo, int hi) {
    extern __shared__ float2 sm[];
    const float2 *tws = load_tw(P, sm);
    const float inv = sc_in ? 1.0f / *sc_in : 1.0f, sc = sc_out ? *sc_out : 1.0f;
    float2 *scr = scratch + (long)blockIdx.x * P.L;
    for (int r = blockIdx.x; r < rows; r += gridDim.x)
        row_view_body<T>(P, in + (long)r * in_ld, out + (long)r * out_ld, chirp_slot, scr, sm, tws,
                         inv, sc, lo, hi);
}

// Batched view pass over rows of many items (views, passes) of uneven length:
// a persistent grid walks the flattened row list (strided: contiguous chunks
// measured slower, rows of one length class still differ in length); the CTA
// reloads the pass structure and twiddle tables when it moves to another item.
template <class T>
__global__ void __launch_bounds__(512) k_rows_view_batch(const PassArgs *__restrict__ args,
                                                         const RowItem *__restrict__ items,
                                                         const int *__restrict__ row_off,
                                                         int nitems, float2 *__restrict__ scratch,
                                                         int scr_stride) {
    extern __shared__ float2 sm[];
    __shared__ PassArgs sP;
    float2 *scr = scratch + (long)blockIdx.x * scr_stride;
    const int total = row_off[nitems];
    int cur = -1, it = 0;
    const float2 *tws = nullptr;
    float inv = 1.0f, sc = 1.0f;
    for (int g = blockIdx.x; g < total; g += gridDim.x) {
        // the item of row g: rows only grow, so walk forward from the last one
        // (every thread alike; no barrier on the critical path)
        while (it + 1 < nitems && __ldg(row_off + it + 1) <= g) ++it;
        const RowItem &I = items[it];
        if (it != cur) {
            if (threadIdx.x == 0) sP = args[I.args];
            __syncthreads();
            tws = load_tw(sP, sm);
            inv = I.sc_in ? 1.0f / *I.sc_in : 1.0f;
            sc = I.sc_out ? *I.sc_out : 1.0f;
            cur = it;
        }
        const int r = g - row_off[it];
        row_view_body<T>(sP, (const T *)I.in + (long)r * I.in_ld, (T *)I.out + (long)r * I.out_ld,
                         I.chirp, scr, sm, tws, inv, sc, I.in_lo, I.in_hi);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------
// Split rows: one view-pass row over a cluster of two CTAs (rows longer than
// one CTA's shared memory holds).  With L the row length and L/2 the length
// each CTA transforms:
//   inverse: X[2k + c] = sum_{n < L/2} (x[n] + (-1)^c x[n + L/2]) W^{-cn}_L W^{-nk}_{L/2},
//            so CTA c folds the row on the way in (radix-2 step, pass 0 of
//            the decimation in frequency) and holds the odd or even outputs;
//   chirp:   pointwise (natural index 2k + c of its slots);
//   forward: X[k] = Z_0[k mod L/2] + W^k_L Z_1[k mod L/2], Z_c the half-length
//            DFT of CTA c's samples (times the odd-half modulation): each CTA
//            leaves Z_c in natural order in shared memory and computes its
//            half of the outputs from both, reading its partner's through
//            distributed shared memory (radix-2 step, pass 0 of the
//            decimation in time).
// ------------------------------------------------------------------------
__device__ __forceinline__ float2 twl_at(const float2 *twl, int n) {  // W_L^n, n < L/2
    return cmul(twl[64 + (n >> 6)], twl[n & 63]);
}

template <int R, class TI>
__device__ __forceinline__ void dif_first_split_r(const PassArgs &P, const TI *__restrict__ irow,
                                                  float inv, float2 *sm, const float2 *tws,
                                                  const float2 *twl, int c, int lo, int hi) {
    const int s = P.stride[0], Lh = P.L;
    const float2 zero = make_float2(0.f, 0.f);
    for (int o = threadIdx.x; o < s; o += blockDim.x) {
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int n = o + i * s;
            const float2 x0 = n >= lo && n < hi ? ld_cs(irow, n, inv) : zero;
            const float2 x1 = n + Lh >= lo && n + Lh < hi ? ld_cs(irow, n + Lh, inv) : zero;
            x[i] = c ? cmulc(csub(x0, x1), twl_at(twl, n)) : cadd(x0, x1);
        }
        Dft<R, true>::run(x);
        if (o) {
            float2 W[R];
            tw_powers<R>(tw_base(tws, o), W);
#pragma unroll
            for (int k = 1; k < R; ++k) x[k] = twmul<true>(x[k], W[k]);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) sm[phys(o + k * s)] = x[k];
    }
}

// last forward DIT pass kept in shared memory: natural-order outputs
template <int R>
__device__ __forceinline__ void dit_last_smem_r(const PassArgs &P, float2 *sm, const float2 *tws) {
    const int s = P.stride[0];
    for (int o = threadIdx.x; o < s; o += blockDim.x) {
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = sm[phys(o + i * s)];
        if (o) {
            float2 W[R];
            tw_powers<R>(tw_base(tws, o), W);
#pragma unroll
            for (int i = 1; i < R; ++i) x[i] = twmul<false>(x[i], W[i]);
        }
        Dft<R, false>::run(x);
#pragma unroll
        for (int k = 0; k < R; ++k) sm[phys(o + k * s)] = x[k];
    }
}

__device__ void forward_tail_smem(const PassArgs &P, float2 *sm, const float2 *tws) {
    for (int j = P.npass - 2; j >= 1; --j) {
        mid_pass<false, true>(P, j, sm, tws);
        __syncthreads();
    }
#define C_(R) dit_last_smem_r<R>(P, sm, tws)
    NUFDS_RADIX_SWITCH(P.radix[0], C_)
#undef C_
}

// outputs k = c L/2 + k' of half a: (-1)^k (Z_0[k'] + W_L^k Z_1[k']), W_L^{L/2} = -1,
// stored in the plane layout at a L + k
template <class TO>
__device__ __forceinline__ void split_combine(const PassArgs &P, const float2 *sm,
                                              const float2 *peer, const float2 *twl, int c,
                                              TO *__restrict__ orow, float sc, int a) {
    const int Lh = P.L;
    for (int k = threadIdx.x; k < Lh; k += blockDim.x) {
        const float2 zo = sm[phys(k)], zp = peer[phys(k)];
        const float2 z0 = c ? zp : zo, z1 = c ? zo : zp;
        float2 t = cmul(z1, twl_at(twl, k));
        if (c) t = make_float2(-t.x, -t.y);
        float2 v = cadd(z0, t);
        const int f = c * Lh + k;
        if (f & 1) v = make_float2(-v.x, -v.y);
        st_cs(orow, (long)a * P.Lfull + f, v, sc);
    }
}

template <class T>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512)
    k_rows_view_split(PassArgs P, const T *__restrict__ in, long in_ld,
                      const float2 *__restrict__ chirp_slot, T *__restrict__ out, long out_ld,
                      int rows, float2 *__restrict__ scratch, const float *sc_in,
                      const float *sc_out, int lo, int hi) {
    extern __shared__ float2 sm[];
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const float2 *peer = cl.map_shared_rank(sm, c ^ 1);
    const float2 *tws = load_tw(P, sm);
    float2 *twl = sm + phys(P.L) + 1 + 64 + P.ncoarse;
    for (int i = threadIdx.x; i < 64 + (P.L + 63) / 64; i += blockDim.x) twl[i] = P.twL[i];
    __syncthreads();
    const float inv = sc_in ? 1.0f / *sc_in : 1.0f, sc = sc_out ? *sc_out : 1.0f;
    float2 *scr = scratch + (long)blockIdx.x * P.L;
    const float2 *chirp = chirp_slot + (long)c * P.L, *mod = P.mod1_slot + (long)c * P.L;
    const int RL = P.radix[P.npass - 1];
    for (int r = blockIdx.x >> 1; r < rows; r += gridDim.x >> 1) {
        const T *irow = in + (long)r * in_ld;
        T *orow = out + (long)r * out_ld;
#define C_(R) dif_first_split_r<R, T>(P, irow, inv, sm, tws, twl, c, lo, hi)
        NUFDS_RADIX_SWITCH(P.radix[0], C_)
#undef C_
        __syncthreads();
        for (int j = 1; j < P.npass - 1; ++j) {
            mid_pass<true, false>(P, j, sm, tws);
            __syncthreads();
        }
#define C_(R) fused_mid_r<R>(P, sm, chirp, scr)
        NUFDS_RADIX_SWITCH(RL, C_)
#undef C_
        __syncthreads();
        forward_tail_smem(P, sm, tws);
        cl.sync();
        split_combine<T>(P, sm, peer, twl, c, orow, sc, 0);
        cl.sync();
#define C_(R) odd_first_r<R>(P, sm, scr, mod)
        NUFDS_RADIX_SWITCH(RL, C_)
#undef C_
        __syncthreads();
        forward_tail_smem(P, sm, tws);
        cl.sync();
        split_combine<T>(P, sm, peer, twl, c, orow, sc, 1);
        cl.sync();
    }
}

// Padded forward pass of a split row (the hologram's passes when N > kMaxRowL):
// CTA c transforms the samples 2m + c (times the deapodisation and, for the
// odd half, the modulation), then the halves combine as in split_combine.
template <int R, class TI>
__device__ __forceinline__ void pad_first_split_r(const PassArgs &P, const TI *__restrict__ irow,
                                                  float inv, float2 *sm, int a, int c) {
    const int nb = P.L / R;
    for (int n = threadIdx.x; n < nb; n += blockDim.x) {
        float2 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int m = 2 * (n + i * nb) + c;
            float2 v = cscale(ld_cs(irow, m, inv), __ldg(P.pad_pre + m));
            x[i] = a ? cmul(v, __ldg(P.mod1 + m)) : v;
        }
        Dft<R, false>::run(x);
        uint32_t q = n;
        int base = 0;
        for (int j = 0; j < P.npass - 1; ++j) {
            uint32_t q2 = udiv(q, P.mag_radix[j]);
            base += (int)(q - q2 * P.radix[j]) * P.stride[j];
            q = q2;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) sm[phys(base + k)] = x[k];
    }
}

// outputs k = c L/2 + k' of half a of a split padded row, (-1)^k (Z_0[k'] +
// W_L^k Z_1[k']), in the layout P.natural_out selects (2: the even half waits
// in pscr, this CTA's L/2 entries, and each fine pair is stored together)
template <class TO>
__device__ __forceinline__ void split_combine_pad(const PassArgs &P, const float2 *sm,
                                                  const float2 *peer, const float2 *twl, int c,
                                                  TO *__restrict__ orow, float sc, int a,
                                                  float2 *__restrict__ pscr) {
    const int Lh = P.L;
    for (int k = threadIdx.x; k < Lh; k += blockDim.x) {
        const float2 zo = sm[phys(k)], zp = peer[phys(k)];
        const float2 z0 = c ? zp : zo, z1 = c ? zo : zp;
        float2 t = cmul(z1, twl_at(twl, k));
        if (c) t = make_float2(-t.x, -t.y);
        float2 v = cadd(z0, t);
        const long f = (long)c * Lh + k;
        if (f & 1) v = make_float2(-v.x, -v.y);
        if (P.natural_out == 2) {
            if (a == 0) pscr[k] = v;
            else st_pair(orow, f, pscr[k], v, sc);
        } else {
            st_cs(orow, P.natural_out ? 2 * f + a : a * P.Lfull + f, v, sc);
        }
    }
}

template <class TI, class TO>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512)
    k_rows_pad2_split(PassArgs P, const TI *__restrict__ in, long in_ld, TO *__restrict__ out,
                      long out_ld, int rows, const float *sc_in, const float *sc_out,
                      float2 *pair_scr) {
    extern __shared__ float2 sm[];
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const float2 *peer = cl.map_shared_rank(sm, c ^ 1);
    const float2 *tws = load_tw(P, sm);
    float2 *twl = sm + phys(P.L) + 1 + 64 + P.ncoarse;
    for (int i = threadIdx.x; i < 64 + (P.L + 63) / 64; i += blockDim.x) twl[i] = P.twL[i];
    __syncthreads();
    const float inv = sc_in ? 1.0f / *sc_in : 1.0f, sc = sc_out ? *sc_out : 1.0f;
    const int RL = P.radix[P.npass - 1];
    float2 *pscr = pair_scr ? pair_scr + (long)blockIdx.x * P.L : nullptr;
    for (int r = blockIdx.x >> 1; r < rows; r += gridDim.x >> 1) {
        const TI *irow = in + (long)r * in_ld;
        TO *orow = out + (long)r * out_ld;
        for (int a = 0; a < 2; ++a) {
#define C_(R) pad_first_split_r<R, TI>(P, irow, inv, sm, a, c)
            NUFDS_RADIX_SWITCH(RL, C_)
#undef C_
            __syncthreads();
            forward_tail_smem(P, sm, tws);
            cl.sync();
            split_combine_pad<TO>(P, sm, peer, twl, c, orow, sc, a, pscr);
            cl.sync();
        }
    }
}

// ------------------------------------------------------------------------
// host side: plans and tables
// ------------------------------------------------------------------------
static const int kRadices[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

static int host_phys(int p) { return p + (p >> 4) + (p >> 8); }

// all multisets of radices (non-increasing) with the fewest factors
static void factor_sets(int L, std::vector<int> &cur, std::vector<std::vector<int>> &out,
                        int &best) {
    if (L == 1) {
        if ((int)cur.size() < best) {
            best = (int)cur.size();
            out.clear();
        }
        if ((int)cur.size() == best) out.push_back(cur);
        return;
    }
    if ((int)cur.size() >= best || (int)cur.size() >= kMaxPasses) return;
    for (int r : kRadices) {
        if (L % r || (!cur.empty() && r > cur.back())) continue;
        cur.push_back(r);
        factor_sets(L / r, cur, out, best);
        cur.pop_back();
    }
}

// shared-memory wavefronts of one warp access (8-byte elements, 32 banks)
static int waves(const int *slots, int n) {
    int cnt[32];
    int words[32][64];
    for (int b = 0; b < 32; ++b) cnt[b] = 0;
    int worst = 0;
    for (int t = 0; t < n; ++t) {
        int ph = host_phys(slots[t]);
        for (int w = 2 * ph; w <= 2 * ph + 1; ++w) {
            int b = w & 31, seen = 0;
            for (int k = 0; k < cnt[b]; ++k) seen |= words[b][k] == w;
            if (!seen && cnt[b] < 64) words[b][cnt[b]++] = w;
            if (cnt[b] > worst) worst = cnt[b];
        }
    }
    return worst;
}

// bank-conflict cost of a radix order: middle passes and the padded-pass scatter
static double order_cost(const std::vector<int> &rad) {
    const int P = (int)rad.size();
    int L = 1;
    for (int r : rad) L *= r;
    std::vector<int> st(P);
    int rem = L;
    for (int j = 0; j < P; ++j) st[j] = (rem /= rad[j]);
    double sum = 0, mx = 0;
    int slots[32];
    for (int j = 1; j < P; ++j) {
        const int R = rad[j], B = R * st[j];
        double w = 0;
        for (int i = 0; i < R; ++i) {
            for (int t = 0; t < 32; ++t) slots[t] = (t / st[j]) * B + t % st[j] + i * st[j];
            w += waves(slots, 32);
        }
        w /= 2.0 * R;
        sum += w;
        mx = std::max(mx, w);
    }
    const int R = rad[P - 1];
    double w = 0;
    for (int k = 0; k < R; ++k) {
        for (int t = 0; t < 32; ++t) {
            int q = t, p = 0;
            for (int j = 0; j < P - 1; ++j) {
                p += (q % rad[j]) * st[j];
                q /= rad[j];
            }
            slots[t] = p + k;
        }
        w += waves(slots, 32);
    }
    w /= 2.0 * R;
    return sum + w + std::max(mx, w);
}

static bool choose_radices(int L, FftPlan &p) {
    std::vector<int> cur;
    std::vector<std::vector<int>> sets;
    int best = kMaxPasses + 1;
    factor_sets(L, cur, sets, best);
    if (sets.empty() || best < 2) return false;
    // lowest bank-conflict cost; among equal costs the most balanced radices
    // (smallest sum of squares: fewer values live in registers in the largest
    // passes), then the smallest first radix.  Measured over every minimum-
    // pass order of 23040 and 16384, this picks the fastest order of each
    // (10 x 12 x 12 x 16: view passes 20.54 ms against 21.31 ms for the first
    // equal-cost order found; 8 x 8 x 16 x 16 for the spectrum passes).
    auto sq = [](const std::vector<int> &r) {
        int m = 0;
        for (int x : r) m += x * x;
        return m;
    };
    double bc = 1e30;
    std::vector<int> bo;
    for (auto &m : sets) {
        std::vector<int> perm = m;
        std::sort(perm.begin(), perm.end());
        do {
            double c = order_cost(perm);
            const bool better =
                c < bc - 1e-9 ||
                (c < bc + 1e-9 &&
                 (sq(perm) < sq(bo) || (sq(perm) == sq(bo) && perm[0] < bo[0])));
            if (better) {
                bc = c;
                bo = perm;
            }
        } while (std::next_permutation(perm.begin(), perm.end()));
    }
    p.L = L;
    p.npass = (int)bo.size();
    int pre = 1, rem = L;
    for (int j = 0; j < p.npass; ++j) {
        p.radix[j] = bo[j];
        p.prefix[j] = pre;
        pre *= bo[j];
        rem /= bo[j];
        p.stride[j] = rem;
    }
    return true;
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

static std::mutex g_mu;
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

// Plan of length L and its host tables:
//   f2: fine[64] | coarse[ncoarse] | mod1[L] | mod1_slot[L] [| twL fine[64] | twL coarse[ncl]];
//   dea[L]; pad[L]
// (for a split row the twiddles fine/coarse are those of the half length, and
// twL holds W_L^n, n < L/2, for the radix-2 steps between the halves)
static int split_ncoarse(int L) { return fft_needs_split(L) ? (L / 2 + 63) / 64 : 0; }

static int plan_host(int L, FftPlan &p, std::vector<float2> &f2, std::vector<double> &dea,
                     std::vector<float> &pad) {
    if (L < 64 || (L % 4)) return -3;
    const int split = fft_needs_split(L) ? 2 : 1, Lh = L / split;
    if ((Lh % 4) || Lh < 64 || !choose_radices(Lh, p)) return -3;
    p.L = L;
    p.split = split;
    int t = (Lh / 16 + 31) / 32 * 32;
    p.threads = t < 64 ? 64 : (t > 512 ? 512 : t);
    p.pad_threads = p.threads;
    p.ncoarse = (Lh + 63) / 64;
    const int ncl = split_ncoarse(L);
    p.smem_bytes = sizeof(float2) * (size_t)(host_phys(Lh) + 1 + 64 + p.ncoarse +
                                             (split == 2 ? 64 + ncl : 0));
    if (p.smem_bytes > 227 * 1024 - 1024) return -3;
    // a split row whose halves fit two CTAs per SM: blocks small enough that
    // two of them also fit the register file
    if (split == 2 && 2 * (p.smem_bytes + 1024) <= 227 * 1024) p.threads = p.pad_threads = 256;
    f2.assign(fft_tw_count(L), make_float2(0.f, 0.f));
    for (int j = 0; j < 64; ++j) {
        double a = -2.0 * M_PI * j / Lh;
        f2[j] = make_float2((float)cos(a), (float)sin(a));
    }
    for (int i = 0; i < p.ncoarse; ++i) {
        double a = -2.0 * M_PI * (double)(64L * i % Lh) / Lh;
        f2[64 + i] = make_float2((float)cos(a), (float)sin(a));
    }
    float2 *mod1 = f2.data() + 64 + p.ncoarse, *mod1s = mod1 + L;
    for (int n = 0; n < L; ++n) {
        double a = -M_PI * (n - L / 2) / (double)L;
        mod1[n] = make_float2((float)cos(a), (float)sin(a));
    }
    for (int q = 0; q < L; ++q) mod1s[fft_gm_pos(p, q)] = mod1[fft_index_of_slot(p, q)];
    if (split == 2) {
        float2 *tl = mod1s + L;
        for (int j = 0; j < 64; ++j) {
            double a = -2.0 * M_PI * j / L;
            tl[j] = make_float2((float)cos(a), (float)sin(a));
        }
        for (int i = 0; i < ncl; ++i) {
            double a = -2.0 * M_PI * (double)(64L * i) / L;
            tl[64 + i] = make_float2((float)cos(a), (float)sin(a));
        }
    }
    std::vector<double> ft;
    es_fourier(L, ft);
    dea.resize(L);
    pad.resize(L);
    p.dmax = 0;
    for (int n = 0; n < L; ++n) {
        dea[n] = 1.0 / ft[n];
        pad[n] = (float)((n & 1) ? -dea[n] : dea[n]);
        p.dmax = std::max(p.dmax, fabs(dea[n]));
    }
    return 0;
}

static void plan_point(FftPlan &p, const float2 *tw, const double *dea, const float *pad) {
    p.tw = tw;
    p.mod1 = tw + 64 + p.ncoarse;
    p.mod1_slot = p.mod1 + p.L;
    p.twL = p.split == 2 ? p.mod1_slot + p.L : nullptr;
    p.deapod = dea;
    p.pad_pre = pad;
}

struct LenEntry {
    FftPlan plan;
    float2 *dev = nullptr;
    double *deapod = nullptr;
    float *pad_pre = nullptr;
};
static std::map<std::pair<int, int>, LenEntry *> g_cache;  // (device, L)

static void set_smem_attrs(size_t bytes);

static int grid_for(const void *fn, const FftPlan &p, int rows);

// Autotuner of the row passes: time the view pass and the padded pass with
// each candidate block size on zeroed buffers and keep the fastest of each
// (per device and length, once).  The probe gives every resident CTA four rows, so it measures
// the steady state rather than a one-row tail.  Falls back to the default on
// any failure.
static void autotune_threads(FftPlan &p) {
    const int L = p.L;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_rows_view<float2>, 128,
                                                  p.smem_bytes);
    const long cap = (512L << 20) / (24L * L);  // in + 2x out + scratch under ~512 MB
    const int rows = (int)std::max(1L, std::min(4L * std::max(sms, 1) * std::max(per, 1), cap));
    int cands[5] = {128, 192, 256, 384, 512}, best_t = p.threads, best_pad = p.pad_threads;
    float best = 1e30f;
    float2 *in = nullptr, *out = nullptr, *scr = nullptr, *chirp = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t nin = (size_t)rows * L, nout = 2 * nin;
    bool ok = cudaMalloc(&in, nin * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&out, nout * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&chirp, (size_t)L * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&scr, (size_t)rows * L * sizeof(float2)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (ok) {
        cudaMemsetAsync(in, 0, nin * sizeof(float2), st);
        cudaMemsetAsync(chirp, 0, (size_t)L * sizeof(float2), st);
        const PassArgs a = fft_pass_args(p);
        for (int kind = 0; kind < 2; ++kind) {  // 0: view pass, 1: padded pass
            best = 1e30f;
            for (int t : cands) {
                if (t < 64 || t > 512) continue;
                FftPlan q = p;
                q.threads = t;
                const void *fn = kind == 0 ? (const void *)k_rows_view<float2>
                                           : (const void *)k_rows_pad2<float2, float2>;
                const int grid = grid_for(fn, q, rows);
                for (int rep = 0; rep < 4; ++rep) {
                    if (rep == 1) cudaEventRecord(e0, st);
                    if (kind == 0)
                        k_rows_view<float2><<<grid, t, p.smem_bytes, st>>>(
                            a, in, L, chirp, out, 2 * L, rows, scr, nullptr, nullptr, 0, L);
                    else
                        k_rows_pad2<float2, float2><<<grid, t, p.smem_bytes, st>>>(
                            a, in, L, out, 2 * L, rows, nullptr, nullptr, nullptr);
                }
                cudaEventRecord(e1, st);
                float ms = 0;
                const bool timed = cudaEventSynchronize(e1) == cudaSuccess &&
                                   cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
                if (getenv("NUFDS_DEBUG"))
                    fprintf(stderr, "nufds: autotune L=%d %s threads=%d: %.4f ms (%d rows)\n", L,
                            kind == 0 ? "view" : "pad", t, timed ? ms / 3 : -1.0f, rows);
                if (timed && ms < best) {
                    best = ms;
                    (kind == 0 ? best_t : best_pad) = t;
                }
            }
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(in);
    cudaFree(out);
    cudaFree(chirp);
    cudaFree(scr);
    p.threads = best_t;
    p.pad_threads = best_pad;
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
    LenEntry *e = new LenEntry();
    std::vector<float2> f2;
    std::vector<double> dea;
    std::vector<float> pad;
    if ((rc = plan_host(L, e->plan, f2, dea, pad))) {
        delete e;
        return rc;
    }
    if (cudaMalloc(&e->dev, sizeof(float2) * f2.size()) != cudaSuccess ||
        cudaMalloc(&e->deapod, sizeof(double) * L) != cudaSuccess ||
        cudaMalloc(&e->pad_pre, sizeof(float) * L) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(e->dev);
        cudaFree(e->deapod);
        delete e;
        return -2;
    }
    cudaMemcpy(e->dev, f2.data(), sizeof(float2) * f2.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(e->deapod, dea.data(), sizeof(double) * L, cudaMemcpyHostToDevice);
    cudaMemcpy(e->pad_pre, pad.data(), sizeof(float) * L, cudaMemcpyHostToDevice);
    plan_point(e->plan, e->dev, e->deapod, e->pad_pre);
    set_smem_attrs(e->plan.smem_bytes);
    if (e->plan.split == 1) autotune_threads(e->plan);  // split rows: the default block size
    g_cache[key] = e;
    *out = &e->plan;
    return 0;
}

// Plan and tables of length L written into caller-provided device memory (no
// allocation): d_tw holds fft_tw_count(L) float2, d_deapod L doubles, d_pad L
// floats.  Tables are computed on the host in FP64 and copied on st.
int fft_plan_fill(int L, FftPlan *p, float2 *d_tw, double *d_deapod, float *d_pad,
                  cudaStream_t st) {
    std::vector<float2> f2;
    std::vector<double> dea;
    std::vector<float> pad;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        int rc = init_constants();
        if (rc) return rc;
        *p = FftPlan();
        if ((rc = plan_host(L, *p, f2, dea, pad))) return rc;
    }
    if (p->smem_bytes > 48 * 1024) return -3;
    if (cudaMemcpyAsync(d_tw, f2.data(), sizeof(float2) * f2.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_deapod, dea.data(), sizeof(double) * L, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_pad, pad.data(), sizeof(float) * L, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return -4;
    // pageable sources: keep them alive until the copies have been consumed
    if (cudaStreamSynchronize(st) != cudaSuccess) return -4;
    plan_point(*p, d_tw, d_deapod, d_pad);
    return 0;
}

size_t fft_tw_count(int L) {
    const int ncl = split_ncoarse(L), Lh = ncl ? L / 2 : L;
    return 64 + (size_t)(Lh + 63) / 64 + 2 * (size_t)L + (ncl ? 64 + (size_t)ncl : 0);
}

PassArgs fft_pass_args(const FftPlan &p) {
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.L = p.L / p.split;
    a.Lfull = p.L;
    a.twL = p.twL;
    a.npass = p.npass;
    a.ncoarse = p.ncoarse;
    for (int j = 0; j < p.npass; ++j) {
        a.radix[j] = p.radix[j];
        a.stride[j] = p.stride[j];
        a.mag_stride[j] = p.stride[j] == 1 ? 0u : (uint32_t)(((1ull << 32) + p.stride[j] - 1) / p.stride[j]);
        a.mag_radix[j] = (uint32_t)(((1ull << 32) + p.radix[j] - 1) / p.radix[j]);
    }
    a.tw = p.tw;
    a.mod1 = p.mod1;
    a.mod1_slot = p.mod1_slot;
    a.pad_pre = p.pad_pre;
    return a;
}

static void set_smem_attrs(size_t bytes) {
    if (bytes > 48 * 1024) {
        const int m = 227 * 1024 - 1024;  // leave room for static shared memory
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaFuncSetAttribute(k_rows_pad2<float2, float2>, a, m);
        cudaFuncSetAttribute(k_rows_pad2<float2, __half2>, a, m);
        cudaFuncSetAttribute(k_rows_pad2<float2, __nv_bfloat162>, a, m);
        cudaFuncSetAttribute(k_rows_pad2<__half2, __half2>, a, m);
        cudaFuncSetAttribute(k_rows_pad2<__nv_bfloat162, __nv_bfloat162>, a, m);
        cudaFuncSetAttribute(k_rows_view<float2>, a, m);
        cudaFuncSetAttribute(k_rows_view<__half2>, a, m);
        cudaFuncSetAttribute(k_rows_view<__nv_bfloat162>, a, m);
        cudaFuncSetAttribute(k_rows_view_batch<float2>, a, m);
        cudaFuncSetAttribute(k_rows_view_batch<__half2>, a, m);
        cudaFuncSetAttribute(k_rows_view_batch<__nv_bfloat162>, a, m);
        cudaFuncSetAttribute(k_rows_view_split<float2>, a, m);
        cudaFuncSetAttribute(k_rows_pad2_split<float2, float2>, a, m);
        cudaFuncSetAttribute(k_rows_pad2_split<float2, __half2>, a, m);
        cudaFuncSetAttribute(k_rows_pad2_split<float2, __nv_bfloat162>, a, m);
        cudaFuncSetAttribute(k_rows_pad2_split<__half2, __half2>, a, m);
        cudaFuncSetAttribute(k_rows_pad2_split<__nv_bfloat162, __nv_bfloat162>, a, m);
        cudaFuncSetAttribute(k_rows_view_split<__half2>, a, m);
        cudaFuncSetAttribute(k_rows_view_split<__nv_bfloat162>, a, m);
    }
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

int rows_view_grid(const FftPlan &p, int rows) {
    if (p.split == 1) return grid_for((const void *)k_rows_view<float2>, p, rows);
    // two CTAs per row: an even grid of at most the resident CTAs
    int dev, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_rows_view_split<float2>,
                                                  p.threads, p.smem_bytes);
    long g = (long)sms * (per < 1 ? 1 : per);
    g = std::min(g, 2L * rows);
    return (int)std::max(2L, g & ~1L);
}

int launch_rows_pad2(const FftPlan &p, const void *in, int in_prec, long in_ld, void *out,
                     int prec, long out_ld, int rows, const float *sc_in, const float *sc_out,
                     cudaStream_t st, int natural_out, const float *pre, float2 *pair_scr,
                     size_t pair_cap) {
    if (rows <= 0) return 0;
    FftPlan q = p;
    q.threads = p.pad_threads;
    int grid;
    if (p.split == 2) {  // two CTAs per row: an even grid of at most the resident CTAs
        int dev, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per, (const void *)k_rows_pad2_split<float2, float2>, q.threads, p.smem_bytes);
        long g = std::min((long)sms * (per < 1 ? 1 : per), 2L * rows);
        grid = (int)std::max(2L, g & ~1L);
    } else {
        grid = grid_for((const void *)k_rows_pad2<float2, float2>, q, rows);
    }
    PassArgs a = fft_pass_args(p);
    a.natural_out = natural_out;
    if (pre) a.pad_pre = pre;
    if (!natural_out || (size_t)grid * p.L > pair_cap) pair_scr = nullptr;
    if (pair_scr) a.natural_out = 2;
    if (p.split == 2) {
#define L_(TI, TO)                                                                         \
    k_rows_pad2_split<TI, TO><<<grid, q.threads, p.smem_bytes, st>>>(                      \
        a, (const TI *)in, in_ld, (TO *)out, out_ld, rows, sc_in, sc_out, pair_scr)
        if (in_prec == PREC_F32 && prec == PREC_F32) L_(float2, float2);
        else if (in_prec == PREC_F32 && prec == PREC_F16) L_(float2, __half2);
        else if (in_prec == PREC_F32 && prec == PREC_BF16) L_(float2, __nv_bfloat162);
        else if (in_prec == PREC_F16 && prec == PREC_F16) L_(__half2, __half2);
        else if (in_prec == PREC_BF16 && prec == PREC_BF16) L_(__nv_bfloat162, __nv_bfloat162);
        else return -3;
#undef L_
        count_launch();
        return check_launch();
    }
#define L_(TI, TO)                                                                        \
    k_rows_pad2<TI, TO><<<grid, q.threads, p.smem_bytes, st>>>(a, (const TI *)in, in_ld,  \
                                                              (TO *)out, out_ld, rows,    \
                                                              sc_in, sc_out, pair_scr)
    if (in_prec == PREC_F32 && prec == PREC_F32) L_(float2, float2);
    else if (in_prec == PREC_F32 && prec == PREC_F16) L_(float2, __half2);
    else if (in_prec == PREC_F32 && prec == PREC_BF16) L_(float2, __nv_bfloat162);
    else if (in_prec == PREC_F16 && prec == PREC_F16) L_(__half2, __half2);
    else if (in_prec == PREC_BF16 && prec == PREC_BF16) L_(__nv_bfloat162, __nv_bfloat162);
    else return -3;
#undef L_
    count_launch();
    return check_launch();
}

int launch_rows_view(const FftPlan &p, const void *in, long in_ld, const float2 *chirp, void *out,
                     long out_ld, int rows, float2 *scratch, int grid, int prec,
                     const float *sc_in, const float *sc_out, cudaStream_t st, int in_lo,
                     int in_hi) {
    if (rows <= 0) return 0;
    in_lo = std::max(in_lo, 0);
    in_hi = std::min(in_hi, p.L);
    const PassArgs a = fft_pass_args(p);
    if (p.split == 2) {
        if (grid & 1) return -3;
#define L_(T)                                                                              \
    k_rows_view_split<T><<<grid, p.threads, p.smem_bytes, st>>>(a, (const T *)in, in_ld,   \
                                                               chirp, (T *)out, out_ld,    \
                                                               rows, scratch, sc_in, sc_out, \
                                                               in_lo, in_hi)
        if (prec == PREC_F32) L_(float2);
        else if (prec == PREC_F16) L_(__half2);
        else if (prec == PREC_BF16) L_(__nv_bfloat162);
        else return -3;
#undef L_
        count_launch();
        return check_launch();
    }
#define L_(T)                                                                               \
    k_rows_view<T><<<grid, p.threads, p.smem_bytes, st>>>(a, (const T *)in, in_ld, chirp,   \
                                                         (T *)out, out_ld, rows, scratch,   \
                                                         sc_in, sc_out, in_lo, in_hi)
    if (prec == PREC_F32) L_(float2);
    else if (prec == PREC_F16) L_(__half2);
    else if (prec == PREC_BF16) L_(__nv_bfloat162);
    else return -3;
#undef L_
    count_launch();
    return check_launch();
}

// ------------------------------------------------------------------------
// transpose
// ------------------------------------------------------------------------
// 32 x 32 tiles moved by 32 x kTrRows threads (eight elements each): measured
// against 8 and 16 rows and 64 x 64 tiles on the 16K workload (view transpose
// 3.19 -> 3.00 ms, spectrum transpose 1.59 -> 1.51 ms)
constexpr int kTrRows = 4;
template <class T>
__global__ void k_transpose(const T *__restrict__ in, long in_ld, T *__restrict__ out,
                            long out_ld, int rows, int cols) {
    __shared__ T tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += kTrRows) {
        int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[(long)r * in_ld + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += kTrRows) {
        int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(long)c * out_ld + r] = tile[threadIdx.x][i];
    }
}

int launch_transpose(const void *in, long in_ld, void *out, long out_ld, int rows, int cols,
                     int prec, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return 0;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    if (prec_bytes(prec) == 8)
        k_transpose<float2><<<grid, dim3(32, kTrRows), 0, st>>>((const float2 *)in, in_ld, (float2 *)out,
                                                          out_ld, rows, cols);
    else
        k_transpose<uint32_t><<<grid, dim3(32, kTrRows), 0, st>>>((const uint32_t *)in, in_ld,
                                                            (uint32_t *)out, out_ld, rows, cols);
    count_launch();
    return check_launch();
}

int rows_view_batch_grid(int threads, size_t smem, int total_rows) {
    int dev, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rows_view_batch<float2>, threads, smem);
    if (per < 1) per = 1;
    long g = (long)sms * per;
    return (int)(g < total_rows ? g : total_rows);
}

int launch_rows_view_batch(const PassArgs *d_args, const RowItem *d_items, const int *d_row_off,
                           int nitems, int total_rows, int threads, size_t smem, float2 *scratch,
                           int scr_stride, int grid, int prec, cudaStream_t st) {
    if (total_rows <= 0) return 0;
#define L_(T)                                                                             \
    k_rows_view_batch<T><<<grid, threads, smem, st>>>(d_args, d_items, d_row_off, nitems, \
                                                      scratch, scr_stride)
    if (prec == PREC_F32) L_(float2);
    else if (prec == PREC_F16) L_(__half2);
    else if (prec == PREC_BF16) L_(__nv_bfloat162);
    else return -3;
#undef L_
    count_launch();
    return check_launch();
}

template <class T>
__global__ void k_transpose_batch(const TrItem *__restrict__ items, const int *__restrict__ off,
                                  int nitems) {
    __shared__ T tile[32][33];
    __shared__ int s_item;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int lo = 0, hi = nitems - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_item = lo;
    }
    __syncthreads();
    const TrItem &I = items[s_item];
    const int t = blockIdx.x - off[s_item];
    const int c0 = (t % I.tiles_x) * 32, r0 = (t / I.tiles_x) * 32;
    const T *in = (const T *)I.in;
    T *out = (T *)I.out;
    for (int i = threadIdx.y; i < 32; i += kTrRows) {
        int r = r0 + i, c = c0 + threadIdx.x;
        if (r < I.rows && c < I.cols) tile[i][threadIdx.x] = in[(long)r * I.in_ld + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += kTrRows) {
        int c = c0 + i, r = r0 + threadIdx.x;
        if (r < I.rows && c < I.cols) out[(long)c * I.out_ld + r] = tile[threadIdx.x][i];
    }
}

int launch_transpose_batch(const TrItem *d_items, const int *d_tile_off, int nitems,
                           int total_tiles, int prec, cudaStream_t st) {
    if (total_tiles <= 0) return 0;
    if (prec_bytes(prec) == 8)
        k_transpose_batch<float2><<<total_tiles, dim3(32, kTrRows), 0, st>>>(d_items, d_tile_off, nitems);
    else
        k_transpose_batch<uint32_t><<<total_tiles, dim3(32, kTrRows), 0, st>>>(d_items, d_tile_off,
                                                                        nitems);
    count_launch();
    return check_launch();
}

// Weighted energies of the hologram for the FP16 scales of the padded passes:
// acc[0] += sum |h|^2 dx[ix]^2, acc[1] += sum |h|^2 dx[ix]^2 dy[iy]^2.  Terms in
// FP32, summed in FP32 over runs of kNormRun rows of a thread's kNormCols
// columns and in FP64 across runs (the scales need a bound, not an exact sum: k_scales_load
// widens it).  Block (x, y) takes the column chunk y (kNormCols per thread,
// 256 threads) of the rows x, x + gridDim.x, ...: the column weights are
// converted once per thread and each row issues kNormCols independent loads.
constexpr int kNormCols = 4;
constexpr int kNormThreads = 256;
constexpr int kNormRun = 16;
__global__ void __launch_bounds__(kNormThreads)
    k_norms(const float2 *__restrict__ H, int nx, int ny, const double *__restrict__ dx,
            const double *__restrict__ dy, double *acc) {
    const int c0 = blockIdx.y * kNormCols * kNormThreads + threadIdx.x;
    float w2[kNormCols];
#pragma unroll
    for (int j = 0; j < kNormCols; ++j) {
        const int ix = c0 + j * kNormThreads;
        const float w = ix < nx ? (float)dx[ix] : 0.f;
        w2[j] = w * w;
    }
    double s0 = 0, s1 = 0;
    float r0 = 0.f, r1 = 0.f;
    int k = 0;
    for (int iy = blockIdx.x; iy < ny; iy += gridDim.x) {
        const float2 *row = H + (long)iy * nx;
        float2 v[kNormCols];
#pragma unroll
        for (int j = 0; j < kNormCols; ++j) {
            const int ix = c0 + j * kNormThreads;
            v[j] = ix < nx ? __ldcs(row + ix) : make_float2(0.f, 0.f);
        }
        float r = 0.f;
#pragma unroll
        for (int j = 0; j < kNormCols; ++j) r = fmaf(fmaf(v[j].x, v[j].x, v[j].y * v[j].y), w2[j], r);
        const float wy = (float)dy[iy];
        r0 += r;
        r1 = fmaf(r, wy * wy, r1);
        if (++k == kNormRun) {  // FP32 runs of kNormRun rows, FP64 across runs
            s0 += r0;
            s1 += r1;
            r0 = r1 = 0.f;
            k = 0;
        }
    }
    s0 += r0;
    s1 += r1;
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, s0);
        atomicAdd(acc + 1, s1);
    }
}

__device__ __forceinline__ float energy4(uint4 u) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    const float2 c = __half22float2(*reinterpret_cast<const __half2 *>(&u.z));
    const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&u.w));
    return fmaf(a.x, a.x, a.y * a.y) + fmaf(b.x, b.x, b.y * b.y) + fmaf(c.x, c.x, c.y * c.y) +
           fmaf(d.x, d.x, d.y * d.y);
}

// ||S||^2 of the stretched band for the FP16 scales of the view passes, from
// the stored S (count elements held as S sc).  The body is read as 16-byte
// vectors (four per thread and iteration, independent), the unaligned head
// and the tail element by element; FP32 over runs of kNormRun iterations,
// FP64 across runs, one atomic per warp spread over kEnergySlots slots.
__global__ void k_energy(const __half2 *__restrict__ S, long count, const float *sc_s,
                         double *slots) {
    const float inv = 1.0f / *sc_s;
    const long head = min(count, (long)((4 - (((uintptr_t)S >> 2) & 3)) & 3));
    const long nvec = (count - head) >> 2, tail0 = head + 4 * nvec;
    const uint4 *V = reinterpret_cast<const uint4 *>(S + head);
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x, nth = (long)gridDim.x * blockDim.x;
    double s = 0;
    float r = 0.f;
    if (tid < head) {
        const float2 v = __half22float2(S[tid]);
        r = fmaf(v.x, v.x, fmaf(v.y, v.y, r));
    }
    if (tid < count - tail0) {
        const float2 v = __half22float2(S[tail0 + tid]);
        r = fmaf(v.x, v.x, fmaf(v.y, v.y, r));
    }
    s += r;
    long i = tid;
    int k = 0;
    r = 0.f;
    for (; i + 3 * nth < nvec; i += 4 * nth) {
        const uint4 a = __ldcs(V + i), b = __ldcs(V + i + nth), c = __ldcs(V + i + 2 * nth),
                    d = __ldcs(V + i + 3 * nth);
        r += (energy4(a) + energy4(b)) + (energy4(c) + energy4(d));
        if (++k == kNormRun) {  // FP32 runs of kNormRun iterations, FP64 across runs
            s += r;
            r = 0.f;
            k = 0;
        }
    }
    for (; i < nvec; i += nth) r += energy4(__ldcs(V + i));
    s += r;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0)
        atomicAdd(slots + ((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (kEnergySlots - 1)),
                  s * (double)inv * (double)inv);
}

int launch_energy(const void *S, long count, const float *sc_s, double *slots, cudaStream_t st) {
    if (cudaMemsetAsync(slots, 0, kEnergySlots * sizeof(double), st) != cudaSuccess) return -4;
    if (count <= 0) return 0;
    int dev, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long blocks = std::max(1L, std::min((long)sms * 4, (count / 4 + 255) / 256));
    k_energy<<<(int)blocks, 256, 0, st>>>((const __half2 *)S, count, sc_s, slots);
    count_launch();
    return check_launch();
}

int launch_norms(const float2 *H, int nx, int ny, const double *dx, const double *dy, double *acc,
                 cudaStream_t st) {
    if (cudaMemsetAsync(acc, 0, 4 * sizeof(double), st) != cudaSuccess) return -4;
    int dev, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int chunks = (nx + kNormCols * kNormThreads - 1) / (kNormCols * kNormThreads);
    const int rows = std::max(1, std::min(ny, sms * 8 / chunks + 1));
    k_norms<<<dim3(rows, chunks), kNormThreads, 0, st>>>(H, nx, ny, dx, dy, acc);
    count_launch();
    return check_launch();
}

__device__ __forceinline__ float pow2_scale(double bound) {
    // largest power of two s with s * bound <= 2^15
    if (!(bound > 0)) return 1.0f;
    int e = (int)floor(log2(32768.0 / bound));
    e = e > 100 ? 100 : (e < -100 ? -100 : e);
    return (float)ldexp(1.0, e);
}

// Parseval bounds (max |.| <= Frobenius norm):
//   |T1| <= sqrt(2 Nx) ||h dx||,  |G| <= 2 sqrt(Nx Ny) ||h dx dy||,  |S| <= K2 |G|
__global__ void k_scales_load(float *sc, const double *acc, int nx, int ny, double k2) {
    // the energies are sums of FP32 terms: widen by 1e-3 to keep the bounds
    const double bT1 = sqrt(2.0 * nx * acc[0] * 1.001);
    const double bG = 2.0 * sqrt((double)nx * ny * acc[1] * 1.001);
    sc[0] = pow2_scale(bT1);
    sc[1] = pow2_scale(bG);
    sc[2] = pow2_scale(k2 * bG);
}

//   |T_T| <= sqrt(2) dy' ||S||,  |Q| <= 2 dx' dy' ||S||  (||S||^2 in kEnergySlots parts)
__global__ void k_scales_view(float *sc, const double *acc, double dxp, double dyp) {
    double e = 0;
    for (int k = 0; k < kEnergySlots; ++k) e += acc[kEnergyAcc + k];
    const double nS = sqrt(e * 1.01);  // from FP16-rounded S, summed in FP32 runs: widened
    sc[3] = pow2_scale(sqrt(2.0) * dyp * nS);
    sc[4] = sc[3];
    sc[5] = pow2_scale(2.0 * dxp * dyp * nS);
}

int launch_scales_load(float *sc, const double *acc, int nx, int ny, double k2, cudaStream_t st) {
    k_scales_load<<<1, 1, 0, st>>>(sc, acc, nx, ny, k2);
    count_launch();
    return check_launch();
}

int launch_scales_view(float *sc, const double *acc, double dxp, double dyp, cudaStream_t st) {
    k_scales_view<<<1, 1, 0, st>>>(sc, acc, dxp, dyp);
    count_launch();
    return check_launch();
}

}  // namespace nufds
