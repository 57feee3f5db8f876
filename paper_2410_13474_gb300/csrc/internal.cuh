// Internal declarations shared by the CUDA sources of libnufds (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

namespace nufds {

// Interpolation kernel of the oversampled-grid resampling ("exponential of
// semicircle", Barnett, Magland & af Klinteberg, SIAM J. Sci. Comput. 2019):
//   psi(s) = exp(beta (sqrt(1 - (2 s / W)^2) - 1)),  |s| < W/2 fine cells.
// Oversampling 2 in each axis.
constexpr int kW = 8;
constexpr double kBeta = 2.30 * kW;
constexpr int kSigma = 2;

// Storage of the cached spectrum and the inter-pass arrays (arithmetic is FP32).
enum Prec { PREC_F32 = 0, PREC_F16 = 1, PREC_BF16 = 2 };
inline size_t prec_bytes(int prec) { return prec == PREC_F32 ? 8 : 4; }

// load/store of one complex sample in a storage type; FP16 samples are held
// multiplied by a power-of-two scale (sc on store, inv = 1/sc on load)
__device__ __forceinline__ float2 ld_c(const float2 *p, long i, float) { return __ldg(p + i); }
__device__ __forceinline__ float2 ld_c(const __half2 *p, long i, float inv) {
    float2 v = __half22float2(__ldg(p + i));
    return make_float2(v.x * inv, v.y * inv);
}
__device__ __forceinline__ float2 ld_c(const __nv_bfloat162 *p, long i, float) {
    return __bfloat1622float2(__ldg(p + i));
}
// streaming variants: data read or written once (keep L2 for reused data)
__device__ __forceinline__ float2 ld_cs(const float2 *p, long i, float) { return __ldcs(p + i); }
__device__ __forceinline__ float2 ld_cs(const __half2 *p, long i, float inv) {
    float2 v = __half22float2(__ldcs(p + i));
    return make_float2(v.x * inv, v.y * inv);
}
__device__ __forceinline__ float2 ld_cs(const __nv_bfloat162 *p, long i, float) {
    return __bfloat1622float2(__ldcs(p + i));
}
__device__ __forceinline__ void st_cs(float2 *p, long i, float2 v, float) { __stcs(p + i, v); }
__device__ __forceinline__ void st_cs(__half2 *p, long i, float2 v, float sc) {
    __stcs(p + i, __float22half2_rn(make_float2(v.x * sc, v.y * sc)));
}
__device__ __forceinline__ void st_cs(__nv_bfloat162 *p, long i, float2 v, float) {
    __stcs(p + i, __float22bfloat162_rn(v));
}
// A row on the 2x grid is stored as two planes: fine index m = 2k + a sits at
// a * L + k (L = unpadded length), so each half is written contiguously.
__device__ __forceinline__ int fine_pos(int m, int L) { return (m & 1) * L + (m >> 1); }

__device__ __forceinline__ void st_c(float2 *p, long i, float2 v, float) { p[i] = v; }
__device__ __forceinline__ void st_c(__half2 *p, long i, float2 v, float sc) {
    p[i] = __float22half2_rn(make_float2(v.x * sc, v.y * sc));
}
__device__ __forceinline__ void st_c(__nv_bfloat162 *p, long i, float2 v, float) {
    p[i] = __float22bfloat162_rn(v);
}

// Entry of a coordinate table: a point on a fine (2x oversampled) grid as
// centred integer base (floor of 2t, in the pull-back table as its offset
// from 2k) and fraction in [0, 1).  base.x == kMasked marks a point that is
// zeroed.
constexpr int16_t kMasked = -32768;

// ---------------------------------------------------------------------------
// Row FFT passes (fft_rows.cu)
// ---------------------------------------------------------------------------
constexpr int kMaxPasses = 8;

// Rows longer than kMaxRowL points do not fit one CTA's shared memory; such a
// row is split over a cluster of two CTAs (split = 2): a radix-2 step on the
// way in (inverse) and out (forward), a half-length transform of L / 2 points
// in each CTA, and the halves exchanged through distributed shared memory.
// The pass structure (npass, radix, stride, prefix, ncoarse, tw) is then that
// of the half-length transform; L, deapod, pad_pre and mod1 stay full length.
constexpr int kMaxRowL = 24576;
inline bool fft_needs_split(int L) { return L > kMaxRowL; }

struct FftPlan {
    int L = 0;
    int split = 1;                     // 2: the row is split over a 2-CTA cluster
    int npass = 0;
    int radix[kMaxPasses] = {};
    int stride[kMaxPasses] = {};   // s_j = L / (r_1 ... r_j)
    int prefix[kMaxPasses] = {};   // r_1 ... r_{j-1}
    int threads = 0;                   // block size of the view passes
    int pad_threads = 0;               // block size of the padded (spectrum) passes
    int ncoarse = 0;                   // ceil(L / 64)
    double dmax = 0;                   // max_n 1 / psi_hat(n - L/2)
    size_t smem_bytes = 0;
    // device tables (owned by the length cache, or caller memory)
    const float2 *tw = nullptr;        // W_L^j (j < 64) | W_L^{64 i} (i < ncoarse)
    const float2 *mod1 = nullptr;      // e^{-i pi (n - L/2)/L}, natural order
    const float2 *mod1_slot = nullptr; // the same per slot, group-major order (fft_gm_pos)
    const double *deapod = nullptr;    // 1 / psi_hat(n - L/2)
    const float *pad_pre = nullptr;    // (-1)^n / psi_hat(n - L/2)
    const float2 *twL = nullptr;       // split rows: W_L^j (j < 64) | W_L^{64 i} (i < ncoarse)
};

struct PassArgs {
    int L, npass, ncoarse;            // of the (half-length, for split rows) transform
    int radix[kMaxPasses], stride[kMaxPasses];
    uint32_t mag_stride[kMaxPasses];  // ceil(2^32 / stride), 0 for stride 1
    uint32_t mag_radix[kMaxPasses];   // ceil(2^32 / radix)
    const float2 *tw;                 // fine[64] | coarse[ncoarse]: W_L^q = coarse[q>>6] fine[q&63]
    const float2 *mod1, *mod1_slot;   // e^{-i pi (n - L/2)/L}: natural / per slot, group-major
    const float *pad_pre;             // (-1)^n / psi_hat(n - L/2), natural order
    int natural_out;                  // padded output: 0 plane-wise (a L + k), 1 natural (2k + a),
                                      // 2 natural, stored in pairs through a scratch row
    int Lfull;                        // row length (2 L for split rows)
    const float2 *twL;                // split rows: W_Lfull fine | coarse, as tw
};

// kernel arguments of plan p
PassArgs fft_pass_args(const FftPlan &p);

// Batched work: one item per (view, pass); rows [row_off[i], row_off[i+1]) of
// a launch belong to item i.
struct RowItem {
    const void *in;
    void *out;
    const float2 *chirp;
    long in_ld, out_ld;
    int args;               // index into the PassArgs array
    const float *sc_in, *sc_out;
    int in_lo, in_hi;       // input elements outside [in_lo, in_hi) are zero (not read)
};
struct TrItem {
    const void *in;
    void *out;
    long in_ld, out_ld;
    int rows, cols, tiles_x;
};
int launch_rows_view_batch(const PassArgs *d_args, const RowItem *d_items, const int *d_row_off,
                           int nitems, int total_rows, int threads, size_t smem, float2 *scratch,
                           int scr_stride, int grid, int prec, cudaStream_t st);
int rows_view_batch_grid(int threads, size_t smem, int total_rows);
int launch_transpose_batch(const TrItem *d_items, const int *d_tile_off, int nitems,
                           int total_tiles, int prec, cudaStream_t st);

// Natural index of a digit-reversed slot of plan p (host and device).  For a
// split row, slot c L/2 + q is slot q of half c, which holds index 2 n_q + c.
__host__ __device__ inline int fft_index_of_slot(const FftPlan &p, int slot) {
    const int Lh = p.L / p.split, c = slot / Lh, q = slot - c * Lh;
    int n = 0;
    for (int j = 0; j < p.npass; ++j) n += ((q / p.stride[j]) % p.radix[j]) * p.prefix[j];
    return p.split * n + c;
}
// Position of digit-reversed slot q in the group-major order of the last
// pass (radix R, L / R groups): element k of group g (slot g R + k) at
// k (L / R) + g, so that lanes handling consecutive groups touch
// consecutive addresses.  The per-slot tables (chirp, odd-half modulation)
// and the odd-half scratch are kept in this order.
__host__ __device__ inline int fft_gm_pos(const FftPlan &p, int slot) {
    const int R = p.radix[p.npass - 1], Lh = p.L / p.split, c = slot / Lh, q = slot - c * Lh;
    return c * Lh + (q % R) * (Lh / R) + q / R;
}
// float2 count of the twiddle/modulation table of length L
size_t fft_tw_count(int L);

// Build (or fetch from the per-device cache) the plan and tables of length L.
int fft_plan_get(int L, const FftPlan **out);
// Same plan with its tables written into caller-provided device memory.
int fft_plan_fill(int L, FftPlan *p, float2 *d_tw, double *d_deapod, float *d_pad,
                  cudaStream_t st);

// Padded forward pass: rows of length L (in, row stride in_ld elements) ->
// rows of length 2L (out, row stride out_ld), fine index 2k + a stored at a L + k:
//   out[r][a L + k] = (-1)^k sum_n in[r][n] pre[n] e^{-i pi a (n - L/2)/L} e^{-2 pi i n k/L}
// with pre = pad_pre (or the given pre[L], e.g. (-1)^n alone).  This is the
// centred DFT on the 2x oversampled grid of the deapodised row.
// in_prec: storage of in (PREC_F32 for the hologram); out: storage prec.
// sc_in / sc_out: device pointers to the FP16 scales of in and out (ignored otherwise).
// natural_out = 1 stores fine index 2k + a at 2k + a (natural order) instead;
// with pair_scr (device float2 scratch of pair_cap elements, grid x L needed,
// else ignored) the even half waits there and both halves of a fine pair are
// stored together (full sectors instead of half-sector writes).
int launch_rows_pad2(const FftPlan &p, const void *in, int in_prec, long in_ld, void *out,
                     int prec, long out_ld, int rows, const float *sc_in, const float *sc_out,
                     cudaStream_t st, int natural_out = 0, const float *pre = nullptr,
                     float2 *pair_scr = nullptr, size_t pair_cap = 0);

// View pass: rows of length L: inverse centred DFT (input already carries
// (-1)^k), multiply by chirp[n] (complex, includes deapodisation and 1/L),
// then the padded forward pass as above (output 2L per row).  scratch holds
// grid-size * L float2.  Input elements outside [in_lo, in_hi) are taken as
// zero and not read (the band of a view whose spectrum is zero elsewhere).
int launch_rows_view(const FftPlan &p, const void *in, long in_ld, const float2 *chirp, void *out,
                     long out_ld, int rows, float2 *scratch, int grid, int prec,
                     const float *sc_in, const float *sc_out, cudaStream_t st, int in_lo = 0,
                     int in_hi = 1 << 30);
int rows_view_grid(const FftPlan &p, int rows);

// out[c][r] = in[r][c]
int launch_transpose(const void *in, long in_ld, void *out, long out_ld, int rows, int cols,
                     int prec, cudaStream_t st);

// ---------------------------------------------------------------------------
// FP64 maps and tables (maps.cu)
// ---------------------------------------------------------------------------
double host_g(double s);                       // int_0^s (1 - t^2)^(-3/4) dt
// The function of Eq. 16's 2F1 used by the maps: exact (series of its integral
// form), or the paper's surrogate (Section 4, initialisation step 1): a
// degree-8 polynomial P(s), s = lambda f, fitted by least squares to 51
// frequencies spread uniformly over the band |f| <= 1/(2 pitch) at f_y = 0,
// used as 2F1(..; w) ~ P(lambda f_x / a_y).
struct MapFn {
    int poly = 0;
    double c[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};
void map_fit_paper_poly(double lam, double pitch, MapFn *m);
void host_phi(double u, double v, double *up, double *vp,
              const MapFn &m = MapFn());  // stretch of Eqs. 9, 10, 16
double g_at_one();

// Pull-back table over lattice [kx0, kx0+nkx) x [ky0, ky0+nky), layout [kx][ky].
// With coarse (device memory of pullback_coarse_count(nkx, nky) double2),
// the pre-images of every kPullbackStep-th point are solved first and seed
// the others' Newton iterations.
constexpr int kPullbackStep = 16;
int pullback_coarse_count(int nkx, int nky);
int launch_pullback_table(double lam, double pitch, int nx, int ny, long kx0, int nkx, long ky0,
                          int nky, short2 *base, float2 *frac, cudaStream_t st,
                          const MapFn &m = MapFn(), double2 *coarse = nullptr);
// Output-map table for pixels x_o = cx + (i - ox/2) px etc. at distance z,
// layout [j][i]; t' in stretched-lattice units, stored as b = floor(2t') and
// the fraction 2t' - b in 0.32 fixed point (exact to 2^-32 of a fine cell:
// the output chirp changes by up to thousands of radians per fine cell at
// the paper's depths, so an FP32 fraction would cost 1e-4 rad).
// plain = 1: the identity map x' = x_o of the plain Fresnel transform instead.
int launch_remap_table(double lam, double pitch, int nx, int ny, double z, double cx, double cy,
                       double px, double py, int ox, int oy, int2 *base, uint2 *frac,
                       cudaStream_t st, int plain = 0, const MapFn &m = MapFn());
// chirp[slot] = e^{i pi x_n^2/(lambda z)} deapod[n] / L (linear: 1 / L) at n = natural index of the
// slot (digit-reversed order of plan fp), x_n = (n - L/2) window / L
// linear = 1: without the deapodisation factor (the bilinear output variant)
int launch_chirp_table(const FftPlan &fp, double window_m, double lam, double z, float2 *chirp,
                       cudaStream_t st, int linear = 0);
// Batched chirp tables: item i fills its table with blocks [off[i], off[i+1])
// of a 1-D grid of 256-thread blocks.
struct ChirpItem {
    FftPlan fp;
    double window_m, lam, z;
    float2 *chirp;
    int linear;
};
int launch_chirp_table_batch(const ChirpItem *d_items, const int *d_off, int nitems,
                             int total_blocks, cudaStream_t st);
inline int chirp_blocks(int L) { return (L + 255) / 256; }
// Output chirp e^{i kappa (b + f)^2 / 4} per axis (b fine base, f its
// fraction), split so that every large argument is reduced exactly:
//   e  = e^{i kappa b^2 / 4}          (FP64 phase, reduced, stored FP32),
//   K  = kappa b / (4 pi)             (turns per unit of f, 32.32 fixed point,
//                                      so K f mod 1 is exact integer arithmetic),
// and the f^2 term kappa / (8 pi) f^2 turns from one per-axis constant.
struct __align__(16) OutChirp {
    float2 e;
    unsigned int klo;  // low word of round(K 2^32)
    int khi;           // high word (two's complement)
};
// E[b - b0] for b in [b0, b0 + nb); fails (-3) if |K| would pass 2^30 turns
int launch_outchirp_table(double kappa, long b0, int nb, OutChirp *E, cudaStream_t st);
// x 2^32 in two's complement, as (low word, high word); |turns| < 2^30
inline uint2 turns_fx32(double turns) {
    const long long v = llrint(turns * 4294967296.0);
    return make_uint2((unsigned int)(v & 0xffffffffLL), (unsigned int)(v >> 32));
}

// ---------------------------------------------------------------------------
// Gathers (gather.cu)
// ---------------------------------------------------------------------------
struct StretchArgs {
    const void *G;          // oversampled spectrum, layout [mx][my], 2Nx x 2Ny
    int Nx, Ny;
    const short2 *pb_base;  // pull-back table, layout [kx][ky]: fine base - 2 k (kMasked: zero)
    const float2 *pb_frac;
    long pb_kx0, pb_ky0;
    int pb_nkx, pb_nky;
    long klo_x, khi_x, klo_y, khi_y, kc_x, kc_y;
    int npx, npy;
    int jx0, jn;            // rows jx0 .. jx0 + jn - 1 of S are computed (jn = 0: all npx)
    // G's fine columns (y) in natural order, rows (x) plane-wise
    void *S;                // output, layout [jx][jy], npx x npy
    int prec;               // storage of G and S
    const float *sc_g, *sc_s;
    int plain;              // 1: no stretch, S(f'_k) = DTFT at f = f'_k (plain FrT)
    int linear;             // 1: bilinear on the unpadded DFT grid (G's even samples of
                            //    the hologram loaded without deapodisation)
};
int launch_stretch(const StretchArgs &a, cudaStream_t st);
// batched: item i owns blocks [off[i], off[i+1]) of a 1-D grid (32 x 8 tiles)
int launch_stretch_batch(const StretchArgs *d_items, const int *d_off, int nitems, int total,
                         int prec, cudaStream_t st);
// band rows of a stretch CTA (32 band points along y each): four rows, eight
// CTAs per SM measured faster than 1, 2, 8 or 16 rows (16K stretch 15.25 ms
// against 15.89 ms at eight rows)
constexpr int kStretchRows = 4;
inline int stretch_tiles(int rows, int npy) {
    return ((npy + 31) / 32) * ((rows + kStretchRows - 1) / kStretchRows);
}

struct RemapArgs {
    const void *Q;          // oversampled FrT output, layout [my][mx], 2npy x 2npx
    int npx, npy;
    long kc_x, kc_y;
    const int2 *rm_base;    // output-map table, layout [j][i], row length rm_ld
    const uint2 *rm_frac;   // its fractions, 0.32 fixed point
    long rm_ld, rm_i0, rm_j0;
    long rm_count;          // entries of the table (the debug build's bounds checks)
    int ox, oy;
    int kind;               // 0 intensity f32, 1 field c64, 2 intensity f32 added to out
    const OutChirp *Ex, *Ey;  // output chirp tables (field only)
    long ex_b0, ey_b0;
    uint2 k2x, k2y;           // kappa / (8 pi) turns, 32.32 fixed point (low, high)
    void *out;
    int prec;               // storage of Q
    const float *sc_q;
    int linear;             // 1: bilinear on the native FrT grid (Q's even samples,
                            //    chirp without deapodisation)
};
int launch_remap(const RemapArgs &a, cudaStream_t st);
int launch_remap_batch(const RemapArgs *d_items, const int *d_off, int nitems, int total, int prec,
                       cudaStream_t st);
// Debug build (NUFDS_BOUNDS_CHECK): gather reads found outside their arrays
// since the last reset (first: the first offending element offset, -1 if
// none); -3 in the product build, -4 on a CUDA error.
int bounds_violations(int reset, long long *first);
// output rows of a remap CTA (32 pixels along x each), measured as for the stretch
constexpr int kRemapRows = 4;
inline int remap_tiles(int ox, int oy) {
    return ((ox + 31) / 32) * ((oy + kRemapRows - 1) / kRemapRows);
}

// FP16 scales (device floats sc[]) from exact energy bounds (max |.| <= the
// Frobenius norm, which Parseval gives for every DFT stage):
//   sc[0] T1, sc[1] G, sc[2] S, sc[3] T_T, sc[4] T, sc[5] Q; each the largest
//   power of two with scale * bound <= 2^15.  acc[] (device doubles): [0], [1]
//   weighted hologram energies (launch_norms), [kEnergyAcc, kEnergyAcc +
//   kEnergySlots) partial sums of ||S||^2 (launch_energy).
constexpr int kEnergySlots = 16;
constexpr int kEnergyAcc = 8;
int launch_norms(const float2 *H, int nx, int ny, const double *dx, const double *dy, double *acc,
                 cudaStream_t st);
// ||S||^2 of count FP16 elements stored as S sc_s, into slots[0 .. kEnergySlots)
// (zeroed first)
int launch_energy(const void *S, long count, const float *sc_s, double *slots, cudaStream_t st);
int launch_scales_load(float *sc, const double *acc, int nx, int ny, double k2, cudaStream_t st);
int launch_scales_view(float *sc, const double *acc, double dxp, double dyp, cudaStream_t st);

// launch bookkeeping
void count_launch();
int check_launch();

}  // namespace nufds
