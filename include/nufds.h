/*
 * nufds.h -- C ABI of the GB300 NU-FDS reconstruction library (libnufds.so).
 *
 * NU-FDS (Kozacki et al., "Non-uniform Fourier Domain Stretching method for
 * ultra-wide-angle wave propagation") reconstructs the object field of a
 * wide-angle computer-generated hologram at distance z:
 *   step two (Section 4, Fig. 3): FT of the hologram, the non-uniform
 *     frequency stretch f' = (f_x m_x, f_y m_y) of Eqs. 9, 10 with the
 *     magnification of Eq. 16, resampling onto a uniform f' grid, inverse FT;
 *   step three: the Fresnel transform of Eq. 2 (chirp, FT, chirp);
 *   step five: the output remap O(x_o) = O'(x_o') with x_o' from Eqs. 17-18,
 *     sampled on a uniform grid of the requested (full or partial) view.
 * Problem statement followed by the parameters: wavelength, pixel pitch,
 * N_x x N_y hologram (Section 2), distance z_o, output window and sampling
 * (Section 4, output-grid choice; partial view: Section 4, last part).
 *
 * Conventions.  Hologram sample (ix, iy) sits at x = (ix - N_x/2) pitch,
 * y = (iy - N_y/2) pitch.  Output pixel (i, j) of a view sits at
 * x_o = center_x + (i - out_nx/2) * width/out_nx (same for y).  Transform
 * kernel e^{-2 pi i x f}; chirps e^{+i pi r^2/(lambda z)}; no 1/(i lambda z)
 * factor (Eq. 2 has none); forward DFT unnormalised, inverse DFT scaled by
 * 1/N'^2.  A unit point source focused at the view centre gives |O|^2 ~ N^4.
 *
 * Buffers.  Every pointer called d_* is a DEVICE pointer owned by the caller.
 * Holograms are row-major interleaved complex64 (8 bytes per sample, 8-byte
 * aligned), N_y rows of N_x samples.  Outputs are row-major out_ny x out_nx,
 * float32 intensity |O|^2 (4 bytes per pixel) or interleaved complex64 field
 * (8 bytes per pixel).  cuda_stream is a cudaStream_t (NULL = legacy
 * default stream).  Calls are asynchronous on that stream unless stated.
 *
 * Host-only calls (no GPU work, no device memory): nufds_view_plan,
 * nufds_output_map, nufds_output_map_inverse, nufds_wavefront_error,
 * nufds_status_string.
 *
 * Errors.  Every int-returning call returns NUFDS_OK (0) or a negative code;
 * nufds_status_string() names it.  No C++ exception crosses the ABI.  A plan
 * is used by one host thread at a time; different plans are independent.
 */
#ifndef NUFDS_H
#define NUFDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NUFDS_OK 0
#define NUFDS_EINVAL (-1)       /* bad argument: lambda >= 2 pitch, z <= 0, sizes, NULL */
#define NUFDS_ENOMEM (-2)       /* HBM budget exceeded or cudaMalloc failed             */
#define NUFDS_EUNSUPPORTED (-3) /* valid but not supported (size limits, view outside FoV) */
#define NUFDS_ECUDA (-4)        /* a CUDA runtime call failed                            */
#define NUFDS_ETIMEOUT (-5)     /* a bounded device-side wait gave up                    */

/* storage of the cached spectrum and of the inter-pass arrays (arithmetic is FP32) */
#define NUFDS_FP32 0
#define NUFDS_FP16_STORE 1
#define NUFDS_BF16_STORE 2

#define NUFDS_OUT_INTENSITY_F32 0
#define NUFDS_OUT_FIELD_C64 1
/* |O|^2 added to the float32 values already in d_out (not overwritten): the
 * mean intensity over several holograms -- the speckle averaging over
 * random-phase CGHs of Section 5 -- is K such calls into one zeroed buffer,
 * then a division by K.  Calls accumulating into one buffer must be ordered
 * (same stream). */
#define NUFDS_OUT_INTENSITY_ACCUM_F32 2

/* plan flags */
/* The paper's own surrogate for Eq. 16 (Section 4, initialisation step 1): 2F1
 * replaced by a degree-8 polynomial in s = lambda f, least-squares fitted to 51
 * frequencies uniformly spread over |f| <= 1/(2 pitch) at f_y = 0, applied as
 * 2F1(..; lambda^2 f_x^2 / a_y^2) ~ P(lambda f_x / a_y) in the pull-back, the
 * output map (Eq. 17) and the view planner.  A paper-literal variant whose
 * distance from the exact method is reported; not in nufds_reconstruct_noalloc. */
#define NUFDS_FLAG_PAPER_POLY_M 1
/* The paper-literal resampling (Section 4, steps two and five name an
 * interpolation without its kernel; read as linear, separable in x and y):
 * S(f'_k) by bilinear interpolation of the unpadded centred DFT of the
 * hologram at the pulled-back frequency, and O(x_o) by bilinear interpolation
 * of the native Fresnel-transform grid at x'(x_o) of Eq. 17, both periodic
 * like the DFT, instead of the ideal (band-limited) resampling.  A variant
 * whose distance from the exact method is reported.  NUFDS_FP32 storage only
 * (else NUFDS_EUNSUPPORTED from nufds_plan_create); single-view calls and
 * sweeps only (a batch gives its views NUFDS_EUNSUPPORTED); combines with
 * NUFDS_FLAG_PAPER_POLY_M; not in nufds_reconstruct_noalloc. */
#define NUFDS_FLAG_PAPER_LINEAR 2

/* reconstruction method of a view */
#define NUFDS_MODE_NUFDS 0     /* the NU-FDS method (stretch, FrT, Eq. 17 remap)          */
#define NUFDS_MODE_PLAIN_FRT 1 /* Eq. 2 alone at z: no stretch, x' = x_o (the paper's Fig.
                                * 10b comparison).  Band from the view's own extent; views
                                * needing N' > 49152 are NUFDS_EUNSUPPORTED; not available
                                * in nufds_reconstruct_noalloc */

typedef struct nufds_plan nufds_plan;

typedef struct nufds_params {
    double wavelength_m;       /* lambda > 0, lambda < 2 pitch (Eq. 1)                  */
    double pitch_m;            /* hologram pixel pitch Delta                            */
    int32_t nx, ny;            /* hologram size; 5-smooth, 64 <= n <= 32768, a multiple
                                * of 4 (of 8 above 24576) (else NUFDS_EUNSUPPORTED)      */
    int32_t precision;         /* NUFDS_FP32, NUFDS_FP16_STORE or NUFDS_BF16_STORE      */
    int32_t flags;             /* 0, or NUFDS_FLAG_PAPER_POLY_M and/or _PAPER_LINEAR   */
    uint64_t hbm_budget_bytes; /* cap on device memory the plan may allocate; 0 = none  */
} nufds_params;

typedef struct nufds_view {
    double z_m;                /* reconstruction distance z_o > 0                       */
    double center_x_m;         /* view centre in the object plane                       */
    double center_y_m;
    double width_m;            /* view size; 0,0 = full view B = 2 z tan(asin(l/2D))    */
    double height_m;
    int32_t out_nx, out_ny;    /* output pixels; 0,0 = N_x, N_y                         */
    int32_t out_kind;          /* NUFDS_OUT_INTENSITY_F32, _FIELD_C64 or _INTENSITY_ACCUM_F32 */
    int32_t mode;              /* NUFDS_MODE_NUFDS or NUFDS_MODE_PLAIN_FRT              */
} nufds_view;

/* What the planner decided for one view (Section 4 output grid; band from Eq. 17). */
typedef struct nufds_view_info {
    int64_t out_nx, out_ny;
    int64_t k_lo_x, k_hi_x, k_lo_y, k_hi_y; /* stretched-spectrum band, lattice 1/(N pitch) */
    int64_t np_x, np_y;                     /* FFT size N' of the band per axis             */
    int64_t k_c_x, k_c_y;                   /* band centre, at index N'/2                   */
    double pitch_out_x_m, pitch_out_y_m;
    double width_m, height_m;
    int32_t on_full_view_lattice;           /* 1: pixels are a window of the full view's   */
    int32_t reserved;
    uint64_t workspace_bytes;               /* device workspace this view needs             */
} nufds_view_info;

/*
 * Create a plan for one hologram geometry and (optionally) load a hologram.
 * Builds, on the device, the FP64-derived tables of the inverse stretch
 * (Eqs. 9, 10, 16) on the full-view band and of the output map (Eq. 17) on
 * the full-view pixel lattice -- once per (device, wavelength, pitch, size,
 * map function, i.e. NUFDS_FLAG_PAPER_POLY_M): plans of the same geometry share them, reference counted, and
 * nufds_plan_device_bytes counts them in each plan -- then, if
 * d_hologram_c64 is not NULL, computes and caches its oversampled spectrum
 * (step two, "FT of the hologram").  Synchronises cuda_stream before
 * returning; the caller may free the hologram afterwards.  *out receives the
 * plan (NULL on error).
 */
int nufds_plan_create(const nufds_params *params, const void *d_hologram_c64,
                      void *cuda_stream, nufds_plan **out);

/*
 * Replace the plan's hologram (same geometry): recompute the cached
 * oversampled spectrum from d_hologram_c64.  Asynchronous on cuda_stream;
 * the hologram must stay valid until the stream reaches this point.
 */
int nufds_plan_load(nufds_plan *plan, const void *d_hologram_c64, void *cuda_stream);

/*
 * Plan one view for a hologram geometry without touching the GPU (host FP64
 * only; fills *info).  Band: floor/ceil of the Eq. 17 image, in stretched-
 * lattice units N pitch f', of every boundary pixel centre of the view; FFT
 * size N' = nice(max(band width, ceil((N pitch)^2/(lambda z)))) with nice(n)
 * the smallest 2^a 3^b 5^c >= n, a >= 6, b <= 2, c <= 1.
 */
int nufds_view_plan(const nufds_params *params, const nufds_view *view, nufds_view_info *info);

/*
 * Reconstruct one view of the loaded hologram into d_out (out_ny x out_nx,
 * float32 intensity or complex64 field).  Asynchronous on cuda_stream.  The
 * plan's workspace grows on first use of a larger view (that call allocates
 * and synchronises).  Calls on different streams may use one plan: each
 * waits, on its stream, for the previous call's use of the plan's workspace.
 * Views whose band leaves the full-view band, or that need N' > 49152 on an
 * axis, are NUFDS_EUNSUPPORTED (rows of N' > 24576 run split over two CTAs).
 */
int nufds_reconstruct(nufds_plan *plan, const nufds_view *view, void *d_out, void *cuda_stream);

/*
 * Reconstruct count views, each of its own plan (plans may repeat, sizes may
 * differ), on cuda_stream.  Views are grouped into waves whose working memory
 * fits a cap (environment variable NUFDS_BATCH_WS_GB, default 48); each wave
 * runs as one CUDA graph: per-view tables, then one persistent launch per
 * stage over all views.  Results are bitwise those of nufds_reconstruct.
 * The batch workspace is kept per (device, stream), so batches on different
 * streams may run concurrently (their plans' spectra are only read).  Views
 * with N' > 24576 on an axis run one by one as nufds_reconstruct, on
 * cuda_stream, in batch order.
 * statuses (may be NULL) receives one code per view; a failing view does not
 * stop the others (views of a plan created with NUFDS_FLAG_PAPER_LINEAR get
 * NUFDS_EUNSUPPORTED).  Returns NUFDS_OK if every view succeeded, else the
 * first error code.
 */
int nufds_reconstruct_batch(nufds_plan *const *plans, const nufds_view *views,
                            void *const *d_outs, int32_t count, void *cuda_stream,
                            int32_t *statuses);

/*
 * Focal sweep (several depths, or several views, of one loaded hologram).
 * Section 4: the magnification m(f) does not depend on z, so the pull-back of
 * the stretched lattice and therefore the stretched spectrum S of a band
 * depend only on the band (its bounds and centre) and N'.  Views are
 * reconstructed in order; a view whose band and N' equal those of the
 * previous successful view reuses its S and runs only the Fresnel transform
 * at its own z (Eq. 2) and the output remap (Eq. 17).  Full views at the
 * paper's depths (0.5-3 m) all share one band.  Results are bitwise those of
 * nufds_reconstruct.  The workspace holds one extra N'_x N'_y array (S).
 * views[i] -> d_outs[i] as in nufds_reconstruct, on cuda_stream; statuses (may
 * be NULL) receives one code per view.  Returns NUFDS_OK or the first error.
 */
int nufds_reconstruct_sweep(nufds_plan *plan, const nufds_view *views, void *const *d_outs,
                            int32_t count, void *cuda_stream, int32_t *statuses);

/* Free the plan and its device memory (synchronises its streams).  NULL-safe. */
void nufds_destroy(nufds_plan *plan);

/* Bytes of device memory the plan holds. */
uint64_t nufds_plan_device_bytes(const nufds_plan *plan);

/* Static name of a status code. */
const char *nufds_status_string(int status);

/* Per-stage timing of the launches a plan issued while profiling was on. */
typedef struct nufds_stage_stat {
    char name[24];     /* stage name, e.g. "view_rows_x"                              */
    int64_t launches;  /* kernel launches recorded                                    */
    double total_ms;   /* summed CUDA-event durations of those launches (device time) */
    double bytes;      /* summed algorithmic bytes: compulsory reads + writes         */
} nufds_stage_stat;

/*
 * enable = 1: clear and start recording a CUDA event pair around every kernel
 * the plan launches (on the launching stream); 0: stop recording.
 */
int nufds_profile(nufds_plan *plan, int32_t enable);

/*
 * Aggregate what was recorded, one entry per stage (at most max entries into
 * out; *count receives the number of stages).  Waits for the recorded events.
 */
int nufds_profile_read(nufds_plan *plan, nufds_stage_stat *out, int32_t max, int32_t *count);

/*
 * Allocation-free reconstruction of a small hologram (no counterpart in the
 * paper; an interface for callers).  For callers that must not call
 * cudaMalloc or cudaFree -- for example a display or capture loop whose
 * device memory is reserved up front by another framework's allocator, or one
 * that cannot take the device-wide synchronisation that cudaFree implies --
 * this runs the whole path (FP64 geometry tables, the oversampled spectrum of
 * d_hologram_c64, and the view) without allocating device memory.  All working
 * memory (tables, spectrum, pass buffers and the per-CTA scratch rows of the
 * view passes) lives in one 6 MiB array in the library's static device
 * memory, which every GPU that loads the library holds until the process
 * exits.  Limits: nx, ny <= 128, FFT size N' <= 256 per axis, and off-lattice
 * views of at most 16384 pixels; larger requests return NUFDS_EUNSUPPORTED.
 * Arguments, layouts and results are those of nufds_plan_create followed by
 * nufds_reconstruct with the same params and view.
 * The first call on a device looks up the array's device address there (do
 * that first call before any stream capture).  Each call synchronises
 * cuda_stream while it uploads its FFT tables, then enqueues its kernels.
 * Every call uses the same array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.  No
 * part of the array needs to start at zero; each kernel writes what the next
 * one reads.
 */
int nufds_reconstruct_noalloc(const nufds_params *params, const nufds_view *view,
                              const void *d_hologram_c64, void *d_out, void *cuda_stream);

/*
 * Output coordinate map of Eq. 17 (host only, FP64, the map function the
 * params' flags select): the FrT output position (xp, yp) at which NU-FDS
 * reconstructs an object point at (xo, yo) and depth z, all in metres.
 * NUFDS_EINVAL for bad geometry (as in nufds_wavefront_error), z <= 0 or NULL
 * outputs.
 */
int nufds_output_map(const nufds_params *params, double z, double xo, double yo, double *xp,
                     double *yp);

/*
 * The paper's fixed-point iteration for the inverse of Eq. 17 (Section 4, the
 * second Eq. 18), host only: x_o(1) = x_o', then steps - 1 updates
 * x_o(k) = x_o' R(k-1) / (z m_x(f_0(k-1))) (and likewise y); the paper uses 4
 * steps, which reach half a pixel over most of the window (Fig. 4c).  The
 * library's own remap does not need it (it gathers through Eq. 17 directly).
 * NUFDS_EINVAL for bad geometry, z <= 0, steps < 1 or NULL outputs.
 */
int nufds_output_map_inverse(const nufds_params *params, double z, double xp, double yp,
                             int32_t steps, double *xo, double *yo);

/*
 * Wavefront error of the object point (xo, yo, zo) reconstructed from its
 * hologram (Section 2, Figs. 2c and 2f; Section 4, Fig. 5), in waves, along
 * the hologram's central row: the phase of the point's spectrum (stationary
 * phase of e^{-ikR_o} at the local frequency of Eq. 4 of each hologram
 * pixel) minus the paraxial phase that the Fresnel transform focuses, with
 * its value at the hologram centre removed.
 *   mode NUFDS_MODE_NUFDS: frequencies stretched by Eqs. 9-10 (the plan's
 *     map function: exact 2F1, or the polynomial with NUFDS_FLAG_PAPER_POLY_M),
 *     focus at z_o and x_o' of Eq. 17; z_r is ignored.
 *   mode NUFDS_MODE_PLAIN_FRT: the plain transform at distance z_r (z_o when
 *     z_r <= 0, the paper's Fig. 2c; 1/|c_xl(0,0)| of Eq. 5 gives Fig. 2f),
 *     focused at z_r lambda f_xl(0,0).
 * Sample j sits at x_j = (j - (samples-1)/2) nx pitch / samples (metres);
 * x (may be NULL) and w (may be NULL) receive `samples` doubles; w_j is NaN
 * where the local frequency leaves the band |lambda f| < lambda/(2 pitch) per
 * axis or is evanescent.  *max_abs = max |w_j| over the others (0 if none).
 * Host only: uses no GPU and allocates nothing.  Errors: NUFDS_EINVAL for
 * NULL params or max_abs, samples < 1, zo <= 0, wavelength or pitch <= 0,
 * wavelength >= 2 pitch, nx <= 0 (ny is not used), an unknown mode or flag.
 */
int nufds_wavefront_error(const nufds_params *params, double xo, double yo, double zo,
                          int32_t mode, double z_r, int32_t samples, double *x, double *w,
                          double *max_abs);

/*
 * Number of kernel launches issued by this library on the calling thread
 * since the last reset (reset = 1 zeroes it after reading).  Lets a caller
 * count the GPU work a call made.
 */
int64_t nufds_launch_count(int32_t reset);

/*
 * Debug builds only (the library compiled with NUFDS_BOUNDS_CHECK defined,
 * libnufds_bc.so): the two gathers of Section 4 (the stretch of step two and
 * the output remap of step five, Eq. 17), their batched and paper-literal
 * bilinear forms, check every read of the spectrum, of Q and of the FP64
 * tables against the extent of the row and array it reads.  A read outside
 * is skipped (its taps count as zero) and recorded instead of faulting.
 * Returns the number of such reads since the last reset (>= 0; saturates at
 * INT32_MAX) after synchronising the device, with the element offset of the
 * first one in *first_offset (-1 if none; first_offset may be NULL);
 * reset = 1 zeroes both after reading.  The product build returns
 * NUFDS_EUNSUPPORTED; NUFDS_ECUDA on a CUDA error.
 */
int nufds_debug_bounds_violations(int32_t reset, int64_t *first_offset);

#ifdef __cplusplus
}
#endif

#endif /* NUFDS_H */
