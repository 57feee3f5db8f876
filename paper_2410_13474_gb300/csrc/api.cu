// C ABI of libnufds: plans, the view planner, workspace and the launch sequence.
//
// Launch sequence of one view (Section 4, Fig. 3, steps two, three and five):
//   stretch     S_T[jx][jy] = H~(f(f'_k)) (-1)^(jx+jy)       gather from G (cached)
//   rows_view   along y: inverse DFT, chirp_y, 2x-oversampled forward DFT
//   transpose
//   rows_view   along x: the same -> Q, the oversampled Fresnel transform
//   remap       O(x_o) = Q at x'(x_o) (Eq. 17), |O|^2 or O * chirp_out
// Hologram load (step two, "FT of the hologram"):
//   rows_pad2 along x, transpose, rows_pad2 along y -> G[mx][my]
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/nufds.h"
#include "internal.cuh"

namespace nufds {

static bool kind_ok(int k) {
    return k == NUFDS_OUT_INTENSITY_F32 || k == NUFDS_OUT_FIELD_C64 ||
           k == NUFDS_OUT_INTENSITY_ACCUM_F32;
}

static thread_local int64_t t_launches = 0;

// With NUFDS_DEBUG set, report the CUDA error behind an NUFDS_ECUDA return.
static int cuda_fail(const char *what, int line) {
    cudaError_t e = cudaGetLastError();
    if (getenv("NUFDS_DEBUG"))
        fprintf(stderr, "nufds: %s failed at api.cu:%d: %s\n", what, line, cudaGetErrorString(e));
    return NUFDS_ECUDA;
}
#define CUDA_FAIL(what) cuda_fail(what, __LINE__)
void count_launch() { ++t_launches; }
int check_launch() {
    cudaError_t e = cudaPeekAtLastError();
    if (e == cudaSuccess) return 0;
    if (getenv("NUFDS_DEBUG")) fprintf(stderr, "nufds: launch error: %s\n", cudaGetErrorString(e));
    return NUFDS_ECUDA;
}

struct Geom {
    double lam, pitch;
    int nx, ny;
    MapFn mf;  // exact 2F1 or the paper's polynomial surrogate
};

struct ViewPlan {
    int ox, oy;
    long klo_x, khi_x, klo_y, khi_y, kc_x, kc_y;
    int npx, npy;
    double px, py, w, h, z, cx, cy;
    bool lattice;
    bool plain;  // NUFDS_MODE_PLAIN_FRT
    long i0, j0;
};

struct ViewKey {
    double z, cx, cy, w, h;
    int ox, oy, mode, pad;
    bool operator==(const ViewKey &o) const { return memcmp(this, &o, sizeof(ViewKey)) == 0; }
};

struct GeomTables;

}  // namespace nufds

using namespace nufds;

struct nufds_plan {
    int device = 0;
    double lam = 0, pitch = 0;
    int nx = 0, ny = 0;
    Geom geom;  // geometry and map function (exact or polynomial surrogate)
    uint64_t budget = 0;
    const FftPlan *fx = nullptr, *fy = nullptr;
    // full-view band (z independent in lattice units) and its pull-back table
    long pb_kx0 = 0, pb_ky0 = 0;
    int pb_nkx = 0, pb_nky = 0;
    short2 *pb_base = nullptr;
    float2 *pb_frac = nullptr;
    // output map on the full-view pixel lattice (z independent)
    int2 *rm_base = nullptr;
    uint2 *rm_frac = nullptr;
    nufds::GeomTables *tab = nullptr;  // owner of the four tables above (shared)
    // cached oversampled spectrum, [mx][my], in the plan's storage precision
    int prec = NUFDS_FP32;
    void *G = nullptr;
    float *sc = nullptr;   // FP16 scales (see launch_scales_load / _view)
    double *acc = nullptr; // energies behind the FP16 scales
    bool loaded = false;
    // paper-literal linear interpolation (NUFDS_FLAG_PAPER_LINEAR): the
    // hologram is loaded with (-1)^n alone (lin_pre: nx, then ny floats)
    bool linear = false;
    float *lin_pre = nullptr;
    // workspace arena
    char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t fixed_bytes = 0;
    std::list<std::pair<ViewKey, ViewPlan>> vcache;
    // profiling: an event pair per recorded launch
    bool prof = false;
    struct Rec {
        int stage;
        double bytes;
        int ev;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> events;
    // the workspace's last user: calls on another stream wait for it (two
    // streams may drive one plan, e.g. serving slots)
    cudaEvent_t ws_ev = nullptr;
    cudaStream_t ws_stream = nullptr;
};

namespace nufds {

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

enum Stage {
    ST_PAD_ROWS_X, ST_PAD_TRANSPOSE, ST_PAD_ROWS_Y, ST_TABLES, ST_STRETCH, ST_VIEW_ROWS_Y,
    ST_VIEW_TRANSPOSE, ST_VIEW_ROWS_X, ST_REMAP, ST_COUNT
};
static const char *kStageName[ST_COUNT] = {"pad_rows_x", "pad_transpose", "pad_rows_y",
                                           "tables", "stretch", "view_rows_y",
                                           "view_transpose", "view_rows_x", "remap"};

// run one launch, bracketed by CUDA events on its stream when profiling
template <class F>
static int stage(nufds_plan *P, int st_id, double bytes, cudaStream_t st, F &&launch) {
    if (!P->prof) return launch();
    size_t k = P->recs.size();
    while (P->events.size() < 2 * (k + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return NUFDS_ECUDA;
        P->events.push_back(e);
    }
    cudaEventRecord(P->events[2 * k], st);
    int rc = launch();
    cudaEventRecord(P->events[2 * k + 1], st);
    P->recs.push_back({st_id, bytes, (int)k});
    return rc;
}

static double full_width(double lam, double pitch, double z) {
    double st = lam / (2.0 * pitch);
    return 2.0 * z * st / sqrt(1.0 - st * st);  // Eq. 1
}

// smallest 2^a 3^b 5^c >= n with a >= 6, b <= 2, c <= 1
static long nice_size(long n) {
    long best = -1;
    const long bases[6] = {1, 3, 9, 5, 15, 45};
    for (long b : bases) {
        long v = 64 * b;
        while (v < n) v *= 2;
        if (best < 0 || v < best) best = v;
    }
    return best;
}

// The planner: band = floor/ceil of the Eq. 17 image of all boundary pixel
// centres in lattice units N pitch f'; N' = nice(max(band, (N pitch)^2/(lambda z))).

constexpr int kKnownFlags = NUFDS_FLAG_PAPER_POLY_M | NUFDS_FLAG_PAPER_LINEAR;

static Geom make_geom(double lam, double pitch, int nx, int ny, int flags) {
    Geom g;
    g.lam = lam;
    g.pitch = pitch;
    g.nx = nx;
    g.ny = ny;
    if (flags & NUFDS_FLAG_PAPER_POLY_M) map_fit_paper_poly(lam, pitch, &g.mf);
    return g;
}

static int plan_view_impl(const Geom *P, const nufds_view *v, ViewPlan *o) {
    if (!v || !(v->z_m > 0)) return NUFDS_EINVAL;
    if (v->mode != NUFDS_MODE_NUFDS && v->mode != NUFDS_MODE_PLAIN_FRT) return NUFDS_EINVAL;
    if (!kind_ok(v->out_kind))
        return NUFDS_EINVAL;
    o->plain = v->mode == NUFDS_MODE_PLAIN_FRT;
    const double lam = P->lam, pitch = P->pitch, z = v->z_m;
    double w = v->width_m, h = v->height_m;
    const double B = full_width(lam, pitch, z);
    if (w <= 0 || h <= 0) {
        if (w != 0 || h != 0) return NUFDS_EINVAL;
        w = B;
        h = B;
    }
    int ox = v->out_nx, oy = v->out_ny;
    if (ox <= 0 || oy <= 0) {
        if (ox != 0 || oy != 0) return NUFDS_EINVAL;
        ox = P->nx;
        oy = P->ny;
    }
    if (ox > 65536 || oy > 65536) return NUFDS_EUNSUPPORTED;
    o->ox = ox;
    o->oy = oy;
    o->px = w / ox;
    o->py = h / oy;
    o->w = w;
    o->h = h;
    o->z = z;
    o->cx = v->center_x_m;
    o->cy = v->center_y_m;
    // Extremes of the Eq. 17 image over the boundary pixels.  With u = x/R,
    // v = y/R: u / sqrt(1 - v^2) = x / sqrt(x^2 + z^2) does not depend on y, so
    // k_x = N pitch (1 - v^2)^(1/4) g(x / sqrt(x^2 + z^2)) / lambda falls in
    // magnitude with |y| along a vertical edge and grows with x along a
    // horizontal one (and x <-> y for k_y).  The extremes over the boundary are
    // therefore at the corners or at the edge pixels nearest the axes; those
    // candidates give the same min/max as evaluating every boundary pixel.
    // (The plain Fresnel transform maps x' = x_o: the extremes are corners.)
    double kmin[2] = {1e300, 1e300}, kmax[2] = {-1e300, -1e300};
    auto eval = [&](int i, int j) {
        i = i < 0 ? 0 : (i >= ox ? ox - 1 : i);
        j = j < 0 ? 0 : (j >= oy ? oy - 1 : j);
        double xo = o->cx + (i - 0.5 * ox) * o->px, yo = o->cy + (j - 0.5 * oy) * o->py;
        double kx, ky;
        if (o->plain) {
            kx = xo * P->nx * pitch / (lam * z);
            ky = yo * P->ny * pitch / (lam * z);
        } else {
            double R0 = sqrt(xo * xo + yo * yo + z * z);
            double up, vp;
            host_phi(xo / R0, yo / R0, &up, &vp, P->mf);
            kx = P->nx * pitch * up / lam;
            ky = P->ny * pitch * vp / lam;
        }
        kmin[0] = fmin(kmin[0], kx);
        kmax[0] = fmax(kmax[0], kx);
        kmin[1] = fmin(kmin[1], ky);
        kmax[1] = fmax(kmax[1], ky);
    };
    // pixel index nearest the axis: x_o = c + (i - n/2) p = 0
    const int ia = (int)floor(0.5 * ox - o->cx / o->px), ja = (int)floor(0.5 * oy - o->cy / o->py);
    for (int d = -1; d <= 2; ++d) {
        eval(0, ja + d);
        eval(ox - 1, ja + d);
        eval(ia + d, 0);
        eval(ia + d, oy - 1);
    }
    eval(0, 0);
    eval(ox - 1, 0);
    eval(0, oy - 1);
    eval(ox - 1, oy - 1);
    o->klo_x = (long)floor(kmin[0]);
    o->khi_x = (long)ceil(kmax[0]);
    o->klo_y = (long)floor(kmin[1]);
    o->khi_y = (long)ceil(kmax[1]);
    double chx = ceil((P->nx * pitch) * (P->nx * pitch) / (lam * z));
    double chy = ceil((P->ny * pitch) * (P->ny * pitch) / (lam * z));
    long wx = o->khi_x - o->klo_x + 1, wy = o->khi_y - o->klo_y + 1;
    long npx = nice_size(wx > (long)chx ? wx : (long)chx);
    long npy = nice_size(wy > (long)chy ? wy : (long)chy);
    // rows up to kMaxRowL in one CTA's shared memory, up to twice that over a
    // 2-CTA cluster
    if (npx > 2 * kMaxRowL || npy > 2 * kMaxRowL) return NUFDS_EUNSUPPORTED;
    o->npx = (int)npx;
    o->npy = (int)npy;
    o->kc_x = (long)floor(0.5 * (double)(o->klo_x + o->khi_x));
    o->kc_y = (long)floor(0.5 * (double)(o->klo_y + o->khi_y));
    // pixels on the full view's lattice?  (then the plan's output-map table serves)
    const double fpx = B / P->nx, fpy = B / P->ny;
    o->lattice = false;
    if (!o->plain && fabs(o->px - fpx) <= 1e-12 * fpx && fabs(o->py - fpy) <= 1e-12 * fpy) {
        double ri = o->cx / fpx - 0.5 * ox + 0.5 * P->nx;
        double rj = o->cy / fpy - 0.5 * oy + 0.5 * P->ny;
        double ii = rint(ri), jj = rint(rj);
        if (fabs(ri - ii) < 1e-9 && fabs(rj - jj) < 1e-9 && ii >= 0 && jj >= 0 &&
            ii + ox <= P->nx && jj + oy <= P->ny) {
            o->lattice = true;
            o->i0 = (long)ii;
            o->j0 = (long)jj;
        }
    }
    return NUFDS_OK;
}

static int plan_view_cached(nufds_plan *P, const nufds_view *v, ViewPlan *o) {
    ViewKey key;
    memset(&key, 0, sizeof key);
    key.z = v->z_m;
    key.cx = v->center_x_m;
    key.cy = v->center_y_m;
    key.w = v->width_m;
    key.h = v->height_m;
    key.ox = v->out_nx;
    key.oy = v->out_ny;
    key.mode = v->mode;
    for (auto it = P->vcache.begin(); it != P->vcache.end(); ++it)
        if (it->first == key) {
            *o = it->second;
            P->vcache.splice(P->vcache.begin(), P->vcache, it);
            return kind_ok(v->out_kind) ? NUFDS_OK : NUFDS_EINVAL;
        }
    Geom g = P->geom;
    int rc = plan_view_impl(&g, v, o);
    if (rc) return rc;
    P->vcache.emplace_front(key, *o);
    if (P->vcache.size() > 64) P->vcache.pop_back();
    return NUFDS_OK;
}

// Workspace layout of one view (bytes): A (Q and the first pass output),
// B (S and the transposed pass input), scratch of the view passes, tables.
struct ViewWs {
    size_t A, B, scr, chirp, outc, rm, keep, total;
    int grid_y, grid_x;
    long ex_b0, ey_b0;
    int nbx, nby;
};

static int view_ws(const nufds_plan *P, const ViewPlan &V, const FftPlan *fpx, const FftPlan *fpy,
                   int kind, ViewWs *w, bool keep_band = false) {
    const size_t np = (size_t)V.npx * V.npy, eb = prec_bytes(P->prec);
    w->A = align256(eb * 4 * np);
    w->B = align256(eb * 2 * np);
    w->grid_y = rows_view_grid(*fpy, V.npx);
    w->grid_x = rows_view_grid(*fpx, 2 * V.npy);
    size_t sy = (size_t)w->grid_y * V.npy, sx = (size_t)w->grid_x * V.npx;
    w->scr = align256(sizeof(float2) * (sy > sx ? sy : sx));
    w->chirp = align256(sizeof(float2) * (V.npx + V.npy));
    w->ex_b0 = 2 * V.klo_x - 8;
    w->ey_b0 = 2 * V.klo_y - 8;
    w->nbx = (int)(2 * (V.khi_x - V.klo_x) + 17);
    w->nby = (int)(2 * (V.khi_y - V.klo_y) + 17);
    w->outc = kind == NUFDS_OUT_FIELD_C64 ? align256(sizeof(OutChirp) * (w->nbx + w->nby)) : 0;
    w->rm = V.lattice ? 0 : align256((sizeof(int2) + sizeof(uint2)) * (size_t)V.ox * V.oy + 256);
    // a focal sweep keeps the stretched band (S_T) apart from B, which the
    // Fresnel passes of each depth overwrite
    w->keep = keep_band ? align256(eb * np) : 0;
    w->total = w->A + w->B + w->scr + w->chirp + w->outc + w->rm + w->keep;
    (void)P;
    return NUFDS_OK;
}

// Order uses of the plan's workspace across streams: wait for the last user
// (when it was another stream), and mark this stream as the last user.
static int ws_acquire(nufds_plan *P, cudaStream_t st) {
    if (P->ws_ev && P->ws_stream != st && cudaStreamWaitEvent(st, P->ws_ev, 0) != cudaSuccess)
        return NUFDS_ECUDA;
    return NUFDS_OK;
}
static int ws_release(nufds_plan *P, cudaStream_t st) {
    if (!P->ws_ev && cudaEventCreateWithFlags(&P->ws_ev, cudaEventDisableTiming) != cudaSuccess)
        return NUFDS_ECUDA;
    if (cudaEventRecord(P->ws_ev, st) != cudaSuccess) return NUFDS_ECUDA;
    P->ws_stream = st;
    return NUFDS_OK;
}

static int ensure_ws(nufds_plan *P, size_t need) {
    if (need <= P->ws_bytes) return NUFDS_OK;
    if (P->budget && P->fixed_bytes + need > P->budget) return NUFDS_ENOMEM;
    if (P->ws) {
        cudaDeviceSynchronize();
        cudaFree(P->ws);
        P->ws = nullptr;
        P->ws_bytes = 0;
    }
    if (cudaMalloc(&P->ws, need) != cudaSuccess) {
        cudaGetLastError();
        return NUFDS_ENOMEM;
    }
    P->ws_bytes = need;
    return NUFDS_OK;
}

// max over f of the kernel's tap sum, squared: bound of a 2-D gather's gain
static double kernel_gain2() {
    double best = 0;
    for (int t = 0; t <= 1000; ++t) {
        double f = t / 1000.0, s = 0;
        for (int i = 0; i < kW; ++i) {
            double d = f + (kW / 2 - 1 - i), u = 2.0 * d / kW;
            if (fabs(u) < 1.0) s += exp(kBeta * (sqrt(1.0 - u * u) - 1.0));
        }
        best = fmax(best, s);
    }
    return best * best;
}

static const float *scale_ptr(const nufds_plan *P, int k) {
    return P->prec == NUFDS_FP16_STORE ? P->sc + k : nullptr;
}

static int load_impl(nufds_plan *P, const void *d_holo, cudaStream_t st) {
    const size_t eb = prec_bytes(P->prec);
    const size_t half = align256(eb * 2 * (size_t)P->nx * P->ny);
    int rc = ensure_ws(P, 2 * half);
    if (rc || (rc = ws_acquire(P, st))) return rc;
    void *A = P->ws, *Bf = P->ws + half;
    const float2 *H = (const float2 *)d_holo;
    const double n2 = (double)P->nx * P->ny, q = eb / 8.0;
    if (P->prec == NUFDS_FP16_STORE) {
        static const double k2 = kernel_gain2();
        if ((rc = stage(P, ST_TABLES, 8.0 * n2, st, [&] {
                 int r = launch_norms(H, P->nx, P->ny, P->fx->deapod, P->fy->deapod, P->acc, st);
                 return r ? r : launch_scales_load(P->sc, P->acc, P->nx, P->ny, k2, st);
             })))
            return rc;
    }
    // along x: rows of H (ny rows of nx) -> A (ny x 2nx)
    if ((rc = stage(P, ST_PAD_ROWS_X, (8.0 + 16.0 * q) * n2, st, [&] {
             return launch_rows_pad2(*P->fx, H, PREC_F32, P->nx, A, P->prec, 2 * P->nx, P->ny,
                                     nullptr, scale_ptr(P, 0), st, 0, P->lin_pre);
         })))
        return rc;
    // A (ny x 2nx) -> Bf (2nx x ny)
    if ((rc = stage(P, ST_PAD_TRANSPOSE, 32.0 * q * n2, st, [&] {
             return launch_transpose(A, 2 * P->nx, Bf, P->ny, P->ny, 2 * P->nx, P->prec, st);
         })))
        return rc;
    // along y: rows of Bf (2nx rows of ny) -> G (2nx x 2ny)
    if ((rc = stage(P, ST_PAD_ROWS_Y, 48.0 * q * n2, st, [&] {
             return launch_rows_pad2(*P->fy, Bf, P->prec, P->ny, P->G, P->prec, 2 * P->ny,
                                     2 * P->nx, scale_ptr(P, 0), scale_ptr(P, 1), st,
                                     1,  // G's columns in natural order (the stretch's reads)
                                     P->lin_pre ? P->lin_pre + P->nx : nullptr,
                                     (float2 *)A, half / sizeof(float2));  // A is free here
         })))
        return rc;
    P->loaded = true;
    return ws_release(P, st);
}

// Stretched band kept across the views of a focal sweep: the pull-back and
// the band depend on the geometry, not on z (Section 4: m is independent of
// z), so views with the same band, band centre and N' share S.
struct Sweep {
    bool valid = false;
    long klo_x, khi_x, klo_y, khi_y, kc_x, kc_y;
    int npx, npy;
    bool plain;
    bool same(const ViewPlan &V) const {
        return valid && plain == V.plain && klo_x == V.klo_x && khi_x == V.khi_x && klo_y == V.klo_y &&
               khi_y == V.khi_y && kc_x == V.kc_x && kc_y == V.kc_y && npx == V.npx &&
               npy == V.npy;
    }
    void set(const ViewPlan &V) {
        valid = true;
        plain = V.plain;
        klo_x = V.klo_x;
        khi_x = V.khi_x;
        klo_y = V.klo_y;
        khi_y = V.khi_y;
        kc_x = V.kc_x;
        kc_y = V.kc_y;
        npx = V.npx;
        npy = V.npy;
    }
};

// The part of a view's arrays its passes need (the partial view processes
// its spectral sub-band, Section 4): S is zero outside the band's rows
// [bx0, bx1) (x) and columns [by0, by1) (y), so the stretch and the y pass run
// on the band rows only and both passes read the band columns only; the remap
// reads only the fine rows of Q within a window of the band's y extent,
// [m0, m1), which sit in plane a at rows a npy + [k0[a], k1[a]), so the
// transpose and the x pass produce only those (all rows when a window would
// wrap around the periodic grid).
struct BandWork {
    int bx0, bx1, by0, by1;
    int k0[2], k1[2];
    int rows_x() const { return (k1[0] - k0[0]) + (k1[1] - k0[1]); }
};
static BandWork band_work(const ViewPlan &V) {
    BandWork b;
    b.bx0 = (int)std::max(0L, V.klo_x - V.kc_x + V.npx / 2);
    b.bx1 = (int)std::min((long)V.npx, V.khi_x - V.kc_x + V.npx / 2 + 1);
    b.by0 = (int)std::max(0L, V.klo_y - V.kc_y + V.npy / 2);
    b.by1 = (int)std::min((long)V.npy, V.khi_y - V.kc_y + V.npy / 2 + 1);
    long m0 = 2 * (V.klo_y - V.kc_y) + V.npy - kW / 2 - 2;
    long m1 = 2 * (V.khi_y - V.kc_y) + V.npy + kW / 2 + 3;
    if (m0 < 0 || m1 > 2L * V.npy) {
        m0 = 0;
        m1 = 2L * V.npy;
    }
    for (int a = 0; a < 2; ++a) {  // plane a holds fine rows 2k + a at row a npy + k
        b.k0[a] = (int)((m0 - a + 1) / 2);
        b.k1[a] = (int)((m1 - a + 1) / 2);
    }
    return b;
}

static int reconstruct_impl(nufds_plan *P, const nufds_view *v, void *d_out, cudaStream_t st,
                            Sweep *sw = nullptr) {
    if (!P || !v || !d_out) return NUFDS_EINVAL;
    if (!P->loaded) return NUFDS_EINVAL;
    int rc;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return NUFDS_EINVAL;
    ViewPlan V;
    if ((rc = plan_view_cached(P, v, &V))) return rc;
    if (!V.plain && (V.klo_x < P->pb_kx0 || V.khi_x >= P->pb_kx0 + P->pb_nkx ||
                     V.klo_y < P->pb_ky0 || V.khi_y >= P->pb_ky0 + P->pb_nky))
        return NUFDS_EUNSUPPORTED;
    const FftPlan *fpx, *fpy;
    if ((rc = fft_plan_get(V.npx, &fpx))) return rc;
    if ((rc = fft_plan_get(V.npy, &fpy))) return rc;
    ViewWs W;
    view_ws(P, V, fpx, fpy, v->out_kind, &W, sw != nullptr);
    if (sw && W.total > P->ws_bytes) sw->valid = false;  // the workspace moves
    if ((rc = ensure_ws(P, W.total)) || (rc = ws_acquire(P, st))) return rc;
    char *p = P->ws;
    void *A = p;
    p += W.A;
    void *Bf = p;
    p += W.B;
    float2 *scr = (float2 *)p;
    p += W.scr;
    float2 *chx = (float2 *)p, *chy = chx + V.npx;
    p += W.chirp;
    void *S = W.keep ? (void *)p : Bf;  // where the stretch writes S_T
    p += W.keep;
    OutChirp *Ex = (OutChirp *)p, *Ey = Ex + W.nbx;
    p += W.outc;
    int2 *rmb = P->rm_base;
    uint2 *rmf = P->rm_frac;
    long rm_ld = P->nx, rm_i0 = 0, rm_j0 = 0;
    if (V.lattice) {
        rm_i0 = V.i0;
        rm_j0 = V.j0;
    } else {
        rmf = (uint2 *)p;
        rmb = (int2 *)(p + align256(sizeof(uint2) * (size_t)V.ox * V.oy));
        rm_ld = V.ox;
        if ((rc = stage(P, ST_TABLES, 16.0 * V.ox * V.oy, st, [&] {
                 return launch_remap_table(P->lam, P->pitch, P->nx, P->ny, V.z, V.cx, V.cy, V.px,
                                           V.py, V.ox, V.oy, rmb, rmf, st, V.plain, P->geom.mf);
             })))
            return rc;
    }
    // chirp tables (FP64 phases), window N pitch, x_n = (n - N'/2) N pitch / N'
    if ((rc = stage(P, ST_TABLES, 16.0 * V.npx, st, [&] {
             return launch_chirp_table(*fpx, P->nx * P->pitch, P->lam, V.z, chx, st, P->linear);
         })))
        return rc;
    if ((rc = stage(P, ST_TABLES, 16.0 * V.npy, st, [&] {
             return launch_chirp_table(*fpy, P->ny * P->pitch, P->lam, V.z, chy, st, P->linear);
         })))
        return rc;
    const double kx = M_PI * P->lam * V.z / ((P->nx * P->pitch) * (P->nx * P->pitch));
    const double ky = M_PI * P->lam * V.z / ((P->ny * P->pitch) * (P->ny * P->pitch));
    if (v->out_kind == NUFDS_OUT_FIELD_C64) {
        if ((rc = stage(P, ST_TABLES, 16.0 * (W.nbx + W.nby), st, [&] {
                 int r = launch_outchirp_table(kx, W.ex_b0, W.nbx, Ex, st);
                 return r ? r : launch_outchirp_table(ky, W.ey_b0, W.nby, Ey, st);
             })))
            return rc;
    }
    // work only where the view needs it (band_work)
    const BandWork bw = band_work(V);
    const int bx0 = bw.bx0, bx1 = bw.bx1, by0 = bw.by0, by1 = bw.by1;
    const int *k0 = bw.k0, *k1 = bw.k1;
    const int nbr = bx1 - bx0, nqr = bw.rows_x();
    const size_t ebv = prec_bytes(P->prec);
    // step two: stretch gather -> S_T in Bf (npx x npy)
    StretchArgs sa = {};
    sa.G = P->G;
    sa.Nx = P->nx;
    sa.Ny = P->ny;
    sa.pb_base = P->pb_base;
    sa.pb_frac = P->pb_frac;
    sa.pb_kx0 = P->pb_kx0;
    sa.pb_ky0 = P->pb_ky0;
    sa.pb_nkx = P->pb_nkx;
    sa.pb_nky = P->pb_nky;
    sa.klo_x = V.klo_x;
    sa.khi_x = V.khi_x;
    sa.klo_y = V.klo_y;
    sa.khi_y = V.khi_y;
    sa.kc_x = V.kc_x;
    sa.kc_y = V.kc_y;
    sa.npx = V.npx;
    sa.npy = V.npy;
    sa.jx0 = bx0;
    sa.jn = nbr;
    sa.S = S;
    sa.plain = V.plain;
    sa.linear = P->linear;
    sa.prec = P->prec;
    sa.sc_g = scale_ptr(P, 1);
    sa.sc_s = scale_ptr(P, 2);
    const double np2 = (double)V.npx * V.npy, q = prec_bytes(P->prec) / 8.0;
    const double nbx = (double)(V.khi_x - V.klo_x + 1), nby = (double)(V.khi_y - V.klo_y + 1);
    // algorithmic bytes of the gather: table entries of the band, the part of
    // G the band pulls back to (in proportion to the full band), S written
    const double g_frac = (nbx * nby) / ((double)P->pb_nkx * P->pb_nky);
    const double st_bytes =
        12.0 * nbx * nby + 32.0 * q * P->nx * P->ny * g_frac + 8.0 * q * nbr * V.npy;
    if (!(sw && sw->same(V))) {  // a sweep reuses the band of an earlier depth
        if ((rc = stage(P, ST_STRETCH, st_bytes, st, [&] { return launch_stretch(sa, st); })))
            return rc;
        // the FP16 scales of the passes depend on S's energy only (its band rows)
        if (P->prec == NUFDS_FP16_STORE &&
            (rc = stage(P, ST_TABLES, 4.0 * nbr * V.npy, st, [&] {
                 int r = launch_energy((const char *)S + ebv * bx0 * V.npy, (long)nbr * V.npy,
                                       scale_ptr(P, 2), P->acc + kEnergyAcc, st);
                 return r ? r : launch_scales_view(P->sc, P->acc, fpx->dmax, fpy->dmax, st);
             })))
            return rc;
        if (sw) sw->set(V);
    }
    (void)np2;
    // steps two/three along y: S_T band rows (of npy, read in [by0, by1)) -> A (npx x 2npy)
    if ((rc = stage(P, ST_VIEW_ROWS_Y, 8.0 * q * nbr * (by1 - by0) + 16.0 * q * nbr * V.npy, st,
                    [&] {
             return launch_rows_view(*fpy, (const char *)S + ebv * bx0 * V.npy, V.npy, chy,
                                     (char *)A + ebv * bx0 * 2 * V.npy, 2 * V.npy, nbr, scr,
                                     rows_view_grid(*fpy, nbr), P->prec, scale_ptr(P, 2),
                                     scale_ptr(P, 3), st, by0, by1);
         })))
        return rc;
    // A (band rows x the needed fine rows) -> Bf (needed fine rows x band columns)
    if ((rc = stage(P, ST_VIEW_TRANSPOSE, 16.0 * q * nbr * nqr, st, [&] {
             int r = 0;
             for (int a = 0; a < 2 && !r; ++a)
                 if (k1[a] > k0[a])
                     r = launch_transpose(
                         (const char *)A + ebv * ((size_t)bx0 * 2 * V.npy + (size_t)a * V.npy + k0[a]),
                         2 * V.npy, (char *)Bf + ebv * (((size_t)a * V.npy + k0[a]) * V.npx + bx0),
                         V.npx, nbr, k1[a] - k0[a], P->prec, st);
             return r;
         })))
        return rc;
    // along x: the needed rows of Bf (read in [bx0, bx1)) -> those rows of A = Q (2npy x 2npx)
    if ((rc = stage(P, ST_VIEW_ROWS_X, 8.0 * q * nqr * nbr + 16.0 * q * nqr * V.npx, st, [&] {
             int r = 0;
             for (int a = 0; a < 2 && !r; ++a)
                 if (k1[a] > k0[a]) {
                     const size_t row = (size_t)a * V.npy + k0[a];
                     r = launch_rows_view(*fpx, (const char *)Bf + ebv * row * V.npx, V.npx, chx,
                                          (char *)A + ebv * row * 2 * V.npx, 2 * V.npx,
                                          k1[a] - k0[a], scr, rows_view_grid(*fpx, k1[a] - k0[a]),
                                          P->prec, scale_ptr(P, 4), scale_ptr(P, 5), st, bx0, bx1);
                 }
             return r;
         })))
        return rc;
    // step five: remap
    RemapArgs ra = {};
    ra.Q = A;
    ra.npx = V.npx;
    ra.npy = V.npy;
    ra.kc_x = V.kc_x;
    ra.kc_y = V.kc_y;
    ra.rm_base = rmb;
    ra.rm_frac = rmf;
    ra.rm_count = V.lattice ? (long)P->nx * P->ny : (long)V.ox * V.oy;
    ra.rm_ld = rm_ld;
    ra.rm_i0 = rm_i0;
    ra.rm_j0 = rm_j0;
    ra.ox = V.ox;
    ra.oy = V.oy;
    ra.kind = v->out_kind;
    ra.Ex = Ex;
    ra.Ey = Ey;
    ra.ex_b0 = W.ex_b0;
    ra.ey_b0 = W.ey_b0;
    ra.k2x = turns_fx32(kx / (8.0 * M_PI));
    ra.k2y = turns_fx32(ky / (8.0 * M_PI));
    ra.out = d_out;
    ra.prec = P->prec;
    ra.sc_q = scale_ptr(P, 5);
    ra.linear = P->linear;
    // Q region the view maps into, its table, the output
    const double rm_bytes = 32.0 * q * nbx * nby + 16.0 * V.ox * V.oy +
                            (v->out_kind == NUFDS_OUT_INTENSITY_F32 ? 4.0 : 8.0) * V.ox * V.oy;
    if ((rc = stage(P, ST_REMAP, rm_bytes, st, [&] { return launch_remap(ra, st); })))
        return rc;
    return ws_release(P, st);
}

// The FP64-derived tables of a geometry (pull-back on the full-view band,
// output map on the full-view pixel lattice) depend only on (device, lambda,
// pitch, nx, ny, map function): plans of one geometry share them, reference
// counted (e.g. one resident hologram per precision, or many holograms of
// one display).
struct GeomTables {
    int device, nx, ny, flags;
    double lam, pitch;
    short2 *pb_base = nullptr;
    float2 *pb_frac = nullptr;
    int2 *rm_base = nullptr;
    uint2 *rm_frac = nullptr;
    int refs = 0;
};
static std::mutex g_tab_mu;
static std::vector<GeomTables *> g_tabs;

static void tables_free(GeomTables *t) {
    cudaFree(t->pb_base);
    cudaFree(t->pb_frac);
    cudaFree(t->rm_base);
    cudaFree(t->rm_frac);
    delete t;
}

static void tables_release(GeomTables *t) {
    if (!t) return;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (--t->refs > 0) return;
    for (size_t i = 0; i < g_tabs.size(); ++i)
        if (g_tabs[i] == t) g_tabs.erase(g_tabs.begin() + (long)i);
    tables_free(t);
}

// Find or build (on st, waited for) the tables of P's geometry.
static int tables_acquire(nufds_plan *P, int flags, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    for (GeomTables *t : g_tabs)
        if (t->device == P->device && t->lam == P->lam && t->pitch == P->pitch &&
            t->nx == P->nx && t->ny == P->ny && t->flags == flags) {
            t->refs++;
            P->tab = t;
            return NUFDS_OK;
        }
    GeomTables *t = new (std::nothrow) GeomTables();
    if (!t) return NUFDS_ENOMEM;
    t->device = P->device;
    t->lam = P->lam;
    t->pitch = P->pitch;
    t->nx = P->nx;
    t->ny = P->ny;
    t->flags = flags;
    const size_t npb = (size_t)P->pb_nkx * P->pb_nky, npix = (size_t)P->nx * P->ny;
    if (cudaMalloc(&t->pb_base, npb * sizeof(short2)) != cudaSuccess ||
        cudaMalloc(&t->pb_frac, npb * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&t->rm_base, npix * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&t->rm_frac, npix * sizeof(uint2)) != cudaSuccess) {
        cudaGetLastError();
        tables_free(t);
        return NUFDS_ENOMEM;
    }
    // inverse stretch on the full-view band; output map on the full-view pixel
    // lattice (computed at z = 1, valid at every z)
    const double B1 = full_width(P->lam, P->pitch, 1.0);
    int rc;
    // coarse pre-images seeding the table's Newton solves (freed below; the
    // table is built without them if the allocation fails)
    double2 *coarse = nullptr;
    if (cudaMalloc(&coarse, sizeof(double2) * (size_t)pullback_coarse_count(P->pb_nkx, P->pb_nky)) !=
        cudaSuccess) {
        cudaGetLastError();
        coarse = nullptr;
    }
    if ((rc = launch_pullback_table(P->lam, P->pitch, P->nx, P->ny, P->pb_kx0, P->pb_nkx,
                                    P->pb_ky0, P->pb_nky, t->pb_base, t->pb_frac, st,
                                    P->geom.mf, coarse)) ||
        (rc = launch_remap_table(P->lam, P->pitch, P->nx, P->ny, 1.0, 0.0, 0.0, B1 / P->nx,
                                 B1 / P->ny, P->nx, P->ny, t->rm_base, t->rm_frac, st, 0,
                                 P->geom.mf))) {
        cudaStreamSynchronize(st);
        cudaFree(coarse);
        tables_free(t);
        return rc;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(coarse);
        tables_free(t);
        return NUFDS_ECUDA;
    }
    cudaFree(coarse);
    t->refs = 1;
    g_tabs.push_back(t);
    P->tab = t;
    return NUFDS_OK;
}

static void free_plan(nufds_plan *P) {
    if (!P) return;
    tables_release(P->tab);
    cudaFree(P->G);
    cudaFree(P->sc);
    cudaFree(P->lin_pre);
    cudaFree(P->ws);
    for (cudaEvent_t e : P->events) cudaEventDestroy(e);
    if (P->ws_ev) cudaEventDestroy(P->ws_ev);
    delete P;
}

// hologram sides: 64 .. 32768, 5-smooth, a multiple of 4 (of 8 above kMaxRowL,
// whose rows split over two CTAs into halves that are multiples of 4)
static bool fft_size_ok(int n) {
    if (n < 64 || n > 32768 || n % 4) return false;  // row FFTs need L >= 64
    if (fft_needs_split(n) && n % 8) return false;
    int m = n;
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

// ---------------------------------------------------------------------------
// Batched reconstruction: many views (of one or several plans, of uneven
// sizes) per launch.  Views are grouped into waves that fit the batch
// workspace; each wave is one CUDA graph: the per-view FP64 tables, then one
// persistent launch per stage over all views' work items (stretch tiles, row
// passes, transpose tiles, remap tiles).
// ---------------------------------------------------------------------------
struct BatchView {
    int idx;
    nufds_plan *P;
    ViewPlan V;
    const FftPlan *fpx, *fpy;
    int kind;
    void *out;
    size_t off, bytes;  // region in the batch workspace
};

struct BatchWs {
    char *dev = nullptr;
    size_t bytes = 0;
    // pinned descriptor staging: a ring of buffers, each reused only after
    // the upload that last read it has executed
    static constexpr int kRing = 4;
    char *host[kRing] = {};
    size_t host_bytes[kRing] = {};
    cudaEvent_t host_ev[kRing] = {};
    int ring = 0;
    struct Graph {
        std::string key;
        cudaGraphExec_t exec = nullptr;
    };
    std::list<Graph> graphs;
    cudaStream_t cap = nullptr;  // private stream the graphs are captured on
    cudaEvent_t last = nullptr;  // recorded after the last wave that used this workspace
    uint64_t used = 0;           // recency, for eviction
    int busy = 0;                // host threads inside run_wave with it
};
static std::mutex g_batch_mu;
static std::map<std::pair<int, cudaStream_t>, BatchWs *> g_batch;  // per (device, stream)
static uint64_t g_batch_clock = 0;
// Batch workspaces kept per device.  A caller that runs batches on ever new
// streams would otherwise keep one workspace per stream it ever used (up to
// the batch cap each); the least recently used idle one is freed instead.
constexpr int kMaxBatchWs = 4;

static void batch_ws_free(BatchWs *B) {
    if (B->last) cudaEventSynchronize(B->last);
    for (auto &g : B->graphs) cudaGraphExecDestroy(g.exec);
    cudaFree(B->dev);
    for (int i = 0; i < BatchWs::kRing; ++i) {
        if (B->host_ev[i]) {
            cudaEventSynchronize(B->host_ev[i]);
            cudaEventDestroy(B->host_ev[i]);
        }
        cudaFreeHost(B->host[i]);
    }
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->last) cudaEventDestroy(B->last);
    delete B;
}

// The workspace of (dev, st), marked busy until release; evicts the least
// recently used idle workspace of the device beyond kMaxBatchWs.
static BatchWs *batch_ws_acquire(int dev, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    const auto key = std::make_pair(dev, st);
    auto it = g_batch.find(key);
    if (it == g_batch.end()) {
        for (;;) {
            int count = 0;
            auto lru = g_batch.end();
            for (auto jt = g_batch.begin(); jt != g_batch.end(); ++jt) {
                if (jt->first.first != dev) continue;
                ++count;
                if (!jt->second->busy && (lru == g_batch.end() || jt->second->used < lru->second->used))
                    lru = jt;
            }
            if (count < kMaxBatchWs || lru == g_batch.end()) break;
            batch_ws_free(lru->second);
            g_batch.erase(lru);
        }
        it = g_batch.emplace(key, new BatchWs()).first;
    }
    BatchWs *B = it->second;
    B->used = ++g_batch_clock;
    B->busy++;
    return B;
}
struct BatchWsHold {
    BatchWs *B;
    ~BatchWsHold() {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        B->busy--;
    }
};

static size_t batch_cap_bytes() {
    const char *e = getenv("NUFDS_BATCH_WS_GB");
    double gb = e ? atof(e) : 48.0;
    return (size_t)(gb * (1ull << 30));
}

static size_t view_batch_bytes(const BatchView &b, int prec) {
    const size_t np = (size_t)b.V.npx * b.V.npy, eb = prec_bytes(prec);
    size_t t = align256(eb * 4 * np) + align256(eb * 2 * np) +
               align256(sizeof(float2) * (b.V.npx + b.V.npy)) + 256;
    if (b.kind == NUFDS_OUT_FIELD_C64)
        t += align256(sizeof(OutChirp) * (4 * (b.V.khi_x - b.V.klo_x) + 4 * (b.V.khi_y - b.V.klo_y) + 68));
    if (!b.V.lattice) t += 2 * align256((sizeof(int2) + sizeof(uint2)) * (size_t)b.V.ox * b.V.oy);
    return t;
}

// Classes of the batched row passes: FFT length (L <= 1024, 2048, .., larger)
// x autotuned block size
constexpr int kLenClasses = 6;
constexpr int kThreadClasses = 5;
constexpr int kThreadSizes[kThreadClasses] = {128, 192, 256, 384, 512};
constexpr int kRowClasses = kLenClasses * kThreadClasses;

static int run_wave(std::vector<BatchView> &w, int prec, cudaStream_t st, int32_t *statuses) {
    // ---- sizes and the workspace
    int maxL = 0, threads = 64;
    size_t scr_elems = 0, views_bytes = 0;
    std::vector<const FftPlan *> fps;
    auto fidx = [&](const FftPlan *f) {
        for (size_t i = 0; i < fps.size(); ++i)
            if (fps[i] == f) return (int)i;
        fps.push_back(f);
        return (int)fps.size() - 1;
    };
    for (auto &b : w) {
        for (const FftPlan *f : {b.fpx, b.fpy}) fidx(f);
        b.off = views_bytes;
        b.bytes = view_batch_bytes(b, prec);
        views_bytes += b.bytes;
    }
    const int n = (int)w.size();
    // Row items of each pass grouped by FFT-length class (L <= 1024, 2048, ..)
    // and by the block size the autotuner picked for their length: one launch
    // per class with that class's shared memory, block size and grid, so short
    // rows are not run at the occupancy or block size of the longest.
    auto len_class = [](int L) {
        int c = 0;
        while (c < kLenClasses - 1 && L > (1024 << c)) ++c;
        return c;
    };
    auto row_class = [&](const FftPlan *f) {
        int t = 0;
        while (t < kThreadClasses - 1 && f->threads > kThreadSizes[t]) ++t;
        return len_class(f->L) * kThreadClasses + t;
    };
    struct RowClass {
        int first = 0, count = 0, rows = 0, threads = 64, maxL = 0, grid = 0;
        size_t smem = 0;
    };
    // Row items: the y pass one per view on its band rows, the x pass one per
    // view and plane of the rows of Q its remap reads (band_work)
    struct Slot {
        int view, plane, rows;
        const FftPlan *f;
    };
    std::vector<BandWork> bws(n);
    std::vector<Slot> slots[2];
    for (int i = 0; i < n; ++i) {
        const BandWork &bw = bws[i] = band_work(w[i].V);
        slots[0].push_back({i, -1, bw.bx1 - bw.bx0, w[i].fpy});
        for (int a = 0; a < 2; ++a)
            if (bw.k1[a] > bw.k0[a]) slots[1].push_back({i, a, bw.k1[a] - bw.k0[a], w[i].fpx});
    }
    const int nri = (int)(slots[0].size() + slots[1].size()), ntr = (int)slots[1].size();
    RowClass cls[2][kRowClasses];
    std::vector<int> order[2];  // slot indices of the y and x items, by class
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < kRowClasses; ++c) {
            RowClass &rc = cls[pass][c];
            rc.first = (int)order[pass].size();
            for (size_t q = 0; q < slots[pass].size(); ++q) {
                const Slot &sl = slots[pass][q];
                const FftPlan *f = sl.f;
                if (row_class(f) != c) continue;
                order[pass].push_back((int)q);
                rc.count++;
                rc.rows += sl.rows;
                rc.threads = std::max(rc.threads, std::min(512, f->threads));
                rc.maxL = std::max(rc.maxL, f->L);
                rc.smem = std::max(rc.smem, f->smem_bytes);
            }
            if (rc.count) {
                rc.grid = rows_view_batch_grid(rc.threads, rc.smem, rc.rows);
                maxL = std::max(maxL, rc.maxL);
                threads = std::max(threads, rc.threads);
                scr_elems = std::max(scr_elems, (size_t)rc.grid * rc.maxL);
            }
        }
    }
    const size_t scr_bytes = align256(sizeof(float2) * scr_elems);
    // descriptors: PassArgs[], RowItem[2n], row offsets, TrItem[n], tile offsets,
    // StretchArgs[n], RemapArgs[n], offsets
    const size_t desc_bytes = align256(sizeof(PassArgs) * fps.size()) +
                              align256(sizeof(RowItem) * nri) +
                              align256(sizeof(int) * (nri + 2 * kRowClasses)) +
                              align256(sizeof(TrItem) * ntr) + align256(sizeof(int) * (ntr + 1)) +
                              align256(sizeof(StretchArgs) * n) + align256(sizeof(int) * (n + 1)) +
                              align256(sizeof(RemapArgs) * n) + align256(sizeof(int) * (n + 1)) +
                              align256(sizeof(ChirpItem) * 2 * n) + align256(sizeof(int) * (2 * n + 1));
    const size_t need = views_bytes + scr_bytes + desc_bytes;
    int dev;
    cudaGetDevice(&dev);
    BatchWs *B = batch_ws_acquire(dev, st);
    BatchWsHold hold{B};
    // a stream handle can be reused after its stream was destroyed: order
    // after the last wave that used this workspace
    if (B->last && cudaStreamWaitEvent(st, B->last, 0) != cudaSuccess)
        return CUDA_FAIL("cudaStreamWaitEvent");
    if (need > B->bytes) {
        cudaStreamSynchronize(st);
        for (auto &g : B->graphs) cudaGraphExecDestroy(g.exec);
        B->graphs.clear();
        cudaFree(B->dev);
        B->dev = nullptr;
        B->bytes = 0;
        if (cudaMalloc(&B->dev, need) != cudaSuccess) {
            cudaGetLastError();
            return NUFDS_ENOMEM;
        }
        B->bytes = need;
    }
    const int slot = B->ring;
    B->ring = (B->ring + 1) % BatchWs::kRing;
    if (B->host_ev[slot]) cudaEventSynchronize(B->host_ev[slot]);
    else if (cudaEventCreateWithFlags(&B->host_ev[slot], cudaEventDisableTiming) != cudaSuccess)
        return CUDA_FAIL("cudaEventCreate");
    if (desc_bytes > B->host_bytes[slot]) {
        cudaFreeHost(B->host[slot]);
        B->host[slot] = nullptr;
        if (cudaMallocHost(&B->host[slot], desc_bytes) != cudaSuccess) {
            cudaGetLastError();
            B->host_bytes[slot] = 0;
            return NUFDS_ENOMEM;
        }
        B->host_bytes[slot] = desc_bytes;
    }
    char *dbase = B->dev, *scr_base = dbase + views_bytes, *ddesc = scr_base + scr_bytes;
    char *hdesc = B->host[slot];
    memset(hdesc, 0, desc_bytes);  // padding too: the bytes are the graph's cache key
    // ---- descriptors (host), mirrored at ddesc
    size_t o = 0;
    auto carve = [&](size_t bytes) { size_t r = o; o += align256(bytes); return r; };
    const size_t o_pa = carve(sizeof(PassArgs) * fps.size()), o_ri = carve(sizeof(RowItem) * nri),
                 o_roff = carve(sizeof(int) * (nri + 2 * kRowClasses)),
                 o_tr = carve(sizeof(TrItem) * ntr),
                 o_toff = carve(sizeof(int) * (ntr + 1)), o_sa = carve(sizeof(StretchArgs) * n),
                 o_soff = carve(sizeof(int) * (n + 1)), o_ra = carve(sizeof(RemapArgs) * n),
                 o_roff2 = carve(sizeof(int) * (n + 1)), o_ch = carve(sizeof(ChirpItem) * 2 * n),
                 o_choff = carve(sizeof(int) * (2 * n + 1));
    PassArgs *hpa = (PassArgs *)(hdesc + o_pa);
    RowItem *hri = (RowItem *)(hdesc + o_ri);
    int *hroff = (int *)(hdesc + o_roff);
    TrItem *htr = (TrItem *)(hdesc + o_tr);
    int *htoff = (int *)(hdesc + o_toff);
    StretchArgs *hsa = (StretchArgs *)(hdesc + o_sa);
    int *hsoff = (int *)(hdesc + o_soff);
    RemapArgs *hra = (RemapArgs *)(hdesc + o_ra);
    int *hrmoff = (int *)(hdesc + o_roff2);
    ChirpItem *hch = (ChirpItem *)(hdesc + o_ch);
    int *hchoff = (int *)(hdesc + o_choff);
    int tch = 0;
    for (size_t i = 0; i < fps.size(); ++i) hpa[i] = fft_pass_args(*fps[i]);
    const size_t eb = prec_bytes(prec);
    struct Regions {
        void *A, *Bf;
        float2 *chx, *chy;
        OutChirp *Ex, *Ey;
        int2 *rmb;
        uint2 *rmf;
        float *sc;
        double *acc;
        long ex_b0, ey_b0;
        int nbx, nby;
    };
    std::vector<Regions> R(n);
    std::vector<const float *> scSv(n), scTv(n), scQv(n);
    int ttr = 0, tst = 0, trm = 0, itr = 0;
    for (int i = 0; i < n; ++i) {
        BatchView &b = w[i];
        const ViewPlan &V = b.V;
        nufds_plan *P = b.P;
        char *p = dbase + b.off;
        const size_t np = (size_t)V.npx * V.npy;
        Regions &g = R[i];
        g.A = p;
        p += align256(eb * 4 * np);
        g.Bf = p;
        p += align256(eb * 2 * np);
        g.chx = (float2 *)p;
        g.chy = g.chx + V.npx;
        p += align256(sizeof(float2) * (V.npx + V.npy));
        g.sc = (float *)p;
        g.acc = (double *)(p + 64);
        p += 256;
        g.ex_b0 = 2 * V.klo_x - 8;
        g.ey_b0 = 2 * V.klo_y - 8;
        g.nbx = (int)(2 * (V.khi_x - V.klo_x) + 17);
        g.nby = (int)(2 * (V.khi_y - V.klo_y) + 17);
        g.Ex = g.Ey = nullptr;
        if (b.kind == NUFDS_OUT_FIELD_C64) {
            g.Ex = (OutChirp *)p;
            g.Ey = g.Ex + g.nbx;
            p += align256(sizeof(OutChirp) * (g.nbx + g.nby));
        }
        g.rmb = P->rm_base;
        g.rmf = P->rm_frac;
        long rm_ld = P->nx, rm_i0 = 0, rm_j0 = 0;
        if (V.lattice) {
            rm_i0 = V.i0;
            rm_j0 = V.j0;
        } else {
            g.rmf = (uint2 *)p;
            g.rmb = (int2 *)(p + align256(sizeof(uint2) * (size_t)V.ox * V.oy));
            rm_ld = V.ox;
        }
        for (int a = 0; a < 2; ++a) {
            ChirpItem &c = hch[2 * i + a];
            c.fp = a == 0 ? *b.fpx : *b.fpy;
            c.window_m = (a == 0 ? P->nx : P->ny) * P->pitch;
            c.lam = P->lam;
            c.z = V.z;
            c.chirp = a == 0 ? g.chx : g.chy;
            hchoff[2 * i + a] = tch;
            tch += chirp_blocks(c.fp.L);
        }
        const float *scG = prec == NUFDS_FP16_STORE ? P->sc + 1 : nullptr;
        const float *scS = prec == NUFDS_FP16_STORE ? P->sc + 2 : nullptr;
        const float *scT = prec == NUFDS_FP16_STORE ? g.sc + 3 : nullptr;
        const float *scQ = prec == NUFDS_FP16_STORE ? g.sc + 5 : nullptr;
        StretchArgs &sa = hsa[i];
        sa.G = P->G;
        sa.Nx = P->nx;
        sa.Ny = P->ny;
        sa.pb_base = P->pb_base;
        sa.pb_frac = P->pb_frac;
        sa.pb_kx0 = P->pb_kx0;
        sa.pb_ky0 = P->pb_ky0;
        sa.pb_nkx = P->pb_nkx;
        sa.pb_nky = P->pb_nky;
        sa.klo_x = V.klo_x;
        sa.khi_x = V.khi_x;
        sa.klo_y = V.klo_y;
        sa.khi_y = V.khi_y;
        sa.kc_x = V.kc_x;
        sa.kc_y = V.kc_y;
        sa.npx = V.npx;
        sa.npy = V.npy;
        sa.jx0 = bws[i].bx0;
        sa.jn = bws[i].bx1 - bws[i].bx0;
        sa.S = g.Bf;
        sa.plain = V.plain;
        sa.prec = prec;
        sa.sc_g = scG;
        sa.sc_s = scS;
        hsoff[i] = tst;
        tst += stretch_tiles(sa.jn, V.npy);
        scSv[i] = scS;
        scTv[i] = scT;
        scQv[i] = scQ;
        // the band rows of A by the needed columns (fine rows of Q), per plane
        const BandWork &bw = bws[i];
        for (int a = 0; a < 2; ++a) {
            if (bw.k1[a] <= bw.k0[a]) continue;
            TrItem &tr = htr[itr];
            tr.in = (char *)g.A + eb * ((size_t)bw.bx0 * 2 * V.npy + (size_t)a * V.npy + bw.k0[a]);
            tr.out = (char *)g.Bf + eb * (((size_t)a * V.npy + bw.k0[a]) * V.npx + bw.bx0);
            tr.in_ld = 2 * V.npy;
            tr.out_ld = V.npx;
            tr.rows = bw.bx1 - bw.bx0;
            tr.cols = bw.k1[a] - bw.k0[a];
            tr.tiles_x = (tr.cols + 31) / 32;
            htoff[itr++] = ttr;
            ttr += tr.tiles_x * ((tr.rows + 31) / 32);
        }
        RemapArgs &ra = hra[i];
        ra.Q = g.A;
        ra.npx = V.npx;
        ra.npy = V.npy;
        ra.kc_x = V.kc_x;
        ra.kc_y = V.kc_y;
        ra.rm_base = g.rmb;
        ra.rm_frac = g.rmf;
        ra.rm_count = V.lattice ? (long)P->nx * P->ny : (long)V.ox * V.oy;
        ra.rm_ld = rm_ld;
        ra.rm_i0 = rm_i0;
        ra.rm_j0 = rm_j0;
        ra.ox = V.ox;
        ra.oy = V.oy;
        ra.kind = b.kind;
        ra.Ex = g.Ex;
        ra.Ey = g.Ey;
        ra.ex_b0 = g.ex_b0;
        ra.ey_b0 = g.ey_b0;
        ra.k2x = turns_fx32(P->lam * V.z / ((P->nx * P->pitch) * (P->nx * P->pitch)) / 8.0);
        ra.k2y = turns_fx32(P->lam * V.z / ((P->ny * P->pitch) * (P->ny * P->pitch)) / 8.0);
        ra.out = b.out;
        ra.prec = prec;
        ra.sc_q = scQ;
        hrmoff[i] = trm;
        trm += remap_tiles(V.ox, V.oy);
    }
    // row items in class order; per class an offsets array starting at 0
    int *coff[2][kRowClasses];
    {
        int k = 0, off = 0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int c = 0; c < kRowClasses; ++c) {
                RowClass &rc = cls[pass][c];
                coff[pass][c] = hroff + off;
                int rows = 0;
                for (int q = 0; q < rc.count; ++q) {
                    const Slot &sl = slots[pass][order[pass][rc.first + q]];
                    const int i = sl.view;
                    const ViewPlan &V = w[i].V;
                    const BandWork &bw = bws[i];
                    const Regions &g = R[i];
                    RowItem it;
                    memset(&it, 0, sizeof it);
                    if (pass == 0) {  // S band rows (read in [by0, by1)) -> A
                        it.in = (char *)g.Bf + eb * (size_t)bw.bx0 * V.npy;
                        it.out = (char *)g.A + eb * (size_t)bw.bx0 * 2 * V.npy;
                        it.chirp = g.chy;
                        it.in_ld = V.npy;
                        it.out_ld = 2 * V.npy;
                        it.args = fidx(w[i].fpy);
                        it.sc_in = scSv[i];
                        it.sc_out = scTv[i];
                        it.in_lo = bw.by0;
                        it.in_hi = bw.by1;
                    } else {  // the needed rows of one plane (read in [bx0, bx1)) -> Q
                        const size_t row = (size_t)sl.plane * V.npy + bw.k0[sl.plane];
                        it.in = (char *)g.Bf + eb * row * V.npx;
                        it.out = (char *)g.A + eb * row * 2 * V.npx;
                        it.chirp = g.chx;
                        it.in_ld = V.npx;
                        it.out_ld = 2 * V.npx;
                        it.args = fidx(w[i].fpx);
                        it.sc_in = scTv[i];
                        it.sc_out = scQv[i];
                        it.in_lo = bw.bx0;
                        it.in_hi = bw.bx1;
                    }
                    hri[k++] = it;
                    hroff[off++] = rows;
                    rows += sl.rows;
                }
                hroff[off++] = rows;
            }
        }
    }
    htoff[ntr] = ttr;
    hchoff[2 * n] = tch;
    hsoff[n] = tst;
    hrmoff[n] = trm;
    // the upload is outside the graph; the graph reads ddesc
    if (cudaMemcpyAsync(ddesc, hdesc, o, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaEventRecord(B->host_ev[slot], st) != cudaSuccess)
        return CUDA_FAIL("descriptor upload");
    const PassArgs *dpa = (const PassArgs *)(ddesc + o_pa);
    const RowItem *dri = (const RowItem *)(ddesc + o_ri);
    const int *droff = (const int *)(ddesc + o_roff);
    // ---- the graph: key = the descriptor bytes and the table-launch parameters
    std::string key(hdesc, o);
    key.append((const char *)&dbase, sizeof(dbase));
    for (int i = 0; i < n; ++i) {
        key.append((const char *)&w[i].V, sizeof(ViewPlan));
        key.append((const char *)&w[i].kind, sizeof(int));
    }
    cudaGraphExec_t exec = nullptr;
    for (auto it = B->graphs.begin(); it != B->graphs.end(); ++it)
        if (it->key == key) {
            exec = it->exec;
            B->graphs.splice(B->graphs.begin(), B->graphs, it);
            break;
        }
    if (!exec) {
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph is launched on st
        if (!B->cap && cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess)
            return CUDA_FAIL("cudaStreamCreate");
        const cudaStream_t caller = st;
        st = B->cap;
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return CUDA_FAIL("cudaStreamBeginCapture");
        int rc = launch_chirp_table_batch((const ChirpItem *)(ddesc + o_ch),
                                          (const int *)(ddesc + o_choff), 2 * n, tch, st);
        for (int i = 0; i < n && !rc; ++i) {
            BatchView &b = w[i];
            nufds_plan *P = b.P;
            const ViewPlan &V = b.V;
            Regions &g = R[i];
            if (b.kind == NUFDS_OUT_FIELD_C64) {
                const double kx = M_PI * P->lam * V.z / ((P->nx * P->pitch) * (P->nx * P->pitch));
                const double ky = M_PI * P->lam * V.z / ((P->ny * P->pitch) * (P->ny * P->pitch));
                rc = launch_outchirp_table(kx, g.ex_b0, g.nbx, g.Ex, st);
                if (!rc) rc = launch_outchirp_table(ky, g.ey_b0, g.nby, g.Ey, st);
            }
            if (!rc && !V.lattice)
                rc = launch_remap_table(P->lam, P->pitch, P->nx, P->ny, V.z, V.cx, V.cy, V.px, V.py,
                                        V.ox, V.oy, g.rmb, g.rmf, st, V.plain, P->geom.mf);
            if (!rc && prec == NUFDS_FP16_STORE &&
                cudaMemsetAsync(g.acc, 0, (kEnergyAcc + kEnergySlots) * sizeof(double), st) !=
                    cudaSuccess)
                rc = NUFDS_ECUDA;
        }
        const char *where = "tables";
        if (!rc) {
            where = "stretch";
            rc = launch_stretch_batch((const StretchArgs *)(ddesc + o_sa),
                                      (const int *)(ddesc + o_soff), n, tst, prec, st);
        }
        for (int i = 0; i < n && !rc && prec == NUFDS_FP16_STORE; ++i) {
            const BandWork &bw = bws[i];
            rc = launch_energy((const char *)R[i].Bf + eb * (size_t)bw.bx0 * w[i].V.npy,
                               (long)(bw.bx1 - bw.bx0) * w[i].V.npy, scSv[i],
                               R[i].acc + kEnergyAcc, st);
            if (!rc)
                rc = launch_scales_view(R[i].sc, R[i].acc, w[i].fpx->dmax, w[i].fpy->dmax, st);
        }
        auto rows_pass = [&](int pass) {
            int r = 0, item0 = pass == 0 ? 0 : (int)slots[0].size();
            for (int c = 0; c < kRowClasses && !r; ++c) {
                const RowClass &k = cls[pass][c];
                if (!k.count) continue;
                r = launch_rows_view_batch(dpa, dri + item0 + k.first,
                                           droff + (coff[pass][c] - hroff), k.count, k.rows,
                                           k.threads, k.smem, (float2 *)scr_base, k.maxL,
                                           k.grid, prec, st);
            }
            return r;
        };
        if (!rc) {
            where = "rows_y";
            rc = rows_pass(0);
        }
        if (!rc) {
            where = "transpose";
            rc = launch_transpose_batch((const TrItem *)(ddesc + o_tr),
                                        (const int *)(ddesc + o_toff), ntr, ttr, prec, st);
        }
        if (!rc) {
            where = "rows_x";
            rc = rows_pass(1);
        }
        if (!rc) {
            where = "remap";
            rc = launch_remap_batch((const RemapArgs *)(ddesc + o_ra),
                                    (const int *)(ddesc + o_roff2), n, trm, prec, st);
        }
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (rc || ce != cudaSuccess) {
            if (ce == cudaSuccess) cudaGraphDestroy(graph);
            if (getenv("NUFDS_DEBUG"))
                fprintf(stderr, "nufds: batch capture stage %s (max threads %d, max L %d)\n",
                        where, threads, maxL);
            int r2 = CUDA_FAIL(rc ? "a launch during capture" : "cudaStreamEndCapture");
            return rc ? rc : r2;
        }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return CUDA_FAIL("cudaGraphInstantiate");
        B->graphs.push_front({key, exec});
        if (B->graphs.size() > 16) {
            cudaGraphExecDestroy(B->graphs.back().exec);
            B->graphs.pop_back();
        }
        st = caller;
    }
    if (cudaGraphLaunch(exec, st) != cudaSuccess) return CUDA_FAIL("cudaGraphLaunch");
    count_launch();
    if ((!B->last && cudaEventCreateWithFlags(&B->last, cudaEventDisableTiming) != cudaSuccess) ||
        cudaEventRecord(B->last, st) != cudaSuccess)
        return CUDA_FAIL("cudaEventRecord");
    for (auto &b : w)
        if (statuses) statuses[b.idx] = NUFDS_OK;
    return NUFDS_OK;
}

static int batch_impl(nufds_plan *const *plans, const nufds_view *views, void *const *outs,
                      int32_t count, cudaStream_t st, int32_t *statuses) {
    int first = NUFDS_OK;
    auto fail = [&](int i, int rc) {
        if (statuses) statuses[i] = rc;
        if (first == NUFDS_OK) first = rc;
    };
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return NUFDS_ECUDA;
    std::vector<BatchView> all;
    for (int32_t i = 0; i < count; ++i) {
        nufds_plan *P = plans[i];
        if (!P || !outs[i] || !P->loaded || P->device != dev) {
            fail(i, NUFDS_EINVAL);
            continue;
        }
        BatchView b;
        b.idx = i;
        b.P = P;
        b.kind = views[i].out_kind;
        b.out = outs[i];
        // the linear variant has single-view kernels only
        int rc = P->linear ? NUFDS_EUNSUPPORTED : plan_view_cached(P, &views[i], &b.V);
        if (!rc && !b.V.plain &&
            (b.V.klo_x < P->pb_kx0 || b.V.khi_x >= P->pb_kx0 + P->pb_nkx ||
             b.V.klo_y < P->pb_ky0 || b.V.khi_y >= P->pb_ky0 + P->pb_nky))
            rc = NUFDS_EUNSUPPORTED;
        if (!rc) rc = fft_plan_get(b.V.npx, &b.fpx);
        if (!rc) rc = fft_plan_get(b.V.npy, &b.fpy);
        if (!rc && (b.fpx->split != 1 || b.fpy->split != 1)) {
            // rows split over a CTA pair have single-view kernels only: such a
            // view runs on its own, on the batch's stream, in its batch order
            rc = reconstruct_impl(P, &views[i], outs[i], st);
            if (rc) fail(i, rc);
            else if (statuses) statuses[i] = NUFDS_OK;
            continue;
        }
        if (rc) {
            fail(i, rc);
            continue;
        }
        all.push_back(b);
    }
    // views of one plan next to each other (in order of the plan's first
    // appearance): their stretch gathers then read the same spectrum while it
    // is in L2, and a wave holds fewer distinct spectra
    {
        std::vector<const nufds_plan *> seen;
        auto rank = [&](const nufds_plan *P) {
            for (size_t k = 0; k < seen.size(); ++k)
                if (seen[k] == P) return (int)k;
            seen.push_back(P);
            return (int)seen.size() - 1;
        };
        std::vector<std::pair<int, int>> key(all.size());
        for (size_t i = 0; i < all.size(); ++i) key[i] = {rank(all[i].P), (int)i};
        std::sort(key.begin(), key.end());
        std::vector<BatchView> sorted;
        sorted.reserve(all.size());
        for (auto &k : key) sorted.push_back(all[k.second]);
        all.swap(sorted);
    }
    const size_t cap = batch_cap_bytes();
    for (int prec : {NUFDS_FP32, NUFDS_FP16_STORE, NUFDS_BF16_STORE}) {
        std::vector<BatchView> wave;
        size_t bytes = 0;
        auto flush = [&]() {
            if (wave.empty()) return;
            int rc = run_wave(wave, prec, st, statuses);
            if (rc)
                for (auto &b : wave) fail(b.idx, rc);
            wave.clear();
            bytes = 0;
        };
        for (auto &b : all) {
            if (b.P->prec != prec) continue;
            size_t vb = view_batch_bytes(b, prec);
            if (!wave.empty() && bytes + vb > cap) flush();
            wave.push_back(b);
            bytes += vb;
        }
        flush();
    }
    return first;
}

}  // namespace nufds

extern "C" {

const char *nufds_status_string(int s) {
    switch (s) {
        case NUFDS_OK: return "ok";
        case NUFDS_EINVAL: return "invalid argument";
        case NUFDS_ENOMEM: return "out of device memory or HBM budget";
        case NUFDS_EUNSUPPORTED: return "unsupported";
        case NUFDS_ECUDA: return "CUDA error";
        case NUFDS_ETIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

int64_t nufds_launch_count(int32_t reset) {
    int64_t v = t_launches;
    if (reset) t_launches = 0;
    return v;
}

int nufds_debug_bounds_violations(int32_t reset, int64_t *first_offset) {
    long long f = -1;
    const int n = bounds_violations(reset, &f);
    if (first_offset) *first_offset = f;
    return n == -3 ? NUFDS_EUNSUPPORTED : (n < 0 ? NUFDS_ECUDA : n);
}

int nufds_plan_create(const nufds_params *prm, const void *d_holo, void *stream, nufds_plan **out) {
    if (!out) return NUFDS_EINVAL;
    *out = nullptr;
    if (!prm || !(prm->wavelength_m > 0) || !(prm->pitch_m > 0) ||
        !(prm->wavelength_m < 2.0 * prm->pitch_m) ||
        (prm->flags & ~kKnownFlags) != 0 || prm->nx <= 0 || prm->ny <= 0 ||
        prm->nx % 4 || prm->ny % 4)
        return NUFDS_EINVAL;
    if (prm->precision != NUFDS_FP32 && prm->precision != NUFDS_FP16_STORE &&
        prm->precision != NUFDS_BF16_STORE)
        return NUFDS_EINVAL;
    if ((prm->flags & NUFDS_FLAG_PAPER_LINEAR) && prm->precision != NUFDS_FP32)
        return NUFDS_EUNSUPPORTED;
    if (!fft_size_ok(prm->nx) || !fft_size_ok(prm->ny)) return NUFDS_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    nufds_plan *P = new (std::nothrow) nufds_plan();
    if (!P) return NUFDS_ENOMEM;
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        delete P;
        return NUFDS_ECUDA;
    }
    P->lam = prm->wavelength_m;
    P->pitch = prm->pitch_m;
    P->nx = prm->nx;
    P->ny = prm->ny;
    P->budget = prm->hbm_budget_bytes;
    P->prec = prm->precision;
    P->geom = make_geom(P->lam, P->pitch, P->nx, P->ny, prm->flags);
    P->linear = (prm->flags & NUFDS_FLAG_PAPER_LINEAR) != 0;
    int rc;
    if ((rc = fft_plan_get(P->nx, &P->fx)) || (rc = fft_plan_get(P->ny, &P->fy))) {
        free_plan(P);
        return rc;
    }
    // full-view band (z = 1: lattice units do not depend on z)
    nufds_view fv;
    memset(&fv, 0, sizeof fv);
    fv.z_m = 1.0;
    ViewPlan V;
    Geom g = P->geom;
    if ((rc = plan_view_impl(&g, &fv, &V))) {
        free_plan(P);
        return rc;
    }
    P->pb_kx0 = V.klo_x;
    P->pb_ky0 = V.klo_y;
    P->pb_nkx = (int)(V.khi_x - V.klo_x + 1);
    P->pb_nky = (int)(V.khi_y - V.klo_y + 1);
    const size_t npb = (size_t)P->pb_nkx * P->pb_nky, npix = (size_t)P->nx * P->ny;
    P->fixed_bytes = npb * 12 + npix * 16 + npix * 4 * prec_bytes(P->prec) + 64;
    if (P->budget && P->fixed_bytes > P->budget) {
        free_plan(P);
        return NUFDS_ENOMEM;
    }
    if (cudaMalloc(&P->G, 4 * npix * prec_bytes(P->prec)) != cudaSuccess ||
        cudaMalloc(&P->sc, 256) != cudaSuccess) {
        cudaGetLastError();
        free_plan(P);
        return NUFDS_ENOMEM;
    }
    P->acc = (double *)(P->sc + 16);
    if (P->linear) {
        std::vector<float> sg(P->nx + P->ny);
        for (int n = 0; n < P->nx; ++n) sg[n] = (n & 1) ? -1.0f : 1.0f;
        for (int n = 0; n < P->ny; ++n) sg[P->nx + n] = (n & 1) ? -1.0f : 1.0f;
        if (cudaMalloc(&P->lin_pre, sizeof(float) * sg.size()) != cudaSuccess ||
            cudaMemcpy(P->lin_pre, sg.data(), sizeof(float) * sg.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            cudaGetLastError();
            free_plan(P);
            return NUFDS_ENOMEM;
        }
    }
    // the tables depend on the map function only
    if ((rc = tables_acquire(P, prm->flags & NUFDS_FLAG_PAPER_POLY_M, st))) {
        free_plan(P);
        return rc;
    }
    P->pb_base = P->tab->pb_base;
    P->pb_frac = P->tab->pb_frac;
    P->rm_base = P->tab->rm_base;
    P->rm_frac = P->tab->rm_frac;
    if (d_holo && (rc = load_impl(P, d_holo, st))) {
        free_plan(P);
        return rc;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        free_plan(P);
        return NUFDS_ECUDA;
    }
    *out = P;
    return NUFDS_OK;
}

int nufds_plan_load(nufds_plan *P, const void *d_holo, void *stream) {
    if (!P || !d_holo) return NUFDS_EINVAL;
    return load_impl(P, d_holo, (cudaStream_t)stream);
}

// Wavefront error along the hologram's central row (Sections 2 and 4).  In
// direction-cosine units (u = lambda f) the point's spectrum has, by
// stationary phase, the phase -(u x_o + w z_o)/lambda cycles, w = sqrt(1 - |u|^2);
// the Fresnel transform at z_r focuses -(u' x_r + z_r (1 - |u'|^2 / 2))/lambda,
// with u' the stretched frequency (NU-FDS) or u itself (plain transform).
int nufds_wavefront_error(const nufds_params *prm, double xo, double yo, double zo, int32_t mode,
                          double z_r, int32_t samples, double *x, double *w, double *max_abs) {
    if (!prm || !max_abs || samples < 1 || !(zo > 0)) return NUFDS_EINVAL;
    const double lam = prm->wavelength_m, pitch = prm->pitch_m;
    if (!(lam > 0) || !(pitch > 0) || !(lam < 2.0 * pitch) || prm->nx <= 0 ||
        (prm->flags & ~kKnownFlags))
        return NUFDS_EINVAL;
    if (mode != NUFDS_MODE_NUFDS && mode != NUFDS_MODE_PLAIN_FRT) return NUFDS_EINVAL;
    const Geom g = make_geom(lam, pitch, prm->nx, prm->ny, prm->flags);
    const double R0 = sqrt(xo * xo + yo * yo + zo * zo);
    const double u0 = xo / R0, v0 = yo / R0;  // lambda f_l at the hologram centre (Eq. 4)
    double zf = zo, xf, yf;                   // the focus of the transform
    if (mode == NUFDS_MODE_NUFDS) {
        double a, b;
        host_phi(u0, v0, &a, &b, g.mf);       // Eq. 17: x_o' = z lambda f_0'
        xf = zo * a;
        yf = zo * b;
    } else {
        if (z_r > 0) zf = z_r;
        xf = zf * u0;
        yf = zf * v0;
    }
    auto err = [&](double u, double v) {      // cycles, before the piston
        double up = u, vp = v;
        if (mode == NUFDS_MODE_NUFDS) host_phi(u, v, &up, &vp, g.mf);
        const double obj = u * xo + v * yo + zo * sqrt(1.0 - u * u - v * v);
        const double par = up * xf + vp * yf + zf * (1.0 - 0.5 * (up * up + vp * vp));
        return (par - obj) / lam;
    };
    const double e0 = err(u0, v0), ub = 0.5 * lam / pitch, aperture = prm->nx * pitch;
    double mx = 0;
    for (int j = 0; j < samples; ++j) {
        const double xh = aperture * (j - 0.5 * (samples - 1)) / samples;
        const double R = sqrt((xh - xo) * (xh - xo) + yo * yo + zo * zo);
        const double u = (xo - xh) / R, v = yo / R;
        double e = NAN;
        if (fabs(u) < ub && fabs(v) < ub && u * u + v * v < 1.0) {
            e = err(u, v) - e0;
            mx = fmax(mx, fabs(e));
        }
        if (x) x[j] = xh;
        if (w) w[j] = e;
    }
    *max_abs = mx;
    return NUFDS_OK;
}

static bool host_geom_ok(const nufds_params *prm) {
    return prm && prm->wavelength_m > 0 && prm->pitch_m > 0 &&
           prm->wavelength_m < 2.0 * prm->pitch_m && prm->nx > 0 && prm->ny > 0 &&
           !(prm->flags & ~kKnownFlags);
}

// Eq. 17: x_o' = z lambda f_0' with f_0 = (x_o, y_o) / (lambda R_0)
int nufds_output_map(const nufds_params *prm, double z, double xo, double yo, double *xp,
                     double *yp) {
    if (!host_geom_ok(prm) || !(z > 0) || !xp || !yp) return NUFDS_EINVAL;
    const Geom g = make_geom(prm->wavelength_m, prm->pitch_m, prm->nx, prm->ny, prm->flags);
    const double R = sqrt(xo * xo + yo * yo + z * z);
    double up, vp;
    host_phi(xo / R, yo / R, &up, &vp, g.mf);
    *xp = z * up;
    *yp = z * vp;
    return NUFDS_OK;
}

// The paper's fixed-point iteration for the inverse of Eq. 17 (Section 4,
// the second Eq. 18): x_o(1) = x_o', x_o(k) = x_o' R(k-1) / (z m_x(f_0(k-1))),
// m_x = f_0x' / f_0x from the same map function as the plan.
int nufds_output_map_inverse(const nufds_params *prm, double z, double xp, double yp,
                             int32_t steps, double *xo, double *yo) {
    if (!host_geom_ok(prm) || !(z > 0) || steps < 1 || !xo || !yo) return NUFDS_EINVAL;
    const Geom g = make_geom(prm->wavelength_m, prm->pitch_m, prm->nx, prm->ny, prm->flags);
    double x = xp, y = yp;
    for (int k = 2; k <= steps; ++k) {
        const double R = sqrt(x * x + y * y + z * z), u = x / R, v = y / R;
        double up, vp;
        host_phi(u, v, &up, &vp, g.mf);
        // x' R / (z m_x) with m_x = u' / u, i.e. x' R u / (z u')
        const double xn = u != 0.0 ? xp * R * u / (z * up) : 0.0;
        const double yn = v != 0.0 ? yp * R * v / (z * vp) : 0.0;
        x = xn;
        y = yn;
    }
    *xo = x;
    *yo = y;
    return NUFDS_OK;
}

int nufds_view_plan(const nufds_params *prm, const nufds_view *v, nufds_view_info *info) {
    if (!prm || !v || !info) return NUFDS_EINVAL;
    if (!(prm->wavelength_m > 0) || !(prm->pitch_m > 0) ||
        !(prm->wavelength_m < 2.0 * prm->pitch_m) || prm->nx <= 0 || prm->ny <= 0)
        return NUFDS_EINVAL;
    ViewPlan V;
    if (prm->flags & ~kKnownFlags) return NUFDS_EINVAL;
    Geom g = make_geom(prm->wavelength_m, prm->pitch_m, prm->nx, prm->ny, prm->flags);
    int rc = plan_view_impl(&g, v, &V);
    if (rc) return rc;
    memset(info, 0, sizeof *info);
    info->out_nx = V.ox;
    info->out_ny = V.oy;
    info->k_lo_x = V.klo_x;
    info->k_hi_x = V.khi_x;
    info->k_lo_y = V.klo_y;
    info->k_hi_y = V.khi_y;
    info->np_x = V.npx;
    info->np_y = V.npy;
    info->k_c_x = V.kc_x;
    info->k_c_y = V.kc_y;
    info->pitch_out_x_m = V.px;
    info->pitch_out_y_m = V.py;
    info->width_m = V.w;
    info->height_m = V.h;
    info->on_full_view_lattice = V.lattice ? 1 : 0;
    const size_t np = (size_t)V.npx * V.npy;
    info->workspace_bytes = sizeof(float2) * 6 * np;
    return NUFDS_OK;
}

int nufds_reconstruct(nufds_plan *P, const nufds_view *v, void *d_out, void *stream) {
    return reconstruct_impl(P, v, d_out, (cudaStream_t)stream);
}

int nufds_reconstruct_sweep(nufds_plan *P, const nufds_view *views, void *const *d_outs,
                            int32_t count, void *stream, int32_t *statuses) {
    if (!P || count < 0 || (count > 0 && (!views || !d_outs))) return NUFDS_EINVAL;
    Sweep sw;
    int first = NUFDS_OK;
    for (int32_t i = 0; i < count; ++i) {
        const int rc = reconstruct_impl(P, &views[i], d_outs[i], (cudaStream_t)stream, &sw);
        if (rc) sw.valid = false;
        if (statuses) statuses[i] = rc;
        if (rc && first == NUFDS_OK) first = rc;
    }
    return first;
}

int nufds_reconstruct_batch(nufds_plan *const *plans, const nufds_view *views,
                            void *const *d_outs, int32_t count, void *stream, int32_t *statuses) {
    if (count < 0 || (count > 0 && (!plans || !views || !d_outs))) return NUFDS_EINVAL;
    return batch_impl(plans, views, d_outs, count, (cudaStream_t)stream, statuses);
}

void nufds_destroy(nufds_plan *P) {
    if (!P) return;
    cudaDeviceSynchronize();
    free_plan(P);
}

int nufds_profile(nufds_plan *P, int32_t enable) {
    if (!P) return NUFDS_EINVAL;
    if (enable) P->recs.clear();
    P->prof = enable != 0;
    return NUFDS_OK;
}

int nufds_profile_read(nufds_plan *P, nufds_stage_stat *out, int32_t max, int32_t *count) {
    if (!P || !count || (max > 0 && !out)) return NUFDS_EINVAL;
    nufds_stage_stat agg[ST_COUNT];
    memset(agg, 0, sizeof agg);
    for (const auto &r : P->recs) {
        if (cudaEventSynchronize(P->events[2 * r.ev + 1]) != cudaSuccess) return NUFDS_ECUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P->events[2 * r.ev], P->events[2 * r.ev + 1]) != cudaSuccess)
            return NUFDS_ECUDA;
        agg[r.stage].launches += 1;
        agg[r.stage].total_ms += ms;
        agg[r.stage].bytes += r.bytes;
    }
    int n = 0;
    for (int s = 0; s < ST_COUNT; ++s) {
        if (!agg[s].launches) continue;
        if (n < max) {
            out[n] = agg[s];
            strncpy(out[n].name, kStageName[s], sizeof(out[n].name) - 1);
        }
        ++n;
    }
    *count = n;
    return NUFDS_OK;
}

uint64_t nufds_plan_device_bytes(const nufds_plan *P) {
    if (!P) return 0;
    return P->fixed_bytes + P->ws_bytes;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free reconstruction for small holograms.
//
// Everything the reconstruction needs besides the caller's hologram and output
// (tables, the oversampled spectrum, the pass buffers and the per-CTA scratch
// rows of the view passes) lives in one file-scope device array.  Host code
// only ever uses its device address from cudaGetSymbolAddress (taken once per
// device, on the first call there); the symbol itself is a host-side stand-in.
// ---------------------------------------------------------------------------
namespace nufds {

constexpr int kNoAllocMaxN = 128;        // hologram side
constexpr int kNoAllocMaxNp = 256;       // FFT size N' of a view
constexpr int kNoAllocMaxOutPix = 16384; // pixels of an off-lattice view
constexpr size_t kNoAllocBytes = 6u << 20;

static __device__ __align__(256) unsigned char g_noalloc_arena[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static std::map<int, char *> g_noalloc_base;  // device -> address of g_noalloc_arena

static int noalloc_base(char **out) {
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return NUFDS_ECUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_base.find(dev);
    if (it == g_noalloc_base.end()) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_arena) != cudaSuccess || !p) {
            cudaGetLastError();
            return NUFDS_ECUDA;
        }
        it = g_noalloc_base.emplace(dev, (char *)p).first;
    }
    *out = it->second;
    return NUFDS_OK;
}

struct Carver {
    char *p;
    size_t left;
    template <class T> T *take(size_t count) {
        size_t b = align256(sizeof(T) * count);
        if (b > left) return nullptr;
        T *r = (T *)p;
        p += b;
        left -= b;
        return r;
    }
};

static int noalloc_fft(Carver &c, int L, FftPlan *fp, cudaStream_t st) {
    float2 *tw = c.take<float2>(fft_tw_count(L));
    double *dea = c.take<double>(L);
    float *pad = c.take<float>(L);
    if (!tw || !dea || !pad) return NUFDS_EUNSUPPORTED;
    int rc = fft_plan_fill(L, fp, tw, dea, pad, st);
    return rc == -3 ? NUFDS_EUNSUPPORTED : (rc ? NUFDS_ECUDA : NUFDS_OK);
}

}  // namespace nufds

extern "C" int nufds_reconstruct_noalloc(const nufds_params *prm, const nufds_view *v,
                                         const void *d_holo, void *d_out, void *stream) {
    if (!prm || !v || !d_holo || !d_out) return NUFDS_EINVAL;
    if (!(prm->wavelength_m > 0) || !(prm->pitch_m > 0) ||
        !(prm->wavelength_m < 2.0 * prm->pitch_m) || prm->flags != 0 || prm->nx <= 0 ||
        prm->ny <= 0 || prm->nx % 4 || prm->ny % 4)
        return NUFDS_EINVAL;
    if (prm->precision != NUFDS_FP32) return NUFDS_EUNSUPPORTED;
    if (prm->nx > kNoAllocMaxN || prm->ny > kNoAllocMaxN || !fft_size_ok(prm->nx) ||
        !fft_size_ok(prm->ny))
        return NUFDS_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const Geom g = make_geom(prm->wavelength_m, prm->pitch_m, prm->nx, prm->ny, 0);
    const int nx = prm->nx, ny = prm->ny;
    ViewPlan F, V;
    nufds_view fv;
    memset(&fv, 0, sizeof fv);
    fv.z_m = 1.0;
    int rc;
    if ((rc = plan_view_impl(&g, &fv, &F))) return rc;
    if ((rc = plan_view_impl(&g, v, &V))) return rc;
    if (V.plain) return NUFDS_EUNSUPPORTED;
    if (V.npx > kNoAllocMaxNp || V.npy > kNoAllocMaxNp) return NUFDS_EUNSUPPORTED;
    if (!V.lattice && (long)V.ox * V.oy > kNoAllocMaxOutPix) return NUFDS_EUNSUPPORTED;
    const long pb_kx0 = F.klo_x, pb_ky0 = F.klo_y;
    const int pb_nkx = (int)(F.khi_x - F.klo_x + 1), pb_nky = (int)(F.khi_y - F.klo_y + 1);
    if (V.klo_x < pb_kx0 || V.khi_x >= pb_kx0 + pb_nkx || V.klo_y < pb_ky0 ||
        V.khi_y >= pb_ky0 + pb_nky)
        return NUFDS_EUNSUPPORTED;
    char *base;
    if ((rc = noalloc_base(&base))) return rc;
    Carver c{base, kNoAllocBytes};
    const size_t npix = (size_t)nx * ny, np2 = (size_t)V.npx * V.npy;
    float2 *G = c.take<float2>(4 * npix);
    short2 *pbb = c.take<short2>((size_t)pb_nkx * pb_nky);
    float2 *pbf = c.take<float2>((size_t)pb_nkx * pb_nky);
    int2 *rmb = c.take<int2>(npix);
    uint2 *rmf = c.take<uint2>(npix);
    float2 *A = c.take<float2>(4 * (np2 > npix ? np2 : npix));
    float2 *Bf = c.take<float2>(2 * (np2 > npix ? np2 : npix));
    float2 *chx = c.take<float2>(V.npx), *chy = c.take<float2>(V.npy);
    if (!G || !pbb || !pbf || !rmb || !rmf || !A || !Bf || !chx || !chy) return NUFDS_EUNSUPPORTED;
    FftPlan fx, fy, fpx, fpy;
    if ((rc = noalloc_fft(c, nx, &fx, st)) || (rc = noalloc_fft(c, ny, &fy, st)) ||
        (rc = noalloc_fft(c, V.npx, &fpx, st)) || (rc = noalloc_fft(c, V.npy, &fpy, st)))
        return rc;
    const int grid_y = rows_view_grid(fpy, V.npx), grid_x = rows_view_grid(fpx, 2 * V.npy);
    const size_t sy = (size_t)grid_y * V.npy, sx = (size_t)grid_x * V.npx;
    float2 *scr = c.take<float2>(sy > sx ? sy : sx);
    const long ex_b0 = 2 * V.klo_x - 8, ey_b0 = 2 * V.klo_y - 8;
    const int nbx = (int)(2 * (V.khi_x - V.klo_x) + 17), nby = (int)(2 * (V.khi_y - V.klo_y) + 17);
    OutChirp *Ex = nullptr, *Ey = nullptr;
    if (v->out_kind == NUFDS_OUT_FIELD_C64) {
        Ex = c.take<OutChirp>(nbx);
        Ey = c.take<OutChirp>(nby);
        if (!Ex || !Ey) return NUFDS_EUNSUPPORTED;
    }
    int2 *vrb = rmb;
    uint2 *vrf = rmf;
    long rm_ld = nx, rm_i0 = 0, rm_j0 = 0;
    if (V.lattice) {
        rm_i0 = V.i0;
        rm_j0 = V.j0;
    } else {
        vrb = c.take<int2>((size_t)V.ox * V.oy);
        vrf = c.take<uint2>((size_t)V.ox * V.oy);
        rm_ld = V.ox;
    }
    if (!scr || !vrb || !vrf) return NUFDS_EUNSUPPORTED;
    // geometry tables (FP64): inverse stretch on the full-view band, output map
    const double B1 = full_width(g.lam, g.pitch, 1.0);
    if ((rc = launch_pullback_table(g.lam, g.pitch, nx, ny, pb_kx0, pb_nkx, pb_ky0, pb_nky, pbb,
                                    pbf, st)))
        return rc;
    if (V.lattice) {
        if ((rc = launch_remap_table(g.lam, g.pitch, nx, ny, 1.0, 0.0, 0.0, B1 / nx, B1 / ny, nx,
                                     ny, rmb, rmf, st)))
            return rc;
    } else if ((rc = launch_remap_table(g.lam, g.pitch, nx, ny, V.z, V.cx, V.cy, V.px, V.py, V.ox,
                                        V.oy, vrb, vrf, st))) {
        return rc;
    }
    // oversampled spectrum of the hologram
    const float2 *H = (const float2 *)d_holo;
    if ((rc = launch_rows_pad2(fx, H, PREC_F32, nx, A, PREC_F32, 2 * nx, ny, nullptr, nullptr,
                               st)) ||
        (rc = launch_transpose(A, 2 * nx, Bf, ny, ny, 2 * nx, PREC_F32, st)) ||
        (rc = launch_rows_pad2(fy, Bf, PREC_F32, ny, G, PREC_F32, 2 * ny, 2 * nx, nullptr,
                               nullptr, st, 1)))
        return rc;
    // the view
    if ((rc = launch_chirp_table(fpx, nx * g.pitch, g.lam, V.z, chx, st)) ||
        (rc = launch_chirp_table(fpy, ny * g.pitch, g.lam, V.z, chy, st)))
        return rc;
    const double kx = M_PI * g.lam * V.z / ((nx * g.pitch) * (nx * g.pitch));
    const double ky = M_PI * g.lam * V.z / ((ny * g.pitch) * (ny * g.pitch));
    if (v->out_kind == NUFDS_OUT_FIELD_C64 &&
        ((rc = launch_outchirp_table(kx, ex_b0, nbx, Ex, st)) ||
         (rc = launch_outchirp_table(ky, ey_b0, nby, Ey, st))))
        return rc;
    StretchArgs sa = {};
    sa.G = G;
    sa.Nx = nx;
    sa.Ny = ny;
    sa.pb_base = pbb;
    sa.pb_frac = pbf;
    sa.pb_kx0 = pb_kx0;
    sa.pb_ky0 = pb_ky0;
    sa.pb_nkx = pb_nkx;
    sa.pb_nky = pb_nky;
    sa.klo_x = V.klo_x;
    sa.khi_x = V.khi_x;
    sa.klo_y = V.klo_y;
    sa.khi_y = V.khi_y;
    sa.kc_x = V.kc_x;
    sa.kc_y = V.kc_y;
    sa.npx = V.npx;
    sa.npy = V.npy;
    sa.S = Bf;
    sa.prec = PREC_F32;
    sa.sc_g = nullptr;
    sa.sc_s = nullptr;
    sa.plain = 0;
    if ((rc = launch_stretch(sa, st)) ||
        (rc = launch_rows_view(fpy, Bf, V.npy, chy, A, 2 * V.npy, V.npx, scr, grid_y, PREC_F32,
                               nullptr, nullptr, st)) ||
        (rc = launch_transpose(A, 2 * V.npy, Bf, V.npx, V.npx, 2 * V.npy, PREC_F32, st)) ||
        (rc = launch_rows_view(fpx, Bf, V.npx, chx, A, 2 * V.npx, 2 * V.npy, scr, grid_x,
                               PREC_F32, nullptr, nullptr, st)))
        return rc;
    RemapArgs ra = {};
    ra.Q = A;
    ra.npx = V.npx;
    ra.npy = V.npy;
    ra.kc_x = V.kc_x;
    ra.kc_y = V.kc_y;
    ra.rm_base = vrb;
    ra.rm_frac = vrf;
    ra.rm_count = V.lattice ? (long)nx * ny : (long)V.ox * V.oy;
    ra.rm_ld = rm_ld;
    ra.rm_i0 = rm_i0;
    ra.rm_j0 = rm_j0;
    ra.ox = V.ox;
    ra.oy = V.oy;
    ra.kind = v->out_kind;
    ra.Ex = Ex;
    ra.Ey = Ey;
    ra.ex_b0 = ex_b0;
    ra.ey_b0 = ey_b0;
    ra.k2x = turns_fx32(kx / (8.0 * M_PI));
    ra.k2y = turns_fx32(ky / (8.0 * M_PI));
    ra.out = d_out;
    ra.prec = PREC_F32;
    ra.sc_q = nullptr;
    return launch_remap(ra, st);
}
