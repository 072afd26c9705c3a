/*
 * Azimuthal-integration ORACLE -- test infrastructure, not product code.
 *
 * A plain, slow, double-precision CPU statement of azimuthal integration with pixel
 * splitting as described by Kieffer & Ashiotis, "PyFAI: a Python library for high
 * performance azimuthal integration on GPU" (EuroSciPy 2014).  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline arm may load this library.  It
 * shares no code with the CUDA path: it has its own geometry, its own binning, its own
 * polygon clipping (Sutherland-Hodgman + shoelace, a textbook routine deliberately
 * different from the line-integral method of Sec. 4.2) and its own sparse assembly.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fPIC -shared  (no FMA contraction, so every
 * rounding step is the one written below; the same flags are used on x86-64 and AArch64).
 *
 * Conventions (readings of the paper, listed in the design notes):
 *   image: ny rows (dim1, slow) x nx columns (dim2, fast), pixel index p = i*nx + j.
 *   geometry: t = Rz(rot3) Ry(rot2) Rx(rot1) (d1 - poni1, d2 - poni2, dist)^T;
 *             2theta = atan2(sqrt(t1^2 + t2^2), t3), chi = atan2(t1, t2)   (Sec. 3 list).
 *   radial bins: data range [lo, hi] of the positions used by the split mode over unmasked
 *             pixels, delta = (hi - lo) / npt, f = (x - lo) / delta        (Sec. 3.2, 3.3).
 *   chi bins: fixed range [-180, 180) degrees, npt_azim bins.
 *   CSR: rows = bins (2D row = chi_bin * npt_rad + rad_bin), columns = pixels, ascending
 *        within a row, one entry per (bin, pixel)                          (Sec. 5.2.1).
 *
 * Parity pins: every function here is checked by the non-GPU tests against closed forms,
 * library routines (numpy.histogram, scipy rotations, scipy.sparse), brute-force sub-pixel
 * sampling and hand-derived fixtures.  The singular-pixel rule (a pixel whose azimuthal
 * span exceeds 180 degrees after unwrapping, i.e. a pixel containing the beam centre) has
 * no statement in the paper: it is a stated reading (radial bounding box, in 2D times a
 * uniform azimuth), pinned to that reading by hand-derived fixtures.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_UNIT_2TH_DEG = 0, ORC_UNIT_Q_NM = 1, ORC_UNIT_R_MM = 2 };
enum { ORC_SPLIT_NONE = 0, ORC_SPLIT_BBOX = 1, ORC_SPLIT_FULL = 2 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ESHAPE = -2, ORC_ENOMEM = -3, ORC_ERANGE = -8 };

/* Relative area below which a 2D full-split candidate rectangle is dropped. */
#define ORC_KEEP_2D 1e-12

typedef struct {
    double dist, poni1, poni2, rot1, rot2, rot3, pixel1, pixel2, wavelength;
} orc_geom;

/* ------------------------------------------------------------------------------------ */
/* Geometry (Sec. 3, coordinate list; the generic detector geometry is only referenced   */
/* by the paper, so the rotation convention is a stated reading).                        */
/* ------------------------------------------------------------------------------------ */

static void matmul3(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

/* R = Rz(rot3) . Ry(rot2) . Rx(rot1), right-handed active rotations. */
void orc_rotation(double rot1, double rot2, double rot3, double R[9])
{
    double c1 = cos(rot1), s1 = sin(rot1);
    double c2 = cos(rot2), s2 = sin(rot2);
    double c3 = cos(rot3), s3 = sin(rot3);
    double Rx[9] = {1, 0, 0, 0, c1, -s1, 0, s1, c1};
    double Ry[9] = {c2, 0, s2, 0, 1, 0, -s2, 0, c2};
    double Rz[9] = {c3, -s3, 0, s3, c3, 0, 0, 0, 1};
    double T[9];
    matmul3(Ry, Rx, T);
    matmul3(Rz, T, R);
}

/* Sample-to-point vector in the laboratory frame for detector coordinates (d1, d2) [m]. */
static void lab_vector(const orc_geom *g, const double R[9], double d1, double d2, double t[3])
{
    double x[3] = {d1 - g->poni1, d2 - g->poni2, g->dist};
    for (int i = 0; i < 3; ++i) t[i] = R[3 * i] * x[0] + R[3 * i + 1] * x[1] + R[3 * i + 2] * x[2];
}

/* 2theta = atan(r / d) generalised to a tilted detector: angle between t and the beam. */
static double two_theta(const double t[3]) { return atan2(sqrt(t[0] * t[0] + t[1] * t[1]), t[2]); }

/* chi = atan(y / x) with y along dim1 and x along dim2, in degrees in [-180, 180]. */
static double chi_deg(const double t[3]) { return atan2(t[0], t[1]) * (180.0 / M_PI); }

/* Radial value in the requested unit: 2theta in degrees, q = 4 pi sin(2theta / 2) / lambda
 * in nm^-1, or r = dist * tan(2theta) in mm. */
static double radial(const orc_geom *g, int unit, const double t[3])
{
    double tth = two_theta(t);
    if (unit == ORC_UNIT_2TH_DEG) return tth * (180.0 / M_PI);
    if (unit == ORC_UNIT_Q_NM) return 4.0 * M_PI * sin(0.5 * tth) / g->wavelength * 1e-9;
    return g->dist * sqrt(t[0] * t[0] + t[1] * t[1]) / t[2] * 1e3;
}

/* Radial value and chi at an arbitrary detector point (d1, d2) [m]. */
void orc_position_at(const orc_geom *g, int unit, double d1, double d2, double *rad, double *chi)
{
    double R[9], t[3];
    orc_rotation(g->rot1, g->rot2, g->rot3, R);
    lab_vector(g, R, d1, d2, t);
    *rad = radial(g, unit, t);
    *chi = chi_deg(t);
}

/* Pixel corners (a, b), a in [0, ny], b in [0, nx]: arrays of (ny+1)*(nx+1), row-major. */
void orc_corner_positions(const orc_geom *g, int ny, int nx, int unit, double *rad, double *chi)
{
    double R[9], t[3];
    orc_rotation(g->rot1, g->rot2, g->rot3, R);
    for (int a = 0; a <= ny; ++a)
        for (int b = 0; b <= nx; ++b) {
            lab_vector(g, R, a * g->pixel1, b * g->pixel2, t);
            size_t k = (size_t)a * (nx + 1) + b;
            rad[k] = radial(g, unit, t);
            if (chi) chi[k] = chi_deg(t);
        }
}

/* Pixel centres (i + 1/2, j + 1/2): arrays of ny*nx, row-major. */
void orc_centre_positions(const orc_geom *g, int ny, int nx, int unit, double *rad, double *chi)
{
    double R[9], t[3];
    orc_rotation(g->rot1, g->rot2, g->rot3, R);
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            lab_vector(g, R, (i + 0.5) * g->pixel1, (j + 0.5) * g->pixel2, t);
            size_t k = (size_t)i * nx + j;
            rad[k] = radial(g, unit, t);
            if (chi) chi[k] = chi_deg(t);
        }
}

/* Solid-angle correction at pixel centres, relative to the PONI: (dist / |t|)^3, where
 * |t| is the sample-to-pixel distance (a pixel seen at incidence alpha from distance d
 * subtends A cos(alpha) / d^2 and cos(alpha) = dist / d).  The correction is named in
 * Sec. 5.3 (kernel timings); its formula is the textbook one. */
void orc_solid_angle(const orc_geom *g, int ny, int nx, double *out)
{
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            double x1 = (i + 0.5) * g->pixel1 - g->poni1;
            double x2 = (j + 0.5) * g->pixel2 - g->poni2;
            double d = sqrt(x1 * x1 + x2 * x2 + g->dist * g->dist);
            double c = g->dist / d;
            out[(size_t)i * nx + j] = c * c * c;
        }
}

/* Polarisation correction at pixel centres for a beam with polarisation factor f:
 * P = (1 + cos^2 2theta - f cos(2 chi) sin^2 2theta) / 2.  Named in Sec. 5.3; textbook
 * linear-polarisation formula, chi measured from the dim2 axis. */
void orc_polarization(const orc_geom *g, int ny, int nx, double f, double *out)
{
    double R[9], t[3];
    orc_rotation(g->rot1, g->rot2, g->rot3, R);
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            lab_vector(g, R, (i + 0.5) * g->pixel1, (j + 0.5) * g->pixel2, t);
            double tth = two_theta(t);
            double chi = atan2(t[0], t[1]);
            double c2t = cos(tth), s2t = sin(tth);
            out[(size_t)i * nx + j] = 0.5 * (1.0 + c2t * c2t - f * cos(2.0 * chi) * s2t * s2t);
        }
}

/* ------------------------------------------------------------------------------------ */
/* Polygon clipping and area (textbook Sutherland-Hodgman + shoelace).                   */
/* ------------------------------------------------------------------------------------ */

#define MAXV 32

/* Keep the part of polygon (ix, iy, n) with coordinate `axis` >= bound (keep_ge) or
 * <= bound (!keep_ge).  Returns the vertex count of the clipped polygon. */
static int clip_half(const double *ix, const double *iy, int n, double *ox, double *oy,
                     int axis, double bound, int keep_ge)
{
    int m = 0;
    for (int k = 0; k < n; ++k) {
        int k1 = (k + 1) % n;
        double cv = axis ? iy[k] : ix[k];
        double nv = axis ? iy[k1] : ix[k1];
        int cin = keep_ge ? (cv >= bound) : (cv <= bound);
        int nin = keep_ge ? (nv >= bound) : (nv <= bound);
        if (cin) {
            ox[m] = ix[k];
            oy[m] = iy[k];
            ++m;
        }
        if (cin != nin) {
            double s = (bound - cv) / (nv - cv);
            if (axis == 0) {
                ox[m] = bound;
                oy[m] = iy[k] + s * (iy[k1] - iy[k]);
            } else {
                ox[m] = ix[k] + s * (ix[k1] - ix[k]);
                oy[m] = bound;
            }
            ++m;
        }
    }
    return m;
}

static double shoelace(const double *x, const double *y, int n)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        int k1 = (k + 1) % n;
        s += x[k] * y[k1] - x[k1] * y[k];
    }
    return 0.5 * s;
}

/* |area| of quad (qx, qy) inside [xlo, xhi] x [ylo, yhi]; an infinite bound is skipped. */
static double clipped_area(const double qx[4], const double qy[4], double xlo, double xhi,
                           double ylo, double yhi)
{
    double ax[MAXV], ay[MAXV], bx[MAXV], by[MAXV];
    int n = 4;
    for (int k = 0; k < 4; ++k) {
        ax[k] = qx[k];
        ay[k] = qy[k];
    }
    if (!isinf(xlo)) { n = clip_half(ax, ay, n, bx, by, 0, xlo, 1); memcpy(ax, bx, sizeof(double) * n); memcpy(ay, by, sizeof(double) * n); }
    if (!isinf(xhi)) { n = clip_half(ax, ay, n, bx, by, 0, xhi, 0); memcpy(ax, bx, sizeof(double) * n); memcpy(ay, by, sizeof(double) * n); }
    if (!isinf(ylo)) { n = clip_half(ax, ay, n, bx, by, 1, ylo, 1); memcpy(ax, bx, sizeof(double) * n); memcpy(ay, by, sizeof(double) * n); }
    if (!isinf(yhi)) { n = clip_half(ax, ay, n, bx, by, 1, yhi, 0); memcpy(ax, bx, sizeof(double) * n); memcpy(ay, by, sizeof(double) * n); }
    if (n < 3) return 0.0;
    return fabs(shoelace(ax, ay, n));
}

/* ------------------------------------------------------------------------------------ */
/* Per-pixel contributions (Sec. 4).                                                      */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int32_t *bin;
    double *w;
    int n, cap;
} entry_list;

static int push(entry_list *L, int bin, double w)
{
    if (L->n == L->cap) {
        int cap = L->cap ? 2 * L->cap : 64;
        int32_t *b = (int32_t *)realloc(L->bin, sizeof(int32_t) * cap);
        if (!b) return ORC_ENOMEM;
        L->bin = b;
        double *ww = (double *)realloc(L->w, sizeof(double) * cap);
        if (!ww) return ORC_ENOMEM;
        L->w = ww;
        L->cap = cap;
    }
    L->bin[L->n] = bin;
    L->w[L->n] = w;
    ++L->n;
    return ORC_OK;
}

/* Sort one pixel's entries by bin and merge duplicates (same bin) by summing. */
static void sort_merge(entry_list *L, int start)
{
    for (int a = start + 1; a < L->n; ++a) {
        int32_t b = L->bin[a];
        double w = L->w[a];
        int c = a - 1;
        while (c >= start && L->bin[c] > b) {
            L->bin[c + 1] = L->bin[c];
            L->w[c + 1] = L->w[c];
            --c;
        }
        L->bin[c + 1] = b;
        L->w[c + 1] = w;
    }
    int m = start;
    for (int a = start; a < L->n; ++a) {
        if (m > start && L->bin[m - 1] == L->bin[a]) {
            L->w[m - 1] += L->w[a];
        } else {
            L->bin[m] = L->bin[a];
            L->w[m] = L->w[a];
            ++m;
        }
    }
    L->n = m;
}

/* Radial bin of a single position (no splitting): floor(f), last bin closed on the right
 * like numpy.histogram (Sec. 3.3). */
static int bin_none(double f, int npt)
{
    int b = (int)floor(f);
    return b > npt - 1 ? npt - 1 : b;
}

/* Bounding-box candidate range [*lo, *hi] of an interval [fmin, fmax] (Sec. 4.1): the
 * first bin holds fmin, the last bin is the one whose right edge reaches fmax. */
static void bbox_range(double fmin, double fmax, int clamp_top, int npt, int *lo, int *hi)
{
    int b0 = (int)floor(fmin);
    if (clamp_top && b0 > npt - 1) b0 = npt - 1;
    int b1 = (int)ceil(fmax) - 1;
    if (b1 < b0) b1 = b0;
    if (clamp_top && b1 > npt - 1) b1 = npt - 1;
    *lo = b0;
    *hi = b1;
}

/* Bounding-box weight of bin b for the interval [fmin, fmax] with candidate range
 * [blo, bhi] (Sec. 4.1): outermost bins get the part of the box they hold, the inner bins
 * share the rest evenly. */
static double bbox_weight(double fmin, double fmax, int blo, int bhi, int b)
{
    if (blo == bhi) return 1.0;
    double span = fmax - fmin;
    if (b == blo) return ((double)(blo + 1) - fmin) / span;
    if (b == bhi) return (fmax - (double)bhi) / span;
    return 1.0 / span;
}

/* Unwrap the azimuth of the four corners across the +-180 degree cut.  Returns 1 when the
 * span still exceeds 180 degrees (the pixel contains the beam centre: "singular"). */
static int unwrap_chi(double c[4])
{
    double mn = c[0], mx = c[0];
    for (int k = 1; k < 4; ++k) {
        if (c[k] < mn) mn = c[k];
        if (c[k] > mx) mx = c[k];
    }
    if (mx - mn <= 180.0) return 0;
    for (int k = 0; k < 4; ++k)
        if (c[k] < 0.0) c[k] += 360.0;
    mn = c[0];
    mx = c[0];
    for (int k = 1; k < 4; ++k) {
        if (c[k] < mn) mn = c[k];
        if (c[k] > mx) mx = c[k];
    }
    return (mx - mn > 180.0) ? 1 : 0;
}

typedef struct {
    int ny, nx, npt_rad, npt_azim, split;
    double lo, delta, dchi;
    const double *rad, *chi; /* corners or centres, per split */
} build_ctx;

static void corner_ids(const build_ctx *B, int i, int j, size_t k[4])
{
    size_t W = (size_t)B->nx + 1;
    k[0] = (size_t)i * W + j;           /* (i,   j)   */
    k[1] = (size_t)i * W + j + 1;       /* (i,   j+1) */
    k[2] = (size_t)(i + 1) * W + j + 1; /* (i+1, j+1) */
    k[3] = (size_t)(i + 1) * W + j;     /* (i+1, j)   */
}

/* 1D contributions of pixel (i, j). */
static int pixel_1d(const build_ctx *B, int i, int j, entry_list *L)
{
    int npt = B->npt_rad;
    if (B->split == ORC_SPLIT_NONE) {
        double f = (B->rad[(size_t)i * B->nx + j] - B->lo) / B->delta;
        return push(L, bin_none(f, npt), 1.0);
    }
    size_t k[4];
    corner_ids(B, i, j, k);
    double f[4];
    for (int c = 0; c < 4; ++c) f[c] = (B->rad[k[c]] - B->lo) / B->delta;
    double fmin = f[0], fmax = f[0];
    for (int c = 1; c < 4; ++c) {
        if (f[c] < fmin) fmin = f[c];
        if (f[c] > fmax) fmax = f[c];
    }
    int blo, bhi;
    bbox_range(fmin, fmax, 1, npt, &blo, &bhi);
    int use_bbox = (B->split == ORC_SPLIT_BBOX) || blo == bhi;
    double area[4096];
    double *areas = area;
    double total = 0.0;
    if (!use_bbox) {
        double chi[4];
        for (int c = 0; c < 4; ++c) chi[c] = B->chi[k[c]];
        if (unwrap_chi(chi)) {
            use_bbox = 1; /* singular pixel: the stated reading (radial bounding box) */
        } else {
            /* Sec. 4.2: area of the quad (straight edges in the radial/azimuth plane) inside
             * each bin, in coordinates relative to the first corner. */
            double qx[4], qy[4];
            for (int c = 0; c < 4; ++c) {
                qx[c] = f[c] - f[0];
                qy[c] = chi[c] - chi[0];
            }
            int nb = bhi - blo + 1;
            if (nb > 4096) areas = (double *)malloc(sizeof(double) * nb);
            if (!areas) return ORC_ENOMEM;
            for (int b = blo; b <= bhi; ++b) {
                double xlo = (b == 0) ? -INFINITY : (double)b - f[0];
                double xhi = (b == npt - 1) ? INFINITY : (double)(b + 1) - f[0];
                areas[b - blo] = clipped_area(qx, qy, xlo, xhi, -INFINITY, INFINITY);
                total += areas[b - blo];
            }
            if (!(total > 0.0)) use_bbox = 1; /* degenerate quad */
        }
    }
    int rc = ORC_OK;
    for (int b = blo; b <= bhi && rc == ORC_OK; ++b) {
        double w = use_bbox ? bbox_weight(fmin, fmax, blo, bhi, b) : areas[b - blo] / total;
        rc = push(L, b, w);
    }
    if (areas != area) free(areas);
    return rc;
}

/* 2D contributions of pixel (i, j): rows are chi_bin * npt_rad + rad_bin. */
static int pixel_2d(const build_ctx *B, int i, int j, entry_list *L)
{
    int npt = B->npt_rad, nch = B->npt_azim;
    int start = L->n;
    int rc = ORC_OK;
    if (B->split == ORC_SPLIT_NONE) {
        size_t p = (size_t)i * B->nx + j;
        double f = (B->rad[p] - B->lo) / B->delta;
        double gch = (B->chi[p] + 180.0) / B->dchi;
        int kc = (int)floor(gch) % nch;
        return push(L, kc * npt + bin_none(f, npt), 1.0);
    }
    size_t k[4];
    corner_ids(B, i, j, k);
    double f[4], chi[4], gc[4];
    for (int c = 0; c < 4; ++c) {
        f[c] = (B->rad[k[c]] - B->lo) / B->delta;
        chi[c] = B->chi[k[c]];
    }
    int singular = unwrap_chi(chi);
    for (int c = 0; c < 4; ++c) gc[c] = (chi[c] + 180.0) / B->dchi;
    double fmin = f[0], fmax = f[0], gmin = gc[0], gmax = gc[0];
    for (int c = 1; c < 4; ++c) {
        if (f[c] < fmin) fmin = f[c];
        if (f[c] > fmax) fmax = f[c];
        if (gc[c] < gmin) gmin = gc[c];
        if (gc[c] > gmax) gmax = gc[c];
    }
    int blo, bhi, klo, khi;
    bbox_range(fmin, fmax, 1, npt, &blo, &bhi);
    bbox_range(gmin, gmax, 0, nch, &klo, &khi);

    if (singular) {
        /* The stated reading for a singular pixel: radial bounding box times a uniform azimuth. */
        for (int b = blo; b <= bhi && rc == ORC_OK; ++b) {
            double wr = bbox_weight(fmin, fmax, blo, bhi, b);
            for (int kc = 0; kc < nch && rc == ORC_OK; ++kc) rc = push(L, kc * npt + b, wr / nch);
        }
        return rc;
    }
    int use_bbox = (B->split == ORC_SPLIT_BBOX);
    if (!use_bbox) {
        /* Sec. 4.2 in two dimensions: area of the quad inside each (radial, chi) bin. */
        double qx[4], qy[4];
        for (int c = 0; c < 4; ++c) {
            qx[c] = f[c] - f[0];
            qy[c] = gc[c] - gc[0];
        }
        int nr = bhi - blo + 1, nc = khi - klo + 1;
        double *areas = (double *)malloc(sizeof(double) * (size_t)nr * nc);
        if (!areas) return ORC_ENOMEM;
        double total = 0.0;
        for (int b = blo; b <= bhi; ++b) {
            double xlo = (b == 0) ? -INFINITY : (double)b - f[0];
            double xhi = (b == npt - 1) ? INFINITY : (double)(b + 1) - f[0];
            for (int kc = klo; kc <= khi; ++kc) {
                double a = clipped_area(qx, qy, xlo, xhi, (double)kc - gc[0], (double)(kc + 1) - gc[0]);
                areas[(size_t)(b - blo) * nc + (kc - klo)] = a;
                total += a;
            }
        }
        if (total > 0.0) {
            double kept = 0.0;
            for (size_t q = 0; q < (size_t)nr * nc; ++q)
                if (areas[q] > ORC_KEEP_2D * total) kept += areas[q];
            for (int b = blo; b <= bhi && rc == ORC_OK; ++b)
                for (int kc = klo; kc <= khi && rc == ORC_OK; ++kc) {
                    double a = areas[(size_t)(b - blo) * nc + (kc - klo)];
                    if (a > ORC_KEEP_2D * total) rc = push(L, (kc % nch) * npt + b, a / kept);
                }
        } else {
            use_bbox = 1; /* degenerate quad */
        }
        free(areas);
        if (rc != ORC_OK) return rc;
    }
    if (use_bbox) {
        /* Sec. 4.1 in two dimensions: product of the radial and azimuthal box fractions. */
        for (int b = blo; b <= bhi && rc == ORC_OK; ++b) {
            double wr = bbox_weight(fmin, fmax, blo, bhi, b);
            for (int kc = klo; kc <= khi && rc == ORC_OK; ++kc)
                rc = push(L, (kc % nch) * npt + b, wr * bbox_weight(gmin, gmax, klo, khi, kc));
        }
    }
    if (rc == ORC_OK) sort_merge(L, start);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* CSR assembly (Sec. 5.2 scatter-to-gather and 5.2.1 CSR).                               */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int ny, nx, npt_rad, npt_azim, nrows, split;
    double lo, hi, delta;
    int64_t nnz;
    int64_t *indptr; /* nrows + 1 */
    int32_t *indices;
    double *data;
} orc_csr;

void orc_csr_free(orc_csr *A)
{
    if (!A) return;
    free(A->indptr);
    free(A->indices);
    free(A->data);
    free(A);
}

/*
 * Build the bins x pixels weight matrix.
 *   split NONE: rad (and chi for 2D) are pixel-centre arrays of ny*nx.
 *   split BBOX/FULL: rad (and chi for 2D or 1D FULL) are corner arrays of (ny+1)*(nx+1).
 *   npt_azim == 0 selects 1D.  mask (nullable): nonzero = masked pixel, contributes nothing.
 * Returns NULL and sets *err on error (ORC_ERANGE: no unmasked pixel or zero radial range).
 */
orc_csr *orc_csr_build(int ny, int nx, const double *rad, const double *chi, const uint8_t *mask,
                       int npt_rad, int npt_azim, int split, int *err)
{
    *err = ORC_OK;
    if (ny <= 0 || nx <= 0) { *err = ORC_ESHAPE; return NULL; }
    if (npt_rad <= 0 || npt_azim < 0 || split < 0 || split > 2) { *err = ORC_EINVAL; return NULL; }
    int two_d = npt_azim > 0;
    if ((two_d || split == ORC_SPLIT_FULL) && !chi) { *err = ORC_EINVAL; return NULL; }

    /* Radial range: min and max over unmasked pixels of the positions the split reads. */
    double lo = INFINITY, hi = -INFINITY;
    size_t unmasked = 0;
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            size_t p = (size_t)i * nx + j;
            if (mask && mask[p]) continue;
            ++unmasked;
            if (split == ORC_SPLIT_NONE) {
                if (rad[p] < lo) lo = rad[p];
                if (rad[p] > hi) hi = rad[p];
            } else {
                build_ctx tmp;
                tmp.nx = nx;
                size_t k[4];
                corner_ids(&tmp, i, j, k);
                for (int c = 0; c < 4; ++c) {
                    if (rad[k[c]] < lo) lo = rad[k[c]];
                    if (rad[k[c]] > hi) hi = rad[k[c]];
                }
            }
        }
    if (unmasked == 0 || !(hi > lo)) { *err = ORC_ERANGE; return NULL; }

    build_ctx B;
    B.ny = ny; B.nx = nx; B.npt_rad = npt_rad; B.npt_azim = npt_azim; B.split = split;
    B.lo = lo;
    B.delta = (hi - lo) / npt_rad;
    B.dchi = two_d ? 360.0 / npt_azim : 0.0;
    B.rad = rad;
    B.chi = chi;

    /* Pixel-ordered triplet list (the "scatter" view). */
    entry_list L = {0, 0, 0, 0};
    int32_t *pix = NULL;
    size_t pix_cap = 0;
    for (int i = 0; i < ny && *err == ORC_OK; ++i)
        for (int j = 0; j < nx && *err == ORC_OK; ++j) {
            size_t p = (size_t)i * nx + j;
            if (mask && mask[p]) continue;
            int before = L.n;
            int rc = two_d ? pixel_2d(&B, i, j, &L) : pixel_1d(&B, i, j, &L);
            if (rc != ORC_OK) { *err = rc; break; }
            if ((size_t)L.n > pix_cap) {
                size_t cap = (size_t)L.cap;
                int32_t *np = (int32_t *)realloc(pix, sizeof(int32_t) * cap);
                if (!np) { *err = ORC_ENOMEM; break; }
                pix = np;
                pix_cap = cap;
            }
            for (int e = before; e < L.n; ++e) pix[e] = (int32_t)p;
        }
    if (*err != ORC_OK) { free(L.bin); free(L.w); free(pix); return NULL; }

    /* Counting sort by row: stable, so each row keeps ascending pixel order (the "gather"
     * view used for the matrix-vector product). */
    int nrows = two_d ? npt_rad * npt_azim : npt_rad;
    orc_csr *A = (orc_csr *)calloc(1, sizeof(orc_csr));
    if (!A) { *err = ORC_ENOMEM; free(L.bin); free(L.w); free(pix); return NULL; }
    A->ny = ny; A->nx = nx; A->npt_rad = npt_rad; A->npt_azim = npt_azim; A->nrows = nrows;
    A->split = split; A->lo = lo; A->hi = hi; A->delta = B.delta; A->nnz = L.n;
    A->indptr = (int64_t *)calloc((size_t)nrows + 1, sizeof(int64_t));
    A->indices = (int32_t *)malloc(sizeof(int32_t) * (L.n ? L.n : 1));
    A->data = (double *)malloc(sizeof(double) * (L.n ? L.n : 1));
    int64_t *fill = (int64_t *)calloc((size_t)nrows, sizeof(int64_t));
    if (!A->indptr || !A->indices || !A->data || !fill) {
        *err = ORC_ENOMEM;
        free(fill); free(L.bin); free(L.w); free(pix); orc_csr_free(A);
        return NULL;
    }
    for (int e = 0; e < L.n; ++e) A->indptr[L.bin[e] + 1] += 1;
    for (int r = 0; r < nrows; ++r) A->indptr[r + 1] += A->indptr[r];
    for (int e = 0; e < L.n; ++e) {
        int r = L.bin[e];
        int64_t pos = A->indptr[r] + fill[r]++;
        A->indices[pos] = pix[e];
        A->data[pos] = L.w[e];
    }
    free(fill); free(L.bin); free(L.w); free(pix);
    return A;
}

int64_t orc_csr_nnz(const orc_csr *A) { return A->nnz; }
int orc_csr_nrows(const orc_csr *A) { return A->nrows; }
void orc_csr_range(const orc_csr *A, double out[3]) { out[0] = A->lo; out[1] = A->hi; out[2] = A->delta; }

void orc_csr_copy(const orc_csr *A, int64_t *indptr, int32_t *indices, double *data)
{
    memcpy(indptr, A->indptr, sizeof(int64_t) * ((size_t)A->nrows + 1));
    memcpy(indices, A->indices, sizeof(int32_t) * (size_t)A->nnz);
    memcpy(data, A->data, sizeof(double) * (size_t)A->nnz);
}

/* ------------------------------------------------------------------------------------ */
/* Forward and adjoint (Sec. 5.2: integration as a sparse matrix-vector product).         */
/* ------------------------------------------------------------------------------------ */

/*
 * For every bin b: S_b = sum_p A_bp (img_p - dark_p), N_b = sum_p A_bp flat_p Omega_p P_p,
 * C_b = sum_p A_bp, I_b = S_b / N_b (0 where N_b == 0).  Null correction arrays mean
 * dark = 0, flat = Omega = P = 1.  Accumulated in double, in row order.
 */
void orc_integrate(int nrows, const int64_t *indptr, const int32_t *indices, const double *data,
                   const double *img, const double *dark, const double *flat, const double *sa,
                   const double *pol, double *I, double *S, double *N, double *C)
{
    for (int b = 0; b < nrows; ++b) {
        double s = 0.0, n = 0.0, c = 0.0;
        for (int64_t e = indptr[b]; e < indptr[b + 1]; ++e) {
            int32_t p = indices[e];
            double w = data[e];
            double v = img[p] - (dark ? dark[p] : 0.0);
            double nrm = (flat ? flat[p] : 1.0) * (sa ? sa[p] : 1.0) * (pol ? pol[p] : 1.0);
            s += w * v;
            n += w * nrm;
            c += w;
        }
        S[b] = s;
        N[b] = n;
        C[b] = c;
        I[b] = (n != 0.0) ? s / n : 0.0;
    }
}

/*
 * The paper's own normalisation (Sec. 6.4, the correction pass then the integration, whose
 * outputs are the ratio of two histograms): each pixel is corrected first,
 * c_p = (img_p - dark_p) / (flat_p Omega_p P_p), then U_b = sum_p A_bp c_p, C_b = sum_p A_bp
 * and I_b = U_b / C_b (0 where C_b = 0).  Absent corrections are 0 (dark) and 1.
 */
void orc_integrate_pixelnorm(int nrows, const int64_t *indptr, const int32_t *indices,
                             const double *data, const double *img, const double *dark,
                             const double *flat, const double *sa, const double *pol, double *I,
                             double *U, double *C)
{
    for (int b = 0; b < nrows; ++b) {
        double u = 0.0, c = 0.0;
        for (int64_t e = indptr[b]; e < indptr[b + 1]; ++e) {
            int32_t p = indices[e];
            double w = data[e];
            double v = img[p] - (dark ? dark[p] : 0.0);
            double nrm = (flat ? flat[p] : 1.0) * (sa ? sa[p] : 1.0) * (pol ? pol[p] : 1.0);
            u += w * (v / nrm);
            c += w;
        }
        U[b] = u;
        C[b] = c;
        I[b] = (c != 0.0) ? u / c : 0.0;
    }
}

/*
 * Propagated variance of the signal sum.  The paper states no error model; the reading used
 * here is counting statistics: a pixel's counts have a Poisson variance equal to their value
 * (clipped at 0), the dark current is a constant, and pixels are independent, so
 * V_b = sum_p A_bp^2 max(img_p, 0), and the standard error of I_b is sqrt(V_b) / N_b.
 */
void orc_variance(int nrows, const int64_t *indptr, const int32_t *indices, const double *data,
                  const double *img, double *V)
{
    for (int b = 0; b < nrows; ++b) {
        double v = 0.0;
        for (int64_t e = indptr[b]; e < indptr[b + 1]; ++e) {
            double w = data[e];
            double x = img[indices[e]];
            v += w * w * (x > 0.0 ? x : 0.0);
        }
        V[b] = v;
    }
}

/*
 * Adjoint of the forward with respect to the image and the flat field, for an upstream
 * gradient g_b = dL/dI_b:  dL/dimg_p = sum_b A_bp g_b / N_b,
 * dL/dflat_p = -Omega_p P_p sum_b A_bp g_b I_b / N_b (bins with N_b == 0 contribute 0).
 * Written as the transpose product (A^T u)_p = sum_b A_bp u_b, scattered row by row.
 * Either output may be NULL.
 */
void orc_backward(int nrows, int64_t npix, const int64_t *indptr, const int32_t *indices,
                  const double *data, const double *g, const double *I, const double *N,
                  const double *sa, const double *pol, double *g_img, double *g_flat)
{
    double *acc = (double *)calloc(npix ? (size_t)npix : 1, sizeof(double));
    if (g_img) memset(g_img, 0, sizeof(double) * (size_t)npix);
    for (int b = 0; b < nrows; ++b) {
        double u = (N[b] != 0.0) ? g[b] / N[b] : 0.0;
        double v = u * I[b];
        for (int64_t e = indptr[b]; e < indptr[b + 1]; ++e) {
            int32_t p = indices[e];
            double w = data[e];
            if (g_img) g_img[p] += w * u;
            if (acc) acc[p] += w * v;
        }
    }
    if (g_flat)
        for (int64_t p = 0; p < npix; ++p)
            g_flat[p] = -(sa ? sa[p] : 1.0) * (pol ? pol[p] : 1.0) * (acc ? acc[p] : 0.0);
    free(acc);
}

/*
 * Look-up-table layout of the matrix (Sec. 5.2, "scatter to gather"): for every output bin,
 * the pixels it takes its value from, as (pixel index, coefficient) pairs.  Every bin gets
 * the same number of slots, `width` = the largest number of entries in any bin; bin b's
 * slots hold its matrix row in column order, then padding pairs (index -1, coefficient 0).
 * Row-major: slot k of bin b is element b * width + k.
 */
int64_t orc_lut_width(int nrows, const int64_t *indptr)
{
    int64_t w = 0;
    for (int b = 0; b < nrows; ++b)
        if (indptr[b + 1] - indptr[b] > w) w = indptr[b + 1] - indptr[b];
    return w;
}

void orc_lut_from_csr(int nrows, const int64_t *indptr, const int32_t *indices, const double *data,
                      int64_t width, int32_t *idx, double *coef)
{
    for (int b = 0; b < nrows; ++b) {
        int64_t k = 0;
        for (int64_t e = indptr[b]; e < indptr[b + 1]; ++e, ++k) {
            idx[(int64_t)b * width + k] = indices[e];
            coef[(int64_t)b * width + k] = data[e];
        }
        for (; k < width; ++k) {
            idx[(int64_t)b * width + k] = -1;
            coef[(int64_t)b * width + k] = 0.0;
        }
    }
}

/*
 * The forward (the sums of orc_integrate) through the look-up table: each bin's slots in
 * order; a padding pair contributes nothing.
 */
void orc_integrate_lut(int nrows, int64_t width, const int32_t *idx, const double *coef,
                       const double *img, const double *dark, const double *flat, const double *sa,
                       const double *pol, double *I, double *S, double *N, double *C)
{
    for (int b = 0; b < nrows; ++b) {
        double s = 0.0, n = 0.0, c = 0.0;
        for (int64_t k = 0; k < width; ++k) {
            int32_t p = idx[(int64_t)b * width + k];
            if (p < 0) continue;
            double w = coef[(int64_t)b * width + k];
            double v = img[p] - (dark ? dark[p] : 0.0);
            double nrm = (flat ? flat[p] : 1.0) * (sa ? sa[p] : 1.0) * (pol ? pol[p] : 1.0);
            s += w * v;
            n += w * nrm;
            c += w;
        }
        S[b] = s;
        N[b] = n;
        C[b] = c;
        I[b] = (n != 0.0) ? s / n : 0.0;
    }
}
