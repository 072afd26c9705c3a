// FP64 detector geometry (Sec. 3 coordinate list): pixel-corner / pixel-centre radial
// positions and azimuth, solid-angle and polarisation corrections.
//
// Compiled with -fmad=false: every product and sum below is rounded on its own, in the
// order written, so positions depend only on the libm-quality of sqrt (exact), atan2 and
// sin.  The rotation matrix is formed once on the host.
#include <cmath>

#include "common.cuh"

namespace azint {

namespace {

__device__ __forceinline__ void lab_vector(const GeomParams &g, double d1, double d2,
                                           double t[3]) {
    const double x0 = d1 - g.poni1, x1 = d2 - g.poni2, x2 = g.dist;
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = g.R[3 * i] * x0 + g.R[3 * i + 1] * x1 + g.R[3 * i + 2] * x2;
}

// Radial value in `unit` for the laboratory vector t (2theta in degrees, q in nm^-1,
// r = dist tan 2theta in mm).
__device__ __forceinline__ double radial_value(const GeomParams &g, int unit, const double t[3]) {
    const double rho = sqrt(t[0] * t[0] + t[1] * t[1]);
    const double tth = atan2(rho, t[2]);
    if (unit == AZ_UNIT_2TH_DEG) return tth * (180.0 / M_PI);
    if (unit == AZ_UNIT_Q_NM) return 4.0 * M_PI * sin(0.5 * tth) / g.wavelength * 1e-9;
    return g.dist * rho / t[2] * 1e3;
}

__global__ void positions_kernel(GeomParams g, int ny, int nx, int unit, int corners,
                                 double *__restrict__ rad, double *__restrict__ chi) {
    const int64_t w = corners ? (int64_t)nx + 1 : (int64_t)nx;
    const int64_t h = corners ? (int64_t)ny + 1 : (int64_t)ny;
    const int64_t n = w * h;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = k / w, b = k - a * w;
        double d1, d2;
        if (corners) {
            d1 = (double)a * g.pixel1;
            d2 = (double)b * g.pixel2;
        } else {
            d1 = ((double)a + 0.5) * g.pixel1;
            d2 = ((double)b + 0.5) * g.pixel2;
        }
        double t[3];
        lab_vector(g, d1, d2, t);
        rad[k] = radial_value(g, unit, t);
        if (chi) chi[k] = atan2(t[0], t[1]) * (180.0 / M_PI);
    }
}

__global__ void solid_angle_kernel(GeomParams g, int ny, int nx, float *__restrict__ out) {
    const int64_t n = (int64_t)ny * nx;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / nx, j = k - i * nx;
        const double x1 = ((double)i + 0.5) * g.pixel1 - g.poni1;
        const double x2 = ((double)j + 0.5) * g.pixel2 - g.poni2;
        const double d = sqrt(x1 * x1 + x2 * x2 + g.dist * g.dist);
        const double c = g.dist / d;
        out[k] = (float)(c * c * c);
    }
}

__global__ void polarization_kernel(GeomParams g, int ny, int nx, double f,
                                    float *__restrict__ out) {
    const int64_t n = (int64_t)ny * nx;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / nx, j = k - i * nx;
        double t[3];
        lab_vector(g, ((double)i + 0.5) * g.pixel1, ((double)j + 0.5) * g.pixel2, t);
        const double tth = atan2(sqrt(t[0] * t[0] + t[1] * t[1]), t[2]);
        const double chi = atan2(t[0], t[1]);
        const double c2t = cos(tth), s2t = sin(tth);
        out[k] = (float)(0.5 * (1.0 + c2t * c2t - f * cos(2.0 * chi) * s2t * s2t));
    }
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 32;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

int launch_positions(const GeomParams &g, int ny, int nx, int unit, int where, double *rad,
                     double *chi, cudaStream_t s) {
    const int corners = where == AZ_WHERE_CORNERS;
    const int64_t n = corners ? (int64_t)(ny + 1) * (nx + 1) : (int64_t)ny * nx;
    positions_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, ny, nx, unit, corners, rad, chi);
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}

}  // namespace azint

using namespace azint;

extern "C" int az_geometry_create(double dist, double poni1, double poni2, double rot1,
                                  double rot2, double rot3, double pixel1, double pixel2,
                                  double wavelength, az_geometry **out) {
    clear_error();
    if (!out) return fail(AZ_EINVAL, "az_geometry_create: out is NULL");
    *out = nullptr;
    if (!finite_pos(dist) || !finite_pos(pixel1) || !finite_pos(pixel2) || !finite_pos(wavelength))
        return fail(AZ_EINVAL, "az_geometry_create: dist, pixel sizes and wavelength must be finite and > 0");
    if (!std::isfinite(poni1) || !std::isfinite(poni2) || !std::isfinite(rot1) ||
        !std::isfinite(rot2) || !std::isfinite(rot3))
        return fail(AZ_EINVAL, "az_geometry_create: non-finite PONI or rotation");
    az_geometry *g = new (std::nothrow) az_geometry;
    if (!g) return fail(AZ_ENOMEM, "az_geometry_create: out of host memory");
    const double c1 = std::cos(rot1), s1 = std::sin(rot1);
    const double c2 = std::cos(rot2), s2 = std::sin(rot2);
    const double c3 = std::cos(rot3), s3 = std::sin(rot3);
    // Rz(rot3) Ry(rot2) Rx(rot1), expanded.
    const double R[9] = {c3 * c2, c3 * s2 * s1 - s3 * c1, c3 * s2 * c1 + s3 * s1,
                         s3 * c2, s3 * s2 * s1 + c3 * c1, s3 * s2 * c1 - c3 * s1,
                         -s2,     c2 * s1,                c2 * c1};
    for (int k = 0; k < 9; ++k) g->g.R[k] = R[k];
    g->g.dist = dist;
    g->g.poni1 = poni1;
    g->g.poni2 = poni2;
    g->g.pixel1 = pixel1;
    g->g.pixel2 = pixel2;
    g->g.wavelength = wavelength;
    g->rot1 = rot1;
    g->rot2 = rot2;
    g->rot3 = rot3;
    *out = g;
    return AZ_OK;
}

extern "C" void az_geometry_destroy(az_geometry *geom) { delete geom; }

extern "C" int az_geometry_rotation(const az_geometry *geom, double *R_host) {
    clear_error();
    if (!geom || !R_host) return fail(AZ_EINVAL, "az_geometry_rotation: NULL argument");
    for (int k = 0; k < 9; ++k) R_host[k] = geom->g.R[k];
    return AZ_OK;
}

extern "C" int az_geometry_positions(const az_geometry *geom, int ny, int nx, int unit,
                                     int where, double *rad_dev, double *chi_dev,
                                     az_stream_t stream) {
    clear_error();
    if (!geom || !rad_dev) return fail(AZ_EINVAL, "az_geometry_positions: NULL argument");
    if (ny < 1 || nx < 1) return fail(AZ_ESHAPE, "az_geometry_positions: ny, nx must be >= 1");
    if (unit < AZ_UNIT_2TH_DEG || unit > AZ_UNIT_R_MM)
        return fail(AZ_EINVAL, "az_geometry_positions: bad unit %d", unit);
    if (where != AZ_WHERE_CORNERS && where != AZ_WHERE_CENTRES)
        return fail(AZ_EINVAL, "az_geometry_positions: bad where %d", where);
    return launch_positions(geom->g, ny, nx, unit, where, rad_dev, chi_dev, (cudaStream_t)stream);
}

extern "C" int az_geometry_solid_angle(const az_geometry *geom, int ny, int nx, float *out_dev,
                                       az_stream_t stream) {
    clear_error();
    if (!geom || !out_dev) return fail(AZ_EINVAL, "az_geometry_solid_angle: NULL argument");
    if (ny < 1 || nx < 1) return fail(AZ_ESHAPE, "az_geometry_solid_angle: ny, nx must be >= 1");
    const int64_t n = (int64_t)ny * nx;
    solid_angle_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(geom->g, ny, nx, out_dev);
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}

extern "C" int az_geometry_polarization(const az_geometry *geom, int ny, int nx, double factor,
                                        float *out_dev, az_stream_t stream) {
    clear_error();
    if (!geom || !out_dev) return fail(AZ_EINVAL, "az_geometry_polarization: NULL argument");
    if (ny < 1 || nx < 1) return fail(AZ_ESHAPE, "az_geometry_polarization: ny, nx must be >= 1");
    if (!std::isfinite(factor)) return fail(AZ_EINVAL, "az_geometry_polarization: bad factor");
    const int64_t n = (int64_t)ny * nx;
    polarization_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(geom->g, ny, nx,
                                                                          factor, out_dev);
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}
