// Adjoint of the forward integration with respect to the image and the flat field.
//
// With I_b = S_b / N_b, S_b = sum_p A_bp (img_p - dark_p), N_b = sum_p A_bp flat_p Om_p P_p:
//   dL/dimg_p  = sum_b A_bp g_b / N_b
//   dL/dflat_p = -Om_p P_p sum_b A_bp g_b I_b / N_b
// for an upstream gradient g_b = dL/dI_b.  The products A^T u are formed as a gather over
// the pixel-major (CSC) copy of the matrix built with the forward one: one thread per pixel
// reads its own column and writes its own outputs, so there are no atomics and the result
// is bit-reproducible.  FP32 column sums are Kahan-compensated.
#include <algorithm>

#include "common.cuh"

namespace azint {

namespace {

template <class AT>
__global__ void adjoint_rows_kernel(const AT *__restrict__ g, const AT *__restrict__ I,
                                    const AT *__restrict__ N, int nrows, AT *__restrict__ u,
                                    AT *__restrict__ v) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
        const AT n = N[r];
        const AT uu = n != AT(0) ? g[r] / n : AT(0);
        u[r] = uu;
        v[r] = uu * I[r];
    }
}

template <class AT, class WT>
__global__ void adjoint_pixels_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ row,
                                      const WT *__restrict__ w, const AT *__restrict__ u,
                                      const AT *__restrict__ v, const float *__restrict__ sa,
                                      const float *__restrict__ pol, int64_t npix,
                                      AT *__restrict__ g_img, AT *__restrict__ g_flat) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int a = ptr[p], b = ptr[p + 1];
        if (sizeof(AT) == 8) {
            double su = 0.0, sv = 0.0;
            for (int e = a; e < b; ++e) {
                const int r = row[e];
                const double ww = (double)w[e];
                su += ww * (double)u[r];
                sv += ww * (double)v[r];
            }
            if (g_img) g_img[p] = (AT)su;
            if (g_flat)
                g_flat[p] = (AT)(-(sa ? (double)sa[p] : 1.0) * (pol ? (double)pol[p] : 1.0) * sv);
        } else {
            Kahan ku{0.f, 0.f}, kv{0.f, 0.f};
            for (int e = a; e < b; ++e) {
                const int r = row[e];
                const float ww = (float)w[e];
                kahan_add(ku, ww, (float)u[r]);
                kahan_add(kv, ww, (float)v[r]);
            }
            if (g_img) g_img[p] = (AT)kahan_value(ku);
            if (g_flat)
                g_flat[p] = (AT)(-(sa ? sa[p] : 1.f) * (pol ? pol[p] : 1.f) * kahan_value(kv));
        }
    }
}

template <class AT, class WT>
int run_adjoint(const az_integrator *h, const AT *g, const AT *I, const AT *N, const float *sa,
                const float *pol, AT *g_img, AT *g_flat, const WT *w, cudaStream_t s) {
    AT *u = h->adj.as<AT>(), *v = u + h->nrows;  // [2][nrows] scratch owned by the integrator
    const int rb = std::min((h->nrows + 255) / 256, num_sms() * 4);
    adjoint_rows_kernel<AT><<<std::max(rb, 1), 256, 0, s>>>(g, I, N, h->nrows, u, v);
    AZ_CUDA(cudaGetLastError());
    const int64_t npix = (int64_t)h->ny * h->nx;
    const int64_t pb = std::min<int64_t>((npix + 255) / 256, (int64_t)num_sms() * 16);
    adjoint_pixels_kernel<AT, WT><<<(unsigned)std::max<int64_t>(pb, 1), 256, 0, s>>>(
        h->csc_ptr.as<int32_t>(), h->csc_row.as<int32_t>(), w, u, v, sa, pol, npix, g_img, g_flat);
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}

}  // namespace

int backward(const az_integrator *h, const void *g, const void *I, const void *N, const float *sa,
             const float *pol, int precision, void *g_img, void *g_flat, cudaStream_t s) {
    if (precision == AZ_PREC_FP64)
        return run_adjoint<double, double>(h, (const double *)g, (const double *)I, (const double *)N,
                                           sa, pol, (double *)g_img, (double *)g_flat,
                                           h->csc_w64.as<double>(), s);
    return run_adjoint<float, float>(h, (const float *)g, (const float *)I, (const float *)N, sa, pol,
                                     (float *)g_img, (float *)g_flat, h->csc_w32.as<float>(), s);
}

}  // namespace azint
