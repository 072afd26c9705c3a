// The look-up-table (LUT) layout of the matrix (Sec. 5.2) and the forward through it.
//
// The table lists, for every output row, the (pixel index, coefficient) pairs the row gathers
// from, every row padded with pairs (-1, 0) to the length of the longest row (the width).  It
// is an array of pairs (Sec. 5.2.1 contrasts this array-of-structures form with the
// structure-of-arrays CSR), stored slot-major on the device, [width][nrows]: the threads of a
// warp take consecutive rows, so at every step they read 32 consecutive pairs.
//
// One frame through the table is three launches, mirroring the steps of Sec. 6.4:
//   lut_correct_kernel  cast and correction pass over the pixels: (img - dark, flat * Omega * P)
//                       per pixel, one 8- or 16-byte pair, so that a table entry costs one
//                       gather whatever corrections are given;
//   lut_sums_kernel     every row cut into chunks of kc slots; thread (row, chunk) sums
//                       w * value, w * normalisation and w over its slots in order and stops
//                       at the first padding pair (rows end in padding only);
//   lut_finish_kernel   per row, the chunk sums combined in chunk order (FP32: compensated),
//                       then I = S / N (0 where N = 0).
// The chunking keeps the GPU busy when there are few rows (1000 bins of a 1D pattern): the
// grid has about 2048 threads per SM whatever the number of rows.
#include <algorithm>

#include "common.cuh"

using namespace azint;

namespace {

struct Pair32 {
    int32_t pix;
    float w;
};
struct __align__(16) Pair64 {
    int32_t pix, pad;
    double w;
};
static_assert(sizeof(Pair32) == 8 && sizeof(Pair64) == 16, "table pair sizes");

// Streaming loads of one pair (the table is read once per frame).
__device__ __forceinline__ Pair32 load_pair(const Pair32 *p) {
    const int2 v = __ldcs(reinterpret_cast<const int2 *>(p));
    return Pair32{v.x, __int_as_float(v.y)};
}
__device__ __forceinline__ Pair64 load_pair(const Pair64 *p) {
    const int4 v = __ldcs(reinterpret_cast<const int4 *>(p));
    Pair64 r;
    r.pix = v.x;
    r.pad = v.y;
    r.w = __hiloint2double(v.w, v.z);
    return r;
}

constexpr int kFinishWarpMin = 8;  // from this many chunks on, one warp combines a row

__global__ void row_len_max_kernel(const int32_t *ptr, int nrows, int *out) {
    int m = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nrows; b += gridDim.x * blockDim.x)
        m = max(m, ptr[b + 1] - ptr[b]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

template <class P>
__global__ void lut_fill_kernel(const int32_t *ptr, const int32_t *idx, const double *w64, int nrows,
                                int64_t width, P *lut) {
    const int64_t total = width * (int64_t)nrows;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / nrows;
        const int b = (int)(t - k * nrows);
        const int32_t e0 = ptr[b], len = ptr[b + 1] - e0;
        P p{};
        if (k < len) {
            p.pix = idx[e0 + k];
            p.w = (decltype(p.w))w64[e0 + k];
        } else {
            p.pix = -1;
            p.w = 0;
        }
        lut[t] = p;
    }
}

template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <class T, int DT>
__device__ __forceinline__ T cast_pixel(const void *img, int64_t p) {
    if (DT == AZ_DTYPE_F32) return (T) static_cast<const float *>(img)[p];
    if (DT == AZ_DTYPE_U32) {
        const uint32_t u = static_cast<const uint32_t *>(img)[p];
        if constexpr (sizeof(T) == 4) return __uint2float_rn(u);
        else return (T)u;
    }
    const int32_t i = static_cast<const int32_t *>(img)[p];
    if constexpr (sizeof(T) == 4) return __int2float_rn(i);
    else return (T)i;
}

// Pixel pass: (cast(img) - dark, ((1 * flat) * Omega) * P) per pixel.
template <class T, int DT>
__global__ void lut_correct_kernel(const void *img, const float *dark, const float *flat, const float *sa,
                                   const float *pol, int64_t npix, typename Vec2<T>::type *vals) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        T v = cast_pixel<T, DT>(img, p);
        if (dark) v = v - (T)__ldg(dark + p);
        T n = (T)1;
        if (flat) n = n * (T)__ldg(flat + p);
        if (sa) n = n * (T)__ldg(sa + p);
        if (pol) n = n * (T)__ldg(pol + p);
        typename Vec2<T>::type o;
        o.x = v;
        o.y = n;
        vals[p] = o;
    }
}

// Accumulators: compensated FP32 (Sec. 5.2.2) or plain FP64.
struct AccF {
    Kahan k{0.f, 0.f};
    __device__ __forceinline__ void add(float w, float v) { kahan_add(k, w, v); }
    __device__ __forceinline__ float value() const { return kahan_value(k); }
};
struct AccD {
    double s = 0.0;
    __device__ __forceinline__ void add(double w, double v) { s = __fma_rn(w, v, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <class T> struct AccOf;
template <> struct AccOf<float> { using type = AccF; };
template <> struct AccOf<double> { using type = AccD; };

// Thread (row b, chunk c) sums slots [c kc, min((c + 1) kc, width)) of row b.  Pairs are read
// four at a time (all four lie inside the table, padding included) so that four loads and
// then four gathers are in flight; a padding pair ends the row.  Partial sums are written to
// part[q][b][c], q = 0 signal, 1 normalisation, 2 count.
template <class T, class P>
__global__ void __launch_bounds__(256) lut_sums_kernel(const P *__restrict__ lut,
                                                       const typename Vec2<T>::type *__restrict__ vals,
                                                       int nrows, int64_t width, int64_t kc, int nchunk,
                                                       T *__restrict__ part) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (b >= nrows) return;
    using A = typename AccOf<T>::type;
    A S, N, C;
    const int64_t k0 = (int64_t)c * kc, k1 = min(width, k0 + kc);
    const P *col = lut + b;
    bool done = false;
    int64_t k = k0;
    for (; k + 4 <= k1 && !done; k += 4) {
        P p[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = load_pair(col + (k + j) * nrows);
        typename Vec2<T>::type x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (p[j].pix >= 0) x[j] = __ldg(vals + p[j].pix);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (p[j].pix < 0) {
                done = true;
                break;
            }
            S.add((T)p[j].w, x[j].x);
            N.add((T)p[j].w, x[j].y);
            C.add((T)p[j].w, (T)1);
        }
    }
    for (; k < k1 && !done; ++k) {
        const P p = load_pair(col + k * nrows);
        if (p.pix < 0) break;
        const typename Vec2<T>::type x = __ldg(vals + p.pix);
        S.add((T)p.w, x.x);
        N.add((T)p.w, x.y);
        C.add((T)p.w, (T)1);
    }
    const size_t o = (size_t)b * nchunk + c, q = (size_t)nrows * nchunk;
    part[o] = S.value();
    part[q + o] = N.value();
    part[2 * q + o] = C.value();
}

template <class T> struct Sum;
template <> struct Sum<float> {
    Kahan k{0.f, 0.f};
    __device__ __forceinline__ void add(float v) { kahan_add(k, 1.f, v); }
    __device__ __forceinline__ void merge_lower_left(int m) {
        const Kahan o = shfl_xor(k, m);
        if ((threadIdx.x & m) != 0) {
            Kahan l = o;
            kahan_merge(l, k);
            k = l;
        } else {
            kahan_merge(k, o);
        }
    }
    __device__ __forceinline__ float value() const { return kahan_value(k); }
};
template <> struct Sum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ void merge_lower_left(int m) {
        const double o = __shfl_xor_sync(0xffffffffu, s, m);
        s = (threadIdx.x & m) != 0 ? o + s : s + o;
    }
    __device__ __forceinline__ double value() const { return s; }
};

template <class T>
__device__ __forceinline__ void write_row(int b, T s, T n, T c, T *oI, T *oS, T *oN, T *oC) {
    if (oS) oS[b] = s;
    if (oN) oN[b] = n;
    if (oC) oC[b] = c;
    if (oI) oI[b] = n != (T)0 ? s / n : (T)0;
}

// Few chunks: one thread per row adds its chunks in order.
template <class T>
__global__ void lut_finish_thread_kernel(const T *part, int nrows, int nchunk, T *oI, T *oS, T *oN, T *oC) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nrows) return;
    const size_t q = (size_t)nrows * nchunk;
    Sum<T> s, n, c;
    for (int j = 0; j < nchunk; ++j) {
        const size_t o = (size_t)b * nchunk + j;
        s.add(part[o]);
        n.add(part[q + o]);
        c.add(part[2 * q + o]);
    }
    write_row<T>(b, s.value(), n.value(), c.value(), oI, oS, oN, oC);
}

// Many chunks: one warp per row; lane l adds chunks l, l + 32, ... in order, then the lanes
// are combined by a butterfly with the lower lane's sum on the left.
template <class T>
__global__ void lut_finish_warp_kernel(const T *part, int nrows, int nchunk, T *oI, T *oS, T *oN, T *oC) {
    const int b = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nrows) return;  // whole warps leave together
    const size_t q = (size_t)nrows * nchunk;
    Sum<T> s, n, c;
    for (int j = lane; j < nchunk; j += 32) {
        const size_t o = (size_t)b * nchunk + j;
        s.add(part[o]);
        n.add(part[q + o]);
        c.add(part[2 * q + o]);
    }
    for (int m = 1; m < 32; m <<= 1) {
        s.merge_lower_left(m);
        n.merge_lower_left(m);
        c.merge_lower_left(m);
    }
    if (lane == 0) write_row<T>(b, s.value(), n.value(), c.value(), oI, oS, oN, oC);
}

int blocks_for(int64_t n, int per) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, (int64_t)num_sms() * 16));
}

// Chunks per row: about 2048 threads per SM in all, at least 16 slots per chunk.
void chunking(const az_integrator *h, int &nchunk, int64_t &kc) {
    const int64_t want = ((int64_t)num_sms() * 2048 + h->nrows - 1) / std::max(h->nrows, 1);
    const int64_t most = std::max<int64_t>(1, (h->lut_width + 15) / 16);
    nchunk = (int)std::max<int64_t>(1, std::min<int64_t>({want, most, 65535}));
    kc = (h->lut_width + nchunk - 1) / nchunk;
    if (kc < 1) kc = 1;
    nchunk = (int)std::max<int64_t>(1, (h->lut_width + kc - 1) / kc);
}

template <class T, class P>
int lut_run(const az_integrator *h, const void *img, int dtype, const float *dark, const float *flat,
            const float *sa, const float *pol, void *oI, void *oS, void *oN, void *oC, cudaStream_t s) {
    const int64_t npix = (int64_t)h->ny * h->nx;
    using V = typename Vec2<T>::type;
    V *vals = h->lut_vals.as<V>();
    {
        ProfScope ps(&h->prof, 4, s);
        const int g = blocks_for(npix, 256);
        switch (dtype) {
            case AZ_DTYPE_F32: lut_correct_kernel<T, AZ_DTYPE_F32><<<g, 256, 0, s>>>(img, dark, flat, sa, pol, npix, vals); break;
            case AZ_DTYPE_U32: lut_correct_kernel<T, AZ_DTYPE_U32><<<g, 256, 0, s>>>(img, dark, flat, sa, pol, npix, vals); break;
            default: lut_correct_kernel<T, AZ_DTYPE_I32><<<g, 256, 0, s>>>(img, dark, flat, sa, pol, npix, vals); break;
        }
        AZ_CUDA(cudaGetLastError());
    }
    int nchunk = 1;
    int64_t kc = 1;
    chunking(h, nchunk, kc);
    T *part = h->lut_part.as<T>();
    const P *lut = static_cast<const P *>(sizeof(T) == 4 ? h->lut32.p : h->lut64.p);
    {
        ProfScope ps(&h->prof, 2, s);
        if (h->lut_width > 0) {
            dim3 grid((unsigned)((h->nrows + 255) / 256), (unsigned)nchunk);
            lut_sums_kernel<T, P><<<grid, 256, 0, s>>>(lut, vals, h->nrows, h->lut_width, kc, nchunk, part);
        } else {
            AZ_CUDA(cudaMemsetAsync(part, 0, sizeof(T) * 3 * (size_t)h->nrows, s));
        }
        AZ_CUDA(cudaGetLastError());
    }
    {
        ProfScope ps(&h->prof, 3, s);
        T *I = static_cast<T *>(oI), *S = static_cast<T *>(oS), *N = static_cast<T *>(oN), *C = static_cast<T *>(oC);
        if (nchunk >= kFinishWarpMin)
            lut_finish_warp_kernel<T><<<(unsigned)(((int64_t)h->nrows * 32 + 255) / 256), 256, 0, s>>>(part, h->nrows, nchunk, I, S, N, C);
        else
            lut_finish_thread_kernel<T><<<(unsigned)((h->nrows + 255) / 256), 256, 0, s>>>(part, h->nrows, nchunk, I, S, N, C);
        AZ_CUDA(cudaGetLastError());
    }
    return AZ_OK;
}

}  // namespace

namespace azint {

int lut_build(az_integrator *h, int precision, cudaStream_t s) {
    if (precision != AZ_PREC_FP64 && precision != AZ_PREC_FP32_COMP)
        return fail(AZ_EINVAL, "az_lut_build: bad precision %d", precision);
    DevBuf wmax;
    AZ_TRY(wmax.alloc(sizeof(int)));
    AZ_CUDA(cudaMemsetAsync(wmax.p, 0, sizeof(int), s));
    row_len_max_kernel<<<blocks_for(h->nrows, 256), 256, 0, s>>>(h->csr_ptr.as<int32_t>(), h->nrows, wmax.as<int>());
    AZ_CUDA(cudaGetLastError());
    int width = 0;
    AZ_CUDA(cudaMemcpyAsync(&width, wmax.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    const bool fp64 = precision == AZ_PREC_FP64;
    const int64_t slots = (int64_t)width * h->nrows;
    DevBuf &tab = fp64 ? h->lut64 : h->lut32;
    // a table of the other precision built for another width is dropped
    if ((fp64 ? h->lut32 : h->lut64).p && h->lut_width != width) (fp64 ? h->lut32 : h->lut64).release();
    AZ_TRY(tab.alloc((size_t)std::max<int64_t>(slots, 1) * (fp64 ? sizeof(Pair64) : sizeof(Pair32))));
    h->lut_width = width;
    const size_t val_bytes = (size_t)h->ny * h->nx * (fp64 ? sizeof(double2) : sizeof(float2));
    if (h->lut_vals.bytes < val_bytes) AZ_TRY(h->lut_vals.alloc(val_bytes));
    int nchunk = 1;
    int64_t kc = 1;
    chunking(h, nchunk, kc);
    const size_t part_bytes = 3 * (size_t)h->nrows * (size_t)nchunk * (fp64 ? sizeof(double) : sizeof(float));
    if (h->lut_part.bytes < part_bytes) AZ_TRY(h->lut_part.alloc(part_bytes));
    if (slots > 0) {
        const int g = blocks_for(slots, 256);
        if (fp64)
            lut_fill_kernel<Pair64><<<g, 256, 0, s>>>(h->csr_ptr.as<int32_t>(), h->csr_idx.as<int32_t>(),
                                                      h->csr_w64.as<double>(), h->nrows, width, h->lut64.as<Pair64>());
        else
            lut_fill_kernel<Pair32><<<g, 256, 0, s>>>(h->csr_ptr.as<int32_t>(), h->csr_idx.as<int32_t>(),
                                                      h->csr_w64.as<double>(), h->nrows, width, h->lut32.as<Pair32>());
        AZ_CUDA(cudaGetLastError());
    }
    return AZ_OK;
}

int lut_forward(const az_integrator *h, const void *img, int dtype, const float *dark, const float *flat,
                const float *sa, const float *pol, int precision, void *oI, void *oS, void *oN, void *oC,
                cudaStream_t s) {
    az_integrator *m = const_cast<az_integrator *>(h);  // the table is built on first use
    if (precision == AZ_PREC_FP64) {
        if (!h->lut64.p) AZ_TRY(lut_build(m, AZ_PREC_FP64, s));
        return lut_run<double, Pair64>(h, img, dtype, dark, flat, sa, pol, oI, oS, oN, oC, s);
    }
    if (!h->lut32.p) AZ_TRY(lut_build(m, AZ_PREC_FP32_COMP, s));
    return lut_run<float, Pair32>(h, img, dtype, dark, flat, sa, pol, oI, oS, oN, oC, s);
}

int lut_export(const az_integrator *h, int64_t *width, int32_t *pix, float *c32, double *c64) {
    if (width) *width = h->lut_width;
    if (!pix && !c32 && !c64) return AZ_OK;
    if ((c64 && !h->lut64.p) || (c32 && !h->lut32.p) || (pix && !h->lut32.p && !h->lut64.p))
        return fail(AZ_EINVAL, "az_lut_export: the table of that precision is not built");
    const int64_t slots = h->lut_width * h->nrows;
    const bool use64 = c64 || !h->lut32.p;
    std::vector<Pair64> t64;
    std::vector<Pair32> t32;
    if (c64 || (pix && use64)) {
        t64.resize((size_t)slots);
        AZ_CUDA(cudaMemcpy(t64.data(), h->lut64.p, sizeof(Pair64) * (size_t)slots, cudaMemcpyDeviceToHost));
    }
    if (c32 || (pix && !use64)) {
        t32.resize((size_t)slots);
        AZ_CUDA(cudaMemcpy(t32.data(), h->lut32.p, sizeof(Pair32) * (size_t)slots, cudaMemcpyDeviceToHost));
    }
    // device order [width][nrows] -> row-major [nrows][width]
    for (int64_t k = 0; k < h->lut_width; ++k)
        for (int b = 0; b < h->nrows; ++b) {
            const size_t dsrc = (size_t)(k * h->nrows + b), ddst = (size_t)((int64_t)b * h->lut_width + k);
            if (pix) pix[ddst] = use64 ? t64[dsrc].pix : t32[dsrc].pix;
            if (c64) c64[ddst] = t64[dsrc].w;
            if (c32) c32[ddst] = t32[dsrc].w;
        }
    return AZ_OK;
}

}  // namespace azint

extern "C" int az_lut_build(az_integrator *h, int precision, az_stream_t stream) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_lut_build: NULL integrator");
    return lut_build(h, precision, (cudaStream_t)stream);
}

extern "C" int az_lut_export(const az_integrator *h, int64_t *width, int32_t *pixel_host, float *coef32_host,
                             double *coef64_host) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_lut_export: NULL integrator");
    return lut_export(h, width, pixel_host, coef32_host, coef64_host);
}

extern "C" int az_integrate_lut(az_integrator *h, const void *image_dev, int image_dtype, const float *dark,
                                const float *flat, const float *solid_angle, const float *polarization,
                                int precision, void *out_I, void *out_sum_signal, void *out_sum_norm,
                                void *out_count, az_stream_t stream) {
    clear_error();
    AZ_TRY(check_forward(h, image_dev, image_dtype, dark, flat, solid_angle, polarization, "az_integrate_lut"));
    if (precision != AZ_PREC_FP64 && precision != AZ_PREC_FP32_COMP)
        return fail(AZ_EINVAL, "az_integrate_lut: bad precision %d", precision);
    h->last_stream = (cudaStream_t)stream;
    return lut_forward(h, image_dev, image_dtype, dark, flat, solid_angle, polarization, precision, out_I,
                       out_sum_signal, out_sum_norm, out_count, (cudaStream_t)stream);
}

extern "C" int az_set_layout(az_integrator *h, int layout) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_set_layout: NULL integrator");
    if (layout != AZ_LAYOUT_TILED && layout != AZ_LAYOUT_LUT)
        return fail(AZ_EINVAL, "az_set_layout: bad layout %d", layout);
    h->layout = layout;
    return AZ_OK;
}
