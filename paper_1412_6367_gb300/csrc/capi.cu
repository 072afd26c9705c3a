// C ABI of the library: argument validation, handle lifetime, error strings, build
// orchestration, the end-to-end host-buffer path and the tuner.  The device work is done by
// the kernels in geometry.cu, csr_build.cu, integrate.cu, lut.cu and backward.cu (the
// allocation-free entry point and the wait self-test have their own files); the only kernel
// here fills the tuner's synthetic frames.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"

namespace azint {

namespace {
thread_local char g_err[512] = "";

bool aligned4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

__global__ void fill_frames_kernel(uint32_t *out, int64_t n, uint32_t seed) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)k * 2654435761u ^ seed;
        x ^= x >> 16;
        x *= 2246822519u;
        x ^= x >> 13;
        out[k] = x & 1023u;
    }
}

int alloc_scratch(az_integrator *h) {
    const size_t nseg = (size_t)std::max(h->tl.nseg, 1);
    const size_t single = 3 * nseg * sizeof(double);
    const size_t frames = (size_t)kMaxFramesPerLaunch * nseg * sizeof(float);
    h->partial_bytes = std::max(single, frames);
    AZ_TRY(h->partial.alloc(h->partial_bytes));
    AZ_TRY(h->norm.alloc(sizeof(float) * 2 * (size_t)h->nrows));
    AZ_TRY(h->adj.alloc(sizeof(double) * 2 * (size_t)h->nrows));
    return AZ_OK;
}

int finish_build(az_integrator *h, cudaStream_t s) {
    // defaults measured on the Pilatus-6M workload (1D) and the 2048 x 2048 cake (2D, whose
    // bins are compact in both directions); az_autotune refines them per matrix
    int th = h->npt_azim > 0 ? 32 : 8, tw = h->npt_azim > 0 ? 64 : 224;
    if (build_tiled_layout(h, th, tw, s) != AZ_OK) {  // a denser matrix: smaller tiles
        th = 8;
        tw = 64;
        AZ_TRY(build_tiled_layout(h, th, tw, s));
    }
    h->frames_per_pass = 8;
    h->rows_per_warp = 32 / h->frames_per_pass;
    AZ_TRY(alloc_scratch(h));
    AZ_TRY(h->status.alloc(sizeof(int)));
    AZ_CUDA(cudaMemsetAsync(h->status.p, 0, sizeof(int), s));
    AZ_CUDA(cudaStreamSynchronize(s));
    // the allocation-free entry point's fixed array and kernels, loaded at set-up
    return noalloc_setup();
}

int check_build_args(int ny, int nx, int npt_rad, int npt_azim, int unit, int split) {
    if (ny < 1 || nx < 1) return fail(AZ_ESHAPE, "csr_build: ny, nx must be >= 1 (got %d, %d)", ny, nx);
    if ((int64_t)ny * nx >= INT32_MAX) return fail(AZ_ESHAPE, "csr_build: more than 2^31 - 1 pixels");
    if (npt_rad < 1) return fail(AZ_EINVAL, "csr_build: npt_rad must be >= 1");
    if (npt_azim < 0) return fail(AZ_EINVAL, "csr_build: npt_azim must be >= 0");
    if ((int64_t)npt_rad * std::max(npt_azim, 1) >= (1ll << 30))
        return fail(AZ_EINVAL, "csr_build: too many bins");
    if (unit < AZ_UNIT_2TH_DEG || unit > AZ_UNIT_R_MM) return fail(AZ_EINVAL, "csr_build: bad unit %d", unit);
    if (split < AZ_SPLIT_NONE || split > AZ_SPLIT_FULL) return fail(AZ_EINVAL, "csr_build: bad split %d", split);
    return AZ_OK;
}

int build_common(int ny, int nx, const double *rad, const double *chi, int npt_rad, int npt_azim,
                 int unit, int split, const uint8_t *mask, cudaStream_t s, az_integrator **out) {
    az_integrator *h = new (std::nothrow) az_integrator;
    if (!h) return fail(AZ_ENOMEM, "csr_build: out of host memory");
    cudaGetDevice(&h->device);
    int rc = build_integrator(ny, nx, rad, chi, npt_rad, npt_azim, unit, split, mask, s, h);
    if (rc == AZ_OK) rc = finish_build(h, s);
    if (rc != AZ_OK) {
        cudaStreamSynchronize(s);
        delete h;
        return rc;
    }
    *out = h;
    return AZ_OK;
}

}  // namespace

int check_forward(const az_integrator *h, const void *image, int dtype, const float *dark,
                  const float *flat, const float *sa, const float *pol, const char *who) {
    if (!h) return fail(AZ_EINVAL, "%s: NULL integrator", who);
    if (!image) return fail(AZ_EINVAL, "%s: NULL image", who);
    if (dtype < AZ_DTYPE_F32 || dtype > AZ_DTYPE_I32) return fail(AZ_EINVAL, "%s: bad image dtype %d", who, dtype);
    const void *ptrs[5] = {image, dark, flat, sa, pol};
    for (const void *p : ptrs)
        if (p && !aligned4(p)) return fail(AZ_EINVAL, "%s: arrays must be 4-byte aligned", who);
    return AZ_OK;
}

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

int multi_create(az_integrator *const *hs, int n, const void *const *images, int dtype,
                 const float *const *darks, const float *const *flats, const float *const *sas,
                 const float *const *pols, float *const *oI, float *const *oS, float *const *oN,
                 float *const *oC, void **out);
int multi_launch(void *plan, int use_graph, cudaStream_t s);
void multi_destroy(void *plan);

}  // namespace azint

using namespace azint;

struct az_multi {
    void *plan = nullptr;
};

extern "C" const char *az_last_error(void) { return g_err; }

extern "C" int az_csr_build(const az_geometry *geom, int ny, int nx, int npt_rad, int npt_azim,
                            int unit, int split, const uint8_t *mask_dev, az_stream_t stream,
                            az_integrator **out) {
    clear_error();
    if (!geom || !out) return fail(AZ_EINVAL, "az_csr_build: NULL argument");
    *out = nullptr;
    AZ_TRY(check_build_args(ny, nx, npt_rad, npt_azim, unit, split));
    cudaStream_t s = (cudaStream_t)stream;
    const bool corners = split != AZ_SPLIT_NONE;
    const bool need_chi = npt_azim > 0 || split == AZ_SPLIT_FULL;
    const int64_t npos = corners ? (int64_t)(ny + 1) * (nx + 1) : (int64_t)ny * nx;
    DevBuf rad, chi;
    AZ_TRY(rad.alloc(sizeof(double) * npos));
    if (need_chi) AZ_TRY(chi.alloc(sizeof(double) * npos));
    AZ_TRY(launch_positions(geom->g, ny, nx, unit, corners ? AZ_WHERE_CORNERS : AZ_WHERE_CENTRES,
                            rad.as<double>(), need_chi ? chi.as<double>() : nullptr, s));
    const int rc = build_common(ny, nx, rad.as<double>(), need_chi ? chi.as<double>() : nullptr,
                                npt_rad, npt_azim, unit, split, mask_dev, s, out);
    cudaStreamSynchronize(s);
    return rc;
}

extern "C" int az_csr_build_from_positions(int ny, int nx, const double *rad_dev,
                                           const double *chi_dev, int npt_rad, int npt_azim,
                                           int split, const uint8_t *mask_dev,
                                           az_stream_t stream, az_integrator **out) {
    clear_error();
    if (!rad_dev || !out) return fail(AZ_EINVAL, "az_csr_build_from_positions: NULL argument");
    *out = nullptr;
    AZ_TRY(check_build_args(ny, nx, npt_rad, npt_azim, AZ_UNIT_2TH_DEG, split));
    if ((npt_azim > 0 || split == AZ_SPLIT_FULL) && !chi_dev)
        return fail(AZ_EINVAL, "az_csr_build_from_positions: chi positions are required");
    return build_common(ny, nx, rad_dev, (npt_azim > 0 || split == AZ_SPLIT_FULL) ? chi_dev : nullptr,
                        npt_rad, npt_azim, -1, split, mask_dev, (cudaStream_t)stream, out);
}

extern "C" int az_csr_import(int ny, int nx, int npt_rad, int npt_azim, int unit, int split,
                             const int32_t *indptr_host, const int32_t *indices_host,
                             const double *data_host, double lo, double hi, az_stream_t stream,
                             az_integrator **out) {
    clear_error();
    const char *who = "az_csr_import";
    if (!out || !indptr_host) return fail(AZ_EINVAL, "%s: NULL argument", who);
    *out = nullptr;
    AZ_TRY(check_build_args(ny, nx, npt_rad, npt_azim, unit, split));
    if (!(std::isfinite(lo) && std::isfinite(hi) && lo < hi))
        return fail(AZ_EINVAL, "%s: the radial range [%g, %g] must be finite with lo < hi", who, lo, hi);
    // the whole matrix is checked on the host before any device work
    const int nrows = npt_azim > 0 ? npt_rad * npt_azim : npt_rad;
    const int64_t npix = (int64_t)ny * nx;
    if (indptr_host[0] != 0) return fail(AZ_EINVAL, "%s: indptr[0] must be 0", who);
    for (int r = 0; r < nrows; ++r)
        if (indptr_host[r + 1] < indptr_host[r])
            return fail(AZ_EINVAL, "%s: indptr decreases at row %d", who, r);
    const int64_t nnz = indptr_host[nrows];
    if (nnz == 0) return fail(AZ_ERANGE, "%s: the matrix has no entries", who);
    if (!indices_host || !data_host) return fail(AZ_EINVAL, "%s: NULL indices or data", who);
    for (int r = 0; r < nrows; ++r)
        for (int32_t k = indptr_host[r]; k < indptr_host[r + 1]; ++k) {
            const int32_t p = indices_host[k];
            if (p < 0 || p >= npix)
                return fail(AZ_EINVAL, "%s: entry %d of row %d has pixel %d outside [0, %lld)", who, (int)k, r,
                            (int)p, (long long)npix);
            if (k > indptr_host[r] && p <= indices_host[k - 1])
                return fail(AZ_EINVAL, "%s: the pixels of row %d are not strictly ascending", who, r);
            if (!std::isfinite(data_host[k]))
                return fail(AZ_EINVAL, "%s: entry %d has a non-finite weight", who, (int)k);
        }
    cudaStream_t s = (cudaStream_t)stream;
    az_integrator *h = new (std::nothrow) az_integrator;
    if (!h) return fail(AZ_ENOMEM, "%s: out of host memory", who);
    cudaGetDevice(&h->device);
    h->ny = ny; h->nx = nx; h->npt_rad = npt_rad; h->npt_azim = npt_azim; h->nrows = nrows;
    h->unit = unit; h->split = split; h->nnz = nnz;
    h->lo = lo; h->hi = hi; h->delta = (hi - lo) / npt_rad;
    int rc = import_csr(h, indptr_host, indices_host, data_host, s);
    if (rc == AZ_OK) rc = finish_build(h, s);
    if (rc != AZ_OK) {
        cudaStreamSynchronize(s);
        delete h;
        return rc;
    }
    *out = h;
    return AZ_OK;
}

extern "C" int az_integrator_info(const az_integrator *h, az_info *out) {
    clear_error();
    if (!h || !out) return fail(AZ_EINVAL, "az_integrator_info: NULL argument");
    memset(out, 0, sizeof(*out));
    out->ny = h->ny; out->nx = h->nx; out->npt_rad = h->npt_rad; out->npt_azim = h->npt_azim;
    out->nrows = h->nrows; out->unit = h->unit; out->split = h->split;
    out->n_unmasked = h->n_unmasked; out->nnz = h->nnz;
    out->lo = h->lo; out->hi = h->hi; out->delta = h->delta;
    out->tile_h = h->tl.th; out->tile_w = h->tl.tw;
    out->rows_per_warp = h->rows_per_warp; out->frames_per_pass = h->frames_per_pass;
    out->n_tiles = h->tl.ntiles; out->n_segments = h->tl.nseg;
    out->copy_engine = h->copy_engine;
    out->n_items = h->tl.n_active;
    out->layout = h->layout;
    out->lut_width = h->lut_width;
    const DevBuf *bufs[] = {&h->csr_ptr, &h->csr_idx, &h->csr_w64, &h->csc_ptr, &h->csc_row,
                            &h->csc_w64, &h->csc_w32, &h->tl.tile_seg_ptr, &h->tl.tile_ent_ptr,
                            &h->tl.active_tiles, &h->tl.seg_ent_ptr, &h->tl.seg_slot,
                            &h->tl.row_slot_ptr, &h->tl.ent_loc, &h->tl.ent_loc_p, &h->tl.ent_w32, &h->tl.ent_w64,
                            &h->partial, &h->norm, &h->adj, &h->status, &h->host_stage,
                            &h->tl.tile_desc, &h->tl.tile_rec, &h->tl.ent_pix, &h->tl.ent_dark,
                            &h->tl.norm_frames, &h->tl.ent_wnorm, &h->lut32, &h->lut64,
                            &h->lut_vals, &h->lut_part, &h->one_planes, &h->bound_ent_dark,
                            &h->bound_norm};
    int64_t tot = 0;
    for (const DevBuf *b : bufs) tot += (int64_t)b->bytes;
    out->device_bytes = tot;
    return AZ_OK;
}

extern "C" int az_csr_export(const az_integrator *h, int32_t *indptr_host, int32_t *indices_host,
                             double *data_host) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_csr_export: NULL integrator");
    if (indptr_host)
        AZ_CUDA(cudaMemcpy(indptr_host, h->csr_ptr.p, sizeof(int32_t) * (h->nrows + 1), cudaMemcpyDeviceToHost));
    if (indices_host)
        AZ_CUDA(cudaMemcpy(indices_host, h->csr_idx.p, sizeof(int32_t) * h->nnz, cudaMemcpyDeviceToHost));
    if (data_host)
        AZ_CUDA(cudaMemcpy(data_host, h->csr_w64.p, sizeof(double) * h->nnz, cudaMemcpyDeviceToHost));
    return AZ_OK;
}

extern "C" int az_radial_axis(const az_integrator *h, double *out_host) {
    clear_error();
    if (!h || !out_host) return fail(AZ_EINVAL, "az_radial_axis: NULL argument");
    for (int k = 0; k < h->npt_rad; ++k) out_host[k] = h->lo + ((double)k + 0.5) * h->delta;
    return AZ_OK;
}

extern "C" int az_integrator_status(az_integrator *h) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_integrator_status: NULL integrator");
    AZ_CUDA(cudaStreamSynchronize(h->last_stream));
    int st = 0;
    AZ_CUDA(cudaMemcpy(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost));
    AZ_CUDA(cudaMemset(h->status.p, 0, sizeof(int)));
    if (st != AZ_OK) return fail(st, "a bounded device-side wait gave up");
    return AZ_OK;
}

extern "C" void az_integrator_destroy(az_integrator *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (cudaEvent_t e : h->copy_events)
        if (e) cudaEventDestroy(e);
    delete h;
}

static int integrate_common(const az_integrator *h, const void *image, int dtype, const float *dark,
                            const float *flat, const float *sa, const float *pol, int precision,
                            void *oI, void *oS, void *oN, void *oC, az_stream_t stream, bool two_d,
                            const char *who) {
    clear_error();
    AZ_TRY(check_forward(h, image, dtype, dark, flat, sa, pol, who));
    if (precision != AZ_PREC_FP64 && precision != AZ_PREC_FP32_COMP)
        return fail(AZ_EINVAL, "%s: bad precision %d", who, precision);
    if (two_d && h->npt_azim == 0) return fail(AZ_ESHAPE, "%s: integrator is 1D", who);
    if (!two_d && h->npt_azim != 0) return fail(AZ_ESHAPE, "%s: integrator is 2D", who);
    const_cast<az_integrator *>(h)->last_stream = (cudaStream_t)stream;
    if (h->layout == AZ_LAYOUT_LUT)
        return lut_forward(h, image, dtype, dark, flat, sa, pol, precision, oI, oS, oN, oC, (cudaStream_t)stream);
    if (precision == AZ_PREC_FP32_COMP) {
        // the batched machinery on a batch of one frame: the same arithmetic per frame as
        // the single-frame kernel (which remains the path without the tensor-copy engine)
        const int rc = forward_batch_one(const_cast<az_integrator *>(h), image, dtype, dark, flat, sa, pol,
                                         static_cast<float *>(oI), static_cast<float *>(oS),
                                         static_cast<float *>(oN), static_cast<float *>(oC),
                                         (cudaStream_t)stream);
        if (rc != AZ_EUNSUPPORTED) return rc;
    }
    return forward_single(h, image, dtype, dark, flat, sa, pol, precision, oI, oS, oN, oC,
                          (cudaStream_t)stream);
}

extern "C" int az_integrate1d(const az_integrator *h, const void *image_dev, int image_dtype,
                              const float *dark, const float *flat, const float *solid_angle,
                              const float *polarization, int precision, void *out_I,
                              void *out_sum_signal, void *out_sum_norm, void *out_count,
                              az_stream_t stream) {
    return integrate_common(h, image_dev, image_dtype, dark, flat, solid_angle, polarization,
                            precision, out_I, out_sum_signal, out_sum_norm, out_count, stream,
                            false, "az_integrate1d");
}

extern "C" int az_integrate2d(const az_integrator *h, const void *image_dev, int image_dtype,
                              const float *dark, const float *flat, const float *solid_angle,
                              const float *polarization, int precision, void *out_I,
                              void *out_sum_signal, void *out_sum_norm, void *out_count,
                              az_stream_t stream) {
    return integrate_common(h, image_dev, image_dtype, dark, flat, solid_angle, polarization,
                            precision, out_I, out_sum_signal, out_sum_norm, out_count, stream,
                            true, "az_integrate2d");
}

extern "C" int az_integrate_batch(az_integrator *h, const void *frames_dev, int n_frames,
                                  int image_dtype, const float *dark, const float *flat,
                                  const float *solid_angle, const float *polarization,
                                  float *out_I, float *out_sum_signal, float *out_sum_norm,
                                  float *out_count, az_stream_t stream) {
    clear_error();
    if (n_frames < 0) return fail(AZ_ESHAPE, "az_integrate_batch: n_frames < 0");
    // with no frames only N and C are formed: the frames pointer may be NULL
    static const uint32_t no_frames = 0;
    AZ_TRY(check_forward(h, n_frames == 0 ? &no_frames : frames_dev, image_dtype, dark, flat,
                         solid_angle, polarization, "az_integrate_batch"));
    h->last_stream = (cudaStream_t)stream;
    if (n_frames == 0 && !out_sum_norm && !out_count) return AZ_OK;
    return forward_batch(h, frames_dev, n_frames, image_dtype, dark, flat, solid_angle,
                         polarization, out_I, out_sum_signal, out_sum_norm, out_count,
                         (cudaStream_t)stream);
}

extern "C" int az_set_corrections(az_integrator *h, const float *dark, const float *flat,
                                  const float *solid_angle, const float *polarization,
                                  az_stream_t stream) {
    clear_error();
    static const uint32_t no_frames = 0;
    AZ_TRY(check_forward(h, &no_frames, AZ_DTYPE_F32, dark, flat, solid_angle, polarization,
                         "az_set_corrections"));
    h->last_stream = (cudaStream_t)stream;
    return bind_corrections(h, dark, flat, solid_angle, polarization, (cudaStream_t)stream);
}

extern "C" int az_integrate_batch_bound(az_integrator *h, const void *frames_dev, int n_frames,
                                        int image_dtype, float *out_I, float *out_sum_signal,
                                        float *out_sum_norm, float *out_count, az_stream_t stream) {
    clear_error();
    if (n_frames < 0) return fail(AZ_ESHAPE, "az_integrate_batch_bound: n_frames < 0");
    static const uint32_t no_frames = 0;
    AZ_TRY(check_forward(h, n_frames == 0 ? &no_frames : frames_dev, image_dtype, nullptr, nullptr,
                         nullptr, nullptr, "az_integrate_batch_bound"));
    h->last_stream = (cudaStream_t)stream;
    return forward_batch_bound(h, frames_dev, n_frames, image_dtype, out_I, out_sum_signal, out_sum_norm,
                               out_count, (cudaStream_t)stream);
}

extern "C" int az_integrate_batch_pixelnorm(az_integrator *h, const void *frames_dev, int n_frames,
                                            int image_dtype, const float *dark, const float *flat,
                                            const float *solid_angle, const float *polarization,
                                            float *out_I, float *out_sum_corrected, float *out_count,
                                            az_stream_t stream) {
    clear_error();
    if (n_frames < 0) return fail(AZ_ESHAPE, "az_integrate_batch_pixelnorm: n_frames < 0");
    static const uint32_t no_frames = 0;
    AZ_TRY(check_forward(h, n_frames == 0 ? &no_frames : frames_dev, image_dtype, dark, flat,
                         solid_angle, polarization, "az_integrate_batch_pixelnorm"));
    h->last_stream = (cudaStream_t)stream;
    return batch_pixelnorm(h, frames_dev, n_frames, image_dtype, dark, flat, solid_angle, polarization,
                           out_I, out_sum_corrected, out_count, (cudaStream_t)stream);
}

extern "C" int az_integrate_variance(az_integrator *h, const void *frames_dev, int n_frames,
                                     int image_dtype, float *out_sum_variance, az_stream_t stream) {
    clear_error();
    if (n_frames < 0) return fail(AZ_ESHAPE, "az_integrate_variance: n_frames < 0");
    if (n_frames == 0) return AZ_OK;
    AZ_TRY(check_forward(h, frames_dev, image_dtype, nullptr, nullptr, nullptr, nullptr,
                         "az_integrate_variance"));
    if (!out_sum_variance) return fail(AZ_EINVAL, "az_integrate_variance: NULL output");
    h->last_stream = (cudaStream_t)stream;
    return batch_variance(h, frames_dev, n_frames, image_dtype, out_sum_variance, (cudaStream_t)stream);
}

extern "C" int az_integrate_batch_host(az_integrator *h, const void *frames_host, int n_frames,
                                       int image_dtype, const float *dark, const float *flat,
                                       const float *solid_angle, const float *polarization,
                                       float *out_I_host, float *out_sum_signal_host,
                                       az_stream_t stream) {
    clear_error();
    AZ_TRY(check_forward(h, frames_host, image_dtype, dark, flat, solid_angle, polarization,
                         "az_integrate_batch_host"));
    if (n_frames < 0) return fail(AZ_ESHAPE, "az_integrate_batch_host: n_frames < 0");
    if (n_frames == 0) return AZ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fbytes = (size_t)h->ny * h->nx * 4u;
    const size_t obytes = (size_t)h->nrows * sizeof(float);
    const int chunk = std::max(1, std::min(16, n_frames));
    // two device buffers of `chunk` frames and their outputs
    const size_t per = chunk * (fbytes + 2 * obytes);
    if (h->host_stage.bytes < 2 * per) AZ_TRY(h->host_stage.alloc(2 * per));
    char *base = h->host_stage.as<char>();
    char *fr[2] = {base, base + per};
    float *oi[2], *os[2];
    for (int b = 0; b < 2; ++b) {
        oi[b] = reinterpret_cast<float *>(fr[b] + chunk * fbytes);
        os[b] = oi[b] + (size_t)chunk * h->nrows;
    }
    int rc = AZ_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == AZ_OK) rc = fail(AZ_ECUDA, "az_integrate_batch_host: %s", cudaGetErrorString(e));
    };
    // the upload stream and its events live with the integrator (created once)
    if (!h->copy_stream) ck(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t &e : h->copy_events)
        if (!e) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (rc != AZ_OK) return rc;
    cudaStream_t cp = h->copy_stream;
    cudaEvent_t start = h->copy_events[0];
    cudaEvent_t up[2] = {h->copy_events[1], h->copy_events[2]};
    cudaEvent_t done[2] = {h->copy_events[3], h->copy_events[4]};
    if (rc == AZ_OK) {
        ck(cudaEventRecord(start, s));
        ck(cudaStreamWaitEvent(cp, start, 0));
        rc = batch_norm(h, flat, solid_angle, polarization, nullptr, nullptr, s);
    }
    const int nchunks = (n_frames + chunk - 1) / chunk;
    // upload chunk 0 (and 1) ahead, then: compute k on `s` while `cp` uploads k+1
    auto upload = [&](int k) {
        const int b = k & 1, f0 = k * chunk, nf = std::min(chunk, n_frames - f0);
        ck(cudaMemcpyAsync(fr[b], static_cast<const char *>(frames_host) + (size_t)f0 * fbytes,
                           (size_t)nf * fbytes, cudaMemcpyHostToDevice, cp));
        ck(cudaEventRecord(up[b], cp));
    };
    if (rc == AZ_OK) upload(0);
    for (int k = 0; k < nchunks && rc == AZ_OK; ++k) {
        const int b = k & 1, f0 = k * chunk, nf = std::min(chunk, n_frames - f0);
        if (k + 1 < nchunks) {
            if (k >= 1) ck(cudaStreamWaitEvent(cp, done[(k + 1) & 1], 0));  // buffer free again
            upload(k + 1);
        }
        ck(cudaStreamWaitEvent(s, up[b], 0));
        if (rc == AZ_OK) rc = batch_frames(h, fr[b], nf, image_dtype, dark, oi[b], os[b], 0, s);
        if (out_I_host)
            ck(cudaMemcpyAsync(out_I_host + (size_t)f0 * h->nrows, oi[b], (size_t)nf * obytes,
                               cudaMemcpyDeviceToHost, s));
        if (out_sum_signal_host)
            ck(cudaMemcpyAsync(out_sum_signal_host + (size_t)f0 * h->nrows, os[b], (size_t)nf * obytes,
                               cudaMemcpyDeviceToHost, s));
        ck(cudaEventRecord(done[b], s));
    }
    ck(cudaStreamSynchronize(s));
    ck(cudaStreamSynchronize(cp));
    h->last_stream = s;
    return rc;
}

extern "C" int az_integrate_backward(const az_integrator *h, const void *grad_I, const void *I,
                                     const void *sum_norm, const float *solid_angle,
                                     const float *polarization, int precision,
                                     void *out_grad_image, void *out_grad_flat,
                                     az_stream_t stream) {
    clear_error();
    if (!h || !grad_I || !I || !sum_norm) return fail(AZ_EINVAL, "az_integrate_backward: NULL argument");
    if (precision != AZ_PREC_FP64 && precision != AZ_PREC_FP32_COMP)
        return fail(AZ_EINVAL, "az_integrate_backward: bad precision %d", precision);
    if (!out_grad_image && !out_grad_flat) return AZ_OK;
    const_cast<az_integrator *>(h)->last_stream = (cudaStream_t)stream;
    return backward(h, grad_I, I, sum_norm, solid_angle, polarization, precision, out_grad_image,
                    out_grad_flat, (cudaStream_t)stream);
}

extern "C" int az_multi_create(az_integrator *const *handles, int n, const void *const *images,
                               int image_dtype, const float *const *darks,
                               const float *const *flats, const float *const *solid_angles,
                               const float *const *polarizations, float *const *out_I,
                               float *const *out_sum_signal, float *const *out_sum_norm,
                               float *const *out_count, az_multi **out) {
    clear_error();
    if (!handles || !images || !out || n < 1) return fail(AZ_EINVAL, "az_multi_create: bad arguments");
    *out = nullptr;
    if (image_dtype < AZ_DTYPE_F32 || image_dtype > AZ_DTYPE_I32)
        return fail(AZ_EINVAL, "az_multi_create: bad image dtype %d", image_dtype);
    for (int k = 0; k < n; ++k) {
        if (!handles[k] || !images[k]) return fail(AZ_EINVAL, "az_multi_create: NULL handle or image %d", k);
        AZ_TRY(check_forward(handles[k], images[k], image_dtype, darks ? darks[k] : nullptr,
                             flats ? flats[k] : nullptr, solid_angles ? solid_angles[k] : nullptr,
                             polarizations ? polarizations[k] : nullptr, "az_multi_create"));
    }
    az_multi *m = new (std::nothrow) az_multi;
    if (!m) return fail(AZ_ENOMEM, "az_multi_create: out of host memory");
    int rc = multi_create(handles, n, images, image_dtype, darks, flats, solid_angles, polarizations,
                          out_I, out_sum_signal, out_sum_norm, out_count, &m->plan);
    if (rc != AZ_OK) {
        delete m;
        return rc;
    }
    *out = m;
    return AZ_OK;
}

extern "C" int az_multi_launch(az_multi *plan, int use_graph, az_stream_t stream) {
    clear_error();
    if (!plan || !plan->plan) return fail(AZ_EINVAL, "az_multi_launch: NULL plan");
    return multi_launch(plan->plan, use_graph, (cudaStream_t)stream);
}

extern "C" void az_multi_destroy(az_multi *plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    multi_destroy(plan->plan);
    delete plan;
}

extern "C" int az_profile_enable(az_integrator *h, int enable) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_profile_enable: NULL integrator");
    h->prof.on = enable != 0;
    return AZ_OK;
}

extern "C" int az_profile_read(az_integrator *h, az_profile *out) {
    clear_error();
    if (!h || !out) return fail(AZ_EINVAL, "az_profile_read: NULL argument");
    memset(out, 0, sizeof(*out));
    int rc = AZ_OK;
    for (auto &r : h->prof.recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess && rc == AZ_OK) rc = fail(AZ_ECUDA, "az_profile_read: %s", cudaGetErrorString(e));
        if (r.kind >= 0 && r.kind < AZ_PROF_KINDS) {
            out->launches[r.kind] += 1;
            out->total_ms[r.kind] += ms;
        }
        h->prof.pool.push_back(r.a);
        h->prof.pool.push_back(r.b);
    }
    h->prof.recs.clear();
    return rc;
}

extern "C" int az_set_copy_engine(az_integrator *h, int engine) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_set_copy_engine: NULL integrator");
    if (engine != AZ_COPY_TMA && engine != AZ_COPY_ASYNC)
        return fail(AZ_EINVAL, "az_set_copy_engine: bad engine %d", engine);
    h->copy_engine = engine;
    return AZ_OK;
}

extern "C" int az_set_tuning(az_integrator *h, int tile_h, int tile_w, int rows_per_warp,
                             int frames_per_pass) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_set_tuning: NULL integrator");
    if (tile_h < 0 || tile_w < 0 || (tile_w % 4) != 0)
        return fail(AZ_EINVAL, "az_set_tuning: tile_w must be a multiple of 4");
    auto pow2_upto32 = [](int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32; };
    if (rows_per_warp && !pow2_upto32(rows_per_warp))
        return fail(AZ_EINVAL, "az_set_tuning: rows_per_warp must be 1, 2, 4, 8, 16 or 32");
    if (frames_per_pass && !pow2_upto32(frames_per_pass))
        return fail(AZ_EINVAL, "az_set_tuning: frames_per_pass must be 1, 2, 4, 8, 16 or 32");
    if (rows_per_warp && frames_per_pass && rows_per_warp * frames_per_pass != 32)
        return fail(AZ_EINVAL, "az_set_tuning: rows_per_warp * frames_per_pass must be 32");
    const int th = tile_h ? tile_h : h->tl.th, tw = tile_w ? tile_w : h->tl.tw;
    if (th != h->tl.th || tw != h->tl.tw) {
        if ((int64_t)th * (tw + 8) > 65535 || th < 1 || tw < 4)
            return fail(AZ_EINVAL, "az_set_tuning: tile %dx%d out of range", th, tw);
        cudaDeviceSynchronize();
        AZ_TRY(build_tiled_layout(h, th, tw, nullptr));
        AZ_TRY(alloc_scratch(h));
        AZ_CUDA(cudaDeviceSynchronize());
    }
    if (rows_per_warp) h->frames_per_pass = 32 / rows_per_warp;
    if (frames_per_pass) h->frames_per_pass = frames_per_pass;
    h->rows_per_warp = 32 / h->frames_per_pass;
    return AZ_OK;
}

// One FP32 frame through the tiled form and through the look-up table; the faster becomes
// the single-frame layout.  The table is built for the trial if missing and small enough
// (at most four times the bytes of the matrix's entries), and freed again if it loses.
static int tune_layout(az_integrator *h, const void *frame, const float *dark, cudaStream_t s) {
    const bool had_table = h->lut32.p != nullptr;
    if (!had_table) {
        int64_t wmax = 0;
        {
            std::vector<int32_t> ptr((size_t)h->nrows + 1);
            AZ_CUDA(cudaMemcpy(ptr.data(), h->csr_ptr.p, sizeof(int32_t) * ptr.size(), cudaMemcpyDeviceToHost));
            for (int b = 0; b < h->nrows; ++b) wmax = std::max<int64_t>(wmax, ptr[b + 1] - ptr[b]);
        }
        if (wmax * h->nrows > 4 * std::max<int64_t>(h->nnz, 1)) return AZ_OK;  // the tiled form stays
        if (lut_build(h, AZ_PREC_FP32_COMP, s) != AZ_OK) {
            clear_error();
            return AZ_OK;
        }
    }
    DevBuf out;
    AZ_TRY(out.alloc(sizeof(float) * 4 * (size_t)h->nrows));
    float *o = out.as<float>();
    const int rows = h->nrows;
    cudaEvent_t e0, e1;
    AZ_CUDA(cudaEventCreate(&e0));
    AZ_CUDA(cudaEventCreate(&e1));
    double t[2] = {1e30, 1e30};
    for (int lay = 0; lay < 2; ++lay) {
        h->layout = lay;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            int rc;
            if (lay == AZ_LAYOUT_LUT) {
                rc = lut_forward(h, frame, AZ_DTYPE_U32, dark, nullptr, nullptr, nullptr, AZ_PREC_FP32_COMP, o,
                                 o + rows, o + 2 * rows, o + 3 * rows, s);
            } else {
                // what az_integrate1d/2d run in FP32 with the tiled form
                rc = forward_batch_one(h, frame, AZ_DTYPE_U32, dark, nullptr, nullptr, nullptr, o, o + rows,
                                       o + 2 * rows, o + 3 * rows, s);
                if (rc == AZ_EUNSUPPORTED)
                    rc = forward_single(h, frame, AZ_DTYPE_U32, dark, nullptr, nullptr, nullptr, AZ_PREC_FP32_COMP,
                                        o, o + rows, o + 2 * rows, o + 3 * rows, s);
            }
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rc != AZ_OK) {
                clear_error();
                break;
            }
            if (rep > 0) t[lay] = std::min<double>(t[lay], ms);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->layout = t[AZ_LAYOUT_LUT] < t[AZ_LAYOUT_TILED] ? AZ_LAYOUT_LUT : AZ_LAYOUT_TILED;
    if (h->layout == AZ_LAYOUT_TILED && !had_table) {
        h->lut32.release();
        if (!h->lut64.p) {
            h->lut_vals.release();
            h->lut_part.release();
            h->lut_width = 0;
        }
    }
    return AZ_OK;
}

extern "C" int az_autotune(az_integrator *h, int n_trial_frames, az_stream_t stream,
                           double *best_ms) {
    clear_error();
    if (!h) return fail(AZ_EINVAL, "az_autotune: NULL integrator");
    if (n_trial_frames < 1) return fail(AZ_EINVAL, "az_autotune: n_trial_frames must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npix = (int64_t)h->ny * h->nx;
    DevBuf frames, outI, outS, dark;
    AZ_TRY(frames.alloc(sizeof(uint32_t) * npix * n_trial_frames));
    AZ_TRY(outI.alloc(sizeof(float) * (size_t)h->nrows * n_trial_frames));
    AZ_TRY(outS.alloc(sizeof(float) * (size_t)h->nrows * n_trial_frames));
    AZ_TRY(dark.alloc(sizeof(float) * npix));
    AZ_CUDA(cudaMemsetAsync(dark.p, 0, sizeof(float) * npix, s));
    fill_frames_kernel<<<num_sms() * 8, 256, 0, s>>>(frames.as<uint32_t>(), npix * n_trial_frames, 12345u);
    AZ_CUDA(cudaGetLastError());
    AZ_TRY(batch_norm(h, nullptr, nullptr, nullptr, nullptr, nullptr, s));
    cudaEvent_t e0, e1;
    AZ_CUDA(cudaEventCreate(&e0));
    AZ_CUDA(cudaEventCreate(&e1));
    const int tiles[][2] = {{8, 224}, {8, 192}, {16, 64}, {16, 96}, {8, 128}, {16, 128}, {32, 64}, {8, 64}};
    const int fpps[] = {4, 8, 16};
    const int engines[] = {AZ_COPY_TMA, AZ_COPY_ASYNC};
    double best = 1e30;
    int bt = -1, bf = h->frames_per_pass, be = h->copy_engine;
    const int tile_count = (int)(sizeof(tiles) / sizeof(tiles[0]));
    for (int ti = 0; ti < tile_count; ++ti) {
        if (build_tiled_layout(h, tiles[ti][0], tiles[ti][1], s) != AZ_OK) { clear_error(); continue; }
        AZ_TRY(alloc_scratch(h));
        AZ_TRY(batch_norm(h, nullptr, nullptr, nullptr, nullptr, nullptr, s));
        for (int eg : engines)
            for (int f : fpps) {
                h->frames_per_pass = f;
                h->copy_engine = eg;
                float best_t = 1e30f;
                bool ok = true;
                for (int rep = 0; rep < 3 && ok; ++rep) {
                    cudaEventRecord(e0, s);
                    ok = batch_frames(h, frames.p, n_trial_frames, AZ_DTYPE_U32, dark.as<float>(),
                                      outI.as<float>(), outS.as<float>(), 0, s) == AZ_OK;
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) best_t = std::min(best_t, ms);
                }
                clear_error();
                if (ok && best_t < best) {
                    best = best_t;
                    bt = ti; bf = f; be = eg;
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best >= 1e30) return fail(AZ_EUNSUPPORTED, "az_autotune: no configuration ran");
    if (bt < 0) return fail(AZ_EUNSUPPORTED, "az_autotune: no configuration ran");
    AZ_TRY(build_tiled_layout(h, tiles[bt][0], tiles[bt][1], s));
    AZ_TRY(alloc_scratch(h));
    h->frames_per_pass = bf;
    h->rows_per_warp = 32 / bf;
    h->copy_engine = be;
    AZ_TRY(tune_layout(h, frames.p, dark.as<float>(), s));
    AZ_CUDA(cudaStreamSynchronize(s));
    if (best_ms) *best_ms = best / n_trial_frames;
    return AZ_OK;
}
