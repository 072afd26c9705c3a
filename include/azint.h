/*
 * azint.h -- C ABI of the GB300 (sm_103a) azimuthal-integration library.
 *
 * The library reduces a corrected 2D X-ray detector image to a 1D (2theta, q or r) pattern
 * or a 2D (radial x chi) "cake", with no, bounding-box or full pixel splitting, by applying
 * a precomputed sparse bins x pixels matrix to every frame.  This is the method of
 * Kieffer & Ashiotis, "PyFAI: a Python library for high performance azimuthal integration
 * on GPU" (EuroSciPy 2014): coordinates in Sec. 3, pixel splitting in Sec. 4, the
 * scatter-to-gather transformation and the CSR matrix in Sec. 5.2, compensated single
 * precision in Sec. 5.2.2, the per-frame pipeline (cast, correction, integrate) in Sec. 6.4.
 *
 * General conventions
 *   - Images are C-contiguous, row-major [ny][nx] (ny rows along dim1, nx columns along
 *     dim2); pixel index p = i * nx + j.  Frame batches are [n_frames][ny][nx].
 *   - Every array argument marked "device" is a device pointer owned by the CALLER; the
 *     library never frees it.  "host" pointers are ordinary host memory.  Device arrays of
 *     4-byte elements must be 4-byte aligned (any cudaMalloc'd pointer is).
 *   - Handles (az_geometry, az_integrator, az_multi) are owned by the LIBRARY and freed by
 *     the matching *_destroy call.  A handle is not thread-safe: do not use one handle
 *     from two host threads at once.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Integration calls are
 *     asynchronous on that stream and do not synchronise.  Build calls (az_csr_build*)
 *     synchronise `stream` because they size their allocations from device results.
 *   - Every call returns AZ_OK (0) or a negative AZ_E* code and sets a thread-local message
 *     readable with az_last_error().  Arguments are validated before any launch; nothing
 *     aborts the process.  Device-side waits are bounded; a kernel that gives up records
 *     it in the integrator's status word (az_integrator_status).
 *   - Units: distances and pixel sizes in metres, angles in radians, wavelength in metres.
 */
#ifndef AZINT_H
#define AZINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *az_stream_t; /* same type as cudaStream_t */

/* ---- status codes ------------------------------------------------------------------- */
#define AZ_OK 0
#define AZ_EINVAL (-1)       /* bad argument (null handle, bad enum, misaligned pointer) */
#define AZ_ESHAPE (-2)       /* bad or inconsistent sizes */
#define AZ_ENOMEM (-3)       /* device or host allocation failed */
#define AZ_EOVERFLOW (-4)    /* more than 2^31 - 1 matrix entries */
#define AZ_ECUDA (-5)        /* a CUDA runtime call failed */
#define AZ_EUNSUPPORTED (-6) /* valid request this build does not implement */
#define AZ_ETIMEOUT (-7)     /* a bounded device-side wait gave up */
#define AZ_ERANGE (-8)       /* empty radial range: no unmasked pixel, or all positions equal */

/* ---- enumerations (the paper's `unit=` and `method=` keywords, Sec. 3) ------------------ */
enum az_unit { AZ_UNIT_2TH_DEG = 0, AZ_UNIT_Q_NM = 1, AZ_UNIT_R_MM = 2 };
enum az_split { AZ_SPLIT_NONE = 0, AZ_SPLIT_BBOX = 1, AZ_SPLIT_FULL = 2 };
enum az_precision { AZ_PREC_FP64 = 0, AZ_PREC_FP32_COMP = 1 };
enum az_dtype { AZ_DTYPE_F32 = 0, AZ_DTYPE_U32 = 1, AZ_DTYPE_I32 = 2 };
enum az_where { AZ_WHERE_CORNERS = 0, AZ_WHERE_CENTRES = 1 };
enum az_copy_engine { AZ_COPY_TMA = 0, AZ_COPY_ASYNC = 1 };

typedef struct az_geometry az_geometry;
typedef struct az_integrator az_integrator;
typedef struct az_multi az_multi;

/* Summary of a built integrator. */
typedef struct {
    int32_t ny, nx;            /* detector shape */
    int32_t npt_rad, npt_azim; /* bins; npt_azim == 0 for 1D */
    int32_t nrows;             /* npt_rad (1D) or npt_azim * npt_rad (2D) */
    int32_t unit, split;
    int32_t n_unmasked;        /* pixels that contribute */
    int64_t nnz;               /* matrix entries */
    double lo, hi, delta;      /* radial range and bin width, in the unit */
    int32_t tile_h, tile_w;    /* pixel tile staged in shared memory by the forward */
    int32_t rows_per_warp;     /* matrix rows a warp reduces at once in the batched forward
                                  (one lane per row and frame: 32 / frames_per_pass) */
    int32_t frames_per_pass;   /* frames sharing one pass over the matrix (batched forward) */
    int64_t n_tiles, n_segments;
    int64_t device_bytes;      /* device memory owned by the integrator */
    int32_t copy_engine;       /* AZ_COPY_TMA or AZ_COPY_ASYNC */
    int32_t n_items;           /* work items of the forward: tiles, heavy ones cut in several */
    int32_t layout;            /* AZ_LAYOUT_TILED or AZ_LAYOUT_LUT: what az_integrate1d/2d use */
    int64_t lut_width;         /* slots per row of the look-up table (0 until it is built) */
} az_info;

/* ---- geometry (Sec. 3) ---------------------------------------------------------------- */

/*
 * PONI-style geometry: the sample sits at `dist` from the detector plane, whose foot
 * point (PONI) is at (poni1, poni2) in detector coordinates.  A detector point (d1, d2)
 * maps to the laboratory vector t = Rz(rot3) Ry(rot2) Rx(rot1) (d1 - poni1, d2 - poni2,
 * dist); 2theta = atan2(sqrt(t1^2 + t2^2), t3), chi = atan2(t1, t2) (Sec. 3 coordinate
 * list: r, chi, 2theta = atan(r/d), q = 4 pi sin(2theta/2)/lambda).  Pixel (i, j) spans
 * d1 in [i, i+1] * pixel1, d2 in [j, j+1] * pixel2.  dist, pixel1, pixel2 and wavelength
 * must be > 0 and finite.  *out receives a host-side handle (no device memory).
 */
int az_geometry_create(double dist, double poni1, double poni2, double rot1, double rot2,
                       double rot3, double pixel1, double pixel2, double wavelength,
                       az_geometry **out);
void az_geometry_destroy(az_geometry *geom);

/* The laboratory rotation Rz(rot3) Ry(rot2) Rx(rot1) of the geometry, row-major, into host
 * double[9].  Host-only (no device work). */
int az_geometry_rotation(const az_geometry *geom, double *R_host);

/*
 * FP64 positions (Sec. 3): radial value in `unit` (2theta in degrees, q in nm^-1, r =
 * dist tan 2theta in mm) and chi in degrees in [-180, 180], at pixel corners
 * ((ny+1) x (nx+1) values, where == AZ_WHERE_CORNERS) or centres (ny x nx values).
 * rad_dev, chi_dev: device double arrays of that size; chi_dev may be NULL.
 */
int az_geometry_positions(const az_geometry *geom, int ny, int nx, int unit, int where,
                          double *rad_dev, double *chi_dev, az_stream_t stream);

/* Solid-angle correction at pixel centres, (dist / |t|)^3 (named in Sec. 6.4, textbook
 * formula); out_dev: device float [ny][nx]. */
int az_geometry_solid_angle(const az_geometry *geom, int ny, int nx, float *out_dev,
                            az_stream_t stream);

/* Polarisation correction at pixel centres, (1 + cos^2 2theta - factor cos 2chi
 * sin^2 2theta) / 2 (named in Sec. 6.4, textbook formula); out_dev: device float [ny][nx]. */
int az_geometry_polarization(const az_geometry *geom, int ny, int nx, double factor,
                             float *out_dev, az_stream_t stream);

/* ---- sparse matrix build (Sec. 4 splitting, Sec. 5.2 scatter-to-gather, CSR) --------- */

/*
 * Build the bins x pixels weight matrix for one detector on the device: FP64 positions,
 * radial range [lo, hi] = min/max over unmasked pixels of the positions the split reads
 * (centres for NONE, corners otherwise), delta = (hi - lo) / npt_rad; chi bins cover
 * [-180, 180) in npt_azim bins (npt_azim == 0: 1D).  Weights: NONE = whole pixel in the
 * bin of its centre; BBOX = bounding box of the corners (Sec. 4.1); FULL = area of the
 * straight-edged corner quadrilateral in the (radial, chi) plane inside each bin, divided
 * by the sum of those areas (Sec. 4.2).  The matrix is assembled as count -> exclusive scan
 * -> fill -> stable sort by row (rows ascending by pixel) and kept in three layouts:
 * scipy-compatible CSR, pixel-major CSC (for the adjoint) and a pixel-tiled layout used by
 * the forward kernels.  mask_dev: device uint8 [ny][nx], nonzero = masked, may be NULL.
 * Synchronises `stream`.  Errors: AZ_ESHAPE (ny, nx < 1), AZ_EINVAL (enums, npt_rad < 1,
 * npt_azim < 0), AZ_ERANGE (empty range), AZ_EOVERFLOW (nnz > 2^31 - 1), AZ_ENOMEM.
 */
int az_csr_build(const az_geometry *geom, int ny, int nx, int npt_rad, int npt_azim,
                 int unit, int split, const uint8_t *mask_dev, az_stream_t stream,
                 az_integrator **out);

/*
 * Same as az_csr_build from caller-supplied FP64 positions (device arrays): centre arrays
 * [ny][nx] for split NONE, corner arrays [ny+1][nx+1] otherwise.  chi_dev (degrees) is
 * required for 2D and for 1D FULL, ignored otherwise (may be NULL).  Lets a caller bring
 * its own geometry, and lets two implementations be compared on identical positions.
 */
int az_csr_build_from_positions(int ny, int nx, const double *rad_dev, const double *chi_dev,
                                int npt_rad, int npt_azim, int split, const uint8_t *mask_dev,
                                az_stream_t stream, az_integrator **out);

int az_integrator_info(const az_integrator *h, az_info *out);

/* Copy the CSR matrix to host memory: indptr int32[nrows + 1], indices int32[nnz] (pixel
 * ids, ascending within a row), data double[nnz] (any of the three may be NULL).  Loads
 * directly into scipy.sparse.csr_matrix (Sec. 5.2.1).  Synchronous. */
int az_csr_export(const az_integrator *h, int32_t *indptr_host, int32_t *indices_host,
                  double *data_host);

/*
 * A new integrator from a bins x pixels matrix in host memory, in the scipy-compatible CSR form
 * that az_csr_export writes (Sec. 5.2.1): indptr int32[nrows + 1] (indptr[0] = 0, non-
 * decreasing), indices int32[nnz] (pixel ids p = i * nx + j < ny * nx, strictly ascending
 * within a row), data double[nnz] (finite weights), nrows = npt_rad (npt_azim == 0) or
 * npt_azim * npt_rad (row = chi_bin * npt_rad + rad_bin).  lo < hi is the radial range the
 * bins cover (az_radial_axis gives lo + (k + 1/2) (hi - lo) / npt_rad); unit and split are
 * kept as labels only (az_integrator_info).  Lets a matrix built elsewhere -- another
 * program's, a stored one, or a reference implementation's -- be applied by this library's
 * kernels.  The matrix is checked on the host, then copied to the device and laid out as
 * az_csr_build's (pixel-major CSC for the adjoint, tiled layout for the forward), so
 * az_csr_export of the result returns the three arrays bit for bit.  Synchronises `stream`.
 * Errors, before any device work: AZ_EINVAL (NULL arrays, indptr or indices out of order or
 * range, non-finite weight, lo >= hi, bad enums), AZ_ESHAPE (ny, nx < 1), AZ_ERANGE (no
 * entries); afterwards AZ_ENOMEM or AZ_ECUDA.
 */
int az_csr_import(int ny, int nx, int npt_rad, int npt_azim, int unit, int split,
                  const int32_t *indptr_host, const int32_t *indices_host, const double *data_host,
                  double lo, double hi, az_stream_t stream, az_integrator **out);

/* Radial bin centres lo + (k + 1/2) delta, k < npt_rad, into host double[npt_rad]. */
int az_radial_axis(const az_integrator *h, double *out_host);

/* Reads and clears the integrator's device status word (synchronises the last stream
 * used): AZ_OK, or AZ_ETIMEOUT if a bounded device-side wait gave up. */
int az_integrator_status(az_integrator *h);

void az_integrator_destroy(az_integrator *h);

/* ---- forward (Sec. 5.2 sparse matrix-vector product, Sec. 6.4 corrections) ----------- */

/*
 * One frame.  For every bin b:
 *   S_b = sum_p A_bp (img_p - dark_p)            (out_sum_signal)
 *   N_b = sum_p A_bp flat_p solid_angle_p pol_p  (out_sum_norm)
 *   C_b = sum_p A_bp                             (out_count)
 *   I_b = S_b / N_b, 0 where N_b == 0            (out_I)
 * with no output zeroing (Sec. 6.4's "memset").  FP64: one fused pass, the cast of the image
 * (Sec. 6.4 "cast"), the corrections ("correction") and the reduction ("integrate") in one
 * kernel.  FP32: a pixel pass forms cast(img) - dark and flat * solid_angle * polarization,
 * which the batched kernel then reduces (the bits of that frame in any batch); C is kept per
 * layout.  With az_set_layout(AZ_LAYOUT_LUT) both go through the look-up table instead.
 * image_dev: device [ny][nx] of image_dtype.  dark/flat/solid_angle/polarization: device
 * float [ny][nx], each may be NULL (dark = 0, the others = 1).  precision AZ_PREC_FP64:
 * FP64 weights and accumulation, outputs are device double[nrows]; AZ_PREC_FP32_COMP:
 * FP32 weights, Kahan-compensated FP32 sums (Sec. 5.2.2), outputs device float[nrows].
 * Any output pointer may be NULL.  Deterministic: the same inputs give the same bits.
 */
int az_integrate1d(const az_integrator *h, const void *image_dev, int image_dtype,
                   const float *dark, const float *flat, const float *solid_angle,
                   const float *polarization, int precision, void *out_I,
                   void *out_sum_signal, void *out_sum_norm, void *out_count,
                   az_stream_t stream);

/* 2D (cake) form of az_integrate1d for an integrator built with npt_azim > 0; outputs are
 * [npt_azim][npt_rad] row-major (row = chi_bin * npt_rad + rad_bin). */
int az_integrate2d(const az_integrator *h, const void *image_dev, int image_dtype,
                   const float *dark, const float *flat, const float *solid_angle,
                   const float *polarization, int precision, void *out_I,
                   void *out_sum_signal, void *out_sum_norm, void *out_count,
                   az_stream_t stream);

/*
 * az_integrate1d / az_integrate2d (by the integrator's kind) without any device allocation
 * by the call.  The paper has no counterpart: this entry point exists for callers that may
 * not call cudaMalloc while they run -- for instance a plugin inside a host program whose own
 * memory pool has reserved the device memory, or an acquisition loop that forbids
 * allocations (which can block and synchronise the device) once set-up is over.  The
 * integrator itself must have been built beforehand.
 *
 * It always runs the tiled single-pass form (the one-launch reduction of FP64 frames, for
 * both precisions), whatever az_set_layout chose, so its FP32 bits may differ from
 * az_integrate1d's by rounding order (both within the stated tolerances).
 *
 * The partial sums the forward keeps between its two kernels go to one fixed array of
 * AZ_NOALLOC_SCRATCH_BYTES compiled into this library; every GPU on which an integrator is
 * built holds that memory from then until the process exits.  A call needs 3 * segments * 8 bytes (FP64) or
 * 3 * segments * 4 bytes (FP32 compensated), segments = az_info.n_segments; a larger need is
 * refused with AZ_ESHAPE and a message giving both sizes.  Nothing in the array has to start
 * at zero: each call writes every partial sum it later reads.
 *
 * All calls on a device share the array and it keeps the last call's contents, so calls
 * that overlap on the GPU (different streams, or host threads without ordering) race and
 * give wrong results: order them on one stream.  Building an integrator on a device (the
 * set-up) looks up the array's device address (cudaGetSymbolAddress, with that device
 * current) and loads the kernels this call runs; under the CUDA runtime's lazy module
 * loading (the default) that is when the array's memory is reserved on that device, so the
 * calls themselves take none.  A call made with a device current on which no integrator was
 * built does that look-up itself: make such a first call before any stream capture.  If a
 * bounded device-side wait gives up during a call (az_integrator_status then reports
 * AZ_ETIMEOUT), that call's outputs are not valid: they may hold sums left in the array by
 * an earlier call.  Arguments, outputs and errors are otherwise those of az_integrate1d.
 */
#define AZ_NOALLOC_SCRATCH_BYTES (8u << 20)
int az_integrate_noalloc(const az_integrator *h, const void *image_dev, int image_dtype,
                         const float *dark, const float *flat, const float *solid_angle,
                         const float *polarization, int precision, void *out_I,
                         void *out_sum_signal, void *out_sum_norm, void *out_count,
                         az_stream_t stream);

/*
 * Many frames through one matrix ("several detectors / frames", Sec. 5.2.2 end): frames
 * device [n_frames][ny][nx]; the frame-independent sums N and C are formed once per call
 * and each matrix entry is applied to frames_per_pass frames per read.  FP32 compensated.
 * out_I, out_sum_signal: device float [n_frames][nrows] (either may be NULL);
 * out_sum_norm, out_count: device float [nrows] (may be NULL).  With n_frames == 0 only N and
 * C are formed and frames_dev may be NULL.
 */
int az_integrate_batch(az_integrator *h, const void *frames_dev, int n_frames,
                       int image_dtype, const float *dark, const float *flat,
                       const float *solid_angle, const float *polarization, float *out_I,
                       float *out_sum_signal, float *out_sum_norm, float *out_count,
                       az_stream_t stream);

/*
 * Bind the correction arrays of a detector to the integrator once (Sec. 6.4 names dark, flat,
 * solid-angle and polarisation corrections; they do not change from frame to frame): the
 * frame-independent part of az_integrate_batch -- the dark of every matrix entry's pixel, and
 * per bin N = sum w flat solid_angle pol and C = sum w -- is formed now, on `stream`, into
 * buffers the integrator owns.  The arrays (device float [ny][nx], any may be NULL: dark = 0,
 * the others = 1) are not read again: later changes to them take effect only when they are
 * bound again.  A new binding replaces the old one; a change of the tiled layout
 * (az_set_tuning, az_autotune) drops it.  Errors: those of az_integrate_batch's arguments.
 */
int az_set_corrections(az_integrator *h, const float *dark, const float *flat,
                       const float *solid_angle, const float *polarization, az_stream_t stream);

/*
 * az_integrate_batch with the corrections bound by az_set_corrections: frames device
 * [n_frames][ny][nx]; out_I, out_sum_signal device float [n_frames][nrows]; out_sum_norm,
 * out_count device float [nrows] receive the bound N and C (each may be NULL).  The bits equal
 * az_integrate_batch's with the same corrections.  AZ_EINVAL when nothing is bound or the
 * layout changed since the binding.
 */
int az_integrate_batch_bound(az_integrator *h, const void *frames_dev, int n_frames,
                             int image_dtype, float *out_I, float *out_sum_signal,
                             float *out_sum_norm, float *out_count, az_stream_t stream);

/*
 * The paper's own normalisation (Sec. 6.4: a correction pass, then the integration, whose
 * result is a ratio of two histograms): each pixel is corrected first,
 * c = (img - dark) / (flat * solid_angle * polarization), then U = sum w c, C = sum w and
 * I = U / C (0 where C = 0).  frames device [n_frames][ny][nx]; corrections as in
 * az_integrate_batch (NULL = absent); out_I, out_sum_corrected device float
 * [n_frames][nrows], out_count device float [nrows] (any may be NULL).  FP32 compensated;
 * computed with the weights divided by each pixel's flat * solid_angle * polarization once
 * per call.  Through the batched kernel (tensor-copy engine; AZ_EUNSUPPORTED for tiles
 * wider than 236 pixels or with AZ_COPY_ASYNC).  With no flat, solid angle or polarisation
 * the result equals az_integrate_batch's I and S bit for bit.
 */
int az_integrate_batch_pixelnorm(az_integrator *h, const void *frames_dev, int n_frames,
                                 int image_dtype, const float *dark, const float *flat,
                                 const float *solid_angle, const float *polarization,
                                 float *out_I, float *out_sum_corrected, float *out_count,
                                 az_stream_t stream);

/*
 * Propagated variance of each bin's signal sum under counting statistics (an extension:
 * the paper states no error model): a pixel's counts have a Poisson variance equal to their
 * value, clipped at 0, the dark current is a constant and pixels are independent, so
 * V_b = sum_p A_bp^2 max(img_p, 0); the standard error of I_b is sqrt(V_b) / N_b.
 * frames device [n_frames][ny][nx]; out_sum_variance device float [n_frames][nrows].
 * FP32 compensated, through the batched kernel (tensor-copy engine; AZ_EUNSUPPORTED for
 * tiles wider than 236 pixels or with AZ_COPY_ASYNC).
 */
int az_integrate_variance(az_integrator *h, const void *frames_dev, int n_frames,
                          int image_dtype, float *out_sum_variance, az_stream_t stream);

/*
 * End-to-end form of az_integrate_batch on HOST buffers: frames_host [n_frames][ny][nx]
 * (pinned memory gives overlapped copies; pageable memory works but copies serialise),
 * outputs out_I_host / out_sum_signal_host [n_frames][nrows] float (either may be NULL).
 * Correction arrays stay on the device.  Frames are copied in chunks on two internal
 * streams so that the upload of chunk k+1 overlaps the integration of chunk k.  Returns
 * after all results are in host memory.
 */
int az_integrate_batch_host(az_integrator *h, const void *frames_host, int n_frames,
                            int image_dtype, const float *dark, const float *flat,
                            const float *solid_angle, const float *polarization,
                            float *out_I_host, float *out_sum_signal_host, az_stream_t stream);

/* ---- adjoint (differentiation of the forward; gather over the pixel-major matrix) ---- */

/*
 * Given g_b = dL/dI_b and the forward's I and N (same precision), writes
 *   grad_image_p = sum_b A_bp g_b / N_b                       (= -dL/ddark_p)
 *   grad_flat_p  = -solid_angle_p pol_p sum_b A_bp g_b I_b / N_b
 * (bins with N_b == 0 contribute nothing), one thread per pixel gathering its own column,
 * no atomics.  precision FP64: grad_I, I, sum_norm and the outputs are double; FP32_COMP:
 * float with compensated sums.  Outputs: device [ny][nx]; either may be NULL.
 */
int az_integrate_backward(const az_integrator *h, const void *grad_I, const void *I,
                          const void *sum_norm, const float *solid_angle,
                          const float *polarization, int precision, void *out_grad_image,
                          void *out_grad_flat, az_stream_t stream);

/* ---- batched heterogeneous launch (several detectors in one persistent launch) ------- */

/*
 * A plan over n integrators of uneven shape and bin count, bound to fixed device buffers:
 * images[k] (device [ny_k][nx_k] of image_dtype), optional corrections per instance
 * (arrays of n pointers, or NULL for all-NULL), outputs out_I[k] / out_sum_signal[k] /
 * out_sum_norm[k] / out_count[k] (device float[nrows_k]; the pointer arrays may be NULL).
 * The plan flattens every (instance, tile) pair into one work list processed by one
 * persistent FP32-compensated launch, followed by one finalising launch.  The pointer
 * arrays are copied; the integrators must outlive the plan.
 */
int az_multi_create(az_integrator *const *handles, int n, const void *const *images,
                    int image_dtype, const float *const *darks, const float *const *flats,
                    const float *const *solid_angles, const float *const *polarizations,
                    float *const *out_I, float *const *out_sum_signal,
                    float *const *out_sum_norm, float *const *out_count, az_multi **out);

/* Run the plan on `stream`.  use_graph != 0: the first call captures the launches into a
 * CUDA graph (on `stream`), later calls replay it. */
int az_multi_launch(az_multi *plan, int use_graph, az_stream_t stream);
void az_multi_destroy(az_multi *plan);

/* ---- tuning ----------------------------------------------------------------------------- */

/*
 * Pick the pixel tile shape, rows per warp and frames per pass for this integrator by
 * timing the batched forward on n_trial_frames synthetic frames (allocated and freed
 * inside), then keep the fastest.  Rebuilds the tiled layout if the tile shape changes.
 * Then times one FP32 frame through the tiled form and through the look-up table (built for
 * the trial if missing, unless it would take more than four times the memory of the CSR
 * matrix's entries) and sets the single-frame layout (az_set_layout) to the faster; a table
 * built only for the trial is freed again if it loses.  Synchronises `stream`.  *best_ms
 * (may be NULL) receives the best time per frame of the batched forward.
 */
int az_autotune(az_integrator *h, int n_trial_frames, az_stream_t stream, double *best_ms);

/* Set the tuning by hand (0 keeps the current value).  tile_w must be a multiple of 4;
 * frames_per_pass is 1, 2, 4, 8, 16 or 32 and rows_per_warp = 32 / frames_per_pass (either
 * may be given; both must agree). */
int az_set_tuning(az_integrator *h, int tile_h, int tile_w, int rows_per_warp,
                  int frames_per_pass);

/* ---- look-up-table layout (Sec. 5.2) ------------------------------------------------------ */

/*
 * The matrix as a look-up table (Sec. 5.2, "scatter to gather"): for every output row the
 * (pixel index, coefficient) pairs it gathers from, in column order, padded with pairs
 * (-1, 0) to the length of the longest row, the table's width.  It is the paper's
 * array-of-structures alternative to the CSR form (Sec. 5.2.1, 6.1, 6.3), kept here as a
 * candidate layout of the single-frame forward.  Device storage is slot-major ([width][nrows]
 * pairs, so that the threads of a warp, which take consecutive rows, read consecutive pairs):
 * 8-byte pairs {int32 pixel, float coefficient} for AZ_PREC_FP32_COMP, 16-byte pairs
 * {int32 pixel, int32 0, double coefficient} for AZ_PREC_FP64, plus a per-pixel buffer of the
 * corrected frame and the per-chunk partial sums.  Owned by the integrator, freed with it.
 */
#define AZ_LAYOUT_TILED 0 /* the tiled CSR form (default) */
#define AZ_LAYOUT_LUT 1   /* the look-up table */

/* Build (or rebuild) the table of `precision` from the integrator's matrix on `stream`;
 * synchronises `stream` (the width is read back).  AZ_ENOMEM if it does not fit. */
int az_lut_build(az_integrator *h, int precision, az_stream_t stream);

/* The table as built.  *width (may be NULL) receives the slots per row (0 if no table was
 * built).  The host arrays, each NULL or [nrows][width] row-major with the padding:
 * pixel_host the pixel indices, coef32_host / coef64_host the coefficients of the FP32 /
 * FP64 table.  AZ_EINVAL if an array is asked of a table that is not built. Synchronous. */
int az_lut_export(const az_integrator *h, int64_t *width, int32_t *pixel_host, float *coef32_host,
                  double *coef64_host);

/*
 * One frame through the table: the four outputs of az_integrate1d / az_integrate2d (same
 * arguments, shapes, output types and error codes).  Three launches: a correction pass over
 * the pixels (cast, dark subtracted, flat * solid angle * polarisation formed: the separate
 * correction step of Sec. 6.4), the gather over each row's pairs, every row cut into chunks
 * summed by separate threads, and a pass that combines each row's chunk sums in a fixed order
 * (FP32: compensated) and forms I = S / N (0 where N = 0).  Deterministic.  Builds the table
 * of `precision` first if it is missing (allocates, synchronises `stream`).
 */
int az_integrate_lut(az_integrator *h, const void *image_dev, int image_dtype, const float *dark,
                     const float *flat, const float *solid_angle, const float *polarization,
                     int precision, void *out_I, void *out_sum_signal, void *out_sum_norm,
                     void *out_count, az_stream_t stream);

/* Which layout az_integrate1d / az_integrate2d use: AZ_LAYOUT_TILED or AZ_LAYOUT_LUT (the
 * table of the call's precision is built on the first call that needs it).  The batched,
 * variance, adjoint and many-instance entry points always use the tiled form.  az_autotune
 * sets it to whichever layout integrates one frame faster.  AZ_EINVAL for another value. */
int az_set_layout(az_integrator *h, int layout);

/* ---- failure detection ------------------------------------------------------------------ */

/*
 * Self-test of the bounded device-side wait (no counterpart in the paper).  Every staged
 * kernel of the library waits on shared-memory barriers with a bound, after which it records
 * AZ_ETIMEOUT in a status word and returns instead of hanging.  This launches one warp that
 * waits, with a bound of limit_cycles SM clock cycles (1 .. 2e9, about one second), on a
 * barrier that nothing completes (arrive == 0) or that the warp's first thread completes
 * first (arrive != 0), then writes the outcome to *out_status (host int): AZ_ETIMEOUT or
 * AZ_OK.  Synchronises `stream`; the context stays usable.  AZ_EINVAL for a NULL status
 * or a bound outside the range, before any launch.
 */
int az_selftest_wait(int arrive, int64_t limit_cycles, int *out_status, az_stream_t stream);

/* ---- kernel timing --------------------------------------------------------------------- */

/* Per-kernel totals recorded while profiling is enabled.  Kinds: 0 = phase-1 frames kernel
 * (az_integrate_batch*), 1 = phase-1 kernel of the frame-independent sums N and C,
 * 2 = phase-1 single-frame kernel (az_integrate1d/2d; with the look-up table, its gather),
 * 3 = phase-2 (finalise) kernel (with the look-up table, the chunk combination),
 * 4 = per-call preparation (per-entry dark gather, per-pixel flat * solid angle *
 * polarisation of az_integrate_batch*; the look-up table's correction pass). */
#define AZ_PROF_KINDS 5
typedef struct {
    int64_t launches[AZ_PROF_KINDS];
    double total_ms[AZ_PROF_KINDS];
} az_profile;

/* enable != 0: bracket every forward launch of this integrator with CUDA events on its
 * stream (a few microseconds per launch).  enable == 0 stops recording. */
int az_profile_enable(az_integrator *h, int enable);

/* Synchronise the recorded events, add up their durations per kernel kind into *out, and
 * clear the record. */
int az_profile_read(az_integrator *h, az_profile *out);

/* How the forward stages a pixel tile into shared memory.  AZ_COPY_TMA (the default) loads
 * each tile as four 2-D tensor boxes, one per class of rows with equal index mod 4 (rows of
 * one class are 16 * width bytes apart, which meets the tensor-map stride rule for any
 * width); it applies to tiles up to 236 pixels wide, wider tiles use AZ_COPY_ASYNC.
 * AZ_COPY_ASYNC issues 16-byte cp.async copies spread over the producer warps.  Results are
 * identical; only speed differs.  Defaults: 8 x 224 pixel tiles (32 x 64 for 2D integrators),
 * 8 frames per pass. */
int az_set_copy_engine(az_integrator *h, int engine);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *az_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AZINT_H */
