// Internal declarations shared by the CUDA translation units of the azint library.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "azint.h"

namespace azint {

// ------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------
int fail(int code, const char *fmt, ...);
void clear_error();

#define AZ_CUDA(expr)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::azint::fail(e_ == cudaErrorMemoryAllocation ? AZ_ENOMEM : AZ_ECUDA,  \
                                 "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),   \
                                 __FILE__, __LINE__);                                      \
    } while (0)

#define AZ_TRY(expr)                                                                       \
    do {                                                                                   \
        int rc_ = (expr);                                                                  \
        if (rc_ != AZ_OK) return rc_;                                                      \
    } while (0)

// Device allocation owned by the library (freed in the destructor).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t n) {
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(AZ_ENOMEM, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
        }
        bytes = n;
        return AZ_OK;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// ------------------------------------------------------------------------------------
// host-side objects
// ------------------------------------------------------------------------------------
struct GeomParams {
    double R[9];   // laboratory rotation Rz(rot3) Ry(rot2) Rx(rot1), row-major
    double dist, poni1, poni2, pixel1, pixel2, wavelength;
};

// Pixel-tiled layout of the matrix used by the forward kernels.  Entries are grouped by
// (tile, row, pixel); a "segment" is the run of one matrix row inside one tile.  Each
// tile's entries start on a multiple of 8 entries so that they can be bulk-copied.
struct TiledLayout {
    int th = 0, tw = 0, srow = 0;      // tile rows/cols, shared-memory row pitch (tw + 4 words)
    int ss = 0;                        // words per row-class slot (tile rows of equal index mod 4)
    int ntx = 0, nty = 0, ntiles = 0;  // tile grid
    int n_active = 0;                  // tiles with at least one entry
    int nseg = 0;
    int max_tile_entries = 0;          // padded entry count of the largest tile
    int max_tile_segments = 0;
    int64_t padded_nnz = 0;
    DevBuf tile_seg_ptr;    // int32 [ntiles + 1]
    DevBuf tile_ent_ptr;    // int32 [ntiles + 1]  (padded start of each tile's entries)
    DevBuf active_tiles;    // int32 [n_active]
    DevBuf seg_ent_ptr;     // int32 [nseg + 1]    (absolute, in the padded entry arrays)
    DevBuf seg_slot;        // int32 [nseg]        (position of the segment in row order)
    DevBuf row_slot_ptr;    // int32 [nrows + 1]
    DevBuf ent_loc;         // uint16 [padded_nnz] (shared-memory word offset in the tile)
    // Frame-pair layout of the batched frames kernel (srow_p == 0: none for this tile shape).
    // Frames F and F + 4 of a stage share a region of pw_p words: F's row-class slots at
    // sl * ss_p, F + 4's slot_p words (16 mod 32: other banks) later, rows at pitch srow_p.
    int srow_p = 0, ss_p = 0, slot_p = 0, pw_p = 0;
    DevBuf ent_loc_p;       // uint16 [padded_nnz] (word offset in the frame-pair layout)
    DevBuf ent_w32;         // float  [padded_nnz]
    DevBuf ent_w64;         // double [padded_nnz]
    DevBuf ent_pix;         // int32  [padded_nnz] (pixel of the entry; -1 for padding)
    DevBuf ent_dark;        // float  [padded_nnz] (dark of the entry's pixel, per batch call)
    DevBuf norm_frames;     // float  [2][ny][nx]: flat * solid angle * polarisation, then ones
    DevBuf ent_wnorm;       // float  [padded_nnz]: weight / (flat * solid angle * polarisation)
    // Per active tile: a 32-byte descriptor {tile, record offset (words), record words,
    // entry offset, padded entry count, segment count, 0, 0} and a 16-byte aligned record
    // {tile, ns, entry offset, entry count, slot[ns], uint16 start[ns + 1]} that the forward
    // copies into shared memory with the tile.
    DevBuf tile_desc;       // int32 [n_active][8]
    DevBuf tile_rec;        // int32 [sum of record words]
    int max_rec_words = 0;
};

}  // namespace azint

struct az_geometry {
    azint::GeomParams g;
    double rot1, rot2, rot3;
};

namespace azint {
// CUDA-event kernel timing (az_profile_enable / az_profile_read).
struct Profiler {
    bool on = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    ~Profiler() {
        for (auto &r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Optional CUDA-event bracket around one launch.
struct ProfScope {
    Profiler *p;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    ProfScope(Profiler *p_, int kind_, cudaStream_t s_) : p(p_ && p_->on ? p_ : nullptr), kind(kind_), s(s_) {
        if (p) { a = p->get(); cudaEventRecord(a, s); }
    }
    ~ProfScope() {
        if (p) {
            cudaEvent_t b = p->get();
            cudaEventRecord(b, s);
            p->recs.push_back({kind, a, b});
        }
    }
};
}  // namespace azint

// Frames one launch of the batched forward covers (its per-segment partial sums are kept
// for all of them): the matrix is read once per launch.
constexpr int kMaxFramesPerLaunch = 64;

struct az_integrator {
    int device = 0;
    int ny = 0, nx = 0, npt_rad = 0, npt_azim = 0, nrows = 0, unit = 0, split = 0;
    int n_unmasked = 0;
    int64_t nnz = 0;
    double lo = 0, hi = 0, delta = 0;
    // canonical CSR (rows = bins)
    azint::DevBuf csr_ptr, csr_idx, csr_w64;
    // pixel-major CSC (columns = pixels) for the adjoint
    azint::DevBuf csc_ptr, csc_row, csc_w64, csc_w32;
    azint::TiledLayout tl;
    // tuning
    int rows_per_warp = 4, frames_per_pass = 8, copy_engine = AZ_COPY_TMA;
    bool count_ready = false;  // norm[nrows..] holds C for the current tiled layout
    // scratch: per-segment partial sums and per-row frame-independent sums
    azint::DevBuf partial;     // float or double [planes][nseg]
    size_t partial_bytes = 0;
    azint::DevBuf norm;        // [2][nrows] (N, C) in the batch accumulation type
    azint::DevBuf adj;         // [2][nrows] doubles: adjoint row factors g/N and g I/N
    azint::DevBuf status;      // int32 device status word
    // look-up-table layout (built on request): [width][nrows] pairs, per-pixel corrected
    // (value, normalisation) of the current frame, per-chunk partial sums
    azint::DevBuf lut32, lut64, lut_vals, lut_part;
    // single FP32 frame through the frames kernel: [2][ny*nx] corrected frame and normalisation
    azint::DevBuf one_planes;
    int64_t lut_width = 0;
    int layout = AZ_LAYOUT_TILED;  // what az_integrate1d/2d use
    // corrections bound by az_set_corrections: per-entry darks, N and C of the current layout
    bool corr_bound = false, corr_dark = false;
    azint::DevBuf bound_ent_dark;  // float [padded_nnz]
    azint::DevBuf bound_norm;      // float [2][nrows]: N, C
    // host copies for the end-to-end path
    azint::DevBuf host_stage;  // device frames buffer for az_integrate_batch_host
    cudaStream_t copy_stream = nullptr;          // its upload stream, created on first use
    cudaEvent_t copy_events[5] = {};             // start, uploaded[2], consumed[2]
    cudaStream_t last_stream = nullptr;
    mutable azint::Profiler prof;
};

namespace azint {

// ------------------------------------------------------------------------------------
// launch helpers implemented in the .cu files
// ------------------------------------------------------------------------------------
int num_sms();
int launch_positions(const GeomParams &g, int ny, int nx, int unit, int where, double *rad,
                     double *chi, cudaStream_t s);
int build_integrator(int ny, int nx, const double *rad, const double *chi, int npt_rad,
                     int npt_azim, int unit, int split, const uint8_t *mask, cudaStream_t s,
                     az_integrator *h);
int build_tiled_layout(az_integrator *h, int th, int tw, cudaStream_t s);
int import_csr(az_integrator *h, const int32_t *indptr, const int32_t *indices, const double *data,
               cudaStream_t s);

// scan / sort primitives (csr_build.cu)
int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
int exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
int stable_sort_pairs(uint32_t *keys, int32_t *vals, int64_t n, int key_bits, cudaStream_t s);

// forward / backward launchers (integrate.cu, backward.cu)
int forward_single(const az_integrator *h, const void *image, int dtype, const float *dark,
                   const float *flat, const float *sa, const float *pol, int precision,
                   void *oI, void *oS, void *oN, void *oC, cudaStream_t s);
int forward_single_into(const az_integrator *h, const void *image, int dtype, const float *dark,
                        const float *flat, const float *sa, const float *pol, int precision,
                        void *oI, void *oS, void *oN, void *oC, void *partial, cudaStream_t s);
int preload_single_pass();
// set-up of the allocation-free entry point on the current device (noalloc.cu)
int noalloc_setup();
int forward_batch(az_integrator *h, const void *frames, int n, int dtype, const float *dark,
                  const float *flat, const float *sa, const float *pol, float *oI, float *oS,
                  float *oN, float *oC, cudaStream_t s);
int backward(const az_integrator *h, const void *g, const void *I, const void *N, const float *sa,
             const float *pol, int precision, void *g_img, void *g_flat, cudaStream_t s);
int batch_variance(az_integrator *h, const void *frames, int n, int dtype, float *oV, cudaStream_t s);
int batch_pixelnorm(az_integrator *h, const void *frames, int n, int dtype, const float *dark,
                    const float *flat, const float *sa, const float *pol, float *oI, float *oU,
                    float *oC, cudaStream_t s);
// argument checks shared by the forward entry points (NULL, dtype, 4-byte alignment)
int check_forward(const az_integrator *h, const void *image, int dtype, const float *dark,
                  const float *flat, const float *sa, const float *pol, const char *who);
int lut_build(az_integrator *h, int precision, cudaStream_t s);
int lut_forward(const az_integrator *h, const void *img, int dtype, const float *dark, const float *flat,
                const float *sa, const float *pol, int precision, void *oI, void *oS, void *oN, void *oC,
                cudaStream_t s);
int lut_export(const az_integrator *h, int64_t *width, int32_t *pix, float *c32, double *c64);
int forward_batch_one(az_integrator *h, const void *image, int dtype, const float *dark,
                      const float *flat, const float *sa, const float *pol, float *oI, float *oS,
                      float *oN, float *oC, cudaStream_t s);
int batch_norm(az_integrator *h, const float *flat, const float *sa, const float *pol, float *oN,
               float *oC, cudaStream_t s);
int batch_frames(az_integrator *h, const void *frames, int n, int dtype, const float *dark,
                 float *oI, float *oS, int frame_out0, cudaStream_t s,
                 const float *ent_dark_given = nullptr, const float *norm = nullptr);
int bind_corrections(az_integrator *h, const float *dark, const float *flat, const float *sa,
                     const float *pol, cudaStream_t s);
int forward_batch_bound(az_integrator *h, const void *frames, int n, int dtype, float *oI, float *oS,
                        float *oN, float *oC, cudaStream_t s);
int max_smem_per_block();

// ------------------------------------------------------------------------------------
// device helpers
// ------------------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    uint64_t st;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(smem_addr(bar)) : "memory");
    (void)st;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One try with the thread suspended by the hardware until the phase completes or `hint_ns`
// nanoseconds pass (no polling loop keeps the warp issuing while it waits).
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up (returns false) after about two seconds of
// the SM's clock, however long each suspended try lasts.
constexpr long long kWaitLimitCycles = 4000000000LL;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long limit = kWaitLimitCycles) {
    if (mbar_try_wait_hint(bar, parity, 1000000u)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait_hint(bar, parity, 1000000u))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Bulk (non-tensor) TMA copy global -> shared; 16-byte aligned addresses, size % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Kahan-compensated FP32 accumulation (Sec. 5.2.2): the running sum s and the compensation
// c (value = s - c).  The product is fused into the first subtraction (one rounding).
// Kahan accumulator with the compensation kept negated (nc = -c), so that one step is a
// fused multiply-add and three additions: y = w v + nc, t = s + y, nc = y - (t - s), s = t.
struct Kahan {
    float s, nc;
};
__device__ __forceinline__ void kahan_add(Kahan &k, float w, float v) {
    float y = __fmaf_rn(w, v, k.nc);
    float t = __fadd_rn(k.s, y);
    k.nc = __fsub_rn(y, __fsub_rn(t, k.s));
    k.s = t;
}
// Merge b into a with an error-free TwoSum of the running sums.
__device__ __forceinline__ void kahan_merge(Kahan &a, const Kahan &b) {
    float t = __fadd_rn(a.s, b.s);
    float z = __fsub_rn(t, a.s);
    float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(b.s, z));
    a.nc = __fadd_rn(__fadd_rn(a.nc, b.nc), e);
    a.s = t;
}
__device__ __forceinline__ float kahan_value(const Kahan &k) { return __fadd_rn(k.s, k.nc); }

__device__ __forceinline__ Kahan shfl_xor(const Kahan &k, int m) {
    Kahan r;
    r.s = __shfl_xor_sync(0xffffffffu, k.s, m);
    r.nc = __shfl_xor_sync(0xffffffffu, k.nc, m);
    return r;
}
#endif

}  // namespace azint
