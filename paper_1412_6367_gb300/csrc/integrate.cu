// Fused correction + sparse matrix-vector product (Sec. 5.2, Sec. 6.4) on the pixel-tiled
// layout.  Every form ends with the same deterministic phase 2; phase 1 comes in two kernels:
//
//   frames_kernel (persistent, one CTA per SM): a work item is a pixel tile (or a piece of
//     a heavy one) for every frame of the launch.  One producer warp copies the item's
//     record and entries (location, weight, per-entry dark) once into a ring of entry
//     buffers and streams the tile's pixels, G frames at a time, into a ring of plane stages
//     (bulk and tensor TMA, mbarrier-tracked, every wait bounded); 15 consumer warps give
//     lanes (segment, frame) pairs and write one partial sum per (segment, frame).  It serves
//     batches, the frame-independent sums N and C, the propagated variance, the per-pixel-
//     corrected form and single FP32 frames (after single_planes_kernel forms the corrected
//     frame and its normalisation per pixel).
//   phase1_kernel (persistent): one item per tile with all planes of one frame (image, dark,
//     flat, solid angle, polarisation) and the tile's entries in a ring of stages; four
//     lanes per segment form S, N and C.  It serves FP64 frames, the many-instance launch,
//     the allocation-free entry point and the cp.async copy engine.
//   phase 2: per (row, frame), the row's segment partials summed in a fixed order; then
//     S, N, C and I = S / N.
//
// Where a segment is one matrix row's entries inside one tile.  The image cast, the dark
// and flat * solid angle * polarisation are applied inside these kernels or in one per-pixel
// pass (the paper runs separate cast / correction / memset / integrate kernels).  FP32 sums
// are Kahan-compensated (Sec. 5.2.2); FP64 sums are plain.  No atomics touch the sums, so
// results are bit-reproducible run to run, and a frame gives the same bits alone or in any
// batch.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace azint {

namespace {

constexpr int kProducers = 4;                               // producer warps per CTA
constexpr int kConsumers = 16;                              // consumer warps per CTA
constexpr int kThreads = 32 * (kProducers + kConsumers);
constexpr uint32_t kFullCount = 32u * kProducers + 1u;       // arrivals completing a stage
constexpr int kMaxPlanes = 12;
constexpr int kMaxStages = 8;

enum Mode { MODE_SINGLE = 0, MODE_NORM = 1, MODE_FRAMES = 2 };

// Everything phase 1 and phase 2 need about one integrator and its inputs.
struct Inst {
    // tiled layout
    const int32_t *tile_seg_ptr, *tile_ent_ptr, *active_tiles;
    const int32_t *seg_start, *seg_end, *seg_slot, *row_slot_ptr;
    const uint16_t *ent_loc;
    const void *ent_w;
    int ny, nx, th, tw, srow, ss, ntx, rpw, nseg, nrows;
    int64_t npix;
    // inputs
    const char *img;  // first frame of this launch
    int n_frames, fpi, n_groups;
    const float *dark, *flat, *sa, *pol;
    // scratch and outputs
    void *partial;       // [planes][nseg] in the accumulation type
    float *norm;         // [2][nrows] N, C (FP32 batched path)
    void *oI, *oS, *oN, *oC;
    int frame_out0;      // first output frame of this launch
    int norm_rows;       // norm pass: 2 = partials hold N and C, 1 = N only
    int64_t item_begin, row_begin;
    int n_items;
    int stage_entries;
    int *status;
    const int32_t *tile_desc, *tile_rec;  // per active tile: descriptor [8] and record
    const float *ent_dark;                // frames pass: dark of each entry's pixel (or NULL)
    const CUtensorMap *maps;              // many-instance launch: this instance's [5][4] maps
    int single_nc;  // single-frame phase 2 in FP32: 0 S, N, C from the partials; 1 C from
                    // the per-layout cache norm[nrows..]; 2 N and C from that cache (N == C)
};

struct StageGeom {
    uint32_t plane_words;   // words per plane slot
    uint32_t plane_region;  // bytes of the plane region
    uint32_t ent_cap;       // entry capacity (staged entries)
    uint32_t stage_bytes;   // bytes per stage (multiple of 128)
    uint32_t rec_cap;       // bytes reserved for the tile record
    int ent_dk;             // entries carry a staged per-entry dark (frames pass)
    int nstages;            // pipeline depth
};

// Number of planes staged per item and the base address of plane `pl`: image frames
// first, then the corrections the mode reads (dark for single/frames; flat, solid angle,
// polarisation for single/norm), skipping absent ones.
template <int MODE>
__device__ __forceinline__ int plane_count(const Inst &d, int nimg) {
    int n = nimg;
    if (MODE == MODE_SINGLE && d.dark) ++n;
    if (MODE != MODE_FRAMES) n += (d.flat != nullptr) + (d.sa != nullptr) + (d.pol != nullptr);
    return n;
}

template <int MODE>
__device__ __forceinline__ const char *plane_base(const Inst &d, int f0, int nimg, int pl, int &kind) {
    if (pl < nimg) { kind = 0; return d.img + (size_t)(f0 + pl) * (size_t)d.npix * 4u; }
    int k = pl - nimg;
    if (MODE == MODE_SINGLE && d.dark) { if (k == 0) { kind = 1; return (const char *)d.dark; } --k; }
    if (MODE != MODE_FRAMES) {
        if (d.flat) { if (k == 0) { kind = 2; return (const char *)d.flat; } --k; }
        if (d.sa) { if (k == 0) { kind = 3; return (const char *)d.sa; } --k; }
        if (d.pol) { if (k == 0) { kind = 4; return (const char *)d.pol; } --k; }
    }
    kind = -1;
    return nullptr;
}

__device__ __forceinline__ const Inst &inst_of(const Inst &single, const Inst *multi, int n_inst,
                                               int64_t item) {
    if (!multi) return single;
    int lo = 0, hi = n_inst;  // last instance with item_begin <= item
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (multi[mid].item_begin <= item) lo = mid; else hi = mid;
    }
    return multi[lo];
}

struct TileDesc {
    int t, rec_off, rec_words, e_off, ne, ns;
};

__device__ __forceinline__ TileDesc load_desc(const Inst &d, int64_t local) {
    const int a = (int)(local / d.n_groups);
    const int4 *p = reinterpret_cast<const int4 *>(d.tile_desc) + 2 * (size_t)a;
    const int4 x = __ldg(p), y = __ldg(p + 1);
    return TileDesc{x.x, x.y, x.z, x.w, y.x, y.y};
}

// Words between two staged planes: four 128-byte aligned row-class slots and a band of 32
// words that holds zeros (the padding entries of the matrix point there: their weight is 0
// and the value they read is 0, whatever the image holds).  Planes are spread over the
// shared-memory banks by per-plane shifts of 4 * s words that the copies apply.
constexpr uint32_t kZeroBand = 32;
__host__ __device__ __forceinline__ uint32_t plane_stride(int ss) { return 4u * (uint32_t)ss + kZeroBand; }

// Zero words band_from .. pw - 1 of every plane of every stage (never written by the copies):
// the band after a plane, or in the frame-pair layout the tail of a region that holds both
// frames' bands.
__device__ __forceinline__ void zero_bands(unsigned char *first_plane, uint32_t stage_bytes, int nstages,
                                           int planes, uint32_t pw, uint32_t band_from) {
    const int band = (int)(pw - band_from);
    const int per_stage = planes * band;
    for (int i = threadIdx.x; i < nstages * per_stage; i += blockDim.x) {
        const int st = i / per_stage, r = i - st * per_stage;
        const int pl = r / band, w = r - pl * band;
        reinterpret_cast<uint32_t *>(first_plane + (size_t)st * stage_bytes)[(size_t)pl * pw + band_from + w] = 0u;
    }
}

// Four 2D tensor maps per staged array, one per tile-row class (rows of equal index mod 4,
// 16 * nx bytes apart).  Index: 0 image, 1 dark, 2 flat, 3 solid angle, 4 polarisation.
// pair: the image's four class maps in three dimensions (x, class row, period of four
// frames) for the frame-pair layout of the frames kernel.
struct TmaSet {
    CUtensorMap m[5][4];
    CUtensorMap pair[4];
};

// Stage layout: [header 256 B][tile record][planes][entry locs][entry weights].
// Header ints: 0 ns, 1 group, 2 nimg, 3..6 word offsets of dark, flat, solid angle,
// polarisation in the plane region (-1 = absent), 7 tile, 8 entry offset, 16.. image planes.
constexpr uint32_t kHeaderBytes = 256;

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Producer warps: stage work item `local` of instance d.  Warp 0 writes the item header and
// bulk-copies (TMA) the tile record and entries.  Each plane of the tile is staged as four
// row classes (tile rows of equal index mod 4, which are 16 * nx bytes apart in global
// memory): with the TMA engine one 2D tensor copy per class -- a box of srow x (th / 4)
// words into a 128-byte aligned slot -- and with the cp.async engine the same words in
// 16-byte pieces spread over all producer lanes.  For a plane whose base address is beta
// words mod 4 and whose first tile row is global row g0, class k goes to slot
// s = (k - g0) mod 4, and the box starts at column X = c0 - 4 (flag + spread) where
// off_k = (beta + k nx) mod 4, c_s = (nx s) mod 4, phi = (beta + nx g0) mod 4,
// flag = (c_s + phi - off_k) / 4 in {0, 1} and spread = plane mod 4.  Pixel (ly, c0 + lx)
// then sits at the build-time offset plus phi + 4 spread, the per-plane shift the consumers
// add.  Every producer thread makes one arrival per item (deferred until its cp.async copies
// land) and lane 0 of warp 0 one more after publishing the header: kFullCount arrivals.
template <int MODE, class WT, bool TMA>
__device__ void produce(const Inst &d, const TmaSet &tm, int64_t local, const TileDesc &td,
                        unsigned char *stage, const StageGeom &sg, uint64_t *bar, int *ctr,
                        int pwarp) {
    const int lane = threadIdx.x & 31;
    const int group = (int)(local % d.n_groups);
    const int t = td.t;
    const int ti = t / d.ntx, tj = t - ti * d.ntx;
    const int r0 = ti * d.th, c0 = tj * d.tw;
    const int f0 = group * d.fpi;
    const int nimg = MODE == MODE_SINGLE ? 1 : (MODE == MODE_FRAMES ? min(d.fpi, d.n_frames - f0) : 0);
    const int np = plane_count<MODE>(d, nimg);
    const uint32_t pw = plane_stride(d.ss);
    const int nu = d.nx & 3;
    const int rows4 = d.th >> 2;          // rows per class in a tile
    const int boxw = d.srow;              // words per staged row (tw + 20)
    unsigned char *rec_dst = stage + kHeaderBytes;
    uint32_t *planes = reinterpret_cast<uint32_t *>(stage + kHeaderBytes + sg.rec_cap);
    unsigned char *eloc = stage + kHeaderBytes + sg.rec_cap + sg.plane_region;
    unsigned char *ew = eloc + sg.ent_cap * 2u;
    const uint32_t ne = (uint32_t)td.ne;
    const bool stage_e = d.stage_entries != 0;

    // plane geometry: array base, first global row of the tile in that array, rows in it
    auto plane_geo = [&](int pl, const char *&arr, int64_t &g0, int64_t &rows_total, int &kind) {
        if (pl < nimg) {
            kind = 0;
            arr = d.img;
            g0 = (int64_t)(f0 + pl) * d.ny + r0;
            rows_total = (int64_t)d.n_frames * d.ny;
        } else {
            plane_base<MODE>(d, f0, nimg, pl, kind);
            arr = kind == 1 ? (const char *)d.dark : kind == 2 ? (const char *)d.flat
                : kind == 3 ? (const char *)d.sa : (const char *)d.pol;
            g0 = r0;
            rows_total = d.ny;
        }
    };

    if (pwarp == 0) {
        uint32_t mine = 0;
        if (TMA) {
            // lane pl * 4 + k copies class k of plane pl
            for (int job = lane; job < 4 * np; job += 32) {
                const int pl = job >> 2, k = job & 3;
                const char *arr;
                int64_t g0, rows_total;
                int kind;
                plane_geo(pl, arr, g0, rows_total, kind);
                const int phi = (int)(g0 & 3);
                const int sl = (k - phi) & 3;
                if (g0 + sl < rows_total) mine += (uint32_t)(boxw * rows4 * 4);
            }
        }
        const bool dk = MODE == MODE_FRAMES && d.ent_dark != nullptr && stage_e;
        if (lane == 0) {
            mine += (uint32_t)td.rec_words * 4u;
            if (stage_e) mine += ne * 2u + ne * (uint32_t)sizeof(WT);
            if (dk) mine += ne * 4u;
        }
        fence_proxy_async_smem();
        if (mine)
            asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
                         "r"(mine)
                         : "memory");
        if (lane == 0) {
            bulk_g2s(rec_dst, d.tile_rec + td.rec_off, (uint32_t)td.rec_words * 4u, bar);
            if (stage_e && ne) {
                bulk_g2s(eloc, d.ent_loc + td.e_off, ne * 2u, bar);
                bulk_g2s(ew, static_cast<const WT *>(d.ent_w) + td.e_off, ne * (uint32_t)sizeof(WT), bar);
            }
            if (dk && ne) bulk_g2s(ew + sg.ent_cap * (uint32_t)sizeof(WT), d.ent_dark + td.e_off, ne * 4u, bar);
        }
        if (TMA) {
            for (int job = lane; job < 4 * np; job += 32) {
                const int pl = job >> 2, k = job & 3;
                const char *arr;
                int64_t g0, rows_total;
                int kind;
                plane_geo(pl, arr, g0, rows_total, kind);
                const int beta = (int)((reinterpret_cast<uintptr_t>(arr) >> 2) & 3u);
                const int phi_row = (int)(g0 & 3);
                const int sl = (k - phi_row) & 3;
                if (g0 + sl >= rows_total) continue;
                const int phi = (beta + nu * phi_row) & 3;
                const int offk = (beta + k * nu) & 3;
                const int cs = (nu * sl) & 3;
                const int flag = (cs + phi - offk) >> 2;
                const int x = c0 - 4 * (flag + (pl & 3));
                uint32_t *dst = planes + (size_t)pl * pw + (size_t)sl * d.ss;
                const int y = (int)((g0 + sl - k) >> 2);
                const CUtensorMap *map = d.maps ? d.maps + 4 * kind + k : &tm.m[kind][k];
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
                    "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
                    : "memory");
            }
        }
    }
    if (!TMA) {
        // the same words as the tensor copies: for every (plane, class, row in class) a run of
        // boxw / 4 16-byte pieces from column c0 - off_k; eight lanes per run
        const int sub = lane >> 3, l8 = lane & 7;
        const int runs = np * 4 * rows4;
        const int nchunk = boxw >> 2;
        for (int r = pwarp * 4 + sub; r < runs; r += 4 * kProducers) {
            const int pl = r / (4 * rows4);
            const int rem = r - pl * 4 * rows4;
            const int k = rem / rows4, jj = rem - k * rows4;
            const char *arr;
            int64_t g0, rows_total;
            int kind;
            plane_geo(pl, arr, g0, rows_total, kind);
            const int beta = (int)((reinterpret_cast<uintptr_t>(arr) >> 2) & 3u);
            const int phi_row = (int)(g0 & 3);
            const int sl = (k - phi_row) & 3;
            const int64_t g = g0 + sl + 4 * (int64_t)jj;  // global row of this run
            if (g >= rows_total) continue;
            const int phi = (beta + nu * phi_row) & 3;
            const int offk = (beta + k * nu) & 3;
            const int cs = (nu * sl) & 3;
            const int flag = (cs + phi - offk) >> 2;
            const int x = c0 - 4 * (flag + (pl & 3));
            uint32_t *dst = planes + (size_t)pl * pw + (size_t)sl * d.ss + (size_t)jj * boxw;
            const int64_t e0 = g * d.nx + x - offk;       // first element of the run (in the array)
            const int64_t elems = rows_total * d.nx;
            const char *src = arr + 4 * e0;               // 16-byte aligned by construction
            for (int c = l8; c < nchunk; c += 8) {
                // copy every piece that overlaps the array; a piece is 16-byte aligned, so the
                // words it holds outside the array share a 16-byte granule with one inside it
                const int64_t ec = e0 + 4 * c;
                if (ec + 3 >= 0 && ec < elems) cp_async16(dst + 4 * c, src + 16 * c);
            }
        }
        cp_async_arrive(bar);  // deferred arrival when this thread's copies have landed
    } else {
        mbar_arrive(bar);
    }
    if (pwarp == 0) {
        // the zero band of every plane of this item (planes of different instances have
        // different strides, so the bands move from item to item)
        for (int pl = 0; pl < np; ++pl) planes[(size_t)pl * pw + pw - kZeroBand + lane] = 0u;
        __syncwarp();
    }
    if (pwarp == 0 && lane == 0) {
        int *h = reinterpret_cast<int *>(stage);
        h[0] = td.ns; h[1] = group; h[2] = nimg; h[3] = h[4] = h[5] = h[6] = -1;
        h[7] = t; h[8] = td.e_off;
        for (int pl = 0; pl < np; ++pl) {
            const char *arr;
            int64_t g0, rows_total;
            int kind;
            plane_geo(pl, arr, g0, rows_total, kind);
            const int beta = (int)((reinterpret_cast<uintptr_t>(arr) >> 2) & 3u);
            const int phi = (beta + nu * (int)(g0 & 3)) & 3;
            const int o = (int)(pl * pw + phi + 4 * (pl & 3));
            if (kind == 0) h[16 + pl] = o; else h[2 + kind] = o;
        }
        *ctr = 0;          // segment claim counter of this stage
        mbar_arrive(bar);  // publishes the header and the counter
    }
}

template <int DT>
__device__ __forceinline__ float img_f32(uint32_t w) {
    if (DT == AZ_DTYPE_F32) return __uint_as_float(w);
    if (DT == AZ_DTYPE_U32) return __uint2float_rn(w);
    return __int2float_rn((int)w);
}
template <int DT>
__device__ __forceinline__ double img_f64(uint32_t w) {
    if (DT == AZ_DTYPE_F32) return (double)__uint_as_float(w);
    if (DT == AZ_DTYPE_U32) return (double)w;
    return (double)(int)w;
}

// Accumulators: Kahan (FP32 compensated) or plain double.
template <class A> struct Acc;
template <> struct Acc<float> {
    Kahan k;
    __device__ void zero() { k.s = 0.f; k.nc = 0.f; }
    __device__ void add(float w, float v) { kahan_add(k, w, v); }
    __device__ void merge(const Acc<float> &o) { kahan_merge(k, o.k); }
    __device__ void merge_xor(int m) {
        // lower lane's partial sum on the left: every lane ends with lane 0's value
        const Kahan o = shfl_xor(k, m);
        if ((threadIdx.x & m) != 0) {
            Kahan l = o;
            kahan_merge(l, k);
            k = l;
        } else {
            kahan_merge(k, o);
        }
    }
    // the partner lane's sum merged in, the lower lane's on the left (its value is right on
    // the lower lane of each pair; the upper lane ends with the pair in the other order)
    __device__ void merge_lower_left(int m) {
        const Kahan o = shfl_xor(k, m);
        if ((threadIdx.x & m) == 0) kahan_merge(k, o);
    }
    __device__ float value() const { return kahan_value(k); }
};
template <> struct Acc<double> {
    double s;
    __device__ void zero() { s = 0.0; }
    __device__ void add(double w, double v) { s = __fma_rn(w, v, s); }
    __device__ void merge(const Acc<double> &o) { s += o.s; }
    __device__ void merge_xor(int m) { s += __shfl_xor_sync(0xffffffffu, s, m); }
    __device__ void merge_lower_left(int m) {
        const double o = __shfl_xor_sync(0xffffffffu, s, m);
        if ((threadIdx.x & m) == 0) s = s + o;
    }
    __device__ double value() const { return s; }
};

// What a consumer needs about its instance, loaded once per item into registers.
struct ConsumerParams {
    void *partial;
    const uint16_t *ent_loc;
    const void *ent_w;
    const float *ent_dark;
    int nseg, fpi, stage_entries;
};

__device__ __forceinline__ ConsumerParams consumer_params(const Inst &d) {
    return ConsumerParams{d.partial, d.ent_loc, d.ent_w, d.ent_dark, d.nseg, d.fpi, d.stage_entries};
}

template <class WT> struct W4;
template <> struct W4<float> {
    static __device__ __forceinline__ void load(const float *p, float w[4]) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
};
template <> struct W4<double> {
    static __device__ __forceinline__ void load(const double *p, double w[4]) {
        const double2 a = *reinterpret_cast<const double2 *>(p);
        const double2 b = *reinterpret_cast<const double2 *>(p + 2);
        w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
    }
};

// One lane per (segment, quantity).  A warp takes 32 / Q segments at a time from the stage's
// claim counter; the Q lanes of a segment share its entry stream (broadcast reads) and each
// sums one quantity over all of the segment's entries:
//   frames pass: quantity q = frame q of the item, value = cast(image) - dark;
//   norm pass:   q = 0: flat * solid angle * polarisation, q = 1: 1 (the count).
// Segments start on a multiple of 4 entries and hold whole quads (the layout pads them with
// entries of weight 0 that read the plane's zero band).  Entries are read four at a time (one
// 8-byte read of the locations, 16-byte reads of the weights and per-entry darks); entry e
// goes to accumulator e mod 4 and the four are combined as ((a0 + a1) + (a2 + a3)).  Every quantity of every pass is reduced
// by this same sequence of operations, so a flat image with unit corrections gives S == N bit
// for bit, and a frame integrated alone or in a batch gives the same bits.
template <int Q, class AT, class WT, int MODE, int DT, bool SE>
__device__ void consume_serial(const ConsumerParams &cp, const unsigned char *stage,
                               const StageGeom &sg, int *ctr) {
    static_assert(MODE != MODE_SINGLE, "the single pass has its own consumer");
    constexpr int R = 32 / Q;
    const int lane = threadIdx.x & 31;
    const int sub = lane / Q, q = lane % Q;
    const int *h = reinterpret_cast<const int *>(stage);
    const int ns = h[0], group = h[1], nimg = h[2];
    const int odark = h[3], oflat = h[4], osa = h[5], opol = h[6];
    const int oimg = h[16 + (MODE == MODE_FRAMES ? q : 0)];
    const bool active = MODE == MODE_FRAMES ? q < nimg : true;
    const int *slots = reinterpret_cast<const int *>(stage + kHeaderBytes) + 4;
    const uint16_t *starts = reinterpret_cast<const uint16_t *>(slots + ns);
    const uint32_t *planes = reinterpret_cast<const uint32_t *>(stage + kHeaderBytes + sg.rec_cap);
    const uint16_t *L;
    const WT *W;
    const float *DK;
    if constexpr (SE) {
        const unsigned char *eb = stage + kHeaderBytes + sg.rec_cap + sg.plane_region;
        L = reinterpret_cast<const uint16_t *>(eb);
        W = reinterpret_cast<const WT *>(eb + sg.ent_cap * 2u);
        DK = reinterpret_cast<const float *>(eb + sg.ent_cap * (2u + (uint32_t)sizeof(WT)));
    } else {
        L = cp.ent_loc + h[8];
        W = static_cast<const WT *>(cp.ent_w) + h[8];
        DK = cp.ent_dark ? cp.ent_dark + h[8] : nullptr;
    }
    const bool has_dk = MODE == MODE_FRAMES && sg.ent_dk;
    size_t orow;
    if (MODE == MODE_FRAMES) orow = (size_t)(group * cp.fpi + q) * cp.nseg;
    else orow = (size_t)q * cp.nseg;
    AT *out = static_cast<AT *>(cp.partial) + orow;
    while (true) {
        int b = 0;
        if (lane == 0) b = atomicAdd(ctr, R);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= ns) break;
        const int sl = b + sub;
        int e0 = 0, e1 = 0, slot = 0;
        if (sl < ns) {
            e0 = starts[sl];
            e1 = starts[sl + 1];
            slot = slots[sl];
        }
        if (!active) e1 = e0;
        Acc<AT> acc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j].zero();
        for (int qd = e0; qd < e1; qd += 4) {
            const uint2 l2 = *reinterpret_cast<const uint2 *>(L + qd);
            const int loc[4] = {(int)(l2.x & 0xffffu), (int)(l2.x >> 16), (int)(l2.y & 0xffffu),
                                (int)(l2.y >> 16)};
            WT w[4];
            W4<WT>::load(W + qd, w);
            float dk[4] = {0.f, 0.f, 0.f, 0.f};
            if (has_dk) {
                const float4 v = *reinterpret_cast<const float4 *>(DK + qd);
                dk[0] = v.x; dk[1] = v.y; dk[2] = v.z; dk[3] = v.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                AT x;
                if (MODE == MODE_FRAMES) {
                    float v = img_f32<DT>(planes[oimg + loc[j]]);
                    if (has_dk) v = __fsub_rn(v, dk[j]);
                    x = (AT)v;
                } else {
                    AT n = AT(1);
                    if (q == 0) {
                        if (oflat >= 0) n = n * (AT)__uint_as_float(planes[oflat + loc[j]]);
                        if (osa >= 0) n = n * (AT)__uint_as_float(planes[osa + loc[j]]);
                        if (opol >= 0) n = n * (AT)__uint_as_float(planes[opol + loc[j]]);
                    }
                    x = n;
                }
                acc[j].add((AT)w[j], x);
            }
        }
        acc[0].merge(acc[1]);
        acc[2].merge(acc[3]);
        acc[0].merge(acc[2]);
        if (sl < ns && active) out[slot] = acc[0].value();
    }
}

// Single-frame mode, four lanes per segment: lane j of a segment keeps accumulator j of each
// of the three sums (the entries e = j mod 4, in order), with per entry x = image - dark,
// n = ((1 flat) solid angle) polarisation and 1, each added with its weight (FP32:
// compensated; FP64: fused multiply-adds); the four lanes are merged by shuffles as
// ((a0 + a1) + (a2 + a3)), the order every other reduction of the library uses, so a frame's
// FP32 sums have the bits of the frames kernel's.  A quarter of the chain per lane, every
// lane busy, eight segments per claim.  Without flat, solid angle and polarisation n = 1 for
// every entry, so N is C and is not formed twice.
template <class AT, class WT, int DT, bool SE>
__device__ void consume_single_split(const ConsumerParams &cp, const unsigned char *stage,
                                     const StageGeom &sg, int *ctr) {
    const int lane = threadIdx.x & 31;
    const int j = lane & 3, sub = lane >> 2;
    const int *h = reinterpret_cast<const int *>(stage);
    const int ns = h[0];
    const int odark = h[3], oflat = h[4], osa = h[5], opol = h[6];
    const int oimg = h[16];
    const bool norm1 = oflat < 0 && osa < 0 && opol < 0;
    const int *slots = reinterpret_cast<const int *>(stage + kHeaderBytes) + 4;
    const uint16_t *starts = reinterpret_cast<const uint16_t *>(slots + ns);
    const uint32_t *planes = reinterpret_cast<const uint32_t *>(stage + kHeaderBytes + sg.rec_cap);
    const uint16_t *L;
    const WT *W;
    if constexpr (SE) {
        const unsigned char *eb = stage + kHeaderBytes + sg.rec_cap + sg.plane_region;
        L = reinterpret_cast<const uint16_t *>(eb);
        W = reinterpret_cast<const WT *>(eb + sg.ent_cap * 2u);
    } else {
        L = cp.ent_loc + h[8];
        W = static_cast<const WT *>(cp.ent_w) + h[8];
    }
    AT *out = static_cast<AT *>(cp.partial);
    while (true) {
        int b = 0;
        if (lane == 0) b = atomicAdd(ctr, 8);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= ns) break;
        const int sl = b + sub;
        const bool live = sl < ns;
        const int e0 = live ? starts[sl] : 0, e1 = live ? starts[sl + 1] : 0, slot = live ? slots[sl] : 0;
        Acc<AT> aS, aN, aC;
        aS.zero(); aN.zero(); aC.zero();
        for (int e = e0 + j; e < e1; e += 4) {
            const int loc = L[e];
            const AT w = (AT)W[e];
            AT x, n = AT(1);
            if (sizeof(AT) == 8) {
                x = (AT)img_f64<DT>(planes[oimg + loc]);
                if (odark >= 0) x = x - (AT)__uint_as_float(planes[odark + loc]);
            } else {
                float v = img_f32<DT>(planes[oimg + loc]);
                if (odark >= 0) v = __fsub_rn(v, __uint_as_float(planes[odark + loc]));
                x = (AT)v;
            }
            if (oflat >= 0) n = n * (AT)__uint_as_float(planes[oflat + loc]);
            if (osa >= 0) n = n * (AT)__uint_as_float(planes[osa + loc]);
            if (opol >= 0) n = n * (AT)__uint_as_float(planes[opol + loc]);
            aS.add(w, x);
            if (!norm1) aN.add(w, n);
            aC.add(w, AT(1));
        }
        // lanes 0 and 2 form a0 + a1 and a2 + a3 (lower lane on the left); lane 0 adds them
        aS.merge_lower_left(1); aC.merge_lower_left(1);
        aS.merge_lower_left(2); aC.merge_lower_left(2);
        if (!norm1) { aN.merge_lower_left(1); aN.merge_lower_left(2); }
        if (live && j == 0) {
            out[slot] = aS.value();
            out[(size_t)cp.nseg + slot] = norm1 ? aC.value() : aN.value();
            out[2 * (size_t)cp.nseg + slot] = aC.value();
        }
    }
}

template <class AT, class WT, int MODE, int NIMG, int DT>
__device__ __forceinline__ void consume_dispatch(const ConsumerParams &cp, const unsigned char *stage,
                                                 const StageGeom &sg, int *ctr) {
    if constexpr (MODE == MODE_SINGLE) {
        if (cp.stage_entries) consume_single_split<AT, WT, DT, true>(cp, stage, sg, ctr);
        else consume_single_split<AT, WT, DT, false>(cp, stage, sg, ctr);
    } else {
        constexpr int Q = MODE == MODE_FRAMES ? NIMG : 2;
        if (cp.stage_entries) consume_serial<Q, AT, WT, MODE, DT, true>(cp, stage, sg, ctr);
        else consume_serial<Q, AT, WT, MODE, DT, false>(cp, stage, sg, ctr);
    }
}

// Warp-specialised persistent kernel.  Warp 0 produces: for each work item of this CTA
// (static round robin) it waits until the stage is free (empty barrier), copies the item
// into it and arms the full barrier.  Warps 1..kConsumers consume: they wait for the item's
// full barrier, claim and reduce its segments, and release the stage (empty barrier, one
// arrival per consumer warp).  Every wait is bounded; a wait that gives up records
// AZ_ETIMEOUT in the status word, raises the CTA's abort flag and leaves, the producer
// first giving its own copies in flight a bounded grace period.
template <class AT, class WT, int MODE, int NIMG, int DT, bool TMA>
__global__ void __launch_bounds__(kThreads, 1)
phase1_kernel(const __grid_constant__ Inst single, const Inst *__restrict__ multi, int n_inst,
              int64_t n_items, StageGeom sg, const __grid_constant__ TmaSet tm) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // tensor copies want 128-byte aligned destinations: align explicitly (128 bytes of slack)
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127u) & ~static_cast<uintptr_t>(127u));
    const int S = sg.nstages;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * sg.stage_bytes);
    uint64_t *empty = full + S;
    int *ctr = reinterpret_cast<int *>(empty + S);
    volatile int *abort_flag = ctr + S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *status = single.status ? single.status : multi[0].status;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], kFullCount);
            mbar_init(&empty[s], kConsumers);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (warp < kProducers) {
        int k = 0;
        int64_t item = blockIdx.x;
        // the instance of the current and of the next item, searched for again only when an
        // item leaves the range of the last one found
        const Inst *dc = &single, *dn = &single;
        auto find = [&](int64_t it, const Inst *hint) -> const Inst * {
            if (!multi || (it >= hint->item_begin && it < hint->item_begin + hint->n_items)) return hint;
            return &inst_of(single, multi, n_inst, it);
        };
        TileDesc td{};
        if (item < n_items) {
            if (multi) dc = dn = &inst_of(single, multi, n_inst, item);
            td = load_desc(*dc, item - dc->item_begin);
        }
        for (; item < n_items; item += gridDim.x, ++k) {
            const int s = k % S, n = k / S;
            // prefetch the next item's descriptor while this one is staged
            const int64_t next = item + gridDim.x;
            TileDesc tn{};
            dc = dn;
            if (next < n_items) {
                dn = find(next, dc);
                tn = load_desc(*dn, next - dn->item_begin);
            }
            bool ok = true;
            if (n > 0) ok = mbar_wait_bounded(&empty[s], (uint32_t)((n - 1) & 1));
            ok = __all_sync(0xffffffffu, ok);
            if (__any_sync(0xffffffffu, !ok || *abort_flag != 0)) {  // warp-uniform decision
                if (lane == 0) {
                    if (!ok) atomicExch(status, AZ_ETIMEOUT);
                    *abort_flag = 1;
                    for (int j = k - 1; j >= 0 && j >= k - S; --j)  // grace for own copies
                        mbar_wait_bounded(&full[j % S], (uint32_t)((j / S) & 1));
                }
                asm volatile("cp.async.wait_all;" ::: "memory");
                break;
            }
            produce<MODE, WT, TMA>(*dc, tm, item - dc->item_begin, td, smem + (size_t)s * sg.stage_bytes,
                                   sg, &full[s], &ctr[s], warp);
            td = tn;
        }
    } else {
        int k = 0;
        // a CTA's items (every gridDim.x-th) mostly stay in one instance for many rounds:
        // the instance's parameters are looked up again only when the item leaves its range
        ConsumerParams cp = consumer_params(single);
        int64_t cur_begin = 0, cur_end = multi ? 0 : n_items;
        for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x, ++k) {
            const int s = k % S, n = k / S;
            if (item < cur_begin || item >= cur_end) {
                const Inst &d = inst_of(single, multi, n_inst, item);
                cp = consumer_params(d);
                cur_begin = d.item_begin;
                cur_end = d.item_begin + d.n_items;
            }
            bool ok = mbar_wait_bounded(&full[s], (uint32_t)(n & 1));
            ok = __all_sync(0xffffffffu, ok);
            if (__any_sync(0xffffffffu, !ok || *abort_flag != 0)) {  // warp-uniform decision
                if (lane == 0) {
                    if (!ok) atomicExch(status, AZ_ETIMEOUT);
                    *abort_flag = 1;
                }
                break;
            }
            consume_dispatch<AT, WT, MODE, NIMG, DT>(cp, smem + (size_t)s * sg.stage_bytes, sg, &ctr[s]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
}

// ------------------------------------------------------------------------------------
// frames pass with tile-resident entries
// ------------------------------------------------------------------------------------
// The batched frames pass spends most of its bytes on pixels, so a work item is one pixel
// tile for every frame of the launch: the tile's record and entries (location, weight,
// dark) are copied once into one of two entry buffers and stay there while the tile's
// pixels stream through a ring of plane stages, G frames per stage.  One producer warp
// issues every copy (bulk and tensor TMA); 15 consumer warps reduce (16 warps in all, four
// per scheduler: with 16 consumers the 64-frame Pilatus pass took 2.5% longer, with 20 or
// 24 longer still).  The consumer
// arithmetic is exactly that of the frames mode of phase1_kernel: the same entry order,
// accumulator assignment and merge, so results do not depend on the kernel that made them.
constexpr int kFrConsumers = 15;
constexpr int kFrThreads = 32 * (1 + kFrConsumers);
constexpr int kFrMaxStages = 8;
constexpr int kFrMaxEbufs = 6;
// What the frames kernel sums per entry: w (img), w (img - dark), or w^2 max(img, 0) (the
// propagated Poisson variance of the signal sum).
enum ValueMode { VM_PLAIN = 0, VM_DARK = 1, VM_VAR = 2 };
constexpr uint32_t kFrStageHeader = 128;  // per plane stage: nimg, group, G plane offsets

struct FrArgs {
    const char *img;                      // first frame of this launch
    int n_frames, n_groups, n_tiles;      // frames in the launch, groups of G, active tiles
    const int32_t *tile_desc, *tile_rec;  // per active tile: descriptor [8] and record
    const uint16_t *ent_loc;
    const float *ent_w, *ent_dark;        // ent_dark: NULL without a dark
    float *partial;                       // [n_frames][nseg]
    int nseg, ny, nx, th, tw, srow, ss, ntx;
    int *status;
    int var;                              // sum w^2 max(img, 0) instead of w img
    int pair;                             // frame-pair layout (8 frames per stage, whole stages)
    int slot;                             // its offset of frame F + 4 from frame F (words)
};

struct FrGeom {
    uint32_t rec_cap;       // bytes for the tile record (multiple of 128)
    uint32_t ent_cap;       // entry capacity (multiple of 8)
    uint32_t ebuf_bytes;    // one entry buffer (multiple of 128)
    int nebufs;             // entry buffers in the ring (2 .. kFrMaxEbufs)
    uint32_t plane_words;   // words per plane (frame-pair layout: per region of two frames)
    uint32_t band_from;     // first word of a plane's zero band
    uint32_t pstage_bytes;  // one plane stage: G planes (G / 2 regions)
    int nstages;            // plane stages
    int dk;                 // entries carry a dark
};

__device__ __forceinline__ TileDesc fr_desc(const FrArgs &a, int item) {
    const int4 *p = reinterpret_cast<const int4 *>(a.tile_desc) + 2 * (size_t)item;
    const int4 x = __ldg(p), y = __ldg(p + 1);
    return TileDesc{x.x, x.y, x.z, x.w, y.x, y.y};
}

// One thread: the tile's record, entry locations, weights and darks into entry buffer `eb`.
__device__ __forceinline__ void fr_stage_entries(const FrArgs &a, const FrGeom &fg, const TileDesc &td,
                                                 unsigned char *eb, uint64_t *bar) {
    const uint32_t ne = (uint32_t)td.ne;
    const uint32_t bytes = (uint32_t)td.rec_words * 4u + ne * (fg.dk ? 10u : 6u);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(eb, a.tile_rec + td.rec_off, (uint32_t)td.rec_words * 4u, bar);
    if (ne) {
        unsigned char *el = eb + fg.rec_cap;
        unsigned char *ew = el + fg.ent_cap * 2u;
        bulk_g2s(el, a.ent_loc + td.e_off, ne * 2u, bar);
        bulk_g2s(ew, a.ent_w + td.e_off, ne * 4u, bar);
        if (fg.dk) bulk_g2s(ew + fg.ent_cap * 4u, a.ent_dark + td.e_off, ne * 4u, bar);
    }
}

// The producer warp in the frame-pair layout (a whole stage of 8 frames): frames q and q + 4
// (q < 4) share region q of the stage, and one 3D tensor copy per (q, row class) moves that
// class of both frames -- periods m and m + 1 of the pair maps, m = (f0 + q) / 4 -- so a
// stage takes 16 copies.  Frame q's box starts 4 s_q words early as in fr_stage_planes (s_q =
// (q / P) mod 4 for the phase period P of the first four frames); frame q + 4, whose rows are
// 4 ny rows later, has frame q's word phase and shift, and its plane is a.slot words after
// frame q's.  Lane 0 then publishes the stage header and resets the stage's claim counter.
__device__ __forceinline__ void fr_stage_pairs(const FrArgs &a, const TmaSet &tm, const TileDesc &td, int g,
                                               uint32_t *planes, int *hdr, const FrGeom &fg, uint64_t *bar,
                                               int *ctr) {
    const int lane = threadIdx.x & 31;
    const int f0 = g * 8;
    if (a.n_frames - f0 < 8) {
        // a partial stage (the host launches whole stages only): no frames, an error status
        if (lane == 0) {
            atomicExch(a.status, AZ_EINVAL);
            hdr[0] = 0;
            hdr[1] = g;
            *ctr = 0;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(bar);
        return;
    }
    const int ti = td.t / a.ntx, tj = td.t - ti * a.ntx;
    const int r0 = ti * a.th, c0 = tj * a.tw;
    const int nu = a.nx & 3;
    const int rows4 = a.th >> 2;
    const uint32_t pw = fg.plane_words;
    const int beta = (int)((reinterpret_cast<uintptr_t>(a.img) >> 2) & 3u);
    const int c = (nu * (a.ny & 3)) & 3;
    const int lp = c == 0 ? 0 : (c == 2 ? 1 : 2);  // log2 of the phase period P
    const int q = (lane >> 2) & 3, k = lane & 3;     // lanes 0..15: (frame q, class k)
    const int phi_row = (int)(((int64_t)(f0 + q) * a.ny + r0) & 3);
    const int phi = (beta + nu * phi_row) & 3;
    const int sq = (q >> lp) & 3;
    fence_proxy_async_smem();
    if (lane == 0)
        asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
                     "r"((uint32_t)(16 * a.srow * rows4 * 2 * 4))
                     : "memory");
    __syncwarp();
    if (lane < 16) {
        const int sl = (k - phi_row) & 3;
        const int offk = (beta + k * nu) & 3;
        const int flag = (((nu * sl) & 3) + phi - offk) >> 2;
        const int x = c0 - 4 * (flag + sq);
        const int y = (q * a.ny + r0 + sl - k) >> 2;  // class row within the period (exact)
        const int m = (f0 + q) >> 2;
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(planes + (size_t)q * pw + (size_t)sl * a.ss)),
            "l"(reinterpret_cast<uint64_t>(&tm.pair[k])), "r"(x), "r"(y), "r"(m), "r"(smem_addr(bar))
            : "memory");
    }
    if (lane < 8) {
        const int qa = lane & 3;
        const int pha = (beta + nu * (int)(((int64_t)(f0 + qa) * a.ny + r0) & 3)) & 3;
        hdr[2 + lane] = (int)(qa * pw) + (lane >> 2) * a.slot + pha + 4 * ((qa >> lp) & 3);
    }
    if (lane == 0) {
        hdr[0] = 8;
        hdr[1] = g;
        *ctr = 0;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);  // publishes the header and the counter
}

// The producer warp: frames f0 .. f0 + nimg - 1 of the tile into plane stage `planes`, one
// tensor copy per (frame, row class), as in produce(); G <= 16, so a lane has at most two
// copies.  Frame q's box starts 4 * s_q words early, s_q = (number of earlier frames of the
// group whose rows have the same word phase) mod 4, so that the frames of a group fall on
// different shared-memory banks for as many frames as the phases and shifts allow.  Lane 0
// then publishes the stage header and resets the stage's claim counter.
template <int G>
__device__ __forceinline__ void fr_stage_planes(const FrArgs &a, const TmaSet &tm, const TileDesc &td,
                                                int g, uint32_t *planes, int *hdr, const FrGeom &fg,
                                                uint64_t *bar, int *ctr) {
    static_assert(G >= 1 && G <= 16, "a plane stage holds at most 16 frames");
    if constexpr (G == 8) {
        if (a.pair) {
            fr_stage_pairs(a, tm, td, g, planes, hdr, fg, bar, ctr);
            return;
        }
    }
    const int lane = threadIdx.x & 31;
    const int ti = td.t / a.ntx, tj = td.t - ti * a.ntx;
    const int r0 = ti * a.th, c0 = tj * a.tw;
    const int f0 = g * G;
    const int nimg = min(G, a.n_frames - f0);
    const int nu = a.nx & 3;
    const int rows4 = a.th >> 2;
    const int64_t rows_total = (int64_t)a.n_frames * a.ny;
    const uint32_t pw = fg.plane_words;
    const int beta = (int)((reinterpret_cast<uintptr_t>(a.img) >> 2) & 3u);
    // lane q < nimg: word phase of frame q's tile rows and its shift (earlier frames of the
    // group with the same phase, mod 4)
    const int64_t gl = (int64_t)(f0 + lane) * a.ny + r0;
    const int ph = (beta + nu * (int)(gl & 3)) & 3;
    const unsigned same = __match_any_sync(0xffffffffu, lane < nimg ? ph : 4 + lane);
    const int sh = __popc(same & ((1u << lane) - 1u)) & 3;
    // a lane's jobs are (frame, class) = (lane / 4, lane % 4) and (8 + lane / 4, lane % 4)
    const int shj[2] = {__shfl_sync(0xffffffffu, sh, lane >> 2), __shfl_sync(0xffffffffu, sh, 8 + (lane >> 2))};
    uint32_t mine = 0;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        const int job = lane + 32 * h2;
        if (job >= 4 * nimg) break;
        const int q = job >> 2, k = job & 3;
        const int64_t g0 = (int64_t)(f0 + q) * a.ny + r0;
        const int sl = (k - (int)(g0 & 3)) & 3;
        if (g0 + sl < rows_total) mine += (uint32_t)(a.srow * rows4 * 4);
    }
    fence_proxy_async_smem();
    if (mine)
        asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
                     "r"(mine)
                     : "memory");
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        const int job = lane + 32 * h2;
        if (job >= 4 * nimg) break;
        const int q = job >> 2, k = job & 3;
        const int64_t g0 = (int64_t)(f0 + q) * a.ny + r0;
        const int phi_row = (int)(g0 & 3);
        const int sl = (k - phi_row) & 3;
        if (g0 + sl >= rows_total) continue;
        const int phi = (beta + nu * phi_row) & 3;
        const int offk = (beta + k * nu) & 3;
        const int cs = (nu * sl) & 3;
        const int flag = (cs + phi - offk) >> 2;
        const int x = c0 - 4 * (flag + shj[h2]);
        uint32_t *dst = planes + (size_t)q * pw + (size_t)sl * a.ss;
        const int y = (int)((g0 + sl - k) >> 2);
        const CUtensorMap *map = &tm.m[0][k];
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
            "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
            : "memory");
    }
    if (lane < nimg) hdr[2 + lane] = (int)(lane * pw) + ph + 4 * sh;
    if (lane == 0) {
        hdr[0] = nimg;
        hdr[1] = g;
        *ctr = 0;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);  // publishes the header and the counter
}

// Load of a 4-byte word of shared memory at a 32-bit shared-window address (the gathers of
// the consumers index the staged planes with 32-bit arithmetic).
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Two FP32 values in one 64-bit register, operated on by the packed f32x2 instructions
// (round to nearest, no flush): each half gives exactly the scalar result.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 x, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// Two Kahan accumulators stepped together: the same operations as kahan_add on each half.
__device__ __forceinline__ void kahan2_add(f32x2 &s, f32x2 &nc, f32x2 w, f32x2 v) {
    const f32x2 y = f2_fma(w, v, nc);
    const f32x2 t = f2_add(s, y);
    nc = f2_sub(y, f2_sub(t, s));
    s = t;
}

// Consumer warps: lane (sub, q) reduces segment b + sub for frame q of the stage, with the
// entry stream of the tile's entry buffer, exactly as consume_serial does in frames mode (same
// entry order, accumulator assignment and merge); accumulators (0, 1) and (2, 3) are stepped
// as packed f32x2 pairs.
template <int G, int DT, int VM>
__device__ __forceinline__ void fr_consume(const FrArgs &a, const FrGeom &fg, const unsigned char *eb,
                                           const uint32_t *planes, const int *hdr, int *ctr) {
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, q = lane % G;
    const int *rec = reinterpret_cast<const int *>(eb);
    const int ns = rec[1];
    const int *slots = rec + 4;
    const uint16_t *starts = reinterpret_cast<const uint16_t *>(slots + ns);
    const uint16_t *L = reinterpret_cast<const uint16_t *>(eb + fg.rec_cap);
    const float *W = reinterpret_cast<const float *>(eb + fg.rec_cap + fg.ent_cap * 2u);
    const float *D = W + fg.ent_cap;
    const int nimg = hdr[0], g = hdr[1];
    const bool active = q < nimg;
    const uint32_t P = smem_addr(planes + hdr[2 + (active ? q : 0)]);
    float *out = a.partial + (size_t)(g * G + q) * (size_t)a.nseg;
    while (true) {
        int b = 0;
        if (lane == 0) b = atomicAdd(ctr, R);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= ns) break;
        const int sl = b + sub;
        int e0 = 0, e1 = 0, slot = 0;
        if (sl < ns) {
            e0 = starts[sl];
            e1 = starts[sl + 1];
            slot = slots[sl];
        }
        if (!active) e1 = e0;
        // Segments start on a quad and hold whole quads (padding entries add w = 0 times 0).
        f32x2 s01 = 0ull, n01 = 0ull, s23 = 0ull, n23 = 0ull;
        for (int qd = e0; qd < e1; qd += 4) {
            const uint2 l2 = *reinterpret_cast<const uint2 *>(L + qd);
            const float4 w4 = *reinterpret_cast<const float4 *>(W + qd);
            float v[4];
            v[0] = img_f32<DT>(lds_u32(P + ((l2.x & 0xffffu) << 2)));
            v[1] = img_f32<DT>(lds_u32(P + ((l2.x >> 16) << 2)));
            v[2] = img_f32<DT>(lds_u32(P + ((l2.y & 0xffffu) << 2)));
            v[3] = img_f32<DT>(lds_u32(P + ((l2.y >> 16) << 2)));
            if (VM == VM_VAR) {
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = fmaxf(v[j], 0.f);
            }
            f32x2 v01 = f2_pack(v[0], v[1]), v23 = f2_pack(v[2], v[3]);
            if (VM == VM_DARK) {
                const float4 d4 = *reinterpret_cast<const float4 *>(D + qd);
                v01 = f2_sub(v01, f2_pack(d4.x, d4.y));
                v23 = f2_sub(v23, f2_pack(d4.z, d4.w));
            }
            f32x2 w01 = f2_pack(w4.x, w4.y), w23 = f2_pack(w4.z, w4.w);
            if (VM == VM_VAR) {
                w01 = f2_mul(w01, w01);
                w23 = f2_mul(w23, w23);
            }
            kahan2_add(s01, n01, w01, v01);
            kahan2_add(s23, n23, w23, v23);
        }
        Kahan k[4];
        f2_unpack(s01, k[0].s, k[1].s);
        f2_unpack(n01, k[0].nc, k[1].nc);
        f2_unpack(s23, k[2].s, k[3].s);
        f2_unpack(n23, k[2].nc, k[3].nc);
        kahan_merge(k[0], k[1]);
        kahan_merge(k[2], k[3]);
        kahan_merge(k[0], k[2]);
        if (sl < ns && active) out[slot] = kahan_value(k[0]);
    }
}

// One or two frames per stage: a warp would take 32 or 16 segments at once and run each
// segment's whole entry stream on one lane, while a tile has only some tens of segments.  Here
// four lanes share a (segment, frame): lane j keeps accumulator j (the entries e = j mod 4 of
// every quad, in order, exactly as one lane of fr_consume steps its accumulator j), and the
// four are merged by shuffles as ((a0 + a1) + (a2 + a3)), the merge of fr_consume.  Same
// operations on the same values, so the same bits, with a quarter of the chain per lane and
// 8 / G segments per claim.
template <int G, int DT, int VM>
__device__ __forceinline__ void fr_consume_split(const FrArgs &a, const FrGeom &fg, const unsigned char *eb,
                                                 const uint32_t *planes, const int *hdr, int *ctr) {
    static_assert(G == 1 || G == 2, "split consumer is for one or two frames per stage");
    constexpr int R = 8 / G;
    const int lane = threadIdx.x & 31;
    const int j = lane & 3, q = (lane >> 2) % G, sub = lane / (4 * G);
    const int *rec = reinterpret_cast<const int *>(eb);
    const int ns = rec[1];
    const int *slots = rec + 4;
    const uint16_t *starts = reinterpret_cast<const uint16_t *>(slots + ns);
    const uint16_t *L = reinterpret_cast<const uint16_t *>(eb + fg.rec_cap);
    const float *W = reinterpret_cast<const float *>(eb + fg.rec_cap + fg.ent_cap * 2u);
    const float *D = W + fg.ent_cap;
    const int nimg = hdr[0], g = hdr[1];
    const bool active = q < nimg;
    const uint32_t P = smem_addr(planes + hdr[2 + (active ? q : 0)]);
    float *out = a.partial + (size_t)(g * G + q) * (size_t)a.nseg;
    while (true) {
        int b = 0;
        if (lane == 0) b = atomicAdd(ctr, R);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= ns) break;
        const int sl = b + sub;
        int e0 = 0, e1 = 0, slot = 0;
        if (sl < ns) {
            e0 = starts[sl];
            e1 = starts[sl + 1];
            slot = slots[sl];
        }
        if (!active) e1 = e0;
        Kahan k{0.f, 0.f};
        for (int e = e0 + j; e < e1; e += 4) {
            float v = img_f32<DT>(lds_u32(P + ((uint32_t)L[e] << 2)));
            float w = W[e];
            if (VM == VM_VAR) {
                v = fmaxf(v, 0.f);
                w = __fmul_rn(w, w);
            }
            if (VM == VM_DARK) v = __fsub_rn(v, D[e]);
            kahan_add(k, w, v);
        }
        // lanes j = 0, 2 take (a0 + a1), (a2 + a3); lane 0 then adds the second to the first
        Kahan o = shfl_xor(k, 1);
        kahan_merge(k, o);
        o = shfl_xor(k, 2);
        kahan_merge(k, o);
        if (j == 0 && sl < ns && active) out[slot] = kahan_value(k);
    }
}

// Bounded grace wait for copies this CTA issued before giving up (every wait is bounded).
__device__ __forceinline__ void fr_drain(uint64_t *bar, uint32_t parity) { (void)mbar_wait_bounded(bar, parity); }

template <int G, int DT, int VM>
__global__ void __launch_bounds__(kFrThreads, 1)
frames_kernel(const __grid_constant__ FrArgs a, FrGeom fg, const __grid_constant__ TmaSet tm) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127u) & ~static_cast<uintptr_t>(127u));
    const int S = fg.nstages;
    unsigned char *ebuf0 = smem;
    const int NE = fg.nebufs;
    unsigned char *pst = smem + (size_t)NE * fg.ebuf_bytes;
    int *hdrs = reinterpret_cast<int *>(pst + (size_t)S * fg.pstage_bytes);
    uint64_t *efull = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(hdrs) +
                                                   (size_t)S * kFrStageHeader);
    uint64_t *eempty = efull + NE;
    uint64_t *pfull = eempty + NE;
    uint64_t *pempty = pfull + S;
    int *ctr = reinterpret_cast<int *>(pempty + S);
    volatile int *abort_flag = ctr + S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NE; ++i) {
            mbar_init(&efull[i], 1);
            mbar_init(&eempty[i], kFrConsumers);
        }
        for (int i = 0; i < S; ++i) {
            mbar_init(&pfull[i], 1);
            mbar_init(&pempty[i], kFrConsumers);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    zero_bands(pst, fg.pstage_bytes, S, (int)(fg.pstage_bytes / (fg.plane_words * 4u)), fg.plane_words,
               fg.band_from);
    __syncthreads();
    if (warp == 0) {
        int k = 0, issued = 0;  // items seen, items whose entries were issued
        uint32_t j = 0;         // plane stages issued
        bool stop = false;
        // descriptors are read two items ahead: with one or two frame groups per item the
        // producer would otherwise wait for a descriptor from DRAM on every item
        TileDesc ahead[2] = {};
        for (int u = 0; u < 2; ++u)
            if (blockIdx.x + u * gridDim.x < (unsigned)a.n_tiles) ahead[u] = fr_desc(a, blockIdx.x + u * gridDim.x);
        for (int item = blockIdx.x; item < a.n_tiles && !stop; item += gridDim.x, ++k) {
            const TileDesc td = ahead[0];
            ahead[0] = ahead[1];
            const int64_t far = (int64_t)item + 2 * (int64_t)gridDim.x;
            if (far < a.n_tiles) ahead[1] = fr_desc(a, (int)far);
            const int eb = k % NE;
            bool ok = true;
            if (k >= NE) ok = mbar_wait_bounded(&eempty[eb], (uint32_t)(((k / NE) - 1) & 1));
            ok = __all_sync(0xffffffffu, ok);
            if (!ok || *abort_flag != 0) { stop = true; if (!ok && lane == 0) atomicExch(a.status, AZ_ETIMEOUT); break; }
            if (lane == 0) fr_stage_entries(a, fg, td, ebuf0 + (size_t)eb * fg.ebuf_bytes, &efull[eb]);
            issued = k + 1;
            for (int g = 0; g < a.n_groups; ++g, ++j) {
                const int s = (int)(j % (uint32_t)S);
                ok = true;
                if (j >= (uint32_t)S) ok = mbar_wait_bounded(&pempty[s], ((j / S) - 1) & 1);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok || *abort_flag != 0) { stop = true; if (!ok && lane == 0) atomicExch(a.status, AZ_ETIMEOUT); break; }
                fr_stage_planes<G>(a, tm, td, g, reinterpret_cast<uint32_t *>(pst + (size_t)s * fg.pstage_bytes),
                                   hdrs + s * (kFrStageHeader / 4), fg, &pfull[s], &ctr[s]);
            }
        }
        if (stop && lane == 0) {
            *abort_flag = 1;
            // grace for this CTA's own copies still in flight
            for (uint32_t jj = j > (uint32_t)S ? j - S : 0; jj < j; ++jj) fr_drain(&pfull[jj % S], (jj / S) & 1);
            for (int kk = issued > NE ? issued - NE : 0; kk < issued; ++kk)
                fr_drain(&efull[kk % NE], (uint32_t)((kk / NE) & 1));
        }
    } else {
        int k = 0;
        uint32_t j = 0;
        bool stop = false;
        for (int item = blockIdx.x; item < a.n_tiles && !stop; item += gridDim.x, ++k) {
            const int eb = k % NE;
            bool ok = mbar_wait_bounded(&efull[eb], (uint32_t)((k / NE) & 1));
            ok = __all_sync(0xffffffffu, ok);
            if (!ok || *abort_flag != 0) {
                if (!ok && lane == 0) { atomicExch(a.status, AZ_ETIMEOUT); *abort_flag = 1; }
                break;
            }
            const unsigned char *ebp = ebuf0 + (size_t)eb * fg.ebuf_bytes;
            for (int g = 0; g < a.n_groups; ++g, ++j) {
                const int s = (int)(j % (uint32_t)S);
                ok = mbar_wait_bounded(&pfull[s], (j / S) & 1);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok || *abort_flag != 0) {
                    if (!ok && lane == 0) { atomicExch(a.status, AZ_ETIMEOUT); *abort_flag = 1; }
                    stop = true;
                    break;
                }
                const uint32_t *pl = reinterpret_cast<const uint32_t *>(pst + (size_t)s * fg.pstage_bytes);
                if constexpr (G <= 2)
                    fr_consume_split<G, DT, VM>(a, fg, ebp, pl, hdrs + s * (kFrStageHeader / 4), &ctr[s]);
                else
                    fr_consume<G, DT, VM>(a, fg, ebp, pl, hdrs + s * (kFrStageHeader / 4), &ctr[s]);
                __syncwarp();
                if (lane == 0) mbar_arrive(&pempty[s]);
            }
            if (stop) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&eempty[eb]);
        }
    }
}

// ------------------------------------------------------------------------------------
// phase 2: per-row sums of the partials in a fixed order
// ------------------------------------------------------------------------------------
template <class AT>
__device__ __forceinline__ AT row_sum(const AT *p, int a, int b) {
    const int lane = threadIdx.x & 31;
    Acc<AT> acc;
    acc.zero();
    for (int s = a + lane; s < b; s += 32) acc.add(AT(1), p[s]);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) acc.merge_xor(m);
    return acc.value();
}

__device__ __forceinline__ const Inst &inst_of_row(const Inst &single, const Inst *multi,
                                                   int n_inst, int64_t row) {
    if (!multi) return single;
    int lo = 0, hi = n_inst;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (multi[mid].row_begin <= row) lo = mid; else hi = mid;
    }
    return multi[lo];
}

// The value row_sum<float> computes, formed by one thread: the 32 lanes' strided Kahan sums
// and the same lower-lane-left merge tree, each virtual lane's sum kept in registers.  For
// rows with few slots (2D patterns: ~1-2 segments per row) this replaces a warp per row and
// frame by a thread; the bits are the same.
__device__ __forceinline__ Kahan kahan_one(float v) {
    Kahan k{0.f, 0.f};
    kahan_add(k, 1.f, v);
    return k;
}

__device__ __forceinline__ float row_sum_thread(const float *p, int a, int b) {
    // Up to four slots: the tree's only non-trivial merges (a merge with an empty lane's
    // {+0, +0} changes no bit), in the tree's order.
    const int n = b - a;
    if (n <= 0) return 0.f;
    if (n == 1) return kahan_value(kahan_one(p[a]));
    if (n <= 4) {
        Kahan x0 = kahan_one(p[a]), x1 = kahan_one(p[a + 1]);
        if (n == 2) {
            kahan_merge(x0, x1);
            return kahan_value(x0);
        }
        kahan_merge(x0, kahan_one(p[a + 2]));       // lanes 0 and 2 at the pairs-of-two level
        if (n == 4) kahan_merge(x1, kahan_one(p[a + 3]));
        kahan_merge(x0, x1);
        return kahan_value(x0);
    }
    Kahan v[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) {
        v[l].s = 0.f;
        v[l].nc = 0.f;
        for (int s = a + l; s < b; s += 32) kahan_add(v[l], 1.f, p[s]);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1)
#pragma unroll
        for (int l = 0; l < m; ++l) kahan_merge(v[l], v[l + m]);
    return kahan_value(v[0]);
}

// Frames-mode phase 2 with one thread per (row, frame), for rows of few slots.
__global__ void phase2_frames_thread_kernel(const __grid_constant__ Inst d, int64_t n_jobs) {
    for (int64_t job = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; job < n_jobs;
         job += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(job / d.nrows), r = (int)(job - (int64_t)f * d.nrows);
        const int a = d.row_slot_ptr[r], b = d.row_slot_ptr[r + 1];
        const float S = row_sum_thread(static_cast<const float *>(d.partial) + (size_t)f * d.nseg, a, b);
        const float N = d.norm[r];
        const size_t o = (size_t)(d.frame_out0 + f) * d.nrows + r;
        if (d.oS) static_cast<float *>(d.oS)[o] = S;
        if (d.oI) static_cast<float *>(d.oI)[o] = N != 0.f ? __fdiv_rn(S, N) : 0.f;
    }
}

template <class AT, int MODE>
__global__ void phase2_kernel(const __grid_constant__ Inst single, const Inst *__restrict__ multi,
                              int n_inst, int64_t n_jobs, int n_frames) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t job = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); job < n_jobs;
         job += nw) {
        if (MODE == MODE_FRAMES) {
            // job = frame * nrows + row (single instance)
            const Inst &d = single;
            const int f = (int)(job / d.nrows), r = (int)(job - (int64_t)f * d.nrows);
            const int a = d.row_slot_ptr[r], b = d.row_slot_ptr[r + 1];
            const AT S = row_sum<AT>(static_cast<const AT *>(d.partial) + (size_t)f * d.nseg, a, b);
            if (lane == 0) {
                const float N = d.norm[r];
                const size_t o = (size_t)(d.frame_out0 + f) * d.nrows + r;
                if (d.oS) static_cast<float *>(d.oS)[o] = (float)S;
                if (d.oI) static_cast<float *>(d.oI)[o] = N != 0.f ? __fdiv_rn((float)S, N) : 0.f;
            }
        } else {
            const Inst &d = inst_of_row(single, multi, n_inst, job);
            const int r = (int)(job - d.row_begin);
            const int a = d.row_slot_ptr[r], b = d.row_slot_ptr[r + 1];
            const AT *P = static_cast<const AT *>(d.partial);
            if (MODE == MODE_SINGLE) {
                const AT S = row_sum<AT>(P, a, b);
                const AT N = d.single_nc == 2 ? (AT)d.norm[d.nrows + r] : row_sum<AT>(P + d.nseg, a, b);
                const AT C = d.single_nc ? (AT)d.norm[d.nrows + r] : row_sum<AT>(P + 2 * (size_t)d.nseg, a, b);
                if (lane == 0) {
                    const AT I = N != AT(0) ? S / N : AT(0);
                    if (d.oI) static_cast<AT *>(d.oI)[r] = I;
                    if (d.oS) static_cast<AT *>(d.oS)[r] = S;
                    if (d.oN) static_cast<AT *>(d.oN)[r] = N;
                    if (d.oC) static_cast<AT *>(d.oC)[r] = C;
                }
            } else {
                const AT N = row_sum<AT>(P, a, b);
                const AT C = d.norm_rows == 2 ? row_sum<AT>(P + d.nseg, a, b) : AT(0);
                if (lane == 0) {
                    d.norm[r] = (float)N;
                    if (d.oN) static_cast<float *>(d.oN)[r] = (float)N;
                    if (d.norm_rows == 2) {
                        d.norm[d.nrows + r] = (float)C;
                        if (d.oC) static_cast<float *>(d.oC)[r] = (float)C;
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
int g_num_sms = 0;
int g_max_smem = 0;

// Stage dimensions: plane slots of `plane_words` words, `planes` of them, plus (when the
// entries are staged) room for `ent_cap` entries of (uint16 loc, wbytes weight).
constexpr uint32_t kBarrierBytes = 256 + 128;  // barriers, counters, abort flag; alignment slack

StageGeom stage_geom(uint32_t plane_words, int planes, uint32_t ent_cap, int wbytes, uint32_t rec_words,
                     int ent_dk = 0) {
    StageGeom sg;
    sg.plane_words = plane_words;
    sg.plane_region = (uint32_t)planes * plane_words * 4u;
    sg.ent_cap = ent_cap;
    sg.ent_dk = ent_dk;
    sg.rec_cap = (rec_words * 4u + 127u) & ~127u;  // keeps the plane region 128-byte aligned
    uint32_t bytes = kHeaderBytes + sg.rec_cap + sg.plane_region +
                     ent_cap * (2u + (uint32_t)wbytes + (ent_dk ? 4u : 0u));
    sg.stage_bytes = (bytes + 127u) & ~127u;
    // as many stages as fit (at least two, at most kMaxStages)
    const int avail = max_smem_per_block() - (int)kBarrierBytes;
    sg.nstages = std::min(kMaxStages, std::max(2, avail / (int)sg.stage_bytes));
    return sg;
}

uint32_t smem_for(const StageGeom &sg) { return (uint32_t)sg.nstages * sg.stage_bytes + kBarrierBytes; }

// Stage the entries when the largest tile fits twice next to the planes; otherwise the
// reduction reads the entries from global memory.
StageGeom choose_stage(uint32_t plane_words, int planes, uint32_t max_entries, int wbytes,
                       uint32_t rec_words, int &stage_entries, int ent_dk = 0) {
    StageGeom sg = stage_geom(plane_words, planes, max_entries, wbytes, rec_words, ent_dk);
    if ((int)smem_for(sg) <= max_smem_per_block()) {
        stage_entries = 1;
        return sg;
    }
    stage_entries = 0;
    return stage_geom(plane_words, planes, 0, wbytes, rec_words, ent_dk);
}

Inst make_inst(const az_integrator *h, bool fp64) {
    Inst d{};
    const TiledLayout &L = h->tl;
    d.tile_seg_ptr = L.tile_seg_ptr.as<int32_t>();
    d.tile_ent_ptr = L.tile_ent_ptr.as<int32_t>();
    d.active_tiles = L.active_tiles.as<int32_t>();
    d.seg_start = L.seg_ent_ptr.as<int32_t>();
    d.seg_end = L.seg_ent_ptr.as<int32_t>() + L.nseg;
    d.seg_slot = L.seg_slot.as<int32_t>();
    d.row_slot_ptr = L.row_slot_ptr.as<int32_t>();
    d.ent_loc = L.ent_loc.as<uint16_t>();
    d.ent_w = fp64 ? (const void *)L.ent_w64.p : (const void *)L.ent_w32.p;
    d.ny = h->ny; d.nx = h->nx; d.th = L.th; d.tw = L.tw; d.srow = L.srow; d.ss = L.ss; d.ntx = L.ntx;
    d.rpw = 32 / h->frames_per_pass; d.nseg = L.nseg; d.nrows = h->nrows;
    d.npix = (int64_t)h->ny * h->nx;
    d.n_frames = 1; d.fpi = 1; d.n_groups = 1;
    d.norm_rows = 2;
    d.partial = h->partial.p;
    d.norm = h->norm.as<float>();
    d.status = h->status.as<int>();
    d.n_items = L.n_active;
    d.tile_desc = L.tile_desc.as<int32_t>();
    d.tile_rec = L.tile_rec.as<int32_t>();
    return d;
}

template <class AT, class WT, int MODE, int NIMG, int DT, bool TMA>
int run_phase1(const Inst &single, const Inst *multi, int n_inst, int64_t n_items,
               const StageGeom &sg, const TmaSet &tm, cudaStream_t s, Profiler *prof = nullptr) {
    if (n_items <= 0) return AZ_OK;
    const uint32_t smem = smem_for(sg);
    if ((int)smem > max_smem_per_block())
        return fail(AZ_EUNSUPPORTED, "forward: %u bytes of shared memory needed (%d available)",
                    smem, max_smem_per_block());
    auto kern = phase1_kernel<AT, WT, MODE, NIMG, DT, TMA>;
    AZ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    AZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::min<int64_t>(n_items, (int64_t)num_sms() * per_sm);
    {
        ProfScope ps(prof, MODE == MODE_FRAMES ? 0 : (MODE == MODE_NORM ? 1 : 2), s);
        kern<<<(unsigned)grid, kThreads, smem, s>>>(single, multi, n_inst, n_items, sg, tm);
    }
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}

template <class AT, int MODE>
int run_phase2(const Inst &single, const Inst *multi, int n_inst, int64_t n_jobs, int n_frames,
               cudaStream_t s, Profiler *prof = nullptr) {
    if (n_jobs <= 0) return AZ_OK;
    if (MODE == MODE_FRAMES && sizeof(AT) == 4 && !multi && (int64_t)single.nseg <= 8 * (int64_t)single.nrows) {
        // few slots per row: a thread per (row, frame)
        const int64_t blocks = std::min<int64_t>((n_jobs + 255) / 256, (int64_t)num_sms() * 16);
        ProfScope ps(prof, 3, s);
        phase2_frames_thread_kernel<<<(unsigned)blocks, 256, 0, s>>>(single, n_jobs);
        AZ_CUDA(cudaGetLastError());
        return AZ_OK;
    }
    const int warps_per_block = 8;
    int64_t blocks = (n_jobs + warps_per_block - 1) / warps_per_block;
    blocks = std::min<int64_t>(blocks, (int64_t)num_sms() * 16);
    {
        ProfScope ps(prof, 3, s);
        phase2_kernel<AT, MODE><<<(unsigned)blocks, warps_per_block * 32, 0, s>>>(single, multi, n_inst,
                                                                               n_jobs, n_frames);
    }
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}

template <class AT, class WT, int MODE, int NIMG, int DT>
int run_phase1_eng(int engine, const Inst &single, const Inst *multi, int n_inst, int64_t n_items,
                   const StageGeom &sg, const TmaSet &tm, cudaStream_t s, Profiler *prof) {
    if (engine == AZ_COPY_ASYNC)
        return run_phase1<AT, WT, MODE, NIMG, DT, false>(single, multi, n_inst, n_items, sg, tm, s, prof);
    return run_phase1<AT, WT, MODE, NIMG, DT, true>(single, multi, n_inst, n_items, sg, tm, s, prof);
}

template <class AT, class WT, int MODE, int NIMG>
int run_phase1_dt(int dtype, int engine, const Inst &single, const Inst *multi, int n_inst,
                  int64_t n_items, const StageGeom &sg, const TmaSet &tm, cudaStream_t s,
                  Profiler *prof = nullptr) {
    switch (dtype) {
        case AZ_DTYPE_F32:
            return run_phase1_eng<AT, WT, MODE, NIMG, AZ_DTYPE_F32>(engine, single, multi, n_inst, n_items, sg, tm, s, prof);
        case AZ_DTYPE_U32:
            return run_phase1_eng<AT, WT, MODE, NIMG, AZ_DTYPE_U32>(engine, single, multi, n_inst, n_items, sg, tm, s, prof);
        default:
            return run_phase1_eng<AT, WT, MODE, NIMG, AZ_DTYPE_I32>(engine, single, multi, n_inst, n_items, sg, tm, s, prof);
    }
}

// Dark of each tiled entry's pixel (0 for padding entries), gathered once per batch call.
__global__ void gather_dark_kernel(const int32_t *__restrict__ pix, const float *__restrict__ dark,
                                   int64_t n, float *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = pix[e];
        out[e] = p >= 0 ? dark[p] : 0.f;
    }
}

// ---- tensor maps for the TMA engine --------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int get_encoder() {
    if (g_encode) return AZ_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(AZ_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return AZ_OK;
}

// Four maps over `rows_total` rows of nx 4-byte words starting at `arr`: map k covers rows
// g = 4 y + k (16 * nx bytes apart) from the 16-byte aligned address just before row k, so
// that element (x, y) is column x - off_k of row g, off_k = (beta + k nx) mod 4.  Reads
// outside [0, nx + off_k) x [0, rows of class k) return zeros, so no copy reads past a row or
// the array.
int encode_class_maps(const void *arr, int64_t rows_total, int nx, int box_w, int box_h,
                      CUtensorMap out[4]) {
    AZ_TRY(get_encoder());
    const uintptr_t base = reinterpret_cast<uintptr_t>(arr);
    const int beta = (int)((base >> 2) & 3u), nu = nx & 3;
    for (int k = 0; k < 4; ++k) {
        const int offk = (beta + k * nu) & 3;
        const int64_t rows_k = rows_total > k ? (rows_total - k + 3) / 4 : 0;
        if (rows_k == 0) {
            memset(&out[k], 0, sizeof(CUtensorMap));  // never used: the producer skips the class
            continue;
        }
        void *basek = reinterpret_cast<void *>(base + 4u * (uintptr_t)k * (uintptr_t)nx - 4u * (uintptr_t)offk);
        cuuint64_t dims[2] = {(cuuint64_t)(nx + offk), (cuuint64_t)rows_k};
        cuuint64_t strides[1] = {(cuuint64_t)16 * (cuuint64_t)nx};
        cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = g_encode(&out[k], CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, basek, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(AZ_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    return AZ_OK;
}

// The engine a launch really uses: the TMA engine needs boxes of at most 256 words.
int engine_for(const az_integrator *h) {
    if (h->copy_engine == AZ_COPY_TMA && h->tl.srow <= 256) return AZ_COPY_TMA;
    return AZ_COPY_ASYNC;
}

// Maps for the arrays a launch stages (image rows_img rows from img; corrections ny rows).
int make_maps(const az_integrator *h, int engine, const void *img, int64_t rows_img, const float *dark,
              const float *flat, const float *sa, const float *pol, TmaSet &tm) {
    memset(&tm, 0, sizeof(tm));
    if (engine != AZ_COPY_TMA) return AZ_OK;
    const int bw = h->tl.srow, bh = h->tl.th / 4;
    const void *arrs[5] = {img, dark, flat, sa, pol};
    for (int i = 0; i < 5; ++i) {
        if (!arrs[i]) continue;
        AZ_TRY(encode_class_maps(arrs[i], i == 0 ? rows_img : h->ny, h->nx, bw, bh, tm.m[i]));
    }
    return AZ_OK;
}

uint32_t plane_words_of(const az_integrator *h) { return plane_stride(h->tl.ss); }
uint32_t rec_words_of(const az_integrator *h) { return (uint32_t)h->tl.max_rec_words; }

// ---- frames kernel with tile-resident entries -----------------------------------------
constexpr uint32_t kFrFixedBytes = 128 + 384;  // alignment slack; barriers, counters, flag

// The image's row-class maps for the frame-pair layout, in three dimensions: x, the ny class
// rows of a period of four frames (class k holds rows k, k + 4, ... of the stacked frames, so
// a period is 4 ny rows = ny class rows), and the period (16 npix bytes, a multiple of 16).
// Class k of frames F and F + 4 are the same class rows of consecutive periods, so a box of
// depth 2 copies both.  Only the nf / 4 whole periods of the nf frames are mapped.
int encode_pair_maps(const void *img, int nf, int ny, int nx, int box_w, int box_h, CUtensorMap out[4]) {
    AZ_TRY(get_encoder());
    const uintptr_t base = reinterpret_cast<uintptr_t>(img);
    const int beta = (int)((base >> 2) & 3u), nu = nx & 3;
    for (int k = 0; k < 4; ++k) {
        const int offk = (beta + k * nu) & 3;
        void *basek = reinterpret_cast<void *>(base + 4u * (uintptr_t)k * (uintptr_t)nx - 4u * (uintptr_t)offk);
        cuuint64_t dims[3] = {(cuuint64_t)(nx + offk), (cuuint64_t)ny, (cuuint64_t)(nf / 4)};
        cuuint64_t strides[2] = {(cuuint64_t)16 * (cuuint64_t)nx, (cuuint64_t)16 * (cuuint64_t)nx * (cuuint64_t)ny};
        cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 2};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = g_encode(&out[k], CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, basek, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(AZ_ECUDA, "cuTensorMapEncodeTiled (pairs) failed (%d)", (int)r);
    }
    return AZ_OK;
}

// Sizes for G frames per plane stage (pair: the frame-pair layout, G / 2 regions of two
// frames); false unless two entry buffers and two plane stages fit.
bool fr_geom(const az_integrator *h, int G, int dk, int n_groups, FrGeom &fg, bool pair = false) {
    fg.rec_cap = (rec_words_of(h) * 4u + 127u) & ~127u;
    fg.ent_cap = ((uint32_t)h->tl.max_tile_entries + 7u) & ~7u;
    fg.dk = dk;
    fg.ebuf_bytes = (fg.rec_cap + fg.ent_cap * (dk ? 10u : 6u) + 127u) & ~127u;
    if (pair) {
        fg.plane_words = (uint32_t)h->tl.pw_p;
        fg.band_from = 4u * (uint32_t)h->tl.ss_p;
        fg.pstage_bytes = (uint32_t)(G / 2) * fg.plane_words * 4u;
    } else {
        fg.plane_words = plane_words_of(h);
        fg.band_from = fg.plane_words - kZeroBand;
        fg.pstage_bytes = (uint32_t)G * fg.plane_words * 4u;
    }
    // two entry buffers and as many plane stages as fit; then, when a work item has few
    // frame groups (the entries dominate its copies), more entry buffers in what is left
    const int64_t per = (int64_t)fg.pstage_bytes + kFrStageHeader;
    const int64_t avail = (int64_t)max_smem_per_block() - 2 * (int64_t)fg.ebuf_bytes - kFrFixedBytes;
    fg.nstages = (int)std::min<int64_t>(kFrMaxStages, avail > 0 ? avail / per : 0);
    fg.nebufs = 2;
    if (n_groups <= 2 && fg.nstages >= 2) {
        // every item takes n_groups plane stages: grow both rings together, so that as many
        // items are in flight for their planes as for their entries
        for (int e = 2; e <= kFrMaxEbufs; ++e) {
            const int ns = std::min(kFrMaxStages, std::max(2, n_groups * e));
            const int64_t need = (int64_t)e * fg.ebuf_bytes + (int64_t)ns * per + kFrFixedBytes;
            if (need > (int64_t)max_smem_per_block()) break;
            fg.nebufs = e;
            fg.nstages = ns;
        }
    }
    return fg.nstages >= 2;
}

uint32_t fr_smem(const FrGeom &fg) {
    return (uint32_t)fg.nebufs * fg.ebuf_bytes + (uint32_t)fg.nstages * (fg.pstage_bytes + kFrStageHeader) +
           kFrFixedBytes;
}

template <int G, int DT, int VM>
int fr_launch(const FrArgs &a, const FrGeom &fg, const TmaSet &tm, cudaStream_t s, Profiler *prof,
              int prof_kind) {
    if (a.n_tiles <= 0) return AZ_OK;
    const uint32_t smem = fr_smem(fg);
    auto kern = frames_kernel<G, DT, VM>;
    AZ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = std::min(a.n_tiles, num_sms());
    {
        ProfScope ps(prof, prof_kind, s);
        kern<<<grid, kFrThreads, smem, s>>>(a, fg, tm);
    }
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}

template <int G>
int fr_launch_dt(int dtype, const FrArgs &a, const FrGeom &fg, const TmaSet &tm, cudaStream_t s,
                 Profiler *prof, int kind) {
    const int vm = a.var ? VM_VAR : (a.ent_dark != nullptr ? VM_DARK : VM_PLAIN);
    switch (dtype) {
        case AZ_DTYPE_F32:
            return vm == VM_DARK ? fr_launch<G, AZ_DTYPE_F32, VM_DARK>(a, fg, tm, s, prof, kind)
                 : vm == VM_VAR  ? fr_launch<G, AZ_DTYPE_F32, VM_VAR>(a, fg, tm, s, prof, kind)
                                 : fr_launch<G, AZ_DTYPE_F32, VM_PLAIN>(a, fg, tm, s, prof, kind);
        case AZ_DTYPE_U32:
            return vm == VM_DARK ? fr_launch<G, AZ_DTYPE_U32, VM_DARK>(a, fg, tm, s, prof, kind)
                 : vm == VM_VAR  ? fr_launch<G, AZ_DTYPE_U32, VM_VAR>(a, fg, tm, s, prof, kind)
                                 : fr_launch<G, AZ_DTYPE_U32, VM_PLAIN>(a, fg, tm, s, prof, kind);
        default:
            return vm == VM_DARK ? fr_launch<G, AZ_DTYPE_I32, VM_DARK>(a, fg, tm, s, prof, kind)
                 : vm == VM_VAR  ? fr_launch<G, AZ_DTYPE_I32, VM_VAR>(a, fg, tm, s, prof, kind)
                                 : fr_launch<G, AZ_DTYPE_I32, VM_PLAIN>(a, fg, tm, s, prof, kind);
    }
}

// Frames kernel over `nf` frames starting at `img` (nf <= the partial buffer's frames from
// frame0 on): per-segment partials [nf][nseg] in h->partial from frame frame0.  With 8 frames
// per stage, whole stages go through the frame-pair layout when the tile shape has one and
// its stages fit; the frames of a last partial stage then go through the plain layout in a
// second launch (a frame's sums do not depend on the layout it is read through: the entry
// order is the same).  Returns AZ_EUNSUPPORTED (without error text) when the TMA engine or
// the shared memory it needs is not available.
int frames_v3(az_integrator *h, const void *img, int nf, int dtype, const float *ent_dark,
              int prof_kind, cudaStream_t s, bool var = false, const float *ent_weights = nullptr,
              int frame0 = 0, bool allow_pair = true) {
    if (engine_for(h) != AZ_COPY_TMA) return AZ_EUNSUPPORTED;
    int G = h->frames_per_pass >= 16 ? 16 : (h->frames_per_pass >= 8 ? 8 : 4);
    FrGeom fg;
    // one frame (any image type, with or without a dark), or two frames of float values
    // without a dark (the norm pass): one lane per segment and frame
    const bool small = nf == 1 || (nf == 2 && dtype == AZ_DTYPE_F32 && ent_dark == nullptr && !var);
    if (small) G = nf;
    else if (nf < G) G = nf <= 4 ? 4 : (nf <= 8 ? 8 : G);
    bool fits = fr_geom(h, G, ent_dark != nullptr, (nf + G - 1) / G, fg);
    while (!fits && G > 4 && !small) {
        G >>= 1;
        fits = fr_geom(h, G, ent_dark != nullptr, (nf + G - 1) / G, fg);
    }
    if (!fits) return AZ_EUNSUPPORTED;
    const TiledLayout &L = h->tl;
    const int nf8 = nf & ~7;
    FrGeom fp;
    const bool pair = allow_pair && G == 8 && !small && L.srow_p > 0 && nf8 > 0 &&
                      fr_geom(h, 8, ent_dark != nullptr, nf8 / 8, fp, true);
    if (pair) fg = fp;
    const int nrun = pair ? nf8 : nf;
    FrArgs a{};
    a.img = static_cast<const char *>(img);
    a.n_frames = nrun; a.n_groups = (nrun + G - 1) / G; a.n_tiles = L.n_active;
    a.tile_desc = L.tile_desc.as<int32_t>(); a.tile_rec = L.tile_rec.as<int32_t>();
    a.ent_loc = pair ? L.ent_loc_p.as<uint16_t>() : L.ent_loc.as<uint16_t>();
    a.ent_w = ent_weights ? ent_weights : L.ent_w32.as<float>();
    a.ent_dark = ent_dark;
    a.var = var ? 1 : 0;
    a.partial = h->partial.as<float>() + (size_t)frame0 * (size_t)L.nseg;
    a.nseg = L.nseg; a.ny = h->ny; a.nx = h->nx; a.th = L.th; a.tw = L.tw;
    a.srow = pair ? L.srow_p : L.srow;
    a.ss = pair ? L.ss_p : L.ss;
    a.ntx = L.ntx;
    a.pair = pair ? 1 : 0;
    a.slot = L.slot_p;
    a.status = h->status.as<int>();
    TmaSet tm;
    if (pair) {
        memset(&tm, 0, sizeof(tm));
        AZ_TRY(encode_pair_maps(img, nrun, h->ny, h->nx, L.srow_p, L.th / 4, tm.pair));
        AZ_TRY(fr_launch_dt<8>(dtype, a, fg, tm, s, &h->prof, prof_kind));
        if (nrun == nf) return AZ_OK;
        return frames_v3(h, static_cast<const char *>(img) + (size_t)nrun * (size_t)h->ny * (size_t)h->nx * 4u,
                         nf - nrun, dtype, ent_dark, prof_kind, s, var, ent_weights, frame0 + nrun, false);
    }
    AZ_TRY(make_maps(h, AZ_COPY_TMA, img, (int64_t)nf * h->ny, nullptr, nullptr, nullptr, nullptr, tm));
    if (small)
        return G == 1 ? fr_launch_dt<1>(dtype, a, fg, tm, s, &h->prof, prof_kind)
                      : fr_launch<2, AZ_DTYPE_F32, VM_PLAIN>(a, fg, tm, s, &h->prof, prof_kind);
    switch (G) {
        case 4: return fr_launch_dt<4>(dtype, a, fg, tm, s, &h->prof, prof_kind);
        case 8: return fr_launch_dt<8>(dtype, a, fg, tm, s, &h->prof, prof_kind);
        default: return fr_launch_dt<16>(dtype, a, fg, tm, s, &h->prof, prof_kind);
    }
}

// flat * solid angle * polarisation per pixel, multiplied in that order from 1 (absent = 1):
// the value the norm reduction multiplies by each weight.
__global__ void norm_pixels_kernel(const float *__restrict__ flat, const float *__restrict__ sa,
                                   const float *__restrict__ pol, int64_t n, float *__restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        float v = 1.f;
        if (flat) v = __fmul_rn(v, flat[p]);
        if (sa) v = __fmul_rn(v, sa[p]);
        if (pol) v = __fmul_rn(v, pol[p]);
        out[p] = v;
    }
}

// Weight of each entry divided by its pixel's flat * solid angle * polarisation (0 for
// padding entries): the weights of the per-pixel-corrected form.
__global__ void gather_wnorm_kernel(const int32_t *__restrict__ pix, const float *__restrict__ w,
                                    const float *__restrict__ npx, int64_t n, float *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = pix[e];
        out[e] = p >= 0 ? __fdiv_rn(w[e], npx[p]) : 0.f;
    }
}

// One frame's two planes for the frames kernel: [cast(img) - dark] and, with corrections,
// [((1 * flat) * solid angle) * polarisation] -- the values the batched path forms per entry
// (dark) and in its norm pass, with the same roundings.
template <int DT>
__global__ void single_planes_kernel(const void *__restrict__ img, const float *__restrict__ dark,
                                     const float *__restrict__ flat, const float *__restrict__ sa,
                                     const float *__restrict__ pol, int64_t n, int with_norm,
                                     float *__restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        float v = img_f32<DT>(static_cast<const uint32_t *>(img)[p]);
        if (dark) v = __fsub_rn(v, dark[p]);
        out[p] = v;
        if (with_norm) {
            float m = 1.f;
            if (flat) m = __fmul_rn(m, flat[p]);
            if (sa) m = __fmul_rn(m, sa[p]);
            if (pol) m = __fmul_rn(m, pol[p]);
            out[n + p] = m;
        }
    }
}

__global__ void fill_f32_kernel(float *__restrict__ out, int64_t n, float v) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        out[p] = v;
}

}  // namespace

int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

int max_smem_per_block() {
    if (!g_max_smem) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (g_max_smem <= 0) g_max_smem = 48 * 1024;
    }
    return g_max_smem;
}

int forward_single(const az_integrator *h, const void *image, int dtype, const float *dark,
                   const float *flat, const float *sa, const float *pol, int precision, void *oI,
                   void *oS, void *oN, void *oC, cudaStream_t s) {
    const bool fp64 = precision == AZ_PREC_FP64;
    Inst d = make_inst(h, fp64);
    d.img = static_cast<const char *>(image);
    d.dark = dark; d.flat = flat; d.sa = sa; d.pol = pol;
    d.oI = oI; d.oS = oS; d.oN = oN; d.oC = oC;
    const int planes = 1 + (dark != nullptr) + (flat != nullptr) + (sa != nullptr) + (pol != nullptr);
    StageGeom sg = choose_stage(plane_words_of(h), planes, (uint32_t)h->tl.max_tile_entries,
                                fp64 ? 8 : 4, rec_words_of(h), d.stage_entries);
    const int eng = engine_for(h);
    TmaSet tm;
    AZ_TRY(make_maps(h, eng, image, h->ny, dark, flat, sa, pol, tm));
    if (fp64) {
        AZ_TRY((run_phase1_dt<double, double, MODE_SINGLE, 1>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof)));
        AZ_TRY((run_phase2<double, MODE_SINGLE>(d, nullptr, 1, h->nrows, 1, s, &h->prof)));
    } else {
        AZ_TRY((run_phase1_dt<float, float, MODE_SINGLE, 1>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof)));
        AZ_TRY((run_phase2<float, MODE_SINGLE>(d, nullptr, 1, h->nrows, 1, s, &h->prof)));
    }
    return AZ_OK;
}

// forward_single with the per-segment partial sums in a buffer the caller supplies (at least
// 3 * nseg values of the accumulation type) instead of the integrator's own; no profiling.
// Loads, without launching them, the kernels forward_single_into can launch (both
// precisions, every image type, both copy engines, and phase 2).  Under the CUDA runtime's
// lazy loading a kernel's code is otherwise loaded, and may take device memory, at its first
// launch.
template <class K> int preload_kernel(K k) {
    cudaFuncAttributes fa;
    AZ_CUDA(cudaFuncGetAttributes(&fa, k));
    return AZ_OK;
}
template <class AT, int DT> int preload_single_dt() {
    AZ_TRY(preload_kernel(phase1_kernel<AT, AT, MODE_SINGLE, 1, DT, true>));
    return preload_kernel(phase1_kernel<AT, AT, MODE_SINGLE, 1, DT, false>);
}
int preload_single_pass() {
    AZ_TRY((preload_single_dt<double, AZ_DTYPE_F32>()));
    AZ_TRY((preload_single_dt<double, AZ_DTYPE_U32>()));
    AZ_TRY((preload_single_dt<double, AZ_DTYPE_I32>()));
    AZ_TRY((preload_single_dt<float, AZ_DTYPE_F32>()));
    AZ_TRY((preload_single_dt<float, AZ_DTYPE_U32>()));
    AZ_TRY((preload_single_dt<float, AZ_DTYPE_I32>()));
    AZ_TRY(preload_kernel(phase2_kernel<double, MODE_SINGLE>));
    return preload_kernel(phase2_kernel<float, MODE_SINGLE>);
}

int forward_single_into(const az_integrator *h, const void *image, int dtype, const float *dark,
                        const float *flat, const float *sa, const float *pol, int precision,
                        void *oI, void *oS, void *oN, void *oC, void *partial, cudaStream_t s) {
    const bool fp64 = precision == AZ_PREC_FP64;
    Inst d = make_inst(h, fp64);
    d.partial = partial;
    d.img = static_cast<const char *>(image);
    d.dark = dark; d.flat = flat; d.sa = sa; d.pol = pol;
    d.oI = oI; d.oS = oS; d.oN = oN; d.oC = oC;
    const int planes = 1 + (dark != nullptr) + (flat != nullptr) + (sa != nullptr) + (pol != nullptr);
    StageGeom sg = choose_stage(plane_words_of(h), planes, (uint32_t)h->tl.max_tile_entries,
                                fp64 ? 8 : 4, rec_words_of(h), d.stage_entries);
    const int eng = engine_for(h);
    TmaSet tm;
    AZ_TRY(make_maps(h, eng, image, h->ny, dark, flat, sa, pol, tm));
    if (fp64) {
        AZ_TRY((run_phase1_dt<double, double, MODE_SINGLE, 1>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s)));
        AZ_TRY((run_phase2<double, MODE_SINGLE>(d, nullptr, 1, h->nrows, 1, s)));
    } else {
        AZ_TRY((run_phase1_dt<float, float, MODE_SINGLE, 1>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s)));
        AZ_TRY((run_phase2<float, MODE_SINGLE>(d, nullptr, 1, h->nrows, 1, s)));
    }
    return AZ_OK;
}

int batch_norm(az_integrator *h, const float *flat, const float *sa, const float *pol, float *oN,
               float *oC, cudaStream_t s) {
    Inst d = make_inst(h, false);
    d.flat = flat; d.sa = sa; d.pol = pol;
    d.oN = oN; d.oC = oC;
    if (engine_for(h) == AZ_COPY_TMA && h->partial_bytes >= 2 * sizeof(float) * (size_t)h->tl.nseg) {
        // Through the frames kernel.  C = sum w does not depend on the inputs: the first call
        // after a layout change reduces [flat * solid angle * polarisation; ones] as a
        // two-frame batch and keeps C; later calls reduce the first frame only (N), and
        // without flat, solid angle and polarisation N equals C.  Each weight meets the same
        // value as in the norm mode below, through the same accumulation.
        const int64_t npix = (int64_t)h->ny * h->nx;
        const int nrows = h->nrows;
        float *Cdev = h->norm.as<float>() + nrows;
        const bool corr = flat || sa || pol;
        if (h->count_ready && !corr) {
            AZ_CUDA(cudaMemcpyAsync(h->norm.as<float>(), Cdev, sizeof(float) * nrows, cudaMemcpyDeviceToDevice, s));
            if (oN) AZ_CUDA(cudaMemcpyAsync(oN, Cdev, sizeof(float) * nrows, cudaMemcpyDeviceToDevice, s));
            if (oC) AZ_CUDA(cudaMemcpyAsync(oC, Cdev, sizeof(float) * nrows, cudaMemcpyDeviceToDevice, s));
            return AZ_OK;
        }
        const int64_t blocks = std::min<int64_t>((npix + 255) / 256, (int64_t)num_sms() * 8);
        if (h->tl.norm_frames.bytes < 2 * sizeof(float) * (size_t)npix) {
            AZ_TRY(h->tl.norm_frames.alloc(2 * sizeof(float) * (size_t)npix));
            fill_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>(h->tl.norm_frames.as<float>() + npix, npix, 1.f);
            AZ_CUDA(cudaGetLastError());
        }
        {
            ProfScope ps(&h->prof, 4, s);
            norm_pixels_kernel<<<(unsigned)blocks, 256, 0, s>>>(flat, sa, pol, npix, h->tl.norm_frames.as<float>());
            AZ_CUDA(cudaGetLastError());
        }
        const int nf = h->count_ready ? 1 : 2;
        const int rc = frames_v3(h, h->tl.norm_frames.p, nf, AZ_DTYPE_F32, nullptr, 1, s);
        if (rc == AZ_OK) {
            d.norm_rows = nf;
            AZ_TRY((run_phase2<float, MODE_NORM>(d, nullptr, 1, h->nrows, 1, s, &h->prof)));
            if (nf == 1 && oC) AZ_CUDA(cudaMemcpyAsync(oC, Cdev, sizeof(float) * nrows, cudaMemcpyDeviceToDevice, s));
            h->count_ready = true;
            return AZ_OK;
        }
        if (rc != AZ_EUNSUPPORTED) return rc;
    }
    const int planes = (flat != nullptr) + (sa != nullptr) + (pol != nullptr);
    StageGeom sg = choose_stage(plane_words_of(h), planes, (uint32_t)h->tl.max_tile_entries, 4,
                                rec_words_of(h), d.stage_entries);
    const int eng = engine_for(h);
    TmaSet tm;
    AZ_TRY(make_maps(h, eng, nullptr, 0, nullptr, flat, sa, pol, tm));
    AZ_TRY((run_phase1_eng<float, float, MODE_NORM, 1, AZ_DTYPE_F32>(eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof)));
    AZ_TRY((run_phase2<float, MODE_NORM>(d, nullptr, 1, h->nrows, 1, s, &h->prof)));
    return AZ_OK;
}

int batch_frames(az_integrator *h, const void *frames, int n, int dtype, const float *dark,
                 float *oI, float *oS, int frame_out0, cudaStream_t s, const float *ent_dark_given,
                 const float *norm) {
    // the dark of every entry, in entry order, so that the frames pass reads it with the
    // weights instead of staging a dark plane with every group of frames (given: bound once
    // by az_set_corrections)
    const int ent_dk = dark != nullptr || ent_dark_given != nullptr;
    if (dark && !ent_dark_given) {
        TiledLayout &L = h->tl;
        if (L.ent_dark.bytes < sizeof(float) * (size_t)L.padded_nnz)
            AZ_TRY(L.ent_dark.alloc(sizeof(float) * (size_t)L.padded_nnz));
        const int64_t blocks = std::min<int64_t>((L.padded_nnz + 255) / 256, (int64_t)num_sms() * 8);
        ProfScope ps(&h->prof, 4, s);
        gather_dark_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(
            L.ent_pix.as<int32_t>(), dark, L.padded_nnz, L.ent_dark.as<float>());
        AZ_CUDA(cudaGetLastError());
    }
    const float *ent_dark = ent_dark_given ? ent_dark_given : h->tl.ent_dark.as<float>();
    // frames per pass as tuned, halved while two stages of that many frame planes do not fit,
    // or while the tile's entries would not fit beside them (down to 4 frames per pass)
    int fpi = h->frames_per_pass;
    while (fpi > 1) {
        int se = 0;
        const StageGeom g = choose_stage(plane_words_of(h), fpi, (uint32_t)h->tl.max_tile_entries, 4,
                                         rec_words_of(h), se, ent_dk);
        if ((int)smem_for(g) <= max_smem_per_block() && (se || fpi <= 4)) break;
        fpi >>= 1;
    }
    const int64_t cap = (int64_t)(h->partial_bytes / (sizeof(float) * (size_t)std::max(h->tl.nseg, 1)));
    const int chunk_max = (int)std::max<int64_t>(fpi, (cap / fpi) * fpi);
    const int planes = fpi;
    int stage_e = 0;
    StageGeom sg = choose_stage(plane_words_of(h), planes, (uint32_t)h->tl.max_tile_entries, 4,
                                rec_words_of(h), stage_e, ent_dk);
    const int eng = engine_for(h);
    if (eng == AZ_COPY_TMA) {
        // tile-resident entries (frames_kernel), up to kMaxFramesPerLaunch frames per launch
        const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(cap, kMaxFramesPerLaunch));
        for (int f0 = 0; f0 < n; f0 += chunk) {
            const int nf = std::min(chunk, n - f0);
            Inst d = make_inst(h, false);
            d.img = static_cast<const char *>(frames) + (size_t)f0 * (size_t)d.npix * 4u;
            const int rc = frames_v3(h, d.img, nf, dtype, ent_dk ? ent_dark : nullptr, 0, s);
            if (rc == AZ_EUNSUPPORTED && f0 == 0) break;  // the general kernel below
            AZ_TRY(rc);
            if (norm) d.norm = const_cast<float *>(norm);
            d.n_frames = nf;
            d.oI = oI; d.oS = oS; d.frame_out0 = frame_out0 + f0;
            AZ_TRY((run_phase2<float, MODE_FRAMES>(d, nullptr, 1, (int64_t)nf * h->nrows, nf, s, &h->prof)));
            if (f0 + nf >= n) return AZ_OK;
        }
    }
    for (int f0 = 0; f0 < n; f0 += chunk_max) {
        const int nf = std::min(chunk_max, n - f0);
        Inst d = make_inst(h, false);
        d.img = static_cast<const char *>(frames) + (size_t)f0 * (size_t)d.npix * 4u;
        d.n_frames = nf; d.fpi = fpi; d.n_groups = (nf + fpi - 1) / fpi;
        d.rpw = 32 / fpi;
        d.dark = dark;
        d.ent_dark = ent_dk ? ent_dark : nullptr;
        if (norm) d.norm = const_cast<float *>(norm);
        d.oI = oI; d.oS = oS; d.frame_out0 = frame_out0 + f0;
        d.stage_entries = stage_e;
        d.n_items = h->tl.n_active * d.n_groups;
        TmaSet tm;
        AZ_TRY(make_maps(h, eng, d.img, (int64_t)nf * h->ny, nullptr, nullptr, nullptr, nullptr, tm));
        switch (fpi) {
            case 1: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 1>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof))); break;
            case 2: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 2>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof))); break;
            case 4: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 4>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof))); break;
            case 8: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 8>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof))); break;
            case 16: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 16>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof))); break;
            default: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 32>(dtype, eng, d, nullptr, 1, d.n_items, sg, tm, s, &h->prof))); break;
        }
        AZ_TRY((run_phase2<float, MODE_FRAMES>(d, nullptr, 1, (int64_t)nf * h->nrows, nf, s, &h->prof)));
    }
    return AZ_OK;
}

// The paper's per-pixel-corrected form for n frames: U = sum (w / (flat Omega P)) (img - dark)
// and I = U / C, C = sum w (kept per layout).  Through the frames kernel with the weights
// divided by each pixel's normalisation once per call.
int batch_pixelnorm(az_integrator *h, const void *frames, int n, int dtype, const float *dark,
                    const float *flat, const float *sa, const float *pol, float *oI, float *oU,
                    float *oC, cudaStream_t s) {
    if (engine_for(h) != AZ_COPY_TMA || h->partial_bytes < 2 * sizeof(float) * (size_t)h->tl.nseg)
        return fail(AZ_EUNSUPPORTED, "az_integrate_batch_pixelnorm: needs the tensor-copy engine (tiles up to 236 pixels wide)");
    TiledLayout &L = h->tl;
    const int64_t npix = (int64_t)h->ny * h->nx;
    const int nrows = h->nrows;
    // C (and, incidentally, N = C) for the current layout
    if (!h->count_ready) AZ_TRY(batch_norm(h, nullptr, nullptr, nullptr, nullptr, nullptr, s));
    const float *Cdev = h->norm.as<float>() + nrows;
    if (oC) AZ_CUDA(cudaMemcpyAsync(oC, Cdev, sizeof(float) * nrows, cudaMemcpyDeviceToDevice, s));
    if (n == 0) return AZ_OK;
    // per-pixel normalisation, per-entry corrected weights and darks
    const int64_t pblocks = std::min<int64_t>((npix + 255) / 256, (int64_t)num_sms() * 8);
    const int64_t eblocks = std::max<int64_t>(1, std::min<int64_t>((L.padded_nnz + 255) / 256, (int64_t)num_sms() * 8));
    if (L.norm_frames.bytes < 2 * sizeof(float) * (size_t)npix) {
        AZ_TRY(L.norm_frames.alloc(2 * sizeof(float) * (size_t)npix));
        fill_f32_kernel<<<(unsigned)pblocks, 256, 0, s>>>(L.norm_frames.as<float>() + npix, npix, 1.f);
        AZ_CUDA(cudaGetLastError());
    }
    if (L.ent_wnorm.bytes < sizeof(float) * (size_t)L.padded_nnz)
        AZ_TRY(L.ent_wnorm.alloc(sizeof(float) * (size_t)L.padded_nnz));
    {
        ProfScope ps(&h->prof, 4, s);
        norm_pixels_kernel<<<(unsigned)pblocks, 256, 0, s>>>(flat, sa, pol, npix, L.norm_frames.as<float>());
        gather_wnorm_kernel<<<(unsigned)eblocks, 256, 0, s>>>(L.ent_pix.as<int32_t>(), L.ent_w32.as<float>(),
                                                              L.norm_frames.as<float>(), L.padded_nnz,
                                                              L.ent_wnorm.as<float>());
        AZ_CUDA(cudaGetLastError());
    }
    const float *ent_dk = nullptr;
    if (dark) {
        if (L.ent_dark.bytes < sizeof(float) * (size_t)L.padded_nnz)
            AZ_TRY(L.ent_dark.alloc(sizeof(float) * (size_t)L.padded_nnz));
        ProfScope ps(&h->prof, 4, s);
        gather_dark_kernel<<<(unsigned)eblocks, 256, 0, s>>>(L.ent_pix.as<int32_t>(), dark, L.padded_nnz,
                                                             L.ent_dark.as<float>());
        AZ_CUDA(cudaGetLastError());
        ent_dk = L.ent_dark.as<float>();
    }
    const int64_t cap = (int64_t)(h->partial_bytes / (sizeof(float) * (size_t)std::max(L.nseg, 1)));
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(cap, kMaxFramesPerLaunch));
    for (int f0 = 0; f0 < n; f0 += chunk) {
        const int nf = std::min(chunk, n - f0);
        Inst d = make_inst(h, false);
        d.img = static_cast<const char *>(frames) + (size_t)f0 * (size_t)d.npix * 4u;
        const int rc = frames_v3(h, d.img, nf, dtype, ent_dk, 0, s, false, L.ent_wnorm.as<float>());
        if (rc == AZ_EUNSUPPORTED)
            return fail(AZ_EUNSUPPORTED, "az_integrate_batch_pixelnorm: the tiles do not fit in shared memory");
        AZ_TRY(rc);
        d.n_frames = nf;
        d.norm = const_cast<float *>(Cdev);  // I = U / C
        d.oI = oI; d.oS = oU; d.frame_out0 = f0;
        AZ_TRY((run_phase2<float, MODE_FRAMES>(d, nullptr, 1, (int64_t)nf * nrows, nf, s, &h->prof)));
    }
    return AZ_OK;
}

// Propagated variance of the signal sums, V = sum w^2 max(img, 0), for n frames through the
// frames kernel (chunks of up to kMaxFramesPerLaunch frames), written to oV [n][nrows].
int batch_variance(az_integrator *h, const void *frames, int n, int dtype, float *oV, cudaStream_t s) {
    if (engine_for(h) != AZ_COPY_TMA)
        return fail(AZ_EUNSUPPORTED, "az_integrate_variance: needs the tensor-copy engine (tiles up to 236 pixels wide)");
    const int64_t cap = (int64_t)(h->partial_bytes / (sizeof(float) * (size_t)std::max(h->tl.nseg, 1)));
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(cap, kMaxFramesPerLaunch));
    for (int f0 = 0; f0 < n; f0 += chunk) {
        const int nf = std::min(chunk, n - f0);
        Inst d = make_inst(h, false);
        d.img = static_cast<const char *>(frames) + (size_t)f0 * (size_t)d.npix * 4u;
        const int rc = frames_v3(h, d.img, nf, dtype, nullptr, 0, s, true);
        if (rc == AZ_EUNSUPPORTED)
            return fail(AZ_EUNSUPPORTED, "az_integrate_variance: the tiles do not fit in shared memory");
        AZ_TRY(rc);
        d.n_frames = nf;
        d.oI = nullptr; d.oS = oV; d.frame_out0 = f0;
        AZ_TRY((run_phase2<float, MODE_FRAMES>(d, nullptr, 1, (int64_t)nf * h->nrows, nf, s, &h->prof)));
    }
    return AZ_OK;
}

// One frame through the batched path (TMA engine only; AZ_EUNSUPPORTED, without error
// text, otherwise).  The N pass needs two frames of partials.
int forward_batch_one(az_integrator *h, const void *image, int dtype, const float *dark,
                      const float *flat, const float *sa, const float *pol, float *oI, float *oS,
                      float *oN, float *oC, cudaStream_t s) {
    if (engine_for(h) != AZ_COPY_TMA || h->partial_bytes < 2 * sizeof(float) * (size_t)h->tl.nseg)
        return AZ_EUNSUPPORTED;
    // C of the current layout, once
    if (!h->count_ready) AZ_TRY(batch_norm(h, nullptr, nullptr, nullptr, nullptr, nullptr, s));
    // Three launches: the frame's planes [img - dark; flat * Omega * P], the frames kernel over
    // them as a batch of two frames (S and N per segment, the accumulation of every other
    // frame), and phase 2 with C from the cache.  Without flat, solid angle and polarisation
    // only the first plane is reduced and N = C.
    const int64_t npix = (int64_t)h->ny * h->nx;
    const bool corr = flat || sa || pol;
    if (h->one_planes.bytes < 2 * sizeof(float) * (size_t)npix)
        AZ_TRY(h->one_planes.alloc(2 * sizeof(float) * (size_t)npix));
    float *planes = h->one_planes.as<float>();
    {
        ProfScope ps(&h->prof, 4, s);
        const unsigned g = (unsigned)std::min<int64_t>((npix + 255) / 256, (int64_t)num_sms() * 8);
        const int wn = corr ? 1 : 0;
        switch (dtype) {
            case AZ_DTYPE_F32: single_planes_kernel<AZ_DTYPE_F32><<<g, 256, 0, s>>>(image, dark, flat, sa, pol, npix, wn, planes); break;
            case AZ_DTYPE_U32: single_planes_kernel<AZ_DTYPE_U32><<<g, 256, 0, s>>>(image, dark, flat, sa, pol, npix, wn, planes); break;
            default: single_planes_kernel<AZ_DTYPE_I32><<<g, 256, 0, s>>>(image, dark, flat, sa, pol, npix, wn, planes); break;
        }
        AZ_CUDA(cudaGetLastError());
    }
    const int rc = frames_v3(h, planes, corr ? 2 : 1, AZ_DTYPE_F32, nullptr, 2, s);
    if (rc != AZ_OK) return rc;
    Inst d = make_inst(h, false);
    d.oI = oI; d.oS = oS; d.oN = oN; d.oC = oC;
    d.single_nc = corr ? 1 : 2;
    return run_phase2<float, MODE_SINGLE>(d, nullptr, 1, h->nrows, 1, s, &h->prof);
}

int forward_batch(az_integrator *h, const void *frames, int n, int dtype, const float *dark,
                  const float *flat, const float *sa, const float *pol, float *oI, float *oS,
                  float *oN, float *oC, cudaStream_t s) {
    AZ_TRY(batch_norm(h, flat, sa, pol, oN, oC, s));
    return batch_frames(h, frames, n, dtype, dark, oI, oS, 0, s);
}

// az_set_corrections: the frame-independent work of a batch formed once -- each entry's dark
// (gathered from `dark`) and N, C per row -- into buffers of their own, which later calls of
// az_integrate_batch do not touch.  The caller's arrays are not read again.
int bind_corrections(az_integrator *h, const float *dark, const float *flat, const float *sa,
                     const float *pol, cudaStream_t s) {
    TiledLayout &L = h->tl;
    h->corr_bound = false;
    h->corr_dark = dark != nullptr;
    if (dark) {
        if (h->bound_ent_dark.bytes < sizeof(float) * (size_t)L.padded_nnz)
            AZ_TRY(h->bound_ent_dark.alloc(sizeof(float) * (size_t)L.padded_nnz));
        const int64_t blocks = std::min<int64_t>((L.padded_nnz + 255) / 256, (int64_t)num_sms() * 8);
        ProfScope ps(&h->prof, 4, s);
        gather_dark_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(
            L.ent_pix.as<int32_t>(), dark, L.padded_nnz, h->bound_ent_dark.as<float>());
        AZ_CUDA(cudaGetLastError());
    }
    if (h->bound_norm.bytes < 2 * sizeof(float) * (size_t)h->nrows)
        AZ_TRY(h->bound_norm.alloc(2 * sizeof(float) * (size_t)h->nrows));
    float *bN = h->bound_norm.as<float>();
    AZ_TRY(batch_norm(h, flat, sa, pol, bN, bN + h->nrows, s));
    h->corr_bound = true;
    return AZ_OK;
}

// Frames through the bound corrections: the frames pass with the bound per-entry darks and
// phase 2 with the bound N.  oN, oC (may be NULL) receive copies of the bound N and C.
int forward_batch_bound(az_integrator *h, const void *frames, int n, int dtype, float *oI, float *oS,
                        float *oN, float *oC, cudaStream_t s) {
    if (!h->corr_bound)
        return fail(AZ_EINVAL, "az_integrate_batch_bound: no corrections are bound (az_set_corrections), "
                               "or the tiled layout changed since they were");
    const float *bN = h->bound_norm.as<float>();
    const size_t rb = sizeof(float) * (size_t)h->nrows;
    if (oN) AZ_CUDA(cudaMemcpyAsync(oN, bN, rb, cudaMemcpyDeviceToDevice, s));
    if (oC) AZ_CUDA(cudaMemcpyAsync(oC, bN + h->nrows, rb, cudaMemcpyDeviceToDevice, s));
    if (n == 0) return AZ_OK;
    return batch_frames(h, frames, n, dtype, nullptr, oI, oS, 0, s,
                        h->corr_dark ? h->bound_ent_dark.as<float>() : nullptr, bN);
}

// ------------------------------------------------------------------------------------
// heterogeneous instances in one persistent launch
// ------------------------------------------------------------------------------------
struct MultiPlan {
    std::vector<Inst> host;
    DevBuf dev;
    DevBuf maps;  // TMA engine: n TmaSets, one per instance, read by the producers
    int n = 0;
    int dtype = 0, engine = 0;
    int64_t n_items = 0, n_rows = 0;
    StageGeom sg{};
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

int multi_create(az_integrator *const *hs, int n, const void *const *images, int dtype,
                 const float *const *darks, const float *const *flats, const float *const *sas,
                 const float *const *pols, float *const *oI, float *const *oS, float *const *oN,
                 float *const *oC, void **out) {
    MultiPlan *P = new (std::nothrow) MultiPlan;
    if (!P) return fail(AZ_ENOMEM, "az_multi_create: out of host memory");
    P->n = n;
    P->dtype = dtype;
    int64_t items = 0, rows = 0;
    uint32_t pw = 0, ecap = 0, rw = 0;
    // The TMA engine when every instance can use it: each instance's tensor maps then live in
    // device memory (a launch parameter holds one set only) and the producers read them there.
    P->engine = AZ_COPY_TMA;
    for (int k = 0; k < n; ++k)
        if (engine_for(hs[k]) != AZ_COPY_TMA) P->engine = AZ_COPY_ASYNC;
    std::vector<TmaSet> maps;
    if (P->engine == AZ_COPY_TMA) {
        maps.resize((size_t)n);
        int rc = P->maps.alloc(sizeof(TmaSet) * (size_t)n);
        for (int k = 0; k < n && rc == AZ_OK; ++k)
            rc = make_maps(hs[k], AZ_COPY_TMA, images[k], hs[k]->ny, darks ? darks[k] : nullptr,
                           flats ? flats[k] : nullptr, sas ? sas[k] : nullptr, pols ? pols[k] : nullptr,
                           maps[(size_t)k]);
        if (rc == AZ_OK) {
            cudaError_t e = cudaMemcpy(P->maps.p, maps.data(), sizeof(TmaSet) * (size_t)n, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) rc = fail(AZ_ECUDA, "az_multi_create: %s", cudaGetErrorString(e));
        }
        if (rc != AZ_OK) {
            delete P;
            return rc;
        }
    }
    int planes = 0;
    for (int k = 0; k < n; ++k) {
        const az_integrator *h = hs[k];
        Inst d = make_inst(h, false);
        d.img = static_cast<const char *>(images[k]);
        d.dark = darks ? darks[k] : nullptr;
        d.flat = flats ? flats[k] : nullptr;
        d.sa = sas ? sas[k] : nullptr;
        d.pol = pols ? pols[k] : nullptr;
        d.oI = oI ? oI[k] : nullptr;
        d.oS = oS ? oS[k] : nullptr;
        d.oN = oN ? oN[k] : nullptr;
        d.oC = oC ? oC[k] : nullptr;
        if (P->engine == AZ_COPY_TMA) d.maps = &P->maps.as<TmaSet>()[k].m[0][0];
        d.item_begin = items;
        d.row_begin = rows;
        items += d.n_items;
        rows += h->nrows;
        pw = std::max(pw, plane_words_of(h));
        ecap = std::max(ecap, (uint32_t)h->tl.max_tile_entries);
        rw = std::max(rw, rec_words_of(h));
        planes = std::max(planes, 1 + (d.dark != nullptr) + (d.flat != nullptr) + (d.sa != nullptr) +
                                      (d.pol != nullptr));
        P->host.push_back(d);
    }
    int stage_e = 0;
    P->sg = choose_stage(pw, planes, ecap, 4, rw, stage_e);
    for (auto &d : P->host) d.stage_entries = stage_e;
    P->n_items = items;
    P->n_rows = rows;
    int rc = P->dev.alloc(sizeof(Inst) * (size_t)n);
    if (rc == AZ_OK) {
        cudaError_t e = cudaMemcpy(P->dev.p, P->host.data(), sizeof(Inst) * (size_t)n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = fail(AZ_ECUDA, "az_multi_create: %s", cudaGetErrorString(e));
    }
    if (rc != AZ_OK) {
        delete P;
        return rc;
    }
    *out = P;
    return AZ_OK;
}

int multi_enqueue(void *plan, cudaStream_t s) {
    MultiPlan *P = static_cast<MultiPlan *>(plan);
    const Inst *dev = P->dev.as<Inst>();
    static TmaSet no_maps;  // zero: the producers read each instance's maps from Inst::maps
    AZ_TRY((run_phase1_dt<float, float, MODE_SINGLE, 1>(P->dtype, P->engine, P->host[0], dev, P->n, P->n_items, P->sg, no_maps, s)));
    AZ_TRY((run_phase2<float, MODE_SINGLE>(P->host[0], dev, P->n, P->n_rows, 1, s)));
    return AZ_OK;
}

int multi_launch(void *plan, int use_graph, cudaStream_t s) {
    MultiPlan *P = static_cast<MultiPlan *>(plan);
    if (!use_graph) return multi_enqueue(plan, s);
    if (!P->exec) {
        // Run once eagerly (this call's results; it also configures the kernels), then
        // capture the two launches on a private stream: the caller's stream may be the
        // legacy default stream, which cannot be captured.
        AZ_TRY(multi_enqueue(plan, s));
        cudaStream_t cs = nullptr;
        AZ_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        int rc = e == cudaSuccess ? multi_enqueue(plan, cs)
                                  : fail(AZ_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraph_t g = nullptr;
        if (e == cudaSuccess) {
            e = cudaStreamEndCapture(cs, &g);
            if (e != cudaSuccess && rc == AZ_OK) rc = fail(AZ_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        cudaStreamDestroy(cs);
        if (rc != AZ_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        P->graph = g;
        AZ_CUDA(cudaGraphInstantiate(&P->exec, g, 0));
        return AZ_OK;
    }
    AZ_CUDA(cudaGraphLaunch(P->exec, s));
    return AZ_OK;
}

void multi_destroy(void *plan) {
    MultiPlan *P = static_cast<MultiPlan *>(plan);
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    delete P;
}

}  // namespace azint
