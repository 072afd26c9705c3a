// Fused correction + sparse matrix-vector product (Sec. 5.2, Sec. 6.4) on the pixel-tiled
// layout, in two deterministic launches:
//
//   phase 1 (persistent): each CTA walks a static round-robin list of work items (an active
//     pixel tile, and for many frames a group of frames).  Warp 0 bulk-copies (TMA,
//     cp.async.bulk + mbarrier) the tile's rows of every needed plane -- image frames,
//     dark, flat, solid angle, polarisation -- and the tile's matrix entries into one of two
//     shared-memory stages while the CTA reduces the previous item from the other stage.
//     Groups of 32/R lanes each reduce one matrix row ("segment") of the tile from shared
//     memory, R rows per warp, and write one partial sum per (segment, plane).
//   phase 2: one warp per (row, frame) sums the row's partials in a fixed order and forms
//     S, N, C and I = S / N.
//
// Casting the image, subtracting the dark, forming flat * solid angle * polarisation and
// the reduction happen in the same pass (the paper's separate cast / correction / memset /
// integrate kernels).  FP32 sums are Kahan-compensated (Sec. 5.2.2); FP64 sums are plain.
// No atomics are used, so results are bit-reproducible run to run.
#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

namespace azint {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxPlanes = 12;

enum Mode { MODE_SINGLE = 0, MODE_NORM = 1, MODE_FRAMES = 2 };

// Everything phase 1 and phase 2 need about one integrator and its inputs.
struct Inst {
    // tiled layout
    const int32_t *tile_seg_ptr, *tile_ent_ptr, *active_tiles;
    const int32_t *seg_start, *seg_end, *seg_slot, *row_slot_ptr;
    const uint16_t *ent_loc;
    const void *ent_w;
    int ny, nx, th, tw, srow, ntx, rpw, nseg, nrows;
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
    int64_t item_begin, row_begin;
    int n_items;
    int stage_entries;
    int *status;
};

struct StageGeom {
    uint32_t plane_words;   // words per plane slot
    uint32_t plane_region;  // bytes of the plane region
    uint32_t ent_cap;       // entry capacity (staged entries)
    uint32_t stage_bytes;   // bytes per stage (multiple of 128)
};

template <int MODE, int NIMG>
__device__ __forceinline__ int plane_list(const Inst &d, int group, const char **base, int &nimg,
                                          int &p_dark, int &p_flat, int &p_sa, int &p_pol) {
    int n = 0;
    nimg = 0;
    if (MODE == MODE_SINGLE) {
        base[n++] = d.img;
        nimg = 1;
    } else if (MODE == MODE_FRAMES) {
        const int f0 = group * d.fpi;
        const int nf = min(d.fpi, d.n_frames - f0);
        for (int f = 0; f < nf; ++f) base[n++] = d.img + (size_t)(f0 + f) * (size_t)d.npix * 4u;
        nimg = nf;
    }
    p_dark = p_flat = p_sa = p_pol = -1;
    if (MODE != MODE_NORM && d.dark) { p_dark = n; base[n++] = (const char *)d.dark; }
    if (MODE != MODE_FRAMES) {
        if (d.flat) { p_flat = n; base[n++] = (const char *)d.flat; }
        if (d.sa) { p_sa = n; base[n++] = (const char *)d.sa; }
        if (d.pol) { p_pol = n; base[n++] = (const char *)d.pol; }
    }
    return n;
}

__device__ __forceinline__ const Inst &inst_of(const Inst &single, const Inst *multi, int n_inst,
                                               int64_t item, int &k) {
    if (!multi) { k = 0; return single; }
    int lo = 0, hi = n_inst;  // last instance with item_begin <= item
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (multi[mid].item_begin <= item) lo = mid; else hi = mid;
    }
    k = lo;
    return multi[lo];
}

template <int MODE, int NIMG, class WT>
__device__ void issue_item(const Inst &d, int64_t local, unsigned char *stage, const StageGeom &sg,
                           uint64_t *bar) {
    const int lane = threadIdx.x & 31;
    const int a = (int)(local / d.n_groups), group = (int)(local % d.n_groups);
    const int t = d.active_tiles[a];
    const int ti = t / d.ntx, tj = t - ti * d.ntx;
    const int r0 = ti * d.th, c0 = tj * d.tw;
    const int rows = min(d.th, d.ny - r0), tweff = min(d.tw, d.nx - c0);
    const char *base[kMaxPlanes];
    int nimg, pd, pf, ps, pp;
    const int np = plane_list<MODE, NIMG>(d, group, base, nimg, pd, pf, ps, pp);
    uint32_t *planes = reinterpret_cast<uint32_t *>(stage);
    const uint32_t pw = (uint32_t)d.th * d.srow;

    // bytes this lane will copy
    uint32_t mine = 0;
    for (int pl = 0; pl < np; ++pl)
        for (int ly = lane; ly < rows; ly += 32) {
            const int64_t q = (int64_t)(r0 + ly) * d.nx + c0;
            const uintptr_t src = reinterpret_cast<uintptr_t>(base[pl]) + 4u * (uintptr_t)q;
            const uintptr_t lo = src & ~(uintptr_t)15;
            const uintptr_t hi = (src + 4u * (uintptr_t)tweff + 15u) & ~(uintptr_t)15;
            mine += (uint32_t)(hi - lo);
        }
    const int e0 = d.tile_ent_ptr[t], e1 = d.tile_ent_ptr[t + 1];
    const uint32_t ne = (uint32_t)(e1 - e0);
    if (d.stage_entries && lane == 0) mine += ne * 2u + ne * (uint32_t)sizeof(WT);

    fence_proxy_async_smem();
    if (mine) asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(
                               smem_addr(bar)), "r"(mine)
                           : "memory");
    for (int pl = 0; pl < np; ++pl) {
        const int dlt = (int)((reinterpret_cast<uintptr_t>(base[pl]) >> 2) & 3u);
        for (int ly = lane; ly < rows; ly += 32) {
            const int64_t q = (int64_t)(r0 + ly) * d.nx + c0;
            const uintptr_t src = reinterpret_cast<uintptr_t>(base[pl]) + 4u * (uintptr_t)q;
            const uintptr_t lo = src & ~(uintptr_t)15;
            const uintptr_t hi = (src + 4u * (uintptr_t)tweff + 15u) & ~(uintptr_t)15;
            const int m0 = (int)(q & 3);
            const int dst_off = (m0 + dlt) >= 4 ? 4 : 0;
            uint32_t *dst = planes + (size_t)pl * pw + (size_t)ly * d.srow + dst_off;
            bulk_g2s(dst, reinterpret_cast<const void *>(lo), (uint32_t)(hi - lo), bar);
        }
    }
    if (d.stage_entries && lane == 0 && ne) {
        unsigned char *eloc = stage + sg.plane_region;
        unsigned char *ew = eloc + sg.ent_cap * 2u;
        bulk_g2s(eloc, d.ent_loc + e0, ne * 2u, bar);
        bulk_g2s(ew, static_cast<const WT *>(d.ent_w) + e0, ne * (uint32_t)sizeof(WT), bar);
    }
    __syncwarp();
    if (lane == 0) {
        uint64_t st;
        asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(smem_addr(bar)) : "memory");
        (void)st;
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
    __device__ void zero() { k.s = 0.f; k.c = 0.f; }
    __device__ void add(float w, float v) { kahan_add(k, w, v); }
    __device__ void merge_xor(int m) { Kahan o = shfl_xor(k, m); kahan_merge(k, o); }
    __device__ float value() const { return kahan_value(k); }
};
template <> struct Acc<double> {
    double s;
    __device__ void zero() { s = 0.0; }
    __device__ void add(double w, double v) { s = __fma_rn(w, v, s); }
    __device__ void merge_xor(int m) { s += __shfl_xor_sync(0xffffffffu, s, m); }
    __device__ double value() const { return s; }
};

template <int R, class AT, class WT, int MODE, int NIMG, int DT>
__device__ void reduce_tile(const Inst &d, int64_t local, const unsigned char *stage,
                            const StageGeom &sg) {
    constexpr int G = 32 / R;
    constexpr int NACC = MODE == MODE_SINGLE ? 3 : (MODE == MODE_NORM ? 2 : NIMG);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G, li = lane % G;
    const int a = (int)(local / d.n_groups), group = (int)(local % d.n_groups);
    const int t = d.active_tiles[a];
    const char *base[kMaxPlanes];
    int nimg, pd, pf, ps, pp;
    plane_list<MODE, NIMG>(d, group, base, nimg, pd, pf, ps, pp);
    const uint32_t *planes = reinterpret_cast<const uint32_t *>(stage);
    const uint32_t pw = (uint32_t)d.th * d.srow;
    auto off = [&](int pl) -> int {
        return pl < 0 ? 0 : (int)(pl * pw + ((reinterpret_cast<uintptr_t>(base[pl]) >> 2) & 3u));
    };
    int oimg[NIMG > 0 ? NIMG : 1];
#pragma unroll
    for (int f = 0; f < (NIMG > 0 ? NIMG : 1); ++f) oimg[f] = off(f < nimg ? f : -1);
    const int odark = off(pd), oflat = off(pf), osa = off(ps), opol = off(pp);
    const int tile_e0 = d.tile_ent_ptr[t];
    const uint16_t *L;
    const WT *W;
    if (d.stage_entries) {
        L = reinterpret_cast<const uint16_t *>(stage + sg.plane_region);
        W = reinterpret_cast<const WT *>(stage + sg.plane_region + sg.ent_cap * 2u);
    } else {
        L = d.ent_loc + tile_e0;
        W = static_cast<const WT *>(d.ent_w) + tile_e0;
    }
    const int s0 = d.tile_seg_ptr[t], ns = d.tile_seg_ptr[t + 1] - s0;
    for (int b = 0; b < ns; b += kWarps * R) {
        const int sl = b + warp * R + grp;
        const bool has = sl < ns;
        int e0 = 0, e1 = 0, slot = 0;
        if (has) {
            e0 = d.seg_start[s0 + sl] - tile_e0;
            e1 = d.seg_end[s0 + sl] - tile_e0;
            slot = d.seg_slot[s0 + sl];
        }
        Acc<AT> acc[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[k].zero();
#pragma unroll 4
        for (int e = e0 + li; e < e1; e += G) {
            const int loc = L[e];
            const AT w = (AT)W[e];
            if (MODE == MODE_SINGLE) {
                AT v, n = AT(1);
                if (sizeof(AT) == 8) {
                    v = (AT)img_f64<DT>(planes[oimg[0] + loc]);
                    if (pd >= 0) v = v - (AT)__uint_as_float(planes[odark + loc]);
                } else {
                    v = (AT)img_f32<DT>(planes[oimg[0] + loc]);
                    if (pd >= 0) v = __fsub_rn((float)v, __uint_as_float(planes[odark + loc]));
                }
                if (pf >= 0) n = n * (AT)__uint_as_float(planes[oflat + loc]);
                if (ps >= 0) n = n * (AT)__uint_as_float(planes[osa + loc]);
                if (pp >= 0) n = n * (AT)__uint_as_float(planes[opol + loc]);
                acc[0].add(w, v);
                acc[1].add(w, n);
                acc[2].add(w, AT(1));
            } else if (MODE == MODE_NORM) {
                AT n = AT(1);
                if (pf >= 0) n = n * (AT)__uint_as_float(planes[oflat + loc]);
                if (ps >= 0) n = n * (AT)__uint_as_float(planes[osa + loc]);
                if (pp >= 0) n = n * (AT)__uint_as_float(planes[opol + loc]);
                acc[0].add(w, n);
                acc[1].add(w, AT(1));
            } else {
                const float dk = pd >= 0 ? __uint_as_float(planes[odark + loc]) : 0.f;
#pragma unroll
                for (int f = 0; f < NIMG; ++f) {
                    if (f < nimg) {
                        float v = img_f32<DT>(planes[oimg[f] + loc]);
                        if (pd >= 0) v = __fsub_rn(v, dk);
                        acc[f].add((float)w, v);
                    }
                }
            }
        }
#pragma unroll
        for (int m = G / 2; m > 0; m >>= 1)
#pragma unroll
            for (int k = 0; k < NACC; ++k) acc[k].merge_xor(m);
        if (has && li == 0) {
            AT *out = static_cast<AT *>(d.partial);
            if (MODE == MODE_FRAMES) {
                const int f0 = group * d.fpi;
#pragma unroll
                for (int f = 0; f < NACC; ++f)
                    if (f < nimg) out[(size_t)(f0 + f) * d.nseg + slot] = acc[f].value();
            } else {
#pragma unroll
                for (int k = 0; k < NACC; ++k) out[(size_t)k * d.nseg + slot] = acc[k].value();
            }
        }
    }
}

template <class AT, class WT, int MODE, int NIMG, int DT>
__device__ __forceinline__ void reduce_dispatch(const Inst &d, int64_t local,
                                                const unsigned char *stage, const StageGeom &sg) {
    switch (d.rpw) {
        case 1: reduce_tile<1, AT, WT, MODE, NIMG, DT>(d, local, stage, sg); break;
        case 2: reduce_tile<2, AT, WT, MODE, NIMG, DT>(d, local, stage, sg); break;
        case 4: reduce_tile<4, AT, WT, MODE, NIMG, DT>(d, local, stage, sg); break;
        default: reduce_tile<8, AT, WT, MODE, NIMG, DT>(d, local, stage, sg); break;
    }
}

template <class AT, class WT, int MODE, int NIMG, int DT>
__global__ void __launch_bounds__(kThreads, 1)
phase1_kernel(const __grid_constant__ Inst single, const Inst *__restrict__ multi, int n_inst,
              int64_t n_items, StageGeom sg) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * (size_t)sg.stage_bytes);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    int64_t item = blockIdx.x;
    if (item < n_items && warp == 0) {
        int k;
        const Inst &d = inst_of(single, multi, n_inst, item, k);
        issue_item<MODE, NIMG, WT>(d, item - d.item_begin, smem, sg, &bars[0]);
    }
    for (int it = 0; item < n_items; ++it, item += gridDim.x) {
        const int st = it & 1;
        const int64_t next = item + gridDim.x;
        if (next < n_items && warp == 0) {
            int k;
            const Inst &dn = inst_of(single, multi, n_inst, next, k);
            issue_item<MODE, NIMG, WT>(dn, next - dn.item_begin, smem + (size_t)(st ^ 1) * sg.stage_bytes,
                                       sg, &bars[st ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((it >> 1) & 1));
        int k;
        const Inst &d = inst_of(single, multi, n_inst, item, k);
        if (!__syncthreads_and(ok)) {
            // A copy never completed: record it, give in-flight copies a bounded grace
            // period, and leave.
            if (threadIdx.x == 0) {
                atomicExch(d.status, AZ_ETIMEOUT);
                mbar_wait_bounded(&bars[st], (uint32_t)((it >> 1) & 1));
                if (next < n_items) mbar_wait_bounded(&bars[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            return;
        }
        reduce_dispatch<AT, WT, MODE, NIMG, DT>(d, item - d.item_begin, smem + (size_t)st * sg.stage_bytes, sg);
        __syncthreads();
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
                const AT N = row_sum<AT>(P + d.nseg, a, b);
                const AT C = row_sum<AT>(P + 2 * (size_t)d.nseg, a, b);
                if (lane == 0) {
                    const AT I = N != AT(0) ? S / N : AT(0);
                    if (d.oI) static_cast<AT *>(d.oI)[r] = I;
                    if (d.oS) static_cast<AT *>(d.oS)[r] = S;
                    if (d.oN) static_cast<AT *>(d.oN)[r] = N;
                    if (d.oC) static_cast<AT *>(d.oC)[r] = C;
                }
            } else {
                const AT N = row_sum<AT>(P, a, b);
                const AT C = row_sum<AT>(P + d.nseg, a, b);
                if (lane == 0) {
                    d.norm[r] = (float)N;
                    d.norm[d.nrows + r] = (float)C;
                    if (d.oN) static_cast<float *>(d.oN)[r] = (float)N;
                    if (d.oC) static_cast<float *>(d.oC)[r] = (float)C;
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
StageGeom stage_geom(uint32_t plane_words, int planes, uint32_t ent_cap, int wbytes) {
    StageGeom sg;
    sg.plane_words = plane_words;
    sg.plane_region = (uint32_t)planes * plane_words * 4u;
    sg.ent_cap = ent_cap;
    uint32_t bytes = sg.plane_region + ent_cap * (2u + (uint32_t)wbytes);
    sg.stage_bytes = (bytes + 127u) & ~127u;
    return sg;
}

uint32_t smem_for(const StageGeom &sg) { return 2u * sg.stage_bytes + 64u; }

// Stage the entries when the largest tile fits twice next to the planes; otherwise the
// reduction reads the entries from global memory.
StageGeom choose_stage(uint32_t plane_words, int planes, uint32_t max_entries, int wbytes,
                       int &stage_entries) {
    StageGeom sg = stage_geom(plane_words, planes, max_entries, wbytes);
    if ((int)smem_for(sg) <= max_smem_per_block()) {
        stage_entries = 1;
        return sg;
    }
    stage_entries = 0;
    return stage_geom(plane_words, planes, 0, wbytes);
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
    d.ny = h->ny; d.nx = h->nx; d.th = L.th; d.tw = L.tw; d.srow = L.srow; d.ntx = L.ntx;
    d.rpw = h->rows_per_warp; d.nseg = L.nseg; d.nrows = h->nrows;
    d.npix = (int64_t)h->ny * h->nx;
    d.n_frames = 1; d.fpi = 1; d.n_groups = 1;
    d.partial = h->partial.p;
    d.norm = h->norm.as<float>();
    d.status = h->status.as<int>();
    d.n_items = L.n_active;
    return d;
}

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

template <class AT, class WT, int MODE, int NIMG, int DT>
int run_phase1(const Inst &single, const Inst *multi, int n_inst, int64_t n_items,
               const StageGeom &sg, cudaStream_t s, Profiler *prof = nullptr) {
    if (n_items <= 0) return AZ_OK;
    const uint32_t smem = smem_for(sg);
    if ((int)smem > max_smem_per_block())
        return fail(AZ_EUNSUPPORTED, "forward: %u bytes of shared memory needed (%d available)",
                    smem, max_smem_per_block());
    auto kern = phase1_kernel<AT, WT, MODE, NIMG, DT>;
    AZ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    AZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::min<int64_t>(n_items, (int64_t)num_sms() * per_sm);
    {
        ProfScope ps(prof, MODE == MODE_FRAMES ? 0 : (MODE == MODE_NORM ? 1 : 2), s);
        kern<<<(unsigned)grid, kThreads, smem, s>>>(single, multi, n_inst, n_items, sg);
    }
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}

template <class AT, int MODE>
int run_phase2(const Inst &single, const Inst *multi, int n_inst, int64_t n_jobs, int n_frames,
               cudaStream_t s, Profiler *prof = nullptr) {
    if (n_jobs <= 0) return AZ_OK;
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

template <class AT, class WT, int MODE, int NIMG>
int run_phase1_dt(int dtype, const Inst &single, const Inst *multi, int n_inst, int64_t n_items,
                  const StageGeom &sg, cudaStream_t s, Profiler *prof = nullptr) {
    switch (dtype) {
        case AZ_DTYPE_F32:
            return run_phase1<AT, WT, MODE, NIMG, AZ_DTYPE_F32>(single, multi, n_inst, n_items, sg, s, prof);
        case AZ_DTYPE_U32:
            return run_phase1<AT, WT, MODE, NIMG, AZ_DTYPE_U32>(single, multi, n_inst, n_items, sg, s, prof);
        default:
            return run_phase1<AT, WT, MODE, NIMG, AZ_DTYPE_I32>(single, multi, n_inst, n_items, sg, s, prof);
    }
}

uint32_t plane_words_of(const az_integrator *h) { return (uint32_t)h->tl.th * h->tl.srow; }

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
                                fp64 ? 8 : 4, d.stage_entries);
    if (fp64) {
        AZ_TRY((run_phase1_dt<double, double, MODE_SINGLE, 1>(dtype, d, nullptr, 1, d.n_items, sg, s, &h->prof)));
        AZ_TRY((run_phase2<double, MODE_SINGLE>(d, nullptr, 1, h->nrows, 1, s, &h->prof)));
    } else {
        AZ_TRY((run_phase1_dt<float, float, MODE_SINGLE, 1>(dtype, d, nullptr, 1, d.n_items, sg, s, &h->prof)));
        AZ_TRY((run_phase2<float, MODE_SINGLE>(d, nullptr, 1, h->nrows, 1, s, &h->prof)));
    }
    return AZ_OK;
}

int batch_norm(az_integrator *h, const float *flat, const float *sa, const float *pol, float *oN,
               float *oC, cudaStream_t s) {
    Inst d = make_inst(h, false);
    d.flat = flat; d.sa = sa; d.pol = pol;
    d.oN = oN; d.oC = oC;
    const int planes = (flat != nullptr) + (sa != nullptr) + (pol != nullptr);
    StageGeom sg = choose_stage(plane_words_of(h), planes, (uint32_t)h->tl.max_tile_entries, 4,
                                d.stage_entries);
    AZ_TRY((run_phase1<float, float, MODE_NORM, 1, AZ_DTYPE_F32>(d, nullptr, 1, d.n_items, sg, s, &h->prof)));
    AZ_TRY((run_phase2<float, MODE_NORM>(d, nullptr, 1, h->nrows, 1, s, &h->prof)));
    return AZ_OK;
}

int batch_frames(az_integrator *h, const void *frames, int n, int dtype, const float *dark,
                 float *oI, float *oS, int frame_out0, cudaStream_t s) {
    const int fpi = h->frames_per_pass;
    const int64_t cap = (int64_t)(h->partial_bytes / (sizeof(float) * (size_t)std::max(h->tl.nseg, 1)));
    const int chunk_max = (int)std::max<int64_t>(fpi, (cap / fpi) * fpi);
    const int planes = fpi + (dark != nullptr);
    int stage_e = 0;
    StageGeom sg = choose_stage(plane_words_of(h), planes, (uint32_t)h->tl.max_tile_entries, 4, stage_e);
    for (int f0 = 0; f0 < n; f0 += chunk_max) {
        const int nf = std::min(chunk_max, n - f0);
        Inst d = make_inst(h, false);
        d.img = static_cast<const char *>(frames) + (size_t)f0 * (size_t)d.npix * 4u;
        d.n_frames = nf; d.fpi = fpi; d.n_groups = (nf + fpi - 1) / fpi;
        d.dark = dark;
        d.oI = oI; d.oS = oS; d.frame_out0 = frame_out0 + f0;
        d.stage_entries = stage_e;
        d.n_items = h->tl.n_active * d.n_groups;
        switch (fpi) {
            case 1: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 1>(dtype, d, nullptr, 1, d.n_items, sg, s, &h->prof))); break;
            case 2: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 2>(dtype, d, nullptr, 1, d.n_items, sg, s, &h->prof))); break;
            case 4: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 4>(dtype, d, nullptr, 1, d.n_items, sg, s, &h->prof))); break;
            default: AZ_TRY((run_phase1_dt<float, float, MODE_FRAMES, 8>(dtype, d, nullptr, 1, d.n_items, sg, s, &h->prof))); break;
        }
        AZ_TRY((run_phase2<float, MODE_FRAMES>(d, nullptr, 1, (int64_t)nf * h->nrows, nf, s, &h->prof)));
    }
    return AZ_OK;
}

int forward_batch(az_integrator *h, const void *frames, int n, int dtype, const float *dark,
                  const float *flat, const float *sa, const float *pol, float *oI, float *oS,
                  float *oN, float *oC, cudaStream_t s) {
    AZ_TRY(batch_norm(h, flat, sa, pol, oN, oC, s));
    return batch_frames(h, frames, n, dtype, dark, oI, oS, 0, s);
}

// ------------------------------------------------------------------------------------
// heterogeneous instances in one persistent launch
// ------------------------------------------------------------------------------------
struct MultiPlan {
    std::vector<Inst> host;
    DevBuf dev;
    int n = 0;
    int dtype = 0;
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
    uint32_t pw = 0, ecap = 0;
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
        d.item_begin = items;
        d.row_begin = rows;
        items += d.n_items;
        rows += h->nrows;
        pw = std::max(pw, plane_words_of(h));
        ecap = std::max(ecap, (uint32_t)h->tl.max_tile_entries);
        planes = std::max(planes, 1 + (d.dark != nullptr) + (d.flat != nullptr) + (d.sa != nullptr) +
                                      (d.pol != nullptr));
        P->host.push_back(d);
    }
    int stage_e = 0;
    P->sg = choose_stage(pw, planes, ecap, 4, stage_e);
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
    AZ_TRY((run_phase1_dt<float, float, MODE_SINGLE, 1>(P->dtype, P->host[0], dev, P->n, P->n_items, P->sg, s)));
    AZ_TRY((run_phase2<float, MODE_SINGLE>(P->host[0], dev, P->n, P->n_rows, 1, s)));
    return AZ_OK;
}

int multi_launch(void *plan, int use_graph, cudaStream_t s) {
    MultiPlan *P = static_cast<MultiPlan *>(plan);
    if (!use_graph) return multi_enqueue(plan, s);
    if (!P->exec) {
        // configure the kernels once outside the capture, then capture the two launches
        AZ_TRY(multi_enqueue(plan, s));
        AZ_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        int rc = multi_enqueue(plan, s);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (rc != AZ_OK) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return fail(AZ_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        P->graph = g;
        AZ_CUDA(cudaGraphInstantiate(&P->exec, g, 0));
        return AZ_OK;  // the eager launch above produced this call's results
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
