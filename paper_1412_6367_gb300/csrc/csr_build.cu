// Sparse bins x pixels matrix build on the device (Sec. 4 pixel splitting, Sec. 5.2
// scatter-to-gather, Sec. 5.2.1 CSR):
//   range (min/max reduction) -> per-pixel entry count -> exclusive scan -> pixel-major fill
//   -> stable LSD radix sort by row -> CSR; then a second stable sort by pixel tile gives the
//   tiled layout the forward kernels stream through shared memory.
//
// Compiled with -fmad=false so that the bin coordinate f = (x - lo) / delta, the bounding-box
// fractions and the azimuth unwrap are rounded exactly as written (they decide integer bin
// indices).  The full-split areas use the line-integral method of Sec. 4.2: the signed area
// of the pixel quadrilateral inside a bin is the sum over its four straight edges of the
// integral of the edge's line function over the bin bounds.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace azint {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr double kKeep2D = 1e-12;  // relative area below which a 2D candidate is dropped

int blocks_for(int64_t n, int per_block) { return (int)((n + per_block - 1) / per_block); }

int grid_stride_blocks(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    return (int)std::max<int64_t>(b, 1);
}

// ------------------------------------------------------------------------------------
// exclusive scan (out[0..n] = prefix sums of in[0..n-1], out[n] = total)
// ------------------------------------------------------------------------------------
template <class T>
__device__ T block_inclusive_scan(T v, T *warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        T x = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < nw) warp_tot[lane] = x;
    }
    __syncthreads();
    if (wid > 0) v += warp_tot[wid - 1];
    __syncthreads();
    return v;
}

template <class T>
__global__ void scan_tiles_kernel(const T *__restrict__ in, T *__restrict__ out, int64_t n_in,
                                  int64_t n_out, T *__restrict__ tile_sums) {
    __shared__ T warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T x[kScanItems];
    T local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        x[k] = (i < n_in) ? in[i] : T(0);
        local += x[k];
    }
    const T incl = block_inclusive_scan<T>(local, warp_tot);
    T run = incl - local;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        if (i < n_out) out[i] = run;
        run += x[k];
    }
    if (threadIdx.x == blockDim.x - 1) tile_sums[blockIdx.x] = incl;
}

template <class T>
__global__ void add_tile_offsets_kernel(T *__restrict__ out, int64_t n_out,
                                        const T *__restrict__ offs) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const T o = offs[blockIdx.x];
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
        const int64_t i = base + k;
        if (i < n_out) out[i] += o;
    }
}

template <class T>
int exclusive_scan_impl(const T *in, T *out, int64_t n, cudaStream_t s) {
    const int64_t n_out = n + 1;
    const int tiles = blocks_for(n_out, kScanTile);
    DevBuf sums, offs;
    AZ_TRY(sums.alloc(sizeof(T) * (tiles + 1)));
    AZ_TRY(offs.alloc(sizeof(T) * (tiles + 1)));
    scan_tiles_kernel<T><<<tiles, kScanThreads, 0, s>>>(in, out, n, n_out, sums.as<T>());
    AZ_CUDA(cudaGetLastError());
    if (tiles > 1) {
        AZ_TRY(exclusive_scan_impl<T>(sums.as<T>(), offs.as<T>(), tiles, s));
        add_tile_offsets_kernel<T><<<tiles, 256, 0, s>>>(out, n_out, offs.as<T>());
        AZ_CUDA(cudaGetLastError());
    }
    return AZ_OK;
}

// ------------------------------------------------------------------------------------
// stable LSD radix sort of (uint32 key, int32 value) pairs, 8-bit digits
// ------------------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsChunks = 8;  // 32-item chunks per warp
constexpr int kRsTile = kRsThreads * kRsChunks;

__global__ void rs_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, int shift,
                               int32_t *__restrict__ hist, int nblocks) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        const int64_t k = base + i;
        if (k < n) atomicAdd(&h[(keys[k] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Each warp owns a contiguous run of kRsChunks * 32 items of the block's tile; items are
// ranked in order with __match_any_sync, so equal keys keep their input order.
__global__ void rs_scatter_kernel(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                  uint32_t *__restrict__ kout, int32_t *__restrict__ vout,
                                  int64_t n, int shift, const int32_t *__restrict__ offs,
                                  int nblocks) {
    __shared__ int wbase[kRsWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRsWarps * 256; d += kRsThreads) (&wbase[0][0])[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)w * (kRsChunks * 32);
    uint32_t key[kRsChunks], dig[kRsChunks];
    int32_t val[kRsChunks];
#pragma unroll
    for (int c = 0; c < kRsChunks; ++c) {
        const int64_t k = base + c * 32 + lane;
        const bool ok = k < n;
        key[c] = ok ? kin[k] : 0u;
        val[c] = ok ? vin[k] : 0;
        dig[c] = ok ? ((key[c] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, dig[c]);
        if (ok && lane == __ffs(peers) - 1) wbase[w][dig[c]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // one digit per thread (256 threads)
        int run = offs[(int64_t)d * nblocks + blockIdx.x];
        for (int ww = 0; ww < kRsWarps; ++ww) {
            const int c = wbase[ww][d];
            wbase[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int c = 0; c < kRsChunks; ++c) {
        const int64_t k = base + c * 32 + lane;
        const bool ok = k < n;
        const unsigned peers = __match_any_sync(0xffffffffu, dig[c]);
        int pos = 0;
        if (ok) pos = wbase[w][dig[c]] + __popc(peers & lt);
        __syncwarp();
        if (ok) {
            kout[pos] = key[c];
            vout[pos] = val[c];
            if (lane == __ffs(peers) - 1) wbase[w][dig[c]] += __popc(peers);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------
// radial range: min / max over unmasked pixels of the positions the split reads
// ------------------------------------------------------------------------------------
__global__ void range_partial_kernel(const double *__restrict__ rad,
                                     const uint8_t *__restrict__ mask, int ny, int nx,
                                     int corners, double *__restrict__ pmin,
                                     double *__restrict__ pmax, int *__restrict__ pcnt) {
    __shared__ double smin[32], smax[32];
    __shared__ int scnt[32];
    double lo = INFINITY, hi = -INFINITY;
    int cnt = 0;
    const int64_t n = (int64_t)ny * nx;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (mask && mask[p]) continue;
        ++cnt;
        if (corners) {
            const int64_t i = p / nx, j = p - i * nx, W = (int64_t)nx + 1;
            const double v[4] = {rad[i * W + j], rad[i * W + j + 1], rad[(i + 1) * W + j + 1],
                                 rad[(i + 1) * W + j]};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                lo = fmin(lo, v[c]);
                hi = fmax(hi, v[c]);
            }
        } else {
            lo = fmin(lo, rad[p]);
            hi = fmax(hi, rad[p]);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) { smin[wid] = lo; smax[wid] = hi; scnt[wid] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            lo = fmin(lo, smin[k]);
            hi = fmax(hi, smax[k]);
            cnt += scnt[k];
        }
        pmin[blockIdx.x] = lo;
        pmax[blockIdx.x] = hi;
        pcnt[blockIdx.x] = cnt;
    }
}

__global__ void range_final_kernel(const double *pmin, const double *pmax, const int *pcnt,
                                   int nb, double *out, int *cnt_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo = INFINITY, hi = -INFINITY;
    long long c = 0;
    for (int k = 0; k < nb; ++k) {
        lo = fmin(lo, pmin[k]);
        hi = fmax(hi, pmax[k]);
        c += pcnt[k];
    }
    out[0] = lo;
    out[1] = hi;
    *cnt_out = (int)c;
}

// ------------------------------------------------------------------------------------
// per-pixel split (the paper's Sec. 4 rules; readings shared with the documented design)
// ------------------------------------------------------------------------------------
struct SplitParams {
    const double *rad;
    const double *chi;
    const uint8_t *mask;
    int ny, nx, npt, nch, split;
    double lo, delta, dchi;
};

__device__ __forceinline__ int bin_none(double f, int npt) {
    const int b = (int)floor(f);
    return b > npt - 1 ? npt - 1 : b;
}

__device__ __forceinline__ void bbox_range(double fmin, double fmax, bool clamp_top, int npt,
                                           int &lo, int &hi) {
    int b0 = (int)floor(fmin);
    if (clamp_top && b0 > npt - 1) b0 = npt - 1;
    int b1 = (int)ceil(fmax) - 1;
    if (b1 < b0) b1 = b0;
    if (clamp_top && b1 > npt - 1) b1 = npt - 1;
    lo = b0;
    hi = b1;
}

__device__ __forceinline__ double bbox_weight(double fmin, double fmax, int blo, int bhi, int b) {
    if (blo == bhi) return 1.0;
    const double span = fmax - fmin;
    if (b == blo) return ((double)(blo + 1) - fmin) / span;
    if (b == bhi) return (fmax - (double)bhi) / span;
    return 1.0 / span;
}

// Azimuth unwrap across +-180 degrees; true when the pixel still spans > 180 degrees.
__device__ __forceinline__ bool unwrap_singular(double c[4]) {
    double mn = c[0], mx = c[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        if (c[k] < mn) mn = c[k];
        if (c[k] > mx) mx = c[k];
    }
    if (mx - mn <= 180.0) return false;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (c[k] < 0.0) c[k] += 360.0;
    mn = c[0];
    mx = c[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        if (c[k] < mn) mn = c[k];
        if (c[k] > mx) mx = c[k];
    }
    return mx - mn > 180.0;
}

// Sec. 4.2: area of the quad (x, y) with x in [lo, hi], as |sum over the four edges of the
// integral of the edge's line function over the clamped edge span|.  An infinite bound
// (outermost bins) is not clamped.
__device__ double slab_area(const double x[4], const double y[4], double lo, double hi,
                            bool lo_inf, bool hi_inf) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double x0 = x[k], y0 = y[k], x1 = x[(k + 1) & 3], y1 = y[(k + 1) & 3];
        if (x0 == x1) continue;
        double u = x0, v = x1;
        if (!lo_inf) { u = fmax(u, lo); v = fmax(v, lo); }
        if (!hi_inf) { u = fmin(u, hi); v = fmin(v, hi); }
        if (u == v) continue;
        const double slope = (y1 - y0) / (x1 - x0);
        const double yu = y0 + (u - x0) * slope;
        const double yv = y0 + (v - x0) * slope;
        s += (v - u) * (yu + yv) * 0.5;
    }
    return fabs(s);
}

// 2D form: area of the quad inside [lo, hi] x [c, d]: the edge integrand is the line
// function clamped to [c, d] (minus c); a clamped line is piecewise linear, so each edge
// contributes (v - u) times the mean of the clamped value over its span.
__device__ double rect_area(const double x[4], const double y[4], double lo, double hi,
                            bool lo_inf, bool hi_inf, double c, double d) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double x0 = x[k], y0 = y[k], x1 = x[(k + 1) & 3], y1 = y[(k + 1) & 3];
        if (x0 == x1) continue;
        double u = x0, v = x1;
        if (!lo_inf) { u = fmax(u, lo); v = fmax(v, lo); }
        if (!hi_inf) { u = fmin(u, hi); v = fmin(v, hi); }
        if (u == v) continue;
        const double slope = (y1 - y0) / (x1 - x0);
        const double yu = y0 + (u - x0) * slope;
        const double yv = y0 + (v - x0) * slope;
        const double p = fmin(yu, yv), q = fmax(yu, yv);
        double mean;
        if (q <= c) {
            continue;
        } else if (p >= d) {
            mean = d - c;
        } else if (q == p) {
            mean = p - c;
        } else {
            const double len = q - p;
            const double below = fmin(fmax((c - p) / len, 0.0), 1.0);
            const double above = fmin(fmax((q - d) / len, 0.0), 1.0);
            const double mid = 1.0 - below - above;
            mean = above * (d - c) + mid * (0.5 * (fmax(p, c) + fmin(q, d)) - c);
        }
        s += (v - u) * mean;
    }
    return fabs(s);
}

__device__ __forceinline__ void corner_ids(int nx, int64_t i, int64_t j, int64_t k[4]) {
    const int64_t W = (int64_t)nx + 1;
    k[0] = i * W + j;
    k[1] = i * W + j + 1;
    k[2] = (i + 1) * W + j + 1;
    k[3] = (i + 1) * W + j;
}

template <class Emit>
__device__ void visit_1d(const SplitParams &P, int64_t p, Emit &emit) {
    if (P.split == AZ_SPLIT_NONE) {
        const double f = (P.rad[p] - P.lo) / P.delta;
        emit(bin_none(f, P.npt), 1.0);
        return;
    }
    const int64_t i = p / P.nx, j = p - i * P.nx;
    int64_t k[4];
    corner_ids(P.nx, i, j, k);
    double f[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) f[c] = (P.rad[k[c]] - P.lo) / P.delta;
    double fmin = f[0], fmax = f[0];
#pragma unroll
    for (int c = 1; c < 4; ++c) {
        if (f[c] < fmin) fmin = f[c];
        if (f[c] > fmax) fmax = f[c];
    }
    int blo, bhi;
    bbox_range(fmin, fmax, true, P.npt, blo, bhi);
    bool use_bbox = P.split == AZ_SPLIT_BBOX || blo == bhi;
    double x[4], y[4], total = 0.0;
    if (!use_bbox) {
        double ch[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) ch[c] = P.chi[k[c]];
        if (unwrap_singular(ch)) {
            use_bbox = true;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                x[c] = f[c] - f[0];
                y[c] = ch[c] - ch[0];
            }
            for (int b = blo; b <= bhi; ++b)
                total += slab_area(x, y, (double)b - f[0], (double)(b + 1) - f[0], b == 0,
                                   b == P.npt - 1);
            if (!(total > 0.0)) use_bbox = true;
        }
    }
    for (int b = blo; b <= bhi; ++b) {
        double w;
        if (use_bbox)
            w = bbox_weight(fmin, fmax, blo, bhi, b);
        else
            w = slab_area(x, y, (double)b - f[0], (double)(b + 1) - f[0], b == 0,
                          b == P.npt - 1) / total;
        emit(b, w);
    }
}

template <class Emit>
__device__ void visit_2d(const SplitParams &P, int64_t p, Emit &emit) {
    const int npt = P.npt, nch = P.nch;
    if (P.split == AZ_SPLIT_NONE) {
        const double f = (P.rad[p] - P.lo) / P.delta;
        const double g = (P.chi[p] + 180.0) / P.dchi;
        const int kc = ((int)floor(g)) % nch;
        emit(kc * npt + bin_none(f, npt), 1.0);
        return;
    }
    const int64_t i = p / P.nx, j = p - i * P.nx;
    int64_t k[4];
    corner_ids(P.nx, i, j, k);
    double f[4], ch[4], g[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        f[c] = (P.rad[k[c]] - P.lo) / P.delta;
        ch[c] = P.chi[k[c]];
    }
    const bool singular = unwrap_singular(ch);
#pragma unroll
    for (int c = 0; c < 4; ++c) g[c] = (ch[c] + 180.0) / P.dchi;
    double fmin = f[0], fmax = f[0], gmin = g[0], gmax = g[0];
#pragma unroll
    for (int c = 1; c < 4; ++c) {
        if (f[c] < fmin) fmin = f[c];
        if (f[c] > fmax) fmax = f[c];
        if (g[c] < gmin) gmin = g[c];
        if (g[c] > gmax) gmax = g[c];
    }
    int blo, bhi, klo, khi;
    bbox_range(fmin, fmax, true, npt, blo, bhi);
    bbox_range(gmin, gmax, false, nch, klo, khi);
    const int nc = khi - klo + 1;
    const int nres = nc < nch ? nc : nch;  // distinct chi bins after the modulo
    if (singular) {
        for (int b = blo; b <= bhi; ++b) {
            const double wr = bbox_weight(fmin, fmax, blo, bhi, b);
            for (int kc = 0; kc < nch; ++kc) emit(kc * npt + b, wr / (double)nch);
        }
        return;
    }
    bool use_bbox = P.split == AZ_SPLIT_BBOX;
    if (!use_bbox) {
        double x[4], y[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            x[c] = f[c] - f[0];
            y[c] = g[c] - g[0];
        }
        double total = 0.0;
        for (int b = blo; b <= bhi; ++b)
            for (int kc = klo; kc <= khi; ++kc)
                total += rect_area(x, y, (double)b - f[0], (double)(b + 1) - f[0], b == 0,
                                   b == npt - 1, (double)kc - g[0], (double)(kc + 1) - g[0]);
        if (total > 0.0) {
            const double thr = kKeep2D * total;
            double kept = 0.0;
            for (int b = blo; b <= bhi; ++b)
                for (int kc = klo; kc <= khi; ++kc) {
                    const double a = rect_area(x, y, (double)b - f[0], (double)(b + 1) - f[0],
                                               b == 0, b == npt - 1, (double)kc - g[0],
                                               (double)(kc + 1) - g[0]);
                    if (a > thr) kept += a;
                }
            for (int b = blo; b <= bhi; ++b)
                for (int r = 0; r < nres; ++r) {
                    double w = 0.0;
                    bool any = false;
                    for (int kc = klo + r; kc <= khi; kc += nch) {
                        const double a = rect_area(x, y, (double)b - f[0], (double)(b + 1) - f[0],
                                                   b == 0, b == npt - 1, (double)kc - g[0],
                                                   (double)(kc + 1) - g[0]);
                        if (a > thr) {
                            w += a / kept;
                            any = true;
                        }
                    }
                    if (any) emit(((klo + r) % nch) * npt + b, w);
                }
            return;
        }
        use_bbox = true;  // degenerate quad
    }
    for (int b = blo; b <= bhi; ++b) {
        const double wr = bbox_weight(fmin, fmax, blo, bhi, b);
        for (int r = 0; r < nres; ++r) {
            double w = 0.0;
            for (int kc = klo + r; kc <= khi; kc += nch)
                w += wr * bbox_weight(gmin, gmax, klo, khi, kc);
            emit(((klo + r) % nch) * npt + b, w);
        }
    }
}

struct CountEmit {
    int64_t n = 0;
    __device__ void operator()(int, double) { ++n; }
};

struct FillEmit {
    int64_t pos;
    int32_t pix;
    int32_t *row;
    double *w64;
    int32_t *pixel;
    __device__ void operator()(int r, double w) {
        row[pos] = r;
        w64[pos] = w;
        pixel[pos] = pix;
        ++pos;
    }
};

__global__ void count_kernel(SplitParams P, int64_t *__restrict__ count) {
    const int64_t n = (int64_t)P.ny * P.nx;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (P.mask && P.mask[p]) {
            count[p] = 0;
            continue;
        }
        CountEmit e;
        if (P.nch > 0) visit_2d(P, p, e); else visit_1d(P, p, e);
        count[p] = e.n;
    }
}

__global__ void fill_kernel(SplitParams P, const int64_t *__restrict__ ptr,
                            int32_t *__restrict__ row, double *__restrict__ w64,
                            int32_t *__restrict__ pixel) {
    const int64_t n = (int64_t)P.ny * P.nx;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (P.mask && P.mask[p]) continue;
        FillEmit e{ptr[p], (int32_t)p, row, w64, pixel};
        if (P.nch > 0) visit_2d(P, p, e); else visit_1d(P, p, e);
    }
}

// ------------------------------------------------------------------------------------
// small element-wise kernels
// ------------------------------------------------------------------------------------
__global__ void iota_kernel(int32_t *v, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        v[k] = (int32_t)k;
}

__global__ void to_u32_kernel(const int32_t *in, uint32_t *out, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (uint32_t)in[k];
}

__global__ void i64_to_i32_kernel(const int64_t *in, int32_t *out, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (int32_t)in[k];
}

__global__ void count_keys_kernel(const int32_t *__restrict__ key, int64_t n,
                                  int32_t *__restrict__ cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[key[k]], 1);
}

__global__ void csr_gather_kernel(const int32_t *__restrict__ perm, const int32_t *__restrict__ pix,
                                  const double *__restrict__ w, int32_t *__restrict__ idx_out,
                                  double *__restrict__ w_out, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = perm[k];
        idx_out[k] = pix[e];
        w_out[k] = w[e];
    }
}

__global__ void f64_to_f32_kernel(const double *in, float *out, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (float)in[k];
}

// Row of each CSR entry (upper bound in indptr).
__global__ void csr_rows_kernel(const int32_t *__restrict__ ptr, int nrows, int64_t nnz,
                                int32_t *__restrict__ row) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nrows;  // find the last r with ptr[r] <= k
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ptr[mid] <= k) lo = mid; else hi = mid;
        }
        row[k] = lo;
    }
}

// Pixels with at least one entry (column pointers ptr[npix + 1]).
__global__ void nonempty_kernel(const int32_t *__restrict__ ptr, int64_t n, int *__restrict__ count) {
    int c = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        c += ptr[p + 1] > ptr[p];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

struct TileGeom {
    int nx, th, tw, srow, ss, ntx;
};

__device__ __forceinline__ int tile_of(const TileGeom &T, int32_t p) {
    const int i = p / T.nx, j = p - (p / T.nx) * T.nx;
    return (i / T.th) * T.ntx + j / T.tw;
}

// Shared-memory word offset of pixel p inside its staged tile.  Tile rows are grouped by
// their index modulo 4 into four 128-byte aligned slots of `ss` words: rows ly = 4 jj + s sit
// in slot s at pitch srow = tw + 20, starting c_s = (nx * s) mod 4 words into the row.  This
// is where one 2D copy per row class (rows of equal index mod 4 are 16 * nx bytes apart, a
// multiple of 16) puts them; the copy adds a per-plane shift of 0..15 words that depends only
// on the plane (base address, first row, plane index), so the offset below is the same for
// every frame.
__device__ __forceinline__ int tile_loc(const TileGeom &T, int32_t p) {
    const int i = p / T.nx, j = p - i * T.nx;
    const int ti = i / T.th, tj = j / T.tw;
    const int ly = i - ti * T.th, lx = j - tj * T.tw;
    const int sl = ly & 3, jj = ly >> 2;
    const int cs = ((T.nx & 3) * sl) & 3;
    return sl * T.ss + cs + jj * T.srow + lx;
}

// Offsets of the padded entries in the frame-pair layout (geometry Tp): the same formula at
// the pair layout's row pitch and slot stride; padding entries read the zero band at 4 ss.
__global__ void pair_loc_kernel(TileGeom Tp, const int32_t *__restrict__ pix, int64_t n,
                                uint16_t *__restrict__ loc) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = pix[e];
        loc[e] = (uint16_t)(p >= 0 ? tile_loc(Tp, p) : 4 * Tp.ss);
    }
}

__global__ void tile_keys_kernel(TileGeom T, const int32_t *__restrict__ idx, int64_t n,
                                 uint32_t *__restrict__ key) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        key[k] = (uint32_t)tile_of(T, idx[k]);
}

// Per segment (flagged first entry e, segment id s): first entry, row and tile.
__global__ void seg_info_kernel(const int32_t *__restrict__ flag, const int32_t *__restrict__ segid,
                                const int32_t *__restrict__ perm, const int32_t *__restrict__ csr_row,
                                const uint32_t *__restrict__ tkey, int64_t n,
                                int32_t *__restrict__ first, int32_t *__restrict__ row,
                                int32_t *__restrict__ tile) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[e]) continue;
        const int32_t s = segid[e];
        first[s] = (int32_t)e;
        row[s] = csr_row[perm[e]];
        tile[s] = (int32_t)tkey[e];
    }
}

// Segment lengths rounded up to whole quads of entries.
__global__ void quad_len_kernel(const int32_t *__restrict__ len, int64_t n, int32_t *__restrict__ plen) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        plen[k] = (len[k] + 3) & ~3;
}

// Padded entries of a tile: its segments' quad-rounded lengths, rounded up to 8.
__global__ void tile_pad_kernel(const int32_t *__restrict__ tile_seg_ptr, const int32_t *__restrict__ pstart,
                                int ntiles, int32_t *__restrict__ tpad) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles;
         t += (int64_t)gridDim.x * blockDim.x)
        tpad[t] = (pstart[tile_seg_ptr[t + 1]] - pstart[tile_seg_ptr[t]] + 7) & ~7;
}

// Padded start and end of every segment.
__global__ void seg_span_kernel(const int32_t *__restrict__ seg_tile, const int32_t *__restrict__ pstart,
                                const int32_t *__restrict__ plen, const int32_t *__restrict__ tile_seg_ptr,
                                const int32_t *__restrict__ tile_ent_ptr, int nseg,
                                int32_t *__restrict__ start, int32_t *__restrict__ end) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int t = seg_tile[s];
        const int32_t a = tile_ent_ptr[t] + pstart[s] - pstart[tile_seg_ptr[t]];
        start[s] = a;
        end[s] = a + plen[s];
    }
}

__global__ void fill_u16_kernel(uint16_t *__restrict__ out, int64_t n, uint16_t v) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = v;
}

// Tile key of each entry of a permuted entry list.
__global__ void tile_keys_perm_kernel(TileGeom T, const int32_t *__restrict__ idx,
                                      const int32_t *__restrict__ perm, int64_t n,
                                      uint32_t *__restrict__ key) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        key[k] = (uint32_t)tile_of(T, idx[perm[k]]);
}

// Segment of each entry from the segment-start flags and their exclusive scan.
__global__ void seg_index_kernel(const int32_t *__restrict__ flag, const int32_t *__restrict__ segid,
                                 int64_t n, int32_t *__restrict__ seg) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        seg[e] = segid[e] - 1 + flag[e];
}

// Sort key putting the longer segments of a tile first: max_len - length of the segment.
__global__ void seg_len_key_kernel(const int32_t *__restrict__ seg, const int32_t *__restrict__ len,
                                   int32_t max_len, int64_t n, uint32_t *__restrict__ key) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        key[e] = (uint32_t)(max_len - len[seg[e]]);
}


__global__ void seg_flags_kernel(const uint32_t *__restrict__ tkey, const int32_t *__restrict__ perm,
                                 const int32_t *__restrict__ csr_row, int64_t n,
                                 int32_t *__restrict__ flag) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int f = 1;
        if (e > 0) f = (tkey[e] != tkey[e - 1]) || (csr_row[perm[e]] != csr_row[perm[e - 1]]);
        flag[e] = f;
    }
}

struct TiledFillArgs {
    TileGeom T;
    const int32_t *perm, *csr_idx;
    const double *csr_w;
    const int32_t *segx, *seg_first, *seg_start;
    uint16_t *loc;
    int32_t *pix;
    float *w32;
    double *w64;
    int64_t n;
};

__global__ void tiled_fill_kernel(TiledFillArgs A) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A.n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = A.segx[e];
        const int64_t pe = (int64_t)A.seg_start[s] + (e - A.seg_first[s]);
        const int32_t k = A.perm[e];
        const int32_t p = A.csr_idx[k];
        A.loc[pe] = (uint16_t)tile_loc(A.T, p);
        const double w = A.csr_w[k];
        A.w64[pe] = w;
        A.w32[pe] = (float)w;
        A.pix[pe] = p;
    }
}

__global__ void scatter_slots_kernel(const int32_t *__restrict__ perm, int nseg,
                                     int32_t *__restrict__ slot) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
         s += (int64_t)gridDim.x * blockDim.x)
        slot[perm[s]] = (int32_t)s;
}

__global__ void max_kernel(const int32_t *a, int n, int32_t *out) {
    __shared__ int32_t sm[32];
    int32_t m = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) m = max(m, a[k]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = max(m, sm[k]);
        *out = m;
    }
}

__global__ void diff_kernel(const int32_t *ptr, int n, int32_t *out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        out[t] = ptr[t + 1] - ptr[t];
}

// Work items: a tile's segments (longest first) cut into runs whose entries, counted from
// the run's first entry rounded down to a multiple of 8, stay within `cap` (a single longer
// segment makes an item of its own).  One thread per tile; `fill` = 0 counts the items,
// 1 writes (tile, first segment, end segment) for each.
__global__ void chunk_kernel(const int32_t *__restrict__ tile_seg_ptr, const int32_t *__restrict__ seg_start,
                             const int32_t *__restrict__ seg_end, int ntiles, int cap, int fill,
                             int32_t *__restrict__ count, const int32_t *__restrict__ offs,
                             int32_t *__restrict__ chunks) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s0 = tile_seg_ptr[t], s1 = tile_seg_ptr[t + 1];
        int n = 0, i = s0;
        while (i < s1) {
            const int e0 = seg_start[i] & ~7;
            int j = i + 1;
            while (j < s1 && seg_end[j] - e0 <= cap) ++j;
            if (fill) {
                int32_t *c = chunks + 3 * (size_t)(offs[t] + n);
                c[0] = (int32_t)t; c[1] = i; c[2] = j;
            }
            ++n;
            i = j;
        }
        if (!fill) count[t] = n;
    }
}

// Record size (int32 words, multiple of 4) of one work item.
__global__ void rec_words_kernel(const int32_t *__restrict__ chunks, int n_items, int32_t *__restrict__ words) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_items;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int ns = chunks[3 * a + 2] - chunks[3 * a + 1];
        const int w = 4 + ns + (ns + 2) / 2;  // header, slots, uint16 starts[ns + 1]
        words[a] = (w + 3) & ~3;
    }
}

// Record {tile, ns, first entry, entries, slots[ns], uint16 starts[ns + 1]} and descriptor
// {tile, record offset, record words, first entry, entries, ns} of one work item.  The
// item's entries start at its first segment rounded down to a multiple of 8 entries (16-byte
// aligned locations for the bulk copy) and end at its last segment's end rounded up to 8.
__global__ void rec_fill_kernel(const int32_t *__restrict__ chunks, int n_items,
                                const int32_t *__restrict__ seg_start, const int32_t *__restrict__ seg_end,
                                const int32_t *__restrict__ seg_slot, const int32_t *__restrict__ rec_off,
                                int32_t *__restrict__ rec, int32_t *__restrict__ desc,
                                int32_t *__restrict__ item_entries, int32_t *__restrict__ item_segments) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_items;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int t = chunks[3 * a], s0 = chunks[3 * a + 1], ns = chunks[3 * a + 2] - s0;
        const int e0 = seg_start[s0] & ~7;
        const int ne = ((seg_end[s0 + ns - 1] - e0) + 7) & ~7;
        const int off = rec_off[a], words = rec_off[a + 1] - off;
        int32_t *r = rec + off;
        r[0] = t; r[1] = ns; r[2] = e0; r[3] = ne;
        for (int i = 0; i < ns; ++i) r[4 + i] = seg_slot[s0 + i];
        uint16_t *st = reinterpret_cast<uint16_t *>(r + 4 + ns);
        for (int i = 0; i < ns; ++i) st[i] = (uint16_t)(seg_start[s0 + i] - e0);
        st[ns] = (uint16_t)(seg_end[s0 + ns - 1] - e0);
        for (int k = 4 + ns + (ns + 2) / 2; k < words; ++k) r[k] = 0;
        int32_t *dd = desc + 8 * a;
        dd[0] = t; dd[1] = off; dd[2] = words; dd[3] = e0;
        dd[4] = ne; dd[5] = ns; dd[6] = 0; dd[7] = 0;
        item_entries[a] = ne;
        item_segments[a] = ns;
    }
}

int bits_for(int64_t maxval) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) <= maxval) ++b;
    return b;
}

template <class K, class... Args>
int launch_gs(K kernel, int64_t n, cudaStream_t s, Args... args) {
    kernel<<<grid_stride_blocks(n, 256), 256, 0, s>>>(args...);
    AZ_CUDA(cudaGetLastError());
    return AZ_OK;
}

}  // namespace

int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return exclusive_scan_impl<int64_t>(in, out, n, s);
}
int exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    return exclusive_scan_impl<int32_t>(in, out, n, s);
}

int stable_sort_pairs(uint32_t *keys, int32_t *vals, int64_t n, int key_bits, cudaStream_t s) {
    if (n <= 1) return AZ_OK;
    const int nblocks = blocks_for(n, kRsTile);
    DevBuf k2, v2, hist, offs;
    AZ_TRY(k2.alloc(sizeof(uint32_t) * n));
    AZ_TRY(v2.alloc(sizeof(int32_t) * n));
    AZ_TRY(hist.alloc(sizeof(int32_t) * 256 * (size_t)nblocks));
    AZ_TRY(offs.alloc(sizeof(int32_t) * (256 * (size_t)nblocks + 1)));
    uint32_t *ka = keys, *kb = k2.as<uint32_t>();
    int32_t *va = vals, *vb = v2.as<int32_t>();
    const int passes = (key_bits + 7) / 8;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        rs_hist_kernel<<<nblocks, kRsThreads, 0, s>>>(ka, n, shift, hist.as<int32_t>(), nblocks);
        AZ_CUDA(cudaGetLastError());
        AZ_TRY(exclusive_scan_i32(hist.as<int32_t>(), offs.as<int32_t>(), 256 * (int64_t)nblocks, s));
        rs_scatter_kernel<<<nblocks, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift,
                                                         offs.as<int32_t>(), nblocks);
        AZ_CUDA(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        AZ_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        AZ_CUDA(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    AZ_CUDA(cudaStreamSynchronize(s));  // k2/v2 are freed on return
    return AZ_OK;
}

int build_integrator(int ny, int nx, const double *rad, const double *chi, int npt_rad,
                     int npt_azim, int unit, int split, const uint8_t *mask, cudaStream_t s,
                     az_integrator *h) {
    const int64_t npix = (int64_t)ny * nx;
    const int corners = split != AZ_SPLIT_NONE;

    // 1. radial range over unmasked pixels
    const int rb = std::min<int64_t>(grid_stride_blocks(npix, 256), 1024);
    DevBuf pmin, pmax, pcnt, rng, rcnt;
    AZ_TRY(pmin.alloc(sizeof(double) * rb));
    AZ_TRY(pmax.alloc(sizeof(double) * rb));
    AZ_TRY(pcnt.alloc(sizeof(int) * rb));
    AZ_TRY(rng.alloc(sizeof(double) * 2));
    AZ_TRY(rcnt.alloc(sizeof(int)));
    range_partial_kernel<<<rb, 256, 0, s>>>(rad, mask, ny, nx, corners, pmin.as<double>(),
                                            pmax.as<double>(), pcnt.as<int>());
    AZ_CUDA(cudaGetLastError());
    range_final_kernel<<<1, 32, 0, s>>>(pmin.as<double>(), pmax.as<double>(), pcnt.as<int>(), rb,
                                        rng.as<double>(), rcnt.as<int>());
    AZ_CUDA(cudaGetLastError());
    double lohi[2];
    int unmasked = 0;
    AZ_CUDA(cudaMemcpyAsync(lohi, rng.p, sizeof(lohi), cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaMemcpyAsync(&unmasked, rcnt.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    if (unmasked == 0) return fail(AZ_ERANGE, "csr_build: every pixel is masked");
    if (!(lohi[1] > lohi[0]) || !std::isfinite(lohi[0]) || !std::isfinite(lohi[1]))
        return fail(AZ_ERANGE, "csr_build: empty radial range [%g, %g]", lohi[0], lohi[1]);

    h->ny = ny; h->nx = nx; h->npt_rad = npt_rad; h->npt_azim = npt_azim;
    h->nrows = npt_azim > 0 ? npt_rad * npt_azim : npt_rad;
    h->unit = unit; h->split = split; h->n_unmasked = unmasked;
    h->lo = lohi[0]; h->hi = lohi[1];
    h->delta = (h->hi - h->lo) / npt_rad;

    SplitParams P;
    P.rad = rad; P.chi = chi; P.mask = mask; P.ny = ny; P.nx = nx; P.npt = npt_rad;
    P.nch = npt_azim; P.split = split; P.lo = h->lo; P.delta = h->delta;
    P.dchi = npt_azim > 0 ? 360.0 / npt_azim : 0.0;

    // 2. per-pixel counts -> 3. exclusive scan
    DevBuf cnt, ptr64;
    AZ_TRY(cnt.alloc(sizeof(int64_t) * npix));
    AZ_TRY(ptr64.alloc(sizeof(int64_t) * (npix + 1)));
    AZ_TRY(launch_gs(count_kernel, npix, s, P, cnt.as<int64_t>()));
    AZ_TRY(exclusive_scan_i64(cnt.as<int64_t>(), ptr64.as<int64_t>(), npix, s));
    int64_t nnz = 0;
    AZ_CUDA(cudaMemcpyAsync(&nnz, ptr64.as<int64_t>() + npix, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    if (nnz > INT32_MAX) return fail(AZ_EOVERFLOW, "csr_build: %lld entries exceed 2^31 - 1", (long long)nnz);
    if (nnz == 0) return fail(AZ_ERANGE, "csr_build: the matrix has no entries");
    h->nnz = nnz;
    cnt.release();

    // 4. pixel-major fill (the "scatter" view, kept as the CSC for the adjoint)
    AZ_TRY(h->csc_ptr.alloc(sizeof(int32_t) * (npix + 1)));
    AZ_TRY(h->csc_row.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(h->csc_w64.alloc(sizeof(double) * nnz));
    AZ_TRY(h->csc_w32.alloc(sizeof(float) * nnz));
    DevBuf pix;
    AZ_TRY(pix.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(launch_gs(fill_kernel, npix, s, P, ptr64.as<int64_t>(), h->csc_row.as<int32_t>(),
                     h->csc_w64.as<double>(), pix.as<int32_t>()));
    AZ_TRY(launch_gs(i64_to_i32_kernel, npix + 1, s, ptr64.as<int64_t>(), h->csc_ptr.as<int32_t>(),
                     npix + 1));
    AZ_TRY(launch_gs(f64_to_f32_kernel, nnz, s, h->csc_w64.as<double>(), h->csc_w32.as<float>(), nnz));
    ptr64.release();

    // 5. stable sort by row -> CSR (the "gather" view, rows ascending by pixel)
    DevBuf keys, perm, rowcnt;
    AZ_TRY(keys.alloc(sizeof(uint32_t) * nnz));
    AZ_TRY(perm.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(launch_gs(to_u32_kernel, nnz, s, h->csc_row.as<int32_t>(), keys.as<uint32_t>(), nnz));
    AZ_TRY(launch_gs(iota_kernel, nnz, s, perm.as<int32_t>(), nnz));
    AZ_TRY(stable_sort_pairs(keys.as<uint32_t>(), perm.as<int32_t>(), nnz, bits_for(h->nrows - 1), s));
    AZ_TRY(h->csr_ptr.alloc(sizeof(int32_t) * (h->nrows + 1)));
    AZ_TRY(h->csr_idx.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(h->csr_w64.alloc(sizeof(double) * nnz));
    AZ_TRY(launch_gs(csr_gather_kernel, nnz, s, perm.as<int32_t>(), pix.as<int32_t>(),
                     h->csc_w64.as<double>(), h->csr_idx.as<int32_t>(), h->csr_w64.as<double>(), nnz));
    AZ_TRY(rowcnt.alloc(sizeof(int32_t) * h->nrows));
    AZ_CUDA(cudaMemsetAsync(rowcnt.p, 0, sizeof(int32_t) * h->nrows, s));
    AZ_TRY(launch_gs(count_keys_kernel, nnz, s, h->csc_row.as<int32_t>(), nnz, rowcnt.as<int32_t>()));
    AZ_TRY(exclusive_scan_i32(rowcnt.as<int32_t>(), h->csr_ptr.as<int32_t>(), h->nrows, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    return AZ_OK;
}

// The integrator's matrix from a host CSR (already checked by the caller): the CSR copied to
// the device, the pixel-major CSC formed by a stable sort of the entries by pixel (so each
// pixel's entries keep ascending row order), and the count of pixels that have entries.
int import_csr(az_integrator *h, const int32_t *indptr, const int32_t *indices, const double *data,
               cudaStream_t s) {
    const int64_t npix = (int64_t)h->ny * h->nx, nnz = h->nnz;
    AZ_TRY(h->csr_ptr.alloc(sizeof(int32_t) * (h->nrows + 1)));
    AZ_TRY(h->csr_idx.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(h->csr_w64.alloc(sizeof(double) * nnz));
    AZ_CUDA(cudaMemcpyAsync(h->csr_ptr.p, indptr, sizeof(int32_t) * (h->nrows + 1), cudaMemcpyHostToDevice, s));
    AZ_CUDA(cudaMemcpyAsync(h->csr_idx.p, indices, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
    AZ_CUDA(cudaMemcpyAsync(h->csr_w64.p, data, sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    DevBuf rows, keys, perm, cnt, nonempty;
    AZ_TRY(rows.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(keys.alloc(sizeof(uint32_t) * nnz));
    AZ_TRY(perm.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(launch_gs(csr_rows_kernel, nnz, s, h->csr_ptr.as<int32_t>(), h->nrows, nnz, rows.as<int32_t>()));
    AZ_TRY(launch_gs(to_u32_kernel, nnz, s, h->csr_idx.as<int32_t>(), keys.as<uint32_t>(), nnz));
    AZ_TRY(launch_gs(iota_kernel, nnz, s, perm.as<int32_t>(), nnz));
    AZ_TRY(stable_sort_pairs(keys.as<uint32_t>(), perm.as<int32_t>(), nnz, bits_for(npix - 1), s));
    AZ_TRY(h->csc_ptr.alloc(sizeof(int32_t) * (npix + 1)));
    AZ_TRY(h->csc_row.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(h->csc_w64.alloc(sizeof(double) * nnz));
    AZ_TRY(h->csc_w32.alloc(sizeof(float) * nnz));
    AZ_TRY(launch_gs(csr_gather_kernel, nnz, s, perm.as<int32_t>(), rows.as<int32_t>(), h->csr_w64.as<double>(),
                     h->csc_row.as<int32_t>(), h->csc_w64.as<double>(), nnz));
    AZ_TRY(launch_gs(f64_to_f32_kernel, nnz, s, h->csc_w64.as<double>(), h->csc_w32.as<float>(), nnz));
    AZ_TRY(cnt.alloc(sizeof(int32_t) * npix));
    AZ_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * npix, s));
    AZ_TRY(launch_gs(count_keys_kernel, nnz, s, h->csr_idx.as<int32_t>(), nnz, cnt.as<int32_t>()));
    AZ_TRY(exclusive_scan_i32(cnt.as<int32_t>(), h->csc_ptr.as<int32_t>(), npix, s));
    AZ_TRY(nonempty.alloc(sizeof(int)));
    AZ_CUDA(cudaMemsetAsync(nonempty.p, 0, sizeof(int), s));
    AZ_TRY(launch_gs(nonempty_kernel, npix, s, h->csc_ptr.as<int32_t>(), npix, nonempty.as<int>()));
    int n_unmasked = 0;
    AZ_CUDA(cudaMemcpyAsync(&n_unmasked, nonempty.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    h->n_unmasked = n_unmasked;
    return AZ_OK;
}

int build_tiled_layout(az_integrator *h, int th, int tw, cudaStream_t s) {
    TiledLayout &L = h->tl;
    h->count_ready = false;  // the accumulation order of C depends on the layout
    h->corr_bound = false;   // bound corrections are per layout too (entry order, sums)
    const int64_t nnz = h->nnz;
    if (th < 4 || (th % 4) != 0 || tw < 4 || (tw % 4) != 0)
        return fail(AZ_EINVAL, "tile %dx%d: both sides must be positive multiples of 4", th, tw);
    TileGeom T;
    T.nx = h->nx; T.th = th; T.tw = tw; T.srow = tw + 20;
    T.ss = ((th / 4) * T.srow + 31) & ~31;
    T.ntx = (h->nx + tw - 1) / tw;
    const int nty = (h->ny + th - 1) / th;
    const int ntiles = T.ntx * nty;
    if ((int64_t)4 * T.ss + 32 > 65535) return fail(AZ_EINVAL, "tile %dx%d too large", th, tw);

    // row of each CSR entry, tile key of each CSR entry, stable sort by tile
    DevBuf csr_row, tkey, perm;
    AZ_TRY(csr_row.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(tkey.alloc(sizeof(uint32_t) * nnz));
    AZ_TRY(perm.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(launch_gs(csr_rows_kernel, nnz, s, h->csr_ptr.as<int32_t>(), h->nrows, nnz,
                     csr_row.as<int32_t>()));
    AZ_TRY(launch_gs(tile_keys_kernel, nnz, s, T, h->csr_idx.as<int32_t>(), nnz, tkey.as<uint32_t>()));
    AZ_TRY(launch_gs(iota_kernel, nnz, s, perm.as<int32_t>(), nnz));
    AZ_TRY(stable_sort_pairs(tkey.as<uint32_t>(), perm.as<int32_t>(), nnz, bits_for(ntiles - 1), s));
    {
        // Within a tile, order the segments (runs of one row) by decreasing length, rows in
        // increasing order among equal lengths; the entries of a segment keep pixel order.
        // Warps that take consecutive segments then get runs of similar length.
        DevBuf f0, id0, seg0, len0, mx0, key2;
        AZ_TRY(f0.alloc(sizeof(int32_t) * nnz));
        AZ_TRY(id0.alloc(sizeof(int32_t) * (nnz + 1)));
        AZ_TRY(seg0.alloc(sizeof(int32_t) * nnz));
        AZ_TRY(launch_gs(seg_flags_kernel, nnz, s, tkey.as<uint32_t>(), perm.as<int32_t>(),
                         csr_row.as<int32_t>(), nnz, f0.as<int32_t>()));
        AZ_TRY(exclusive_scan_i32(f0.as<int32_t>(), id0.as<int32_t>(), nnz, s));
        int32_t nseg0 = 0;
        AZ_CUDA(cudaMemcpyAsync(&nseg0, id0.as<int32_t>() + nnz, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AZ_CUDA(cudaStreamSynchronize(s));
        AZ_TRY(launch_gs(seg_index_kernel, nnz, s, f0.as<int32_t>(), id0.as<int32_t>(), nnz,
                         seg0.as<int32_t>()));
        AZ_TRY(len0.alloc(sizeof(int32_t) * std::max(nseg0, 1)));
        AZ_CUDA(cudaMemsetAsync(len0.p, 0, sizeof(int32_t) * std::max(nseg0, 1), s));
        AZ_TRY(launch_gs(count_keys_kernel, nnz, s, seg0.as<int32_t>(), nnz, len0.as<int32_t>()));
        AZ_TRY(mx0.alloc(sizeof(int32_t)));
        max_kernel<<<1, 1024, 0, s>>>(len0.as<int32_t>(), nseg0, mx0.as<int32_t>());
        AZ_CUDA(cudaGetLastError());
        int32_t max_len = 0;
        AZ_CUDA(cudaMemcpyAsync(&max_len, mx0.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AZ_CUDA(cudaStreamSynchronize(s));
        AZ_TRY(key2.alloc(sizeof(uint32_t) * nnz));
        AZ_TRY(launch_gs(seg_len_key_kernel, nnz, s, seg0.as<int32_t>(), len0.as<int32_t>(), max_len,
                         nnz, key2.as<uint32_t>()));
        AZ_TRY(stable_sort_pairs(key2.as<uint32_t>(), perm.as<int32_t>(), nnz, bits_for(max_len), s));
        AZ_TRY(launch_gs(tile_keys_perm_kernel, nnz, s, T, h->csr_idx.as<int32_t>(), perm.as<int32_t>(),
                         nnz, tkey.as<uint32_t>()));
        AZ_TRY(stable_sort_pairs(tkey.as<uint32_t>(), perm.as<int32_t>(), nnz, bits_for(ntiles - 1), s));
    }

    // Segments (runs of one row inside a tile) in the final entry order.  Each segment is
    // padded to whole quads of entries with dummy entries of weight 0 whose location is the
    // zero band after every staged plane (pixel -1), so that reductions read whole quads only.
    DevBuf flag, segid, segx;
    AZ_TRY(flag.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(segid.alloc(sizeof(int32_t) * (nnz + 1)));
    AZ_TRY(segx.alloc(sizeof(int32_t) * nnz));
    AZ_TRY(launch_gs(seg_flags_kernel, nnz, s, tkey.as<uint32_t>(), perm.as<int32_t>(),
                     csr_row.as<int32_t>(), nnz, flag.as<int32_t>()));
    AZ_TRY(exclusive_scan_i32(flag.as<int32_t>(), segid.as<int32_t>(), nnz, s));
    int32_t nseg = 0;
    AZ_CUDA(cudaMemcpyAsync(&nseg, segid.as<int32_t>() + nnz, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    AZ_TRY(launch_gs(seg_index_kernel, nnz, s, flag.as<int32_t>(), segid.as<int32_t>(), nnz,
                     segx.as<int32_t>()));
    DevBuf seg_first, seg_row, seg_tile, seg_len, seg_plen, pstart;
    AZ_TRY(seg_first.alloc(sizeof(int32_t) * nseg));
    AZ_TRY(seg_row.alloc(sizeof(int32_t) * nseg));
    AZ_TRY(seg_tile.alloc(sizeof(int32_t) * nseg));
    AZ_TRY(seg_len.alloc(sizeof(int32_t) * nseg));
    AZ_TRY(seg_plen.alloc(sizeof(int32_t) * nseg));
    AZ_TRY(pstart.alloc(sizeof(int32_t) * (nseg + 1)));
    AZ_TRY(launch_gs(seg_info_kernel, nnz, s, flag.as<int32_t>(), segid.as<int32_t>(), perm.as<int32_t>(),
                     csr_row.as<int32_t>(), tkey.as<uint32_t>(), nnz, seg_first.as<int32_t>(),
                     seg_row.as<int32_t>(), seg_tile.as<int32_t>()));
    AZ_CUDA(cudaMemsetAsync(seg_len.p, 0, sizeof(int32_t) * nseg, s));
    AZ_TRY(launch_gs(count_keys_kernel, nnz, s, segx.as<int32_t>(), nnz, seg_len.as<int32_t>()));
    AZ_TRY(launch_gs(quad_len_kernel, nseg, s, seg_len.as<int32_t>(), (int64_t)nseg, seg_plen.as<int32_t>()));
    AZ_TRY(exclusive_scan_i32(seg_plen.as<int32_t>(), pstart.as<int32_t>(), nseg, s));

    // segments per tile -> tile_seg_ptr; padded entries per tile (multiple of 8) -> tile_ent_ptr
    DevBuf scnt, tpadcnt;
    AZ_TRY(scnt.alloc(sizeof(int32_t) * ntiles));
    AZ_TRY(tpadcnt.alloc(sizeof(int32_t) * ntiles));
    AZ_CUDA(cudaMemsetAsync(scnt.p, 0, sizeof(int32_t) * ntiles, s));
    AZ_TRY(launch_gs(count_keys_kernel, nseg, s, seg_tile.as<int32_t>(), (int64_t)nseg, scnt.as<int32_t>()));
    AZ_TRY(L.tile_seg_ptr.alloc(sizeof(int32_t) * (ntiles + 1)));
    AZ_TRY(exclusive_scan_i32(scnt.as<int32_t>(), L.tile_seg_ptr.as<int32_t>(), ntiles, s));
    AZ_TRY(launch_gs(tile_pad_kernel, ntiles, s, L.tile_seg_ptr.as<int32_t>(), pstart.as<int32_t>(), ntiles,
                     tpadcnt.as<int32_t>()));
    L.tile_ent_ptr.release();
    AZ_TRY(L.tile_ent_ptr.alloc(sizeof(int32_t) * (ntiles + 1)));
    AZ_TRY(exclusive_scan_i32(tpadcnt.as<int32_t>(), L.tile_ent_ptr.as<int32_t>(), ntiles, s));
    int32_t padded = 0;
    AZ_CUDA(cudaMemcpyAsync(&padded, L.tile_ent_ptr.as<int32_t>() + ntiles, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));

    // padded entry arrays
    L.ent_loc.release(); L.ent_w32.release(); L.ent_w64.release();
    AZ_TRY(L.ent_loc.alloc(sizeof(uint16_t) * (size_t)padded));
    AZ_TRY(L.ent_w32.alloc(sizeof(float) * (size_t)padded));
    AZ_TRY(L.ent_w64.alloc(sizeof(double) * (size_t)padded));
    AZ_TRY(L.ent_pix.alloc(sizeof(int32_t) * (size_t)padded));
    L.ent_dark.release();
    AZ_TRY(launch_gs(fill_u16_kernel, padded, s, L.ent_loc.as<uint16_t>(), (int64_t)padded,
                     (uint16_t)(4 * T.ss)));  // dummies read the zero band
    AZ_CUDA(cudaMemsetAsync(L.ent_w32.p, 0, L.ent_w32.bytes, s));
    AZ_CUDA(cudaMemsetAsync(L.ent_w64.p, 0, L.ent_w64.bytes, s));
    AZ_CUDA(cudaMemsetAsync(L.ent_pix.p, 0xff, L.ent_pix.bytes, s));  // padding entries: -1
    AZ_TRY(L.seg_ent_ptr.alloc(sizeof(int32_t) * 2 * (size_t)nseg));  // [start | end]
    AZ_TRY(launch_gs(seg_span_kernel, nseg, s, seg_tile.as<int32_t>(), pstart.as<int32_t>(),
                     seg_plen.as<int32_t>(), L.tile_seg_ptr.as<int32_t>(), L.tile_ent_ptr.as<int32_t>(),
                     nseg, L.seg_ent_ptr.as<int32_t>(), L.seg_ent_ptr.as<int32_t>() + nseg));
    TiledFillArgs A;
    A.T = T; A.perm = perm.as<int32_t>(); A.csr_idx = h->csr_idx.as<int32_t>();
    A.csr_w = h->csr_w64.as<double>(); A.segx = segx.as<int32_t>();
    A.seg_first = seg_first.as<int32_t>(); A.seg_start = L.seg_ent_ptr.as<int32_t>();
    A.loc = L.ent_loc.as<uint16_t>(); A.w32 = L.ent_w32.as<float>(); A.w64 = L.ent_w64.as<double>();
    A.pix = L.ent_pix.as<int32_t>(); A.n = nnz;
    AZ_TRY(launch_gs(tiled_fill_kernel, nnz, s, A));

    // Frame-pair layout: a 3D copy of one row class of frames F and F + 4 writes the two
    // frames' boxes (th / 4 rows of srow_p words each) back to back, so F + 4 sits slot_p =
    // (th / 4) srow_p words after F.  slot_p = 16 mod 32 puts the two frames on different
    // banks; slots of 2 slot_p words keep F's slots 128-byte aligned; boxes are at most 256
    // words wide.  Tile shapes without such a pitch use the plain layout only.
    int srow_p = 0, ss_p = 0, slot_p = 0, pw_p = 0;
    for (int sr = T.srow; sr <= 256 && !srow_p; sr += 4)
        if (((th / 4) * sr) % 32 == 16) srow_p = sr;
    if (srow_p) {
        slot_p = (th / 4) * srow_p;
        ss_p = 2 * slot_p;
        pw_p = (4 * ss_p + slot_p + 32 + 31) & ~31;
        if (pw_p > 65535) srow_p = 0;
    }
    L.ent_loc_p.release();
    if (srow_p) {
        TileGeom Tp = T;
        Tp.srow = srow_p;
        Tp.ss = ss_p;
        AZ_TRY(L.ent_loc_p.alloc(sizeof(uint16_t) * (size_t)padded));
        AZ_TRY(launch_gs(pair_loc_kernel, padded, s, Tp, L.ent_pix.as<int32_t>(), (int64_t)padded,
                         L.ent_loc_p.as<uint16_t>()));
    } else {
        ss_p = slot_p = pw_p = 0;
    }

    // slots: segments in row order (stable sort of segment ids by row)
    DevBuf skey, sperm, rcnt;
    AZ_TRY(skey.alloc(sizeof(uint32_t) * nseg));
    AZ_TRY(sperm.alloc(sizeof(int32_t) * nseg));
    AZ_TRY(launch_gs(to_u32_kernel, nseg, s, seg_row.as<int32_t>(), skey.as<uint32_t>(), (int64_t)nseg));
    AZ_TRY(launch_gs(iota_kernel, nseg, s, sperm.as<int32_t>(), (int64_t)nseg));
    AZ_TRY(stable_sort_pairs(skey.as<uint32_t>(), sperm.as<int32_t>(), nseg, bits_for(h->nrows - 1), s));
    AZ_TRY(L.seg_slot.alloc(sizeof(int32_t) * nseg));
    AZ_TRY(launch_gs(scatter_slots_kernel, nseg, s, sperm.as<int32_t>(), nseg, L.seg_slot.as<int32_t>()));
    AZ_TRY(rcnt.alloc(sizeof(int32_t) * h->nrows));
    AZ_CUDA(cudaMemsetAsync(rcnt.p, 0, sizeof(int32_t) * h->nrows, s));
    AZ_TRY(launch_gs(count_keys_kernel, nseg, s, seg_row.as<int32_t>(), (int64_t)nseg, rcnt.as<int32_t>()));
    AZ_TRY(L.row_slot_ptr.alloc(sizeof(int32_t) * (h->nrows + 1)));
    AZ_TRY(exclusive_scan_i32(rcnt.as<int32_t>(), L.row_slot_ptr.as<int32_t>(), h->nrows, s));

    // Work items: a tile whose entries would not fit, twice, beside two stages of four frame
    // planes in shared memory is cut at segment boundaries (about 11.5 bytes of shared memory
    // per entry: location, weight, dark and its share of the record).
    const int64_t plane_bytes = 4 * ((int64_t)4 * T.ss + 32);
    const int64_t budget = ((int64_t)max_smem_per_block() - 1024 - 2 * (4 * plane_bytes + 256)) / 2;
    const int kItemEntries = (int)std::max<int64_t>(1024, std::min<int64_t>(60000, budget * 2 / 23) & ~7);
    DevBuf icnt, ioff, chunks, mx;
    AZ_TRY(icnt.alloc(sizeof(int32_t) * ntiles));
    AZ_TRY(ioff.alloc(sizeof(int32_t) * (ntiles + 1)));
    AZ_TRY(mx.alloc(sizeof(int32_t) * 3));
    AZ_TRY(launch_gs(chunk_kernel, ntiles, s, L.tile_seg_ptr.as<int32_t>(), L.seg_ent_ptr.as<int32_t>(),
                     L.seg_ent_ptr.as<int32_t>() + nseg, ntiles, kItemEntries, 0, icnt.as<int32_t>(),
                     (const int32_t *)nullptr, (int32_t *)nullptr));
    AZ_TRY(exclusive_scan_i32(icnt.as<int32_t>(), ioff.as<int32_t>(), ntiles, s));
    int32_t n_items = 0;
    AZ_CUDA(cudaMemcpyAsync(&n_items, ioff.as<int32_t>() + ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    AZ_TRY(chunks.alloc(sizeof(int32_t) * 3 * (size_t)std::max(n_items, 1)));
    AZ_TRY(launch_gs(chunk_kernel, ntiles, s, L.tile_seg_ptr.as<int32_t>(), L.seg_ent_ptr.as<int32_t>(),
                     L.seg_ent_ptr.as<int32_t>() + nseg, ntiles, kItemEntries, 1, icnt.as<int32_t>(),
                     (const int32_t *)ioff.as<int32_t>(), chunks.as<int32_t>()));

    // per-item records and descriptors, and the largest item
    DevBuf rwords, roff, ient, iseg;
    AZ_TRY(rwords.alloc(sizeof(int32_t) * std::max(n_items, 1)));
    AZ_TRY(roff.alloc(sizeof(int32_t) * (n_items + 1)));
    AZ_TRY(ient.alloc(sizeof(int32_t) * std::max(n_items, 1)));
    AZ_TRY(iseg.alloc(sizeof(int32_t) * std::max(n_items, 1)));
    AZ_TRY(launch_gs(rec_words_kernel, n_items, s, chunks.as<int32_t>(), n_items, rwords.as<int32_t>()));
    AZ_TRY(exclusive_scan_i32(rwords.as<int32_t>(), roff.as<int32_t>(), n_items, s));
    int32_t rec_total = 0;
    AZ_CUDA(cudaMemcpyAsync(&rec_total, roff.as<int32_t>() + n_items, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    AZ_TRY(L.tile_rec.alloc(sizeof(int32_t) * std::max(rec_total, 4)));
    AZ_TRY(L.tile_desc.alloc(sizeof(int32_t) * 8 * (size_t)std::max(n_items, 1)));
    AZ_TRY(launch_gs(rec_fill_kernel, n_items, s, chunks.as<int32_t>(), n_items,
                     L.seg_ent_ptr.as<int32_t>(), L.seg_ent_ptr.as<int32_t>() + nseg,
                     L.seg_slot.as<int32_t>(), roff.as<int32_t>(), L.tile_rec.as<int32_t>(),
                     L.tile_desc.as<int32_t>(), ient.as<int32_t>(), iseg.as<int32_t>()));
    max_kernel<<<1, 1024, 0, s>>>(ient.as<int32_t>(), n_items, mx.as<int32_t>());
    AZ_CUDA(cudaGetLastError());
    max_kernel<<<1, 1024, 0, s>>>(iseg.as<int32_t>(), n_items, mx.as<int32_t>() + 1);
    AZ_CUDA(cudaGetLastError());
    max_kernel<<<1, 1024, 0, s>>>(rwords.as<int32_t>(), n_items, mx.as<int32_t>() + 2);
    AZ_CUDA(cudaGetLastError());
    int32_t maxes[3];
    AZ_CUDA(cudaMemcpyAsync(maxes, mx.p, sizeof(maxes), cudaMemcpyDeviceToHost, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    if (maxes[0] > 65535)
        return fail(AZ_EUNSUPPORTED, "a %dx%d tile item holds %d matrix entries (limit 65535): use smaller tiles",
                    th, tw, maxes[0]);
    // tile of every item (kept for accounting)
    AZ_TRY(L.active_tiles.alloc(sizeof(int32_t) * std::max(n_items, 1)));
    if (n_items > 0)
        AZ_CUDA(cudaMemcpy2DAsync(L.active_tiles.p, sizeof(int32_t), chunks.p, 3 * sizeof(int32_t),
                                  sizeof(int32_t), (size_t)n_items, cudaMemcpyDeviceToDevice, s));
    AZ_CUDA(cudaStreamSynchronize(s));
    const int32_t n_active = n_items;
    const int32_t max_rec = maxes[2];

    L.th = th; L.tw = tw; L.srow = T.srow; L.ss = T.ss; L.ntx = T.ntx; L.nty = nty; L.ntiles = ntiles;
    L.srow_p = srow_p; L.ss_p = ss_p; L.slot_p = slot_p; L.pw_p = pw_p;
    L.n_active = n_active; L.nseg = nseg; L.padded_nnz = padded;
    L.max_tile_entries = maxes[0]; L.max_tile_segments = maxes[1];
    L.max_rec_words = max_rec;
    return AZ_OK;
}

}  // namespace azint
