/*
 * Multi-core CPU baseline of the forward -- test infrastructure, not product code.
 *
 * The scheme of the paper's multi-threaded CPU histograms (Sec. 3.4.1, "OpenMP support in
 * Cython"): the pixels are shared among the threads, each thread scatters its pixels'
 * contributions into histograms of its own (no two threads write the same memory, so no
 * atomic operations are needed), and the per-thread histograms are added at the end.  With
 * pixel splitting each pixel scatters into every bin of its column of the weight matrix, so
 * the matrix is read pixel-major (CSC: column pointers, row indices, weights).  FP64 sums;
 * the per-thread histograms are added in thread order, so a run with a given thread count is
 * deterministic.  The same quantities as orc_integrate: S_b = sum_p w_bp (img_p - dark_p),
 * N_b = sum_p w_bp flat_p Omega_p P_p, C_b = sum_p w_bp, I_b = S_b / N_b (0 where N_b = 0).
 *
 * Only the benchmark's CPU-baseline leg (timing) and the tests (its sums against the
 * oracle's) load it; it shares no code with the CUDA path.
 *
 * Build: gcc -O2 -std=c99 -fopenmp -ffp-contract=off -fPIC -shared
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Threads the next parallel region will use. */
int omp_threads(void) { return omp_get_max_threads(); }

/*
 * img: uint32 counts [npix]; dark, flat, sa, pol: float [npix] or NULL (0 and 1).
 * colptr int64 [npix + 1], rows int32 [nnz], w double [nnz].  Outputs double [nrows].
 * Returns the number of threads used, or -1 if the per-thread histograms could not be
 * allocated.
 */
int omp_integrate(int nrows, int64_t npix, const int64_t *colptr, const int32_t *rows,
                  const double *w, const uint32_t *img, const float *dark, const float *flat,
                  const float *sa, const float *pol, double *I, double *S, double *N, double *C)
{
    const int nt = omp_get_max_threads();
    double *hist = (double *)calloc((size_t)nt * 3 * (size_t)nrows, sizeof(double));
    if (!hist) return -1;
    int used = 1;
#pragma omp parallel
    {
        const int t = omp_get_thread_num();
#pragma omp single
        used = omp_get_num_threads();
        double *hs = hist + (size_t)t * 3 * (size_t)nrows;
        double *hn = hs + nrows, *hc = hn + nrows;
#pragma omp for schedule(static)
        for (int64_t p = 0; p < npix; ++p) {
            const int64_t e0 = colptr[p], e1 = colptr[p + 1];
            if (e0 == e1) continue;
            const double v = (double)img[p] - (dark ? (double)dark[p] : 0.0);
            const double nrm = (flat ? (double)flat[p] : 1.0) * (sa ? (double)sa[p] : 1.0) *
                               (pol ? (double)pol[p] : 1.0);
            for (int64_t e = e0; e < e1; ++e) {
                const int32_t b = rows[e];
                hs[b] += w[e] * v;
                hn[b] += w[e] * nrm;
                hc[b] += w[e];
            }
        }
    }
    for (int b = 0; b < nrows; ++b) {
        double s = 0.0, n = 0.0, c = 0.0;
        for (int t = 0; t < used; ++t) {
            const double *h = hist + (size_t)t * 3 * (size_t)nrows;
            s += h[b];
            n += h[nrows + b];
            c += h[2 * (size_t)nrows + b];
        }
        S[b] = s;
        N[b] = n;
        C[b] = c;
        I[b] = (n != 0.0) ? s / n : 0.0;
    }
    free(hist);
    return used;
}
