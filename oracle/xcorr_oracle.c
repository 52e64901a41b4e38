/*
 * CPU oracle for the X stage of an FX correlator -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The product path (the CUDA library under the package's
 * csrc/) never calls, links or includes it, and this file includes nothing of
 * the product.
 *
 * What it computes (Wayth, Greenhill & Briggs, "A GPU based real-time software
 * correlation system for the MWA prototype"):
 *
 *   For every channel c and every input pair 0 <= i <= j < N (autos included,
 *   N(N+1)/2 products, Sec. 2), the channel-by-channel product of the first
 *   spectrum with the complex conjugate of the second (Sec. 2, the `X' stage),
 *   added into an accumulator over the time samples of one dump (Fig. 1):
 *
 *       V_ij(c) = sum_t x_i(c,t) * conj(x_j(c,t))
 *       Re V_ij = sum_t (ar*br + ai*bi),  Im V_ij = sum_t (ai*br - ar*bi)
 *
 *   with a = x_i, b = x_j.  The matrix over (i,j) is the outer product of the
 *   per-channel sample vector with its conjugate (Sec. 4, Fig. 2); only the
 *   upper triangle i <= j is stored.
 *
 * Output layout: vis[c][b][2] (re, im), b = i*N - i*(i-1)/2 + (j - i), the
 * row-major upper triangle.  Integer samples accumulate in int64 (exact);
 * float samples accumulate in double.
 *
 * Input layout: packed samples [T][C][N], input index fastest within one time
 * instant (Sec. 3: the samples of all inputs for one instant are grouped).
 *   bits = 4: one byte per sample, high nibble = re, low nibble = im, two's
 *             complement (the "1-byte mode" of Sec. 5; nibble order is this
 *             oracle's reading, the paper does not print one)
 *   bits = 8: two bytes per sample, re then im, each two's complement
 *   float:    two float32 per sample, re then im
 *
 * Each sample is unpacked by this file's own routine; nothing is shared with
 * the GPU library.  The loops are the plain definition: no blocking, no
 * reordering beyond channel-level threading (channels are independent, Fig. 2).
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int64_t oracle_baseline_index(int64_t n, int64_t i, int64_t j)
{
    /* row-major upper triangle, 0 <= i <= j < n */
    return i * n - (i * (i - 1)) / 2 + (j - i);
}

int64_t oracle_n_baselines(int64_t n) { return n * (n + 1) / 2; }

static int sign_extend(int v, int nbits)
{
    int half = 1 << (nbits - 1);
    return v >= half ? v - (1 << nbits) : v;
}

/* Unpack one complex integer sample.  idx = (t*C + c)*N + i. */
void oracle_unpack_sample(const uint8_t *packed, int bits, int64_t idx, int *re, int *im)
{
    if (bits == 4) {
        int byte = packed[idx];
        *re = sign_extend((byte >> 4) & 0xF, 4);
        *im = sign_extend(byte & 0xF, 4);
    } else {
        *re = sign_extend(packed[2 * idx], 8);
        *im = sign_extend(packed[2 * idx + 1], 8);
    }
}

/* Unpack a whole [T][C][N] block into int32 re/im arrays of the same shape. */
int oracle_unpack(const uint8_t *packed, int n_inputs, int n_chan, int n_time, int bits,
                  int32_t *re, int32_t *im)
{
    if (bits != 4 && bits != 8) return 1;
    int64_t total = (int64_t)n_time * n_chan * n_inputs;
    for (int64_t idx = 0; idx < total; ++idx) {
        int r, m;
        oracle_unpack_sample(packed, bits, idx, &r, &m);
        re[idx] = r;
        im[idx] = m;
    }
    return 0;
}

int oracle_threads_used(int requested)
{
#ifdef _OPENMP
    if (requested > 0) return requested;
    return omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

/*
 * Integer X stage.  chans (length n_sel) lists the channels to compute (NULL:
 * all, n_sel = n_chan); vis receives [n_sel][P][2] int64.  Returns 0 on success.
 */
int oracle_xcorr_int(const uint8_t *packed, int n_inputs, int n_chan, int n_time, int bits,
                     const int32_t *chans, int n_sel, int64_t *vis, int n_threads)
{
    if (bits != 4 && bits != 8) return 1;
    if (n_inputs < 1 || n_chan < 1 || n_time < 0) return 1;
    if (chans == NULL) n_sel = n_chan;
    const int64_t N = n_inputs;
    const int64_t P = oracle_n_baselines(N);
    int status = 0;

#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(| : status)
#else
    (void)n_threads;
#endif
    for (int s = 0; s < n_sel; ++s) {
        int c = chans ? chans[s] : s;
        if (c < 0 || c >= n_chan) { status |= 1; continue; }
        /* this channel's samples, unpacked: x[i][t] */
        int32_t *xr = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)(n_time > 0 ? n_time : 1));
        int32_t *xi = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)(n_time > 0 ? n_time : 1));
        if (!xr || !xi) { free(xr); free(xi); status |= 2; continue; }
        for (int t = 0; t < n_time; ++t)
            for (int64_t i = 0; i < N; ++i) {
                int r, m;
                oracle_unpack_sample(packed, bits, ((int64_t)t * n_chan + c) * N + i, &r, &m);
                xr[i * n_time + t] = r;
                xi[i * n_time + t] = m;
            }
        int64_t *out = vis + (int64_t)s * P * 2;
        for (int64_t i = 0; i < N; ++i) {
            for (int64_t j = i; j < N; ++j) {
                int64_t acc_re = 0, acc_im = 0;
                const int32_t *ar = xr + i * n_time, *ai = xi + i * n_time;
                const int32_t *br = xr + j * n_time, *bi = xi + j * n_time;
                for (int t = 0; t < n_time; ++t) {
                    /* x_i * conj(x_j) */
                    acc_re += (int64_t)ar[t] * br[t] + (int64_t)ai[t] * bi[t];
                    acc_im += (int64_t)ai[t] * br[t] - (int64_t)ar[t] * bi[t];
                }
                int64_t b = oracle_baseline_index(N, i, j);
                out[2 * b] = acc_re;
                out[2 * b + 1] = acc_im;
            }
        }
        free(xr);
        free(xi);
    }
    return status;
}

/*
 * Float X stage in double precision.  x is [T][C][N][2] float32 (re, im);
 * vis receives [n_sel][P][2] double.
 */
int oracle_xcorr_f64(const float *x, int n_inputs, int n_chan, int n_time,
                     const int32_t *chans, int n_sel, double *vis, int n_threads)
{
    if (n_inputs < 1 || n_chan < 1 || n_time < 0) return 1;
    if (chans == NULL) n_sel = n_chan;
    const int64_t N = n_inputs;
    const int64_t P = oracle_n_baselines(N);
    int status = 0;

#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(| : status)
#else
    (void)n_threads;
#endif
    for (int s = 0; s < n_sel; ++s) {
        int c = chans ? chans[s] : s;
        if (c < 0 || c >= n_chan) { status |= 1; continue; }
        double *xr = (double *)malloc(sizeof(double) * (size_t)N * (size_t)(n_time > 0 ? n_time : 1));
        double *xi = (double *)malloc(sizeof(double) * (size_t)N * (size_t)(n_time > 0 ? n_time : 1));
        if (!xr || !xi) { free(xr); free(xi); status |= 2; continue; }
        for (int t = 0; t < n_time; ++t)
            for (int64_t i = 0; i < N; ++i) {
                int64_t idx = ((int64_t)t * n_chan + c) * N + i;
                xr[i * n_time + t] = (double)x[2 * idx];
                xi[i * n_time + t] = (double)x[2 * idx + 1];
            }
        double *out = vis + (int64_t)s * P * 2;
        for (int64_t i = 0; i < N; ++i) {
            for (int64_t j = i; j < N; ++j) {
                double acc_re = 0.0, acc_im = 0.0;
                const double *ar = xr + i * n_time, *ai = xi + i * n_time;
                const double *br = xr + j * n_time, *bi = xi + j * n_time;
                for (int t = 0; t < n_time; ++t) {
                    acc_re += ar[t] * br[t] + ai[t] * bi[t];
                    acc_im += ai[t] * br[t] - ar[t] * bi[t];
                }
                int64_t b = oracle_baseline_index(N, i, j);
                out[2 * b] = acc_re;
                out[2 * b + 1] = acc_im;
            }
        }
        free(xr);
        free(xi);
    }
    return status;
}
