/*
 * oracle.c -- plain FP64 CPU reference of the MWAX FX correlator's GPU stage.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this code.  It shares no code, header, table or
 * constant generator with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes is the plain FX definition, written out step by step:
 *   1. x_p[s] = complex(int8 re, int8 im); path p = 2*tile + pol            (Sec. 2.5)
 *   2. frame m = samples [mN, (m+1)N); X_p[m,k] = sum_n x_p[mN+n] e^{-2 pi i k n/N}
 *      (unnormalised forward DFT; radix-2 FFT when N is a power of two, Bluestein's
 *      chirp-z on a radix-2 FFT otherwise, direct DFT available for checks) (Sec. 2.5.1)
 *   3. centre-symmetric channel order: bin k -> offset u (k if k < N - N/2, else k - N),
 *      channel c = u + floor(N/2); f_u = u Fs / N; u = 0 is DC              (Sec. 2.6)
 *   4. delay/phase correction, tau_p(t) = c0 + c1 t + c2 t^2 at the frame centre
 *      t_m = (m + 1/2) N / Fs:  Y = X exp(+2 pi i (nu + f_u) tau_p(t_m))    (Sec. 2.5.1, 4.3)
 *   5. cross-power summed over the frames of integration w:
 *      C_w[p,q,u] = sum_m Y_p[m,u] conj(Y_q[m,u])                           (Sec. 2.5.2)
 *   6. channel averaging by fscrunch F into M = N/F channels, centre-symmetric;
 *      even F sums F+1 bins with the two end bins weighted 1/2; DC excluded from
 *      the centre channel when F > 1; result re-scaled by the weight sum     (Sec. 2.6)
 *   7. MWAX_ORDER [integration][baseline][channel][pol], baselines (i<=j) row-major,
 *      pols xx, xy, yx, yy; weights [baseline][pol] = 1.0 after each set    (Sec. 2.7)
 *   8. integer mode (N = 1, F = 1, no delay): the same sums in exact int64.
 * Readings of points the paper leaves open are listed in the project's design notes
 * and repeated at each step below.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_FS 1280000.0
static const double ORA_PI = 3.14159265358979323846264338327950288;

typedef struct {
    int n_tiles;           /* T; paths n = 2T                                   */
    int fft_len;           /* N, points per frame                               */
    int fine_avg;          /* F (fscrunch); output channels M = N / F           */
    long long int_frames;  /* K, frames per integration                         */
    long long n_samples;   /* samples per path in the call (whole integrations) */
    int block_samples;     /* samples per path per data block (64,000 in MWAX) */
    double sky_freq_hz;    /* nu                                                */
    int dc_exclude;        /* exclude u = 0 from the centre channel when F > 1  */
} ora_desc;

/* ------------------------------------------------------------------ DFT / FFT */

/* Direct O(N^2) forward DFT, twiddle angle reduced exactly as (k n mod N). */
void ora_dft(int n, const double complex* x, double complex* X)
{
    for (int k = 0; k < n; ++k) {
        double complex acc = 0;
        for (int j = 0; j < n; ++j) {
            long long r = ((long long)k * j) % n;
            acc += x[j] * cexp(-2.0 * ORA_PI * I * (double)r / (double)n);
        }
        X[k] = acc;
    }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* In-place iterative radix-2 (Cooley-Tukey, bit-reversed input order). sign = -1 forward. */
static void fft_radix2_inplace(int n, double complex* a, int sign)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double complex t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int i = 0; i < n; i += len) {
            for (int k = 0; k < len / 2; ++k) {
                double complex w = cexp(sign * 2.0 * ORA_PI * I * (double)k / (double)len);
                double complex u = a[i + k];
                double complex v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

/* Bluestein: X_k = conj(b_k) sum_j (x_j conj(b_j)) b_{k-j}, b_j = e^{i pi j^2 / N},
 * the convolution done with radix-2 FFTs of length >= 2N-1. */
static void fft_bluestein(int n, const double complex* x, double complex* X)
{
    int m = 1;
    while (m < 2 * n - 1) m <<= 1;
    double complex* a = calloc((size_t)m, sizeof(double complex));
    double complex* b = calloc((size_t)m, sizeof(double complex));
    double complex* w = malloc(sizeof(double complex) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        long long r = ((long long)j * j) % (2LL * n); /* j^2 mod 2N keeps the angle exact */
        w[j] = cexp(I * ORA_PI * (double)r / (double)n);
    }
    for (int j = 0; j < n; ++j) a[j] = x[j] * conj(w[j]);
    b[0] = w[0];
    for (int j = 1; j < n; ++j) b[j] = b[m - j] = w[j];
    fft_radix2_inplace(m, a, -1);
    fft_radix2_inplace(m, b, -1);
    for (int i = 0; i < m; ++i) a[i] *= b[i];
    fft_radix2_inplace(m, a, +1);
    for (int k = 0; k < n; ++k) X[k] = conj(w[k]) * a[k] / (double)m;
    free(a);
    free(b);
    free(w);
}

/* Forward unnormalised DFT of length n by the fast routes above. */
void ora_fft(int n, const double complex* x, double complex* X)
{
    if (n == 1) {
        X[0] = x[0];
    } else if (is_pow2(n)) {
        memcpy(X, x, sizeof(double complex) * (size_t)n);
        fft_radix2_inplace(n, X, -1);
    } else {
        fft_bluestein(n, x, X);
    }
}

/* ---------------------------------------------------------- channel geometry */

/* Frequency offset u (in ultrafine bins) of channel c: c = u + floor(N/2). */
int ora_offset_of_channel(int N, int c) { return c - N / 2; }

/* Channel c holding FFT bin k (fftshift). */
static int channel_of_bin(int N, int k)
{
    int u = (k < N - N / 2) ? k : k - N;
    return u + N / 2;
}

/*
 * Weights of output channel j over the N ultrafine channels (indexed by c), Sec. 2.6.
 * Centre output channel j0 = floor(M/2) sits on DC; channel j is centred on
 * offset (j - j0) F.  Odd F: bins centre +- (F-1)/2, weight 1.  Even F: bins
 * centre +- F/2, the two end bins weight 1/2.  Bins outside [-N/2, N - N/2 - 1]
 * are dropped (the edge half-channels of even M are still emitted).  With
 * dc_exclude and F > 1 the DC bin gets weight 0.  Returns the weight sum.
 */
double ora_avg_weights(int N, int F, int dc_exclude, int j, double* w)
{
    int M = N / F;
    int j0 = M / 2;
    long long centre = (long long)(j - j0) * F;
    int half = F / 2; /* even F: F/2 with half-weight ends; odd F: (F-1)/2 */
    double sum = 0.0;
    for (int c = 0; c < N; ++c) w[c] = 0.0;
    for (long long u = centre - half; u <= centre + half; ++u) {
        double wt = 1.0;
        if (F % 2 == 0 && (u == centre - half || u == centre + half)) wt = 0.5;
        if (dc_exclude && F > 1 && u == 0) wt = 0.0;
        long long c = u + N / 2;
        if (c < 0 || c >= N) continue;
        w[c] = wt;
        sum += wt;
    }
    return sum;
}

/* ---------------------------------------------------------------- baselines */

long long ora_n_baselines(int T) { return (long long)T * (T + 1) / 2; }

/* Baseline b -> tiles (i, j), i <= j, row-major over the upper triangle (Sec. 2.7). */
void ora_baseline_tiles(int T, long long b, int* ti, int* tj)
{
    int i = 0;
    long long start = 0;
    while (start + (T - i) <= b) {
        start += T - i;
        ++i;
    }
    *ti = i;
    *tj = i + (int)(b - start);
}

/* Paths of (baseline, pol): pol 0..3 = xx, xy, yx, yy, p = 2i + a, q = 2j + e. */
static void baseline_paths(int T, long long b, int pol, int* p, int* q)
{
    int i, j;
    ora_baseline_tiles(T, b, &i, &j);
    *p = 2 * i + (pol >> 1);
    *q = 2 * j + (pol & 1);
}

/* ---------------------------------------------------------------- F step */

static inline double complex volt_at(const ora_desc* d, const int8_t* volt, int p, long long s)
{
    int n_paths = 2 * d->n_tiles;
    long long blk = s / d->block_samples, i = s % d->block_samples;
    const int8_t* v = volt + ((blk * n_paths + p) * (long long)d->block_samples + i) * 2;
    return (double)v[0] + I * (double)v[1];
}

/*
 * Spectra of path p for frames [m0, m0 + nm): Y[m - m0][c], FFT, channel shift and
 * delay correction (steps 1-4).  delay = [n_paths][3] (c0, c1, c2) or NULL.
 */
void ora_spectra(const ora_desc* d, const int8_t* volt, const double* delay, int p, long long m0,
                 long long nm, double complex* Y)
{
    int N = d->fft_len;
    double complex* x = malloc(sizeof(double complex) * (size_t)N);
    double complex* X = malloc(sizeof(double complex) * (size_t)N);
    for (long long m = m0; m < m0 + nm; ++m) {
        for (int n = 0; n < N; ++n) x[n] = volt_at(d, volt, p, m * N + n);
        ora_fft(N, x, X);
        double complex* out = Y + (m - m0) * N;
        for (int k = 0; k < N; ++k) out[channel_of_bin(N, k)] = X[k];
        if (delay) {
            double t = ((double)m + 0.5) * (double)N / ORA_FS;
            double tau = delay[3 * p] + delay[3 * p + 1] * t + delay[3 * p + 2] * t * t;
            for (int c = 0; c < N; ++c) {
                double f = (double)ora_offset_of_channel(N, c) * ORA_FS / (double)N;
                double cyc = (d->sky_freq_hz + f) * tau;
                out[c] *= cexp(2.0 * ORA_PI * I * cyc);
            }
        }
    }
    free(x);
    free(X);
}

/* --------------------------------------------------------- validation */

int ora_check(const ora_desc* d)
{
    if (d->n_tiles < 1 || d->fft_len < 1 || d->fine_avg < 1 || d->int_frames < 1) return -1;
    if (d->block_samples < 1 || d->block_samples % d->fft_len) return -1;
    if (d->fft_len % d->fine_avg) return -1;
    if (d->n_samples < 1 || d->n_samples % ((long long)d->int_frames * d->fft_len)) return -1;
    if (d->n_samples % d->block_samples) return -1;
    return 0;
}

/* ---------------------------------------------------------- X + averaging */

/*
 * Full correlation (steps 1-7).  vis: double complex [ints][B][M][4];
 * weights: double [ints][B][4] (all 1.0, the paper's current occupancy weights).
 * Memory: holds every path's spectra for one integration (n K N complex).
 */
int ora_correlate(const ora_desc* d, const int8_t* volt, const double* delay, double complex* vis,
                  double* weights)
{
    if (ora_check(d)) return -1;
    int T = d->n_tiles, n = 2 * T, N = d->fft_len, F = d->fine_avg, M = N / F;
    long long K = d->int_frames, n_ints = d->n_samples / (K * N), B = ora_n_baselines(T);
    double complex* Y = malloc(sizeof(double complex) * (size_t)n * (size_t)K * (size_t)N);
    double* wts = malloc(sizeof(double) * (size_t)M * (size_t)N);
    double* wsum = malloc(sizeof(double) * (size_t)M);
    if (!Y || !wts || !wsum) {
        free(Y);
        free(wts);
        free(wsum);
        return -2;
    }
    for (int j = 0; j < M; ++j) wsum[j] = ora_avg_weights(N, F, d->dc_exclude, j, wts + (size_t)j * N);
    for (long long w = 0; w < n_ints; ++w) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int p = 0; p < n; ++p) ora_spectra(d, volt, delay, p, w * K, K, Y + (size_t)p * K * N);
#pragma omp parallel for schedule(dynamic, 1)
        for (long long bp = 0; bp < B * 4; ++bp) {
            long long b = bp / 4;
            int pol = (int)(bp % 4), p, q;
            baseline_paths(T, b, pol, &p, &q);
            for (int j = 0; j < M; ++j) {
                double complex acc = 0;
                for (int c = 0; c < N; ++c) {
                    double wt = wts[(size_t)j * N + c];
                    if (wt == 0.0) continue;
                    double complex cpq = 0; /* C_w[p,q,c], brute force over frames */
                    for (long long m = 0; m < K; ++m)
                        cpq += Y[((size_t)p * K + m) * N + c] * conj(Y[((size_t)q * K + m) * N + c]);
                    acc += wt * cpq;
                }
                vis[((w * B + b) * M + j) * 4 + pol] = acc / wsum[j];
            }
            weights[(w * B + b) * 4 + pol] = 1.0;
        }
    }
    free(Y);
    free(wts);
    free(wsum);
    return 0;
}

/*
 * Full n x n cross-power matrix of channel c, integration w, both triangles computed
 * independently by brute force (for the Hermitian check): C[p*n + q].
 */
int ora_xmatrix(const ora_desc* d, const int8_t* volt, const double* delay, long long w, int c,
                double complex* C)
{
    if (ora_check(d)) return -1;
    int n = 2 * d->n_tiles, N = d->fft_len;
    long long K = d->int_frames;
    double complex* Y = malloc(sizeof(double complex) * (size_t)n * (size_t)K * (size_t)N);
    if (!Y) return -2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < n; ++p) ora_spectra(d, volt, delay, p, w * K, K, Y + (size_t)p * K * N);
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double complex acc = 0;
            for (long long m = 0; m < K; ++m) acc += Y[((size_t)p * K + m) * N + c] * conj(Y[((size_t)q * K + m) * N + c]);
            C[(size_t)p * n + q] = acc;
        }
    free(Y);
    return 0;
}

/*
 * Selected outputs only: req[4 r .. 4 r + 3] = (w, b, j, pol) -> out[r] (step 6/7
 * value of that one visibility).  Spectra are made for just the paths requested,
 * one integration at a time, so full-size workloads can be spot-checked.
 */
int ora_correlate_sampled(const ora_desc* d, const int8_t* volt, const double* delay, long long n_req,
                          const long long* req, double complex* out)
{
    if (ora_check(d)) return -1;
    int T = d->n_tiles, n = 2 * T, N = d->fft_len, F = d->fine_avg;
    long long K = d->int_frames;
    char* need = malloc((size_t)n);
    int* slot = malloc(sizeof(int) * (size_t)n);
    char* done = calloc((size_t)n_req, 1);
    double* wts = malloc(sizeof(double) * (size_t)N);
    for (long long r0 = 0; r0 < n_req; ++r0) {
        if (done[r0]) continue;
        long long w = req[4 * r0];
        memset(need, 0, (size_t)n);
        for (long long r = r0; r < n_req; ++r) {
            if (req[4 * r] != w) continue;
            int p, q;
            baseline_paths(T, req[4 * r + 1], (int)req[4 * r + 3], &p, &q);
            need[p] = need[q] = 1;
        }
        int n_need = 0;
        for (int p = 0; p < n; ++p) slot[p] = need[p] ? n_need++ : -1;
        double complex* Y = malloc(sizeof(double complex) * (size_t)n_need * (size_t)K * (size_t)N);
        if (!Y) return -2;
#pragma omp parallel for schedule(dynamic, 1)
        for (int p = 0; p < n; ++p)
            if (slot[p] >= 0) ora_spectra(d, volt, delay, p, w * K, K, Y + (size_t)slot[p] * K * N);
        for (long long r = r0; r < n_req; ++r) {
            if (req[4 * r] != w) continue;
            int p, q, j = (int)req[4 * r + 2];
            baseline_paths(T, req[4 * r + 1], (int)req[4 * r + 3], &p, &q);
            double ws = ora_avg_weights(N, F, d->dc_exclude, j, wts);
            double complex acc = 0;
            for (int c = 0; c < N; ++c) {
                if (wts[c] == 0.0) continue;
                double complex cpq = 0;
                const double complex* yp = Y + (size_t)slot[p] * K * N;
                const double complex* yq = Y + (size_t)slot[q] * K * N;
                for (long long m = 0; m < K; ++m) cpq += yp[m * N + c] * conj(yq[m * N + c]);
                acc += wts[c] * cpq;
            }
            out[r] = acc / ws;
            done[r] = 1;
        }
        free(Y);
    }
    free(need);
    free(slot);
    free(done);
    free(wts);
    return 0;
}

/*
 * Integer mode (N = 1, F = 1, no delay correction): exact int64 sums.
 * vis: int64 [ints][B][4][2] (re, im); weights: double [ints][B][4] = 1.0.
 */
int ora_correlate_int(const ora_desc* d, const int8_t* volt, long long* vis, double* weights)
{
    if (ora_check(d) || d->fft_len != 1 || d->fine_avg != 1) return -1;
    int T = d->n_tiles;
    long long K = d->int_frames, n_ints = d->n_samples / K, B = ora_n_baselines(T);
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (long long w = 0; w < n_ints; ++w)
        for (long long bp = 0; bp < B * 4; ++bp) {
            long long b = bp / 4;
            int pol = (int)(bp % 4), p, q;
            baseline_paths(T, b, pol, &p, &q);
            long long re = 0, im = 0;
            int n_paths = 2 * T, bs = d->block_samples;
            for (long long s = w * K; s < (w + 1) * K; ++s) {
                long long blk = s / bs, i = s % bs;
                const int8_t* a = volt + ((blk * n_paths + p) * (long long)bs + i) * 2;
                const int8_t* e = volt + ((blk * n_paths + q) * (long long)bs + i) * 2;
                /* (ar + i ai)(er - i ei) */
                re += (long long)a[0] * e[0] + (long long)a[1] * e[1];
                im += (long long)a[1] * e[0] - (long long)a[0] * e[1];
            }
            vis[((w * B + b) * 4 + pol) * 2] = re;
            vis[((w * B + b) * 4 + pol) * 2 + 1] = im;
            weights[(w * B + b) * 4 + pol] = 1.0;
        }
    return 0;
}

/* ============================================================================
 * Roadmap extensions (Sec. 4), each a plain restatement of what the paper describes:
 *   - zeroing flags and visibility weights (Sec. 2.4.2, 4.1): a flagged 50 ms block of
 *     a path holds no data (its samples count as zero); the weight of a baseline/pol in
 *     an integration is the fraction of the integration's frames whose blocks are
 *     unflagged in both paths; optionally the visibility is divided by that weight;
 *   - tabulated fractional delays (Sec. 2.4.1, 4.3): one value per path per table step
 *     (5 ms = 6,400 samples in MWAX), held constant over the step; frame m uses the step
 *     containing its centre sample (m + 1/2) N;
 *   - passband de-ripple (Sec. 4.2): a real magnitude gain per ultrafine channel
 *     multiplies every spectral value together with the delay phasor;
 *   - oversampled coarse channels (Sec. 4.5): the coarse channel is sampled at a rate
 *     above its spacing; only the keep_bins ultrafine channels around DC are passed to
 *     the X step and averaged (M = keep_bins / F), the rest are discarded.
 * ========================================================================== */

typedef struct {
    double sample_rate_hz;       /* coarse-channel sample rate Fs; 0 = 1.28 MS/s       */
    int keep_bins;               /* ultrafine channels kept around DC; 0 = all N       */
    const double* delay_table;   /* [n_paths][table_steps] seconds, or NULL            */
    long long table_step;        /* samples per table step                             */
    long long table_steps;       /* entries per path                                   */
    const double* passband;      /* [N] gain per ultrafine channel c, or NULL          */
    const uint8_t* zero_flags;   /* [n_blocks][n_paths], nonzero = zeroed, or NULL     */
    int normalise;               /* divide visibilities by their occupancy weight      */
} ora_ext;

static double ext_fs(const ora_ext* e) { return (e && e->sample_rate_hz > 0.0) ? e->sample_rate_hz : ORA_FS; }

static int ext_keep(const ora_desc* d, const ora_ext* e) { return (e && e->keep_bins > 0) ? e->keep_bins : d->fft_len; }

static int ext_flagged(const ora_desc* d, const ora_ext* e, int p, long long s)
{
    if (!e || !e->zero_flags) return 0;
    long long blk = s / d->block_samples;
    return e->zero_flags[blk * (2LL * d->n_tiles) + p] != 0;
}

/*
 * Averaging weights of output channel j when only the keep ultrafine channels around DC
 * are used: M = keep / F output channels centred as in Sec. 2.6, bins outside
 * [-keep/2, keep - keep/2 - 1] dropped.  keep = N gives ora_avg_weights.
 */
double ora_avg_weights_keep(int N, int keep, int F, int dc_exclude, int j, double* w)
{
    int M = keep / F;
    int j0 = M / 2;
    long long centre = (long long)(j - j0) * F;
    int half = F / 2;
    double sum = 0.0;
    for (int c = 0; c < N; ++c) w[c] = 0.0;
    for (long long u = centre - half; u <= centre + half; ++u) {
        double wt = 1.0;
        if (F % 2 == 0 && (u == centre - half || u == centre + half)) wt = 0.5;
        if (dc_exclude && F > 1 && u == 0) wt = 0.0;
        if (u < -(keep / 2) || u > keep - keep / 2 - 1) continue;
        w[u + N / 2] = wt;
        sum += wt;
    }
    return sum;
}

/* Fractional delay of path p for the frame starting at sample s0 (N samples), seconds. */
static double ext_tau(const ora_desc* d, const ora_ext* e, const double* delay, int p, long long s0)
{
    int N = d->fft_len;
    if (e && e->delay_table) {
        long long step = (2 * s0 + N) / (2 * e->table_step);   /* step holding sample s0 + N/2 */
        if (step >= e->table_steps) step = e->table_steps - 1;
        return e->delay_table[(long long)p * e->table_steps + step];
    }
    double t = ((double)(s0 / N) + 0.5) * (double)N / ext_fs(e);   /* frame centre */
    return delay[3 * p] + delay[3 * p + 1] * t + delay[3 * p + 2] * t * t;
}

/* ora_spectra with the extensions: sample rate, flags, delay table, passband gains. */
void ora_spectra_ext(const ora_desc* d, const ora_ext* e, const int8_t* volt, const double* delay, int p,
                     long long m0, long long nm, double complex* Y)
{
    int N = d->fft_len;
    double fs = ext_fs(e);
    int have_delay = delay != NULL || (e && e->delay_table);
    double complex* x = malloc(sizeof(double complex) * (size_t)N);
    double complex* X = malloc(sizeof(double complex) * (size_t)N);
    for (long long m = m0; m < m0 + nm; ++m) {
        long long s0 = m * N;
        int zero = ext_flagged(d, e, p, s0); /* frames never straddle a block (N | block) */
        for (int n = 0; n < N; ++n) x[n] = zero ? 0.0 : volt_at(d, volt, p, s0 + n);
        ora_fft(N, x, X);
        double complex* out = Y + (m - m0) * N;
        for (int k = 0; k < N; ++k) out[channel_of_bin(N, k)] = X[k];
        double tau = have_delay ? ext_tau(d, e, delay, p, s0) : 0.0;
        for (int c = 0; c < N; ++c) {
            if (have_delay) {
                double f = (double)ora_offset_of_channel(N, c) * fs / (double)N;
                double cyc = (d->sky_freq_hz + f) * tau;
                out[c] *= cexp(2.0 * ORA_PI * I * cyc);
            }
            if (e && e->passband) out[c] *= e->passband[c];
        }
    }
    free(x);
    free(X);
}

/* Occupancy weight of paths (p, q) over integration w: fraction of its K frames whose
 * block is unflagged in both paths (Sec. 4.1).  1.0 without flags. */
double ora_occupancy(const ora_desc* d, const ora_ext* e, long long w, int p, int q)
{
    long long K = d->int_frames, good = 0;
    int N = d->fft_len;
    for (long long m = w * K; m < (w + 1) * K; ++m)
        if (!ext_flagged(d, e, p, m * N) && !ext_flagged(d, e, q, m * N)) ++good;
    return (double)good / (double)K;
}

int ora_check_ext(const ora_desc* d, const ora_ext* e)
{
    if (ora_check(d)) return -1;
    if (!e) return 0;
    int keep = ext_keep(d, e);
    if (keep < 1 || keep > d->fft_len || keep % d->fine_avg) return -1;
    if (e->delay_table && (e->table_step < 1 || e->table_steps < 1)) return -1;
    return 0;
}

/*
 * Full correlation with the extensions.  vis: [ints][B][M][4] with M = keep / F;
 * weights: [ints][B][4] occupancy (1.0 without flags); with normalise, each visibility
 * is divided by its weight (left at 0 where the weight is 0).
 */
int ora_correlate_ext(const ora_desc* d, const ora_ext* e, const int8_t* volt, const double* delay,
                      double complex* vis, double* weights)
{
    if (ora_check_ext(d, e)) return -1;
    int T = d->n_tiles, n = 2 * T, N = d->fft_len, F = d->fine_avg, keep = ext_keep(d, e), M = keep / F;
    long long K = d->int_frames, n_ints = d->n_samples / (K * N), B = ora_n_baselines(T);
    double complex* Y = malloc(sizeof(double complex) * (size_t)n * (size_t)K * (size_t)N);
    double* wts = malloc(sizeof(double) * (size_t)M * (size_t)N);
    double* wsum = malloc(sizeof(double) * (size_t)M);
    if (!Y || !wts || !wsum) {
        free(Y);
        free(wts);
        free(wsum);
        return -2;
    }
    for (int j = 0; j < M; ++j) wsum[j] = ora_avg_weights_keep(N, keep, F, d->dc_exclude, j, wts + (size_t)j * N);
    for (long long w = 0; w < n_ints; ++w) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int p = 0; p < n; ++p) ora_spectra_ext(d, e, volt, delay, p, w * K, K, Y + (size_t)p * K * N);
#pragma omp parallel for schedule(dynamic, 1)
        for (long long bp = 0; bp < B * 4; ++bp) {
            long long b = bp / 4;
            int pol = (int)(bp % 4), p, q;
            baseline_paths(T, b, pol, &p, &q);
            double occ = ora_occupancy(d, e, w, p, q);
            for (int j = 0; j < M; ++j) {
                double complex acc = 0;
                for (int c = 0; c < N; ++c) {
                    double wt = wts[(size_t)j * N + c];
                    if (wt == 0.0) continue;
                    double complex cpq = 0;
                    for (long long m = 0; m < K; ++m)
                        cpq += Y[((size_t)p * K + m) * N + c] * conj(Y[((size_t)q * K + m) * N + c]);
                    acc += wt * cpq;
                }
                double complex v = acc / wsum[j];
                if (e && e->normalise) v = occ > 0.0 ? v / occ : 0.0;
                vis[((w * B + b) * M + j) * 4 + pol] = v;
            }
            weights[(w * B + b) * 4 + pol] = occ;
        }
    }
    free(Y);
    free(wts);
    free(wsum);
    return 0;
}

/* Integer mode with zeroing flags: flagged samples count as zero, weights = occupancy
 * (no normalisation: the sums stay exact integers). */
int ora_correlate_int_ext(const ora_desc* d, const ora_ext* e, const int8_t* volt, long long* vis, double* weights)
{
    if (ora_check_ext(d, e) || d->fft_len != 1 || d->fine_avg != 1 || (e && e->normalise)) return -1;
    int T = d->n_tiles;
    long long K = d->int_frames, n_ints = d->n_samples / K, B = ora_n_baselines(T);
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (long long w = 0; w < n_ints; ++w)
        for (long long bp = 0; bp < B * 4; ++bp) {
            long long b = bp / 4;
            int pol = (int)(bp % 4), p, q;
            baseline_paths(T, b, pol, &p, &q);
            long long re = 0, im = 0;
            int n_paths = 2 * T, bs = d->block_samples;
            for (long long s = w * K; s < (w + 1) * K; ++s) {
                if (ext_flagged(d, e, p, s) || ext_flagged(d, e, q, s)) continue;
                long long blk = s / bs, i = s % bs;
                const int8_t* a = volt + ((blk * n_paths + p) * (long long)bs + i) * 2;
                const int8_t* c = volt + ((blk * n_paths + q) * (long long)bs + i) * 2;
                re += (long long)a[0] * c[0] + (long long)a[1] * c[1];
                im += (long long)a[1] * c[0] - (long long)a[0] * c[1];
            }
            vis[((w * B + b) * 4 + pol) * 2] = re;
            vis[((w * B + b) * 4 + pol) * 2 + 1] = im;
            weights[(w * B + b) * 4 + pol] = ora_occupancy(d, e, w, p, q);
        }
    return 0;
}

/* ============================================================================
 * Tied-array beamformer (Sec. 4.4), plain FP64.  The spectra of every path are formed
 * without the correlator's delay correction (steps 1-3); coherent beam b of polarisation
 * a is the delay-steered sum over tiles t of path p = 2t + a:
 *     B_b,a[m, c] = sum_t Y_p[m, c] exp(+2 pi i (nu + f_u) tau_b,p(step(m)))
 * with tau from the beam's table of fractional delays (one value per path per step of
 * table_step samples, a frame taking the step that holds its centre, as in Sec. 2.4.1).
 * Detected outputs over integrations of int_frames frames (when int_frames > 0):
 *     P_b[w, c] = sum_{m in w} |B_b,x[m, c]|^2 + |B_b,y[m, c]|^2   (Stokes I)
 *     I[w, a, c] = sum_{m in w} sum_t |Y_{2t+a}[m, c]|^2             (incoherent beam)
 * ========================================================================== */
int ora_beamform(const ora_desc* d, double fs_in, const int8_t* volt, int n_beams, const double* beam_tab,
                 long long table_step, long long table_steps, long long int_frames, double complex* beams,
                 double* power, double* incoh)
{
    if (ora_check(d) || n_beams < 1 || table_step < 1 || table_steps < 1) return -1;
    int T = d->n_tiles, n = 2 * T, N = d->fft_len;
    double fs = fs_in > 0.0 ? fs_in : ORA_FS;
    long long frames = d->n_samples / N;
    long long n_det = int_frames > 0 ? frames / int_frames : 0;
    double complex* Y = malloc(sizeof(double complex) * (size_t)n * (size_t)frames * (size_t)N);
    if (!Y) return -2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < n; ++p) ora_spectra(d, volt, NULL, p, 0, frames, Y + (size_t)p * frames * N);
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int b = 0; b < n_beams; ++b)
        for (int a = 0; a < 2; ++a)
            for (long long m = 0; m < frames; ++m) {
                long long step = (2 * m * N + N) / (2 * table_step);
                if (step >= table_steps) step = table_steps - 1;
                for (int c = 0; c < N; ++c) {
                    double f = (double)ora_offset_of_channel(N, c) * fs / (double)N;
                    double complex acc = 0;
                    for (int t = 0; t < T; ++t) {
                        int p = 2 * t + a;
                        double tau = beam_tab[((long long)b * n + p) * table_steps + step];
                        double cyc = (d->sky_freq_hz + f) * tau;
                        acc += Y[((size_t)p * frames + m) * N + c] * cexp(2.0 * ORA_PI * I * cyc);
                    }
                    beams[(((size_t)b * 2 + a) * frames + m) * N + c] = acc;
                }
            }
    for (long long w = 0; w < n_det; ++w)
        for (int c = 0; c < N; ++c) {
            for (int b = 0; b < n_beams; ++b) {
                double s = 0.0;
                for (long long m = w * int_frames; m < (w + 1) * int_frames; ++m)
                    for (int a = 0; a < 2; ++a) {
                        double complex v = beams[(((size_t)b * 2 + a) * frames + m) * N + c];
                        s += creal(v) * creal(v) + cimag(v) * cimag(v);
                    }
                if (power) power[((size_t)b * n_det + w) * N + c] = s;
            }
            for (int a = 0; a < 2; ++a) {
                double s = 0.0;
                for (long long m = w * int_frames; m < (w + 1) * int_frames; ++m)
                    for (int t = 0; t < T; ++t) {
                        double complex v = Y[((size_t)(2 * t + a) * frames + m) * N + c];
                        s += creal(v) * creal(v) + cimag(v) * cimag(v);
                    }
                if (incoh) incoh[((size_t)w * 2 + a) * N + c] = s;
            }
        }
    free(Y);
    return 0;
}
