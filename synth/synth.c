/*
 * synth.c -- seeded, counter-based synthetic coarse-channel voltages.
 *
 * This module is shared input plumbing: the FP64 oracle, the tests, bench.py and
 * the GPU path all read voltages made here.  It holds none of the correlator's
 * arithmetic (no FFT, no delay correction, no cross-multiply): it only draws
 * Gaussian noise and adds complex sinusoids, then rounds to int8.
 *
 * Signal model (the paper's workloads, Sec. 2.5 and Sec. 3.1):
 *   x_p[n] = clip127( rint( g_p[n] + sum_t a_t exp(i phi_t)
 *                            * exp(2 pi i (f_t (t_n - tau_p(t_n)) - nu tau_p(t_n))) ) )
 *   - g_p[n]: iid complex Gaussian noise, sigma per component (Box-Muller on a
 *     SplitMix64 counter stream keyed by (seed, path, sample));
 *   - tone t is either common to all paths (a point source seen by every
 *     signal path with that path's delay) or private to one path (the paper's
 *     hand-crafted digital-phase-rotator test vectors, Sec. 3.1);
 *   - tau_p(t) = c0 + c1 t + c2 t^2 (seconds), t_n = n / Fs, Fs = 1.28 MS/s;
 *   - rint() rounds half to even; values are clipped to [-127, 127].
 * Each tone's phase is a quadratic A + B n + C n^2 in the sample index, so it is
 * advanced per sample by a rotation whose angle B + C (2n + 1) itself grows by the
 * fixed 2C per sample (one extra complex multiply when C != 0); both are re-seeded
 * from exact FP64 phases at the start of every 50 ms block (no drift across blocks).
 *
 * Voltage layout: int8 [block][path][block_samples][2] (re, im), i.e. the
 * sub-observation is a sequence of data blocks, each holding every signal
 * path's samples for that block (Sec. 2.5: 64,000 samples per path per 50 ms).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define SYNTH_FS 1280000.0
static const double SYNTH_TWO_PI = 6.283185307179586476925286766559;

/* SplitMix64 output function (Steele, Lea & Flood 2014). */
static inline uint64_t sm64_mix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Counter-based stream: word k of (seed, path, sample). */
static inline uint64_t synth_word(uint64_t seed, uint64_t path, uint64_t sample, uint64_t k)
{
    uint64_t key = sm64_mix(seed ^ 0x4D57415853594E54ULL);
    return sm64_mix(key ^ sm64_mix((path << 40) ^ (sample << 2) ^ k));
}

/* Uniform in (0, 1) with 53 random bits. */
static inline double u01_open(uint64_t w) { return ((double)(w >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

static inline int8_t clip_round(double v)
{
    double r = nearbyint(v); /* default rounding mode: half to even */
    if (r > 127.0) r = 127.0;
    if (r < -127.0) r = -127.0;
    return (int8_t)r;
}

/* Complex Gaussian sample (sigma per component) for (seed, path, sample). */
void synth_gauss(uint64_t seed, uint64_t path, uint64_t sample, double sigma, double* re, double* im)
{
    double u1 = u01_open(synth_word(seed, path, sample, 0));
    double u2 = u01_open(synth_word(seed, path, sample, 1));
    double r = sigma * sqrt(-2.0 * log(u1));
    double th = SYNTH_TWO_PI * u2;
    *re = r * cos(th);
    *im = r * sin(th);
}

/*
 * Fill out[n_blocks][n_paths][block_samples][2].
 *   seed, sigma        : noise stream and its per-component standard deviation
 *   n_tones            : number of sinusoids
 *   tone_freq_hz[t]    : baseband frequency of tone t (Hz, relative to the coarse-channel centre)
 *   tone_amp[t]        : amplitude a_t
 *   tone_phase[t]      : starting phase phi_t (radians)
 *   tone_path[t]       : -1 = common to all paths, else the only path that carries it
 *   delay_poly         : [n_paths][3] (c0 s, c1 s/s, c2 s/s^2) or NULL (no delay)
 *   sky_freq_hz        : nu, sky frequency of the coarse-channel centre
 *   sample0            : absolute index of the first sample (lets callers make any window)
 */
void synth_voltages(uint64_t seed, int n_paths, long long n_blocks, int block_samples, double sigma,
                    int n_tones, const double* tone_freq_hz, const double* tone_amp,
                    const double* tone_phase, const int* tone_path, const double* delay_poly,
                    double sky_freq_hz, long long sample0, int8_t* out)
{
    long long n_units = n_blocks * (long long)n_paths;
#pragma omp parallel
    {
        int nt_cap = n_tones > 0 ? n_tones : 1;
        /* per tone: current value, per-sample rotation, and the rotation's own per-sample
         * rotation (quadratic phase) */
        double* buf = (double*)malloc(sizeof(double) * (size_t)(6 * nt_cap));
        double *cur_re = buf, *cur_im = buf + nt_cap, *rot_re = buf + 2 * nt_cap, *rot_im = buf + 3 * nt_cap;
        double *acc_re = buf + 4 * nt_cap, *acc_im = buf + 5 * nt_cap;
        int* quad = (int*)malloc(sizeof(int) * (size_t)nt_cap);
#pragma omp for schedule(dynamic, 4)
        for (long long unit = 0; unit < n_units; ++unit) {
            long long blk = unit / n_paths;
            int p = (int)(unit % n_paths);
            long long s0 = sample0 + blk * (long long)block_samples;
            double c0 = delay_poly ? delay_poly[3 * p] : 0.0;
            double c1 = delay_poly ? delay_poly[3 * p + 1] : 0.0;
            double c2 = delay_poly ? delay_poly[3 * p + 2] : 0.0;
            /* phase(n) in cycles = phi/2pi + f (t - tau(t)) - nu tau(t), t = n/Fs,
             * tau(t) = c0 + c1 t + c2 t^2, i.e.  A + B n + C n^2                     */
            int nt = 0;
            for (int t = 0; t < n_tones; ++t) {
                if (tone_path[t] >= 0 && tone_path[t] != p) continue;
                double f = tone_freq_hz[t];
                double A = tone_phase[t] / SYNTH_TWO_PI - (f + sky_freq_hz) * c0;
                double B = (f - (f + sky_freq_hz) * c1) / SYNTH_FS;
                double C = -(f + sky_freq_hz) * c2 / (SYNTH_FS * SYNTH_FS);
                double sd = (double)s0;
                /* exact phase at s0 and the step from s0 to s0 + 1, each reduced to [0,1)
                 * cycles before the trig call */
                double cyc = A + B * sd + C * sd * sd;
                cyc -= floor(cyc);
                double stp = B + C * (2.0 * sd + 1.0);
                stp -= floor(stp);
                cur_re[nt] = tone_amp[t] * cos(SYNTH_TWO_PI * cyc);
                cur_im[nt] = tone_amp[t] * sin(SYNTH_TWO_PI * cyc);
                rot_re[nt] = cos(SYNTH_TWO_PI * stp);
                rot_im[nt] = sin(SYNTH_TWO_PI * stp);
                quad[nt] = C != 0.0;
                acc_re[nt] = cos(SYNTH_TWO_PI * 2.0 * C);   /* the step grows by 2C per sample */
                acc_im[nt] = sin(SYNTH_TWO_PI * 2.0 * C);
                ++nt;
            }
            int8_t* o = out + (size_t)unit * (size_t)block_samples * 2;
            for (int i = 0; i < block_samples; ++i) {
                double re = 0.0, im = 0.0;
                if (sigma > 0.0) synth_gauss(seed, (uint64_t)p, (uint64_t)(s0 + i), sigma, &re, &im);
                for (int k = 0; k < nt; ++k) {
                    re += cur_re[k];
                    im += cur_im[k];
                    double nr = cur_re[k] * rot_re[k] - cur_im[k] * rot_im[k];
                    double ni = cur_re[k] * rot_im[k] + cur_im[k] * rot_re[k];
                    cur_re[k] = nr;
                    cur_im[k] = ni;
                    if (quad[k]) {
                        double rr = rot_re[k] * acc_re[k] - rot_im[k] * acc_im[k];
                        double ri = rot_re[k] * acc_im[k] + rot_im[k] * acc_re[k];
                        rot_re[k] = rr;
                        rot_im[k] = ri;
                    }
                }
                o[2 * i] = clip_round(re);
                o[2 * i + 1] = clip_round(im);
            }
        }
        free(buf);
        free(quad);
    }
}

/* Uniform doubles in [0,1) from a counter stream (for tone phases, delays). */
void synth_uniform(uint64_t seed, long long n, double* out)
{
    for (long long i = 0; i < n; ++i)
        out[i] = (double)(synth_word(seed, 0xFFFFFULL, (uint64_t)i, 3) >> 11) * (1.0 / 9007199254740992.0);
}
