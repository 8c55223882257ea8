// Tied-array multibeam beamformer (Sec. 4.4) on the correlator's F-step.
//
// The voltages are channelised by the same F-step kernels as the correlator, without
// delay correction (FP32 planar spectra Y[c][plane][p][k] for a chunk of frames).  Each
// beam then steers every path with its own tabulated fractional delays (one value per
// path per step of table_step samples, a frame taking the step that holds its centre,
// as the correlator's tables do) and sums the tiles of each polarisation:
//     B_b,a[m, c] = sum_t Y_{2t+a}[m, c] exp(+2 pi i (nu + f_u) tau_b,2t+a(step(m)))
// For one channel and one step that is a small complex matrix product, beams x tiles
// times tiles x frames, whose left factor W[b][t] depends on (channel, step) only.  A CTA
// takes one step's frames (up to 32), 8 channels and up to 8 beams of one polarisation:
// it builds W for 16 tiles at a time in shared memory (one sincospi per beam and tile, the
// other channels by the exact phasor ratio e^{2 pi i tau Fs / N}) while the next 16 tiles'
// spectra stream in by asynchronous copies (two stages), and each thread accumulates an
// 8-beam x 2-frame complex register tile.  The
// incoherent beam (sum over tiles of |Y|^2) is accumulated from the same staged spectra.
// Detected Stokes I is formed afterwards from the coherent beams.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "plan.cuh"

namespace mwax {
namespace {

constexpr int CB = 8;      // channels per CTA
constexpr int FMAX = 32;   // frames per CTA
constexpr int TC = 16;     // tiles per shared-memory chunk
constexpr int BG = 8;      // beams per CTA
constexpr int NT = 128;    // threads: 8 channels x 16 pairs of frames
// two stages of (spectra Re, Im planes + steering phasors): 80 KB
constexpr size_t kStageY = sizeof(float) * CB * TC * FMAX;
constexpr size_t kStageW = sizeof(float2) * CB * TC * BG;
constexpr size_t kBeamSmem = 2 * (2 * kStageY + kStageW);

struct BeamUnit {
    int m_lo, m_hi;   // frames of the chunk (relative to its first frame)
    long long step;   // table step of those frames
};

// Per (beam, path, step): phi0 = frac(nu tau), d = tau Fs / N split into d_hi (12
// significant bits, so that u d_hi is exact for |u| < 4096) and d_lo.
__global__ void beam_params_kernel(const double* __restrict__ tab, long long total, double nu, double fs, int N,
                                   float4* __restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double tau = tab[i];
        const double ph = nu * tau;
        const double d = tau * fs / (double)N;
        const float dh = __uint_as_float(__float_as_uint((float)d) & 0xFFFFF000u);
        out[i] = make_float4((float)(ph - floor(ph)), dh, (float)(d - (double)dh), 0.0f);
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// 4-byte asynchronous copy global -> shared; src_bytes = 0 fills the destination with zero.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct BeamArgs {
    const float* Y;         // chunk spectra, slot 0: [N][2][n][Kpad]
    const float4* params;   // [nb][n][steps]
    const BeamUnit* units;
    float2* beams;          // [nb][2][frames][N]
    float* incoh;           // [n_det][2][N] or nullptr
    long long Kpad, steps, frames, f0;   // f0: first frame of the chunk in the call
    int T, n, N, nb, int_frames;
    long long n_det;
};

__global__ void __launch_bounds__(NT) beam_kernel(const BeamArgs a)
{
    extern __shared__ __align__(16) unsigned char beam_smem[];
    const BeamUnit un = a.units[blockIdx.x];
    const int c0 = blockIdx.y * CB;
    const int pol = blockIdx.z & 1, bg = blockIdx.z >> 1;
    const int tid = threadIdx.x;
    const int ch = tid / 16, fg = tid % 16;   // channel, frames 2 fg and 2 fg + 1
    const int nfr = un.m_hi - un.m_lo;
    const int n_chunks = (a.T + TC - 1) / TC;

    auto Yr = [&](int st) { return reinterpret_cast<float (*)[TC][FMAX]>(beam_smem + st * (2 * kStageY + kStageW)); };
    auto Yi = [&](int st) {
        return reinterpret_cast<float (*)[TC][FMAX]>(beam_smem + st * (2 * kStageY + kStageW) + kStageY);
    };
    auto Wt = [&](int st) {
        return reinterpret_cast<float2 (*)[TC][BG]>(beam_smem + st * (2 * kStageY + kStageW) + 2 * kStageY);
    };

    // stage the spectra of tile chunk k (16 tiles x 8 channels x the unit's frames, zero
    // past the end) with asynchronous copies
    auto stage = [&](int k, int st) {
        float (*yr)[TC][FMAX] = Yr(st);
        float (*yi)[TC][FMAX] = Yi(st);
        for (int i = tid; i < 2 * CB * TC * FMAX; i += NT) {
            const int m = i % FMAX, r = i / FMAX;
            const int t = r % TC, cp = r / TC;
            const int c = cp % CB, plane = cp / CB;
            const int tt = k * TC + t;
            const bool ok = m < nfr && tt < a.T;
            const long long p = 2 * (long long)(ok ? tt : 0) + pol;
            const float* src = a.Y + (((long long)(c0 + c) * 2 + plane) * a.n + p) * a.Kpad + un.m_lo + (ok ? m : 0);
            cp_async4(plane ? &yi[c][t][m] : &yr[c][t][m], src, ok ? 4 : 0);
        }
        cp_async_commit();
    };

    float2 acc[BG][2];
#pragma unroll
    for (int b = 0; b < BG; ++b) acc[b][0] = acc[b][1] = make_float2(0.0f, 0.0f);
    float pw[2] = {0.0f, 0.0f};
    const bool want_incoh = a.incoh != nullptr && bg == 0;

    stage(0, 0);
    for (int k = 0; k < n_chunks; ++k) {
        const int st = k & 1;
        if (k + 1 < n_chunks) stage(k + 1, st ^ 1);
        // steering phasors of 8 beams x 16 tiles for the 8 channels: one sincospi at the
        // first channel, the others by the exact ratio e^{2 pi i d}
        {
            const int t = tid / BG, b = tid % BG;
            const int tt = k * TC + t, bb = bg * BG + b;
            float2 w[CB];
            if (tt < a.T && bb < a.nb) {
                const float4 pr = __ldg(a.params + ((long long)bb * a.n + 2 * tt + pol) * a.steps + un.step);
                const int u0 = c0 - a.N / 2;
                float x = (float)u0 * pr.y;
                x -= rintf(x);
                float y = pr.x + x + (float)u0 * pr.z;
                y -= rintf(y);
                float sn, cs;
                sincospif(2.0f * y, &sn, &cs);
                w[0] = make_float2(cs, sn);
                float dd = pr.y - rintf(pr.y) + pr.z;
                sincospif(2.0f * dd, &sn, &cs);
                const float2 R = make_float2(cs, sn);
#pragma unroll
                for (int q = 1; q < CB; ++q) w[q] = cmul(w[q - 1], R);
            } else {
#pragma unroll
                for (int q = 0; q < CB; ++q) w[q] = make_float2(0.0f, 0.0f);
            }
            float2 (*W)[TC][BG] = Wt(st);
#pragma unroll
            for (int q = 0; q < CB; ++q) W[q][t][b] = w[q];
        }
        if (k + 1 < n_chunks) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();
        float (*yr)[TC][FMAX] = Yr(st);
        float (*yi)[TC][FMAX] = Yi(st);
        float2 (*W)[TC][BG] = Wt(st);
#pragma unroll 4
        for (int t = 0; t < TC; ++t) {
            const float2 r2 = *reinterpret_cast<const float2*>(&yr[ch][t][2 * fg]);
            const float2 i2 = *reinterpret_cast<const float2*>(&yi[ch][t][2 * fg]);
            const float y_r[2] = {r2.x, r2.y}, y_i[2] = {i2.x, i2.y};
#pragma unroll
            for (int b2 = 0; b2 < BG / 2; ++b2) {
                const float4 ww = *reinterpret_cast<const float4*>(&W[ch][t][2 * b2]);
                const float2 wv[2] = {make_float2(ww.x, ww.y), make_float2(ww.z, ww.w)};
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int f = 0; f < 2; ++f) {
                        float2& s = acc[2 * b2 + h][f];
                        s.x = fmaf(wv[h].x, y_r[f], fmaf(-wv[h].y, y_i[f], s.x));
                        s.y = fmaf(wv[h].x, y_i[f], fmaf(wv[h].y, y_r[f], s.y));
                    }
            }
            if (want_incoh) {
#pragma unroll
                for (int f = 0; f < 2; ++f) pw[f] = fmaf(y_r[f], y_r[f], fmaf(y_i[f], y_i[f], pw[f]));
            }
        }
        __syncthreads();   // stage st is refilled two iterations on
    }

    const int c = c0 + ch;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const int m = 2 * fg + f;
        if (m >= nfr) continue;
        const long long fr = a.f0 + un.m_lo + m;   // frame in the call
#pragma unroll
        for (int b = 0; b < BG; ++b) {
            const int bb = bg * BG + b;
            if (bb < a.nb) a.beams[(((long long)bb * 2 + pol) * a.frames + fr) * a.N + c] = acc[b][f];
        }
        if (want_incoh && a.int_frames > 0) {
            const long long w = fr / a.int_frames;
            if (w < a.n_det) atomicAdd(a.incoh + (w * 2 + pol) * a.N + c, pw[f]);
        }
    }
}

// Stokes I of each beam summed over the frames of each detection interval.
__global__ void detect_kernel(const float2* __restrict__ beams, float* __restrict__ power, int nb, long long frames,
                              int N, int int_frames, long long n_det)
{
    const long long total = (long long)nb * n_det * N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % N);
        const long long r = i / N;
        const long long w = r % n_det;
        const int b = (int)(r / n_det);
        float s = 0.0f;
        for (int a = 0; a < 2; ++a) {
            const float2* row = beams + ((long long)b * 2 + a) * frames * N;
            for (long long m = w * int_frames; m < (w + 1) * int_frames; ++m) {
                const float2 v = row[m * N + c];
                s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
            }
        }
        power[i] = s;
    }
}

}  // namespace
}  // namespace mwax

using namespace mwax;

struct mwax_beamformer {
    mwax_beam_desc desc;
    int T = 0, n = 0, N = 0, nb = 0, bs = 0, int_frames = 0;
    long long S = 0, frames = 0, tab_step = 0, n_det = 0, Kc = 0, Kpad = 0;
    double fs = 0.0, nu = 0.0;
    float* Y = nullptr;
    float2* tw = nullptr;
    float* gain = nullptr;
    float4* params = nullptr;
    size_t params_cap = 0;
    double* d_tab = nullptr;
    size_t tab_cap = 0;
    BeamUnit* units = nullptr;
    long long units_cap = 0;
    std::vector<BeamUnit> h_units;
    cudaStream_t stream = nullptr;
    int device = 0;
    long long launches = 0;
};

namespace {

void free_beam(mwax_beamformer* b)
{
    if (!b) return;
    cudaFree(b->Y);
    cudaFree(b->tw);
    cudaFree(b->gain);
    cudaFree(b->params);
    cudaFree(b->d_tab);
    cudaFree(b->units);
    delete b;
}

#define BEAM_CUDA(call)                                                  \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);             \
    } while (0)

mwax_status beam_setup(mwax_beamformer* b, const mwax_beam_desc& d)
{
    if (d.n_tiles < 1) return set_error(MWAX_EINVAL, "n_tiles must be >= 1");
    if (d.n_beams < 1) return set_error(MWAX_EINVAL, "n_beams must be >= 1");
    if (d.fft_len < 16 || d.fft_len % CB || !fft_len_supported(d.fft_len))
        return set_error(MWAX_EUNSUPPORTED, "beamformer fft_len must be a built FFT length >= 16");
    const int bs = d.block_samples ? d.block_samples : kDefaultBlock;
    if (bs % d.fft_len) return set_error(MWAX_EINVAL, "block_samples must be a multiple of fft_len");
    if (d.samples_per_call < 1 || d.samples_per_call % bs)
        return set_error(MWAX_EINVAL, "samples_per_call must be a whole number of blocks");
    if (d.sample_rate_hz < 0.0) return set_error(MWAX_EINVAL, "sample_rate_hz must be >= 0");
    if (d.table_step_samples < 0 || d.int_frames < 0) return set_error(MWAX_EINVAL, "negative table step or int_frames");
    b->desc = d;
    b->T = d.n_tiles;
    b->n = 2 * d.n_tiles;
    b->N = d.fft_len;
    b->nb = d.n_beams;
    b->bs = bs;
    b->S = d.samples_per_call;
    b->frames = b->S / b->N;
    b->fs = d.sample_rate_hz > 0.0 ? d.sample_rate_hz : kFs;
    b->nu = d.sky_freq_hz;
    b->tab_step = d.table_step_samples ? d.table_step_samples : 6400;
    b->int_frames = d.int_frames;
    b->n_det = d.int_frames > 0 ? b->frames / d.int_frames : 0;
    BEAM_CUDA(cudaGetDevice(&b->device));

    // spectra of a chunk of frames: workspace_limit (default 4 GiB) of FP32 operands
    const size_t limit = d.workspace_limit ? d.workspace_limit : ((size_t)4 << 30);
    const size_t per_frame = (size_t)b->N * 2 * b->n * sizeof(float);
    long long kc = (long long)(limit / per_frame) / kKAlign * kKAlign;
    if (kc < kKAlign) return set_error(MWAX_ENOMEM, "workspace_limit too small for 128 frames");
    const long long need = (b->frames + kKAlign - 1) / kKAlign * kKAlign;
    b->Kc = std::min(kc, need);
    b->Kpad = b->Kc;
    BEAM_CUDA(cudaMalloc(&b->Y, per_frame * (size_t)b->Kpad));
    BEAM_CUDA(cudaMemset(b->Y, 0, per_frame * (size_t)b->Kpad));
    std::vector<float2> tw(b->N);
    for (int k = 0; k < b->N; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)b->N;
        tw[k] = make_float2((float)cos(ang), (float)sin(ang));
    }
    BEAM_CUDA(cudaMalloc(&b->tw, sizeof(float2) * b->N));
    BEAM_CUDA(cudaMemcpy(b->tw, tw.data(), sizeof(float2) * b->N, cudaMemcpyHostToDevice));
    std::vector<float> ones(b->N, 1.0f);
    BEAM_CUDA(cudaMalloc(&b->gain, sizeof(float) * b->N));
    BEAM_CUDA(cudaMemcpy(b->gain, ones.data(), sizeof(float) * b->N, cudaMemcpyHostToDevice));
    b->units_cap = b->Kc + 64;
    BEAM_CUDA(cudaMalloc(&b->units, sizeof(BeamUnit) * b->units_cap));
    return MWAX_OK;
}

// Work units of frames [f0, f0 + nfr): per table step, its frames in pieces of FMAX.
void build_units(const mwax_beamformer* b, long long f0, long long nfr, long long steps, std::vector<BeamUnit>& u)
{
    u.clear();
    long long m = 0;
    while (m < nfr) {
        const long long fr = f0 + m;
        long long step = (2 * fr * b->N + b->N) / (2 * b->tab_step);
        if (step >= steps) step = steps - 1;
        long long e = m + 1;
        while (e < nfr && e - m < FMAX) {
            long long s2 = (2 * (f0 + e) * b->N + b->N) / (2 * b->tab_step);
            if (s2 >= steps) s2 = steps - 1;
            if (s2 != step) break;
            ++e;
        }
        u.push_back(BeamUnit{(int)m, (int)e, step});
        m = e;
    }
}

}  // namespace

extern "C" {

mwax_beamformer* mwax_beam_create(const mwax_beam_desc* desc)
{
    if (!desc) {
        set_error(MWAX_EINVAL, "desc is NULL");
        return nullptr;
    }
    mwax_beamformer* b = new mwax_beamformer();
    if (beam_setup(b, *desc) != MWAX_OK) {
        free_beam(b);
        return nullptr;
    }
    return b;
}

mwax_status mwax_beam_set_stream(mwax_beamformer* b, void* stream)
{
    if (!b) return set_error(MWAX_EINVAL, "beamformer is NULL");
    b->stream = (cudaStream_t)stream;
    return MWAX_OK;
}

size_t mwax_beam_output_bytes(const mwax_beamformer* b, int which)
{
    if (!b) return 0;
    switch (which) {
        case 0: return (size_t)b->nb * 2 * b->frames * b->N * sizeof(float2);
        case 1: return (size_t)b->nb * b->n_det * b->N * sizeof(float);
        case 2: return (size_t)b->n_det * 2 * b->N * sizeof(float);
        default: return 0;
    }
}

mwax_status mwax_beam_form(mwax_beamformer* b, const int8_t* volt, const double* beam_delay, long long steps,
                           void* beams_out, float* power_out, float* incoh_out)
{
    if (!b || !volt || !beam_delay || !beams_out) return set_error(MWAX_EINVAL, "NULL beamformer, voltages, delays or beams_out");
    if (steps < 1) return set_error(MWAX_EINVAL, "table_steps must be >= 1");
    if ((power_out || incoh_out) && b->n_det < 1)
        return set_error(MWAX_EINVAL, "detected outputs need int_frames in [1, frames]");
    if (((uintptr_t)volt & 15) || ((uintptr_t)beams_out & 15))
        return set_error(MWAX_EINVAL, "voltages and beams_out must be 16-byte aligned");
    cudaStream_t s = b->stream;
    BEAM_CUDA(cudaSetDevice(b->device));

    // steering tables -> per (beam, path, step) phase terms
    const size_t entries = (size_t)b->nb * b->n * steps;
    if (entries * sizeof(double) > b->tab_cap) {
        cudaFree(b->d_tab);
        cudaFree(b->params);
        b->d_tab = nullptr;
        b->params = nullptr;
        b->tab_cap = 0;
        BEAM_CUDA(cudaMalloc(&b->d_tab, entries * sizeof(double)));
        BEAM_CUDA(cudaMalloc(&b->params, entries * sizeof(float4)));
        b->tab_cap = entries * sizeof(double);
    }
    BEAM_CUDA(cudaMemcpyAsync(b->d_tab, beam_delay, entries * sizeof(double), cudaMemcpyDefault, s));
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, beam_delay) == cudaSuccess && at.type == cudaMemoryTypeHost)
        BEAM_CUDA(cudaStreamSynchronize(s));
    cudaGetLastError();
    beam_params_kernel<<<2 * 148, 256, 0, s>>>(b->d_tab, (long long)entries, b->nu, b->fs, b->N, b->params);
    BEAM_CUDA(cudaGetLastError());
    if (incoh_out) BEAM_CUDA(cudaMemsetAsync(incoh_out, 0, mwax_beam_output_bytes(b, 2), s));

    for (long long f0 = 0; f0 < b->frames; f0 += b->Kc) {
        const long long nfr = std::min(b->Kc, b->frames - f0);
        FArgs fa;
        memset(&fa, 0, sizeof fa);
        fa.volt = volt;
        fa.Y = b->Y;
        fa.tw = b->tw;
        fa.gain = b->gain;
        fa.m_begin = f0;
        fa.n_frames = nfr;
        fa.n_store = nfr;
        fa.Kc = b->Kpad;
        fa.Kpad = b->Kpad;
        fa.n = b->n;
        fa.bs = b->bs;
        fa.nu = b->nu;
        fa.fs = b->fs;
        BEAM_CUDA(launch_fstep(b->N, FOUT_F32, fa, s, 0));
        build_units(b, f0, nfr, steps, b->h_units);
        BEAM_CUDA(cudaMemcpyAsync(b->units, b->h_units.data(), sizeof(BeamUnit) * b->h_units.size(),
                                  cudaMemcpyHostToDevice, s));
        BeamArgs ba;
        ba.Y = b->Y;
        ba.params = b->params;
        ba.units = b->units;
        ba.beams = static_cast<float2*>(beams_out);
        ba.incoh = incoh_out;
        ba.Kpad = b->Kpad;
        ba.steps = steps;
        ba.frames = b->frames;
        ba.f0 = f0;
        ba.T = b->T;
        ba.n = b->n;
        ba.N = b->N;
        ba.nb = b->nb;
        ba.int_frames = b->int_frames;
        ba.n_det = b->n_det;
        dim3 grid((unsigned)b->h_units.size(), (unsigned)(b->N / CB), (unsigned)(2 * ((b->nb + BG - 1) / BG)));
        static bool attr_done = false;
        if (!attr_done) {
            BEAM_CUDA(cudaFuncSetAttribute(beam_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBeamSmem));
            attr_done = true;
        }
        beam_kernel<<<grid, NT, kBeamSmem, s>>>(ba);
        BEAM_CUDA(cudaGetLastError());
        b->launches += 2;
    }
    if (power_out) {
        detect_kernel<<<4 * 148, 256, 0, s>>>(static_cast<const float2*>(beams_out), power_out, b->nb, b->frames, b->N,
                                              b->int_frames, b->n_det);
        BEAM_CUDA(cudaGetLastError());
        b->launches += 1;
    }
    return MWAX_OK;
}

mwax_status mwax_beam_sync(mwax_beamformer* b)
{
    if (!b) return set_error(MWAX_EINVAL, "beamformer is NULL");
    BEAM_CUDA(cudaSetDevice(b->device));
    BEAM_CUDA(cudaStreamSynchronize(b->stream));
    return MWAX_OK;
}

void mwax_beam_destroy(mwax_beamformer* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    free_beam(b);
}

}  // extern "C"
