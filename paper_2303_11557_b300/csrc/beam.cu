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
// Detected Stokes I is formed afterwards from the coherent beams.  That CUDA-core engine
// (FP32) is engine 1; engine 0, the default, runs the same products on the tensor cores
// (below).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "plan.cuh"
#include "tc_ptx.cuh"

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

// ------------------------------------------------------------------ tensor-core engine
// The same product on tcgen05: per (step unit of <= 64 frames, 4 consecutive channels, one
// polarisation, 16 beams) a CTA accumulates, channel by channel, D[m][b] = sum_t Y[t][m]
// W[b][t] in tensor memory (M = frames, N = beams, K = tiles in chunks of 64).  Both
// operands are staged by the CUDA cores into shared memory in the no-swizzle K-major layout
// as FP16 hi/lo pairs (v = hi + lo, 22 significant bits; the spectra pre-scaled by a power
// of two that keeps them in FP16 range, undone exactly at the end), and each complex term
// takes three FP16 products per real product (hi hi, hi lo, lo hi; the dropped lo lo is
// 2^-22 of it): the FP32 engine's accuracy on the tensor cores.  The steering phasors of
// a chunk are made once per (beam, tile) at the first channel and advanced to the next
// channel by the exact ratio e^{2 pi i tau Fs / N}.
constexpr int TM = 128;                 // MMA M (rows = frames)
constexpr int TMU = 64;                 // frames per unit (rows past it are never read back)
constexpr int TNB = 16;                 // beams per CTA (MMA N)
constexpr int TCQ = 4;                  // channels per CTA
constexpr int TKC = 64;                 // tiles per K chunk
constexpr int TNT = 256;                // threads per CTA
constexpr uint32_t T_LBO_A = 16 * 128 + 16;   // A: 128 frame rows; K core stride (+16 B: bank spread)
constexpr uint32_t T_APLANE = (TKC / 8) * T_LBO_A;
constexpr uint32_t T_LBO_B = 2 * 128 + 16;    // B: 16 beam rows
constexpr uint32_t T_BPLANE = (TKC / 8) * T_LBO_B;
constexpr size_t kBeamTcSmem = 4 * T_APLANE + 6 * T_BPLANE + sizeof(float) * TCQ * TM + 1024;

struct BeamTcShared {
    uint64_t bar;       // MMA completion
    uint64_t drained;   // after an abort: every MMA issued has completed
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ uint64_t plain_desc(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(128u >> 4) << 32;   // SBO: next 8-row group
    d |= (uint64_t)1 << 46;             // tcgen05 descriptor; no swizzle
    return d;
}

__device__ __forceinline__ uint32_t plain_at(int r, int k, uint32_t lbo)
{
    return (uint32_t)(k >> 3) * lbo + (uint32_t)(r >> 3) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void split_half(float v, __half& hi, __half& lo)
{
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));   // the difference is exact in FP32
}

__device__ __forceinline__ void beam_tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__global__ void __launch_bounds__(TNT, 2) beam_tc_kernel(const BeamArgs a, float prescale, float unscale, int* status)
{
    extern __shared__ __align__(1024) unsigned char beam_tc_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(beam_tc_raw) + 127) & ~(uintptr_t)127);
    unsigned char* Ap[4];   // yr hi, yr lo, yi hi, yi lo
    for (int i = 0; i < 4; ++i) Ap[i] = sm + i * T_APLANE;
    unsigned char* Bp[6];   // wr hi, wr lo, wi hi, wi lo, -wi hi, -wi lo
    for (int i = 0; i < 6; ++i) Bp[i] = sm + 4 * T_APLANE + i * T_BPLANE;
    float* inc = reinterpret_cast<float*>(sm + 4 * T_APLANE + 6 * T_BPLANE);   // [TCQ][TM]
    BeamTcShared& S = *reinterpret_cast<BeamTcShared*>(inc + TCQ * TM);

    const BeamUnit un = a.units[blockIdx.x];
    const int c0 = blockIdx.y * TCQ;
    const int pol = blockIdx.z & 1, bg = blockIdx.z >> 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nfr = un.m_hi - un.m_lo;
    const bool want_incoh = a.incoh != nullptr && bg == 0;
    const int n_kc = (a.T + TKC - 1) / TKC;

    for (int i = tid; i < TCQ * TM; i += TNT) inc[i] = 0.0f;
    if (tid == 0) {
        tc::mbar_init(&S.bar, 1);
        tc::mbar_init(&S.drained, 1);
        S.abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, 128);   // D of the 4 channels: (16 re + 16 im) columns each
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t idesc = tc::idesc(0, TM, TNB, false);
    uint64_t desc_a[4], desc_b[6];   // operand planes at K step 0
#pragma unroll
    for (int i = 0; i < 4; ++i) desc_a[i] = plain_desc(tc::smem_u32(Ap[i]), T_LBO_A);
#pragma unroll
    for (int i = 0; i < 6; ++i) desc_b[i] = plain_desc(tc::smem_u32(Bp[i]), T_LBO_B);
    const long long lim = (long long)tc::kDefaultSpin * 1000LL;
    uint32_t parity = 0;
    bool issued = false, waiting = false;
    // a thread's own timeout (bad) decides nothing alone: every exit is taken by all threads
    // at the same barrier, from __syncthreads_or of the threads' flags (stop)
    bool bad = false, stop = false;

    // spectra loaded one (chunk, channel) step ahead: a thread takes frames mh + 16 j of
    // the tile pairs tp0 and tp0 + 16 of the chunk, so a warp reads 64-byte runs of 4 tile
    // rows per plane; frames past the unit and tiles past T read as zero
    const int nj = (nfr + 15) >> 4;
    float yv[TMU / 16][2][2][2];   // [j][pair][tile of the pair][re, im]
    auto load_step = [&](int kc, int ci) {
        const int mh = tid & 15, tp0 = tid >> 4;
        const int c = c0 + ci;
#pragma unroll
        for (int j = 0; j < TMU / 16; ++j) {
            const int m = mh + 16 * j;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int tt = kc * TKC + 2 * (tp0 + 16 * h) + e;
                    yv[j][h][e][0] = yv[j][h][e][1] = 0.0f;
                    if (j < nj && m < nfr && tt < a.T) {
                        const long long row = ((long long)c * 2 * a.n + 2 * tt + pol) * a.Kpad + un.m_lo + m;
                        yv[j][h][e][0] = __ldg(a.Y + row);
                        yv[j][h][e][1] = __ldg(a.Y + row + (long long)a.n * a.Kpad);
                    }
                }
        }
    };
    load_step(0, 0);

    // steering role of this thread: beam b = tid / 16, tiles 4 (tid % 16) .. + 3 of a chunk
    const int wb = tid >> 4, wt4 = tid & 15;
    const int bb = bg * TNB + wb;
    for (int kc = 0; kc < n_kc && !stop; ++kc) {
        float2 w[4], R[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int tt = kc * TKC + 4 * wt4 + j;
            w[j] = R[j] = make_float2(0.0f, 0.0f);
            if (tt < a.T && bb < a.nb) {
                const float4 pr = __ldg(a.params + ((long long)bb * a.n + 2 * tt + pol) * a.steps + un.step);
                const int u0 = c0 - a.N / 2;
                float x = (float)u0 * pr.y;
                x -= rintf(x);
                float y = pr.x + x + (float)u0 * pr.z;
                y -= rintf(y);
                float sn, cs;
                sincospif(2.0f * y, &sn, &cs);
                w[j] = make_float2(cs, sn);
                const float dd = pr.y - rintf(pr.y) + pr.z;
                sincospif(2.0f * dd, &sn, &cs);
                R[j] = make_float2(cs, sn);
            }
        }
        for (int ci = 0; ci < TCQ; ++ci) {
            const int c = c0 + ci;
            // the previous MMAs read the operands about to be overwritten
            if (waiting) {
                const long long t0 = clock64();
                bool ok = true;
                while (!tc::mbar_try_wait(&S.bar, parity)) {
                    if (*reinterpret_cast<volatile int*>(&S.abort) || clock64() - t0 > lim) {
                        ok = false;
                        break;
                    }
                }
                if (ok) {
                    parity ^= 1u;
                } else {
                    bad = true;
                    S.abort = 1;   // lets the other threads' waits give up early
                    if (status) atomicOr(status, 4096);
                }
                waiting = false;
            }
            // A: Y^T (rows = frames, K = tiles) from the values loaded one step ahead, FP32 ->
            // pre-scaled FP16 hi/lo; both tiles of a pair as one 4-byte word
            {
                const int mh = tid & 15, tp0 = tid >> 4;
#pragma unroll
                for (int j = 0; j < TMU / 16; ++j) {
                    if (j >= nj) break;
                    const int m = mh + 16 * j;
                    const bool mok = m < nfr;
                    if (want_incoh) {
                        float pw = 0.0f;
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int e = 0; e < 2; ++e)
                                pw = fmaf(yv[j][h][e][0], yv[j][h][e][0], fmaf(yv[j][h][e][1], yv[j][h][e][1], pw));
                        pw += __shfl_xor_sync(0xffffffffu, pw, 16);   // lanes L, L + 16: same frame
                        if (lane < 16 && mok) atomicAdd(&inc[ci * TM + m], pw);
                    }
                    if (!mok) continue;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        __half hv[4][2];   // [yr hi, yr lo, yi hi, yi lo][tile of the pair]
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            split_half(yv[j][h][e][0] * prescale, hv[0][e], hv[1][e]);
                            split_half(yv[j][h][e][1] * prescale, hv[2][e], hv[3][e]);
                        }
                        const uint32_t o = plain_at(m, 2 * (tp0 + 16 * h), T_LBO_A);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            *reinterpret_cast<__half2*>(Ap[i] + o) = __halves2half2(hv[i][0], hv[i][1]);
                    }
                }
            }
            // B: the steering phasors of this channel (rows = beams, K = tiles)
            {
                __half hr[2][4], hi[2][4], hn[2][4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    split_half(w[j].x, hr[0][j], hr[1][j]);
                    split_half(w[j].y, hi[0][j], hi[1][j]);
                    split_half(-w[j].y, hn[0][j], hn[1][j]);
                    w[j] = cmul(w[j], R[j]);   // next channel
                }
                const uint32_t o = plain_at(wb, 4 * wt4, T_LBO_B);
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    *reinterpret_cast<uint2*>(Bp[0 + l] + o) = *reinterpret_cast<const uint2*>(hr[l]);
                    *reinterpret_cast<uint2*>(Bp[2 + l] + o) = *reinterpret_cast<const uint2*>(hi[l]);
                    *reinterpret_cast<uint2*>(Bp[4 + l] + o) = *reinterpret_cast<const uint2*>(hn[l]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::fence_before();
            if ((stop = __syncthreads_or(bad))) break;
            if (tid == 0) {
                tc::fence_after();
                const uint32_t dre = tmem + 32u * ci, dim = dre + 16u;
#pragma unroll
                for (int ks = 0; ks < TKC / 16; ++ks) {
                    const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                    // the start address field counts 16-byte units: step ks is 2 K core columns on
                    uint64_t da[4], db[6];
#pragma unroll
                    for (int i = 0; i < 4; ++i) da[i] = desc_a[i] + (uint64_t)((ks * 2u * T_LBO_A) >> 4);
#pragma unroll
                    for (int i = 0; i < 6; ++i) db[i] = desc_b[i] + (uint64_t)((ks * 2u * T_LBO_B) >> 4);
                    // re: yr wr - yi wi;  im: yr wi + yi wr  (hi hi, hi lo, lo hi of each)
                    tc::mma_f16(dre, da[0], db[0], idesc, acc);
                    tc::mma_f16(dre, da[0], db[1], idesc, 1u);
                    tc::mma_f16(dre, da[1], db[0], idesc, 1u);
                    tc::mma_f16(dre, da[2], db[4], idesc, 1u);
                    tc::mma_f16(dre, da[2], db[5], idesc, 1u);
                    tc::mma_f16(dre, da[3], db[4], idesc, 1u);
                    tc::mma_f16(dim, da[0], db[2], idesc, acc);
                    tc::mma_f16(dim, da[0], db[3], idesc, 1u);
                    tc::mma_f16(dim, da[1], db[2], idesc, 1u);
                    tc::mma_f16(dim, da[2], db[0], idesc, 1u);
                    tc::mma_f16(dim, da[2], db[1], idesc, 1u);
                    tc::mma_f16(dim, da[3], db[0], idesc, 1u);
                }
                tc::mma_commit(&S.bar);
                issued = true;
            }
            waiting = true;
            // the next step's spectra load while these MMAs run
            if (ci + 1 < TCQ) load_step(kc, ci + 1);
            else if (kc + 1 < n_kc) load_step(kc + 1, 0);
        }
    }
    if (waiting && !stop) {
        const long long t0 = clock64();
        bool ok = true;
        while (!tc::mbar_try_wait(&S.bar, parity)) {
            if (*reinterpret_cast<volatile int*>(&S.abort) || clock64() - t0 > lim) {
                ok = false;
                break;
            }
        }
        if (!ok) {
            bad = true;
            S.abort = 1;
            if (status) atomicOr(status, 4096);
        }
    }
    tc::fence_after();
    stop = __syncthreads_or(bad);

    // epilogue: row m = 32 (warp % 4) + lane, beams 8 (warp / 4) .. + 7; four channels per
    // beam and frame are one 32-byte store
    if (!stop) {
        const int q = warp & 3, h = warp >> 2;
        const int m = 32 * q + lane;
        const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
        float2 v[TCQ][8];
#pragma unroll
        for (int ci = 0; ci < TCQ; ++ci) {
            uint32_t re[8], im[8];
            beam_tmem_ld8(tq + 32u * ci + 8u * h, re);
            beam_tmem_ld8(tq + 32u * ci + 16u + 8u * h, im);
            tc::tmem_wait_ld();
#pragma unroll
            for (int b = 0; b < 8; ++b)
                v[ci][b] = make_float2(__uint_as_float(re[b]) * unscale, __uint_as_float(im[b]) * unscale);
        }
        if (m < nfr) {
            const long long fr = a.f0 + un.m_lo + m;   // frame in the call
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int beam = bg * TNB + 8 * h + b;
                if (beam >= a.nb) continue;
                float4* dst = reinterpret_cast<float4*>(a.beams + (((long long)beam * 2 + pol) * a.frames + fr) * a.N + c0);
                dst[0] = make_float4(v[0][b].x, v[0][b].y, v[1][b].x, v[1][b].y);
                dst[1] = make_float4(v[2][b].x, v[2][b].y, v[3][b].x, v[3][b].y);
            }
        }
    }
    if (!stop && want_incoh && a.int_frames > 0)
        for (int i = tid; i < TCQ * nfr; i += TNT) {
            const int ci = i / nfr, m = i % nfr;
            const long long fr = a.f0 + un.m_lo + m;
            const long long wdet = fr / a.int_frames;
            if (wdet < a.n_det) atomicAdd(a.incoh + (wdet * 2 + pol) * a.N + c0 + ci, inc[ci * TM + m]);
        }

    if (tid == 0 && stop && issued) {
        tc::mma_commit(&S.drained);
        if (!tc::wait_bounded(&S.drained, 0u, tc::kDrainCycles) && status) atomicOr(status, tc::kDrainGaveUp);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 128);
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
    int* status = nullptr;    // bounded waits of the tensor-core engine
    int engine = 0;           // 0: tcgen05 (FP16 hi/lo pairs), 1: FP32 CUDA cores
    float prescale = 1.0f;    // power of two keeping the spectra in FP16 range (engine 0)
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
    cudaFree(b->status);
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
    if (d.engine != 0 && d.engine != 1) return set_error(MWAX_EINVAL, "engine must be 0 (tensor cores) or 1 (CUDA cores)");
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
    b->engine = d.engine;
    // |Re Y|, |Im Y| <= 128 sqrt(2) N: scaled by 2^-k below 2^15 for the FP16 operands
    while (181.0 * b->N * b->prescale > 32768.0) b->prescale *= 0.5f;
    BEAM_CUDA(cudaGetDevice(&b->device));
    BEAM_CUDA(cudaMalloc(&b->status, sizeof(int)));
    BEAM_CUDA(cudaMemset(b->status, 0, sizeof(int)));

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

// Work units of frames [f0, f0 + nfr): per table step, its frames in pieces of at most
// fmax (32 for the CUDA-core engine, 64 for the tensor-core engine).
void build_units(const mwax_beamformer* b, long long f0, long long nfr, long long steps, int fmax,
                 std::vector<BeamUnit>& u)
{
    u.clear();
    long long m = 0;
    while (m < nfr) {
        const long long fr = f0 + m;
        long long step = (2 * fr * b->N + b->N) / (2 * b->tab_step);
        if (step >= steps) step = steps - 1;
        long long e = m + 1;
        while (e < nfr && e - m < fmax) {
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
        build_units(b, f0, nfr, steps, b->engine == 0 ? TMU : FMAX, b->h_units);
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
        if (b->engine == 0) {
            dim3 grid((unsigned)b->h_units.size(), (unsigned)(b->N / TCQ), (unsigned)(2 * ((b->nb + TNB - 1) / TNB)));
            static bool tc_attr_done = false;
            if (!tc_attr_done) {
                BEAM_CUDA(cudaFuncSetAttribute(beam_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kBeamTcSmem));
                tc_attr_done = true;
            }
            beam_tc_kernel<<<grid, TNT, kBeamTcSmem, s>>>(ba, b->prescale, 1.0f / b->prescale, b->status);
        } else {
            dim3 grid((unsigned)b->h_units.size(), (unsigned)(b->N / CB), (unsigned)(2 * ((b->nb + BG - 1) / BG)));
            static bool attr_done = false;
            if (!attr_done) {
                BEAM_CUDA(cudaFuncSetAttribute(beam_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBeamSmem));
                attr_done = true;
            }
            beam_kernel<<<grid, NT, kBeamSmem, s>>>(ba);
        }
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
    int st = 0;
    BEAM_CUDA(cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        BEAM_CUDA(cudaMemset(b->status, 0, sizeof(int)));
        return set_error(MWAX_ETIMEOUT, "a device-side bounded wait of the beamformer gave up");
    }
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
