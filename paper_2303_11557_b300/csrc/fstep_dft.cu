// Tensor-core F-step for the short fine-channel FFTs (Sec. 2.5.1, N = 32, 64, 128): the
// N-point DFT of 128 frames at once as one matrix product on tcgen05,
//     D[f][k] = sum_n x_f[n] e^{-2 pi i k n / N}      (M = 128 frames, N = N bins, K = N samples)
// then, per frame and bin, the delay phasor (Sec. 4.3), the channel gain (averaging weight,
// passband, FP16 pre-scale) and the store of the K-major operand planes
// Y[slot][c][plane][p][Kpad], c = fftshift(k), as the CUDA-core F-steps do.
//
// The frames' int8 samples are exact in FP16 (the A operand, one frame per row, samples
// along K: the voltages' own order).  The DFT matrix (the B operand) is FP16 for FP16
// operands out (2^-12 per entry, below the FP16 rounding of the result), and an FP16 hi/lo
// pair (F = hi + lo, 2^-23) for FP32 and FP16 hi/lo operands out: two products per real
// product, FP32-level spectra.  Complex products on planar operands with the A-negate bit
// for the -Im(x) Im(F) term.
//
// A persistent CTA per SM runs four roles on items of 128 consecutive frames of one signal
// path, connected by mbarriers (every wait bounded):
//   thread 0        bulk-copies the next item's int8 frames into the stage;
//   warps 0-3       convert the stage into the A operand (FP16, no-swizzle K-major);
//   warp 4 lane 0   issues the MMAs into one of two tensor-memory accumulators;
//   warps 5-12      read an accumulator (lane = frame), apply phasor and gain, store: a
//                   warp writes 32 consecutive frames of one operand row at a time.
// Converting item i + 1 overlaps the MMAs and the stores of item i.
#include "mwax_internal.cuh"
#include "tc_ptx.cuh"

namespace mwax {
namespace {

constexpr int kFrames = 128;      // frames per item (MMA M)
constexpr int kConv = 128;        // converter threads (warps 0-3)
constexpr int kEpi = 256;         // epilogue threads (warps 5-12)
constexpr int kThreads = 416;

template <int N, int OUTK>
struct Dft {
    static constexpr bool PAIR = OUTK != FOUT_F16;         // hi/lo DFT matrix: two products
    static constexpr int NB = PAIR ? 4 : 2;                // B planes: Fr, Fi (, Fr lo, Fi lo)
    static constexpr uint32_t LBO_A = 16 * 128 + 16;       // A: 128 frame rows per K core column
    static constexpr uint32_t APLANE = (N / 8) * LBO_A;
    static constexpr uint32_t LBO_B = (N / 8) * 128;       // B: N bin rows per K core column
    static constexpr uint32_t BPLANE = (N / 8) * LBO_B;
    static constexpr uint32_t STAGE = kFrames * N * 2;     // int8 (re, im) of the item's frames
    static constexpr uint32_t DCOLS = 2 * N;               // one accumulator: re, im
    static constexpr uint32_t TMEM = 4 * N <= 32 ? 32u : (4 * N <= 64 ? 64u : (4 * N <= 128 ? 128u : (4 * N <= 256 ? 256u : 512u)));
    static constexpr size_t SMEM = 2 * APLANE + NB * BPLANE + STAGE + sizeof(float) * N + 1024;
    static_assert(N % 16 == 0 && N <= 128, "bins per MMA");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct DftShared {
    uint64_t st_full, st_empty;   // stage: copied / read by the converters
    uint64_t a_full, a_empty;     // A operand: written / read by the MMAs
    uint64_t d_full[2], d_empty[2];
    uint64_t drained;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ uint64_t desc_plain(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(128u >> 4) << 32;   // SBO: next 8-row group
    d |= (uint64_t)1 << 46;             // tcgen05 descriptor, no swizzle
    return d;
}

__device__ __forceinline__ uint32_t plain_off(int r, int k, uint32_t lbo)
{
    return (uint32_t)(k >> 3) * lbo + (uint32_t)(r >> 3) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) { tc::tmem_ld16(taddr, r); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// e^{2 pi i (phi0 + u d)}, d = d_hi + d_lo with d_hi holding 12 significant bits (|u| < 4096).
__device__ __forceinline__ float2 phasor_u(float phi0, float d_hi, float d_lo, int u)
{
    const float uf = (float)u;
    float x = uf * d_hi;
    x -= rintf(x);
    float y = phi0 + x + uf * d_lo;
    y -= rintf(y);
    float s, c;
    sincospif(2.0f * y, &s, &c);
    return make_float2(c, s);
}

// Bounded wait; on expiry raises the abort flag and records the status bit.
__device__ __forceinline__ bool wait_phase(DftShared& S, uint64_t* bar, uint32_t parity, int* status, int code)
{
    const long long lim = (long long)tc::kDefaultSpin * 1000LL;
    if (tc::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*reinterpret_cast<volatile int*>(&S.abort)) return false;
        if (clock64() - t0 > lim) {
            S.abort = 1;
            if (status) atomicOr(status, code);
            return false;
        }
    }
    return true;
}

// Frame f of item `item` (path, first frame).
__device__ __forceinline__ void item_of(const FArgs& a, long long item, int* p, long long* f0)
{
    const long long n_fb = (a.n_store + kFrames - 1) / kFrames;
    *p = (int)(item / n_fb);
    *f0 = (item % n_fb) * kFrames;
}

template <int N>
__device__ __forceinline__ bool frame_has_data(const FArgs& a, int p, long long f)
{
    return f < a.n_frames && !frame_zeroed(a, p, (a.m_begin + f) * (long long)N);
}

template <int N, int OUTK>
__device__ __forceinline__ void store_value(const FArgs& a, long long at, long long ps, float2 v)
{
    if (OUTK == FOUT_F32) {
        float* Y = static_cast<float*>(a.Y);
        Y[at] = v.x;
        Y[at + ps] = v.y;
    } else if (OUTK == FOUT_F16) {
        __half* Y = static_cast<__half*>(a.Y);
        Y[at] = __float2half_rn(v.x);
        Y[at + ps] = __float2half_rn(v.y);
    } else {   // FP16 hi/lo pairs: lo values half a row further on
        __half* Y = static_cast<__half*>(a.Y);
        const long long lo = a.Kpad >> 1;
        const __half hr = __float2half_rn(v.x), hi = __float2half_rn(v.y);
        Y[at] = hr;
        Y[at + ps] = hi;
        Y[at + lo] = __float2half_rn(v.x - __half2float(hr));
        Y[at + ps + lo] = __float2half_rn(v.y - __half2float(hi));
    }
}

template <int N, int OUTK>
__global__ void __launch_bounds__(kThreads, 1) fstep_dft_kernel(const FArgs a, long long n_items)
{
    using C = Dft<N, OUTK>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    unsigned char* a_re = sm;
    unsigned char* a_im = a_re + C::APLANE;
    unsigned char* bpl = a_im + C::APLANE;                        // Fr hi, Fi hi (, Fr lo, Fi lo)
    int8_t* stage = reinterpret_cast<int8_t*>(bpl + C::NB * C::BPLANE);
    float* gain = reinterpret_cast<float*>(stage + C::STAGE);
    DftShared& S = *reinterpret_cast<DftShared*>(gain + N);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int* status = a.status;

    // ---- set-up: the DFT matrix (B: rows = bins k, K = samples n), gains, barriers, TMEM
    for (int e = tid; e < N * N; e += kThreads) {
        const int k = e / N, n = e % N;
        double s, c;
        sincospi(-2.0 * (double)((k * n) % N) / (double)N, &s, &c);
        const uint32_t o = plain_off(k, n, C::LBO_B);
        const __half hr = __double2half(c), hi = __double2half(s);
        *reinterpret_cast<__half*>(bpl + o) = hr;
        *reinterpret_cast<__half*>(bpl + C::BPLANE + o) = hi;
        if (C::PAIR) {
            *reinterpret_cast<__half*>(bpl + 2 * C::BPLANE + o) = __double2half(c - (double)__half2float(hr));
            *reinterpret_cast<__half*>(bpl + 3 * C::BPLANE + o) = __double2half(s - (double)__half2float(hi));
        }
    }
    for (int i = tid; i < N; i += kThreads) gain[i] = __ldg(&a.gain[i]);
    if (tid == 0) {
        tc::mbar_init(&S.st_full, 1);
        tc::mbar_init(&S.st_empty, kConv);
        tc::mbar_init(&S.a_full, kConv);
        tc::mbar_init(&S.a_empty, 1);
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&S.d_full[b], 1);
            tc::mbar_init(&S.d_empty[b], kEpi);
        }
        tc::mbar_init(&S.drained, 1);
        S.abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 4) {
        tc::tmem_alloc(&S.tmem, C::TMEM);
        tc::tmem_relinquish();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B written by the generic proxy
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;

    if (warp < 4) {
        // ------------------------------------------------ producer (thread 0) + converters
        bool pending = false;   // thread 0: a bulk copy not yet waited for
        uint32_t it = 0;
        // first item's frames
        if (tid == 0 && blockIdx.x < n_items) {
            int p;
            long long f0;
            item_of(a, blockIdx.x, &p, &f0);
            uint32_t bytes = 0;
            for (int f = 0; f < kFrames && f0 + f < a.n_frames; ++f)
                if (frame_has_data<N>(a, p, f0 + f)) bytes += 2 * N;
            tc::mbar_arrive_expect_tx(&S.st_full, bytes);
            for (int f = 0; f < kFrames && f0 + f < a.n_frames;) {
                if (!frame_has_data<N>(a, p, f0 + f)) {
                    ++f;
                    continue;
                }
                // a run of frames inside one data block
                const long long s0 = (a.m_begin + f0 + f) * (long long)N;
                const long long blk = s0 / a.bs, off = s0 % a.bs;
                int run = 1;
                while (f + run < kFrames && f0 + f + run < a.n_frames && (off + (long long)run * N) < a.bs &&
                       !frame_zeroed(a, p, s0 + (long long)run * N))
                    ++run;
                bulk_copy(stage + f * 2 * N, a.volt + ((blk * a.n + p) * (long long)a.bs + off) * 2, (uint32_t)run * 2 * N,
                          &S.st_full);
                f += run;
            }
            pending = true;
        }
        for (long long item = blockIdx.x; item < n_items; item += gridDim.x, ++it) {
            int p;
            long long f0;
            item_of(a, item, &p, &f0);
            if (!wait_phase(S, &S.st_full, it & 1, status, 2048)) break;
            if (tid == 0) pending = false;
            // the A operand is free once the previous item's MMAs completed
            if (it > 0 && !wait_phase(S, &S.a_empty, (it - 1) & 1, status, 2048)) break;
            // 8-sample chunks: a warp reads 512 contiguous stage bytes per step
            constexpr int CH = N / 8;
            for (int e = tid; e < kFrames * CH; e += kConv) {
                const int f = e / CH, kk = e % CH;
                int4 raw = make_int4(0, 0, 0, 0);
                if (frame_has_data<N>(a, p, f0 + f)) raw = *reinterpret_cast<const int4*>(stage + (f * CH + kk) * 16);
                const uint32_t w[4] = {(uint32_t)raw.x, (uint32_t)raw.y, (uint32_t)raw.z, (uint32_t)raw.w};
                uint32_t hr[4], hi[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __half2 r2 = __halves2half2(__int2half_rn((int)(int8_t)(w[q])), __int2half_rn((int)(int8_t)(w[q] >> 16)));
                    const __half2 i2 = __halves2half2(__int2half_rn((int)(int8_t)(w[q] >> 8)), __int2half_rn((int)(int8_t)(w[q] >> 24)));
                    hr[q] = *reinterpret_cast<const uint32_t*>(&r2);
                    hi[q] = *reinterpret_cast<const uint32_t*>(&i2);
                }
                const uint32_t o = plain_off(f, 8 * kk, C::LBO_A);
                *reinterpret_cast<uint4*>(a_re + o) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
                *reinterpret_cast<uint4*>(a_im + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::mbar_arrive(&S.st_empty);
            tc::mbar_arrive(&S.a_full);
            // thread 0: the next item's frames into the stage once every converter has read it
            const long long next = item + gridDim.x;
            if (tid == 0 && next < n_items) {
                if (!wait_phase(S, &S.st_empty, it & 1, status, 2048)) break;
                int pn;
                long long fn;
                item_of(a, next, &pn, &fn);
                uint32_t bytes = 0;
                for (int f = 0; f < kFrames && fn + f < a.n_frames; ++f)
                    if (frame_has_data<N>(a, pn, fn + f)) bytes += 2 * N;
                tc::mbar_arrive_expect_tx(&S.st_full, bytes);
                for (int f = 0; f < kFrames && fn + f < a.n_frames;) {
                    if (!frame_has_data<N>(a, pn, fn + f)) {
                        ++f;
                        continue;
                    }
                    const long long s0 = (a.m_begin + fn + f) * (long long)N;
                    const long long blk = s0 / a.bs, off = s0 % a.bs;
                    int run = 1;
                    while (f + run < kFrames && fn + f + run < a.n_frames && (off + (long long)run * N) < a.bs &&
                           !frame_zeroed(a, pn, s0 + (long long)run * N))
                        ++run;
                    bulk_copy(stage + f * 2 * N, a.volt + ((blk * a.n + pn) * (long long)a.bs + off) * 2,
                              (uint32_t)run * 2 * N, &S.st_full);
                    f += run;
                }
                pending = true;
            }
        }
        // a bulk copy still in flight lands before the CTA can exit
        if (tid == 0 && pending && !tc::wait_bounded(&S.st_full, it & 1, tc::kDrainCycles) && status)
            atomicOr(status, tc::kDrainGaveUp);
    } else if (warp == 4) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool issued = false;
            uint32_t it = 0;
            const uint32_t idesc = tc::idesc(0, kFrames, N, false), idesc_neg = tc::idesc(0, kFrames, N, true);
            const uint64_t dar = desc_plain(tc::smem_u32(a_re), C::LBO_A), dai = desc_plain(tc::smem_u32(a_im), C::LBO_A);
            uint64_t db[4];
            for (int i = 0; i < C::NB; ++i) db[i] = desc_plain(tc::smem_u32(bpl + i * C::BPLANE), C::LBO_B);
            for (long long item = blockIdx.x; item < n_items; item += gridDim.x, ++it) {
                const int b = it & 1;
                if (!wait_phase(S, &S.a_full, it & 1, status, 2048)) break;
                if (it >= 2 && !wait_phase(S, &S.d_empty[b], ((it >> 1) - 1) & 1, status, 2048)) break;
                tc::fence_after();
                const uint32_t dre = tmem + b * C::DCOLS, dim = dre + N;
#pragma unroll
                for (int ks = 0; ks < N / 16; ++ks) {
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    const uint64_t oa = (uint64_t)((ks * 2u * C::LBO_A) >> 4), ob = (uint64_t)((ks * 2u * C::LBO_B) >> 4);
                    // re = xr Fr - xi Fi,  im = xr Fi + xi Fr  (hi, then lo parts of F)
                    tc::mma_f16(dre, dar + oa, db[0] + ob, idesc, acc);
                    tc::mma_f16(dre, dai + oa, db[1] + ob, idesc_neg, 1u);
                    tc::mma_f16(dim, dar + oa, db[1] + ob, idesc, acc);
                    tc::mma_f16(dim, dai + oa, db[0] + ob, idesc, 1u);
                    if (C::PAIR) {
                        tc::mma_f16(dre, dar + oa, db[2] + ob, idesc, 1u);
                        tc::mma_f16(dre, dai + oa, db[3] + ob, idesc_neg, 1u);
                        tc::mma_f16(dim, dar + oa, db[3] + ob, idesc, 1u);
                        tc::mma_f16(dim, dai + oa, db[2] + ob, idesc, 1u);
                    }
                }
                tc::mma_commit(&S.a_empty);
                tc::mma_commit(&S.d_full[b]);
                issued = true;
            }
            if (S.abort && issued) {
                tc::mma_commit(&S.drained);
                if (!tc::wait_bounded(&S.drained, 0u, tc::kDrainCycles) && status) atomicOr(status, tc::kDrainGaveUp);
            }
        }
    } else {
        // ------------------------------------------------ epilogue: lane = frame
        const int e = warp - 5;                    // 0..7
        const int q = warp & 3;                    // tensor-memory lane quarter
        const int h = e >> 2;                      // bins [h N/2, (h + 1) N/2)
        const int f = 32 * q + lane;
        const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
        uint32_t it = 0;
        for (long long item = blockIdx.x; item < n_items; item += gridDim.x, ++it) {
            const int b = it & 1;
            int p;
            long long f0;
            item_of(a, item, &p, &f0);
            // frame terms (FP64 delay polynomial at the frame centre, Sec. 4.3)
            const long long fl = f0 + f;
            const bool live = fl < a.n_store;
            const long long slot = live ? fl / a.Kc : 0, kf = live ? fl % a.Kc : 0;
            const bool delayed = (a.delay != nullptr || a.delay_tab != nullptr) && fl < a.n_frames;
            float phi0 = 0.0f, d_hi = 0.0f, d_lo = 0.0f;
            if (delayed) {
                const double tau = frame_delay(a, p, a.m_begin + fl, N);
                const double ph = a.nu * tau;
                phi0 = (float)(ph - floor(ph));
                const double d = tau * a.fs_over_n;
                d_hi = __uint_as_float(__float_as_uint((float)d) & 0xFFFFF000u);
                d_lo = (float)(d - (double)d_hi);
            }
            if (!wait_phase(S, &S.d_full[b], (it >> 1) & 1, status, 2048)) break;
            tc::fence_after();
            const long long cs = 2LL * a.n * a.Kpad, ps = (long long)a.n * a.Kpad;
            const long long base = (slot * N * 2LL * a.n + p) * a.Kpad + kf;
            // bins k of this half: u = k (lower half) or k - N (upper half); no wrap inside
#pragma unroll 1
            for (int k0 = h * (N / 2); k0 < (h + 1) * (N / 2); k0 += 16) {
                uint32_t vr[16], vi[16];
                tmem_ld16(tq + b * C::DCOLS + k0, vr);
                tmem_ld16(tq + b * C::DCOLS + N + k0, vi);
                tc::tmem_wait_ld();
                // exact phasor at the chunk's first bin, the ratio e^{2 pi i d} for the next
                float2 E = make_float2(1.0f, 0.0f), R = make_float2(1.0f, 0.0f);
                if (delayed) {
                    E = phasor_u(phi0, d_hi, d_lo, h ? k0 - N : k0);
                    R = phasor_u(0.0f, d_hi, d_lo, 1);
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int k = k0 + j;
                    const int c = h ? k - N / 2 : k + N / 2;   // fftshift
                    float2 y = make_float2(__uint_as_float(vr[j]), __uint_as_float(vi[j]));
                    if (delayed) {
                        y = cmul(y, E);
                        E = cmul(E, R);
                    }
                    const float g = gain[c];
                    if (live) store_value<N, OUTK>(a, base + c * cs, ps, make_float2(y.x * g, y.y * g));
                }
            }
            tc::fence_before();
            tc::mbar_arrive(&S.d_empty[b]);
        }
    }

    tc::fence_before();
    __syncthreads();
    if (warp == 4) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, C::TMEM);
    }
}

template <int N, int OUTK>
cudaError_t launch_dft(const FArgs& a, cudaStream_t s)
{
    using C = Dft<N, OUTK>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fstep_dft_kernel<N, OUTK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const long long n_items = (long long)a.n * ((a.n_store + kFrames - 1) / kFrames);
    if (n_items <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = n_items < sms ? n_items : sms;
    fstep_dft_kernel<N, OUTK><<<(unsigned)grid, kThreads, C::SMEM, s>>>(a, n_items);
    return cudaGetLastError();
}

template <int OUTK>
cudaError_t launch_dft_n(int N, const FArgs& a, cudaStream_t s)
{
    switch (N) {
        case 32: return launch_dft<32, OUTK>(a, s);
        case 64: return launch_dft<64, OUTK>(a, s);
        case 128: return launch_dft<128, OUTK>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool fstep_dft_supported(int N, int out_kind)
{
    return (N == 32 || N == 64 || N == 128) && (out_kind == FOUT_F32 || out_kind == FOUT_F16 || out_kind == FOUT_F16X3);
}

cudaError_t launch_fstep_dft(int N, int out_kind, const FArgs& a, cudaStream_t s)
{
    switch (out_kind) {
        case FOUT_F32: return launch_dft_n<FOUT_F32>(N, a, s);
        case FOUT_F16: return launch_dft_n<FOUT_F16>(N, a, s);
        case FOUT_F16X3: return launch_dft_n<FOUT_F16X3>(N, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mwax
