// Tensor-core F-step for the long fine-channel FFTs (Sec. 2.5.1: N = 80 N2, here 6400 and
// 1280) with FP16 operands out (the FP16 and FP8 forms).  The N-point DFT of a frame is
// taken as two small DFT-matrix products (the four-step decomposition N = N1 N2, N1 = 80):
//   sample n = N2 n1 + n2, bin k = k1 + 80 k2,
//   stage A (tcgen05, both operands in shared memory):
//       Y[k1, n2]  = sum_n1 F80[k1, n1] x[N2 n1 + n2]
//   twiddle (CUDA cores, tensor memory -> registers -> tensor memory):
//       Y'[k1, n2] = Y[k1, n2] e^{-2 pi i n2 k1 / N}
//   stage B (tcgen05, A operand read from tensor memory, B in shared memory):
//       X[k1 + 80 k2] = sum_n2 Y'[k1, n2] F_N2[k2, n2]
// F_L[a, b] = e^{-2 pi i a b / L}.  Then the delay phasor (Sec. 4.3), the channel gain
// (averaging weight, passband, FP16 pre-scale) and the FP16 store of the K-major operand
// planes Y[slot][c][plane][p][Kpad], c = fftshift(k), exactly as the CUDA-core F-steps do.
//
// Complex products on planar operands: re = ar br - ai bi, im = ar bi + ai br, with a
// stored -Im plane of the DFT matrices for the minus sign.  The DFT matrices are rounded to
// FP16 (2^-12 relative); stage A's inputs (int8) are exact; Y' is rounded to FP16 once: the
// FP16 form's error bar (2e-3 of the auto scale) holds with a wide margin.
//
// A persistent CTA (256 threads; one per SM holding all 512 tensor-memory columns, or two
// with 256 each) loops over items of G consecutive frames of one signal path.  Shared-memory operands use the no-swizzle K-major canonical layout (8 x 16 B
// core matrices; LBO = K-direction stride between core matrices, SBO = M/N-direction
// stride).  The next item's int8 samples are loaded into registers while the current
// item's outputs are stored.  Every wait on the tensor cores is bounded (status word).
#include "mwax_internal.cuh"
#include "tc_ptx.cuh"

namespace mwax {
namespace {

constexpr int kN1 = 80;                     // stage-A DFT length (rows k1 of the M = 128 tile)
constexpr int kNT = 256;                    // threads per CTA
constexpr uint32_t kFPlane = 10 * 2048;     // F80 plane: 128 rows x 80 K, LBO 2048, SBO 128

template <int N2, int G, int CTAS>
struct TcDft {
    static constexpr int N = kN1 * N2;
    static constexpr int NA = G * N2;                 // stage-A N (frames x n2)
    static constexpr int N2P = N2;                    // stage-B K and N (N2 a multiple of 16)
    static_assert(N2 % 16 == 0 && NA % 16 == 0 && NA <= 256, "MMA shapes");
    static constexpr int COLS_D = 2 * NA;             // D_A (re, im); D_B reuses its columns
    static constexpr int A0 = COLS_D;                 // Y' (stage-B A operand), FP16 pairs
    static constexpr int COLS = COLS_D + G * N2P;
    // CTAS CTAs share an SM: 512 / CTAS tensor-memory columns each
    static constexpr uint32_t TMEM = CTAS == 1 ? 512u : 256u;
    static_assert(COLS <= (int)TMEM && 2 * G * N2P <= COLS_D, "tensor memory budget");
    static constexpr uint32_t LBO_X = NA * 16;        // X plane: NA rows x 80 K
    static constexpr uint32_t XPLANE = 10 * LBO_X;
    // F_N2 as the stage-B B operand: F80 itself when N2 = 80, else its own planes
    static constexpr bool OWN_F2 = N2 != kN1;
    static constexpr uint32_t LBO_F2 = OWN_F2 ? (N2 / 8) * 128 : 2048;
    static constexpr uint32_t F2PLANE = OWN_F2 ? (N2 / 8) * LBO_F2 : 0;
    static constexpr int BLOCKS = G * 10 * (N2 / 8);  // 8 x 8 sample blocks per item
    static_assert(BLOCKS <= kNT, "one 8 x 8 block per thread");
    // shared memory: F80 (re, im, -im), X (re, im), F_N2 (re, im, -im), the int8 stage,
    // the channel gains (one CTA per SM; with two the gains are read through the read-only
    // cache), frame info.  At least 1/(CTAS + 1) of the SM's shared memory, so that no more
    // than CTAS CTAs (512 TMEM columns) share an SM.
    static constexpr size_t STAGE = (size_t)G * 2 * N;   // int8 samples of an item's frames
    static constexpr bool GAIN_SMEM = CTAS == 1;
    static constexpr size_t SMEM_USED =
        3 * kFPlane + 2 * XPLANE + 3 * F2PLANE + STAGE + (GAIN_SMEM ? sizeof(float) * N : 0) + 1024;
    static constexpr size_t SMEM_MIN = CTAS == 1 ? 116 * 1024 : 80 * 1024;
    static constexpr size_t SMEM = SMEM_USED < SMEM_MIN ? SMEM_MIN : SMEM_USED;
    static constexpr int H = N2 / 2;           // n2 (twiddle) or k2 (store) per warp half
    static constexpr int CHUNKS = (H + 7) / 8;
};

struct TcFrame {
    long long slot, k;       // operand slot and frame within it (slot -1: not stored)
    float phi0, d_hi, d_lo;  // delay terms (see delay_phasor_u in the CUDA-core F-step)
    int delay;
    float2 step80;           // e^{2 pi i 80 d}: phasor ratio between bins k and k + 80
};

struct TcShared {
    uint64_t ld_bar;         // int8 samples of the next item staged (bulk copies)
    unsigned ld_mask;        // frames of that item with data
    uint64_t bar;            // MMA completion (stage A, then stage B, alternating phases)
    uint64_t drained;        // after an abort: every MMA issued has completed
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ uint64_t desc_plain(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05; swizzle bits 0: none
    return d;
}

// D[tmem] (+)= A[tmem] * B[smem]^T, 16-bit inputs, FP32 accumulate (A: M rows on the lanes,
// two K elements per 32-bit column).
__device__ __forceinline__ void mma_f16_tmem_a(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n"
        "}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}

// CW consecutive columns (8 or 4) of this warp's lanes.
template <int CW>
__device__ __forceinline__ void tmem_ldw(uint32_t taddr, uint32_t (&r)[CW])
{
    if constexpr (CW == 8) tmem_ld8(taddr, r);
    else tmem_ld4(taddr, r);
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&r)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3])
                 : "memory");
}

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

// Byte offset of element (row r, k) in a no-swizzle K-major plane with the given LBO.
__device__ __forceinline__ uint32_t plain_off(int r, int k, uint32_t lbo)
{
    return (uint32_t)(k >> 3) * lbo + (uint32_t)(r >> 3) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// Bounded wait for the MMA barrier phase; false (abort raised, status recorded) on expiry.
__device__ __forceinline__ bool wait_mma(TcShared& S, uint32_t parity, int* status)
{
    const long long lim = (long long)tc::kDefaultSpin * 1000LL;
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(&S.bar, parity)) {
        if (*reinterpret_cast<volatile int*>(&S.abort)) return false;
        if (clock64() - t0 > lim) {
            S.abort = 1;
            if (status) atomicOr(status, 1024);
            return false;
        }
    }
    return true;
}

// 1-D bulk copy global -> shared, completing on an mbarrier's transaction count (16-byte
// aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}

// Issue the copies of an item's frames (2N bytes each, one bulk copy per frame with data)
// into the int8 stage and publish the mask of frames copied (the others are read as zero:
// past the call's data, or a zeroed block).  One thread.
template <int N2, int G>
__device__ __forceinline__ void issue_item(const FArgs& a, long long item, unsigned char* stage, uint64_t* bar, unsigned* mask_out)
{
    constexpr int N = kN1 * N2;
    const long long n_fg = (a.n_store + G - 1) / G;
    const int p = (int)(item / n_fg);
    const long long f0 = (item % n_fg) * G;
    unsigned mask = 0;
    long long srcs[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const long long f = f0 + g;
        srcs[g] = -1;
        if (f >= a.n_frames) continue;
        const long long s0 = (a.m_begin + f) * (long long)N;
        if (frame_zeroed(a, p, s0)) continue;
        const long long blk = s0 / a.bs, off = s0 % a.bs;
        srcs[g] = ((blk * a.n + p) * (long long)a.bs + off) * 2;
        mask |= 1u << g;
    }
    // the mask is published before the arrive (release): a waiter that sees the phase
    // complete (at once when no frame is copied) reads this item's mask
    *mask_out = mask;
    tc::mbar_arrive_expect_tx(bar, (uint32_t)(__popc(mask) * 2 * N));
#pragma unroll
    for (int g = 0; g < G; ++g)
        if (mask & (1u << g)) bulk_copy(stage + g * 2 * N, a.volt + srcs[g], 2u * N, bar);
}

// Transpose one 8 x 8 block of staged int8 samples (rows n1 = 8 b1 + i, samples n2 = 8 b2 ..
// 8 b2 + 7 of frame g) into the X operand as FP16: row r = g N2 + n2 (B row), K = n1.  Row
// j of the core matrix takes sample j of each of the 8 staged rows; rows are visited in an
// order rotated by the thread index so that a warp's 16-byte stores spread over the banks.
template <int N2, int G, int CTAS>
__device__ __forceinline__ void stage_to_x(const unsigned char* stage, unsigned mask, unsigned char* xre,
                                           unsigned char* xim, int t)
{
    using C = TcDft<N2, G, CTAS>;
    constexpr int PB = 10 * (N2 / 8);
    if (t >= C::BLOCKS) return;
    const int g = t / PB, rem = t % PB, b1 = rem / (N2 / 8), b2 = rem % (N2 / 8);
    int4 raw[8];
    const bool live = (mask >> g) & 1u;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        raw[i] = live ? *reinterpret_cast<const int4*>(stage + g * 2 * C::N + 2 * ((8 * b1 + i) * N2 + 8 * b2))
                      : make_int4(0, 0, 0, 0);
    const uint32_t base = (uint32_t)b1 * C::LBO_X + (uint32_t)(g * (N2 / 8) + b2) * 128u;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        const int j = (jj + t) & 7;
        uint32_t wr[4], wi[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            // sample j of rows 2h and 2h + 1: bytes 2j (re) and 2j + 1 (im) of each
            const int4 c0 = raw[2 * h], c1 = raw[2 * h + 1];
            const uint32_t w0 = (j < 2) ? (uint32_t)c0.x : (j < 4) ? (uint32_t)c0.y : (j < 6) ? (uint32_t)c0.z : (uint32_t)c0.w;
            const uint32_t w1 = (j < 2) ? (uint32_t)c1.x : (j < 4) ? (uint32_t)c1.y : (j < 6) ? (uint32_t)c1.z : (uint32_t)c1.w;
            const int sh = (j & 1) * 16;
            const int r0 = (int)(int8_t)(w0 >> sh), i0 = (int)(int8_t)(w0 >> (sh + 8));
            const int r1 = (int)(int8_t)(w1 >> sh), i1 = (int)(int8_t)(w1 >> (sh + 8));
            const __half2 hr = __halves2half2(__int2half_rn(r0), __int2half_rn(r1));
            const __half2 hi = __halves2half2(__int2half_rn(i0), __int2half_rn(i1));
            wr[h] = *reinterpret_cast<const uint32_t*>(&hr);
            wi[h] = *reinterpret_cast<const uint32_t*>(&hi);
        }
        *reinterpret_cast<uint4*>(xre + base + 16u * j) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
        *reinterpret_cast<uint4*>(xim + base + 16u * j) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
    }
}

template <int N2, int G, int CTAS>
__global__ void __launch_bounds__(kNT, CTAS) fstep_tc_kernel(const FArgs a, long long n_items)
{
    using C = TcDft<N2, G, CTAS>;
    constexpr int N = C::N;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    unsigned char* f_re = sm;
    unsigned char* f_im = f_re + kFPlane;
    unsigned char* f_nim = f_im + kFPlane;
    unsigned char* x_re = f_nim + kFPlane;
    unsigned char* x_im = x_re + C::XPLANE;
    unsigned char* g_re = C::OWN_F2 ? x_im + C::XPLANE : f_re;
    unsigned char* g_im = C::OWN_F2 ? g_re + C::F2PLANE : f_im;
    unsigned char* g_nim = C::OWN_F2 ? g_im + C::F2PLANE : f_nim;
    unsigned char* stage = x_im + C::XPLANE + 3 * C::F2PLANE;   // 16-byte aligned (plane sizes)
    float* gain_s = reinterpret_cast<float*>(stage + C::STAGE);
    const float* gain = C::GAIN_SMEM ? gain_s : a.gain;
    TcFrame* fr = reinterpret_cast<TcFrame*>(stage + C::STAGE + (C::GAIN_SMEM ? sizeof(float) * N : 0));
    TcShared& S = *reinterpret_cast<TcShared*>(fr + G);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int* status = a.status;

    // ---- one-time set-up: DFT matrices (FP16), gains, barriers, tensor memory
    for (int e = tid; e < 128 * kN1; e += kNT) {
        const int r = e / kN1, k = e % kN1;
        float s = 0.0f, c = 0.0f;
        if (r < kN1) sincospif(-2.0f * (float)((r * k) % kN1) / (float)kN1, &s, &c);
        const uint32_t o = plain_off(r, k, 2048);
        *reinterpret_cast<__half*>(f_re + o) = __float2half_rn(c);
        *reinterpret_cast<__half*>(f_im + o) = __float2half_rn(s);
        *reinterpret_cast<__half*>(f_nim + o) = __float2half_rn(-s);
    }
    if (C::OWN_F2)
        for (int e = tid; e < N2 * N2; e += kNT) {
            const int r = e / N2, k = e % N2;
            float s, c;
            sincospif(-2.0f * (float)((r * k) % N2) / (float)N2, &s, &c);
            const uint32_t o = plain_off(r, k, C::LBO_F2);
            *reinterpret_cast<__half*>(g_re + o) = __float2half_rn(c);
            *reinterpret_cast<__half*>(g_im + o) = __float2half_rn(s);
            *reinterpret_cast<__half*>(g_nim + o) = __float2half_rn(-s);
        }
    if (C::GAIN_SMEM)
        for (int i = tid; i < N; i += kNT) gain_s[i] = __ldg(&a.gain[i]);
    long long item = blockIdx.x;
    if (tid == 0) {
        tc::mbar_init(&S.bar, 1);
        tc::mbar_init(&S.drained, 1);
        tc::mbar_init(&S.ld_bar, 1);
        S.abort = 0;
        tc::fence_mbar_init();
        if (item < n_items) issue_item<N2, G>(a, item, stage, &S.ld_bar, &S.ld_mask);   // first item
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, C::TMEM);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t idA = tc::idesc(0, 128, C::NA, false), idB = tc::idesc(0, 128, C::N2P, false);
    const int q = warp & 3;                 // tensor-memory lane quarter: rows k1 = 32 q + lane
    const int k1 = 32 * q + lane;
    const bool hi_half = warp >= 4;         // n2 (twiddle) or k2 (store) in [N2/2, N2)
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
    uint32_t parity = 0, ld_parity = 0;
    bool issued = false;
    // a thread's own timeout (bad) decides nothing alone: every exit is taken by all threads
    // at the same barrier, from __syncthreads_or of the threads' flags (stop)
    bool bad = false, stop = false;
    bool ld_pending = tid == 0 && blockIdx.x < n_items;   // a bulk copy not yet waited for
    // twiddles of this thread's row k1 and n2 range, the same for every item: the value at
    // the range's first n2 and the ratio between neighbouring n2 (a recurrence over at
    // most 40 steps: ~1e-6 relative, far below the FP16 rounding of Y')
    float2 tw0, tw1;
    {
        const int n2b = hi_half ? C::H : 0;
        float sn, cs;
        sincospif(-2.0f * (float)((n2b * k1) % N) / (float)N, &sn, &cs);
        tw0 = make_float2(cs, sn);
        sincospif(-2.0f * (float)k1 / (float)N, &sn, &cs);
        tw1 = make_float2(cs, sn);
    }

    for (; item < n_items; item += gridDim.x) {
        const long long n_fg = (a.n_store + G - 1) / G;
        const int p = (int)(item / n_fg);
        const long long f0 = (item % n_fg) * G;

        // ---- X operand of this item from the staged samples, frame terms (FP64 delay
        // polynomial, Sec. 4.3)
        {
            const long long lim = (long long)tc::kDefaultSpin * 1000LL, t0 = clock64();
            bool ok = true;
            while (!tc::mbar_try_wait(&S.ld_bar, ld_parity))
                if (clock64() - t0 > lim) {
                    ok = false;
                    break;
                }
            if (ok) {
                ld_parity ^= 1u;
                if (tid == 0) ld_pending = false;
            } else {
                bad = true;
                S.abort = 1;   // lets the other threads' waits give up early
                if (status) atomicOr(status, 2048);
            }
        }
        stage_to_x<N2, G, CTAS>(stage, S.ld_mask, x_re, x_im, tid);
        if (tid < G) {
            const long long f = f0 + tid;
            TcFrame fi;
            fi.slot = (f < a.n_store) ? f / a.Kc : -1;
            fi.k = (f < a.n_store) ? f % a.Kc : 0;
            fi.delay = 0;
            fi.phi0 = fi.d_hi = fi.d_lo = 0.0f;
            fi.step80 = make_float2(1.0f, 0.0f);
            if ((a.delay != nullptr || a.delay_tab != nullptr) && f < a.n_frames) {
                const double tau = frame_delay(a, p, a.m_begin + f, N);
                const double ph = a.nu * tau;
                fi.phi0 = (float)(ph - floor(ph));
                const double d = tau * a.fs_over_n;
                const float dh = __uint_as_float(__float_as_uint((float)d) & 0xFFFFF000u);
                fi.d_hi = dh;
                fi.d_lo = (float)(d - (double)dh);
                fi.delay = 1;
                const double st = 80.0 * d;
                float sn, cs;
                sincospif(2.0f * (float)(st - rint(st)), &sn, &cs);
                fi.step80 = make_float2(cs, sn);
            }
            fr[tid] = fi;
        }
        fence_proxy_async_smem();   // X written by the generic proxy, read by the tensor cores
        tc::fence_before();
        if ((stop = __syncthreads_or(bad))) break;
        // the stage is free: the next item's samples copy in while this one is processed
        {
            const long long next = item + gridDim.x;
            if (tid == 0 && next < n_items) {
                issue_item<N2, G>(a, next, stage, &S.ld_bar, &S.ld_mask);
                ld_pending = true;
            }
        }

        // ---- stage A: Y = F80 X (4 real products per complex term, K = n1 in 5 steps of 16)
        if (tid == 0) {
            tc::fence_after();
            const uint32_t fr0 = tc::smem_u32(f_re), fi0 = tc::smem_u32(f_im), fn0 = tc::smem_u32(f_nim);
            const uint32_t xr0 = tc::smem_u32(x_re), xi0 = tc::smem_u32(x_im);
            const uint32_t dre = tmem, dim = tmem + C::NA;
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const uint32_t acc = s > 0 ? 1u : 0u;
                const uint64_t ar = desc_plain(fr0 + s * 4096u, 2048, 128), ai = desc_plain(fi0 + s * 4096u, 2048, 128);
                const uint64_t an = desc_plain(fn0 + s * 4096u, 2048, 128);
                const uint64_t br = desc_plain(xr0 + s * 2u * C::LBO_X, C::LBO_X, 128);
                const uint64_t bi = desc_plain(xi0 + s * 2u * C::LBO_X, C::LBO_X, 128);
                tc::mma_f16(dre, ar, br, idA, acc);
                tc::mma_f16(dre, an, bi, idA, 1u);
                tc::mma_f16(dim, ar, bi, idA, acc);
                tc::mma_f16(dim, ai, br, idA, 1u);
            }
            tc::mma_commit(&S.bar);
            issued = true;
        }
        const bool okA = wait_mma(S, parity, status);
        parity ^= 1u;
        tc::fence_after();
        bad = bad || !okA;
        const bool skipA = __any_sync(0xffffffffu, bad);   // warp-uniform (collective TMEM access)

        // ---- twiddle: Y' = Y W_N^{n2 k1}, FP16 pairs into tensor memory (stage B's A)
        if (!skipA && q < 3) {
            constexpr int H = C::H;   // n2 per warp half
            const int n2b = hi_half ? H : 0;
#pragma unroll 1
            for (int g = 0; g < G; ++g) {
                float2 E = tw0;
#pragma unroll 1
                for (int ci = 0; ci < C::CHUNKS; ++ci) {
                    const int n20 = n2b + 8 * ci;
                    uint32_t vr[8], vi[8];
                    tmem_ld8(tq + (uint32_t)(g * N2 + n20), vr);
                    tmem_ld8(tq + (uint32_t)(C::NA + g * N2 + n20), vi);
                    tc::tmem_wait_ld();
                    const float2 w1 = tw1;
                    uint32_t pr[4], pi[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const float2 y0 = cmul(make_float2(__uint_as_float(vr[e]), __uint_as_float(vi[e])), E);
                        E = cmul(E, w1);
                        const float2 y1 = cmul(make_float2(__uint_as_float(vr[e + 1]), __uint_as_float(vi[e + 1])), E);
                        E = cmul(E, w1);
                        const __half2 hr = __floats2half2_rn(y0.x, y1.x), hi = __floats2half2_rn(y0.y, y1.y);
                        pr[e / 2] = *reinterpret_cast<const uint32_t*>(&hr);
                        pi[e / 2] = *reinterpret_cast<const uint32_t*>(&hi);
                    }
                    const uint32_t col = C::A0 + g * C::N2P + n20 / 2;
                    tmem_st4(tq + col, pr);
                    tmem_st4(tq + col + C::N2P / 2, pi);
                }
            }
            tc::tmem_wait_st();
        }
        tc::fence_before();
        if ((stop = __syncthreads_or(bad))) break;

        // ---- stage B: X = Y' F_N2 per frame (A from tensor memory)
        if (tid == 0) {
            tc::fence_after();
            const uint32_t gr0 = tc::smem_u32(g_re), gi0 = tc::smem_u32(g_im), gn0 = tc::smem_u32(g_nim);
#pragma unroll 1
            for (int g = 0; g < G; ++g) {
                const uint32_t dre = tmem + (uint32_t)(g * 2 * C::N2P), dim = dre + C::N2P;
                const uint32_t are = tmem + C::A0 + (uint32_t)(g * C::N2P), aim = are + C::N2P / 2;
#pragma unroll
                for (int s = 0; s < C::N2P / 16; ++s) {
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    const uint64_t br = desc_plain(gr0 + s * 2u * C::LBO_F2, C::LBO_F2, 128);
                    const uint64_t bi = desc_plain(gi0 + s * 2u * C::LBO_F2, C::LBO_F2, 128);
                    const uint64_t bn = desc_plain(gn0 + s * 2u * C::LBO_F2, C::LBO_F2, 128);
                    mma_f16_tmem_a(dre, are + 8u * s, br, idB, acc);
                    mma_f16_tmem_a(dre, aim + 8u * s, bn, idB, 1u);
                    mma_f16_tmem_a(dim, are + 8u * s, bi, idB, acc);
                    mma_f16_tmem_a(dim, aim + 8u * s, br, idB, 1u);
                }
            }
            tc::mma_commit(&S.bar);
        }
        const bool okB = wait_mma(S, parity, status);
        parity ^= 1u;
        tc::fence_after();
        bad = bad || !okB;
        const bool skipB = __any_sync(0xffffffffu, bad);

        // ---- phasor, gain, FP16 store: bins k = k1 + 80 k2, k2 in this warp's half
        // (the tensor-memory loads are warp-collective: every lane of a quarter takes part,
        // only rows k1 < 80 store)
        if (!skipB && q < 3) {
            constexpr int H = N2 / 2;
            const int k2b = hi_half ? H : 0;
            const bool row_ok = k1 < kN1;
            TcFrame fi[G];
            float2 E[G];
            bool live_all = true;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                fi[g] = fr[g];
                // bins past N/2 are u = k - N: exactly the upper half of k2 (80 divides N/2)
                const int u = k1 + kN1 * k2b - (hi_half ? N : 0);
                E[g] = fi[g].delay ? phasor_u(fi[g].phi0, fi[g].d_hi, fi[g].d_lo, u) : make_float2(1.0f, 0.0f);
                live_all = live_all && fi[g].slot == fi[0].slot && fi[g].slot >= 0;
            }
            // all G frames in one slot from a multiple of G: one store of G values per plane
            const bool packed = live_all && (fi[0].k % G) == 0;
            const long long ps = (long long)a.n * a.Kpad;
            __half* Y = static_cast<__half*>(a.Y);
            constexpr int CW = G >= 4 ? 4 : 8;   // columns per load (registers: G x 2 x CW)
#pragma unroll 1
            for (int c8 = 0; c8 < H; c8 += CW) {
                uint32_t vr[G][CW], vi[G][CW];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    tmem_ldw<CW>(tq + (uint32_t)(g * 2 * C::N2P + k2b + c8), vr[g]);
                    tmem_ldw<CW>(tq + (uint32_t)(g * 2 * C::N2P + C::N2P + k2b + c8), vi[g]);
                }
                tc::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < CW; ++e) {
                    const int k2 = k2b + c8 + e;
                    const int c = k1 + kN1 * k2 + (hi_half ? -(N / 2) : N / 2);   // fftshift
                    const float gn = gain[c];
                    __half hr[G], hi[G];
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        float2 y = make_float2(__uint_as_float(vr[g][e]), __uint_as_float(vi[g][e]));
                        if (fi[g].delay) {
                            y = cmul(y, E[g]);
                            E[g] = cmul(E[g], fi[g].step80);
                        }
                        hr[g] = __float2half_rn(y.x * gn);
                        hi[g] = __float2half_rn(y.y * gn);
                    }
                    if (!row_ok) continue;
                    if (packed) {
                        // G consecutive frames of one slot from a multiple of G: one 2 G-byte
                        // store per plane
                        const long long at = ((fi[0].slot * N + c) * 2LL * a.n + p) * a.Kpad + fi[0].k;
                        if constexpr (G == 1) {
                            Y[at] = hr[0];
                            Y[at + ps] = hi[0];
                        } else {
                            uint32_t wr[G / 2], wi[G / 2];
#pragma unroll
                            for (int h = 0; h < G / 2; ++h) {
                                const __half2 a2 = __halves2half2(hr[2 * h], hr[2 * h + 1]);
                                const __half2 b2 = __halves2half2(hi[2 * h], hi[2 * h + 1]);
                                wr[h] = *reinterpret_cast<const uint32_t*>(&a2);
                                wi[h] = *reinterpret_cast<const uint32_t*>(&b2);
                            }
                            if constexpr (G == 8) {
                                *reinterpret_cast<uint4*>(Y + at) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
                                *reinterpret_cast<uint4*>(Y + at + ps) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
                            } else if constexpr (G == 4) {
                                *reinterpret_cast<uint2*>(Y + at) = make_uint2(wr[0], wr[1]);
                                *reinterpret_cast<uint2*>(Y + at + ps) = make_uint2(wi[0], wi[1]);
                            } else {
                                static_assert(G == 2, "frames per item: 1, 2, 4 or 8");
                                *reinterpret_cast<uint32_t*>(Y + at) = wr[0];
                                *reinterpret_cast<uint32_t*>(Y + at + ps) = wi[0];
                            }
                        }
                    } else {
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            if (fi[g].slot < 0) continue;
                            const long long at = ((fi[g].slot * N + c) * 2LL * a.n + p) * a.Kpad + fi[g].k;
                            Y[at] = hr[g];
                            Y[at + ps] = hi[g];
                        }
                    }
                }
            }
        }
        tc::fence_before();
        if ((stop = __syncthreads_or(bad))) break;
    }

    // ---- wind-down: after an abort let the MMAs and the bulk copy in flight finish before
    // the tensor memory is freed and the CTA exits
    if (tid == 0 && stop) {
        if (issued) {
            tc::mma_commit(&S.drained);
            if (!tc::wait_bounded(&S.drained, 0u, tc::kDrainCycles) && status) atomicOr(status, tc::kDrainGaveUp);
        }
        if (ld_pending && !tc::wait_bounded(&S.ld_bar, ld_parity, tc::kDrainCycles) && status)
            atomicOr(status, tc::kDrainGaveUp);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, C::TMEM);
    }
}

template <int N2, int G, int CTAS>
cudaError_t launch_tc(const FArgs& a, cudaStream_t s)
{
    using C = TcDft<N2, G, CTAS>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fstep_tc_kernel<N2, G, CTAS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const long long n_items = (long long)a.n * ((a.n_store + G - 1) / G);
    if (n_items <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = n_items < (long long)CTAS * sms ? n_items : (long long)CTAS * sms;
    fstep_tc_kernel<N2, G, CTAS><<<(unsigned)grid, kNT, C::SMEM, s>>>(a, n_items);
    return cudaGetLastError();
}

}  // namespace

bool fstep_tc_supported(int N) { return N == 6400 || N == 1280; }

cudaError_t launch_fstep_tc(int N, const FArgs& a, cudaStream_t s)
{
    switch (N) {
        // measured (256 tiles, FP16, per 0.5 s): N = 6400 with 2-frame items, one CTA per SM,
        // 3.5 ms (1-frame items, two CTAs per SM: 8.0 ms); N = 1280 with 4-frame items, two
        // CTAs per SM, 3.7 ms (8-frame items, one CTA: 4.9 ms)
        case 6400: return launch_tc<80, 2, 1>(a, s);
        case 1280: return launch_tc<16, 4, 2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mwax
