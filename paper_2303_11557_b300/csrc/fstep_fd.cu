// Tensor-core F-step for the short fine-channel FFTs (Sec. 2.5.1: N = 32, 64, 128) with the
// frames on the accumulator lanes, FP16 or e4m3 operands out (the FP16 and FP8 forms).  An
// item is 128 consecutive frames of one path; the N-point DFT of all of them is one product
//   X[g, k] = sum_n x_g[n] F_N[k, n]        (tcgen05: M = 128 frames g, N = N bins k, K = N)
// with both operands in shared memory: the frames' int8 samples as FP16 (exact) and the DFT
// matrix F_N[k, n] = e^{-2 pi i k n / N}, each row scaled by its channel's gain, rounded to
// FP16 (2^-12 per entry).  Then per lane (one frame) and bin: the delay phasor (Sec. 4.3; a
// ratio recurrence along the bins from one sincospi per frame and warp) and the store of
// the K-major operand planes Y[slot][c][plane][p][Kpad], c = fftshift(k): a warp's 32
// lanes are 32 consecutive frames, so each store instruction writes 64 (FP16) or 32 (e4m3)
// contiguous bytes of one operand row.
//
// A persistent CTA (16 worker warps and a control warp, one CTA per SM) loops over the items,
// software-pipelined as the 128-row F-step: the control warp copies item j + 3's samples
// and frame terms in (bulk copies, one per run of frames within a data block; two stage
// buffers, so each copy has two items' time to land) and issues item j + 1's MMAs into the
// other half of tensor memory while the workers convert item j + 1's samples, then run the
// epilogue of item j; one CTA barrier per item.  Every wait is
// bounded.  The frames' delay terms (FP64) come from a small kernel launched first: inside
// this one they held every item's barrier (one warp's FP64 sequence on this GPU's narrow
// FP64 pipe).
#include "mwax_internal.cuh"
#include "tc_ptx.cuh"

#include <type_traits>

namespace mwax {
namespace {

constexpr int kF = 128;              // frames per item (MMA M, tensor-memory lanes)
// int8 stage buffers: with one, each copy was issued one item ahead and the workers waited
// on it for over a third of the item
constexpr int kST = 2;
constexpr int kNFR = kST + 2;        // frame-term slots: items j .. j + kST + 1
constexpr int kW = 512;              // worker threads (4 warps per lane quarter)
constexpr int kT = kW + 32;          // plus the control warp

template <int N>
struct FD {
    static_assert(N == 32 || N == 64 || N == 128, "direct-DFT lengths");
    static constexpr uint32_t LBO_A = kF * 16 + 16;    // data: 128 rows; K core columns padded by 16 B
    static constexpr uint32_t APLANE = (N / 8) * LBO_A;
    static constexpr uint32_t LBO_B = N * 16;          // DFT matrix: N rows x N K
    static constexpr uint32_t BPLANE = (N / 8) * LBO_B;
    static constexpr uint32_t STAGE = kF * N * 2;      // int8 (re, im) of the item's frames
    static constexpr uint32_t BUF = 2 * N;             // accumulator columns (re, im) per buffer
    static constexpr uint32_t TMEM = 4 * N < 32 ? 32 : 4 * N;   // two buffers (a power of two)
    static constexpr int QB = N / 4;                   // bins per worker warp of a lane quarter
    static constexpr int NCH = QB / 8;                 // 8-column loads per warp and plane
    static constexpr int TASKS = kF * (N / 8);         // conversion tasks (8 samples each)
    static_assert(TASKS % kW == 0, "whole conversion tasks per thread");
};

struct __align__(16) FDTerm {   // two 16-byte stores
    long long base;          // element of (slot, c = 0, re plane, p, k) or -1: not stored
    float phi0, d_hi, d_lo;  // delay terms: the phasor of bin offset u is e^{2 pi i (phi0 + u d)}
    int delay;
    float2 step;             // e^{2 pi i d}: phasor ratio between bins k and k + 1
};
static_assert(sizeof(FDTerm) == 32, "frame terms: 32 bytes (an item's 128 travel by bulk copy)");

struct FDShared {
    uint64_t ld_bar[kST];    // an item's int8 frames staged, per stage buffer
    uint64_t bar;            // an item's MMAs complete
    uint64_t drained;        // after an abort: every MMA issued has completed
    unsigned mask[kST][kF / 32];   // frames of the staged item with data, per stage buffer
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

// Byte offset of element (row r, K index k) of a K-major no-swizzle operand.
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

__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
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

// Bounded wait on an mbarrier phase; on a timeout or another thread's abort: false.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, const int* abort)
{
    const long long lim = (long long)tc::kDefaultSpin * 1000LL, t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity))
        if (*reinterpret_cast<const volatile int*>(abort) || clock64() - t0 > lim) return false;
    return true;
}

// Issue the copies of an item's frames: one bulk copy per run of frames with data inside
// one data block (frames never straddle blocks: a block is a multiple of N samples), and of
// its 128 frame terms (fd_terms_kernel), on one mbarrier transaction.  The mask of frames
// copied is published before the arrive (a waiter that sees the phase complete reads this
// item's mask); the other frames are read as zero.  One thread.
template <int N>
__device__ __forceinline__ void issue_item(const FArgs& a, unsigned item, unsigned n_fg, int8_t* stage,
                                           uint64_t* bar, unsigned* mask_out, const FDTerm* tab, FDTerm* terms)
{
    // frame numbers below 2^31 (launcher): 32-bit division
    const unsigned p = item / n_fg;
    const unsigned f0 = (item - p * n_fg) * (unsigned)kF, mb = (unsigned)a.m_begin;
    const unsigned fpb = (unsigned)(a.bs / N);   // frames per data block
    const unsigned fend = (long long)f0 + kF < a.n_frames ? f0 + kF : (unsigned)a.n_frames;
    unsigned m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;   // frames with data (bits of frames 0..127)
    uint32_t bytes = 0;
    // first pass: the runs and the mask; second pass: the copies (after the arrive)
    for (unsigned f = f0; f < fend;) {
        const unsigned mf = mb + f, blk = mf / fpb;
        unsigned run = (blk + 1) * fpb - mb;   // first frame of the next block
        if (run > fend) run = fend;
        if (a.flags == nullptr || a.flags[(long long)blk * a.n + p] == 0) {
            const int lo = (int)(f - f0), hi = (int)(run - f0);   // frames [lo, hi) of the item
            auto bits = [&](int w) {
                const int a0 = max(lo - 32 * w, 0), a1 = min(hi - 32 * w, 32);
                return a1 <= a0 ? 0u : ((a1 - a0 == 32) ? 0xFFFFFFFFu : (((1u << (a1 - a0)) - 1u) << a0));
            };
            m0 |= bits(0);
            m1 |= bits(1);
            m2 |= bits(2);
            m3 |= bits(3);
            bytes += (uint32_t)((run - f) * 2 * N);
        }
        f = run;
    }
    const unsigned mask[kF / 32] = {m0, m1, m2, m3};
#pragma unroll
    for (int i = 0; i < kF / 32; ++i) mask_out[i] = mask[i];
    tc::mbar_arrive_expect_tx(bar, bytes + (uint32_t)(kF * sizeof(FDTerm)));
    bulk_copy(terms, tab + (size_t)item * kF, (uint32_t)(kF * sizeof(FDTerm)), bar);
    for (unsigned f = f0; f < fend;) {
        const unsigned mf = mb + f, blk = mf / fpb;
        unsigned run = (blk + 1) * fpb - mb;
        if (run > fend) run = fend;
        if (a.flags == nullptr || a.flags[(long long)blk * a.n + p] == 0) {
            const long long src = (((long long)blk * a.n + p) * (long long)a.bs + (long long)(mf - blk * fpb) * N) * 2;
            bulk_copy(stage + (f - f0) * 2 * N, a.volt + src, (uint32_t)((run - f) * 2 * N), bar);
        }
        f = run;
    }
}

// Operand position of frame g of an item (frame numbers below 2^31: 32-bit division).
template <int N>
__device__ __forceinline__ long long frame_base(const FArgs& a, unsigned item, unsigned n_fg, int g)
{
    const unsigned p = item / n_fg, f = (item - p * n_fg) * (unsigned)kF + (unsigned)g;
    if ((long long)f >= a.n_store) return -1;
    const unsigned kc = (unsigned)a.Kc, slot = f / kc, k = f - slot * kc;
    return ((long long)slot * N * 2LL * a.n + p) * a.Kpad + k;
}

// Frame terms of frame g of an item: its operand position and delay phasor terms (the FP64
// delay polynomial or table, Sec. 4.3), one frame at a time.
template <int N>
__device__ __forceinline__ FDTerm frame_terms(const FArgs& a, unsigned item, unsigned n_fg, int g)
{
    const unsigned p = item / n_fg;
    const long long f = (long long)(item - p * n_fg) * kF + g;
    FDTerm fi;
    fi.base = frame_base<N>(a, item, n_fg, g);
    fi.step = make_float2(1.0f, 0.0f);
    fi.delay = 0;
    fi.phi0 = fi.d_hi = fi.d_lo = 0.0f;
    if ((a.delay != nullptr || a.delay_tab != nullptr) && f < a.n_frames) {
        const double tau = frame_delay(a, (int)p, a.m_begin + f, N);
        const double ph = a.nu * tau;
        fi.phi0 = (float)(ph - floor(ph));
        const double d = tau * a.fs_over_n;
        const float dh = __uint_as_float(__float_as_uint((float)d) & 0xFFFFF000u);
        fi.d_hi = dh;
        fi.d_lo = (float)(d - (double)dh);
        fi.delay = 1;
        fi.step = phasor_u(0.0f, fi.d_hi, fi.d_lo, 1);
    }
    return fi;
}

// x rounded toward zero to `bits` significant bits: products with integers of up to 24 - bits
// bits are exact in FP32.
__device__ __forceinline__ float sig_bits(float x, int bits)
{
    return __uint_as_float(__float_as_uint(x) & (0xFFFFFFFFu << (24 - bits)));
}

// The delay polynomial along an item's frames (Sec. 4.3): with t_j = t_0 + j dt,
//   tau_j = tau_0 + j rate + j^2 acc,  rate = dt (c1 + 2 c2 t_0),  acc = c2 dt^2,
// so the phase nu tau_j (cycles) is nu tau_0 + j (nu rate) + j^2 (nu acc) and only its value
// mod 1 matters: one FP64 evaluation per item gives frac(nu tau_0) and the two differences
// reduced mod 1 (j, j^2 integers), each split hi + lo with hi short enough that j hi and
// j^2 hi are exact in FP32; every frame then adds them in FP32.  The bin slope
// d_j = tau_j fs / N likewise: d_0 split as the per-frame terms do, plus FP32 increments.
struct FDBase {
    float P0, Rh, Rl, Ah, Al;   // phase: frac(nu tau_0), nu rate mod 1 (hi, lo), nu acc mod 1 (hi, lo)
    float dh, dl0, ddr, dda;    // slope: d_0 = dh + dl0; per frame and per frame^2
    long long row0;             // operand element of (slot of frame 0, c = 0, re, p, k = 0)
    unsigned f0, k0;            // the item's first frame in the launch, and within its slot
};

// The item's position terms (any delay model): its first frame, that frame's slot and
// place in it, so that each frame's operand position takes no division by the slot length
// unless the item runs into the next slot.
template <int N>
__device__ __forceinline__ void item_position(const FArgs& a, unsigned item, unsigned n_fg, FDBase& B)
{
    const unsigned p = item / n_fg, kc = (unsigned)a.Kc;
    B.f0 = (item - p * n_fg) * (unsigned)kF;
    const unsigned slot = B.f0 / kc;
    B.k0 = B.f0 - slot * kc;
    B.row0 = ((long long)slot * N * 2LL * a.n + p) * a.Kpad;
}

template <int N>
__device__ __forceinline__ FDBase item_base(const FArgs& a, unsigned item, unsigned n_fg)
{
    const unsigned p = item / n_fg;
    const long long f0 = (long long)(item - p * n_fg) * kF;
    const double dt = a.frame_dt;
    const double t0 = ((double)(a.m_begin + f0) + 0.5) * dt;
    const double c0 = a.delay[3 * p], c1 = a.delay[3 * p + 1], c2 = a.delay[3 * p + 2];
    const double tau0 = fma(t0, fma(t0, c2, c1), c0);
    const double rate = fma(2.0 * c2, t0, c1) * dt, acc = c2 * dt * dt;
    FDBase B;
    const double ph = a.nu * tau0;
    B.P0 = (float)(ph - floor(ph));
    double r = a.nu * rate;
    r -= rint(r);
    B.Rh = sig_bits((float)r, 12);   // j < 2^7
    B.Rl = (float)(r - (double)B.Rh);
    double q = a.nu * acc;
    q -= rint(q);
    B.Ah = sig_bits((float)q, 8);    // j^2 < 2^14
    B.Al = (float)(q - (double)B.Ah);
    const double d0 = tau0 * a.fs_over_n;
    B.dh = sig_bits((float)d0, 12);
    B.dl0 = (float)(d0 - (double)B.dh);
    B.ddr = (float)(rate * a.fs_over_n);
    B.dda = (float)(acc * a.fs_over_n);
    return B;
}

template <int N>
__device__ __forceinline__ FDTerm frame_from_base(const FArgs& a, const FDBase& B, int g)
{
    const long long f = (long long)B.f0 + g;
    FDTerm fi;
    fi.base = -1;
    if (f < a.n_store) {
        const unsigned kc = (unsigned)a.Kc, kk = B.k0 + (unsigned)g;
        const unsigned ds = kk < kc ? 0u : kk / kc;   // slots past the item's first
        fi.base = B.row0 + (long long)ds * N * 2LL * a.n * a.Kpad + (kk - ds * kc);
    }
    fi.step = make_float2(1.0f, 0.0f);
    fi.delay = 0;
    fi.phi0 = fi.d_hi = fi.d_lo = 0.0f;
    if (f < a.n_frames) {
        const float jf = (float)g, j2 = (float)(g * g);
        float x1 = jf * B.Rh, x2 = j2 * B.Ah;   // exact
        x1 -= rintf(x1);
        x2 -= rintf(x2);
        float ph = B.P0 + x1 + x2 + fmaf(jf, B.Rl, j2 * B.Al);
        fi.phi0 = ph - floorf(ph);
        fi.d_hi = B.dh;
        fi.d_lo = B.dl0 + fmaf(jf, B.ddr, j2 * B.dda);
        fi.delay = 1;
        fi.step = phasor_u(0.0f, fi.d_hi, fi.d_lo, 1);
    }
    return fi;
}

// Before the F kernel: the terms of every frame of the launch into the table a.Yt
// [item][128].  A block takes 32 items: with a delay polynomial, lane i of the first warp
// evaluates item i's FP64 base (one FP64 sequence per 32 items: this GPU's FP64 pipe is
// narrow), then 8 threads per item derive its frames from it in FP32, the base held in
// registers (read once per thread: per frame, its fields' shared-memory loads throttled
// the kernel); with a delay table (or none), frame by frame.
constexpr int kTermItems = 32;
template <int N>
__global__ void __launch_bounds__(256) fd_terms_kernel(const FArgs a, unsigned n_items, unsigned n_fg)
{
    __shared__ FDBase base[kTermItems];
    const unsigned item0 = blockIdx.x * (unsigned)kTermItems;
    const bool poly = a.delay != nullptr && a.delay_tab == nullptr;
    if (poly && threadIdx.x < kTermItems && item0 + threadIdx.x < n_items) {
        FDBase B = item_base<N>(a, item0 + threadIdx.x, n_fg);
        item_position<N>(a, item0 + threadIdx.x, n_fg, B);
        base[threadIdx.x] = B;
    }
    __syncthreads();
    static_assert(kTermItems * 8 == 256, "8 threads per item");
    FDTerm* tab = static_cast<FDTerm*>(a.Yt);
    const int ii = threadIdx.x >> 3, sub = threadIdx.x & 7;
    const unsigned item = item0 + (unsigned)ii;
    if (item >= n_items) return;
    FDTerm* out = tab + (size_t)item * kF;
    if (poly) {
        const FDBase B = base[ii];
#pragma unroll 4
        for (int g = sub; g < kF; g += 8) out[g] = frame_from_base<N>(a, B, g);
    } else {
        for (int g = sub; g < kF; g += 8) out[g] = frame_terms<N>(a, item, n_fg, g);
    }
}

template <int N, bool E4M3>
__global__ void __launch_bounds__(kT, 1) fstep_fd_kernel(const FArgs a, unsigned n_items, unsigned n_fg)
{
    using C = FD<N>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    unsigned char* f_re = sm;                    // DFT matrix (B: rows k, K = n)
    unsigned char* f_im = f_re + C::BPLANE;
    unsigned char* x_re = f_im + C::BPLANE;      // the item's samples (A: rows g, K = n)
    unsigned char* x_im = x_re + C::APLANE;
    int8_t* stage = reinterpret_cast<int8_t*>(x_im + C::APLANE);   // kST buffers
    // frame terms of kNFR items x 128: the CTA's j-th item in slot j mod kNFR (item j in
    // stage E, j + 1 converted, j + 2 and j + 3 staged or being copied)
    FDTerm* frs = reinterpret_cast<FDTerm*>(stage + kST * C::STAGE);
    const FDTerm* tab = static_cast<const FDTerm*>(a.Yt);
    FDShared& S = *reinterpret_cast<FDShared*>(frs + kNFR * kF);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = tid < kW, ctl = tid == kW;
    int* status = a.status;
    unsigned n_cp[kST] = {0u, 0u};   // copies issued per stage buffer (control thread)
    // copy the CTA's j-th item `itj` into stage buffer j mod kST
    auto issue_copy = [&](int j, unsigned itj) {
        const int b = j % kST;
        issue_item<N>(a, itj, n_fg, stage + b * C::STAGE, &S.ld_bar[b], S.mask[b], tab, frs + (j % kNFR) * kF);
        ++n_cp[b];
    };

    // ---- set-up: the DFT matrix, barriers, tensor memory, the first kST items' copies
    // row k carries the gain of its output channel c(k) = fftshift(k): the product is the
    // gained spectrum
    for (int e = tid; e < N * N; e += kT) {
        const int k = e / N, n = e % N;
        float s, c;
        sincospif(-2.0f * (float)((k * n) % N) / (float)N, &s, &c);   // argument exact
        const float gk = __ldg(&a.gain[k < N / 2 ? k + N / 2 : k - N / 2]);
        const uint32_t o = plain_off(k, n, C::LBO_B);
        *reinterpret_cast<__half*>(f_re + o) = __float2half_rn(c * gk);
        *reinterpret_cast<__half*>(f_im + o) = __float2half_rn(s * gk);
    }
    unsigned cur = blockIdx.x;
    if (ctl) {
        for (int b = 0; b < kST; ++b) tc::mbar_init(&S.ld_bar[b], 1);
        tc::mbar_init(&S.bar, 1);
        tc::mbar_init(&S.drained, 1);
        S.abort = 0;
        tc::fence_mbar_init();
        for (int j = 0; j < kST; ++j) {
            const unsigned itj = cur + (unsigned)j * gridDim.x;
            if (itj < n_items) issue_copy(j, itj);
        }
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, C::TMEM);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    const int q = warp & 3, h = (warp >> 2) & 3;   // lane quarter; quarter of the bins
    const int g = 32 * q + lane;                   // a worker lane's frame
    uint32_t mma_par = 0;
    bool bad = false, stop = false, issued = false;

    // conversion of the CTA's j-th item (workers; stage buffer j mod kST, its (j / kST)-th
    // copy): 8 samples of one frame per task, FP16 rows
    auto stage_p = [&](int ji) {
        const int bs = ji % kST;
        if (!wait_phase(&S.ld_bar[bs], (uint32_t)(ji / kST) & 1u, &S.abort)) {
            bad = true;
            S.abort = 1;
            if (status) atomicOr(status, 2048);
            return;
        }
        const unsigned* mk = S.mask[bs];
        const int8_t* sb = stage + bs * C::STAGE;
#pragma unroll
        for (int i = 0; i < C::TASKS / kW; ++i) {
            const int t = tid + kW * i;
            const int j = t % (N / 8), fr = t / (N / 8);
            uint32_t wr[4] = {0u, 0u, 0u, 0u}, wi[4] = {0u, 0u, 0u, 0u};
            if ((mk[fr >> 5] >> (fr & 31)) & 1u) {
                const uint4 raw = *reinterpret_cast<const uint4*>(sb + fr * 2 * N + 16 * j);
                const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};   // (re, im) int8 of 2 samples each
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __half2 r2 = __halves2half2(__short2half_rn((signed char)(w[e] & 0xFF)),
                                                      __short2half_rn((signed char)((w[e] >> 16) & 0xFF)));
                    const __half2 i2 = __halves2half2(__short2half_rn((signed char)((w[e] >> 8) & 0xFF)),
                                                      __short2half_rn((signed char)(w[e] >> 24)));
                    wr[e] = *reinterpret_cast<const uint32_t*>(&r2);
                    wi[e] = *reinterpret_cast<const uint32_t*>(&i2);
                }
            }
            const uint32_t o = plain_off(fr, 8 * j, C::LBO_A);
            *reinterpret_cast<uint4*>(x_re + o) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
            *reinterpret_cast<uint4*>(x_im + o) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
        }
    };

    // the item's DFT into accumulator buffer `buf` (control thread): re = Xr Fr - Xi Fi,
    // im = Xr Fi + Xi Fr
    auto stage_a = [&](int buf) {
        const uint32_t id = tc::idesc(0, kF, N, false), id_neg = tc::idesc(0, kF, N, true);
        const uint64_t ar = desc_plain(tc::smem_u32(x_re), C::LBO_A), ai = desc_plain(tc::smem_u32(x_im), C::LBO_A);
        const uint64_t br = desc_plain(tc::smem_u32(f_re), C::LBO_B), bi = desc_plain(tc::smem_u32(f_im), C::LBO_B);
        const uint32_t dre = tmem + (uint32_t)buf * C::BUF, dim = dre + N;
#pragma unroll
        for (int ks = 0; ks < N / 16; ++ks) {
            const uint32_t acc = ks > 0 ? 1u : 0u;
            const uint64_t oa = (uint64_t)((ks * 2u * C::LBO_A) >> 4), ob = (uint64_t)((ks * 2u * C::LBO_B) >> 4);
            tc::mma_f16(dre, ar + oa, br + ob, id, acc);
            tc::mma_f16(dre, ai + oa, bi + ob, id_neg, 1u);
            tc::mma_f16(dim, ar + oa, bi + ob, id, acc);
            tc::mma_f16(dim, ai + oa, br + ob, id, 1u);
        }
        tc::mma_commit(&S.bar);
        issued = true;
    };

    // the epilogue of an item (workers): lane = frame g, bins k of this warp's quarter (the
    // upper half is u = k - N); phasor recurrence along the bins, conversion, stores
    // (the bins of a quarter are consecutive channels: one pointer step per bin)
    auto stage_e = [&](int buf, const FDTerm* fr) {
        constexpr int QB = C::QB;
        const FDTerm fi = fr[g];
        const bool live = fi.base >= 0;
        const bool upper = h >= 2;                       // k >= N/2: u = k - N, c = k - N/2
        const int k0 = h * QB;
        float2 P = fi.delay ? phasor_u(fi.phi0, fi.d_hi, fi.d_lo, upper ? k0 - N : k0) : make_float2(1.0f, 0.0f);
        const float2 st = fi.step;
        const long long cs = 2LL * a.n * a.Kpad, ps = (long long)a.n * a.Kpad;
        const int c0 = upper ? k0 - N / 2 : k0 + N / 2;   // fftshift of the quarter's first bin
        using T = typename std::conditional<E4M3, uint8_t, __half>::type;
        T* yp = static_cast<T*>(a.Y) + (live ? fi.base : 0) + (long long)c0 * cs;
        const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * C::BUF + (uint32_t)k0;
        uint32_t vr[8], vi[8], nr[8], ni[8];
        ld8(tb, vr);
        ld8(tb + (uint32_t)N, vi);
        tc::tmem_wait_ld();
#pragma unroll
        for (int ch = 0; ch < C::NCH; ++ch) {
            if (ch + 1 < C::NCH) {
                ld8(tb + (uint32_t)(8 * (ch + 1)), nr);
                ld8(tb + (uint32_t)(N + 8 * (ch + 1)), ni);
            }
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const float2 y = cmul(make_float2(__uint_as_float(vr[b]), __uint_as_float(vi[b])), P);
                P = cmul(P, st);
                if (live) {
                    if constexpr (E4M3) {
                        const uint32_t v = e4m3x2(y);
                        yp[0] = (uint8_t)(v & 0xFFu);
                        yp[ps] = (uint8_t)(v >> 8);
                    } else {
                        const __half2 v = __floats2half2_rn(y.x, y.y);
                        yp[0] = __low2half(v);
                        yp[ps] = __high2half(v);
                    }
                }
                yp += cs;
            }
            if (ch + 1 < C::NCH) {
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    vr[i] = nr[i];
                    vi[i] = ni[i];
                }
            }
        }
    };

    // ---- prologue: conversion and MMAs of the first item, the copy of item kST into the
    // buffer the first has left
    if (worker && cur < n_items) stage_p(0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // A operand: generic writes, MMA reads
    tc::fence_before();
    stop = __syncthreads_or(bad);
    if (!stop && ctl && cur < n_items) {
        tc::fence_after();
        stage_a(0);
        const unsigned itj = cur + (unsigned)kST * gridDim.x;
        if (itj < n_items) issue_copy(kST, itj);
    }

    // ---- steady state, item `cur` in buffer it & 1 (as the 128-row F-step)
    int it = 0;
    for (; !stop && cur < n_items; cur += gridDim.x, ++it) {
        const unsigned nxt = cur + gridDim.x;
        if (worker) {
            if (wait_phase(&S.bar, mma_par, &S.abort)) {
                mma_par ^= 1u;
            } else {
                bad = true;
                S.abort = 1;
                if (status) atomicOr(status, 1024);
            }
            tc::fence_after();
            if (!bad && nxt < n_items) stage_p(it + 1);   // the next item's conversion
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc::fence_before();
        if ((stop = __syncthreads_or(bad))) break;
        tc::fence_after();
        if (ctl && nxt < n_items) {
            stage_a((it + 1) & 1);
            // item it + 1 + kST into the buffer item it + 1 has just left
            const unsigned itj = nxt + (unsigned)kST * gridDim.x;
            if (itj < n_items) issue_copy(it + 1 + kST, itj);
        }
        if (worker) stage_e(it & 1, frs + (it % kNFR) * kF);
    }

    // ---- wind-down: after an abort the MMAs and the bulk copies in flight finish before the
    // CTA releases its tensor memory and exits (at most one copy per stage buffer)
    if (ctl && stop) {
        if (issued) {
            tc::mma_commit(&S.drained);
            if (!tc::wait_bounded(&S.drained, 0u, tc::kDrainCycles) && status) atomicOr(status, tc::kDrainGaveUp);
        }
        for (int b = 0; b < kST; ++b)
            if (n_cp[b] > 0 && !tc::wait_bounded(&S.ld_bar[b], (n_cp[b] - 1) & 1u, tc::kDrainCycles) && status)
                atomicOr(status, tc::kDrainGaveUp);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, C::TMEM);
    }
}

template <int N, bool E4M3>
cudaError_t launch_fd(const FArgs& a, cudaStream_t s)
{
    using C = FD<N>;
    constexpr size_t smem = 2 * C::BPLANE + 2 * C::APLANE + kST * C::STAGE + kNFR * kF * sizeof(FDTerm) +
                            sizeof(FDShared) + 128;
    static_assert(smem <= 227 * 1024, "shared memory");
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fstep_fd_kernel<N, E4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    if (a.bs % N != 0 || a.ktile != 0) return cudaErrorInvalidValue;
    const long long n_fg = (a.n_store + kF - 1) / kF, n_items = (long long)a.n * n_fg;
    if (n_items <= 0) return cudaSuccess;
    // the frame-term table in the scratch; frame numbers below 2^31 (32-bit block arithmetic)
    if (n_items >= (1LL << 31) || a.Kc <= 0 || a.Kc >= (1LL << 31) || a.Yt == nullptr ||
        a.m_begin + a.n_frames >= (1LL << 31) ||
        n_fg * kF >= (1LL << 31) ||
        (size_t)a.Yt_bytes < fstep_fd_scratch_bytes(N, a.n, a.n_store))
        return cudaErrorInvalidValue;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = n_items < sms ? n_items : sms;
    fd_terms_kernel<N><<<(unsigned)((n_items + kTermItems - 1) / kTermItems), 256, 0, s>>>(a, (unsigned)n_items,
                                                                                          (unsigned)n_fg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fstep_fd_kernel<N, E4M3><<<(unsigned)grid, kT, smem, s>>>(a, (unsigned)n_items, (unsigned)n_fg);
    count_extra_launches(1);   // the frame-term kernel
    return cudaGetLastError();
}

}  // namespace

size_t fstep_fd_scratch_bytes(int N, int n, long long n_store)
{
    (void)N;
    return (size_t)n * (size_t)((n_store + kF - 1) / kF) * kF * sizeof(FDTerm);
}

bool fstep_fd_supported(int N, int out_kind)
{
    return (N == 32 || N == 64 || N == 128) && (out_kind == FOUT_F16 || out_kind == FOUT_E4M3);
}

cudaError_t launch_fstep_fd(int N, int out_kind, const FArgs& a, cudaStream_t s)
{
    const bool e8 = out_kind == FOUT_E4M3;
    switch (N) {
        case 32: return e8 ? launch_fd<32, true>(a, s) : launch_fd<32, false>(a, s);
        case 64: return e8 ? launch_fd<64, true>(a, s) : launch_fd<64, false>(a, s);
        case 128: return e8 ? launch_fd<128, true>(a, s) : launch_fd<128, false>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mwax
