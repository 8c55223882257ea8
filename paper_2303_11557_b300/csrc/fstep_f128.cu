// Tensor-core F-step for the long fine-channel FFTs with full 128-row MMAs (Sec. 2.5.1:
// N = 128 N2, here 1280 = 128 x 10 and 6400 = 128 x 50), FP16 or e4m3 operands out (the
// FP16 and FP8 forms).  Four-step decomposition with the 128-point DFT on the tensor cores:
//   sample n = n1 + 128 n2, bin k = N2 k1 + k2,
//   stage P (CUDA cores, one thread per n1 of a frame, in registers):
//       Z[n1, k2] = e^{-2 pi i n1 k2 / N} sum_n2 x[n1 + 128 n2] e^{-2 pi i n2 k2 / N2}
//   stage A (tcgen05, both operands in shared memory, M = 128 bins k1, K = 128 samples n1):
//       X[N2 k1 + k2] = sum_n1 e^{-2 pi i k1 n1 / 128} Z[n1, k2]
//   stage E (CUDA cores, one lane per k1): the delay phasor (Sec. 4.3), the channel gain,
//       FP16 (re, im) into a shared-memory tile, then copied whole (coalesced) into the
//       item's frame-major scratch tile Yt[p][group][c][g], c = fftshift(k);
//   transpose (one launch per slot after the F-step's): Yt to the K-major operand planes
//       Y[slot][c][plane][p][Kpad] (FP16, or e4m3 when the gains carry the FP8 scales).
// Each frame's delay terms (FP64) and each item's mask of frames with data come from a small
// kernel launched before the F kernel: on this GPU's narrow FP64 pipe one lane's FP64 work
// costs a whole warp's issue time, and inside the F kernel it held every item's barrier.
// Writing the K-major rows straight from the bins (each item holds only G frames, so each
// lane's store lands in its own row and 2 MB page) measured several times slower than
// the whole F-step: the address translation of scattered rows, not DRAM, bounds it.
// Every accumulator lane is a bin row k1.  The B operand's rows are ordered (half of k2,
// k2 within the half, frame): a warp's lanes read the G frames of one bin from adjacent
// tensor-memory columns and write them as one row of the shared tile.  Z is rounded to
// FP16 once and the 128-point DFT matrix is FP16 (2^-12 per entry): the FP16 form's error
// bar holds widely.
//
// A persistent CTA (one per SM: 8 or 16 worker warps and a control warp) loops over the items (G
// frames of one path) of one integration slot, software-pipelined: while the worker warps run
// stage E of item j, the tensor cores run stage A of item j + 1 into the other half of
// tensor memory and the bulk copies of later items' int8 samples land; the control warp
// issues both; one CTA barrier per item.  Every
// wait is bounded (status word); loop exits are taken by all threads at that barrier.
#include "mwax_internal.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstring>

namespace mwax {
namespace {

constexpr int kM = 128;                 // bins k1 (MMA rows), samples n1 (MMA K)
// Worker threads (stages P and E) per length: 16 warps at N = 1280 (registers allow it),
// 8 at N = 6400 (the length-50 DFT holds 100 registers per thread); plus one control warp
// (copies, MMAs).
__host__ __device__ constexpr int f128_workers(int N2) { return N2 == 10 ? 512 : 256; }
constexpr uint32_t kLboF = 16 * 128;    // DFT matrix: 128 rows per K core column
constexpr uint32_t kFPlane = 16 * kLboF;
constexpr uint32_t kBufCols = 256;      // tensor-memory columns per accumulator buffer

template <int N2, int G>
struct F128 {
    static constexpr int N = kM * N2;
    static constexpr int H = N2 / 2;                          // bins k2 per warp half
    static constexpr int HS = (H * G + 7) / 8 * 8;            // B rows per half (padded)
    static constexpr int NA = 2 * HS;                         // MMA N
    static_assert(N2 % 2 == 0 && NA % 16 == 0 && 2 * NA <= (int)kBufCols, "MMA shape");
    static_assert(G == 2 || G == 4 || G == 8, "frames per item");
    // K core-column stride padded by 16 B: the 2- and 4-byte stores of stage P, whose
    // lanes walk along K, spread over all banks
    static constexpr uint32_t LBO_X = NA * 16 + 16;
    static constexpr uint32_t XPLANE = 16 * LBO_X;
    static constexpr uint32_t STAGE = G * 2 * N;              // int8 (re, im) of the item's frames
    // int8 stage buffers: two at N = 1280 (a short item's copy, issued one item ahead, did
    // not land in time: the workers waited on it for a third of the item), one at N = 6400
    // (its longer items hide the copy: a second buffer measured 3 % slower)
    static constexpr int ST = N2 == 10 ? 2 : 1;
    // stage P: one thread per sample n1 of a frame, or per pair (n1, n1 + 1) when there
    // are enough pairs for every thread (4-byte stores)
    static constexpr int W = f128_workers(N2);                // worker threads
    static constexpr int T = W + 32;                          // plus the control warp
    static constexpr int FS = W / 256;                        // frame groups of stage E
    static constexpr int FG = G / FS;                         // frames per stage-E warp
    static_assert(FG == G || FG == 4, "stage-E frame split");
    static constexpr bool PAIR = G * kM / 2 >= W;
    static constexpr int TASKS = PAIR ? G * kM / 2 : G * kM;
    static_assert(TASKS % W == 0, "whole tasks per thread");
    static constexpr int PER = TASKS / W;
    static constexpr int CB = 8 / G;                          // bins per 8-column load
    static constexpr int NCH = (H + CB - 1) / CB;             // loads per half and plane
    // stage E's tile in shared memory: channel c's G words at c * TS (16-byte rows padded so
    // that the lanes of a store phase, N2 channels apart, spread over the banks)
    static constexpr int TS = G == 8 ? 12 : G;
    static constexpr uint32_t TILE = (uint32_t)N * TS * 4;
    static_assert((NCH * CB - 1) * G + G <= HS, "loads stay inside the half's columns");
};

struct F128Frame {
    float phi0, d_hi, d_lo;  // delay terms: the phasor of bin offset u is e^{2 pi i (phi0 + u d)}
    int delay;
    float2 step;             // e^{2 pi i d}: phasor ratio between bins k and k + 1
};
// an item's G frame terms travel by bulk copy (16-byte multiples)
static_assert(sizeof(F128Frame) == 24, "frame terms: 24 bytes");

// Frames per item, and the bytes of one launch's scratch tiles (FP16 re, im words [item][c][g]).
constexpr int f128_frames(int N) { return N == 1280 ? 8 : 2; }
inline size_t f128_tiles_bytes(int N, int n, long long Kc)
{
    const int G = f128_frames(N);
    return (size_t)n * (size_t)((Kc + G - 1) / G) * G * (size_t)N * 4;
}

// Items of one launch: one integration slot, path-major, groups of G frames.
struct F128Items {
    unsigned n_items;    // paths x groups
    unsigned groups;     // groups of G frames per slot: ceil(Kc / G)
    unsigned slot;       // slot of the launch group
    F128Frame* tab;      // frame terms [item][G] (f128_terms_kernel)
    unsigned* masks;     // frames with data per item (f128_terms_kernel)
};

// Path, first frame (of the call) and frames in the slot (at most G) of an item.
template <int G>
__device__ __forceinline__ void item_pos(const F128Items& m, long long Kc, unsigned item, unsigned& p, long long& f0,
                                         int& nv)
{
    p = item / m.groups;
    const unsigned fg = item - p * m.groups;
    f0 = (long long)m.slot * Kc + (long long)fg * G;
    const long long left = Kc - (long long)fg * G;
    nv = left < G ? (int)left : G;
}

struct F128Shared {
    uint64_t ld_bar[2];      // an item's int8 frames staged, per stage buffer
    uint64_t bar;            // an item's stage-A MMAs complete
    uint64_t drained;        // after an abort: every MMA issued has completed
    unsigned ld_mask[2];     // frames of the staged item with data, per stage buffer
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

// Byte offset of element (row r, K index k) of a K-major no-swizzle operand: 8-row x 16-byte
// core matrices, 8-row groups 128 B apart, K core columns lbo apart.
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

__device__ __forceinline__ void ld4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}

// Bounded wait on an mbarrier phase; on a timeout or another thread's abort: false.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, const int* abort)
{
    const long long lim = (long long)tc::kDefaultSpin * 1000LL, t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity))
        if (*reinterpret_cast<const volatile int*>(abort) || clock64() - t0 > lim) return false;
    return true;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

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

// Forward DFTs X[k] = sum_n x[n] e^{-2 pi i n k / L} in registers, in place, natural order.
__device__ __forceinline__ void dft5(float2& x0, float2& x1, float2& x2, float2& x3, float2& x4)
{
    const float c1 = 0.30901699437494745f, s1 = 0.9510565162951535f;   // cos, sin 2 pi / 5
    const float c2 = -0.8090169943749473f, s2 = 0.5877852522924732f;   // cos, sin 4 pi / 5
    const float2 a1 = cadd(x1, x4), b1 = csub(x1, x4), a2 = cadd(x2, x3), b2 = csub(x2, x3);
    const float2 p1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
    const float2 p2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
    // X1 = p1 - i (s1 b1 + s2 b2), X2 = p2 - i (s2 b1 - s1 b2); X4, X3 their mirrors
    const float2 q1 = make_float2(s1 * b1.y + s2 * b2.y, -(s1 * b1.x + s2 * b2.x));
    const float2 q2 = make_float2(s2 * b1.y - s1 * b2.y, -(s2 * b1.x - s1 * b2.x));
    x0 = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
    x1 = cadd(p1, q1);
    x4 = csub(p1, q1);
    x2 = cadd(p2, q2);
    x3 = csub(p2, q2);
}

// Length 10 = 5 x 2: n = 2 a + b, k = k' + 5 k'': X = sum_b W10^{b k'} (-1)^{b k''} DFT5_a(x[2a+b])
__device__ __forceinline__ void dft10(float2 (&x)[10])
{
    const float2 e0[5] = {x[0], x[2], x[4], x[6], x[8]};
    float2 o[5] = {x[1], x[3], x[5], x[7], x[9]};
    float2 e[5] = {e0[0], e0[1], e0[2], e0[3], e0[4]};
    dft5(e[0], e[1], e[2], e[3], e[4]);
    dft5(o[0], o[1], o[2], o[3], o[4]);
    // W10^k' = e^{-2 pi i k' / 10}: cos / sin of 36 and 72 degrees
    const float ca = 0.8090169943749475f, sa = 0.5877852522924731f, cb = 0.30901699437494745f,
                sb = 0.9510565162951535f;
    o[1] = cmul(o[1], make_float2(ca, -sa));
    o[2] = cmul(o[2], make_float2(cb, -sb));
    o[3] = cmul(o[3], make_float2(-cb, -sb));
    o[4] = cmul(o[4], make_float2(-ca, -sa));
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        x[k] = cadd(e[k], o[k]);
        x[k + 5] = csub(e[k], o[k]);
    }
}

// Length 50 = 5 x 10: n = 10 a + b, k = k' + 5 k'': a length-5 DFT over a for each b, the
// twiddles W50^{b k'} (table w[j] = W50^j), then a length-10 DFT over b for each k', in
// place: bin k ends in slot 10 (k mod 5) + k / 5 (bin_slot).
__device__ __forceinline__ void dft50(float2 (&x)[50], const float2* w)
{
#pragma unroll
    for (int b = 0; b < 10; ++b) dft5(x[b], x[10 + b], x[20 + b], x[30 + b], x[40 + b]);
#pragma unroll
    for (int kp = 0; kp < 5; ++kp) {
        float2 z[10];
#pragma unroll
        for (int b = 0; b < 10; ++b) z[b] = (b * kp == 0) ? x[10 * kp + b] : cmul(x[10 * kp + b], w[b * kp]);
        dft10(z);
#pragma unroll
        for (int kk = 0; kk < 10; ++kk) x[10 * kp + kk] = z[kk];
    }
}

template <int L>
__host__ __device__ constexpr int bin_slot(int k)
{
    return L == 50 ? 10 * (k % 5) + k / 5 : k;
}

template <int L>
__device__ __forceinline__ void dft_n2(float2 (&x)[L], const float2* w)
{
    static_assert(L == 10 || L == 50, "stage-B lengths");
    if constexpr (L == 10) dft10(x);
    else dft50(x, w);
}

// The frames of an item with data: the others are read as zero (past the call's data or the
// slot, or in a zeroed block).  A frame never straddles a data block, whose length is a
// multiple of N.
template <int N2, int G>
__device__ __forceinline__ unsigned item_mask(const FArgs& a, const F128Items& m, unsigned item)
{
    constexpr int N = kM * N2;
    unsigned p;
    long long f0;
    int nv;
    item_pos<G>(m, a.Kc, item, p, f0, nv);
    const unsigned fpb = (unsigned)(a.bs / N);   // frames per data block
    const unsigned mf0 = (unsigned)(a.m_begin + f0), blk0 = mf0 / fpb;
    unsigned blk = blk0, fb = mf0 - blk0 * fpb, mask = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g < nv && f0 + g < a.n_frames && (a.flags == nullptr || a.flags[(long long)blk * a.n + p] == 0))
            mask |= 1u << g;
        if (++fb == fpb) {   // frame g + 1 lies in the next block
            fb = 0;
            ++blk;
        }
    }
    return mask;
}

// Stage an item: its frames with data (the mask of f128_terms_kernel; one bulk copy per run
// of consecutive frames with data in one data block) and its G frame terms, on one mbarrier
// transaction; publish the mask.  One thread.
template <int N2, int G>
__device__ __forceinline__ void issue_item(const FArgs& a, const F128Items& m, unsigned item, int8_t* stage,
                                               uint64_t* bar, unsigned* mask_out, const unsigned* masks,
                                               const F128Frame* tab, F128Frame* terms)
{
    constexpr int N = kM * N2;
    unsigned p;
    long long f0;
    int nv;
    item_pos<G>(m, a.Kc, item, p, f0, nv);
    const unsigned fpb = (unsigned)(a.bs / N);   // frames per data block
    const unsigned mf0 = (unsigned)(a.m_begin + f0), blk0 = mf0 / fpb, fb0 = mf0 - blk0 * fpb;
    const unsigned mask = __ldg(&masks[item]);
    // the mask is published before the arrive (release): a waiter that sees the phase
    // complete reads this item's mask
    *mask_out = mask;
    tc::mbar_arrive_expect_tx(bar, (uint32_t)(__popc(mask) * 2 * N) + (uint32_t)(G * sizeof(F128Frame)));
    bulk_copy(terms, tab + (size_t)item * G, (uint32_t)(G * sizeof(F128Frame)), bar);
    // one copy per run of consecutive frames with data inside one block (contiguous there)
    unsigned blk = blk0, fb = fb0;
    int g_run = -1;
    long long src_run = 0;
#pragma unroll
    for (int g = 0; g <= G; ++g) {
        const bool in = g < G && ((mask >> g) & 1u);
        if (g_run >= 0 && (!in || fb == 0)) {   // close the open run at a gap or a block edge
            bulk_copy(stage + g_run * 2 * N, a.volt + src_run, (uint32_t)((g - g_run) * 2 * N), bar);
            g_run = -1;
        }
        if (in && g_run < 0) {
            g_run = g;
            src_run = (((long long)blk * a.n + p) * (long long)a.bs + (long long)fb * N) * 2;
        }
        if (g < G && ++fb == fpb) {
            fb = 0;
            ++blk;
        }
    }
}

// B-operand row of bin k2 of frame g: rows grouped by half of k2, then bin, then frame.
template <int N2, int G>
__host__ __device__ constexpr int z_row(int k2, int g)
{
    return (k2 >= N2 / 2 ? F128<N2, G>::HS : 0) + (k2 % (N2 / 2)) * G + g;
}

// Stage P of one task: the length-N2 DFT over n2 of sample n1 of frame g (two samples n1,
// n1 + 1 with PAIR), the twiddles e^{-2 pi i n1 k2 / N}, FP16 rows of the B operand.
template <int N2, int G, bool PAIR>
__device__ __forceinline__ void stage_p_task(const int8_t* stage, bool live, int g, int n1, const float2* tw,
                                             const float2* w2, unsigned char* xre, unsigned char* xim)
{
    using C = F128<N2, G>;
    constexpr int N = C::N;
    constexpr int NS = PAIR ? 2 : 1;
    float2 x[NS][N2];
    const int8_t* src = stage + g * 2 * N + 2 * n1;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
        if constexpr (PAIR) {
            const char4 v = live ? *reinterpret_cast<const char4*>(src + 2 * kM * n2) : make_char4(0, 0, 0, 0);
            x[0][n2] = make_float2((float)v.x, (float)v.y);
            x[1][n2] = make_float2((float)v.z, (float)v.w);
        } else {
            const char2 v = live ? *reinterpret_cast<const char2*>(src + 2 * kM * n2) : make_char2(0, 0);
            x[0][n2] = make_float2((float)v.x, (float)v.y);
        }
    }
    float2 w[NS], E[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        dft_n2<N2>(x[s], w2);
        w[s] = __ldg(&tw[n1 + s]);   // e^{-2 pi i (n1 + s) / N}
        E[s] = w[s];
    }
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
        float2 z[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            z[s] = x[s][bin_slot<N2>(k2)];
            if (k2 > 0) {
                z[s] = cmul(z[s], E[s]);
                E[s] = cmul(E[s], w[s]);
            }
        }
        const uint32_t o = plain_off(z_row<N2, G>(k2, g), n1, C::LBO_X);
        if constexpr (PAIR) {
            const __half2 r2 = __floats2half2_rn(z[0].x, z[1].x), i2 = __floats2half2_rn(z[0].y, z[1].y);
            *reinterpret_cast<__half2*>(xre + o) = r2;
            *reinterpret_cast<__half2*>(xim + o) = i2;
        } else {
            *reinterpret_cast<__half*>(xre + o) = __float2half_rn(z[0].x);
            *reinterpret_cast<__half*>(xim + o) = __float2half_rn(z[0].y);
        }
    }
}

// Frame terms of an item's frame g: the delay phasor terms (the FP64 delay polynomial or
// table, Sec. 4.3).
template <int N2, int G>
__device__ __forceinline__ F128Frame frame_terms(const FArgs& a, const F128Items& m, unsigned item, int g)
{
    constexpr int N = kM * N2;
    unsigned p;
    long long f0;
    int nv;
    item_pos<G>(m, a.Kc, item, p, f0, nv);
    const long long f = f0 + g;
    F128Frame fi;
    fi.delay = 0;
    fi.phi0 = fi.d_hi = fi.d_lo = 0.0f;
    fi.step = make_float2(1.0f, 0.0f);
    if ((a.delay != nullptr || a.delay_tab != nullptr) && g < nv && f < a.n_frames) {
        const double tau = frame_delay(a, (int)p, a.m_begin + f, N);
        const double ph = a.nu * tau;
        fi.phi0 = (float)(ph - floor(ph));
        const double d = tau * a.fs_over_n;
        const float dh = __uint_as_float(__float_as_uint((float)d) & 0xFFFFF000u);
        fi.d_hi = dh;
        fi.d_lo = (float)(d - (double)dh);
        fi.delay = 1;
        float sn, cs;
        sincospif(2.0f * (float)(d - rint(d)), &sn, &cs);
        fi.step = make_float2(cs, sn);
    }
    return fi;
}

// Per launch, before the F kernel: every item's frame terms and mask, one thread per frame.
// The FP64 work runs here at full occupancy; the F kernel's control thread copies an item's
// terms into shared memory with its samples.
template <int N2, int G>
__global__ void __launch_bounds__(256) f128_terms_kernel(const FArgs a, const F128Items m)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)m.n_items * G) return;
    const unsigned item = (unsigned)(e / G);
    const int g = (int)(e - (long long)item * G);
    m.tab[e] = frame_terms<N2, G>(a, m, item, g);
    if (g == 0) m.masks[item] = item_mask<N2, G>(a, m, item);
}

// Rows (channels) per tensor-store box of an item's tile (padded tiles, N = 1280).
constexpr int kTileRows = 256;

template <int N2, int G>
__global__ void __launch_bounds__(F128<N2, G>::T, 1)
    fstep_f128_kernel(const FArgs a, const F128Items m, const __grid_constant__ CUtensorMap tm_tile)
{
    using C = F128<N2, G>;
    constexpr int N = C::N, H = C::H, HS = C::HS, NA = C::NA;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    unsigned char* f_re = sm;
    unsigned char* f_im = f_re + kFPlane;
    unsigned char* x_re = f_im + kFPlane;
    unsigned char* x_im = x_re + C::XPLANE;
    int8_t* stage = reinterpret_cast<int8_t*>(x_im + C::XPLANE);
    uint32_t* T = reinterpret_cast<uint32_t*>(stage + C::ST * C::STAGE);  // stage E tile [c][TS]
    float2* w2 = reinterpret_cast<float2*>(stage + C::ST * C::STAGE + C::TILE);   // W_N2^j, j < N2 (64 slots)
    // frame terms of ST + 2 items x G: items j .. j + ST + 1 are staged or in use while the
    // CTA's j-th item is in stage E
    F128Frame* frs = reinterpret_cast<F128Frame*>(w2 + 64);
    constexpr int NFR = C::ST + 2;
    F128Shared& S = *reinterpret_cast<F128Shared*>(frs + NFR * G);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kW = C::W, kT = C::T;
    const bool worker = tid < kW, ctl = tid == kW;   // ctl: lane 0 of the control warp
    int* status = a.status;
    unsigned n_cp[2] = {0u, 0u};   // copies issued per stage buffer (control thread)
    // copy item `itj`, the j-th of this CTA, into stage buffer j mod ST
    auto issue_copy = [&](int j, unsigned itj) {
        const int b = j % C::ST;
        issue_item<N2, G>(a, m, itj, stage + b * C::STAGE, &S.ld_bar[b], &S.ld_mask[b], m.masks, m.tab,
                          frs + (j % NFR) * G);
        ++n_cp[b];
    };

    // ---- set-up: the 128-point DFT matrix (A: rows k1, K = n1), the B operand zeroed (its
    // padding rows stay zero), the length-N2 twiddles, barriers, tensor memory
    for (int e = tid; e < kM * kM; e += kT) {
        const int k = e / kM, n = e % kM;
        float s, c;
        sincospif(-2.0f * (float)((k * n) % kM) / (float)kM, &s, &c);   // argument exact
        const uint32_t o = plain_off(k, n, kLboF);
        *reinterpret_cast<__half*>(f_re + o) = __float2half_rn(c);
        *reinterpret_cast<__half*>(f_im + o) = __float2half_rn(s);
    }
    for (uint32_t i = tid; i < 2 * C::XPLANE / 16; i += kT) reinterpret_cast<uint4*>(x_re)[i] = make_uint4(0, 0, 0, 0);
    for (int j = tid; j < N2; j += kT) w2[j] = __ldg(&a.tw[j * kM]);   // e^{-2 pi i 128 j / N} = W_N2^j
    unsigned cur = blockIdx.x;
    if (ctl) {
        tc::mbar_init(&S.ld_bar[0], 1);
        tc::mbar_init(&S.ld_bar[1], 1);
        tc::mbar_init(&S.bar, 1);
        tc::mbar_init(&S.drained, 1);
        S.abort = 0;
        tc::fence_mbar_init();
        // the first ST items' copies, one per stage buffer
        for (int j = 0; j < C::ST; ++j) {
            const unsigned itj = cur + (unsigned)j * gridDim.x;
            if (itj < m.n_items) issue_copy(j, itj);
        }
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, 2 * kBufCols);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    const int q = warp & 3, h = (warp >> 2) & 1, fq = warp >> 3;   // lane quarter, bin half, frame group
    const int k1 = 32 * q + lane;                  // a worker lane's bin row
    uint32_t mma_par = 0;
    bool bad = false, stop = false, issued = false;

    // stage P of an item (worker threads): its staged samples to the B operand
    auto stage_p = [&](int j) {   // the CTA's j-th item: stage buffer j mod ST, its (j / ST)-th copy
        const int b = j % C::ST;
        if (!wait_phase(&S.ld_bar[b], (uint32_t)(j / C::ST) & 1u, &S.abort)) {
            bad = true;
            S.abort = 1;   // lets the other threads' waits give up early
            if (status) atomicOr(status, 2048);
            return;
        }
        const unsigned mask = S.ld_mask[b];
        const int8_t* sb = stage + b * C::STAGE;
#pragma unroll
        for (int i = 0; i < C::PER; ++i) {
            const int t = tid + kW * i;
            const int g = C::PAIR ? t / (kM / 2) : t / kM;
            const int n1 = C::PAIR ? 2 * (t % (kM / 2)) : t % kM;
            stage_p_task<N2, G, C::PAIR>(sb, (mask >> g) & 1u, g, n1, a.tw, w2, x_re, x_im);
        }
    };

    // stage A of the item staged in the B operand, into accumulator buffer `buf` (control
    // thread): re = Fr Zr - Fi Zi, im = Fr Zi + Fi Zr
    auto stage_a = [&](int buf) {
        const uint32_t id = tc::idesc(0, kM, NA, false), id_neg = tc::idesc(0, kM, NA, true);
        const uint64_t ar = desc_plain(tc::smem_u32(f_re), kLboF), ai = desc_plain(tc::smem_u32(f_im), kLboF);
        const uint64_t br = desc_plain(tc::smem_u32(x_re), C::LBO_X), bi = desc_plain(tc::smem_u32(x_im), C::LBO_X);
        const uint32_t dre = tmem + (uint32_t)buf * kBufCols, dim = dre + NA;
#pragma unroll
        for (int ks = 0; ks < kM / 16; ++ks) {
            const uint32_t acc = ks > 0 ? 1u : 0u;
            const uint64_t oa = (uint64_t)((ks * 2u * kLboF) >> 4), ob = (uint64_t)((ks * 2u * C::LBO_X) >> 4);
            tc::mma_f16(dre, ar + oa, br + ob, id, acc);
            tc::mma_f16(dre, ai + oa, bi + ob, id_neg, 1u);
            tc::mma_f16(dim, ar + oa, bi + ob, id, acc);
            tc::mma_f16(dim, ai + oa, br + ob, id, 1u);
        }
        tc::mma_commit(&S.bar);
        issued = true;
    };

    // stage E of an item from accumulator buffer `buf` (worker threads): bins
    // k = N2 k1 + k2, k2 in this warp's half; phasor, gain, FP16 (re, im) of the G frames
    // into the shared-memory tile T
    auto stage_e_all = [&](int buf, const F128Frame* fr) {
        const bool lowk = k1 < kM / 2;                  // k < N/2: u = k; else u = k - N
        const int k0 = N2 * k1 + H * h;                 // this lane's first bin
        float2 P[G], st[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const F128Frame& fi = fr[g];
            P[g] = fi.delay ? phasor_u(fi.phi0, fi.d_hi, fi.d_lo, lowk ? k0 : k0 - N) : make_float2(1.0f, 0.0f);
            st[g] = fi.step;
        }
        const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * kBufCols + (uint32_t)(h * HS);
        // chunk ch + 1's tensor-memory columns and gains load while chunk ch is processed
        uint32_t vr[8], vi[8], nr[8], ni[8];
        float gc[C::CB], gnx[C::CB];
        auto gains = [&](int ch, float (&gv)[C::CB]) {
#pragma unroll
            for (int b = 0; b < C::CB; ++b) {
                const int k = k0 + min(ch * C::CB + b, H - 1);
                gv[b] = __ldg(&a.gain[lowk ? k + N / 2 : k - N / 2]);
            }
        };
        ld8(tb, vr);
        ld8(tb + (uint32_t)NA, vi);
        gains(0, gc);
        tc::tmem_wait_ld();
#pragma unroll
        for (int ch = 0; ch < C::NCH; ++ch) {
            if (ch + 1 < C::NCH) {
                ld8(tb + (uint32_t)(8 * (ch + 1)), nr);
                ld8(tb + (uint32_t)(NA + 8 * (ch + 1)), ni);
                gains(ch + 1, gnx);
            }
#pragma unroll
            for (int b = 0; b < C::CB; ++b) {
                const int kk = ch * C::CB + b;
                if (kk >= H) break;
                const int k = k0 + kk;
                const int c = lowk ? k + N / 2 : k - N / 2;   // fftshift
                const float gn = gc[b];
                uint32_t hv[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    float2 y = make_float2(__uint_as_float(vr[b * G + g]), __uint_as_float(vi[b * G + g]));
                    y = cmul(y, P[g]);
                    P[g] = cmul(P[g], st[g]);
                    const __half2 v = __floats2half2_rn(y.x * gn, y.y * gn);
                    hv[g] = *reinterpret_cast<const uint32_t*>(&v);
                }
                uint32_t* t = T + c * C::TS;
                if constexpr (G == 8) {
                    reinterpret_cast<uint4*>(t)[0] = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                    reinterpret_cast<uint4*>(t)[1] = make_uint4(hv[4], hv[5], hv[6], hv[7]);
                } else if constexpr (G == 4) {
                    *reinterpret_cast<uint4*>(t) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                } else {
                    *reinterpret_cast<uint2*>(t) = make_uint2(hv[0], hv[1]);
                }
            }
            if (ch + 1 < C::NCH) {
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    vr[i] = nr[i];
                    vi[i] = ni[i];
                }
#pragma unroll
                for (int b = 0; b < C::CB; ++b) gc[b] = gnx[b];
            }
        }
    };

    // stage E with the frames split over two warp groups (16 worker warps): warp group fq
    // takes frames FG fq .. FG fq + FG - 1 of every bin of its half; per bin one 4-column
    // tensor-memory load per plane, the next bin's loads and gain in flight
    auto stage_e_split = [&](int buf, const F128Frame* fr) {
        constexpr int FG = C::FG;
        const int g0 = fq * FG;
        const bool lowk = k1 < kM / 2;
        const int k0 = N2 * k1 + H * h;
        float2 P[FG], st[FG];
#pragma unroll
        for (int j = 0; j < FG; ++j) {
            const F128Frame& fi = fr[g0 + j];
            P[j] = fi.delay ? phasor_u(fi.phi0, fi.d_hi, fi.d_lo, lowk ? k0 : k0 - N) : make_float2(1.0f, 0.0f);
            st[j] = fi.step;
        }
        const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * kBufCols + (uint32_t)(h * HS + g0);
        auto gain_of = [&](int kk) {
            const int k = k0 + kk;
            return __ldg(&a.gain[lowk ? k + N / 2 : k - N / 2]);
        };
        uint32_t vr[4], vi[4], nr[4], ni[4];
        ld4(tb, vr);
        ld4(tb + (uint32_t)NA, vi);
        float gc = gain_of(0), gnx = 0.0f;
        tc::tmem_wait_ld();
#pragma unroll
        for (int kk = 0; kk < H; ++kk) {
            if (kk + 1 < H) {
                ld4(tb + (uint32_t)((kk + 1) * G), nr);
                ld4(tb + (uint32_t)(NA + (kk + 1) * G), ni);
                gnx = gain_of(kk + 1);
            }
            const int k = k0 + kk;
            const int c = lowk ? k + N / 2 : k - N / 2;   // fftshift
            uint32_t hv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 y = make_float2(__uint_as_float(vr[j]), __uint_as_float(vi[j]));
                y = cmul(y, P[j]);
                P[j] = cmul(P[j], st[j]);
                const __half2 v = __floats2half2_rn(y.x * gc, y.y * gc);
                hv[j] = *reinterpret_cast<const uint32_t*>(&v);
            }
            *reinterpret_cast<uint4*>(T + c * C::TS + g0) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
            if (kk + 1 < H) {
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    vr[i] = nr[i];
                    vi[i] = ni[i];
                }
                gc = gnx;
            }
        }
    };
    auto stage_e = [&](int buf, const F128Frame* fr) {
        if constexpr (C::FS == 1) stage_e_all(buf, fr);
        else stage_e_split(buf, fr);
    };

    // the tile of an item into its scratch tile Yt[c][g].  The padded tile (N = 1280): tensor
    // stores by the bulk-copy engine (one worker thread, after the workers' fence and
    // barrier) whose boxes end past the rows, so the padding is not written; the workers go
    // on to the next item.  The dense tile (N = 6400): the worker threads, 16-byte copies, a
    // warp writing 512 contiguous bytes (one 51 KB bulk store per item measured 9 % slower over
    // the F-step, the stores draining long after the item loop; 16 bulk stores of 3.2 KB, 1.5 %).
    constexpr bool kTmaTile = C::TS != G;
    auto store_tile = [&](unsigned item) {
#pragma unroll
        for (int i = 0; i < N / kTileRows; ++i)
            tc::tma_store_2d(&tm_tile, T + i * kTileRows * C::TS, 0, (int)(item * (unsigned)N) + i * kTileRows);
        tc::bulk_commit();
    };
    auto copy_out = [&](unsigned item) {
        uint4* dst = reinterpret_cast<uint4*>(static_cast<uint32_t*>(a.Yt) + (size_t)item * N * G);
        for (int q = tid; q < N * G / 4; q += kW) {
            const int c = q / (G / 4 > 0 ? G / 4 : 1);
            uint4 v;
            if constexpr (G >= 4) {
                v = *reinterpret_cast<const uint4*>(T + c * C::TS + 4 * (q % (G / 4)));
            } else {
                // G = 2: two channels per 16 bytes
                const uint2 lo = *reinterpret_cast<const uint2*>(T + (2 * q) * C::TS);
                const uint2 hi = *reinterpret_cast<const uint2*>(T + (2 * q + 1) * C::TS);
                v = make_uint4(lo.x, lo.y, hi.x, hi.y);
            }
            dst[q] = v;
        }
    };

    // ---- prologue: stage P and stage A of the first item, the copy of the second
    if (worker && cur < m.n_items) stage_p(0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B operand: generic writes, MMA reads
    tc::fence_before();
    stop = __syncthreads_or(bad);
    if (!stop && ctl && cur < m.n_items) {
        tc::fence_after();
        stage_a(0);
        const unsigned itj = cur + (unsigned)C::ST * gridDim.x;   // item ST, into buffer 0
        if (itj < m.n_items) issue_copy(C::ST, itj);
    }

    // ---- steady state, item `cur` in buffer it & 1.  Workers: wait for its MMAs, stage P of
    // the next item.  Barrier.  Then the control thread issues stage A of the next item and
    // the copy of a later one (samples and frame terms; the control warp shares its scheduler
    // with four worker warps, so its own work is kept short), and the workers run stage E of
    // `cur`.
    int it = 0;
    for (; !stop && cur < m.n_items; cur += gridDim.x, ++it) {
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
            if (!bad && nxt < m.n_items) stage_p(it + 1);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (kTmaTile && tid == 0) tc::bulk_wait_read_all();   // the last tile read out: stage E may rewrite it
        tc::fence_before();
        if ((stop = __syncthreads_or(bad))) break;
        tc::fence_after();
        if (ctl && nxt < m.n_items) {
            stage_a((it + 1) & 1);
            // item it + 1 + ST into the buffer item it + 1 has just left
            const unsigned itj = nxt + (unsigned)C::ST * gridDim.x;
            if (itj < m.n_items) issue_copy(it + 1 + C::ST, itj);
        }
        if (worker) {
            stage_e(it & 1, frs + (it % NFR) * G);
            if constexpr (kTmaTile) tc::fence_proxy_async();
            asm volatile("bar.sync 1, %0;" ::"n"(kW) : "memory");   // the worker warps' tile complete
            if constexpr (kTmaTile) {
                if (tid == 0) store_tile(cur);
            } else {
                copy_out(cur);
            }
        }
    }

    // ---- wind-down: after an abort the MMAs and the bulk copies in flight finish before the
    // CTA releases its tensor memory and exits (at most one copy per stage buffer)
    if (ctl && stop) {
        if (issued) {
            tc::mma_commit(&S.drained);
            if (!tc::wait_bounded(&S.drained, 0u, tc::kDrainCycles) && status) atomicOr(status, tc::kDrainGaveUp);
        }
        for (int b = 0; b < C::ST; ++b)
            if (n_cp[b] > 0 && !tc::wait_bounded(&S.ld_bar[b], (n_cp[b] - 1) & 1u, tc::kDrainCycles) && status)
                atomicOr(status, tc::kDrainGaveUp);
    }
    if (kTmaTile && tid == 0) tc::bulk_wait_all();   // the tile stores complete before the CTA exits
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 2 * kBufCols);
    }
}

// Transpose of one slot's scratch tiles Yt[p][group][c][g] (FP16 re, im) into the K-major
// operand planes of that slot, Y[c][plane][p][Kpad]: a CTA takes one path, kTrC channels
// and up to 8192 / kTrC frames; it reads the groups' kTrC-channel runs (whole sectors),
// turns them in shared memory and writes 2 kTrC rows of up to 16384 / kTrC bytes.  (Run
// beside the next slot's F-step on a second stream it gained little: the F-step's CTAs
// fill the SMs, and a transpose thin enough to fit beside them is latency-bound.)
constexpr int kTrWords = 8192;   // 32 KB tile
template <int G, int kTrC, bool E4M3>
__global__ void __launch_bounds__(256) f128_transpose_kernel(const uint32_t* __restrict__ Yt, void* __restrict__ Yv,
                                                             int N, int n, long long Kpad, unsigned groups, int kn)
{
    constexpr int kTrK = kTrWords / kTrC;
    __shared__ __align__(16) uint32_t S[kTrC][kTrK + 4];
    const int cblocks = N / kTrC, kblocks = (int)((Kpad + kTrK - 1) / kTrK);
    const long long tiles = (long long)n * cblocks * kblocks;
    for (long long b = blockIdx.x; b < tiles; b += gridDim.x) {
    const int kb = (int)(b % kblocks), cb = (int)((b / kblocks) % cblocks), p = (int)(b / ((long long)kblocks * cblocks));
    const int c0 = cb * kTrC, k0 = kb * kTrK;
    const int kt = max(0, min(kTrK, kn - k0));              // frames with data in this tile
    const int kw = (int)min((long long)kTrK, Kpad - k0);    // frames written: whole rows to Kpad
    const int ng = (kt + G - 1) / G;   // groups in this tile
    // read: group fg's words (c0 .. c0 + kTrC - 1) x G are contiguous 16-byte chunks
    constexpr int CH = kTrC * G / 4;
    const uint4* src = reinterpret_cast<const uint4*>(Yt + ((size_t)p * groups + k0 / G) * N * G + (size_t)c0 * G);
#pragma unroll 4
    for (int e = threadIdx.x; e < ng * CH; e += blockDim.x) {
        const int fg = e / CH, r4 = e % CH;
        const uint4 v = __ldg(src + (size_t)fg * (N * G / 4) + r4);
        if constexpr (G >= 4) {
            const int c = 4 * r4 / G, g = 4 * r4 % G;
            *reinterpret_cast<uint4*>(&S[c][fg * G + g]) = v;
        } else {
            const int c = 2 * r4;   // G = 2: two channels per chunk
            *reinterpret_cast<uint2*>(&S[c][fg * 2]) = make_uint2(v.x, v.y);
            *reinterpret_cast<uint2*>(&S[c + 1][fg * 2]) = make_uint2(v.z, v.w);
        }
    }
    __syncthreads();
    // write: row (c, plane), frames k0 .. k0 + kw - 1 (zeros past the data: whole rows up to
    // Kpad, so every store fills its sectors), 8 frames per thread step
    const long long ps = (long long)n * Kpad;
    const int segs = kw / 8;   // Kpad is a multiple of 8
    for (int e = threadIdx.x; e < kTrC * 2 * segs; e += blockDim.x) {
        const int j = e % segs, row = e / segs, c = row >> 1, plane = row & 1;
        const long long at = ((long long)(c0 + c) * 2 * n + p) * Kpad + plane * ps + k0 + 8 * j;
        uint32_t w8[8];   // the tile's (re, im) words of the 8 frames, 0 past the data
        if (8 * j + 8 <= kt) {
            const uint4 a0 = *reinterpret_cast<const uint4*>(&S[c][8 * j]);
            const uint4 a1 = *reinterpret_cast<const uint4*>(&S[c][8 * j + 4]);
            w8[0] = a0.x; w8[1] = a0.y; w8[2] = a0.z; w8[3] = a0.w;
            w8[4] = a1.x; w8[5] = a1.y; w8[6] = a1.z; w8[7] = a1.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) w8[i] = 8 * j + i < kt ? S[c][8 * j + i] : 0u;
        }
        const uint32_t sel = plane ? 0x7632u : 0x5410u;   // the re (low) or im (high) halves
        if constexpr (E4M3) {
            // the FP8 form: the tile holds v / s as FP16; e4m3 bytes, 8 frames per 8 bytes
            uint32_t w[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const uint32_t h01 = __byte_perm(w8[4 * i], w8[4 * i + 1], sel);
                const uint32_t h23 = __byte_perm(w8[4 * i + 2], w8[4 * i + 3], sel);
                const float2 f01 = __half22float2(*reinterpret_cast<const __half2*>(&h01));
                const float2 f23 = __half22float2(*reinterpret_cast<const __half2*>(&h23));
                w[i] = e4m3x2(f01) | (e4m3x2(f23) << 16);
            }
            *reinterpret_cast<uint2*>(static_cast<uint8_t*>(Yv) + at) = make_uint2(w[0], w[1]);
        } else {
            *reinterpret_cast<uint4*>(static_cast<__half*>(Yv) + at) =
                make_uint4(__byte_perm(w8[0], w8[1], sel), __byte_perm(w8[2], w8[3], sel),
                           __byte_perm(w8[4], w8[5], sel), __byte_perm(w8[6], w8[7], sel));
        }
    }
    __syncthreads();   // S is refilled by the next tile
    }
}

template <int N2, int G, bool E4M3>
cudaError_t launch_f128(const FArgs& a, cudaStream_t s)
{
    using C = F128<N2, G>;
    constexpr size_t smem = 2 * kFPlane + 2 * C::XPLANE + C::ST * C::STAGE + C::TILE + sizeof(float2) * 64 +
                            (C::ST + 2) * G * sizeof(F128Frame) + sizeof(F128Shared) + 128;
    static_assert(smem <= 227 * 1024, "shared memory");
    static_assert(G == f128_frames(C::N), "frames per item");
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fstep_f128_kernel<N2, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    if (a.bs % C::N != 0 || a.Kc <= 0 || a.m_begin + a.n_frames >= (1LL << 31)) return cudaErrorInvalidValue;
    if (a.n_store <= 0 || a.n <= 0) return cudaSuccess;
    const long long groups = (a.Kc + G - 1) / G, slots = (a.n_store + a.Kc - 1) / a.Kc;
    const long long n_items = (long long)a.n * groups;
    // tile rows (item x N) are 32-bit tensor coordinates
    if (n_items * C::N >= (1LL << 31) || (size_t)a.Yt_bytes < fstep_f128_scratch_bytes(C::N, a.n, a.Kc))
        return cudaErrorInvalidValue;
    CUtensorMap tm_tile;
    memset(&tm_tile, 0, sizeof tm_tile);
    if constexpr (C::TS != G) {
        static_assert(C::N % kTileRows == 0 && (C::TS * 4) % 16 == 0, "tile boxes");
        cudaError_t e = make_rows_tmap(&tm_tile, a.Yt, G, n_items * C::N, C::TS, kTileRows);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = n_items < sms ? n_items : sms;
    const long long slot_elems = (long long)C::N * 2 * a.n * a.Kpad;
    // behind the scratch tiles: the frame terms and masks of one launch
    char* tail = static_cast<char*>(a.Yt) + f128_tiles_bytes(C::N, a.n, a.Kc);
    for (long long sl = 0; sl < slots; ++sl) {
        F128Items m;
        m.n_items = (unsigned)n_items;
        m.groups = (unsigned)groups;
        m.slot = (unsigned)sl;
        m.tab = reinterpret_cast<F128Frame*>(tail);
        m.masks = reinterpret_cast<unsigned*>(tail + (size_t)n_items * G * sizeof(F128Frame));
        f128_terms_kernel<N2, G><<<(unsigned)((n_items * G + 255) / 256), 256, 0, s>>>(a, m);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        fstep_f128_kernel<N2, G><<<(unsigned)grid, C::T, smem, s>>>(a, m, tm_tile);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const long long left = a.n_store - sl * a.Kc;
        const int kn = (int)(left < a.Kc ? left : a.Kc);   // frames stored in this slot
        constexpr int TRC = G >= 8 ? 32 : 64, TRK = kTrWords / TRC;   // channels, frames per transpose tile
        const long long tiles = (long long)a.n * (C::N / TRC) * ((a.Kpad + TRK - 1) / TRK);
        void* ys = static_cast<char*>(a.Y) + sl * slot_elems * (E4M3 ? 1 : 2);
        f128_transpose_kernel<G, TRC, E4M3><<<(unsigned)tiles, 256, 0, s>>>(static_cast<const uint32_t*>(a.Yt), ys, C::N,
                                                                           a.n, a.Kpad, (unsigned)groups, kn);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        count_extra_launches(sl == 0 ? 2 : 3);   // frame terms, F kernel, transpose per slot
    }
    return cudaSuccess;
}

}  // namespace

bool fstep_f128_supported(int N) { return N == 1280 || N == 6400; }

size_t fstep_f128_scratch_bytes(int N, int n, long long Kc)
{
    const int G = f128_frames(N);
    const size_t items = (size_t)n * (size_t)((Kc + G - 1) / G);
    return f128_tiles_bytes(N, n, Kc) + items * (G * sizeof(F128Frame) + sizeof(unsigned));
}

cudaError_t launch_fstep_f128(int N, int out_kind, const FArgs& a, cudaStream_t s)
{
    const bool e4m3 = out_kind == FOUT_E4M3;
    if (!e4m3 && out_kind != FOUT_F16) return cudaErrorInvalidValue;
    switch (N) {
        case 1280: return e4m3 ? launch_f128<10, 8, true>(a, s) : launch_f128<10, 8, false>(a, s);
        case 6400: return e4m3 ? launch_f128<50, 2, true>(a, s) : launch_f128<50, 2, false>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mwax
