// F-step of the MWAX FX correlator (Sec. 2.5.1): int8 unpack, fine-channel FFT,
// per-path delay/phase correction (Sec. 2.5.1, 4.3), channel shift (Sec. 2.6) and the
// store of X-engine operands.
//
// One CTA transforms FB consecutive frames of one signal path.  The frames' int8
// samples are staged in shared memory with 16-byte loads, then an out-of-place Stockham
// FFT runs pass by pass in shared memory (radix-R butterflies in registers, ping-pong
// buffers), and the last pass multiplies by the delay phasor and writes the operand
// planes straight to global memory.  Lanes of a warp take consecutive frames, so the
// final stores are contiguous along the frame (K) axis of the K-major operand layout
//     Y[slot][c][plane][p][Kpad]   (plane 0 = re, 1 = im).
#include "mwax_internal.cuh"

namespace mwax {
namespace {

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_mul_negi(float2 a) { return make_float2(a.y, -a.x); }  // -i a

// In-register forward DFTs, X_k = sum_r v_r e^{-2 pi i r k / R}.
template <int R>
struct Dft;

template <>
struct Dft<2> {
    __device__ __forceinline__ static void run(float2 (&v)[2])
    {
        float2 a = v[0], b = v[1];
        v[0] = c_add(a, b);
        v[1] = c_sub(a, b);
    }
};

template <>
struct Dft<4> {
    __device__ __forceinline__ static void run(float2 (&v)[4])
    {
        float2 t0 = c_add(v[0], v[2]), t1 = c_sub(v[0], v[2]);
        float2 t2 = c_add(v[1], v[3]), t3 = c_mul_negi(c_sub(v[1], v[3]));
        v[0] = c_add(t0, t2);
        v[2] = c_sub(t0, t2);
        v[1] = c_add(t1, t3);
        v[3] = c_sub(t1, t3);
    }
};

template <>
struct Dft<5> {
    __device__ __forceinline__ static void run(float2 (&v)[5])
    {
        const float c1 = 0.30901699437494745f, s1 = 0.9510565162951535f;   // cos, sin 2pi/5
        const float c2 = -0.8090169943749473f, s2 = 0.5877852522924732f;   // cos, sin 4pi/5
        float2 a1 = c_add(v[1], v[4]), b1 = c_sub(v[1], v[4]);
        float2 a2 = c_add(v[2], v[3]), b2 = c_sub(v[2], v[3]);
        float2 x0 = v[0];
        float2 p1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
        float2 p2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
        float2 q1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
        float2 q2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
        v[0] = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
        v[1] = c_add(p1, c_mul_negi(q1));
        v[4] = c_sub(p1, c_mul_negi(q1));
        v[2] = c_add(p2, c_mul_negi(q2));
        v[3] = c_sub(p2, c_mul_negi(q2));
    }
};

template <>
struct Dft<8> {
    __device__ __forceinline__ static void run(float2 (&v)[8])
    {
        const float h = 0.7071067811865476f;
        float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4>::run(e);
        Dft<4>::run(o);
        o[1] = c_mul(o[1], make_float2(h, -h));
        o[2] = c_mul_negi(o[2]);
        o[3] = c_mul(o[3], make_float2(-h, -h));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = c_add(e[k], o[k]);
            v[k + 4] = c_sub(e[k], o[k]);
        }
    }
};

template <>
struct Dft<16> {
    __device__ __forceinline__ static void run(float2 (&v)[16])
    {
        // e^{-2 pi i k / 16}, k = 0..7
        const float2 w[8] = {make_float2(1.0f, 0.0f),
                             make_float2(0.9238795325112867f, -0.3826834323650898f),
                             make_float2(0.7071067811865476f, -0.7071067811865475f),
                             make_float2(0.38268343236508984f, -0.9238795325112867f),
                             make_float2(0.0f, -1.0f),
                             make_float2(-0.3826834323650897f, -0.9238795325112867f),
                             make_float2(-0.7071067811865475f, -0.7071067811865476f),
                             make_float2(-0.9238795325112867f, -0.3826834323650899f)};
        float2 e[8], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        Dft<8>::run(e);
        Dft<8>::run(o);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float2 t = (k == 0) ? o[0] : (k == 4 ? c_mul_negi(o[4]) : c_mul(o[k], w[k]));
            v[k] = c_add(e[k], t);
            v[k + 8] = c_sub(e[k], t);
        }
    }
};

template <>
struct Dft<32> {
    __device__ __forceinline__ static void run(float2 (&v)[32])
    {
        // e^{-2 pi i k / 32}, k = 0..15
        const float2 w[16] = {make_float2(1.0f, 0.0f),
                              make_float2(0.9807852804032304f, -0.19509032201612825f),
                              make_float2(0.9238795325112867f, -0.3826834323650898f),
                              make_float2(0.8314696123025452f, -0.5555702330196022f),
                              make_float2(0.7071067811865476f, -0.7071067811865475f),
                              make_float2(0.5555702330196023f, -0.8314696123025452f),
                              make_float2(0.38268343236508984f, -0.9238795325112867f),
                              make_float2(0.19509032201612833f, -0.9807852804032304f),
                              make_float2(0.0f, -1.0f),
                              make_float2(-0.1950903220161282f, -0.9807852804032304f),
                              make_float2(-0.3826834323650897f, -0.9238795325112867f),
                              make_float2(-0.555570233019602f, -0.8314696123025455f),
                              make_float2(-0.7071067811865475f, -0.7071067811865476f),
                              make_float2(-0.8314696123025453f, -0.5555702330196022f),
                              make_float2(-0.9238795325112867f, -0.3826834323650899f),
                              make_float2(-0.9807852804032304f, -0.1950903220161286f)};
        float2 e[16], o[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        Dft<16>::run(e);
        Dft<16>::run(o);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float2 t = (k == 0) ? o[0] : (k == 8 ? c_mul_negi(o[8]) : c_mul(o[k], w[k]));
            v[k] = c_add(e[k], t);
            v[k + 16] = c_sub(e[k], t);
        }
    }
};

template <int R>
struct DftIf {   // radix-1 "DFT" is the identity
    __device__ __forceinline__ static void run(float2 (&v)[R]) { Dft<R>::run(v); }
};
template <>
struct DftIf<1> {
    __device__ __forceinline__ static void run(float2 (&)[1]) {}
};

// Radix schedule per FFT length (applied in this order).
template <int N>
struct Sched;
#define MWAX_SCHED(NN, FBV, NTV, ...)                                             \
    template <>                                                                   \
    struct Sched<NN> {                                                            \
        static constexpr int fb = FBV;                                            \
        static constexpr int nt = NTV;                                            \
        static constexpr int radix[4] = {__VA_ARGS__};                            \
        static constexpr int passes = sizeof(radix) / sizeof(int) - count1(radix); \
    };
__host__ __device__ constexpr int count1(const int (&r)[4])
{
    return (r[0] == 1) + (r[1] == 1) + (r[2] == 1) + (r[3] == 1);
}
// (N, frames per CTA, threads per CTA, radices).  Above N = 512 the frames and threads are
// chosen so that two ping-pong buffers of fb frames still leave 16 warps resident per SM.
#ifndef MWAX_FB640
#define MWAX_FB640 16
#endif
#ifndef MWAX_NT640
#define MWAX_NT640 512
#endif
#ifndef MWAX_FB1280
#define MWAX_FB1280 8
#endif
#ifndef MWAX_NT1280
#define MWAX_NT1280 512
#endif
#ifndef MWAX_FB3200
#define MWAX_FB3200 2
#endif
#ifndef MWAX_NT3200
#define MWAX_NT3200 256
#endif
#ifndef MWAX_FB6400
#define MWAX_FB6400 2
#endif
#ifndef MWAX_NT6400
#define MWAX_NT6400 512
#endif
MWAX_SCHED(16, 32, 256, 16, 1, 1, 1)
MWAX_SCHED(32, 32, 256, 8, 4, 1, 1)
MWAX_SCHED(64, 32, 256, 8, 8, 1, 1)
MWAX_SCHED(128, 32, 256, 16, 8, 1, 1)
MWAX_SCHED(256, 32, 256, 16, 16, 1, 1)
MWAX_SCHED(512, 16, 256, 8, 8, 8, 1)
MWAX_SCHED(640, MWAX_FB640, MWAX_NT640, 16, 8, 5, 1)
MWAX_SCHED(1280, MWAX_FB1280, MWAX_NT1280, 16, 16, 5, 1)
MWAX_SCHED(3200, MWAX_FB3200, MWAX_NT3200, 16, 8, 5, 5)
MWAX_SCHED(6400, MWAX_FB6400, MWAX_NT6400, 16, 16, 5, 5)
#undef MWAX_SCHED

template <int N, int P>
struct PassNs {  // product of the radices before pass P
    static constexpr int value = PassNs<N, P - 1>::value * Sched<N>::radix[P - 1];
};
template <int N>
struct PassNs<N, 0> {
    static constexpr int value = 1;
};


// Per-frame data shared by the CTA.
struct FrameInfo {
    long long slot;   // operand slot (integration within the launch), -1 = no frame
    long long k;      // frame index within the slot
    float phi0;       // frac(nu * tau) [cycles]
    float d_hi;       // tau Fs / N [cycles per bin], top 12 significant bits
    float d_lo;       // the rest
    int delay;
    float2 step;      // e^{2 pi i (N/R_last) d}: phasor ratio between a thread's outputs
    float2 wrap;      // e^{-2 pi i N d}: outputs past N/2 sit at u = k - N
};

template <int N, int OUTK>
struct Store {
    // Write one corrected spectral value: real plane at element `at`, imaginary plane at
    // `at + plane_stride` of the operand buffer (FP32, or FP16, v already carrying the
    // power-of-two pre-scale through the channel gain;
    // FP16 pairs: the remainder v - hi, exact in FP32, rounded again to FP16 half a row
    // further on, so hi + lo carries 22 significant bits).
    __device__ __forceinline__ static void run(const FArgs& a, long long at, long long plane_stride, float2 v,
                                               long long /*slot*/, int /*c*/, int /*p*/)
    {
        if (OUTK == FOUT_F32) {
            float* Y = static_cast<float*>(a.Y);
            Y[at] = v.x;
            Y[at + plane_stride] = v.y;
        } else if (OUTK == FOUT_F16X3) {
            __half* Y = static_cast<__half*>(a.Y);
            const long long lo = a.Kpad >> 1;
            const float xr = v.x, xi = v.y;
            const __half hr = __float2half_rn(xr), hi = __float2half_rn(xi);
            Y[at] = hr;
            Y[at + plane_stride] = hi;
            Y[at + lo] = __float2half_rn(xr - __half2float(hr));
            Y[at + plane_stride + lo] = __float2half_rn(xi - __half2float(hi));
        } else if (OUTK == FOUT_E4M3) {
            uint8_t* Y = static_cast<uint8_t*>(a.Y);
            const uint32_t q = e4m3x2(v);
            Y[at] = (uint8_t)(q & 0xFFu);
            Y[at + plane_stride] = (uint8_t)(q >> 8);
        } else {
            __half* Y = static_cast<__half*>(a.Y);
            Y[at] = __float2half_rn(v.x);
            Y[at + plane_stride] = __float2half_rn(v.y);
        }
    }
};

// Two frames per CTA (the largest FFT lengths): lanes 2i and 2i + 1 hold frames 0 and 1 of
// the same output, which are neighbours along K.  They swap halves with one shuffle so that
// the even lane writes both frames' real parts and the odd lane both imaginary parts, each
// as one word: half the scattered stores.  `at` is this lane's own element (the odd lane's
// frame-0 element is at - 1); paired = both frames in one slot starting at an even index
// (the same for both lanes); otherwise each live lane stores its own values.  Every lane
// must call this (the shuffle).
template <int OUTK>
__device__ __forceinline__ void store_frame_pair(const FArgs& a, long long at, long long ps, float2 y, bool odd,
                                                 bool paired, bool live)
{
    if (OUTK == FOUT_F32) {
        const float other = __shfl_xor_sync(0xffffffffu, odd ? y.x : y.y, 1);
        float* Y = static_cast<float*>(a.Y);
        if (paired) {
            if (odd) *reinterpret_cast<float2*>(Y + at - 1 + ps) = make_float2(other, y.y);
            else *reinterpret_cast<float2*>(Y + at) = make_float2(y.x, other);
        } else if (live) {
            Y[at] = y.x;
            Y[at + ps] = y.y;
        }
    } else if (OUTK == FOUT_F16) {
        const __half2 h2 = __floats2half2_rn(y.x, y.y);
        const uint32_t hu = *reinterpret_cast<const uint32_t*>(&h2);
        const uint32_t other = __shfl_xor_sync(0xffffffffu, hu, 1);
        __half* Y = static_cast<__half*>(a.Y);
        if (paired) {
            if (odd) *reinterpret_cast<uint32_t*>(Y + at - 1 + ps) = __byte_perm(other, hu, 0x7632);
            else *reinterpret_cast<uint32_t*>(Y + at) = __byte_perm(hu, other, 0x5410);
        } else if (live) {
            Y[at] = __low2half(h2);
            Y[at + ps] = __high2half(h2);
        }
    } else if (OUTK == FOUT_E4M3) {
        const uint32_t q = e4m3x2(y);   // (re, im) bytes
        const uint32_t other = __shfl_xor_sync(0xffffffffu, q, 1);
        uint8_t* Y = static_cast<uint8_t*>(a.Y);
        if (paired) {
            // even lane: (frame 0 re, frame 1 re); odd lane: (frame 0 im, frame 1 im)
            if (odd) *reinterpret_cast<uint16_t*>(Y + at - 1 + ps) = (uint16_t)__byte_perm(other, q, 0x0051);
            else *reinterpret_cast<uint16_t*>(Y + at) = (uint16_t)__byte_perm(q, other, 0x0040);
        } else if (live) {
            Y[at] = (uint8_t)(q & 0xFFu);
            Y[at + ps] = (uint8_t)(q >> 8);
        }
    } else {   // FP16 hi/lo pairs: lo values half a row further on
        const float xr = y.x, xi = y.y;
        const __half2 h2 = __floats2half2_rn(xr, xi);
        const float2 hf = __half22float2(h2);
        const __half2 l2 = __floats2half2_rn(xr - hf.x, xi - hf.y);
        const uint32_t hu = *reinterpret_cast<const uint32_t*>(&h2), lu = *reinterpret_cast<const uint32_t*>(&l2);
        // even lane sends (im hi, im lo), odd lane (re hi, re lo)
        const uint32_t send = odd ? __byte_perm(hu, lu, 0x5410) : __byte_perm(hu, lu, 0x7632);
        const uint32_t other = __shfl_xor_sync(0xffffffffu, send, 1);
        const long long lo = a.Kpad >> 1;
        __half* Y = static_cast<__half*>(a.Y);
        if (paired) {
            if (odd) {
                uint32_t* w = reinterpret_cast<uint32_t*>(Y + at - 1 + ps);
                w[0] = __byte_perm(other, hu, 0x7610);          // (frame 0 im hi, frame 1 im hi)
                w[lo >> 1] = __byte_perm(other, lu, 0x7632);    // (frame 0 im lo, frame 1 im lo)
            } else {
                uint32_t* w = reinterpret_cast<uint32_t*>(Y + at);
                w[0] = __byte_perm(hu, other, 0x5410);          // (frame 0 re hi, frame 1 re hi)
                w[lo >> 1] = __byte_perm(lu, other, 0x7610);    // (frame 0 re lo, frame 1 re lo)
            }
        } else if (live) {
            Y[at] = __low2half(h2);
            Y[at + ps] = __high2half(h2);
            Y[at + lo] = __low2half(l2);
            Y[at + ps + lo] = __high2half(l2);
        }
    }
}

// Two neighbouring frames of one output channel (frame 0 at element `at`, an even index;
// frame 1 at at + 1) written by one thread: each plane's two values as one word (FP32: 8
// bytes, FP16: 4 bytes; FP16 pairs: hi and lo words, lo half a row further on).
template <int OUTK>
__device__ __forceinline__ void store_two_frames(const FArgs& a, long long at, long long ps, float2 y0, float2 y1)
{
    if (OUTK == FOUT_F32) {
        float* Y = static_cast<float*>(a.Y);
        *reinterpret_cast<float2*>(Y + at) = make_float2(y0.x, y1.x);
        *reinterpret_cast<float2*>(Y + at + ps) = make_float2(y0.y, y1.y);
    } else if (OUTK == FOUT_F16) {
        __half* Y = static_cast<__half*>(a.Y);
        *reinterpret_cast<__half2*>(Y + at) = __floats2half2_rn(y0.x, y1.x);
        *reinterpret_cast<__half2*>(Y + at + ps) = __floats2half2_rn(y0.y, y1.y);
    } else if (OUTK == FOUT_E4M3) {
        uint8_t* Y = static_cast<uint8_t*>(a.Y);
        *reinterpret_cast<uint16_t*>(Y + at) = (uint16_t)e4m3x2(make_float2(y0.x, y1.x));
        *reinterpret_cast<uint16_t*>(Y + at + ps) = (uint16_t)e4m3x2(make_float2(y0.y, y1.y));
    } else {
        __half* Y = static_cast<__half*>(a.Y);
        const long long lo = a.Kpad >> 1;
        const __half2 hr = __floats2half2_rn(y0.x, y1.x), hi = __floats2half2_rn(y0.y, y1.y);
        const float2 fr = __half22float2(hr), fi = __half22float2(hi);
        *reinterpret_cast<__half2*>(Y + at) = hr;
        *reinterpret_cast<__half2*>(Y + at + ps) = hi;
        *reinterpret_cast<__half2*>(Y + at + lo) = __floats2half2_rn(y0.x - fr.x, y1.x - fr.y);
        *reinterpret_cast<__half2*>(Y + at + ps + lo) = __floats2half2_rn(y0.y - fi.x, y1.y - fi.y);
    }
}

// Delay phasor e^{2 pi i (phi0 + u d)} of ultrafine offset u (|u| < 4096), d = d_hi + d_lo
// with d_hi holding 12 significant bits so that u * d_hi is exact in FP32.
__device__ __forceinline__ float2 delay_phasor_u(float phi0, float d_hi, float d_lo, int u)
{
    float uf = (float)u;
    float x = uf * d_hi;
    x -= rintf(x);
    float y = phi0 + x + uf * d_lo;
    y -= rintf(y);
    float s, c;
    sincospif(2.0f * y, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ float2 delay_phasor(const FrameInfo& fi, int u)
{
    float uf = (float)u;
    float x = uf * fi.d_hi;       // exact: 12-bit by 12-bit significands
    x -= rintf(x);                // exact
    float y = fi.phi0 + x + uf * fi.d_lo;
    y -= rintf(y);
    float s, c;
    sincospif(2.0f * y, &s, &c);
    return make_float2(c, s);
}

// Twiddle e^{-2 pi i k / N}: straight from the full table when it sits in shared memory
// (N <= 1280); above that from two small shared tables, T1[k mod 128] T2[k / 128]
// (T1[a] = e^{-2 pi i a / N}, T2[b] = e^{-2 pi i 128 b / N}), one complex multiply
// instead of an uncached load from a table larger than what L1 has left.
template <int N>
__device__ __forceinline__ float2 twiddle(const float2* tw, int k)
{
    static_assert(N <= 1280 || N % 128 == 0, "two-level twiddles need N % 128 == 0");
    if (N <= 1280) return tw[k];
    return c_mul(tw[k & 127], tw[128 + (k >> 7)]);
}

// Shared-memory layout of the generic kernel's frames: element i of a frame sits at
// smem_pad(i) (one float2 of padding per 16, so the first pass's radix-R writes, R float2
// apart, fall in different banks), and frame f's row starts at f * ROW with ROW = 16 / FB
// (mod 16 float2): the FB frames x 16 / FB butterflies of a half-warp then cover all banks.
__host__ __device__ constexpr int smem_pad(int i) { return i + (i >> 4); }

template <int N>
__host__ __device__ constexpr int fstep_row()
{
    return (smem_pad(N - 1) + 1) +
           (((Sched<N>::fb >= 16 ? 1 : 16 / Sched<N>::fb) - (smem_pad(N - 1) + 1) % 16) % 16 + 16) % 16;
}

template <int N, int OUTK, int P>
struct Pass {
    static constexpr int R = Sched<N>::radix[P];
    static constexpr int NS = PassNs<N, P>::value;
    static constexpr int NB = N / R;
    static constexpr int FB = Sched<N>::fb;
    static constexpr int ROW = fstep_row<N>();     // padded float2 row per frame
    static constexpr int SROW = 2 * N + 4;         // padded int8 staging row (bytes)
    static constexpr bool FIRST = (P == 0);
    static constexpr bool LAST = (P == Sched<N>::passes - 1);

    __device__ __forceinline__ static void run(const FArgs& a, const FrameInfo* finfo, float2* buf0,
                                               float2* buf1, const int8_t* stage, int p, const float2* tw,
                                               const float* gain)
    {
        float2* in = (P % 2 == 0) ? buf1 : buf0;   // pass 0 reads the staging area in buf1
        float2* out = (P % 2 == 0) ? buf0 : buf1;
        // A thread keeps one frame (the CTA size is a multiple of FB) and walks its
        // butterflies j; padded offsets of the R inputs (outputs) are compile-time steps from
        // the first one whenever their stride is a multiple of 16 (or the first pass's
        // radix divides 16), so each access is one shared load or store.
        constexpr int NT = Sched<N>::nt;
        static_assert(NT % FB == 0, "a thread keeps one frame");
        const int f = threadIdx.x % FB;
        const float2* in_f = in + f * ROW;
        float2* out_f = out + f * ROW;
        const int8_t* st_f = stage + f * SROW;
        for (int j = threadIdx.x / FB; j < NB; j += NT / FB) {
            float2 v[R];
            const int pj = smem_pad(j);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (FIRST) {
                    const char2 s = *reinterpret_cast<const char2*>(st_f + 2 * j + 2 * r * NB);
                    v[r] = make_float2((float)s.x, (float)s.y);
                } else if (NB % 16 == 0) {
                    v[r] = in_f[pj + r * (NB + NB / 16)];
                } else {
                    v[r] = in_f[smem_pad(j + r * NB)];
                }
            }
            if (NS > 1) {
                const int tj = (j % NS) * (N / (NS * R));
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], twiddle<N>(tw, tj * r));
            }
            // last pass: the outputs' channel gains, loaded before the butterfly so that
            // their latency (global memory above N = 1280) overlaps its arithmetic
            float gk[LAST ? R : 1];
            if (LAST) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int k = j + r * NB;
                    gk[r] = gain[(k < N - N / 2) ? k + N / 2 : k - (N - N / 2)];
                }
            }
            Dft<R>::run(v);
            if (!LAST) {
                const int d = (j / NS) * NS * R + (j % NS);
                const int pd = smem_pad(d);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (NS % 16 == 0) out_f[pd + r * (NS + NS / 16)] = v[r];
                    else if (NS == 1 && 16 % R == 0) out_f[pd + r] = v[r];   // d = j R: no carry into d / 16
                    else out_f[smem_pad(d + r * NS)] = v[r];
                }
            } else {
                const FrameInfo fi = finfo[f];
                // two frames per CTA: neighbouring lanes pair their stores (every lane stays
                // in the loop for the shuffles; FB * NB is a multiple of the CTA size)
                constexpr bool PAIR = FB == 2;
                static_assert(!PAIR || !LAST || (FB * NB) % Sched<N>::nt == 0, "paired stores need uniform iterations");
                const bool live = fi.slot >= 0;
                const bool paired =
                    PAIR && finfo[0].slot >= 0 && finfo[1].slot == finfo[0].slot && (finfo[0].k & 1) == 0;
                if (!PAIR && !live) continue;
                // outputs k = j + r NB, r = 0..R-1; channel c = (k + N/2) mod N
                float2 E = make_float2(1.0f, 0.0f);
                if (fi.delay) E = delay_phasor(fi, j);   // u = j for r = 0 (j < NB <= N/2)
                const long long cs = 2LL * a.n * a.Kpad;                 // channel stride
                const long long ps = (long long)a.n * a.Kpad;            // plane stride
                const long long base = (fi.slot * N * 2LL * a.n + p) * a.Kpad + fi.k;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int k = j + r * NB;
                    const int c = (k < N - N / 2) ? k + N / 2 : k - (N - N / 2);
                    float2 y = v[r];
                    if (fi.delay) {
                        y = c_mul(y, (k < N - N / 2) ? E : c_mul(E, fi.wrap));
                        E = c_mul(E, fi.step);
                    }
                    const float gn = gk[r];
                    y.x *= gn;
                    y.y *= gn;
                    if (PAIR)
                        store_frame_pair<OUTK>(a, base + c * cs, ps, y, f == 1, paired, live);
                    else
                        Store<N, OUTK>::run(a, base + c * cs, ps, y, fi.slot, c, p);
                }
            }
        }
        if (!LAST) __syncthreads();
    }
};

template <int N, int OUTK, int P, bool DONE = (P >= Sched<N>::passes)>
struct PassChain {
    __device__ __forceinline__ static void run(const FArgs& a, const FrameInfo* fi, float2* b0, float2* b1,
                                               const int8_t* st, int p, const float2* tw, const float* gn)
    {
        Pass<N, OUTK, P>::run(a, fi, b0, b1, st, p, tw, gn);
        PassChain<N, OUTK, P + 1>::run(a, fi, b0, b1, st, p, tw, gn);
    }
};
template <int N, int OUTK, int P>
struct PassChain<N, OUTK, P, true> {
    __device__ __forceinline__ static void run(const FArgs&, const FrameInfo*, float2*, float2*, const int8_t*, int,
                                               const float2*, const float*)
    {
    }
};

// Twiddle and gain tables live in shared memory for N <= 1280; above that the twiddles
// are two small tables there (128 + N / 128 entries) and the gains stay in global memory
// (read once per output, coalesced).
template <int N>
__host__ __device__ constexpr bool tables_in_smem()
{
    return N <= 1280;
}

template <int N>
__host__ __device__ constexpr size_t fstep_smem()
{
    return 2 * sizeof(float2) * (size_t)Sched<N>::fb * fstep_row<N>() + sizeof(FrameInfo) * Sched<N>::fb +
           (tables_in_smem<N>() ? (sizeof(float2) + sizeof(float)) * N : sizeof(float2) * (128 + N / 128));
}

template <int N, int OUTK>
__global__ void __launch_bounds__(Sched<N>::nt) fstep_kernel(const FArgs a)
{
    constexpr int FB = Sched<N>::fb;
    constexpr int ROW = fstep_row<N>();
    constexpr int SROW = 2 * N + 4;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* buf0 = reinterpret_cast<float2*>(smem);
    float2* buf1 = buf0 + FB * ROW;
    FrameInfo* finfo = reinterpret_cast<FrameInfo*>(buf1 + FB * ROW);
    int8_t* stage = reinterpret_cast<int8_t*>(buf1);
    const float2* tw = a.tw;
    const float* gain = a.gain;
    if (tables_in_smem<N>()) {
        float2* tws = reinterpret_cast<float2*>(finfo + FB);
        float* gns = reinterpret_cast<float*>(tws + N);
        for (int i = threadIdx.x; i < N; i += Sched<N>::nt) {
            tws[i] = __ldg(&a.tw[i]);
            gns[i] = __ldg(&a.gain[i]);
        }
        tw = tws;
        gain = gns;
    } else {
        float2* tws = reinterpret_cast<float2*>(finfo + FB);
        for (int i = threadIdx.x; i < 128 + N / 128; i += Sched<N>::nt)
            tws[i] = __ldg(&a.tw[i < 128 ? i : 128 * (i - 128)]);
        tw = tws;
    }

    const int p = blockIdx.y;
    const long long f0 = (long long)blockIdx.x * FB;

    // Frame metadata: slot, index within the slot, FP64 delay polynomial (Sec. 4.3).
    if (threadIdx.x < FB) {
        const int f = threadIdx.x;
        FrameInfo fi;
        const long long fl = f0 + f;
        fi.slot = (fl < a.n_store) ? fl / a.Kc : -1;
        fi.k = (fl < a.n_store) ? fl % a.Kc : 0;
        fi.delay = 0;
        fi.phi0 = fi.d_hi = fi.d_lo = 0.0f;
        if ((a.delay != nullptr || a.delay_tab != nullptr) && fl < a.n_frames) {
            const double tau = frame_delay(a, p, a.m_begin + fl, N);
            const double ph = a.nu * tau;
            fi.phi0 = (float)(ph - floor(ph));
            const double d = tau * a.fs_over_n;
            const float dh = __uint_as_float(__float_as_uint((float)d) & 0xFFFFF000u);
            fi.d_hi = dh;
            fi.d_lo = (float)(d - (double)dh);
            fi.delay = 1;
            constexpr int NBL = N / Sched<N>::radix[Sched<N>::passes - 1];
            const double st = (double)NBL * d, wr = -(double)N * d;
            float sn, cs;
            sincospif(2.0f * (float)(st - rint(st)), &sn, &cs);
            fi.step = make_float2(cs, sn);
            sincospif(2.0f * (float)(wr - rint(wr)), &sn, &cs);
            fi.wrap = make_float2(cs, sn);
        }
        finfo[f] = fi;
    }

    // Stage the frames' int8 samples (2N bytes per frame, 16-byte loads).
    constexpr int CH = 2 * N / 16;   // 16-byte chunks per frame
    for (int i = threadIdx.x; i < FB * CH; i += Sched<N>::nt) {
        const int f = i / CH, ch = i % CH;
        const long long fl = f0 + f;
        int4 w = make_int4(0, 0, 0, 0);
        if (fl < a.n_frames && !frame_zeroed(a, p, (a.m_begin + fl) * (long long)N)) {
            const long long s = (a.m_begin + fl) * (long long)N;   // absolute first sample
            const long long blk = s / a.bs, off = s % a.bs;
            const int8_t* src = a.volt + ((blk * a.n + p) * (long long)a.bs + off) * 2;
            w = __ldg(reinterpret_cast<const int4*>(src) + ch);
        }
        int* dst = reinterpret_cast<int*>(stage + f * SROW + ch * 16);
        dst[0] = w.x;
        dst[1] = w.y;
        dst[2] = w.z;
        dst[3] = w.w;
    }
    __syncthreads();

    PassChain<N, OUTK, 0>::run(a, finfo, buf0, buf1, stage, p, tw, gain);
}


// -------------------------------------------------------------------------------------
// Two-pass variant for N = 32 T (T = 1, 2, 4, 8, 16): pass 1 reads each frame's int8
// samples straight from global memory, decimated by T (thread t of a frame takes samples
// t, t + T, ...), and does a 32-point DFT in registers; pass 2 does radix-T butterflies
// across those sub-transforms, with the twiddles W_N^{j r}, and its epilogue applies the
// delay phasor and channel gain and stores.  Each pass-2 thread takes consecutive
// butterflies j of one frame, so the phasor e^{2 pi i (phi0 + u d)} advances by fixed
// ratios (j -> j+1: e^{2 pi i d}; output r -> r+1: e^{2 pi i 32 d}; past N/2:
// e^{-2 pi i N d}) and only one sincospi is needed per thread and frame.
template <int N>
struct R32 {
    static constexpr int T = N / 32;
    static constexpr int FB = (N <= 256) ? 32 : 16;     // frames per CTA
    static constexpr int NT = 128;                      // threads per CTA
    static constexpr int JPT = 32 * FB / NT;            // pass-2 butterflies per thread
    // Shared-memory strides chosen for conflict-free access by both passes: pass 1 (lanes
    // = T sub-sequences x 32/T frames) writes row f, sub-row t; pass 2 (lanes = frames)
    // reads across sub-rows.  SR = 32 + 16/T (mod 16 == 16/T), ROW = 1 (mod 16).
    static constexpr int SR = (T == 1) ? 32 : 32 + 16 / T;
    static constexpr int ROW = (T == 1) ? 33 : T * SR + 1;
};

struct FrameR32 {
    long long slot, k;
    float phi0, d_hi, d_lo;
    int delay;
    float2 step1, step32, wrap;
};

template <int N>
__host__ __device__ constexpr size_t r32_smem()
{
    return sizeof(float2) * (size_t)R32<N>::FB * R32<N>::ROW + sizeof(FrameR32) * R32<N>::FB +
           (sizeof(float2) + sizeof(float)) * N;
}

template <int N, int OUTK>
__global__ void __launch_bounds__(128) fstep_r32_kernel(const FArgs a)
{
    using P = R32<N>;
    constexpr int T = P::T, FB = P::FB, NT = P::NT, ROW = P::ROW, SR = P::SR;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    FrameR32* finfo = reinterpret_cast<FrameR32*>(buf + FB * ROW);
    float2* tw = reinterpret_cast<float2*>(finfo + FB);
    float* gain = reinterpret_cast<float*>(tw + N);

    const int p = blockIdx.y;
    const long long f0 = (long long)blockIdx.x * FB;


    for (int i = threadIdx.x; i < N; i += NT) {
        tw[i] = __ldg(&a.tw[i]);
        gain[i] = __ldg(&a.gain[i]);
    }
    // Per-frame delay terms (Sec. 4.3): the FP64 polynomial once per frame (the FP64 pipe is
    // narrow on this GPU), the phasor ratios from its FP32 split d_hi + d_lo (u d_hi exact
    // for |u| < 4096: u = 1, 32, -N).
    if (threadIdx.x < FB) {
        const int f = threadIdx.x;
        const long long fl = f0 + f;
        const bool live = (a.delay != nullptr || a.delay_tab != nullptr) && fl < a.n_frames;
        FrameR32& fi = finfo[f];
        fi.slot = (fl < a.n_store) ? fl / a.Kc : -1;
        fi.k = (fl < a.n_store) ? fl % a.Kc : 0;
        fi.delay = live ? 1 : 0;
        fi.phi0 = fi.d_hi = fi.d_lo = 0.0f;
        fi.step1 = fi.step32 = fi.wrap = make_float2(1.0f, 0.0f);
        if (live) {
            const double tau = frame_delay(a, p, a.m_begin + fl, N);
            const double d = tau * a.fs_over_n;
            const double ph = a.nu * tau;
            fi.phi0 = (float)(ph - floor(ph));
            const float dh = __uint_as_float(__float_as_uint((float)d) & 0xFFFFF000u);
            fi.d_hi = dh;
            fi.d_lo = (float)(d - (double)dh);
            fi.step1 = delay_phasor_u(0.0f, fi.d_hi, fi.d_lo, 1);
            fi.step32 = delay_phasor_u(0.0f, fi.d_hi, fi.d_lo, 32);
            fi.wrap = delay_phasor_u(0.0f, fi.d_hi, fi.d_lo, -N);
        }
    }

    // Two frames per pass-2 thread for N <= 128: frames 2i and 2i + 1 (neighbours along K)
    // are stored as words.  Pass 1 writes frame f to row (f % 2) FB/2 + f / 2, so that the
    // two rows a thread reads (i and i + FB/2) and the rows of a half-warp stay in distinct
    // banks.
    constexpr bool PAIRS2 = T <= 4;
    static_assert(!PAIRS2 || FB % 2 == 0, "frame pairs");

    // ---- pass 1: 32-point DFTs of the T decimated sub-sequences of each frame
    for (int idx = threadIdx.x; idx < FB * T; idx += NT) {
        const int t = idx % T, row = idx / T;
        const int f = PAIRS2 ? 2 * (row % (FB / 2)) + row / (FB / 2) : row;
        const long long fl = f0 + f;
        float2 v[32];
        if (fl < a.n_frames && !frame_zeroed(a, p, (a.m_begin + fl) * (long long)N)) {
            const long long s0 = (a.m_begin + fl) * (long long)N;   // first sample of the frame
            const long long blk = s0 / a.bs, off = s0 % a.bs;
            const char2* src = reinterpret_cast<const char2*>(a.volt + ((blk * a.n + p) * (long long)a.bs + off) * 2);
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                const char2 x = __ldg(src + t + T * m);
                v[m] = make_float2((float)x.x, (float)x.y);
            }
        } else {
#pragma unroll
            for (int m = 0; m < 32; ++m) v[m] = make_float2(0.0f, 0.0f);
        }
        Dft<32>::run(v);
#pragma unroll
        for (int r = 0; r < 32; ++r) buf[row * ROW + SR * t + r] = v[r];
    }
    __syncthreads();

    if constexpr (PAIRS2) {
        // ---- pass 2, frame pairs: radix-T butterflies j of frames 2i and 2i + 1 (rows i and
        // i + FB/2), sharing the twiddle and gain loads; phasor per frame; word stores
        constexpr int PP = FB / 2;
        constexpr int JP = 32 * PP / NT;   // butterflies per thread
        static_assert(JP * NT == 32 * PP, "whole butterflies per thread");
        const int fp = threadIdx.x % PP;
        const int jb = (threadIdx.x / PP) * JP;
        const FrameR32 fi0 = finfo[2 * fp], fi1 = finfo[2 * fp + 1];
        const bool live0 = fi0.slot >= 0, live1 = fi1.slot >= 0;
        if (!live0 && !live1) return;
        // both frames in one slot, frame 0 at an even index: one word per value
        const bool paired = live0 && live1 && fi1.slot == fi0.slot && (fi0.k & 1) == 0;
        const long long cs = 2LL * a.n * a.Kpad;
        const long long ps = (long long)a.n * a.Kpad;
        const long long base0 = (fi0.slot * N * 2LL * a.n + p) * a.Kpad + fi0.k;
        const long long d1 = (fi1.slot * N * 2LL * a.n + p) * a.Kpad + fi1.k - base0;   // frame 1 - frame 0
        long long at[T];
#pragma unroll
        for (int r = 0; r < T; ++r) {
            const int k = jb + 32 * r;
            const bool low = (T >= 2) ? (r < T / 2) : (k < N - N / 2);
            at[r] = base0 + (long long)(low ? k + N / 2 : k - (N - N / 2)) * cs;
        }
        float2 Ej0 = make_float2(1.0f, 0.0f), Ej1 = Ej0;
        if (fi0.delay) Ej0 = delay_phasor_u(fi0.phi0, fi0.d_hi, fi0.d_lo, jb);
        if (fi1.delay) Ej1 = delay_phasor_u(fi1.phi0, fi1.d_hi, fi1.d_lo, jb);
        for (int jj = 0; jj < JP; ++jj) {
            const int j = jb + jj;
            float2 v0[T], v1[T];
#pragma unroll
            for (int r = 0; r < T; ++r) {
                v0[r] = buf[fp * ROW + SR * r + j];
                v1[r] = buf[(fp + PP) * ROW + SR * r + j];
                if (r > 0) {
                    const float2 w = tw[j * r];
                    v0[r] = c_mul(v0[r], w);
                    v1[r] = c_mul(v1[r], w);
                }
            }
            DftIf<T>::run(v0);
            DftIf<T>::run(v1);
            float2 E0 = Ej0, E1 = Ej1;
#pragma unroll
            for (int r = 0; r < T; ++r) {
                const int k = j + 32 * r;
                const bool low = (T >= 2) ? (r < T / 2) : (k < N - N / 2);
                const int c = low ? k + N / 2 : k - (N - N / 2);
                float2 y0 = v0[r], y1 = v1[r];
                if (fi0.delay) {
                    if (T >= 2) {
                        if (r == T / 2) E0 = c_mul(E0, fi0.wrap);
                        y0 = c_mul(y0, E0);
                    } else {
                        y0 = c_mul(y0, low ? E0 : c_mul(E0, fi0.wrap));
                    }
                    E0 = c_mul(E0, fi0.step32);
                }
                if (fi1.delay) {
                    if (T >= 2) {
                        if (r == T / 2) E1 = c_mul(E1, fi1.wrap);
                        y1 = c_mul(y1, E1);
                    } else {
                        y1 = c_mul(y1, low ? E1 : c_mul(E1, fi1.wrap));
                    }
                    E1 = c_mul(E1, fi1.step32);
                }
                const float gn = gain[c];
                y0 = make_float2(y0.x * gn, y0.y * gn);
                y1 = make_float2(y1.x * gn, y1.y * gn);
                if (paired) {
                    store_two_frames<OUTK>(a, at[r], ps, y0, y1);
                } else {
                    if (live0) Store<N, OUTK>::run(a, at[r], ps, y0, fi0.slot, c, p);
                    if (live1) Store<N, OUTK>::run(a, at[r] + d1, ps, y1, fi1.slot, c, p);
                }
                at[r] += cs;
            }
            if (fi0.delay) Ej0 = c_mul(Ej0, fi0.step1);
            if (fi1.delay) Ej1 = c_mul(Ej1, fi1.step1);
        }
        return;
    }

    // ---- pass 2: radix-T butterflies j = 0..31 of each frame, then phasor, gain, store
    const int f = threadIdx.x % FB;
    const int jb = (threadIdx.x / FB) * P::JPT;
    const FrameR32 fi = finfo[f];
    if (fi.slot < 0) return;
    const long long cs = 2LL * a.n * a.Kpad;
    const long long ps = (long long)a.n * a.Kpad;
    const long long base = (fi.slot * N * 2LL * a.n + p) * a.Kpad + fi.k;
    // output r of butterfly j goes to channel c_r(j) = c_r(jb) + (j - jb): one element offset
    // per r, advanced by a channel stride per butterfly
    long long at[T];
#pragma unroll
    for (int r = 0; r < T; ++r) {
        const int k = jb + 32 * r;
        const bool low = (T >= 2) ? (r < T / 2) : (k < N - N / 2);
        at[r] = base + (long long)(low ? k + N / 2 : k - (N - N / 2)) * cs;
    }
    float2 Ej = make_float2(1.0f, 0.0f);
    if (fi.delay) Ej = delay_phasor_u(fi.phi0, fi.d_hi, fi.d_lo, jb);
#pragma unroll 2
    for (int jj = 0; jj < P::JPT; ++jj) {
        const int j = jb + jj;
        float2 v[T];
#pragma unroll
        for (int r = 0; r < T; ++r) {
            v[r] = buf[f * ROW + SR * r + j];
            if (r > 0) v[r] = c_mul(v[r], tw[j * r]);
        }
        DftIf<T>::run(v);
        float2 E = Ej;
#pragma unroll
        for (int r = 0; r < T; ++r) {
            const int k = j + 32 * r;   // natural-order bin
            // j < 32: for T >= 2 the bins past N/2 are exactly the outputs r >= T/2
            const bool low = (T >= 2) ? (r < T / 2) : (k < N - N / 2);
            const int c = low ? k + N / 2 : k - (N - N / 2);
            float2 y = v[r];
            if (fi.delay) {
                if (T >= 2) {
                    if (r == T / 2) E = c_mul(E, fi.wrap);   // u = k - N from here on
                    y = c_mul(y, E);
                } else {
                    y = c_mul(y, low ? E : c_mul(E, fi.wrap));
                }
                E = c_mul(E, fi.step32);
            }
            const float gn = gain[c];
            y = make_float2(y.x * gn, y.y * gn);
            Store<N, OUTK>::run(a, at[r], ps, y, fi.slot, c, p);
            at[r] += cs;
        }
        if (fi.delay) Ej = c_mul(Ej, fi.step1);
    }
}

// N = 1: no FFT.  One thread per (path, 8 samples).  The common case (no delay, no flags,
// FP32/FP16 output, the 8 samples in one data block and one operand slot) is one 16-byte
// load and 16-byte stores per plane with the index arithmetic done once; everything else
// (phasor e^{2 pi i nu tau}, flags, FP8 maxima, group edges) takes the per-sample path.
// Operand element of frame k of a slot for path p (real plane; the imaginary plane is
// *ps further on): rows of Kpad frames, or in the integer mode rows of one K tile
// (Y[slot][K tile][plane][p][ktile]).
__device__ __forceinline__ long long unpack_at(const FArgs& a, long long slot, long long k, int p, long long* ps)
{
    if (a.ktile > 0) {   // the integer mode's tile is kIntKTile (a power of two: shifts, not divisions)
        constexpr long long KT = kIntKTile;
        static_assert((KT & (KT - 1)) == 0, "K tile must be a power of two");
        *ps = (long long)a.n * KT;
        return ((slot * (a.Kpad / KT) + k / KT) * 2LL * a.n + p) * KT + (k & (KT - 1));
    }
    *ps = (long long)a.n * a.Kpad;
    return (slot * 2LL * a.n + p) * a.Kpad + k;
}

template <int OUTK>
__global__ void __launch_bounds__(256) unpack_kernel(const FArgs a)
{
    const int p = blockIdx.y;
    const long long i8 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long f_first = i8 * 8;
    if (f_first >= a.n_store) return;
    if ((OUTK == FOUT_F32 || OUTK == FOUT_F16) && a.delay == nullptr && a.delay_tab == nullptr &&
        a.flags == nullptr && f_first + 8 <= a.n_frames) {
        const long long s0 = a.m_begin + f_first;
        const long long blk = s0 / a.bs, off = s0 % a.bs;
        const long long slot = f_first / a.Kc, k = f_first % a.Kc;
        const int8_t* src = a.volt + ((blk * a.n + p) * (long long)a.bs + off) * 2;
        if (off + 8 <= a.bs && k + 8 <= a.Kc && (k & 7) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            const int4 raw = __ldg(reinterpret_cast<const int4*>(src));
            const char2* x = reinterpret_cast<const char2*>(&raw);
            const float g = __ldg(&a.gain[0]);
            long long ps;
            const long long at = unpack_at(a, slot, k, p, &ps);   // 8 frames in one row (tiles are multiples of 8)
            if (OUTK == FOUT_F16) {
                __half2 re[4], im[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    re[e] = __floats2half2_rn((float)x[2 * e].x * g, (float)x[2 * e + 1].x * g);
                    im[e] = __floats2half2_rn((float)x[2 * e].y * g, (float)x[2 * e + 1].y * g);
                }
                __half* Y = static_cast<__half*>(a.Y);
                *reinterpret_cast<uint4*>(Y + at) = *reinterpret_cast<const uint4*>(re);
                *reinterpret_cast<uint4*>(Y + at + ps) = *reinterpret_cast<const uint4*>(im);
            } else {
                float re[8], im[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    re[e] = (float)x[e].x * g;
                    im[e] = (float)x[e].y * g;
                }
                float* Y = static_cast<float*>(a.Y);
                *reinterpret_cast<float4*>(Y + at) = make_float4(re[0], re[1], re[2], re[3]);
                *reinterpret_cast<float4*>(Y + at + 4) = make_float4(re[4], re[5], re[6], re[7]);
                *reinterpret_cast<float4*>(Y + at + ps) = make_float4(im[0], im[1], im[2], im[3]);
                *reinterpret_cast<float4*>(Y + at + ps + 4) = make_float4(im[4], im[5], im[6], im[7]);
            }
            return;
        }
    }
    for (int e = 0; e < 8; ++e) {
        const long long fl = f_first + e;
        if (fl >= a.n_store) break;
        const long long s = a.m_begin + fl;
        float2 v = make_float2(0.0f, 0.0f);
        if (fl < a.n_frames && !frame_zeroed(a, p, s)) {
            const long long blk = s / a.bs, off = s % a.bs;
            const char2 x = *reinterpret_cast<const char2*>(a.volt + ((blk * a.n + p) * (long long)a.bs + off) * 2);
            v = make_float2((float)x.x, (float)x.y);
        }
        if ((a.delay != nullptr || a.delay_tab != nullptr) && fl < a.n_frames) {
            const double tau = frame_delay(a, p, s, 1);   // N = 1: frame = sample
            const double ph = a.nu * tau;
            float sn, cs;
            sincospif(2.0f * (float)(ph - floor(ph)), &sn, &cs);
            v = c_mul(v, make_float2(cs, sn));
        }
        const float gn = __ldg(&a.gain[0]);
        long long ps;
        const long long at = unpack_at(a, fl / a.Kc, fl % a.Kc, p, &ps);
        Store<1, OUTK>::run(a, at, ps, make_float2(v.x * gn, v.y * gn), fl / a.Kc, 0, p);
    }
}

template <int N, int OUTK>
cudaError_t launch_n(const FArgs& a, cudaStream_t s)
{
    constexpr size_t smem = fstep_smem<N>();
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fstep_kernel<N, OUTK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((unsigned)((a.n_store + Sched<N>::fb - 1) / Sched<N>::fb), (unsigned)a.n);
    fstep_kernel<N, OUTK><<<grid, Sched<N>::nt, smem, s>>>(a);
    return cudaGetLastError();
}

template <int N, int OUTK>
cudaError_t launch_r32(const FArgs& a, cudaStream_t s)
{
    constexpr size_t smem = r32_smem<N>();
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(fstep_r32_kernel<N, OUTK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((unsigned)((a.n_store + R32<N>::FB - 1) / R32<N>::FB), (unsigned)a.n);
    fstep_r32_kernel<N, OUTK><<<grid, R32<N>::NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int OUTK>
cudaError_t launch_kind(int N, const FArgs& a, cudaStream_t s, int variant)
{
    if (variant == 1) {
        switch (N) {
            case 32: return launch_n<32, OUTK>(a, s);
            case 64: return launch_n<64, OUTK>(a, s);
            case 128: return launch_n<128, OUTK>(a, s);
            case 256: return launch_n<256, OUTK>(a, s);
            case 512: return launch_n<512, OUTK>(a, s);
            default: break;
        }
    }
    switch (N) {
        case 1: {
            dim3 grid((unsigned)((a.n_store + 2047) / 2048), (unsigned)a.n);
            unpack_kernel<OUTK><<<grid, 256, 0, s>>>(a);
            return cudaGetLastError();
        }
        case 16: return launch_n<16, OUTK>(a, s);
        case 32: return launch_r32<32, OUTK>(a, s);
        case 64: return launch_r32<64, OUTK>(a, s);
        case 128: return launch_r32<128, OUTK>(a, s);
        case 256: return launch_r32<256, OUTK>(a, s);
        case 512: return launch_r32<512, OUTK>(a, s);
        case 640: return launch_n<640, OUTK>(a, s);
        case 1280: return launch_n<1280, OUTK>(a, s);
        case 3200: return launch_n<3200, OUTK>(a, s);
        case 6400: return launch_n<6400, OUTK>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

// FP8: e4m3 operands from the FP16 ones, q = h * 448 / amax[slot][group(c)][p] with
// saturation (|q| <= 448 by construction).  One CTA per operand row (slot, c, plane, p),
// 8 consecutive frames per thread and step.
__global__ void __launch_bounds__(256) quantise_e4m3_kernel(const __half* __restrict__ Y16,
                                                            __nv_fp8_storage_t* __restrict__ Y8,
                                                            const float* __restrict__ amax,
                                                            const int* __restrict__ chan_group, int n_groups, int N,
                                                            int n, long long Kpad, long long rows)
{
    // One warp per operand row (grid-stride over rows); a lane converts 16 FP16 values
    // (two 16-byte loads) into one 16-byte store of e4m3 codes per step.
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
        const int p = (int)(row % n);
        const long long sc = row / (2LL * n);       // slot * N + c
        const int c = (int)(sc % N);
        const long long slot = sc / N;
        const int g = __ldg(&chan_group[c]);
        if (g < 0) continue;                        // zero-weight channel: never read
        const float am = __ldg(&amax[(slot * n_groups + g) * (long long)n + p]);
        const float inv = am > 0.0f ? 448.0f / am : 0.0f;
        const uint4* src = reinterpret_cast<const uint4*>(Y16 + row * Kpad);
        uint4* dst = reinterpret_cast<uint4*>(Y8 + row * Kpad);
        for (long long k16 = lane; k16 < Kpad / 16; k16 += 32) {
            const uint4 h[2] = {__ldg(src + 2 * k16), __ldg(src + 2 * k16 + 1)};
            const __half2* hp = reinterpret_cast<const __half2*>(h);
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float2 v0 = __half22float2(hp[2 * e]), v1 = __half22float2(hp[2 * e + 1]);
                v0.x *= inv;
                v0.y *= inv;
                v1.x *= inv;
                v1.y *= inv;
                const uint32_t q0 = __nv_cvt_float2_to_fp8x2(v0, __NV_SATFINITE, __NV_E4M3);
                const uint32_t q1 = __nv_cvt_float2_to_fp8x2(v1, __NV_SATFINITE, __NV_E4M3);
                w[e] = q0 | (q1 << 16);
            }
            dst[k16] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Zero each integration's visibility set and write its weights table (1.0, Sec. 2.7).
__global__ void init_output_kernel(char* out, long long n_ints, long long vis_words, long long wt_words)
{
    const long long per = vis_words + wt_words;
    const long long total = n_ints * per;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i % per;
        reinterpret_cast<float*>(out)[i] = (r < vis_words) ? 0.0f : 1.0f;
    }
}

// Occupancy weight of (integration w, baseline b, pol): the fraction of the integration's K
// frames whose data block is unflagged in both paths (Sec. 4.1).  One thread per
// (w, tile i, tile j >= i, pol); frames never straddle a block (N divides the block).
__global__ void weights_kernel(char* out, long long n_ints, long long int_stride, long long vis_set_bytes, int T,
                               int M, long long K, int N, int bs, int n, const uint8_t* __restrict__ flags,
                               int normalise)
{
    const long long total = n_ints * (long long)T * T * 4;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int pol = (int)(idx % 4);
        const long long r = idx / 4;
        const int j = (int)(r % T), i = (int)((r / T) % T);
        const long long w = r / ((long long)T * T);
        if (j < i) continue;
        const int p = 2 * i + (pol >> 1), q = 2 * j + (pol & 1);
        const long long s_begin = w * K * N, s_end = (w + 1) * K * N;
        long long good = 0;
        for (long long blk = s_begin / bs; blk * bs < s_end; ++blk) {
            const long long lo = max(blk * bs, s_begin), hi = min((blk + 1) * bs, s_end);
            if (!flags[blk * n + p] && !flags[blk * n + q]) good += (hi - lo) / N;
        }
        const float wt = (float)((double)good / (double)K);
        const long long b = (long long)i * (2 * T - i + 1) / 2 + (j - i);
        char* set = out + w * int_stride;
        reinterpret_cast<float*>(set + vis_set_bytes)[b * 4 + pol] = wt;
        if (normalise) {
            const float inv = wt > 0.0f ? 1.0f / wt : 0.0f;
            float2* v = reinterpret_cast<float2*>(set);
            for (int ch = 0; ch < M; ++ch) {
                float2 x = v[(b * M + ch) * 4 + pol];
                v[(b * M + ch) * 4 + pol] = make_float2(x.x * inv, x.y * inv);
            }
        }
    }
}

}  // namespace

bool fft_len_supported(int N)
{
    switch (N) {
        case 1: case 16: case 32: case 64: case 128: case 256: case 512: case 640: case 1280: case 3200: case 6400:
            return true;
        default:
            return false;
    }
}

cudaError_t launch_fstep(int N, int out_kind, const FArgs& a_in, cudaStream_t s, int variant)
{
    FArgs a = a_in;
    a.frame_dt = (double)N / a.fs;
    a.fs_over_n = a.fs / (double)N;
    if (variant == 4) {
        if (fstep_fd_supported(N, out_kind) && a.ktile == 0) return launch_fstep_fd(N, out_kind, a, s);
        variant = 0;
    }
    if (variant == 3) {
        if ((out_kind == FOUT_F16 || out_kind == FOUT_E4M3) && fstep_f128_supported(N) && a.Yt)
            return launch_fstep_f128(N, out_kind, a, s);
        variant = 2;
    }
    if (variant == 2) {
        if (out_kind == FOUT_F16 && fstep_tc_supported(N)) return launch_fstep_tc(N, a, s);
        if (fstep_dft_supported(N, out_kind) && a.ktile == 0) return launch_fstep_dft(N, out_kind, a, s);
        variant = 0;
    }
    switch (out_kind) {
        case FOUT_F32: return launch_kind<FOUT_F32>(N, a, s, variant);
        case FOUT_F16: return launch_kind<FOUT_F16>(N, a, s, variant);
        case FOUT_F16X3: return launch_kind<FOUT_F16X3>(N, a, s, variant);
        case FOUT_E4M3: return launch_kind<FOUT_E4M3>(N, a, s, variant);
        default: return cudaErrorInvalidValue;
    }
}

// FP8 form, after an FP16 F-step: per (slot, channel group g, path p) one warp reads the
// FP16 operand rows of the group's channels (both planes, 16-byte loads) and stores the
// largest magnitude over the slot's kvalid frames in amax[slot][g][p] (the e4m3 scale is
// amax / 448): the same maxima as gathering them inside the F-step.
__global__ void __launch_bounds__(256) amax_e4m3_kernel(const __half* __restrict__ Y16, float* __restrict__ amax,
                                                        const int* __restrict__ chan_group,
                                                        const Group* __restrict__ groups, int n_groups, int N, int n,
                                                        long long Kpad, long long kvalid, long long slots)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long tasks = slots * n_groups * (long long)n;
    for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < tasks; t += warps) {
        const int p = (int)(t % n);
        const int g = (int)((t / n) % n_groups);
        const long long slot = t / ((long long)n * n_groups);
        const Group gr = groups[g];
        __half2 m2 = __float2half2_rn(0.0f);
        for (int c = gr.c0; c < gr.c1; ++c) {
            if (__ldg(&chan_group[c]) != g) continue;
            for (int plane = 0; plane < 2; ++plane) {
                const uint4* row = reinterpret_cast<const uint4*>(Y16 + (((slot * N + c) * 2 + plane) * n + p) * Kpad);
                for (long long k8 = lane; 8 * k8 < kvalid; k8 += 32) {
                    const uint4 h = __ldg(row + k8);
                    const __half2* hp = reinterpret_cast<const __half2*>(&h);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        __half2 v = __habs2(hp[e]);
                        // frames past kvalid were not written by the F-step: leave them out
                        const long long f0 = 8 * k8 + 2 * e;
                        if (f0 + 1 >= kvalid) v = (f0 >= kvalid) ? __float2half2_rn(0.0f)
                                                                : __halves2half2(__low2half(v), __float2half(0.0f));
                        m2 = __hmax2(m2, v);
                    }
                }
            }
        }
        float m = fmaxf(__low2float(m2), __high2float(m2));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) amax[(slot * n_groups + g) * (long long)n + p] = m;
    }
}

__global__ void __launch_bounds__(256) fill_amax_kernel(float* __restrict__ amax, const float* __restrict__ amax_static,
                                                        int n_groups, int n, long long total)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        amax[i] = __ldg(&amax_static[(i / n) % n_groups]);
}

cudaError_t launch_fill_amax(float* amax, const float* amax_static, int n_groups, int n, long long slots,
                             cudaStream_t s)
{
    const long long total = slots * n_groups * (long long)n;
    if (total <= 0) return cudaSuccess;
    fill_amax_kernel<<<(unsigned)std::min<long long>((total + 255) / 256, 148LL * 8), 256, 0, s>>>(amax, amax_static,
                                                                                                  n_groups, n, total);
    return cudaGetLastError();
}

cudaError_t launch_amax_e4m3(const __half* Y16, float* amax, const int* chan_group, const Group* groups, int n_groups,
                             long long slots, int N, int n, long long Kpad, long long kvalid, cudaStream_t s)
{
    const long long tasks = slots * n_groups * (long long)n;
    if (tasks <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((tasks + 7) / 8, 148LL * 16);   // 8 tasks (warps) per block
    amax_e4m3_kernel<<<(unsigned)blocks, 256, 0, s>>>(Y16, amax, chan_group, groups, n_groups, N, n, Kpad, kvalid,
                                                      slots);
    return cudaGetLastError();
}

cudaError_t launch_quantise_e4m3(const __half* Y16, __nv_fp8_storage_t* Y8, const float* amax,
                                 const int* chan_group, int n_groups, long long slots, int N, int n, long long Kpad,
                                 cudaStream_t s)
{
    const long long rows = slots * (long long)N * 2 * n;
    if (rows <= 0) return cudaSuccess;
    if (rows > 0x7fffffffLL) return cudaErrorInvalidValue;
    const long long blocks = std::min<long long>((rows + 7) / 8, 148LL * 16);   // 8 rows (warps) per block
    quantise_e4m3_kernel<<<(unsigned)blocks, 256, 0, s>>>(Y16, Y8, amax, chan_group, n_groups, N, n, Kpad, rows);
    return cudaGetLastError();
}

cudaError_t launch_weights(char* out, long long n_ints, long long int_stride, long long vis_set_bytes, int T, int M,
                           long long K, int N, int bs, int n, const uint8_t* flags, int normalise, cudaStream_t s)
{
    weights_kernel<<<4 * 148, 256, 0, s>>>(out, n_ints, int_stride, vis_set_bytes, T, M, K, N, bs, n, flags,
                                           normalise);
    return cudaGetLastError();
}

cudaError_t launch_init_output(char* out, long long n_ints, long long vis_set_bytes, long long weights_bytes,
                               cudaStream_t s)
{
    init_output_kernel<<<4 * 148, 256, 0, s>>>(out, n_ints, vis_set_bytes / 4, weights_bytes / 4);
    return cudaGetLastError();
}

}  // namespace mwax
