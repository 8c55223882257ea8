// X-step, FP32 CUDA-core form (the paper's xGPU-style single-precision cross-multiply,
// Sec. 2.5.2), with time integration (Sec. 2.5.2), channel averaging (Sec. 2.6) and
// MWAX_ORDER output (Sec. 2.7) fused into the epilogue.
//
// CTA = one 64 x 64 tile of signal-path pairs (p rows, q columns; tiles on or above the
// block diagonal only) x one run of output channels x one integration slot.  For every
// group of ultrafine channels feeding the run, the CTA forms
//     C[p,q] = sum_{c in group} sum_k Y_p[k,c] conj(Y_q[k,c])
// (the F-step has already weighted channel c by sqrt(w_c)) with a 4 x 4 complex register
// tile per thread (two-level FP32 accumulation: a fresh partial per 32-frame chunk, added
// into the running total), and adds coef * C into every output channel the group feeds.
// Each output element is owned by exactly one CTA, so the read-modify-write needs no
// atomics.
#include "mwax_internal.cuh"

namespace mwax {
namespace {

constexpr int TP = 64;    // paths per tile side
constexpr int KT = 32;    // frames per chunk
constexpr int LDA = 68;   // padded smem row (floats): conflict-free transposed stores

struct SimtSmem {
    float a[2][2][KT][LDA];   // [buffer][plane][k][p]
    float b[2][2][KT][LDA];
};

__device__ __forceinline__ long long baseline_of(int i, int j, int T)
{
    return (long long)i * (2 * T - i + 1) / 2 + (j - i);
}

// Load one 4x4 (rows x frames) block of a plane tile into registers.
__device__ __forceinline__ void load_block(const float* __restrict__ base, long long Kpad, int rows_valid, int r0,
                                           long long k0, long long klen, float4 (&v)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + i;
        if (r < rows_valid && k0 + 3 < klen) {
            v[i] = __ldg(reinterpret_cast<const float4*>(base + (long long)r * Kpad + k0));
        } else {
            float t[4] = {0.f, 0.f, 0.f, 0.f};
            if (r < rows_valid)
                for (int e = 0; e < 4; ++e)
                    if (k0 + e < klen) t[e] = base[(long long)r * Kpad + k0 + e];
            v[i] = make_float4(t[0], t[1], t[2], t[3]);
        }
    }
}

__device__ __forceinline__ void store_block(float (*dst)[LDA], int r0, int k0, const float4 (&v)[4])
{
    *reinterpret_cast<float4*>(&dst[k0 + 0][r0]) = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
    *reinterpret_cast<float4*>(&dst[k0 + 1][r0]) = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
    *reinterpret_cast<float4*>(&dst[k0 + 2][r0]) = make_float4(v[0].z, v[1].z, v[2].z, v[3].z);
    *reinterpret_cast<float4*>(&dst[k0 + 3][r0]) = make_float4(v[0].w, v[1].w, v[2].w, v[3].w);
}

__global__ void __launch_bounds__(256, 2) xstep_simt_kernel(const XArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SimtSmem& sm = *reinterpret_cast<SimtSmem*>(smem_raw);

    const int4 tile = a.tiles[blockIdx.x];
    const RunInfo run = a.runs[blockIdx.y];
    const long long slot = blockIdx.z;
    const int p0 = tile.x, q0 = tile.y;
    const bool diag = (p0 == q0);
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;

    // Loader role: one 4x4 block of the A tile (plane = tid / 128) and, unless the tile
    // is on the diagonal, the same block of the B tile.
    const int lplane = tid / 128, lblk = tid % 128;
    const int lrow = (lblk / 8) * 4, lk = (lblk % 8) * 4;
    const int rows_a = min(TP, a.n - p0), rows_b = min(TP, a.n - q0);
    const float* Yf = static_cast<const float*>(a.Y);

    for (int g = run.g0; g < run.g1; ++g) {
        const Group gr = a.groups[g];
        const bool use_a = gr.ja >= run.j0 && gr.ja < run.j1;
        const bool use_b = gr.jb >= run.j0 && gr.jb < run.j1;
        if (!use_a && !use_b) continue;

        float tre[4][4], tim[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) tre[i][j] = tim[i][j] = 0.f;

        for (int c = gr.c0; c < gr.c1; ++c) {
            if (__ldg(&a.gain[c]) == 0.0f) continue;
            const float* plane_base = Yf + ((slot * a.N + c) * 2) * (long long)a.n * a.Kpad;
            const float* abase = plane_base + ((long long)lplane * a.n + p0) * a.Kpad;
            const float* bbase = plane_base + ((long long)lplane * a.n + q0) * a.Kpad;

            const long long nchunks = (a.klen + KT - 1) / KT;
            float4 ra[4], rb[4];
            load_block(abase, a.Kpad, rows_a, lrow, lk, a.klen, ra);
            if (!diag) load_block(bbase, a.Kpad, rows_b, lrow, lk, a.klen, rb);
            __syncthreads();   // previous channel's readers are done with both buffers
            store_block(sm.a[0][lplane], lrow, lk, ra);
            if (!diag) store_block(sm.b[0][lplane], lrow, lk, rb);
            __syncthreads();

            for (long long ch = 0; ch < nchunks; ++ch) {
                const int cur = (int)(ch & 1);
                const bool more = ch + 1 < nchunks;
                if (more) {
                    const long long k0 = (ch + 1) * KT + lk;
                    load_block(abase, a.Kpad, rows_a, lrow, k0, a.klen, ra);
                    if (!diag) load_block(bbase, a.Kpad, rows_b, lrow, k0, a.klen, rb);
                }
                const float(*Ar)[LDA] = sm.a[cur][0];
                const float(*Ai)[LDA] = sm.a[cur][1];
                const float(*Br)[LDA] = diag ? sm.a[cur][0] : sm.b[cur][0];
                const float(*Bi)[LDA] = diag ? sm.a[cur][1] : sm.b[cur][1];
                float pre[4][4], pim[4][4];
    #pragma unroll
                for (int i = 0; i < 4; ++i)
    #pragma unroll
                    for (int j = 0; j < 4; ++j) pre[i][j] = pim[i][j] = 0.f;
    #pragma unroll 8
                for (int k = 0; k < KT; ++k) {
                    const float4 ar = *reinterpret_cast<const float4*>(&Ar[k][ty * 4]);
                    const float4 ai = *reinterpret_cast<const float4*>(&Ai[k][ty * 4]);
                    const float4 br = *reinterpret_cast<const float4*>(&Br[k][tx * 4]);
                    const float4 bi = *reinterpret_cast<const float4*>(&Bi[k][tx * 4]);
                    const float xr[4] = {ar.x, ar.y, ar.z, ar.w}, xi[4] = {ai.x, ai.y, ai.z, ai.w};
                    const float yr[4] = {br.x, br.y, br.z, br.w}, yi[4] = {bi.x, bi.y, bi.z, bi.w};
    #pragma unroll
                    for (int i = 0; i < 4; ++i)
    #pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            // (xr + i xi)(yr - i yi)
                            pre[i][j] = fmaf(xr[i], yr[j], pre[i][j]);
                            pre[i][j] = fmaf(xi[i], yi[j], pre[i][j]);
                            pim[i][j] = fmaf(xi[i], yr[j], pim[i][j]);
                            pim[i][j] = fmaf(-xr[i], yi[j], pim[i][j]);
                        }
                }
    #pragma unroll
                for (int i = 0; i < 4; ++i)
    #pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        tre[i][j] += pre[i][j];
                        tim[i][j] += pim[i][j];
                    }
                if (more) {
                    store_block(sm.a[cur ^ 1][lplane], lrow, lk, ra);
                    if (!diag) store_block(sm.b[cur ^ 1][lplane], lrow, lk, rb);
                }
                __syncthreads();
            }
        }   // channels of the group

        // Epilogue: add coef * C into MWAX_ORDER output of every channel the group feeds
        // (the first group feeding a channel stores; a row's loads precede its stores).
        float2* ob = reinterpret_cast<float2*>(a.out + slot * a.out_stride);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int p = p0 + ty * 4 + i;
            int off[4];
            float2 va[4], vb[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = q0 + tx * 4 + j;
                const bool ok = p < a.n && q < a.n && (p >> 1) <= (q >> 1);
                const int pol = ((p & 1) << 1) | (q & 1);
                off[j] = ok ? (int)(baseline_of(p >> 1, q >> 1, a.T) * a.M * 4 + pol) : -1;
                va[j] = (ok && use_a && !(gr.first_a & a.first_store)) ? ob[off[j] + gr.ja * 4] : make_float2(0.f, 0.f);
                vb[j] = (ok && use_b && !(gr.first_b & a.first_store)) ? ob[off[j] + gr.jb * 4] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (off[j] < 0) continue;
                const int q = q0 + tx * 4 + j;
                const float vr = tre[i][j] * a.post_scale;
                const float vi = (p == q) ? 0.0f : tim[i][j] * a.post_scale;   // autos are real
                if (use_a) ob[off[j] + gr.ja * 4] = make_float2(fmaf(gr.ca, vr, va[j].x), fmaf(gr.ca, vi, va[j].y));
                if (use_b) ob[off[j] + gr.jb * 4] = make_float2(fmaf(gr.cb, vr, vb[j].x), fmaf(gr.cb, vi, vb[j].y));
            }
        }
    }
}

}  // namespace

cudaError_t launch_xstep_simt(const XArgs& a, int n_tiles, int n_runs, int slots, cudaStream_t s)
{
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(xstep_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(SimtSmem));
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((unsigned)n_tiles, (unsigned)n_runs, (unsigned)slots);
    xstep_simt_kernel<<<grid, 256, sizeof(SimtSmem), s>>>(a);
    return cudaGetLastError();
}

}  // namespace mwax
