// X-step, FP32 CUDA-core form (the paper's xGPU-style single-precision cross-multiply,
// Sec. 2.5.2), with time integration (Sec. 2.5.2), channel averaging (Sec. 2.6) and
// MWAX_ORDER output (Sec. 2.7) fused into the epilogue.
//
// CTA = one 64 x 64 tile of signal-path pairs (p rows, q columns; tiles on or above the
// block diagonal only) x one run of output channels x one integration slot, taken from a
// work list sorted by estimated cost (longest first, so the short ones fill the tail).
// On a diagonal tile a thread skips its register sub-blocks (i, j) with j < 2 i: their
// rows ty + 16 i >= 16 i exceed their columns tx + 8 j <= 8 j + 7 for every thread, so
// they hold only pairs below the diagonal (9 of the 32 complex accumulators).  For every
// group of ultrafine channels feeding the run, the CTA forms
//     C[p,q] = sum_{c in group} sum_k Y_p[k,c] conj(Y_q[k,c])
// (the F-step has already weighted channel c by sqrt(w_c)) and adds coef * C into every
// output channel the group feeds.  Each output element is owned by exactly one CTA, so
// the read-modify-write needs no atomics.
//
// Operands stay in the F-step's K-major planes Y[slot][c][plane][p][Kpad].  32-frame
// chunks of the A and B tiles (both planes, 64 rows x 128 B each) stream through a
// three-stage shared-memory ring by TMA with 128-byte swizzle.  Four warps consume every
// chunk; the warp that releases a stage last refills it with the chunk three ahead, so
// two chunks are always in flight and no thread blocks on a producer role.  A thread owns
// a 4 x 8 complex register tile (rows ty + 16 i, columns tx + 8 j) and reads MWAX_SIMT_VEC
// frames of an operand row per shared load (the swizzle keeps the 4-row A reads and the
// 8-row B reads of a warp conflict-free).  Accumulation is two-level: a fresh FP32
// partial per chunk, added into the running group total (keeps the rounding error of
// 10^4-term sums near the FP32 unit).  Waits are bounded: a stalled wait sets a status
// bit and the CTA drains its in-flight copies and returns.
#include "mwax_internal.cuh"
#include "tc_ptx.cuh"

#ifndef MWAX_SIMT_VEC
#define MWAX_SIMT_VEC 2   // frames per shared load: 2 (8-byte loads) or 4 (16-byte loads)
#endif

namespace mwax {
namespace {

constexpr int TP = 64;                        // paths per tile side
constexpr int KT = 32;                        // frames per chunk (128 B of one row)
constexpr int STAGES = 3;                     // TMA ring depth
constexpr int PLANE_BYTES = TP * KT * 4;      // 8 KB: one plane of one operand tile
constexpr int TILE_BYTES = 2 * PLANE_BYTES;   // Re and Im planes
constexpr int NTHREADS = 128;
constexpr int NWARPS = NTHREADS / 32;

struct SimtBars {
    uint64_t full[STAGES];
    unsigned int released[STAGES];   // warps done with the stage, counted modulo NWARPS
    unsigned int issued;             // chunks copied so far
    int abort;
    int local_status;
};

constexpr size_t simt_smem_bytes() { return 1024 + 2 * STAGES * TILE_BYTES + sizeof(SimtBars); }

__device__ __forceinline__ long long baseline_of(int i, int j, int T)
{
    return (long long)i * (2 * T - i + 1) / 2 + (j - i);
}

// Position in the chunk sequence every role walks identically: groups of the run that
// feed it, their channels with non-zero weight, the 32-frame chunks of each.
struct Cursor {
    int g, c;
    long long ch;
    bool valid;
};

// From (g, c) on, find the next (group, channel) whose chunks the CTA consumes.
__device__ __forceinline__ bool next_source(const XArgs& a, const RunInfo& run, int& g, int& c)
{
    for (; g < run.g1; ++g, c = -1) {
        const Group gr = a.groups[g];
        if (!(gr.ja >= run.j0 && gr.ja < run.j1) && !(gr.jb >= run.j0 && gr.jb < run.j1)) continue;
        if (c < gr.c0) c = gr.c0;
        for (; c < gr.c1; ++c)
            if (__ldg(&a.gain[c]) != 0.0f) return true;
    }
    return false;
}

__device__ __forceinline__ Cursor cursor_begin(const XArgs& a, const RunInfo& run, long long nchunks)
{
    Cursor u{run.g0, -1, 0, false};
    u.valid = nchunks > 0 && next_source(a, run, u.g, u.c);
    return u;
}

__device__ __forceinline__ void cursor_next(const XArgs& a, const RunInfo& run, long long nchunks, Cursor& u)
{
    if (!u.valid) return;
    if (++u.ch == nchunks) {
        u.ch = 0;
        ++u.c;
        u.valid = next_source(a, run, u.g, u.c);
    }
}

// Copy chunk `u` of the A (and, off the diagonal, B) tile into `stage`.
__device__ __forceinline__ void issue_chunk(const CUtensorMap* map, SimtBars& S, unsigned char* ring_a,
                                            unsigned char* ring_b, int stage, const Cursor& u, int slot, int N,
                                            int p0, int q0, bool diag)
{
    const int z = (slot * N + u.c) * 2;
    tc::mbar_arrive_expect_tx(&S.full[stage], diag ? TILE_BYTES : 2 * TILE_BYTES);
    tc::tma_load_3d(ring_a + stage * TILE_BYTES, map, &S.full[stage], (int)(u.ch * KT), p0, z);
    if (!diag) tc::tma_load_3d(ring_b + stage * TILE_BYTES, map, &S.full[stage], (int)(u.ch * KT), q0, z);
    atomicAdd(&S.issued, 1u);
}

template <bool first>
__device__ __forceinline__ void cmac(float xr, float xi, float yr, float yi, float& re, float& im)
{
    // re + i im += (xr + i xi)(yr - i yi)
    if (first) {
        re = xr * yr;
        im = xi * yr;
    } else {
        re = fmaf(xr, yr, re);
        im = fmaf(xi, yr, im);
    }
    re = fmaf(xi, yi, re);
    im = fmaf(-xr, yi, im);
}

// The four frames of one 16-byte column chunk into the thread's partial.  oa / ob: byte
// offsets of the thread's first A row (ty) and first B row (tx) at this column chunk
// (swizzle applied); A rows step by 16 (2 KB), B rows by 8 (1 KB).  DIAG: a diagonal tile
// (sub-blocks j < 2 i lie below the diagonal and are skipped; they stay 0).
template <bool first, bool DIAG>
__device__ __forceinline__ void column_chunk(const unsigned char* sa, const unsigned char* sb, uint32_t oa,
                                             uint32_t ob, float (&pre)[4][8], float (&pim)[4][8])
{
#if MWAX_SIMT_VEC == 4
    float4 ar[4], ai[4], br[8], bi[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        ar[i] = *reinterpret_cast<const float4*>(sa + oa + i * 2048);
        ai[i] = *reinterpret_cast<const float4*>(sa + PLANE_BYTES + oa + i * 2048);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        br[j] = *reinterpret_cast<const float4*>(sb + ob + j * 1024);
        bi[j] = *reinterpret_cast<const float4*>(sb + PLANE_BYTES + ob + j * 1024);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (DIAG && j < 2 * i) {
                if (first) pre[i][j] = pim[i][j] = 0.f;
                continue;
            }
            cmac<first>(ar[i].x, ai[i].x, br[j].x, bi[j].x, pre[i][j], pim[i][j]);
            cmac<false>(ar[i].y, ai[i].y, br[j].y, bi[j].y, pre[i][j], pim[i][j]);
            cmac<false>(ar[i].z, ai[i].z, br[j].z, bi[j].z, pre[i][j], pim[i][j]);
            cmac<false>(ar[i].w, ai[i].w, br[j].w, bi[j].w, pre[i][j], pim[i][j]);
        }
#else
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float2 ar[4], ai[4], br[8], bi[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ar[i] = *reinterpret_cast<const float2*>(sa + oa + i * 2048 + h * 8);
            ai[i] = *reinterpret_cast<const float2*>(sa + PLANE_BYTES + oa + i * 2048 + h * 8);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            br[j] = *reinterpret_cast<const float2*>(sb + ob + j * 1024 + h * 8);
            bi[j] = *reinterpret_cast<const float2*>(sb + PLANE_BYTES + ob + j * 1024 + h * 8);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (DIAG && j < 2 * i) {
                    if (first && h == 0) pre[i][j] = pim[i][j] = 0.f;
                    continue;
                }
                if (h == 0)
                    cmac<first>(ar[i].x, ai[i].x, br[j].x, bi[j].x, pre[i][j], pim[i][j]);
                else
                    cmac<false>(ar[i].x, ai[i].x, br[j].x, bi[j].x, pre[i][j], pim[i][j]);
                cmac<false>(ar[i].y, ai[i].y, br[j].y, bi[j].y, pre[i][j], pim[i][j]);
            }
    }
#endif
}

// The 32 frames of one staged chunk into the thread's partials.
template <bool DIAG>
__device__ __forceinline__ void chunk_partials(const unsigned char* sa, const unsigned char* sb, int ty, int tx,
                                               float (&pre)[4][8], float (&pim)[4][8])
{
    column_chunk<true, DIAG>(sa, sb, ty * 128 + ((ty & 7) << 4), tx * 128 + (tx << 4), pre, pim);
#pragma unroll 1
    for (int ck = 1; ck < KT / 4; ++ck)
        column_chunk<false, DIAG>(sa, sb, ty * 128 + ((ck ^ (ty & 7)) << 4), tx * 128 + ((ck ^ tx) << 4), pre, pim);
}

// order: work list (tile, run, slot) indexed by blockIdx.x, or nullptr for a 3-D grid
// (x = tile, y = run, z = slot).
__global__ void __launch_bounds__(NTHREADS, 2)
    xstep_simt_kernel(const __grid_constant__ CUtensorMap map, const XArgs a, const XItem* __restrict__ order)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);   // swizzle atom
    unsigned char* ring_a = base;                              // [STAGES][2 planes][64 rows][128 B]
    unsigned char* ring_b = base + STAGES * TILE_BYTES;
    SimtBars& S = *reinterpret_cast<SimtBars*>(base + 2 * STAGES * TILE_BYTES);

    int tile_i = blockIdx.x, run_i = blockIdx.y, slot = blockIdx.z;
    if (order != nullptr) {
        const XItem w = order[blockIdx.x];
        tile_i = w.tile;
        run_i = w.run;
        slot = w.slot;
    }
    const int4 tile = a.tiles[tile_i];
    const RunInfo run = a.runs[run_i];
    const int p0 = tile.x, q0 = tile.y;
    const bool diag = (p0 == q0);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const long long nchunks = (a.klen + KT - 1) / KT;
    const long long lim = (long long)(a.spin_limit > 0 ? a.spin_limit : tc::kDefaultSpin) * 1000LL;
    volatile int* abort = &S.abort;
    int* status = a.status ? a.status : &S.local_status;

    // Each warp's cursor runs STAGES chunks ahead of the chunk it consumes: it names the
    // chunk to copy when this warp is the last to release a stage.
    Cursor ahead = cursor_begin(a, run, nchunks);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&S.full[s], 1);
            S.released[s] = 0;
        }
        S.issued = 0;
        S.abort = 0;
        S.local_status = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&map);
    }
    __syncthreads();
    for (int s = 0; s < STAGES; ++s) {
        if (tid == 0 && ahead.valid) issue_chunk(&map, S, ring_a, ring_b, s, ahead, slot, a.N, p0, q0, diag);
        cursor_next(a, run, nchunks, ahead);
    }

    const int ty = tid >> 3, tx = tid & 7;   // rows ty + 16 i (i < 4), columns tx + 8 j (j < 8)
    const unsigned char* a_ring = ring_a;
    const unsigned char* b_ring = diag ? ring_a : ring_b;
    long long it = 0;
    bool ok = true;

    for (int g = run.g0; g < run.g1 && ok; ++g) {
        const Group gr = a.groups[g];
        const bool use_a = gr.ja >= run.j0 && gr.ja < run.j1;
        const bool use_b = gr.jb >= run.j0 && gr.jb < run.j1;
        if (!use_a && !use_b) continue;

        float tre[4][8], tim[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) tre[i][j] = tim[i][j] = 0.f;

        for (int c = gr.c0; c < gr.c1 && ok; ++c) {
            if (__ldg(&a.gain[c]) == 0.0f) continue;
            for (long long ch = 0; ch < nchunks; ++ch, ++it) {
                const int s = (int)(it % STAGES);
                if (!tc::mbar_wait(&S.full[s], (uint32_t)((it / STAGES) & 1), abort, status, 128, lim)) {
                    ok = false;
                    break;
                }
                const unsigned char* sa = a_ring + s * TILE_BYTES;
                const unsigned char* sb = b_ring + s * TILE_BYTES;
                float pre[4][8], pim[4][8];
                if (diag)
                    chunk_partials<true>(sa, sb, ty, tx, pre, pim);
                else
                    chunk_partials<false>(sa, sb, ty, tx, pre, pim);
                // Release the stage (every shared-memory read of it has returned: its values
                // are used above); the last warp to release it copies the chunk STAGES ahead.
                __syncwarp();
                if (lane == 0 && atomicAdd(&S.released[s], 1u) % NWARPS == NWARPS - 1 && ahead.valid)
                    issue_chunk(&map, S, ring_a, ring_b, s, ahead, slot, a.N, p0, q0, diag);
                cursor_next(a, run, nchunks, ahead);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        tre[i][j] += pre[i][j];
                        tim[i][j] += pim[i][j];
                    }
            }
        }   // channels of the group
        if (!ok) break;

        // Epilogue: add coef * C into MWAX_ORDER output of every channel the group feeds
        // (the first group feeding a channel stores; a row's loads precede its stores).
        float2* ob = reinterpret_cast<float2*>(a.out + slot * a.out_stride);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int p = p0 + ty + 16 * i;
            int off[8];
            float2 va[8], vb[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int q = q0 + tx + 8 * j;
                const bool in = p < a.n && q < a.n && (p >> 1) <= (q >> 1);
                const int pol = ((p & 1) << 1) | (q & 1);
                off[j] = in ? (int)(baseline_of(p >> 1, q >> 1, a.T) * a.M * 4 + pol) : -1;
                va[j] = (in && use_a && !(gr.first_a & a.first_store)) ? ob[off[j] + gr.ja * 4] : make_float2(0.f, 0.f);
                vb[j] = (in && use_b && !(gr.first_b & a.first_store)) ? ob[off[j] + gr.jb * 4] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (off[j] < 0) continue;
                const int q = q0 + tx + 8 * j;
                const float vr = tre[i][j] * a.post_scale;
                const float vi = (p == q) ? 0.0f : tim[i][j] * a.post_scale;   // autos are real
                if (use_a) ob[off[j] + gr.ja * 4] = make_float2(fmaf(gr.ca, vr, va[j].x), fmaf(gr.ca, vi, va[j].y));
                if (use_b) ob[off[j] + gr.jb * 4] = make_float2(fmaf(gr.cb, vr, vb[j].x), fmaf(gr.cb, vi, vb[j].y));
            }
        }
    }

    // Drain: the last copy issued into each stage has landed before the CTA exits (already
    // true unless a wait gave up; copies from valid addresses always land, so the bound is
    // the fixed drain bound, not the spin limit that may have fired).
    __syncthreads();
    if (tid == 0) {
        const long long issued = S.issued;
        for (int st = 0; st < STAGES; ++st) {
            if (issued <= st) continue;
            const long long last = issued - 1 - ((issued - 1 - st) % STAGES);   // last chunk copied into st
            if (!tc::wait_bounded(&S.full[st], (uint32_t)((last / STAGES) & 1), tc::kDrainCycles))
                atomicOr(status, tc::kDrainGaveUp);
        }
    }
}

}  // namespace

cudaError_t simt_attributes()
{
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(xstep_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)simt_smem_bytes());
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    return cudaSuccess;
}

cudaError_t launch_xstep_simt(const CUtensorMap& map, const XArgs& a, int n_tiles, int n_runs, int slots,
                              cudaStream_t s)
{
    cudaError_t e = simt_attributes();
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)n_tiles, (unsigned)n_runs, (unsigned)slots);
    xstep_simt_kernel<<<grid, NTHREADS, simt_smem_bytes(), s>>>(map, a, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_xstep_simt_items(const CUtensorMap& map, const XArgs& a, const XItem* items, int n_items,
                                    cudaStream_t s)
{
    cudaError_t e = simt_attributes();
    if (e != cudaSuccess) return e;
    xstep_simt_kernel<<<(unsigned)n_items, NTHREADS, simt_smem_bytes(), s>>>(map, a, items);
    return cudaGetLastError();
}

int simt_resident_ctas()
{
    int n = 0;
    if (simt_attributes() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, xstep_simt_kernel, NTHREADS, simt_smem_bytes()) !=
            cudaSuccess)
        return 2;
    return n > 0 ? n : 1;
}

}  // namespace mwax
