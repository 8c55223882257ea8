// X-step on the 5th-generation tensor cores (tcgen05, TMEM accumulators, TMA operand
// staging) for the FP16, FP8-e4m3 and FP16 hi/lo pair forms, with the same fused epilogue
// as the CUDA-core form: integration over the frames of a slot (Sec. 2.5.2), channel
// averaging (Sec. 2.6) and MWAX_ORDER output (Sec. 2.7); and for the exact integer mode
// (no FFT, int64 sums of the int8 voltages).
//
// The complex product C = Y_p conj(Y_q) is four real MMAs on planar operands:
//     Re C = Ar Br^T + Ai Bi^T,      Im C = Ai Br^T - Ar Bi^T
// (the last with the instruction's A-negate bit).  Operands are K-major planes
// Y[slot][c][plane][p][Kpad] loaded by TMA with 64-byte swizzle.
//
// The kernel is persistent: one CTA per SM claims work items (job, tile, run of output
// channels, slot) from a global counter, most expensive first (the host sorts the list
// by estimated cost); the producer warp claims and publishes each item index to the MMA
// and epilogue warps through a small shared-memory ring.  A job is one plan's launch (its operand
// tensor map and arguments), so one launch serves a single plan or a batch of coarse
// channels of mixed shapes and precisions.  The TMA ring, MMA and epilogue pipelines run
// on across item boundaries.  A tile is 128 rows (paths p) by a window of 256 (or, at
// the right edge, 128) columns (paths q).  Windows start at
// the tile's own diagonal, so for those the 128 A rows are the first 128 rows of the B
// window and only B is loaded; elsewhere A and B are loaded separately.  For each group of
// ultrafine channels (pre-weighted by sqrt(w) in the F-step) the MMAs of every frame of
// every channel in the group accumulate into one TMEM accumulator pair (Re: columns
// [0, 256), Im: [256, 512)), which the epilogue drains once per group.  When every tile of
// the launch is at most 128 columns wide the pair needs only 256 columns, and two pairs
// alternate (buffer b: Re [256 b, 256 b + 128), Im [256 b + 128, 256 b + 256)): the MMAs
// of the next group run while the epilogue drains the previous one.
//
// 10 warps: warp 0 issues TMA loads into a 4-stage ring, warp 1 owns TMEM and issues the
// MMAs from one thread, warps 2-9 drain the accumulators (TMEM lane quarter = warp % 4,
// column half = (warp - 2) / 4; one TMEM lane = one path p).
//
// Integer mode: sm_103a has no integer MMA, but every int8 value is exact in FP16 and every
// product of two is exact in FP32.  The MMAs of 512 samples go into a fresh TMEM partial
// (every partial sum an integer of magnitude at most 512 * 2 * 128^2 = 2^24, so exact),
// two partial buffers alternate, and the epilogue adds each partial into int32 register
// totals.  A work item is (tile, segment of at most 51,200 samples, slot), so the totals
// stay below 2^31; at its end they go into the int64 output by 64-bit atomic adds (integer
// addition: the order of the segments does not matter).  The operands of this mode are
// K-tiled, [slot][K tile][re/im][p][2048], so that the rows of one TMA box lie close together.
//
// FP16 hi/lo pair form (FP32-accurate products on the tensor cores): every operand value
// v is held as hi = fp16(v) and lo = fp16(v - hi) (22 significant bits), and each complex
// product is (Ah + Al)(Bh + Bl)^H less the Al Bl^H term, i.e. twelve real MMAs whose
// products are exact in FP32; the dropped term is 2^-22 of the product.  The MMAs of 128
// frames at a time go into a fresh TMEM partial (two partial buffers alternate), and the
// epilogue adds each partial into FP32 register totals: the two-level sum keeps the
// accumulation error of an integration of thousands of frames at the FP32 level, where
// one MMA accumulation over all of them would not be.  Tiles are 128 x 128 (the register
// totals hold one row's 64 columns per epilogue thread); the ring has 3 stages of the 8
// planes (re, im x hi, lo of A and B).
#include "mwax_internal.cuh"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>

#include <type_traits>

namespace mwax {
namespace {

constexpr int TM = 128;                        // rows (paths p) per tile
constexpr int TNMAX = 256;                     // columns (paths q) per tile
constexpr int ROWB = 64;                       // bytes of K per operand row in a stage
constexpr int A_PLANE = TM * ROWB;             // 8 KB
constexpr int B_PLANE = TNMAX * ROWB;          // 16 KB
constexpr int NTHREADS = 320;
constexpr int EPI_THREADS = 256;
constexpr uint32_t TMEM_COLS = 512;
constexpr int MAX_STAGES = 4;

// Kernel modes: one FP16 / e4m3 product per term, accumulated per channel group in TMEM;
// FP16 hi/lo pairs (three products per term) in chunked partial sums added into FP32
// register totals; integer mode (int8 values held in FP16) in exact 512-sample partials
// added into int32 register totals and flushed as int64 atomics per segment.
constexpr int MODE_ONE = 0, MODE_PAIRS = 1, MODE_INT = 2;

// Ring geometry.  One-product and integer modes: 4 stages of Br, Bi (256 rows) and Ar, Ai
// (48 KB).  Pairs (128-column windows only): 3 stages of Br, Bi, Br', Bi', Ar, Ai, Ar',
// Ai' (' = low halves; 8 planes of 128 rows, 64 KB).
template <int MODE>
struct Ring {
    static constexpr int stages = MODE == MODE_PAIRS ? 3 : 4;
    static constexpr int stage_bytes = MODE == MODE_PAIRS ? 8 * A_PLANE : 2 * B_PLANE + 2 * A_PLANE;
};

// k-blocks (32 frames each) per TMEM partial sum in the chunked modes.  Pairs: 128 frames,
// so no tensor-core accumulation runs longer than 48 MMAs (64 frames measured 1-5 % slower
// in the X-step, same accuracy bar).  Integer mode: 512 samples,
// every partial an integer of magnitude at most 512 * 2 * 128^2 = 2^24, exact in FP32.
template <int MODE>
__host__ __device__ constexpr int chunk_kb()
{
    return MODE == MODE_PAIRS ? 4 : 16;
}

constexpr int IRING = 4;   // claimed work items in flight between the roles

struct TcSmem {
    uint64_t full[MAX_STAGES];
    uint64_t empty[MAX_STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t item_full[IRING];    // producer -> MMA + epilogue: item index published
    uint64_t item_empty[IRING];   // MMA + epilogue -> producer: slot free again
    int item[IRING];              // claimed item index, -1 = no more work
    uint64_t drained;             // after an abort: the MMA issuer's last commit (all its MMAs done)
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ long long baseline_of(int i, int j, int T)
{
    return (long long)i * (2 * T - i + 1) / 2 + (j - i);
}

__device__ __forceinline__ bool item_feeds(const Group& gr, const RunInfo& run)
{
    return (gr.ja >= run.j0 && gr.ja < run.j1) || (gr.jb >= run.j0 && gr.jb < run.j1);
}

// Ultrafine channels of a group that carry weight (the others are skipped).
__device__ __forceinline__ int live_channels(const XArgs& a, const Group& gr)
{
    int live = 0;
    for (int c = gr.c0; c < gr.c1; ++c) live += __ldg(&a.gain[c]) != 0.0f;
    return live;
}

// Add coef x (re, im) of row p and the 8 consecutive columns q = qc .. qc + 7 into the
// output channels ja / jb that the group feeds (MWAX_ORDER), or store where this group is
// the channel's first.  Every load of the old values is issued before any store, so the
// read-modify-writes overlap instead of serialising.
__device__ __forceinline__ void emit8(const XArgs& a, const Group& gr, bool use_a, bool use_b, float2* ob, int p,
                                      int qc, const float (&re)[8], const float (&im)[8])
{
    const int T = a.T, M = a.M, n = a.n, first_store = a.first_store;
    const int ti = p >> 1;
    int off[8];
    float2 va[8], vb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int q = qc + i;
        const int tj = q >> 1;
        const bool okq = q < n && ti <= tj;
        const int pol = ((p & 1) << 1) | (q & 1);
        off[i] = okq ? (int)(baseline_of(ti, tj, T) * M * 4 + pol) : -1;
        va[i] = (okq && use_a && !(gr.first_a & first_store)) ? ob[off[i] + gr.ja * 4] : make_float2(0.f, 0.f);
        vb[i] = (okq && use_b && !(gr.first_b & first_store)) ? ob[off[i] + gr.jb * 4] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (off[i] < 0) continue;
        const float vi = (p == qc + i) ? 0.0f : im[i];   // autocorrelation: exactly real
        if (use_a) ob[off[i] + gr.ja * 4] = make_float2(fmaf(gr.ca, re[i], va[i].x), fmaf(gr.ca, vi, va[i].y));
        if (use_b) ob[off[i] + gr.jb * 4] = make_float2(fmaf(gr.cb, re[i], vb[i].x), fmaf(gr.cb, vi, vb[i].y));
    }
}

// Write-out of row p's columns [col, col + 32 pieces) of the accumulator whose real part
// starts at TMEM column re0 (imaginary part im_off further on): scale (post_scale, and the
// e4m3 scales of p and q for FP8), then emit8.  Every lane of the warp takes part in the
// TMEM loads.
__device__ __forceinline__ void drain(const XArgs& a, const Group& gr, bool use_a, bool use_b, float2* ob, int p,
                                      int q0, uint32_t tlane, uint32_t re0, uint32_t im_off, int col, int pieces,
                                      float sp, const float* qscale)
{
    const int n = a.n;
#pragma unroll 1
    for (int ch = 0; ch < pieces; ++ch) {
        const int c = col + ch * 32;
        uint32_t vr[32], vi[32];
        tc::tmem_ld32(tlane + re0 + c, vr);
        tc::tmem_ld32(tlane + re0 + c + im_off, vi);
        tc::tmem_wait_ld();
        if (p >= n) continue;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float re[8], im[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = q0 + c + h * 8 + i;
                float s = sp;
                if (qscale != nullptr) s *= (q < n) ? e4m3_scale(__ldg(qscale + q)) : 0.0f;
                re[i] = __uint_as_float(vr[h * 8 + i]) * s;
                im[i] = __uint_as_float(vi[h * 8 + i]) * s;
            }
            emit8(a, gr, use_a, use_b, ob, p, q0 + c + h * 8, re, im);
        }
    }
}

// Integer mode: add row p's int32 segment sums for columns [col, col + 64) (TMEM: real
// part at tre, imaginary part 128 columns further on) into the int64 (re, im) MWAX_ORDER
// output (one channel) with 64-bit atomic adds: integer addition, so the result does not
// depend on the order in which segments arrive.  Every lane takes part in the TMEM loads.
__device__ __forceinline__ void flush_int(const XArgs& a, char* obase, int p, int q0, uint32_t tre, int col)
{
    const int n = a.n, ti = p >> 1;
    long long* ob64 = reinterpret_cast<long long*>(obase);
#pragma unroll 1
    for (int ch = 0; ch < 2; ++ch) {
        const int c = col + ch * 32;
        uint32_t re[32], im[32];
        tc::tmem_ld32(tre + c, re);
        tc::tmem_ld32(tre + 128 + c, im);
        tc::tmem_wait_ld();
        if (p >= n) continue;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int q = q0 + c + i;
            if (q < n && ti <= (q >> 1)) {
                const int pol = ((p & 1) << 1) | (q & 1);
                unsigned long long* o =
                    reinterpret_cast<unsigned long long*>(ob64 + (baseline_of(ti, q >> 1, a.T) * 4 + pol) * 2);
                const long long vi = (p == q) ? 0LL : (long long)(int)im[i];
                atomicAdd(o, (unsigned long long)(long long)(int)re[i]);   // two's complement add
                if (vi != 0) atomicAdd(o + 1, (unsigned long long)vi);
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
    xstep_tc_kernel(const __grid_constant__ XLaunch L, const XItem* __restrict__ items, int n_items, int* counter,
                    int* status, unsigned int spin_limit, int dbuf)
{
    constexpr bool SPLIT = MODE == MODE_PAIRS;
    constexpr bool CHUNKED = MODE != MODE_ONE;
    constexpr int CHUNK_KB = chunk_kb<MODE>();
    constexpr int STAGES = Ring<MODE>::stages;
    constexpr int STAGE_BYTES = Ring<MODE>::stage_bytes;
    const XJob* jobs = L.jobs;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    TcSmem& S = *reinterpret_cast<TcSmem*>(ring + STAGES * STAGE_BYTES);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const long long lim = (long long)spin_limit * 1000LL;   // cycles
    if (CHUNKED) dbuf = 1;   // the partial sums always alternate between two buffers

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&S.full[s], 1);
            tc::mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&S.acc_full[b], 1);
            tc::mbar_init(&S.acc_empty[b], EPI_THREADS);
        }
        for (int r = 0; r < IRING; ++r) {
            tc::mbar_init(&S.item_full[r], 1);
            tc::mbar_init(&S.item_empty[r], 1 + EPI_THREADS);
        }
        tc::mbar_init(&S.drained, 1);
        S.abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&S.tmem_base, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem_base;
    volatile int* abort = &S.abort;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[STAGES];
            for (int s = 0; s < STAGES; ++s) issued_phase[s] = -1;
            int ir = 0;
            uint32_t iphase = 0;
            for (;;) {
                // claim the next item and publish it (-1 = done) to the other roles
                if (!tc::mbar_wait(&S.item_empty[ir], iphase ^ 1, abort, status, 32, lim)) break;
                const int it = atomicAdd(counter, 1);
                S.item[ir] = (it < n_items) ? it : -1;
                tc::mbar_arrive(&S.item_full[ir]);
                if (++ir == IRING) {
                    ir = 0;
                    iphase ^= 1;
                }
                if (it >= n_items || *abort) break;
                const XItem w = items[it];
                const XJob* J = jobs + w.job;
                const XArgs& a = J->a;
                const CUtensorMap* tm = &J->tmap;
                tc::prefetch_tmap(tm);
                const int4 tile = a.tiles[w.tile];
                const RunInfo run = a.runs[MODE == MODE_INT ? 0 : w.run];
                const int KF = (J->op == 1) ? 64 : 32;   // frames per 64-byte operand row
                const int nkb = (int)((a.klen + KF - 1) / KF);
                // k-blocks of this item: all of the slot's, or (integer mode) segment w.run's
                const int kb_lo = MODE == MODE_INT ? w.run * (int)(a.seg_frames / KF) : 0;
                const int kb_hi = MODE == MODE_INT ? min(nkb, kb_lo + (int)(a.seg_frames / KF)) : nkb;
                const int nbox = tile.z / TM;             // 128-row boxes of the B window
                const bool a_in_b = tile.w != 0;
                const uint32_t bytes = SPLIT ? (uint32_t)((a_in_b ? 4 : 8) * A_PLANE)
                                             : (uint32_t)(2 * nbox * A_PLANE + (a_in_b ? 0 : 2 * A_PLANE));
                const int klo = (int)a.Kpad;   // hi/lo pairs: the low halves start Kpad frames into a row
                for (int g = run.g0; g < run.g1 && !*abort; ++g) {
                    const Group gr = a.groups[g];
                    if (!item_feeds(gr, run)) continue;
                    for (int c = gr.c0; c < gr.c1 && !*abort; ++c) {
                        if (__ldg(&a.gain[c]) == 0.0f) continue;
                        int zr = (w.slot * a.N + c) * 2, zi = zr + 1;
                        for (int kb = kb_lo; kb < kb_hi; ++kb) {
                            int kx = kb * KF;
                            if (MODE == MODE_INT) {
                                // K-tiled operand planes [slot][K tile][re/im] (one channel)
                                const int kt = (int)(kx / a.ktile);
                                zr = (int)((w.slot * (a.Kpad / a.ktile) + kt) * 2);
                                zi = zr + 1;
                                kx -= (int)(kt * a.ktile);
                            }
                            if (!tc::mbar_wait(&S.empty[stage], phase ^ 1, abort, status, 2, lim)) break;
                            unsigned char* st = ring + stage * STAGE_BYTES;
                            uint64_t* fb = &S.full[stage];
                            tc::mbar_arrive_expect_tx(fb, bytes);
                            if (SPLIT) {
                                const int kl = klo + kx;
                                tc::tma_load_3d(st, tm, fb, kx, tile.y, zr);
                                tc::tma_load_3d(st + A_PLANE, tm, fb, kx, tile.y, zi);
                                tc::tma_load_3d(st + 2 * A_PLANE, tm, fb, kl, tile.y, zr);
                                tc::tma_load_3d(st + 3 * A_PLANE, tm, fb, kl, tile.y, zi);
                                if (!a_in_b) {
                                    tc::tma_load_3d(st + 4 * A_PLANE, tm, fb, kx, tile.x, zr);
                                    tc::tma_load_3d(st + 5 * A_PLANE, tm, fb, kx, tile.x, zi);
                                    tc::tma_load_3d(st + 6 * A_PLANE, tm, fb, kl, tile.x, zr);
                                    tc::tma_load_3d(st + 7 * A_PLANE, tm, fb, kl, tile.x, zi);
                                }
                            } else {
                                for (int b = 0; b < nbox; ++b) {
                                    tc::tma_load_3d(st + b * A_PLANE, tm, fb, kx, tile.y + b * TM, zr);
                                    tc::tma_load_3d(st + B_PLANE + b * A_PLANE, tm, fb, kx, tile.y + b * TM, zi);
                                }
                                if (!a_in_b) {
                                    tc::tma_load_3d(st + 2 * B_PLANE, tm, fb, kx, tile.x, zr);
                                    tc::tma_load_3d(st + 2 * B_PLANE + A_PLANE, tm, fb, kx, tile.x, zi);
                                }
                            }
                            issued_phase[stage] = (int)phase;
                            if (++stage == STAGES) {
                                stage = 0;
                                phase ^= 1;
                            }
                        }
                    }
                }
            }
            if (*abort) {
                // let the last load issued into each stage land before the CTA can exit
                // (loads from valid addresses always land: the bound is not the spin limit)
                for (int s = 0; s < STAGES; ++s)
                    if (issued_phase[s] >= 0 && !tc::wait_bounded(&S.full[s], (uint32_t)issued_phase[s], tc::kDrainCycles))
                        atomicOr(status, tc::kDrainGaveUp);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, gcount = 0;   // gcount: accumulator uses so far (groups; chunks for pairs)
            int cur_b = 0;
            uint32_t cur_ph = 0;
            const uint32_t sbase = tc::smem_u32(ring);
            bool issued = false;
            int ir = 0;
            uint32_t iphase = 0;
            for (;;) {
                if (!tc::mbar_wait(&S.item_full[ir], iphase, abort, status, 32, lim)) break;
                const int it = S.item[ir];
                tc::mbar_arrive(&S.item_empty[ir]);
                if (++ir == IRING) {
                    ir = 0;
                    iphase ^= 1;
                }
                if (it < 0 || *abort) break;
                const XItem w = items[it];
                const XJob* J = jobs + w.job;
                const XArgs& a = J->a;
                const int op = J->op;
                const int4 tile = a.tiles[w.tile];
                const RunInfo run = a.runs[MODE == MODE_INT ? 0 : w.run];
                const int KF = (op == 1) ? 64 : 32;
                const int nkb = (int)((a.klen + KF - 1) / KF);
                const int kb_lo = MODE == MODE_INT ? w.run * (int)(a.seg_frames / KF) : 0;
                const int kb_hi = MODE == MODE_INT ? min(nkb, kb_lo + (int)(a.seg_frames / KF)) : nkb;
                const bool a_in_b = tile.w != 0;
                const uint32_t id = tc::idesc(0, TM, tile.z, false), id_neg = tc::idesc(0, TM, tile.z, true);
                for (int g = run.g0; g < run.g1 && !*abort; ++g) {
                    const Group gr = a.groups[g];
                    if (!item_feeds(gr, run)) continue;
                    if (CHUNKED) {
                        // a fresh partial per CHUNK_KB k-blocks, alternating buffers
                        const int total = live_channels(a, gr) * (kb_hi - kb_lo);
                        int done = 0;
                        bool first = true;
                        uint32_t d_re = 0, d_im = 0;
                        for (int c = gr.c0; c < gr.c1 && !*abort; ++c) {
                            if (__ldg(&a.gain[c]) == 0.0f) continue;
                            for (int kb = kb_lo; kb < kb_hi; ++kb) {
                                if (done % CHUNK_KB == 0) {
                                    cur_b = (int)(gcount & 1);
                                    cur_ph = (gcount >> 1) & 1;
                                    d_re = tmem + 256u * cur_b;
                                    d_im = d_re + 128u;
                                    if (!tc::mbar_wait(&S.acc_empty[cur_b], cur_ph ^ 1, abort, status, 4, lim)) break;
                                    tc::fence_after();
                                    first = true;
                                }
                                if (!tc::mbar_wait(&S.full[stage], phase, abort, status, 8, lim)) break;
                                tc::fence_after();
                                const uint32_t st = sbase + stage * STAGE_BYTES;
                                if (!SPLIT) {
                                    // integer mode: int8 values held in FP16, one product per term
                                    const uint64_t dbr = tc::sw64_desc(st), dbi = tc::sw64_desc(st + B_PLANE);
                                    const uint64_t dar = a_in_b ? dbr : tc::sw64_desc(st + 2 * B_PLANE);
                                    const uint64_t dai = a_in_b ? dbi : tc::sw64_desc(st + 2 * B_PLANE + A_PLANE);
#pragma unroll
                                    for (int k = 0; k < ROWB / 32; ++k) {
                                        const uint64_t off = (uint64_t)(k * 32) >> 4;
                                        const uint32_t acc = first ? 0u : 1u;
                                        first = false;
                                        tc::mma_f16(d_re, dar + off, dbr + off, id, acc);
                                        tc::mma_f16(d_re, dai + off, dbi + off, id, 1u);
                                        tc::mma_f16(d_im, dai + off, dbr + off, id, acc);
                                        tc::mma_f16(d_im, dar + off, dbi + off, id_neg, 1u);
                                    }
                                } else {
                                    const uint64_t brh = tc::sw64_desc(st), bih = tc::sw64_desc(st + A_PLANE);
                                    const uint64_t brl = tc::sw64_desc(st + 2 * A_PLANE);
                                    const uint64_t bil = tc::sw64_desc(st + 3 * A_PLANE);
                                    const uint64_t arh = a_in_b ? brh : tc::sw64_desc(st + 4 * A_PLANE);
                                    const uint64_t aih = a_in_b ? bih : tc::sw64_desc(st + 5 * A_PLANE);
                                    const uint64_t arl = a_in_b ? brl : tc::sw64_desc(st + 6 * A_PLANE);
                                    const uint64_t ail = a_in_b ? bil : tc::sw64_desc(st + 7 * A_PLANE);
#pragma unroll
                                    for (int k = 0; k < ROWB / 32; ++k) {
                                        const uint64_t off = (uint64_t)(k * 32) >> 4;
                                        const uint32_t acc = first ? 0u : 1u;
                                        first = false;
                                        // (Ah + Al)(Bh + Bl)^H without the Al Bl^H term
                                        tc::mma_f16(d_re, arh + off, brh + off, id, acc);
                                        tc::mma_f16(d_re, aih + off, bih + off, id, 1u);
                                        tc::mma_f16(d_re, arh + off, brl + off, id, 1u);
                                        tc::mma_f16(d_re, aih + off, bil + off, id, 1u);
                                        tc::mma_f16(d_re, arl + off, brh + off, id, 1u);
                                        tc::mma_f16(d_re, ail + off, bih + off, id, 1u);
                                        tc::mma_f16(d_im, aih + off, brh + off, id, acc);
                                        tc::mma_f16(d_im, arh + off, bih + off, id_neg, 1u);
                                        tc::mma_f16(d_im, aih + off, brl + off, id, 1u);
                                        tc::mma_f16(d_im, arh + off, bil + off, id_neg, 1u);
                                        tc::mma_f16(d_im, ail + off, brh + off, id, 1u);
                                        tc::mma_f16(d_im, arl + off, bih + off, id_neg, 1u);
                                    }
                                }
                                issued = true;
                                tc::mma_commit(&S.empty[stage]);
                                if (++stage == STAGES) {
                                    stage = 0;
                                    phase ^= 1;
                                }
                                if (++done % CHUNK_KB == 0 || done == total) {
                                    tc::mma_commit(&S.acc_full[cur_b]);
                                    ++gcount;
                                }
                            }
                        }
                        if (*abort) break;
                        continue;
                    }
                    // accumulator buffer of this group and the parity of its use
                    cur_b = dbuf ? (int)(gcount & 1) : 0;
                    cur_ph = dbuf ? ((gcount >> 1) & 1) : (gcount & 1);
                    const uint32_t d_re = tmem + (dbuf ? 256u * cur_b : 0u), d_im = d_re + (dbuf ? 128u : 256u);
                    if (!tc::mbar_wait(&S.acc_empty[cur_b], cur_ph ^ 1, abort, status, 4, lim)) break;
                    tc::fence_after();
                    bool first = true;
                    for (int c = gr.c0; c < gr.c1 && !*abort; ++c) {
                        if (__ldg(&a.gain[c]) == 0.0f) continue;
                        for (int kb = 0; kb < nkb; ++kb) {
                            if (!tc::mbar_wait(&S.full[stage], phase, abort, status, 8, lim)) break;
                            tc::fence_after();
                            const uint32_t st = sbase + stage * STAGE_BYTES;
                            const uint64_t dbr = tc::sw64_desc(st), dbi = tc::sw64_desc(st + B_PLANE);
                            const uint64_t dar = a_in_b ? dbr : tc::sw64_desc(st + 2 * B_PLANE);
                            const uint64_t dai = a_in_b ? dbi : tc::sw64_desc(st + 2 * B_PLANE + A_PLANE);
#pragma unroll
                            for (int k = 0; k < ROWB / 32; ++k) {
                                const uint64_t off = (uint64_t)(k * 32) >> 4;   // 32 bytes of K per step
                                const uint32_t acc = first ? 0u : 1u;
                                first = false;
                                if (op == 0) {
                                    tc::mma_f16(d_re, dar + off, dbr + off, id, acc);
                                    tc::mma_f16(d_re, dai + off, dbi + off, id, 1u);
                                    tc::mma_f16(d_im, dai + off, dbr + off, id, acc);
                                    tc::mma_f16(d_im, dar + off, dbi + off, id_neg, 1u);
                                } else {
                                    tc::mma_f8(d_re, dar + off, dbr + off, id, acc);
                                    tc::mma_f8(d_re, dai + off, dbi + off, id, 1u);
                                    tc::mma_f8(d_im, dai + off, dbr + off, id, acc);
                                    tc::mma_f8(d_im, dar + off, dbi + off, id_neg, 1u);
                                }
                            }
                            issued = true;
                            tc::mma_commit(&S.empty[stage]);
                            if (++stage == STAGES) {
                                stage = 0;
                                phase ^= 1;
                            }
                        }
                    }
                    if (*abort) break;
                    tc::mma_commit(&S.acc_full[cur_b]);
                    ++gcount;
                }
            }
            if (*abort && issued) {
                // wait for the MMAs in flight before TMEM is released: a commit on a barrier
                // of its own arrives once every MMA issued so far has completed
                tc::mma_commit(&S.drained);
                if (!tc::wait_bounded(&S.drained, 0u, tc::kDrainCycles)) atomicOr(status, tc::kDrainGaveUp);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int g4 = warp & 3;                 // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;        // column half of the window
        uint32_t gcount = 0;
        int ir = 0;
        uint32_t iphase = 0;
        for (;;) {
            bool okit = tc::mbar_wait(&S.item_full[ir], iphase, abort, status, 32, lim);
            if (!__all_sync(0xffffffffu, okit)) break;
            const int it = S.item[ir];
            tc::mbar_arrive(&S.item_empty[ir]);
            if (++ir == IRING) {
                ir = 0;
                iphase ^= 1;
            }
            if (it < 0 || *abort) break;
            const XItem w = items[it];
            const XJob* J = jobs + w.job;
            const XArgs& a = J->a;
            const int op = J->op;
            const int4 tile = a.tiles[w.tile];
            const RunInfo run = a.runs[MODE == MODE_INT ? 0 : w.run];
            const int p0 = tile.x, q0 = tile.y, nq = tile.z;
            const int p = p0 + g4 * 32 + lane;
            const bool cols = half * 128 < nq;
            char* obase = a.out + (long long)w.slot * a.out_stride;
            float2* ob = reinterpret_cast<float2*>(obase);
            const int n = a.n;
            const int nkb = (int)((a.klen + 31) / 32);   // chunked modes: FP16, 32 frames per k-block
            const int kb_lo = MODE == MODE_INT ? w.run * (int)(a.seg_frames / 32) : 0;
            const int kb_hi = MODE == MODE_INT ? min(nkb, kb_lo + (int)(a.seg_frames / 32)) : nkb;
            for (int g = run.g0; g < run.g1 && !*abort; ++g) {
                const Group gr = a.groups[g];
                if (!item_feeds(gr, run)) continue;
                const bool use_a = gr.ja >= run.j0 && gr.ja < run.j1;
                const bool use_b = gr.jb >= run.j0 && gr.jb < run.j1;
                const uint32_t tlane = tmem + ((uint32_t)(g4 * 32) << 16);
                if (CHUNKED) {
                    // columns [64 half, 64 half + 64) of the 128-column window, summed over
                    // the group's chunk partials in registers (pairs: FP32, the totals then
                    // go back into the last partial's buffer, still held, for the write-out;
                    // integer mode: int32, flushed into the int64 output by atomic adds)
                    using Tot = typename std::conditional<MODE == MODE_INT, int, float>::type;
                    const int col0 = half * 64;
                    const int nch = (live_channels(a, gr) * (kb_hi - kb_lo) + CHUNK_KB - 1) / CHUNK_KB;
                    Tot tr[64], tq[64];
#pragma unroll
                    for (int i = 0; i < 64; ++i) {
                        tr[i] = 0;
                        tq[i] = 0;
                    }
                    bool ok = true;
                    int b = 0;
                    for (int ck = 0; ck < nch; ++ck) {
                        b = (int)(gcount & 1);
                        const uint32_t ph = (gcount >> 1) & 1;
                        ok = tc::mbar_wait(&S.acc_full[b], ph, abort, status, 16, lim);
                        if (!__all_sync(0xffffffffu, ok)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint32_t taddr = tlane + 256u * b + col0;
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            uint32_t vr[16], vi[16];
                            tc::tmem_ld16(taddr + 16 * h, vr);
                            tc::tmem_ld16(taddr + 128 + 16 * h, vi);
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                if (MODE == MODE_INT) {   // exact integers in FP32
                                    tr[16 * h + i] += __float2int_rn(__uint_as_float(vr[i]));
                                    tq[16 * h + i] += __float2int_rn(__uint_as_float(vi[i]));
                                } else {
                                    tr[16 * h + i] += __uint_as_float(vr[i]);
                                    tq[16 * h + i] += __uint_as_float(vi[i]);
                                }
                            }
                        }
                        if (ck + 1 < nch) {
                            tc::fence_before();
                            tc::mbar_arrive(&S.acc_empty[b]);
                            ++gcount;
                        }
                    }
                    if (!ok) break;
                    if (nch == 0) continue;   // no channel with weight: nothing accumulated
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        uint32_t vr[16], vi[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {   // FP32 totals, or int32 totals as their bits
                            vr[i] = MODE == MODE_INT ? (uint32_t)tr[16 * h + i] : __float_as_uint((float)tr[16 * h + i]);
                            vi[i] = MODE == MODE_INT ? (uint32_t)tq[16 * h + i] : __float_as_uint((float)tq[16 * h + i]);
                        }
                        tc::tmem_st16(tlane + 256u * b + col0 + 16 * h, vr);
                        tc::tmem_st16(tlane + 256u * b + 128 + col0 + 16 * h, vi);
                    }
                    tc::tmem_wait_st();
                    if (MODE == MODE_INT)
                        flush_int(a, obase, p, q0, tlane + 256u * b, col0);
                    else
                        drain(a, gr, use_a, use_b, ob, p, q0, tlane, 256u * b, 128u, col0, 2, a.post_scale, nullptr);
                    tc::fence_before();
                    tc::mbar_arrive(&S.acc_empty[b]);
                    ++gcount;
                    continue;
                }
                const int b = dbuf ? (int)(gcount & 1) : 0;
                const uint32_t ph = dbuf ? ((gcount >> 1) & 1) : (gcount & 1);
                const uint32_t re0 = dbuf ? 256u * b : 0u, im_off = dbuf ? 128u : 256u;
                bool ok = tc::mbar_wait(&S.acc_full[b], ph, abort, status, 16, lim);
                if (!__all_sync(0xffffffffu, ok)) break;   // keep the warp's TMEM loads uniform
                tc::fence_after();
                if (cols) {
                    float sp = a.post_scale;
                    const float* qscale = nullptr;
                    if (op == 1) {
                        const float* sc = a.scale + ((long long)w.slot * a.n_groups + g) * n;
                        sp *= (p < n) ? e4m3_scale(__ldg(sc + p)) : 0.0f;
                        qscale = sc;
                    }
                    drain(a, gr, use_a, use_b, ob, p, q0, tlane, re0, im_off, half * 128, 4, sp, qscale);
                }
                tc::fence_before();
                tc::mbar_arrive(&S.acc_empty[b]);
                ++gcount;
            }
        }
    }

    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

template <int MODE>
constexpr size_t tc_smem_bytes()
{
    return 1024 + Ring<MODE>::stages * Ring<MODE>::stage_bytes + sizeof(TcSmem);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

// Tensor map over the operand planes: dims (Kpad, n, slots * N * 2), box (64 B of K,
// 128 rows, 1 plane), 64-byte swizzle, zero fill outside the rows / frames.
cudaError_t make_operand_tmap(CUtensorMap* map, const void* Y, int elem_bytes, long long Kpad, int n,
                              long long planes)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)n, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)Kpad * elem_bytes, (cuuint64_t)Kpad * elem_bytes * n};
    cuuint32_t box[3] = {(cuuint32_t)(ROWB / elem_bytes), (cuuint32_t)TM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                    const_cast<void*>(Y), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map over `rows` rows of `row_words` 32-bit words (rows contiguous), box
// (box_words, box_rows), no swizzle.  A box wider than the rows is allowed for stores: the
// words past a row's end are outside the tensor and not written (a padded shared tile
// stored into dense rows).
cudaError_t make_rows_tmap(CUtensorMap* map, const void* base, int row_words, long long rows, int box_words,
                           int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)row_words, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)row_words * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_words, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_simt_tmap(CUtensorMap* map, const void* Y, long long Kpad, int n, long long planes)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)n, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)Kpad * 4, (cuuint64_t)Kpad * 4 * n};
    cuuint32_t box[3] = {32, 64, 2};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(Y), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int MODE>
cudaError_t launch_tc_kernel(const XLaunch& L, const XItem* items, int n_items, int* counter, int* status, int dbuf,
                             cudaStream_t s)
{
    static bool attr_done = false;
    const size_t smem = tc_smem_bytes<MODE>();
    if (!attr_done) {
        cudaError_t e =
            cudaFuncSetAttribute(xstep_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    if (n_items <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    unsigned int spin = 0;   // x 1000 cycles per bounded wait: the largest of the jobs' limits
    for (int j = 0; j < L.n_jobs; ++j) spin = L.jobs[j].a.spin_limit > spin ? L.jobs[j].a.spin_limit : spin;
    xstep_tc_kernel<MODE><<<n_items < sms ? n_items : sms, NTHREADS, smem, s>>>(L, items, n_items, counter, status,
                                                                                 spin ? spin : tc::kDefaultSpin, dbuf);
    return cudaGetLastError();
}

cudaError_t launch_xstep_tc(const XLaunch& L, const XItem* items, int n_items, int* counter, int* status,
                            cudaStream_t s)
{
    // one kernel mode per launch: every job FP16 / e4m3 (op 0, 1), every job FP16 hi/lo
    // pairs (op 2) or every job integer mode (op 3); the last two on 128-column tiles only
    int mode = -1;
    for (int j = 0; j < L.n_jobs; ++j) {
        const int op = L.jobs[j].op;
        const int mj = op == 2 ? MODE_PAIRS : (op == 3 ? MODE_INT : MODE_ONE);
        if (mode >= 0 && mj != mode) return cudaErrorInvalidValue;
        mode = mj;
        if (mj != MODE_ONE && L.jobs[j].max_cols > TM) return cudaErrorInvalidValue;
        if (mj == MODE_INT && (L.jobs[j].a.seg_frames <= 0 || L.jobs[j].a.seg_frames % 512 != 0 ||
                               L.jobs[j].a.seg_frames > 100 * 512))
            return cudaErrorInvalidValue;   // segments of whole exact chunks, int32-safe
        if (mj == MODE_INT && (L.jobs[j].a.ktile <= 0 || L.jobs[j].a.ktile % 32 != 0 ||
                               L.jobs[j].a.Kpad % L.jobs[j].a.ktile != 0))
            return cudaErrorInvalidValue;   // K-tiled operands: whole k-blocks per tile
    }
    if (mode == MODE_PAIRS) return launch_tc_kernel<MODE_PAIRS>(L, items, n_items, counter, status, 1, s);
    if (mode == MODE_INT) return launch_tc_kernel<MODE_INT>(L, items, n_items, counter, status, 1, s);
    int dbuf = 1;   // double-buffered accumulators when every job's tiles are at most 128 columns wide
    for (int j = 0; j < L.n_jobs; ++j) dbuf &= (L.jobs[j].max_cols <= TM) ? 1 : 0;
    return launch_tc_kernel<MODE_ONE>(L, items, n_items, counter, status, dbuf, s);
}

// Tile list of the tensor-core X-step: for each 128-row block, column windows of
// `window` (256 or 128) starting at its own diagonal (a 256 window at the right edge
// shrinks to 128 when only that much is left).
int build_tc_tiles(int n, int window, int4* out, int cap)
{
    const int wmax = (window == TM) ? TM : TNMAX;
    int k = 0;
    for (int p0 = 0; p0 < n; p0 += TM) {
        for (int q0 = p0; q0 < n; q0 += wmax) {
            const int nq = (n - q0 > TM) ? wmax : TM;
            if (k < cap) out[k] = make_int4(p0, q0, nq, q0 == p0 ? 1 : 0);
            ++k;
        }
    }
    return k;
}

}  // namespace mwax
