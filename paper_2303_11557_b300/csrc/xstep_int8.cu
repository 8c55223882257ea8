// X-step of the integer mode (no FFT, N = F = 1, 1.28 MHz channels): exact cross-power
// sums of the int8 voltages on the tcgen05 tensor cores.
//
// sm_103a has no integer tensor-core MMA, but every int8 value is exact in FP16 and every
// product of two is exact in FP32.  The MMAs accumulate chunks of 512 samples in FP32
// TMEM: every partial sum of (re re + im im) or (im re - re im) within a chunk is an
// integer of magnitude at most 512 * 2 * 128^2 = 2^24, so it is exact.  After each chunk
// the epilogue converts the sums and adds them into int32 accumulators kept in the other
// half of TMEM; every 100 chunks (51,200 samples: at most 100 * 2^24 < 2^31) the int32
// sums are added into the int64 output.  Result: bit-exact int64 visibilities.
//
// CTA = one 128 x 128 tile of path pairs x one segment of the slot's samples x one slot;
// the segments' int64 sums are combined with 64-bit atomic adds into the zeroed output
// (integer addition, so the result does not depend on their order).  TMEM columns: FP32 chunk sums
// (Re [0,128), Im [128,256)), int32 running sums (Re [256,384), Im [384,512)).
// Warps: 0 = TMA producer, 1 = MMA issuer (+ TMEM owner), 2-9 = epilogue (lane quarter
// warp % 4, column half (warp - 2) / 4).
#include "mwax_internal.cuh"
#include "tc_ptx.cuh"

namespace mwax {
namespace {

constexpr int TM = 128;
constexpr int STAGES = 4;
constexpr int ROWB = 64;                      // 32 FP16 samples per operand row in a stage
constexpr int KF = 32;                        // samples per stage
constexpr int PLANE = TM * ROWB;              // 8 KB
constexpr int STAGE_BYTES = 4 * PLANE;        // Br, Bi, Ar, Ai
constexpr int CHUNK_STAGES = 16;              // 512 samples per exact FP32 chunk
constexpr int FLUSH_CHUNKS = 100;             // 51,200 samples per int32 flush
constexpr int NTHREADS = 320;
constexpr int EPI_THREADS = 256;

struct I8Smem {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full;
    uint64_t acc_empty;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ long long baseline_of(int i, int j, int T)
{
    return (long long)i * (2 * T - i + 1) / 2 + (j - i);
}

__global__ void __launch_bounds__(NTHREADS, 1) xstep_int8_kernel(const __grid_constant__ CUtensorMap tmap, const XArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    I8Smem& S = *reinterpret_cast<I8Smem*>(ring + STAGES * STAGE_BYTES);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int4 tile = a.tiles[blockIdx.x];
    const int slot = blockIdx.z;
    const int p0 = tile.x, q0 = tile.y;
    const bool a_in_b = tile.w != 0;
    // this CTA's segment: stages [kb0, kb1) of the slot, a whole number of chunks
    const int nkb_all = (int)((a.klen + KF - 1) / KF);
    const int seg_stages = (int)a.seg_frames / KF;
    const int kb0 = blockIdx.y * seg_stages;
    const int kb1 = min(nkb_all, kb0 + seg_stages);
    const int nkb = max(0, kb1 - kb0);
    const int nchunks = (nkb + CHUNK_STAGES - 1) / CHUNK_STAGES;
    const long long lim = (long long)a.spin_limit * 1000LL;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&S.full[s], 1);
            tc::mbar_init(&S.empty[s], 1);
        }
        tc::mbar_init(&S.acc_full, 1);
        tc::mbar_init(&S.acc_empty, EPI_THREADS);
        S.abort = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tmap);
    }
    if (warp == 1) {
        tc::tmem_alloc(&S.tmem_base, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem_base;
    volatile int* abort = &S.abort;
    const int zr = slot * 2, zi = zr + 1;   // the single ultrafine channel c = 0

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[STAGES];
            for (int s = 0; s < STAGES; ++s) issued_phase[s] = -1;
            const uint32_t bytes = a_in_b ? 2 * PLANE : 4 * PLANE;
            for (int kb = 0; kb < nkb && !*abort; ++kb) {
                if (!tc::mbar_wait(&S.empty[stage], phase ^ 1, abort, a.status, 2, lim)) break;
                unsigned char* st = ring + stage * STAGE_BYTES;
                uint64_t* fb = &S.full[stage];
                tc::mbar_arrive_expect_tx(fb, bytes);
                const int kx = (kb0 + kb) * KF;
                tc::tma_load_3d(st, &tmap, fb, kx, q0, zr);
                tc::tma_load_3d(st + PLANE, &tmap, fb, kx, q0, zi);
                if (!a_in_b) {
                    tc::tma_load_3d(st + 2 * PLANE, &tmap, fb, kx, p0, zr);
                    tc::tma_load_3d(st + 3 * PLANE, &tmap, fb, kx, p0, zi);
                }
                issued_phase[stage] = (int)phase;
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1;
                }
            }
            if (*abort) {
                for (int s = 0; s < STAGES; ++s) {
                    if (issued_phase[s] < 0) continue;
                    const long long t0 = clock64();
                    while (!tc::mbar_try_wait(&S.full[s], (uint32_t)issued_phase[s]) && clock64() - t0 < lim) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = tc::idesc(0, TM, TM, false), id_neg = tc::idesc(0, TM, TM, true);
            const uint32_t sbase = tc::smem_u32(ring);
            const uint32_t d_re = tmem, d_im = tmem + 128;
            int stage = 0;
            uint32_t phase = 0, cphase = 0;
            bool issued = false;
            int kb = 0;
            for (int ch = 0; ch < nchunks && !*abort; ++ch) {
                if (!tc::mbar_wait(&S.acc_empty, cphase ^ 1, abort, a.status, 4, lim)) break;
                tc::fence_after();
                bool first = true;
                for (int i = 0; i < CHUNK_STAGES && kb < nkb; ++i, ++kb) {
                    if (!tc::mbar_wait(&S.full[stage], phase, abort, a.status, 8, lim)) break;
                    tc::fence_after();
                    const uint32_t st = sbase + stage * STAGE_BYTES;
                    const uint64_t dbr = tc::sw64_desc(st), dbi = tc::sw64_desc(st + PLANE);
                    const uint64_t dar = a_in_b ? dbr : tc::sw64_desc(st + 2 * PLANE);
                    const uint64_t dai = a_in_b ? dbi : tc::sw64_desc(st + 3 * PLANE);
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
                    issued = true;
                    tc::mma_commit(&S.empty[stage]);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (*abort) break;
                tc::mma_commit(&S.acc_full);
                cphase ^= 1;
            }
            if (*abort && issued) {
                tc::mma_commit(&S.acc_full);
                const long long t0 = clock64();
                while (!tc::mbar_try_wait(&S.acc_full, cphase) && clock64() - t0 < lim) {
                }
            }
        }
    } else {
        const int g4 = warp & 3;
        const int half = (warp - 2) >> 2;
        const int p = p0 + g4 * 32 + lane;
        const int ti = p >> 1;
        const uint32_t lane_off = (uint32_t)(g4 * 32) << 16;
        long long* ob = reinterpret_cast<long long*>(a.out + (long long)slot * a.out_stride);
        uint32_t cphase = 0;
        int since_flush = 0;
        for (int ch = 0; ch < nchunks && !*abort; ++ch) {
            bool ok = tc::mbar_wait(&S.acc_full, cphase, abort, a.status, 16, lim);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc::fence_after();
            // fold the chunk's exact FP32 sums into the int32 accumulators
#pragma unroll 1
            for (int cb = 0; cb < 2; ++cb) {
                const int col = half * 64 + cb * 32;
#pragma unroll 1
                for (int part = 0; part < 2; ++part) {   // 0 = Re, 1 = Im
                    uint32_t fv[32], iv[32];
                    tc::tmem_ld32(tmem + lane_off + part * 128 + col, fv);
                    if (since_flush > 0) tc::tmem_ld32(tmem + lane_off + 256 + part * 128 + col, iv);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int x = __float2int_rn(__uint_as_float(fv[i]));
                        iv[i] = (since_flush > 0) ? (uint32_t)((int)iv[i] + x) : (uint32_t)x;
                    }
                    tc::tmem_st32(tmem + lane_off + 256 + part * 128 + col, iv);
                }
            }
            tc::tmem_wait_st();
            tc::fence_before();
            tc::mbar_arrive(&S.acc_empty);
            cphase ^= 1;
            ++since_flush;
            if (since_flush == FLUSH_CHUNKS || ch == nchunks - 1) {
                // add the int32 sums into the int64 MWAX_ORDER output
#pragma unroll 1
                for (int cb = 0; cb < 2; ++cb) {
                    const int col = half * 64 + cb * 32;
                    uint32_t re[32], im[32];
                    tc::tmem_ld32(tmem + lane_off + 256 + col, re);
                    tc::tmem_ld32(tmem + lane_off + 384 + col, im);
                    tc::tmem_wait_ld();
                    if (p < a.n) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int q = q0 + col + i;
                            if (q < a.n && ti <= (q >> 1)) {
                                const int pol = ((p & 1) << 1) | (q & 1);
                                unsigned long long* o = reinterpret_cast<unsigned long long*>(
                                    ob + (baseline_of(ti, q >> 1, a.T) * 4 + pol) * 2);
                                const long long vr = (long long)(int)re[i];
                                const long long vi = (p == q) ? 0LL : (long long)(int)im[i];
                                atomicAdd(o, (unsigned long long)vr);   // two's complement add
                                if (vi != 0) atomicAdd(o + 1, (unsigned long long)vi);
                            }
                        }
                    }
                }
                since_flush = 0;
            }
        }
    }

    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

constexpr size_t i8_smem_bytes() { return 1024 + STAGES * STAGE_BYTES + sizeof(I8Smem); }

}  // namespace

cudaError_t launch_xstep_int8(const CUtensorMap& map, const XArgs& a, int n_tiles, int segments, int slots,
                              cudaStream_t s)
{
    static bool attr_done = false;
    const size_t smem = i8_smem_bytes();
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(xstep_int8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((unsigned)n_tiles, (unsigned)segments, (unsigned)slots);
    xstep_int8_kernel<<<grid, NTHREADS, smem, s>>>(map, a);
    return cudaGetLastError();
}

}  // namespace mwax
