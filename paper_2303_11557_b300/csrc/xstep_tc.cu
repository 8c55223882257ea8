// X-step on the 5th-generation tensor cores (tcgen05, TMEM accumulators, TMA operand
// staging) for the FP16 and FP8-e4m3 precision forms, with the same fused epilogue as the
// CUDA-core form: integration over the frames of a slot (Sec. 2.5.2), channel averaging
// (Sec. 2.6) and MWAX_ORDER output (Sec. 2.7).
//
// The complex product C = Y_p conj(Y_q) is four real MMAs on planar operands:
//     Re C = Ar Br^T + Ai Bi^T,      Im C = Ai Br^T - Ar Bi^T
// (the last with the instruction's A-negate bit).  Operands are K-major planes
// Y[slot][c][plane][p][Kpad] loaded by TMA with 128-byte swizzle.
//
// CTA = one 128 x 128 tile of path pairs x one run of output channels x one slot;
// 6 warps: warp 0 issues TMA loads into a 3-stage ring, warp 1 owns TMEM and issues
// the MMAs from one thread, warps 2-5 drain the accumulators (one TMEM lane = one path
// p per thread).  Each ultrafine bin accumulates into one of two TMEM buffers (Re and
// Im, 128 columns each), so the epilogue of bin c overlaps the MMAs of bin c+1.
#include "mwax_internal.cuh"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>

namespace mwax {
namespace {

constexpr int TM = 128;           // paths per tile side
constexpr int STAGES = 3;
constexpr int ROWB = 128;         // bytes per operand row in a stage (one swizzle row)
constexpr int PLANE_BYTES = TM * ROWB;   // 16 KB
constexpr int STAGE_BYTES = 4 * PLANE_BYTES;
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 512;

struct TcSmem {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ long long baseline_of(int i, int j, int T)
{
    return (long long)i * (2 * T - i + 1) / 2 + (j - i);
}

// OP: 0 = FP16 (kind::f16, 16 frames per MMA), 1 = e4m3 (kind::f8f6f4, 32 frames per MMA)
template <int OP>
__global__ void __launch_bounds__(NTHREADS, 1) xstep_tc_kernel(const __grid_constant__ CUtensorMap tmap, const XArgs a)
{
    constexpr int ELEM = (OP == 0) ? 2 : 1;
    constexpr int KB = ROWB / ELEM;           // frames per stage
    constexpr int KSTEP = 32 / ELEM;          // frames per MMA (32 bytes of K)
    constexpr int NSTEPS = KB / KSTEP;        // MMAs per plane pair per stage (4)
    constexpr uint32_t ID = tc::idesc(0, TM, TM, false);
    constexpr uint32_t ID_NEG = tc::idesc(0, TM, TM, true);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // operand ring at a 1024-byte aligned offset, control block after it
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    TcSmem& S = *reinterpret_cast<TcSmem*>(ring + STAGES * STAGE_BYTES);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int2 tile = a.tiles[blockIdx.x];
    const RunInfo run = a.runs[blockIdx.y];
    const int slot = blockIdx.z;
    const int p0 = tile.x * TM, q0 = tile.y * TM;
    const bool diag = tile.x == tile.y;
    const int nkb = (int)((a.klen + KB - 1) / KB);
    const long long lim = (long long)a.spin_limit * 1000LL;   // cycles

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&S.full[s], 1);
            tc::mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&S.acc_full[b], 1);
            tc::mbar_init(&S.acc_empty[b], 128);
        }
        S.abort = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tmap);
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
            const uint32_t bytes = diag ? 2 * PLANE_BYTES : 4 * PLANE_BYTES;
            for (int c = run.c0; c < run.c1 && !*abort; ++c) {
                const BinCoef bc = a.bins[c];
                if (!((bc.ja >= run.j0 && bc.ja < run.j1) || (bc.jb >= run.j0 && bc.jb < run.j1))) continue;
                const int zr = (slot * a.N + c) * 2, zi = zr + 1;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!tc::mbar_wait(&S.empty[stage], phase ^ 1, abort, a.status, 2, lim)) break;
                    unsigned char* st = ring + stage * STAGE_BYTES;
                    tc::mbar_arrive_expect_tx(&S.full[stage], bytes);
                    tc::tma_load_3d(st, &tmap, &S.full[stage], kb * KB, p0, zr);
                    tc::tma_load_3d(st + PLANE_BYTES, &tmap, &S.full[stage], kb * KB, p0, zi);
                    if (!diag) {
                        tc::tma_load_3d(st + 2 * PLANE_BYTES, &tmap, &S.full[stage], kb * KB, q0, zr);
                        tc::tma_load_3d(st + 3 * PLANE_BYTES, &tmap, &S.full[stage], kb * KB, q0, zi);
                    }
                    issued_phase[stage] = (int)phase;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            if (*abort) {
                // let the last load issued into each stage land before the CTA can exit
                for (int s = 0; s < STAGES; ++s) {
                    if (issued_phase[s] < 0) continue;
                    const long long t0 = clock64();
                    while (!tc::mbar_try_wait(&S.full[s], (uint32_t)issued_phase[s]) && clock64() - t0 < lim) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int buf = 0;
            uint32_t aphase = 0;
            const uint32_t sbase = tc::smem_u32(ring);
            bool issued = false;
            for (int c = run.c0; c < run.c1 && !*abort; ++c) {
                const BinCoef bc = a.bins[c];
                if (!((bc.ja >= run.j0 && bc.ja < run.j1) || (bc.jb >= run.j0 && bc.jb < run.j1))) continue;
                if (!tc::mbar_wait(&S.acc_empty[buf], aphase ^ 1, abort, a.status, 4, lim)) break;
                tc::fence_after();
                const uint32_t d_re = tmem + buf * 256, d_im = d_re + 128;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!tc::mbar_wait(&S.full[stage], phase, abort, a.status, 8, lim)) break;
                    tc::fence_after();
                    const uint32_t st = sbase + stage * STAGE_BYTES;
                    const uint64_t dar = tc::sw128_desc(st), dai = tc::sw128_desc(st + PLANE_BYTES);
                    const uint64_t dbr = diag ? dar : tc::sw128_desc(st + 2 * PLANE_BYTES);
                    const uint64_t dbi = diag ? dai : tc::sw128_desc(st + 3 * PLANE_BYTES);
#pragma unroll
                    for (int k = 0; k < NSTEPS; ++k) {
                        const uint64_t off = (uint64_t)(k * 32) >> 4;   // 32 bytes of K per step
                        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                        if (OP == 0) {
                            tc::mma_f16(d_re, dar + off, dbr + off, ID, acc);
                            tc::mma_f16(d_re, dai + off, dbi + off, ID, 1u);
                            tc::mma_f16(d_im, dai + off, dbr + off, ID, acc);
                            tc::mma_f16(d_im, dar + off, dbi + off, ID_NEG, 1u);
                        } else {
                            tc::mma_f8(d_re, dar + off, dbr + off, ID, acc);
                            tc::mma_f8(d_re, dai + off, dbi + off, ID, 1u);
                            tc::mma_f8(d_im, dai + off, dbr + off, ID, acc);
                            tc::mma_f8(d_im, dar + off, dbi + off, ID_NEG, 1u);
                        }
                    }
                    issued = true;
                    tc::mma_commit(&S.empty[stage]);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (*abort) break;
                tc::mma_commit(&S.acc_full[buf]);
                if (++buf == 2) {
                    buf = 0;
                    aphase ^= 1;
                }
            }
            if (*abort && issued) {
                // wait for the MMAs in flight before TMEM is released
                uint64_t* done = &S.acc_full[buf];
                tc::mma_commit(done);
                const long long t0 = clock64();
                while (!tc::mbar_try_wait(done, aphase) && clock64() - t0 < lim) {
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int g = warp & 3;                  // TMEM lane quarter of this warp
        const int row = g * 32 + lane;
        const int p = p0 + row;
        int buf = 0;
        uint32_t aphase = 0;
        for (int c = run.c0; c < run.c1 && !*abort; ++c) {
            const BinCoef bc = a.bins[c];
            const bool use_a = bc.ja >= run.j0 && bc.ja < run.j1;
            const bool use_b = bc.jb >= run.j0 && bc.jb < run.j1;
            if (!use_a && !use_b) continue;
            bool ok = tc::mbar_wait(&S.acc_full[buf], aphase, abort, a.status, 16, lim);
            if (!__all_sync(0xffffffffu, ok)) break;   // keep the warp's TMEM loads uniform
            tc::fence_after();
            float sp = a.post_scale;
            const float* qscale = nullptr;
            if (OP == 1) {
                const float* sc = a.scale + ((long long)slot * a.N + c) * a.n;
                sp *= (p < a.n) ? __ldg(sc + p) : 0.0f;
                qscale = sc;
            }
            const int ti = p >> 1;
            char* obase = a.out + (long long)slot * a.out_stride;
#pragma unroll 1
            for (int ch = 0; ch < TM / 32; ++ch) {
                uint32_t vr[32], vi[32];
                const uint32_t taddr = tmem + ((uint32_t)(g * 32) << 16) + buf * 256 + ch * 32;
                tc::tmem_ld32(taddr, vr);
                tc::tmem_ld32(taddr + 128, vi);
                tc::tmem_wait_ld();
                if (p >= a.n) continue;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int q = q0 + ch * 32 + i;
                    const int tj = q >> 1;
                    if (q < a.n && ti <= tj) {
                        float s = sp;
                        if (OP == 1) s *= __ldg(qscale + q);
                        const float re = __uint_as_float(vr[i]) * s;
                        const float im = (p == q) ? 0.0f : __uint_as_float(vi[i]) * s;
                        const int pol = ((p & 1) << 1) | (q & 1);
                        float2* o =
                            reinterpret_cast<float2*>(obase) + (baseline_of(ti, tj, a.T) * a.M) * 4 + pol;
                        if (use_a) {
                            float2 cur = o[(long long)bc.ja * 4];
                            cur.x = fmaf(bc.ca, re, cur.x);
                            cur.y = fmaf(bc.ca, im, cur.y);
                            o[(long long)bc.ja * 4] = cur;
                        }
                        if (use_b) {
                            float2 cur = o[(long long)bc.jb * 4];
                            cur.x = fmaf(bc.cb, re, cur.x);
                            cur.y = fmaf(bc.cb, im, cur.y);
                            o[(long long)bc.jb * 4] = cur;
                        }
                    }
                }
            }
            tc::fence_before();
            tc::mbar_arrive(&S.acc_empty[buf]);
            if (++buf == 2) {
                buf = 0;
                aphase ^= 1;
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

constexpr size_t tc_smem_bytes() { return 1024 + STAGES * STAGE_BYTES + sizeof(TcSmem); }

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

// Tensor map over the operand planes: dims (Kpad, n, slots * N * 2), box (128 B of K,
// 128 rows, 1 plane), 128-byte swizzle, zero fill outside the rows / frames.
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
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_xstep_tc(int op, const CUtensorMap& map, const XArgs& a, int n_tiles, int n_runs, int slots,
                            cudaStream_t s)
{
    static bool attr_done[2] = {false, false};
    const size_t smem = tc_smem_bytes();
    dim3 grid((unsigned)n_tiles, (unsigned)n_runs, (unsigned)slots);
    if (op == 0) {
        if (!attr_done[0]) {
            cudaError_t e = cudaFuncSetAttribute(xstep_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            attr_done[0] = true;
        }
        xstep_tc_kernel<0><<<grid, NTHREADS, smem, s>>>(map, a);
    } else {
        if (!attr_done[1]) {
            cudaError_t e = cudaFuncSetAttribute(xstep_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            attr_done[1] = true;
        }
        xstep_tc_kernel<1><<<grid, NTHREADS, smem, s>>>(map, a);
    }
    return cudaGetLastError();
}

}  // namespace mwax
