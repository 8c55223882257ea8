// Allocation-free entry point: the FP32 correlation of a small job with every piece of
// device working memory (the X-step operand planes, the F/X tables and a status word) in
// fixed, file-scope device arrays.  It serves callers that cannot call cudaMalloc: a
// process whose device memory is owned by another allocator (a framework's caching pool
// that has reserved the whole GPU), a plug-in whose host application forbids it to
// allocate, or a real-time service that bans allocation after start-up because an
// allocation can block or fail at an arbitrary time.  The F-step and the CUDA-core X-step
// are the library's own launchers, unchanged.
//
// The arrays are part of the library image: every GPU that loads the library holds them
// (about 33.6 MB) until the process exits.  Their host-side names are only stand-ins, so
// host code looks their device addresses up with cudaGetSymbolAddress, once per device and
// context, with that device current, on the first call made there (under a lock; a new
// context after cudaDeviceReset is looked up again).  Device code names them directly: a
// one-block set-up kernel writes the tables from the job's shape passed by value, so no
// host buffer is read after the call returns.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <mutex>

#include "avg_groups.cuh"
#include "mwax_internal.cuh"
#include "plan.cuh"

namespace {

using namespace mwax;

constexpr size_t kScratchBytes = (size_t)32 << 20;   // operand planes of one call
constexpr int kMaxN = 512;
constexpr int kMaxPaths = 64;                          // 32 tiles: one 64 x 64 X-step tile
constexpr int kRunLen = 4;                             // output channels per X-step run
constexpr int kMaxRuns = kMaxN / kRunLen;
constexpr int kMaxDevices = 64;

// Everything but the operands, in one array.
struct Tables {
    float2 tw[kMaxN];               // e^{-2 pi i k / N}
    float gain[kMaxN];              // sqrt of each ultrafine channel's averaging weight
    Group groups[kMaxN];            // at most one group per channel
    RunInfo runs[kMaxRuns];
    int4 tile;                      // the one 64 x 64 path-pair tile
    double delay[3 * kMaxPaths];    // the caller's delay polynomial, when it was in host memory
    int status;                     // 0, or the code of a bounded device wait that gave up
    // scratch of the group builder (set-up kernel, thread 0): in the array rather than in
    // per-thread local memory, which would make the driver grow its local-memory pool
    double w[kMaxN], wsum[kMaxN];
    int fa[kMaxN], fb[kMaxN];
    char seen[kMaxN];
};

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];
__device__ __align__(256) Tables g_tab;

// Shape of the job, and the delay polynomial by value when the caller's copy is in host
// memory (the kernel parameters are captured at launch, so the host copy may go at once).
struct SetupArgs {
    int N, F, keep, dc_excl, n;
    int copy_delay;
    double delay[3 * kMaxPaths];
};

// One block: twiddles and the delay copy by all threads; averaging groups, runs and the
// tile by thread 0 (N <= 512: microseconds); status cleared for this call.
__global__ void __launch_bounds__(256) noalloc_setup_kernel(const SetupArgs a)
{
    for (int k = threadIdx.x; k < a.N; k += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)k / (double)a.N, &s, &c);
        g_tab.tw[k] = make_float2((float)c, (float)s);
    }
    if (a.copy_delay)
        for (int i = threadIdx.x; i < 3 * a.n; i += blockDim.x) g_tab.delay[i] = a.delay[i];
    if (threadIdx.x == 0) {
        const int ng = build_avg_groups(a.N, a.keep, a.F, a.dc_excl, g_tab.gain, g_tab.groups, kMaxN, g_tab.w,
                                        g_tab.fa, g_tab.fb, g_tab.wsum, g_tab.seen);
        // the host ran the same builder on the same shape before launching: ng >= 0 here
        const int M = a.keep / a.F;
        for (int r = 0, j0 = 0; j0 < M; ++r, j0 += kRunLen) {
            RunInfo& run = g_tab.runs[r];
            run.j0 = j0;
            run.j1 = j0 + kRunLen < M ? j0 + kRunLen : M;
            run.g0 = ng;
            run.g1 = 0;
            for (int g = 0; g < ng; ++g) {
                const Group& gr = g_tab.groups[g];
                const bool in = (gr.ja >= run.j0 && gr.ja < run.j1) || (gr.jb >= run.j0 && gr.jb < run.j1);
                if (in) {
                    run.g0 = g < run.g0 ? g : run.g0;
                    run.g1 = g + 1 > run.g1 ? g + 1 : run.g1;
                }
            }
        }
        g_tab.tile = make_int4(0, 0, 64, 1);
        g_tab.status = ng >= 0 ? 0 : MWAX_EINVAL;
    }
}

// After the X-step: if a bounded wait gave up (or the set-up failed), the call's
// visibilities are incomplete, and every weight is set to 0 (no valid data) so the caller
// can tell from the output alone.
__global__ void noalloc_finish_kernel(char* out, long long n_ints, long long vis_set, long long n_weights,
                                      long long stride)
{
    if (g_tab.status == 0) return;
    const long long total = n_ints * n_weights;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long w = i / n_weights, k = i % n_weights;
        reinterpret_cast<float*>(out + w * stride + vis_set)[k] = 0.0f;
    }
}

struct DeviceArrays {
    bool ready;
    unsigned long long ctx;   // the context the addresses belong to
    unsigned char* scratch;
    Tables* tab;
};

// Device address of a member of the table array (host code must not dereference it).
template <typename T>
T* member(Tables* tab, size_t offset)
{
    return reinterpret_cast<T*>(reinterpret_cast<char*>(tab) + offset);
}
std::mutex g_mu;
DeviceArrays g_dev[kMaxDevices];

// Unique id of the calling thread's current context (0 if it cannot be read).
unsigned long long current_context_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
        tried = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur && get_id && get_cur(&ctx) == CUDA_SUCCESS && ctx) get_id(ctx, &id);
    return id;
}

// Device addresses of the arrays on device `dev` (current), looked up once per context.
mwax_status lookup(int dev, DeviceArrays* out)
{
    std::lock_guard<std::mutex> lock(g_mu);   // also guards the driver entry points above
    const unsigned long long ctx = current_context_id();
    DeviceArrays& d = g_dev[dev];
    if (!d.ready || d.ctx != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_error(e, "scratch array address");
        d.scratch = static_cast<unsigned char*>(p);
        if ((e = cudaGetSymbolAddress(&p, g_tab)) != cudaSuccess) return cuda_error(e, "table array address");
        d.tab = static_cast<Tables*>(p);
        d.ctx = current_context_id();   // the look-up made the primary context current if it was not
        d.ready = true;
    }
    *out = d;
    return MWAX_OK;
}

}  // namespace

extern "C" mwax_status mwax_correlate_noalloc(const mwax_plan_desc* desc, const int8_t* voltages,
                                              const double* delay_poly, void* vis_out, void* cuda_stream)
{
    if (!desc || !voltages || !vis_out) return set_error(MWAX_EINVAL, "NULL desc, voltages or vis_out");
    if (((uintptr_t)voltages & 15) || ((uintptr_t)vis_out & 15))
        return set_error(MWAX_EINVAL, "voltages and vis_out must be 16-byte aligned");
    const mwax_plan_desc& d = *desc;
    const int N = d.fft_len, F = d.fine_avg, T = d.n_tiles, n = 2 * T;
    const int bs = d.block_samples ? d.block_samples : kDefaultBlock;
    if (d.precision != MWAX_FP32) return set_error(MWAX_EUNSUPPORTED, "the allocation-free call runs FP32 only");
    if (T < 1 || n > kMaxPaths) return set_error(MWAX_EINVAL, "allocation-free call: 1 to 32 tiles");
    if (N != 32 && N != 64 && N != 128 && N != 256 && N != 512)
        return set_error(MWAX_EUNSUPPORTED, "allocation-free call: fft_len 32, 64, 128, 256 or 512");
    if (F < 1 || N % F) return set_error(MWAX_EINVAL, "fine_avg must divide fft_len");
    if (bs % N) return set_error(MWAX_EINVAL, "block_samples must be a multiple of fft_len");
    if (!(d.int_time_s > 0.0)) return set_error(MWAX_EINVAL, "int_time_s must be > 0");
    if (d.keep_bins != 0 && d.keep_bins != N)
        return set_error(MWAX_EUNSUPPORTED, "allocation-free call: all fft_len bins are kept");
    if (d.sample_rate_hz < 0.0) return set_error(MWAX_EINVAL, "sample_rate_hz must be >= 0");
    const double fs = d.sample_rate_hz > 0.0 ? d.sample_rate_hz : kFs;
    const double isd = d.int_time_s * fs;
    const long long is = llround(isd);
    if (is < 1 || fabs(isd - (double)is) > 1e-9 * isd || is % N)
        return set_error(MWAX_EINVAL, "integration must be a whole number of frames");
    const long long S = d.samples_per_call ? d.samples_per_call : is;
    if (S % is || S % bs) return set_error(MWAX_EINVAL, "samples_per_call must be whole integrations and blocks");
    const long long K = is / N, n_ints = S / is;
    const long long Kpad = (K + kKAlign - 1) / kKAlign * kKAlign;
    const size_t need = (size_t)n_ints * N * 2 * n * Kpad * sizeof(float);
    if (need > kScratchBytes)
        return set_error(MWAX_EINVAL, "allocation-free call: operands exceed the 32 MiB device scratch array");

    // The averaging tables (Sec. 2.6) are validated here with the builder the set-up
    // kernel runs, on stack arrays; only their group count leaves the host.
    const int M = N / F, dc_excl = d.keep_dc ? 0 : 1;
    int ng;
    {
        float gain[kMaxN];
        Group groups[kMaxN];
        double w[kMaxN], wsum[kMaxN];
        int fa[kMaxN], fb[kMaxN];
        char seen[kMaxN];
        ng = build_avg_groups(N, N, F, dc_excl, gain, groups, kMaxN, w, fa, fb, wsum, seen);
        if (ng < 0) return set_error(MWAX_EINVAL, "channel averaging leaves an empty channel");
    }
    const int nr = (M + kRunLen - 1) / kRunLen;

    SetupArgs sa;
    memset(&sa, 0, sizeof sa);
    sa.N = N;
    sa.F = F;
    sa.keep = N;
    sa.dc_excl = dc_excl;
    sa.n = n;
    bool delay_in_device_memory = false;
    if (delay_poly) {
        cudaPointerAttributes at;
        cudaError_t e = cudaPointerGetAttributes(&at, delay_poly);
        if (e != cudaSuccess) return cuda_error(e, "delay_poly attributes");
        delay_in_device_memory = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
        if (!delay_in_device_memory) {   // host memory: read now, into the kernel parameters
            memcpy(sa.delay, delay_poly, sizeof(double) * 3 * n);
            sa.copy_delay = 1;
        }
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(MWAX_EUNSUPPORTED, "device index too large");
    DeviceArrays A;
    mwax_status st = lookup(dev, &A);
    if (st != MWAX_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // tables and status from the job's shape, then the zero padding of the operand planes
    // (the array keeps the previous call's data)
    noalloc_setup_kernel<<<1, 256, 0, s>>>(sa);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "set-up launch");
    if ((e = cudaMemsetAsync(A.scratch, 0, need, s)) != cudaSuccess) return cuda_error(e, "operand clear");

    const long long B = (long long)T * (T + 1) / 2;
    const size_t vis_set = (size_t)B * M * 4 * 8, wts = (size_t)B * 4 * 4;
    if ((e = launch_init_output(static_cast<char*>(vis_out), n_ints, (long long)vis_set, (long long)wts, s)) != cudaSuccess)
        return cuda_error(e, "output init");
    FArgs fa_;
    memset(&fa_, 0, sizeof fa_);
    fa_.volt = voltages;
    fa_.delay = delay_poly ? (delay_in_device_memory ? delay_poly : member<double>(A.tab, offsetof(Tables, delay))) : nullptr;
    fa_.Y = A.scratch;
    fa_.tw = member<float2>(A.tab, offsetof(Tables, tw));
    fa_.gain = member<float>(A.tab, offsetof(Tables, gain));
    fa_.m_begin = 0;
    fa_.n_frames = n_ints * K;
    fa_.n_store = n_ints * K;
    fa_.Kc = K;
    fa_.Kpad = Kpad;
    fa_.n = n;
    fa_.bs = bs;
    fa_.nu = d.sky_freq_hz;
    fa_.fs = fs;
    if ((e = launch_fstep(N, FOUT_F32, fa_, s, 0)) != cudaSuccess) return cuda_error(e, "F-step launch");
    XArgs xa;
    memset(&xa, 0, sizeof xa);
    xa.Y = A.scratch;
    xa.out = static_cast<char*>(vis_out);
    xa.out_stride = (long long)(vis_set + wts);
    xa.Kpad = Kpad;
    xa.klen = K;
    xa.n = n;
    xa.T = T;
    xa.N = N;
    xa.M = M;
    xa.n_groups = ng;
    xa.B = B;
    xa.groups = member<Group>(A.tab, offsetof(Tables, groups));
    xa.runs = member<RunInfo>(A.tab, offsetof(Tables, runs));
    xa.gain = member<float>(A.tab, offsetof(Tables, gain));
    xa.tiles = member<int4>(A.tab, offsetof(Tables, tile));
    xa.post_scale = 1.0f;
    xa.first_store = 1;
    xa.status = member<int>(A.tab, offsetof(Tables, status));
    xa.spin_limit = 2000000;
    CUtensorMap map;   // encoded on the host into the launch parameters: no device memory
    if ((e = make_simt_tmap(&map, A.scratch, Kpad, n, n_ints * N * 2)) != cudaSuccess)
        return cuda_error(e, "operand tensor map");
    if ((e = launch_xstep_simt(map, xa, 1, nr, (int)n_ints, s)) != cudaSuccess) return cuda_error(e, "X-step launch");
    noalloc_finish_kernel<<<8, 256, 0, s>>>(static_cast<char*>(vis_out), n_ints, (long long)vis_set, B * 4,
                                            (long long)(vis_set + wts));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "finish launch");
    return MWAX_OK;
}
