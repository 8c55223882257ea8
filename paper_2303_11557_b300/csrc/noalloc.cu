// Allocation-free entry point: the FP32 correlation of a small plan with every piece of
// device working memory (the X-step operand planes and the F/X tables) in fixed,
// file-scope device arrays, for callers that cannot call cudaMalloc (for example code
// that runs inside a CUDA-graph capture it does not control, in a process whose device
// memory is owned by another allocator, or under a policy that forbids allocation after
// start-up).  It reuses the library's F-step and CUDA-core X-step launchers unchanged.
//
// The arrays are part of the library image: every GPU that loads the library holds them
// (about 33 MB) until the process exits.  Their host-side names are only stand-ins, so
// their device addresses are looked up with cudaGetSymbolAddress once per device, with
// that device current, on the first call made there.
#include <math.h>
#include <string.h>

#include "mwax_internal.cuh"
#include "plan.cuh"

namespace {

using namespace mwax;

constexpr size_t kScratchBytes = (size_t)32 << 20;   // operand planes of one call
constexpr int kMaxN = 512;
constexpr int kMaxPaths = 64;                          // 32 tiles: one 64 x 64 X-step tile
constexpr int kMaxGroups = 2 * kMaxN;
constexpr int kMaxRuns = kMaxN;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];
__device__ __align__(256) float2 g_tw[kMaxN];
__device__ __align__(256) float g_gain[kMaxN];
__device__ __align__(256) Group g_groups[kMaxGroups];
__device__ __align__(256) RunInfo g_runs[kMaxRuns];
__device__ __align__(256) int4 g_tiles[1];
__device__ __align__(256) double g_delay[3 * kMaxPaths];

struct DeviceArrays {
    bool ready;
    unsigned char* scratch;
    float2* tw;
    float* gain;
    Group* groups;
    RunInfo* runs;
    int4* tiles;
    double* delay;
};
DeviceArrays g_dev[kMaxDevices];

template <typename T>
mwax_status symbol_address(T** dst, const void* symbol, const char* what)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, symbol);
    if (e != cudaSuccess) return cuda_error(e, what);
    *dst = static_cast<T*>(p);
    return MWAX_OK;
}

// Device addresses of the arrays on device `dev` (looked up once, with `dev` current).
mwax_status lookup(int dev, DeviceArrays* out)
{
    DeviceArrays& d = g_dev[dev];
    if (!d.ready) {
        mwax_status st;
        if ((st = symbol_address(&d.scratch, g_scratch, "scratch address")) != MWAX_OK) return st;
        if ((st = symbol_address(&d.tw, g_tw, "twiddle address")) != MWAX_OK) return st;
        if ((st = symbol_address(&d.gain, g_gain, "gain address")) != MWAX_OK) return st;
        if ((st = symbol_address(&d.groups, g_groups, "group address")) != MWAX_OK) return st;
        if ((st = symbol_address(&d.runs, g_runs, "run address")) != MWAX_OK) return st;
        if ((st = symbol_address(&d.tiles, g_tiles, "tile address")) != MWAX_OK) return st;
        if ((st = symbol_address(&d.delay, g_delay, "delay address")) != MWAX_OK) return st;
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

    // averaging: gains sqrt(w) per ultrafine channel and groups (Sec. 2.6), in fixed arrays
    const int M = N / F, jc = M / 2, half = F / 2, dc_excl = d.keep_dc ? 0 : 1;
    float gain[kMaxN];
    double w[kMaxN], wsum[kMaxN];
    int fa[kMaxN], fb[kMaxN];
    for (int c = 0; c < N; ++c) {
        w[c] = 0.0;
        fa[c] = fb[c] = -1;
    }
    for (int j = 0; j < M; ++j) {
        wsum[j] = 0.0;
        const long long mid = (long long)(j - jc) * F;
        for (long long u = mid - half; u <= mid + half; ++u) {
            const long long c = u + N / 2;
            if (c < 0 || c >= N) continue;
            double wt = (F % 2 == 0 && (u == mid - half || u == mid + half)) ? 0.5 : 1.0;
            if (dc_excl && F > 1 && u == 0) wt = 0.0;
            if (wt == 0.0) continue;
            w[c] = wt;
            if (fa[c] < 0) fa[c] = j;
            else fb[c] = j;
            wsum[j] += wt;
        }
    }
    Group groups[kMaxGroups];
    RunInfo runs[kMaxRuns];
    int ng = 0;
    bool seen[kMaxN];
    for (int j = 0; j < M; ++j) seen[j] = false;
    for (int c = 0; c < N; ++c) {
        gain[c] = (float)sqrt(w[c]);
        if (w[c] == 0.0) continue;
        if (ng > 0 && groups[ng - 1].ja == fa[c] && groups[ng - 1].jb == fb[c]) {
            groups[ng - 1].c1 = c + 1;
            continue;
        }
        Group& g = groups[ng++];
        g.c0 = c;
        g.c1 = c + 1;
        g.ja = fa[c];
        g.jb = fb[c];
        g.ca = (float)(1.0 / wsum[fa[c]]);
        g.cb = fb[c] >= 0 ? (float)(1.0 / wsum[fb[c]]) : 0.0f;
        g.first_a = !seen[g.ja];
        seen[g.ja] = true;
        g.first_b = 0;
        if (g.jb >= 0) {
            g.first_b = !seen[g.jb];
            seen[g.jb] = true;
        }
    }
    // runs of 4 output channels
    int nr = 0;
    for (int j0 = 0; j0 < M; j0 += 4) {
        RunInfo& r = runs[nr++];
        r.j0 = j0;
        r.j1 = j0 + 4 < M ? j0 + 4 : M;
        r.g0 = ng;
        r.g1 = 0;
        for (int g = 0; g < ng; ++g) {
            const bool in = (groups[g].ja >= r.j0 && groups[g].ja < r.j1) || (groups[g].jb >= r.j0 && groups[g].jb < r.j1);
            if (in) {
                r.g0 = g < r.g0 ? g : r.g0;
                r.g1 = g + 1 > r.g1 ? g + 1 : r.g1;
            }
        }
    }
    float2 tw[kMaxN];
    for (int k = 0; k < N; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)N;
        tw[k] = make_float2((float)cos(a), (float)sin(a));
    }
    const int4 tile = make_int4(0, 0, 64, 1);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(MWAX_EUNSUPPORTED, "device index too large");
    DeviceArrays A;
    mwax_status st = lookup(dev, &A);
    if (st != MWAX_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // tables (copied from host memory: the call returns once they are staged), delays,
    // and the zero padding of the operand planes (the array keeps the previous call's data)
    if ((e = cudaMemcpyAsync(A.tw, tw, sizeof(float2) * N, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A.gain, gain, sizeof(float) * N, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A.groups, groups, sizeof(Group) * ng, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A.runs, runs, sizeof(RunInfo) * nr, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A.tiles, &tile, sizeof(int4), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(A.scratch, 0, need, s)) != cudaSuccess)
        return cuda_error(e, "table upload");
    if (delay_poly && (e = cudaMemcpyAsync(A.delay, delay_poly, sizeof(double) * 3 * n, cudaMemcpyDefault, s)) != cudaSuccess)
        return cuda_error(e, "delay upload");

    const long long B = (long long)T * (T + 1) / 2;
    const size_t vis_set = (size_t)B * M * 4 * 8, wts = (size_t)B * 4 * 4;
    if ((e = launch_init_output(static_cast<char*>(vis_out), n_ints, (long long)vis_set, (long long)wts, s)) != cudaSuccess)
        return cuda_error(e, "output init");
    FArgs fa_;
    memset(&fa_, 0, sizeof fa_);
    fa_.volt = voltages;
    fa_.delay = delay_poly ? A.delay : nullptr;
    fa_.Y = A.scratch;
    fa_.tw = A.tw;
    fa_.gain = A.gain;
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
    xa.groups = A.groups;
    xa.runs = A.runs;
    xa.gain = A.gain;
    xa.tiles = A.tiles;
    xa.post_scale = 1.0f;
    xa.first_store = 1;
    xa.spin_limit = 2000000;
    CUtensorMap map;   // encoded on the host into the launch parameters: no device memory
    if ((e = make_simt_tmap(&map, A.scratch, Kpad, n, n_ints * N * 2)) != cudaSuccess)
        return cuda_error(e, "operand tensor map");
    if ((e = launch_xstep_simt(map, xa, 1, nr, (int)n_ints, s)) != cudaSuccess) return cuda_error(e, "X-step launch");
    return MWAX_OK;
}
