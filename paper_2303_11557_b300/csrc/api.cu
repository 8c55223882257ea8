// C ABI of the MWAX B300 correlator: plan creation and validation, the channel-averaging
// tables, device workspace, and the per-call launch sequence
//   init output -> for each group of integrations: F-step -> X-step.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <queue>
#include <string>
#include <vector>

#include "avg_groups.cuh"
#include "plan.cuh"

using namespace mwax;

namespace {

thread_local std::string g_err;

mwax_status fail(mwax_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
mwax_status fail(mwax_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define MWAX_CUDA(call)                                                                                  \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? MWAX_ENOMEM : MWAX_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                     \
    } while (0)

// Channel-averaging gains and groups (Sec. 2.6) of a plan, from the shared builder.
bool build_groups(int N, int keep, int F, int dc_excl, std::vector<float>& gain, std::vector<Group>& groups)
{
    const int M = keep / F;
    std::vector<double> w(N), wsum(M);
    std::vector<int> fa(N), fb(N);
    std::vector<char> seen(M);
    gain.assign(N, 0.0f);
    groups.assign(N, Group{});
    const int ng = build_avg_groups(N, keep, F, dc_excl, gain.data(), groups.data(), N, w.data(), fa.data(), fb.data(),
                                    wsum.data(), seen.data());
    if (ng < 0) return false;
    groups.resize(ng);
    return true;
}

int prec_elem_bytes(int prec)
{
    switch (prec) {
        case MWAX_FP32: return 4;
        case MWAX_FP16: return 2;
        case MWAX_FP8: return 1;   // e4m3 operands (F-step variant 2's FP16 staging comes with that variant)
        case MWAX_INT8: return 2;   // int8 held exactly in FP16 operands
        case MWAX_FP16X3: return 4;   // an FP16 hi/lo pair per value
        default: return 0;
    }
}

void free_plan(mwax_plan* p)
{
    if (!p) return;
    cudaFree(p->Y);
    cudaFree(p->Y16);
    cudaFree(p->Yt);
    cudaFree(p->tw);
    cudaFree(p->delay);
    cudaFree(p->groups);
    cudaFree(p->gain);
    cudaFree(p->chan_group);
    cudaFree(p->amax);
    cudaFree(p->gain8);
    cudaFree(p->amax_static);
    cudaFree(p->runs);
    cudaFree(p->tiles);
    cudaFree(p->status);
    cudaFree(p->counter);
    for (auto& h : p->hbuf) {
        cudaFree(h.dvolt);
        cudaFree(h.dout);
        for (auto e : h.copied) cudaEventDestroy(e);
        if (h.free_ev) cudaEventDestroy(h.free_ev);
        if (h.done_ev) cudaEventDestroy(h.done_ev);
        if (h.out_ev) cudaEventDestroy(h.out_ev);
    }
    if (p->back_stream) cudaStreamDestroy(p->back_stream);
    cudaFree(p->d_table);
    cudaFree(p->d_flags);
    for (auto& it : p->item_lists) cudaFree(it.items);
    for (auto e : p->ev_pool) cudaEventDestroy(e);
    for (auto& u : p->ev_used) {
        cudaEventDestroy(u.second.first);
        cudaEventDestroy(u.second.second);
    }
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    delete p;
}

mwax_status validate(const mwax_plan_desc& d, mwax_plan& p)
{
    if (d.n_tiles < 1) return fail(MWAX_EINVAL, "n_tiles must be >= 1 (got %d)", d.n_tiles);
    if (d.fft_len < 1) return fail(MWAX_EINVAL, "fft_len must be >= 1 (got %d)", d.fft_len);
    if (d.fine_avg < 1 || d.fft_len % d.fine_avg)
        return fail(MWAX_EINVAL, "fine_avg (%d) must divide fft_len (%d)", d.fine_avg, d.fft_len);
    const int bs = d.block_samples ? d.block_samples : kDefaultBlock;
    if (bs < 1 || bs % d.fft_len)
        return fail(MWAX_EINVAL, "block_samples (%d) must be a multiple of fft_len (%d)", bs, d.fft_len);
    if (!(d.int_time_s > 0.0)) return fail(MWAX_EINVAL, "int_time_s must be > 0");
    if (d.sample_rate_hz < 0.0 || !(d.sample_rate_hz < 1e12))
        return fail(MWAX_EINVAL, "sample_rate_hz must be >= 0 (0 = 1.28 MS/s)");
    const double fs = d.sample_rate_hz > 0.0 ? d.sample_rate_hz : kFs;
    const int keep = d.keep_bins ? d.keep_bins : d.fft_len;
    if (keep < 1 || keep > d.fft_len || keep % d.fine_avg)
        return fail(MWAX_EINVAL, "keep_bins (%d) must be in [1, fft_len] and a multiple of fine_avg (%d)", keep,
                    d.fine_avg);
    const double int_samples_d = d.int_time_s * fs;
    const long long int_samples = llround(int_samples_d);
    if (fabs(int_samples_d - (double)int_samples) > 1e-9 * std::max(1.0, int_samples_d) || int_samples < 1)
        return fail(MWAX_EINVAL, "int_time_s * Fs must be a whole number of samples");
    if (int_samples % d.fft_len)
        return fail(MWAX_EINVAL, "integration (%lld samples) must be a whole number of %d-sample frames",
                    int_samples, d.fft_len);
    const long long S = d.samples_per_call ? d.samples_per_call : int_samples;
    if (S < 1 || S % int_samples)
        return fail(MWAX_EINVAL, "samples_per_call (%lld) must be a multiple of the integration (%lld)", S,
                    int_samples);
    if (S % bs) return fail(MWAX_EINVAL, "samples_per_call (%lld) must be a multiple of block_samples (%d)", S, bs);
    if (d.precision < MWAX_FP32 || d.precision > MWAX_FP16X3)
        return fail(MWAX_EINVAL, "unknown precision %d", d.precision);
    if (d.precision == MWAX_INT8 && (d.fft_len != 1 || d.fine_avg != 1))
        return fail(MWAX_EINVAL, "MWAX_INT8 needs fft_len = fine_avg = 1 (no FFT)");
    if (!fft_len_supported(d.fft_len)) return fail(MWAX_EUNSUPPORTED, "fft_len %d is not built", d.fft_len);
    if (d.fft_len > 1 && d.fft_len < 16) return fail(MWAX_EUNSUPPORTED, "fft_len %d is not built", d.fft_len);

    p.desc = d;
    p.T = d.n_tiles;
    p.n = 2 * d.n_tiles;
    p.N = d.fft_len;
    p.F = d.fine_avg;
    p.keep = keep;
    p.fs = fs;
    p.M = keep / d.fine_avg;
    p.bs = bs;
    p.prec = d.precision;
    p.dc_excl = d.keep_dc ? 0 : 1;
    p.nu = d.sky_freq_hz;
    p.K = int_samples / d.fft_len;
    p.S = S;
    p.n_ints = S / int_samples;
    p.B = (long long)p.T * (p.T + 1) / 2;
    p.n_blocks = S / bs;
    if (p.prec == MWAX_INT8) {
        p.vis_set_bytes = (size_t)p.B * 4 * 16;
    } else {
        p.vis_set_bytes = (size_t)p.B * p.M * 4 * 8;
    }
    p.weights_bytes = (size_t)p.B * 4 * 4;
    p.int_stride = p.vis_set_bytes + p.weights_bytes;
    p.input_bytes = (size_t)p.n_blocks * p.n * bs * 2;
    p.elem_bytes = prec_elem_bytes(p.prec);
    return MWAX_OK;
}

}  // namespace

namespace mwax {

// (Re)build the X-step tile list and the runs of output channels.  run_len = output
// channels per work item (0: chosen from the grid size), window = width of a tensor-core
// tile's column window (128 or 256).  Drops cached item lists.
// Ultrafine channels (with non-zero weight) that a run [j0, j1) of output channels
// consumes: every group feeding one of them, shared boundary groups included.
int run_bins(const mwax_plan& p, int j0, int j1)
{
    int bins = 0;
    for (const Group& gr : p.h_groups) {
        if (!((gr.ja >= j0 && gr.ja < j1) || (gr.jb >= j0 && gr.jb < j1))) continue;
        for (int c = gr.c0; c < gr.c1; ++c) bins += p.h_gain[c] > 0.0f;
    }
    return bins;
}

// Run length of the X-step: short runs make more work items (a fuller last wave) but
// recompute the boundary channels that neighbouring runs share.  Each candidate's items
// (cost = channels consumed x the tile's relative cost, + a fixed epilogue share) are
// placed longest first on the resident CTA slots (CUDA cores: the sorted work list as
// launched; tensor cores: one persistent CTA per SM claiming the sorted list); the
// candidate whose launches finish first wins.
int model_run_len(const mwax_plan& p, const std::vector<int4>& tiles)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int resident = p.tensor_cores ? sms : sms * simt_resident_ctas();
    // relative cost of a tile, as in plan_items
    auto tile_cost = [&](const int4& tl) {
        return p.tensor_cores ? tl.z / 256.0 * (tl.w ? 1.0 : 1.25) : (tl.w ? 23.0 / 32.0 : 1.0);
    };
    std::vector<long long> launch_slots;
    for (long long w0 = 0; w0 < p.n_ints; w0 += p.slots)
        for (int ch = 0; ch < p.chunks; ++ch) launch_slots.push_back(std::min(p.slots, p.n_ints - w0));
    std::vector<int> cand;
    for (int rl = 1; rl <= 8; ++rl) cand.push_back(rl);
    for (int rl = 12; rl <= 32; rl += 4) cand.push_back(rl);
    for (int rl = 48; rl < p.M; rl *= 2) cand.push_back(rl);
    cand.push_back(p.M);
    int best = p.M;
    double best_t = 1e300;
    for (int rl : cand) {
        if (rl > p.M) continue;
        std::vector<double> run_cost;
        for (int j0 = 0; j0 < p.M; j0 += rl) run_cost.push_back(run_bins(p, j0, std::min(p.M, j0 + rl)) + 0.25);
        const double ctas = (double)run_cost.size() * tiles.size() * launch_slots[0];
        if (ctas > 400000.0 && rl < p.M) continue;   // far more CTAs than the GPU holds
        double t = 0.0;
        for (long long ns : launch_slots) {
            std::vector<double> c;
            for (long long sl = 0; sl < ns; ++sl)
                for (double rc : run_cost)
                    for (const int4& tl : tiles) c.push_back(rc * tile_cost(tl));
            std::sort(c.begin(), c.end(), std::greater<double>());
            std::priority_queue<double, std::vector<double>, std::greater<double>> q;
            for (int k = 0; k < resident; ++k) q.push(0.0);
            double end = 0.0;
            for (double w : c) {
                const double f = q.top() + w;
                q.pop();
                q.push(f);
                end = std::max(end, f);
            }
            t += end;
        }
        if (t < best_t * 0.999) {
            best_t = t;
            best = rl;
        }
    }
    return best;
}

mwax_status configure_x(mwax_plan& p, int run_len_req, int window)
{
    for (auto& it : p.item_lists) cudaFree(it.items);
    p.item_lists.clear();
    cudaFree(p.tiles);
    cudaFree(p.runs);
    p.tiles = nullptr;
    p.runs = nullptr;
    const std::vector<Group>& groups = p.h_groups;

    // tiles of path pairs on or above the diagonal
    std::vector<int4> tiles;
    if (p.prec == MWAX_INT8) {
        for (int i = 0; i < p.n; i += 128)
            for (int j = i; j < p.n; j += 128) tiles.push_back(make_int4(i, j, 128, i == j ? 1 : 0));
    } else if (p.tensor_cores) {
        if (p.prec == MWAX_FP16X3) window = 128;   // the pair form's register totals hold 128 columns
        tiles.resize(build_tc_tiles(p.n, window, nullptr, 0));
        build_tc_tiles(p.n, window, tiles.data(), (int)tiles.size());
    } else {
        for (int i = 0; i < p.n; i += 64)
            for (int j = i; j < p.n; j += 64) tiles.push_back(make_int4(i, j, 64, i == j ? 1 : 0));
    }
    p.n_tiles = (int)tiles.size();
    p.h_tiles = tiles;
    MWAX_CUDA(cudaMalloc(&p.tiles, sizeof(int4) * tiles.size()));
    MWAX_CUDA(cudaMemcpy(p.tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice));

    // runs of output channels: by default the run length whose longest-first schedule
    // finishes first (model_run_len); the integer mode has one output channel
    int run_len = run_len_req;
    if (run_len <= 0 && p.prec != MWAX_INT8) run_len = model_run_len(p, tiles);
    if (run_len <= 0) {
        const long long items_wo_runs = (long long)p.n_tiles * p.slots;
        const long long want_items = p.tensor_cores ? 6LL * 148 : 8LL * 148;
        const int want_runs = (int)std::max<long long>(1, (want_items + items_wo_runs - 1) / items_wo_runs);
        run_len = std::max(4, (p.M + want_runs - 1) / want_runs);
    }
    run_len = std::max(1, std::min(run_len, p.M));
    p.run_len = run_len;
    std::vector<RunInfo> runs;
    for (int j0 = 0; j0 < p.M; j0 += run_len) {
        RunInfo r;
        r.j0 = j0;
        r.j1 = std::min(p.M, j0 + run_len);
        r.g0 = p.n_groups;
        r.g1 = 0;
        for (int g = 0; g < p.n_groups; ++g) {
            const Group& gr = groups[g];
            const bool in = (gr.ja >= r.j0 && gr.ja < r.j1) || (gr.jb >= r.j0 && gr.jb < r.j1);
            if (in) {
                r.g0 = std::min(r.g0, g);
                r.g1 = std::max(r.g1, g + 1);
            }
        }
        runs.push_back(r);
    }
    p.n_runs = (int)runs.size();
    p.h_runs = runs;
    p.window = window;
    MWAX_CUDA(cudaMalloc(&p.runs, sizeof(RunInfo) * runs.size()));
    MWAX_CUDA(cudaMemcpy(p.runs, runs.data(), sizeof(RunInfo) * runs.size(), cudaMemcpyHostToDevice));
    return MWAX_OK;
}

}  // namespace mwax

namespace {

// FP16 / FP8 operands: power-of-two pre-scale keeping |Re X|, |Im X| <= 181 N g (int8
// magnitude 128 sqrt 2 summed over N samples, times a passband gain g <= 2) below 2^15;
// undone exactly after the MMA.  Fixed at plan creation, so de-ripple gains can change
// without touching launch arguments captured in graphs.
constexpr double kMaxPassband = 2.0;

// The F-step's per-channel gains as the device holds them: sqrt(w_c) x passband gain x the
// power-of-two pre-scale of the FP16 operand forms (1 otherwise), one multiply per value.
//
// FP8 form: the F-step writes e4m3 directly with a static scale per channel group g,
// s_g = A_g / 448 with A_g = 181.02 N max_{c in g} gain_c (pre-scaled), the bound on any
// |Re X|, |Im X| of the group: no value saturates, and the values of an ordinary sky sit
// well inside e4m3's normal range, whose relative step (2^-3) is the same at any scale.
mwax_status upload_gains(mwax_plan& p)
{
    std::vector<float> g(p.N);
    for (int c = 0; c < p.N; ++c) g[c] = p.h_gain[c] * p.out_scale;   // exact: a power of two
    MWAX_CUDA(cudaMemcpy(p.gain, g.data(), sizeof(float) * p.N, cudaMemcpyHostToDevice));
    if (p.prec == MWAX_FP8) {
        std::vector<float> g8(p.N, 0.0f), a8(p.n_groups, 448.0f);
        for (int gi = 0; gi < p.n_groups; ++gi) {
            const Group& gr = p.h_groups[gi];
            double gmax = 0.0;
            for (int c = gr.c0; c < gr.c1; ++c) gmax = std::max(gmax, (double)g[c]);
            if (gmax <= 0.0) continue;
            const double A = 181.02 * p.N * gmax;
            a8[gi] = (float)A;
            for (int c = gr.c0; c < gr.c1; ++c) g8[c] = (float)((double)g[c] * 448.0 / A);
        }
        if (!p.gain8) MWAX_CUDA(cudaMalloc(&p.gain8, sizeof(float) * p.N));
        if (!p.amax_static) MWAX_CUDA(cudaMalloc(&p.amax_static, sizeof(float) * std::max(1, p.n_groups)));
        MWAX_CUDA(cudaMemcpy(p.gain8, g8.data(), sizeof(float) * p.N, cudaMemcpyHostToDevice));
        MWAX_CUDA(cudaMemcpy(p.amax_static, a8.data(), sizeof(float) * p.n_groups, cudaMemcpyHostToDevice));
    }
    return MWAX_OK;
}

void set_prescale(mwax_plan& p)
{
    if (p.prec != MWAX_FP16 && p.prec != MWAX_FP8 && p.prec != MWAX_FP16X3) return;
    int k = 0;
    while (181.02 * p.N * kMaxPassband / (double)(1 << k) > 32768.0) ++k;
    p.out_scale = ldexpf(1.0f, -k);
    p.post_scale = ldexpf(1.0f, 2 * k);
}

// Copy into plan-owned device memory in stream order; a pinned host source is waited for
// so that the caller may reuse it when the call returns (pageable sources are staged by
// the copy itself, device sources are read in stream order).
mwax_status copy_in(mwax_plan* p, void* dst, const void* src, size_t bytes)
{
    MWAX_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, p->stream));
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeHost)
        MWAX_CUDA(cudaStreamSynchronize(p->stream));
    cudaGetLastError();   // an unregistered pointer is not an error here
    return MWAX_OK;
}

mwax_status setup(mwax_plan& p)
{
    MWAX_CUDA(cudaGetDevice(&p.device));

    // workspace: operand slots
    const size_t limit = p.desc.workspace_limit ? p.desc.workspace_limit : ((size_t)16 << 30);
    // integer mode: frames come in whole K tiles
    const long long align = (p.prec == MWAX_INT8) ? kIntKTile : kKAlign;
    p.ktile = (p.prec == MWAX_INT8) ? kIntKTile : 0;
    const long long Kpad_full = (p.K + align - 1) / align * align;
    const size_t per_slot = (size_t)p.N * 2 * p.n * Kpad_full * p.elem_bytes;
    if (per_slot <= limit) {
        p.slots = std::min<long long>(p.n_ints, (long long)(limit / per_slot));
        p.Kc = p.K;
        p.Kpad = Kpad_full;
        p.chunks = 1;
    } else {
        const size_t per_frame = (size_t)p.N * 2 * p.n * p.elem_bytes;
        long long kc = (long long)(limit / per_frame) / align * align;
        if (kc < align) return fail(MWAX_ENOMEM, "workspace_limit too small for one %lld-frame chunk", align);
        p.slots = 1;
        p.Kc = kc;
        p.Kpad = kc;
        p.chunks = (int)((p.K + kc - 1) / kc);
    }
    const size_t elems = (size_t)p.slots * p.N * 2 * p.n * p.Kpad;
    p.Y_bytes = elems * p.elem_bytes;
    MWAX_CUDA(cudaMalloc(&p.Y, p.Y_bytes));
    MWAX_CUDA(cudaMemset(p.Y, 0, p.Y_bytes));
    // N = 1280, 6400 with FP16 operands out: the 128-row tensor-core F-step by default (the
    // fastest measured there), with its one-slot scratch
    if (fstep_f128_supported(p.N) && (p.prec == MWAX_FP16 || p.prec == MWAX_FP8)) {
        const mwax_status st = ensure_fstep_scratch(&p, 3);
        if (st != MWAX_OK) return st;
        p.fvariant = 3;
    }

    // twiddles e^{-2 pi i k / N}, rounded from FP64
    std::vector<float2> tw(p.N);
    for (int k = 0; k < p.N; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)p.N;
        tw[k] = make_float2((float)cos(a), (float)sin(a));
    }
    MWAX_CUDA(cudaMalloc(&p.tw, sizeof(float2) * p.N));
    MWAX_CUDA(cudaMemcpy(p.tw, tw.data(), sizeof(float2) * p.N, cudaMemcpyHostToDevice));
    MWAX_CUDA(cudaMalloc(&p.delay, sizeof(double) * 3 * p.n));

    // averaging: per-channel gains (applied in the F-step) and channel groups
    std::vector<float> gain;
    std::vector<Group> groups;
    if (!build_groups(p.N, p.keep, p.F, p.dc_excl, gain, groups))
        return fail(MWAX_EINVAL, "channel averaging with fscrunch %d leaves an empty channel", p.F);
    p.n_groups = (int)groups.size();
    MWAX_CUDA(cudaMalloc(&p.gain, sizeof(float) * p.N));
    MWAX_CUDA(cudaMalloc(&p.groups, sizeof(Group) * groups.size()));
    MWAX_CUDA(cudaMemcpy(p.groups, groups.data(), sizeof(Group) * groups.size(), cudaMemcpyHostToDevice));
    p.h_groups = groups;
    p.h_gain = gain;
    p.h_avg_gain = gain;
    p.passband.assign(p.N, 1.0f);

    // FP16 operands: power-of-two pre-scale keeping |Re X|, |Im X| <= 181 N (int8
    // magnitude 128 sqrt 2 summed over N samples) below 2^15; undone exactly after the MMA
    set_prescale(p);
    {
        mwax_status st = upload_gains(p);
        if (st != MWAX_OK) return st;
    }
    p.tensor_cores = p.prec != MWAX_FP32;
    if (p.prec == MWAX_FP8) {
        std::vector<int> cg(p.N, -1);
        for (int g = 0; g < p.n_groups; ++g)
            for (int c = groups[g].c0; c < groups[g].c1; ++c)
                if (gain[c] > 0.0f) cg[c] = g;
        MWAX_CUDA(cudaMalloc(&p.chan_group, sizeof(int) * p.N));
        MWAX_CUDA(cudaMemcpy(p.chan_group, cg.data(), sizeof(int) * p.N, cudaMemcpyHostToDevice));
        p.amax_bytes = sizeof(float) * (size_t)p.slots * p.n_groups * p.n;
        MWAX_CUDA(cudaMalloc(&p.amax, p.amax_bytes));
    }
    if (p.prec == MWAX_FP32)
        MWAX_CUDA(make_simt_tmap(&p.tmap, p.Y, p.Kpad, p.n, p.slots * p.N * 2));
    else if (p.prec == MWAX_FP16X3)   // FP16 rows of 2 Kpad: hi frames, then lo frames
        MWAX_CUDA(make_operand_tmap(&p.tmap, p.Y, 2, 2 * p.Kpad, p.n, p.slots * p.N * 2));
    else if (p.prec == MWAX_INT8)     // rows of one K tile: planes [slot][K tile][re/im]
        MWAX_CUDA(make_operand_tmap(&p.tmap, p.Y, 2, p.ktile, p.n, p.slots * (p.Kpad / p.ktile) * 2));
    else
        MWAX_CUDA(make_operand_tmap(&p.tmap, p.Y, p.prec == MWAX_FP8 ? 1 : 2, p.Kpad, p.n, p.slots * p.N * 2));

    {
        mwax_status st = configure_x(p, 0, p.prec == MWAX_INT8 ? 128 : 256);
        if (st != MWAX_OK) return st;
    }

    MWAX_CUDA(cudaMalloc(&p.counter, sizeof(int)));
    MWAX_CUDA(cudaMalloc(&p.status, sizeof(int)));
    MWAX_CUDA(cudaMemset(p.status, 0, sizeof(int)));
    return MWAX_OK;
}

}  // namespace

namespace mwax {

// Work items of one X launch of plan p (as job `job`) with their sort key; the tiles'
// relative costs: tensor cores, the B window width with A rows outside it costing extra;
// CUDA cores, a diagonal tile skipping 9 of its 32 register sub-blocks.
// Tensor cores: the key is the cost of the item's run of output channels (active
// ultrafine channels x frame blocks) and within each (slot, run) the tiles are listed most
// expensive first, so after the stable sort the big runs start first and all tiles of one
// (slot, run) sit side by side: the CTAs running together stream the same channels of the
// same integration, which then come from L2 instead of HBM (the persistent kernel is fed by
// HBM; this ordering took 4-5 % off its time).  CUDA cores (bound by FMA issue, not by
// HBM): the key is the item's own cost, longest first.
// Integer mode: samples per K segment of the tensor-core X-step (one work item each): the
// slot's samples split evenly into segments of whole 512-sample chunks, at most 100
// chunks (51,200 samples) each so the int32 register sums cannot overflow.
long long int8_seg_frames(long long klen)
{
    const long long chunks = std::max<long long>(1, (klen + 511) / 512);
    const long long nseg = (chunks + 99) / 100;
    return (chunks + nseg - 1) / nseg * 512;
}

void plan_items(const mwax_plan& p, int job, long long nslots, long long klen, std::vector<std::pair<double, XItem>>& out)
{
    if (p.prec == MWAX_INT8) {
        // (slot, segment) groups with all tiles side by side (they stream the same samples
        // through L2); the key is the segment's length, so a short last segment goes last
        const long long seg = int8_seg_frames(klen);
        const int nseg = (int)((klen + seg - 1) / seg);
        for (long long sl = 0; sl < nslots; ++sl)
            for (int sg = 0; sg < nseg; ++sg)
                for (int t = 0; t < p.n_tiles; ++t)
                    out.push_back({(double)std::min(seg, klen - sg * seg), XItem{job, t, sg, (int)sl}});
        return;
    }
    const int KF = (p.prec == MWAX_FP8) ? 64 : 32;
    const double nkb = (double)((klen + KF - 1) / KF);
    std::vector<int> bins(p.n_runs, 0);
    for (int r = 0; r < p.n_runs; ++r) {
        const RunInfo& run = p.h_runs[r];
        for (int g = run.g0; g < run.g1; ++g) {
            const Group& gr = p.h_groups[g];
            if (!((gr.ja >= run.j0 && gr.ja < run.j1) || (gr.jb >= run.j0 && gr.jb < run.j1))) continue;
            for (int c = gr.c0; c < gr.c1; ++c) bins[r] += p.h_gain[c] > 0.0f;
        }
    }
    std::vector<int> tiles(p.n_tiles);
    std::vector<double> tcost(p.n_tiles);
    for (int t = 0; t < p.n_tiles; ++t) {
        const int4 tl = p.h_tiles[t];
        tiles[t] = t;
        tcost[t] = tl.z * (p.tensor_cores ? (tl.w ? 1.0 : 1.25) : (tl.w ? 23.0 / 32.0 : 1.0));
    }
    std::stable_sort(tiles.begin(), tiles.end(), [&](int x, int y) { return tcost[x] > tcost[y]; });
    for (long long sl = 0; sl < nslots; ++sl)
        for (int r = 0; r < p.n_runs; ++r)
            for (int t : tiles)
                out.push_back({p.tensor_cores ? bins[r] * nkb + 1.0 : bins[r] * nkb * tcost[t] + 1.0,
                               XItem{job, t, r, (int)sl}});
}

// Items in decreasing key (stable): claimed or launched in this order.
void sort_items(std::vector<std::pair<double, XItem>>& v, std::vector<XItem>& order)
{
    std::stable_sort(v.begin(), v.end(), [](const std::pair<double, XItem>& a, const std::pair<double, XItem>& b) {
        return a.first > b.first;
    });
    order.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) order[i] = v[i].second;
}

}  // namespace mwax

namespace {

int sm_count()
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Device item list of a single-plan launch, most expensive first (cached per slot count
// and frames).
mwax_status single_items(mwax_plan* p, long long nslots, long long klen, XItem** items, int* n)
{
    const long long key = nslots * 1000003LL + klen;
    for (auto& e : p->item_lists)
        if (e.key == key) {
            *items = e.items;
            *n = e.n;
            return MWAX_OK;
        }
    std::vector<std::pair<double, XItem>> v;
    plan_items(*p, 0, nslots, klen, v);
    std::vector<XItem> order;
    sort_items(v, order);
    XItem* d = nullptr;
    MWAX_CUDA(cudaMalloc(&d, sizeof(XItem) * std::max<size_t>(1, order.size())));
    MWAX_CUDA(cudaMemcpy(d, order.data(), sizeof(XItem) * order.size(), cudaMemcpyHostToDevice));
    p->item_lists.push_back({key, d, (int)order.size()});
    *items = d;
    *n = (int)order.size();
    return MWAX_OK;
}

cudaEvent_t take_event(mwax_plan* p)
{
    if (!p->ev_pool.empty()) {
        cudaEvent_t e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one launch of `stage` with events when timing is on; count its kernels either way.
template <typename F>
cudaError_t timed(mwax_plan* p, int stage, cudaStream_t s, F&& launch)
{
    const long long x0 = extra_launches();
    cudaError_t e;
    if (!p->timing) {
        e = launch();
    } else {
        cudaEvent_t a = take_event(p), b = take_event(p);
        cudaEventRecord(a, s);
        e = launch();
        cudaEventRecord(b, s);
        p->ev_used.push_back({stage, {a, b}});
    }
    p->launches[stage] += 1 + (extra_launches() - x0);
    return e;
}

// Launch groups of one call.  max_slots > 0 (host-input path) splits each group of
// whole integrations into groups of at most max_slots, so the F- and X-steps of the
// first integrations run while the later ones are still being copied in.
std::vector<LaunchGroup> call_groups(const mwax_plan* p, long long max_slots)
{
    std::vector<LaunchGroup> v = plan_groups(p);
    if (max_slots <= 0 || p->chunks != 1) return v;
    std::vector<LaunchGroup> out;
    for (const LaunchGroup& g : v)
        for (long long s0 = 0; s0 < g.nslots; s0 += max_slots) {
            LaunchGroup h = g;
            h.w0 = g.w0 + s0;
            h.nslots = std::min(max_slots, g.nslots - s0);
            h.nframes = h.nslots * p->K;
            h.m_begin = h.w0 * p->K;
            out.push_back(h);
        }
    return out;
}

mwax_status enqueue(mwax_plan* p, const int8_t* volt, bool have_delay, char* out, cudaEvent_t* wait_events,
                    long long events_per_block, long long max_slots = 0)
{
    cudaStream_t s = p->stream;
    mwax_status st = enqueue_init(p, out, s);
    if (st != MWAX_OK) return st;
    for (const LaunchGroup& g : call_groups(p, max_slots)) {
        if (wait_events) {
            // host-input path: wait for the copy of the last block this launch reads
            const long long last_sample = (g.m_begin + g.nframes) * p->N - 1;
            const long long blk = last_sample / p->bs;
            MWAX_CUDA(cudaStreamWaitEvent(s, wait_events[blk / events_per_block], 0));
        }
        st = enqueue_fstep(p, g, volt, have_delay, s);
        if (st != MWAX_OK) return st;
        st = enqueue_xstep_single(p, g, make_xargs(p, g, out), s);
        if (st != MWAX_OK) return st;
    }
    return MWAX_OK;
}

mwax_status load_delay(mwax_plan* p, const double* delay_poly)
{
    if (!delay_poly) return MWAX_OK;
    MWAX_CUDA(cudaMemcpyAsync(p->delay, delay_poly, sizeof(double) * 3 * p->n, cudaMemcpyDefault, p->stream));
    return MWAX_OK;
}

// One host-memory call on staging set b: the voltages go to the device in 16 chunks on the
// copy stream (after the set's previous call has read it), each launch group of the
// correlation waits for the chunks it reads, and the result is copied back on the
// read-back stream (the set's next correlation waits until that copy is done).  split: launch groups of a quarter of the plan's (the synchronous call, whose
// own upload is all there is to overlap with); otherwise the plan's groups (streaming:
// the next call's upload overlaps this correlation).  Returns once all is enqueued.
mwax_status host_call(mwax_plan* p, const int8_t* volt, const double* delay_poly, void* vis_out, int b, bool split)
{
    if (!p || !volt || !vis_out) return fail(MWAX_EINVAL, "NULL plan, voltages or vis_out");
    if (p->prec == MWAX_INT8 && delay_poly) return fail(MWAX_EINVAL, "MWAX_INT8 takes no delay correction");
    MWAX_CUDA(cudaSetDevice(p->device));
    const size_t out_bytes = (size_t)p->n_ints * p->int_stride;
    const long long blocks_per_copy = std::max<long long>(1, p->n_blocks / 16);
    const long long n_copies = (p->n_blocks + blocks_per_copy - 1) / blocks_per_copy;
    if (!p->copy_stream) MWAX_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    if (!p->back_stream) MWAX_CUDA(cudaStreamCreateWithFlags(&p->back_stream, cudaStreamNonBlocking));
    mwax_plan::HostBuf& h = p->hbuf[b];
    if (!h.dvolt) {
        MWAX_CUDA(cudaMalloc(&h.dvolt, p->input_bytes));
        MWAX_CUDA(cudaMalloc(&h.dout, out_bytes));
        h.copied.resize(n_copies);
        for (auto& e : h.copied) MWAX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (cudaEvent_t* e : {&h.free_ev, &h.done_ev, &h.out_ev}) {
            MWAX_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
            MWAX_CUDA(cudaEventRecord(*e, p->stream));
        }
    }
    MWAX_CUDA(cudaStreamWaitEvent(p->copy_stream, h.free_ev, 0));
    MWAX_CUDA(cudaStreamWaitEvent(p->stream, h.out_ev, 0));   // the set's last output was read back
    const size_t block_bytes = (size_t)p->n * p->bs * 2;
    for (long long c = 0; c < n_copies; ++c) {
        const long long b0 = c * blocks_per_copy, b1 = std::min(p->n_blocks, b0 + blocks_per_copy);
        MWAX_CUDA(cudaMemcpyAsync(h.dvolt + b0 * block_bytes, volt + b0 * block_bytes, (b1 - b0) * block_bytes,
                                  cudaMemcpyHostToDevice, p->copy_stream));
        MWAX_CUDA(cudaEventRecord(h.copied[c], p->copy_stream));
    }
    mwax_status st = load_delay(p, delay_poly);
    if (st != MWAX_OK) return st;
    // split: a quarter of the launch group per launch, so compute follows the copies
    // while each X-step still fills the GPU several times over
    const long long host_slots = split ? std::max<long long>(1, (p->slots + 3) / 4) : 0;
    st = enqueue(p, h.dvolt, delay_poly != nullptr, h.dout, h.copied.data(), blocks_per_copy, host_slots);
    if (st != MWAX_OK) return st;
    MWAX_CUDA(cudaEventRecord(h.free_ev, p->stream));
    MWAX_CUDA(cudaEventRecord(h.done_ev, p->stream));
    MWAX_CUDA(cudaStreamWaitEvent(p->back_stream, h.done_ev, 0));
    MWAX_CUDA(cudaMemcpyAsync(vis_out, h.dout, out_bytes, cudaMemcpyDeviceToHost, p->back_stream));
    MWAX_CUDA(cudaEventRecord(h.out_ev, p->back_stream));
    return MWAX_OK;
}

}  // namespace

namespace mwax {

mwax_status set_error(mwax_status st, const char* msg) { return fail(st, "%s", msg); }

namespace {
thread_local long long t_extra_launches = 0;
}

void count_extra_launches(long long k) { t_extra_launches += k; }
long long extra_launches() { return t_extra_launches; }

mwax_status cuda_error(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return MWAX_OK;
    return fail(e == cudaErrorMemoryAllocation ? MWAX_ENOMEM : MWAX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

std::vector<LaunchGroup> plan_groups(const mwax_plan* p)
{
    std::vector<LaunchGroup> v;
    for (long long w0 = 0; w0 < p->n_ints; w0 += p->slots) {
        const long long nslots = std::min(p->slots, p->n_ints - w0);
        for (int ch = 0; ch < p->chunks; ++ch) {
            LaunchGroup g;
            g.w0 = w0;
            g.nslots = nslots;
            g.ch = ch;
            g.kbeg = (long long)ch * p->Kc;
            g.klen = std::min(p->Kc, p->K - g.kbeg);
            g.nframes = (p->chunks == 1) ? nslots * p->K : g.klen;
            g.m_begin = w0 * p->K + g.kbeg;
            v.push_back(g);
        }
    }
    return v;
}

mwax_status enqueue_init(mwax_plan* p, char* out, cudaStream_t s)
{
    MWAX_CUDA(timed(p, 0, s, [&] {
        return launch_init_output(out, p->n_ints, (long long)p->vis_set_bytes, (long long)p->weights_bytes, s);
    }));
    return MWAX_OK;
}

mwax_status enqueue_fstep(mwax_plan* p, const LaunchGroup& g, const int8_t* volt, bool have_delay, cudaStream_t s)
{
    FArgs fa;
    memset(&fa, 0, sizeof fa);
    fa.volt = volt;
    fa.delay = have_delay ? p->delay : nullptr;
    fa.Y = p->Y;
    fa.tw = p->tw;
    fa.gain = p->gain;
    fa.m_begin = g.m_begin;
    fa.n_frames = g.nframes;
    // a short last chunk of a split integration overwrites the previous chunk's frames
    // up to the next 128-frame boundary with zeros
    fa.n_store = (p->chunks == 1) ? g.nframes : std::min(p->Kpad, (g.nframes + kKAlign - 1) / kKAlign * kKAlign);
    fa.Kc = (p->chunks == 1) ? p->K : p->Kc;
    fa.Kpad = p->Kpad;
    fa.ktile = p->ktile;
    fa.n = p->n;
    fa.bs = p->bs;
    fa.nu = p->nu;
    fa.fs = p->fs;
    fa.delay_tab = p->cur_table;
    fa.tab_steps = p->cur_steps;
    fa.tab_step = p->cur_step;
    fa.flags = p->cur_flags;
    fa.status = p->status;
    fa.Yt = p->Yt;
    fa.Yt_bytes = (long long)p->Yt_bytes;
    if (p->prec == MWAX_FP8 && p->fvariant != 2) {
        // e4m3 straight from the F-step, with the plan's static per-group scales
        fa.gain = p->gain8;
        MWAX_CUDA(timed(p, 1, s, [&] { return launch_fstep(p->N, FOUT_E4M3, fa, s, p->fvariant); }));
        MWAX_CUDA(timed(p, 1, s, [&] { return launch_fill_amax(p->amax, p->amax_static, p->n_groups, p->n, g.nslots, s); }));
    } else if (p->prec == MWAX_FP8) {
        // the tensor-core DFT-product F-steps write FP16: then per path and channel group
        // the max magnitude, then e4m3 (the FP16 staging is allocated with the variant)
        if (!p->Y16) return fail(MWAX_EINVAL, "FP8 plan with F-step variant 2 and no FP16 staging");
        fa.Y = p->Y16;
        MWAX_CUDA(timed(p, 1, s, [&] { return launch_fstep(p->N, FOUT_F16, fa, s, p->fvariant); }));
        MWAX_CUDA(timed(p, 1, s, [&] {
            return launch_amax_e4m3(static_cast<const __half*>(p->Y16), p->amax, p->chan_group, p->groups,
                                    p->n_groups, g.nslots, p->N, p->n, p->Kpad, g.klen, s);
        }));
        MWAX_CUDA(timed(p, 1, s, [&] {
            return launch_quantise_e4m3(static_cast<const __half*>(p->Y16), static_cast<__nv_fp8_storage_t*>(p->Y),
                                        p->amax, p->chan_group, p->n_groups, g.nslots, p->N, p->n, p->Kpad, s);
        }));
    } else {
        const int fout = (p->prec == MWAX_FP32) ? FOUT_F32 : (p->prec == MWAX_FP16X3 ? FOUT_F16X3 : FOUT_F16);
        if (p->prec == MWAX_FP16X3) fa.Kpad = 2 * p->Kpad;   // row length: hi frames, then lo frames
        MWAX_CUDA(timed(p, 1, s, [&] { return launch_fstep(p->N, fout, fa, s, p->fvariant); }));
    }
    return MWAX_OK;
}

XArgs make_xargs(const mwax_plan* p, const LaunchGroup& g, char* out)
{
    XArgs xa;
    memset(&xa, 0, sizeof xa);
    xa.Y = p->Y;
    xa.out = out + g.w0 * (long long)p->int_stride;
    xa.out_stride = (long long)p->int_stride;
    xa.Kpad = p->Kpad;
    xa.ktile = p->ktile;
    xa.klen = g.klen;
    xa.n = p->n;
    xa.T = p->T;
    xa.N = p->N;
    xa.M = p->M;
    xa.B = p->B;
    xa.groups = p->groups;
    xa.n_groups = p->n_groups;
    xa.gain = p->gain;
    xa.runs = p->runs;
    xa.tiles = p->tiles;
    xa.post_scale = p->post_scale;
    xa.first_store = (g.ch == 0) ? 1 : 0;
    xa.status = p->status;
    xa.spin_limit = p->spin_limit;   // x 1000 cycles; 0: the kernels' default (~1 s per wait)
    xa.scale = p->amax;
    return xa;
}

mwax_status enqueue_xstep_single(mwax_plan* p, const LaunchGroup& g, const XArgs& xa_in, cudaStream_t s)
{
    XArgs xa = xa_in;
    if (p->tensor_cores) {
        XItem* items = nullptr;
        int n_items = 0;
        mwax_status st = single_items(p, g.nslots, g.klen, &items, &n_items);
        if (st != MWAX_OK) return st;
        static thread_local XLaunch L;   // large: keep it off the stack
        L.n_jobs = 1;
        L.jobs[0].tmap = p->tmap;
        L.jobs[0].a = xa;
        L.jobs[0].op = (p->prec == MWAX_FP8) ? 1 : (p->prec == MWAX_FP16X3 ? 2 : (p->prec == MWAX_INT8 ? 3 : 0));
        if (p->prec == MWAX_INT8) L.jobs[0].a.seg_frames = int8_seg_frames(g.klen);
        L.jobs[0].max_cols = 0;
        for (const int4& tl : p->h_tiles) L.jobs[0].max_cols = std::max(L.jobs[0].max_cols, tl.z);
        MWAX_CUDA(timed(p, 2, s, [&] { return launch_xstep_tc(L, items, n_items, p->counter, p->status, s); }));
    } else {
        XItem* items = nullptr;
        int n_items = 0;
        mwax_status st = single_items(p, g.nslots, g.klen, &items, &n_items);
        if (st != MWAX_OK) return st;
        MWAX_CUDA(timed(p, 2, s, [&] { return launch_xstep_simt_items(p->tmap, xa, items, n_items, s); }));
    }
    return MWAX_OK;
}

}  // namespace mwax

namespace mwax {

// X-step flops of one call (8 per complex multiply-accumulate): the algorithmic count over
// unique pairs, frames and feeding channels, and what the kernels execute with the
// current tiles and runs (see mwax_plan_info).
void x_flops(const mwax_plan& p, double* alg, double* issued)
{
    double used = 0.0;
    for (const Group& gr : p.h_groups)
        for (int c = gr.c0; c < gr.c1; ++c) used += p.h_gain[c] > 0.0f;
    *alg = 8.0 * ((double)p.n * (p.n + 1) / 2) * (double)p.K * (double)p.n_ints * used;
    double tile_pairs = 0.0;
    for (const int4& t : p.h_tiles) {
        if (p.tensor_cores) tile_pairs += 128.0 * t.z;                         // whole MMA rectangles
        else tile_pairs += 64.0 * 64.0 * (t.w ? 23.0 / 32.0 : 1.0);          // diagonal sub-block skip
    }
    double run_chan = 0.0;
    for (const RunInfo& r : p.h_runs) run_chan += run_bins(p, r.j0, r.j1);
    const long long KF = (p.prec == MWAX_FP8) ? 64 : 32;
    double frames = 0.0;
    for (const LaunchGroup& g : plan_groups(&p)) frames += (double)g.nslots * ((g.klen + KF - 1) / KF * KF);
    *issued = 8.0 * tile_pairs * run_chan * frames;
}

}  // namespace mwax

extern "C" {

const char* mwax_version(void) { return "mwax-b300 0.1 (sm_103a)"; }

const char* mwax_last_error(void) { return g_err.c_str(); }

mwax_plan* mwax_plan_create_ex(const mwax_plan_desc* desc)
{
    g_err.clear();
    if (!desc) {
        fail(MWAX_EINVAL, "desc is NULL");
        return nullptr;
    }
    mwax_plan* p = new mwax_plan();
    if (validate(*desc, *p) != MWAX_OK || setup(*p) != MWAX_OK) {
        std::string keep = g_err;
        free_plan(p);
        g_err = keep;
        return nullptr;
    }
    return p;
}

mwax_plan* mwax_plan_create(int n_tiles, int fft_len, double int_time_s, int fine_avg)
{
    mwax_plan_desc d;
    memset(&d, 0, sizeof d);
    d.n_tiles = n_tiles;
    d.fft_len = fft_len;
    d.int_time_s = int_time_s;
    d.fine_avg = fine_avg;
    return mwax_plan_create_ex(&d);
}

mwax_status mwax_plan_get_info(const mwax_plan* p, mwax_plan_info* info)
{
    if (!p || !info) return fail(MWAX_EINVAL, "NULL argument");
    info->n_paths = p->n;
    info->n_baselines = p->B;
    info->n_chan_out = p->M;
    info->frames_per_int = p->K;
    info->n_ints = p->n_ints;
    info->input_bytes = p->input_bytes;
    info->vis_set_bytes = p->vis_set_bytes;
    info->weights_bytes = p->weights_bytes;
    info->output_bytes = (size_t)p->n_ints * p->int_stride;
    // operands, FP8 variant 2's FP16 staging, F-step scratch
    info->workspace_bytes = p->Y_bytes + (p->Y16 ? 2 * p->Y_bytes : 0) + p->Yt_bytes;
    info->precision = p->prec;
    mwax::x_flops(*p, &info->x_flop_alg, &info->x_flop_issued);
    return MWAX_OK;
}

size_t mwax_plan_output_bytes(const mwax_plan* p) { return p ? (size_t)p->n_ints * p->int_stride : 0; }

size_t mwax_plan_input_bytes(const mwax_plan* p) { return p ? p->input_bytes : 0; }

mwax_status mwax_plan_set_stream(mwax_plan* p, void* stream)
{
    if (!p) return fail(MWAX_EINVAL, "plan is NULL");
    p->stream = (cudaStream_t)stream;
    return MWAX_OK;
}

mwax_status mwax_correlate(mwax_plan* p, const int8_t* volt, const double* delay_poly, void* vis_out)
{
    if (!p || !volt || !vis_out) return fail(MWAX_EINVAL, "NULL plan, voltages or vis_out");
    if (((uintptr_t)volt & 15) || ((uintptr_t)vis_out & 15))
        return fail(MWAX_EINVAL, "voltages and vis_out must be 16-byte aligned");
    if (p->prec == MWAX_INT8 && delay_poly) return fail(MWAX_EINVAL, "MWAX_INT8 takes no delay correction");
    MWAX_CUDA(cudaSetDevice(p->device));
    mwax_status st = load_delay(p, delay_poly);
    if (st != MWAX_OK) return st;
    return enqueue(p, volt, delay_poly != nullptr, static_cast<char*>(vis_out), nullptr, 1);
}

mwax_status mwax_correlate_ex(mwax_plan* p, const mwax_call* c)
{
    if (!p || !c) return fail(MWAX_EINVAL, "NULL plan or call");
    if (!c->voltages || !c->vis_out) return fail(MWAX_EINVAL, "NULL voltages or vis_out");
    if (((uintptr_t)c->voltages & 15) || ((uintptr_t)c->vis_out & 15))
        return fail(MWAX_EINVAL, "voltages and vis_out must be 16-byte aligned");
    if (c->delay_poly && c->delay_table) return fail(MWAX_EINVAL, "delay_poly and delay_table are exclusive");
    if (p->prec == MWAX_INT8 && (c->delay_poly || c->delay_table))
        return fail(MWAX_EINVAL, "MWAX_INT8 takes no delay correction");
    if (p->prec == MWAX_INT8 && c->normalise)
        return fail(MWAX_EINVAL, "normalise needs a float precision (MWAX_INT8 sums stay exact integers)");
    const long long step = c->table_step_samples ? c->table_step_samples : 6400;
    if (c->delay_table && (c->table_steps < 1 || step < 1))
        return fail(MWAX_EINVAL, "delay_table needs table_steps >= 1 and table_step_samples >= 0");
    MWAX_CUDA(cudaSetDevice(p->device));
    mwax_status st = load_delay(p, c->delay_poly);
    if (st != MWAX_OK) return st;
    if (c->delay_table) {
        const size_t bytes = sizeof(double) * (size_t)p->n * (size_t)c->table_steps;
        if (bytes > p->table_cap) {
            cudaFree(p->d_table);   // synchronises with work still reading the old table
            p->d_table = nullptr;
            p->table_cap = 0;
            MWAX_CUDA(cudaMalloc(&p->d_table, bytes));
            p->table_cap = bytes;
        }
        if ((st = copy_in(p, p->d_table, c->delay_table, bytes)) != MWAX_OK) return st;
    }
    if (c->zero_flags) {
        const size_t bytes = (size_t)p->n_blocks * p->n;
        if (!p->d_flags) MWAX_CUDA(cudaMalloc(&p->d_flags, bytes));
        if ((st = copy_in(p, p->d_flags, c->zero_flags, bytes)) != MWAX_OK) return st;
    }
    p->cur_table = c->delay_table ? p->d_table : nullptr;
    p->cur_steps = c->table_steps;
    p->cur_step = step;
    p->cur_flags = c->zero_flags ? p->d_flags : nullptr;
    char* out = static_cast<char*>(c->vis_out);
    st = enqueue(p, c->voltages, c->delay_poly != nullptr, out, nullptr, 1);
    if (st == MWAX_OK && c->zero_flags) {
        cudaError_t e = timed(p, 0, p->stream, [&] {
            return launch_weights(out, p->n_ints, (long long)p->int_stride, (long long)p->vis_set_bytes, p->T, p->M,
                                  p->K, p->N, p->bs, p->n, p->d_flags, c->normalise ? 1 : 0, p->stream);
        });
        if (e != cudaSuccess) st = cuda_error(e, "weights launch");
    }
    p->cur_table = nullptr;
    p->cur_flags = nullptr;
    return st;
}

mwax_status mwax_plan_set_passband(mwax_plan* p, const float* gain)
{
    if (!p) return fail(MWAX_EINVAL, "plan is NULL");
    if (p->prec == MWAX_INT8) return fail(MWAX_EUNSUPPORTED, "MWAX_INT8 sums stay exact integers: no passband gains");
    std::vector<float> g(p->N, 1.0f);
    if (gain) {
        for (int c = 0; c < p->N; ++c) {
            if (!(gain[c] > 0.0f) || !(gain[c] <= (float)kMaxPassband))
                return fail(MWAX_EINVAL, "passband gain[%d] = %g must be in (0, %g]", c, (double)gain[c], kMaxPassband);
            g[c] = gain[c];
        }
    }
    MWAX_CUDA(cudaSetDevice(p->device));
    MWAX_CUDA(cudaStreamSynchronize(p->stream));   // earlier calls may still read the table
    p->passband = g;
    for (int c = 0; c < p->N; ++c) p->h_gain[c] = p->h_avg_gain[c] * g[c];
    return upload_gains(*p);
}

mwax_status mwax_correlate_host(mwax_plan* p, const int8_t* volt, const double* delay_poly, void* vis_out)
{
    mwax_status st = host_call(p, volt, delay_poly, vis_out, 0, true);
    if (st != MWAX_OK) return st;
    return mwax_plan_sync(p);
}

mwax_status mwax_correlate_host_async(mwax_plan* p, const int8_t* volt, const double* delay_poly, void* vis_out)
{
    if (!p) return fail(MWAX_EINVAL, "plan is NULL");
    const int b = p->hnext;
    mwax_status st = host_call(p, volt, delay_poly, vis_out, b, false);
    if (st == MWAX_OK) p->hnext ^= 1;
    return st;
}

mwax_status mwax_plan_sync(mwax_plan* p)
{
    if (!p) return fail(MWAX_EINVAL, "plan is NULL");
    MWAX_CUDA(cudaSetDevice(p->device));
    MWAX_CUDA(cudaStreamSynchronize(p->stream));
    if (p->back_stream) MWAX_CUDA(cudaStreamSynchronize(p->back_stream));
    int st = 0;
    MWAX_CUDA(cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        MWAX_CUDA(cudaMemset(p->status, 0, sizeof(int)));
        return fail(MWAX_ETIMEOUT, "a device-side bounded wait gave up (status %d)", st);
    }
    return MWAX_OK;
}

mwax_status mwax_plan_set_wait_limit(mwax_plan* p, unsigned int kilocycles)
{
    if (!p) return fail(MWAX_EINVAL, "plan is NULL");
    p->spin_limit = kilocycles;
    return MWAX_OK;
}

mwax_status mwax_plan_enable_timing(mwax_plan* p, int enable)
{
    if (!p) return fail(MWAX_EINVAL, "plan is NULL");
    p->timing = enable != 0;
    return MWAX_OK;
}

mwax_status mwax_plan_stage_times(mwax_plan* p, double ms[3], long long launches[3])
{
    if (!p || !ms || !launches) return fail(MWAX_EINVAL, "NULL argument");
    MWAX_CUDA(cudaSetDevice(p->device));
    MWAX_CUDA(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < 3; ++i) {
        ms[i] = 0.0;
        launches[i] = p->launches[i];
        p->launches[i] = 0;
    }
    for (auto& u : p->ev_used) {
        float t = 0.0f;
        MWAX_CUDA(cudaEventElapsedTime(&t, u.second.first, u.second.second));
        ms[u.first] += t;
        p->ev_pool.push_back(u.second.first);
        p->ev_pool.push_back(u.second.second);
    }
    p->ev_used.clear();
    return MWAX_OK;
}

void mwax_plan_destroy(mwax_plan* p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    cudaStreamSynchronize(p->stream);
    if (p->copy_stream) cudaStreamSynchronize(p->copy_stream);   // host calls still in flight
    if (p->back_stream) cudaStreamSynchronize(p->back_stream);
    free_plan(p);
}

}  // extern "C"
