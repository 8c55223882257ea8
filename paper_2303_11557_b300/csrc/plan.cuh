// The plan object behind the C ABI's opaque mwax_plan, and the launch building blocks
// shared by the single-plan path (api.cu) and the batch path (batch.cu).
#pragma once

#include <string>
#include <vector>

#include "mwax_internal.cuh"

using mwax::Group;
using mwax::RunInfo;
using mwax::XItem;

struct mwax_plan {
    mwax_plan_desc desc;
    int T = 0, n = 0, N = 0, F = 0, M = 0, bs = 0, prec = 0, dc_excl = 1;
    int keep = 0;             // ultrafine channels passed to the X step (centred on DC)
    double fs = 0.0;          // coarse-channel sample rate
    long long K = 0, S = 0, n_ints = 0, B = 0, n_blocks = 0;
    double nu = 0.0;
    size_t vis_set_bytes = 0, weights_bytes = 0, int_stride = 0, input_bytes = 0;

    // integration grouping: `slots` integrations per launch, or one integration split
    // into `chunks` launches of at most Kc frames
    long long slots = 1, Kc = 0, Kpad = 0;
    int chunks = 1;
    int elem_bytes = 4;
    long long ktile = 0;      // integer mode: K tile of the operand layout (kIntKTile), else 0

    // device memory
    void* Y = nullptr;      // X-step operands (FP8: e4m3)
    void* Y16 = nullptr;    // FP8 with F-step variant 2 only: the FP16 operands the e4m3 ones
                            //   are quantised from (2 x Y_bytes), allocated with the variant
    void* Yt = nullptr;     // F-step variants 3 and 4: their scratch (frame terms; variant 3
                            //   also the frame-major spectra of one slot)
    size_t Yt_bytes = 0;
    size_t Y_bytes = 0;
    float2* tw = nullptr;
    double* delay = nullptr;
    Group* groups = nullptr;
    int n_groups = 0;
    float* gain = nullptr;
    int* chan_group = nullptr;   // FP8: group of each ultrafine channel
    float* amax = nullptr;       // FP8: [slots][groups][n] per-path max magnitude
    size_t amax_bytes = 0;
    float* gain8 = nullptr;      // FP8, e4m3 from the F-step: gains carrying 1 / (static scale)
    float* amax_static = nullptr;   // FP8: [groups] bound on the group's magnitudes
    RunInfo* runs = nullptr;
    int n_runs = 0;
    int4* tiles = nullptr;
    int n_tiles = 0;
    int* status = nullptr;
    int* counter = nullptr;   // work-item counter of the persistent X-step
    float out_scale = 1.0f, post_scale = 1.0f;
    bool tensor_cores = false;   // tcgen05 X-step (FP16 / FP8 / INT8) vs CUDA-core FP32
    int tile = 64;               // paths per tile side of the X-step
    int run_len = 0;             // output channels per X work item (autotuned)
    int window = 256;            // tensor-core tile column window (autotuned: 128 or 256)
    int fvariant = 0;            // F-step kernel: 0 = two-pass radix-32 where built, 1 = generic,
                                 //   2 = tensor-core DFT products, 3 = 128-row tensor-core
    CUtensorMap tmap;            // operand planes, for the tcgen05 X-step

    // host copies of the tables (work-item costs) and the tcgen05 item lists by slot count
    std::vector<int4> h_tiles;
    std::vector<RunInfo> h_runs;
    std::vector<Group> h_groups;
    std::vector<float> h_gain;
    std::vector<float> h_avg_gain;   // sqrt of each channel's averaging weight
    std::vector<float> passband;     // de-ripple gain per channel (1 = flat)

    // extended calls: device copies of the delay table and zeroing flags, and what the
    // call being enqueued uses (nullptr outside mwax_correlate_ex)
    double* d_table = nullptr;
    size_t table_cap = 0;
    uint8_t* d_flags = nullptr;
    const double* cur_table = nullptr;
    long long cur_steps = 0, cur_step = 0;
    const uint8_t* cur_flags = nullptr;
    struct ItemList {
        long long key;
        XItem* items;
        int n;
    };
    std::vector<ItemList> item_lists;   // per (slot count, frames) of a launch

    // host-input path: two device staging sets used alternately by the streaming call
    // (the synchronous one always takes set 0)
    struct HostBuf {
        int8_t* dvolt = nullptr;
        char* dout = nullptr;
        std::vector<cudaEvent_t> copied;   // per copy chunk of the voltages
        cudaEvent_t free_ev = nullptr;     // the last call that used the set has read it
        cudaEvent_t done_ev = nullptr;     // its correlation is complete (output written)
        cudaEvent_t out_ev = nullptr;      // its output has been copied back
    };
    HostBuf hbuf[2];
    int hnext = 0;
    cudaStream_t copy_stream = nullptr;   // uploads
    cudaStream_t back_stream = nullptr;   // read-backs

    cudaStream_t stream = nullptr;
    int device = 0;
    unsigned int spin_limit = 0;   // bounded device waits, x 1000 cycles (0: the kernels' default)

    // stage timing: event pairs per launch, drained by mwax_plan_stage_times
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    long long launches[3] = {0, 0, 0};
};


namespace mwax {

// One launch group of a call: `nslots` integrations from w0, or chunk `ch` of integration w0.
struct LaunchGroup {
    long long w0, nslots, kbeg, klen, nframes, m_begin;
    int ch;
};

std::vector<LaunchGroup> plan_groups(const mwax_plan* p);
mwax_status enqueue_init(mwax_plan* p, char* out, cudaStream_t s);
mwax_status enqueue_fstep(mwax_plan* p, const LaunchGroup& g, const int8_t* volt, bool have_delay, cudaStream_t s);
XArgs make_xargs(const mwax_plan* p, const LaunchGroup& g, char* out);
mwax_status enqueue_xstep_single(mwax_plan* p, const LaunchGroup& g, const XArgs& xa, cudaStream_t s);
void plan_items(const mwax_plan& p, int job, long long nslots, long long klen,
                std::vector<std::pair<double, XItem>>& out);
// F-step variant 3: allocate its scratch (once; set-up time, never inside a call).
mwax_status ensure_fstep_scratch(mwax_plan* p, int variant);
// Integer mode: samples per K segment of the tensor-core X-step (one work item each).
long long int8_seg_frames(long long klen);
void sort_items(std::vector<std::pair<double, XItem>>& v, std::vector<XItem>& order);
mwax_status set_error(mwax_status st, const char* msg);
mwax_status configure_x(mwax_plan& p, int run_len, int window);
mwax_status cuda_error(cudaError_t e, const char* what);

}  // namespace mwax
