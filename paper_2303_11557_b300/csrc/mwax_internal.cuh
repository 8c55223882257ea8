// Internal declarations of the MWAX B300 correlator library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/mwax.h"

namespace mwax {

constexpr double kFs = 1280000.0;        // coarse-channel sample rate (Sec. 2.5)
constexpr int kDefaultBlock = 64000;     // samples per path per 50 ms data block (Sec. 2.5)
constexpr int kKAlign = 128;             // frames per operand row are padded to this
// Integer mode: the K axis of the operands is cut into tiles of this many samples, laid out
// Y[slot][K tile][plane][p][kIntKTile], so that the 128 rows of one TMA box lie within
// 512 KB (a whole 1 s row per path would put them 2.56 MB apart, one memory page each).
constexpr int kIntKTile = 2048;

// Output-type selector of the F-step.
// FOUT_F16X3: each value v (pre-scaled) as an FP16 pair hi = fp16(v), lo = fp16(v - hi),
// hi in the first half of the operand row and lo in the second (the launch's Kpad is then
// the row length, twice the frame capacity).
// FOUT_E4M3: the FP8 form written directly, v / s rounded to e4m3 (saturating), with the
// plan's per-channel-group scale s folded into the gains (fp8_static_amax); otherwise the
// FP8 form quantises an FP16 F-step's output with measured maxima afterwards.
enum FOut : int { FOUT_F32 = 0, FOUT_F16 = 1, FOUT_F16X3 = 2, FOUT_E4M3 = 3 };

// e4m3 bytes of (v.x, v.y), saturating: x in the low byte.
__device__ __forceinline__ uint32_t e4m3x2(float2 v)
{
    return (uint32_t)__nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
}

// Channel averaging (Sec. 2.6) is split in two: the F-step multiplies ultrafine channel
// c by gain[c] = sqrt(w_c) (w_c = 1, 1/2 for the end bins of an even fscrunch, 0 for an
// excluded DC bin), so C'(c) = w_c C(c); the X-step then sums C' over a *group* of
// consecutive channels that feed the same output channels, and adds coef * sum into
// each of them, coef = 1 / sum(w) of that output channel.  j = -1 marks "none".
struct Group {
    int c0, c1;     // ultrafine channels [c0, c1) (zero-gain channels inside are skipped)
    int ja, jb;     // output channels fed
    float ca, cb;   // their 1 / sum(w)
    int first_a;    // 1: the first group (in channel order) that feeds ja; it stores
    int first_b;    //    instead of adding (same for jb)
};

// A run of consecutive output channels [j0, j1) handled by one X CTA and the groups
// [g0, g1) that feed it (groups shared with a neighbouring run add only to j in [j0, j1)).
struct RunInfo {
    int j0, j1, g0, g1;
};

// Arguments of one F-step launch: frames [m_begin, m_begin + n_frames) of the call,
// written to operand slots of Kc frames each (slot = frame / Kc).
struct FArgs {
    const int8_t* volt;   // [blk][n][bs][2]
    const double* delay;  // [n][3] or nullptr
    void* Y;              // operands [slot][N][2][n][Kpad]
    const float2* tw;     // e^{-2 pi i k / N}, k < N
    const float* gain;    // [N] sqrt of each ultrafine channel's averaging weight (x passband gain,
                          //   x the FP16 forms' power-of-two pre-scale keeping |X| in range)
    long long m_begin;
    long long n_frames;   // frames with data
    long long n_store;    // frames stored (>= n_frames: the rest are written as zeros)
    long long Kc;
    long long Kpad;
    int n;
    int bs;
    double nu;
    double fs;            // coarse-channel sample rate (1.28 MS/s unless oversampled)
    const double* delay_tab;   // [n][tab_steps] tabulated fractional delays (s), or nullptr
    long long tab_steps;
    long long tab_step;        // samples per table entry
    const uint8_t* flags;      // [n_blocks][n] zeroing flags (nonzero: block holds no data), or nullptr
    long long ktile;           // integer mode: K tile length (kIntKTile); 0 = rows of Kpad frames
    // set by launch_fstep from fs and N (so no kernel divides in FP64 per frame)
    double frame_dt;           // N / fs: seconds per frame
    double fs_over_n;          // fs / N: frames per second
    int* status;               // device status word of the kernels with bounded waits (tensor-core
                               //   F-step), or nullptr
    void* Yt;                  // F-step scratch: variant 3, frame-major spectra of one slot and
                               //   the frame terms (fstep_f128_scratch_bytes); variant 4, the
                               //   frame terms (fstep_fd_scratch_bytes); or nullptr
    long long Yt_bytes;
};

// Delay (s) of path p for frame m of the call (N samples from absolute sample m N): the
// FP64 polynomial at the frame centre t = (m + 1/2) N / Fs (Sec. 4.3), or the table entry
// of the step that holds the frame centre (Sec. 2.4.1).
__device__ __forceinline__ double frame_delay(const FArgs& a, int p, long long m, int N)
{
    if (a.delay_tab != nullptr) {
        long long step = (2 * m * N + N) / (2 * a.tab_step);
        if (step >= a.tab_steps) step = a.tab_steps - 1;
        return a.delay_tab[(long long)p * a.tab_steps + step];
    }
    const double t = ((double)m + 0.5) * a.frame_dt;
    return fma(t, fma(t, a.delay[3 * p + 2], a.delay[3 * p + 1]), a.delay[3 * p]);
}

// True when the data block holding sample s0 of path p is flagged as zeroed (Sec. 2.4.2):
// its samples are excluded (read as zero) whatever the buffer holds.
__device__ __forceinline__ bool frame_zeroed(const FArgs& a, int p, long long s0)
{
    return a.flags != nullptr && a.flags[(s0 / a.bs) * (long long)a.n + p] != 0;
}

// Arguments of one X-step launch over `slots` operand slots.
struct XArgs {
    const void* Y;         // operands [slot][N][2][n][Kpad]
    const float* scale;    // FP8: amax [slot][group][n]; the scale is s = amax / 448
    char* out;             // output of slot 0's integration
    long long out_stride;  // bytes from one integration's output to the next
    long long Kpad;
    long long klen;        // valid frames per slot in this launch
    int n, T, N, M;
    int n_groups;
    long long B;
    const Group* groups;
    const RunInfo* runs;
    const float* gain;     // [N]; channels with gain 0 are skipped
    const int4* tiles;     // (p0, q0, column count, A rows inside the B window) per tile
    float post_scale;      // multiplies every product (undoes the FP16 pre-scale)
    long long seg_frames;  // integer mode: frames per K segment, one work item each (a multiple
                           //   of 512, at most 51,200)
    int first_store;       // 1: a channel's first group stores (output not yet written by an
                           //    earlier frame chunk of the same integration); 0: all add
    int* status;           // device status word (bounded waits)
    unsigned int spin_limit;
    long long ktile;       // integer mode: K tile length of the operand layout (see kIntKTile)
};

// One launch's worth of tensor-core X-step work for one plan ("job"): its operand tensor
// map and arguments, resident in device memory.
struct XJob {
    CUtensorMap tmap;
    XArgs a;
    int op;         // 0 = FP16 (kind::f16), 1 = e4m3 (kind::f8f6f4), 2 = FP16 hi/lo pairs
                    //   (three products per complex term, chunked two-level accumulation),
                    //   3 = integer mode (int8 held in FP16, exact chunks, int64 output)
    int max_cols;   // widest tile (columns) of the job: 128 lets the launch double-buffer TMEM
};

// One work item of the persistent tensor-core X-step.
struct XItem {
    int job, tile, run, slot;
};

// The jobs of one persistent X-step launch, passed by value (kernel parameter space).
constexpr int kMaxJobs = 40;
struct XLaunch {
    int n_jobs;
    XJob jobs[kMaxJobs];
};

// Launchers (each returns the cudaError_t of its launch).
// variant 0: two-pass radix-32 kernel for N = 32..512 (generic elsewhere); 1: generic
// Stockham passes for every N; 2: a tensor-core F-step where one is built (the direct DFT
// product for N = 32, 64, 128, every output kind; the four-step DFT for FP16 output at
// N = 1280 and 6400), variant 0 elsewhere; 3: the 128-row tensor-core F-step (FP16 or e4m3
// output, N = 1280 and 6400), variant 2 elsewhere; 4: the direct DFT with the frames on
// the accumulator lanes (FP16 or e4m3 output, N = 32, 64, 128), variant 0 elsewhere.
cudaError_t launch_fstep(int N, int out_kind, const FArgs& a, cudaStream_t s, int variant);
// Kernels launched beyond the first by a launcher that issues several (the F-step variants
// with a frame-term kernel and a transpose), counted per host thread: a plan's launch count
// is the number of kernels.
void count_extra_launches(long long k);
long long extra_launches();
// The tensor-core four-step F-step (FP16 output), N = 1280 or 6400.
bool fstep_tc_supported(int N);
cudaError_t launch_fstep_tc(int N, const FArgs& a, cudaStream_t s);
// The 128-row tensor-core F-step (FP16 or e4m3 output), N = 1280 or 6400; it needs the
// scratch a.Yt of fstep_f128_scratch_bytes (one slot of frame-major spectra).
bool fstep_f128_supported(int N);
size_t fstep_f128_scratch_bytes(int N, int n, long long Kc);
cudaError_t launch_fstep_f128(int N, int out_kind, const FArgs& a, cudaStream_t s);
// The tensor-core direct-DFT F-step with the frames on the accumulator lanes (variant 4),
// N = 32, 64, 128, FP16 or e4m3 output; it needs the scratch a.Yt of fstep_fd_scratch_bytes
// for a launch of n_store frames (the frames' delay terms).
bool fstep_fd_supported(int N, int out_kind);
size_t fstep_fd_scratch_bytes(int N, int n, long long n_store);
cudaError_t launch_fstep_fd(int N, int out_kind, const FArgs& a, cudaStream_t s);
// The tensor-core direct-DFT F-step, N = 32, 64, 128 (FP32, FP16 or FP16 hi/lo output).
bool fstep_dft_supported(int N, int out_kind);
cudaError_t launch_fstep_dft(int N, int out_kind, const FArgs& a, cudaStream_t s);

// e4m3 scale of a path's spectra from their max magnitude: 448 is e4m3's largest finite.
__host__ __device__ __forceinline__ float e4m3_scale(float amax) { return amax > 0.0f ? amax * (1.0f / 448.0f) : 1.0f; }
cudaError_t launch_quantise_e4m3(const __half* Y16, __nv_fp8_storage_t* Y8, const float* amax,
                                 const int* chan_group, int n_groups, long long slots, int N, int n, long long Kpad,
                                 cudaStream_t s);
// FP8 form after an FP16 F-step: per (slot, group, path) the max magnitude of the FP16
// values over frames [0, kvalid) into amax (then launch_quantise_e4m3).
cudaError_t launch_amax_e4m3(const __half* Y16, float* amax, const int* chan_group, const Group* groups, int n_groups,
                             long long slots, int N, int n, long long Kpad, long long kvalid, cudaStream_t s);
// FP8 form written by the F-step (FOUT_E4M3): the scales are static per channel group,
// amax[slot][g][p] = amax_static[g] for the launch's slots.
cudaError_t launch_fill_amax(float* amax, const float* amax_static, int n_groups, int n, long long slots,
                             cudaStream_t s);
cudaError_t launch_init_output(char* out, long long n_ints, long long vis_set_bytes, long long weights_bytes,
                               cudaStream_t s);
// Occupancy weights from zeroing flags (Sec. 4.1) over each integration's weights table;
// with normalise (float output only) the visibilities are divided by them.
cudaError_t launch_weights(char* out, long long n_ints, long long int_stride, long long vis_set_bytes, int T, int M,
                           long long K, int N, int bs, int n, const uint8_t* flags, int normalise, cudaStream_t s);
cudaError_t launch_xstep_simt(const CUtensorMap& map, const XArgs& a, int n_tiles, int n_runs, int slots,
                              cudaStream_t s);
// Same over a work list (tile, run, slot per CTA, in launch order).
cudaError_t launch_xstep_simt_items(const CUtensorMap& map, const XArgs& a, const XItem* items, int n_items,
                                    cudaStream_t s);
int simt_resident_ctas();   // CTAs of the FP32 X-step resident per SM
// FP32 operand planes for the CUDA-core X-step: 32 frames x 64 rows x both planes per box,
// 128-byte swizzle.
cudaError_t make_simt_tmap(CUtensorMap* map, const void* Y, long long Kpad, int n, long long planes);
cudaError_t make_rows_tmap(CUtensorMap* map, const void* base, int row_words, long long rows, int box_words,
                           int box_rows);
cudaError_t make_operand_tmap(CUtensorMap* map, const void* Y, int elem_bytes, long long Kpad, int n,
                              long long planes);
cudaError_t launch_xstep_tc(const XLaunch& L, const XItem* items, int n_items, int* counter, int* status,
                            cudaStream_t s);
int build_tc_tiles(int n, int window, int4* out, int cap);
bool fft_len_supported(int N);

}  // namespace mwax
