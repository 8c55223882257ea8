// Real-time serving loop: sub-observations (8 s of one coarse channel, as the paper's
// FX-engine receives them through its input ring buffer, Sec. 2.5) arrive from the host
// and are admitted onto the GPU as device lanes and HBM free up.
//
// A scheduler thread owns every CUDA call of the server.  Submitted requests wait in a
// FIFO; the head is admitted when a lane is idle and its device footprint (input and
// output buffers, plus the plan workspace if the lane has no plan of that shape yet) fits
// the HBM budget.  A lane is a CUDA stream with its own plan cache and device buffers
// (reused, grown on demand); on admission it runs H2D copy -> mwax_correlate -> D2H copy
// and records an event.  Requests on different lanes run concurrently on the device
// (continuous batching).  Completion is the event firing; latency is submission to
// completion on the host clock.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "plan.cuh"

using namespace mwax;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long id;
    mwax_plan_desc desc;
    const int8_t* volt;
    const double* delay;
    void* out;
    double deadline_s;
    Clock::time_point submitted;
    int status = 0;   // 0 pending, 1 done, <0 -error
    bool cold = false;   // its admission created a plan
};

// Plans are cached per shape: ordered on the descriptor's fields (never on its bytes, so
// padding a caller left uninitialised cannot create a new plan per request).
struct PlanKey {
    mwax_plan_desc d;
    auto fields() const
    {
        return std::tie(d.n_tiles, d.fft_len, d.fine_avg, d.int_time_s, d.samples_per_call, d.block_samples,
                        d.precision, d.sky_freq_hz, d.keep_dc, d.workspace_limit, d.sample_rate_hz, d.keep_bins);
    }
    bool operator<(const PlanKey& o) const { return fields() < o.fields(); }
};

struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::map<PlanKey, mwax_plan*> plans;
    size_t plan_bytes = 0;
    int8_t* dvolt = nullptr;
    size_t dvolt_bytes = 0;
    char* dout = nullptr;
    size_t dout_bytes = 0;
    Request* running = nullptr;
};

}  // namespace

struct mwax_server {
    mwax_server_desc cfg;
    int device = 0;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Request*> queue;
    std::map<long long, Request*> all;
    long long next_id = 0;
    bool stop = false;
    std::thread thr;
    size_t hbm_in_use = 0;
    std::vector<double> latencies_ms;
    std::vector<double> warm_latencies_ms;   // requests whose lane already held their plan
    long long completed = 0, failed = 0, misses = 0, submitted = 0;
    long long cold = 0;   // admissions that had to create a plan
    long long reset_completed = 0, reset_failed = 0;   // counts at the last statistics reset
    std::string init_error;
    bool ready = false;
};

namespace {

size_t footprint_new_plan(const mwax_plan_desc& d)
{
    // the plan's workspace is bounded by its workspace_limit (the server sets it)
    return d.workspace_limit + ((size_t)64 << 20);
}

mwax_plan* lane_plan(mwax_server* S, Lane& L, const mwax_plan_desc& d)
{
    auto it = L.plans.find(PlanKey{d});
    if (it != L.plans.end()) return it->second;
    mwax_plan* p = mwax_plan_create_ex(&d);
    if (!p) return nullptr;
    mwax_plan_set_stream(p, L.stream);
    mwax_plan_info info;
    mwax_plan_get_info(p, &info);
    L.plans[PlanKey{d}] = p;
    L.plan_bytes += info.workspace_bytes;
    S->hbm_in_use += info.workspace_bytes;
    return p;
}

// Make room for `need` more bytes by dropping idle lanes' cached plans (largest first).
void evict_for(mwax_server* S, size_t need)
{
    while (S->hbm_in_use + need > S->cfg.hbm_budget) {
        Lane* victim = nullptr;
        for (auto& L : S->lanes)
            if (!L.running && !L.plans.empty() && (!victim || L.plan_bytes > victim->plan_bytes)) victim = &L;
        if (!victim) return;
        for (auto& kv : victim->plans) mwax_plan_destroy(kv.second);
        victim->plans.clear();
        S->hbm_in_use -= victim->plan_bytes;
        victim->plan_bytes = 0;
    }
}

bool grow(mwax_server* S, void** buf, size_t* have, size_t need)
{
    if (*have >= need) return true;
    if (*buf) {
        cudaFree(*buf);
        S->hbm_in_use -= *have;
    }
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) return false;
    *have = need;
    S->hbm_in_use += need;
    return true;
}

// Try to start the queue head on an idle lane.  Called with the mutex held.
bool try_admit(mwax_server* S)
{
    if (S->queue.empty()) return false;
    Request* r = S->queue.front();
    Lane* lane = nullptr;
    for (auto& L : S->lanes)   // prefer an idle lane that already has this shape's plan
        if (!L.running && L.plans.count(PlanKey{r->desc})) {
            lane = &L;
            break;
        }
    if (!lane)
        for (auto& L : S->lanes)
            if (!L.running) {
                lane = &L;
                break;
            }
    if (!lane) return false;
    // device footprint of this request on this lane
    const mwax_plan_desc& d = r->desc;
    const bool has_plan = lane->plans.count(PlanKey{d}) != 0;
    mwax_plan* probe = has_plan ? lane->plans[PlanKey{d}] : nullptr;
    size_t in_b = 0, out_b = 0;
    if (probe) {
        in_b = mwax_plan_input_bytes(probe);
        out_b = mwax_plan_output_bytes(probe);
    } else {
        const double bs = d.block_samples ? d.block_samples : 64000;
        const double fs = d.sample_rate_hz > 0.0 ? d.sample_rate_hz : kFs;
        const long long S_ = d.samples_per_call ? d.samples_per_call : llround(d.int_time_s * fs);
        in_b = (size_t)S_ * 2 * d.n_tiles * 2;
        const long long ints = S_ / std::max(1LL, llround(d.int_time_s * fs));
        const long long B = (long long)d.n_tiles * (d.n_tiles + 1) / 2;
        const int M = (d.keep_bins ? d.keep_bins : d.fft_len) / std::max(1, d.fine_avg);
        out_b = (size_t)ints * (d.precision == MWAX_INT8 ? B * 4 * 16 : B * M * 4 * 8) + (size_t)ints * B * 16;
        (void)bs;
    }
    const size_t extra = (in_b > lane->dvolt_bytes ? in_b - lane->dvolt_bytes : 0) +
                         (out_b > lane->dout_bytes ? out_b - lane->dout_bytes : 0) +
                         (has_plan ? 0 : footprint_new_plan(d));
    if (S->hbm_in_use + extra > S->cfg.hbm_budget) {
        evict_for(S, extra);
        if (S->hbm_in_use + extra > S->cfg.hbm_budget) {
            bool any_running = false;
            for (auto& L : S->lanes) any_running |= L.running != nullptr;
            if (any_running) return false;   // wait for memory to free up
        }
    }
    S->queue.pop_front();
    if (!has_plan) S->cold += 1;
    r->cold = !has_plan;
    mwax_plan* p = lane_plan(S, *lane, d);
    bool ok = p && grow(S, reinterpret_cast<void**>(&lane->dvolt), &lane->dvolt_bytes, mwax_plan_input_bytes(p)) &&
              grow(S, reinterpret_cast<void**>(&lane->dout), &lane->dout_bytes, mwax_plan_output_bytes(p));
    if (ok) {
        ok = cudaMemcpyAsync(lane->dvolt, r->volt, mwax_plan_input_bytes(p), cudaMemcpyHostToDevice, lane->stream) ==
                 cudaSuccess &&
             mwax_correlate(p, lane->dvolt, r->delay, lane->dout) == MWAX_OK &&
             cudaMemcpyAsync(r->out, lane->dout, mwax_plan_output_bytes(p), cudaMemcpyDeviceToHost, lane->stream) ==
                 cudaSuccess &&
             cudaEventRecord(lane->done, lane->stream) == cudaSuccess;
    }
    if (!ok) {
        r->status = -MWAX_ECUDA;
        S->failed += 1;
        S->done_cv.notify_all();
        return true;
    }
    lane->running = r;
    return true;
}

void reap(mwax_server* S)
{
    for (auto& L : S->lanes) {
        if (!L.running) continue;
        const cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        Request* r = L.running;
        L.running = nullptr;
        const double ms =
            std::chrono::duration<double, std::milli>(Clock::now() - r->submitted).count();
        if (q == cudaSuccess) {
            r->status = 1;
            S->completed += 1;
            S->latencies_ms.push_back(ms);
            if (!r->cold) S->warm_latencies_ms.push_back(ms);
            if (r->deadline_s > 0 && ms > 1e3 * r->deadline_s) S->misses += 1;
        } else {
            r->status = -MWAX_ECUDA;
            S->failed += 1;
        }
        S->done_cv.notify_all();
    }
}

void scheduler(mwax_server* S)
{
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (cudaSetDevice(S->device) != cudaSuccess) S->init_error = "cudaSetDevice failed";
        for (auto& L : S->lanes) {
            if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess)
                S->init_error = "stream/event creation failed";
        }
        S->ready = true;
        S->done_cv.notify_all();
    }
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        reap(S);
        while (try_admit(S)) {
        }
        bool busy = false;
        for (auto& L : S->lanes) busy |= L.running != nullptr;
        if (S->stop && !busy && S->queue.empty()) break;
        if (busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(100));
            lk.lock();
        } else {
            S->cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
    for (auto& L : S->lanes) {
        cudaStreamSynchronize(L.stream);
        for (auto& kv : L.plans) mwax_plan_destroy(kv.second);
        cudaFree(L.dvolt);
        cudaFree(L.dout);
        cudaEventDestroy(L.done);
        cudaStreamDestroy(L.stream);
    }
}

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

mwax_server* mwax_server_create(const mwax_server_desc* desc)
{
    mwax_server* S = new mwax_server();
    memset(&S->cfg, 0, sizeof S->cfg);
    if (desc) S->cfg = *desc;
    if (!S->cfg.hbm_budget) S->cfg.hbm_budget = (size_t)64 << 30;
    if (S->cfg.n_lanes <= 0) S->cfg.n_lanes = 4;
    if (!S->cfg.workspace_limit) S->cfg.workspace_limit = (size_t)2 << 30;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        set_error(MWAX_ECUDA, "no CUDA device");
        delete S;
        return nullptr;
    }
    S->lanes.resize(S->cfg.n_lanes);
    S->thr = std::thread(scheduler, S);
    std::unique_lock<std::mutex> lk(S->mu);
    S->done_cv.wait(lk, [&] { return S->ready; });
    if (!S->init_error.empty()) {
        std::string e = S->init_error;
        S->stop = true;
        lk.unlock();
        S->cv.notify_all();
        S->thr.join();
        set_error(MWAX_ECUDA, e.c_str());
        delete S;
        return nullptr;
    }
    return S;
}

long long mwax_server_submit(mwax_server* S, const mwax_plan_desc* desc, const int8_t* voltages,
                             const double* delay_poly, void* vis_out, double deadline_s)
{
    if (!S || !desc || !voltages || !vis_out) {
        set_error(MWAX_EINVAL, "NULL server, desc, voltages or vis_out");
        return -1;
    }
    Request* r = new Request();
    r->desc = *desc;
    r->desc.workspace_limit = desc->workspace_limit ? desc->workspace_limit : S->cfg.workspace_limit;
    r->volt = voltages;
    r->delay = delay_poly;
    r->out = vis_out;
    r->deadline_s = deadline_s;
    r->submitted = Clock::now();
    {
        std::lock_guard<std::mutex> g(S->mu);
        r->id = S->next_id++;
        S->all[r->id] = r;
        S->queue.push_back(r);
        S->submitted += 1;
    }
    S->cv.notify_all();
    return r->id;
}

int mwax_server_poll(mwax_server* S, long long id)
{
    if (!S) return -MWAX_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return -MWAX_EINVAL;
    return it->second->status;
}

mwax_status mwax_server_wait(mwax_server* S, long long id)
{
    if (!S) return set_error(MWAX_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return set_error(MWAX_EINVAL, "unknown request id");
    Request* r = it->second;
    S->done_cv.wait(lk, [&] { return r->status != 0; });
    return r->status == 1 ? MWAX_OK : set_error((mwax_status)(-r->status), "request failed");
}

mwax_status mwax_server_drain(mwax_server* S)
{
    if (!S) return set_error(MWAX_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    S->done_cv.wait(lk, [&] { return S->completed + S->failed + S->reset_completed + S->reset_failed == S->submitted; });
    return S->failed ? set_error(MWAX_ECUDA, "some requests failed") : MWAX_OK;
}

mwax_status mwax_server_reset_stats(mwax_server* S)
{
    if (!S) return set_error(MWAX_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    S->reset_completed += S->completed;
    S->reset_failed += S->failed;
    S->completed = S->failed = S->misses = S->cold = 0;
    S->latencies_ms.clear();
    S->warm_latencies_ms.clear();
    return MWAX_OK;
}

mwax_status mwax_server_get_stats(mwax_server* S, mwax_server_stats* st)
{
    if (!S || !st) return set_error(MWAX_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    st->submitted = S->submitted - S->reset_completed - S->reset_failed;
    st->completed = S->completed;
    st->failed = S->failed;
    st->queued = (long long)S->queue.size();
    st->in_flight = 0;
    for (auto& L : S->lanes) st->in_flight += L.running != nullptr;
    st->p50_ms = percentile(S->latencies_ms, 0.50);
    st->p99_ms = percentile(S->latencies_ms, 0.99);
    st->max_ms = S->latencies_ms.empty() ? 0.0 : *std::max_element(S->latencies_ms.begin(), S->latencies_ms.end());
    st->deadline_misses = S->misses;
    st->hbm_in_use = S->hbm_in_use;
    st->cold_starts = S->cold;
    st->p50_warm_ms = percentile(S->warm_latencies_ms, 0.50);
    st->p99_warm_ms = percentile(S->warm_latencies_ms, 0.99);
    return MWAX_OK;
}

void mwax_server_destroy(mwax_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    S->thr.join();
    for (auto& kv : S->all) delete kv.second;
    delete S;
}

}  // extern "C"
