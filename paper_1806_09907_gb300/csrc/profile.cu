// Optional per-kernel timing of the library's own launches with CUDA events
// recorded on the launching stream (off by default; see al_profile_enable).
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "airgb.h"
#include "profile.h"

namespace airgb {

namespace {

struct Pending {
    const char *name;
    cudaEvent_t start, stop;
};

struct Totals {
    std::string name;
    double ms;
    long long launches;
};

std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
std::vector<Totals> g_totals;
thread_local cudaEvent_t t_open = nullptr;
thread_local const char *t_name = nullptr;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess)
        return nullptr;
    return e;
}

}  // namespace

void prof_begin(cudaStream_t s, const char *name)
{
    if (!g_on)
        return;
    // a stream being captured into a CUDA graph records nothing: an event
    // recorded there would become a graph node, not a timestamp
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    t_open = take_event();
    t_name = name;
    if (t_open)
        cudaEventRecord(t_open, s);
}

void prof_end(cudaStream_t s)
{
    if (!g_on || !t_open)
        return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t stop = take_event();
    if (!stop) {
        g_pool.push_back(t_open);
        t_open = nullptr;
        return;
    }
    cudaEventRecord(stop, s);
    g_pending.push_back({t_name, t_open, stop});
    t_open = nullptr;
}

}  // namespace airgb

using namespace airgb;

extern "C" {

al_status al_profile_enable(int32_t on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return AL_OK;
}

int32_t al_profile_collect(char *names, size_t names_bytes, double *total_ms, int64_t *launches,
                           int32_t max_kernels)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Pending &p : g_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            Totals *t = nullptr;
            for (Totals &x : g_totals)
                if (x.name == p.name)
                    t = &x;
            if (!t) {
                g_totals.push_back({p.name, 0.0, 0});
                t = &g_totals.back();
            }
            t->ms += ms;
            t->launches += 1;
        }
        g_pool.push_back(p.start);
        g_pool.push_back(p.stop);
    }
    g_pending.clear();
    const int n = (int)g_totals.size();
    if (names && names_bytes > 0)
        names[0] = '\0';
    size_t used = 0;
    for (int i = 0; i < n && i < max_kernels; ++i) {
        if (total_ms)
            total_ms[i] = g_totals[i].ms;
        if (launches)
            launches[i] = g_totals[i].launches;
        if (names) {
            const size_t len = g_totals[i].name.size();
            if (used + len + 2 <= names_bytes) {
                memcpy(names + used, g_totals[i].name.c_str(), len);
                used += len;
                names[used++] = '\n';
                names[used] = '\0';
            }
        }
    }
    return n;
}

al_status al_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Pending &p : g_pending) {
        cudaEventSynchronize(p.stop);
        g_pool.push_back(p.start);
        g_pool.push_back(p.stop);
    }
    g_pending.clear();
    g_totals.clear();
    return AL_OK;
}

}  // extern "C"
