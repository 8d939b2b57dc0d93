// Per-kernel timing: when a handle's profiler is on, every kernel the handle
// launches is bracketed by two CUDA events recorded on the launching stream.
// Reading the profiler waits for the recorded events and accumulates, per
// kernel label, the number of launches and the summed device time.
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "weo_internal.h"

namespace weo {

struct ProfRec {
    std::string label;
    cudaEvent_t start, stop;
};

struct ProfStat {
    long long launches = 0;
    double ms = 0.0;
};

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<ProfRec> pending;
    std::map<std::string, ProfStat> stats;

    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return e;
    }
    int drain()
    {
        for (auto &r : pending) {
            cudaError_t e = cudaEventSynchronize(r.stop);
            if (e != cudaSuccess) return fail_cuda(e, "cudaEventSynchronize", __FILE__, __LINE__);
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, r.start, r.stop);
            if (e != cudaSuccess) return fail_cuda(e, "cudaEventElapsedTime", __FILE__, __LINE__);
            ProfStat &s = stats[r.label];
            s.launches += 1;
            s.ms += ms;
            pool.push_back(r.start);
            pool.push_back(r.stop);
        }
        pending.clear();
        return WEO_OK;
    }
    ~Profiler()
    {
        for (auto &r : pending) {
            cudaEventDestroy(r.start);
            cudaEventDestroy(r.stop);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

void prof_destroy(wilson_eo_s *h)
{
    delete h->prof;
    h->prof = nullptr;
}

int prof_begin(wilson_eo_s *h, const char *label, cudaStream_t s)
{
    if (!h->prof || !h->prof->on) return -1;
    ProfRec r;
    r.label = label;
    r.start = h->prof->get();
    r.stop = h->prof->get();
    if (!r.start || !r.stop) return -1;
    if (cudaEventRecord(r.start, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    h->prof->pending.push_back(r);
    return (int)h->prof->pending.size() - 1;
}

void prof_end(wilson_eo_s *h, int token, cudaStream_t s)
{
    if (token < 0 || !h->prof) return;
    if (cudaEventRecord(h->prof->pending[token].stop, s) != cudaSuccess) (void)cudaGetLastError();
}

std::string kernel_label(const char *kind, int prec, int fmt, bool dag, bool axpy)
{
    static const char *pn[] = {"f64", "f32", "f16", "bf16", "ff"};
    std::string l = kind;
    l += "_";
    l += (prec >= 0 && prec < 5) ? pn[prec] : "?";
    l += fmt == WEO_LINK12 ? "_l12" : "_l18";
    if (axpy) l += "_axpy";
    if (dag) l += "_dag";
    return l;
}

}  // namespace weo

using namespace weo;

extern "C" {

int wilson_eo_profile(wilson_eo_t h, int enable)
{
    try {
        if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
        if (!h->prof) h->prof = new Profiler();
        h->prof->on = enable != 0;
        return WEO_OK;
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_profile");
    }
}

int wilson_eo_profile_read(wilson_eo_t h, int max_kernels, char *names, int name_len,
                           double *total_ms, long long *launches, int *n_kernels, int reset)
{
    try {
        if (!h || !n_kernels) return set_error(WEO_ERR_ARG, "NULL handle or n_kernels");
        *n_kernels = 0;
        if (!h->prof) return WEO_OK;
        WEO_TRY(h->prof->drain());
        int k = 0;
        for (auto &kv : h->prof->stats) {
            if (k >= max_kernels) break;
            if (names && name_len > 0) {
                strncpy(names + (size_t)k * name_len, kv.first.c_str(), name_len - 1);
                names[(size_t)k * name_len + name_len - 1] = '\0';
            }
            if (total_ms) total_ms[k] = kv.second.ms;
            if (launches) launches[k] = kv.second.launches;
            ++k;
        }
        *n_kernels = k;
        if (reset) h->prof->stats.clear();
        return WEO_OK;
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_profile_read");
    }
}

}  // extern "C"
