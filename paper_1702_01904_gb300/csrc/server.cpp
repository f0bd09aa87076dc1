// server.cpp -- continuous-batching request engine over the plan API (include/prism.h).
//
// A worker thread owns all CUDA work.  Requests (cell + potential + probe + scan + detector)
// queue in arrival order; the worker admits a request as soon as an in-flight slot is free and
// its device-memory footprint fits the server's HBM budget, launches its S-matrix build (unless an
// S-matrix with the request's key is resident) and its scan on the stream of its plan, and keeps
// polling the in-flight requests' completion events.  Requests for different S-matrices run on
// different streams and overlap on the device; requests that share a key reuse the resident
// S-matrix (the S-matrix serves every later probe configuration, Varying Probe Size section).
// Idle resident S-matrices are evicted least-recently-used when a new one needs the memory.
// Every wait is bounded.  Results are bitwise identical to running the request alone: the
// kernels are deterministic and nothing is shared between in-flight requests but read-only S.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "prism.h"

using Clock = std::chrono::steady_clock;

namespace {

double ms_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Resident {  // a plan with its S-matrix, resident on the device
    prism_plan *plan = nullptr;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;
    prism_grid grid{};
    std::vector<double> slice_dz;
    int users = 0;
    bool built = false;
    Clock::time_point last_use;
};

struct Job {
    unsigned long long ticket = 0;
    prism_grid grid{};
    std::vector<double> slice_dz;
    const float *V_host = nullptr;
    unsigned long long key = 0;
    prism_probe probe{};
    std::vector<double> x0, y0;
    int px = 0, py = 0;
    prism_detector det{};
    float *out_host = nullptr;
    // runtime
    std::shared_ptr<Resident> res;
    float *out_dev = nullptr;
    float *out_pinned = nullptr;
    size_t out_bytes = 0;
    cudaEvent_t done = nullptr;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // device timestamps of the request's work
    double dev_start_ms = -1.0, dev_end_ms = -1.0;
    Clock::time_point t_submit, t_admit, t_done;
    int status = PRISM_OK;
    int reused = 0;
    bool finished = false;
    bool cancelled = false;
    std::string error;
};

bool same_grid(const prism_grid &a, const std::vector<double> &adz, const prism_grid &b, const std::vector<double> &bdz) {
    return a.nx == b.nx && a.ny == b.ny && a.n_slices == b.n_slices && a.cell_x == b.cell_x && a.cell_y == b.cell_y &&
           a.dz == b.dz && a.kv == b.kv && a.f == b.f && a.downsample == b.downsample && a.aa_frac == b.aa_frac &&
           a.alpha_max_mrad == b.alpha_max_mrad && adz == bdz;
}

}  // namespace

struct prism_server {
    size_t budget = 0;
    int max_inflight = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    unsigned long long next_ticket = 1;
    std::deque<std::shared_ptr<Job>> pending;
    std::list<std::shared_ptr<Job>> running;
    std::map<unsigned long long, std::shared_ptr<Job>> jobs;  // by ticket, until waited for
    std::map<unsigned long long, std::shared_ptr<Resident>> cache;  // by key
    std::vector<std::shared_ptr<Resident>> anonymous;             // key 0: freed after the request
    size_t used = 0, peak_used = 0;
    long admitted = 0, completed = 0;
    cudaEvent_t ref = nullptr;  // device-time origin of the request timestamps
    // worker-side helpers (called with mu held)
    void loop();
    bool try_admit(std::shared_ptr<Job> &j);
    void reap();
    size_t footprint(const Job &j, bool need_plan) const;
    bool evict_for(size_t need);
    void fail_job(const std::shared_ptr<Job> &j, int code, const std::string &msg);
};

static size_t plan_bytes_estimate(const prism_grid &g) {
    // transmission + row transform of t_0 + wave stack of all beams + S-matrix + tables, matching
    // prism_plan_create
    const double lam = prism_wavelength(g.kv);
    const double a = g.alpha_max_mrad * 1e-3;
    const double rx = a / (lam * g.f / g.cell_x), ry = a / (lam * (g.f_y > 0 ? g.f_y : g.f) / g.cell_y);
    const double beams = 3.15 * (rx + 1) * (ry + 1) + 8;
    const size_t px = (size_t)g.nx * g.ny;
    const size_t s16 = g.precision != PRISM_PRECISION_FP32
                           ? (size_t)((beams + 8) * 4 * px / (g.downsample * g.downsample)) * (g.precision == PRISM_PRECISION_FP16X2 ? 2 : 1)
                           : 0;
    return (size_t)(g.n_slices + 1) * px * 8 + (size_t)(beams * px * 8) + (size_t)(beams * px / (g.downsample * g.downsample) * 8) +
           s16 + ((size_t)2 << 20) + (size_t)g.n_slices * px * 4;
}

// window scratch a scan of this job can grow its plan's to: 32 complex windows per probe block, one
// slot per resident CTA (at most 2 per SM) plus one per block split over idle CTAs
static size_t scan_scratch_estimate(const Job &j) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 160;
    }
    const int ds = j.grid.downsample > 0 ? j.grid.downsample : 1;
    const int fx = j.grid.f > 0 ? j.grid.f : 1, fy = j.grid.f_y > 0 ? j.grid.f_y : fx;
    const size_t win = (size_t)(j.grid.nx / ds / fx) * (size_t)(j.grid.ny / ds / fy) * 8;
    const size_t blocks = ((size_t)j.px + 3) / 4 * (((size_t)j.py + 3) / 4);  // bounds 4 x 8 and 8 x 4 blocks
    const size_t cap = (size_t)2 * sms;
    return (std::min(blocks, cap) + std::min(blocks, cap)) * 32 * win + cap * sizeof(int);
}

size_t prism_server::footprint(const Job &j, bool need_plan) const {
    size_t b = j.out_bytes + (size_t)j.x0.size() * 16 + 4096 + scan_scratch_estimate(j);
    if (need_plan) b += plan_bytes_estimate(j.grid);
    return b;
}

bool prism_server::evict_for(size_t need) {
    while (budget && used + need > budget) {
        // least-recently-used idle resident plan
        auto victim = cache.end();
        for (auto it = cache.begin(); it != cache.end(); ++it)
            if (it->second->users == 0 && (victim == cache.end() || it->second->last_use < victim->second->last_use))
                victim = it;
        if (victim == cache.end()) return false;
        prism_plan_destroy(victim->second->plan);
        cudaStreamDestroy(victim->second->stream);
        used -= victim->second->bytes;
        cache.erase(victim);
    }
    return true;
}

void prism_server::fail_job(const std::shared_ptr<Job> &j, int code, const std::string &msg) {
    j->status = code;
    j->error = msg;
    j->finished = true;
    j->t_done = Clock::now();
    if (j->t_admit.time_since_epoch().count() == 0) j->t_admit = j->t_done;
    completed++;
    cv_done.notify_all();
}

bool prism_server::try_admit(std::shared_ptr<Job> &j) {
    std::shared_ptr<Resident> res;
    if (j->key) {
        auto it = cache.find(j->key);
        if (it != cache.end()) {
            if (!same_grid(it->second->grid, it->second->slice_dz, j->grid, j->slice_dz)) {
                fail_job(j, PRISM_ERR_INVALID, "smatrix_key reused with a different grid");
                return true;
            }
            res = it->second;
        }
    }
    const bool need_plan = !res;
    const size_t need = footprint(*j, need_plan);
    if (budget && need > budget) {
        fail_job(j, PRISM_ERR_BUDGET, "request needs " + std::to_string(need) + " bytes, server budget " + std::to_string(budget));
        return true;
    }
    if (budget && used + need > budget && !evict_for(need)) return false;  // wait for memory
    cudaError_t e;
    int rc;
    if (need_plan) {
        res = std::make_shared<Resident>();
        if ((e = cudaStreamCreateWithFlags(&res->stream, cudaStreamNonBlocking)) != cudaSuccess) {
            fail_job(j, PRISM_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            return true;
        }
        prism_grid g = j->grid;
        g.slice_dz = j->slice_dz.empty() ? nullptr : j->slice_dz.data();
        const size_t plan_budget = budget ? budget - used - (need - plan_bytes_estimate(j->grid)) : 0;
        if ((rc = prism_plan_create(&g, plan_budget, res->stream, &res->plan)) != PRISM_OK) {
            cudaStreamDestroy(res->stream);
            fail_job(j, rc, prism_last_error());
            return true;
        }
        prism_info info;
        prism_plan_info(res->plan, &info);
        res->bytes = info.device_bytes;
        res->grid = j->grid;
        res->slice_dz = j->slice_dz;
        used += res->bytes;
        if (j->key)
            cache[j->key] = res;
        else
            anonymous.push_back(res);
    } else {
        j->reused = 1;
    }
    res->users++;
    res->last_use = Clock::now();
    j->res = res;
    j->t_admit = Clock::now();
    cudaStream_t st = res->stream;
    const size_t extra = j->out_bytes + j->x0.size() * 16 + 4096;
    used += extra;
    peak_used = std::max(peak_used, used);
    auto bail = [&](int code, const std::string &msg) {
        fail_job(j, code, msg);
        if (j->ev_start) cudaEventDestroy(j->ev_start);
        j->ev_start = nullptr;
        res->users--;
        used -= extra;
        if (j->out_dev) cudaFreeAsync(j->out_dev, st);
        if (j->out_pinned) cudaFreeHost(j->out_pinned);
        if (!j->key) {  // a private plan dies with its request
            anonymous.erase(std::remove(anonymous.begin(), anonymous.end(), res), anonymous.end());
            prism_plan_destroy(res->plan);
            cudaStreamDestroy(res->stream);
            used -= res->bytes;
        }
        j->res.reset();
        return true;
    };
    if ((e = cudaMallocAsync(&j->out_dev, j->out_bytes ? j->out_bytes : 16, st)) != cudaSuccess)
        return bail(PRISM_ERR_CUDA, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    if ((e = cudaMallocHost(&j->out_pinned, j->out_bytes ? j->out_bytes : 16)) != cudaSuccess)
        return bail(PRISM_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    if (ref && (cudaEventCreate(&j->ev_start) != cudaSuccess || cudaEventRecord(j->ev_start, st) != cudaSuccess)) {
        if (j->ev_start) cudaEventDestroy(j->ev_start);
        j->ev_start = nullptr;
    }
    if (!res->built) {
        if ((rc = prism_build_smatrix_host(res->plan, j->V_host)) != PRISM_OK) return bail(rc, prism_last_error());
        res->built = true;
    }
    prism_scan sc{j->px, j->py, j->x0.data(), j->y0.data()};
    if ((rc = prism_scan_run(res->plan, &j->probe, &sc, &j->det, j->out_dev)) != PRISM_OK) return bail(rc, prism_last_error());
    if (j->out_bytes && (e = cudaMemcpyAsync(j->out_pinned, j->out_dev, j->out_bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return bail(PRISM_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    if ((e = cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(j->done, st)) != cudaSuccess)
        return bail(PRISM_ERR_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
    if (j->ev_start && (cudaEventCreate(&j->ev_end) != cudaSuccess || cudaEventRecord(j->ev_end, st) != cudaSuccess)) {
        if (j->ev_end) cudaEventDestroy(j->ev_end);
        j->ev_end = nullptr;
    }
    running.push_back(j);
    admitted++;
    return true;
}

void prism_server::reap() {
    for (auto it = running.begin(); it != running.end();) {
        auto &j = *it;
        const cudaError_t q = cudaEventQuery(j->done);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        if (q != cudaSuccess) {
            j->status = PRISM_ERR_CUDA;
            j->error = std::string("request failed on the device: ") + cudaGetErrorString(q);
        } else if (j->cancelled) {
            j->status = PRISM_ERR_CANCELLED;
            j->error = "request " + std::to_string(j->ticket) + " was cancelled (its result was discarded)";
        } else if (j->out_bytes) {
            std::memcpy(j->out_host, j->out_pinned, j->out_bytes);
        }
        if (q == cudaSuccess && j->ev_start && j->ev_end) {
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, ref, j->ev_start) == cudaSuccess && cudaEventElapsedTime(&b, ref, j->ev_end) == cudaSuccess) {
                j->dev_start_ms = a;
                j->dev_end_ms = b;
            }
        }
        if (j->ev_start) cudaEventDestroy(j->ev_start);
        if (j->ev_end) cudaEventDestroy(j->ev_end);
        j->ev_start = j->ev_end = nullptr;
        cudaEventDestroy(j->done);
        cudaFreeAsync(j->out_dev, j->res->stream);
        cudaFreeHost(j->out_pinned);
        used -= j->out_bytes + j->x0.size() * 16 + 4096;
        j->res->users--;
        j->res->last_use = Clock::now();
        if (!j->key) {  // private plan: release it
            auto &an = anonymous;
            an.erase(std::remove(an.begin(), an.end(), j->res), an.end());
            prism_plan_destroy(j->res->plan);
            cudaStreamDestroy(j->res->stream);
            used -= j->res->bytes;
        }
        j->res.reset();
        j->finished = true;
        j->t_done = Clock::now();
        completed++;
        it = running.erase(it);
        cv_done.notify_all();
    }
}

void prism_server::loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    while (true) {
        reap();
        // admit in arrival order; a request that does not fit yet does not block later ones
        for (auto it = pending.begin(); it != pending.end() && (int)running.size() < max_inflight;) {
            if (try_admit(*it))
                it = pending.erase(it);
            else
                ++it;
        }
        if (stop && pending.empty() && running.empty()) break;
        // bounded wait: new work, or poll the in-flight requests again shortly
        cv_work.wait_for(lock, std::chrono::microseconds(running.empty() ? 2000 : 50));
    }
}

// ------------------------------------------------------------------ C ABI
extern "C" int prism_server_create(size_t hbm_budget_bytes, int max_inflight, prism_server **out) {
    if (!out) return prism::internal_fail(PRISM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (max_inflight < 1 || max_inflight > 256) return prism::internal_fail(PRISM_ERR_INVALID, "max_inflight must be in [1, 256]");
    prism_server *S = new prism_server();
    S->budget = hbm_budget_bytes;
    S->max_inflight = max_inflight;
    cudaGetDevice(&S->device);
    // device-time origin for the requests' timestamps (recorded once, completed before any request)
    cudaStream_t s0 = nullptr;
    if (cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) == cudaSuccess) {
        if (cudaEventCreate(&S->ref) != cudaSuccess || cudaEventRecord(S->ref, s0) != cudaSuccess ||
            cudaStreamSynchronize(s0) != cudaSuccess) {
            if (S->ref) cudaEventDestroy(S->ref);
            S->ref = nullptr;
        }
        cudaStreamDestroy(s0);
    }
    S->worker = std::thread([S] { S->loop(); });
    *out = S;
    return PRISM_OK;
}

extern "C" int prism_server_submit(prism_server *S, const prism_request *r, unsigned long long *ticket) {
    if (!S || !r || !ticket) return prism::internal_fail(PRISM_ERR_INVALID, "NULL argument");
    if (!r->V_host) return prism::internal_fail(PRISM_ERR_INVALID, "V_host is NULL");
    if (r->scan.px < 0 || r->scan.py < 0 || ((long long)r->scan.px * r->scan.py > 0 && (!r->scan.x0 || !r->scan.y0)))
        return prism::internal_fail(PRISM_ERR_INVALID, "bad scan");
    if (r->det.nbins < 1 || !r->out_host) return prism::internal_fail(PRISM_ERR_INVALID, "bad detector or out_host");
    auto j = std::make_shared<Job>();
    j->grid = r->grid;
    if (r->grid.slice_dz) j->slice_dz.assign(r->grid.slice_dz, r->grid.slice_dz + r->grid.n_slices);
    j->grid.slice_dz = nullptr;
    j->V_host = r->V_host;
    j->key = r->smatrix_key;
    j->probe = r->probe;
    j->px = r->scan.px;
    j->py = r->scan.py;
    const size_t n = (size_t)r->scan.px * r->scan.py;
    j->x0.assign(r->scan.x0, r->scan.x0 + n);
    j->y0.assign(r->scan.y0, r->scan.y0 + n);
    j->det = r->det;
    j->out_host = r->out_host;
    j->out_bytes = n * r->det.nbins * sizeof(float);
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) return prism::internal_fail(PRISM_ERR_INVALID, "server is shutting down");
        j->ticket = S->next_ticket++;
        S->jobs[j->ticket] = j;
        S->pending.push_back(j);
    }
    S->cv_work.notify_one();
    *ticket = j->ticket;
    return PRISM_OK;
}

extern "C" int prism_server_wait(prism_server *S, unsigned long long ticket, double timeout_s, prism_request_stats *stats) {
    if (!S) return prism::internal_fail(PRISM_ERR_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return prism::internal_fail(PRISM_ERR_INVALID, "unknown ticket");
    auto j = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!j->finished) {
        if (S->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && !j->finished)
            return prism::internal_fail(PRISM_ERR_DEVICE, ("timed out waiting for request " + std::to_string(ticket)).c_str());
    }
    if (stats) {
        stats->queued_ms = ms_since(j->t_submit, j->t_admit);
        stats->total_ms = ms_since(j->t_submit, j->t_done);
        stats->smatrix_reused = j->reused;
        stats->status = j->status;
        stats->device_start_ms = j->dev_start_ms;
        stats->device_end_ms = j->dev_end_ms;
    }
    S->jobs.erase(it);
    if (j->status != PRISM_OK) return prism::internal_fail(j->status, j->error.c_str());
    return PRISM_OK;
}

extern "C" int prism_server_stats(prism_server *S, prism_server_info *out) {
    if (!S || !out) return prism::internal_fail(PRISM_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    out->pending = (int)S->pending.size();
    out->running = (int)S->running.size();
    out->resident = (int)S->cache.size();
    out->admitted = S->admitted;
    out->completed = S->completed;
    out->used_bytes = S->used;
    out->peak_bytes = S->peak_used;
    return PRISM_OK;
}

extern "C" int prism_server_cancel(prism_server *S, unsigned long long ticket) {
    if (!S) return prism::internal_fail(PRISM_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end() || it->second->finished)
        return prism::internal_fail(PRISM_ERR_INVALID, ("no queued or running request " + std::to_string(ticket)).c_str());
    auto j = it->second;
    auto q = std::find(S->pending.begin(), S->pending.end(), j);
    if (q != S->pending.end()) {  // still queued: leaves the queue now
        S->pending.erase(q);
        S->fail_job(j, PRISM_ERR_CANCELLED, "request " + std::to_string(ticket) + " was cancelled before it ran");
        return PRISM_OK;
    }
    j->cancelled = true;  // running: the worker discards its result when its device work is done
    return PRISM_OK;
}

extern "C" void prism_server_destroy(prism_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_one();
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->cache) {
        prism_plan_destroy(kv.second->plan);
        cudaStreamDestroy(kv.second->stream);
    }
    if (S->ref) cudaEventDestroy(S->ref);
    delete S;
}
