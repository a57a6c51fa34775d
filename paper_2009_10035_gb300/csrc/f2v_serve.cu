// f2v_serve.cu -- the job server of include/f2v_serve.h: a host thread that
// admits queued jobs under a device-memory budget, steps every running job
// one epoch at a time in the batched form (one BatchEngine per group of jobs
// sharing model, s, minibatch and precision, each on its own stream), and
// retires jobs that reached their epoch count.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "f2v.h"
#include "f2v_batch_engine.h"
#include "f2v_internal.h"
#include "f2v_serve.h"

using namespace f2v;

namespace {

using Clock = std::chrono::steady_clock;
using GroupKey = std::tuple<int, int, int, int>;   // model, s, minibatch, precision

struct Job {
    f2v_job spec{};
    f2v_job_info info{};
    std::string err;
    int64_t pairs_per_epoch = 0;
    GroupKey key{};
    int engine_id = -1;        // graph id inside the group's engine
};

}  // namespace

struct f2v_server {
    int device = 0;
    size_t budget = 0;
    int max_active = 1;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work;     // the loop waits for submissions
    std::condition_variable cv_done;     // callers wait for completions
    bool stopping = false;
    std::vector<std::unique_ptr<Job>> jobs;   // by id
    std::deque<int64_t> queue;                // queued ids, arrival order
    std::vector<int64_t> running;
    size_t in_use = 0, peak = 0;
    int64_t steps = 0, pairs_done = 0, done = 0, failed = 0;
    double busy_s = 0.0;
    std::string err;

    // CSRs already validated by this server (pointers and sizes): a graph
    // submitted again (the caller keeps it unchanged) is not re-checked
    std::set<std::tuple<const int32_t *, const int32_t *, int32_t, int64_t>> checked;

    // owned by the loop thread only
    std::map<GroupKey, std::unique_ptr<BatchEngine>> groups;
    std::thread loop;

    double now() const
    {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }
};

namespace {

f2v_status sfail(f2v_server *srv, f2v_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (srv) {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->err = buf;
    } else {
        set_global_error(buf);
    }
    return st;
}

// Marks a job finished (caller holds the lock).
void finish(f2v_server *srv, Job &j, f2v_status st, const std::string &msg)
{
    j.info.finish_s = srv->now();
    j.info.status = st;
    j.info.state = (st == F2V_OK) ? F2V_JOB_DONE : F2V_JOB_FAILED;
    j.err = msg;
    if (st == F2V_OK)
        ++srv->done;
    else
        ++srv->failed;
}

BatchEngine *group_engine(f2v_server *srv, const GroupKey &key, std::string *err)
{
    auto it = srv->groups.find(key);
    if (it != srv->groups.end()) return it->second.get();
    std::unique_ptr<BatchEngine> eng(new (std::nothrow) BatchEngine());
    if (!eng) {
        *err = "host allocation failed";
        return nullptr;
    }
    cudaSetDevice(srv->device);
    if (eng->init(std::get<0>(key), std::get<1>(key), std::get<2>(key), std::get<3>(key) == 1,
                  nullptr) != F2V_OK) {
        *err = eng->err();
        return nullptr;
    }
    BatchEngine *p = eng.get();
    srv->groups[key] = std::move(eng);
    return p;
}

void serve_loop(f2v_server *srv)
{
    cudaSetDevice(srv->device);
    std::vector<int64_t> admit;
    for (;;) {
        // ---- admission: arrival order, within the budget and slot count
        admit.clear();
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] {
                return srv->stopping || !srv->queue.empty() || !srv->running.empty();
            });
            if (srv->stopping) break;
            while (!srv->queue.empty() &&
                   (int)(srv->running.size() + admit.size()) < srv->max_active) {
                Job &j = *srv->jobs[(size_t)srv->queue.front()];
                if (srv->in_use + j.info.device_bytes > srv->budget) break;
                srv->in_use += j.info.device_bytes;
                srv->peak = std::max(srv->peak, srv->in_use);
                admit.push_back(srv->queue.front());
                srv->queue.pop_front();
            }
        }
        for (int64_t id : admit) {
            Job &j = *srv->jobs[(size_t)id];
            std::string msg;
            BatchEngine *eng = group_engine(srv, j.key, &msg);
            f2v_status st = F2V_ECUDA;
            int gid = -1;
            if (eng) {
                gid = eng->add_graph(j.spec.row_ptr, j.spec.col_idx, j.spec.n, j.spec.d,
                                     j.spec.seed, j.spec.lr, (int)F2V_LR_LINEAR, j.spec.epochs,
                                     &st, /*validated=*/true);
                if (gid < 0) msg = eng->err();
            }
            std::lock_guard<std::mutex> lk(srv->mu);
            if (gid < 0) {
                srv->in_use -= j.info.device_bytes;
                finish(srv, j, st, msg);
                srv->cv_done.notify_all();
            } else {
                j.engine_id = gid;
                j.info.state = F2V_JOB_RUNNING;
                j.info.admit_s = srv->now();
                srv->running.push_back(id);
            }
        }
        std::vector<int64_t> running;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            running = srv->running;
        }
        if (running.empty()) continue;

        // ---- one step: an epoch of every running job, groups on their streams
        const double t_step = srv->now();
        std::map<GroupKey, f2v_status> gst;
        for (auto &kv : srv->groups)
            if (kv.second->num_graphs() > 0) gst[kv.first] = kv.second->run(1);
        for (auto &kv : gst)
            if (kv.second == F2V_OK) kv.second = srv->groups[kv.first]->sync();
        int64_t step_pairs = 0;
        std::vector<int64_t> finished;
        for (int64_t id : running) {
            Job &j = *srv->jobs[(size_t)id];
            BatchEngine *eng = srv->groups[j.key].get();
            const f2v_status st = gst.count(j.key) ? gst[j.key] : F2V_OK;
            if (st != F2V_OK) {
                finished.push_back(id);
                continue;
            }
            step_pairs += j.pairs_per_epoch;
            j.info.epochs_done = eng->graph_epoch(j.engine_id);
            if (j.info.epochs_done >= j.spec.epochs) finished.push_back(id);
        }
        // ---- retire: results to the callers' buffers, memory back to the budget
        for (int64_t id : finished) {
            Job &j = *srv->jobs[(size_t)id];
            BatchEngine *eng = srv->groups[j.key].get();
            f2v_status st = gst.count(j.key) ? gst[j.key] : F2V_OK;
            std::string msg;
            if (st == F2V_OK) {
                st = eng->get_z(j.engine_id, j.spec.out, (size_t)j.spec.n * j.spec.d);
                if (st == F2V_OK) st = eng->remove_graph(j.engine_id);
            }
            if (st != F2V_OK) msg = eng->err();
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->running.erase(std::find(srv->running.begin(), srv->running.end(), id));
            srv->in_use -= j.info.device_bytes;
            finish(srv, j, st, msg);
        }
        // a group that failed cannot run again: its other jobs fail with it
        for (auto &kv : gst) {
            if (kv.second == F2V_OK) continue;
            srv->groups.erase(kv.first);
        }
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            ++srv->steps;
            srv->pairs_done += step_pairs;
            srv->busy_s += srv->now() - t_step;
        }
        srv->cv_done.notify_all();
    }
    // ---- stop: everything still running or queued fails
    std::lock_guard<std::mutex> lk(srv->mu);
    for (int64_t id : srv->running)
        finish(srv, *srv->jobs[(size_t)id], F2V_ESTATE, "server stopped");
    for (int64_t id : srv->queue)
        finish(srv, *srv->jobs[(size_t)id], F2V_ESTATE, "server stopped");
    srv->running.clear();
    srv->queue.clear();
    srv->cv_done.notify_all();
}

}  // namespace

extern "C" {

f2v_status f2v_server_create(size_t budget_bytes, int32_t max_active, f2v_server **out)
{
    if (!out) return sfail(nullptr, F2V_EINVAL, "out is NULL");
    *out = nullptr;
    if (budget_bytes == 0) return sfail(nullptr, F2V_EINVAL, "budget must be > 0");
    if (max_active < 1) return sfail(nullptr, F2V_EINVAL, "max_active = %d, must be >= 1", max_active);
    f2v_server *srv = new (std::nothrow) f2v_server();
    if (!srv) return sfail(nullptr, F2V_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return sfail(nullptr, F2V_ECUDA, "no CUDA device");
    }
    srv->budget = budget_bytes;
    srv->max_active = max_active;
    srv->t0 = Clock::now();
    try {
        srv->loop = std::thread(serve_loop, srv);
    } catch (...) {
        delete srv;
        return sfail(nullptr, F2V_ENOMEM, "could not start the server thread");
    }
    *out = srv;
    return F2V_OK;
}

f2v_status f2v_server_submit(f2v_server *srv, const f2v_job *job, int64_t *id)
{
    if (!srv || !job || !id) return sfail(srv, F2V_EINVAL, "null argument");
    const f2v_job &j = *job;
    if (j.n < 1) return sfail(srv, F2V_EINVAL, "n = %d, must be >= 1", j.n);
    if (batch_size_index(j.d) < 0)
        return sfail(srv, F2V_EINVAL, "d = %d; jobs take d in {2, 4, 8, 16, 32, 64, 128}", j.d);
    if (j.s < 0 || j.s > 65534) return sfail(srv, F2V_EINVAL, "s = %d, must be in [0, 65534]", j.s);
    if (j.minibatch < 1) return sfail(srv, F2V_EINVAL, "minibatch = %d, must be >= 1", j.minibatch);
    if (!(j.lr > 0.f) || !std::isfinite(j.lr)) return sfail(srv, F2V_EINVAL, "lr must be finite and > 0");
    if (j.epochs < 1) return sfail(srv, F2V_EINVAL, "epochs = %d, must be >= 1", j.epochs);
    if (j.model != F2V_TDIST && j.model != F2V_SIGMOID)
        return sfail(srv, F2V_EINVAL, "unknown model %d", (int)j.model);
    if (j.precision != F2V_FP32 && j.precision != F2V_BF16)
        return sfail(srv, F2V_EINVAL, "unknown precision %d", (int)j.precision);
    if (!j.out) return sfail(srv, F2V_EINVAL, "out is NULL");
    if (!j.row_ptr) return sfail(srv, F2V_EINVAL, "row_ptr is NULL");
    const auto ckey = std::make_tuple(j.row_ptr, j.col_idx, j.n, (int64_t)j.row_ptr[j.n]);
    bool known;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        known = srv->checked.count(ckey) != 0;
    }
    if (!known) {
        if (check_csr(j.row_ptr, j.col_idx, j.n, 0) != F2V_OK)
            return sfail(srv, F2V_EINVAL, "%s", global_error().c_str());
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->checked.insert(ckey);
    }
    std::unique_ptr<Job> p(new (std::nothrow) Job());
    if (!p) return sfail(srv, F2V_ENOMEM, "host allocation failed");
    p->spec = j;
    const int64_t nnz = j.row_ptr[j.n];
    int64_t pairs = 0;
    for (int32_t u = 0; u < j.n; ++u)
        pairs += std::max<int64_t>(1, (int64_t)(j.row_ptr[u + 1] - j.row_ptr[u]) + j.s);
    p->pairs_per_epoch = pairs;
    p->key = GroupKey{(int)j.model, j.s, j.minibatch, (int)j.precision};
    // bytes charged: the graph's arrays and its share of the work tables
    size_t bytes = 0;
    {
        // the estimate needs no device: sizes only
        const size_t es = j.precision == F2V_BF16 ? 2 : 4;
        auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
        bytes = a256((size_t)(j.n + 1) * 4) + a256((size_t)std::max<int64_t>(nnz, 1) * 4) +
                a256((size_t)(j.n + 1) * 8) + 2 * a256((size_t)j.n * j.d * es) +
                a256((size_t)j.n * 4) + (j.precision == F2V_BF16 ? a256((size_t)j.n * j.d * 4) : 0);
        const int64_t items = pairs / 64 + ((int64_t)j.n + j.minibatch - 1) / j.minibatch + 1;
        bytes += (size_t)items * (4 + 8 + 2 * 2 * (size_t)j.d * 4 + 16) +
                 (size_t)(((int64_t)j.n + j.minibatch - 1) / j.minibatch + 1) * 64;
    }
    p->info.state = F2V_JOB_QUEUED;
    p->info.admit_s = -1.0;
    p->info.finish_s = -1.0;
    p->info.pairs = pairs * j.epochs;
    p->info.device_bytes = bytes;
    p->info.status = F2V_OK;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (bytes > srv->budget) {
        srv->err = "job needs more device memory than the whole budget";
        return F2V_EINVAL;
    }
    if (srv->stopping) {
        srv->err = "server stopping";
        return F2V_ESTATE;
    }
    p->info.submit_s = srv->now();
    *id = (int64_t)srv->jobs.size();
    srv->jobs.push_back(std::move(p));
    srv->queue.push_back(*id);
    srv->cv_work.notify_one();
    return F2V_OK;
}

f2v_status f2v_server_job(f2v_server *srv, int64_t id, f2v_job_info *info)
{
    if (!srv || !info) return sfail(srv, F2V_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    if (id < 0 || id >= (int64_t)srv->jobs.size()) {
        srv->err = "no such job";
        return F2V_EINVAL;
    }
    *info = srv->jobs[(size_t)id]->info;
    return F2V_OK;
}

f2v_status f2v_server_wait(f2v_server *srv, int64_t id)
{
    if (!srv) return sfail(srv, F2V_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    if (id < 0 || id >= (int64_t)srv->jobs.size()) {
        srv->err = "no such job";
        return F2V_EINVAL;
    }
    Job &j = *srv->jobs[(size_t)id];
    srv->cv_done.wait(lk, [&] {
        return j.info.state == F2V_JOB_DONE || j.info.state == F2V_JOB_FAILED;
    });
    return j.info.status;
}

f2v_status f2v_server_wait_all(f2v_server *srv)
{
    if (!srv) return sfail(srv, F2V_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv_done.wait(lk, [&] { return srv->done + srv->failed == (int64_t)srv->jobs.size(); });
    return srv->failed ? F2V_ESTATE : F2V_OK;
}

f2v_status f2v_server_get_stats(f2v_server *srv, f2v_server_stats *st)
{
    if (!srv || !st) return sfail(srv, F2V_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    st->submitted = (int64_t)srv->jobs.size();
    st->done = srv->done;
    st->failed = srv->failed;
    st->running = (int64_t)srv->running.size();
    st->queued = (int64_t)srv->queue.size();
    st->steps = srv->steps;
    st->pairs_done = srv->pairs_done;
    st->bytes_in_use = srv->in_use;
    st->peak_bytes = srv->peak;
    st->budget = srv->budget;
    st->busy_s = srv->busy_s;
    return F2V_OK;
}

void f2v_server_destroy(f2v_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
    }
    srv->cv_work.notify_all();
    if (srv->loop.joinable()) srv->loop.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    srv->groups.clear();
    if (prev >= 0) cudaSetDevice(prev);
    delete srv;
}

const char *f2v_server_last_error(const f2v_server *srv)
{
    static thread_local std::string msg;
    if (!srv) {
        msg = global_error();
    } else {
        std::lock_guard<std::mutex> lk(const_cast<f2v_server *>(srv)->mu);
        msg = srv->err;
    }
    return msg.c_str();
}

const char *f2v_server_job_error(f2v_server *srv, int64_t id)
{
    static thread_local std::string msg;
    msg.clear();
    if (srv) {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (id >= 0 && id < (int64_t)srv->jobs.size()) msg = srv->jobs[(size_t)id]->err;
    }
    return msg.c_str();
}

}  // extern "C"
