// Request server: continuous admission of likelihood (Eq. 1) and cokriging
// (Eq. 3) requests of different sizes on one GPU.
//
// * `slots` worker threads, each with its own context and CUDA stream, so the
//   kernels of concurrent requests overlap on the device.
// * Admission by device memory.  Every worker publishes its footprint: idle,
//   the bytes its context holds (cached workspaces and kept factors) plus its
//   staging buffers; running, that plus an upper bound of what the request
//   may allocate.  A free worker takes the oldest queued request for which the
//   sum of footprints stays within the budget, dropping its own cached
//   workspaces first when that is what makes the request fit; when a request
//   cannot be admitted, idle workers drop theirs.  Later, smaller requests may
//   start while a large one waits.
// * A likelihood request may keep its factor on the device under a dataset
//   key; cokriging requests for that key run on the worker that owns the
//   factor (affinity), reuse it, and the last one may release it.
// * Every result is computed by the same kernels with the same reduction
//   order whatever else runs: a request's result is the same alone and in the mix.
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "geo_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    long long id;
    int kind, keep, release, escalate;
    long long dataset;
    int n, m, p;
    std::vector<double> locs, z, new_locs, sigma2, nu, beta;
    double a;
    geo_opts opts;
    double *zhat_out;   // caller's host buffer (PREDICT)
    size_t bytes;       // upper bound of the device bytes the request may add
    int affinity;       // worker index, or -1
    double t_submit;
};

struct Worker;

}  // namespace

struct geo_server {
    int device = 0;
    size_t budget = 0, reserved = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::vector<geo_result> done;
    std::vector<Worker *> workers;
    std::map<long long, std::pair<int, geo_factor *>> factors;   // dataset -> (worker, factor)
    std::atomic<long long> next_id{1};
    int inflight = 0;
    bool stop = false;
    bool starved = false;   // a queued request did not fit: idle workers drop their caches
};

namespace {

struct Worker {
    int index;
    geo_server *srv;
    geo_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread th;
    double *d_locs = nullptr, *d_z = nullptr, *d_new = nullptr, *d_zhat = nullptr;
    size_t cap_locs = 0, cap_z = 0, cap_new = 0, cap_zhat = 0;
    // published under the server lock
    size_t foot = 0;     // device bytes held now (running: plus the request's bound)
    size_t kept = 0;     // bytes of the factors kept in this worker's context
    bool busy = false;
};

size_t staging_bytes(const Worker *w) { return sizeof(double) * (w->cap_locs + w->cap_z + w->cap_new + w->cap_zhat); }

// Upper bound of the device bytes a request adds to its worker (staging
// buffers included).  Predictions: the weight vector w = Sigma^-1 Z (computed
// once per factor) and the new locations and predictions.
size_t request_bytes(const geo_server *S, const Req &r, int N_factor) {
    if (r.kind == GEO_REQ_PREDICT)
        return sizeof(double) * ((size_t)N_factor + 2 * (size_t)r.m + (size_t)GEO_PMAX * r.m) + 4096;
    const size_t N = (size_t)r.p * r.n;
    return loglik_device_bytes(S->device, r.n, r.p, &r.opts) + sizeof(double) * (2 * (size_t)r.n + N);
}

bool grow(double **p, size_t *cap, size_t n) {
    if (*cap >= n) return true;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    *cap = n;
    return true;
}

void run_request(Worker *w, Req *r, geo_result *res) {
    geo_server *S = w->srv;
    res->id = r->id;
    res->kind = r->kind;
    res->dataset = r->dataset;
    res->status = GEO_OK;
    res->loglik = 0.0;
    geo_theta th{r->p, r->sigma2.data(), r->nu.data(), r->beta.data(), r->a};
    if (r->kind == GEO_REQ_LOGLIK) {
        const size_t N = (size_t)r->p * r->n;
        if (!grow(&w->d_locs, &w->cap_locs, 2 * (size_t)r->n) || !grow(&w->d_z, &w->cap_z, N)) {
            res->status = GEO_ENOMEM;
            return;
        }
        cudaMemcpyAsync(w->d_locs, r->locs.data(), sizeof(double) * 2 * r->n, cudaMemcpyHostToDevice, w->stream);
        cudaMemcpyAsync(w->d_z, r->z.data(), sizeof(double) * N, cudaMemcpyHostToDevice, w->stream);
        geo_factor *f = nullptr;
        double ll = 0.0;
        int info = 0;
        res->prec = r->opts.prec;
        res->status = geo_loglik(w->ctx, w->d_locs, r->n, w->d_z, &th, &r->opts, &ll, r->keep ? &f : nullptr, &info,
                                 w->stream);
        if (res->status == GEO_ENOTSPD && r->escalate && r->opts.prec != GEO_PREC_FP64) {
            // the reduced form lost positive definiteness: the FP64 form decides
            geo_opts o64;
            geo_opts_default(&o64);
            o64.nb = 0;
            o64.morton = r->opts.morton;
            res->prec = GEO_PREC_FP64;
            res->status = geo_loglik(w->ctx, w->d_locs, r->n, w->d_z, &th, &o64, &ll, r->keep ? &f : nullptr, &info,
                                     w->stream);
        }
        res->loglik = ll;
        if (r->keep) {
            // a failed likelihood leaves a null factor: its predictions complete with an error
            size_t fb = 0;
            if (res->status == GEO_OK && f) {
                geo_factor_stats st;
                geo_factor_stats_get(f, &st);
                fb = (size_t)st.device_bytes;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            S->factors[r->dataset] = {w->index, (res->status == GEO_OK) ? f : nullptr};
            w->kept += fb;
        }
    } else {
        geo_factor *f = nullptr;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            auto it = S->factors.find(r->dataset);
            if (it != S->factors.end()) f = it->second.second;
        }
        if (!f) {
            res->status = GEO_EINVAL;
            if (r->release) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->factors.erase(r->dataset);
            }
            return;
        }
        geo_factor_stats fs;
        geo_factor_stats_get(f, &fs);
        const size_t pm = (size_t)fs.p * r->m;
        if (!grow(&w->d_new, &w->cap_new, 2 * (size_t)r->m) || !grow(&w->d_zhat, &w->cap_zhat, pm)) {
            res->status = GEO_ENOMEM;
            return;
        }
        cudaMemcpyAsync(w->d_new, r->new_locs.data(), sizeof(double) * 2 * r->m, cudaMemcpyHostToDevice, w->stream);
        res->status = geo_predict(w->ctx, f, w->d_new, r->m, w->d_zhat, w->stream);
        if (res->status == GEO_OK && r->zhat_out)
            cudaMemcpyAsync(r->zhat_out, w->d_zhat, sizeof(double) * pm, cudaMemcpyDeviceToHost, w->stream);
        cudaStreamSynchronize(w->stream);
        if (r->release) {
            geo_factor_stats st;
            geo_factor_stats_get(f, &st);
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->factors.erase(r->dataset);
                w->kept -= std::min(w->kept, (size_t)st.device_bytes);
            }
            geo_factor_free(f);
        }
    }
}

// Publish the worker's idle footprint (called with the lock held).
void publish_idle(Worker *w) {
    w->foot = ctx_device_bytes(w->ctx) + staging_bytes(w);
    w->busy = false;
}

void trim_unlocked(Worker *w, std::unique_lock<std::mutex> &lk) {
    lk.unlock();
    ctx_trim(w->ctx, w->stream);
    lk.lock();
    publish_idle(w);
}

void worker_loop(Worker *w) {
    geo_server *S = w->srv;
    cudaSetDevice(S->device);
    for (;;) {
        Req *r = nullptr;
        bool trim_first = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop && S->queue.empty()) return;
                size_t others = 0;
                for (Worker *v : S->workers)
                    if (v != w) others += v->foot;
                const size_t cached = w->foot - std::min(w->foot, w->kept + staging_bytes(w));
                // the oldest request that is routed here (or anywhere) and fits in the budget
                for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
                    Req *q = *it;
                    if (q->affinity >= 0 && q->affinity != w->index) continue;
                    int Nf = 0;
                    if (q->kind == GEO_REQ_PREDICT) {
                        auto f = S->factors.find(q->dataset);
                        if (f == S->factors.end()) continue;   // its factor is not ready yet
                        q->affinity = f->second.first;
                        if (q->affinity != w->index) continue;
                        if (f->second.second) {
                            geo_factor_stats st;
                            geo_factor_stats_get(f->second.second, &st);
                            Nf = st.N;
                        }
                        q->bytes = request_bytes(S, *q, Nf);
                    }
                    if (S->budget) {
                        if (others + w->foot + q->bytes > S->budget) {
                            if (others + (w->foot - cached) + q->bytes > S->budget) {
                                S->starved = true;
                                continue;
                            }
                            trim_first = true;
                        }
                    }
                    r = q;
                    S->queue.erase(it);
                    w->foot += q->bytes;
                    w->busy = true;
                    S->reserved = others + w->foot;
                    S->inflight += 1;
                    break;
                }
                if (r) break;
                if (S->starved && cached > 0) {
                    // another request waits for memory: give back this idle worker's cache
                    trim_unlocked(w, lk);
                    S->starved = false;
                    S->cv_work.notify_all();
                    continue;
                }
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
        if (trim_first) ctx_trim(w->ctx, w->stream);
        geo_result res;
        memset(&res, 0, sizeof(res));
        res.t_submit = r->t_submit;
        res.t_start = now_s();
        run_request(w, r, &res);
        res.t_end = now_s();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            publish_idle(w);
            if (S->starved) {
                trim_unlocked(w, lk);
                S->starved = false;
            }
            size_t tot = 0;
            for (Worker *v : S->workers) tot += v->foot;
            S->reserved = tot;
            S->inflight -= 1;
            S->done.push_back(res);
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
        delete r;
    }
}

}  // namespace

extern "C" {

int geo_server_create(geo_server **out, int device, size_t hbm_budget_bytes, int slots) {
    if (!out || slots < 1 || slots > 64) return GEO_EINVAL;
    *out = nullptr;
    geo_server *S = new geo_server();
    S->device = device;
    S->budget = hbm_budget_bytes;
    for (int k = 0; k < slots; ++k) {
        Worker *w = new Worker();
        w->index = k;
        w->srv = S;
        int rc = geo_create(&w->ctx, device, 0);
        if (rc != GEO_OK) {
            delete w;
            geo_server_destroy(S);
            return rc;
        }
        int cur;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            geo_destroy(w->ctx);
            delete w;
            geo_server_destroy(S);
            return GEO_ECUDA;
        }
        cudaSetDevice(cur);
        S->workers.push_back(w);
    }
    for (Worker *w : S->workers) w->th = std::thread(worker_loop, w);
    *out = S;
    return GEO_OK;
}

int geo_server_submit(geo_server *S, const geo_request *q, double *zhat_host, long long *id) {
    if (!S || !q) return GEO_EINVAL;
    Req *r = new Req();
    r->id = S->next_id++;
    r->kind = q->kind;
    r->keep = q->keep;
    r->release = q->release;
    r->escalate = q->escalate;
    r->dataset = q->dataset;
    r->n = q->n;
    r->m = q->m;
    r->zhat_out = zhat_host;
    r->affinity = -1;
    r->t_submit = now_s();
    if (q->kind == GEO_REQ_LOGLIK) {
        const int p = q->theta.p;
        if (p < 1 || p > GEO_PMAX || q->n <= 0 || !q->locs_host || !q->z_host) {
            delete r;
            return GEO_EINVAL;
        }
        r->p = p;
        r->locs.assign(q->locs_host, q->locs_host + 2 * (size_t)q->n);
        r->z.assign(q->z_host, q->z_host + (size_t)p * q->n);
        r->sigma2.assign(q->theta.sigma2, q->theta.sigma2 + p);
        r->nu.assign(q->theta.nu, q->theta.nu + p);
        r->beta.assign((size_t)p * p, 0.0);
        for (int i = 0; i < p; ++i) r->beta[i * p + i] = 1.0;
        if (q->theta.beta) r->beta.assign(q->theta.beta, q->theta.beta + (size_t)p * p);
        r->a = q->theta.a;
        if (q->opts)
            r->opts = *q->opts;
        else
            geo_opts_default(&r->opts);
    } else if (q->kind == GEO_REQ_PREDICT) {
        if (q->m <= 0 || !q->new_locs_host) {
            delete r;
            return GEO_EINVAL;
        }
        r->p = GEO_PMAX;
        r->new_locs.assign(q->new_locs_host, q->new_locs_host + 2 * (size_t)q->m);
        geo_opts_default(&r->opts);
    } else {
        delete r;
        return GEO_EINVAL;
    }
    r->bytes = request_bytes(S, *r, 0);
    if (S->budget && r->kind == GEO_REQ_LOGLIK && r->bytes > S->budget) {
        delete r;
        return GEO_ENOMEM;
    }
    if (id) *id = r->id;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->queue.push_back(r);
    }
    S->cv_work.notify_all();
    return GEO_OK;
}

int geo_server_poll(geo_server *S, geo_result *out, int max, int *nout, int wait_ms) {
    if (!S || !out || !nout || max < 0) return GEO_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
    const int k = std::min<int>(max, (int)S->done.size());
    for (int i = 0; i < k; ++i) out[i] = S->done[i];
    S->done.erase(S->done.begin(), S->done.begin() + k);
    *nout = k;
    return GEO_OK;
}

int geo_server_pending(geo_server *S, int *queued, int *inflight, long long *reserved_bytes) {
    if (!S) return GEO_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int)S->queue.size();
    if (inflight) *inflight = S->inflight;
    if (reserved_bytes) *reserved_bytes = (long long)S->reserved;
    return GEO_OK;
}

int geo_server_profile_read(geo_server *S, geo_kstat *out) {
    if (!S || !out) return GEO_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->queue.empty() || S->inflight) return GEO_EINVAL;
    }
    for (int k = 0; k < GEO_K_COUNT; ++k) out[k] = geo_kstat{0, 0.0, 0.0, 0.0, 0, 0.0};
    for (Worker *w : S->workers) {
        geo_kstat ks[GEO_K_COUNT];
        int rc = geo_profile_read(w->ctx, ks);
        if (rc != GEO_OK) return rc;
        for (int k = 0; k < GEO_K_COUNT; ++k) {
            out[k].launches += ks[k].launches;
            out[k].ms += ks[k].ms;
            out[k].flops += ks[k].flops;
            out[k].bytes += ks[k].bytes;
            out[k].timed += ks[k].timed;
            out[k].tensor_flops += ks[k].tensor_flops;
        }
    }
    return GEO_OK;
}

int geo_server_destroy(geo_server *S) {
    if (!S) return GEO_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // requests that can never run (their factor is gone) are dropped
        for (Req *r : S->queue) delete r;
        S->queue.clear();
    }
    S->cv_work.notify_all();
    for (Worker *w : S->workers)
        if (w->th.joinable()) w->th.join();
    for (auto &kv : S->factors) geo_factor_free(kv.second.second);
    for (Worker *w : S->workers) {
        cudaSetDevice(S->device);
        if (w->d_locs) cudaFree(w->d_locs);
        if (w->d_z) cudaFree(w->d_z);
        if (w->d_new) cudaFree(w->d_new);
        if (w->d_zhat) cudaFree(w->d_zhat);
        if (w->stream) cudaStreamDestroy(w->stream);
        if (w->ctx) geo_destroy(w->ctx);
        delete w;
    }
    delete S;
    return GEO_OK;
}

}  // extern "C"
