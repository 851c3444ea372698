// Request server: continuous admission of forward + adjoint rollouts by slot
// and HBM budget, with host-side preparation pipelined ahead of the GPU.
//
//   submit --> [prep threads: mesh ordering, factor, fronts, footprint] -->
//   ready queue (submission order) --> [slot threads: admit when a slot is free
//   and the footprint fits the budget; upload, rollout, backward on the slot's
//   stream; free] --> results, collected by dc_server_wait.
//
// Every request is its own one-instance context, so its numbers do not depend
// on what else runs (bitwise equal to running it alone).
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "dc_ctx.h"

namespace {

struct Request {
    int64_t ticket = 0;
    std::vector<double> rest, x0, v0, gx, gv;
    std::vector<int32_t> tris, pins;
    int n_steps = 0;
    dc_params prm{};
    bool solo = false;   // runs in a context of its own (after its batch failed)
    // results
    bool done = false;
    dc_status status = DC_OK;
    std::string err;
    int slot = -1;
    std::vector<double> xN, vN, dx0, dv0;
    double dth[3] = {0, 0, 0};
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t bytes = 0, peak = 0;
    long long adj_iters = 0;
};

// One or more requests prepared as one context (a batch when max_batch > 1).
struct Job {
    std::vector<Request*> reqs;
    dc_ctx* c = nullptr;
    MeshPrep mp;
    ParamPrep pp;
    size_t bytes = 0;
};

}  // namespace

struct dc_server {
    dc_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv;     // any state change
    std::deque<Request*> to_prep;
    std::map<int64_t, Job*> ready;       // prepared, by the ticket of their first request
    std::map<int64_t, Request*> all;
    int64_t next_ticket = 1;
    size_t reserved = 0, peak_reserved = 0;
    int64_t in_flight = 0, peak_in_flight = 0, submitted = 0, completed = 0, failed = 0, steps = 0;
    int64_t batch_retries = 0;   // batches whose requests were run again one by one
    int preparing = 0;
    bool stop = false;
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;
    std::vector<double*> pinned;
    size_t pinned_doubles = 0;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void finish(dc_server* s, Request* r, dc_status st, const std::string& err) {
    // caller holds s->mu
    r->status = st;
    r->err = err;
    r->done = true;
    r->t_done = s->now();
    if (st == DC_OK) {
        s->completed++;
        s->steps += r->n_steps;
    } else {
        s->failed++;
    }
    s->cv.notify_all();
}

void finish_job(dc_server* s, Job* j, dc_status st, const std::string& err) {
    for (Request* r : j->reqs) finish(s, r, st, err);
}

// The oldest queued request and up to max_batch - 1 others whose shared
// parameters agree with it leave the preparation queue together (caller holds
// s->mu).  A batch runs as many steps as its longest request, so among the
// compatible requests those with the step counts closest to the first one's are
// taken (the older one on ties).  Solo requests go alone.
std::vector<Request*> take_group(dc_server* s) {
    std::vector<Request*> g;
    const int cap = std::max(1, s->cfg.max_batch);
    g.push_back(s->to_prep.front());
    s->to_prep.pop_front();
    if (g[0]->solo || cap == 1) return g;
    std::vector<std::pair<long long, size_t>> cand;   // (|step difference|, queue position)
    for (size_t q = 0; q < s->to_prep.size(); ++q) {
        const Request* r = s->to_prep[q];
        if (!r->solo && dc_same_batch_fields(r->prm, g[0]->prm))
            cand.push_back({std::llabs((long long)r->n_steps - g[0]->n_steps), q});
    }
    const size_t take = std::min(cand.size(), (size_t)cap - 1);
    std::partial_sort(cand.begin(), cand.begin() + take, cand.end());
    std::vector<size_t> pos;
    for (size_t k = 0; k < take; ++k) pos.push_back(cand[k].second);
    std::sort(pos.begin(), pos.end());
    for (size_t k = pos.size(); k-- > 0;) {
        g.push_back(s->to_prep[pos[k]]);
        s->to_prep.erase(s->to_prep.begin() + (long)pos[k]);
    }
    std::sort(g.begin() + 1, g.end(), [](const Request* a, const Request* b) { return a->ticket < b->ticket; });
    return g;
}

// Host preparation of one job (meshes, ordering, factorisation, fronts,
// footprint), without the server lock.  On failure j->c stays null.
dc_status prepare_job(Job* j, std::string& err) {
    const int B = (int)j->reqs.size();
    dc_ctx* c = new dc_ctx();
    c->async_alloc = true;
    c->blocking_sync = true;
    c->ihm.resize(B);
    for (int i = 0; i < B; ++i) {
        Request* r = j->reqs[i];
        err = dc_build_mesh(c->ihm[i], (int)(r->rest.size() / 3), r->rest.data(), (int)(r->tris.size() / 3),
                            r->tris.data(), (int)r->pins.size(), r->pins.empty() ? nullptr : r->pins.data());
        if (!err.empty()) {
            delete c;
            return DC_ERR_INVALID;
        }
    }
    prep_mesh_host(c, j->mp);
    std::vector<dc_params> q;
    int max_steps = 0;
    for (Request* r : j->reqs) {
        q.push_back(r->prm);
        max_steps = std::max(max_steps, r->n_steps);
    }
    dc_status st = prep_params_host(c, q, j->pp);
    if (st) {
        err = c->err;
        delete c;
        return st;
    }
    j->c = c;
    j->bytes = estimate_device_bytes(c, j->mp, j->pp, max_steps) + 4 * (size_t)B + 64;
    return DC_OK;
}

void prep_loop(dc_server* s) {
    for (;;) {
        std::vector<Request*> group;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // while stopping, a thread leaves only once nothing is queued and no
            // job runs (a failed batch puts its requests back in the queue)
            s->cv.wait(lk, [&] {
                const bool can = !s->to_prep.empty() && (int)s->ready.size() + s->preparing < s->cfg.max_prepared;
                return can || (s->stop && s->to_prep.empty() && s->in_flight == 0);
            });
            if (s->to_prep.empty()) return;   // stop with nothing left
            group = take_group(s);
            s->preparing++;
        }
        // a group that fails is prepared again request by request, so that a bad
        // request fails alone and the others still run
        std::vector<Job*> jobs(1, new Job());
        jobs[0]->reqs = group;
        std::vector<dc_status> st(1);
        std::vector<std::string> err(1);
        st[0] = prepare_job(jobs[0], err[0]);
        if (st[0] && group.size() > 1) {
            delete jobs[0];
            jobs.clear();
            st.clear();
            err.clear();
            for (Request* r : group) {
                Job* j = new Job();
                j->reqs.push_back(r);
                std::string e;
                st.push_back(prepare_job(j, e));
                err.push_back(e);
                jobs.push_back(j);
            }
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->preparing--;
        for (size_t q = 0; q < jobs.size(); ++q) {
            Job* j = jobs[q];
            if (st[q]) {
                finish_job(s, j, st[q], err[q]);
                delete j;
            } else if (j->bytes > (size_t)s->cfg.hbm_budget_bytes) {
                delete j->c;
                finish_job(s, j, DC_ERR_OOM,
                           "request needs " + std::to_string(j->bytes) + " device bytes, more than the server's budget");
                delete j;
            } else {
                s->ready[j->reqs[0]->ticket] = j;
            }
        }
        s->cv.notify_all();
    }
}

// Runs one admitted job on the slot's stream; returns the context's status, and
// in inst[i] that of request i (a non-converged adjoint concerns only the
// instances whose steps stopped above adj_tol).
dc_status run_job(dc_server* s, Job* j, int slot, std::string& err, std::vector<dc_status>& inst) {
    dc_ctx* c = j->c;
    const int B = (int)j->reqs.size();
    c->stream = s->streams[slot];
    c->device = s->cfg.device;
    c->kt.stream = c->stream;
    c->hpin = s->pinned[slot];
    c->hpin_cap = s->pinned_doubles;
    c->hpin_external = true;
    dc_status st = upload_mesh(c, j->mp);
    if (!st) st = upload_params(c, j->pp);
    j->mp = MeshPrep();
    j->pp = ParamPrep();
    // concatenated inputs; instance i's nodes are [ext_off_i, ext_off_i + m_i)
    std::vector<double> x0, v0, gx, gv;
    std::vector<int32_t> steps(B);
    bool any_gv = false;
    int max_steps = 0;
    for (int i = 0; i < B; ++i) {
        Request* r = j->reqs[i];
        x0.insert(x0.end(), r->x0.begin(), r->x0.end());
        v0.insert(v0.end(), r->v0.begin(), r->v0.end());
        gx.insert(gx.end(), r->gx.begin(), r->gx.end());
        any_gv |= !r->gv.empty();
        steps[i] = r->n_steps;
        max_steps = std::max(max_steps, r->n_steps);
    }
    if (any_gv)
        for (int i = 0; i < B; ++i) {
            Request* r = j->reqs[i];
            if (r->gv.empty())
                gv.insert(gv.end(), r->x0.size(), 0.0);
            else
                gv.insert(gv.end(), r->gv.begin(), r->gv.end());
        }
    const size_t n3 = x0.size();
    std::vector<double> xN(n3), vN(n3), dx0(n3), dv0(n3), dth(3 * (size_t)B);
    if (!st && B > 1) st = dc_set_instance_steps(c, steps.data());
    if (!st) st = dc_rollout(c, max_steps, x0.data(), v0.data(), xN.data(), vN.data(), nullptr);
    if (!st)
        st = dc_backward(c, gx.data(), any_gv ? gv.data() : nullptr, nullptr, dx0.data(), dv0.data(), dth.data());
    if (st) err = c->err;
    inst.assign(B, st);
    if (st == DC_ERR_NONCONVERGED)
        for (int i = 0; i < B; ++i)
            inst[i] = (i < (int)c->inst_noncv.size() && c->inst_noncv[i] > 0) ? DC_ERR_NONCONVERGED : DC_OK;
    for (int i = 0; i < B; ++i) {
        Request* r = j->reqs[i];
        const size_t lo = 3 * (size_t)c->inst[i].ext_off, hi = lo + r->x0.size();
        r->xN.assign(xN.begin() + lo, xN.begin() + hi);
        r->vN.assign(vN.begin() + lo, vN.begin() + hi);
        r->dx0.assign(dx0.begin() + lo, dx0.begin() + hi);
        r->dv0.assign(dv0.begin() + lo, dv0.begin() + hi);
        for (int k = 0; k < 3; ++k) r->dth[k] = dth[3 * i + k];
        r->adj_iters = c->adj_iters;
        r->peak = c->dev_peak;
        r->bytes = j->bytes;
    }
    dc_destroy(c);
    j->c = nullptr;
    return st;
}

void slot_loop(dc_server* s, int slot) {
    cudaSetDevice(s->cfg.device);
    for (;;) {
        Job* j;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (!s->ready.empty()) {
                    Job* h = s->ready.begin()->second;
                    if (s->reserved + h->bytes <= (size_t)s->cfg.hbm_budget_bytes) return true;
                }
                return s->stop && s->ready.empty() && s->to_prep.empty() && s->preparing == 0 && s->in_flight == 0;
            });
            if (s->ready.empty()) return;
            j = s->ready.begin()->second;
            s->ready.erase(s->ready.begin());
            s->reserved += j->bytes;
            s->peak_reserved = std::max(s->peak_reserved, s->reserved);
            s->in_flight += (int64_t)j->reqs.size();
            s->peak_in_flight = std::max(s->peak_in_flight, s->in_flight);
            const double t = s->now();
            for (Request* r : j->reqs) {
                r->slot = slot;
                r->t_admit = t;
            }
            s->cv.notify_all();   // a prep thread may now prepare the next job
        }
        std::string err;
        std::vector<dc_status> inst;
        dc_status st = run_job(s, j, slot, err, inst);
        std::lock_guard<std::mutex> lk(s->mu);
        s->reserved -= j->bytes;
        s->in_flight -= (int64_t)j->reqs.size();
        if (st != DC_OK && st != DC_ERR_NONCONVERGED && j->reqs.size() > 1) {
            // one request can fail a whole batch (a non-finite state, say): run
            // each of them again in a context of its own, ahead of the queue
            for (size_t q = j->reqs.size(); q-- > 0;) {
                j->reqs[q]->solo = true;
                s->to_prep.push_front(j->reqs[q]);
            }
            s->batch_retries++;
            s->cv.notify_all();
        } else {
            for (size_t q = 0; q < j->reqs.size(); ++q)
                finish(s, j->reqs[q], inst[q], inst[q] == DC_OK ? std::string() : err);
        }
        delete j;
    }
}

}  // namespace

extern "C" {

dc_status dc_server_create(dc_server** out, const dc_server_config* cfg) {
    if (!out || !cfg || cfg->n_slots < 1 || cfg->n_prep_threads < 1 || cfg->hbm_budget_bytes <= 0 ||
        cfg->max_prepared < 1)
        return DC_ERR_INVALID;
    *out = nullptr;
    if (cudaSetDevice(cfg->device) != cudaSuccess) return DC_ERR_CUDA;
    // keep freed blocks in the stream-ordered pool of this process for the next request
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, cfg->device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    dc_server* s = new dc_server();
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    // pinned host scratch of a slot: what the batched GMRES needs for max_batch
    // instances at the largest restart length (dc_ctx::hpin)
    const size_t mb = (size_t)std::max(1, cfg->max_batch);
    s->pinned_doubles = std::max<size_t>(1024, 3 * 257 * mb + 4 * mb + 64);
    for (int i = 0; i < cfg->n_slots; ++i) {
        cudaStream_t st;
        double* h;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&h, s->pinned_doubles * sizeof(double)) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            for (double* x : s->pinned) cudaFreeHost(x);
            delete s;
            return DC_ERR_CUDA;
        }
        s->streams.push_back(st);
        s->pinned.push_back(h);
    }
    for (int i = 0; i < cfg->n_prep_threads; ++i) s->threads.emplace_back(prep_loop, s);
    for (int i = 0; i < cfg->n_slots; ++i) s->threads.emplace_back(slot_loop, s, i);
    *out = s;
    return DC_OK;
}

dc_status dc_server_submit(dc_server* s, const dc_request* q, int64_t* ticket) {
    if (!s || !q || !ticket || q->n_nodes <= 0 || q->n_tris <= 0 || q->n_pins < 0 || q->n_steps < 0 ||
        !q->rest_pos || !q->tris || (q->n_pins > 0 && !q->pins) || !q->x0 || !q->v0 || !q->dL_dx_final)
        return DC_ERR_INVALID;
    Request* r = new Request();
    const size_t n3 = 3 * (size_t)q->n_nodes;
    r->rest.assign(q->rest_pos, q->rest_pos + n3);
    r->x0.assign(q->x0, q->x0 + n3);
    r->v0.assign(q->v0, q->v0 + n3);
    r->gx.assign(q->dL_dx_final, q->dL_dx_final + n3);
    if (q->dL_dv_final) r->gv.assign(q->dL_dv_final, q->dL_dv_final + n3);
    r->tris.assign(q->tris, q->tris + 3 * (size_t)q->n_tris);
    if (q->n_pins > 0) r->pins.assign(q->pins, q->pins + q->n_pins);
    r->n_steps = q->n_steps;
    r->prm = q->params;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete r;
        return DC_ERR_STATE;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = s->now();
    s->all[r->ticket] = r;
    s->to_prep.push_back(r);
    s->submitted++;
    *ticket = r->ticket;
    s->cv.notify_all();
    return DC_OK;
}

dc_status dc_server_wait(dc_server* s, int64_t ticket, dc_result* out) {
    if (!s || !out) return DC_ERR_INVALID;
    Request* r;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return DC_ERR_INVALID;
        r = it->second;
        s->cv.wait(lk, [&] { return r->done; });
        s->all.erase(it);
    }
    const size_t nb = r->xN.size() * sizeof(double);
    if (r->status == DC_OK) {
        if (out->x_final) std::memcpy(out->x_final, r->xN.data(), nb);
        if (out->v_final) std::memcpy(out->v_final, r->vN.data(), nb);
        if (out->dL_dx0) std::memcpy(out->dL_dx0, r->dx0.data(), nb);
        if (out->dL_dv0) std::memcpy(out->dL_dv0, r->dv0.data(), nb);
    }
    out->status = r->status;
    out->slot = r->slot;
    for (int k = 0; k < 3; ++k) out->dL_dparams[k] = r->dth[k];
    out->t_submit = r->t_submit;
    out->t_admit = r->t_admit;
    out->t_done = r->t_done;
    out->device_bytes = (int64_t)r->bytes;   // the footprint of its job (a batch: all its requests)
    out->device_bytes_peak = (int64_t)r->peak;
    out->adj_iters = r->adj_iters;
    std::snprintf(out->message, sizeof(out->message), "%s", r->err.c_str());
    delete r;
    return DC_OK;
}

dc_status dc_server_get_stats(dc_server* s, dc_server_stats* o) {
    if (!s || !o) return DC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->failed = s->failed;
    o->in_flight = s->in_flight;
    o->peak_in_flight = s->peak_in_flight;
    o->bytes_reserved = (int64_t)s->reserved;
    o->peak_bytes_reserved = (int64_t)s->peak_reserved;
    o->cloth_steps = s->steps;
    o->batch_retries = s->batch_retries;
    return DC_OK;
}

void dc_server_destroy(dc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    for (auto& t : s->threads) t.join();
    for (auto& kv : s->ready) {
        if (kv.second->c) dc_destroy(kv.second->c);
        delete kv.second;
    }
    for (auto& kv : s->all) delete kv.second;
    for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
    for (double* x : s->pinned) cudaFreeHost(x);
    delete s;
}

}  // extern "C"
