// Serving loop: simulation requests of different lattice sizes, schemes and
// kernels arrive over time; each admitted case keeps its populations and
// markers resident on the device; admission is by HBM budget and slot count;
// every tick advances all resident cases together with the batched launch
// sequence (continuous batching), retires the finished ones and admits queued
// ones while the device works.  Time-to-result is measured from submission.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <vector>

#include <cuda_runtime.h>

#include "iblbm.h"
#include "internal.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum { Q_QUEUED = 0, Q_RESIDENT = 1, Q_DONE = 2 };

struct Request {
    long long id = 0;
    iblbm_lattice_desc desc{};
    int collision = 0;
    double tau = 0;
    bool has_body = false;
    iblbm_body_desc body{};
    std::vector<double> xy;
    double ds = 0;
    int kernel = 0, scheme = 0;
    int nsteps = 0;
    long long remaining = 0;
    double t_submit = 0, t_done = 0;
    int state = Q_QUEUED;
    int error = 0;
    size_t bytes = 0;
    iblbm_ctx* ctx = nullptr;
    std::vector<double> history;   // force history of the body, 3 per step
};

}  // namespace

struct iblbm_server {
    size_t budget = 0, used = 0;
    int max_slots = 1;
    void* stream = nullptr;
    long long next_id = 1;
    std::deque<Request*> queue;
    std::vector<Request*> resident;
    std::map<long long, Request*> all;
    int use_graphs = 1;   // ticks replay the batch plan's captured step graphs
};

namespace {

size_t estimate(const Request* r) {
    double reach = 0.0;
    const int n = (int)r->xy.size() / 2;
    for (int k = 0; k < n; ++k)
        reach = std::max(reach, std::hypot(r->xy[2 * k] - r->body.xc, r->xy[2 * k + 1] - r->body.yc));
    return iblbm_internal_estimate_bytes(&r->desc, r->has_body ? n : 0, reach, r->kernel, r->body.history_cap);
}

// Creates the case on the device; returns a status code.
int materialise(iblbm_server* s, Request* r) {
    iblbm_lattice_desc d = r->desc;
    d.cuda_stream = s->stream;
    int rc = iblbm_create(&d, r->collision, r->tau, &r->ctx);
    if (rc) return rc;
    if (r->has_body) {
        int id = 0;
        rc = iblbm_add_body(r->ctx, r->xy.data(), (int)r->xy.size() / 2, r->ds, r->kernel, r->scheme, &r->body, &id);
        if (rc) {
            iblbm_destroy(r->ctx);
            r->ctx = nullptr;
            return rc;
        }
    }
    r->bytes = iblbm_device_bytes(r->ctx);
    return IBLBM_OK;
}

// Admits queued requests in arrival order while a slot and the budget allow.
int admit(iblbm_server* s) {
    int admitted = 0;
    while (!s->queue.empty() && (int)s->resident.size() < s->max_slots) {
        Request* r = s->queue.front();
        const size_t need = estimate(r);
        if (s->used + need > s->budget) {
            if (s->resident.empty() && need > s->budget) {   // can never fit
                s->queue.pop_front();
                r->state = Q_DONE;
                r->error = IBLBM_ERR_NOT_ADMITTED;
                r->t_done = now_s();
                continue;
            }
            break;
        }
        s->queue.pop_front();
        const int rc = materialise(s, r);
        if (rc) {
            r->state = Q_DONE;
            r->error = rc;
            r->t_done = now_s();
            continue;
        }
        s->used += r->bytes;
        r->state = Q_RESIDENT;
        s->resident.push_back(r);
        ++admitted;
    }
    return admitted;
}

void retire(iblbm_server* s, Request* r) {
    if (r->has_body && r->error == 0) {
        int got = 0;
        r->history.assign(3 * (size_t)r->nsteps, 0.0);
        const int rc = iblbm_force_history(r->ctx, 0, r->history.data(), r->nsteps, &got);
        if (rc < 0) r->error = rc;
        r->history.resize(3 * (size_t)std::max(got, 0));
    }
    iblbm_destroy(r->ctx);
    r->ctx = nullptr;
    s->used -= std::min(s->used, r->bytes);
    r->state = Q_DONE;
    r->t_done = now_s();
}

}  // namespace

extern "C" {

int iblbm_server_create(size_t hbm_budget, int max_slots, void* stream, iblbm_server** out) {
    if (!out || max_slots < 1 || hbm_budget == 0) return IBLBM_ERR_INVALID_ARG;
    iblbm_server* s = new iblbm_server();
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    s->stream = stream;
    *out = s;
    return IBLBM_OK;
}

void iblbm_server_destroy(iblbm_server* s) {
    if (!s) return;
    for (auto* r : s->resident)
        if (r->ctx) iblbm_destroy(r->ctx);
    for (auto& kv : s->all) delete kv.second;
    delete s;
}

int iblbm_server_submit(iblbm_server* s, const iblbm_lattice_desc* desc, int collision, double tau,
                        const iblbm_body_desc* body, const double* xy, int n, double ds, int kernel, int scheme,
                        int nsteps, long long* req_id) {
    if (!s || !desc || nsteps < 1 || !req_id || n < 0 || (n > 0 && (!xy || !body))) return IBLBM_ERR_INVALID_ARG;
    Request* r = new Request();
    r->id = s->next_id++;
    r->desc = *desc;
    r->collision = collision;
    r->tau = tau;
    r->has_body = n > 0;
    if (n > 0) {
        r->body = *body;
        r->xy.assign(xy, xy + 2 * (size_t)n);
    }
    r->ds = ds;
    r->kernel = kernel;
    r->scheme = scheme;
    r->nsteps = nsteps;
    r->remaining = nsteps;
    r->t_submit = now_s();
    s->all[r->id] = r;
    s->queue.push_back(r);
    *req_id = r->id;
    return IBLBM_OK;
}

int iblbm_server_tick(iblbm_server* s, int max_steps, int* resident, int* queued) {
    if (!s || max_steps < 1) return IBLBM_ERR_INVALID_ARG;
    int rc = IBLBM_OK;
    if (s->resident.empty()) admit(s);
    int done = 0;
    if (!s->resident.empty()) {
        long long step = max_steps;
        for (auto* r : s->resident) step = std::min(step, r->remaining);
        std::vector<iblbm_ctx*> ctxs;
        for (auto* r : s->resident) ctxs.push_back(r->ctx);
        rc = iblbm_internal_step_batch(ctxs.data(), (int)ctxs.size(), (int)step, s->use_graphs);
        // while the device works, bring in requests that fit next to the running ones
        std::vector<Request*> before = s->resident;
        admit(s);
        std::vector<Request*> keep;
        for (auto* r : s->resident) {
            const bool stepped = std::find(before.begin(), before.end(), r) != before.end();
            if (stepped) {
                const int st = iblbm_sync(r->ctx);
                if (st < 0) r->error = st;
                r->remaining -= rc ? 0 : step;
                if (r->remaining <= 0 || r->error) {
                    retire(s, r);
                    ++done;
                    continue;
                }
            }
            keep.push_back(r);
        }
        s->resident.swap(keep);
    }
    if (resident) *resident = (int)s->resident.size();
    if (queued) *queued = (int)s->queue.size();
    return rc < 0 ? rc : done;
}

int iblbm_server_poll(iblbm_server* s, long long req_id, double* forces_out, int cap, int* n, double* latency_s) {
    if (!s) return IBLBM_ERR_INVALID_ARG;
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return IBLBM_ERR_NOT_FOUND;
    Request* r = it->second;
    if (r->state != Q_DONE) return 0;
    if (r->error < 0) return r->error;
    const int have = (int)(r->history.size() / 3);
    const int m = std::min(have, std::max(cap, 0));
    if (forces_out && m > 0) std::copy(r->history.end() - 3 * (size_t)m, r->history.end(), forces_out);
    if (n) *n = m;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    return 1;
}

int iblbm_server_set_graphs(iblbm_server* s, int enable) {
    if (!s) return IBLBM_ERR_INVALID_ARG;
    s->use_graphs = enable ? 1 : 0;
    return IBLBM_OK;
}

int iblbm_server_stats(const iblbm_server* s, size_t* used_bytes, int* resident, int* queued) {
    if (!s) return IBLBM_ERR_INVALID_ARG;
    if (used_bytes) *used_bytes = s->used;
    if (resident) *resident = (int)s->resident.size();
    if (queued) *queued = (int)s->queue.size();
    return IBLBM_OK;
}

}  // extern "C"
