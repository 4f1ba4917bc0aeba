// Serving loop: many forward solves against shared, device-resident adjoint
// snapshot sets.  Requests queue in arrival order; a request is admitted as
// soon as a slot is free and its projected device memory fits the budget
// (continuous admission: requests that arrive while others run join as
// slots and memory free up).  Each slot is a worker thread with its own CUDA
// stream, so the kernels of all admitted requests overlap on the device.
// Each request's arithmetic depends only on its own inputs (own arenas, no
// cross-request reduction), so its result is the same alone and in a mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

struct Req {
    long long ticket = 0;
    adjamr_params p;
    adjamr_medium m;
    std::vector<double> iface, f0, f1;
    adjamr_adjoint *adj = nullptr;
    adjamr_target t;
    size_t bytes = 0;
    adjamr_result res;
};

double now_s(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" size_t adjamr_estimate_bytes(const adjamr_params *p)
{
    if (!p || p->nlevels < 1 || p->nlevels > ADJAMR_MAX_LEVELS) return 0;
    for (int l = 0; l < p->nlevels - 1; l++)
        if (p->ratio[l] < 2 || p->ratio[l] > adjamr::kMaxSubsteps) return 0;  // as hierarchy creation refuses them
    const int m = (p->dim == 2) ? 3 : 2;
    const int per = 2 * m + adjamr::naux_of(p->eqn) + adjamr::nmed_of(p->eqn);
    long long N = p->n0[0], M = (p->dim == 2) ? p->n0[1] : 1;
    size_t total = 0;
    long long prev = 0;  // storage cells of the coarser level
    for (int l = 0; l < p->nlevels; l++) {
        // upper bound: every level fully refined, ghost rings included
        long long cells = (N + 4 * (N / 8 + 1)) * (p->dim == 2 ? (M + 4 * (M / 8 + 1)) : 1);
        total += (size_t)cells * per * sizeof(double);
        // descriptors (ghost maps, average-down maps, work-lists), generous
        total += (size_t)cells * 24;
        // coarse stencil values of the ghost cells (3 per coarse cell, field
        // and substep), their marks, and the list of coarse cells
        if (l > 0) total += (size_t)prev * (3 * sizeof(double) * m * p->ratio[l - 1] + sizeof(int)) + (size_t)cells * 8;
        // conservation fix-up: arena map and records (refluxing runs only)
        if (p->reflux) total += (size_t)cells * 8;
        // error-estimate flagging: the extended patches (rings of 4 cells: at
        // most 4.5x the cells of patches of 8 or more cells a side) with their
        // coarsened copies (a quarter), state, first-step state and
        // coefficients, and the estimate itself
        if ((p->flag_mode == ADJAMR_FLAG_ERROR || p->flag_mode == ADJAMR_FLAG_RICHARDSON) && l < p->nlevels - 1)
            total += (size_t)cells * sizeof(double) * ((size_t)per * 45 / 10 * 5 / 4 + (size_t)m);
        prev = cells;
        if (l < p->nlevels - 1) {
            N *= p->ratio[l];
            if (p->dim == 2) M *= p->ratio[l];
        }
    }
    return total;
}

struct adjamr_server {
    size_t budget = 0, used = 0;
    int max_slots = 0, active = 0, dev = 0;
    long long next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::map<long long, Req *> all;
    std::vector<std::thread> workers;
    bool stop = false;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
};

namespace {

void run_request(adjamr_server *srv, Req *r, cudaStream_t s)
{
    adjamr_params p = r->p;
    p.stream = (void *)s;
    adjamr_ctx *ctx = nullptr;
    adjamr_status st = adjamr_init_grid_hierarchy(&p, &ctx);
    if (st == ADJAMR_OK) {
        // admitted bytes stay the projected bytes: no block cache, no coefficient tables
        adjamr::ctx_set_block_cache(ctx, 0);
        adjamr::ctx_set_aux_tables(ctx, false);
    }
    if (st == ADJAMR_OK) st = adjamr_set_medium(ctx, &r->m);
    if (st == ADJAMR_OK) st = adjamr_set_adjoint(ctx, r->adj);
    if (st == ADJAMR_OK) st = adjamr_regrid(ctx, 0, 1);
    int nsteps = 0;
    if (st == ADJAMR_OK) st = adjamr_time_info(ctx, nullptr, &nsteps);
    if (st == ADJAMR_OK) st = adjamr_advance_level(ctx, 0, nsteps);
    double J = 0.0;
    if (st == ADJAMR_OK) st = adjamr_integrate_functional(ctx, &r->t, &J);
    adjamr_stats stats;
    std::memset(&stats, 0, sizeof stats);
    if (ctx) adjamr_get_stats(ctx, &stats);
    if (st != ADJAMR_OK && ctx) std::strncpy(r->res.error, adjamr_last_error(ctx), sizeof(r->res.error) - 1);
    adjamr_destroy(ctx);
    r->res.status = st;
    r->res.J = J;
    r->res.cell_updates = stats.cell_updates;
    r->res.kernel_launches = stats.kernel_launches;
    (void)srv;
}

void worker(adjamr_server *srv)
{
    cudaSetDevice(srv->dev);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        Req *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] {
                return srv->stop ||
                       (!srv->queue.empty() && srv->used + srv->queue.front()->bytes <= srv->budget);
            });
            if (srv->stop && srv->queue.empty()) break;
            if (srv->stop) break;
            r = srv->queue.front();
            srv->queue.pop_front();
            srv->used += r->bytes;
            srv->active++;
            r->res.t_admit = now_s(srv->t0);
        }
        run_request(srv, r, s);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            r->res.t_finish = now_s(srv->t0);
            r->res.done = 1;
            srv->used -= r->bytes;
            srv->active--;
            adjamr_adjoint_release(r->adj);
            r->adj = nullptr;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
    if (s) cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

adjamr_status adjamr_server_create(size_t budget_bytes, int max_slots, adjamr_server **out)
{
    if (!out || max_slots < 1 || budget_bytes == 0) return ADJAMR_EINVAL;
    adjamr_server *srv = new (std::nothrow) adjamr_server();
    if (!srv) return ADJAMR_ENOMEM;
    srv->budget = budget_bytes;
    srv->max_slots = max_slots;
    if (cudaGetDevice(&srv->dev) != cudaSuccess) {
        delete srv;
        return ADJAMR_ECUDA;
    }
    try {
        for (int k = 0; k < max_slots; k++) srv->workers.emplace_back(worker, srv);
    } catch (...) {
        adjamr_server_destroy(srv);
        return ADJAMR_ENOMEM;
    }
    *out = srv;
    return ADJAMR_OK;
}

adjamr_status adjamr_server_submit(adjamr_server *srv, const adjamr_request *rq, long long *ticket)
{
    if (!srv || !rq || !rq->adjoint || rq->medium.kind != ADJAMR_MEDIUM_LAYERED || rq->medium.nlayers < 1 ||
        rq->medium.nlayers > 32)
        return ADJAMR_EINVAL;
    Req *r = new (std::nothrow) Req();
    if (!r) return ADJAMR_ENOMEM;
    r->p = rq->params;
    r->m = rq->medium;
    int nl = rq->medium.nlayers;
    r->iface.assign(rq->medium.iface, rq->medium.iface + (nl > 1 ? nl - 1 : 0));
    r->f0.assign(rq->medium.f0, rq->medium.f0 + nl);
    r->f1.assign(rq->medium.f1, rq->medium.f1 + nl);
    r->m.iface = r->iface.empty() ? nullptr : r->iface.data();
    r->m.f0 = r->f0.data();
    r->m.f1 = r->f1.data();
    r->t = rq->target;
    r->bytes = adjamr_estimate_bytes(&rq->params);
    std::memset(&r->res, 0, sizeof r->res);
    if (r->bytes == 0) {  // parameters the estimate (and the hierarchy) refuse
        delete r;
        return ADJAMR_EINVAL;
    }
    if (r->bytes > srv->budget) {
        delete r;
        return ADJAMR_EBUDGET;
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        r->ticket = srv->next_ticket++;
        r->adj = rq->adjoint;
        r->adj->refs++;
        r->res.t_submit = now_s(srv->t0);
        r->res.bytes_reserved = r->bytes;
        srv->all[r->ticket] = r;
        srv->queue.push_back(r);
        if (ticket) *ticket = r->ticket;
    }
    srv->cv_work.notify_all();
    return ADJAMR_OK;
}

adjamr_status adjamr_server_poll(adjamr_server *srv, long long ticket, adjamr_result *out)
{
    if (!srv || !out) return ADJAMR_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) return ADJAMR_EINVAL;
    *out = it->second->res;
    return ADJAMR_OK;
}

adjamr_status adjamr_server_wait(adjamr_server *srv, long long ticket, adjamr_result *out)
{
    if (!srv) return ADJAMR_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) return ADJAMR_EINVAL;
    Req *r = it->second;
    srv->cv_done.wait(lk, [&] { return r->res.done != 0; });
    if (out) *out = r->res;
    return ADJAMR_OK;
}

adjamr_status adjamr_server_info(adjamr_server *srv, size_t *used, int *active, int *queued)
{
    if (!srv) return ADJAMR_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (used) *used = srv->used;
    if (active) *active = srv->active;
    if (queued) *queued = (int)srv->queue.size();
    return ADJAMR_OK;
}

double adjamr_server_now(adjamr_server *srv) { return srv ? now_s(srv->t0) : 0.0; }

void adjamr_server_destroy(adjamr_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        // queued requests that never ran drop their adjoint references
        for (Req *r : srv->queue) {
            adjamr_adjoint_release(r->adj);
            r->adj = nullptr;
            r->res.status = ADJAMR_ESTATE;
            r->res.done = 1;
        }
        srv->queue.clear();
    }
    srv->cv_work.notify_all();
    for (std::thread &t : srv->workers)
        if (t.joinable()) t.join();
    for (auto &kv : srv->all) delete kv.second;
    delete srv;
}

}  // extern "C"
